// common.cuh -- device-side descriptors shared by the kernels and the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace mhd {

// Device copy of one patch for a launch.  Array index a_d of a cell runs over
// [0, N_d); the interior is [g, g + n_d).  All eight arrays share s1 (y
// stride) and s2 (z stride); the x stride is 1.
struct DPatch {
  void* U[5];
  void* B[3];
  int64_t s1, s2;
  int64_t nelem;     // elements of one array (s2 * (N_2 + 1))
  int64_t snelem;    // stride of the library's scratch planes: nelem rounded
                     // up to 8, so that vector groups of planes stay aligned
  int64_t scr;       // offset of this patch's scratch in the arena (elements)
  int32_t n[3];      // interior cells
  int32_t N[3];      // cells including ghosts
  int32_t g;         // ghost layers
  int32_t k;         // update box = interior grown by k
  int32_t glo[3];    // global index of array index 0 (interior lo - g)
  int32_t flags;     // bit 0: the fused advance also stores fluxes for captures
  double dx[3];
  double dt_scale;   // dt of this patch = (*d_dt) * dt_scale
  double cfl_scale;  // scale factor of the CFL candidate dt
  float dxf[3];      // dx rounded to FP32 (FP32 kernels read no doubles per thread)
  int32_t pad2;
  double rdx[3];     // 1 / dx (FP64): the FP32-state refluxing multiplies by it
};

// Cell width along d in the arithmetic type of a kernel.
template <typename R> __device__ __forceinline__ R dx_of(const DPatch& p, int d);
template <> __device__ __forceinline__ double dx_of<double>(const DPatch& p, int d) { return p.dx[d]; }
template <> __device__ __forceinline__ float dx_of<float>(const DPatch& p, int d) { return p.dxf[d]; }

// q = floor(e / d) and e - q d for 0 <= e < 2^24 without an integer
// division: the single-precision quotient is within one of the true one and
// is corrected.
__device__ __forceinline__ int divmod24(int e, int d, int& r) {
  int q = __float2int_rz(__int2float_rn(e) * __frcp_rn(__int2float_rn(d)));
  r = e - q * d;
  if (r < 0) {
    q -= 1;
    r += d;
  } else if (r >= d) {
    q += 1;
    r -= d;
  }
  return q;
}

// One block of a batched launch: the patch it works on and the first linear
// element (within that patch's launch region) of its threads.
struct BlockTask {
  int32_t patch;
  int32_t start;
};

constexpr int kThreads = 256;

// Packed block tables: the elements of consecutive items (boxes of a list)
// laid end to end and cut into blocks of kThreads, so that small items share
// blocks.  starts[i] is the first element of item i (starts[n] the total);
// a block's task holds the item its first element lies in (patch) and that
// element's offset in it (start).  Every item holds at least one element, so
// a block spans at most kThreads items.  Returns false past the last element.
__device__ __forceinline__ bool packed_elem(const BlockTask& t, const int64_t* __restrict__ starts, int nitems,
                                            int& item, int& e) {
  const int64_t G = starts[t.patch] + t.start + threadIdx.x;
  if (G >= starts[nitems]) return false;
  int lo = t.patch, hi = nitems - 1 < t.patch + kThreads ? nitems - 1 : t.patch + kThreads;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (starts[mid] <= G) lo = mid;
    else hi = mid - 1;
  }
  item = lo;
  e = (int)(G - starts[lo]);
  return true;
}

// Element of an item list under either block table: aligned (packed == 0:
// every block inside one item, the task's item and offset as given, threads
// past the item's end idle) or packed (packed_elem).
__device__ __forceinline__ bool list_elem(const BlockTask& t, const int64_t* __restrict__ starts, int nitems,
                                          int packed, int& item, int& e) {
  if (packed) return packed_elem(t, starts, nitems, item, e);
  item = t.patch;
  e = t.start + threadIdx.x;
  return e < starts[item + 1] - starts[item];
}

// Component q of element x in a vector group of scratch planes (the 8 slots
// from g on, plane stride sn): FP32 groups are two planes of float4 (values
// 0-3, 4-7), FP64 four planes of double2.
template <typename R> __device__ __forceinline__ R* vgroup_at(R* g, int64_t sn, int64_t x, int q) {
  constexpr int W = 16 / (int)sizeof(R);
  return g + (int64_t)(q / W) * W * sn + W * x + (q % W);
}

// Tile of the tiled predictor (cells, x fastest; one thread per cell) per
// element type; the host builds one block per tile of each patch's UB+1.
constexpr int kPredTile32[3] = {32, 4, 2};
constexpr int kPredTile64[3] = {16, 4, 4};

// One work item of the fused advance: an x-y tile of the update box with
// lower corner (x0, y0) (array indices) and the planes [z0, z1).
struct FusedItem {
  int32_t patch, x0, y0, z0, z1;
  int32_t tx, ty;    // fused pass: this tile's x and y extents (at most its build's tile)
  int32_t pad;
};

// One ghost-fill copy, resolved to array indices of both patches.
struct DCopy {
  int32_t src, dst;
  int32_t lo[3];     // destination array indices of the box corner
  int32_t ext[3];    // box extents
  int32_t off[3];    // source array index = destination array index + off
  int32_t xr, nx;    // the copy's bottom-layer rectangles: DExcl xr .. xr + nx - 1
};

// A rectangle of a copy box's bottom layer along `axis` whose lower faces
// another copy of the same destination writes (as the upper faces of its top
// layer): the two transverse axes in increasing order, destination array
// indices, inclusive.
struct DExcl {
  int32_t axis;
  int32_t lo[2], hi[2];
};

// scratch arrays of the staged advance (offsets in units of one array)
enum : int {
  SC_W = 0,      // 8 primitives on UB+2
  SC_EN = 8,     // 3 cell-centred E^n = -v x Bc on UB+2
  SC_WF = 11,    // 48 predicted face states (d, side, q) on UB+1
  SC_ER = 59,    // 3 reference cell EMFs from U^{n+1/2} on UB+1
  SC_EE = 62,    // 3 edge E^n averages
  SC_F = 65,     // 24 face fluxes (d, q); slot 5+d holds the contact side
  SC_ED = 89,    // 3 edge EMFs of the update
  SC_COUNT = 92
};


// Records a device status code (the first one raised wins).  The status word
// is read first, so that once it is set the threads that meet further bad
// cells (a whole region of them, say) issue no atomic on the one address.
__device__ __forceinline__ void raise_status(int* status, int code) {
  if (*(volatile int*)status == 0) atomicCAS(status, 0, code);
}

// Kernel ids of the per-kernel event timer (mhd_timing_*).
enum KernelId : int {
  K_PRIM = 0, K_PRED, K_EDGE, K_FLUX, K_EMF, K_UPDATE, K_CFL, K_GHOST, K_SUMS, K_REFLUX, K_FUSED, K_COMMIT,
  K_PROLONG, K_RESTRICT, K_CAPTURE, K_PF, K_COUNT
};

// Optional hook that records CUDA events around each launch on its stream.
struct KernelTimer {
  void* self;
  void (*mark)(void* self, int kernel, int phase, cudaStream_t s);
};

#define MHD_TIMED(tm, id, s, launch)                      \
  do {                                                     \
    if (tm) (tm)->mark((tm)->self, (id), 0, (s));          \
    launch;                                                \
    if (tm) (tm)->mark((tm)->self, (id), 1, (s));          \
  } while (0)

}  // namespace mhd
