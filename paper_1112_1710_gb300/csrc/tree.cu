// tree.cu -- the AMR tree on the device: parents of the patches of a level and
// the neighbour relations of a level inherited from the level above
// (Sec. 3.1).  Integer box algebra only.
//
// Because grids are nested, the neighbours of a node's children are children
// of the node's neighbours (Sec. 3.1): a child c of level l+1 can only
// interact with children of the patches that interact with c's parents.  Here
// "interact" means that box(c') shifted by s periodic domain lengths meets
// box(c) grown by r cells; with r = g + 1 these are exactly the pairs that
// carry ghost copies.  Completeness: take a cell x of box(c') + s N within r
// of the cell y of box(c) nearest to it; the coarse cells x/2 and y/2 (floor)
// are at most ceil(r/2) <= r apart per axis, y/2 lies in a parent P of c and
// x/2 in a parent P' of c' shifted by s (the fine boxes lie inside the union
// of the coarse ones, and the fine domain is twice the coarse one), so
// (P', s) is an interaction of P at range r.  A child may have several
// parents (the patches of level l its coarsened box meets).  Each kernel runs in two passes: without an output
// list it writes per-child counts, with one it writes the entries at the
// given offsets, in loop order (parents, their interactions, their children).
#include <cuda_runtime.h>

#include <cstdint>

#include "mhd_gpu.h"

namespace mhd {
namespace {

struct IBox {
  int lo[3], hi[3];
};

__device__ __forceinline__ IBox load_box(const int32_t* lo, const int32_t* hi, int i) {
  IBox b;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    b.lo[d] = lo[3 * i + d];
    b.hi[d] = hi[3 * i + d];
  }
  return b;
}

// Floor division by 2 for negative indices too (coarsening of a fine index).
__device__ __forceinline__ int half_floor(int v) { return v >= 0 ? v / 2 : -((-v + 1) / 2); }

// Parents: coarse boxes that meet the coarsened fine box [lo/2, hi/2].
__global__ void k_parents(const int32_t* __restrict__ flo, const int32_t* __restrict__ fhi, int nf,
                          const int32_t* __restrict__ clo, const int32_t* __restrict__ chi, int nc,
                          const int64_t* __restrict__ off, int32_t* __restrict__ count, int32_t* __restrict__ list) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  const IBox F = load_box(flo, fhi, f);
  int cl[3], ch[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    cl[d] = half_floor(F.lo[d]);
    ch[d] = half_floor(F.hi[d]);
  }
  int32_t n = 0;
  int64_t o = list ? off[f] : 0;
  for (int c = 0; c < nc; ++c) {
    bool meet = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) meet = meet && clo[3 * c + d] <= ch[d] && chi[3 * c + d] >= cl[d];
    if (!meet) continue;
    if (list) list[o + n] = c;
    ++n;
  }
  if (!list) count[f] = n;
}

// Inherited interactions of the children: for child c, every (c', s) with c'
// a child of P', (P', s) an interaction of a parent P of c, and box(c') + s N
// meeting box(c) grown by r.
__global__ void k_inherit(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi, int n, int ndom, int r,
                          const int64_t* __restrict__ par_off, const int32_t* __restrict__ par,
                          const int64_t* __restrict__ int_off, const int32_t* __restrict__ inter,
                          const int8_t* __restrict__ int_shift, const int64_t* __restrict__ kid_off,
                          const int32_t* __restrict__ kid, const int64_t* __restrict__ out_off,
                          int32_t* __restrict__ count, int32_t* __restrict__ out, int8_t* __restrict__ out_shift) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const IBox C = load_box(lo, hi, c);
  int gl[3], gh[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    gl[d] = C.lo[d] - r;
    gh[d] = C.hi[d] + r;
  }
  int32_t m = 0;
  const int64_t o = out ? out_off[c] : 0;
  for (int64_t pi = par_off[c]; pi < par_off[c + 1]; ++pi) {
    const int P = par[pi];
    for (int64_t ii = int_off[P]; ii < int_off[P + 1]; ++ii) {
      const int P2 = inter[ii];
      const int s0 = int_shift[3 * ii], s1 = int_shift[3 * ii + 1], s2 = int_shift[3 * ii + 2];
      const int sh[3] = {s0 * ndom, s1 * ndom, s2 * ndom};
      for (int64_t ki = kid_off[P2]; ki < kid_off[P2 + 1]; ++ki) {
        const int c2 = kid[ki];
        bool meet = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) meet = meet && lo[3 * c2 + d] + sh[d] <= gh[d] && hi[3 * c2 + d] + sh[d] >= gl[d];
        if (!meet) continue;
        if (out) {
          out[o + m] = c2;
          out_shift[3 * (o + m)] = (int8_t)s0;
          out_shift[3 * (o + m) + 1] = (int8_t)s1;
          out_shift[3 * (o + m) + 2] = (int8_t)s2;
        }
        ++m;
      }
    }
  }
  if (!out) count[c] = m;
}

}  // namespace
}  // namespace mhd

using namespace mhd;

extern "C" mhd_status mhd_tree_parents(const int32_t* d_flo, const int32_t* d_fhi, int32_t nf, const int32_t* d_clo,
                                       const int32_t* d_chi, int32_t nc, const int64_t* d_off, int32_t* d_count,
                                       int32_t* d_list, void* stream) {
  if (nf < 0 || nc < 0) return MHD_EINVAL;
  if (nf == 0) return MHD_OK;
  if (!d_flo || !d_fhi || (nc > 0 && (!d_clo || !d_chi))) return MHD_EINVAL;
  if (d_list ? !d_off : !d_count) return MHD_EINVAL;
  k_parents<<<(nf + 127) / 128, 128, 0, (cudaStream_t)stream>>>(d_flo, d_fhi, nf, d_clo, d_chi, nc, d_off, d_count,
                                                                 d_list);
  return cudaGetLastError() == cudaSuccess ? MHD_OK : MHD_ECUDA;
}

extern "C" mhd_status mhd_tree_inherit(const int32_t* d_lo, const int32_t* d_hi, int32_t n, int32_t ndom, int32_t r,
                                       const int64_t* d_par_off, const int32_t* d_par, const int64_t* d_int_off,
                                       const int32_t* d_int, const int8_t* d_int_shift, const int64_t* d_kid_off,
                                       const int32_t* d_kid, const int64_t* d_out_off, int32_t* d_count,
                                       int32_t* d_out, int8_t* d_out_shift, void* stream) {
  if (n < 0 || ndom < 1 || r < 0) return MHD_EINVAL;
  if (n == 0) return MHD_OK;
  if (!d_lo || !d_hi || !d_par_off || !d_par || !d_int_off || !d_int || !d_int_shift || !d_kid_off || !d_kid)
    return MHD_EINVAL;
  if (d_out ? (!d_out_off || !d_out_shift) : !d_count) return MHD_EINVAL;
  k_inherit<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(d_lo, d_hi, n, ndom, r, d_par_off, d_par, d_int_off,
                                                                d_int, d_int_shift, d_kid_off, d_kid, d_out_off,
                                                                d_count, d_out, d_out_shift);
  return cudaGetLastError() == cudaSuccess ? MHD_OK : MHD_ECUDA;
}
