// hilbert.cu -- space-filling-curve ordering and Hilbert splitting of grids
// (Sec. 5.1 grid assignments, Sec. 5.2 Hilbert splitting).  Integer keys on
// the device, the recursive bisection on the host.
//
// Hilbert index: Skilling's transposed-axes construction (J. Skilling,
// "Programming the Hilbert curve", AIP Conf. Proc. 707, 381 (2004)): from the
// top bit down, a set bit Q of coordinate i inverts the bits below Q of
// coordinate 0, a clear one exchanges them with coordinate i's; the
// coordinates are then Gray-coded across the axes, a parity mask from the
// last coordinate is applied to all, and the index is read off the
// transposed bits, the top bit of coordinate 0 first.  The children of a
// cell take one contiguous block of 2^dim indices, so child order follows
// parent order (Sec. 5.1).
//
// Distance of a grid along the curve: the sum of the indices of its 2^dim
// corner cells (Sec. 5.1 samples a grid by its corners); only order and
// differences are used.
//
// Built with FP contraction off: the splitter's costs must round as written.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

#include "mhd_gpu.h"

namespace mhd {
namespace {

constexpr uint64_t kBadKey = ~0ull;
constexpr int64_t kBadDist = INT64_MAX;

// Largest curve resolution per dimension: 2-D keys use 2 bits per level and
// 3-D keys 3; a corner sum of 2^dim keys must stay below 2^63.
__host__ __device__ inline int max_bits(int dim) { return dim == 2 ? 30 : 20; }

// Spreads the low 21 bits of v to every third bit (bit j -> bit 3 j).
__host__ __device__ inline uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x1fffffu;
  x = (x | (x << 32)) & 0x001f00000000ffffull;
  x = (x | (x << 16)) & 0x001f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

// Spreads the low 32 bits of v to every second bit (bit j -> bit 2 j).
__host__ __device__ inline uint64_t spread2(uint32_t v) {
  uint64_t x = v;
  x = (x | (x << 16)) & 0x0000ffff0000ffffull;
  x = (x | (x << 8)) & 0x00ff00ff00ff00ffull;
  x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}

// Hilbert index of the cell x[0..dim) at resolution `bits` (every coordinate
// in [0, 2^bits) is the caller's precondition).  The exchange step is
// written without branches (a mask selects inversion or exchange), and the
// transposed bits are read off as a bit interleave: bit j of coordinate i
// becomes bit dim j + (dim - 1 - i) of the index.
__host__ __device__ inline uint64_t hilbert_key(const int32_t* x, int dim, int bits) {
  uint32_t X[3] = {0, 0, 0};
  for (int i = 0; i < dim; ++i) X[i] = (uint32_t)x[i];
  if (bits == 0) return 0;
  const uint32_t top = 1u << (bits - 1);
  for (uint32_t Q = top; Q > 1; Q >>= 1) {
    const uint32_t P = Q - 1;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if (i >= dim) break;
      const uint32_t inv = (X[i] & Q) ? P : 0u;          // bit set: invert
      const uint32_t t = (X[0] ^ X[i]) & (P & ~inv);     // bit clear: exchange
      X[0] ^= inv | t;
      X[i] ^= t;
    }
  }
  for (int i = 1; i < dim; ++i) X[i] ^= X[i - 1];
  uint32_t t = 0;
  for (uint32_t Q = top; Q > 1; Q >>= 1) t ^= (X[dim - 1] & Q) ? Q - 1 : 0u;
  for (int i = 0; i < dim; ++i) X[i] ^= t;
  return dim == 3 ? (spread3(X[0]) << 2) | (spread3(X[1]) << 1) | spread3(X[2])
                  : (spread2(X[0]) << 1) | spread2(X[1]);
}

__host__ __device__ inline bool in_curve(const int32_t* x, int dim, int bits) {
  for (int i = 0; i < dim; ++i)
    if (x[i] < 0 || (int64_t)x[i] >= ((int64_t)1 << bits)) return false;
  return true;
}

// Corner-sum distance of the inclusive box [lo, hi]; kBadDist if it is empty
// or leaves the curve's domain.
__host__ __device__ inline int64_t box_distance(const int32_t* lo, const int32_t* hi, int dim, int bits) {
  for (int d = 0; d < dim; ++d)
    if (hi[d] < lo[d]) return kBadDist;
  if (!in_curve(lo, dim, bits) || !in_curve(hi, dim, bits)) return kBadDist;
  uint64_t s = 0;
  for (int k = 0; k < (1 << dim); ++k) {
    int32_t c[3];
    for (int d = 0; d < dim; ++d) c[d] = ((k >> d) & 1) ? hi[d] : lo[d];
    s += hilbert_key(c, dim, bits);
  }
  return (int64_t)s;
}

// One thread per point: its key, or kBadKey outside [0, 2^bits)^dim.
__global__ void k_hilbert_keys(const int32_t* __restrict__ pts, int64_t n, int dim, int bits,
                               uint64_t* __restrict__ keys) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t x[3];
  for (int d = 0; d < dim; ++d) x[d] = pts[i * dim + d];
  keys[i] = in_curve(x, dim, bits) ? hilbert_key(x, dim, bits) : kBadKey;
}

// One thread per box: its corner-sum distance.
__global__ void k_box_distances(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi, int64_t n,
                                int dim, int bits, int64_t* __restrict__ dist) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t a[3], b[3];
  for (int d = 0; d < dim; ++d) {
    a[d] = lo[i * dim + d];
    b[d] = hi[i * dim + d];
  }
  dist[i] = box_distance(a, b, dim, bits);
}

// ------------------------------------------------------------ splitting
struct Box {
  int32_t lo[3], hi[3];
};

// Cells of the box grown by g ghost layers (its advance cost).
double advance_cost(const Box& b, int dim, int g) {
  double c = 1.0;
  for (int d = 0; d < dim; ++d) c *= (double)(b.hi[d] - b.lo[d] + 1 + 2 * g);
  return c;
}

double wsum(const double* w, int a, int b) {  // w[a] + ... + w[b - 1], in order
  double s = 0.0;
  for (int k = a; k < b; ++k) s += w[k];
  return s;
}

constexpr double kComparable = 0.01;

// Recursive bisection of box b over weights w[a..e) (Sec. 5.2); appends one
// box per weight, in weight order.  False if a box has no axis to cut.
bool split_rec(const Box& b, const double* w, int a, int e, int dim, int bits, int g, std::vector<Box>& out) {
  if (e - a == 1) {
    out.push_back(b);
    return true;
  }
  // step 1: the prefix / suffix cut of the weights with the least difference
  // of sums, ties to the shorter prefix
  int cut = a + 1;
  double best = -1.0;
  for (int k = a + 1; k < e; ++k) {
    const double dif = std::fabs(wsum(w, a, k) - wsum(w, k, e));
    if (best < 0.0 || dif < best) {
      best = dif;
      cut = k;
    }
  }
  const double wa = wsum(w, a, cut), wb = wsum(w, cut, e), tot = wa + wb;
  const double sa = wa / tot, sb = wb / tot;
  // steps 2-4: candidates (axis, prefix side, cut at the floor or ceiling of
  // the proportional point), least cost, then the largest lead of the suffix
  // piece over the prefix piece along the curve among comparable costs
  struct Cand {
    double cost;
    int64_t gain;
    Box pa, pb;
  };
  std::vector<Cand> cands;
  for (int d = 0; d < dim; ++d) {
    const int L = b.hi[d] - b.lo[d] + 1;
    if (L < 2) continue;
    for (int high = 0; high < 2; ++high) {
      const double share_low = (high ? wb : wa) / tot;
      const double pos = share_low * (double)L;
      int cf = (int)std::floor(pos), cc = (int)std::ceil(pos);
      cf = cf < 1 ? 1 : (cf > L - 1 ? L - 1 : cf);
      cc = cc < 1 ? 1 : (cc > L - 1 ? L - 1 : cc);
      const int cuts[2] = {cf, cc};
      for (int ci = 0; ci < (cf == cc ? 1 : 2); ++ci) {
        Box lowb = b, highb = b;
        lowb.hi[d] = b.lo[d] + cuts[ci] - 1;
        highb.lo[d] = b.lo[d] + cuts[ci];
        Cand c;
        c.pa = high ? highb : lowb;
        c.pb = high ? lowb : highb;
        const double ca = advance_cost(c.pa, dim, g) / sa, cb = advance_cost(c.pb, dim, g) / sb;
        c.cost = ca > cb ? ca : cb;
        c.gain = box_distance(c.pb.lo, c.pb.hi, dim, bits) - box_distance(c.pa.lo, c.pa.hi, dim, bits);
        cands.push_back(c);
      }
    }
  }
  if (cands.empty()) return false;
  double least = cands[0].cost;
  for (const Cand& c : cands) least = c.cost < least ? c.cost : least;
  const Cand* pick = nullptr;
  for (const Cand& c : cands)
    if (c.cost <= least * (1.0 + kComparable) && (!pick || c.gain > pick->gain)) pick = &c;
  const Box pa = pick->pa, pb = pick->pb;
  return split_rec(pa, w, a, cut, dim, bits, g, out) && split_rec(pb, w, cut, e, dim, bits, g, out);
}

inline unsigned grid_for(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace
}  // namespace mhd

using namespace mhd;

extern "C" mhd_status mhd_hilbert_keys(const int32_t* d_pts, int64_t n_pts, int32_t dim, int32_t bits,
                                       uint64_t* d_keys, void* stream) {
  if (n_pts < 0 || (dim != 2 && dim != 3) || bits < 0 || bits > max_bits(dim)) return MHD_EINVAL;
  if (n_pts == 0) return MHD_OK;
  if (!d_pts || !d_keys || grid_for(n_pts) > 0x7fffffffu) return MHD_EINVAL;
  k_hilbert_keys<<<grid_for(n_pts), 256, 0, (cudaStream_t)stream>>>(d_pts, n_pts, dim, bits, d_keys);
  return cudaGetLastError() == cudaSuccess ? MHD_OK : MHD_ECUDA;
}

extern "C" mhd_status mhd_box_distances(const int32_t* d_lo, const int32_t* d_hi, int64_t n_boxes, int32_t dim,
                                        int32_t bits, int64_t* d_dist, void* stream) {
  if (n_boxes < 0 || (dim != 2 && dim != 3) || bits < 0 || bits > max_bits(dim)) return MHD_EINVAL;
  if (n_boxes == 0) return MHD_OK;
  if (!d_lo || !d_hi || !d_dist || grid_for(n_boxes) > 0x7fffffffu) return MHD_EINVAL;
  k_box_distances<<<grid_for(n_boxes), 256, 0, (cudaStream_t)stream>>>(d_lo, d_hi, n_boxes, dim, bits, d_dist);
  return cudaGetLastError() == cudaSuccess ? MHD_OK : MHD_ECUDA;
}

extern "C" mhd_status mhd_hilbert_split(const int32_t* lo, const int32_t* hi, int32_t dim, const double* weights,
                                        int32_t n_weights, int32_t bits, int32_t ghost, int32_t* out_lo,
                                        int32_t* out_hi) {
  if ((dim != 2 && dim != 3) || n_weights < 1 || bits < 0 || bits > max_bits(dim) || ghost < 0) return MHD_EINVAL;
  if (!lo || !hi || !weights || !out_lo || !out_hi) return MHD_EINVAL;
  for (int k = 0; k < n_weights; ++k)
    if (!(weights[k] > 0.0) || !std::isfinite(weights[k])) return MHD_EINVAL;
  Box b{};
  for (int d = 0; d < dim; ++d) {
    b.lo[d] = lo[d];
    b.hi[d] = hi[d];
  }
  if (box_distance(b.lo, b.hi, dim, bits) == kBadDist) return MHD_EINVAL;
  std::vector<Box> out;
  out.reserve(n_weights);
  if (!split_rec(b, weights, 0, n_weights, dim, bits, ghost, out)) return MHD_EINVAL;
  for (int k = 0; k < n_weights; ++k)
    for (int d = 0; d < dim; ++d) {
      out_lo[k * dim + d] = out[k].lo[d];
      out_hi[k * dim + d] = out[k].hi[d];
    }
  return MHD_OK;
}
