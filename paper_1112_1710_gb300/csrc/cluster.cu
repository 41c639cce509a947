// cluster.cu -- grid generation for regridding (Sec. 2.1): the boxes that
// cover the cells a level flags for refinement.  The paper leaves the rule
// open and cites Berger's AMR papers; this is the point-clustering algorithm
// of Berger & Rigoutsos (IEEE Trans. SMC 21, 1278 (1991)).  Host code.
//
// A candidate box is shrunk to the bounding box of its flags and accepted
// when flagged cells / cells >= eff, or when no axis is at least 2 min_size
// long.  Otherwise it is cut between two slices of one axis, both pieces at
// least min_size long: at a hole of the signature (the flag count of each
// slice normal to the axis) nearest the box centre, ties to the lower slice,
// axes tried in order; else at the sign change of the signature's second
// difference with the largest jump over all axes, ties to the position
// nearer the centre, then the lower axis and slice; else at the middle of
// the longest axis.  Both pieces are clustered again, low piece first.
#include <cstdint>
#include <cstdlib>
#include <vector>

#include "mhd_gpu.h"

namespace mhd {
namespace {

struct Grid {
  const uint8_t* f;
  int dim;
  int64_t n[3];
  int64_t at(const int* x) const {
    int64_t i = 0;
    for (int d = 0; d < dim; ++d) i = i * n[d] + x[d];
    return i;
  }
};

struct CBox {
  int lo[3], hi[3];
};

// Visits every cell of box b (any order), calling fn(index array).
template <typename F> void for_cells(const Grid& g, const CBox& b, F&& fn) {
  int x[3] = {b.lo[0], b.lo[1], b.lo[2]};
  for (;;) {
    fn(x);
    int d = g.dim - 1;
    while (d >= 0) {
      if (++x[d] <= b.hi[d]) break;
      x[d] = b.lo[d];
      --d;
    }
    if (d < 0) return;
  }
}

// Signatures of box b along every axis, and the flag count.
int64_t signatures(const Grid& g, const CBox& b, std::vector<int64_t> (&sig)[3]) {
  for (int d = 0; d < g.dim; ++d) sig[d].assign(b.hi[d] - b.lo[d] + 1, 0);
  int64_t total = 0;
  for_cells(g, b, [&](const int* x) {
    if (g.f[g.at(x)]) {
      ++total;
      for (int d = 0; d < g.dim; ++d) ++sig[d][x[d] - b.lo[d]];
    }
  });
  return total;
}

struct Cut {
  int axis, after;  // cut after slice `after` (relative to lo)
};

bool choose_cut(const CBox& b, int dim, const std::vector<int64_t> (&sig)[3], int min_size, Cut& out) {
  // holes
  for (int d = 0; d < dim; ++d) {
    const int L = b.hi[d] - b.lo[d] + 1, c2 = L - 1;
    bool found = false;
    int64_t bk0 = 0, bk1 = 0, bk2 = 0;
    int bcut = 0;
    for (int i = 0; i < L; ++i) {
      if (sig[d][i] != 0) continue;
      for (int cut = i - 1; cut <= i; ++cut) {
        if (cut + 1 < min_size || L - cut - 1 < min_size) continue;
        const int64_t k0 = std::llabs((int64_t)2 * i - c2), k1 = i, k2 = cut;
        if (!found || k0 < bk0 || (k0 == bk0 && (k1 < bk1 || (k1 == bk1 && k2 < bk2)))) {
          found = true;
          bk0 = k0;
          bk1 = k1;
          bk2 = k2;
          bcut = cut;
        }
      }
    }
    if (found) {
      out = Cut{d, bcut};
      return true;
    }
  }
  // inflections
  bool found = false;
  int64_t bjump = 0, bdist = 0;
  Cut best{0, 0};
  for (int d = 0; d < dim; ++d) {
    const int L = b.hi[d] - b.lo[d] + 1;
    if (L < 4) continue;
    const std::vector<int64_t>& s = sig[d];
    for (int i = 1; i < L - 2; ++i) {
      const int64_t a = s[i - 1] - 2 * s[i] + s[i + 1];
      const int64_t c = s[i] - 2 * s[i + 1] + s[i + 2];
      if (!((a < 0 && c > 0) || (c < 0 && a > 0))) continue;
      if (i + 1 < min_size || L - i - 1 < min_size) continue;
      const int64_t jump = std::llabs(c - a), dist = std::llabs((int64_t)2 * i + 1 - (L - 1));
      // key (-jump, dist, axis, i); axes and slices come in increasing order
      if (!found || jump > bjump || (jump == bjump && dist < bdist)) {
        found = true;
        bjump = jump;
        bdist = dist;
        best = Cut{d, i};
      }
    }
  }
  if (found) {
    out = best;
    return true;
  }
  // the middle of the longest axis (the lower axis on ties)
  int d = 0;
  for (int k = 1; k < dim; ++k)
    if (b.hi[k] - b.lo[k] > b.hi[d] - b.lo[d]) d = k;
  const int L = b.hi[d] - b.lo[d] + 1;
  if (L < 2 * min_size) return false;
  out = Cut{d, L / 2 - 1};
  return true;
}

void cluster_rec(const Grid& g, CBox b, double eff, int min_size, std::vector<CBox>& out) {
  std::vector<int64_t> sig[3];
  const int64_t n = signatures(g, b, sig);
  if (n == 0) return;
  // shrink to the flags' bounding box
  for (int d = 0; d < g.dim; ++d) {
    int a = 0, z = b.hi[d] - b.lo[d];
    while (sig[d][a] == 0) ++a;
    while (sig[d][z] == 0) --z;
    b.hi[d] = b.lo[d] + z;
    b.lo[d] = b.lo[d] + a;
  }
  signatures(g, b, sig);
  int64_t cells = 1;
  for (int d = 0; d < g.dim; ++d) cells *= b.hi[d] - b.lo[d] + 1;
  if ((double)n * 1.0 >= eff * (double)cells) {
    out.push_back(b);
    return;
  }
  Cut c;
  if (!choose_cut(b, g.dim, sig, min_size, c)) {
    out.push_back(b);
    return;
  }
  CBox lo = b, hi = b;
  lo.hi[c.axis] = b.lo[c.axis] + c.after;
  hi.lo[c.axis] = b.lo[c.axis] + c.after + 1;
  cluster_rec(g, lo, eff, min_size, out);
  cluster_rec(g, hi, eff, min_size, out);
}

}  // namespace
}  // namespace mhd

using namespace mhd;

extern "C" mhd_status mhd_cluster_flags(const uint8_t* flags, int32_t dim, const int32_t* shape, double eff,
                                        int32_t min_size, int32_t max_boxes, int32_t* out_lo, int32_t* out_hi,
                                        int32_t* n_out) {
  if (!flags || !shape || !n_out || (dim != 2 && dim != 3) || min_size < 1 || max_boxes < 0) return MHD_EINVAL;
  if (!(eff > 0.0) || !(eff <= 1.0)) return MHD_EINVAL;
  if (max_boxes > 0 && (!out_lo || !out_hi)) return MHD_EINVAL;
  Grid g{flags, dim, {1, 1, 1}};
  CBox all{};
  for (int d = 0; d < dim; ++d) {
    if (shape[d] < 1) return MHD_EINVAL;
    g.n[d] = shape[d];
    all.lo[d] = 0;
    all.hi[d] = shape[d] - 1;
  }
  std::vector<CBox> out;
  cluster_rec(g, all, eff, min_size, out);
  *n_out = (int32_t)out.size();
  if ((int64_t)out.size() > max_boxes) return MHD_ETOOBIG;
  for (size_t k = 0; k < out.size(); ++k)
    for (int d = 0; d < dim; ++d) {
      out_lo[k * dim + d] = out[k].lo[d];
      out_hi[k * dim + d] = out[k].hi[d];
    }
  return MHD_OK;
}
