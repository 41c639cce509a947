// launch.h -- host entry points of the kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace mhd {

struct AdvanceArgs {
  const DPatch* patches;   // device
  int npatches;
  const BlockTask* tasks;  // device, blocks over each patch's UB+2
  int nblocks;
  const BlockTask* tasks1;  // device, blocks over each patch's UB+1
  int nblocks1;
  const BlockTask* tasksu;  // device, blocks over [lo, hi + 1] of each patch's UB
  int nblocksu;
  const BlockTask* ptasks;  // device, tiles of the tiled predictor (npblocks 0: untiled)
  int npblocks;
  void* scratch;           // device arena of the call's element type
  void* stepc;             // device, npatches x 8 elements of that type (in the arena)
  double gamma, eps_up;
  int limiter, emf;
  const double* d_dt;      // device
  int* d_status;           // device
  const KernelTimer* timer;  // nullable
  // fused advance (one persistent kernel over the work items, then k_commit)
  bool fused;
  const FusedItem* items;    // device
  int nitems;
  int* counter;              // device, the work-queue head (zeroed by the launch)
  const BlockTask* ctasks;   // device, k_commit blocks over each UB + 1
  int nctasks;
  int variant;               // index into the variant table of the element type
  bool commit;               // false: leave the new state in the output copies
  // staged only: non-null makes k_prim compute the step's CFL dt into this
  // device double (the same one as d_dt) before the step constants read it
  unsigned long long* cfl_out;
  double cfl;
  // pressure floor after the update (0: none) and the device count of the
  // cells it raised
  double p_floor, rho_floor;
  unsigned long long* d_floors;
  // primitive + predictor + Riemann passes fused (k_pf over x-y tiles of UB+1
  // and z-chunks, items in the FusedItem layout; shape `variant` of
  // kPfVariants), then the staged update
  bool pf;
  const FusedItem* pf_items;  // device
  int npf;
  // fused kernel without commit: the copy-back writes through these patches'
  // arrays instead (device; the autotuner's scratch destinations)
  const DPatch* commit_patches;
};

// Compiled shapes of the fused primitive / predictor / Riemann pass (k_pf):
// the largest x-y tile and the blocks per SM its registers and shared memory
// allow (FP32: 16 x 16 at 2, 92 KB; 16 x 12 and 24 x 8 at 3, 71-72 KB;
// 16 x 8 at 4, 50 KB).
struct PfVariant {
  int tx, ty, minb;
};
constexpr PfVariant kPfVariants32[] = {{16, 16, 2}, {16, 12, 3}, {24, 8, 3}, {16, 8, 4}};
constexpr PfVariant kPfVariants64[] = {{8, 8, 2}};
constexpr int kNumPf32 = sizeof(kPfVariants32) / sizeof(kPfVariants32[0]);
constexpr int kNumPf64 = sizeof(kPfVariants64) / sizeof(kPfVariants64[0]);

// Compiled shapes of the fused advance: x-y tile and threads per CTA (one CTA
// per SM; FP64 fits smaller tiles, its intermediates being twice as large).
struct FusedVariant {
  int bx, by, nt;
};
constexpr FusedVariant kFusedVariants32[] = {{16, 16, 512}, {16, 16, 384}, {16, 12, 384}, {24, 8, 384}};
constexpr FusedVariant kFusedVariants64[] = {{8, 8, 128}};
constexpr int kNumFused32 = sizeof(kFusedVariants32) / sizeof(kFusedVariants32[0]);
constexpr int kNumFused64 = sizeof(kFusedVariants64) / sizeof(kFusedVariants64[0]);

// Launch regions of the staged advance (UB = [lo, hi]): the predictor and
// flux stages run over UB grown by region_m1 on each side, the update stages
// over [lo - region_mu, hi + region_mu_top]: the regions the stages fill
// (UB+1; [lo, hi + 1]), which saves the idle threads of small patches.  The
// alternative, UB+2 for every stage (a thread's element is then its storage
// element), measured on GB300 in FP32: a 128^3 patch 0.432 against 0.428 ms
// per step, a 64^3 patch 0.084 against 0.085 ms, and the AMR hierarchy of
// 8-48 cell patches 65.9 against 63.1 ms per coarse step; FP64 is faster
// over the tight regions at every size.
constexpr int region_m1(size_t) { return 1; }
constexpr int region_mu(size_t) { return 0; }
constexpr int region_mu_top(size_t) { return 1; }

// Kernel launches of one staged advance: step constants, k_prim, k_pred,
// k_flux, k_update, and k_edge and k_emf in FP64 (one more, the dt reset,
// when k_prim computes the CFL dt).
inline int staged_launches(size_t elem) { return elem == 8 ? 7 : 5; }

cudaError_t advance_f64(const AdvanceArgs& a, cudaStream_t s);
cudaError_t advance_f64c(const AdvanceArgs& a, cudaStream_t s);
cudaError_t advance_f32(const AdvanceArgs& a, cudaStream_t s);
// The floors of AdvanceArgs (p_floor, rho_floor, d_floors) over the cells of
// each patch's interior (tasksu over [lo, hi + 1] with k = 0).
cudaError_t floor_f64(const AdvanceArgs& a, cudaStream_t s);
cudaError_t floor_f32(const AdvanceArgs& a, cudaStream_t s);

// CFL candidate minimum over the interiors (tasks span interiors).
cudaError_t cfl_dt_launch(int dtype, const DPatch* patches, const BlockTask* tasks, int nblocks,
                          double gamma, double cfl, double* d_out, int* d_status,
                          const KernelTimer* tm, cudaStream_t s);

// Conservation sums (tasks span interiors); partials holds nblocks*8 doubles.
cudaError_t sums_launch(int dtype, const DPatch* patches, const BlockTask* tasks, int nblocks,
                        double* partials, double* d_out8, const KernelTimer* tm, cudaStream_t s);

// Regridding's error flags of the interiors (tasks span interiors; flags of
// patch p start at off[p]).
cudaError_t flag_launch(int dtype, const DPatch* patches, const BlockTask* tasks, int nblocks, const int64_t* off,
                        double gamma, double theta, uint8_t* flags, cudaStream_t s);

}  // namespace mhd
