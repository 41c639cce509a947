// advance_f32.cu -- FP32 instantiation of the staged patch advance (the bulk
// precision of the mixed-precision mode; flux registers and conservation sums
// stay in FP64).  Built with multiply-add contraction enabled.
#include "advance.cuh"
#include "launch.h"

namespace mhd {

cudaError_t advance_f32(const AdvanceArgs& a, cudaStream_t s) {
  SolverConsts<float> sc;
  sc.gamma = (float)a.gamma;
  sc.gm1 = sc.gamma - 1.0f;
  sc.igm1 = 1.0f / sc.gm1;
  sc.eps_up = (float)a.eps_up;
  sc.limiter = a.limiter;
  sc.emf = a.emf;
  return launch_advance<float>(a.patches, a.npatches, a.tasks, a.nblocks, (float*)a.scratch,
                               (float*)a.stepc, sc, a.d_dt, a.d_status, a.timer, s);
}

}  // namespace mhd
