// advance_f64.cu -- FP64 instantiation of the staged patch advance.  Built with
// --fmad=false: no multiply-add contraction, so every result is the correctly
// rounded value of the expression as written.
#include "advance.cuh"
#include "launch.h"

namespace mhd {

cudaError_t advance_f64(const AdvanceArgs& a, cudaStream_t s) {
  SolverConsts<double> sc;
  sc.gamma = a.gamma;
  sc.gm1 = a.gamma - 1.0;
  sc.igm1 = 1.0 / sc.gm1;
  sc.eps_up = a.eps_up;
  sc.limiter = a.limiter;
  sc.emf = a.emf;
  return launch_advance<double>(a.patches, a.npatches, a.tasks, a.nblocks, (double*)a.scratch,
                                (double*)a.stepc, sc, a.d_dt, a.d_status, a.timer, s);
}

}  // namespace mhd
