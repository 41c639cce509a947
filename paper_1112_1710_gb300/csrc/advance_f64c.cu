// advance_f64c.cu -- FP64 instantiation of the staged patch advance built with
// multiply-add contraction (--fmad=true): the same expressions with a*b+c
// fused into one rounding, which takes about a quarter fewer FP64 pipe
// instructions.  Results differ from the parity build by rounding only.
#define MHD_ADVANCE_NS contracted64
#define MHD_FAST_RECIP 1
#include "advance.cuh"

namespace mhd {

cudaError_t advance_f64c(const AdvanceArgs& a, cudaStream_t s) { return contracted64::run_advance<double>(a, s); }

}  // namespace mhd
