// advance_f64.cu -- FP64 instantiation of the staged patch advance, the
// parity build: --fmad=false, so every result is the correctly rounded value
// of the expression as written, in the oracle's order.
#define MHD_ADVANCE_NS exact64
#define MHD_FAST_RECIP 0
#include "advance.cuh"

namespace mhd {

cudaError_t advance_f64(const AdvanceArgs& a, cudaStream_t s) { return exact64::run_advance<double>(a, s); }
cudaError_t floor_f64(const AdvanceArgs& a, cudaStream_t s) { return exact64::run_floor<double>(a, s); }

}  // namespace mhd
