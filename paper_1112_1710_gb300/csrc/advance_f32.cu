// advance_f32.cu -- FP32 instantiation of the staged patch advance (the bulk
// precision of the mixed-precision mode; flux registers and conservation sums
// stay in FP64).  Built with multiply-add contraction and fast FP32 division,
// reciprocal and square root.
#define MHD_ADVANCE_NS fast32
#define MHD_FAST_RECIP 1
#include "advance.cuh"

namespace mhd {

cudaError_t advance_f32(const AdvanceArgs& a, cudaStream_t s) { return fast32::run_advance<float>(a, s); }
cudaError_t floor_f32(const AdvanceArgs& a, cudaStream_t s) { return fast32::run_floor<float>(a, s); }

}  // namespace mhd
