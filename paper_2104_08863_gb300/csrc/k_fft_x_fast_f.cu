// FP32 instantiations of the x-transform kernels (FP32 field, FP32 half spectrum).
#include "k_fft_x_fast.cuh"

namespace pp {
cudaError_t launch_fwd_x_fast_ff(const Geometry& g, const DevTables& tb, FwdMode mode, const FwdArgs& args,
                                 cplx<float>* spec, cudaStream_t st) {
  return launch_fwd_x_fast_impl<float, float>(g, tb, tb.f, mode, args, spec, st);
}
cudaError_t launch_inv_x_fast_ff(const Geometry& g, const DevTables& tb, InvMode mode, const cplx<float>* spec,
                                 float* out, double scale, bool accumulate, cudaStream_t st, PairArgs pair) {
  return launch_inv_x_fast_impl<float, float>(g, tb, tb.f, mode, spec, out, scale, accumulate, st,
                                                 pair);
}
}  // namespace pp
