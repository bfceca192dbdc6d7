// FP32-spectrum instantiations with FP64 fields: the FP64 right-hand side (plain or the
// refinement residual) into the FP32 half spectrum, and the FP64 assembly of the refined
// pressure.
#include "k_fft_x_fast.cuh"

namespace pp {
cudaError_t launch_fwd_x_fast_fd(const Geometry& g, const DevTables& tb, FwdMode mode, const FwdArgs& args,
                                 cplx<float>* spec, cudaStream_t st) {
  return launch_fwd_x_fast_impl<float, double>(g, tb, tb.f, mode, args, spec, st);
}
cudaError_t launch_inv_x_fast_fd(const Geometry& g, const DevTables& tb, InvMode mode, const cplx<float>* spec,
                                 double* out, double scale, bool accumulate, cudaStream_t st, PairArgs pair) {
  return launch_inv_x_fast_impl<float, double>(g, tb, tb.f, mode, spec, out, scale, accumulate, st,
                                                 pair);
}
}  // namespace pp
