// FP64 instantiations of the specialised x-transform kernels.
#include "k_fft_x_fast.cuh"

namespace pp {
cudaError_t launch_fwd_x_fast_dd(const Geometry& g, const DevTables& tb, FwdMode mode, const FwdArgs& args,
                                 cplx<double>* spec, cudaStream_t st) {
  return launch_fwd_x_fast_impl<double, double>(g, tb, tb.d, mode, args, spec, st);
}
cudaError_t launch_inv_x_fast_dd(const Geometry& g, const DevTables& tb, InvMode mode, const cplx<double>* spec,
                                 double* out, double scale, bool accumulate, cudaStream_t st, PairArgs pair) {
  return launch_inv_x_fast_impl<double, double>(g, tb, tb.d, mode, spec, out, scale, accumulate, st,
                                                 pair);
}
}  // namespace pp
