/*
 * dg_mixed_sym.cu -- the mixed-precision element kernel (dg_mixed_tc.cuh)
 * instantiated for the fully symmetric volume rules of degree 2p (3 / 6 / 12 /
 * 16 / 25 points at p = 1..5), in a translation unit of its own.
 */
#include "dg_mixed_tc.cuh"

namespace dg {

int tc_tables_sym(dg_mesh *m) { return tc_tables_rule<true>(m); }

int launch_element_tc_sym(const dg_mesh *m, int split3, const double *c, const double *u0, double *out,
                          float *trace_out, const float *fhat, const double *fmean, const StageUpdate &su,
                          int mode, void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
  return split3 ? dispatch_tc<true, true>(m, c, u0, out, trace_out, fhat, fmean, su, mode, s)
                : dispatch_tc<false, true>(m, c, u0, out, trace_out, fhat, fmean, su, mode, s);
}

}  // namespace dg
