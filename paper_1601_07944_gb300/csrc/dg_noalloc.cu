/*
 * dg_noalloc.cu -- dg_rhs_noalloc: the right-hand side of dg_rhs for callers
 * that cannot allocate device memory when they evaluate it.
 *
 * Some callers cannot call cudaMalloc at that point: a host that hands the whole
 * GPU to another allocator (a framework's caching pool that has already reserved
 * the device memory, where a raw cudaMalloc fails or fragments that pool), or a
 * time-critical loop that must not pay an allocation's latency and implicit
 * device synchronisation.  The RHS needs work space beyond its input and output
 * (the edge traces and the edge fluxes); this entry point takes it from one
 * fixed array of kScratchDoubles doubles (64 MiB) that lives in this file as a
 * static device variable.  Every GPU that loads this part of the library keeps
 * that array until the process exits.
 *
 * The array's name is only a host-side stand-in for the symbol; its device
 * address is fetched once per device with cudaGetSymbolAddress, on the first
 * call made while that device is current, and cached.  That first call should
 * therefore come before any stream capture.
 */
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "dg_internal.h"

namespace {

constexpr size_t kScratchDoubles = size_t(8) << 20;   // 8,388,608 doubles = 64 MiB

static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {};                // device address per device

}  // namespace

extern "C" dg_status dg_rhs_noalloc(dg_mesh *m, const double *c, double *r, dg_precision prec, void *stream) {
  if (!m || !c || !r) return dg::set_error(DG_EINVAL, "dg_rhs_noalloc: null argument");
  if (c == r) return dg::set_error(DG_EINVAL, "dg_rhs_noalloc: c and r alias");
  if (prec != DG_FP64 && prec != DG_TF32X1 && prec != DG_TF32X3)
    return dg::set_error(DG_EINVAL, "dg_rhs_noalloc: unknown precision %d", (int)prec);
  if (!m->bstate_set)
    return dg::set_error(DG_EINVAL, "dg_rhs_noalloc: the mesh has DG_BC_STATE faces and no boundary state was set");
  const size_t n_trace = (size_t)m->N * 3 * m->ne * dg::M;
  const size_t n_flux = (size_t)m->F * m->ne * dg::M;
  if (n_trace + n_flux > kScratchDoubles)
    return dg::set_error(DG_EINVAL,
                         "dg_rhs_noalloc: this mesh needs %zu doubles of work space (edge traces %zu + edge "
                         "fluxes %zu); the static array holds %zu (64 MiB); use dg_rhs",
                         n_trace + n_flux, n_trace, n_flux, kScratchDoubles);
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();     // leave no stale error for the next launch check
    return dg::set_error(DG_ECUDA, "dg_rhs_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
  }
  if (dev != m->device)
    return dg::set_error(DG_EINVAL, "dg_rhs_noalloc: current device %d is not the mesh's device %d", dev, m->device);
  if (dev < 0 || dev >= kMaxDevices) return dg::set_error(DG_EINVAL, "dg_rhs_noalloc: device %d out of range", dev);
  double *scratch;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
      double *ptr = nullptr;
      e = cudaGetSymbolAddress((void **)&ptr, g_scratch);
      if (e != cudaSuccess || !ptr) {
        cudaGetLastError();   // leave no stale error for the next launch check
        return dg::set_error(DG_ECUDA, "dg_rhs_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      }
      g_scratch_ptr[dev] = ptr;
    }
    scratch = g_scratch_ptr[dev];
  }
  // Every trace and flux slot is written before it is read, so nothing in the
  // array needs clearing between calls.
  // The mixed modes use the first half of each block (float32 traces and fluxes,
  // and the fluxes' float64 mean-mode integrals), in the same launches as dg_rhs.
  double *trace = scratch, *fhat = scratch + n_trace;
  if (prec == DG_FP64) {
    if ((e = (cudaError_t)dg::launch_traces(m, c, trace, stream)) != cudaSuccess ||
        (e = (cudaError_t)dg::launch_face_flux(m, trace, fhat, stream)) != cudaSuccess ||
        (e = (cudaError_t)dg::launch_element(m, c, nullptr, r, nullptr, fhat, 0.0, 0.0, 0.0, 0, stream)) !=
            cudaSuccess)
      return dg::set_error(DG_ECUDA, "dg_rhs_noalloc: %s", cudaGetErrorString(e));
  } else {
    const int split3 = prec == DG_TF32X3 ? 1 : 0;
    const dg::MixedBuffers b = dg::mixed_buffers(m, trace, fhat);
    if ((e = (cudaError_t)dg::launch_element_tc(m, split3, c, nullptr, nullptr, b.trace, nullptr, nullptr, 0.0,
                                                0.0, 0.0, 2, stream)) != cudaSuccess ||
        (e = (cudaError_t)dg::launch_face_flux_mixed(m, b, stream)) != cudaSuccess ||
        (e = (cudaError_t)dg::launch_element_tc(m, split3, c, nullptr, r, nullptr, b.fhat, b.fmean, 0.0, 0.0, 0.0,
                                                0, stream)) != cudaSuccess)
      return dg::set_error(DG_ECUDA, "dg_rhs_noalloc: %s", cudaGetErrorString(e));
  }
  return DG_OK;
}
