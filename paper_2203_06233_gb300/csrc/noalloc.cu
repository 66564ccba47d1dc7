// stap_run_cpi_noalloc: the whole STAP chain for one CPI with its scratch in a
// fixed-size device array that the library itself owns, so the caller never
// allocates device memory.  It drives the same plan and kernels as
// stap_run_cpi; only the origin of the scratch differs.
#include <mutex>

#include "stap_internal.cuh"

namespace {

// Scratch shared by every call on a device: status, tables and the dop / cov /
// wts intermediates of the CPI being processed.
static __device__ __align__(256) unsigned char g_noalloc_scratch[STAP_NOALLOC_SCRATCH_BYTES];

std::mutex g_setup_mutex;
void* g_scratch_addr[64] = {nullptr};  // device address of g_noalloc_scratch, per device

// Once per device, with that device current: the host-side name of the array
// is not a device address, so ask the runtime for the real one.
stap_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return STAP_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return STAP_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return STAP_OK;
}

}  // namespace

extern "C" stap_status stap_run_cpi_noalloc(const stap_dims* dims, const stap_options* opt,
                                            void* cuda_stream, const void* cube_c64, float* out,
                                            int64_t* n_failed_systems) {
  if (!dims || !cube_c64 || !out) return STAP_ERR_INVALID_ARG;
  stap_plan plan = nullptr;
  size_t need = 0;
  stap_status st = stap_plan_create(dims, 1, opt, cuda_stream, &plan, &need);
  if (st != STAP_OK) return st;
  if (need > (size_t)STAP_NOALLOC_SCRATCH_BYTES) {  // rejected before any CUDA call
    stap_plan_destroy(plan);
    return STAP_ERR_NO_WORKSPACE;
  }
  void* scratch = nullptr;
  st = scratch_address(&scratch);
  // set_workspace clears the status block and uploads this CPI's tables, so
  // nothing left in the array by an earlier call is read.
  if (st == STAP_OK) st = stap_plan_set_workspace(plan, scratch, STAP_NOALLOC_SCRATCH_BYTES);
  const void* cubes[1] = {cube_c64};
  float* outs[1] = {out};
  if (st == STAP_OK) st = stap_run_cpi(plan, cubes, outs);
  if (st == STAP_OK && n_failed_systems) {
    st = stap_get_status(plan, n_failed_systems);
  }
  stap_plan_destroy(plan);  // host metadata only; the launched work needs none of it
  return st;
}
