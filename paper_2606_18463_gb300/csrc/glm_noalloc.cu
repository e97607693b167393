// glm_noalloc.cu -- glm_sample_indices_noalloc: the host-output form of the
// index-stream draw (Algorithm 1's sampling step: Philox4x64-10 mapped to
// floor(U m / 2^64)) with its device staging buffer held in a fixed
// file-scope __device__ array instead of a per-call cudaMalloc/cudaFree.
//
// The scratch array is one per device (one copy per CUDA context), so two
// calls whose work overlaps on the same GPU race on it; callers serialise
// them.  The first call on a device resolves the array's address with
// cudaGetSymbolAddress (which may load this module), so make that first call
// before any stream capture begins.  The resolved address is kept for the
// life of the process: cudaDeviceReset ends the context it belongs to, so the
// entry point must not be called on a device after that device was reset.
#include <mutex>

#include "glm_internal.cuh"

namespace {

// 2^20 indices (4 MiB) of staging: every entry the kernel writes is copied
// back, and nothing is read before it is written, so nothing needs clearing.
constexpr int64_t kNoAllocMaxCount = GLM_SAMPLE_NOALLOC_MAX;
static __device__ __align__(256) int32_t g_sample_scratch[kNoAllocMaxCount];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
int32_t *g_scratch_addr[kMaxDevices] = {};

// Resolves the scratch address on the current device once; later calls read
// the cached pointer.
int scratch_for_current_device(int32_t **out) {
  int dev = -1;
  GLM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices)
    return glm::set_error(GLM_EUNSUPPORTED, "glm_sample_indices_noalloc: device ordinal >= 64");
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_sample_scratch);
    if (e != cudaSuccess || !p)
      return glm::cuda_error(e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                             "cudaGetSymbolAddress(g_sample_scratch)");
    g_scratch_addr[dev] = static_cast<int32_t *>(p);
  }
  *out = g_scratch_addr[dev];
  return GLM_OK;
}

}  // namespace

extern "C" int glm_sample_indices_noalloc(uint64_t seed, uint32_t problem, int64_t first_draw,
                                          int64_t count, int64_t m, int32_t *out) {
  glm::set_error(GLM_OK, "");
  if (count < 0 || first_draw < 0)
    return glm::set_error(GLM_EINVAL, "count/first_draw must be >= 0");
  if (m < 1 || m >= (1ll << 31)) return glm::set_error(GLM_EINVAL, "m must be in [1, 2^31)");
  if (count > kNoAllocMaxCount)
    return glm::set_error(GLM_EINVAL,
                          "glm_sample_indices_noalloc: count exceeds the static scratch of "
                          "GLM_SAMPLE_NOALLOC_MAX (1048576) indices");
  if (count == 0) return GLM_OK;
  if (!out) return glm::set_error(GLM_EINVAL, "out is NULL");
  {  // the output must be host memory (a device pointer would make the copy
     // below a device-to-device copy described as device-to-host)
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, out) != cudaSuccess) {
      cudaGetLastError();
    } else if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
      return glm::set_error(GLM_EINVAL, "glm_sample_indices_noalloc: out must be host memory");
    }
  }
  int32_t *d = nullptr;
  GLM_TRY(scratch_for_current_device(&d));
  GLM_TRY(glm::launch_sample(seed, problem, first_draw, count, m, d, 0));
  GLM_CUDA_TRY(cudaMemcpy(out, d, (size_t)count * 4, cudaMemcpyDeviceToHost));
  return GLM_OK;
}
