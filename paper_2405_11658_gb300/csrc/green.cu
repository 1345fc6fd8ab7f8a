// green.cu -- contexts restricted to a subset of the GPU's SMs.
//
// A green context (CUDA driver API) is the device's primary context with a
// provisioned share of its SMs: kernels launched on its streams run on those
// SMs only, while memory stays shared with the primary context.  A leiden_ctx
// created on one lets the whole pipeline run on k SMs, the GPU counterpart of
// running the paper's implementation on fewer threads (Sec. 5.2, strong
// scaling).  The driver entry points are resolved through the runtime
// (cudaGetDriverEntryPointByVersion), so the library needs no link-time
// dependency on the driver library.
#include <cuda.h>
#include <cuda_runtime.h>

#include "internal.h"

namespace lk {

namespace {

struct Api {
  CUresult (*DeviceGetDevResource)(CUdevice, CUdevResource *, CUdevResourceType) = nullptr;
  CUresult (*DevSmResourceSplitByCount)(CUdevResource *, unsigned int *, const CUdevResource *, CUdevResource *,
                                        unsigned int, unsigned int) = nullptr;
  CUresult (*DevResourceGenerateDesc)(CUdevResourceDesc *, CUdevResource *, unsigned int) = nullptr;
  CUresult (*GreenCtxCreate)(CUgreenCtx *, CUdevResourceDesc, CUdevice, unsigned int) = nullptr;
  CUresult (*GreenCtxDestroy)(CUgreenCtx) = nullptr;
  CUresult (*CtxFromGreenCtx)(CUcontext *, CUgreenCtx) = nullptr;
  CUresult (*CtxPushCurrent)(CUcontext) = nullptr;
  CUresult (*CtxPopCurrent)(CUcontext *) = nullptr;
  CUresult (*DeviceGet)(CUdevice *, int) = nullptr;
  bool ok = false;
};

template <typename F>
bool entry(const char *name, F *fn) {
  cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
  void *p = nullptr;
  if (cudaGetDriverEntryPointByVersion(name, &p, 12040, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !p) {
    cudaGetLastError();
    return false;
  }
  *fn = reinterpret_cast<F>(p);
  return true;
}

const Api &api() {
  static Api a = [] {
    Api x;
    x.ok = entry("cuDeviceGetDevResource", &x.DeviceGetDevResource) &&
           entry("cuDevSmResourceSplitByCount", &x.DevSmResourceSplitByCount) &&
           entry("cuDevResourceGenerateDesc", &x.DevResourceGenerateDesc) &&
           entry("cuGreenCtxCreate", &x.GreenCtxCreate) && entry("cuGreenCtxDestroy", &x.GreenCtxDestroy) &&
           entry("cuCtxFromGreenCtx", &x.CtxFromGreenCtx) && entry("cuCtxPushCurrent", &x.CtxPushCurrent) &&
           entry("cuCtxPopCurrent", &x.CtxPopCurrent) && entry("cuDeviceGet", &x.DeviceGet);
    return x;
  }();
  return a;
}

}  // namespace

int green_create(int device, int sm_count, GreenCtx *out) {
  *out = GreenCtx{};
  const Api &a = api();
  if (!a.ok) return LEIDEN_ECUDA;
  if (cudaSetDevice(device) != cudaSuccess || cudaFree(nullptr) != cudaSuccess) {  // primary context up
    cudaGetLastError();
    return LEIDEN_ECUDA;
  }
  CUdevice dev;
  if (a.DeviceGet(&dev, device) != CUDA_SUCCESS) return LEIDEN_ECUDA;
  CUdevResource all{}, part{}, rest{};
  if (a.DeviceGetDevResource(dev, &all, CU_DEV_RESOURCE_TYPE_SM) != CUDA_SUCCESS) return LEIDEN_ECUDA;
  if (sm_count < 1 || (unsigned)sm_count > all.sm.smCount) return LEIDEN_EINVAL;
  unsigned int groups = 1;
  if (a.DevSmResourceSplitByCount(&part, &groups, &all, &rest, 0, (unsigned)sm_count) != CUDA_SUCCESS ||
      groups < 1)
    return LEIDEN_EINVAL;
  CUdevResourceDesc desc;
  if (a.DevResourceGenerateDesc(&desc, &part, 1) != CUDA_SUCCESS) return LEIDEN_ECUDA;
  CUgreenCtx g;
  if (a.GreenCtxCreate(&g, desc, dev, CU_GREEN_CTX_DEFAULT_STREAM) != CUDA_SUCCESS) return LEIDEN_ECUDA;
  CUcontext cu;
  if (a.CtxFromGreenCtx(&cu, g) != CUDA_SUCCESS) {
    a.GreenCtxDestroy(g);
    return LEIDEN_ECUDA;
  }
  out->green = g;
  out->cu = cu;
  out->sms = (int)part.sm.smCount;
  return LEIDEN_OK;
}

void green_destroy(GreenCtx *g) {
  if (g->green) api().GreenCtxDestroy(static_cast<CUgreenCtx>(g->green));
  *g = GreenCtx{};
}

bool green_push(const GreenCtx &g) {
  return g.cu && api().CtxPushCurrent(static_cast<CUcontext>(g.cu)) == CUDA_SUCCESS;
}

void green_pop() {
  CUcontext prev;
  api().CtxPopCurrent(&prev);
}

}  // namespace lk
