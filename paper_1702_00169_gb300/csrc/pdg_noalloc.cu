// pdg_get_w_noalloc: the moments w = P f read into host memory without any device
// allocation.
//
// pdg_get_w with a host destination stages w in a device buffer that the context
// allocates with cudaMalloc on first use.  Some callers cannot allow that: code that
// runs while a custom or pooled allocator owns the device memory budget, a process
// whose allocation calls are intercepted or forbidden after start-up, or a caller
// that must not grow the context's footprint between two checkpoints.  This variant
// stages w in a fixed array compiled into the library instead.
//
// The staging array is a file-scope __device__ array of PDG_NOALLOC_W_MAX doubles
// (8 MiB).  Every GPU that loads the library holds it until the process exits.  In
// host code the array's name is only a host-side stand-in, so its device address is
// looked up once per device with cudaGetSymbolAddress (on the first call on that
// device, with that device current) and passed to the kernel.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/pdg.h"
#include "pdg_internal.h"

namespace {

constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_w_scratch[PDG_NOALLOC_W_MAX];

std::mutex g_mu;
double* g_addr[kMaxDevices] = {nullptr};

// Writes every element of [0, m * P) of `scratch`: nothing has to start at zero.
__global__ void get_w_scratch_kernel(const double* __restrict__ f, double* __restrict__ scratch, long long P,
                                     int m, int nv) {
  for (long long pt = blockIdx.x * (long long)blockDim.x + threadIdx.x; pt < P;
       pt += (long long)gridDim.x * blockDim.x) {
    for (int k = 0; k < m; ++k) {
      double s = 0.0;
      for (int i = 0; i < nv; ++i) s += f[(long long)(k * nv + i) * P + pt];
      scratch[(long long)k * P + pt] = s;
    }
  }
}

// Device address of the staging array on the current device (looked up once per device).
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_w_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int pdg_get_w_noalloc(pdg_ctx* c, double* out, size_t len) try {
  if (!c) return PDG_ERR_ARG;
  PdgStateView v;
  if (!pdg_internal_view(c, &v)) return pdg_internal_fail(c, PDG_ERR_STATE, "no state");
  if (!out) return pdg_internal_fail(c, PDG_ERR_ARG, "out is NULL");
  if (v.prec != PDG_PREC_FP64)
    return pdg_internal_fail(c, PDG_ERR_UNSUPPORTED, "pdg_get_w_noalloc reads FP64 states only");
  if (v.m * v.nv != v.nf)
    return pdg_internal_fail(c, PDG_ERR_UNSUPPORTED, "pdg_get_w_noalloc reads vectorial (DnQ2n) states only");
  const size_t need = (size_t)v.m * (size_t)v.npoints;
  if (len != need) return pdg_internal_fail(c, PDG_ERR_ARG, "w length mismatch");
  if (need > (size_t)PDG_NOALLOC_W_MAX)
    return pdg_internal_fail(c, PDG_ERR_ARG,
                             "pdg_get_w_noalloc: w has " + std::to_string(need) +
                                 " doubles, more than the static staging array of " +
                                 std::to_string((long long)PDG_NOALLOC_W_MAX) + " doubles; use pdg_get_w");
  double* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess)
    return pdg_internal_fail(c, PDG_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  const int threads = 256;
  long long blocks = ((long long)v.npoints + threads - 1) / threads;
  if (blocks > 32LL * pdg_sm_count()) blocks = 32LL * pdg_sm_count();
  if (blocks < 1) blocks = 1;
  get_w_scratch_kernel<<<(int)blocks, threads, 0, v.stream>>>(v.f, scratch, v.npoints, v.m, v.nv);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, scratch, sizeof(double) * need, cudaMemcpyDeviceToHost, v.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(v.stream);
  if (e != cudaSuccess)
    return pdg_internal_fail(c, PDG_ERR_CUDA, std::string("pdg_get_w_noalloc: ") + cudaGetErrorString(e));
  return PDG_OK;
} catch (...) {
  return pdgapi::abi_exception(nullptr);
}
