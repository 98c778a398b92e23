// Measured FMA throughput of the current device: the denominators of the "alu" roofline
// of the FP64 kernels (FP64 pipe) and of the double-float kernels (FP32 pipe).
//
// Every thread runs kChains independent multiply-add chains x <- x * a + b for `iters`
// iterations.  With a = 1 - 2^-20 and b = 2^-30 the chains converge towards b / (1 - a)
// = 2^-10 and never overflow, underflow or reach a fixed point that the compiler could
// know, so every FMA is executed.  The grid is 4 blocks of 256 threads per SM (1024
// resident threads, 32 warps: enough independent chains to hide the FMA latency).  One
// value per thread is stored so that nothing is dead code.
#include <cuda_runtime.h>

#include "../../include/pdg.h"
#include "pdg_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <class T>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(T* out, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * (long long)blockDim.x + threadIdx.x] = s;
}

template <class T>
int measure(double* tflops, double* ms_out, cudaStream_t st) {
  const int sms = pdg_sm_count();
  const int blocks = 4 * sms;
  const int iters = sizeof(T) == 8 ? 4096 : 65536;
  T* out = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&out, sizeof(T) * (size_t)blocks * kThreads, st);
  if (e != cudaSuccess) return PDG_ERR_OOM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float best = 1e30f;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const T a = (T)(1.0 - 1.0 / 1048576.0), b = (T)(1.0 / 1073741824.0);
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first run warms up
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
      fma_chain_kernel<T><<<blocks, kThreads, 0, st>>>(out, iters, a, b);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && ms < best) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(out, st);
  if (e != cudaSuccess) return PDG_ERR_CUDA;
  const double flops = 2.0 * kChains * (double)iters * blocks * kThreads;
  if (tflops) *tflops = flops / (best * 1e-3) / 1e12;
  if (ms_out) *ms_out = best;
  return PDG_OK;
}

}  // namespace

extern "C" int pdg_measure_fma_peak(int fp64, double* tflops, double* ms, void* stream) try {
  if (!tflops) return PDG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int r = fp64 ? measure<double>(tflops, ms, st) : measure<float>(tflops, ms, st);
  if (r != PDG_OK) cudaGetLastError();
  return r;
} catch (...) {
  return pdgapi::abi_exception(nullptr);
}
