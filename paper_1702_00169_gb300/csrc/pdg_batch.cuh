// Batched persistent kernel (templated on the number type; instantiated in
// pdg_batch.cu for FP64 and pdg_batch_df.cu for double-float).
//
// A stage is a list of entries (pass descriptor, number of thread-block work
// items).  Entries are sorted by the cost of one work item, largest first, and the
// persistent blocks claim work items in that order with an atomic counter, so
// the long items start first and the short ones fill the tail.  A work item is
// exactly one block of the single-mesh pass kernel (same lines, same segments,
// same arithmetic), so a mesh gives bitwise the same result alone or in a batch
// as long as its launch shape is the same.
#pragma once
#include <cuda_runtime.h>

#include "pdg_device.cuh"

namespace pdgdev {

constexpr int kBatchThreads = 256;
constexpr int kDescWords = (int)((sizeof(PdgPass) + 7) / 8);

template <int NP, int MV, class T>
__global__ void __launch_bounds__(kBatchThreads)
    batch_kernel(const PdgPass* __restrict__ descs, const int* __restrict__ ent_desc,
                 const long long* __restrict__ ent_start, int nent, long long total,
                 unsigned long long* counter) {
  extern __shared__ double smem[];
  __shared__ long long s_item;
  __shared__ int s_desc;
  PdgPass* sp = reinterpret_cast<PdgPass*>(smem);
  double* carry = smem + kDescWords;
  int loaded = -1;
  for (;;) {
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1ULL);
    __syncthreads();
    const long long g = s_item;
    if (g >= total) break;
    if (threadIdx.x == 0) {
      int lo = 0, hi = nent - 1;  // last entry with ent_start <= g
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ent_start[mid] <= g) lo = mid; else hi = mid - 1;
      }
      s_desc = lo;
    }
    __syncthreads();
    const int e = s_desc;
    const int di = ent_desc[e];
    const int bid = (int)(g - ent_start[e]);
    if (di != loaded) {
      const long long* src = reinterpret_cast<const long long*>(descs + di);
      long long* dst = reinterpret_cast<long long*>(smem);
      for (int i = threadIdx.x; i < kDescWords; i += blockDim.x) dst[i] = src[i];
      loaded = di;
      __syncthreads();
    }
    pass_body<NP, MV, T>(*sp, bid, carry);
    __syncthreads();  // s_item / s_desc / descriptor are rewritten by the next item
  }
}

// Host side: the kernel of one (degree NP, model variant MV) and its persistent grid.
template <int NP, int MV, class T>
int launch_variant(const PdgPass* d_descs, const int* d_ent_desc, const long long* d_ent_start, int nent,
                   long long total, unsigned long long* d_counter, size_t smem, cudaStream_t st) {
  static int grid = 0;  // blocks per SM x SMs, computed once per process and variant
  auto kern = batch_kernel<NP, MV, T>;
  if (grid == 0) {
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess && smem > 48 * 1024)
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kBatchThreads, smem);
    if (e != cudaSuccess) return (int)e;
    grid = sms * (per < 1 ? 1 : per);
  }
  kern<<<grid, kBatchThreads, smem, st>>>(d_descs, d_ent_desc, d_ent_start, nent, total, d_counter);
  return (int)cudaGetLastError();
}

template <int NP, class T>
int launch_np(int mv, const PdgPass* a, const int* b, const long long* c, int n, long long t,
              unsigned long long* k, size_t smem, cudaStream_t st) {
  switch (mv) {
    case MV_ADV: return launch_variant<NP, MV_ADV, T>(a, b, c, n, t, k, smem, st);
    case MV_SW: return launch_variant<NP, MV_SW, T>(a, b, c, n, t, k, smem, st);
    case MV_EU1: return launch_variant<NP, MV_EU1, T>(a, b, c, n, t, k, smem, st);
    case MV_EU2: return launch_variant<NP, MV_EU2, T>(a, b, c, n, t, k, smem, st);
    case MV_EU3: return launch_variant<NP, MV_EU3, T>(a, b, c, n, t, k, smem, st);
    case MV_NONE: return launch_variant<NP, MV_NONE, T>(a, b, c, n, t, k, smem, st);
  }
  return (int)cudaErrorInvalidValue;
}

template <class T>
int launch_batch_t(int np, int mv, const PdgPass* d_descs, const int* d_ent_desc, const long long* d_ent_start,
                   int nent, long long total, unsigned long long* d_counter, size_t smem, void* stream) {
  if (nent <= 0 || total <= 0) return 0;
  cudaStream_t st = (cudaStream_t)stream;
  switch (np) {
    case 2: return launch_np<2, T>(mv, d_descs, d_ent_desc, d_ent_start, nent, total, d_counter, smem, st);
    case 3: return launch_np<3, T>(mv, d_descs, d_ent_desc, d_ent_start, nent, total, d_counter, smem, st);
    case 4: return launch_np<4, T>(mv, d_descs, d_ent_desc, d_ent_start, nent, total, d_counter, smem, st);
    case 5: return launch_np<5, T>(mv, d_descs, d_ent_desc, d_ent_start, nent, total, d_counter, smem, st);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace pdgdev
