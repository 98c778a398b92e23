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

template <int NP, class T>
__device__ __forceinline__ void dispatch_mv(const PdgPass& p, int mv, int bid, double* sm) {
  switch (mv) {
    case MV_ADV: pass_body<NP, MV_ADV, T>(p, bid, sm); break;
    case MV_SW: pass_body<NP, MV_SW, T>(p, bid, sm); break;
    case MV_EU2: pass_body<NP, MV_EU2, T>(p, bid, sm); break;
    case MV_EU3: pass_body<NP, MV_EU3, T>(p, bid, sm); break;
    case MV_EU1: pass_body<NP, MV_EU1, T>(p, bid, sm); break;
    default: pass_body<NP, MV_NONE, T>(p, bid, sm); break;
  }
}

template <class T>
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
    const int np = sp->npl / sp->ncell;
    const int mv = sp->mv;
    switch (np) {
      case 2: dispatch_mv<2, T>(*sp, mv, bid, carry); break;
      case 3: dispatch_mv<3, T>(*sp, mv, bid, carry); break;
      case 4: dispatch_mv<4, T>(*sp, mv, bid, carry); break;
      case 5: dispatch_mv<5, T>(*sp, mv, bid, carry); break;
      default: break;
    }
    __syncthreads();  // s_item / s_desc / descriptor are rewritten by the next item
  }
}

template <class T>
int batch_grid_t(size_t smem, int* grid) {
  int dev = 0, sms = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return (int)e;
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(batch_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
  }
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_kernel<T>, kBatchThreads, smem);
  if (e != cudaSuccess) return (int)e;
  if (per < 1) per = 1;
  *grid = sms * per;
  return 0;
}

template <class T>
int launch_batch_t(const PdgPass* d_descs, const int* d_ent_desc, const long long* d_ent_start, int nent,
                   long long total, unsigned long long* d_counter, int grid, size_t smem, void* stream) {
  if (nent <= 0 || total <= 0) return 0;
  batch_kernel<T><<<grid, kBatchThreads, smem, (cudaStream_t)stream>>>(d_descs, d_ent_desc, d_ent_start, nent,
                                                                        total, d_counter);
  return (int)cudaGetLastError();
}

}  // namespace pdgdev
