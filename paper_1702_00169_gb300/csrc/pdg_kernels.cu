// CUDA kernels (sm_103a, FP64) of the PDG hot path.
//
// pass_kernel<NP, MV> runs one "pass" over whole periodic lines of one axis:
// a short list of operations chosen from
//   T  the theta transport sub-step of eq. (3.11) (exact periodic solve), applied
//      to the 2m populations whose velocity is along the pass axis;
//   C  the collision of eq. (3.12), f <- omega f^eq(w) + (1 - omega) f with
//      w = P f (eq. (2.2)), applied to all populations of every point of the tile.
// A thread block owns `lpb` complete lines (all populations at those points), so
// every operation is done in place and the exact periodic closure needs no
// global synchronisation.  Inside a block, each line is cut into `nseg` segments;
// a segment's inflow value is obtained from a first pass over (the end of) the
// upwind segment -- the affine aggregate of the scalar recurrence
// x_c = alpha_c + beta x_{c-1} -- then the segment is swept once more to write
// the new values.  This replaces the topological ordering and wavefronts of
// Section 4.1-4.2 (a periodic line is a cycle, not a DAG) by an exact cyclic
// solve:
//   * "full" mode: segment aggregates Y_s cover the whole segment and the ring
//     is closed exactly, x = sum_j (prod beta^len) Y_{s-1-j} / (1 - beta^N);
//   * "window" mode (|beta|^W <= 2^-60 with W <= segment length): Y_{s-1} taken
//     over the last W cells equals the inflow value to within 2^-60 relative.
#include <cuda_runtime.h>

#include "pdg_device.cuh"

namespace {
using namespace pdgdev;

template <int NP, int MV>
__global__ void __launch_bounds__(512) pass_kernel(const __grid_constant__ PdgPass p) {
  extern __shared__ double sm[];
  pass_body<NP, MV>(p, blockIdx.x, sm);
}

// ---------------------------------------------------------------------------
template <int MV>
__global__ void set_feq_kernel(double* __restrict__ f, long long P, const __grid_constant__ PdgModel M) {
  constexpr int NF = NFields<MV>::value;
  const int m = M.m, nv = M.nv;
  for (long long pt = blockIdx.x * (long long)blockDim.x + threadIdx.x; pt < P;
       pt += (long long)gridDim.x * blockDim.x) {
    // w_k sits in field slot k (copied there by the host); read all before writing.
    double w[PDG_MAXM];
#pragma unroll
    for (int k = 0; k < PDG_MAXM; ++k)
      if (k < m) w[k] = f[(long long)k * P + pt];
    // f^eq: start from populations that sum to w_k with zero first moment, then one
    // collision with omega = 1 turns them into f^eq(w) exactly as in the sweep.
    double v[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) v[k] = 0.0;
    for (int k = 0; k < m; ++k) v[k * nv] = w[k];
    PdgModel M1 = M;
    M1.omega = 1.0;
    collide<MV>(v, M1);
#pragma unroll
    for (int k = 0; k < NF; ++k)
      if (k < m * nv) f[(long long)k * P + pt] = v[k];
  }
}

__global__ void get_w_kernel(const double* __restrict__ f, double* __restrict__ w, long long P, int m,
                             int nv) {
  for (long long pt = blockIdx.x * (long long)blockDim.x + threadIdx.x; pt < P;
       pt += (long long)gridDim.x * blockDim.x) {
    for (int k = 0; k < m; ++k) {
      double s = 0.0;
      for (int i = 0; i < nv; ++i) s += f[(long long)(k * nv + i) * P + pt];
      w[(long long)k * P + pt] = s;
    }
  }
}

template <int NP, int MV>
int launch_pass_t(const PdgPass& p, cudaStream_t st) {
  const int threads = p.lpb * p.nseg * p.ngroup;
  const size_t smem = sizeof(double) * 2 * (size_t)p.ntf * p.nseg * p.lpb;
  auto kern = pass_kernel<NP, MV>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
  }
  const int blocks = (p.nlines + p.lpb - 1) / p.lpb;
  kern<<<blocks, threads, smem, st>>>(p);
  return (int)cudaGetLastError();
}

template <int NP>
int launch_pass_np(const PdgPass& p, cudaStream_t st) {
  switch (p.mv) {
    case MV_NONE: return launch_pass_t<NP, MV_NONE>(p, st);
    case MV_ADV: return launch_pass_t<NP, MV_ADV>(p, st);
    case MV_SW: return launch_pass_t<NP, MV_SW>(p, st);
    case MV_EU1: return launch_pass_t<NP, MV_EU1>(p, st);
    case MV_EU2: return launch_pass_t<NP, MV_EU2>(p, st);
    case MV_EU3: return launch_pass_t<NP, MV_EU3>(p, st);
  }
  return (int)cudaErrorInvalidValue;
}

template <int MV>
int launch_feq_t(double* f, long long P, const PdgModel& m, cudaStream_t st) {
  const int threads = 256;
  long long blocks = (P + threads - 1) / threads;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks < 1) blocks = 1;
  set_feq_kernel<MV><<<(int)blocks, threads, 0, st>>>(f, P, m);
  return (int)cudaGetLastError();
}

}  // namespace

int pdg_model_variant(const PdgModel& m) {
  switch (m.kind) {
    case PDG_MODEL_ADVECTION: return MV_ADV;
    case PDG_MODEL_SHALLOW_WATER: return MV_SW;
    case PDG_MODEL_EULER: return m.dim == 1 ? MV_EU1 : (m.dim == 2 ? MV_EU2 : MV_EU3);
  }
  return -1;
}

int pdg_launch_pass(const PdgPass& p, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  switch (p.ncell > 0 ? p.npl / p.ncell : 0) {
    case 2: return launch_pass_np<2>(p, st);
    case 3: return launch_pass_np<3>(p, st);
    case 4: return launch_pass_np<4>(p, st);
    case 5: return launch_pass_np<5>(p, st);
  }
  return (int)cudaErrorInvalidValue;
}

int pdg_launch_set_feq(double* f, long long P, const PdgModel& m, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  switch (pdg_model_variant(m)) {
    case MV_ADV: return launch_feq_t<MV_ADV>(f, P, m, st);
    case MV_SW: return launch_feq_t<MV_SW>(f, P, m, st);
    case MV_EU1: return launch_feq_t<MV_EU1>(f, P, m, st);
    case MV_EU2: return launch_feq_t<MV_EU2>(f, P, m, st);
    case MV_EU3: return launch_feq_t<MV_EU3>(f, P, m, st);
  }
  return (int)cudaErrorInvalidValue;
}

int pdg_launch_get_w(const double* f, double* w, long long P, const PdgModel& m, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const int threads = 256;
  long long blocks = (P + threads - 1) / threads;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks < 1) blocks = 1;
  get_w_kernel<<<(int)blocks, threads, 0, st>>>(f, w, P, m.m, m.nv);
  return (int)cudaGetLastError();
}
