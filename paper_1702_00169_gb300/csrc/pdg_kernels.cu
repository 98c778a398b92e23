// FP64 instantiation of the pass kernels (see pdg_pass_kernels.cuh), the dispatch by
// precision, and the state kernels at the API boundary (equilibrium start, moments,
// FP64 <-> double-float conversion).
#include <atomic>
#include <cuda_runtime.h>

#include "pdg_pass_kernels.cuh"

int pdg_launch_pass_df(const PdgPass& p, void* stream);

// Streaming multiprocessors of the current device, read once per device from its
// properties; 152 (GB300) when no device answers (host-only use of the planners).
int pdg_sm_count() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cached[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    cudaGetLastError();
    return 152;
  }
  int v = cached[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
    cudaGetLastError();
    return 152;
  }
  cached[dev].store(v, std::memory_order_relaxed);
  return v;
}

namespace {
using namespace pdgdev;

// f := f^eq(w) in place: w_k sits (as FP64) in field slot k; a thread reads all w_k of
// its point before writing.  Populations summing to w_k with zero first moment pass
// through one collision with omega = 1 (the model M1 carries the omega = 1 constants),
// which yields f^eq(w) with the sweep's own arithmetic.
template <int MV, class T>
__global__ void set_feq_kernel(double* __restrict__ f, long long P, long long n, const __grid_constant__ PdgModel M1) {
  constexpr int NF = NFields<MV>::value;
  const int m = M1.m, nv = M1.nv;
  for (long long pt = blockIdx.x * (long long)blockDim.x + threadIdx.x; pt < n;
       pt += (long long)gridDim.x * blockDim.x) {
    double w[PDG_MAXM];
#pragma unroll
    for (int k = 0; k < PDG_MAXM; ++k)
      if (k < m) w[k] = f[(long long)k * P + pt];
    T v[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) v[k] = zero<T>();
    for (int k = 0; k < m; ++k) v[k * nv] = from_double<T>(w[k]);
    collide<MV, T>(v, M1);
#pragma unroll
    for (int k = 0; k < NF; ++k)
      if (k < m * nv) st(f + (long long)k * P + pt, v[k]);
  }
}

template <class T>
__global__ void get_w_kernel(const double* __restrict__ f, double* __restrict__ w, long long P, long long n,
                             int m, int nv) {
  for (long long pt = blockIdx.x * (long long)blockDim.x + threadIdx.x; pt < n;
       pt += (long long)gridDim.x * blockDim.x) {
    for (int k = 0; k < m; ++k) {
      T s = zero<T>();
      for (int i = 0; i < nv; ++i) s = s + ld<T>(f + (long long)(k * nv + i) * P + pt);
      w[(long long)k * P + pt] = to_double(s);
    }
  }
}

// D2Q9: w = (rho, rho u_x, rho u_y) in slots 0-2 -> f = f^eq(w) in slots 0-8 (M1 has
// omega = 1, so the relaxation returns f^eq).
template <class T>
__global__ void set_feq_q9_kernel(double* __restrict__ f, long long P, long long n, const __grid_constant__ PdgModel M1) {
  for (long long pt = blockIdx.x * (long long)blockDim.x + threadIdx.x; pt < n;
       pt += (long long)gridDim.x * blockDim.x) {
    const T rho = from_double<T>(f[pt]);
    const T ilam = PDG_K(T, M1, PDG_K_ILAM);
    const T jx = from_double<T>(f[P + pt]) * ilam, jy = from_double<T>(f[2 * P + pt]) * ilam;
    T v[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) v[i] = zero<T>();
    d2q9_relax<T>(v, rho, jx, jy, M1);
#pragma unroll
    for (int i = 0; i < 9; ++i) st(f + (long long)i * P + pt, v[i]);
  }
}

// D2Q9: w = P f = (sum f_i, lambda sum f_i xi_i).
template <class T>
__global__ void get_w_q9_kernel(const double* __restrict__ f, double* __restrict__ w, long long P, long long n,
                                const __grid_constant__ PdgModel M) {
  for (long long pt = blockIdx.x * (long long)blockDim.x + threadIdx.x; pt < n;
       pt += (long long)gridDim.x * blockDim.x) {
    T v[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) v[i] = ld<T>(f + (long long)i * P + pt);
    const T rho = (((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]))) + v[8];
    const T jx = (v[1] - v[3]) + ((v[5] - v[6]) + (v[8] - v[7]));
    const T jy = (v[2] - v[4]) + ((v[5] + v[6]) - (v[7] + v[8]));
    const T lam = PDG_K(T, M, PDG_K_LAM);
    w[pt] = to_double(rho);
    w[P + pt] = to_double(lam * jx);
    w[2 * P + pt] = to_double(lam * jy);
  }
}

// D3Q19: w = (rho, rho u) in slots 0-3 -> f = f^eq(w) in slots 0-18.
template <class T>
__global__ void set_feq_q19_kernel(double* __restrict__ f, long long P, long long n, const __grid_constant__ PdgModel M1) {
  for (long long pt = blockIdx.x * (long long)blockDim.x + threadIdx.x; pt < n;
       pt += (long long)gridDim.x * blockDim.x) {
    const T rho = from_double<T>(f[pt]);
    const T ilam = PDG_K(T, M1, PDG_K_ILAM);
    const T jx = from_double<T>(f[P + pt]) * ilam, jy = from_double<T>(f[2 * P + pt]) * ilam;
    const T jz = from_double<T>(f[3 * P + pt]) * ilam;
    T e[19];
    d3q19_e<T>(rho, jx, jy, jz, M1, e);
    const T a0 = PDG_K(T, M1, PDG_K_Q9W0) * rho, a1 = PDG_K(T, M1, PDG_K_Q9W1) * rho;
    const T a2 = PDG_K(T, M1, PDG_K_Q9W2) * rho;
#pragma unroll
    for (int i = 0; i < 19; ++i) st(f + (long long)i * P + pt, (i == 0 ? a0 : (i < 7 ? a1 : a2)) * e[i]);
  }
}

// D3Q19: w = P f = (sum f_i, lambda sum f_i xi_i).
template <class T>
__global__ void get_w_q19_kernel(const double* __restrict__ f, double* __restrict__ w, long long P, long long n,
                                 const __grid_constant__ PdgModel M) {
  for (long long pt = blockIdx.x * (long long)blockDim.x + threadIdx.x; pt < n;
       pt += (long long)gridDim.x * blockDim.x) {
    T v[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) v[i] = ld<T>(f + (long long)i * P + pt);
    T rho, jx, jy, jz;
    d3q19_moments<T>(v, &rho, &jx, &jy, &jz);
    const T lam = PDG_K(T, M, PDG_K_LAM);
    w[pt] = to_double(rho);
    w[P + pt] = to_double(lam * jx);
    w[2 * P + pt] = to_double(lam * jy);
    w[3 * P + pt] = to_double(lam * jz);
  }
}

// D3Q15 / D3Q27: w = (rho, rho u) in slots 0-3 -> f = f^eq(w).  rho goes to the rest
// population and +-j_a/2 to the two axis populations of axis a (moments (rho, j) exactly);
// one relaxation with omega = 1 (M1) then returns f^eq with the sweep's own arithmetic.
template <class T, bool EDGES>
__global__ void set_feq_corner_kernel(double* __restrict__ f, long long P, long long n, const __grid_constant__ PdgModel M1) {
  constexpr int NV = EDGES ? 27 : 15;
  for (long long pt = blockIdx.x * (long long)blockDim.x + threadIdx.x; pt < n;
       pt += (long long)gridDim.x * blockDim.x) {
    const T ilam = PDG_K(T, M1, PDG_K_ILAM), hf = from_double<T>(0.5);
    T v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = zero<T>();
    v[0] = from_double<T>(f[pt]);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const T ja = from_double<T>(f[(a + 1) * P + pt]) * ilam * hf;
      v[1 + 2 * a] = ja;
      v[2 + 2 * a] = -ja;
    }
    d3q_lattice_collide<T, EDGES, true>(v, M1);
#pragma unroll
    for (int i = 0; i < NV; ++i) st(f + (long long)i * P + pt, v[i]);
  }
}

// D3Q15 / D3Q27: w = P f = (sum f_i, lambda sum f_i xi_i).
template <class T, bool EDGES>
__global__ void get_w_corner_kernel(const double* __restrict__ f, double* __restrict__ w, long long P, long long n,
                                    const __grid_constant__ PdgModel M) {
  constexpr int NV = EDGES ? 27 : 15, C0 = EDGES ? 19 : 7;
  for (long long pt = blockIdx.x * (long long)blockDim.x + threadIdx.x; pt < n;
       pt += (long long)gridDim.x * blockDim.x) {
    T v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = ld<T>(f + (long long)i * P + pt);
    T rho, jx, jy, jz;
    if constexpr (EDGES) {
      d3q19_moments<T>(v, &rho, &jx, &jy, &jz);
    } else {
      rho = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + v[6]);
      jx = v[1] - v[2];
      jy = v[3] - v[4];
      jz = v[5] - v[6];
    }
    T cr, cx, cy, cz;
    corner_moments<T>(v + C0, &cr, &cx, &cy, &cz);
    const T lam = PDG_K(T, M, PDG_K_LAM);
    w[pt] = to_double(rho + cr);
    w[P + pt] = to_double(lam * (jx + cx));
    w[2 * P + pt] = to_double(lam * (jy + cy));
    w[3 * P + pt] = to_double(lam * (jz + cz));
  }
}

__global__ void convert_kernel(double* __restrict__ f, long long n, int to_df) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (to_df) st(f + i, dd_from_double(f[i]));
    else f[i] = dd_to_double(ld<dd>(f + i));
  }
}

int grid_for(long long n, int threads) {
  long long blocks = (n + threads - 1) / threads;
  const long long cap = 32LL * pdg_sm_count();
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

template <int MV>
int launch_feq_t(double* f, long long P, long long p0, long long n, const PdgModel& m1, cudaStream_t st) {
  if (m1.prec == PDG_PREC_DF32)
    set_feq_kernel<MV, dd><<<grid_for(n, 256), 256, 0, st>>>(f + p0, P, n, m1);
  else
    set_feq_kernel<MV, double><<<grid_for(n, 256), 256, 0, st>>>(f + p0, P, n, m1);
  return (int)cudaGetLastError();
}

}  // namespace

int pdg_model_variant(const PdgModel& m) {
  switch (m.kind) {
    case PDG_MODEL_ADVECTION: return MV_ADV;
    case PDG_MODEL_SHALLOW_WATER: return MV_SW;
    case PDG_MODEL_EULER: return m.dim == 1 ? MV_EU1 : (m.dim == 2 ? MV_EU2 : MV_EU3);
    case PDG_MODEL_ISOTHERMAL_D2Q9: return MV_D2Q9;
    case PDG_MODEL_ISOTHERMAL_D3Q19: return MV_D3Q19;
    case PDG_MODEL_ISOTHERMAL_D3Q15: return MV_D3Q15;
    case PDG_MODEL_ISOTHERMAL_D3Q27: return MV_D3Q27;
  }
  return -1;
}

int pdg_launch_pass(const PdgPass& p, void* stream) {
  if (p.prec == PDG_PREC_DF32) return pdg_launch_pass_df(p, stream);
  return launch_pass_typed<double>(p, (cudaStream_t)stream);
}

int pdg_launch_set_feq(double* f, long long P, const PdgModel& m, void* stream) {
  return pdg_launch_set_feq_range(f, P, 0, P, m, stream);
}

int pdg_launch_set_feq_range(double* f, long long P, long long p0, long long n, const PdgModel& m, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  PdgModel m1 = m;
  m1.omega = 1.0;
  pdg_model_constants(&m1);
  switch (pdg_model_variant(m)) {
    case MV_ADV: return launch_feq_t<MV_ADV>(f, P, p0, n, m1, st);
    case MV_SW: return launch_feq_t<MV_SW>(f, P, p0, n, m1, st);
    case MV_EU1: return launch_feq_t<MV_EU1>(f, P, p0, n, m1, st);
    case MV_EU2: return launch_feq_t<MV_EU2>(f, P, p0, n, m1, st);
    case MV_EU3: return launch_feq_t<MV_EU3>(f, P, p0, n, m1, st);
    case MV_D2Q9:
      if (m1.prec == PDG_PREC_DF32)
        set_feq_q9_kernel<dd><<<grid_for(n, 256), 256, 0, st>>>(f + p0, P, n, m1);
      else
        set_feq_q9_kernel<double><<<grid_for(n, 256), 256, 0, st>>>(f + p0, P, n, m1);
      return (int)cudaGetLastError();
    case MV_D3Q19:
      if (m1.prec == PDG_PREC_DF32)
        set_feq_q19_kernel<dd><<<grid_for(n, 256), 256, 0, st>>>(f + p0, P, n, m1);
      else
        set_feq_q19_kernel<double><<<grid_for(n, 256), 256, 0, st>>>(f + p0, P, n, m1);
      return (int)cudaGetLastError();
    case MV_D3Q15:
      if (m1.prec == PDG_PREC_DF32)
        set_feq_corner_kernel<dd, false><<<grid_for(n, 256), 256, 0, st>>>(f + p0, P, n, m1);
      else
        set_feq_corner_kernel<double, false><<<grid_for(n, 256), 256, 0, st>>>(f + p0, P, n, m1);
      return (int)cudaGetLastError();
    case MV_D3Q27:
      if (m1.prec == PDG_PREC_DF32)
        set_feq_corner_kernel<dd, true><<<grid_for(n, 256), 256, 0, st>>>(f + p0, P, n, m1);
      else
        set_feq_corner_kernel<double, true><<<grid_for(n, 256), 256, 0, st>>>(f + p0, P, n, m1);
      return (int)cudaGetLastError();
  }
  return (int)cudaErrorInvalidValue;
}

int pdg_launch_get_w(const double* f, double* w, long long P, const PdgModel& m, void* stream) {
  return pdg_launch_get_w_range(f, w, P, 0, P, m, stream);
}

int pdg_launch_get_w_range(const double* f, double* w, long long P, long long p0, long long n, const PdgModel& m,
                           void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (m.kind == PDG_MODEL_ISOTHERMAL_D3Q19) {
    if (m.prec == PDG_PREC_DF32)
      get_w_q19_kernel<dd><<<grid_for(n, 256), 256, 0, st>>>(f + p0, w + p0, P, n, m);
    else
      get_w_q19_kernel<double><<<grid_for(n, 256), 256, 0, st>>>(f + p0, w + p0, P, n, m);
    return (int)cudaGetLastError();
  }
  if (m.kind == PDG_MODEL_ISOTHERMAL_D3Q15 || m.kind == PDG_MODEL_ISOTHERMAL_D3Q27) {
    const bool q27 = m.kind == PDG_MODEL_ISOTHERMAL_D3Q27;
    if (m.prec == PDG_PREC_DF32) {
      if (q27) get_w_corner_kernel<dd, true><<<grid_for(n, 256), 256, 0, st>>>(f + p0, w + p0, P, n, m);
      else get_w_corner_kernel<dd, false><<<grid_for(n, 256), 256, 0, st>>>(f + p0, w + p0, P, n, m);
    } else {
      if (q27) get_w_corner_kernel<double, true><<<grid_for(n, 256), 256, 0, st>>>(f + p0, w + p0, P, n, m);
      else get_w_corner_kernel<double, false><<<grid_for(n, 256), 256, 0, st>>>(f + p0, w + p0, P, n, m);
    }
    return (int)cudaGetLastError();
  }
  if (m.kind == PDG_MODEL_ISOTHERMAL_D2Q9) {
    if (m.prec == PDG_PREC_DF32)
      get_w_q9_kernel<dd><<<grid_for(n, 256), 256, 0, st>>>(f + p0, w + p0, P, n, m);
    else
      get_w_q9_kernel<double><<<grid_for(n, 256), 256, 0, st>>>(f + p0, w + p0, P, n, m);
    return (int)cudaGetLastError();
  }
  if (m.prec == PDG_PREC_DF32)
    get_w_kernel<dd><<<grid_for(n, 256), 256, 0, st>>>(f + p0, w + p0, P, n, m.m, m.nv);
  else
    get_w_kernel<double><<<grid_for(n, 256), 256, 0, st>>>(f + p0, w + p0, P, n, m.m, m.nv);
  return (int)cudaGetLastError();
}

int pdg_launch_convert(double* f, long long n, int to_df, void* stream) {
  convert_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(f, n, to_df);
  return (int)cudaGetLastError();
}
