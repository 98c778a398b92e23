// Pass kernel and its launcher.  The kernels are instantiated in pdg_pass_inst.cu (one
// object per group of model variants and number type); pdg_kernels.cu and
// pdg_kernels_df.cu hold the dispatch by number type.
//
// pass_kernel<NP, MV, T> runs one "pass" over whole periodic lines of one axis:
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
#pragma once
#include <cuda_runtime.h>

#include "pdg_device.cuh"

namespace pdgdev {

template <int NP, int MV, class T>
__global__ void __launch_bounds__(512) pass_kernel(const __grid_constant__ PdgPass p) {
  extern __shared__ double sm[];
  pass_body<NP, MV, T>(p, blockIdx.x, sm);
}

// The 3-D lattices (15 to 27 populations live in the collision): the same body, compiled
// for one block of 512 threads per SM, so that ptxas may use all 128 registers a thread
// can have there instead of spilling.
template <int NP, int MV, class T>
__global__ void __launch_bounds__(512, 1) pass_kernel_lat(const __grid_constant__ PdgPass p) {
  extern __shared__ double sm[];
  pass_body<NP, MV, T>(p, blockIdx.x, sm);
}

template <int NP, int MV, class T>
int launch_pass_t(const PdgPass& p, cudaStream_t st) {
  const int threads = p.lpb * p.nseg * p.ngroup;
  const size_t smem = sizeof(double) * 3 * (size_t)p.ntf * p.nseg * p.lpb;
  const int blocks = p.nblocks > 0 ? p.nblocks : (p.nlines + p.lpb - 1) / p.lpb;
  auto go = [&](auto kern) -> int {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return (int)e;
    }
    kern<<<blocks, threads, smem, st>>>(p);
    return (int)cudaGetLastError();
  };
  if constexpr (MV == MV_D3Q19 || MV == MV_D3Q15 || MV == MV_D3Q27)
    return go(pass_kernel_lat<NP, MV, T>);
  else
    return go(pass_kernel<NP, MV, T>);
}

// All degrees of one model variant.  Explicitly instantiated per (variant, number type) in
// pdg_pass_inst.cu, which is compiled once per group of variants (build.py), so the
// instantiations compile in parallel; every other translation unit sees the extern
// declarations below.
template <int MV, class T>
int launch_pass_mv(const PdgPass& p, cudaStream_t st) {
  switch (p.ncell > 0 ? p.npl / p.ncell : 0) {
    case 2: return launch_pass_t<2, MV, T>(p, st);
    case 3: return launch_pass_t<3, MV, T>(p, st);
    case 4: return launch_pass_t<4, MV, T>(p, st);
    case 5: return launch_pass_t<5, MV, T>(p, st);
  }
  return (int)cudaErrorInvalidValue;
}

#define PDG_PASS_EXTERN(MV)                                                       \
  extern template int launch_pass_mv<MV, double>(const PdgPass&, cudaStream_t); \
  extern template int launch_pass_mv<MV, dd>(const PdgPass&, cudaStream_t);
PDG_PASS_EXTERN(MV_NONE)
PDG_PASS_EXTERN(MV_ADV)
PDG_PASS_EXTERN(MV_SW)
PDG_PASS_EXTERN(MV_EU1)
PDG_PASS_EXTERN(MV_EU2)
PDG_PASS_EXTERN(MV_EU3)
PDG_PASS_EXTERN(MV_D2Q9)
PDG_PASS_EXTERN(MV_D3Q19)
PDG_PASS_EXTERN(MV_D3Q15)
PDG_PASS_EXTERN(MV_D3Q27)
#undef PDG_PASS_EXTERN

template <class T>
int launch_pass_typed(const PdgPass& p, cudaStream_t st) {
  switch (p.mv) {
    case MV_NONE: return launch_pass_mv<MV_NONE, T>(p, st);
    case MV_ADV: return launch_pass_mv<MV_ADV, T>(p, st);
    case MV_SW: return launch_pass_mv<MV_SW, T>(p, st);
    case MV_EU1: return launch_pass_mv<MV_EU1, T>(p, st);
    case MV_EU2: return launch_pass_mv<MV_EU2, T>(p, st);
    case MV_EU3: return launch_pass_mv<MV_EU3, T>(p, st);
    case MV_D2Q9: return launch_pass_mv<MV_D2Q9, T>(p, st);
    case MV_D3Q19: return launch_pass_mv<MV_D3Q19, T>(p, st);
    case MV_D3Q15: return launch_pass_mv<MV_D3Q15, T>(p, st);
    case MV_D3Q27: return launch_pass_mv<MV_D3Q27, T>(p, st);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace pdgdev
