// Pass kernel and its launcher, instantiated once per number type (FP64 in
// pdg_kernels.cu, double-float in pdg_kernels_df.cu) so the two compile in parallel.
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

template <int NP, int MV, class T>
int launch_pass_t(const PdgPass& p, cudaStream_t st) {
  const int threads = p.lpb * p.nseg * p.ngroup;
  const size_t smem = sizeof(double) * 3 * (size_t)p.ntf * p.nseg * p.lpb;
  auto kern = pass_kernel<NP, MV, T>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
  }
  const int blocks = p.nblocks > 0 ? p.nblocks : (p.nlines + p.lpb - 1) / p.lpb;
  kern<<<blocks, threads, smem, st>>>(p);
  return (int)cudaGetLastError();
}

template <int NP, class T>
int launch_pass_np(const PdgPass& p, cudaStream_t st) {
  switch (p.mv) {
    case MV_NONE: return launch_pass_t<NP, MV_NONE, T>(p, st);
    case MV_ADV: return launch_pass_t<NP, MV_ADV, T>(p, st);
    case MV_SW: return launch_pass_t<NP, MV_SW, T>(p, st);
    case MV_EU1: return launch_pass_t<NP, MV_EU1, T>(p, st);
    case MV_EU2: return launch_pass_t<NP, MV_EU2, T>(p, st);
    case MV_EU3: return launch_pass_t<NP, MV_EU3, T>(p, st);
    case MV_D2Q9: return launch_pass_t<NP, MV_D2Q9, T>(p, st);
    case MV_D3Q19: return launch_pass_t<NP, MV_D3Q19, T>(p, st);
    case MV_D3Q15: return launch_pass_t<NP, MV_D3Q15, T>(p, st);
    case MV_D3Q27: return launch_pass_t<NP, MV_D3Q27, T>(p, st);
  }
  return (int)cudaErrorInvalidValue;
}

template <class T>
int launch_pass_typed(const PdgPass& p, cudaStream_t st) {
  switch (p.ncell > 0 ? p.npl / p.ncell : 0) {
    case 2: return launch_pass_np<2, T>(p, st);
    case 3: return launch_pass_np<3, T>(p, st);
    case 4: return launch_pass_np<4, T>(p, st);
    case 5: return launch_pass_np<5, T>(p, st);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace pdgdev
