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

// Line-resident form of the pass kernel: the block's lines (every field the pass touches,
// over the whole line length) are copied into shared memory with coalesced cp.async, the op
// list runs there unchanged (pass_body on a copy of the descriptor, in shared memory, that
// points at the staged lines), and the lines are written back once.  Each value of the
// block's lines crosses DRAM once each way, and the block requests all of its data at the
// start, instead of one cell per thread and sweep step through global memory.  Periodic
// lines of the DnQ2n models (no inflow data, no lattice slots, no source stage).
// Shared memory: nload fields x lpb lines x pdg_resident_ls(npl) values (16-byte aligned
// lines on different banks), then the segment aggregates of pass_body.
__device__ __forceinline__ bool pass_has_collision(const PdgPass& p) {
  for (int o = 0; o < p.nops; ++o)
    if (p.op[o] == PDG_OP_C) return true;
  return false;
}

__device__ __forceinline__ void cp_async8_line(double* smem, const double* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}

// Copies between the block's lines in global memory and their shared-memory image, with
// no division per element: unit-stride lines with consecutive threads on consecutive
// points, strided lines with consecutive threads on consecutive lines (adjacent points of
// the fastest axis; a thread keeps one line and steps along it).
template <bool LOAD>
__device__ __forceinline__ void resident_copy(const PdgPass& p, double* lines, int l0, int cnt, int nload,
                                              bool all) {
  const int LS = pdg_resident_ls(p.npl);
  const long long FS = (long long)p.lpb * LS;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (p.stride == 1) {
    for (int j = 0; j < nload; ++j) {
      const long long fo = (long long)(all ? j : p.tfield[j]) * p.field_stride;
      for (int l = 0; l < cnt; ++l) {
        double* g = p.f + fo + line_base(p, l0 + l);
        double* sp = lines + j * FS + (long long)l * LS;
        for (int pt = tid; pt < p.npl; pt += nt) {
          if (LOAD)
            cp_async8_line(sp + pt, g + pt);
          else
            g[pt] = sp[pt];
        }
      }
    }
  } else {
    const int tpl = nt / cnt;                 // threads per line
    const int l = tid % cnt, t0 = tid / cnt;
    if (t0 >= tpl) return;
    const long long lb = line_base(p, l0 + l);
    for (int j = 0; j < nload; ++j) {
      double* g = p.f + (long long)(all ? j : p.tfield[j]) * p.field_stride + lb;
      double* sp = lines + j * FS + (long long)l * LS;
      for (int pt = t0; pt < p.npl; pt += tpl) {
        if (LOAD)
          cp_async8_line(sp + pt, g + (long long)pt * p.stride);
        else
          g[(long long)pt * p.stride] = sp[pt];
      }
    }
  }
}

template <int NP, int MV, class T>
__global__ void __launch_bounds__(512) pass_resident_kernel(const __grid_constant__ PdgPass p) {
  extern __shared__ __align__(16) double sm[];
  __shared__ PdgPass q;
  int l0, cnt;
  block_lines(p, blockIdx.x, &l0, &cnt);
  const bool all = pass_has_collision(p);
  const int nload = all ? p.model.nf : p.ntf;
  const int LS = pdg_resident_ls(p.npl);
  const long long FS = (long long)p.lpb * LS;
  double* lines = sm;
  double* aux = sm + (size_t)nload * FS;
  resident_copy<true>(p, lines, l0, cnt, nload, all);
  {   // the descriptor, copied word by word by all threads
    const int* src = reinterpret_cast<const int*>(&p);
    int* dst = reinterpret_cast<int*>(&q);
    for (int i = threadIdx.x; i < (int)(sizeof(PdgPass) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    q.f = lines;
    q.field_stride = FS;
    q.stride = 1;
    q.lineA = 0x40000000;
    q.s1 = LS;
    q.s2 = 0;
    q.nlines = cnt;
    q.nblocks = 0;
    q.tmap = 1;
    if (!all)
      for (int phi = 0; phi < p.ntf; ++phi) q.tfield[phi] = phi;
  }
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  pass_body<NP, MV, T>(q, 0, aux);
  __syncthreads();
  resident_copy<false>(p, lines, l0, cnt, nload, all);
}

// Dynamic shared memory (bytes) of the line-resident kernel for a pass descriptor.
inline size_t resident_smem(const PdgPass& p, int nf) {
  bool all = false;
  for (int o = 0; o < p.nops; ++o)
    if (p.op[o] == PDG_OP_C) all = true;
  const size_t nload = all ? (size_t)nf : (size_t)p.ntf;
  return sizeof(double) * (nload * (size_t)p.lpb * (size_t)pdg_resident_ls(p.npl) + 3 * (size_t)p.ntf * p.nseg * p.lpb);
}

template <int NP, int MV, class T>
int launch_pass_t(const PdgPass& p, cudaStream_t st) {
  const int threads = p.lpb * p.nseg * p.ngroup;
  const int blocks = p.nblocks > 0 ? p.nblocks : (p.nlines + p.lpb - 1) / p.lpb;
  if constexpr (MV != MV_D2Q9 && MV != MV_D3Q19 && MV != MV_D3Q15 && MV != MV_D3Q27) {
    if (p.resident) {
      const size_t smem = resident_smem(p, p.model.nf);
      auto kern = pass_resident_kernel<NP, MV, T>;
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return (int)e;
      kern<<<blocks, threads, smem, st>>>(p);
      return (int)cudaGetLastError();
    }
  }
  const size_t smem = sizeof(double) * 3 * (size_t)p.ntf * p.nseg * p.lpb;
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
