// Transport of the corner populations of D3Q15 / D3Q27 (velocities lambda (+-1, +-1, +-1)).
//
// Section 3.1, eq. (3.7) on a Cartesian cell splits into one line operator per axis, so
// the theta step of eq. (3.11) couples cell c to the NEW values on the downwind faces of
// its three upwind neighbours (traversal orientation: -x, -y and -z):
//   fn_c = Binv r_c - c1 f_c,   r_c = f_c / theta + kx S_x Lt + ky S_y Bt + kz S_z Zt
// (PdgCornerCoef).  The faces obey a 3-D recurrence, periodic along all three axes: the
// analogue of the macrocell wavefronts of Section 4.2 on a cyclic mesh.
//
// Exact solve by truncated boxes.  A block owns a box of tx x ty x tz output cells of one
// population and sweeps the region that starts wx columns, wy rows and wz layers upwind of
// it.  At the region's three upwind boundaries the new face values are replaced by the old
// ones; the host chose the widths so that this start changes no output cell by more than
// 2^-57 of max|f| per boundary (pdg_plan_corner).  The region is swept layer by layer
// along z; inside a layer, column j handles row t - j at step t (a skewed 2-D wavefront:
// every cell of an anti-diagonal is independent).  The +x and +y faces pass between the
// steps of a layer through shared memory (double-buffered by step parity); the +z face of
// every cell of the layer's region is kept until the cell above reads it.
// No block waits on another block.  Reads come from the input slots and writes go to the
// output slots, so overlapping regions of neighbouring boxes never see a new value.
//
// Work split per step: (A) the block builds r_c for every cell of the anti-diagonal in
// shared memory, (B) the threads form the output nodes as dot products with r_c (Binv sits
// in shared memory transposed, so the threads of a cell read consecutive words; the FP64
// pipe, not shared memory, bounds this loop): all n^3 nodes of an output cell, only the
// face nodes of a cell of the upwind start.  The state of the next anti-diagonal (and the
// +z faces it reads) is copied into shared memory with cp.async while (B) runs.
//
// Memory: the +z faces of a layer (one face per cell of the region, the largest per-block
// array) live in a global scratch slice of the block (PdgCornerPass::zt, L2-resident),
// which keeps shared memory for the staging buffers and lets boxes grow; each entry is
// written one layer before it is staged again, with many barriers in between.
#pragma once
#include <cuda_runtime.h>

#include "pdg_diag.cuh"

namespace pdgdev {

struct CornerGeom {
  const double* fin;
  double* fout;
  double* zt;              // this block's +z faces: [nrow][ncol][n^2] (global scratch)
  int sx, sy, sz;
  long long sa, sb, sc;
  int ncol, nrow, nlay, wx, wy, wz;
  int X0, Y0, Z0, ncx, ncy, ncz;
  // inflow starts: the region begins at the domain's inflow face of that axis, and the
  // values entering its first column (row, layer) are this population's boundary data
  int bx, by, bz;
  const double* fbx;
  const double* fby;
  const double* fbz;
  long long fls[3][3];
  const long long* colx;   // [ncol + 1]: offset of traversal node 0 of region column j - 1
  const long long* rowy;   // [nrow + 1]
  const long long* layz;   // [nlay + 1]
};

// Offset of node (iz, iy, ix) (traversal orientation) of region cell (j, r, k), j, r, k >= -1.
__device__ __forceinline__ long long corner_off(const CornerGeom& g, int j, int r, int k, int iz, int iy, int ix) {
  return g.layz[k + 1] + (long long)(g.sz * iz) * g.sc + g.rowy[r + 1] + (long long)(g.sy * iy) * g.sb +
         g.colx[j + 1] + (long long)(g.sx * ix) * g.sa;
}

// Point coordinates (along x, y, z) of traversal node i of region column j, row r, layer k.
template <int NP>
__device__ __forceinline__ long long corner_px(const CornerGeom& g, int j, int i) {
  const int tc = wrap_cell(g.X0 - g.wx + j, g.ncx);
  return g.sx > 0 ? (long long)tc * NP + i : (long long)(g.ncx - 1 - tc) * NP + (NP - 1 - i);
}
template <int NP>
__device__ __forceinline__ long long corner_py(const CornerGeom& g, int r, int i) {
  const int tc = wrap_cell(g.Y0 - g.wy + r, g.ncy);
  return g.sy > 0 ? (long long)tc * NP + i : (long long)(g.ncy - 1 - tc) * NP + (NP - 1 - i);
}
template <int NP>
__device__ __forceinline__ long long corner_pz(const CornerGeom& g, int k, int i) {
  const int tc = wrap_cell(g.Z0 - g.wz + k, g.ncz);
  return g.sz > 0 ? (long long)tc * NP + i : (long long)(g.ncz - 1 - tc) * NP + (NP - 1 - i);
}

// Row of one cell in the staging buffers: its n^3 state values, then the n^2 values on the
// +z face of the cell below it (the face it reads), padded to 16 bytes.
template <int NP>
struct CornerRow {
  static constexpr int NF = NP * NP, NN = NF * NP, RS = (NN + NF + 1) & ~1;
};

// Stage the state and the entering +z faces of every cell of anti-diagonal t of layer k,
// and, on the region's upwind x and y edges, the old face values entering it.
// stage_z = false: the entering +z faces are left out (a caller that reads them later,
// directly from the scratch, because the layer below writes them one step before).
template <int NP>
__device__ __forceinline__ void corner_stage(const CornerGeom& g, int k, int t, double* fb, double* lbnd,
                                             double* bbnd, bool stage_z = true) {
  constexpr int NF = CornerRow<NP>::NF, NN = CornerRow<NP>::NN, RS = CornerRow<NP>::RS;
  const int jlo = max(0, t - g.nrow + 1), jhi = min(g.ncol - 1, t);
  const int A = jhi - jlo + 1;
  const int per = stage_z ? NN + NF : NN;
  for (int i = threadIdx.x; i < A * per; i += blockDim.x) {
    const int c = i / per, q = i % per;
    const int j = jlo + c, r = t - j;
    const double* src = q < NN ? g.fin + corner_off(g, j, r, k, q / NF, (q / NP) % NP, q % NP)
                               : g.zt + ((long long)r * g.ncol + j) * NF + (q - NN);
    cp_async8(fb + c * RS + q, src);
  }
  const int tid = threadIdx.x;
  if (jlo == 0 && tid < NF) {   // column 0 at row t: +x face of the cell upwind of it
    const int iz = tid / NP, iy = tid % NP;
    if (g.bx)                   // the inflow face: boundary value at the node's (y, z) point
      cp_async8(lbnd + tid, g.fbx + corner_py<NP>(g, t, iy) * g.fls[0][1] + corner_pz<NP>(g, k, iz) * g.fls[0][2]);
    else
      cp_async8(lbnd + tid, g.fin + corner_off(g, -1, t, k, iz, iy, NP - 1));
  }
  if (jhi == t && tid >= NF && tid < 2 * NF) {   // row 0 at column t: +y face of the cell below
    const int u = tid - NF, iz = u / NP, ix = u % NP;
    if (g.by)
      cp_async8(bbnd + u, g.fby + corner_px<NP>(g, t, ix) * g.fls[1][0] + corner_pz<NP>(g, k, iz) * g.fls[1][2]);
    else
      cp_async8(bbnd + u, g.fin + corner_off(g, t, -1, k, iz, NP - 1, ix));
  }
}

template <int NP, class T>
__device__ __forceinline__ void corner_body(const PdgCornerPass& p, double* sm) {
  constexpr int NF = CornerRow<NP>::NF, NN = CornerRow<NP>::NN, RS = CornerRow<NP>::RS;
  constexpr int NFF = NN - (NP - 1) * (NP - 1) * (NP - 1);   // nodes on the three downwind faces
  int b = blockIdx.x;
  const int txi = b % p.ntx;
  b /= p.ntx;
  const int tyi = b % p.nty;
  b /= p.nty;
  const int tzi = b % p.ntz;
  const int pop = b / p.ntz;
  const PdgCornerCoef& C = p.c;
  const int CM = p.tx + C.wx, RM = p.ty + C.wy;   // column / row capacities of any box
  const int amax = min(CM, RM);                   // longest anti-diagonal

  CornerGeom g;
  g.fin = p.fin[pop];
  g.fout = p.fout[pop];
  g.sx = p.sx[pop];
  g.sy = p.sy[pop];
  g.sz = p.sz[pop];
  g.sa = p.sa;
  g.sb = p.sb;
  g.sc = p.sc;
  const int X0 = txi * p.tx, Y0 = tyi * p.ty, Z0 = tzi * p.tz;
  // periodic axis: the truncated start; inflow axis: at most back to the inflow face
  g.wx = p.per[0] ? C.wx : min(C.wx, X0);
  g.wy = p.per[1] ? C.wy : min(C.wy, Y0);
  g.wz = p.per[2] ? C.wz : min(C.wz, Z0);
  g.bx = !p.per[0] && X0 - g.wx == 0;
  g.by = !p.per[1] && Y0 - g.wy == 0;
  g.bz = !p.per[2] && Z0 - g.wz == 0;
  g.X0 = X0;
  g.Y0 = Y0;
  g.Z0 = Z0;
  g.ncx = p.ncx;
  g.ncy = p.ncy;
  g.ncz = p.ncz;
  const double* fbs[3];
  for (int a = 0; a < 3; ++a) {
    fbs[a] = p.fb[a] ? p.fb[a] + (long long)(p.bside[a][pop] * p.nent + p.bent[a][pop]) * p.flines[a] : nullptr;
    for (int b = 0; b < 3; ++b) g.fls[a][b] = p.fls[a][b];
  }
  g.fbx = fbs[0];
  g.fby = fbs[1];
  g.fbz = fbs[2];
  g.ncol = min(p.tx, p.ncx - X0) + g.wx;
  g.nrow = min(p.ty, p.ncy - Y0) + g.wy;
  g.nlay = min(p.tz, p.ncz - Z0) + g.wz;
  g.zt = p.zt + (long long)blockIdx.x * RM * CM * NF;
  const int T_steps = g.ncol + g.nrow - 1;

  // shared memory: BinvT[NN][NN] | rbuf[amax][RS] | fbuf[2][amax][RS] | Lt[2][CM+1][NF] |
  //                Bt[2][CM][NF] | lbnd[2][NF] | bbnd[2][NF] | fnode[NFF] (int) |
  //                colx[CM+1] | rowy[RM+1] | layz[tz+wz+1] (64-bit offsets)
  T* BinvT = reinterpret_cast<T*>(sm);
  T* rbuf = BinvT + NN * NN;
  T* fbuf = rbuf + (size_t)amax * RS;
  T* Lt = fbuf + (size_t)2 * amax * RS;
  T* Bt = Lt + (size_t)2 * (CM + 1) * NF;
  T* lbnd = Bt + (size_t)2 * CM * NF;
  T* bbnd = lbnd + 2 * NF;
  long long* colx = reinterpret_cast<long long*>(bbnd + 2 * NF);
  long long* rowy = colx + (CM + 1);
  long long* layz = rowy + (RM + 1);
  int* fnode = reinterpret_cast<int*>(layz + (p.tz + C.wz + 1));
  const int LtS = CM + 1, BtS = CM;
  for (int i = threadIdx.x; i < NN * NN; i += blockDim.x) {
    const int row = i % NN, col = i / NN;   // BinvT[col][row] = Binv[row][col]
    if constexpr (__is_same(T, double)) {
      BinvT[i] = p.binv[row * NN + col];
    } else {
      const float* bf = p.binv_f + 2 * (row * NN + col);
      BinvT[i] = T{bf[0], bf[1]};
    }
  }
  if (threadIdx.x == 0) {   // the face nodes, in node order
    int f = 0;
    for (int q = 0; q < NN; ++q)
      if (q % NP == NP - 1 || (q / NP) % NP == NP - 1 || q / NF == NP - 1) fnode[f++] = q;
  }
  for (int j = threadIdx.x; j <= g.ncol; j += blockDim.x) {
    const int tc = wrap_cell(X0 - g.wx + j - 1, p.ncx);
    colx[j] = (long long)(g.sx > 0 ? tc * NP : (p.ncx - 1 - tc) * NP + (NP - 1)) * g.sa;
  }
  for (int r = threadIdx.x; r <= g.nrow; r += blockDim.x) {
    const int tr = wrap_cell(Y0 - g.wy + r - 1, p.ncy);
    rowy[r] = (long long)(g.sy > 0 ? tr * NP : (p.ncy - 1 - tr) * NP + (NP - 1)) * g.sb;
  }
  for (int k = threadIdx.x; k <= g.nlay; k += blockDim.x) {
    const int tl = wrap_cell(Z0 - g.wz + k - 1, p.ncz);
    layz[k] = (long long)(g.sz > 0 ? tl * NP : (p.ncz - 1 - tl) * NP + (NP - 1)) * g.sc;
  }
  g.colx = colx;
  g.rowy = rowy;
  g.layz = layz;
  __syncthreads();
  // the region's lower z boundary: old +z faces of the layer below the region, or at the
  // inflow face the boundary values at the nodes' (x, y) points
  for (int i = threadIdx.x; i < g.nrow * g.ncol * NF; i += blockDim.x) {
    const int cell = i / NF, u = i % NF;
    const int r = cell / g.ncol, j = cell % g.ncol;
    g.zt[i] = g.bz ? g.fbz[corner_px<NP>(g, j, u % NP) * g.fls[2][0] + corner_py<NP>(g, r, u / NP) * g.fls[2][1]]
                   : g.fin[corner_off(g, j, r, -1, NP - 1, u / NP, u % NP)];
  }
  __syncthreads();
  const T rth = PDG_DC(T, C, rtheta), c1 = PDG_DC(T, C, c1);
  const T th = PDG_DC(T, C, theta);
  const T kx = PDG_DC(T, C, kx), ky = PDG_DC(T, C, ky), kz = PDG_DC(T, C, kz);

  corner_stage<NP>(g, 0, 0, reinterpret_cast<double*>(fbuf), reinterpret_cast<double*>(lbnd),
                   reinterpret_cast<double*>(bbnd));
  cp_async_wait_all();
  __syncthreads();
  int s = 0;   // steps so far (all layers): the parity of the double buffers
  for (int k = 0; k < g.nlay; ++k) {
    const bool out_layer = k >= g.wz;
    for (int t = 0; t < T_steps; ++t, ++s) {
      const int par = s & 1, prv = par ^ 1;
      const int jlo = max(0, t - g.nrow + 1), jhi = min(g.ncol - 1, t);
      const int A = jhi - jlo + 1;
      const T* fc = fbuf + (size_t)par * amax * RS;
      // (A) r_c of every cell of the anti-diagonal
      for (int i = threadIdx.x; i < A * NN; i += blockDim.x) {
        const int c = i / NN, q = i % NN;
        const int j = jlo + c, r = t - j;
        const int iz = q / NF, iy = (q / NP) % NP, ix = q % NP;
        T rv = fc[c * RS + q] * rth;
        if (ix == 0)
          rv = fma(kx, j == 0 ? lbnd[par * NF + iz * NP + iy] : Lt[((size_t)prv * LtS + j) * NF + iz * NP + iy], rv);
        if (iy == 0)
          rv = fma(ky, r == 0 ? bbnd[par * NF + iz * NP + ix] : Bt[((size_t)prv * BtS + j) * NF + iz * NP + ix], rv);
        if (iz == 0) rv = fma(kz, fc[c * RS + NN + iy * NP + ix], rv);
        rbuf[c * RS + q] = rv;
      }
      __syncthreads();
      {   // stage the next anti-diagonal (the first one of the next layer after the last)
        double* nf = reinterpret_cast<double*>(fbuf + (size_t)prv * amax * RS);
        double* nl = reinterpret_cast<double*>(lbnd + prv * NF);
        double* nb = reinterpret_cast<double*>(bbnd + prv * NF);
        if (t + 1 < T_steps) corner_stage<NP>(g, k, t + 1, nf, nl, nb);
        else if (k + 1 < g.nlay) corner_stage<NP>(g, k + 1, 0, nf, nl, nb);
      }
      // (B) output cells [h1, h2] (columns >= wx, rows >= wy, in a layer >= wz): every node;
      // the cells of the upwind start: only their face nodes.  Items are (cell, node)
      // pairs, output cells first, consecutive threads on consecutive nodes of a cell.
      int h1 = jhi + 1, h2 = jhi;
      if (out_layer) {
        h1 = max(jlo, min(g.wx, jhi + 1));
        h2 = max(h1 - 1, min(jhi, t - g.wy));
      }
      const int nout = (h2 - h1 + 1) * NN, nlo = (h1 - jlo) * NFF;
      const int items = nout + (A * NFF - (h2 - h1 + 1) * NFF);
      for (int it = threadIdx.x; it < items; it += blockDim.x) {
        int j, q;
        if (it < nout) {
          j = h1 + it / NN;
          q = it % NN;
        } else if (it - nout < nlo) {
          j = jlo + (it - nout) / NFF;
          q = fnode[(it - nout) % NFF];
        } else {
          j = h2 + 1 + (it - nout - nlo) / NFF;
          q = fnode[(it - nout - nlo) % NFF];
        }
        const int c = j - jlo, r = t - j;
        const T* rc = rbuf + c * RS;
        T acc;
        if constexpr (__is_same(T, double)) {
          // two chains: the FP64 pipe (2 DFMA per SM and clock) hides their latency
          double a0 = 0.0, a1 = 0.0;
#pragma unroll
          for (int m = 0; m + 1 < NN; m += 2) {
            a0 = fma(BinvT[m * NN + q], rc[m], a0);
            a1 = fma(BinvT[(m + 1) * NN + q], rc[m + 1], a1);
          }
          if (NN % 2) a0 = fma(BinvT[(NN - 1) * NN + q], rc[NN - 1], a0);
          acc = a0 + a1;
        } else {
          // compensated dot product (see dot_acc): exact high products and sums, the
          // rounding errors and cross terms gathered in one FP32 accumulator
          float S = 0.0f, L = 0.0f;
#pragma unroll 8
          for (int m = 0; m < NN; ++m) {
            const T a = BinvT[m * NN + q], bv = rc[m];
            const dd pr = dd_two_prod(a.hi, bv.hi);
            const float cross = __fmaf_rn(a.hi, bv.lo, __fmul_rn(a.lo, bv.hi));
            const dd sm2 = dd_two_sum(S, pr.hi);
            S = sm2.hi;
            L = __fadd_rn(L, __fadd_rn(sm2.lo, __fadd_rn(pr.lo, cross)));
          }
          acc = dd_fast_two_sum(S, L);
        }
        const int qz = q / NF, qy = (q / NP) % NP, qx = q % NP;
        if (it < nout) st(g.fout + corner_off(g, j, r, k, qz, qy, qx), acc - c1 * fc[c * RS + q]);
        if (qx == NP - 1 || qy == NP - 1 || qz == NP - 1) {
          // theta fn + (1 - theta) f = theta (Binv r) - (1 - theta) f + (1 - theta) f
          const T face = th * acc;
          if (qx == NP - 1) Lt[((size_t)par * LtS + j + 1) * NF + qz * NP + qy] = face;
          if (qy == NP - 1) Bt[((size_t)par * BtS + j) * NF + qz * NP + qx] = face;
          if (qz == NP - 1) st(g.zt + ((long long)r * g.ncol + j) * NF + qy * NP + qx, face);
        }
      }
      cp_async_wait_all();
      __syncthreads();
    }
  }
}

template <int NP, class T>
__global__ void __launch_bounds__(512, 1) corner_kernel(const __grid_constant__ PdgCornerPass p) {
  extern __shared__ double sm[];
  corner_body<NP, T>(p, sm);
}

template <class T>
int launch_corner_typed(const PdgCornerPass& p, size_t smem, cudaStream_t st) {
  const long long blocks = (long long)p.ntx * p.nty * p.ntz * p.npop;
  if (blocks > 0x7fffffffLL || blocks < 1) return (int)cudaErrorInvalidConfiguration;
  auto go = [&](auto kern) -> int {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return (int)e;
    }
    kern<<<(unsigned)blocks, p.threads, smem, st>>>(p);
    return (int)cudaGetLastError();
  };
  switch (p.n) {
    case 2: return go(corner_kernel<2, T>);
    case 3: return go(corner_kernel<3, T>);
    case 4: return go(corner_kernel<4, T>);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace pdgdev
