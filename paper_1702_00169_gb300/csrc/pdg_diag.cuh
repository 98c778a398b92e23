// Transport of the D2Q9 diagonal populations (velocities lambda (+-1, +-1)).
//
// Section 3.1, eq. (3.7) on a Cartesian cell splits into one line operator per axis, so
// the theta step of eq. (3.11) couples cell c to the NEW values on the downwind faces of
// its two upwind neighbours (traversal orientation: -x and -y):
//   fn_c = Binv r_c - c1 f_c,   r_c = f_c / theta + kx S_x Lt + ky S_y Bt
// (PdgDiagCoef).  The faces obey a 2-D recurrence along both axes, periodic in both: the
// analogue of the macrocell wavefronts of Section 4.2 on a cyclic mesh.
//
// Exact solve by truncated tiles.  A block owns a tile of tx x ty output cells of one
// population and sweeps the region that starts wx columns and wy rows upwind of it.  At
// the region's upwind edges the new face values are replaced by the old ones; the host
// chose wx, wy so that this start changes no output cell by more than 2^-56 of max|f|
// (pdg_plan_diag).  Inside the region, column j handles row t - j at step t (a skewed
// wavefront: every cell of an anti-diagonal is independent), with the faces passed
// between steps through shared memory, double-buffered by step parity.  No block waits
// on another block.  Reads come from the input slots and writes go to the output slots,
// so overlapping regions of neighbouring tiles never see a new value.
//
// Work split.  One step of the wavefront = one anti-diagonal of cells: (A) the block
// builds r_c for every cell of it in shared memory, (B) the block forms the output
// nodes as dot products with r_c (Binv sits in shared memory transposed, so the threads
// of a cell read consecutive words).  The cells of the upwind start only pass faces on,
// so (B) computes just their 2n-1 face nodes.  The block forms theta r_c, whose product
// with Binv is the face value passed on, theta fn + (1 - theta) f = theta (Binv r_c).  The
// state of the next anti-diagonal is copied into shared memory with cp.async while (B)
// runs (double-buffered by parity).
#pragma once
#include <cuda_runtime.h>

#include "pdg_device.cuh"

namespace pdgdev {

// Coefficient accessors of PdgDiagCoef (FP64 value or float pair).
#define PDG_DC(T, C, name) cval<T>(&(C).name, (C).name##_f, 0)

__device__ __forceinline__ int wrap_cell(int c, int n) {
  int r = c % n;
  return r < 0 ? r + n : r;
}

struct DiagGeom {
  const double* fin;
  double* fout;
  int sx, sy, ncx, ncy;
  long long sa, sb;        // point strides along the plane's axes a ("x") and b ("y")
  int X0, Y0, wx, wy, ncol, nrow;
  const long long* colx;   // [ncol + 1]: offset of traversal node 0 of region column j - 1
  const long long* rowy;   // [nrow + 1]: offset of traversal node row 0 of region row r - 1
  // inflow faces: when bx (by) is set the region starts at the domain's inflow face and
  // the values entering column 0 (row 0) are the boundary data fbx (fby)
  int bx, by;
  const double* fbx;       // values of this population at its x inflow face (this plane)
  const double* fby;       // values at its y inflow face
  long long fbx_ls, fby_ls;   // line-index stride of the point coordinate along y (x) there
};

// Offset of node (iy, ix) (traversal orientation) of region cell (j, r), j, r >= -1.
template <int NP>
__device__ __forceinline__ long long diag_off(const DiagGeom& g, int j, int r, int iy, int ix) {
  return g.rowy[r + 1] + (long long)(g.sy * iy) * g.sb + g.colx[j + 1] + (long long)(g.sx * ix) * g.sa;
}

// Asynchronous 8-byte copy global -> shared (cp.async, cached in L1) and its fences.
__device__ __forceinline__ void cp_async8(void* smem, const double* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Face node f of a cell: f < n: node (f, n-1) of the +x face; else node (n-1, f-n) of the
// +y face (the corner belongs to the first set).
template <int NP>
__device__ __forceinline__ int face_node(int f) {
  return f < NP ? f * NP + (NP - 1) : (NP - 1) * NP + (f - NP);
}

// Stage the state of every cell of anti-diagonal t (all n^2 nodes) and, on the region's
// upwind edges, the old face values entering it, into buffer set `b`.
template <int NP, class T>
__device__ __forceinline__ void diag_stage(const DiagGeom& g, int t, T* fb, T* lbnd, T* bbnd) {
  constexpr int NN = NP * NP, RS = NN + 2;
  const int jlo = max(0, t - g.nrow + 1), jhi = min(g.ncol - 1, t);
  const int A = jhi - jlo + 1;
  for (int i = threadIdx.x; i < A * NN; i += blockDim.x) {
    const int c = i / NN, q = i % NN;
    const int j = jlo + c;
    cp_async8(fb + c * RS + q, g.fin + diag_off<NP>(g, j, t - j, q / NP, q % NP));
  }
  const int tid = threadIdx.x;
  if (jlo == 0 && tid < NP) {   // column 0 at row t: +x face of the cell upwind of it
    if (g.bx) {                 // the inflow face: boundary value at the node's y point
      const int tr = wrap_cell(g.Y0 - g.wy + t, g.ncy);   // y may be periodic
      const int pcy = g.sy > 0 ? tr : g.ncy - 1 - tr;
      cp_async8(lbnd + tid, g.fbx + (long long)(pcy * NP + (g.sy > 0 ? tid : NP - 1 - tid)) * g.fbx_ls);
    } else {
      cp_async8(lbnd + tid, g.fin + diag_off<NP>(g, -1, t, tid, NP - 1));
    }
  }
  if (jhi == t && tid >= NP && tid < 2 * NP) {   // row 0 at column t: +y face of the cell below
    const int ix = tid - NP;
    if (g.by) {
      const int tc = wrap_cell(g.X0 - g.wx + t, g.ncx);   // x may be periodic
      const int pcx = g.sx > 0 ? tc : g.ncx - 1 - tc;
      cp_async8(bbnd + ix, g.fby + (long long)(pcx * NP + (g.sx > 0 ? ix : NP - 1 - ix)) * g.fby_ls);
    } else {
      cp_async8(bbnd + ix, g.fin + diag_off<NP>(g, t, -1, NP - 1, ix));
    }
  }
}

template <int NP, class T>
__device__ __forceinline__ void diag_body(const PdgDiagPass& p, double* sm) {
  constexpr int NN = NP * NP, NF = 2 * NP - 1, RS = NN + 2;   // RS: 16-byte aligned rows
  // block order: plane fastest (neighbouring planes share cache sectors), then tiles
  int b = blockIdx.x;
  const int plane = b % p.nplane;
  b /= p.nplane;
  const int txi = b % p.ntx;
  b /= p.ntx;
  const int tyi = b % p.nty;
  const int pop = b / p.nty;
  const PdgDiagCoef& C = p.c;

  DiagGeom g;
  g.fin = p.fin[pop] + (long long)plane * p.sc;
  g.fout = p.fout[pop] + (long long)plane * p.sc;
  g.sx = p.sx[pop];
  g.sy = p.sy[pop];
  g.ncx = p.ncx;
  g.ncy = p.ncy;
  g.sa = p.sa;
  g.sb = p.sb;
  g.X0 = txi * p.tx;
  g.Y0 = tyi * p.ty;
  // periodic axis: the truncated start; inflow axis: at most back to the inflow face
  g.wx = p.perx ? C.wx : min(C.wx, g.X0);
  g.wy = p.pery ? C.wy : min(C.wy, g.Y0);
  g.bx = !p.perx && g.X0 - g.wx == 0;
  g.by = !p.pery && g.Y0 - g.wy == 0;
  g.fbx = p.fbx ? p.fbx + (long long)(p.bxside[pop] * p.nent + p.bxent[pop]) * p.fbx_lines + plane * p.fbx_ps
                : nullptr;
  g.fby = p.fby ? p.fby + (long long)(p.byside[pop] * p.nent + p.byent[pop]) * p.fby_lines + plane * p.fby_ps
                : nullptr;
  g.fbx_ls = p.fbx_ls;
  g.fby_ls = p.fby_ls;
  const int ox = min(p.tx, p.ncx - g.X0), oy = min(p.ty, p.ncy - g.Y0);
  g.ncol = ox + g.wx;
  g.nrow = oy + g.wy;
  const int T_steps = g.ncol + g.nrow - 1;
  const int amax = min(p.tx + C.wx, p.ty + C.wy);   // longest anti-diagonal of any tile

  // shared memory: BinvT[NN][NN] | rbuf[amax][RS] | fbuf[2][amax][RS] | Lt[2][ncol+1][NP] |
  //                Bt[2][ncol][NP] | lbnd[2][NP] | bbnd[2][NP] | rowy[nrow+1] | colx[ncol+1]
  //                (rowy, colx: 64-bit offsets)
  T* BinvT = reinterpret_cast<T*>(sm);
  T* rbuf = BinvT + NN * NN;
  T* fbuf = rbuf + (size_t)amax * RS;
  T* Lt = fbuf + (size_t)2 * amax * RS;
  T* Bt = Lt + (size_t)2 * (p.tx + C.wx + 1) * NP;
  T* lbnd = Bt + (size_t)2 * (p.tx + C.wx) * NP;
  T* bbnd = lbnd + 2 * NP;
  long long* rowy = reinterpret_cast<long long*>(bbnd + 2 * NP);
  long long* colx = rowy + (p.ty + C.wy + 1);
  const int LtS = p.tx + C.wx + 1, BtS = p.tx + C.wx;   // per-parity strides (columns)
  for (int i = threadIdx.x; i < NN * NN; i += blockDim.x) {
    const int row = i % NN, col = i / NN;   // BinvT[col][row] = Binv[row][col]
    BinvT[i] = cval<T>(&C.Binv[row * NN + col], &C.Binv_f[row * NN + col], 0);
  }
  for (int j = threadIdx.x; j <= g.ncol; j += blockDim.x) {
    const int tc = wrap_cell(g.X0 - g.wx + j - 1, g.ncx);
    colx[j] = (long long)(g.sx > 0 ? tc * NP : (g.ncx - 1 - tc) * NP + (NP - 1)) * g.sa;
  }
  for (int r = threadIdx.x; r <= g.nrow; r += blockDim.x) {
    const int tr = wrap_cell(g.Y0 - g.wy + r - 1, g.ncy);
    rowy[r] = (long long)(g.sy > 0 ? tr * NP : (g.ncy - 1 - tr) * NP + (NP - 1)) * g.sb;
  }
  g.colx = colx;
  g.rowy = rowy;
  __syncthreads();
  // output-cell mapping: thread (k, q) computes node q of cells h1 + k, h1 + k + K, ...
  const int K = blockDim.x / NN;
  const int kq = threadIdx.x / NN, qq = threadIdx.x % NN;
  T creg[NN];
#pragma unroll
  for (int i = 0; i < NN; ++i) creg[i] = BinvT[i * NN + qq];
  // the block forms theta r_c = f_c + theta kx S_x Lt + theta ky S_y Bt: its product with
  // Binv is the face value theta (Binv r_c) itself, and fn = (Binv (theta r) - (1 - theta) f)
  // / theta
  const T rth = PDG_DC(T, C, rtheta), omth = PDG_DC(T, C, omtheta);
  const T th = PDG_DC(T, C, theta);
  const T tkx = th * PDG_DC(T, C, kx), tky = th * PDG_DC(T, C, ky);

  diag_stage<NP, T>(g, 0, fbuf, lbnd, bbnd);
  cp_async_wait_all();
  __syncthreads();
  for (int t = 0; t < T_steps; ++t) {
    const int par = t & 1, prv = par ^ 1;
    const int jlo = max(0, t - g.nrow + 1), jhi = min(g.ncol - 1, t);
    const int A = jhi - jlo + 1;
    const T* fc = fbuf + (size_t)par * amax * RS;
    // (A) theta r_c of every cell of the anti-diagonal
    for (int i = threadIdx.x; i < A * NN; i += blockDim.x) {
      const int c = i / NN, q = i % NN;
      const int j = jlo + c, iy = q / NP, ix = q % NP;
      T rv = fc[c * RS + q];
      if (ix == 0) rv = fma(tkx, j == 0 ? lbnd[par * NP + iy] : Lt[((size_t)prv * LtS + j) * NP + iy], rv);
      if (iy == 0) rv = fma(tky, j == t ? bbnd[par * NP + ix] : Bt[((size_t)prv * BtS + j) * NP + ix], rv);
      rbuf[c * RS + q] = rv;
    }
    __syncthreads();
    if (t + 1 < T_steps)
      diag_stage<NP, T>(g, t + 1, fbuf + (size_t)prv * amax * RS, lbnd + prv * NP, bbnd + prv * NP);
    // (B) outputs.  Cells [jlo, h1) and (h2, jhi] belong to the upwind start (column < wx
    // or row < wy): only their 2n-1 face nodes are needed.  Cells [h1, h2] are output
    // cells: every node, with the thread's row of Binv held in registers.
    const int h1 = max(jlo, min(g.wx, jhi + 1));
    const int h2 = max(h1 - 1, min(jhi, t - g.wy));
    auto finish = [&](int j, int q, T acc) {
      const int c = j - jlo, r = t - j, iy = q / NP, ix = q % NP;
      if (j >= g.wx && r >= g.wy) st(g.fout + diag_off<NP>(g, j, r, iy, ix), (acc - omth * fc[c * RS + q]) * rth);
      if (ix == NP - 1 || iy == NP - 1) {
        // theta fn + (1 - theta) f = theta (Binv r) = Binv (theta r)
        const T face = acc;
        if (ix == NP - 1) Lt[((size_t)par * LtS + j + 1) * NP + iy] = face;
        if (iy == NP - 1) Bt[((size_t)par * BtS + j) * NP + ix] = face;
      }
    };
    if (kq < K) {
      for (int j = h1 + kq; j <= h2; j += K) {
        const T* rc = rbuf + (j - jlo) * RS;
        T acc;
        if constexpr (__is_same(T, double)) {
          // one chain: a dependent DFMA chain per warp keeps its SM sub-partition's FP64
          // unit busy, so more chains would only add the adds that join them
          double a = 0.0;
#pragma unroll
          for (int k = 0; k < NN; ++k) a = fma(creg[k], rc[k], a);
          acc = a;
        } else {
          T bb[NN];
#pragma unroll
          for (int k = 0; k < NN; ++k) bb[k] = rc[k];
          acc = dot_acc<NN>(creg, bb, zero<T>());
        }
        finish(j, qq, acc);
      }
    }
    const int n1 = (h1 - jlo) * NF, n2 = (jhi - h2) * NF;
    for (int i = threadIdx.x; i < n1 + n2; i += blockDim.x) {
      const int j = i < n1 ? jlo + i / NF : h2 + 1 + (i - n1) / NF;
      const int q = face_node<NP>(i < n1 ? i % NF : (i - n1) % NF);
      const T* rc = rbuf + (j - jlo) * RS;
      T acc;
      if constexpr (__is_same(T, double)) {
        double a = 0.0;
#pragma unroll
        for (int k = 0; k < NN; ++k) a = fma(BinvT[k * NN + q], rc[k], a);
        acc = a;
      } else {
        T a[NN], bb[NN];
#pragma unroll
        for (int k = 0; k < NN; ++k) {
          a[k] = BinvT[k * NN + q];
          bb[k] = rc[k];
        }
        acc = dot_acc<NN>(a, bb, zero<T>());
      }
      finish(j, q, acc);
    }
    cp_async_wait_all();
    __syncthreads();
  }
}

template <int NP, class T>
__global__ void __launch_bounds__(512, 1) diag_kernel(const __grid_constant__ PdgDiagPass p) {
  extern __shared__ double sm[];
  diag_body<NP, T>(p, sm);
}

template <class T>
int launch_diag_typed(const PdgDiagPass& p, size_t smem, cudaStream_t st) {
  const int threads = p.threads;
  const long long blocks = (long long)p.ntx * p.nty * p.npop * p.nplane;
  if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidConfiguration;
  auto go = [&](auto kern) -> int {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return (int)e;
    }
    kern<<<(unsigned)blocks, threads, smem, st>>>(p);
    return (int)cudaGetLastError();
  };
  switch (p.n) {
    case 2: return go(diag_kernel<2, T>);
    case 3: return go(diag_kernel<3, T>);
    case 4: return go(diag_kernel<4, T>);
    case 5: return go(diag_kernel<5, T>);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace pdgdev
