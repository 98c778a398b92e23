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
// Work split.  Each cell is computed by n^2 threads, thread q owning output node q; Binv
// sits in shared memory transposed (column-major), so the threads of a cell read
// consecutive words; kpar cells of an anti-diagonal are processed per round
// (threads = kpar n^2).  A round: (A) every thread builds entry q of r_c in shared
// memory; (B) every thread forms its output node as a dot product with r_c.  The next
// round's state value is loaded before (B) so that its latency overlaps the arithmetic.
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
  long long row;
  int X0, Y0, wx, wy, ncol, nrow;
};

// Offset of node (iy, ix) (traversal orientation) of region cell (j, r).
template <int NP>
__device__ __forceinline__ long long diag_off(const DiagGeom& g, int j, int r, int iy, int ix) {
  const int tc = wrap_cell(g.X0 - g.wx + j, g.ncx);
  const int tr = wrap_cell(g.Y0 - g.wy + r, g.ncy);
  const int pcx = g.sx > 0 ? tc : g.ncx - 1 - tc;
  const int pcy = g.sy > 0 ? tr : g.ncy - 1 - tr;
  const int x = pcx * NP + (g.sx > 0 ? ix : NP - 1 - ix);
  const int y = pcy * NP + (g.sy > 0 ? iy : NP - 1 - iy);
  return (long long)y * g.row + x;
}

// Values a thread needs from memory for one round: its state value and, on the
// region's upwind edges, the old face value entering its node.
template <class T>
struct DiagLoad {
  T f, lb, bb;
};

template <int NP, class T>
__device__ __forceinline__ void diag_fetch(const DiagGeom& g, int t, int j, int iy, int ix, bool act,
                                          DiagLoad<T>& L) {
  if (!act) return;
  const int r = t - j;
  L.f = ld<T>(g.fin + diag_off<NP>(g, j, r, iy, ix));
  if (j == 0 && ix == 0) L.lb = ld<T>(g.fin + diag_off<NP>(g, -1, r, iy, NP - 1));
  if (r == 0 && iy == 0) L.bb = ld<T>(g.fin + diag_off<NP>(g, j, -1, NP - 1, ix));
}

template <int NP, class T>
__device__ __forceinline__ void diag_body(const PdgDiagPass& p, double* sm) {
  constexpr int NN = NP * NP;
  const int K = p.kpar;
  int b = blockIdx.x;
  const int txi = b % p.ntx;
  b /= p.ntx;
  const int tyi = b % p.nty;
  const int pop = b / p.nty;
  const PdgDiagCoef& C = p.c;

  DiagGeom g;
  g.fin = p.fin[pop];
  g.fout = p.fout[pop];
  g.sx = p.sx[pop];
  g.sy = p.sy[pop];
  g.ncx = p.ncx;
  g.ncy = p.ncy;
  g.row = p.row;
  g.X0 = txi * p.tx;
  g.Y0 = tyi * p.ty;
  g.wx = C.wx;
  g.wy = C.wy;
  const int ox = min(p.tx, p.ncx - g.X0), oy = min(p.ty, p.ncy - g.Y0);
  g.ncol = ox + g.wx;
  g.nrow = oy + g.wy;
  const int T_steps = g.ncol + g.nrow - 1;

  const int tid = threadIdx.x;
  const int k = tid / NN, q = tid % NN;
  const int iy = q / NP, ix = q % NP;
  const bool lane_ok = k < K;

  // shared memory: BinvT[NN][NN] | rbuf[K][NN + 1] | Lt[2][ncol + 1][NP] | Bt[2][ncol][NP]
  T* BinvT = reinterpret_cast<T*>(sm);
  T* rbuf = BinvT + NN * NN;
  T* Lt = rbuf + (size_t)K * (NN + 1);
  T* Bt = Lt + (size_t)2 * (g.ncol + 1) * NP;
  for (int i = threadIdx.x; i < NN * NN; i += blockDim.x) {
    const int row = i % NN, col = i / NN;   // BinvT[col][row] = Binv[row][col]
    BinvT[i] = cval<T>(&C.Binv[row * NN + col], &C.Binv_f[row * NN + col], 0);
  }
  const T rth = PDG_DC(T, C, rtheta), c1 = PDG_DC(T, C, c1);
  const T th = PDG_DC(T, C, theta), omth = PDG_DC(T, C, omtheta);
  const T kx = PDG_DC(T, C, kx), ky = PDG_DC(T, C, ky);

  auto jlo = [&](int t) { return max(0, t - g.nrow + 1); };
  auto jhi = [&](int t) { return min(g.ncol - 1, t); };

  // first round
  int t = 0, base = 0;
  DiagLoad<T> cur{}, nxt{};
  diag_fetch<NP, T>(g, t, base + k, iy, ix, lane_ok && base + k <= jhi(t), cur);
  while (t < T_steps) {
    const int j = base + k;
    const bool act = lane_ok && j <= jhi(t);
    const int r = t - j;
    const int par = t & 1, prv = par ^ 1;
    // (A) entry q of r_c
    if (act) {
      T rv = cur.f * rth;
      if (ix == 0) {
        const T lin = (j == 0) ? cur.lb : Lt[((size_t)prv * (g.ncol + 1) + j) * NP + iy];
        rv = fma(kx, lin, rv);
      }
      if (iy == 0) {
        const T bin = (r == 0) ? cur.bb : Bt[((size_t)prv * g.ncol + j) * NP + ix];
        rv = fma(ky, bin, rv);
      }
      rbuf[k * (NN + 1) + q] = rv;
    }
    __syncthreads();
    // next round, and its loads
    int t2 = t, base2 = base + K;
    if (base2 > jhi(t2)) {
      t2 = t + 1;
      base2 = jlo(t2);
    }
    if (t2 < T_steps) diag_fetch<NP, T>(g, t2, base2 + k, iy, ix, lane_ok && base2 + k <= jhi(t2), nxt);
    // (B) output node q
    if (act) {
      const T* rc = rbuf + k * (NN + 1);
      T acc = zero<T>();
      if constexpr (__is_same(T, double)) {
#pragma unroll
        for (int i = 0; i < NN; ++i) acc = fma(BinvT[i * NN + q], rc[i], acc);
      } else {
        T a[NN], bb[NN];
#pragma unroll
        for (int i = 0; i < NN; ++i) {
          a[i] = BinvT[i * NN + q];
          bb[i] = rc[i];
        }
        acc = dot_acc<NN>(a, bb, acc);
      }
      const T out = acc - c1 * cur.f;
      if (j >= g.wx && r >= g.wy) st(g.fout + diag_off<NP>(g, j, r, iy, ix), out);
      if (ix == NP - 1 || iy == NP - 1) {
        const T face = fma(th, out, omth * cur.f);
        if (ix == NP - 1) Lt[((size_t)par * (g.ncol + 1) + j + 1) * NP + iy] = face;
        if (iy == NP - 1) Bt[((size_t)par * g.ncol + j) * NP + ix] = face;
      }
    }
    __syncthreads();
    cur = nxt;
    t = t2;
    base = base2;
  }
}

template <int NP, class T>
__global__ void __launch_bounds__(512) diag_kernel(const __grid_constant__ PdgDiagPass p) {
  extern __shared__ double sm[];
  diag_body<NP, T>(p, sm);
}

template <class T>
int launch_diag_typed(const PdgDiagPass& p, size_t smem, cudaStream_t st) {
  const int NN = p.n * p.n;
  const int threads = p.kpar * NN;
  const int blocks = p.ntx * p.nty * p.npop;
  auto go = [&](auto kern) -> int {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return (int)e;
    }
    kern<<<blocks, threads, smem, st>>>(p);
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
