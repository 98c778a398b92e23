// Transport of the corner populations of D3Q15 / D3Q27 by hyperplane sweeps of the whole
// periodic domain.
//
// The operator is that of pdg_corner.cuh (Section 3.1, eq. (3.7) split by axis, the theta
// step of eq. (3.11)): fn_c = Binv r_c - c1 f_c, r_c = f_c / theta + kx S_x Lt + ky S_y Bt +
// kz S_z Zt, the faces passed on being theta (Binv r_c).  A cell depends on its three
// upwind neighbours only, so the cells of a hyperplane j + r + k = s of the (column, row,
// layer) grid are independent: the 3-D form of the wavefronts of Section 4.2.
//
// Region.  Each population sweeps ONE region: the whole mesh plus, along every periodic
// axis, the start that begins wx (wy, wz) cells upwind (pdg_plan_corner: starting from the
// old face values there changes no output cell by more than 2^-57 of max|f| per
// boundary), or, along an inflow axis, the mesh from its inflow face.  The truncated start
// is paid once per population instead of once per box: at 128^3 cells and a width of 16
// the region holds 1.42x the output cells (face nodes only in the start), against about
// 2x for boxes of one block each.
//
// Blocks.  G blocks share a population (a cooperative launch of npop x G blocks, all
// resident at once).  At step s the cells of hyperplane s, enumerated layer by layer
// (row inside a layer), are cut into G contiguous ranges of equal work (n^3 nodes per
// output cell, the face nodes per start cell); a block processes its range in batches
// of nb cells: (A) r_c of every node of a batch in shared memory, (B) the dot products
// with Binv (row-major in shared memory, rows padded so that the 16-byte pair loads of
// neighbouring nodes fall on different banks) for every node of an output cell and for
// the face nodes of a start cell, while the next batch is copied in with cp.async.  The
// first batch of the next hyperplane is planned and its state copied in before the blocks
// meet (the state does not depend on the other blocks; the faces do).
//
// Faces.  The faces a cell passes on go to a global buffer (L2-resident), slot [layer]
// [row] of the RECEIVING cell, in the half of the step parity that reads it: x faces to
// (k, r) itself, y faces to (k, r + 1), z faces to (k + 1, r).  Every slot has one
// writer per step.  After a step the G blocks of the population meet at a counter in
// global memory (release / acquire at GPU scope); the faces are then read with cp.async.cg
// (L2, never a stale L1 line: the same addresses were read two steps before).  The
// region's upwind boundaries read the old face values (or the inflow data) instead.
//
// Waits.  A block waits only at that counter, and only for blocks of the same launch
// (all resident).  The wait is bounded (about two seconds of SM clock): if it runs out,
// or another block has given up, the block records PDG_HP_ERR_TIMEOUT in the launch's
// error word and returns; the host reports PDG_ERR_TIMEOUT at the next synchronising
// call.  The copies in flight at the counter (the next state) are waited for before the
// block returns.  The test switch p.stall makes every block wait for a count that no
// block reaches, with a bound of about 0.5 ms, so that the failure path runs without
// any fault.
#pragma once
#include <cuda_runtime.h>

#include "pdg_corner.cuh"
#include "pdg_corner_tc.cuh"

#define PDG_HP_ERR_TIMEOUT 2

namespace pdgdev {

// Shared-memory layout of the hyperplane kernel.
template <int NP>
struct HpShape {
  static constexpr int NF = NP * NP, NN = NF * NP;
  static constexpr int NFF = NN - (NP - 1) * (NP - 1) * (NP - 1);   // face nodes of a cell
  static constexpr int NN2 = (NN + 1) & ~1, NF2 = (NF + 1) & ~1;     // 16-byte rows
  static constexpr int RS = NN2 + 3 * NF2;   // staged row: state, then the x, y, z inflow faces
  static constexpr int BS = NN2 + ((NN2 / 2) % 2 == 0 ? 2 : 0);   // Binv row stride: odd in 16-byte units
  static constexpr int RB = BS;   // row stride of theta r in shared memory (the same rule)
};

// tc != 0: the tensor-core form (nb = 128 cells, one product row each) adds, first and
// 128-byte aligned, the two TF32 splits of the A operand (128 x K) and of Binv (N x K),
// x~ of the batch, the residual stencil and the mbarriers; it keeps no Binv of its own and
// no item table.
struct HpSmem {
  size_t aop, bop, xt, kt, ktf, mbar;
  size_t binv, stage, rbuf, off0, nodeoff, colx, rowy, layz, rcell, ritem, cr, ck, cit, icell, misc, total;
  __host__ __device__ HpSmem(int n, int nb, int RX, int RY, int RZ, int tc = 0) {
    const int NF = n * n, NN = NF * n, NN2 = (NN + 1) & ~1, NF2 = (NF + 1) & ~1, RS = NN2 + 3 * NF2;
    const int BS = NN2 + ((NN2 / 2) % 2 == 0 ? 2 : 0);
    const int KP = (NN + 7) & ~7, NPAD = KP < 16 ? 16 : KP;
    size_t o = 0;
    auto take = [&](size_t bytes) {
      o = (o + 15) / 16 * 16;
      const size_t at = o;
      o += bytes;
      return at;
    };
    aop = bop = xt = kt = ktf = mbar = 0;
    if (tc) {
      aop = take(sizeof(float) * 2 * 128 * KP);
      bop = take(sizeof(float) * 2 * NPAD * KP);
      xt = take(sizeof(float) * 128 * NN);
      kt = take(sizeof(double) * 3 * n * n);
      ktf = take(sizeof(float) * 2 * 3 * n * n);
      mbar = take(32);   // mbarrier (8 bytes), an idle mbarrier (8), TMEM base (4)
    }
    binv = take(tc ? 0 : sizeof(double) * NN * BS);
    stage = take(sizeof(double) * 2 * (size_t)nb * RS);
    rbuf = take(sizeof(double) * (size_t)nb * BS);
    off0 = take(sizeof(long long) * 2 * nb);
    nodeoff = take(sizeof(long long) * NN);
    colx = take(sizeof(long long) * (RX + 1));
    rowy = take(sizeof(long long) * (RY + 1));
    layz = take(sizeof(long long) * (RZ + 1));
    rcell = take(sizeof(int) * (RZ + 1));
    ritem = take(sizeof(int) * (RZ + 1));
    cr = take(sizeof(int) * 2 * nb);
    ck = take(sizeof(int) * 2 * nb);
    cit = take(sizeof(int) * 2 * (nb + 1));
    icell = take(tc ? 0 : sizeof(unsigned short) * 2 * (size_t)nb * NN);   // cell of each item of a batch
    misc = take(sizeof(int) * 96);   // fnode[NFF <= 37], range bounds, abort flag, warp sums
    total = o;
  }
};

// 16-byte copy global -> shared that bypasses L1 (cp.async.cg): face slots written by
// other blocks since this block last read the same addresses.
__device__ __forceinline__ void cp_async16_cg(void* smem, const double* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Rows of hyperplane s in layer k: r in [rlo, rhi] (j = s - r - k in [0, RX)); returns the
// count (0 when the layer does not meet the hyperplane).
__device__ __forceinline__ int hp_rows(int s, int k, int RX, int RY, int* rlo, int* rhi) {
  *rlo = max(0, s - k - (RX - 1));
  *rhi = min(RY - 1, s - k);
  return max(0, *rhi - *rlo + 1);
}

// Output rows of layer k on hyperplane s: [olo, ohi] (j >= wx, r >= wy, k >= wz).
__device__ __forceinline__ int hp_out_rows(int s, int k, int rlo, int rhi, int wx, int wy, int wz, int* olo) {
  if (k < wz) {
    *olo = 0;
    return 0;
  }
  *olo = max(rlo, wy);
  const int ohi = min(rhi, s - k - wx);
  return max(0, ohi - *olo + 1);
}

// Two consecutive 8-byte words of shared memory (16-byte aligned) in one load.
__device__ __forceinline__ void ld_pair(const double* p, double& a, double& b) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  a = v.x;
  b = v.y;
}

// TC = 0: FP64 or double-float dot products with Binv (T = double or dd).  TC = 1 / 2: the
// tensor-core form (T = double, FP64 state): per batch of at most 128 cells, the products
// X~ = (theta R) Binv^T as three TF32 split products on tcgen05 (rows = cells), the residual
// theta r - B x~ through the Kronecker sum (TC = 1: FP64; 2: double-float), a second split
// product for the correction d, and x = x~ + d, the face values (pdg_corner_tc.cuh has the
// same arithmetic on box anti-diagonals).
template <int NP, class T, int TC>
__device__ __forceinline__ void corner_hp_body(const PdgCornerPass& p, unsigned char* smraw) {
  using S = HpShape<NP>;
  constexpr int NF = S::NF, NN = S::NN, NFF = S::NFF, NN2 = S::NN2, NF2 = S::NF2, RS = S::RS, BS = S::BS;
  constexpr int RB = S::RB;
  constexpr int NT = 512;
  const int G = p.hg, nb = p.hnb;
  const int pop = blockIdx.x / G, gi = blockIdx.x % G;
  const PdgCornerCoef& C = p.c;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  CornerGeom g;
  g.fin = p.fin[pop];
  g.fout = p.fout[pop];
  g.sx = p.sx[pop];
  g.sy = p.sy[pop];
  g.sz = p.sz[pop];
  g.sa = p.sa;
  g.sb = p.sb;
  g.sc = p.sc;
  g.wx = p.per[0] ? C.wx : 0;
  g.wy = p.per[1] ? C.wy : 0;
  g.wz = p.per[2] ? C.wz : 0;
  g.bx = !p.per[0];
  g.by = !p.per[1];
  g.bz = !p.per[2];
  g.X0 = g.Y0 = g.Z0 = 0;
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
  const int RX = p.ncx + g.wx, RY = p.ncy + g.wy, RZ = p.ncz + g.wz;
  g.ncol = RX;
  g.nrow = RY;
  g.nlay = RZ;
  g.zt = nullptr;

  const HpSmem L(NP, nb, RX, RY, RZ, TC);
  T* Bq = reinterpret_cast<T*>(smraw + L.binv);        // Binv[q][m] at q * BS + m
  T* stage = reinterpret_cast<T*>(smraw + L.stage);    // 8-byte words (FP64 or a float pair)
  T* rbuf = reinterpret_cast<T*>(smraw + L.rbuf);      // theta r of cell c at c * RB
  long long* off0 = reinterpret_cast<long long*>(smraw + L.off0);        // node (0, 0, 0) of a cell
  long long* nodeoff = reinterpret_cast<long long*>(smraw + L.nodeoff);  // node q from node 0
  long long* colx = reinterpret_cast<long long*>(smraw + L.colx);
  long long* rowy = reinterpret_cast<long long*>(smraw + L.rowy);
  long long* layz = reinterpret_cast<long long*>(smraw + L.layz);
  int* rcell = reinterpret_cast<int*>(smraw + L.rcell);
  int* ritem = reinterpret_cast<int*>(smraw + L.ritem);
  int* cr = reinterpret_cast<int*>(smraw + L.cr);
  int* ck = reinterpret_cast<int*>(smraw + L.ck);
  int* cit = reinterpret_cast<int*>(smraw + L.cit);
  unsigned short* icell = reinterpret_cast<unsigned short*>(smraw + L.icell);
  int* misc = reinterpret_cast<int*>(smraw + L.misc);
  int* fnode = misc;            // [NFF]
  int* range = misc + 40;       // [2]: this block's cells [range[0], range[1]) of the step
  volatile int* abort_flag = misc + 42;
  int* wsum = misc + 48;        // [16]: per-warp sums
  int* wsum2 = misc + 64;       // [16]

  for (int i = tid; i < (TC ? 0 : NN * BS); i += NT) {
    const int q = i / BS, m = i % BS;
    if constexpr (__is_same(T, double)) {
      Bq[i] = m < NN ? p.binv[q * NN + m] : 0.0;
    } else {
      Bq[i] = m < NN ? T{p.binv_f[2 * (q * NN + m)], p.binv_f[2 * (q * NN + m) + 1]} : T{0.0f, 0.0f};
    }
  }
  for (int q = tid; q < NN; q += NT)
    nodeoff[q] = (long long)(g.sz * (q / NF)) * g.sc + (long long)(g.sy * ((q / NP) % NP)) * g.sb +
                 (long long)(g.sx * (q % NP)) * g.sa;
  if (tid == 0) {
    int f = 0;
    for (int q = 0; q < NN; ++q)
      if (q % NP == NP - 1 || (q / NP) % NP == NP - 1 || q / NF == NP - 1) fnode[f++] = q;
    *abort_flag = 0;
  }
  for (int j = tid; j <= RX; j += NT) {
    const int tc = wrap_cell(j - 1 - g.wx, p.ncx);
    colx[j] = (long long)(g.sx > 0 ? tc * NP : (p.ncx - 1 - tc) * NP + (NP - 1)) * g.sa;
  }
  for (int r = tid; r <= RY; r += NT) {
    const int tr = wrap_cell(r - 1 - g.wy, p.ncy);
    rowy[r] = (long long)(g.sy > 0 ? tr * NP : (p.ncy - 1 - tr) * NP + (NP - 1)) * g.sb;
  }
  for (int k = tid; k <= RZ; k += NT) {
    const int tl = wrap_cell(k - 1 - g.wz, p.ncz);
    layz[k] = (long long)(g.sz > 0 ? tl * NP : (p.ncz - 1 - tl) * NP + (NP - 1)) * g.sc;
  }
  g.colx = colx;
  g.rowy = rowy;
  g.layz = layz;
  // tensor-core form: TMEM columns for the accumulator, the mbarriers, both A splits zero
  // (rows beyond a batch and columns k >= NN stay finite), both Binv splits from the host's
  // layout, the stencil of B
  using TS = TcShape<NP>;
  float* aop = reinterpret_cast<float*>(smraw + L.aop);
  float* bop = reinterpret_cast<float*>(smraw + L.bop);
  float* xt = reinterpret_cast<float*>(smraw + L.xt);
  double* kt = reinterpret_cast<double*>(smraw + L.kt);
  float* ktf = reinterpret_cast<float*>(smraw + L.ktf);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smraw + L.mbar);
  uint64_t* idle = mbar + 1;   // no thread or product ever arrives on it (the stall test waits here)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smraw + L.mbar + 16);
  if constexpr (TC != 0) {
    if (warp == 0) tc::tmem_alloc(tslot, TS::NCOL);
    if (tid == 0) {
      tc::mbar_init(mbar, 1);
      tc::mbar_init(idle, 1);
    }
    for (int i = tid; i < 2 * TS::AOPS; i += NT) aop[i] = 0.0f;
    for (int i = tid; i < 2 * TS::BOPS; i += NT) bop[i] = p.binv_tc[i];
    for (int i = tid; i < 3 * NP * NP; i += NT) {
      kt[i] = p.c.kt[i / (NP * NP)][i % (NP * NP)];
      ktf[2 * i] = p.c.kt_f[i / (NP * NP)][i % (NP * NP)][0];
      ktf[2 * i + 1] = p.c.kt_f[i / (NP * NP)][i % (NP * NP)][1];
    }
    tc::fence_before_sync();
  }
  __syncthreads();
  uint32_t tmem = 0;
  if constexpr (TC != 0) {
    tc::fence_after_sync();
    tmem = *tslot;
  }

  // theta r_c = f_c + theta kx S_x Lt + ... is what the block forms: its product with
  // Binv is the face value theta (Binv r_c) itself, and fn = (Binv (theta r) - (1 - theta) f)
  // / theta
  const T rth = PDG_DC(T, C, rtheta), omth = PDG_DC(T, C, omtheta);
  const T th = PDG_DC(T, C, theta);
  const T tkx = th * PDG_DC(T, C, kx), tky = th * PDG_DC(T, C, ky), tkz = th * PDG_DC(T, C, kz);
  // face slots of this population: [parity][face a][layer][row][NF2]
  const long long slab = (long long)RZ * RY * NF2;
  double* hf = p.hface + (long long)pop * 6 * slab;
  unsigned* bar = p.hbar + pop;
  const int NS = RX + RY + RZ - 2;

  // sum of ws[0 .. this warp) (the per-warp partial sums of a block scan): one load per lane
  // and a butterfly, instead of a serial loop over the earlier warps
  auto warps_before = [&](const int* ws) {
    int x = (lane < NT / 32 && lane < warp) ? ws[lane] : 0;
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
    return x;
  };

  // (0) cells and items of hyperplane s per layer, exclusive prefixes over the layers
  // (rcell, ritem), then (1) this block's cells: those whose first item lies in
  // [I gi / G, I (gi + 1) / G) (range).  Barriers inside; rcell / ritem are overwritten.
  auto plan_step = [&](int s) {
    const int per_t = (RZ + NT - 1) / NT, k0 = tid * per_t;
    int cs = 0, is = 0;
    for (int k = k0; k < min(RZ, k0 + per_t); ++k) {
      int rlo, rhi, olo;
      const int n = hp_rows(s, k, RX, RY, &rlo, &rhi);
      const int no = n ? hp_out_rows(s, k, rlo, rhi, g.wx, g.wy, g.wz, &olo) : 0;
      cs += n;
      is += n * NFF + no * (NN - NFF);
    }
    int vc = cs, vi = is;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int uc = __shfl_up_sync(0xffffffffu, vc, d), ui = __shfl_up_sync(0xffffffffu, vi, d);
      if (lane >= d) {
        vc += uc;
        vi += ui;
      }
    }
    if (lane == 31) {
      wsum[warp] = vc;
      wsum2[warp] = vi;
    }
    __syncthreads();
    const int bc = warps_before(wsum), bi = warps_before(wsum2);
    int pc = bc + vc - cs, pi = bi + vi - is;   // exclusive prefixes at k0
    for (int k = k0; k < min(RZ, k0 + per_t); ++k) {
      rcell[k] = pc;
      ritem[k] = pi;
      int rlo, rhi, olo;
      const int n = hp_rows(s, k, RX, RY, &rlo, &rhi);
      const int no = n ? hp_out_rows(s, k, rlo, rhi, g.wx, g.wy, g.wz, &olo) : 0;
      pc += n;
      pi += n * NFF + no * (NN - NFF);
    }
    if (tid == NT - 1) {
      rcell[RZ] = pc;
      ritem[RZ] = pi;
    }
    __syncthreads();
    if (warp < 2) {   // warp 0: the first cell of this block's range, warp 1: of the next
      const long long I = ritem[RZ];
      const int P = (int)(I * (gi + warp) / G);
      int le = 0;   // layers k with ritem[k] <= P (a non-decreasing table from ritem[0] = 0)
      for (int k = lane; k < RZ; k += 32) le += ritem[k] <= P ? 1 : 0;
#pragma unroll
      for (int d = 16; d >= 1; d >>= 1) le += __shfl_xor_sync(0xffffffffu, le, d);
      int c = rcell[RZ];
      if (lane == 0 && P < I) {
        const int lo = le - 1;   // layer with ritem[k] <= P < ritem[k + 1]
        int rlo, rhi, olo;
        hp_rows(s, lo, RX, RY, &rlo, &rhi);
        const int no = hp_out_rows(s, lo, rlo, rhi, g.wx, g.wy, g.wz, &olo);
        int a = rlo, b = rhi + 1;   // first row of the layer whose first item is >= P
        while (a < b) {
          const int m = (a + b) >> 1;
          const int before_out = no ? max(0, min(m, olo + no) - olo) : 0;
          const int start = ritem[lo] + (m - rlo) * NFF + before_out * (NN - NFF);
          if (start >= P) b = m;
          else a = m + 1;
        }
        c = rcell[lo] + (a - rlo);
      }
      if (lane == 0) range[warp] = c;
    }
    __syncthreads();
  };

  // cells [c0, c0 + cnt) of hyperplane s into table buffer buf: coordinates, offset of
  // node 0, the start of each cell's items (n^3 for an output cell, NFF else) and the
  // cell of every item.  One barrier inside; the tables are complete after the caller's
  // next barrier.
  auto batch_info = [&](int s, int c0, int cnt, int buf) {
    int items = 0;
    if (tid < cnt) {
      const int c = c0 + tid;
      int lo = 0, hi = RZ - 1;   // the layer: last k with rcell[k] <= c
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (rcell[mid] <= c) lo = mid;
        else hi = mid - 1;
      }
      int rlo, rhi;
      hp_rows(s, lo, RX, RY, &rlo, &rhi);
      const int r = rlo + (c - rcell[lo]);
      const int j = s - r - lo;
      cr[buf * nb + tid] = r;
      ck[buf * nb + tid] = lo;
      off0[buf * nb + tid] = layz[lo + 1] + rowy[r + 1] + colx[j + 1];
      items = (j >= g.wx && r >= g.wy && lo >= g.wz) ? NN : NFF;
    }
    int v = items;   // exclusive scan of items over the batch (cnt <= nb <= 512)
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, v, d);
      if (lane >= d) v += u;
    }
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    const int base = warps_before(wsum);
    if (tid < cnt) {
      cit[buf * (nb + 1) + tid] = base + v - items;
      if constexpr (TC == 0) {   // the tensor-core form maps one thread row to one cell
        unsigned short* ic = icell + (size_t)buf * nb * NN + (base + v - items);
        for (int i = 0; i < items; ++i) ic[i] = (unsigned short)tid;
      }
    }
    if (tid == cnt - 1) cit[buf * (nb + 1) + cnt] = base + v;
  };

  // copy the state (what & 1) and the inflow faces (what & 2) of the batch's cells into
  // stage[buf]; the faces of hyperplane s must be complete (after the blocks met)
  auto stage_batch = [&](int s, int cnt, int buf, int what) {
    double* sb = reinterpret_cast<double*>(stage + (size_t)buf * nb * RS);
    const int par = s & 1;
    if (what & 1)
      for (int i = tid; i < cnt * NN; i += NT) {
        const int c = i / NN, e = i % NN;
        cp_async8(sb + (size_t)c * RS + e, g.fin + off0[buf * nb + c] + nodeoff[e]);
      }
    if (what & 2) {   // one item per 16-byte chunk of a face slot
      constexpr int CH = NF2 / 2, per = 3 * CH;
      for (int i = tid; i < cnt * per; i += NT) {
        const int c = i / per, e = i % per;
        const int a = e / CH, u0 = 2 * (e % CH);
        const int r = cr[buf * nb + c], k = ck[buf * nb + c], j = s - r - k;
        double* dst = sb + (size_t)c * RS + NN2 + a * NF2 + u0;
        const bool edge = a == 0 ? j == 0 : (a == 1 ? r == 0 : k == 0);
        if (!edge) {
          cp_async16_cg(dst, hf + ((long long)(par * 3 + a) * RZ + k) * RY * NF2 + (long long)r * NF2 + u0);
          continue;
        }
        for (int u = u0; u < min(u0 + 2, NF); ++u) {   // the region's upwind boundary: old faces
          const int u1 = u / NP, u2 = u % NP;
          const double* src;
          if (a == 0) {   // +x face of the cell upwind of column 0: node (iz, iy) = (u1, u2)
            src = g.bx ? g.fbx + corner_py<NP>(g, r, u2) * g.fls[0][1] + corner_pz<NP>(g, k, u1) * g.fls[0][2]
                       : g.fin + corner_off(g, -1, r, k, u1, u2, NP - 1);
          } else if (a == 1) {   // +y face below row 0: node (iz, ix) = (u1, u2)
            src = g.by ? g.fby + corner_px<NP>(g, j, u2) * g.fls[1][0] + corner_pz<NP>(g, k, u1) * g.fls[1][2]
                       : g.fin + corner_off(g, j, -1, k, u1, NP - 1, u2);
          } else {   // +z face under layer 0: node (iy, ix) = (u1, u2)
            src = g.bz ? g.fbz + corner_px<NP>(g, j, u2) * g.fls[2][0] + corner_py<NP>(g, r, u1) * g.fls[2][1]
                       : g.fin + corner_off(g, j, r, -1, NP - 1, u1, u2);
          }
          cp_async8(dst + (u - u0), src);
        }
      }
    }
  };

  // Pipeline.  Table and stage buffers alternate with a running batch count (nbt) across
  // hyperplanes.  Before the blocks meet after hyperplane s, the block has planned
  // hyperplane s + 1, filled the tables of its first batch and started copying that
  // batch's state; after the meeting it copies the batch's faces.
  // tensor-core form: one thread issues the three split products of a solve (then commits
  // them to the mbarrier) and later waits for them, boundedly
  constexpr uint32_t IDESC = tc::idesc_tf32(128, TS::NPAD);
  uint32_t phase = 0;
  // descriptors of the operand splits at K-step 0; a K-step of 8 moves the start address by
  // two core-matrix columns (the address field is the byte address / 16, and shared
  // memory addresses stay below 2^18 bytes, so the offsets add without a carry)
  const uint64_t adesc[2] = {tc::smem_desc(tc::smem_u32(aop), 16 * 128, 128),
                             tc::smem_desc(tc::smem_u32(aop + TS::AOPS), 16 * 128, 128)};
  const uint64_t bdesc[2] = {tc::smem_desc(tc::smem_u32(bop), (TS::NPAD / 8) * 128, 128),
                             tc::smem_desc(tc::smem_u32(bop + TS::BOPS), (TS::NPAD / 8) * 128, 128)};
  auto mma_issue = [&]() {   // tid 0 only
    tc::fence_after_sync();
#pragma unroll
    for (int sp = 0; sp < 3; ++sp) {   // (hi, hi), (lo, hi), (hi, lo)
#pragma unroll
      for (int ks = 0; ks < TS::KP / 8; ++ks) {
        const uint64_t ad = adesc[sp == 1 ? 1 : 0] + (uint64_t)((ks * 2 * 16 * 128) >> 4);
        const uint64_t bd = bdesc[sp == 2 ? 1 : 0] + (uint64_t)((ks * 2 * (TS::NPAD / 8) * 128) >> 4);
        tc::mma_tf32(tmem, ad, bd, IDESC, (sp | ks) ? 1u : 0u);
      }
    }
    tc::commit(mbar);
  };
  auto mma_wait = [&]() {    // tid 0 only; records a timeout for the whole block
    const bool ok = p.stall ? tc::mbar_wait_bounded(idle, 0, 1000000LL)
                            : tc::mbar_wait_bounded(mbar, phase & 1, 2000000000LL);
    ++phase;
    if (!ok) {
      *abort_flag = 1;
      atomicExch(p.err, PDG_TC_ERR_TIMEOUT);
    }
  };
  const int lq = warp & 3, cc = warp >> 2;        // TMEM lane quarter, column block
  const int trow = 32 * lq + lane;                // this thread's TMEM row (cell of the batch)
  const uint32_t taddr = tmem + ((uint32_t)(32 * lq) << 16) + (uint32_t)(cc * TS::CW);
  bool aborted = false;

  int nbt = 0;
  plan_step(0);
  int cb = range[0], ce = range[1];
  if (ce > cb) {
    batch_info(0, cb, min(nb, ce - cb), 0);
    __syncthreads();
    stage_batch(0, min(nb, ce - cb), 0, 1);
  }
  for (int s = 0; s < NS; ++s) {
    const int nbat = (ce - cb + nb - 1) / nb;
    if (nbat > 0) stage_batch(s, min(nb, ce - cb), nbt & 1, 2);
    for (int bI = 0; bI < nbat && !aborted; ++bI, ++nbt) {
      const int buf = nbt & 1;
      const int c0 = cb + bI * nb, cnt = min(nb, ce - c0);
      cp_async_wait_all();
      __syncthreads();
      // (A) theta r_c of every node of the batch.  The item order is the one each form ran
      // fastest with (measured): double-float (T = dd), item i is node i / nb of cell i % nb
      // (nb a power of two: a warp takes one node of 32 cells, so its face terms are
      // warp-uniform); FP64, consecutive nodes of a cell; tensor-core form, item i of a group
      // of 32 is (cell 8 cg + i / 4, node 4 qg + i % 4), whose operand words are consecutive
      // in the core-matrix layout (i = tc::op_index(c, q, 128), no bank conflict)
      const T* sb = stage + (size_t)buf * nb * RS;
      constexpr int QG = (NN + 3) / 4;
      const int lgnb = __ffs(nb) - 1;
      constexpr bool by_node = !__is_same(T, double);
      for (int i = tid; i < (TC ? QG * 16 * 32 : (by_node ? (NN << lgnb) : cnt * NN)); i += NT) {
        int c, q;
        if constexpr (TC != 0) {
          c = 8 * ((i >> 5) & 15) + ((i & 31) >> 2);
          q = 4 * (i >> 9) + (i & 3);
          if (c >= cnt || q >= NN) continue;
        } else if constexpr (by_node) {
          q = i >> lgnb;
          c = i & (nb - 1);
          if (c >= cnt) continue;
        } else {
          c = i / NN;
          q = i % NN;
        }
        const int iz = q / NF, iy = (q / NP) % NP, ix = q % NP;
        const T* row = sb + (size_t)c * RS;
        T rv = row[q];
        if (ix == 0) rv = fma(tkx, row[NN2 + iz * NP + iy], rv);
        if (iy == 0) rv = fma(tky, row[NN2 + NF2 + iz * NP + ix], rv);
        if (iz == 0) rv = fma(tkz, row[NN2 + 2 * NF2 + iy * NP + ix], rv);
        rbuf[(size_t)c * RB + q] = rv;
        if constexpr (TC != 0) {   // row c of the A operand: theta r_c split into TF32 parts
          float hi, lo;
          tc::split_tf32_fast(rv, &hi, &lo);
          aop[i] = hi;
          aop[TS::AOPS + i] = lo;
        }
      }
      const bool more = bI + 1 < nbat;
      if (more) batch_info(s, c0 + nb, min(nb, ce - c0 - nb), buf ^ 1);   // has its own barrier
      const int par1 = (s + 1) & 1;
      if constexpr (TC != 0) {
        tc::fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) mma_issue();
        if (more) stage_batch(s, min(nb, ce - c0 - nb), buf ^ 1, 3);   // while the products run
        if (tid == 0) mma_wait();
        __syncthreads();
        if (*abort_flag) {
          aborted = true;
          break;
        }
        // (L1) x~ from TMEM (rows = cells, this warp's block of node columns)
        tc::fence_after_sync();
        float xr[TS::CW];
        tc::tmem_ld<TS::CW>(taddr, xr);
        if (trow < cnt) {
#pragma unroll
          for (int e = 0; e < TS::CW; ++e)
            if (cc * TS::CW + e < NN) xt[trow * NN + cc * TS::CW + e] = xr[e];
        }
        tc::fence_before_sync();
        __syncthreads();
        // (R) residual theta r - B x~ of every node, split into the operand
        for (int i = tid; i < QG * 16 * 32; i += NT) {   // i = tc::op_index(c, q, 128)
          const int c = 8 * ((i >> 5) & 15) + ((i & 31) >> 2), q = 4 * (i >> 9) + (i & 3);
          if (c >= cnt || q >= NN) continue;
          const int qz = q / NF, qy = (q / NP) % NP, qx = q % NP;
          const int idx = i;
          if constexpr (TC == 1) {
            const double res = tc_residual<NP>(rbuf[(size_t)c * RB + q], xt + c * NN, kt, qz, qy, qx);
            float hi, lo;
            tc::split_tf32_fast(res, &hi, &lo);
            aop[idx] = hi;
            aop[TS::AOPS + idx] = lo;
          } else {
            const dd res = tc_residual_dd<NP>(rbuf[(size_t)c * RB + q], xt + c * NN, ktf, qz, qy, qx);
            const float hi = tc::tf32_rna(res.hi);
            aop[idx] = hi;
            aop[TS::AOPS + idx] = tc::tf32_rna(__fadd_rn(__fsub_rn(res.hi, hi), res.lo));
          }
        }
        tc::fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
          mma_issue();
          mma_wait();
        }
        __syncthreads();
        if (*abort_flag) {
          aborted = true;
          break;
        }
        // (L2) x = x~ + d (= theta Binv r: the face value); outputs and faces
        tc::fence_after_sync();
        float dv[TS::CW];
        tc::tmem_ld<TS::CW>(taddr, dv);
        if (trow < cnt) {
          const int r = cr[buf * nb + trow], k = ck[buf * nb + trow], j = s - r - k;
          const bool out = cit[buf * (nb + 1) + trow + 1] - cit[buf * (nb + 1) + trow] == NN;
          const long long o0 = off0[buf * nb + trow];
          double* fx = hf + (long long)par1 * 3 * slab + ((long long)k * RY + r) * NF2;
#pragma unroll
          for (int e = 0; e < TS::CW; ++e) {
            const int q = cc * TS::CW + e;
            if (q < NN) {
              const double x = tc::f64_from_f32_bits(xr[e]) + tc::f64_from_f32_bits(dv[e]);
              const int qz = q / NF, qy = (q / NP) % NP, qx = q % NP;
              if (out) st(g.fout + o0 + nodeoff[q], (x - omth * sb[(size_t)trow * RS + q]) * rth);
              if (qx == NP - 1 && j + 1 < RX) st(fx + qz * NP + qy, x);
              if (qy == NP - 1 && r + 1 < RY) st(fx + slab + NF2 + qz * NP + qx, x);
              if (qz == NP - 1 && k + 1 < RZ) st(fx + 2 * slab + (long long)RY * NF2 + qy * NP + qx, x);
            }
          }
        }
        tc::fence_before_sync();
        continue;
      }
      __syncthreads();
      // (B) items of the batch: every node of an output cell, the face nodes of a start cell;
      // each thread issues its share of the next batch's copies after its first item
      const int* itb = cit + buf * (nb + 1);
      const unsigned short* icb = icell + (size_t)buf * nb * NN;
      const int nitems = itb[cnt];
      bool staged = !more;
      for (int it = tid; it < nitems; it += NT) {
        const int c = icb[it], loc = it - itb[c];
        const bool out = itb[c + 1] - itb[c] == NN;
        const int q = out ? loc : fnode[loc];
        const T* rc = rbuf + (size_t)c * RB;
        const T* br = Bq + (size_t)q * BS;
        T acc;
        if constexpr (__is_same(T, double)) {
          // one chain (one warp per SM sub-partition keeps its FP64 unit busy with a
          // dependent chain), 16-byte pair loads of Binv[q][m..m+1] and r[m..m+1]
          double a = 0.0;
#pragma unroll
          for (int m = 0; m + 1 < NN; m += 2) {
            double b0, b1, x0, x1;
            ld_pair(br + m, b0, b1);
            ld_pair(rc + m, x0, x1);
            a = fma(b0, x0, a);
            a = fma(b1, x1, a);
          }
          if constexpr (NN % 2) a = fma(br[NN - 1], rc[NN - 1], a);
          acc = a;
        } else {
          // compensated dot product (see dot_acc): exact high products and sums, the
          // rounding errors and cross terms gathered in one FP32 accumulator
          float Sh = 0.0f, Ll = 0.0f;
#pragma unroll 8
          for (int m = 0; m < NN; ++m) {
            const T a = br[m], bv = rc[m];
            const dd pr = dd_two_prod(a.hi, bv.hi);
            const float cross = __fmaf_rn(a.hi, bv.lo, __fmul_rn(a.lo, bv.hi));
            const dd sm2 = dd_two_sum(Sh, pr.hi);
            Sh = sm2.hi;
            Ll = __fadd_rn(Ll, __fadd_rn(sm2.lo, __fadd_rn(pr.lo, cross)));
          }
          acc = dd_fast_two_sum(Sh, Ll);
        }
        const int qz = q / NF, qy = (q / NP) % NP, qx = q % NP;
        if (out) st(g.fout + off0[buf * nb + c] + nodeoff[q], (acc - omth * sb[(size_t)c * RS + q]) * rth);
        if (qx == NP - 1 || qy == NP - 1 || qz == NP - 1) {
          const int r = cr[buf * nb + c], k = ck[buf * nb + c], j = s - r - k;
          const T face = acc;
          double* fx = hf + (long long)par1 * 3 * slab + ((long long)k * RY + r) * NF2;
          if (qx == NP - 1 && j + 1 < RX) st(fx + qz * NP + qy, face);
          if (qy == NP - 1 && r + 1 < RY) st(fx + slab + NF2 + qz * NP + qx, face);
          if (qz == NP - 1 && k + 1 < RZ) st(fx + 2 * slab + (long long)RY * NF2 + qy * NP + qx, face);
        }
        if (!staged) {
          stage_batch(s, min(nb, ce - c0 - nb), buf ^ 1, 3);
          staged = true;
        }
      }
      if (!staged) stage_batch(s, min(nb, ce - c0 - nb), buf ^ 1, 3);
    }
    if (aborted) break;
    // (2) plan hyperplane s + 1 and start copying the state of its first batch; then the
    // population's blocks meet: every face of step s is written before any block reads it
    // at step s + 1
    if (s + 1 < NS) {
      plan_step(s + 1);   // its barriers also end this step's work on the tables
      cb = range[0];
      ce = range[1];
      if (ce > cb) {
        batch_info(s + 1, cb, min(nb, ce - cb), nbt & 1);
        __syncthreads();
        stage_batch(s + 1, min(nb, ce - cb), nbt & 1, 1);
      }
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      atomicAdd(bar, 1u);
      // test switch (p.stall): a count no block reaches, with a bound of about 0.5 ms
      const unsigned target = p.stall ? 0xffffffffu : (unsigned)G * (unsigned)(s + 1);
      const long long limit = p.stall ? 1000000LL : 4000000000LL;
      const long long t0 = clock64();
      int ok = 1;
      while (ld_acquire_gpu(bar) < target) {
        if (*(volatile int*)p.err != 0 || clock64() - t0 > limit) {
          atomicCAS(p.err, 0, PDG_HP_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
      __threadfence();
      if (!ok) *abort_flag = 1;
    }
    __syncthreads();
    if (*abort_flag) {
      aborted = true;
      break;
    }
  }
  // the copies in flight (after a failed wait: the next state's), then, tensor-core form,
  // the products in flight after a timed-out wait (bounded) and the TMEM columns
  if constexpr (TC != 0)
    if (aborted && tid == 0) tc::mbar_wait_bounded(mbar, (phase - 1) & 1, 2000000000LL);
  cp_async_wait_all();
  if constexpr (TC != 0) {
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
      tc::fence_after_sync();
      tc::tmem_dealloc(tmem, TS::NCOL);
    }
  }
}

template <int NP, class T, int TC>
__global__ void __launch_bounds__(512, 1) corner_hp_kernel(const __grid_constant__ PdgCornerPass p) {
  extern __shared__ __align__(128) unsigned char smraw[];
  corner_hp_body<NP, T, TC>(p, smraw);
}

// Blocks of the kernel for n that fit one SM with smem bytes of shared memory.
template <class T, int TC>
int hp_blocks_per_sm(int n, size_t smem) {
  auto occ = [&](auto kern) -> int {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, 512, smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return b;
  };
  switch (n) {
    case 2: return occ(corner_hp_kernel<2, T, TC>);
    case 3: return occ(corner_hp_kernel<3, T, TC>);
    case 4:
      if constexpr (TC == 0) return occ(corner_hp_kernel<4, T, TC>);
  }
  return 0;
}

// Cooperative launch of npop x hg blocks of 512 threads (the host sized hg so that all are
// resident).
template <class T, int TC>
int launch_corner_hp_typed(const PdgCornerPass& p, size_t smem, cudaStream_t st) {
  auto go = [&](auto kern) -> int {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    e = cudaMemsetAsync(p.hbar, 0, sizeof(unsigned) * 8, st);
    if (e != cudaSuccess) return (int)e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(p.npop * p.hg));
    cfg.blockDim = dim3(512);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, p);
    return (int)e;
  };
  switch (p.n) {
    case 2: return go(corner_hp_kernel<2, T, TC>);
    case 3: return go(corner_hp_kernel<3, T, TC>);
    case 4:
      if constexpr (TC == 0) return go(corner_hp_kernel<4, T, TC>);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace pdgdev
