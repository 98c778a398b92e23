// Tensor-core form of the corner transport (D3Q15 / D3Q27 velocities lambda (+-1,+-1,+-1)):
// the dense cell-inverse applications x = Binv r of the truncated-box sweep (pdg_corner.cuh)
// run on the Blackwell tensor cores, and one refinement step restores FP64-level accuracy.
//
// The cells of one anti-diagonal of a box layer are independent, so their cell solves are
// one matrix product X = R Binv^T with R = [r_c] (cells x NN) and Binv (NN x NN, the inverse
// of B = I + theta sum_a nu_a K_a of Section 3.1, eq. (3.7) under the theta step of eq.
// (3.11)): the (Np x Np) . (Np x cells) contraction.  It runs as tcgen05.mma kind::tf32
// (M = 128 rows of cells, N = K = the NN nodes padded to 16 / 32 / 64), FP32 accumulation
// in TMEM, each operand split into two TF32 parts (v = hi + lo, 22 significant bits):
//   X~ = R_hi Binv_hi + R_lo Binv_hi + R_hi Binv_lo    (relative error ~1e-6)
// (the FP64 values split into TF32 parts, and FP32 results widened, by integer operations on
// the bit patterns, which keeps these conversions off the FP64 pipe),
// then the residual of the cell system, through the Kronecker sum B (1 + 3n FMA per node),
//   res = r - B x~ = r - x~ - sum_a (theta nu_a K) x~ along axis a
// in FP64 (RES = 0) or in double-float on the FP32 pipes (RES = 1), a second split
// product D = Res Binv^T and x = x~ + d (relative error ~1e-13 on the cell systems of the
// sweep).  The state stays FP64; the face values and outputs are formed from x as in the
// FP64 kernel: fn = x - c1 f, faces theta x.
//
// Per anti-diagonal step: (A) r_c of every cell (FP64) and its split into the MMA operand;
// one thread issues the MMAs and commits them to an mbarrier while the block stages the
// next anti-diagonal with cp.async; (L1) the tensor results are read from TMEM (a warp
// reads the TMEM lanes of its quarter: rows = cells, a block of columns = nodes); (R) the
// residual and its split; second MMA; (L2) x = x~ + d, outputs and faces.  Only one
// thread waits on the mbarrier, with a bound of about one second; if the bound runs out it
// records PDG_TC_ERR_TIMEOUT in the launch's error word, and the whole block (which reads
// the decision from shared memory after a barrier) waits once more, boundedly, for its
// MMAs in flight, waits for its copies, frees its TMEM and returns.
#pragma once
#include <cuda_runtime.h>

#include "pdg_corner.cuh"
#include "pdg_tc.cuh"

#define PDG_TC_ERR_TIMEOUT 1

namespace pdgdev {

template <int NP>
struct TcShape {
  static constexpr int NN = NP * NP * NP;
  static constexpr int KP = (NN + 7) & ~7;              // contraction length (multiple of 8)
  static constexpr int NPAD = KP < 16 ? 16 : KP;         // MMA N (M = 128 needs N % 16 == 0)
  static constexpr int NCOL = NPAD < 32 ? 32 : NPAD;     // TMEM columns (power of 2 >= 32)
  static constexpr int THREADS = 512;                    // 16 warps: 4 per TMEM lane quarter
  static constexpr int CW = NPAD / 4;                    // columns per warp in a TMEM load
  static constexpr int AOPS = 128 * KP;                  // floats of one A split
  static constexpr int BOPS = NPAD * KP;                 // floats of one B split
};

// Shared-memory carve-up of the tensor-core corner kernel (offsets in bytes) for `layers`
// box layers swept together (their anti-diagonals' cells share one product).
template <int NP>
struct TcSmem {
  size_t aop, bop, rbuf, fbuf, xt, lt, bt, lbnd, bbnd, kt, ktf, colx, rowy, layz, mbar, total;
  __host__ __device__ TcSmem(int CM, int RM, int LM, int layers) {
    using S = TcShape<NP>;
    constexpr int NF = CornerRow<NP>::NF, NN = CornerRow<NP>::NN, RS = CornerRow<NP>::RS;
    const int amax = CM < RM ? CM : RM;
    size_t o = 0;
    auto take = [&](size_t bytes, size_t align) {
      o = (o + align - 1) / align * align;
      const size_t at = o;
      o += bytes;
      return at;
    };
    aop = take(sizeof(float) * 2 * S::AOPS, 128);
    bop = take(sizeof(float) * 2 * S::BOPS, 128);
    rbuf = take(sizeof(double) * layers * amax * NN, 16);
    fbuf = take(sizeof(double) * 2 * layers * amax * RS, 16);
    xt = take(sizeof(float) * layers * amax * NN, 16);
    lt = take(sizeof(double) * layers * 2 * (CM + 1) * NF, 16);
    bt = take(sizeof(double) * layers * 2 * CM * NF, 16);
    lbnd = take(sizeof(double) * layers * 2 * NF, 16);
    bbnd = take(sizeof(double) * layers * 2 * NF, 16);
    kt = take(sizeof(double) * 3 * NP * NP, 16);
    ktf = take(sizeof(float) * 2 * 3 * NP * NP, 16);
    colx = take(sizeof(long long) * (CM + 1), 16);
    rowy = take(sizeof(long long) * (RM + 1), 16);
    layz = take(sizeof(long long) * (LM + 1), 16);
    mbar = take(32, 16);   // mbarrier (8 bytes), an idle mbarrier (8), TMEM base (4), timeout decision (4)
    total = o;
  }
};

// r - (x~ + sum_a Kt_a x~ along a) for node (qz, qy, qx) of one cell; x~ in FP32.
template <int NP>
__device__ __forceinline__ double tc_residual(double r, const float* xc, const double* kt, int qz, int qy, int qx) {
  using tc::f64_from_f32_bits;
  double s = f64_from_f32_bits(xc[(qz * NP + qy) * NP + qx]);
#pragma unroll
  for (int i = 0; i < NP; ++i) s = fma(kt[qx * NP + i], f64_from_f32_bits(xc[(qz * NP + qy) * NP + i]), s);
#pragma unroll
  for (int i = 0; i < NP; ++i)
    s = fma(kt[NP * NP + qy * NP + i], f64_from_f32_bits(xc[(qz * NP + i) * NP + qx]), s);
#pragma unroll
  for (int i = 0; i < NP; ++i)
    s = fma(kt[2 * NP * NP + qz * NP + i], f64_from_f32_bits(xc[(i * NP + qy) * NP + qx]), s);
  return r - s;
}

// The same residual in double-float arithmetic: exact products of the coefficient's high
// part with x~ (two_prod), the high sum kept exactly (two_sum), rounding errors and the
// coefficient's low part gathered in one FP32 accumulator; r - s with the accurate
// double-word addition (the two nearly cancel).  Returns the residual as a float pair.
template <int NP>
__device__ __forceinline__ dd tc_residual_dd(double r, const float* xc, const float* ktf, int qz, int qy, int qx) {
  float S = xc[(qz * NP + qy) * NP + qx], L = 0.0f;
  auto term = [&](int a, int row, int i, float x) {
    const float kh = ktf[2 * ((a * NP + row) * NP + i)], kl = ktf[2 * ((a * NP + row) * NP + i) + 1];
    const dd p = dd_two_prod(kh, x);
    const dd s = dd_two_sum(S, p.hi);
    S = s.hi;
    L = __fadd_rn(L, __fadd_rn(s.lo, __fmaf_rn(kl, x, p.lo)));
  };
#pragma unroll
  for (int i = 0; i < NP; ++i) term(0, qx, i, xc[(qz * NP + qy) * NP + i]);
#pragma unroll
  for (int i = 0; i < NP; ++i) term(1, qy, i, xc[(qz * NP + i) * NP + qx]);
#pragma unroll
  for (int i = 0; i < NP; ++i) term(2, qz, i, xc[(i * NP + qy) * NP + qx]);
  const dd s = dd_fast_two_sum(S, L);
  dd rr;
  tc::split_dd_fast(r, &rr.hi, &rr.lo);
  return dd_add_accurate(rr, dd{-s.hi, -s.lo});
}

template <int NP, int RES, int LAYERS>
__device__ __forceinline__ void corner_tc_body(const PdgCornerPass& p, unsigned char* smem) {
  using S = TcShape<NP>;
  constexpr int NF = CornerRow<NP>::NF, NN = CornerRow<NP>::NN, RS = CornerRow<NP>::RS;
  constexpr int KP = S::KP, NPAD = S::NPAD, CW = S::CW;
  constexpr uint32_t IDESC = tc::idesc_tf32(128, NPAD);
  int b = blockIdx.x;
  const int txi = b % p.ntx;
  b /= p.ntx;
  const int tyi = b % p.nty;
  b /= p.nty;
  const int tzi = b % p.ntz;
  const int pop = b / p.ntz;
  const PdgCornerCoef& C = p.c;
  const int CM = p.tx + C.wx, RM = p.ty + C.wy;
  const int amax = min(CM, RM);
  const TcSmem<NP> L(CM, RM, p.tz + C.wz, LAYERS);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

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
    for (int bb = 0; bb < 3; ++bb) g.fls[a][bb] = p.fls[a][bb];
  }
  g.fbx = fbs[0];
  g.fby = fbs[1];
  g.fbz = fbs[2];
  g.ncol = min(p.tx, p.ncx - X0) + g.wx;
  g.nrow = min(p.ty, p.ncy - Y0) + g.wy;
  g.nlay = min(p.tz, p.ncz - Z0) + g.wz;
  g.zt = p.zt + (long long)blockIdx.x * RM * CM * NF;
  const int T_steps = g.ncol + g.nrow - 1;

  float* aop = reinterpret_cast<float*>(smem + L.aop);
  float* bop = reinterpret_cast<float*>(smem + L.bop);
  double* rbuf = reinterpret_cast<double*>(smem + L.rbuf);   // [layer][amax][NN]
  double* fbuf = reinterpret_cast<double*>(smem + L.fbuf);   // [parity][layer][amax][RS]
  float* xt = reinterpret_cast<float*>(smem + L.xt);         // [layer][amax][NN]
  double* Lt = reinterpret_cast<double*>(smem + L.lt);       // [layer][parity][CM + 1][NF]
  double* Bt = reinterpret_cast<double*>(smem + L.bt);       // [layer][parity][CM][NF]
  double* lbnd = reinterpret_cast<double*>(smem + L.lbnd);   // [layer][parity][NF]
  double* bbnd = reinterpret_cast<double*>(smem + L.bbnd);
  double* kt = reinterpret_cast<double*>(smem + L.kt);
  float* ktf = reinterpret_cast<float*>(smem + L.ktf);
  long long* colx = reinterpret_cast<long long*>(smem + L.colx);
  long long* rowy = reinterpret_cast<long long*>(smem + L.rowy);
  long long* layz = reinterpret_cast<long long*>(smem + L.layz);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L.mbar);
  uint64_t* idle = mbar + 1;   // no thread or MMA ever arrives on it (the stall test waits here)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L.mbar + 16);
  int* abort_flag = reinterpret_cast<int*>(smem + L.mbar + 20);
  const int LtS = CM + 1, BtS = CM;
  auto FB = [&](int par, int ls) { return fbuf + ((size_t)par * LAYERS + ls) * amax * RS; };
  auto LT = [&](int ls, int par) { return Lt + ((size_t)ls * 2 + par) * LtS * NF; };
  auto BT = [&](int ls, int par) { return Bt + ((size_t)ls * 2 + par) * BtS * NF; };
  auto LB = [&](int ls, int par) { return lbnd + ((size_t)ls * 2 + par) * NF; };
  auto BB = [&](int ls, int par) { return bbnd + ((size_t)ls * 2 + par) * NF; };

  // set-up: TMEM columns for the accumulator, the mbarriers, both A splits zero (the padded
  // columns k >= NN stay zero), both B splits from the host's layout, the stencil of B
  if (warp == 0) tc::tmem_alloc(tslot, S::NCOL);
  if (tid == 0) {
    tc::mbar_init(mbar, 1);
    tc::mbar_init(idle, 1);
    *abort_flag = 0;
  }
  for (int i = tid; i < 2 * S::AOPS; i += blockDim.x) aop[i] = 0.0f;
  for (int i = tid; i < 2 * S::BOPS; i += blockDim.x) bop[i] = p.binv_tc[i];
  for (int i = tid; i < 3 * NP * NP; i += blockDim.x) {
    kt[i] = p.c.kt[i / (NP * NP)][i % (NP * NP)];
    ktf[2 * i] = p.c.kt_f[i / (NP * NP)][i % (NP * NP)][0];
    ktf[2 * i + 1] = p.c.kt_f[i / (NP * NP)][i % (NP * NP)][1];
  }
  for (int j = tid; j <= g.ncol; j += blockDim.x) {
    const int tc_ = wrap_cell(X0 - g.wx + j - 1, p.ncx);
    colx[j] = (long long)(g.sx > 0 ? tc_ * NP : (p.ncx - 1 - tc_) * NP + (NP - 1)) * g.sa;
  }
  for (int r = tid; r <= g.nrow; r += blockDim.x) {
    const int tr = wrap_cell(Y0 - g.wy + r - 1, p.ncy);
    rowy[r] = (long long)(g.sy > 0 ? tr * NP : (p.ncy - 1 - tr) * NP + (NP - 1)) * g.sb;
  }
  for (int k = tid; k <= g.nlay; k += blockDim.x) {
    const int tl = wrap_cell(Z0 - g.wz + k - 1, p.ncz);
    layz[k] = (long long)(g.sz > 0 ? tl * NP : (p.ncz - 1 - tl) * NP + (NP - 1)) * g.sc;
  }
  g.colx = colx;
  g.rowy = rowy;
  g.layz = layz;
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  for (int i = tid; i < g.nrow * g.ncol * NF; i += blockDim.x) {
    const int cell = i / NF, u = i % NF;
    const int r = cell / g.ncol, j = cell % g.ncol;
    g.zt[i] = g.bz ? g.fbz[corner_px<NP>(g, j, u % NP) * g.fls[2][0] + corner_py<NP>(g, r, u / NP) * g.fls[2][1]]
                   : g.fin[corner_off(g, j, r, -1, NP - 1, u / NP, u % NP)];
  }
  __syncthreads();
  const double rth = C.rtheta, c1 = C.c1, th = C.theta, kx = C.kx, ky = C.ky, kz = C.kz;

  // step s (all groups) uses parity s & 1; the first step stages layer 0's anti-diagonal 0
  corner_stage<NP>(g, 0, 0, FB(0, 0), LB(0, 0), BB(0, 0));
  cp_async_wait_all();
  __syncthreads();

  // one thread issues the three split products of a solve (then commits them to the
  // mbarrier), and later waits for them
  uint32_t phase = 0;
  auto mma_issue = [&]() {   // tid 0 only
    tc::fence_after_sync();
#pragma unroll 1
    for (int sp = 0; sp < 3; ++sp) {
      const int sa = sp == 1 ? 1 : 0, sb = sp == 2 ? 1 : 0;   // (hi, hi), (lo, hi), (hi, lo)
#pragma unroll 1
      for (int ks = 0; ks < KP / 8; ++ks) {
        const uint64_t ad = tc::smem_desc(tc::smem_u32(aop + sa * S::AOPS) + ks * 2 * 16 * 128, 16 * 128, 128);
        const uint64_t bd =
            tc::smem_desc(tc::smem_u32(bop + sb * S::BOPS) + ks * 2 * (NPAD / 8) * 128, (NPAD / 8) * 128, 128);
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
  const int trow = 32 * lq + lane;                // this thread's TMEM row (cell)
  const uint32_t taddr = tmem + ((uint32_t)(32 * lq) << 16) + (uint32_t)(cc * CW);
  bool aborted = false;

  // Layers k0 .. k0 + nl - 1 are swept together: at group step tau, layer k0 + ls handles
  // its anti-diagonal tau - ls.  A layer's +z faces come from the layer below: for the first
  // layer of a group that layer finished in an earlier group and the faces are staged with
  // the state; for the others it wrote them one step before, after that step's staging, so
  // they are read from the scratch directly.  Rows of the products: the cells of layer k0's
  // anti-diagonal, then those of layer k0 + 1.
  int s = 0;
  for (int k0 = 0; k0 < g.nlay && !aborted; k0 += LAYERS) {
    const int nl = min(LAYERS, g.nlay - k0);
    const int tsteps = T_steps + nl - 1;
    for (int tau = 0; tau < tsteps; ++tau, ++s) {
      const int par = s & 1, prv = par ^ 1;
      int jlo[LAYERS], jhi[LAYERS], Acnt[LAYERS], roff[LAYERS];
      int Atot = 0;
#pragma unroll
      for (int ls = 0; ls < LAYERS; ++ls) {
        const int tt = tau - ls;
        const bool on = ls < nl && tt >= 0 && tt < T_steps;
        jlo[ls] = on ? max(0, tt - g.nrow + 1) : 0;
        jhi[ls] = on ? min(g.ncol - 1, tt) : -1;
        Acnt[ls] = on ? jhi[ls] - jlo[ls] + 1 : 0;
        roff[ls] = Atot;
        Atot += Acnt[ls];
      }
      // row c of the products -> (layer slot, cell index in its anti-diagonal)
      auto row_slot = [&](int c) { return (LAYERS > 1 && c >= Acnt[0]) ? 1 : 0; };
      // (A) r_c of every cell, kept in FP64 and split into the operand
      for (int i = tid; i < Atot * NN; i += blockDim.x) {
        const int c = i / NN, q = i % NN;
        const int ls = row_slot(c), cl = c - roff[ls], tt = tau - ls;
        const int j = jlo[ls] + cl, r = tt - j;
        const int iz = q / NF, iy = (q / NP) % NP, ix = q % NP;
        const double* fc = FB(par, ls);
        double rv = fc[cl * RS + q] * rth;
        if (ix == 0)
          rv = fma(kx, j == 0 ? LB(ls, par)[iz * NP + iy] : LT(ls, prv)[(size_t)j * NF + iz * NP + iy], rv);
        if (iy == 0)
          rv = fma(ky, r == 0 ? BB(ls, par)[iz * NP + ix] : BT(ls, prv)[(size_t)j * NF + iz * NP + ix], rv);
        if (iz == 0) {
          const double zf = ls == 0 ? fc[cl * RS + NN + iy * NP + ix]
                                    : g.zt[((long long)r * g.ncol + j) * NF + iy * NP + ix];
          rv = fma(kz, zf, rv);
        }
        rbuf[((size_t)ls * amax + cl) * NN + q] = rv;
        float hi, lo;
        tc::split_f64_bits<11>(rv, &hi, &lo);
        const int idx = tc::op_index(c, q, 128);
        aop[idx] = hi;
        aop[S::AOPS + idx] = lo;
      }
      tc::fence_proxy_async_smem();
      __syncthreads();
      if (tid == 0) mma_issue();
      {   // stage the next step: each layer's next anti-diagonal, or the next group's first
#pragma unroll
        for (int ls = 0; ls < LAYERS; ++ls) {
          const int tn = tau + 1 - ls;
          if (ls < nl && tn >= 0 && tn < T_steps)
            corner_stage<NP>(g, k0 + ls, tn, FB(prv, ls), LB(ls, prv), BB(ls, prv), ls == 0);
        }
        if (tau + 1 == tsteps && k0 + LAYERS < g.nlay) corner_stage<NP>(g, k0 + LAYERS, 0, FB(prv, 0), LB(0, prv), BB(0, prv));
      }
      if (tid == 0) mma_wait();
      __syncthreads();
      if (*abort_flag) {
        aborted = true;
        break;
      }
      // (L1) x~ from TMEM (rows = cells, this warp's block of node columns)
      tc::fence_after_sync();
      float xr[CW];
      tc::tmem_ld<CW>(taddr, xr);
      if (trow < Atot) {
        const int ls = row_slot(trow), cl = trow - roff[ls];
#pragma unroll
        for (int e = 0; e < CW; ++e)
          if (cc * CW + e < NN) xt[((size_t)ls * amax + cl) * NN + cc * CW + e] = xr[e];
      }
      tc::fence_before_sync();
      __syncthreads();
      // (R) residual r - B x~ of every node, split into the operand
      for (int i = tid; i < Atot * NN; i += blockDim.x) {
        const int c = i / NN, q = i % NN;
        const int ls = row_slot(c), cl = c - roff[ls];
        const int qz = q / NF, qy = (q / NP) % NP, qx = q % NP;
        const int idx = tc::op_index(c, q, 128);
        const size_t cr = ((size_t)ls * amax + cl) * NN;
        if constexpr (RES == 0) {
          const double res = tc_residual<NP>(rbuf[cr + q], xt + cr, kt, qz, qy, qx);
          float hi, lo;
          tc::split_f64_bits<11>(res, &hi, &lo);
          aop[idx] = hi;
          aop[S::AOPS + idx] = lo;
        } else {
          const dd res = tc_residual_dd<NP>(rbuf[cr + q], xt + cr, ktf, qz, qy, qx);
          const float hi = tc::tf32_rna(res.hi);
          aop[idx] = hi;
          aop[S::AOPS + idx] = tc::tf32_rna(__fadd_rn(__fsub_rn(res.hi, hi), res.lo));
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
      // (L2) x = x~ + d; outputs (cells of the box) and the faces passed downwind
      tc::fence_after_sync();
      float dv[CW];
      tc::tmem_ld<CW>(taddr, dv);
      if (trow < Atot) {
        const int ls = row_slot(trow), cl = trow - roff[ls], tt = tau - ls, k = k0 + ls;
        const int j = jlo[ls] + cl, r = tt - j;
        const bool out_layer = k >= g.wz;
        int h1 = jhi[ls] + 1, h2 = jhi[ls];
        if (out_layer) {
          h1 = max(jlo[ls], min(g.wx, jhi[ls] + 1));
          h2 = max(h1 - 1, min(jhi[ls], tt - g.wy));
        }
        const bool out_cell = j >= h1 && j <= h2;
        const double* fc = FB(par, ls);
        double* lt = LT(ls, par);
        double* bt = BT(ls, par);
#pragma unroll
        for (int e = 0; e < CW; ++e) {
          const int q = cc * CW + e;
          if (q < NN) {
            const double x = tc::f64_from_f32_bits(xr[e]) + tc::f64_from_f32_bits(dv[e]);
            const int qz = q / NF, qy = (q / NP) % NP, qx = q % NP;
            if (out_cell) st(g.fout + corner_off(g, j, r, k, qz, qy, qx), x - c1 * fc[cl * RS + q]);
            if (qx == NP - 1 || qy == NP - 1 || qz == NP - 1) {
              const double face = th * x;
              if (qx == NP - 1) lt[(size_t)(j + 1) * NF + qz * NP + qy] = face;
              if (qy == NP - 1) bt[(size_t)j * NF + qz * NP + qx] = face;
              if (qz == NP - 1) st(g.zt + ((long long)r * g.ncol + j) * NF + qy * NP + qx, face);
            }
          }
        }
      }
      cp_async_wait_all();
      tc::fence_before_sync();
      __syncthreads();
    }
  }
  if (aborted && tid == 0) tc::mbar_wait_bounded(mbar, (phase - 1) & 1, 2000000000LL);   // MMAs in flight
  cp_async_wait_all();
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, S::NCOL);
  }
}

template <int NP, int RES, int LAYERS>
__global__ void __launch_bounds__(512, 1) corner_tc_kernel(const __grid_constant__ PdgCornerPass p) {
  extern __shared__ __align__(128) unsigned char tc_smem[];
  corner_tc_body<NP, RES, LAYERS>(p, tc_smem);
}

}  // namespace pdgdev
