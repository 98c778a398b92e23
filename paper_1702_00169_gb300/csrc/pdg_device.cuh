// Device code shared by the single-instance kernels (pdg_kernels*.cu) and the
// batched persistent kernels (pdg_batch*.cu): collision of eq. (3.12), the two-phase
// exact periodic transport sweep of eq. (3.11), and the pass body.
//
// Everything is templated on the number type T of the state and of the arithmetic:
//   T = double : FP64 storage and FP64 arithmetic;
//   T = dd     : double-float numbers (an unevaluated sum hi + lo of two FP32 values,
//                about 48 significant bits) stored as a float pair in the same 8 bytes,
//                with arithmetic built from error-free transformations on the FP32
//                pipes (GB300 executes FP32 FMAs at 61x its FP64 rate).
#pragma once
#include <cuda_runtime.h>

#include "pdg_internal.h"
#include "../../include/pdg.h"

namespace pdgdev {

#ifndef PDG_PREFETCH_DIST
#define PDG_PREFETCH_DIST 2   // cells ahead prefetched into L2 on strided sweeps
#endif

enum { MV_ADV = 0, MV_SW = 1, MV_EU1 = 2, MV_EU2 = 3, MV_EU3 = 4, MV_NONE = 5, MV_D2Q9 = 6, MV_D3Q19 = 7,
       MV_D3Q15 = 8, MV_D3Q27 = 9 };

// ---------------------------------------------------------------------------
// Double-float arithmetic.  Error-free transformations (all with explicit
// round-to-nearest intrinsics so that no FMA contraction can alter them):
//   two_sum  (Knuth):  a + b = s + e exactly;
//   fast_two_sum (Dekker, |a| >= |b|): a + b = s + e exactly;
//   two_prod (with FMA): a * b = p + e exactly.
// Double-word operations follow Joldes, Muller & Popescu, "Tight and rigorous error
// bounds for basic building blocks of double-word arithmetic", ACM TOMS 44 (2017):
//   add = SloppyDWPlusDW (Dekker) below, AccurateDWPlusDW (relative error
//         <= 3u^2 + 13u^3) where cancellation must not cost relative accuracy,
//   mul = DWTimesDW with FMA (relative error <= 5u^2), u = 2^-24.
struct __align__(8) dd {
  float hi, lo;
};

__device__ __forceinline__ dd dd_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ dd dd_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dd dd_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
// Addition: Dekker's double-word sum (SloppyDWPlusDW, 11 operations).  Its error is
// bounded by about 2u^2 (|x| + |y|): relative to the operands rather than to the sum,
// which on this scheme's O(1) populations is an absolute error of ~1e-15; the
// accurate variant (AccurateDWPlusDW, 20 operations) is kept for the recurrences.
__device__ __forceinline__ dd operator+(dd x, dd y) {
  const dd s = dd_two_sum(x.hi, y.hi);
  const float v = __fadd_rn(x.lo, y.lo);
  return dd_fast_two_sum(s.hi, __fadd_rn(s.lo, v));
}
__device__ __forceinline__ dd dd_add_accurate(dd x, dd y) {
  const dd s = dd_two_sum(x.hi, y.hi);
  const dd t = dd_two_sum(x.lo, y.lo);
  const dd v = dd_fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return dd_fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}
__device__ __forceinline__ dd operator-(dd x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ dd operator-(dd x, dd y) { return x + (-y); }
__device__ __forceinline__ dd operator*(dd x, dd y) {
  const dd c = dd_two_prod(x.hi, y.hi);
  const float tl = __fmul_rn(x.lo, y.lo);
  const float cl = __fmaf_rn(x.lo, y.hi, __fmaf_rn(x.hi, y.lo, tl));
  return dd_fast_two_sum(c.hi, __fadd_rn(c.lo, cl));
}
__device__ __forceinline__ dd fma(dd a, dd b, dd c) { return a * b + c; }
// keep the FP64 fma visible next to the double-float overload
__device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
// 1/x: FP32 reciprocal seed refined by one Newton step in double-word arithmetic.
__device__ __forceinline__ dd recip(dd x) {
  const float r0 = __frcp_rn(x.hi);
  const dd one = {1.0f, 0.0f};
  const dd e = one - x * dd{r0, 0.0f};          // ~2^-23
  return dd{r0, 0.0f} + dd{r0, 0.0f} * e;
}
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// (1 - omega) f + omega f^eq for the double-float state: with omega = 2 the factor
// 1 - omega = -1 is exact and the product is a sign flip.
__device__ __forceinline__ dd relax(dd om1, dd v, dd e) {
  if (om1.hi == -1.0f && om1.lo == 0.0f) return e - v;
  return om1 * v + e;
}

template <class T> __device__ __forceinline__ T zero();
template <> __device__ __forceinline__ double zero<double>() { return 0.0; }
template <> __device__ __forceinline__ dd zero<dd>() { return {0.0f, 0.0f}; }

// loads / stores of the state (the same 8-byte slots in both modes)
template <class T> __device__ __forceinline__ T ld(const double* p);
template <> __device__ __forceinline__ double ld<double>(const double* p) { return *p; }
template <> __device__ __forceinline__ dd ld<dd>(const double* p) {
  const float2 v = *reinterpret_cast<const float2*>(p);
  return {v.x, v.y};
}
__device__ __forceinline__ void st(double* p, double v) { *p = v; }
__device__ __forceinline__ void st(double* p, dd v) { *reinterpret_cast<float2*>(p) = make_float2(v.hi, v.lo); }

// FP64 <-> double-float conversion (only at the API boundary)
__device__ __forceinline__ dd dd_from_double(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double dd_to_double(dd x) { return (double)x.hi + (double)x.lo; }
__device__ __forceinline__ double to_double(double x) { return x; }
__device__ __forceinline__ double to_double(dd x) { return dd_to_double(x); }
template <class T> __device__ __forceinline__ T from_double(double x);
template <> __device__ __forceinline__ double from_double<double>(double x) { return x; }
template <> __device__ __forceinline__ dd from_double<dd>(double x) { return dd_from_double(x); }

// coefficient accessors: value i of a (double array, float-pair array) couple
template <class T> __device__ __forceinline__ T cval(const double* d, const float (*f)[2], int i);
template <> __device__ __forceinline__ double cval<double>(const double* d, const float (*)[2], int i) {
  return d[i];
}
template <> __device__ __forceinline__ dd cval<dd>(const double*, const float (*f)[2], int i) {
  return {f[i][0], f[i][1]};
}
#define PDG_C(T, C, name, i) cval<T>((C).name, (C).name##_f, (i))
#define PDG_S(T, C, name) cval<T>(&(C).name, (C).name##_f, 0)
#define PDG_K(T, M, i) cval<T>((M).k, (M).k_f, (i))

// Dot product acc + sum_j a_j b_j.  FP64: an FMA chain.  Double-float: compensated
// accumulation in the spirit of Ogita, Rump & Oishi ("Accurate sum and dot product",
// SIAM J. Sci. Comput. 2005): exact products of the high parts (two_prod), the
// high sum kept exactly with two_sum, every rounding error and the cross terms
// a.hi b.lo + a.lo b.hi collected in one FP32 accumulator, then renormalised.
template <int K>
__device__ __forceinline__ double dot_acc(const double* a, const double* b, double acc) {
#pragma unroll
  for (int j = 0; j < K; ++j) acc = fma(a[j], b[j], acc);
  return acc;
}
template <int K>
__device__ __forceinline__ dd dot_acc(const dd* a, const dd* b, dd acc) {
  float S = acc.hi, L = acc.lo;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const dd p = dd_two_prod(a[j].hi, b[j].hi);
    const float cross = __fmaf_rn(a[j].hi, b[j].lo, __fmul_rn(a[j].lo, b[j].hi));
    const dd s = dd_two_sum(S, p.hi);
    S = s.hi;
    L = __fadd_rn(L, __fadd_rn(s.lo, __fadd_rn(p.lo, cross)));
  }
  return dd_fast_two_sum(S, L);
}

// ---------------------------------------------------------------------------
// Collision at one point (eq. (3.12)); v holds the m * 2D populations.
// f^eq_{k,i} = w_k/(2D) + (v_i . q_k(w))/(2 lambda^2) = w_k/(2D) + s_i q^a_k / (2 lambda)
// for v_i = s_i lambda e_a.  Model constants (index PDG_K_*) come precomputed from
// the host in FP64 and as float pairs.
template <int MV, class T>
__device__ __forceinline__ void collide(T* v, const PdgModel& M);

template <int MV, class T>
struct Collide;

template <class T>
struct Collide<MV_ADV, T> {
  static __device__ __forceinline__ void run(T* v, const PdgModel& M) {
    const int nv = M.nv;
    T w = zero<T>();
#pragma unroll
    for (int i = 0; i < 6; ++i)
      if (i < nv) w = w + v[i];
    const T om1 = PDG_K(T, M, PDG_K_OM1);
#pragma unroll
    for (int i = 0; i < 6; ++i)
      if (i < nv) v[i] = fma(PDG_K(T, M, PDG_K_CADV + i), w, om1 * v[i]);
  }
};

template <class T>
struct Collide<MV_SW, T> {
  static __device__ __forceinline__ void run(T* v, const PdgModel& M) {
    // w = (h, hu, hv), populations k*4 + {+x, -x, +y, -y}
    T w[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) w[k] = (v[4 * k] + v[4 * k + 1]) + (v[4 * k + 2] + v[4 * k + 3]);
    const T h = w[0], hu = w[1], hv = w[2];
    const T ih = recip(h);
    const T u = hu * ih, vv = hv * ih;
    const T p = (PDG_K(T, M, PDG_K_HALFG) * h) * h;
    const T qx[3] = {hu, fma(hu, u, p), hv * u};
    const T qy[3] = {hv, hu * vv, fma(hv, vv, p)};
    const T om1 = PDG_K(T, M, PDG_K_OM1);
    const T c0 = PDG_K(T, M, PDG_K_C0);   // omega / (2D)
    const T c1 = PDG_K(T, M, PDG_K_C1);   // omega / (2 lambda)
    const T mc1 = -c1;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const T b = c0 * w[k];
      if constexpr (sizeof(T) == sizeof(dd) && !__is_same(T, double)) {
        // double-float: b +- c1 q shared by the two opposite populations
        const T tx = c1 * qx[k], ty = c1 * qy[k];
        v[4 * k + 0] = relax(om1, v[4 * k + 0], b + tx);
        v[4 * k + 1] = relax(om1, v[4 * k + 1], b - tx);
        v[4 * k + 2] = relax(om1, v[4 * k + 2], b + ty);
        v[4 * k + 3] = relax(om1, v[4 * k + 3], b - ty);
      } else {
        v[4 * k + 0] = fma(om1, v[4 * k + 0], fma(c1, qx[k], b));
        v[4 * k + 1] = fma(om1, v[4 * k + 1], fma(mc1, qx[k], b));
        v[4 * k + 2] = fma(om1, v[4 * k + 2], fma(c1, qy[k], b));
        v[4 * k + 3] = fma(om1, v[4 * k + 3], fma(mc1, qy[k], b));
      }
    }
  }
};

template <int D, class T>
__device__ __forceinline__ void collide_euler(T* v, const PdgModel& M) {
  constexpr int m = D + 2, nv = 2 * D;
  T w[m];
#pragma unroll
  for (int k = 0; k < m; ++k) {
    T s = zero<T>();
#pragma unroll
    for (int i = 0; i < nv; ++i) s = s + v[k * nv + i];
    w[k] = s;
  }
  const T rho = w[0], E = w[D + 1];
  const T ir = recip(rho);
  T u[D];
  T ke = zero<T>();
#pragma unroll
  for (int b = 0; b < D; ++b) {
    u[b] = w[1 + b] * ir;
    ke = fma(w[1 + b], u[b], ke);
  }
  const T p = PDG_K(T, M, PDG_K_GM1) * (E - PDG_K(T, M, PDG_K_HALF) * ke);
  const T om1 = PDG_K(T, M, PDG_K_OM1);
  const T c0 = PDG_K(T, M, PDG_K_C0);
  const T c1 = PDG_K(T, M, PDG_K_C1);
  const T mc1 = -c1;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    T q[m];
    q[0] = w[1 + a];
#pragma unroll
    for (int b = 0; b < D; ++b) q[1 + b] = (a == b) ? fma(w[1 + b], u[a], p) : w[1 + b] * u[a];
    q[D + 1] = (E + p) * u[a];
#pragma unroll
    for (int k = 0; k < m; ++k) {
      const T bse = c0 * w[k];
      if constexpr (!__is_same(T, double)) {
        const T t = c1 * q[k];
        v[k * nv + 2 * a] = relax(om1, v[k * nv + 2 * a], bse + t);
        v[k * nv + 2 * a + 1] = relax(om1, v[k * nv + 2 * a + 1], bse - t);
      } else {
        v[k * nv + 2 * a] = fma(om1, v[k * nv + 2 * a], fma(c1, q[k], bse));
        v[k * nv + 2 * a + 1] = fma(om1, v[k * nv + 2 * a + 1], fma(mc1, q[k], bse));
      }
    }
  }
}

template <class T>
struct Collide<MV_EU1, T> {
  static __device__ __forceinline__ void run(T* v, const PdgModel& M) { collide_euler<1, T>(v, M); }
};
template <class T>
struct Collide<MV_EU2, T> {
  static __device__ __forceinline__ void run(T* v, const PdgModel& M) { collide_euler<2, T>(v, M); }
};
template <class T>
struct Collide<MV_EU3, T> {
  static __device__ __forceinline__ void run(T* v, const PdgModel& M) { collide_euler<3, T>(v, M); }
};
// D2Q9 (Section 5.1): with j = sum_i f_i xi_i (lattice units, v_i = lambda xi_i) and
// s = 3 j / rho = u . xi / c^2 per unit xi, the equilibrium is
// f^eq_i = W_i rho e_i, e_i = 1 + s.xi_i + (s.xi_i)^2 / 2 - |s|^2 / 6.  v holds the nine
// populations in the velocity order of Section 5.1; M carries omega W_i (omega = 1 gives
// f^eq itself when 1 - omega = 0).
template <class T>
__device__ __forceinline__ void d2q9_relax(T* v, T rho, T jx, T jy, const PdgModel& M) {
  const T three = from_double<T>(3.0);
  const T ir = recip(rho);
  const T sx = three * (jx * ir), sy = three * (jy * ir);
  const T half = PDG_K(T, M, PDG_K_HALF);
  const T base = from_double<T>(1.0) - PDG_K(T, M, PDG_K_SIXTH) * fma(sx, sx, sy * sy);
  const T a0 = PDG_K(T, M, PDG_K_Q9W0) * rho, a1 = PDG_K(T, M, PDG_K_Q9W1) * rho;
  const T a2 = PDG_K(T, M, PDG_K_Q9W2) * rho;
  const T om1 = PDG_K(T, M, PDG_K_OM1);
  const T sp = sx + sy, sm = sy - sx;
  // e(+t) = base + t + t^2/2, e(-t) = base - t + t^2/2
  const T bx = fma(half * sx, sx, base), by = fma(half * sy, sy, base);
  const T bp = fma(half * sp, sp, base), bm = fma(half * sm, sm, base);
  const T e[9] = {base, bx + sx, by + sy, bx - sx, by - sy, bp + sp, bm + sm, bp - sp, bm - sm};
  if constexpr (!__is_same(T, double)) {
    v[0] = relax(om1, v[0], a0 * e[0]);
#pragma unroll
    for (int i = 1; i < 5; ++i) v[i] = relax(om1, v[i], a1 * e[i]);
#pragma unroll
    for (int i = 5; i < 9; ++i) v[i] = relax(om1, v[i], a2 * e[i]);
  } else if (M.omega == 2.0) {
    // omega = 2: (1 - omega) f + omega f^eq = W_i rho e_i (times 2) - f, one FMA
    v[0] = fma(a0, e[0], -v[0]);
#pragma unroll
    for (int i = 1; i < 5; ++i) v[i] = fma(a1, e[i], -v[i]);
#pragma unroll
    for (int i = 5; i < 9; ++i) v[i] = fma(a2, e[i], -v[i]);
  } else {
    v[0] = fma(om1, v[0], a0 * e[0]);
#pragma unroll
    for (int i = 1; i < 5; ++i) v[i] = fma(om1, v[i], a1 * e[i]);
#pragma unroll
    for (int i = 5; i < 9; ++i) v[i] = fma(om1, v[i], a2 * e[i]);
  }
}

// D2Q9 equilibrium f^eq_i(rho, j) = W_i rho e_i (unscaled weights), j in lattice units.
template <class T>
__device__ __forceinline__ void d2q9_feq(T rho, T jx, T jy, const PdgModel& M, T* out) {
  const T three = from_double<T>(3.0);
  const T ir = recip(rho);
  const T sx = three * (jx * ir), sy = three * (jy * ir);
  const T half = PDG_K(T, M, PDG_K_HALF);
  const T base = from_double<T>(1.0) - PDG_K(T, M, PDG_K_SIXTH) * fma(sx, sx, sy * sy);
  const T sp = sx + sy, sm = sy - sx;
  const T bx = fma(half * sx, sx, base), by = fma(half * sy, sy, base);
  const T bp = fma(half * sp, sp, base), bm = fma(half * sm, sm, base);
  const T a0 = from_double<T>(4.0 / 9.0) * rho, a1 = from_double<T>(1.0 / 9.0) * rho;
  const T a2 = from_double<T>(1.0 / 36.0) * rho;
  out[0] = a0 * base;
  out[1] = a1 * (bx + sx);
  out[2] = a1 * (by + sy);
  out[3] = a1 * (bx - sx);
  out[4] = a1 * (by - sy);
  out[5] = a2 * (bp + sp);
  out[6] = a2 * (bm + sm);
  out[7] = a2 * (bp - sp);
  out[8] = a2 * (bm - sm);
}

// Source stages around the collision, S(delta) C S(delta) (pdg_set_source).  S is the theta
// step of d/dt w = s(w) for w = (rho, rho u), s = (0, rho g) - K (w - w_s), applied to the
// equilibrium part: f' = f + f^eq(w') - f^eq(w).  Its theta system is lower triangular:
// rho' first, then rho u' with the gravity term taken at both levels.  Composed:
//   w -> w1 -> w2 (C keeps w),  f_out = f^eq(w2) + (1 - omega) (f - f^eq(w)),
// since S keeps f - f^eq and C scales it by 1 - omega (f^eq(w1) cancels).
template <class T>
__device__ __forceinline__ void d2q9_source_collide(T* v, const PdgSrc& S, const PdgModel& M, long long off) {
  const T rho = (((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]))) + v[8];
  const T jx = (v[1] - v[3]) + ((v[5] - v[6]) + (v[8] - v[7]));
  const T jy = (v[2] - v[4]) + ((v[5] + v[6]) - (v[7] + v[8]));
  const T lam = PDG_K(T, M, PDG_K_LAM), ilam = PDG_K(T, M, PDG_K_ILAM);
  const T dl = PDG_S(T, S, delta), th = PDG_S(T, S, theta), omth = PDG_S(T, S, omtheta);
  const T K = (S.flags & PDG_SOURCE_PENALIZATION) ? from_double<T>(S.kfield[off]) : zero<T>();
  const T dK = dl * K;
  const T ia = recip(fma(th, dK, from_double<T>(1.0)));
  const T bb = from_double<T>(1.0) - omth * dK;
  const T gx = PDG_C(T, S, g, 0), gy = PDG_C(T, S, g, 1);
  const T kr = dK * PDG_C(T, S, ws, 0), kmx = dK * PDG_C(T, S, ws, 1), kmy = dK * PDG_C(T, S, ws, 2);
  // S(delta) twice
  const T rho1 = fma(bb, rho, kr) * ia;
  const T rg1 = dl * fma(omth, rho, th * rho1);
  const T mx1 = fma(bb, lam * jx, fma(rg1, gx, kmx)) * ia;
  const T my1 = fma(bb, lam * jy, fma(rg1, gy, kmy)) * ia;
  const T rho2 = fma(bb, rho1, kr) * ia;
  const T rg2 = dl * fma(omth, rho1, th * rho2);
  const T mx2 = fma(bb, mx1, fma(rg2, gx, kmx)) * ia;
  const T my2 = fma(bb, my1, fma(rg2, gy, kmy)) * ia;
  T e0[9], e2[9];
  d2q9_feq<T>(rho, jx, jy, M, e0);
  d2q9_feq<T>(rho2, mx2 * ilam, my2 * ilam, M, e2);
  const T om1 = PDG_K(T, M, PDG_K_OM1);
#pragma unroll
  for (int i = 0; i < 9; ++i) v[i] = fma(om1, v[i] - e0[i], e2[i]);
}

template <class T>
struct Collide<MV_D2Q9, T> {
  static __device__ __forceinline__ void run(T* v, const PdgModel& M) {
    const T rho = (((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]))) + v[8];
    const T jx = (v[1] - v[3]) + ((v[5] - v[6]) + (v[8] - v[7]));
    const T jy = (v[2] - v[4]) + ((v[5] + v[6]) - (v[7] + v[8]));
    d2q9_relax<T>(v, rho, jx, jy, M);
  }
};

// D3Q19 (order of PDG_Q19_*): f^eq_i = W_i rho e_i with the same e as D2Q9 per velocity,
// s = 3 j / rho.  Edge velocities of plane (a, b) in the order (+,+), (-,+), (-,-), (+,-)
// have s.xi = +-(s_a + s_b), +-(s_b - s_a).
template <class T>
__device__ __forceinline__ void d3q19_e(T rho, T jx, T jy, T jz, const PdgModel& M, T* e) {
  const T three = from_double<T>(3.0);
  const T ir = recip(rho);
  const T s[3] = {three * (jx * ir), three * (jy * ir), three * (jz * ir)};
  const T half = PDG_K(T, M, PDG_K_HALF);
  const T base = from_double<T>(1.0) - PDG_K(T, M, PDG_K_SIXTH) * fma(s[0], s[0], fma(s[1], s[1], s[2] * s[2]));
  e[0] = base;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const T q = fma(half * s[a], s[a], base);
    e[1 + 2 * a] = q + s[a];
    e[2 + 2 * a] = q - s[a];
  }
  const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
#pragma unroll
  for (int o = 0; o < 3; ++o) {
    const T t1 = s[pa[o]] + s[pb[o]], t2 = s[pb[o]] - s[pa[o]];
    const T q1 = fma(half * t1, t1, base), q2 = fma(half * t2, t2, base);
    e[7 + 4 * o] = q1 + t1;
    e[8 + 4 * o] = q2 + t2;
    e[9 + 4 * o] = q1 - t1;
    e[10 + 4 * o] = q2 - t2;
  }
}

template <class T>
__device__ __forceinline__ void d3q19_moments(const T* v, T* rho, T* jx, T* jy, T* jz) {
  *rho = ((((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]))) +
          (((v[8] + v[9]) + (v[10] + v[11])) + ((v[12] + v[13]) + (v[14] + v[15])))) + ((v[16] + v[17]) + v[18]);
  // x: axis 1 - 2; xy edges 7 - 8 - 9 + 10; xz edges 11 - 12 - 13 + 14
  *jx = (v[1] - v[2]) + ((v[7] - v[8]) + (v[10] - v[9])) + ((v[11] - v[12]) + (v[14] - v[13]));
  // y: axis 3 - 4; xy edges 7 + 8 - 9 - 10; yz edges 15 - 16 - 17 + 18
  *jy = (v[3] - v[4]) + ((v[7] + v[8]) - (v[9] + v[10])) + ((v[15] - v[16]) + (v[18] - v[17]));
  // z: axis 5 - 6; xz edges 11 + 12 - 13 - 14; yz edges 15 + 16 - 17 - 18
  *jz = (v[5] - v[6]) + ((v[11] + v[12]) - (v[13] + v[14])) + ((v[15] + v[16]) - (v[17] + v[18]));
}

// Corner velocities (D3Q15 / D3Q27) in the order (s_x, s_y, s_z) = (+,+,+), (-,+,+), (-,-,+),
// (+,-,+), (+,+,-), (-,+,-), (-,-,-), (+,-,-): sums of the eight populations c[0..7] (mass
// and the three first moments).  Their s.xi_i are +-t_1..t_4 (pairs (0,6), (1,7), (2,4),
// (3,5)), t_1 = s_x + s_y + s_z, t_2 = s_y + s_z - s_x, t_3 = s_z - s_x - s_y, t_4 = s_x + s_z - s_y.
template <class T>
__device__ __forceinline__ void corner_moments(const T* c, T* rho, T* jx, T* jy, T* jz) {
  *rho = ((c[0] + c[1]) + (c[2] + c[3])) + ((c[4] + c[5]) + (c[6] + c[7]));
  *jx = ((c[0] - c[1]) + (c[3] - c[2])) + ((c[4] - c[5]) + (c[7] - c[6]));
  *jy = ((c[0] + c[1]) - (c[2] + c[3])) + ((c[4] + c[5]) - (c[6] + c[7]));
  *jz = ((c[0] + c[1]) + (c[2] + c[3])) - ((c[4] + c[5]) + (c[6] + c[7]));
}

// 3-D lattice collision (D3Q19: EDGES; D3Q15: CORNERS; D3Q27: both).  Populations 0 (rest),
// 1-6 (axis), then the twelve edges (order of PDG_Q19_*), then the eight corners;
// f^eq_i = W_i rho e_i with s = 3 j / rho (see d3q19_e and corner_moments).  Each equilibrium
// factor is formed right where its population is relaxed, so that only the populations
// and a few scalars stay live (the pass kernels run at most 128 registers per thread).
template <class T, bool EDGES, bool CORNERS>
__device__ __forceinline__ void d3q_lattice_collide(T* v, const PdgModel& M) {
  constexpr int E0 = 7, C0 = EDGES ? 19 : 7;
  T rho = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + v[6]);
  T jx = v[1] - v[2], jy = v[3] - v[4], jz = v[5] - v[6];
  if constexpr (EDGES) {
    rho = rho + ((((v[E0] + v[E0 + 1]) + (v[E0 + 2] + v[E0 + 3])) + ((v[E0 + 4] + v[E0 + 5]) + (v[E0 + 6] + v[E0 + 7]))) +
                 ((v[E0 + 8] + v[E0 + 9]) + (v[E0 + 10] + v[E0 + 11])));
    // x: xy edges 0 - 1 - 2 + 3, xz edges 4 - 5 - 6 + 7; y: xy 0 + 1 - 2 - 3, yz 8 - 9 - 10 + 11;
    // z: xz 4 + 5 - 6 - 7, yz 8 + 9 - 10 - 11 (edge indices relative to population 7)
    jx = jx + (((v[E0] - v[E0 + 1]) + (v[E0 + 3] - v[E0 + 2])) + ((v[E0 + 4] - v[E0 + 5]) + (v[E0 + 7] - v[E0 + 6])));
    jy = jy + (((v[E0] + v[E0 + 1]) - (v[E0 + 2] + v[E0 + 3])) + ((v[E0 + 8] - v[E0 + 9]) + (v[E0 + 11] - v[E0 + 10])));
    jz = jz + (((v[E0 + 4] + v[E0 + 5]) - (v[E0 + 6] + v[E0 + 7])) + ((v[E0 + 8] + v[E0 + 9]) - (v[E0 + 10] + v[E0 + 11])));
  }
  if constexpr (CORNERS) {
    T cr, cx, cy, cz;
    corner_moments<T>(v + C0, &cr, &cx, &cy, &cz);
    rho = rho + cr;
    jx = jx + cx;
    jy = jy + cy;
    jz = jz + cz;
  }
  const T three = from_double<T>(3.0);
  const T ir = recip(rho);
  const T sx = three * (jx * ir), sy = three * (jy * ir), sz = three * (jz * ir);
  const T half = PDG_K(T, M, PDG_K_HALF);
  const T base = from_double<T>(1.0) - PDG_K(T, M, PDG_K_SIXTH) * fma(sx, sx, fma(sy, sy, sz * sz));
  const T om1 = PDG_K(T, M, PDG_K_OM1);
  const bool two = M.omega == 2.0;
  // v_i <- omega W_i rho e_i + (1 - omega) v_i  (a = omega W_i rho)
  auto upd = [&](int i, T a, T e) {
    if constexpr (!__is_same(T, double)) {
      v[i] = relax(om1, v[i], a * e);
    } else {
      v[i] = two ? fma(a, e, -v[i]) : fma(om1, v[i], a * e);
    }
  };
  // one velocity pair +-t: e = q +- t, q = base + t^2 / 2
  auto pair = [&](int ip, int im, T a, T t) {
    const T q = fma(half * t, t, base);
    upd(ip, a, q + t);
    upd(im, a, q - t);
  };
  upd(0, PDG_K(T, M, PDG_K_Q9W0) * rho, base);
  {
    const T a1 = PDG_K(T, M, PDG_K_Q9W1) * rho;
    pair(1, 2, a1, sx);
    pair(3, 4, a1, sy);
    pair(5, 6, a1, sz);
  }
  if constexpr (EDGES) {   // plane (a, b): (+,+) / (-,-) carry s_a + s_b, (-,+) / (+,-) carry s_b - s_a
    const T a2 = PDG_K(T, M, PDG_K_Q9W2) * rho;
    pair(E0 + 0, E0 + 2, a2, sx + sy);
    pair(E0 + 1, E0 + 3, a2, sy - sx);
    pair(E0 + 4, E0 + 6, a2, sx + sz);
    pair(E0 + 5, E0 + 7, a2, sz - sx);
    pair(E0 + 8, E0 + 10, a2, sy + sz);
    pair(E0 + 9, E0 + 11, a2, sz - sy);
  }
  if constexpr (CORNERS) {   // the corner order of corner_moments
    const T a3 = PDG_K(T, M, PDG_K_Q9W3) * rho;
    pair(C0 + 0, C0 + 6, a3, (sx + sy) + sz);
    pair(C0 + 1, C0 + 7, a3, (sy + sz) - sx);
    pair(C0 + 2, C0 + 4, a3, sz - (sx + sy));
    pair(C0 + 3, C0 + 5, a3, (sx + sz) - sy);
  }
}

template <class T>
struct Collide<MV_D3Q19, T> {
  static __device__ __forceinline__ void run(T* v, const PdgModel& M) { d3q_lattice_collide<T, true, false>(v, M); }
};

template <class T>
struct Collide<MV_D3Q15, T> {
  static __device__ __forceinline__ void run(T* v, const PdgModel& M) { d3q_lattice_collide<T, false, true>(v, M); }
};

template <class T>
struct Collide<MV_D3Q27, T> {
  static __device__ __forceinline__ void run(T* v, const PdgModel& M) { d3q_lattice_collide<T, true, true>(v, M); }
};

template <class T>
struct Collide<MV_NONE, T> {
  static __device__ __forceinline__ void run(T*, const PdgModel&) {}
};

template <int MV, class T>
__device__ __forceinline__ void collide(T* v, const PdgModel& M) {
  Collide<MV, T>::run(v, M);
}

template <int MV>
struct NFields { static constexpr int value = PDG_MAXF; };
template <> struct NFields<MV_SW> { static constexpr int value = 12; };
template <> struct NFields<MV_EU1> { static constexpr int value = 6; };
template <> struct NFields<MV_EU2> { static constexpr int value = 16; };
template <> struct NFields<MV_EU3> { static constexpr int value = 30; };
template <> struct NFields<MV_ADV> { static constexpr int value = 6; };
template <> struct NFields<MV_NONE> { static constexpr int value = 1; };
template <> struct NFields<MV_D2Q9> { static constexpr int value = 9; };
template <> struct NFields<MV_D3Q19> { static constexpr int value = 19; };
template <> struct NFields<MV_D3Q15> { static constexpr int value = 15; };
template <> struct NFields<MV_D3Q27> { static constexpr int value = 27; };

// State slot of population k at collision time (D2Q9: the diagonal populations 5-8 sit
// in slots dslot..dslot+3, see PDG_Q9_SLOTS).
template <int MV>
__device__ __forceinline__ int coll_slot(int k, int dslot) {
  if constexpr (MV == MV_D2Q9) return k < PDG_Q9_DIAG ? k : dslot + (k - PDG_Q9_DIAG);
  if constexpr (MV == MV_D3Q19) return k < PDG_Q19_DIAG ? k : dslot + (k - PDG_Q19_DIAG);
  if constexpr (MV == MV_D3Q15) return k < PDG_Q15_DIAG ? k : dslot + (k - PDG_Q15_DIAG);
  if constexpr (MV == MV_D3Q27) return k < PDG_Q27_DIAG ? k : dslot + (k - PDG_Q27_DIAG);
  return k;
}

// ---------------------------------------------------------------------------
// Transport phases for one population along one line.  lp points at traversal
// index 0 of the line, dstep is the signed stride between traversal indices.

// 16-byte vector access to two consecutive state slots (x-axis lines are contiguous).
__device__ __forceinline__ void ld2(const double* p, double* a, double* b) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  *a = v.x;
  *b = v.y;
}
__device__ __forceinline__ void ld2(const double* p, dd* a, dd* b) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  *a = dd{v.x, v.y};
  *b = dd{v.z, v.w};
}
__device__ __forceinline__ void st2(double* p, double a, double b) {
  *reinterpret_cast<double2*>(p) = make_double2(a, b);
}
__device__ __forceinline__ void st2(double* p, dd a, dd b) {
  *reinterpret_cast<float4*>(p) = make_float4(a.hi, a.lo, b.hi, b.lo);
}

// Cell c of a line: NP values in traversal order.  On unit-stride lines (dstep = +-1)
// with an even NP the cell is one 16-byte aligned block (lines start on 16-byte
// boundaries and every cell holds NP * 8 bytes): vector loads, reversed in registers
// for the backward direction.
template <int NP, class T>
__device__ __forceinline__ void load_cell(const double* lp, long long dstep, int c, T* v) {
  const double* p0 = lp + (long long)c * NP * dstep;
  if constexpr (NP % 2 == 0) {
    if (dstep == 1) {
#pragma unroll
      for (int j = 0; j < NP; j += 2) ld2(p0 + j, &v[j], &v[j + 1]);
      return;
    }
    if (dstep == -1) {
      const double* b = p0 - (NP - 1);
#pragma unroll
      for (int j = 0; j < NP; j += 2) ld2(b + j, &v[NP - 1 - j], &v[NP - 2 - j]);
      return;
    }
  }
#pragma unroll
  for (int j = 0; j < NP; ++j) v[j] = ld<T>(p0 + j * dstep);
}

template <int NP, class T>
__device__ __forceinline__ void store_cell(double* lp, long long dstep, int c, const T* v) {
  double* p0 = lp + (long long)c * NP * dstep;
  if constexpr (NP % 2 == 0) {
    if (dstep == 1) {
#pragma unroll
      for (int j = 0; j < NP; j += 2) st2(p0 + j, v[j], v[j + 1]);
      return;
    }
    if (dstep == -1) {
      double* b = p0 - (NP - 1);
#pragma unroll
      for (int j = 0; j < NP; j += 2) st2(b + j, v[NP - 1 - j], v[NP - 2 - j]);
      return;
    }
  }
#pragma unroll
  for (int j = 0; j < NP; ++j) st(p0 + j * dstep, v[j]);
}

// L2 prefetch of the NP values of cell c (strided lines: no register is spent on it).
template <int NP>
__device__ __forceinline__ void prefetch_cell(const double* lp, long long dstep, int c) {
  const double* p0 = lp + (long long)c * NP * dstep;
#pragma unroll
  for (int j = 0; j < NP; ++j) asm volatile("prefetch.global.L2 [%0];" ::"l"(p0 + j * dstep));
}

template <int NP, class T>
__device__ __forceinline__ void load_row(const PdgCoef& C, int r, T* row) {
#pragma unroll
  for (int j = 0; j < NP; ++j) row[j] = PDG_C(T, C, E, r * NP + j);
}

// Phase 1: aggregate Y of the recurrence over cells [wstart, c1) starting from 0,
// and the old last-node value of cell c1 - 1.
template <int NP, class T>
__device__ __forceinline__ void phase_aggregate(const double* lp, long long dstep, int N, int wstart, int c1,
                                                const PdgCoef& C, T* Y, T* U, const T* inflow) {
  int cp = wstart - 1;
  if (cp < 0) cp += N;
  T u = (wstart == 0 && inflow) ? *inflow : ld<T>(lp + ((long long)cp * NP + (NP - 1)) * dstep);
  T y = zero<T>();
  const T qz = PDG_C(T, C, q, NP - 1) * PDG_S(T, C, zb);
  const T beta = PDG_S(T, C, beta);
  T row[NP];
  load_row<NP, T>(C, NP - 1, row);
  for (int c = wstart; c < c1; ++c) {
    T v[NP];
    load_cell<NP, T>(lp, dstep, c, v);
    const T alpha = dot_acc<NP>(row, v, qz * u);
    y = fma(beta, y, alpha);
    u = v[NP - 1];
  }
  *Y = y;
  *U = u;
}

// Phase 2: sweep cells [c0, c1) with inflow (x, u) and write the new values in place.
// On unit-stride lines the next cell is loaded before the current one is stored (they
// never alias), so its memory latency overlaps the arithmetic; strided lines are
// coalesced across the warp and keep the lighter loop.
template <int NP, class T>
__device__ __forceinline__ void phase_sweep(double* lp, long long dstep, int c0, int c1, T x, T u,
                                            const PdgCoef& C) {
  const T za = PDG_S(T, C, za), zb = PDG_S(T, C, zb);
  if (dstep == 1 || dstep == -1) {
    T v[NP];
    if (c0 < c1) load_cell<NP, T>(lp, dstep, c0, v);
    for (int c = c0; c < c1; ++c) {
      T vn[NP];
      if (c + 1 < c1) load_cell<NP, T>(lp, dstep, c + 1, vn);
      const T z = fma(za, x, zb * u);
      T out[NP];
#pragma unroll
      for (int r = 0; r < NP; ++r) {
        T row[NP];
        load_row<NP, T>(C, r, row);
        out[r] = dot_acc<NP>(row, v, PDG_C(T, C, q, r) * z);
      }
      store_cell<NP, T>(lp, dstep, c, out);
      x = out[NP - 1];
      u = v[NP - 1];
#pragma unroll
      for (int j = 0; j < NP; ++j) v[j] = vn[j];
    }
    return;
  }
  for (int c = c0; c < c1; ++c) {
    if (c + PDG_PREFETCH_DIST < c1) prefetch_cell<NP>(lp, dstep, c + PDG_PREFETCH_DIST);
    T v[NP];
    load_cell<NP, T>(lp, dstep, c, v);
    const T z = fma(za, x, zb * u);
    double* p0 = lp + (long long)c * NP * dstep;
    T last = zero<T>();
#pragma unroll
    for (int r = 0; r < NP; ++r) {
      T row[NP];
      load_row<NP, T>(C, r, row);
      const T acc = dot_acc<NP>(row, v, PDG_C(T, C, q, r) * z);
      st(p0 + r * dstep, acc);
      if (r == NP - 1) last = acc;
    }
    x = last;
    u = v[NP - 1];
  }
}

// Reverse mode (|beta| > 1): x_{c-1} = gamma (x_c - alpha_c).
// Phase 1: y = x_{c0-1} from the first cells [c0, cend) of the segment, given the
// old last-node value u0 of cell c0 - 1.
template <int NP, class T>
__device__ __forceinline__ void phase_aggregate_rev(const double* lp, long long dstep, int c0, int cend, T u0,
                                                    const PdgCoef& C, T* Y) {
  T y = zero<T>();
  const T qz = PDG_C(T, C, q, NP - 1) * PDG_S(T, C, zb);
  const T gamma = PDG_S(T, C, gamma);
  T row[NP];
  load_row<NP, T>(C, NP - 1, row);
  for (int c = cend - 1; c >= c0; --c) {
    T v[NP];
    load_cell<NP, T>(lp, dstep, c, v);
    const T u = (c > c0) ? ld<T>(lp + ((long long)(c - 1) * NP + (NP - 1)) * dstep) : u0;
    const T alpha = dot_acc<NP>(row, v, qz * u);
    y = gamma * (y - alpha);
  }
  *Y = y;
}

// Phase 2 (reverse): sweep cells c1-1 down to c0 from x = x_{c1-1}; u0 = old value of
// the last node of cell c0 - 1 (saved before any write).
template <int NP, class T>
__device__ __forceinline__ void phase_sweep_rev(double* lp, long long dstep, int c0, int c1, T x, T u0,
                                                const PdgCoef& C) {
  const T qz = PDG_C(T, C, q, NP - 1) * PDG_S(T, C, zb);
  const T gamma = PDG_S(T, C, gamma);
  const T za = PDG_S(T, C, za), zb = PDG_S(T, C, zb);
  for (int c = c1 - 1; c >= c0; --c) {
    T v[NP];
    load_cell<NP, T>(lp, dstep, c, v);
    const T u = (c > c0) ? ld<T>(lp + ((long long)(c - 1) * NP + (NP - 1)) * dstep) : u0;
    T rowl[NP];
    load_row<NP, T>(C, NP - 1, rowl);
    const T alpha = dot_acc<NP>(rowl, v, qz * u);
    const T xm = gamma * (x - alpha);
    const T z = fma(za, xm, zb * u);
    double* p0 = lp + (long long)c * NP * dstep;
#pragma unroll
    for (int r = 0; r < NP; ++r) {
      T row[NP];
      load_row<NP, T>(C, r, row);
      st(p0 + r * dstep, dot_acc<NP>(row, v, PDG_C(T, C, q, r) * z));
    }
    x = xm;
  }
}

// Composed double sub-step T T (forward recurrence, window mode; see PdgCoef):
// phase 1 aggregates the pair recurrence X_c = A_c + [[beta, 0], [gamma1, beta]] X_{c-1}
// over the last cells [wstart, c1) of the segment, from X = 0.
template <int NP, class T>
__device__ __forceinline__ void phase_aggregate_tt(const double* lp, long long dstep, int N, int wstart, int c1,
                                                   const PdgCoef& C, T* Y1, T* Y2, T* U, const T* inflow) {
  int cp = wstart - 1;
  if (cp < 0) cp += N;
  T u = (wstart == 0 && inflow) ? *inflow : ld<T>(lp + ((long long)cp * NP + (NP - 1)) * dstep);
  T y1 = zero<T>(), y2 = zero<T>();
  const T zb = PDG_S(T, C, zb);
  const T qz = PDG_C(T, C, q, NP - 1) * zb;
  const T eqz = PDG_C(T, C, Eq, NP - 1) * zb;
  const T beta = PDG_S(T, C, beta), g1 = PDG_S(T, C, gamma1);
  T rowE[NP], rowE2[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    rowE[j] = PDG_C(T, C, E, (NP - 1) * NP + j);
    rowE2[j] = PDG_C(T, C, E2, (NP - 1) * NP + j);
  }
  for (int c = wstart; c < c1; ++c) {
    T v[NP];
    load_cell<NP, T>(lp, dstep, c, v);
    const T a1 = dot_acc<NP>(rowE, v, qz * u);
    const T a2 = dot_acc<NP>(rowE2, v, eqz * u);
    y2 = fma(beta, y2, fma(g1, y1, a2));
    y1 = fma(beta, y1, a1);
    u = v[NP - 1];
  }
  *Y1 = y1;
  *Y2 = y2;
  *U = u;
}

// Phase 2 of T T: sweep [c0, c1) from the inflow pair (x, xp) and old value u.
template <int NP, class T>
__device__ __forceinline__ void phase_sweep_tt(double* lp, long long dstep, int c0, int c1, T x, T xp, T u,
                                               const PdgCoef& C) {
  const T za = PDG_S(T, C, za), zb = PDG_S(T, C, zb);
  const T qn = PDG_C(T, C, q, NP - 1);
  T rowE[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) rowE[j] = PDG_C(T, C, E, (NP - 1) * NP + j);
  for (int c = c0; c < c1; ++c) {
    T v[NP];
    load_cell<NP, T>(lp, dstep, c, v);
    const T z = fma(za, x, zb * u);
    const T zp = fma(za, xp, zb * x);
    T out[NP];
#pragma unroll
    for (int r = 0; r < NP; ++r) {
      T row[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) row[j] = PDG_C(T, C, E2, r * NP + j);
      out[r] = dot_acc<NP>(row, v, fma(PDG_C(T, C, Eq, r), z, PDG_C(T, C, q, r) * zp));
    }
    const T xn = dot_acc<NP>(rowE, v, qn * z);
    store_cell<NP, T>(lp, dstep, c, out);
    xp = out[NP - 1];
    x = xn;
    u = v[NP - 1];
  }
}

// Offset of line `line` of a pass.  Line indices and lineA are below 2^31 (lineA <= the
// lines of one axis), so the division runs in 32-bit arithmetic.
__device__ __forceinline__ long long line_base(const PdgPass& p, int line) {
  const unsigned la = (unsigned)min(p.lineA, 0x7fffffffLL);
  const unsigned u = (unsigned)line;
  return (long long)(u % la) * p.s1 + (long long)(u / la) * p.s2;
}

__device__ __forceinline__ int seg_begin(int s, int N, int S) { return (int)(((long long)s * N) / S); }

// Inflow boundary value of transported population phi on line `line` (non-periodic axes).
template <class T>
__device__ __forceinline__ T inflow_value(const PdgPass& p, int phi, int line) {
  const int side = p.tdir[phi] > 0 ? 0 : 1;
  return ld<T>(p.fb + ((long long)(side * p.fbnent + p.fbent[phi]) * p.nlines + line));
}

template <int NP, class T>
__device__ void transport_op(const PdgPass& p, const PdgCoef& C, T* smY, T* smU, int l_in, int s, int grp,
                             bool active, int line, int bid) {
  const int N = p.ncell, S = p.nseg, LPB = p.lpb, G = p.ngroup;
  const int c0 = seg_begin(s, N, S), c1 = seg_begin(s + 1, N, S);
  const long long base = active ? line_base(p, line) : 0;
  __syncthreads();  // previous writes of the block are visible; nobody writes in phase 1
  if (active) {
    for (int phi = grp; phi < p.ntf; phi += G) {
      const int dir = p.tdir[phi];
      double* fl = p.f + (long long)p.tfield[phi] * p.field_stride + base;
      const long long dstep = dir > 0 ? p.stride : -p.stride;
      double* lp = dir > 0 ? fl : fl + (long long)(p.npl - 1) * p.stride;
      T Y, U;
      if (!C.rev) {
        const int wstart = C.full ? c0 : c1 - C.W;
        T bval;
        const T* inflow = nullptr;
        if (!p.periodic) {
          bval = inflow_value<T>(p, phi, line);
          inflow = &bval;
        }
        phase_aggregate<NP, T>(lp, dstep, N, wstart, c1, C, &Y, &U, inflow);
      } else {
        const int cp = (c0 == 0) ? N - 1 : c0 - 1;
        U = ld<T>(lp + ((long long)cp * NP + (NP - 1)) * dstep);
        phase_aggregate_rev<NP, T>(lp, dstep, c0, C.full ? c1 : c0 + C.W, U, C, &Y);
      }
      const int o = (phi * S + s) * LPB + l_in;
      smY[o] = Y;
      smU[o] = U;
    }
  }
  __syncthreads();
  if (active) {
    const int Lbase = N / S;
    const T bL0 = PDG_S(T, C, betaL0), bL1 = PDG_S(T, C, betaL1);
    for (int phi = grp; phi < p.ntf; phi += G) {
      const int dir = p.tdir[phi];
      double* fl = p.f + (long long)p.tfield[phi] * p.field_stride + base;
      const long long dstep = dir > 0 ? p.stride : -p.stride;
      double* lp = dir > 0 ? fl : fl + (long long)(p.npl - 1) * p.stride;
      if (!C.rev && !p.periodic) {
        // open chain from the inflow boundary (fictitious cell value b, constant in time)
        const T b = inflow_value<T>(p, phi, line);
        T x, u;
        if (s == 0) {
          x = b;
          u = b;
        } else {
          u = smU[(phi * S + s - 1) * LPB + l_in];
          if (!C.full) {
            x = smY[(phi * S + s - 1) * LPB + l_in];
          } else {
            T acc = zero<T>(), cf = from_double<T>(1.0);
            for (int t = s - 1; t >= 0; --t) {
              acc = fma(cf, smY[(phi * S + t) * LPB + l_in], acc);
              const int len = seg_begin(t + 1, N, S) - seg_begin(t, N, S);
              cf = cf * ((len == Lbase) ? bL0 : bL1);
            }
            x = fma(cf, b, acc);
          }
        }
        phase_sweep<NP, T>(lp, dstep, c0, c1, x, u, C);
      } else if (!C.rev) {
        // inflow from the upwind segment s-1 (ring)
        const int sp = (s == 0) ? S - 1 : s - 1;
        const T u = smU[(phi * S + sp) * LPB + l_in];
        T x;
        if (!C.full) {
          x = smY[(phi * S + sp) * LPB + l_in];
        } else {
          T acc = zero<T>(), cf = from_double<T>(1.0);
          int t = sp;
          for (int j = 0; j < S; ++j) {
            acc = fma(cf, smY[(phi * S + t) * LPB + l_in], acc);
            const int len = seg_begin(t + 1, N, S) - seg_begin(t, N, S);
            cf = cf * ((len == Lbase) ? bL0 : bL1);
            t = (t == 0) ? S - 1 : t - 1;
          }
          x = acc * PDG_S(T, C, inv_ring);
        }
        phase_sweep<NP, T>(lp, dstep, c0, c1, x, u, C);
      } else {
        // outflow value of the own segment from the downwind segment s+1 (ring)
        const int sn = (s == S - 1) ? 0 : s + 1;
        const T u0 = smU[(phi * S + s) * LPB + l_in];
        T x;
        if (!C.full) {
          x = smY[(phi * S + sn) * LPB + l_in];
        } else {
          T acc = zero<T>(), cf = from_double<T>(1.0);
          int t = sn;
          for (int j = 0; j < S; ++j) {
            acc = fma(cf, smY[(phi * S + t) * LPB + l_in], acc);
            const int len = seg_begin(t + 1, N, S) - seg_begin(t, N, S);
            cf = cf * ((len == Lbase) ? bL0 : bL1);
            t = (t == S - 1) ? 0 : t + 1;
          }
          x = acc * PDG_S(T, C, inv_ring);
        }
        phase_sweep_rev<NP, T>(lp, dstep, c0, c1, x, u0, C);
      }
    }
  }
}

template <int NP, class T>
__device__ void transport_op_tt(const PdgPass& p, const PdgCoef& C, T* smY, T* smY2, T* smU, int l_in, int s,
                                int grp, bool active, int line) {
  const int N = p.ncell, S = p.nseg, LPB = p.lpb, G = p.ngroup;
  const int c0 = seg_begin(s, N, S), c1 = seg_begin(s + 1, N, S);
  const long long base = active ? line_base(p, line) : 0;
  __syncthreads();
  if (active) {
    for (int phi = grp; phi < p.ntf; phi += G) {
      const int dir = p.tdir[phi];
      double* fl = p.f + (long long)p.tfield[phi] * p.field_stride + base;
      const long long dstep = dir > 0 ? p.stride : -p.stride;
      double* lp = dir > 0 ? fl : fl + (long long)(p.npl - 1) * p.stride;
      T Y1, Y2, U;
      T bval;
      const T* inflow = nullptr;
      if (!p.periodic) {
        bval = inflow_value<T>(p, phi, line);
        inflow = &bval;
      }
      phase_aggregate_tt<NP, T>(lp, dstep, N, c1 - C.W2, c1, C, &Y1, &Y2, &U, inflow);
      const int o = (phi * S + s) * LPB + l_in;
      smY[o] = Y1;
      smY2[o] = Y2;
      smU[o] = U;
    }
  }
  __syncthreads();
  if (active) {
    for (int phi = grp; phi < p.ntf; phi += G) {
      const int dir = p.tdir[phi];
      double* fl = p.f + (long long)p.tfield[phi] * p.field_stride + base;
      const long long dstep = dir > 0 ? p.stride : -p.stride;
      double* lp = dir > 0 ? fl : fl + (long long)(p.npl - 1) * p.stride;
      if (!p.periodic && s == 0) {
        const T b = inflow_value<T>(p, phi, line);   // both sub-steps see the constant fictitious value
        phase_sweep_tt<NP, T>(lp, dstep, c0, c1, b, b, b, C);
      } else {
        const int o = (phi * S + ((s == 0) ? S - 1 : s - 1)) * LPB + l_in;
        phase_sweep_tt<NP, T>(lp, dstep, c0, c1, smY[o], smY2[o], smU[o], C);
      }
    }
  }
}

// Lines [*l0, *l0 + *cnt) of block bid (see PdgPass::nblocks); *cnt <= lpb.
__device__ __forceinline__ void block_lines(const PdgPass& p, int bid, int* l0, int* cnt) {
  if (p.nblocks > 0) {
    const long long a = (long long)bid * p.nlines / p.nblocks;
    const long long b = (long long)(bid + 1) * p.nlines / p.nblocks;
    *l0 = (int)a;
    *cnt = (int)(b - a);
  } else {
    *l0 = bid * p.lpb;
    *cnt = min(p.lpb, p.nlines - *l0);
  }
}

template <int MV, class T>
__device__ void collision_op(const PdgPass& p, int bid) {
  __syncthreads();
  constexpr int NF = NFields<MV>::value;
  int l0, cnt;
  block_lines(p, bid, &l0, &cnt);
  const int tile = cnt * p.npl;   // at most lpb * npl points: 32-bit index arithmetic
  for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) {
    const int l_in = idx % cnt;
    const int tpos = idx / cnt;
    const int line = l0 + l_in;
    const long long off = line_base(p, line) + tpos * p.stride;
    const int nf = p.model.nf;
    T v[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k)
      v[k] = (k < nf) ? ld<T>(p.f + (long long)coll_slot<MV>(k, p.dslot) * p.field_stride + off) : zero<T>();
    bool done = false;
    if constexpr (MV == MV_D2Q9) {
      if (p.src.flags) {
        d2q9_source_collide<T>(v, p.src, p.model, off);
        done = true;
      }
    }
    if (!done) collide<MV, T>(v, p.model);
#pragma unroll
    for (int k = 0; k < NF; ++k)
      if (k < nf) st(p.f + (long long)coll_slot<MV>(k, p.dslot) * p.field_stride + off, v[k]);
  }
}

// One pass over block `bid` of a pass descriptor: the op list of p applied to the
// lpb lines owned by the block.  sm: 3 * ntf * nseg * lpb 8-byte words.  All threads
// of the block must call it (it contains __syncthreads); threads with index >=
// lpb * nseg * ngroup take part in the barriers and in the collision phase only.
template <int NP, int MV, class T>
__device__ __forceinline__ void pass_body(const PdgPass& p, int bid, double* sm) {
  const int LPB = p.lpb, S = p.nseg, G = p.ngroup;
  const int t = threadIdx.x;
  const int nthr = LPB * S * G;
  // thread -> (line, segment, field group): lines fastest (coalesced streaming from global
  // memory), or field groups fastest (tmap = 1, the line-resident kernel: consecutive
  // threads then sweep different populations, whose staged copies start on different banks,
  // instead of segments of one line, which share banks)
  const int l_in = p.tmap ? t / (G * S) : t % LPB;
  const int s = p.tmap ? (t / G) % S : (t / LPB) % S;
  const int grp = p.tmap ? t % G : t / (LPB * S);
  int l0, cnt;
  block_lines(p, bid, &l0, &cnt);
  const int line = l0 + l_in;
  const bool active = (t < nthr) && l_in < cnt;
  const int cap = p.ntf * S * LPB;
  T* smY = reinterpret_cast<T*>(sm);
  T* smU = smY + cap;
  T* smY2 = smU + cap;
  for (int o = 0; o < p.nops; ++o) {
    if (p.op[o] == PDG_OP_T) {
      if (p.opcoef[o] == 0)
        transport_op<NP, T>(p, p.coef[0], smY, smU, l_in, s, grp, active, line, bid);
      else
        transport_op<NP, T>(p, p.coef[1], smY, smU, l_in, s, grp, active, line, bid);
    } else if (p.op[o] == PDG_OP_TT) {
      transport_op_tt<NP, T>(p, p.coef[p.opcoef[o]], smY, smY2, smU, l_in, s, grp, active, line);
    } else if (p.op[o] == PDG_OP_C) {
      if constexpr (MV != MV_NONE) collision_op<MV, T>(p, bid);
    }
  }
}

}  // namespace pdgdev
