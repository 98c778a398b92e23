// Device code shared by the single-instance kernels (pdg_kernels.cu) and the
// batched persistent kernel (pdg_batch.cu): collision of eq. (3.12), the two-phase
// exact periodic transport sweep of eq. (3.11), and the pass body.
#pragma once
#include <cuda_runtime.h>

#include "pdg_internal.h"
#include "../../include/pdg.h"

namespace pdgdev {

enum { MV_ADV = 0, MV_SW = 1, MV_EU1 = 2, MV_EU2 = 3, MV_EU3 = 4, MV_NONE = 5 };

// ---------------------------------------------------------------------------
// Collision at one point (eq. (3.12)); v holds the m * 2D populations.
// f^eq_{k,i} = w_k/(2D) + (v_i . q_k(w))/(2 lambda^2) = w_k/(2D) + s_i q^a_k / (2 lambda)
// for v_i = s_i lambda e_a.
template <int MV>
__device__ __forceinline__ void collide(double* v, const PdgModel& M);

template <>
__device__ __forceinline__ void collide<MV_ADV>(double* v, const PdgModel& M) {
  const int nv = M.nv;
  double w = 0.0;
#pragma unroll
  for (int i = 0; i < 6; ++i)
    if (i < nv) w += v[i];
  const double om = M.omega, om1 = 1.0 - M.omega;
#pragma unroll
  for (int i = 0; i < 6; ++i)
    if (i < nv) v[i] = fma(om * M.cadv[i], w, om1 * v[i]);
}

template <>
__device__ __forceinline__ void collide<MV_SW>(double* v, const PdgModel& M) {
  // w = (h, hu, hv), populations k*4 + {+x, -x, +y, -y}
  double w[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) w[k] = (v[4 * k] + v[4 * k + 1]) + (v[4 * k + 2] + v[4 * k + 3]);
  const double h = w[0], hu = w[1], hv = w[2];
  const double ih = 1.0 / h;
  const double u = hu * ih, vv = hv * ih;
  const double p = 0.5 * M.gravity * h * h;
  const double qx[3] = {hu, fma(hu, u, p), hv * u};
  const double qy[3] = {hv, hu * vv, fma(hv, vv, p)};
  const double om = M.omega, om1 = 1.0 - M.omega;
  const double c0 = 0.25 * om;                 // omega / (2D)
  const double c1 = om / (2.0 * M.lambda);     // omega / (2 lambda)
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double b = c0 * w[k];
    v[4 * k + 0] = fma(om1, v[4 * k + 0], fma(c1, qx[k], b));
    v[4 * k + 1] = fma(om1, v[4 * k + 1], fma(-c1, qx[k], b));
    v[4 * k + 2] = fma(om1, v[4 * k + 2], fma(c1, qy[k], b));
    v[4 * k + 3] = fma(om1, v[4 * k + 3], fma(-c1, qy[k], b));
  }
}

template <int D>
__device__ __forceinline__ void collide_euler(double* v, const PdgModel& M) {
  constexpr int m = D + 2, nv = 2 * D;
  double w[m];
#pragma unroll
  for (int k = 0; k < m; ++k) {
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < nv; ++i) s += v[k * nv + i];
    w[k] = s;
  }
  const double rho = w[0], E = w[D + 1];
  const double ir = 1.0 / rho;
  double u[D];
  double ke = 0.0;
#pragma unroll
  for (int b = 0; b < D; ++b) {
    u[b] = w[1 + b] * ir;
    ke = fma(w[1 + b], u[b], ke);
  }
  const double p = (M.gamma - 1.0) * (E - 0.5 * ke);
  const double om = M.omega, om1 = 1.0 - M.omega;
  const double c0 = om / (2.0 * D);
  const double c1 = om / (2.0 * M.lambda);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    double q[m];
    q[0] = w[1 + a];
#pragma unroll
    for (int b = 0; b < D; ++b) q[1 + b] = (a == b) ? fma(w[1 + b], u[a], p) : w[1 + b] * u[a];
    q[D + 1] = (E + p) * u[a];
#pragma unroll
    for (int k = 0; k < m; ++k) {
      const double bse = c0 * w[k];
      v[k * nv + 2 * a] = fma(om1, v[k * nv + 2 * a], fma(c1, q[k], bse));
      v[k * nv + 2 * a + 1] = fma(om1, v[k * nv + 2 * a + 1], fma(-c1, q[k], bse));
    }
  }
}

template <>
__device__ __forceinline__ void collide<MV_EU1>(double* v, const PdgModel& M) { collide_euler<1>(v, M); }
template <>
__device__ __forceinline__ void collide<MV_EU2>(double* v, const PdgModel& M) { collide_euler<2>(v, M); }
template <>
__device__ __forceinline__ void collide<MV_EU3>(double* v, const PdgModel& M) { collide_euler<3>(v, M); }
template <>
__device__ __forceinline__ void collide<MV_NONE>(double*, const PdgModel&) {}

template <int MV>
struct NFields { static constexpr int value = PDG_MAXF; };
template <> struct NFields<MV_SW> { static constexpr int value = 12; };
template <> struct NFields<MV_EU1> { static constexpr int value = 6; };
template <> struct NFields<MV_EU2> { static constexpr int value = 16; };
template <> struct NFields<MV_EU3> { static constexpr int value = 30; };
template <> struct NFields<MV_ADV> { static constexpr int value = 6; };
template <> struct NFields<MV_NONE> { static constexpr int value = 1; };

// ---------------------------------------------------------------------------
// Transport phases for one population along one line.  lp points at traversal
// index 0 of the line, dstep is the signed stride between traversal indices.

template <int NP>
__device__ __forceinline__ void load_cell(const double* lp, long long dstep, int c, double* v) {
  const double* p0 = lp + (long long)c * NP * dstep;
#pragma unroll
  for (int j = 0; j < NP; ++j) v[j] = p0[j * dstep];
}

// Phase 1: aggregate Y of the recurrence over cells [wstart, c1) starting from 0,
// and the old last-node value of cell c1 - 1.
template <int NP>
__device__ __forceinline__ void phase_aggregate(const double* lp, long long dstep, int N, int wstart,
                                                int c1, const PdgCoef& C, double* Y, double* U) {
  int cp = wstart - 1;
  if (cp < 0) cp += N;
  double u = lp[((long long)cp * NP + (NP - 1)) * dstep];
  double y = 0.0;
  const double qz = C.q[NP - 1] * C.zb;
  for (int c = wstart; c < c1; ++c) {
    double v[NP];
    load_cell<NP>(lp, dstep, c, v);
    double alpha = qz * u;
#pragma unroll
    for (int j = 0; j < NP; ++j) alpha = fma(C.E[(NP - 1) * NP + j], v[j], alpha);
    y = fma(C.beta, y, alpha);
    u = v[NP - 1];
  }
  *Y = y;
  *U = u;
}

// Phase 2: sweep cells [c0, c1) with inflow (x, u) and write the new values in place.
template <int NP>
__device__ __forceinline__ void phase_sweep(double* lp, long long dstep, int c0, int c1, double x,
                                            double u, const PdgCoef& C) {
  for (int c = c0; c < c1; ++c) {
    double v[NP];
    load_cell<NP>(lp, dstep, c, v);
    const double z = fma(C.za, x, C.zb * u);
    double* p0 = lp + (long long)c * NP * dstep;
    double last = 0.0;
#pragma unroll
    for (int r = 0; r < NP; ++r) {
      double acc = C.q[r] * z;
#pragma unroll
      for (int j = 0; j < NP; ++j) acc = fma(C.E[r * NP + j], v[j], acc);
      p0[r * dstep] = acc;
      if (r == NP - 1) last = acc;
    }
    x = last;
    u = v[NP - 1];
  }
}

// Reverse mode (|beta| > 1): x_{c-1} = gamma (x_c - alpha_c).
// Phase 1: y = x_{c0-1} from the first cells [c0, cend) of the segment, given the
// old last-node value u0 of cell c0 - 1.
template <int NP>
__device__ __forceinline__ void phase_aggregate_rev(const double* lp, long long dstep, int c0, int cend,
                                                    double u0, const PdgCoef& C, double* Y) {
  double y = 0.0;
  const double qz = C.q[NP - 1] * C.zb;
  for (int c = cend - 1; c >= c0; --c) {
    double v[NP];
    load_cell<NP>(lp, dstep, c, v);
    const double u = (c > c0) ? lp[((long long)(c - 1) * NP + (NP - 1)) * dstep] : u0;
    double alpha = qz * u;
#pragma unroll
    for (int j = 0; j < NP; ++j) alpha = fma(C.E[(NP - 1) * NP + j], v[j], alpha);
    y = C.gamma * (y - alpha);
  }
  *Y = y;
}

// Phase 2 (reverse): sweep cells c1-1 down to c0 from x = x_{c1-1}; u0 = old value of
// the last node of cell c0 - 1 (saved before any write).
template <int NP>
__device__ __forceinline__ void phase_sweep_rev(double* lp, long long dstep, int c0, int c1, double x,
                                                double u0, const PdgCoef& C) {
  const double qz = C.q[NP - 1] * C.zb;
  for (int c = c1 - 1; c >= c0; --c) {
    double v[NP];
    load_cell<NP>(lp, dstep, c, v);
    const double u = (c > c0) ? lp[((long long)(c - 1) * NP + (NP - 1)) * dstep] : u0;
    double alpha = qz * u;
#pragma unroll
    for (int j = 0; j < NP; ++j) alpha = fma(C.E[(NP - 1) * NP + j], v[j], alpha);
    const double xm = C.gamma * (x - alpha);
    const double z = fma(C.za, xm, C.zb * u);
    double* p0 = lp + (long long)c * NP * dstep;
#pragma unroll
    for (int r = 0; r < NP; ++r) {
      double acc = C.q[r] * z;
#pragma unroll
      for (int j = 0; j < NP; ++j) acc = fma(C.E[r * NP + j], v[j], acc);
      p0[r * dstep] = acc;
    }
    x = xm;
  }
}

__device__ __forceinline__ long long line_base(const PdgPass& p, int line) {
  return (long long)(line % p.lineA) * p.s1 + (long long)(line / p.lineA) * p.s2;
}

__device__ __forceinline__ int seg_begin(int s, int N, int S) { return (int)(((long long)s * N) / S); }

template <int NP>
__device__ void transport_op(const PdgPass& p, const PdgCoef& C, double* smY, double* smU, int l_in,
                             int s, int grp, bool active, int line, int bid) {
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
      double Y, U;
      if (!C.rev) {
        const int wstart = C.full ? c0 : c1 - C.W;
        phase_aggregate<NP>(lp, dstep, N, wstart, c1, C, &Y, &U);
      } else {
        const int cp = (c0 == 0) ? N - 1 : c0 - 1;
        U = lp[((long long)cp * NP + (NP - 1)) * dstep];
        phase_aggregate_rev<NP>(lp, dstep, c0, C.full ? c1 : c0 + C.W, U, C, &Y);
      }
      const int o = (phi * S + s) * LPB + l_in;
      smY[o] = Y;
      smU[o] = U;
    }
  }
  __syncthreads();
  if (active) {
    const int Lbase = N / S;
    for (int phi = grp; phi < p.ntf; phi += G) {
      const int dir = p.tdir[phi];
      double* fl = p.f + (long long)p.tfield[phi] * p.field_stride + base;
      const long long dstep = dir > 0 ? p.stride : -p.stride;
      double* lp = dir > 0 ? fl : fl + (long long)(p.npl - 1) * p.stride;
      if (!C.rev) {
        // inflow from the upwind segment s-1 (ring)
        const int sp = (s == 0) ? S - 1 : s - 1;
        const double u = smU[(phi * S + sp) * LPB + l_in];
        double x;
        if (!C.full) {
          x = smY[(phi * S + sp) * LPB + l_in];
        } else {
          double acc = 0.0, cf = 1.0;
          int t = sp;
          for (int j = 0; j < S; ++j) {
            acc = fma(cf, smY[(phi * S + t) * LPB + l_in], acc);
            const int len = seg_begin(t + 1, N, S) - seg_begin(t, N, S);
            cf *= (len == Lbase) ? C.betaL0 : C.betaL1;
            t = (t == 0) ? S - 1 : t - 1;
          }
          x = acc * C.inv_ring;
        }
        phase_sweep<NP>(lp, dstep, c0, c1, x, u, C);
      } else {
        // outflow value of the own segment from the downwind segment s+1 (ring)
        const int sn = (s == S - 1) ? 0 : s + 1;
        const double u0 = smU[(phi * S + s) * LPB + l_in];
        double x;
        if (!C.full) {
          x = smY[(phi * S + sn) * LPB + l_in];
        } else {
          double acc = 0.0, cf = 1.0;
          int t = sn;
          for (int j = 0; j < S; ++j) {
            acc = fma(cf, smY[(phi * S + t) * LPB + l_in], acc);
            const int len = seg_begin(t + 1, N, S) - seg_begin(t, N, S);
            cf *= (len == Lbase) ? C.betaL0 : C.betaL1;
            t = (t == S - 1) ? 0 : t + 1;
          }
          x = acc * C.inv_ring;
        }
        phase_sweep_rev<NP>(lp, dstep, c0, c1, x, u0, C);
      }
    }
  }
}

template <int MV>
__device__ void collision_op(const PdgPass& p, int bid) {
  __syncthreads();
  constexpr int NF = NFields<MV>::value;
  const int LPB = p.lpb;
  const long long tile = (long long)LPB * p.npl;
  for (long long idx = threadIdx.x; idx < tile; idx += blockDim.x) {
    const int l_in = (int)(idx % LPB);
    const long long tpos = idx / LPB;
    const int line = bid * LPB + l_in;
    if (line >= p.nlines) continue;
    const long long off = line_base(p, line) + tpos * p.stride;
    const int nf = p.model.m * p.model.nv;
    double v[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) v[k] = (k < nf) ? p.f[(long long)k * p.field_stride + off] : 0.0;
    collide<MV>(v, p.model);
#pragma unroll
    for (int k = 0; k < NF; ++k)
      if (k < nf) p.f[(long long)k * p.field_stride + off] = v[k];
  }
}


// One pass over block `bid` of a pass descriptor: the op list of p applied to the
// lpb lines owned by the block.  sm: 2 * ntf * nseg * lpb doubles.  All threads of
// the block must call it (it contains __syncthreads); threads with index >=
// lpb * nseg * ngroup take part in the barriers and in the collision phase only.
template <int NP, int MV>
__device__ __forceinline__ void pass_body(const PdgPass& p, int bid, double* sm) {
  const int LPB = p.lpb, S = p.nseg;
  const int t = threadIdx.x;
  const int nthr = LPB * S * p.ngroup;
  const int l_in = t % LPB;
  const int s = (t / LPB) % S;
  const int grp = t / (LPB * S);
  const int line = bid * LPB + l_in;
  const bool active = (t < nthr) && line < p.nlines;
  const int cap = p.ntf * S * LPB;
  double* smY = sm;
  double* smU = sm + cap;
  for (int o = 0; o < p.nops; ++o) {
    if (p.op[o] == PDG_OP_T) {
      if (p.opcoef[o] == 0)
        transport_op<NP>(p, p.coef[0], smY, smU, l_in, s, grp, active, line, bid);
      else
        transport_op<NP>(p, p.coef[1], smY, smU, l_in, s, grp, active, line, bid);
    } else if (p.op[o] == PDG_OP_C) {
      if constexpr (MV != MV_NONE) collision_op<MV>(p, bid);
    }
  }
}

}  // namespace pdgdev
