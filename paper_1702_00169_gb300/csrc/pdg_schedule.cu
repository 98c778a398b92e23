// The pass schedule of the palindromic compositions.
//
// Schedule.  M2(dt) = T(dt/2) C(dt) T(dt/2) (Section 3.2) with T the product of
// the per-population transports; transports along different axes act on
// different populations, so they commute exactly.  Between two collisions every
// population therefore sees its axis' trailing T(dt/2) of one step and leading T(dt/2) of
// the next, in that order, whatever the order of the axes.  With L the axis whose pass
// carries the collision (the last axis, or the one PDG_OPT_COLLISION_AXIS names), nsteps
// steps are issued as
//   for a != L: pass_a [T(dt/2)];   pass_L [T(dt/2), C]
//   repeat nsteps - 1:  for a != L: pass_a [T(dt/2), T(dt/2)];   pass_L [T(dt/2), T(dt/2), C]
//   for a != L: pass_a [T(dt/2)];   pass_L [T(dt/2)]
// which applies to every population exactly the sequence of the naive order, and puts
// every pair of half steps of one axis into one pass (the issue composes it into one
// T T sweep), the collision at the end of the last axis' pass.
// The collapsed scheme of Section 5.1 merges interior half steps into T(dt).
// The passes are generated one at a time into a sink: pdg_step issues each as it comes, so
// its host memory does not grow with the step count; the other callers collect them.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "pdg_ctx.h"

namespace pdgapi {

// Fill the launch-dependent fields of a coefficient set for segments of a line of
// N cells.  Returns 0, or -1 when the periodic system is singular (|beta| = 1 with
// beta^N = 1).
int finish_coef(PdgCoef* C, int N, int S, bool periodic) {
  const int Lbase = N / S;
  const double ab = std::fabs(C->beta);
  C->rev = ab > 1.0 ? 1 : 0;
  C->gamma = C->rev ? 1.0 / C->beta : 0.0;
  const double r = C->rev ? C->gamma : C->beta;
  const int W = pdg_plan_window(r);
  C->W = W;
  C->full = (W > Lbase) ? 1 : 0;
  C->betaL0 = std::pow(r, (double)Lbase);
  C->betaL1 = std::pow(r, (double)(Lbase + 1));
  const double rN = std::pow(r, (double)N);
  if (periodic && !(std::fabs(1.0 - rN) > 1e-12)) return -1;
  C->inv_ring = periodic ? 1.0 / (1.0 - rN) : 0.0;
  pdg_coef_split(C);
  return 0;
}

// Window of a coefficient set in the stable direction.
int stable_window(const PdgCoef& C) {
  const double ab = std::fabs(C.beta);
  return pdg_plan_window(ab > 1.0 ? 1.0 / C.beta : C.beta);
}

int plan_line_coef(const pdg_ctx* c, int axis, double delta, PdgCoef* C) {
  const double nu = 2.0 * c->model.lambda * delta / c->h[axis];
  return pdg_plan_coef(c->order, nu, c->theta, C);
}

// Kind of a pass: 0 = transport only, 1 = contains the collision.
int pass_kind(const PdgPassSpec& sp) {
  for (int o = 0; o < sp.nops; ++o)
    if (sp.op[o] == PDG_OP_C) return 1;
  return 0;
}

PdgPassSpec spec(int axis, int nops, const int* ops, const int* ci, const PdgCoef* cs, int ncs) {
  PdgPassSpec sp;
  std::memset(&sp, 0, sizeof(sp));
  sp.axis = axis;
  sp.nops = nops;
  for (int o = 0; o < nops; ++o) {
    sp.op[o] = ops[o];
    sp.opcoef[o] = ci[o];
  }
  sp.ncs = ncs;
  for (int i = 0; i < ncs; ++i) sp.cs[i] = cs[i];
  return sp;
}

// The line passes of nsteps palindromic steps (see the schedule at the top of this file),
// in order, into `sink`.  Every argument check comes before the first pass; after a sink
// error no further pass reaches it and that error is returned.
int emit_line_schedule(pdg_ctx* c, double dt, int nsteps, const PassSink& sink) {
  if (nsteps <= 0) return PDG_OK;
  const int D = c->dim, L = (c->caxis >= 0 && c->caxis < D) ? c->caxis : D - 1;
  int rc = PDG_OK;
  auto put = [&](const PdgPassSpec& sp) {
    if (rc == PDG_OK) rc = sink(sp);
  };
  PdgCoef half[3], full[3];
  for (int a = 0; a < D; ++a) {
    if (plan_line_coef(c, a, 0.5 * dt, &half[a])) return fail(c, PDG_ERR_ARG, "singular transport step");
    if (plan_line_coef(c, a, dt, &full[a])) return fail(c, PDG_ERR_ARG, "singular transport step");
    PdgCoef t0 = half[a], t1 = full[a];
    if (finish_coef(&t0, c->N[a], 1, c->periodic[a]) ||
        (c->scheme == PDG_SCHEME_M2_COLLAPSED && finish_coef(&t1, c->N[a], 1, c->periodic[a])))
      return fail(c, PDG_ERR_ARG, "singular periodic transport system (|beta| = 1)");
    if (!c->periodic[a] && (t0.rev || (c->scheme == PDG_SCHEME_M2_COLLAPSED && t1.rev)))
      return fail(c, PDG_ERR_UNSUPPORTED, "time steps with |beta| > 1 on an inflow (non-periodic) axis");
  }
  const int T = PDG_OP_T, C = PDG_OP_C;
  const int z1[1] = {0}, z2[2] = {0, 0}, z3[3] = {0, 0, 0};
  const int o1[1] = {T}, o2[2] = {T, T};
  if (c->scheme == PDG_SCHEME_M2KIN) {
    // T(dt/4) C T(dt/2) C T(dt/4) per step.  The collisions split the run into the
    // transport segments seg_0 = T(q), then alternately T(h) and T(q) T(q) (the trailing
    // quarter of a step and the leading quarter of the next), and seg_2n = T(q).  Each
    // collision runs in a last-axis pass together with the last axis' transports around
    // it; the other axes transport each segment in passes between the collisions.
    PdgCoef qc[3], hc[3];
    for (int a = 0; a < D; ++a) {
      if (plan_line_coef(c, a, 0.25 * dt, &qc[a]) || plan_line_coef(c, a, 0.5 * dt, &hc[a]))
        return fail(c, PDG_ERR_ARG, "singular transport step");
      PdgCoef t0 = qc[a], t1 = hc[a];
      if (finish_coef(&t0, c->N[a], 1, c->periodic[a]) || finish_coef(&t1, c->N[a], 1, c->periodic[a]))
        return fail(c, PDG_ERR_ARG, "singular periodic transport system (|beta| = 1)");
      if (!c->periodic[a] && (t0.rev || t1.rev))
        return fail(c, PDG_ERR_UNSUPPORTED, "time steps with |beta| > 1 on an inflow (non-periodic) axis");
    }
    const long long nseg = 2LL * nsteps + 1;
    // segment j: number of sub-steps and their coefficient index (0 = quarter, 1 = half)
    auto seg_n = [&](long long j) { return (j == 0 || j == nseg - 1) ? 1 : ((j % 2 == 1) ? 1 : 2); };
    auto seg_ci = [&](long long j) { return (j % 2 == 1) ? 1 : 0; };
    auto other_axes = [&](long long j) {
      for (int a = 0; a < D; ++a) {
        if (a == L) continue;
        PdgCoef cs[2] = {qc[a], hc[a]};
        const int ops[2] = {T, T}, ci[2] = {seg_ci(j), seg_ci(j)};
        put(spec(a, seg_n(j), ops, ci, cs, 2));
      }
    };
    PdgCoef csL[2] = {qc[L], hc[L]};
    other_axes(0);
    {
      const int ops[3] = {T, C, T}, ci[3] = {seg_ci(0), 0, seg_ci(1)};
      put(spec(L, 3, ops, ci, csL, 2));
    }
    for (long long j = 1; j < nseg - 1 && rc == PDG_OK; ++j) {
      other_axes(j);
      int ops[3] = {C, T, T}, ci[3] = {0, seg_ci(j + 1), seg_ci(j + 1)};
      put(spec(L, 1 + seg_n(j + 1), ops, ci, csL, 2));
    }
    other_axes(nseg - 1);
    return rc;
  }
  if (c->scheme == PDG_SCHEME_M2) {
    const int otc[2] = {T, C}, ottc[3] = {T, T, C};
    for (int a = 0; a < D; ++a)
      if (a != L) put(spec(a, 1, o1, z1, &half[a], 1));
    put(spec(L, 2, otc, z2, &half[L], 1));
    for (int s = 1; s < nsteps && rc == PDG_OK; ++s) {
      for (int a = 0; a < D; ++a)
        if (a != L) put(spec(a, 2, o2, z2, &half[a], 1));
      put(spec(L, 3, ottc, z3, &half[L], 1));
    }
    for (int a = 0; a < D; ++a)
      if (a != L) put(spec(a, 1, o1, z1, &half[a], 1));
    put(spec(L, 1, o1, z1, &half[L], 1));
  } else {
    for (int a = 0; a < D; ++a)
      if (a != L) put(spec(a, 1, o1, z1, &half[a], 1));
    for (int s = 0; s < nsteps && rc == PDG_OK; ++s) {
      PdgCoef cs[2] = {half[L], full[L]};
      const int ops[2] = {T, C}, ci[2] = {s == 0 ? 0 : 1, 0};
      put(spec(L, 2, ops, ci, cs, 2));
      for (int a = 0; a < D; ++a)
        if (a != L) put(spec(a, 1, o1, z1, s < nsteps - 1 ? &full[a] : &half[a], 1));
    }
    put(spec(L, 1, o1, z1, &half[L], 1));
  }
  return rc;
}

// The full pass list.  D2Q9 adds the diagonal transports: the sub-steps between two
// collisions (and before the first / after the last) run as diagonal passes issued
// just before the line pass that holds the next collision (transports of different
// populations commute); each diagonal pass swaps the slot set of populations 5-8, the
// collision reads them where they are, and a final copy returns them to slots 5-8.
int emit_schedule_one(pdg_ctx* c, double dt, int nsteps, const PassSink& sink) {
  Lattice Lat;
  if (!lattice_of(c->model.kind, &Lat) || nsteps <= 0) return emit_line_schedule(c, dt, nsteps, sink);
  if (!(dt > 0.0)) return fail(c, PDG_ERR_UNSUPPORTED, "diagonal transport needs dt > 0");
  if (c->src.flags && c->scheme == PDG_SCHEME_M2KIN)
    return fail(c, PDG_ERR_UNSUPPORTED, "sources are defined for M2 and M2_collapsed");
  // diagonal sub-steps of transport segment j (the segments between the collisions, in
  // order): nseg segments, one more than the collisions
  const double h = 0.5 * dt, q = 0.25 * dt;
  const int scheme = c->scheme;
  const long long nseg = scheme == PDG_SCHEME_M2KIN ? 2LL * nsteps + 1 : (long long)nsteps + 1;
  auto seg = [&](long long j, double* dl) -> int {
    const bool end = j == 0 || j == nseg - 1;
    if (scheme == PDG_SCHEME_M2) {
      dl[0] = dl[1] = h;
      return end ? 1 : 2;
    }
    if (scheme == PDG_SCHEME_M2_COLLAPSED) {
      dl[0] = end ? h : dt;
      return 1;
    }
    if (end || j % 2 == 0) {       // M2^kin: T(dt/4) at the ends, T(dt/4) T(dt/4) between steps
      dl[0] = dl[1] = q;
      return end ? 1 : 2;
    }
    dl[0] = h;                     // the middle of a step
    return 1;
  };
  int slot = Lat.diag;
  long long ci = 0;
  auto diag = [&](double delta) {
    PdgPassSpec d;
    std::memset(&d, 0, sizeof(d));
    d.axis = -1;
    d.ddelta = delta;
    d.dslot_in = slot;
    slot = (slot == Lat.diag) ? Lat.scratch : Lat.diag;
    return sink(d);
  };
  auto segment = [&](long long j) {
    double dl[2];
    const int k = seg(j, dl);
    for (int i = 0; i < k; ++i)
      if (int r = diag(dl[i])) return r;
    return (int)PDG_OK;
  };
  int r = emit_line_schedule(c, dt, nsteps, [&](const PdgPassSpec& line) -> int {
    PdgPassSpec sp = line;
    if (pass_kind(sp)) {
      if (ci >= nseg) return fail(c, PDG_ERR_ARG, "internal: schedule segments");
      if (int e = segment(ci)) return e;
      ++ci;
      sp.dslot = slot;
      sp.sdelta = c->src.flags ? 0.5 * dt : 0.0;   // S(dt/2) C(dt) S(dt/2)
    }
    return sink(sp);
  });
  if (r) return r;
  if (ci + 1 != nseg) return fail(c, PDG_ERR_ARG, "internal: schedule segments");
  if (int e = segment(ci)) return e;
  if (slot != Lat.diag) {
    PdgPassSpec cp;
    std::memset(&cp, 0, sizeof(cp));
    cp.axis = -2;   // copy slots 9-12 back to 5-8
    return sink(cp);
  }
  return PDG_OK;
}

// The pass list of nsteps steps of the context's scheme.  M4^kin (PDG_SCHEME_M4KIN) is the
// triple jump M2^kin(g1 dt) M2^kin(g2 dt) M2^kin(g1 dt) per step (Section 3.2: palindromic
// compositions of M2^kin; H. Yoshida, Phys. Lett. A 150 (1990)), g1 = 1/(2 - 2^(1/3)),
// g2 = 1 - 2 g1 < 0: three M2^kin schedules per step, the middle one backwards in time.
// Its steps are all alike, so one step is generated first without a sink to check the
// arguments of all three sub-steps before any pass is emitted.
int emit_schedule(pdg_ctx* c, double dt, int nsteps, const PassSink& sink) {
  if (c->scheme != PDG_SCHEME_M4KIN) return emit_schedule_one(c, dt, nsteps, sink);
  Lattice L;
  if (lattice_of(c->model.kind, &L))
    return fail(c, PDG_ERR_UNSUPPORTED, "M4^kin has a backward sub-step: not available for diagonal velocities");
  if (c->src.flags) return fail(c, PDG_ERR_UNSUPPORTED, "sources are defined for M2 and M2_collapsed");
  const double g1 = 1.0 / (2.0 - std::cbrt(2.0)), g2 = 1.0 - 2.0 * g1;
  const PassSink none = [](const PdgPassSpec&) { return (int)PDG_OK; };
  c->scheme = PDG_SCHEME_M2KIN;
  int r = PDG_OK;
  try {
    for (double g : {g1, g2, g1})
      if (nsteps > 0 && r == PDG_OK) r = emit_schedule_one(c, g * dt, 1, none);
    for (int s = 0; s < nsteps && r == PDG_OK; ++s)
      for (double g : {g1, g2, g1}) {
        if ((r = emit_schedule_one(c, g * dt, 1, sink)) != PDG_OK) break;
      }
  } catch (...) {
    c->scheme = PDG_SCHEME_M4KIN;
    throw;
  }
  c->scheme = PDG_SCHEME_M4KIN;
  return r;
}

int build_schedule(pdg_ctx* c, double dt, int nsteps, std::vector<PdgPassSpec>& out) {
  out.clear();
  if (nsteps > 0) out.reserve((2 * (size_t)nsteps + 1) * (size_t)c->dim);   // at least the passes of every scheme
  return emit_schedule(c, dt, nsteps, [&](const PdgPassSpec& sp) {
    out.push_back(sp);
    return (int)PDG_OK;
  });
}

// build_schedule for the C entry points: the pass list lives in host memory (about 2.3 KB
// per pass, a few passes per step), and a failed allocation is reported as PDG_ERR_OOM
// instead of letting the exception cross the C ABI.
int build_schedule_checked(pdg_ctx* c, double dt, int nsteps, std::vector<PdgPassSpec>& out) {
  try {
    return build_schedule(c, dt, nsteps, out);
  } catch (const std::bad_alloc&) {
    std::vector<PdgPassSpec>().swap(out);
    return fail(c, PDG_ERR_OOM, "no host memory for the pass list of this many steps: split the call");
  } catch (const std::length_error&) {
    std::vector<PdgPassSpec>().swap(out);
    return fail(c, PDG_ERR_OOM, "no host memory for the pass list of this many steps: split the call");
  }
}

}  // namespace pdgapi
