// Issue of the passes of a schedule: launch descriptors of the line, diagonal and corner
// passes (launch shapes, plans, coefficient uploads), their launches with optional kernel
// timing, and the CUDA-graph capture of a step sequence.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "pdg_ctx.h"

namespace pdgapi {

// Launch shape heuristic for one pass (lines per block, segments, field groups)
// with at most max_threads threads; ov (if ov[0] > 0) forces the shape.
void choose_shape(const int* ov, int max_threads, int nlines, int ncell, int ntf, int W, int* lpb, int* nseg,
                  int* ngroup) {
  if (ov && ov[0] > 0) {
    *lpb = ov[0];
    *nseg = ov[1] < ncell ? ov[1] : ncell;
    *ngroup = ov[2] < ntf ? ov[2] : ntf;
    while ((long long)(*lpb) * (*nseg) * (*ngroup) > max_threads && *nseg > 1) --(*nseg);
    while ((long long)(*lpb) * (*nseg) * (*ngroup) > max_threads && *ngroup > 1) --(*ngroup);
    while ((long long)(*lpb) * (*nseg) * (*ngroup) > max_threads && *lpb > 1) --(*lpb);
    return;
  }
  int L = 8;
  if (nlines < L) L = nlines < 1 ? 1 : nlines;
  if (L > max_threads) L = max_threads;
  int G = ntf;
  const long long target = (long long)pdg_sm_count() * 1024;
  long long s_target = (target + (long long)nlines * G - 1) / ((long long)nlines * G);
  int s_max_threads = max_threads / (L * G);
  if (s_max_threads < 1) {
    G = max_threads / L;
    if (G < 1) G = 1;
    s_max_threads = 1;
  }
  long long S = s_target;
  if (S > s_max_threads) S = s_max_threads;
  int s_win = ncell / (2 * (W > 0 ? W : 1));
  if (s_win < 1) s_win = 1;
  if (S > s_win) S = s_win;
  if (S > ncell) S = ncell;
  if (S < 1) S = 1;
  *lpb = L;
  *nseg = (int)S;
  *ngroup = G;
}

// Fill a launch descriptor for one pass of context c (shape from ov or the heuristic).
int make_pass(pdg_ctx* c, const PdgPassSpec& sp, int max_threads, const int* ov, PdgPass* out) {
  PdgPass& p = *out;
  std::memset(&p, 0, sizeof(p));
  const int axis = sp.axis;
  p.f = c->f;
  p.field_stride = c->npoints;
  const long long Px = c->P[0], Py = c->P[1], Pz = c->P[2];
  if (axis == 0) {
    p.stride = 1;
    p.lineA = Py * Pz;
    p.s1 = Px;
    p.s2 = 0;
    p.nlines = (int)(Py * Pz);
  } else if (axis == 1) {
    p.stride = Px;
    p.lineA = Px;
    p.s1 = 1;
    p.s2 = Px * Py;
    p.nlines = (int)(Px * Pz);
  } else {
    p.stride = Px * Py;
    p.lineA = Px * Py;
    p.s1 = 1;
    p.s2 = 0;
    p.nlines = (int)(Px * Py);
  }
  p.npl = c->P[axis];
  p.ncell = c->N[axis];
  const int m = c->model.m, nv = c->model.nv;
  if (c->model.kind == PDG_MODEL_ISOTHERMAL_D2Q9) {
    // populations 1 + axis (+lambda e_axis) and 3 + axis (-lambda e_axis); each is the
    // first of the three populations entering through its face
    p.ntf = 2;
    p.tfield[0] = 1 + axis;
    p.tdir[0] = +1;
    p.tfield[1] = 3 + axis;
    p.tdir[1] = -1;
    p.fbnent = 3;
    p.fbent[0] = p.fbent[1] = 0;
  } else if (c->model.kind == PDG_MODEL_ISOTHERMAL_D3Q19 || c->model.kind == PDG_MODEL_ISOTHERMAL_D3Q15 ||
             c->model.kind == PDG_MODEL_ISOTHERMAL_D3Q27) {
    // populations 1 + 2 axis (+lambda e_axis) and 2 + 2 axis (-lambda e_axis); each is the
    // first of the populations entering through its face
    p.ntf = 2;
    p.tfield[0] = 1 + 2 * axis;
    p.tdir[0] = +1;
    p.tfield[1] = 2 + 2 * axis;
    p.tdir[1] = -1;
    p.fbnent = inflow_entries(c->model);
    p.fbent[0] = p.fbent[1] = 0;
  } else {
    p.ntf = 2 * m;
    for (int k = 0; k < m; ++k) {
      p.tfield[2 * k] = k * nv + 2 * axis;
      p.tdir[2 * k] = +1;
      p.tfield[2 * k + 1] = k * nv + 2 * axis + 1;
      p.tdir[2 * k + 1] = -1;
      p.fbent[2 * k] = p.fbent[2 * k + 1] = k;
    }
    p.fbnent = m;
  }
  p.dslot = sp.dslot;
  p.nops = sp.nops;
  for (int o = 0; o < sp.nops; ++o) {
    p.op[o] = sp.op[o];
    p.opcoef[o] = sp.opcoef[o];
  }
  const int kind = pass_kind(sp);
  p.mv = kind ? pdg_model_variant(c->model) : 5 /* no collision */;
  if (kind && c->src.flags && sp.sdelta != 0.0) {
    p.src = c->src;
    p.src.kfield = c->kfield;
    p.src.delta = sp.sdelta;
    pdg_split(p.src.delta, p.src.delta_f[0]);
  }
  p.prec = c->model.prec;
  int Wmax = 1;
  for (int i = 0; i < sp.ncs; ++i) {
    int W = stable_window(sp.cs[i]);
    if (W > Wmax) Wmax = W;
  }
  choose_shape(ov, max_threads, p.nlines, p.ncell, p.ntf, Wmax, &p.lpb, &p.nseg, &p.ngroup);
  p.periodic = c->periodic[axis] ? 1 : 0;
  p.fb = c->periodic[axis] ? nullptr : c->fb[axis];
  for (int i = 0; i < sp.ncs && i < 2; ++i) {
    p.coef[i] = sp.cs[i];
    if (finish_coef(&p.coef[i], p.ncell, p.nseg, c->periodic[axis]))
      return fail(c, PDG_ERR_ARG, "singular periodic transport system (|beta| = 1)");
    if (!p.periodic && p.coef[i].rev)
      return fail(c, PDG_ERR_UNSUPPORTED, "time steps with |beta| > 1 on an inflow (non-periodic) axis");
  }
  // Two consecutive transports with the same coefficients become one composed T T
  // op when the pair recurrence can use the window closure on these segments.
  for (int o = 0; o + 1 < p.nops; ++o) {
    if (p.op[o] != PDG_OP_T || p.op[o + 1] != PDG_OP_T || p.opcoef[o] != p.opcoef[o + 1]) continue;
    PdgCoef& cf = p.coef[p.opcoef[o]];
    if (cf.rev || cf.full || !c->compose) continue;
    const int W2 = pdg_plan_compose(c->n, &cf);
    if (W2 <= 0 || W2 > p.ncell / p.nseg) continue;
    cf.W2 = W2;
    pdg_coef_split(&cf);
    p.op[o] = PDG_OP_TT;
    for (int q = o + 1; q + 1 < p.nops; ++q) {
      p.op[q] = p.op[q + 1];
      p.opcoef[q] = p.opcoef[q + 1];
    }
    p.nops -= 1;
  }
  p.model = c->model;
  return PDG_OK;
}

int launch_timed(pdg_ctx* c, const PdgPass& p, int kind) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->timing) {
    e0 = get_event(c);
    e1 = get_event(c);
    if (!e0 || !e1) return fail(c, PDG_ERR_CUDA, "cudaEventCreate failed");
    PDG_CUDA(c, cudaEventRecord(e0, c->stream));
  }
  int e = pdg_launch_pass(p, (void*)c->stream);
  if (e != 0) return cuda_fail(c, (cudaError_t)e, "pass_kernel launch");
  if (c->timing) {
    PDG_CUDA(c, cudaEventRecord(e1, c->stream));
    c->pending.push_back({kind, e0, e1});
  }
  return PDG_OK;
}

// Launch descriptor of one orientation o of a diagonal pass: the four populations whose
// velocity lies in plane (a, b) (D2Q9: 5-8 in the x-y plane; D3Q19: 7 + 4 o .. 10 + 4 o in
// plane xy, xz, yz), read from slot set dslot_in and written to the other set.  The tile
// counts minimise the swept region of one block (output cells plus the upwind start)
// times the number of blocks per SM.
int make_diag(pdg_ctx* c, const PdgPassSpec& sp, int o, PdgDiagPass* out) {
  PdgDiagPass& p = *out;
  std::memset(&p, 0, sizeof(p));
  Lattice L;
  if (!lattice_of(c->model.kind, &L)) return fail(c, PDG_ERR_ARG, "internal: diagonal pass of a DnQ2n model");
  static const int oa[3] = {0, 0, 1}, ob[3] = {1, 2, 2};
  const int ax = oa[o], ay = ob[o], az = 3 - ax - ay;   // az: the plane axis in 3-D
  const double nux = 2.0 * c->model.lambda * sp.ddelta / c->h[ax];
  const double nuy = 2.0 * c->model.lambda * sp.ddelta / c->h[ay];
  // plans are cached: the width search costs up to a few ms on the host
  const PdgDiagCoef* hit = nullptr;
  for (const auto& e : c->diag_plans)
    if (e.order == c->order && e.nux == nux && e.nuy == nuy && e.theta == c->theta) hit = &e.c;
  if (hit) {
    p.c = *hit;
  } else {
    if (pdg_plan_diag(c->order, nux, nuy, c->theta, &p.c))
      return fail(c, PDG_ERR_UNSUPPORTED,
                  "diagonal transport: no truncation width <= 128 cells for this time step (dt must be > 0)");
    if (c->diag_plans.size() >= 8) c->diag_plans.erase(c->diag_plans.begin());
    c->diag_plans.push_back({c->order, nux, nuy, c->theta, p.c});
  }
  const int in = sp.dslot_in, outs = sp.dslot_in == L.diag ? L.scratch : L.diag;
  static const int sx[4] = {+1, -1, -1, +1}, sy[4] = {+1, +1, -1, -1};   // (+,+) (-,+) (-,-) (+,-)
  p.npop = 4;
  for (int i = 0; i < 4; ++i) {
    const int pop = L.diag + 4 * o + i;   // population index (slots diag.. hold it or scratch..)
    p.fin[i] = c->f + (long long)(in + 4 * o + i) * c->npoints;
    p.fout[i] = c->f + (long long)(outs + 4 * o + i) * c->npoints;
    p.sx[i] = sx[i];
    p.sy[i] = sy[i];
    p.bxside[i] = sx[i] > 0 ? 0 : 1;
    p.byside[i] = sy[i] > 0 ? 0 : 1;
    p.bxent[i] = inflow_entry(c->model.kind, ax, pop);
    p.byent[i] = inflow_entry(c->model.kind, ay, pop);
  }
  p.perx = c->periodic[ax] ? 1 : 0;
  p.pery = c->periodic[ay] ? 1 : 0;
  p.fbx = c->periodic[ax] ? nullptr : c->fb[ax];
  p.fby = c->periodic[ay] ? nullptr : c->fb[ay];
  p.nent = inflow_entries(c->model);
  p.fbx_lines = c->npoints / c->P[ax];
  p.fby_lines = c->npoints / c->P[ay];
  p.fbx_ls = face_line_stride(c, ax, ay);
  p.fby_ls = face_line_stride(c, ay, ax);
  p.fbx_ps = c->dim == 3 ? face_line_stride(c, ax, az) : 0;
  p.fby_ps = c->dim == 3 ? face_line_stride(c, ay, az) : 0;
  p.n = c->n;
  p.ncx = c->N[ax];
  p.ncy = c->N[ay];
  const long long stride[3] = {1, c->P[0], (long long)c->P[0] * c->P[1]};
  p.sa = stride[ax];
  p.sb = stride[ay];
  p.sc = c->dim == 3 ? stride[az] : 0;
  p.nplane = c->dim == 3 ? c->P[az] : 1;
  p.prec = c->model.prec;
  // cells of at most 9 nodes (degree <= 2) carry little work between the two barriers of
  // a wavefront step: two 256-thread blocks per SM then overlap one block's barriers with
  // the other's FP64 work; larger cells keep one 512-thread block per SM
  const bool small_cells = c->n * c->n <= 9;
  p.threads = c->dshape[0] ? c->dshape[0] : (small_cells ? 256 : 512);
  const int slots = (p.threads <= 256 ? 2 : 1) * pdg_sm_count();   // blocks per wave
  const double NN = (double)c->n * c->n, NF = 2.0 * c->n - 1.0;
  double best = 1e300;
  if (c->dshape[0]) {
    p.tx = std::min(c->dshape[1], p.ncx);
    p.ty = std::min(c->dshape[2], p.ncy);
    p.ntx = (p.ncx + p.tx - 1) / p.tx;
    p.nty = (p.ncy + p.ty - 1) / p.ty;
  }
  // cost of one block: output cells, start cells at the face-node share of their work, and
  // a per-step overhead of about 8 cells (two barriers per anti-diagonal)
  for (int ntx = 1; ntx <= std::min(p.ncx, 64) && !c->dshape[0]; ++ntx) {
    const int tx = (p.ncx + ntx - 1) / ntx;
    if ((long long)tx * (ntx - 1) >= p.ncx) continue;   // the last tile would be empty
    for (int nty = 1; nty <= std::min(p.ncy, 64); ++nty) {
      const int ty = (p.ncy + nty - 1) / nty;
      if ((long long)ty * (nty - 1) >= p.ncy) continue;
      const long long blocks = 4LL * ntx * nty * p.nplane;
      const long long waves = (blocks + slots - 1) / slots;
      const double region = (double)(tx + p.c.wx) * (double)(ty + p.c.wy), out = (double)tx * ty;
      const double cost = (double)waves * (out + (region - out) * NF / NN + 8.0 * (tx + p.c.wx + ty + p.c.wy));
      if (cost < best) {
        best = cost;
        p.tx = tx;
        p.ty = ty;
        p.ntx = ntx;
        p.nty = nty;
      }
    }
  }
  if (pdg_diag_smem(p) > 200 * 1024) return fail(c, PDG_ERR_UNSUPPORTED, "diagonal tile too large");
  return PDG_OK;
}

// The hyperplane form of the corner pass (pdg_corner_hp.cuh): batch size, blocks per
// population and the face slots.  Returns 1 when planned, 0 when the form does not apply
// here (the caller plans boxes), -1 on a failed allocation (the context error is set).
int plan_corner_hyper(pdg_ctx* c, PdgCornerPass* pp) {
  PdgCornerPass& p = *pp;
  int dev = 0, coop = 0;   // cooperative launches (every GB300 has them)
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess)
    coop = 0;
  cudaGetLastError();
  if (!coop || !c->dev_err) return 0;
  const int RX = p.ncx + (p.per[0] ? p.c.wx : 0), RY = p.ncy + (p.per[1] ? p.c.wy : 0);
  const int RZ = p.ncz + (p.per[2] ? p.c.wz : 0);
  const long long NN = (long long)p.n * p.n * p.n, NF2 = ((long long)p.n * p.n + 1) & ~1LL;
  if ((long long)RY * RZ * NN >= (1LL << 30)) return 0;   // item counts of a step in 32 bits
  if (p.tc && p.n > 3) return 0;   // the tensor-core form's batches are 128 cells: degree <= 2 fits
  p.hyper = 1;
  p.threads = 512;
  p.hnb = p.tc ? 128 : (p.n == 2 ? 256 : (p.n == 3 ? 128 : 64));
  if (p.tc && pdg_corner_smem(p) > 220 * 1024) {
    p.hyper = 0;
    return 0;
  }
  while (p.hnb > 16 && pdg_corner_smem(p) > 220 * 1024) p.hnb /= 2;
  if (pdg_corner_smem(p) > 220 * 1024) {
    p.hyper = 0;
    return 0;
  }
  // blocks per population: all resident (cooperative launch), and no more than the
  // largest hyperplane has cells for (about 32 cells per block)
  long long maxcells = 0;
  for (int s = 0; s < RX + RY + RZ - 2; ++s) {
    long long n = 0;
    for (int k = 0; k < RZ; ++k) {
      const int rlo = std::max(0, s - k - (RX - 1)), rhi = std::min(RY - 1, s - k);
      if (rhi >= rlo) n += rhi - rlo + 1;
    }
    maxcells = std::max(maxcells, n);
  }
  const int per_sm = pdg_corner_hp_blocks_per_sm(p, pdg_corner_smem(p));
  if (per_sm < 1) {
    p.hyper = 0;
    return 0;
  }
  const long long resident = (long long)per_sm * pdg_sm_count();
  long long G = std::min<long long>(resident / p.npop, std::max<long long>(1, maxcells / 32));
  if (G < 1) {
    p.hyper = 0;
    return 0;
  }
  p.hg = (int)G;
  const size_t words = (size_t)p.npop * 6 * RZ * RY * NF2;
  if (words > c->czt_cap) {
    if (c->czt) cudaFree(c->czt);
    c->czt = nullptr;
    c->czt_cap = 0;
    cudaError_t e = cudaMalloc((void**)&c->czt, sizeof(double) * words);
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->czt = nullptr;
      fail(c, PDG_ERR_OOM, std::string("corner face slots: ") + cudaGetErrorString(e));
      return -1;
    }
    c->czt_cap = words;
  }
  p.hface = c->czt;
  p.hbar = reinterpret_cast<unsigned*>(c->dev_err + 16);
  return 1;
}

// Launch descriptor of the corner pass of a diagonal sub-step: the eight corner populations
// (slots diag + 4 norient ..), read from slot set dslot_in and written to the other set.
// The box counts minimise the swept volume per SM (output cells plus the upwind start,
// and a per-step overhead of about 8 cells) within the shared-memory budget.
int make_corner(pdg_ctx* c, const PdgPassSpec& sp, const Lattice& L, PdgCornerPass* out) {
  PdgCornerPass& p = *out;
  std::memset(&p, 0, sizeof(p));
  double nu[3];
  for (int a = 0; a < 3; ++a) nu[a] = 2.0 * c->model.lambda * sp.ddelta / c->h[a];
  const pdg_ctx::CornerPlan* hit = nullptr;
  for (const auto& e : c->corner_plans)
    if (e.order == c->order && e.nu[0] == nu[0] && e.nu[1] == nu[1] && e.nu[2] == nu[2] && e.theta == c->theta)
      hit = &e;
  if (!hit) {
    if (!c->cbuf) return fail(c, PDG_ERR_STATE, "internal: corner coefficients not allocated");
    pdg_ctx::CornerPlan pl;
    pl.order = c->order;
    for (int a = 0; a < 3; ++a) pl.nu[a] = nu[a];
    pl.theta = c->theta;
    std::vector<double> binv(64 * 64);
    std::vector<float> binv_f(2 * 64 * 64);
    if (pdg_plan_corner(c->order, nu[0], nu[1], nu[2], c->theta, &pl.c, binv.data(), binv_f.data()))
      return fail(c, PDG_ERR_UNSUPPORTED,
                  "corner transport: no start width <= 64 cells for this time step (dt must be > 0)");
    // reuse the oldest slot when all are taken (the stream orders the upload after the
    // launches that read the old coefficients)
    int slot = (int)c->corner_plans.size();
    if (slot >= PDG_CORNER_PLANS) {
      slot = c->corner_plans.front().slot;
      c->corner_plans.erase(c->corner_plans.begin());
    }
    pl.slot = slot;
    char* base = c->cbuf + (size_t)slot * kCornerSlotBytes;
    const size_t NN = (size_t)c->n * c->n * c->n;
    PDG_CUDA(c, cudaMemcpyAsync(base, binv.data(), sizeof(double) * NN * NN, cudaMemcpyHostToDevice, c->stream));
    PDG_CUDA(c, cudaMemcpyAsync(base + sizeof(double) * 64 * 64, binv_f.data(), sizeof(float) * 2 * NN * NN,
                                cudaMemcpyHostToDevice, c->stream));
    std::vector<float> ops(2 * 64 * 64);
    const int nops = pdg_corner_tc_operands(c->n, binv.data(), ops.data());
    PDG_CUDA(c, cudaMemcpyAsync(base + kCornerTcOffset, ops.data(), sizeof(float) * nops, cudaMemcpyHostToDevice,
                                c->stream));
    // pageable sources: the copies above return once the data are staged
    c->corner_plans.push_back(pl);
    hit = &c->corner_plans.back();
  }
  p.c = hit->c;
  const char* base = c->cbuf + (size_t)hit->slot * kCornerSlotBytes;
  p.binv = reinterpret_cast<const double*>(base);
  p.binv_f = reinterpret_cast<const float*>(base + sizeof(double) * 64 * 64);
  p.binv_tc = reinterpret_cast<const float*>(base + kCornerTcOffset);
  p.tc = c->tc;
  p.err = c->dev_err;
  p.stall = c->tc_stall;
  p.tc_layers = c->tc ? c->tc_layers : 1;
  const int in = sp.dslot_in, outs = sp.dslot_in == L.diag ? L.scratch : L.diag;
  const int c0 = 4 * L.norient;   // first corner among the moving populations
  static const int sx[8] = {+1, -1, -1, +1, +1, -1, -1, +1}, sy[8] = {+1, +1, -1, -1, +1, +1, -1, -1};
  static const int sz[8] = {+1, +1, +1, +1, -1, -1, -1, -1};
  p.npop = 8;
  for (int i = 0; i < 8; ++i) {
    p.fin[i] = c->f + (long long)(in + c0 + i) * c->npoints;
    p.fout[i] = c->f + (long long)(outs + c0 + i) * c->npoints;
    p.sx[i] = sx[i];
    p.sy[i] = sy[i];
    p.sz[i] = sz[i];
  }
  p.n = c->n;
  p.ncx = c->N[0];
  p.ncy = c->N[1];
  p.ncz = c->N[2];
  p.sa = 1;
  p.sb = c->P[0];
  p.sc = (long long)c->P[0] * c->P[1];
  p.nent = inflow_entries(c->model);
  const int* sgn[3] = {sx, sy, sz};
  for (int a = 0; a < 3; ++a) {
    p.per[a] = c->periodic[a] ? 1 : 0;
    p.fb[a] = c->periodic[a] ? nullptr : c->fb[a];
    p.flines[a] = c->npoints / c->P[a];
    for (int b = 0; b < 3; ++b) p.fls[a][b] = b == a ? 0 : face_line_stride(c, a, b);
    for (int i = 0; i < 8; ++i) {
      p.bside[a][i] = sgn[a][i] > 0 ? 0 : 1;
      p.bent[a][i] = inflow_entry(c->model.kind, a, L.diag + c0 + i);
    }
  }
  p.prec = c->model.prec;
  p.threads = c->cshape[0] && !p.tc ? c->cshape[0] : 512;   // the tensor-core kernel runs 16 warps
  // hyperplane sweep of the whole region (default; not for forced box shapes), when its
  // tables fit shared memory and its blocks can all be resident
  if (c->corner_sweep && !c->cshape[1]) {
    int r = plan_corner_hyper(c, &p);
    if (r < 0) return fail(c, PDG_ERR_UNSUPPORTED, "internal: corner hyperplane plan");
    if (r == 1) return PDG_OK;
  }
  if (c->cshape[1]) {
    p.tx = std::min(c->cshape[1], p.ncx);
    p.ty = std::min(c->cshape[2], p.ncy);
    p.tz = std::min(c->cshape[3], p.ncz);
    p.ntx = (p.ncx + p.tx - 1) / p.tx;
    p.nty = (p.ncy + p.ty - 1) / p.ty;
    p.ntz = (p.ncz + p.tz - 1) / p.tz;
  } else {
    // cost of one block in node dot products: output cells (all NN nodes) and start cells
    // (NFF face nodes) of every layer, plus about 4 cells of overhead per wavefront step;
    // one block per SM (512 threads at ~86 registers)
    const double NN = (double)c->n * c->n * c->n, NFF = NN - (double)(c->n - 1) * (c->n - 1) * (c->n - 1);
    double best = 1e300;
    auto tiles = [](int N, int cap) {   // candidate (count, size) pairs with a non-empty last box
      std::vector<std::pair<int, int>> v;
      for (int k = 1; k <= std::min(N, cap); ++k) {
        const int t = (N + k - 1) / k;
        if ((long long)t * (k - 1) >= N) continue;
        if (!v.empty() && v.back().second == t) continue;
        v.push_back({k, t});
      }
      return v;
    };
    const auto TX = tiles(p.ncx, 64), TY = tiles(p.ncy, 64), TZ = tiles(p.ncz, 64);
    const long long sms = pdg_sm_count();   // one block per SM
    for (auto [ntx, tx] : TX)
      for (auto [nty, ty] : TY)
        for (auto [ntz, tz] : TZ) {
          PdgCornerPass q = p;
          q.tx = tx;
          q.ty = ty;
          q.tz = tz;
          if (p.tc && q.tc_layers * std::min(tx + p.c.wx, ty + p.c.wy) > 128) q.tc_layers = 1;
          if (pdg_corner_smem(q) > 200 * 1024) continue;
          if (p.tc && std::min(tx + p.c.wx, ty + p.c.wy) > 128) continue;
          const long long blocks = 8LL * ntx * nty * ntz;
          const long long waves = (blocks + sms - 1) / sms;
          const double region = (double)(tx + p.c.wx) * (double)(ty + p.c.wy), out = (double)tx * ty;
          const double steps = (double)(tx + p.c.wx + ty + p.c.wy);
          // tensor-core kernel: every cell of the region forms all its nodes and the full
          // residual (start cells included), and a step carries six barriers and two MMA waits
          const double work = p.tc ? (double)(tz + p.c.wz) * (region * NN + 16.0 * NN * steps / q.tc_layers)
                                   : tz * (out * NN + (region - out) * NFF) + p.c.wz * region * NFF +
                                         (double)(tz + p.c.wz) * 4.0 * NN * steps;
          const double cost = (double)waves * work;
          if (cost < best) {
            best = cost;
            p.tx = tx;
            p.ty = ty;
            p.tz = tz;
            p.ntx = ntx;
            p.nty = nty;
            p.ntz = ntz;
            p.tc_layers = q.tc_layers;
          }
        }
    if (best == 1e300) return fail(c, PDG_ERR_UNSUPPORTED, "corner box too large for shared memory");
  }
  if (p.tc && p.tc_layers * std::min(p.tx + p.c.wx, p.ty + p.c.wy) > 128) p.tc_layers = 1;
  if (p.tc && pdg_corner_smem(p) > 200 * 1024) p.tc_layers = 1;
  if (pdg_corner_smem(p) > 200 * 1024) return fail(c, PDG_ERR_UNSUPPORTED, "corner box too large");
  if (p.threads < 64 || p.threads > 512) return fail(c, PDG_ERR_ARG, "corner pass: threads per block");
  if (p.tc && std::min(p.tx + p.c.wx, p.ty + p.c.wy) > 128)
    return fail(c, PDG_ERR_UNSUPPORTED, "tensor-core corner pass: more than 128 cells on an anti-diagonal");
  // +z face scratch of the launch (grown on demand; cudaFree waits for the device)
  const size_t words = pdg_corner_scratch(p);
  if (words > c->czt_cap) {
    if (c->czt) cudaFree(c->czt);
    c->czt = nullptr;
    c->czt_cap = 0;
    cudaError_t e = cudaMalloc((void**)&c->czt, sizeof(double) * words);
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->czt = nullptr;
      return fail(c, PDG_ERR_OOM, std::string("corner face scratch: ") + cudaGetErrorString(e));
    }
    c->czt_cap = words;
  }
  p.zt = c->czt;
  return PDG_OK;
}

// The diagonal launches of one sub-step (the corner pass first, then the edge planes) act
// on disjoint populations.  With more than one, they fork from the context stream onto
// the context's auxiliary streams and join back, so the last partial wave of one overlaps
// the next (events only: a graph capture records them as parallel branches).  Their
// descriptors, and the corner plans' uploads on the context stream, come before the fork.
int issue_diag(pdg_ctx* c, const PdgPassSpec& sp) {
  Lattice L;
  if (!lattice_of(c->model.kind, &L)) return fail(c, PDG_ERR_ARG, "internal: diagonal pass of a DnQ2n model");
  PdgCornerPass cp;
  PdgDiagPass dp[3];
  if (L.ncorner)
    if (int r = make_corner(c, sp, L, &cp)) return r;
  for (int o = 0; o < L.norient; ++o)
    if (int r = make_diag(c, sp, o, &dp[o])) return r;
  const int nl = L.norient + (L.ncorner ? 1 : 0);
  const bool fork = nl > 1;
  if (fork) {
    for (int i = 0; i < nl; ++i) {
      if (!c->dstream[i]) PDG_CUDA(c, cudaStreamCreateWithFlags(&c->dstream[i], cudaStreamNonBlocking));
      if (!c->djoin[i]) PDG_CUDA(c, cudaEventCreateWithFlags(&c->djoin[i], cudaEventDisableTiming));
    }
    if (!c->dfork) PDG_CUDA(c, cudaEventCreateWithFlags(&c->dfork, cudaEventDisableTiming));
    PDG_CUDA(c, cudaEventRecord(c->dfork, c->stream));
    for (int i = 0; i < nl; ++i) PDG_CUDA(c, cudaStreamWaitEvent(c->dstream[i], c->dfork, 0));
  }
  for (int i = 0; i < nl; ++i) {
    const bool corner = L.ncorner && i == 0;
    cudaStream_t st = fork ? c->dstream[i] : c->stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->timing) {
      e0 = get_event(c);
      e1 = get_event(c);
      if (!e0 || !e1) return fail(c, PDG_ERR_CUDA, "cudaEventCreate failed");
      PDG_CUDA(c, cudaEventRecord(e0, st));
    }
    const int e = corner ? pdg_launch_corner(cp, (void*)st) : pdg_launch_diag(dp[i - (L.ncorner ? 1 : 0)], (void*)st);
    if (e != 0) return cuda_fail(c, (cudaError_t)e, corner ? "corner_kernel launch" : "diag_kernel launch");
    if (c->timing) {
      PDG_CUDA(c, cudaEventRecord(e1, st));
      c->pending.push_back({corner ? 4 : 3, e0, e1});
    }
  }
  if (fork)
    for (int i = 0; i < nl; ++i) {
      PDG_CUDA(c, cudaEventRecord(c->djoin[i], c->dstream[i]));
      PDG_CUDA(c, cudaStreamWaitEvent(c->stream, c->djoin[i], 0));
    }
  return PDG_OK;
}

// Single-mesh launch shape: when ceil(nlines / lpb) blocks would leave more than 5 % of
// the SMs idle in their last round, the block count is rounded up to a multiple of the
// SM count, the lines are spread evenly over the blocks, and lpb shrinks to the largest
// share, so that every SM gets the same number of lines and few thread slots stay idle.
void balance_blocks(PdgPass* p) {
  const int sms = pdg_sm_count();
  const int nb0 = (p->nlines + p->lpb - 1) / p->lpb;
  // keep the plain split (aligned line groups) when the last round of blocks already
  // keeps 95 % of the SMs busy
  const long long rounds = ((long long)nb0 + sms - 1) / sms;
  if (nb0 < sms / 2 || (double)nb0 >= 0.95 * (double)(rounds * sms)) {
    p->nblocks = nb0;
    return;
  }
  const long long nb = std::min<long long>(((long long)nb0 + sms - 1) / sms * sms, p->nlines);
  p->nblocks = (int)nb;
  p->lpb = (int)(((long long)p->nlines + nb - 1) / nb);
}

// Launch shape of the line-resident kernel (pass_resident_kernel) for a line pass, or false
// when the pass runs the streaming kernel: the option is off, the axis has inflow faces,
// the model is a lattice or has a source stage, or the staged lines of one block would
// not fit in shared memory.  Shape: the kind's override (launch kinds 7 / 8) or one line
// per block on unit-stride lines (two when they stay under ~110 KB, two blocks per SM) and
// four adjacent lines on strided ones (32-byte runs of the fastest axis; fewer when the
// staged lines pass ~220 KB), segments of about eight cells (never shorter than the
// transport window), all transported fields in flight, at most 512 threads.
bool resident_shape(const pdg_ctx* c, const PdgPassSpec& sp, int kind, int* shape) {
  Lattice Lat;
  if (!c->resident || sp.axis < 0 || !c->periodic[sp.axis] || c->src.flags || lattice_of(c->model.kind, &Lat))
    return false;
  const int axis = sp.axis, npl = c->P[axis], ncell = c->N[axis], ntf = 2 * c->model.m;
  const size_t nload = kind ? (size_t)c->model.nf : (size_t)ntf;
  int W = 1;
  for (int i = 0; i < sp.ncs; ++i) W = std::max(W, stable_window(sp.cs[i]));
  auto smem = [&](int lpb, int nseg) {
    return sizeof(double) * (nload * (size_t)lpb * (size_t)pdg_resident_ls(npl) + 3 * (size_t)ntf * nseg * lpb);
  };
  const size_t cap = 220 * 1024;
  int lpb, nseg, ngroup;
  const int* ov = c->rshape[kind];
  if (ov[0] > 0) {
    lpb = ov[0];
    nseg = std::min(ov[1], ncell);
    ngroup = std::min(ov[2], ntf);
  } else {
    nseg = std::max(1, ncell / 8);
    if (ncell / nseg < W) nseg = std::max(1, ncell / W);
    ngroup = ntf;
    if (axis == 0) {
      lpb = smem(2, nseg) <= 110 * 1024 ? 2 : 1;
    } else {
      lpb = 4;
      while (lpb > 1 && smem(lpb, nseg) > cap) lpb /= 2;
    }
    while (lpb * nseg * ngroup > 512 && ngroup > 1) {
      int g = ngroup - 1;
      while (g > 1 && ntf % g) --g;
      ngroup = g;
    }
    while (lpb * nseg * ngroup > 512 && nseg > 1) nseg = (nseg + 1) / 2;
  }
  if (lpb < 1 || nseg < 1 || ngroup < 1 || lpb * nseg * ngroup > 512 || smem(lpb, nseg) > cap) return false;
  if (axis > 0 && lpb < 2 && ov[0] <= 0) return false;   // strided lines: at least 16-byte runs
  shape[0] = lpb;
  shape[1] = nseg;
  shape[2] = ngroup;
  return true;
}

int issue_pass(pdg_ctx* c, const PdgPassSpec& sp) {
  if (sp.axis == -2) {
    Lattice L;
    if (!lattice_of(c->model.kind, &L)) return fail(c, PDG_ERR_ARG, "internal: copy of a DnQ2n model");
    PDG_CUDA(c, cudaMemcpyAsync(c->f + (long long)L.diag * c->npoints, c->f + (long long)L.scratch * c->npoints,
                                sizeof(double) * L.ndiag * (size_t)c->npoints, cudaMemcpyDeviceToDevice,
                                c->stream));
    return PDG_OK;
  }
  if (sp.axis < 0) return issue_diag(c, sp);
  PdgPass p;
  const int kind = pass_kind(sp);
  int rs[3];
  if (resident_shape(c, sp, kind, rs)) {
    if (int r = make_pass(c, sp, 512, rs, &p)) return r;
    p.resident = 1;
  } else {
    if (int r = make_pass(c, sp, 512, c->launch[kind], &p)) return r;
  }
  balance_blocks(&p);
  return launch_timed(c, p, kind);
}

// Capture the passes of (dt, nsteps) into a CUDA graph on the private stream.  Plans,
// coefficient uploads and scratch allocations happen first, outside the capture (the
// corner passes' plans are made by a dry make_corner), so the graph holds launches and
// device-to-device copies only.
int capture_steps(pdg_ctx* c, double dt, int nsteps, const std::vector<PdgPassSpec>& sched) {
  Lattice L;
  if (lattice_of(c->model.kind, &L) && L.ncorner)
    for (const auto& sp : sched)
      if (sp.axis == -1) {
        PdgCornerPass p;
        if (int r = make_corner(c, sp, L, &p)) return r;
      }
  if (!c->gstream) PDG_CUDA(c, cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
  if (!c->g_in) PDG_CUDA(c, cudaEventCreateWithFlags(&c->g_in, cudaEventDisableTiming));
  if (!c->g_out) PDG_CUDA(c, cudaEventCreateWithFlags(&c->g_out, cudaEventDisableTiming));
  if (c->gexec) {
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  // (the corner uploads above went to the context stream, which every replay waits for)
  PDG_CUDA(c, cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal));
  cudaStream_t user = c->stream;
  c->stream = c->gstream;
  int r = PDG_OK;
  for (const auto& sp : sched)
    if ((r = issue_pass(c, sp)) != PDG_OK) break;
  c->stream = user;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->gstream, &g);
  if (r != PDG_OK) {
    if (g) cudaGraphDestroy(g);
    return r;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&c->gexec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    c->gexec = nullptr;
    return cuda_fail(c, e, "graph capture of pdg_step");
  }
  c->g_dt = dt;
  c->g_nsteps = nsteps;
  c->g_gen = c->gen;
  return PDG_OK;
}

}  // namespace pdgapi
