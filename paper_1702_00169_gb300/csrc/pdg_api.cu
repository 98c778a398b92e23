// C ABI of the PDG solver: context, device state, and the pass schedule of the
// palindromic step.
//
// Schedule.  M2(dt) = T(dt/2) C(dt) T(dt/2) (Section 3.2) with T the product of
// the per-population transports; transports along different axes act on
// different populations, so they commute exactly.  For D axes with last axis L,
// nsteps steps are issued as
//   for a < L: pass_a [T(dt/2)]
//   repeat nsteps:  pass_L [T(dt/2), C, T(dt/2)]
//                   for a < L: pass_a [T(dt/2), T(dt/2)]   (last step: [T(dt/2)])
// which applies to every population exactly the sequence of the naive order.
// The collapsed scheme of Section 5.1 merges interior half steps into T(dt).
#include <cuda_runtime.h>

#include <atomic>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/pdg.h"
#include "pdg_internal.h"

struct PdgTimedLaunch {
  int kind;
  cudaEvent_t e0, e1;
};

struct pdg_ctx {
  int dim = 0, order = 0, n = 0;
  int nmacro[3] = {1, 1, 1}, nsub[3] = {1, 1, 1}, N[3] = {1, 1, 1}, P[3] = {1, 1, 1};
  double len[3] = {1, 1, 1}, h[3] = {1, 1, 1};
  long long npoints = 0;
  cudaStream_t stream = nullptr;
  bool has_model = false;
  PdgModel model{};
  int scheme = 0, precision = 0;
  double theta = 0.5;
  double* f = nullptr;
  long long f_cap = 0;
  bool has_state = false;
  double* wstage = nullptr;
  long long wstage_cap = 0;
  bool periodic[3] = {true, true, true};
  double* fb[3] = {nullptr, nullptr, nullptr};  // inflow data per non-periodic axis: [2][m][lines]
  bool async_alloc = false;   // state from the stream-ordered pool (cudaMallocAsync / cudaFreeAsync)
  bool compose = true;        // compose consecutive equal transports into one T T sweep
  int launch[2][3] = {{0, 0, 0}, {0, 0, 0}};   // single-mesh shape overrides per pass kind
  int bshape[2][3] = {{0, 0, 0}, {0, 0, 0}};   // shapes inside batched launches (<= 256 threads)
  int dshape[3] = {0, 0, 0};                   // D2Q9 diagonal pass: threads, tile x, tile y
  PdgSrc src{};                                // source stage (flags 0 = none); delta set per pass
  struct DiagPlan {
    int order;
    double nux, nuy, theta;
    PdgDiagCoef c;
  };
  std::vector<DiagPlan> diag_plans;            // planned diagonal sub-steps (a few sizes per run)
  // corner sub-steps (D3Q15 / D3Q27): host plans and their B^-1 in cbuf (device memory
  // allocated by pdg_set_model, PDG_CORNER_PLANS slots of FP64 and double-float copies)
  struct CornerPlan {
    int order;
    double nu[3], theta;
    PdgCornerCoef c;
    int slot;
  };
  std::vector<CornerPlan> corner_plans;
  char* cbuf = nullptr;
  int tc = 0;                                  // corner cell inverse on the tensor cores: 0 off,
                                               // 1 FP64 residual, 2 double-float residual
  int* dev_err = nullptr;                      // error word of the tensor-core kernel (in cbuf)
  int tc_stall = 0;                            // PDG_OPT_DEBUG_TC_STALL
  double* czt = nullptr;                       // corner pass: per-block +z face scratch
  // CUDA-graph replay of pdg_step (PDG_OPT_GRAPH): the captured step sequence, its key
  // (dt, nsteps, configuration generation) and the private capture / replay stream
  bool use_graph = false;
  unsigned long long gen = 0;                  // bumped by every call that changes the passes
  cudaStream_t gstream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  double g_dt = 0.0;
  int g_nsteps = -1;
  unsigned long long g_gen = ~0ULL;
  cudaEvent_t g_in = nullptr, g_out = nullptr;
  // auxiliary streams of the diagonal launches of a 3-D lattice sub-step (issue_diag)
  cudaStream_t dstream[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t dfork = nullptr, djoin[4] = {nullptr, nullptr, nullptr, nullptr};
  size_t czt_cap = 0;                          // its capacity (8-byte words)
  int cshape[4] = {0, 0, 0, 0};                // corner pass: threads, box x, y, z (0 = heuristic)
  double* kfield = nullptr;                    // penalisation K at every point
  bool timing = false;
  long long t_launches[5] = {0, 0, 0, 0, 0};   // per kind: 0 line, 1 line + C, 2 state, 3 diag, 4 corner
  double t_ms[5] = {0, 0, 0, 0, 0};
  std::vector<PdgTimedLaunch> pending;
  std::vector<cudaEvent_t> event_pool;
  std::string err;
};

struct pdg_batch {
  std::vector<pdg_ctx*> inst;
  cudaStream_t stream = nullptr;       // the caller's stream (may be the legacy default stream)
  cudaStream_t cap = nullptr;          // private blocking stream used for graph capture and replay
  size_t smem = 0;
  // device tables of the last pdg_batch_step (kept alive for the captured graph)
  PdgPass* d_desc = nullptr;
  int* d_ent_desc = nullptr;
  long long* d_ent_start = nullptr;
  unsigned long long* d_counter = nullptr;
  size_t cap_desc = 0, cap_ent = 0, cap_es = 0, cap_cnt = 0;
  bool realloc = false;                // a table moved: the cached graph must be recaptured
  // per launch (one per stage and (precision, degree, model) group present): first entry,
  // entries, work items, group
  std::vector<int> st_off, st_nent, st_prec, st_np, st_mv;
  std::vector<long long> st_total;
  std::vector<char> sig;                      // signature of the tables (graph cache key)
  cudaGraphExec_t gexec = nullptr;
  std::vector<char> gsig;
  cudaEvent_t e0 = nullptr, e1 = nullptr, ej = nullptr;
  long long last_launches = 0;
  std::string err;
};

namespace {

int fail(pdg_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(pdg_ctx* c, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(c, PDG_ERR_CUDA, m);
}

#define PDG_CUDA(ctx, call)                                   \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call); \
  } while (0)

// After a synchronisation of the context stream: a bounded wait of the tensor-core corner
// kernel that ran out (its error word set) is reported once as PDG_ERR_TIMEOUT, and the
// word is cleared.  The state of the steps in flight then is incomplete.
int check_device_error(pdg_ctx* c) {
  if (!c->dev_err || !c->tc) return 0;
  int v = 0;
  PDG_CUDA(c, cudaMemcpyAsync(&v, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  PDG_CUDA(c, cudaStreamSynchronize(c->stream));
  if (!v) return 0;
  PDG_CUDA(c, cudaMemsetAsync(c->dev_err, 0, sizeof(int), c->stream));
  PDG_CUDA(c, cudaStreamSynchronize(c->stream));
  return fail(c, PDG_ERR_TIMEOUT,
              "tensor-core corner pass: a bounded wait for the tensor cores ran out; the state is incomplete");
}

cudaEvent_t get_event(pdg_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Drain pending timed launches into the counters (requires completed events).
int drain_timing(pdg_ctx* c) {
  for (auto& t : c->pending) {
    float ms = 0.f;
    cudaError_t e = cudaEventElapsedTime(&ms, t.e0, t.e1);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventElapsedTime");
    c->t_launches[t.kind] += 1;
    c->t_ms[t.kind] += ms;
    c->event_pool.push_back(t.e0);
    c->event_pool.push_back(t.e1);
  }
  c->pending.clear();
  return PDG_OK;
}

// Lattice models (one set of populations for all variables): D2Q9, D3Q19, D3Q15, D3Q27.
// Their non-axis populations [diag, diag + ndiag) run in diagonal passes, out of place
// between slots diag.. and scratch..: first norient planes of four edge velocities (a, b),
// then ncorner corner velocities.
struct Lattice {
  int slots, diag, scratch, ndiag, norient, ncorner;
};
bool lattice_of(int kind, Lattice* L) {
  if (kind == PDG_MODEL_ISOTHERMAL_D2Q9) {
    *L = {PDG_Q9_SLOTS, PDG_Q9_DIAG, PDG_Q9_SCRATCH, 4, 1, 0};
    return true;
  }
  if (kind == PDG_MODEL_ISOTHERMAL_D3Q19) {
    *L = {PDG_Q19_SLOTS, PDG_Q19_DIAG, PDG_Q19_SCRATCH, 12, 3, 0};
    return true;
  }
  if (kind == PDG_MODEL_ISOTHERMAL_D3Q15) {
    *L = {PDG_Q15_SLOTS, PDG_Q15_DIAG, PDG_Q15_SCRATCH, 8, 0, 8};
    return true;
  }
  if (kind == PDG_MODEL_ISOTHERMAL_D3Q27) {
    *L = {PDG_Q27_SLOTS, PDG_Q27_DIAG, PDG_Q27_SCRATCH, 20, 3, 8};
    return true;
  }
  return false;
}

// Unit velocities xi_i of the lattice models in population order (the orders of pdg.h):
// components (x, y, z); nullptr for the DnQ2n models.
struct LatticeTables {
  int q9[9][3], q19[19][3], q15[15][3], q27[27][3];
};
LatticeTables make_lattice_tables() {
  LatticeTables t{};
  // rest, +-x, +-y, +-z; edges by plane xy, xz, yz; corners z = +1 then z = -1
  const int q9[9][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
                        {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
  const int axis[7][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
  const int sa[4] = {1, -1, -1, 1}, sb[4] = {1, 1, -1, -1};
  const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
  int edge[12][3] = {}, corner[8][3] = {};
  for (int o = 0; o < 3; ++o)
    for (int k = 0; k < 4; ++k) {
      edge[4 * o + k][pa[o]] = sa[k];
      edge[4 * o + k][pb[o]] = sb[k];
    }
  for (int h = 0; h < 2; ++h)
    for (int k = 0; k < 4; ++k) {
      corner[4 * h + k][0] = sa[k];
      corner[4 * h + k][1] = sb[k];
      corner[4 * h + k][2] = h == 0 ? 1 : -1;
    }
  for (int i = 0; i < 9; ++i)
    for (int a = 0; a < 3; ++a) t.q9[i][a] = q9[i][a];
  for (int i = 0; i < 7; ++i)
    for (int a = 0; a < 3; ++a) t.q19[i][a] = t.q15[i][a] = t.q27[i][a] = axis[i][a];
  for (int i = 0; i < 12; ++i)
    for (int a = 0; a < 3; ++a) t.q19[7 + i][a] = t.q27[7 + i][a] = edge[i][a];
  for (int i = 0; i < 8; ++i)
    for (int a = 0; a < 3; ++a) {
      t.q15[7 + i][a] = corner[i][a];
      t.q27[19 + i][a] = corner[i][a];
    }
  return t;
}

// Unit velocities xi_i of the lattice models in population order (the orders of pdg.h):
// components (x, y, z); nullptr for the DnQ2n models.
const int* lattice_xi(int kind, int* q) {
  static const LatticeTables t = make_lattice_tables();
  switch (kind) {
    case PDG_MODEL_ISOTHERMAL_D2Q9: *q = 9; return &t.q9[0][0];
    case PDG_MODEL_ISOTHERMAL_D3Q19: *q = 19; return &t.q19[0][0];
    case PDG_MODEL_ISOTHERMAL_D3Q15: *q = 15; return &t.q15[0][0];
    case PDG_MODEL_ISOTHERMAL_D3Q27: *q = 27; return &t.q27[0][0];
  }
  *q = 0;
  return nullptr;
}

// Inflow data entries per face side: the conserved variables of a DnQ2n model (its +-e_a
// population of each variable), or for a lattice the populations entering through the face.
int inflow_entries(const PdgModel& m) {
  int q = 0;
  const int* xi = lattice_xi(m.kind, &q);
  if (!xi) return m.m;
  int n = 0;
  for (int i = 0; i < q; ++i) n += xi[3 * i] > 0;
  return n;
}

// Entry of lattice population i in the data of the face normal to `axis` that it enters
// through (low face for xi_axis > 0, high face for < 0): its rank among the populations
// entering through that face, in population order.
int inflow_entry(int kind, int axis, int i) {
  int q = 0;
  const int* xi = lattice_xi(kind, &q);
  const int s = xi[3 * i + axis];
  int e = 0;
  for (int j = 0; j < i; ++j) e += xi[3 * j + axis] == s;
  return e;
}

// Stride, in the line index of the face normal to axis A (C order over the other axes, x
// fastest), of the point coordinate along axis b != A.
long long face_line_stride(const pdg_ctx* c, int A, int b) {
  long long st = 1;
  for (int a = 0; a < b; ++a)
    if (a != A) st *= c->P[a];
  return st;
}

// Corner coefficient slots in pdg_ctx::cbuf: FP64 B^-1 (64 x 64 at most), its
// double-float copy, then its two TF32 operands of the tensor-core kernel, per slot; after
// the slots, the tensor-core kernel's error word.
#define PDG_CORNER_PLANS 4
constexpr size_t kCornerSlotBytes = 64 * 64 * (sizeof(double) + 2 * sizeof(float) + 2 * sizeof(float));
constexpr size_t kCornerTcOffset = 64 * 64 * (sizeof(double) + 2 * sizeof(float));
constexpr size_t kCornerErrBytes = 256;

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

// Fill the launch-dependent fields of a coefficient set for segments of a line of
// N cells.  Returns 0, or -1 when the periodic system is singular (|beta| = 1 with
// beta^N = 1).
int finish_coef(PdgCoef* C, int N, int S, bool periodic = true) {
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
          if (pdg_corner_smem(q) > 200 * 1024) continue;
          if (p.tc && std::min(tx + p.c.wx, ty + p.c.wy) > 128) continue;
          const long long blocks = 8LL * ntx * nty * ntz;
          const long long waves = (blocks + sms - 1) / sms;
          const double region = (double)(tx + p.c.wx) * (double)(ty + p.c.wy), out = (double)tx * ty;
          const double steps = (double)(tx + p.c.wx + ty + p.c.wy);
          // tensor-core kernel: every cell of the region forms all its nodes and the full
          // residual (start cells included), and a step carries six barriers and two MMA waits
          const double work = p.tc ? (double)(tz + p.c.wz) * (region * NN + 16.0 * NN * steps)
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
          }
        }
    if (best == 1e300) return fail(c, PDG_ERR_UNSUPPORTED, "corner box too large for shared memory");
  }
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
  if (int r = make_pass(c, sp, 512, c->launch[kind], &p)) return r;
  balance_blocks(&p);
  return launch_timed(c, p, kind);
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

// The line passes of nsteps palindromic steps (see the schedule at the top of this file).
int build_line_schedule(pdg_ctx* c, double dt, int nsteps, std::vector<PdgPassSpec>& out) {
  out.clear();
  if (nsteps <= 0) return PDG_OK;
  const int D = c->dim, L = D - 1;
  out.reserve((2 * (size_t)nsteps + 1) * (size_t)D);   // at least the passes of every scheme
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
  const int o1[1] = {T}, o2[2] = {T, T}, o3[3] = {T, C, T};
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
    const int nseg = 2 * nsteps + 1;
    // segment j: number of sub-steps and their coefficient index (0 = quarter, 1 = half)
    auto seg_n = [&](int j) { return (j == 0 || j == nseg - 1) ? 1 : ((j % 2 == 1) ? 1 : 2); };
    auto seg_ci = [&](int j) { return (j % 2 == 1) ? 1 : 0; };
    auto other_axes = [&](int j) {
      for (int a = 0; a < L; ++a) {
        PdgCoef cs[2] = {qc[a], hc[a]};
        const int ops[2] = {T, T}, ci[2] = {seg_ci(j), seg_ci(j)};
        out.push_back(spec(a, seg_n(j), ops, ci, cs, 2));
      }
    };
    PdgCoef csL[2] = {qc[L], hc[L]};
    other_axes(0);
    {
      const int ops[3] = {T, C, T}, ci[3] = {seg_ci(0), 0, seg_ci(1)};
      out.push_back(spec(L, 3, ops, ci, csL, 2));
    }
    for (int j = 1; j < nseg - 1; ++j) {
      other_axes(j);
      int ops[3] = {C, T, T}, ci[3] = {0, seg_ci(j + 1), seg_ci(j + 1)};
      out.push_back(spec(L, 1 + seg_n(j + 1), ops, ci, csL, 2));
    }
    other_axes(nseg - 1);
    return PDG_OK;
  }
  if (c->scheme == PDG_SCHEME_M2) {
    for (int a = 0; a < L; ++a) out.push_back(spec(a, 1, o1, z1, &half[a], 1));
    for (int s = 0; s < nsteps; ++s) {
      out.push_back(spec(L, 3, o3, z3, &half[L], 1));
      for (int a = 0; a < L; ++a) out.push_back(spec(a, s < nsteps - 1 ? 2 : 1, o2, z2, &half[a], 1));
    }
  } else {
    for (int a = 0; a < L; ++a) out.push_back(spec(a, 1, o1, z1, &half[a], 1));
    for (int s = 0; s < nsteps; ++s) {
      PdgCoef cs[2] = {half[L], full[L]};
      const int ops[2] = {T, C}, ci[2] = {s == 0 ? 0 : 1, 0};
      out.push_back(spec(L, 2, ops, ci, cs, 2));
      for (int a = 0; a < L; ++a) out.push_back(spec(a, 1, o1, z1, s < nsteps - 1 ? &full[a] : &half[a], 1));
    }
    out.push_back(spec(L, 1, o1, z1, &half[L], 1));
  }
  return PDG_OK;
}

// The full pass list.  D2Q9 adds the diagonal transports: the sub-steps between two
// collisions (and before the first / after the last) run as diagonal passes issued
// just before the line pass that holds the next collision (transports of different
// populations commute); each diagonal pass swaps the slot set of populations 5-8, the
// collision reads them where they are, and a final copy returns them to slots 5-8.
int build_schedule_one(pdg_ctx* c, double dt, int nsteps, std::vector<PdgPassSpec>& out) {
  if (int r = build_line_schedule(c, dt, nsteps, out)) return r;
  Lattice Lat;
  if (!lattice_of(c->model.kind, &Lat) || nsteps <= 0) return PDG_OK;
  if (!(dt > 0.0)) return fail(c, PDG_ERR_UNSUPPORTED, "diagonal transport needs dt > 0");
  if (c->src.flags && c->scheme == PDG_SCHEME_M2KIN)
    return fail(c, PDG_ERR_UNSUPPORTED, "sources are defined for M2 and M2_collapsed");
  // diagonal sub-steps of each transport segment, in order
  std::vector<std::vector<double>> seg;
  const double h = 0.5 * dt, q = 0.25 * dt;
  if (c->scheme == PDG_SCHEME_M2) {
    seg.push_back({h});
    for (int s = 1; s < nsteps; ++s) seg.push_back({h, h});
    seg.push_back({h});
  } else if (c->scheme == PDG_SCHEME_M2_COLLAPSED) {
    seg.push_back({h});
    for (int s = 1; s < nsteps; ++s) seg.push_back({dt});
    seg.push_back({h});
  } else {
    seg.push_back({q});
    for (int s = 0; s < nsteps; ++s) {
      seg.push_back({h});
      if (s < nsteps - 1) seg.push_back({q, q});
    }
    seg.push_back({q});
  }
  std::vector<PdgPassSpec> res;
  res.reserve(out.size() + 3 * seg.size() + 1);
  int slot = Lat.diag;
  size_t ci = 0;
  auto diag = [&](double delta) {
    PdgPassSpec d;
    std::memset(&d, 0, sizeof(d));
    d.axis = -1;
    d.ddelta = delta;
    d.dslot_in = slot;
    res.push_back(d);
    slot = (slot == Lat.diag) ? Lat.scratch : Lat.diag;
  };
  for (auto sp : out) {
    if (pass_kind(sp)) {
      if (ci >= seg.size()) return fail(c, PDG_ERR_ARG, "internal: schedule segments");
      for (double dl : seg[ci]) diag(dl);
      ++ci;
      sp.dslot = slot;
      sp.sdelta = c->src.flags ? 0.5 * dt : 0.0;   // S(dt/2) C(dt) S(dt/2)
    }
    res.push_back(sp);
  }
  if (ci + 1 != seg.size()) return fail(c, PDG_ERR_ARG, "internal: schedule segments");
  for (double dl : seg[ci]) diag(dl);
  if (slot != Lat.diag) {
    PdgPassSpec cp;
    std::memset(&cp, 0, sizeof(cp));
    cp.axis = -2;   // copy slots 9-12 back to 5-8
    res.push_back(cp);
  }
  out.swap(res);
  return PDG_OK;
}

// The pass list of nsteps steps of the context's scheme.  M4^kin (PDG_SCHEME_M4KIN) is the
// triple jump M2^kin(g1 dt) M2^kin(g2 dt) M2^kin(g1 dt) per step (Section 3.2: palindromic
// compositions of M2^kin; H. Yoshida, Phys. Lett. A 150 (1990)), g1 = 1/(2 - 2^(1/3)),
// g2 = 1 - 2 g1 < 0: three M2^kin schedules per step, the middle one backwards in time.
int build_schedule(pdg_ctx* c, double dt, int nsteps, std::vector<PdgPassSpec>& out) {
  if (c->scheme != PDG_SCHEME_M4KIN) return build_schedule_one(c, dt, nsteps, out);
  Lattice L;
  if (lattice_of(c->model.kind, &L))
    return fail(c, PDG_ERR_UNSUPPORTED, "M4^kin has a backward sub-step: not available for diagonal velocities");
  if (c->src.flags) return fail(c, PDG_ERR_UNSUPPORTED, "sources are defined for M2 and M2_collapsed");
  const double g1 = 1.0 / (2.0 - std::cbrt(2.0)), g2 = 1.0 - 2.0 * g1;
  out.clear();
  std::vector<PdgPassSpec> part;
  c->scheme = PDG_SCHEME_M2KIN;
  int r = PDG_OK;
  try {
    out.reserve(3 * (size_t)nsteps * 3 * (size_t)c->dim);
    for (int s = 0; s < nsteps && r == PDG_OK; ++s)
      for (double g : {g1, g2, g1}) {
        if ((r = build_schedule_one(c, g * dt, 1, part)) != PDG_OK) break;
        out.insert(out.end(), part.begin(), part.end());
      }
  } catch (...) {
    c->scheme = PDG_SCHEME_M4KIN;
    throw;
  }
  c->scheme = PDG_SCHEME_M4KIN;
  return r;
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

// State slots of the current model (D2Q9: nine populations and four scratch slots).
long long state_slots(const pdg_ctx* c) {
  Lattice L;
  return lattice_of(c->model.kind, &L) ? L.slots : (long long)c->model.nf;
}

// Allocate the kinetic state for the current model if it does not fit yet.
int ensure_state(pdg_ctx* c) {
  const long long need = state_slots(c) * c->npoints;
  if (need <= c->f_cap) return PDG_OK;
  c->gen++;
  double* nf = nullptr;
  cudaError_t e = pdg_fault_take_alloc() ? cudaErrorMemoryAllocation   // injected on the host (tests)
                  : c->async_alloc ? cudaMallocAsync((void**)&nf, sizeof(double) * (size_t)need, c->stream)
                                   : cudaMalloc((void**)&nf, sizeof(double) * (size_t)need);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, e == cudaErrorMemoryAllocation ? PDG_ERR_OOM : PDG_ERR_CUDA,
                std::string("cudaMalloc(f): ") + cudaGetErrorString(e));
  }
  if (c->f) {
    if (c->async_alloc) cudaFreeAsync(c->f, c->stream);
    else cudaFree(c->f);
  }
  c->f = nf;
  c->f_cap = need;
  c->has_state = false;
  return PDG_OK;
}

size_t fields_of(const pdg_ctx* c) { return (size_t)c->model.nf; }

// Lines of a pass along axis a (= points of the other axes).
long long lines_of(const pdg_ctx* c, int a) { return c->npoints / c->P[a]; }

// Allocate (zeroed) inflow data for every non-periodic axis of the current model.
int ensure_inflow(pdg_ctx* c) {
  for (int a = 0; a < c->dim; ++a) {
    if (c->periodic[a] || c->fb[a]) continue;
    const size_t n = 2 * (size_t)inflow_entries(c->model) * (size_t)lines_of(c, a);
    cudaError_t e = cudaMalloc((void**)&c->fb[a], sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->fb[a], 0, sizeof(double) * n, c->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(c, PDG_ERR_OOM, std::string("inflow data: ") + cudaGetErrorString(e));
    }
  }
  return PDG_OK;
}

void free_inflow(pdg_ctx* c) {
  for (int a = 0; a < 3; ++a)
    if (c->fb[a]) {
      cudaFree(c->fb[a]);
      c->fb[a] = nullptr;
    }
}

}  // namespace

// Host-side fault injection: the next n state allocations fail as if the device were out
// of memory (pdg_debug_fail_allocs).
static std::atomic<int> g_fail_allocs{0};

int pdg_fault_take_alloc() {
  int n = g_fail_allocs.load();
  while (n > 0 && !g_fail_allocs.compare_exchange_weak(n, n - 1)) {
  }
  return n > 0 ? 1 : 0;
}

bool pdg_internal_view(const pdg_ctx* c, PdgStateView* v) {
  if (!c || !c->has_state || !c->f) return false;
  v->f = c->f;
  v->npoints = c->npoints;
  v->m = c->model.m;
  v->nv = c->model.nv;
  v->nf = c->model.nf;
  v->prec = c->model.prec;
  v->stream = c->stream;
  return true;
}

int pdg_internal_fail(pdg_ctx* c, int code, const std::string& msg) { return fail(c, code, msg); }

void pdg_internal_set_async_alloc(pdg_ctx* c, bool on) { c->async_alloc = on; }

int pdg_internal_set_w_async(pdg_ctx* c, const double* w_host_pinned) {
  if (!c || !c->has_model || !w_host_pinned) return PDG_ERR_ARG;
  if (int r = ensure_state(c)) return r;
  const size_t need = (size_t)c->model.m * c->npoints;
  PDG_CUDA(c, cudaMemcpyAsync(c->f, w_host_pinned, sizeof(double) * need, cudaMemcpyHostToDevice, c->stream));
  int e = pdg_launch_set_feq(c->f, c->npoints, c->model, (void*)c->stream);
  if (e) return cuda_fail(c, (cudaError_t)e, "set_feq launch");
  c->has_state = true;
  return PDG_OK;
}

int pdg_internal_batch_set(pdg_batch* b, int n, pdg_ctx* const* ctxs) {
  if (!b || n < 0 || (n > 0 && !ctxs)) return PDG_ERR_ARG;
  b->inst.assign(ctxs, ctxs + n);
  return PDG_OK;
}

extern "C" {

const char* pdg_status_string(int s) {
  switch (s) {
    case PDG_OK: return "PDG_OK";
    case PDG_ERR_ARG: return "PDG_ERR_ARG";
    case PDG_ERR_OOM: return "PDG_ERR_OOM";
    case PDG_ERR_CUDA: return "PDG_ERR_CUDA";
    case PDG_ERR_STATE: return "PDG_ERR_STATE";
    case PDG_ERR_TIMEOUT: return "PDG_ERR_TIMEOUT";
    case PDG_ERR_UNSUPPORTED: return "PDG_ERR_UNSUPPORTED";
  }
  return "PDG_ERR_UNKNOWN";
}

const char* pdg_last_error(const pdg_ctx* c) { return c ? c->err.c_str() : "null context"; }

int pdg_debug_fail_allocs(int n) {
  if (n < 0) return PDG_ERR_ARG;
  g_fail_allocs.store(n);
  return PDG_OK;
}

int pdg_create_mesh(pdg_ctx** out, int dim, const int n_macro[3], const int n_sub[3], int order,
                    const double length[3], unsigned periodic_mask, void* cuda_stream) {
  if (!out) return PDG_ERR_ARG;
  *out = nullptr;
  if (dim < 1 || dim > 3 || !n_macro || !n_sub || order < 1 || order > PDG_MAXN - 1) return PDG_ERR_ARG;
  for (int a = 0; a < dim; ++a) {
    if (n_macro[a] < 1 || n_sub[a] < 1) return PDG_ERR_ARG;
    if ((long long)n_macro[a] * n_sub[a] * (order + 1) > (1LL << 30)) return PDG_ERR_ARG;
    if (length && !(length[a] > 0.0 && std::isfinite(length[a]))) return PDG_ERR_ARG;
  }
  pdg_ctx* c = new (std::nothrow) pdg_ctx();
  if (!c) return PDG_ERR_OOM;
  c->dim = dim;
  c->order = order;
  c->n = order + 1;
  for (int a = 0; a < dim; ++a) c->periodic[a] = (periodic_mask >> a) & 1u;
  long long np = 1;
  for (int a = 0; a < 3; ++a) {
    if (a < dim) {
      c->nmacro[a] = n_macro[a];
      c->nsub[a] = n_sub[a];
      c->N[a] = n_macro[a] * n_sub[a];
      c->P[a] = c->N[a] * c->n;
      c->len[a] = length ? length[a] : 1.0;
      c->h[a] = c->len[a] / c->N[a];
    }
    np *= c->P[a];
  }
  if (np > (1LL << 40)) {
    delete c;
    return PDG_ERR_ARG;
  }
  c->npoints = np;
  c->stream = (cudaStream_t)cuda_stream;
  *out = c;
  return PDG_OK;
}

int pdg_set_model(pdg_ctx* c, const pdg_model_desc* d) {
  if (!c || !d) return PDG_ERR_ARG;
  c->gen++;
  if (d->kind < PDG_MODEL_ADVECTION || d->kind > PDG_MODEL_ISOTHERMAL_D3Q27)
    return fail(c, PDG_ERR_ARG, "unknown model kind");
  if (d->scheme != PDG_SCHEME_M2 && d->scheme != PDG_SCHEME_M2_COLLAPSED && d->scheme != PDG_SCHEME_M2KIN &&
      d->scheme != PDG_SCHEME_M4KIN)
    return fail(c, PDG_ERR_ARG, "unknown scheme");
  if (d->precision != PDG_PREC_FP64 && d->precision != PDG_PREC_DF32 && d->precision != PDG_PREC_TF32 &&
      d->precision != PDG_PREC_TF32_DFRES)
    return fail(c, PDG_ERR_UNSUPPORTED, "precision not available");
  const bool tcp = d->precision == PDG_PREC_TF32 || d->precision == PDG_PREC_TF32_DFRES;
  if (tcp && d->kind != PDG_MODEL_ISOTHERMAL_D3Q15 && d->kind != PDG_MODEL_ISOTHERMAL_D3Q27)
    return fail(c, PDG_ERR_UNSUPPORTED,
                "the tensor-core precision forms apply to the dense cell inverses of the corner sweeps "
                "(D3Q15, D3Q27)");
  if (!(d->lambda > 0.0 && std::isfinite(d->lambda))) return fail(c, PDG_ERR_ARG, "lambda must be > 0");
  if (!std::isfinite(d->omega) || d->omega == 0.0) return fail(c, PDG_ERR_ARG, "omega must be finite and != 0");
  if (!(d->theta >= 0.0 && d->theta <= 1.0)) return fail(c, PDG_ERR_ARG, "theta must be in [0, 1]");
  if (d->kind == PDG_MODEL_SHALLOW_WATER && c->dim != 2)
    return fail(c, PDG_ERR_UNSUPPORTED, "shallow water needs dim = 2");
  const bool q9 = d->kind == PDG_MODEL_ISOTHERMAL_D2Q9, q19 = d->kind == PDG_MODEL_ISOTHERMAL_D3Q19;
  const bool q15 = d->kind == PDG_MODEL_ISOTHERMAL_D3Q15, q27 = d->kind == PDG_MODEL_ISOTHERMAL_D3Q27;
  const bool q3d = q19 || q15 || q27, lat = q9 || q3d;
  if (q9 && c->dim != 2) return fail(c, PDG_ERR_UNSUPPORTED, "D2Q9 needs dim = 2");
  if (q3d && c->dim != 3) return fail(c, PDG_ERR_UNSUPPORTED, "D3Q15 / D3Q19 / D3Q27 need dim = 3");
  if ((q15 || q27) && c->n > PDG_MAXN_CORNER)
    return fail(c, PDG_ERR_UNSUPPORTED, "D3Q15 / D3Q27 support degrees 1 to 3");
  if (lat && !(d->theta > 0.0)) return fail(c, PDG_ERR_UNSUPPORTED, "diagonal velocities need theta > 0");
  PdgModel M{};
  M.kind = d->kind;
  M.dim = c->dim;
  M.m = d->kind == PDG_MODEL_ADVECTION ? 1
        : (d->kind == PDG_MODEL_SHALLOW_WATER ? 3 : (lat ? c->dim + 1 : c->dim + 2));
  M.nv = q9 ? 9 : (q19 ? 19 : (q15 ? 15 : (q27 ? 27 : 2 * c->dim)));
  M.nf = lat ? M.nv : M.m * M.nv;
  M.lambda = d->lambda;
  M.omega = d->omega;
  for (int a = 0; a < 3; ++a) M.a[a] = d->a[a];
  M.gravity = d->gravity;
  M.gamma = d->gamma;
  for (int i = 0; i < M.nv && !lat; ++i) {
    const double s = (i % 2 == 0) ? 1.0 : -1.0;
    M.cadv[i] = 1.0 / (2.0 * c->dim) + s * d->a[i / 2] / (2.0 * d->lambda);
  }
  // the tensor-core forms keep an FP64 state: every kernel but the corner pass is the FP64 one
  M.prec = tcp ? PDG_PREC_FP64 : d->precision;
  pdg_model_constants(&M);
  if ((q15 || q27) && !c->cbuf) {
    cudaError_t e = cudaMalloc((void**)&c->cbuf, PDG_CORNER_PLANS * kCornerSlotBytes + kCornerErrBytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->cbuf = nullptr;
      return fail(c, PDG_ERR_OOM, std::string("corner coefficients: ") + cudaGetErrorString(e));
    }
    c->dev_err = reinterpret_cast<int*>(c->cbuf + PDG_CORNER_PLANS * kCornerSlotBytes);
    PDG_CUDA(c, cudaMemsetAsync(c->dev_err, 0, sizeof(int), c->stream));
  }
  c->tc = d->precision == PDG_PREC_TF32 ? 1 : (d->precision == PDG_PREC_TF32_DFRES ? 2 : 0);
  c->corner_plans.clear();
  // a different number of fields or a different state format invalidates the state
  if (c->has_model && (c->model.m != M.m || c->model.nf != M.nf || c->model.prec != M.prec)) {
    c->has_state = false;
    free_inflow(c);   // layout / format of the boundary data changes too (reset to zero)
  }
  c->model = M;
  c->src.flags = 0;   // a new model starts without a source
  c->scheme = d->scheme;
  c->precision = d->precision;
  c->theta = d->theta;
  c->has_model = true;
  return PDG_OK;
}

int pdg_set_w(pdg_ctx* c, const double* w, size_t len, int on_device) {
  if (!c) return PDG_ERR_ARG;
  if (!c->has_model) return fail(c, PDG_ERR_STATE, "pdg_set_w before pdg_set_model");
  if (!w) return fail(c, PDG_ERR_ARG, "w is NULL");
  const size_t need = (size_t)c->model.m * c->npoints;
  if (len != need) return fail(c, PDG_ERR_ARG, "w length mismatch");
  if (int r = ensure_state(c)) return r;
  if (int r = ensure_inflow(c)) return r;
  // w_k goes to field slot k; the kernel reads all w_k of a point before writing.
  PDG_CUDA(c, cudaMemcpyAsync(c->f, w, sizeof(double) * need,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  int e = pdg_launch_set_feq(c->f, c->npoints, c->model, (void*)c->stream);
  if (e) return cuda_fail(c, (cudaError_t)e, "set_feq launch");
  if (!on_device) PDG_CUDA(c, cudaStreamSynchronize(c->stream));
  c->has_state = true;
  return PDG_OK;
}

int pdg_set_f(pdg_ctx* c, const double* f, size_t len, int on_device) {
  if (!c) return PDG_ERR_ARG;
  if (!c->has_model) return fail(c, PDG_ERR_STATE, "pdg_set_f before pdg_set_model");
  if (!f) return fail(c, PDG_ERR_ARG, "f is NULL");
  const size_t need = fields_of(c) * c->npoints;
  if (len != need) return fail(c, PDG_ERR_ARG, "f length mismatch");
  if (int r = ensure_state(c)) return r;
  if (int r = ensure_inflow(c)) return r;
  PDG_CUDA(c, cudaMemcpyAsync(c->f, f, sizeof(double) * need,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  if (c->model.prec == PDG_PREC_DF32) {
    int e = pdg_launch_convert(c->f, (long long)need, 1, (void*)c->stream);
    if (e) return cuda_fail(c, (cudaError_t)e, "convert launch");
  }
  if (!on_device) PDG_CUDA(c, cudaStreamSynchronize(c->stream));
  c->has_state = true;
  return PDG_OK;
}

int pdg_get_f(pdg_ctx* c, double* out, size_t len, int on_device) {
  if (!c) return PDG_ERR_ARG;
  if (!c->has_state) return fail(c, PDG_ERR_STATE, "no state");
  if (!out) return fail(c, PDG_ERR_ARG, "out is NULL");
  const size_t need = fields_of(c) * c->npoints;
  if (len != need) return fail(c, PDG_ERR_ARG, "f length mismatch");
  const bool df = c->model.prec == PDG_PREC_DF32;
  // double-float state: convert to FP64 in place, copy, convert back (the round trip
  // pair -> double -> pair is exact)
  if (df) {
    int e = pdg_launch_convert(c->f, (long long)need, 0, (void*)c->stream);
    if (e) return cuda_fail(c, (cudaError_t)e, "convert launch");
  }
  PDG_CUDA(c, cudaMemcpyAsync(out, c->f, sizeof(double) * need,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  if (df) {
    int e = pdg_launch_convert(c->f, (long long)need, 1, (void*)c->stream);
    if (e) return cuda_fail(c, (cudaError_t)e, "convert launch");
  }
  if (!on_device) {
    PDG_CUDA(c, cudaStreamSynchronize(c->stream));
    if (int r = check_device_error(c)) return r;
  }
  return PDG_OK;
}

int pdg_get_w(pdg_ctx* c, double* out, size_t len, int on_device) {
  if (!c) return PDG_ERR_ARG;
  if (!c->has_state) return fail(c, PDG_ERR_STATE, "no state");
  if (!out) return fail(c, PDG_ERR_ARG, "out is NULL");
  const size_t need = (size_t)c->model.m * c->npoints;
  if (len != need) return fail(c, PDG_ERR_ARG, "w length mismatch");
  double* dst = out;
  if (!on_device) {
    if (c->wstage_cap < (long long)need) {
      double* nb = nullptr;
      cudaError_t e = cudaMalloc((void**)&nb, sizeof(double) * need);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, PDG_ERR_OOM, std::string("cudaMalloc(w staging): ") + cudaGetErrorString(e));
      }
      if (c->wstage) cudaFree(c->wstage);
      c->wstage = nb;
      c->wstage_cap = (long long)need;
    }
    dst = c->wstage;
  }
  int e = pdg_launch_get_w(c->f, dst, c->npoints, c->model, (void*)c->stream);
  if (e) return cuda_fail(c, (cudaError_t)e, "get_w launch");
  if (!on_device) {
    PDG_CUDA(c, cudaMemcpyAsync(out, dst, sizeof(double) * need, cudaMemcpyDeviceToHost, c->stream));
    PDG_CUDA(c, cudaStreamSynchronize(c->stream));
    if (int r = check_device_error(c)) return r;
  }
  return PDG_OK;
}

int pdg_set_source(pdg_ctx* c, const pdg_source_desc* d) {
  if (!c) return PDG_ERR_ARG;
  c->gen++;
  if (!c->has_model) return fail(c, PDG_ERR_STATE, "pdg_set_source before pdg_set_model");
  if (!d || d->flags == 0) {
    c->src.flags = 0;
    return PDG_OK;
  }
  if (c->model.kind != PDG_MODEL_ISOTHERMAL_D2Q9)
    return fail(c, PDG_ERR_UNSUPPORTED, "sources are available for the D2Q9 model");
  if (c->scheme == PDG_SCHEME_M2KIN || c->scheme == PDG_SCHEME_M4KIN)
    return fail(c, PDG_ERR_UNSUPPORTED, "sources are defined for M2 and M2_collapsed");
  if (d->flags & ~(PDG_SOURCE_GRAVITY | PDG_SOURCE_PENALIZATION)) return fail(c, PDG_ERR_ARG, "unknown source flag");
  if (!(d->theta >= 0.0 && d->theta <= 1.0)) return fail(c, PDG_ERR_ARG, "source theta must be in [0, 1]");
  const bool pen = d->flags & PDG_SOURCE_PENALIZATION;
  for (int a = 0; a < 2; ++a)
    if (!std::isfinite(d->gravity[a]) || !std::isfinite(d->x_c[a])) return fail(c, PDG_ERR_ARG, "non-finite source value");
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(d->w_s[k])) return fail(c, PDG_ERR_ARG, "non-finite source value");
  if (pen && !(d->K_s >= 0.0 && std::isfinite(d->K_s) && d->kappa >= 0.0 && std::isfinite(d->kappa)))
    return fail(c, PDG_ERR_ARG, "penalisation needs finite K_s >= 0 and kappa >= 0");
  PdgSrc S{};
  S.flags = d->flags;
  const bool grav = d->flags & PDG_SOURCE_GRAVITY;
  for (int a = 0; a < 2; ++a) S.g[a] = grav ? d->gravity[a] : 0.0;
  for (int k = 0; k < 3; ++k) S.ws[k] = d->w_s[k];
  S.theta = d->theta;
  S.omtheta = 1.0 - d->theta;
  for (int a = 0; a < 2; ++a) pdg_split(S.g[a], S.g_f[a]);
  for (int k = 0; k < 3; ++k) pdg_split(S.ws[k], S.ws_f[k]);
  pdg_split(S.theta, S.theta_f[0]);
  pdg_split(S.omtheta, S.omtheta_f[0]);
  if (pen) {
    // K(x) = K_s exp(-kappa |x - x_c|^2) at the GL points, computed on the host once; a
    // host allocation failure returns PDG_ERR_OOM with the source left unchanged
    std::vector<double> xs[2];
    std::vector<double> K;
    try {
      for (int a = 0; a < 2; ++a) xs[a].resize(c->P[a]);
      K.resize((size_t)c->npoints);
    } catch (const std::bad_alloc&) {
      return fail(c, PDG_ERR_OOM, "no host memory for the penalisation field");
    } catch (const std::length_error&) {
      return fail(c, PDG_ERR_OOM, "no host memory for the penalisation field");
    }
    for (int a = 0; a < 2; ++a)
      if (pdg_get_points(c, a, xs[a].data(), xs[a].size())) return fail(c, PDG_ERR_ARG, "points");
    for (int y = 0; y < c->P[1]; ++y) {
      const double dy = xs[1][y] - d->x_c[1];
      for (int x = 0; x < c->P[0]; ++x) {
        const double dx = xs[0][x] - d->x_c[0];
        K[(size_t)y * c->P[0] + x] = d->K_s * std::exp(-d->kappa * (dx * dx + dy * dy));
      }
    }
    if (!c->kfield) {
      cudaError_t e = cudaMalloc((void**)&c->kfield, sizeof(double) * (size_t)c->npoints);
      if (e != cudaSuccess) {
        cudaGetLastError();
        c->kfield = nullptr;
        return fail(c, PDG_ERR_OOM, std::string("cudaMalloc(K): ") + cudaGetErrorString(e));
      }
    }
    PDG_CUDA(c, cudaMemcpyAsync(c->kfield, K.data(), sizeof(double) * K.size(), cudaMemcpyHostToDevice, c->stream));
    PDG_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  c->src = S;
  return PDG_OK;
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

int pdg_step(pdg_ctx* c, double dt, int nsteps) {
  if (!c) return PDG_ERR_ARG;
  if (!c->has_state) return fail(c, PDG_ERR_STATE, "pdg_step before pdg_set_w / pdg_set_f");
  if (nsteps < 0 || !std::isfinite(dt)) return fail(c, PDG_ERR_ARG, "bad dt or nsteps");
  if (nsteps == 0) return PDG_OK;
  const bool graph = c->use_graph && !c->timing;
  if (graph && c->gexec && c->g_gen == c->gen && c->g_dt == dt && c->g_nsteps == nsteps) {
    PDG_CUDA(c, cudaEventRecord(c->g_in, c->stream));
    PDG_CUDA(c, cudaStreamWaitEvent(c->gstream, c->g_in, 0));
    PDG_CUDA(c, cudaGraphLaunch(c->gexec, c->gstream));
    PDG_CUDA(c, cudaEventRecord(c->g_out, c->gstream));
    PDG_CUDA(c, cudaStreamWaitEvent(c->stream, c->g_out, 0));
    return PDG_OK;
  }
  std::vector<PdgPassSpec> sched;
  if (int r = build_schedule_checked(c, dt, nsteps, sched)) return r;
  if (graph) {
    if (int r = capture_steps(c, dt, nsteps, sched)) return r;
    return pdg_step(c, dt, nsteps);   // replay
  }
  for (const auto& sp : sched)
    if (int r = issue_pass(c, sp)) return r;
  return PDG_OK;
}

int pdg_set_inflow(pdg_ctx* c, int axis, const double* fb, size_t len, int on_device) {
  if (!c) return PDG_ERR_ARG;
  c->gen++;
  if (!c->has_model) return fail(c, PDG_ERR_STATE, "pdg_set_inflow before pdg_set_model");
  if (axis < 0 || axis >= c->dim || c->periodic[axis]) return fail(c, PDG_ERR_ARG, "axis is not an inflow axis");
  if (!fb) return fail(c, PDG_ERR_ARG, "fb is NULL");
  const size_t need = 2 * (size_t)inflow_entries(c->model) * (size_t)lines_of(c, axis);
  if (len != need) return fail(c, PDG_ERR_ARG, "inflow data length mismatch");
  if (int r = ensure_inflow(c)) return r;
  PDG_CUDA(c, cudaMemcpyAsync(c->fb[axis], fb, sizeof(double) * need,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  if (c->model.prec == PDG_PREC_DF32) {
    int e = pdg_launch_convert(c->fb[axis], (long long)need, 1, (void*)c->stream);
    if (e) return cuda_fail(c, (cudaError_t)e, "convert launch");
  }
  if (!on_device) PDG_CUDA(c, cudaStreamSynchronize(c->stream));
  return PDG_OK;
}

int pdg_get_points(const pdg_ctx* c, int axis, double* out, size_t len) {
  if (!c || !out || axis < 0 || axis >= c->dim) return PDG_ERR_ARG;
  if (len != (size_t)c->P[axis]) return PDG_ERR_ARG;
  double x[PDG_MAXN], w[PDG_MAXN];
  if (pdg_plan_gl(c->order, x, w)) return PDG_ERR_ARG;
  const double h = c->h[axis];
  for (int cell = 0; cell < c->N[axis]; ++cell)
    for (int j = 0; j < c->n; ++j) out[(size_t)cell * c->n + j] = cell * h + 0.5 * h * (1.0 + x[j]);
  return PDG_OK;
}

int pdg_get_info(const pdg_ctx* c, pdg_info* info) {
  if (!c || !info) return PDG_ERR_ARG;
  std::memset(info, 0, sizeof(*info));
  info->dim = c->dim;
  info->order = c->order;
  info->m = c->has_model ? c->model.m : 0;
  info->nv = c->has_model ? c->model.nv : 2 * c->dim;
  for (int a = 0; a < 3; ++a) {
    info->ncell[a] = c->N[a];
    info->npts[a] = c->P[a];
    info->h[a] = a < c->dim ? c->h[a] : 0.0;
  }
  info->npoints = c->npoints;
  info->nfields = c->has_model ? (long long)c->model.nf : 0;
  info->w_len = (long long)info->m * c->npoints;
  info->f_len = info->nfields * c->npoints;
  return PDG_OK;
}

int pdg_get_line_coefs(const pdg_ctx* c, int axis, double delta, double* E, double* q, double* beta) {
  if (!c) return PDG_ERR_ARG;
  if (!c->has_model) return PDG_ERR_STATE;
  if (axis < 0 || axis >= c->dim || !E || !q || !beta) return PDG_ERR_ARG;
  PdgCoef C;
  if (plan_line_coef(c, axis, delta, &C)) return PDG_ERR_ARG;
  const int n = c->n;
  for (int i = 0; i < n * n; ++i) E[i] = C.E[i];
  for (int i = 0; i < n; ++i) q[i] = C.q[i];
  *beta = C.beta;
  return PDG_OK;
}

int pdg_get_schedule(pdg_ctx* c, double dt, int nsteps, int* ints, double* dbls, int max_passes, int* npasses) {
  if (!c || !npasses || nsteps < 0 || max_passes < 0 || !std::isfinite(dt)) return PDG_ERR_ARG;
  if (!c->has_model) return PDG_ERR_STATE;
  std::vector<PdgPassSpec> sched;
  if (int r = build_schedule_checked(c, dt, nsteps, sched)) return r;
  if (sched.size() > (size_t)0x7fffffff) return fail(c, PDG_ERR_ARG, "more passes than an int counts");
  *npasses = (int)sched.size();
  if (!ints && !dbls) return PDG_OK;
  if (!ints || !dbls || (int)sched.size() > max_passes) return PDG_ERR_ARG;
  static_assert(PDG_MAXOPS <= 4, "four operation slots per pass");
  for (size_t i = 0; i < sched.size(); ++i) {
    const PdgPassSpec& sp = sched[i];
    int* I = ints + 8 * i;
    double* X = dbls + 10 * i;
    for (int k = 0; k < 8; ++k) I[k] = 0;
    for (int k = 0; k < 10; ++k) X[k] = 0.0;
    I[0] = sp.axis >= 0 ? 0 : (sp.axis == -1 ? 1 : 2);
    I[1] = sp.axis;
    if (sp.axis >= 0) {
      I[2] = sp.nops;
      for (int o = 0; o < sp.nops; ++o) {
        I[3 + o] = sp.op[o];
        if (sp.op[o] == PDG_OP_T) {
          const PdgCoef& cf = sp.cs[sp.opcoef[o]];
          X[2 * o] = cf.E[0];
          X[2 * o + 1] = cf.beta;
        }
      }
      I[7] = sp.dslot;
      X[9] = sp.sdelta;
    } else if (sp.axis == -1) {
      I[7] = sp.dslot_in;
      X[8] = sp.ddelta;
    }
  }
  return PDG_OK;
}

int pdg_synchronize(pdg_ctx* c) {
  if (!c) return PDG_ERR_ARG;
  PDG_CUDA(c, cudaStreamSynchronize(c->stream));
  return check_device_error(c);
}

int pdg_timing_enable(pdg_ctx* c, int enable) {
  if (!c) return PDG_ERR_ARG;
  if (!c->pending.empty()) {
    PDG_CUDA(c, cudaStreamSynchronize(c->stream));
    int r = drain_timing(c);
    if (r) return r;
  }
  c->timing = enable != 0;
  for (int k = 0; k < 5; ++k) {
    c->t_launches[k] = 0;
    c->t_ms[k] = 0.0;
  }
  return PDG_OK;
}

int pdg_timing_read(pdg_ctx* c, long long* launches, double* ms, int max_kinds) {
  if (!c || max_kinds < 0) return PDG_ERR_ARG;
  PDG_CUDA(c, cudaStreamSynchronize(c->stream));
  int r = drain_timing(c);
  if (r) return r;
  for (int k = 0; k < max_kinds && k < 5; ++k) {
    if (launches) launches[k] = c->t_launches[k];
    if (ms) ms[k] = c->t_ms[k];
  }
  return PDG_OK;
}

int pdg_set_launch(pdg_ctx* c, int kind, int lpb, int nseg, int ngroup) {
  if (!c || kind < 0 || kind > 6) return PDG_ERR_ARG;
  c->gen++;
  if (kind == 6) {   // corner box along x, y, z; the threads stay as kind 5 set them
    if (lpb == 0 && nseg == 0 && ngroup == 0) {
      c->cshape[1] = c->cshape[2] = c->cshape[3] = 0;
      return PDG_OK;
    }
    if (lpb < 1 || nseg < 1 || ngroup < 1) return fail(c, PDG_ERR_ARG, "bad corner box shape");
    c->cshape[1] = lpb;
    c->cshape[2] = nseg;
    c->cshape[3] = ngroup;
    return PDG_OK;
  }
  if (kind == 5) {
    if (lpb == 0 && nseg == 0 && ngroup == 0) {
      c->cshape[0] = c->cshape[1] = c->cshape[2] = c->cshape[3] = 0;
      return PDG_OK;
    }
    if (lpb < 64 || lpb > 512 || lpb % 32 || nseg < 1 || ngroup < 1)
      return fail(c, PDG_ERR_ARG, "bad corner launch shape");
    c->cshape[0] = lpb;
    c->cshape[1] = c->cshape[2] = nseg;
    c->cshape[3] = ngroup;
    return PDG_OK;
  }
  if (kind == 4) {
    if (lpb == 0 && nseg == 0 && ngroup == 0) {
      c->dshape[0] = c->dshape[1] = c->dshape[2] = 0;
      return PDG_OK;
    }
    if (lpb < 64 || lpb > 512 || lpb % 32 || nseg < 1 || ngroup < 1)
      return fail(c, PDG_ERR_ARG, "bad diagonal launch shape");
    c->dshape[0] = lpb;
    c->dshape[1] = nseg;
    c->dshape[2] = ngroup;
    return PDG_OK;
  }
  int* slot = kind < 2 ? c->launch[kind] : c->bshape[kind - 2];
  const int maxt = kind < 2 ? 512 : pdg_batch_threads();
  if (lpb == 0 && nseg == 0 && ngroup == 0) {
    slot[0] = slot[1] = slot[2] = 0;
    return PDG_OK;
  }
  if (lpb < 1 || nseg < 1 || ngroup < 1 || (long long)lpb * nseg * ngroup > maxt)
    return fail(c, PDG_ERR_ARG, "bad launch shape");
  slot[0] = lpb;
  slot[1] = nseg;
  slot[2] = ngroup;
  return PDG_OK;
}

int pdg_destroy(pdg_ctx* c) {
  if (!c) return PDG_OK;
  if (!c->async_alloc && (c->stream || c->f)) cudaStreamSynchronize(c->stream);
  for (auto& t : c->pending) {
    cudaEventDestroy(t.e0);
    cudaEventDestroy(t.e1);
  }
  for (auto e : c->event_pool) cudaEventDestroy(e);
  if (c->f) {
    if (c->async_alloc) cudaFreeAsync(c->f, c->stream);
    else cudaFree(c->f);
  }
  if (c->wstage) cudaFree(c->wstage);
  if (c->kfield) cudaFree(c->kfield);
  if (c->cbuf) cudaFree(c->cbuf);
  if (c->czt) cudaFree(c->czt);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->gstream) {
    cudaStreamSynchronize(c->gstream);
    cudaStreamDestroy(c->gstream);
  }
  if (c->g_in) cudaEventDestroy(c->g_in);
  if (c->g_out) cudaEventDestroy(c->g_out);
  for (int i = 0; i < 4; ++i) {
    if (c->dstream[i]) {
      cudaStreamSynchronize(c->dstream[i]);
      cudaStreamDestroy(c->dstream[i]);
    }
    if (c->djoin[i]) cudaEventDestroy(c->djoin[i]);
  }
  if (c->dfork) cudaEventDestroy(c->dfork);
  free_inflow(c);
  delete c;
  return PDG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Autotuner: time candidate launch shapes of the two pass kinds on a scratch copy
// of the state and keep the fastest.

namespace {

struct Shape {
  int lpb, nseg, ngroup;
};

std::vector<Shape> shape_candidates(int max_threads, int ncell, int ntf, int W) {
  std::vector<Shape> out;
  const int lpbs[] = {4, 8, 16, 32};
  const int segs[] = {1, 2, 4, 8, 16, 32};
  const int groups[] = {1, 2, ntf / 2, ntf};
  for (int L : lpbs)
    for (int S : segs) {
      if (S > ncell) continue;
      if (S > 1 && ncell / S < W) continue;  // keep the window closure
      for (int gi = 0; gi < 4; ++gi) {
        const int G = groups[gi];
        if (G < 1 || ntf % G) continue;
        if (gi > 0 && G == groups[gi - 1]) continue;
        const int t = L * S * G;
        if (t > max_threads || t < max_threads / 4) continue;
        out.push_back({L, S, G});
      }
    }
  if (out.empty()) out.push_back({8, 1, 1});
  return out;
}

// Runs `reps` launches of one pass on a scratch copy of the state and returns the mean ms.
template <class LaunchFn>
int time_launches(pdg_ctx* c, int reps, LaunchFn fn, float* ms) {
  cudaEvent_t a, b;
  PDG_CUDA(c, cudaEventCreate(&a));
  PDG_CUDA(c, cudaEventCreate(&b));
  int r = fn();  // warm-up
  if (r) return r;
  PDG_CUDA(c, cudaEventRecord(a, c->stream));
  for (int i = 0; i < reps; ++i)
    if ((r = fn())) return r;
  PDG_CUDA(c, cudaEventRecord(b, c->stream));
  PDG_CUDA(c, cudaEventSynchronize(b));
  float t = 0.f;
  PDG_CUDA(c, cudaEventElapsedTime(&t, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms = t / (reps > 0 ? reps : 1);
  return PDG_OK;
}

// Representative pass specs of kind 0 and 1 for time step dt.
int representative_specs(pdg_ctx* c, double dt, PdgPassSpec* sp, bool* have) {
  std::vector<PdgPassSpec> sched;
  if (int r = build_schedule_checked(c, dt, 2, sched)) return r;
  have[0] = have[1] = false;
  for (const auto& s : sched) {
    if (s.axis < 0) continue;   // diagonal passes and copies have no line shape
    const int k = pass_kind(s);
    // prefer the steady-state passes (T T and T C T)
    if (!have[k] || s.nops > sp[k].nops) {
      sp[k] = s;
      have[k] = true;
    }
  }
  return PDG_OK;
}

}  // namespace

extern "C" {

int pdg_autotune(pdg_ctx* c, double dt, int reps) {
  if (c) c->gen++;
  if (!c) return PDG_ERR_ARG;
  if (!c->has_state) return fail(c, PDG_ERR_STATE, "pdg_autotune needs a state (pdg_set_w)");
  if (!std::isfinite(dt) || dt == 0.0 || reps < 1) return fail(c, PDG_ERR_ARG, "bad dt or reps");
  PdgPassSpec sp[2];
  bool have[2];
  if (int r = representative_specs(c, dt, sp, have)) return r;
  const size_t bytes = sizeof(double) * (size_t)state_slots(c) * c->npoints;
  double* scratch = nullptr;
  cudaError_t e = cudaMalloc((void**)&scratch, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, PDG_ERR_OOM, "pdg_autotune: no memory for the scratch state");
  }
  double* keep = c->f;
  int status = PDG_OK;
  e = cudaMemcpyAsync(scratch, c->f, bytes, cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) status = cuda_fail(c, e, "pdg_autotune copy");
  c->f = scratch;
  const bool tim = c->timing;
  c->timing = false;
  for (int k = 0; k < 2 && status == PDG_OK; ++k) {
    if (!have[k]) continue;
    PdgPass p0;
    if ((status = make_pass(c, sp[k], 512, nullptr, &p0))) break;
    int W = 1;
    for (int i = 0; i < sp[k].ncs; ++i) W = std::max(W, stable_window(sp[k].cs[i]));
    float best = 1e30f;
    Shape bs{0, 0, 0};
    for (const Shape& s : shape_candidates(512, p0.ncell, p0.ntf, W)) {
      int ov[3] = {s.lpb, s.nseg, s.ngroup};
      PdgPass p;
      if ((status = make_pass(c, sp[k], 512, ov, &p))) break;
      balance_blocks(&p);
      float ms = 0.f;
      status = time_launches(c, reps, [&]() {
        int er = pdg_launch_pass(p, (void*)c->stream);
        return er ? cuda_fail(c, (cudaError_t)er, "autotune launch") : PDG_OK;
      }, &ms);
      if (status) break;
      if (ms < best) {
        best = ms;
        bs = s;
      }
    }
    if (status == PDG_OK && bs.lpb > 0) {
      c->launch[k][0] = bs.lpb;
      c->launch[k][1] = bs.nseg;
      c->launch[k][2] = bs.ngroup;
    }
  }
  c->timing = tim;
  c->f = keep;
  cudaStreamSynchronize(c->stream);
  cudaFree(scratch);
  return status;
}

int pdg_set_option(pdg_ctx* c, int option, int value) {
  if (!c) return PDG_ERR_ARG;
  c->gen++;
  switch (option) {
    case PDG_OPT_COMPOSE_TT:
      c->compose = value != 0;
      return PDG_OK;
    case PDG_OPT_GRAPH:
      c->use_graph = value != 0;
      return PDG_OK;
    case PDG_OPT_DEBUG_TC_STALL:
      c->tc_stall = value != 0;
      return PDG_OK;
  }
  return fail(c, PDG_ERR_ARG, "unknown option");
}

int pdg_get_launch(const pdg_ctx* c, int kind, int* lpb, int* nseg, int* ngroup) {
  if (!c || kind < 0 || kind > 6 || !lpb || !nseg || !ngroup) return PDG_ERR_ARG;
  if (kind == 6) {
    *lpb = c->cshape[1];
    *nseg = c->cshape[2];
    *ngroup = c->cshape[3];
    return PDG_OK;
  }
  if (kind == 5) {
    *lpb = c->cshape[0];
    *nseg = c->cshape[1];
    *ngroup = c->cshape[3];
    return PDG_OK;
  }
  const int* slot = kind < 2 ? c->launch[kind] : (kind < 4 ? c->bshape[kind - 2] : c->dshape);
  *lpb = slot[0];
  *nseg = slot[1];
  *ngroup = slot[2];
  return PDG_OK;
}

// ---------------------------------------------------------------------------
// Batched execution of many independent meshes.

}  // extern "C"

extern "C" const char* pdg_batch_last_error(const pdg_batch* b) { return b ? b->err.c_str() : "null batch"; }

extern "C" {

int pdg_batch_create(pdg_batch** out, int n, pdg_ctx* const* ctxs, void* cuda_stream) {
  if (!out) return PDG_ERR_ARG;
  *out = nullptr;
  if (n < 1 || !ctxs) return PDG_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i] || !ctxs[i]->has_model) return PDG_ERR_STATE;
    Lattice L;
    if (lattice_of(ctxs[i]->model.kind, &L)) return PDG_ERR_UNSUPPORTED;
  }
  pdg_batch* b = new (std::nothrow) pdg_batch();
  if (!b) return PDG_ERR_OOM;
  b->inst.assign(ctxs, ctxs + n);
  b->stream = (cudaStream_t)cuda_stream;
  // carry arrays sized for the largest population count (any instance list fits)
  const int maxcarry = 3 * (2 * PDG_MAXM) * pdg_batch_threads();
  b->smem = pdg_batch_smem(maxcarry);
  int e = 0;
  // Graphs cannot be captured on the legacy default stream: capture and replay on a
  // private blocking stream joined to the caller's stream with events.
  if (e || cudaEventCreate(&b->e0) != cudaSuccess || cudaEventCreate(&b->e1) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ej, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap, cudaStreamDefault) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return PDG_ERR_CUDA;
  }
  *out = b;
  return PDG_OK;
}

}  // extern "C"

namespace {

int bfail(pdg_batch* b, int code, const std::string& m) {
  b->err = m;
  return code;
}

template <class T>
int ensure_dev(pdg_batch* b, T** p, size_t* cap, size_t need) {
  if (need <= *cap) return PDG_OK;
  // the cached graph holds the old address: it is replayed no more (and freed first)
  if (b->gexec) {
    cudaStreamSynchronize(b->cap);
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  b->realloc = true;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * need);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, PDG_ERR_OOM, "batch table allocation failed");
  }
  *cap = need;
  return PDG_OK;
}

double item_cost(const PdgPass& p) {
  int nt = 0, nc = 0;
  for (int o = 0; o < p.nops; ++o) {
    nt += p.op[o] == PDG_OP_T;
    nc += p.op[o] == PDG_OP_C;
  }
  const int np = p.npl / p.ncell;
  const double per_point = (double)p.ntf * nt * (np + 2) + (double)nc * p.model.m * p.model.nv * 6.0;
  return (double)p.lpb * p.npl * per_point;
}

// Build the stage tables for dt[i], nsteps[i] and upload them.
int batch_prepare(pdg_batch* b, const double* dt, const int* nsteps) {
  const int n = (int)b->inst.size();
  std::vector<PdgPass> descs;
  std::vector<std::vector<int>> plist(n);  // per instance: descriptor index per pass
  std::vector<std::vector<long long>> pblocks(n);
  for (int i = 0; i < n; ++i) {
    pdg_ctx* c = b->inst[i];
    if (!c->has_state) return bfail(b, PDG_ERR_STATE, "batch instance without state");
    Lattice L;
    if (lattice_of(c->model.kind, &L))
      return bfail(b, PDG_ERR_UNSUPPORTED, "lattice (D2Q9 / D3Qq) instances run through pdg_step only");
    if (nsteps[i] < 0 || !std::isfinite(dt[i])) return bfail(b, PDG_ERR_ARG, "bad dt or nsteps");
    std::vector<PdgPassSpec> sched;
    if (int r = build_schedule_checked(c, dt[i], nsteps[i], sched)) return bfail(b, r, c->err);
    for (const auto& sp : sched) {
      const int kind = pass_kind(sp);
      PdgPass p;
      if (int r = make_pass(c, sp, pdg_batch_threads(), c->bshape[kind], &p)) return bfail(b, r, c->err);
      // reuse the previous identical descriptor of this instance (steady-state passes repeat)
      int idx = -1;
      for (int j = (int)descs.size() - 1; j >= 0 && j >= (int)descs.size() - 4; --j)
        if (std::memcmp(&descs[j], &p, sizeof(PdgPass)) == 0) {
          idx = j;
          break;
        }
      if (idx < 0) {
        idx = (int)descs.size();
        descs.push_back(p);
      }
      plist[i].push_back(idx);
      pblocks[i].push_back((p.nlines + p.lpb - 1) / p.lpb);
    }
  }
  size_t nst = 0;
  for (int i = 0; i < n; ++i) nst = std::max(nst, plist[i].size());
  std::vector<int> ent_desc;
  std::vector<long long> ent_start;
  b->st_off.clear();
  b->st_nent.clear();
  b->st_total.clear();
  b->st_prec.clear();
  b->st_np.clear();
  b->st_mv.clear();
  for (size_t t = 0; t < nst; ++t) {
    // groups of this stage: one persistent launch per (precision, degree, model) variant
    std::vector<int> keys;
    for (int i = 0; i < n; ++i)
      if (t < plist[i].size()) {
        const PdgPass& d = descs[plist[i][t]];
        const int key = (d.prec * 8 + d.npl / d.ncell) * 8 + d.mv;
        if (std::find(keys.begin(), keys.end(), key) == keys.end()) keys.push_back(key);
      }
    std::sort(keys.begin(), keys.end());
    for (int key : keys) {
      std::vector<std::pair<double, int>> order;  // (cost per item, instance)
      for (int i = 0; i < n; ++i)
        if (t < plist[i].size()) {
          const PdgPass& d = descs[plist[i][t]];
          if ((d.prec * 8 + d.npl / d.ncell) * 8 + d.mv == key) order.push_back({item_cost(d), i});
        }
      std::stable_sort(order.begin(), order.end(), [](const std::pair<double, int>& x,
                                                      const std::pair<double, int>& y) { return x.first > y.first; });
      b->st_off.push_back((int)ent_desc.size());
      long long acc = 0;
      for (auto& o : order) {
        ent_desc.push_back(plist[o.second][t]);
        ent_start.push_back(acc);
        acc += pblocks[o.second][t];
      }
      b->st_nent.push_back((int)order.size());
      b->st_total.push_back(acc);
      b->st_prec.push_back(key / 64);
      b->st_np.push_back((key / 8) % 8);
      b->st_mv.push_back(key % 8);
    }
  }
  nst = b->st_off.size();
  if (int r = ensure_dev(b, &b->d_desc, &b->cap_desc, std::max<size_t>(1, descs.size()))) return r;
  if (int r = ensure_dev(b, &b->d_ent_desc, &b->cap_ent, std::max<size_t>(1, ent_desc.size()))) return r;
  if (int r = ensure_dev(b, &b->d_ent_start, &b->cap_es, std::max<size_t>(1, ent_start.size()))) return r;
  if (int r = ensure_dev(b, &b->d_counter, &b->cap_cnt, std::max<size_t>(1, nst))) return r;
  cudaError_t e = cudaSuccess;
  e = cudaMemcpyAsync(b->d_desc, descs.data(), sizeof(PdgPass) * descs.size(), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_ent_desc, ent_desc.data(), sizeof(int) * ent_desc.size(), cudaMemcpyHostToDevice,
                        b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_ent_start, ent_start.data(), sizeof(long long) * ent_start.size(),
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // host vectors die at return
  if (e != cudaSuccess) return bfail(b, PDG_ERR_CUDA, std::string("batch upload: ") + cudaGetErrorString(e));
  // signature: the tables themselves
  b->sig.clear();
  auto app = [&](const void* p, size_t nb) {
    const char* q = (const char*)p;
    b->sig.insert(b->sig.end(), q, q + nb);
  };
  app(descs.data(), sizeof(PdgPass) * descs.size());
  app(ent_desc.data(), sizeof(int) * ent_desc.size());
  app(ent_start.data(), sizeof(long long) * ent_start.size());
  return PDG_OK;
}

int batch_issue(pdg_batch* b, cudaStream_t st) {
  const size_t nst = b->st_nent.size();
  cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long) * std::max<size_t>(1, nst), st);
  if (e != cudaSuccess) return bfail(b, PDG_ERR_CUDA, std::string("batch counters: ") + cudaGetErrorString(e));
  long long launches = 0;
  for (size_t t = 0; t < nst; ++t) {
    int r = pdg_launch_batch(b->d_desc, b->d_ent_desc + b->st_off[t], b->d_ent_start + b->st_off[t],
                             b->st_nent[t], b->st_total[t], b->d_counter + t, b->smem, b->st_prec[t],
                             b->st_np[t], b->st_mv[t], (void*)st);
    if (r) return bfail(b, PDG_ERR_CUDA, std::string("batch launch: ") + cudaGetErrorString((cudaError_t)r));
    launches += b->st_total[t] > 0;
  }
  b->last_launches = launches;
  return PDG_OK;
}

// End a capture left open by an error so that the stream is usable again.
void abort_capture(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(st, &g);
    if (g) cudaGraphDestroy(g);
  }
  cudaGetLastError();
}

}  // namespace

extern "C" {

int pdg_batch_step(pdg_batch* b, const double* dt, const int* nsteps, int use_graph) {
  if (!b || !dt || !nsteps) return PDG_ERR_ARG;
  if (int r = batch_prepare(b, dt, nsteps)) return r;
  cudaError_t e = cudaEventRecord(b->e0, b->stream);
  if (e != cudaSuccess) return bfail(b, PDG_ERR_CUDA, cudaGetErrorString(e));
  if (!use_graph) {
    if (int r = batch_issue(b, b->stream)) return r;
  } else {
    if (!b->gexec || b->gsig != b->sig) {
      if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
      }
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) {
        abort_capture(b->cap);
        return bfail(b, PDG_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
      }
      int r = batch_issue(b, b->cap);
      e = cudaStreamEndCapture(b->cap, &g);
      if (r || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        abort_capture(b->cap);
        return r ? r : bfail(b, PDG_ERR_CUDA, std::string("capture end: ") + cudaGetErrorString(e));
      }
      e = cudaGraphInstantiate(&b->gexec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        b->gexec = nullptr;
        return bfail(b, PDG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
      }
      b->gsig = b->sig;
    }
    // order: caller stream -> capture stream (graph) -> caller stream
    e = cudaEventRecord(b->ej, b->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->ej, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->gexec, b->cap);
    if (e == cudaSuccess) e = cudaEventRecord(b->ej, b->cap);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ej, 0);
    if (e != cudaSuccess) return bfail(b, PDG_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  }
  e = cudaEventRecord(b->e1, b->stream);
  if (e != cudaSuccess) return bfail(b, PDG_ERR_CUDA, cudaGetErrorString(e));
  return PDG_OK;
}

int pdg_batch_elapsed(pdg_batch* b, double* ms, long long* launches) {
  if (!b) return PDG_ERR_ARG;
  cudaError_t e = cudaEventSynchronize(b->e1);
  if (e != cudaSuccess) return bfail(b, PDG_ERR_CUDA, cudaGetErrorString(e));
  float t = 0.f;
  e = cudaEventElapsedTime(&t, b->e0, b->e1);
  if (e != cudaSuccess) return bfail(b, PDG_ERR_CUDA, cudaGetErrorString(e));
  if (ms) *ms = t;
  if (launches) *launches = b->last_launches;
  return PDG_OK;
}

}  // extern "C"

namespace {
// Autotuning classes: cells per line rounded to a power of two, CFL number rounded to
// a power of two (the window of the periodic closure depends on it).
int size_bucket(const pdg_ctx* c) {
  int m = 0;
  for (int a = 0; a < c->dim; ++a) m = std::max(m, c->N[a]);
  int b = 0;
  while ((1 << b) < m) ++b;
  return b;
}
int cfl_bucket(const pdg_ctx* c, double dt) {
  const double nu = std::fabs(2.0 * c->model.lambda * dt / c->h[0]);
  return (int)std::floor(std::log2(nu + 1e-300) + 0.5);
}
}  // namespace

extern "C" {

int pdg_batch_autotune(pdg_batch* b, const double* dt, int reps) {
  if (!b || !dt || reps < 1) return PDG_ERR_ARG;
  const int n = (int)b->inst.size();
  // one representative per class (dimension, degree, cells per axis, model)
  std::vector<int> rep(n, -1);
  for (int i = 0; i < n; ++i) {
    pdg_ctx* ci = b->inst[i];
    for (int j = 0; j < i && rep[i] < 0; ++j) {
      pdg_ctx* cj = b->inst[j];
      if (rep[j] == j && ci->dim == cj->dim && ci->order == cj->order && ci->model.kind == cj->model.kind &&
          size_bucket(ci) == size_bucket(cj) && cfl_bucket(ci, dt[i]) == cfl_bucket(cj, dt[j]))
        rep[i] = j;
    }
    if (rep[i] < 0) rep[i] = i;
  }
  for (int i = 0; i < n; ++i) {
    if (rep[i] != i) continue;
    pdg_ctx* c = b->inst[i];
    if (!c->has_state) return bfail(b, PDG_ERR_STATE, "batch instance without state");
    PdgPassSpec sp[2];
    bool have[2];
    if (int r = representative_specs(c, dt[i], sp, have)) return bfail(b, r, c->err);
    const size_t bytes = sizeof(double) * (size_t)c->model.m * c->model.nv * c->npoints;
    double* scratch = nullptr;
    if (cudaMalloc((void**)&scratch, bytes) != cudaSuccess) {
      cudaGetLastError();
      return bfail(b, PDG_ERR_OOM, "autotune scratch");
    }
    cudaMemcpyAsync(scratch, c->f, bytes, cudaMemcpyDeviceToDevice, c->stream);
    double* keep = c->f;
    c->f = scratch;
    int status = PDG_OK;
    int* d_ent = nullptr;
    long long* d_start = nullptr;
    unsigned long long* d_cnt = nullptr;
    PdgPass* d_p = nullptr;
    if (cudaMalloc((void**)&d_ent, sizeof(int)) || cudaMalloc((void**)&d_start, sizeof(long long)) ||
        cudaMalloc((void**)&d_cnt, sizeof(unsigned long long)) || cudaMalloc((void**)&d_p, sizeof(PdgPass))) {
      cudaGetLastError();
      status = bfail(b, PDG_ERR_OOM, "autotune tables");
    }
    const int zero_i = 0;
    const long long zero_l = 0;
    if (status == PDG_OK) {
      cudaMemcpy(d_ent, &zero_i, sizeof(int), cudaMemcpyHostToDevice);
      cudaMemcpy(d_start, &zero_l, sizeof(long long), cudaMemcpyHostToDevice);
    }
    int best_shape[2][3] = {{0, 0, 0}, {0, 0, 0}};
    for (int k = 0; k < 2 && status == PDG_OK; ++k) {
      if (!have[k]) continue;
      PdgPass p0;
      if ((status = make_pass(c, sp[k], pdg_batch_threads(), nullptr, &p0))) break;
      int W = 1;
      for (int q = 0; q < sp[k].ncs; ++q) W = std::max(W, stable_window(sp[k].cs[q]));
      float best = 1e30f;
      for (const Shape& s : shape_candidates(pdg_batch_threads(), p0.ncell, p0.ntf, W)) {
        int ov[3] = {s.lpb, s.nseg, s.ngroup};
        PdgPass p;
        if ((status = make_pass(c, sp[k], pdg_batch_threads(), ov, &p))) break;
        cudaMemcpyAsync(d_p, &p, sizeof(PdgPass), cudaMemcpyHostToDevice, c->stream);
        const long long total = (p.nlines + p.lpb - 1) / p.lpb;
        float ms = 0.f;
        status = time_launches(c, reps, [&]() {
          cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), c->stream);
          int er = pdg_launch_batch(d_p, d_ent, d_start, 1, total, d_cnt, b->smem, p.prec, p.npl / p.ncell, p.mv,
                                    (void*)c->stream);
          return er ? cuda_fail(c, (cudaError_t)er, "batch autotune launch") : PDG_OK;
        }, &ms);
        if (status) break;
        if (ms < best) {
          best = ms;
          best_shape[k][0] = s.lpb;
          best_shape[k][1] = s.nseg;
          best_shape[k][2] = s.ngroup;
        }
      }
    }
    cudaStreamSynchronize(c->stream);
    c->f = keep;
    cudaFree(scratch);
    cudaFree(d_ent);
    cudaFree(d_start);
    cudaFree(d_cnt);
    cudaFree(d_p);
    if (status) return bfail(b, status, c->err);
    for (int j = 0; j < n; ++j)
      if (rep[j] == i)
        for (int k = 0; k < 2; ++k)
          for (int q = 0; q < 3; ++q) b->inst[j]->bshape[k][q] = best_shape[k][q];
  }
  return PDG_OK;
}

int pdg_batch_destroy(pdg_batch* b) {
  if (!b) return PDG_OK;
  cudaStreamSynchronize(b->stream);
  if (b->cap) cudaStreamSynchronize(b->cap);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->d_desc) cudaFree(b->d_desc);
  if (b->d_ent_desc) cudaFree(b->d_ent_desc);
  if (b->d_ent_start) cudaFree(b->d_ent_start);
  if (b->d_counter) cudaFree(b->d_counter);
  if (b->e0) cudaEventDestroy(b->e0);
  if (b->e1) cudaEventDestroy(b->e1);
  if (b->ej) cudaEventDestroy(b->ej);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
  return PDG_OK;
}

}  // extern "C"
