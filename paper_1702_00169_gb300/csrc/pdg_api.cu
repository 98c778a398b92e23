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

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
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
  int launch[2][3] = {{0, 0, 0}, {0, 0, 0}};
  bool timing = false;
  long long t_launches[3] = {0, 0, 0};
  double t_ms[3] = {0, 0, 0};
  std::vector<PdgTimedLaunch> pending;
  std::vector<cudaEvent_t> event_pool;
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

// Launch shape heuristic for one pass (lines per block, segments, field groups).
void choose_shape(const pdg_ctx* c, int kind, int nlines, int ncell, int ntf, int W, int* lpb, int* nseg,
                  int* ngroup) {
  const int* ov = c->launch[kind];
  if (ov[0] > 0) {
    *lpb = ov[0];
    *nseg = ov[1] < ncell ? ov[1] : ncell;
    *ngroup = ov[2] < ntf ? ov[2] : ntf;
    return;
  }
  int L = 8;
  if (nlines < L) L = nlines < 1 ? 1 : nlines;
  int G = ntf;
  const long long target = 152LL * 1024;
  long long s_target = (target + (long long)nlines * G - 1) / ((long long)nlines * G);
  int s_max_threads = 512 / (L * G);
  if (s_max_threads < 1) {
    G = 512 / L;
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
int finish_coef(PdgCoef* C, int N, int S) {
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
  if (!(std::fabs(1.0 - rN) > 1e-12)) return -1;
  C->inv_ring = 1.0 / (1.0 - rN);
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

// Issue one pass along `axis` with the op list (ops: PDG_OP_*, coef: index into cs).
int issue_pass(pdg_ctx* c, int axis, int nops, const int* ops, const int* coefidx, const PdgCoef* cs,
               int ncs) {
  PdgPass p;
  std::memset(&p, 0, sizeof(p));
  const int D = c->dim;
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
  p.ntf = 2 * m;
  for (int k = 0; k < m; ++k) {
    p.tfield[2 * k] = k * nv + 2 * axis;
    p.tdir[2 * k] = +1;
    p.tfield[2 * k + 1] = k * nv + 2 * axis + 1;
    p.tdir[2 * k + 1] = -1;
  }
  bool has_c = false;
  p.nops = nops;
  for (int o = 0; o < nops; ++o) {
    p.op[o] = ops[o];
    p.opcoef[o] = coefidx[o];
    has_c |= ops[o] == PDG_OP_C;
  }
  const int kind = has_c ? 1 : 0;
  int Wmax = 1;
  for (int i = 0; i < ncs; ++i) {
    int W = stable_window(cs[i]);
    if (W > Wmax) Wmax = W;
  }
  choose_shape(c, kind, p.nlines, p.ncell, p.ntf, Wmax, &p.lpb, &p.nseg, &p.ngroup);
  for (int i = 0; i < ncs && i < 2; ++i) {
    p.coef[i] = cs[i];
    if (finish_coef(&p.coef[i], p.ncell, p.nseg))
      return fail(c, PDG_ERR_ARG, "singular periodic transport system (|beta| = 1)");
  }
  p.model = c->model;
  (void)D;
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

// Allocate the kinetic state for the current model if it does not fit yet.
int ensure_state(pdg_ctx* c) {
  const long long need = (long long)c->model.m * c->model.nv * c->npoints;
  if (need <= c->f_cap) return PDG_OK;
  double* nf = nullptr;
  cudaError_t e = cudaMalloc((void**)&nf, sizeof(double) * (size_t)need);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, e == cudaErrorMemoryAllocation ? PDG_ERR_OOM : PDG_ERR_CUDA,
                std::string("cudaMalloc(f): ") + cudaGetErrorString(e));
  }
  if (c->f) cudaFree(c->f);
  c->f = nf;
  c->f_cap = need;
  c->has_state = false;
  return PDG_OK;
}

size_t fields_of(const pdg_ctx* c) { return (size_t)c->model.m * c->model.nv; }

}  // namespace

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
  const unsigned need = (1u << dim) - 1u;
  if ((periodic_mask & need) != need) return PDG_ERR_UNSUPPORTED;
  pdg_ctx* c = new (std::nothrow) pdg_ctx();
  if (!c) return PDG_ERR_OOM;
  c->dim = dim;
  c->order = order;
  c->n = order + 1;
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
  if (d->kind < PDG_MODEL_ADVECTION || d->kind > PDG_MODEL_EULER)
    return fail(c, PDG_ERR_ARG, "unknown model kind");
  if (d->scheme != PDG_SCHEME_M2 && d->scheme != PDG_SCHEME_M2_COLLAPSED)
    return fail(c, PDG_ERR_ARG, "unknown scheme");
  if (d->precision != PDG_PREC_FP64) return fail(c, PDG_ERR_UNSUPPORTED, "precision not available");
  if (!(d->lambda > 0.0 && std::isfinite(d->lambda))) return fail(c, PDG_ERR_ARG, "lambda must be > 0");
  if (!std::isfinite(d->omega) || d->omega == 0.0) return fail(c, PDG_ERR_ARG, "omega must be finite and != 0");
  if (!(d->theta >= 0.0 && d->theta <= 1.0)) return fail(c, PDG_ERR_ARG, "theta must be in [0, 1]");
  if (d->kind == PDG_MODEL_SHALLOW_WATER && c->dim != 2)
    return fail(c, PDG_ERR_UNSUPPORTED, "shallow water needs dim = 2");
  PdgModel M{};
  M.kind = d->kind;
  M.dim = c->dim;
  M.m = d->kind == PDG_MODEL_ADVECTION ? 1 : (d->kind == PDG_MODEL_SHALLOW_WATER ? 3 : c->dim + 2);
  M.nv = 2 * c->dim;
  M.lambda = d->lambda;
  M.omega = d->omega;
  for (int a = 0; a < 3; ++a) M.a[a] = d->a[a];
  M.gravity = d->gravity;
  M.gamma = d->gamma;
  for (int i = 0; i < M.nv; ++i) {
    const double s = (i % 2 == 0) ? 1.0 : -1.0;
    M.cadv[i] = 1.0 / (2.0 * c->dim) + s * d->a[i / 2] / (2.0 * d->lambda);
  }
  if (c->has_model && c->model.m != M.m) c->has_state = false;
  c->model = M;
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
  PDG_CUDA(c, cudaMemcpyAsync(c->f, f, sizeof(double) * need,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
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
  PDG_CUDA(c, cudaMemcpyAsync(out, c->f, sizeof(double) * need,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  if (!on_device) PDG_CUDA(c, cudaStreamSynchronize(c->stream));
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
  }
  return PDG_OK;
}

int pdg_step(pdg_ctx* c, double dt, int nsteps) {
  if (!c) return PDG_ERR_ARG;
  if (!c->has_state) return fail(c, PDG_ERR_STATE, "pdg_step before pdg_set_w / pdg_set_f");
  if (nsteps < 0 || !std::isfinite(dt)) return fail(c, PDG_ERR_ARG, "bad dt or nsteps");
  if (nsteps == 0) return PDG_OK;
  const int D = c->dim, L = D - 1;
  PdgCoef half[3], full[3];
  for (int a = 0; a < D; ++a) {
    if (plan_line_coef(c, a, 0.5 * dt, &half[a])) return fail(c, PDG_ERR_ARG, "singular transport step");
    if (plan_line_coef(c, a, dt, &full[a])) return fail(c, PDG_ERR_ARG, "singular transport step");
    // validate the periodic closure of every coefficient set before issuing any pass
    PdgCoef t0 = half[a], t1 = full[a];
    if (finish_coef(&t0, c->N[a], 1) || (c->scheme == PDG_SCHEME_M2_COLLAPSED && finish_coef(&t1, c->N[a], 1)))
      return fail(c, PDG_ERR_ARG, "singular periodic transport system (|beta| = 1)");
  }
  const int T = PDG_OP_T, C = PDG_OP_C;
  int r;
  if (c->scheme == PDG_SCHEME_M2) {
    for (int a = 0; a < L; ++a) {
      const int ops[1] = {T}, ci[1] = {0};
      if ((r = issue_pass(c, a, 1, ops, ci, &half[a], 1))) return r;
    }
    for (int s = 0; s < nsteps; ++s) {
      const int ops[3] = {T, C, T}, ci[3] = {0, 0, 0};
      if ((r = issue_pass(c, L, 3, ops, ci, &half[L], 1))) return r;
      for (int a = 0; a < L; ++a) {
        const int ops2[2] = {T, T}, ci2[2] = {0, 0};
        if ((r = issue_pass(c, a, s < nsteps - 1 ? 2 : 1, ops2, ci2, &half[a], 1))) return r;
      }
    }
  } else {
    for (int a = 0; a < L; ++a) {
      const int ops[1] = {T}, ci[1] = {0};
      if ((r = issue_pass(c, a, 1, ops, ci, &half[a], 1))) return r;
    }
    for (int s = 0; s < nsteps; ++s) {
      PdgCoef cs[2] = {half[L], full[L]};
      const int ops[2] = {T, C}, ci[2] = {s == 0 ? 0 : 1, 0};
      if ((r = issue_pass(c, L, 2, ops, ci, cs, 2))) return r;
      for (int a = 0; a < L; ++a) {
        const int ops2[1] = {T}, ci2[1] = {0};
        if ((r = issue_pass(c, a, 1, ops2, ci2, s < nsteps - 1 ? &full[a] : &half[a], 1))) return r;
      }
    }
    const int ops[1] = {T}, ci[1] = {0};
    if ((r = issue_pass(c, L, 1, ops, ci, &half[L], 1))) return r;
  }
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
  info->nv = 2 * c->dim;
  for (int a = 0; a < 3; ++a) {
    info->ncell[a] = c->N[a];
    info->npts[a] = c->P[a];
    info->h[a] = a < c->dim ? c->h[a] : 0.0;
  }
  info->npoints = c->npoints;
  info->nfields = (long long)info->m * info->nv;
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

int pdg_synchronize(pdg_ctx* c) {
  if (!c) return PDG_ERR_ARG;
  PDG_CUDA(c, cudaStreamSynchronize(c->stream));
  return PDG_OK;
}

int pdg_timing_enable(pdg_ctx* c, int enable) {
  if (!c) return PDG_ERR_ARG;
  if (!c->pending.empty()) {
    PDG_CUDA(c, cudaStreamSynchronize(c->stream));
    int r = drain_timing(c);
    if (r) return r;
  }
  c->timing = enable != 0;
  for (int k = 0; k < 3; ++k) {
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
  for (int k = 0; k < max_kinds && k < 3; ++k) {
    if (launches) launches[k] = c->t_launches[k];
    if (ms) ms[k] = c->t_ms[k];
  }
  return PDG_OK;
}

int pdg_set_launch(pdg_ctx* c, int kind, int lpb, int nseg, int ngroup) {
  if (!c || kind < 0 || kind > 1) return PDG_ERR_ARG;
  if (lpb == 0 && nseg == 0 && ngroup == 0) {
    c->launch[kind][0] = c->launch[kind][1] = c->launch[kind][2] = 0;
    return PDG_OK;
  }
  if (lpb < 1 || nseg < 1 || ngroup < 1 || (long long)lpb * nseg * ngroup > 512)
    return fail(c, PDG_ERR_ARG, "bad launch shape");
  c->launch[kind][0] = lpb;
  c->launch[kind][1] = nseg;
  c->launch[kind][2] = ngroup;
  return PDG_OK;
}

int pdg_destroy(pdg_ctx* c) {
  if (!c) return PDG_OK;
  if (c->stream || c->f) cudaStreamSynchronize(c->stream);
  for (auto& t : c->pending) {
    cudaEventDestroy(t.e0);
    cudaEventDestroy(t.e1);
  }
  for (auto e : c->event_pool) cudaEventDestroy(e);
  if (c->f) cudaFree(c->f);
  if (c->wstage) cudaFree(c->wstage);
  delete c;
  return PDG_OK;
}

}  // extern "C"
