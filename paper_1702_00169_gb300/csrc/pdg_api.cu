// C ABI of the PDG solver (include/pdg.h): mesh and model set-up, state transfer, the
// time step, inspection, timing and launch options of one context.  Every entry point
// returns a status; none lets a C++ exception through.
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

using namespace pdgapi;

namespace {
// pdg_set_w / pdg_get_w with host buffers: a state of at least kXferChunks * kXferChunkMin
// points moves in kXferChunks chunks of points, the copy of each chunk overlapping the
// equilibrium or moment kernel of its neighbour (smaller states: one copy, one kernel).
constexpr int kXferChunks = 8;
constexpr long long kXferChunkMin = 1LL << 19;
static_assert(kXferChunks + 1 <= (int)(sizeof(pdg_ctx::xev) / sizeof(cudaEvent_t)), "one event per chunk and one more");

int ensure_xfer(pdg_ctx* c) {
  if (!c->xstream) PDG_CUDA(c, cudaStreamCreateWithFlags(&c->xstream, cudaStreamNonBlocking));
  for (auto& e : c->xev)
    if (!e) PDG_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  return PDG_OK;
}
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

int pdg_debug_fail_allocs(int n) try {
  if (n < 0) return PDG_ERR_ARG;
  g_fail_allocs.store(n);
  return PDG_OK;
} catch (...) {
  return pdgapi::abi_exception(nullptr);
}

int pdg_create_mesh(pdg_ctx** out, int dim, const int n_macro[3], const int n_sub[3], int order,
                    const double length[3], unsigned periodic_mask, void* cuda_stream) try {
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
} catch (...) {
  return pdgapi::abi_exception(nullptr);
}

int pdg_set_model(pdg_ctx* c, const pdg_model_desc* d) try {
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
  if (lat && c->caxis >= 0 && c->caxis != c->dim - 1)
    return fail(c, PDG_ERR_UNSUPPORTED, "lattice models carry the collision in the last-axis pass");
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
} catch (...) {
  return pdgapi::abi_exception(c ? &c->err : nullptr);
}

int pdg_set_w(pdg_ctx* c, const double* w, size_t len, int on_device) try {
  if (!c) return PDG_ERR_ARG;
  if (!c->has_model) return fail(c, PDG_ERR_STATE, "pdg_set_w before pdg_set_model");
  if (!w) return fail(c, PDG_ERR_ARG, "w is NULL");
  const size_t need = (size_t)c->model.m * c->npoints;
  if (len != need) return fail(c, PDG_ERR_ARG, "w length mismatch");
  if (int r = ensure_state(c)) return r;
  if (int r = ensure_inflow(c)) return r;
  // w_k goes to field slot k; the kernel reads all w_k of a point before writing.
  if (!on_device && c->npoints >= kXferChunkMin * kXferChunks) {
    // large host state: chunk j's copies on the private stream, its equilibrium kernel on the
    // context stream after them, so that the kernel of chunk j runs during the copies of j + 1
    if (int r = ensure_xfer(c)) return r;
    const int m = c->model.m;
    const long long P = c->npoints;
    PDG_CUDA(c, cudaEventRecord(c->xev[kXferChunks], c->stream));   // earlier work on f first
    PDG_CUDA(c, cudaStreamWaitEvent(c->xstream, c->xev[kXferChunks], 0));
    // (a copy from pageable memory may return only once staged: each kernel is issued right
    // after its chunk's copies, before the next chunk's)
    for (int j = 0; j < kXferChunks; ++j) {
      const long long p0 = P * j / kXferChunks, p1 = P * (j + 1) / kXferChunks;
      for (int k = 0; k < m; ++k)
        PDG_CUDA(c, cudaMemcpyAsync(c->f + (long long)k * P + p0, w + (long long)k * P + p0,
                                    sizeof(double) * (size_t)(p1 - p0), cudaMemcpyHostToDevice, c->xstream));
      PDG_CUDA(c, cudaEventRecord(c->xev[j], c->xstream));
      PDG_CUDA(c, cudaStreamWaitEvent(c->stream, c->xev[j], 0));
      int e = pdg_launch_set_feq_range(c->f, P, p0, p1 - p0, c->model, (void*)c->stream);
      if (e) return cuda_fail(c, (cudaError_t)e, "set_feq launch");
    }
    PDG_CUDA(c, cudaStreamSynchronize(c->stream));
    c->has_state = true;
    return PDG_OK;
  }
  PDG_CUDA(c, cudaMemcpyAsync(c->f, w, sizeof(double) * need,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  int e = pdg_launch_set_feq(c->f, c->npoints, c->model, (void*)c->stream);
  if (e) return cuda_fail(c, (cudaError_t)e, "set_feq launch");
  if (!on_device) PDG_CUDA(c, cudaStreamSynchronize(c->stream));
  c->has_state = true;
  return PDG_OK;
} catch (...) {
  return pdgapi::abi_exception(c ? &c->err : nullptr);
}

int pdg_set_f(pdg_ctx* c, const double* f, size_t len, int on_device) try {
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
} catch (...) {
  return pdgapi::abi_exception(c ? &c->err : nullptr);
}

int pdg_get_f(pdg_ctx* c, double* out, size_t len, int on_device) try {
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
} catch (...) {
  return pdgapi::abi_exception(c ? &c->err : nullptr);
}

int pdg_get_w(pdg_ctx* c, double* out, size_t len, int on_device) try {
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
  if (!on_device && c->npoints >= kXferChunkMin * kXferChunks) {
    // large host result: chunk j's moment kernel on the context stream, its copies on the
    // private stream after it, so that the copies of chunk j run during the kernel of j + 1
    if (int r = ensure_xfer(c)) return r;
    const int m = c->model.m;
    const long long P = c->npoints;
    // the kernel of chunk j + 1 is issued before the copies of chunk j (a copy to pageable
    // memory may return only once it has completed)
    auto kernel = [&](int j) -> int {
      const long long p0 = P * j / kXferChunks, p1 = P * (j + 1) / kXferChunks;
      int e = pdg_launch_get_w_range(c->f, dst, P, p0, p1 - p0, c->model, (void*)c->stream);
      if (e) return cuda_fail(c, (cudaError_t)e, "get_w launch");
      PDG_CUDA(c, cudaEventRecord(c->xev[j], c->stream));
      return PDG_OK;
    };
    if (int r = kernel(0)) return r;
    for (int j = 0; j < kXferChunks; ++j) {
      if (j + 1 < kXferChunks)
        if (int r = kernel(j + 1)) return r;
      const long long p0 = P * j / kXferChunks, p1 = P * (j + 1) / kXferChunks;
      PDG_CUDA(c, cudaStreamWaitEvent(c->xstream, c->xev[j], 0));
      for (int k = 0; k < m; ++k)
        PDG_CUDA(c, cudaMemcpyAsync(out + (long long)k * P + p0, dst + (long long)k * P + p0,
                                    sizeof(double) * (size_t)(p1 - p0), cudaMemcpyDeviceToHost, c->xstream));
    }
    PDG_CUDA(c, cudaStreamSynchronize(c->xstream));
    PDG_CUDA(c, cudaStreamSynchronize(c->stream));
    return check_device_error(c);
  }
  int e = pdg_launch_get_w(c->f, dst, c->npoints, c->model, (void*)c->stream);
  if (e) return cuda_fail(c, (cudaError_t)e, "get_w launch");
  if (!on_device) {
    PDG_CUDA(c, cudaMemcpyAsync(out, dst, sizeof(double) * need, cudaMemcpyDeviceToHost, c->stream));
    PDG_CUDA(c, cudaStreamSynchronize(c->stream));
    if (int r = check_device_error(c)) return r;
  }
  return PDG_OK;
} catch (...) {
  return pdgapi::abi_exception(c ? &c->err : nullptr);
}

int pdg_set_source(pdg_ctx* c, const pdg_source_desc* d) try {
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
} catch (...) {
  return pdgapi::abi_exception(c ? &c->err : nullptr);
}

int pdg_step(pdg_ctx* c, double dt, int nsteps) try {
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
  if (graph) {
    std::vector<PdgPassSpec> sched;
    if (int r = build_schedule_checked(c, dt, nsteps, sched)) return r;
    if (int r = capture_steps(c, dt, nsteps, sched)) return r;
    return pdg_step(c, dt, nsteps);   // replay
  }
  // each pass is issued as it is generated: no pass list is held on the host
  return emit_schedule(c, dt, nsteps, [c](const PdgPassSpec& sp) { return issue_pass(c, sp); });
} catch (...) {
  return pdgapi::abi_exception(c ? &c->err : nullptr);
}

int pdg_set_inflow(pdg_ctx* c, int axis, const double* fb, size_t len, int on_device) try {
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
} catch (...) {
  return pdgapi::abi_exception(c ? &c->err : nullptr);
}

int pdg_get_points(const pdg_ctx* c, int axis, double* out, size_t len) try {
  if (!c || !out || axis < 0 || axis >= c->dim) return PDG_ERR_ARG;
  if (len != (size_t)c->P[axis]) return PDG_ERR_ARG;
  double x[PDG_MAXN], w[PDG_MAXN];
  if (pdg_plan_gl(c->order, x, w)) return PDG_ERR_ARG;
  const double h = c->h[axis];
  for (int cell = 0; cell < c->N[axis]; ++cell)
    for (int j = 0; j < c->n; ++j) out[(size_t)cell * c->n + j] = cell * h + 0.5 * h * (1.0 + x[j]);
  return PDG_OK;
} catch (...) {
  return pdgapi::abi_exception(nullptr);
}

int pdg_get_info(const pdg_ctx* c, pdg_info* info) try {
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
} catch (...) {
  return pdgapi::abi_exception(nullptr);
}

int pdg_get_line_coefs(const pdg_ctx* c, int axis, double delta, double* E, double* q, double* beta) try {
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
} catch (...) {
  return pdgapi::abi_exception(nullptr);
}

int pdg_get_schedule(pdg_ctx* c, double dt, int nsteps, int* ints, double* dbls, int max_passes, int* npasses) try {
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
} catch (...) {
  return pdgapi::abi_exception(c ? &c->err : nullptr);
}

int pdg_synchronize(pdg_ctx* c) try {
  if (!c) return PDG_ERR_ARG;
  PDG_CUDA(c, cudaStreamSynchronize(c->stream));
  return check_device_error(c);
} catch (...) {
  return pdgapi::abi_exception(c ? &c->err : nullptr);
}

int pdg_timing_enable(pdg_ctx* c, int enable) try {
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
} catch (...) {
  return pdgapi::abi_exception(c ? &c->err : nullptr);
}

int pdg_timing_read(pdg_ctx* c, long long* launches, double* ms, int max_kinds) try {
  if (!c || max_kinds < 0) return PDG_ERR_ARG;
  PDG_CUDA(c, cudaStreamSynchronize(c->stream));
  int r = drain_timing(c);
  if (r) return r;
  for (int k = 0; k < max_kinds && k < 5; ++k) {
    if (launches) launches[k] = c->t_launches[k];
    if (ms) ms[k] = c->t_ms[k];
  }
  return PDG_OK;
} catch (...) {
  return pdgapi::abi_exception(c ? &c->err : nullptr);
}

int pdg_set_launch(pdg_ctx* c, int kind, int lpb, int nseg, int ngroup) try {
  if (!c || kind < 0 || kind > 8) return PDG_ERR_ARG;
  c->gen++;
  if (kind == 7 || kind == 8) {   // line-resident kernel, pass kinds 0 / 1
    int* slot = c->rshape[kind - 7];
    if (lpb == 0 && nseg == 0 && ngroup == 0) {
      slot[0] = slot[1] = slot[2] = 0;
      return PDG_OK;
    }
    if (lpb < 1 || nseg < 1 || ngroup < 1 || (long long)lpb * nseg * ngroup > 512)
      return fail(c, PDG_ERR_ARG, "bad line-resident launch shape");
    slot[0] = lpb;
    slot[1] = nseg;
    slot[2] = ngroup;
    return PDG_OK;
  }
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
} catch (...) {
  return pdgapi::abi_exception(c ? &c->err : nullptr);
}

int pdg_destroy(pdg_ctx* c) try {
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
  if (c->xstream) {
    cudaStreamSynchronize(c->xstream);
    cudaStreamDestroy(c->xstream);
  }
  for (auto e : c->xev)
    if (e) cudaEventDestroy(e);
  free_inflow(c);
  delete c;
  return PDG_OK;
} catch (...) {
  return pdgapi::abi_exception(c ? &c->err : nullptr);
}

int pdg_set_option(pdg_ctx* c, int option, int value) try {
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
    case PDG_OPT_TC_LAYERS:
      if (value != 1 && value != 2) return fail(c, PDG_ERR_ARG, "tensor-core layers: 1 or 2");
      c->tc_layers = value;
      return PDG_OK;
    case PDG_OPT_RESIDENT:
      c->resident = value != 0;
      return PDG_OK;
    case PDG_OPT_CORNER_SWEEP:
      c->corner_sweep = value != 0;
      return PDG_OK;
    case PDG_OPT_COLLISION_AXIS: {
      Lattice Lat;
      if (value < -1 || value >= c->dim) return fail(c, PDG_ERR_ARG, "collision axis out of range");
      if (value >= 0 && value != c->dim - 1 && c->has_model && lattice_of(c->model.kind, &Lat))
        return fail(c, PDG_ERR_UNSUPPORTED, "lattice models carry the collision in the last-axis pass");
      c->caxis = value;
      return PDG_OK;
    }
  }
  return fail(c, PDG_ERR_ARG, "unknown option");
} catch (...) {
  return pdgapi::abi_exception(c ? &c->err : nullptr);
}

int pdg_get_launch(const pdg_ctx* c, int kind, int* lpb, int* nseg, int* ngroup) try {
  if (!c || kind < 0 || kind > 8 || !lpb || !nseg || !ngroup) return PDG_ERR_ARG;
  if (kind == 7 || kind == 8) {
    *lpb = c->rshape[kind - 7][0];
    *nseg = c->rshape[kind - 7][1];
    *ngroup = c->rshape[kind - 7][2];
    return PDG_OK;
  }
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
} catch (...) {
  return pdgapi::abi_exception(nullptr);
}

}  // extern "C"
