// The project's autotuners: launch shapes of the line passes of one mesh (pdg_autotune)
// and of the batched classes of a batch (pdg_batch_autotune), timed with CUDA events on a
// scratch copy of the state.
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

}  // namespace pdgapi

using namespace pdgapi;

extern "C" {

int pdg_autotune(pdg_ctx* c, double dt, int reps) try {
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
} catch (...) {
  return pdgapi::abi_exception(c ? &c->err : nullptr);
}

int pdg_batch_autotune(pdg_batch* b, const double* dt, int reps) try {
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
} catch (...) {
  return pdgapi::abi_exception(b ? &b->err : nullptr);
}

}  // extern "C"
