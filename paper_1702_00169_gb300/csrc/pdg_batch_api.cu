// Batched execution of many independent meshes: persistent launches per stage and
// (precision, degree, model) group, work items claimed through an atomic counter, and the
// CUDA graph of a step sequence.
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

}  // namespace pdgapi

using namespace pdgapi;

// ---------------------------------------------------------------------------
// Batched execution of many independent meshes.


extern "C" const char* pdg_batch_last_error(const pdg_batch* b) { return b ? b->err.c_str() : "null batch"; }

extern "C" {

int pdg_batch_create(pdg_batch** out, int n, pdg_ctx* const* ctxs, void* cuda_stream) try {
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
} catch (...) {
  return pdgapi::abi_exception(nullptr);
}

int pdg_batch_step(pdg_batch* b, const double* dt, const int* nsteps, int use_graph) try {
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
} catch (...) {
  return pdgapi::abi_exception(b ? &b->err : nullptr);
}

int pdg_batch_elapsed(pdg_batch* b, double* ms, long long* launches) try {
  if (!b) return PDG_ERR_ARG;
  cudaError_t e = cudaEventSynchronize(b->e1);
  if (e != cudaSuccess) return bfail(b, PDG_ERR_CUDA, cudaGetErrorString(e));
  float t = 0.f;
  e = cudaEventElapsedTime(&t, b->e0, b->e1);
  if (e != cudaSuccess) return bfail(b, PDG_ERR_CUDA, cudaGetErrorString(e));
  if (ms) *ms = t;
  if (launches) *launches = b->last_launches;
  return PDG_OK;
} catch (...) {
  return pdgapi::abi_exception(b ? &b->err : nullptr);
}

int pdg_batch_destroy(pdg_batch* b) try {
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
} catch (...) {
  return pdgapi::abi_exception(b ? &b->err : nullptr);
}

}  // extern "C"
