// Serving loop with continuous batching: requests (independent PDG solves) are
// admitted into resident slots while the device memory budget allows, all resident
// solves advance together by batched launches (pdg_batch_step) in chunks of steps,
// and finished solves retire (result copied to host, state freed), which admits the
// next waiting requests.  Latency = completion time - arrival time (server clock).
//
// Built on the public C ABI (contexts, batches) plus two internal hooks: state from
// the stream-ordered pool, and an unsynchronised pdg_set_w from pinned host memory.
#include <cuda_runtime.h>

#include <chrono>
#include <cstring>
#include <deque>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/pdg.h"
#include "pdg_internal.h"

namespace {

struct Req {
  long long id = 0;
  pdg_request desc{};
  std::vector<double> w0;     // host copy of the initial state (released at admission)
  size_t w_len = 0;
  size_t state_bytes = 0;     // device footprint while resident
  long long dofs = 0;
  double t_arrival = 0, t_admit = 0, t_done = 0;
  int remaining = 0;
  pdg_ctx* ctx = nullptr;
};

struct Done {
  long long id;
  double t_arrival, t_admit, t_done;
};

}  // namespace

struct pdg_server {
  size_t budget = 0, resident_bytes = 0, peak_bytes = 0;
  int chunk = 10;
  int use_graph = 0;
  cudaStream_t stream = nullptr;
  std::chrono::steady_clock::time_point t0;
  long long next_id = 1;
  std::deque<Req*> waiting;
  std::vector<Req*> resident;
  std::deque<Done> done;                                    // not yet polled
  std::unordered_map<long long, std::vector<double>> results;  // not yet fetched
  std::unordered_map<long long, int> failed;                   // admission failed: status (not yet fetched)
  std::unordered_map<long long, char> cancelled;               // cancelled ids (not yet fetched)
  pdg_batch* batch = nullptr;
  long long iterations = 0, dof_updates = 0, admitted = 0, completed = 0, nfailed = 0, ncancelled = 0;
  std::string err;
};

namespace {

double now_s(const pdg_server* s) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

int sfail(pdg_server* s, int code, const std::string& m) {
  s->err = m;
  return code;
}

void free_req(Req* r) {
  if (r->ctx) pdg_destroy(r->ctx);
  delete r;
}

// Create the context of an admitted request and start its initial state upload.
int start_req(pdg_server* s, Req* r) {
  const pdg_request& d = r->desc;
  int st = pdg_create_mesh(&r->ctx, d.dim, d.n_macro, d.n_sub, d.order, nullptr, (1u << d.dim) - 1u,
                           (void*)s->stream);
  if (st) return sfail(s, st, "pdg_create_mesh failed for request " + std::to_string(r->id));
  pdg_internal_set_async_alloc(r->ctx, true);
  if ((st = pdg_set_model(r->ctx, &d.model))) return sfail(s, st, pdg_last_error(r->ctx));
  // pageable source: the copy has left r->w0 when the call returns
  if ((st = pdg_internal_set_w_async(r->ctx, r->w0.data()))) return sfail(s, st, pdg_last_error(r->ctx));
  std::vector<double>().swap(r->w0);
  return PDG_OK;
}

}  // namespace

extern "C" {

const char* pdg_server_last_error(const pdg_server* s) { return s ? s->err.c_str() : "null server"; }

int pdg_server_create(pdg_server** out, size_t mem_budget_bytes, int chunk_steps, int use_graph,
                      void* cuda_stream) try {
  if (!out) return PDG_ERR_ARG;
  *out = nullptr;
  if (mem_budget_bytes == 0 || chunk_steps < 1) return PDG_ERR_ARG;
  pdg_server* s = new (std::nothrow) pdg_server();
  if (!s) return PDG_ERR_OOM;
  s->budget = mem_budget_bytes;
  s->chunk = chunk_steps;
  s->use_graph = use_graph;
  s->stream = (cudaStream_t)cuda_stream;
  s->t0 = std::chrono::steady_clock::now();
  *out = s;
  return PDG_OK;
} catch (...) {
  return pdgapi::abi_exception(nullptr);
}

double pdg_server_now(const pdg_server* s) { return s ? now_s(s) : 0.0; }

int pdg_server_submit(pdg_server* s, const pdg_request* req, long long* id) try {
  if (!s || !req || !req->w0) return PDG_ERR_ARG;
  if (req->dim < 1 || req->dim > 3 || req->order < 1 || req->order > 4 || req->nsteps < 0 ||
      !(req->dt == req->dt))
    return sfail(s, PDG_ERR_ARG, "bad request");
  if (req->model.kind >= PDG_MODEL_ISOTHERMAL_D2Q9)
    return sfail(s, PDG_ERR_UNSUPPORTED, "lattice models (D2Q9 / D3Qq) run through pdg_step only");
  // sizes through a throw-away context (no device work)
  pdg_ctx* probe = nullptr;
  int st = pdg_create_mesh(&probe, req->dim, req->n_macro, req->n_sub, req->order, nullptr,
                           (1u << req->dim) - 1u, nullptr);
  if (st) return sfail(s, st, "bad request mesh");
  st = pdg_set_model(probe, &req->model);
  pdg_info info;
  if (!st) st = pdg_get_info(probe, &info);
  std::string perr = pdg_last_error(probe);
  pdg_destroy(probe);
  if (st) return sfail(s, st, "bad request model: " + perr);
  if (req->w0_len != (size_t)info.w_len) return sfail(s, PDG_ERR_ARG, "request w0 length mismatch");
  const size_t bytes = sizeof(double) * (size_t)info.f_len;
  if (bytes > s->budget) return sfail(s, PDG_ERR_ARG, "request larger than the memory budget");
  Req* r = new (std::nothrow) Req();
  if (!r) return sfail(s, PDG_ERR_OOM, "host allocation");
  r->id = s->next_id++;
  r->desc = *req;
  r->w_len = req->w0_len;
  r->state_bytes = bytes;
  r->dofs = info.f_len;
  r->remaining = req->nsteps;
  r->t_arrival = req->t_arrival;
  try {
    r->w0.assign(req->w0, req->w0 + r->w_len);
  } catch (...) {
    delete r;
    return sfail(s, PDG_ERR_OOM, "host allocation");
  }
  r->desc.w0 = nullptr;
  s->waiting.push_back(r);
  if (id) *id = r->id;
  return PDG_OK;
} catch (...) {
  return pdgapi::abi_exception(s ? &s->err : nullptr);
}

int pdg_server_iterate(pdg_server* s, int* n_resident, int* n_done) try {
  if (!s) return PDG_ERR_ARG;
  // 1. admission, first come first served, while the memory budget allows
  while (!s->waiting.empty()) {
    Req* r = s->waiting.front();
    if (s->resident_bytes + r->state_bytes > s->budget) break;
    s->waiting.pop_front();
    if (int st = start_req(s, r)) {
      // the request fails alone (e.g. the device is out of memory beyond the budget): its
      // status is kept for pdg_server_result and the others are served
      s->failed[r->id] = st;
      s->nfailed++;
      free_req(r);
      continue;
    }
    r->t_admit = now_s(s);
    s->resident_bytes += r->state_bytes;
    if (s->resident_bytes > s->peak_bytes) s->peak_bytes = s->resident_bytes;
    s->resident.push_back(r);
    s->admitted++;
  }
  int finished = 0;
  if (!s->resident.empty()) {
    // 2. one chunk of steps for every resident solve, in batched launches
    std::vector<pdg_ctx*> ctxs;
    std::vector<double> dts;
    std::vector<int> ns;
    for (Req* r : s->resident) {
      ctxs.push_back(r->ctx);
      dts.push_back(r->desc.dt);
      ns.push_back(r->remaining < s->chunk ? r->remaining : s->chunk);
    }
    int st;
    if (!s->batch) {
      if ((st = pdg_batch_create(&s->batch, (int)ctxs.size(), ctxs.data(), (void*)s->stream)))
        return sfail(s, st, "pdg_batch_create failed");
    } else if ((st = pdg_internal_batch_set(s->batch, (int)ctxs.size(), ctxs.data()))) {
      return sfail(s, st, "batch update failed");
    }
    if ((st = pdg_batch_step(s->batch, dts.data(), ns.data(), s->use_graph)))
      return sfail(s, st, pdg_batch_last_error(s->batch));
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return sfail(s, PDG_ERR_CUDA, cudaGetErrorString(e));
    s->iterations++;
    // 3. retirement
    std::vector<Req*> keep;
    for (size_t i = 0; i < s->resident.size(); ++i) {
      Req* r = s->resident[i];
      r->remaining -= ns[i];
      s->dof_updates += r->dofs * (long long)ns[i];
      if (r->remaining > 0) {
        keep.push_back(r);
        continue;
      }
      // moments through a stream-ordered temporary (no cudaMalloc / cudaFree synchronisation)
      std::vector<double> w(r->w_len);
      double* wdev = nullptr;
      e = cudaMallocAsync((void**)&wdev, sizeof(double) * r->w_len, s->stream);
      if (e != cudaSuccess) return sfail(s, PDG_ERR_OOM, std::string("result buffer: ") + cudaGetErrorString(e));
      if ((st = pdg_get_w(r->ctx, wdev, w.size(), 1))) {
        cudaFreeAsync(wdev, s->stream);
        return sfail(s, st, pdg_last_error(r->ctx));
      }
      e = cudaMemcpyAsync(w.data(), wdev, sizeof(double) * r->w_len, cudaMemcpyDeviceToHost, s->stream);
      cudaFreeAsync(wdev, s->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
      if (e != cudaSuccess) return sfail(s, PDG_ERR_CUDA, std::string("result copy: ") + cudaGetErrorString(e));
      r->t_done = now_s(s);
      s->results[r->id] = std::move(w);
      s->done.push_back({r->id, r->t_arrival, r->t_admit, r->t_done});
      s->resident_bytes -= r->state_bytes;
      s->completed++;
      finished++;
      free_req(r);
    }
    s->resident.swap(keep);
  }
  if (n_resident) *n_resident = (int)s->resident.size();
  if (n_done) *n_done = finished;
  return PDG_OK;
} catch (...) {
  return pdgapi::abi_exception(s ? &s->err : nullptr);
}

int pdg_server_pending(const pdg_server* s, int* n_waiting, int* n_resident) try {
  if (!s) return PDG_ERR_ARG;
  if (n_waiting) *n_waiting = (int)s->waiting.size();
  if (n_resident) *n_resident = (int)s->resident.size();
  return PDG_OK;
} catch (...) {
  return pdgapi::abi_exception(nullptr);
}

int pdg_server_poll(pdg_server* s, long long* ids, double* t_arrival, double* t_admit, double* t_done, int max,
                    int* count) try {
  if (!s || max < 0 || !count) return PDG_ERR_ARG;
  int n = 0;
  while (n < max && !s->done.empty()) {
    const Done& d = s->done.front();
    if (ids) ids[n] = d.id;
    if (t_arrival) t_arrival[n] = d.t_arrival;
    if (t_admit) t_admit[n] = d.t_admit;
    if (t_done) t_done[n] = d.t_done;
    s->done.pop_front();
    ++n;
  }
  *count = n;
  return PDG_OK;
} catch (...) {
  return pdgapi::abi_exception(s ? &s->err : nullptr);
}

int pdg_server_cancel(pdg_server* s, long long id) try {
  if (!s) return PDG_ERR_ARG;
  for (auto it = s->waiting.begin(); it != s->waiting.end(); ++it)
    if ((*it)->id == id) {
      free_req(*it);
      s->waiting.erase(it);
      s->cancelled[id] = 1;
      s->ncancelled++;
      return PDG_OK;
    }
  for (size_t i = 0; i < s->resident.size(); ++i)
    if (s->resident[i]->id == id) {
      // between iterations no launch of the server is in flight; pdg_destroy frees the
      // stream-ordered state after the server stream's pending work
      Req* r = s->resident[i];
      s->resident_bytes -= r->state_bytes;
      s->resident.erase(s->resident.begin() + (long)i);
      free_req(r);
      s->cancelled[id] = 1;
      s->ncancelled++;
      return PDG_OK;
    }
  return sfail(s, PDG_ERR_STATE, "no waiting or resident request with this id");
} catch (...) {
  return pdgapi::abi_exception(s ? &s->err : nullptr);
}

int pdg_server_result(pdg_server* s, long long id, double* w, size_t len) try {
  if (!s || !w) return PDG_ERR_ARG;
  auto fit = s->failed.find(id);
  if (fit != s->failed.end()) {
    const int st = fit->second;
    s->failed.erase(fit);
    return sfail(s, st, "request " + std::to_string(id) + " failed at admission");
  }
  auto cit = s->cancelled.find(id);
  if (cit != s->cancelled.end()) {
    s->cancelled.erase(cit);
    return sfail(s, PDG_ERR_STATE, "request " + std::to_string(id) + " was cancelled");
  }
  auto it = s->results.find(id);
  if (it == s->results.end()) return sfail(s, PDG_ERR_STATE, "no result for this id (not finished or fetched)");
  if (it->second.size() != len) return sfail(s, PDG_ERR_ARG, "result length mismatch");
  std::memcpy(w, it->second.data(), sizeof(double) * len);
  s->results.erase(it);
  return PDG_OK;
} catch (...) {
  return pdgapi::abi_exception(s ? &s->err : nullptr);
}

int pdg_server_stats(const pdg_server* s, long long* iterations, long long* dof_updates, long long* completed,
                     size_t* peak_bytes) try {
  if (!s) return PDG_ERR_ARG;
  if (iterations) *iterations = s->iterations;
  if (dof_updates) *dof_updates = s->dof_updates;
  if (completed) *completed = s->completed;
  if (peak_bytes) *peak_bytes = s->peak_bytes;
  return PDG_OK;
} catch (...) {
  return pdgapi::abi_exception(nullptr);
}

int pdg_server_destroy(pdg_server* s) try {
  if (!s) return PDG_OK;
  cudaStreamSynchronize(s->stream);
  if (s->batch) pdg_batch_destroy(s->batch);
  for (Req* r : s->resident) free_req(r);
  for (Req* r : s->waiting) free_req(r);
  cudaStreamSynchronize(s->stream);
  delete s;
  return PDG_OK;
} catch (...) {
  return pdgapi::abi_exception(s ? &s->err : nullptr);
}

}  // extern "C"
