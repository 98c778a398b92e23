// Helpers of the host-side context: error reporting, kernel timing, lattice tables, state
// and boundary-data allocation, the host-side fault injection, and the read-only views that
// other translation units use.
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

int abi_exception(std::string* err) noexcept {
  int code = PDG_ERR_ARG;
  const char* msg = "internal error";
  try {
    throw;
  } catch (const std::bad_alloc&) {
    code = PDG_ERR_OOM;
    msg = "host memory exhausted";
  } catch (const std::length_error&) {
    code = PDG_ERR_OOM;
    msg = "host memory exhausted";
  } catch (...) {
  }
  if (err) {
    try {
      *err = msg;
    } catch (...) {
    }
  }
  return code;
}

// Host-side fault injection: the next n state allocations fail as if the device were out
// of memory (pdg_debug_fail_allocs).
std::atomic<int> g_fail_allocs{0};

int fail(pdg_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(pdg_ctx* c, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(c, PDG_ERR_CUDA, m);
}

// After a synchronisation of the context stream: a bounded wait of a corner kernel that
// ran out (its error word set: the tensor-core kernel's wait for its products, or the
// hyperplane kernel's wait for the other blocks of its population) is reported once as
// PDG_ERR_TIMEOUT, and the word is cleared.  The state of the steps in flight then is
// incomplete.
int check_device_error(pdg_ctx* c) {
  if (!c->dev_err) return 0;
  int v = 0;
  PDG_CUDA(c, cudaMemcpyAsync(&v, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  PDG_CUDA(c, cudaStreamSynchronize(c->stream));
  if (!v) return 0;
  PDG_CUDA(c, cudaMemsetAsync(c->dev_err, 0, sizeof(int), c->stream));
  PDG_CUDA(c, cudaStreamSynchronize(c->stream));
  return fail(c, PDG_ERR_TIMEOUT, v == 2 ? "corner pass: a bounded wait for the other blocks of a hyperplane ran "
                                           "out; the state is incomplete"
                                         : "tensor-core corner pass: a bounded wait for the tensor cores ran out; "
                                           "the state is incomplete");
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

}  // namespace pdgapi

using namespace pdgapi;

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
