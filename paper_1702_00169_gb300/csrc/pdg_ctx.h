// Internal host-side state of the C ABI: the context, the batch, and the helpers shared by
// the ABI (pdg_api.cu), the pass schedule (pdg_schedule.cu), the pass issue
// (pdg_issue.cu), the autotuners (pdg_autotune.cu) and the batched execution
// (pdg_batch_api.cu).  Not installed; the public interface is include/pdg.h.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <functional>
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
  int tc_layers = 2;                           // PDG_OPT_TC_LAYERS
  int corner_sweep = 1;                        // PDG_OPT_CORNER_SWEEP (1 hyperplanes, 0 boxes)
  int resident = 0;                            // PDG_OPT_RESIDENT
  int rshape[2][3] = {{0, 0, 0}, {0, 0, 0}};   // line-resident shapes per pass kind (0 = heuristic)
  int caxis = -1;                              // PDG_OPT_COLLISION_AXIS (-1: the last axis)
  double* czt = nullptr;                       // corner pass: per-block +z face scratch (boxes) or
                                               // the face slots of the hyperplane sweep
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
  // host <-> device copies of pdg_set_w / pdg_get_w in chunks of points, overlapped with the
  // equilibrium and moment kernels of the neighbouring chunks (private stream and events)
  cudaStream_t xstream = nullptr;
  cudaEvent_t xev[9] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
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

namespace pdgapi {

#define PDG_CUDA(ctx, call)                                   \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return ::pdgapi::cuda_fail((ctx), e_, #call); \
  } while (0)

// Lattice models (one set of populations for all variables): D2Q9, D3Q19, D3Q15, D3Q27.
// Their non-axis populations [diag, diag + ndiag) run in diagonal passes, out of place
// between slots diag.. and scratch..: first norient planes of four edge velocities (a, b),
// then ncorner corner velocities.
struct Lattice {
  int slots, diag, scratch, ndiag, norient, ncorner;
};

// Unit velocities xi_i of the lattice models in population order (the orders of pdg.h):
// components (x, y, z); nullptr for the DnQ2n models.
struct LatticeTables {
  int q9[9][3], q19[19][3], q15[15][3], q27[27][3];
};

// Corner coefficient slots in pdg_ctx::cbuf: FP64 B^-1 (64 x 64 at most), its
// double-float copy, then its two TF32 operands of the tensor-core kernel, per slot; after
// the slots, the tensor-core kernel's error word.
#define PDG_CORNER_PLANS 4
constexpr size_t kCornerSlotBytes = 64 * 64 * (sizeof(double) + 2 * sizeof(float) + 2 * sizeof(float));
constexpr size_t kCornerTcOffset = 64 * 64 * (sizeof(double) + 2 * sizeof(float));
constexpr size_t kCornerErrBytes = 256;

// ---------------------------------------------------------------------------
// Autotuner: time candidate launch shapes of the two pass kinds on a scratch copy
// of the state and keep the fastest.


struct Shape {
  int lpb, nseg, ngroup;
};

// Pending injected allocation failures (pdg_debug_fail_allocs).
extern std::atomic<int> g_fail_allocs;

int fail(pdg_ctx* c, int code, const std::string& msg);
int cuda_fail(pdg_ctx* c, cudaError_t e, const char* what);
int check_device_error(pdg_ctx* c);
cudaEvent_t get_event(pdg_ctx* c);
int drain_timing(pdg_ctx* c);
bool lattice_of(int kind, Lattice* L);
LatticeTables make_lattice_tables();
const int* lattice_xi(int kind, int* q);
int inflow_entries(const PdgModel& m);
int inflow_entry(int kind, int axis, int i);
long long face_line_stride(const pdg_ctx* c, int A, int b);
long long state_slots(const pdg_ctx* c);
int ensure_state(pdg_ctx* c);
size_t fields_of(const pdg_ctx* c);
long long lines_of(const pdg_ctx* c, int a);
int ensure_inflow(pdg_ctx* c);
void free_inflow(pdg_ctx* c);
int finish_coef(PdgCoef* C, int N, int S, bool periodic = true);
int stable_window(const PdgCoef& C);
int plan_line_coef(const pdg_ctx* c, int axis, double delta, PdgCoef* C);
int pass_kind(const PdgPassSpec& sp);
PdgPassSpec spec(int axis, int nops, const int* ops, const int* ci, const PdgCoef* cs, int ncs);
// Receives the passes of a schedule in order; a non-zero return (a PDG_ERR_*) stops it.
using PassSink = std::function<int(const PdgPassSpec&)>;
int emit_line_schedule(pdg_ctx* c, double dt, int nsteps, const PassSink& sink);
int emit_schedule_one(pdg_ctx* c, double dt, int nsteps, const PassSink& sink);
int emit_schedule(pdg_ctx* c, double dt, int nsteps, const PassSink& sink);
int build_schedule(pdg_ctx* c, double dt, int nsteps, std::vector<PdgPassSpec>& out);
int build_schedule_checked(pdg_ctx* c, double dt, int nsteps, std::vector<PdgPassSpec>& out);
void choose_shape(const int* ov, int max_threads, int nlines, int ncell, int ntf, int W, int* lpb, int* nseg,
                  int* ngroup);
int make_pass(pdg_ctx* c, const PdgPassSpec& sp, int max_threads, const int* ov, PdgPass* out);
int launch_timed(pdg_ctx* c, const PdgPass& p, int kind);
int make_diag(pdg_ctx* c, const PdgPassSpec& sp, int o, PdgDiagPass* out);
int make_corner(pdg_ctx* c, const PdgPassSpec& sp, const Lattice& L, PdgCornerPass* out);
int issue_diag(pdg_ctx* c, const PdgPassSpec& sp);
void balance_blocks(PdgPass* p);
int issue_pass(pdg_ctx* c, const PdgPassSpec& sp);
bool resident_shape(const pdg_ctx* c, const PdgPassSpec& sp, int kind, int* shape);
int capture_steps(pdg_ctx* c, double dt, int nsteps, const std::vector<PdgPassSpec>& sched);
int bfail(pdg_batch* b, int code, const std::string& m);
std::vector<Shape> shape_candidates(int max_threads, int ncell, int ntf, int W);
int representative_specs(pdg_ctx* c, double dt, PdgPassSpec* sp, bool* have);

}  // namespace pdgapi
