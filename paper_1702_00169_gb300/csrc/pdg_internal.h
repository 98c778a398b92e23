// Internal declarations shared by the host plan, the kernels and the C ABI layer.
#pragma once

#include <cstddef>
#include <cstdint>

#define PDG_MAXN 5          // GL points per cell and axis (degree <= 4)
#define PDG_MAXM 5          // conserved variables (3-D Euler)
#define PDG_MAXF 30         // fields m * 2D
#define PDG_MAXOPS 4        // operations fused in one pass

// Per-cell coefficients of one theta transport sub-step along one axis, for the
// traversal direction of the velocity (negative velocities traverse the line
// backwards, which maps them onto the positive case: the GL nodes are symmetric).
//
// For cell c (traversal order) with old values f_c and new values fn_c:
//   fn_c = E f_c + q z_{c-1},   z_{c-1} = za x_{c-1} + zb u_{c-1},
// where x_{c-1} is the NEW and u_{c-1} the OLD value at the last node of the
// upwind cell.  The last node obeys the scalar periodic recurrence
//   x_c = alpha_c + beta x_{c-1},  alpha_c = (E f_c)_{n-1} + q_{n-1} zb u_{c-1},
//   beta = q_{n-1} za.
struct PdgCoef {
  double E[PDG_MAXN * PDG_MAXN];  // row-major n x n
  double q[PDG_MAXN];
  double za, zb, beta;
  // Launch-dependent fields.  With |beta| < 1 the recurrence runs downwind with
  // ratio r = beta; with |beta| > 1 (negative time steps) it runs upwind,
  // x_{c-1} = gamma (x_c - alpha_c) with r = gamma = 1/beta (rev = 1), which is
  // the stable direction.
  double gamma;           // 1 / beta when rev
  double betaL0, betaL1;  // r^Lbase, r^(Lbase+1): segment lengths of the launch
  double inv_ring;        // 1 / (1 - r^N)
  int W;                  // window (cells) when truncated
  int full;               // 1: aggregate whole segments and close the ring exactly
  int rev;                // 1: upwind recurrence (|beta| > 1)
  int W2;                 // window of the composed double step (0: not composable)
  // Two consecutive sub-steps T T with these coefficients, composed (forward, window mode):
  //   gn_c = E2 f_c + Eq z_{c-1} + q z'_{c-1},  E2 = E E,  Eq = E q,
  //   z = za x + zb u (first step), z' = za x' + zb x (second step),
  //   (x, x') last-node values of the two steps: x_c = (E f_c)_{n-1} + q_{n-1} z_{c-1},
  //   x'_c = (gn_c)_{n-1};  the pair obeys X_c = A_c + [[beta, 0], [gamma1, beta]] X_{c-1}
  //   with gamma1 = Eq_{n-1} za + q_{n-1} zb.
  double E2[PDG_MAXN * PDG_MAXN];
  double Eq[PDG_MAXN];
  double gamma1;
  // the same values as double-float pairs (hi, lo) for the double-float kernels
  float E_f[PDG_MAXN * PDG_MAXN][2];
  float q_f[PDG_MAXN][2];
  float za_f[1][2], zb_f[1][2], beta_f[1][2], gamma_f[1][2];
  float betaL0_f[1][2], betaL1_f[1][2], inv_ring_f[1][2];
  float E2_f[PDG_MAXN * PDG_MAXN][2];
  float Eq_f[PDG_MAXN][2];
  float gamma1_f[1][2];
};

// Model constants precomputed on the host (FP64 and as float pairs).
enum {
  PDG_K_OM1 = 0,    // 1 - omega
  PDG_K_C0 = 1,     // omega / (2D)
  PDG_K_C1 = 2,     // omega / (2 lambda)
  PDG_K_HALFG = 3,  // gravity / 2
  PDG_K_GM1 = 4,    // gamma - 1
  PDG_K_HALF = 5,   // 1/2
  PDG_K_CADV = 6,   // omega (1/(2D) + s_i a_axis / (2 lambda)), 6 entries
  PDG_K_N = 13
};
// The lattice models reuse the advection slots: omega W_0, omega W_axis, omega W_diag
// (edge), 1/6, 1/lambda, lambda, and one more slot for omega W_corner (D3Q15 / D3Q27).
enum { PDG_K_Q9W0 = 6, PDG_K_Q9W1 = 7, PDG_K_Q9W2 = 8, PDG_K_SIXTH = 9, PDG_K_ILAM = 10, PDG_K_LAM = 11,
       PDG_K_Q9W3 = 12 };

// D2Q9 state slots: populations 0-8 in the velocity order of Section 5.1, then four
// scratch slots.  The diagonal transport (populations 5-8) is computed out of place,
// so between the two diagonal sub-steps of a step the diagonal populations live in
// slots 9-12 (PdgPass::dslot tells the collision where they are).
#define PDG_Q9_SLOTS 13
#define PDG_Q9_DIAG 5
#define PDG_Q9_SCRATCH 9
// D3Q19: populations 0-18 (rest, six axis, twelve edge velocities: four per plane xy, xz,
// yz), then twelve scratch slots for the edge populations 7-18.
#define PDG_Q19_SLOTS 31
#define PDG_Q19_DIAG 7
#define PDG_Q19_SCRATCH 19
// D3Q15: populations 0-14 (rest, six axis, eight corners), then eight scratch slots for
// the corner populations 7-14.
#define PDG_Q15_SLOTS 23
#define PDG_Q15_DIAG 7
#define PDG_Q15_SCRATCH 15
// D3Q27: populations 0-26 (rest, six axis, twelve edges as in D3Q19, eight corners), then
// twenty scratch slots for populations 7-26.
#define PDG_Q27_SLOTS 47
#define PDG_Q27_DIAG 7
#define PDG_Q27_SCRATCH 27

struct PdgModel {
  int kind;      // PDG_MODEL_*
  int dim;       // D
  int m;         // conserved variables
  int nv;        // 2D
  int prec;      // PDG_PREC_*
  int nf;        // populations in f: m * nv (DnQ2n) or 9 (D2Q9)
  double lambda;
  double omega;
  double a[3];
  double gravity;
  double gamma;
  double cadv[6];  // advection: 1/(2D) + s_i a_axis / (2 lambda) per population (f^eq_i / w)
  double k[PDG_K_N];
  float k_f[PDG_K_N][2];
};

enum { PDG_OP_NONE = 0, PDG_OP_T = 1, PDG_OP_C = 2, PDG_OP_TT = 3 };

// Source stage S(delta) applied before and after the collision (see pdg_set_source):
// theta step of d/dt w = s(w) on (rho, rho u), gravity g and penalisation K(x) (w_s - w).
struct PdgSrc {
  int flags;               // PDG_SOURCE_* bits
  int pad_;
  const double* kfield;    // K at every point (FP64), when penalising
  double g[2], ws[3], theta, omtheta, delta;
  float g_f[2][2], ws_f[3][2], theta_f[1][2], omtheta_f[1][2], delta_f[1][2];
};

struct PdgPass {
  double* f;
  long long field_stride;  // points per field
  long long stride;        // point stride along the line
  long long lineA, s1, s2; // base(l) = (l % lineA) * s1 + (l / lineA) * s2
  int nlines;              // line positions in the pass
  int nblocks;             // > 0: blocks of the launch, lines spread evenly over them
                           //      (block b owns lines [b nlines / nblocks, (b+1) nlines / nblocks));
                           // 0: block b owns lines [b lpb, (b+1) lpb) (batched launches)
  int npl;                 // points per line, P = ncell * n
  int ncell;               // cells per line
  int nseg, lpb, ngroup;   // launch shape
  int nops;
  int op[PDG_MAXOPS];
  int opcoef[PDG_MAXOPS];
  int ntf;                     // transported fields
  int tfield[2 * PDG_MAXM];    // field index (k * 2D + i)
  int tdir[2 * PDG_MAXM];      // +1 / -1
  int mv;                      // model variant of the collision (MV_* of pdg_device.cuh)
  int prec;                    // PDG_PREC_* of the state and arithmetic
  int periodic;                // 1: periodic lines; 0: inflow boundary data fb
  int dslot;                   // D2Q9 collision: state slot of population 5 (5 or 9)
  int resident;                // 1: the line-resident kernel (the block's lines staged in shared
                               //    memory for the whole op list; periodic DnQ2n passes)
  int tmap;                    // thread map of the transport sweeps: 0 lines fastest, 1 field
                               //    groups fastest (set by the line-resident kernel)
  const double* fb;            // non-periodic: inflow values [2 sides][fbnent][nlines] (state format)
  int fbnent;                  // entries per side of fb (m; 3 for D2Q9)
  int fbent[2 * PDG_MAXM];     // entry of each transported population within its side
  PdgSrc src;                  // source stage around the collision (D2Q9), flags 0 = none
  PdgCoef coef[2];
  PdgModel model;
};

// A pass of the schedule before its launch shape is chosen.  axis >= 0: a line pass
// (ops on the populations along that axis, C on all); axis = -1: the D2Q9 diagonal
// transport T(ddelta) of populations 5-8 from slots dslot_in.. to the other slot set.
struct PdgPassSpec {
  int axis;
  int nops;
  int op[PDG_MAXOPS];
  int opcoef[PDG_MAXOPS];
  int ncs;
  int dslot;      // line pass with C on D2Q9: slot of population 5
  int dslot_in;   // diagonal pass: input slot of population 5 (output: the other set)
  double ddelta;  // diagonal pass: sub-step
  double sdelta;  // line pass with C: sub-step of the source stages around it (0: none)
  PdgCoef cs[2];
};

// Coefficients of one diagonal theta sub-step on an n x n-node cell (node p = iy n + ix,
// traversal orientation: the upwind neighbours are at -x and -y):
//   fn = Binv r - c1 f,  r = f / theta + kx S_x Lt + ky S_y Bt,  c1 = (1 - theta) / theta,
//   Lt = (1 - theta) L^old + theta L^new (values on the +x face of the -x neighbour,
//   one per row iy, entering node (iy, 0)), Bt likewise from the -y neighbour (one per
//   column ix, entering node (0, ix)); Binv = (I + theta (nu_x I(x)K + nu_y K(x)I))^-1,
//   kx = nu_x / w_0, ky = nu_y / w_0.
#define PDG_MAXNN (PDG_MAXN * PDG_MAXN)
struct PdgDiagCoef {
  double Binv[PDG_MAXNN * PDG_MAXNN];   // row-major NN x NN
  double rtheta, c1, theta, omtheta, kx, ky;
  int wx, wy;                            // halo columns / warm-up rows (cells)
  float Binv_f[PDG_MAXNN * PDG_MAXNN][2];
  float rtheta_f[1][2], c1_f[1][2], theta_f[1][2], omtheta_f[1][2], kx_f[1][2], ky_f[1][2];
};

// Launch descriptor of a diagonal pass: npop populations whose velocity has components
// along two axes a ("x") and b ("y") (traversal signs sx, sy), on an ncx x ncy cell grid
// of the (a, b) plane, repeated over nplane planes of points along the remaining axis;
// tiles of tx x ty output cells, each swept from wx columns and wy rows upwind.
struct PdgDiagPass {
  const double* fin[4];
  double* fout[4];
  int sx[4], sy[4];
  // inflow axes (per axis: 1 = periodic); boundary data [2 sides][nent][lines] of the faces
  // normal to a ("x") and b ("y") and each population's side and entry in it.  A point of
  // such a face has line index (coordinate along the other plane axis) * f?_ls +
  // (plane index) * f?_ps; f?_lines = lines of the face (the entry stride).
  int perx, pery;
  const double* fbx;
  const double* fby;
  int bxside[4], bxent[4], byside[4], byent[4];
  int nent;
  long long fbx_lines, fby_lines, fbx_ls, fbx_ps, fby_ls, fby_ps;
  int npop, n, ncx, ncy;
  long long sa, sb;       // point strides along a and b
  long long sc;           // point stride between planes
  int nplane;             // planes (points along the third axis; 1 in 2-D)
  int tx, ty, ntx, nty;   // tile shape and counts
  int threads;            // threads per block
  int prec;
  PdgDiagCoef c;
};

// Coefficients of one corner sub-step (velocity lambda (+-1, +-1, +-1)) on an n^3-node
// cell (node p = (iz n + iy) n + ix, traversal orientation: the upwind neighbours are at
// -x, -y and -z):
//   fn = Binv r - c1 f,  r = f / theta + kx S_x Lt + ky S_y Bt + kz S_z Zt,
//   Binv = (I + theta (nu_x I(x)I(x)K + nu_y I(x)K(x)I + nu_z K(x)I(x)I))^-1,
// Lt, Bt, Zt the theta-weighted values on the +x / +y / +z faces of the upwind
// neighbours (n^2 each), entering the nodes with ix = 0 / iy = 0 / iz = 0.  Binv itself
// (up to 64 x 64) lives in device memory (PdgCornerPass::binv).
#define PDG_MAXN_CORNER 4
struct PdgCornerCoef {
  double rtheta, c1, theta, omtheta, kx, ky, kz;
  int wx, wy, wz;   // upwind start widths (cells) along x, y, z
  float rtheta_f[1][2], c1_f[1][2], theta_f[1][2], omtheta_f[1][2], kx_f[1][2], ky_f[1][2], kz_f[1][2];
  // theta nu_a K (n x n, row-major) for a = x, y, z: B x = x + sum_a (theta nu_a K) x along a,
  // the residual stencil of the tensor-core form (FP64 and as float pairs)
  double kt[3][PDG_MAXN_CORNER * PDG_MAXN_CORNER];
  float kt_f[3][PDG_MAXN_CORNER * PDG_MAXN_CORNER][2];
};

// Launch descriptor of a corner pass: npop (<= 8) populations with traversal signs
// (sx, sy, sz) on an ncx x ncy x ncz periodic cell grid, in tiles of tx x ty x tz output
// cells, each swept from wx columns, wy rows and wz layers upwind.
struct PdgCornerPass {
  const double* fin[8];
  double* fout[8];
  int sx[8], sy[8], sz[8];
  int npop, n, ncx, ncy, ncz;
  long long sa, sb, sc;            // point strides along x, y, z
  int tx, ty, tz, ntx, nty, ntz;   // tile shape and counts
  int threads, prec;
  int tc;                          // 0: FP64 / double-float kernel; 1: tensor-core cell inverse with
                                   // an FP64 residual; 2: with a double-float residual
  const double* binv;              // device: NN x NN row-major (FP64)
  const float* binv_f;             // device: NN x NN (hi, lo) pairs (double-float)
  const float* binv_tc;            // device: Binv split into two TF32 MMA operands (tc != 0)
  int* err;                        // device error word of the tensor-core kernel (tc != 0)
  int stall;                       // test switch: the MMA wait watches an mbarrier nothing arrives
                                   // on, with a bound of about 0.5 ms, so it runs out
  int tc_layers;                   // tensor-core kernel: box layers swept together (1 or 2; 2 when
                                   // two anti-diagonals fit the 128 rows of a product)
  double* zt;                      // device scratch: per block [ty + wy][tx + wx][n^2] +z faces
  // hyperplane sweep of the whole region (hyper != 0; pdg_corner_hp.cuh): hg blocks per
  // population in a cooperative launch, batches of hnb cells, face slots hface
  // ([npop][2][3][nlay][nrow][n^2 rounded to even]) and one step counter per population
  int hyper, hg, hnb;
  double* hface;
  unsigned* hbar;
  // inflow axes (per axis a: per[a] = 1 periodic); boundary data fb[a] = [2 sides][nent][lines]
  // of the faces normal to a, each population's side and entry there; a face point's line
  // index is sum over the other axes b of (point coordinate along b) * fls[a][b]
  int per[3];
  const double* fb[3];
  int bside[3][8], bent[3][8];
  int nent;
  long long flines[3], fls[3][3];
  PdgCornerCoef c;
};

// Shared-memory line stride (8-byte words) of the line-resident kernel: the line length
// rounded up to an even count plus two words at most.  Staged lines then start 16-byte
// aligned, as lines do in global memory (unit-stride sweeps of even-degree cells move
// 16-byte pairs), and consecutive lines start on different banks.
#ifdef __CUDACC__
__host__ __device__
#endif
inline int pdg_resident_ls(int npl) { return (npl + 2) & ~1; }

// ---- read-only view of a context for entry points outside pdg_api.cu ----
#include <cuda_runtime.h>
#include <string>
struct pdg_ctx;
struct PdgStateView {
  const double* f;
  long long npoints;
  int m, nv, nf;
  int prec;
  cudaStream_t stream;
};
// Fills v and returns true when the context has a state.
bool pdg_internal_view(const pdg_ctx* c, PdgStateView* v);
// Records msg as the context's last error and returns code.
int pdg_internal_fail(pdg_ctx* c, int code, const std::string& msg);
namespace pdgapi {
// Status of a C++ exception that reached an exported entry point (every one of them catches
// all): PDG_ERR_OOM for a failed host allocation, PDG_ERR_ARG for anything else; the message
// goes to *err when given.  No exception crosses the C ABI.
int abi_exception(std::string* err) noexcept;
}  // namespace pdgapi
// Take the state of c from the stream-ordered pool (no device-wide synchronisation on free).
void pdg_internal_set_async_alloc(pdg_ctx* c, bool on);
// pdg_set_w without the final stream synchronisation (pageable sources are staged
// by the copy call itself; pinned sources must stay valid until the stream passes).
int pdg_internal_set_w_async(pdg_ctx* c, const double* w_host_pinned);
// Replace the instance list of a batch (the contexts must have models).
struct pdg_batch;
int pdg_internal_batch_set(pdg_batch* b, int n, pdg_ctx* const* ctxs);

// Host-side fault injection (pdg_debug_fail_allocs): 1 when the caller's device allocation
// must fail as out of memory (the counter of injected failures is decremented).
int pdg_fault_take_alloc();

// Capacity (doubles) of the static staging array of pdg_get_w_noalloc (8 MiB).
#define PDG_NOALLOC_W_MAX (1LL << 20)

// ---- host plan (pdg_plan.cpp) ----
// Gauss-Lobatto nodes/weights of degree d (ascending) and Dm[j*n+i] = l_i'(x_j).
int pdg_plan_gl(int d, double* x, double* w);
void pdg_plan_dmat(int n, const double* x, double* Dm);
// Transport coefficients for degree d, nu = 2 lambda delta / h, weight theta.
// Fills E, q, za, zb, beta (not the launch-dependent fields).  Returns 0 on success.
int pdg_plan_coef(int d, double nu, double theta, PdgCoef* c);
// Smallest K >= 1 with |beta|^K <= 2^-60 (window that makes truncation exact to rounding).
int pdg_plan_window(double beta);
// Fill E2, Eq, gamma1 of a coefficient set (n = order + 1) and return the window of the
// composed recurrence (|beta|^K and K |gamma1| |beta|^(K-1) <= 2^-60), 0 if |beta| >= 1.
int pdg_plan_compose(int n, PdgCoef* c);

// Split a double into a double-float pair (hi = nearest float, lo = nearest float of the rest).
inline void pdg_split(double x, float out[2]) {
  const float h = (float)x;
  out[0] = h;
  out[1] = (float)(x - (double)h);
}
// Fill the float-pair copies of a coefficient set / of the model constants.
void pdg_coef_split(PdgCoef* c);
void pdg_model_constants(PdgModel* m);
// Diagonal sub-step coefficients for degree d, nu_x, nu_y > 0, 0 < theta <= 1, and the
// halo / warm-up widths of the truncated tile start (influence <= 2^-56).  Returns 0, or
// -1 when the theta system is singular or no width <= 128 meets the bound.
int pdg_plan_diag(int d, double nux, double nuy, double theta, PdgDiagCoef* c);
// Corner sub-step coefficients for degree d <= 3, nu_x, nu_y, nu_z > 0, 0 < theta <= 1:
// fills c, binv[NN * NN] and binv_f[NN * NN * 2] (NN = (d+1)^3) and the start widths
// (influence <= 2^-57 per upwind face set).  Returns 0, or -1 when the system is singular
// or no width <= 64 meets the bound.
int pdg_plan_corner(int d, double nux, double nuy, double nuz, double theta, PdgCornerCoef* c, double* binv,
                    float* binv_f);

// ---- kernels (pdg_corner.cu, pdg_corner_tc.cu) ----
int pdg_launch_corner(const PdgCornerPass& p, void* stream);
size_t pdg_corner_smem(const PdgCornerPass& p);
int pdg_launch_corner_tc(const PdgCornerPass& p, size_t smem, void* stream);
size_t pdg_corner_tc_smem(const PdgCornerPass& p);
// Hyperplane form (pdg_corner_hp.cu): launch, shared memory of a block, and how many of
// its blocks fit one SM (0 when none does).
int pdg_launch_corner_hp(const PdgCornerPass& p, size_t smem, void* stream);
size_t pdg_corner_hp_smem(const PdgCornerPass& p);
int pdg_corner_hp_blocks_per_sm(const PdgCornerPass& p, size_t smem);
// The tensor-core operands of a corner plan: for n = d + 1, NN = n^3, K = NN rounded up to
// a multiple of 8 and N = max(16, K), two arrays (TF32 high parts, then low parts) of N x K
// floats each in the MMA's core-matrix layout (pdg_tc.cuh), zero beyond NN.  Returns the
// number of floats written (2 N K).
int pdg_corner_tc_operands(int n, const double* binv, float* out);
// 8-byte words of the +z face scratch (PdgCornerPass::zt) of a launch
size_t pdg_corner_scratch(const PdgCornerPass& p);

// ---- kernels (pdg_diag.cu) ----
int pdg_launch_diag(const PdgDiagPass& p, void* stream);
// dynamic shared memory (bytes) of one diagonal block
size_t pdg_diag_smem(const PdgDiagPass& p);

// ---- kernels (pdg_kernels.cu) ----
// Streaming multiprocessors of the current device (152 when no device answers).
int pdg_sm_count();
// All return a cudaError_t cast to int.
int pdg_launch_pass(const PdgPass& p, void* stream);
int pdg_launch_set_feq(double* f, long long npoints, const PdgModel& m, void* stream);
int pdg_launch_get_w(const double* f, double* w, long long npoints, const PdgModel& m, void* stream);
// The same on points [p0, p0 + n) of the npoints (field stride npoints).
int pdg_launch_set_feq_range(double* f, long long npoints, long long p0, long long n, const PdgModel& m,
                             void* stream);
int pdg_launch_get_w_range(const double* f, double* w, long long npoints, long long p0, long long n,
                           const PdgModel& m, void* stream);
// In-place conversion of n state values between FP64 and double-float (to_df != 0: FP64 -> pair).
int pdg_launch_convert(double* f, long long n, int to_df, void* stream);
// Model variant index used by the kernels (MV_* in pdg_device.cuh) for a model / pass.
int pdg_model_variant(const PdgModel& m);

// ---- batched persistent kernel (pdg_batch.cu) ----
int pdg_batch_threads();
size_t pdg_batch_smem(int max_carry_doubles);
// One persistent launch over the entries of one (precision, degree NP, model variant) group.
int pdg_launch_batch(const PdgPass* d_descs, const int* d_ent_desc, const long long* d_ent_start, int nent,
                     long long total, unsigned long long* d_counter, size_t smem, int prec, int np, int mv,
                     void* stream);
