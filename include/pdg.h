/*
 * pdg.h -- C ABI of the GB300 (sm_103a) Palindromic Discontinuous Galerkin solver.
 *
 * The library advances the kinetic BGK system of Badwaik et al., "Task-based
 * parallelization of an implicit kinetic scheme" (arXiv:1702.00169):
 *   - Section 2, eq. (2.1) kin_bgk: n_v = 2D transport equations at constant
 *     velocities +-lambda e_a, coupled by the relaxation towards f^eq(P f);
 *   - Section 3.1, eq. (3.7) DG_reduit: upwind nodal DG on Gauss-Lobatto points;
 *   - Section 3.2, eq. (3.11) transport_cn and eq. (3.12) collision_cn, composed
 *     as the palindrome M2(dt) = T(dt/2) C(dt) T(dt/2).
 * Meshes are periodic Cartesian boxes split into n_macro x n_sub cells per axis
 * (the macrocell / subcell structure of Section 4.3).
 *
 * Conventions common to every entry point
 *   - Every call returns a pdg_status (0 = PDG_OK, negative = error).  No C++
 *     exception crosses the ABI.  On error the context is left unchanged
 *     (except for the text returned by pdg_last_error) unless stated.
 *   - The caller owns every buffer it passes; the library never keeps a
 *     caller pointer after the call returns.  The context owns its device
 *     state (allocated with cudaMalloc on the current device).
 *   - A context is not thread-safe; distinct contexts are independent.
 *   - Work is issued on the context's CUDA stream.  Calls with host buffers
 *     synchronise that stream before returning; calls with device buffers and
 *     pdg_step are asynchronous with respect to the host.
 *
 * Data layout (both host and device buffers, FP64, C order):
 *   point index along axis a:  g_a = cell_a * (d+1) + node_a  (face points are
 *     duplicated, as in any DG method; P_a = N_a (d+1) with N_a = n_macro_a n_sub_a);
 *   one scalar field:          [P_z][P_y][P_x]  (x fastest; absent axes have P = 1);
 *   macroscopic state w:       [m][P_z][P_y][P_x];
 *   kinetic state f:           [m][2D][P_z][P_y][P_x], population i in the order
 *                              +x, -x, +y, -y, +z, -z;
 *                              D2Q9 (PDG_MODEL_ISOTHERMAL_D2Q9): [9][P_y][P_x] in the
 *                              velocity order of Section 5.1, lambda (0,0), (1,0), (0,1),
 *                              (-1,0), (0,-1), (1,1), (-1,1), (-1,-1), (1,-1);
 *                              D3Q19, D3Q15, D3Q27: [19 / 15 / 27][P_z][P_y][P_x] in
 *                              the orders of PDG_MODEL_ISOTHERMAL_D3Q19 / _D3Q15 / _D3Q27.
 */
#ifndef PDG_H
#define PDG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pdg_ctx pdg_ctx;

/* Status codes. */
enum {
  PDG_OK = 0,
  PDG_ERR_ARG = -1,         /* invalid argument (null pointer, size, range) */
  PDG_ERR_OOM = -2,         /* device or host allocation failed */
  PDG_ERR_CUDA = -3,        /* a CUDA runtime call failed (text in pdg_last_error) */
  PDG_ERR_STATE = -4,       /* call out of order (e.g. pdg_step before pdg_set_w) */
  PDG_ERR_TIMEOUT = -5,     /* a bounded device wait ran out */
  PDG_ERR_UNSUPPORTED = -6  /* valid request that this build does not implement */
};

/* Kinetic model kinds.  0-2: vectorial DnQ2n, each conserved variable has 2D
 * populations.  3: the D2Q9 lattice of Section 5.1 (Euler with gravity), one set of
 * nine populations for the isothermal Euler variables. */
enum {
  PDG_MODEL_ADVECTION = 0,     /* m = 1, flux q^a = a_a w                          */
  PDG_MODEL_SHALLOW_WATER = 1, /* D = 2, m = 3, w = (h, hu, hv), gravity g          */
  PDG_MODEL_EULER = 2,         /* D = 2 or 3, m = D + 2, w = (rho, rho u, E), gamma */
  PDG_MODEL_ISOTHERMAL_D2Q9 = 3, /* D = 2, m = 3, w = (rho, rho u_x, rho u_y), nine
                                  velocities lambda xi_i (xi in {-1,0,1}^2), equilibrium
                                  f_i = W_i rho (1 + u.v_i/c^2 + (u.v_i)^2/(2c^4)
                                  - u.u/(2c^2)), c = lambda/sqrt(3), W = 4/9, 1/9, 1/36
                                  (Section 5.1).  The four diagonal velocities couple each
                                  cell to two upwind faces: their transport is the 2-D
                                  recurrence of pdg_step's documentation.  Periodic or
                                  inflow axes (pdg_set_inflow); 0 < theta <= 1; dt > 0. */
  PDG_MODEL_ISOTHERMAL_D3Q19 = 4, /* D = 3, m = 4, w = (rho, rho u): the D3Q19 lattice of the
                                  paper's 3-D scaling runs (Section 4.5), velocities 0, the
                                  six lambda(+-e_a) (+x, -x, +y, -y, +z, -z) and the twelve
                                  lambda(+-e_a +- e_b) (planes xy, xz, yz, each (+,+), (-,+),
                                  (-,-), (+,-)); the equilibrium of the D2Q9 model with weights
                                  1/3, 1/18, 1/36 (reading: the paper prints no 3-D one).
                                  Each edge velocity acts in planes: its transport is the
                                  D2Q9 diagonal recurrence on every plane of points.
                                  Periodic or inflow axes; 0 < theta <= 1; dt > 0. */
  PDG_MODEL_ISOTHERMAL_D3Q15 = 5, /* D = 3, m = 4, w = (rho, rho u): the D3Q15 lattice of
                                  Section 4.5: velocities 0, the six lambda(+-e_a) and the
                                  eight corners lambda(+-1, +-1, +-1), ordered z = +1 first,
                                  then z = -1, each as (x, y) = (+,+), (-,+), (-,-), (+,-);
                                  the same equilibrium with weights 2/9, 1/9, 1/72.  A corner
                                  velocity couples each cell to three upwind faces: its
                                  transport is the 3-D recurrence of pdg_step's
                                  documentation.  Periodic or inflow axes; degree <= 3;
                                  0 < theta <= 1; dt > 0. */
  PDG_MODEL_ISOTHERMAL_D3Q27 = 6 /* D = 3, m = 4, w = (rho, rho u): the D3Q27 lattice of
                                  Section 4.5: the nineteen velocities of D3Q19 in its order,
                                  then the eight corners in the order of D3Q15; weights 8/27,
                                  2/27, 1/54, 1/216.  Periodic or inflow axes; degree <= 3;
                                  0 < theta <= 1; dt > 0. */
};

/* Time schemes (Section 3.2 and Section 5.1). */
enum {
  PDG_SCHEME_M2 = 0,          /* T(dt/2) C(dt) T(dt/2) per step                   */
  PDG_SCHEME_M2_COLLAPSED = 1, /* consecutive half transports merged into T(dt)   */
  PDG_SCHEME_M2KIN = 2,        /* T(dt/4) C(dt/2) T(dt/2) C(dt/2) T(dt/4): second order
                                  also as tau -> 0 (Section 3.2); omega is the weight of
                                  each C(dt/2) */
  PDG_SCHEME_M4KIN = 3         /* M2KIN(g1 dt) M2KIN(g2 dt) M2KIN(g1 dt), g1 = 1/(2 - 2^(1/3)),
                                  g2 = 1 - 2 g1 < 0: the symmetric triple jump of M2^kin,
                                  fourth order when M2^kin is time-symmetric (omega = 2);
                                  Section 3.2 states that palindromic compositions of M2^kin
                                  give any even order.  The middle sub-step runs backwards
                                  (anti-dissipative): stable for moderate Courant numbers
                                  only.  DnQ2n models on periodic axes (an inflow axis
                                  refuses the backward step); no sources. */
};

/* State format and arithmetic. */
enum {
  PDG_PREC_FP64 = 0, /* FP64 storage and FP64 arithmetic on every step */
  PDG_PREC_DF32 = 1, /* double-float: the state is stored as a pair of FP32 values
                        (hi + lo, about 48 significant bits, same 8 bytes per value) and
                        every step -- transport, moments, equilibrium, relaxation -- uses
                        double-word arithmetic built from error-free FP32 transformations
                        (GB300 runs FP32 at 61x its FP64 rate).  The ABI still exchanges
                        FP64 buffers: states are converted on pdg_set_w / pdg_set_f /
                        pdg_get_w / pdg_get_f (pair -> FP64 is exact).  Not a paper
                        feature: an accuracy/speed trade-off of this implementation
                        (relative L2 vs the FP64 reference <= 1e-12 on the tested
                        workloads). */
  PDG_PREC_TF32 = 2, /* the precision form of the dense cell inverses on the tensor cores
                        (D3Q15 / D3Q27 only; the state and every other step stay FP64):
                        the cell solves x = B^-1 r of the cells on a wavefront of the corner
                        sweep (B of eq. (3.7) under the theta step of eq. (3.11), Np x Np with
                        Np = (d+1)^3) run as one (cells x Np) . (Np x Np) product on the
                        tensor cores (tcgen05, TF32 operands, FP32 accumulation), each
                        operand split into two TF32 parts (hi + lo), then one refinement:
                        the residual r - B x in FP64 through the Kronecker sum B, a second
                        split product for the correction.  Error vs the FP64 path: about
                        1e-13 per cell solve; the tests hold it to relative L2 <= 1e-10. */
  PDG_PREC_TF32_DFRES = 3 /* as PDG_PREC_TF32, with the refinement residual in double-float
                             arithmetic on the FP32 pipes instead of FP64 */
};

/*
 * Model description.  Equilibrium (Section 2; the paper gives no DnQ2n formula,
 * reading): f^eq_{k,i} = w_k/(2D) + (v_i . q_k(w)) / (2 lambda^2), which satisfies
 * P f^eq = w and P V^a f^eq = q^a(w).
 *   kind       PDG_MODEL_*
 *   scheme     PDG_SCHEME_*
 *   precision  PDG_PREC_*
 *   lambda     lattice speed (> 0): velocities are +-lambda e_a
 *   a[3]       advection velocity (PDG_MODEL_ADVECTION)
 *   gravity    g (PDG_MODEL_SHALLOW_WATER)
 *   gamma      ratio of specific heats (PDG_MODEL_EULER)
 *   omega      relaxation weight of eq. (3.12): omega = 2 dt/(2 tau + dt); finite, != 0
 *              (physical range (0, 2]; a negative dt gives a negative omega)
 *   theta      implicit weight of the transport step, 0 <= theta <= 1 (1/2 = eq. (3.11))
 */
typedef struct pdg_model_desc {
  int kind;
  int scheme;
  int precision;
  int reserved;
  double lambda;
  double a[3];
  double gravity;
  double gamma;
  double omega;
  double theta;
} pdg_model_desc;

/* Sizes of a context (filled by pdg_get_info). */
typedef struct pdg_info {
  int dim;            /* D */
  int order;          /* d (d+1 GL points per cell and axis) */
  int m;              /* conserved variables (0 before pdg_set_model) */
  int nv;             /* populations per variable, 2D (D2Q9 / D3Q19: 9 / 19 in all) */
  int ncell[3];       /* N_a = n_macro_a n_sub_a (1 for absent axes) */
  int npts[3];        /* P_a = N_a (d+1) (1 for absent axes) */
  long long npoints;  /* prod_a P_a */
  long long nfields;  /* populations in f: m * 2D (D2Q9: 9, D3Q19: 19) */
  long long w_len;    /* m * npoints: doubles in w */
  long long f_len;    /* nfields * npoints: doubles in f */
  double h[3];        /* cell edge per axis */
} pdg_info;

/*
 * pdg_create_mesh -- create a context on a periodic Cartesian mesh.
 * Defines the mesh of Section 3.1 (cells L with the affine map tau_L, GL points
 * eq. (3.3)) grouped as in Section 4.3 (macrocells split into regular subcells).
 *   out            receives the new context (set to NULL on error)
 *   dim            D in {1, 2, 3}
 *   n_macro, n_sub macrocells and subcells per macrocell along x, y, z (first
 *                  dim entries read; each >= 1)
 *   order          DG degree d in {1, 2, 3, 4}
 *   length         box edge lengths (> 0; first dim entries read); NULL = unit box
 *   periodic_mask  bit a set = axis a periodic; bit clear = the axis ends at inflow /
 *                  outflow boundaries (eq. (2.6): each population takes the boundary
 *                  datum f^b at its inflow face, through the fictitious cells of
 *                  eq. (3.8); f^b = 0 until set with pdg_set_inflow)
 *   cuda_stream    cudaStream_t for all work of this context; NULL = legacy default stream
 * Allocates no device memory.  Errors: PDG_ERR_ARG, PDG_ERR_OOM.
 */
int pdg_create_mesh(pdg_ctx** out, int dim, const int n_macro[3], const int n_sub[3], int order,
                    const double length[3], unsigned periodic_mask, void* cuda_stream);

/*
 * pdg_set_model -- choose the kinetic model and time scheme (Section 2, Section 3.2).
 * Allocates nothing.  If the number of conserved variables changes, the previous
 * state is discarded and pdg_set_w or pdg_set_f must follow before pdg_step.
 * Errors: PDG_ERR_ARG, PDG_ERR_UNSUPPORTED (e.g. shallow water with D != 2).
 */
int pdg_set_model(pdg_ctx* ctx, const pdg_model_desc* desc);

/*
 * pdg_set_w -- set f := f^eq(w) at every GL point (equilibrium start; the paper
 * is silent on the initial kinetic data).
 *   w          macroscopic state, layout [m][P_z][P_y][P_x], len = m * npoints doubles
 *   on_device  1: w is a device pointer (read on the context stream, asynchronous);
 *              0: w is host memory (copied, then the stream is synchronised)
 * The first pdg_set_w / pdg_set_f after a model change allocates the device state
 * f (f_len doubles, cudaMalloc).  From host memory, a state of at least 8 * 2^19 points is
 * copied in 8 chunks of points on a private stream of the context (created on first use,
 * ordered after the work already on the context stream), each chunk's equilibrium kernel
 * running on the context stream during the next chunk's copy; the result is bitwise that
 * of one copy and one kernel.
 * Errors: PDG_ERR_STATE (no model), PDG_ERR_ARG (len mismatch, NULL), PDG_ERR_OOM, PDG_ERR_CUDA.
 */
int pdg_set_w(pdg_ctx* ctx, const double* w, size_t len, int on_device);

/*
 * Source terms of the split scheme M2^s(dt) = T(dt/2) S(dt/2) C(dt) S(dt/2) T(dt/2)
 * (Section 3.2; collapsed form of Section 5.1 with PDG_SCHEME_M2_COLLAPSED).  S is a
 * theta step of d/dt w = s(w) applied to the equilibrium part of f:
 *   w' = w + delta [theta s(w') + (1 - theta) s(w)],   f' = f + f^eq(w') - f^eq(w)
 * (reading: the paper applies the source "on the equilibrium part"; P f' = w').
 *   PDG_SOURCE_GRAVITY       s = (0, rho g)            (Section 5.1; g = gravity[0..1])
 *   PDG_SOURCE_PENALIZATION  s = -K(x) (w - w_s), K(x) = K_s exp(-kappa |x - x_c|^2) at the
 *                            GL points (Section 5.2; the paper prints the opposite sign
 *                            while describing a relaxation towards w_s)
 * Both may be combined.  Available for PDG_MODEL_ISOTHERMAL_D2Q9 (the model of both
 * source test cases of the paper) with PDG_SCHEME_M2 or PDG_SCHEME_M2_COLLAPSED.
 */
enum { PDG_SOURCE_GRAVITY = 1, PDG_SOURCE_PENALIZATION = 2 };
typedef struct pdg_source_desc {
  int flags;          /* PDG_SOURCE_* bits; 0 = no source */
  int reserved;
  double gravity[3];  /* g (x, y used) */
  double K_s;         /* penalisation amplitude (>= 0) */
  double kappa;       /* penalisation decay (>= 0) */
  double x_c[3];      /* penalisation centre (box coordinates; x, y used) */
  double w_s[5];      /* target state (rho, rho u_x, rho u_y) */
  double theta;       /* implicit weight of S, 0 <= theta <= 1 (1/2 = second order) */
} pdg_source_desc;

/*
 * pdg_set_source -- set (or, with desc NULL or flags 0, remove) the source of a context.
 * The penalisation frequency K(x) is evaluated once here at every GL point and kept on
 * the device (npoints doubles, cudaMalloc).  pdg_set_model removes the source.
 * Errors: PDG_ERR_STATE (no model), PDG_ERR_UNSUPPORTED (model or scheme without
 * sources), PDG_ERR_ARG (bad values), PDG_ERR_OOM, PDG_ERR_CUDA.
 */
int pdg_set_source(pdg_ctx* ctx, const pdg_source_desc* desc);

/*
 * pdg_step -- advance nsteps palindromic steps of size dt (Section 3.2):
 * M2(dt) = T(dt/2) C(dt) T(dt/2), with T the theta step
 * (I - theta delta L_h) F^new = (I + (1-theta) delta L_h) F^old of eq. (3.11),
 * solved exactly on the periodic mesh, and C eq. (3.12).  With
 * PDG_SCHEME_M2_COLLAPSED the interior half transports are merged into T(dt)
 * (collapsed Strang of Section 5.1); PDG_SCHEME_M2KIN advances M2^kin steps,
 * PDG_SCHEME_M4KIN steps of its triple-jump composition.
 * Asynchronous on the context stream.
 * dt may be negative (time-symmetric use).  nsteps = 0 is a no-op.
 * D2Q9 diagonal velocities v = lambda (s_x, s_y): on a Cartesian cell eq. (3.7) splits
 * into one line operator per axis, and the theta step couples a cell to the NEW values
 * on the faces of its two upwind neighbours,
 *   f_c^new = B^-1 [f_c/theta + (nu_x/w_0) S_x Lt + (nu_y/w_0) S_y Bt] - ((1-theta)/theta) f_c,
 *   B = I + theta (nu_x I (x) K + nu_y K (x) I),  Lt = (1-theta) L^old + theta L^new
 * (L, B: downwind-face values of the upwind neighbours along x and y).  The periodic
 * 2-D recurrence is solved on tiles swept as wavefronts; every tile starts W cells
 * upwind along both axes, W chosen on the host so that the influence of the
 * truncated start (bounded by the sum over lattice paths of the face recurrence's
 * transfer matrices) is below 2^-56 of the state's magnitude.  dt must be > 0 there
 * (PDG_ERR_UNSUPPORTED otherwise, or when no such W <= 128 exists).  On an inflow axis
 * the tiles that reach the inflow face start there, from the exact boundary data.
 * D3Q15 / D3Q27 corner velocities v = lambda (s_x, s_y, s_z): the same form with three
 * upwind faces, B = I + theta (nu_x I(x)I(x)K + nu_y I(x)K(x)I + nu_z K(x)I(x)I) on the
 * n^3 nodes of a cell.  By default each corner population sweeps the whole mesh, from a
 * start W cells upwind along every periodic axis, cell hyperplane by cell hyperplane
 * (PDG_OPT_CORNER_SWEEP); otherwise boxes of cells are swept layer by layer along z, each
 * layer as a 2-D wavefront, every box starting W cells upwind along all three axes (bound
 * 2^-57 per upwind boundary; W <= 64, otherwise PDG_ERR_UNSUPPORTED).  The first step with
 * a new (dt, scheme) plan copies the corner coefficients to the device (a few tens of KB,
 * in memory allocated by pdg_set_model).  The corner pass keeps the faces passed between
 * cells in a device scratch buffer (hyperplanes: 6 slots of n^2 doubles, rounded up to an
 * even count, per (layer, row) of each population's region, about 80 MB at 384^3 points;
 * boxes: the +z faces of each box's region); the first step that needs a larger one
 * allocates it with cudaMalloc (after a cudaFree of the old one, which waits for the
 * device), so issue a first step before any stream capture.
 * Pass order (M2): transports of different axes act on different populations and commute,
 * so between two collisions the trailing T(dt/2) of one step and the leading T(dt/2) of the
 * next run in one pass per axis (composed, PDG_OPT_COMPOSE_TT), the collision at the end of
 * the last axis' pass; each population sees the order of the definition.
 * Host memory: the passes are generated and issued one at a time, so the host memory of the
 * call does not depend on nsteps.  The schedule's own checks (time step, scheme, model) come
 * before the first pass is issued; a pass that cannot be planned (PDG_ERR_UNSUPPORTED) ends
 * the call after the passes before it.  With PDG_OPT_GRAPH the call first builds its pass
 * list for the capture, about 2.3 KB per pass (D passes per step for M2 and the collapsed
 * form, about 2D for M2^kin and 6D for M4^kin, plus one per diagonal sub-step of the
 * lattices); a list that cannot be allocated fails the call with PDG_ERR_OOM before anything
 * is issued.
 * Errors: PDG_ERR_STATE (no state), PDG_ERR_ARG (nsteps < 0, non-finite dt), PDG_ERR_OOM,
 *         PDG_ERR_CUDA, PDG_ERR_UNSUPPORTED.
 */
int pdg_step(pdg_ctx* ctx, double dt, int nsteps);

/*
 * pdg_get_w -- moments w_k = sum_i f_{k,i} (eq. (2.2) micro_to_macro), FP64.
 *   out        layout [m][P_z][P_y][P_x], len = m * npoints doubles
 *   on_device  1: out is a device pointer (written on the context stream, asynchronous);
 *              0: host memory (the stream is synchronised before returning)
 * A host read uses a device staging buffer of len doubles, allocated on first use; from a
 * state of at least 8 * 2^19 points it is copied out in 8 chunks of points on the private
 * stream of pdg_set_w, each during the moment kernel of the next chunk.
 * Errors: PDG_ERR_STATE, PDG_ERR_ARG, PDG_ERR_OOM, PDG_ERR_CUDA.
 */
int pdg_get_w(pdg_ctx* ctx, double* out, size_t len, int on_device);

/*
 * pdg_get_f / pdg_set_f -- read or overwrite the kinetic state f (the only state
 * the scheme keeps, the "low-storage" property of Section 4.4); a get/set pair
 * is a checkpoint / restore.  Layout [m][2D][P_z][P_y][P_x], len = f_len doubles.
 * on_device as for pdg_get_w / pdg_set_w.  Errors: PDG_ERR_STATE, PDG_ERR_ARG, PDG_ERR_CUDA.
 */
int pdg_get_f(pdg_ctx* ctx, double* out, size_t len, int on_device);
int pdg_set_f(pdg_ctx* ctx, const double* f, size_t len, int on_device);

/*
 * pdg_set_inflow -- boundary data f^b of a non-periodic axis (eq. (2.6) with the
 * fictitious cells of eq. (3.8): f^b is constant in time).  On such an axis the upwind
 * graph is acyclic (Section 4.1) and each line is swept from its inflow face with no
 * cyclic closure.
 *   fb   [2][m][lines] doubles: side 0 = the low face (x_a = 0), read by the +lambda e_a
 *        populations; side 1 = the high face, read by the -lambda e_a populations; lines
 *        are the points of the other axes in C order ([P_z][P_y] for axis 0, [P_z][P_x]
 *        for axis 1, [P_y][P_x] for axis 2); len = 2 * m * lines.
 *        Lattice models: [2][q_f][lines], the q_f populations entering through that face
 *        (xi_a > 0 at the low face, xi_a < 0 at the high face) in increasing population
 *        index; len = 2 * q_f * lines.  D2Q9: q_f = 3 (low x face: 1, 5, 8; high x face:
 *        3, 6, 7; low y face: 2, 5, 6; high y face: 4, 7, 8).  D3Q19 and D3Q15: q_f = 5
 *        (low x face: 1, 7, 10, 11, 14 in both orders); D3Q27: q_f = 9 (low x face: 1, 7,
 *        10, 11, 14, 19, 22, 23, 26).
 *   on_device as for pdg_set_w.  Kept until the next pdg_set_inflow or a model change
 *   (which resets it to zero).  Time steps that make |beta| > 1 (dt < 0) are not
 *   supported on inflow axes (pdg_step returns PDG_ERR_UNSUPPORTED).
 * Errors: PDG_ERR_STATE (no model), PDG_ERR_ARG (periodic axis, length), PDG_ERR_OOM, PDG_ERR_CUDA.
 */
int pdg_set_inflow(pdg_ctx* ctx, int axis, const double* fb, size_t len, int on_device);

/*
 * pdg_get_points -- physical GL coordinates along one axis (eq. (3.3) map_GL:
 * x = c h + (h/2)(1 + x^_j)), computed by the library's own quadrature.
 *   axis  0..dim-1;  out: host buffer of len = P_axis doubles.
 * Errors: PDG_ERR_ARG.
 */
int pdg_get_points(const pdg_ctx* ctx, int axis, double* out, size_t len);

/* pdg_get_info -- sizes of the context (see pdg_info).  Errors: PDG_ERR_ARG. */
int pdg_get_info(const pdg_ctx* ctx, pdg_info* info);

/*
 * pdg_get_line_coefs -- the per-cell transport coefficients the sweep uses for
 * axis-aligned velocity +lambda e_axis and sub-step delta (host, for inspection
 * and tests): E = B^{-1}(I - (1-theta) nu K) (n x n, row-major), the inflow
 * vector q, and the ratio beta of the periodic inflow recurrence, where
 * nu = 2 lambda delta / h_axis, K = Dm + w_0^{-1} e_0 e_0^T, B = I + theta nu K.
 *   E: n*n doubles, q: n doubles, beta: 1 double (n = order + 1).
 * Errors: PDG_ERR_STATE (no model), PDG_ERR_ARG.
 */
int pdg_get_line_coefs(const pdg_ctx* ctx, int axis, double delta, double* E, double* q, double* beta);

/*
 * pdg_get_schedule -- the pass list pdg_step(ctx, dt, nsteps) would issue, for inspection
 * and tests (host only: builds the list and launches nothing; needs a model, no state).
 * Section 3.2's compositions (M2, the collapsed form of Section 5.1, M2^kin, M4^kin) are
 * issued as passes over the axes: transports of different populations commute, so the
 * transports of each axis between two collisions are grouped into line passes, and the
 * collision is fused in the pass of the last axis.  Pass i is written as 8 ints at
 * ints[8 i] and 10 doubles at dbls[10 i]:
 *   ints   kind (0 line pass, 1 diagonal sub-step: the tile / box launches of every
 *          velocity with several nonzero components, 2 copy of those populations back to
 *          their home slots), axis (line pass; -1 / -2 otherwise), nops and op[4] (line pass:
 *          1 = transport T, 2 = collision C, in order), slot (line pass: where the collision
 *          reads the diagonal populations; diagonal sub-step: the slot set it reads)
 *   dbls   per op o of a line pass, 2 o and 2 o + 1: E[0][0] and beta of the transport's line
 *          plan (as pdg_plan_line returns them for its sub-step; 0 for C); 8: the sub-step of a
 *          diagonal sub-step; 9: the sub-step of the source stages around a collision (0: none)
 *   npasses receives the number of passes.  ints = dbls = NULL queries the count only.
 * Errors: PDG_ERR_STATE (no model), PDG_ERR_ARG (NULL npasses, nsteps < 0, dt not finite,
 * max_passes below the count, a singular step), PDG_ERR_OOM (no host memory for the list, as
 * pdg_step), PDG_ERR_UNSUPPORTED (as pdg_step).
 */
int pdg_get_schedule(pdg_ctx* ctx, double dt, int nsteps, int* ints, double* dbls, int max_passes, int* npasses);

/*
 * pdg_get_w_noalloc -- pdg_get_w into HOST memory without allocating device memory.
 * The paper has no counterpart: this entry point exists for callers that cannot let
 * the library call cudaMalloc (a pooled or custom allocator owns the device budget,
 * allocation calls are intercepted or forbidden after start-up, or the footprint must
 * not grow between two checkpoints).  pdg_get_w stages a host read in a device buffer
 * it allocates on first use; this variant stages it in a static array compiled into
 * the library instead: 1,048,576 doubles (8 MiB), held on every GPU that loads the
 * library until the process exits.  It calls no cudaMalloc / cudaFree.
 *   out  host buffer of len = m * npoints doubles, layout [m][P_z][P_y][P_x]
 * Behaviour: writes the whole staged range before copying it (nothing in the array
 * needs to start at zero); synchronises the context stream before returning.  The
 * first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current and keeps it for the life of the process; make that first
 * call before any stream capture.  The kept address assumes the device's primary
 * context lives as long as the library: a caller that runs cudaDeviceReset must not
 * call this entry point on that device afterwards (the reset unloads the array).  All
 * calls share the one array: calls whose GPU work overlaps (other contexts on other
 * streams, or other host threads) race on it and must be serialised by the caller.
 * Errors: PDG_ERR_STATE (no state), PDG_ERR_ARG (NULL, len mismatch, or len greater
 * than 1,048,576: use pdg_get_w), PDG_ERR_UNSUPPORTED (a PDG_PREC_DF32 state, or a
 * lattice model: D2Q9, D3Q15, D3Q19, D3Q27, whose w is not a sum of m groups of 2D
 * populations; use pdg_get_w for those), PDG_ERR_CUDA.
 */
int pdg_get_w_noalloc(pdg_ctx* ctx, double* out, size_t len);

/* pdg_synchronize -- wait for all work issued on the context stream.  Errors: PDG_ERR_CUDA,
 * PDG_ERR_TIMEOUT (a tensor-core corner pass gave up a bounded wait for its tensor-core
 * work, about one second; the state is incomplete; reported once, also by the host paths
 * of pdg_get_w / pdg_get_f). */
int pdg_synchronize(pdg_ctx* ctx);

/*
 * Kernel timing.  When enabled, pdg_step records CUDA events on the context
 * stream around every launch and accumulates, per kernel kind, the number of
 * launches and their summed duration (read back after a synchronisation).
 *   kind 0 = transport pass (axes before the last; T or T T, no collision)
 *   kind 1 = last-axis pass (T, fused collision, T)
 *   kind 2 = state kernels (set_w / get_w)
 *   kind 3 = diagonal transport pass (D2Q9 diagonals, D3Q19 / D3Q27 edges)
 *   kind 4 = corner transport pass (D3Q15 / D3Q27)
 * pdg_timing_enable(ctx, 1) resets the counters.  pdg_timing_read fills up to
 * max_kinds entries of launches[] and ms[] and synchronises the stream.
 */
int pdg_timing_enable(pdg_ctx* ctx, int enable);
int pdg_timing_read(pdg_ctx* ctx, long long* launches, double* ms, int max_kinds);

/*
 * pdg_set_launch -- override the launch shape of one pass kind: kind 0 / 1 as above
 * for pdg_step launches (lpb*nseg*ngroup <= 512), kind 2 / 3 for the same pass kinds
 * inside batched launches (lpb*nseg*ngroup <= 256):
 *   lpb    lines per thread block (>= 1), nseg: segments per line (>= 1),
 *   ngroup field groups per block (>= 1).
 * kind 4 = D2Q9 diagonal pass: lpb = threads per block (a multiple of 32, 64..512),
 *   nseg x ngroup = output cells per tile along x and y (>= 1; the tile counts follow).
 * kind 5 = D3Q15 / D3Q27 corner pass: lpb = threads per block (a multiple of 32, 64..512,
 *   at least (d+1)^3), nseg = output cells per box along x and y, ngroup = along z.
 * kind 6 = the corner box alone: lpb, nseg, ngroup = output cells per box along x, y, z
 *   (>= 1 each); the threads per block stay as kind 5 set them (512 when unset).
 * kind 7 / 8 = the line-resident kernel (PDG_OPT_RESIDENT) for pass kinds 0 / 1: lines per
 *   block, segments per line, field groups (lpb*nseg*ngroup <= 512); a shape whose staged
 *   lines exceed ~220 KB of shared memory makes the pass run the streaming kernel.
 * All zeros restores the built-in heuristic (kind 6: the box only).  Used by the
 * autotuners and by tests that force a box shape.
 * Errors: PDG_ERR_ARG.
 */
int pdg_set_launch(pdg_ctx* ctx, int kind, int lpb, int nseg, int ngroup);

/*
 * pdg_set_option -- implementation switches of a context.
 *   PDG_OPT_COMPOSE_TT (default 1): two consecutive transport sub-steps with the same
 *     coefficients (the T(dt/2) T(dt/2) of consecutive palindromic steps) run as one
 *     composed sweep, fn = E^2 f + (E q) z + q z', with a 2x2 inflow recurrence; the
 *     same operator, about 27 % fewer operations per cell at degree 3, results equal
 *     up to rounding.  0 runs them as two sweeps.
 *   PDG_OPT_GRAPH (default 0): pdg_step captures its launches for (dt, nsteps) into a CUDA
 *     graph on a private stream and replays it while dt, nsteps and the configuration stay
 *     the same (any set_model / set_w reallocation / set_inflow / set_source / set_launch /
 *     set_option / autotune call forces a new capture); the replay is ordered after the
 *     work already on the context stream, and that stream waits for it.  The same
 *     launches, bitwise the same results, fewer launch overheads for small meshes.  Plans
 *     and scratch are prepared before the capture.  Ignored while kernel timing is on;
 *     not to be combined with a capture of the context stream by the caller.
 *   PDG_OPT_DEBUG_TC_STALL (default 0): a test switch of the failure path of the bounded
 *     waits of the corner passes.  Tensor-core form (PDG_PREC_TF32 / PDG_PREC_TF32_DFRES):
 *     its one waiting thread watches an mbarrier that nothing arrives on, with a bound of
 *     about 0.5 ms, so the bounded wait runs out; the pass then records the timeout, waits
 *     (boundedly) for its tensor-core work in flight, frees its tensor memory and returns.
 *     Hyperplane sweep (PDG_OPT_CORNER_SWEEP): every block waits for a count that no block
 *     reaches, with the same bound, records the timeout and returns.  Either way the next
 *     synchronising call reports PDG_ERR_TIMEOUT once.  The context stays usable: with the
 *     switch off, later steps run normally (from the state left by the aborted passes).
 *   PDG_OPT_TC_LAYERS (default 2): box layers the tensor-core corner pass sweeps together
 *     (PDG_PREC_TF32 / PDG_PREC_TF32_DFRES): 2 = layer k + 1 follows layer k one
 *     anti-diagonal behind, and the cells of both anti-diagonals share one product (half the
 *     products and barriers) when they fit its 128 rows; 1 = one layer at a time.  Same
 *     arithmetic per cell either way.
 *   PDG_OPT_RESIDENT (default 0): line passes of periodic axes of the DnQ2n models (no
 *     source stage) run the line-resident kernel: a block copies its lines -- every
 *     population the pass touches, over the whole line -- into shared memory, runs the
 *     pass's operations there and writes the lines back once, so each value crosses DRAM
 *     once each way per pass and the block requests all of its data at once.  The same
 *     operations in the same order as the streaming kernel (the segment closure may round
 *     differently when the launch shape differs).  Passes whose staged lines do not fit
 *     run the streaming kernel.
 *   PDG_OPT_COLLISION_AXIS (default -1): the axis whose line pass carries the collision
 *     (M2: the pair of half steps between two collisions, composed, then the collision,
 *     T(dt/2) T(dt/2) C; M2^kin: T C T as in Section 3.2); -1 = the last axis.  Transports
 *     along different axes commute, so
 *     any axis gives the same scheme (results equal up to rounding); axis 0 has
 *     unit-stride lines, which the line-resident kernel stages most cheaply.  Lattice
 *     models keep the last axis (other values: PDG_ERR_UNSUPPORTED).
 *   PDG_OPT_CORNER_SWEEP (default 1): how the corner pass of D3Q15 / D3Q27 (FP64 and
 *     PDG_PREC_DF32) is organised.  1 = hyperplane sweeps: each corner population sweeps
 *     the whole mesh once, from one truncated upwind start per periodic axis, cell
 *     hyperplane by hyperplane (column + row + layer = s), each hyperplane shared by the
 *     blocks of a cooperative launch that meet at a bounded counter wait after every
 *     hyperplane (a wait that runs out is reported as PDG_ERR_TIMEOUT at the next
 *     synchronising call); 0 = boxes: one block per box of output cells with its own
 *     truncated start, no block waiting on another.  Forced box shapes (pdg_set_launch,
 *     kind 6) and the tensor-core forms at degree 3 use boxes; the tensor-core forms at
 *     degree <= 2 sweep hyperplanes too, one batch of 128 cells per product.  Results
 *     agree to rounding.
 * Errors: PDG_ERR_ARG (unknown option, axis out of range), PDG_ERR_UNSUPPORTED.
 */
enum {
  PDG_OPT_COMPOSE_TT = 1,
  PDG_OPT_GRAPH = 2,
  PDG_OPT_DEBUG_TC_STALL = 3,
  PDG_OPT_RESIDENT = 4,
  PDG_OPT_COLLISION_AXIS = 5,
  PDG_OPT_TC_LAYERS = 6,
  PDG_OPT_CORNER_SWEEP = 7
};
int pdg_set_option(pdg_ctx* ctx, int option, int value);

/* pdg_get_launch -- read the launch shape override of a kind 0..8 (zeros = heuristic). */
int pdg_get_launch(const pdg_ctx* ctx, int kind, int* lpb, int* nseg, int* ngroup);

/*
 * pdg_autotune -- pick the launch shapes of both pass kinds for this mesh and model.
 * Every candidate (lines per block, segments, field groups) is timed with CUDA events
 * over `reps` launches of the steady-state pass of a step of size dt, on a scratch
 * copy of the state (the state is not modified; a temporary of f_len doubles is
 * allocated and freed), and the fastest is stored as the pdg_set_launch override.
 * Results are unchanged up to rounding (the segment split changes the summation
 * order of the periodic closure).  Synchronises the stream.
 * Errors: PDG_ERR_STATE (no state), PDG_ERR_ARG, PDG_ERR_OOM, PDG_ERR_CUDA.
 */
int pdg_autotune(pdg_ctx* ctx, double dt, int reps);

/*
 * Batched execution (many independent meshes of different size, degree and model
 * in one persistent launch per stage).  Stage t runs the t-th pass of the schedule
 * of every instance that has one (the schedule of pdg_step); inside a stage the work
 * items (one thread block's lines of one pass) are ordered by cost, largest first,
 * and claimed by persistent blocks through an atomic counter.  A work item does the
 * arithmetic of the single-mesh kernel with the same launch shape, so an instance
 * gives the same result whatever its batch neighbours are.
 *
 * pdg_batch_create -- group n contexts (each with a model; the batch keeps the
 *   context handles, which must outlive it) on one CUDA stream (NULL = default).
 *   Errors: PDG_ERR_ARG, PDG_ERR_STATE (a context without model), PDG_ERR_OOM, PDG_ERR_CUDA.
 * pdg_batch_step -- advance instance i by nsteps[i] palindromic steps of size dt[i]
 *   (nsteps[i] = 0 leaves it untouched).  use_graph != 0 captures the stage launches
 *   in a CUDA graph, cached and replayed while dt[] and nsteps[] repeat.
 *   Asynchronous; the per-call work tables (a few bytes per pass and per instance)
 *   live in device memory owned by the batch.
 *   Errors: PDG_ERR_STATE (an instance without state), PDG_ERR_ARG, PDG_ERR_OOM, PDG_ERR_CUDA.
 * pdg_batch_elapsed -- device time (ms) of the last pdg_batch_step (CUDA events; waits
 *   for it) and the number of kernel launches it issued.
 * pdg_batch_autotune -- per class of instances (dimension, degree, cells per axis,
 *   model, dt) time the candidate shapes of the batched kernel on a scratch copy of
 *   one representative state and apply the fastest to the whole class.
 * pdg_batch_destroy -- release the batch (not its contexts).
 */
typedef struct pdg_batch pdg_batch;
int pdg_batch_create(pdg_batch** out, int n, pdg_ctx* const* ctxs, void* cuda_stream);
int pdg_batch_step(pdg_batch* batch, const double* dt, const int* nsteps, int use_graph);
int pdg_batch_elapsed(pdg_batch* batch, double* ms, long long* launches);
int pdg_batch_autotune(pdg_batch* batch, const double* dt, int reps);
int pdg_batch_destroy(pdg_batch* batch);
const char* pdg_batch_last_error(const pdg_batch* batch);

/*
 * Serving with continuous batching.  A server owns a FIFO of submitted solves and a
 * set of resident ones.  pdg_server_iterate (1) admits waiting requests, first come
 * first served, while the sum of the resident states stays within the memory budget
 * (each admitted request gets its own context; its state comes from the CUDA
 * stream-ordered pool, so admission and retirement do not synchronise the device),
 * (2) advances every resident solve by min(remaining, chunk_steps) palindromic steps
 * through one pdg_batch_step (all their launches overlap on the device), then (3)
 * retires the finished ones: their moments w are copied to a host result and their
 * device state is freed, which lets the next waiting requests in.  A solve's
 * arithmetic does not depend on the other solves in flight, on when it was admitted
 * or on the chunking (chunk boundaries only split fused transport passes).
 * Times are seconds on the server clock (pdg_server_now, a monotonic clock).
 *
 * pdg_request:  mesh (dim, n_macro, n_sub, order; unit box, periodic), model,
 *   dt and nsteps, w0 = initial macroscopic state in host memory (m * npoints doubles,
 *   copied at submission), t_arrival = arrival time on the server clock.
 * pdg_server_create -- budget in bytes of resident kinetic state, chunk of steps per
 *   iteration (>= 1), use_graph as in pdg_batch_step, CUDA stream (NULL = default).
 * pdg_server_submit -- validate and enqueue a request; *id receives its id (> 0).
 *   Errors: PDG_ERR_ARG (bad request, w0 length, larger than the budget), PDG_ERR_OOM,
 *   PDG_ERR_UNSUPPORTED (lattice models: they run through pdg_step only).
 * pdg_server_iterate -- one admission / batched chunk / retirement round (synchronous).
 *   A request whose admission fails (its state cannot be allocated, e.g. the device holds
 *   less free memory than the budget) fails alone: it leaves the queue, pdg_server_result
 *   returns its status, and the other requests are served.
 * pdg_server_cancel -- drop a waiting or resident request between iterations (its state is
 *   freed); pdg_server_result then returns PDG_ERR_STATE for it.
 *   Errors: PDG_ERR_STATE (no waiting or resident request with this id), PDG_ERR_ARG.
 * pdg_server_pending -- waiting and resident counts.
 * pdg_server_poll -- up to max finished requests not yet polled: ids, arrival,
 *   admission and completion times; *count receives how many were written.
 * pdg_server_result -- copy the final w of a finished request (once; then released).
 *   Errors: PDG_ERR_STATE (unknown, unfinished, cancelled or already fetched id),
 *   PDG_ERR_ARG, or the status of a request whose admission failed (e.g. PDG_ERR_OOM).
 * pdg_server_stats -- iterations, DOF-updates done, requests completed, peak resident bytes.
 * pdg_server_destroy -- free everything, including unfinished requests.
 */
typedef struct pdg_request {
  int dim;
  int n_macro[3];
  int n_sub[3];
  int order;
  pdg_model_desc model;
  double dt;
  int nsteps;
  int reserved;
  const double* w0;
  size_t w0_len;
  double t_arrival;
} pdg_request;
typedef struct pdg_server pdg_server;
int pdg_server_create(pdg_server** out, size_t mem_budget_bytes, int chunk_steps, int use_graph,
                      void* cuda_stream);
double pdg_server_now(const pdg_server* server);
int pdg_server_submit(pdg_server* server, const pdg_request* req, long long* id);
int pdg_server_iterate(pdg_server* server, int* n_resident, int* n_done);
int pdg_server_pending(const pdg_server* server, int* n_waiting, int* n_resident);
int pdg_server_poll(pdg_server* server, long long* ids, double* t_arrival, double* t_admit, double* t_done,
                    int max, int* count);
int pdg_server_result(pdg_server* server, long long id, double* w, size_t len);
int pdg_server_cancel(pdg_server* server, long long id);
int pdg_server_stats(const pdg_server* server, long long* iterations, long long* dof_updates,
                     long long* completed, size_t* peak_bytes);
int pdg_server_destroy(pdg_server* server);
const char* pdg_server_last_error(const pdg_server* server);

/*
 * pdg_plan_line -- the line plan of an axis-aligned velocity, for inspection and tests (host
 * only: needs no context and no GPU).  With the line reduction of eq. (3.7) and the theta
 * step of eq. (3.11), for degree d, Courant number nu = 2 lambda delta / h and weight theta,
 * the update of cell c is
 *     fn_c = E f_c + q (za x_{c-1} + zb u_{c-1}),
 * x and u the new and old values of the last node of the upwind cell, and the last node
 * obeys the recurrence x_c = alpha_c + beta x_{c-1}.
 *   d        1..4
 *   nu       finite (negative for delta < 0)
 *   theta    in [0, 1]
 *   E        NULL or n*n doubles (n = d + 1), row-major: B^{-1}(I - (1-theta) nu K),
 *            B = I + theta nu K, K = Dm + w_0^{-1} e_0 e_0^T
 *   q        NULL or n doubles: the inflow vector
 *   scalars  NULL or 4 doubles: beta, za, zb, and gamma1, the coupling of the composed double
 *            step (its second last-node value gains gamma1 x_{c-1}; gamma1 = (E q)_d za + q_d zb)
 *   windows  NULL or 2 ints: W, the window of the recurrence in its stable direction
 *            (|r|^W <= 2^-60 with r = beta, or 1/beta when |beta| > 1; 1 when beta = 0), and
 *            W2, that of the composed double step (|beta|^W2 <= 2^-60 and
 *            W2 |gamma1| |beta|^(W2-1) <= 2^-60; 0 when |beta| >= 1, where it is not composed)
 * Errors: PDG_ERR_ARG (d, nu or theta out of range, or a singular cell system).
 */
int pdg_plan_line(int d, double nu, double theta, double* E, double* q, double* scalars, int* windows);

/*
 * pdg_plan_sweep -- the truncated-start plan of the wavefront sweeps, for inspection and
 * tests (host only: needs no context and no GPU).  ncomp = 2: the tile sweep of velocities
 * with two nonzero components (D2Q9 diagonals, D3Q19 / D3Q27 edges, Section 4.1's
 * wavefronts cut into independent tiles); ncomp = 3: the box sweep of the corner velocities
 * of D3Q15 / D3Q27.
 *   d       DG degree: 1..4 (ncomp 2), 1..3 (ncomp 3)
 *   nu      ncomp Courant numbers nu_a = 2 |v_a| delta / h_a (> 0, finite), in the order of
 *           the velocity's nonzero axes
 *   theta   weight of the theta step, in (0, 1]
 *   widths  receives ncomp ints: the cells every tile / box is swept from upwind along each
 *           axis, the smallest widths whose signed lattice-path bound on the error of the
 *           truncated start is <= 2^-57 max |f| per upwind edge
 *   binv    NULL, or (d+1)^(2 ncomp) doubles: the inverse of the cell system
 *           B = I + theta sum_a nu_a K_a of eq. (3.7) split by axis (K = Dm + w_0^{-1} e_0 e_0^T
 *           acting along axis a), row-major, nodes numbered with x fastest
 * Errors: PDG_ERR_ARG (ncomp, d, nu or theta out of range, NULL nu / widths),
 * PDG_ERR_UNSUPPORTED (no width within the limit: 128 cells for tiles, 64 for boxes).
 */
int pdg_plan_sweep(int ncomp, int d, const double* nu, double theta, int* widths, double* binv);

/*
 * pdg_measure_fma_peak -- measured multiply-add throughput of the current device, for
 * the roofline of the arithmetic-bound kernels (no counterpart in the paper: a
 * measurement utility).  A kernel of 4 blocks of 256 threads per SM runs 8 independent
 * FMA chains per thread, in FP64 (fp64 != 0, the FP64 pipe that bounds the FP64 passes)
 * or FP32 (the pipe of the double-float passes); the best of three timed launches after
 * one warm-up, CUDA events on `stream` (NULL = default stream).
 *   tflops  receives 2 x FMAs / seconds / 1e12;  ms (may be NULL) the kernel time.
 * Allocates and frees a small device buffer (stream-ordered).  Synchronises the stream.
 * Errors: PDG_ERR_ARG (tflops NULL), PDG_ERR_OOM, PDG_ERR_CUDA.
 */
int pdg_measure_fma_peak(int fp64, double* tflops, double* ms, void* stream);

/*
 * pdg_debug_fail_allocs -- host-side fault injection for tests: the next n device
 * allocations of kinetic states (any context, this process) fail as if the device were
 * out of memory, without calling the CUDA allocator; n = 0 disarms.  The failing call
 * returns PDG_ERR_OOM and leaves its context as it was.  Errors: PDG_ERR_ARG (n < 0).
 */
int pdg_debug_fail_allocs(int n);

/* pdg_destroy -- free the context and its device memory (NULL is a no-op). */
int pdg_destroy(pdg_ctx* ctx);

/* pdg_last_error -- text of the last error of ctx (never NULL; "" if none). */
const char* pdg_last_error(const pdg_ctx* ctx);

/* pdg_status_string -- static text of a status code. */
const char* pdg_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* PDG_H */
