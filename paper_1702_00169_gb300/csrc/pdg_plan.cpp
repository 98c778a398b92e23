// Host plan: Gauss-Lobatto quadrature and the per-cell transport coefficients.
//
// Section 3.1: nodal DG on the (d+1) Gauss-Lobatto points of [-1, 1] with the
// Lagrange basis; eq. (3.7) DG_reduit on an affine Cartesian cell of edge h
// reduces, for v = +lambda e_a, to the line system
//     d/dt f_c = -(2 lambda / h) [K f_c - w_0^{-1} e_0 f_{c-1, d}],
//     K = Dm + w_0^{-1} e_0 e_0^T,  Dm[j][i] = l_i'(x_j),
// using the summation-by-parts identity W Dm + Dm^T W = e_d e_d^T - e_0 e_0^T of
// GL quadrature.  The theta step of eq. (3.11) (theta = 1/2) with nu = 2 lambda delta / h:
//     B fn_c - theta nu w_0^{-1} e_0 x_{c-1} = (I - (1-theta) nu K) f_c + (1-theta) nu w_0^{-1} e_0 u_{c-1}
// with B = I + theta nu K, hence fn_c = E f_c + g (x_{c-1} + ((1-theta)/theta) u_{c-1}),
// E = B^{-1}(I - (1-theta) nu K), g = B^{-1} theta nu w_0^{-1} e_0.
//
// Everything is computed in double with FP contraction disabled (build flag), so
// the x86-64 and aarch64 builds produce identical coefficients.
#include <cmath>
#include <utility>
#include <cstring>
#include <vector>

#include "pdg.h"
#include "pdg_internal.h"

// Legendre P_k(x) and its derivative by the three-term recurrence.
static void legendre(int k, double x, double* p, double* dp) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (k == 0) { *p = 1.0; *dp = 0.0; return; }
  for (int j = 2; j <= k; ++j) {
    double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
    double d2 = d0 + (2.0 * j - 1.0) * p1;  // P_j' = P_{j-2}' + (2j-1) P_{j-1}
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *p = p1; *dp = d1;
}

// GL nodes: x_0 = -1, x_d = +1 and the roots of P_d' (Newton on P_d' with
// P_d'' = (2x P_d' - d(d+1) P_d) / (1 - x^2), started from Chebyshev-Lobatto points);
// weights w_j = 2 / (d (d+1) P_d(x_j)^2).
int pdg_plan_gl(int d, double* x, double* w) {
  if (d < 1 || d > 16) return -1;
  const double pi = 3.14159265358979323846;
  for (int j = 0; j <= d; ++j) {
    if (j == 0) { x[j] = -1.0; continue; }
    if (j == d) { x[j] = 1.0; continue; }
    double t = -std::cos(pi * j / d);
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(d, t, &p, &dp);
      double ddp = (2.0 * t * dp - d * (d + 1.0) * p) / (1.0 - t * t);
      double step = dp / ddp;
      t -= step;
      if (std::fabs(step) < 1e-17) break;
    }
    x[j] = t;
  }
  // exact symmetry of the node set
  for (int j = 0; j <= d / 2; ++j) {
    double s = 0.5 * (x[d - j] - x[j]);
    x[j] = -s; x[d - j] = s;
  }
  if (d % 2 == 0) x[d / 2] = 0.0;
  for (int j = 0; j <= d; ++j) {
    double p, dp;
    legendre(d, x[j], &p, &dp);
    w[j] = 2.0 / (d * (d + 1.0) * p * p);
  }
  return 0;
}

// Dm[j*n + i] = l_i'(x_j) by the barycentric formula (Berrut & Trefethen, SIAM Review 2004):
// with b_i = 1 / prod_{k != i} (x_i - x_k): l_i'(x_j) = (b_i / b_j) / (x_j - x_i), j != i,
// and the diagonal from sum_i l_i' = 0.
void pdg_plan_dmat(int n, const double* x, double* Dm) {
  double b[16];
  for (int i = 0; i < n; ++i) {
    double p = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != i) p *= (x[i] - x[k]);
    b[i] = 1.0 / p;
  }
  for (int j = 0; j < n; ++j) {
    double diag = 0.0;
    for (int i = 0; i < n; ++i) {
      if (i == j) continue;
      double v = (b[i] / b[j]) / (x[j] - x[i]);
      Dm[j * n + i] = v;
      diag -= v;
    }
    Dm[j * n + j] = diag;
  }
}

// Solve A X = R (n x n, k right-hand sides, row-major) by Gaussian elimination
// with partial pivoting; A and R are overwritten.  Returns 0 on success.
static int solve(int n, int k, double* A, double* R) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) return -1;
    if (piv != c) {
      for (int j = 0; j < n; ++j) { double t = A[c * n + j]; A[c * n + j] = A[piv * n + j]; A[piv * n + j] = t; }
      for (int j = 0; j < k; ++j) { double t = R[c * k + j]; R[c * k + j] = R[piv * k + j]; R[piv * k + j] = t; }
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double fct = A[r * n + c] / A[c * n + c];
      if (fct == 0.0) continue;
      for (int j = c; j < n; ++j) A[r * n + j] -= fct * A[c * n + j];
      for (int j = 0; j < k; ++j) R[r * k + j] -= fct * R[c * k + j];
    }
  }
  for (int r = 0; r < n; ++r) {
    double inv = A[r * n + r];
    for (int j = 0; j < k; ++j) R[r * k + j] /= inv;
  }
  return 0;
}

int pdg_plan_coef(int d, double nu, double theta, PdgCoef* c) {
  const int n = d + 1;
  if (n > PDG_MAXN || !(theta >= 0.0 && theta <= 1.0) || !std::isfinite(nu)) return -1;
  double x[PDG_MAXN], w[PDG_MAXN], Dm[PDG_MAXN * PDG_MAXN];
  if (pdg_plan_gl(d, x, w)) return -1;
  pdg_plan_dmat(n, x, Dm);
  double K[PDG_MAXN * PDG_MAXN];
  std::memcpy(K, Dm, sizeof(double) * n * n);
  K[0] += 1.0 / w[0];
  // A = B = I + theta nu K ; right-hand sides: [I - (1-theta) nu K | theta nu/w0 e0 | (1-theta) nu/w0 e0]
  double A[PDG_MAXN * PDG_MAXN];
  const int k = n + 2;
  double R[PDG_MAXN * (PDG_MAXN + 2)];
  for (int r = 0; r < n; ++r) {
    for (int j = 0; j < n; ++j) {
      double id = (r == j) ? 1.0 : 0.0;
      A[r * n + j] = id + theta * nu * K[r * n + j];
      R[r * k + j] = id - (1.0 - theta) * nu * K[r * n + j];
    }
    R[r * k + n] = (r == 0) ? theta * nu / w[0] : 0.0;
    R[r * k + n + 1] = (r == 0) ? (1.0 - theta) * nu / w[0] : 0.0;
  }
  if (solve(n, k, A, R)) return -1;
  std::memset(c, 0, sizeof(*c));
  for (int r = 0; r < n; ++r)
    for (int j = 0; j < n; ++j) c->E[r * n + j] = R[r * k + j];
  if (theta > 0.0) {
    for (int r = 0; r < n; ++r) c->q[r] = R[r * k + n];  // g
    c->za = 1.0;
    c->zb = (1.0 - theta) / theta;
  } else {
    for (int r = 0; r < n; ++r) c->q[r] = R[r * k + n + 1];  // p (explicit step)
    c->za = 0.0;
    c->zb = 1.0;
  }
  c->beta = c->q[n - 1] * c->za;
  return 0;
}

int pdg_plan_window(double beta) {
  double a = std::fabs(beta);
  if (a == 0.0) return 1;
  if (a >= 1.0) return 1 << 30;
  double K = std::ceil(-60.0 * std::log(2.0) / std::log(a));
  if (K < 1.0) K = 1.0;
  if (K > (double)(1 << 30)) return 1 << 30;
  return (int)K;
}

int pdg_plan_compose(int n, PdgCoef* c) {
  for (int r = 0; r < n; ++r) {
    for (int j = 0; j < n; ++j) {
      double acc = 0.0;
      for (int k = 0; k < n; ++k) acc += c->E[r * n + k] * c->E[k * n + j];
      c->E2[r * n + j] = acc;
    }
    double acc = 0.0;
    for (int k = 0; k < n; ++k) acc += c->E[r * n + k] * c->q[k];
    c->Eq[r] = acc;
  }
  c->gamma1 = c->Eq[n - 1] * c->za + c->q[n - 1] * c->zb;
  const double b = std::fabs(c->beta), g = std::fabs(c->gamma1);
  if (b >= 1.0) return 0;
  const double tol = std::ldexp(1.0, -60);
  double bk = 1.0;  // |beta|^(K-1)
  for (int K = 1; K < (1 << 20); ++K) {
    const double bK = bk * b;
    if (bK <= tol && (double)K * g * bk <= tol) return K;
    if (b == 0.0 && K >= 2) return K;
    bk = bK;
  }
  return 0;
}

void pdg_coef_split(PdgCoef* c) {
  for (int i = 0; i < PDG_MAXN * PDG_MAXN; ++i) pdg_split(c->E[i], c->E_f[i]);
  for (int i = 0; i < PDG_MAXN; ++i) pdg_split(c->q[i], c->q_f[i]);
  pdg_split(c->za, c->za_f[0]);
  pdg_split(c->zb, c->zb_f[0]);
  pdg_split(c->beta, c->beta_f[0]);
  pdg_split(c->gamma, c->gamma_f[0]);
  pdg_split(c->betaL0, c->betaL0_f[0]);
  pdg_split(c->betaL1, c->betaL1_f[0]);
  pdg_split(c->inv_ring, c->inv_ring_f[0]);
  for (int i = 0; i < PDG_MAXN * PDG_MAXN; ++i) pdg_split(c->E2[i], c->E2_f[i]);
  for (int i = 0; i < PDG_MAXN; ++i) pdg_split(c->Eq[i], c->Eq_f[i]);
  pdg_split(c->gamma1, c->gamma1_f[0]);
}

void pdg_model_constants(PdgModel* m) {
  const double om = m->omega;
  for (int i = 0; i < PDG_K_N; ++i) m->k[i] = 0.0;
  m->k[PDG_K_OM1] = 1.0 - om;
  m->k[PDG_K_C0] = m->kind == 1 ? 0.25 * om : om / (2.0 * m->dim);
  m->k[PDG_K_C1] = om / (2.0 * m->lambda);
  m->k[PDG_K_HALFG] = 0.5 * m->gravity;
  m->k[PDG_K_GM1] = m->gamma - 1.0;
  m->k[PDG_K_HALF] = 0.5;
  if (m->kind >= 3 && m->kind <= 6) {  // lattice weights: rest, axis, edge, corner
    // D2Q9 (Section 5.1), D3Q19, D3Q15, D3Q27
    static const double W[4][4] = {{4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0, 0.0},
                                   {1.0 / 3.0, 1.0 / 18.0, 1.0 / 36.0, 0.0},
                                   {2.0 / 9.0, 1.0 / 9.0, 0.0, 1.0 / 72.0},
                                   {8.0 / 27.0, 2.0 / 27.0, 1.0 / 54.0, 1.0 / 216.0}};
    const double* w = W[m->kind - 3];
    m->k[PDG_K_Q9W0] = om * w[0];
    m->k[PDG_K_Q9W1] = om * w[1];
    m->k[PDG_K_Q9W2] = om * w[2];
    m->k[PDG_K_Q9W3] = om * w[3];
    m->k[PDG_K_SIXTH] = 1.0 / 6.0;
    m->k[PDG_K_ILAM] = 1.0 / m->lambda;
    m->k[PDG_K_LAM] = m->lambda;
  } else {
    for (int i = 0; i < 6; ++i) m->k[PDG_K_CADV + i] = om * m->cadv[i];
  }
  for (int i = 0; i < PDG_K_N; ++i) pdg_split(m->k[i], m->k_f[i]);
}

// ---------------------------------------------------------------------------
// Diagonal velocities (D2Q9).  On a Cartesian cell eq. (3.7) splits by axis, so for
// v = lambda (s_x, s_y), in the traversal orientation (s = -1 mirrors that axis),
//   B fn_c = (I - (1-theta) K2) f_c + (nu_x/w_0) S_x Lt + (nu_y/w_0) S_y Bt,
//   K2 = nu_x I(x)K + nu_y K(x)I,  B = I + theta K2,
// and B^-1 (I - (1-theta) K2) = B^-1 / theta - ((1-theta)/theta) I, which gives the form
// of PdgDiagCoef (one dense NN x NN product per cell).
//
// Truncation width.  The new face values s_c = (R_c, T_c) (R: nodes (i, n-1), T: nodes
// (n-1, i)) obey s_c = a_c + A s_{c-x} + B s_{c-y}, A and B the theta-weighted injection
// columns of B^-1 restricted to the face rows.  A tile swept from W columns upwind starts
// with the old face values instead of the new ones (error <= 2 max|f| per entry).  An
// error entering at row k of the upwind edge reaches the cell of column j, row k + r,
// through the sum over lattice paths G(j, r) = A G(j-1, r) + B G(j, r-1) of products of A
// and B (signs kept), so its effect on any cell of column j is bounded by
// 2 max|f| g sum_r ||G(j, r)||_inf (g: largest gain of a cell value per unit change of the
// inflow faces).  W is the smallest width for which that bound is <= 2^-57 max|f|, for
// each of the two edges (rows: A and B exchanged).  Rows are summed up to 256, far past
// the decay of the terms.
static int diag_width(int n, const double* A, const double* B, int edge, double g) {
  const int m = 2 * n, mm = m * m, R = 256;
  std::vector<double> bufA((size_t)R * mm), bufB((size_t)R * mm);
  double* prev = bufA.data();
  double* cur = bufB.data();
  const double* X = edge == 0 ? A : B;   // step across the edge
  const double* Y = edge == 0 ? B : A;   // step along the edge
  for (int i = 0; i < R * mm; ++i) prev[i] = 0.0;
  for (int s = 0; s < n; ++s) {          // unit error on the faces crossing the edge
    const int f = edge == 0 ? s : n + s;
    prev[f * m + f] = 1.0;
  }
  const double tol = std::ldexp(1.0, -57);
  for (int W = 1; W <= 128; ++W) {
    double total = 0.0;
    for (int r = 0; r < R; ++r) {
      double* G = cur + (size_t)r * mm;
      const double* P = prev + (size_t)r * mm;
      const double* L = r > 0 ? cur + (size_t)(r - 1) * mm : nullptr;
      double nrm = 0.0;
      for (int i = 0; i < m; ++i) {
        double rs = 0.0;
        for (int j = 0; j < m; ++j) {
          double acc = 0.0;
          for (int k = 0; k < m; ++k) {
            acc += X[i * m + k] * P[k * m + j];
            if (L) acc += Y[i * m + k] * L[k * m + j];
          }
          G[i * m + j] = acc;
          rs += std::fabs(acc);
        }
        if (rs > nrm) nrm = rs;
      }
      total += nrm;
    }
    if (!(total < 1e300)) return -1;
    if (2.0 * g * total <= tol) return W;
    double* t = prev;
    prev = cur;
    cur = t;
  }
  return -1;
}

int pdg_plan_diag(int d, double nux, double nuy, double theta, PdgDiagCoef* c) {
  const int n = d + 1, NN = n * n;
  if (n > PDG_MAXN || !(theta > 0.0 && theta <= 1.0) || !(nux > 0.0) || !(nuy > 0.0) ||
      !std::isfinite(nux) || !std::isfinite(nuy))
    return -1;
  double x[PDG_MAXN], w[PDG_MAXN], K[PDG_MAXN * PDG_MAXN];
  if (pdg_plan_gl(d, x, w)) return -1;
  pdg_plan_dmat(n, x, K);
  K[0] += 1.0 / w[0];
  std::vector<double> Av((size_t)PDG_MAXNN * PDG_MAXNN), Rv((size_t)PDG_MAXNN * PDG_MAXNN);
  double* A = Av.data();
  double* R = Rv.data();
  for (int p = 0; p < NN; ++p) {
    const int iy = p / n, ix = p % n;
    for (int q = 0; q < NN; ++q) {
      const int jy = q / n, jx = q % n;
      double k2 = 0.0;
      if (iy == jy) k2 += nux * K[ix * n + jx];
      if (ix == jx) k2 += nuy * K[iy * n + jy];
      A[p * NN + q] = (p == q ? 1.0 : 0.0) + theta * k2;
      R[p * NN + q] = (p == q ? 1.0 : 0.0);
    }
  }
  if (solve(NN, NN, A, R)) return -1;
  std::memset(c, 0, sizeof(*c));
  for (int i = 0; i < NN * NN; ++i) c->Binv[i] = R[i];
  c->theta = theta;
  c->omtheta = 1.0 - theta;
  c->rtheta = 1.0 / theta;
  c->c1 = (1.0 - theta) / theta;
  c->kx = nux / w[0];
  c->ky = nuy / w[0];
  // face transfer matrices (signed), state index s < n: R_s, s >= n: T_{s-n}
  const int m = 2 * n;
  auto fnode = [&](int s) { return s < n ? s * n + (n - 1) : (n - 1) * n + (s - n); };
  double Ab[4 * PDG_MAXN * PDG_MAXN], Bb[4 * PDG_MAXN * PDG_MAXN];
  for (int s = 0; s < m; ++s)
    for (int t = 0; t < m; ++t) {
      Ab[s * m + t] = t < n ? theta * c->kx * c->Binv[fnode(s) * NN + t * n] : 0.0;
      Bb[s * m + t] = t >= n ? theta * c->ky * c->Binv[fnode(s) * NN + (t - n)] : 0.0;
    }
  double g = 0.0;   // largest cell value change per unit change of the inflow faces
  for (int p = 0; p < NN; ++p) {
    double acc = 0.0;
    for (int q = 0; q < n; ++q)
      acc += std::fabs(theta * c->kx * c->Binv[p * NN + q * n]) + std::fabs(theta * c->ky * c->Binv[p * NN + q]);
    if (acc > g) g = acc;
  }
  c->wx = diag_width(n, Ab, Bb, 0, g);
  c->wy = diag_width(n, Ab, Bb, 1, g);
  if (c->wx < 0 || c->wy < 0) return -1;
  for (int i = 0; i < NN * NN; ++i) pdg_split(c->Binv[i], c->Binv_f[i]);
  pdg_split(c->rtheta, c->rtheta_f[0]);
  pdg_split(c->c1, c->c1_f[0]);
  pdg_split(c->theta, c->theta_f[0]);
  pdg_split(c->omtheta, c->omtheta_f[0]);
  pdg_split(c->kx, c->kx_f[0]);
  pdg_split(c->ky, c->ky_f[0]);
  return 0;
}

// ---------------------------------------------------------------------------
// Corner velocities (D3Q15 / D3Q27).  eq. (3.7) splits by axis on a Cartesian cell (as for
// the diagonal velocities above), so for v = lambda (s_x, s_y, s_z), in the traversal
// orientation,
//   B fn_c = (I - (1-theta) K3) f_c + k_x S_x Lt + k_y S_y Bt + k_z S_z Zt,
//   K3 = nu_x I(x)I(x)K + nu_y I(x)K(x)I + nu_z K(x)I(x)I,  B = I + theta K3,
// on the node vector p = (iz n + iy) n + ix, and B^-1 (I - (1-theta) K3) = B^-1/theta - c1 I.
//
// Start widths.  The theta-weighted values on the three downwind faces of a cell,
// s_c = (R_c, T_c, U_c) (R: nodes (iz, iy, n-1), T: (iz, n-1, ix), U: (n-1, iy, ix)), obey
// s_c = a_c + X_x R_{c-x} + X_y T_{c-y} + X_z U_{c-z}, X_a = theta k_a (rows of B^-1 at the
// face nodes, columns at the nodes the face a enters).  A region swept from W cells
// upwind along x starts from the old face values on its x edge (error <= 2 max|f| per
// entry); an error entering there reaches the cell W columns downwind, r rows and k
// layers along the edge, through the signed lattice-path sum
//   G(j, r, k) = X_x G(j-1, r, k) + X_y G(j, r-1, k) + X_z G(j, r, k-1),
// so the effect on any cell of that column is at most 2 max|f| g sum_{r,k} ||G(W, r, k)||_inf
// (g: largest change of a cell value per unit change of its inflow faces).  W is the
// smallest width for which this is <= 2^-57 max|f|, for each of the three edges (the y and
// z edges exchange the roles of the directions).  The sums run over r, k < 48, far past
// the decay of the terms; the plan is refused when the last row or layer of the sum still
// carries more than 2^-67 of the total.
static int corner_width(int n, const std::vector<double>& X, int edge, double g) {
  const int nn = n * n, m = 3 * nn, R = 48, RR = R * R;
  const size_t msz = (size_t)m * nn;
  std::vector<double> bufA((size_t)RR * msz, 0.0), bufB((size_t)RR * msz, 0.0);
  double* prev = bufA.data();
  double* cur = bufB.data();
  const int dir[3] = {edge, (edge + 1) % 3, (edge + 2) % 3};   // across, along 1, along 2
  for (int c = 0; c < nn; ++c) prev[(size_t)(edge * nn + c) * nn + c] = 1.0;
  const double tol = std::ldexp(1.0, -57);
  // acc += X_a (block a of the face state of G)
  auto apply = [&](int a, const double* G, double* acc) {
    const double* Xa = X.data() + (size_t)a * m * nn;
    for (int s = 0; s < m; ++s) {
      double* out = acc + (size_t)s * nn;
      for (int t = 0; t < nn; ++t) {
        const double x = Xa[s * nn + t];
        if (x == 0.0) continue;
        const double* row = G + (size_t)(a * nn + t) * nn;
        for (int c = 0; c < nn; ++c) out[c] += x * row[c];
      }
    }
  };
  for (int W = 1; W <= 64; ++W) {
    double total = 0.0, rim = 0.0;
    for (int r = 0; r < R; ++r)
      for (int k = 0; k < R; ++k) {
        double* G = cur + (size_t)(r * R + k) * msz;
        for (size_t i = 0; i < msz; ++i) G[i] = 0.0;
        apply(dir[0], prev + (size_t)(r * R + k) * msz, G);
        if (r > 0) apply(dir[1], cur + (size_t)((r - 1) * R + k) * msz, G);
        if (k > 0) apply(dir[2], cur + (size_t)(r * R + k - 1) * msz, G);
        double nrm = 0.0;
        for (int s = 0; s < m; ++s) {
          double rs = 0.0;
          for (int c = 0; c < nn; ++c) rs += std::fabs(G[(size_t)s * nn + c]);
          if (rs > nrm) nrm = rs;
        }
        total += nrm;
        if (r == R - 1 || k == R - 1) rim += nrm;
      }
    if (!(total < 1e300)) return -1;
    if (2.0 * g * total <= tol) return 2.0 * g * rim <= std::ldexp(tol, -10) ? W : -1;
    std::swap(prev, cur);
  }
  return -1;
}

int pdg_plan_corner(int d, double nux, double nuy, double nuz, double theta, PdgCornerCoef* c, double* binv,
                    float* binv_f) {
  const int n = d + 1, nn = n * n, NN = nn * n;
  if (n < 2 || n > PDG_MAXN_CORNER || !(theta > 0.0 && theta <= 1.0) || !(nux > 0.0) || !(nuy > 0.0) ||
      !(nuz > 0.0) || !std::isfinite(nux) || !std::isfinite(nuy) || !std::isfinite(nuz))
    return -1;
  double x[PDG_MAXN], w[PDG_MAXN], K[PDG_MAXN * PDG_MAXN];
  if (pdg_plan_gl(d, x, w)) return -1;
  pdg_plan_dmat(n, x, K);
  K[0] += 1.0 / w[0];
  std::vector<double> A((size_t)NN * NN), R((size_t)NN * NN);
  for (int p = 0; p < NN; ++p) {
    const int iz = p / nn, iy = (p / n) % n, ix = p % n;
    for (int q = 0; q < NN; ++q) {
      const int jz = q / nn, jy = (q / n) % n, jx = q % n;
      double k3 = 0.0;
      if (iz == jz && iy == jy) k3 += nux * K[ix * n + jx];
      if (iz == jz && ix == jx) k3 += nuy * K[iy * n + jy];
      if (iy == jy && ix == jx) k3 += nuz * K[iz * n + jz];
      A[(size_t)p * NN + q] = (p == q ? 1.0 : 0.0) + theta * k3;
      R[(size_t)p * NN + q] = (p == q ? 1.0 : 0.0);
    }
  }
  if (solve(NN, NN, A.data(), R.data())) return -1;
  std::memset(c, 0, sizeof(*c));
  for (int i = 0; i < NN * NN; ++i) {
    binv[i] = R[i];
    pdg_split(R[i], binv_f + 2 * i);
  }
  c->theta = theta;
  c->omtheta = 1.0 - theta;
  c->rtheta = 1.0 / theta;
  c->c1 = (1.0 - theta) / theta;
  c->kx = nux / w[0];
  c->ky = nuy / w[0];
  c->kz = nuz / w[0];
  const double ka[3] = {c->kx, c->ky, c->kz};
  auto idx = [&](int iz, int iy, int ix) { return (iz * n + iy) * n + ix; };
  auto fnode = [&](int s) {
    const int a = s / nn, u = (s % nn) / n, v = s % n;
    return a == 0 ? idx(u, v, n - 1) : (a == 1 ? idx(u, n - 1, v) : idx(n - 1, u, v));
  };
  auto inj = [&](int a, int t) {
    const int u = t / n, v = t % n;
    return a == 0 ? idx(u, v, 0) : (a == 1 ? idx(u, 0, v) : idx(0, u, v));
  };
  const int m = 3 * nn;
  std::vector<double> X((size_t)3 * m * nn);
  for (int a = 0; a < 3; ++a)
    for (int s = 0; s < m; ++s)
      for (int t = 0; t < nn; ++t)
        X[((size_t)a * m + s) * nn + t] = theta * ka[a] * R[(size_t)fnode(s) * NN + inj(a, t)];
  double g = 0.0;
  for (int p = 0; p < NN; ++p) {
    double acc = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int t = 0; t < nn; ++t) acc += std::fabs(theta * ka[a] * R[(size_t)p * NN + inj(a, t)]);
    if (acc > g) g = acc;
  }
  c->wx = corner_width(n, X, 0, g);
  // equal Courant numbers: the three edges are images of each other under a permutation
  // of the axes, which maps the node and face orderings onto each other
  const bool cubic = nux == nuy && nuy == nuz;
  c->wy = cubic ? c->wx : corner_width(n, X, 1, g);
  c->wz = cubic ? c->wx : corner_width(n, X, 2, g);
  if (c->wx < 0 || c->wy < 0 || c->wz < 0) return -1;
  pdg_split(c->rtheta, c->rtheta_f[0]);
  pdg_split(c->c1, c->c1_f[0]);
  pdg_split(c->theta, c->theta_f[0]);
  pdg_split(c->omtheta, c->omtheta_f[0]);
  pdg_split(c->kx, c->kx_f[0]);
  pdg_split(c->ky, c->ky_f[0]);
  pdg_split(c->kz, c->kz_f[0]);
  const double nua[3] = {nux, nuy, nuz};
  for (int a = 0; a < 3; ++a)
    for (int i = 0; i < n * n; ++i) {
      c->kt[a][i] = theta * nua[a] * K[i];
      pdg_split(c->kt[a][i], c->kt_f[a][i]);
    }
  return 0;
}

// Inspection entry point of the line plan (declared in pdg.h).
int pdg_plan_line(int d, double nu, double theta, double* E, double* q, double* scalars, int* windows) try {
  if (d < 1 || d + 1 > PDG_MAXN || !(theta >= 0.0 && theta <= 1.0) || !std::isfinite(nu)) return PDG_ERR_ARG;
  PdgCoef c;
  if (pdg_plan_coef(d, nu, theta, &c)) return PDG_ERR_ARG;
  const int n = d + 1;
  const int W2 = pdg_plan_compose(n, &c);
  if (E)
    for (int i = 0; i < n * n; ++i) E[i] = c.E[i];
  if (q)
    for (int i = 0; i < n; ++i) q[i] = c.q[i];
  if (scalars) {
    scalars[0] = c.beta;
    scalars[1] = c.za;
    scalars[2] = c.zb;
    scalars[3] = c.gamma1;
  }
  if (windows) {
    windows[0] = pdg_plan_window(std::fabs(c.beta) > 1.0 ? 1.0 / c.beta : c.beta);
    windows[1] = W2;
  }
  return PDG_OK;
} catch (...) {
  return pdgapi::abi_exception(nullptr);
}

// Inspection entry point of the tile and box plans (declared in pdg.h).
int pdg_plan_sweep(int ncomp, int d, const double* nu, double theta, int* widths, double* binv) try {
  if (!nu || !widths || (ncomp != 2 && ncomp != 3)) return PDG_ERR_ARG;
  if (d < 1 || d + 1 > (ncomp == 2 ? PDG_MAXN : PDG_MAXN_CORNER)) return PDG_ERR_ARG;
  if (!(theta > 0.0 && theta <= 1.0)) return PDG_ERR_ARG;
  for (int a = 0; a < ncomp; ++a)
    if (!(nu[a] > 0.0) || !std::isfinite(nu[a])) return PDG_ERR_ARG;
  const int n = d + 1;
  if (ncomp == 2) {
    std::vector<PdgDiagCoef> c(1);
    if (pdg_plan_diag(d, nu[0], nu[1], theta, c.data())) return PDG_ERR_UNSUPPORTED;
    widths[0] = c[0].wx;
    widths[1] = c[0].wy;
    if (binv)
      for (int i = 0; i < n * n * n * n; ++i) binv[i] = c[0].Binv[i];
    return PDG_OK;
  }
  const int NN = n * n * n;
  PdgCornerCoef c;
  std::vector<double> b((size_t)NN * NN);
  std::vector<float> bf((size_t)NN * NN * 2);
  if (pdg_plan_corner(d, nu[0], nu[1], nu[2], theta, &c, b.data(), bf.data())) return PDG_ERR_UNSUPPORTED;
  widths[0] = c.wx;
  widths[1] = c.wy;
  widths[2] = c.wz;
  if (binv)
    for (int i = 0; i < NN * NN; ++i) binv[i] = b[i];
  return PDG_OK;
} catch (...) {
  return pdgapi::abi_exception(nullptr);
}
