"""Source step S_2 of the split scheme (oracle; test infrastructure only).

Section 3.2 builds, for tau > 0 and a source, the five-stage palindrome
  M_2^s(dt) = T_2(dt/2) S_2(dt/2) C_2(dt) S_2(dt/2) T_2(dt/2);
Section 5.1 uses it (and its collapsed form) for the isothermal Euler equations
with gravity on the D2Q9 model, and Section 5.2 a penalisation source.  Every
stage is a weighted implicit (theta) step.

Readings (the paper states these in words only):
  * the source acts on the macroscopic variables, d/dt w = s(w), and "on the
    equilibrium part of the distribution function": the step advances w by the
    theta scheme and replaces the equilibrium part of f, keeping f - f^eq(w):
        w'  solves  w' = w + delta [theta s(w') + (1 - theta) s(w)],
        f' = f + f^eq(w') - f^eq(w);
    P f' = w' follows from P f^eq(w) = w;
  * both sources are linear in w, s(w) = A(x) w + b(x), so the theta step is the
    linear system (I - theta delta A) w' = (I + (1 - theta) delta A) w + delta b,
    solved here as it stands at every point (for gravity alone A is nilpotent
    and one Picard iteration is already exact, as the paper remarks);
  * gravity (Section 5.1): s = (0, rho g) for w = (rho, rho u), g a constant
    vector (g = -g e_y in the paper);
  * penalisation (Section 5.2): the paper prints s = K(x)(w - w_s) and calls its
    effect a stiff relaxation TOWARDS w_s; the relaxation reading
    s = -K(x)(w - w_s) is used, with K(x) = K_s exp(-kappa |x - x_c|^2) evaluated
    at the Gauss-Lobatto points (Euclidean distance in the box coordinates).
"""
import numpy as np


class Source:
    """A linear source s(w) = A(x) w + b(x) for the isothermal D2Q9 variables
    w = (rho, rho u_x, rho u_y): gravity vector g, penalisation (K_s, kappa, x_c, w_s)."""

    def __init__(self, gravity=(0.0, 0.0), K_s=0.0, kappa=0.0, x_c=(0.0, 0.0), w_s=(1.0, 0.0, 0.0), theta=0.5):
        self.g = np.asarray(gravity, dtype=np.float64)
        self.K_s, self.kappa = float(K_s), float(kappa)
        self.x_c = np.asarray(x_c, dtype=np.float64)
        self.w_s = np.asarray(w_s, dtype=np.float64)
        self.theta = float(theta)

    def K(self, mesh):
        """Penalisation frequency at every point (field-shaped)."""
        X = mesh.coords1d(0)[None, :]
        Y = mesh.coords1d(1)[:, None]
        return self.K_s * np.exp(-self.kappa * ((X - self.x_c[0]) ** 2 + (Y - self.x_c[1]) ** 2))

    def operator(self, mesh):
        """A (3, 3, *grid) and b (3, *grid) of s(w) = A w + b."""
        K = self.K(mesh)
        A = np.zeros((3, 3) + K.shape)
        for k in range(3):
            A[k, k] = -K
        A[1, 0] += self.g[0]
        A[2, 0] += self.g[1]
        b = K[None] * self.w_s[:, None, None]
        return A, b


def source_step(f, model, mesh, src, delta):
    """S_theta(delta): theta step of d/dt w = s(w), applied to the equilibrium part of f."""
    w = model.moments(f)
    A, b = src.operator(mesh)
    th = src.theta
    n = w.shape[1:]
    Am = np.moveaxis(A.reshape(3, 3, -1), -1, 0)            # (P, 3, 3)
    wv = w.reshape(3, -1).T                                  # (P, 3)
    bv = b.reshape(3, -1).T
    I = np.eye(3)[None]
    lhs = I - th * delta * Am
    rhs = np.einsum("pij,pj->pi", I + (1.0 - th) * delta * Am, wv) + delta * bv
    wn = np.linalg.solve(lhs, rhs[..., None])[..., 0].T.reshape((3,) + n)
    return f + model.feq(wn) - model.feq(w)
