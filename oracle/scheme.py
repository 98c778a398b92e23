"""Collision integrator and palindromic time steps (oracle; test infrastructure only).

Section 3.2:
  eq. (3.12) collision_cn: C_2(dt) F = ((2 tau - dt) F + 2 dt F^eq(F)) / (2 tau + dt),
      i.e. F <- omega F^eq + (1 - omega) F with omega = 2 dt / (2 tau + dt);
      omega = 2 is tau = 0, where C_2 F = 2 F^eq - F.
  M_2(dt) = T_2(dt/2) C_2(dt) T_2(dt/2)  (source-less three-stage palindrome,
      the method the paper retains for its results).
  Section 5.1, collapsed Strang: the last transport sub-step of a step and the
      first of the next are merged into one T_2(dt), except at the two ends.
  M_2^kin(dt) = T_2(dt/4) C_2(dt/2) T_2(dt/2) C_2(dt/2) T_2(dt/4) (Section 3.2): the
      composition that stays second order when tau -> 0; `omega` is then the weight of
      each C_2(dt/2).
  With a source (oracle.source): M_2^s(dt) = T_2(dt/2) S_2(dt/2) C_2(dt) S_2(dt/2) T_2(dt/2)
      (Section 3.2), also in the collapsed form of Section 5.1.
  M_4^kin(dt) = M_2^kin(g1 dt) M_2^kin(g2 dt) M_2^kin(g1 dt): Section 3.2 states that
      palindromic compositions of M_2^kin reach any even order without giving one; this is
      the symmetric triple jump (H. Yoshida, Phys. Lett. A 150 (1990) 262), whose
      coefficients solve 2 g1 + g2 = 1 and 2 g1^3 + g2^3 = 0:
      g1 = 1 / (2 - 2^(1/3)), g2 = 1 - 2 g1 (negative).  It is fourth order when the
      composed step is time-symmetric (eq. (3.13)), which M_2^kin is at omega = 2
      (C_2 is then an involution); its negative sub-step runs the transport backwards,
      which is stable only for moderate Courant numbers.

The steps are applied in the naive order: every population is transported
along its own velocity, then the collision acts on all populations, then every
population is transported again.
"""
import numpy as np

from .dg import CartesianMesh
from .source import source_step
from .transport import DirectTransport, bloch_transport, bloch_transport_2d, bloch_transport_3d, bloch_transport_planes


def collision(f, model, omega):
    """eq. (3.12): f <- omega f^eq(P f) + (1 - omega) f, pointwise."""
    w = model.moments(f)
    return omega * model.feq(w) + (1.0 - omega) * f


class Transporter:
    """Applies T_theta(delta) to every population (each along its velocity).

    method = "direct": sparse LU of the assembled eq. (3.7) system (tiny meshes);
    method = "bloch":  Fourier closed form (any size): per line for axis-aligned
                       velocities, per 2-D mode for the diagonal D2Q9 velocities and
                       (plane by plane) the D3Q19 edges, per 3-D mode for the corners
                       of D3Q15 / D3Q27; rest velocities are not transported.
    """

    def __init__(self, mesh, model, theta=0.5, method="direct", fb=None):
        """fb: boundary data f^b, array (m, 2D, *grid) whose values at the inflow face
        points of each population are used on non-periodic axes (direct method only)."""
        self.mesh, self.model, self.theta, self.method = mesh, model, theta, method
        self.fb = fb
        self._cache = {}

    def _direct(self, i, delta):
        key = (i, delta)
        if key not in self._cache:
            v = self.model.velocities()[i]
            self._cache[key] = DirectTransport(self.mesh, v, delta, self.theta)
        return self._cache[key]

    def field(self, g, i, delta, fb=None):
        """Transport one population array g (grid-shaped) with velocity v_i over delta."""
        if self.method == "direct":
            return self._direct(i, delta)(g, fb)
        assert all(self.mesh.periodic), "the Bloch solver is periodic only"
        v = self.model.velocities()[i]
        nz = np.flatnonzero(v)
        if nz.size == 0:
            return np.array(g, dtype=np.float64, copy=True)
        if nz.size == 1:
            a = int(nz[0])
            nu = 2.0 * abs(v[a]) * delta / self.mesh.h[a]
            return bloch_transport(g, self.mesh.axis_np(a), 1 if v[a] > 0 else -1, self.mesh.d, nu,
                                   self.theta)
        if self.mesh.dim == 2:
            return bloch_transport_2d(g, v, self.mesh.h, self.mesh.d, delta, self.theta)
        if nz.size == 2:
            return bloch_transport_planes(g, v, self.mesh.h, self.mesh.d, delta, self.theta)
        return bloch_transport_3d(g, v, self.mesh.h, self.mesh.d, delta, self.theta)

    def __call__(self, f, delta):
        out = np.empty_like(f)
        for k in range(f.shape[0]):
            for i in range(f.shape[1]):
                out[k, i] = self.field(f[k, i], i, delta, None if self.fb is None else self.fb[k, i])
        return out


def m2_step(f, transporter, model, dt, omega, source=None):
    """M_2(dt) = T(dt/2) C(dt) T(dt/2), Section 3.2; with a source M_2^s(dt)."""
    f = transporter(f, 0.5 * dt)
    f = source_collision(f, transporter, model, dt, omega, source)
    return transporter(f, 0.5 * dt)


def source_collision(f, transporter, model, dt, omega, source=None):
    """C_2(dt), or S_2(dt/2) C_2(dt) S_2(dt/2) with a source."""
    if source is None:
        return collision(f, model, omega)
    f = source_step(f, model, transporter.mesh, source, 0.5 * dt)
    f = collision(f, model, omega)
    return source_step(f, model, transporter.mesh, source, 0.5 * dt)


def run(f0, transporter, model, dt, nsteps, omega, scheme="M2", source=None):
    """nsteps palindromic steps from f0.  scheme: "M2", "M2_collapsed" (Section 5.1),
    "M2_kin" (Section 3.2) or "M4_kin" (the triple jump of M2_kin); source: an
    oracle.source.Source (M2 and M2_collapsed)."""
    f = np.array(f0, dtype=np.float64, copy=True)
    if nsteps <= 0:
        return f
    if scheme == "M2":
        for _ in range(nsteps):
            f = m2_step(f, transporter, model, dt, omega, source)
        return f
    if scheme == "M2_collapsed":
        f = transporter(f, 0.5 * dt)
        for s in range(nsteps):
            f = source_collision(f, transporter, model, dt, omega, source)
            f = transporter(f, dt if s < nsteps - 1 else 0.5 * dt)
        return f
    if source is not None:
        raise ValueError("sources are defined for M2 and M2_collapsed (Section 3.2, Section 5.1)")
    if scheme == "M2_kin":
        for _ in range(nsteps):
            f = m2kin_step(f, transporter, model, dt, omega)
        return f
    if scheme == "M4_kin":
        g1, g2 = triple_jump()
        for _ in range(nsteps):
            for g in (g1, g2, g1):
                f = m2kin_step(f, transporter, model, g * dt, omega)
        return f
    raise ValueError(scheme)


def m2kin_step(f, transporter, model, dt, omega):
    """M_2^kin(dt) = T_2(dt/4) C_2(dt/2) T_2(dt/2) C_2(dt/2) T_2(dt/4) (Section 3.2)."""
    f = transporter(f, 0.25 * dt)
    f = collision(f, model, omega)
    f = transporter(f, 0.5 * dt)
    f = collision(f, model, omega)
    return transporter(f, 0.25 * dt)


def triple_jump():
    """Coefficients (g1, g2) of the symmetric triple jump M(g1 dt) M(g2 dt) M(g1 dt)."""
    g1 = 1.0 / (2.0 - 2.0 ** (1.0 / 3.0))
    return g1, 1.0 - 2.0 * g1


def initial_state(model, w0):
    """Equilibrium initialisation f^0 = f^eq(w^0) (reading: the paper is silent)."""
    return model.feq(np.asarray(w0, dtype=np.float64))


def weighted_total(mesh, w):
    """sum over points of omega_{L,i} w_k: the discrete integral of each variable."""
    M = mesh.mass_weights()
    return np.array([np.sum(M * w[k]) for k in range(w.shape[0])])


def make_mesh(dim, ncells, d, lengths=None, periodic=None):
    return CartesianMesh(dim, ncells, d, lengths, periodic)
