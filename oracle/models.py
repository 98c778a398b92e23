"""Kinetic models: velocity sets, moments, fluxes, equilibria (oracle; test infrastructure only).

Section 2, eq. (2.1) kin_bgk: n_v transport equations at constant velocities
v_i coupled by the BGK relaxation towards f^eq; eq. (2.2) micro_to_macro:
w = P f; the macroscopic flux is q^k(w) = P V^k f^eq (Section 2).

Velocity sets used here (vectorial DnQ2n): for each conserved variable k the
2D velocities +lambda e_1, -lambda e_1, ..., +lambda e_D, -lambda e_D, in that
order; P sums the 2D populations of each variable: w_k = sum_i f_{k,i}.

Equilibrium (reading; the paper cites the kinetic-representation literature
but prints no DnQ2n formula): f^eq_{k,i} = w_k/(2D) + (v_i . q_k(w))/(2 lambda^2).
It satisfies P f^eq = w and P V^a f^eq = q^a(w) (the two requirements of
Section 2), and for q = a w it is the advection equilibrium
w/4 + (a . v_i) w/(2 lambda^2) of the D2Q4 advection workload.
"""
import numpy as np

ADVECTION, SHALLOW_WATER, EULER = 0, 1, 2


class Model:
    """kind in {ADVECTION, SHALLOW_WATER, EULER}; dim D; lam = lattice speed lambda."""

    def __init__(self, kind, dim, lam, a=None, gravity=9.81, gamma=1.4):
        self.kind = kind
        self.dim = int(dim)
        self.lam = float(lam)
        self.a = np.asarray(a if a is not None else np.zeros(dim), dtype=np.float64)
        self.gravity = float(gravity)
        self.gamma = float(gamma)
        if kind == ADVECTION:
            self.m = 1
        elif kind == SHALLOW_WATER:
            assert self.dim == 2
            self.m = 3
        elif kind == EULER:
            self.m = self.dim + 2
        else:
            raise ValueError(kind)
        self.nv = 2 * self.dim

    def velocities(self):
        """(2D, D) array: row i is v_i, order +e_1, -e_1, +e_2, -e_2, ..."""
        V = np.zeros((self.nv, self.dim))
        for a in range(self.dim):
            V[2 * a, a] = self.lam
            V[2 * a + 1, a] = -self.lam
        return V

    def moments(self, f):
        """eq. (2.2): w_k = sum_i f_{k,i}; f has shape (m, 2D, *grid)."""
        return np.sum(f, axis=1)

    def flux(self, w):
        """q^a_k(w) as an array (D, m, *grid): physical flux of each variable along axis a."""
        D = self.dim
        if self.kind == ADVECTION:
            return np.stack([self.a[a] * w for a in range(D)])
        if self.kind == SHALLOW_WATER:
            h, hu, hv = w[0], w[1], w[2]
            u, v = hu / h, hv / h
            p = 0.5 * self.gravity * h * h
            qx = np.stack([hu, hu * u + p, hv * u])
            qy = np.stack([hv, hu * v, hv * v + p])
            return np.stack([qx, qy])
        # Euler: w = (rho, rho u_1..rho u_D, E), p = (gamma-1)(E - |rho u|^2/(2 rho))
        rho = w[0]
        mom = w[1:1 + D]
        E = w[1 + D]
        u = mom / rho
        p = (self.gamma - 1.0) * (E - 0.5 * np.sum(mom * u, axis=0))
        out = []
        for a in range(D):
            comps = [mom[a]]
            for b in range(D):
                comps.append(mom[b] * u[a] + (p if a == b else 0.0))
            comps.append((E + p) * u[a])
            out.append(np.stack(comps))
        return np.stack(out)

    def feq(self, w):
        """f^eq_{k,i} = w_k/(2D) + (v_i . q_k)/(2 lambda^2); returns (m, 2D, *grid)."""
        q = self.flux(w)                                  # (D, m, *grid)
        V = self.velocities()
        out = np.empty((self.m, self.nv) + w.shape[1:])
        for i in range(self.nv):
            vq = np.tensordot(V[i], q, axes=(0, 0))       # (m, *grid)
            out[:, i] = w / (2.0 * self.dim) + vq / (2.0 * self.lam ** 2)
        return out
