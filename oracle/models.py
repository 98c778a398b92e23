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

D2Q9 (Section 5.1, Euler with gravity): ONE set of nine populations for the three
isothermal Euler variables w = (rho, rho u_x, rho u_y); velocities lambda (0,0),
(1,0), (0,1), (-1,0), (0,-1), (1,1), (-1,1), (-1,-1), (1,-1) in that order;
P = [1; v_x; v_y] (rho = sum f_i, rho u = sum f_i v_i); equilibrium
f_i = W_i rho (1 + u.v_i/c^2 + (u.v_i)^2/(2 c^4) - u.u/(2 c^2)), c = lambda/sqrt(3),
W = 4/9 (rest), 1/9 (axis), 1/36 (diagonal).  Its second moment is the isothermal
flux Pi = rho c^2 I + rho u u^T (the paper prints the yy entry without its rho; the
moment identity fixes it).  Arrays keep the layout (groups, populations, *grid) with
one group of nine populations.
"""
import numpy as np

ADVECTION, SHALLOW_WATER, EULER, ISOTHERMAL_D2Q9 = 0, 1, 2, 3

D2Q9_XI = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]],
                   dtype=np.float64)
D2Q9_W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


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
        elif kind == ISOTHERMAL_D2Q9:
            assert self.dim == 2
            self.m = 3
        else:
            raise ValueError(kind)
        self.nv = 9 if kind == ISOTHERMAL_D2Q9 else 2 * self.dim
        self.groups = 1 if kind == ISOTHERMAL_D2Q9 else self.m

    @property
    def sound_speed(self):
        """D2Q9: c = lambda / sqrt(3)."""
        return self.lam / np.sqrt(3.0)

    def velocities(self):
        """(n_v, D) array: row i is v_i; DnQ2n order +e_1, -e_1, +e_2, -e_2, ...;
        D2Q9 in the order of the module doc."""
        if self.kind == ISOTHERMAL_D2Q9:
            return self.lam * D2Q9_XI
        V = np.zeros((self.nv, self.dim))
        for a in range(self.dim):
            V[2 * a, a] = self.lam
            V[2 * a + 1, a] = -self.lam
        return V

    def moments(self, f):
        """eq. (2.2) w = P f.  DnQ2n: w_k = sum_i f_{k,i}, f of shape (m, 2D, *grid).
        D2Q9: f of shape (1, 9, *grid), w = (sum_i f_i, sum_i f_i v_i)."""
        if self.kind == ISOTHERMAL_D2Q9:
            V = self.velocities()
            g = f[0]
            return np.stack([np.sum(g, axis=0), np.tensordot(V[:, 0], g, axes=(0, 0)),
                             np.tensordot(V[:, 1], g, axes=(0, 0))])
        return np.sum(f, axis=1)

    def flux(self, w):
        """q^a_k(w) as an array (D, m, *grid): physical flux of each variable along axis a."""
        D = self.dim
        if self.kind == ADVECTION:
            return np.stack([self.a[a] * w for a in range(D)])
        if self.kind == ISOTHERMAL_D2Q9:
            rho, mx, my = w[0], w[1], w[2]
            c2 = self.sound_speed ** 2
            qx = np.stack([mx, mx * mx / rho + rho * c2, mx * my / rho])
            qy = np.stack([my, mx * my / rho, my * my / rho + rho * c2])
            return np.stack([qx, qy])
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
        """DnQ2n: f^eq_{k,i} = w_k/(2D) + (v_i . q_k)/(2 lambda^2), shape (m, 2D, *grid).
        D2Q9: the polynomial equilibrium of the module doc, shape (1, 9, *grid)."""
        if self.kind == ISOTHERMAL_D2Q9:
            rho = w[0]
            u = np.stack([w[1] / rho, w[2] / rho])
            c2 = self.sound_speed ** 2
            uu = u[0] * u[0] + u[1] * u[1]
            out = np.empty((1, 9) + w.shape[1:])
            for i, v in enumerate(self.velocities()):
                uv = u[0] * v[0] + u[1] * v[1]
                out[0, i] = D2Q9_W[i] * rho * (1.0 + uv / c2 + uv * uv / (2.0 * c2 * c2) - uu / (2.0 * c2))
            return out
        q = self.flux(w)                                  # (D, m, *grid)
        V = self.velocities()
        out = np.empty((self.m, self.nv) + w.shape[1:])
        for i in range(self.nv):
            vq = np.tensordot(V[i], q, axes=(0, 0))       # (m, *grid)
            out[:, i] = w / (2.0 * self.dim) + vq / (2.0 * self.lam ** 2)
        return out
