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

D3Q19 (one of the lattices of the paper's 3-D scaling runs, Section 4.5; the paper
prints no 3-D equilibrium): the same polynomial equilibrium for the 3-D isothermal
Euler variables w = (rho, rho u), c = lambda/sqrt(3), on the velocities 0, the six
lambda (+-e_a) (order +x, -x, +y, -y, +z, -z) and the twelve lambda (+-e_a +- e_b),
four per plane in the order xy, xz, yz, each as (+,+), (-,+), (-,-), (+,-); weights
1/3, 1/18, 1/36.

D3Q15 and D3Q27 (the other two lattices of the Section 4.5 scaling runs; again no
equilibrium is printed): the same polynomial equilibrium and c = lambda/sqrt(3) on
  D3Q15: 0, the six axis velocities, the eight corners lambda (+-1, +-1, +-1);
         weights 2/9, 1/9, 1/72;
  D3Q27: 0, the six axis velocities, the twelve edges of D3Q19, the eight corners;
         weights 8/27, 2/27, 1/54, 1/216
(the standard weights that make the lattice moments isotropic up to fourth order).
Corners are ordered z = +1 first, then z = -1, each as (x, y) = (+,+), (-,+), (-,-), (+,-).
"""
import numpy as np

ADVECTION, SHALLOW_WATER, EULER, ISOTHERMAL_D2Q9, ISOTHERMAL_D3Q19 = 0, 1, 2, 3, 4
ISOTHERMAL_D3Q15, ISOTHERMAL_D3Q27 = 5, 6

D2Q9_XI = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]],
                   dtype=np.float64)
D2Q9_W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


_REST_AXIS = [[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]]


def _edges():
    xi = []
    for a, b in ((0, 1), (0, 2), (1, 2)):
        for sa, sb in ((1, 1), (-1, 1), (-1, -1), (1, -1)):
            v = [0, 0, 0]
            v[a], v[b] = sa, sb
            xi.append(v)
    return xi


def _corners():
    return [[sx, sy, sz] for sz in (1, -1) for sx, sy in ((1, 1), (-1, 1), (-1, -1), (1, -1))]


D3Q19_XI = np.array(_REST_AXIS + _edges(), dtype=np.float64)
D3Q19_W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
D3Q15_XI = np.array(_REST_AXIS + _corners(), dtype=np.float64)
D3Q15_W = np.array([2 / 9] + [1 / 9] * 6 + [1 / 72] * 8)
D3Q27_XI = np.array(_REST_AXIS + _edges() + _corners(), dtype=np.float64)
D3Q27_W = np.array([8 / 27] + [2 / 27] * 6 + [1 / 54] * 12 + [1 / 216] * 8)
LATTICES = {ISOTHERMAL_D2Q9: (D2Q9_XI, D2Q9_W), ISOTHERMAL_D3Q19: (D3Q19_XI, D3Q19_W),
            ISOTHERMAL_D3Q15: (D3Q15_XI, D3Q15_W), ISOTHERMAL_D3Q27: (D3Q27_XI, D3Q27_W)}


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
        elif kind in LATTICES:
            assert self.dim == LATTICES[kind][0].shape[1]
            self.m = self.dim + 1
        else:
            raise ValueError(kind)
        self.lattice = kind in LATTICES
        self.nv = len(LATTICES[kind][1]) if self.lattice else 2 * self.dim
        self.groups = 1 if self.lattice else self.m

    @property
    def sound_speed(self):
        """D2Q9 / D3Q15 / D3Q19 / D3Q27: c = lambda / sqrt(3)."""
        return self.lam / np.sqrt(3.0)

    def velocities(self):
        """(n_v, D) array: row i is v_i; DnQ2n order +e_1, -e_1, +e_2, -e_2, ...;
        D2Q9 in the order of the module doc."""
        if self.lattice:
            return self.lam * LATTICES[self.kind][0]
        V = np.zeros((self.nv, self.dim))
        for a in range(self.dim):
            V[2 * a, a] = self.lam
            V[2 * a + 1, a] = -self.lam
        return V

    def moments(self, f):
        """eq. (2.2) w = P f.  DnQ2n: w_k = sum_i f_{k,i}, f of shape (m, 2D, *grid).
        D2Q9: f of shape (1, 9, *grid), w = (sum_i f_i, sum_i f_i v_i)."""
        if self.lattice:
            V = self.velocities()
            g = f[0]
            return np.stack([np.sum(g, axis=0)] + [np.tensordot(V[:, a], g, axes=(0, 0))
                                                   for a in range(self.dim)])
        return np.sum(f, axis=1)

    def flux(self, w):
        """q^a_k(w) as an array (D, m, *grid): physical flux of each variable along axis a."""
        D = self.dim
        if self.kind == ADVECTION:
            return np.stack([self.a[a] * w for a in range(D)])
        if self.lattice:
            rho, mom = w[0], w[1:]
            c2 = self.sound_speed ** 2
            out = []
            for a in range(self.dim):
                comps = [mom[a]] + [mom[a] * mom[b] / rho + (rho * c2 if a == b else 0.0)
                                    for b in range(self.dim)]
                out.append(np.stack(comps))
            return np.stack(out)
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
        if self.lattice:
            W = LATTICES[self.kind][1]
            rho = w[0]
            u = [w[1 + a] / rho for a in range(self.dim)]
            c2 = self.sound_speed ** 2
            uu = sum(ua * ua for ua in u)
            out = np.empty((1, self.nv) + w.shape[1:])
            for i, v in enumerate(self.velocities()):
                uv = sum(u[a] * v[a] for a in range(self.dim))
                out[0, i] = W[i] * rho * (1.0 + uv / c2 + uv * uv / (2.0 * c2 * c2) - uu / (2.0 * c2))
            return out
        q = self.flux(w)                                  # (D, m, *grid)
        V = self.velocities()
        out = np.empty((self.m, self.nv) + w.shape[1:])
        for i in range(self.nv):
            vq = np.tensordot(V[i], q, axes=(0, 0))       # (m, *grid)
            out[:, i] = w / (2.0 * self.dim) + vq / (2.0 * self.lam ** 2)
        return out
