"""Nodal upwind DG transport matrix on an affine periodic Cartesian mesh (oracle).

Test infrastructure only.  Assembles L_h of eq. (3.9) linear_ODE for ONE
constant velocity v, term by term from eq. (3.7) DG_reduit (Section 3.1):

  d/dt f_{L,i} =  (1/omega_{L,i}) sum_j  v . c_{L,j} grad^phi_i(x^_j) f_{L,j} omega_j
               -  (1/omega_{L,i}) sum_eps mu_i^eps ( (v . c_{L,i} n^_eps)^+ f_{L,i}
                                                   + (v . c_{L,i} n^_eps)^- f_{R,i'} )

with omega_{L,i} = omega_i det tau_L' (eq. (3.3) map_GL), the cofactor
c = co(tau_L') = det(tau_L') tau_L'^{-T} (eq. (3.6) co_mat), reference face
weights mu_i^eps (product of the 1-D GL weights of the other directions, zero
off the face) and conformal matching x_{L,i} = x_{R,i'}.

Reading (the configurations are Cartesian): every cell is the box
prod_a [c_a h_a, (c_a+1) h_a] and tau_L(x^) = centre + diag(h_a/2) x^, so
det tau_L' = prod_a h_a/2 and c = diag(det * 2/h_a).  All faces are periodic:
the neighbour across the face (a, +) of cell c is c + e_a modulo N_a.

Point numbering (both sides of the test-suite use it): along axis a the global
index is g_a = c_a (d+1) + i_a, so face points are duplicated (DG); arrays are
stored numpy-C-order with axis x LAST: shape (P_z, P_y, P_x) in 3-D,
(P_y, P_x) in 2-D, flat index = g_x + P_x (g_y + P_y g_z).
"""
import itertools

import numpy as np
import scipy.sparse as sp

from .quadrature import gauss_lobatto, lagrange_derivative


class CartesianMesh:
    """Periodic Cartesian DG mesh: dim D, N_a cells per axis, degree d, box lengths.

    The paper's macrocell/subcell split (Section 4.3) only groups cells; on a
    regular grid N_a = n_macro_a * n_sub_a and the discrete problem depends on
    N_a alone.
    """

    def __init__(self, dim, ncells, d, lengths=None, periodic=None):
        self.dim = int(dim)
        self.periodic = tuple(bool(p) for p in (periodic if periodic is not None else (True,) * dim))
        self.N = tuple(int(v) for v in ncells)
        assert len(self.N) == self.dim
        self.d = int(d)
        self.n = self.d + 1
        self.lengths = tuple(float(v) for v in (lengths or (1.0,) * self.dim))
        self.h = tuple(self.lengths[a] / self.N[a] for a in range(self.dim))
        self.P = tuple(self.N[a] * self.n for a in range(self.dim))
        self.xhat, self.what = gauss_lobatto(self.d)

    @property
    def shape(self):
        """numpy shape of one field: axes reversed so that x is last."""
        return tuple(reversed(self.P))

    @property
    def npoints(self):
        return int(np.prod(self.P))

    def axis_np(self, a):
        """numpy axis (negative) of geometric axis a (0=x, 1=y, 2=z)."""
        return -1 - a

    def coords1d(self, a):
        """Physical GL coordinates along axis a, eq. (3.3): x = c h + (h/2)(1 + x^)."""
        h = self.h[a]
        c = np.arange(self.N[a])[:, None]
        return (c * h + 0.5 * h * (1.0 + self.xhat[None, :])).reshape(-1)

    def weights1d(self, a):
        """Per-point 1-D weight w_{i_a} h_a / 2 along axis a."""
        return np.tile(self.what * (0.5 * self.h[a]), self.N[a])

    def mass_weights(self):
        """omega_{L,i} = omega_i det tau_L' at every point (eq. (3.3)), field-shaped."""
        out = np.ones(())
        for a in reversed(range(self.dim)):
            out = np.multiply.outer(out, self.weights1d(a))
        return out

    def flat_index(self, g):
        """Flat index of global point multi-index g = (g_x, g_y, ...)."""
        idx = 0
        stride = 1
        for a in range(self.dim):
            idx = idx + g[a] * stride
            stride *= self.P[a]
        return idx


def assemble_transport(mesh, v, with_boundary=False):
    """Sparse L_h (npoints x npoints) for constant velocity v; eq. (3.7) DG_reduit.

    Every term of eq. (3.7) is added literally, for every local pair (i, j) and
    every face eps, vectorised over the cells (uniform affine cells share the
    coefficients).

    Non-periodic axes (mesh.periodic[a] False) end at the domain boundary.  There the
    neighbour value f_{R,i'} is the boundary datum f^b at the same face point (the
    fictitious cell of eq. (3.8)); its coefficient - (1/omega_{L,i}) mu (v.c n^)^- is
    returned, per point, in `bcoef` when with_boundary is True: the semi-discrete
    system is d/dt f = L_h f + bcoef * f^b (only inflow face points have bcoef != 0).
    """
    D = mesh.dim
    n = mesh.n
    v = np.asarray(v, dtype=np.float64)
    assert v.shape == (D,)
    Dm = lagrange_derivative(mesh.xhat)          # Dm[j, i] = l_i'(x_j)
    w1 = mesh.what
    det = float(np.prod([0.5 * h for h in mesh.h]))
    cof = np.array([det * 2.0 / mesh.h[a] for a in range(D)])   # diagonal of co(tau')

    # cell multi-indices, x fastest
    cell_axes = [np.arange(mesh.N[a]) for a in range(D)]
    grids = np.meshgrid(*cell_axes, indexing="ij")
    cells = [g.reshape(-1) for g in grids]         # cells[a][q] = c_a of cell q

    def gidx(cellc, loc):
        return mesh.flat_index([cellc[a] * n + loc[a] for a in range(D)])

    rows, cols, vals = [], [], []
    brows, bvals = [], []
    locs = list(itertools.product(range(n), repeat=D))   # loc[a] = i_a
    for i in locs:
        omega_i = float(np.prod([w1[i[a]] for a in range(D)]))
        omega_Li = omega_i * det
        row = gidx(cells, i)
        # volume term: + (1/omega_Li) sum_j v.c grad^phi_i(x^_j) f_j omega_j
        for j in locs:
            grad = np.zeros(D)
            for a in range(D):
                others = all(i[b] == j[b] for b in range(D) if b != a)
                grad[a] = Dm[j[a], i[a]] if others else 0.0
            coef = float(np.dot(v, cof * grad))
            if coef == 0.0:
                continue
            omega_j = float(np.prod([w1[j[a]] for a in range(D)]))
            rows.append(row)
            cols.append(gidx(cells, j))
            vals.append(np.full(row.shape, coef * omega_j / omega_Li))
        # face terms: - (1/omega_Li) mu_i^eps ((v.c n^)^+ f_L,i + (v.c n^)^- f_R,i')
        for a in range(D):
            for s in (-1, +1):
                on_face = i[a] == (n - 1 if s > 0 else 0)
                if not on_face:
                    continue                       # mu_i^eps = 0
                mu = float(np.prod([w1[i[b]] for b in range(D) if b != a]))
                vn = s * v[a] * cof[a]             # v . c n^_eps, n^ = s e_a
                vp, vm = max(vn, 0.0), min(vn, 0.0)
                if vp != 0.0:
                    rows.append(row)
                    cols.append(row)
                    vals.append(np.full(row.shape, -mu * vp / omega_Li))
                if vm != 0.0:
                    ncell = [c.copy() for c in cells]
                    ncell[a] = (cells[a] + s) % mesh.N[a]
                    ip = list(i)
                    ip[a] = 0 if s > 0 else n - 1   # matching point x_{L,i} = x_{R,i'}
                    inside = np.ones(row.shape, dtype=bool)
                    if not mesh.periodic[a]:
                        inside = (cells[a] + s >= 0) & (cells[a] + s < mesh.N[a])
                    coef = -mu * vm / omega_Li
                    rows.append(row[inside])
                    cols.append(gidx(ncell, ip)[inside])
                    vals.append(np.full(int(inside.sum()), coef))
                    if not inside.all():             # fictitious cell: f_R = f^b at the face point
                        brows.append(row[~inside])
                        bvals.append(np.full(int((~inside).sum()), coef))
    N = mesh.npoints
    if not rows:                                   # v = 0: every term of eq. (3.7) vanishes
        rows, cols, vals = [np.zeros(0, dtype=np.int64)], [np.zeros(0, dtype=np.int64)], [np.zeros(0)]
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    L = sp.coo_matrix((vals, (rows, cols)), shape=(N, N)).tocsr()
    if not with_boundary:
        return L
    bcoef = np.zeros(N)
    if brows:
        np.add.at(bcoef, np.concatenate(brows), np.concatenate(bvals))
    return L, bcoef.reshape(mesh.shape)
