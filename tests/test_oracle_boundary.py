"""Pins of the inflow-boundary oracle (eq. (2.6) boundary_conditions, eq. (3.8)
fictitious cells, Section 4.1 triangular structure)."""
import numpy as np
import pytest

from golden_util import expr, rows
from oracle import models as M
from oracle import scheme as S
from oracle.dg import CartesianMesh, assemble_transport
from oracle.transport import DirectTransport

CASES = [(1, (5,), 3, (False,)), (2, (3, 4), 2, (False, True)), (2, (3, 3), 1, (False, False)),
         (3, (2, 3, 2), 2, (True, False, False))]


def _energy_with_boundary(mesh, F, v):
    """-1/2 sum over interior faces of |v.n| (weight) [f]^2 - 1/2 sum over boundary faces
    of |v.n| (weight) f^2 (zero boundary data)."""
    n = mesh.n
    s = 0.0
    for a in range(mesh.dim):
        Fa = np.moveaxis(F, mesh.axis_np(a), -1)
        Wo = np.ones(())
        for b in reversed(range(mesh.dim)):
            if b != a:
                Wo = np.multiply.outer(Wo, mesh.weights1d(b))
        right = Fa[..., n - 1::n]
        left = Fa[..., 0::n]
        if mesh.periodic[a]:
            jump = right - np.roll(left, -1, axis=-1)
            s += -0.5 * abs(v[a]) * np.sum(Wo[..., None] * jump ** 2)
        else:
            jump = right[..., :-1] - left[..., 1:]
            s += -0.5 * abs(v[a]) * np.sum(Wo[..., None] * jump ** 2)
            s += -0.5 * abs(v[a]) * np.sum(Wo * (left[..., 0] ** 2 + right[..., -1] ** 2))
    return s


@pytest.mark.parametrize("dim,N,d,per", CASES)
def test_energy_identity_with_boundaries(dim, N, d, per):
    """Upwind dissipation with inflow data zero: boundary faces dissipate |v.n| f^2 / 2."""
    rng = np.random.default_rng(70 + dim + d)
    m = CartesianMesh(dim, N, d, lengths=tuple(rng.uniform(0.5, 2.0, dim)), periodic=per)
    v = rng.standard_normal(dim)
    L = assemble_transport(m, v)
    for _ in range(3):
        F = rng.standard_normal(m.shape)
        lhs = np.sum(F * m.mass_weights() * (L @ F.reshape(-1)).reshape(m.shape))
        rhs = _energy_with_boundary(m, F, v)
        assert lhs <= 0 and abs(lhs - rhs) <= 1e-13 * abs(rhs)


@pytest.mark.parametrize("dim,N,d,per", CASES)
def test_constant_state_with_matching_inflow_is_steady(dim, N, d, per):
    rng = np.random.default_rng(80 + dim)
    m = CartesianMesh(dim, N, d, periodic=per)
    L, bcoef = assemble_transport(m, rng.standard_normal(dim), with_boundary=True)
    c = 1.7
    r = (L @ np.full(m.npoints, c)).reshape(m.shape) + bcoef * c
    assert np.max(np.abs(r)) < 1e-12 * np.max(np.abs(L.data))


def test_block_triangular_in_upwind_order():
    """Section 4.1: with inflow boundaries the dependency graph is a DAG; for a velocity
    with positive components, every coupling goes from a cell to a cell with no larger
    index along any axis (block lower-triangular in that order)."""
    m = CartesianMesh(2, (4, 3), 2, periodic=(False, False))
    L = assemble_transport(m, np.array([0.7, 1.3])).tocoo()
    n = m.n
    gx_r, gy_r = L.row % m.P[0], L.row // m.P[0]
    gx_c, gy_c = L.col % m.P[0], L.col // m.P[0]
    assert np.all(gx_c // n <= gx_r // n) and np.all(gy_c // n <= gy_r // n)
    # and the periodic mesh is not triangular (the graph has cycles)
    Lp = assemble_transport(CartesianMesh(2, (4, 3), 2), np.array([0.7, 1.3])).tocoo()
    assert np.any((Lp.col % m.P[0]) // n > (Lp.row % m.P[0]) // n)


def test_d1_inflow_recurrence_golden():
    """d = 1, theta = 1/2, nu = 1, inflow datum b at the left face: the fictitious cell
    is constant, so fn_0 = E f_0 + g (b + b) and fn_c = E f_c + g (f_{c-1,1} + x_{c-1})
    with the hand-computed E, g of tests/golden (an open chain: no cyclic closure)."""
    gd = {k: expr(v) for k, v in rows("line_d1_theta_half_nu1.txt")}
    E = np.array([[gd["E00"], gd["E01"]], [gd["E10"], gd["E11"]]])
    g = np.array([gd["g0"], gd["g1"]])
    N, lam, b = 6, 2.0, 0.37
    m = CartesianMesh(1, (N,), 1, periodic=(False,))
    delta = m.h[0] / (2.0 * lam)
    F = np.random.default_rng(81).standard_normal(2 * N)
    fb = np.zeros(2 * N)
    fb[0] = b
    got = DirectTransport(m, np.array([lam]), delta, 0.5)(F, fb)
    fc = F.reshape(N, 2)
    out = np.empty((N, 2))
    xprev, uprev = b, b
    for c in range(N):
        out[c] = E @ fc[c] + g * (uprev + xprev)
        xprev, uprev = out[c, 1], fc[c, 1]
    np.testing.assert_allclose(got, out.reshape(-1), rtol=0, atol=1e-14)


def test_m2_constant_equilibrium_with_matching_inflow():
    """M2 with inflow data f^b = f^eq(w_c) keeps the constant equilibrium f^eq(w_c)."""
    model = M.Model(M.SHALLOW_WATER, 2, 8.0)
    m = CartesianMesh(2, (3, 2), 2, periodic=(False, True))
    w = np.array([1.1, 0.2, -0.1]).reshape(3, 1, 1) * np.ones(m.shape)
    f0 = S.initial_state(model, w)
    tr = S.Transporter(m, model, method="direct", fb=f0)
    f = S.run(f0, tr, model, 0.5 * m.h[0] / model.lam, 3, 2.0)
    np.testing.assert_allclose(f, f0, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("kind,q", [(M.ISOTHERMAL_D3Q19, 19), (M.ISOTHERMAL_D3Q15, 15), (M.ISOTHERMAL_D3Q27, 27)])
def test_3d_lattice_constant_equilibrium_with_matching_inflow(kind, q):
    """The 3-D lattices on a box with inflow faces on every axis: boundary data f^b =
    f^eq(w_c) keep the constant equilibrium under M2 (edge and corner velocities included;
    the oracle the 3-D inflow GPU tests compare with)."""
    model = M.Model(kind, 3, 1.0)
    m = CartesianMesh(3, (2, 2, 3), 1, periodic=(False, False, False))
    w = np.array([1.05, 0.02, -0.01, 0.03]).reshape(4, 1, 1, 1) * np.ones(m.shape)
    f0 = S.initial_state(model, w)
    assert f0.shape == (1, q) + m.shape
    tr = S.Transporter(m, model, method="direct", fb=f0)
    f = S.run(f0, tr, model, 0.5 * min(m.h) / model.lam, 2, 2.0)
    np.testing.assert_allclose(f, f0, rtol=1e-13, atol=1e-13)
