"""Pins of oracle.dg: the transport matrix L_h assembled from eq. (3.7) DG_reduit."""
import numpy as np
import pytest

from oracle.dg import CartesianMesh, assemble_transport
from oracle.quadrature import gauss_lobatto, lagrange_derivative

CASES = [(1, (5,), 3), (2, (3, 4), 2), (2, (3, 3), 4), (3, (2, 3, 2), 1), (3, (2, 2, 3), 2)]


def _jump_energy(mesh, F, v):
    """-1/2 sum over faces of |v . n| (face weight) [f]^2 (closed form of F^T M L_h F)."""
    n = mesh.n
    s = 0.0
    for a in range(mesh.dim):
        Fa = np.moveaxis(F, mesh.axis_np(a), -1)
        Wo = np.ones(())
        for b in reversed(range(mesh.dim)):
            if b != a:
                Wo = np.multiply.outer(Wo, mesh.weights1d(b))
        jump = Fa[..., n - 1::n] - np.roll(Fa[..., 0::n], -1, axis=-1)
        s += -0.5 * abs(v[a]) * np.sum(Wo[..., None] * jump ** 2)
    return s


@pytest.mark.parametrize("dim,N,d", CASES)
def test_constants_in_kernel(dim, N, d):
    """Section 3.1: L_h F = 0 when all components of F are equal."""
    rng = np.random.default_rng(10 + dim)
    m = CartesianMesh(dim, N, d, lengths=tuple(rng.uniform(0.5, 2.0, dim)))
    L = assemble_transport(m, rng.standard_normal(dim))
    assert np.max(np.abs(L @ np.full(m.npoints, 3.25))) < 1e-12 * np.max(np.abs(L.data))


@pytest.mark.parametrize("dim,N,d", CASES)
def test_energy_identity_upwind_dissipation(dim, N, d):
    """Section 3.1: F^T M L_h F <= 0; with SBP it equals minus half the upwind jump energy."""
    rng = np.random.default_rng(20 + dim + d)
    m = CartesianMesh(dim, N, d, lengths=tuple(rng.uniform(0.5, 2.0, dim)))
    v = rng.standard_normal(dim)
    L = assemble_transport(m, v)
    for _ in range(3):
        F = rng.standard_normal(m.shape)
        lhs = np.sum(F * m.mass_weights() * (L @ F.reshape(-1)).reshape(m.shape))
        rhs = _jump_energy(m, F, v)
        assert lhs <= 0.0
        assert abs(lhs - rhs) <= 1e-13 * abs(rhs)


@pytest.mark.parametrize("dim,N,d", CASES)
def test_weighted_conservation(dim, N, d):
    """1^T M L_h = 0: the quadrature-weighted total of f is invariant (periodic mesh)."""
    rng = np.random.default_rng(30 + dim)
    m = CartesianMesh(dim, N, d, lengths=tuple(rng.uniform(0.5, 2.0, dim)))
    L = assemble_transport(m, rng.standard_normal(dim))
    col = L.T @ m.mass_weights().reshape(-1)
    assert np.max(np.abs(col)) < 1e-12 * np.max(np.abs(L.data)) * np.max(m.mass_weights())


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_polynomial_exactness_away_from_seam(d):
    """On cells whose upwind neighbours hold the same polynomial of degree <= d per axis,
    L_h f = -v . grad f exactly (no jumps; exact nodal derivative).  Checks the 2/h
    scaling, the sign and the axis of every term."""
    rng = np.random.default_rng(40 + d)
    m = CartesianMesh(2, (4, 5), d, lengths=(1.3, 0.7))
    v = np.array([0.8, 1.7])                      # both components positive
    L = assemble_transport(m, v)
    cx = rng.standard_normal(d + 1)
    cy = rng.standard_normal(d + 1)
    X = m.coords1d(0)[None, :]
    Y = m.coords1d(1)[:, None]
    px = np.polyval(cx, X)
    py = np.polyval(cy, Y)
    f = px * py
    grad = v[0] * np.polyval(np.polyder(cx), X) * py + v[1] * px * np.polyval(np.polyder(cy), Y)
    Lf = (L @ f.reshape(-1)).reshape(m.shape)
    n = m.n
    interior = (slice(n, None), slice(n, None))  # skip the cells fed across the periodic seam
    np.testing.assert_allclose(Lf[interior], -grad[interior], rtol=0,
                               atol=1e-11 * np.max(np.abs(grad)))


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_axis_velocity_reduces_to_line_operator(d):
    """v = lambda e_a: L_h is block bidiagonal along a with diagonal -(2 lambda/h) K,
    K = Dm + w_0^{-1} e_0 e_0^T, and upwind coupling (2 lambda/h) w_0^{-1} e_0 e_d^T
    (hand reduction of eq. (3.7) with the SBP identity)."""
    lam, N = 1.7, 4
    m = CartesianMesh(1, (N,), d, lengths=(0.9,))
    x, w = gauss_lobatto(d)
    K = lagrange_derivative(x)
    K[0, 0] += 1.0 / w[0]
    mu = 2.0 * lam / m.h[0]
    n = d + 1
    ref = np.zeros((N * n, N * n))
    for c in range(N):
        ref[c * n:(c + 1) * n, c * n:(c + 1) * n] = -mu * K
        cp = (c - 1) % N
        ref[c * n, cp * n + n - 1] += mu / w[0]
    for sgn in (+1, -1):
        L = assemble_transport(m, np.array([sgn * lam])).toarray()
        R = ref if sgn > 0 else ref[::-1, ::-1]      # mirror image for -lambda
        np.testing.assert_allclose(L, R, atol=1e-12 * mu)
