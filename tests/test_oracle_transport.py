"""Pins of oracle.transport: the theta / Crank-Nicolson step of eq. (3.11)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from golden_util import expr, rows
from oracle.dg import CartesianMesh, assemble_transport
from oracle.transport import DirectTransport, bloch_transport


def _dirs(dim, lam):
    for a in range(dim):
        for sgn in (+1, -1):
            v = np.zeros(dim)
            v[a] = sgn * lam
            yield a, sgn, v


@pytest.mark.parametrize("dim,N,d", [(2, (3, 4), 1), (2, (4, 3), 3), (3, (2, 3, 2), 2), (2, (2, 2), 4)])
@pytest.mark.parametrize("theta", [0.5, 0.75, 1.0])
@pytest.mark.parametrize("nu", [1.0, 2.0, 7.5])
def test_direct_equals_bloch(dim, N, d, theta, nu):
    """Sparse LU of the assembled eq. (3.7) system == hand-derived per-line Fourier form."""
    rng = np.random.default_rng(hash((dim, N, d)) % 1000)
    lam = 1.3
    m = CartesianMesh(dim, N, d, lengths=tuple(rng.uniform(0.5, 1.5, dim)))
    for a, sgn, v in _dirs(dim, lam):
        delta = nu * m.h[a] / (2.0 * lam)
        F = rng.standard_normal(m.shape)
        r1 = DirectTransport(m, v, delta, theta)(F)
        r2 = bloch_transport(F, m.axis_np(a), sgn, d, nu, theta)
        np.testing.assert_allclose(r1, r2, rtol=0, atol=1e-13 * np.max(np.abs(F)))


def test_d1_closed_form_recurrence():
    """d = 1, theta = 1/2, nu = 1: f_c^new = E f_c + g (f^old_{c-1,1} + x_{c-1}) with the
    hand-computed E, g and ratio beta = 1/13 of tests/golden (exact cyclic closure)."""
    gd = {k: expr(v) for k, v in rows("line_d1_theta_half_nu1.txt")}
    E = np.array([[gd["E00"], gd["E01"]], [gd["E10"], gd["E11"]]])
    g = np.array([gd["g0"], gd["g1"]])
    beta = gd["beta"]
    N, lam = 7, 2.0
    m = CartesianMesh(1, (N,), 1)
    delta = m.h[0] / (2.0 * lam)                  # nu = 2 lambda delta / h = 1
    rng = np.random.default_rng(5)
    F = rng.standard_normal(2 * N)
    got = DirectTransport(m, np.array([lam]), delta, 0.5)(F)
    fc = F.reshape(N, 2)
    # alpha_c: new last value with zero new inflow; then the cyclic closure
    alpha = np.array([(E @ fc[c])[1] + g[1] * fc[(c - 1) % N, 1] for c in range(N)])
    xlast = sum(beta ** k * alpha[N - 1 - k] for k in range(N)) / (1.0 - beta ** N)
    x = np.empty(N)
    prev = xlast
    for c in range(N):
        x[c] = alpha[c] + beta * prev
        prev = x[c]
    ref = np.array([E @ fc[c] + g * (fc[(c - 1) % N, 1] + x[(c - 1) % N]) for c in range(N)])
    np.testing.assert_allclose(got, ref.reshape(-1), rtol=0, atol=1e-14)
    np.testing.assert_allclose(ref[:, 1], x, rtol=0, atol=1e-15)


@pytest.mark.parametrize("theta", [0.5, 0.3, 1.0])
def test_time_symmetry(theta):
    """eq. (3.13) prop_sym: T_theta(-delta) T_{1-theta}(delta) = I (theta = 1/2: T(-dt) = T(dt)^-1)."""
    rng = np.random.default_rng(7)
    m = CartesianMesh(2, (3, 4), 2)
    v = np.array([0.9, -1.4])
    F = rng.standard_normal(m.shape)
    fwd = DirectTransport(m, v, 0.03, 1.0 - theta)(F)
    back = DirectTransport(m, v, -0.03, theta)(fwd)
    np.testing.assert_allclose(back, F, atol=1e-13)


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_constant_and_weighted_total_preserved(d):
    """L_h 1 = 0 => T 1 = 1; 1^T M L_h = 0 => sum M T F = sum M F."""
    rng = np.random.default_rng(8 + d)
    m = CartesianMesh(2, (3, 3), d)
    for a, sgn, v in _dirs(2, 2.0):
        T = DirectTransport(m, v, 0.7 * m.h[a], 0.5)
        np.testing.assert_allclose(T(np.full(m.shape, 2.5)), 2.5, atol=1e-13)
        F = rng.standard_normal(m.shape)
        M = m.mass_weights()
        assert abs(np.sum(M * T(F)) - np.sum(M * F)) < 1e-14 * np.sum(M * np.abs(F))


def test_crank_nicolson_third_order_local_error():
    """T_2(delta) = exp(delta L_h) + O(delta^3): compared with scipy's expm_multiply,
    the local error drops by ~8 when delta is halved."""
    rng = np.random.default_rng(9)
    m = CartesianMesh(2, (4, 4), 2)
    v = np.array([1.0, 0.6])
    L = assemble_transport(m, v)
    F = rng.standard_normal(m.npoints)
    errs = []
    for delta in (0.002, 0.001, 0.0005):
        t = DirectTransport(m, v, delta, 0.5)(F)
        e = spla.expm_multiply(delta * L, F)
        errs.append(np.linalg.norm(t - e))
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(7.5 < r < 8.5 for r in ratios), ratios
