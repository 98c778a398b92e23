"""Pins of oracle.quadrature (Section 3.1: GL points, weights, nodal basis)."""
import numpy as np
import pytest

from golden_util import expr, rows
from oracle.quadrature import gauss_lobatto, lagrange_derivative, lagrange_eval


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_gl_nodes_weights_textbook(d):
    """Nodes/weights equal the closed forms of Abramowitz & Stegun 25.4.32 (tests/golden)."""
    ref = [(expr(x), expr(w)) for dd, x, w in rows("gauss_lobatto.txt") if int(dd) == d]
    x, w = gauss_lobatto(d)
    assert len(x) == d + 1 == len(ref)
    np.testing.assert_allclose(x, [r[0] for r in ref], rtol=0, atol=4.5e-16)
    np.testing.assert_allclose(w, [r[1] for r in ref], rtol=2e-15, atol=0)


@pytest.mark.parametrize("d", [1, 2, 3, 4, 6, 9])
def test_gl_exact_degree(d):
    """GL with d+1 points integrates x^p exactly for p <= 2d-1 and not for p = 2d."""
    x, w = gauss_lobatto(d)
    for p in range(0, 2 * d):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert abs(np.sum(w * x ** p) - exact) < 1e-14
    p = 2 * d
    assert abs(np.sum(w * x ** p) - 2.0 / (p + 1)) > 1e-8


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_derivative_matrix_exact_on_polynomials(d):
    """(Dm f)_j = f'(x_j) for every polynomial f of degree <= d (Dm[j,i] = l_i'(x_j))."""
    x, _ = gauss_lobatto(d)
    Dm = lagrange_derivative(x)
    for p in range(d + 1):
        f = x ** p
        fp = p * x ** (p - 1) if p > 0 else np.zeros_like(x)
        np.testing.assert_allclose(Dm @ f, fp, atol=2e-14)


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_sbp_identity(d):
    """W Dm + Dm^T W = e_d e_d^T - e_0 e_0^T (integration by parts, exact GL quadrature)."""
    x, w = gauss_lobatto(d)
    Dm = lagrange_derivative(x)
    W = np.diag(w)
    Bd = np.zeros((d + 1, d + 1))
    Bd[0, 0], Bd[d, d] = -1.0, 1.0
    np.testing.assert_allclose(W @ Dm + Dm.T @ W, Bd, atol=3e-15)


def test_d1_derivative_closed_form():
    """Two-point basis l_0 = (1-x)/2, l_1 = (1+x)/2: Dm = [[-1/2, 1/2], [-1/2, 1/2]] (golden)."""
    g = {k: expr(v) for k, v in rows("line_d1_theta_half_nu1.txt")}
    Dm = lagrange_derivative(gauss_lobatto(1)[0])
    np.testing.assert_array_equal(Dm, [[g["Dm00"], g["Dm01"]], [g["Dm10"], g["Dm11"]]])


@pytest.mark.parametrize("d", [2, 3, 4])
def test_interpolation_property(d):
    """eq. (3.4): phi_i(x_j) = delta_ij."""
    x, _ = gauss_lobatto(d)
    for i in range(d + 1):
        np.testing.assert_allclose(lagrange_eval(x, i, x), np.eye(d + 1)[i], atol=1e-15)
