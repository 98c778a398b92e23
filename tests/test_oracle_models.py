"""Pins of oracle.models: moments, fluxes and equilibria (Section 2)."""
import numpy as np
import pytest

from oracle import models as M


def _rand_state(model, rng, shape=(5, 4)):
    if model.kind == M.ADVECTION:
        return rng.uniform(0.5, 1.5, (1,) + shape)
    if model.kind == M.SHALLOW_WATER:
        h = rng.uniform(0.8, 1.2, shape)
        return np.stack([h, h * rng.uniform(-0.3, 0.3, shape), h * rng.uniform(-0.3, 0.3, shape)])
    D = model.dim
    rho = rng.uniform(0.8, 1.2, shape)
    u = rng.uniform(-0.3, 0.3, (D,) + shape)
    p = rng.uniform(0.8, 1.2, shape)
    E = p / (model.gamma - 1.0) + 0.5 * rho * np.sum(u * u, axis=0)
    return np.concatenate([rho[None], rho[None] * u, E[None]])


MODELS = [M.Model(M.ADVECTION, 2, 2.0, a=(1.0, 0.5)), M.Model(M.ADVECTION, 3, 3.0, a=(1.0, -0.5, 0.25)),
          M.Model(M.SHALLOW_WATER, 2, 8.0), M.Model(M.EULER, 2, 5.0), M.Model(M.EULER, 3, 5.0)]


@pytest.mark.parametrize("model", MODELS, ids=lambda m: f"k{m.kind}d{m.dim}")
def test_equilibrium_moments(model):
    """Section 2: P f^eq = w and P V^a f^eq = q^a(w) (the macroscopic flux)."""
    rng = np.random.default_rng(1)
    w = _rand_state(model, rng)
    feq = model.feq(w)
    np.testing.assert_allclose(model.moments(feq), w, rtol=1e-15, atol=1e-15)
    V = model.velocities()
    q = model.flux(w)
    for a in range(model.dim):
        first = np.tensordot(V[:, a], feq, axes=(0, 1))
        np.testing.assert_allclose(first, q[a], rtol=1e-14, atol=1e-14)


def test_advection_equilibrium_matches_workload_formula():
    """D2Q4 advection workload: f_i^eq = w/4 + (a . v_i) w / (2 lambda^2)."""
    model = M.Model(M.ADVECTION, 2, 2.0, a=(1.0, 0.5))
    w = np.random.default_rng(2).uniform(0.5, 1.5, (1, 3, 3))
    feq = model.feq(w)
    V = model.velocities()
    for i in range(4):
        ref = w[0] / 4 + (1.0 * V[i, 0] + 0.5 * V[i, 1]) * w[0] / (2 * 2.0 ** 2)
        np.testing.assert_allclose(feq[0, i], ref, rtol=1e-15)


def _jacobian_eigs(model, w, a):
    """Eigenvalues of d q^a / d w by complex-step differentiation (exact to round-off)."""
    m = model.m
    J = np.zeros((m, m))
    eps = 1e-30
    for j in range(m):
        wc = w.astype(complex)
        wc[j] += 1j * eps
        J[:, j] = np.imag(model.flux(wc)[a]) / eps
    return np.sort(np.linalg.eigvals(J).real)


def test_shallow_water_flux_wave_speeds():
    """Textbook: the SW flux Jacobian along x has eigenvalues u - c, u, u + c, c = sqrt(g h)."""
    model = M.Model(M.SHALLOW_WATER, 2, 8.0, gravity=9.81)
    h, u, v = 1.3, 0.4, -0.2
    w = np.array([h, h * u, h * v])
    for a, ua in ((0, u), (1, v)):
        c = np.sqrt(9.81 * h)
        np.testing.assert_allclose(_jacobian_eigs(model, w, a), [ua - c, ua, ua + c], rtol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_euler_flux_wave_speeds(dim):
    """Textbook: the Euler flux Jacobian along a has eigenvalues u_a - c, u_a (D times), u_a + c,
    c = sqrt(gamma p / rho)."""
    model = M.Model(M.EULER, dim, 5.0, gamma=1.4)
    rho, p = 1.1, 0.9
    u = np.array([0.3, -0.2, 0.1])[:dim]
    E = p / 0.4 + 0.5 * rho * np.dot(u, u)
    w = np.concatenate([[rho], rho * u, [E]])
    c = np.sqrt(1.4 * p / rho)
    for a in range(dim):
        ref = np.sort([u[a] - c] + [u[a]] * dim + [u[a] + c])
        np.testing.assert_allclose(_jacobian_eigs(model, w, a), ref, rtol=1e-12, atol=1e-12)
