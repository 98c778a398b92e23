"""Pins of oracle.source: the source step S_2 of M_2^s (Section 3.2) with the gravity
(Section 5.1) and penalisation (Section 5.2) sources of the D2Q9 test cases."""
import numpy as np
import pytest

from oracle import models as M
from oracle import scheme as S
from oracle.dg import CartesianMesh
from oracle.source import Source, source_step


def _setup(N=(4, 3), d=2):
    mesh = CartesianMesh(2, N, d)
    model = M.Model(M.ISOTHERMAL_D2Q9, 2, 1.0)
    return mesh, model


def _uniform(mesh, w):
    return np.stack([np.full(mesh.shape, v) for v in w])


def _state(mesh, rng):
    X = mesh.coords1d(0)[None, :]
    Y = mesh.coords1d(1)[:, None]
    rho = 1.0 + 0.05 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y + 0.4)
    return np.stack([rho, rho * 0.04 * np.cos(2 * np.pi * Y) + 0 * X, rho * 0.03 * np.sin(2 * np.pi * X)])


def test_gravity_step_closed_form():
    """rho is unchanged and rho u gains delta rho g exactly (constant source in rho u);
    the non-equilibrium part of f is kept and P f' = w'."""
    rng = np.random.default_rng(1)
    mesh, model = _setup()
    w = _state(mesh, rng)
    f = model.feq(w) + 1e-3 * rng.standard_normal((1, 9) + mesh.shape)
    src = Source(gravity=(0.3, -1.7))
    delta = 0.05
    g = source_step(f, model, mesh, src, delta)
    wg = model.moments(g)
    wf = model.moments(f)
    np.testing.assert_allclose(wg[0], wf[0], atol=1e-15)
    np.testing.assert_allclose(wg[1], wf[1] + delta * 0.3 * wf[0], atol=1e-14)
    np.testing.assert_allclose(wg[2], wf[2] - delta * 1.7 * wf[0], atol=1e-14)
    np.testing.assert_allclose(g - model.feq(wg), f - model.feq(wf), atol=1e-14)


@pytest.mark.parametrize("theta", [0.5, 1.0])
def test_penalisation_step_closed_form(theta):
    """Constant K (kappa = 0): w' - w_s = (1 - (1-theta) delta K) / (1 + theta delta K) (w - w_s)."""
    mesh, model = _setup()
    w = _uniform(mesh, (1.2, 0.05, -0.02))
    ws = (1.0, 0.0, 0.01)
    src = Source(K_s=30.0, kappa=0.0, w_s=ws, theta=theta)
    delta = 0.04
    g = source_step(model.feq(w), model, mesh, src, delta)
    fac = (1 - (1 - theta) * delta * 30.0) / (1 + theta * delta * 30.0)
    wg = model.moments(g)
    for k in range(3):
        np.testing.assert_allclose(wg[k], ws[k] + fac * (w[k] - ws[k]), atol=1e-14)


def test_penalisation_profile():
    """K(x) = K_s exp(-kappa |x - x_c|^2) at the GL points: K_s at a point placed on x_c."""
    mesh, _ = _setup((4, 4), 2)
    xc = (mesh.coords1d(0)[5], mesh.coords1d(1)[7])
    K = Source(K_s=300.0, kappa=40.0, x_c=xc).K(mesh)
    assert abs(K[7, 5] - 300.0) < 1e-12
    x, y = mesh.coords1d(0)[0], mesh.coords1d(1)[0]
    assert abs(K[0, 0] - 300.0 * np.exp(-40.0 * ((x - xc[0]) ** 2 + (y - xc[1]) ** 2))) < 1e-12


def test_source_step_time_symmetry():
    """theta = 1/2: S(-delta) S(delta) = I (eq. (3.13) for the source stage)."""
    rng = np.random.default_rng(2)
    mesh, model = _setup()
    f = model.feq(_state(mesh, rng)) + 1e-3 * rng.standard_normal((1, 9) + mesh.shape)
    src = Source(gravity=(0.0, -2.0), K_s=50.0, kappa=10.0, x_c=(0.4, 0.6))
    back = source_step(source_step(f, model, mesh, src, 0.03), model, mesh, src, -0.03)
    np.testing.assert_allclose(back, f, atol=1e-13)


@pytest.mark.parametrize("scheme", ["M2", "M2_collapsed"])
def test_uniform_fall(scheme):
    """A uniform state under gravity stays uniform and rho u grows by rho g t exactly:
    transport leaves it unchanged, C keeps w, every S(dt/2) adds dt/2 rho g."""
    mesh, model = _setup((3, 3), 1)
    w0 = _uniform(mesh, (1.3, 0.02, 0.01))
    src = Source(gravity=(0.5, -2.0))
    tr = S.Transporter(mesh, model, 0.5, "bloch")
    dt, n = 0.05, 5
    f = S.run(S.initial_state(model, w0), tr, model, dt, n, 2.0, scheme, source=src)
    w = model.moments(f)
    np.testing.assert_allclose(w[0], 1.3, atol=1e-14)
    np.testing.assert_allclose(w[1], 0.02 + n * dt * 1.3 * 0.5, atol=1e-13)
    np.testing.assert_allclose(w[2], 0.01 - n * dt * 1.3 * 2.0, atol=1e-13)


def test_m2s_second_order_and_palindrome():
    """M_2^s with gravity and a penalisation bump: second order self-convergence of w, and
    M_2^s(-dt) M_2^s(dt) = I for tau > 0."""
    rng = np.random.default_rng(3)
    mesh, model = _setup((6, 6), 2)
    w0 = _state(mesh, rng)
    src = Source(gravity=(0.0, -1.0), K_s=20.0, kappa=30.0, x_c=(0.5, 0.5), w_s=(1.0, 0.0, 0.0))
    tr = S.Transporter(mesh, model, 0.5, "bloch")
    T = 0.1
    sols = []
    for k in (2, 4, 8, 16):
        f = S.run(S.initial_state(model, w0), tr, model, T / k, k, 2.0, "M2", source=src)
        sols.append(model.moments(f))
    e = [np.linalg.norm(sols[i] - sols[i + 1]) for i in range(3)]
    r = [e[i] / e[i + 1] for i in range(2)]
    assert all(3.4 < x < 4.7 for x in r), r
    tau, dt = 0.05, 0.01
    om = lambda t: 2 * t / (2 * tau + t)
    f = model.feq(w0) + 1e-3 * rng.standard_normal((1, 9) + mesh.shape)
    g = S.m2_step(f, tr, model, dt, om(dt), src)
    np.testing.assert_allclose(S.m2_step(g, tr, model, -dt, om(-dt), src), f, atol=1e-12)


def test_hydrostatic_state_time_order():
    """Section 5.1: at rest under gravity, with the exact hydrostatic state
    rho_0 exp(-g y / c^2) as initial state and as inflow data on the y faces (x periodic),
    M_2^s keeps the state to discretisation accuracy, and its error in time is of second
    order (self-convergence of w at fixed mesh)."""
    mesh = CartesianMesh(2, (2, 12), 2, periodic=(True, False))
    model = M.Model(M.ISOTHERMAL_D2Q9, 2, 1.0)
    g, c2 = 1.0, 1.0 / 3.0
    Y = mesh.coords1d(1)[:, None] + 0 * mesh.coords1d(0)[None, :]
    wex = np.stack([np.exp(-g * Y / c2), 0 * Y, 0 * Y])
    fb = model.feq(wex)
    tr = S.Transporter(mesh, model, 0.5, "direct", fb=fb)
    src = Source(gravity=(0.0, -g))
    T = 0.12
    sols = []
    for k in (3, 6, 12, 24):
        f = S.run(S.initial_state(model, wex), tr, model, T / k, k, 2.0, "M2", source=src)
        sols.append(model.moments(f))
    assert np.linalg.norm(sols[-1][0] - wex[0]) / np.linalg.norm(wex[0]) < 1e-3
    e = [np.linalg.norm(sols[i] - sols[i + 1]) for i in range(3)]
    r = [e[i] / e[i + 1] for i in range(2)]
    assert all(3.3 < x < 4.8 for x in r), r
