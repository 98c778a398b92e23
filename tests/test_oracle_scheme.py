"""Pins of oracle.scheme: collision (eq. (3.12)) and the palindromic step M2 (Section 3.2)."""
import numpy as np
import pytest

from oracle import models as M
from oracle import scheme as S
from oracle.dg import CartesianMesh


def _sw_state(mesh, rng):
    X = mesh.coords1d(0)[None, :]
    Y = mesh.coords1d(1)[:, None]
    h = 1.0 + 0.1 * np.sin(2 * np.pi * X + 0.3) * np.cos(2 * np.pi * Y)
    hu = 0.05 * np.cos(2 * np.pi * Y) + 0 * X
    hv = 0.03 * np.sin(2 * np.pi * X) + 0 * Y
    return np.stack([h, hu, hv])


def _euler3_state(mesh):
    X = mesh.coords1d(0)[None, None, :]
    Y = mesh.coords1d(1)[None, :, None]
    Z = mesh.coords1d(2)[:, None, None]
    rho = 1.0 + 0.05 * np.sin(2 * np.pi * (X + Y)) + 0 * Z
    u = [0.1 * np.cos(2 * np.pi * Z) + 0 * X + 0 * Y, 0.05 * np.sin(2 * np.pi * X) + 0 * Y + 0 * Z,
         0.02 + 0 * X + 0 * Y + 0 * Z]
    E = 1.0 / 0.4 + 0.5 * rho * sum(v * v for v in u)
    return np.stack([rho] + [rho * v for v in u] + [E])


def test_collision_conserves_moments_and_is_involution():
    """eq. (3.12): C keeps w = P f; omega = 2 (tau = 0) gives C F = 2 F^eq - F, so C o C = I;
    omega = 1 returns F^eq."""
    rng = np.random.default_rng(3)
    model = M.Model(M.SHALLOW_WATER, 2, 8.0)
    mesh = CartesianMesh(2, (2, 3), 2)
    f = model.feq(_sw_state(mesh, rng)) + 1e-2 * rng.standard_normal((3, 4) + mesh.shape)
    c2 = S.collision(f, model, 2.0)
    np.testing.assert_allclose(model.moments(c2), model.moments(f), atol=1e-14)
    np.testing.assert_allclose(S.collision(c2, model, 2.0), f, atol=1e-14)
    np.testing.assert_allclose(S.collision(f, model, 1.0), model.feq(model.moments(f)), atol=1e-15)


def test_collision_time_symmetry_positive_tau():
    """eq. (3.13) for C_2 (tau > 0): C_2(-dt) C_2(dt) = I, with omega(dt) = 2 dt / (2 tau + dt)."""
    rng = np.random.default_rng(4)
    model = M.Model(M.EULER, 2, 5.0)
    mesh = CartesianMesh(2, (2, 2), 1)
    X = mesh.coords1d(0)[None, :]
    w = np.stack([1 + 0.1 * np.sin(2 * np.pi * X) + 0 * X.T, 0.1 + 0 * X + 0 * X.T,
                  -0.05 + 0 * X + 0 * X.T, 2.5 + 0 * X + 0 * X.T])
    f = model.feq(w) + 1e-2 * rng.standard_normal((4, 4) + mesh.shape)
    tau, dt = 0.3, 0.1
    om = lambda t: 2 * t / (2 * tau + t)
    back = S.collision(S.collision(f, model, om(dt)), model, om(-dt))
    np.testing.assert_allclose(back, f, atol=1e-13)


def test_m2_time_symmetric_for_positive_tau():
    """eq. (3.13) for the palindrome: M2(-dt) M2(dt) = I when tau > 0 (nonlinear SW model).
    A non-palindromic ordering of T and C would break it."""
    rng = np.random.default_rng(5)
    model = M.Model(M.SHALLOW_WATER, 2, 8.0)
    mesh = CartesianMesh(2, (3, 3), 2)
    f = model.feq(_sw_state(mesh, rng)) + 1e-3 * rng.standard_normal((3, 4) + mesh.shape)
    tr = S.Transporter(mesh, model, method="direct")
    tau, dt = 0.02, 0.01
    om = lambda t: 2 * t / (2 * tau + t)
    g = S.m2_step(f, tr, model, dt, om(dt))
    back = S.m2_step(g, tr, model, -dt, om(-dt))
    np.testing.assert_allclose(back, f, atol=1e-12)


def test_m2_tau_zero_limit():
    """Section 3.2: with tau = 0, M2(0) F = 2 F^eq(F) - F."""
    rng = np.random.default_rng(6)
    model = M.Model(M.ADVECTION, 2, 2.0, a=(1.0, 0.5))
    mesh = CartesianMesh(2, (2, 2), 3)
    f = rng.uniform(0.1, 1.0, (1, 4) + mesh.shape)
    tr = S.Transporter(mesh, model, method="direct")
    np.testing.assert_allclose(S.m2_step(f, tr, model, 0.0, 2.0), 2 * model.feq(model.moments(f)) - f,
                               atol=1e-14)


@pytest.mark.parametrize("model,dim", [(M.Model(M.ADVECTION, 2, 2.0, a=(1.0, 0.5)), 2),
                                       (M.Model(M.SHALLOW_WATER, 2, 8.0), 2),
                                       (M.Model(M.EULER, 3, 5.0), 3)])
def test_m2_constant_state_invariant(model, dim):
    """A constant equilibrium is a fixed point of M2 (L_h 1 = 0 and C F^eq = F^eq)."""
    mesh = CartesianMesh(dim, (2,) * dim, 2)
    wc = {M.ADVECTION: [1.3], M.SHALLOW_WATER: [1.1, 0.2, -0.1], M.EULER: [1.2, 0.1, -0.2, 0.05, 2.9]}
    w = np.array(wc[model.kind]).reshape((-1,) + (1,) * dim) * np.ones(mesh.shape)
    f0 = S.initial_state(model, w)
    tr = S.Transporter(mesh, model, method="bloch")
    f = S.run(f0, tr, model, 0.5 * mesh.h[0] / model.lam, 3, 2.0)
    np.testing.assert_allclose(f, f0, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("scheme", ["M2", "M2_collapsed"])
def test_m2_weighted_conservation(scheme):
    """sum_points omega_{L,i} w_k is conserved by T and C, hence by M2 (SW and 3-D Euler)."""
    rng = np.random.default_rng(7)
    for model, mesh, w in [
        (M.Model(M.SHALLOW_WATER, 2, 8.0), CartesianMesh(2, (3, 4), 3), None),
        (M.Model(M.EULER, 3, 5.0), CartesianMesh(3, (2, 2, 3), 2), None),
    ]:
        w = _sw_state(mesh, rng) if model.kind == M.SHALLOW_WATER else _euler3_state(mesh)
        f0 = S.initial_state(model, w)
        tr = S.Transporter(mesh, model, method="bloch")
        f = S.run(f0, tr, model, mesh.h[0] / model.lam, 4, 2.0, scheme)
        t0 = S.weighted_total(mesh, model.moments(f0))
        t1 = S.weighted_total(mesh, model.moments(f))
        np.testing.assert_allclose(t1, t0, rtol=0, atol=1e-14 * np.max(np.abs(t0)) + 1e-15)


def test_m2_plain_sum_not_invariant_for_d2():
    """Reading of 'conservation of sum(w)': the plain unweighted point sum is NOT invariant
    for d >= 2 (the GL weights differ); the weighted sum is (previous test)."""
    model = M.Model(M.ADVECTION, 2, 2.0, a=(1.0, 0.5))
    mesh = CartesianMesh(2, (4, 4), 2)
    X = mesh.coords1d(0)[None, :]
    Y = mesh.coords1d(1)[:, None]
    w = (1.0 + np.exp(-((X - 0.3) ** 2 + (Y - 0.6) ** 2) / 0.02))[None]
    f = S.run(S.initial_state(model, w), S.Transporter(mesh, model, method="bloch"), model,
              mesh.h[0] / model.lam, 3, 2.0)
    assert abs(np.sum(model.moments(f)) - np.sum(w)) > 1e-6


def _advection_error(d, N, scheme):
    a, lam = np.array([1.0, 0.5]), 2.0
    model = M.Model(M.ADVECTION, 2, lam, a=a)
    mesh = CartesianMesh(2, (N, N), d)
    X = mesh.coords1d(0)[None, :]
    Y = mesh.coords1d(1)[:, None]
    w0 = lambda x, y: 1.0 + np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) + 0.5 * np.cos(2 * np.pi * (x + y))
    dt = mesh.h[0] / lam
    ns = int(round(0.25 / dt))
    f = S.run(S.initial_state(model, w0(X, Y)[None]), S.Transporter(mesh, model, method="bloch"),
              model, dt, ns, 2.0, scheme)
    ex = w0(X - a[0] * ns * dt, Y - a[1] * ns * dt)
    Mw = mesh.mass_weights()
    return np.sqrt(np.sum(Mw * (model.moments(f)[0] - ex) ** 2) / np.sum(Mw * ex ** 2))


@pytest.mark.parametrize("scheme", ["M2", "M2_collapsed"])
@pytest.mark.parametrize("d", [2, 3])
def test_advection_converges_to_exact_translation_second_order(scheme, d):
    """w -> w0(x - a t) on the periodic square at second order (h and dt refined together at
    CFL 1; relative L2 error of w, the measure of Section 5.1)."""
    errs = [_advection_error(d, N, scheme) for N in (8, 16, 32)]
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(slopes > 1.8) and slopes[-1] > 1.9, (errs, slopes)
    assert errs[-1] < 1e-2


def test_collapsed_single_step_equals_m2():
    """With one step the collapsed scheme is exactly M2 (no interior merge)."""
    model = M.Model(M.SHALLOW_WATER, 2, 8.0)
    mesh = CartesianMesh(2, (2, 3), 2)
    f0 = S.initial_state(model, _sw_state(mesh, None))
    tr = S.Transporter(mesh, model, method="bloch")
    dt = mesh.h[0] / model.lam
    np.testing.assert_allclose(S.run(f0, tr, model, dt, 1, 2.0, "M2_collapsed"),
                               S.run(f0, tr, model, dt, 1, 2.0, "M2"), atol=0, rtol=0)


def test_m2kin_zero_step_is_identity_unlike_m2():
    """Section 3.2: with tau = 0, M2(0) F = 2 F^eq - F != F, while
    M2^kin(0) = C_2 C_2 = I (the collision is an involution at omega = 2)."""
    rng = np.random.default_rng(61)
    model = M.Model(M.SHALLOW_WATER, 2, 8.0)
    mesh = CartesianMesh(2, (2, 3), 2)
    f = model.feq(_sw_state(mesh, rng)) + 1e-2 * rng.standard_normal((3, 4) + mesh.shape)
    tr = S.Transporter(mesh, model, method="direct")
    np.testing.assert_allclose(S.run(f, tr, model, 0.0, 1, 2.0, "M2_kin"), f, atol=1e-14)
    assert np.max(np.abs(S.run(f, tr, model, 0.0, 1, 2.0, "M2") - f)) > 1e-3


def test_m2kin_time_symmetric_for_positive_tau():
    """The palindrome M2^kin with C_2(dt/2) weights omega(dt/2) = dt/(2 tau + dt/2):
    M2^kin(-dt) M2^kin(dt) = I when tau > 0."""
    rng = np.random.default_rng(62)
    model = M.Model(M.SHALLOW_WATER, 2, 8.0)
    mesh = CartesianMesh(2, (3, 2), 2)
    f = model.feq(_sw_state(mesh, rng)) + 1e-3 * rng.standard_normal((3, 4) + mesh.shape)
    tr = S.Transporter(mesh, model, method="direct")
    tau, dt = 0.02, 0.01
    om = lambda t: 2 * (t / 2) / (2 * tau + t / 2)
    g = S.run(f, tr, model, dt, 1, om(dt), "M2_kin")
    back = S.run(g, tr, model, -dt, 1, om(-dt), "M2_kin")
    np.testing.assert_allclose(back, f, atol=1e-12)


@pytest.mark.parametrize("d", [2, 3])
def test_m2kin_second_order(d):
    errs = [_advection_error(d, N, "M2_kin") for N in (8, 16, 32)]
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(slopes > 1.8) and slopes[-1] > 1.9, (errs, slopes)


def test_triple_jump_coefficients():
    """The order conditions of the symmetric triple jump: consistency 2 g1 + g2 = 1 and
    cancellation of the third-order error term 2 g1^3 + g2^3 = 0 (g2 < 0)."""
    g1, g2 = S.triple_jump()
    assert abs(2 * g1 + g2 - 1.0) < 1e-15
    assert abs(2 * g1 ** 3 + g2 ** 3) < 1e-14
    assert g2 < 0 < g1


def test_m4kin_time_symmetric_and_conservative():
    """omega = 2: M4^kin(-dt) M4^kin(dt) = I (composition of time-symmetric steps), and
    the weighted totals of w are kept."""
    rng = np.random.default_rng(63)
    model = M.Model(M.SHALLOW_WATER, 2, 8.0)
    mesh = CartesianMesh(2, (3, 2), 2)
    f = model.feq(_sw_state(mesh, rng)) + 1e-3 * rng.standard_normal((3, 4) + mesh.shape)
    tr = S.Transporter(mesh, model, method="bloch")
    dt = 0.2 * min(mesh.h) / model.lam
    g = S.run(f, tr, model, dt, 1, 2.0, "M4_kin")
    np.testing.assert_allclose(S.run(g, tr, model, -dt, 1, 2.0, "M4_kin"), f, atol=1e-12)
    np.testing.assert_allclose(S.weighted_total(mesh, model.moments(g)), S.weighted_total(mesh, model.moments(f)),
                               rtol=0, atol=1e-13)


def test_m4kin_fourth_order_in_time():
    """Fixed mesh, dt halved: successive differences of w shrink by about 2^4 for the
    triple jump (2^2 for M2^kin itself), on the advection workload at omega = 2."""
    import dataclasses
    from paper_1702_00169_gb300 import workloads as W
    cfg = dataclasses.replace(W.ADVECTION_D2Q4, n_macro=(4, 4), n_sub=(2, 2), order=3)
    mesh = CartesianMesh(2, cfg.ncells, cfg.order)
    model = M.Model(M.ADVECTION, 2, cfg.lam, a=cfg.a[:2])
    w0 = W.initial_w(cfg, [mesh.coords1d(a) for a in range(2)])
    tr = S.Transporter(mesh, model, 0.5, "bloch")
    T = 0.05
    for scheme, lo, hi in (("M2_kin", 3.7, 4.3), ("M4_kin", 13.0, 19.0)):
        res = [model.moments(S.run(S.initial_state(model, w0), tr, model, T / N, N, 2.0, scheme))
               for N in (8, 16, 32)]
        e = [np.abs(res[0] - res[1]).max(), np.abs(res[1] - res[2]).max()]
        assert lo < e[0] / e[1] < hi, (scheme, e)


def test_backward_steps_amplify_rounding_forward_steps_do_not():
    """The conditioning behind the pointwise bar of time-reversed GPU runs: the backward theta
    step (the inverse of the forward one, eq. (3.13)) is anti-dissipative, so a one-ulp
    perturbation of the input grows to ~1e-12 of max|f| in three backward M2 steps, while
    three forward steps keep it at ~1e-14.  Two correct FP64 evaluations that round
    differently can therefore differ pointwise by more than 1e-12 only when run backwards."""
    import dataclasses
    import os
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    from gpu_common import TOL_POINTWISE_REVERSED, oracle_mesh, oracle_model, oracle_w0
    from paper_1702_00169_gb300 import workloads as W
    worst_b = []
    for order in (2, 3):
        cfg = dataclasses.replace(W.SW_D2Q4, n_macro=(3, 2), n_sub=(3, 4), order=order)
        model = oracle_model(cfg)
        tr = S.Transporter(oracle_mesh(cfg), model, theta=cfg.theta, method="bloch")
        f0 = S.initial_state(model, oracle_w0(cfg))
        rng = np.random.default_rng(order)
        pert = f0 * (1 + 2.0 ** -52 * rng.standard_normal(f0.shape))
        for sign, store in ((-1, worst_b), (1, None)):
            a = S.run(f0, tr, model, sign * cfg.dt, 3, cfg.omega)
            b = S.run(pert, tr, model, sign * cfg.dt, 3, cfg.omega)
            e = np.max(np.abs(a - b)) / np.max(np.abs(a))
            if store is None:
                assert e < 1e-13, (order, e)
            else:
                store.append(e)
    assert max(worst_b) > 1e-12
    assert max(worst_b) < 0.5 * TOL_POINTWISE_REVERSED
