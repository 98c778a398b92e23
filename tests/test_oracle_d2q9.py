"""Pins of the D2Q9 parts of the oracle: the isothermal equilibrium of Section 5.1 and the
transport of the diagonal velocities (eq. (3.7) with v = lambda (+-1, +-1))."""
import numpy as np
import pytest

from oracle import models as M
from oracle import scheme as S
from oracle.dg import CartesianMesh, assemble_transport
from oracle.transport import DirectTransport, bloch_transport, bloch_transport_2d


def _state(mesh, rng, amp=0.05, mach=0.05):
    X = mesh.coords1d(0)[None, :]
    Y = mesh.coords1d(1)[:, None]
    ph = rng.uniform(0, 2 * np.pi, 4)
    rho = 1.0 + amp * np.sin(2 * np.pi * X + ph[0]) * np.cos(2 * np.pi * Y + ph[1])
    ux = mach * np.cos(2 * np.pi * Y + ph[2]) + 0 * X
    uy = mach * np.sin(2 * np.pi * (X + Y) + ph[3])
    return np.stack([rho, rho * ux, rho * uy])


def test_lattice_weights_isotropy():
    """The D2Q9 weights: sum W_i = 1, sum W_i xi_i = 0, sum W_i xi_i xi_i^T = I/3 (so that
    c^2 = lambda^2/3), and the fourth moment sum W xi_x^2 xi_y^2 = 1/9."""
    W, X = M.D2Q9_W, M.D2Q9_XI
    assert abs(W.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(W @ X, 0.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", W, X, X), np.eye(2) / 3.0, atol=1e-16)
    assert abs(np.sum(W * X[:, 0] ** 2 * X[:, 1] ** 2) - 1.0 / 9.0) < 1e-16


@pytest.mark.parametrize("lam", [1.0, 2.5])
def test_equilibrium_moments(lam):
    """P f^eq(w) = w, and the second moment is the isothermal Euler flux of Section 5.1,
    Pi = rho c^2 I + rho u u^T (c = lambda / sqrt(3))."""
    rng = np.random.default_rng(11)
    model = M.Model(M.ISOTHERMAL_D2Q9, 2, lam)
    rho = 1.0 + 0.3 * rng.random(50)
    u = 0.2 * lam * (rng.random((2, 50)) - 0.5)
    w = np.stack([rho, rho * u[0], rho * u[1]])
    f = model.feq(w)
    assert f.shape == (1, 9, 50)
    np.testing.assert_allclose(model.moments(f), w, rtol=0, atol=1e-14)
    V = model.velocities()
    Pi = np.einsum("ia,ib,in->abn", V, V, f[0])
    c2 = lam * lam / 3.0
    for a in range(2):
        for b in range(2):
            ref = rho * c2 * (a == b) + rho * u[a] * u[b]
            np.testing.assert_allclose(Pi[a, b], ref, rtol=0, atol=1e-14 * lam * lam)
    q = model.flux(w)                                      # (D, m, n): rows of Pi as momentum fluxes
    np.testing.assert_allclose(q[0, 1], Pi[0, 0], rtol=1e-13)
    np.testing.assert_allclose(q[1, 2], Pi[1, 1], rtol=1e-13)
    np.testing.assert_allclose(q[0, 2], Pi[0, 1], rtol=0, atol=1e-14 * lam * lam)


def test_equilibrium_at_rest_is_weights():
    """u = 0: f^eq_i = W_i rho."""
    model = M.Model(M.ISOTHERMAL_D2Q9, 2, 1.0)
    w = np.array([[1.7], [0.0], [0.0]])
    np.testing.assert_allclose(model.feq(w)[0, :, 0], 1.7 * M.D2Q9_W, rtol=1e-15)


def test_split_by_axis():
    """eq. (3.7) on a Cartesian mesh: L_h(v_x, v_y) = L_h(v_x, 0) + L_h(0, v_y) for every sign
    pattern (the face upwinding of a face normal to x sees v_x only)."""
    m = CartesianMesh(2, (3, 2), 2, lengths=(0.8, 1.1))
    for sx in (1, -1):
        for sy in (1, -1):
            L = assemble_transport(m, np.array([1.3 * sx, 0.9 * sy]))
            Lx = assemble_transport(m, np.array([1.3 * sx, 0.0]))
            Ly = assemble_transport(m, np.array([0.0, 0.9 * sy]))
            assert abs(L - Lx - Ly).max() < 1e-13


@pytest.mark.parametrize("d,N", [(1, (3, 4)), (2, (4, 3)), (3, (2, 3)), (4, (2, 2))])
@pytest.mark.parametrize("theta", [0.5, 0.75, 1.0])
@pytest.mark.parametrize("nu", [1.0, 2.0, 5.0])
def test_bloch2d_equals_direct(d, N, theta, nu):
    """Sparse LU of the assembled system == the 2-D Fourier form, every diagonal velocity,
    rectangular cells."""
    rng = np.random.default_rng(d * 100 + N[0])
    m = CartesianMesh(2, N, d, lengths=(0.7, 1.2))
    lam = 1.4
    delta = nu * min(m.h) / (2 * lam)
    for sx in (1, -1):
        for sy in (1, -1):
            v = np.array([sx * lam, sy * lam])
            F = rng.standard_normal(m.shape)
            r1 = DirectTransport(m, v, delta, theta)(F)
            r2 = bloch_transport_2d(F, v, m.h, d, delta, theta)
            np.testing.assert_allclose(r1, r2, rtol=0, atol=2e-13 * np.abs(F).max())


@pytest.mark.parametrize("d", [1, 3])
def test_bloch2d_axis_velocity_is_line_form(d):
    """With one zero component the 2-D form reduces to the per-line form."""
    rng = np.random.default_rng(3)
    m = CartesianMesh(2, (5, 3), d)
    F = rng.standard_normal(m.shape)
    for a, v in ((0, (-2.0, 0.0)), (1, (0.0, 2.0))):
        nu = 2 * 2.0 * 0.02 / m.h[a]
        r1 = bloch_transport_2d(F, v, m.h, d, 0.02, 0.5)
        r2 = bloch_transport(F, m.axis_np(a), 1 if sum(v) > 0 else -1, d, nu, 0.5)
        np.testing.assert_allclose(r1, r2, atol=1e-14)


def test_zero_velocity_is_identity():
    """v = 0 (the D2Q9 rest population): L_h = 0, the transport step is the identity."""
    rng = np.random.default_rng(4)
    m = CartesianMesh(2, (3, 3), 2)
    F = rng.standard_normal(m.shape)
    np.testing.assert_allclose(bloch_transport_2d(F, (0.0, 0.0), m.h, 2, 0.3, 0.5), F, rtol=0, atol=1e-15)
    np.testing.assert_allclose(DirectTransport(m, np.zeros(2), 0.3)(F), F, rtol=0, atol=1e-15)
    model = M.Model(M.ISOTHERMAL_D2Q9, 2, 1.0)
    np.testing.assert_array_equal(S.Transporter(m, model, 0.5, "bloch").field(F, 0, 0.3), F)


@pytest.mark.parametrize("d", [1, 2, 4])
def test_diagonal_invariants(d):
    """Diagonal transport keeps constants and the weighted total, is time-symmetric
    (eq. (3.13)), and does not increase the M-norm (energy identity of Section 3.1)."""
    rng = np.random.default_rng(5 + d)
    m = CartesianMesh(2, (4, 5), d)
    v = np.array([-1.0, 1.0])
    delta = 0.6 * min(m.h)
    Mw = m.mass_weights()
    F = rng.standard_normal(m.shape)
    np.testing.assert_allclose(bloch_transport_2d(np.full(m.shape, 3.0), v, m.h, d, delta), 3.0, atol=1e-13)
    G = bloch_transport_2d(F, v, m.h, d, delta)
    assert abs(np.sum(Mw * G) - np.sum(Mw * F)) < 1e-13 * np.sum(Mw * np.abs(F))
    assert np.sum(Mw * G * G) <= np.sum(Mw * F * F) * (1 + 1e-14)
    back = bloch_transport_2d(G, v, m.h, d, -delta)
    np.testing.assert_allclose(back, F, atol=1e-12)


def _d2q9(N=(6, 6), d=2, lam=1.0):
    mesh = CartesianMesh(2, N, d)
    model = M.Model(M.ISOTHERMAL_D2Q9, 2, lam)
    return mesh, model


def test_collision_d2q9():
    """eq. (3.12) with the D2Q9 equilibrium: moments kept, C o C = I at omega = 2,
    omega = 1 gives f^eq."""
    rng = np.random.default_rng(6)
    mesh, model = _d2q9((2, 3))
    f = model.feq(_state(mesh, rng)) + 1e-3 * rng.standard_normal((1, 9) + mesh.shape)
    c2 = S.collision(f, model, 2.0)
    np.testing.assert_allclose(model.moments(c2), model.moments(f), atol=1e-14)
    np.testing.assert_allclose(S.collision(c2, model, 2.0), f, atol=1e-14)
    np.testing.assert_allclose(S.collision(f, model, 1.0), model.feq(model.moments(f)), atol=1e-15)


@pytest.mark.parametrize("scheme", ["M2", "M2_collapsed", "M2_kin"])
def test_d2q9_constant_state_and_conservation(scheme):
    """A uniform equilibrium is a fixed point of every scheme; the weighted totals of
    rho, rho u_x, rho u_y are conserved on the periodic mesh; Bloch == direct."""
    rng = np.random.default_rng(7)
    mesh, model = _d2q9((4, 4), 1)
    w_c = np.stack([np.full(mesh.shape, 1.2), np.full(mesh.shape, 0.06), np.full(mesh.shape, -0.03)])
    tr = S.Transporter(mesh, model, 0.5, "bloch")
    dt = mesh.h[0] / model.lam
    f = S.run(S.initial_state(model, w_c), tr, model, dt, 3, 2.0, scheme)
    np.testing.assert_allclose(f, S.initial_state(model, w_c), atol=1e-14)
    w0 = _state(mesh, rng)
    f1 = S.run(S.initial_state(model, w0), tr, model, dt, 4, 2.0, scheme)
    f2 = S.run(S.initial_state(model, w0), S.Transporter(mesh, model, 0.5, "direct"), model, dt, 4, 2.0, scheme)
    np.testing.assert_allclose(f1, f2, atol=1e-13)
    np.testing.assert_allclose(S.weighted_total(mesh, model.moments(f1)), S.weighted_total(mesh, w0),
                               rtol=0, atol=1e-14)


def test_d2q9_m2_second_order_in_time():
    """M2 is second order: the self-convergence ratio of w at fixed mesh is ~4."""
    rng = np.random.default_rng(8)
    mesh, model = _d2q9((6, 6), 2)
    w0 = _state(mesh, rng, amp=0.05, mach=0.05)
    tr = S.Transporter(mesh, model, 0.5, "bloch")
    T = 0.12
    sols = []
    for k in (3, 6, 12, 24):
        f = S.run(S.initial_state(model, w0), tr, model, T / k, k, 2.0, "M2")
        sols.append(model.moments(f))
    e = [np.linalg.norm(sols[i] - sols[i + 1]) for i in range(3)]
    r = [e[i] / e[i + 1] for i in range(2)]
    assert all(3.5 < x < 4.6 for x in r), r


def test_d2q9_m2_time_symmetric_positive_tau():
    """eq. (3.13) for the palindrome with tau > 0: M2(-dt) M2(dt) = I."""
    rng = np.random.default_rng(9)
    mesh, model = _d2q9((3, 3), 1)
    f = model.feq(_state(mesh, rng)) + 1e-3 * rng.standard_normal((1, 9) + mesh.shape)
    tr = S.Transporter(mesh, model, 0.5, "bloch")
    tau, dt = 0.05, 0.02
    om = lambda t: 2 * t / (2 * tau + t)
    g = S.m2_step(f, tr, model, dt, om(dt))
    back = S.m2_step(g, tr, model, -dt, om(-dt))
    np.testing.assert_allclose(back, f, atol=1e-12)


def test_d2q9_linear_acoustics_second_order():
    """Small-amplitude isothermal Euler (Section 5.1 model, tau = 0): a density wave
    rho = 1 + eps cos(2 pi x) at rest oscillates as cos(2 pi c t) with c = lambda/sqrt(3).
    M2 at CFL 1 converges to it at second order (h and dt refined together) and keeps u_y = 0."""
    eps, T = 1e-4, 0.5
    errs = []
    for N in (16, 32):
        mesh = CartesianMesh(2, (N, 1), 3)
        model = M.Model(M.ISOTHERMAL_D2Q9, 2, 1.0)
        X = mesh.coords1d(0)[None, :] + 0 * mesh.coords1d(1)[:, None]
        w0 = np.stack([1 + eps * np.cos(2 * np.pi * X), 0 * X, 0 * X])
        tr = S.Transporter(mesh, model, 0.5, "bloch")
        f = S.run(S.initial_state(model, w0), tr, model, T / (N // 2), N // 2, 2.0, "M2")
        w = model.moments(f)
        ref = 1 + eps * np.cos(2 * np.pi * X) * np.cos(2 * np.pi * model.sound_speed * T)
        errs.append(np.abs(w[0] - ref).max() / eps)
        assert np.abs(w[2]).max() < 1e-14
    assert errs[0] < 0.02 and errs[0] / errs[1] > 3.5, errs
