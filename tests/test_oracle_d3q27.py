"""Pins of the D3Q15 / D3Q27 parts of the oracle: lattices, equilibrium moments, and the
transport of the corner velocities lambda (+-1, +-1, +-1) (eq. (3.7)), whose operator acts
along all three axes (the 3-D Fourier form of oracle.transport.bloch_transport_3d)."""
import numpy as np
import pytest

from oracle import models as M
from oracle import scheme as S
from oracle.dg import CartesianMesh
from oracle.transport import DirectTransport, bloch_transport_3d, bloch_transport_planes

LATTICES = [(M.ISOTHERMAL_D3Q15, 15), (M.ISOTHERMAL_D3Q27, 27)]


@pytest.mark.parametrize("kind,q", LATTICES)
def test_lattice(kind, q):
    """sum W = 1, sum W xi = 0, sum W xi xi^T = I/3, fourth moments 1/3 (aaaa) and 1/9
    (aabb), odd third moments zero; the velocity order of the model doc."""
    X, W = M.LATTICES[kind]
    assert X.shape == (q, 3)
    assert len({tuple(r) for r in X}) == q
    assert abs(W.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(W @ X, 0.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", W, X, X), np.eye(3) / 3.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib,ic->abc", W, X, X, X), 0.0, atol=1e-16)
    for a in range(3):
        assert abs(np.sum(W * X[:, a] ** 4) - 1 / 3) < 1e-15
        for b in range(3):
            if a != b:
                assert abs(np.sum(W * X[:, a] ** 2 * X[:, b] ** 2) - 1 / 9) < 1e-15
    np.testing.assert_array_equal(X[:7], M.D3Q19_XI[:7])
    np.testing.assert_array_equal(X[q - 8], [1, 1, 1])
    np.testing.assert_array_equal(X[q - 6], [-1, -1, 1])
    np.testing.assert_array_equal(X[q - 1], [1, -1, -1])
    if q == 27:
        np.testing.assert_array_equal(X[7:19], M.D3Q19_XI[7:])


@pytest.mark.parametrize("kind,q", LATTICES)
@pytest.mark.parametrize("lam", [1.0, 3.0])
def test_equilibrium_moments(kind, q, lam):
    rng = np.random.default_rng(5)
    model = M.Model(kind, 3, lam)
    assert model.nv == q and model.m == 4
    rho = 1.0 + 0.3 * rng.random(40)
    u = 0.2 * lam * (rng.random((3, 40)) - 0.5)
    w = np.concatenate([rho[None], rho[None] * u])
    f = model.feq(w)
    np.testing.assert_allclose(model.moments(f), w, rtol=0, atol=1e-14)
    V = model.velocities()
    Pi = np.einsum("ia,ib,in->abn", V, V, f[0])
    c2 = lam * lam / 3.0
    for a in range(3):
        for b in range(3):
            np.testing.assert_allclose(Pi[a, b], rho * c2 * (a == b) + rho * u[a] * u[b], rtol=0,
                                       atol=1e-14 * lam * lam)


@pytest.mark.parametrize("d", [1, 2])
def test_corner_transport_fourier_equals_direct(d):
    """Sparse LU of the assembled 3-D system == the 3-D Fourier form, for every corner
    velocity, rectangular cells, theta = 1/2 and 0.8."""
    rng = np.random.default_rng(10 + d)
    m = CartesianMesh(3, (3, 2, 4), d, lengths=(0.8, 1.1, 1.3))
    lam = 1.2
    for theta in (0.5, 0.8):
        delta = 0.7 * min(m.h) / lam
        for v in M.D3Q15_XI[7:]:
            F = rng.standard_normal(m.shape)
            r1 = DirectTransport(m, lam * v, delta, theta)(F)
            r2 = bloch_transport_3d(F, lam * v, m.h, d, delta, theta)
            np.testing.assert_allclose(r1, r2, rtol=0, atol=2e-13 * np.abs(F).max())


def test_fourier_3d_reduces_to_planes_and_identity():
    """With a zero component the 3-D form is the plane-wise form of the D3Q19 edges; with
    v = 0 it is the identity."""
    rng = np.random.default_rng(3)
    m = CartesianMesh(3, (2, 3, 2), 2, lengths=(1.0, 0.9, 1.2))
    delta = 0.5 * min(m.h)
    for v in M.D3Q19_XI[7:]:
        F = rng.standard_normal(m.shape)
        np.testing.assert_allclose(bloch_transport_3d(F, v, m.h, 2, delta),
                                   bloch_transport_planes(F, v, m.h, 2, delta), rtol=0, atol=1e-13)
    F = rng.standard_normal(m.shape)
    np.testing.assert_allclose(bloch_transport_3d(F, np.zeros(3), m.h, 2, delta), F, rtol=0, atol=1e-15)


def test_corner_transport_translates_a_constant_and_dissipates():
    """L_h 1 = 0 (a constant is kept) and the theta = 1/2 step does not increase the
    GL-weighted L2 norm (the upwind energy identity, Section 3.1)."""
    rng = np.random.default_rng(7)
    m = CartesianMesh(3, (3, 3, 2), 2)
    delta = min(m.h)
    one = np.ones(m.shape)
    np.testing.assert_allclose(bloch_transport_3d(one, (1, -1, 1), m.h, 2, delta), one, atol=1e-14)
    Wm = m.mass_weights()
    for v in M.D3Q15_XI[7:]:
        F = rng.standard_normal(m.shape)
        G = bloch_transport_3d(F, v, m.h, 2, delta)
        assert np.sum(Wm * G * G) <= np.sum(Wm * F * F) * (1 + 1e-14)


def _state(mesh):
    X = mesh.coords1d(0)[None, None, :]
    Y = mesh.coords1d(1)[None, :, None]
    Z = mesh.coords1d(2)[:, None, None]
    rho = 1.0 + 0.04 * np.sin(2 * np.pi * (X + Z)) + 0 * Y
    u = [0.03 * np.cos(2 * np.pi * Y) + 0 * X + 0 * Z, 0.02 * np.sin(2 * np.pi * Z) + 0 * X + 0 * Y,
         0.01 + 0 * X + 0 * Y + 0 * Z]
    return np.stack([rho] + [rho * ua for ua in u])


@pytest.mark.parametrize("kind,q", LATTICES)
@pytest.mark.parametrize("scheme", ["M2", "M2_collapsed"])
def test_constant_state_and_conservation(kind, q, scheme):
    mesh = CartesianMesh(3, (2, 3, 2), 1)
    model = M.Model(kind, 3, 1.0)
    tr = S.Transporter(mesh, model, 0.5, "bloch")
    dt = min(mesh.h) / model.lam
    wc = np.stack([np.full(mesh.shape, v) for v in (1.1, 0.02, -0.01, 0.03)])
    f = S.run(S.initial_state(model, wc), tr, model, dt, 2, 2.0, scheme)
    np.testing.assert_allclose(f, S.initial_state(model, wc), atol=1e-14)
    w0 = _state(mesh)
    f1 = S.run(S.initial_state(model, w0), tr, model, dt, 2, 2.0, scheme)
    np.testing.assert_allclose(S.weighted_total(mesh, model.moments(f1)), S.weighted_total(mesh, w0),
                               rtol=0, atol=1e-14)


@pytest.mark.parametrize("kind,q", LATTICES)
def test_linear_acoustics_along_the_diagonal(kind, q):
    """A density wave rho = 1 + eps cos(2 pi (x + y + z)) at rest has |k| = 2 pi sqrt(3) and
    oscillates as cos(2 pi sqrt(3) c t), c = lambda/sqrt(3); M2 at CFL 1 converges to it at
    second order (h and dt refined together).  Every corner velocity carries it."""
    eps, T = 1e-4, 0.25
    errs = []
    for N in (4, 8):
        mesh = CartesianMesh(3, (N, N, N), 2)
        model = M.Model(kind, 3, 1.0)
        X = mesh.coords1d(0)[None, None, :]
        Y = mesh.coords1d(1)[None, :, None]
        Z = mesh.coords1d(2)[:, None, None]
        phase = np.cos(2 * np.pi * (X + Y + Z))
        w0 = np.stack([1 + eps * phase, 0 * phase, 0 * phase, 0 * phase])
        tr = S.Transporter(mesh, model, 0.5, "bloch")
        nsteps = N // 2
        f = S.run(S.initial_state(model, w0), tr, model, T / nsteps, nsteps, 2.0, "M2")
        w = model.moments(f)
        ref = 1 + eps * phase * np.cos(2 * np.pi * np.sqrt(3.0) * model.sound_speed * T)
        errs.append(np.abs(w[0] - ref).max() / eps)
    assert errs[0] < 0.25 and errs[0] / errs[1] > 3.5, errs
