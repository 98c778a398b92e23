"""Pins of the D3Q19 parts of the oracle: lattice, equilibrium moments, and the transport of
the edge velocities lambda (+-e_a +- e_b) (eq. (3.7)), which act in planes."""
import numpy as np
import pytest

from oracle import models as M
from oracle import scheme as S
from oracle.dg import CartesianMesh
from oracle.transport import DirectTransport, bloch_transport_planes


def test_lattice():
    """sum W = 1, sum W xi = 0, sum W xi xi^T = I/3, fourth moments 1/3 (aaaa), 1/9 (aabb);
    the velocity order of the model doc."""
    W, X = M.D3Q19_W, M.D3Q19_XI
    assert X.shape == (19, 3)
    assert abs(W.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(W @ X, 0.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", W, X, X), np.eye(3) / 3.0, atol=1e-16)
    for a in range(3):
        assert abs(np.sum(W * X[:, a] ** 4) - 1 / 3) < 1e-15
        for b in range(3):
            if a != b:
                assert abs(np.sum(W * X[:, a] ** 2 * X[:, b] ** 2) - 1 / 9) < 1e-15
    np.testing.assert_array_equal(X[7], [1, 1, 0])
    np.testing.assert_array_equal(X[12], [-1, 0, 1])
    np.testing.assert_array_equal(X[18], [0, 1, -1])


@pytest.mark.parametrize("lam", [1.0, 3.0])
def test_equilibrium_moments(lam):
    rng = np.random.default_rng(2)
    model = M.Model(M.ISOTHERMAL_D3Q19, 3, lam)
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
def test_edge_transport_plane_form_equals_direct(d):
    """Sparse LU of the assembled 3-D system == the plane-wise 2-D Fourier form, for every
    edge velocity, rectangular cells, theta = 1/2 and 0.8."""
    rng = np.random.default_rng(d)
    m = CartesianMesh(3, (3, 2, 4), d, lengths=(0.8, 1.1, 1.3))
    lam = 1.2
    for theta in (0.5, 0.8):
        delta = 0.7 * min(m.h) / lam
        for v in M.D3Q19_XI[7:]:
            F = rng.standard_normal(m.shape)
            r1 = DirectTransport(m, lam * v, delta, theta)(F)
            r2 = bloch_transport_planes(F, lam * v, m.h, d, delta, theta)
            np.testing.assert_allclose(r1, r2, rtol=0, atol=2e-13 * np.abs(F).max())


def _state(mesh, rng):
    X = mesh.coords1d(0)[None, None, :]
    Y = mesh.coords1d(1)[None, :, None]
    Z = mesh.coords1d(2)[:, None, None]
    rho = 1.0 + 0.04 * np.sin(2 * np.pi * (X + Z)) + 0 * Y
    u = [0.03 * np.cos(2 * np.pi * Y) + 0 * X + 0 * Z, 0.02 * np.sin(2 * np.pi * Z) + 0 * X + 0 * Y,
         0.01 + 0 * X + 0 * Y + 0 * Z]
    return np.stack([rho] + [rho * ua for ua in u])


@pytest.mark.parametrize("scheme", ["M2", "M2_collapsed"])
def test_constant_state_and_conservation(scheme):
    rng = np.random.default_rng(4)
    mesh = CartesianMesh(3, (2, 3, 2), 1)
    model = M.Model(M.ISOTHERMAL_D3Q19, 3, 1.0)
    tr = S.Transporter(mesh, model, 0.5, "bloch")
    dt = min(mesh.h) / model.lam
    wc = np.stack([np.full(mesh.shape, v) for v in (1.1, 0.02, -0.01, 0.03)])
    f = S.run(S.initial_state(model, wc), tr, model, dt, 2, 2.0, scheme)
    np.testing.assert_allclose(f, S.initial_state(model, wc), atol=1e-14)
    w0 = _state(mesh, rng)
    f1 = S.run(S.initial_state(model, w0), tr, model, dt, 2, 2.0, scheme)
    np.testing.assert_allclose(S.weighted_total(mesh, model.moments(f1)), S.weighted_total(mesh, w0),
                               rtol=0, atol=1e-14)


def test_linear_acoustics_along_z():
    """A density wave along z at rest oscillates as cos(2 pi c t), c = lambda/sqrt(3); M2 at
    CFL 1 converges to it at second order (h and dt refined together)."""
    eps, T = 1e-4, 0.5
    errs = []
    for N in (8, 16):
        mesh = CartesianMesh(3, (1, 1, N), 3)
        model = M.Model(M.ISOTHERMAL_D3Q19, 3, 1.0)
        Z = mesh.coords1d(2)[:, None, None] + np.zeros(mesh.shape)
        w0 = np.stack([1 + eps * np.cos(2 * np.pi * Z), 0 * Z, 0 * Z, 0 * Z])
        tr = S.Transporter(mesh, model, 0.5, "bloch")
        f = S.run(S.initial_state(model, w0), tr, model, T / (N // 2), N // 2, 2.0, "M2")
        w = model.moments(f)
        ref = 1 + eps * np.cos(2 * np.pi * Z) * np.cos(2 * np.pi * model.sound_speed * T)
        errs.append(np.abs(w[0] - ref).max() / eps)
        assert np.abs(w[1:3]).max() < 1e-14
    assert errs[0] < 0.06 and errs[0] / errs[1] > 3.5, errs
