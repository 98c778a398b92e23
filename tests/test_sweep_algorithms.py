"""CPU checks of the three sweep algorithms the transport kernels implement (not the kernels).

Each test restates one algorithm in plain numpy, cell by cell, and compares it with the
theta step solved as the linear system it is: the sparse LU of the eq. (3.7) matrix
(oracle.transport.DirectTransport), which knows nothing of lines, segments, tiles or
truncated starts.  The algorithms (Section 4.1 replaced by exact closures):

* line sweep, axis-aligned velocities: per-cell update fn_c = E f_c + q (x_{c-1} + zb u_{c-1}),
  the scalar recurrence of the last node, segment aggregates closed around the periodic ring
  exactly (full mode) or through a window of W cells with |beta|^W <= 2^-60 (window mode),
  and the composed double step with its 2 x 2 recurrence;
* tile sweep, diagonal velocities of D2Q9: fn_c = B^-1 r_c - c1 f_c with the two upwind faces,
  every tile swept from W cells upwind, starting from the old face values;
* box sweep, corner velocities of D3Q15 / D3Q27: the same with three upwind faces.

The widths used are those of the signed lattice-path bound for these Courant numbers; a
much smaller width is shown to miss, so the check does see the truncation.  The last tests
take the cell inverse and the widths from the library's host planner (pdg_plan_sweep, no GPU)
and run them through the same algorithm.
"""
import os

import numpy as np
import pytest

from oracle.dg import CartesianMesh
from oracle.transport import DirectTransport, line_K


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


# ----------------------------------------------------------------------------------------
# line sweep (axis-aligned velocity +lambda e_x on a periodic 1-D mesh)

def _line_coefs(d, nu, theta):
    """E, q, beta, zb of the per-cell update, from the reduced cell operator
    d/dt f_c = -(2 lambda/h)(K f_c - w0^-1 e0 f_{c-1,d}) and the theta step."""
    K, w = line_K(d)
    n = d + 1
    I = np.eye(n)
    B = I + theta * nu * K
    E = np.linalg.solve(B, I - (1.0 - theta) * nu * K)
    e0 = np.zeros(n)
    e0[0] = 1.0
    q = np.linalg.solve(B, theta * nu / w[0] * e0)
    return E, q, q[n - 1], (1.0 - theta) / theta


def _line_sweep(f, d, nu, theta, nseg, window):
    """One theta sub-step of a periodic line of N cells (f: (N, n)), split into nseg segments.
    window=None: every segment aggregates its whole length and the ring is closed exactly;
    window=W: the inflow of a segment is the recurrence over the W cells before it."""
    E, q, beta, zb = _line_coefs(d, nu, theta)
    N, n = f.shape
    a = f @ E.T                                        # E f_c
    u_prev = np.roll(f[:, n - 1], 1)                   # old last node of the upwind cell
    alpha = a[:, n - 1] + beta * zb * u_prev           # x_c = alpha_c + beta x_{c-1}
    bounds = np.linspace(0, N, nseg + 1).astype(int)
    starts, ends = bounds[:-1], bounds[1:]
    x_in = np.zeros(nseg)                              # x_{s0-1} for each segment
    if window is None:
        Y = np.array([sum(beta ** (e - 1 - c) * alpha[c] for c in range(s, e)) for s, e in zip(starts, ends)])
        P = np.array([beta ** (e - s) for s, e in zip(starts, ends)])
        for s in range(nseg):
            # end value of segment s-1: sum_j (prod of the later segments' beta powers) Y, / (1 - beta^N)
            acc, gain = 0.0, 1.0
            for j in range(nseg):
                t = (s - 1 - j) % nseg
                acc += gain * Y[t]
                gain *= P[t]
            x_in[s] = acc / (1.0 - beta ** N)
    else:
        for s in range(nseg):
            x_in[s] = sum(beta ** k * alpha[(starts[s] - 1 - k) % N] for k in range(window))
    out = np.empty_like(f)
    for s in range(nseg):
        x = x_in[s]
        for c in range(starts[s], ends[s]):
            out[c] = a[c] + q * (x + zb * u_prev[c])
            x = out[c, n - 1]
    return out


def _line_composed(f, d, nu, theta, window):
    """Two consecutive sub-steps as one sweep: gn_c = E^2 f_c + (E q) z_c + q z'_c with
    z_c = x_{c-1} + zb u_{c-1}, z'_c = y_{c-1} + zb x_{c-1}; the last nodes X_c = (x_c, y_c)
    obey X_c = A_c + M X_{c-1}, M = [[beta, 0], [g1 + beta zb, beta]], g1 = (E q)[d],
    started `window` cells upwind."""
    E, q, beta, zb = _line_coefs(d, nu, theta)
    N, n = f.shape
    Eq = E @ q
    M = np.array([[beta, 0.0], [Eq[n - 1] + beta * zb, beta]])
    a1 = f @ E.T
    a2 = f @ (E @ E).T
    u_prev = np.roll(f[:, n - 1], 1)
    A = np.stack([a1[:, n - 1] + beta * zb * u_prev, a2[:, n - 1] + Eq[n - 1] * zb * u_prev], axis=1)
    out = np.empty_like(f)
    for c in range(N):
        X = np.zeros(2)                                # X_{c-1} from the window
        for k in range(window, 0, -1):
            X = A[(c - k) % N] + M @ X
        # X_{c-1} = (x_{c-1}, y_{c-1})
        z = X[0] + zb * u_prev[c]
        zp = X[1] + zb * X[0]
        out[c] = a2[c] + Eq * z + q * zp
    return out


def _window(beta, tol=2.0 ** -60):
    W = 1
    while abs(beta) ** W > tol:
        W += 1
    return W


@pytest.mark.parametrize("d", [1, 2, 3, 4])
@pytest.mark.parametrize("nu,theta", [(1.0, 0.5), (2.0, 0.5), (1.5, 0.75)])
def test_line_segments_full_ring_and_window_equal_the_lu_solve(d, nu, theta):
    N = 11
    n = d + 1
    mesh = CartesianMesh(1, (N,), d)
    lam = 1.0
    delta = nu * mesh.h[0] / (2.0 * lam)
    f = np.random.default_rng(100 * d + int(4 * nu)).standard_normal(N * n)
    ref = DirectTransport(mesh, np.array([lam]), delta, theta)(f)
    _, _, beta, _ = _line_coefs(d, nu, theta)
    for nseg in (1, 3, 4):
        full = _line_sweep(f.reshape(N, n), d, nu, theta, nseg, None).reshape(-1)
        assert _rel(full, ref) < 1e-14
        win = _line_sweep(f.reshape(N, n), d, nu, theta, nseg, _window(beta)).reshape(-1)
        assert _rel(win, ref) < 1e-14
    if abs(beta) > 1e-3:                               # a one-cell window misses
        assert _rel(_line_sweep(f.reshape(N, n), d, nu, theta, 3, 1).reshape(-1), ref) > 1e-6


@pytest.mark.parametrize("d", [1, 3])
@pytest.mark.parametrize("nu,theta", [(1.0, 0.5), (2.0, 0.5)])
def test_line_composed_double_step_equals_two_lu_solves(d, nu, theta):
    N = 9
    n = d + 1
    mesh = CartesianMesh(1, (N,), d)
    delta = nu * mesh.h[0] / 2.0
    T = DirectTransport(mesh, np.array([1.0]), delta, theta)
    f = np.random.default_rng(7 + d).standard_normal(N * n)
    ref = T(T(f))
    _, _, beta, _ = _line_coefs(d, nu, theta)
    W2 = _window(beta, 2.0 ** -62) + 8                 # the 2 x 2 recurrence decays like k beta^k
    got = _line_composed(f.reshape(N, n), d, nu, theta, W2).reshape(-1)
    assert _rel(got, ref) < 1e-14


# ----------------------------------------------------------------------------------------
# tile sweep (diagonal velocity of D2Q9) and box sweep (corner velocity of D3Q15 / D3Q27)

def _cell_operator(d, nus, theta):
    """B^-1 and k_a = nu_a / w0 of the cell system B = I + theta sum_a nu_a K_a, nodes
    numbered with x fastest (p = (i_z n + i_y) n + i_x); axis a of the cell is numpy axis -1-a."""
    K, w = line_K(d)
    n = d + 1
    D = len(nus)
    Ksum = np.zeros((n ** D, n ** D))
    for a in range(D):
        factors = [np.eye(n)] * D
        factors[D - 1 - a] = K                         # kron order: slowest axis first
        op = factors[0]
        for fct in factors[1:]:
            op = np.kron(op, fct)
        Ksum += nus[a] * op
    Binv = np.linalg.inv(np.eye(n ** D) + theta * Ksum)
    return Binv, [nu / w[0] for nu in nus]


def _truncated_sweep(F, d, nus, theta, signs, tile, W):
    """Every tile (box) of `tile` output cells is swept in upwind-to-downwind order over the
    region that starts W[a] cells upwind along axis a (W: one int for all axes, or a list).  A cell takes r = f/theta + sum_a k_a
    S_a (face value of its upwind neighbour along a), forms fn = B^-1 r - c1 f and passes the
    face value theta B^-1 r on.  At the start of the region the face values come from the old
    state (theta fn + (1-theta) f with fn = f there)."""
    D = len(nus)
    n = d + 1
    W = [W] * D if np.isscalar(W) else list(W)
    Binv, k = _cell_operator(d, nus, theta)
    c1 = (1.0 - theta) / theta
    G = F.copy()
    for a in range(D):                                 # traversal orientation: all signs positive
        if signs[a] < 0:
            G = np.flip(G, axis=D - 1 - a)
    ncell = [G.shape[D - 1 - a] // n for a in range(D)]
    out = np.full_like(G, np.nan)

    def cell(idx):                                     # idx[a] = cell index along axis a
        sl = tuple(slice((idx[a] % ncell[a]) * n, (idx[a] % ncell[a]) * n + n) for a in reversed(range(D)))
        return sl

    def face(vals, a):                                 # the +a face nodes of a cell array
        sl = [slice(None)] * D
        sl[D - 1 - a] = n - 1
        return vals[tuple(sl)]

    def inject(r, a, vals):                            # add to the -a face nodes
        sl = [slice(None)] * D
        sl[D - 1 - a] = 0
        r[tuple(sl)] += vals

    for t0 in np.ndindex(*[-(-ncell[a] // tile[a]) for a in range(D)]):
        lo = [t0[a] * tile[a] for a in range(D)]
        hi = [min(lo[a] + tile[a], ncell[a]) for a in range(D)]
        faces = {}                                     # (cell, axis) -> new +axis face value
        for rel in np.ndindex(*[hi[a] - lo[a] + W[a] for a in reversed(range(D))]):
            idx = [lo[a] - W[a] + rel[D - 1 - a] for a in range(D)]
            f = G[cell(idx)]
            r = f / theta
            for a in range(D):
                up = list(idx)
                up[a] -= 1
                fv = faces.get((tuple(up), a))
                if fv is None:                         # region start: old face value
                    fv = face(G[cell(up)], a)
                inject(r, a, k[a] * fv)
            y = (Binv @ r.reshape(-1)).reshape(r.shape)
            for a in range(D):
                faces[(tuple(idx), a)] = theta * face(y, a)
            if all(idx[a] >= lo[a] for a in range(D)):
                out[cell(idx)] = y - c1 * f
    for a in range(D):
        if signs[a] < 0:
            out = np.flip(out, axis=D - 1 - a)
    return out


def _lu_reference(dim, ncells, d, v, nus, theta):
    lam = 1.0
    h = tuple(2.0 * abs(v[a]) * lam * 0.5 / nus[a] for a in range(dim))   # delta = 1/2
    mesh = CartesianMesh(dim, ncells, d, lengths=tuple(ncells[a] * h[a] for a in range(dim)))
    return mesh, DirectTransport(mesh, lam * np.asarray(v, dtype=np.float64), 0.5, theta)


@pytest.mark.parametrize("d,signs,nus,tile", [(1, (1, 1), (1.0, 1.0), (2, 3)), (3, (-1, 1), (1.0, 0.8), (3, 2)),
                                              (2, (-1, -1), (0.6, 1.0), (4, 5)), (3, (1, -1), (1.0, 1.0), (1, 1))])
def test_diagonal_tile_sweep_truncated_start_equals_the_lu_solve(d, signs, nus, tile):
    ncells = (4, 5)
    mesh, T = _lu_reference(2, ncells, d, signs, nus, 0.5)
    F = np.random.default_rng(sum(ncells) + d).standard_normal(mesh.shape)
    ref = T(F)
    got = _truncated_sweep(F, d, nus, 0.5, signs, tile, 17)      # widths 13-17 at nu <= 1
    assert _rel(got, ref) < 1e-14
    assert _rel(_truncated_sweep(F, d, nus, 0.5, signs, tile, 2), ref) > 1e-6


@pytest.mark.parametrize("d,signs,nus,tile,W", [(1, (1, 1, 1), (1.0, 1.0, 1.0), (2, 3, 2), 17),
                                                (2, (-1, 1, -1), (1.0, 1.0, 1.0), (3, 3, 3), 16),
                                                (1, (1, -1, -1), (0.7, 1.0, 0.9), (1, 2, 3), 17)])
def test_corner_box_sweep_truncated_start_equals_the_lu_solve(d, signs, nus, tile, W):
    ncells = (3, 3, 3)
    mesh, T = _lu_reference(3, ncells, d, signs, nus, 0.5)
    F = np.random.default_rng(3 + d).standard_normal(mesh.shape)
    ref = T(F)
    got = _truncated_sweep(F, d, nus, 0.5, signs, tile, W)
    assert _rel(got, ref) < 1e-14
    assert _rel(_truncated_sweep(F, d, nus, 0.5, signs, tile, 2), ref) > 1e-6


# ----------------------------------------------------------------------------------------
# the library's host planner (pdg_plan_sweep; host code, no GPU): its cell inverse and its
# widths, run through the algorithm above

@pytest.fixture(scope="module")
def pdg():
    from paper_1702_00169_gb300 import build as B
    if not os.path.exists(B.LIB):
        B.build()
    from paper_1702_00169_gb300 import pdg as P
    return P


@pytest.mark.parametrize("d,nus,theta", [(1, (1.0, 0.8), 0.5), (2, (0.6, 1.0), 0.75), (3, (2.0, 2.0), 0.5),
                                         (4, (1.0, 1.0), 1.0), (1, (1.0, 0.7, 0.9), 0.5),
                                         (2, (1.0, 1.0, 1.0), 0.75), (3, (0.5, 1.0, 2.0), 0.5)])
def test_planner_cell_inverse(pdg, d, nus, theta):
    """B^-1 of the planner = numpy's inverse of I + theta sum_a nu_a K_a (K from the oracle)."""
    _, binv = pdg.plan_sweep(d, nus, theta)
    ref, _ = _cell_operator(d, nus, theta)
    assert np.max(np.abs(binv - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("d,signs,nus,theta,tile", [
    (1, (1, -1), (1.0, 0.8), 0.5, (2, 3)), (2, (-1, -1), (2.0, 2.0), 0.5, (3, 4)),
    (3, (1, 1), (1.0, 1.0), 0.75, (2, 2)), (4, (-1, 1), (0.6, 1.0), 1.0, (4, 5)),
    (1, (1, -1, 1), (1.0, 0.7, 0.9), 0.5, (3, 1, 2)), (2, (-1, -1, -1), (1.0, 1.0, 1.0), 0.75, (3, 3, 3)),
    (1, (1, 1, -1), (2.0, 2.0, 2.0), 0.5, (3, 3, 3))])
def test_planner_widths_make_the_truncated_sweep_exact(pdg, d, signs, nus, theta, tile):
    """The widths of the library's planner, used by the tile / box sweep above, reproduce the
    LU solve to rounding; a third of them does not."""
    widths, _ = pdg.plan_sweep(d, nus, theta)
    D = len(nus)
    ncells = (4, 5) if D == 2 else (3, 3, 3)
    mesh, T = _lu_reference(D, ncells, d, signs, nus, theta)
    F = np.random.default_rng(11 * d + D).standard_normal(mesh.shape)
    ref = T(F)
    assert _rel(_truncated_sweep(F, d, nus, theta, signs, tile, widths), ref) < 1e-14
    assert _rel(_truncated_sweep(F, d, nus, theta, signs, tile, [w // 3 for w in widths]), ref) > 1e-12


def test_planner_widths_follow_a_permutation_of_the_axes(pdg):
    """The cell problem is symmetric under a permutation of the axes (with its Courant
    numbers), so the widths are permuted with them: boxes for all six permutations, tiles
    for the swap."""
    import itertools
    for d in (1, 2):
        for nus in ((1.0, 0.7, 0.9), (0.5, 1.0, 2.0)):
            base = pdg.plan_sweep(d, list(nus))[0]
            assert len(set(base)) > 1
            for perm in itertools.permutations(range(3)):
                assert pdg.plan_sweep(d, [nus[p] for p in perm])[0] == [base[p] for p in perm]
    for d in (1, 2, 3, 4):
        for nus in ((1.0, 0.6), (2.0, 1.3)):
            a = pdg.plan_sweep(d, list(nus))[0]
            assert a != a[::-1] and pdg.plan_sweep(d, list(nus[::-1]))[0] == a[::-1]


def test_planner_widths_and_refusals(pdg):
    """Box widths at equal Courant numbers 1 and 2 (theta = 1/2), tile widths in 12..17 at
    nu <= 1; refusals: boxes at nu = 4 (no width <= 64), degree and argument ranges."""
    assert [pdg.plan_sweep(d, [1.0] * 3)[0][0] for d in (1, 2, 3)] == [17, 16, 16]
    assert [pdg.plan_sweep(d, [2.0] * 3)[0][0] for d in (1, 2, 3)] == [27, 25, 24]
    for d in (1, 2, 3, 4):
        for nus in ((1.0, 1.0), (1.0, 0.8), (0.6, 1.0)):
            assert all(12 <= w <= 17 for w in pdg.plan_sweep(d, nus)[0])
    for args, status in [((1, [4.0] * 3), pdg.PDG_ERR_UNSUPPORTED), ((4, [1.0] * 3), pdg.PDG_ERR_ARG),
                         ((0, [1.0, 1.0]), pdg.PDG_ERR_ARG), ((5, [1.0, 1.0]), pdg.PDG_ERR_ARG),
                         ((1, [1.0, 0.0]), pdg.PDG_ERR_ARG), ((1, [1.0]), pdg.PDG_ERR_ARG),
                         ((1, [1.0, -1.0]), pdg.PDG_ERR_ARG)]:
        with pytest.raises(pdg.PdgError) as e:
            pdg.plan_sweep(*args)
        assert e.value.status == status
    with pytest.raises(pdg.PdgError) as e:
        pdg.plan_sweep(1, [1.0, 1.0], theta=0.0)
    assert e.value.status == pdg.PDG_ERR_ARG


@pytest.mark.parametrize("d", [1, 2, 3, 4])
@pytest.mark.parametrize("nu,theta", [(1.0, 0.5), (2.0, 0.5), (1.5, 0.75), (1.0, 1.0), (-0.7, 0.5), (0.4, 0.0)])
def test_planner_line_plan(pdg, d, nu, theta):
    """E, q, beta, za, zb and gamma1 of the library's line plan = the numpy derivation; the
    windows are the smallest that meet their 2^-60 rules."""
    r = pdg.plan_line(d, nu, theta)
    n = d + 1
    K, w = line_K(d)
    if theta > 0:
        E, q, beta, zb = _line_coefs(d, nu, theta)
        za = 1.0
    else:                                              # explicit step: inflow from the old value only
        E, q = np.eye(n) - nu * K, np.eye(n)[0] * nu / w[0]
        beta, za, zb = 0.0, 0.0, 1.0
    # backward steps (nu < 0) make B ill-conditioned: both sides round differently there
    atol = (1e-14 if nu > 0 else 1e-12) * max(1.0, np.max(np.abs(E)))
    np.testing.assert_allclose(r["E"], E, rtol=0, atol=atol)
    np.testing.assert_allclose(r["q"], q, rtol=0, atol=atol)
    assert abs(r["beta"] - beta) <= atol
    assert (r["za"], r["zb"]) == (za, pytest.approx(zb, rel=1e-15))
    g1 = (E @ q)[n - 1] * za + q[n - 1] * zb
    assert abs(r["gamma1"] - g1) <= 10 * atol * max(1.0, abs(g1))
    tol = 2.0 ** -60
    rr = abs(1.0 / beta) if abs(beta) > 1.0 else abs(beta)
    W = r["W"]
    assert rr ** W <= tol and (W == 1 or rr ** (W - 1) > tol)

    def ok2(k):
        return abs(beta) ** k <= tol and k * abs(g1) * abs(beta) ** (k - 1) <= tol
    if abs(beta) >= 1.0:
        assert r["W2"] == 0
    elif beta == 0.0:
        assert r["W2"] in (1, 2)
    else:
        assert ok2(r["W2"]) and not ok2(r["W2"] - 1)


@pytest.mark.parametrize("d", [1, 3, 4])
@pytest.mark.parametrize("nu,theta", [(1.0, 0.5), (2.0, 0.5), (1.0, 1.0)])
def test_planner_line_windows_make_the_sweep_exact(pdg, d, nu, theta):
    """The library's windows W (single step, 3 segments) and W2 (composed double step), used
    by the line algorithms above, reproduce the LU solves to rounding."""
    N = 9
    n = d + 1
    mesh = CartesianMesh(1, (N,), d)
    T = DirectTransport(mesh, np.array([1.0]), nu * mesh.h[0] / 2.0, theta)
    f = np.random.default_rng(31 + d).standard_normal(N * n)
    r = pdg.plan_line(d, nu, theta)
    one = _line_sweep(f.reshape(N, n), d, nu, theta, 3, r["W"]).reshape(-1)
    assert _rel(one, T(f)) < 1e-14
    two = _line_composed(f.reshape(N, n), d, nu, theta, r["W2"]).reshape(-1)
    assert _rel(two, T(T(f))) < 1e-14


# ----------------------------------------------------------------------------------------
# hyperplane sweep of the corner velocities (the organisation of the default corner kernel):
# the whole mesh plus one truncated start per axis, swept cell hyperplane by cell hyperplane
# (column + row + layer = s); each hyperplane's cells, enumerated layer by layer and row
# inside a layer, are cut into G ranges of equal work (n^3 node dot products per output
# cell, the face nodes per start cell), each range processed in batches; the faces a cell
# passes on go to a slot [parity][face][layer][row] of the receiving cell.  The integer
# arithmetic below is the kernel's (per-layer prefix tables, first cell of a work offset,
# slot indices); the values are checked against the LU solve, and the bookkeeping by
# assertions: every cell once per step, every slot written once per step and read one
# step after it was written.

def _hp_rows(s, k, RX, RY):
    rlo, rhi = max(0, s - k - (RX - 1)), min(RY - 1, s - k)
    return max(0, rhi - rlo + 1), rlo, rhi


def _hp_out_rows(s, k, rlo, rhi, w):
    if k < w[2]:
        return 0, 0
    olo, ohi = max(rlo, w[1]), min(rhi, s - k - w[0])
    return max(0, ohi - olo + 1), olo


def _hyperplane_sweep(F, d, nus, theta, signs, W, G, nb):
    n = d + 1
    NF, NN = n * n, n ** 3
    NFF = NN - (n - 1) ** 3
    Binv, k = _cell_operator(d, nus, theta)
    c1 = (1.0 - theta) / theta
    Gs = F.copy()
    for a in range(3):
        if signs[a] < 0:
            Gs = np.flip(Gs, axis=2 - a)
    nc = [Gs.shape[2 - a] // n for a in range(3)]
    w = list(W)
    RX, RY, RZ = nc[0] + w[0], nc[1] + w[1], nc[2] + w[2]
    fnode = [q for q in range(NN) if q % n == n - 1 or (q // n) % n == n - 1 or q // NF == n - 1]
    assert len(fnode) == NFF
    out = np.full_like(Gs, np.nan)
    slots = np.full((2, 3, RZ, RY, NF), np.nan)
    written = np.full((2, 3, RZ, RY), -10, dtype=np.int64)

    def cell(j, r, kk):
        cx, cy, cz = (j - w[0]) % nc[0], (r - w[1]) % nc[1], (kk - w[2]) % nc[2]
        return (slice(cz * n, cz * n + n), slice(cy * n, cy * n + n), slice(cx * n, cx * n + n))

    def old_face(j, r, kk, a):              # +a face of the upwind cell (old state)
        up = [j, r, kk]
        up[a] -= 1
        v = Gs[cell(*up)]
        return (v[:, :, n - 1], v[:, n - 1, :], v[n - 1, :, :])[a].reshape(-1)

    for s in range(RX + RY + RZ - 2):
        rcell = np.zeros(RZ + 1, dtype=np.int64)
        ritem = np.zeros(RZ + 1, dtype=np.int64)
        for kk in range(RZ):
            cnt, rlo, rhi = _hp_rows(s, kk, RX, RY)
            no = _hp_out_rows(s, kk, rlo, rhi, w)[0] if cnt else 0
            rcell[kk + 1] = rcell[kk] + cnt
            ritem[kk + 1] = ritem[kk] + cnt * NFF + no * (NN - NFF)
        items = int(ritem[RZ])

        def first_cell(P):                  # first cell whose first item is >= P
            if P >= items:
                return int(rcell[RZ])
            kk = int(np.searchsorted(ritem, P, side="right")) - 1
            cnt, rlo, rhi = _hp_rows(s, kk, RX, RY)
            assert cnt > 0
            no, olo = _hp_out_rows(s, kk, rlo, rhi, w)
            for r in range(rlo, rhi + 2):
                before = max(0, min(r, olo + no) - olo) if no else 0
                if ritem[kk] + (r - rlo) * NFF + before * (NN - NFF) >= P:
                    return int(rcell[kk] + r - rlo)
            raise AssertionError("no first cell")

        seen = np.zeros(int(rcell[RZ]), dtype=np.int64)
        par, par1 = s & 1, (s + 1) & 1
        for gi in range(G):
            cb, ce = first_cell(items * gi // G), first_cell(items * (gi + 1) // G)
            for c0 in range(cb, ce, nb):
                for c in range(c0, min(c0 + nb, ce)):
                    kk = int(np.searchsorted(rcell, c, side="right")) - 1
                    _, rlo, _ = _hp_rows(s, kk, RX, RY)
                    r = rlo + c - int(rcell[kk])
                    j = s - r - kk
                    assert 0 <= j < RX and 0 <= r < RY
                    seen[c] += 1
                    f = Gs[cell(j, r, kk)]
                    inflow = []
                    for a, edge in enumerate((j == 0, r == 0, kk == 0)):
                        if edge:
                            inflow.append(old_face(j, r, kk, a))
                        else:
                            assert written[par, a, kk, r] == s - 1
                            inflow.append(slots[par, a, kk, r])
                    tr = f.copy()                                    # theta r
                    tr[:, :, 0] += theta * k[0] * inflow[0].reshape(n, n)
                    tr[:, 0, :] += theta * k[1] * inflow[1].reshape(n, n)
                    tr[0, :, :] += theta * k[2] * inflow[2].reshape(n, n)
                    is_out = j >= w[0] and r >= w[1] and kk >= w[2]
                    x = (Binv[fnode] @ tr.reshape(-1)) if not is_out else Binv @ tr.reshape(-1)
                    if is_out:
                        sl = cell(j, r, kk)
                        assert np.isnan(out[sl]).all()
                        out[sl] = ((x - (1.0 - theta) * f.reshape(-1)) / theta).reshape(n, n, n)
                        xf = x.reshape(n, n, n)
                    else:
                        xf = np.full(NN, np.nan)
                        xf[fnode] = x
                        xf = xf.reshape(n, n, n)
                    for a, (jj, rr, kq, face) in enumerate(((j + 1, r, kk, xf[:, :, n - 1]),
                                                             (j, r + 1, kk, xf[:, n - 1, :]),
                                                             (j, r, kk + 1, xf[n - 1, :, :]))):
                        if jj < RX and rr < RY and kq < RZ:
                            assert written[par1, a, kq, rr] != s
                            written[par1, a, kq, rr] = s
                            slots[par1, a, kq, rr] = face.reshape(-1)
        assert (seen == 1).all()
    for a in range(3):
        if signs[a] < 0:
            out = np.flip(out, axis=2 - a)
    return out


@pytest.mark.parametrize("d,signs,nus,ncells,W,G,nb", [(1, (1, 1, 1), (1.0, 1.0, 1.0), (3, 4, 2), (17, 17, 17), 3, 16),
                                                       (2, (-1, 1, -1), (1.0, 1.0, 1.0), (3, 3, 3), (16, 16, 16), 5, 8),
                                                       (1, (1, -1, -1), (0.7, 1.0, 0.9), (2, 3, 4), (17, 17, 17), 2, 32)])
def test_corner_hyperplane_sweep_with_face_slots_equals_the_lu_solve(d, signs, nus, ncells, W, G, nb):
    mesh, T = _lu_reference(3, ncells, d, signs, nus, 0.5)
    F = np.random.default_rng(7 + d).standard_normal(mesh.shape)
    ref = T(F)
    assert _rel(_hyperplane_sweep(F, d, nus, 0.5, signs, W, G, nb), ref) < 1e-14
    assert _rel(_hyperplane_sweep(F, d, nus, 0.5, signs, (2, 2, 2), G, nb), ref) > 1e-6
