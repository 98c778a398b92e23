"""GPU parity of the D2Q9 path on meshes with inflow axes (eq. (2.6), fictitious cells of
eq. (3.8)): the tiles of the diagonal sweep that reach an inflow face start there from the
boundary data, the others from their truncated upwind start.  Against the oracle's
sparse LU of the assembled system with the same boundary data.  Includes the paper's
Section 5.1 configuration: isothermal Euler at rest in a gravity field, exact hydrostatic
state rho_0 exp(-g y / c^2) imposed at the y faces, x periodic."""
import dataclasses

import numpy as np
import pytest

from gpu_common import assert_parity, oracle_mesh, oracle_model, oracle_w0, rel_l2
from paper_1702_00169_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12
LOW = {0: (1, 5, 8), 1: (2, 5, 6)}
HIGH = {0: (3, 6, 7), 1: (4, 7, 8)}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1702_00169_gb300 import pdg  # noqa: F401


def _fb_gpu(fbf, axis):
    """[2][3][lines] from the field-shaped boundary populations fbf (9, P_y, P_x)."""
    if axis == 1:
        lo = [fbf[p, 0, :] for p in LOW[1]]
        hi = [fbf[p, -1, :] for p in HIGH[1]]
    else:
        lo = [fbf[p, :, 0] for p in LOW[0]]
        hi = [fbf[p, :, -1] for p in HIGH[0]]
    return np.ascontiguousarray(np.stack([np.stack(lo), np.stack(hi)]))


def _run(cfg, w0, wb, periodic, nsteps, scheme="M2", source=None, precision=0):
    from oracle import scheme as OS
    from oracle.dg import CartesianMesh
    from oracle.source import Source
    from paper_1702_00169_gb300 import pdg
    model = oracle_model(cfg)
    mesh = CartesianMesh(2, cfg.ncells, cfg.order, lengths=cfg.lengths[:2], periodic=periodic)
    fbf = model.feq(wb)                                   # (1, 9, P_y, P_x)
    tr = OS.Transporter(mesh, model, cfg.theta, "direct", fb=fbf)
    src = None if source is None else Source(**source)
    f_ref = OS.run(OS.initial_state(model, w0), tr, model, cfg.dt, nsteps, cfg.omega, scheme, source=src)
    s = pdg.Solver(2, cfg.n_macro, cfg.n_sub, cfg.order, lengths=cfg.lengths[:2], periodic=periodic)
    s.set_model(cfg.kind, cfg.lam, theta=cfg.theta, omega=cfg.omega, scheme=scheme, precision=precision)
    if source is not None:
        s.set_source(**source)
    s.set_w(np.ascontiguousarray(w0.reshape(-1)))
    for a in range(2):
        if not periodic[a]:
            s.set_inflow(a, _fb_gpu(fbf[0], a).reshape(-1))
    s.step(cfg.dt, nsteps)
    f = s.get_f().reshape((1, 9) + w0.shape[1:])
    s.close()
    return f, f_ref


def _cfg(nm, ns, order):
    return dataclasses.replace(W.D2Q9_ISO, n_macro=nm, n_sub=ns, order=order)


def _wb(cfg, shift=0.0):
    """A smooth boundary state (different from the initial state)."""
    mesh = oracle_mesh(cfg)
    X = mesh.coords1d(0)[None, :]
    Y = mesh.coords1d(1)[:, None]
    rho = 1.0 + 0.03 * np.cos(2 * np.pi * (X + shift)) + 0.02 * np.sin(2 * np.pi * Y)
    return np.stack([rho, rho * 0.04 * np.cos(2 * np.pi * Y), rho * 0.03 * np.sin(2 * np.pi * X)])


@pytest.mark.parametrize("periodic", [(True, False), (False, True), (False, False)],
                         ids=["y_inflow", "x_inflow", "both_inflow"])
@pytest.mark.parametrize("order", [1, 3])
def test_inflow_axes(periodic, order):
    """8x6 macrocells x 5x5 subcells: several tiles per axis, some starting at an inflow face,
    the others with a truncated start."""
    cfg = _cfg((8, 6), (5, 5), order)
    w0 = oracle_w0(cfg)
    f, f_ref = _run(cfg, w0, _wb(cfg), periodic, 4)
    assert_parity(f, f_ref, TOL)


@pytest.mark.parametrize("scheme", ["M2_collapsed", "M2_kin"])
def test_inflow_schemes(scheme):
    cfg = _cfg((4, 4), (3, 3), 2)
    w0 = oracle_w0(cfg)
    f, f_ref = _run(cfg, w0, _wb(cfg, 0.2), (False, False), 3, scheme=scheme)
    assert_parity(f, f_ref, TOL)


@pytest.mark.parametrize("precision", [0, 1])
def test_hydrostatic_gravity(precision):
    """Section 5.1: isothermal fluid at rest under gravity g = -g e_y; the exact stationary
    state rho = rho_0 exp(-g y / c^2) is the initial state and the inflow data at the y
    faces; x periodic.  GPU == oracle, and the state stays hydrostatic to discretisation
    accuracy."""
    cfg = dataclasses.replace(_cfg((4, 4), (4, 4), 2), cfl=0.25)
    mesh = oracle_mesh(cfg)
    g, c2 = 1.0, cfg.lam ** 2 / 3.0
    Y = mesh.coords1d(1)[:, None] + 0 * mesh.coords1d(0)[None, :]
    rho = np.exp(-g * Y / c2)
    wex = np.stack([rho, 0 * rho, 0 * rho])
    src = dict(gravity=(0.0, -g))
    nsteps = 8                                  # t = 0.125, the paper's t_max of about 0.12
    f, f_ref = _run(cfg, wex, wex, (True, False), nsteps, source=src, precision=precision)
    assert_parity(f, f_ref, TOL)
    from oracle import models as OM
    w = OM.Model(OM.ISOTHERMAL_D2Q9, 2, cfg.lam).moments(f)
    assert rel_l2(w[0], wex[0]) < 2e-3          # discretisation error, rho spans 1 .. 0.05
    assert np.max(np.abs(w[1:])) < 2e-3
