"""Inflow boundaries (eq. (2.6), fictitious cells of eq. (3.8)) on the GPU against the
oracle's sparse-LU solve of the assembled system with boundary data.

Boundary data: f^b = f^eq(w^b) of a smooth boundary state, evaluated at the inflow
face points of every population."""
import dataclasses

import numpy as np
import pytest

from gpu_common import assert_parity, oracle_model, oracle_w0
from oracle import scheme as OS
from oracle.dg import CartesianMesh
from paper_1702_00169_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _mesh(cfg, periodic):
    return CartesianMesh(cfg.dim, cfg.ncells, cfg.order, lengths=cfg.lengths[:cfg.dim], periodic=periodic)


def _boundary_f(cfg, mesh):
    """f^b on the whole grid (only inflow face values are used): f^eq of a perturbed state."""
    w = oracle_w0(cfg)
    X = mesh.coords1d(0)
    bump = 1.0 + 0.05 * np.cos(2 * np.pi * X)
    wb = w.copy()
    wb[0] = w[0] * bump
    return oracle_model(cfg).feq(wb)


def _faces(cfg, Fb, axis):
    """[2][m][lines] slices of Fb for the GPU: side 0 = (k, +axis) at the low face,
    side 1 = (k, -axis) at the high face; lines in C order of the other axes."""
    gax = 1 + (cfg.dim - 1 - axis)          # numpy axis of the grid in Fb[:, i] (x is last)
    lo = np.take(Fb[:, 2 * axis], 0, axis=gax)
    hi = np.take(Fb[:, 2 * axis + 1], -1, axis=gax)
    return np.ascontiguousarray(np.stack([lo.reshape(cfg.m, -1), hi.reshape(cfg.m, -1)]))


def _run(cfg, periodic, nsteps, precision=0, scheme="M2", launch=None, dt=None):
    from paper_1702_00169_gb300 import pdg
    mesh = _mesh(cfg, periodic)
    Fb = _boundary_f(cfg, mesh)
    w0 = oracle_w0(cfg)
    dt = cfg.dt if dt is None else dt
    model = oracle_model(cfg)
    tr = OS.Transporter(mesh, model, theta=cfg.theta, method="direct", fb=Fb)
    f_ref = OS.run(OS.initial_state(model, w0), tr, model, dt, nsteps, cfg.omega, scheme)
    s = pdg.Solver(cfg.dim, cfg.n_macro, cfg.n_sub, cfg.order, lengths=cfg.lengths[:cfg.dim], periodic=periodic)
    s.set_model(cfg.kind, cfg.lam, a=cfg.a, gravity=cfg.gravity, gamma=cfg.gamma, omega=cfg.omega,
                theta=cfg.theta, scheme=scheme, precision=precision)
    if launch:
        for k, sh in launch.items():
            s.set_launch(k, *sh)
    s.set_w(np.ascontiguousarray(w0.reshape(-1)))
    for a in range(cfg.dim):
        if not periodic[a]:
            s.set_inflow(a, _faces(cfg, Fb, a))
    s.step(dt, nsteps)
    f = s.get_f().reshape(f_ref.shape)
    s.close()
    return f, f_ref


@pytest.mark.parametrize("order", [1, 2, 3, 4])
@pytest.mark.parametrize("periodic", [(False, True), (True, False), (False, False)])
def test_shallow_water_inflow(order, periodic):
    cfg = dataclasses.replace(W.SW_D2Q4, n_macro=(3, 2), n_sub=(2, 3), order=order)
    f, f_ref = _run(cfg, periodic, 4)
    assert_parity(f, f_ref, TOL)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("shape", [None, (4, 3, 2), (2, 6, 1)])
def test_inflow_shapes_windows_and_full_chain(precision, shape):
    """Forced shapes: window mode and, at CFL 8, segments shorter than the window (full
    open chain from the boundary); composed T T on the x axis."""
    cfg = dataclasses.replace(W.SW_D2Q4, n_macro=(3, 3), n_sub=(2, 2), order=3, cfl=8.0 if shape else 1.0)
    f, f_ref = _run(cfg, (False, False), 3, precision=precision,
                    launch=None if shape is None else {0: shape, 1: shape})
    assert_parity(f, f_ref, TOL)


def test_euler_3d_inflow_and_m2kin():
    cfg = dataclasses.replace(W.EULER_D3Q6, n_macro=(2, 2, 2), n_sub=(2, 1, 2), order=2)
    f, f_ref = _run(cfg, (False, True, False), 3)
    assert_parity(f, f_ref, TOL)
    cfg2 = dataclasses.replace(W.SW_D2Q4, n_macro=(2, 3), n_sub=(2, 2), order=2)
    f, f_ref = _run(cfg2, (False, True), 2, scheme="M2_kin")
    assert_parity(f, f_ref, TOL)


def test_negative_dt_on_inflow_axis_unsupported():
    from paper_1702_00169_gb300 import pdg
    cfg = dataclasses.replace(W.SW_D2Q4, n_macro=(2, 2), n_sub=(2, 2), order=3)
    s = pdg.Solver(2, cfg.n_macro, cfg.n_sub, cfg.order, periodic=(False, True))
    s.set_model(cfg.kind, cfg.lam, gravity=cfg.gravity)
    s.set_w(np.ascontiguousarray(oracle_w0(cfg).reshape(-1)))
    with pytest.raises(pdg.PdgError) as e:
        s.step(-cfg.dt, 1)
    assert e.value.status == pdg.PDG_ERR_UNSUPPORTED
    s.close()
