"""GPU parity of the 3-D lattices (D3Q15, D3Q19, D3Q27) on meshes with inflow axes (eq. (2.6),
fictitious cells of eq. (3.8)): axis populations through the line passes, edge populations
through the plane-wise diagonal sweep and corner populations through the hyperplane sweep
(the default; boxes where a launch shape forces them); a region that reaches an inflow face
starts there from the boundary data, the others from their truncated upwind start.  Against the oracle's sparse LU of the assembled
system with the same boundary data.  Bar: relative L2 <= 1e-12."""
import dataclasses

import numpy as np
import pytest

from gpu_common import assert_parity, oracle_model, oracle_w0
from paper_1702_00169_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12
BASES = {"q19": W.D3Q19_ISO, "q15": W.D3Q15_ISO, "q27": W.D3Q27_ISO}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1702_00169_gb300 import pdg  # noqa: F401


def _face_data(model, fbf, axis):
    """[2][q_f][lines]: the populations entering through the low (xi_a > 0) and the high
    (xi_a < 0) face normal to `axis`, in population order, at that face's points (lines in
    C order of the other axes)."""
    xi = model.velocities() / model.lam
    npax = 2 - axis                                   # numpy axis of geometric axis `axis`
    lo = [np.take(fbf[i], 0, axis=npax).reshape(-1) for i in range(len(xi)) if xi[i, axis] > 0]
    hi = [np.take(fbf[i], -1, axis=npax).reshape(-1) for i in range(len(xi)) if xi[i, axis] < 0]
    return np.ascontiguousarray(np.stack([np.stack(lo), np.stack(hi)]))


def _run(cfg, periodic, nsteps, scheme="M2", precision=0, launch=None):
    from oracle import scheme as OS
    from oracle.dg import CartesianMesh
    from paper_1702_00169_gb300 import pdg
    model = oracle_model(cfg)
    mesh = CartesianMesh(3, cfg.ncells, cfg.order, lengths=cfg.lengths[:3], periodic=periodic)
    w0 = oracle_w0(cfg)
    X = mesh.coords1d(0)[None, None, :]
    Y = mesh.coords1d(1)[None, :, None]
    Z = mesh.coords1d(2)[:, None, None]
    wb = w0.copy()                                    # a smooth boundary state != the initial one
    wb[0] = w0[0] * (1.0 + 0.05 * np.cos(2 * np.pi * (X + 0.5 * Y)) * np.cos(np.pi * Z))
    wb[1] = w0[1] + 0.02 * wb[0]
    fbf = model.feq(wb)[0]                            # (q, P_z, P_y, P_x)
    tr = OS.Transporter(mesh, model, cfg.theta, "direct", fb=fbf[None])
    f_ref = OS.run(OS.initial_state(model, w0), tr, model, cfg.dt, nsteps, cfg.omega, scheme)
    s = pdg.Solver(3, cfg.n_macro, cfg.n_sub, cfg.order, lengths=cfg.lengths[:3], periodic=periodic)
    s.set_model(cfg.kind, cfg.lam, theta=cfg.theta, omega=cfg.omega, scheme=scheme, precision=precision)
    if launch:
        for k, sh in launch.items():
            s.set_launch(k, *sh)
    s.set_w(np.ascontiguousarray(w0.reshape(-1)))
    for a in range(3):
        if not periodic[a]:
            s.set_inflow(a, _face_data(model, fbf, a).reshape(-1))
    s.step(cfg.dt, nsteps)
    f = s.get_f().reshape(f_ref.shape)
    s.close()
    return f, f_ref


def _cfg(lat, nm, ns, order, **kw):
    return dataclasses.replace(BASES[lat], n_macro=nm, n_sub=ns, order=order, **kw)


@pytest.mark.parametrize("lat,periodic,order", [
    ("q19", (False, True, True), 1), ("q19", (True, False, False), 2),
    ("q15", (False, True, True), 2), ("q15", (True, True, False), 1),
    ("q27", (False, False, False), 1), ("q27", (True, False, True), 2),
])
def test_inflow_axes(lat, periodic, order):
    cfg = _cfg(lat, (3, 2, 2), (1, 2, 2), order)
    f, f_ref = _run(cfg, periodic, 3)
    assert_parity(f, f_ref, TOL)


@pytest.mark.parametrize("lat", ["q15", "q27"])
def test_long_inflow_axis_truncated_boxes(lat):
    """24 cells along the inflow axis x with 4-cell boxes: the boxes near the inflow face
    start there, the others 17 cells upwind from the old values (truncated start)."""
    cfg = _cfg(lat, (12, 1, 2), (2, 2, 1), 1)
    f, f_ref = _run(cfg, (False, True, True), 2, launch={5: (256, 4, 2)})
    assert_parity(f, f_ref, TOL)


def test_inflow_schemes_df32():
    cfg = _cfg("q27", (2, 2, 2), (1, 2, 2), 1)
    f, f_ref = _run(cfg, (False, True, False), 2, scheme="M2_collapsed", precision=1)
    assert_parity(f, f_ref, TOL)
    f, f_ref = _run(cfg, (True, False, True), 2, scheme="M2_kin")
    assert_parity(f, f_ref, TOL)


@pytest.mark.parametrize("precision", [2, 3])
@pytest.mark.parametrize("lat,periodic", [("q15", (False, True, False)), ("q27", (True, False, True)),
                                          ("q27", (False, False, False))])
def test_tensor_core_corner_pass_with_inflow(lat, periodic, precision):
    """The tensor-core precision forms (split-TF32 cell inverse with an FP64 or a
    double-float refinement residual) on inflow axes, at the mixed-precision bar 1e-10."""
    cfg = _cfg(lat, (2, 2, 3), (2, 3, 2), 2)
    f, f_ref = _run(cfg, periodic, 2, precision=precision)
    assert_parity(f, f_ref, 1e-10)
