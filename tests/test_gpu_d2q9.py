"""GPU parity of the D2Q9 path (Section 5.1 model): the diagonal-velocity transport of the
CUDA library against the oracle's 2-D Fourier solver, through the C ABI.

Bar: relative L2 error <= 1e-12 over the nine populations.  Cases: every degree, the
three schemes (their diagonal sub-step counts leave the populations in either slot set),
theta != 1/2, rectangular cells (nu_x != nu_y), meshes smaller than the truncation width
(the tile's upwind start wraps around the torus several times), meshes that need several
tiles along both axes with ragged last tiles, both precisions, and the full 2048^2-point
workload in the launch configuration the benchmark times.
"""
import dataclasses

import numpy as np
import pytest

from gpu_common import assert_parity, oracle_mesh, oracle_model, oracle_w0, run_gpu, run_oracle
from paper_1702_00169_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12
BASE = W.D2Q9_ISO


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1702_00169_gb300 import pdg  # noqa: F401  (fails loudly if the library is missing)


def _cfg(nm, ns, order, **kw):
    return dataclasses.replace(BASE, n_macro=nm, n_sub=ns, order=order, **kw)


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_orders_multi_tile_ragged(order):
    """5x3 macrocells x 7x9 subcells (35 x 27 cells): several tiles per axis, ragged."""
    cfg = _cfg((5, 3), (7, 9), order)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 5)
    f = run_gpu(cfg, w0, cfg.dt, 5)
    assert_parity(f, f_ref, TOL)


@pytest.mark.parametrize("scheme,nsteps", [("M2", 3), ("M2_collapsed", 4), ("M2_collapsed", 3),
                                           ("M2_kin", 3), ("M2_kin", 2)])
def test_schemes(scheme, nsteps):
    cfg = _cfg((4, 4), (4, 4), 2)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, nsteps, scheme=scheme)
    f = run_gpu(cfg, w0, cfg.dt, nsteps, scheme=scheme)
    assert_parity(f, f_ref, TOL)


@pytest.mark.parametrize("theta,cfl", [(0.7, 1.0), (1.0, 1.0), (0.5, 2.0), (0.5, 4.0), (0.5, 0.3)])
def test_theta_and_cfl(theta, cfl):
    cfg = _cfg((3, 5), (5, 3), 3, theta=theta, cfl=cfl)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 4)
    f = run_gpu(cfg, w0, cfg.dt, 4)
    assert_parity(f, f_ref, TOL)


@pytest.mark.parametrize("ncells,order", [((1, 1), 2), ((2, 3), 1), ((3, 2), 4), ((1, 7), 3)])
def test_tiny_meshes_wrap(ncells, order):
    """Meshes far smaller than the truncation width: the swept region wraps the torus."""
    cfg = _cfg(ncells, (1, 1), order)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 3)
    f = run_gpu(cfg, w0, cfg.dt, 3)
    assert_parity(f, f_ref, TOL)


def test_rectangular_cells():
    """lengths (1.0, 0.6): nu_x != nu_y, dt = h_min / lambda."""
    cfg = _cfg((6, 4), (3, 3), 2, lengths=(1.0, 0.6, 1.0))
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 4)
    f = run_gpu(cfg, w0, cfg.dt, 4)
    assert_parity(f, f_ref, TOL)


def test_df32():
    cfg = _cfg((5, 3), (7, 9), 3)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 6)
    f = run_gpu(cfg, w0, cfg.dt, 6, precision=1)
    assert_parity(f, f_ref, TOL)


def test_moments_and_checkpoint():
    """get_w equals P f of the oracle state; get_f / set_f round trip continues exactly."""
    from paper_1702_00169_gb300 import pdg
    cfg = _cfg((4, 3), (4, 4), 2)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 3)
    s = pdg.solver_for(cfg)
    s.set_w(np.ascontiguousarray(w0.reshape(-1)))
    s.step(cfg.dt, 3)
    w = s.get_w().reshape(w0.shape)
    w_ref = oracle_model(cfg).moments(f_ref)
    assert_parity(w, w_ref, TOL)
    f3 = s.get_f()
    s.step(cfg.dt, 2)
    f5 = s.get_f()
    s.set_f(f3)
    s.step(cfg.dt, 2)
    np.testing.assert_array_equal(s.get_f(), f5)
    s.close()


def test_unsupported_requests():
    """dt <= 0 and theta = 0 are refused with PDG_ERR_UNSUPPORTED; a batch refuses D2Q9
    instances."""
    from paper_1702_00169_gb300 import pdg
    cfg = _cfg((2, 2), (2, 2), 1)
    w0 = oracle_w0(cfg)
    s = pdg.solver_for(cfg)
    s.set_w(np.ascontiguousarray(w0.reshape(-1)))
    with pytest.raises(pdg.PdgError) as e:
        s.step(-cfg.dt, 1)
    assert e.value.status == pdg.PDG_ERR_UNSUPPORTED
    with pytest.raises(pdg.PdgError) as e:
        s.set_model("isothermal_d2q9", cfg.lam, theta=0.0)
    assert e.value.status == pdg.PDG_ERR_UNSUPPORTED
    with pytest.raises(pdg.PdgError):
        pdg.Batch([s])
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_one_step_vs_oracle(precision):
    """The 2048^2-point D2Q9 workload (512^2 cells, d = 3), one step, whole state."""
    from paper_1702_00169_gb300 import pdg
    cfg = BASE
    w0 = oracle_w0(cfg)
    s = pdg.solver_for(cfg, precision=precision)
    s.set_w(np.ascontiguousarray(w0.reshape(-1)))
    s.step(cfg.dt, 1)
    f = s.get_f().reshape((1, 9) + w0.shape[1:])
    s.close()
    f_ref = run_oracle(cfg, w0, cfg.dt, 1)
    assert_parity(f, f_ref, TOL)


def test_full_size_conservation():
    """The workload's steps at full size: weighted totals of rho, rho u conserved."""
    from oracle import scheme as OS
    from paper_1702_00169_gb300 import pdg
    cfg = BASE
    w0 = oracle_w0(cfg)
    s = pdg.solver_for(cfg)
    s.set_w(np.ascontiguousarray(w0.reshape(-1)))
    s.step(cfg.dt, cfg.steps)
    w = s.get_w().reshape(w0.shape)
    s.close()
    mesh = oracle_mesh(cfg)
    t0, t1 = OS.weighted_total(mesh, w0), OS.weighted_total(mesh, w)
    assert np.all(np.isfinite(w))
    assert np.max(np.abs(t1 - t0)) <= 1e-12 * max(1.0, np.max(np.abs(t0)))
