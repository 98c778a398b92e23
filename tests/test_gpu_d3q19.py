"""GPU parity of the D3Q19 path: axis populations through the line passes, the twelve
edge populations through the diagonal sweep on every plane of points (three launches
per diagonal sub-step, planes xy, xz, yz), against the oracle's plane-wise Fourier form.
Bar: relative L2 <= 1e-12 over the nineteen populations."""
import dataclasses

import numpy as np
import pytest

from gpu_common import assert_parity, oracle_mesh, oracle_model, oracle_w0, run_gpu, run_oracle
from paper_1702_00169_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12
BASE = W.D3Q19_ISO


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1702_00169_gb300 import pdg  # noqa: F401


def _cfg(nm, ns, order, **kw):
    return dataclasses.replace(BASE, n_macro=nm, n_sub=ns, order=order, **kw)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_orders_ragged(order):
    cfg = _cfg((3, 2, 4), (2, 3, 2), order)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 3)
    f = run_gpu(cfg, w0, cfg.dt, 3)
    assert_parity(f, f_ref, TOL)


@pytest.mark.parametrize("scheme,nsteps", [("M2_collapsed", 3), ("M2_kin", 2)])
def test_schemes(scheme, nsteps):
    cfg = _cfg((2, 3, 2), (2, 2, 2), 2)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, nsteps, scheme=scheme)
    f = run_gpu(cfg, w0, cfg.dt, nsteps, scheme=scheme)
    assert_parity(f, f_ref, TOL)


@pytest.mark.parametrize("theta,cfl", [(0.7, 1.0), (0.5, 2.0)])
def test_theta_cfl_rectangular(theta, cfl):
    cfg = _cfg((2, 2, 3), (3, 2, 2), 2, theta=theta, cfl=cfl, lengths=(1.0, 0.7, 1.2))
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 3)
    f = run_gpu(cfg, w0, cfg.dt, 3)
    assert_parity(f, f_ref, TOL)


def test_tiny_mesh_wraps():
    cfg = _cfg((1, 1, 2), (1, 1, 1), 2)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 3)
    f = run_gpu(cfg, w0, cfg.dt, 3)
    assert_parity(f, f_ref, TOL)


def test_df32():
    cfg = _cfg((3, 2, 2), (2, 2, 3), 2)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 4)
    f = run_gpu(cfg, w0, cfg.dt, 4, precision=1)
    assert_parity(f, f_ref, TOL)


def test_larger_mesh_two_steps():
    """24^3 cells, d = 2 (72^3 points): several tiles or whole planes per block."""
    cfg = _cfg((6, 6, 6), (4, 4, 4), 2)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 2)
    f = run_gpu(cfg, w0, cfg.dt, 2)
    assert_parity(f, f_ref, TOL)


def test_moments_checkpoint_and_refusals():
    from paper_1702_00169_gb300 import pdg
    cfg = _cfg((2, 2, 2), (2, 2, 2), 1)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 2)
    s = pdg.solver_for(cfg)
    s.set_w(np.ascontiguousarray(w0.reshape(-1)))
    s.step(cfg.dt, 2)
    assert_parity(s.get_w().reshape(w0.shape), oracle_model(cfg).moments(f_ref), TOL)
    f2 = s.get_f()
    s.step(cfg.dt, 1)
    f3 = s.get_f()
    s.set_f(f2)
    s.step(cfg.dt, 1)
    np.testing.assert_array_equal(s.get_f(), f3)
    with pytest.raises(pdg.PdgError):
        pdg.Batch([s])
    s.close()
    s2 = pdg.Solver(3, (2, 2, 2), (2, 2, 2), 1)
    with pytest.raises(pdg.PdgError) as e:       # the D3Q lattices need dim = 3
        s2.set_model("isothermal_d2q9", 1.0)
    assert e.value.status == pdg.PDG_ERR_UNSUPPORTED
    s2.close()


def test_full_size_conservation():
    """The 384^3-point workload (19 populations, 31 state slots, 14 GB): weighted totals of
    rho and rho u conserved over the workload's steps, state finite."""
    from oracle import scheme as OS
    from paper_1702_00169_gb300 import pdg
    cfg = BASE
    mesh = oracle_mesh(cfg)
    w0 = oracle_w0(cfg)
    s = pdg.solver_for(cfg)
    s.set_w(np.ascontiguousarray(w0.reshape(-1)))
    s.step(cfg.dt, cfg.steps)
    w = s.get_w().reshape(w0.shape)
    s.close()
    t0, t1 = OS.weighted_total(mesh, w0), OS.weighted_total(mesh, w)
    assert np.all(np.isfinite(w))
    assert np.max(np.abs(t1 - t0)) <= 1e-12 * max(1.0, np.max(np.abs(t0)))


@pytest.mark.parametrize("ncells", [(128, 128, 4), (4, 128, 128)])
def test_edge_tiles_at_the_benchmark_shape(ncells):
    """The diagonal kernel on the edge planes at the tile shape of the 384^3-point benchmark:
    one 128 x 128-cell tile per plane and population (256 threads), swept from 15 cells
    upwind, so the start region wraps around the periodic plane.  (128, 128, 4) puts the xy
    planes at that shape, (4, 128, 128) the yz planes; the xz planes run 128 x 4 tiles.
    One M2 step, d = 2, against the oracle's plane-wise Fourier form, every value compared."""
    nm = tuple(c // 4 if c % 4 == 0 else c for c in ncells)
    ns = tuple(4 if c % 4 == 0 else 1 for c in ncells)
    cfg = _cfg(nm, ns, 2)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 1)
    f = run_gpu(cfg, w0, cfg.dt, 1, launch={4: (256, 128, 128)})
    assert_parity(f, f_ref, TOL)
