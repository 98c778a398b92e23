"""GPU parity of the D3Q15 and D3Q27 paths: axis populations through the line passes, the
D3Q27 edge populations through the plane-wise diagonal sweep, and the eight corner
populations lambda (+-1, +-1, +-1) through the 3-D hyperplane sweep (the default) or, where a
launch shape forces it, the box sweep (layer-by-layer wavefronts), both from a truncated
upwind start, against the oracle's 3-D Fourier form.
Bar: relative L2 <= 1e-12 over all populations."""
import dataclasses

import numpy as np
import pytest

from gpu_common import assert_parity, oracle_mesh, oracle_model, oracle_w0, run_gpu, run_oracle
from paper_1702_00169_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12
BASES = {"q15": W.D3Q15_ISO, "q27": W.D3Q27_ISO}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1702_00169_gb300 import pdg  # noqa: F401


def _cfg(lat, nm, ns, order, **kw):
    return dataclasses.replace(BASES[lat], n_macro=nm, n_sub=ns, order=order, **kw)


@pytest.mark.parametrize("lat", ["q15", "q27"])
@pytest.mark.parametrize("order", [1, 2, 3])
def test_orders_ragged(lat, order):
    cfg = _cfg(lat, (3, 2, 4), (2, 3, 2), order)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 3)
    f = run_gpu(cfg, w0, cfg.dt, 3)
    assert_parity(f, f_ref, TOL)


@pytest.mark.parametrize("lat", ["q15", "q27"])
@pytest.mark.parametrize("scheme,nsteps", [("M2_collapsed", 3), ("M2_kin", 2)])
def test_schemes(lat, scheme, nsteps):
    cfg = _cfg(lat, (2, 3, 2), (2, 2, 2), 2)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, nsteps, scheme=scheme)
    f = run_gpu(cfg, w0, cfg.dt, nsteps, scheme=scheme)
    assert_parity(f, f_ref, TOL)


@pytest.mark.parametrize("theta,cfl", [(0.7, 1.0), (0.5, 2.0)])
def test_theta_cfl_rectangular(theta, cfl):
    """Different Courant numbers per axis (rectangular cells): three different start widths."""
    cfg = _cfg("q15", (2, 2, 3), (3, 2, 2), 2, theta=theta, cfl=cfl, lengths=(1.0, 0.7, 1.2))
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 3)
    f = run_gpu(cfg, w0, cfg.dt, 3)
    assert_parity(f, f_ref, TOL)


@pytest.mark.parametrize("lat", ["q15", "q27"])
def test_tiny_mesh_wraps(lat):
    """Meshes smaller than the start width: the region wraps around the torus many times."""
    cfg = _cfg(lat, (1, 1, 2), (1, 1, 1), 2)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 3)
    f = run_gpu(cfg, w0, cfg.dt, 3)
    assert_parity(f, f_ref, TOL)


@pytest.mark.parametrize("shape", [(128, 3, 2), (64, 1, 1), (512, 5, 4)])
def test_forced_boxes_ragged(shape):
    """Forced box shapes (threads, box x = box y, box z): many boxes, ragged last boxes."""
    cfg = _cfg("q27", (2, 3, 5), (3, 2, 1), 1)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 2)
    f = run_gpu(cfg, w0, cfg.dt, 2, launch={5: shape})
    assert_parity(f, f_ref, TOL)


@pytest.mark.parametrize("lat", ["q15", "q27"])
def test_df32(lat):
    cfg = _cfg(lat, (3, 2, 2), (2, 2, 3), 2)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 4)
    f = run_gpu(cfg, w0, cfg.dt, 4, precision=1)
    assert_parity(f, f_ref, TOL)


def test_larger_mesh_two_steps():
    """16^3 cells, d = 2 (48^3 points): several boxes per population."""
    cfg = _cfg("q27", (4, 4, 4), (4, 4, 4), 2)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 2)
    f = run_gpu(cfg, w0, cfg.dt, 2)
    assert_parity(f, f_ref, TOL)


@pytest.mark.parametrize("lat", ["q15", "q27"])
def test_moments_checkpoint_and_refusals(lat):
    from paper_1702_00169_gb300 import pdg
    cfg = _cfg(lat, (2, 2, 2), (2, 2, 2), 1)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 2)
    s = pdg.solver_for(cfg)
    s.set_w(np.ascontiguousarray(w0.reshape(-1)))
    np.testing.assert_allclose(s.get_w().reshape(w0.shape), w0, rtol=0, atol=1e-15)
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
    with pytest.raises(pdg.PdgError) as e:
        s.step(-cfg.dt, 1)
    assert e.value.status == pdg.PDG_ERR_UNSUPPORTED
    s.close()
    kind = cfg.kind
    s3 = pdg.Solver(3, (1, 1, 1), (2, 2, 2), 4)
    with pytest.raises(pdg.PdgError) as e:
        s3.set_model(kind, 1.0)
    assert e.value.status == pdg.PDG_ERR_UNSUPPORTED
    s3.close()


@pytest.mark.parametrize("lat", ["q15", "q27"])
def test_full_size_conservation(lat):
    """The 384^3-point workload (D3Q27: 27 populations, 47 state slots, 21 GB): weighted
    totals of rho and rho u conserved over the workload's steps, state finite."""
    from oracle import scheme as OS
    from paper_1702_00169_gb300 import pdg
    cfg = BASES[lat]
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


_BOX_REF = {}


@pytest.mark.parametrize("precision", [0, 1])
def test_corner_box_at_the_benchmark_shape(precision):
    """The corner kernel at the box shape the planner picks for the 384^3-point benchmark
    (64 x 43 x 43 output cells, start width 16 along every axis, the +z faces in the global
    scratch slice of each block), forced on an 80 x 50 x 50-cell D3Q15 mesh, d = 2: two full
    boxes and a ragged one per axis.  One M2 step against the oracle's 3-D Fourier form,
    every value compared (box starts included)."""
    cfg = _cfg("q15", (20, 25, 25), (4, 2, 2), 2)
    w0 = oracle_w0(cfg)
    if "f" not in _BOX_REF:
        _BOX_REF["f"] = run_oracle(cfg, w0, cfg.dt, 1)
    f = run_gpu(cfg, w0, cfg.dt, 1, precision=precision, launch={6: (64, 43, 43)})
    assert_parity(f, _BOX_REF["f"], TOL)
