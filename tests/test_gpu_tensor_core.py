"""GPU parity of the tensor-core precision form (PDG_PREC_TF32 / PDG_PREC_TF32_DFRES).

The dense cell solves x = B^-1 r of the corner sweeps (D3Q15 / D3Q27 velocities
lambda (+-1, +-1, +-1); B of eq. (3.7) under the theta step of eq. (3.11), an
(n^3 x n^3) matrix) run as split-TF32 products on the tensor cores with one refinement
(residual in FP64, or in double-float); every other step stays FP64.  Against the oracle's
3-D Fourier form the bar is the mixed-precision one, relative L2 <= 1e-10 and every value
within 1e-10 max|f|; against the FP64 GPU path the difference must stay far below it.
The failure path of the kernel's bounded waits is exercised without any fault: a test
switch makes the wait watch an mbarrier nothing arrives on, and the host must then see
PDG_ERR_TIMEOUT once and a usable context."""
import dataclasses

import numpy as np
import pytest

from gpu_common import assert_parity, oracle_w0, rel_l2, run_gpu, run_oracle
from paper_1702_00169_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL_MIXED = 1e-10
BASES = {"q15": W.D3Q15_ISO, "q27": W.D3Q27_ISO}
PRECS = ("tf32", "tf32_df")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1702_00169_gb300 import pdg  # noqa: F401


def _cfg(lat, nm, ns, order, **kw):
    return dataclasses.replace(BASES[lat], n_macro=nm, n_sub=ns, order=order, **kw)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("lat", ["q15", "q27"])
@pytest.mark.parametrize("order", [1, 2, 3])
def test_orders_ragged_vs_oracle(lat, order, prec):
    cfg = _cfg(lat, (3, 2, 2), (2, 3, 2), order)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 3)
    f = run_gpu(cfg, w0, cfg.dt, 3, precision=prec)
    assert_parity(f, f_ref, TOL_MIXED)
    f64 = run_gpu(cfg, w0, cfg.dt, 3)
    assert rel_l2(f, f64) <= 1e-11


@pytest.mark.parametrize("prec", PRECS)
def test_schemes_theta_and_rectangular_cells(prec):
    """theta = 0.7, CFL 2 (three different start widths on rectangular cells), collapsed and
    M2^kin schemes."""
    for scheme, kw in (("M2_collapsed", {}), ("M2_kin", {}),
                       ("M2", dict(theta=0.7, cfl=2.0, lengths=(1.0, 1.5, 0.75)))):
        cfg = _cfg("q27", (2, 3, 2), (3, 2, 3), 2, **kw)
        w0 = oracle_w0(cfg)
        f_ref = run_oracle(cfg, w0, cfg.dt, 2, scheme=scheme)
        f = run_gpu(cfg, w0, cfg.dt, 2, scheme=scheme, precision=prec)
        assert_parity(f, f_ref, TOL_MIXED, scheme)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", [(5, 3, 2), (1, 1, 1), (9, 7, 4)])
def test_forced_boxes_ragged(prec, shape):
    """Forced box shapes (x, y, z cells): many boxes, ragged last boxes, one-cell boxes."""
    cfg = _cfg("q15", (2, 3, 5), (3, 2, 1), 2)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 2)
    f = run_gpu(cfg, w0, cfg.dt, 2, precision=prec, launch={6: shape})
    assert_parity(f, f_ref, TOL_MIXED)


def test_mesh_smaller_than_the_start_width():
    cfg = _cfg("q27", (1, 1, 2), (1, 1, 1), 2)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 3)
    for prec in PRECS:
        assert_parity(run_gpu(cfg, w0, cfg.dt, 3, precision=prec), f_ref, TOL_MIXED, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_corner_box_at_the_benchmark_shape(prec):
    """The 64 x 43 x 43-cell box of the 384^3-point run (start width 16), forced on an
    80 x 50 x 50-cell D3Q15 mesh: one M2 step, every value against the oracle."""
    cfg = _cfg("q15", (20, 25, 25), (4, 2, 2), 2)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 1)
    f = run_gpu(cfg, w0, cfg.dt, 1, precision=prec, launch={6: (64, 43, 43)})
    assert_parity(f, f_ref, TOL_MIXED)


def test_checkpoint_and_graph_replay():
    from paper_1702_00169_gb300 import pdg
    cfg = _cfg("q27", (2, 2, 2), (2, 2, 2), 2)
    w0 = oracle_w0(cfg)
    s = pdg.solver_for(cfg, precision="tf32")
    s.set_w(np.ascontiguousarray(w0.reshape(-1)))
    s.step(cfg.dt, 2)
    f2 = s.get_f()
    s.step(cfg.dt, 1)
    f3 = s.get_f()
    s.set_f(f2)
    s.step(cfg.dt, 1)
    np.testing.assert_array_equal(s.get_f(), f3)     # deterministic: bitwise the same
    s.set_f(f2)
    s.set_option(pdg.PDG_OPT_GRAPH, 1)
    s.step(cfg.dt, 1)                                # capture + replay
    np.testing.assert_array_equal(s.get_f(), f3)
    s.close()


def test_bounded_wait_runs_out_and_the_context_stays_usable():
    """PDG_OPT_DEBUG_TC_STALL: the kernel's waiting thread watches an mbarrier nothing
    arrives on; the bound (about 0.5 ms) runs out, every block drains its tensor-core work,
    frees its tensor memory and returns; the host reads PDG_ERR_TIMEOUT once.  Then the
    same context, switch off, reproduces the oracle."""
    from paper_1702_00169_gb300 import pdg
    cfg = _cfg("q15", (2, 2, 2), (2, 2, 2), 2)
    w0 = oracle_w0(cfg)
    s = pdg.solver_for(cfg, precision="tf32")
    s.set_w(np.ascontiguousarray(w0.reshape(-1)))
    s.set_option(pdg.PDG_OPT_DEBUG_TC_STALL, 1)
    s.step(cfg.dt, 1)                                # asynchronous: the launch itself succeeds
    with pytest.raises(pdg.PdgError) as e:
        s.synchronize()
    assert e.value.status == pdg.PDG_ERR_TIMEOUT
    s.synchronize()                                  # reported once
    s.set_option(pdg.PDG_OPT_DEBUG_TC_STALL, 0)
    s.set_w(np.ascontiguousarray(w0.reshape(-1)))
    s.step(cfg.dt, 2)
    f = s.get_f().reshape((1, cfg.nv) + w0.shape[1:])
    s.close()
    assert_parity(f, run_oracle(cfg, w0, cfg.dt, 2), TOL_MIXED)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("lat,order", [("q15", 1), ("q27", 2), ("q15", 3)])
def test_layer_pairs_equal_single_layers_bitwise(prec, lat, order):
    """PDG_OPT_TC_LAYERS: sweeping two box layers together (layer k + 1 one anti-diagonal
    behind layer k, both anti-diagonals in one product) changes where a cell's row sits in
    the product, not its arithmetic: the result is bitwise that of one layer at a time, and
    both match the oracle.  Odd layer counts leave a last single layer."""
    from paper_1702_00169_gb300 import pdg
    cfg = _cfg(lat, (3, 2, 3), (2, 3, 1), order)
    w0 = oracle_w0(cfg)
    out = {}
    for layers in (1, 2):
        s = pdg.solver_for(cfg, precision=prec)
        s.set_option(pdg.PDG_OPT_CORNER_SWEEP, 0)      # layer pairs belong to the box sweep
        s.set_option(pdg.PDG_OPT_TC_LAYERS, layers)
        s.set_w(np.ascontiguousarray(w0.reshape(-1)))
        s.step(cfg.dt, 3)
        out[layers] = s.get_f()
        s.close()
    np.testing.assert_array_equal(out[1], out[2])
    f_ref = run_oracle(cfg, w0, cfg.dt, 3)
    assert_parity(out[2].reshape(f_ref.shape), f_ref, TOL_MIXED)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("lat,order", [("q15", 1), ("q27", 2), ("q15", 2)])
def test_hyperplane_and_box_forms_match_the_oracle(prec, lat, order):
    """The tensor-core form on hyperplanes (default for degree <= 2: batches of up to 128
    cells of one hyperplane, one product row each) and on box anti-diagonals both reach
    the oracle within the mixed-precision bar; they differ by the refinement's rounding."""
    from paper_1702_00169_gb300 import pdg
    cfg = _cfg(lat, (3, 2, 3), (2, 3, 1), order)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 3)
    out = {}
    for sweep in (1, 0):
        s = pdg.solver_for(cfg, precision=prec)
        s.set_option(pdg.PDG_OPT_CORNER_SWEEP, sweep)
        s.set_w(np.ascontiguousarray(w0.reshape(-1)))
        s.step(cfg.dt, 3)
        out[sweep] = s.get_f().reshape(f_ref.shape)
        s.close()
        assert_parity(out[sweep], f_ref, TOL_MIXED, ("sweep", sweep))
    assert rel_l2(out[1], out[0]) <= 1e-11


@pytest.mark.parametrize("prec", PRECS)
def test_hyperplane_form_at_scale(prec):
    """80 x 50 x 50 cells, d = 2 (D3Q15): 226 hyperplanes, 19 blocks per population, many
    batches of 128 cells per block and step.  One M2 step, every value against the oracle."""
    cfg = _cfg("q15", (20, 25, 25), (4, 2, 2), 2)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 1)
    f = run_gpu(cfg, w0, cfg.dt, 1, precision=prec)
    assert_parity(f, f_ref, TOL_MIXED)
