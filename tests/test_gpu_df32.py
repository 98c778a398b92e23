"""Double-float precision mode (PDG_PREC_DF32): state stored as FP32 pairs, every step
in double-word arithmetic on the FP32 pipes.

Bar: relative L2 error against the FP64 oracle <= 1e-12 (the FP64 bar) on the same
cases as the FP64 parity tests; the checkpoint round trip (get_f / set_f) is exact;
mixed FP64 / double-float batches and servers give each instance the result it has
alone.
"""
import dataclasses

import numpy as np
import pytest

from gpu_common import TOL_POINTWISE_REVERSED, TOL_POINTWISE_REVERSED_DF, assert_parity, oracle_model, oracle_w0, run_gpu, run_oracle
from paper_1702_00169_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12
DF = 1


def test_advection_workload_df32():
    cfg = W.ADVECTION_D2Q4
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, cfg.steps, method="direct")
    f = run_gpu(cfg, w0, cfg.dt, cfg.steps, precision=DF)
    assert_parity(f, f_ref, TOL)


@pytest.mark.parametrize("order", [1, 2, 3, 4])
@pytest.mark.parametrize("cfl", [1.0, 4.0])
def test_shallow_water_orders_df32(order, cfl):
    cfg = dataclasses.replace(W.SW_D2Q4, n_macro=(3, 2), n_sub=(3, 5), order=order, cfl=cfl)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 6)
    f = run_gpu(cfg, w0, cfg.dt, 6, precision=DF)
    assert_parity(f, f_ref, TOL)


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_negative_time_step_df32(order):
    """dt < 0 runs the anti-dissipative backward scheme, which amplifies rounding errors
    step after step (the FP64 path itself loses up to ~6e-13 here).  Double-word
    operations carry 3-5 u^2 error bounds (u = 2^-24), about 100-160 times the FP64 unit
    roundoff, so the time-reversed case is held to the mixed-precision bar 1e-10."""
    cfg = dataclasses.replace(W.SW_D2Q4, n_macro=(3, 2), n_sub=(3, 4), order=order)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, -cfg.dt, 3)
    e64 = assert_parity(run_gpu(cfg, w0, -cfg.dt, 3), f_ref, TOL, tol_pt=TOL_POINTWISE_REVERSED)
    e32 = assert_parity(run_gpu(cfg, w0, -cfg.dt, 3, precision=DF), f_ref, 1e-10, tol_pt=TOL_POINTWISE_REVERSED_DF)
    print(f"dt<0 d={order}: fp64 {e64} df32 {e32}")


@pytest.mark.parametrize("shape", [(1, 1, 1), (8, 3, 2), (3, 9, 4)])
def test_launch_shapes_full_ring_df32(shape):
    cfg = dataclasses.replace(W.SW_D2Q4, n_macro=(3, 3), n_sub=(3, 3), order=3, cfl=8.0)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 4)
    f = run_gpu(cfg, w0, cfg.dt, 4, launch={0: shape, 1: shape}, precision=DF)
    assert_parity(f, f_ref, TOL)


@pytest.mark.parametrize("theta", [0.0, 0.75, 1.0])
def test_theta_variants_df32(theta):
    cfl = 0.1 if theta == 0.0 else 2.0
    cfg = dataclasses.replace(W.ADVECTION_D2Q4, n_macro=(3, 4), n_sub=(2, 3), order=3, theta=theta, cfl=cfl)
    w0 = oracle_w0(cfg)
    assert_parity(run_gpu(cfg, w0, cfg.dt, 5, precision=DF), run_oracle(cfg, w0, cfg.dt, 5), TOL)


def test_euler_and_collapsed_df32():
    for cfg, scheme in ((dataclasses.replace(W.EULER_D3Q6, n_macro=(2, 3, 2), n_sub=(3, 2, 3), order=2), "M2"),
                        (dataclasses.replace(W.EULER_D3Q6, dim=2, n_macro=(3, 2), n_sub=(2, 3), order=3), "M2"),
                        (dataclasses.replace(W.SW_D2Q4, n_macro=(2, 3), n_sub=(4, 2), order=2), "M2_collapsed")):
        w0 = oracle_w0(cfg)
        f_ref = run_oracle(cfg, w0, cfg.dt, 3, scheme=scheme)
        assert_parity(run_gpu(cfg, w0, cfg.dt, 3, scheme=scheme, precision=DF), f_ref, TOL)


def test_shallow_water_100_steps_reduced_df32():
    cfg = W.SW_D2Q4.scaled(n_macro=(4, 4))
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, cfg.steps)
    f = run_gpu(cfg, w0, cfg.dt, cfg.steps, precision=DF)
    err = assert_parity(f, f_ref, TOL)
    print(f"df32 SW 100 steps (rel L2, pointwise) = {err}")


def test_checkpoint_roundtrip_exact_and_moments_df32():
    from paper_1702_00169_gb300 import pdg
    cfg = dataclasses.replace(W.SW_D2Q4, n_macro=(3, 2), n_sub=(4, 4), order=2)
    w0 = oracle_w0(cfg)
    s = pdg.solver_for(cfg, precision=DF)
    s.set_w(np.ascontiguousarray(w0.reshape(-1)))
    s.step(cfg.dt, 3)
    snap = s.get_f().copy()
    s.step(cfg.dt, 4)
    ref = s.get_f().copy()
    s.set_f(snap)
    np.testing.assert_array_equal(s.get_f(), snap)
    s.step(cfg.dt, 4)
    np.testing.assert_array_equal(s.get_f(), ref)
    w = s.get_w().reshape(w0.shape)
    f = s.get_f().reshape((cfg.m, 4) + w0.shape[1:])
    np.testing.assert_allclose(w, f.sum(axis=1), rtol=0, atol=1e-13 * np.max(np.abs(w)))
    s.close()


def test_mixed_precision_batch_and_server():
    from paper_1702_00169_gb300 import pdg
    cfgs = [dataclasses.replace(W.SW_D2Q4, n_macro=(3, 2), n_sub=(3, 5), order=3, seed=41),
            dataclasses.replace(W.ADVECTION_D2Q4, n_macro=(4, 3), n_sub=(2, 3), order=2, seed=42),
            dataclasses.replace(W.EULER_D3Q6, n_macro=(2, 2, 2), n_sub=(2, 3, 2), order=2, seed=43)]
    precs = [DF, 0, DF]
    alone = []
    for c, pr in zip(cfgs, precs):
        s = pdg.solver_for(c, precision=pr)
        s.set_w(np.ascontiguousarray(oracle_w0(c).reshape(-1)))
        b = pdg.Batch([s])
        b.step([c.dt], [4])
        alone.append(s.get_f().copy())
        b.close()
        s.close()
    sol = []
    for c, pr in zip(cfgs, precs):
        s = pdg.solver_for(c, precision=pr)
        s.set_w(np.ascontiguousarray(oracle_w0(c).reshape(-1)))
        sol.append(s)
    b = pdg.Batch(sol)
    b.step([c.dt for c in cfgs], [4] * 3, use_graph=True)
    for s, c, ref in zip(sol, cfgs, alone):
        f = s.get_f()
        np.testing.assert_array_equal(f, ref)
        fr = run_oracle(c, oracle_w0(c), c.dt, 4)
        assert_parity(f.reshape(fr.shape), fr, TOL)
    b.close()
    for s in sol:
        s.close()
    srv = pdg.Server(1 << 33, chunk_steps=3)
    ids = {srv.submit(c, oracle_w0(c), 5, precision=pr): (c, pr) for c, pr in zip(cfgs, precs)}
    got = {}
    while len(got) < len(ids):
        srv.iterate()
        for rid, ta, tb, tc in srv.poll():
            c, pr = ids[rid]
            got[rid] = srv.result(rid, c.m * c.npoints)
    srv.close()
    for rid, (c, pr) in ids.items():
        w_ref = oracle_model(c).moments(run_oracle(c, oracle_w0(c), c.dt, 5))
        assert_parity(got[rid].reshape(w_ref.shape), w_ref, TOL)


def test_noalloc_rejects_df32():
    from paper_1702_00169_gb300 import pdg
    cfg = dataclasses.replace(W.SW_D2Q4, n_macro=(2, 2), n_sub=(2, 2), order=2)
    s = pdg.solver_for(cfg, precision=DF)
    s.set_w(np.ascontiguousarray(oracle_w0(cfg).reshape(-1)))
    out = np.empty(s.info().w_len)
    assert pdg.pdg_get_w_noalloc(s.ctx, out.ctypes.data, out.size) == pdg.PDG_ERR_UNSUPPORTED
    s.close()
