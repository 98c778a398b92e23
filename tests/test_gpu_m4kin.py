"""GPU parity of M4^kin, the triple-jump composition M2^kin(g1 dt) M2^kin(g2 dt) M2^kin(g1 dt)
of Section 3.2's palindromic step (g2 < 0: the middle sub-step runs backwards in time).
Bar: relative L2 <= 1e-12 against the oracle in FP64; the double-float state is held to the
mixed-precision bar 1e-10 (backward transports are anti-dissipative and amplify rounding)."""
import dataclasses

import numpy as np
import pytest

from gpu_common import assert_parity, oracle_w0, run_gpu, run_oracle
from paper_1702_00169_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1702_00169_gb300 import pdg  # noqa: F401


CASES = {
    "advection": dataclasses.replace(W.ADVECTION_D2Q4, n_macro=(3, 2), n_sub=(3, 5), order=2, cfl=0.25),
    "shallow_water": dataclasses.replace(W.SW_D2Q4, n_macro=(2, 3), n_sub=(4, 3), order=3, cfl=0.25),
    "euler3d": dataclasses.replace(W.EULER_D3Q6, n_macro=(2, 2, 3), n_sub=(2, 3, 2), order=1, cfl=0.25),
    "sw_degree4": dataclasses.replace(W.SW_D2Q4, n_macro=(2, 2), n_sub=(2, 3), order=4, cfl=0.2),
}


@pytest.mark.parametrize("name", list(CASES))
def test_m4kin_parity(name):
    cfg = CASES[name]
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 3, scheme="M4_kin")
    f = run_gpu(cfg, w0, cfg.dt, 3, scheme="M4_kin")
    assert_parity(f, f_ref, TOL)


def test_m4kin_df32():
    cfg = CASES["shallow_water"]
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 3, scheme="M4_kin")
    f = run_gpu(cfg, w0, cfg.dt, 3, scheme="M4_kin", precision=1)
    assert_parity(f, f_ref, 1e-10)


def test_m4kin_batch_equals_alone_bitwise():
    from paper_1702_00169_gb300 import pdg
    cfgs = [CASES["advection"], CASES["shallow_water"], CASES["euler3d"]]
    solo = []
    for c in cfgs:
        s = pdg.solver_for(c, scheme="M4_kin")
        s.set_w(np.ascontiguousarray(oracle_w0(c).reshape(-1)))
        s.step(c.dt, 2)
        solo.append(s.get_f())
        s.close()
    sol = []
    for c in cfgs:
        s = pdg.solver_for(c, scheme="M4_kin")
        s.set_w(np.ascontiguousarray(oracle_w0(c).reshape(-1)))
        sol.append(s)
    b = pdg.Batch(sol)
    b.step([c.dt for c in cfgs], [2, 2, 2])
    for s, f in zip(sol, solo):
        np.testing.assert_array_equal(s.get_f(), f)
    b.close()
    for s in sol:
        s.close()


def test_m4kin_refusals():
    from paper_1702_00169_gb300 import pdg
    q9 = dataclasses.replace(W.D2Q9_ISO, n_macro=(2, 2), n_sub=(2, 2), order=1)
    s = pdg.solver_for(q9, scheme="M4_kin")
    s.set_w(np.ascontiguousarray(oracle_w0(q9).reshape(-1)))
    with pytest.raises(pdg.PdgError) as e:
        s.step(q9.dt, 1)
    assert e.value.status == pdg.PDG_ERR_UNSUPPORTED
    with pytest.raises(pdg.PdgError) as e:
        s.set_source(gravity=(0.0, -1.0))
    assert e.value.status == pdg.PDG_ERR_UNSUPPORTED
    s.close()
