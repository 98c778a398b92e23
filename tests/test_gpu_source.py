"""GPU parity of the source stage S_2 of M_2^s (Section 3.2) on the D2Q9 path: gravity
(Section 5.1) and penalisation (Section 5.2), against oracle.source through the C ABI.
Bar: relative L2 <= 1e-12 over the nine populations."""
import dataclasses

import numpy as np
import pytest

from gpu_common import assert_parity, oracle_w0, run_gpu, run_oracle
from paper_1702_00169_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12
GRAV = dict(gravity=(0.3, -2.0))
PEN = dict(K_s=300.0, kappa=40.0, x_c=(0.35, 0.6), w_s=(1.0, 0.0, 0.0))
BOTH = dict(gravity=(0.0, -1.0), K_s=50.0, kappa=20.0, x_c=(0.5, 0.5), w_s=(1.02, 0.01, -0.01))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1702_00169_gb300 import pdg  # noqa: F401


def _cfg(order=2, nm=(4, 3), ns=(4, 5)):
    return dataclasses.replace(W.D2Q9_ISO, n_macro=nm, n_sub=ns, order=order)


@pytest.mark.parametrize("src", [GRAV, PEN, BOTH], ids=["gravity", "penalization", "both"])
@pytest.mark.parametrize("scheme", ["M2", "M2_collapsed"])
def test_sources(src, scheme):
    cfg = _cfg()
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 4, scheme=scheme, source=src)
    f = run_gpu(cfg, w0, cfg.dt, 4, scheme=scheme, source=src)
    assert_parity(f, f_ref, TOL)


@pytest.mark.parametrize("order", [1, 3, 4])
def test_source_orders_and_theta(order):
    src = dict(BOTH, theta=1.0)
    cfg = _cfg(order, (3, 3), (3, 4))
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 3, source=src)
    f = run_gpu(cfg, w0, cfg.dt, 3, source=src)
    assert_parity(f, f_ref, TOL)


def test_source_df32():
    cfg = _cfg(3)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 5, source=BOTH)
    f = run_gpu(cfg, w0, cfg.dt, 5, source=BOTH, precision=1)
    assert_parity(f, f_ref, TOL)


def test_uniform_fall_on_gpu():
    """Uniform state under gravity: rho u = rho u_0 + rho g t exactly up to the rounding of
    the transports (the diagonal sweeps round at about 1e-15 per step)."""
    from paper_1702_00169_gb300 import pdg
    cfg = _cfg(2, (2, 2), (3, 3))
    s = pdg.solver_for(cfg)
    P = cfg.npoints
    w0 = np.concatenate([np.full(P, 1.3), np.full(P, 0.02), np.full(P, 0.01)])
    s.set_w(w0)
    s.set_source(gravity=(0.5, -2.0))
    s.step(cfg.dt, 6)
    w = s.get_w().reshape(3, P)
    s.close()
    t = 6 * cfg.dt
    np.testing.assert_allclose(w[0], 1.3, rtol=0, atol=1e-12)
    np.testing.assert_allclose(w[1], 0.02 + 1.3 * 0.5 * t, rtol=0, atol=1e-12)
    np.testing.assert_allclose(w[2], 0.01 - 1.3 * 2.0 * t, rtol=0, atol=1e-12)


def test_source_refusals():
    from paper_1702_00169_gb300 import pdg
    s = pdg.solver_for(_cfg(), scheme="M2_kin")
    with pytest.raises(pdg.PdgError) as e:
        s.set_source(**GRAV)
    assert e.value.status == pdg.PDG_ERR_UNSUPPORTED
    s.close()
    sw = pdg.solver_for(dataclasses.replace(W.SW_D2Q4, n_macro=(2, 2), n_sub=(2, 2)))
    with pytest.raises(pdg.PdgError) as e:
        sw.set_source(**GRAV)
    assert e.value.status == pdg.PDG_ERR_UNSUPPORTED
    sw.close()
