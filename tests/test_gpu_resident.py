"""GPU parity of the line-resident pass kernel (PDG_OPT_RESIDENT) and of the collision carried by
another axis' pass (PDG_OPT_COLLISION_AXIS).

The resident kernel stages a block's lines in shared memory, runs the pass's operations there
(the same segment closure of the periodic theta step, eq. (3.11), and the collision of eq.
(3.12)) and writes them back once; moving the collision to another axis' pass reorders only
transports of different populations, which commute.  Both must reproduce the oracle at the
FP64 bar (relative L2 <= 1e-12 and every value within 1e-12 max|f|), in both precisions, for
every DnQ2n model, degree, scheme and launch shape, ring closures included."""
import dataclasses

import numpy as np
import pytest

from gpu_common import TOL_POINTWISE_REVERSED, assert_parity, oracle_w0, rel_l2, run_oracle
from paper_1702_00169_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1702_00169_gb300 import pdg  # noqa: F401


def _run(cfg, w0, dt, nsteps, scheme="M2", precision=0, caxis=-1, resident=1, shapes=None):
    from paper_1702_00169_gb300 import pdg
    s = pdg.solver_for(cfg, scheme=scheme, precision=precision)
    s.set_option(pdg.PDG_OPT_RESIDENT, resident)
    s.set_option(pdg.PDG_OPT_COLLISION_AXIS, caxis)
    for kind, sh in (shapes or {}).items():
        s.set_launch(kind, *sh)
    s.set_w(np.ascontiguousarray(w0.reshape(-1)))
    s.step(dt, nsteps)
    f = s.get_f().reshape((cfg.m, 2 * cfg.dim) + w0.shape[1:])
    s.close()
    return f


MODELS = {
    "advection": dataclasses.replace(W.ADVECTION_D2Q4, n_macro=(3, 4), n_sub=(3, 2)),
    "shallow_water": dataclasses.replace(W.SW_D2Q4, n_macro=(2, 3), n_sub=(4, 3)),
    "euler2": dataclasses.replace(W.EULER_D3Q6, dim=2, n_macro=(3, 2), n_sub=(2, 3)),
    "euler3": dataclasses.replace(W.EULER_D3Q6, n_macro=(2, 3, 2), n_sub=(3, 2, 2)),
}


@pytest.mark.parametrize("model", list(MODELS))
@pytest.mark.parametrize("order", [1, 2, 3, 4])
@pytest.mark.parametrize("caxis", [-1, 0])
def test_models_degrees_and_collision_axis(model, order, caxis):
    cfg = dataclasses.replace(MODELS[model], order=order)
    if model == "euler3" and order == 4:
        cfg = dataclasses.replace(cfg, n_macro=(2, 2, 2), n_sub=(2, 2, 2))
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 3)
    for precision in (0, 1):
        f = _run(cfg, w0, cfg.dt, 3, precision=precision, caxis=caxis)
        assert_parity(f, f_ref, TOL, (model, order, caxis, precision))


@pytest.mark.parametrize("scheme", ["M2_collapsed", "M2_kin"])
@pytest.mark.parametrize("caxis", [-1, 0, 1])
def test_schemes(scheme, caxis):
    cfg = dataclasses.replace(MODELS["euler3"], order=2)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 3, scheme=scheme)
    assert_parity(_run(cfg, w0, cfg.dt, 3, scheme=scheme, caxis=caxis), f_ref, TOL)


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 2), (4, 7, 3), (3, 16, 6)])
def test_forced_resident_shapes_and_ring_closure(shape):
    """Forced shapes (lines per block, segments, field groups) for both pass kinds; at CFL 8
    the window exceeds the segments, so the exact ring closure runs in shared memory."""
    for cfl in (1.0, 8.0):
        cfg = dataclasses.replace(W.SW_D2Q4, n_macro=(3, 3), n_sub=(3, 3), order=3, cfl=cfl)
        w0 = oracle_w0(cfg)
        f_ref = run_oracle(cfg, w0, cfg.dt, 3)
        f = _run(cfg, w0, cfg.dt, 3, shapes={7: shape, 8: shape}, caxis=0)
        assert_parity(f, f_ref, TOL, (shape, cfl))


def test_time_reversed_steps():
    cfg = dataclasses.replace(W.SW_D2Q4, n_macro=(3, 2), n_sub=(3, 4), order=3)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, -cfg.dt, 3)
    f = _run(cfg, w0, -cfg.dt, 3, caxis=0)
    assert_parity(f, f_ref, TOL, tol_pt=TOL_POINTWISE_REVERSED)


def test_equals_the_streaming_kernel():
    """The resident and the streaming kernel run the same operations: with the same launch
    shape they agree to rounding (the staged copy changes nothing in the arithmetic)."""
    cfg = dataclasses.replace(MODELS["shallow_water"], order=2)
    w0 = oracle_w0(cfg)
    sh = (2, 3, 2)
    a = _run(cfg, w0, cfg.dt, 4, resident=0, shapes={0: sh, 1: sh})
    b = _run(cfg, w0, cfg.dt, 4, resident=1, shapes={7: sh, 8: sh})
    assert rel_l2(b, a) <= 1e-15


@pytest.mark.parametrize("precision", [0, 1])
def test_euler_96cube_collision_on_x(precision):
    """3-D Euler D3Q6 at 8^3 macrocells x 4^3 subcells (96^3 points, 30 populations), the
    collision in the x pass and every pass line-resident, two steps against the oracle."""
    cfg = W.EULER_D3Q6.scaled(n_macro=(8, 8, 8))
    w0 = oracle_w0(cfg)
    f = _run(cfg, w0, cfg.dt, 2, precision=precision, caxis=0)
    assert_parity(f, run_oracle(cfg, w0, cfg.dt, 2), TOL)
