"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bar: relative L2 error <= 1e-12 over all populations (FP64 path), on seeded
synthetic inputs shared by both sides.  Sizes span several thread blocks, ragged
tails (line counts not divisible by the block shape, cells not divisible by
the segment count), both closure modes of the periodic recurrence (window and
full ring), every degree, every model, both schemes and theta != 1/2.
"""
import dataclasses

import numpy as np
import pytest

from gpu_common import TOL_POINTWISE_REVERSED, assert_parity, oracle_w0, rel_l2, run_gpu, run_oracle
from paper_1702_00169_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1702_00169_gb300 import pdg  # noqa: F401  (fails loudly if the library is missing)


def test_advection_d2q4_workload_full_size_direct_oracle():
    """8x8 macrocells x 4x4 subcells, d = 2, 10 steps: oracle = sparse LU of eq. (3.7)."""
    cfg = W.ADVECTION_D2Q4
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, cfg.steps, method="direct")
    f = run_gpu(cfg, w0, cfg.dt, cfg.steps)
    assert_parity(f, f_ref, TOL)
    assert np.max(np.abs(f - f_ref)) <= 1e-12 * np.max(np.abs(f_ref))


@pytest.mark.parametrize("order", [1, 2, 3, 4])
@pytest.mark.parametrize("cfl", [1.0, 4.0])
def test_shallow_water_orders_ragged(order, cfl):
    """SW D2Q4 on 3x2 macrocells x 3x5 subcells (ragged line/block counts), all degrees,
    CFL 1 (window closure) and CFL 4 (larger beta)."""
    cfg = dataclasses.replace(W.SW_D2Q4, n_macro=(3, 2), n_sub=(3, 5), order=order, cfl=cfl)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 6)
    f = run_gpu(cfg, w0, cfg.dt, 6)
    assert_parity(f, f_ref, TOL)


@pytest.mark.parametrize("shape", [(1, 1, 1), (8, 3, 2), (5, 7, 1), (3, 9, 4), (16, 1, 12)])
def test_launch_shapes_and_full_ring_closure(shape):
    """Forced launch shapes (lines per block, segments, field groups), including segments
    shorter than the window (full ring closure) at CFL 8."""
    cfg = dataclasses.replace(W.SW_D2Q4, n_macro=(3, 3), n_sub=(3, 3), order=3, cfl=8.0)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 4)
    f = run_gpu(cfg, w0, cfg.dt, 4, launch={0: shape, 1: shape})
    assert_parity(f, f_ref, TOL)


@pytest.mark.parametrize("theta", [0.0, 0.75, 1.0])
def test_theta_variants(theta):
    """Weighted transport step (Section 5.1): explicit (theta = 0), 3/4 and implicit Euler.
    theta = 0 uses a small CFL (explicit upwind DG is only conditionally stable)."""
    cfl = 0.1 if theta == 0.0 else 2.0
    cfg = dataclasses.replace(W.ADVECTION_D2Q4, n_macro=(3, 4), n_sub=(2, 3), order=3, theta=theta, cfl=cfl)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 5)
    f = run_gpu(cfg, w0, cfg.dt, 5)
    assert_parity(f, f_ref, TOL)


@pytest.mark.parametrize("nsteps", [1, 2, 7])
def test_collapsed_scheme(nsteps):
    cfg = dataclasses.replace(W.SW_D2Q4, n_macro=(2, 3), n_sub=(4, 2), order=2)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, nsteps, scheme="M2_collapsed")
    f = run_gpu(cfg, w0, cfg.dt, nsteps, scheme="M2_collapsed")
    assert_parity(f, f_ref, TOL)


@pytest.mark.parametrize("order", [1, 2, 4])
def test_euler_d3q6_reduced(order):
    """3-D Euler D3Q6 (30 populations) on 2x3x2 macrocells x 3x2x3 subcells."""
    cfg = dataclasses.replace(W.EULER_D3Q6, n_macro=(2, 3, 2), n_sub=(3, 2, 3), order=order)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 3)
    f = run_gpu(cfg, w0, cfg.dt, 3)
    assert_parity(f, f_ref, TOL)


def test_euler_d2q4_and_d1():
    for dim, nm, ns in ((2, (3, 2), (2, 3)), (1, (5,), (3,))):
        cfg = dataclasses.replace(W.EULER_D3Q6, dim=dim, n_macro=nm, n_sub=ns, order=3)
        w0 = oracle_w0(cfg)
        f_ref = run_oracle(cfg, w0, cfg.dt, 4)
        f = run_gpu(cfg, w0, cfg.dt, 4)
        assert_parity(f, f_ref, TOL)


def test_advection_3d_and_omega_below_two():
    cfg = dataclasses.replace(W.ADVECTION_D2Q4, dim=3, n_macro=(2, 2, 3), n_sub=(2, 3, 2), order=2,
                              a=(1.0, -0.5, 0.25), lam=3.0)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 4, omega=1.6)
    f = run_gpu(cfg, w0, cfg.dt, 4, omega=1.6)
    assert_parity(f, f_ref, TOL)


def test_shallow_water_100_steps_reduced():
    """The SW workload's 100 steps on a reduced mesh (4x4 macrocells x 8x8 subcells, d = 3)."""
    cfg = W.SW_D2Q4.scaled(n_macro=(4, 4))
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, cfg.steps)
    f = run_gpu(cfg, w0, cfg.dt, cfg.steps)
    assert_parity(f, f_ref, TOL)


@pytest.mark.parametrize("order", [1, 2, 3, 4])
@pytest.mark.parametrize("shape", [None, (4, 3, 2), (2, 7, 1)])
def test_negative_time_step_reverse_recurrence(order, shape):
    """dt < 0 (time reversal): |beta| > 1 for several degrees, where the inflow recurrence
    runs upwind with ratio 1/beta; window and full-ring closures via forced shapes."""
    cfg = dataclasses.replace(W.SW_D2Q4, n_macro=(3, 2), n_sub=(3, 4), order=order)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, -cfg.dt, 3)
    f = run_gpu(cfg, w0, -cfg.dt, 3, launch=None if shape is None else {0: shape, 1: shape})
    assert_parity(f, f_ref, TOL, tol_pt=TOL_POINTWISE_REVERSED)


def test_time_symmetry_on_gpu():
    """eq. (3.13): with tau > 0 (omega < 2) the palindrome satisfies M2(-dt) M2(dt) = I."""
    from paper_1702_00169_gb300 import pdg
    cfg = dataclasses.replace(W.SW_D2Q4, n_macro=(3, 3), n_sub=(4, 4), order=3)
    w0 = oracle_w0(cfg)
    tau = cfg.dt
    om = lambda t: 2 * t / (2 * tau + t)
    s = pdg.solver_for(dataclasses.replace(cfg, omega=om(cfg.dt)))
    s.set_w(np.ascontiguousarray(w0.reshape(-1)))
    f0 = s.get_f().copy()
    s.step(cfg.dt, 1)
    s.set_model(cfg.kind, cfg.lam, gravity=cfg.gravity, omega=om(-cfg.dt))
    s.step(-cfg.dt, 1)
    f1 = s.get_f()
    s.close()
    assert rel_l2(f1, f0) <= 1e-13


def test_checkpoint_restore_bitwise():
    """get_f / set_f is a checkpoint: k + j steps == k steps, save, restore, j steps (bitwise)."""
    from paper_1702_00169_gb300 import pdg
    cfg = dataclasses.replace(W.SW_D2Q4, n_macro=(3, 2), n_sub=(4, 4), order=2)
    w0 = oracle_w0(cfg)
    s = pdg.solver_for(cfg)
    s.set_w(np.ascontiguousarray(w0.reshape(-1)))
    s.step(cfg.dt, 3)
    snap = s.get_f().copy()
    s.step(cfg.dt, 4)
    ref = s.get_f().copy()
    s.set_f(snap)
    s.step(cfg.dt, 4)
    again = s.get_f()
    s.close()
    np.testing.assert_array_equal(again, ref)


def test_device_buffers_and_moments():
    """set_w / get_w with device pointers (torch tensors); w = P f (eq. (2.2)) equals the
    oracle's moments of the same state."""
    import torch
    from paper_1702_00169_gb300 import pdg
    from oracle import models as OM
    cfg = dataclasses.replace(W.EULER_D3Q6, n_macro=(2, 2, 2), n_sub=(2, 3, 2), order=3)
    w0 = oracle_w0(cfg)
    stream = torch.cuda.current_stream()
    s = pdg.solver_for(cfg, stream=stream.cuda_stream)
    wd = torch.from_numpy(np.ascontiguousarray(w0.reshape(-1))).cuda()
    s.set_w(wd)
    s.step(cfg.dt, 2)
    out = torch.empty_like(wd)
    s.get_w(out)
    stream.synchronize()
    f = s.get_f().reshape((cfg.m, 6) + w0.shape[1:])
    s.close()
    np.testing.assert_allclose(out.cpu().numpy().reshape(w0.shape), np.sum(f, axis=1), rtol=0,
                               atol=1e-14 * np.max(np.abs(w0)))
    f_ref = run_oracle(cfg, w0, cfg.dt, 2)
    assert_parity(out.cpu().numpy().reshape(w0.shape), OM.Model(OM.EULER, 3, cfg.lam).moments(f_ref), TOL)


def test_degenerate_single_cell_lines():
    """One cell per axis (each line is a one-cell ring) and one GL line per block."""
    cfg = dataclasses.replace(W.SW_D2Q4, n_macro=(1, 1), n_sub=(1, 2), order=1)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 3, method="direct")
    f = run_gpu(cfg, w0, cfg.dt, 3)
    assert_parity(f, f_ref, TOL)


def test_zero_steps_is_identity_and_equilibrium_start():
    cfg = dataclasses.replace(W.SW_D2Q4, n_macro=(2, 2), n_sub=(2, 2), order=2)
    w0 = oracle_w0(cfg)
    f = run_gpu(cfg, w0, cfg.dt, 0)
    from gpu_common import oracle_model
    np.testing.assert_allclose(f, oracle_model(cfg).feq(w0), rtol=0, atol=1e-15)


def test_get_w_host_path_matches_moments():
    """pdg_get_w into host memory (device staging buffer + copy) equals sum_i f_{k,i} of the
    state read back with pdg_get_f, bitwise (same FP64 additions in the same order), on
    several calls in a row and two models."""
    from paper_1702_00169_gb300 import pdg
    for cfg in (dataclasses.replace(W.SW_D2Q4, n_macro=(3, 2), n_sub=(2, 3), order=3),
                dataclasses.replace(W.EULER_D3Q6, n_macro=(2, 2, 2), n_sub=(2, 2, 3), order=2)):
        w0 = oracle_w0(cfg)
        s = pdg.solver_for(cfg)
        s.set_w(np.ascontiguousarray(w0.reshape(-1)))
        for _ in range(3):
            s.step(cfg.dt, 2)
            w = s.get_w().reshape(w0.shape)
            f = s.get_f().reshape((cfg.m, 2 * cfg.dim) + w0.shape[1:])
            ref = f[:, 0].copy()
            for i in range(1, 2 * cfg.dim):
                ref = ref + f[:, i]
            np.testing.assert_allclose(w, ref, rtol=0, atol=1e-15 * np.max(np.abs(ref)))
        s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_composed_double_sweep_matches_two_sweeps(precision):
    """PDG_OPT_COMPOSE_TT: the composed T T sweep and two single sweeps are the same
    operator; both match the oracle (1e-12) and each other to rounding."""
    from paper_1702_00169_gb300 import pdg
    cfg = dataclasses.replace(W.SW_D2Q4, n_macro=(3, 4), n_sub=(5, 3), order=3)
    w0 = oracle_w0(cfg)
    out = []
    for compose in (1, 0):
        s = pdg.solver_for(cfg, precision=precision)
        s.set_option(pdg.PDG_OPT_COMPOSE_TT, compose)
        s.set_w(np.ascontiguousarray(w0.reshape(-1)))
        s.step(cfg.dt, 7)
        out.append(s.get_f().reshape((cfg.m, 4) + w0.shape[1:]))
        s.close()
    f_ref = run_oracle(cfg, w0, cfg.dt, 7)
    assert_parity(out[0], f_ref, TOL)
    assert_parity(out[1], f_ref, TOL)
    assert rel_l2(out[0], out[1]) <= 1e-13


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("nsteps", [1, 2, 5])
def test_m2kin_scheme(precision, nsteps):
    """M2^kin (Section 3.2) for shallow water and 3-D Euler against the oracle."""
    for cfg in (dataclasses.replace(W.SW_D2Q4, n_macro=(2, 3), n_sub=(4, 3), order=3),
                dataclasses.replace(W.EULER_D3Q6, n_macro=(2, 2, 2), n_sub=(2, 3, 2), order=2)):
        w0 = oracle_w0(cfg)
        f_ref = run_oracle(cfg, w0, cfg.dt, nsteps, scheme="M2_kin")
        f = run_gpu(cfg, w0, cfg.dt, nsteps, scheme="M2_kin", precision=precision)
        assert_parity(f, f_ref, TOL)


@pytest.mark.parametrize("shape", [None, (8, 4, 2)])
def test_balanced_line_split(shape):
    """A pass whose ceil(lines / lpb) blocks would leave SMs idle (700 y-lines, lpb 8 -> 88
    blocks): the lines are spread evenly over 152 blocks of 4-5 lines; parity unchanged."""
    cfg = dataclasses.replace(W.SW_D2Q4, n_macro=(70, 14), n_sub=(5, 5), order=1)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 3)
    f = run_gpu(cfg, w0, cfg.dt, 3, launch=None if shape is None else {0: shape, 1: shape})
    assert_parity(f, f_ref, TOL)
