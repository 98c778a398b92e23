"""Full-size parity: the benchmark workloads at their real sizes, in the launch
configuration bench.py times (autotuned shapes), against the oracle where it can
follow (a few steps through the per-line Bloch solver) and through properties that
hold at any size otherwise.  The two precisions are both checked."""
import numpy as np
import pytest

from gpu_common import assert_parity, oracle_mesh, oracle_w0, rel_l2, run_oracle
from paper_1702_00169_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _solver(cfg, precision, w0):
    from paper_1702_00169_gb300 import pdg
    s = pdg.solver_for(cfg, precision=precision)
    s.set_w(np.ascontiguousarray(w0.reshape(-1)))
    s.autotune(cfg.dt, reps=2)
    return s


@pytest.mark.parametrize("precision", [0, 1])
def test_shallow_water_full_size_two_steps_vs_oracle(precision):
    cfg = W.SW_D2Q4                                  # 2048 x 2048 points, 12 populations
    w0 = oracle_w0(cfg)
    s = _solver(cfg, precision, w0)
    s.step(cfg.dt, 2)
    f = s.get_f().reshape((cfg.m, 4) + w0.shape[1:])
    s.close()
    f_ref = run_oracle(cfg, w0, cfg.dt, 2)
    assert_parity(f, f_ref, TOL)


@pytest.mark.parametrize("precision", [0, 1])
def test_shallow_water_full_size_100_steps_properties(precision):
    """The workload's 100 steps at full size: the quadrature-weighted totals of w are
    conserved to round-off and the state stays finite; a constant equilibrium state is
    a fixed point (L_h 1 = 0, C f^eq = f^eq)."""
    cfg = W.SW_D2Q4
    mesh = oracle_mesh(cfg)
    M = mesh.mass_weights()
    w0 = oracle_w0(cfg)
    s = _solver(cfg, precision, w0)
    s.step(cfg.dt, cfg.steps)
    w = s.get_w().reshape(w0.shape)
    assert np.all(np.isfinite(w))
    for k in range(cfg.m):
        t0, t1 = np.sum(M * w0[k]), np.sum(M * w[k])
        assert abs(t1 - t0) <= 1e-12 * np.sum(M * np.abs(w0[k])) + 1e-15
    wc = np.stack([np.full(w0.shape[1:], 1.05), np.full(w0.shape[1:], 0.1), np.full(w0.shape[1:], -0.05)])
    s.set_w(np.ascontiguousarray(wc.reshape(-1)))
    f0 = s.get_f().copy()
    s.step(cfg.dt, 5)
    assert rel_l2(s.get_f(), f0) <= 1e-13
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_euler_d3q6_8cube_macrocells_vs_oracle(precision):
    """3-D Euler D3Q6 at 8^3 macrocells x 4^3 subcells, d = 2 (96^3 points, 30 populations)."""
    cfg = W.EULER_D3Q6.scaled(n_macro=(8, 8, 8))
    w0 = oracle_w0(cfg)
    s = _solver(cfg, precision, w0)
    s.step(cfg.dt, 2)
    f = s.get_f().reshape((cfg.m, 6) + w0.shape[1:])
    s.close()
    assert_parity(f, run_oracle(cfg, w0, cfg.dt, 2), TOL)


def test_euler_d3q6_full_size_properties():
    """Full Euler workload (32^3 macrocells x 4^3 subcells: 384^3 points, 30 populations,
    13.6 GB): one step keeps the weighted totals of w and a finite state."""
    cfg = W.EULER_D3Q6
    from paper_1702_00169_gb300 import pdg
    s = pdg.solver_for(cfg)
    coords = [s.points(a) for a in range(3)]
    w0 = W.initial_w(cfg, coords)
    s.set_w(np.ascontiguousarray(w0.reshape(-1)))
    s.step(cfg.dt, 1)
    w = s.get_w().reshape(w0.shape)
    s.close()
    mesh = oracle_mesh(cfg)
    wts = [mesh.weights1d(a) for a in range(3)]
    for k in range(cfg.m):
        def tot(a):
            return np.einsum("zyx,z,y,x->", a, wts[2], wts[1], wts[0])
        t0, t1 = tot(w0[k]), tot(w[k])
        assert np.all(np.isfinite(w[k]))
        assert abs(t1 - t0) <= 1e-12 * tot(np.abs(w0[k])) + 1e-15
