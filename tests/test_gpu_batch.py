"""Batched form: many independent meshes of uneven size, degree and model advanced by
one persistent launch per stage (optionally replayed from a CUDA graph).

Bars: every instance matches the FP64 oracle (relative L2 <= 1e-12); an instance gives
bitwise the same result alone and in a mix; graph replay equals direct launches bitwise.
"""
import dataclasses

import numpy as np
import pytest

from gpu_common import assert_parity, oracle_w0, run_oracle
from paper_1702_00169_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _mix():
    """Eight instances: 2-D SW/advection and 3-D Euler, degrees 1-4, ragged sizes."""
    return [
        dataclasses.replace(W.SW_D2Q4, n_macro=(3, 2), n_sub=(3, 5), order=3, seed=11),
        dataclasses.replace(W.SW_D2Q4, n_macro=(5, 5), n_sub=(2, 2), order=1, seed=12),
        dataclasses.replace(W.ADVECTION_D2Q4, n_macro=(4, 3), n_sub=(2, 3), order=2, seed=13),
        dataclasses.replace(W.SW_D2Q4, n_macro=(2, 2), n_sub=(4, 4), order=4, seed=14, cfl=3.0),
        dataclasses.replace(W.EULER_D3Q6, n_macro=(2, 3, 2), n_sub=(2, 2, 3), order=2, seed=15),
        dataclasses.replace(W.ADVECTION_D2Q4, n_macro=(7, 1), n_sub=(1, 5), order=4, seed=16),
        dataclasses.replace(W.SW_D2Q4, n_macro=(1, 1), n_sub=(1, 2), order=2, seed=17),
        dataclasses.replace(W.EULER_D3Q6, dim=2, n_macro=(3, 2), n_sub=(2, 3), order=3, seed=18),
    ]


def _solvers(cfgs, stream=None):
    from paper_1702_00169_gb300 import pdg
    out = []
    for c in cfgs:
        s = pdg.solver_for(c, stream=stream)
        s.set_w(np.ascontiguousarray(oracle_w0(c).reshape(-1)))
        out.append(s)
    return out


def _f(s, c):
    return s.get_f().reshape((c.m, 2 * c.dim) + tuple(reversed(c.npoints_axis)))


def test_batch_matches_oracle_per_instance():
    from paper_1702_00169_gb300 import pdg
    cfgs = _mix()
    nsteps = [3, 4, 2, 5, 3, 0, 1, 4]
    sol = _solvers(cfgs)
    b = pdg.Batch(sol)
    b.step([c.dt for c in cfgs], nsteps)
    for s, c, k in zip(sol, cfgs, nsteps):
        f_ref = run_oracle(c, oracle_w0(c), c.dt, k)
        assert_parity(_f(s, c), f_ref, TOL, c)
    b.close()
    for s in sol:
        s.close()


def test_alone_and_in_the_mix_bitwise_and_graph_replay():
    from paper_1702_00169_gb300 import pdg
    cfgs = _mix()
    dts = [c.dt for c in cfgs]
    alone = []
    for c in cfgs:
        (s,) = _solvers([c])
        b = pdg.Batch([s])
        b.step([c.dt], [3])
        alone.append(_f(s, c).copy())
        b.close()
        s.close()
    sol = _solvers(cfgs)
    b = pdg.Batch(sol)
    b.step(dts, [3] * len(cfgs))
    for s, c, ref in zip(sol, cfgs, alone):
        np.testing.assert_array_equal(_f(s, c), ref)
    b.close()
    # graph replay: 2 x (3 steps) through a captured graph == the same launches without a graph
    sol_g = _solvers(cfgs)
    sol_d = _solvers(cfgs)
    bg, bd = pdg.Batch(sol_g), pdg.Batch(sol_d)
    for _ in range(2):
        bg.step(dts, [3] * len(cfgs), use_graph=True)
        bd.step(dts, [3] * len(cfgs), use_graph=False)
    for sg, sd, c in zip(sol_g, sol_d, cfgs):
        np.testing.assert_array_equal(_f(sg, c), _f(sd, c))
    bg.close()
    bd.close()
    for s in sol + sol_g + sol_d:
        s.close()


def test_batched_kernel_equals_single_kernel_with_same_shape():
    """A work item of the persistent kernel is one block of the single-mesh kernel: with the
    same launch shape on pdg_step (kinds 0/1) and in the batch (kinds 2/3) the results are
    bitwise equal."""
    from paper_1702_00169_gb300 import pdg
    c = dataclasses.replace(W.SW_D2Q4, n_macro=(3, 3), n_sub=(3, 3), order=3, seed=21)
    (s1,) = _solvers([c])
    (s2,) = _solvers([c])
    for kind in (0, 1):
        s1.set_launch(kind, 4, 3, 2)
        s2.set_launch(kind + 2, 4, 3, 2)
    s1.step(c.dt, 4)
    b = pdg.Batch([s2])
    b.step([c.dt], [4])
    b.close()
    np.testing.assert_array_equal(_f(s2, c), _f(s1, c))
    assert_parity(_f(s1, c), run_oracle(c, oracle_w0(c), c.dt, 4), TOL)
    s1.close()
    s2.close()


def test_autotuned_shapes_keep_parity():
    from paper_1702_00169_gb300 import pdg
    cfgs = _mix()[:5]
    sol = _solvers(cfgs)
    b = pdg.Batch(sol)
    b.autotune([c.dt for c in cfgs], reps=2)
    b.step([c.dt for c in cfgs], [3] * len(cfgs), use_graph=True)
    for s, c in zip(sol, cfgs):
        assert_parity(_f(s, c), run_oracle(c, oracle_w0(c), c.dt, 3), TOL)
    b.close()
    c = cfgs[0]
    s = sol[0]
    s.set_w(np.ascontiguousarray(oracle_w0(c).reshape(-1)))
    s.autotune(c.dt, reps=2)
    assert s.get_launch(0)[0] > 0 and s.get_launch(1)[0] > 0
    s.step(c.dt, 3)
    assert_parity(_f(s, c), run_oracle(c, oracle_w0(c), c.dt, 3), TOL)
    for s in sol:
        s.close()
