"""CUDA-graph replay of pdg_step (PDG_OPT_GRAPH): the replayed launches are the direct ones,
so results are bitwise those of direct stepping; a new dt, a new step count or a changed
launch shape is recaptured; the lattice paths (diagonal, edge and corner sweeps, whose plans
and scratch are prepared before the capture) replay too."""
import dataclasses

import numpy as np
import pytest

from gpu_common import assert_parity, oracle_w0, run_oracle
from paper_1702_00169_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = {
    "advection": dataclasses.replace(W.ADVECTION_D2Q4, n_macro=(3, 2), n_sub=(3, 5), order=2),
    "shallow_water": dataclasses.replace(W.SW_D2Q4, n_macro=(2, 3), n_sub=(4, 3), order=3),
    "d2q9": dataclasses.replace(W.D2Q9_ISO, n_macro=(2, 3), n_sub=(3, 2), order=2),
    "d3q27": dataclasses.replace(W.D3Q27_ISO, n_macro=(2, 1, 2), n_sub=(1, 2, 1), order=1),
}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1702_00169_gb300 import pdg  # noqa: F401


def _solver(cfg, graph, scheme="M2"):
    from paper_1702_00169_gb300 import pdg
    s = pdg.solver_for(cfg, scheme=scheme)
    s.set_option(pdg.PDG_OPT_GRAPH, 1 if graph else 0)
    s.set_w(np.ascontiguousarray(oracle_w0(cfg).reshape(-1)))
    return s


@pytest.mark.parametrize("name", list(CASES))
def test_graph_replay_equals_direct(name):
    cfg = CASES[name]
    a, b = _solver(cfg, False), _solver(cfg, True)
    for dt, n in ((cfg.dt, 3), (cfg.dt, 3), (0.5 * cfg.dt, 2), (cfg.dt, 3)):   # replay, then recaptures
        a.step(dt, n)
        b.step(dt, n)
        np.testing.assert_array_equal(b.get_f(), a.get_f())
    a.close()
    b.close()


def test_graph_recaptures_after_launch_change_and_matches_oracle():
    from paper_1702_00169_gb300 import pdg
    cfg = CASES["shallow_water"]
    s = _solver(cfg, True, scheme="M2_kin")
    s.step(cfg.dt, 2)
    s.set_launch(0, 1, 1, 1)          # new shapes: the next step must not replay the old graph
    s.set_launch(1, 3, 2, 2)
    s.step(cfg.dt, 2)
    f = s.get_f().reshape((cfg.m, 4) + tuple(reversed(cfg.npoints_axis)))
    s.close()
    assert_parity(f, run_oracle(cfg, oracle_w0(cfg), cfg.dt, 4, scheme="M2_kin"), 1e-12)
