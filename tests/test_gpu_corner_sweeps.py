"""GPU parity of the two organisations of the D3Q15 / D3Q27 corner pass (PDG_OPT_CORNER_SWEEP):
hyperplane sweeps of the whole region (default: one truncated start per population, the
cells of each hyperplane column + row + layer = s shared by the blocks of a cooperative
launch, faces passed through global face slots, a bounded counter wait per hyperplane) and
boxes with their own truncated starts.  Both solve the theta step of eq. (3.11) on the 3-D
recurrence of eq. (3.7); against the oracle's 3-D Fourier form every value is compared
(relative L2 and pointwise <= 1e-12)."""
import dataclasses

import numpy as np
import pytest

from gpu_common import assert_parity, oracle_w0, rel_l2, run_oracle
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


def _run(cfg, w0, nsteps, sweep, precision=0, scheme="M2"):
    from paper_1702_00169_gb300 import pdg
    s = pdg.solver_for(cfg, scheme=scheme, precision=precision)
    s.set_option(pdg.PDG_OPT_CORNER_SWEEP, sweep)
    s.set_w(np.ascontiguousarray(w0.reshape(-1)))
    s.step(cfg.dt, nsteps)
    f = s.get_f().reshape((cfg.groups, cfg.nv) + tuple(reversed(cfg.npoints_axis)))
    s.close()
    return f


@pytest.mark.parametrize("lat", ["q15", "q27"])
@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("precision", [0, 1])
def test_hyperplanes_and_boxes_match_the_oracle(lat, order, precision):
    """Ragged meshes, both sweeps, both precisions; hyperplanes and boxes agree to rounding."""
    cfg = _cfg(lat, (3, 2, 4), (2, 3, 2), order)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, 3)
    fh = _run(cfg, w0, 3, 1, precision)
    fb = _run(cfg, w0, 3, 0, precision)
    assert_parity(fh, f_ref, TOL, ("hyperplanes", lat, order, precision))
    assert_parity(fb, f_ref, TOL, ("boxes", lat, order, precision))
    assert rel_l2(fh, fb) <= (1e-14 if precision == 0 else 1e-12)


@pytest.mark.parametrize("theta,cfl,lengths", [(0.7, 1.0, (1.0, 0.7, 1.2)), (0.5, 2.0, (1.0, 0.7, 1.2)),
                                               (0.5, 1.0, (1.3, 1.0, 0.6))])
def test_hyperplanes_three_start_widths(theta, cfl, lengths):
    """Different Courant numbers per axis: three different start widths (region extents)."""
    cfg = _cfg("q15", (2, 2, 3), (3, 2, 2), 2, theta=theta, cfl=cfl, lengths=lengths)
    w0 = oracle_w0(cfg)
    assert_parity(_run(cfg, w0, 3, 1), run_oracle(cfg, w0, cfg.dt, 3), TOL)


@pytest.mark.parametrize("scheme,nsteps", [("M2_collapsed", 3), ("M2_kin", 2)])
def test_hyperplanes_schemes(scheme, nsteps):
    """The collapsed and kinetic schemes (Courant number 2 in the interior sub-steps: wider
    starts)."""
    cfg = _cfg("q27", (2, 3, 2), (2, 2, 2), 2)
    w0 = oracle_w0(cfg)
    f_ref = run_oracle(cfg, w0, cfg.dt, nsteps, scheme=scheme)
    assert_parity(_run(cfg, w0, nsteps, 1, scheme=scheme), f_ref, TOL)


@pytest.mark.parametrize("nm,ns", [((1, 1, 1), (1, 1, 1)), ((1, 2, 1), (1, 1, 3)), ((5, 1, 1), (1, 1, 1))])
def test_hyperplanes_tiny_and_flat_meshes(nm, ns):
    """Meshes smaller than the start width along some or all axes (the region wraps around
    the torus), and flat ones (few cells along one axis)."""
    cfg = _cfg("q27", nm, ns, 2)
    w0 = oracle_w0(cfg)
    assert_parity(_run(cfg, w0, 3, 1), run_oracle(cfg, w0, cfg.dt, 3), TOL)


_REF = {}


@pytest.mark.parametrize("precision", [0, 1])
def test_hyperplanes_at_scale(precision):
    """80 x 50 x 50 cells, d = 2 (D3Q15): regions of 96 x 66 x 66 cells, 226 hyperplanes, the
    largest one cut into 19 block ranges of several batches each.  One M2 step against the
    oracle's 3-D Fourier form, every value compared."""
    cfg = _cfg("q15", (20, 25, 25), (4, 2, 2), 2)
    w0 = oracle_w0(cfg)
    if "f" not in _REF:
        _REF["f"] = run_oracle(cfg, w0, cfg.dt, 1)
    assert_parity(_run(cfg, w0, 1, 1, precision), _REF["f"], TOL)


def test_hyperplane_wait_runs_out_and_the_context_stays_usable():
    """PDG_OPT_DEBUG_TC_STALL: every block waits for a count that no block reaches, with a
    bound of about 0.5 ms; the next synchronising call reports PDG_ERR_TIMEOUT once, and
    with the switch off the same context reproduces the oracle."""
    from paper_1702_00169_gb300 import pdg
    cfg = _cfg("q27", (2, 2, 2), (2, 2, 2), 2)
    w0 = oracle_w0(cfg)
    s = pdg.solver_for(cfg)
    s.set_w(np.ascontiguousarray(w0.reshape(-1)))
    s.set_option(pdg.PDG_OPT_DEBUG_TC_STALL, 1)
    s.step(cfg.dt, 1)                                    # asynchronous: the launch succeeds
    with pytest.raises(pdg.PdgError) as e:
        s.synchronize()
    assert e.value.status == pdg.PDG_ERR_TIMEOUT
    assert "hyperplane" in str(e.value)
    s.synchronize()                                      # reported once
    s.set_option(pdg.PDG_OPT_DEBUG_TC_STALL, 0)
    s.set_w(np.ascontiguousarray(w0.reshape(-1)))
    s.step(cfg.dt, 3)
    f = s.get_f().reshape((cfg.groups, cfg.nv) + tuple(reversed(cfg.npoints_axis)))
    s.close()
    assert_parity(f, run_oracle(cfg, w0, cfg.dt, 3), TOL)


def test_hyperplanes_graph_replay_and_checkpoint():
    """A captured CUDA graph (the cooperative launch and the counter reset inside it) gives
    bitwise the direct launches' result for the same calls (2 + 2 steps); 2 steps from the
    checkpoint after the first 2 give bitwise the same again."""
    from paper_1702_00169_gb300 import pdg
    cfg = _cfg("q27", (3, 2, 2), (2, 2, 3), 2)
    w0 = oracle_w0(cfg)
    out = {}
    for graph in (0, 1):
        s = pdg.solver_for(cfg)
        s.set_option(pdg.PDG_OPT_GRAPH, graph)
        s.set_w(np.ascontiguousarray(w0.reshape(-1)))
        s.step(cfg.dt, 2)
        ck = s.get_f()
        s.step(cfg.dt, 2)
        out[graph] = s.get_f()
        s.set_f(ck)
        s.step(cfg.dt, 2)
        out[graph + 2] = s.get_f()
        s.close()
    np.testing.assert_array_equal(out[1], out[0])
    np.testing.assert_array_equal(out[2], out[0])
    np.testing.assert_array_equal(out[3], out[0])
