"""Serving with continuous batching (pdg_server_*).

Bars: every request's result equals the FP64 oracle (relative L2 <= 1e-12) and is
bitwise the same whether the request ran alone or mixed with others that arrived
while it was on the GPU; admission never exceeds the memory budget; time stamps are
ordered.
"""
import dataclasses

import numpy as np
import pytest

from gpu_common import assert_parity, oracle_model, oracle_w0, run_oracle
from paper_1702_00169_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _requests():
    base = [
        (dataclasses.replace(W.SW_D2Q4, n_macro=(3, 2), n_sub=(3, 5), order=3, seed=31), 7),
        (dataclasses.replace(W.ADVECTION_D2Q4, n_macro=(4, 3), n_sub=(2, 3), order=2, seed=32), 12),
        (dataclasses.replace(W.SW_D2Q4, n_macro=(2, 2), n_sub=(4, 4), order=4, seed=33), 3),
        (dataclasses.replace(W.SW_D2Q4, n_macro=(5, 5), n_sub=(2, 2), order=1, seed=34), 9),
        (dataclasses.replace(W.ADVECTION_D2Q4, n_macro=(7, 1), n_sub=(1, 5), order=4, seed=35), 5),
        (dataclasses.replace(W.EULER_D3Q6, n_macro=(2, 2, 2), n_sub=(2, 3, 2), order=2, seed=36), 4),
        (dataclasses.replace(W.SW_D2Q4, n_macro=(3, 3), n_sub=(2, 3), order=2, seed=37), 11),
    ]
    return base


def _w_len(cfg):
    return cfg.m * cfg.npoints


def _run(reqs, budget, chunk, stagger):
    """Submit requests (all at once, or one more after every iteration) and serve them all."""
    from paper_1702_00169_gb300 import pdg
    srv = pdg.Server(budget, chunk_steps=chunk)
    ids = {}
    pending = list(range(len(reqs)))
    while pending and not stagger:
        i = pending.pop(0)
        ids[srv.submit(reqs[i][0], oracle_w0(reqs[i][0]), reqs[i][1])] = i
    done = {}
    guard = 0
    while len(done) < len(reqs):
        if stagger and pending:
            i = pending.pop(0)
            ids[srv.submit(reqs[i][0], oracle_w0(reqs[i][0]), reqs[i][1])] = i
        srv.iterate()
        for rid, ta, tb, tc in srv.poll():
            assert ta <= tb <= tc
            done[ids[rid]] = srv.result(rid, _w_len(reqs[ids[rid]][0]))
        guard += 1
        assert guard < 1000
    st = srv.stats()
    srv.close()
    return done, st


def test_mixed_results_equal_alone_and_oracle():
    reqs = _requests()
    sizes = [8 * c.nfields * c.npoints for c, _ in reqs]
    budget = sum(sorted(sizes)[-3:])       # forces queueing: at most ~3 resident solves
    mixed, st = _run(reqs, budget, chunk=4, stagger=True)
    assert st["peak_bytes"] <= budget and st["completed"] == len(reqs)
    for i, (cfg, ns) in enumerate(reqs):
        alone, _ = _run([(cfg, ns)], budget, chunk=4, stagger=False)
        np.testing.assert_array_equal(mixed[i], alone[0])
        w_ref = oracle_model(cfg).moments(run_oracle(cfg, oracle_w0(cfg), cfg.dt, ns))
        assert_parity(mixed[i].reshape(w_ref.shape), w_ref, TOL)


def test_chunking_does_not_change_results():
    """Chunk boundaries only split the transport passes of consecutive steps: the same
    operator, evaluated as two sweeps instead of one composed sweep, so results agree
    to rounding."""
    reqs = _requests()[:4]
    big = 1 << 34
    a, _ = _run(reqs, big, chunk=1, stagger=False)
    b, _ = _run(reqs, big, chunk=100, stagger=True)
    for i in range(len(reqs)):
        assert np.linalg.norm(a[i] - b[i]) <= 1e-13 * np.linalg.norm(b[i])


def test_request_larger_than_budget_rejected():
    from paper_1702_00169_gb300 import pdg
    cfg, ns = _requests()[0]
    srv = pdg.Server(1024, chunk_steps=2)
    with pytest.raises(pdg.PdgError) as e:
        srv.submit(cfg, oracle_w0(cfg), ns)
    assert e.value.status == pdg.PDG_ERR_ARG
    srv.close()
