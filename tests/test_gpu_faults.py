"""Failure paths made on the host (no GPU fault, trap or hang): an injected allocation
failure (pdg_debug_fail_allocs: the library's next state allocations report out of
memory without calling the CUDA allocator), a request cancelled while waiting and one
cancelled while resident, and a lattice request refused at submission.  Bars: the failing
call returns PDG_ERR_OOM and its context stays usable; a failed or cancelled request
leaves the others' results bitwise unchanged (the same as when it was never submitted)."""
import dataclasses

import numpy as np
import pytest

from gpu_common import assert_parity, oracle_w0, run_oracle
from paper_1702_00169_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _disarm():
    from paper_1702_00169_gb300 import pdg
    pdg.pdg_debug_fail_allocs(0)
    yield
    pdg.pdg_debug_fail_allocs(0)


def _reqs():
    return [
        (dataclasses.replace(W.SW_D2Q4, n_macro=(3, 2), n_sub=(3, 5), order=3, seed=41), 6),
        (dataclasses.replace(W.ADVECTION_D2Q4, n_macro=(4, 3), n_sub=(2, 3), order=2, seed=42), 9),
        (dataclasses.replace(W.SW_D2Q4, n_macro=(2, 2), n_sub=(4, 4), order=4, seed=43), 5),
        (dataclasses.replace(W.EULER_D3Q6, n_macro=(2, 2, 2), n_sub=(2, 2, 2), order=2, seed=44), 4),
    ]


def _serve(reqs, budget, actions=()):
    """Submit all requests, then iterate; actions: {iteration: callable(server, ids)} run
    before that iteration.  Returns {index: result or status}."""
    from paper_1702_00169_gb300 import pdg
    srv = pdg.Server(budget, chunk_steps=2)
    ids = [srv.submit(c, oracle_w0(c), ns, t_arrival=0.0) for c, ns in reqs]
    actions = dict(actions)
    it = 0
    while True:
        if it in actions:
            actions[it](srv, ids)
        nw, nr = srv.pending()
        if nw == 0 and nr == 0:
            break
        srv.iterate()
        it += 1
        assert it < 1000
    out = {}
    for i, (c, _) in enumerate(reqs):
        try:
            out[i] = srv.result(ids[i], c.m * c.npoints)
        except pdg.PdgError as e:
            out[i] = e.status
    srv.close()
    return out


def test_injected_oom_leaves_context_usable():
    from paper_1702_00169_gb300 import pdg
    cfg = dataclasses.replace(W.SW_D2Q4, n_macro=(2, 3), n_sub=(2, 2), order=2)
    w0 = np.ascontiguousarray(oracle_w0(cfg).reshape(-1))
    s = pdg.solver_for(cfg)
    pdg.pdg_debug_fail_allocs(1)
    with pytest.raises(pdg.PdgError) as e:
        s.set_w(w0)
    assert e.value.status == pdg.PDG_ERR_OOM
    with pytest.raises(pdg.PdgError) as e:   # still no state: the failed call changed nothing
        s.step(cfg.dt, 1)
    assert e.value.status == pdg.PDG_ERR_STATE
    s.set_w(w0)                              # the injection was used up: this one succeeds
    s.step(cfg.dt, 3)
    f = s.get_f().reshape((cfg.m, 4) + tuple(reversed(cfg.npoints_axis)))
    s.close()
    assert_parity(f, run_oracle(cfg, oracle_w0(cfg), cfg.dt, 3), 1e-12)


def test_server_isolates_failed_admission():
    from paper_1702_00169_gb300 import pdg
    reqs = _reqs()
    budget = max(8 * c.nfields * c.npoints for c, _ in reqs)   # one resident request at a time
    ref = _serve(reqs, budget)
    # one injected failure before the first iteration: the first admission (request 0)
    # fails, the server admits request 1 in its place and serves the rest
    got = _serve(reqs, budget, actions={0: lambda srv, ids: pdg.pdg_debug_fail_allocs(1)})
    failed = [i for i in got if not isinstance(got[i], np.ndarray)]
    assert failed == [0] and got[0] == pdg.PDG_ERR_OOM
    for i in range(1, len(reqs)):
        np.testing.assert_array_equal(got[i], ref[i])


def test_server_cancel_waiting_and_resident():
    from paper_1702_00169_gb300 import pdg
    reqs = _reqs()[:2] + [
        (dataclasses.replace(W.SW_D2Q4, n_macro=(2, 2), n_sub=(2, 2), order=3, seed=45), 5),
        (dataclasses.replace(W.ADVECTION_D2Q4, n_macro=(3, 4), n_sub=(3, 2), order=2, seed=46), 7),
    ]
    size = [8 * c.nfields * c.npoints for c, _ in reqs]
    budget = size[0] + size[1]            # requests 0 and 1 resident, 2 and 3 waiting
    assert size[0] + size[1] + min(size[2], size[3]) > budget and max(size[2:]) <= budget
    ref = _serve(reqs, budget)

    def cancel(srv, ids):
        nw, nr = srv.pending()
        assert nr == 2 and nw == 2
        srv.cancel(ids[1])   # resident
        srv.cancel(ids[3])   # waiting
        with pytest.raises(pdg.PdgError) as e:
            srv.cancel(ids[3])
        assert e.value.status == pdg.PDG_ERR_STATE
    got = _serve(reqs, budget, actions={1: cancel})
    assert got[1] == pdg.PDG_ERR_STATE and got[3] == pdg.PDG_ERR_STATE
    for i in (0, 2):
        np.testing.assert_array_equal(got[i], ref[i])


def test_server_refuses_lattice_requests():
    from paper_1702_00169_gb300 import pdg
    cfg = dataclasses.replace(W.D2Q9_ISO, n_macro=(2, 2), n_sub=(2, 2), order=1)
    srv = pdg.Server(1 << 30)
    with pytest.raises(pdg.PdgError) as e:
        srv.submit(cfg, oracle_w0(cfg), 2)
    assert e.value.status == pdg.PDG_ERR_UNSUPPORTED
    srv.close()
