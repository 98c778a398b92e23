"""The pass schedule on the host (no GPU): pdg_get_schedule against Section 3.2's compositions.

pdg_step issues each composition as passes over the axes (line passes; the collision fused in
the pass of the last axis; diagonal sub-steps for the D2Q9 diagonals).  Transports of
different populations commute, so the schedule is correct when every class of populations
(each axis, and the diagonals) meets exactly the sequence of sub-steps and collisions the
composition defines, in order:

  M2(dt)        T(dt/2) C T(dt/2)
  collapsed     T(dt/2) C T(dt) C ... T(dt) C T(dt/2)            (Section 5.1)
  M2^kin(dt)    T(dt/4) C T(dt/2) C T(dt/4)
  M4^kin(dt)    M2^kin(g1 dt) M2^kin(g2 dt) M2^kin(g1 dt),  g1 = 1/(2 - 2^(1/3)), g2 = 1 - 2 g1

A transport is identified by its line plan (E[0][0] and beta, compared with pdg_plan_line for
the expected sub-step on that axis); a diagonal sub-step by its sub-step.  For D2Q9 the slot
bookkeeping is checked too: every diagonal sub-step reads the slot set the previous one wrote,
every collision reads the diagonals where they are, and a copy brings them home at the end
exactly when they ended in the scratch set.
"""
import os

import numpy as np
import pytest

T_OP, C_OP = 1, 2
HOME, SCRATCH = 5, 9                                  # D2Q9 slots of population 5


@pytest.fixture(scope="module")
def pdg():
    from paper_1702_00169_gb300 import build as B
    if not os.path.exists(B.LIB):
        B.build()
    from paper_1702_00169_gb300 import pdg as P
    return P


def _m2kin(dt):
    return [("T", 0.25 * dt), "C", ("T", 0.5 * dt), "C", ("T", 0.25 * dt)]


def expected(scheme, dt, nsteps):
    if scheme == "M2":
        return [e for _ in range(nsteps) for e in (("T", 0.5 * dt), "C", ("T", 0.5 * dt))]
    if scheme == "M2_collapsed":
        seq = [("T", 0.5 * dt)]
        for s in range(nsteps):
            seq += ["C", ("T", dt if s < nsteps - 1 else 0.5 * dt)]
        return seq
    if scheme == "M2_kin":
        return [e for _ in range(nsteps) for e in _m2kin(dt)]
    g1 = 1.0 / (2.0 - np.cbrt(2.0))
    g2 = 1.0 - 2.0 * g1
    return [e for _ in range(nsteps) for g in (g1, g2, g1) for e in _m2kin(g * dt)]


def classes_from_schedule(sched, dim, diagonal):
    """Per class (axis a, or 'diag'): the sequence of ('T', plan or sub-step) and 'C'."""
    ev = {a: [] for a in range(dim)}
    if diagonal:
        ev["diag"] = []
    for p in sched:
        if p["kind"] == 0:
            for op, plan in zip(p["ops"], p["plans"]):
                if op == T_OP:
                    ev[p["axis"]].append(("T", plan))
                else:
                    assert op == C_OP
                    for k in ev:
                        ev[k].append("C")
        elif p["kind"] == 1:
            ev["diag"].append(("T", p["ddelta"]))
    return ev


def check_line_class(pdg, got, exp, d, lam, h, theta):
    assert len(got) == len(exp), (got, exp)
    for g, e in zip(got, exp):
        if e == "C":
            assert g == "C"
            continue
        assert g != "C"
        r = pdg.plan_line(d, 2.0 * lam * e[1] / h, theta)
        E00, beta = g[1]
        assert E00 == pytest.approx(r["E"][0, 0], rel=1e-12, abs=1e-15)
        assert beta == pytest.approx(r["beta"], rel=1e-12, abs=1e-15)


def check_diag_class(got, exp):
    assert len(got) == len(exp), (got, exp)
    for g, e in zip(got, exp):
        assert (g == "C") == (e == "C")
        if e != "C":
            assert g[1] == pytest.approx(e[1], rel=1e-14)


def check_slots(sched):
    slot = HOME
    for p in sched:
        if p["kind"] == 1:
            assert p["slot"] == slot
            slot = SCRATCH if slot == HOME else HOME
        elif p["kind"] == 0 and C_OP in p["ops"]:
            assert p["slot"] == slot
        elif p["kind"] == 2:
            assert slot == SCRATCH
            slot = HOME
    assert slot == HOME
    assert sum(p["kind"] == 2 for p in sched) <= 1 and all(p["kind"] != 2 for p in sched[:-1])


CASES = [  # (dim, model, lambda, lengths, d, theta)
    (1, "advection", 2.0, (1.0,), 2, 0.5),
    (2, "shallow_water", 8.0, (1.0, 0.7), 3, 0.5),
    (3, "euler", 5.0, (1.0, 0.8, 1.3), 1, 0.75),
]


@pytest.mark.parametrize("dim,model,lam,lengths,d,theta", CASES, ids=[c[1] for c in CASES])
@pytest.mark.parametrize("scheme", ["M2", "M2_collapsed", "M2_kin", "M4_kin"])
@pytest.mark.parametrize("nsteps", [1, 2, 3])
def test_line_schedule_follows_the_composition(pdg, dim, model, lam, lengths, d, theta, scheme, nsteps):
    s = pdg.Solver(dim, (3,) * dim, (2,) * dim, d, lengths=lengths)
    kw = {"a": tuple([1.0, -0.5, 0.25][:dim])} if model == "advection" else {}
    s.set_model(model, lam, scheme=scheme, theta=theta, **kw)
    info = s.info()
    dt = 0.6 * min(info.h[a] for a in range(dim)) / lam
    sched = s.schedule(dt, nsteps)
    assert all(p["kind"] == 0 for p in sched)
    assert all(p["axis"] == dim - 1 for p in sched if C_OP in p["ops"])    # collision in the last-axis pass
    ev = classes_from_schedule(sched, dim, False)
    exp = expected(scheme, dt, nsteps)
    for a in range(dim):
        check_line_class(pdg, ev[a], exp, d, lam, info.h[a], theta)
    assert s.schedule(dt, 0) == []
    s.close()


@pytest.mark.parametrize("scheme", ["M2", "M2_collapsed", "M2_kin"])
@pytest.mark.parametrize("nsteps", [1, 2, 3, 4])
@pytest.mark.parametrize("source", [False, True])
def test_d2q9_schedule_diagonals_and_slots(pdg, scheme, nsteps, source):
    if source and scheme == "M2_kin":
        pytest.skip("sources are defined for M2 and the collapsed form")
    s = pdg.Solver(2, (3, 2), (2, 2), 2, lengths=(1.0, 0.6))
    lam, theta = 1.0, 0.5
    s.set_model("isothermal_d2q9", lam, scheme=scheme, theta=theta)
    if source:
        s.set_source(gravity=(0.0, -1.0))
    info = s.info()
    dt = 0.5 * min(info.h[0], info.h[1]) / lam
    sched = s.schedule(dt, nsteps)
    ev = classes_from_schedule(sched, 2, True)
    exp = expected(scheme, dt, nsteps)
    for a in range(2):
        check_line_class(pdg, ev[a], exp, 2, lam, info.h[a], theta)
    check_diag_class(ev["diag"], exp)
    check_slots(sched)
    for p in sched:
        if p["kind"] == 0 and C_OP in p["ops"]:
            assert p["sdelta"] == (pytest.approx(0.5 * dt) if source else 0.0)
    s.close()


def test_schedule_refusals_and_arguments(pdg):
    s = pdg.Solver(2, (3, 2), (2, 2), 2)
    with pytest.raises(pdg.PdgError) as e:
        s.schedule(0.01, 1)
    assert e.value.status == pdg.PDG_ERR_STATE                  # no model yet
    s.set_model("isothermal_d2q9", 1.0, scheme="M4_kin")
    with pytest.raises(pdg.PdgError) as e:
        s.schedule(0.01, 1)
    assert e.value.status == pdg.PDG_ERR_UNSUPPORTED            # backward sub-step on diagonals
    s.set_model("isothermal_d2q9", 1.0)
    with pytest.raises(pdg.PdgError) as e:
        s.schedule(-0.01, 1)
    assert e.value.status == pdg.PDG_ERR_UNSUPPORTED            # diagonal transport needs dt > 0
    for args in ((float("nan"), 1), (0.01, -1)):
        with pytest.raises(pdg.PdgError) as e:
            s.schedule(*args)
        assert e.value.status == pdg.PDG_ERR_ARG
    s.set_model("isothermal_d2q9", 1.0, scheme="M2_kin")
    with pytest.raises(pdg.PdgError) as e:
        s.set_source(gravity=(0.0, -1.0))
    assert e.value.status == pdg.PDG_ERR_UNSUPPORTED            # sources: M2 and collapsed only
    assert len(s.schedule(0.01, 2)) > 0
    s.close()


def _overcommit_refuses_huge_requests():
    try:
        with open("/proc/sys/vm/overcommit_memory") as fh:
            return fh.read().strip() in ("0", "2")
    except OSError:
        return False


@pytest.mark.skipif(not _overcommit_refuses_huge_requests(),
                    reason="needs a kernel that refuses allocations far beyond its memory")
@pytest.mark.parametrize("scheme", ["M2", "M4_kin"])
def test_pass_list_beyond_host_memory_fails_cleanly(pdg, scheme):
    """2^31 - 1 steps need tens of TB of pass list: the call returns PDG_ERR_OOM at once (no
    exception crosses the C ABI), and the context keeps working, its scheme unchanged."""
    s = pdg.Solver(3, (2, 2, 2), (2, 2, 2), 1)
    s.set_model("euler", 5.0, scheme=scheme)
    with pytest.raises(pdg.PdgError) as e:
        s.schedule(0.01, 2 ** 31 - 1)
    assert e.value.status == pdg.PDG_ERR_OOM
    sched = s.schedule(0.01, 2)
    ev = classes_from_schedule(sched, 3, False)
    info = s.info()
    for a in range(3):
        check_line_class(pdg, ev[a], expected(scheme, 0.01, 2), 1, 5.0, info.h[a], 0.5)
    s.close()


def test_failed_calls_leave_the_context_unchanged(pdg):
    """A refused pdg_set_model / pdg_set_source keeps the model, scheme and source that were
    set before (seen through pdg_get_info and the pass list)."""
    s = pdg.Solver(2, (3, 2), (2, 2), 2)
    s.set_model("isothermal_d2q9", 1.0, scheme="M2_collapsed", theta=0.75)
    s.set_source(gravity=(0.0, -1.0))
    info0 = bytes(s.info())
    sched0 = s.schedule(0.01, 3)
    for kw in ({"theta": 1.5}, {"omega": 0.0}, {"scheme": 7}, {"theta": 0.0}):
        with pytest.raises(pdg.PdgError):
            s.set_model("isothermal_d2q9", 1.0, **kw)
    with pytest.raises(pdg.PdgError):
        s.set_model("isothermal_d3q19", 1.0)                     # a 3-D lattice on a 2-D mesh
    assert bytes(s.info()) == info0
    assert s.schedule(0.01, 3) == sched0
    with pytest.raises(pdg.PdgError):
        s.set_source(gravity=(0.0, -1.0), theta=1.5)
    assert bytes(s.info()) == info0
    assert s.schedule(0.01, 3) == sched0
    s.close()


@pytest.mark.parametrize("dim,model,lam,lengths,d,theta", CASES[1:], ids=[c[1] for c in CASES[1:]])
@pytest.mark.parametrize("scheme", ["M2", "M2_collapsed", "M2_kin", "M4_kin"])
@pytest.mark.parametrize("nsteps", [1, 3])
def test_any_axis_can_carry_the_collision(pdg, dim, model, lam, lengths, d, theta, scheme, nsteps):
    """PDG_OPT_COLLISION_AXIS: transports along different axes commute, so the pass holding
    T(dt/2) C T(dt/2) may be any axis' pass; every class still meets the composition."""
    for ca in range(dim):
        s = pdg.Solver(dim, (3,) * dim, (2,) * dim, d, lengths=lengths)
        s.set_model(model, lam, scheme=scheme, theta=theta)
        s.set_option(pdg.PDG_OPT_COLLISION_AXIS, ca)
        info = s.info()
        dt = 0.6 * min(info.h[a] for a in range(dim)) / lam
        sched = s.schedule(dt, nsteps)
        assert all(p["axis"] == ca for p in sched if C_OP in p["ops"])
        assert any(C_OP in p["ops"] for p in sched)
        ev = classes_from_schedule(sched, dim, False)
        exp = expected(scheme, dt, nsteps)
        for a in range(dim):
            check_line_class(pdg, ev[a], exp, d, lam, info.h[a], theta)
        s.close()


def test_collision_axis_and_resident_options(pdg):
    s = pdg.Solver(3, (2, 2, 2), (2, 2, 2), 2)
    for bad in (-2, 3):
        with pytest.raises(pdg.PdgError) as e:
            s.set_option(pdg.PDG_OPT_COLLISION_AXIS, bad)
        assert e.value.status == pdg.PDG_ERR_ARG
    s.set_option(pdg.PDG_OPT_COLLISION_AXIS, 0)
    with pytest.raises(pdg.PdgError) as e:        # lattices keep the last axis
        s.set_model("isothermal_d3q19", 1.0)
    assert e.value.status == pdg.PDG_ERR_UNSUPPORTED
    s.set_option(pdg.PDG_OPT_COLLISION_AXIS, -1)
    s.set_model("isothermal_d3q19", 1.0)
    with pytest.raises(pdg.PdgError) as e:
        s.set_option(pdg.PDG_OPT_COLLISION_AXIS, 1)
    assert e.value.status == pdg.PDG_ERR_UNSUPPORTED
    s.set_option(pdg.PDG_OPT_COLLISION_AXIS, 2)   # the last axis itself is fine
    s.set_option(pdg.PDG_OPT_RESIDENT, 1)
    for bad in ((0, 1, 1), (1, 0, 1), (8, 8, 10)):
        with pytest.raises(pdg.PdgError):
            s.set_launch(7, *bad)
    s.set_launch(8, 1, 16, 10)
    assert s.get_launch(8) == (1, 16, 10)
    s.set_launch(8, 0, 0, 0)
    assert s.get_launch(8) == (0, 0, 0)
    s.close()


@pytest.mark.parametrize("model", ["euler", "isothermal_d2q9", "isothermal_d3q19"])
@pytest.mark.parametrize("scheme", ["M2", "M2_collapsed", "M2_kin", "M4_kin"])
def test_long_runs_repeat_one_step_pattern(pdg, model, scheme):
    """Long runs: the pass lists of 200 and 202 steps share their first and last passes, and
    their middle repeats with the passes of two steps (two, because the diagonal sub-steps
    alternate the slot set of the D2Q9 / D3Q19 diagonals).  The class sequences of the
    200-step list still follow the composition (the diagonal class included), and the D2Q9
    slots stay consistent."""
    dim = 2 if model == "isothermal_d2q9" else 3
    lattice = model.startswith("isothermal")
    if lattice and scheme == "M4_kin":
        pytest.skip("M4^kin is refused for diagonal velocities (test_schedule_refusals_and_arguments)")
    s = pdg.Solver(dim, (2,) * dim, (2,) * dim, 2, lengths=(1.0, 0.7, 1.3)[:dim])
    s.set_model(model, 1.0 if lattice else 5.0, scheme=scheme)
    dt, n = 0.01, 200
    a, b = s.schedule(dt, n), s.schedule(dt, n + 2)
    k = len(b) - len(a)
    assert k > 0 and len(a) > 8 * k
    edge = len(a) // 4
    assert b[:edge] == a[:edge] and b[-edge:] == a[-edge:]
    for i in range(2 * k, len(a) - 2 * k):
        assert a[i] == a[i + k], i
    for i in range(edge, len(b) - edge - k):
        assert b[i] == b[i + k], i
    ev = classes_from_schedule(a, dim, lattice)
    info = s.info()
    exp = expected(scheme, dt, n)
    for ax in range(dim):
        if not lattice:
            check_line_class(pdg, ev[ax], exp, 2, 5.0, info.h[ax], 0.5)
        else:
            assert [e == "C" for e in ev[ax]] == [e == "C" for e in exp]
    if lattice:
        check_diag_class(ev["diag"], exp)
    if model == "isothermal_d2q9":
        check_slots(a)
    s.close()
