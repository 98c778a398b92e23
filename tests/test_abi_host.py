"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every
entry point declared in include/pdg.h, and validates arguments before touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

from golden_util import expr, rows

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pdg():
    from paper_1702_00169_gb300 import build as B
    if not os.path.exists(B.LIB):
        B.build()
    from paper_1702_00169_gb300 import pdg as P
    return P


def _declared():
    src = open(os.path.join(ROOT, "include", "pdg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pdg_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(pdg):
    names = _declared()
    assert len(names) >= 17
    for n in names:
        assert hasattr(pdg.lib, n), n
        assert n in pdg.EXPORTED, n


def test_create_mesh_validation(pdg):
    ctx = ctypes.c_void_p()
    nm = (ctypes.c_int * 3)(4, 4, 1)
    ns = (ctypes.c_int * 3)(2, 2, 1)
    assert pdg.pdg_create_mesh(ctypes.byref(ctx), 4, nm, ns, 2, None, 15, None) == pdg.PDG_ERR_ARG
    assert pdg.pdg_create_mesh(ctypes.byref(ctx), 2, nm, ns, 0, None, 3, None) == pdg.PDG_ERR_ARG
    assert pdg.pdg_create_mesh(ctypes.byref(ctx), 2, nm, ns, 5, None, 3, None) == pdg.PDG_ERR_ARG
    assert pdg.pdg_create_mesh(ctypes.byref(ctx), 2, nm, ns, 2, None, 1, None) == pdg.PDG_OK  # y: inflow axis
    assert pdg.pdg_destroy(ctx) == pdg.PDG_OK
    bad = (ctypes.c_int * 3)(0, 4, 1)
    assert pdg.pdg_create_mesh(ctypes.byref(ctx), 2, bad, ns, 2, None, 3, None) == pdg.PDG_ERR_ARG
    assert pdg.pdg_create_mesh(None, 2, nm, ns, 2, None, 3, None) == pdg.PDG_ERR_ARG
    assert pdg.pdg_create_mesh(ctypes.byref(ctx), 2, nm, ns, 2, None, 3, None) == pdg.PDG_OK
    assert pdg.pdg_destroy(ctx) == pdg.PDG_OK
    assert pdg.pdg_destroy(None) == pdg.PDG_OK


def test_model_validation_and_state_order(pdg):
    s = pdg.Solver(3, (2, 2, 2), (2, 2, 2), 2)
    with pytest.raises(pdg.PdgError) as e:
        s.set_model("shallow_water", 8.0)
    assert e.value.status == pdg.PDG_ERR_UNSUPPORTED
    for kw in ({"omega": 0.0}, {"omega": float("nan")}, {"theta": 1.5}):
        with pytest.raises(pdg.PdgError) as e:
            s.set_model("euler", 5.0, **kw)
        assert e.value.status == pdg.PDG_ERR_ARG
    with pytest.raises(pdg.PdgError) as e:
        s.set_model("euler", -1.0)
    assert e.value.status == pdg.PDG_ERR_ARG
    with pytest.raises(pdg.PdgError) as e:
        s.step(0.01, 1)
    assert e.value.status == pdg.PDG_ERR_STATE
    s.set_model("euler", 5.0)
    info = s.info()
    assert (info.m, info.nv, info.nfields) == (5, 6, 30)
    assert list(info.npts) == [12, 12, 12] and info.npoints == 12 ** 3
    with pytest.raises(pdg.PdgError) as e:
        s.set_w(np.zeros(7))
    assert e.value.status == pdg.PDG_ERR_ARG
    with pytest.raises(pdg.PdgError) as e:
        s.get_w()
    assert e.value.status == pdg.PDG_ERR_STATE
    s.close()


def test_points_match_gl_closed_form(pdg):
    """Library GL coordinates (its own quadrature) = cell h + (h/2)(1 + x^) with the
    textbook nodes of tests/golden/gauss_lobatto.txt."""
    for d in (1, 2, 3, 4):
        s = pdg.Solver(2, (3, 2), (2, 1), d, lengths=(1.5, 0.5))
        s.set_model("advection", 2.0, a=(1.0, 0.5))
        nodes = [expr(x) for dd, x, w in rows("gauss_lobatto.txt") if int(dd) == d]
        for a, (L, N) in enumerate(((1.5, 6), (0.5, 2))):
            h = L / N
            ref = np.array([c * h + 0.5 * h * (1 + x) for c in range(N) for x in nodes])
            np.testing.assert_allclose(s.points(a), ref, rtol=0, atol=4e-16 * L)
        s.close()


def test_line_coefficients_d1_golden(pdg):
    """E, q, beta computed by the library for d = 1, theta = 1/2, nu = 1 equal the hand
    derivation of tests/golden/line_d1_theta_half_nu1.txt."""
    g = {k: expr(v) for k, v in rows("line_d1_theta_half_nu1.txt")}
    s = pdg.Solver(1, (7,), (1,), 1)
    s.set_model("advection", 2.0, a=(0.5,))
    h = 1.0 / 7
    E, q, beta = s.line_coefs(0, h / (2 * 2.0))
    np.testing.assert_allclose(E, [[g["E00"], g["E01"]], [g["E10"], g["E11"]]], rtol=0, atol=2e-16)
    np.testing.assert_allclose(q, [g["g0"], g["g1"]], rtol=0, atol=2e-16)
    assert abs(beta - g["beta"]) < 2e-16
    s.close()


@pytest.mark.parametrize("d", [1, 2, 3, 4])
@pytest.mark.parametrize("nu,theta", [(1.0, 0.5), (2.0, 0.5), (5.0, 0.75), (1.0, 1.0)])
def test_line_coefficients_vs_oracle_bloch_zero_mode(pdg, d, nu, theta):
    """The per-cell operator of one CN step applied to one isolated periodic cell (N = 1,
    so x_{c-1} is the cell itself) equals the oracle's Bloch step at kappa = 0."""
    from oracle.transport import bloch_transport
    s = pdg.Solver(1, (1,), (1,), d)
    lam = 2.0
    s.set_model("advection", lam, a=(0.5,), theta=theta)
    delta = nu * 1.0 / (2 * lam)
    E, q, beta = s.line_coefs(0, delta)
    n = d + 1
    f = np.random.default_rng(d).standard_normal(n)
    # one cell ring: x = fn[n-1] solves x = alpha + beta x
    if theta > 0:
        za, zb = 1.0, (1 - theta) / theta
    else:
        za, zb = 0.0, 1.0
    alpha = (E @ f)[n - 1] + q[n - 1] * zb * f[n - 1]
    x = alpha / (1 - beta)
    fn = E @ f + q * (za * x + zb * f[n - 1])
    ref = bloch_transport(f, -1, +1, d, nu, theta)
    np.testing.assert_allclose(fn, ref, rtol=0, atol=1e-13)
    s.close()


def test_inflow_validation_host(pdg):
    s = pdg.Solver(2, (3, 2), (2, 2), 2, periodic=(False, True))
    with pytest.raises(pdg.PdgError) as e:
        s.set_inflow(0, np.zeros(4))
    assert e.value.status == pdg.PDG_ERR_STATE
    s.set_model("shallow_water", 8.0)
    for axis, n in ((1, 2 * 3 * 18), (0, 7)):   # periodic axis, wrong length
        with pytest.raises(pdg.PdgError) as e:
            s.set_inflow(axis, np.zeros(n))
        assert e.value.status == pdg.PDG_ERR_ARG
    s.close()


def test_d2q9_and_source_validation(pdg):
    """D2Q9 model checks and pdg_set_source argument checks (no device memory is touched:
    the gravity-only source allocates nothing)."""
    s3 = pdg.Solver(3, (2, 2, 2), (2, 2, 2), 1)
    with pytest.raises(pdg.PdgError) as e:
        s3.set_model("isothermal_d2q9", 1.0)
    assert e.value.status == pdg.PDG_ERR_UNSUPPORTED           # D2Q9 is 2-D
    s3.close()
    s = pdg.Solver(2, (2, 2), (2, 2), 2)
    with pytest.raises(pdg.PdgError) as e:
        s.set_source(gravity=(0.0, -1.0))
    assert e.value.status == pdg.PDG_ERR_STATE                 # no model yet
    with pytest.raises(pdg.PdgError) as e:
        s.set_model("isothermal_d2q9", 1.0, theta=0.0)
    assert e.value.status == pdg.PDG_ERR_UNSUPPORTED           # the diagonal form needs theta > 0
    s.set_model("isothermal_d2q9", 1.0)
    i = s.info()
    assert (i.m, i.nv, i.nfields, i.w_len, i.f_len) == (3, 9, 9, 3 * i.npoints, 9 * i.npoints)
    s.set_source(gravity=(0.0, -1.0))                          # accepted, nothing allocated
    with pytest.raises(pdg.PdgError) as e:
        s.set_source(gravity=(0.0, -1.0), theta=1.5)
    assert e.value.status == pdg.PDG_ERR_ARG
    with pytest.raises(pdg.PdgError) as e:
        s.set_source(K_s=-1.0)
    assert e.value.status == pdg.PDG_ERR_ARG
    with pytest.raises(pdg.PdgError) as e:
        s.set_source(gravity=(float("nan"), 0.0))
    assert e.value.status == pdg.PDG_ERR_ARG
    s.set_source()                                             # removes the source
    s.set_model("shallow_water", 8.0)
    with pytest.raises(pdg.PdgError) as e:
        s.set_source(gravity=(0.0, -1.0))
    assert e.value.status == pdg.PDG_ERR_UNSUPPORTED           # sources: D2Q9 only
    s.close()


def test_diagonal_launch_override_validation(pdg):
    s = pdg.Solver(2, (2, 2), (2, 2), 2)
    for bad in ((32, 8, 8), (520, 8, 8), (100, 8, 8), (256, 0, 8)):
        with pytest.raises(pdg.PdgError):
            s.set_launch(4, *bad)
    s.set_launch(4, 256, 40, 30)
    assert s.get_launch(4) == (256, 40, 30)
    s.set_launch(4, 0, 0, 0)
    assert s.get_launch(4) == (0, 0, 0)
    s.close()


def test_corner_launch_override_and_options(pdg):
    """Launch kind 5 (corner boxes) and the options, validated on the host."""
    s = pdg.Solver(3, (2, 2, 2), (2, 2, 2), 2)
    for bad in ((32, 8, 8), (520, 8, 8), (100, 8, 8), (256, 0, 8), (256, 8, 0)):
        with pytest.raises(pdg.PdgError):
            s.set_launch(5, *bad)
    s.set_launch(5, 256, 12, 7)
    assert s.get_launch(5) == (256, 12, 7)
    s.set_launch(5, 0, 0, 0)
    assert s.get_launch(5) == (0, 0, 0)
    # kind 6: the box alone (x, y, z may differ); threads stay as kind 5 set them
    for bad in ((0, 8, 8), (64, 0, 43), (64, 43, -1)):
        with pytest.raises(pdg.PdgError):
            s.set_launch(6, *bad)
    s.set_launch(5, 256, 12, 7)
    s.set_launch(6, 64, 43, 41)
    assert s.get_launch(6) == (64, 43, 41)
    assert s.get_launch(5) == (256, 64, 41)
    s.set_launch(6, 0, 0, 0)
    assert s.get_launch(6) == (0, 0, 0)
    assert s.get_launch(5)[0] == 256
    s.set_launch(5, 0, 0, 0)
    with pytest.raises(pdg.PdgError):
        s.set_launch(9, 1, 1, 1)
    s.set_option(pdg.PDG_OPT_GRAPH, 1)
    s.set_option(pdg.PDG_OPT_GRAPH, 0)
    s.set_option(pdg.PDG_OPT_COMPOSE_TT, 1)
    with pytest.raises(pdg.PdgError) as e:
        s.set_option(99, 1)
    assert e.value.status == pdg.PDG_ERR_ARG
    s.close()


def test_lattice_3d_model_checks_and_inflow_lengths(pdg):
    """D3Q19 on an inflow mesh: accepted; its inflow data hold the five populations
    entering through each face (2 x 5 x lines); M4^kin is refused for lattices only when
    stepping (it needs a backward diagonal sub-step)."""
    s = pdg.Solver(3, (2, 1, 1), (1, 2, 1), 1, periodic=(False, True, True))
    s.set_model("isothermal_d3q19", 1.0)
    i = s.info()
    assert (i.m, i.nv, i.nfields) == (4, 19, 19)
    lines = i.npoints // i.npts[0]
    with pytest.raises(pdg.PdgError) as e:
        s.set_inflow(0, np.zeros(2 * 4 * lines))                 # m entries: wrong for a lattice
    assert e.value.status == pdg.PDG_ERR_ARG
    s.close()
    s2 = pdg.Solver(2, (2, 2), (2, 2), 3)
    with pytest.raises(pdg.PdgError) as e:
        s2.set_model("isothermal_d3q27", 1.0)                     # 3-D lattices need dim = 3
    assert e.value.status == pdg.PDG_ERR_UNSUPPORTED
    s2.close()


def test_server_host_paths(pdg):
    """Server calls that need no device: unknown ids, fault-injection arguments, lattice
    requests refused at submission."""
    import dataclasses
    from paper_1702_00169_gb300 import workloads as W
    assert pdg.pdg_debug_fail_allocs(-1) == pdg.PDG_ERR_ARG
    assert pdg.pdg_debug_fail_allocs(0) == pdg.PDG_OK
    srv = pdg.Server(1 << 20)
    with pytest.raises(pdg.PdgError) as e:
        srv.cancel(12345)
    assert e.value.status == pdg.PDG_ERR_STATE
    with pytest.raises(pdg.PdgError) as e:
        srv.result(12345, 4)
    assert e.value.status == pdg.PDG_ERR_STATE
    cfg = dataclasses.replace(W.D2Q9_ISO, n_macro=(1, 1), n_sub=(2, 2), order=1)
    with pytest.raises(pdg.PdgError) as e:
        srv.submit(cfg, np.zeros(cfg.m * cfg.npoints), 2, t_arrival=0.0)
    assert e.value.status == pdg.PDG_ERR_UNSUPPORTED
    assert srv.pending() == (0, 0)
    srv.close()


def test_tensor_core_precisions_only_for_corner_lattices(pdg):
    """PDG_PREC_TF32 / PDG_PREC_TF32_DFRES apply to the dense cell inverses of the corner
    sweeps (D3Q15 / D3Q27); every other model refuses them before allocating anything, and a
    refused call leaves the context without a model."""
    for dim, kind in ((2, "advection"), (2, "shallow_water"), (3, "euler"), (2, "isothermal_d2q9"),
                      (3, "isothermal_d3q19")):
        s = pdg.Solver(dim, (2,) * dim, (2,) * dim, 2)
        for prec in (pdg.PDG_PREC_TF32, pdg.PDG_PREC_TF32_DFRES):
            with pytest.raises(pdg.PdgError) as e:
                s.set_model(kind, 2.0, precision=prec)
            assert e.value.status == pdg.PDG_ERR_UNSUPPORTED
            assert "corner" in pdg.pdg_last_error(s.ctx).decode()
        with pytest.raises(pdg.PdgError) as e:
            s.set_model(kind, 2.0, precision=4)
        assert e.value.status == pdg.PDG_ERR_UNSUPPORTED
        s.close()
    assert pdg.PRECISION["tf32"] == pdg.PDG_PREC_TF32 == 2 and pdg.PRECISION["tf32_df"] == 3


def test_every_exported_status_function_catches_all_exceptions():
    """No C++ exception crosses the C ABI: every exported function that returns a status is a
    function-try-block whose handler maps the exception to a status (a failed host
    allocation to PDG_ERR_OOM)."""
    import glob
    import re
    csrc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1702_00169_gb300", "csrc")
    seen = set()
    for fn in glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cpp")):
        src = open(fn).read()
        for m in re.finditer(r'^(?:extern "C" )?int (pdg_[a-z_0-9]+)\(([^{;]*?)\)( try)? \{', src, re.M):
            name = m.group(1)
            if name.startswith(("pdg_internal_", "pdg_plan_", "pdg_launch_", "pdg_corner_", "pdg_diag_",
                                "pdg_batch_threads", "pdg_sm_count", "pdg_fault_take", "pdg_model_variant")) \
                    and name not in ("pdg_plan_line", "pdg_plan_sweep"):
                continue
            assert m.group(3), f"{os.path.basename(fn)}: {name} is not a function-try-block"
            seen.add(name)
    header = open(os.path.join(os.path.dirname(csrc), "..", "include", "pdg.h")).read()
    declared = set(re.findall(r'^int (pdg_[a-z_0-9]+)\(', header, re.M))
    assert declared <= seen, sorted(declared - seen)
