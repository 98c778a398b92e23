"""Helpers shared by the GPU parity tests: run a problem through the C ABI and
through the oracle on identical seeded inputs."""
import numpy as np

from oracle import models as OM
from oracle import scheme as OS
from oracle.dg import CartesianMesh

ORACLE_KIND = {"advection": OM.ADVECTION, "shallow_water": OM.SHALLOW_WATER, "euler": OM.EULER,
               "isothermal_d2q9": OM.ISOTHERMAL_D2Q9, "isothermal_d3q19": OM.ISOTHERMAL_D3Q19,
               "isothermal_d3q15": OM.ISOTHERMAL_D3Q15, "isothermal_d3q27": OM.ISOTHERMAL_D3Q27}


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def max_rel(a, b):
    """Largest pointwise difference, relative to the largest magnitude of the reference."""
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


# Pointwise bar of time-reversed runs (dt < 0).  The backward theta step is
# anti-dissipative (the inverse of the forward one, eq. (3.13)), so it amplifies rounding:
# the oracle alone, given the shallow-water parity case perturbed by one ulp, moves by up to
# 4.4e-12 max|f| after three backward steps (1.5e-13 to 4.4e-12 for degrees 1-4, against
# 4e-15 to 9e-15 forward).  Two correct FP64 evaluations that round differently therefore
# differ by that much pointwise; the relative L2 bar stays 1e-12.
TOL_POINTWISE_REVERSED = 1e-11
# The same for the double-float state: its unit roundoff is 100-160 times FP64's (double-word
# operations carry 3-5 u^2 bounds, u = 2^-24), so the amplified rounding reaches ~1e-10.
TOL_POINTWISE_REVERSED_DF = 1e-9


def assert_parity(got, ref, tol, what="", tol_pt=None):
    """The parity bar of a GPU result against the oracle, in two parts:
    the relative L2 error over the whole state (the stated tolerance), and every single
    value within tol * max|ref| of the oracle's (tol_pt * max|ref| when given), so that a
    few wrong values at tile or box starts cannot hide in the norm (a norm dilutes a local
    error by the square root of the state size)."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    assert got.shape == ref.shape or got.size == ref.size, (what, got.shape, ref.shape)
    got = got.reshape(ref.shape)
    assert np.all(np.isfinite(got)), (what, "non-finite values")
    e2 = rel_l2(got, ref)
    em = max_rel(got, ref)
    assert e2 <= tol, (what, "relative L2", e2, tol)
    tp = tol if tol_pt is None else tol_pt
    if em > tp:
        idx = np.unravel_index(int(np.argmax(np.abs(got - ref))), ref.shape)
        raise AssertionError((what, "pointwise", em, tp, "worst index", tuple(int(i) for i in idx)))
    return e2, em


def oracle_mesh(cfg):
    return CartesianMesh(cfg.dim, cfg.ncells, cfg.order, lengths=cfg.lengths[:cfg.dim])


def oracle_model(cfg):
    return OM.Model(ORACLE_KIND[cfg.kind], cfg.dim, cfg.lam, a=cfg.a[:cfg.dim], gravity=cfg.gravity,
                    gamma=cfg.gamma)


def oracle_w0(cfg):
    from paper_1702_00169_gb300 import workloads as W
    mesh = oracle_mesh(cfg)
    return W.initial_w(cfg, [mesh.coords1d(a) for a in range(cfg.dim)])


def run_oracle(cfg, w0, dt, nsteps, scheme="M2", method="bloch", omega=None, source=None):
    """source: keyword arguments of oracle.source.Source (and of Solver.set_source)."""
    from oracle.source import Source
    mesh = oracle_mesh(cfg)
    model = oracle_model(cfg)
    tr = OS.Transporter(mesh, model, theta=cfg.theta, method=method)
    om = cfg.omega if omega is None else omega
    src = None if source is None else Source(**source)
    return OS.run(OS.initial_state(model, w0), tr, model, dt, nsteps, om, scheme, source=src)


def run_gpu(cfg, w0, dt, nsteps, scheme="M2", launch=None, omega=None, stream=None, precision=0, source=None):
    from paper_1702_00169_gb300 import pdg
    import dataclasses
    c = cfg if omega is None else dataclasses.replace(cfg, omega=omega)
    s = pdg.solver_for(c, scheme=scheme, stream=stream, precision=precision)
    if source is not None:
        s.set_source(**source)
    if launch:
        for kind, shape in launch.items():
            s.set_launch(kind, *shape)
    s.set_w(np.ascontiguousarray(w0.reshape(-1)))
    s.step(dt, nsteps)
    f = s.get_f().reshape((cfg.groups, cfg.nv) + tuple(reversed(cfg.npoints_axis)))
    s.close()
    return f
