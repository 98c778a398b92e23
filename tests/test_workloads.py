"""The seeded input recipes (paper_1702_00169_gb300.workloads; CPU): determinism, the
separable mode-sum evaluation against a point-by-point sum, the normalisation, and the
value ranges and workload totals the recipes state."""
import dataclasses
import math

import numpy as np
import pytest

from oracle.dg import CartesianMesh
from paper_1702_00169_gb300 import workloads as W


def _coords(cfg):
    m = CartesianMesh(cfg.dim, cfg.ncells, cfg.order, lengths=cfg.lengths[:cfg.dim])
    return [m.coords1d(a) for a in range(cfg.dim)]


@pytest.mark.parametrize("D", [1, 2, 3])
def test_mode_sum_equals_the_pointwise_sum(D):
    rng = np.random.default_rng(40 + D)
    ks = W._modes(rng, D, 6, 3)
    amps, phases = rng.standard_normal(6), rng.uniform(0, 2 * math.pi, 6)
    xs = [np.sort(rng.uniform(0, 1, 5 + a)) for a in range(D)]
    got = W._mode_sum(W._grid(xs), ks, amps, phases)
    ref = np.zeros(tuple(len(xs[a]) for a in reversed(range(D))))
    for idx in np.ndindex(*ref.shape):
        x = [xs[a][idx[D - 1 - a]] for a in range(D)]
        ref[idx] = sum(amps[j] * math.cos(2 * math.pi * float(np.dot(ks[j], x)) + phases[j]) for j in range(6))
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)
    assert np.all(np.any(ks != 0, axis=1)) and np.all(np.abs(ks) <= 3)


def test_normalised_field_has_unit_maximum_on_its_reference_grid():
    for D, ref in ((2, 256), (3, 48)):
        F = W._normalised_field(np.random.default_rng(7), D, 16, 4 if D == 2 else 2, ref)
        grid = W._grid([np.arange(ref) / ref] * D)
        assert abs(np.max(np.abs(F(grid))) - 1.0) < 1e-12


def test_recipes_are_seeded_and_in_their_stated_ranges():
    small = {k: c.scaled(n_macro=tuple([4] * c.dim)) for k, c in W.CONFIGS.items()}
    for name, cfg in small.items():
        X = _coords(cfg)
        w = W.initial_w(cfg, X)
        assert w.shape == (cfg.m,) + tuple(reversed(cfg.npoints_axis))
        np.testing.assert_array_equal(w, W.initial_w(cfg, X))                 # seeded
        assert not np.array_equal(w, W.initial_w(dataclasses.replace(cfg, seed=cfg.seed + 1), X))
    sw = W.initial_w(small["shallow_water_d2q4_64x64x8x8_d3"], _coords(small["shallow_water_d2q4_64x64x8x8_d3"]))
    assert 0.89 < sw[0].min() and sw[0].max() < 1.11 and not sw[1:].any()
    cfg = small["euler_d3q6_32c3x4c3_d2"]
    e = W.initial_w(cfg, _coords(cfg))
    rho, mom, E = e[0], e[1:4], e[4]
    p = (cfg.gamma - 1.0) * (E - 0.5 * np.sum(mom * mom, axis=0) / rho)
    np.testing.assert_allclose(p, 1.0, rtol=0, atol=1e-13)
    assert 0.94 < rho.min() and rho.max() < 1.06
    for name in ("isothermal_d2q9_64x64x8x8_d3", "isothermal_d3q27_32c3x4c3_d2"):
        cfg = small[name]
        w = W.initial_w(cfg, _coords(cfg))
        u = w[1:] / w[0]
        mach = np.sqrt(np.sum(u * u, axis=0)).max() / (cfg.lam / math.sqrt(3.0))
        assert 0.94 < w[0].min() and w[0].max() < 1.06
        assert mach <= 0.05 * math.sqrt(3.0 * cfg.dim) * 1.05


def test_benchmark_grids_mach_number():
    cfg = W.D2Q9_ISO
    w = W.initial_w(cfg, _coords(cfg))
    u = w[1:] / w[0]
    assert np.sqrt(np.sum(u * u, axis=0)).max() * math.sqrt(3.0) == pytest.approx(0.101, abs=5e-4)


def test_batched_and_serving_streams():
    b = W.batched_instances()
    assert len(b) == 256 and len({c.seed for c in b}) == 256
    assert all(8 <= c.n_macro[0] <= 96 and c.n_macro[0] == c.n_macro[1] and c.order in (1, 2, 3, 4) for c in b)
    assert sum(c.dofs for c in b) == 2_248_980_480
    r = W.serving_requests()
    t = np.array([x[0] for x in r])
    assert len(r) == 1000 and np.all(np.diff(t) > 0)
    assert abs(np.diff(t).mean() * 200.0 - 1.0) < 0.1
    assert all(10 <= n <= 1000 and 16 <= c.n_macro[0] <= 128 for _, c, n in r)
    assert 0.45 < np.mean([c.kind == "advection" for _, c, _ in r]) < 0.55
