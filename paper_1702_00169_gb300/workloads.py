"""Seeded synthetic workloads (configurations and initial macroscopic states).

This module holds no arithmetic of the scheme: only problem sizes and the
recipes of the initial states w^0, evaluated at point coordinates that the
caller supplies (each side computes its own Gauss-Lobatto coordinates).  It
is shared by the tests (which feed the same arrays to the oracle and to the
CUDA library) and by ``bench.py``.

Recipes (the paper prints no data for these workloads; all inputs are
synthetic and drawn from ``numpy.random.default_rng(seed)``):

* advection: a periodised Gaussian bump (sigma = 0.1, centre (1/2, ..., 1/2),
  3^D periodic images) plus 8 Fourier modes of amplitude 1e-2 with wave vectors
  drawn from {-4..4}^D minus 0 and phases from U[0, 2 pi).
* shallow water: h = 1 + 0.1 F, hu = hv = 0, F a sum of 16 Fourier modes
  (|k|_inf <= 4, N(0,1) amplitudes, U[0,2 pi) phases) scaled so that
  max |F| = 1 on a fixed uniform reference grid.
* Euler: rho = 1 + 0.05 F_rho, u_a = 0.1 F_a, p = 1, with independent fields
  built like F above (|k|_inf <= 2 in 3-D); w = (rho, rho u, E) with
  E = p/(gamma-1) + rho |u|^2 / 2.
* isothermal D2Q9 (the model of the paper's Euler-with-gravity test, without the
  source): rho = 1 + 0.05 F_rho, u_a = 0.05 F_a with independent fields built like
  F above; w = (rho, rho u_x, rho u_y); lambda = 1 (sound speed 1/sqrt(3); Mach number at
  most 0.05 sqrt(3 D) max|F_a|, about 0.1 on the workload grids).
* isothermal D3Q19, D3Q15, D3Q27 (the lattices of the paper's 3-D scaling runs): the
  same recipe in 3-D (|k|_inf <= 2), w = (rho, rho u).
"""
import math
from dataclasses import dataclass, field
from typing import Tuple

import numpy as np

KINDS = ("advection", "shallow_water", "euler", "isothermal_d2q9", "isothermal_d3q19", "isothermal_d3q15",
         "isothermal_d3q27")


@dataclass
class Config:
    name: str
    kind: str
    dim: int
    n_macro: Tuple[int, ...]
    n_sub: Tuple[int, ...]
    order: int
    lam: float
    steps: int
    seed: int
    a: Tuple[float, ...] = (0.0, 0.0, 0.0)
    gravity: float = 9.81
    gamma: float = 1.4
    theta: float = 0.5
    omega: float = 2.0
    cfl: float = 1.0
    lengths: Tuple[float, ...] = (1.0, 1.0, 1.0)

    @property
    def m(self):
        return {"advection": 1, "shallow_water": 3, "euler": self.dim + 2, "isothermal_d2q9": 3,
                "isothermal_d3q19": 4, "isothermal_d3q15": 4, "isothermal_d3q27": 4}[self.kind]

    @property
    def groups(self):
        """Leading axis of f: conserved variables (DnQ2n) or one set of nine (D2Q9)."""
        return 1 if self.kind.startswith("isothermal") else self.m

    @property
    def nv(self):
        """Populations per group: 2D (DnQ2n), 9 (D2Q9), 15 / 19 / 27 (D3Qq)."""
        return {"isothermal_d2q9": 9, "isothermal_d3q19": 19, "isothermal_d3q15": 15,
                "isothermal_d3q27": 27}.get(self.kind, 2 * self.dim)

    @property
    def ncells(self):
        return tuple(self.n_macro[a] * self.n_sub[a] for a in range(self.dim))

    @property
    def npoints_axis(self):
        return tuple(c * (self.order + 1) for c in self.ncells)

    @property
    def npoints(self):
        return int(np.prod(self.npoints_axis))

    @property
    def nfields(self):
        return self.groups * self.nv

    @property
    def dofs(self):
        """Kinetic degrees of freedom: one f value at one GL point."""
        return self.nfields * self.npoints

    @property
    def h(self):
        """Sub-cell edge (all axes have the same edge in these workloads)."""
        return min(self.lengths[a] / self.ncells[a] for a in range(self.dim))

    @property
    def dt(self):
        """Time step dt = cfl * h / lambda."""
        return self.cfl * self.h / self.lam

    def scaled(self, n_macro=None, n_sub=None, steps=None, name=None):
        import dataclasses
        return dataclasses.replace(
            self, n_macro=tuple(n_macro or self.n_macro), n_sub=tuple(n_sub or self.n_sub),
            steps=self.steps if steps is None else steps, name=name or self.name)


ADVECTION_D2Q4 = Config("advection_d2q4_8x8x4x4_d2", "advection", 2, (8, 8), (4, 4), 2,
                        lam=2.0, steps=10, seed=1, a=(1.0, 0.5, 0.0))
SW_D2Q4 = Config("shallow_water_d2q4_64x64x8x8_d3", "shallow_water", 2, (64, 64), (8, 8), 3,
                 lam=8.0, steps=100, seed=2)
EULER_D3Q6 = Config("euler_d3q6_32c3x4c3_d2", "euler", 3, (32, 32, 32), (4, 4, 4), 2,
                    lam=5.0, steps=10, seed=3)

D2Q9_ISO = Config("isothermal_d2q9_64x64x8x8_d3", "isothermal_d2q9", 2, (64, 64), (8, 8), 3,
                  lam=1.0, steps=20, seed=6)

D3Q19_ISO = Config("isothermal_d3q19_32c3x4c3_d2", "isothermal_d3q19", 3, (32, 32, 32), (4, 4, 4), 2,
                   lam=1.0, steps=10, seed=7)
D3Q15_ISO = Config("isothermal_d3q15_32c3x4c3_d2", "isothermal_d3q15", 3, (32, 32, 32), (4, 4, 4), 2,
                   lam=1.0, steps=4, seed=8)
D3Q27_ISO = Config("isothermal_d3q27_32c3x4c3_d2", "isothermal_d3q27", 3, (32, 32, 32), (4, 4, 4), 2,
                   lam=1.0, steps=4, seed=9)

CONFIGS = {c.name: c for c in (ADVECTION_D2Q4, SW_D2Q4, EULER_D3Q6, D2Q9_ISO, D3Q19_ISO, D3Q15_ISO, D3Q27_ISO)}


def _grid(coords):
    """Broadcastable coordinate arrays, numpy axis order (z, y, x) i.e. x last."""
    D = len(coords)
    out = []
    for a in range(D):
        shape = [1] * D
        shape[D - 1 - a] = len(coords[a])
        out.append(np.asarray(coords[a], dtype=np.float64).reshape(shape))
    return out


def _modes(rng, D, count, kmax):
    ks = []
    while len(ks) < count:
        k = rng.integers(-kmax, kmax + 1, size=D)
        if np.any(k != 0):
            ks.append(k)
    return np.array(ks, dtype=np.float64)


def _mode_sum(X, ks, amps, phases):
    """sum_j amps_j cos(2 pi k_j . x + phases_j) on the tensor grid X, evaluated as the real
    part of a rank-(number of modes) sum of separable complex exponentials (one matrix
    product), not point by point."""
    D = len(X)
    xs = [np.asarray(X[a]).reshape(-1) for a in range(D)]          # 1-D coordinates, axis a
    wj = amps * np.exp(1j * phases)
    Ea = [np.exp(2j * np.pi * np.outer(ks[:, a], xs[a])) for a in range(D)]   # (J, P_a)
    # A[j, rest] = w_j prod_{a >= 1} E_a[j, .] (numpy order: highest axis first)
    A = wj[:, None]
    for a in reversed(range(1, D)):
        A = (A[:, :, None] * Ea[a][:, None, :]).reshape(len(wj), -1)
    F = np.real(A.T @ Ea[0])                                        # (prod_{a>=1} P_a, P_0)
    shape = tuple(len(xs[a]) for a in reversed(range(D)))
    return F.reshape(shape)


def _normalised_field(rng, D, count, kmax, ref_pts):
    ks = _modes(rng, D, count, kmax)
    amps = rng.standard_normal(count)
    phases = rng.uniform(0.0, 2.0 * math.pi, count)
    ref = _grid([np.arange(ref_pts) / ref_pts] * D)
    scale = np.max(np.abs(_mode_sum(ref, ks, amps, phases)))
    return lambda X: _mode_sum(X, ks, amps / scale, phases)


def initial_w(cfg, coords):
    """w^0 of shape (m, *grid) (x last) at the tensor grid ``coords`` = [x, y(, z)]."""
    D = cfg.dim
    X = _grid(coords)
    shape = tuple(len(coords[a]) for a in reversed(range(D)))
    rng = np.random.default_rng(cfg.seed)
    if cfg.kind == "advection":
        sigma = 0.1
        # periodised Gaussian: the sum over the 3^D images factorises per axis
        g = 1.0
        for a in range(D):
            ga = sum(np.exp(-(X[a] - 0.5 - s) ** 2 / (2.0 * sigma * sigma)) for s in (-1.0, 0.0, 1.0))
            g = g * ga
        ks = _modes(rng, D, 8, 4)
        phases = rng.uniform(0.0, 2.0 * math.pi, 8)
        w = g + _mode_sum(X, ks, np.full(8, 1e-2), phases)
        return np.broadcast_to(w, shape)[None].astype(np.float64).copy()
    if cfg.kind == "shallow_water":
        F = _normalised_field(rng, D, 16, 4, 256)
        h = np.broadcast_to(1.0 + 0.1 * F(X), shape)
        z = np.zeros(shape)
        return np.stack([h, z, z.copy()]).astype(np.float64)
    if cfg.kind == "euler":
        kmax = 4 if D == 2 else 2
        ref = 256 if D == 2 else 48
        Fr = _normalised_field(rng, D, 16, kmax, ref)
        Fu = [_normalised_field(rng, D, 16, kmax, ref) for _ in range(D)]
        rho = np.broadcast_to(1.0 + 0.05 * Fr(X), shape)
        u = [np.broadcast_to(0.1 * Fu[a](X), shape) for a in range(D)]
        p = 1.0
        E = p / (cfg.gamma - 1.0) + 0.5 * rho * sum(ua * ua for ua in u)
        return np.stack([rho] + [rho * ua for ua in u] + [E]).astype(np.float64)
    if cfg.kind.startswith("isothermal"):
        kmax, ref = (4, 256) if D == 2 else (2, 48)
        Fr = _normalised_field(rng, D, 16, kmax, ref)
        Fu = [_normalised_field(rng, D, 16, kmax, ref) for _ in range(D)]
        rho = np.broadcast_to(1.0 + 0.05 * Fr(X), shape)
        u = [np.broadcast_to(0.05 * Fu[a](X), shape) for a in range(D)]
        return np.stack([rho] + [rho * ua for ua in u]).astype(np.float64)
    raise ValueError(cfg.kind)


def batched_instances(n=256, seed=4, m_range=(8, 96), n_sub=4, orders=(1, 2, 3, 4), kind="shallow_water"):
    """Independent shallow-water instances of the batched workload: macrocell grid M x M
    with M ~ U{m_range}, n_sub x n_sub subcells, degree ~ U{orders}; instance i has its
    own initial-state seed (1000 * seed + i); dt from CFL 1 per instance."""
    rng = np.random.default_rng(seed)
    base = SW_D2Q4 if kind == "shallow_water" else ADVECTION_D2Q4
    out = []
    for i in range(n):
        M = int(rng.integers(m_range[0], m_range[1] + 1))
        d = int(rng.choice(orders))
        out.append(base.scaled(n_macro=(M, M), n_sub=(n_sub, n_sub), name=f"{kind}_{i}_M{M}_d{d}"))
        import dataclasses
        out[-1] = dataclasses.replace(out[-1], order=d, seed=1000 * seed + i, steps=20)
    return out


def serving_requests(n=1000, seed=5, rate=200.0, m_range=(16, 128), n_sub=4, orders=(1, 2, 3, 4),
                     steps_range=(10, 1000)):
    """Seeded Poisson request stream of the serving workload: arrival times (s) with mean
    rate `rate`, each request a 2-D advection or shallow-water solve (50/50) on M x M
    macrocells (M ~ U{m_range}) x n_sub^2 subcells, degree ~ U{orders}, steps
    log-uniform in steps_range, dt at CFL 1.  Returns [(t_arrival, Config, nsteps)]."""
    import dataclasses
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += float(rng.exponential(1.0 / rate))
        kind = "advection" if rng.random() < 0.5 else "shallow_water"
        M = int(rng.integers(m_range[0], m_range[1] + 1))
        d = int(rng.choice(orders))
        lo, hi = np.log(steps_range[0]), np.log(steps_range[1])
        ns = int(round(float(np.exp(rng.uniform(lo, hi)))))
        base = ADVECTION_D2Q4 if kind == "advection" else SW_D2Q4
        cfg = dataclasses.replace(base.scaled(n_macro=(M, M), n_sub=(n_sub, n_sub), name=f"req{i}_{kind}_M{M}_d{d}"),
                                  order=d, seed=100000 * seed + i, steps=ns)
        out.append((t, cfg, ns))
    return out
