"""The arithmetic of the tensor-core precision form, emulated on the CPU.

The dense cell solves x = B^-1 r of the wavefront sweeps (B = I + theta sum_a nu_a K_a, the
cell system of eq. (3.7) under the theta step of eq. (3.11), split by axis) run on the
tensor cores in TF32 (operands rounded to 10 explicit mantissa bits) with FP32
accumulation.  Two ways to recover FP64-level accuracy are measured here on the cell
systems of the corner boxes (D = 3) and of the tiles (D = 2):

* plain TF32 operands and repeated refinement x += B~^-1 (r - B x): 3 applications reach
  1e-10 and 4 reach 1e-12 (BF16: 4-5 and 5), each refinement an FP64 residual of
  1 + D n FMA per node through the Kronecker sum B, so the FP64 work of the residuals is at
  least that of the direct FP64 product (n^D FMA per node) for tiles and for boxes up to
  degree 2;
* each operand split into two TF32 parts, v = hi + lo, and the three products
  hi.hi + lo.hi + hi.lo accumulated in FP32 (what corner_tc_kernel does): one application
  is accurate to about 1e-6, and ONE refinement (residual in FP64, or in double-float)
  reaches about 1e-13.  The FP64 work per node is then 1 + D n FMA against n^D for the
  direct product (10 against 27 at degree 2, 13 against 64 at degree 3), and the
  double-float residual needs none.

The emulation rounds exactly as the kernel does (cvt.rna.tf32.f32: to nearest, ties away)
and accumulates in FP32 in the order of the MMA sequence, one product at a time; the
tensor cores may round their internal sums differently, which the GPU tests bound.
"""
import numpy as np
import pytest

from oracle.transport import line_K


def _round(x, bits):
    """Round to `bits` explicit mantissa bits, to nearest (ties to even); exponent unbounded."""
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    s = 2.0 ** (bits + 1)
    return np.ldexp(np.round(m * s) / s, e)


def _tf32(x):
    """FP32 value rounded to TF32 (10 explicit mantissa bits), to nearest, ties away."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return ((b + 0x1000) & 0xFFFFE000).astype(np.uint32).view(np.float32)


def _split(x64):
    hi = _tf32(np.asarray(x64).astype(np.float32))
    lo = _tf32((np.asarray(x64) - hi.astype(np.float64)).astype(np.float32))
    return hi, lo


def _tc_apply(Bh, Bl, r64):
    """Split products (r_hi, B_hi), (r_lo, B_hi), (r_hi, B_lo), FP32 accumulation in order."""
    rh, rl = _split(r64)
    acc = np.zeros((Bh.shape[0], r64.shape[1]), dtype=np.float32)
    for A, X in ((Bh, rh), (Bh, rl), (Bl, rh)):
        for k in range(A.shape[1]):
            acc = (acc + A[:, k:k + 1] * X[k:k + 1, :]).astype(np.float32)
    return acc.astype(np.float64)


def _df(x):
    """x rounded to a double-float pair (about 48 significant bits)."""
    hi = np.asarray(x).astype(np.float32)
    return hi.astype(np.float64) + (np.asarray(x) - hi.astype(np.float64)).astype(np.float32).astype(np.float64)


def _cell_system(d, D, nu=1.0, theta=0.5):
    K, _ = line_K(d)
    n = d + 1
    Ks = np.zeros((n ** D, n ** D))
    for a in range(D):
        f = [np.eye(n)] * D
        f[D - 1 - a] = K
        op = f[0]
        for g in f[1:]:
            op = np.kron(op, g)
        Ks += nu * op
    return np.eye(n ** D) + theta * Ks


def _rhs(n, D, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n ** D, 64)) * np.exp(rng.uniform(-3, 3, (1, 64)))


def _applications(B, R, bits, bar, max_it=12):
    X = np.linalg.solve(B, R)
    Bl = _round(np.linalg.inv(B), bits).astype(np.float32)
    x = np.zeros_like(R)
    for k in range(1, max_it + 1):
        res = R - B @ x                                          # FP64 residual
        x = x + (Bl @ _round(res, bits).astype(np.float32)).astype(np.float64)   # FP32 accumulation
        if np.max(np.abs(x - X)) <= bar * np.max(np.abs(X)):
            return k
    return None


@pytest.mark.parametrize("d,D", [(1, 3), (2, 3), (3, 3), (2, 2), (3, 2), (4, 2)])
@pytest.mark.parametrize("fmt,bits", [("tf32", 10), ("bf16", 7)])
def test_plain_low_precision_needs_several_refinements(d, D, fmt, bits):
    n = d + 1
    B = _cell_system(d, D)
    R = np.random.default_rng(10 * d + D).standard_normal((n ** D, 64))
    k10, k12 = _applications(B, R, bits, 1e-10), _applications(B, R, bits, 1e-12)
    assert k10 is not None and k12 is not None
    assert k10 >= (3 if fmt == "tf32" else 4) and k12 >= k10
    residual_fma = (k12 - 1) * (1 + D * n)                       # FP64 FMA per node (first residual is R)
    if (d, D) == (3, 3):
        assert 0.5 * n ** D <= residual_fma < n ** D, (k12, residual_fma)
    else:
        assert residual_fma >= n ** D, (k12, residual_fma, n ** D)


@pytest.mark.parametrize("d,D", [(1, 3), (2, 3), (3, 3), (2, 2), (3, 2)])
@pytest.mark.parametrize("nu,theta", [(1.0, 0.5), (2.0, 0.5), (1.0, 0.75)])
def test_split_tf32_with_one_refinement_reaches_fp64_level(d, D, nu, theta):
    n = d + 1
    B = _cell_system(d, D, nu, theta)
    Binv = np.linalg.inv(B)
    Bh, Bl = _split(Binv)
    R = _rhs(n, D, 100 * d + D)
    X = np.linalg.solve(B, R)
    scale = np.max(np.abs(X), axis=0)
    x1 = _tc_apply(Bh, Bl, R)
    e1 = np.max(np.abs(x1 - X) / scale)
    assert 1e-8 < e1 < 5e-6, e1                                  # the split product alone: FP32 level
    x_fp64 = x1 + _tc_apply(Bh, Bl, R - B @ x1)                  # residual in FP64
    x_df = x1 + _tc_apply(Bh, Bl, _df(R) - _df(B) @ x1)          # residual from double-float operands
    for x in (x_fp64, x_df):
        assert np.max(np.abs(x - X) / scale) <= 2e-12
    # FP64 work per node of the refined form against the direct FP64 product
    assert 1 + D * n < n ** D or (d, D) == (1, 2)


def test_dropping_a_split_term_is_caught():
    """Without the (hi, lo) cross term the split product is no better than plain TF32 and one
    refinement no longer reaches 1e-11: the three products are all needed."""
    d, D = 2, 3
    n = d + 1
    B = _cell_system(d, D)
    Bh, Bl = _split(np.linalg.inv(B))
    R = _rhs(n, D, 7)
    X = np.linalg.solve(B, R)
    scale = np.max(np.abs(X), axis=0)

    def two_terms(r64):
        rh, rl = _split(r64)
        return (Bh.astype(np.float64) @ rh + Bh.astype(np.float64) @ rl).astype(np.float32).astype(np.float64)

    x1 = two_terms(R)
    x2 = x1 + two_terms(R - B @ x1)
    assert np.max(np.abs(x2 - X) / scale) > 1e-11
