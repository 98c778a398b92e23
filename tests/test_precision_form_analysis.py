"""Why the precision form runs in double-float arithmetic and not on the tensor cores (CPU).

The tensor-core form would apply the cell inverse B^-1 in TF32 or BF16 (operands rounded to
10 or 7 mantissa bits, FP32 accumulation) and recover accuracy by refinement: x += low(B^-1)
(r - B x), the residual in FP64 through the Kronecker-sum B = I + theta sum_a nu_a K_a, which
costs 1 + D n FMA per node.  This test measures, for the cell systems of the sweeps (corner
boxes: D = 3, tiles: D = 2), how many low-precision applications that takes to reach the
1e-10 and 1e-12 bars (TF32: 3 and 4, BF16: 4-5 and 5), and checks the consequence: the FP64
residual work alone is at least the FP64 work of the direct product with B^-1 (n^D FMA per
node) for every tile and for boxes up to degree 2, so there the tensor cores cannot make the
refined form cheaper on the FP64 pipe, which is what bounds the FP64 path.  The exception is
the degree-3 box (64 FMA per node), where the TF32 residuals take 39 and the BF16 ones 52.
"""
import numpy as np
import pytest

from oracle.transport import line_K


def _round(x, bits):
    """Round to `bits` explicit mantissa bits, to nearest (ties to even); exponent unbounded."""
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    s = 2.0 ** (bits + 1)
    return np.ldexp(np.round(m * s) / s, e)


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
def test_refined_low_precision_costs_more_fp64_than_the_direct_product(d, D, fmt, bits):
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
