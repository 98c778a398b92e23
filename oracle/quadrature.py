"""Gauss-Lobatto quadrature and the nodal Lagrange basis (oracle; test infrastructure only).

Section 3.1: the reference cell is ]-1,1[^D; its points and weights are tensor
products of the (d+1) one-dimensional Gauss-Lobatto (GL) points, eq. (3.3)
map_GL, and the basis functions are the Lagrange polynomials attached to those
points, eq. (3.4) interp_property.

Definition used here (textbook, e.g. Abramowitz & Stegun 25.4.32): for degree d
the d+1 GL nodes are -1, +1 and the d-1 roots of P_d'(x) (derivative of the
Legendre polynomial P_d); the weights are w_i = 2 / (d (d+1) P_d(x_i)^2).
"""
import numpy as np
from numpy.polynomial import legendre as _leg


def gauss_lobatto(d):
    """Return (x, w): the d+1 Gauss-Lobatto nodes on [-1,1] (ascending) and weights.

    Section 3.1, eq. (3.3) map_GL (reference points and weights).  d >= 1.
    """
    if d < 1:
        raise ValueError("Gauss-Lobatto needs degree d >= 1 (two end points)")
    c = np.zeros(d + 1)
    c[d] = 1.0                                   # P_d in the Legendre basis
    if d >= 2:
        inner = np.sort(np.real(_leg.legroots(_leg.legder(c))))
    else:
        inner = np.zeros(0)
    x = np.concatenate(([-1.0], inner, [1.0]))
    pd = _leg.legval(x, c)
    w = 2.0 / (d * (d + 1) * pd * pd)
    return x, w


def lagrange_derivative(x):
    """D[j, i] = l_i'(x_j): derivative of the i-th Lagrange polynomial at node j.

    Section 3.1 (basis functions with phi_i(x_j) = delta_ij, eq. (3.4)).  Plain
    product-rule formula:  l_i'(x) = sum_{k != i} 1/(x_i - x_k)
    prod_{m != i,k} (x - x_m)/(x_i - x_m).
    """
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            s = 0.0
            for k in range(n):
                if k == i:
                    continue
                p = 1.0 / (x[i] - x[k])
                for m in range(n):
                    if m == i or m == k:
                        continue
                    p *= (x[j] - x[m]) / (x[i] - x[m])
                s += p
            D[j, i] = s
    return D


def lagrange_eval(x, i, t):
    """Value of the i-th Lagrange polynomial on nodes x at points t."""
    t = np.asarray(t, dtype=np.float64)
    out = np.ones_like(t)
    for m in range(len(x)):
        if m != i:
            out = out * (t - x[m]) / (x[i] - x[m])
    return out
