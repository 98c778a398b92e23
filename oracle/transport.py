"""Theta / Crank-Nicolson transport step (oracle; test infrastructure only).

Section 3.2, eq. (3.11) transport_cn: T_2(dt) = (I + dt/2 L_h)(I - dt/2 L_h)^{-1}.
Section 5.1 uses the theta-weighted form of the same step; with weight theta
and sub-step delta the new state solves

    (I - theta delta L_h) F^new = (I + (1 - theta) delta L_h) F^old,      (*)

theta = 1/2 being eq. (3.11).  Reading: eq. (4.2) crank_nicolson prints the
same system without the factors 1/2; (*) is used (it is eq. (3.11) for
theta = 1/2).  The periodic system is cyclic (the paper treats inflow
boundaries only, Section 2); (*) is solved exactly as the linear system it is.

Two independent routes:
  DirectTransport  sparse LU of (*) with the L_h assembled from eq. (3.7)
                   (the plain definition; tiny and medium meshes);
  bloch_transport  per-line Fourier (Bloch) closed form of (*) for an
                   axis-aligned velocity, derived by hand from eq. (3.7) on a
                   Cartesian cell (any size).  Derivation: with
                   K = Dm + w_0^{-1} e_0 e_0^T (Dm[j,i] = l_i'(x_j)), the
                   summation-by-parts identity of GL quadrature reduces
                   eq. (3.7) for v = +lambda e_a on line cell c to
                   d/dt f_c = -(2 lambda / h)(K f_c - w_0^{-1} e_0 f_{c-1,d});
                   for the Fourier mode exp(i kappa c), f_{c-1} -> exp(-i kappa) f_c.
                   v = -lambda e_a is the mirror image (points reversed).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .dg import assemble_transport
from .quadrature import gauss_lobatto, lagrange_derivative


class DirectTransport:
    """Solve (*) for one velocity v and sub-step delta with a sparse LU (SuperLU).

    On non-periodic axes the boundary data f^b enter through the fictitious cells of
    eq. (3.8) (d/dt f_R = 0): with the augmented unknowns (f, f_R) the theta step
    reduces to (I - theta delta L) f^new = (I + (1-theta) delta L) f^old
    + delta * bcoef * f^b.
    """

    def __init__(self, mesh, v, delta, theta=0.5):
        self.mesh = mesh
        self.delta = delta
        L, self.bcoef = assemble_transport(mesh, v, with_boundary=True)
        I = sp.identity(mesh.npoints, format="csr")
        self.A = (I - theta * delta * L).tocsc()
        self.B = (I + (1.0 - theta) * delta * L).tocsr()
        self.lu = spla.splu(self.A)

    def __call__(self, field, fb=None):
        rhs = self.B @ np.asarray(field, dtype=np.float64).reshape(-1)
        if fb is not None:
            rhs = rhs + self.delta * (self.bcoef * np.asarray(fb, dtype=np.float64)).reshape(-1)
        return self.lu.solve(rhs).reshape(np.shape(field))


def line_K(d):
    """K = Dm + w_0^{-1} e_0 e_0^T of the reduced 1-D cell operator (see module doc)."""
    x, w = gauss_lobatto(d)
    K = lagrange_derivative(x).copy()
    K[0, 0] += 1.0 / w[0]
    return K, w


def bloch_transport(field, axis_np, sign, d, nu, theta=0.5):
    """Solve (*) for v = sign * lambda e_a along numpy axis ``axis_np`` by Fourier modes.

    nu = 2 lambda delta / h.  For mode m (kappa = 2 pi m / N) the cell block obeys
      [I + theta nu (K - w0^{-1} e^{-i kappa} e_0 e_d^T)] f^new
          = [I - (1-theta) nu (K - w0^{-1} e^{-i kappa} e_0 e_d^T)] f^old.
    """
    n = d + 1
    K, w = line_K(d)
    f = np.moveaxis(np.asarray(field, dtype=np.float64), axis_np, -1)
    if sign < 0:
        f = f[..., ::-1]
    P = f.shape[-1]
    N = P // n
    assert N * n == P
    fc = f.reshape(f.shape[:-1] + (N, n))
    kappa = 2.0 * np.pi * np.arange(N) / N
    e0ed = np.zeros((n, n))
    e0ed[0, n - 1] = 1.0 / w[0]
    Kk = K[None, :, :] - np.exp(-1j * kappa)[:, None, None] * e0ed[None, :, :]
    I = np.eye(n)[None]
    Am = I + theta * nu * Kk
    Bm = I - (1.0 - theta) * nu * Kk
    Tm = np.linalg.solve(Am, Bm)                      # (N, n, n)
    Fh = np.fft.fft(fc, axis=-2)
    Fh = np.einsum("mij,...mj->...mi", Tm, Fh)
    fnew = np.real(np.fft.ifft(Fh, axis=-2)).reshape(f.shape)
    if sign < 0:
        fnew = fnew[..., ::-1]
    return np.ascontiguousarray(np.moveaxis(fnew, -1, axis_np))


def bloch_transport_2d(field, v, h, d, delta, theta=0.5):
    """Solve (*) on a periodic 2-D mesh for ANY constant velocity v = (v_x, v_y) by
    2-D Fourier modes over the cells (field shape (P_y, P_x), x last; h = (h_x, h_y)).

    On a Cartesian cell the terms of eq. (3.7) split by axis: the x part of the volume
    term involves Dm along x only, the faces normal to x carry (v_x n_x)^+- only, and the
    GL weight of the other direction cancels against omega_{L,i}.  Hence
    L_h = v_x-line operator (acting along every row of nodes) + v_y-line operator
    (along every column), each the 1-D reduction of ``bloch_transport``.  For the mode
    exp(i (kappa_x c_x + kappa_y c_y)), in the traversal orientation of each axis
    (negative components mirror that axis),
      K2 = nu_x (I (x) K_x(kappa_x)) + nu_y (K_y(kappa_y) (x) I),
      K_a(kappa) = K - w0^{-1} e^{-i kappa} e_0 e_d^T,  nu_a = 2 |v_a| delta / h_a,
    on the node vector p = i_y n + i_x, and [I + theta K2] f^new = [I - (1-theta) K2] f^old.
    A zero component drops its term; v = 0 is the identity.
    """
    n = d + 1
    K, w = line_K(d)
    f = np.asarray(field, dtype=np.float64)
    if v[0] < 0:
        f = f[:, ::-1]
    if v[1] < 0:
        f = f[::-1, :]
    Py, Px = f.shape
    Ny, Nx = Py // n, Px // n
    assert Ny * n == Py and Nx * n == Px
    nux = 2.0 * abs(v[0]) * delta / h[0]
    nuy = 2.0 * abs(v[1]) * delta / h[1]
    fc = f.reshape(Ny, n, Nx, n).transpose(0, 2, 1, 3).reshape(Ny, Nx, n * n)
    Fh = np.fft.fft2(fc, axes=(0, 1))
    e0ed = np.zeros((n, n))
    e0ed[0, n - 1] = 1.0 / w[0]
    I = np.eye(n)
    kx = 2.0 * np.pi * np.arange(Nx) / Nx
    ky = 2.0 * np.pi * np.arange(Ny) / Ny
    Kx = K[None] - np.exp(-1j * kx)[:, None, None] * e0ed[None]            # (Nx, n, n)
    Ky = K[None] - np.exp(-1j * ky)[:, None, None] * e0ed[None]            # (Ny, n, n)
    out = np.empty_like(Fh)
    Inn = np.eye(n * n)
    for jy in range(Ny):
        K2 = (nux * np.einsum("ab,mij->maibj", I, Kx).reshape(Nx, n * n, n * n)
              + nuy * np.kron(Ky[jy], I)[None])
        A = Inn[None] + theta * K2
        B = Inn[None] - (1.0 - theta) * K2
        out[jy] = np.linalg.solve(A, np.einsum("mpq,mq->mp", B, Fh[jy])[..., None])[..., 0]
    fn = np.real(np.fft.ifft2(out, axes=(0, 1)))
    fn = fn.reshape(Ny, Nx, n, n).transpose(0, 2, 1, 3).reshape(Py, Px)
    if v[1] < 0:
        fn = fn[::-1, :]
    if v[0] < 0:
        fn = fn[:, ::-1]
    return np.ascontiguousarray(fn)


def bloch_transport_planes(field, v, h, d, delta, theta=0.5):
    """Solve (*) on a periodic 3-D mesh for a velocity with exactly one zero component c
    (the edge velocities of D3Q19).  The operator acts along the other two axes only, so
    every plane of points normal to c is an independent 2-D problem, solved by
    ``bloch_transport_2d`` (field shape (P_z, P_y, P_x))."""
    v = np.asarray(v, dtype=np.float64)
    c = int(np.flatnonzero(v == 0)[0])
    a, b = [x for x in range(3) if x != c]
    f = np.asarray(field, dtype=np.float64)
    out = np.empty_like(f)
    npc = 2 - c                                  # numpy axis of geometric axis c
    for k in range(f.shape[npc]):
        sl = [slice(None)] * 3
        sl[npc] = k
        out[tuple(sl)] = bloch_transport_2d(f[tuple(sl)], (v[a], v[b]), (h[a], h[b]), d, delta, theta)
    return out


def bloch_transport_3d(field, v, h, d, delta, theta=0.5):
    """Solve (*) on a periodic 3-D mesh for ANY constant velocity v = (v_x, v_y, v_z) by 3-D
    Fourier modes over the cells (field shape (P_z, P_y, P_x), x last; h = (h_x, h_y, h_z)).

    The axis split of eq. (3.7) on a Cartesian cell (see ``bloch_transport_2d``) gives, for
    the mode exp(i (kappa_x c_x + kappa_y c_y + kappa_z c_z)) in the traversal orientation of
    each axis (negative components mirror that axis), on the node vector
    p = (i_z n + i_y) n + i_x,
      K3 = nu_x (I (x) I (x) K_x) + nu_y (I (x) K_y (x) I) + nu_z (K_z (x) I (x) I),
    K_a = K - w0^{-1} e^{-i kappa_a} e_0 e_d^T, nu_a = 2 |v_a| delta / h_a, and
    [I + theta K3] f^new = [I - (1-theta) K3] f^old.  Zero components drop their term.
    This is the form of the corner velocities lambda (+-1, +-1, +-1) of D3Q15 / D3Q27."""
    n = d + 1
    K, w = line_K(d)
    f = np.asarray(field, dtype=np.float64)
    flips = [v[0] < 0, v[1] < 0, v[2] < 0]
    for a, fl in enumerate(flips):
        if fl:
            f = np.flip(f, axis=2 - a)
    Pz, Py, Px = f.shape
    Nz, Ny, Nx = Pz // n, Py // n, Px // n
    assert Nz * n == Pz and Ny * n == Py and Nx * n == Px
    nu = [2.0 * abs(v[a]) * delta / h[a] for a in range(3)]
    nn = n ** 3
    fc = f.reshape(Nz, n, Ny, n, Nx, n).transpose(0, 2, 4, 1, 3, 5).reshape(Nz, Ny, Nx, nn)
    Fh = np.fft.fftn(fc, axes=(0, 1, 2))
    e0ed = np.zeros((n, n))
    e0ed[0, n - 1] = 1.0 / w[0]
    I = np.eye(n)
    I2 = np.eye(n * n)

    def Kmodes(N):
        kap = 2.0 * np.pi * np.arange(N) / N
        return K[None] - np.exp(-1j * kap)[:, None, None] * e0ed[None]   # (N, n, n)

    Kx, Ky, Kz = Kmodes(Nx), Kmodes(Ny), Kmodes(Nz)
    Tx = np.stack([np.kron(I2, Kx[i]) for i in range(Nx)])                 # acts on i_x
    Ty = np.stack([np.kron(np.kron(I, Ky[i]), I) for i in range(Ny)])      # acts on i_y
    Tz = np.stack([np.kron(Kz[i], I2) for i in range(Nz)])                 # acts on i_z
    Inn = np.eye(nn)
    out = np.empty_like(Fh)
    for jz in range(Nz):
        for jy in range(Ny):
            K3 = nu[0] * Tx + (nu[1] * Ty[jy] + nu[2] * Tz[jz])[None]
            A = Inn[None] + theta * K3
            B = Inn[None] - (1.0 - theta) * K3
            rhs = np.einsum("mpq,mq->mp", B, Fh[jz, jy])
            out[jz, jy] = np.linalg.solve(A, rhs[..., None])[..., 0]
    fn = np.real(np.fft.ifftn(out, axes=(0, 1, 2)))
    fn = fn.reshape(Nz, Ny, Nx, n, n, n).transpose(0, 3, 1, 4, 2, 5).reshape(Pz, Py, Px)
    for a, fl in enumerate(flips):
        if fl:
            fn = np.flip(fn, axis=2 - a)
    return np.ascontiguousarray(fn)
