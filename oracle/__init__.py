"""FP64 CPU oracle for the Palindromic Discontinuous Galerkin (PDG) kinetic scheme.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of what the scheme computes (Badwaik et al., "Task-based
parallelization of an implicit kinetic scheme", arXiv:1702.00169).  Only the
test-suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import or run it.  The product
path (the CUDA library under ``paper_1702_00169_gb300/``) never imports it, and
it imports nothing from the product path.

Modules
-------
quadrature  Gauss-Lobatto nodes/weights and the Lagrange derivative matrix
            (Section 3.1, eq. (3.3) map_GL and the nodal basis).
dg          Generic D-dimensional assembly of the transport matrix L_h on an
            affine periodic Cartesian mesh, literally from eq. (3.7) DG_reduit
            with the cofactor formula eq. (3.6).
transport   The theta / Crank-Nicolson transport step (eq. (3.11)
            transport_cn, with the weight theta of Section 5.1), solved
            (a) directly with a sparse LU and (b) by a Bloch/FFT closed form
            (per line, per 2-D mode, per 3-D mode).
models      Velocity sets (DnQ2n, D2Q9, D3Q15, D3Q19, D3Q27), the moment map P
            (eq. (2.2)), the macroscopic fluxes and the equilibrium f_eq.
source      The source stage S_2 of M2^s (Section 3.2): gravity, penalisation.
scheme      Collision integrator (eq. (3.12) collision_cn) and the palindromic
            step M2 = T(dt/2) C(dt) T(dt/2) of Section 3.2, in the naive order.

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
textbook values, invariants or special cases (see each test's docstring).
"""
