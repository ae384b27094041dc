"""Plain, slow FP64 CPU oracle for the multi-body Nystrom operator of
"A Spectral Solver for Acoustic Scattering by Multiple Quasi-Axisymmetric
Structures" (Lai & Li).

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package; only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline and
reference legs) may call it.  It shares no code with the CUDA path: the only
common module is ``scenes`` (seeded input descriptors, no arithmetic of the
method).

Modules, each following the paper's steps in its order and notation:

* ``geometry``  -- surface map, tangents, normals, Jacobian; composite
                   Gauss-Legendre x trapezoidal nodes (Eq. para_quasi, Sec. 3.1).
* ``special``   -- complete elliptic integrals (AGM), half-integer Legendre
                   functions Q_{m-1/2} and their chi-derivatives (Eqs. modal0,
                   leg_recur, dleg_recur).
* ``modal``     -- modal Green's functions G_m^(k) and the source-derivative
                   modal kernels for k >= 0 (Eqs. modalgreen, conv, I1, Sec. 3.3),
                   and the Lagrange weights W_j (inverse DFT, Sec. 3.1).
* ``selfblock`` -- product-integration self block with adaptive outer
                   quadrature (Sec. 3.4; GGQ tables replaced, see header).
* ``operator``  -- the inter-body smooth rule (Eq. multi2part), the full
                   operator apply, the incident field and the far field.
* ``solve``     -- dense LU and restarted GMRES (Sec. 6, solver description).
* ``nearfield`` -- the layer potential of the interpolated density at
                   off-surface points as a plain adaptive 2-D integral (the
                   field near a surface, Sec. 6).

Parity status of every function is stated in its module header.
"""
