"""Independent CPU FP64 oracle for the three-body tensor-product scheme.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  The CUDA library never calls it and shares no code with it.

It computes, plainly and slowly, what the GPU path computes quickly:

* ``grid``        -- periodic Fourier grid and the dense second-derivative
                     matrix D2, built two independent ways.
* ``hamiltonian`` -- masses -> kinetic coefficients (Sec. 2), the heavy-light
                     pair potential (Eq. definition_potential), the
                     Kronecker-sum Hamiltonian assembled explicitly (Eqs.
                     discretized_Schroedinger_equation_1D and Ham2D).
* ``sector``      -- the heavy-exchange parity sectors (Sec. 5.1, parity
                     selection rule).
* ``two_body``    -- well depth v0 from a two-body binding energy (Sec. 2,
                     generalized eigenvalue problem of Sec. 5.1).
* ``precond``     -- the shifted kinetic preconditioner as the Sylvester
                     equation of Sec. 4.2 (Bartels-Stewart via SciPy) and as a
                     dense linear solve.
* ``eig``         -- lowest eigenpairs: dense LAPACK eigh, or LOBPCG with
                     the Sylvester preconditioner for large grids, plus the
                     Weyl / Kato-Temple residual certificates.
* ``blocks``      -- the small block-linear-algebra definitions used by the
                     Jacobi-Davidson steps (Gram matrices, Rayleigh-Ritz,
                     projected correction equation, Sec. 4.1).

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
brute force, invariants or printed values of the paper (Table 1).
"""
