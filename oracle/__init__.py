"""Plain FP64 CPU oracle of the structure-preserving FDTD reduction.

TEST INFRASTRUCTURE ONLY.  This package restates, slowly and literally, what
the paper computes: the Yee system in the matrix form of Sec. II-A, the SPRIM
reduction of Sec. II-C with the expansion points and shifted solves of
Sec. IV, the projection of Eq. (R_and_Freduced), the perturbation of
Sec. III-A and the reduced leap-frog.  Only the test-suite,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  It shares no code with the CUDA library and never calls it.

Modules
-------
yee      -- grid assembly (D_eps, D_mu, D_sigma, K, B, C), full FDTD, CFL,
            discrete energy, dispersion relation of the uniform PEC box.
mor      -- expansion points, Krylov chains with sparse LU, SPRIM split and
            Gram-Schmidt, projection, SVD perturbation, reduced leap-frog,
            transfer functions and moments.
adjoint  -- discrete adjoint of the full FDTD recursion, gradient of a probe
            loss with respect to per-cell relative permittivity.

Parity status: every function is pinned by a ``-m "not gpu"`` test; none is
"parity unpinned".
"""
