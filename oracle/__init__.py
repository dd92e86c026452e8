"""FP64 CPU oracle for the IOBM transport solve (test infrastructure only).

This package is the independent reference that the CUDA path is checked
against.  Only the test-suite, the smoke check and the CPU-baseline leg of the
benchmark may import it; the library itself never does, and it shares no code,
tables or constants with the CUDA path (both only draw their inputs from the
seeded generator in ``iobm_synth``).

What it computes, in plain FP64 NumPy/SciPy and in the paper's order:

* ``fd``        -- finite-difference second-derivative weights c_n (Eq. 1),
                  solved exactly from the Taylor conditions.
* ``modes``     -- lateral plane-wave modes (Eq. 19), the generalised Bloch
                  roots of the electrode recurrence (Eqs. 8.5-9, Appendix
                  Eq. A-08), their velocities, the per-mode self-energy
                  (Eqs. 17-1/17-2, 18-2) and the incident-wave source (Eq. 7).
* ``operator``  -- the truncated Hamiltonian H_T (Eqs. 2-4) with the local
                  potential and KB projectors, the dense real-space
                  self-energy blocks (Eq. 8), the assembled sparse matrix
                  E - H_T - H~ (Eqs. 7, 7-2) and the preconditioner P (Eq. 10).
* ``transport`` -- the exact solution of Eq. 7 for every incident channel by
                  sparse LU, projection of the solved waves onto electrode
                  channels (Eq. 6), T, R, Landauer conductance, and the adjoint
                  gradient dG/dV(r).

Parity status of every function is listed in its module docstring.
"""
