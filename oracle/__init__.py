"""Plain FP64 CPU oracle for HEOM-2DVS (test infrastructure).

This package is the independent reference that the CUDA path is checked
against.  It is written from the paper (arXiv 2601.20550), step by step, in
double precision with dense matrices and a plain loop over hierarchy elements.
It shares no code with the library under ``paper_2601_20550_gb300``; the only
common module is ``workloads`` (seeded parameter sets, no arithmetic).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The product path never calls it.

Modules
-------
model : mode eigenbases, system operators, Drude/Pade bath coefficients and the
        hierarchy index set (Sec. II.A, II.B; Eqs. Total Hamiltonian .. Pade2).
heom  : right-hand side of Eq. HEOM_DB, classic RK4, equilibration, dipole
        kicks, traces, the 2D procedure and the 2D Fourier transforms
        (Sec. II.C; Eqs. R1, RFTIRI, echo, virtual-echo, 2D-rephasing,
        2D-nonrephasing, correlation-spectrum).
adjoint : the squared misfit of S_C against a reference spectrum and its gradient
        with respect to twelve model parameters, by central differences.

Parity status: every function is pinned by a test in tests/test_oracle_*.py
against closed forms, invariants, special cases or brute force; see the module
docstrings for which pin covers which function.
"""
