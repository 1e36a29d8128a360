"""Oracle for the IRKGL16 second-order step: TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, obviously-correct CPU restatement of the
method in arXiv 2511.03655 (Sec. 2), written to check the CUDA library.
Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import, call or execute it.
The CUDA product path never routes through it and shares no code with it:
the coefficient tables, the step and the right-hand sides are derived and
written here independently.

Modules
-------
coeffs    Gauss-Legendre collocation coefficients c, b, A, alpha, beta and the
          floating-point forms mu, eta, nu (Sec. 2.2-2.4), in 80-digit
          ``decimal`` arithmetic, rounded once to FP64.
irkgl     The second-order step (Eqs. IRK_init2, IRK_FP2, stopping rule
          Eqs. Delta_n/stopping, update Eq. qnvn2 with compensated sums),
          generic over the scalar type (float, Decimal, Dual), plus the
          right-hand sides and Hamiltonians of the test problems.
cbind     ctypes binding to ``irkgl_oracle.c``, the same FP64 algorithm in
          plain C (scalar loops, no FMA contraction), used where the Python
          form would be too slow.

Parity status of each function is stated in its own docstring; functions
without an independent pin say "parity unpinned".
"""
