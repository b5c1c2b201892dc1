"""CPU oracle for the Volterra / spectral-recurrence TDSE solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: it is used by ``tests/``, by ``__graft_entry__.smoke()``
(to check one small GPU run) and by ``bench.py``'s CPU-baseline leg.

It is a plain, slow, FP64 restatement of the method of Kaye, Barnett and
Greengard (arXiv:2001.06113):
  * ``adams``    -- implicit Adams weights from the Vandermonde system
                    (Sec. 2.2, Table 1);
  * ``fields``   -- phi(t) = int_0^t A(s) ds (eq. phi), closed form for the
                    sin^2 pulse and Gauss-Legendre for a general A;
  * ``periodic`` -- the periodic marching scheme: direct O(M^2) DFT sums per
                    dimension (eq. ftperdisc), the trapezoidal recurrence
                    (eq. utrapkdisc), the n-th order implicit Adams scheme
                    (eq. uadamsk) and iterated Richardson start-up (Sec. 2.2).

It shares no code with the CUDA path; the only common module is ``synth``,
which samples input data and holds none of the method's arithmetic.
Every function is pinned by a ``-m "not gpu"`` test against closed forms,
textbook special cases or brute force (see ``tests/test_oracle_*.py``).
"""
from . import adams, fields, periodic  # noqa: F401
from .periodic import PeriodicOracle, rel_l2  # noqa: F401
