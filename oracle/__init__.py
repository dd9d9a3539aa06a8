"""CPU oracle for the Chebyshev--Jacobi transform (test infrastructure only).

Only tests, the smoke check and the benchmark's CPU-baseline leg import this
package.  Functions whose parity is pinned, and by what, are listed in the
module docstrings; every function here is pinned by at least one
``-m "not gpu"`` test in ``tests/test_oracle_pins.py``.
"""
