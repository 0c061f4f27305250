"""CPU oracle for the L1 Caputo time-marching schemes (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The product library never does.
"""
