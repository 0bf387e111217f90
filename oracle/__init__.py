"""CPU oracle for the NS / GS estimators (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg import this package.  The product library never does.
"""
