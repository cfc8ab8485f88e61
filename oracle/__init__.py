"""FP64 CPU oracle of the coupled LBM-PSM-DEM step (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg import
this package. Functions with no independent pin are listed as "parity unpinned" in the
oracle header comment of ``ledds_oracle.c``; currently every function has a pin in
``tests/test_oracle_*.py``.
"""
