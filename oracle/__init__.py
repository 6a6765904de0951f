"""CPU oracle for alias-table construction and sampling (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never uses it.
"""
