"""CPU oracle (test infrastructure): plain FP64 restatement of the paper's method.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import it.
"""
