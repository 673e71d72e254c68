"""ORACLE -- test infrastructure (plain FP64 CPU rendering of the method).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may use
this package.  The product path never imports it.
"""
