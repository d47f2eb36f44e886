"""CPU FP64 oracle of the generalized Block CG method. Test infrastructure only: used by tests/,
__graft_entry__.smoke() and bench.py's CPU-baseline leg, never by the product path."""
