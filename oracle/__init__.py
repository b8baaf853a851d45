"""CPU FP64 oracle of the paper's method.  Test infrastructure only: imported by
tests/, __graft_entry__.smoke() and bench.py's CPU-baseline arm, never by the
product path."""
