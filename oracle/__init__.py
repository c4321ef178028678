"""CPU oracle of the 3DGS training step.  Test infrastructure only: used by
tests/, __graft_entry__.smoke() and bench.py's CPU baseline, never by the
product path."""
