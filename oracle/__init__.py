"""FP64 CPU oracle of the pencil-beam dose model (test infrastructure only).

Only tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py may
import this package.  The product path (paper_2512_18863_gb300) never does.
"""
