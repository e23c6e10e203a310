"""CPU FP64 oracle for the CBIE N-Mueller operator (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import this package.  It shares no code with the CUDA library.
"""
