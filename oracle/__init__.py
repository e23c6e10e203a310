"""CPU FP64 oracle for the CBIE N-Mueller operator (test infrastructure only).

``cbie``: the unaccelerated operator, RHS, solve and fields; ``ifgf``: the IFGF
approximation of the far-field sums, step by step; ``mie``: the Mie series.
Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import this package.  It shares no code with the CUDA library.
"""
