"""FP64 CPU oracle for the Yee FDTD update (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import this package.  It shares no code with the CUDA library.
"""
from .yee import YeeOracle, COMPONENTS  # noqa: F401
