"""FP64 CPU oracle for the variable-order fractional wave solver.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import, call or
execute anything in this package.  The product path (the CUDA library and its
Python binding) never routes through it and never falls back to it.

Everything here is a plain, slow, obviously-correct restatement of the
equations of arXiv 2311.13049 in float64 NumPy; each function names the
passage it follows.  It shares no code with the CUDA path.
"""
from .vofl_oracle import *  # noqa: F401,F403
from .vofl_oracle import __all__  # noqa: F401
