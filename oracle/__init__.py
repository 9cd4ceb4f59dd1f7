"""FP64 CPU oracle for the PDHG photoacoustic reconstruction hot path.

Test infrastructure only: the test-suite, the smoke check and the benchmark's
CPU-baseline / reference leg are its only users.  The CUDA library never imports,
links or runs it, and the two share no code.  See ``pat_oracle`` for the functions,
their citations and the readings taken where the paper is silent.
"""
from .pat_oracle import *  # noqa: F401,F403
from .pat_oracle import REG_DTV, REG_TGV, REG_TV  # noqa: F401
