"""CPU oracle for the Holstein DQMC engine (plain FP64 numpy/scipy).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU-baseline
leg of bench.py may import it; the CUDA path never does, and the two share no code.
"""
from . import philox, dqmc, autocorr  # noqa: F401
