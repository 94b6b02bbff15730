"""TFHE oracle for VeLoPIR's hot path -- TEST INFRASTRUCTURE ONLY.

A plain CPU implementation (tfhe_oracle.c) used by tests/, by
__graft_entry__.smoke() and by bench.py's CPU-baseline leg to check and time
the CUDA library.  The CUDA library never imports, links or executes anything
here; the two share no code.  Inputs come from paper_2506_12761_gb300.synth,
which draws random numbers only.
"""
from .oracle import *  # noqa: F401,F403
