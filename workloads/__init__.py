"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package builds the *inputs* of the cascade (continuous HiPPO-LegS state
matrices, random B, C, D, step sizes, input sequences, ragged batch layouts).
It holds none of the method's arithmetic: no discretisation, no powers, no
cascade.  Both the CPU oracle and the tests/bench of the CUDA path draw from it.
"""
from .synth import *  # noqa: F401,F403
