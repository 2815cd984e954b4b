"""Seeded synthetic inputs shared by the oracle-side tests and the CUDA path.

This module draws random numbers and assembles op lists; it contains none of
the method's arithmetic (no Kraus map is ever applied here).
"""
from .synth import *  # noqa: F401,F403
