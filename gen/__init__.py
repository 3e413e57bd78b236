"""Seeded synthetic input generators shared by the oracle and the CUDA path (no solver arithmetic)."""
from .problems import *  # noqa: F401,F403
