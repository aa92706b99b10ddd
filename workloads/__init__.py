"""Seeded synthetic input generators (random numbers only; no search arithmetic)."""
from .synth import *  # noqa: F401,F403
from .synth import __all__  # noqa: F401
