"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark."""
from .synth import *  # noqa: F401,F403
