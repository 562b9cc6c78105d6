"""Seeded synthetic inputs shared by the tests, the bench and the oracle's callers.

This package holds only input construction (random numbers, prescribed spectra,
Householder test matrices, start blocks). It contains none of the eigensolver's
arithmetic.
"""
from .problems import (  # noqa: F401
    Problem,
    complex_normal,
    config_problem,
    uniform01,
)
