"""Seeded synthetic hyperspectral cubes shared by the tests, the smoke check and
the benchmark.  Holds input generation and evaluation metrics only: none of the
denoiser's arithmetic lives here."""
from .hsi import *  # noqa: F401,F403
from .hsi import __all__  # noqa: F401
