"""Plain FP64 CPU oracle of the coupled FCD time step (arXiv 2410.11129).

Test infrastructure only: tests/, the smoke check and the benchmark's CPU
baseline import it; the product package never does.
"""
from .oracle import *  # noqa: F401,F403
