"""Plain FP64 CPU oracle of the ADI heat step.  TEST INFRASTRUCTURE ONLY."""
from .oracle import Oracle, build, max_threads, pulse, set_threads, thomas  # noqa: F401
