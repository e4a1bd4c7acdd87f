"""Plain FP64 CPU oracle of the ADI heat step.  TEST INFRASTRUCTURE ONLY."""
from .oracle import Oracle, thomas, build, set_threads, max_threads  # noqa: F401
