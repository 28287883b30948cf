"""CPU FP64 oracle (test infrastructure only; see ``vne_oracle``)."""
from . import rng  # noqa: F401
from .vne_oracle import *  # noqa: F401,F403
