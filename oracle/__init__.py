"""FP64 CPU oracle of the SIFT extraction path.

Test infrastructure: imported only by tests/, __graft_entry__.smoke() and the
benchmark's CPU-baseline / reference arm. The product package never imports it.
"""
from .sift_oracle import *  # noqa: F401,F403
from .sift_oracle import Params, extract  # noqa: F401
