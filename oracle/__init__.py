"""FP64 CPU oracle (test infrastructure only; never imported by the product path)."""
from .cc_oracle import *  # noqa: F401,F403
from .cc_oracle import CC_SN, CC_U, grid_size, track_one, track_batch, track_batch_parallel  # noqa: F401
