"""FP64 CPU oracle (test infrastructure only; see cgmimo_oracle)."""

from .cgmimo_oracle import *  # noqa: F401,F403
from .cgmimo_oracle import (STATUS_BREAKDOWN, STATUS_MU_NONPOS, STATUS_OK,  # noqa: F401
                            _gray_inverse)
