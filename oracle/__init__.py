"""FP64 CPU oracle (test infrastructure only; see scint_oracle's header)."""
from .scint_oracle import *  # noqa: F401,F403
from .scint_oracle import ScreenParams  # noqa: F401
