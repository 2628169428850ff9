"""FP64 CPU oracle (test infrastructure only; see nadmm_oracle)."""
from .nadmm_oracle import *  # noqa: F401,F403
from .nadmm_oracle_eval import *  # noqa: F401,F403
from .nadmm_oracle_grad import *  # noqa: F401,F403
from .nadmm_oracle_pyramid import *  # noqa: F401,F403
