"""FP64 CPU oracle of the modified IDM simulator, its adjoint and the fit.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the product library
never does, and it shares no code with the CUDA path.
"""
from .ref import (  # noqa: F401
    build,
    forward,
    mse_seed,
    adjoint,
    adam_step,
    lr_schedule,
    fit,
    layout,
    PARAM_NAMES,
)
from . import mlp_oracle  # noqa: F401,E402
from . import recon  # noqa: F401,E402
from . import lanes  # noqa: F401,E402
