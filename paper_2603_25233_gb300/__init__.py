"""GB300 (sm_103a) library for the rank-adaptive sweep-based SI-DSA of the steady 2D x-y
S_N radiative transfer equation: C ABI in include/rte.h, kernels in csrc/, the Python
binding in api.py (torch device tensors and streams as plumbing)."""
from ._lib import (RTE_FP32, RTE_FP64, RTE_MODE_FR, RTE_MODE_LR, RteError,  # noqa: F401
                   load as load_library)


def __getattr__(name):
    if name in ("Handle", "default_opts", "sweep_batch", "si_dsa_solve_batch", "detector_response"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
