"""GB300 (sm_103a) implementation of the hot path of the four-equation
multi-phase multi-component solver of arXiv 2504.14063: the finite-volume
right-hand side of every SSP-RK3 stage, behind the C ABI of include/mpmc.h.

`workloads` (seeded synthetic inputs) and `build` import without a GPU
library; the binding names (`Context`, `init_state`, `rhs`, `rk_step`,
`step_n`, `rhs_adjoint`, ...) load libmpmc.so and raise if it is missing.
"""
import importlib

from . import workloads  # noqa: F401

_BINDING_NAMES = {"Context", "create", "init_state", "rhs", "rk_step", "step_n", "rhs_adjoint", "MpmcError",
                  "FP64", "MIXED", "lib"}


def __getattr__(name):
    if name in _BINDING_NAMES:
        return getattr(importlib.import_module(__name__ + ".binding"), name)
    raise AttributeError(name)
