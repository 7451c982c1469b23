"""GB300-native (sm_103a) hot path of BSGD for tomographic reconstruction.

Block stochastic gradient descent (Gao, Biguri and Blumensath, arXiv:1903.11874):
on-the-fly Siddon forward projection of a sampled row block, the matched back
projection into a sampled column block, the aggregated block gradient step,
device-side block sampling and the TV proximal step, behind the C ABI in
include/bsgd.h. The Python names below forward to that ABI (binding.py);
`synth` draws seeded synthetic inputs. Importing the package loads nothing;
the CUDA library is loaded on first use and every call fails loudly without it.
"""
_BINDING_NAMES = {
    "Geometry", "State", "SolveParams", "BSGDError", "bsgd_geometry_create",
    "bsgd_forward_project", "bsgd_back_project", "bsgd_count_updates", "bsgd_power_iteration",
    "bsgd_tv_prox", "bsgd_state_create", "bsgd_block_step", "bsgd_state_query", "bsgd_solve",
    "F32", "BF16", "F16", "STEP_STRIP", "STEP_BLOCK", "STEP_FIXED", "PAIRS_UNIFORM",
    "PAIRS_RESIDUAL", "CELLS_NONE", "CELLS_GEOMETRIC", "CELLS_UNIFORM",
}


def __getattr__(name):
    if name in _BINDING_NAMES:
        from . import binding
        return getattr(binding, name)
    raise AttributeError(name)
