"""GB300-native conflict-driven answer-set solving (arXiv 1909.01786).

The solver is the CUDA library ``libaspgpu.so`` behind the C ABI in
``include/aspgpu.h``; ``aspgpu`` is its Python binding.
"""
from .aspgpu import (AspError, Program, SAT, UNSAT, UNKNOWN, LEARN_FWD, LEARN_RES,  # noqa: F401
                     BACKJUMP_H_MINUS_1, BACKJUMP_ASSERTING, lib, solve_batch, words_to_models)
