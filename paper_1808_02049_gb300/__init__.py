"""GB300-native deterministic, sort-based Epstein-Nesbet PT2 (arXiv:1808.02049).

The computation lives in the CUDA library libpt2 (include/pt2.h); ``pt2`` is
its ctypes binding and ``inputs`` the seeded synthetic workload generator.
"""

from . import inputs  # noqa: F401
