"""GB300-native (sm_103a) hot path of Probabilistic Domain Decomposition
(Bernal, dos Reis, Smith, arXiv:1705.03666): Monte Carlo Feynman-Kac estimates
at interface nodes, branching diffusions, and the deterministic stage two.

The compute path is libpdd.so (CUDA C++, C ABI in include/pdd.h); ``api``
binds it to torch tensors.  ``workloads`` holds the seeded input generators.
Importing the package does not load the library; the first call does, and
fails loudly if it has not been built.
"""
from . import workloads  # noqa: F401  (input generators only)

__all__ = ["workloads", "Context", "interface_solve_host", "build"]


def __getattr__(name):
    if name in ("Context", "interface_solve_host"):
        from . import api
        return getattr(api, name)
    if name == "build":
        from .build import build
        return build
    raise AttributeError(name)
