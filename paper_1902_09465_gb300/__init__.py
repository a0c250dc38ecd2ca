"""GB300-native adaptive k-nearest-neighbour search (LeJeune, Baraniuk and
Heckel, "Adaptive Estimation for Approximate k-Nearest-Neighbor Computations",
AISTATS 2019).

The compute path is a C-ABI CUDA library (``csrc/``, built for sm_103a);
``knn`` is its thin Python binding. ``synth`` holds the seeded input
generators.
"""

import importlib

__all__ = ["knn", "synth", "build", "runtime"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
