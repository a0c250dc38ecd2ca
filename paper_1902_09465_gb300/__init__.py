"""GB300-native adaptive k-nearest-neighbour search (LeJeune, Baraniuk and
Heckel, "Adaptive Estimation for Approximate k-Nearest-Neighbor Computations",
AISTATS 2019).

The compute path is a C-ABI CUDA library (``csrc/``, built for sm_103a);
``knn`` is its thin Python binding. ``synth`` holds the seeded input
generators.
"""

__all__ = ["knn", "synth"]


def __getattr__(name):
    if name == "knn":
        from . import knn as _knn
        return _knn
    if name == "synth":
        from . import synth as _synth
        return _synth
    raise AttributeError(name)
