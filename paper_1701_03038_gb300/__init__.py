"""GB300-native Viterbi and forward-backward decoding with large, sparse,
epsilon-free weighted finite-state transducers (Argueta & Chiang, EACL 2017).

The compute path is the C-ABI library ``libfstgpu.so`` (hand-written CUDA
kernels for sm_103a); this package marshals arguments to it.  Importing the
package does not load the library; ``Fst`` and friends do, and they raise if
it has not been built (there is no CPU fallback).
"""
from .synth import FstArrays, Strings  # noqa: F401

__all__ = ["FstArrays", "Strings"]
