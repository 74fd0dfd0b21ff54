"""dfsnufft: GB300-native type-2 NUFFT for the spectral interpolation step of the
double-Fourier-sphere semi-implicit semi-Lagrangian shallow-water scheme.

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/dfsnufft.h``); :mod:`.nufft` is its Python binding and :mod:`.synth`
draws seeded synthetic inputs.
"""
__all__ = ["Plan", "Options", "Ensemble", "nufft", "synth"]


def __getattr__(name):
    if name in ("Plan", "Options", "Ensemble"):
        from . import nufft
        return getattr(nufft, name)
    raise AttributeError(name)
