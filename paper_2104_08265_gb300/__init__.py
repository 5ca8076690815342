"""GB300-native LArTPC signal simulation (drift, rasterize, scatter-add, FFT convolution).

The compute path lives in the CUDA library ``libwcsim.so`` built from ``csrc/``; the Python
binding in :mod:`paper_2104_08265_gb300.wcsim` only marshals arguments to its C-ABI.
Import of the binding is lazy so that the input generators in :mod:`.synth` can be used
without a GPU.
"""

__all__ = ["synth", "wcsim"]


def __getattr__(name):
    if name == "wcsim":
        from . import wcsim as _w
        return _w
    raise AttributeError(name)
