"""GB300-native LArTPC signal simulation (drift, rasterize, scatter-add, FFT convolution).

The compute path lives in the CUDA library ``libwcsim.so`` built from ``csrc/``; the Python
binding in :mod:`paper_2104_08265_gb300.wcsim` only marshals arguments to its C-ABI.
Submodules are imported explicitly (``from paper_2104_08265_gb300 import wcsim``) so that
the input generators in :mod:`.synth` can be used without the CUDA library.
"""
