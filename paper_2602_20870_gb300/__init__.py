"""GB300-native FGFRFT online hot path (fast graph fractional Fourier transform).

The compute path lives in the C-ABI library ``libfgfrft.so`` built from
``csrc/``; ``fgfrft`` is its thin Python binding.  Import ``fgfrft`` (or call
``load()``) to load the library; importing the package itself loads nothing.
"""
__all__ = ["workloads"]
