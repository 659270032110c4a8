"""Exact word-frequency counting on one GB300 GPU (sm_103a).

The CUDA library (csrc/, built into _build/libwc.so by build.py) implements
the MapReduce word count of arXiv 2206.05269 on the device: letters-only
tokenisation with lowercasing (the map of Sec. 2 / Sec. 3.1), exact counts per
document, per class and overall (the reduce of Sec. 3.3), sorted by count
descending then word ascending.  ``wc`` is the thin ctypes binding.
"""
from . import wc  # noqa: F401
