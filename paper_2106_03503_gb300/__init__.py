"""libedt: exact squared Euclidean distance transform and feature map on GB300.

The compute path is the CUDA shared library built from ``csrc/`` and called
through the C ABI declared in ``include/edt.h``; ``edt`` is its thin Python
binding.  Importing this package loads nothing: ``from paper_2106_03503_gb300
import edt`` loads the library and fails loudly when it is missing.
"""
__all__ = ["edt", "inputs"]
