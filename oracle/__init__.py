"""ORACLE -- test infrastructure, not part of the product.

A plain, slow, float64 CPU implementation of RandRAND written from the paper
(arXiv 2509.19747), used only to check the CUDA library: by ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``.  The
library never imports, links or executes anything here, and nothing here
imports the library.
"""
from . import philox, randrand  # noqa: F401
