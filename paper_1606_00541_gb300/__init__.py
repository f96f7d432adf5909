"""GB300-native level-scheduled sparse triangular solves on the HEC format (arXiv 1606.00541).

The compute path is the C-ABI library ``libhec.so`` built from ``csrc/`` (hand-written CUDA for
sm_103a).  ``paper_1606_00541_gb300.hec`` is its thin Python binding; importing it loads the
library and fails loudly when the library is missing.  ``synth`` builds seeded test problems.
Importing this package itself loads nothing.
"""
__all__ = ["hec", "synth"]
