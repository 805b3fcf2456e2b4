"""GB300-native staggered-grid acoustic modelling, RTM and FWI gradients
(the hot path of SMIwiz, arXiv 2311.02293).

The compute path is the C-ABI library ``libsmi.so`` (CUDA, sm_103a) built
from ``csrc/``; ``smi`` is its thin Python binding.  Importing this package
does not load the library; ``from paper_2311_02293_gb300 import smi`` does.
"""
__all__ = ["smi", "synth"]
