"""B300-native graph-based static timing analysis (HeteroSTA hot path).

``paper_2511_11660_b300.sta`` binds the C-ABI library ``libsta.so`` built
from ``csrc/``; ``synth`` draws seeded synthetic designs.  Submodules are
imported on demand so that the generator can be used without a GPU.
"""
__all__ = ["sta", "synth", "autograd"]
