"""GB300-native importance-sampled generalized Feynman-Kac (GFK) walk for helium.

The compute path is the CUDA library ``libgfk.so`` (sm_103a), reached through a
C ABI (``include/gfk.h``).  ``gfk`` is its thin Python binding; ``workloads``
holds the seeded synthetic inputs.  Nothing here falls back to the CPU: if the
library cannot be built or loaded, the binding raises.  Submodules are imported
on demand (``from paper_1703_08977_gb300 import gfk``).
"""
