"""GB300 (sm_103a) implementation of the DVNR hot path (arXiv 2304.10516):
hash-grid INR training per partition, decoding and ray-marching, behind the C
ABI of ``libdvnr.so`` (``include/dvnr.h``).

Importing the package loads nothing; ``paper_2304_10516_gb300.model`` loads
the CUDA library on first use and raises if it is missing.
"""

__all__ = ["model", "volumes", "build"]
