"""GB300-native indexed k-means (Dask-means, arXiv 2412.02244).

The compute path lives in ``libdkm.so`` (hand-written sm_103a CUDA behind
the C ABI declared in ``include/dkm.h``).  ``paper_2412_02244_gb300.dkm``
is the thin ctypes binding with the same function names; importing this
package does not load the library, so the seeded input generators in
``paper_2412_02244_gb300.synth`` stay usable on machines without a GPU.
"""

__all__ = ["dkm", "synth"]
