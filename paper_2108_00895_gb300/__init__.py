"""Exact sparse spherical k-means on one GB300 GPU (sm_103a).

Method: Knittel, Koch, Ertl, "Efficient Sparse Spherical k-Means for Document
Clustering", DocEng 2021 -- the Lloyd assignment step (Sec. 2) with the
non-changing-clusters skip (Sec. 3.1), a deterministic centroid update, and FP64
rescoring of near ties.

Modules (imported on demand so that input generation needs no GPU):
  skm        ctypes binding of the C ABI in include/skm.h (libskm.so) and
             ``SphericalKMeans``, the owner of one context.
  build      nvcc build of libskm.so.
  synth      seeded synthetic tf-idf corpora (input generation only).
  workloads  the named workloads used by tests and the benchmark.
"""
__all__ = ["skm", "build", "synth", "workloads"]
