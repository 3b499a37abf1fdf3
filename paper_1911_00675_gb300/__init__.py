"""GB300-native ProbMinHash: signatures of weighted sets for the probability
Jaccard similarity J_P (Ertl, arXiv 1911.00675) and equal-component J_P
estimation, computed by hand-written sm_103a CUDA kernels behind a C ABI.

``paper_1911_00675_gb300.pmh`` is the thin Python binding (argument
marshalling only); ``paper_1911_00675_gb300.workloads`` draws seeded synthetic
inputs.  Importing the package does not load the CUDA library.
"""
__all__ = ["pmh", "workloads"]
