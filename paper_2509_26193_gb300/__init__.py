"""GB300-native Barnes-Hut connectivity update of the Model of Structural
Plasticity (arXiv 2509.26193), backed by hand-written sm_103a CUDA kernels.

Importing the package loads nothing native; the first call into
``paper_2509_26193_gb300.relearn`` loads ``librelearn.so`` and raises if it is
missing (there is no CPU fallback).
"""
__all__ = ["relearn", "workloads"]
