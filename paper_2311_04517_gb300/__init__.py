"""GB300 (sm_103a) HPClust hot path: sampling, K-means++ seeding, Lloyd and
the full-data objective of minimum sum-of-squares clustering (arXiv
2311.04517), as CUDA kernels behind the C ABI of include/hpclust.h.

``hpclust`` is the Python binding of that ABI; ``synth`` generates the seeded
synthetic Gaussian-mixture inputs.
"""
