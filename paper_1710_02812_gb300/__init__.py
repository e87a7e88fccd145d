"""GB300-native hierarchical merge-and-truncate rank-k SVD (arXiv:1710.02812).

The compute path is the C-ABI library ``libhsvd.so`` (CUDA for sm_103a);
``hsvd`` is its thin Python binding and ``workloads`` the seeded synthetic
inputs.  Importing this package does not load the library; the first call
into ``hsvd`` does, and raises if it has not been built.
"""
from . import workloads  # noqa: F401
