"""GB300-native grid-filtered spatial join (PIP and P2P) after Zhang & You,
"Large-Scale Geospatial Processing on Multi-Core and Many-Core Processors"
(arXiv 1403.0802).

The compute path is libsj.so (hand-written CUDA for sm_103a behind the C ABI
of include/sj.h); `paper_1403_0802_gb300.api` marshals torch tensors / numpy
arrays into it.  The CUDA library is loaded on first use and its absence is an
error.  Submodules are imported on demand (`from paper_1403_0802_gb300 import api`).
"""
