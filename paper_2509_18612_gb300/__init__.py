"""GB300 (sm_103a) hot path of the DECO MaxCut solver (arXiv 2509.18612).

The computation lives in libdeco.so (hand-written CUDA kernels behind the C
ABI declared in include/deco.h).  This package is its thin Python binding;
importing it loads the library and fails loudly if it has not been built.
"""
from ._lib import *  # noqa: F401,F403
from ._lib import lib, Graph, DecoError, graph_from, last_error  # noqa: F401
