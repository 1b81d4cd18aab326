"""GB300-native PEOs routing for graph ANNS (arXiv 2402.11354): batched graph
beam search with the PEOs probabilistic edge test, as a CUDA library (sm_103a)
behind a C ABI (include/peos.h) with this thin Python binding."""
from .peos import (Codes, Graph, PeosError, build_codes, edge_stats, knn_bruteforce, load, projections,  # noqa: F401
                   release_workspace, search, search_host, search_noalloc, version, COUNTER_NAMES, NCOUNTERS)
