"""GB300-native PEOs routing for graph ANNS (arXiv 2402.11354): batched graph
beam search with the PEOs probabilistic edge test, as a CUDA library (sm_103a)
behind a C ABI (include/peos.h) with this thin Python binding."""
from .peos import (Codes, Graph, Hierarchy, PeosError, Server, StoredBase, build_codes, build_simhash, check_read, crc32,
                   dim_permutation, edge_stats, hier_entry, knn_bruteforce, load_codes, selftest_bounded_wait,
                   knn_tensor, load,  # noqa: F401
                   projections, quantize, release_workspace, search, search_batch, batch_workspace_size, search_host,
                   search_noalloc, trace_enable, trace_read, version,
                   COUNTER_NAMES, NCOUNTERS)
