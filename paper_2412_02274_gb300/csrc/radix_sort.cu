// radix_sort.cu -- sizes of the radix sorts' per-tile histograms.
//
// The sorts themselves: inside one thread-block cluster for survivor sets and
// skylines of at most kClusterSortMax rows (cluster.cuh), and in one
// cooperative launch above that (radix.cuh).
#include "radix.cuh"

namespace gres {

// Tiles of kRxTile items: the per-digit histogram has this many columns.
int64_t sort_blocks(int64_t n) { return (n + kRxTile - 1) / kRxTile; }

}  // namespace gres
