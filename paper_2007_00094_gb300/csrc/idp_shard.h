// Row partition of the stage for domain decomposition (Sec. 4.1, Fig. 1-2):
// contiguous ranges of rows, each shard holding its rows and one ghost layer
// (the neighbours of its rows that other shards own), and the lists of the
// values that shards exchange at the stage's synchronisation points.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace idp {

struct ShardLocal {
  // Global ids of the shard's nodes (its rows and its ghosts), increasing;
  // the local id of a node is its index here, so local ids keep the global
  // order and every row keeps its global column order.
  std::vector<int64_t> nodes;
  int64_t own_lo = 0, own_hi = 0;  // local ids of the shard's own rows: [own_lo, own_hi)
  // Local CSR: every node's entries to nodes of the shard (all entries for an
  // own row, a subset for a ghost row), local column ids, and the global CSR
  // entry each local entry is.
  std::vector<int64_t> rowptr, col, entry;
  // Exchange lists per peer shard q (empty for q == this shard), in the order
  // of global ids, so that the sender's list and the receiver's list of the
  // same link enumerate the same values:
  //   send_nodes[q]   own rows that are ghosts of q (local ids here)
  //   recv_nodes[q]   ghosts here that q owns (local ids here)
  //   send_entries[q] entries (g, i) of own rows g with i owned by q (local entry ids here)
  //   recv_entries[q] entries (g, i) of ghost rows g owned by q with i an own row here
  std::vector<std::vector<int64_t>> send_nodes, recv_nodes, send_entries, recv_entries;
};

struct ShardPlan {
  int64_t n = 0, nnz = 0;
  int n_shards = 0;
  std::vector<int64_t> row_begin;  // n_shards + 1 global row offsets
  std::vector<ShardLocal> shard;
};

// Builds the plan of a structurally symmetric CSR pattern (rowptr n+1, col
// nnz, columns increasing within each row) for the given row ranges
// (row_begin[0] = 0, strictly increasing so that every shard owns a row,
// row_begin[n_shards] = n).
// Returns an empty string on success, else what is wrong with the input.
std::string build_shard_plan(int64_t n, const int64_t* rowptr, const int64_t* col, int n_shards,
                             const int64_t* row_begin, ShardPlan& plan);

}  // namespace idp
