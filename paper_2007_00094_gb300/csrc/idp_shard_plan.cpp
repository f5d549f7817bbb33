// Host construction of the row partition and exchange lists (idp_shard.h).
#include <algorithm>

#include "idp_shard.h"

namespace idp {

std::string build_shard_plan(int64_t n, const int64_t* rowptr, const int64_t* col, int n_shards,
                             const int64_t* row_begin, ShardPlan& plan) {
  if (n <= 0 || !rowptr || !col || n_shards < 1 || !row_begin) return "bad partition arguments";
  if (row_begin[0] != 0 || row_begin[n_shards] != n) return "row ranges must start at 0 and end at n";
  for (int s = 0; s < n_shards; ++s)
    if (row_begin[s + 1] <= row_begin[s]) return "every shard needs at least one row";
  if (rowptr[0] != 0) return "rowptr[0] must be 0";
  for (int64_t i = 0; i < n; ++i) {
    if (rowptr[i + 1] < rowptr[i]) return "rowptr must not decrease";
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      if (col[k] < 0 || col[k] >= n) return "column index out of range";
      if (k > rowptr[i] && col[k] <= col[k - 1]) return "columns must increase within a row";
    }
  }
  plan = ShardPlan{};
  plan.n = n;
  plan.nnz = rowptr[n];
  plan.n_shards = n_shards;
  plan.row_begin.assign(row_begin, row_begin + n_shards + 1);
  plan.shard.resize(n_shards);
  auto owner = [&](int64_t g) {
    return (int)(std::upper_bound(plan.row_begin.begin(), plan.row_begin.end(), g) - plan.row_begin.begin()) - 1;
  };
  std::vector<int64_t> local(n, -1);  // global -> local id of the shard being built
  for (int s = 0; s < n_shards; ++s) {
    ShardLocal& S = plan.shard[s];
    const int64_t a = row_begin[s], b = row_begin[s + 1];
    // nodes: own rows and every column of them, in global order
    std::vector<int64_t>& nodes = S.nodes;
    for (int64_t i = a; i < b; ++i)
      for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) nodes.push_back(col[k]);
    for (int64_t i = a; i < b; ++i) nodes.push_back(i);
    std::sort(nodes.begin(), nodes.end());
    nodes.erase(std::unique(nodes.begin(), nodes.end()), nodes.end());
    for (size_t l = 0; l < nodes.size(); ++l) local[nodes[l]] = (int64_t)l;
    S.own_lo = local[a];
    S.own_hi = local[b - 1] + 1;
    // local CSR: entries to nodes of the shard, in the global column order
    S.rowptr.assign(1, 0);
    for (int64_t g : nodes) {
      for (int64_t k = rowptr[g]; k < rowptr[g + 1]; ++k) {
        const int64_t lc = local[col[k]];
        if (lc < 0) continue;
        S.col.push_back(lc);
        S.entry.push_back(k);
      }
      S.rowptr.push_back((int64_t)S.col.size());
    }
    S.send_nodes.assign(n_shards, {});
    S.recv_nodes.assign(n_shards, {});
    S.send_entries.assign(n_shards, {});
    S.recv_entries.assign(n_shards, {});
    const int64_t nl = (int64_t)nodes.size();
    for (int64_t l = 0; l < nl; ++l) {
      const int64_t g = nodes[l];
      const bool own = l >= S.own_lo && l < S.own_hi;
      if (!own) {
        const int q = owner(g);
        S.recv_nodes[q].push_back(l);
        // entries (g, i) of the ghost row with i an own row: l_gi comes from q
        for (int64_t e = S.rowptr[l]; e < S.rowptr[l + 1]; ++e) {
          const int64_t c = S.col[e];
          if (c >= S.own_lo && c < S.own_hi) S.recv_entries[q].push_back(e);
        }
        continue;
      }
      // an own row is a ghost of every other shard that owns one of its
      // columns (the pattern is symmetric); entries to those shards' rows
      // are what they read of this row
      int last = -1;
      for (int64_t e = S.rowptr[l]; e < S.rowptr[l + 1]; ++e) {
        const int64_t c = S.col[e];
        if (c >= S.own_lo && c < S.own_hi) continue;
        const int q = owner(nodes[c]);
        S.send_entries[q].push_back(e);
        if (q != last) {
          // columns increase, so the ghosts of one shard come together; a row
          // is listed once per shard
          auto& sn = S.send_nodes[q];
          if (sn.empty() || sn.back() != l) sn.push_back(l);
          last = q;
        }
      }
    }
    for (int64_t g : nodes) local[g] = -1;
  }
  // the pattern must be structurally symmetric for the lists to match
  for (int s = 0; s < n_shards; ++s)
    for (int q = 0; q < n_shards; ++q) {
      const ShardLocal &A = plan.shard[s], &B = plan.shard[q];
      if (A.send_nodes[q].size() != B.recv_nodes[s].size() || A.send_entries[q].size() != B.recv_entries[s].size())
        return "sparsity pattern is not structurally symmetric";
      for (size_t k = 0; k < A.send_nodes[q].size(); ++k)
        if (A.nodes[A.send_nodes[q][k]] != B.nodes[B.recv_nodes[s][k]])
          return "sparsity pattern is not structurally symmetric";
      for (size_t k = 0; k < A.send_entries[q].size(); ++k)
        if (A.entry[A.send_entries[q][k]] != B.entry[B.recv_entries[s][k]])
          return "sparsity pattern is not structurally symmetric";
    }
  return std::string();
}

}  // namespace idp
