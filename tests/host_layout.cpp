// Test harness (test infrastructure only): runs the library's host set-up,
// Q1 assembly and the sliced-ELL layout, on a mesh and checks the layout's
// invariants on the CPU, counting violations.
#include <cstdint>
#include <cstdlib>
#include <string>

#include "idp_internal.h"

extern "C" int host_layout(int dim, int64_t n, int64_t nc, const int64_t* cells, const double* x, int renumber,
                           int64_t* perm_out, int64_t* stats) {
  idp::HostMatrices M;
  std::string msg = dim == 3 ? idp::assemble_q1(n, nc, cells, x, M) : idp::assemble_q1_2d(n, nc, cells, x, M);
  if (!msg.empty()) return 1;
  M.bc.assign(n, 0);
  idp::SellLayout L;
  if (!idp::build_sell(M, L, renumber).empty()) return 2;
  int64_t bad_perm = 0, bad_tpos = 0, bad_upper = 0, bad_diag = 0, bad_col = 0, bad_skew = 0, bad_map = 0;
  int64_t bandwidth = 0;
  for (int64_t i = 0; i < n; ++i) {
    perm_out[i] = L.perm[i];
    if (L.perm[i] < 0 || L.perm[i] >= n || L.iperm[L.perm[i]] != i) ++bad_perm;
  }
  std::vector<char> used(L.n_slots, 0);
  for (int64_t i = 0; i < n; ++i) {
    const int64_t r = L.perm[i];
    int diag = 0;
    for (int64_t e = M.rowptr[i]; e < M.rowptr[i + 1]; ++e) {
      const int64_t p = L.slot_of_entry[e], j = M.col[e];
      if (p < 0 || p >= L.n_slots || used[p]) {
        ++bad_map;
        continue;
      }
      used[p] = 1;
      // slot p belongs to row r: slice of r, lane r % 32
      if ((p - L.slice_ptr[r / 32]) % 32 != r % 32) ++bad_map;
      if (L.col[p] != L.perm[j]) ++bad_col;
      const int64_t pt = L.tpos[p];
      if (pt < 0 || pt >= L.n_slots || L.tpos[pt] != p || L.col[pt] != r) ++bad_tpos;
      const int64_t dist = std::llabs(L.perm[j] - r);
      if (dist > bandwidth) bandwidth = dist;
      if (j == i) {
        ++diag;
        if (!(L.flags[p] & idp::kEntryDiag) || (L.flags[p] & idp::kEntryUpper)) ++bad_diag;
      } else {
        // exactly one orientation of a pair is the upper one: the smaller caller
        // id's row (Morton order: the row from which the other lies at a
        // positive cell offset)
        const bool up = L.flags[p] & idp::kEntryUpper, up_t = L.flags[pt] & idp::kEntryUpper;
        const bool want = renumber == 2 ? M.offset[e] > 13 : j > i;
        if (up == up_t || up != want) ++bad_upper;
        const bool sk = L.flags[p] & idp::kEntrySkew, sk_t = L.flags[pt] & idp::kEntrySkew;
        if (sk != sk_t) ++bad_skew;
      }
    }
    if (diag != 1) ++bad_diag;
  }
  for (int64_t p = 0; p < L.n_slots; ++p)
    if (!used[p] && !(L.flags[p] & idp::kEntryPad)) ++bad_map;
  const int64_t s[9] = {L.n_slots, bad_perm, bad_tpos, bad_upper, bad_diag, bad_col, bad_skew, bad_map, bandwidth};
  for (int k = 0; k < 9; ++k) stats[k] = s[k];
  return 0;
}
