// Internal declarations of libidp (not part of the C ABI in include/idp.h).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "idp.h"

namespace idp {

constexpr int kFields = 5;  // (rho, m_x, m_y, m_z, E), d + 2 with d = 3
constexpr int kSlice = 32;  // SELL-C slice height: one warp of rows

// Entry flags of the sliced-ELL layout.
enum : uint8_t {
  kEntryUpper = 1,  // j > i: this row evaluates the wavespeed of edge {i, j}
  kEntrySkew = 2,   // c_ji == -c_ij bitwise: one lambda_max evaluation suffices
  kEntryDiag = 4,   // j == i
  kEntryPad = 8     // padding slot of a slice
};

// Host-side mesh matrices in the caller's numbering (CSR, sorted columns).
struct HostMatrices {
  int64_t n = 0;
  std::vector<int64_t> rowptr, col;
  std::vector<double> mij, cij[3], mi;
  bool lumped_given = false;           // mi is the caller's (else m_i = sum_j m_ij)
  std::vector<uint8_t> boundary_pair;  // entry (i,j) lies on a common boundary face
  std::vector<int32_t> bc;
  std::vector<double> xyz;  // 3n node coordinates (mesh uploads; empty for pre-assembled matrices)
  // per entry (i, j): offset of j from i in the reference cell of the first
  // cell holding both, (dz+1) 9 + (dy+1) 3 + (dx+1) (mesh uploads; else empty)
  std::vector<uint8_t> offset;
};

// Sparsity pattern and exact Q1 matrices of Sec. 3.1 eq. (matrices); returns
// an empty string on success or a message describing the bad input.
std::string assemble_q1(int64_t n_nodes, int64_t n_cells, const int64_t* cells, const double* cell_xyz,
                        HostMatrices& out);
// The same for Q1 quadrilaterals in 2D (4 vertices per cell, v = a + 2b,
// 2 coordinates per vertex); the z components of c_ij are zero.
std::string assemble_q1_2d(int64_t n_nodes, int64_t n_cells, const int64_t* cells, const double* cell_xy,
                           HostMatrices& out);

// Sliced-ELL (C = 32) layout of the matrices in the library's row order.
struct SellLayout {
  int64_t n = 0, n_slices = 0, n_slots = 0;
  std::vector<int64_t> perm;      // library row of caller node i
  std::vector<int64_t> iperm;     // caller node of library row r
  std::vector<int32_t> slice_ptr; // n_slices + 1 slot offsets
  std::vector<int32_t> row_len;   // n
  std::vector<int32_t> col, tpos; // n_slots (library ids / slot of the transposed entry)
  std::vector<uint8_t> flags;     // n_slots
  std::vector<double> cx, cy, cz, mij;  // n_slots
  std::vector<double> cn, inv_cn;       // n_slots: |c_ij| and 1/|c_ij| (0 for c_ij = 0)
  std::vector<double> mi, inv_mi, lam;  // n (lam = 1 / (card I(i) - 1))
  std::vector<double> csx, csy, csz;    // n: row sums sum_j c_ij (zero up to rounding)
  std::vector<int32_t> bc;              // n
  std::vector<int64_t> slot_of_entry;   // caller CSR entry -> slot
};

// Row order: renumber 0 = the caller's order, 1 = reverse Cuthill-McKee over
// the stencil graph (each row's entries keep the caller's column order), 2 =
// Morton (Z-order) of the node coordinates M.xyz (an error without them),
// each row's entries ordered by their cell offset M.offset, then library
// column.
std::string build_sell(const HostMatrices& M, SellLayout& L, int renumber = 0);

}  // namespace idp
