// Host set-up of libidp: stencil sparsity, exact Q1 matrices (Sec. 3.1
// eq. "matrices"), boundary-pair detection and the sliced-ELL device layout
// (Sec. 4.3, with slice height 32 = one warp instead of the AVX-512 width).
//
// Runs once per mesh, off the time loop (Sec. 3.2: "avoid all assembly
// operations during the time loop").
#include <algorithm>
#include <cmath>
#include <cstring>

#include "idp_internal.h"

namespace idp {

namespace {

// 3-point Gauss-Legendre rule per direction on [0,1]^D: exact for
// polynomials of degree 5 per direction, enough for phi_i phi_j det J and
// phi_i cof(J) grad^ phi_j of a multilinear map (degree <= 4 per direction).
template <int D>
struct Quadrature {
  static constexpr int NQ = D == 3 ? 27 : 9, NV = 1 << D;
  double w[NQ];
  double phi[NQ][NV];
  double dphi[NQ][NV][D];
  Quadrature() {
    const double r = std::sqrt(15.0) / 10.0;
    const double x1[3] = {0.5 - r, 0.5, 0.5 + r};
    const double w1[3] = {5.0 / 18.0, 4.0 / 9.0, 5.0 / 18.0};
    for (int q = 0; q < NQ; ++q) {
      int qi[3] = {q % 3, (q / 3) % 3, q / 9};
      w[q] = 1.0;
      for (int d = 0; d < D; ++d) w[q] *= w1[qi[d]];
      for (int v = 0; v < NV; ++v) {
        double sh[3], ds[3];
        for (int d = 0; d < D; ++d) {
          const double x = x1[qi[d]];
          const bool hi = (v >> d) & 1;
          sh[d] = hi ? x : 1.0 - x;
          ds[d] = hi ? 1.0 : -1.0;
        }
        phi[q][v] = 1.0;
        for (int d = 0; d < D; ++d) phi[q][v] *= sh[d];
        for (int e = 0; e < D; ++e) {
          double g = ds[e];
          for (int d = 0; d < D; ++d)
            if (d != e) g *= sh[d];
          dphi[q][v][e] = g;
        }
      }
    }
  }
};

// Local matrices of one cell: m_ab, c_ab (3 components; the z component is 0
// in 2D) and int phi_a.  Uses det(J) grad phi_b = cof(J) grad^ phi_b, with
// cof(J) the cofactor matrix; X holds D coordinates per vertex.
template <int D>
bool local_matrices(const Quadrature<D>& Q, const double* X, double (*M)[1 << D], double (*Cm)[1 << D][1 << D],
                    double* m) {
  constexpr int NV = 1 << D, NQ = Quadrature<D>::NQ;
  for (int a = 0; a < NV; ++a) {
    m[a] = 0.0;
    for (int b = 0; b < NV; ++b) {
      M[a][b] = 0.0;
      for (int r = 0; r < 3; ++r) Cm[r][a][b] = 0.0;
    }
  }
  for (int q = 0; q < NQ; ++q) {
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int v = 0; v < NV; ++v)
      for (int r = 0; r < D; ++r)
        for (int t = 0; t < D; ++t) J[r][t] += X[D * v + r] * Q.dphi[q][v][t];
    double K[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};  // cofactors
    double det;
    if (D == 3) {
      K[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
      K[0][1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
      K[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
      K[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
      K[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
      K[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
      K[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
      K[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
      K[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      det = J[0][0] * K[0][0] + J[0][1] * K[0][1] + J[0][2] * K[0][2];
    } else {
      K[0][0] = J[1][1];
      K[0][1] = -J[1][0];
      K[1][0] = -J[0][1];
      K[1][1] = J[0][0];
      det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    }
    if (!(det > 0.0)) return false;
    double G[NV][3];
    for (int b = 0; b < NV; ++b)
      for (int r = 0; r < 3; ++r) {
        double g = 0.0;
        if (r < D)
          for (int t = 0; t < D; ++t) g += K[r][t] * Q.dphi[q][b][t];
        G[b][r] = g;
      }
    for (int a = 0; a < NV; ++a) {
      const double wa = Q.w[q] * Q.phi[q][a];
      m[a] += wa * det;
      for (int b = 0; b < NV; ++b) {
        M[a][b] += wa * Q.phi[q][b] * det;
        for (int r = 0; r < D; ++r) Cm[r][a][b] += wa * G[b][r];
      }
    }
  }
  return true;
}

// Local vertices of the faces of a cell (v = a + 2b + 4c): six quadrilaterals
// of a hexahedron, four edges of a quadrilateral.
const int kFace3[6][4] = {{0, 2, 4, 6}, {1, 3, 5, 7}, {0, 1, 4, 5}, {2, 3, 6, 7}, {0, 1, 2, 3}, {4, 5, 6, 7}};
const int kFace2[4][4] = {{0, 2, -1, -1}, {1, 3, -1, -1}, {0, 1, -1, -1}, {2, 3, -1, -1}};

template <int D>
std::string assemble_impl(int64_t n, int64_t nc, const int64_t* cells, const double* xyz, HostMatrices& out) {
  constexpr int NV = 1 << D, NF = 2 * D, FV = 1 << (D - 1);
  const int(*kFace)[4] = D == 3 ? kFace3 : kFace2;
  if (n <= 0 || nc <= 0) return "empty mesh";
  for (int64_t q = 0; q < NV * nc; ++q)
    if (cells[q] < 0 || cells[q] >= n) return "cell references a node id out of range";
  // node -> cell incidence
  std::vector<int64_t> inc_ptr(n + 1, 0), inc;
  for (int64_t q = 0; q < NV * nc; ++q) inc_ptr[cells[q] + 1]++;
  for (int64_t i = 0; i < n; ++i) inc_ptr[i + 1] += inc_ptr[i];
  inc.resize(inc_ptr[n]);
  {
    std::vector<int64_t> fill(inc_ptr.begin(), inc_ptr.end() - 1);
    for (int64_t c = 0; c < nc; ++c)
      for (int v = 0; v < NV; ++v) inc[fill[cells[NV * c + v]]++] = c;
  }
  for (int64_t i = 0; i < n; ++i)
    if (inc_ptr[i + 1] == inc_ptr[i]) return "a node belongs to no cell";

  // node coordinates, as the first cell around the node sees them (a node on
  // a periodic seam has one position per side; either serves for ordering)
  out.xyz.assign(3 * (size_t)n, 0.0);
  for (int64_t i = 0; i < n; ++i) {
    const int64_t c = inc[inc_ptr[i]];
    for (int v = 0; v < NV; ++v)
      if (cells[NV * c + v] == i) {
        for (int d = 0; d < D; ++d) out.xyz[3 * i + d] = xyz[(NV * c + v) * D + d];
        break;
      }
  }

  // stencil I(i): union of the vertices of the cells around node i (sorted)
  out.n = n;
  out.rowptr.assign(n + 1, 0);
  std::vector<std::vector<int64_t>> rows(n);
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < n; ++i) {
    std::vector<int64_t>& r = rows[i];
    for (int64_t q = inc_ptr[i]; q < inc_ptr[i + 1]; ++q)
      for (int v = 0; v < NV; ++v) r.push_back(cells[NV * inc[q] + v]);
    std::sort(r.begin(), r.end());
    r.erase(std::unique(r.begin(), r.end()), r.end());
  }
  for (int64_t i = 0; i < n; ++i) out.rowptr[i + 1] = out.rowptr[i] + (int64_t)rows[i].size();
  const int64_t nnz = out.rowptr[n];
  out.col.resize(nnz);
  for (int64_t i = 0; i < n; ++i) std::copy(rows[i].begin(), rows[i].end(), out.col.begin() + out.rowptr[i]);
  rows.clear();
  rows.shrink_to_fit();

  out.mij.assign(nnz, 0.0);
  for (int d = 0; d < 3; ++d) out.cij[d].assign(nnz, 0.0);
  out.mi.assign(n, 0.0);
  out.offset.assign(nnz, 0xff);
  auto find = [&](int64_t i, int64_t j) -> int64_t {
    const int64_t* b = out.col.data() + out.rowptr[i];
    const int64_t* e = out.col.data() + out.rowptr[i + 1];
    const int64_t* p = std::lower_bound(b, e, j);
    return (p != e && *p == j) ? (p - out.col.data()) : -1;
  };

  // cell matrices, computed in parallel chunks and added in cell order so the
  // sums do not depend on the thread count
  static const Quadrature<D> Q;
  const int64_t chunk = 1 << 16;
  struct Local {
    double M[NV][NV], C[3][NV][NV], m[NV];
  };
  std::vector<Local> loc(std::min<int64_t>(chunk, nc));
  for (int64_t c0 = 0; c0 < nc; c0 += chunk) {
    const int64_t c1 = std::min(nc, c0 + chunk);
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t c = c0; c < c1; ++c) {
      Local& L = loc[c - c0];
      if (!local_matrices<D>(Q, xyz + D * NV * c, L.M, L.C, L.m)) bad |= 1;
    }
    if (bad) return "a cell has a non-positive Jacobian determinant";
    for (int64_t c = c0; c < c1; ++c) {
      const Local& L = loc[c - c0];
      const int64_t* vn = cells + NV * c;
      for (int a = 0; a < NV; ++a) {
        out.mi[vn[a]] += L.m[a];
        for (int b = 0; b < NV; ++b) {
          const int64_t k = find(vn[a], vn[b]);
          out.mij[k] += L.M[a][b];
          for (int d = 0; d < 3; ++d) out.cij[d][k] += L.C[d][a][b];
          if (out.offset[k] == 0xff) {
            // reference-corner offset of vertex b from vertex a (v = x + 2y + 4z bits)
            const int dx = (b & 1) - (a & 1), dy = ((b >> 1) & 1) - ((a >> 1) & 1),
                      dz = ((b >> 2) & 1) - ((a >> 2) & 1);
            out.offset[k] = (uint8_t)((dz + 1) * 9 + (dy + 1) * 3 + (dx + 1));
          }
        }
      }
    }
  }

  // boundary faces: faces of exactly one cell.  Entries (i, j) with both
  // nodes on a common boundary face carry the boundary term
  // c_ij + c_ji = int_dOmega phi_i phi_j n; all others are skew in exact
  // arithmetic and are made skew bitwise here.
  out.boundary_pair.assign(nnz, 0);
  std::vector<uint8_t> on_boundary(n, 0);
  std::vector<uint8_t> face_free(NF * nc, 0);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nc; ++c) {
    const int64_t* vn = cells + NV * c;
    for (int f = 0; f < NF; ++f) {
      const int64_t a = vn[kFace[f][0]];
      bool shared = false;
      for (int64_t q = inc_ptr[a]; q < inc_ptr[a + 1] && !shared; ++q) {
        const int64_t o = inc[q];
        if (o == c) continue;
        const int64_t* on = cells + NV * o;
        int hit = 0;
        for (int v = 0; v < NV; ++v)
          for (int p = 1; p < FV; ++p) hit += on[v] == vn[kFace[f][p]];
        shared = hit >= FV - 1;
      }
      face_free[NF * c + f] = shared ? 0 : 1;
    }
  }
  for (int64_t c = 0; c < nc; ++c) {
    const int64_t* vn = cells + NV * c;
    for (int f = 0; f < NF; ++f) {
      if (!face_free[NF * c + f]) continue;
      int64_t fn[4];
      for (int p = 0; p < FV; ++p) fn[p] = vn[kFace[f][p]];
      for (int p = 0; p < FV; ++p) {
        on_boundary[fn[p]] = 1;
        for (int r = 0; r < FV; ++r) {
          const int64_t k = find(fn[p], fn[r]);
          if (k >= 0) out.boundary_pair[k] = 1;
        }
      }
    }
  }
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t k = out.rowptr[i]; k < out.rowptr[i + 1]; ++k) {
      const int64_t j = out.col[k];
      if (j == i) {
        if (!on_boundary[i])
          for (int d = 0; d < 3; ++d) out.cij[d][k] = 0.0;
        continue;
      }
      if (j < i || out.boundary_pair[k]) continue;
      const int64_t kt = find(j, i);
      for (int d = 0; d < 3; ++d) {
        const double s = 0.5 * (out.cij[d][k] - out.cij[d][kt]);
        out.cij[d][k] = s;
        out.cij[d][kt] = -s;
      }
    }
  }
  return "";
}

}  // namespace

std::string assemble_q1(int64_t n, int64_t nc, const int64_t* cells, const double* xyz, HostMatrices& out) {
  return assemble_impl<3>(n, nc, cells, xyz, out);
}

std::string assemble_q1_2d(int64_t n, int64_t nc, const int64_t* cells, const double* xy, HostMatrices& out) {
  return assemble_impl<2>(n, nc, cells, xy, out);
}

// Reverse Cuthill-McKee order of the stencil graph: per connected component
// (taken in order of their smallest node id) a breadth-first order from a
// pseudo-peripheral node (the lowest-degree node of the last level of a
// breadth-first search from the component's smallest id), neighbours visited
// by increasing degree, then id; the whole sequence reversed.  Returns the
// caller node of each row.
std::vector<int64_t> rcm_order(const HostMatrices& M) {
  const int64_t n = M.n;
  std::vector<int64_t> order, level(n, -1), queue;
  order.reserve(n);
  queue.reserve(n);
  std::vector<char> done(n, 0);
  auto deg = [&](int64_t i) { return M.rowptr[i + 1] - M.rowptr[i]; };
  std::vector<int64_t> nb;
  for (int64_t s0 = 0; s0 < n; ++s0) {
    if (done[s0]) continue;
    // breadth-first levels from s0 to find a pseudo-peripheral start
    queue.clear();
    queue.push_back(s0);
    level[s0] = 0;
    for (size_t h = 0; h < queue.size(); ++h) {
      const int64_t u = queue[h];
      for (int64_t e = M.rowptr[u]; e < M.rowptr[u + 1]; ++e) {
        const int64_t v = M.col[e];
        if (level[v] < 0) {
          level[v] = level[u] + 1;
          queue.push_back(v);
        }
      }
    }
    int64_t start = queue.back();
    for (int64_t u : queue)
      if (level[u] == level[queue.back()] && (deg(u) < deg(start) || (deg(u) == deg(start) && u < start))) start = u;
    for (int64_t u : queue) level[u] = -1;
    // Cuthill-McKee order of the component from start
    const size_t first = order.size();
    order.push_back(start);
    done[start] = 1;
    for (size_t h = first; h < order.size(); ++h) {
      const int64_t u = order[h];
      nb.clear();
      for (int64_t e = M.rowptr[u]; e < M.rowptr[u + 1]; ++e)
        if (!done[M.col[e]]) nb.push_back(M.col[e]);
      std::sort(nb.begin(), nb.end(), [&](int64_t a, int64_t b) { return deg(a) != deg(b) ? deg(a) < deg(b) : a < b; });
      for (int64_t v : nb) {
        done[v] = 1;
        order.push_back(v);
      }
    }
  }
  std::reverse(order.begin(), order.end());
  return order;
}

// Morton (Z-order) of the node coordinates: each coordinate scaled by the
// largest extent of the bounding box to 21 bits, the bits interleaved (x
// lowest), rows sorted by key and then by caller id.  Consecutive rows, and
// so the 32 rows of a slice, are nodes of a compact block of space (4 x 4 x 2
// on a uniform grid), whose stencils overlap; build_sell also orders each
// row's entries by their offset in the reference cell, whatever order the
// caller's ids give them.
std::vector<int64_t> morton_order(const HostMatrices& M) {
  const int64_t n = M.n;
  double lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    lo[d] = INFINITY;
    hi[d] = -INFINITY;
  }
  for (int64_t i = 0; i < n; ++i)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], M.xyz[3 * i + d]);
      hi[d] = std::max(hi[d], M.xyz[3 * i + d]);
    }
  const double ext = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]});
  const double s = ext > 0.0 ? (double)((1 << 21) - 1) / ext : 0.0;
  auto spread = [](uint64_t v) {  // 21 bits -> every third bit
    v &= 0x1fffffull;
    v = (v | v << 32) & 0x1f00000000ffffull;
    v = (v | v << 16) & 0x1f0000ff0000ffull;
    v = (v | v << 8) & 0x100f00f00f00f00full;
    v = (v | v << 4) & 0x10c30c30c30c30c3ull;
    v = (v | v << 2) & 0x1249249249249249ull;
    return v;
  };
  std::vector<std::pair<uint64_t, int64_t>> key(n);
  for (int64_t i = 0; i < n; ++i) {
    uint64_t k = 0;
    for (int d = 0; d < 3; ++d) {
      double q = (M.xyz[3 * i + d] - lo[d]) * s;
      q = std::min(std::max(q, 0.0), (double)((1 << 21) - 1));
      k |= spread((uint64_t)q) << d;
    }
    key[i] = {k, i};
  }
  std::sort(key.begin(), key.end());
  std::vector<int64_t> order(n);
  for (int64_t r = 0; r < n; ++r) order[r] = key[r].second;
  return order;
}

std::string build_sell(const HostMatrices& M, SellLayout& L, int renumber) {
  const int64_t n = M.n;
  L.n = n;
  L.perm.resize(n);
  L.iperm.resize(n);
  if (renumber == 2 && (M.xyz.size() != 3 * (size_t)n || M.offset.size() != M.col.size()))
    return "Morton row order needs node coordinates and cell offsets (a mesh upload)";
  if (renumber == 1 || renumber == 2) {
    L.iperm = renumber == 1 ? rcm_order(M) : morton_order(M);
    for (int64_t r = 0; r < n; ++r) L.perm[L.iperm[r]] = r;
  } else {
    for (int64_t i = 0; i < n; ++i) L.perm[i] = L.iperm[i] = i;  // caller order keeps mesh locality
  }
  L.n_slices = (n + kSlice - 1) / kSlice;
  L.slice_ptr.assign(L.n_slices + 1, 0);
  L.row_len.assign(n, 0);
  int64_t slots = 0;
  for (int64_t s = 0; s < L.n_slices; ++s) {
    int64_t w = 0;
    for (int64_t r = s * kSlice; r < std::min(n, (s + 1) * kSlice); ++r) {
      const int64_t i = L.iperm[r];
      w = std::max(w, M.rowptr[i + 1] - M.rowptr[i]);
    }
    slots += w * kSlice;
    if (slots > INT32_MAX) return "too many matrix entries for 32-bit slot indices";
    L.slice_ptr[s + 1] = (int32_t)slots;
  }
  L.n_slots = slots;
  L.col.assign(slots, 0);
  L.tpos.assign(slots, 0);
  L.flags.assign(slots, kEntryPad);
  L.cx.assign(slots, 0.0);
  L.cy.assign(slots, 0.0);
  L.cz.assign(slots, 0.0);
  L.mij.assign(slots, 0.0);
  L.cn.assign(slots, 0.0);
  L.inv_cn.assign(slots, 0.0);
  L.csx.assign(n, 0.0);
  L.csy.assign(n, 0.0);
  L.csz.assign(n, 0.0);
  L.mi.resize(n);
  L.inv_mi.resize(n);
  L.lam.resize(n);
  L.bc.assign(n, 0);
  L.slot_of_entry.assign(M.rowptr[n], -1);
  auto slot = [&](int64_t r, int64_t k) -> int64_t { return L.slice_ptr[r / kSlice] + k * kSlice + (r % kSlice); };
  std::vector<int64_t> ord;
  for (int64_t r = 0; r < n; ++r) {
    const int64_t i = L.iperm[r];
    const int64_t len = M.rowptr[i + 1] - M.rowptr[i];
    if (len < 2) return "a node has no neighbours";
    L.row_len[r] = (int32_t)len;
    // the lumped mass m_i = int phi_i equals the row sum of m_ij (partition of
    // unity); pre-assembled matrices may bring their own
    double m = 0.0;
    for (int64_t k = M.rowptr[i]; k < M.rowptr[i + 1]; ++k) m += M.mij[k];
    if (M.lumped_given) m = M.mi[i];
    L.mi[r] = m;
    L.inv_mi[r] = 1.0 / m;
    L.lam[r] = 1.0 / (double)(len - 1);
    L.bc[r] = M.bc.empty() ? 0 : M.bc[i];
    const int64_t w = (L.slice_ptr[r / kSlice + 1] - L.slice_ptr[r / kSlice]) / kSlice;
    for (int64_t k = 0; k < w; ++k) {  // padding slots point at the row itself
      const int64_t p = slot(r, k);
      L.col[p] = (int32_t)r;
      L.tpos[p] = (int32_t)p;
    }
    // the row's entries in the caller's column order, or (Morton order) by
    // their offset in the reference cell, then library column: the lanes of
    // a warp then gather, at each slot, the neighbours at one offset, as in a
    // lexicographic grid order
    ord.resize(len);
    for (int64_t k = 0; k < len; ++k) ord[k] = M.rowptr[i] + k;
    if (renumber == 2)
      std::sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) {
        const int oa = M.offset[a], ob = M.offset[b];
        return oa != ob ? oa < ob : L.perm[M.col[a]] < L.perm[M.col[b]];
      });
    for (int64_t k = 0; k < len; ++k) {
      const int64_t e = ord[k];
      const int64_t p = slot(r, k);
      const int64_t j = L.perm[M.col[e]];
      L.slot_of_entry[e] = p;
      L.col[p] = (int32_t)j;
      L.cx[p] = M.cij[0][e];
      L.cy[p] = M.cij[1][e];
      L.cz[p] = M.cij[2][e];
      L.mij[p] = M.mij[e];
      // |c_ij| and 1/|c_ij| once here (n_ij = c_ij/|c_ij|, Sec. 3.2): on GB300
      // a square root and a division cost more FP64 issue than loading them
      const double nc = std::sqrt(L.cx[p] * L.cx[p] + L.cy[p] * L.cy[p] + L.cz[p] * L.cz[p]);
      L.cn[p] = nc;
      L.inv_cn[p] = nc > 0.0 ? 1.0 / nc : 0.0;
      L.csx[r] += L.cx[p];
      L.csy[r] += L.cy[p];
      L.csz[r] += L.cz[p];
      uint8_t f = 0;
      if (j == r) f |= kEntryDiag;
      // the row of the smaller caller id evaluates the pair's wavespeed, so the
      // orientation does not depend on the row order; in Morton order the row
      // from which the other lies at a positive cell offset ((dz, dy, dx) > 0
      // lexicographically), so that the lanes of a warp agree at each slot
      if (renumber == 2 ? M.offset[e] > 13 : M.col[e] > i) f |= kEntryUpper;
      L.flags[p] = f;
    }
  }
  // transposed slots and bitwise skew pairs
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t e = M.rowptr[i]; e < M.rowptr[i + 1]; ++e) {
      const int64_t j = M.col[e];
      const int64_t* b = M.col.data() + M.rowptr[j];
      const int64_t* x = M.col.data() + M.rowptr[j + 1];
      const int64_t* q = std::lower_bound(b, x, i);
      if (q == x || *q != i) return "sparsity pattern is not structurally symmetric";
      const int64_t et = q - M.col.data();
      const int64_t p = L.slot_of_entry[e], pt = L.slot_of_entry[et];
      L.tpos[p] = (int32_t)pt;
      if (j != i && M.cij[0][et] == -M.cij[0][e] && M.cij[1][et] == -M.cij[1][e] && M.cij[2][et] == -M.cij[2][e])
        L.flags[p] |= kEntrySkew;
    }
  }
  return "";
}

}  // namespace idp
