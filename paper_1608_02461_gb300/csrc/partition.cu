// Partition of one FMM apply across ranks (host code only, no CUDA call).
//
// The octree of Sec. 5.1.1 is cut along the Morton curve of its leaf level
// into one contiguous range of leaves per rank, balanced by a per-leaf cost;
// this is the domain decomposition the paper's distributed runs use (MPI
// ranks, Sec. 7).  A rank owns the sources and targets of its leaves.  Its
// locally essential tree (LET) is what it needs from the other ranks for one
// apply:
//  - near field (P2P): the leaves of other ranks that hold sources and lie in
//    the near list of one of its target leaves;
//  - far field (M2L): at every level l >= 2, the cells in the M2L list of one
//    of its target cells (a cell holding one of its target leaves) that hold
//    a source leaf of another rank.  Each rank sends, for such a cell, the
//    partial multipole of its own leaves in it (the M of a cell is a sum over
//    its sources, so partial multipoles add).
// The lists are the library's own (the separation test of common.cuh, the
// near and M2L offset rules of the tree build).

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace {

bool valid_ranges(int64_t nleaf, int nranks, const int64_t* b) {
  if (b[0] != 0 || b[nranks] != nleaf) return false;
  for (int r = 0; r < nranks; ++r)
    if (b[r + 1] < b[r]) return false;
  return true;
}

// near offsets: cells of one level that are not well separated
std::vector<int> near_offsets(int64_t num, int64_t den) {
  const int R = (int)(den / num) + 1;
  std::vector<int> out;
  for (int dz = -R; dz <= R; ++dz)
    for (int dy = -R; dy <= R; ++dy)
      for (int dx = -R; dx <= R; ++dx)
        if (!separated(dx * dx + dy * dy + dz * dz, num, den)) {
          out.push_back(dx);
          out.push_back(dy);
          out.push_back(dz);
        }
  return out;
}

// M2L offsets of parity class b (bit 0 x, 1 y, 2 z): separated offsets whose
// parents are not separated
std::vector<int> m2l_offsets(int64_t num, int64_t den, int b) {
  const int Rn = (int)(den / num), box_r = 2 * Rn + 1;
  const int bx = b & 1, by = (b >> 1) & 1, bz = (b >> 2) & 1;
  std::vector<int> out;
  for (int dz = -box_r; dz <= box_r; ++dz)
    for (int dy = -box_r; dy <= box_r; ++dy)
      for (int dx = -box_r; dx <= box_r; ++dx) {
        if (!separated(dx * dx + dy * dy + dz * dz, num, den)) continue;
        const int px = floor_half(bx + dx), py = floor_half(by + dy), pz = floor_half(bz + dz);
        if (separated(px * px + py * py + pz * pz, num, den)) continue;
        out.push_back(dx);
        out.push_back(dy);
        out.push_back(dz);
      }
  return out;
}

}  // namespace

extern "C" int hfmm_partition_ranges(int L, const double* leaf_cost, int nranks, int64_t* leaf_begin) {
  if (L < 2 || L > HFMM_MAX_LEVEL - 1 || nranks < 1 || !leaf_begin) return HFMM_ERR_INVALID_ARG;
  const int64_t nleaf = (int64_t)1 << (3 * L);
  if (nranks > nleaf) return HFMM_ERR_INVALID_ARG;
  double total = 0.0;
  if (leaf_cost) {
    for (int64_t m = 0; m < nleaf; ++m) {
      const double c = leaf_cost[m];
      if (!(c >= 0.0) || !std::isfinite(c)) return HFMM_ERR_INVALID_ARG;
      total += c;
    }
  }
  const bool uniform = !leaf_cost || !(total > 0.0);
  if (uniform) total = (double)nleaf;
  auto cost = [&](int64_t m) { return uniform ? 1.0 : leaf_cost[m]; };
  std::vector<int64_t> b(nranks + 1);
  b[0] = 0;
  b[nranks] = nleaf;
  // rank r starts at the leaf where the running cost comes closest to
  // r / nranks of the total; every range holds at least one leaf
  int64_t m = 0;
  double pre = 0.0;  // cost of the leaves below m
  for (int r = 1; r < nranks; ++r) {
    const double target = total * r / nranks;
    while (m < nleaf && pre + cost(m) <= target) pre += cost(m++);
    int64_t cut = m;
    if (m < nleaf && (pre + cost(m)) - target < target - pre) cut = m + 1;
    cut = std::max(cut, b[r - 1] + 1);
    cut = std::min(cut, nleaf - (nranks - r));
    b[r] = cut;
    while (m < cut) pre += cost(m++);
  }
  std::copy(b.begin(), b.end(), leaf_begin);
  return HFMM_OK;
}

extern "C" int hfmm_partition_let(int L, double theta, int nranks, const int64_t* leaf_begin, int rank,
                                  const uint8_t* leaf_tgt, const uint8_t* leaf_src, int64_t* near_leaves,
                                  int64_t near_cap, int64_t* n_near, int64_t* cells, int64_t cells_cap,
                                  int64_t* cell_count) {
  if (L < 2 || L > HFMM_MAX_LEVEL - 1 || nranks < 1 || !leaf_begin || !n_near || !cell_count)
    return HFMM_ERR_INVALID_ARG;
  if (!(theta > 0.0 && theta <= 0.55) || rank < 0 || rank >= nranks) return HFMM_ERR_INVALID_ARG;
  const int64_t nleaf = (int64_t)1 << (3 * L);
  if (!valid_ranges(nleaf, nranks, leaf_begin)) return HFMM_ERR_INVALID_ARG;
  int64_t num = 0, den = 1;
  theta_rational(theta, num, den);
  const int64_t b0 = leaf_begin[rank], b1 = leaf_begin[rank + 1];
  auto tgt = [&](int64_t m) { return !leaf_tgt || leaf_tgt[m] != 0; };
  auto src = [&](int64_t m) { return !leaf_src || leaf_src[m] != 0; };
  auto mine = [&](int64_t m) { return m >= b0 && m < b1; };

  // near field: foreign source leaves in the near lists of the rank's target leaves
  const std::vector<int> noff = near_offsets(num, den);
  const int s = 1 << L;
  std::vector<uint8_t> need(nleaf, 0);
  for (int64_t m = b0; m < b1; ++m) {
    if (!tgt(m)) continue;
    int ix, iy, iz;
    morton_decode((uint64_t)m, ix, iy, iz);
    for (size_t i = 0; i < noff.size(); i += 3) {
      const int jx = ix + noff[i], jy = iy + noff[i + 1], jz = iz + noff[i + 2];
      if (jx < 0 || jy < 0 || jz < 0 || jx >= s || jy >= s || jz >= s) continue;
      const int64_t mj = (int64_t)morton_encode(jx, jy, jz);
      if (!mine(mj) && src(mj)) need[mj] = 1;
    }
  }
  std::vector<int64_t> nl;
  for (int64_t m = 0; m < nleaf; ++m)
    if (need[m]) nl.push_back(m);

  // far field, level by level
  std::vector<std::vector<int>> moff(8);
  for (int b = 0; b < 8; ++b) moff[b] = m2l_offsets(num, den, b);
  std::vector<int64_t> cl;
  int64_t cnt[HFMM_MAX_LEVEL + 1] = {0};
  for (int l = 2; l <= L; ++l) {
    const int shift = 3 * (L - l), sl = 1 << l;
    const int64_t ncell = (int64_t)1 << (3 * l);
    std::vector<uint8_t> tcell(ncell, 0), foreign(ncell, 0), want(ncell, 0);
    for (int64_t m = b0; m < b1; ++m)
      if (tgt(m)) tcell[m >> shift] = 1;
    for (int64_t m = 0; m < nleaf; ++m)
      if (!mine(m) && src(m)) foreign[m >> shift] = 1;
    for (int64_t c = 0; c < ncell; ++c) {
      if (!tcell[c]) continue;
      int ix, iy, iz;
      morton_decode((uint64_t)c, ix, iy, iz);
      const std::vector<int>& o = moff[(ix & 1) | ((iy & 1) << 1) | ((iz & 1) << 2)];
      for (size_t i = 0; i < o.size(); i += 3) {
        const int jx = ix + o[i], jy = iy + o[i + 1], jz = iz + o[i + 2];
        if (jx < 0 || jy < 0 || jz < 0 || jx >= sl || jy >= sl || jz >= sl) continue;
        const int64_t cj = (int64_t)morton_encode(jx, jy, jz);
        if (foreign[cj]) want[cj] = 1;
      }
    }
    for (int64_t c = 0; c < ncell; ++c)
      if (want[c]) {
        cl.push_back(c);
        ++cnt[l];
      }
  }
  if ((near_leaves == nullptr) != (cells == nullptr)) return HFMM_ERR_INVALID_ARG;
  if (near_leaves) {
    if (near_cap < (int64_t)nl.size() || cells_cap < (int64_t)cl.size()) return HFMM_ERR_INVALID_ARG;
    std::copy(nl.begin(), nl.end(), near_leaves);
    std::copy(cl.begin(), cl.end(), cells);
  }
  *n_near = (int64_t)nl.size();
  for (int l = 0; l <= L; ++l) cell_count[l] = cnt[l];
  return HFMM_OK;
}
