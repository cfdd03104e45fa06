// Tree construction on the device (Sec. 5.1.1: recursive subdivision of the
// cube into eight cells down to a uniform leaf level; Sec. 5.3: constant
// boundary elements centred at the boundary grid nodes off the edges).
//
//  - geometry: interior nodes (i,j,l) h and boundary panels, or caller points
//  - leaf keys: Morton code of floor(x 2^L) clamped to 2^L - 1
//  - counting sort into leaf order; inside a leaf, volume points first, then
//    boundary points, each set by original index (deterministic)
//  - per-level occupancy flags (bit 0 volume, bit 1 boundary)
//  - near list and per-parity M2L lists from the acceptance test
//    theta |d| > 1 (d in cell widths) evaluated in integers
//  - singular self terms of a cell and of a panel
#include <algorithm>
#include <cmath>
#include <vector>

#include "special.cuh"
#include "tree.cuh"

namespace {

__global__ void k_lattice_points(int n, double h, int64_t n_vol, int64_t n_bnd, double* xyz) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n_vol) {
    int64_t a = i % n, b = (i / n) % n, c = i / ((int64_t)n * n);
    xyz[3 * i + 0] = (a + 1) * h;
    xyz[3 * i + 1] = (b + 1) * h;
    xyz[3 * i + 2] = (c + 1) * h;
  } else if (i < n_vol + n_bnd) {
    int64_t j = i - n_vol;
    int64_t per = (int64_t)n * n;
    int face = (int)(j / per);
    int64_t r = j % per;
    int64_t u = r % n, v = r / n;
    int axis = face / 2;
    double val = (face & 1) ? 1.0 : 0.0;
    int f0 = axis == 0 ? 1 : 0;
    int f1 = axis == 2 ? 1 : 2;
    double x[3];
    x[axis] = val;
    x[f0] = (u + 1) * h;
    x[f1] = (v + 1) * h;
    xyz[3 * i + 0] = x[0];
    xyz[3 * i + 1] = x[1];
    xyz[3 * i + 2] = x[2];
  }
}

__device__ __forceinline__ int cell_coord(double x, int nl) {
  int c = (int)floor(x * nl);
  return c < 0 ? 0 : (c >= nl ? nl - 1 : c);
}

__global__ void k_leaf_keys_count(const double* xyz, int64_t n_vol, int64_t n_pts, int nl,
                                  int* key, int* cnt_vol, int* cnt_bnd) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_pts) return;
  int ix = cell_coord(xyz[3 * i], nl), iy = cell_coord(xyz[3 * i + 1], nl),
      iz = cell_coord(xyz[3 * i + 2], nl);
  int m = (int)morton_encode(ix, iy, iz);
  key[i] = m;
  atomicAdd(i < n_vol ? &cnt_vol[m] : &cnt_bnd[m], 1);
}

// exclusive scan of cnt_vol + cnt_bnd over nleaf entries; one block
__global__ void k_scan_leaves(const int* cnt_vol, const int* cnt_bnd, int nleaf, int* leaf_start,
                              int* leaf_mid, int* cursor_vol, int* cursor_bnd) {
  __shared__ int partial[1024];
  int tid = threadIdx.x;
  int chunk = (nleaf + blockDim.x - 1) / blockDim.x;
  int lo = tid * chunk, hi = min(nleaf, lo + chunk);
  int s = 0;
  for (int i = lo; i < hi; ++i) s += cnt_vol[i] + cnt_bnd[i];
  partial[tid] = s;
  __syncthreads();
  if (tid == 0) {
    int run = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) {
      int v = partial[i];
      partial[i] = run;
      run += v;
    }
    leaf_start[nleaf] = run;
  }
  __syncthreads();
  int run = partial[tid];
  for (int i = lo; i < hi; ++i) {
    leaf_start[i] = run;
    leaf_mid[i] = run + cnt_vol[i];
    cursor_vol[i] = run;
    cursor_bnd[i] = run + cnt_vol[i];
    run += cnt_vol[i] + cnt_bnd[i];
  }
}

__global__ void k_scatter(const int* key, int64_t n_vol, int64_t n_pts, int* cursor_vol,
                          int* cursor_bnd, int64_t* orig) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_pts) return;
  int m = key[i];
  int pos = atomicAdd(i < n_vol ? &cursor_vol[m] : &cursor_bnd[m], 1);
  orig[pos] = i;
}

// Order each leaf's volume and boundary segments by original id: the rank of
// an element is the number of smaller ids in its segment.
__global__ void k_sort_segments(const int* leaf_start, const int* leaf_mid, int64_t* orig,
                                int64_t* tmp) {
  int leaf = blockIdx.x;
  for (int part = 0; part < 2; ++part) {
    int lo = part == 0 ? leaf_start[leaf] : leaf_mid[leaf];
    int hi = part == 0 ? leaf_mid[leaf] : leaf_start[leaf + 1];
    int cnt = hi - lo;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      int64_t v = orig[lo + e];
      int rank = 0;
      for (int f = 0; f < cnt; ++f) rank += orig[lo + f] < v;
      tmp[lo + rank] = v;
    }
  }
}

// sorted FP64 coordinates, FP32 coordinates relative to the point's leaf
// centre (small numbers: differences inside the near field keep their
// relative precision in FP32), and the inverse permutation
__global__ void k_finalize_points(const int64_t* orig, const double* xyz_in, int64_t n_pts, int nl,
                                  double* xyz, float* xyz32, int64_t* pos_of) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_pts) return;
  int64_t o = orig[i];
  double x = xyz_in[3 * o], y = xyz_in[3 * o + 1], z = xyz_in[3 * o + 2];
  xyz[3 * i] = x;
  xyz[3 * i + 1] = y;
  xyz[3 * i + 2] = z;
  double w = 1.0 / nl;
  xyz32[4 * i] = (float)(x - (cell_coord(x, nl) + 0.5) * w);
  xyz32[4 * i + 1] = (float)(y - (cell_coord(y, nl) + 0.5) * w);
  xyz32[4 * i + 2] = (float)(z - (cell_coord(z, nl) + 0.5) * w);
  xyz32[4 * i + 3] = 0.f;
  pos_of[o] = i;
}

__global__ void k_leaf_flags(const int* cnt_vol, const int* cnt_bnd, int nleaf, int* flags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nleaf) return;
  flags[i] = (cnt_vol[i] > 0 ? 1 : 0) | (cnt_bnd[i] > 0 ? 2 : 0);
}

__global__ void k_parent_flags(const int* child_flags, int ncells, int* flags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ncells) return;
  int f = 0;
  for (int c = 0; c < 8; ++c) f |= child_flags[8 * i + c];
  flags[i] = f;
}

// ---- lists

__device__ __forceinline__ int pack_off(int dx, int dy, int dz) {
  return (dx + 128) | ((dy + 128) << 8) | ((dz + 128) << 16);
}

__global__ void k_near_list(int64_t num, int64_t den, int R, int* out, int* count) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int c = 0;
  for (int dz = -R; dz <= R; ++dz)
    for (int dy = -R; dy <= R; ++dy)
      for (int dx = -R; dx <= R; ++dx)
        if (!separated(dx * dx + dy * dy + dz * dz, num, den)) out[c++] = pack_off(dx, dy, dz);
  *count = c;
}

// one thread per parity class b = (bx, by, bz): offsets v in the box that are
// separated and whose parents (at offset floor((b + v)/2)) are not
__global__ void k_m2l_list(int64_t num, int64_t den, int box_r, int cap, int* off, int* box_index,
                           int* count) {
  int b = threadIdx.x;
  if (b >= 8 || blockIdx.x != 0) return;
  int bx = b & 1, by = (b >> 1) & 1, bz = (b >> 2) & 1;
  int w = 2 * box_r + 1;
  int c = 0;
  for (int dz = -box_r; dz <= box_r; ++dz)
    for (int dy = -box_r; dy <= box_r; ++dy)
      for (int dx = -box_r; dx <= box_r; ++dx) {
        if (!separated(dx * dx + dy * dy + dz * dz, num, den)) continue;
        int px = floor_half(bx + dx), py = floor_half(by + dy), pz = floor_half(bz + dz);
        if (separated(px * px + py * py + pz * pz, num, den)) continue;
        if (c < cap) {
          off[b * cap + c] = pack_off(dx, dy, dz);
          box_index[b * cap + c] = (dx + box_r) + w * ((dy + box_r) + w * (dz + box_r));
        }
        ++c;
      }
  count[b] = c;
}

// Distinct M2L offsets over the eight classes get operator slots in box
// order; the lists are repacked to stride `count[0]` and their box indices
// replaced by slots.  One thread (tiny, one-time).
__global__ void k_m2l_slots(int box, const int* count, int* off, int* box_index, int* slot,
                            int* slot_off, int* nslots) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int cnt = count[0];
  for (int i = 0; i < box; ++i) slot[i] = -1;
  for (int b = 0; b < 8; ++b)
    for (int i = 0; i < cnt; ++i) slot[box_index[b * box + i]] = 0;
  int ns = 0;
  for (int i = 0; i < box; ++i)
    if (slot[i] == 0) slot[i] = ns++;
  for (int b = 0; b < 8; ++b)
    for (int i = 0; i < cnt; ++i) {
      int o = off[b * box + i];
      int sl = slot[box_index[b * box + i]];
      slot_off[sl] = o;
      off[b * cnt + i] = o;
      box_index[b * cnt + i] = sl;
    }
  *nslots = ns;
}

// ---- active cells: one thread per (level, mask), Morton order

__global__ void k_active_cells(int L, const int* flags, const int64_t* level_off, int64_t stride, int* cells,
                               int* counts) {
  const int l = blockIdx.x, mi = threadIdx.x;
  if (mi >= 3 || l > L) return;
  const int mask = mi + 1;
  const int64_t off = level_off[l];
  const int nc = 1 << (3 * l);
  int* out = cells + mi * stride + off;
  int c = 0;
  for (int i = 0; i < nc; ++i)
    if (flags[off + i] & mask) out[c++] = i;
  counts[mi * (HFMM_MAX_LEVEL + 1) + l] = c;
}

// ---- M2L target tiles

// cells of level 2 + blockIdx.x whose flags meet mask blockIdx.y + 1, one
// thread per parity class b, in Morton order; region of class b at
// level_off[l] + b 8^(l-1)
__global__ void k_m2l_cells(const int* flags, const int64_t* level_off_dev, int* cells_all,
                            int64_t cells_stride, int* counts) {
  const int l = 2 + blockIdx.x;
  const int mask = blockIdx.y + 1;
  const int b = threadIdx.x;
  if (b >= 8) return;
  const int64_t off = level_off_dev[l];
  const int per = 1 << (3 * (l - 1));
  int* cells = cells_all + (mask - 1) * cells_stride + off + (int64_t)b * per;
  // grouped by the first cube face the cell touches (x=0, x=1, y=0, y=1,
  // z=0, z=1, none), Morton order within a group: cells of one tile then
  // share most of their far-field source pattern when only boundary cells
  // hold sources
  const int sl = 1 << l;
  int c = 0;
  for (int g = 0; g < 7; ++g)
    for (int j = 0; j < per; ++j) {
      int cell = 8 * j + b;
      if (!(flags[off + cell] & mask)) continue;
      int ix, iy, iz;
      morton_decode((uint64_t)cell, ix, iy, iz);
      int key = ix == 0 ? 0 : ix == sl - 1 ? 1 : iy == 0 ? 2 : iy == sl - 1 ? 3 : iz == 0 ? 4
                : iz == sl - 1 ? 5 : 6;
      if (key == g) cells[c++] = cell;
    }
  counts[((mask - 1) * (HFMM_MAX_LEVEL + 1) + l) * 8 + b] = c;
}

// one thread per mask: tiles of at most tc cells of one (level, class)
__global__ void k_m2l_tiles(int L, int tc, const int64_t* level_off_dev, const int* counts,
                            int4* tiles_all, int64_t tiles_stride, int* ntiles) {
  const int mi = threadIdx.x;
  if (mi >= 3) return;
  int4* tiles = tiles_all + mi * tiles_stride;
  int n = 0;
  for (int l = 2; l <= L; ++l) {
    const int per = 1 << (3 * (l - 1));
    for (int b = 0; b < 8; ++b) {
      int cnt = counts[(mi * (HFMM_MAX_LEVEL + 1) + l) * 8 + b];
      int64_t base = level_off_dev[l] + (int64_t)b * per;
      for (int st = 0; st < cnt; st += tc) tiles[n++] = make_int4(l, b, (int)(base + st), min(tc, cnt - st));
    }
  }
  ntiles[mi] = n;
}

// ---- algorithmic work counts (statistics and roofline accounting)

__global__ void k_count_m2l(int level, const int* flags, const int* m2l_off, int m2l_count,
                            unsigned long long* cnt) {
  __shared__ unsigned long long loc[16];
  if (threadIdx.x < 16) loc[threadIdx.x] = 0;
  __syncthreads();
  int cell = blockIdx.x * blockDim.x + threadIdx.x;
  int s = 1 << level;
  if (cell < s * s * s) {
    int ft = flags[cell];
    int b = cell & 7;
    int ix, iy, iz;
    morton_decode((uint64_t)cell, ix, iy, iz);
    unsigned long long c[4] = {0, 0, 0, 0};
    for (int i = 0; i < m2l_count; ++i) {
      int o = m2l_off[b * m2l_count + i];
      int jx = ix + (o & 255) - 128, jy = iy + ((o >> 8) & 255) - 128, jz = iz + ((o >> 16) & 255) - 128;
      if (jx < 0 || jy < 0 || jz < 0 || jx >= s || jy >= s || jz >= s) continue;
      c[flags[morton_encode(jx, jy, jz)]]++;
    }
    for (int f = 0; f < 4; ++f)
      if (c[f]) atomicAdd(&loc[ft * 4 + f], c[f]);
  }
  __syncthreads();
  if (threadIdx.x < 16 && loc[threadIdx.x]) atomicAdd(&cnt[threadIdx.x], loc[threadIdx.x]);
}

__global__ void k_count_p2p(int L, const int* leaf_start, const int* leaf_mid, const int* near_off,
                            int near_count, unsigned long long* cnt) {
  int leaf = blockIdx.x * blockDim.x + threadIdx.x;
  int s = 1 << L;
  if (leaf >= s * s * s) return;
  unsigned long long tv = leaf_mid[leaf] - leaf_start[leaf], tb = leaf_start[leaf + 1] - leaf_mid[leaf];
  if (tv + tb == 0) return;
  int ix, iy, iz;
  morton_decode((uint64_t)leaf, ix, iy, iz);
  unsigned long long sv = 0, sb = 0;
  for (int i = 0; i < near_count; ++i) {
    int o = near_off[i];
    int jx = ix + (o & 255) - 128, jy = iy + ((o >> 8) & 255) - 128, jz = iz + ((o >> 16) & 255) - 128;
    if (jx < 0 || jy < 0 || jz < 0 || jx >= s || jy >= s || jz >= s) continue;
    int m = (int)morton_encode(jx, jy, jz);
    sv += leaf_mid[m] - leaf_start[m];
    sb += leaf_start[m + 1] - leaf_mid[m];
  }
  atomicAdd(&cnt[0], tv * sv);
  atomicAdd(&cnt[1], tv * sb);
  atomicAdd(&cnt[2], tb * sv);
  atomicAdd(&cnt[3], tb * sb);
}

// ---- self terms

// radial integrals along a ray of length R from the singular point:
//   Iv(a) = int_0^1 s e^{i a s} ds   (volume: s^2 ds times 1/(s R))
//   Ip(a) = int_0^1 e^{i a s} ds     (panel:  s ds times 1/(s R))
__device__ double2 radial_vol(double a) {
  if (a < 1.0) {  // sum_m (i a)^m / (m! (m + 2))
    double2 s = make_double2(0, 0), t = make_double2(1, 0);  // t = (ia)^m / m!
    for (int m = 0; m < 40; ++m) {
      s.x += t.x / (m + 2);
      s.y += t.y / (m + 2);
      double2 tn = make_double2(-t.y * a / (m + 1), t.x * a / (m + 1));
      t = tn;
    }
    return s;
  }
  double sa, ca;
  sincos(a, &sa, &ca);
  // e^{ia}/(ia) + (e^{ia} - 1)/a^2
  return make_double2(sa / a + (ca - 1.0) / (a * a), -ca / a + sa / (a * a));
}
__device__ double2 radial_panel(double a) {
  if (a < 1.0) {  // sum_m (i a)^m / (m + 1)!
    double2 s = make_double2(0, 0), t = make_double2(1, 0);  // (ia)^m / (m+1)!
    for (int m = 0; m < 40; ++m) {
      s.x += t.x;
      s.y += t.y;
      double2 tn = make_double2(-t.y * a / (m + 2), t.x * a / (m + 2));
      t = tn;
    }
    return s;
  }
  double sa, ca;
  sincos(a, &sa, &ca);
  // (e^{ia} - 1)/(ia)
  return make_double2(sa / a, (1.0 - ca) / a);
}

// s_vol = 6 (h/2) int_{face} Iv(k R) / (4 pi R) dA,  R = |(h/2, u, v)|
// s_bnd = 4 (h/2) int_{edge} Ip(k R) / (4 pi R) du,  R = |(h/2, u)|
// (pyramids / triangles with apex at the singular point, radial part exact)
// and their k-derivatives, from d/dk Iv(k R) = R Iv'(k R), Iv'(a) = i int_0^1 s^2 e^{ias} ds,
// Ip'(a) = i int_0^1 s e^{ias} ds = i Iv(a).
__device__ double2 radial_vol_d(double a) {  // i int_0^1 s^2 e^{ias} ds
  double2 v;
  if (a < 1.0) {  // sum_m (i a)^m / (m! (m + 3))
    double2 s = make_double2(0, 0), t = make_double2(1, 0);
    for (int m = 0; m < 40; ++m) {
      s.x += t.x / (m + 3);
      s.y += t.y / (m + 3);
      double2 tn = make_double2(-t.y * a / (m + 1), t.x * a / (m + 1));
      t = tn;
    }
    v = s;
  } else {  // e^{ia}/(ia) - (2/(ia)) Iv(a)
    double sa, ca;
    sincos(a, &sa, &ca);
    double2 I = radial_vol(a);
    // 1/(ia) = -i/a
    double2 e = make_double2(sa / a, -ca / a);
    double2 t2 = make_double2(2.0 * I.y / a, -2.0 * I.x / a);  // (2/(ia)) I = -2i I / a
    v = make_double2(e.x - t2.x, e.y - t2.y);
  }
  return make_double2(-v.y, v.x);  // times i
}

__global__ void k_self_terms(double h, double k, double2* out) {
  constexpr int NQ = 32;
  __shared__ double xg[NQ], wg[NQ];
  __shared__ double2 red[256], red2[256];
  if (threadIdx.x == 0) gauss_legendre(NQ, xg, wg);
  __syncthreads();
  const double hh = 0.5 * h;
  const double inv4pi = 0.25 / M_PI;
  double2 acc = make_double2(0, 0), accd = make_double2(0, 0);
  for (int q = threadIdx.x; q < NQ * NQ; q += blockDim.x) {
    int i = q % NQ, j = q / NQ;
    double u = hh * xg[i], v = hh * xg[j];
    double R = sqrt(hh * hh + u * u + v * v);
    double2 I = radial_vol(k * R);
    double2 Id = radial_vol_d(k * R);
    double wt = hh * wg[i] * hh * wg[j] * inv4pi;
    acc.x += wt / R * I.x;
    acc.y += wt / R * I.y;
    accd.x += wt * Id.x;
    accd.y += wt * Id.y;
  }
  red[threadIdx.x] = acc;
  red2[threadIdx.x] = accd;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      red[threadIdx.x].x += red[threadIdx.x + s].x;
      red[threadIdx.x].y += red[threadIdx.x + s].y;
      red2[threadIdx.x].x += red2[threadIdx.x + s].x;
      red2[threadIdx.x].y += red2[threadIdx.x + s].y;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = make_double2(6 * hh * red[0].x, 6 * hh * red[0].y);
    out[2] = make_double2(6 * hh * red2[0].x, 6 * hh * red2[0].y);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 a2 = make_double2(0, 0), a2d = make_double2(0, 0);
    for (int i = 0; i < NQ; ++i) {
      double u = hh * xg[i];
      double R = sqrt(hh * hh + u * u);
      double2 I = radial_panel(k * R);
      double2 Iv = radial_vol(k * R);  // Ip'(a) = i Iv(a)
      double wt = hh * wg[i] * inv4pi;
      a2.x += wt / R * I.x;
      a2.y += wt / R * I.y;
      a2d.x += wt * (-Iv.y);
      a2d.y += wt * Iv.x;
    }
    out[1] = make_double2(4 * hh * a2.x, 4 * hh * a2.y);
    out[3] = make_double2(4 * hh * a2d.x, 4 * hh * a2d.y);
  }
}


// ---------------------------------------------------------------- lattice near-field table

// integer lattice coordinates of each leaf's points: min and max per axis
// (min > max for an empty leaf)
__global__ void k_leaf_lat_box(const double* __restrict__ xyz, const int* __restrict__ leaf_start, int nleaf,
                               double inv_h, int* __restrict__ box) {
  const int leaf = blockIdx.x * blockDim.x + threadIdx.x;
  if (leaf >= nleaf) return;
  int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
  for (int i = leaf_start[leaf]; i < leaf_start[leaf + 1]; ++i)
    for (int a = 0; a < 3; ++a) {
      const int c = (int)llrint(xyz[3 * (int64_t)i + a] * inv_h);
      lo[a] = min(lo[a], c);
      hi[a] = max(hi[a], c);
    }
  for (int a = 0; a < 3; ++a) {
    box[6 * leaf + a] = lo[a];
    box[6 * leaf + 3 + a] = hi[a];
  }
}

// largest |offset component| between points of a leaf and of its near leaves
__global__ void k_lat_max_offset(const int* __restrict__ box, int L, const int* __restrict__ near_off,
                                 int near_count, int* __restrict__ dmax) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int nleaf = 1 << (3 * L);
  if (tid >= (int64_t)nleaf * near_count) return;
  const int leaf = (int)(tid / near_count), q = (int)(tid % near_count);
  const int* bt = box + 6 * leaf;
  if (bt[0] > bt[3]) return;
  const int o = near_off[q];
  int ix, iy, iz;
  morton_decode((uint64_t)leaf, ix, iy, iz);
  const int s = 1 << L;
  const int jx = ix + (o & 255) - 128, jy = iy + ((o >> 8) & 255) - 128, jz = iz + ((o >> 16) & 255) - 128;
  if (jx < 0 || jy < 0 || jz < 0 || jx >= s || jy >= s || jz >= s) return;
  const int* bs = box + 6 * (int)morton_encode(jx, jy, jz);
  if (bs[0] > bs[3]) return;
  int m = 0;
  for (int a = 0; a < 3; ++a) m = max(m, max(bt[3 + a] - bs[a], bs[3 + a] - bt[a]));
  atomicMax(dmax, m);
}

__global__ void k_lat_lin(const double* __restrict__ xyz, int64_t n, double inv_h, int Sy, int Sz,
                          int* __restrict__ lin) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int cx = (int)llrint(xyz[3 * i] * inv_h), cy = (int)llrint(xyz[3 * i + 1] * inv_h),
            cz = (int)llrint(xyz[3 * i + 2] * inv_h);
  lin[i] = cx + Sy * cy + Sz * cz;
}

// signed residue of r modulo m in [-(m/2), m - m/2)
__device__ __forceinline__ int64_t balanced_mod(int64_t r, int64_t m) {
  int64_t v = ((r % m) + m) % m;
  if (v >= m - m / 2) v -= m;
  return v;
}

// half table over delta = dx + Sy dy + Sz dz >= 0 (dx, dy, dz in [-D, D],
// Sy > 2D, Sz = (2D + 1) Sy): G(h d) = e^{i k h |d|} / (4 pi h |d|) (the 3D
// Green's function of Sec. 5.2 on the lattice), zero at d = 0 and at codes
// that no offset of the box produces
__global__ void k_lat_table(int D, int Sy, int Sz, double h, double k, int64_t nhalf, int64_t npad,
                            double2* __restrict__ t64, float2* __restrict__ t32) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= npad) return;
  double2 g = make_double2(0.0, 0.0);
  if (e < nhalf) {
    const int64_t dx = balanced_mod(e, Sy);
    const int64_t r = (e - dx) / Sy;  // dy + (Sz / Sy) dz
    const int64_t W = Sz / Sy;
    const int64_t dy = balanced_mod(r, W);
    const int64_t dz = (r - dy) / W;
    const bool inbox = dx >= -D && dx <= D && dy >= -D && dy <= D && dz >= -D && dz <= D;
    const int64_t d2 = dx * dx + dy * dy + dz * dz;
    if (inbox && d2 > 0) {
      const double rr = h * sqrt((double)d2);
      double sn, cs;
      sincos(k * rr, &sn, &cs);
      const double a = 0.07957747154594766788 / rr;
      g = make_double2(a * cs, a * sn);
    }
  }
  t64[e] = g;
  t32[e] = make_float2((float)g.x, (float)g.y);
}

}  // namespace

int build_geometry_and_sort(fmm_tree* t, const double* d_vol, const double* d_bnd, cudaStream_t s) {
  const int64_t N = t->n_pts;
  const int nleaf = 1 << (3 * t->L);
  double* xyz_in = nullptr;
  int *key = nullptr, *cnt_vol = nullptr, *cnt_bnd = nullptr, *cur_vol = nullptr, *cur_bnd = nullptr;
  int64_t* tmp = nullptr;
  HFMM_CUDA_TRY(cudaMallocAsync((void**)&xyz_in, sizeof(double) * 3 * std::max<int64_t>(N, 1), s));
  HFMM_CUDA_TRY(cudaMallocAsync((void**)&key, sizeof(int) * std::max<int64_t>(N, 1), s));
  HFMM_CUDA_TRY(cudaMallocAsync((void**)&cnt_vol, sizeof(int) * nleaf * 4, s));
  HFMM_CUDA_TRY(cudaMallocAsync((void**)&tmp, sizeof(int64_t) * std::max<int64_t>(N, 1), s));
  cnt_bnd = cnt_vol + nleaf;
  cur_vol = cnt_vol + 2 * nleaf;
  cur_bnd = cnt_vol + 3 * nleaf;
  HFMM_CUDA_TRY(cudaMemsetAsync(cnt_vol, 0, sizeof(int) * nleaf * 2, s));

  if (t->lattice) {
    k_lattice_points<<<ceil_div(N, 256), 256, 0, s>>>(t->n, t->h, t->n_vol, t->n_bnd, xyz_in);
  } else {
    if (t->n_vol) HFMM_CUDA_TRY(cudaMemcpyAsync(xyz_in, d_vol, sizeof(double) * 3 * t->n_vol,
                                                cudaMemcpyDeviceToDevice, s));
    if (t->n_bnd) HFMM_CUDA_TRY(cudaMemcpyAsync(xyz_in + 3 * t->n_vol, d_bnd,
                                                sizeof(double) * 3 * t->n_bnd,
                                                cudaMemcpyDeviceToDevice, s));
  }
  k_leaf_keys_count<<<ceil_div(N, 256), 256, 0, s>>>(xyz_in, t->n_vol, N, t->nlv, key, cnt_vol,
                                                     cnt_bnd);
  k_scan_leaves<<<1, 1024, 0, s>>>(cnt_vol, cnt_bnd, nleaf, t->leaf_start, t->leaf_mid, cur_vol,
                                   cur_bnd);
  k_scatter<<<ceil_div(N, 256), 256, 0, s>>>(key, t->n_vol, N, cur_vol, cur_bnd, t->orig);
  k_sort_segments<<<nleaf, 128, 0, s>>>(t->leaf_start, t->leaf_mid, t->orig, tmp);
  HFMM_CUDA_TRY(cudaMemcpyAsync(t->orig, tmp, sizeof(int64_t) * N, cudaMemcpyDeviceToDevice, s));
  k_finalize_points<<<ceil_div(N, 256), 256, 0, s>>>(t->orig, xyz_in, N, t->nlv, t->xyz,
                                                     t->xyz32, t->pos_of);
  // occupancy flags, leaf level then upwards
  k_leaf_flags<<<ceil_div(nleaf, 256), 256, 0, s>>>(cnt_vol, cnt_bnd, nleaf,
                                                    t->flags + t->level_off[t->L]);
  for (int l = t->L - 1; l >= 0; --l) {
    int nc = 1 << (3 * l);
    k_parent_flags<<<ceil_div(nc, 256), 256, 0, s>>>(t->flags + t->level_off[l + 1], nc,
                                                     t->flags + t->level_off[l]);
  }
  HFMM_TRY(hfmm_last_launch());
  // near-field pair count (statistics)
  std::vector<int> hv(nleaf), hb(nleaf);
  HFMM_CUDA_TRY(cudaMemcpyAsync(hv.data(), cnt_vol, sizeof(int) * nleaf, cudaMemcpyDeviceToHost, s));
  HFMM_CUDA_TRY(cudaMemcpyAsync(hb.data(), cnt_bnd, sizeof(int) * nleaf, cudaMemcpyDeviceToHost, s));
  HFMM_CUDA_TRY(cudaStreamSynchronize(s));
  t->p2p_pairs = 0;
  {
    const int R = (int)(t->th_den / t->th_num) + 1;
    for (int m = 0; m < nleaf; ++m) {
      int64_t cm = hv[m] + hb[m];
      if (!cm) continue;
      int ix, iy, iz;
      morton_decode((uint64_t)m, ix, iy, iz);
      for (int dz = -R; dz <= R; ++dz)
        for (int dy = -R; dy <= R; ++dy)
          for (int dx = -R; dx <= R; ++dx) {
            int64_t d2 = dx * dx + dy * dy + dz * dz;
            if (t->th_num * t->th_num * d2 > t->th_den * t->th_den) continue;
            int jx = ix + dx, jy = iy + dy, jz = iz + dz;
            if (jx < 0 || jy < 0 || jz < 0 || jx >= t->nlv || jy >= t->nlv || jz >= t->nlv) continue;
            int o = (int)morton_encode(jx, jy, jz);
            t->p2p_pairs += cm * (hv[o] + hb[o]);
          }
    }
    t->p2p_pairs -= N;  // j != i
  }
  cudaFreeAsync(xyz_in, s);
  cudaFreeAsync(key, s);
  cudaFreeAsync(cnt_vol, s);
  cudaFreeAsync(tmp, s);
  return hfmm_last_launch();
}

int build_lists(fmm_tree* t, cudaStream_t s) {
  const int Rn = (int)(t->th_den / t->th_num);  // floor(1/theta): near offsets lie in [-Rn, Rn]
  t->box_r = 2 * Rn + 1;                         // M2L offsets: 2u + c - b with |u| <= Rn
  const int w = 2 * t->box_r + 1;
  const int box = w * w * w;
  int* d_count = nullptr;
  int* d_slot = nullptr;
  HFMM_CUDA_TRY(cudaMallocAsync((void**)&d_count, sizeof(int) * 16, s));
  HFMM_CUDA_TRY(cudaMallocAsync((void**)&d_slot, sizeof(int) * box, s));
  const int near_cap = (2 * Rn + 3) * (2 * Rn + 3) * (2 * Rn + 3);
  HFMM_TRY(tree_alloc_t(t, &t->near_off, near_cap));
  k_near_list<<<1, 1, 0, s>>>(t->th_num, t->th_den, Rn + 1, t->near_off, d_count);
  HFMM_TRY(tree_alloc_t(t, &t->m2l_off, 8 * box));
  HFMM_TRY(tree_alloc_t(t, &t->m2l_box_index, 8 * box));
  HFMM_TRY(tree_alloc_t(t, &t->m2l_slot_off, box));
  k_m2l_list<<<1, 32, 0, s>>>(t->th_num, t->th_den, t->box_r, box, t->m2l_off, t->m2l_box_index,
                              d_count + 1);
  k_m2l_slots<<<1, 1, 0, s>>>(box, d_count + 1, t->m2l_off, t->m2l_box_index, d_slot,
                              t->m2l_slot_off, d_count + 9);
  HFMM_TRY(hfmm_last_launch());
  int hc[10];
  HFMM_CUDA_TRY(cudaMemcpyAsync(hc, d_count, sizeof(int) * 10, cudaMemcpyDeviceToHost, s));
  HFMM_CUDA_TRY(cudaStreamSynchronize(s));
  cudaFreeAsync(d_count, s);
  cudaFreeAsync(d_slot, s);
  t->near_count = hc[0];
  for (int b = 1; b < 8; ++b)
    if (hc[1 + b] != hc[1]) return HFMM_ERR_UNSUPPORTED;
  t->m2l_count = hc[1];
  t->box_cells = hc[9];  // number of distinct M2L offsets = operator slots per level
  // statistics: far-field cell pairs over all levels, every cell a target
  std::vector<int> off(8 * (size_t)box);
  HFMM_CUDA_TRY(cudaMemcpy(off.data(), t->m2l_off, sizeof(int) * off.size(), cudaMemcpyDeviceToHost));
  t->m2l_pairs = 0;
  for (int l = 2; l <= t->L; ++l) {
    int sl = 1 << l;
    for (int b = 0; b < 8; ++b) {
      int bb[3] = {b & 1, (b >> 1) & 1, (b >> 2) & 1};
      for (int i = 0; i < t->m2l_count; ++i) {
        int o = off[(size_t)b * t->m2l_count + i];
        int d[3] = {(o & 255) - 128, ((o >> 8) & 255) - 128, ((o >> 16) & 255) - 128};
        int64_t cnt = 1;
        for (int ax = 0; ax < 3; ++ax) {
          int64_t c = 0;
          for (int x = bb[ax]; x < sl; x += 2)
            if (x + d[ax] >= 0 && x + d[ax] < sl) ++c;
          cnt *= c;
        }
        t->m2l_pairs += cnt;
      }
    }
  }
  return HFMM_OK;
}

int build_self_terms(fmm_tree* t, cudaStream_t s) {
  if (!t->lattice) {
    t->s_vol = t->s_bnd = t->sigma_vol = t->sigma_bnd = make_double2(0, 0);
    return HFMM_OK;
  }
  double2* d = nullptr;
  HFMM_CUDA_TRY(cudaMallocAsync((void**)&d, sizeof(double2) * 4, s));
  k_self_terms<<<1, 256, 0, s>>>(t->h, t->k, d);
  HFMM_TRY(hfmm_last_launch());
  double2 hs[4];
  HFMM_CUDA_TRY(cudaMemcpyAsync(hs, d, sizeof(hs), cudaMemcpyDeviceToHost, s));
  HFMM_CUDA_TRY(cudaStreamSynchronize(s));
  cudaFreeAsync(d, s);
  t->s_vol = hs[0];
  t->s_bnd = hs[1];
  const double h3 = t->h * t->h * t->h, h2 = t->h * t->h;
  t->sigma_vol = make_double2(hs[0].x / h3, hs[0].y / h3);
  t->sigma_bnd = make_double2(hs[1].x / h2, hs[1].y / h2);
  t->dsigma_vol = make_double2(hs[2].x / h3, hs[2].y / h3);
  t->dsigma_bnd = make_double2(hs[3].x / h2, hs[3].y / h2);
  return HFMM_OK;
}

int build_pair_counts(fmm_tree* t, cudaStream_t s) {
  unsigned long long* d = nullptr;
  const int nc = (HFMM_MAX_LEVEL + 1) * 16 + 4;
  HFMM_CUDA_TRY(cudaMallocAsync((void**)&d, sizeof(unsigned long long) * nc, s));
  HFMM_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(unsigned long long) * nc, s));
  for (int l = 2; l <= t->L; ++l) {
    int ncell = 1 << (3 * l);
    k_count_m2l<<<ceil_div(ncell, 128), 128, 0, s>>>(l, t->flags + t->level_off[l], t->m2l_off,
                                                      t->m2l_count, d + l * 16);
  }
  int nleaf = 1 << (3 * t->L);
  k_count_p2p<<<ceil_div(nleaf, 128), 128, 0, s>>>(t->L, t->leaf_start, t->leaf_mid, t->near_off,
                                                    t->near_count, d + (HFMM_MAX_LEVEL + 1) * 16);
  HFMM_TRY(hfmm_last_launch());
  std::vector<unsigned long long> h(nc);
  HFMM_CUDA_TRY(cudaMemcpyAsync(h.data(), d, sizeof(unsigned long long) * nc, cudaMemcpyDeviceToHost, s));
  HFMM_CUDA_TRY(cudaStreamSynchronize(s));
  cudaFreeAsync(d, s);
  for (int l = 0; l <= HFMM_MAX_LEVEL; ++l)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) t->m2l_cnt[l][a][b] = (int64_t)h[l * 16 + a * 4 + b];
  for (int i = 0; i < 4; ++i) t->p2p_cnt[i] = (int64_t)h[(HFMM_MAX_LEVEL + 1) * 16 + i];
  return HFMM_OK;
}

double p2p_work(const fmm_tree* t, int src_set, int tgt_set) {
  double w = 0;
  for (int ti = 0; ti < 2; ++ti)
    for (int si = 0; si < 2; ++si)
      if ((tgt_set & (1 << ti)) && (src_set & (1 << si))) w += (double)t->p2p_cnt[2 * ti + si];
  // j != i: a point that is both source and target does not meet itself
  if ((src_set & tgt_set) & HFMM_SET_VOL) w -= (double)t->n_vol;
  if ((src_set & tgt_set) & HFMM_SET_BND) w -= (double)t->n_bnd;
  return w;
}

double m2l_work(const fmm_tree* t, int src_set, int tgt_set) {
  double pairs = 0;
  for (int l = 2; l <= t->L; ++l)
    for (int ft = 0; ft < 4; ++ft)
      for (int fs = 0; fs < 4; ++fs)
        if ((ft & tgt_set) && (fs & src_set)) pairs += (double)t->m2l_cnt[l][ft][fs];
  return 8.0 * t->P * t->P * pairs;
}

int build_m2l_tiles(fmm_tree* t, cudaStream_t s) {
  // tile width: 32 target cells (the offset lists are split over blocks when
  // that gives too few tiles for the GPU)
  int64_t cells_l = 0;
  for (int l = 2; l <= t->L; ++l) cells_l += (int64_t)1 << (3 * l);
  t->m2l_tc = 32;
  const int64_t cstride = t->total_cells;
  const int64_t tstride = cells_l / t->m2l_tc + 8 * (t->L + 1) + 8;
  int* cells = nullptr;
  int4* tiles = nullptr;
  HFMM_TRY(tree_alloc_t(t, &cells, 3 * cstride));
  HFMM_TRY(tree_alloc_t(t, &tiles, 3 * tstride));
  int* d_counts = nullptr;
  int64_t* d_off = nullptr;
  const int ncount = 3 * (HFMM_MAX_LEVEL + 1) * 8 + 4;
  HFMM_CUDA_TRY(cudaMallocAsync((void**)&d_counts, sizeof(int) * ncount, s));
  HFMM_CUDA_TRY(cudaMallocAsync((void**)&d_off, sizeof(t->level_off), s));
  HFMM_CUDA_TRY(cudaMemsetAsync(d_counts, 0, sizeof(int) * ncount, s));
  HFMM_CUDA_TRY(cudaMemcpyAsync(d_off, t->level_off, sizeof(t->level_off), cudaMemcpyHostToDevice, s));
  k_m2l_cells<<<dim3(t->L - 1, 3), 32, 0, s>>>(t->flags, d_off, cells, cstride, d_counts);
  k_m2l_tiles<<<1, 32, 0, s>>>(t->L, t->m2l_tc, d_off, d_counts, tiles, tstride,
                               d_counts + 3 * (HFMM_MAX_LEVEL + 1) * 8);
  HFMM_TRY(hfmm_last_launch());
  int nt[3];
  HFMM_CUDA_TRY(cudaMemcpyAsync(nt, d_counts + 3 * (HFMM_MAX_LEVEL + 1) * 8, sizeof(nt),
                                cudaMemcpyDeviceToHost, s));
  HFMM_CUDA_TRY(cudaStreamSynchronize(s));
  cudaFreeAsync(d_counts, s);
  cudaFreeAsync(d_off, s);
  for (int i = 0; i < 3; ++i) {
    t->m2l_cells[i] = cells + i * cstride;
    t->m2l_tiles[i] = tiles + i * tstride;
    t->m2l_ntiles[i] = nt[i];
    // tiles are in level order: count those below each level
    std::vector<int4> ht(nt[i]);
    if (nt[i] > 0)
      HFMM_CUDA_TRY(cudaMemcpy(ht.data(), t->m2l_tiles[i], sizeof(int4) * nt[i], cudaMemcpyDeviceToHost));
    for (int l = 0; l <= HFMM_MAX_LEVEL + 1; ++l) {
      int c = 0;
      for (const int4& tl : ht) c += tl.x < l ? 1 : 0;
      t->m2l_tiles_lt[i][l] = c;
    }
  }
  return HFMM_OK;
}

int build_active_lists(fmm_tree* t, cudaStream_t s) {
  int* cells = nullptr;
  HFMM_TRY(tree_alloc_t(t, &cells, 3 * t->total_cells));
  int* d_cnt = nullptr;
  const int nc = 3 * (HFMM_MAX_LEVEL + 1);
  HFMM_CUDA_TRY(cudaMallocAsync((void**)&d_cnt, sizeof(int) * nc, s));
  HFMM_CUDA_TRY(cudaMemsetAsync(d_cnt, 0, sizeof(int) * nc, s));
  k_active_cells<<<t->L + 1, 32, 0, s>>>(t->L, t->flags, t->level_off_dev, t->total_cells, cells, d_cnt);
  HFMM_TRY(hfmm_last_launch());
  int h[3 * (HFMM_MAX_LEVEL + 1)];
  HFMM_CUDA_TRY(cudaMemcpyAsync(h, d_cnt, sizeof(h), cudaMemcpyDeviceToHost, s));
  HFMM_CUDA_TRY(cudaStreamSynchronize(s));
  cudaFreeAsync(d_cnt, s);
  for (int m = 0; m < 3; ++m) {
    t->act_cells[m] = cells + m * t->total_cells;
    for (int l = 0; l <= HFMM_MAX_LEVEL; ++l) t->act_count[m][l] = h[m * (HFMM_MAX_LEVEL + 1) + l];
  }
  return HFMM_OK;
}

int build_lattice_table(fmm_tree* t, cudaStream_t s) {
  t->lat_D = 0;
  if (!t->lattice || t->near_count == 0) return HFMM_OK;
  const int nleaf = 1 << (3 * t->L);
  const double inv_h = 1.0 / t->h;
  int *box = nullptr, *dmax = nullptr;
  HFMM_CUDA_TRY(cudaMallocAsync((void**)&box, sizeof(int) * 6 * nleaf + sizeof(int) * 64, s));
  dmax = box + 6 * nleaf;
  HFMM_CUDA_TRY(cudaMemsetAsync(dmax, 0, sizeof(int), s));
  k_leaf_lat_box<<<ceil_div(nleaf, 128), 128, 0, s>>>(t->xyz, t->leaf_start, nleaf, inv_h, box);
  k_lat_max_offset<<<ceil_div((int64_t)nleaf * t->near_count, 256), 256, 0, s>>>(box, t->L, t->near_off,
                                                                                 t->near_count, dmax);
  HFMM_TRY(hfmm_last_launch());
  int D = 0;
  HFMM_CUDA_TRY(cudaMemcpyAsync(&D, dmax, sizeof(int), cudaMemcpyDeviceToHost, s));
  HFMM_CUDA_TRY(cudaStreamSynchronize(s));
  cudaFreeAsync(box, s);
  // strides of the offset code: Sy > 2D with Sy = 12 (mod 16), so that a
  // 4 x 4 patch of lattice nodes (a half-warp's sources) reads 16 distinct
  // 8-byte banks of the table; Sz = (2D + 1) Sy keeps the code one-to-one
  const int W = 2 * D + 1;
  int Sy = W;
  while (Sy % 16 != 12) ++Sy;
  const int Sz = W * Sy;
  const int64_t nhalf = (int64_t)D * (1 + Sy + Sz) + 1;
  const int64_t npad = (nhalf + 1) / 2 * 2;  // multiple of 16 bytes in both precisions
  const int64_t maxc = (int64_t)(t->n + 1) * (1 + Sy + Sz);
  // the table is staged whole in shared memory by the near-field kernel
  if (D < 1 || npad * (int64_t)sizeof(float2) > HFMM_LAT_TABLE_MAX_BYTES || maxc >= (1ll << 31))
    return HFMM_OK;
  HFMM_TRY(tree_alloc_t(t, &t->lat_lin, t->n_pts));
  HFMM_TRY(tree_alloc_t(t, &t->lat_tab32, npad));
  HFMM_TRY(tree_alloc_t(t, &t->lat_tab64, npad));
  k_lat_lin<<<ceil_div(t->n_pts, 256), 256, 0, s>>>(t->xyz, t->n_pts, inv_h, Sy, Sz, t->lat_lin);
  k_lat_table<<<ceil_div(npad, 256), 256, 0, s>>>(D, Sy, Sz, t->h, t->k, nhalf, npad, t->lat_tab64, t->lat_tab32);
  HFMM_TRY(hfmm_last_launch());
  t->lat_half = npad;
  // FP64: table, window of 32-byte staged sources and 4 KB of static shared memory
  t->lat_tab64_fits = npad * (int64_t)sizeof(double2) + (int64_t)HFMM_LAT_WS * 32 + 4096 <= HFMM_SMEM_MAX;
  t->lat_D = D;
  t->lat_Sy = Sy;
  t->lat_Sz = Sz;
  return HFMM_OK;
}
