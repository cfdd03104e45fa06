// The FMM flow of Sec. 5.1.2 over the sorted point set of a tree:
//   P2M -> M2M (upward) -> M2L (far field, per level) -> L2L (downward)
//   -> L2P, plus P2P (near field) and the singular self term.
//
// Expansions (spherical waves, degrees n < p, coefficient a = n^2 + n + m):
//   multipole about c   phi(x) = i k sum_a M_a h_n(k|x-c|) Y_a(x-c),
//                       M_a = sum_j q_j j_n(k|y_j-c|) conj(Y_a(y_j-c))
//   local about c       phi(x) = i k sum_a L_a j_n(k|x-c|) Y_a(x-c)
// Kernels are templated on the arithmetic type T (double: plain FP64 form;
// float: FP32 form with complex numbers as float pairs).
#include <cmath>
#include <map>
#include <mutex>
#include <utility>

#include "m2l_product.cuh"
#include "special.cuh"
#include "tree.cuh"

namespace {

template <typename T>
int set_smem(const void* fn, size_t bytes);

// cells of level l holding points of a set mask (count, device list)
inline int act_n(const fmm_tree* t, int mask, int l) { return t->act_count[mask - 1][l]; }
inline const int* act_list(const fmm_tree* t, int mask, int l) {
  return t->act_cells[mask - 1] + t->level_off[l];
}

template <typename T>
struct FmmDev {
  const double* xyz;     // sorted coordinates, FP64
  const float4* xyz32;   // sorted coordinates relative to their leaf centre, FP32
  const int* leaf_start;
  const int* leaf_mid;
  const int* flags;      // all levels
  C<T>* M;               // all levels
  C<T>* Lc;
  const C<T>* qs;
  C<T>* phis;
  int p, P, L;
  T k;
  const int* skip;  // when set and nonzero, every kernel of the pass returns at once
  C<T>* near;       // when set: P2P writes its sums here (=) and L2P adds them
  // lattice trees: sorted position -> original id, for the face (and outward
  // normal) of a boundary panel: face = (orig - n_vol) / nn, nn = n^2, faces
  // x=0, x=1, y=0, y=1, z=0, z=1 with normals -e_x, +e_x, -e_y, ...
  const int64_t* orig;
  int64_t n_vol, nn;
};

// face of the boundary panel at sorted position j (lattice trees)
template <typename T>
__device__ __forceinline__ int panel_face(const FmmDev<T>& d, int j) {
  return (int)((d.orig[j] - d.n_vol) / d.nn);
}

// P2P result of target i: into the near-field buffer, or added to phis
template <typename T>
__device__ __forceinline__ void p2p_store(const FmmDev<T>& d, int i, C<T> v) {
  if (d.near)
    d.near[i] = v;
  else
    d.phis[i] = cadd<T>(d.phis[i], v);
}

// L2P result of target i (plus the near field when it went to its own buffer)
template <typename T>
__device__ __forceinline__ void l2p_store(const FmmDev<T>& d, int i, C<T> v) {
  d.phis[i] = d.near ? cadd<T>(v, d.near[i]) : v;
}

#define HFMM_SKIP_IF(d) \
  if ((d).skip && *(d).skip) return

// source/target range of a leaf for a point-set mask
__device__ __forceinline__ void leaf_range(const int* start, const int* mid, int leaf, int set,
                                           int& lo, int& hi) {
  int s0 = start[leaf], s1 = mid[leaf], s2 = start[leaf + 1];
  lo = (set & HFMM_SET_VOL) ? s0 : s1;
  hi = (set & HFMM_SET_BND) ? s2 : s1;
}

// R_a(v) = j_n(k|v|) Y_n^m(v^) for all a < P, written as conj(R_a) * q (P2M, conj = true)
// or R_a (L2P, conj = false) into out[a].
template <typename T, bool CONJ>
__device__ void regular_basis(int p, T k, T dx, T dy, T dz, C<T> q, C<T>* out) {
  T r, ct, st, cp, sp;
  direction<T>(dx, dy, dz, r, ct, st, cp, sp);
  T jn[HFMM_MAX_P];
  T pl[HFMM_MAX_P * (HFMM_MAX_P + 1) / 2];
  sph_bessel_j<T>(k * r, p, jn);
  legendre_bar<T>(ct, st, p, pl);
  T er = T(1), ei = T(0);  // e^{i m phi}
  for (int m = 0; m < p; ++m) {
    for (int n = m; n < p; ++n) {
      T v = jn[n] * pl[n * (n + 1) / 2 + m];
      C<T> R = mkc<T>(v * er, v * ei);  // R_{n,m}
      if (CONJ) {
        out[n * n + n + m] = cmul<T>(conjc<T>(R), q);
        if (m > 0) {  // conj(R_{n,-m}) = (-1)^m R_{n,m}
          C<T> Rm = (m & 1) ? mkc<T>(-R.x, -R.y) : R;
          out[n * n + n - m] = cmul<T>(Rm, q);
        }
      } else {
        out[n * n + n + m] = R;
        if (m > 0) {  // R_{n,-m} = (-1)^m conj(R_{n,m})
          C<T> Rc = conjc<T>(R);
          out[n * n + n - m] = (m & 1) ? mkc<T>(-Rc.x, -Rc.y) : Rc;
        }
      }
    }
    T nr = er * cp - ei * sp, ni = er * sp + ei * cp;
    er = nr;
    ei = ni;
  }
}

template <typename T>
__device__ __forceinline__ void local_coords(const FmmDev<T>& d, int i, int leaf, T& dx, T& dy, T& dz) {
  if constexpr (sizeof(T) == 4) {
    float4 v = d.xyz32[i];
    dx = v.x;
    dy = v.y;
    dz = v.z;
  } else {
    int ix, iy, iz;
    morton_decode((uint64_t)leaf, ix, iy, iz);
    double w = ldexp(1.0, -d.L);
    dx = d.xyz[3 * i] - (ix + 0.5) * w;
    dy = d.xyz[3 * i + 1] - (iy + 0.5) * w;
    dz = d.xyz[3 * i + 2] - (iz + 0.5) * w;
  }
}

// ---------------------------------------------------------------- P2M
// one block per leaf; CHUNK points' basis rows staged in shared memory, then
// summed per coefficient
// conj(dR_a/dk)(v) * q = |v| j_n'(k|v|) conj(Y_a(v^)) * q for all a < P, with
// (2n+1) j_n' = n j_{n-1} - (n+1) j_{n+1} (no division by k|v|)
template <typename T>
__device__ void regular_basis_dk_conj(int p, T k, T dx, T dy, T dz, C<T> q, C<T>* out) {
  T r, ct, st, cp, sp;
  direction<T>(dx, dy, dz, r, ct, st, cp, sp);
  T jn[HFMM_MAX_P + 1];
  T pl[HFMM_MAX_P * (HFMM_MAX_P + 1) / 2];
  sph_bessel_j<T>(k * r, p + 1, jn);
  legendre_bar<T>(ct, st, p, pl);
  T er = T(1), ei = T(0);
  for (int m = 0; m < p; ++m) {
    for (int n = m; n < p; ++n) {
      T djn = (n > 0 ? T(n) * jn[n - 1] : T(0)) - T(n + 1) * jn[n + 1];
      djn = r * djn / T(2 * n + 1);
      T v = djn * pl[n * (n + 1) / 2 + m];
      C<T> R = mkc<T>(v * er, v * ei);
      out[n * n + n + m] = cmul<T>(conjc<T>(R), q);
      if (m > 0) {
        C<T> Rm = (m & 1) ? mkc<T>(-R.x, -R.y) : R;
        out[n * n + n - m] = cmul<T>(Rm, q);
      }
    }
    T nr = er * cp - ei * sp, ni = er * sp + ei * cp;
    er = nr;
    ei = ni;
  }
}

// conj(n . grad R_a)(v) * q for all a < P: the multipole row of a dipole of
// strength q with the outward normal n of boundary face `face` (n = -e_x for
// x=0, +e_x for x=1, ...), Sec. 5.2 (normal derivative in the double-layer
// term of Eq. (bem)).  With d+- = d/dx +- i d/dy the gradient of R_l^m =
// j_l Y_l^m (orthonormal Y, Condon-Shortley phase) is exact in the degrees
// l -+ 1:
//   d/dz R_l^m = k (A R_{l-1}^m - B R_{l+1}^m)
//   d+   R_l^m = k (C R_{l-1}^{m+1} + D R_{l+1}^{m+1})
//   d-   R_l^m = -k (E R_{l-1}^{m-1} + F R_{l+1}^{m-1})
//   A = sqrt((l^2 - m^2) / ((2l-1)(2l+1))),   B = sqrt(((l+1)^2 - m^2) / ((2l+1)(2l+3))),
//   C = sqrt((l-m)(l-m-1) / ((2l-1)(2l+1))),  D = sqrt((l+m+1)(l+m+2) / ((2l+1)(2l+3))),
//   E = sqrt((l+m)(l+m-1) / ((2l-1)(2l+1))),  F = sqrt((l-m+1)(l-m+2) / ((2l+1)(2l+3))),
// terms of order |m'| > l' being zero; so R is needed up to degree p, and no
// division by sin(theta) occurs (points on the polar axis are regular).
template <typename T>
__device__ void regular_basis_dn_conj(int p, T k, T dx, T dy, T dz, int face, C<T> q, C<T>* out) {
  T r, ct, st, cp, sp;
  direction<T>(dx, dy, dz, r, ct, st, cp, sp);
  T jn[HFMM_MAX_P + 1];
  T pl[(HFMM_MAX_P + 1) * (HFMM_MAX_P + 2) / 2];
  C<T> em[HFMM_MAX_P + 1];  // e^{i m phi}, m <= p
  sph_bessel_j<T>(k * r, p + 1, jn);
  legendre_bar<T>(ct, st, p + 1, pl);
  em[0] = mkc<T>(1, 0);
  for (int m = 1; m <= p; ++m) em[m] = mkc<T>(em[m - 1].x * cp - em[m - 1].y * sp, em[m - 1].x * sp + em[m - 1].y * cp);
  // R_n^m for 0 <= n <= p, zero outside |m| <= n
  auto Rnm = [&](int n, int m) -> C<T> {
    const int am = m < 0 ? -m : m;
    if (n < 0 || am > n) return mkc<T>(0, 0);
    const T v = jn[n] * pl[n * (n + 1) / 2 + am];
    C<T> R = mkc<T>(v * em[am].x, v * em[am].y);
    if (m < 0) {  // R_n^{-m} = (-1)^m conj(R_n^m)
      R = conjc<T>(R);
      if (am & 1) R = mkc<T>(-R.x, -R.y);
    }
    return R;
  };
  const int axis = face >> 1;
  const T sgn = (face & 1) ? T(1) : T(-1);
  for (int l = 0; l < p; ++l) {
    const T den_lo = T((2 * l - 1) * (2 * l + 1)), den_hi = T((2 * l + 1) * (2 * l + 3));
    for (int m = -l; m <= l; ++m) {
      C<T> g;  // d/d(axis) R_l^m
      if (axis == 2) {
        const T A = l > 0 ? sqrt(T(l * l - m * m) / den_lo) : T(0);
        const T B = sqrt(T((l + 1) * (l + 1) - m * m) / den_hi);
        const C<T> lo = Rnm(l - 1, m), hi = Rnm(l + 1, m);
        g = mkc<T>(k * (A * lo.x - B * hi.x), k * (A * lo.y - B * hi.y));
      } else {
        const T Cc = l > 0 ? sqrt(T((l - m) * (l - m - 1)) / den_lo) : T(0);
        const T Dd = sqrt(T((l + m + 1) * (l + m + 2)) / den_hi);
        const T Ee = l > 0 ? sqrt(T((l + m) * (l + m - 1)) / den_lo) : T(0);
        const T Ff = sqrt(T((l - m + 1) * (l - m + 2)) / den_hi);
        const C<T> a1 = Rnm(l - 1, m + 1), a2 = Rnm(l + 1, m + 1);
        const C<T> b1 = Rnm(l - 1, m - 1), b2 = Rnm(l + 1, m - 1);
        const C<T> dp = mkc<T>(k * (Cc * a1.x + Dd * a2.x), k * (Cc * a1.y + Dd * a2.y));
        const C<T> dm = mkc<T>(-k * (Ee * b1.x + Ff * b2.x), -k * (Ee * b1.y + Ff * b2.y));
        if (axis == 0)  // d/dx = (d+ + d-) / 2
          g = mkc<T>(T(0.5) * (dp.x + dm.x), T(0.5) * (dp.y + dm.y));
        else            // d/dy = (d+ - d-) / (2 i)
          g = mkc<T>(T(0.5) * (dp.y - dm.y), -T(0.5) * (dp.x - dm.x));
      }
      out[l * l + l + m] = cmul<T>(conjc<T>(mkc<T>(sgn * g.x, sgn * g.y)), q);
    }
  }
}

// one block per leaf; CHUNK points' basis rows staged in shared memory, then
// summed per coefficient.  Output Mout (leaf level), weights times `fac`;
// BASIS 0: R_a; 1: derivative of the basis with respect to k; 2: normal
// derivative at boundary panels (dipole sources).
template <typename T, int BASIS>
__global__ void k_p2m(FmmDev<T> d, C<T>* Mout, int64_t leaf_off, int src_set, int chunk, C<T> fac,
                      const int* __restrict__ list) {
  HFMM_SKIP_IF(d);
  extern __shared__ unsigned char smem_raw[];
  C<T>* basis = reinterpret_cast<C<T>*>(smem_raw);
  const int leaf = list ? list[blockIdx.x] : blockIdx.x;
  const int P = d.P;
  C<T>* M = Mout + (leaf_off + leaf) * P;
  int lo, hi;
  leaf_range(d.leaf_start, d.leaf_mid, leaf, src_set, lo, hi);
  if (hi <= lo) {
    for (int a = threadIdx.x; a < P; a += blockDim.x) M[a] = mkc<T>(0, 0);
    return;
  }
  C<T> acc[4];
  for (int i = 0; i < 4; ++i) acc[i] = mkc<T>(0, 0);
  for (int base = lo; base < hi; base += chunk) {
    for (int jj = threadIdx.x; jj < chunk; jj += blockDim.x) {
      int j = base + jj;
      C<T>* row = basis + (int64_t)jj * P;
      if (j < hi) {
        T dx, dy, dz;
        local_coords<T>(d, j, leaf, dx, dy, dz);
        C<T> q = cmul<T>(d.qs[j], fac);
        if constexpr (BASIS == 1)
          regular_basis_dk_conj<T>(d.p, d.k, dx, dy, dz, q, row);
        else if constexpr (BASIS == 2)
          regular_basis_dn_conj<T>(d.p, d.k, dx, dy, dz, panel_face<T>(d, j), q, row);
        else
          regular_basis<T, true>(d.p, d.k, dx, dy, dz, q, row);
      } else {
        for (int a = 0; a < P; ++a) row[a] = mkc<T>(0, 0);
      }
    }
    __syncthreads();
    for (int s = 0; s < 4; ++s) {
      int a = threadIdx.x + s * blockDim.x;
      if (a < P)
        for (int jj = 0; jj < chunk; ++jj) acc[s] = cadd<T>(acc[s], basis[(int64_t)jj * P + a]);
    }
    __syncthreads();
  }
  for (int s = 0; s < 4; ++s) {
    int a = threadIdx.x + s * blockDim.x;
    if (a < P) M[a] = acc[s];
  }
}

// Regular basis table: row i holds R_a(x_i - c) (a < P) for every sorted
// point i and the centre c of its leaf, evaluated in FP64 once per tree and
// stored in the precision of the form.  P2M and L2P then reduce to short
// complex dot products over the rows (no special functions per apply).
template <typename T>
__global__ void k_basis_table(const double* __restrict__ xyz, const int* __restrict__ leaf_start, int L, int p,
                              double k, C<T>* __restrict__ R) {
  const int leaf = blockIdx.x;
  const int P = p * p;
  int ix, iy, iz;
  morton_decode((uint64_t)leaf, ix, iy, iz);
  const double w = ldexp(1.0, -L);
  for (int i = leaf_start[leaf] + threadIdx.x; i < leaf_start[leaf + 1]; i += blockDim.x) {
    const double dx = xyz[3 * (int64_t)i] - (ix + 0.5) * w;
    const double dy = xyz[3 * (int64_t)i + 1] - (iy + 0.5) * w;
    const double dz = xyz[3 * (int64_t)i + 2] - (iz + 0.5) * w;
    double r, ct, st, cp, sp;
    direction<double>(dx, dy, dz, r, ct, st, cp, sp);
    double jn[HFMM_MAX_P];
    double pl[HFMM_MAX_P * (HFMM_MAX_P + 1) / 2];
    sph_bessel_j<double>(k * r, p, jn);
    legendre_bar<double>(ct, st, p, pl);
    C<T>* out = R + (int64_t)i * P;
    double er = 1.0, ei = 0.0;  // e^{i m phi}
    for (int m = 0; m < p; ++m) {
      for (int n = m; n < p; ++n) {
        const double v = jn[n] * pl[n * (n + 1) / 2 + m];
        const double Rx = v * er, Ry = v * ei;  // R_{n,m}
        out[n * n + n + m] = mkc<T>(T(Rx), T(Ry));
        if (m > 0) {  // R_{n,-m} = (-1)^m conj(R_{n,m})
          const double sg = (m & 1) ? -1.0 : 1.0;
          out[n * n + n - m] = mkc<T>(T(sg * Rx), T(-sg * Ry));
        }
      }
      const double nr = er * cp - ei * sp, ni = er * sp + ei * cp;
      er = nr;
      ei = ni;
    }
  }
}

// M_a(leaf) = fac sum_i conj(R_ia) q_i over the leaf's points of src_set
template <typename T>
__global__ void __launch_bounds__(64) k_p2m_tab(FmmDev<T> d, const C<T>* __restrict__ R, C<T>* Mout,
                                                int64_t leaf_off, int src_set, C<T> fac,
                                                const int* __restrict__ list) {
  HFMM_SKIP_IF(d);
  __shared__ C<T> qsh[64];
  const int leaf = list ? list[blockIdx.x] : blockIdx.x;
  const int P = d.P;
  C<T>* M = Mout + (leaf_off + leaf) * P;
  int lo, hi;
  leaf_range(d.leaf_start, d.leaf_mid, leaf, src_set, lo, hi);
  for (int a0 = 0; a0 < P; a0 += 64) {
    const int a = a0 + threadIdx.x;
    C<T> acc = mkc<T>(0, 0);
    for (int base = lo; base < hi; base += 64) {
      const int nb = min(64, hi - base);
      __syncthreads();
      if ((int)threadIdx.x < nb) qsh[threadIdx.x] = d.qs[base + threadIdx.x];
      __syncthreads();
      if (a < P) {
        const C<T>* Rc = R + (int64_t)base * P + a;
#pragma unroll 8
        for (int jj = 0; jj < nb; ++jj) cfma_conj<T>(acc, Rc[(int64_t)jj * P], qsh[jj]);
      }
    }
    if (a < P) M[a] = cmul<T>(fac, acc);
  }
}

// phi_i = fac sum_a L_a R_ia over the leaf's points of tgt_set; eight lanes
// per point, each a strided share of the coefficients
template <typename T>
__global__ void __launch_bounds__(256) k_l2p_tab(FmmDev<T> d, const C<T>* __restrict__ R, int64_t leaf_off,
                                                 int tgt_set, C<T> fac, const int* __restrict__ list) {
  HFMM_SKIP_IF(d);
  extern __shared__ unsigned char smem_raw[];
  C<T>* Ls = reinterpret_cast<C<T>*>(smem_raw);
  const int leaf = list ? list[blockIdx.x] : blockIdx.x;
  const int P = d.P;
  int lo, hi;
  leaf_range(d.leaf_start, d.leaf_mid, leaf, tgt_set, lo, hi);
  if (hi <= lo) return;
  for (int e = threadIdx.x; e < P; e += blockDim.x) Ls[e] = d.Lc[(leaf_off + leaf) * P + e];
  __syncthreads();
  const int sub = threadIdx.x & 7, grp = threadIdx.x >> 3;
  for (int ib = lo; ib < hi; ib += 32) {
    const int i = ib + grp;
    const bool act = i < hi;
    C<T> acc = mkc<T>(0, 0);
    if (act) {
      const C<T>* Ri = R + (int64_t)i * P;
      for (int a = sub; a < P; a += 8) cfma<T>(acc, Ls[a], Ri[a]);
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (act && sub == 0) l2p_store<T>(d, i, cmul<T>(fac, acc));
  }
}

// ---------------------------------------------------------------- M2M / L2L
// out[a'] = sum_a T(a', a) in[a] with T column-major (entry (a', a) at a*P + a');
// one thread per a', so a warp reads consecutive words of each column
template <typename T>
__device__ __forceinline__ C<T> matvec_row(const C<T>* Tcol, int ap, const C<T>* x, int P) {
  C<T> acc = mkc<T>(0, 0);
  for (int a = 0; a < P; ++a) cfma<T>(acc, Tcol[(int64_t)a * P + ap], x[a]);
  return acc;
}

// Mout(parent) (+)= sum over children holding sources of T_o Min(child).
// With a list, only the listed parents (those holding sources) are visited;
// expansions of cells without sources are never read (they may be stale).
// Four threads per output row (thread `sub` takes octants sub and sub + 4),
// combined with warp shuffles; block = 4 P threads rounded up to a warp.
template <typename T>
__global__ void k_m2m(FmmDev<T> d, int level, int64_t off_par, int64_t off_child, const C<T>* Min, C<T>* Mout,
                      const C<T>* __restrict__ ops, int src_set, int accumulate, const int* __restrict__ list) {
  HFMM_SKIP_IF(d);
  extern __shared__ unsigned char smem_raw[];
  C<T>* xs = reinterpret_cast<C<T>*>(smem_raw);  // [8][P]
  __shared__ int has[8];
  const int cell = list ? list[blockIdx.x] : blockIdx.x;
  const int P = d.P;
  C<T>* Mp = Mout + (off_par + cell) * P;
  if (!(d.flags[off_par + cell] & src_set)) {
    if (!accumulate)
      for (int a = threadIdx.x; a < P; a += blockDim.x) Mp[a] = mkc<T>(0, 0);
    return;
  }
  if (threadIdx.x < 8) has[threadIdx.x] = (d.flags[off_child + 8 * (int64_t)cell + threadIdx.x] & src_set) != 0;
  __syncthreads();
  const C<T>* ch = Min + (off_child + 8 * (int64_t)cell) * P;
  for (int o = 0; o < 8; ++o) {
    const bool h = has[o];
    for (int a = threadIdx.x; a < P; a += blockDim.x) xs[o * P + a] = h ? ch[o * P + a] : mkc<T>(0, 0);
  }
  __syncthreads();
  const int ap = threadIdx.x >> 2, sub = threadIdx.x & 3;
  C<T> acc = mkc<T>(0, 0);
  if (ap < P) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int o = sub + 4 * q;
      if (!has[o]) continue;
      const C<T>* Tc = ops + (int64_t)o * P * P + ap;
      const C<T>* x = xs + o * P;
      for (int a = 0; a < P; ++a) cfma<T>(acc, Tc[(int64_t)a * P], x[a]);
    }
  }
  acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
  acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
  acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
  acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
  if (ap < P && sub == 0) Mp[ap] = accumulate ? cadd<T>(Mp[ap], acc) : acc;
}

// Lout(child) += T_octant Lin(parent); four threads per output row, each a
// quarter of the columns, combined with warp shuffles
template <typename T>
__global__ void k_l2l(FmmDev<T> d, int64_t off_par, int64_t off_child, const C<T>* Lin, C<T>* Lout,
                      const C<T>* __restrict__ ops, int tgt_set, const int* __restrict__ list) {
  HFMM_SKIP_IF(d);
  extern __shared__ unsigned char smem_raw[];
  C<T>* xs = reinterpret_cast<C<T>*>(smem_raw);
  const int cell = list ? list[blockIdx.x] : blockIdx.x;  // child
  const int P = d.P;
  if (!(d.flags[off_child + cell] & tgt_set)) return;
  const int parent = cell >> 3, o = cell & 7;
  for (int e = threadIdx.x; e < P; e += blockDim.x) xs[e] = Lin[(off_par + parent) * P + e];
  __syncthreads();
  C<T>* Lch = Lout + (off_child + cell) * P;
  const int ap = threadIdx.x >> 2, sub = threadIdx.x & 3;
  C<T> acc = mkc<T>(0, 0);
  if (ap < P) {
    const C<T>* Tc = ops + (int64_t)o * P * P + ap;
    for (int a = sub; a < P; a += 4) cfma<T>(acc, Tc[(int64_t)a * P], xs[a]);
  }
  acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
  acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
  acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
  acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
  if (ap < P && sub == 0) Lch[ap] = cadd<T>(Lch[ap], acc);
}

// ---------------------------------------------------------------- M2L
// one block per target cell of the level: L_T = sum over the cell's list of
// T_{slot} M_S, sources skipped when they hold no point of the source set
template <typename T>
__global__ void k_m2l(FmmDev<T> d, int level, int64_t off, const C<T>* ops, const int* m2l_off,
                      const int* m2l_slot, int m2l_count, int src_set, int tgt_set, int accumulate) {
  HFMM_SKIP_IF(d);
  extern __shared__ unsigned char smem_raw[];
  C<T>* xs = reinterpret_cast<C<T>*>(smem_raw);
  const int cell = blockIdx.x;
  const int P = d.P;
  if (!(d.flags[off + cell] & tgt_set)) return;
  const int b = cell & 7;
  int ix, iy, iz;
  morton_decode((uint64_t)cell, ix, iy, iz);
  const int s = 1 << level;
  C<T> acc[4];
  for (int i = 0; i < 4; ++i) acc[i] = mkc<T>(0, 0);
  for (int i = 0; i < m2l_count; ++i) {
    int o = m2l_off[b * m2l_count + i];
    int jx = ix + (o & 255) - 128, jy = iy + ((o >> 8) & 255) - 128, jz = iz + ((o >> 16) & 255) - 128;
    if (jx < 0 || jy < 0 || jz < 0 || jx >= s || jy >= s || jz >= s) continue;
    int64_t src = (int64_t)morton_encode(jx, jy, jz);
    if (!(d.flags[off + src] & src_set)) continue;
    __syncthreads();
    for (int e = threadIdx.x; e < P; e += blockDim.x) xs[e] = d.M[(off + src) * P + e];
    __syncthreads();
    const C<T>* Top = ops + (int64_t)m2l_slot[b * m2l_count + i] * P * P;
    for (int q = 0; q < 4; ++q) {
      int ap = threadIdx.x + q * blockDim.x;
      if (ap < P) {  // row-major operator: row ap is contiguous
        C<T> v = mkc<T>(0, 0);
        for (int a = 0; a < P; ++a) cfma<T>(v, Top[(int64_t)ap * P + a], xs[a]);
        acc[q] = cadd<T>(acc[q], v);
      }
    }
  }
  for (int q = 0; q < 4; ++q) {
    int ap = threadIdx.x + q * blockDim.x;
    if (ap < P) {
      C<T>* dst = d.Lc + (off + cell) * P + ap;
      *dst = accumulate ? cadd<T>(*dst, acc[q]) : acc[q];
    }
  }
}

// Tiled M2L over all levels in one launch.  A block owns a tile of TC target
// cells of one level and parity class (so they share their offset list); for
// each offset it stages the operator (P x P, column-major) and the TC source
// expansions in shared memory and forms the P x TC complex product with a
// register tile of R rows x CM columns per thread (128 threads as 16 row
// groups x 8 column groups).  Offsets whose sources hold no point of the
// source set in the whole tile are skipped.
template <typename T, int R, int CM>
__global__ void __launch_bounds__(128) k_m2l_tiled(FmmDev<T> d, const int4* __restrict__ tiles,
                                                   const int* __restrict__ cells,
                                                   const int64_t* __restrict__ level_off,
                                                   const C<T>* __restrict__ ops, int64_t box_cells,
                                                   const int* __restrict__ m2l_off,
                                                   const int* __restrict__ m2l_slot, int m2l_count,
                                                   int src_set, int accumulate) {
  HFMM_SKIP_IF(d);
  constexpr int CT = 8, RT = 16, TC = CT * CM;
  extern __shared__ unsigned char smem_raw[];
  const int P = d.P;
  C<T>* Ts = reinterpret_cast<C<T>*>(smem_raw);           // [P][P] column-major
  C<T>* Ms = Ts + (size_t)P * P;                          // [P][TC + 1]
  int* scell = reinterpret_cast<int*>(Ms + (size_t)P * (TC + 1));
  int* tcell = scell + TC;
  int* tco = tcell + TC;                                  // [TC][3] target coordinates
  const int4 tile = tiles[blockIdx.x];
  const int level = tile.x, b = tile.y, first = tile.z, cnt = tile.w;
  const int64_t off = level_off[level];
  const int s = 1 << level;
  const int tid = threadIdx.x;
  const int r0 = tid / CT, c0 = tid % CT;
  if (tid < TC) {
    int cell = tid < cnt ? cells[first + tid] : -1;
    tcell[tid] = cell;
    int ix = 0, iy = 0, iz = 0;
    if (cell >= 0) morton_decode((uint64_t)cell, ix, iy, iz);
    tco[3 * tid] = ix;
    tco[3 * tid + 1] = iy;
    tco[3 * tid + 2] = iz;
  }
  C<T> acc[R][CM];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int j = 0; j < CM; ++j) acc[r][j] = mkc<T>(0, 0);
  const C<T>* opsl = ops + (int64_t)level * box_cells * P * P;
  __syncthreads();
  for (int i = 0; i < m2l_count; ++i) {
    const int o = m2l_off[b * m2l_count + i];
    bool valid = false;
    if (tid < TC) {
      int src = -1;
      if (tcell[tid] >= 0) {
        int jx = tco[3 * tid] + (o & 255) - 128, jy = tco[3 * tid + 1] + ((o >> 8) & 255) - 128,
            jz = tco[3 * tid + 2] + ((o >> 16) & 255) - 128;
        if (jx >= 0 && jy >= 0 && jz >= 0 && jx < s && jy < s && jz < s) {
          int c = (int)morton_encode(jx, jy, jz);
          if (d.flags[off + c] & src_set) src = c;
        }
      }
      scell[tid] = src;
      valid = src >= 0;
    }
    if (!__syncthreads_or(valid)) continue;
    const C<T>* Top = opsl + (int64_t)m2l_slot[b * m2l_count + i] * P * P;
    for (int e = tid; e < P * P; e += 128) Ts[e] = Top[e];
    for (int e = tid; e < P * TC; e += 128) {
      int c = e / P, a = e - c * P;
      int sc = scell[c];
      Ms[a * (TC + 1) + c] = sc >= 0 ? d.M[(off + sc) * P + a] : mkc<T>(0, 0);
    }
    __syncthreads();
    for (int a = 0; a < P; ++a) {
      C<T> tv[R], mv[CM];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        int ap = r0 + r * RT;
        tv[r] = ap < P ? Ts[ap * P + a] : mkc<T>(0, 0);
      }
#pragma unroll
      for (int j = 0; j < CM; ++j) mv[j] = Ms[a * (TC + 1) + c0 + j * CT];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int j = 0; j < CM; ++j) cfma<T>(acc[r][j], tv[r], mv[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int j = 0; j < CM; ++j) {
      int ap = r0 + r * RT, c = c0 + j * CT;
      if (ap < P && c < cnt) {
        C<T>* dst = d.Lc + (off + tcell[c]) * P + ap;
        *dst = accumulate ? cadd<T>(*dst, acc[r][j]) : acc[r][j];
      }
    }
}

// ---- TMA-staged, split-offset M2L (even p: rows are multiples of 16 bytes)
//
// Same tiling as k_m2l_tiled, but (1) the offsets of a tile whose sources hold
// no point of the source set are dropped up front, (2) the operator and the
// source rows of the next offset are fetched with 1D bulk copies
// (cp.async.bulk, completion on an mbarrier) while the current one is
// multiplied (two stages), and (3) a tile's offset list may be split over
// gridDim.y blocks whose partial sums go to a scratch array, reduced in a
// fixed order afterwards (deterministic).

__device__ int g_fmm_error;  // set when a bounded wait gives up (HFMM_ERR_TIMEOUT)

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// bounded wait: gives up (false) after one second of wall time
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (global_ns() - t0 < 1000000000ull)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Valid offsets of every tile for one source-set mask: the offsets (in list
// order) for which at least one tile cell has a source cell holding points of
// the set, with the mask of those columns.  One block per tile, one-time.
__global__ void k_m2l_valid(const int4* __restrict__ tiles, const int* __restrict__ cells,
                            const int* __restrict__ flags, const int64_t* __restrict__ level_off,
                            const int* __restrict__ m2l_off, int m2l_count, int src_set,
                            int* __restrict__ vlist, unsigned* __restrict__ vmask, int* __restrict__ nval) {
  extern __shared__ unsigned char smem_raw[];
  unsigned* msk = reinterpret_cast<unsigned*>(smem_raw);  // [m2l_count]
  __shared__ int tco[32][3];
  __shared__ int tval[32];
  const int4 tile = tiles[blockIdx.x];
  const int level = tile.x, b = tile.y, first = tile.z, cnt = tile.w;
  const int64_t off = level_off[level];
  const int s = 1 << level;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  if (tid < 32) {
    int cell = tid < cnt ? cells[first + tid] : -1;
    int ix = 0, iy = 0, iz = 0;
    if (cell >= 0) morton_decode((uint64_t)cell, ix, iy, iz);
    tco[tid][0] = ix;
    tco[tid][1] = iy;
    tco[tid][2] = iz;
    tval[tid] = cell >= 0;
  }
  __syncthreads();
  for (int i = warp; i < m2l_count; i += nw) {
    const int o = m2l_off[b * m2l_count + i];
    bool v = false;
    if (tval[lane]) {
      int jx = tco[lane][0] + (o & 255) - 128, jy = tco[lane][1] + ((o >> 8) & 255) - 128,
          jz = tco[lane][2] + ((o >> 16) & 255) - 128;
      if (jx >= 0 && jy >= 0 && jz >= 0 && jx < s && jy < s && jz < s)
        v = (flags[off + morton_encode(jx, jy, jz)] & src_set) != 0;
    }
    unsigned m = __ballot_sync(0xffffffffu, v);
    if (lane == 0) msk[i] = m;
  }
  __syncthreads();
  if (tid == 0) {
    int n = 0;
    int* vl = vlist + (int64_t)blockIdx.x * m2l_count;
    unsigned* vm = vmask + (int64_t)blockIdx.x * m2l_count;
    for (int i = 0; i < m2l_count; ++i)
      if (msk[i]) {
        vl[n] = i;
        vm[n] = msk[i];
        ++n;
      }
    nval[blockIdx.x] = n;
  }
}

template <typename T, int R, int CM, int RT>
__global__ void __launch_bounds__(RT * 8) k_m2l_tma(FmmDev<T> d, const int4* __restrict__ tiles,
                                                    const int* __restrict__ cells,
                                                    const int64_t* __restrict__ level_off,
                                                    const C<T>* __restrict__ ops, int64_t box_cells,
                                                    const int* __restrict__ m2l_off,
                                                    const int* __restrict__ m2l_slot, int m2l_count,
                                                    const int* __restrict__ vlist_all,
                                                    const unsigned* __restrict__ vmask_all,
                                                    const int* __restrict__ nval_all,
                                                    const C<T>* __restrict__ zero_row,
                                                    C<T>* __restrict__ part, int64_t part_stride, int accumulate) {
  HFMM_SKIP_IF(d);
  constexpr int CT = 8, TC = CT * CM, NT = RT * CT;
  const int P = d.P;
  const int MS = P + 2;  // padded source row (16-byte multiple, spreads banks)
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);  // [2]
  int* tcell = reinterpret_cast<int*>(smem_raw + 16);      // [TC]
  int* tco = tcell + TC;                                   // [TC][3]
  C<T>* Ts = reinterpret_cast<C<T>*>(smem_raw + 1024);     // [2][P*P]
  C<T>* Ms = Ts + 2 * (size_t)P * P;                       // [2][TC][MS]

  const int4 tile = tiles[blockIdx.x];
  const int level = tile.x, b = tile.y, first = tile.z, cnt = tile.w;
  const int64_t off = level_off[level];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r0 = tid / CT, c0 = tid % CT;
  const int* vlist = vlist_all + (int64_t)blockIdx.x * m2l_count;
  const unsigned* vmask = vmask_all + (int64_t)blockIdx.x * m2l_count;
  if (tid < TC) {
    int cell = tid < cnt ? cells[first + tid] : -1;
    tcell[tid] = cell;
    int ix = 0, iy = 0, iz = 0;
    if (cell >= 0) morton_decode((uint64_t)cell, ix, iy, iz);
    tco[3 * tid] = ix;
    tco[3 * tid + 1] = iy;
    tco[3 * tid + 2] = iz;
  }
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int nv = nval_all[blockIdx.x];
  const int ks = blockIdx.y, kn = gridDim.y;
  const int sbeg = (int)((int64_t)nv * ks / kn), send = (int)((int64_t)nv * (ks + 1) / kn);
  const C<T>* opsl = ops + (int64_t)level * box_cells * P * P;
  const uint32_t op_bytes = (uint32_t)((size_t)P * P * sizeof(C<T>));
  const uint32_t row_bytes = (uint32_t)((size_t)P * sizeof(C<T>));

  // warp 0 issues the copies of step `st` into stage (st - sbeg) & 1: the
  // operator, and for each of the TC columns either its source row or a row
  // of zeros (so that the product needs no masking)
  auto issue = [&](int st) {
    const int i = vlist[st];
    const unsigned m = vmask[st];
    const int stg = (st - sbeg) & 1;
    if (lane == 0) {
      fence_async_shared();
      mbar_expect_tx(&bar[stg], op_bytes + (uint32_t)TC * row_bytes);
    }
    __syncwarp();
    if (lane == 0)
      bulk_copy_g2s(Ts + (size_t)stg * P * P, opsl + (int64_t)m2l_slot[b * m2l_count + i] * P * P, op_bytes,
                    &bar[stg]);
    if (lane < TC) {
      const C<T>* src = zero_row;
      if ((m >> lane) & 1u) {
        const int o = m2l_off[b * m2l_count + i];
        int jx = tco[3 * lane] + (o & 255) - 128, jy = tco[3 * lane + 1] + ((o >> 8) & 255) - 128,
            jz = tco[3 * lane + 2] + ((o >> 16) & 255) - 128;
        src = d.M + (off + (int64_t)morton_encode(jx, jy, jz)) * P;
      }
      bulk_copy_g2s(Ms + ((size_t)stg * TC + lane) * MS, src, row_bytes, &bar[stg]);
    }
  };

  C<T> acc[R][CM];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int j = 0; j < CM; ++j) acc[r][j] = mkc<T>(0, 0);

  if (warp == 0 && sbeg < send) issue(sbeg);
  int failed_at = -1;
  for (int st = sbeg; st < send; ++st) {
    const int stg = (st - sbeg) & 1;
    if (warp == 0 && st + 1 < send) issue(st + 1);
    const uint32_t parity = (uint32_t)(((st - sbeg) >> 1) & 1);
    bool ok = mbar_wait_bounded(&bar[stg], parity);
    if (__syncthreads_or(!ok)) {
      failed_at = st;
      break;
    }
    m2l_block_product<T, R, CM, RT>(Ts + (size_t)stg * P * P, Ms + (size_t)stg * TC * MS, P, MS, r0, c0, acc);
    __syncthreads();  // stage free for the copy issued in the next step
  }
  if (failed_at >= 0) {
    // record the error, then give the copies still in flight (the step that
    // timed out and the one issued after it) a bounded time to land before
    // the block's shared memory is released
    if (tid == 0) {
      atomicExch(&g_fmm_error, HFMM_ERR_TIMEOUT);
      for (int st = failed_at; st < send && st <= failed_at + 1; ++st)
        mbar_wait_bounded(&bar[(st - sbeg) & 1], (uint32_t)(((st - sbeg) >> 1) & 1));
    }
    __syncthreads();
    return;
  }
  C<T>* out = part ? part + (int64_t)ks * part_stride : nullptr;
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int j = 0; j < CM; ++j) {
      int ap = r0 + r * RT, c = c0 + j * CT;
      if (ap < P && c < cnt) {
        if (out) {
          out[(int64_t)(first + c) * P + ap] = acc[r][j];
        } else {
          C<T>* dst = d.Lc + (off + tcell[c]) * P + ap;
          *dst = accumulate ? cadd<T>(*dst, acc[r][j]) : acc[r][j];
        }
      }
    }
  (void)NT;
}

// Warp-specialised form of k_m2l_tma: one producer warp streams the
// operator and source rows of each valid offset through NSTG shared-memory
// stages with bulk copies (full barrier per stage, completed by the copies'
// byte count), and RT * 8 consumer threads multiply; consumers release a
// stage through its empty barrier (one arrival per consumer warp), so no
// block-wide barrier sits in the main loop.  Every wait is bounded; a wait
// that gives up raises a block-wide abort flag, records HFMM_ERR_TIMEOUT and
// the block leaves without writing results.
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_wait_abortable(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (global_ns() - t0 < 1000000000ull) {
    if (*abort_flag) return false;
    if (mbar_try_wait(bar, parity)) return true;
  }
  *abort_flag = 1;
  return false;
}

template <typename T, int R, int CM, int RT, int NSTG>
__global__ void __launch_bounds__(RT * 8 + 32) k_m2l_ws(FmmDev<T> d, const int4* __restrict__ tiles,
                                                        const int* __restrict__ cells,
                                                        const int64_t* __restrict__ level_off,
                                                        const C<T>* __restrict__ ops, int64_t box_cells,
                                                        const int* __restrict__ m2l_off,
                                                        const int* __restrict__ m2l_slot, int m2l_count,
                                                        const int* __restrict__ vlist_all,
                                                        const unsigned* __restrict__ vmask_all,
                                                        const int* __restrict__ nval_all,
                                                        const C<T>* __restrict__ zero_row,
                                                        C<T>* __restrict__ part, int64_t part_stride, int accumulate) {
  HFMM_SKIP_IF(d);
  constexpr int CT = 8, TC = CT * CM, NC = RT * CT, NCW = NC / 32;
  const int P = d.P;
  const int MS = P + 2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);           // [NSTG]
  uint64_t* empty = full + NSTG;                                     // [NSTG]
  int* abort_flag = reinterpret_cast<int*>(empty + NSTG);
  int* tcell = abort_flag + 4;                                       // [TC]
  int* tco = tcell + TC;                                             // [TC][3]
  C<T>* Ts = reinterpret_cast<C<T>*>(smem_raw + 1024);              // [NSTG][P*P]
  C<T>* Ms = Ts + NSTG * (size_t)P * P;                              // [NSTG][TC][MS]

  const int4 tile = tiles[blockIdx.x];
  const int level = tile.x, b = tile.y, first = tile.z, cnt = tile.w;
  const int64_t off = level_off[level];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int* vlist = vlist_all + (int64_t)blockIdx.x * m2l_count;
  const unsigned* vmask = vmask_all + (int64_t)blockIdx.x * m2l_count;
  if (tid < TC) {
    int cell = tid < cnt ? cells[first + tid] : -1;
    tcell[tid] = cell;
    int ix = 0, iy = 0, iz = 0;
    if (cell >= 0) morton_decode((uint64_t)cell, ix, iy, iz);
    tco[3 * tid] = ix;
    tco[3 * tid + 1] = iy;
    tco[3 * tid + 2] = iz;
  }
  if (tid == 0) {
    for (int q = 0; q < NSTG; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], NCW);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int nv = nval_all[blockIdx.x];
  const int ks = blockIdx.y, kn = gridDim.y;
  const int sbeg = (int)((int64_t)nv * ks / kn), send = (int)((int64_t)nv * (ks + 1) / kn);
  const int nsteps = send - sbeg;
  volatile int* abf = abort_flag;

  if (warp == NCW) {
    // ---------------- producer warp
    const C<T>* opsl = ops + (int64_t)level * box_cells * P * P;
    const uint32_t op_bytes = (uint32_t)((size_t)P * P * sizeof(C<T>));
    const uint32_t row_bytes = (uint32_t)((size_t)P * sizeof(C<T>));
    for (int kk = 0; kk < nsteps; ++kk) {
      const int stg = kk % NSTG;
      bool ok = true;
      if (kk >= NSTG) ok = mbar_wait_abortable(&empty[stg], (uint32_t)(((kk / NSTG) - 1) & 1), abf);
      if (!__all_sync(0xffffffffu, ok)) break;
      const int st = sbeg + kk;
      const int i = vlist[st];
      const unsigned m = vmask[st];
      if (lane == 0) {
        fence_async_shared();
        mbar_expect_tx(&full[stg], op_bytes + (uint32_t)TC * row_bytes);
      }
      __syncwarp();
      if (lane == 0)
        bulk_copy_g2s(Ts + (size_t)stg * P * P, opsl + (int64_t)m2l_slot[b * m2l_count + i] * P * P,
                      op_bytes, &full[stg]);
      if (lane < TC) {
        const C<T>* src = zero_row;
        if ((m >> lane) & 1u) {
          const int o = m2l_off[b * m2l_count + i];
          int jx = tco[3 * lane] + (o & 255) - 128, jy = tco[3 * lane + 1] + ((o >> 8) & 255) - 128,
              jz = tco[3 * lane + 2] + ((o >> 16) & 255) - 128;
          src = d.M + (off + (int64_t)morton_encode(jx, jy, jz)) * P;
        }
        bulk_copy_g2s(Ms + ((size_t)stg * TC + lane) * MS, src, row_bytes, &full[stg]);
      }
    }
    // wait for the copies of the last stages to land before leaving
    for (int kk = (nsteps > NSTG ? nsteps - NSTG : 0); kk < nsteps; ++kk)
      if (lane == 0) mbar_wait_abortable(&full[kk % NSTG], (uint32_t)((kk / NSTG) & 1), abf);
    __syncwarp();
  } else {
    // ---------------- consumer warps
    const int r0 = tid / CT, c0 = tid % CT;
    C<T> acc[R][CM];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int j = 0; j < CM; ++j) acc[r][j] = mkc<T>(0, 0);
    bool ok = true;
    for (int kk = 0; kk < nsteps; ++kk) {
      const int stg = kk % NSTG;
      ok = mbar_wait_abortable(&full[stg], (uint32_t)((kk / NSTG) & 1), abf);
      if (!__all_sync(0xffffffffu, ok)) {
        ok = false;
        break;
      }
      m2l_block_product<T, R, CM, RT>(Ts + (size_t)stg * P * P, Ms + (size_t)stg * TC * MS, P, MS, r0, c0,
                                      acc);
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[stg]);
    }
    if (ok && !*abf) {
      C<T>* out = part ? part + (int64_t)ks * part_stride : nullptr;
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int j = 0; j < CM; ++j) {
          int ap = r0 + r * RT, c = c0 + j * CT;
          if (ap < P && c < cnt) {
            if (out) {
              out[(int64_t)(first + c) * P + ap] = acc[r][j];
            } else {
              C<T>* dst = d.Lc + (off + tcell[c]) * P + ap;
              *dst = accumulate ? cadd<T>(*dst, acc[r][j]) : acc[r][j];
            }
          }
        }
    }
  }
  __syncthreads();
  if (tid == 0 && *abf) atomicExch(&g_fmm_error, HFMM_ERR_TIMEOUT);
}

// L of every tile cell = sum over the split parts, in part order
template <typename T>
__global__ void k_m2l_reduce(FmmDev<T> d, const int4* __restrict__ tiles, const int* __restrict__ cells,
                             const int64_t* __restrict__ level_off, const C<T>* __restrict__ part,
                             int64_t part_stride, int nsplit, int accumulate) {
  HFMM_SKIP_IF(d);
  const int4 tile = tiles[blockIdx.x];
  const int P = d.P;
  const int64_t off = level_off[tile.x];
  for (int e = threadIdx.x; e < tile.w * P; e += blockDim.x) {
    int c = e / P, a = e - c * P;
    int64_t slot = (int64_t)(tile.z + c) * P + a;
    C<T> v = part[slot];
    for (int k = 1; k < nsplit; ++k) v = cadd<T>(v, part[k * part_stride + slot]);
    C<T>* dst = d.Lc + (off + cells[tile.z + c]) * P + a;
    *dst = accumulate ? cadd<T>(*dst, v) : v;
  }
}

// valid-offset lists of the tiles of target mask tm for source mask sm,
// built on first use and kept by the handle
int m2l_valid_lists(fmm_tree* t, int sm, int tm, cudaStream_t s) {
  const int ci = (tm - 1) * 3 + (sm - 1);
  if (t->m2l_vlist[ci]) return HFMM_OK;
  const int nt = t->m2l_ntiles[tm - 1];
  HFMM_TRY(tree_alloc_t(t, &t->m2l_vlist[ci], (size_t)nt * t->m2l_count + 1));
  HFMM_TRY(tree_alloc_t(t, &t->m2l_vmask[ci], (size_t)nt * t->m2l_count + 1));
  HFMM_TRY(tree_alloc_t(t, &t->m2l_nval[ci], (size_t)nt + 1));
  if (nt == 0) return HFMM_OK;
  k_m2l_valid<<<nt, 128, sizeof(unsigned) * t->m2l_count, s>>>(
      t->m2l_tiles[tm - 1], t->m2l_cells[tm - 1], t->flags, t->level_off_dev, t->m2l_off, t->m2l_count,
      sm, t->m2l_vlist[ci], t->m2l_vmask[ci], t->m2l_nval[ci]);
  count_launches(1);
  return hfmm_last_launch();
}

// ---- pair-list M2L (passes whose targets are the boundary cells)
//
// For a boundary-target pass most columns of a 32-cell tile would be empty
// for most offsets.  Here the valid (target, source) cell pairs are listed
// once per (target mask, source mask), grouped by (level, operator slot) and
// multiplied in chunks of 32 pairs that share one operator (bulk copies of
// the operator and the 32 source rows); each pair's product is a row of a
// buffer, and each target sums its rows in its own fixed order (deterministic).

// per tile cell: number of valid offsets (pass 1) or the pairs (pass 2)
__global__ void k_pairs_list(const int4* __restrict__ tiles, const int* __restrict__ cells,
                             const int* __restrict__ flags, const int64_t* __restrict__ level_off,
                             const int* __restrict__ m2l_off, const int* __restrict__ m2l_slot, int m2l_count,
                             int src_set, int* __restrict__ cnt, const int* __restrict__ csr,
                             int* __restrict__ ptgt, int* __restrict__ psrc, int* __restrict__ pkey,
                             int nslots) {
  const int4 tile = tiles[blockIdx.x];
  const int c = threadIdx.x;
  if (c >= tile.w) return;
  const int level = tile.x, b = tile.y;
  const int cell = cells[tile.z + c];
  const int64_t off = level_off[level];
  const int s = 1 << level;
  int ix, iy, iz;
  morton_decode((uint64_t)cell, ix, iy, iz);
  int n = 0;
  int base = csr ? csr[tile.z + c] : 0;
  for (int i = 0; i < m2l_count; ++i) {
    const int o = m2l_off[b * m2l_count + i];
    int jx = ix + (o & 255) - 128, jy = iy + ((o >> 8) & 255) - 128, jz = iz + ((o >> 16) & 255) - 128;
    if (jx < 0 || jy < 0 || jz < 0 || jx >= s || jy >= s || jz >= s) continue;
    int sc = (int)morton_encode(jx, jy, jz);
    if (!(flags[off + sc] & src_set)) continue;
    if (csr) {
      ptgt[base + n] = cell;
      psrc[base + n] = sc;
      pkey[base + n] = level * nslots + m2l_slot[b * m2l_count + i];
    }
    ++n;
  }
  if (!csr) cnt[tile.z + c] = n;
}

// exclusive scan of n counts (one block)
__global__ void k_scan_counts(const int* cnt, int n, int* out) {
  __shared__ int part[1024];
  const int tid = threadIdx.x;
  const int chunk = (n + blockDim.x - 1) / blockDim.x;
  const int lo = tid * chunk, hi = min(n, lo + chunk);
  int sum = 0;
  for (int i = lo; i < hi; ++i) sum += cnt[i];
  part[tid] = sum;
  __syncthreads();
  if (tid == 0) {
    int run = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) {
      int v = part[i];
      part[i] = run;
      run += v;
    }
    out[n] = run;
  }
  __syncthreads();
  int run = part[tid];
  for (int i = lo; i < hi; ++i) {
    out[i] = run;
    run += cnt[i];
  }
}

// group pair indices by key with per-group cursors (order inside a group is
// irrelevant to the result: each pair owns its output row)
__global__ void k_pairs_group(int64_t npairs, const int* __restrict__ pkey, int* __restrict__ cursor,
                              int* __restrict__ grouped) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= npairs) return;
  int pos = atomicAdd(&cursor[pkey[p]], 1);
  grouped[pos] = (int)p;
}
__global__ void k_count_keys(int64_t npairs, const int* __restrict__ pkey, int* __restrict__ kcnt) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p < npairs) atomicAdd(&kcnt[pkey[p]], 1);
}
// chunks of <= 32 pairs per key (one thread)
__global__ void k_pairs_chunks(int nkeys, int nslots, const int* __restrict__ kstart, int4* __restrict__ chunks,
                               int* __restrict__ nchunks) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int n = 0;
  for (int g = 0; g < nkeys; ++g) {
    int a = kstart[g], e = kstart[g + 1];
    for (int st = a; st < e; st += 32) chunks[n++] = make_int4(g / nslots, g % nslots, st, min(32, e - st));
  }
  *nchunks = n;
}

// one block per chunk: buf[pair] = T_slot M[source of pair] for its 32 pairs
template <typename T, int R, int CM, int RT>
__global__ void __launch_bounds__(RT * 8) k_m2l_pairs(FmmDev<T> d, const int4* __restrict__ chunks,
                                                      const int* __restrict__ grouped,
                                                      const int* __restrict__ psrc,
                                                      const int64_t* __restrict__ level_off,
                                                      const C<T>* __restrict__ ops, int64_t box_cells,
                                                      C<T>* __restrict__ buf) {
  HFMM_SKIP_IF(d);
  constexpr int CT = 8, TC = CT * CM;
  const int P = d.P;
  const int MS = P + 2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  int* pid = reinterpret_cast<int*>(smem_raw + 16);  // [TC]
  C<T>* Ts = reinterpret_cast<C<T>*>(smem_raw + 256);
  C<T>* Ms = Ts + (size_t)P * P;
  const int4 ch = chunks[blockIdx.x];
  const int level = ch.x, slot = ch.y, first = ch.z, cnt = ch.w;
  const int64_t off = level_off[level];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < TC) pid[tid] = tid < cnt ? grouped[first + tid] : -1;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const uint32_t op_bytes = (uint32_t)((size_t)P * P * sizeof(C<T>));
  const uint32_t row_bytes = (uint32_t)((size_t)P * sizeof(C<T>));
  if (warp == 0) {
    if (lane == 0) mbar_expect_tx(&bar[0], op_bytes + (uint32_t)TC * row_bytes);
    __syncwarp();
    if (lane == 0)
      bulk_copy_g2s(Ts, ops + ((int64_t)level * box_cells + slot) * P * P, op_bytes, &bar[0]);
    if (lane < TC) {
      const int p = pid[lane];
      const C<T>* row = p >= 0 ? d.M + (off + psrc[p]) * P : d.M + off * P;  // any valid row for padding
      bulk_copy_g2s(Ms + (size_t)lane * MS, row, row_bytes, &bar[0]);
    }
  }
  const bool ok = mbar_wait_bounded(&bar[0], 0);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) {
      atomicExch(&g_fmm_error, HFMM_ERR_TIMEOUT);
      mbar_wait_bounded(&bar[0], 0);
    }
    __syncthreads();
    return;
  }
  const int r0 = tid / CT, c0 = tid % CT;
  C<T> acc[R][CM];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int j = 0; j < CM; ++j) acc[r][j] = mkc<T>(0, 0);
  m2l_block_product<T, R, CM, RT>(Ts, Ms, P, MS, r0, c0, acc);
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int j = 0; j < CM; ++j) {
      int ap = r0 + r * RT, c = c0 + j * CT;
      if (ap < P && c < cnt) buf[(int64_t)pid[c] * P + ap] = acc[r][j];
    }
}

// L of each tile cell = (L +) sum of its pair rows, in its CSR order; one
// block per (tile, cell), one thread per coefficient (coalesced row reads)
template <typename T>
__global__ void k_pairs_reduce(FmmDev<T> d, const int4* __restrict__ tiles, const int* __restrict__ cells,
                               const int64_t* __restrict__ level_off, const int* __restrict__ csr,
                               const C<T>* __restrict__ buf, int accumulate) {
  HFMM_SKIP_IF(d);
  const int4 tile = tiles[blockIdx.x];
  const int c = blockIdx.y;
  if (c >= tile.w) return;
  const int P = d.P;
  const int64_t off = level_off[tile.x];
  const int lo = csr[tile.z + c], hi = csr[tile.z + c + 1];
  C<T>* dst = d.Lc + (off + cells[tile.z + c]) * P;
  for (int a = threadIdx.x; a < P; a += blockDim.x) {
    C<T> v0 = mkc<T>(0, 0), v1 = mkc<T>(0, 0);
    int q = lo;
    for (; q + 1 < hi; q += 2) {  // two independent chains, then combined
      v0 = cadd<T>(v0, buf[(int64_t)q * P + a]);
      v1 = cadd<T>(v1, buf[(int64_t)(q + 1) * P + a]);
    }
    if (q < hi) v0 = cadd<T>(v0, buf[(int64_t)q * P + a]);
    C<T> v = cadd<T>(v0, v1);
    dst[a] = accumulate ? cadd<T>(dst[a], v) : v;
  }
}

// builds the pair lists of (target mask tm, source mask sm) on first use
int m2l_pair_lists(fmm_tree* t, int sm, int tm, size_t csz, cudaStream_t s) {
  const int ci = (tm - 1) * 3 + (sm - 1);
  if (t->pr_csr[ci]) return HFMM_OK;
  const int mi = tm - 1;
  const int nt = t->m2l_ntiles[mi];
  const int64_t ncell = t->total_cells;  // tile cells index the cells array of the mask
  int* cnt = nullptr;
  HFMM_TRY(tree_alloc_t(t, &t->pr_csr[ci], ncell + 1));
  HFMM_CUDA_TRY(cudaMallocAsync((void**)&cnt, sizeof(int) * (ncell + 1), s));
  HFMM_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int) * (ncell + 1), s));
  if (nt) k_pairs_list<<<nt, 32, 0, s>>>(t->m2l_tiles[mi], t->m2l_cells[mi], t->flags, t->level_off_dev, t->m2l_off,
                                         t->m2l_box_index, t->m2l_count, sm, cnt, nullptr, nullptr, nullptr,
                                         nullptr, (int)t->box_cells);
  k_scan_counts<<<1, 1024, 0, s>>>(cnt, (int)ncell, t->pr_csr[ci]);
  HFMM_TRY(hfmm_last_launch());
  int np = 0;
  HFMM_CUDA_TRY(cudaMemcpyAsync(&np, t->pr_csr[ci] + ncell, sizeof(int), cudaMemcpyDeviceToHost, s));
  HFMM_CUDA_TRY(cudaStreamSynchronize(s));
  t->pr_npairs[ci] = np;
  const int nkeys = (t->L + 1) * (int)t->box_cells;
  int *pkey = nullptr, *kcnt = nullptr, *kstart = nullptr;
  HFMM_TRY(tree_alloc_t(t, &t->pr_tgt[ci], (size_t)np + 1));
  HFMM_TRY(tree_alloc_t(t, &t->pr_src[ci], (size_t)np + 1));
  HFMM_TRY(tree_alloc_t(t, &t->pr_grouped[ci], (size_t)np + 1));
  HFMM_TRY(tree_alloc_t(t, &t->pr_chunks[ci], (size_t)np / 32 + nkeys + 1));
  HFMM_CUDA_TRY(cudaMallocAsync((void**)&pkey, sizeof(int) * ((size_t)np + 1), s));
  HFMM_CUDA_TRY(cudaMallocAsync((void**)&kcnt, sizeof(int) * (nkeys + 1), s));
  HFMM_CUDA_TRY(cudaMallocAsync((void**)&kstart, sizeof(int) * (nkeys + 2), s));
  HFMM_CUDA_TRY(cudaMemsetAsync(kcnt, 0, sizeof(int) * (nkeys + 1), s));
  if (nt)
    k_pairs_list<<<nt, 32, 0, s>>>(t->m2l_tiles[mi], t->m2l_cells[mi], t->flags, t->level_off_dev, t->m2l_off,
                                   t->m2l_box_index, t->m2l_count, sm, nullptr, t->pr_csr[ci], t->pr_tgt[ci],
                                   t->pr_src[ci], pkey, (int)t->box_cells);
  if (np) k_count_keys<<<ceil_div(np, 256), 256, 0, s>>>(np, pkey, kcnt);
  k_scan_counts<<<1, 1024, 0, s>>>(kcnt, nkeys, kstart);
  HFMM_CUDA_TRY(cudaMemcpyAsync(kcnt, kstart, sizeof(int) * nkeys, cudaMemcpyDeviceToDevice, s));
  if (np) k_pairs_group<<<ceil_div(np, 256), 256, 0, s>>>(np, pkey, kcnt, t->pr_grouped[ci]);
  int* d_n = kcnt + nkeys;
  k_pairs_chunks<<<1, 1, 0, s>>>(nkeys, (int)t->box_cells, kstart, t->pr_chunks[ci], d_n);
  HFMM_TRY(hfmm_last_launch());
  int nchunks = 0;
  HFMM_CUDA_TRY(cudaMemcpyAsync(&nchunks, d_n, sizeof(int), cudaMemcpyDeviceToHost, s));
  HFMM_CUDA_TRY(cudaStreamSynchronize(s));
  t->pr_nchunks[ci] = nchunks;
  cudaFreeAsync(cnt, s);
  cudaFreeAsync(pkey, s);
  cudaFreeAsync(kcnt, s);
  cudaFreeAsync(kstart, s);
  if (np > t->pr_buf_pairs) {  // product buffer sized for the largest list
    HFMM_TRY(tree_alloc(t, &t->pr_buf, csz * (size_t)np * t->P));
    t->pr_buf_pairs = np;
  }
  count_launches(6);
  return HFMM_OK;
}

template <typename T, int R, int CM, int RT>
int launch_m2l_pairs_rt(fmm_tree* t, const FmmDev<T>& d, const C<T>* ops, int src_set, int tgt_set,
                        int accumulate, cudaStream_t s) {
  const int P = t->P, mi = tgt_set - 1, ci = mi * 3 + (src_set - 1);
  HFMM_TRY(m2l_pair_lists(t, src_set, tgt_set, sizeof(C<T>), s));
  const int TC = 8 * CM;
  const size_t sm = 256 + ((size_t)P * P + (size_t)TC * (P + 2)) * sizeof(C<T>);
  C<T>* buf = reinterpret_cast<C<T>*>(t->pr_buf);
  if (t->pr_nchunks[ci] > 0) {
    HFMM_TRY(set_smem<T>((const void*)k_m2l_pairs<T, R, CM, RT>, sm));
    k_m2l_pairs<T, R, CM, RT><<<t->pr_nchunks[ci], RT * 8, sm, s>>>(
        d, t->pr_chunks[ci], t->pr_grouped[ci], t->pr_src[ci], t->level_off_dev, ops, t->box_cells, buf);
  }
  if (t->m2l_ntiles[mi] > 0)
    k_pairs_reduce<T><<<dim3(t->m2l_ntiles[mi], t->m2l_tc), 64, 0, s>>>(
        d, t->m2l_tiles[mi], t->m2l_cells[mi], t->level_off_dev, t->pr_csr[ci], buf, accumulate);
  count_launches(2);
  return hfmm_last_launch();
}

template <typename T>
int launch_m2l_pairs(fmm_tree* t, const FmmDev<T>& d, const C<T>* ops, int src_set, int tgt_set, int accumulate,
                     cudaStream_t s) {
  const int P = t->P;
  if (P <= 16) return launch_m2l_pairs_rt<T, 1, 4, 16>(t, d, ops, src_set, tgt_set, accumulate, s);
  if (P <= 32) return launch_m2l_pairs_rt<T, 2, 4, 16>(t, d, ops, src_set, tgt_set, accumulate, s);
  if (P <= 36) return launch_m2l_pairs_rt<T, 3, 4, 12>(t, d, ops, src_set, tgt_set, accumulate, s);
  if (P <= 48) return launch_m2l_pairs_rt<T, 3, 4, 16>(t, d, ops, src_set, tgt_set, accumulate, s);
  if (P <= 64) return launch_m2l_pairs_rt<T, 4, 4, 16>(t, d, ops, src_set, tgt_set, accumulate, s);
  if (P <= 96) return launch_m2l_pairs_rt<T, 6, 4, 16>(t, d, ops, src_set, tgt_set, accumulate, s);
  return HFMM_ERR_UNSUPPORTED;
}

template <typename T, int CM, int R, int RT>
int launch_m2l_tma_rt(fmm_tree* t, const FmmDev<T>& d, const C<T>* ops, int src_set, int tgt_set,
                      int accumulate, cudaStream_t s, int nt_limit) {
  const int P = t->P, mi = tgt_set - 1;
  const int TC = 8 * CM;
  const int nt = nt_limit >= 0 ? std::min(nt_limit, t->m2l_ntiles[mi]) : t->m2l_ntiles[mi];
  if (nt == 0) return HFMM_OK;
  HFMM_TRY(m2l_valid_lists(t, src_set, tgt_set, s));
  const int ci = mi * 3 + (src_set - 1);
  size_t sm = 1024 + (2 * (size_t)P * P + 2 * (size_t)TC * (P + 2)) * sizeof(C<T>);
  // split the offset lists so that the grid fills the GPU a few times over
  const int tci = mi * 3 + (src_set - 1);
  const int variant = t->tuned_variant[tci] >= 0 ? t->tuned_variant[tci] : t->m2l_variant;
  const int fill = t->tuned_variant[tci] >= 0 ? t->tuned_fill[tci] : t->m2l_fill;
  int nsplit = (fill * 152 + nt - 1) / nt;
  if (nsplit > t->m2l_part_max) nsplit = t->m2l_part_max;
  if (nsplit < 1) nsplit = 1;
  C<T>* part = nsplit > 1 ? reinterpret_cast<C<T>*>(t->m2l_part) : nullptr;
  const int64_t pstride = t->total_cells * (int64_t)P;
  constexpr int NSTG = 3;
  size_t smw = 1024 + (NSTG * (size_t)P * P + NSTG * (size_t)TC * (P + 2)) * sizeof(C<T>);
  if (variant == 1 && smw <= 200 * 1024 && (RT * 8) % 32 == 0) {
    HFMM_TRY(set_smem<T>((const void*)k_m2l_ws<T, R, CM, RT, NSTG>, smw));
    k_m2l_ws<T, R, CM, RT, NSTG><<<dim3(nt, nsplit), RT * 8 + 32, smw, s>>>(
        d, t->m2l_tiles[mi], t->m2l_cells[mi], t->level_off_dev, ops, t->box_cells, t->m2l_off,
        t->m2l_box_index, t->m2l_count, t->m2l_vlist[ci], t->m2l_vmask[ci], t->m2l_nval[ci],
        reinterpret_cast<const C<T>*>(t->zero_row), part, pstride, accumulate);
  } else {
    HFMM_TRY(set_smem<T>((const void*)k_m2l_tma<T, R, CM, RT>, sm));
    k_m2l_tma<T, R, CM, RT><<<dim3(nt, nsplit), RT * 8, sm, s>>>(
        d, t->m2l_tiles[mi], t->m2l_cells[mi], t->level_off_dev, ops, t->box_cells, t->m2l_off,
        t->m2l_box_index, t->m2l_count, t->m2l_vlist[ci], t->m2l_vmask[ci], t->m2l_nval[ci],
        reinterpret_cast<const C<T>*>(t->zero_row), part, pstride, accumulate);
  }
  if (nsplit > 1)
    k_m2l_reduce<T><<<nt, 128, 0, s>>>(d, t->m2l_tiles[mi], t->m2l_cells[mi], t->level_off_dev, part,
                                       pstride, nsplit, accumulate);
  count_launches(nsplit > 1 ? 2 : 1);
  return hfmm_last_launch();
}

template <typename T, int CM>
int launch_m2l_tma(fmm_tree* t, const FmmDev<T>& d, const C<T>* ops, int src_set, int tgt_set,
                   int accumulate, cudaStream_t s, int nt_limit = -1) {
  const int P = t->P;
  if (P <= 16) return launch_m2l_tma_rt<T, CM, 1, 16>(t, d, ops, src_set, tgt_set, accumulate, s, nt_limit);
  if (P <= 32) return launch_m2l_tma_rt<T, CM, 2, 16>(t, d, ops, src_set, tgt_set, accumulate, s, nt_limit);
  if (P <= 36) return launch_m2l_tma_rt<T, CM, 3, 12>(t, d, ops, src_set, tgt_set, accumulate, s, nt_limit);
  if (P <= 48) return launch_m2l_tma_rt<T, CM, 3, 16>(t, d, ops, src_set, tgt_set, accumulate, s, nt_limit);
  if (P <= 64) return launch_m2l_tma_rt<T, CM, 4, 16>(t, d, ops, src_set, tgt_set, accumulate, s, nt_limit);
  if (P <= 96) return launch_m2l_tma_rt<T, CM, 6, 16>(t, d, ops, src_set, tgt_set, accumulate, s, nt_limit);
  return HFMM_ERR_UNSUPPORTED;
}

template <typename T, int CM>
int launch_m2l_tiled(fmm_tree* t, const FmmDev<T>& d, const C<T>* ops, const int64_t* level_off_dev,
                     int src_set, int tgt_set, int accumulate, cudaStream_t s) {
  const int P = t->P, mi = tgt_set - 1;
  const int TC = 8 * CM;
  size_t sm = ((size_t)P * P + (size_t)P * (TC + 1)) * sizeof(C<T>) + 5 * TC * sizeof(int);
  const int R = (P + 15) / 16;
  const void* fn = nullptr;
#define HFMM_M2L_CASE(RR)                                               \
  if (R <= RR) {                                                        \
    fn = (const void*)k_m2l_tiled<T, RR, CM>;                           \
    HFMM_TRY(set_smem<T>(fn, sm));                                      \
    k_m2l_tiled<T, RR, CM><<<t->m2l_ntiles[mi], 128, sm, s>>>(          \
        d, t->m2l_tiles[mi], t->m2l_cells[mi], level_off_dev, ops, t->box_cells, t->m2l_off, \
        t->m2l_box_index, t->m2l_count, src_set, accumulate);           \
    return hfmm_last_launch();                                          \
  }
  HFMM_M2L_CASE(1)
  HFMM_M2L_CASE(2)
  HFMM_M2L_CASE(3)
  HFMM_M2L_CASE(4)
  HFMM_M2L_CASE(6)
#undef HFMM_M2L_CASE
  return HFMM_ERR_UNSUPPORTED;
}

// ---------------------------------------------------------------- L2P
// phi_i = fac * sum_a L_a R_a(x_i - c)   (forward fac = i k; adjoint fac = 1)
template <typename T>
__global__ void k_l2p(FmmDev<T> d, int64_t leaf_off, int tgt_set, C<T> fac, const int* __restrict__ list) {
  HFMM_SKIP_IF(d);
  extern __shared__ unsigned char smem_raw[];
  C<T>* Ls = reinterpret_cast<C<T>*>(smem_raw);
  const int leaf = list ? list[blockIdx.x] : blockIdx.x;
  const int P = d.P;
  int lo, hi;
  leaf_range(d.leaf_start, d.leaf_mid, leaf, tgt_set, lo, hi);
  if (hi <= lo) return;
  for (int e = threadIdx.x; e < P; e += blockDim.x) Ls[e] = d.Lc[(leaf_off + leaf) * P + e];
  __syncthreads();
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    T dx, dy, dz;
    local_coords<T>(d, i, leaf, dx, dy, dz);
    T r, ct, st, cp, sp;
    direction<T>(dx, dy, dz, r, ct, st, cp, sp);
    T jn[HFMM_MAX_P];
    T pl[HFMM_MAX_P * (HFMM_MAX_P + 1) / 2];
    sph_bessel_j<T>(d.k * r, d.p, jn);
    legendre_bar<T>(ct, st, d.p, pl);
    C<T> acc = mkc<T>(0, 0);
    T er = T(1), ei = T(0);
    for (int m = 0; m < d.p; ++m) {
      for (int n = m; n < d.p; ++n) {
        T v = jn[n] * pl[n * (n + 1) / 2 + m];
        C<T> R = mkc<T>(v * er, v * ei);
        cfma<T>(acc, Ls[n * n + n + m], R);
        if (m > 0) {
          C<T> Rc = conjc<T>(R);
          if (m & 1) Rc = mkc<T>(-Rc.x, -Rc.y);
          cfma<T>(acc, Ls[n * n + n - m], Rc);
        }
      }
      T nr = er * cp - ei * sp, ni = er * sp + ei * cp;
      er = nr;
      ei = ni;
    }
    l2p_store<T>(d, i, cmul<T>(fac, acc));
  }
}

// d(phi_i)/dk = sum_a [(i L_a + i k dL_a) R_a + i k L_a dR_a/dk],
// dR_a/dk = |v| j_n'(k|v|) Y_a (tangent of L2P, written to `out`)
template <typename T>
__global__ void k_l2p_dk(FmmDev<T> d, const C<T>* __restrict__ Lv, const C<T>* __restrict__ Ldv,
                         C<T>* __restrict__ out, int64_t leaf_off, int tgt_set, const int* __restrict__ list) {
  HFMM_SKIP_IF(d);
  extern __shared__ unsigned char smem_raw[];
  C<T>* Ls = reinterpret_cast<C<T>*>(smem_raw);
  const int leaf = list ? list[blockIdx.x] : blockIdx.x;
  const int P = d.P;
  int lo, hi;
  leaf_range(d.leaf_start, d.leaf_mid, leaf, tgt_set, lo, hi);
  if (hi <= lo) return;
  C<T>* Lds = Ls + P;
  for (int e = threadIdx.x; e < P; e += blockDim.x) {
    Ls[e] = Lv[(leaf_off + leaf) * P + e];
    Lds[e] = Ldv[(leaf_off + leaf) * P + e];
  }
  __syncthreads();
  const T k = d.k;
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    T dx, dy, dz;
    local_coords<T>(d, i, leaf, dx, dy, dz);
    T r, ct, st, cp, sp;
    direction<T>(dx, dy, dz, r, ct, st, cp, sp);
    T jn[HFMM_MAX_P + 1];
    T pl[HFMM_MAX_P * (HFMM_MAX_P + 1) / 2];
    sph_bessel_j<T>(k * r, d.p + 1, jn);
    legendre_bar<T>(ct, st, d.p, pl);
    C<T> a1 = mkc<T>(0, 0), a2 = mkc<T>(0, 0), a3 = mkc<T>(0, 0);  // L.R, dL.R, L.dR
    T er = T(1), ei = T(0);
    for (int m = 0; m < d.p; ++m) {
      for (int n = m; n < d.p; ++n) {
        T pv = pl[n * (n + 1) / 2 + m];
        T v = jn[n] * pv;
        T djn = r * ((n > 0 ? T(n) * jn[n - 1] : T(0)) - T(n + 1) * jn[n + 1]) / T(2 * n + 1);
        T dv = djn * pv;
        C<T> R = mkc<T>(v * er, v * ei), dR = mkc<T>(dv * er, dv * ei);
        const int ap = n * n + n + m, am = n * n + n - m;
        cfma<T>(a1, Ls[ap], R);
        cfma<T>(a2, Lds[ap], R);
        cfma<T>(a3, Ls[ap], dR);
        if (m > 0) {
          C<T> Rc = conjc<T>(R), dRc = conjc<T>(dR);
          if (m & 1) {
            Rc = mkc<T>(-Rc.x, -Rc.y);
            dRc = mkc<T>(-dRc.x, -dRc.y);
          }
          cfma<T>(a1, Ls[am], Rc);
          cfma<T>(a2, Lds[am], Rc);
          cfma<T>(a3, Ls[am], dRc);
        }
      }
      T nr = er * cp - ei * sp, ni = er * sp + ei * cp;
      er = nr;
      ei = ni;
    }
    // i a1 + i k (a2 + a3)
    C<T> s = mkc<T>(a1.x + k * (a2.x + a3.x), a1.y + k * (a2.y + a3.y));
    out[i] = mkc<T>(-s.y, s.x);
  }
}

// ---------------------------------------------------------------- P2P
// One block per target leaf, one thread per target point (loops if more);
// source leaves of the near list staged through shared memory; j != i by
// sorted index.  FP32: partial sums per source leaf are added with Kahan
// compensation.  Self term s_i q_i added at the end.
template <typename T>
struct SrcPt {
  T x, y, z;
  int idx;
  C<T> q;
};

template <typename T>
__global__ void k_p2p(FmmDev<T> d, const int* near_off, int near_count, int src_set, int tgt_set,
                      double2 sig_vol, double2 sig_bnd) {
  HFMM_SKIP_IF(d);
  constexpr int TILE = 128;
  __shared__ SrcPt<T> tile[TILE];
  const int leaf = blockIdx.x;
  int tlo, thi;
  leaf_range(d.leaf_start, d.leaf_mid, leaf, tgt_set, tlo, thi);
  if (thi <= tlo) return;
  int ix, iy, iz;
  morton_decode((uint64_t)leaf, ix, iy, iz);
  const int s = 1 << d.L;
  const T w = T(ldexp(1.0, -d.L));
  const T k = d.k;
  const T inv4pi = T(0.07957747154594766788);
  for (int tbase = tlo; tbase < thi; tbase += blockDim.x) {
    const int i = tbase + threadIdx.x;
    const bool active = i < thi;
    T xi = 0, yi = 0, zi = 0;
    if (active) local_coords<T>(d, i, leaf, xi, yi, zi);
    C<T> tot = mkc<T>(0, 0), comp = mkc<T>(0, 0);
    for (int nb = 0; nb < near_count; ++nb) {
      int o = near_off[nb];
      int ox = (o & 255) - 128, oy = ((o >> 8) & 255) - 128, oz = ((o >> 16) & 255) - 128;
      int jx = ix + ox, jy = iy + oy, jz = iz + oz;
      if (jx < 0 || jy < 0 || jz < 0 || jx >= s || jy >= s || jz >= s) continue;
      int sleaf = (int)morton_encode(jx, jy, jz);
      int slo, shi;
      leaf_range(d.leaf_start, d.leaf_mid, sleaf, src_set, slo, shi);
      if (shi <= slo) continue;
      // source coordinates relative to the target leaf centre
      const T sx = T(ox) * w, sy = T(oy) * w, sz = T(oz) * w;
      C<T> part = mkc<T>(0, 0);
      for (int sbase = slo; sbase < shi; sbase += TILE) {
        __syncthreads();
        for (int e = threadIdx.x; e < TILE && sbase + e < shi; e += blockDim.x) {
          int j = sbase + e;
          T lx, ly, lz;
          local_coords<T>(d, j, sleaf, lx, ly, lz);
          tile[e].x = lx + sx;
          tile[e].y = ly + sy;
          tile[e].z = lz + sz;
          tile[e].idx = j;
          tile[e].q = d.qs[j];
        }
        __syncthreads();
        const int cnt = min(TILE, shi - sbase);
        if (active) {
          for (int e = 0; e < cnt; ++e) {
            T dx = xi - tile[e].x, dy = yi - tile[e].y, dz = zi - tile[e].z;
            T r2 = dx * dx + dy * dy + dz * dz;
            if (tile[e].idx == i) continue;
            T r = sqrt(r2);
            T sn, cs;
            if constexpr (sizeof(T) == 8) {
              sincos(k * r, &sn, &cs);
            } else {
              sincosf(k * r, &sn, &cs);
            }
            T g = inv4pi / r;
            C<T> G = mkc<T>(cs * g, sn * g);
            cfma<T>(part, G, tile[e].q);
          }
        }
      }
      if constexpr (sizeof(T) == 4) {  // Kahan addition of the leaf-pair sum
        T yx = part.x - comp.x, yy = part.y - comp.y;
        T tx = tot.x + yx, ty = tot.y + yy;
        comp.x = (tx - tot.x) - yx;
        comp.y = (ty - tot.y) - yy;
        tot.x = tx;
        tot.y = ty;
      } else {
        tot = cadd<T>(tot, part);
      }
    }
    if (active) {
      // self term for targets that are also sources
      int vol_end = d.leaf_mid[leaf];
      bool is_vol = i < vol_end;
      if ((is_vol && (src_set & HFMM_SET_VOL)) || (!is_vol && (src_set & HFMM_SET_BND))) {
        double2 sg = is_vol ? sig_vol : sig_bnd;
        cfma<T>(tot, mkc<T>(T(sg.x), T(sg.y)), d.qs[i]);
      }
      p2p_store<T>(d, i, tot);
    }
  }
}

// P2P, second form.  One block of 256 threads per target leaf.  The sources
// of all near leaves are staged in shared memory in windows of up to W
// points (coordinates relative to the target leaf centre, weights scaled by
// 1/(4 pi)); each target is served by `tpt` threads (a power of two chosen so
// that targets x tpt fills the block), each summing a strided share of the
// window, and the shares are combined with warp shuffles.  A source at zero
// distance from the target is the target itself (points are distinct) and
// contributes nothing.  Window sums are added with Kahan compensation.
template <typename T>
struct StagedSrc {
  T x, y, z, pad;
};

template <typename T>
__device__ __forceinline__ void sincos_kr(T ph, T& sn, T& cs) {
  if constexpr (sizeof(T) == 8) {
    sincos(ph, &sn, &cs);
  } else {
    // reduce to [-pi, pi] (one-constant Cody-Waite step), then the SFU
    const float n = rintf(ph * 0.15915494309189535f);
    const float r = fmaf(-n, 6.28318530717958648f, ph);
    sn = __sinf(r);
    cs = __cosf(r);
  }
}

template <typename T>
__device__ __forceinline__ T rsqrt_t(T x) {
  if constexpr (sizeof(T) == 8) return rsqrt(x);
  else return rsqrtf(x);
}

// KMODE 0: G = e^{ikr}/(4 pi r); 1: conj(G) (adjoint); 2: dG/dk = i e^{ikr}/(4 pi) (tangent);
// 3: dG/dn_y = (i k r - 1) e^{ikr} / (4 pi r^2) (y - x).n_y / r, boundary
// sources of a lattice tree (double layer; the staged record's fourth word
// carries the source's normal as +-(axis + 1)); no self term (the own flat
// panel contributes nothing)
template <typename T, int W, int KMODE>
__global__ void __launch_bounds__(256) k_p2p_v2(FmmDev<T> d, const int* __restrict__ near_off,
                                                int near_count, int src_set, int tgt_set,
                                                double2 sig_vol, double2 sig_bnd,
                                                const int* __restrict__ list) {
  HFMM_SKIP_IF(d);
  __shared__ StagedSrc<T> spos[W];
  __shared__ C<T> sq[W];
  __shared__ int nb_leaf[128], nb_lo[128], nb_cnt[128], nb_pre[129];
  __shared__ T nb_sh[128][3];
  __shared__ int n_nb;
  const int leaf = list ? list[blockIdx.x] : blockIdx.x;
  int tlo, thi;
  leaf_range(d.leaf_start, d.leaf_mid, leaf, tgt_set, tlo, thi);
  const int ntgt = thi - tlo;
  if (ntgt <= 0) return;
  const int tid = threadIdx.x;
  int ix, iy, iz;
  morton_decode((uint64_t)leaf, ix, iy, iz);
  const int s = 1 << d.L;
  const T w = T(ldexp(1.0, -d.L));
  // near leaves with sources: ranges and prefix sums
  if (tid < 32) {
    int base = 0;
    for (int c0 = 0; c0 < near_count; c0 += 32) {
      int i = c0 + tid;
      int cnt = 0, lo = 0, sl = 0, ox = 0, oy = 0, oz = 0;
      if (i < near_count) {
        int o = near_off[i];
        ox = (o & 255) - 128;
        oy = ((o >> 8) & 255) - 128;
        oz = ((o >> 16) & 255) - 128;
        int jx = ix + ox, jy = iy + oy, jz = iz + oz;
        if (jx >= 0 && jy >= 0 && jz >= 0 && jx < s && jy < s && jz < s) {
          sl = (int)morton_encode(jx, jy, jz);
          int hi;
          leaf_range(d.leaf_start, d.leaf_mid, sl, src_set, lo, hi);
          cnt = hi > lo ? hi - lo : 0;
        }
      }
      unsigned has = __ballot_sync(0xffffffffu, cnt > 0);
      int pos = base + __popc(has & ((1u << tid) - 1u));
      int v = cnt;  // inclusive scan of counts over the compacted lanes
      if (cnt > 0) {
        nb_leaf[pos] = sl;
        nb_lo[pos] = lo;
        nb_cnt[pos] = cnt;
        nb_sh[pos][0] = T(ox) * w;
        nb_sh[pos][1] = T(oy) * w;
        nb_sh[pos][2] = T(oz) * w;
      }
      (void)v;
      base += __popc(has);
    }
    if (tid == 0) {
      n_nb = base;
      int run = 0;
      for (int q = 0; q < base; ++q) {
        nb_pre[q] = run;
        run += nb_cnt[q];
      }
      nb_pre[base] = run;
    }
  }
  __syncthreads();
  const int nnb = n_nb;
  const int total = nb_pre[nnb];
  const T inv4pi = T(0.07957747154594766788);
  const T k = d.k;
  // threads per target
  int tpt = 1;
  while (tpt < 32 && (tpt * 2) * ntgt <= 256) tpt *= 2;
  const int tslots = 256 / tpt;
  const int sub = tid % tpt;
  for (int tb = 0; tb < ntgt; tb += tslots) {
    const int ti = tb + tid / tpt;
    const bool active = ti < ntgt;
    const int i = tlo + (active ? ti : 0);
    T xi, yi, zi;
    local_coords<T>(d, i, leaf, xi, yi, zi);
    C<T> tot = mkc<T>(0, 0), comp = mkc<T>(0, 0);
    for (int wb = 0; wb < total; wb += W) {
      const int wn = min(W, total - wb);
      __syncthreads();
      for (int e = tid; e < wn; e += 256) {
        const int g = wb + e;
        int lo = 0, hi = nnb;  // leaf of staged source g: last q with nb_pre[q] <= g
        while (hi - lo > 1) {
          int mid = (lo + hi) >> 1;
          if (nb_pre[mid] <= g) lo = mid;
          else hi = mid;
        }
        const int j = nb_lo[lo] + (g - nb_pre[lo]);
        T lx, ly, lz;
        local_coords<T>(d, j, nb_leaf[lo], lx, ly, lz);
        StagedSrc<T> sp;
        sp.x = lx + nb_sh[lo][0];
        sp.y = ly + nb_sh[lo][1];
        sp.z = lz + nb_sh[lo][2];
        sp.pad = T(0);
        if constexpr (KMODE == 3) {
          const int f = panel_face<T>(d, j);
          sp.pad = T((f & 1) ? (f >> 1) + 1 : -((f >> 1) + 1));
        }
        spos[e] = sp;
        sq[e] = cscale<T>(d.qs[j], inv4pi);
      }
      __syncthreads();
      C<T> part = mkc<T>(0, 0);
      if (active) {
#pragma unroll 4
        for (int e = sub; e < wn; e += tpt) {
          const StagedSrc<T> sp = spos[e];
          const T dx = xi - sp.x, dy = yi - sp.y, dz = zi - sp.z;
          const T r2 = fma(dx, dx, fma(dy, dy, dz * dz));
          T rinv = rsqrt_t<T>(r2);
          rinv = r2 > T(0) ? rinv : T(0);
          const T r = r2 * rinv;
          T sn, cs;
          sincos_kr<T>(k * r, sn, cs);
          const C<T> q = sq[e];
          if constexpr (KMODE == 0) {
            const T wr = q.x * rinv, wi = q.y * rinv;
            part.x = fma(cs, wr, fma(-sn, wi, part.x));
            part.y = fma(cs, wi, fma(sn, wr, part.y));
          } else if constexpr (KMODE == 1) {
            const T wr = q.x * rinv, wi = q.y * rinv;
            part.x = fma(cs, wr, fma(sn, wi, part.x));
            part.y = fma(cs, wi, fma(-sn, wr, part.y));
          } else if constexpr (KMODE == 2) {  // i e^{ikr} q (zero-distance pairs masked through rinv)
            const T m = rinv > T(0) ? T(1) : T(0);
            const T gr = -sn * m, gi = cs * m;
            part.x = fma(gr, q.x, fma(-gi, q.y, part.x));
            part.y = fma(gr, q.y, fma(gi, q.x, part.y));
          } else {  // (i k r - 1) e^{ikr} (y - x).n / r^3 q; y - x = -(dx, dy, dz)
            const int code = (int)sp.pad;
            const int ax = (code < 0 ? -code : code) - 1;
            const T dn = ax == 0 ? dx : (ax == 1 ? dy : dz);
            const T g = (code > 0 ? -dn : dn) * rinv * rinv * rinv;  // zero at zero distance
            const T kr = k * r;
            const T gr = g * (-cs - kr * sn), gi = g * (kr * cs - sn);
            part.x = fma(gr, q.x, fma(-gi, q.y, part.x));
            part.y = fma(gr, q.y, fma(gi, q.x, part.y));
          }
        }
      }
      if constexpr (sizeof(T) == 4) {
        T yx = part.x - comp.x, yy = part.y - comp.y;
        T tx = tot.x + yx, ty = tot.y + yy;
        comp.x = (tx - tot.x) - yx;
        comp.y = (ty - tot.y) - yy;
        tot.x = tx;
        tot.y = ty;
      } else {
        tot = cadd<T>(tot, part);
      }
    }
    // combine the tpt shares (consecutive lanes of one warp)
    for (int o = tpt >> 1; o > 0; o >>= 1) {
      tot.x += __shfl_xor_sync(0xffffffffu, tot.x, o);
      tot.y += __shfl_xor_sync(0xffffffffu, tot.y, o);
    }
    if (active && sub == 0) {
      const bool is_vol = i < d.leaf_mid[leaf];
      if (KMODE != 3 && ((is_vol && (src_set & HFMM_SET_VOL)) || (!is_vol && (src_set & HFMM_SET_BND)))) {
        double2 sg = is_vol ? sig_vol : sig_bnd;
        cfma<T>(tot, mkc<T>(T(sg.x), T(sg.y)), d.qs[i]);
      }
      p2p_store<T>(d, i, tot);
    }
  }
}

// P2P on lattice trees.  Every point is a node of h Z^3, so the kernel
// between a target and a source depends only on their integer offset d.
// With lin = (iz W + iy) W + ix (W = 2D + 1, D the largest offset component
// between near leaves) the offset is coded by delta = lin_t - lin_s, a
// bijection of [-D, D]^3 onto [-(W^3-1)/2, (W^3-1)/2] with -d <-> -delta;
// G(d) = G(-d), so the entry of the pair is tab[|delta|].  The half table is
// staged once per block in shared memory with bulk copies; blocks are
// persistent (two per SM in FP32, so that one block's leaf setup overlaps the
// other's sums) and take target leaves in turn.  Per pair: one broadcast read
// of the staged source {q, lin}, one table read and a complex multiply-add;
// no transcendental functions.  In FP32 a thread holds four consecutive
// targets, so each staged-source read (a 16-byte load, which the shared
// memory serves a quarter warp at a time) feeds four pairs; tpt threads per
// group of targets sum strided shares of a window of staged sources
// (consecutive sources of a leaf are consecutive lattice nodes, so the table
// reads of a warp fall in distinct banks); FP32 window sums are added with
// Kahan compensation.  KMODE 0: G; 1: conj(G) (adjoint).
template <typename T> struct LatSrc;
template <> struct LatSrc<float> { float4 v; };                       // q.x, q.y, lin (bits), 0
template <> struct LatSrc<double> { double2 q; int lin; int pad[3]; };

constexpr int LAT_THREADS = 512;
constexpr int LAT_WS = HFMM_LAT_WS;  // staged sources per window

__device__ __forceinline__ void lat_stage(LatSrc<float>& o, float2 q, int l) {
  o.v = make_float4(q.x, q.y, __int_as_float(l), 0.f);
}
__device__ __forceinline__ void lat_stage(LatSrc<double>& o, double2 q, int l) {
  o.q = q;
  o.lin = l;
}
__device__ __forceinline__ void lat_read(const LatSrc<float>& o, float2& q, int& l) {
  const float4 v = o.v;
  q = make_float2(v.x, v.y);
  l = __float_as_int(v.z);
}
__device__ __forceinline__ void lat_read(const LatSrc<double>& o, double2& q, int& l) {
  q = o.q;
  l = o.lin;
}

// TILE (FP32 only): the staged window is cut into groups of four consecutive
// staged sources {q0..q3, lin0..lin3}.  When a thread's four targets and a
// group are both runs of x-consecutive lattice nodes (lin, lin + 1, lin + 2,
// lin + 3), the 16 pairs use only the seven offsets delta - 3 .. delta + 3,
// delta = lin_t0 - lin_s0: seven table reads instead of sixteen; other
// groups take one table read per pair.  A partial last group is padded with
// zero weights at the group's first node (always a valid table offset).
struct LatGrp {
  float4 q01, q23;  // q0, q1 / q2, q3
  int4 l;           // lin0 .. lin3
};

template <typename T, int KMODE, bool TILE = false>
__global__ void __launch_bounds__(LAT_THREADS, sizeof(T) == 4 ? 2 : 1)
    k_p2p_lat(FmmDev<T> d, const int* __restrict__ near_off, int near_count, int src_set, int tgt_set,
              double2 sig_vol, double2 sig_bnd, const int* __restrict__ list, int nlist,
              const C<T>* __restrict__ tab, uint32_t tab_bytes, const int* __restrict__ lin, int tpt_max) {
  HFMM_SKIP_IF(d);
  extern __shared__ __align__(128) unsigned char lat_smem[];
  const C<T>* stab = reinterpret_cast<const C<T>*>(lat_smem);
  LatSrc<T>* ssrc = reinterpret_cast<LatSrc<T>*>(lat_smem + tab_bytes);
  __shared__ __align__(8) uint64_t bar;
  __shared__ int q_lo[128], q_cnt[128];
  __shared__ int nb_lo[128], nb_pre[129];
  __shared__ int n_nb;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    mbar_expect_tx(&bar, tab_bytes);
    constexpr uint32_t CH = 32768;
    for (uint32_t off = 0; off < tab_bytes; off += CH)
      bulk_copy_g2s(lat_smem + off, reinterpret_cast<const unsigned char*>(tab) + off,
                    tab_bytes - off < CH ? tab_bytes - off : CH, &bar);
  }
  const bool ok = mbar_wait_bounded(&bar, 0);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) {
      atomicExch(&g_fmm_error, HFMM_ERR_TIMEOUT);
      mbar_wait_bounded(&bar, 0);
    }
    __syncthreads();
    return;
  }
  const int s = 1 << d.L;
  for (int li = blockIdx.x; li < nlist; li += gridDim.x) {
    const int leaf = list[li];
    int tlo, thi;
    leaf_range(d.leaf_start, d.leaf_mid, leaf, tgt_set, tlo, thi);
    const int ntgt = thi - tlo;
    if (ntgt <= 0) continue;  // uniform over the block
    int ix, iy, iz;
    morton_decode((uint64_t)leaf, ix, iy, iz);
    __syncthreads();  // the previous leaf is done with the lists and the window
    // source ranges of the near leaves, one offset per thread
    for (int q = tid; q < near_count; q += LAT_THREADS) {
      int cnt = 0, lo = 0;
      const int o = near_off[q];
      const int jx = ix + (o & 255) - 128, jy = iy + ((o >> 8) & 255) - 128, jz = iz + ((o >> 16) & 255) - 128;
      if (jx >= 0 && jy >= 0 && jz >= 0 && jx < s && jy < s && jz < s) {
        int hi;
        leaf_range(d.leaf_start, d.leaf_mid, (int)morton_encode(jx, jy, jz), src_set, lo, hi);
        cnt = hi > lo ? hi - lo : 0;
      }
      q_lo[q] = lo;
      q_cnt[q] = cnt;
    }
    __syncthreads();
    // compaction and prefix sums of the non-empty ones (warp 0)
    if (warp == 0) {
      int base = 0, run = 0;
      for (int c0 = 0; c0 < near_count; c0 += 32) {
        const int q = c0 + lane;
        const int cnt = q < near_count ? q_cnt[q] : 0;
        const unsigned has = __ballot_sync(0xffffffffu, cnt > 0);
        int v = cnt;
        for (int o = 1; o < 32; o <<= 1) {
          const int u = __shfl_up_sync(0xffffffffu, v, o);
          if (lane >= o) v += u;
        }
        const int pos = base + __popc(has & ((1u << lane) - 1u));
        if (cnt > 0) {
          nb_lo[pos] = q_lo[q];
          nb_pre[pos + 1] = run + v;
        }
        run += __shfl_sync(0xffffffffu, v, 31);
        base += __popc(has);
      }
      if (lane == 0) {
        nb_pre[0] = 0;
        n_nb = base;
      }
    }
    __syncthreads();
    const int nnb = n_nb;
    const int total = nb_pre[nnb];
    // NT consecutive targets per thread share each source read; tpt threads
    // per group of NT targets (a power of two up to tpt_max <= 32) take
    // strided shares of the window
    constexpr int NT = sizeof(T) == 4 ? 4 : 1;
    const int nq = (ntgt + NT - 1) / NT;
    int tpt = 1;
    while (tpt < tpt_max && (tpt * 2) * nq <= LAT_THREADS) tpt *= 2;
    const int qslots = LAT_THREADS / tpt;
    const int sub = tid & (tpt - 1);
    for (int qb = 0; qb < nq; qb += qslots) {
      const int qi = qb + tid / tpt;
      const bool active = qi < nq;
      int lt[NT];
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const int ti = NT * qi + j;
        lt[j] = lin[tlo + ((active && ti < ntgt) ? ti : 0)];
      }
      C<T> tot[NT], comp[NT];
#pragma unroll
      for (int j = 0; j < NT; ++j) tot[j] = comp[j] = mkc<T>(0, 0);
      for (int wb = 0; wb < total; wb += LAT_WS) {
        const int wn = min(LAT_WS, total - wb);
        __syncthreads();
        if constexpr (TILE) {
          LatGrp* sgrp = reinterpret_cast<LatGrp*>(lat_smem + tab_bytes);
          for (int gi = tid; 4 * gi < wn; gi += LAT_THREADS) {
            float qx[4], qy[4];
            int ll[4];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
              const int e = 4 * gi + jj;
              if (e < wn) {
                const int g = wb + e;
                int lo = 0, hi = nnb;
                while (hi - lo > 1) {
                  const int mid = (lo + hi) >> 1;
                  if (nb_pre[mid] <= g) lo = mid;
                  else hi = mid;
                }
                const int j = nb_lo[lo] + (g - nb_pre[lo]);
                const C<T> qj = d.qs[j];
                qx[jj] = qj.x;
                qy[jj] = qj.y;
                ll[jj] = lin[j];
              } else {
                qx[jj] = 0.f;
                qy[jj] = 0.f;
                ll[jj] = ll[0];
              }
            }
            LatGrp G;
            G.q01 = make_float4(qx[0], qy[0], qx[1], qy[1]);
            G.q23 = make_float4(qx[2], qy[2], qx[3], qy[3]);
            G.l = make_int4(ll[0], ll[1], ll[2], ll[3]);
            sgrp[gi] = G;
          }
        } else {
          for (int e = tid; e < wn; e += LAT_THREADS) {
            const int g = wb + e;
            int lo = 0, hi = nnb;  // near leaf of staged source g: last q with nb_pre[q] <= g
            while (hi - lo > 1) {
              const int mid = (lo + hi) >> 1;
              if (nb_pre[mid] <= g) lo = mid;
              else hi = mid;
            }
            const int j = nb_lo[lo] + (g - nb_pre[lo]);
            lat_stage(ssrc[e], d.qs[j], lin[j]);
          }
        }
        __syncthreads();
        C<T> part[NT];
#pragma unroll
        for (int j = 0; j < NT; ++j) part[j] = mkc<T>(0, 0);
        if constexpr (TILE) {
          static_assert(sizeof(T) == 4, "the tiled near field is the FP32 form's");
          const LatGrp* sgrp = reinterpret_cast<const LatGrp*>(lat_smem + tab_bytes);
          const bool tcons = lt[1] == lt[0] + 1 && lt[2] == lt[0] + 2 && lt[3] == lt[0] + 3;
          const int ngw = active ? (wn + 3) >> 2 : 0;
          for (int gi = sub; gi < ngw; gi += tpt) {
            const float4 a = sgrp[gi].q01, b = sgrp[gi].q23;
            const int4 l4 = sgrp[gi].l;
            const C<T> q[4] = {mkc<T>(a.x, a.y), mkc<T>(a.z, a.w), mkc<T>(b.x, b.y), mkc<T>(b.z, b.w)};
            if (tcons && l4.y == l4.x + 1 && l4.z == l4.x + 2 && l4.w == l4.x + 3) {
              // pair (target i, source j): delta = D + i - j -> e[i - j + 3]
              const int D = lt[0] - l4.x;
              C<T> e[7];
#pragma unroll
              for (int m = 0; m < 7; ++m) e[m] = stab[abs(D + m - 3)];
#pragma unroll
              for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                  const C<T> g = e[i - j + 3];
                  if constexpr (KMODE == 0) {
                    part[i].x = fma(g.x, q[j].x, fma(-g.y, q[j].y, part[i].x));
                    part[i].y = fma(g.x, q[j].y, fma(g.y, q[j].x, part[i].y));
                  } else {
                    part[i].x = fma(g.x, q[j].x, fma(g.y, q[j].y, part[i].x));
                    part[i].y = fma(g.x, q[j].y, fma(-g.y, q[j].x, part[i].y));
                  }
                }
            } else {
              const int ls[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
              for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                  const C<T> g = stab[abs(lt[i] - ls[j])];
                  if constexpr (KMODE == 0) {
                    part[i].x = fma(g.x, q[j].x, fma(-g.y, q[j].y, part[i].x));
                    part[i].y = fma(g.x, q[j].y, fma(g.y, q[j].x, part[i].y));
                  } else {
                    part[i].x = fma(g.x, q[j].x, fma(g.y, q[j].y, part[i].x));
                    part[i].y = fma(g.x, q[j].y, fma(-g.y, q[j].x, part[i].y));
                  }
                }
            }
          }
        } else if (active) {
#pragma unroll 4
          for (int e = sub; e < wn; e += tpt) {
            C<T> q;
            int ls;
            lat_read(ssrc[e], q, ls);
#pragma unroll
            for (int j = 0; j < NT; ++j) {
              const C<T> g = stab[abs(lt[j] - ls)];
              if constexpr (KMODE == 0) {
                part[j].x = fma(g.x, q.x, fma(-g.y, q.y, part[j].x));
                part[j].y = fma(g.x, q.y, fma(g.y, q.x, part[j].y));
              } else {
                part[j].x = fma(g.x, q.x, fma(g.y, q.y, part[j].x));
                part[j].y = fma(g.x, q.y, fma(-g.y, q.x, part[j].y));
              }
            }
          }
        }
#pragma unroll
        for (int j = 0; j < NT; ++j) {
          if constexpr (sizeof(T) == 4) {
            const T yx = part[j].x - comp[j].x, yy = part[j].y - comp[j].y;
            const T tx = tot[j].x + yx, ty = tot[j].y + yy;
            comp[j].x = (tx - tot[j].x) - yx;
            comp[j].y = (ty - tot[j].y) - yy;
            tot[j].x = tx;
            tot[j].y = ty;
          } else {
            tot[j] = cadd<T>(tot[j], part[j]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < NT; ++j)
        for (int o = tpt >> 1; o > 0; o >>= 1) {
          tot[j].x += __shfl_xor_sync(0xffffffffu, tot[j].x, o);
          tot[j].y += __shfl_xor_sync(0xffffffffu, tot[j].y, o);
        }
      if (active && sub == 0) {
#pragma unroll
        for (int j = 0; j < NT; ++j) {
          const int ti = NT * qi + j;
          if (ti >= ntgt) break;
          const int i = tlo + ti;
          C<T> v = tot[j];
          const bool is_vol = i < d.leaf_mid[leaf];
          if ((is_vol && (src_set & HFMM_SET_VOL)) || (!is_vol && (src_set & HFMM_SET_BND))) {
            const double2 sg = is_vol ? sig_vol : sig_bnd;  // conjugated by the caller in adjoint mode
            cfma<T>(v, mkc<T>(T(sg.x), T(sg.y)), d.qs[i]);
          }
          p2p_store<T>(d, i, v);
        }
      }
    }
  }
}

// ---------------------------------------------------------------- gather / scatter

// qs[pos(o)] = scale q[o] for the original indices o of the point sets in
// `src_set` (points outside the set keep stale values: no kernel reads them);
// the boundary vector is complex128 or complex64 (QB)
template <typename T, typename QB>
__global__ void k_gather(const int64_t* __restrict__ pos_of, int64_t o0, int64_t o1, int64_t n_vol,
                         const double2* __restrict__ q_vol, double s_vol, const QB* __restrict__ q_bnd,
                         double s_bnd, C<T>* qs, const int* skip) {
  if (skip && *skip) return;
  const int64_t o = o0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (o >= o1) return;
  C<T> v;
  if (o < n_vol) {
    const double2 q = q_vol[o];
    v = mkc<T>(T(q.x * s_vol), T(q.y * s_vol));
  } else {
    const QB q = q_bnd[o - n_vol];
    v = mkc<T>(T(q.x * s_bnd), T(q.y * s_bnd));
  }
  qs[pos_of[o]] = v;
}

// out[o] = phis[pos(o)] for the original indices o of `tgt_set`
template <typename T, typename OB>
__global__ void k_scatter(const int64_t* __restrict__ pos_of, int64_t o0, int64_t o1, int64_t n_vol,
                          const C<T>* __restrict__ phis, double2* phi_vol, OB* phi_bnd, const int* skip) {
  if (skip && *skip) return;
  const int64_t o = o0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (o >= o1) return;
  const C<T> v = phis[pos_of[o]];
  if (o < n_vol)
    phi_vol[o] = make_double2((double)v.x, (double)v.y);
  else
    phi_bnd[o - n_vol] = mkc<decltype(phi_bnd->x)>(v.x, v.y);
}

template <typename T>
FmmDev<T> make_dev(fmm_tree* t) {
  FmmDev<T> d;
  d.xyz = t->xyz;
  d.xyz32 = reinterpret_cast<const float4*>(t->xyz32);
  d.leaf_start = t->leaf_start;
  d.leaf_mid = t->leaf_mid;
  d.flags = t->flags;
  d.M = reinterpret_cast<C<T>*>(t->M);
  d.Lc = reinterpret_cast<C<T>*>(t->Lc);
  d.qs = reinterpret_cast<const C<T>*>(t->qs);
  d.phis = reinterpret_cast<C<T>*>(t->phis);
  d.p = t->p;
  d.P = t->P;
  d.L = t->L;
  d.k = T(t->k);
  d.skip = t->skip;
  d.near = nullptr;
  d.orig = t->orig;
  d.n_vol = t->n_vol;
  d.nn = (int64_t)t->n * t->n;
  return d;
}

int threads_for(int P) {  // four threads per expansion coefficient (M2M / L2L)
  int th = ((4 * P + 31) / 32) * 32;
  if (th > 1024) th = 1024;
  return th;
}

// Raises a kernel's dynamic shared-memory limit to at least `bytes`.  The
// limit is process-wide state of the function, and handles driven from
// several host threads (batched solves) launch the same kernel with
// different sizes, so it is only ever raised (under a lock), never lowered.
template <typename T>
int set_smem(const void* fn, size_t bytes) {
  if (bytes <= 48 * 1024) return HFMM_OK;
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> limit;
  int dev = 0;
  HFMM_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = limit[{dev, fn}];
  if (cur >= bytes) return HFMM_OK;
  HFMM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  cur = bytes;
  return HFMM_OK;
}

// M2L over all levels with the kernel that fits P and the precision;
// reads d.M, writes (or adds to) d.Lc
template <typename T>
int m2l_stage(fmm_tree* t, const FmmDev<T>& d, const C<T>* m2l, int src_set, int tgt_set, int accumulate,
              cudaStream_t s, int* nlaunch) {
  const int P = t->P, L = t->L;
  const int64_t PP = (int64_t)P * P;
  const bool tiled = (sizeof(T) == 4 && P <= 81) || (sizeof(T) == 8 && P <= 64);
  const bool tma = tiled && (P % 2 == 0);  // rows are 16-byte multiples; pairs of columns per load
  if (tma) {
    *nlaunch = 0;  // counted by the launcher
    const int ci = (tgt_set - 1) * 3 + (src_set - 1);
    const bool pairs = t->tuned_variant[ci] >= 0 ? t->tuned_variant[ci] == 2
                                                 : (t->m2l_pairs_enabled && tgt_set == HFMM_SET_BND &&
                                                    src_set == HFMM_SET_BND);
    if (pairs) return launch_m2l_pairs<T>(t, d, m2l, src_set, tgt_set, accumulate, s);
    // tensor cores for the levels >= lmin of the forward far field (volume
    // targets by default), the tiled kernel for the levels below
    if constexpr (sizeof(T) == 4) {
      const int lmin = m2l_tc_lmin(t);
      const bool fwd = (const void*)m2l == (const void*)t->op_m2l32 && (void*)d.M == t->M && (void*)d.Lc == t->Lc;
      const bool pass_ok = t->use_m2l_tcore >= 2 || (tgt_set & HFMM_SET_VOL);
      if (lmin && fwd && pass_ok) {
        const int nlow = t->m2l_tiles_lt[tgt_set - 1][lmin];
        if (nlow > 0) {
          if (t->m2l_tc == 32) HFMM_TRY(launch_m2l_tma<T, 4>(t, d, m2l, src_set, tgt_set, accumulate, s, nlow));
          else HFMM_TRY(launch_m2l_tma<T, 2>(t, d, m2l, src_set, tgt_set, accumulate, s, nlow));
        }
        int ntc = 0;
        HFMM_TRY(m2l_tc_stage(t, src_set, tgt_set, accumulate, s, &ntc));
        count_launches(ntc);
        return HFMM_OK;
      }
    }
    if (t->m2l_tc == 32) return launch_m2l_tma<T, 4>(t, d, m2l, src_set, tgt_set, accumulate, s);
    return launch_m2l_tma<T, 2>(t, d, m2l, src_set, tgt_set, accumulate, s);
  }
  if (tiled) {
    *nlaunch = 1;
    if (t->m2l_tc == 32)  // tiles hold up to 32 cells: 8 column groups x 4
      return launch_m2l_tiled<T, 4>(t, d, m2l, t->level_off_dev, src_set, tgt_set, accumulate, s);
    return launch_m2l_tiled<T, 2>(t, d, m2l, t->level_off_dev, src_set, tgt_set, accumulate, s);
  }
  const int th = threads_for(P);
  const size_t sm1 = (size_t)P * sizeof(C<T>);
  for (int l = 2; l <= L; ++l)
    k_m2l<T><<<1 << (3 * l), th, sm1, s>>>(d, l, t->level_off[l], m2l + (int64_t)l * t->box_cells * PP,
                                            t->m2l_off, t->m2l_box_index, t->m2l_count, src_set, tgt_set,
                                            accumulate);
  *nlaunch = L - 1;
  return hfmm_last_launch();
}

static int sm_count() {
  static int c = 0;
  if (!c) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    c = v > 0 ? v : 1;
  }
  return c;
}

template <typename T>
int launch_p2m(fmm_tree* t, const FmmDev<T>& d, C<T>* Mout, int src_set, C<T> fac, cudaStream_t s) {
  const int L = t->L, P = t->P;
  const int na = act_n(t, src_set, L);
  if (!na) return HFMM_OK;
  if (t->rtab && t->use_rtab) {
    k_p2m_tab<T><<<na, 64, 0, s>>>(d, reinterpret_cast<const C<T>*>(t->rtab), Mout, t->level_off[L], src_set, fac,
                                   act_list(t, src_set, L));
    return hfmm_last_launch();
  }
  const int chunk = 32;
  const size_t sm_p2m = (size_t)chunk * P * sizeof(C<T>);
  HFMM_TRY(set_smem<T>((const void*)k_p2m<T, 0>, sm_p2m));
  k_p2m<T, 0><<<na, 64, sm_p2m, s>>>(d, Mout, t->level_off[L], src_set, chunk, fac, act_list(t, src_set, L));
  return hfmm_last_launch();
}

// dipole P2M over the boundary panels (double layer): generic kernel, the
// basis rows being normal derivatives
template <typename T>
int launch_p2m_dipole(fmm_tree* t, const FmmDev<T>& d, C<T>* Mout, cudaStream_t s) {
  const int L = t->L, P = t->P;
  const int na = act_n(t, HFMM_SET_BND, L);
  if (!na) return HFMM_OK;
  const int chunk = 32;
  const size_t sm_p2m = (size_t)chunk * P * sizeof(C<T>);
  HFMM_TRY(set_smem<T>((const void*)k_p2m<T, 2>, sm_p2m));
  k_p2m<T, 2><<<na, 64, sm_p2m, s>>>(d, Mout, t->level_off[L], HFMM_SET_BND, chunk, mkc<T>(1, 0),
                                     act_list(t, HFMM_SET_BND, L));
  return hfmm_last_launch();
}

template <typename T>
int launch_l2p(fmm_tree* t, const FmmDev<T>& d, int tgt_set, C<T> fac, cudaStream_t s) {
  const int L = t->L, P = t->P;
  const int na = act_n(t, tgt_set, L);
  if (!na) return HFMM_OK;
  const size_t sm1 = (size_t)P * sizeof(C<T>);
  if (t->rtab && t->use_rtab) {
    k_l2p_tab<T><<<na, 256, sm1, s>>>(d, reinterpret_cast<const C<T>*>(t->rtab), t->level_off[L], tgt_set, fac,
                                      act_list(t, tgt_set, L));
    return hfmm_last_launch();
  }
  k_l2p<T><<<na, 64, sm1, s>>>(d, t->level_off[L], tgt_set, fac, act_list(t, tgt_set, L));
  return hfmm_last_launch();
}

template <typename T, int KMODE>
int launch_p2p_lat(fmm_tree* t, const FmmDev<T>& d, int src_set, int tgt_set, double2 sv, double2 sb,
                   cudaStream_t s) {
  const int na = act_n(t, tgt_set, t->L);
  if (!na) return HFMM_OK;
  const int64_t nh = t->lat_half;  // half-table entries, padded to 16 bytes
  const uint32_t tab_bytes = (uint32_t)(nh * sizeof(C<T>));
  const size_t smem = tab_bytes + (size_t)LAT_WS * sizeof(LatSrc<T>);
  // the autotuner's choice for this pass, else the defaults
  const int ci = 3 * (tgt_set - 1) + (src_set - 1);
  const bool tuned = t->tuned_p2p_tpt[ci] > 0;
  const bool tile = tuned ? t->tuned_p2p_tile[ci] != 0 : t->lat_tile != 0;
  const int tpt_max = tuned ? t->tuned_p2p_tpt[ci] : 32;
  auto kern = k_p2p_lat<T, KMODE, false>;
  if constexpr (sizeof(T) == 4) {
    if (tile) kern = k_p2p_lat<T, KMODE, true>;
  }
  HFMM_TRY(set_smem<T>((const void*)kern, smem));
  int per_sm = 0;
  HFMM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, LAT_THREADS, smem));
  if (per_sm < 1) return HFMM_ERR_UNSUPPORTED;
  if (tuned) {
    if (t->tuned_p2p_blocks[ci] > 0) per_sm = std::min(per_sm, t->tuned_p2p_blocks[ci]);
  } else if (d.near && !(src_set & HFMM_SET_VOL)) {
    // boundary-only near field on the side stream (concurrent with the far
    // field): one block per SM, so that the far-field kernels find shared
    // memory next to it (with volume sources the near field is the larger
    // part and keeps two)
    per_sm = 1;
  }
  const int grid = std::min(na, per_sm * sm_count());
  kern<<<grid, LAT_THREADS, smem, s>>>(d, t->near_off, t->near_count, src_set, tgt_set, sv, sb,
                                       act_list(t, tgt_set, t->L), na,
                                       reinterpret_cast<const C<T>*>(sizeof(T) == 4 ? (const void*)t->lat_tab32
                                                                                    : (const void*)t->lat_tab64),
                                       tab_bytes, t->lat_lin, tpt_max);
  return hfmm_last_launch();
}

template <typename T, int KMODE>
int p2p_stage(fmm_tree* t, const FmmDev<T>& d, int src_set, int tgt_set, double2 sv, double2 sb,
              cudaStream_t s) {
  const int nleaf = 1 << (3 * t->L);
  if constexpr (KMODE == 0 || KMODE == 1) {
    if (t->lat_D > 0 && t->use_lattice_p2p && t->near_count <= 128 &&
        (sizeof(T) == 4 || t->lat_tab64_fits))
      return launch_p2p_lat<T, KMODE>(t, d, src_set, tgt_set, sv, sb, s);
  }
  if (t->near_count <= 128) {
    const int na = act_n(t, tgt_set, t->L);
    if (na)
      k_p2p_v2<T, (sizeof(T) == 4 ? 1536 : 768), KMODE><<<na, 256, 0, s>>>(
          d, t->near_off, t->near_count, src_set, tgt_set, sv, sb, act_list(t, tgt_set, t->L));
    return hfmm_last_launch();
  }
  if (KMODE != 0) return HFMM_ERR_UNSUPPORTED;
  k_p2p<T><<<nleaf, 128, 0, s>>>(d, t->near_off, t->near_count, src_set, tgt_set, sv, sb);
  return hfmm_last_launch();
}

template <typename T>
const C<T>* ops_of(const fmm_tree* t, const double2* o64, const float2* o32) {
  return reinterpret_cast<const C<T>*>(sizeof(T) == 4 ? (const void*)o32 : (const void*)o64);
}

// Adjoint pass (every stage conjugate-transposed, in reverse order).  The
// weights y in qs live on the forward targets (tgt_set); the result on the
// forward sources (src_set) goes to phis.  With S' = tgt_set, T' = src_set:
//   Lh_L  = (-i k) P2M(y)                       (L2P^H)
//   Lh_l  = sum_o L2L_o^H Lh_{l+1}              (L2L^H, upward)
//   Mh_l  = M2L^H Lh_l                          (slot of -v, conjugate transpose)
//   Mh_{l+1} += M2M_o^H Mh_l                    (M2M^H, downward)
//   phi   = L2P(Mh_L) without the i k factor    (P2M^H)
//   phi  += conj(G) y near field + conj(s) y    (P2P^H, self term)
template <typename T>
int core_adjoint_impl(fmm_tree* t, int src_set, int tgt_set, cudaStream_t s) {
  HFMM_TRY(build_operators_adjoint(t, s));
  FmmDev<T> d = make_dev<T>(t);
  const int P = t->P, L = t->L;
  const int64_t PP = (int64_t)P * P;
  const int th = threads_for(P);
  const C<T>* m2m_h = ops_of<T>(t, t->op_m2m_h, t->op_m2m_h32);
  const C<T>* l2l_h = ops_of<T>(t, t->op_l2l_h, t->op_l2l_h32);
  const C<T>* m2l_h = ops_of<T>(t, t->op_m2l_h, t->op_m2l_h32);
  C<T>* Lh = d.Lc;  // cotangents of the local expansions
  C<T>* Mh = d.M;   // cotangents of the multipole expansions
  const int Sp = tgt_set, Tp = src_set;
  HFMM_TRY(launch_p2m<T>(t, d, Lh, Sp, mkc<T>(0, -d.k), s));
  size_t sm8 = 8 * (size_t)P * sizeof(C<T>);
  HFMM_TRY(set_smem<T>((const void*)k_m2m<T>, sm8));
  for (int l = L - 1; l >= 2; --l)
    if (act_n(t, Sp, l))
      k_m2m<T><<<act_n(t, Sp, l), th, sm8, s>>>(d, l, t->level_off[l], t->level_off[l + 1], Lh, Lh,
                                            l2l_h + (int64_t)l * 8 * PP, Sp, 0, act_list(t, Sp, l));
  FmmDev<T> dm = d;
  dm.M = Lh;
  dm.Lc = Mh;
  int nm = 0;
  HFMM_TRY(m2l_stage<T>(t, dm, m2l_h, Sp, Tp, 0, s, &nm));
  size_t sm1 = (size_t)P * sizeof(C<T>);
  for (int l = 2; l < L; ++l)
    if (act_n(t, Tp, l + 1))
      k_l2l<T><<<act_n(t, Tp, l + 1), th, sm1, s>>>(d, t->level_off[l], t->level_off[l + 1], Mh, Mh,
                                                  m2m_h + (int64_t)l * 8 * PP, Tp, act_list(t, Tp, l + 1));
  FmmDev<T> dl = d;
  dl.Lc = Mh;
  HFMM_TRY(launch_l2p<T>(t, dl, Tp, mkc<T>(1, 0), s));
  const double2 cv = make_double2(t->sigma_vol.x, -t->sigma_vol.y);
  const double2 cb = make_double2(t->sigma_bnd.x, -t->sigma_bnd.y);
  HFMM_TRY(p2p_stage<T, 1>(t, d, Sp, Tp, cv, cb, s));
  count_launches(4 + 2 * (L > 2 ? L - 2 : 0) + nm);
  return hfmm_last_launch();
}

// Tangent pass: d(phi)/dk for fixed weights q (in qs), into phis_d.
//   M, dM  = P2M(q), P2M_k(q)
//   dM_l   = T dM_{l+1} + dT M_{l+1}            (M2M)
//   dL_l   = T dM + dT M                        (M2L)
//   dL_{l+1} += T dL_l + dT L_l                 (L2L)
//   dphi   = i L.R + i k dL.R + i k L.dR        (L2P)
//   dphi  += dG/dk near field + ds/dk q          (P2P, self term)
template <typename T>
int core_dk_impl(fmm_tree* t, int src_set, int tgt_set, cudaStream_t s) {
  HFMM_TRY(build_operators_deriv(t, s));
  const int P = t->P, L = t->L;
  const size_t csz = sizeof(C<T>);
  if (!t->Md) {
    HFMM_TRY(tree_alloc(t, &t->Md, csz * t->total_cells * P));
    HFMM_TRY(tree_alloc(t, &t->Ld, csz * t->total_cells * P));
    HFMM_TRY(tree_alloc(t, &t->phis_d, csz * t->n_pts));
    HFMM_CUDA_TRY(cudaMemsetAsync(t->Md, 0, csz * t->total_cells * P, s));
    HFMM_CUDA_TRY(cudaMemsetAsync(t->Ld, 0, csz * t->total_cells * P, s));
  }
  FmmDev<T> d = make_dev<T>(t);
  const int64_t PP = (int64_t)P * P;
  const int th = threads_for(P);
  const C<T>* m2m = ops_of<T>(t, t->op_m2m, t->op_m2m32);
  const C<T>* l2l = ops_of<T>(t, t->op_l2l, t->op_l2l32);
  const C<T>* m2l = ops_of<T>(t, t->op_m2l, t->op_m2l32);
  const C<T>* m2m_d = ops_of<T>(t, t->op_m2m_d, t->op_m2m_d32);
  const C<T>* l2l_d = ops_of<T>(t, t->op_l2l_d, t->op_l2l_d32);
  const C<T>* m2l_d = ops_of<T>(t, t->op_m2l_d, t->op_m2l_d32);
  C<T>* Md = reinterpret_cast<C<T>*>(t->Md);
  C<T>* Ld = reinterpret_cast<C<T>*>(t->Ld);
  C<T>* phd = reinterpret_cast<C<T>*>(t->phis_d);
  const int chunk = 32;
  size_t sm_p2m = (size_t)chunk * P * csz;
  HFMM_TRY(set_smem<T>((const void*)k_p2m<T, 1>, sm_p2m));
  HFMM_TRY(launch_p2m<T>(t, d, d.M, src_set, mkc<T>(1, 0), s));
  if (act_n(t, src_set, L))
    k_p2m<T, 1><<<act_n(t, src_set, L), 64, sm_p2m, s>>>(d, Md, t->level_off[L], src_set, chunk, mkc<T>(1, 0), act_list(t, src_set, L));
  size_t sm8 = 8 * (size_t)P * csz;
  HFMM_TRY(set_smem<T>((const void*)k_m2m<T>, sm8));
  for (int l = L - 1; l >= 2; --l) {
    const int64_t o = (int64_t)l * 8 * PP;
    if (act_n(t, src_set, l))
      k_m2m<T><<<act_n(t, src_set, l), th, sm8, s>>>(d, l, t->level_off[l], t->level_off[l + 1], d.M, d.M, m2m + o,
                                            src_set, 0, act_list(t, src_set, l));
    if (act_n(t, src_set, l))
      k_m2m<T><<<act_n(t, src_set, l), th, sm8, s>>>(d, l, t->level_off[l], t->level_off[l + 1], Md, Md, m2m + o,
                                            src_set, 0, act_list(t, src_set, l));
    if (act_n(t, src_set, l))
      k_m2m<T><<<act_n(t, src_set, l), th, sm8, s>>>(d, l, t->level_off[l], t->level_off[l + 1], d.M, Md, m2m_d + o,
                                            src_set, 1, act_list(t, src_set, l));
  }
  int n1 = 0, n2 = 0, n3 = 0;
  HFMM_TRY(m2l_stage<T>(t, d, m2l, src_set, tgt_set, 0, s, &n1));  // L
  FmmDev<T> dd = d;
  dd.M = Md;
  dd.Lc = Ld;
  HFMM_TRY(m2l_stage<T>(t, dd, m2l, src_set, tgt_set, 0, s, &n2));  // dL = T dM
  FmmDev<T> dx = d;
  dx.Lc = Ld;
  HFMM_TRY(m2l_stage<T>(t, dx, m2l_d, src_set, tgt_set, 1, s, &n3));  // dL += dT M
  size_t sm1 = (size_t)P * csz;
  for (int l = 2; l < L; ++l) {
    const int64_t o = (int64_t)l * 8 * PP;
    if (act_n(t, tgt_set, l + 1))
      k_l2l<T><<<act_n(t, tgt_set, l + 1), th, sm1, s>>>(d, t->level_off[l], t->level_off[l + 1], d.Lc, d.Lc, l2l + o,
                                                  tgt_set, act_list(t, tgt_set, l + 1));
    if (act_n(t, tgt_set, l + 1))
      k_l2l<T><<<act_n(t, tgt_set, l + 1), th, sm1, s>>>(d, t->level_off[l], t->level_off[l + 1], Ld, Ld, l2l + o,
                                                  tgt_set, act_list(t, tgt_set, l + 1));
    if (act_n(t, tgt_set, l + 1))
      k_l2l<T><<<act_n(t, tgt_set, l + 1), th, sm1, s>>>(d, t->level_off[l], t->level_off[l + 1], d.Lc, Ld,
                                                  l2l_d + o, tgt_set, act_list(t, tgt_set, l + 1));
  }
  if (act_n(t, tgt_set, L))
    k_l2p_dk<T><<<act_n(t, tgt_set, L), 64, 2 * sm1, s>>>(d, d.Lc, Ld, phd, t->level_off[L], tgt_set,
                                                          act_list(t, tgt_set, L));
  FmmDev<T> dp = d;
  dp.phis = phd;
  HFMM_TRY(p2p_stage<T, 2>(t, dp, src_set, tgt_set, t->dsigma_vol, t->dsigma_bnd, s));
  count_launches(4 + 6 * (L > 2 ? L - 2 : 0) + n1 + n2 + n3);
  return hfmm_last_launch();
}

// dipole: double-layer pass (boundary sources with their outward normals,
// dipole P2M and P2P, no self term); otherwise the single-layer pass
template <typename T>
int core_impl(fmm_tree* t, int src_set, int tgt_set, cudaStream_t s, bool dipole = false) {
  FmmDev<T> d = make_dev<T>(t);
  const int P = t->P, L = t->L;
  const int nleaf = 1 << (3 * L);
  const C<T>* m2m = reinterpret_cast<const C<T>*>(sizeof(T) == 4 ? (void*)t->op_m2m32 : (void*)t->op_m2m);
  const C<T>* l2l = reinterpret_cast<const C<T>*>(sizeof(T) == 4 ? (void*)t->op_l2l32 : (void*)t->op_l2l);
  const C<T>* m2l = reinterpret_cast<const C<T>*>(sizeof(T) == 4 ? (void*)t->op_m2l32 : (void*)t->op_m2l);
  const int64_t PP = (int64_t)P * P;
  const int th = threads_for(P);
  (void)nleaf;

  StageTimer& tm = t->timer;
  // near field on its own stream, concurrent with the far-field chain, by
  // default when the targets are the boundary points: there the far-field
  // kernels are small and latency-bound and leave most SMs idle (with volume
  // targets both chains are compute-bound); fmm_autotune may choose per pass
  const int oci = 3 * (tgt_set - 1) + (src_set - 1);
  const bool ov_pass = t->tuned_overlap[oci] >= 0 ? t->tuned_overlap[oci] != 0 : !(tgt_set & HFMM_SET_VOL);
  // volume targets of a regular lattice: the volume sources' near field as
  // dense blocks on the tensor cores, after L2P (adding into phis)
  const bool near_tc = !dipole && near_tc_usable(t, src_set, tgt_set, s);
  const bool overlap = !dipole && !near_tc && t->overlap_near && t->near_stream && t->phis_near && ov_pass;
  if (overlap) {
    d.near = reinterpret_cast<C<T>*>(t->phis_near);
    cudaStream_t sn = t->near_stream;
    HFMM_CUDA_TRY(cudaEventRecord(t->ev_fork, s));
    HFMM_CUDA_TRY(cudaStreamWaitEvent(sn, t->ev_fork, 0));
    tm.begin(HFMM_STAGE_P2P, sn);
    HFMM_TRY(p2p_stage<T, 0>(t, d, src_set, tgt_set, t->sigma_vol, t->sigma_bnd, sn));
    tm.end(1, sn, tm.on ? p2p_work(t, src_set, tgt_set) : 0.0);
    HFMM_CUDA_TRY(cudaEventRecord(t->ev_join, sn));
  }
  // P2M
  tm.begin(HFMM_STAGE_P2M, s);
  if (dipole)
    HFMM_TRY(launch_p2m_dipole<T>(t, d, d.M, s));
  else
    HFMM_TRY(launch_p2m<T>(t, d, d.M, src_set, mkc<T>(1, 0), s));
  tm.end(1, s);
  count_launches(1);
  // M2M, levels L-1 .. 2
  size_t sm8 = 8 * (size_t)P * sizeof(C<T>);
  HFMM_TRY(set_smem<T>((const void*)k_m2m<T>, sm8));
  if (L > 2) {
    tm.begin(HFMM_STAGE_M2M, s);
    for (int l = L - 1; l >= 2; --l)
      if (act_n(t, src_set, l))
      k_m2m<T><<<act_n(t, src_set, l), th, sm8, s>>>(d, l, t->level_off[l], t->level_off[l + 1], d.M, d.M,
                                              m2m + (int64_t)l * 8 * PP, src_set, 0, act_list(t, src_set, l));
    tm.end(L - 2, s);
    count_launches(L - 2);
  }
  // M2L, levels 2 .. L
  tm.begin(HFMM_STAGE_M2L, s);
  int nm2l = 0;
  HFMM_TRY(m2l_stage<T>(t, d, m2l, src_set, tgt_set, 0, s, &nm2l));
  tm.end(nm2l > 0 ? nm2l : 1, s, tm.on ? m2l_work(t, src_set, tgt_set) : 0.0);
  count_launches(nm2l);
  // L2L, levels 2 .. L-1 into their children
  size_t sm1 = (size_t)P * sizeof(C<T>);
  if (L > 2) {
    tm.begin(HFMM_STAGE_L2L, s);
    for (int l = 2; l < L; ++l)
      if (act_n(t, tgt_set, l + 1))
      k_l2l<T><<<act_n(t, tgt_set, l + 1), th, sm1, s>>>(d, t->level_off[l], t->level_off[l + 1], d.Lc, d.Lc,
                                                    l2l + (int64_t)l * 8 * PP, tgt_set, act_list(t, tgt_set, l + 1));
    tm.end(L - 2, s);
    count_launches(L - 2);
  }
  // L2P (adds the near field when it ran concurrently), else L2P then P2P (adds)
  if (overlap) HFMM_CUDA_TRY(cudaStreamWaitEvent(s, t->ev_join, 0));
  tm.begin(HFMM_STAGE_L2P, s);
  HFMM_TRY(launch_l2p<T>(t, d, tgt_set, mkc<T>(0, d.k), s));
  tm.end(1, s);
  if (!overlap) {
    tm.begin(HFMM_STAGE_P2P, s);
    int nl = 1;
    if (dipole) {
      HFMM_TRY(p2p_stage<T, 3>(t, d, src_set, tgt_set, t->sigma_vol, t->sigma_bnd, s));
    } else if (near_tc) {
      HFMM_TRY(near_tc_stage(t, s, &nl));
      count_launches(nl);
      if (src_set & HFMM_SET_BND) {
        HFMM_TRY(p2p_stage<T, 0>(t, d, HFMM_SET_BND, tgt_set, t->sigma_vol, t->sigma_bnd, s));
        ++nl;
      }
    } else {
      HFMM_TRY(p2p_stage<T, 0>(t, d, src_set, tgt_set, t->sigma_vol, t->sigma_bnd, s));
    }
    tm.end(nl, s, tm.on ? p2p_work(t, src_set, tgt_set) : 0.0);
  }
  count_launches(2);
  return hfmm_last_launch();
}

}  // namespace

int build_basis_table(fmm_tree* t, cudaStream_t s) {
  const size_t csz = t->precision == HFMM_FP32 ? sizeof(float2) : sizeof(double2);
  const size_t bytes = csz * (size_t)t->n_pts * (size_t)t->P;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return HFMM_OK;
  }
  if (bytes > fr / 4) return HFMM_OK;  // no table: P2M and L2P evaluate the basis at every apply
  HFMM_TRY(tree_alloc(t, &t->rtab, bytes));
  const int nleaf = 1 << (3 * t->L);
  if (t->precision == HFMM_FP32)
    k_basis_table<float><<<nleaf, 64, 0, s>>>(t->xyz, t->leaf_start, t->L, t->p, t->k,
                                              reinterpret_cast<float2*>(t->rtab));
  else
    k_basis_table<double><<<nleaf, 64, 0, s>>>(t->xyz, t->leaf_start, t->L, t->p, t->k,
                                               reinterpret_cast<double2*>(t->rtab));
  return hfmm_last_launch();
}

namespace {

// original-index range [o0, o1) of a set mask (volume ids, then boundary)
inline void set_range(const fmm_tree* t, int set, int64_t& o0, int64_t& o1) {
  o0 = (set & HFMM_SET_VOL) ? 0 : t->n_vol;
  o1 = (set & HFMM_SET_BND) ? t->n_pts : t->n_vol;
}

template <typename QB>
int gather_impl(fmm_tree* t, int src_set, const double2* q_vol, double scale_vol, const QB* q_bnd,
                double scale_bnd, cudaStream_t s) {
  int64_t o0, o1;
  set_range(t, src_set, o0, o1);
  t->timer.begin(HFMM_STAGE_GATHER, s);
  if (o1 > o0) {
    const unsigned g = ceil_div(o1 - o0, 256);
    if (t->precision == HFMM_FP32)
      k_gather<float, QB><<<g, 256, 0, s>>>(t->pos_of, o0, o1, t->n_vol, q_vol, scale_vol, q_bnd, scale_bnd,
                                            reinterpret_cast<float2*>(t->qs), t->skip);
    else
      k_gather<double, QB><<<g, 256, 0, s>>>(t->pos_of, o0, o1, t->n_vol, q_vol, scale_vol, q_bnd, scale_bnd,
                                             reinterpret_cast<double2*>(t->qs), t->skip);
  }
  t->timer.end(1, s);
  count_launches(1);
  return hfmm_last_launch();
}

template <typename OB>
int scatter_impl(fmm_tree* t, const void* sorted, int tgt_set, double2* phi_vol, OB* phi_bnd, cudaStream_t s) {
  int64_t o0, o1;
  set_range(t, tgt_set, o0, o1);
  t->timer.begin(HFMM_STAGE_GATHER, s);
  if (o1 > o0) {
    const unsigned g = ceil_div(o1 - o0, 256);
    if (t->precision == HFMM_FP32)
      k_scatter<float, OB><<<g, 256, 0, s>>>(t->pos_of, o0, o1, t->n_vol, reinterpret_cast<const float2*>(sorted),
                                             phi_vol, phi_bnd, t->skip);
    else
      k_scatter<double, OB><<<g, 256, 0, s>>>(t->pos_of, o0, o1, t->n_vol,
                                              reinterpret_cast<const double2*>(sorted), phi_vol, phi_bnd, t->skip);
  }
  t->timer.end(1, s);
  count_launches(1);
  return hfmm_last_launch();
}

}  // namespace

int fmm_gather(fmm_tree* t, int src_set, const double2* q_vol, double scale_vol, const double2* q_bnd,
               double scale_bnd, cudaStream_t s) {
  return gather_impl<double2>(t, src_set, q_vol, scale_vol, q_bnd, scale_bnd, s);
}

int fmm_gather(fmm_tree* t, int src_set, const double2* q_vol, double scale_vol, const float2* q_bnd,
               double scale_bnd, cudaStream_t s) {
  return gather_impl<float2>(t, src_set, q_vol, scale_vol, q_bnd, scale_bnd, s);
}

int fmm_device_error(cudaStream_t s, bool clear) {
  int h = 0;
  HFMM_CUDA_TRY(cudaMemcpyFromSymbolAsync(&h, g_fmm_error, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
  HFMM_CUDA_TRY(cudaStreamSynchronize(s));
  if (h && clear) {
    int z = 0;
    HFMM_CUDA_TRY(cudaMemcpyToSymbolAsync(g_fmm_error, &z, sizeof(int), 0, cudaMemcpyHostToDevice, s));
  }
  if (m2l_tc_error(s, clear)) h = HFMM_ERR_TIMEOUT;
  if (bnd_op_error(s, clear)) h = HFMM_ERR_TIMEOUT;
  return h;
}

int set_smem_any(const void* fn, size_t bytes) { return set_smem<float>(fn, bytes); }

int fmm_pair_lists(fmm_tree* t, int src_set, int tgt_set, cudaStream_t s) {
  const size_t csz = t->precision == HFMM_FP32 ? sizeof(float2) : sizeof(double2);
  return m2l_pair_lists(t, src_set, tgt_set, csz, s);
}

int fmm_core(fmm_tree* t, int src_set, int tgt_set, cudaStream_t s) {
  if (t->precision == HFMM_FP32) return core_impl<float>(t, src_set, tgt_set, s);
  return core_impl<double>(t, src_set, tgt_set, s);
}

int fmm_core_dlp(fmm_tree* t, int tgt_set, cudaStream_t s) {
  if (!t->lattice || !t->orig) return HFMM_ERR_UNSUPPORTED;
  if (t->precision == HFMM_FP32) return core_impl<float>(t, HFMM_SET_BND, tgt_set, s, true);
  return core_impl<double>(t, HFMM_SET_BND, tgt_set, s, true);
}

int fmm_core_adjoint(fmm_tree* t, int src_set, int tgt_set, cudaStream_t s) {
  if (t->precision == HFMM_FP32) return core_adjoint_impl<float>(t, src_set, tgt_set, s);
  return core_adjoint_impl<double>(t, src_set, tgt_set, s);
}

int fmm_core_dk(fmm_tree* t, int src_set, int tgt_set, cudaStream_t s) {
  if (t->precision == HFMM_FP32) return core_dk_impl<float>(t, src_set, tgt_set, s);
  return core_dk_impl<double>(t, src_set, tgt_set, s);
}

int fmm_scatter(fmm_tree* t, int tgt_set, double2* phi_vol, double2* phi_bnd, cudaStream_t s) {
  return scatter_impl<double2>(t, t->phis, tgt_set, phi_vol, phi_bnd, s);
}

int fmm_scatter(fmm_tree* t, int tgt_set, double2* phi_vol, float2* phi_bnd, cudaStream_t s) {
  return scatter_impl<float2>(t, t->phis, tgt_set, phi_vol, phi_bnd, s);
}

int fmm_scatter_from(fmm_tree* t, const void* sorted, int tgt_set, double2* phi_vol, double2* phi_bnd,
                     cudaStream_t s) {
  return scatter_impl<double2>(t, sorted, tgt_set, phi_vol, phi_bnd, s);
}
