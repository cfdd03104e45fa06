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

#include "special.cuh"
#include "tree.cuh"

namespace {

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
};

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
template <typename T>
__global__ void k_p2m(FmmDev<T> d, int64_t leaf_off, int src_set, int chunk) {
  extern __shared__ unsigned char smem_raw[];
  C<T>* basis = reinterpret_cast<C<T>*>(smem_raw);
  const int leaf = blockIdx.x;
  const int P = d.P;
  C<T>* M = d.M + (leaf_off + leaf) * P;
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
        regular_basis<T, true>(d.p, d.k, dx, dy, dz, d.qs[j], row);
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

// ---------------------------------------------------------------- M2M / L2L
// out[a'] (+)= sum_a T[a'][a] in[a]; thread per a' (a' = tid + s*blockDim)
template <typename T>
__device__ __forceinline__ C<T> matvec_row(const C<T>* Trow, const C<T>* x, int P) {
  C<T> acc = mkc<T>(0, 0);
  for (int a = 0; a < P; ++a) cfma<T>(acc, Trow[a], x[a]);
  return acc;
}

template <typename T>
__global__ void k_m2m(FmmDev<T> d, int level, int64_t off_par, int64_t off_child, const C<T>* ops,
                      int src_set) {
  extern __shared__ unsigned char smem_raw[];
  C<T>* xs = reinterpret_cast<C<T>*>(smem_raw);
  const int cell = blockIdx.x;
  const int P = d.P;
  C<T>* Mp = d.M + (off_par + cell) * P;
  if (!(d.flags[off_par + cell] & src_set)) {
    for (int a = threadIdx.x; a < P; a += blockDim.x) Mp[a] = mkc<T>(0, 0);
    return;
  }
  for (int e = threadIdx.x; e < 8 * P; e += blockDim.x) xs[e] = d.M[(off_child + 8 * (int64_t)cell) * P + e];
  __syncthreads();
  for (int ap = threadIdx.x; ap < P; ap += blockDim.x) {
    C<T> acc = mkc<T>(0, 0);
    for (int o = 0; o < 8; ++o) {
      const C<T>* Trow = ops + ((int64_t)o * P + ap) * P;
      C<T> v = matvec_row<T>(Trow, xs + o * P, P);
      acc = cadd<T>(acc, v);
    }
    Mp[ap] = acc;
  }
}

template <typename T>
__global__ void k_l2l(FmmDev<T> d, int64_t off_par, int64_t off_child, const C<T>* ops, int tgt_set) {
  extern __shared__ unsigned char smem_raw[];
  C<T>* xs = reinterpret_cast<C<T>*>(smem_raw);
  const int cell = blockIdx.x;  // child
  const int P = d.P;
  if (!(d.flags[off_child + cell] & tgt_set)) return;
  const int parent = cell >> 3, o = cell & 7;
  for (int e = threadIdx.x; e < P; e += blockDim.x) xs[e] = d.Lc[(off_par + parent) * P + e];
  __syncthreads();
  C<T>* Lch = d.Lc + (off_child + cell) * P;
  for (int ap = threadIdx.x; ap < P; ap += blockDim.x) {
    C<T> v = matvec_row<T>(ops + ((int64_t)o * P + ap) * P, xs, P);
    Lch[ap] = cadd<T>(Lch[ap], v);
  }
}

// ---------------------------------------------------------------- M2L
// one block per target cell of the level: L_T = sum over the cell's list of
// T_{slot} M_S, sources skipped when they hold no point of the source set
template <typename T>
__global__ void k_m2l(FmmDev<T> d, int level, int64_t off, const C<T>* ops, const int* m2l_off,
                      const int* m2l_slot, int m2l_count, int src_set, int tgt_set) {
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
      if (ap < P) acc[q] = cadd<T>(acc[q], matvec_row<T>(Top + (int64_t)ap * P, xs, P));
    }
  }
  for (int q = 0; q < 4; ++q) {
    int ap = threadIdx.x + q * blockDim.x;
    if (ap < P) d.Lc[(off + cell) * P + ap] = acc[q];
  }
}

// ---------------------------------------------------------------- L2P
template <typename T>
__global__ void k_l2p(FmmDev<T> d, int64_t leaf_off, int tgt_set) {
  extern __shared__ unsigned char smem_raw[];
  C<T>* Ls = reinterpret_cast<C<T>*>(smem_raw);
  const int leaf = blockIdx.x;
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
    // phi = i k acc
    d.phis[i] = mkc<T>(-d.k * acc.y, d.k * acc.x);
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
      d.phis[i] = cadd<T>(d.phis[i], tot);
    }
  }
}

// ---------------------------------------------------------------- gather / scatter

template <typename T>
__global__ void k_gather(const int64_t* orig, int64_t n_pts, int64_t n_vol, int src_set,
                         const double2* q_vol, double s_vol, const double2* q_bnd, double s_bnd,
                         C<T>* qs) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_pts) return;
  int64_t o = orig[i];
  double2 v = make_double2(0, 0);
  if (o < n_vol) {
    if (src_set & HFMM_SET_VOL) {
      double2 q = q_vol[o];
      v = make_double2(q.x * s_vol, q.y * s_vol);
    }
  } else if (src_set & HFMM_SET_BND) {
    double2 q = q_bnd[o - n_vol];
    v = make_double2(q.x * s_bnd, q.y * s_bnd);
  }
  qs[i] = mkc<T>(T(v.x), T(v.y));
}

template <typename T>
__global__ void k_scatter(const int64_t* pos_of, int64_t n_vol, int64_t n_bnd, int tgt_set,
                          const C<T>* phis, double2* phi_vol, double2* phi_bnd) {
  int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (o < n_vol) {
    if (tgt_set & HFMM_SET_VOL) {
      C<T> v = phis[pos_of[o]];
      phi_vol[o] = make_double2((double)v.x, (double)v.y);
    }
  } else if (o < n_vol + n_bnd) {
    if (tgt_set & HFMM_SET_BND) {
      C<T> v = phis[pos_of[o]];
      phi_bnd[o - n_vol] = make_double2((double)v.x, (double)v.y);
    }
  }
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
  return d;
}

int threads_for(int P) {
  int th = ((P + 31) / 32) * 32;
  if (th > 256) th = 256;
  if (th < 32) th = 32;
  return th;
}

template <typename T>
int set_smem(const void* fn, size_t bytes) {
  if (bytes > 48 * 1024)
    HFMM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return HFMM_OK;
}

template <typename T>
int core_impl(fmm_tree* t, int src_set, int tgt_set, cudaStream_t s) {
  FmmDev<T> d = make_dev<T>(t);
  const int P = t->P, L = t->L;
  const int nleaf = 1 << (3 * L);
  const C<T>* m2m = reinterpret_cast<const C<T>*>(sizeof(T) == 4 ? (void*)t->op_m2m32 : (void*)t->op_m2m);
  const C<T>* l2l = reinterpret_cast<const C<T>*>(sizeof(T) == 4 ? (void*)t->op_l2l32 : (void*)t->op_l2l);
  const C<T>* m2l = reinterpret_cast<const C<T>*>(sizeof(T) == 4 ? (void*)t->op_m2l32 : (void*)t->op_m2l);
  const int64_t PP = (int64_t)P * P;
  const int th = threads_for(P);

  // P2M
  const int chunk = 32;
  size_t sm_p2m = (size_t)chunk * P * sizeof(C<T>);
  HFMM_TRY(set_smem<T>((const void*)k_p2m<T>, sm_p2m));
  k_p2m<T><<<nleaf, 64, sm_p2m, s>>>(d, t->level_off[L], src_set, chunk);
  // M2M, levels L-1 .. 2
  size_t sm8 = 8 * (size_t)P * sizeof(C<T>);
  HFMM_TRY(set_smem<T>((const void*)k_m2m<T>, sm8));
  for (int l = L - 1; l >= 2; --l)
    k_m2m<T><<<1 << (3 * l), th, sm8, s>>>(d, l, t->level_off[l], t->level_off[l + 1],
                                            m2m + (int64_t)l * 8 * PP, src_set);
  // M2L, levels 2 .. L
  size_t sm1 = (size_t)P * sizeof(C<T>);
  for (int l = 2; l <= L; ++l)
    k_m2l<T><<<1 << (3 * l), th, sm1, s>>>(d, l, t->level_off[l], m2l + (int64_t)l * t->box_cells * PP,
                                            t->m2l_off, t->m2l_box_index, t->m2l_count, src_set,
                                            tgt_set);
  // L2L, levels 2 .. L-1 into their children
  for (int l = 2; l < L; ++l)
    k_l2l<T><<<1 << (3 * (l + 1)), th, sm1, s>>>(d, t->level_off[l], t->level_off[l + 1],
                                                  l2l + (int64_t)l * 8 * PP, tgt_set);
  // L2P then P2P (adds)
  k_l2p<T><<<nleaf, 64, sm1, s>>>(d, t->level_off[L], tgt_set);
  k_p2p<T><<<nleaf, 128, 0, s>>>(d, t->near_off, t->near_count, src_set, tgt_set, t->sigma_vol,
                                  t->sigma_bnd);
  return hfmm_last_launch();
}

}  // namespace

int fmm_gather(fmm_tree* t, int src_set, const double2* q_vol, double scale_vol, const double2* q_bnd,
               double scale_bnd, cudaStream_t s) {
  unsigned g = ceil_div(t->n_pts, 256);
  if (t->precision == HFMM_FP32)
    k_gather<float><<<g, 256, 0, s>>>(t->orig, t->n_pts, t->n_vol, src_set, q_vol, scale_vol, q_bnd,
                                      scale_bnd, reinterpret_cast<float2*>(t->qs));
  else
    k_gather<double><<<g, 256, 0, s>>>(t->orig, t->n_pts, t->n_vol, src_set, q_vol, scale_vol, q_bnd,
                                       scale_bnd, reinterpret_cast<double2*>(t->qs));
  return hfmm_last_launch();
}

int fmm_core(fmm_tree* t, int src_set, int tgt_set, cudaStream_t s) {
  if (t->precision == HFMM_FP32) return core_impl<float>(t, src_set, tgt_set, s);
  return core_impl<double>(t, src_set, tgt_set, s);
}

int fmm_scatter(fmm_tree* t, int tgt_set, double2* phi_vol, double2* phi_bnd, cudaStream_t s) {
  unsigned g = ceil_div(t->n_pts, 256);
  if (t->precision == HFMM_FP32)
    k_scatter<float><<<g, 256, 0, s>>>(t->pos_of, t->n_vol, t->n_bnd, tgt_set,
                                       reinterpret_cast<const float2*>(t->phis), phi_vol, phi_bnd);
  else
    k_scatter<double><<<g, 256, 0, s>>>(t->pos_of, t->n_vol, t->n_bnd, tgt_set,
                                        reinterpret_cast<const double2*>(t->phis), phi_vol, phi_bnd);
  return hfmm_last_launch();
}
