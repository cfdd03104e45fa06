// Krylov kernels: the 7-point Helmholtz operator (Sec. 2) and restarted
// (flexible) GMRES (Sec. 3-4) on device vectors.  The vectors are complex of
// the real type R (double: complex128; float: complex64, used for the inner
// solve of the FP32 form, where FP64 arithmetic would dominate: this GPU runs
// FP64 at a small fraction of its FP32 rate).  Dot products are summed per
// block in R and across blocks in FP64; the Hessenberg matrix, the Givens
// rotations and the least-squares solution are FP64 in both cases.
#include <algorithm>
#include <cmath>
#include <complex>

#include "krylov.cuh"
#include "tree.cuh"

namespace {

constexpr int RT = 128;      // threads of the reduction kernels
constexpr int RMAXB = 608;   // at most 4 reduction blocks per SM (152 SMs)
constexpr int KV = 8;        // vectors accumulated per pass over a block's elements
static_assert(RMAXB <= RE_DOT_PARTS, "re_dot_dev's scratch holds one partial per block");

static inline int red_blocks(int64_t N) {
  int64_t b = (N + RT - 1) / RT;
  return (int)(b < 1 ? 1 : (b > RMAXB ? RMAXB : b));
}

// (A u)_i = (6 u_i - sum of six neighbours)/h^2 - k^2 u_i, zero outside
__global__ void k_fdm(int n, double inv_h2, double k2, const double2* __restrict__ u,
                      double2* __restrict__ out) {
  int64_t N = (int64_t)n * n * n;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  int a = (int)(i % n), b = (int)((i / n) % n), c = (int)(i / ((int64_t)n * n));
  int64_t nn = (int64_t)n * n;
  double2 ui = u[i];
  double sx = 0, sy = 0;
  if (a > 0) { sx += u[i - 1].x; sy += u[i - 1].y; }
  if (a < n - 1) { sx += u[i + 1].x; sy += u[i + 1].y; }
  if (b > 0) { sx += u[i - n].x; sy += u[i - n].y; }
  if (b < n - 1) { sx += u[i + n].x; sy += u[i + n].y; }
  if (c > 0) { sx += u[i - nn].x; sy += u[i - nn].y; }
  if (c < n - 1) { sx += u[i + nn].x; sy += u[i + nn].y; }
  double d = 6.0 * inv_h2 - k2;
  out[i] = make_double2(d * ui.x - inv_h2 * sx, d * ui.y - inv_h2 * sy);
}

// Block sums of acc[0..nv) to partial[(i0 + q) * gridDim.x + blockIdx.x]
// (complex of real type R).
// FP64 arithmetic is scarce on this GPU, so the block sum uses few adds per
// thread: the 2 nv real columns go through shared memory, 16 threads sum a
// column's rows in 8 chunks, and the chunks are combined by one shuffle and
// one pass over the four warps.
template <typename R>
__device__ __forceinline__ void group_to_partials(C<R> (&acc)[KV], int nv, int i0, double2* partial) {
  static_assert(RT == 128 && KV == 8, "block layout assumes 128 threads and 16 real columns");
  __shared__ R red[RT][2 * KV + 1];
  __shared__ R wsum[RT / 32][2 * KV];
  const int tid = threadIdx.x;
#pragma unroll
  for (int q = 0; q < KV; ++q) {
    if (q < nv) {
      red[tid][2 * q] = acc[q].x;
      red[tid][2 * q + 1] = acc[q].y;
    }
  }
  __syncthreads();
  const int c = tid & 15, part = tid >> 4;
  R v = R(0);
  if (c < 2 * nv) {
#pragma unroll
    for (int k = 0; k < RT / 8; ++k) v += red[part + 8 * k][c];
  }
  v += __shfl_xor_sync(0xffffffffu, v, 16);
  if ((tid & 31) < 16) wsum[tid >> 5][c] = v;
  __syncthreads();
  if (tid < 2 * nv) {
    const R t = (wsum[0][tid] + wsum[1][tid]) + (wsum[2][tid] + wsum[3][tid]);
    reinterpret_cast<R*>(partial)[2 * ((int64_t)(i0 + (tid >> 1)) * gridDim.x + blockIdx.x) + (tid & 1)] = t;
  }
  __syncthreads();
}

// true in every thread of the block that finishes last; it resets the counter
__device__ __forceinline__ bool last_block(unsigned* counter) {
  __shared__ int is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned t = atomicAdd(counter, 1u);
    is_last = (t == gridDim.x - 1);
    if (is_last) *counter = 0u;
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last != 0;
}

// Hessenberg column j from the CGS2 coefficients, previous rotations, a new
// complex Givens rotation c = |a|/nu, s = (a/|a|) conj(b)/nu, update of g,
// residual estimate and breakdown flag; run by the whole block, the serial
// part by thread 0 on shared-memory copies, in the arithmetic of R.
// scal: [0] ||w|| before orthogonalisation, [1] h_{j+1,j}, [2] relres,
//       [3] breakdown, [4] ||b||
template <typename R>
__device__ void arnoldi_block(int j, int m, const double2* dots, double2* H, double* cs, double2* sn,
                              double2* g, double* scal, int* done, int* jdone, double rtol, R hnext,
                              C<R>* col, R* css, C<R>* sns) {
  const int ld = m + 1;
  for (int i = threadIdx.x; i <= j; i += blockDim.x)
    col[i] = mkc<R>(R(dots[i].x + dots[ld + i].x), R(dots[i].y + dots[ld + i].y));
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    css[i] = R(cs[i]);
    sns[i] = mkc<R>(R(sn[i].x), R(sn[i].y));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    col[j + 1] = mkc<R>(hnext, R(0));
    scal[1] = (double)hnext;
    scal[3] = ((double)hnext <= 1e-14 * scal[0]) ? 1.0 : 0.0;
    for (int i = 0; i < j; ++i) {
      const C<R> a = col[i], b = col[i + 1];
      const R c = css[i];
      const C<R> s = sns[i];
      // a' = c a + s b ; b' = -conj(s) a + c b
      col[i] = mkc<R>(c * a.x + s.x * b.x - s.y * b.y, c * a.y + s.x * b.y + s.y * b.x);
      col[i + 1] = mkc<R>(-(s.x * a.x + s.y * a.y) + c * b.x, -(s.x * a.y - s.y * a.x) + c * b.y);
    }
    const C<R> a = col[j], b = col[j + 1];
    const R aa = hypot(a.x, a.y);
    R c;
    C<R> s;
    if (aa == R(0)) {
      c = R(0);
      s = mkc<R>(R(1), R(0));
    } else {
      const R nu = sqrt(aa * aa + b.x * b.x + b.y * b.y);
      c = aa / nu;
      const C<R> ph = mkc<R>(a.x / aa, a.y / aa);  // a/|a|
      const C<R> cb = mkc<R>(b.x / nu, -b.y / nu);  // conj(b)/nu
      s = mkc<R>(ph.x * cb.x - ph.y * cb.y, ph.x * cb.y + ph.y * cb.x);
    }
    cs[j] = (double)c;
    sn[j] = make_double2((double)s.x, (double)s.y);
    col[j] = mkc<R>(c * a.x + s.x * b.x - s.y * b.y, c * a.y + s.x * b.y + s.y * b.x);
    col[j + 1] = mkc<R>(R(0), R(0));
    const C<R> gj = mkc<R>(R(g[j].x), R(g[j].y));
    const C<R> g1 = mkc<R>(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));
    g[j + 1] = make_double2((double)g1.x, (double)g1.y);
    g[j] = make_double2((double)(c * gj.x), (double)(c * gj.y));
    scal[2] = (double)hypot(g1.x, g1.y) / scal[4];
    if (jdone) *jdone = j + 1;
    if (done && (scal[2] < rtol || scal[3] != 0.0 || !(scal[2] == scal[2]))) *done = 1;
  }
  __syncthreads();
  double2* Hc = H + (int64_t)j * ld;
  for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) Hc[i] = make_double2((double)col[i].x, (double)col[i].y);
}

// One pass of classical Gram-Schmidt over the block's share of w, with the
// final reduction in the last block to finish (no second launch):
//   MODE 0: dots[i] = <V_i, w> (i < nvec); nrm = ||w|| when nrm != null
//   MODE 1: w -= sum_i coef[i] V_i, then dots[i] = <V_i, w>
//   MODE 2: w -= sum_i coef[i] V_i, then h = ||w||, and the Arnoldi update of
//           column j (arnoldi_block) in the last block
// <a, b> = sum conj(a) b.  Partial sums are combined in block order, so the
// result does not depend on the order in which blocks finish.
template <int MODE, typename R>
__global__ void __launch_bounds__(RT) k_cgs(const C<R>* __restrict__ V, int64_t ld, int nvec,
                                            const double2* __restrict__ coef, C<R>* w, int64_t N,
                                            double2* partial, unsigned* counter, double2* dots, double* nrm,
                                            const int* skip, int j, int m, const double2* adots, double2* H,
                                            double* cs, double2* sn, double2* g, double* scal, int* done,
                                            int* jdone, double rtol) {
  extern __shared__ double2 dyn[];
  if (skip && *skip) return;
  const int64_t stride = (int64_t)gridDim.x * RT;
  const int64_t e0 = blockIdx.x * (int64_t)RT + threadIdx.x;
  if (MODE >= 1) {
    C<R>* cf = reinterpret_cast<C<R>*>(dyn);  // nvec coefficients
    for (int i = threadIdx.x; i < nvec; i += RT) cf[i] = mkc<R>(R(coef[i].x), R(coef[i].y));
    __syncthreads();
    for (int64_t e = e0; e < N; e += stride) {
      C<R> acc = w[e];
      for (int i = 0; i < nvec; ++i) {
        const C<R> c = cf[i], v = V[(int64_t)i * ld + e];
        acc.x -= c.x * v.x - c.y * v.y;
        acc.y -= c.x * v.y + c.y * v.x;
      }
      w[e] = acc;
    }
  }
  int nrow = 0;
  if (MODE <= 1) {
    for (int i0 = 0; i0 < nvec; i0 += KV) {
      const int nv = min(KV, nvec - i0);
      C<R> acc[KV];
#pragma unroll
      for (int q = 0; q < KV; ++q) acc[q] = mkc<R>(0, 0);
      for (int64_t e = e0; e < N; e += stride) {
        const C<R> b = w[e];
#pragma unroll
        for (int q = 0; q < KV; ++q) {
          if (q < nv) {
            const C<R> a = V[(int64_t)(i0 + q) * ld + e];
            acc[q].x += a.x * b.x + a.y * b.y;
            acc[q].y += a.x * b.y - a.y * b.x;
          }
        }
      }
      group_to_partials<R>(acc, nv, i0, partial);
    }
    nrow = nvec;
  }
  const bool want_norm = (MODE == 2) || nrm != nullptr;
  if (want_norm) {
    C<R> acc[KV];
#pragma unroll
    for (int q = 0; q < KV; ++q) acc[q] = mkc<R>(0, 0);
    for (int64_t e = e0; e < N; e += stride) {
      const C<R> b = w[e];
      acc[0].x += b.x * b.x + b.y * b.y;
    }
    group_to_partials<R>(acc, 1, nrow, partial);
  }
  if (!last_block(counter)) return;
  __shared__ R sums_norm;
  const int rows = nrow + (want_norm ? 1 : 0);
  // rows 0..nrow-1 go to dots, the norm row to shared memory; each warp
  // sums four rows at a time so that their loads are in flight together
  {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nb = gridDim.x;
    const C<R>* pr = reinterpret_cast<const C<R>*>(partial);
    for (int i0 = 4 * wid; i0 < rows; i0 += 4 * (RT / 32)) {
      R x[4] = {0, 0, 0, 0}, y[4] = {0, 0, 0, 0};
#pragma unroll 3
      for (int b = lane; b < nb; b += 32) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          if (i0 + r < rows) {
            const C<R> v = __ldcg(&pr[(int64_t)(i0 + r) * nb + b]);
            x[r] += v.x;
            y[r] += v.y;
          }
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        for (int o = 16; o > 0; o >>= 1) {
          x[r] += __shfl_xor_sync(0xffffffffu, x[r], o);
          y[r] += __shfl_xor_sync(0xffffffffu, y[r], o);
        }
        const int i = i0 + r;
        if (lane == 0 && i < rows) {
          if (i < nrow)
            dots[i] = make_double2((double)x[r], (double)y[r]);
          else
            sums_norm = sqrt(x[r]);
        }
      }
    }
  }
  __syncthreads();
  if (MODE == 2) {
    C<R>* col = reinterpret_cast<C<R>*>(dyn);  // j + 2
    C<R>* sns = col + (j + 2);
    R* css = reinterpret_cast<R*>(sns + j);
    arnoldi_block<R>(j, m, adots, H, cs, sn, g, scal, done, jdone, rtol, sums_norm, col, css, sns);
  } else if (want_norm && threadIdx.x == 0) {
    *nrm = (double)sums_norm;
  }
}

// w += sign * sum_i coef[i] V_i (coefficients staged in shared memory in R)
template <typename R>
__global__ void k_axpy_multi(const C<R>* __restrict__ V, int64_t ld, int nvec, const double2* __restrict__ coef,
                             double sign, C<R>* w, int64_t N, const int* skip, const int* nvec_dev) {
  extern __shared__ double2 dyn[];
  if (skip && *skip) return;
  if (nvec_dev) nvec = *nvec_dev;
  C<R>* cf = reinterpret_cast<C<R>*>(dyn);
  for (int i = threadIdx.x; i < nvec; i += blockDim.x)
    cf[i] = mkc<R>(R(sign * coef[i].x), R(sign * coef[i].y));
  __syncthreads();
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= N) return;
  C<R> acc = w[e];
  for (int i = 0; i < nvec; ++i) {
    const C<R> c = cf[i], v = V[(int64_t)i * ld + e];
    acc.x += c.x * v.x - c.y * v.y;
    acc.y += c.x * v.y + c.y * v.x;
  }
  w[e] = acc;
}

template <typename R>
__global__ void k_sub(const C<R>* a, const C<R>* b, C<R>* out, int64_t N) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < N) out[e] = mkc<R>(a[e].x - b[e].x, a[e].y - b[e].y);
}

// dst = src / *nrm (no-op when the norm is zero); one reciprocal per thread
template <typename R>
__global__ void k_scale_by(const C<R>* src, const double* nrm, C<R>* dst, int64_t N, const int* skip) {
  if (skip && *skip) return;
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const double d = *nrm;
  if (e < N && d > 0) {
    const R r = R(1.0 / d);
    dst[e] = mkc<R>(src[e].x * r, src[e].y * r);
  }
}

// start of a cycle: g = (beta, 0, ...)
__global__ void k_cycle_init(int m, const double* beta, double2* g) {
  for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = make_double2(i == 0 ? *beta : 0.0, 0.0);
}

// y = H(0:k,0:k)^-1 g(0:k), upper triangular, column by column: after y_i
// is known, every row q < i drops H(q,i) y_i (one thread per row).  Columns
// are staged in shared memory up front when the triangle is small (BS_MAX).
constexpr int BS_MAX = 40;
template <typename R>
__global__ void k_backsolve(int kdim, int m, const double2* H, const double2* g, double2* y, const int* kdim_dev) {
  __shared__ C<R> acc[BS_MAX];
  __shared__ C<R> Hs[BS_MAX * BS_MAX];
  __shared__ C<R> yi_s;
  extern __shared__ double2 dynb[];  // kdim accumulators, when kdim > BS_MAX
  if (kdim_dev) kdim = *kdim_dev;
  const int ld = m + 1;
  const bool small = kdim <= BS_MAX;
  C<R>* a = small ? acc : reinterpret_cast<C<R>*>(dynb);
  for (int q = threadIdx.x; q < kdim; q += blockDim.x) a[q] = mkc<R>(R(g[q].x), R(g[q].y));
  if (small)
    for (int e = threadIdx.x; e < kdim * kdim; e += blockDim.x) {
      const int c = e / kdim, r = e % kdim;
      const double2 h = r <= c ? H[(int64_t)c * ld + r] : make_double2(0.0, 0.0);
      Hs[e] = mkc<R>(R(h.x), R(h.y));
    }
  __syncthreads();
  for (int i = kdim - 1; i >= 0; --i) {
    if (threadIdx.x == 0) {
      const C<R> v0 = a[i];
      const double2 dd = small ? make_double2(0.0, 0.0) : H[(int64_t)i * ld + i];
      const C<R> d = small ? Hs[(int64_t)i * kdim + i] : mkc<R>(R(dd.x), R(dd.y));
      const R inv = R(1) / (d.x * d.x + d.y * d.y);
      const C<R> v = mkc<R>((v0.x * d.x + v0.y * d.y) * inv, (v0.y * d.x - v0.x * d.y) * inv);
      y[i] = make_double2((double)v.x, (double)v.y);
      yi_s = v;
    }
    __syncthreads();
    const C<R> v = yi_s;
    for (int q = threadIdx.x; q < i; q += blockDim.x) {
      C<R> h;
      if (small) {
        h = Hs[(int64_t)i * kdim + q];
      } else {
        const double2 hd = H[(int64_t)i * ld + q];
        h = mkc<R>(R(hd.x), R(hd.y));
      }
      a[q].x -= h.x * v.x - h.y * v.y;
      a[q].y -= h.x * v.y + h.y * v.x;
    }
    __syncthreads();
  }
}

}  // namespace

int fdm_apply_dev(int n, double h, double k, const double2* u, double2* out, cudaStream_t s) {
  int64_t N = (int64_t)n * n * n;
  k_fdm<<<ceil_div(N, 256), 256, 0, s>>>(n, 1.0 / (h * h), k * k, u, out);
  count_launches(1);
  return hfmm_last_launch();
}

template <typename R>
int gmres_work_reserve(GmresWorkT<R>& W, int64_t N, int m, bool flexible) {
  if (W.base && W.N == N && W.m >= m && (W.flexible || !flexible)) return HFMM_OK;
  gmres_work_free(W);
  W.N = N;
  W.m = m;
  W.flexible = flexible;
  const size_t esz = sizeof(C<R>);
  size_t nv = (size_t)(m + 1) + (flexible ? m : 0) + 2;
  size_t bytes = nv * N * esz;
  bytes += (size_t)RMAXB * (m + 2) * sizeof(double2) + 256;  // partials, block counter
  bytes += (2 * (m + 1) + (m + 1) * m + m + m + 1 + m) * sizeof(double2) + m * sizeof(double) +
           32 * sizeof(double) + 4096;
  if (cudaMalloc(&W.base, bytes) != cudaSuccess) {
    W.base = nullptr;
    return HFMM_ERR_NOMEM;
  }
  if (cudaMallocHost((void**)&W.host, 32 * sizeof(double)) != cudaSuccess) {
    cudaFree(W.base);
    W.base = nullptr;
    return HFMM_ERR_NOMEM;
  }
  W.bytes = bytes;
  char* p = (char*)W.base;
  auto take = [&](size_t b) {
    char* q = p;
    p += (b + 255) / 256 * 256;
    return (void*)q;
  };
  W.V = (C<R>*)take((size_t)(m + 1) * N * esz);
  W.Z = flexible ? (C<R>*)take((size_t)m * N * esz) : nullptr;
  W.w = (C<R>*)take(N * esz);
  W.r = (C<R>*)take(N * esz);
  W.partial = (double*)take((size_t)RMAXB * (m + 2) * sizeof(double2));
  W.counter = (unsigned*)take(256);
  if (cudaMemset(W.counter, 0, 256) != cudaSuccess) {
    gmres_work_free(W);
    return HFMM_ERR_CUDA;
  }
  W.dots = (double2*)take(2 * (m + 1) * sizeof(double2));
  W.H = (double2*)take((size_t)(m + 1) * m * sizeof(double2));
  W.cs = (double*)take(m * sizeof(double));
  W.sn = (double2*)take(m * sizeof(double2));
  W.g = (double2*)take((m + 1) * sizeof(double2));
  W.y = (double2*)take(m * sizeof(double2));
  W.scal = (double*)take(32 * sizeof(double));
  return HFMM_OK;
}

template <typename R>
void gmres_work_free(GmresWorkT<R>& W) {
  if (W.base) cudaFree(W.base);
  if (W.host) cudaFreeHost(W.host);
  W = GmresWorkT<R>();
}

namespace {

// out = scale Re sum_i conj(a_i) b_i in FP64: each thread sums its strided
// elements in index order, each block folds its threads in a fixed tree and
// writes one partial; k_re_dot_final adds the partials in block order, so
// the result does not depend on the order in which blocks run
__global__ void __launch_bounds__(RT) k_re_dot_part(const double2* __restrict__ a, const double2* __restrict__ b,
                                                    int64_t N, double* __restrict__ part) {
  __shared__ double sh[RT / 32];
  const int64_t stride = (int64_t)gridDim.x * RT;
  double acc = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)RT + threadIdx.x; e < N; e += stride) {
    const double2 x = a[e], y = b[e];
    acc = fma(x.x, y.x, acc);
    acc = fma(x.y, y.y, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < RT / 32; ++w) s += sh[w];
    part[blockIdx.x] = s;
  }
}

__global__ void __launch_bounds__(32) k_re_dot_final(const double* __restrict__ part, int nb, double scale,
                                                     double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < nb; i += 32) acc += part[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (threadIdx.x == 0) *out = scale * acc;
}

}  // namespace

int re_dot_dev(const double2* a, const double2* b, int64_t N, double scale, double* part, double* out,
               cudaStream_t s) {
  const int nb = red_blocks(N);
  k_re_dot_part<<<nb, RT, 0, s>>>(a, b, N, part);
  k_re_dot_final<<<1, 32, 0, s>>>(part, nb, scale, out);
  count_launches(2);
  return hfmm_last_launch();
}

template <typename R>
int dev_norm(GmresWorkT<R>& W, const C<R>* x, int64_t N, double* out_dev, cudaStream_t s) {
  k_cgs<0, R><<<red_blocks(N), RT, 0, s>>>(nullptr, 0, 0, nullptr, const_cast<C<R>*>(x), N, (double2*)W.partial,
                                           W.counter, nullptr, out_dev, W.skip, 0, 0, nullptr, nullptr, nullptr,
                                           nullptr, nullptr, nullptr, nullptr, nullptr, 0.0);
  count_launches(1);
  return hfmm_last_launch();
}

namespace {

// Classical Gram-Schmidt applied twice to W.w against V_0..V_j, then the
// Arnoldi update of Hessenberg column j (three launches).  skip: kernels
// return at once when set; done/jdone/rtol: convergence flags of the device-
// driven form (null on the host-driven path).
template <typename R>
int cgs2_step(GmresWorkT<R>& W, int j, int m, const int* skip, int* done, int* jdone, double rtol, cudaStream_t s) {
  const int64_t N = W.N;
  const int nb = red_blocks(N);
  const int nvec = j + 1;
  double2* P = (double2*)W.partial;
  double2* d1 = W.dots;
  double2* d2 = W.dots + (m + 1);
  k_cgs<0, R><<<nb, RT, 0, s>>>(W.V, N, nvec, nullptr, W.w, N, P, W.counter, d1, W.scal + 0, skip, 0, 0, nullptr,
                                nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0.0);
  k_cgs<1, R><<<nb, RT, nvec * sizeof(double2), s>>>(W.V, N, nvec, d1, W.w, N, P, W.counter, d2, nullptr, skip, 0,
                                                     0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                     nullptr, nullptr, 0.0);
  const size_t sh3 = std::max<size_t>(nvec * sizeof(double2),
                                      (size_t)(2 * j + 2) * sizeof(double2) + (size_t)j * sizeof(double));
  k_cgs<2, R><<<nb, RT, sh3, s>>>(W.V, N, nvec, d2, W.w, N, P, W.counter, nullptr, nullptr, skip, j, m, W.dots,
                                  W.H, W.cs, W.sn, W.g, W.scal, done, jdone, rtol);
  count_launches(3);
  return hfmm_last_launch();
}

// start of a device-driven cycle: beta = ||b|| (x0 = 0), g = (beta, 0...),
// done = 1 when b is zero or not finite, jdone = 0
__global__ void k_cycle_start(int m, double* scal, double2* g, int* done, int* jdone) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double beta = scal[5];
  scal[4] = beta;
  for (int i = 0; i <= m; ++i) g[i] = make_double2(i == 0 ? beta : 0.0, 0.0);
  *done = (beta > 0.0 && beta < 1e300) ? 0 : 1;
  *jdone = 0;
}

__global__ void k_count_add(const int* jdone, int* total) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *total += *jdone;
}

}  // namespace

template <typename R>
int gmres_run(GmresWorkT<R>& W, const DevOpT<R>& A, const DevOpT<R>* M, const C<R>* b, C<R>* x, int m,
              double rtol, int maxit, bool x0_zero, bool true_residual, GmresResult* res,
              double* history, int history_len, cudaStream_t s) {
  const int64_t N = W.N;
  const size_t esz = sizeof(C<R>);
  const unsigned gN = ceil_div(N, 256);
  const size_t shc = (size_t)m * sizeof(double2);  // staged coefficients of k_axpy_multi
  GmresResult Res;
  HFMM_TRY(dev_norm<R>(W, b, N, W.scal + 4, s));
  HFMM_CUDA_TRY(cudaMemcpyAsync(W.host, W.scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
  HFMM_CUDA_TRY(cudaStreamSynchronize(s));
  const double bnorm = W.host[4];
  if (!std::isfinite(bnorm)) return HFMM_ERR_NONFINITE;
  if (bnorm == 0.0) {
    HFMM_CUDA_TRY(cudaMemsetAsync(x, 0, N * esz, s));
    Res.converged = 1;
    if (res) *res = Res;
    return HFMM_OK;
  }
  double relres = 1.0;
  bool stop = false;
  while (true) {
    // r = b - A x, beta = ||r||
    if (x0_zero && Res.iters == 0) {
      HFMM_CUDA_TRY(cudaMemcpyAsync(W.r, b, N * esz, cudaMemcpyDeviceToDevice, s));
    } else {
      HFMM_TRY(A(x, W.w));
      k_sub<R><<<gN, 256, 0, s>>>(b, W.w, W.r, N);
      count_launches(1);
    }
    HFMM_TRY(dev_norm<R>(W, W.r, N, W.scal + 5, s));
    HFMM_CUDA_TRY(cudaMemcpyAsync(W.host, W.scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
    HFMM_CUDA_TRY(cudaStreamSynchronize(s));
    relres = W.host[5] / bnorm;
    if (!std::isfinite(relres)) return HFMM_ERR_NONFINITE;
    if (relres < rtol) {
      Res.converged = 1;
      break;
    }
    if (Res.iters >= maxit) break;
    k_cycle_init<<<1, 64, 0, s>>>(m, W.scal + 5, W.g);
    k_scale_by<R><<<gN, 256, 0, s>>>(W.r, W.scal + 5, W.V, N, nullptr);
    count_launches(2);
    int jdone = 0;
    for (int j = 0; j < m; ++j) {
      C<R>* vj = W.V + (int64_t)j * N;
      C<R>* zj = vj;
      if (M) {
        zj = W.Z + (int64_t)j * N;
        HFMM_TRY((*M)(vj, zj));
      }
      HFMM_TRY(A(zj, W.w));
      HFMM_TRY(cgs2_step<R>(W, j, m, nullptr, nullptr, nullptr, 0.0, s));
      if (j + 1 < m) {
        k_scale_by<R><<<gN, 256, 0, s>>>(W.w, W.scal + 1, W.V + (int64_t)(j + 1) * N, N, nullptr);
        count_launches(1);
      }
      HFMM_TRY(hfmm_last_launch());
      HFMM_CUDA_TRY(cudaMemcpyAsync(W.host, W.scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
      HFMM_CUDA_TRY(cudaStreamSynchronize(s));
      relres = W.host[2];
      if (history && Res.iters < history_len) history[Res.iters] = relres;
      Res.iters++;
      jdone = j + 1;
      if (!std::isfinite(relres)) return HFMM_ERR_NONFINITE;
      bool breakdown = W.host[3] != 0.0;
      if (relres < rtol || breakdown || Res.iters >= maxit) {
        stop = true;
        if (relres < rtol || breakdown) Res.converged = 1;
        break;
      }
    }
    k_backsolve<R><<<1, 128, (size_t)m * sizeof(double2), s>>>(jdone, m, W.H, W.g, W.y, nullptr);
    k_axpy_multi<R><<<gN, 256, shc, s>>>(M ? W.Z : W.V, N, jdone, W.y, 1.0, x, N, nullptr, nullptr);
    count_launches(2);
    HFMM_TRY(hfmm_last_launch());
    if (stop) break;
    Res.restarts++;
  }
  Res.relres_est = relres;
  if (!true_residual) {
    Res.relres_true = -1.0;
    if (res) *res = Res;
    return HFMM_OK;
  }
  // true residual
  HFMM_TRY(A(x, W.w));
  k_sub<R><<<gN, 256, 0, s>>>(b, W.w, W.r, N);
  count_launches(1);
  HFMM_TRY(dev_norm<R>(W, W.r, N, W.scal + 6, s));
  HFMM_CUDA_TRY(cudaMemcpyAsync(W.host, W.scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
  HFMM_CUDA_TRY(cudaStreamSynchronize(s));
  Res.relres_true = W.host[6] / bnorm;
  if (res) *res = Res;
  return HFMM_OK;
}

// ---------------------------------------------------------------- graph form

template <typename R>
int gmres_cycle_device(GmresWorkT<R>& W, const DevOpT<R>& A, const C<R>* b, C<R>* x, int m, double rtol,
                       int* d_done, int* d_jdone, int* d_total, cudaStream_t s) {
  const int64_t N = W.N;
  const unsigned gN = ceil_div(N, 256);
  if (W.m < m) return HFMM_ERR_INVALID_ARG;
  HFMM_CUDA_TRY(cudaMemsetAsync(x, 0, N * sizeof(C<R>), s));
  W.skip = nullptr;
  HFMM_TRY(dev_norm<R>(W, b, N, W.scal + 5, s));
  k_cycle_start<<<1, 1, 0, s>>>(m, W.scal, W.g, d_done, d_jdone);
  W.skip = d_done;
  k_scale_by<R><<<gN, 256, 0, s>>>(b, W.scal + 5, W.V, N, d_done);
  count_launches(2);
  for (int j = 0; j < m; ++j) {
    C<R>* vj = W.V + (int64_t)j * N;
    HFMM_TRY(A(vj, W.w));
    HFMM_TRY(cgs2_step<R>(W, j, m, d_done, d_done, d_jdone, rtol, s));
    if (j + 1 < m) {
      k_scale_by<R><<<gN, 256, 0, s>>>(W.w, W.scal + 1, W.V + (int64_t)(j + 1) * N, N, d_done);
      count_launches(1);
    }
  }
  W.skip = nullptr;
  k_backsolve<R><<<1, 128, (size_t)m * sizeof(double2), s>>>(0, m, W.H, W.g, W.y, d_jdone);
  k_axpy_multi<R><<<gN, 256, (size_t)m * sizeof(double2), s>>>(W.V, N, 0, W.y, 1.0, x, N, nullptr, d_jdone);
  k_count_add<<<1, 1, 0, s>>>(d_jdone, d_total);
  count_launches(3);
  return hfmm_last_launch();
}

// ---------------------------------------------------------------- BiCGSTAB

namespace {

// p = r + beta (p - omega v)
__global__ void k_bicg_p(double2* __restrict__ p, const double2* __restrict__ r, const double2* __restrict__ v,
                         double2 beta, double2 omega, int64_t N) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= N) return;
  const double2 pe = p[e], ve = v[e], re = r[e];
  const double2 d = make_double2(pe.x - (omega.x * ve.x - omega.y * ve.y), pe.y - (omega.x * ve.y + omega.y * ve.x));
  p[e] = make_double2(re.x + beta.x * d.x - beta.y * d.y, re.y + beta.x * d.y + beta.y * d.x);
}

// out = a - c b
__global__ void k_bicg_sub(double2* __restrict__ out, const double2* __restrict__ a, const double2* __restrict__ b,
                           double2 c, int64_t N) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= N) return;
  const double2 ae = a[e], be = b[e];
  out[e] = make_double2(ae.x - (c.x * be.x - c.y * be.y), ae.y - (c.x * be.y + c.y * be.x));
}

// x += alpha phat + omega shat; r = s - omega t (r may be null: x only)
__global__ void k_bicg_x(double2* __restrict__ x, double2* __restrict__ r, const double2* __restrict__ phat,
                         const double2* __restrict__ shat, const double2* __restrict__ sv,
                         const double2* __restrict__ t, double2 alpha, double2 omega, int64_t N) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= N) return;
  const double2 ph = phat[e];
  double2 xe = x[e];
  xe.x += alpha.x * ph.x - alpha.y * ph.y;
  xe.y += alpha.x * ph.y + alpha.y * ph.x;
  if (shat) {
    const double2 sh = shat[e];
    xe.x += omega.x * sh.x - omega.y * sh.y;
    xe.y += omega.x * sh.y + omega.y * sh.x;
  }
  x[e] = xe;
  if (r) {
    const double2 se = sv[e], te = t[e];
    r[e] = make_double2(se.x - (omega.x * te.x - omega.y * te.y), se.y - (omega.x * te.y + omega.y * te.x));
  }
}

}  // namespace

int bicg_work_reserve(BicgWork& W, int64_t N) {
  if (W.base && W.N == N) return HFMM_OK;
  bicg_work_free(W);
  W.N = N;
  const size_t vec = (size_t)N * sizeof(double2);
  const size_t vb = (vec + 255) / 256 * 256;
  const size_t bytes = 8 * vb + (size_t)RMAXB * 4 * sizeof(double2) + 256 + 4 * 256;
  if (cudaMalloc(&W.base, bytes) != cudaSuccess) {
    W.base = nullptr;
    return HFMM_ERR_NOMEM;
  }
  if (cudaMallocHost((void**)&W.host, 8 * sizeof(double)) != cudaSuccess) {
    cudaFree(W.base);
    W.base = nullptr;
    return HFMM_ERR_NOMEM;
  }
  char* q = (char*)W.base;
  double2** vecs[8] = {&W.r, &W.rhat, &W.p, &W.v, &W.s, &W.t, &W.phat, &W.shat};
  for (int i = 0; i < 8; ++i) {
    *vecs[i] = (double2*)q;
    q += vb;
  }
  W.partial = (double2*)q;
  q += (size_t)RMAXB * 4 * sizeof(double2);
  W.counter = (unsigned*)q;
  q += 256;
  W.dots = (double2*)q;  // [0] dot, [1] norm in .x
  if (cudaMemset(W.counter, 0, 256) != cudaSuccess) {
    bicg_work_free(W);
    return HFMM_ERR_CUDA;
  }
  return HFMM_OK;
}

void bicg_work_free(BicgWork& W) {
  if (W.base) cudaFree(W.base);
  if (W.host) cudaFreeHost(W.host);
  W = BicgWork();
}

// <a, b> = sum conj(a) b and, when want_norm, ||b||; read back to the host
static int bicg_dot(BicgWork& W, const double2* a, const double2* b, bool want_norm, std::complex<double>* dot,
                    double* nrm, cudaStream_t s) {
  const int64_t N = W.N;
  k_cgs<0, double><<<red_blocks(N), RT, 0, s>>>(a, N, a ? 1 : 0, nullptr, const_cast<double2*>(b), N, W.partial,
                                                W.counter, W.dots, want_norm ? (double*)(W.dots + 1) : nullptr,
                                                nullptr, 0, 0, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                nullptr, nullptr, nullptr, 0.0);
  count_launches(1);
  HFMM_TRY(hfmm_last_launch());
  HFMM_CUDA_TRY(cudaMemcpyAsync(W.host, W.dots, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  HFMM_CUDA_TRY(cudaStreamSynchronize(s));
  if (dot) *dot = std::complex<double>(W.host[0], W.host[1]);
  if (nrm) *nrm = W.host[2];
  return HFMM_OK;
}

static inline double2 d2(std::complex<double> z) { return make_double2(z.real(), z.imag()); }

int bicgstab_run(BicgWork& W, const DevOp& A, const DevOp* M, const double2* b, double2* x, double rtol, int maxit,
                 bool x0_zero, BicgResult* res, double* history, int history_len, cudaStream_t s) {
  using cd = std::complex<double>;
  const int64_t N = W.N;
  const unsigned gN = ceil_div(N, 256);
  BicgResult R;
  double bnorm = 0.0;
  HFMM_TRY(bicg_dot(W, nullptr, b, true, nullptr, &bnorm, s));
  if (!std::isfinite(bnorm)) return HFMM_ERR_NONFINITE;
  if (bnorm == 0.0) {
    HFMM_CUDA_TRY(cudaMemsetAsync(x, 0, N * sizeof(double2), s));
    R.converged = 1;
    if (res) *res = R;
    return HFMM_OK;
  }
  if (x0_zero) {
    HFMM_CUDA_TRY(cudaMemcpyAsync(W.r, b, N * sizeof(double2), cudaMemcpyDeviceToDevice, s));
  } else {
    HFMM_TRY(A(x, W.v));
    k_bicg_sub<<<gN, 256, 0, s>>>(W.r, b, W.v, make_double2(1.0, 0.0), N);
    count_launches(1);
  }
  double rn = 0.0;
  HFMM_TRY(bicg_dot(W, nullptr, W.r, true, nullptr, &rn, s));
  double relres = rn / bnorm;
  if (relres < rtol) R.converged = 1;
  HFMM_CUDA_TRY(cudaMemcpyAsync(W.rhat, W.r, N * sizeof(double2), cudaMemcpyDeviceToDevice, s));
  HFMM_CUDA_TRY(cudaMemsetAsync(W.p, 0, N * sizeof(double2), s));
  HFMM_CUDA_TRY(cudaMemsetAsync(W.v, 0, N * sizeof(double2), s));
  cd rho_old(1.0, 0.0), alpha(1.0, 0.0), omega(1.0, 0.0);
  for (int it = 1; it <= maxit && !R.converged && !R.breakdown; ++it) {
    R.iters = it;
    cd rho;
    HFMM_TRY(bicg_dot(W, W.rhat, W.r, false, &rho, nullptr, s));
    if (rho == cd(0.0, 0.0)) {
      R.breakdown = 1;
      break;
    }
    const cd beta = it == 1 ? cd(0.0, 0.0) : (rho / rho_old) * (alpha / omega);
    k_bicg_p<<<gN, 256, 0, s>>>(W.p, W.r, W.v, d2(beta), d2(it == 1 ? cd(0.0, 0.0) : omega), N);
    count_launches(1);
    const double2* ph = W.p;
    if (M) {
      HFMM_TRY((*M)(W.p, W.phat));
      ph = W.phat;
      R.precond_applies++;
    }
    HFMM_TRY(A(ph, W.v));
    cd rv;
    HFMM_TRY(bicg_dot(W, W.rhat, W.v, false, &rv, nullptr, s));
    alpha = rho / rv;
    k_bicg_sub<<<gN, 256, 0, s>>>(W.s, W.r, W.v, d2(alpha), N);
    count_launches(1);
    double sn = 0.0;
    HFMM_TRY(bicg_dot(W, nullptr, W.s, true, nullptr, &sn, s));
    if (!std::isfinite(sn)) return HFMM_ERR_NONFINITE;
    if (sn / bnorm < rtol) {  // half step
      k_bicg_x<<<gN, 256, 0, s>>>(x, nullptr, ph, nullptr, nullptr, nullptr, d2(alpha), make_double2(0, 0), N);
      count_launches(1);
      relres = sn / bnorm;
      if (history && it - 1 < history_len) history[it - 1] = relres;
      R.converged = 1;
      break;
    }
    const double2* sh = W.s;
    if (M) {
      HFMM_TRY((*M)(W.s, W.shat));
      sh = W.shat;
      R.precond_applies++;
    }
    HFMM_TRY(A(sh, W.t));
    cd ts, tt;
    HFMM_TRY(bicg_dot(W, W.t, W.s, false, &ts, nullptr, s));
    HFMM_TRY(bicg_dot(W, W.t, W.t, false, &tt, nullptr, s));
    omega = tt != cd(0.0, 0.0) ? ts / tt : cd(0.0, 0.0);
    k_bicg_x<<<gN, 256, 0, s>>>(x, W.r, ph, sh, W.s, W.t, d2(alpha), d2(omega), N);
    count_launches(1);
    HFMM_TRY(bicg_dot(W, nullptr, W.r, true, nullptr, &rn, s));
    relres = rn / bnorm;
    if (!std::isfinite(relres)) return HFMM_ERR_NONFINITE;
    if (history && it - 1 < history_len) history[it - 1] = relres;
    rho_old = rho;
    if (relres < rtol) R.converged = 1;
    else if (omega == cd(0.0, 0.0)) R.breakdown = 1;
  }
  R.relres_est = relres;
  // true residual
  HFMM_TRY(A(x, W.v));
  k_bicg_sub<<<gN, 256, 0, s>>>(W.r, b, W.v, make_double2(1.0, 0.0), N);
  count_launches(1);
  HFMM_TRY(bicg_dot(W, nullptr, W.r, true, nullptr, &rn, s));
  R.relres_true = rn / bnorm;
  if (res) *res = R;
  return HFMM_OK;
}

#define HFMM_KRYLOV_INSTANTIATE(R)                                                                        \
  template int gmres_work_reserve<R>(GmresWorkT<R>&, int64_t, int, bool);                                 \
  template void gmres_work_free<R>(GmresWorkT<R>&);                                                       \
  template int dev_norm<R>(GmresWorkT<R>&, const C<R>*, int64_t, double*, cudaStream_t);                  \
  template int gmres_run<R>(GmresWorkT<R>&, const DevOpT<R>&, const DevOpT<R>*, const C<R>*, C<R>*, int,   \
                            double, int, bool, bool, GmresResult*, double*, int, cudaStream_t);           \
  template int gmres_cycle_device<R>(GmresWorkT<R>&, const DevOpT<R>&, const C<R>*, C<R>*, int, double,   \
                                     int*, int*, int*, cudaStream_t);
HFMM_KRYLOV_INSTANTIATE(double)
HFMM_KRYLOV_INSTANTIATE(float)
