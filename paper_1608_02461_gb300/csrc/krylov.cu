// Krylov kernels: the 7-point Helmholtz operator (Sec. 2) and restarted
// (flexible) GMRES (Sec. 3-4) on device vectors, FP64 complex.
#include <cmath>

#include "krylov.cuh"
#include "tree.cuh"

namespace {

constexpr int RED_BLOCKS = 304;  // 2 x 152 SMs
constexpr int RED_THREADS = 256;

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

__device__ __forceinline__ double2 block_sum2(double2 v) {
  __shared__ double2 red[RED_THREADS / 32];
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : make_double2(0, 0);
    for (int o = 16; o > 0; o >>= 1) {
      v.x += __shfl_down_sync(0xffffffffu, v.x, o);
      v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
  }
  return v;  // valid in thread 0
}

// partial[i * gridDim.x + blk] = sum over the block's share of conj(V_i) w
__global__ void k_mdot_partial(const double2* __restrict__ V, int64_t ld, int nvec,
                               const double2* __restrict__ w, int64_t N, double2* partial, const int* skip) {
  if (skip && *skip) return;
  const int i = blockIdx.y;
  const double2* v = V + (int64_t)i * ld;
  double2 acc = make_double2(0, 0);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    double2 a = v[e], b = w[e];
    acc.x += a.x * b.x + a.y * b.y;
    acc.y += a.x * b.y - a.y * b.x;
  }
  acc = block_sum2(acc);
  if (threadIdx.x == 0) partial[(int64_t)i * gridDim.x + blockIdx.x] = acc;
}

__global__ void k_mdot_final(const double2* partial, int nblk, double2* out, const int* skip) {
  if (skip && *skip) return;
  const int i = blockIdx.x;
  double2 acc = make_double2(0, 0);
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
    double2 v = partial[(int64_t)i * nblk + b];
    acc.x += v.x;
    acc.y += v.y;
  }
  acc = block_sum2(acc);
  if (threadIdx.x == 0) out[i] = acc;
}

__global__ void k_norm_partial(const double2* __restrict__ x, int64_t N, double* partial, const int* skip) {
  if (skip && *skip) return;
  double2 acc = make_double2(0, 0);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    double2 a = x[e];
    acc.x += a.x * a.x + a.y * a.y;
  }
  acc = block_sum2(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc.x;
}

__global__ void k_norm_final(const double* partial, int nblk, double* out, const int* skip) {
  if (skip && *skip) return;
  double2 acc = make_double2(0, 0);
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc.x += partial[b];
  acc = block_sum2(acc);
  if (threadIdx.x == 0) *out = sqrt(acc.x);
}

// w += sign * sum_i coef[i] V_i
__global__ void k_axpy_multi(const double2* __restrict__ V, int64_t ld, int nvec,
                             const double2* __restrict__ coef, double sign, double2* w, int64_t N,
                             const int* skip, const int* nvec_dev) {
  if (skip && *skip) return;
  if (nvec_dev) nvec = *nvec_dev;
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= N) return;
  double2 acc = w[e];
  for (int i = 0; i < nvec; ++i) {
    double2 c = coef[i], v = V[(int64_t)i * ld + e];
    acc.x += sign * (c.x * v.x - c.y * v.y);
    acc.y += sign * (c.x * v.y + c.y * v.x);
  }
  w[e] = acc;
}

__global__ void k_sub(const double2* a, const double2* b, double2* out, int64_t N) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < N) out[e] = make_double2(a[e].x - b[e].x, a[e].y - b[e].y);
}

// dst = src / *nrm (no-op when the norm is zero)
__global__ void k_scale_by(const double2* src, const double* nrm, double2* dst, int64_t N, const int* skip) {
  if (skip && *skip) return;
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double d = *nrm;
  if (e < N && d > 0) dst[e] = make_double2(src[e].x / d, src[e].y / d);
}

// start of a cycle: g = (beta, 0, ...)
__global__ void k_cycle_init(int m, const double* beta, double2* g) {
  for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = make_double2(i == 0 ? *beta : 0.0, 0.0);
}

// Hessenberg column j from the CGS2 coefficients, previous rotations, a new
// complex Givens rotation, update of g, residual estimate and breakdown flag.
// scal: [0] ||w|| before orthogonalisation, [1] h_{j+1,j}, [2] relres,
//       [3] breakdown, [4] ||b||
__global__ void k_arnoldi(int j, int m, const double2* dots, double2* H, double* cs, double2* sn,
                          double2* g, double* scal, int* done, int* jdone, double rtol) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (done && *done) return;
  const int ld = m + 1;
  double2* col = H + (int64_t)j * ld;
  for (int i = 0; i <= j; ++i) col[i] = make_double2(dots[i].x + dots[ld + i].x, dots[i].y + dots[ld + i].y);
  double hnext = scal[1];
  col[j + 1] = make_double2(hnext, 0.0);
  scal[3] = (hnext <= 1e-14 * scal[0]) ? 1.0 : 0.0;
  for (int i = 0; i < j; ++i) {
    double2 a = col[i], b = col[i + 1];
    double c = cs[i];
    double2 s = sn[i];
    // a' = c a + s b ; b' = -conj(s) a + c b
    col[i] = make_double2(c * a.x + s.x * b.x - s.y * b.y, c * a.y + s.x * b.y + s.y * b.x);
    col[i + 1] = make_double2(-(s.x * a.x + s.y * a.y) + c * b.x, -(s.x * a.y - s.y * a.x) + c * b.y);
  }
  double2 a = col[j], b = col[j + 1];
  double aa = hypot(a.x, a.y);
  double c;
  double2 s;
  if (aa == 0.0) {
    c = 0.0;
    s = make_double2(1.0, 0.0);
  } else {
    double nu = sqrt(aa * aa + b.x * b.x + b.y * b.y);
    c = aa / nu;
    double2 ph = make_double2(a.x / aa, a.y / aa);           // a/|a|
    double2 cb = make_double2(b.x / nu, -b.y / nu);           // conj(b)/nu
    s = make_double2(ph.x * cb.x - ph.y * cb.y, ph.x * cb.y + ph.y * cb.x);
  }
  cs[j] = c;
  sn[j] = s;
  col[j] = make_double2(c * a.x + s.x * b.x - s.y * b.y, c * a.y + s.x * b.y + s.y * b.x);
  col[j + 1] = make_double2(0.0, 0.0);
  double2 gj = g[j];
  g[j + 1] = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));
  g[j] = make_double2(c * gj.x, c * gj.y);
  scal[2] = hypot(g[j + 1].x, g[j + 1].y) / scal[4];
  if (jdone) *jdone = j + 1;
  if (done && (scal[2] < rtol || scal[3] != 0.0 || !(scal[2] == scal[2]))) *done = 1;
}

// y = H(0:k,0:k)^-1 g(0:k), upper triangular
__global__ void k_backsolve(int kdim, int m, const double2* H, const double2* g, double2* y, const int* kdim_dev) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (kdim_dev) kdim = *kdim_dev;
  const int ld = m + 1;
  for (int i = kdim - 1; i >= 0; --i) {
    double2 acc = g[i];
    for (int q = i + 1; q < kdim; ++q) {
      double2 h = H[(int64_t)q * ld + i], v = y[q];
      acc.x -= h.x * v.x - h.y * v.y;
      acc.y -= h.x * v.y + h.y * v.x;
    }
    double2 d = H[(int64_t)i * ld + i];
    double den = d.x * d.x + d.y * d.y;
    y[i] = make_double2((acc.x * d.x + acc.y * d.y) / den, (acc.y * d.x - acc.x * d.y) / den);
  }
}

}  // namespace

int fdm_apply_dev(int n, double h, double k, const double2* u, double2* out, cudaStream_t s) {
  int64_t N = (int64_t)n * n * n;
  k_fdm<<<ceil_div(N, 256), 256, 0, s>>>(n, 1.0 / (h * h), k * k, u, out);
  count_launches(1);
  return hfmm_last_launch();
}

int gmres_work_reserve(GmresWork& W, int64_t N, int m, bool flexible) {
  if (W.base && W.N == N && W.m >= m && (W.flexible || !flexible)) return HFMM_OK;
  gmres_work_free(W);
  W.N = N;
  W.m = m;
  W.flexible = flexible;
  size_t nv = (size_t)(m + 1) + (flexible ? m : 0) + 2;
  size_t bytes = nv * N * sizeof(double2);
  bytes += (size_t)RED_BLOCKS * (m + 1) * sizeof(double2) * 2;  // partials
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
  W.V = (double2*)take((size_t)(m + 1) * N * sizeof(double2));
  W.Z = flexible ? (double2*)take((size_t)m * N * sizeof(double2)) : nullptr;
  W.w = (double2*)take(N * sizeof(double2));
  W.r = (double2*)take(N * sizeof(double2));
  W.partial = (double*)take((size_t)RED_BLOCKS * (m + 1) * sizeof(double2));
  W.dots = (double2*)take(2 * (m + 1) * sizeof(double2));
  W.H = (double2*)take((size_t)(m + 1) * m * sizeof(double2));
  W.cs = (double*)take(m * sizeof(double));
  W.sn = (double2*)take(m * sizeof(double2));
  W.g = (double2*)take((m + 1) * sizeof(double2));
  W.y = (double2*)take(m * sizeof(double2));
  W.scal = (double*)take(32 * sizeof(double));
  return HFMM_OK;
}

void gmres_work_free(GmresWork& W) {
  if (W.base) cudaFree(W.base);
  if (W.host) cudaFreeHost(W.host);
  W = GmresWork();
}

int dev_norm(GmresWork& W, const double2* x, int64_t N, double* out_dev, cudaStream_t s) {
  k_norm_partial<<<RED_BLOCKS, RED_THREADS, 0, s>>>(x, N, W.partial, W.skip);
  k_norm_final<<<1, RED_THREADS, 0, s>>>(W.partial, RED_BLOCKS, out_dev, W.skip);
  count_launches(2);
  return hfmm_last_launch();
}

static int mdot(GmresWork& W, const double2* V, int nvec, const double2* w, double2* out, cudaStream_t s) {
  dim3 g(RED_BLOCKS, nvec);
  k_mdot_partial<<<g, RED_THREADS, 0, s>>>(V, W.N, nvec, w, W.N, (double2*)W.partial, W.skip);
  k_mdot_final<<<nvec, RED_THREADS, 0, s>>>((double2*)W.partial, RED_BLOCKS, out, W.skip);
  count_launches(2);
  return hfmm_last_launch();
}

int gmres_run(GmresWork& W, const DevOp& A, const DevOp* M, const double2* b, double2* x, int m,
              double rtol, int maxit, bool x0_zero, bool true_residual, GmresResult* res,
              double* history, int history_len, cudaStream_t s) {
  const int64_t N = W.N;
  const unsigned gN = ceil_div(N, 256);
  GmresResult R;
  HFMM_TRY(dev_norm(W, b, N, W.scal + 4, s));
  HFMM_CUDA_TRY(cudaMemcpyAsync(W.host, W.scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
  HFMM_CUDA_TRY(cudaStreamSynchronize(s));
  const double bnorm = W.host[4];
  if (!std::isfinite(bnorm)) return HFMM_ERR_NONFINITE;
  if (bnorm == 0.0) {
    HFMM_CUDA_TRY(cudaMemsetAsync(x, 0, N * sizeof(double2), s));
    R.converged = 1;
    if (res) *res = R;
    return HFMM_OK;
  }
  double relres = 1.0;
  bool stop = false;
  while (true) {
    // r = b - A x, beta = ||r||
    if (x0_zero && R.iters == 0) {
      HFMM_CUDA_TRY(cudaMemcpyAsync(W.r, b, N * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    } else {
      HFMM_TRY(A(x, W.w));
      k_sub<<<gN, 256, 0, s>>>(b, W.w, W.r, N);
      count_launches(1);
    }
    HFMM_TRY(dev_norm(W, W.r, N, W.scal + 5, s));
    HFMM_CUDA_TRY(cudaMemcpyAsync(W.host, W.scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
    HFMM_CUDA_TRY(cudaStreamSynchronize(s));
    relres = W.host[5] / bnorm;
    if (!std::isfinite(relres)) return HFMM_ERR_NONFINITE;
    if (relres < rtol) {
      R.converged = 1;
      break;
    }
    if (R.iters >= maxit) break;
    k_cycle_init<<<1, 64, 0, s>>>(m, W.scal + 5, W.g);
    k_scale_by<<<gN, 256, 0, s>>>(W.r, W.scal + 5, W.V, N, nullptr);
    count_launches(2);
    int jdone = 0;
    for (int j = 0; j < m; ++j) {
      double2* vj = W.V + (int64_t)j * N;
      double2* zj = vj;
      if (M) {
        zj = W.Z + (int64_t)j * N;
        HFMM_TRY((*M)(vj, zj));
      }
      HFMM_TRY(A(zj, W.w));
      HFMM_TRY(dev_norm(W, W.w, N, W.scal + 0, s));
      // classical Gram-Schmidt, twice
      HFMM_TRY(mdot(W, W.V, j + 1, W.w, W.dots, s));
      k_axpy_multi<<<gN, 256, 0, s>>>(W.V, N, j + 1, W.dots, -1.0, W.w, N, nullptr, nullptr);
      HFMM_TRY(mdot(W, W.V, j + 1, W.w, W.dots + (m + 1), s));
      k_axpy_multi<<<gN, 256, 0, s>>>(W.V, N, j + 1, W.dots + (m + 1), -1.0, W.w, N, nullptr, nullptr);
      HFMM_TRY(dev_norm(W, W.w, N, W.scal + 1, s));
      k_arnoldi<<<1, 1, 0, s>>>(j, m, W.dots, W.H, W.cs, W.sn, W.g, W.scal, nullptr, nullptr, 0.0);
      count_launches(3);
      if (j + 1 < m) {
        k_scale_by<<<gN, 256, 0, s>>>(W.w, W.scal + 1, W.V + (int64_t)(j + 1) * N, N, nullptr);
        count_launches(1);
      }
      HFMM_TRY(hfmm_last_launch());
      HFMM_CUDA_TRY(cudaMemcpyAsync(W.host, W.scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
      HFMM_CUDA_TRY(cudaStreamSynchronize(s));
      relres = W.host[2];
      if (history && R.iters < history_len) history[R.iters] = relres;
      R.iters++;
      jdone = j + 1;
      if (!std::isfinite(relres)) return HFMM_ERR_NONFINITE;
      bool breakdown = W.host[3] != 0.0;
      if (relres < rtol || breakdown || R.iters >= maxit) {
        stop = true;
        if (relres < rtol || breakdown) R.converged = 1;
        break;
      }
    }
    k_backsolve<<<1, 1, 0, s>>>(jdone, m, W.H, W.g, W.y, nullptr);
    k_axpy_multi<<<gN, 256, 0, s>>>(M ? W.Z : W.V, N, jdone, W.y, 1.0, x, N, nullptr, nullptr);
    count_launches(2);
    HFMM_TRY(hfmm_last_launch());
    if (stop) break;
    R.restarts++;
  }
  R.relres_est = relres;
  if (!true_residual) {
    R.relres_true = -1.0;
    if (res) *res = R;
    return HFMM_OK;
  }
  // true residual
  HFMM_TRY(A(x, W.w));
  k_sub<<<gN, 256, 0, s>>>(b, W.w, W.r, N);
  count_launches(1);
  HFMM_TRY(dev_norm(W, W.r, N, W.scal + 6, s));
  HFMM_CUDA_TRY(cudaMemcpyAsync(W.host, W.scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
  HFMM_CUDA_TRY(cudaStreamSynchronize(s));
  R.relres_true = W.host[6] / bnorm;
  if (res) *res = R;
  return HFMM_OK;
}

// ---------------------------------------------------------------- graph form

namespace {

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

int gmres_cycle_device(GmresWork& W, const DevOp& A, const double2* b, double2* x, int m, double rtol, int* d_done,
                       int* d_jdone, int* d_total, cudaStream_t s) {
  const int64_t N = W.N;
  const unsigned gN = ceil_div(N, 256);
  if (W.m < m) return HFMM_ERR_INVALID_ARG;
  HFMM_CUDA_TRY(cudaMemsetAsync(x, 0, N * sizeof(double2), s));
  W.skip = nullptr;
  HFMM_TRY(dev_norm(W, b, N, W.scal + 5, s));
  k_cycle_start<<<1, 1, 0, s>>>(m, W.scal, W.g, d_done, d_jdone);
  W.skip = d_done;
  k_scale_by<<<gN, 256, 0, s>>>(b, W.scal + 5, W.V, N, d_done);
  count_launches(2);
  for (int j = 0; j < m; ++j) {
    double2* vj = W.V + (int64_t)j * N;
    HFMM_TRY(A(vj, W.w));
    HFMM_TRY(dev_norm(W, W.w, N, W.scal + 0, s));
    HFMM_TRY(mdot(W, W.V, j + 1, W.w, W.dots, s));
    k_axpy_multi<<<gN, 256, 0, s>>>(W.V, N, j + 1, W.dots, -1.0, W.w, N, d_done, nullptr);
    HFMM_TRY(mdot(W, W.V, j + 1, W.w, W.dots + (m + 1), s));
    k_axpy_multi<<<gN, 256, 0, s>>>(W.V, N, j + 1, W.dots + (m + 1), -1.0, W.w, N, d_done, nullptr);
    HFMM_TRY(dev_norm(W, W.w, N, W.scal + 1, s));
    k_arnoldi<<<1, 1, 0, s>>>(j, m, W.dots, W.H, W.cs, W.sn, W.g, W.scal, d_done, d_jdone, rtol);
    count_launches(3);
    if (j + 1 < m) {
      k_scale_by<<<gN, 256, 0, s>>>(W.w, W.scal + 1, W.V + (int64_t)(j + 1) * N, N, d_done);
      count_launches(1);
    }
  }
  W.skip = nullptr;
  k_backsolve<<<1, 1, 0, s>>>(0, m, W.H, W.g, W.y, d_jdone);
  k_axpy_multi<<<gN, 256, 0, s>>>(W.V, N, 0, W.y, 1.0, x, N, nullptr, d_jdone);
  k_count_add<<<1, 1, 0, s>>>(d_jdone, d_total);
  count_launches(3);
  return hfmm_last_launch();
}
