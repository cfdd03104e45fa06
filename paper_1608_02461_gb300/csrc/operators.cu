// Translation operators of the FMM (Sec. 5.1.2: M2M, M2L, L2L), built on the
// device for one wavenumber k and every tree level.
//
// Each operator is the exact re-expansion of a truncated spherical-wave
// expansion about a new centre, truncated again to degrees n' < p.  With
// R_a(v) = j_n(k|v|) Y_n^m(v^) and S_a(v) = h_n(k|v|) Y_n^m(v^) the addition
// theorem gives the dense P x P matrices
//
//   T[a'][a] = 4 pi sum_l i^(n'+l-n) F_{l, m-m'}(t) Gaunt(a, a', l),
//   Gaunt(a, a', l) = integral Y_a conj(Y_a') conj(Y_{l, m-m'}) dOmega,
//
// with F = R for M2M (t = c_parent - c_child) and L2L (t = c_child -
// c_parent) and F = S for M2L (t = c_target - c_source).  The Gaunt integrals
// are 2 pi times a 1D integral of three normalised Legendre functions, done
// exactly with a Gauss-Legendre rule of 2p+4 nodes.
#include <cmath>

#include "special.cuh"
#include "tree.cuh"

namespace {

// Pbar_n^m(x) for one (n, m), any sign of m (Pbar_n^{-m} = (-1)^m Pbar_n^m)
__device__ double pbar(int n, int m, double x) {
  int am = m < 0 ? -m : m;
  if (am > n) return 0.0;
  double st = sqrt(fmax(0.0, 1.0 - x * x));
  double pmm = 0.28209479177387814347;
  for (int i = 1; i <= am; ++i) pmm *= -sqrt((2.0 * i + 1.0) / (2.0 * i)) * st;
  double val;
  if (n == am) {
    val = pmm;
  } else {
    double p0 = pmm, p1 = sqrt(2.0 * am + 3.0) * x * pmm;
    for (int j = am + 2; j <= n; ++j) {
      double a = sqrt((4.0 * j * j - 1.0) / ((double)j * j - (double)am * am));
      double b = sqrt(((double)(j - 1) * (j - 1) - (double)am * am) / (4.0 * (j - 1) * (j - 1) - 1.0));
      double p2 = a * (x * p1 - b * p0);
      p0 = p1;
      p1 = p2;
    }
    val = p1;
  }
  if (m < 0 && (am & 1)) val = -val;
  return val;
}

__device__ __forceinline__ void nm_of(int a, int& n, int& m) {
  n = (int)sqrt((double)a);
  while (n * n > a) --n;
  while ((n + 1) * (n + 1) <= a) ++n;
  m = a - n * n - n;
}

// gt[(a * P + ap) * lmax + l]
__global__ void k_gaunt(int p, double* gt) {
  __shared__ double xg[2 * HFMM_MAX_P + 4], wg[2 * HFMM_MAX_P + 4];
  const int nq = 2 * p + 4;
  if (threadIdx.x == 0) gauss_legendre(nq, xg, wg);
  __syncthreads();
  const int P = p * p, lmax = 2 * p - 1;
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)P * P * lmax) return;
  int l = (int)(idx % lmax);
  int ap = (int)((idx / lmax) % P);
  int a = (int)(idx / ((int64_t)lmax * P));
  int n, m, np_, mp;
  nm_of(a, n, m);
  nm_of(ap, np_, mp);
  int mu = m - mp;
  double v = 0.0;
  bool ok = (mu <= l && -mu <= l) && ((n + np_ + l) % 2 == 0) && (l >= abs(n - np_)) && (l <= n + np_);
  if (ok) {
    for (int q = 0; q < nq; ++q) {
      double x = xg[q];
      v += wg[q] * pbar(n, m, x) * pbar(np_, mp, x) * pbar(l, mu, x);
    }
    v *= 2.0 * M_PI;
  }
  gt[idx] = v;
}

// One block per (operator, level).  vec(op, level) gives t; kind 0 = R, 1 = S.
// M2M / L2L are stored column-major: entry (a', a) at
// out[(level * nops + op) * P * P + a * P + a'] (threads owning consecutive
// output rows read consecutive words); M2L operators row-major, entry (a', a)
// at ... + a' * P + a (a thread owning a row reads pairs of consecutive
// columns with one 16-byte load).
struct OpSet {
  int kind;     // 0: regular (j_l), 1: singular (h_l)
  int nops;     // operators per level
  int mode;     // 0: M2L offsets from `off`, 1: M2M child->parent, 2: L2L parent->child
  const int* off;  // packed offsets per slot (mode 0)
  int deriv;    // 1: d/dk of the operator (z_l(k|t|) -> |t| z_l'(k|t|))
};

__global__ void k_translation(int p, double k, int lmin, OpSet set, const double* gt, double2* out) {
  const int op = blockIdx.x;
  const int level = lmin + blockIdx.y;
  const int P = p * p, lmax = 2 * p - 1;
  __shared__ double2 F[(2 * HFMM_MAX_P - 1) * (2 * HFMM_MAX_P - 1)];
  __shared__ double zr[2 * HFMM_MAX_P], zi[2 * HFMM_MAX_P];
  __shared__ double pl[(2 * HFMM_MAX_P) * (2 * HFMM_MAX_P + 1) / 2];
  __shared__ double geo[5];  // r, ct, st, cp, sp
  if (threadIdx.x == 0) {
    double tx, ty, tz;
    if (set.mode == 0) {
      int o = set.off[op];
      int dx = (o & 255) - 128, dy = ((o >> 8) & 255) - 128, dz = ((o >> 16) & 255) - 128;
      double w = ldexp(1.0, -level);
      tx = -dx * w;  // c_T - c_S with S = T + d
      ty = -dy * w;
      tz = -dz * w;
    } else {
      double wc = ldexp(1.0, -(level + 1));  // child width
      int ox = op & 1, oy = (op >> 1) & 1, oz = (op >> 2) & 1;
      double sgn = set.mode == 1 ? 1.0 : -1.0;  // M2M: parent - child; L2L: child - parent
      tx = sgn * (0.5 - ox) * wc;
      ty = sgn * (0.5 - oy) * wc;
      tz = sgn * (0.5 - oz) * wc;
    }
    double r, ct, st, cp, sp;
    direction<double>(tx, ty, tz, r, ct, st, cp, sp);
    geo[0] = r;
    geo[1] = ct;
    geo[2] = st;
    geo[3] = cp;
    geo[4] = sp;
    double jl[2 * HFMM_MAX_P + 1], yl[2 * HFMM_MAX_P + 1];
    sph_bessel_j<double>(k * r, lmax + 1, jl);
    if (set.kind == 1) sph_bessel_y(k * r, lmax + 1, yl);
    for (int l = 0; l < lmax; ++l) {
      double a = jl[l], b = set.kind == 1 ? yl[l] : 0.0;
      if (set.deriv) {
        // d/dk z_l(k r) = r z_l'(k r); z_0' = -z_1, z_l' = z_{l-1} - (l+1)/x z_l
        double x = k * r;
        if (l == 0) {
          a = -jl[1];
          b = set.kind == 1 ? -yl[1] : 0.0;
        } else {
          a = jl[l - 1] - (l + 1) / x * jl[l];
          b = set.kind == 1 ? yl[l - 1] - (l + 1) / x * yl[l] : 0.0;
        }
        a *= r;
        b *= r;
      }
      zr[l] = a;
      zi[l] = b;
    }
    legendre_bar<double>(ct, st, lmax, pl);
  }
  __syncthreads();
  // F_{l,mu} = z_l(k r) Y_l^mu(t^)
  for (int e = threadIdx.x; e < lmax * lmax; e += blockDim.x) {
    int l = (int)sqrt((double)e);
    while (l * l > e) --l;
    while ((l + 1) * (l + 1) <= e) ++l;
    int mu = e - l * l - l;
    int am = mu < 0 ? -mu : mu;
    double ang = am * atan2(geo[4], geo[3]);
    double s_, c_;
    sincos(ang, &s_, &c_);
    double pv = pl[l * (l + 1) / 2 + am];
    double yr = pv * c_, yi = pv * s_;  // Y_l^|mu|
    if (mu < 0) {  // Y_l^{-m} = (-1)^m conj(Y_l^m)
      double sg = (am & 1) ? -1.0 : 1.0;
      yr = sg * yr;
      yi = -sg * yi;
    }
    F[e] = make_double2(zr[l] * yr - zi[l] * yi, zr[l] * yi + zi[l] * yr);
  }
  __syncthreads();
  double2* T = out + ((int64_t)blockIdx.y * set.nops + op) * P * P;
  for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
    int a, ap;
    if (set.mode == 0) {
      ap = e / P;
      a = e % P;
    } else {
      a = e / P;
      ap = e % P;
    }
    int n, m, np_, mp;
    nm_of(a, n, m);
    nm_of(ap, np_, mp);
    int mu = m - mp;
    double sr = 0.0, si = 0.0;
    const double* g = gt + ((int64_t)a * P + ap) * lmax;
    int lo = max(abs(mu), abs(n - np_));
    for (int l = lo; l <= n + np_ && l < lmax; ++l) {
      if ((n + np_ + l) & 1) continue;
      double gv = g[l];
      if (gv == 0.0) continue;
      // i^(n'+l-n) is real here: (-1)^((n'+l-n)/2)
      double sg = (((np_ + l - n) / 2) & 1) ? -1.0 : 1.0;
      double2 f = F[l * l + l + mu];
      sr += sg * gv * f.x;
      si += sg * gv * f.y;
    }
    T[e] = make_double2(4.0 * M_PI * sr, 4.0 * M_PI * si);
  }
}

__global__ void k_to_float(const double2* in, float2* out, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

}  // namespace

int build_operators(fmm_tree* t, cudaStream_t s) {
  const int p = t->p, P = t->P, lmax = 2 * p - 1, L = t->L;
  const int64_t PP = (int64_t)P * P;
  double* gt = nullptr;
  const int64_t ng = PP * lmax;
  HFMM_CUDA_TRY(cudaMallocAsync((void**)&gt, sizeof(double) * ng, s));
  k_gaunt<<<ceil_div(ng, 256), 256, 0, s>>>(p, gt);

  // M2M / L2L: 8 per level, levels 0..L (only 2..L-1 used)
  HFMM_TRY(tree_alloc_t(t, &t->op_m2m, (size_t)(L + 1) * 8 * PP));
  HFMM_TRY(tree_alloc_t(t, &t->op_l2l, (size_t)(L + 1) * 8 * PP));
  HFMM_TRY(tree_alloc_t(t, &t->op_m2l, (size_t)(L + 1) * t->box_cells * PP));
  HFMM_CUDA_TRY(cudaMemsetAsync(t->op_m2m, 0, sizeof(double2) * (L + 1) * 8 * PP, s));
  HFMM_CUDA_TRY(cudaMemsetAsync(t->op_l2l, 0, sizeof(double2) * (L + 1) * 8 * PP, s));
  HFMM_CUDA_TRY(cudaMemsetAsync(t->op_m2l, 0, sizeof(double2) * (L + 1) * t->box_cells * PP, s));

  if (L >= 3) {
    OpSet m2m{0, 8, 1, nullptr, 0}, l2l{0, 8, 2, nullptr, 0};
    dim3 g(8, L - 2);  // levels 2..L-1
    k_translation<<<g, 256, 0, s>>>(p, t->k, 2, m2m, gt, t->op_m2m + 2 * 8 * PP);
    k_translation<<<g, 256, 0, s>>>(p, t->k, 2, l2l, gt, t->op_l2l + 2 * 8 * PP);
  }
  {
    OpSet m2l{1, (int)t->box_cells, 0, t->m2l_slot_off, 0};
    dim3 g((unsigned)t->box_cells, L - 1);  // levels 2..L
    k_translation<<<g, 256, 0, s>>>(p, t->k, 2, m2l, gt, t->op_m2l + 2 * t->box_cells * PP);
  }
  HFMM_TRY(hfmm_last_launch());
  if (t->precision == HFMM_FP32) {
    int64_t n1 = (int64_t)(L + 1) * 8 * PP, n2 = (int64_t)(L + 1) * t->box_cells * PP;
    HFMM_TRY(tree_alloc_t(t, &t->op_m2m32, n1));
    HFMM_TRY(tree_alloc_t(t, &t->op_l2l32, n1));
    HFMM_TRY(tree_alloc_t(t, &t->op_m2l32, n2));
    k_to_float<<<ceil_div(n1, 256), 256, 0, s>>>(t->op_m2m, t->op_m2m32, n1);
    k_to_float<<<ceil_div(n1, 256), 256, 0, s>>>(t->op_l2l, t->op_l2l32, n1);
    k_to_float<<<ceil_div(n2, 256), 256, 0, s>>>(t->op_m2l, t->op_m2l32, n2);
    HFMM_TRY(hfmm_last_launch());
  }
  t->gaunt = gt;  // kept for the derivative operators (freed with the handle)
  return hfmm_last_launch();
}

namespace {

// slot of the negated offset: neg[slot(v)] = slot(-v) (the M2L offset set is
// symmetric); one thread per slot
__global__ void k_slot_neg(int nslots, const int* slot_off, int* neg) {
  int sl = blockIdx.x * blockDim.x + threadIdx.x;
  if (sl >= nslots) return;
  int o = slot_off[sl];
  int dx = (o & 255) - 128, dy = ((o >> 8) & 255) - 128, dz = ((o >> 16) & 255) - 128;
  int want = (-dx + 128) | ((-dy + 128) << 8) | ((-dz + 128) << 16);
  int r = -1;
  for (int q = 0; q < nslots; ++q)
    if (slot_off[q] == want) r = q;
  neg[sl] = r;
}

// Hermitian adjoints.  Column-major (M2M/L2L): out(a', a) = conj(in(a, a'));
// row-major M2L with slot map: out[slot](a', a) = conj(in[neg[slot]](a, a')).
__global__ void k_adjoint_colmajor(const double2* in, double2* out, int P, int64_t nmat) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t PP = (int64_t)P * P;
  if (e >= nmat * PP) return;
  int64_t m = e / PP, r = e % PP;
  int a = (int)(r / P), ap = (int)(r % P);  // element (a', a) at a*P + a'
  double2 v = in[m * PP + (int64_t)ap * P + a];
  out[e] = make_double2(v.x, -v.y);
}
__global__ void k_adjoint_m2l(const double2* in, double2* out, int P, int nslots, int levels,
                              const int* neg) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t PP = (int64_t)P * P;
  if (e >= (int64_t)levels * nslots * PP) return;
  int64_t m = e / PP, r = e % PP;
  int level = (int)(m / nslots), sl = (int)(m % nslots);
  int ap = (int)(r / P), a = (int)(r % P);  // row-major element (a', a)
  int src = neg[sl];
  double2 v = src >= 0 ? in[((int64_t)level * nslots + src) * PP + (int64_t)a * P + ap] : make_double2(0, 0);
  out[e] = make_double2(v.x, -v.y);
}

}  // namespace

// d/dk operators (tangent mode) and Hermitian adjoint operators (adjoint
// mode), built on first use of those modes
int build_operators_deriv(fmm_tree* t, cudaStream_t s) {
  if (t->op_m2l_d) return HFMM_OK;
  const int p = t->p, P = t->P, L = t->L;
  const int64_t PP = (int64_t)P * P;
  const int64_t n1 = (int64_t)(L + 1) * 8 * PP, n2 = (int64_t)(L + 1) * t->box_cells * PP;
  HFMM_TRY(tree_alloc_t(t, &t->op_m2m_d, n1));
  HFMM_TRY(tree_alloc_t(t, &t->op_l2l_d, n1));
  HFMM_TRY(tree_alloc_t(t, &t->op_m2l_d, n2));
  HFMM_CUDA_TRY(cudaMemsetAsync(t->op_m2m_d, 0, sizeof(double2) * n1, s));
  HFMM_CUDA_TRY(cudaMemsetAsync(t->op_l2l_d, 0, sizeof(double2) * n1, s));
  HFMM_CUDA_TRY(cudaMemsetAsync(t->op_m2l_d, 0, sizeof(double2) * n2, s));
  if (L >= 3) {
    OpSet m2m{0, 8, 1, nullptr, 1}, l2l{0, 8, 2, nullptr, 1};
    dim3 g(8, L - 2);
    k_translation<<<g, 256, 0, s>>>(p, t->k, 2, m2m, t->gaunt, t->op_m2m_d + 2 * 8 * PP);
    k_translation<<<g, 256, 0, s>>>(p, t->k, 2, l2l, t->gaunt, t->op_l2l_d + 2 * 8 * PP);
  }
  OpSet m2l{1, (int)t->box_cells, 0, t->m2l_slot_off, 1};
  k_translation<<<dim3((unsigned)t->box_cells, L - 1), 256, 0, s>>>(p, t->k, 2, m2l, t->gaunt,
                                                                    t->op_m2l_d + 2 * t->box_cells * PP);
  HFMM_TRY(hfmm_last_launch());
  if (t->precision == HFMM_FP32) {
    HFMM_TRY(tree_alloc_t(t, &t->op_m2m_d32, n1));
    HFMM_TRY(tree_alloc_t(t, &t->op_l2l_d32, n1));
    HFMM_TRY(tree_alloc_t(t, &t->op_m2l_d32, n2));
    k_to_float<<<ceil_div(n1, 256), 256, 0, s>>>(t->op_m2m_d, t->op_m2m_d32, n1);
    k_to_float<<<ceil_div(n1, 256), 256, 0, s>>>(t->op_l2l_d, t->op_l2l_d32, n1);
    k_to_float<<<ceil_div(n2, 256), 256, 0, s>>>(t->op_m2l_d, t->op_m2l_d32, n2);
  }
  return hfmm_last_launch();
}

int build_operators_adjoint(fmm_tree* t, cudaStream_t s) {
  if (t->op_m2l_h) return HFMM_OK;
  const int P = t->P, L = t->L;
  const int64_t PP = (int64_t)P * P;
  const int64_t n1 = (int64_t)(L + 1) * 8 * PP, n2 = (int64_t)(L + 1) * t->box_cells * PP;
  HFMM_TRY(tree_alloc_t(t, &t->m2l_slot_neg, t->box_cells));
  k_slot_neg<<<ceil_div(t->box_cells, 128), 128, 0, s>>>((int)t->box_cells, t->m2l_slot_off,
                                                         t->m2l_slot_neg);
  HFMM_TRY(tree_alloc_t(t, &t->op_m2m_h, n1));
  HFMM_TRY(tree_alloc_t(t, &t->op_l2l_h, n1));
  HFMM_TRY(tree_alloc_t(t, &t->op_m2l_h, n2));
  k_adjoint_colmajor<<<ceil_div(n1, 256), 256, 0, s>>>(t->op_m2m, t->op_m2m_h, P, (L + 1) * 8);
  k_adjoint_colmajor<<<ceil_div(n1, 256), 256, 0, s>>>(t->op_l2l, t->op_l2l_h, P, (L + 1) * 8);
  k_adjoint_m2l<<<ceil_div(n2, 256), 256, 0, s>>>(t->op_m2l, t->op_m2l_h, P, (int)t->box_cells, L + 1,
                                                  t->m2l_slot_neg);
  HFMM_TRY(hfmm_last_launch());
  if (t->precision == HFMM_FP32) {
    HFMM_TRY(tree_alloc_t(t, &t->op_m2m_h32, n1));
    HFMM_TRY(tree_alloc_t(t, &t->op_l2l_h32, n1));
    HFMM_TRY(tree_alloc_t(t, &t->op_m2l_h32, n2));
    k_to_float<<<ceil_div(n1, 256), 256, 0, s>>>(t->op_m2m_h, t->op_m2m_h32, n1);
    k_to_float<<<ceil_div(n1, 256), 256, 0, s>>>(t->op_l2l_h, t->op_l2l_h32, n1);
    k_to_float<<<ceil_div(n2, 256), 256, 0, s>>>(t->op_m2l_h, t->op_m2l_h32, n2);
  }
  return hfmm_last_launch();
}
