// Device special functions for the spherical-wave expansions of the 3D
// Helmholtz kernel G = exp(i k r) / (4 pi r) (Sec. 5.2):
//   spherical Bessel j_n (power series / upward / Miller downward recurrence),
//   spherical Neumann y_n (upward recurrence), orthonormal spherical harmonics
//   Y_n^m with the Condon-Shortley phase via normalised associated Legendre
//   recurrences.  Coefficient index a = n^2 + n + m.
#pragma once

#include "common.cuh"

// j_n(x) for n = 0..nmax-1 into out[].  Three regimes:
//  x < 1         power series j_n = x^n/(2n+1)!! sum_s (-x^2/2)^s / (s! prod_{i<=s}(2n+2i+1))
//  x >= nmax-1   upward recurrence j_{n+1} = (2n+1)/x j_n - j_{n-1} (stable for n < x)
//  otherwise     Miller's downward recurrence from well above nmax, rescaled on the
//                way and normalised by whichever of j_0, j_1 has the larger size.
template <typename T>
__device__ __forceinline__ void sph_bessel_j(T x, int nmax, T* out) {
  if (x < T(1)) {
    T x2h = T(0.5) * x * x;
    T lead = T(1);  // x^n / (2n+1)!!
    for (int n = 0; n < nmax; ++n) {
      if (n > 0) lead *= x / T(2 * n + 1);
      T term = T(1), sum = T(1);
      for (int s = 1; s < 40; ++s) {
        term *= -x2h / (T(s) * T(2 * n + 2 * s + 1));
        sum += term;
        if (fabs(term) < T(1e-18) * fabs(sum)) break;
      }
      out[n] = lead * sum;
    }
    return;
  }
  T sx, cx;
  if constexpr (sizeof(T) == 8) {
    sincos(x, &sx, &cx);
  } else {
    sincosf(x, &sx, &cx);
  }
  T j0 = sx / x;
  T j1 = sx / (x * x) - cx / x;
  if (x >= T(nmax - 1)) {
    out[0] = j0;
    if (nmax > 1) out[1] = j1;
    for (int n = 1; n + 1 < nmax; ++n) out[n + 1] = T(2 * n + 1) / x * out[n] - out[n - 1];
    return;
  }
  int start = nmax + 24 + (int)(2.0 * sqrt((double)nmax));
  constexpr T tiny = sizeof(T) == 8 ? T(1e-280) : T(1e-30);
  constexpr T scale_big = sizeof(T) == 8 ? T(1e250) : T(1e30);
  T jp1 = T(0), jn = tiny;
  for (int n = start; n >= 1; --n) {
    T jm1 = T(2 * n + 1) / x * jn - jp1;
    jp1 = jn;
    jn = jm1;
    if (n - 1 < nmax) out[n - 1] = jn;
    if (fabs(jn) > scale_big) {  // rescale everything computed so far
      T s = T(1) / scale_big;
      jn *= s;
      jp1 *= s;
      for (int i = n - 1; i < nmax; ++i) out[i] *= s;
    }
  }
  // out[0] ~ c j0, out[1] ~ c j1
  T c = (fabs(j0) >= fabs(j1)) ? j0 / out[0] : j1 / out[1];
  for (int n = 0; n < nmax; ++n) out[n] *= c;
}

// y_n(x), n = 0..nmax-1, upward recurrence (stable), x > 0.
__device__ __forceinline__ void sph_bessel_y(double x, int nmax, double* out) {
  double sx, cx;
  sincos(x, &sx, &cx);
  out[0] = -cx / x;
  if (nmax > 1) out[1] = -cx / (x * x) - sx / x;
  for (int n = 1; n + 1 < nmax; ++n) out[n + 1] = double(2 * n + 1) / x * out[n] - out[n - 1];
}

// Normalised associated Legendre values Pbar_n^m(ct), 0 <= m <= n < nmax, with
// st = sin(theta) >= 0, stored at index n(n+1)/2 + m.
//   Pbar_n^m = sqrt((2n+1)/(4 pi) (n-m)!/(n+m)!) P_n^m, P_n^m with the
//   Condon-Shortley phase, so that Y_n^m = Pbar_n^m e^{i m phi}.
template <typename T>
__device__ __forceinline__ void legendre_bar(T ct, T st, int nmax, T* out) {
  const T inv_sqrt_4pi = T(0.28209479177387814347);
  T pmm = inv_sqrt_4pi;
  for (int m = 0; m < nmax; ++m) {
    if (m > 0) pmm *= -sqrt(T(2 * m + 1) / T(2 * m)) * st;
    out[m * (m + 1) / 2 + m] = pmm;
    if (m + 1 < nmax) {
      T p1 = sqrt(T(2 * m + 3)) * ct * pmm;
      out[(m + 1) * (m + 2) / 2 + m] = p1;
      T p0 = pmm;
      for (int n = m + 2; n < nmax; ++n) {
        T a = sqrt(T(4 * n * n - 1) / T(n * n - m * m));
        T b = sqrt(T((n - 1) * (n - 1) - m * m) / T(4 * (n - 1) * (n - 1) - 1));
        T pn = a * (ct * p1 - b * p0);
        out[n * (n + 1) / 2 + m] = pn;
        p0 = p1;
        p1 = pn;
      }
    }
  }
}

// Angles of a vector: cos/sin of the polar angle and e^{i phi}.
template <typename T>
__device__ __forceinline__ void direction(T dx, T dy, T dz, T& r, T& ct, T& st, T& cp, T& sp) {
  T rxy2 = dx * dx + dy * dy;
  r = sqrt(rxy2 + dz * dz);
  T rxy = sqrt(rxy2);
  if (r > T(0)) {
    ct = dz / r;
    st = rxy / r;
  } else {
    ct = T(1);
    st = T(0);
  }
  if (rxy > T(0)) {
    cp = dx / rxy;
    sp = dy / rxy;
  } else {
    cp = T(1);
    sp = T(0);
  }
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton's method on P_n.
static __device__ __noinline__ void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int j = 2; j <= n; ++j) {
        double p2 = ((2 * j - 1) * z * p1 - (j - 1) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    // recompute P_n' at the converged node for the weight
    double p0 = 1.0, p1 = z;
    for (int j = 2; j <= n; ++j) {
      double p2 = ((2 * j - 1) * z * p1 - (j - 1) * p0) / j;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

