// Shared device helpers: complex arithmetic, Morton codes, error plumbing.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "../../include/hfmm.h"

#define HFMM_MAX_P 16
#define HFMM_MAX_LEVEL 9
// lattice near-field kernel: sources staged per window, and the largest
// table it stages in shared memory (table + window + 4 KB within 227 KB)
#define HFMM_LAT_WS 2048
#define HFMM_SMEM_MAX (227 * 1024)
#define HFMM_LAT_TABLE_MAX_BYTES (180 * 1024)

// ---------------------------------------------------------------- complex

template <typename T> struct cplx;
template <> struct cplx<double> { using type = double2; };
template <> struct cplx<float> { using type = float2; };
template <typename T> using C = typename cplx<T>::type;

template <typename T>
__host__ __device__ __forceinline__ C<T> mkc(T re, T im) {
  C<T> z;
  z.x = re;
  z.y = im;
  return z;
}
template <typename T>
__host__ __device__ __forceinline__ C<T> cadd(C<T> a, C<T> b) { return mkc<T>(a.x + b.x, a.y + b.y); }
template <typename T>
__host__ __device__ __forceinline__ C<T> csub(C<T> a, C<T> b) { return mkc<T>(a.x - b.x, a.y - b.y); }
template <typename T>
__host__ __device__ __forceinline__ C<T> cmul(C<T> a, C<T> b) {
  return mkc<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T>
__host__ __device__ __forceinline__ C<T> conjc(C<T> a) { return mkc<T>(a.x, -a.y); }
template <typename T>
__host__ __device__ __forceinline__ C<T> cscale(C<T> a, T s) { return mkc<T>(a.x * s, a.y * s); }
// acc += a * b
template <typename T>
__host__ __device__ __forceinline__ void cfma(C<T>& acc, C<T> a, C<T> b) {
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
// acc += conj(a) * b
template <typename T>
__host__ __device__ __forceinline__ void cfma_conj(C<T>& acc, C<T> a, C<T> b) {
  acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
}

// ---------------------------------------------------------------- Morton codes

// spread the low 21 bits of v to every third bit
__host__ __device__ __forceinline__ uint64_t spread3(uint64_t v) {
  v &= 0x1fffffULL;
  v = (v | (v << 32)) & 0x1f00000000ffffULL;
  v = (v | (v << 16)) & 0x1f0000ff0000ffULL;
  v = (v | (v << 8)) & 0x100f00f00f00f00fULL;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ULL;
  v = (v | (v << 2)) & 0x1249249249249249ULL;
  return v;
}
__host__ __device__ __forceinline__ uint64_t compact3(uint64_t v) {
  v &= 0x1249249249249249ULL;
  v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ULL;
  v = (v ^ (v >> 4)) & 0x100f00f00f00f00fULL;
  v = (v ^ (v >> 8)) & 0x1f0000ff0000ffULL;
  v = (v ^ (v >> 16)) & 0x1f00000000ffffULL;
  v = (v ^ (v >> 32)) & 0x1fffffULL;
  return v;
}
// bit 0 of each triple = x, bit 1 = y, bit 2 = z
__host__ __device__ __forceinline__ uint64_t morton_encode(int ix, int iy, int iz) {
  return spread3((uint64_t)ix) | (spread3((uint64_t)iy) << 1) | (spread3((uint64_t)iz) << 2);
}
__host__ __device__ __forceinline__ void morton_decode(uint64_t m, int& ix, int& iy, int& iz) {
  ix = (int)compact3(m);
  iy = (int)compact3(m >> 1);
  iz = (int)compact3(m >> 2);
}

// ---------------------------------------------------------------- tree lists
// Two cells of one level whose centres lie d cell widths apart (d2 = |d|^2)
// are well separated iff theta^2 d2 > 1, theta = num / den (the multipole
// acceptance test of the octree, Sec. 5.1.1 with theta of Sec. 7).
__host__ __device__ __forceinline__ bool separated(int d2, int64_t num, int64_t den) {
  return num * num * (int64_t)d2 > den * den;
}
// floor(x / 2) for any sign: the parent offset of a child offset
__host__ __device__ __forceinline__ int floor_half(int x) { return x >= 0 ? x / 2 : -((1 - x) / 2); }

// theta as a rational num / den (smallest den <= 1000 that represents it to
// 1e-9), so that the separation test is exact integer arithmetic
inline void theta_rational(double th, int64_t& num, int64_t& den) {
  for (int64_t d = 1; d <= 1000; ++d) {
    double n = th * d;
    int64_t r = (int64_t)llround(n);
    if (r > 0 && fabs(n - r) < 1e-9 * d) {
      num = r;
      den = d;
      return;
    }
  }
  den = 1000;
  num = (int64_t)llround(th * 1000);
}

// ---------------------------------------------------------------- error plumbing

#define HFMM_CUDA_TRY(...)                               \
  do {                                                   \
    cudaError_t _e = (__VA_ARGS__);                      \
    if (_e != cudaSuccess) return HFMM_ERR_CUDA;         \
  } while (0)

#define HFMM_TRY(...)                                    \
  do {                                                   \
    int _s = (__VA_ARGS__);                              \
    if (_s != HFMM_OK) return _s;                        \
  } while (0)

static inline int hfmm_last_launch() {
  return cudaGetLastError() == cudaSuccess ? HFMM_OK : HFMM_ERR_CUDA;
}

static inline unsigned ceil_div(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }
