// Register-tiled block product of the M2L kernels (shared by the CUDA-core
// M2L pipelines and the boundary-operator kernel).
#pragma once

#include "common.cuh"

namespace {

// RT row groups x 8 column groups of threads; a thread owns rows r0 + r RT
// (r < R) and columns c0 + j 8 (j < CM) of the P x TC output tile.
// acc[r][j] += sum_a T(r0 + r RT, a) M(c0 + 8 j, a) for one staged offset:
// T row-major (P x P), source rows of stride MS; two consecutive a per step
// read with one 16-byte load per row (FP32) or two (FP64).  P is even.
template <typename T, int R, int CM, int RT>
__device__ __forceinline__ void m2l_block_product(const C<T>* __restrict__ Ts, const C<T>* __restrict__ Ms,
                                                  int P, int MS, int r0, int c0, C<T> (&acc)[R][CM]) {
  constexpr int CT = 8;
  const C<T>* trow[R];
  const C<T>* mrow[CM];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    int ap = r0 + r * RT;
    trow[r] = Ts + (size_t)(ap < P ? ap : 0) * P;
  }
#pragma unroll
  for (int j = 0; j < CM; ++j) mrow[j] = Ms + (size_t)(c0 + j * CT) * MS;
#pragma unroll 2
  for (int a = 0; a < P; a += 2) {
    C<T> t0[R], t1[R], m0[CM], m1[CM];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if constexpr (sizeof(T) == 4) {
        float4 v = *reinterpret_cast<const float4*>(trow[r] + a);
        t0[r] = mkc<T>(v.x, v.y);
        t1[r] = mkc<T>(v.z, v.w);
      } else {
        t0[r] = trow[r][a];
        t1[r] = trow[r][a + 1];
      }
    }
#pragma unroll
    for (int j = 0; j < CM; ++j) {
      if constexpr (sizeof(T) == 4) {
        float4 v = *reinterpret_cast<const float4*>(mrow[j] + a);
        m0[j] = mkc<T>(v.x, v.y);
        m1[j] = mkc<T>(v.z, v.w);
      } else {
        m0[j] = mrow[j][a];
        m1[j] = mrow[j][a + 1];
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int j = 0; j < CM; ++j) {
        cfma<T>(acc[r][j], t0[r], m0[j]);
        cfma<T>(acc[r][j], t1[r], m1[j]);
      }
  }
}

}  // namespace
