// M2L on the tensor cores (FP32 form, dense far-field passes).
//
// At a level l >= lmin the multipole expansions are re-laid out per parity
// class of the cells (x, y, z bits 0) as dense lattices X[c][z][y][x][2P]
// (complex interleaved, 2P floats a row; cells without sources of the pass
// hold zeros).  Every cell of a class shares one M2L offset list (Sec. 5.1.2
// interaction lists), and for an offset o the sources of a brick of 8 x 4 x 4
// same-class target cells form a brick of one class at a shifted origin.  So
// one CTA owns two such bricks stacked in z (8 x 4 x 8 cells, 2 x 128 rows)
// and, for each offset of its list and each brick, accumulates the real form
// of the complex product
//     D[cell][2a'+c'] += sum_k X_src[cell][k] B_o[k][2a'+c'],
//     B_o[2a][2a'] = B_o[2a+1][2a'+1] = Re T_o(a', a),
//     B_o[2a][2a'+1] = Im T_o(a', a) = -B_o[2a+1][2a'],
// with tcgen05.mma (kind::tf32, M = 128 cells, N = 2P rounded up to 16,
// K = 8 per instruction) into a TMEM accumulator per brick.  The two source
// bricks arrive by one 5-D TMA load of an 8 x 4 x 8 box per 32-float slice of
// K (zero fill outside the level; rows x fastest, then y, then z, so the
// bricks are the box's first and second 128 rows); the operator slice by a
// 1-D bulk copy of a pre-swizzled image, read by the MMAs of both bricks.
// All use the 128-byte swizzled K-major layout (8-row atoms of 1024 bytes).
//
// FP32 accuracy from TF32 inputs: every operand is split as v = hi + lo with
// hi = v truncated to TF32 (exact in TF32) and lo = v - hi, and the product is
// hi*hi + hi*lo + lo*hi (the lo*lo term is below FP32 rounding).
//
// Warp roles (320 threads): warp 8 lane 0 issues the copies of a ring of
// NSTG stages; warp 9 lane 0 issues the MMAs, commits each stage back to the
// producer, and accumulates chunks of CHUNK offsets alternately into two
// TMEM buffers per brick; warps 0-7 (brick w / 4, TMEM lanes 32 (w % 4) ..
// + 31 = its cells) add each finished chunk to FP32 registers and free its
// buffer, then write the result.  Tensor-core accumulation rounds less carefully than FP32 FMA, so
// bounding its chains to one chunk keeps the FP32 form's accuracy.  Every
// wait is bounded (about one second); on time-out the kernel records
// HFMM_ERR_TIMEOUT, waits (bounded) for its own copies and MMAs in flight,
// frees its TMEM and returns.
#include <cuda.h>

#include <algorithm>
#include <new>
#include <vector>

#include "tc.cuh"
#include "tree.cuh"

namespace {

constexpr int TC_ACC_WARPS = 8;                      // warps that read TMEM (two bricks x lanes 0..127)
constexpr int TC_THREADS = 32 * (TC_ACC_WARPS + 2);  // + producer warp + MMA warp
constexpr int TC_NSTG = 2;
constexpr int TC_CHUNK = 8;       // offsets per tensor-core accumulation chain
constexpr int TC_MAX_NPAD = 128;  // accumulator columns (2P rounded up to 16)
constexpr int TC_TMEM_COLS = 512; // per brick two accumulator buffers of 128 columns
constexpr int BX = 8, BY = 4, BZ = 4;  // brick of same-class target cells (128 rows)
constexpr int NBRK = 2;                // bricks per CTA, stacked in z
constexpr int TC_MAX_COUNT = 2048;     // offsets per class list held in shared memory

__device__ int g_tc_error;  // set when a bounded wait gives up

__device__ __forceinline__ void tc_tma5(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3, int c4,
                                        uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
      "%6}], [%7];" ::"r"(sa(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(sa(bar))
      : "memory");
}

// X_hi / X_lo of level l: per class c and half coordinates, 2P floats a row;
// zero for cells holding no source of src_set
__global__ void k_tc_split(const float* __restrict__ M, const int* __restrict__ flags, int64_t off, int l, int twoP,
                           int src_set, float* __restrict__ xh, float* __restrict__ xl, const int* skip) {
  if (skip && *skip) return;
  const int64_t ncell = (int64_t)1 << (3 * l);
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= ncell * twoP) return;
  const int64_t m = e / twoP;
  const int k = (int)(e - m * twoP);
  int ix, iy, iz;
  morton_decode((uint64_t)m, ix, iy, iz);
  const int h = 1 << (l - 1);
  const int c = (ix & 1) | ((iy & 1) << 1) | ((iz & 1) << 2);
  const int64_t row = (((int64_t)c * h + (iz >> 1)) * h + (iy >> 1)) * h + (ix >> 1);
  const float v = (flags[off + m] & src_set) ? M[(off + m) * twoP + k] : 0.f;
  const float hv = tf32_hi(v);
  xh[row * twoP + k] = hv;
  xl[row * twoP + k] = v - hv;
}

// Pre-swizzled operator images: for each (level, slot), NA slices of
// [Npad rows n][32 floats k] in the 128-byte swizzled K-major layout, hi
// slices then lo slices; B^T[n][k] as in the header comment, zero outside
// n, k < 2P.  One-time, at the first tensor-core M2L of a tree.
__global__ void k_tc_ops(const float2* __restrict__ ops, int P, int64_t box_cells, int lmin, int L, int NA, int Npad,
                         float* __restrict__ img) {
  const int64_t per_slot = (int64_t)2 * NA * Npad * 32;  // floats
  const int64_t nslot = (int64_t)(L - lmin + 1) * box_cells;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nslot * NA * Npad * 32) return;
  const int64_t sl = e / ((int64_t)NA * Npad * 32);
  int64_t r = e - sl * ((int64_t)NA * Npad * 32);
  const int a = (int)(r / (Npad * 32));
  r -= (int64_t)a * Npad * 32;
  const int n = (int)(r / 32), kk = (int)(r % 32);
  const int k = 32 * a + kk;
  const int level = lmin + (int)(sl / box_cells);
  const int64_t slot = sl % box_cells;
  float v = 0.f;
  if (n < 2 * P && k < 2 * P) {
    const int ap = n >> 1, cp = n & 1, ai = k >> 1, ci = k & 1;
    const float2 T = ops[((int64_t)level * box_cells + slot) * P * P + (int64_t)ap * P + ai];
    // B^T[2a'+c'][2a+c]: (c',c) = (0,0) Re T, (0,1) -Im T, (1,0) Im T, (1,1) Re T
    v = (cp == ci) ? T.x : (cp == 0 ? -T.y : T.y);
  }
  const float hv = tf32_hi(v);
  // swizzled position of (n, kk) in the slice: 16-byte chunk (kk / 4) ^ (n % 8)
  const int64_t pos = (int64_t)n * 32 + (((kk >> 2) ^ (n & 7)) << 2) + (kk & 3);
  float* base = img + sl * per_slot + (int64_t)a * Npad * 32;
  base[pos] = hv;
  base[(int64_t)NA * Npad * 32 + pos] = v - hv;
}

struct TcMaps {
  CUtensorMap xh[HFMM_MAX_LEVEL + 1];
  CUtensorMap xl[HFMM_MAX_LEVEL + 1];
};

struct TcArgs {
  const float* img;         // operator images
  const int* m2l_off;       // [8][count] packed offsets
  const int* m2l_slot;      // [8][count] operator slot of each offset
  const int* flags;         // all levels
  const int64_t* level_off; // device copy
  float* Lc;                // local expansions (complex interleaved)
  float* part;              // split partial sums [nsplit][total_cells][2P], or null
  const int* skip;          // every kernel of the pass returns at once when set
  int64_t part_stride;      // floats
  int count;                // offsets per class
  int64_t box_cells;
  int P, NA, Npad, lmin, L;
  int tgt_set, accumulate;
  int brick_first[HFMM_MAX_LEVEL + 2];  // first CTA of each level
};

__device__ __forceinline__ void tc_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa(bar)) : "memory");
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_m2l_tc(const __grid_constant__ TcMaps maps, const TcArgs A) {
  if (A.skip && *A.skip) return;
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  // 1024-byte aligned stage buffers (the launch adds 1024 bytes of slack)
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  __shared__ __align__(8) uint64_t full[TC_NSTG], empty[TC_NSTG], ready[2], drained[2];
  __shared__ uint32_t tmem_base;
  __shared__ int vlist[TC_MAX_COUNT];
  __shared__ unsigned char vflag[TC_MAX_COUNT];
  __shared__ int nvalid;
  __shared__ int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int twoP = 2 * A.P;
  const uint32_t bxbytes = (uint32_t)(BX * BY * BZ * 128);  // one K slice of a brick
  const uint32_t xbytes = NBRK * bxbytes;                    // ... of the CTA's bricks
  const uint32_t bbytes = (uint32_t)A.Npad * 128;          // one K slice of an operator
  const uint32_t stage_bytes = 2 * xbytes + 2 * bbytes;

  // this CTA's brick: level, class, origin in half coordinates
  int level = A.lmin;
  while (level < A.L && (int)blockIdx.x >= A.brick_first[level + 1]) ++level;
  const int h = 1 << (level - 1);
  const int nbx = h / BX, nby = h / BY, nbz = h / (NBRK * BZ);
  int b = (int)blockIdx.x - A.brick_first[level];
  const int cls = b / (nbx * nby * nbz);
  b -= cls * nbx * nby * nbz;
  const int hz0 = (b / (nbx * nby)) * (NBRK * BZ);
  b %= nbx * nby;
  const int hy0 = (b / nbx) * BY, hx0 = (b % nbx) * BX;
  const int cx = cls & 1, cy = (cls >> 1) & 1, cz = (cls >> 2) & 1;

  if (tid == 0) {
    for (int s = 0; s < TC_NSTG; ++s) {
      tc_mbar_init(&full[s], 1);
      tc_mbar_init(&empty[s], 1);
    }
    for (int j = 0; j < 2; ++j) {
      tc_mbar_init(&ready[j], 1);
      tc_mbar_init(&drained[j], TC_ACC_WARPS);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(&tmem_base)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // offsets of this CTA's share of the class list whose source brick meets
  // the level, in list order
  const int ks = blockIdx.y, kn = gridDim.y;
  const int i0 = (int)((int64_t)A.count * ks / kn), i1 = (int)((int64_t)A.count * (ks + 1) / kn);
  for (int i = i0 + tid; i < i1; i += TC_THREADS) {
    const int o = A.m2l_off[cls * A.count + i];
    const int ox = (o & 255) - 128, oy = ((o >> 8) & 255) - 128, oz = ((o >> 16) & 255) - 128;
    const int sx = hx0 + ((cx + ox) >> 1), sy = hy0 + ((cy + oy) >> 1), sz = hz0 + ((cz + oz) >> 1);
    vflag[i - i0] = (sx + BX > 0 && sx < h && sy + BY > 0 && sy < h && sz + NBRK * BZ > 0 && sz < h) ? 1 : 0;
  }
  __syncthreads();
  if (warp == 0) {
    int base = 0;
    for (int c0 = 0; c0 < i1 - i0; c0 += 32) {
      const int j = c0 + lane;
      const bool f = j < i1 - i0 && vflag[j];
      const unsigned bal = __ballot_sync(0xffffffffu, f);
      if (f) vlist[base + __popc(bal & ((1u << lane) - 1u))] = i0 + j;
      base += __popc(bal);
    }
    if (lane == 0) nvalid = base;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const int NA = A.NA;
  const int nv = nvalid;
  const int units = nv * NA;
  const int cunits = TC_CHUNK * NA;                      // units per accumulation chunk
  const int nchunks = (nv + TC_CHUNK - 1) / TC_CHUNK;
  const uint32_t idesc = tc_idesc(128, A.Npad);

  if (warp == TC_ACC_WARPS && lane == 0) {
    // producer: one stage = one K slice of one offset
    for (int u = 0; u < units; ++u) {
      const int s = u % TC_NSTG;
      const uint32_t ph = (uint32_t)((u / TC_NSTG) & 1);
      if (!tc_wait(&empty[s], ph ^ 1u)) {
        atomicExch(&g_tc_error, 1);
        *(volatile int*)&abort_flag = 1;
        break;
      }
      if (*(volatile int*)&abort_flag) break;
      const int i = vlist[u / NA], a = u % NA;
      const int o = A.m2l_off[cls * A.count + i];
      const int ox = (o & 255) - 128, oy = ((o >> 8) & 255) - 128, oz = ((o >> 16) & 255) - 128;
      const int sc = ((cx + ox) & 1) | (((cy + oy) & 1) << 1) | (((cz + oz) & 1) << 2);
      const int sx = hx0 + ((cx + ox) >> 1), sy = hy0 + ((cy + oy) >> 1), sz = hz0 + ((cz + oz) >> 1);
      unsigned char* st = smem + (size_t)s * stage_bytes;
      const int slot = A.m2l_slot[cls * A.count + i];
      const float* img = A.img + (((int64_t)(level - A.lmin) * A.box_cells + slot) * 2 * NA + a) * A.Npad * 32;
      tc_expect_tx(&full[s], stage_bytes);
      tc_tma5(st, &maps.xh[level], 32 * a, sx, sy, sz, sc, &full[s]);
      tc_tma5(st + xbytes, &maps.xl[level], 32 * a, sx, sy, sz, sc, &full[s]);
      tc_bulk_g2s(st + 2 * xbytes, img, bbytes, &full[s]);
      tc_bulk_g2s(st + 2 * xbytes + bbytes, img + (int64_t)NA * A.Npad * 32, bbytes, &full[s]);
    }
  } else if (warp == TC_ACC_WARPS + 1 && lane == 0) {
    // MMA issuer: chunks of TC_CHUNK offsets into alternating TMEM buffers
    // (brick q: columns 256 q + 128 buf)
    for (int u = 0; u < units; ++u) {
      const int g = u / cunits, buf = g & 1;
      const bool first = (u % cunits) == 0;
      if (first && g >= 2 && !tc_wait(&drained[buf], (uint32_t)(((g >> 1) - 1) & 1))) {
        atomicExch(&g_tc_error, 1);
        *(volatile int*)&abort_flag = 1;
        break;
      }
      const int s = u % TC_NSTG;
      const uint32_t ph = (uint32_t)((u / TC_NSTG) & 1);
      if (!tc_wait(&full[s], ph)) {
        atomicExch(&g_tc_error, 1);
        *(volatile int*)&abort_flag = 1;
        break;
      }
      tc_fence_after();
      const int a = u % NA;
      const int kvalid = min(32, twoP - 32 * a);  // K of this slice
      const uint32_t st = sa(smem + (size_t)s * stage_bytes);
      const uint32_t bh = st + 2 * xbytes, bl = st + 2 * xbytes + bbytes;
      for (int q = 0; q < NBRK; ++q) {
        const uint32_t dt = tmem + (uint32_t)(q * 256 + buf * 128);
        const uint32_t xh = st + (uint32_t)q * bxbytes, xl = st + xbytes + (uint32_t)q * bxbytes;
        uint32_t acc = first ? 0u : 1u;
        for (int kk = 0; kk < kvalid; kk += 8) {
          const uint32_t ko = (uint32_t)kk * 4;
          tc_mma(dt, tc_desc(xh + ko), tc_desc(bh + ko), idesc, acc);
          acc = 1;
          tc_mma(dt, tc_desc(xh + ko), tc_desc(bl + ko), idesc, 1);
          tc_mma(dt, tc_desc(xl + ko), tc_desc(bh + ko), idesc, 1);
        }
      }
      tc_commit(&empty[s]);  // the stage is free once these MMAs have read it
      if ((u + 1) % cunits == 0 || u + 1 == units) tc_commit(&ready[buf]);  // chunk complete
    }
  } else if (warp < TC_ACC_WARPS) {
    // accumulator warps: TMEM lane r = brick cell r; each chunk is added to
    // FP32 registers (round to nearest), so no tensor-core accumulation chain
    // is longer than one chunk
    float sum[TC_MAX_NPAD];
#pragma unroll
    for (int c = 0; c < TC_MAX_NPAD; ++c) sum[c] = 0.f;
    bool good = true;
    for (int g = 0; g < nchunks; ++g) {
      const int buf = g & 1;
      if (!tc_wait(&ready[buf], (uint32_t)((g >> 1) & 1))) {
        atomicExch(&g_tc_error, 1);
        *(volatile int*)&abort_flag = 1;
        good = false;
        break;
      }
      tc_fence_after();
      const uint32_t ta = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((warp >> 2) * 256 + buf * 128);
#pragma unroll
      for (int c0 = 0; c0 < TC_MAX_NPAD; c0 += 16) {
        if (c0 < A.Npad) {
          float v[16];
          tc_ld16(ta + (uint32_t)c0, v);
#pragma unroll
          for (int j = 0; j < 16; ++j) sum[c0 + j] += v[j];
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) tc_arrive(&drained[buf]);
    }
    if (good) {
      const int r = (warp & 3) * 32 + lane;
      const int dx = r % BX, dy = (r / BX) % BY, dz = (warp >> 2) * BZ + r / (BX * BY);
      const int X = 2 * (hx0 + dx) + cx, Y = 2 * (hy0 + dy) + cy, Z = 2 * (hz0 + dz) + cz;
      const int64_t cell = A.level_off[level] + (int64_t)morton_encode(X, Y, Z);
      if (A.flags[cell] & A.tgt_set) {
        float* dst = A.part ? A.part + (int64_t)blockIdx.y * A.part_stride + cell * twoP : A.Lc + cell * twoP;
        const bool add = A.part ? false : A.accumulate != 0;
#pragma unroll
        for (int c = 0; c < TC_MAX_NPAD; ++c)
          if (c < twoP) dst[c] = add ? dst[c] + sum[c] : sum[c];
      }
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (*(volatile int*)&abort_flag && tid == 0) {
    // give copies and MMAs in flight a bounded time to land before the
    // shared memory and TMEM are released
    for (int s = 0; s < TC_NSTG; ++s) {
      tc_wait(&full[s], 0);
      tc_wait(&empty[s], 0);
    }
    tc_wait(&ready[0], 0);
    tc_wait(&ready[1], 0);
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
  }
}

// ---- the volume -> volume near field of a regular lattice tree on the
// tensor cores.  When every leaf holds the same s x s x s block of lattice
// nodes (n divisible by 2^L), the kernel block between the nodes of a target
// leaf and those of a source leaf at leaf offset o depends only on o: K_o(t,
// j) = G(h (s o + x_j - x_t)), the same for every leaf pair.  The near field
// of the volume targets from the volume sources is then, per near offset, the
// product of that fixed npl x npl matrix with the weights of the shifted leaf:
// the M2L's structure with the leaf's weights for its multipole and K_o for
// its operator, so the tensor-core M2L kernel computes it unchanged.

// operator images of the near offsets: slot i = near offset i, B^T[n][k] of
// K_o in the real form of the M2L images (n = 2t + c', k = 2j + c), read from
// the lattice table through the codes of a reference leaf and its neighbour
__global__ void k_tc_near_ops(const float2* __restrict__ tab, const int* __restrict__ lin, int ref_first,
                              const int* __restrict__ src_first, int nslot, int npl, int NA, int Npad,
                              float* __restrict__ img) {
  const int64_t per_slot = (int64_t)2 * NA * Npad * 32;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)nslot * NA * Npad * 32) return;
  const int sl = (int)(e / ((int64_t)NA * Npad * 32));
  int64_t r = e - (int64_t)sl * NA * Npad * 32;
  const int a = (int)(r / (Npad * 32));
  r -= (int64_t)a * Npad * 32;
  const int n = (int)(r / 32), kk = (int)(r % 32);
  const int k = 32 * a + kk;
  float v = 0.f;
  if (n < 2 * npl && k < 2 * npl) {
    const int t = n >> 1, cp = n & 1, j = k >> 1, ci = k & 1;
    const int dl = lin[ref_first + t] - lin[src_first[sl] + j];
    const float2 T = tab[dl < 0 ? -dl : dl];
    v = (cp == ci) ? T.x : (cp == 0 ? -T.y : T.y);
  }
  const float hv = tf32_hi(v);
  const int64_t pos = (int64_t)n * 32 + (((kk >> 2) ^ (n & 7)) << 2) + (kk & 3);
  float* base = img + sl * per_slot + (int64_t)a * Npad * 32;
  base[pos] = hv;
  base[(int64_t)NA * Npad * 32 + pos] = v - hv;
}

// X_hi / X_lo of the leaf level from the sorted weights: the row of leaf m is
// its npl volume weights (2 npl reals, padded with zeros to xs reals, a
// multiple of 4 for the tensor map's row stride), zero for leaves without
// volume points
__global__ void k_tc_near_split(const float2* __restrict__ qs, const int* __restrict__ leaf_start,
                                const int* __restrict__ flags, int64_t off, int l, int npl, int xs,
                                float* __restrict__ xh, float* __restrict__ xl, const int* skip) {
  if (skip && *skip) return;
  const int64_t ncell = (int64_t)1 << (3 * l);
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= ncell * xs) return;
  const int64_t m = e / xs;
  const int k = (int)(e - m * xs);
  int ix, iy, iz;
  morton_decode((uint64_t)m, ix, iy, iz);
  const int h = 1 << (l - 1);
  const int c = (ix & 1) | ((iy & 1) << 1) | ((iz & 1) << 2);
  const int64_t row = (((int64_t)c * h + (iz >> 1)) * h + (iy >> 1)) * h + (ix >> 1);
  float v = 0.f;
  if (k < 2 * npl && (flags[off + m] & HFMM_SET_VOL)) {
    const float2 q = qs[leaf_start[m] + (k >> 1)];
    v = (k & 1) ? q.y : q.x;
  }
  const float hv = tf32_hi(v);
  xh[row * xs + k] = hv;
  xl[row * xs + k] = v - hv;
}

// phis += near field + self term, for the volume points of every leaf
__global__ void k_tc_near_add(const float* __restrict__ out, int64_t off, const int* __restrict__ leaf_start,
                              const int* __restrict__ flags, int64_t nleaf, int npl, float2 sig,
                              const float2* __restrict__ qs, float2* __restrict__ phis, const int* skip) {
  if (skip && *skip) return;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nleaf * npl) return;
  const int64_t m = e / npl;
  const int t = (int)(e - m * npl);
  if (!(flags[off + m] & HFMM_SET_VOL)) return;
  const int j = leaf_start[m] + t;
  const float* o = out + (off + m) * 2 * npl + 2 * t;
  const float2 q = qs[j], p = phis[j];
  phis[j] = make_float2(p.x + o[0] + (sig.x * q.x - sig.y * q.y), p.y + o[1] + (sig.x * q.y + sig.y * q.x));
}

// L = (L +) sum over splits of the partial rows, for the target cells of the
// tensor-core levels
__global__ void k_tc_reduce(const float* __restrict__ part, int64_t part_stride, int nsplit,
                            const int* __restrict__ flags, int64_t off0, int64_t ncell, int twoP, int tgt_set,
                            int accumulate, float* __restrict__ Lc, const int* skip) {
  if (skip && *skip) return;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= ncell * twoP) return;
  const int64_t cell = off0 + e / twoP;
  if (!(flags[cell] & tgt_set)) return;
  const int64_t i = off0 * twoP + e;
  float v = part[i];
  for (int k = 1; k < nsplit; ++k) v += part[k * part_stride + i];
  Lc[i] = accumulate ? Lc[i] + v : v;
}

}  // namespace

struct fmm_tc_state {
  int ready = 0;
  int NA = 0, Npad = 0;
  float* img = nullptr;
  float* xh = nullptr;
  float* xl = nullptr;
  int64_t lat_off[HFMM_MAX_LEVEL + 1] = {};  // float offset of each level in xh / xl
  TcMaps maps;
};

void m2l_tc_release(fmm_tree* t) {
  delete t->m2l_tcore;  // its device buffers belong to the handle's allocation list
  t->m2l_tcore = nullptr;
}

// lowest level served by the tensor-core M2L (0: none): FP32 form, even P
// (rows of 16-byte multiples), 2P <= 256 (one MMA N), class lattices of at
// least 8 x 8 x 8 cells (levels >= 4), class lists held in shared memory
int m2l_tc_lmin(const fmm_tree* t) {
  if (!t->use_m2l_tcore || t->precision != HFMM_FP32 || (t->P & 1) || 2 * t->P > 256 ||
      t->m2l_count > TC_MAX_COUNT || t->L < 4)
    return 0;
  return 4;
}

static int tc_prepare(fmm_tree* t, cudaStream_t s) {
  if (t->m2l_tcore && t->m2l_tcore->ready) return HFMM_OK;
  const int lmin = m2l_tc_lmin(t);
  if (!lmin) return HFMM_ERR_UNSUPPORTED;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return HFMM_ERR_UNSUPPORTED;
  if (!t->m2l_tcore) t->m2l_tcore = new (std::nothrow) fmm_tc_state();
  if (!t->m2l_tcore) return HFMM_ERR_NOMEM;
  fmm_tc_state& S = *t->m2l_tcore;
  const int P = t->P, twoP = 2 * P, L = t->L;
  S.NA = (twoP + 31) / 32;
  S.Npad = (twoP + 15) / 16 * 16;
  // operator images
  const int64_t nslot = (int64_t)(L - lmin + 1) * t->box_cells;
  const int64_t img_floats = nslot * 2 * S.NA * S.Npad * 32;
  HFMM_TRY(tree_alloc(t, (void**)&S.img, sizeof(float) * img_floats));
  const int64_t nel = nslot * S.NA * S.Npad * 32;
  k_tc_ops<<<ceil_div(nel, 256), 256, 0, s>>>(t->op_m2l32, P, t->box_cells, lmin, L, S.NA, S.Npad, S.img);
  count_launches(1);
  HFMM_TRY(hfmm_last_launch());
  // lattice arrays and their tensor maps
  int64_t tot = 0;
  for (int l = lmin; l <= L; ++l) {
    S.lat_off[l] = tot;
    tot += ((int64_t)1 << (3 * l)) * twoP;
  }
  HFMM_TRY(tree_alloc(t, (void**)&S.xh, sizeof(float) * tot));
  HFMM_TRY(tree_alloc(t, (void**)&S.xl, sizeof(float) * tot));
  for (int l = lmin; l <= L; ++l) {
    const cuuint64_t hh = (cuuint64_t)1 << (l - 1);
    const cuuint64_t dims[5] = {(cuuint64_t)twoP, hh, hh, hh, 8};
    const cuuint64_t row = (cuuint64_t)twoP * sizeof(float);
    const cuuint64_t strides[4] = {row, row * hh, row * hh * hh, row * hh * hh * hh};
    const cuuint32_t box[5] = {32, BX, BY, NBRK * BZ, 1};
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    for (int w = 0; w < 2; ++w) {
      float* base = (w ? S.xl : S.xh) + S.lat_off[l];
      CUresult r = enc(w ? &S.maps.xl[l] : &S.maps.xh[l], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, base, dims, strides,
                       box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return HFMM_ERR_UNSUPPORTED;
    }
  }
  S.ready = 1;
  return HFMM_OK;
}

// Far field of levels lmin..L on the tensor cores; *nlaunch = kernels launched
int m2l_tc_stage(fmm_tree* t, int src_set, int tgt_set, int accumulate, cudaStream_t s, int* nlaunch) {
  *nlaunch = 0;
  HFMM_TRY(tc_prepare(t, s));
  fmm_tc_state& S = *t->m2l_tcore;
  const int lmin = m2l_tc_lmin(t), L = t->L, P = t->P, twoP = 2 * P;
  const float* M = reinterpret_cast<const float*>(t->M);
  for (int l = lmin; l <= L; ++l) {
    const int64_t n = ((int64_t)1 << (3 * l)) * twoP;
    k_tc_split<<<ceil_div(n, 256), 256, 0, s>>>(M, t->flags, t->level_off[l], l, twoP, src_set, S.xh + S.lat_off[l],
                                                S.xl + S.lat_off[l], t->skip);
    ++*nlaunch;
  }
  TcArgs A;
  A.img = S.img;
  A.m2l_off = t->m2l_off;
  A.m2l_slot = t->m2l_box_index;
  A.flags = t->flags;
  A.level_off = t->level_off_dev;
  A.Lc = reinterpret_cast<float*>(t->Lc);
  A.skip = t->skip;
  A.count = t->m2l_count;
  A.box_cells = t->box_cells;
  A.P = P;
  A.NA = S.NA;
  A.Npad = S.Npad;
  A.lmin = lmin;
  A.L = L;
  A.tgt_set = tgt_set;
  A.accumulate = accumulate;
  int nb = 0;
  for (int l = 0; l <= HFMM_MAX_LEVEL + 1; ++l) A.brick_first[l] = 0;
  for (int l = lmin; l <= L; ++l) {
    A.brick_first[l] = nb;
    const int h = 1 << (l - 1);
    nb += 8 * (h / BX) * (h / BY) * (h / (NBRK * BZ));
  }
  A.brick_first[L + 1] = nb;
  // split the offset lists until the grid covers the GPU about twice
  const int nsplit = std::max(1, std::min(t->m2l_part_max, (2 * 152 + nb - 1) / nb));
  A.part = nsplit > 1 ? reinterpret_cast<float*>(t->m2l_part) : nullptr;
  A.part_stride = t->total_cells * (int64_t)twoP;
  const size_t stage_bytes = 2 * (size_t)(NBRK * BX * BY * BZ * 128) + 2 * (size_t)S.Npad * 128;
  const size_t smem = TC_NSTG * stage_bytes + 1024;
  HFMM_TRY(set_smem_any((const void*)k_m2l_tc, smem));
  k_m2l_tc<<<dim3(nb, nsplit), TC_THREADS, smem, s>>>(S.maps, A);
  ++*nlaunch;
  if (nsplit > 1) {
    const int64_t off0 = t->level_off[lmin];
    const int64_t ncell = t->level_off[L] + ((int64_t)1 << (3 * L)) - off0;
    k_tc_reduce<<<ceil_div(ncell * twoP, 256), 256, 0, s>>>(A.part, A.part_stride, nsplit, t->flags, off0, ncell,
                                                            twoP, tgt_set, accumulate, A.Lc, t->skip);
    ++*nlaunch;
  }
  return hfmm_last_launch();
}

// nonzero when a bounded wait of the tensor-core M2L gave up (synchronises s);
// clears the flag when asked
int m2l_tc_error(cudaStream_t s, bool clear) {
  int h = 0;
  if (cudaMemcpyFromSymbolAsync(&h, g_tc_error, sizeof(int), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return 1;
  if (h && clear) {
    int z = 0;
    cudaMemcpyToSymbolAsync(g_tc_error, &z, sizeof(int), 0, cudaMemcpyHostToDevice, s);
  }
  return h;
}

// ---------------------------------------------------------------- near field on the tensor cores

struct fmm_tc_near_state {
  int ok = 0;        // 1 usable, -1 not for this tree
  int npl = 0, NA = 0, Npad = 0;
  int xs = 0;        // reals per row of the weight lattices (2 npl rounded up to 4)
  float* img = nullptr;
  float* xh = nullptr;
  float* xl = nullptr;
  float* out = nullptr;   // [level_off[L] + 8^L][2 npl] (rows of the leaf level used)
  float* part = nullptr;  // [nsplit][level_off[L] + 8^L][2 npl]
  int nsplit = 1;         // parts of the offset list (grid about two full waves)
  int* offs = nullptr;    // [8][near_count] packed near offsets (every class the same list)
  int* slots = nullptr;   // [8][near_count] slot = offset index
  TcMaps maps;
};

namespace {
constexpr int TC_NEAR_SPLIT = 32;  // at most this many parts of the offset list

// brick pairs of the leaf level
int near_bricks(int L) {
  const int h = 1 << (L - 1);
  return 8 * (h / BX) * (h / BY) * (h / (NBRK * BZ));
}
}

void near_tc_release(fmm_tree* t) {
  delete t->near_tcore;  // device buffers belong to the handle's allocation list
  t->near_tcore = nullptr;
}

// eligibility and set-up (host, once per tree): FP32 lattice tree of depth
// >= 4 whose leaves all hold the same s x s x s block of nodes (checked on the
// lattice codes of every leaf against a reference leaf), npl = s^3 <= 128
static int near_tc_prepare(fmm_tree* t, cudaStream_t s) {
  if (t->near_tcore) return t->near_tcore->ok > 0 ? HFMM_OK : HFMM_ERR_UNSUPPORTED;
  fmm_tc_near_state* S = new (std::nothrow) fmm_tc_near_state();
  if (!S) return HFMM_ERR_NOMEM;
  t->near_tcore = S;
  S->ok = -1;
  const int L = t->L;
  if (!t->lattice || t->precision != HFMM_FP32 || L < 4 || !t->lat_D || !t->lat_tab32 || t->near_count > TC_MAX_COUNT ||
      t->n % (1 << L))
    return HFMM_ERR_UNSUPPORTED;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return HFMM_ERR_UNSUPPORTED;
  const int sn = t->n >> L, npl = sn * sn * sn;
  if (2 * npl > TC_MAX_NPAD) return HFMM_ERR_UNSUPPORTED;
  const int64_t nleaf = (int64_t)1 << (3 * L);
  std::vector<int> ls(nleaf + 1), lm(nleaf), lin(t->n_pts);
  HFMM_CUDA_TRY(cudaStreamSynchronize(s));
  HFMM_CUDA_TRY(cudaMemcpy(ls.data(), t->leaf_start, sizeof(int) * (nleaf + 1), cudaMemcpyDeviceToHost));
  HFMM_CUDA_TRY(cudaMemcpy(lm.data(), t->leaf_mid, sizeof(int) * nleaf, cudaMemcpyDeviceToHost));
  HFMM_CUDA_TRY(cudaMemcpy(lin.data(), t->lat_lin, sizeof(int) * t->n_pts, cudaMemcpyDeviceToHost));
  // every leaf: npl volume points, whose codes are the reference leaf's
  // shifted by one constant (the same node pattern)
  const int half = 1 << (L - 1);
  const int64_t ref = (int64_t)morton_encode(half, half, half);
  for (int64_t m = 0; m < nleaf; ++m) {
    if (lm[m] - ls[m] != npl) return HFMM_ERR_UNSUPPORTED;
    const int sh = lin[ls[m]] - lin[ls[ref]];
    for (int q = 1; q < npl; ++q)
      if (lin[ls[m] + q] - lin[ls[ref] + q] != sh) return HFMM_ERR_UNSUPPORTED;
  }
  // the reference leaf's near neighbours (all inside the level)
  std::vector<int> noff(t->near_count), src_first(t->near_count);
  HFMM_CUDA_TRY(cudaMemcpy(noff.data(), t->near_off, sizeof(int) * t->near_count, cudaMemcpyDeviceToHost));
  const int sl = 1 << L;
  for (int i = 0; i < t->near_count; ++i) {
    const int o = noff[i];
    const int jx = half + (o & 255) - 128, jy = half + ((o >> 8) & 255) - 128, jz = half + ((o >> 16) & 255) - 128;
    if (jx < 0 || jy < 0 || jz < 0 || jx >= sl || jy >= sl || jz >= sl) return HFMM_ERR_UNSUPPORTED;
    src_first[i] = ls[morton_encode(jx, jy, jz)];
  }
  S->npl = npl;
  const int twoP = 2 * npl;
  S->xs = (twoP + 3) & ~3;
  S->NA = (twoP + 31) / 32;
  S->Npad = (twoP + 15) / 16 * 16;
  const int nslot = t->near_count;
  std::vector<int> offs(8 * (size_t)nslot), slots(8 * (size_t)nslot);
  for (int c = 0; c < 8; ++c)
    for (int i = 0; i < nslot; ++i) {
      offs[(size_t)c * nslot + i] = noff[i];
      slots[(size_t)c * nslot + i] = i;
    }
  int* d_src_first = nullptr;
  HFMM_TRY(tree_alloc(t, (void**)&d_src_first, sizeof(int) * nslot));
  HFMM_TRY(tree_alloc(t, (void**)&S->offs, sizeof(int) * offs.size()));
  HFMM_TRY(tree_alloc(t, (void**)&S->slots, sizeof(int) * slots.size()));
  HFMM_CUDA_TRY(cudaMemcpy(d_src_first, src_first.data(), sizeof(int) * nslot, cudaMemcpyHostToDevice));
  HFMM_CUDA_TRY(cudaMemcpy(S->offs, offs.data(), sizeof(int) * offs.size(), cudaMemcpyHostToDevice));
  HFMM_CUDA_TRY(cudaMemcpy(S->slots, slots.data(), sizeof(int) * slots.size(), cudaMemcpyHostToDevice));
  const int64_t img_floats = (int64_t)nslot * 2 * S->NA * S->Npad * 32;
  HFMM_TRY(tree_alloc(t, (void**)&S->img, sizeof(float) * img_floats));
  const int64_t nel = (int64_t)nslot * S->NA * S->Npad * 32;
  k_tc_near_ops<<<ceil_div(nel, 256), 256, 0, s>>>(t->lat_tab32, t->lat_lin, ls[ref], d_src_first, nslot, npl, S->NA,
                                                   S->Npad, S->img);
  count_launches(1);
  HFMM_TRY(hfmm_last_launch());
  const int64_t rows = t->level_off[L] + nleaf;
  HFMM_TRY(tree_alloc(t, (void**)&S->xh, sizeof(float) * nleaf * S->xs));
  HFMM_TRY(tree_alloc(t, (void**)&S->xl, sizeof(float) * nleaf * S->xs));
  HFMM_TRY(tree_alloc(t, (void**)&S->out, sizeof(float) * rows * twoP));
  {
    const int nb = near_bricks(L);
    S->nsplit = std::max(1, std::min(TC_NEAR_SPLIT, (2 * 152 + nb - 1) / nb));
  }
  HFMM_TRY(tree_alloc(t, (void**)&S->part, sizeof(float) * rows * twoP * S->nsplit));
  const cuuint64_t hh = (cuuint64_t)half;
  const cuuint64_t dims[5] = {(cuuint64_t)S->xs, hh, hh, hh, 8};
  const cuuint64_t row = (cuuint64_t)S->xs * sizeof(float);
  const cuuint64_t strides[4] = {row, row * hh, row * hh * hh, row * hh * hh * hh};
  const cuuint32_t box[5] = {32, BX, BY, NBRK * BZ, 1};
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  for (int w = 0; w < 2; ++w) {
    CUresult r = enc(w ? &S->maps.xl[L] : &S->maps.xh[L], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, w ? S->xl : S->xh, dims,
                     strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return HFMM_ERR_UNSUPPORTED;
  }
  HFMM_CUDA_TRY(cudaStreamSynchronize(s));
  S->ok = 1;
  return HFMM_OK;
}

bool near_tc_usable(fmm_tree* t, int src_set, int tgt_set, cudaStream_t s) {
  if (!t->use_near_tcore || t->precision != HFMM_FP32 || tgt_set != HFMM_SET_VOL || !(src_set & HFMM_SET_VOL))
    return false;
  if (!t->near_tcore) {
    // set up on first use, outside any capture only
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
      cudaGetLastError();
      return false;
    }
    const int st = near_tc_prepare(t, s);
    if (st != HFMM_OK && st != HFMM_ERR_UNSUPPORTED) return false;
  }
  return t->near_tcore && t->near_tcore->ok > 0;
}

// phis += the volume -> volume near field and the volume self terms (the
// boundary sources' near field is left to the caller); *nlaunch = kernels
int near_tc_stage(fmm_tree* t, cudaStream_t s, int* nlaunch) {
  *nlaunch = 0;
  HFMM_TRY(near_tc_prepare(t, s));
  fmm_tc_near_state& S = *t->near_tcore;
  const int L = t->L, npl = S.npl, twoP = 2 * npl;
  const int64_t nleaf = (int64_t)1 << (3 * L);
  const int64_t n = nleaf * S.xs;
  k_tc_near_split<<<ceil_div(n, 256), 256, 0, s>>>(reinterpret_cast<const float2*>(t->qs), t->leaf_start, t->flags,
                                                   t->level_off[L], L, npl, S.xs, S.xh, S.xl, t->skip);
  ++*nlaunch;
  TcArgs A;
  A.img = S.img;
  A.m2l_off = S.offs;
  A.m2l_slot = S.slots;
  A.flags = t->flags;
  A.level_off = t->level_off_dev;
  A.Lc = S.out;
  A.skip = t->skip;
  A.count = t->near_count;
  A.box_cells = t->near_count;
  A.P = npl;
  A.NA = S.NA;
  A.Npad = S.Npad;
  A.lmin = L;
  A.L = L;
  A.tgt_set = HFMM_SET_VOL;
  A.accumulate = 0;
  for (int l = 0; l <= HFMM_MAX_LEVEL + 1; ++l) A.brick_first[l] = 0;
  const int nb = near_bricks(L);
  A.brick_first[L] = 0;
  A.brick_first[L + 1] = nb;
  const int nsplit = S.nsplit;
  A.part = nsplit > 1 ? S.part : nullptr;
  A.part_stride = (t->level_off[L] + nleaf) * (int64_t)twoP;
  const size_t stage_bytes = 2 * (size_t)(NBRK * BX * BY * BZ * 128) + 2 * (size_t)S.Npad * 128;
  const size_t smem = TC_NSTG * stage_bytes + 1024;
  HFMM_TRY(set_smem_any((const void*)k_m2l_tc, smem));
  k_m2l_tc<<<dim3(nb, nsplit), TC_THREADS, smem, s>>>(S.maps, A);
  ++*nlaunch;
  if (nsplit > 1) {
    k_tc_reduce<<<ceil_div(nleaf * twoP, 256), 256, 0, s>>>(A.part, A.part_stride, nsplit, t->flags, t->level_off[L],
                                                           nleaf, twoP, HFMM_SET_VOL, 0, A.Lc, t->skip);
    ++*nlaunch;
  }
  const float2 sig = make_float2((float)t->sigma_vol.x, (float)t->sigma_vol.y);
  k_tc_near_add<<<ceil_div(nleaf * npl, 256), 256, 0, s>>>(S.out, t->level_off[L], t->leaf_start, t->flags, nleaf, npl,
                                                           sig, reinterpret_cast<const float2*>(t->qs),
                                                           reinterpret_cast<float2*>(t->phis), t->skip);
  ++*nlaunch;
  return hfmm_last_launch();
}
