// Boundary -> boundary FMM apply as one persistent kernel.
//
// The inner solve of the preconditioner (Sec. 5.2, Eq. (ubound) with u = 0,
// by GMRES with every product an FMM, Sec. 5.3) applies the single-layer
// operator between the boundary panels once per inner iteration: hundreds of
// times per outer solve, on the 6 n^2 panels only.  Launched as the usual
// chain of the FMM flow (Sec. 5.1.2: gather, P2M, M2M per level, M2L, L2L per
// level, L2P, near field, scatter) each stage is a short kernel bound by the
// latency of its dependent loads.  Here the same stages run as phases of one
// cooperative kernel whose CTAs stay resident (one per SM), separated by grid
// barriers whose waits are bounded (about one second; on time-out the kernel
// records HFMM_ERR_TIMEOUT and every CTA returns).  For a leaf level L >= 4:
//   phase 0   P2M at the boundary leaves, M2M into their parents (per parent)
//   phase 1   M2L products of levels L-1 and L: the (target, source) cell
//             pairs grouped by operator slot, 32 per item, operator (bulk
//             copy) and source rows (TMA gathers) double-buffered per group
//             of threads; M2M into level 2; then the near field of the
//             leaves through the lattice kernel table, with the self term
//   phase 2   products of level 2; row sums (pair order) of levels L-1, L
//   then      per level l = 3 .. L: L_l = (its row sum) + L2L of its
//             parent's L; at the leaf level L2P plus the near field, written
//             to the output in the caller's order
// (shallower trees fold the row sums and the near field into the downward
// phases).  Inside the inner solve the kernel runs the whole GMRES cycle:
// per step one apply as above, then classical Gram-Schmidt twice, the Givens
// update, and at the end the back substitution and x = V y.
// Every sum is taken in a fixed order, so results are deterministic.  Input
// and output are boundary vectors in the caller's (original) panel order; the
// kernel reads x through the sorted order itself.
#include <algorithm>
#include <map>
#include <new>
#include <vector>

#include "m2l_product.cuh"
#include "tc.cuh"
#include "tree.cuh"

namespace {

enum BoSegType { SEG_P2M_UP = 0, SEG_P2M = 1, SEG_M2M = 2, SEG_PROD = 3, SEG_DOWN = 4, SEG_ROWS = 5, SEG_NEAR = 6 };
// SEG_DOWN flags (in BoSeg::first): the cell's product rows were summed into
// its L by an earlier SEG_ROWS phase; the leaves' near field is in nearv;
// the leaf item computes its parent's L itself (the parent's rows summed
// earlier, plus L2L of the grandparent's L: its rows at level 2, else Lc), so
// that no downward phase of level L - 1 is needed
constexpr int DOWN_ROWS_PRE = 1, DOWN_NEAR_PRE = 2, DOWN_PARENT = 4;
constexpr int BO_MAX_PH = 12, BO_MAX_SEG = 4, BO_MAX_NG = 5;
constexpr int BO_CHUNK = 32;  // pairs per product item (the pair lists' chunk size)

// product groups per CTA of a configuration (R rows of RT groups per thread)
// and copy stages per group: two stages when at least four groups fit the
// shared memory that way, else one stage with as many groups as fit; at most
// BO_MAX_NG groups and 512 threads.  The launch bound follows, so that the
// smaller CTAs keep more registers.
__host__ __device__ constexpr int bo_fit(int R, int RT, int csz, int nst) {
  const int P = R * RT;  // largest P of the configuration
  const int gbytes = nst * (P * P + 32 * P) * csz;
  const int by_smem = (200 * 1024) / gbytes;
  const int by_thr = 512 / (RT * 8);
  const int n = by_smem < by_thr ? by_smem : by_thr;
  return n < BO_MAX_NG ? (n < 1 ? 1 : n) : BO_MAX_NG;
}
__host__ __device__ constexpr int bo_stages(int R, int RT, int csz) {
  return (bo_fit(R, RT, csz, 2) >= 4 || bo_fit(R, RT, csz, 2) == bo_fit(R, RT, csz, 1)) ? 2 : 1;
}
__host__ __device__ constexpr int bo_groups(int R, int RT, int csz) { return bo_fit(R, RT, csz, bo_stages(R, RT, csz)); }

struct BoSeg {
  int type, level, first, count;
};
struct BoPhase {
  int nseg;
  BoSeg seg[BO_MAX_SEG];
};

constexpr int BO_MAX_LEAF_PTS = 64;  // panels of one leaf held in shared memory
constexpr int BO_MAX_M = 128;        // longest GMRES cycle run inside the kernel

template <typename T, typename IO>
struct BoArgs {
  const IO* x;       // input, original boundary order
  IO* y;             // output, original boundary order
  T scale;           // weights q = scale x
  const int* skip;   // when set and nonzero the kernel returns at once
  int P, L, nb, ng;  // coefficients, leaf level, boundary points, thread groups per CTA
  int nst;           // copy stages per product group (1 or 2)
  T k;
  C<T> sig;          // self coefficient per unit weight
  // boundary points in sorted (leaf-Morton) order
  const int* borig;  // -> original boundary index
  const int2* bcode; // lattice offset codes: {x fastest, y fastest}
  const int* bxf;    // 1 for panels of the x faces
  const int* bfirst; // [8^L + 1] first sorted-boundary index of each leaf
  const C<T>* Rb;    // basis table of the boundary points [nb][P]
  C<T>* qb;          // weights in sorted order (written by the first phase)
  const C<T>* tab;   // lattice kernel half table
  // near field: per boundary leaf (index into the level-L active list) the
  // sorted indices of the panels of its near leaves
  const int* nsrc_ptr;
  const int* nsrc;
  // items of SEG_NEAR: {leaf index, first and end panel within the leaf},
  // the costliest first
  const int4* near_items;
  int64_t tab_len;   // entries of the kernel table
  // the multipoles M as a 2-D tensor (rows of 2P reals) for the TMA gathers
  // of the product items' source rows
  CUtensorMap mrows;
  C<T>* nearv;       // [nb] near field + self term (SEG_NEAR)
  // tree arrays
  const int* flags;
  int64_t loff[HFMM_MAX_LEVEL + 2];
  const int* act;    // active boundary cells, per level at loff[l]
  const int2* rng;   // pair range of each boundary cell, at loff[l] + cell
  C<T>* M;
  C<T>* Lc;
  const C<T>* m2m;   // [level][8][P][P] column-major
  const C<T>* l2l;
  const C<T>* m2l;   // [level][slot][P][P] row-major
  int64_t box_cells;
  // pairs
  const int4* chunks;  // {level, slot, first (grouped), count}
  const int* grouped;  // pair index of each grouped position
  const int* crow;     // [chunk][32] row of M of each column's source (-1: no pair)
  const int* cpid;     // [chunk][32] pair (product row) of each column
  const int* psrc;     // source cell of each pair
  const int* pslot;    // operator slot of each pair
  C<T>* buf;           // [npairs][P] products
  unsigned* bar;       // grid barrier words: count, generation, abort, exits
  // one GMRES cycle of the inner solve inside the kernel (cycle != 0): the
  // Krylov vectors in sorted order, the Arnoldi/Givens state in FP64
  int cycle, m;
  double rtol;
  const IO* b;         // right-hand side, original order
  IO* xout;            // solution of the cycle, original order
  C<T>* Vc;            // [m + 1][nb] basis, sorted order
  C<T>* wc;            // [nb] operator output, sorted order
  double2* part;       // [3][m + 2][gridDim] partial sums of the CTAs, one buffer per pass
  double2* dots;       // [2][m + 1] Gram-Schmidt coefficients of the current step, then
                       // ||w||^2 before them
  double2* H;          // [m][m + 1] Hessenberg columns (after the rotations)
  double* cs;          // [m] Givens cosines
  double2* sn;         // [m] Givens sines
  double2* gv;         // [m + 1] rotated right-hand side
  double* scal;        // [0] ||b||, [1] relative residual, [2] breakdown
  int* cflags;         // [0] done, [1] steps of the cycle, [2] steps summed over cycles
  size_t smem_bytes;   // dynamic shared memory of the launch
  int stage_l2l, stage_tab;  // the leaf level's downward items read these from shared memory
  int near_win;              // near sources staged per group (0: read from global memory)
  int nphase;
  BoPhase ph[BO_MAX_PH];
};

__device__ int g_bo_error;  // HFMM_ERR_TIMEOUT recorded by a bounded wait

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// grid barrier over all CTAs (co-resident: cooperative launch); false when a
// CTA gave up waiting (time-out or another CTA's abort).  bar[0] counts
// arrivals over the whole launch: barrier number `gen` (1, 2, ...) is passed
// once it reaches gen x gridDim.x, so no word needs a reset between barriers.
__device__ __forceinline__ void red_release(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ bool bo_grid_sync(unsigned* bar, unsigned& gen) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    gen += 1;
    const unsigned target = gen * gridDim.x;
    __threadfence();  // the CTA's writes of this phase, ordered before the arrival
    red_release(&bar[0], 1u);
    if ((int)(ld_acquire(&bar[0]) - target) < 0) {
      const uint64_t t0 = tc_now();
      for (int it = 0;; ++it) {
        if ((int)(ld_acquire(&bar[0]) - target) >= 0) break;
        if ((it & 63) == 63) {
          if (ld_acquire(&bar[2]) != 0u) {
            ok = 0;
            break;
          }
          if (tc_now() - t0 > 1000000000ull) {
            atomicExch(&g_bo_error, HFMM_ERR_TIMEOUT);
            atomicExch(&bar[2], 1u);
            ok = 0;
            break;
          }
        }
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// the last CTA to leave resets the barrier words and the item counters
// (bar[4 ...]) for the next launch
__device__ void bo_exit(unsigned* bar) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&bar[3], 1u) == gridDim.x - 1) {
      bar[0] = 0u;
      bar[2] = 0u;
      for (int i = 0; i < BO_MAX_PH * BO_MAX_SEG; ++i) bar[4 + i] = 0u;
      __threadfence();
      bar[3] = 0u;
    }
  }
}

template <typename T>
__device__ __forceinline__ C<T> ldcg(const C<T>* p);
template <>
__device__ __forceinline__ float2 ldcg<float>(const float2* p) { return __ldcg(p); }
template <>
__device__ __forceinline__ double2 ldcg<double>(const double2* p) { return __ldcg(p); }

// two consecutive complex values of data written earlier in this kernel
__device__ __forceinline__ void ldcg2(const float2* p, float2& a, float2& b) {
  const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
  a = make_float2(v.x, v.y);
  b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void ldcg2(const double2* p, double2& a, double2& b) {
  a = __ldcg(p);
  b = __ldcg(p + 1);
}

template <typename T>
__device__ __forceinline__ C<T> to_c(float2 v) { return mkc<T>(T(v.x), T(v.y)); }
template <typename T>
__device__ __forceinline__ C<T> to_c(double2 v) { return mkc<T>(T(v.x), T(v.y)); }
__device__ __forceinline__ void store_io(float2* y, int64_t i, float2 v) { y[i] = v; }
__device__ __forceinline__ void store_io(double2* y, int64_t i, float2 v) { y[i] = make_double2(v.x, v.y); }
__device__ __forceinline__ void store_io(double2* y, int64_t i, double2 v) { y[i] = v; }

// weight of sorted boundary point i, from the input vector
template <typename T, typename IO>
__device__ __forceinline__ C<T> weight(const BoArgs<T, IO>& A, int i) {
  const C<T> v = to_c<T>(A.x[A.borig[i]]);
  return mkc<T>(A.scale * v.x, A.scale * v.y);
}


// named barriers: 1 .. BO_MAX_NG for the thread groups of the product and
// downward items, 8 and 9 for the two teams of the upward items
__device__ __forceinline__ void group_sync(int g, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(nthreads) : "memory");
}
struct BoTeam {
  int tid, nthr, bid;
  __device__ void sync() const { asm volatile("bar.sync %0, %1;" ::"r"(bid), "r"(nthr) : "memory"); }
};

// M_parent = sum over the children o holding panels of T_o M_child (T column-
// major); Mc[8][P] staged children (zero rows for children without panels),
// part[8][P] scratch; all CTA threads
template <typename T>
__device__ void bo_m2m_into(const C<T>* __restrict__ ops, int P, const C<T>* Mc, const unsigned hasmask,
                            C<T>* part, C<T>* out, const BoTeam& tm) {
  const int nt = tm.nthr;
  for (int e = tm.tid; e < 8 * P; e += nt) {
    const int o = e / P, ap = e - o * P;
    C<T> acc = mkc<T>(0, 0);
    if ((hasmask >> o) & 1u) {
      const C<T>* Tc = ops + (int64_t)o * P * P + ap;
      const C<T>* xv = Mc + o * P;
#pragma unroll 12
      for (int a = 0; a < P; ++a) cfma<T>(acc, __ldg(Tc + (int64_t)a * P), xv[a]);
    }
    part[e] = acc;
  }
  tm.sync();
  for (int ap = tm.tid; ap < P; ap += nt) {
    C<T> s = mkc<T>(0, 0);
    for (int o = 0; o < 8; ++o) s = cadd<T>(s, part[o * P + ap]);
    out[ap] = s;
  }
}

// team item SEG_P2M_UP / SEG_P2M: the weights of the item's panels (sorted
// order, written to qb for the near field), P2M of the children (or of the
// leaf itself) and, for P2M_UP, M2M into the parent.  The children of a cell
// are consecutive leaves, so their panels are one sorted range.
template <typename T, typename IO>
__device__ void bo_p2m(const BoArgs<T, IO>& A, int level, int idx, bool up, unsigned char* sm, int* cb,
                       const BoTeam& tm, const C<T>* xsrc, T xs) {
  const int P = A.P, nt = tm.nthr;
  C<T>* Mc = reinterpret_cast<C<T>*>(sm);  // [8][P]
  C<T>* part = Mc + 8 * P;                 // [8][P]
  C<T>* wq = part + 8 * P;                 // [8 * BO_MAX_LEAF_PTS]
  const int cell = A.act[A.loff[level] + idx];
  const int L = A.L;
  const int nch = up ? 8 : 1;
  const int leaf0 = up ? 8 * cell : cell;
  if (tm.tid <= nch) cb[tm.tid] = A.bfirst[leaf0 + tm.tid];
  tm.sync();
  const int base = cb[0], np = cb[nch] - base;
  for (int e = tm.tid; e < np; e += nt) {
    C<T> w;
    if (xsrc) {  // inside a GMRES cycle: the sorted-order vector, scaled
      const C<T> v = ldcg<T>(xsrc + base + e);
      w = mkc<T>(A.scale * xs * v.x, A.scale * xs * v.y);
    } else {
      w = weight(A, base + e);
    }
    wq[e] = w;
    A.qb[base + e] = w;
  }
  unsigned hasmask = 0;
  for (int o = 0; o < nch; ++o)
    if (cb[o + 1] > cb[o]) hasmask |= 1u << o;
  tm.sync();
  for (int e = tm.tid; e < nch * P; e += nt) {
    const int o = e / P, a = e - o * P;
    const int lo = cb[o] - base, hi = cb[o + 1] - base;
    C<T> acc = mkc<T>(0, 0);
#pragma unroll 8
    for (int i = lo; i < hi; ++i) cfma_conj<T>(acc, __ldg(A.Rb + (int64_t)(base + i) * P + a), wq[i]);
    Mc[e] = acc;
    if (hi > lo) A.M[(A.loff[L] + leaf0 + o) * P + a] = acc;
  }
  tm.sync();
  if (up)
    bo_m2m_into<T>(A.m2m + (int64_t)level * 8 * P * P, P, Mc, hasmask, part, A.M + (A.loff[level] + cell) * P,
                   tm);
  tm.sync();
}

// team item SEG_M2M: parent at `level` from its children at level + 1
template <typename T, typename IO>
__device__ void bo_m2m(const BoArgs<T, IO>& A, int level, int idx, unsigned char* sm, const BoTeam& tm) {
  const int P = A.P, nt = tm.nthr;
  C<T>* Mc = reinterpret_cast<C<T>*>(sm);
  C<T>* part = Mc + 8 * P;
  const int cell = A.act[A.loff[level] + idx];
  const int64_t coff = A.loff[level + 1] + 8 * (int64_t)cell;
  unsigned hasmask = 0;
  for (int o = 0; o < 8; ++o)
    if (A.flags[coff + o] & HFMM_SET_BND) hasmask |= 1u << o;
  for (int e = tm.tid; e < 8 * P; e += nt) {
    const int o = e / P;
    Mc[e] = ((hasmask >> o) & 1u) ? ldcg<T>(A.M + coff * P + e) : mkc<T>(0, 0);
  }
  tm.sync();
  bo_m2m_into<T>(A.m2m + (int64_t)level * 8 * P * P, P, Mc, hasmask, part, A.M + (A.loff[level] + cell) * P,
                 tm);
  tm.sync();
}

// L (P values in shared memory) of the boundary leaf `leaf` to its panels,
// y = i k sum_a L_a R_ia + near; `nthr` threads (a multiple of 32), thread
// index tl, in groups of 4 lanes per panel
template <typename T, typename IO>
__device__ void bo_l2p(const BoArgs<T, IO>& A, int leaf, const C<T>* Lv, const C<T>* nearg, bool near_global,
                       int tl, int nthr) {
  const int P = A.P;
  const int lo = A.bfirst[leaf], hi = A.bfirst[leaf + 1];
  const int sub = tl & 3, grp = tl >> 2, ngrp = nthr >> 2;
  for (int ib = lo; ib < hi; ib += ngrp) {
    const int i = ib + grp;
    const bool act = i < hi;
    C<T> acc = mkc<T>(0, 0);
    if (act) {
      const C<T>* Ri = A.Rb + (int64_t)i * P;
#pragma unroll 4
      for (int a = sub; a < P; a += 4) cfma<T>(acc, Lv[a], __ldg(Ri + a));
    }
#pragma unroll
    for (int o = 2; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (act && sub == 0) {
      // the near field: this kernel's global buffer (read past L1), or the
      // group's shared scratch
      const C<T> nv = near_global ? ldcg<T>(nearg + (i - lo)) : nearg[i - lo];
      // i k acc + near
      const C<T> v = mkc<T>(-A.k * acc.y + nv.x, A.k * acc.x + nv.y);
      if (A.cycle)
        A.wc[i] = v;
      else
        store_io(A.y, A.borig[i], v);
    }
  }
}

// near field of the panels of one boundary leaf (index idx in the leaf
// level's active list) through the lattice kernel table, plus the self term,
// into nearg[panel - first panel of the leaf].  The warps of a group take
// blocks of TB targets; lanes stride the leaf's near sources; warp sums in a
// fixed tree.  G depends on |d| only, so a pair may use any axis order for
// its offset code as long as both points use the same one: a target on an x
// face takes the code with y fastest, which keeps a warp's table reads in
// consecutive entries (panels of an x face run along y).
// staged near-field source: weight and both offset codes
template <typename T> struct BoNs;
template <> struct BoNs<float> { float4 v; };                          // q.x, q.y, code x, code y (bits)
template <> struct BoNs<double> { double2 q; int2 c; int pad[2]; };
__device__ __forceinline__ void bo_ns_put(BoNs<float>& d, float2 q, int2 c) {
  d.v = make_float4(q.x, q.y, __int_as_float(c.x), __int_as_float(c.y));
}
__device__ __forceinline__ void bo_ns_put(BoNs<double>& d, double2 q, int2 c) {
  d.q = q;
  d.c = c;
}
__device__ __forceinline__ void bo_ns_get(const BoNs<float>& d, float2& q, int2& c) {
  const float4 v = d.v;
  q = make_float2(v.x, v.y);
  c = make_int2(__float_as_int(v.z), __float_as_int(v.w));
}
__device__ __forceinline__ void bo_ns_get(const BoNs<double>& d, double2& q, int2& c) {
  q = d.q;
  c = d.c;
}

template <typename T, typename IO>
__device__ void bo_near(const BoArgs<T, IO>& A, int idx, int leaf, C<T>* nearg, const C<T>* tab, BoNs<T>* ns_st,
                        int g, int tg, int GT, int t0 = 0, int t1 = -1) {
  constexpr int TB = 6;
  const int lane = tg & 31, wg = tg >> 5, nwg = GT >> 5;
  // panels [t0, t1) of the leaf (t1 < 0: all); nearg is indexed from the leaf's first panel
  const int tall = A.bfirst[leaf + 1] - A.bfirst[leaf];
  const int tlo = A.bfirst[leaf] + t0, nt = (t1 < 0 ? tall : t1) - t0;
  nearg += t0;
  const int s0 = A.nsrc_ptr[idx], s1 = A.nsrc_ptr[idx + 1], nsrc = s1 - s0;
  const bool staged = ns_st && nsrc <= A.near_win;
  if (staged) {  // the leaf's sources into shared memory, in batches of loads
    constexpr int NB = 4;
    for (int e0 = tg; e0 < nsrc; e0 += NB * GT) {
      int js[NB];
#pragma unroll
      for (int u = 0; u < NB; ++u) js[u] = e0 + u * GT < nsrc ? A.nsrc[s0 + e0 + u * GT] : -1;
      C<T> q[NB];
      int2 c[NB];
#pragma unroll
      for (int u = 0; u < NB; ++u)
        if (js[u] >= 0) {
          q[u] = ldcg<T>(A.qb + js[u]);
          c[u] = A.bcode[js[u]];
        }
#pragma unroll
      for (int u = 0; u < NB; ++u)
        if (js[u] >= 0) bo_ns_put(ns_st[e0 + u * GT], q[u], c[u]);
    }
    group_sync(g, GT);
  }
  for (int b0 = wg * TB; b0 < nt; b0 += nwg * TB) {
    int lt[TB];
    bool xa[TB];
    C<T> acc[TB];
#pragma unroll
    for (int j = 0; j < TB; ++j) {
      const int t = tlo + min(b0 + j, nt - 1);
      const int2 c = A.bcode[t];
      xa[j] = A.bxf[t] != 0;
      lt[j] = xa[j] ? c.y : c.x;
      acc[j] = mkc<T>(0, 0);
    }
    if (staged) {
#pragma unroll 2
      for (int e = lane; e < nsrc; e += 32) {
        C<T> q;
        int2 c;
        bo_ns_get(ns_st[e], q, c);
#pragma unroll
        for (int j = 0; j < TB; ++j) cfma<T>(acc[j], tab[abs(lt[j] - (xa[j] ? c.y : c.x))], q);
      }
    } else {
#pragma unroll 2
      for (int e = s0 + lane; e < s1; e += 32) {
        const int js = A.nsrc[e];
        const C<T> q = ldcg<T>(A.qb + js);
        const int2 c = A.bcode[js];
#pragma unroll
        for (int j = 0; j < TB; ++j) cfma<T>(acc[j], tab[abs(lt[j] - (xa[j] ? c.y : c.x))], q);
      }
    }
    C<T> mine = mkc<T>(0, 0);
#pragma unroll
    for (int j = 0; j < TB; ++j) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        acc[j].x += __shfl_xor_sync(0xffffffffu, acc[j].x, o);
        acc[j].y += __shfl_xor_sync(0xffffffffu, acc[j].y, o);
      }
      if (lane == j) mine = acc[j];
    }
    if (lane < TB && b0 + lane < nt) {
      cfma<T>(mine, A.sig, ldcg<T>(A.qb + tlo + b0 + lane));
      nearg[b0 + lane] = mine;
    }
  }
}

// sum of the product rows [r.x, r.y) for the coefficients of this thread
// (GT threads: S = GT / (P / 2) splits of the rows, two coefficients each)
template <typename T, typename IO>
__device__ void bo_rows(const BoArgs<T, IO>& A, int2 r, C<T>* part, int tg, int S) {
  const int P = A.P, P2 = P / 2;
  if (tg < S * P2) {
    const int sp = tg / P2, a2 = 2 * (tg - sp * P2);
    C<T> s0 = mkc<T>(0, 0), s1 = mkc<T>(0, 0);
    // batches of NB rows: all NB loads issued before the first add
    constexpr int NB = 8;
    for (int q0 = r.x + sp; q0 < r.y; q0 += NB * S) {
      C<T> v0[NB], v1[NB];
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        const int q = q0 + u * S;
        if (q < r.y) {
          ldcg2(A.buf + (int64_t)q * P + a2, v0[u], v1[u]);
        } else {
          v0[u] = mkc<T>(0, 0);
          v1[u] = mkc<T>(0, 0);
        }
      }
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        s0 = cadd<T>(s0, v0[u]);
        s1 = cadd<T>(s1, v1[u]);
      }
    }
    part[sp * P + a2] = s0;
    part[sp * P + a2 + 1] = s1;
  }
}

// group item SEG_DOWN: L of a cell at `level` = L2L of its parent's L + the
// sum of its own product rows (pair order).  At level 3 the parent's L (level
// 2, no parent of its own) is the sum of the parent's rows, formed here; at
// level 2 (leaf level 2 only) there is no L2L.  At the leaf level also the
// near field of the leaf's panels and L2P.  The L2L operators and the kernel
// table come from shared memory when the kernel staged them there.
template <typename T, typename IO>
__device__ void bo_down(const BoArgs<T, IO>& A, int level, int idx, int flags, C<T>* gsm, int g, int tg, int GT,
                        const C<T>* l2l_sm, const C<T>* tab, BoNs<T>* ns_st) {
  const int P = A.P, P2 = P / 2;
  const int S = GT / P2;
  C<T>* part = gsm;          // [S][P] own rows
  C<T>* pp = part + S * P;   // [S][P] the level-2 parent's rows
  C<T>* Lp = pp + S * P;     // parent L
  C<T>* Lv = Lp + P;
  C<T>* nearg = Lv + P;      // [BO_MAX_LEAF_PTS] near field of the leaf's panels
  const int cell = A.act[A.loff[level] + idx];
  const int parent = cell >> 3, o = cell & 7;
  const bool rows_pre = (flags & DOWN_ROWS_PRE) != 0;
  if (rows_pre) {  // the row sum is in L already: one "split"
    for (int a = tg; a < P; a += GT) part[a] = ldcg<T>(A.Lc + (A.loff[level] + cell) * P + a);
  } else {
    bo_rows<T, IO>(A, A.rng[A.loff[level] + cell], part, tg, S);
  }
  if (flags & DOWN_PARENT) {
    // the parent's L: its row sum (Lc, from an earlier row-sum phase) plus
    // L2L of the grandparent's L (into Lv as scratch)
    const int pl = level - 1, gp = parent >> 3, op = parent & 7;
    if (pl - 1 == 2) bo_rows<T, IO>(A, A.rng[A.loff[2] + gp], pp, tg, S);
    else
      for (int a = tg; a < P; a += GT) Lv[a] = ldcg<T>(A.Lc + (A.loff[pl - 1] + gp) * P + a);
    group_sync(g, GT);
    if (pl - 1 == 2) {
      for (int a = tg; a < P; a += GT) {
        C<T> v = mkc<T>(0, 0);
        for (int sp = 0; sp < S; ++sp) v = cadd<T>(v, pp[sp * P + a]);
        Lv[a] = v;
      }
      group_sync(g, GT);
    }
    for (int ap = tg; ap < P; ap += GT) {
      C<T> acc = ldcg<T>(A.Lc + (A.loff[pl] + parent) * P + ap);
      const C<T>* Tc = A.l2l + ((int64_t)(pl - 1) * 8 + op) * P * P + ap;
#pragma unroll 12
      for (int a = 0; a < P; ++a) cfma<T>(acc, __ldg(Tc + (int64_t)a * P), Lv[a]);
      Lp[ap] = acc;
    }
  } else if (level == 3) {
    bo_rows<T, IO>(A, A.rng[A.loff[2] + parent], pp, tg, S);
  } else if (level > 3) {
    for (int a = tg; a < P; a += GT) Lp[a] = ldcg<T>(A.Lc + (A.loff[level - 1] + parent) * P + a);
  }
  group_sync(g, GT);
  if (level == 3 && !(flags & DOWN_PARENT)) {
    for (int a = tg; a < P; a += GT) {
      C<T> v = mkc<T>(0, 0);
      for (int sp = 0; sp < S; ++sp) v = cadd<T>(v, pp[sp * P + a]);
      Lp[a] = v;
    }
    group_sync(g, GT);
  }
  for (int ap = tg; ap < P; ap += GT) {
    C<T> acc = mkc<T>(0, 0);
    if (level > 2) {
      if (l2l_sm) {
        const C<T>* Tc = l2l_sm + (int64_t)o * P * P + ap;
#pragma unroll 12
        for (int a = 0; a < P; ++a) cfma<T>(acc, Tc[(int64_t)a * P], Lp[a]);
      } else {
        const C<T>* Tc = A.l2l + ((int64_t)(level - 1) * 8 + o) * P * P + ap;
#pragma unroll 12
        for (int a = 0; a < P; ++a) cfma<T>(acc, __ldg(Tc + (int64_t)a * P), Lp[a]);
      }
    }
    const int ns = rows_pre ? 1 : S;
    for (int sp = 0; sp < ns; ++sp) acc = cadd<T>(acc, part[sp * P + ap]);
    Lv[ap] = acc;
    if (level < A.L) A.Lc[(A.loff[level] + cell) * P + ap] = acc;
  }
  const bool near_pre = (flags & DOWN_NEAR_PRE) != 0;
  if (level == A.L && !near_pre) bo_near<T, IO>(A, idx, cell, nearg, tab, ns_st, g, tg, GT);
  group_sync(g, GT);
  if (level == A.L) bo_l2p<T, IO>(A, cell, Lv, near_pre ? A.nearv + A.bfirst[cell] : nearg, near_pre, tg, GT);
  group_sync(g, GT);
}

// group item SEG_ROWS: the sum of a cell's product rows (pair order), stored
// as its L for the downward item of its level to complete
template <typename T, typename IO>
__device__ void bo_rows_item(const BoArgs<T, IO>& A, int level, int idx, C<T>* gsm, int g, int tg, int GT) {
  const int P = A.P, S = GT / (P / 2);
  C<T>* part = gsm;
  const int cell = A.act[A.loff[level] + idx];
  bo_rows<T, IO>(A, A.rng[A.loff[level] + cell], part, tg, S);
  group_sync(g, GT);
  for (int ap = tg; ap < P; ap += GT) {
    C<T> acc = mkc<T>(0, 0);
    for (int sp = 0; sp < S; ++sp) acc = cadd<T>(acc, part[sp * P + ap]);
    A.Lc[(A.loff[level] + cell) * P + ap] = acc;
  }
  group_sync(g, GT);
}

// products of one staged chunk for the first J column groups (J x 8 pairs)
template <typename T, typename IO, int R, int J, int RT>
__device__ __forceinline__ void bo_prod_cols(const BoArgs<T, IO>& A, const C<T>* Ts, const C<T>* Ms,
                                             const int* pids, int cw, int r0, int c0) {
  constexpr int CT = 8;
  const int P = A.P, MS = P;
  int pid[J];
#pragma unroll
  for (int q = 0; q < J; ++q) {
    const int c = c0 + q * CT;
    pid[q] = c < cw ? pids[c] : -1;
  }
  C<T> acc[R][J];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int q = 0; q < J; ++q) acc[r][q] = mkc<T>(0, 0);
  m2l_block_product<T, R, J, RT>(Ts, Ms, P, MS, r0, c0, acc);
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int q = 0; q < J; ++q) {
      const int ap = r0 + r * RT;
      if (ap < P && pid[q] >= 0) A.buf[(int64_t)pid[q] * P + ap] = acc[r][q];
    }
}

// records of a product chunk in shared memory: the header {level, slot,
// first, count}, the pair (product row) and the source row of each column
struct __align__(16) BoRec {
  int4 ch;
  int pid[BO_CHUNK];
  int row[BO_CHUNK];
};
constexpr int BO_NBAR = 5;  // mbarriers per group: two stages, three record slots

// group items SEG_PROD: chunk i of [first, first + count) -> buf rows, per
// group of GT = RT * 8 threads.  Every copy completes on an mbarrier: the
// records of the item three ahead (bulk copies) into one of three record
// slots, and for the item NST ahead the operator (one bulk copy) and the
// source rows (TMA gathers of four rows each, from the records, issued by
// the first lanes of the group's first warp) into one of NST stages, so that
// all latencies overlap the products of the current item.  Source rows sit
// at a stride of P in a stage (4 P elements = 32 P or 64 P bytes, a multiple
// of 128 for even p, so every gather lands on a 128-byte boundary).  Every
// thread of the group waits for each completion it reads (and all track the
// barriers' phases alike).  Returns false on a wait time-out.
template <typename T, typename IO, int R, int CM, int RT>
__device__ bool bo_products(const BoArgs<T, IO>& A, const BoSeg& sg, unsigned char* sm, uint64_t* mbar,
                            uint32_t& phase_bits, int* gabort, BoRec (*rec)[3]) {
  constexpr int GT = RT * 8, CT = 8, TC = CT * CM;
  static_assert(TC == BO_CHUNK, "one product column per pair of a chunk");
  static_assert(BO_NBAR * BO_MAX_NG <= 32, "phase bits of every group in one word");
  const int P = A.P, MS = P;
  const int g = threadIdx.x / GT, tg = threadIdx.x - g * GT;
  if (g >= A.ng) return true;
  const size_t op_elems = (size_t)P * P, ms_elems = (size_t)TC * MS;
  const int NST = A.nst;
  C<T>* base = reinterpret_cast<C<T>*>(sm) + (size_t)g * NST * (op_elems + ms_elems);
  uint64_t* bar = mbar + BO_NBAR * g;  // [0, 2): stages, [2, 5): record slots
  const int gid = blockIdx.x * A.ng + g, ngt = gridDim.x * A.ng;
  const int nitems = gid < sg.count ? (sg.count - gid + ngt - 1) / ngt : 0;
  const uint32_t op_bytes = (uint32_t)(op_elems * sizeof(C<T>));
  const uint32_t row_bytes = (uint32_t)(P * sizeof(C<T>));
  auto bit = [&](int k) { return 1u << (BO_NBAR * g + k); };
  auto par = [&](int k) { return (phase_bits & bit(k)) ? 1u : 0u; };
  uint32_t pending = 0;  // barriers with a phase issued and not yet consumed
  auto fail = [&]() {
    atomicExch(&g_bo_error, HFMM_ERR_TIMEOUT);
    *(volatile int*)&gabort[g] = 1;
  };
  // records of item j into slot j % 3
  auto rec_issue = [&](int j) {
    if (j >= nitems) return;
    const int s = j % 3, it = sg.first + gid + j * ngt;
    if (tg == 0) {
      uint64_t* rb = &bar[2 + s];
      tc_expect_tx(rb, (uint32_t)sizeof(BoRec));
      tc_bulk_g2s(&rec[g][s].ch, A.chunks + it, 16, rb);
      tc_bulk_g2s(rec[g][s].pid, A.cpid + (int64_t)it * TC, 4 * TC, rb);
      tc_bulk_g2s(rec[g][s].row, A.crow + (int64_t)it * TC, 4 * TC, rb);
    }
    pending |= bit(2 + s);
  };
  // operator and source rows of item j into stage j % NST (the first warp
  // waits for the records of item j without consuming that phase)
  auto stage_issue = [&](int j) {
    if (j >= nitems) return;
    const int st = j % NST, s = j % 3;
    if (tg < 32) {
      const bool ok = tc_wait(&bar[2 + s], par(2 + s));
      if (__all_sync(0xffffffffu, ok)) {
        C<T>* Ts = base + (size_t)st * (op_elems + ms_elems);
        C<T>* Ms = Ts + op_elems;
        const int4 ch = rec[g][s].ch;
        const int ngath = (ch.w + 3) >> 2;
        if (tg == 0) {
          tc_expect_tx(&bar[st], op_bytes + (uint32_t)ngath * 4u * row_bytes);
          tc_bulk_g2s(Ts, A.m2l + ((int64_t)ch.x * A.box_cells + ch.y) * P * P, op_bytes, &bar[st]);
        }
        __syncwarp();
        if (tg < ngath) {
          // rows past the chunk's width repeat its last row (never stored)
          const int* rw = rec[g][s].row;
          const int c0 = 4 * tg, last = ch.w - 1;
          tc_gather4(Ms + (size_t)c0 * MS, &A.mrows, 0, rw[c0], rw[min(c0 + 1, last)], rw[min(c0 + 2, last)],
                     rw[min(c0 + 3, last)], &bar[st]);
        }
      } else if (tg == 0) {
        fail();
      }
    }
    pending |= bit(st);
  };
  for (int j = 0; j < 3; ++j) rec_issue(j);
  for (int j = 0; j < NST; ++j) stage_issue(j);
  bool ok = true;
  for (int j = 0; j < nitems; ++j) {
    const int st = j % NST, s = j % 3;
    // every thread reads the records (width, pair rows) and the stage
    bool w = tc_wait(&bar[2 + s], par(2 + s));
    if (w) {
      phase_bits ^= bit(2 + s);
      pending &= ~bit(2 + s);
      w = tc_wait(&bar[st], par(st));
      if (w) {
        phase_bits ^= bit(st);
        pending &= ~bit(st);
      }
    }
    if (!w) fail();
    group_sync(g, GT);
    if (*(volatile int*)&gabort[g]) {
      ok = false;
      break;
    }
    C<T>* Ts = base + (size_t)st * (op_elems + ms_elems);
    C<T>* Ms = Ts + op_elems;
    const int cw = rec[g][s].ch.w;
    const int* pids = rec[g][s].pid;
    const int r0 = tg / CT, c0 = tg % CT;
    // only the column groups the chunk fills
    switch ((cw + CT - 1) / CT) {
      case 1: bo_prod_cols<T, IO, R, 1, RT>(A, Ts, Ms, pids, cw, r0, c0); break;
      case 2: bo_prod_cols<T, IO, R, 2, RT>(A, Ts, Ms, pids, cw, r0, c0); break;
      case 3: bo_prod_cols<T, IO, R, 3, RT>(A, Ts, Ms, pids, cw, r0, c0); break;
      default: bo_prod_cols<T, IO, R, CM, RT>(A, Ts, Ms, pids, cw, r0, c0); break;
    }
    group_sync(g, GT);  // stage st and record slot s are free again
    rec_issue(j + 3);
    stage_issue(j + NST);
  }
  if (!ok) {
    // copies still in flight after a time-out: let them land, bounded
    for (int k = 0; k < BO_NBAR; ++k)
      if (pending & bit(k)) tc_wait(&bar[k], par(k));
  }
  group_sync(g, GT);
  return ok;
}

// per-CTA state of the kernel (shared memory and the layout of the dynamic
// shared memory)
template <typename T>
struct BoCta {
  unsigned char* smem;
  uint64_t* mbar;
  int* gabort;
  BoRec (*rec)[3];
  int* gnext;        // [BO_MAX_NG] next item of each group (dynamic segments)
  int (*cbt)[9];
  unsigned gen;
  uint32_t phase_bits;
  unsigned napply;  // boundary applies finished in this launch
};

// the phases of one boundary -> boundary apply; xsrc / xs: the input inside a
// GMRES cycle (sorted order, times xs), null for the caller's vector.
// Returns false when a wait gave up.
template <typename T, typename IO, int R, int CM, int RT>
__device__ bool bo_apply_phases(const BoArgs<T, IO>& A, BoCta<T>& S, const C<T>* xsrc, T xs) {
  constexpr int GT = RT * 8;
  __shared__ int abort_s;
  if (threadIdx.x == 0) abort_s = 0;
  const int g = threadIdx.x / GT, tg = threadIdx.x - g * GT;
  const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int P = A.P;
  // two teams of whole warps for the upward items
  const int w0 = nwarp / 2, team = warp < w0 ? 0 : 1;
  const BoTeam tm{team ? (int)threadIdx.x - 32 * w0 : (int)threadIdx.x, team ? (int)blockDim.x - 32 * w0 : 32 * w0,
                  8 + team};
  const size_t team_elems = 16 * (size_t)P + 8 * BO_MAX_LEAF_PTS;
  unsigned char* team_sm = S.smem + (size_t)team * team_elems * sizeof(C<T>);
  // downward items: one scratch region per group, after the leaf level's
  // L2L operators and kernel table when those are staged; the group scratch
  // holds the downward sums, then the staged near sources (whole BoNs
  // records: the element count is rounded to their size)
  constexpr size_t NS_ELEMS = sizeof(BoNs<T>) / sizeof(C<T>);
  const size_t down_sums = ((size_t)(2 * (GT / (P / 2)) + 2) * P + BO_MAX_LEAF_PTS + NS_ELEMS - 1) / NS_ELEMS * NS_ELEMS;
  const size_t down_elems = down_sums + (size_t)A.near_win * NS_ELEMS;
  const size_t l2l_elems = 8 * (size_t)P * P;
  const size_t tab_elems = A.stage_tab ? (size_t)((A.tab_len + 1) & ~(int64_t)1) : 0;
  C<T>* l2l_st = reinterpret_cast<C<T>*>(S.smem);
  C<T>* tab_st = l2l_st + (A.stage_l2l ? l2l_elems : 0);
  C<T>* gsm = tab_st + tab_elems + (size_t)g * down_elems;
  __syncthreads();
  for (int ph = 0; ph < A.nphase; ++ph) {
    if (ph > 0 && !bo_grid_sync(A.bar, S.gen)) return false;
    const BoPhase& Ph = A.ph[ph];
    for (int si = 0; si < Ph.nseg; ++si) {
      const BoSeg sg = Ph.seg[si];
      switch (sg.type) {
        case SEG_PROD:
          if (!bo_products<T, IO, R, CM, RT>(A, sg, S.smem, S.mbar, S.phase_bits, S.gabort, S.rec))
            abort_s = 1;
          break;
        case SEG_DOWN:
        case SEG_ROWS:
        case SEG_NEAR: {
          const bool leaf = sg.type == SEG_DOWN && sg.level == A.L;
          const bool near = sg.type == SEG_NEAR || (leaf && !(sg.first & DOWN_NEAR_PRE));
          const C<T>* l2l_sm = nullptr;
          const C<T>* tab = A.tab;
          if ((leaf && A.stage_l2l) || (near && A.stage_tab)) {
            if (leaf && A.stage_l2l && sg.level > 2) {
              const float4* src = reinterpret_cast<const float4*>(A.l2l + (int64_t)(sg.level - 1) * l2l_elems);
              const int n4 = (int)(l2l_elems * sizeof(C<T>) / 16);
              for (int e = threadIdx.x; e < n4; e += blockDim.x) reinterpret_cast<float4*>(l2l_st)[e] = __ldg(src + e);
              l2l_sm = l2l_st;
            }
            if (near && A.stage_tab) {
              const float4* src = reinterpret_cast<const float4*>(A.tab);
              const int64_t n4 = A.tab_len * (int64_t)sizeof(C<T>) / 16;
              for (int64_t e = threadIdx.x; e < n4; e += blockDim.x)
                reinterpret_cast<float4*>(tab_st)[e] = __ldg(src + e);
              for (int64_t e = n4 * 16 / (int64_t)sizeof(C<T>) + threadIdx.x; e < A.tab_len; e += blockDim.x)
                tab_st[e] = A.tab[e];
              tab = tab_st;
            }
            __syncthreads();
          }
          BoNs<T>* ns_st = A.near_win ? reinterpret_cast<BoNs<T>*>(gsm + down_sums) : nullptr;
          // items handed out one at a time from a counter that grows by
          // count + (groups of the grid) per apply (every group takes one
          // index past the end): the item costs differ, and each item owns
          // its outputs, so results do not depend on which group runs it
          if (g < A.ng) {
            unsigned* ctr = A.bar + 4 + ph * BO_MAX_SEG + si;
            const unsigned base = S.napply * (unsigned)(sg.count + (int)gridDim.x * A.ng);
            if (tg == 0) S.gnext[g] = (int)(atomicAdd(ctr, 1u) - base);
            group_sync(g, GT);
            int i = S.gnext[g];
            while (i < sg.count) {
              unsigned nx = 0u;
              if (tg == 0) nx = atomicAdd(ctr, 1u);  // the next index, while this item runs
              if (sg.type == SEG_DOWN) {
                bo_down<T, IO>(A, sg.level, i, sg.first, gsm, g, tg, GT, l2l_sm, tab, ns_st);
              } else if (sg.type == SEG_ROWS) {
                bo_rows_item<T, IO>(A, sg.level, i, gsm, g, tg, GT);
              } else {
                const int4 it = A.near_items[i];
                const int leafc = A.act[A.loff[A.L] + it.x];
                bo_near<T, IO>(A, it.x, leafc, A.nearv + A.bfirst[leafc], tab, ns_st, g, tg, GT, it.y, it.z);
              }
              group_sync(g, GT);
              if (tg == 0) S.gnext[g] = (int)(nx - base);
              group_sync(g, GT);
              i = S.gnext[g];
            }
          }
          break;
        }
        default: {
          // inside a GMRES cycle CTA 0 also runs the Arnoldi update at the
          // start of each step: the upward items go to the other CTAs
          const int c0 = (A.cycle && gridDim.x > 1) ? 1 : 0;
          if ((int)blockIdx.x < c0) break;
          for (int i = 2 * ((int)blockIdx.x - c0) + team; i < sg.count; i += 2 * ((int)gridDim.x - c0)) {
            if (sg.type == SEG_P2M_UP) bo_p2m<T, IO>(A, sg.level, i, true, team_sm, S.cbt[team], tm, xsrc, xs);
            else if (sg.type == SEG_P2M) bo_p2m<T, IO>(A, sg.level, i, false, team_sm, S.cbt[team], tm, xsrc, xs);
            else if (sg.type == SEG_M2M) bo_m2m<T, IO>(A, sg.level, i, team_sm, tm);
          }
          break;
        }
      }
      __syncthreads();
      if (abort_s) {
        if (threadIdx.x == 0) atomicExch(&A.bar[2], 1u);
        return false;
      }
    }
  }
  S.napply += 1;
  return true;
}

// ---- the inner GMRES cycle (readings of the inner solve: unpreconditioned
//      GMRES from zero, classical Gram-Schmidt twice, complex Givens
//      rotations, stop on the residual estimate) with every vector operation
//      on this CTA's slice [lo, hi) of the sorted order and every reduction
//      over the CTAs' partial sums in CTA order (deterministic)

// sum over the CTAs of partial row k (one warp, fixed order)
__device__ __forceinline__ double2 bo_sum_part(const double2* part, int k, int ncta, int lane) {
  double x = 0.0, y = 0.0;
  for (int c = lane; c < ncta; c += 32) {
    const double2 v = __ldcg(&part[(int64_t)k * ncta + c]);
    x += v.x;
    y += v.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_xor_sync(0xffffffffu, x, o);
    y += __shfl_xor_sync(0xffffffffu, y, o);
  }
  return make_double2(x, y);
}

// partial rows k < nk: <V_k, w> over this CTA's slice (one warp per row), and
// with want_norm the row nk = ||w||^2
template <typename T, typename IO>
__device__ void bo_slice_dots(const BoArgs<T, IO>& A, double2* part, int nk, bool want_norm, int lo, int hi) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int rows = nk + (want_norm ? 1 : 0);
  // in the arithmetic of the form (T); the CTAs' sums are combined in FP64
  for (int k = warp; k < rows; k += nwarp) {
    T x = T(0), y = T(0);
#pragma unroll 4
    for (int e = lo + lane; e < hi; e += 32) {
      const C<T> b = ldcg<T>(A.wc + e);
      if (k < nk) {
        const C<T> a = ldcg<T>(A.Vc + (int64_t)k * A.nb + e);
        x += a.x * b.x + a.y * b.y;
        y += a.x * b.y - a.y * b.x;
      } else {
        x += b.x * b.x + b.y * b.y;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, o);
      y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    if (lane == 0) part[(int64_t)k * gridDim.x + blockIdx.x] = make_double2((double)x, (double)y);
  }
}

// coefficients d_k (k < nk) from the partial rows into shared memory (and,
// from CTA 0, into A.dots + doff for the Arnoldi column); then
// w -= sum_k d_k V_k on this CTA's slice
template <typename T, typename IO>
__device__ void bo_slice_project(const BoArgs<T, IO>& A, const double2* part, int nk, double2* dsm, int doff, int lo,
                                 int hi) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int k = warp; k < nk; k += nwarp) {
    const double2 d = bo_sum_part(part, k, gridDim.x, lane);
    if (lane == 0) {
      dsm[k] = d;
      if (blockIdx.x == 0) A.dots[doff + k] = d;
    }
  }
  __syncthreads();
  // four lanes per element, each a strided quarter of the k, combined in a
  // fixed tree
  const int sub = threadIdx.x & 3;
  for (int e0 = lo; e0 < hi; e0 += (int)(blockDim.x >> 2)) {
    const int e = e0 + (int)(threadIdx.x >> 2);
    const bool on = e < hi;
    T sx = T(0), sy = T(0);
    if (on) {
#pragma unroll 4
      for (int k = sub; k < nk; k += 4) {
        const C<T> v = ldcg<T>(A.Vc + (int64_t)k * A.nb + e);
        const T dx = T(dsm[k].x), dy = T(dsm[k].y);
        sx += dx * v.x - dy * v.y;
        sy += dx * v.y + dy * v.x;
      }
    }
    sx += __shfl_xor_sync(0xffffffffu, sx, 1);
    sy += __shfl_xor_sync(0xffffffffu, sy, 1);
    sx += __shfl_xor_sync(0xffffffffu, sx, 2);
    sy += __shfl_xor_sync(0xffffffffu, sy, 2);
    if (on && sub == 0) {
      const C<T> w = ldcg<T>(A.wc + e);
      A.wc[e] = mkc<T>(w.x - sx, w.y - sy);
    }
  }
  __syncthreads();
}

// Arnoldi column j (CTA 0): H(0:j, j) = d1 + d2, H(j+1, j) = hnext, the
// previous rotations, a new one (c = |a|/nu, s = (a/|a|) conj(b)/nu, c = 0
// and s = 1 when a = 0), the rotated right-hand side and the residual
// estimate; done when below rtol, on breakdown (hnext <= 1e-14 ||w||) or on a
// value that is not finite.  The column and the rotations are staged in
// shared memory by all threads; thread 0 runs the sequential part.
template <typename T, typename IO>
__device__ void bo_arnoldi(const BoArgs<T, IO>& A, int j, double hnext, double wnorm, C<T>* col, T* css,
                           C<T>* sns) {
  const int ld = A.m + 1;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    const double2 d1 = __ldcg(&A.dots[i]), d2 = __ldcg(&A.dots[ld + i]);
    col[i] = mkc<T>(T(d1.x + d2.x), T(d1.y + d2.y));
  }
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    css[i] = T(__ldcg(&A.cs[i]));
    const double2 v = __ldcg(&A.sn[i]);
    sns[i] = mkc<T>(T(v.x), T(v.y));
  }
  __shared__ double2 gj_s;
  __shared__ double bn_s;
  if (threadIdx.x == 32) {
    gj_s = __ldcg(&A.gv[j]);
    bn_s = __ldcg(&A.scal[0]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // in the arithmetic of the form (T)
    col[j + 1] = mkc<T>(T(hnext), T(0));
    for (int i = 0; i < j; ++i) {
      const C<T> a = col[i], b = col[i + 1];
      const T c = css[i];
      const C<T> sv = sns[i];
      col[i] = mkc<T>(c * a.x + sv.x * b.x - sv.y * b.y, c * a.y + sv.x * b.y + sv.y * b.x);
      col[i + 1] = mkc<T>(-(sv.x * a.x + sv.y * a.y) + c * b.x, -(sv.x * a.y - sv.y * a.x) + c * b.y);
    }
    const C<T> a = col[j], b = col[j + 1];
    const T aa = hypot(a.x, a.y);
    T c;
    C<T> sv;
    if (aa == T(0)) {
      c = T(0);
      sv = mkc<T>(T(1), T(0));
    } else {
      const T nu = sqrt(aa * aa + b.x * b.x + b.y * b.y);
      c = aa / nu;
      const C<T> ph = mkc<T>(a.x / aa, a.y / aa);
      const C<T> cb = mkc<T>(b.x / nu, -b.y / nu);
      sv = mkc<T>(ph.x * cb.x - ph.y * cb.y, ph.x * cb.y + ph.y * cb.x);
    }
    A.cs[j] = (double)c;
    A.sn[j] = make_double2((double)sv.x, (double)sv.y);
    col[j] = mkc<T>(c * a.x + sv.x * b.x - sv.y * b.y, c * a.y + sv.x * b.y + sv.y * b.x);
    col[j + 1] = mkc<T>(T(0), T(0));
    const C<T> gj = mkc<T>(T(gj_s.x), T(gj_s.y));
    const C<T> g1 = mkc<T>(-(sv.x * gj.x + sv.y * gj.y), -(sv.x * gj.y - sv.y * gj.x));
    A.gv[j + 1] = make_double2((double)g1.x, (double)g1.y);
    A.gv[j] = make_double2((double)(c * gj.x), (double)(c * gj.y));
    const double relres = (double)hypot(g1.x, g1.y) / bn_s;
    const bool brk = hnext <= 1e-14 * wnorm;
    A.scal[1] = relres;
    A.scal[2] = brk ? 1.0 : 0.0;
    A.cflags[1] = j + 1;
    if (relres < A.rtol || brk || !(relres == relres)) A.cflags[0] = 1;
  }
  __syncthreads();
  double2* Hc = A.H + (int64_t)j * ld;
  for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) Hc[i] = make_double2((double)col[i].x, (double)col[i].y);
}

template <typename T, typename IO, int R, int CM, int RT>
__device__ void bo_cycle(const BoArgs<T, IO>& A, BoCta<T>& S) {
  __shared__ double2 dsm[BO_MAX_M + 1];
  __shared__ C<T> colt[BO_MAX_M + 2];
  __shared__ T cssm[BO_MAX_M];
  __shared__ C<T> snsm[BO_MAX_M];
  __shared__ double hs[2];
  __shared__ int done_s;
  __shared__ int one_pass_s;
  bool analytic = false;    // the next step's norm is the one-pass value (no pass C)
  double next_norm2 = 0.0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nb = A.nb;
  const int lo = (int)((int64_t)nb * blockIdx.x / gridDim.x), hi = (int)((int64_t)nb * (blockIdx.x + 1) / gridDim.x);
  const int m = A.m;
  // partial-sum buffers: pass A (dots and ||w||^2 after the apply), pass B
  // (dots after the first projection), pass C (||w||^2 after the second)
  const int64_t pstride = (int64_t)(m + 2) * gridDim.x;
  double2* pA = A.part;
  double2* pB = A.part + pstride;
  double2* pC = A.part + 2 * pstride;
  // start: V_0 <- b (sorted order), ||b||^2 into pass C's row 0
  for (int e = lo + threadIdx.x; e < hi; e += blockDim.x) {
    const C<T> v = to_c<T>(A.b[A.borig[e]]);
    A.Vc[e] = v;
    A.wc[e] = v;
  }
  __syncthreads();
  bo_slice_dots<T, IO>(A, pC, 0, true, lo, hi);
  if (!bo_grid_sync(A.bar, S.gen)) return;
  int j = 0;
  for (;; ++j) {
    // the norm of w (||b|| at j = 0): v_j = w / norm on this slice, and (CTA
    // 0) the Arnoldi update of column j - 1 or the start of the cycle
    if (warp == 0) {
      const double2 s2 = analytic ? make_double2(next_norm2, 0.0) : bo_sum_part(pC, 0, gridDim.x, lane);
      if (lane == 0) {
        hs[0] = sqrt(s2.x);
        hs[1] = j > 0 && blockIdx.x == 0 ? sqrt(__ldcg(&A.dots[2 * (m + 1)]).x) : 0.0;
      }
    }
    __syncthreads();
    const double nrm = hs[0];
    if (blockIdx.x == 0) {
      if (j == 0) {
        for (int i = threadIdx.x; i <= m; i += blockDim.x) A.gv[i] = make_double2(i == 0 ? nrm : 0.0, 0.0);
        if (threadIdx.x == 0) {
          A.scal[0] = nrm;
          A.cflags[0] = (nrm > 0.0 && nrm < 1e300) ? 0 : 1;
          A.cflags[1] = 0;
        }
      } else {
        bo_arnoldi<T, IO>(A, j - 1, nrm, hs[1], colt, cssm, snsm);
      }
    }
    if (j >= m) break;
    const T inv = nrm > 0.0 ? T(1.0 / nrm) : T(0);
    for (int e = lo + threadIdx.x; e < hi; e += blockDim.x) {
      const C<T> w = ldcg<T>(A.wc + e);
      A.Vc[(int64_t)j * nb + e] = mkc<T>(w.x * inv, w.y * inv);
    }
    // the apply of v_j = w / norm (its first phase reads w, scaled); its
    // last phase overwrites w with the result
    if (!bo_apply_phases<T, IO, R, CM, RT>(A, S, A.wc, inv)) return;
    if (!bo_grid_sync(A.bar, S.gen)) return;
    // stop here when the Arnoldi update of column j - 1 (written by CTA 0
    // before the apply, visible after its barriers) ended the cycle
    if (threadIdx.x == 0) done_s = __ldcg(&A.cflags[0]);
    __syncthreads();
    if (done_s) break;
    // classical Gram-Schmidt with the reorthogonalization test of Daniel,
    // Gragg, Kaufman and Stewart: d1 = V^H w, w -= V d1; with V orthonormal
    // ||w||^2 = ||w0||^2 - |d1|^2, and when that keeps more than half of
    // ||w0||^2 one pass is enough (that norm serves the next step);
    // otherwise d2 = V^H w, w -= V d2 and ||w||^2 summed again.  The test is
    // taken on sums every CTA forms in the same order, so all agree.
    // ||w0||^2 also serves the breakdown test.
    bo_slice_dots<T, IO>(A, pA, j + 1, true, lo, hi);
    if (!bo_grid_sync(A.bar, S.gen)) return;
    if (warp == 0) {
      const double2 s2 = bo_sum_part(pA, j + 1, gridDim.x, lane);
      if (lane == 0) {
        hs[0] = s2.x;
        if (blockIdx.x == 0) A.dots[2 * (m + 1)] = s2;
      }
    }
    bo_slice_project<T, IO>(A, pA, j + 1, dsm, 0, lo, hi);
    if (threadIdx.x == 0) {
      double d2sum = 0.0;
      for (int k = 0; k <= j; ++k) d2sum += dsm[k].x * dsm[k].x + dsm[k].y * dsm[k].y;
      const double w1 = hs[0] - d2sum;
      one_pass_s = (w1 > 0.5 * hs[0]) ? 1 : 0;
      hs[1] = w1;
    }
    __syncthreads();
    if (one_pass_s) {
      if (blockIdx.x == 0)
        for (int k = threadIdx.x; k <= j; k += blockDim.x) A.dots[(m + 1) + k] = make_double2(0.0, 0.0);
      analytic = true;
      next_norm2 = hs[1];
      if (!bo_grid_sync(A.bar, S.gen)) return;
      continue;
    }
    analytic = false;
    bo_slice_dots<T, IO>(A, pB, j + 1, false, lo, hi);
    if (!bo_grid_sync(A.bar, S.gen)) return;
    bo_slice_project<T, IO>(A, pB, j + 1, dsm, m + 1, lo, hi);
    bo_slice_dots<T, IO>(A, pC, 0, true, lo, hi);
    if (!bo_grid_sync(A.bar, S.gen)) return;
  }
  // y = H(0:k, 0:k)^-1 g(0:k), k = steps done, by CTA 0; then x = V y
  if (!bo_grid_sync(A.bar, S.gen)) return;
  const int kdim = __ldcg(&A.cflags[1]);
  if (blockIdx.x == 0) {
    // the triangle and g staged by all threads (dynamic shared memory: the
    // apply's buffers are free here), then back substitution by thread 0
    // (in the arithmetic of the form)
    C<T>* Hs = reinterpret_cast<C<T>*>(S.smem);  // [kdim][kdim], column-major
    const int ld = m + 1;
    for (int e = threadIdx.x; e < kdim * kdim; e += blockDim.x) {
      const int c = e / kdim, r = e - c * kdim;
      const double2 h = r <= c ? __ldcg(&A.H[(int64_t)c * ld + r]) : make_double2(0.0, 0.0);
      Hs[e] = mkc<T>(T(h.x), T(h.y));
    }
    for (int i = threadIdx.x; i < kdim; i += blockDim.x) {
      const double2 gi = __ldcg(&A.gv[i]);
      colt[i] = mkc<T>(T(gi.x), T(gi.y));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int i = kdim - 1; i >= 0; --i) {
        C<T> acc = colt[i];
        for (int q = i + 1; q < kdim; ++q) {
          const C<T> h = Hs[(int64_t)q * kdim + i];
          const C<T> y = mkc<T>(T(dsm[q].x), T(dsm[q].y));
          acc.x -= h.x * y.x - h.y * y.y;
          acc.y -= h.x * y.y + h.y * y.x;
        }
        const C<T> d = Hs[(int64_t)i * kdim + i];
        const T den = d.x * d.x + d.y * d.y;
        dsm[i] = make_double2((double)((acc.x * d.x + acc.y * d.y) / den), (double)((acc.y * d.x - acc.x * d.y) / den));
      }
      A.cflags[2] += kdim;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kdim; i += blockDim.x) A.dots[i] = dsm[i];
  }
  if (!bo_grid_sync(A.bar, S.gen)) return;
  for (int i = threadIdx.x; i < kdim; i += blockDim.x) dsm[i] = __ldcg(&A.dots[i]);
  __syncthreads();
  for (int e = lo + threadIdx.x; e < hi; e += blockDim.x) {
    double x = 0.0, y = 0.0;
    for (int i = 0; i < kdim; ++i) {
      const C<T> v = ldcg<T>(A.Vc + (int64_t)i * nb + e);
      x += dsm[i].x * v.x - dsm[i].y * v.y;
      y += dsm[i].x * v.y + dsm[i].y * v.x;
    }
    store_io(A.xout, A.borig[e], mkc<T>(T(x), T(y)));
  }
}

template <typename T, typename IO, int R, int CM, int RT>
__global__ void __launch_bounds__(RT * 8 * bo_groups(R, RT, (int)sizeof(C<T>)), 1)
    k_bnd_op(const __grid_constant__ BoArgs<T, IO> A) {
  if (A.skip && *A.skip) return;
  extern __shared__ __align__(128) unsigned char bo_smem[];
  __shared__ __align__(8) uint64_t mbar[BO_NBAR * BO_MAX_NG];
  __shared__ int gabort[BO_MAX_NG];
  __shared__ BoRec rec[BO_MAX_NG][3];
  __shared__ int gnext[BO_MAX_NG];
  __shared__ int cbt[2][9];
  if (threadIdx.x == 0) {
    // per group: two stage barriers, three record slots (one expect-tx
    // arrival each)
    for (int i = 0; i < BO_NBAR * BO_MAX_NG; ++i) tc_mbar_init(&mbar[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int i = 0; i < BO_MAX_NG; ++i) gabort[i] = 0;
  }
  __syncthreads();
  BoCta<T> S{bo_smem, mbar, gabort, rec, gnext, cbt, 0u, 0u, 0u};
  if (A.cycle)
    bo_cycle<T, IO, R, CM, RT>(A, S);
  else
    bo_apply_phases<T, IO, R, CM, RT>(A, S, nullptr, T(1));
  bo_exit(A.bar);
}

}  // namespace

// ---------------------------------------------------------------- plan

struct bnd_op_state {
  int ok = 0;                 // 1: usable, -1: not for this tree
  int nb = 0, nbl = 0;
  int *borig = nullptr, *bxf = nullptr, *bfirst = nullptr;
  int2* bcode = nullptr;
  int *nsrc_ptr = nullptr, *nsrc = nullptr;
  int2* rng = nullptr;
  int *pslot = nullptr, *crow = nullptr, *cpid = nullptr;
  int4* near_items = nullptr;
  CUtensorMap mrows;       // the tree's multipoles as rows of 2P reals (TMA gathers)
  int near_win = 0;        // sources of a leaf's near field staged in shared memory (0: none)
  void* Rb = nullptr;     // basis rows of the boundary points, sorted order
  void* qb = nullptr;     // weights, sorted order
  int stage_l2l = 0, stage_tab = 0;
  void* nearv = nullptr;   // near field of the boundary points (sorted order)
  // workspace of the in-kernel GMRES cycle (sized for cyc_m steps)
  int cyc_m = 0;
  void *Vc = nullptr, *wc = nullptr;
  double2 *part = nullptr, *dots = nullptr, *H = nullptr, *sn = nullptr, *gv = nullptr;
  double *cs = nullptr, *scal = nullptr;
  int* cflags = nullptr;
  unsigned* bar = nullptr;
  int chunk_first[HFMM_MAX_LEVEL + 2] = {};
  int chunk_count[HFMM_MAX_LEVEL + 2] = {};
  int nphase = 0;
  BoPhase ph[BO_MAX_PH];
  int grid = 0, threads = 0, ng = 0, nst = 2;
  size_t smem = 0;
};

namespace {

template <typename X>
int to_host(std::vector<X>& h, const X* d, size_t n) {
  h.resize(n);
  if (n) HFMM_CUDA_TRY(cudaMemcpy(h.data(), d, n * sizeof(X), cudaMemcpyDeviceToHost));
  return HFMM_OK;
}
template <typename X>
int to_dev(fmm_tree* t, X** d, const std::vector<X>& h) {
  HFMM_TRY(tree_alloc_t(t, d, std::max<size_t>(1, h.size())));
  if (!h.empty()) HFMM_CUDA_TRY(cudaMemcpy(*d, h.data(), h.size() * sizeof(X), cudaMemcpyHostToDevice));
  return HFMM_OK;
}

// Rb[i][a] = R[bsort[i]][a]: the basis-table rows of the boundary points in
// sorted order (one-time)
template <typename T>
__global__ void k_bo_rows(int64_t nb, int P, const int* __restrict__ bsort, const C<T>* __restrict__ R,
                          C<T>* __restrict__ Rb) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nb * P) return;
  const int64_t i = e / P;
  const int a = (int)(e - i * P);
  Rb[e] = R[(int64_t)bsort[i] * P + a];
}

// kernel configuration per P (the pair-list M2L's register tiles)
struct BoCfg {
  int R, CM, RT;
};
inline bool bo_cfg(int P, BoCfg& c) {
  if (P <= 16) c = {1, 4, 16};
  else if (P <= 36) c = {3, 4, 12};
  else if (P <= 64) c = {4, 4, 16};
  else return false;
  return true;
}

template <typename T, typename IO, int R, int CM, int RT>
const void* bo_kernel() {
  return (const void*)k_bnd_op<T, IO, R, CM, RT>;
}

template <typename T, typename IO>
const void* bo_kernel_for(int P) {
  if (P <= 16) return bo_kernel<T, IO, 1, 4, 16>();
  if (P <= 36) return bo_kernel<T, IO, 3, 4, 12>();
  return bo_kernel<T, IO, 4, 4, 16>();
}

// phase table (see the file comment): the upward pass, then per level the
// M2L products as soon as its multipoles are complete (M2M one level up in
// the same phase) and the sums of a level's product rows in the phase after
// its products, then the downward items level by level; the near field with
// the level above the leaves (inside the leaf level's items when the tree is
// too shallow for that)
void bo_schedule(bnd_op_state* b, int L, int nact[], int chunk_first[], int chunk_count[]) {
  std::vector<std::vector<BoSeg>> phases;
  auto prod_seg = [&](int lhi, int llo) {  // product items of levels llo..lhi (contiguous chunks)
    int first = chunk_first[llo], cnt = 0;
    for (int l = llo; l <= lhi; ++l) cnt += chunk_count[l];
    return BoSeg{SEG_PROD, lhi, first, cnt};
  };
  int cur;  // lowest level whose multipoles are complete
  int plo, phi;  // product levels pending
  if (L == 2) {
    phases.push_back({BoSeg{SEG_P2M, 2, 0, nact[2]}});
    cur = plo = phi = 2;
  } else {
    phases.push_back({BoSeg{SEG_P2M_UP, L - 1, 0, nact[L - 1]}});
    cur = L - 1;
    plo = L - 1;
    phi = L;
  }
  std::vector<int> rows_pre(L + 1, 0);
  int rlo = 0, rhi = -1;  // levels whose rows are summed in the next phase
  while (true) {
    std::vector<BoSeg> ph{prod_seg(phi, plo)};
    for (int l = rhi; l >= std::max(3, rlo); --l) {
      ph.push_back(BoSeg{SEG_ROWS, l, 0, nact[l]});
      rows_pre[l] = 1;
    }
    rlo = plo;
    rhi = phi;
    if (cur == 2) {
      phases.push_back(ph);
      break;
    }
    ph.push_back(BoSeg{SEG_M2M, cur - 1, 0, nact[cur - 1]});
    phases.push_back(ph);
    --cur;
    plo = phi = cur;
  }
  // the near field needs only the sorted weights (phase 0): from L = 4 on it
  // runs after the first products, its items filling the groups that finish
  // their products early
  const bool near_early = L >= 4;
  if (near_early) phases[1].push_back(BoSeg{SEG_NEAR, L, 0, nact[L]});
  // from L = 4 on, with the rows of level L - 1 summed already, the leaves
  // compute their parents' L themselves: no downward phase for level L - 1
  const bool fold = near_early && rows_pre[L - 1];
  for (int l = (L == 2 ? 2 : 3); l <= L; ++l) {
    if (fold && l == L - 1) continue;
    const int fl = (rows_pre[l] ? DOWN_ROWS_PRE : 0) | (l == L && near_early ? DOWN_NEAR_PRE : 0) |
                   (l == L && fold ? DOWN_PARENT : 0);
    phases.push_back({BoSeg{SEG_DOWN, l, fl, nact[l]}});
  }
  b->nphase = (int)phases.size();
  for (size_t i = 0; i < phases.size(); ++i) {
    b->ph[i].nseg = (int)phases[i].size();
    for (size_t j = 0; j < phases[i].size(); ++j) b->ph[i].seg[j] = phases[i][j];
  }
}

int bo_plan(fmm_tree* t, bool fp32, cudaStream_t s) {
  if (t->bop) return t->bop->ok > 0 ? HFMM_OK : HFMM_ERR_UNSUPPORTED;
  bnd_op_state* b = new (std::nothrow) bnd_op_state();
  if (!b) return HFMM_ERR_NOMEM;
  t->bop = b;
  b->ok = -1;
  BoCfg cfg;
  const int L = t->L, P = t->P;
  if (!t->lattice || t->n_bnd == 0 || !t->rtab || t->lat_D <= 0 || !t->use_lattice_p2p || !bo_cfg(P, cfg) ||
      t->near_count > 128 || (t->p & 1) || L + 1 > BO_MAX_PH)
    return HFMM_ERR_UNSUPPORTED;
  if (!fp32 && !t->lat_tab64) return HFMM_ERR_UNSUPPORTED;
  int dev = 0, nsm = 0, coop = 0;
  HFMM_CUDA_TRY(cudaGetDevice(&dev));
  HFMM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  HFMM_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return HFMM_ERR_UNSUPPORTED;
  // pair lists of the boundary -> boundary pass (built on first use)
  HFMM_TRY(fmm_pair_lists(t, HFMM_SET_BND, HFMM_SET_BND, s));
  HFMM_CUDA_TRY(cudaStreamSynchronize(s));
  const int ci = (HFMM_SET_BND - 1) * 3 + (HFMM_SET_BND - 1);
  const int mi = HFMM_SET_BND - 1;
  const int64_t nleaf = (int64_t)1 << (3 * L);
  // sorted boundary points
  std::vector<int> ls, lm;
  std::vector<int64_t> orig;
  std::vector<double> xyz;
  HFMM_TRY(to_host(ls, t->leaf_start, nleaf + 1));
  HFMM_TRY(to_host(lm, t->leaf_mid, nleaf));
  HFMM_TRY(to_host(orig, t->orig, t->n_pts));
  HFMM_TRY(to_host(xyz, t->xyz, 3 * t->n_pts));
  const double inv_h = 1.0 / t->h;
  const int Sy = t->lat_Sy, Sz = t->lat_Sz;
  const int64_t nn = (int64_t)t->n * t->n;
  std::vector<int> borig, bsort, bxf, bfirst(nleaf + 1, 0);
  std::vector<int2> bcode;
  borig.reserve(t->n_bnd);
  for (int64_t leaf = 0; leaf < nleaf; ++leaf) {
    bfirst[leaf] = (int)bsort.size();
    for (int j = lm[leaf]; j < ls[leaf + 1]; ++j) {
      bsort.push_back(j);
      const int64_t ob = orig[j] - t->n_vol;
      borig.push_back((int)ob);
      bxf.push_back(ob < 2 * nn ? 1 : 0);  // faces x = 0 and x = 1 come first
      const int cx = (int)llrint(xyz[3 * j] * inv_h), cy = (int)llrint(xyz[3 * j + 1] * inv_h),
                cz = (int)llrint(xyz[3 * j + 2] * inv_h);
      bcode.push_back(make_int2(cx + Sy * cy + Sz * cz, cy + Sy * cz + Sz * cx));
    }
  }
  bfirst[nleaf] = (int)bsort.size();
  if ((int64_t)bsort.size() != t->n_bnd) return HFMM_ERR_UNSUPPORTED;
  for (int64_t leaf = 0; leaf < nleaf; ++leaf)
    if (bfirst[leaf + 1] - bfirst[leaf] > BO_MAX_LEAF_PTS) return HFMM_ERR_UNSUPPORTED;
  // active boundary cells per level and their pair ranges
  std::vector<int> act;
  HFMM_TRY(to_host(act, t->act_cells[mi], t->total_cells));
  int nact[HFMM_MAX_LEVEL + 1] = {};
  for (int l = 2; l <= L; ++l) nact[l] = t->act_count[mi][l];
  std::vector<int4> tiles;
  std::vector<int> cells, csr;
  HFMM_TRY(to_host(tiles, t->m2l_tiles[mi], t->m2l_ntiles[mi]));
  int ncells_t = 0;
  for (const int4& tl : tiles) ncells_t = std::max(ncells_t, tl.z + tl.w);
  HFMM_TRY(to_host(cells, t->m2l_cells[mi], ncells_t));
  HFMM_TRY(to_host(csr, t->pr_csr[ci], ncells_t + 1));
  std::map<std::pair<int, int>, int2> range_of;
  for (const int4& tl : tiles)
    for (int c = 0; c < tl.w; ++c) range_of[{tl.x, cells[tl.z + c]}] = make_int2(csr[tl.z + c], csr[tl.z + c + 1]);
  std::vector<int2> rng(t->total_cells, make_int2(0, 0));  // by cell
  for (const auto& kv : range_of) rng[t->level_off[kv.first.first] + kv.first.second] = kv.second;
  // chunks by level, slot of every pair
  const int nch = t->pr_nchunks[ci];
  const int64_t npairs = t->pr_npairs[ci];
  std::vector<int4> chunks;
  std::vector<int> grouped, psrc;
  HFMM_TRY(to_host(chunks, t->pr_chunks[ci], nch));
  HFMM_TRY(to_host(grouped, t->pr_grouped[ci], npairs));
  HFMM_TRY(to_host(psrc, t->pr_src[ci], npairs));
  std::vector<int> pslot(std::max<int64_t>(1, npairs), 0);
  // per chunk and column: the source row of M and the pair (product row)
  std::vector<int> crow((size_t)std::max(1, nch) * BO_CHUNK, -1), cpid((size_t)std::max(1, nch) * BO_CHUNK, -1);
  for (int c = 0; c < nch; ++c) {
    const int4 ch = chunks[c];
    for (int k = 0; k < ch.w; ++k) {
      const int pr = grouped[ch.z + k];
      crow[(size_t)c * BO_CHUNK + k] = (int)(t->level_off[ch.x] + psrc[pr]);
      cpid[(size_t)c * BO_CHUNK + k] = pr;
    }
  }
  for (int l = 0; l <= L + 1; ++l) b->chunk_first[l] = 0;
  int prev_level = -1;
  for (int c = 0; c < nch; ++c) {
    const int4 ch = chunks[c];
    if (ch.x < prev_level) return HFMM_ERR_UNSUPPORTED;  // chunks must be grouped by level
    if (ch.x != prev_level) b->chunk_first[ch.x] = c;
    prev_level = ch.x;
    b->chunk_count[ch.x]++;
    for (int g = ch.z; g < ch.z + ch.w; ++g) pslot[grouped[g]] = ch.y;
  }
  for (int l = 2; l <= L; ++l)
    if (!b->chunk_count[l]) b->chunk_first[l] = l > 2 ? b->chunk_first[l - 1] + b->chunk_count[l - 1] : 0;
  // near lists of the boundary leaves
  std::vector<int> noff;
  HFMM_TRY(to_host(noff, t->near_off, t->near_count));
  std::vector<int> nsrc_ptr(1, 0), nsrc;
  const int sl = 1 << L;
  const int* al = act.data() + t->level_off[L];
  for (int i = 0; i < nact[L]; ++i) {
    const int leaf = al[i];
    int ix, iy, iz;
    morton_decode((uint64_t)leaf, ix, iy, iz);
    for (int q = 0; q < t->near_count; ++q) {
      const int o = noff[q];
      const int jx = ix + (o & 255) - 128, jy = iy + ((o >> 8) & 255) - 128, jz = iz + ((o >> 16) & 255) - 128;
      if (jx < 0 || jy < 0 || jz < 0 || jx >= sl || jy >= sl || jz >= sl) continue;
      const int j = (int)morton_encode(jx, jy, jz);
      for (int q2 = bfirst[j]; q2 < bfirst[j + 1]; ++q2) nsrc.push_back(q2);
    }
    nsrc_ptr.push_back((int)nsrc.size());
  }
  int max_ns = 0;
  for (size_t i = 0; i + 1 < nsrc_ptr.size(); ++i) max_ns = std::max(max_ns, nsrc_ptr[i + 1] - nsrc_ptr[i]);
  int* d_bsort = nullptr;
  HFMM_TRY(to_dev(t, &b->borig, borig));
  HFMM_TRY(to_dev(t, &d_bsort, bsort));
  HFMM_TRY(to_dev(t, &b->bcode, bcode));
  HFMM_TRY(to_dev(t, &b->bxf, bxf));
  HFMM_TRY(to_dev(t, &b->bfirst, bfirst));
  HFMM_TRY(to_dev(t, &b->nsrc_ptr, nsrc_ptr));
  HFMM_TRY(to_dev(t, &b->nsrc, nsrc));
  HFMM_TRY(to_dev(t, &b->rng, rng));
  HFMM_TRY(to_dev(t, &b->pslot, pslot));
  HFMM_TRY(to_dev(t, &b->crow, crow));
  HFMM_TRY(to_dev(t, &b->cpid, cpid));
  const size_t cs = fp32 ? sizeof(float2) : sizeof(double2);
  HFMM_TRY(tree_alloc(t, &b->qb, cs * (size_t)t->n_bnd));
  HFMM_TRY(tree_alloc(t, &b->nearv, cs * (size_t)t->n_bnd));
  HFMM_TRY(tree_alloc(t, &b->Rb, cs * (size_t)t->n_bnd * P));
  {
    // M [total_cells][P] complex as a 2-D tensor of rows of 2P reals, box one
    // row high (the products gather their source rows four at a time)
    EncodeTiledFn enc = encode_fn();
    if (!enc || 2 * P > 256) return HFMM_ERR_UNSUPPORTED;
    const cuuint64_t dims[2] = {(cuuint64_t)(2 * P), (cuuint64_t)t->total_cells};
    const cuuint64_t strides[1] = {(cuuint64_t)(2 * P) * (fp32 ? 4u : 8u)};
    const cuuint32_t box[2] = {(cuuint32_t)(2 * P), 1u};
    const cuuint32_t es[2] = {1u, 1u};
    if (enc(&b->mrows, fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, t->M, dims, strides,
            box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return HFMM_ERR_UNSUPPORTED;
  }
  const int64_t nrow = t->n_bnd * (int64_t)P;
  if (fp32)
    k_bo_rows<float><<<ceil_div(nrow, 256), 256, 0, s>>>(t->n_bnd, P, d_bsort, (const float2*)t->rtab, (float2*)b->Rb);
  else
    k_bo_rows<double><<<ceil_div(nrow, 256), 256, 0, s>>>(t->n_bnd, P, d_bsort, (const double2*)t->rtab,
                                                         (double2*)b->Rb);
  HFMM_TRY(hfmm_last_launch());
  HFMM_CUDA_TRY(cudaStreamSynchronize(s));
  // barrier words [0, 4) and the dynamic segments' item counters
  HFMM_TRY(tree_alloc_t(t, &b->bar, 4 + BO_MAX_PH * BO_MAX_SEG));
  HFMM_CUDA_TRY(cudaMemset(b->bar, 0, (4 + BO_MAX_PH * BO_MAX_SEG) * sizeof(unsigned)));
  b->nb = (int)t->n_bnd;
  b->nbl = nact[L];
  bo_schedule(b, L, nact, b->chunk_first, b->chunk_count);
  // the near-field items (one per boundary leaf) costliest first: taken
  // from the counter in that order, the last to finish are cheap ones
  {
    std::vector<std::pair<int64_t, int>> c(nact[L]);
    for (int i = 0; i < nact[L]; ++i) {
      const int leaf = act[t->level_off[L] + i];
      c[i] = {-(int64_t)(bfirst[leaf + 1] - bfirst[leaf]) * (nsrc_ptr[i + 1] - nsrc_ptr[i]), i};
    }
    std::stable_sort(c.begin(), c.end(),
                     [](const std::pair<int64_t, int>& x, const std::pair<int64_t, int>& y) { return x.first < y.first; });
    std::vector<int4> items(std::max(1, nact[L]), make_int4(0, 0, 0, 0));
    for (int k = 0; k < nact[L]; ++k) items[k] = make_int4(c[k].second, 0, -1, 0);
    HFMM_TRY(to_dev(t, &b->near_items, items));
  }
  // launch shape: one CTA per SM, product groups sized to the shared memory
  const size_t csz = fp32 ? sizeof(float2) : sizeof(double2);
  // dynamic shared memory left beside the kernel's static arrays (at most 220 KB)
  const void* kern = fp32 ? bo_kernel_for<float, float2>(P) : bo_kernel_for<double, double2>(P);
  const void* kern2 = fp32 ? bo_kernel_for<float, double2>(P) : kern;
  size_t smem_cap = 220 * 1024;
  {
    int dev = 0, optin = 0;
    HFMM_CUDA_TRY(cudaGetDevice(&dev));
    HFMM_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa1, fa2;
    HFMM_CUDA_TRY(cudaFuncGetAttributes(&fa1, kern));
    HFMM_CUDA_TRY(cudaFuncGetAttributes(&fa2, kern2));
    const size_t stat = std::max(fa1.sharedSizeBytes, fa2.sharedSizeBytes);
    if ((size_t)optin <= stat) return HFMM_ERR_UNSUPPORTED;
    smem_cap = std::min(smem_cap, (size_t)optin - stat);
  }
  const int nst = bo_stages(cfg.R, cfg.RT, (int)csz);
  const size_t group_bytes = (size_t)nst * ((size_t)P * P + (size_t)BO_CHUNK * P) * csz;
  const size_t budget = std::min<size_t>(200 * 1024, smem_cap);
  const int GT = cfg.RT * 8;
  int ng = (int)std::min<size_t>(std::min(BO_MAX_NG, 512 / GT), budget / group_bytes);
  ng = std::min(ng, bo_groups(cfg.R, cfg.RT, (int)csz));  // the kernel's launch bound
  if (ng < 1) return HFMM_ERR_UNSUPPORTED;
  b->ng = ng;
  b->nst = nst;
  b->threads = ng * GT;
  // team items (P2M, M2M): two teams, each 16 P + staged weights
  const size_t team_bytes = 2 * csz * (size_t)(16 * P + 8 * BO_MAX_LEAF_PTS);
  // downward items: per group two [S][P] partial sums, the parent's and its
  // own L and the leaf's near field; at the leaf level the kernel table and
  // the L2L operators staged in front when they fit (and there are enough
  // leaves per CTA to pay for the copy)
  // (record sizes as in the kernel: the sums rounded to whole two-element
  // near-source records, then near_win records)
  const size_t sums = ((size_t)(2 * (GT / (P / 2)) + 2) * P + BO_MAX_LEAF_PTS + 1) / 2 * 2;
  auto down_b = [&](int nw) { return csz * (size_t)ng * (sums + 2 * (size_t)nw); };
  const size_t tab_bytes = csz * (size_t)((t->lat_half + 1) & ~(int64_t)1);
  const size_t l2l_bytes = csz * 8 * (size_t)P * P;
  const bool worth = nact[L] >= 4 * nsm;
  b->stage_tab = worth && down_b(0) + tab_bytes <= smem_cap;
  int nw = std::min(max_ns, 1024);
  while (nw > 0 && down_b(nw) + (b->stage_tab ? tab_bytes : 0) > smem_cap) nw /= 2;
  b->near_win = nw;
  b->stage_l2l = worth && L > 2 && down_b(nw) + (b->stage_tab ? tab_bytes : 0) + l2l_bytes <= smem_cap;
  const size_t down_total = down_b(nw) + (b->stage_tab ? tab_bytes : 0) + (b->stage_l2l ? l2l_bytes : 0);
  b->smem = std::max(std::max((size_t)ng * group_bytes, team_bytes), down_total);
  HFMM_TRY(set_smem_any(kern, b->smem));
  HFMM_TRY(set_smem_any(kern2, b->smem));
  int per_sm = 0;
  HFMM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, b->threads, b->smem));
  int per_sm2 = 0;
  HFMM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, kern2, b->threads, b->smem));
  if (per_sm < 1 || per_sm2 < 1) return HFMM_ERR_UNSUPPORTED;
  b->grid = nsm;
  b->ok = 1;
  return HFMM_OK;
}

template <typename T, typename IO>
int bo_launch(fmm_tree* t, const IO* x, IO* y, double scale, cudaStream_t s, int cycle_m = 0, double rtol = 0.0,
              int* cflags = nullptr) {
  bnd_op_state* b = t->bop;
  BoArgs<T, IO> A;
  A.x = x;
  A.y = y;
  A.skip = nullptr;  // set below for a single apply (a cycle resets its own flags at its start)
  A.cycle = cycle_m > 0 ? 1 : 0;
  A.m = cycle_m;
  A.rtol = rtol;
  A.b = x;
  A.xout = y;
  A.Vc = reinterpret_cast<C<T>*>(b->Vc);
  A.wc = reinterpret_cast<C<T>*>(b->wc);
  A.part = b->part;
  A.dots = b->dots;
  A.H = b->H;
  A.cs = b->cs;
  A.sn = b->sn;
  A.gv = b->gv;
  A.scal = b->scal;
  A.cflags = cflags ? cflags : b->cflags;
  A.scale = T(scale);
  if (!A.cycle) A.skip = t->skip;
  A.P = t->P;
  A.L = t->L;
  A.nb = b->nb;
  A.ng = b->ng;
  A.nst = b->nst;
  A.k = T(t->k);
  A.sig = mkc<T>(T(t->sigma_bnd.x), T(t->sigma_bnd.y));
  A.borig = b->borig;
  A.bcode = b->bcode;
  A.bxf = b->bxf;
  A.bfirst = b->bfirst;
  A.Rb = reinterpret_cast<const C<T>*>(b->Rb);
  A.qb = reinterpret_cast<C<T>*>(b->qb);
  A.tab = reinterpret_cast<const C<T>*>(sizeof(T) == 4 ? (const void*)t->lat_tab32 : (const void*)t->lat_tab64);
  A.nsrc_ptr = b->nsrc_ptr;
  A.nsrc = b->nsrc;
  A.near_items = b->near_items;
  A.mrows = b->mrows;
  A.tab_len = t->lat_half;
  A.nearv = reinterpret_cast<C<T>*>(b->nearv);
  A.flags = t->flags;
  for (int l = 0; l < HFMM_MAX_LEVEL + 2; ++l) A.loff[l] = t->level_off[l];
  const int mi = HFMM_SET_BND - 1, ci = mi * 3 + mi;
  A.act = t->act_cells[mi];
  A.rng = b->rng;
  A.M = reinterpret_cast<C<T>*>(t->M);
  A.Lc = reinterpret_cast<C<T>*>(t->Lc);
  A.m2m = reinterpret_cast<const C<T>*>(sizeof(T) == 4 ? (const void*)t->op_m2m32 : (const void*)t->op_m2m);
  A.l2l = reinterpret_cast<const C<T>*>(sizeof(T) == 4 ? (const void*)t->op_l2l32 : (const void*)t->op_l2l);
  A.m2l = reinterpret_cast<const C<T>*>(sizeof(T) == 4 ? (const void*)t->op_m2l32 : (const void*)t->op_m2l);
  A.box_cells = t->box_cells;
  A.chunks = t->pr_chunks[ci];
  A.grouped = t->pr_grouped[ci];
  A.crow = b->crow;
  A.cpid = b->cpid;
  A.psrc = t->pr_src[ci];
  A.pslot = b->pslot;
  A.buf = reinterpret_cast<C<T>*>(t->pr_buf);
  A.bar = b->bar;
  A.smem_bytes = b->smem;
  A.stage_l2l = b->stage_l2l;
  A.stage_tab = b->stage_tab;
  A.near_win = b->near_win;
  A.nphase = b->nphase;
  for (int i = 0; i < b->nphase; ++i) A.ph[i] = b->ph[i];
  const void* kern = bo_kernel_for<T, IO>(t->P);
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)b->grid);
  lc.blockDim = dim3((unsigned)b->threads);
  lc.dynamicSmemBytes = b->smem;
  lc.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  void* args[] = {(void*)&A};
  HFMM_CUDA_TRY(cudaLaunchKernelExC(&lc, kern, args));
  count_launches(1);
  return HFMM_OK;
}

}  // namespace

int fmm_bnd_apply(fmm_tree* t, const float2* x, float2* y, double scale, cudaStream_t s) {
  if (!t->use_bnd_op || t->precision != HFMM_FP32) return HFMM_ERR_UNSUPPORTED;
  HFMM_TRY(bo_plan(t, true, s));
  return bo_launch<float, float2>(t, x, y, scale, s);
}

int fmm_bnd_apply(fmm_tree* t, const double2* x, double2* y, double scale, cudaStream_t s) {
  if (!t->use_bnd_op) return HFMM_ERR_UNSUPPORTED;
  const bool fp32 = t->precision == HFMM_FP32;
  HFMM_TRY(bo_plan(t, fp32, s));
  if (fp32) return bo_launch<float, double2>(t, x, y, scale, s);
  return bo_launch<double, double2>(t, x, y, scale, s);
}

// workspace of the in-kernel cycle for m steps (grown on demand, outside any
// stream capture)
static int bo_cycle_reserve(fmm_tree* t, int m) {
  bnd_op_state* b = t->bop;
  if (b->cyc_m >= m) return HFMM_OK;
  const size_t cs = t->precision == HFMM_FP32 ? sizeof(float2) : sizeof(double2);
  HFMM_TRY(tree_alloc(t, &b->Vc, cs * (size_t)(m + 1) * t->n_bnd));
  HFMM_TRY(tree_alloc(t, &b->wc, cs * (size_t)t->n_bnd));
  HFMM_TRY(tree_alloc_t(t, &b->part, 3 * (size_t)(m + 2) * b->grid));
  HFMM_TRY(tree_alloc_t(t, &b->dots, 2 * (size_t)(m + 1) + 1));
  HFMM_TRY(tree_alloc_t(t, &b->H, (size_t)m * (m + 1)));
  HFMM_TRY(tree_alloc_t(t, &b->cs, (size_t)m));
  HFMM_TRY(tree_alloc_t(t, &b->sn, (size_t)m));
  HFMM_TRY(tree_alloc_t(t, &b->gv, (size_t)m + 1));
  HFMM_TRY(tree_alloc_t(t, &b->scal, 4));
  if (!b->cflags) {
    HFMM_TRY(tree_alloc_t(t, &b->cflags, 4));
    HFMM_CUDA_TRY(cudaMemset(b->cflags, 0, 4 * sizeof(int)));
  }
  b->cyc_m = m;
  return HFMM_OK;
}

int bnd_op_cycle_ready(fmm_tree* t, int m, cudaStream_t s) {
  if (m < 1 || m > BO_MAX_M) return HFMM_ERR_UNSUPPORTED;
  HFMM_TRY(bnd_op_ready(t, s));
  // the back substitution stages the m x m triangle in the kernel's shared memory
  if ((size_t)m * m * sizeof(double2) > t->bop->smem) return HFMM_ERR_UNSUPPORTED;
  return bo_cycle_reserve(t, m);
}

int fmm_bnd_cycle(fmm_tree* t, const float2* b, float2* x, double scale, int m, double rtol, int* d_flags,
                  cudaStream_t s) {
  if (t->precision != HFMM_FP32 || !t->bop || t->bop->cyc_m < m) return HFMM_ERR_UNSUPPORTED;
  return bo_launch<float, float2>(t, b, x, scale, s, m, rtol, d_flags);
}

int fmm_bnd_cycle(fmm_tree* t, const double2* b, double2* x, double scale, int m, double rtol, int* d_flags,
                  cudaStream_t s) {
  if (t->precision != HFMM_FP64 || !t->bop || t->bop->cyc_m < m) return HFMM_ERR_UNSUPPORTED;
  return bo_launch<double, double2>(t, b, x, scale, s, m, rtol, d_flags);
}

const int* bnd_op_cycle_flags(const fmm_tree* t) { return t->bop ? t->bop->cflags : nullptr; }

bool bnd_op_cycle_planned(const fmm_tree* t, int m) {
  return t->bop && t->bop->ok > 0 && t->bop->cyc_m >= m && m <= BO_MAX_M &&
         (size_t)m * m * sizeof(double2) <= t->bop->smem;
}

int bnd_op_ready(fmm_tree* t, cudaStream_t s) {
  if (!t->use_bnd_op) return HFMM_ERR_UNSUPPORTED;
  return bo_plan(t, t->precision == HFMM_FP32, s);
}

bool bnd_op_planned(const fmm_tree* t) { return t->bop && t->bop->ok > 0; }

int bnd_op_error(cudaStream_t s, bool clear) {
  int h = 0;
  HFMM_CUDA_TRY(cudaMemcpyFromSymbolAsync(&h, g_bo_error, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
  HFMM_CUDA_TRY(cudaStreamSynchronize(s));
  if (h && clear) {
    int z = 0;
    HFMM_CUDA_TRY(cudaMemcpyToSymbolAsync(g_bo_error, &z, sizeof(int), 0, cudaMemcpyHostToDevice, s));
  }
  return h;
}

void bnd_op_release(fmm_tree* t) {
  delete t->bop;  // its device arrays belong to the handle's allocation list
  t->bop = nullptr;
}
