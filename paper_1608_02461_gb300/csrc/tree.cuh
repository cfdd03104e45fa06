// Internal state of an fmm_tree handle and the entry points shared between
// the translation units of the library.
#pragma once

#include <vector>

#include "common.cuh"

// One device allocation tracked by the handle.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

struct fmm_tree_ext;  // solver workspaces (capi.cu)
struct fmm_tc_state;  // tensor-core M2L state (m2l_tc.cu)
struct bnd_op_state;  // boundary -> boundary apply as one kernel (bnd_op.cu)
struct fmm_tc_near_state;  // volume near field on the tensor cores (m2l_tc.cu)

// kernels launched by the library (all handles)
void count_launches(int64_t n);
int64_t launches_so_far();

// Per-stage CUDA-event timing: pairs of events recorded around each stage's
// launches, resolved lazily (flush) so that timing adds no synchronisation.
// While a graph is being captured (`cap` set) each timed stage gets its own
// pair of external events, recorded at every replay of the graph and
// resolved after it (resolve_slots).
struct TimerSlot {
  int stage;
  cudaEvent_t a, b;
  int nlaunch;
  double work;
};

struct StageTimer {
  bool on = false;
  int mask = 0;               // stages timed (bit per stage)
  bool cur = false;           // the current begin() was recorded
  std::vector<TimerSlot>* cap = nullptr;
  std::vector<cudaEvent_t> pool;
  std::vector<int> stage_of;  // per recorded pair
  size_t used = 0;            // events used in the pool
  double ms[HFMM_NSTAGES] = {0};
  int64_t launches[HFMM_NSTAGES] = {0};
  double work[HFMM_NSTAGES] = {0};
  void begin(int stage, cudaStream_t s) {
    cur = on && ((mask >> stage) & 1);
    if (!cur) return;
    if (cap) {
      TimerSlot sl{stage, nullptr, nullptr, 0, 0.0};
      cudaEventCreate(&sl.a);
      cudaEventCreate(&sl.b);
      cudaEventRecordWithFlags(sl.a, s, cudaEventRecordExternal);
      cap->push_back(sl);
      return;
    }
    if (used + 2 > pool.size()) {
      if (pool.size() >= 8192) flush();
      while (used + 2 > pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        pool.push_back(e);
      }
    }
    cudaEventRecord(pool[used], s);
    stage_of.push_back(stage);
  }
  void end(int nlaunch, cudaStream_t s, double w = 0.0) {
    if (!cur) return;
    cur = false;
    if (cap) {
      TimerSlot& sl = cap->back();
      cudaEventRecordWithFlags(sl.b, s, cudaEventRecordExternal);
      sl.nlaunch = nlaunch;
      sl.work = w;
      return;
    }
    cudaEventRecord(pool[used + 1], s);
    launches[stage_of.back()] += nlaunch;
    work[stage_of.back()] += w;
    used += 2;
  }
  void resolve_slots(const std::vector<TimerSlot>& slots) {
    if (slots.empty()) return;
    cudaEventSynchronize(slots.back().b);
    for (const auto& sl : slots) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, sl.a, sl.b) == cudaSuccess) ms[sl.stage] += t;
      launches[sl.stage] += sl.nlaunch;
      work[sl.stage] += sl.work;
    }
    cudaGetLastError();
  }
  void flush() {
    if (used == 0) return;
    cudaEventSynchronize(pool[used - 1]);
    for (size_t i = 0; i < stage_of.size(); ++i) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, pool[2 * i], pool[2 * i + 1]) == cudaSuccess) ms[stage_of[i]] += t;
    }
    cudaGetLastError();
    stage_of.clear();
    used = 0;
  }
  void reset() {
    flush();
    for (int i = 0; i < HFMM_NSTAGES; ++i) {
      ms[i] = 0;
      launches[i] = 0;
      work[i] = 0;
    }
  }
  void destroy() {
    for (auto e : pool) cudaEventDestroy(e);
    pool.clear();
    stage_of.clear();
    used = 0;
  }
};

struct fmm_tree {
  fmm_tree_ext* ext = nullptr;
  // ---- problem
  int n = 0;             // interior nodes per axis (lattice trees)
  int lattice = 1;       // 1: points are the n^3 nodes and 6 n^2 panels
  int64_t n_vol = 0, n_bnd = 0, n_pts = 0;
  double h = 0.0, k = 0.0;
  int p = 0, P = 0;      // order and coefficients per expansion (p^2)
  int precision = HFMM_FP64;
  int leaf_size = 0;
  double theta = 0.0;
  int64_t th_num = 0, th_den = 1;  // theta as a rational number
  int L = 0;             // leaf level
  int nlv = 0;           // lattice leaf cells per axis = 2^L

  // ---- points in sorted (leaf-Morton) order: within a leaf volume points
  //      first, then boundary points, each by original index
  double* xyz = nullptr;        // [n_pts][3] sorted coordinates (FP64)
  float* xyz32 = nullptr;       // [n_pts][4] sorted coordinates (FP32, w unused)
  int64_t* orig = nullptr;      // sorted position -> original id (vol ids, then n_vol + bnd id)
  int64_t* pos_of = nullptr;    // original id -> sorted position
  int* leaf_start = nullptr;    // [8^L + 1] first sorted position of each leaf
  int* leaf_mid = nullptr;      // [8^L] first boundary point of each leaf
  int* flags = nullptr;         // per level, per Morton cell: bit0 volume points, bit1 boundary
  int64_t level_off[HFMM_MAX_LEVEL + 2] = {0};  // first cell of level l in the per-cell arrays
  int64_t* level_off_dev = nullptr;             // device copy
  int64_t total_cells = 0;

  // cells of each level holding points of a set mask (index mask - 1), in
  // Morton order at level_off[l]; counts on the host for grid sizes
  int* act_cells[3] = {nullptr, nullptr, nullptr};
  int act_count[3][HFMM_MAX_LEVEL + 1] = {};

  // ---- interaction lists (offsets in cell units)
  int near_count = 0;
  int* near_off = nullptr;      // [near_count] packed offsets (dx,dy,dz) each in 8 bits + 128
  int box_r = 0;                // M2L offsets lie in [-box_r, box_r]^3
  int m2l_count = 0;            // offsets per parity class (same for all classes)
  int* m2l_off = nullptr;       // [8][m2l_count] packed offsets
  int* m2l_box_index = nullptr; // [8][m2l_count] operator slot of each list entry
  int* m2l_slot_off = nullptr;  // [slots] packed offset of each operator slot
  // target cells of the M2L, per target-set mask (index mask - 1), grouped by
  // level and parity class, and tiles {level, class, first, count} over them
  int m2l_tc = 32;              // target cells per tile
  int* m2l_cells[3] = {nullptr, nullptr, nullptr};
  int4* m2l_tiles[3] = {nullptr, nullptr, nullptr};
  int m2l_ntiles[3] = {0, 0, 0};
  int m2l_tiles_lt[3][HFMM_MAX_LEVEL + 2] = {};  // tiles of the levels below l, per target mask
  // per (target mask, source mask) pair, index 3 (tm-1) + (sm-1): the valid
  // offsets of every tile (built on first use)
  int* m2l_vlist[9] = {};
  unsigned* m2l_vmask[9] = {};
  int* m2l_nval[9] = {};
  void* zero_row = nullptr;     // P complex zeros (bulk-copy source for empty columns)
  // pair-list M2L for sparse passes, per (target mask, source mask) pair:
  // the valid (target, source) cell pairs in target-major order (CSR over the
  // tile cells), the same pairs grouped by (level, operator slot) in chunks
  // of at most 32, and a product buffer with one row per pair
  int* pr_tgt[9] = {};          // [npairs] level-local target cell (CSR order)
  int* pr_src[9] = {};          // [npairs] level-local source cell
  int* pr_csr[9] = {};          // [ncells + 1] pair range of each tile cell (cells in tile order)
  int* pr_grouped[9] = {};      // [npairs] pair indices grouped by (level, slot)
  int4* pr_chunks[9] = {};      // {level, slot, first (grouped), count}
  int pr_nchunks[9] = {};
  int64_t pr_npairs[9] = {};
  void* pr_buf = nullptr;       // [max npairs][P] products (precision T)
  int64_t pr_buf_pairs = 0;
  int m2l_pairs_enabled = 1;    // allow the pair-list form for boundary-target passes
  void* m2l_part = nullptr;     // [m2l_part_max][total_cells][P] split-offset partial sums
  int m2l_part_max = 1;
  int m2l_variant = 1;          // 1: warp-specialised pipeline, 0: two-stage block pipeline
  int m2l_fill = 4;             // split offset lists until the grid holds fill x 152 blocks
  // autotuned (variant, fill) per (target mask, source mask) pair, index 3 (tm-1) + (sm-1);
  // variant -1: not tuned (use the defaults above)
  int tuned_variant[9] = {-1, -1, -1, -1, -1, -1, -1, -1, -1};
  int tuned_fill[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  // autotuned lattice near field per (target mask, source mask) pair, same
  // index: tiled form (FP32), cap on the threads per target group (power of
  // two, 0: not tuned, use the defaults), blocks per SM (0: as many as fit)
  int tuned_p2p_tile[9] = {};
  int tuned_p2p_tpt[9] = {};
  int tuned_p2p_blocks[9] = {};
  // near field concurrent with the far field (1) or after L2P (0) per pass,
  // same index; -1: not tuned (concurrent exactly when the targets are the
  // boundary points)
  int tuned_overlap[9] = {-1, -1, -1, -1, -1, -1, -1, -1, -1};

  // ---- near-field kernel table of lattice trees: every point is a node of
  //      the lattice h Z^3, so the kernel between two points depends only on
  //      their integer offset d in [-D, D]^3 (D: largest offset component
  //      between points of near leaves), coded as delta = lin_t - lin_s with
  //      lin = ix + Sy iy + Sz iz (Sy > 2D, Sz = (2D + 1) Sy: one-to-one on
  //      the box); G(d) = G(-d), so a half table lat_tab[|delta|] =
  //      e^{ik h|d|} / (4 pi h|d|) (0 at d = 0) holds all
  int lat_D = 0;                // 0: no table
  int lat_Sy = 0, lat_Sz = 0;   // strides of the offset code
  int64_t lat_half = 0;         // D (1 + Sy + Sz) + 1 entries, padded to a multiple of 16 bytes (FP64 size)
  int* lat_lin = nullptr;       // [n_pts] lin of each sorted point
  float2* lat_tab32 = nullptr;  // [lat_half] FP32 table
  double2* lat_tab64 = nullptr; // [lat_half] FP64 table
  int lat_tab64_fits = 0;       // the FP64 table fits the near-field kernel's shared memory
  int use_lattice_p2p = 1;      // near field through the table when it exists
  int lat_tile = 0;             // FP32: 4 x 4 target-source tiles over x-runs of the lattice

  // ---- regular basis table [n_pts][P]: R_a(x_i - c) for each sorted point
  //      and its leaf centre (precision of the form); P2M and L2P read it
  //      instead of evaluating Bessel and Legendre functions per apply
  void* rtab = nullptr;
  int use_rtab = 1;

  // ---- tensor-core M2L (FP32 form, levels >= 4): operator images, class
  //      lattices of the multipoles and their TMA descriptors, built on first
  //      use; use_m2l_tcore: 0 off, 1 passes with volume targets, 2 all passes
  fmm_tc_state* m2l_tcore = nullptr;
  int use_m2l_tcore = 1;
  // ---- volume -> volume near field on the tensor cores (FP32 form, regular
  //      lattice trees of depth >= 4: every leaf the same block of nodes, so
  //      the block between two leaves depends only on their offset); set up on
  //      first use; use_near_tcore 0: always the lattice near-field kernel
  fmm_tc_near_state* near_tcore = nullptr;
  int use_near_tcore = 1;

  // ---- near field concurrent with the far field: P2P runs on its own
  //      stream (fork/join through events, also inside captured graphs) into
  //      phis_near, and L2P adds it
  cudaStream_t near_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  void* phis_near = nullptr;    // [n_pts] precision T
  int overlap_near = 1;

  // ---- operators (FP64 master copy; FP32 copy for the FP32 form)
  double2* op_m2m = nullptr;    // [L+1][8][P][P]   row a' (out), column a (in)
  double2* op_l2l = nullptr;    // [L+1][8][P][P]
  double2* op_m2l = nullptr;    // [L+1][box^3][P][P]
  float2* op_m2m32 = nullptr;
  float2* op_l2l32 = nullptr;
  float2* op_m2l32 = nullptr;
  int64_t box_cells = 0;        // distinct M2L offsets = operator slots per level
  double* gaunt = nullptr;      // Gaunt integrals [P][P][2p-1] (operator builds)
  // d/dk operators (tangent mode) and Hermitian adjoints (adjoint mode): same
  // layouts as the forward ones, built on first use
  double2 *op_m2m_d = nullptr, *op_l2l_d = nullptr, *op_m2l_d = nullptr;
  float2 *op_m2m_d32 = nullptr, *op_l2l_d32 = nullptr, *op_m2l_d32 = nullptr;
  double2 *op_m2m_h = nullptr, *op_l2l_h = nullptr, *op_m2l_h = nullptr;
  float2 *op_m2m_h32 = nullptr, *op_l2l_h32 = nullptr, *op_m2l_h32 = nullptr;
  int* m2l_slot_neg = nullptr;  // slot of the negated offset
  // tangent-mode work arrays (precision T), allocated on first use
  void* Md = nullptr;           // dM/dk [total_cells][P]
  void* Ld = nullptr;           // dL/dk [total_cells][P]
  void* phis_d = nullptr;       // dphi/dk sorted [n_pts]
  // singular self coefficients' k-derivatives per unit weight
  double2 dsigma_vol = {0, 0}, dsigma_bnd = {0, 0};

  // ---- singular self coefficients per unit weight
  double2 sigma_vol = {0, 0};   // s_Omega / h^3
  double2 sigma_bnd = {0, 0};   // s_Gamma / h^2
  double2 s_vol = {0, 0}, s_bnd = {0, 0};

  // ---- expansions and sorted work vectors (precision T)
  void* M = nullptr;            // [total_cells][P]
  void* Lc = nullptr;           // [total_cells][P]
  void* qs = nullptr;           // [n_pts] sorted weights
  void* phis = nullptr;         // [n_pts] sorted potentials

  // ---- boundary -> boundary apply of the inner solve as one persistent
  //      kernel (plan built on first use); use_bnd_op 0: the stage chain,
  //      1: the kernel up to P = 36, 2: the kernel for every P it supports
  bnd_op_state* bop = nullptr;
  int use_bnd_op = 1;
  int bnd_op_suspend = 0;       // set while the handle runs inside gmres_solve_batched

  int use_graphs = 1;           // gmres_solve replays the preconditioner as one CUDA graph
  // auxiliary tree over the same points with expansion order inner_p, used
  // for the boundary -> boundary applies of the preconditioner's inner solve
  // (Pass B); nullptr: Pass B uses this tree
  fmm_tree* inner = nullptr;
  int inner_p = 0;
  // device flag read by every FMM kernel: nonzero = return at once (set while
  // capturing the graph of the inner solve, whose late iterations are skipped
  // after convergence); nullptr outside graphs
  const int* skip = nullptr;

  // ---- preconditioner work (complex128)
  double2* g_bnd = nullptr;     // [n_bnd]
  double2* q_bnd = nullptr;     // [n_bnd]
  float2* g_bnd32 = nullptr;    // [n_bnd] the same for the complex64 inner solve of the FP32 form
  float2* q_bnd32 = nullptr;

  // ---- counters
  int64_t m2l_pairs = 0, p2p_pairs = 0;
  // cell pairs per level by (target flags, source flags), and near-field
  // point pairs by (target set, source set) with index 2*(tgt==BND)+(src==BND)
  int64_t m2l_cnt[HFMM_MAX_LEVEL + 1][4][4] = {};
  int64_t p2p_cnt[4] = {0, 0, 0, 0};
  double ms_last_apply = 0.0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  StageTimer timer;

  std::vector<DevBuf> bufs;
  int64_t device_bytes = 0;
};

// allocation helper owned by the handle
int tree_alloc(fmm_tree* t, void** ptr, size_t bytes);
template <typename X>
inline int tree_alloc_t(fmm_tree* t, X** ptr, size_t count) {
  return tree_alloc(t, (void**)ptr, count * sizeof(X));
}

// tree.cu
int build_geometry_and_sort(fmm_tree* t, const double* d_vol, const double* d_bnd, cudaStream_t s);
int build_lists(fmm_tree* t, cudaStream_t s);
int build_self_terms(fmm_tree* t, cudaStream_t s);
int build_pair_counts(fmm_tree* t, cudaStream_t s);
int build_m2l_tiles(fmm_tree* t, cudaStream_t s);
int build_active_lists(fmm_tree* t, cudaStream_t s);
int build_lattice_table(fmm_tree* t, cudaStream_t s);
// fmm.cu: regular basis table (skipped when it would take over a quarter of free memory)
int build_basis_table(fmm_tree* t, cudaStream_t s);
double p2p_work(const fmm_tree* t, int src_set, int tgt_set);
double m2l_work(const fmm_tree* t, int src_set, int tgt_set);

// operators.cu
int build_operators(fmm_tree* t, cudaStream_t s);
int build_operators_deriv(fmm_tree* t, cudaStream_t s);
int build_operators_adjoint(fmm_tree* t, cudaStream_t s);

// fmm.cu: sorted-weight gather, FMM core over the sorted vectors, scatter
int fmm_gather(fmm_tree* t, int src_set, const double2* q_vol, double scale_vol,
               const double2* q_bnd, double scale_bnd, cudaStream_t s);
// the same with a complex64 boundary vector
int fmm_gather(fmm_tree* t, int src_set, const double2* q_vol, double scale_vol,
               const float2* q_bnd, double scale_bnd, cudaStream_t s);
int fmm_core(fmm_tree* t, int src_set, int tgt_set, cudaStream_t s);
// double-layer pass (lattice trees): dipole strengths in qs on the boundary
// panels, phis_i = sum_{j != i} q_j dG/dn_y(x_i, y_j) on tgt_set
int fmm_core_dlp(fmm_tree* t, int tgt_set, cudaStream_t s);
// adjoint pass: weights in qs on the points of tgt_set, result in phis on src_set
int fmm_core_adjoint(fmm_tree* t, int src_set, int tgt_set, cudaStream_t s);
// tangent pass: d(phi)/dk into phis for the weights in qs
int fmm_core_dk(fmm_tree* t, int src_set, int tgt_set, cudaStream_t s);
// HFMM_ERR_TIMEOUT (or 0) recorded by a kernel's bounded wait; synchronises s
int fmm_device_error(cudaStream_t s, bool clear);
// raises a kernel's dynamic shared-memory limit (never lowers it)
int set_smem_any(const void* fn, size_t bytes);

// m2l_tc.cu: tensor-core M2L of the levels >= m2l_tc_lmin(t) (0: not available)
int m2l_tc_lmin(const fmm_tree* t);
int m2l_tc_stage(fmm_tree* t, int src_set, int tgt_set, int accumulate, cudaStream_t s, int* nlaunch);
int m2l_tc_error(cudaStream_t s, bool clear);
void m2l_tc_release(fmm_tree* t);
// m2l_tc.cu: the volume -> volume near field (and volume self terms) added to
// phis on the tensor cores, for passes with volume targets only
bool near_tc_usable(fmm_tree* t, int src_set, int tgt_set, cudaStream_t s);
int near_tc_stage(fmm_tree* t, cudaStream_t s, int* nlaunch);
void near_tc_release(fmm_tree* t);
int fmm_scatter(fmm_tree* t, int tgt_set, double2* phi_vol, double2* phi_bnd, cudaStream_t s);
int fmm_scatter(fmm_tree* t, int tgt_set, double2* phi_vol, float2* phi_bnd, cudaStream_t s);
int fmm_scatter_from(fmm_tree* t, const void* sorted, int tgt_set, double2* phi_vol, double2* phi_bnd,
                     cudaStream_t s);

// bnd_op.cu: y = G~(scale x) between the boundary points (x, y in the original
// boundary order) as one cooperative kernel; HFMM_ERR_UNSUPPORTED when the
// tree does not qualify (the caller then runs the stage chain).  The first
// call builds the plan (host synchronisation: not inside a stream capture).
int fmm_bnd_apply(fmm_tree* t, const float2* x, float2* y, double scale, cudaStream_t s);
int fmm_bnd_apply(fmm_tree* t, const double2* x, double2* y, double scale, cudaStream_t s);
int bnd_op_ready(fmm_tree* t, cudaStream_t s);  // builds the plan; HFMM_OK when usable
bool bnd_op_planned(const fmm_tree* t);          // a usable plan exists
// one GMRES cycle of m <= 128 steps from x = 0 for (G~ scale) x = b between the
// boundary points (b, x in the original order), inside the same kernel; the
// flags (device, or the plan's own when null): [0] done, [1] steps,
// [2] += steps.  bnd_op_cycle_ready builds the plan and the workspace (not
// inside a capture).
int bnd_op_cycle_ready(fmm_tree* t, int m, cudaStream_t s);
int fmm_bnd_cycle(fmm_tree* t, const float2* b, float2* x, double scale, int m, double rtol, int* d_flags,
                  cudaStream_t s);
int fmm_bnd_cycle(fmm_tree* t, const double2* b, double2* x, double scale, int m, double rtol, int* d_flags,
                  cudaStream_t s);
const int* bnd_op_cycle_flags(const fmm_tree* t);
bool bnd_op_cycle_planned(const fmm_tree* t, int m);
int bnd_op_error(cudaStream_t s, bool clear);
void bnd_op_release(fmm_tree* t);
// fmm.cu: pair lists of a (source set, target set) pass, built on first use
int fmm_pair_lists(fmm_tree* t, int src_set, int tgt_set, cudaStream_t s);

// krylov.cu
int fdm_apply_dev(int n, double h, double k, const double2* u, double2* out, cudaStream_t s);
