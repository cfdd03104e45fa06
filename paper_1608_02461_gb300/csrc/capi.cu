// The C ABI declared in include/hfmm.h: handle life cycle, argument checks,
// the FMM apply, the BEM-coupled preconditioner (Sec. 5.2-5.3) and the outer
// preconditioned GMRES (Sec. 3-4, Sec. 6).
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <new>

#include "krylov.cuh"
#include "tree.cuh"

// The preconditioner as one CUDA graph: Pass A, one device-driven inner
// GMRES cycle (its late steps skipped after convergence through a device
// flag), Pass C; on fixed input/output buffers.  Captured on a private
// stream, replayed on the caller's.
struct PrecGraph {
  cudaGraphExec_t exec = nullptr;
  double rtol = -1.0;
  int maxit = -1;
  int timer_mask = -1;
  int bnd_mode = -1;            // boundary operator form captured (1: one kernel, 0: stage chain)
  int eager_its = 0;            // inner steps of the eager apply that preceded a capture
  double2* r_in = nullptr;
  double2* z_out = nullptr;
  int* flags = nullptr;         // [0] done, [1] steps of the last cycle, [2] steps summed over replays
  int64_t kernels = 0;          // kernel nodes per replay
  std::vector<TimerSlot> slots; // timed stages inside the graph
  bool pending = false;         // slots of the last replay not yet resolved
  cudaStream_t cap = nullptr;
};

struct fmm_tree_ext {
  GmresWork inner;   // boundary solve V q = -g (FP64 form)
  GmresWork inner_g; // the same in the graph form
  GmresWorkT<float> inner32;    // the complex64 boundary solve of the FP32 form
  GmresWorkT<float> inner_g32;  // the same in the graph form
  GmresWork outer;   // A x = b
  BicgWork bicg;     // A x = b by BiCGSTAB
  PrecGraph pg;
  void* dl_work = nullptr;  // [max(n_vol, n_bnd)] complex128: double-layer sums of the BEM solve with data
  void* gk_phi = nullptr;   // [n_vol] complex128: dphi/dk of fmm_grad_k
  double* gk_part = nullptr;  // [RE_DOT_PARTS] block partials of the k-gradient reductions
};

// the inner workspaces and boundary vectors of a form
inline GmresWorkT<double>& inner_ws(fmm_tree_ext* e, double, bool graph) { return graph ? e->inner_g : e->inner; }
inline GmresWorkT<float>& inner_ws(fmm_tree_ext* e, float, bool graph) { return graph ? e->inner_g32 : e->inner32; }
inline double2* bnd_g(fmm_tree* t, double) { return t->g_bnd; }
inline double2* bnd_q(fmm_tree* t, double) { return t->q_bnd; }
inline float2* bnd_g(fmm_tree* t, float) { return t->g_bnd32; }
inline float2* bnd_q(fmm_tree* t, float) { return t->q_bnd32; }

// tree of the boundary -> boundary applies of the inner solve (Pass B), with
// the caller's timing state (and, while a graph is captured, its timer slots
// and skip flag)
inline fmm_tree* pass_b_tree(fmm_tree* t) {
  fmm_tree* b = t->inner ? t->inner : t;
  if (b != t) {
    b->timer.on = t->timer.on;
    b->timer.mask = t->timer.mask;
    b->timer.cap = t->timer.cap;
    b->skip = t->skip;
    b->bnd_op_suspend = t->bnd_op_suspend;
  }
  return b;
}

// out = G~_{Gamma,Gamma}(scale in) + self term on the boundary points (the
// operator of the inner solve): one persistent kernel when the tree has a
// plan for it (built on first use, outside any capture), else the stage chain
static bool bnd_op_usable(fmm_tree* t, cudaStream_t s) {
  // not inside gmres_solve_batched: concurrent solves would run several
  // cooperative kernels at once, each waiting for all of its CTAs
  if (!t->use_bnd_op || t->bnd_op_suspend || t->n_bnd == 0) return false;
  if (!t->bop) {  // the plan is built outside any stream capture
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (cs != cudaStreamCaptureStatusNone) return false;
  }
  return bnd_op_ready(t, s) == HFMM_OK;
}

// the inner solve V q = -g as one GMRES cycle inside the boundary operator's
// kernel: when the tree has the plan, the solve is one cycle (inner_m >=
// inner_maxit) and the cycle fits the kernel (at most 128 steps)
static bool bnd_cycle_usable(fmm_tree* tb, int inner_m, int inner_maxit, cudaStream_t s) {
  if (inner_m < inner_maxit || !bnd_op_usable(tb, s)) return false;
  if (!bnd_op_cycle_planned(tb, inner_maxit)) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (cs != cudaStreamCaptureStatusNone) return false;
    if (bnd_op_cycle_ready(tb, inner_maxit, s) != HFMM_OK) return false;
  }
  return true;
}

// form of the inner solve's operator that a captured graph would hold
static int bnd_mode_of(fmm_tree* t) {
  const fmm_tree* b = t->inner ? t->inner : t;
  return (b->use_bnd_op && !t->bnd_op_suspend && bnd_op_planned(b)) ? 1 : 0;
}

template <typename V>
static int bnd_apply(fmm_tree* tb, const V* in, V* out, double scale, cudaStream_t s) {
  if (bnd_op_usable(tb, s)) {
    tb->timer.begin(HFMM_STAGE_BND, s);
    const int st = fmm_bnd_apply(tb, in, out, scale, s);
    tb->timer.end(1, s);
    return st;
  }
  HFMM_TRY(fmm_gather(tb, HFMM_SET_BND, nullptr, 0.0, in, scale, s));
  HFMM_TRY(fmm_core(tb, HFMM_SET_BND, HFMM_SET_BND, s));
  return fmm_scatter(tb, HFMM_SET_BND, nullptr, out, s);
}

static void prec_graph_drop(PrecGraph& G) {
  if (G.exec) cudaGraphExecDestroy(G.exec);
  G.exec = nullptr;
  for (auto& sl : G.slots) {
    cudaEventDestroy(sl.a);
    cudaEventDestroy(sl.b);
  }
  G.slots.clear();
  G.pending = false;
}

namespace {

void release(fmm_tree* t) {
  if (!t) return;
  for (auto& b : t->bufs) cudaFree(b.ptr);
  t->bufs.clear();
  if (t->ev0) cudaEventDestroy(t->ev0);
  if (t->ev1) cudaEventDestroy(t->ev1);
  if (t->ev_fork) cudaEventDestroy(t->ev_fork);
  if (t->ev_join) cudaEventDestroy(t->ev_join);
  if (t->near_stream) cudaStreamDestroy(t->near_stream);
  t->ev_fork = t->ev_join = nullptr;
  t->near_stream = nullptr;
  t->timer.destroy();
  m2l_tc_release(t);
  near_tc_release(t);
  bnd_op_release(t);
  if (t->gaunt) cudaFree(t->gaunt);
  t->gaunt = nullptr;
}

fmm_tree_ext* ext_of(fmm_tree* t) { return t->ext; }

std::atomic<int64_t> g_launches{0};

}  // namespace

void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

int tree_alloc(fmm_tree* t, void** ptr, size_t bytes) {
  *ptr = nullptr;
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return HFMM_ERR_NOMEM;
  }
  t->bufs.push_back({*ptr, bytes});
  t->device_bytes += (int64_t)bytes;
  return HFMM_OK;
}

extern "C" const char* hfmm_error_string(int status) {
  switch (status) {
    case HFMM_OK: return "ok";
    case HFMM_ERR_INVALID_ARG: return "invalid argument";
    case HFMM_ERR_CUDA: return "CUDA error";
    case HFMM_ERR_NOMEM: return "out of device memory";
    case HFMM_ERR_NONFINITE: return "non-finite value encountered";
    case HFMM_ERR_NOT_CONVERGED: return "iteration did not converge";
    case HFMM_ERR_TIMEOUT: return "timeout";
    case HFMM_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
  }
}

static int build_impl(fmm_tree* t, const double* d_vol, const double* d_bnd, cudaStream_t s) {
  const int P = t->P;
  // level offsets of the per-cell arrays
  int64_t off = 0;
  for (int l = 0; l <= t->L; ++l) {
    t->level_off[l] = off;
    off += (int64_t)1 << (3 * l);
  }
  t->level_off[t->L + 1] = off;
  t->total_cells = off;
  HFMM_TRY(tree_alloc_t(t, &t->level_off_dev, HFMM_MAX_LEVEL + 2));
  HFMM_CUDA_TRY(cudaMemcpyAsync(t->level_off_dev, t->level_off, sizeof(t->level_off),
                                cudaMemcpyHostToDevice, s));
  const int64_t nleaf = (int64_t)1 << (3 * t->L);
  const int64_t N = t->n_pts;
  HFMM_TRY(tree_alloc_t(t, &t->xyz, 3 * N));
  HFMM_TRY(tree_alloc_t(t, &t->xyz32, 4 * N));
  HFMM_TRY(tree_alloc_t(t, &t->orig, N));
  HFMM_TRY(tree_alloc_t(t, &t->pos_of, N));
  HFMM_TRY(tree_alloc_t(t, &t->leaf_start, nleaf + 1));
  HFMM_TRY(tree_alloc_t(t, &t->leaf_mid, nleaf));
  HFMM_TRY(tree_alloc_t(t, &t->flags, t->total_cells));
  const size_t csz = t->precision == HFMM_FP32 ? sizeof(float2) : sizeof(double2);
  HFMM_TRY(tree_alloc(t, &t->M, csz * t->total_cells * P));
  HFMM_TRY(tree_alloc(t, &t->Lc, csz * t->total_cells * P));
  HFMM_TRY(tree_alloc(t, &t->qs, csz * N));
  HFMM_TRY(tree_alloc(t, &t->phis, csz * N));
  HFMM_TRY(tree_alloc(t, &t->zero_row, csz * (P + 2)));
  HFMM_CUDA_TRY(cudaMemsetAsync(t->zero_row, 0, csz * (P + 2), s));
  // partial-sum buffers of split offset lists: 32 parts where they take at
  // most 256 MB, else 16 (the tensor-core M2L splits into at most 16)
  t->m2l_part_max = csz * t->total_cells * P * 32 <= ((size_t)256 << 20) ? 32 : 16;
  // M2L pipeline: the warp-specialised form wins once the operator is large
  // (p >= 8), the block-synchronous two-stage form below that (measured)
  t->m2l_variant = P >= 64 ? 1 : 0;
  if (const char* g = getenv("HFMM_GRAPHS")) t->use_graphs = atoi(g) != 0;
  if (const char* v = getenv("HFMM_M2L_VARIANT")) t->m2l_variant = atoi(v);
  if (const char* v = getenv("HFMM_LATTICE_P2P")) t->use_lattice_p2p = atoi(v) != 0;
  if (const char* v = getenv("HFMM_P2P_TILE")) t->lat_tile = atoi(v) != 0;
  if (const char* v = getenv("HFMM_BASIS_TABLE")) t->use_rtab = atoi(v) != 0;
  if (const char* v = getenv("HFMM_OVERLAP_NEAR")) t->overlap_near = atoi(v) != 0;
  if (const char* v = getenv("HFMM_M2L_TC")) t->use_m2l_tcore = atoi(v);
  if (const char* v = getenv("HFMM_NEAR_TC")) t->use_near_tcore = atoi(v);
  if (const char* v = getenv("HFMM_BND_OP")) t->use_bnd_op = atoi(v);
  // 1 (default): the one-kernel boundary operator where it was measured
  // faster than the stage chain (up to p = 6; at p = 8 the products are
  // bound by the FP32 FMA rate and the chain's kernels were faster)
  if (t->use_bnd_op == 1 && P > 36) t->use_bnd_op = 0;
  HFMM_TRY(tree_alloc(t, &t->m2l_part, csz * t->total_cells * P * t->m2l_part_max));
  HFMM_TRY(tree_alloc_t(t, &t->g_bnd, t->n_bnd + 1));
  HFMM_TRY(tree_alloc_t(t, &t->q_bnd, t->n_bnd + 1));
  if (t->precision == HFMM_FP32) {
    HFMM_TRY(tree_alloc_t(t, &t->g_bnd32, t->n_bnd + 1));
    HFMM_TRY(tree_alloc_t(t, &t->q_bnd32, t->n_bnd + 1));
  }
  HFMM_CUDA_TRY(cudaMemsetAsync(t->M, 0, csz * t->total_cells * P, s));
  HFMM_CUDA_TRY(cudaMemsetAsync(t->Lc, 0, csz * t->total_cells * P, s));
  HFMM_TRY(build_geometry_and_sort(t, d_vol, d_bnd, s));
  HFMM_TRY(build_lists(t, s));
  HFMM_TRY(build_self_terms(t, s));
  HFMM_TRY(build_operators(t, s));
  HFMM_TRY(build_pair_counts(t, s));
  HFMM_TRY(build_m2l_tiles(t, s));
  HFMM_TRY(build_active_lists(t, s));
  HFMM_TRY(build_lattice_table(t, s));
  HFMM_TRY(build_basis_table(t, s));
  HFMM_CUDA_TRY(cudaEventCreate(&t->ev0));
  HFMM_CUDA_TRY(cudaEventCreate(&t->ev1));
  HFMM_TRY(tree_alloc(t, &t->phis_near, csz * N));
  HFMM_CUDA_TRY(cudaStreamCreateWithFlags(&t->near_stream, cudaStreamNonBlocking));
  HFMM_CUDA_TRY(cudaEventCreateWithFlags(&t->ev_fork, cudaEventDisableTiming));
  HFMM_CUDA_TRY(cudaEventCreateWithFlags(&t->ev_join, cudaEventDisableTiming));
  HFMM_CUDA_TRY(cudaStreamSynchronize(s));
  return HFMM_OK;
}

extern "C" int fmm_build_tree(int n, const double* d_vol_xyz, int64_t n_vol, const double* d_bnd_xyz,
                              int64_t n_bnd, const hfmm_params* params, void* stream,
                              fmm_tree** out) {
  if (!out) return HFMM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!params) return HFMM_ERR_INVALID_ARG;
  const hfmm_params& pr = *params;
  if (pr.p < 1 || pr.p > HFMM_MAX_P) return HFMM_ERR_INVALID_ARG;
  if (!(pr.theta > 0.0 && pr.theta <= 0.55)) return HFMM_ERR_INVALID_ARG;
  if (pr.leaf_size < 1) return HFMM_ERR_INVALID_ARG;
  if (!(pr.k > 0.0) || !std::isfinite(pr.k)) return HFMM_ERR_INVALID_ARG;
  if (pr.precision != HFMM_FP64 && pr.precision != HFMM_FP32) return HFMM_ERR_INVALID_ARG;
  const bool lattice = d_vol_xyz == nullptr && d_bnd_xyz == nullptr;
  if (lattice) {
    if (n < 2 || n > 1024) return HFMM_ERR_INVALID_ARG;
    n_vol = (int64_t)n * n * n;
    n_bnd = 6 * (int64_t)n * n;
  } else {
    if (d_vol_xyz == nullptr || n_vol < 1 || n_bnd < 0 || (n_bnd > 0 && !d_bnd_xyz))
      return HFMM_ERR_INVALID_ARG;
  }
  if (n_vol + n_bnd > ((int64_t)1 << 30)) return HFMM_ERR_INVALID_ARG;
  fmm_tree* t = new (std::nothrow) fmm_tree();
  if (!t) return HFMM_ERR_NOMEM;
  t->ext = new (std::nothrow) fmm_tree_ext();
  if (!t->ext) {
    delete t;
    return HFMM_ERR_NOMEM;
  }
  t->n = lattice ? n : 0;
  t->lattice = lattice ? 1 : 0;
  t->n_vol = n_vol;
  t->n_bnd = n_bnd;
  t->n_pts = n_vol + n_bnd;
  t->h = lattice ? 1.0 / (n + 1) : 0.0;
  t->k = pr.k;
  t->p = pr.p;
  t->P = pr.p * pr.p;
  t->precision = pr.precision;
  t->leaf_size = pr.leaf_size;
  t->theta = pr.theta;
  theta_rational(pr.theta, t->th_num, t->th_den);
  int L = 2;
  while ((int64_t)pr.leaf_size * ((int64_t)1 << (3 * L)) < n_vol) ++L;
  if (L > HFMM_MAX_LEVEL - 1) {
    delete t->ext;
    delete t;
    return HFMM_ERR_UNSUPPORTED;
  }
  t->L = L;
  t->nlv = 1 << L;
  cudaStream_t s = (cudaStream_t)stream;
  int st = build_impl(t, d_vol_xyz, d_bnd_xyz, s);
  if (st != HFMM_OK) {
    cudaStreamSynchronize(s);
    cudaGetLastError();
    release(t);
    delete t->ext;
    delete t;
    return st;
  }
  *out = t;
  return HFMM_OK;
}

extern "C" void fmm_destroy_tree(fmm_tree* tree) {
  if (!tree) return;
  cudaDeviceSynchronize();
  fmm_tree_ext* e = ext_of(tree);
  gmres_work_free(e->inner);
  gmres_work_free(e->inner_g);
  gmres_work_free(e->inner32);
  gmres_work_free(e->inner_g32);
  gmres_work_free(e->outer);
  bicg_work_free(e->bicg);
  prec_graph_drop(e->pg);
  if (e->pg.cap) cudaStreamDestroy(e->pg.cap);
  if (tree->inner) fmm_destroy_tree(tree->inner);
  release(tree);
  delete e;
  delete tree;
}

extern "C" int fmm_apply(fmm_tree* t, int src_set, int tgt_set, const void* d_q_vol, const void* d_q_bnd,
                         void* d_phi_vol, void* d_phi_bnd, int mode, void* stream) {
  if (!t) return HFMM_ERR_INVALID_ARG;
  const int all = HFMM_SET_VOL | HFMM_SET_BND;
  if (src_set <= 0 || (src_set & ~all) || tgt_set <= 0 || (tgt_set & ~all)) return HFMM_ERR_INVALID_ARG;
  if (mode != HFMM_FWD && mode != HFMM_ADJ && mode != HFMM_DK && mode != HFMM_DLP) return HFMM_ERR_INVALID_ARG;
  if (mode == HFMM_DLP) {
    if (src_set != HFMM_SET_BND) return HFMM_ERR_INVALID_ARG;
    if (!t->lattice || t->n_bnd == 0) return HFMM_ERR_UNSUPPORTED;
  }
  const int in_set = mode == HFMM_ADJ ? tgt_set : src_set;
  const int out_set = mode == HFMM_ADJ ? src_set : tgt_set;
  if ((in_set & HFMM_SET_VOL) && !d_q_vol) return HFMM_ERR_INVALID_ARG;
  if ((in_set & HFMM_SET_BND) && t->n_bnd > 0 && !d_q_bnd) return HFMM_ERR_INVALID_ARG;
  if ((out_set & HFMM_SET_VOL) && !d_phi_vol) return HFMM_ERR_INVALID_ARG;
  if ((out_set & HFMM_SET_BND) && t->n_bnd > 0 && !d_phi_bnd) return HFMM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  HFMM_CUDA_TRY(cudaEventRecord(t->ev0, s));
  if (mode == HFMM_FWD && src_set == HFMM_SET_BND && tgt_set == HFMM_SET_BND && bnd_op_usable(t, s)) {
    t->timer.begin(HFMM_STAGE_BND, s);
    HFMM_TRY(fmm_bnd_apply(t, (const double2*)d_q_bnd, (double2*)d_phi_bnd, 1.0, s));
    t->timer.end(1, s);
    HFMM_CUDA_TRY(cudaEventRecord(t->ev1, s));
    return HFMM_OK;
  }
  HFMM_TRY(fmm_gather(t, in_set, (const double2*)d_q_vol, 1.0, (const double2*)d_q_bnd, 1.0, s));
  if (mode == HFMM_FWD) {
    HFMM_TRY(fmm_core(t, src_set, tgt_set, s));
    HFMM_TRY(fmm_scatter(t, out_set, (double2*)d_phi_vol, (double2*)d_phi_bnd, s));
  } else if (mode == HFMM_ADJ) {
    HFMM_TRY(fmm_core_adjoint(t, src_set, tgt_set, s));
    HFMM_TRY(fmm_scatter(t, out_set, (double2*)d_phi_vol, (double2*)d_phi_bnd, s));
  } else if (mode == HFMM_DLP) {
    HFMM_TRY(fmm_core_dlp(t, tgt_set, s));
    HFMM_TRY(fmm_scatter(t, out_set, (double2*)d_phi_vol, (double2*)d_phi_bnd, s));
  } else {
    HFMM_TRY(fmm_core_dk(t, src_set, tgt_set, s));
    HFMM_TRY(fmm_scatter_from(t, t->phis_d, out_set, (double2*)d_phi_vol, (double2*)d_phi_bnd, s));
  }
  HFMM_CUDA_TRY(cudaEventRecord(t->ev1, s));
  return HFMM_OK;
}

// smallest order >= p_min with p >= ceil(k rho_2) + 1, rho_2 = sqrt(3)/8 the
// half-diagonal of the level-2 cells of the unit cube (the coarsest level
// with M2L); raised to even
extern "C" int hfmm_order_for_k(double k, int p_min) {
  if (!(k >= 0.0) || !(k < 1e6) || p_min < 1 || p_min > HFMM_MAX_P) return HFMM_ERR_INVALID_ARG;
  const double rho2 = std::sqrt(3.0) / 8.0;
  int p = (int)std::ceil(k * rho2) + 1;
  if (p & 1) ++p;
  p = std::max(p, p_min);
  if (p > HFMM_MAX_P) return HFMM_ERR_UNSUPPORTED;
  return p;
}

static int grad_k_scratch(fmm_tree* t, bool phi) {
  fmm_tree_ext* e = ext_of(t);
  if (phi && !e->gk_phi) HFMM_TRY(tree_alloc(t, &e->gk_phi, sizeof(double2) * (size_t)t->n_vol));
  if (!e->gk_part) HFMM_TRY(tree_alloc(t, (void**)&e->gk_part, sizeof(double) * RE_DOT_PARTS));
  return HFMM_OK;
}

// dL/dk = Re sum_i conj(g_i) (dG~/dk q)_i on the volume points: the tangent
// apply into the handle's scratch, then a fixed-order device reduction
extern "C" int fmm_grad_k(fmm_tree* t, const void* d_q_vol, const void* d_g_vol, double* d_out, void* stream) {
  if (!t || !d_q_vol || !d_g_vol || !d_out || t->n_vol == 0) return HFMM_ERR_INVALID_ARG;
  HFMM_TRY(grad_k_scratch(t, true));
  fmm_tree_ext* e = ext_of(t);
  HFMM_TRY(fmm_apply(t, HFMM_SET_VOL, HFMM_SET_VOL, d_q_vol, nullptr, e->gk_phi, nullptr, HFMM_DK, stream));
  return re_dot_dev((const double2*)d_g_vol, (const double2*)e->gk_phi, t->n_vol, 1.0, e->gk_part, d_out,
                    (cudaStream_t)stream);
}

// dL/dk of x = A(k)^-1 b given the adjoint solution lam: A = A^T is real for
// real k and dA/dk = -2k I (Sec. 2), so dL/dk = -Re <lam, dA/dk x> = 2k Re <lam, x>
extern "C" int hfmm_solve_grad_k(fmm_tree* t, const void* d_lam, const void* d_x, double* d_out, void* stream) {
  if (!t || !d_lam || !d_x || !d_out) return HFMM_ERR_INVALID_ARG;
  if (!t->lattice) return HFMM_ERR_UNSUPPORTED;
  HFMM_TRY(grad_k_scratch(t, false));
  return re_dot_dev((const double2*)d_lam, (const double2*)d_x, (int64_t)t->n * t->n * t->n, 2.0 * t->k,
                    ext_of(t)->gk_part, d_out, (cudaStream_t)stream);
}

namespace {

// b_i = f_i + (1/h^2) sum of u_Gamma over the boundary neighbours of interior
// node i (7-point stencil with u = u_Gamma on the boundary nodes; those
// neighbours are the panel centres).  Node (ix, iy, iz), 1-based, x fastest;
// panel of face F = 2 axis + side at free coordinates (a, b) (first free
// coordinate fastest): F n^2 + (b - 1) n + (a - 1).
__global__ void k_dirichlet_rhs(int n, double inv_h2, const double2* __restrict__ f,
                                const double2* __restrict__ ub, double2* __restrict__ b) {
  const int64_t N = (int64_t)n * n * n;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int ix = (int)(i % n) + 1, iy = (int)((i / n) % n) + 1, iz = (int)(i / ((int64_t)n * n)) + 1;
  const int64_t nn = (int64_t)n * n;
  double sx = 0.0, sy = 0.0;
  auto add = [&](int face, int a, int c) {
    const double2 v = ub[face * nn + (int64_t)(c - 1) * n + (a - 1)];
    sx += v.x;
    sy += v.y;
  };
  if (ix == 1) add(0, iy, iz);
  if (ix == n) add(1, iy, iz);
  if (iy == 1) add(2, ix, iz);
  if (iy == n) add(3, ix, iz);
  if (iz == 1) add(4, ix, iy);
  if (iz == n) add(5, ix, iy);
  const double2 fi = f[i];
  b[i] = make_double2(fi.x + inv_h2 * sx, fi.y + inv_h2 * sy);
}

// g_i = g_i - u_i / 2 - d_i on the boundary (right-hand side of the inner
// solve with Dirichlet data, written for (-V) q = g)
template <typename R>
__global__ void k_bnd_data_rhs(int64_t n, C<R>* __restrict__ g, const double2* __restrict__ u,
                               const C<R>* __restrict__ dl) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const C<R> gi = g[i], di = dl[i];
  const double2 ui = u[i];
  g[i] = mkc<R>(gi.x - R(0.5 * ui.x) - di.x, gi.y - R(0.5 * ui.y) - di.y);
}

// z_i = z_i - d_i (interior, complex128)
__global__ void k_sub_inplace(int64_t n, double2* __restrict__ z, const double2* __restrict__ dl) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  z[i] = make_double2(z[i].x - dl[i].x, z[i].y - dl[i].y);
}

}  // namespace

extern "C" int hfmm_dirichlet_rhs(fmm_tree* t, const void* d_f, const void* d_u_bnd, void* d_b, void* stream) {
  if (!t || !d_f || !d_u_bnd || !d_b) return HFMM_ERR_INVALID_ARG;
  if (!t->lattice) return HFMM_ERR_UNSUPPORTED;
  const int64_t N = (int64_t)t->n * t->n * t->n;
  const double inv_h2 = 1.0 / (t->h * t->h);
  k_dirichlet_rhs<<<(unsigned)((N + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      t->n, inv_h2, (const double2*)d_f, (const double2*)d_u_bnd, (double2*)d_b);
  count_launches(1);
  return hfmm_last_launch();
}

// the inner boundary solve (-V) q = g (Sec. 5.2, Eq. (ubound); reading B4:
// GMRES from q = 0 to inner_rtol, at most inner_maxit steps, restart
// inner_m), V x = h^2 G_{Gamma,Gamma} x + s_Gamma x: one cycle inside the
// boundary operator's kernel when that applies, else the stage-by-stage
// GMRES; *inner_iters gets the steps taken (a host read)
template <typename R>
static int inner_solve(fmm_tree* t, fmm_tree* tb, GmresWorkT<R>& W, const C<R>* g, C<R>* q, double h2,
                       double inner_rtol, int inner_maxit, int inner_m, int* inner_iters, cudaStream_t s) {
  if (bnd_cycle_usable(tb, inner_m, inner_maxit, s)) {
    tb->timer.begin(HFMM_STAGE_BND, s);
    HFMM_TRY(fmm_bnd_cycle(tb, g, q, -h2, inner_maxit, inner_rtol, nullptr, s));
    tb->timer.end(1, s);
    int its = 0;
    HFMM_CUDA_TRY(cudaMemcpyAsync(&its, bnd_op_cycle_flags(tb) + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    HFMM_CUDA_TRY(cudaStreamSynchronize(s));
    if (inner_iters) *inner_iters = its;
    return HFMM_OK;
  }
  DevOpT<R> negV = [tb, h2, s](const C<R>* in, C<R>* out) -> int { return bnd_apply(tb, in, out, -h2, s); };
  HFMM_CUDA_TRY(cudaMemsetAsync(q, 0, sizeof(C<R>) * t->n_bnd, s));
  GmresResult ir;
  HFMM_TRY(gmres_run<R>(W, negV, nullptr, g, q, inner_m, inner_rtol, inner_maxit, true, false, &ir, nullptr, 0, s));
  if (inner_iters) *inner_iters = ir.iters;
  return HFMM_OK;
}

// z = M^-1 r (Sec. 5.2-5.3, homogeneous Dirichlet data).  The inner solve
// runs on complex vectors of real type R: the precision of the FMM form.
template <typename R>
static int precond_impl_t(fmm_tree* t, const double2* r, double2* z, double inner_rtol, int inner_maxit,
                          int inner_m, int* inner_iters, cudaStream_t s) {
  const double h = t->h, h2 = h * h, h3 = h2 * h;
  fmm_tree_ext* e = ext_of(t);
  GmresWorkT<R>& W = inner_ws(e, R(0), false);
  C<R>* g = bnd_g(t, R(0));
  C<R>* q = bnd_q(t, R(0));
  const double2* none = nullptr;
  // Pass A: g = G_{Gamma,Omega} (h^3 r)
  HFMM_TRY(fmm_gather(t, HFMM_SET_VOL, r, h3, none, 0.0, s));
  HFMM_TRY(fmm_core(t, HFMM_SET_VOL, HFMM_SET_BND, s));
  HFMM_TRY(fmm_scatter(t, HFMM_SET_BND, nullptr, g, s));
  // inner solve V q = -g with V x = h^2 G_{Gamma,Gamma} x + s_Gamma x (Pass B),
  // written as (-V) q = g
  HFMM_TRY(gmres_work_reserve(W, t->n_bnd, inner_m, false));
  fmm_tree* tb = pass_b_tree(t);
  HFMM_TRY(inner_solve<R>(t, tb, W, g, q, h2, inner_rtol, inner_maxit, inner_m, inner_iters, s));
  // Pass C: z = G_{Omega,Omega} (h^3 r) + G_{Omega,Gamma} (h^2 q) + s_Omega r
  HFMM_TRY(fmm_gather(t, HFMM_SET_VOL | HFMM_SET_BND, r, h3, q, h2, s));
  HFMM_TRY(fmm_core(t, HFMM_SET_VOL | HFMM_SET_BND, HFMM_SET_VOL, s));
  HFMM_TRY(fmm_scatter(t, HFMM_SET_VOL, z, (C<R>*)nullptr, s));
  if (fmm_device_error(s, true)) return HFMM_ERR_TIMEOUT;
  return HFMM_OK;
}

// u = BEM solution with volume data f and Dirichlet data u_Gamma (Sec. 5.2-5.3,
// Eq. (ubound) then Eq. (uinter)); the preconditioner's passes plus the
// double layer D (weights h^2 u_Gamma) and the jump u_Gamma / 2:
//   g = G_{Gamma,Omega} (h^3 f) - u_Gamma / 2 - D_{Gamma,Gamma} u_Gamma
//   solve (-V) q = g                                   (inner GMRES, Pass B)
//   u = G_{Omega,Omega} (h^3 f) + G_{Omega,Gamma} (h^2 q) + s_Omega f - D_{Omega,Gamma} u_Gamma
template <typename R>
static int bem_dirichlet_impl_t(fmm_tree* t, const double2* f, const double2* ub, double2* u, double inner_rtol,
                                int inner_maxit, int inner_m, int* inner_iters, cudaStream_t s) {
  const double h = t->h, h2 = h * h, h3 = h2 * h;
  fmm_tree_ext* e = ext_of(t);
  GmresWorkT<R>& W = inner_ws(e, R(0), false);
  C<R>* g = bnd_g(t, R(0));
  C<R>* q = bnd_q(t, R(0));
  if (!e->dl_work) HFMM_TRY(tree_alloc(t, &e->dl_work, sizeof(double2) * (size_t)std::max(t->n_vol, t->n_bnd)));
  const double2* none = nullptr;
  const unsigned gb = (unsigned)((t->n_bnd + 255) / 256), gv = (unsigned)((t->n_vol + 255) / 256);
  // g = N_{Gamma,Omega} f - u / 2 - D_{Gamma,Gamma} u
  HFMM_TRY(fmm_gather(t, HFMM_SET_VOL, f, h3, none, 0.0, s));
  HFMM_TRY(fmm_core(t, HFMM_SET_VOL, HFMM_SET_BND, s));
  HFMM_TRY(fmm_scatter(t, HFMM_SET_BND, nullptr, g, s));
  C<R>* dl_b = reinterpret_cast<C<R>*>(e->dl_work);
  HFMM_TRY(fmm_gather(t, HFMM_SET_BND, nullptr, 0.0, ub, h2, s));
  HFMM_TRY(fmm_core_dlp(t, HFMM_SET_BND, s));
  HFMM_TRY(fmm_scatter(t, HFMM_SET_BND, nullptr, dl_b, s));
  k_bnd_data_rhs<R><<<gb, 256, 0, s>>>(t->n_bnd, g, ub, dl_b);
  count_launches(1);
  HFMM_TRY(hfmm_last_launch());
  // (-V) q = g
  HFMM_TRY(gmres_work_reserve(W, t->n_bnd, inner_m, false));
  fmm_tree* tb = pass_b_tree(t);
  HFMM_TRY(inner_solve<R>(t, tb, W, g, q, h2, inner_rtol, inner_maxit, inner_m, inner_iters, s));
  // u = N_{Omega,Omega} f + V_{Omega,Gamma} q + s_Omega f - D_{Omega,Gamma} u_Gamma
  HFMM_TRY(fmm_gather(t, HFMM_SET_VOL | HFMM_SET_BND, f, h3, q, h2, s));
  HFMM_TRY(fmm_core(t, HFMM_SET_VOL | HFMM_SET_BND, HFMM_SET_VOL, s));
  HFMM_TRY(fmm_scatter(t, HFMM_SET_VOL, u, (C<R>*)nullptr, s));
  double2* dl_v = reinterpret_cast<double2*>(e->dl_work);
  HFMM_TRY(fmm_gather(t, HFMM_SET_BND, nullptr, 0.0, ub, h2, s));
  HFMM_TRY(fmm_core_dlp(t, HFMM_SET_VOL, s));
  HFMM_TRY(fmm_scatter(t, HFMM_SET_VOL, dl_v, (double2*)nullptr, s));
  k_sub_inplace<<<gv, 256, 0, s>>>(t->n_vol, u, dl_v);
  count_launches(1);
  HFMM_TRY(hfmm_last_launch());
  if (fmm_device_error(s, true)) return HFMM_ERR_TIMEOUT;
  return HFMM_OK;
}

static int precond_impl(fmm_tree* t, const double2* r, double2* z, double inner_rtol, int inner_maxit,
                        int inner_m, int* inner_iters, cudaStream_t s) {
  if (t->precision == HFMM_FP32)
    return precond_impl_t<float>(t, r, z, inner_rtol, inner_maxit, inner_m, inner_iters, s);
  return precond_impl_t<double>(t, r, z, inner_rtol, inner_maxit, inner_m, inner_iters, s);
}

// captured body of the preconditioner graph (all launches on stream c)
template <typename R>
static int prec_graph_body_t(fmm_tree* t, double rtol, int maxit, cudaStream_t c) {
  fmm_tree_ext* e = ext_of(t);
  PrecGraph& G = e->pg;
  GmresWorkT<R>& W = inner_ws(e, R(0), true);
  C<R>* g = bnd_g(t, R(0));
  C<R>* q = bnd_q(t, R(0));
  const double2* none = nullptr;
  const double h = t->h, h2 = h * h, h3 = h2 * h;
  HFMM_TRY(fmm_gather(t, HFMM_SET_VOL, G.r_in, h3, none, 0.0, c));
  HFMM_TRY(fmm_core(t, HFMM_SET_VOL, HFMM_SET_BND, c));
  HFMM_TRY(fmm_scatter(t, HFMM_SET_BND, nullptr, g, c));
  t->skip = G.flags;
  fmm_tree* tb = pass_b_tree(t);
  int st;
  if (bnd_cycle_usable(tb, maxit, maxit, c)) {  // one cycle inside the boundary operator's kernel
    tb->timer.begin(HFMM_STAGE_BND, c);
    st = fmm_bnd_cycle(tb, g, q, -h2, maxit, rtol, G.flags, c);
    tb->timer.end(1, c);
  } else {
    DevOpT<R> negV = [tb, h2, c](const C<R>* in, C<R>* out) -> int { return bnd_apply(tb, in, out, -h2, c); };
    st = gmres_cycle_device<R>(W, negV, g, q, maxit, rtol, G.flags, G.flags + 1, G.flags + 2, c);
  }
  t->skip = nullptr;
  if (tb != t) {
    tb->skip = nullptr;
    tb->timer.cap = nullptr;
  }
  HFMM_TRY(st);
  HFMM_TRY(fmm_gather(t, HFMM_SET_VOL | HFMM_SET_BND, G.r_in, h3, q, h2, c));
  HFMM_TRY(fmm_core(t, HFMM_SET_VOL | HFMM_SET_BND, HFMM_SET_VOL, c));
  return fmm_scatter(t, HFMM_SET_VOL, G.z_out, (C<R>*)nullptr, c);
}

static int prec_graph_body(fmm_tree* t, double rtol, int maxit, cudaStream_t c) {
  if (t->precision == HFMM_FP32) return prec_graph_body_t<float>(t, rtol, maxit, c);
  return prec_graph_body_t<double>(t, rtol, maxit, c);
}

static int prec_graph_build(fmm_tree* t, const double2* r, double2* z, double rtol, int maxit, cudaStream_t s) {
  fmm_tree_ext* e = ext_of(t);
  PrecGraph& G = e->pg;
  prec_graph_drop(G);
  // one eager apply builds everything the passes create on first use (its
  // result is the answer of this call; the first replay recomputes it)
  HFMM_TRY(precond_impl(t, r, z, rtol, maxit, maxit, &G.eager_its, s));
  if (!G.r_in) {
    HFMM_TRY(tree_alloc_t(t, &G.r_in, t->n_vol));
    HFMM_TRY(tree_alloc_t(t, &G.z_out, t->n_vol));
    HFMM_TRY(tree_alloc_t(t, &G.flags, 4));
    HFMM_CUDA_TRY(cudaMemsetAsync(G.flags, 0, 4 * sizeof(int), s));
  }
  if (!G.cap) HFMM_CUDA_TRY(cudaStreamCreateWithFlags(&G.cap, cudaStreamNonBlocking));
  if (t->precision == HFMM_FP32)
    HFMM_TRY(gmres_work_reserve(e->inner_g32, t->n_bnd, maxit, false));
  else
    HFMM_TRY(gmres_work_reserve(e->inner_g, t->n_bnd, maxit, false));
  HFMM_CUDA_TRY(cudaStreamSynchronize(s));
  cudaGraph_t graph = nullptr;
  HFMM_CUDA_TRY(cudaStreamBeginCapture(G.cap, cudaStreamCaptureModeThreadLocal));
  t->timer.cap = &G.slots;
  const int64_t before = launches_so_far();
  int st = prec_graph_body(t, rtol, maxit, G.cap);
  t->timer.cap = nullptr;
  G.kernels = launches_so_far() - before;
  count_launches(-G.kernels);  // captured, not executed
  cudaError_t ce = cudaStreamEndCapture(G.cap, &graph);
  if (st != HFMM_OK || ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    prec_graph_drop(G);
    return st != HFMM_OK ? st : HFMM_ERR_CUDA;
  }
  ce = cudaGraphInstantiate(&G.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) {
    G.exec = nullptr;
    cudaGetLastError();
    return HFMM_ERR_CUDA;
  }
  G.rtol = rtol;
  G.maxit = maxit;
  G.timer_mask = t->timer.on ? t->timer.mask : 0;
  G.bnd_mode = bnd_mode_of(t);
  return HFMM_OK;
}

// z = M^-1 r through the graph (rebuilt when the inner settings or the
// timed stages change)
static int precond_graph(fmm_tree* t, const double2* r, double2* z, double rtol, int maxit, cudaStream_t s) {
  PrecGraph& G = ext_of(t)->pg;
  const int tmask = t->timer.on ? t->timer.mask : 0;
  if (G.pending) {  // the previous replay has completed: the caller synchronised since
    t->timer.resolve_slots(G.slots);
    G.pending = false;
  }
  if (!G.exec || G.rtol != rtol || G.maxit != maxit || G.timer_mask != tmask || G.bnd_mode != bnd_mode_of(t))
    HFMM_TRY(prec_graph_build(t, r, z, rtol, maxit, s));
  HFMM_CUDA_TRY(cudaMemcpyAsync(G.r_in, r, sizeof(double2) * t->n_vol, cudaMemcpyDeviceToDevice, s));
  HFMM_CUDA_TRY(cudaGraphLaunch(G.exec, s));
  HFMM_CUDA_TRY(cudaMemcpyAsync(z, G.z_out, sizeof(double2) * t->n_vol, cudaMemcpyDeviceToDevice, s));
  G.pending = !G.slots.empty();
  count_launches(G.kernels);
  return HFMM_OK;
}

extern "C" int fmm_precond_apply(fmm_tree* t, const void* d_r, void* d_z, double inner_rtol,
                                 int inner_maxit, int inner_m, int* inner_iters, void* stream) {
  if (!t || !d_r || !d_z) return HFMM_ERR_INVALID_ARG;
  if (!t->lattice) return HFMM_ERR_UNSUPPORTED;
  if (!(inner_rtol > 0.0) || inner_maxit < 1 || inner_m < 1 || inner_m > 500) return HFMM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  HFMM_CUDA_TRY(cudaEventRecord(t->ev0, s));
  HFMM_TRY(precond_impl(t, (const double2*)d_r, (double2*)d_z, inner_rtol, inner_maxit, inner_m,
                        inner_iters, s));
  HFMM_CUDA_TRY(cudaEventRecord(t->ev1, s));
  return HFMM_OK;
}

extern "C" int bem_solve_dirichlet(fmm_tree* t, const void* d_f, const void* d_u_bnd, void* d_u, double inner_rtol,
                                   int inner_maxit, int inner_m, int* inner_iters, void* stream) {
  if (!t || !d_f || !d_u_bnd || !d_u) return HFMM_ERR_INVALID_ARG;
  if (!t->lattice || t->n_bnd == 0) return HFMM_ERR_UNSUPPORTED;
  if (!(inner_rtol > 0.0) || inner_maxit < 1 || inner_m < 1 || inner_m > 500) return HFMM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  HFMM_CUDA_TRY(cudaEventRecord(t->ev0, s));
  if (t->precision == HFMM_FP32)
    HFMM_TRY(bem_dirichlet_impl_t<float>(t, (const double2*)d_f, (const double2*)d_u_bnd, (double2*)d_u,
                                         inner_rtol, inner_maxit, inner_m, inner_iters, s));
  else
    HFMM_TRY(bem_dirichlet_impl_t<double>(t, (const double2*)d_f, (const double2*)d_u_bnd, (double2*)d_u,
                                          inner_rtol, inner_maxit, inner_m, inner_iters, s));
  HFMM_CUDA_TRY(cudaEventRecord(t->ev1, s));
  return HFMM_OK;
}

extern "C" int hfmm_fdm_apply(fmm_tree* t, const void* d_u, void* d_out, void* stream) {
  if (!t || !d_u || !d_out) return HFMM_ERR_INVALID_ARG;
  if (!t->lattice) return HFMM_ERR_UNSUPPORTED;
  return fdm_apply_dev(t->n, t->h, t->k, (const double2*)d_u, (double2*)d_out, (cudaStream_t)stream);
}

extern "C" int gmres_solve(fmm_tree* t, const void* d_b, void* d_x, const hfmm_gmres_params* gp,
                           hfmm_gmres_info* info, void* stream) {
  if (!t || !d_b || !d_x || !gp) return HFMM_ERR_INVALID_ARG;
  if (!t->lattice) return HFMM_ERR_UNSUPPORTED;
  if (gp->restart_m < 1 || gp->restart_m > 200 || !(gp->rtol > 0.0) || gp->maxit < 0 ||
      !(gp->inner_rtol > 0.0) || gp->inner_maxit < 1 || gp->inner_m < 1 || gp->inner_m > 500)
    return HFMM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  fmm_tree_ext* e = ext_of(t);
  const int64_t N = t->n_vol;
  HFMM_TRY(gmres_work_reserve(e->outer, N, gp->restart_m, true));
  DevOp A = [t, s](const double2* in, double2* out) -> int {
    t->timer.begin(HFMM_STAGE_FDM, s);
    int st = fdm_apply_dev(t->n, t->h, t->k, in, out, s);
    t->timer.end(1, s);
    return st;
  };
  int inner_total = 0;
  const bool graphs = t->use_graphs && gp->inner_m >= gp->inner_maxit;
  PrecGraph& G = e->pg;
  if (graphs && G.flags) HFMM_CUDA_TRY(cudaMemsetAsync(G.flags + 2, 0, sizeof(int), s));
  G.eager_its = 0;
  DevOp M = [t, gp, s, graphs, &inner_total](const double2* in, double2* out) -> int {
    if (graphs) return precond_graph(t, in, out, gp->inner_rtol, gp->inner_maxit, s);
    int its = 0;
    int st = precond_impl(t, in, out, gp->inner_rtol, gp->inner_maxit, gp->inner_m, &its, s);
    inner_total += its;
    return st;
  };
  const int maxit = gp->maxit > 0 ? gp->maxit : 20 * gp->restart_m;
  GmresResult R;
  int st = gmres_run(e->outer, A, &M, (const double2*)d_b, (double2*)d_x, gp->restart_m, gp->rtol, maxit,
                     false, true, &R, info ? info->history : nullptr, info ? info->history_len : 0, s);
  if (graphs && st == HFMM_OK && G.flags) {
    // inner steps of the graph replays (the first apply ran eagerly when the
    // graph was built and counted nothing there)
    int tot = 0;
    HFMM_CUDA_TRY(cudaMemcpyAsync(&tot, G.flags + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
    HFMM_CUDA_TRY(cudaStreamSynchronize(s));
    // the replay that follows an eager build recomputes that apply: its steps
    // are in `tot` already, so the eager count is not added again
    inner_total = tot;
    if (G.pending) {
      t->timer.resolve_slots(G.slots);
      G.pending = false;
    }
    if (fmm_device_error(s, true)) st = HFMM_ERR_TIMEOUT;
  }
  if (info) {
    info->iters = R.iters;
    info->restarts = R.restarts;
    info->inner_iters_total = inner_total;
    info->relres_est = R.relres_est;
    info->relres_true = R.relres_true;
    info->status = st != HFMM_OK ? st : (R.converged ? HFMM_OK : HFMM_ERR_NOT_CONVERGED);
  }
  if (st != HFMM_OK) return st;
  return R.converged ? HFMM_OK : HFMM_ERR_NOT_CONVERGED;
}

extern "C" int bicgstab_solve(fmm_tree* t, const void* d_b, void* d_x, const hfmm_gmres_params* gp,
                              hfmm_gmres_info* info, void* stream) {
  if (!t || !d_b || !d_x || !gp) return HFMM_ERR_INVALID_ARG;
  if (!t->lattice) return HFMM_ERR_UNSUPPORTED;
  if (!(gp->rtol > 0.0) || gp->maxit < 0 || !(gp->inner_rtol > 0.0) || gp->inner_maxit < 1 || gp->inner_m < 1 ||
      gp->inner_m > 500)
    return HFMM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  fmm_tree_ext* e = ext_of(t);
  HFMM_TRY(bicg_work_reserve(e->bicg, t->n_vol));
  DevOp A = [t, s](const double2* in, double2* out) -> int {
    t->timer.begin(HFMM_STAGE_FDM, s);
    int st = fdm_apply_dev(t->n, t->h, t->k, in, out, s);
    t->timer.end(1, s);
    return st;
  };
  int inner_total = 0;
  const bool graphs = t->use_graphs && gp->inner_m >= gp->inner_maxit;
  PrecGraph& G = e->pg;
  if (graphs && G.flags) HFMM_CUDA_TRY(cudaMemsetAsync(G.flags + 2, 0, sizeof(int), s));
  G.eager_its = 0;
  DevOp M = [t, gp, s, graphs, &inner_total](const double2* in, double2* out) -> int {
    if (graphs) return precond_graph(t, in, out, gp->inner_rtol, gp->inner_maxit, s);
    int its = 0;
    int st = precond_impl(t, in, out, gp->inner_rtol, gp->inner_maxit, gp->inner_m, &its, s);
    inner_total += its;
    return st;
  };
  const int maxit = gp->maxit > 0 ? gp->maxit : 500;
  BicgResult R;
  int st = bicgstab_run(e->bicg, A, &M, (const double2*)d_b, (double2*)d_x, gp->rtol, maxit, false, &R,
                        info ? info->history : nullptr, info ? info->history_len : 0, s);
  if (graphs && st == HFMM_OK && G.flags) {
    int tot = 0;
    HFMM_CUDA_TRY(cudaMemcpyAsync(&tot, G.flags + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
    HFMM_CUDA_TRY(cudaStreamSynchronize(s));
    inner_total = tot;
    if (G.pending) {
      t->timer.resolve_slots(G.slots);
      G.pending = false;
    }
    if (fmm_device_error(s, true)) st = HFMM_ERR_TIMEOUT;
  }
  if (info) {
    info->iters = R.iters;
    info->restarts = R.precond_applies;
    info->inner_iters_total = inner_total;
    info->relres_est = R.relres_est;
    info->relres_true = R.relres_true;
    info->status = st != HFMM_OK ? st : (R.converged ? HFMM_OK : HFMM_ERR_NOT_CONVERGED);
  }
  if (st != HFMM_OK) return st;
  return R.converged ? HFMM_OK : HFMM_ERR_NOT_CONVERGED;
}

extern "C" int fmm_get_stats(const fmm_tree* t, hfmm_stats* st) {
  if (!t || !st) return HFMM_ERR_INVALID_ARG;
  st->L = t->L;
  st->p = t->p;
  st->n_vol = t->n_vol;
  st->n_bnd = t->n_bnd;
  st->leaves = (int64_t)1 << (3 * t->L);
  st->m2l_pairs = t->m2l_pairs;
  st->p2p_pairs = t->p2p_pairs;
  st->device_bytes = t->device_bytes;
  float ms = 0.f;
  fmm_tree* tt = const_cast<fmm_tree*>(t);
  if (tt->ev0 && tt->ev1 && cudaEventElapsedTime(&ms, tt->ev0, tt->ev1) == cudaSuccess)
    tt->ms_last_apply = ms;
  else
    cudaGetLastError();
  st->ms_last_apply = tt->ms_last_apply;
  tt->timer.flush();
  if (tt->ext && tt->ext->pg.pending) {
    tt->timer.resolve_slots(tt->ext->pg.slots);
    tt->ext->pg.pending = false;
  }
  st->launches = launches_so_far();
  for (int i = 0; i < HFMM_NSTAGES; ++i) {
    st->stage_ms[i] = tt->timer.ms[i];
    st->stage_launches[i] = tt->timer.launches[i];
    st->stage_work[i] = tt->timer.work[i];
  }
  if (tt->inner) {  // stages of the inner solve's applies timed eagerly on the auxiliary tree
    tt->inner->timer.flush();
    for (int i = 0; i < HFMM_NSTAGES; ++i) {
      st->stage_ms[i] += tt->inner->timer.ms[i];
      st->stage_launches[i] += tt->inner->timer.launches[i];
      st->stage_work[i] += tt->inner->timer.work[i];
    }
    st->device_bytes += tt->inner->device_bytes;
  }
  return HFMM_OK;
}

extern "C" int fmm_use_graphs(fmm_tree* t, int enable) {
  if (!t || (enable != 0 && enable != 1)) return HFMM_ERR_INVALID_ARG;
  t->use_graphs = enable;
  return HFMM_OK;
}

extern "C" int fmm_set_timing(fmm_tree* t, int stage_mask) {
  if (!t || stage_mask < 0 || stage_mask >= (1 << HFMM_NSTAGES)) return HFMM_ERR_INVALID_ARG;
  t->timer.reset();
  t->timer.on = stage_mask != 0;
  t->timer.mask = stage_mask;
  if (t->inner) {
    t->inner->timer.reset();
    t->inner->timer.on = t->timer.on;
    t->inner->timer.mask = stage_mask;
  }
  return HFMM_OK;
}

extern "C" int fmm_set_inner_order(fmm_tree* t, int p_inner, void* stream) {
  if (!t || p_inner < 0 || p_inner > HFMM_MAX_P) return HFMM_ERR_INVALID_ARG;
  if (p_inner != 0 && p_inner != t->p && !t->lattice) return HFMM_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  HFMM_CUDA_TRY(cudaStreamSynchronize(s));
  prec_graph_drop(ext_of(t)->pg);  // the captured inner solve used the previous tree
  if (t->inner) {
    fmm_destroy_tree(t->inner);
    t->inner = nullptr;
  }
  t->inner_p = 0;
  if (p_inner == 0 || p_inner == t->p) return HFMM_OK;
  hfmm_params prm;
  prm.p = p_inner;
  prm.theta = t->theta;
  prm.leaf_size = t->leaf_size;
  prm.k = t->k;
  prm.precision = t->precision;
  fmm_tree* aux = nullptr;
  HFMM_TRY(fmm_build_tree(t->n, nullptr, 0, nullptr, 0, &prm, stream, &aux));
  t->inner = aux;
  t->inner_p = p_inner;
  return HFMM_OK;
}
