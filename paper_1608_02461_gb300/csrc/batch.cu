// Batched solves and the M2L autotuner.
//
// gmres_solve_batched runs many independent preconditioned solves (uneven
// grid sizes and wavenumbers, one tree each) concurrently: worker host
// threads take solves from a shared counter and drive each on their own CUDA
// stream, so that the small, latency-bound kernels of different solves
// overlap on the GPU.  The caller's stream is ordered before and after the
// batch with events.
//
// fmm_autotune times the M2L kernel variants (two-stage block pipeline,
// warp-specialised three-stage pipeline, pair lists) and the split of the offset lists
// (grid filled to 1, 2, 4 or 8 times the SM count) on the FMM passes the
// preconditioner uses, then, with that M2L, the shapes of the lattice near
// field (tiled 4 x 4 target-source groups or not, at most 8, 16 or 32
// threads per target group, one block per SM or as many as fit) and whether
// the near field runs concurrently with the far field, and keeps the fastest
// per pass in the handle.
#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

#include "tree.cuh"

namespace {

int time_core(fmm_tree* t, int src, int tgt, cudaStream_t s, int reps, float* ms) {
  cudaEvent_t a, b;
  HFMM_CUDA_TRY(cudaEventCreate(&a));
  HFMM_CUDA_TRY(cudaEventCreate(&b));
  int st = fmm_core(t, src, tgt, s);  // warm (valid lists, operators)
  if (st == HFMM_OK) st = fmm_core(t, src, tgt, s);
  if (st == HFMM_OK) {
    cudaEventRecord(a, s);
    for (int r = 0; r < reps && st == HFMM_OK; ++r) st = fmm_core(t, src, tgt, s);
    cudaEventRecord(b, s);
    if (cudaEventSynchronize(b) != cudaSuccess) st = HFMM_ERR_CUDA;
    if (st == HFMM_OK) cudaEventElapsedTime(ms, a, b);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return st;
}

}  // namespace

extern "C" int fmm_autotune(fmm_tree* t, void* stream) {
  if (!t) return HFMM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t csz = t->precision == HFMM_FP32 ? sizeof(float2) : sizeof(double2);
  HFMM_CUDA_TRY(cudaMemsetAsync(t->qs, 0, csz * t->n_pts, s));
  const int passes[4][2] = {{HFMM_SET_VOL, HFMM_SET_BND},
                            {HFMM_SET_BND, HFMM_SET_BND},
                            {HFMM_SET_VOL | HFMM_SET_BND, HFMM_SET_VOL},
                            {HFMM_SET_VOL | HFMM_SET_BND, HFMM_SET_VOL | HFMM_SET_BND}};
  const int fills[5] = {1, 2, 4, 8, 16};
  const bool timer_was_on = t->timer.on;
  t->timer.on = false;
  for (const auto& ps : passes) {
    const int src = ps[0], tgt = ps[1];
    if (t->n_bnd == 0 && ((src | tgt) & HFMM_SET_BND)) continue;
    const int ci = (tgt - 1) * 3 + (src - 1);
    float best = 1e30f;
    int bv = -1, bf = 0;
    for (int v = 0; v < 3; ++v)
      for (int f : fills) {
        if (v == 2 && f != fills[0]) continue;  // the pair-list form has no split
        t->tuned_variant[ci] = v;
        t->tuned_fill[ci] = f;
        float ms = 0.f;
        int st = time_core(t, src, tgt, s, 3, &ms);
        if (st != HFMM_OK) {
          t->timer.on = timer_was_on;
          return st;
        }
        if (ms < best) {
          best = ms;
          bv = v;
          bf = f;
        }
      }
    t->tuned_variant[ci] = bv;
    t->tuned_fill[ci] = bf;
    // near-field shapes (lattice trees whose near field goes through the table)
    const bool lat = t->lat_D > 0 && t->use_lattice_p2p && t->near_count <= 128 &&
                     (t->precision == HFMM_FP32 || t->lat_tab64_fits);
    if (!lat) continue;
    best = 1e30f;
    int btile = 0, btpt = 32, bblk = 0;
    const int ntile = t->precision == HFMM_FP32 ? 2 : 1;
    for (int tile = 0; tile < ntile; ++tile)
      for (int tpt : {8, 16, 32})
        for (int blk : {1, 0}) {
          t->tuned_p2p_tile[ci] = tile;
          t->tuned_p2p_tpt[ci] = tpt;
          t->tuned_p2p_blocks[ci] = blk;
          float ms = 0.f;
          int st = time_core(t, src, tgt, s, 3, &ms);
          if (st != HFMM_OK) {
            t->timer.on = timer_was_on;
            return st;
          }
          if (ms < best) {
            best = ms;
            btile = tile;
            btpt = tpt;
            bblk = blk;
          }
        }
    t->tuned_p2p_tile[ci] = btile;
    t->tuned_p2p_tpt[ci] = btpt;
    t->tuned_p2p_blocks[ci] = bblk;
    // near field concurrent with the far field or after it
    if (!t->overlap_near || !t->near_stream || !t->phis_near) continue;
    best = 1e30f;
    int bov = -1;
    for (int ov = 0; ov < 2; ++ov) {
      t->tuned_overlap[ci] = ov;
      float ms = 0.f;
      int st = time_core(t, src, tgt, s, 3, &ms);
      if (st != HFMM_OK) {
        t->timer.on = timer_was_on;
        return st;
      }
      if (ms < best) {
        best = ms;
        bov = ov;
      }
    }
    t->tuned_overlap[ci] = bov;
  }
  t->timer.on = timer_was_on;
  if (t->inner) return fmm_autotune(t->inner, stream);  // the inner solve's tree
  return HFMM_OK;
}

extern "C" int gmres_solve_batched(fmm_tree** trees, const void** d_b, void** d_x, int count,
                                   const hfmm_gmres_params* gp, hfmm_gmres_info* infos, void* stream) {
  if (count < 0 || !gp || (count > 0 && (!trees || !d_b || !d_x))) return HFMM_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i)
    if (!trees[i] || !d_b[i] || !d_x[i]) return HFMM_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i)
    for (int j = i + 1; j < count; ++j)
      if (trees[i] == trees[j]) return HFMM_ERR_INVALID_ARG;  // a handle is not thread safe
  if (count == 0) return HFMM_OK;
  int dev = 0;
  HFMM_CUDA_TRY(cudaGetDevice(&dev));
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t start;
  HFMM_CUDA_TRY(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  HFMM_CUDA_TRY(cudaEventRecord(start, s));
  const int nw = std::min(count, 8);
  // concurrent solves keep the stage chain for their inner solves (the
  // boundary operator's cooperative kernel wants every SM to itself)
  std::vector<int> was_suspended(count);
  for (int i = 0; i < count; ++i) {
    was_suspended[i] = trees[i]->bnd_op_suspend;
    if (nw > 1) trees[i]->bnd_op_suspend = 1;
  }
  std::atomic<int> next{0};
  std::vector<int> status(count, HFMM_OK);
  std::vector<cudaEvent_t> done(nw, nullptr);
  std::vector<int> wstatus(nw, HFMM_OK);
  auto worker = [&](int w) {
    if (cudaSetDevice(dev) != cudaSuccess) {
      wstatus[w] = HFMM_ERR_CUDA;
      return;
    }
    cudaStream_t ws;
    if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess) {
      wstatus[w] = HFMM_ERR_CUDA;
      return;
    }
    cudaStreamWaitEvent(ws, start, 0);
    for (int i = next.fetch_add(1); i < count; i = next.fetch_add(1))
      status[i] = gmres_solve(trees[i], d_b[i], d_x[i], gp, infos ? &infos[i] : nullptr, ws);
    if (cudaEventCreateWithFlags(&done[w], cudaEventDisableTiming) == cudaSuccess)
      cudaEventRecord(done[w], ws);
    else
      wstatus[w] = HFMM_ERR_CUDA;
    cudaStreamDestroy(ws);  // returns at once; the stream is released when its work completes
  };
  std::vector<std::thread> pool;
  for (int w = 0; w < nw; ++w) pool.emplace_back(worker, w);
  for (auto& th : pool) th.join();
  for (int i = 0; i < count; ++i) trees[i]->bnd_op_suspend = was_suspended[i];
  int rc = HFMM_OK;
  for (int w = 0; w < nw; ++w) {
    if (done[w]) {
      cudaStreamWaitEvent(s, done[w], 0);
      cudaEventDestroy(done[w]);
    }
    if (wstatus[w] != HFMM_OK && rc == HFMM_OK) rc = wstatus[w];
  }
  cudaEventDestroy(start);
  // first hard error, else NOT_CONVERGED when any solve did not converge or
  // broke down on a non-finite value (a numerical outcome of that solve alone,
  // reported in its info; the other solves' results stand)
  auto solve_failed = [](int st) { return st == HFMM_ERR_NOT_CONVERGED || st == HFMM_ERR_NONFINITE; };
  for (int i = 0; i < count && rc == HFMM_OK; ++i)
    if (status[i] != HFMM_OK && !solve_failed(status[i])) rc = status[i];
  if (rc == HFMM_OK)
    for (int i = 0; i < count; ++i)
      if (solve_failed(status[i])) rc = HFMM_ERR_NOT_CONVERGED;
  return rc;
}
