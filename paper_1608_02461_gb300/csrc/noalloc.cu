// Direct Helmholtz sum that allocates no device memory.
//
// Some callers cannot allocate device memory: code running inside another
// framework's memory pool with cudaMalloc forbidden, allocation-free
// real-time paths, or a stream that is being captured where allocation would
// break the capture.  hfmm_direct_sum_noalloc serves them: the caller passes
// the inputs and the output, and the only scratch space (partial sums of the
// source chunks) lives in a fixed-size array in this library's device memory.
// This entry point has no counterpart in the paper; it is a split-source
// variant of the near-field (P2P) kernel applied to whole point sets.
#include <mutex>

#include "common.cuh"

namespace {

// Scratch: partial potentials [chunk][target], complex128.  Every device that
// loads the library holds this array (4 MiB) until the process exits.
constexpr int64_t kScratchEntries = int64_t(1) << 18;
static __device__ __align__(256) double2 g_noalloc_scratch[kScratchEntries];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
double2* g_scratch_ptr[kMaxDevices] = {};

constexpr int kThreads = 128;
constexpr int kTile = 256;
constexpr int64_t kChunkMin = 1024;  // sources per chunk at least
constexpr int kMaxChunks = 32;

// block (target block, chunk): potentials of kThreads targets from the
// sources of one chunk, tiled through shared memory
__global__ void k_direct_chunk(int64_t n_src, const double* __restrict__ sx, const double2* __restrict__ q,
                               int64_t n_tgt, const double* __restrict__ tx, double k, int64_t chunk_len,
                               double2* __restrict__ part) {
  __shared__ double ps[kTile][3];
  __shared__ double2 pq[kTile];
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  const int64_t c = blockIdx.y;
  const int64_t jb = c * chunk_len, je = min(n_src, jb + chunk_len);
  double xi = 0, yi = 0, zi = 0;
  if (i < n_tgt) {
    xi = tx[3 * i];
    yi = tx[3 * i + 1];
    zi = tx[3 * i + 2];
  }
  double2 acc = make_double2(0, 0);
  const double inv4pi = 0.07957747154594766788;
  for (int64_t j0 = jb; j0 < je; j0 += kTile) {
    __syncthreads();
    for (int e = threadIdx.x; e < kTile && j0 + e < je; e += kThreads) {
      ps[e][0] = sx[3 * (j0 + e)];
      ps[e][1] = sx[3 * (j0 + e) + 1];
      ps[e][2] = sx[3 * (j0 + e) + 2];
      pq[e] = q[j0 + e];
    }
    __syncthreads();
    const int cnt = (int)min((int64_t)kTile, je - j0);
    if (i < n_tgt) {
      for (int e = 0; e < cnt; ++e) {
        double dx = xi - ps[e][0], dy = yi - ps[e][1], dz = zi - ps[e][2];
        double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 == 0.0) continue;  // a point does not act on itself
        double r = sqrt(r2);
        double sn, cs;
        sincos(k * r, &sn, &cs);
        double g = inv4pi / r;
        double gr = cs * g, gi = sn * g;
        acc.x += gr * pq[e].x - gi * pq[e].y;
        acc.y += gr * pq[e].y + gi * pq[e].x;
      }
    }
  }
  if (i < n_tgt) part[c * n_tgt + i] = acc;
}

// phi_i = sum over chunks in chunk order (deterministic)
__global__ void k_direct_reduce(int64_t n_tgt, int nchunks, const double2* __restrict__ part,
                                double2* __restrict__ phi) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_tgt) return;
  double2 s = part[i];
  for (int c = 1; c < nchunks; ++c) {
    double2 v = part[c * n_tgt + i];
    s.x += v.x;
    s.y += v.y;
  }
  phi[i] = s;
}

// device address of the scratch array for the current device.  The first
// call on each device looks it up (a first call on a stream that is being
// captured is refused); later calls on a stream that is not being captured
// look it up again, because a device reset or a recreated primary context
// moves the array and a cached address would then be stale.
int scratch_for_current_device(cudaStream_t s, double2** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HFMM_ERR_CUDA;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    cudaGetLastError();
    cap = cudaStreamCaptureStatusActive;  // unknown: do not call the runtime's symbol lookup
  }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev] || cap == cudaStreamCaptureStatusNone) {
    if (cap != cudaStreamCaptureStatusNone) return HFMM_ERR_UNSUPPORTED;  // first call inside a capture
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return HFMM_ERR_CUDA;
    }
    g_scratch_ptr[dev] = reinterpret_cast<double2*>(p);
  }
  *out = g_scratch_ptr[dev];
  return HFMM_OK;
}

}  // namespace

extern "C" int hfmm_direct_sum_noalloc(int64_t n_src, const double* d_src_xyz, const void* d_q,
                                       int64_t n_tgt, const double* d_tgt_xyz, double k, void* d_phi,
                                       void* stream) {
  if (n_src < 0 || n_tgt < 0 || !(k >= 0.0)) return HFMM_ERR_INVALID_ARG;
  if (n_tgt == 0) return HFMM_OK;
  if (!d_tgt_xyz || !d_phi || (n_src > 0 && (!d_src_xyz || !d_q))) return HFMM_ERR_INVALID_ARG;
  if (n_tgt > kScratchEntries) return HFMM_ERR_INVALID_ARG;  // beyond the scratch maximum
  // chunks of the source set: enough blocks to fill the GPU, bounded by the
  // scratch size (n_tgt x nchunks entries)
  int64_t nchunks = n_src / kChunkMin;
  if (nchunks < 1) nchunks = 1;
  if (nchunks > kMaxChunks) nchunks = kMaxChunks;
  if (nchunks * n_tgt > kScratchEntries) nchunks = kScratchEntries / n_tgt;
  const int64_t chunk_len = n_src > 0 ? (n_src + nchunks - 1) / nchunks : 1;
  cudaStream_t s = (cudaStream_t)stream;
  double2* scratch = nullptr;
  HFMM_TRY(scratch_for_current_device(s, &scratch));
  dim3 grid(ceil_div(n_tgt, kThreads), (unsigned)nchunks);
  k_direct_chunk<<<grid, kThreads, 0, s>>>(n_src, d_src_xyz, (const double2*)d_q, n_tgt, d_tgt_xyz, k,
                                           chunk_len, scratch);
  k_direct_reduce<<<ceil_div(n_tgt, 256), 256, 0, s>>>(n_tgt, (int)nchunks, scratch, (double2*)d_phi);
  return hfmm_last_launch();
}
