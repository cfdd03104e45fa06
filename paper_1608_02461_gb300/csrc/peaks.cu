// Pipe-rate probe: the measured throughput of the arithmetic pipes that bound
// the solver's kernels, for the roofline denominators (FP32 FMA for the near
// field and the CUDA-core M2L, FP64 FMA for the FP64 form, the XU for the
// per-pair sin/cos/rsqrt of a direct evaluation, shared-memory loads for the
// table-driven lattice near field, tcgen05 kind::tf32 for the tensor-core
// M2L).  Each rate is the best of a few timed launches (CUDA events) of a
// kernel that keeps one pipe busy on every SM; the GPU's clocks are left as
// they are.
#include <algorithm>

#include "common.cuh"
#include "tc.cuh"

namespace {

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;  // independent dependency chains per thread

// a * b + c on PK_CHAINS chains; the result is written only if it takes an
// impossible value, which keeps every chain live
template <typename T>
__global__ void __launch_bounds__(PK_THREADS) k_peak_fma(int iters, T* out) {
  T a[PK_CHAINS];
#pragma unroll
  for (int i = 0; i < PK_CHAINS; ++i) a[i] = T(1) + T(1e-3) * (T)(threadIdx.x + i);
  const T b = T(0.999999), c = T(1e-7);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int i = 0; i < PK_CHAINS; ++i) a[i] = fma(a[i], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < PK_CHAINS; ++i) s += a[i];
  if (s == T(-1.25)) out[0] = s;
}

// XU (multi-function unit) ops: sine, cosine and reciprocal square root of
// the PTX approximate forms, on independent chains
__global__ void __launch_bounds__(PK_THREADS) k_peak_xu(int iters, float* out) {
  float a[PK_CHAINS];
#pragma unroll
  for (int i = 0; i < PK_CHAINS; ++i) a[i] = 0.5f + 1e-3f * (float)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < PK_CHAINS; ++i) {
      float v = a[i];
      asm volatile("sin.approx.f32 %0, %0;" : "+f"(v));
      asm volatile("cos.approx.f32 %0, %0;" : "+f"(v));
      asm volatile("rsqrt.approx.f32 %0, %0;" : "+f"(v));
      a[i] = v;
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < PK_CHAINS; ++i) s += a[i];
  if (s == -1.25f) out[0] = s;
}

// shared-memory loads: 16-byte loads from conflict-free addresses (a warp's
// load covers 512 consecutive bytes)
constexpr int PK_SMEM_FLOATS = 4096;  // 16 KB
__global__ void __launch_bounds__(PK_THREADS) k_peak_smem(int iters, float* out) {
  __shared__ __align__(16) float buf[PK_SMEM_FLOATS];
  for (int i = threadIdx.x; i < PK_SMEM_FLOATS; i += PK_THREADS) buf[i] = (float)i * 1e-6f;
  __syncthreads();
  const float4* b4 = reinterpret_cast<const float4*>(buf);
  constexpr int N4 = PK_SMEM_FLOATS / 4;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  int idx = threadIdx.x;
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float4 v = b4[(idx + u * 32) & (N4 - 1)];
      acc.x += v.x;
      acc.y += v.y;
      acc.z += v.z;
      acc.w += v.w;
    }
    idx = (idx + 256) & (N4 - 1);
  }
  if (acc.x + acc.y + acc.z + acc.w == -1.25f) out[0] = acc.x;
}

// tcgen05.mma kind::tf32, M = 128, N = 256, K = 8, one CTA per SM, operands
// resident in shared memory (128-byte swizzled K-major, one 32-float K slice:
// four MMAs per slice), accumulating in TMEM; one thread issues, a commit at
// the end arrives on an mbarrier.  The wait is bounded (about one second):
// on time-out the kernel records it, waits again (bounded) for its own MMAs
// and frees its TMEM.
constexpr int PK_TC_M = 128, PK_TC_N = 256;
constexpr uint32_t PK_TC_ABYTES = PK_TC_M * 128, PK_TC_BBYTES = PK_TC_N * 128;

__device__ int g_peak_error;

__global__ void __launch_bounds__(128, 1) k_peak_tf32(int iters, float* out) {
  extern __shared__ __align__(1024) unsigned char pk_smem[];
  __shared__ __align__(8) uint64_t done;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  // 1024-byte aligned operand tiles
  unsigned char* base = pk_smem + ((1024u - (sa(pk_smem) & 1023u)) & 1023u);
  float* fa = reinterpret_cast<float*>(base);
  for (uint32_t i = tid; i < (PK_TC_ABYTES + PK_TC_BBYTES) / 4; i += 128)
    fa[i] = 0.25f + 1e-4f * (float)(i % 1000);
  if (tid == 0) {
    tc_mbar_init(&done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(&tmem_base)),
                 "r"(PK_TC_N)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  if (tid == 0) {
    const uint32_t a0 = sa(base), b0 = a0 + PK_TC_ABYTES;
    const uint32_t idesc = tc_idesc(PK_TC_M, PK_TC_N);
    for (int it = 0; it < iters; ++it)
#pragma unroll
      for (int ks = 0; ks < 4; ++ks)
        tc_mma(tmem, tc_desc(a0 + 32 * ks), tc_desc(b0 + 32 * ks), idesc, (it | ks) ? 1u : 0u);
    tc_commit(&done);
  }
  bool ok = tc_wait(&done, 0);
  if (!ok) {
    atomicExch(&g_peak_error, 1);
    tc_wait(&done, 0);
  }
  tc_fence_after();
  __syncthreads();
  if (ok && warp == 0) {
    float v[16];
    tc_ld16(tmem, v);
    if (v[0] == -1.25f) out[0] = v[0];
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(PK_TC_N) : "memory");
}

int sm_count_here(int* n) {
  int dev = 0;
  HFMM_CUDA_TRY(cudaGetDevice(&dev));
  HFMM_CUDA_TRY(cudaDeviceGetAttribute(n, cudaDevAttrMultiProcessorCount, dev));
  return HFMM_OK;
}

// best time (ms) of `reps` launches after one warm-up
template <typename F>
int best_ms(F launch, cudaStream_t s, int reps, double* ms) {
  cudaEvent_t e0, e1;
  HFMM_CUDA_TRY(cudaEventCreate(&e0));
  HFMM_CUDA_TRY(cudaEventCreate(&e1));
  launch();
  double best = 1e30;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0, s);
    launch();
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return HFMM_ERR_CUDA;
    }
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    best = std::min(best, (double)t);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = best;
  return hfmm_last_launch();
}

}  // namespace

extern "C" int hfmm_pipe_peaks(double* out, void* stream) {
  if (!out) return HFMM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int nsm = 0;
  HFMM_TRY(sm_count_here(&nsm));
  float* sink = nullptr;
  HFMM_CUDA_TRY(cudaMalloc(&sink, 64));
  int st = HFMM_OK;
  const int blocks = nsm * 8;  // 2048 threads per SM resident
  const double threads = (double)blocks * PK_THREADS;
  double ms = 0.0;
  do {
    // FP32 FMA: 2 flop per FMA
    const int it32 = 4096;
    st = best_ms([&] { k_peak_fma<float><<<blocks, PK_THREADS, 0, s>>>(it32, sink); }, s, 3, &ms);
    if (st != HFMM_OK) break;
    out[HFMM_PEAK_FP32_TFLOPS] = 2.0 * 4 * PK_CHAINS * (double)it32 * threads / (ms * 1e-3) / 1e12;
    // FP64 FMA
    const int it64 = 128;
    st = best_ms([&] { k_peak_fma<double><<<blocks, PK_THREADS, 0, s>>>(it64, (double*)sink); }, s, 3, &ms);
    if (st != HFMM_OK) break;
    out[HFMM_PEAK_FP64_TFLOPS] = 2.0 * 4 * PK_CHAINS * (double)it64 * threads / (ms * 1e-3) / 1e12;
    // XU: three ops per chain step
    const int itxu = 512;
    st = best_ms([&] { k_peak_xu<<<blocks, PK_THREADS, 0, s>>>(itxu, sink); }, s, 3, &ms);
    if (st != HFMM_OK) break;
    out[HFMM_PEAK_XU_GOPS] = 3.0 * PK_CHAINS * (double)itxu * threads / (ms * 1e-3) / 1e9;
    // shared-memory loads: 8 x 16 bytes per thread and iteration
    const int itsm = 2048;
    st = best_ms([&] { k_peak_smem<<<blocks, PK_THREADS, 0, s>>>(itsm, sink); }, s, 3, &ms);
    if (st != HFMM_OK) break;
    out[HFMM_PEAK_SMEM_GBS] = 8.0 * 16.0 * (double)itsm * threads / (ms * 1e-3) / 1e9;
    // TF32 tensor cores: 2 M N K flop per MMA, four MMAs per iteration
    const int ittc = 4096;
    // 120 KB of shared memory keeps one CTA per SM (the operands take 49 KB)
    const size_t smem = 120 * 1024;
    if (cudaFuncSetAttribute(k_peak_tf32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      st = HFMM_ERR_CUDA;
      break;
    }
    int zero = 0;
    if (cudaMemcpyToSymbolAsync(g_peak_error, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      st = HFMM_ERR_CUDA;
      break;
    }
    st = best_ms([&] { k_peak_tf32<<<nsm, 128, smem, s>>>(ittc, sink); }, s, 3, &ms);
    if (st != HFMM_OK) break;
    int err = 0;
    if (cudaMemcpyFromSymbol(&err, g_peak_error, sizeof(int)) != cudaSuccess) {
      st = HFMM_ERR_CUDA;
      break;
    }
    if (err) {
      st = HFMM_ERR_TIMEOUT;
      break;
    }
    out[HFMM_PEAK_TF32_TFLOPS] =
        2.0 * PK_TC_M * PK_TC_N * 8 * 4 * (double)ittc * nsm / (ms * 1e-3) / 1e12;
  } while (false);
  if (st != HFMM_OK) cudaGetLastError();
  cudaFree(sink);
  return st;
}
