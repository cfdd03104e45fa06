// Restarted GMRES on device vectors (Sec. 3: GMRES(m); Sec. 4: right
// preconditioning, so the minimised residual is the true one).  FP64
// complex arithmetic throughout; classical Gram-Schmidt applied twice; the
// Hessenberg least-squares problem is updated with complex Givens rotations
// c = |a|/nu, s = (a/|a|) conj(b)/nu on the device.  With a preconditioner
// the flexible variant stores Z = [M^-1 v_1 ...] and updates x with Z y.
#pragma once

#include <functional>

#include "common.cuh"

// operator on complex vectors of real type R (complex128 for double)
template <typename R>
using DevOpT = std::function<int(const C<R>* in, C<R>* out)>;
using DevOp = DevOpT<double>;

template <typename R>
struct GmresWorkT {
  int64_t N = 0;
  int m = 0;
  bool flexible = false;
  C<R>* V = nullptr;         // (m+1) x N
  C<R>* Z = nullptr;         // m x N (flexible)
  C<R>* w = nullptr;         // N
  C<R>* r = nullptr;         // N
  double* partial = nullptr; // reduction partials (per block, FP64)
  unsigned* counter = nullptr; // blocks finished in the current reduction launch (reset by the last)
  double2* dots = nullptr;   // 2 (m+1): CGS2 coefficients
  double2* H = nullptr;      // (m+1) x m, column-major
  double* cs = nullptr;      // m
  double2* sn = nullptr;     // m
  double2* g = nullptr;      // m+1
  double2* y = nullptr;      // m
  double* scal = nullptr;    // device scalars
  double* host = nullptr;    // pinned host mirror of scal
  void* base = nullptr;      // single allocation
  size_t bytes = 0;
  const int* skip = nullptr; // device flag: reductions return at once when set (graph form)
};
using GmresWork = GmresWorkT<double>;

template <typename R>
int gmres_work_reserve(GmresWorkT<R>& W, int64_t N, int m, bool flexible);
template <typename R>
void gmres_work_free(GmresWorkT<R>& W);

struct GmresResult {
  int iters = 0, restarts = 0, converged = 0;
  double relres_est = 0, relres_true = 0;
};

// Solves A x = b (x holds x0 on entry).  M may be null (no preconditioner).
// history (host, optional) receives relres_est per iteration.
// x0_zero: x holds zeros on entry (skips one operator application);
// true_residual: recompute ||b - A x|| at exit (one more application).
template <typename R>
int gmres_run(GmresWorkT<R>& W, const DevOpT<R>& A, const DevOpT<R>* M, const C<R>* b, C<R>* x, int m,
              double rtol, int maxit, bool x0_zero, bool true_residual, GmresResult* res,
              double* history, int history_len, cudaStream_t s);

template <typename R>
int dev_norm(GmresWorkT<R>& W, const C<R>* x, int64_t N, double* out_dev, cudaStream_t s);

// *out = scale Re sum_i conj(a_i) b_i over N complex128 entries (device
// pointers), deterministic; part: RE_DOT_PARTS doubles of scratch
constexpr int RE_DOT_PARTS = 608;
int re_dot_dev(const double2* a, const double2* b, int64_t N, double scale, double* part, double* out,
               cudaStream_t s);

// One GMRES cycle of m steps from x0 = 0 for capture in a CUDA graph: no
// host reads; once the device flag *d_done is set (converged or breakdown)
// the kernels of the remaining steps return at once (the operator's kernels
// must honour the same flag).  x = V y with y from the first *d_jdone steps;
// *d_total += *d_jdone.
template <typename R>
int gmres_cycle_device(GmresWorkT<R>& W, const DevOpT<R>& A, const C<R>* b, C<R>* x, int m, double rtol,
                       int* d_done, int* d_jdone, int* d_total, cudaStream_t s);

// Right-preconditioned BiCGSTAB (van der Vorst), FP64 complex vectors: the
// paper's Sec. 3 short-recurrence alternative to GMRES.  Two operator and two
// preconditioner applications per iteration (one of each when it stops at
// the half step); scalars on the host.
struct BicgWork {
  int64_t N = 0;
  double2 *r = nullptr, *rhat = nullptr, *p = nullptr, *v = nullptr, *s = nullptr, *t = nullptr;
  double2 *phat = nullptr, *shat = nullptr;
  double2* partial = nullptr;  // reduction partials
  unsigned* counter = nullptr; // blocks finished in the current reduction launch
  double2* dots = nullptr;     // [0] inner product, [1].x norm
  double* host = nullptr;      // pinned mirror of dots
  void* base = nullptr;
};

struct BicgResult {
  int iters = 0, converged = 0, breakdown = 0, precond_applies = 0;
  double relres_est = 0, relres_true = 0;
};

int bicg_work_reserve(BicgWork& W, int64_t N);
void bicg_work_free(BicgWork& W);
int bicgstab_run(BicgWork& W, const DevOp& A, const DevOp* M, const double2* b, double2* x, double rtol, int maxit,
                 bool x0_zero, BicgResult* res, double* history, int history_len, cudaStream_t s);
