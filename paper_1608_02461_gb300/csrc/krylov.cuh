// Restarted GMRES on device vectors (Sec. 3: GMRES(m); Sec. 4: right
// preconditioning, so the minimised residual is the true one).  FP64
// complex arithmetic throughout; classical Gram-Schmidt applied twice; the
// Hessenberg least-squares problem is updated with complex Givens rotations
// c = |a|/nu, s = (a/|a|) conj(b)/nu on the device.  With a preconditioner
// the flexible variant stores Z = [M^-1 v_1 ...] and updates x with Z y.
#pragma once

#include <functional>

#include "common.cuh"

using DevOp = std::function<int(const double2* in, double2* out)>;

struct GmresWork {
  int64_t N = 0;
  int m = 0;
  bool flexible = false;
  double2* V = nullptr;      // (m+1) x N
  double2* Z = nullptr;      // m x N (flexible)
  double2* w = nullptr;      // N
  double2* r = nullptr;      // N
  double* partial = nullptr; // reduction partials
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

int gmres_work_reserve(GmresWork& W, int64_t N, int m, bool flexible);
void gmres_work_free(GmresWork& W);

struct GmresResult {
  int iters = 0, restarts = 0, converged = 0;
  double relres_est = 0, relres_true = 0;
};

// Solves A x = b (x holds x0 on entry).  M may be null (no preconditioner).
// history (host, optional) receives relres_est per iteration.
// x0_zero: x holds zeros on entry (skips one operator application);
// true_residual: recompute ||b - A x|| at exit (one more application).
int gmres_run(GmresWork& W, const DevOp& A, const DevOp* M, const double2* b, double2* x, int m,
              double rtol, int maxit, bool x0_zero, bool true_residual, GmresResult* res,
              double* history, int history_len, cudaStream_t s);

int dev_norm(GmresWork& W, const double2* x, int64_t N, double* out_dev, cudaStream_t s);

// One GMRES cycle of m steps from x0 = 0 for capture in a CUDA graph: no
// host reads; once the device flag *d_done is set (converged or breakdown)
// the kernels of the remaining steps return at once (the operator's kernels
// must honour the same flag).  x = V y with y from the first *d_jdone steps;
// *d_total += *d_jdone.
int gmres_cycle_device(GmresWork& W, const DevOp& A, const double2* b, double2* x, int m, double rtol, int* d_done,
                       int* d_jdone, int* d_total, cudaStream_t s);
