/*
 * hfmm.h -- C ABI of the GB300 (sm_103a) FMM-preconditioned Helmholtz solver.
 *
 * Method: Ibeid, Yokota, Keyes, "A Matrix-free Preconditioner for the
 * Helmholtz Equation based on the Fast Multipole Method".  The library solves
 * the 7-point finite-difference discretisation of -Lap u - k^2 u = f on the
 * unit cube with u = 0 on the boundary (Sec. 2, Eq. (helm), Dirichlet case of
 * Sec. 6/7) by right-preconditioned GMRES (Sec. 3-4); the preconditioner is
 * the BEM-coupled FMM of Sec. 5 (FMM flow of Sec. 5.1.2, boundary equation
 * Eq. (ubound), interior representation Eq. (uinter)).
 *
 * Conventions for every entry point
 *  - Pointers named d_* are DEVICE memory owned by the caller; the library
 *    never frees them and keeps no reference after the call returns.
 *  - Complex vectors are interleaved (re, im) float64 pairs (the layout of
 *    complex128 / cuDoubleComplex), whatever the internal precision.
 *  - Interior-node vectors have n^3 entries, node (i, j, l) h with h = 1/(n+1)
 *    at index (i-1) + n (j-1) + n^2 (l-1) (x fastest).
 *  - Boundary vectors have 6 n^2 entries, one constant element (panel) per
 *    boundary grid node off the cube's edges, faces in the order x=0, x=1,
 *    y=0, y=1, z=0, z=1, first free coordinate fastest within a face.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    stream-ordered; entry points that must read a scalar back (GMRES) block
 *    the host on that stream.
 *  - Every call returns an int status (HFMM_OK = 0, negative on error) and
 *    throws nothing.  On an argument error nothing is written.
 *  - The fmm_tree handle owns all its device workspace; it is not thread
 *    safe: calls on one handle must be serialised by the caller.
 */
#ifndef HFMM_H
#define HFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define HFMM_OK                 0
#define HFMM_ERR_INVALID_ARG   -1
#define HFMM_ERR_CUDA          -2
#define HFMM_ERR_NOMEM         -3
#define HFMM_ERR_NONFINITE     -4
#define HFMM_ERR_NOT_CONVERGED -5
#define HFMM_ERR_TIMEOUT       -6
#define HFMM_ERR_UNSUPPORTED   -7

/* internal arithmetic of the FMM stages (Krylov arithmetic is always FP64) */
#define HFMM_FP64 0
#define HFMM_FP32 1

/* point sets */
#define HFMM_SET_VOL 1   /* interior nodes (volume term of Eq. (uinter)) */
#define HFMM_SET_BND 2   /* boundary elements (boundary terms)           */

/* fmm_apply modes */
#define HFMM_FWD 0       /* phi = G~ q                                   */
#define HFMM_ADJ 1       /* phi = G~^H q  (conjugate transpose)          */
#define HFMM_DK  2       /* phi = d(G~ q)/dk                             */
#define HFMM_DLP 3       /* phi = D~ q  (double layer, boundary sources)  */

typedef struct hfmm_params {
    int p;            /* expansion order: degrees 0..p-1 (1 <= p <= 16)  */
    double theta;     /* multipole acceptance parameter, 0 < theta <= 0.55:
                         same-level cells at centre distance d are far iff
                         theta * d > cell width                          */
    int leaf_size;    /* target interior nodes per leaf; the tree is uniform
                         of depth L = max(2, ceil(log8(n_vol / leaf_size)))  */
    double k;         /* wavenumber, k >= 0                              */
    int precision;    /* HFMM_FP64 or HFMM_FP32                          */
} hfmm_params;

typedef struct hfmm_gmres_params {
    int restart_m;     /* outer GMRES restart length m (1..200)            */
    double rtol;       /* stop when |g_{j+1}| < rtol ||b|| (Sec. 6: 1e-6)  */
    int maxit;         /* cap on preconditioner applications (0: 20 m)     */
    double inner_rtol; /* tolerance of the inner boundary solve V q = -g   */
    int inner_maxit;   /* cap on inner iterations per preconditioner apply */
    int inner_m;       /* restart length of the inner GMRES                */
} hfmm_gmres_params;

typedef struct hfmm_gmres_info {
    int iters;             /* preconditioner applications (all restarts)  */
    int restarts;
    int inner_iters_total; /* inner GMRES iterations over all applies     */
    int status;            /* HFMM_OK or HFMM_ERR_NOT_CONVERGED           */
    double relres_est;     /* |g_{j+1}| / ||b|| at exit                   */
    double relres_true;    /* ||b - A x|| / ||b|| at exit                 */
    double* history;       /* optional host array (caller-owned) of length
                              history_len: relres_est per iteration       */
    int history_len;
} hfmm_gmres_info;

/* stages timed by fmm_set_timing (index into hfmm_stats.stage_ms) */
#define HFMM_STAGE_GATHER  0  /* input permutation into leaf order, output scatter */
#define HFMM_STAGE_P2M     1
#define HFMM_STAGE_M2M     2
#define HFMM_STAGE_M2L     3
#define HFMM_STAGE_L2L     4
#define HFMM_STAGE_L2P     5
#define HFMM_STAGE_P2P     6  /* near field and self term                    */
#define HFMM_STAGE_FDM     7  /* 7-point operator inside gmres_solve         */
#define HFMM_STAGE_BND     8  /* boundary -> boundary apply of the inner solve
                                 as one kernel (all its stages together)    */
#define HFMM_NSTAGES       9

typedef struct hfmm_stats {
    int L;                 /* tree depth                                   */
    int p;
    int64_t n_vol, n_bnd;
    int64_t leaves;
    int64_t m2l_pairs;     /* far-field cell pairs over all levels (volume+boundary sets) */
    int64_t p2p_pairs;     /* near-field point pairs, all points as sources and targets */
    int64_t device_bytes;  /* device memory held by the handle              */
    double ms_last_apply;  /* CUDA-event time of the last fmm_apply/precond */
    int64_t launches;      /* kernels this library has launched in this process */
    double stage_ms[HFMM_NSTAGES];     /* CUDA-event time per stage since timing
                                          was switched on (fmm_set_timing)      */
    int64_t stage_launches[HFMM_NSTAGES]; /* kernel launches per stage, same span */
    double stage_work[HFMM_NSTAGES];   /* algorithmic work per stage, same span:
                                          P2P point pairs (j != i), M2L flops
                                          (8 p^4 per cell pair), 0 elsewhere   */
} hfmm_stats;

typedef struct fmm_tree fmm_tree;

/* Text for a status code (static storage). */
const char* hfmm_error_string(int status);

/*
 * fmm_build_tree -- Sec. 5.1.1 (octree decomposition), Sec. 5.3 (constant
 * boundary elements), Sec. 7 (p, theta).
 *
 * Builds the uniform Morton-ordered octree over the interior nodes and the
 * boundary panels of the n^3 grid, the near (P2P) and far (M2L) interaction
 * lists, every translation operator for wavenumber k, and the singular self
 * terms of cells and panels.  All of it runs in device kernels on `stream`.
 *
 *   n          interior nodes per axis (n >= 2); h = 1/(n+1)
 *   d_vol_xyz  NULL: the n^3 lattice nodes.  Otherwise n_vol points (AoS
 *              x,y,z float64, device) in [0,1]^3 that replace them; the
 *              self terms are then zero (no cell volume is implied).
 *   n_vol      number of interior points (n^3 when d_vol_xyz is NULL)
 *   d_bnd_xyz  NULL: the 6 n^2 lattice panels.  Otherwise n_bnd points.
 *   n_bnd      number of boundary points (6 n^2 when d_bnd_xyz is NULL;
 *              0 allowed with explicit points)
 *   params     see hfmm_params
 *   out        receives the handle (NULL on error)
 * Errors: INVALID_ARG (sizes, p, theta, k, precision), NOMEM, CUDA.
 */
int fmm_build_tree(int n, const double* d_vol_xyz, int64_t n_vol,
                   const double* d_bnd_xyz, int64_t n_bnd,
                   const hfmm_params* params, void* stream, fmm_tree** out);

/* Releases the handle and all its device memory (NULL is a no-op). */
void fmm_destroy_tree(fmm_tree* tree);

/*
 * fmm_apply -- Sec. 5.1 N-body sum with the 3D Helmholtz kernel of Sec. 5.2,
 * G(x, y) = exp(i k |x-y|) / (4 pi |x-y|), by the FMM of Sec. 5.1.2.
 *
 *   phi_i = sum_{j in src_set, j != i} q_j G(x_i, x_j) + [i in src_set] s_i q_i
 *
 * for every target i in tgt_set, where s_i is the self coefficient: the
 * integral of G over the point's own cell divided by h^3 (interior node) or
 * over its own panel divided by h^2 (boundary element); zero for explicit
 * points.  Weights are used as given (no quadrature weight is applied).
 * Call this linear map G~ (the truncated FMM operator from src_set to
 * tgt_set).  `mode` selects:
 *   HFMM_FWD  phi = G~ q:        q on src_set, phi on tgt_set
 *   HFMM_ADJ  phi = G~^H q:      q on tgt_set, phi on src_set.  Every FMM
 *             stage is conjugate-transposed and applied in reverse order
 *             (L2P^H, L2L^H, M2L^H, M2M^H, P2M^H, conj(P2P), conj(self)),
 *             so <G~ x, y> = <x, G~^H y> holds to rounding.
 *   HFMM_DK   phi = dG~/dk q:    q on src_set, phi on tgt_set; the exact
 *             k-derivative of the truncated FMM (tangent of every stage:
 *             Bessel functions in P2M/L2P, translation operators, near-field
 *             kernel, self terms).
 *   HFMM_DLP  phi = D~ q:        the double layer of Eq. (bem) (Sec. 5.2):
 *             phi_i = sum_{j != i} q_j dG/dn_y(x_i, y_j),
 *             dG/dn_y = (i k r - 1) e^{ikr} / (4 pi r^2) (y - x).n_y / r,
 *             for boundary sources y_j (src_set must be HFMM_SET_BND) with
 *             the outward normals of their faces; lattice trees only
 *             (UNSUPPORTED otherwise).  The own panel contributes nothing
 *             (it is flat: (y - x).n_y = 0); no jump term is added.  The
 *             FMM is the same but for P2M (normal derivative of the regular
 *             basis: dipole multipoles) and P2P (the kernel above).
 *
 *   src_set, tgt_set  non-zero OR of HFMM_SET_VOL / HFMM_SET_BND
 *   d_q_vol, d_q_bnd  input weights (complex128) per set of the input side;
 *                     a set not on that side may be NULL
 *   d_phi_vol, d_phi_bnd  outputs (complex128) per set of the output side
 *                     (overwritten); a set not on that side may be NULL
 * The adjoint and derivative operators are built on the first call in those
 * modes (device memory held by the handle).
 * FP32 form: the M2L of levels >= 4 with volume targets runs on the tensor
 * cores (three TF32 products per product, FP32 accumulation), and on a
 * regular lattice tree (n divisible by 2^L, every leaf the same block of
 * nodes) so does the volume sources' near field of an HFMM_FWD apply with
 * tgt_set = HFMM_SET_VOL (the block between two leaves depends only on their
 * offset); environment HFMM_M2L_TC=0 / HFMM_NEAR_TC=0 at tree build keeps
 * the CUDA-core kernels.
 * Errors: INVALID_ARG, NOMEM, CUDA.
 */
int fmm_apply(fmm_tree* tree, int src_set, int tgt_set,
              const void* d_q_vol, const void* d_q_bnd,
              void* d_phi_vol, void* d_phi_bnd, int mode, void* stream);

/*
 * fmm_precond_apply -- z = M^-1 r, the BEM-coupled FMM preconditioner of
 * Sec. 5.2-5.3 with homogeneous Dirichlet data:
 *   w = h^3 r;  g = G_{Gamma,Omega} w                         (Pass A)
 *   solve V q = -g, V = h^2 G_{Gamma,Gamma} + self terms      (inner GMRES,
 *                                                              Pass B per step)
 *   z = G_{Omega,Omega} w + G_{Omega,Gamma} (h^2 q) + s_Omega r (Pass C)
 * Requires a lattice tree (d_vol_xyz == NULL at build).
 *   d_r, d_z       n^3 complex128 (device); d_z is overwritten
 *   inner_rtol     relative tolerance of the inner solve (> 0)
 *   inner_maxit    inner iteration cap (>= 1); inner_m its restart length
 *   inner_iters    optional host int receiving the inner iteration count
 * The inner solve stopping at inner_maxit is not an error.
 * Errors: INVALID_ARG, UNSUPPORTED (explicit points), CUDA.
 */
int fmm_precond_apply(fmm_tree* tree, const void* d_r, void* d_z,
                      double inner_rtol, int inner_maxit, int inner_m,
                      int* inner_iters, void* stream);

/*
 * fmm_set_inner_order -- expansion order of the boundary -> boundary FMM
 * applies inside the preconditioner's inner solve (Pass B of
 * fmm_precond_apply, gmres_solve, bicgstab_solve, bem_solve_dirichlet).  The
 * inner solve runs to a loose tolerance (1e-2 in the benchmark), so a lower
 * order than the tree's p can serve it; Passes A and C keep p.  p_inner = 0
 * (or the tree's p) uses the tree itself.  Otherwise an auxiliary tree over
 * the same points with order p_inner is built on `stream` (device memory
 * held by the handle; its stage times are added to fmm_get_stats).  Drops a
 * captured preconditioner graph.  Lattice trees only.
 * Errors: INVALID_ARG (p_inner outside 0..16), UNSUPPORTED, NOMEM, CUDA.
 */
int fmm_set_inner_order(fmm_tree* tree, int p_inner, void* stream);

/*
 * bem_solve_dirichlet -- the BEM solution of -Lap u - k^2 u = f in the cube
 * with Dirichlet data u = u_Gamma on the boundary (Sec. 5.2-5.3: Eq. (ubound)
 * for q = du/dn, then Eq. (uinter) at the interior nodes), every sum by the
 * FMM:
 *   g = G_{Gamma,Omega} (h^3 f) - u_Gamma / 2 - D_{Gamma,Gamma} (h^2 u_Gamma)
 *   solve (-V) q = g                           (inner GMRES, as in
 *                                               fmm_precond_apply)
 *   u = G_{Omega,Omega} (h^3 f) + G_{Omega,Gamma} (h^2 q) + s_Omega f
 *       - D_{Omega,Gamma} (h^2 u_Gamma)
 * with D the double layer of fmm_apply's HFMM_DLP mode.  With u_Gamma = 0 it
 * is fmm_precond_apply (r = f).  A starting iterate for gmres_solve on the
 * system of hfmm_dirichlet_rhs.  Lattice trees only.
 *   d_f        n^3 complex128 volume data (device)
 *   d_u_bnd    6 n^2 complex128 Dirichlet values at the panel centres (device)
 *   d_u        n^3 complex128 result (device, overwritten)
 *   inner_rtol, inner_maxit, inner_m, inner_iters  as in fmm_precond_apply
 * Errors: INVALID_ARG, UNSUPPORTED (explicit points), NOMEM, CUDA, TIMEOUT.
 */
int bem_solve_dirichlet(fmm_tree* tree, const void* d_f, const void* d_u_bnd, void* d_u,
                        double inner_rtol, int inner_maxit, int inner_m,
                        int* inner_iters, void* stream);

/*
 * hfmm_dirichlet_rhs -- right-hand side of the 7-point system (Sec. 2) with
 * Dirichlet data: the stencil's neighbours outside the interior are the
 * boundary grid nodes off the edges, i.e. the panel centres, so with
 * u = u_Gamma there
 *   b_i = f_i + (1/h^2) sum of u_Gamma over the boundary neighbours of node i
 * and hfmm_fdm_apply(u) = b for the interior values u.  Lattice trees only.
 *   d_f      n^3 complex128 (device)
 *   d_u_bnd  6 n^2 complex128 (device), panel order as everywhere
 *   d_b      n^3 complex128 result (device; may be d_f)
 * Errors: INVALID_ARG, UNSUPPORTED, CUDA.
 */
int hfmm_dirichlet_rhs(fmm_tree* tree, const void* d_f, const void* d_u_bnd, void* d_b, void* stream);

/*
 * hfmm_fdm_apply -- the 7-point operator of Sec. 2 (reading: -Lap - k^2):
 *   (A u)_i = (6 u_i - sum of the six neighbours) / h^2 - k^2 u_i,
 * neighbours outside the grid being zero.  d_u, d_out: n^3 complex128.
 */
int hfmm_fdm_apply(fmm_tree* tree, const void* d_u, void* d_out, void* stream);

/*
 * hfmm_order_for_k -- the expansion order to build a lattice tree with for
 * wavenumber k when at least p_min is asked for (host function, no device
 * work).  A multipole or local expansion of order p (degrees below p) of a
 * cell of half-diagonal rho resolves e^{ikr}/r only for p above about
 * k rho (the spherical Bessel functions j_n(k rho) become small for
 * n > k rho; Sec. 5.1.2 expansions).  The coarsest level with M2L
 * interactions is level 2 of the unit cube, rho_2 = sqrt(3)/8, so the
 * order is the smallest even p >= max(p_min, ceil(k rho_2) + 1).  With a
 * fixed order the preconditioner degrades as k grows (GMRES iterations rise
 * and at p = 4, k > 21 the solve stalls); with this order the iteration
 * count stays near that of moderate k.
 * Returns the order (>= 1), or INVALID_ARG (k < 0 or not finite, p_min
 * outside 1..16) or UNSUPPORTED (the rule asks for more than order 16).
 */
int hfmm_order_for_k(double k, int p_min);

/*
 * fmm_grad_k -- the wavenumber gradient of a real loss of phi = G~ q on the
 * volume points (fmm_apply VOL -> VOL, HFMM_FWD):
 *   *d_out = Re sum_i conj(g_i) (dG~/dk q)_i,   g = dL/dphi
 * (PyTorch's convention for complex tensors).  The tangent apply (HFMM_DK)
 * writes into device memory held by the handle (n_vol complex128, allocated
 * on the first call, so the first call must not be inside a stream capture);
 * the sum runs on the device in FP64 in a fixed order (bit-identical on
 * repeated calls).
 *   d_q_vol, d_g_vol  n_vol complex128 (device), read only
 *   d_out             one double (device), overwritten
 * Errors: INVALID_ARG (null pointer, no volume points), NOMEM, CUDA.
 */
int fmm_grad_k(fmm_tree* tree, const void* d_q_vol, const void* d_g_vol, double* d_out, void* stream);

/*
 * hfmm_solve_grad_k -- the wavenumber gradient of a real loss of the solution
 * x = A(k)^-1 b of the 7-point system (Sec. 2).  For real k, A is real and
 * symmetric with dA/dk = -2k I, so with lam the solution of A lam = dL/dx:
 *   *d_out = -Re <lam, (dA/dk) x> = 2k Re sum_i conj(lam_i) x_i
 * summed on the device in FP64 in a fixed order (scratch held by the handle,
 * allocated on the first call of either gradient entry point).
 *   d_lam, d_x  n^3 complex128 (device), read only
 *   d_out       one double (device), overwritten
 * Lattice trees only (UNSUPPORTED otherwise).  Errors: INVALID_ARG, NOMEM, CUDA.
 */
int hfmm_solve_grad_k(fmm_tree* tree, const void* d_lam, const void* d_x, double* d_out, void* stream);

/*
 * gmres_solve -- Sec. 3-4, Sec. 6: flexible right-preconditioned restarted
 * GMRES(m) for A x = b with A the 7-point operator of the tree's (n, k) and
 * M^-1 = fmm_precond_apply.  Classical Gram-Schmidt with reorthogonalisation,
 * complex Givens rotations, FP64 Krylov arithmetic (the preconditioner's
 * inner boundary solve runs in the precision of the tree's FMM form).
 *   d_b     n^3 complex128 right-hand side
 *   d_x     in: initial guess x0; out: solution (written also when the
 *           status is NOT_CONVERGED)
 *   info    host struct, filled on return (history optional)
 * Returns HFMM_OK when converged, HFMM_ERR_NOT_CONVERGED after maxit
 * applications, or another error.
 */
int gmres_solve(fmm_tree* tree, const void* d_b, void* d_x,
                const hfmm_gmres_params* gp, hfmm_gmres_info* info, void* stream);

/*
 * bicgstab_solve -- Sec. 3 (and its GMRES/BiCGSTAB comparison figure):
 * right-preconditioned BiCGSTAB (van der Vorst) for the same system and
 * preconditioner as gmres_solve, FP64 complex vectors.  One iteration
 * applies A and M^-1 twice (once each when it stops at the half step);
 * stops when ||b - A x|| < rtol ||b|| by the recurrence residual, or on a
 * breakdown (rho = 0 or omega = 0).
 *   d_b, d_x  as in gmres_solve (d_x holds x0 on entry)
 *   gp        rtol, maxit (iterations; 0: 500) and the preconditioner's
 *             inner_rtol, inner_maxit, inner_m; restart_m is not used
 *   info      iters = BiCGSTAB iterations, restarts = preconditioner
 *             applications, history[i] = relative residual after iteration i,
 *             relres_true = ||b - A x|| / ||b|| recomputed at exit
 * Returns HFMM_OK when converged, HFMM_ERR_NOT_CONVERGED otherwise (x and
 * info written), or another error.
 */
int bicgstab_solve(fmm_tree* tree, const void* d_b, void* d_x,
                   const hfmm_gmres_params* gp, hfmm_gmres_info* info, void* stream);

/*
 * gmres_solve_batched -- many independent solves of gmres_solve (Sec. 3-4,
 * Sec. 6), e.g. right-hand sides and wavenumbers of uneven grid sizes, one
 * handle per solve.  The solves run concurrently: worker threads drive them
 * on their own streams so that their kernels overlap on the GPU.  Work on
 * `stream` before the call is ordered before the batch, and work queued on
 * `stream` after it waits for the whole batch.
 *   trees[count], d_b[count], d_x[count]   as in gmres_solve; the handles
 *                                          must be distinct
 *   infos                                  optional host array [count]
 * Returns the first hard error, else HFMM_ERR_NOT_CONVERGED if any solve did
 * not converge or stopped on a non-finite value (infos[i].status is then
 * HFMM_ERR_NOT_CONVERGED or HFMM_ERR_NONFINITE for that solve alone), else
 * HFMM_OK.  Blocks the calling thread until done.
 */
int gmres_solve_batched(fmm_tree** trees, const void** d_b, void** d_x, int count,
                        const hfmm_gmres_params* gp, hfmm_gmres_info* infos, void* stream);

/*
 * fmm_autotune -- times the M2L kernel variants (two-stage block pipeline,
 * warp-specialised three-stage pipeline, pair lists) and the split of the
 * per-tile offset lists (grid filled to 1, 2, 4, 8 or 16 x 152 blocks, at
 * most 32 parts per tile, 16 on trees whose 32 partial-sum slots would take
 * more than 256 MB) on the FMM passes of the preconditioner and on the full
 * apply, then, with the
 * chosen M2L, the tile shapes of the lattice near field (tiled 4 x 4
 * target-source groups or not in the FP32 form; at most 8, 16 or 32 threads
 * per group of targets; one block per SM or as many as fit) and whether the
 * near field runs on a side stream concurrently with the far field, and keeps
 * the fastest per pass in the handle.  The choice changes only the order in
 * which contributions are summed (rounding-level differences); a handle's
 * results stay deterministic.  Also tunes the handle's inner-order tree
 * (fmm_set_inner_order) when it has one.
 */
int fmm_autotune(fmm_tree* tree, void* stream);

/*
 * fmm_use_graphs -- enable (1, default) or disable (0) the CUDA-graph form of
 * the preconditioner inside gmres_solve: Pass A, one inner GMRES cycle of
 * inner_maxit steps driven on the device (steps after convergence return at
 * once through a device flag) and Pass C are captured once per (inner_rtol,
 * inner_maxit) and replayed with one launch per application, with no host
 * synchronisation inside.  Used when inner_m >= inner_maxit; results are
 * identical to the host-driven form.
 */
int fmm_use_graphs(fmm_tree* tree, int enable);

/* Sizes and counters of a built tree.  Waits for the handle's pending
 * timing events (host blocks until they complete). */
int fmm_get_stats(const fmm_tree* tree, hfmm_stats* stats);

/*
 * fmm_set_timing -- per-stage CUDA-event timing.  `stage_mask` has bit i set
 * for every stage HFMM_STAGE_i to time (0 switches timing off; (1 << 8) - 1
 * times all stages); the stage accumulators are reset.  While on, each timed
 * stage's launches are bracketed by events on the launching stream;
 * fmm_get_stats resolves them.  Costs two event records per timed stage and
 * no synchronisation.
 */
int fmm_set_timing(fmm_tree* tree, int stage_mask);

/*
 * hfmm_pipe_peaks -- measured throughput of the arithmetic pipes that bound
 * the solver's kernels (the roofline denominators; no counterpart in the
 * paper).  Runs one short kernel per pipe on the current device, on every SM,
 * and reports the best of three launches timed with CUDA events; the clocks
 * are whatever the GPU runs at.  Takes about 50 ms.
 *   out[HFMM_PEAK_FP32_TFLOPS]  FP32 FMA, 2 flop per FMA
 *   out[HFMM_PEAK_FP64_TFLOPS]  FP64 FMA, 2 flop per FMA
 *   out[HFMM_PEAK_XU_GOPS]      multi-function unit ops (sin, cos, rsqrt) per second, 1e9
 *   out[HFMM_PEAK_SMEM_GBS]     shared-memory 16-byte loads, GB/s
 *   out[HFMM_PEAK_TF32_TFLOPS]  tcgen05.mma kind::tf32 (M 128, N 256), dense, 2 flop per MAC
 * out is a host array of HFMM_NPEAKS doubles.  Allocates 64 bytes of device
 * memory for the duration of the call.  Returns HFMM_ERR_TIMEOUT if the
 * tensor-core probe's bounded wait gave up.
 */
#define HFMM_PEAK_FP32_TFLOPS 0
#define HFMM_PEAK_FP64_TFLOPS 1
#define HFMM_PEAK_XU_GOPS     2
#define HFMM_PEAK_SMEM_GBS    3
#define HFMM_PEAK_TF32_TFLOPS 4
#define HFMM_NPEAKS           5
int hfmm_pipe_peaks(double* out, void* stream);

/*
 * Partition of one FMM apply across ranks (host only: these two calls make
 * no CUDA call and run without a GPU).
 *
 * The octree of Sec. 5.1.1 is cut along the Morton curve of its leaf level
 * into one contiguous range of leaves per rank, the domain decomposition of
 * the paper's distributed runs (Sec. 7).  Leaves are addressed by Morton code
 * m in [0, 8^L): bit 3i of m is bit i of the leaf's x index, bit 3i+1 of y,
 * bit 3i+2 of z; the leaf of a point x is floor(x 2^L) per axis, clamped to
 * 2^L - 1; L is the tree depth of fmm_build_tree (the smallest L >= 2 with
 * leaf_size 8^L >= n_vol).  A cell of level l holds the leaves m with
 * m >> 3(L - l) equal to its own Morton code.
 *
 * hfmm_partition_ranges -- contiguous Morton ranges balanced by cost.
 *   L            leaf level, 2 <= L <= 8
 *   leaf_cost    8^L non-negative finite costs in Morton order (host), or
 *                NULL for equal costs (all-zero costs count as equal)
 *   nranks       1 <= nranks <= 8^L
 *   leaf_begin   nranks + 1 int64 (host, written): rank r owns the leaves
 *                leaf_begin[r] <= m < leaf_begin[r + 1]; every range holds at
 *                least one leaf, and rank r starts where the running cost is
 *                closest to r / nranks of the total
 *
 * hfmm_partition_let -- the locally essential tree (LET) of one rank: what it
 * needs from the other ranks for one apply whose targets lie in the leaves
 * flagged by leaf_tgt and whose sources lie in the leaves flagged by leaf_src.
 *   L, theta     the tree's depth and separation parameter (0 < theta <= 0.55;
 *                the lists are the library's own near and M2L lists)
 *   nranks, leaf_begin, rank   a partition (leaf_begin[0] = 0,
 *                non-decreasing, leaf_begin[nranks] = 8^L; empty ranges are
 *                allowed) and the rank, 0 <= rank < nranks
 *   leaf_tgt, leaf_src   8^L flags in Morton order (host, nonzero = holds
 *                targets / sources), or NULL for all leaves
 *   near_leaves  (host, written) ascending Morton codes of the leaves of
 *                other ranks that hold sources and lie in the near list
 *                (P2P, Sec. 5.1.2) of one of the rank's target leaves: their
 *                source weights travel to the rank
 *   cells        (host, written) for l = 2..L in turn, the ascending Morton
 *                codes of the level-l cells in the M2L list of one of the
 *                rank's target cells that hold a source leaf of another rank:
 *                every other rank with source leaves in such a cell sends its
 *                partial multipole of it (multipoles add over sources)
 *   near_cap, cells_cap  capacities of near_leaves and cells (entries)
 *   n_near       (written) entries of near_leaves
 *   cell_count   L + 1 int64 (written): cells of level l at cell_count[l]
 *                (entries 0 and 1 are zero)
 * near_leaves and cells both NULL: only the counts are written (a size
 * query).  Otherwise both must be given with capacity for every entry, else
 * HFMM_ERR_INVALID_ARG and nothing is written.
 */
int hfmm_partition_ranges(int L, const double* leaf_cost, int nranks, int64_t* leaf_begin);
int hfmm_partition_let(int L, double theta, int nranks, const int64_t* leaf_begin, int rank,
                       const uint8_t* leaf_tgt, const uint8_t* leaf_src, int64_t* near_leaves,
                       int64_t near_cap, int64_t* n_near, int64_t* cells, int64_t cells_cap,
                       int64_t* cell_count);

/*
 * hfmm_direct_sum_noalloc -- allocation-free direct Helmholtz sum.
 *
 * The paper has no counterpart to this entry point.  It exists for callers
 * that cannot allocate device memory (a host framework that forbids
 * cudaMalloc, an allocation-free real-time path, ...).  It allocates nothing:
 * its only scratch space, the partial sums of the source chunks, is a fixed
 * array inside the library (2^18 complex128 entries = 4 MiB, held by every
 * device that loads the library until the process exits).
 *
 *   phi_i = sum_{j : |x_i - y_j| > 0} q_j exp(i k |x_i - y_j|) / (4 pi |x_i - y_j|)
 *
 *   n_src, d_src_xyz, d_q   sources: AoS x,y,z float64 and complex128 weights (device)
 *   n_tgt, d_tgt_xyz        targets: AoS x,y,z float64 (device)
 *   k                       wavenumber (>= 0)
 *   d_phi                   n_tgt complex128 outputs (device), overwritten
 * Limits: n_tgt <= 262144 (larger sizes return HFMM_ERR_INVALID_ARG and
 * nothing is launched); the source set is split into at most
 * min(32, 262144 / n_tgt) chunks.  FP64 arithmetic, deterministic.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) for that device; make that first call before any
 * stream capture (a first call made while its stream is being captured
 * returns HFMM_ERR_UNSUPPORTED).  Calls on a stream that is not being
 * captured look the address up again, so a device reset between such calls
 * leaves no stale address behind.
 * Calls share the scratch array, so calls that overlap on the GPU (different
 * streams, or different host threads on one device) race and must be
 * serialised by the caller.  Every scratch entry a call reads is
 * written earlier in the same call, so no clearing is needed.
 */
int hfmm_direct_sum_noalloc(int64_t n_src, const double* d_src_xyz, const void* d_q,
                            int64_t n_tgt, const double* d_tgt_xyz, double k, void* d_phi,
                            void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HFMM_H */
