/*
 * rte.h -- C ABI of the GB300 (sm_103a) library for the rank-adaptive sweep-based SI-DSA
 * of the steady, single-group, first-order discrete-ordinates radiative transfer equation
 * in 2D x-y geometry (Guo & Peng, "Highly efficient rank-adaptive sweep-based SI-DSA for the
 * radiative transfer equation via mild space augmentation").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Status: 0 (RTE_OK) on success, a negative RTE_ERR_* code otherwise; the message of the
 *    last failure on the calling thread is returned by rte_last_error().  No C++ exception
 *    crosses this interface.
 *  - Ownership: the caller owns every buffer it passes (host arrays in rte_problem, device
 *    arrays passed to the compute calls).  The library owns the handle, its device workspace
 *    and the low-rank factors returned by rte_get_factors(), which stay valid until the next
 *    solve on the handle or rte_destroy().
 *  - Streams: every compute call is enqueued on the stream given to rte_setup() (the
 *    caller's CUDA stream, passed as void*).  Calls that return statistics synchronise that
 *    stream before returning; the others are asynchronous.
 *  - Mesh and DOF layout: nx x ny uniform cells on [x0,x1] x [y0,y1]; cell c = iy*nx + ix;
 *    N_x = 4 * nx * ny DOFs, cell-major, the 4 coefficients of a cell in the order of the
 *    orthonormal tensor Legendre basis (0,0), (1,0), (0,1), (1,1) (x degree, y degree).  A
 *    vector of N_x values is one column psi_j or the scalar flux phi (Sec. 2.1).
 *  - Angles: CL(n_theta, n_omz) quadrature (App. A); angle j = j2 * n_theta + j1 with
 *    theta_{j1} = (2 j1 + 1) pi / n_theta and Omega_z the j2-th Gauss-Legendre node.
 *  - Angular-flux blocks are column-major: psi[a * N_x + i] is DOF i of the a-th listed angle.
 *  - Precision: RTE_FP64 buffers are double, RTE_FP32 buffers are float.
 */
#ifndef RTE_H_
#define RTE_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------------------- */
#define RTE_OK                 0
#define RTE_ERR_ARG           -1  /* invalid argument (null pointer, size, index out of range) */
#define RTE_ERR_CUDA          -2  /* a CUDA runtime call failed */
#define RTE_ERR_NOMEM         -3  /* device or host allocation failed */
#define RTE_ERR_NOT_CONVERGED -4  /* outer iteration limit reached before the stop test held */
#define RTE_ERR_DEP_TIMEOUT   -5  /* a bounded device wait ran out (reported, never hangs) */
#define RTE_ERR_SINGULAR      -6  /* a Galerkin system had a zero pivot */
#define RTE_ERR_NAN           -7  /* a non-finite value appeared in the scalar flux */
#define RTE_ERR_STATE         -8  /* call not valid in the handle's current state */

#define RTE_FP64 0
#define RTE_FP32 1
#define RTE_DWF32 2     /* double-word FP32: hi + lo float pairs, about 48 significant bits,
                           computed on the FP32 pipe (low-rank basis passes only) */

#define RTE_UPDATE_MGS2A 0      /* basis update by MGS2-A (Alg. 2) */
#define RTE_UPDATE_MGSQR 1      /* one projection, full QR of the basis on a failed test (Sec. 4.2) */
#define RTE_UPDATE_QR 2         /* one projection, full QR after every inner iteration (Sec. 4.2) */

#define RTE_SAMPLE_RESIDUAL 0   /* residual-based randomized greedy sampling (Sec. 3.2) */
#define RTE_SAMPLE_DEIM 1       /* DEIM sampling (remark in Sec. 3.2) */

#define RTE_MODE_FR 0   /* full-rank SI-DSA (Sec. 2.2) */
#define RTE_MODE_LR 1   /* rank-adaptive low-rank SI-DSA (Sec. 3, Alg. 1) */

typedef struct rte_handle rte_handle;

/*
 * Problem statement (Sec. 2, Eq. rte; S_N-DG system Eq. mat-vec).  All arrays are HOST
 * arrays read during rte_setup() / rte_set_materials() only.
 *   sig_t, sig_s : [nx*ny] per-cell total and scattering cross sections (sigma_t > 0,
 *                  0 <= sigma_s <= sigma_t).
 *   q_cell       : [nx*ny] per-cell constant isotropic source, or NULL for none.
 *   q_rects      : [n_rect*5] rectangles (x0, x1, y0, y1, value) added to the source; the
 *                  moments int q eta_k over each cell are integrated exactly over the overlap.
 *   inflow       : isotropic inflow g on the left, right, bottom, top sides (0 = vacuum).
 *   q_gauss      : [n_gauss*4] isotropic Gaussian sources (xc, yc, a, amp) added to the source,
 *                  amp * exp(-a ((x - xc)^2 + (y - yc)^2)) with a > 0 (the source of the
 *                  experiments of Sec. 4.1, 4.3 and 4.4 is (0, 0, 100, 1)); the moments
 *                  int q eta_k over each cell are integrated exactly (separable erf forms).
 *                  n_gauss = 0 and q_gauss = NULL for none.
 */
typedef struct {
    int nx, ny;
    double x0, x1, y0, y1;
    int n_theta, n_omz;
    const double* sig_t;
    const double* sig_s;
    const double* q_cell;
    int n_rect;
    const double* q_rects;
    double inflow[4];
    int n_gauss;
    const double* q_gauss;
} rte_problem;

/*
 * Solver options.  Defaults (rte_default_opts) follow Sec. 4: eps_si = 1e-6,
 * eps_res = eps_diff = 1e-7, eps_svd = 1e-8, eps_mgs = 1e-10, p = 1, q = 8, 2 mandatory +
 * m_max = 4 adaptive MGS projections, DSA CG relative tolerance 1e-12, phi^(0) = 0.
 * With RTE_FP32 sweeps and sweep_refine = 1 (default) every sweep is followed by one defect
 * correction: r = b - (D_j + Sigma_t) psi in FP64, delta = (D_j + Sigma_t)^{-1} r in FP32,
 * psi + delta formed in FP64 (the S_N fixed point is ill-conditioned where sigma_s ~ sigma_t,
 * so plain FP32 sweeps stall at their rounding level there).
 */
typedef struct {
    int mode;               /* RTE_MODE_FR or RTE_MODE_LR */
    int sweep_precision;    /* RTE_FP64 or RTE_FP32 arithmetic inside the sweeps */
    double eps_si;          /* outer stop: ||phi^(n,*) - phi^(n-1)||_inf <= eps_si (Alg. 1) */
    double eps_res;         /* inner residual test (Eq. residual-chk) */
    double eps_diff;        /* inner scalar-flux test (Eq. phi-diff) */
    double eps_svd;         /* truncation tail ratio (Sec. 3.3) */
    double eps_mgs;         /* MGS2-A orthogonality test (Alg. 2) */
    double eps_break;       /* snapshot not appended when alpha <= eps_break * ||psi|| */
    double dsa_tol;         /* DSA CG relative residual tolerance */
    int dsa_max_iter;       /* DSA CG iteration cap */
    int use_dsa;            /* 0 = plain source iteration */
    int p, q;               /* sampled / candidate angles per inner iteration (Sec. 3.2);
                               1 <= p <= 64.  q >= the number of unsampled angles makes every
                               unsampled angle a candidate: the fully greedy sampling of the
                               remark in Sec. 3.2 (at most 1024 candidates per iteration) */
    int m_max;              /* adaptive MGS projections beyond the mandatory two */
    int mgs_test;           /* 0: |X(:,1)^T psi| as in Alg. 2, 1: max_i |X(:,i)^T psi| */
    int max_outer;          /* N_iter */
    int max_inner;          /* inner iteration cap per outer iteration */
    int truncate;           /* 0: none, 1: SVD of C after each inner loop (Sec. 3.3), 2: after the last outer iteration only */
    int want_factors;       /* 1: form X U, S, V after the last outer iteration */
    uint64_t seed;          /* Philox4x32-10 key for the random angle draws */
    int sweep_refine;       /* RTE_FP32 sweeps: FP64 defect-correction steps (0 or 1) */
    int dsa_precision;      /* RTE_FP64 or RTE_FP32 arithmetic in the DSA CG (FP64 inner products) */
    int basis_precision;    /* RTE_FP64 or RTE_DWF32 for the low-rank passes over the basis X
                               (MGS2-A projections and norms, the border products X^T W, the
                               candidate vectors X c_j and their residuals).  RTE_DWF32 holds X
                               also as hi + lo floats and accumulates by compensated (Dot2) sums:
                               results within about 1e-14 of the sums of absolute products. */
    int tc_projection;      /* RTE_DWF32 basis with r_cap <= 256 only: 1 forms the first MGS2-A
                               projection X^T Psi of each inner iteration's snapshots on the tensor
                               cores (tcgen05, split-TF32 operands, FP32 accumulation: about 1e-7 of
                               the sums of absolute products); the second projection (double-word)
                               removes its error, so the basis and R keep their double-word accuracy
                               (Alg. 2).  0 (default): the first projection in double-word FP32. */
    int sampling;           /* RTE_SAMPLE_RESIDUAL (default) or RTE_SAMPLE_DEIM: every inner iteration
                               forms the Galerkin coefficients C of all angles (Eq. lr_for_allangles)
                               and phi = X C w, stops when the change of phi is within eps_diff, and
                               else samples the DEIM points of the p leading right singular vectors
                               of C among the unsampled angles (q and eps_res are not used). */
    int basis_update;       /* RTE_UPDATE_MGS2A (default) or the ablation of Sec. 4.2 (Table 2):
                               RTE_UPDATE_MGSQR, one projection per snapshot and a full QR of the
                               basis (CholeskyQR2) whenever the orthogonality test fails (use
                               mgs_test = 1: the first-column test misses most single-pass losses);
                               RTE_UPDATE_QR, one projection and a full QR after every inner
                               iteration.  A full QR rebuilds every projected operator and Galerkin
                               factor (the incremental update needs the hierarchical basis).  FP64
                               basis passes only; stats.full_qr counts the full QRs. */
} rte_opts;

/* Statistics of the last solve (valid when the call returns). */
typedef struct {
    int status;
    int converged;
    int outer_iters;
    int total_inner;        /* inner iterations summed over outer iterations */
    int total_sweeps;       /* single-ordinate sweeps performed */
    int max_rank;           /* largest r_k reached */
    int final_rank;         /* r_k of the last inner loop */
    int final_rank_trunc;   /* r' after the last truncation */
    int mgs_failures;       /* Alg. 2 "orthogonality failure" count */
    int breakdowns;         /* snapshots not appended */
    int full_checks;        /* inner iterations that formed all of C */
    int dsa_cg_iters;       /* CG iterations summed over DSA solves */
    double last_diff;       /* last ||phi^(n,*) - phi^(n-1)||_inf */
    long long cell_angle_updates;  /* cells x ordinates swept (each sweep counts N_c) */
    int full_qr;            /* full QRs of the basis (basis_update MGS-QR / QR) */
} rte_stats;

/* Fill *o with the defaults listed above (mode = FR, FP64 sweeps). */
void rte_default_opts(rte_opts* o);

/* Message of the last failure on this thread ("" if none).  Owned by the library. */
const char* rte_last_error(void);

/*
 * Create a handle for one problem (Sec. 2.1, App. A, App. B): computes the CL quadrature,
 * the source moments G, the inflow data and uploads the materials; allocates the device
 * workspace.  stream: cudaStream_t (may be NULL for the legacy default stream).
 * Errors: RTE_ERR_ARG (bad sizes/pointers), RTE_ERR_NOMEM, RTE_ERR_CUDA.
 */
int rte_setup(const rte_problem* prob, void* stream, rte_handle** out);

/* Release the handle and all library-owned device memory.  NULL is accepted. */
int rte_destroy(rte_handle* h);

/* Replace sig_t, sig_s and q_cell (host arrays, [nx*ny]; q_cell may be NULL = keep) of an
 * existing handle, re-deriving G; the mesh, rectangles and quadrature are unchanged. */
int rte_set_materials(rte_handle* h, const double* sig_t, const double* sig_s, const double* q_cell);

/*
 * Failure detection (no paper counterpart).  Every wait of a sweep's band hand-off (one warp
 * waiting for the band below it to finish a column) polls a progress counter at most `spins`
 * times; a wait that runs out sets a device flag, the sweep finishes (its output is then
 * invalid) and the call returns RTE_ERR_DEP_TIMEOUT instead of hanging.  spins = 0 restores the
 * default (2^22 polls, far beyond any legitimate wait); a small limit makes the waits run out
 * on purpose.  Errors: RTE_ERR_ARG.
 */
int rte_set_wait_limit(rte_handle* h, int spins);

/*
 * Host-side failure injection for tests (no paper counterpart).  With code = RTE_ERR_SINGULAR
 * the next low-rank solve on h behaves as if the zero-pivot check of the bordered Galerkin LU
 * (Eq. galerkin-projection) had fired in its first inner iteration: the solve releases its
 * state and returns RTE_ERR_SINGULAR.  (With sigma_t > 0 the Galerkin matrices have a positive
 * definite symmetric part, so valid data never reach a zero pivot; a non-finite pivot, from
 * non-finite data, returns RTE_ERR_NAN.)  code = 0 clears it.  Errors: RTE_ERR_ARG.
 */
int rte_inject_failure(rte_handle* h, int code);

/* Sizes: n_dof = 4*nx*ny, n_angles = n_theta*n_omz (any pointer may be NULL). */
int rte_get_sizes(const rte_handle* h, int* n_dof, int* n_cells, int* n_angles);

/* Copy the quadrature (host outputs, [n_angles] each; any pointer may be NULL). */
int rte_get_quadrature(const rte_handle* h, double* ox, double* oy, double* oz, double* w);

/* Copy the source moments G(k) = int G eta_k (App. B) to a DEVICE buffer [N_x] (double). */
int rte_get_source(const rte_handle* h, double* G_dev);

/*
 * Transport sweeps (Sec. 2.2): for each listed angle j solve (D_j + Sigma_t) psi_j = b_j by
 * one upwind pass over the mesh, cell by cell, with the 4x4 local system solved in
 * registers.  b_j = src (+ g_j^bc when add_inflow).
 *   angles      : HOST [n_angles] angle indices in [0, N_Omega).
 *   src         : DEVICE [N_x] shared by all angles, or [n_angles*N_x] when src_per_angle.
 *   psi_out     : DEVICE [n_angles*N_x] or NULL.
 *   phi_out     : DEVICE [N_x] double or NULL; receives sum_a omega_{j_a} psi_{j_a}.
 *   precision   : RTE_FP64 (double src/psi) or RTE_FP32 (float src/psi).
 *   src, psi_out and phi_out must be 16-byte aligned (RTE_ERR_ARG otherwise).
 * Errors: RTE_ERR_ARG.
 */
int rte_sweep(rte_handle* h, const int* angles, int n_angles, int precision,
              const void* src, int src_per_angle, int add_inflow, void* psi_out, double* phi_out);

/*
 * Adjoint sweeps: solve (D_j + Sigma_t)^T mu_j = src for the listed angles.  With the upwind
 * DG operators, D_x^{+T} = -D_x^- and D_y^{+T} = -D_y^-, so the transposed system is the
 * forward system of the reversed direction -Omega_j with zero inflow; same arguments as
 * rte_sweep (no inflow term).
 */
int rte_sweep_adjoint(rte_handle* h, const int* angles, int n_angles, int precision,
                      const void* src, int src_per_angle, void* mu_out, double* chi_out);

/*
 * Launch configuration of the single-problem sweep (no paper counterpart: the sweep of
 * Sec. 2.2 is the same computation in every configuration, cell by cell in the same order of
 * operations, so psi is bit-identical across configurations).
 *   kernel           : RTE_SWEEP_BAND for meshes of nx >= 32 and ny > 32 (one block per ordinate;
 *                      rows in bands of 32, one warp per band in flight, lanes on the rows of a
 *                      band, anti-diagonal wavefront), else RTE_SWEEP_WARP (one warp per ordinate).
 *   warps            : band kernel: warps per block W in [1, 16], W <= the band count nb; the
 *                      wavefront tile is 32 W rows; W < nb (warps take bands cyclically) needs
 *                      nx >= 32 W + 4.
 *   depth            : band kernel: prefetch depth in wavefront steps (2, 4 or 8).
 *   staged           : band kernel: psi stores gathered per row segment in shared memory (1) or
 *                      one store per lane and cell (0).
 *   angles_per_block : ordinates per block (1, 2 or 4): the warp kernel runs them side by side
 *                      (one warp each), the band kernel one after the other (a persistent grid
 *                      of ceil(n / angles_per_block) blocks).
 *   ms               : time of one launch measured by the autotuner (0 when not measured).
 * The library keeps one configuration per handle, precision, launch width n (ordinates per
 * launch) and whether psi is written.  The first uncaptured sweep of such a kind times every
 * valid configuration on the call's own buffers (a few launches each, not recorded by the
 * profiler) and keeps the fastest; launches inside a graph capture or with a device-side
 * ordinate count use the cached choice, else the built-in default.  A
 * low-rank solve tunes its p-ordinate sweeps before its first capture.
 */
#define RTE_SWEEP_BAND 1
#define RTE_SWEEP_WARP 2
typedef struct rte_sweep_config {
    int kernel;
    int warps;
    int depth;
    int staged;
    int angles_per_block;
    float ms;
} rte_sweep_config;

/*
 * Run the sweep autotuner now for launches of n ordinates (1 <= n <= N_Omega) in `precision`,
 * with psi written (with_psi = 1) or not, on the handle's stream with library scratch buffers
 * (the distinct directions, repeated up to n), cache the winner and return it in *out
 * (may be NULL).  Synchronises the stream.  Errors: RTE_ERR_ARG, RTE_ERR_NOMEM.
 */
int rte_sweep_tune(rte_handle* h, int precision, int n, int with_psi, rte_sweep_config* out);

/*
 * Force the configuration of that kind of launch (validated against the mesh: RTE_ERR_ARG if
 * invalid); cfg = NULL forgets it (the next uncaptured sweep of that kind tunes again).
 */
int rte_sweep_set_config(rte_handle* h, int precision, int n, int with_psi, const rte_sweep_config* cfg);

/*
 * The configuration that kind of launch uses now: the cached one, else the built-in default
 * (ms = 0).  Errors: RTE_ERR_ARG.
 */
int rte_sweep_get_config(rte_handle* h, int precision, int n, int with_psi, rte_sweep_config* out);

/*
 * SI-DSA solve (Sec. 2.2 for RTE_MODE_FR; Sec. 3 and Alg. 1-2 for RTE_MODE_LR).
 *   phi_inout : DEVICE [N_x] double; on entry phi^(0), on exit the converged phi^(n,*).
 *   stats     : may be NULL.
 * Returns RTE_OK when the outer stop test held, RTE_ERR_NOT_CONVERGED at max_outer.
 */
int rte_si_dsa_solve(rte_handle* h, const rte_opts* opts, double* phi_inout, rte_stats* stats);

/*
 * Batched transport sweeps over nprob independent problems in ONE kernel launch (no paper
 * counterpart: many problems of uneven mesh size and ordinate count share the GPU).  Each CTA
 * takes one (problem, ordinate) work item and runs the same upwind pass as rte_sweep (Sec. 2.2).
 *   hs[i]       : distinct handles; the launch runs on hs[0]'s stream after every handle's
 *                 stream has drained.
 *   angles[i]   : HOST [n_angles[i]] angle indices of problem i (0 <= n_angles[i] <= N_Omega_i).
 *   src[i]      : DEVICE [N_x_i] source shared by problem i's angles (FP64 or FP32 as precision).
 *   add_inflow  : add g_j^bc of each problem's inflow data.
 *   psi_out[i]  : DEVICE [n_angles[i] * N_x_i]; src[i] and psi_out[i] 16-byte aligned.
 * If any mesh has ny > 512 (more than 16 bands of 32 rows), or a mesh is too wide for the
 * shared-memory trace ring of the batch's block size, the problems are swept one at a time
 * with rte_sweep; the results are the same.  Errors: RTE_ERR_ARG, RTE_ERR_DEP_TIMEOUT.
 */
int rte_sweep_batch(rte_handle* const* hs, int nprob, const int* const* angles, const int* n_angles,
                    int precision, const void* const* src, int add_inflow, void* const* psi_out);

/*
 * SI-DSA of nprob independent problems in one call (no paper counterpart); opts are shared by
 * all problems and each problem stops on its own test.
 *   RTE_MODE_FR (Sec. 2.2): lock step; per outer iteration one batched sweep launch for all
 *     unconverged problems and one cooperative CG launch for all their DSA corrections.  Runs
 *     on hs[0]'s stream.
 *   RTE_MODE_LR (Alg. 1): the problems' low-rank solves run concurrently, each as the
 *     single-problem rte_si_dsa_solve (same kernels, graphs and results) on one of up to 32
 *     library-owned streams driven by as many host threads, largest problem first; a problem
 *     of low rank finishes early and its thread takes the next one.  Each solve starts after
 *     the work queued on its handle's stream, and that stream waits for the solve.  The
 *     handles must not be used by other threads during the call.
 *   phi[i]    : DEVICE [N_x_i] double, phi^(0) on entry, converged phi on exit; distinct.
 *   stats     : NULL or [nprob].
 * All handles on one device.  Returns RTE_OK when every problem converged, else
 * RTE_ERR_NOT_CONVERGED (stats[i].converged tells which), or the first other error of any
 * problem (RTE_ERR_ARG, RTE_ERR_DEP_TIMEOUT, RTE_ERR_SINGULAR, RTE_ERR_NAN, RTE_ERR_CUDA).
 */
int rte_si_dsa_solve_batch(rte_handle* const* hs, int nprob, const rte_opts* opts, double* const* phi,
                           rte_stats* stats);

/*
 * One backward-Euler step of the time-dependent problem (Sec. 3.7; particle speed 1, step dt):
 *   (D_j + Sigma_t + M/dt) psi_j^{n+1} - Sigma_s phi^{n+1} = G + g_j^bc + M psi_j^n / dt
 * for every ordinate j.  With the orthonormal DG basis the mass matrix M is the identity on
 * every cell, so the step is the steady problem with sigma_t + 1/dt per cell and the extra
 * per-ordinate source psi_j^n / dt.  It is solved by full-rank SI-DSA (Alg. 1's loop and stop
 * test) over every ordinate (no +-Omega_z folding: psi^n need not be symmetric), the DSA
 * correction using the MIP operator of sigma_t + 1/dt.  With RTE_MODE_LR the step runs the
 * low-rank SI-DSA of Alg. 1 on that steady problem instead: the time source of each sampled
 * ordinate in its sweep, its products with the basis columns in the bordered Galerkin
 * right-hand sides, and the source in the candidate residuals; psi^{n+1} = X C of the last
 * inner loop.  psi_prev must then be equal on +-Omega_z twin pairs (RTE_ERR_ARG otherwise: a
 * pair is solved once), with residual sampling, MGS2-A and no tensor-core projection.
 *   opts      : mode RTE_MODE_FR or RTE_MODE_LR; sweep_precision RTE_FP64, or RTE_FP32 with
 *               sweep_refine = 0 (the FP64 defect correction takes a source shared by all
 *               ordinates).
 *   dt        : finite, > 0.
 *   psi_prev  : DEVICE double [N_Omega][N_x] psi^n (ordinate-major).
 *   psi_next  : DEVICE double [N_Omega][N_x] psi^{n+1} out: the last sweep's, consistent with
 *               phi^{n+1}; may alias psi_prev.
 *   phi_inout : DEVICE double [N_x]: the initial guess (phi^n, say) in, phi^{n+1} out.
 *   stats     : may be NULL.
 * The full-rank step allocates 2 N_Omega N_x values of the sweep precision as scratch for the
 * call, the low-rank step (N_Omega / 2) N_x doubles (the time source of the distinct directions).
 * The handle's materials are those of the steady problem before and after the call.
 * Runs on the handle's stream and synchronises it.  Returns RTE_OK, RTE_ERR_NOT_CONVERGED at
 * max_outer, RTE_ERR_ARG, RTE_ERR_NOMEM, RTE_ERR_NAN, RTE_ERR_DEP_TIMEOUT.
 */
int rte_be_step(rte_handle* h, const rte_opts* opts, double dt, const double* psi_prev, double* psi_next,
                double* phi_inout, rte_stats* stats);

/*
 * Low-rank factors of the last RTE_MODE_LR solve with want_factors = 1 (Sec. 3.3):
 * Psi ~ X diag(S) V^T with X [N_x x r'] (DEVICE, column-major), S [r'], V [N_Omega x r']
 * (DEVICE, column-major).  Pointers are library-owned.  Errors: RTE_ERR_STATE.
 */
int rte_get_factors(rte_handle* h, const double** X, const double** S, const double** V, int* rank);

/*
 * Inspection of the low-rank state left by the last RTE_MODE_LR solve (tests, diagnostics): the
 * basis X of its last inner loop and the projected operators bordered incrementally as X grew
 * (Sec. 3.4): X^T D_x^- X, X^T D_y^- X and X^T Sigma_t X.
 *   rank : columns r of X; ld : leading dimension of the operators (r x r used, column-major:
 *          entry (i, k) = x_i^T A x_k at [k * ld + i]).
 *   X    : DEVICE [r][N_x] (column-major N_x x r, FP64).
 * Pointers are library-owned, valid until the next solve or rte_destroy; any may be NULL.
 * Errors: RTE_ERR_ARG, RTE_ERR_STATE (no low-rank solve has left a basis).
 */
int rte_get_lowrank_state(rte_handle* h, int* rank, int* ld, const double** X, const double** Pxm,
                          const double** Pym, const double** T);

/*
 * Gradient of the detector response R = d^T phi at a converged phi with respect to the
 * per-cell sigma_t, sigma_s and the per-cell constant source q (discrete adjoint of
 * Eq. mat-vec-a):  (D_j + Sigma_t)^T mu_j = d + Sigma_s chi,  chi = sum_j omega_j mu_j,
 * dR/dsigma_t,c = -sum_j omega_j mu_j|_c . psi_j|_c,  dR/dsigma_s,c = chi|_c . phi|_c,
 * dR/dq_c = chi|_c . int_c eta.   psi_j is regenerated by a sweep from phi.
 *   phi, det      : DEVICE [N_x] double.
 *   d_sig_t, d_sig_s, d_q : DEVICE [N_c] double outputs (any may be NULL).
 *   opts          : eps_si / DSA settings / sweep precision used for the adjoint solve.
 */
int rte_adjoint_grad(rte_handle* h, const rte_opts* opts, const double* phi, const double* det,
                     double* d_sig_t, double* d_sig_s, double* d_q, rte_stats* stats);

/*
 * Projection of a block of vectors onto a spatial basis on the tensor cores (the first
 * projection "Delta c = X^T psi" of Alg. 2 for a block of snapshots, Sec. 3.1):
 *   out[v * r + k] = sum_i X[k * N_x + i] * Psi[v * N_x + i],   k < r, v < nv <= 8,
 * N_x = the handle's DOF count.  X: DEVICE float [r][N_x] (basis columns, column-major as an
 * N_x x r matrix), Psi: DEVICE float [nv][N_x], both 16-byte aligned; out: DEVICE double [nv * r].
 * tcgen05 MMAs on split-TF32 operands (each FP32 entry as a TF32 high part plus a TF32 low part,
 * four products) with FP32 accumulation in tensor memory: each sum is accurate to a few 1e-7 of
 * the sum of the absolute products.  Runs on the handle's stream and synchronises it (a bounded
 * wait inside the kernel that runs out returns RTE_ERR_DEP_TIMEOUT).  Errors: RTE_ERR_ARG.
 */
int rte_basis_project(rte_handle* h, const float* X, int r, const float* Psi, int nv, double* out);

/* Apply the MIP diffusion operator of the DSA step, y = A_MIP x (DEVICE, double [N_x]). */
int rte_dsa_apply(rte_handle* h, const double* x, double* y);

/* Solve A_MIP dphi = rhs by the library's preconditioned CG (DEVICE double [N_x]);
 * *iters receives the iteration count.  Relative tolerance tol, at most max_iter steps.
 * Preconditioner: block Jacobi on the 4x4 cell blocks plus a multigrid V-cycle on the
 * continuous bilinear (vertex) subspace, the same one the DSA step of rte_si_dsa_solve uses. */
int rte_dsa_solve(rte_handle* h, const double* rhs, double* x, double tol, int max_iter, int* iters);

/*
 * Allocation-free DSA solve.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory (another component owns the device-memory budget
 * through its own pool, the host forbids allocation after start-up so that memory use stays
 * fixed, or the caller must not trigger a synchronising cudaMalloc mid-run).  It solves the
 * same MIP diffusion system as rte_dsa_solve by CG preconditioned with block Jacobi only (no
 * multigrid hierarchy), for the problem given directly by its mesh and DEVICE cross sections,
 * and allocates nothing:
 *   sig_t, sig_s : DEVICE [nx*ny] double; rhs, x : DEVICE [4*nx*ny] double (x is written);
 *   tol, max_iter: CG relative tolerance and iteration cap; iters: host out (may be NULL);
 *   stream       : cudaStream_t the work is enqueued on.
 * Scratch: one file-scope device array of about 5.1 MB (every GPU that loads the library holds
 * it until exit) limits the mesh to 16384 cells; larger meshes return RTE_ERR_ARG.  Every call
 * looks the array's address up (cudaGetSymbolAddress) on the current device; the first call on
 * a device also loads the library's device code there, so make that first call before any
 * stream capture.  All calls share the array and
 * keep the last call's contents (every value is rewritten before use): calls that overlap on
 * the GPU race and must be ordered by the caller.  With iters != NULL the call synchronises
 * the stream.
 */
int rte_dsa_solve_static(int nx, int ny, double x0, double x1, double y0, double y1, const double* sig_t,
                         const double* sig_s, const double* rhs, double* x, double tol, int max_iter, int* iters,
                         void* stream);

/*
 * Instrumentation (measurement only; the paper has no counterpart): per kernel class, CUDA
 * events recorded on the handle's stream around every launch while enabled.
 *   rte_profile_enable: on != 0 starts (and zeroes) the counters, 0 stops recording.
 *   rte_profile_read:   total device time (ms), launch count, algorithmic bytes moved and
 *                       flops of the class since the last enable (synchronises the stream).
 * Classes: RTE_PROF_SWEEP (transport sweeps), RTE_PROF_DSA (diffusion CG), RTE_PROF_BASIS
 * (passes over the spatial basis X: projections, X c products), RTE_PROF_GALERKIN (bordered
 * LU updates and back-substitutions), RTE_PROF_RESID (stencil applications: operator
 * borders and candidate residuals), RTE_PROF_SVD (truncation), RTE_PROF_PASS (the double-word
 * projection pass fused with the next X^T v: v - X dc and X^T (v - X dc) in one read of X),
 * RTE_PROF_XC (the candidate vectors X c_j), RTE_PROF_XT (double-word X^T V passes: the first
 * products of all snapshots, the border products X^T W), RTE_PROF_TC (the first products on the
 * tensor cores, tc_projection = 1).
 * While profiling, the low-rank solve reads the rank and the MGS2-A loop state back from the
 * device at every snapshot, so only launches that do work are issued and counted (kernels
 * whose gate is closed are skipped) and the byte and flop counts use the exact rank.
 */
#define RTE_PROF_SWEEP 0
#define RTE_PROF_DSA 1
#define RTE_PROF_BASIS 2
#define RTE_PROF_GALERKIN 3
#define RTE_PROF_RESID 4
#define RTE_PROF_SVD 5
#define RTE_PROF_PASS 6
#define RTE_PROF_XC 7
#define RTE_PROF_XT 8
#define RTE_PROF_TC 9
#define RTE_PROF_NCLASS 10
int rte_profile_enable(rte_handle* h, int on);
int rte_profile_read(rte_handle* h, int cls, double* ms, long long* launches, double* bytes, double* flops);

#ifdef __cplusplus
}
#endif
#endif /* RTE_H_ */
