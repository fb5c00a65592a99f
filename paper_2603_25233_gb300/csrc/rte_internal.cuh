// Internal declarations of the RTE library (handle layout, kernels' launch wrappers).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <condition_variable>
#include <mutex>
#include <map>
#include <set>
#include <shared_mutex>
#include <utility>
#include <string>
#include <vector>

#include "../../include/rte.h"

namespace rte {

// Thread-local last-error message; set by fail() and returned by rte_last_error().
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);

// Calls that can synchronise the device (allocation and release of device or pinned memory, a
// device-wide synchronisation) invalidate a stream capture in progress on another host thread,
// as in a low-rank batch whose solves run on several threads.  Captures therefore hold
// alloc_capture_mutex() shared and those calls hold it exclusively.  Both locks are reentrant
// per thread, and a thread inside its own capture never takes the exclusive one (any such call
// there fails as a capture error, as it would without the lock).
std::shared_mutex& alloc_capture_mutex();
extern thread_local int tl_capture_depth;
extern thread_local int tl_alloc_depth;
struct AllocLock {
    bool counted;
    AllocLock() : counted(tl_capture_depth == 0) {
        if (counted && tl_alloc_depth++ == 0) alloc_capture_mutex().lock();
    }
    ~AllocLock() {
        if (counted && --tl_alloc_depth == 0) alloc_capture_mutex().unlock();
    }
    AllocLock(const AllocLock&) = delete;
    AllocLock& operator=(const AllocLock&) = delete;
};
struct CaptureLock {
    bool counted;
    CaptureLock() : counted(tl_alloc_depth == 0) {
        if (counted && tl_capture_depth++ == 0) alloc_capture_mutex().lock_shared();
    }
    ~CaptureLock() {
        if (counted && --tl_capture_depth == 0) alloc_capture_mutex().unlock_shared();
    }
    CaptureLock(const CaptureLock&) = delete;
    CaptureLock& operator=(const CaptureLock&) = delete;
};
// The host threads of a low-rank batch enter the batch's gate while they issue CUDA calls and
// leave it while they wait for their stream.  A stream capture holds the gate alone (waiting
// for every other thread to leave it; threads that arrive meanwhile wait), so that no call of
// another thread (an allocation, a kernel's first load, a graph instantiation, ...) can
// invalidate the capture.
class BatchGate {
  public:
    void enter();
    void leave();
    void capture_begin();
    void capture_end();
  private:
    std::mutex m_;
    std::condition_variable cv_;
    int active_ = 0, waiting_ = 0;
    bool capturing_ = false;
};
extern thread_local BatchGate* tl_gate;        // the gate of this batch worker thread, or null
extern thread_local int tl_gate_capture_depth;
struct GateCapture {                            // scope of a capture (reentrant)
    BatchGate* g;
    GateCapture() : g(tl_gate) {
        if (g && tl_gate_capture_depth++ == 0) { g->leave(); g->capture_begin(); }
    }
    ~GateCapture() {
        if (g && --tl_gate_capture_depth == 0) { g->capture_end(); g->enter(); }
    }
    GateCapture(const GateCapture&) = delete;
    GateCapture& operator=(const GateCapture&) = delete;
};
// Wait for a stream outside the gate.
cudaError_t gate_stream_sync(cudaStream_t st);

// Programmatic dependent launch (sm_90 and later): the kernel-to-kernel edges of a captured
// low-rank iteration graph are programmatic, so a kernel may be launched as its predecessor's
// blocks exit, before the predecessor has fully completed; it starts by waiting until the grids it
// depends on have completed and their writes are visible (a no-op when it was not launched with a
// programmatic dependency).  Every kernel of the files whose kernels run in those graphs calls it
// first.  (Letting dependents launch earlier, from this point, measured slower.)
__device__ __forceinline__ void pdl_entry() {
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
}

// Allow a kernel up to `bytes` of dynamic shared memory.  Above the 48 KB default the kernel's
// limit is raised once per device to the opt-in maximum (less its static shared memory), so
// that no launch changes a function attribute while that kernel runs on another stream or a
// capture is in progress.
int smem_optin(const void* func, size_t bytes);
template <typename F>
inline int smem_optin(F* func, size_t bytes) { return smem_optin((const void*)func, bytes); }

// cudaFree / cudaMallocHost / cudaFreeHost under AllocLock.
void dev_free(void* p);
cudaError_t pinned_alloc(void** p, size_t n);
void pinned_free(void* p);

#define RTE_CUDA_TRY(expr)                                                              \
    do {                                                                                \
        cudaError_t _e = (expr);                                                        \
        if (_e != cudaSuccess)                                                          \
            return ::rte::fail(RTE_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
    } while (0)

#define RTE_TRY(expr)               \
    do {                            \
        int _s = (expr);            \
        if (_s != RTE_OK) return _s; \
    } while (0)

// Device allocation that records into the handle's list (freed by rte_destroy).
struct DeviceArena {
    std::vector<void*> ptrs;
    size_t bytes = 0;
    int alloc(void** p, size_t n);
    // (re)allocate *buf to hold at least need bytes (contents are not kept)
    int grow(void** buf, size_t* cap, size_t need);
    void release_all();
};

// Vertex-grid multigrid hierarchy of the DSA preconditioner (kernels in rte_mg.cuh).
constexpr int kMgMaxLevels = 16;
constexpr int kMgCoarseMax = 100;
#ifndef RTE_MG_BLOCK_MAX64
#define RTE_MG_BLOCK_MAX64 300
#endif
#ifndef RTE_MG_BLOCK_MAX32
#define RTE_MG_BLOCK_MAX32 1100
#endif
// V-cycle levels up to this many vertices run in one thread block (below that size a grid-wide
// sync costs more than the level's work); FP32 arithmetic affords larger single-block levels.
constexpr int kMgBlockMax64 = RTE_MG_BLOCK_MAX64;
constexpr int kMgBlockMax32 = RTE_MG_BLOCK_MAX32;

struct MgLevel {
    int nx, ny;       // vertices in x and y
    int cx, cy;       // 1 if that dimension is halved on the next level
    double* S;        // [9][N] stencil, position d = (di + 1) + 3 (dj + 1)
    double* dinv;     // [N] 1 / (l1 norm of the stencil row)
    double* b;        // [N] right-hand side
    double* x;        // [N] scratch (first sweep, residual)
    double* y;        // [N] iterate
    float *S32, *dinv32, *b32, *x32, *y32;   // the same in FP32 (the V-cycle of the FP32 CG)
};

struct MgArgs {
    int L;            // number of vertex levels (the last one is solved directly)
    int ncx, ncy;     // cells of the DG level
    double g;         // sqrt(hx hy)
    double* Ainv;     // [N_{L-1}^2] inverse of the coarsest operator (row-major)
    float* Ainv32;
    int lb64, lb32;   // first level handled by one block (FP64 / FP32 V-cycle), <= L - 1
    MgLevel lv[kMgMaxLevels];
};

// Tensor maps of the tensor-core first projection X^T Psi (rte_tc.cu): the basis [r_cap][N_x]
// and the snapshots [64][N_x], each as a TF32 high part and an FP32 remainder (CUtensorMap
// storage, 128 bytes each).
struct TcProjection {
    alignas(64) unsigned char maps[4 * 128];
    int N = 0, rc = 0;
    bool ready = false;
};
int tc_projection_prepare(TcProjection* P, const float* Xt, const float* Xl, int N, int rc, const float* Vt,
                          const float* Vl, int nv_total);
// x -> (TF32 high part, FP32 remainder), n entries
int tc_split(const float* x, long long n, float* t, float* l, cudaStream_t s);
// part[((b kxtv) + v) rc + k] = rows of block b of X(:, k)^T Psi(:, v0 + v) (k < *rank, v < nv <= 8),
// npart[v nblk + b] = the rows' sum of psi2(:, v0 + v)^2; nothing when *stop
int tc_projection_launch(const TcProjection* P, int v0, int nv, int rows_per_cta, int nblk, const int* stop,
                         const int* rank, double* part, int kxtv, const float2* psi2, double* npart, int* err,
                         cudaStream_t s);

// State of the rank-adaptive low-rank SI (Sec. 3); sized for r_cap basis vectors.
struct LowRankState {
    int r_cap = 0;          // capacity of X (columns)
    int n_dir = 0;          // distinct (Omega_x, Omega_y) directions (twins folded)
    double* X = nullptr;    // [N_x * r_cap] column-major basis (FP64)
    double* R = nullptr;    // [r_cap * r_cap] coefficient columns, column a of R belongs to X column a
    double* Pxm = nullptr;  // [r_cap * r_cap] X^T D_x^- X (column-major, ld r_cap)
    double* Pym = nullptr;  // X^T D_y^- X
    int last_rank = 0;      // rank of the last inner loop of the last solve (inspection)
    double* T = nullptr;    // X^T Sigma_t X
    double* bS = nullptr;   // [r_cap] X^T S   (S = Sigma_s phi + G)
    double* bE = nullptr;   // [4 * r_cap] X^T e_side (inflow side vectors)
    double* LUl = nullptr;  // [n_dir * r_cap * r_cap] unit-lower factors (column-major per direction)
    double* LUu = nullptr;  // [n_dir * r_cap * r_cap] upper factors (row-major per direction)
    double* Udinv = nullptr;// [n_dir * r_cap] reciprocals of the diagonals of the upper factors
    double* Y = nullptr;    // [n_dir * r_cap] forward-substituted right-hand sides
    double* Cdir = nullptr; // [n_dir * r_cap] Galerkin coefficients per direction (when solved)
    double* W = nullptr;    // [N_x * 8] stencil images of the newest column
    double* snap = nullptr; // [N_x * p] snapshots (FP64)
    void* snap_lo = nullptr;// [N_x * p] snapshots in sweep precision
    double* vcand = nullptr;// [N_x * q] X c_j of the candidates
    size_t vcand_bytes = 0, ccand2_bytes = 0;
    void*& vcand_void() { return reinterpret_cast<void*&>(vcand); }
    void*& ccand2_void() { return reinterpret_cast<void*&>(ccand2); }
    float2* X2 = nullptr;   // [N_x * r_cap] X as double-word FP32 (hi, lo), double-word basis passes
    float* Xt = nullptr;    // [N_x * r_cap] TF32 high part of X2's hi (tensor-core first projection)
    float* Xl = nullptr;    // [N_x * r_cap] the FP32 remainder
    float* snap_t = nullptr;// [64 * N_x] the same split of the double-word snapshots' hi
    float* snap_l = nullptr;
    TcProjection tc;
    float2* S2 = nullptr;   // [N_x] S as double-word
    float2* E2 = nullptr;   // [4 N_x] inflow side vectors as double-words
    float2* ccand2 = nullptr;  // [64 * r_cap] candidate coefficients as double-word
    double* red = nullptr;  // reduction scratch
    double* small = nullptr;// [small_len] device small vectors (coefficients, norms, ...)
    int* ints = nullptr;    // device integer state
    double* host_small = nullptr;  // pinned mirror of the status block
    int* host_ints = nullptr;
    double* phi_old = nullptr;     // [N_x]
    double* phi_k = nullptr;       // [N_x]
    double* Cfull = nullptr;       // [r_cap * N_Omega]
    double* svd_A = nullptr;       // [N_Omega * r_cap] work for the Jacobi SVD
    double* svd_W = nullptr;       // [r_cap * r_cap]
    double* svd_s = nullptr;       // [r_cap]
    double* fX = nullptr;          // [N_x * r_cap] factor X U (library-owned output)
    double* fS = nullptr;
    double* fV = nullptr;
    int factor_rank = 0;
    bool ready = false;
};

// CUDA-event timing per kernel class (enabled by rte_profile_enable).
struct Profiler {
    struct Rec {
        int cls;
        cudaEvent_t a, b;
        double bytes, flops;
    };
    bool on = false;
    std::vector<cudaEvent_t> free_ev;
    std::vector<Rec> pending;
    double ms[16] = {0}, bytes[16] = {0}, flops[16] = {0};
    long long launches[16] = {0};
    cudaEvent_t open_ev = nullptr;
    int open_cls = -1;
    cudaEvent_t get_event();
    void begin(int cls, cudaStream_t st);
    int end(int cls, cudaStream_t st, double bytes, double flops);   // index of the record
    void flush();      // caller synchronised the stream
    void reset();
    ~Profiler();
};

}  // namespace rte

struct rte_handle {
    int nx = 0, ny = 0, nc = 0, ndof = 0, nang = 0, n_theta = 0, n_omz = 0;
    double x0 = 0, x1 = 0, y0 = 0, y1 = 0, hx = 0, hy = 0;
    double inflow[4] = {0, 0, 0, 0};
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;   // private stream for CUDA-graph capture
    cudaStream_t cap_stream2 = nullptr;  // capture of conditional-node bodies
    cudaStream_t border_stream = nullptr;   // low-rank border branch of the captured graph
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int num_sms = 0;
    int device = 0;               // CUDA device the handle was created on
    cudaEvent_t ev_pinned = nullptr;  // after the last copy from the pinned staging buffers
    bool pinned_busy = false;          // ev_pinned recorded and not yet waited for
    double* h_wlist = nullptr;         // pinned [nang] weights of an rte_sweep call's phi reduction

    std::vector<double> ox, oy, oz, w;        // quadrature (host)
    std::vector<int> twin;                    // +-Omega_z twin of each angle
    std::vector<int> fold_rep;                // one angle per distinct direction
    std::vector<double> fold_w;               // summed weights of the twins
    std::vector<double> rects;                // source rectangles (host)
    std::vector<double> gauss;                // Gaussian sources (xc, yc, a, amp) (host)
    std::vector<double> sig_t_h, sig_s_h, q_h;
    bool has_q = false;

    rte::DeviceArena arena;
    // materials and data (device)
    double* sig_t = nullptr;
    double* sig_s = nullptr;
    float* sig_t_f = nullptr;
    float* sig_dw = nullptr;      // [2 nc] sigma_t as FP32 hi, lo (double-word defect)
    float* b_dw = nullptr;        // [2 N_x] defect right-hand side as FP32 hi, lo
    double* G = nullptr;          // [N_x] source moments
    double* e_side = nullptr;     // [4 * N_x] boundary vectors int eta_k on the inflow faces
    double* d_ox = nullptr;
    double* d_oy = nullptr;
    double* d_w = nullptr;
    double* d_fold_w = nullptr;
    double* d_wlist = nullptr;    // [nang] per-list weights for rte_sweep
    int* d_fold_rep = nullptr;
    int* d_angles = nullptr;      // [nang] scratch angle list
    int* h_angles = nullptr;      // pinned staging
    int2* d_outcols = nullptr;    // [nang] output columns of the deduplicated sweep items (rte_sweep)
    int2* h_outcols = nullptr;    // pinned staging
    double* h_scalar = nullptr;   // pinned scalars
    // work vectors
    double* phi_star = nullptr;
    double* dphi = nullptr;
    double* tmp = nullptr;
    void* src_w = nullptr;        // [N_x] sweep source in sweep precision
    double* src64 = nullptr;      // [N_x] the same source in FP64 (defect correction)
    void* dpsi_w = nullptr;       // [psi_cap * N_x] defect-correction sweeps
    void* res_w = nullptr;        // [psi_cap * N_x] FP64 residuals stored in the sweep precision
    size_t dpsi_cap_bytes = 0;
    void* psi_w = nullptr;        // [psi_cap * N_x] angular-flux scratch
    size_t psi_cap_bytes = 0;
    double* red = nullptr;        // reduction partials
    int* d_err = nullptr;         // set by a device wait that ran out (sweep hand-offs)
    int wait_limit = 1 << 22;     // polls of a sweep hand-off wait before it gives up (rte_set_wait_limit)
    int inject = 0;               // failure the next solve reports (rte_inject_failure; tests only)
    // DSA (MIP) preconditioned CG
    double* D = nullptr;          // [nc] diffusion coefficient 1/(3 sigma_t)
    double* sig_a = nullptr;      // [nc]
    double* Minv = nullptr;       // [nc*16] inverse diagonal blocks
    double* cg_r = nullptr;
    double* cg_z = nullptr;
    double* cg_p = nullptr;
    double* cg_q = nullptr;
    double* cg_red = nullptr;
    int* cg_iters = nullptr;
    int cg_grid = 0;
    int cg_grid32 = 0;
    int cg_tuned[2] = {0, 0};     // CG grid autotuned (FP64, FP32); a negative grid = one block
    std::map<long long, rte_sweep_config> sweep_cfg;   // sweep launch configurations by kind (rte_sweep.cu)
    void* cg_args_dev = nullptr;  // CG arguments of the block-resident schedule
    void* batch_buf = nullptr;    // batched CG launch arguments (this handle owns a batch)
    size_t batch_cap = 0;
    void* tc_scratch = nullptr;   // partial sums of rte_basis_project
    size_t tc_scratch_cap = 0;
    void* sweep_batch_buf = nullptr;  // batched sweep launch arguments
    size_t sweep_batch_cap = 0;
    rte::MgArgs mg{};                 // DSA two-level preconditioner (mg.L == 0: block Jacobi only)
    rte::MgArgs* mg_dev = nullptr;    // device copy of mg
    double* mg_scratch = nullptr;     // probing scratch [12 N_0]
    float* D32 = nullptr;         // FP32 copies for the FP32 CG
    float* sa32 = nullptr;
    float* Minv32 = nullptr;
    void* cg_w = nullptr;         // [5 N_x] CG work vectors (FP64 or FP32 view)

    rte::LowRankState lr;
    rte::Profiler prof;
    rte_stats last{};
};

namespace rte {

// ---- setup helpers (rte_setup.cu) ----
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);
int upload_materials(rte_handle* h);

// ---- sweeps (rte_sweep.cu) ----
// Sweep n angles (device list d_angles) with source src (stride src_stride per angle, 0 = shared).
// outcols (device, optional): item a writes psi columns outcols[a].x and outcols[a].y (if >= 0);
// n_out = the number of columns written (for the profiler's byte count; -1 = n)
int launch_sweep(rte_handle* h, const int* d_angles, int n, int precision, const void* src,
                 long long src_stride, int add_inflow, int reverse, void* psi, cudaStream_t st,
                 const int* n_dev = nullptr, const int2* outcols = nullptr, int n_out = -1);
int launch_phi_reduce(rte_handle* h, const int* d_angles, const double* d_weight_of_angle,
                      int n, int precision, const void* psi, double* phi, cudaStream_t st);
int launch_source(rte_handle* h, const double* phi, int precision, void* src, cudaStream_t st);
int max_abs_diff(rte_handle* h, const double* a, const double* b, int n, double* host_out, cudaStream_t st);
// the same without the synchronisation: the result lands in h->h_scalar[0] once st has drained
int max_abs_diff_async(rte_handle* h, const double* a, const double* b, int n, cudaStream_t st);
// Read and clear the device wait-timeout flag (synchronises the stream); RTE_ERR_DEP_TIMEOUT if set.
int check_dep_flag(rte_handle* h, cudaStream_t st);
// Sweep with optional FP64 defect correction (FP32 only): psi = sweep(src); when refine,
// dpsi = sweep(b64 (+ g) - L psi).  Consumers add psi + dpsi in FP64.
// Tune the sweep configuration of n-ordinate launches in `precision` (psi written or not) now,
// with scratch buffers, unless one is cached.
int sweep_pretune(rte_handle* h, int precision, int n, int with_psi, cudaStream_t st);
int sweep_refined(rte_handle* h, const int* d_angles, int n, int precision, int refine, const void* src,
                  const double* b64, int add_inflow, int reverse, void* psi, void** dpsi_out, const int* n_dev,
                  cudaStream_t st);
// FP64 defect of FP32 sweeps (psi, stride ndof) into h->res_w (FP32): r = b64 (+ inflow) - L_j psi_j
int launch_defect(rte_handle* h, const int* d_angles, int n, const double* b64, int add_inflow, int reverse,
                  const void* psi, const int* n_dev, cudaStream_t st);
int ensure_refine_scratch(rte_handle* h, int n);
bool batch_supported(rte_handle* const* hs, int nprob, int precision);
int launch_sweep_batch(rte_handle* const* hs, int nprob, const int* const* d_angles, const int* n, int precision,
                       const void* const* src, const long long* src_stride, int add_inflow, int reverse,
                       void* const* psi, cudaStream_t st);
int launch_phi_reduce2(rte_handle* h, const double* d_wlist, int n, int precision, const void* psi,
                       const void* dpsi, double* phi, cudaStream_t st);
int launch_to_double2(rte_handle* h, int n, int precision, const void* psi, const void* dpsi, double* out,
                      cudaStream_t st);

// ---- DSA (rte_dsa.cu) ----
int dsa_prepare(rte_handle* h);
// One kernel per translation unit, whose CUDA library holds all of that unit's kernels.
const void* sweep_kernel_anchor();
const void* dsa_kernel_anchor();
const void* tc_kernel_anchor();
const void* lowrank_kernel_anchor();
// Autotune the handle's CG schedule for a precision now (on its stream), if not done yet.
int dsa_pretune(rte_handle* h, int precision);
int dsa_apply(rte_handle* h, const double* x, double* y, cudaStream_t st);
int dsa_cg(rte_handle* h, const double* rhs, double* x, double tol, int max_iter, int* iters, cudaStream_t st);
// dphi = CG solution of A dphi = sig_s (phi_star - phi); phi = phi_star + dphi
int dsa_correct(rte_handle* h, const rte_opts* o, const double* phi_star, double* phi, int* iters, cudaStream_t st);
// The same for n problems with one batched cooperative CG; synchronises st, iters[i] per problem.
int dsa_correct_batch(rte_handle* const* hs, int n, const rte_opts* o, const double* const* phi_star,
                      double* const* phi, int* iters, cudaStream_t st);

// ---- solvers (rte_solve.cu / rte_lowrank.cu) ----
int solve_full_rank(rte_handle* h, const rte_opts* o, double* phi, rte_stats* st);
// F (optional, DEVICE [ndir][N]): the backward-Euler time source of each distinct direction (the
// previous angular flux over dt); psi_next (optional, DEVICE [nang][N]): receives X C.
int solve_low_rank(rte_handle* h, const rte_opts* o, double* phi, rte_stats* st, const double* F = nullptr,
                   double* psi_next = nullptr);
int ensure_psi_scratch(rte_handle* h, size_t bytes);

#define RTE_PROF_BEGIN(h, cls, st) do { if ((h)->prof.on) (h)->prof.begin((cls), (st)); } while (0)
#define RTE_PROF_END(h, cls, st, by, fl) do { if ((h)->prof.on) (h)->prof.end((cls), (st), (by), (fl)); } while (0)

}  // namespace rte
