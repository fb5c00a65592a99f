// Rank-adaptive low-rank source iteration (Sec. 3.1-3.4, Alg. 1, Alg. 2) on the device.
//
// Inner iteration k of outer iteration n (phi^{(n-1)} fixed, S = Sigma_s phi^{(n-1)} + G):
//   1. sweep the p sampled angles (Eq. sampled-sweep);
//   2. append each snapshot to the basis X by MGS2-A (Alg. 2): two classical projections
//      c += X^T psi, psi -= X (X^T psi), normalisation, then adaptive re-projections while the
//      orthogonality test fails (at most m_max);
//   3. grow the projected operators by their new border (Sec. 3.4): with the upwind DG
//      operators D_x^{+T} = -D_x^-, D_y^{+T} = -D_y^-, so only X^T D_x^- X, X^T D_y^- X and
//      X^T Sigma_t X are kept; the border needs the images D_x^- p, D_x^{-T} p, D_y^- p,
//      D_y^{-T} p, Sigma_t p of the new column p and one pass X^T [..] over the basis;
//   4. Galerkin systems A_j c_j = X^T (S + g_j^bc) (Eq. galerkin-projection) for every
//      unsampled direction are kept factorised, A_j = L_j U_j, and bordered when X grows by
//      one column (u = L^{-1} a, l = U^{-T} b, delta = d - l.u): the symmetric part of A_j is
//      X^T (sym D_j + Sigma_t) X >= sigma_t,min I, so elimination without pivoting is
//      defined; this gives the same c_j as solving each candidate's system anew;
//   5. draw q unsampled candidates (Philox4x32-10 keys, the q smallest (key, index) win),
//      back-substitute their c_j, form X c_j and the residual norms ||S + g_j - (D_j +
//      Sigma_t) X c_j||_2 (Sec. 3.2), select the p largest (ties: smaller index);
//   6. if the largest candidate residual is below eps_res, form C for all angles (columns of
//      R for appended angles, Galerkin solutions for the others), phi^{(n,k)} = X (C w), and
//      stop when ||phi^{(n,k)} - phi_old||_2 <= eps_diff (Sec. 3.3).
// After the inner loop C = U S V^T by one-sided Jacobi, truncated by the tail rule, and
// X U is formed when factors are requested.
//
// +-Omega_z twins share (Omega_x, Omega_y): sweeping one samples both (identical psi), and the
// Galerkin systems are kept once per distinct direction.
#include <cooperative_groups.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <vector>

#include "rte_internal.cuh"
#include "rte_dw.cuh"

namespace cg = cooperative_groups;

namespace rte {

// ---- device integer state -----------------------------------------------------------------
// The whole inner iteration reads its control state from here, so that it can be captured once
// as a CUDA graph and replayed; kernels whose gate is closed return at once.
enum {
    I_R = 0,          // current rank r
    I_NNEW = 1,       // angles to sweep next
    I_STOP = 2,       // inner loop finished
    I_FULL = 3,       // full check requested this iteration
    I_NCAND = 4,      // candidates drawn this iteration
    I_MGSFAIL = 5,
    I_BREAK = 6,
    I_FULLCNT = 7,
    I_SING = 8,       // zero pivot met
    I_APPENDED = 9,   // the current snapshot was appended
    I_MGSDONE = 10,   // adaptive projections finished for the current snapshot
    I_K = 11,         // inner iteration index k
    I_OUTER = 12,     // outer iteration index n
    I_ACTIVE = 13,    // snapshot slot in use
    I_CUR = 14,       // angle of the current snapshot
    I_CURTW = 15,     // its +-Omega_z twin
    I_NEW = 16,       // [64] angles to sweep
    // (80..143 unused: the candidate list lives after the per-angle arrays, cand_arr)
    I_R0 = 144,       // rank at the start of the inner iteration (bordering starts there)
    I_MGSIT = 145,    // adaptive projection round of the current snapshot (graph loop)
    I_CNT_PASS = 146, // completion counters of the kernels that finish their reduction in their
    I_CNT_STEN = 147, // last block (zero between launches)
    I_CNT_FIN = 148,
    I_BCOL = 150,     // [64] column appended by snapshot slot l of this inner iteration, -1 if none
    I_HDR = 256
};
// per-angle arrays after the header: status[nang] (0 unsampled, 1 appended, 2 swept but not
// appended), col_of[nang], then angle_of_col[r_cap], 64 spare, then the candidate list
// [kCandMax] of the current inner iteration
constexpr int kCandMax = 1024;   // candidates per inner iteration (q = every unsampled angle: fully greedy)

enum { G_LIVE = 0, G_SNAP = 1, G_MGS = 2, G_APP = 3, G_FULL = 4, G_ALWAYS = 5 };

// Rank seen by a pass: rsel < 0 -> the current rank; rsel = l >= 0 -> one more than the column that
// snapshot slot l appended (the border work of slot l, which may run after later slots have
// appended), -1 when slot l appended nothing.
__device__ __forceinline__ int rank_sel(const int* st, int rsel) {
    if (rsel < 0) return st[I_R];
    const int col = st[I_BCOL + rsel];
    return col >= 0 ? col + 1 : -1;
}

__device__ __forceinline__ bool gate(const int* st, int mode) {
    if (mode == G_ALWAYS) return true;
    if (st[I_STOP]) return false;
    switch (mode) {
        case G_SNAP: return st[I_ACTIVE] != 0;
        case G_MGS: return st[I_ACTIVE] != 0 && st[I_MGSDONE] == 0;
        case G_APP: return st[I_ACTIVE] != 0 && st[I_APPENDED] != 0;
        case G_FULL: return st[I_FULL] != 0;
        default: return true;
    }
}

// ---- small double state layout (offsets in units of r_cap) ------------------------------
struct SmallLayout {
    int rc;
    static constexpr int Q = kCandMax;
    __host__ __device__ int c() const { return 0; }                     // [rc] accumulated coefficients
    __host__ __device__ int dc() const { return rc; }                   // [rc] projection coefficients
    __host__ __device__ int scal() const { return 2 * rc; }             // [16] scalars
    __host__ __device__ int norms() const { return 2 * rc + 16; }       // [Q] candidate residual norms
    __host__ __device__ int cw() const { return 2 * rc + 16 + Q; }      // [rc]
    __host__ __device__ int border() const { return 3 * rc + 16 + Q; }  // [5 * rc] X^T W
    __host__ __device__ int dots() const { return 8 * rc + 16 + Q; }    // [8]
    __host__ __device__ int ccand() const { return 8 * rc + 32 + Q; }   // [Q * rc]
    __host__ __device__ int total() const { return (8 + Q) * rc + 32 + Q; }
};
enum { S_ALPHA = 0, S_PSINORM = 1, S_TEST = 2, S_DIFF = 3, S_MAXRES = 4 };

struct LRArgs {
    int nx, ny, nc, N, nang, rc, ndir, p, q;
    double hx, hy;
    double ihx, ihy;        // 1 / hx, 1 / hy (formed on the host: no FP64 divisions per thread)
    double g[4];
    const double* ox;
    const double* oy;
    const double* w;
    const int* dir_of;      // [nang] direction of each angle
    const int* dir_rep;     // [ndir] representative angle
    const int* twin;        // [nang] +-Omega_z twin
    const double* sig_t;
    const double* e_side;   // [4 N]
    const double* S;        // [N] FP64 source Sigma_s phi + G
    // backward-Euler time source (Sec. 3.7), or null: F [ndir][N] the previous step's angular flux
    // over dt of each distinct direction; bF [ndir][rc] its products with the basis columns
    const double* F;
    double* bF;
    double* X;
    double* R;
    double* Pxm;
    double* Pym;
    double* T;
    double* bS;
    double* bE;
    double* Lf;             // [ndir][rc][rc] unit lower, column-major
    double* Uf;             // [ndir][rc][rc] upper, row-major
    double* Udinv;          // [ndir][rc] reciprocals of the diagonal of U (no divisions in the solves)
    double* Y;              // [ndir][rc]
    double* Cdir;           // [ndir][rc]
    double* W;              // [5 N]
    double* vcand;          // [q N]
    double* red;            // residual partials [64][nblk]
    double* sm;             // small doubles
    int* st;                // ints
    double* phi_old;
    double* phi_k;
    double* Cfull;          // [nang][rc] (column j of C at j*rc)
    // double-word basis passes (dwb = 1): X2 [rc][N] (hi, lo) of X, S2 [N] of S, sigma_t as
    // hi / lo floats, candidate coefficients [64][rc]; vcand and W then hold double-words
    int dwb;
    float2* X2;
    float* Xt;              // TF32 split of X2's hi for the tensor-core first projection (or null)
    float* Xl;
    float2* S2;
    const float* sig_h;
    const float* sig_l;
    float2* ccand2;
    double eps_mgs, eps_break, eps_res, eps_diff;
    int m_max, mgs_test, max_inner;
    unsigned long long seed;
};

__device__ __forceinline__ int* status_arr(const LRArgs& a) { return a.st + I_HDR; }
__device__ __forceinline__ int* colof_arr(const LRArgs& a) { return a.st + I_HDR + a.nang; }
__device__ __forceinline__ int* angleofcol_arr(const LRArgs& a) { return a.st + I_HDR + 2 * a.nang; }
__device__ __forceinline__ int* cand_arr(const LRArgs& a) { return a.st + I_HDR + 2 * a.nang + a.rc + 64; }
__device__ __forceinline__ double* scal(const LRArgs& a) { return a.sm + SmallLayout{a.rc}.scal(); }

__device__ __forceinline__ double nan_val() { return __longlong_as_double(0x7ff8000000000000ll); }

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// |X(:,1)^T psi_hat| or max_i |X(:,i)^T psi_hat| from dc = X^T v: psi_hat = v (FP64 chain, v
// normalised) or v / alpha (double-word chain, v unnormalised; v = 0 gives 0 as in the FP64 chain)
__device__ __forceinline__ double mgs_test_value(const LRArgs& a) {
    const int r = a.st[I_R];
    const double* dc = a.sm + SmallLayout{a.rc}.dc();
    double t = 0.0;
    if (r > 0) {
        if (a.mgs_test == 0) t = fabs(dc[0]);
        else for (int k = 0; k < r; ++k) t = fmax(t, fabs(dc[k]));
    }
    if (a.dwb) {
        const double alpha = scal(a)[S_ALPHA];
        t = alpha > 0.0 ? t / alpha : 0.0;
    }
    return t;
}

// Append the current snapshot as column r of the basis (or record a breakdown), by one whole block
// once its MGS2-A projections are final: the R column (c, alpha), the angle's status and column,
// the slot's column record, then r + 1.  The column itself is written by copy_col(_dw).
__device__ void append_block(const LRArgs& a, int slot) {
    __shared__ int ok;
    const int r = a.st[I_R];
    const int angle = a.st[I_CUR], twin = a.st[I_CURTW];
    const double* sc = scal(a);
    if (threadIdx.x == 0) {
        const double alpha = sc[S_ALPHA];
        const double psin = sc[S_PSINORM];
        ok = (alpha > a.eps_break * psin) && (r < a.rc) && (alpha == alpha);
        int* status = status_arr(a);
        int* colof = colof_arr(a);
        if (slot >= 0) a.st[I_BCOL + slot] = ok ? r : -1;
        if (ok) {
            status[angle] = 1;
            colof[angle] = r;
            if (twin != angle) { status[twin] = 1; colof[twin] = r; }
            angleofcol_arr(a)[r] = angle;
        } else {
            // not appended: the angle (and its twin) are swept; a direction that already has an
            // R column keeps it (the twin of an appended angle has the same psi)
            if (status[angle] == 0) status[angle] = 2;
            if (twin != angle && status[twin] == 0) status[twin] = 2;
            a.st[I_BREAK] += 1;
        }
    }
    __syncthreads();
    if (!ok) return;
    const double* c = a.sm + SmallLayout{a.rc}.c();
    for (int k = threadIdx.x; k < a.rc; k += blockDim.x)
        a.R[(long long)r * a.rc + k] = k < r ? c[k] : (k == r ? sc[S_ALPHA] : 0.0);
    __syncthreads();
    if (threadIdx.x == 0) {
        a.st[I_R] = r + 1;
        a.st[I_APPENDED] = 1;
    }
}

// ------------------------------------------------------------------ Philox4x32-10
__device__ __forceinline__ unsigned philox_key(unsigned long long seed, unsigned n, unsigned k, unsigned j) {
    unsigned c0 = j, c1 = k, c2 = n, c3 = 0x52544531u;
    unsigned k0 = (unsigned)(seed & 0xffffffffull), k1 = (unsigned)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const unsigned long long p0 = 0xD2511F53ull * (unsigned long long)c0;
        const unsigned long long p1 = 0xCD9E8D57ull * (unsigned long long)c2;
        const unsigned hi0 = (unsigned)(p0 >> 32), lo0 = (unsigned)p0;
        const unsigned hi1 = (unsigned)(p1 >> 32), lo1 = (unsigned)p1;
        const unsigned n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    return c0;
}

// ------------------------------------------------------------------ passes over X (FP64)
// partial[b][v][k] = sum over the rows of row chunk b of X[:,k] V[v]  (k < r, r on the device).
// Grid: (row chunks of kXtRows, groups of 8 columns); warp w of a block takes column 8 y + w, so
// each warp reduction follows kXtRows/32 FMAs per vector.
constexpr int kXtRows = 1024;
__global__ void __launch_bounds__(256) xt_partial(const double* __restrict__ X, int N, const int* __restrict__ st,
                                                   int gm, const double* __restrict__ V, int nv, long long vstride,
                                                   double* __restrict__ part, int rc) {
    pdl_entry();
    extern __shared__ double vs[];
    if (!gate(st, gm)) return;
    const int r = st[I_R];
    if ((int)blockIdx.y * 8 >= r) return;                  // uniform per block
    const int row0 = blockIdx.x * kXtRows;
    const int len = min(kXtRows, N - row0);
    for (int v = 0; v < nv; ++v)
        for (int i = threadIdx.x; i < len; i += blockDim.x) vs[v * kXtRows + i] = V[v * vstride + row0 + i];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int k = blockIdx.y * 8 + wid;
    if (k >= r) return;
    const double* xk = X + (long long)k * N + row0;
    double acc[5] = {0, 0, 0, 0, 0};
    int i = lane;
    for (; i + 96 < len; i += 128) {               // four independent loads in flight per lane
        const double x0 = xk[i], x1 = xk[i + 32], x2 = xk[i + 64], x3 = xk[i + 96];
#pragma unroll
        for (int v = 0; v < 5; ++v)
            if (v < nv) {
                const double* vv = vs + v * kXtRows + i;
                acc[v] = fma(x0, vv[0], fma(x1, vv[32], fma(x2, vv[64], fma(x3, vv[96], acc[v]))));
            }
    }
    for (; i < len; i += 32) {
        const double x = xk[i];
#pragma unroll
        for (int v = 0; v < 5; ++v)
            if (v < nv) acc[v] = fma(x, vs[v * kXtRows + i], acc[v]);
    }
#pragma unroll
    for (int v = 0; v < 5; ++v)
        if (v < nv) {
            const double sv = warp_sum(acc[v]);
            if (lane == 0) part[((long long)blockIdx.x * 5 + v) * rc + k] = sv;
        }
}

// out[v][k] = sum_b partial[b][v][k]: one warp per (v, k)
__global__ void __launch_bounds__(256) xt_final(const double* __restrict__ part, int nblk, const int* __restrict__ st,
                                                 int gm, int nv, int rc, double* __restrict__ out, int rsel = -1,
                                                 int vs = 5) {
    pdl_entry();
    if (!gate(st, gm)) return;
    const int r = rank_sel(st, rsel);
    const int lane = threadIdx.x & 31;
    const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int v = blockIdx.y;
    if (k >= r || v >= nv) return;
    double s = 0.0;
    for (int b = lane; b < nblk; b += 32) s += part[((long long)b * vs + v) * rc + k];
    s = warp_sum(s);
    if (lane == 0) out[v * rc + k] = s;
}

// out[j][i] = sum_k X[k][i] C[j][k] for j0 <= j < min(*njptr, j0 + kXtChunk) (C with leading
// dimension rc); one launch per chunk of kXtChunk columns of C
constexpr int kXtChunk = 64;
__global__ void __launch_bounds__(256) x_times(const double* __restrict__ X, int N, const int* __restrict__ st, int gm,
                                                const double* __restrict__ C, int rc, const int* __restrict__ njptr,
                                                double* __restrict__ out, int j0c) {
    pdl_entry();
    extern __shared__ double cs[];
    if (!gate(st, gm)) return;
    const int r = st[I_R];
    const int nj = min(*njptr - j0c, kXtChunk);
    if (nj <= 0) return;
    C += (long long)j0c * rc;
    out += (long long)j0c * N;
    for (int t = threadIdx.x; t < nj * r; t += blockDim.x) cs[t] = C[(t / r) * rc + (t % r)];
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        for (int j0 = 0; j0 < nj; j0 += 8) {
            double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int k = 0; k < r; ++k) {
                const double x = X[(long long)k * N + i];
#pragma unroll
                for (int jj = 0; jj < 8; ++jj)
                    if (j0 + jj < nj) acc[jj] = fma(x, cs[(j0 + jj) * r + k], acc[jj]);
            }
#pragma unroll
            for (int jj = 0; jj < 8; ++jj)
                if (j0 + jj < nj) out[(long long)(j0 + jj) * N + i] = acc[jj];
        }
    }
}

// ------------------------------------------------------------------ passes over X (double-word FP32)
// The same passes with X, the projected vectors and the coefficients held as double-word FP32
// (rte_dw.cuh): X2[k N + i] = X[k N + i] split into hi + lo (exact, written when the column is
// appended), accumulations by Dot2.  Results about 1e-14 relative to the sums of the absolute
// products, on the FP32 pipe.

// Last-block completion: every block of the launch calls this after writing its partial
// results; it returns true in the one block that finishes last, which then sees all partials
// (read them with __ldcg) and resets the counter for the next launch.
__device__ __forceinline__ bool last_block(int* cnt) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(cnt, 1) == (int)(gridDim.x * gridDim.y) - 1;
    __syncthreads();
    if (s_last) __threadfence();
    return s_last;
}

// sum of n FP64 values (fixed order per thread, then a fixed tree): the whole block, result in
// thread 0
__device__ __forceinline__ double block_sum_strided(const double* p, int n, long long stride) {
    __shared__ double smb[32];
    double s = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) s += __ldcg(p + b * stride);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) smb[threadIdx.x >> 5] = s;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) t += smb[w2];
    __syncthreads();
    return t;
}

// block sum of a double-word value; thread 0 gets the result as FP64
__device__ __forceinline__ double dw_block_sum(DW v) {
    __shared__ float2 smw[32];
    v = dw_warp_sum(v);
    if ((threadIdx.x & 31) == 0) smw[threadIdx.x >> 5] = make_float2(v.h, v.l);
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) t += (double)smw[w2].x + (double)smw[w2].y;
    __syncthreads();
    return t;
}

// partial[b][v][k] = X[chunk b, k]^T V[v][chunk b] at part[((b kXtV) + v) rc + k] (k < r,
// v < nv <= kXtV; V holds nv double-word vectors with stride vstride).  Grid (row chunks of kXtRows,
// groups of 8 columns): warp w of a block takes column 8 y + w over the chunk (Dot2 sums, two
// chains per vector; the arithmetic of each product does not depend on nv).  With npart, the
// blocks of column group 0 also sum V[v]^2 over their chunk into npart[v nblk + b].  The partials
// are added by xt_final / mgs_dots_final / norms_final (one warp per entry).
constexpr int kXtV = 8;
constexpr int kOpenChunks = 32;      // row chunks of snap_open's products with new columns
__global__ void __launch_bounds__(256) xt_dw(const float2* __restrict__ X2, int N, const int* __restrict__ st, int gm,
                                              const float2* __restrict__ V, int nv, long long vstride,
                                              double* __restrict__ part, int rc, double* __restrict__ npart,
                                              int rsel) {
    pdl_entry();
    extern __shared__ float2 vs2[];
    if (!gate(st, gm)) return;                         // uniform over the launch
    const int r = rank_sel(st, rsel);
    if (r < 0) return;
    const bool cols = (int)blockIdx.y * 8 < r;         // uniform per block
    const bool nrm = npart && blockIdx.y == 0;
    if (!cols && !nrm) return;
    const int row0 = blockIdx.x * kXtRows;
    const int len = min(kXtRows, N - row0);
    for (int v = 0; v < nv; ++v)
        for (int i = threadIdx.x; i < len; i += blockDim.x) vs2[v * kXtRows + i] = V[v * vstride + row0 + i];
    __syncthreads();
    if (nrm)
        for (int v = 0; v < nv; ++v) {
            DW acc{0.f, 0.f};
            for (int i = threadIdx.x; i < len; i += blockDim.x) {
                const float2 y = vs2[v * kXtRows + i];
                dw_mac(acc, DW{y.x, y.y}, DW{y.x, y.y});
            }
            const double t = dw_block_sum(dw_norm(acc));
            if (threadIdx.x == 0) npart[(long long)v * gridDim.x + blockIdx.x] = t;
        }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int k = blockIdx.y * 8 + wid;
    if (!cols || k >= r) return;
    const float2* xk = X2 + (long long)k * N + row0;
    DW acc0[kXtV], acc1[kXtV];                      // two Dot2 chains per vector
#pragma unroll
    for (int v = 0; v < kXtV; ++v) acc0[v] = acc1[v] = DW{0.f, 0.f};
    int i = lane;
    for (; i + 96 < len; i += 128) {
        const float2 x0 = xk[i], x1 = xk[i + 32], x2 = xk[i + 64], x3 = xk[i + 96];
#pragma unroll
        for (int v = 0; v < kXtV; ++v)
            if (v < nv) {
                const float2* vv = vs2 + v * kXtRows + i;
                const float2 y0 = vv[0], y1 = vv[32], y2 = vv[64], y3 = vv[96];
                dw_mac(acc0[v], DW{x0.x, x0.y}, DW{y0.x, y0.y});
                dw_mac(acc1[v], DW{x1.x, x1.y}, DW{y1.x, y1.y});
                dw_mac(acc0[v], DW{x2.x, x2.y}, DW{y2.x, y2.y});
                dw_mac(acc1[v], DW{x3.x, x3.y}, DW{y3.x, y3.y});
            }
    }
    for (; i < len; i += 32) {
        const float2 x = xk[i];
#pragma unroll
        for (int v = 0; v < kXtV; ++v)
            if (v < nv) {
                const float2 y = vs2[v * kXtRows + i];
                dw_mac(acc0[v], DW{x.x, x.y}, DW{y.x, y.y});
            }
    }
#pragma unroll
    for (int v = 0; v < kXtV; ++v)
        if (v < nv) {
            const DW sv = dw_warp_sum(dw_add(dw_norm(acc0[v]), dw_norm(acc1[v])));
            if (lane == 0) part[((long long)blockIdx.x * kXtV + v) * rc + k] = dw_to_double(sv);
        }
}

// out[v] = sqrt(sum_b npart[v nblk + b]) for v < nv: one warp per v
__global__ void norms_final(const double* __restrict__ npart, int nblk, int nv, const int* __restrict__ st, int gm,
                            double* __restrict__ out) {
    pdl_entry();
    if (!gate(st, gm)) return;
    const int lane = threadIdx.x & 31, v = threadIdx.x >> 5;
    if (v >= nv) return;
    double s = 0.0;
    for (int b = lane; b < nblk; b += 32) s += npart[(long long)v * nblk + b];
    s = warp_sum(s);
    if (lane == 0) out[v] = sqrt(s);
}

// Opens snapshot slot l of the double-word chain (the state of snap_begin).  The first projection
// needs dc = X^T psi_l: the products with the r0 columns present when the inner iteration started
// come from one pass over X for all slots (dcall, with psn = ||psi_l||); block (b, j) forms the
// partial product over row chunk b with column r0 + j, appended by an earlier slot of this
// iteration, into opart[j nchunk + b] (the first pass adds them up).
__global__ void __launch_bounds__(256) snap_open(LRArgs a, int l, const float2* __restrict__ psi,
                                                 const double* __restrict__ psn, double* __restrict__ opart) {
    pdl_entry();
    const int on = !a.st[I_STOP] && l < a.st[I_NNEW];
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        a.st[I_ACTIVE] = on; a.st[I_MGSDONE] = 0; a.st[I_MGSIT] = 0; a.st[I_APPENDED] = 0;
        if (on) {
            const int ang = a.st[I_NEW + l];
            a.st[I_CUR] = ang;
            a.st[I_CURTW] = a.twin[ang];
            scal(a)[S_PSINORM] = psn[l];
        }
    }
    if (!on) return;
    const int k = a.st[I_R0] + blockIdx.y;
    if (k >= a.st[I_R]) return;                      // uniform per block
    const int chunk = (a.N + gridDim.x - 1) / gridDim.x;
    const int i0 = blockIdx.x * chunk, i1 = min(a.N, i0 + chunk);
    const float2* xk = a.X2 + (long long)k * a.N;
    DW acc0{0.f, 0.f}, acc1{0.f, 0.f};
    int i = i0 + threadIdx.x;
    for (; i + (int)blockDim.x < i1; i += 2 * blockDim.x) {
        const float2 x0 = xk[i], x1 = xk[i + blockDim.x], y0 = psi[i], y1 = psi[i + blockDim.x];
        dw_mac(acc0, DW{x0.x, x0.y}, DW{y0.x, y0.y});
        dw_mac(acc1, DW{x1.x, x1.y}, DW{y1.x, y1.y});
    }
    if (i < i1) {
        const float2 x0 = xk[i], y0 = psi[i];
        dw_mac(acc0, DW{x0.x, x0.y}, DW{y0.x, y0.y});
    }
    const double t = dw_block_sum(dw_add(dw_norm(acc0), dw_norm(acc1)));
    if (threadIdx.x == 0) opart[(long long)blockIdx.y * gridDim.x + blockIdx.x] = t;
}

// One projection pass of Alg. 2 on the double-word snapshot, without normalisation (the
// double-word chain keeps the projected vector v unnormalised and carries alpha = ||v||):
//   c = (first ? 0 : c) + dc;  vout = vin - X dc;  with alpha_out, alpha_out = ||vout|| (last block)
__global__ void __launch_bounds__(256) mgs_pass_dw(LRArgs a, int gm, int first, const float2* vin,
                                                    float2* vout, double* __restrict__ part, int* cnt,
                                                    double* alpha_out) {
    pdl_entry();
    extern __shared__ float2 cs2[];
    if (!gate(a.st, gm)) return;
    const int r = a.st[I_R];
    const double* dc = a.sm + SmallLayout{a.rc}.dc();
    double* c = a.sm + SmallLayout{a.rc}.c();
    for (int k = threadIdx.x; k < r; k += blockDim.x) {
        const double d = dc[k];
        const DW dd = dw_of(d);
        cs2[k] = make_float2(dd.h, dd.l);
        if (blockIdx.x == 0) c[k] = (first ? 0.0 : c[k]) + d;
    }
    __syncthreads();
    const float2* X2 = a.X2;
    DW nrm{0.f, 0.f};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += gridDim.x * blockDim.x) {
        DW a0{0.f, 0.f}, a1{0.f, 0.f};
        int k = 0;
        for (; k + 1 < r; k += 2) {
            const float2 x0 = X2[(long long)k * a.N + i], x1 = X2[(long long)(k + 1) * a.N + i];
            const float2 c0 = cs2[k], c1 = cs2[k + 1];
            dw_mac(a0, DW{x0.x, x0.y}, DW{c0.x, c0.y});
            dw_mac(a1, DW{x1.x, x1.y}, DW{c1.x, c1.y});
        }
        if (k < r) {
            const float2 x0 = X2[(long long)k * a.N + i];
            const float2 c0 = cs2[k];
            dw_mac(a0, DW{x0.x, x0.y}, DW{c0.x, c0.y});
        }
        const DW nv = dw_add(dw_load(vin + i), dw_neg(dw_add(dw_norm(a0), dw_norm(a1))));
        dw_store(vout + i, nv);
        dw_mac(nrm, nv, nv);
    }
    if (!alpha_out) return;
    const double t = dw_block_sum(dw_norm(nrm));
    if (threadIdx.x == 0) part[blockIdx.x * 8] = t;
    if (!last_block(cnt)) return;
    const double s = block_sum_strided(part, gridDim.x, 8);
    if (threadIdx.x == 0) {
        *alpha_out = sqrt(s);
        *cnt = 0;
    }
}

// A projection pass fused with the inner products that follow it (double-word chain):
//   c = (first ? 0 : c) + dc;  vout = vin - X dc;  then per block the partial sums of X^T vout and
//   of ||vout||^2 (part[(b kXtV) rc + k], npart[b]; mgs_dots_final adds them in block order).
// A block of NW warps takes rows_per_block rows in 32-row groups (lane = row); warp w takes the
// columns k = w + NW j (j < KPW): the pass phase reads each X entry of the group from memory once
// (KPW independent loads per lane), the warps' partial sums meet in shared memory, and the product
// phase reads the same entries again from L1.  r <= NW KPW.
// With dcall (the first pass of a slot), dc is not read: its entries below r0 are dcall[k] and the
// others the sums of snap_open's chunk partials opart[(k - r0) nchunk + b] (one warp each).
template <int KPW, int NW>
__global__ void __launch_bounds__(32 * NW) mgs_pass_xt_dw(LRArgs a, int gm, int first, const float2* vin, float2* vout,
                                                       double* __restrict__ part, double* __restrict__ npart,
                                                       int rows_per_block, const double* __restrict__ dcall,
                                                       const double* __restrict__ opart, int nchunk) {
    pdl_entry();
    extern __shared__ float2 cs2[];          // [rc] the coefficients dc as double-words
    __shared__ float2 ps[2][NW][32];         // partial pass sums of the NW warps, double-buffered
    if (!gate(a.st, gm)) return;
    const int r = a.st[I_R];
    const double* dc = a.sm + SmallLayout{a.rc}.dc();
    double* c = a.sm + SmallLayout{a.rc}.c();
    const int r_lo = dcall ? min(r, a.st[I_R0]) : r;
    for (int k = threadIdx.x; k < r_lo; k += blockDim.x) {
        const double d = dcall ? dcall[k] : dc[k];
        const DW dd = dw_of(d);
        cs2[k] = make_float2(dd.h, dd.l);
        if (blockIdx.x == 0) c[k] = (first ? 0.0 : c[k]) + d;
    }
    if (dcall) {
        const int lane_ = threadIdx.x & 31, w_ = threadIdx.x >> 5;
        for (int k = r_lo + w_; k < r; k += NW) {
            double d = 0.0;
            for (int b = lane_; b < nchunk; b += 32) d += opart[(long long)(k - r_lo) * nchunk + b];
            d = warp_sum(d);
            if (lane_ == 0) {
                const DW dd = dw_of(d);
                cs2[k] = make_float2(dd.h, dd.l);
                if (blockIdx.x == 0) c[k] = (first ? 0.0 : c[k]) + d;
            }
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long N = a.N;
    const float2* X2 = a.X2;
    DW acc[KPW];
#pragma unroll
    for (int j = 0; j < KPW; ++j) acc[j] = DW{0.f, 0.f};
    DW nrm{0.f, 0.f};
    const int row_begin = blockIdx.x * rows_per_block;
    const int row_end = min(a.N, row_begin + rows_per_block);
    int buf = 0;
    for (int g0 = row_begin; g0 < row_end; g0 += 32, buf ^= 1) {
        const int i = g0 + lane;
        const bool ok = i < row_end;
        const DW vi = ok ? dw_load(vin + i) : DW{0.f, 0.f};     // read before any warp writes vout
        DW s0{0.f, 0.f}, s1{0.f, 0.f};
        if (ok) {
#pragma unroll
            for (int j = 0; j < KPW; j += 2) {
                const int k0 = w + NW * j, k1 = k0 + NW;
                if (k0 < r) {
                    const float2 x = X2[k0 * N + i], cc = cs2[k0];
                    dw_mac(s0, DW{x.x, x.y}, DW{cc.x, cc.y});
                }
                if (k1 < r) {
                    const float2 x = X2[k1 * N + i], cc = cs2[k1];
                    dw_mac(s1, DW{x.x, x.y}, DW{cc.x, cc.y});
                }
            }
        }
        const DW sw = dw_add(dw_norm(s0), dw_norm(s1));
        ps[buf][w][lane] = make_float2(sw.h, sw.l);
        __syncthreads();
        DW t{ps[buf][0][lane].x, ps[buf][0][lane].y};
#pragma unroll
        for (int u = 1; u < NW; ++u) t = dw_add(t, DW{ps[buf][u][lane].x, ps[buf][u][lane].y});
        const DW vn = ok ? dw_add(vi, dw_neg(t)) : DW{0.f, 0.f};
        if (w == 0) {
            if (ok) dw_store(vout + i, vn);
            dw_mac(nrm, vn, vn);
        }
        if (ok) {
#pragma unroll
            for (int j = 0; j < KPW; ++j) {
                const int k = w + NW * j;
                if (k < r) {
                    const float2 x = X2[k * N + i];
                    dw_mac(acc[j], DW{x.x, x.y}, vn);
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < KPW; ++j) {
        const int k = w + NW * j;
        if (k >= r) break;
        const DW sv = dw_warp_sum(dw_norm(acc[j]));
        if (lane == 0) part[(long long)blockIdx.x * kXtV * a.rc + k] = dw_to_double(sv);
    }
    if (w == 0) {
        const DW sv = dw_warp_sum(dw_norm(nrm));
        if (lane == 0) npart[blockIdx.x] = dw_to_double(sv);
    }
}

// dc[k] = sum_b part[(b kXtV) rc + k] (one warp per k, blocks 0 .. (rc+7)/8 - 1) and, in the last
// block, alpha_out = sqrt(sum_b npart[b]) when asked
__global__ void __launch_bounds__(256) mgs_dots_final(const double* __restrict__ part, const double* __restrict__ npart,
                                                      int nblk, int rc, const int* __restrict__ st, int gm,
                                                      double* __restrict__ dc, double* alpha_out) {
    pdl_entry();
    if (!gate(st, gm)) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (blockIdx.x + 1 < gridDim.x) {
        const int k = blockIdx.x * 8 + w;
        if (k >= st[I_R]) return;
        double s = 0.0;
        for (int b = lane; b < nblk; b += 32) s += part[(long long)b * kXtV * rc + k];
        s = warp_sum(s);
        if (lane == 0) dc[k] = s;
    } else if (alpha_out && w == 0) {
        double s = 0.0;
        for (int b = lane; b < nblk; b += 32) s += npart[b];
        s = warp_sum(s);
        if (lane == 0) *alpha_out = sqrt(s);
    }
}

// mgs_dots_final followed, in the block that finishes last, by the orthogonality test of Alg. 2 on
// the new dc and alpha (as mgs_test_cond): the kernel that ends a projection pass of the captured
// graph also decides whether the conditional re-projection loop runs (again), so the loop needs
// no separate opening and test launches.  When the loop ends, the same block appends the snapshot
// (append_block, slot `slot`).  The handle is set even when the gate is closed.
__global__ void __launch_bounds__(256) mgs_final_test(LRArgs a, const double* __restrict__ part,
                                                      const double* __restrict__ npart, int nblk, int gm,
                                                      int* cnt, cudaGraphConditionalHandle hc, int slot) {
    pdl_entry();
    __shared__ int done;
    if (!gate(a.st, gm)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(hc, 0u);
        return;
    }
    const int rc = a.rc;
    double* dc = a.sm + SmallLayout{rc}.dc();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (blockIdx.x + 1 < gridDim.x) {
        const int k = blockIdx.x * 8 + w;
        if (k < a.st[I_R]) {
            double s = 0.0;
            for (int b = lane; b < nblk; b += 32) s += part[(long long)b * kXtV * rc + k];
            s = warp_sum(s);
            if (lane == 0) dc[k] = s;
        }
    } else if (w == 0) {
        double s = 0.0;
        for (int b = lane; b < nblk; b += 32) s += npart[b];
        s = warp_sum(s);
        if (lane == 0) scal(a)[S_ALPHA] = sqrt(s);
    }
    if (!last_block(cnt)) return;
    if (threadIdx.x == 0) {
        const double t = mgs_test_value(a);
        scal(a)[S_TEST] = t;
        const int m = a.st[I_MGSIT]++;
        if (t <= a.eps_mgs) {
            a.st[I_MGSDONE] = 1;
        } else if (m >= a.m_max) {
            a.st[I_MGSFAIL] += 1;
            a.st[I_MGSDONE] = 1;
        }
        done = a.st[I_MGSDONE];
        cudaGraphSetConditional(hc, done ? 0u : 1u);
        *cnt = 0;
    }
    __syncthreads();
    if (done) append_block(a, slot);
}

// out[j][i] = sum_k X[k][i] C[j][k] for j < nj (double-word C2 with leading dimension rc),
// written as double-word.  blockIdx.y takes the candidates j0 = kXtJ y .. j0 + kXtJ - 1 (one thread
// per row and candidate group, so the grid has rows x groups threads).
constexpr int kXtJ = 16;
__global__ void __launch_bounds__(256) x_times_dw(const float2* __restrict__ X2, int N, const int* __restrict__ st,
                                                   int gm, const float2* __restrict__ C2, int rc,
                                                   const int* __restrict__ njptr, float2* __restrict__ out) {
    pdl_entry();
    extern __shared__ float2 cs2[];                   // [k][jj] of this group: kXtJ rc double-words
    if (!gate(st, gm)) return;
    const int r = st[I_R];
    const int j0 = blockIdx.y * kXtJ;
    const int nj = min(*njptr - j0, kXtJ);
    if (nj <= 0) return;                              // uniform per block
    for (int t = threadIdx.x; t < nj * r; t += blockDim.x) {
        const int jj = t / r, k = t % r;
        cs2[k * kXtJ + jj] = C2[(long long)(j0 + jj) * rc + k];
    }
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        DW acc[kXtJ];
#pragma unroll
        for (int jj = 0; jj < kXtJ; ++jj) acc[jj] = DW{0.f, 0.f};
        for (int k = 0; k < r; ++k) {
            const float2 x = X2[(long long)k * N + i];
            const float2* ck = cs2 + k * kXtJ;
#pragma unroll
            for (int jj = 0; jj < kXtJ; ++jj)
                if (jj < nj) {
                    const float2 cc = ck[jj];
                    dw_mac(acc[jj], DW{x.x, x.y}, DW{cc.x, cc.y});
                }
        }
#pragma unroll
        for (int jj = 0; jj < kXtJ; ++jj)
            if (jj < nj) dw_store(out + (long long)(j0 + jj) * N + i, dw_norm(acc[jj]));
    }
}

// snapshot slots as double-word: psi + dpsi (FP32 sweeps, exact by TwoSum) or the split of the
// FP64 psi (FP64 sweeps); the count of active sweeps is on the device
template <typename T>
__global__ void to_dw_snap(int N, const int* __restrict__ nptr, const T* psi, const T* dpsi, float2* out,
                           float* out_t, float* out_l) {
    pdl_entry();
    const long long n = (long long)(*nptr) * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        DW d;
        if constexpr (sizeof(T) == 4) d = dpsi ? dw_two_sum((float)psi[i], (float)dpsi[i]) : DW{(float)psi[i], 0.f};
        else d = dw_of((double)psi[i]);
        dw_store(out + i, d);
        if (out_t) {                                 // TF32 split of the high part
            const float t = __uint_as_float(__float_as_uint(d.h) & 0xFFFFE000u);
            out_t[i] = t;
            out_l[i] = __fsub_rn(d.h, t);
        }
    }
}

// hi/lo split of an FP64 vector
__global__ void split_dw_g(int n, const double* __restrict__ src, float2* __restrict__ dst) {
    pdl_entry();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dw_store(dst + i, dw_of(src[i]));
}

// part[b*8] = sum over block b of x[i]^2
__global__ void __launch_bounds__(256) sumsq_partial(int n, const double* __restrict__ x, double* __restrict__ part,
                                                      const int* __restrict__ st, int gm) {
    pdl_entry();
    if (!gate(st, gm)) return;
    __shared__ double sm[32];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) acc = fma(x[i], x[i], acc);
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) t += sm[w2];
        part[blockIdx.x * 8] = t;
    }
}

// out[t] = sum_b part[b*8 + t] (t < nsum), square-rooted when take_sqrt; one warp per t
__global__ void finalize_sums(const double* __restrict__ part, int nblk, int nsum, const int* __restrict__ st, int gm,
                              double* __restrict__ out, int take_sqrt) {
    pdl_entry();
    if (!gate(st, gm)) return;
    const int lane = threadIdx.x & 31, t = threadIdx.x >> 5;
    if (t >= nsum) return;
    double s = 0.0;
    for (int b = lane; b < nblk; b += 32) s += part[b * 8 + t];
    s = warp_sum(s);
    if (lane == 0) out[t] = take_sqrt ? sqrt(s) : s;
}

__global__ void copy_vec_g(int n, const double* __restrict__ src, double* __restrict__ dst, const int* __restrict__ st,
                           int gm) {
    pdl_entry();
    if (st && !gate(st, gm)) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[i];
}

// snapshot dst = psi + dpsi (FP64) for the active sweeps (count on the device)
template <typename T>
__global__ void to_double2_g(int N, const int* __restrict__ nptr, const T* __restrict__ psi, const T* __restrict__ dpsi,
                             double* __restrict__ out) {
    pdl_entry();
    const long long n = (long long)(*nptr) * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (double)psi[i] + (dpsi ? (double)dpsi[i] : 0.0);
}

// ------------------------------------------------------------------ MGS2-A (Alg. 2) control
__global__ void snap_begin(LRArgs a, int l) {
    pdl_entry();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int on = !a.st[I_STOP] && l < a.st[I_NNEW];
    a.st[I_ACTIVE] = on;
    a.st[I_MGSDONE] = 0;
    a.st[I_MGSIT] = 0;
    a.st[I_APPENDED] = 0;
    if (on) {
        const int ang = a.st[I_NEW + l];
        a.st[I_CUR] = ang;
        a.st[I_CURTW] = a.twin[ang];
    }
}

// One projection pass of Alg. 2 on the current snapshot v, fused:
//   d = s * dc (s = alpha for an adaptive pass, 1 otherwise);  c = (first ? 0 : c) + d;
//   v = s * v - X d;   part[b*8] = partial sums of v^2 (for the next norm)
__global__ void __launch_bounds__(256) mgs_pass(LRArgs a, int gm, int first, int scale_alpha, double* __restrict__ v,
                                                 double* __restrict__ part) {
    pdl_entry();
    extern __shared__ double cs[];
    if (!gate(a.st, gm)) return;
    const int r = a.st[I_R];
    const double sc_ = scale_alpha ? scal(a)[S_ALPHA] : 1.0;
    const double* dc = a.sm + SmallLayout{a.rc}.dc();
    double* c = a.sm + SmallLayout{a.rc}.c();
    for (int k = threadIdx.x; k < r; k += blockDim.x) {
        const double d = sc_ * dc[k];
        cs[k] = d;
        if (blockIdx.x == 0) c[k] = (first ? 0.0 : c[k]) + d;
    }
    __syncthreads();
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += gridDim.x * blockDim.x) {
        double s0 = sc_ * v[i], s1 = 0.0;
        int k = 0;
        for (; k + 1 < r; k += 2) {
            s0 = fma(-a.X[(long long)k * a.N + i], cs[k], s0);
            s1 = fma(-a.X[(long long)(k + 1) * a.N + i], cs[k + 1], s1);
        }
        if (k < r) s0 = fma(-a.X[(long long)k * a.N + i], cs[k], s0);
        const double nv = s0 + s1;
        v[i] = nv;
        acc = fma(nv, nv, acc);
    }
    acc = warp_sum(acc);
    __shared__ double sm2[32];
    if ((threadIdx.x & 31) == 0) sm2[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) t += sm2[w2];
        part[blockIdx.x * 8] = t;
    }
}

// psi /= alpha (alpha = ||psi|| finalised into scal[S_ALPHA])
__global__ void mgs_normalise(LRArgs a, int gm, double* v) {
    pdl_entry();
    if (!gate(a.st, gm)) return;
    const double alpha = scal(a)[S_ALPHA];
    if (alpha > 0.0) {
        const double inv = 1.0 / alpha;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += gridDim.x * blockDim.x) v[i] *= inv;
    }
}

// orthogonality test of Alg. 2: |X(:,1)^T psi| (mgs_test 0) or max_i |X(:,i)^T psi| (1), from
// the coefficients dc = X^T psi just computed; sets I_MGSDONE when it holds; on the final call
// a failed test is counted.
__global__ void mgs_test_kernel(LRArgs a, int final_check) {
    pdl_entry();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (!gate(a.st, G_MGS)) return;
    const double t = mgs_test_value(a);
    scal(a)[S_TEST] = t;
    if (!final_check) {
        if (t <= a.eps_mgs) a.st[I_MGSDONE] = 1;
    } else if (t > a.eps_mgs) {
        a.st[I_MGSFAIL] += 1;
    }
}

// The adaptive projections as a device-controlled loop of a CUDA graph (a conditional WHILE
// node): mgs_loop_begin opens it for an active snapshot, and mgs_test_cond ends it once the
// orthogonality test holds or after the m_max-th re-projection (counting a failure then), so
// no gated no-op launches are left in the graph.
__global__ void mgs_loop_begin(LRArgs a, cudaGraphConditionalHandle hc) {
    pdl_entry();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    cudaGraphSetConditional(hc, gate(a.st, G_MGS) ? 1u : 0u);
}

__global__ void mgs_test_cond(LRArgs a, cudaGraphConditionalHandle hc) {
    pdl_entry();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double t = mgs_test_value(a);
    scal(a)[S_TEST] = t;
    const int m = a.st[I_MGSIT]++;
    if (t <= a.eps_mgs) {
        a.st[I_MGSDONE] = 1;
    } else if (m >= a.m_max) {
        a.st[I_MGSFAIL] += 1;
        a.st[I_MGSDONE] = 1;                 // leave the loop (the re-projection below is gated off)
    }
    cudaGraphSetConditional(hc, a.st[I_MGSDONE] ? 0u : 1u);
}

// Append the normalised snapshot (or record a breakdown).  One block.
__global__ void mgs_append(LRArgs a, const double* v, int slot) {
    pdl_entry();
    if (!gate(a.st, G_SNAP)) return;
    append_block(a, slot);
}

__global__ void copy_col(LRArgs a, const double* v) {
    pdl_entry();
    if (!gate(a.st, G_APP)) return;
    double* xc = a.X + (long long)(a.st[I_R] - 1) * a.N;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += gridDim.x * blockDim.x) xc[i] = v[i];
}

// the appended column x = v / alpha from the unnormalised double-word snapshot: X2 takes x as a
// double-word, X its exact FP64 value (hi + lo)
__global__ void copy_col_dw(LRArgs a, const float2* v) {
    pdl_entry();
    __shared__ float2 inv_s;
    if (!gate(a.st, G_APP)) return;                 // appended: alpha > 0
    if (threadIdx.x == 0) {
        const DW iv = dw_of(1.0 / scal(a)[S_ALPHA]);
        inv_s = make_float2(iv.h, iv.l);
    }
    __syncthreads();
    const DW inv{inv_s.x, inv_s.y};
    const long long off = (long long)(a.st[I_R] - 1) * a.N;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += gridDim.x * blockDim.x) {
        const DW x = dw_mul(dw_load(v + i), inv);
        a.X2[off + i] = make_float2(x.h, x.l);
        a.X[off + i] = (double)x.h + (double)x.l;
        if (a.Xt) {
            const float t = __uint_as_float(__float_as_uint(x.h) & 0xFFFFE000u);   // TF32 high part
            a.Xt[off + i] = t;
            a.Xl[off + i] = __fsub_rn(x.h, t);
        }
    }
}

// ------------------------------------------------------------------ projected-operator border
// W = [D_x^- p, D_x^{-T} p, D_y^- p, D_y^{-T} p, Sigma_t p] for p = X[:, r-1] (FP64 chain)
__global__ void __launch_bounds__(256) border_stencil(LRArgs a, int gm, int rsel) {
    pdl_entry();
    if (!gate(a.st, gm)) return;
    const int r = rank_sel(a.st, rsel);
    if (r < 1) return;
    const double* p = a.X + (long long)(r - 1) * a.N;
    const double s3 = 1.7320508075688772935;
    const double ihx = a.ihx, ihy = a.ihy;
    double* W0 = a.W;
    double* W1 = a.W + a.N;
    double* W2 = a.W + 2 * (long long)a.N;
    double* W3 = a.W + 3 * (long long)a.N;
    double* W4 = a.W + 4 * (long long)a.N;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.nc; c += gridDim.x * blockDim.x) {
        const int ix = c % a.nx, iy = c / a.nx;
        const double p0 = p[4 * c], p1 = p[4 * c + 1], p2 = p[4 * c + 2], p3 = p[4 * c + 3];
        // x direction, modes j = 0 (p0, p1) and j = 1 (p2, p3); K = [[1, s3], [-s3, 3]]
        double tL0 = 0, tL1 = 0, lR0 = 0, lR1 = 0;
        if (ix > 0) { const double* q = p + 4 * (c - 1); tL0 = q[0] + s3 * q[1]; tL1 = q[2] + s3 * q[3]; }
        if (ix + 1 < a.nx) { const double* q = p + 4 * (c + 1); lR0 = q[0] - s3 * q[1]; lR1 = q[2] - s3 * q[3]; }
        // D_x^- p = (1/hx) [K p - l (rho . p_left)], l = (1, -s3)
        W0[4 * c + 0] = ihx * (p0 + s3 * p1 - tL0);
        W0[4 * c + 1] = ihx * (-s3 * p0 + 3 * p1 + s3 * tL0);
        W0[4 * c + 2] = ihx * (p2 + s3 * p3 - tL1);
        W0[4 * c + 3] = ihx * (-s3 * p2 + 3 * p3 + s3 * tL1);
        // D_x^{-T} p = (1/hx) [K^T p - rho (l . p_right)], rho = (1, s3)
        W1[4 * c + 0] = ihx * (p0 - s3 * p1 - lR0);
        W1[4 * c + 1] = ihx * (s3 * p0 + 3 * p1 - s3 * lR0);
        W1[4 * c + 2] = ihx * (p2 - s3 * p3 - lR1);
        W1[4 * c + 3] = ihx * (s3 * p2 + 3 * p3 - s3 * lR1);
        // y direction, modes i = 0 (p0, p2) and i = 1 (p1, p3)
        double tB0 = 0, tB1 = 0, lT0 = 0, lT1 = 0;
        if (iy > 0) { const double* q = p + 4 * (c - a.nx); tB0 = q[0] + s3 * q[2]; tB1 = q[1] + s3 * q[3]; }
        if (iy + 1 < a.ny) { const double* q = p + 4 * (c + a.nx); lT0 = q[0] - s3 * q[2]; lT1 = q[1] - s3 * q[3]; }
        W2[4 * c + 0] = ihy * (p0 + s3 * p2 - tB0);
        W2[4 * c + 2] = ihy * (-s3 * p0 + 3 * p2 + s3 * tB0);
        W2[4 * c + 1] = ihy * (p1 + s3 * p3 - tB1);
        W2[4 * c + 3] = ihy * (-s3 * p1 + 3 * p3 + s3 * tB1);
        W3[4 * c + 0] = ihy * (p0 - s3 * p2 - lT0);
        W3[4 * c + 2] = ihy * (s3 * p0 + 3 * p2 - s3 * lT0);
        W3[4 * c + 1] = ihy * (p1 - s3 * p3 - lT1);
        W3[4 * c + 3] = ihy * (s3 * p1 + 3 * p3 - s3 * lT1);
        const double sg = a.sig_t[c];
        W4[4 * c + 0] = sg * p0;
        W4[4 * c + 1] = sg * p1;
        W4[4 * c + 2] = sg * p2;
        W4[4 * c + 3] = sg * p3;
    }
}

// border_stencil of the double-word chain: W (double-words, in the W buffer) from the double-word
// column p = X2[:, col] of slot l, in double-word arithmetic on the FP32 pipe.  With S = +sqrt3
// (upwind neighbour below in x or y, D^-) or -sqrt3 (neighbour above, D^{-T}) and the neighbour
// trace t = q0 + S q1 (x: modes (0,1), (2,3); y: modes (0,2), (1,3)), each mode pair (a0, a1) gives
//   h (a0 + S a1 - t),  h (3 a1 + S (t - a0))        (h = 1/hx or 1/hy)
// which is the FP64 kernel's formulas rearranged.  blockIdx.y = v takes the image W_v of its cells
// (five threads per cell); the v = 4 blocks (Sigma_t p) also form the dots of p with S and the
// inflow side vectors (S2, e_side2 double-words), finished by the last block into the dots slots.
__global__ void __launch_bounds__(64) border_stencil_dw(LRArgs a, int rsel, const float2* __restrict__ e2,
                                                        double* __restrict__ dpart, int* cnt) {
    pdl_entry();
    __shared__ float2 kc[3];
    if (!gate(a.st, G_LIVE)) return;
    const int r = rank_sel(a.st, rsel);
    if (r < 1) return;
    if (threadIdx.x == 0) {
        const DW d0 = dw_of(1.7320508075688772935), d1 = dw_of(a.ihx), d2 = dw_of(a.ihy);
        kc[0] = make_float2(d0.h, d0.l); kc[1] = make_float2(d1.h, d1.l); kc[2] = make_float2(d2.h, d2.l);
    }
    __syncthreads();
    const int v = blockIdx.y;
    const DW s3{kc[0].x, kc[0].y}, ms3{-kc[0].x, -kc[0].y};
    const DW h = v < 2 ? DW{kc[1].x, kc[1].y} : DW{kc[2].x, kc[2].y};
    const DW S = (v == 0 || v == 2) ? s3 : ms3;
    const long long N = a.N;
    const float2* p = a.X2 + (long long)(r - 1) * N;
    float2* Wv = reinterpret_cast<float2*>(a.W) + v * N;
    auto lo = [](DW a0, DW a1, DW t, DW S_) { return dw_add(dw_add(a0, dw_mul(S_, a1)), dw_neg(t)); };
    auto hi = [](DW a0, DW a1, DW t, DW S_) { return dw_add(dw_mul_f(a1, 3.f), dw_mul(S_, dw_add(t, dw_neg(a0)))); };
    auto tr = [](const float2* q, int m0, int m1, DW S_) { return dw_add(dw_load(q + m0), dw_mul(S_, dw_load(q + m1))); };
    DW dacc[5];
#pragma unroll
    for (int t = 0; t < 5; ++t) dacc[t] = DW{0.f, 0.f};
    const DW z{0.f, 0.f};
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.nc; c += gridDim.x * blockDim.x) {
        const int ix = c % a.nx, iy = c / a.nx;
        const long long b4 = 4 * (long long)c;
        const DW p0 = dw_load(p + b4), p1 = dw_load(p + b4 + 1), p2 = dw_load(p + b4 + 2), p3 = dw_load(p + b4 + 3);
        if (v < 2) {                                   // x images: modes (0, 1), (2, 3)
            const bool has = v == 0 ? ix > 0 : ix + 1 < a.nx;
            const float2* q = p + b4 + (v == 0 ? -4 : 4);
            const DW t0 = has ? tr(q, 0, 1, S) : z, t1 = has ? tr(q, 2, 3, S) : z;
            dw_store(Wv + b4 + 0, dw_mul(h, lo(p0, p1, t0, S)));
            dw_store(Wv + b4 + 1, dw_mul(h, hi(p0, p1, t0, S)));
            dw_store(Wv + b4 + 2, dw_mul(h, lo(p2, p3, t1, S)));
            dw_store(Wv + b4 + 3, dw_mul(h, hi(p2, p3, t1, S)));
        } else if (v < 4) {                            // y images: modes (0, 2), (1, 3)
            const bool has = v == 2 ? iy > 0 : iy + 1 < a.ny;
            const float2* q = p + b4 + (v == 2 ? -4 * (long long)a.nx : 4 * (long long)a.nx);
            const DW t0 = has ? tr(q, 0, 2, S) : z, t1 = has ? tr(q, 1, 3, S) : z;
            dw_store(Wv + b4 + 0, dw_mul(h, lo(p0, p2, t0, S)));
            dw_store(Wv + b4 + 2, dw_mul(h, hi(p0, p2, t0, S)));
            dw_store(Wv + b4 + 1, dw_mul(h, lo(p1, p3, t1, S)));
            dw_store(Wv + b4 + 3, dw_mul(h, hi(p1, p3, t1, S)));
        } else {                                       // Sigma_t p and the dots
            const DW sg{a.sig_h[c], a.sig_l[c]};
            const DW pv[4] = {p0, p1, p2, p3};
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                dw_store(Wv + b4 + m, dw_mul(sg, pv[m]));
                dw_mac(dacc[0], pv[m], dw_load(a.S2 + b4 + m));
#pragma unroll
                for (int t = 0; t < 4; ++t) dw_mac(dacc[1 + t], pv[m], dw_load(e2 + t * N + b4 + m));
            }
        }
    }
    if (v == 4) {
        __shared__ float2 sm5[2][5];                  // blockDim = 64: two warps
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int t = 0; t < 5; ++t) {
            const DW d = dw_warp_sum(dw_norm(dacc[t]));
            if (lane == 0) sm5[wid][t] = make_float2(d.h, d.l);
        }
        __syncthreads();
        if (threadIdx.x < 5)
            dpart[blockIdx.x * 8 + threadIdx.x] = (double)sm5[0][threadIdx.x].x + (double)sm5[0][threadIdx.x].y +
                                                  ((double)sm5[1][threadIdx.x].x + (double)sm5[1][threadIdx.x].y);
    }
    if (!last_block(cnt)) return;
    double* dots = a.sm + SmallLayout{a.rc}.dots();
#pragma unroll
    for (int t = 0; t < 5; ++t) {
        const double d = block_sum_strided(dpart + t, gridDim.x, 8);
        if (threadIdx.x == 0) dots[t] = d;
    }
    if (threadIdx.x == 0) *cnt = 0;
}

// part[b*8 + t] = partial dots of the newest basis column with S (t = 0) and e_side (t = 1..4)
__global__ void __launch_bounds__(256) newcol_dots_partial(LRArgs a, double* __restrict__ part) {
    pdl_entry();
    if (!gate(a.st, G_APP)) return;
    __shared__ double sm[32][5];
    const double* p = a.X + (long long)(a.st[I_R] - 1) * a.N;
    double acc[5] = {0, 0, 0, 0, 0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += gridDim.x * blockDim.x) {
        const double x = p[i];
        acc[0] = fma(x, a.S[i], acc[0]);
#pragma unroll
        for (int t = 0; t < 4; ++t) acc[1 + t] = fma(x, a.e_side[(long long)t * a.N + i], acc[1 + t]);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < 5; ++t) {
        const double v = warp_sum(acc[t]);
        if (lane == 0) sm[wid][t] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double v = 0.0;
        for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) v += sm[w2][threadIdx.x];
        part[blockIdx.x * 8 + threadIdx.x] = v;
    }
}

// Backward-Euler time source (Sec. 3.7): products of basis column m = rank_sel - 1 with F[d] of
// every distinct direction, the entries the bordered Galerkin right-hand sides take.  Grid
// (row chunks of kXtRows, groups of 8 directions): warp w of block (b, y) forms the chunk-b part
// of F[8 y + w] . x_m into part[b ndir + d]; fsrc_dots_final adds the chunks into bF[d rc + m].
__global__ void __launch_bounds__(256) fsrc_dots_partial(LRArgs a, int gm, int rsel, double* __restrict__ part) {
    pdl_entry();
    __shared__ double xs[1024];
    if (!gate(a.st, gm)) return;
    const int r = rank_sel(a.st, rsel);
    if (r < 1) return;
    const int row0 = blockIdx.x * 1024;
    const int len = min(1024, a.N - row0);
    const double* x = a.X + (long long)(r - 1) * a.N + row0;
    for (int i = threadIdx.x; i < len; i += blockDim.x) xs[i] = x[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, d = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (d >= a.ndir) return;
    const double* f = a.F + (long long)d * a.N + row0;
    double acc = 0.0;
    for (int i = lane; i < len; i += 32) acc = fma(f[i], xs[i], acc);
    acc = warp_sum(acc);
    if (lane == 0) part[(long long)blockIdx.x * a.ndir + d] = acc;
}

__global__ void __launch_bounds__(256) fsrc_dots_final(LRArgs a, int gm, int rsel, const double* __restrict__ part,
                                                       int nblk) {
    pdl_entry();
    if (!gate(a.st, gm)) return;
    const int r = rank_sel(a.st, rsel);
    if (r < 1) return;
    const int lane = threadIdx.x & 31, d = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (d >= a.ndir) return;
    double s_ = 0.0;
    for (int b = lane; b < nblk; b += 32) s_ += part[(long long)b * a.ndir + d];
    s_ = warp_sum(s_);
    if (lane == 0) a.bF[(long long)d * a.rc + (r - 1)] = s_;
}

// Sources of the sampled sweeps with the time source: slot l sweeps angle j = st[I_NEW + l] with
// S + F[dir_of[j]] (rounded once to the sweep precision).
template <typename T>
__global__ void fsrc_sweep_source(LRArgs a, int p, T* __restrict__ out) {
    pdl_entry();
    if (!gate(a.st, G_LIVE)) return;
    const int nn = min(p, a.st[I_NNEW]);
    const long long N = a.N, total = N * nn;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const int l = (int)(k / N);
        const long long i = k - (long long)l * N;
        out[k] = T(a.S[i] + a.F[(long long)a.dir_of[a.st[I_NEW + l]] * N + i]);
    }
}

// Border of X^T D_x^- X, X^T D_y^- X, X^T Sigma_t X (column r-1 and row r-1), bS, bE entries.
__global__ void border_write(LRArgs a, int gm, int rsel) {
    pdl_entry();
    if (!gate(a.st, gm)) return;
    const int r = rank_sel(a.st, rsel);
    if (r < 1) return;
    const int m = r - 1;
    const SmallLayout SL{a.rc};
    const double* B = a.sm + SL.border();   // [5][rc]
    const double* D = a.sm + SL.dots();     // [5]
    const int rc = a.rc;
    for (int k = threadIdx.x; k < r; k += blockDim.x) {
        a.Pxm[(long long)m * rc + k] = B[0 * rc + k];        // X_k^T D_x^- p     (column m)
        a.Pxm[(long long)k * rc + m] = B[1 * rc + k];        // p^T D_x^- X_k     (row m)
        a.Pym[(long long)m * rc + k] = B[2 * rc + k];
        a.Pym[(long long)k * rc + m] = B[3 * rc + k];
        a.T[(long long)m * rc + k] = B[4 * rc + k];
        a.T[(long long)k * rc + m] = B[4 * rc + k];
    }
    if (threadIdx.x == 0) a.bS[m] = D[0];
    if (threadIdx.x >= 1 && threadIdx.x < 5) a.bE[(threadIdx.x - 1) * rc + m] = D[threadIdx.x];
}

// ------------------------------------------------------------------ Galerkin factors
__device__ __forceinline__ void dir_coeffs(const LRArgs& a, int d, double& ox, double& oy, double gc[4]) {
    const int j = a.dir_rep[d];
    ox = a.ox[j];
    oy = a.oy[j];
    gc[0] = fmax(ox, 0.0) * a.g[0];
    gc[1] = -fmin(ox, 0.0) * a.g[1];
    gc[2] = fmax(oy, 0.0) * a.g[2];
    gc[3] = -fmin(oy, 0.0) * a.g[3];
}

// entry (row i, col k) of A_d = Ox Px + Oy Py + T with Px = Pxm (Ox >= 0) or -Pxm^T (Ox < 0)
__device__ __forceinline__ double A_entry(const LRArgs& a, double ox, double oy, int i, int k) {
    const long long rc = a.rc;
    const double px = ox >= 0.0 ? a.Pxm[k * rc + i] : -a.Pxm[i * rc + k];
    const double py = oy >= 0.0 ? a.Pym[k * rc + i] : -a.Pym[i * rc + k];
    return fma(ox, px, fma(oy, py, a.T[k * rc + i]));
}

// cp.async staging of the next kDq columns of a triangular factor (global -> shared).
constexpr int kDq = 4;
__device__ __forceinline__ void cpa8(double* dst, const double* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N_>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N_) : "memory"); }

// One warp sweeps a triangular factor for nrhs right-hand sides at once (vectors vec + t*vstride,
// t < nrhs): the factor column of step k is staged once (kDq - 1 steps ahead) and applied to
// every vector, so the sequential chain has m steps however many vectors there are.
__device__ void tri_sweep_multi(const double* __restrict__ base, long long ld, int m, const double* dinv, double* vec,
                                int vstride, int nrhs, double* stage /*[kDq][rcap]*/, int rcap) {
    const bool divide = dinv != nullptr;     // scale by the reciprocal diagonal (non-unit factor)
    const int lane = threadIdx.x & 31;
    auto issue = [&](int k) {
        if (k < m) {
            double* dst = stage + (size_t)(k % kDq) * rcap;
            const double* src = base + (long long)k * ld;
            for (int i = lane; i < m; i += 32) cpa8(dst + i, src + i);
        }
        cpa_commit();
    };
#pragma unroll
    for (int t = 0; t < kDq - 1; ++t) issue(t);
    for (int k = 0; k < m; ++k) {
        issue(k + kDq - 1);
        cpa_wait<kDq - 1>();
        __syncwarp();
        const double* col = stage + (size_t)(k % kDq) * rcap;
        const double rk = divide ? dinv[k] : 1.0;
        for (int t = 0; t < nrhs; ++t) {
            double* v = vec + (size_t)t * vstride;
            double xk = v[k];
            if (divide) xk *= rk;
            __syncwarp();
            if (divide && lane == 0) v[k] = xk;
            for (int i = k + 1 + lane; i < m; i += 32) v[i] = fma(-col[i], xk, v[i]);
        }
        __syncwarp();
    }
    cpa_wait<0>();
    __syncwarp();
}

constexpr int kBorderWarps = 8;      // most warps per side (L solve / U^T solve) in lu_border
constexpr int kBorderChunk = 8;      // new columns bordered per pass

// Block bordering of the LU factors of every direction that still needs Galerkin solutions by
// the np = r - r0 columns appended in this inner iteration (one launch instead of one per
// column): with A11 = L11 U11 (m0 = r0),
//   U12 = L11^{-1} A12,  L21 = A21 U11^{-1},  S = A22 - L21 U12 = L22 U22 (no pivoting),
//   y2 = L22^{-1} (b2 - L21 y1).
// The same factors as bordering one column at a time (LU without pivoting is unique).  One
// block per direction: warps 0..7 run L11^{-1} on the new columns, warps 8..15 U11^{-T} on the
// new rows, kBorderChunk columns per pass.  A large basis capacity gives each side fewer warps
// (blockDim / 64 per side, each with its own staging ring), which then take several vectors.
__global__ void __launch_bounds__(64 * kBorderWarps) lu_border(LRArgs a) {
    pdl_entry();
    if (!gate(a.st, G_LIVE)) return;
    const int d = blockIdx.x;
    if (d >= a.ndir) return;
    const int rep = a.dir_rep[d];
    if (status_arr(a)[rep] == 1) return;
    const int r = a.st[I_R], r0 = a.st[I_R0];
    if (r <= r0) return;
    extern __shared__ __align__(16) double sh[];
    const int rcp = a.rc;
    double* va = sh;                                             // [chunk][rc] new columns
    double* vb = sh + (size_t)kBorderChunk * rcp;                // [chunk][rc] new rows
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double* stage = sh + (size_t)2 * kBorderChunk * rcp + (size_t)wid * kDq * rcp;
    const long long rc = a.rc;
    double ox, oy, gc[4];
    dir_coeffs(a, d, ox, oy, gc);
    double* L = a.Lf + (long long)d * rc * rc;   // column-major: L[k*rc + i] = L(i, k)
    double* U = a.Uf + (long long)d * rc * rc;   // row-major:    U[i*rc + k] = U(i, k)
    double* Yd = a.Y + (long long)d * rc;
    double* Ud = a.Udinv + (long long)d * rc;
    for (int c0 = r0; c0 < r; c0 += kBorderChunk) {
        const int m0 = c0;                        // factors are complete up to m0
        const int np = min(kBorderChunk, r - c0);
        // new columns c0..c0+np-1: rows 0..m0-1 (col) and cols 0..m0-1 (row)
        for (int idx = threadIdx.x; idx < np * m0; idx += blockDim.x) {
            const int t = idx / m0, i = idx % m0;
            va[(size_t)t * rcp + i] = A_entry(a, ox, oy, i, m0 + t);
            vb[(size_t)t * rcp + i] = A_entry(a, ox, oy, m0 + t, i);
        }
        __syncthreads();
        if (m0 > 0) {
            const int nw = blockDim.x >> 6;          // warps per side
            const int side = wid / nw, wl = wid % nw;
            // warp wl of a side takes vectors wl, wl + nw, ...
            for (int t = wl; t < np; t += nw) {
                if (side == 0) tri_sweep_multi(L, rc, m0, nullptr, va + (size_t)t * rcp, rcp, 1, stage, rcp);
                else tri_sweep_multi(U, rc, m0, Ud, vb + (size_t)t * rcp, rcp, 1, stage, rcp);
            }
        }
        __syncthreads();
        // store U12 (column m0+t of U, rows < m0) and L21 (row m0+t of L, columns < m0)
        for (int idx = threadIdx.x; idx < np * m0; idx += blockDim.x) {
            const int t = idx / m0, i = idx % m0;
            U[(long long)i * rc + m0 + t] = va[(size_t)t * rcp + i];
            L[(long long)i * rc + m0 + t] = vb[(size_t)t * rcp + i];
        }
        // Schur complement and its LU, then y2: warp 0 (np <= kBorderChunk)
        if (wid == 0) {
            __shared__ double Sb[kBorderChunk][kBorderChunk];
            __shared__ double yb[kBorderChunk];
            for (int e = 0; e < np * np; ++e) {
                const int t = e / np, u = e % np;
                double acc = 0.0;
                for (int i = lane; i < m0; i += 32) acc = fma(vb[(size_t)t * rcp + i], va[(size_t)u * rcp + i], acc);
                acc = warp_sum(acc);
                if (lane == 0) Sb[t][u] = A_entry(a, ox, oy, m0 + t, m0 + u) - acc;
            }
            for (int t = 0; t < np; ++t) {
                double acc = 0.0;
                for (int i = lane; i < m0; i += 32) acc = fma(vb[(size_t)t * rcp + i], Yd[i], acc);
                acc = warp_sum(acc);
                if (lane == 0) {
                    double bm = a.bS[m0 + t];
                    for (int s2 = 0; s2 < 4; ++s2) bm = fma(gc[s2], a.bE[s2 * rc + m0 + t], bm);
                    if (a.bF) bm += a.bF[(long long)d * rc + m0 + t];      // time source
                    yb[t] = bm - acc;
                }
            }
            __syncwarp();
            if (lane == 0) {
                // in-place LU of Sb (unit lower below, upper on and above the diagonal)
                for (int k = 0; k < np; ++k) {
                    if (!(fabs(Sb[k][k]) > 0.0)) a.st[I_SING] = Sb[k][k] == 0.0 ? 1 : 2;   // 2: NaN
                    for (int i = k + 1; i < np; ++i) {
                        const double f = Sb[i][k] / Sb[k][k];
                        Sb[i][k] = f;
                        for (int jj = k + 1; jj < np; ++jj) Sb[i][jj] = fma(-f, Sb[k][jj], Sb[i][jj]);
                    }
                }
                for (int t = 0; t < np; ++t) {
                    double y = yb[t];
                    for (int k = 0; k < t; ++k) y = fma(-Sb[t][k], yb[k], y);
                    yb[t] = y;
                    Yd[m0 + t] = y;
                }
                for (int t = 0; t < np; ++t) Ud[m0 + t] = 1.0 / Sb[t][t];
                for (int t = 0; t < np; ++t)
                    for (int u = 0; u < np; ++u) {
                        if (u >= t) U[(long long)(m0 + t) * rc + m0 + u] = Sb[t][u];
                        if (u < t) L[(long long)(m0 + u) * rc + m0 + t] = Sb[t][u];
                        if (u == t) L[(long long)(m0 + t) * rc + m0 + t] = 1.0;
                    }
            }
            __syncwarp();
        }
        __syncthreads();
    }
}

// c = U^{-1} y for direction d by one warp: columns of the row-major U taken from the last
// (strided, U[i*rc + k]) and staged kDq - 1 steps ahead; ws: [rc + kDq*rc] shared scratch.
__device__ void back_subst_warp(const LRArgs& a, int d, int r, double* ws, double* out) {
    const int lane = threadIdx.x & 31;
    const long long rc = a.rc;
    const double* U = a.Uf + (long long)d * rc * rc;
    const double* Yd = a.Y + (long long)d * rc;
    const double* Ud = a.Udinv + (long long)d * rc;
    double* cs = ws;
    double* stage = ws + rc;
    for (int i = lane; i < r; i += 32) cs[i] = Yd[i];
    __syncwarp();
    // step t handles column k = r - 1 - t: entries U[i*rc + k] for i <= k
    auto issue = [&](int t) {
        const int k = r - 1 - t;
        if (k >= 0) {
            double* dst = stage + (size_t)(t % kDq) * rc;
            for (int i = lane; i <= k; i += 32) cpa8(dst + i, U + (long long)i * rc + k);
        }
        cpa_commit();
    };
#pragma unroll
    for (int t = 0; t < kDq - 1; ++t) issue(t);
    for (int t = 0; t < r; ++t) {
        const int k = r - 1 - t;
        issue(t + kDq - 1);
        cpa_wait<kDq - 1>();
        __syncwarp();
        const double* col = stage + (size_t)(t % kDq) * rc;
        const double ck = cs[k] * Ud[k];
        __syncwarp();
        if (lane == 0) cs[k] = ck;
        for (int i = lane; i < k; i += 32) cs[i] = fma(-col[i], ck, cs[i]);
        __syncwarp();
    }
    cpa_wait<0>();
    __syncwarp();
    for (int i = lane; i < r; i += 32) out[i] = cs[i];
}

// ------------------------------------------------------------------ candidates
__global__ void iter_begin(LRArgs a) {
    pdl_entry();
    if (blockIdx.x != 0 || !gate(a.st, G_LIVE)) return;
    for (int l = threadIdx.x; l < 64; l += blockDim.x) a.st[I_BCOL + l] = -1;
    if (threadIdx.x == 0) {
        a.st[I_K] += 1;
        a.st[I_R0] = a.st[I_R];
    }
}

// Draw `count` unsampled angles with the smallest Philox keys at (seed, n, k): into I_NEW
// (dst = I_NEW, the initial sample) or the candidate list (dst = -1).
__global__ void draw_kernel(LRArgs a, int count, int dst, int gm) {
    pdl_entry();
    extern __shared__ unsigned long long keys[];   // [nang] (key << 32 | j), ~0 for excluded
    if (!gate(a.st, gm)) return;
    const int* status = status_arr(a);
    const unsigned n = (unsigned)a.st[I_OUTER], k = (unsigned)a.st[I_K];
    for (int j = threadIdx.x; j < a.nang; j += blockDim.x)
        keys[j] = status[j] == 0 ? (((unsigned long long)philox_key(a.seed, n, k, (unsigned)j) << 32) | (unsigned)j)
                                 : ~0ull;
    __syncthreads();
    __shared__ unsigned long long best[32];
    int got = 0;
    for (int t = 0; t < count; ++t) {
        unsigned long long mn = ~0ull;
        for (int j = threadIdx.x; j < a.nang; j += blockDim.x) mn = min(mn, keys[j]);
        for (int o = 16; o > 0; o >>= 1) mn = min(mn, (unsigned long long)__shfl_xor_sync(0xffffffffu, mn, o));
        if ((threadIdx.x & 31) == 0) best[threadIdx.x >> 5] = mn;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long b = ~0ull;
            for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) b = min(b, best[w2]);
            best[0] = b;
        }
        __syncthreads();
        const unsigned long long b = best[0];
        __syncthreads();
        if (b == ~0ull) break;
        const int j = (int)(b & 0xffffffffull);
        if (threadIdx.x == 0) {
            if (dst == I_NEW) a.st[I_NEW + t] = j;
            else cand_arr(a)[t] = j;
            keys[j] = ~0ull;
        }
        __syncthreads();
        ++got;
    }
    if (threadIdx.x == 0) a.st[dst == I_NEW ? I_NNEW : I_NCAND] = got;
}

// back-substitution for the candidates: Ccand[t] = U^{-1} y of the candidate's direction
__global__ void cand_solve(LRArgs a) {
    pdl_entry();
    extern __shared__ __align__(16) double ws[];
    if (!gate(a.st, G_LIVE)) return;
    const int t = blockIdx.x;
    if (t >= a.st[I_NCAND]) return;
    const int j = cand_arr(a)[t];
    double* out = a.sm + SmallLayout{a.rc}.ccand() + (long long)t * a.rc;
    const int r = a.st[I_R];
    back_subst_warp(a, a.dir_of[j], r, ws, out);
    if (a.dwb)                                       // each lane reads back what it wrote
        for (int i = threadIdx.x & 31; i < r; i += 32) {
            const DW d = dw_of(out[i]);
            a.ccand2[(long long)t * a.rc + i] = make_float2(d.h, d.l);
        }
}

// residual norms: red[t][b] = sum over cells of block b of |S + g_j - (D_j + Sigma_t) v_t|^2
__global__ void __launch_bounds__(256) cand_residual(LRArgs a) {
    pdl_entry();
    if (!gate(a.st, G_LIVE)) return;
    const int t = blockIdx.y;
    if (t >= a.st[I_NCAND]) return;
    const int j = cand_arr(a)[t];
    const double ox = a.ox[j], oy = a.oy[j];
    const double ax = fabs(ox) * a.ihx, ay = fabs(oy) * a.ihy;
    const double s3 = 1.7320508075688772935;
    const double* v = a.vcand + (long long)t * a.N;
    double acc = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.nc; c += gridDim.x * blockDim.x) {
        const int ix = c % a.nx, iy = c / a.nx;
        const double v0 = v[4 * c], v1 = v[4 * c + 1], v2 = v[4 * c + 2], v3 = v[4 * c + 3];
        double y0, y1, y2, y3;
        // x part: Ox >= 0 -> ax [K v - l (rho . v_left)];  Ox < 0 -> ax [K^T v - rho (l . v_right)]
        if (ox >= 0.0) {
            double t0 = 0, t1 = 0;
            if (ix > 0) { const double* q = v + 4 * (c - 1); t0 = q[0] + s3 * q[1]; t1 = q[2] + s3 * q[3]; }
            y0 = ax * (v0 + s3 * v1 - t0);
            y1 = ax * (-s3 * v0 + 3 * v1 + s3 * t0);
            y2 = ax * (v2 + s3 * v3 - t1);
            y3 = ax * (-s3 * v2 + 3 * v3 + s3 * t1);
        } else {
            double t0 = 0, t1 = 0;
            if (ix + 1 < a.nx) { const double* q = v + 4 * (c + 1); t0 = q[0] - s3 * q[1]; t1 = q[2] - s3 * q[3]; }
            y0 = ax * (v0 - s3 * v1 - t0);
            y1 = ax * (s3 * v0 + 3 * v1 - s3 * t0);
            y2 = ax * (v2 - s3 * v3 - t1);
            y3 = ax * (s3 * v2 + 3 * v3 - s3 * t1);
        }
        if (oy >= 0.0) {
            double t0 = 0, t1 = 0;
            if (iy > 0) { const double* q = v + 4 * (c - a.nx); t0 = q[0] + s3 * q[2]; t1 = q[1] + s3 * q[3]; }
            y0 += ay * (v0 + s3 * v2 - t0);
            y2 += ay * (-s3 * v0 + 3 * v2 + s3 * t0);
            y1 += ay * (v1 + s3 * v3 - t1);
            y3 += ay * (-s3 * v1 + 3 * v3 + s3 * t1);
        } else {
            double t0 = 0, t1 = 0;
            if (iy + 1 < a.ny) { const double* q = v + 4 * (c + a.nx); t0 = q[0] - s3 * q[2]; t1 = q[1] - s3 * q[3]; }
            y0 += ay * (v0 - s3 * v2 - t0);
            y2 += ay * (s3 * v0 + 3 * v2 - s3 * t0);
            y1 += ay * (v1 - s3 * v3 - t1);
            y3 += ay * (s3 * v1 + 3 * v3 - s3 * t1);
        }
        const double sg = a.sig_t[c];
        double g0 = 0, g1 = 0, g2 = 0, g3 = 0;
        const double gcx = ox >= 0 ? ox * a.g[0] : -ox * a.g[1];
        const double gcy = oy >= 0 ? oy * a.g[2] : -oy * a.g[3];
        if (gcx != 0.0 && ((ox >= 0 && ix == 0) || (ox < 0 && ix == a.nx - 1))) {
            const double* e = a.e_side + (ox >= 0 ? 0 : (long long)a.N) + 4 * (long long)c;
            g0 += gcx * e[0]; g1 += gcx * e[1]; g2 += gcx * e[2]; g3 += gcx * e[3];
        }
        if (gcy != 0.0 && ((oy >= 0 && iy == 0) || (oy < 0 && iy == a.ny - 1))) {
            const double* e = a.e_side + (oy >= 0 ? 2 : 3) * (long long)a.N + 4 * (long long)c;
            g0 += gcy * e[0]; g1 += gcy * e[1]; g2 += gcy * e[2]; g3 += gcy * e[3];
        }
        if (a.F) {                                       // time source of the candidate's direction
            const double* f = a.F + (long long)a.dir_of[j] * a.N + 4 * (long long)c;
            g0 += f[0]; g1 += f[1]; g2 += f[2]; g3 += f[3];
        }
        const double r0 = a.S[4 * c] + g0 - (y0 + sg * v0);
        const double r1 = a.S[4 * c + 1] + g1 - (y1 + sg * v1);
        const double r2 = a.S[4 * c + 2] + g2 - (y2 + sg * v2);
        const double r3 = a.S[4 * c + 3] + g3 - (y3 + sg * v3);
        acc += r0 * r0 + r1 * r1 + r2 * r2 + r3 * r3;
    }
    acc = warp_sum(acc);
    __shared__ double sm[32];
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) s += sm[w2];
        a.red[(long long)t * gridDim.x + blockIdx.x] = s;
    }
}

// cand_residual in double-word FP32: v = X c_j from x_times_dw, S from S2, sigma_t from its
// hi / lo split.  With S_x = sign(Omega_x) sqrt3 the x part of D_j v in both upwind forms is
//   a_x (v0 + S_x v1 - t0),  a_x (3 v1 + S_x (t0 - v0))   (and v2, v3, t1 likewise),
// t = (q0 + S_x q1, q2 + S_x q3) the upwind x-neighbour's outflow trace; the y part likewise with
// the modes (0, 2), (1, 3).  Inflow terms (boundary cells only) are formed in FP64.
__global__ void __launch_bounds__(256) cand_residual_dw(LRArgs a) {
    pdl_entry();
    __shared__ float2 kc[4];
    if (!gate(a.st, G_LIVE)) return;
    const int t = blockIdx.y;
    if (t >= a.st[I_NCAND]) return;
    const int j = cand_arr(a)[t];
    const double ox = a.ox[j], oy = a.oy[j];
    if (threadIdx.x == 0) {
        const double s3 = 1.7320508075688772935;
        const DW d0 = dw_of(fabs(ox) * a.ihx), d1 = dw_of(fabs(oy) * a.ihy);
        const DW d2 = dw_of(ox >= 0.0 ? s3 : -s3), d3 = dw_of(oy >= 0.0 ? s3 : -s3);
        kc[0] = make_float2(d0.h, d0.l); kc[1] = make_float2(d1.h, d1.l);
        kc[2] = make_float2(d2.h, d2.l); kc[3] = make_float2(d3.h, d3.l);
    }
    __syncthreads();
    const DW ax{kc[0].x, kc[0].y}, ay{kc[1].x, kc[1].y}, Sx{kc[2].x, kc[2].y}, Sy{kc[3].x, kc[3].y};
    const bool px = ox >= 0.0, py = oy >= 0.0;
    const double gcx = px ? ox * a.g[0] : -ox * a.g[1];
    const double gcy = py ? oy * a.g[2] : -oy * a.g[3];
    const float2* v = reinterpret_cast<const float2*>(a.vcand) + (long long)t * a.N;
    DW acc{0.f, 0.f};
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.nc; c += gridDim.x * blockDim.x) {
        const int ix = c % a.nx, iy = c / a.nx;
        const DW v0 = dw_load(v + 4 * c), v1 = dw_load(v + 4 * c + 1), v2 = dw_load(v + 4 * c + 2),
                 v3 = dw_load(v + 4 * c + 3);
        DW t0{0.f, 0.f}, t1{0.f, 0.f}, u0{0.f, 0.f}, u1{0.f, 0.f};
        const int cx = px ? c - 1 : c + 1;
        if (px ? ix > 0 : ix + 1 < a.nx) {
            const float2* q = v + 4 * cx;
            t0 = dw_add(dw_load(q), dw_mul(Sx, dw_load(q + 1)));
            t1 = dw_add(dw_load(q + 2), dw_mul(Sx, dw_load(q + 3)));
        }
        const int cy = py ? c - a.nx : c + a.nx;
        if (py ? iy > 0 : iy + 1 < a.ny) {
            const float2* q = v + 4 * cy;
            u0 = dw_add(dw_load(q), dw_mul(Sy, dw_load(q + 2)));
            u1 = dw_add(dw_load(q + 1), dw_mul(Sy, dw_load(q + 3)));
        }
        // (D_j v) by modes: x pairs (v0, v1; t0), (v2, v3; t1); y pairs (v0, v2; u0), (v1, v3; u1)
        auto lo_part = [](DW a0, DW a1, DW tr, DW s) { return dw_add(dw_add(a0, dw_mul(s, a1)), dw_neg(tr)); };
        auto hi_part = [](DW a0, DW a1, DW tr, DW s) { return dw_add(dw_mul_f(a1, 3.f), dw_mul(s, dw_add(tr, dw_neg(a0)))); };
        const DW y0 = dw_add(dw_mul(ax, lo_part(v0, v1, t0, Sx)), dw_mul(ay, lo_part(v0, v2, u0, Sy)));
        const DW y1 = dw_add(dw_mul(ax, hi_part(v0, v1, t0, Sx)), dw_mul(ay, lo_part(v1, v3, u1, Sy)));
        const DW y2 = dw_add(dw_mul(ax, lo_part(v2, v3, t1, Sx)), dw_mul(ay, hi_part(v0, v2, u0, Sy)));
        const DW y3 = dw_add(dw_mul(ax, hi_part(v2, v3, t1, Sx)), dw_mul(ay, hi_part(v1, v3, u1, Sy)));
        const DW sg{a.sig_h[c], a.sig_l[c]};
        DW r0 = dw_add(dw_load(a.S2 + 4 * c), dw_neg(dw_add(y0, dw_mul(sg, v0))));
        DW r1 = dw_add(dw_load(a.S2 + 4 * c + 1), dw_neg(dw_add(y1, dw_mul(sg, v1))));
        DW r2 = dw_add(dw_load(a.S2 + 4 * c + 2), dw_neg(dw_add(y2, dw_mul(sg, v2))));
        DW r3 = dw_add(dw_load(a.S2 + 4 * c + 3), dw_neg(dw_add(y3, dw_mul(sg, v3))));
        const bool bx = gcx != 0.0 && (px ? ix == 0 : ix == a.nx - 1);
        const bool by = gcy != 0.0 && (py ? iy == 0 : iy == a.ny - 1);
        if (bx || by) {
            double g0 = 0, g1 = 0, g2 = 0, g3 = 0;
            if (bx) {
                const double* e = a.e_side + (px ? 0 : (long long)a.N) + 4 * (long long)c;
                g0 += gcx * e[0]; g1 += gcx * e[1]; g2 += gcx * e[2]; g3 += gcx * e[3];
            }
            if (by) {
                const double* e = a.e_side + (py ? 2 : 3) * (long long)a.N + 4 * (long long)c;
                g0 += gcy * e[0]; g1 += gcy * e[1]; g2 += gcy * e[2]; g3 += gcy * e[3];
            }
            r0 = dw_add(r0, dw_of(g0)); r1 = dw_add(r1, dw_of(g1));
            r2 = dw_add(r2, dw_of(g2)); r3 = dw_add(r3, dw_of(g3));
        }
        if (a.F) {                                       // time source of the candidate's direction
            const double* f = a.F + (long long)a.dir_of[j] * a.N + 4 * (long long)c;
            r0 = dw_add(r0, dw_of(f[0])); r1 = dw_add(r1, dw_of(f[1]));
            r2 = dw_add(r2, dw_of(f[2])); r3 = dw_add(r3, dw_of(f[3]));
        }
        dw_mac(acc, r0, r0);
        dw_mac(acc, r1, r1);
        dw_mac(acc, r2, r2);
        dw_mac(acc, r3, r3);
    }
    const double s = dw_block_sum(dw_norm(acc));
    if (threadIdx.x == 0) a.red[(long long)t * gridDim.x + blockIdx.x] = s;
}

// norms (one warp per candidate), top-p selection (largest first, ties to the smaller index)
// and the residual test of Sec. 3.3
__global__ void __launch_bounds__(1024) select_kernel(LRArgs a, int nblk) {
    pdl_entry();
    if (!gate(a.st, G_LIVE)) return;
    const int nc_ = a.st[I_NCAND];
    double* norms = a.sm + SmallLayout{a.rc}.norms();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int t = wid; t < nc_; t += blockDim.x >> 5) {
        double s = 0.0;
        for (int b = lane; b < nblk; b += 32) s += a.red[(long long)t * nblk + b];
        s = warp_sum(s);
        if (lane == 0) norms[t] = sqrt(s);
    }
    __syncthreads();
    // every candidate finds its place in the order (norm descending, angle index ascending on
    // ties: a strict order, the angles are distinct); the first p places are selected
    __shared__ int any_nan;
    if (threadIdx.x == 0) any_nan = 0;
    __syncthreads();
    if (threadIdx.x < nc_ && !(norms[threadIdx.x] == norms[threadIdx.x])) any_nan = 1;
    __syncthreads();
    const int nsel = min(a.p, nc_);
    if (!any_nan) {
        if (threadIdx.x < nc_) {
            const int t = threadIdx.x;
            const double nt = norms[t];
            const int jt = cand_arr(a)[t];
            int place = 0;
            for (int u = 0; u < nc_; ++u) {
                const double nu = norms[u];
                place += (nu > nt || (nu == nt && cand_arr(a)[u] < jt)) ? 1 : 0;
            }
            if (place < nsel) a.st[I_NEW + place] = jt;
        }
    }
    if (threadIdx.x != 0) return;
    double mx = 0.0;
    for (int t = 0; t < nc_; ++t) mx = fmax(mx, norms[t]);
    scal(a)[S_MAXRES] = any_nan ? nan_val() : mx;
    if (any_nan) {
        // a non-finite residual ends the inner loop at the full check that follows; the angles
        // are picked in candidate order (the order above is not defined for NaN)
        for (int s = 0; s < nsel; ++s) a.st[I_NEW + s] = cand_arr(a)[s];
    }
    a.st[I_NNEW] = nsel;
    a.st[I_FULL] = (nc_ == 0 || mx < a.eps_res || any_nan) ? 1 : 0;
}

// full check: Galerkin solutions of every direction without an R column (one warp each)
__global__ void full_solve(LRArgs a) {
    pdl_entry();
    extern __shared__ __align__(16) double ws_all[];
    if (!gate(a.st, G_FULL)) return;
    const int wl = threadIdx.x >> 5;
    const int d = blockIdx.x * (blockDim.x >> 5) + wl;
    if (d >= a.ndir) return;
    if (status_arr(a)[a.dir_rep[d]] == 1) return;
    back_subst_warp(a, d, a.st[I_R], ws_all + (size_t)wl * (kDq + 1) * a.rc, a.Cdir + (long long)d * a.rc);
}

// C (all angles, column j at j*rc) and Cw = C w
__global__ void full_assemble(LRArgs a) {
    pdl_entry();
    if (!gate(a.st, G_FULL)) return;
    const int r = a.st[I_R];
    const int* status = status_arr(a);
    const int* colof = colof_arr(a);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < r * a.nang; t += gridDim.x * blockDim.x) {
        const int j = t / r, k = t % r;
        double v;
        if (status[j] == 1) v = a.R[(long long)colof[j] * a.rc + k];     // zero below the diagonal entry
        else v = a.Cdir[(long long)a.dir_of[j] * a.rc + k];
        a.Cfull[(long long)j * a.rc + k] = v;
    }
}

__global__ void full_cw(LRArgs a) {
    pdl_entry();
    if (!gate(a.st, G_FULL)) return;
    const int r = a.st[I_R];
    double* cw = a.sm + SmallLayout{a.rc}.cw();
    const int lane = threadIdx.x & 31;
    const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (k >= r) return;
    double s = 0.0;
    for (int j = lane; j < a.nang; j += 32) s = fma(a.Cfull[(long long)j * a.rc + k], a.w[j], s);
    s = warp_sum(s);
    if (lane == 0) cw[k] = s;
}

// phi^{(n,k)} = X (C w); W[0:N] = phi^{(n,k)} - phi_old (for the norm)
__global__ void __launch_bounds__(256) full_phi(LRArgs a) {
    pdl_entry();
    extern __shared__ double cs[];
    if (!gate(a.st, G_FULL)) return;
    const int r = a.st[I_R];
    const double* cw = a.sm + SmallLayout{a.rc}.cw();
    for (int k = threadIdx.x; k < r; k += blockDim.x) cs[k] = cw[k];
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < r; ++k) s = fma(a.X[(long long)k * a.N + i], cs[k], s);
        a.phi_k[i] = s;
        a.W[i] = s - a.phi_old[i];
    }
}

__global__ void full_decide(LRArgs a) {
    pdl_entry();
    if (threadIdx.x != 0 || blockIdx.x != 0 || !gate(a.st, G_FULL)) return;
    const double diff = scal(a)[S_DIFF];
    a.st[I_FULLCNT] += 1;
    if (diff <= a.eps_diff || a.st[I_NCAND] == 0 || !(diff == diff)) {
        a.st[I_STOP] = 1;
        a.st[I_NNEW] = 0;
    }
}

// DEIM sampling (remark in Sec. 3.2), before the full check of every inner iteration: the
// number of unsampled angles stands in for the candidate count (the full check stops the loop
// when it is zero) and the full check is requested.
__global__ void deim_prepare(LRArgs a) {
    pdl_entry();
    if (!gate(a.st, G_LIVE)) return;
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    const int* status = status_arr(a);
    int c = 0;
    for (int j = threadIdx.x; j < a.nang; j += blockDim.x) c += status[j] == 0;
    atomicAdd(&cnt, c);
    __syncthreads();
    if (threadIdx.x == 0) {
        a.st[I_NCAND] = cnt;
        a.st[I_FULL] = 1;
    }
}

// DEIM points (Chaturantabut and Sorensen, 2010) of the p leading right singular vectors of C
// among the unsampled angles, after the SVD of the full check's C: A [r][nang] holds
// sigma_k v_k column by column (one-sided Jacobi), sig the sigma_k.  Point l maximises
// |v_l - V_{<l} (V_{<l}[pts])^{-1} v_l[pts]| over the unsampled angles (ties to the smaller
// index); the column scaling by sigma does not change the points.  One block.
constexpr int kDeimMax = 64;
__global__ void __launch_bounds__(256) deim_select(LRArgs a, const double* __restrict__ A,
                                                   const double* __restrict__ sig) {
    pdl_entry();
    if (!gate(a.st, G_LIVE)) return;
    const int r = a.st[I_R], M = a.nang;
    const int* status = status_arr(a);
    __shared__ int order[kDeimMax], pts[kDeimMax];
    __shared__ double Ms[kDeimMax * kDeimMax], cv[kDeimMax];
    __shared__ double bv[8];
    __shared__ int bi[8];
    __shared__ int got_s;
    const int np = min(min(a.p, r), kDeimMax);
    for (int k = threadIdx.x; k < r; k += blockDim.x) {
        int rank = 0;
        for (int u = 0; u < r; ++u) rank += (sig[u] > sig[k] || (sig[u] == sig[k] && u < k)) ? 1 : 0;
        if (rank < np) order[rank] = k;
    }
    if (threadIdx.x == 0) got_s = 0;
    __syncthreads();
    for (int l = 0; l < np; ++l) {
        const double* vl = A + (long long)order[l] * M;
        if (threadIdx.x == 0 && l > 0) {
            // the l x l interpolation system at the points so far, Gaussian elimination with
            // partial pivoting
            for (int i = 0; i < l; ++i) {
                for (int t = 0; t < l; ++t) Ms[i * kDeimMax + t] = A[(long long)order[t] * M + pts[i]];
                cv[i] = vl[pts[i]];
            }
            for (int c = 0; c < l; ++c) {
                int pv = c;
                for (int i = c + 1; i < l; ++i)
                    if (fabs(Ms[i * kDeimMax + c]) > fabs(Ms[pv * kDeimMax + c])) pv = i;
                if (pv != c) {
                    for (int t = 0; t < l; ++t) {
                        const double tmp = Ms[c * kDeimMax + t];
                        Ms[c * kDeimMax + t] = Ms[pv * kDeimMax + t];
                        Ms[pv * kDeimMax + t] = tmp;
                    }
                    const double tmp = cv[c]; cv[c] = cv[pv]; cv[pv] = tmp;
                }
                const double d = Ms[c * kDeimMax + c];
                for (int i = c + 1; i < l; ++i) {
                    const double f = d != 0.0 ? Ms[i * kDeimMax + c] / d : 0.0;
                    for (int t = c; t < l; ++t) Ms[i * kDeimMax + t] = fma(-f, Ms[c * kDeimMax + t], Ms[i * kDeimMax + t]);
                    cv[i] = fma(-f, cv[c], cv[i]);
                }
            }
            for (int c = l - 1; c >= 0; --c) {
                double x = cv[c];
                for (int t = c + 1; t < l; ++t) x = fma(-Ms[c * kDeimMax + t], cv[t], x);
                const double d = Ms[c * kDeimMax + c];
                cv[c] = d != 0.0 ? x / d : 0.0;
            }
        }
        __syncthreads();
        double best = -1.0;
        int bidx = 0x7fffffff;
        for (int j = threadIdx.x; j < M; j += blockDim.x) {
            if (status[j] != 0) continue;
            double v = vl[j];
            for (int t = 0; t < l; ++t) v = fma(-cv[t], A[(long long)order[t] * M + j], v);
            const double av = fabs(v);
            if (av > best || (av == best && j < bidx)) { best = av; bidx = j; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
            if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
        }
        if ((threadIdx.x & 31) == 0) { bv[threadIdx.x >> 5] = best; bi[threadIdx.x >> 5] = bidx; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = -1.0;
            int ix = 0x7fffffff;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
                if (bv[w] > b || (bv[w] == b && bi[w] < ix)) { b = bv[w]; ix = bi[w]; }
            if (b >= 0.0) {
                pts[l] = ix;
                got_s = l + 1;
            }
        }
        __syncthreads();
        if (got_s <= l) break;                       // no unsampled angle left
    }
    if (threadIdx.x == 0) {
        for (int l = 0; l < got_s; ++l) a.st[I_NEW + l] = pts[l];
        a.st[I_NNEW] = got_s;
    }
}

// phi_old <- phi^{(n,k)} after a full check that did not stop the inner loop
__global__ void full_update_old(LRArgs a) {
    pdl_entry();
    if (!gate(a.st, G_FULL)) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += gridDim.x * blockDim.x) a.phi_old[i] = a.phi_k[i];
}

// start of outer iteration n: clear the header and the per-angle state
__global__ void outer_begin(LRArgs a, int n) {
    pdl_entry();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < I_HDR + 2 * a.nang; i += gridDim.x * blockDim.x) {
        int v = 0;
        if (i >= I_HDR + a.nang) v = -1;           // col_of
        if (i == I_OUTER) v = n;
        a.st[i] = v;
    }
}

__global__ void force_full(LRArgs a) {
    pdl_entry();
    if (threadIdx.x == 0 && blockIdx.x == 0) a.st[I_FULL] = 1;
}

// ------------------------------------------------------------------ full QR of the basis
// The MGS-QR and QR basis updates of the ablation in Sec. 4.2 (Table 2) replace the incremental
// update by a full re-orthogonalisation X = Q T of the whole basis (shifted CholeskyQR3: G =
// X^T X, G (+ shift) = L L^T, X <- X L^{-T}, three times), after which the snapshot coefficients
// R <- L^T R (each pass) and every projected operator and Galerkin factor is rebuilt from scratch.

// G = X^T X for r columns (FP64), 32 x 32 tiles, one thread per entry
__global__ void __launch_bounds__(1024) gram_kernel(const double* __restrict__ X, int N, int r,
                                                    double* __restrict__ G) {
    pdl_entry();
    __shared__ double ti[32][33], tj[32][33];
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    double acc = 0.0;
    for (int n0 = 0; n0 < N; n0 += 32) {
        const int n = n0 + tx;                        // consecutive threads, consecutive rows
        ti[tx][ty] = (n < N && i0 + ty < r) ? X[(long long)(i0 + ty) * N + n] : 0.0;
        tj[tx][ty] = (n < N && j0 + ty < r) ? X[(long long)(j0 + ty) * N + n] : 0.0;
        __syncthreads();
#pragma unroll 8
        for (int m = 0; m < 32; ++m) acc = fma(ti[m][ty], tj[m][tx], acc);
        __syncthreads();
    }
    if (i0 + ty < r && j0 + tx < r) G[(long long)(j0 + tx) * r + i0 + ty] = acc;   // column-major
}

// Cholesky G + shift I = L L^T (column-major r x r, lower part written into L), then
// W = L^{-T} (column-major, W[k + r c] = (L^{-1})[c][k]).  One block.  shift_coef > 0 gives the
// shifted CholeskyQR of Fukaya, Kannan, Nakatsukasa, Yamamoto and Yanagisawa (2020):
// shift = shift_coef * trace(G) = 11 (N r + r (r + 1)) u ||X||_F^2, positive definite for any
// basis with cond(X) below about 1/u; the later unshifted passes restore orthonormality.
__global__ void __launch_bounds__(256) chol_inv_kernel(const double* __restrict__ G, int r, double* __restrict__ L,
                                                       double* __restrict__ W, int* st, double shift_coef) {
    pdl_entry();
    for (int t = threadIdx.x; t < r * r; t += blockDim.x) { L[t] = 0.0; W[t] = 0.0; }
    __shared__ double dk, shift;
    if (threadIdx.x == 0) {
        double tr = 0.0;
        for (int k = 0; k < r; ++k) tr += G[(long long)k * r + k];
        shift = shift_coef * tr;
    }
    __syncthreads();
    for (int k = 0; k < r; ++k) {
        if (threadIdx.x == 0) {
            double d = G[(long long)k * r + k] + shift;
            for (int j = 0; j < k; ++j) d = fma(-L[(long long)j * r + k], L[(long long)j * r + k], d);
            if (!(d > 0.0)) st[I_SING] = d == 0.0 ? 1 : 2;
            dk = d > 0.0 ? sqrt(d) : 1.0;
            L[(long long)k * r + k] = dk;
        }
        __syncthreads();
        for (int i = k + 1 + threadIdx.x; i < r; i += blockDim.x) {
            double v = G[(long long)k * r + i];
            for (int j = 0; j < k; ++j) v = fma(-L[(long long)j * r + i], L[(long long)j * r + k], v);
            L[(long long)k * r + i] = v / dk;
        }
        __syncthreads();
    }
    // column c of L^{-1} by forward substitution (one column per thread); W[i r + c] = L^{-1}(i, c),
    // i.e. W = L^{-T} column-major
    for (int c = threadIdx.x; c < r; c += blockDim.x) {
        for (int i = c; i < r; ++i) {
            double v = i == c ? 1.0 : 0.0;
            for (int j = c; j < i; ++j) v = fma(-L[(long long)j * r + i], W[(long long)j * r + c], v);
            W[(long long)i * r + c] = v / L[(long long)i * r + i];
        }
    }
}

// R[:, a] <- L^T R[:, a] for the r columns of R (upper triangular times upper triangular)
__global__ void rmul_kernel(const double* __restrict__ L, int r, double* __restrict__ R, int rc) {
    pdl_entry();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < r; t += gridDim.x * blockDim.x) {
        double* col = R + (long long)t * rc;
        for (int i = 0; i <= t; ++i) {              // row i of L^T R: sum_{k >= i} L[k][i] R[k][t]
            double v = 0.0;
            for (int k = i; k <= t; ++k) v = fma(L[(long long)i * r + k], col[k], v);
            col[i] = v;                             // rows below i are read before they change
        }
    }
}

// the border chain's view of the rank during the operator rebuild: r = k + 1, the newest
// column k appended
__global__ void set_rank_kernel(LRArgs a, int r, int active) {
    pdl_entry();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    a.st[I_R] = r;
    a.st[I_ACTIVE] = active;
    a.st[I_APPENDED] = active;
}

__global__ void set_r0_kernel(LRArgs a, int r0) {
    pdl_entry();
    if (threadIdx.x == 0 && blockIdx.x == 0) a.st[I_R0] = r0;
}

// ------------------------------------------------------------------ truncation SVD
// One-sided Jacobi on A = C^T (nang x r, column k = row k of C) with accumulated W (r x r):
// A W = U_A Sigma, so C = W Sigma U_A^T: the paper's U = W, V = U_A.  Cooperative kernel,
// round-robin pairing (r/2 disjoint pairs per step, one warp per pair).
struct SvdArgs {
    int m, n, rc, max_sweeps;
    double* A;      // [n][m] columns
    double* W;      // [n][n] columns
    int* flag;      // [max_sweeps] rotation counters
    double tol;
};

__global__ void svd_init(SvdArgs s, const double* __restrict__ C) {
    pdl_entry();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < s.n * s.m; t += gridDim.x * blockDim.x) {
        const int k = t / s.m, j = t % s.m;
        s.A[(long long)k * s.m + j] = C[(long long)j * s.rc + k];
    }
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < s.n * s.n; t += gridDim.x * blockDim.x)
        s.W[t] = (t / s.n == t % s.n) ? 1.0 : 0.0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < s.max_sweeps; t += gridDim.x * blockDim.x) s.flag[t] = 0;
}

__global__ void svd_jacobi(SvdArgs s) {
    pdl_entry();
    cg::grid_group grid = cg::this_grid();
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int n2 = s.n + (s.n & 1);              // pad to even with a dummy column
    for (int sweep = 0; sweep < s.max_sweeps; ++sweep) {
        for (int step = 0; step < n2 - 1; ++step) {
            for (int pr = gw; pr < n2 / 2; pr += nw) {
                // round-robin: position 0 fixed, others rotate
                int i0 = pr == 0 ? 0 : 1 + (pr - 1 + step) % (n2 - 1);
                int i1 = 1 + (n2 - 2 - pr + step) % (n2 - 1);
                int p = min(i0, i1), q = max(i0, i1);
                if (q >= s.n || p == q) continue;
                double* ap = s.A + (long long)p * s.m;
                double* aq = s.A + (long long)q * s.m;
                double al = 0, be = 0, ga = 0;
                for (int j = lane; j < s.m; j += 32) {
                    const double x = ap[j], y = aq[j];
                    al = fma(x, x, al); be = fma(y, y, be); ga = fma(x, y, ga);
                }
                al = warp_sum(al); be = warp_sum(be); ga = warp_sum(ga);
                if (fabs(ga) > s.tol * sqrt(al * be) && ga != 0.0) {
                    const double zeta = (be - al) / (2.0 * ga);
                    const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                    const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
                    for (int j = lane; j < s.m; j += 32) {
                        const double x = ap[j], y = aq[j];
                        ap[j] = c * x - sn * y;
                        aq[j] = sn * x + c * y;
                    }
                    double* wp = s.W + (long long)p * s.n;
                    double* wq = s.W + (long long)q * s.n;
                    for (int j = lane; j < s.n; j += 32) {
                        const double x = wp[j], y = wq[j];
                        wp[j] = c * x - sn * y;
                        wq[j] = sn * x + c * y;
                    }
                    if (lane == 0) atomicAdd(&s.flag[sweep], 1);
                }
            }
            grid.sync();
        }
        if (s.flag[sweep] == 0) break;
        grid.sync();
    }
}

__global__ void svd_norms(SvdArgs s, double* __restrict__ sig) {
    pdl_entry();
    const int lane = threadIdx.x & 31;
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= s.n) return;
    double v = 0.0;
    for (int j = lane; j < s.m; j += 32) v = fma(s.A[(long long)k * s.m + j], s.A[(long long)k * s.m + j], v);
    v = warp_sum(v);
    if (lane == 0) sig[k] = sqrt(v);
}

// fX[:, c] = X W[:, order[c]] for c < r'  (the truncated spatial factor X U)
__global__ void form_xu(const double* __restrict__ X, int N, int r, const double* __restrict__ W, int n,
                        const int* __restrict__ order, int rp, double* __restrict__ out) {
    pdl_entry();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        for (int c = 0; c < rp; ++c) {
            const double* wc = W + (long long)order[c] * n;
            double s = 0.0;
            for (int k = 0; k < r; ++k) s = fma(X[(long long)k * N + i], wc[k], s);
            out[(long long)c * N + i] = s;
        }
}

__global__ void form_v(const double* __restrict__ A, int m, const int* __restrict__ order, const double* __restrict__ sig,
                       int rp, double* __restrict__ V, double* __restrict__ S) {
    pdl_entry();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < rp * m; t += gridDim.x * blockDim.x) {
        const int c = t / m, j = t % m;
        const double sv = sig[order[c]];
        V[(long long)c * m + j] = sv > 0 ? A[(long long)order[c] * m + j] / sv : 0.0;
        if (j == 0) S[c] = sv;
    }
}

// ====================================================================== host side
static int egrid(const rte_handle* h, long long n) {
    long long g = (n + 255) / 256;
    return (int)std::max(1ll, std::min(g, (long long)std::max(h->num_sms, 1) * 8));
}

static int lr_allocate(rte_handle* h) {
    LowRankState& L = h->lr;
    if (L.X) return RTE_OK;
    const int ndir = (int)h->fold_rep.size();
    const int rc = std::min(ndir, h->ndof);
    L.r_cap = rc;
    L.n_dir = ndir;
    const size_t N = h->ndof, R = rc, M = h->nang;
    auto A = [&](void** p, size_t n) { return h->arena.alloc(p, n); };
    RTE_TRY(A((void**)&L.X, 8 * N * R));
    RTE_TRY(A((void**)&L.R, 8 * R * R));
    RTE_TRY(A((void**)&L.Pxm, 8 * R * R));
    RTE_TRY(A((void**)&L.Pym, 8 * R * R));
    RTE_TRY(A((void**)&L.T, 8 * R * R));
    RTE_TRY(A((void**)&L.bS, 8 * R));
    RTE_TRY(A((void**)&L.bE, 8 * 4 * R));
    RTE_TRY(A((void**)&L.LUl, 8 * (size_t)ndir * R * R));
    RTE_TRY(A((void**)&L.LUu, 8 * (size_t)ndir * R * R));
    RTE_TRY(A((void**)&L.Udinv, 8 * (size_t)ndir * R));
    RTE_TRY(A((void**)&L.Y, 8 * (size_t)ndir * R));
    RTE_TRY(A((void**)&L.Cdir, 8 * (size_t)ndir * R));
    RTE_TRY(A((void**)&L.W, 8 * 5 * N));
    RTE_TRY(A((void**)&L.snap, 8 * 64 * N));
    RTE_TRY(A((void**)&L.vcand, 8 * 64 * N));
    L.vcand_bytes = 8 * 64 * N;
    RTE_TRY(A((void**)&L.X2, 8 * N * R));
    RTE_TRY(A((void**)&L.S2, 8 * N));
    RTE_TRY(A((void**)&L.E2, 8 * 4 * N));
    RTE_TRY(A((void**)&L.ccand2, 8 * 64 * R));
    L.ccand2_bytes = 8 * 64 * R;
    RTE_TRY(A((void**)&L.small, 8 * (size_t)SmallLayout{rc}.total()));
    RTE_TRY(A((void**)&L.ints, sizeof(int) * (I_HDR + 2 * M + R + 64 + kCandMax)));
    RTE_TRY(A((void**)&L.phi_old, 8 * N));
    RTE_TRY(A((void**)&L.phi_k, 8 * N));
    RTE_TRY(A((void**)&L.Cfull, 8 * R * M));
    RTE_TRY(A((void**)&L.svd_A, 8 * R * M));
    RTE_TRY(A((void**)&L.svd_W, 8 * R * R));
    RTE_TRY(A((void**)&L.svd_s, 8 * R));
    if (pinned_alloc((void**)&L.host_ints, sizeof(int) * 256) != cudaSuccess ||
        pinned_alloc((void**)&L.host_small, sizeof(double) * 64) != cudaSuccess) {
        cudaGetLastError();
        return fail(RTE_ERR_NOMEM, "low-rank: pinned allocation failed");
    }
    return RTE_OK;
}

// One-sided Jacobi SVD of the full check's C (r x nang): svd_A <- sigma_k v_k, svd_W <- U,
// svd_s <- sigma_k (unsorted).  flag: [40] device rotation counters.
static int svd_of_c(rte_handle* h, int r, int* flag, cudaStream_t st) {
    LowRankState& L = h->lr;
    SvdArgs sa;
    sa.m = h->nang;
    sa.n = r;
    sa.rc = L.r_cap;
    sa.max_sweeps = 40;
    sa.A = L.svd_A;
    sa.W = L.svd_W;
    sa.tol = 1e-15;
    sa.flag = flag;
    svd_init<<<egrid(h, (long long)r * h->nang), 256, 0, st>>>(sa, L.Cfull);
    RTE_CUDA_TRY(cudaGetLastError());
    const int pairs = (r + 1) / 2;
    int blocks = std::max(1, (pairs * 32 + 255) / 256);
    int per_sm = 0;
    RTE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, svd_jacobi, 256, 0));
    blocks = std::min(blocks, std::max(1, per_sm) * std::max(1, h->num_sms));
    void* args[] = {&sa};
    if (r > 1) RTE_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)svd_jacobi, dim3(blocks), dim3(256), args, 0, st));
    svd_norms<<<(r * 32 + 255) / 256, 256, 0, st>>>(sa, L.svd_s);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

// Truncated SVD of C (r x nang) after an inner loop; fills the factors when asked.
static int truncate_c(rte_handle* h, const rte_opts* o, int r, int* rank_out, bool form_factors, cudaStream_t st) {
    LowRankState& L = h->lr;
    const int M = h->nang;
    SvdArgs sa;
    sa.m = M;
    sa.n = r;
    sa.rc = L.r_cap;
    sa.max_sweeps = 40;
    sa.A = L.svd_A;
    sa.W = L.svd_W;
    sa.tol = 1e-15;
    int* flag = nullptr;
    RTE_TRY(h->arena.alloc((void**)&flag, sizeof(int) * 64));
    sa.flag = flag;
    svd_init<<<egrid(h, (long long)r * M), 256, 0, st>>>(sa, L.Cfull);
    RTE_CUDA_TRY(cudaGetLastError());
    const int pairs = (r + 1) / 2;
    int blocks = std::max(1, (pairs * 32 + 255) / 256);
    int per_sm = 0;
    RTE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, svd_jacobi, 256, 0));
    blocks = std::min(blocks, std::max(1, per_sm) * std::max(1, h->num_sms));
    void* args[] = {&sa};
    if (r > 1) RTE_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)svd_jacobi, dim3(blocks), dim3(256), args, 0, st));
    svd_norms<<<(r * 32 + 255) / 256, 256, 0, st>>>(sa, L.svd_s);
    RTE_CUDA_TRY(cudaGetLastError());
    std::vector<double> sig(r);
    RTE_CUDA_TRY(cudaMemcpyAsync(sig.data(), L.svd_s, sizeof(double) * r, cudaMemcpyDeviceToHost, st));
    RTE_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<int> order(r);
    for (int k = 0; k < r; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return sig[x] > sig[y]; });
    double total = 0.0;
    for (double v : sig) total += v;
    int rp = r;
    if (total > 0) {
        double cum = 0.0;
        for (int k = 0; k < r; ++k) {
            cum += sig[order[k]];
            if ((total - cum) / total <= o->eps_svd) { rp = k + 1; break; }
        }
    }
    *rank_out = rp;
    if (form_factors) {
        if (!L.fX) {
            RTE_TRY(h->arena.alloc((void**)&L.fX, sizeof(double) * (size_t)h->ndof * L.r_cap));
            RTE_TRY(h->arena.alloc((void**)&L.fS, sizeof(double) * L.r_cap));
            RTE_TRY(h->arena.alloc((void**)&L.fV, sizeof(double) * (size_t)M * L.r_cap));
        }
        int* d_order = nullptr;
        RTE_TRY(h->arena.alloc((void**)&d_order, sizeof(int) * r));
        RTE_CUDA_TRY(cudaMemcpyAsync(d_order, order.data(), sizeof(int) * r, cudaMemcpyHostToDevice, st));
        form_xu<<<egrid(h, h->ndof), 256, 0, st>>>(L.X, h->ndof, r, L.svd_W, r, d_order, rp, L.fX);
        form_v<<<egrid(h, (long long)rp * M), 256, 0, st>>>(L.svd_A, M, d_order, L.svd_s, rp, L.fV, L.fS);
        RTE_CUDA_TRY(cudaGetLastError());
        RTE_CUDA_TRY(cudaStreamSynchronize(st));
        L.factor_rank = rp;
        auto& v = h->arena.ptrs;
        v.erase(std::remove(v.begin(), v.end(), (void*)d_order), v.end());
        dev_free(d_order);
    }
    RTE_CUDA_TRY(cudaStreamSynchronize(st));
    auto& v = h->arena.ptrs;
    v.erase(std::remove(v.begin(), v.end(), (void*)flag), v.end());
    dev_free(flag);
    return RTE_OK;
}

// shared memory: lu_border (2 chunk + 2 x nw warps x kDq) rc, cand_solve (1 + kDq) rc, full_solve 2 warps x (1 + kDq) rc
constexpr size_t kGalerkinSmemMax = 227 * 1024;
static size_t border_smem(int nw, int rc) { return sizeof(double) * (2 * kBorderChunk + 2 * nw * kDq) * (size_t)rc; }
// warps per side of lu_border: the most (up to kBorderWarps) whose staging rings fit
static int border_warps(int rc) {
    int nw = kBorderWarps;
    while (nw > 1 && border_smem(nw, rc) > kGalerkinSmemMax) nw >>= 1;
    return nw;
}
static void launch_galerkin(int /*unused*/, int which, const LRArgs& a, int ndir, int rc, int q, cudaStream_t st) {
    if (which == 0) {
        const int nw = border_warps(rc);
        lu_border<<<ndir, 64 * nw, border_smem(nw, rc), st>>>(a);
    } else if (which == 1) cand_solve<<<q, 32, sizeof(double) * (1 + kDq) * rc, st>>>(a);
    else full_solve<<<(ndir + 1) / 2, 64, sizeof(double) * 2 * (1 + kDq) * rc, st>>>(a);
}

static int galerkin_smem_setup(int rc) {
    const size_t s0 = border_smem(border_warps(rc), rc),
                 s1 = sizeof(double) * (1 + kDq) * rc,
                 s2 = sizeof(double) * 2 * (1 + kDq) * rc;
    if (s0 > kGalerkinSmemMax || s2 > kGalerkinSmemMax)
        return fail(RTE_ERR_ARG, "low-rank: basis capacity too large for the Galerkin kernels' shared memory");
    RTE_TRY(smem_optin(lu_border, s0));
    RTE_TRY(smem_optin(cand_solve, s1));
    RTE_TRY(smem_optin(full_solve, s2));
    return RTE_OK;
}

// Turn every kernel-to-kernel edge of a captured graph into a programmatic dependency: the
// downstream kernel is launched as the upstream one's blocks pass pdl_entry and waits there for
// the upstream's completion (memory visible).  Edges touching other node types stay as they are.
static int make_edges_programmatic(cudaGraph_t g) {
    size_t ne = 0;
    RTE_CUDA_TRY(cudaGraphGetEdges(g, nullptr, nullptr, nullptr, &ne));
    if (!ne) return RTE_OK;
    std::vector<cudaGraphNode_t> from(ne), to(ne);
    std::vector<cudaGraphEdgeData> ed(ne);
    RTE_CUDA_TRY(cudaGraphGetEdges(g, from.data(), to.data(), ed.data(), &ne));
    for (size_t e = 0; e < ne; ++e) {
        cudaGraphNodeType tf, tt;
        RTE_CUDA_TRY(cudaGraphNodeGetType(from[e], &tf));
        RTE_CUDA_TRY(cudaGraphNodeGetType(to[e], &tt));
        if (tf != cudaGraphNodeTypeKernel || tt != cudaGraphNodeTypeKernel || ed[e].type != cudaGraphDependencyTypeDefault ||
            ed[e].from_port != cudaGraphKernelNodePortDefault)
            continue;
        RTE_CUDA_TRY(cudaGraphRemoveDependencies(g, &from[e], &to[e], &ed[e], 1));
        cudaGraphEdgeData pe_ = {};
        pe_.from_port = cudaGraphKernelNodePortProgrammatic;
        pe_.type = cudaGraphDependencyTypeProgrammatic;
        RTE_CUDA_TRY(cudaGraphAddDependencies(g, &from[e], &to[e], &pe_, 1));
    }
    return RTE_OK;
}

int solve_low_rank(rte_handle* h, const rte_opts* o, double* phi, rte_stats* s, const double* F, double* psi_next) {
    if (o->p < 1 || o->p > 64 || o->q < 1) return fail(RTE_ERR_ARG, "need 1 <= p <= 64 and q >= 1");
    if (F && ((o->sweep_precision == RTE_FP32 && o->sweep_refine) || o->tc_projection ||
              o->sampling != RTE_SAMPLE_RESIDUAL || o->basis_update != RTE_UPDATE_MGS2A))
        return fail(RTE_ERR_ARG, "low-rank time step: residual sampling, MGS2-A, no tensor-core projection, and "
                                 "FP32 sweeps without the defect correction");
    RTE_TRY(lr_allocate(h));
    LowRankState& Ls = h->lr;
    {
        // candidate vectors and coefficients for up to min(q, N_Omega) candidates per inner
        // iteration (q >= the unsampled count: every unsampled angle, the fully greedy variant)
        const size_t qeff = (size_t)std::min(std::min(o->q, h->nang), kCandMax);
        RTE_TRY(h->arena.grow(&Ls.vcand_void(), &Ls.vcand_bytes, 8 * qeff * (size_t)h->ndof));
        RTE_TRY(h->arena.grow(&Ls.ccand2_void(), &Ls.ccand2_bytes, 8 * qeff * (size_t)Ls.r_cap));
    }
    Ls.factor_rank = 0;
    Ls.last_rank = 0;
    cudaStream_t st = h->stream;
    // the p-ordinate sweeps of the inner loop run inside graph captures: tune them now
    RTE_TRY(sweep_pretune(h, o->sweep_precision == RTE_FP32 ? RTE_FP32 : RTE_FP64, o->p, 1, st));
    const int N = h->ndof, M = h->nang, rc = Ls.r_cap, ndir = Ls.n_dir, p = o->p;
    const int q = std::min(o->q, std::min(M, kCandMax));   // candidates beyond N_Omega never exist
    if (rc > 512) return fail(RTE_ERR_ARG, "low-rank: at most 512 distinct directions");
    const int mt = (rc + 31) / 32;
    const int prec = o->sweep_precision == RTE_FP32 ? RTE_FP32 : RTE_FP64;
    const int refine = prec == RTE_FP32 && o->sweep_refine ? 1 : 0;
    const size_t esz = prec == RTE_FP32 ? 4 : 8;
    std::vector<int> dir_of(M), dir_rep(ndir);
    for (int d = 0; d < ndir; ++d) {
        dir_rep[d] = h->fold_rep[d];
        dir_of[h->fold_rep[d]] = d;
        dir_of[h->twin[h->fold_rep[d]]] = d;
    }
    const int nblk_x = (N + kXtRows - 1) / kXtRows;
    // row blocks of the tensor-core first projection (smaller blocks than the CUDA-core pass:
    // its CTAs only stream two tiles per stage through the tensor cores)
    constexpr int kTcRows = 256;
    const int nblk_tc = (N + kTcRows - 1) / kTcRows;
    const int nblk_d = std::min(egrid(h, N), 1024);
    const int nblk_res = std::min(egrid(h, h->nc), 512);
    // fused pass + X^T v (double-word chain): rows per block so that the grid is at most one
    // wave of two blocks per SM (32-row groups); its partials share xpart and npart with xt_dw
    // resident blocks per SM: two of 8 warps (rc <= 128), one of 16 warps (rc <= 256; 16 columns
    // per warp either way, so about 128 registers per thread)
    const int fz_slots = (rc <= 128 ? 2 : 1) * std::max(1, h->num_sms);
    const int fz_groups = std::max(1, ((N + 31) / 32 + fz_slots - 1) / fz_slots);
    const int fz_rows = 32 * fz_groups;
    const int fz_blocks = (N + fz_rows - 1) / fz_rows;
    const size_t red_len = std::max({(size_t)nblk_x * kXtV * rc, (size_t)nblk_tc * kXtV * rc,
                                     (size_t)fz_blocks * kXtV * rc,
                                     (size_t)std::max(64, std::min(q, M)) * nblk_res});
    int *d_dir_of = nullptr, *d_dir_rep = nullptr, *d_twin = nullptr;
    double *S64 = nullptr, *v = nullptr, *part = nullptr, *red = nullptr, *xpart = nullptr, *npart = nullptr;
    double *xpart_b = nullptr, *bpart = nullptr;      // scratch of the border branch
    double *dcall = nullptr, *psn = nullptr;          // X^T psi_l (columns at the start) and ||psi_l||
    double* opart = nullptr;                          // snap_open's chunk partials [64][kOpenChunks]
    // part holds 8 doubles per block of the grid-stride passes (up to egrid blocks) and of
    // the 1024-block reductions
    const int sten_blocks = std::min((h->nc + 63) / 64, 16 * std::max(1, h->num_sms));   // 64-thread blocks
    const size_t part_len = 8 * (size_t)std::max({egrid(h, N), egrid(h, h->nc), sten_blocks, 1024});
    std::vector<void*> call_allocs;
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    auto A = [&](void** ptr, size_t n) {
        int rc_ = h->arena.alloc(ptr, n);
        if (rc_ == RTE_OK) call_allocs.push_back(*ptr);
        return rc_;
    };
    auto release = [&]() {
        cudaStreamSynchronize(st);
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        gexec = nullptr;
        graph = nullptr;
        for (void* ptr : call_allocs) {
            auto& vv = h->arena.ptrs;
            vv.erase(std::remove(vv.begin(), vv.end(), ptr), vv.end());
            dev_free(ptr);
        }
        call_allocs.clear();
    };
#define LR_TRY(expr) do { int _s = (expr); if (_s != RTE_OK) { release(); return _s; } } while (0)
#define LR_CUDA(expr) do { cudaError_t _e = (expr); if (_e != cudaSuccess) { release(); return fail(RTE_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); } } while (0)
    LR_TRY(A((void**)&d_dir_of, sizeof(int) * M));
    LR_TRY(A((void**)&d_dir_rep, sizeof(int) * ndir));
    LR_TRY(A((void**)&d_twin, sizeof(int) * M));
    LR_TRY(A((void**)&S64, sizeof(double) * N));
    LR_TRY(A((void**)&v, sizeof(double) * N));
    LR_TRY(A((void**)&part, sizeof(double) * part_len));
    LR_TRY(A((void**)&npart, sizeof(double) * kXtV * std::max({nblk_x, nblk_tc, fz_blocks})));
    LR_TRY(A((void**)&xpart_b, sizeof(double) * (size_t)nblk_x * kXtV * rc));
    LR_TRY(A((void**)&dcall, sizeof(double) * 64 * (size_t)rc));
    LR_TRY(A((void**)&psn, sizeof(double) * 64));
    LR_TRY(A((void**)&opart, sizeof(double) * 64 * kOpenChunks));
    LR_TRY(A((void**)&bpart, sizeof(double) * 8 * (size_t)sten_blocks));
    LR_TRY(A((void**)&red, sizeof(double) * (size_t)std::max(64, std::min(q, M)) * nblk_res));
    LR_TRY(A((void**)&xpart, sizeof(double) * red_len));
    LR_CUDA(cudaMemcpyAsync(d_dir_of, dir_of.data(), sizeof(int) * M, cudaMemcpyHostToDevice, st));
    LR_CUDA(cudaMemcpyAsync(d_dir_rep, dir_rep.data(), sizeof(int) * ndir, cudaMemcpyHostToDevice, st));
    LR_CUDA(cudaMemcpyAsync(d_twin, h->twin.data(), sizeof(int) * M, cudaMemcpyHostToDevice, st));
    LR_TRY(ensure_psi_scratch(h, esz * (size_t)p * N));
    if (refine) LR_TRY(ensure_refine_scratch(h, p));
    LR_CUDA(cudaStreamSynchronize(st));            // host tables above are temporaries

    LRArgs a;
    memset(&a, 0, sizeof(a));
    a.nx = h->nx; a.ny = h->ny; a.nc = h->nc; a.N = N; a.nang = M; a.rc = rc; a.ndir = ndir;
    a.p = p; a.q = q; a.hx = h->hx; a.hy = h->hy; a.ihx = 1.0 / h->hx; a.ihy = 1.0 / h->hy;
    for (int k = 0; k < 4; ++k) a.g[k] = h->inflow[k];
    a.ox = h->d_ox; a.oy = h->d_oy; a.w = h->d_w;
    a.dir_of = d_dir_of; a.dir_rep = d_dir_rep; a.twin = d_twin;
    a.sig_t = h->sig_t; a.e_side = h->e_side; a.S = S64;
    // backward-Euler time source (Sec. 3.7): F, its products with the basis columns, per-slot sweep
    // sources
    double *bF = nullptr, *fpart = nullptr;
    void* src_pa = nullptr;
    const int nblk_f = (N + 1023) / 1024;
    if (F) {
        LR_TRY(A((void**)&bF, sizeof(double) * (size_t)ndir * rc));
        LR_TRY(A((void**)&fpart, sizeof(double) * (size_t)nblk_f * ndir));
        LR_TRY(A(&src_pa, esz * (size_t)p * N));
    }
    a.F = F;
    a.bF = bF;
    auto fsrc_dots = [&](int gm, int rsel, cudaStream_t sx) {
        if (!F) return;
        fsrc_dots_partial<<<dim3(nblk_f, (ndir + 7) / 8), 256, 0, sx>>>(a, gm, rsel, fpart);
        fsrc_dots_final<<<(ndir + 7) / 8, 256, 0, sx>>>(a, gm, rsel, fpart, nblk_f);
    };
    a.X = Ls.X; a.R = Ls.R; a.Pxm = Ls.Pxm; a.Pym = Ls.Pym; a.T = Ls.T; a.bS = Ls.bS; a.bE = Ls.bE;
    a.Lf = Ls.LUl; a.Uf = Ls.LUu; a.Udinv = Ls.Udinv; a.Y = Ls.Y; a.Cdir = Ls.Cdir; a.W = Ls.W;
    a.vcand = Ls.vcand; a.red = red; a.sm = Ls.small; a.st = Ls.ints; a.phi_old = Ls.phi_old;
    a.phi_k = Ls.phi_k; a.Cfull = Ls.Cfull;
    const bool dwb = o->basis_precision == RTE_DWF32;
    a.dwb = dwb ? 1 : 0; a.X2 = Ls.X2; a.S2 = Ls.S2; a.ccand2 = Ls.ccand2;
    a.sig_h = h->sig_dw; a.sig_l = h->sig_dw + h->nc;
    a.eps_mgs = o->eps_mgs; a.eps_break = o->eps_break; a.eps_res = o->eps_res; a.eps_diff = o->eps_diff;
    a.m_max = o->m_max; a.mgs_test = o->mgs_test; a.max_inner = o->max_inner; a.seed = o->seed;
    const SmallLayout SL{rc};
    double* sc = Ls.small + SL.scal();
    int* ints = Ls.ints;
    const int g = egrid(h, N);
    const size_t xsm = sizeof(double) * (size_t)5 * kXtRows;
    LR_TRY(smem_optin(xt_partial, xsm));
    LR_TRY(smem_optin(xt_dw, sizeof(float2) * kXtV * kXtRows));
    if (sizeof(float2) * kXtJ * rc > 48 * 1024)
        LR_TRY(smem_optin(x_times_dw, sizeof(float2) * kXtJ * rc));
    const size_t xtsm = sizeof(double) * (size_t)std::min(q, kXtChunk) * rc;
    if (xtsm > 48 * 1024) {
        LR_TRY(smem_optin(x_times, xtsm));
    }
    const size_t dsm = sizeof(unsigned long long) * M;
    LR_TRY(galerkin_smem_setup(rc));
    LR_TRY(smem_optin(draw_kernel, dsm));

    cudaStream_t cs_ = st;    // stream the body launches into (a private one while capturing)
    int r_host = 0;    // rank at the last read-back (profiler byte counts only)
    auto pb = [&](int cls) { RTE_PROF_BEGIN(h, cls, cs_); };
    auto pe = [&](int cls, double by, double fl) { RTE_PROF_END(h, cls, cs_, by, fl); };
    // FP64 chain
    auto xt = [&](const double* V, int nv, long long vstride, double* out, int gm) {
        pb(RTE_PROF_BASIS);
        xt_partial<<<dim3(nblk_x, (rc + 7) / 8), 256, sizeof(double) * (size_t)nv * kXtRows, cs_>>>(
            Ls.X, N, ints, gm, V, nv, vstride, xpart, rc);
        xt_final<<<dim3((rc + 7) / 8, nv), 256, 0, cs_>>>(xpart, nblk_x, ints, gm, nv, rc, out);
        pe(RTE_PROF_BASIS, 8.0 * N * (r_host + nv), 2.0 * N * r_host * nv);
    };
    auto xpass = [&](int gm, int first, int scale_alpha) {
        pb(RTE_PROF_BASIS);
        mgs_pass<<<g, 256, sizeof(double) * rc, cs_>>>(a, gm, first, scale_alpha, v, part);
        pe(RTE_PROF_BASIS, 8.0 * N * (r_host + 2), 2.0 * N * r_host);
    };
    auto norm_into = [&](const double* x, int gm, double* out) {
        sumsq_partial<<<nblk_d, 256, 0, cs_>>>(N, x, part, ints, gm);
        finalize_sums<<<1, 32, 0, cs_>>>(part, nblk_d, 1, ints, gm, out, 1);
    };
    // double-word chain (X2, the snapshots, v and W hold double-words: same 8 bytes per entry)
    float2* const v2 = reinterpret_cast<float2*>(v);
    auto xtd = [&](const float2* V, int nv, long long vstride, double* out, int gm, double* nrm_out) {
        pb(RTE_PROF_BASIS);
        xt_dw<<<dim3(nblk_x, (rc + 7) / 8), 256, sizeof(float2) * (size_t)nv * kXtRows, cs_>>>(
            Ls.X2, N, ints, gm, V, nv, vstride, xpart, rc, nrm_out ? npart : nullptr, -1);
        if (nv == 1)
            mgs_dots_final<<<(rc + 7) / 8 + 1, 256, 0, cs_>>>(xpart, npart, nblk_x, rc, ints, gm, out, nrm_out);
        else
            xt_final<<<dim3((rc + 7) / 8, nv), 256, 0, cs_>>>(xpart, nblk_x, ints, gm, nv, rc, out, -1, kXtV);
        pe(RTE_PROF_BASIS, 8.0 * N * (r_host + nv), 2.0 * N * r_host * nv);
    };
    auto passd = [&](int gm, int first, const float2* vin, double* alpha_out) {
        pb(RTE_PROF_BASIS);
        mgs_pass_dw<<<g, 256, sizeof(float2) * rc, cs_>>>(a, gm, first, vin, v2, part, ints + I_CNT_PASS, alpha_out);
        pe(RTE_PROF_BASIS, 8.0 * N * (r_host + 2), 2.0 * N * r_host);
    };
    const bool fused = rc <= 256;           // register-resident products for r <= 256
    // tensor-core first projection: double-word chain with the fused passes (its partials feed
    // the same reductions as the double-word first products)
    const bool use_tc = o->tc_projection && dwb && fused;
    const bool deim = o->sampling == RTE_SAMPLE_DEIM;
    int* svd_flag = nullptr;
    if (deim) LR_TRY(A((void**)&svd_flag, sizeof(int) * 64));
    // basis update of the ablation in Sec. 4.2: one projection per snapshot, full QR of the basis
    // on a failed test (MGS-QR) or after every inner iteration (QR); FP64 basis passes only
    const int bu = o->basis_update;
    const bool bu_qr = bu != RTE_UPDATE_MGS2A;
    if (bu_qr && dwb) LR_TRY(fail(RTE_ERR_ARG, "basis_update MGS-QR / QR needs basis_precision = RTE_FP64"));
    const int n_mand = bu_qr ? 1 : 2;          // mandatory projections per snapshot
    const int m_max_eff = bu_qr ? 0 : o->m_max;
    a.m_max = m_max_eff;
    double *qr_G = nullptr, *qr_L = nullptr, *qr_W = nullptr, *qr_X = nullptr;
    int* qr_iota = nullptr;
    int full_qr_count = 0;
    if (bu_qr) {
        LR_TRY(A((void**)&qr_G, sizeof(double) * (size_t)rc * rc));
        LR_TRY(A((void**)&qr_L, sizeof(double) * (size_t)rc * rc));
        LR_TRY(A((void**)&qr_W, sizeof(double) * (size_t)rc * rc));
        LR_TRY(A((void**)&qr_X, sizeof(double) * (size_t)N * rc));
        LR_TRY(A((void**)&qr_iota, sizeof(int) * rc));
        std::vector<int> io(rc);
        for (int k = 0; k < rc; ++k) io[k] = k;
        LR_CUDA(cudaMemcpyAsync(qr_iota, io.data(), sizeof(int) * rc, cudaMemcpyHostToDevice, st));
        LR_CUDA(cudaStreamSynchronize(st));
    }
    if (o->tc_projection && !use_tc)
        LR_TRY(fail(RTE_ERR_ARG, "tc_projection needs basis_precision = RTE_DWF32 and at most 256 distinct directions"));
    a.Xt = a.Xl = nullptr;
    if (use_tc) {
        if (!Ls.Xt) {
            LR_TRY(h->arena.alloc((void**)&Ls.Xt, sizeof(float) * (size_t)N * rc));
            LR_TRY(h->arena.alloc((void**)&Ls.Xl, sizeof(float) * (size_t)N * rc));
            LR_TRY(h->arena.alloc((void**)&Ls.snap_t, sizeof(float) * 64 * (size_t)N));
            LR_TRY(h->arena.alloc((void**)&Ls.snap_l, sizeof(float) * 64 * (size_t)N));
        }
        if (!Ls.tc.ready) LR_TRY(tc_projection_prepare(&Ls.tc, Ls.Xt, Ls.Xl, N, rc, Ls.snap_t, Ls.snap_l, 64));
        a.Xt = Ls.Xt;
        a.Xl = Ls.Xl;
    }
    // Full QR of the basis and a rebuild of every projected operator (MGS-QR / QR ablation): the
    // basis columns, R, then the border of each column k in turn with the chain's rank set to
    // k + 1; the Galerkin factors are re-bordered from column 0 at this inner iteration's LU step.
    // Uncaptured only (the rank is read back).
    std::function<int()> full_qr_rebuild = [&]() -> int {
        int r_now = 0;
        LR_CUDA(cudaMemcpyAsync(&r_now, ints + I_R, sizeof(int), cudaMemcpyDeviceToHost, st));
        LR_CUDA(cudaStreamSynchronize(st));
        if (r_now <= 0) return RTE_OK;
        const int tiles = (r_now + 31) / 32;
        // shifted CholeskyQR3: a shifted pass (robust to the nearly dependent columns a single
        // projection can leave), then two plain passes
        const double u = 1.1102230246251565e-16;
        const double shift_coef = 11.0 * ((double)N * r_now + (double)r_now * (r_now + 1)) * u;
        for (int pass = 0; pass < 3; ++pass) {
            gram_kernel<<<dim3(tiles, tiles), dim3(32, 32), 0, st>>>(Ls.X, N, r_now, qr_G);
            chol_inv_kernel<<<1, 256, 0, st>>>(qr_G, r_now, qr_L, qr_W, ints, pass == 0 ? shift_coef : 0.0);
            form_xu<<<g, 256, 0, st>>>(Ls.X, N, r_now, qr_W, r_now, qr_iota, r_now, qr_X);
            LR_CUDA(cudaMemcpyAsync(Ls.X, qr_X, sizeof(double) * (size_t)N * r_now, cudaMemcpyDeviceToDevice, st));
            rmul_kernel<<<(r_now + 127) / 128, 128, 0, st>>>(qr_L, r_now, Ls.R, rc);
        }
        for (int k = 0; k < r_now; ++k) {
            set_rank_kernel<<<1, 32, 0, st>>>(a, k + 1, 1);
            border_stencil<<<egrid(h, h->nc), 256, 0, st>>>(a, G_APP, -1);
            xt(Ls.W, 5, N, Ls.small + SL.border(), G_APP);
            newcol_dots_partial<<<nblk_d, 256, 0, st>>>(a, part);
            finalize_sums<<<1, 160, 0, st>>>(part, nblk_d, 5, ints, G_APP, Ls.small + SL.dots(), 0);
            border_write<<<1, 256, 0, st>>>(a, G_APP, -1);
        }
        set_rank_kernel<<<1, 32, 0, st>>>(a, r_now, 1);
        set_r0_kernel<<<1, 32, 0, st>>>(a, 0);
        LR_CUDA(cudaGetLastError());
        ++full_qr_count;
        return RTE_OK;
    };
    auto passxt = [&](int gm, int first, const float2* vin, double* alpha_out, const double* dcall_l,
                      cudaGraphConditionalHandle hc = 0, int slot = -1) {
        // algorithmic traffic: X (8 N r bytes, double-words) once, v in and out; 2 double-word
        // multiply-adds per X entry counted as the 4 flops of the FP64 operations they replace
        pb(RTE_PROF_PASS);
        if (rc <= 128)
            mgs_pass_xt_dw<16, 8><<<fz_blocks, 256, sizeof(float2) * rc, cs_>>>(a, gm, first, vin, v2, xpart, npart, fz_rows,
                                                                             dcall_l, opart, kOpenChunks);
        else
            mgs_pass_xt_dw<16, 16><<<fz_blocks, 512, sizeof(float2) * rc, cs_>>>(a, gm, first, vin, v2, xpart, npart, fz_rows,
                                                                             dcall_l, opart, kOpenChunks);
        pe(RTE_PROF_PASS, 8.0 * N * (r_host + 2), 4.0 * N * r_host);
        pb(RTE_PROF_BASIS);
        if (hc)          // the test of Alg. 2 in the same launch (captured graph, alpha_out = S_ALPHA)
            mgs_final_test<<<(rc + 7) / 8 + 1, 256, 0, cs_>>>(a, xpart, npart, fz_blocks, gm, ints + I_CNT_FIN, hc,
                                                              slot);
        else
            mgs_dots_final<<<(rc + 7) / 8 + 1, 256, 0, cs_>>>(xpart, npart, fz_blocks, rc, ints, gm, Ls.small + SL.dc(),
                                                              alpha_out);
        pe(RTE_PROF_BASIS, 8.0 * fz_blocks * r_host, 1.0 * fz_blocks * r_host);
    };
    const void* src_sweep = prec == RTE_FP32 ? h->src_w : (const void*)S64;
    void* out_sweep = prec == RTE_FP32 ? h->psi_w : (void*)Ls.snap;

    // one inner iteration, every launch gated on the device state (capturable)
    bool capturing = false;   // body() is being captured into the inner-iteration graph
    std::vector<cudaGraph_t> cond_bodies;                   // bodies of the captured WHILE nodes
    auto body = [&]() -> int {
        bool forked = false;
        if (capturing && dwb && !h->border_stream) {
            LR_CUDA(cudaStreamCreateWithFlags(&h->border_stream, cudaStreamNonBlocking));
            LR_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
            LR_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
        }
        iter_begin<<<1, 32, 0, cs_>>>(a);
        void* dpsi = nullptr;
        if (F) {                  // per-slot sources S + F of the sampled directions (no defect correction)
            if (prec == RTE_FP32) fsrc_sweep_source<float><<<g, 256, 0, cs_>>>(a, p, (float*)src_pa);
            else fsrc_sweep_source<double><<<g, 256, 0, cs_>>>(a, p, (double*)src_pa);
            LR_CUDA(cudaGetLastError());
            RTE_TRY(launch_sweep(h, ints + I_NEW, p, prec, src_pa, N, 1, 0, out_sweep, cs_, ints + I_NNEW));
        } else {
            RTE_TRY(sweep_refined(h, ints + I_NEW, p, prec, refine, src_sweep, S64, 1, 0, out_sweep, &dpsi,
                                  ints + I_NNEW, cs_));
        }
        float2* snap2 = reinterpret_cast<float2*>(Ls.snap);
        if (prec == RTE_FP32 && dwb)
            to_dw_snap<float><<<g, 256, 0, cs_>>>(N, ints + I_NNEW, (const float*)h->psi_w, (const float*)dpsi, snap2,
                                                   use_tc ? Ls.snap_t : nullptr, Ls.snap_l);
        else if (prec == RTE_FP32)
            to_double2_g<float><<<g, 256, 0, cs_>>>(N, ints + I_NNEW, (const float*)h->psi_w, (const float*)dpsi, Ls.snap);
        else if (dwb)                                                       // in place, entry by entry
            to_dw_snap<double><<<g, 256, 0, cs_>>>(N, ints + I_NNEW, Ls.snap, nullptr, snap2, use_tc ? Ls.snap_t : nullptr, Ls.snap_l);
        // adaptive re-projections of Alg. 2: a conditional WHILE node when capturing (round(true, .)
        // launches one round, its test ends the loop), else m_max + 1 gated rounds
        // open(hc), when given, launches the work before the loop and sets the handle itself (it is
        // called with 0 when not capturing, and then sets nothing)
        auto adaptive = [&](auto&& round, auto&& open) -> int {
            if (!capturing) {
                open((cudaGraphConditionalHandle)0);
                for (int m = 0; m <= m_max_eff; ++m)
                    if (!round(false, m, (cudaGraphConditionalHandle)0)) break;
                return RTE_OK;
            }
            cudaStreamCaptureStatus cst;
            cudaGraph_t cgraph = nullptr;
            const cudaGraphNode_t* deps = nullptr;
            size_t ndep = 0;
            LR_CUDA(cudaStreamGetCaptureInfo(cs_, &cst, nullptr, &cgraph, &deps, nullptr, &ndep));
            cudaGraphConditionalHandle hc;
            LR_CUDA(cudaGraphConditionalHandleCreate(&hc, cgraph, 0, 0));
            if (!open(hc)) mgs_loop_begin<<<1, 32, 0, cs_>>>(a, hc);
            LR_CUDA(cudaStreamGetCaptureInfo(cs_, &cst, nullptr, &cgraph, &deps, nullptr, &ndep));
            cudaGraphNodeParams cp = {};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = hc;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            cudaGraphNode_t cnode;
            LR_CUDA(cudaGraphAddNode(&cnode, cgraph, deps, nullptr, ndep, &cp));
            LR_CUDA(cudaStreamUpdateCaptureDependencies(cs_, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies));
            if (!h->cap_stream2) LR_CUDA(cudaStreamCreateWithFlags(&h->cap_stream2, cudaStreamNonBlocking));
            cudaStream_t outer = cs_;
            cs_ = h->cap_stream2;
            GateCapture gate_capture;            // both held by the enclosing capture already
            CaptureLock capture_lock;
            LR_CUDA(cudaStreamBeginCaptureToGraph(cs_, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal));
            round(true, 0, hc);
            cudaGraph_t bodyg = nullptr;
            const cudaError_t be = cudaStreamEndCapture(cs_, &bodyg);
            if (be == cudaSuccess && bodyg) cond_bodies.push_back(bodyg);
            cs_ = outer;
            if (be != cudaSuccess) return fail(RTE_ERR_CUDA, std::string("loop capture: ") + cudaGetErrorString(be));
            return RTE_OK;
        };
        // profiling (uncaptured, launches one by one): read device state back so that only launches
        // that do work are issued and their byte counts use the current rank
        auto dev_int = [&](int idx) {
            int v_ = 0;
            cudaMemcpyAsync(&v_, ints + idx, sizeof(int), cudaMemcpyDeviceToHost, cs_);
            cudaStreamSynchronize(cs_);
            return v_;
        };
        // the orthogonality test of one round; false ends the uncaptured loop
        auto test = [&](bool cond, int m, cudaGraphConditionalHandle hc) {
            if (cond) {
                mgs_test_cond<<<1, 32, 0, cs_>>>(a, hc);
                return true;
            }
            mgs_test_kernel<<<1, 32, 0, cs_>>>(a, m == m_max_eff);
            if (h->prof.on && dev_int(I_MGSDONE)) return false;
            return m < m_max_eff;
        };
        if (dwb && fused) {
            // X^T psi_l over the columns present now and ||psi_l||, every slot in one pass per 8
            for (int l0 = 0; l0 < p; l0 += kXtV) {
                const int nv = std::min(kXtV, p - l0);
                if (use_tc) {
                    // tensor cores, split TF32 (rte_tc.cu): X hi read once, FP32 accumulation
                    pb(RTE_PROF_TC);
                    RTE_TRY(tc_projection_launch(&Ls.tc, l0, nv, kTcRows, nblk_tc, ints + I_STOP, ints + I_R, xpart,
                                                 kXtV, snap2, npart, h->d_err, cs_));
                    // bytes: X split in two FP32 arrays, the split snapshots and the double-word ones
                    pe(RTE_PROF_TC, 8.0 * N * (r_host + nv) + 8.0 * N * nv, 8.0 * N * r_host * nv);
                } else {
                    pb(RTE_PROF_XT);
                    xt_dw<<<dim3(nblk_x, (rc + 7) / 8), 256, sizeof(float2) * (size_t)nv * kXtRows, cs_>>>(
                        Ls.X2, N, ints, G_LIVE, snap2 + (size_t)l0 * N, nv, N, xpart, rc, npart, -1);
                    pe(RTE_PROF_XT, 8.0 * N * (r_host + nv), 2.0 * N * r_host * nv);
                }
                const int nbf = use_tc ? nblk_tc : nblk_x;
                pb(RTE_PROF_BASIS);
                xt_final<<<dim3((rc + 7) / 8, nv), 256, 0, cs_>>>(xpart, nbf, ints, G_LIVE, nv, rc,
                                                                 dcall + (size_t)l0 * rc, -1, kXtV);
                norms_final<<<1, 32 * kXtV, 0, cs_>>>(npart, nbf, nv, ints, G_LIVE, psn + l0);
                pe(RTE_PROF_BASIS, 8.0 * nbf * r_host * nv, 1.0 * nbf * r_host * nv);
            }
        }
        for (int l = 0; l < p; ++l) {
            if (dwb && fused)
                snap_open<<<dim3(kOpenChunks, std::max(1, l)), 256, 0, cs_>>>(a, l, snap2 + (size_t)l * N, psn, opart);
            else snap_begin<<<1, 32, 0, cs_>>>(a, l);
            if (h->prof.on && !capturing) {
                if (!dev_int(I_ACTIVE)) continue;        // an idle slot: every launch below is gated off
                r_host = dev_int(I_R);
            }
            if (dwb) {
                // two projections on the unnormalised snapshot (||psi|| and the first X^T psi from
                // snap_open, or formed here)
                const float2* sl = snap2 + (size_t)l * N;
                if (!fused) xtd(sl, 1, 0, Ls.small + SL.dc(), G_SNAP, sc + S_PSINORM);
                if (fused) {
                    // each pass also forms X^T v of its result: the next pass's coefficients, or
                    // the test's
                    passxt(G_SNAP, 1, sl, nullptr, dcall + (size_t)l * rc);
                    // captured: each pass's final launch runs the test and sets the loop handle
                    // (captured: the pass that ends the loop also appends the snapshot)
                    RTE_TRY(adaptive([&](bool cond, int m, cudaGraphConditionalHandle hc) {
                        if (cond) {
                            passxt(G_MGS, 0, v2, sc + S_ALPHA, nullptr, hc, l);
                            return true;
                        }
                        if (!test(cond, m, hc)) return false;
                        passxt(G_MGS, 0, v2, sc + S_ALPHA, nullptr);
                        return true;
                    }, [&](cudaGraphConditionalHandle hc) {
                        passxt(G_SNAP, 0, v2, sc + S_ALPHA, nullptr, hc, l);
                        return hc != 0;
                    }));
                } else {
                    passd(G_SNAP, 1, sl, nullptr);
                    xtd(v2, 1, 0, Ls.small + SL.dc(), G_SNAP, nullptr);
                    passd(G_SNAP, 0, v2, sc + S_ALPHA);
                    RTE_TRY(adaptive([&](bool cond, int m, cudaGraphConditionalHandle hc) {
                        xtd(v2, 1, 0, Ls.small + SL.dc(), G_MGS, nullptr);
                        if (!test(cond, m, hc)) return false;
                        passd(G_MGS, 0, v2, sc + S_ALPHA);
                        return true;
                    }, [](cudaGraphConditionalHandle) { return false; }));
                }
                if (!(fused && capturing)) mgs_append<<<1, 256, 0, cs_>>>(a, v, l);
                copy_col_dw<<<g, 256, 0, cs_>>>(a, v2);
                // border of the projected operators by the column of slot l (stencil images, X^T W,
                // the border rows): nothing later in this inner iteration's snapshot loop reads
                // it, so in a captured graph it is a branch of its own that runs beside the next
                // slots' projections (slots in order; joined before the factors are bordered)
                cudaStream_t bs = cs_;
                if (capturing) {
                    LR_CUDA(cudaEventRecord(h->ev_fork, cs_));
                    LR_CUDA(cudaStreamWaitEvent(h->border_stream, h->ev_fork, 0));
                    bs = h->border_stream;
                    forked = true;
                }
                pb(RTE_PROF_RESID);
                border_stencil_dw<<<dim3(sten_blocks, 5), 64, 0, bs>>>(a, l, Ls.E2, bpart, ints + I_CNT_STEN);
                pe(RTE_PROF_RESID, 8.0 * N * 7, 60.0 * N);
                pb(RTE_PROF_XT);
                xt_dw<<<dim3(nblk_x, (rc + 7) / 8), 256, sizeof(float2) * 5 * kXtRows, bs>>>(
                    Ls.X2, N, ints, G_LIVE, reinterpret_cast<const float2*>(Ls.W), 5, N, xpart_b, rc, nullptr, l);
                pe(RTE_PROF_XT, 8.0 * N * (r_host + 5), 10.0 * N * r_host);
                pb(RTE_PROF_BASIS);
                xt_final<<<dim3((rc + 7) / 8, 5), 256, 0, bs>>>(xpart_b, nblk_x, ints, G_LIVE, 5, rc,
                                                                Ls.small + SL.border(), l, kXtV);
                pe(RTE_PROF_BASIS, 8.0 * nblk_x * r_host * 5, 1.0 * nblk_x * r_host * 5);
                border_write<<<1, 256, 0, bs>>>(a, G_LIVE, l);
                fsrc_dots(G_LIVE, l, bs);
                continue;
            }
            copy_vec_g<<<g, 256, 0, cs_>>>(N, Ls.snap + (size_t)l * N, v, ints, G_SNAP);
            norm_into(v, G_SNAP, sc + S_PSINORM);
            const int fails_before = bu == RTE_UPDATE_MGSQR ? dev_int(I_MGSFAIL) : 0;
            for (int t = 0; t < n_mand; ++t) {                             // two projections (one: MGS-QR, QR)
                xt(v, 1, 0, Ls.small + SL.dc(), G_SNAP);
                xpass(G_SNAP, t == 0, 0);
            }
            finalize_sums<<<1, 32, 0, cs_>>>(part, g, 1, ints, G_SNAP, sc + S_ALPHA, 1);
            mgs_normalise<<<g, 256, 0, cs_>>>(a, G_SNAP, v);
            RTE_TRY(adaptive([&](bool cond, int m, cudaGraphConditionalHandle hc) {
                xt(v, 1, 0, Ls.small + SL.dc(), G_MGS);
                if (!test(cond, m, hc)) return false;
                xpass(G_MGS, 0, 1);
                finalize_sums<<<1, 32, 0, cs_>>>(part, g, 1, ints, G_MGS, sc + S_ALPHA, 1);
                mgs_normalise<<<g, 256, 0, cs_>>>(a, G_MGS, v);
                return true;
            }, [](cudaGraphConditionalHandle) { return false; }));
            mgs_append<<<1, 256, 0, cs_>>>(a, v, -1);
            copy_col<<<g, 256, 0, cs_>>>(a, v);
            pb(RTE_PROF_RESID);
            border_stencil<<<egrid(h, h->nc), 256, 0, cs_>>>(a, G_APP, -1);
            pe(RTE_PROF_RESID, 8.0 * N * 7, 60.0 * N);
            xt(Ls.W, 5, N, Ls.small + SL.border(), G_APP);
            newcol_dots_partial<<<nblk_d, 256, 0, cs_>>>(a, part);
            finalize_sums<<<1, 160, 0, cs_>>>(part, nblk_d, 5, ints, G_APP, Ls.small + SL.dots(), 0);
            border_write<<<1, 256, 0, cs_>>>(a, G_APP, -1);
            fsrc_dots(G_APP, -1, cs_);
            if (bu == RTE_UPDATE_MGSQR && dev_int(I_MGSFAIL) > fails_before) RTE_TRY(full_qr_rebuild());
        }
        if (bu == RTE_UPDATE_QR && dev_int(I_R) > 0) RTE_TRY(full_qr_rebuild());
        if (forked) {                                   // join the border branch
            LR_CUDA(cudaEventRecord(h->ev_join, h->border_stream));
            LR_CUDA(cudaStreamWaitEvent(cs_, h->ev_join, 0));
        }
        pb(RTE_PROF_GALERKIN);
        launch_galerkin(mt, 0, a, ndir, rc, q, cs_);     // border the factors by this iteration's columns
        pe(RTE_PROF_GALERKIN, 8.0 * ndir * p * (1.0 * r_host * r_host + 6.0 * r_host), 2.0 * ndir * p * r_host * r_host);
        if (deim) {
            deim_prepare<<<1, 256, 0, cs_>>>(a);
        } else {
        draw_kernel<<<1, 256, dsm, cs_>>>(a, q, -1, G_LIVE);
        pb(RTE_PROF_GALERKIN);
        launch_galerkin(mt, 1, a, ndir, rc, q, cs_);
        pe(RTE_PROF_GALERKIN, 8.0 * q * r_host * r_host / 2, 1.0 * q * r_host * r_host);
        pb(RTE_PROF_XC);
        if (dwb)
            x_times_dw<<<dim3(g, (q + kXtJ - 1) / kXtJ), 256, sizeof(float2) * kXtJ * rc, cs_>>>(Ls.X2, N, ints, G_LIVE, Ls.ccand2, rc,
                                                                        ints + I_NCAND, reinterpret_cast<float2*>(Ls.vcand));
        else
            for (int j0c = 0; j0c < q; j0c += kXtChunk)
                x_times<<<g, 256, xtsm, cs_>>>(Ls.X, N, ints, G_LIVE, Ls.small + SL.ccand(), rc, ints + I_NCAND,
                                               Ls.vcand, j0c);
        pe(RTE_PROF_XC, 8.0 * N * (r_host + q), 2.0 * N * r_host * q);
        pb(RTE_PROF_RESID);
        if (dwb) cand_residual_dw<<<dim3(nblk_res, q), 256, 0, cs_>>>(a);
        else cand_residual<<<dim3(nblk_res, q), 256, 0, cs_>>>(a);
        pe(RTE_PROF_RESID, 8.0 * N * (q + 2), 80.0 * N * q);
        select_kernel<<<1, 1024, 0, cs_>>>(a, nblk_res);
        }
        launch_galerkin(mt, 2, a, ndir, rc, q, cs_);
        full_assemble<<<egrid(h, (long long)rc * M), 256, 0, cs_>>>(a);
        full_cw<<<(rc + 7) / 8, 256, 0, cs_>>>(a);
        full_phi<<<g, 256, sizeof(double) * rc, cs_>>>(a);
        norm_into(Ls.W, G_FULL, sc + S_DIFF);
        full_decide<<<1, 32, 0, cs_>>>(a);
        full_update_old<<<g, 256, 0, cs_>>>(a);
        RTE_CUDA_TRY(cudaGetLastError());
        if (deim && !dev_int(I_STOP)) {
            // DEIM sampling: SVD of this iteration's C, then the next p angles (uncaptured loop)
            const int r_now = dev_int(I_R);
            pb(RTE_PROF_SVD);
            RTE_TRY(svd_of_c(h, r_now, svd_flag, cs_));
            deim_select<<<1, 256, 0, cs_>>>(a, Ls.svd_A, Ls.svd_s);
            pe(RTE_PROF_SVD, 8.0 * r_now * M * 2, 40.0 * r_now * r_now * M);
            RTE_CUDA_TRY(cudaGetLastError());
        }
        return RTE_OK;
    };

    // DEIM sampling and the full-QR basis updates read the rank back every iteration
    const bool use_graph = !h->prof.on && !deim && !bu_qr;
    const int batch = 4;
    s->converged = 0;
    for (int n = 1; n <= o->max_outer; ++n) {
        LR_TRY(launch_source(h, phi, RTE_FP64, S64, st));
        if (dwb) split_dw_g<<<g, 256, 0, st>>>(N, S64, Ls.S2);
        if (dwb && n == 1) split_dw_g<<<g, 256, 0, st>>>(4 * N, h->e_side, Ls.E2);   // inflow side vectors
        if (prec == RTE_FP32) LR_TRY(launch_source(h, phi, RTE_FP32, h->src_w, st));
        outer_begin<<<egrid(h, I_HDR + 2 * M), 256, 0, st>>>(a, n);
        copy_vec_g<<<g, 256, 0, st>>>(N, phi, Ls.phi_old, nullptr, G_ALWAYS);
        draw_kernel<<<1, 256, dsm, st>>>(a, p, I_NEW, G_ALWAYS);      // initial random angles (k = 0)
        LR_CUDA(cudaGetLastError());
        if (use_graph && !gexec) {
            // capture on a private non-blocking stream (the caller's may be the legacy stream),
            // launch the instantiated graph on the caller's stream
            if (!h->cap_stream) LR_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
            cs_ = h->cap_stream;
            cudaGraph_t gr = nullptr;
            int brc = RTE_OK;
            cudaError_t ce = cudaSuccess;
            {
                GateCapture gate_capture;        // no CUDA call of another batch thread meanwhile
                CaptureLock capture_lock;        // no device-synchronising call of another thread meanwhile
                const cudaError_t bc = cudaStreamBeginCapture(cs_, cudaStreamCaptureModeThreadLocal);
                if (bc != cudaSuccess) {
                    ce = bc;
                } else {
                    capturing = true;
                    brc = body();
                    capturing = false;
                    ce = cudaStreamEndCapture(cs_, &gr);
                }
            }
            cs_ = st;
            if (brc != RTE_OK) { if (gr) cudaGraphDestroy(gr); release(); return brc; }
            if (ce != cudaSuccess) { release(); return fail(RTE_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce)); }
            graph = gr;
            // programmatic dependent launch between the graph's consecutive kernels (and inside
            // the WHILE bodies)
            LR_TRY(make_edges_programmatic(graph));
            for (cudaGraph_t b : cond_bodies) LR_TRY(make_edges_programmatic(b));
            LR_CUDA(cudaGraphInstantiate(&gexec, graph, 0));
        }
        bool stop = false;
        while (!stop) {
            const int nb = use_graph ? batch : 1;
            for (int b = 0; b < nb; ++b) {
                if (use_graph) LR_CUDA(cudaGraphLaunch(gexec, st));
                else LR_TRY(body());
            }
            LR_CUDA(cudaMemcpyAsync(Ls.host_ints, ints, sizeof(int) * 128, cudaMemcpyDeviceToHost, st));
            LR_CUDA(gate_stream_sync(st));
            if (h->inject == RTE_ERR_SINGULAR && !Ls.host_ints[I_SING]) {
                h->inject = 0;                   // host-injected: as if the pivot check had fired
                Ls.host_ints[I_SING] = 1;
            }
            if (Ls.host_ints[I_SING] == 2) { release(); return fail(RTE_ERR_NAN, "low-rank: non-finite pivot in a Galerkin system"); }
            if (Ls.host_ints[I_SING]) { release(); return fail(RTE_ERR_SINGULAR, "low-rank: zero pivot in a Galerkin system"); }
            r_host = Ls.host_ints[I_R];
            stop = Ls.host_ints[I_STOP] != 0;
            if (!stop && Ls.host_ints[I_K] >= o->max_inner) {
                // force a full check so that phi^{(n,k)} is defined
                force_full<<<1, 32, 0, st>>>(a);
                launch_galerkin(mt, 2, a, ndir, rc, q, st);
                full_assemble<<<egrid(h, (long long)rc * M), 256, 0, st>>>(a);
                full_cw<<<(rc + 7) / 8, 256, 0, st>>>(a);
                full_phi<<<g, 256, sizeof(double) * rc, st>>>(a);
                LR_CUDA(cudaGetLastError());
                stop = true;
            }
        }
        LR_TRY(check_dep_flag(h, st));
        const int r = Ls.host_ints[I_R];
        r_host = 0;
        s->total_inner += Ls.host_ints[I_K];
        s->final_rank = r;
        Ls.last_rank = r;
        s->max_rank = std::max(s->max_rank, r);
        if (!bu_qr) s->mgs_failures += Ls.host_ints[I_MGSFAIL];   // failures became full QRs otherwise
        s->breakdowns += Ls.host_ints[I_BREAK];
        s->full_checks += Ls.host_ints[I_FULLCNT];
        // sweeps: one per appended or broken-down snapshot (twice with the defect correction)
        const int swept = r + Ls.host_ints[I_BREAK];
        s->total_sweeps += swept * (refine ? 2 : 1);
        s->cell_angle_updates += (long long)swept * h->nc * (refine ? 2 : 1);
        double diff = 0.0;
        LR_TRY(max_abs_diff(h, Ls.phi_k, phi, N, &diff, st));
        s->outer_iters = n;
        s->last_diff = diff;
        if (!(diff == diff) || isinf(diff)) { release(); return fail(RTE_ERR_NAN, "low-rank SI-DSA: non-finite scalar flux"); }
        const bool done = diff <= o->eps_si;
        const bool last = done || n == o->max_outer;
        if (o->truncate && r > 0 && (o->truncate == 1 || last)) {
            int rp = r;
            pb(RTE_PROF_SVD);
            LR_TRY(truncate_c(h, o, r, &rp, last && o->want_factors, st));
            pe(RTE_PROF_SVD, 8.0 * r * M * 2, 40.0 * r * r * M);
            s->final_rank_trunc = rp;
        }
        if (done) {
            copy_vec_g<<<g, 256, 0, st>>>(N, Ls.phi_k, phi, nullptr, G_ALWAYS);
            s->converged = 1;
            break;
        }
        if (o->use_dsa) {
            int it = 0;
            LR_TRY(dsa_correct(h, o, Ls.phi_k, phi, &it, st));
            s->dsa_cg_iters += it;
        } else {
            copy_vec_g<<<g, 256, 0, st>>>(N, Ls.phi_k, phi, nullptr, G_ALWAYS);
        }
    }
    if (F && psi_next && s->outer_iters > 0) {
        // psi^{n+1} = X C of the last inner loop, every angle (chunks of kXtChunk columns of C)
        int* d_m = nullptr;
        LR_TRY(A((void**)&d_m, sizeof(int)));
        LR_CUDA(cudaMemcpyAsync(d_m, &M, sizeof(int), cudaMemcpyHostToDevice, st));
        const size_t sm_x = sizeof(double) * (size_t)kXtChunk * rc;
        LR_TRY(smem_optin(x_times, sm_x));
        for (int j0c = 0; j0c < M; j0c += kXtChunk)
            x_times<<<g, 256, sm_x, st>>>(Ls.X, N, ints, G_ALWAYS, Ls.Cfull, rc, d_m, psi_next, j0c);
        LR_CUDA(cudaGetLastError());
    }
    LR_CUDA(cudaStreamSynchronize(st));
    release();
#undef LR_TRY
#undef LR_CUDA
    s->full_qr = full_qr_count;
    return s->converged ? RTE_OK : fail(RTE_ERR_NOT_CONVERGED, "low-rank SI-DSA: max_outer reached");
}

// A kernel of this translation unit (its CUDA library is enumerated by preload_all_kernels).
const void* lowrank_kernel_anchor() { return (const void*)xt_partial; }

}  // namespace rte
