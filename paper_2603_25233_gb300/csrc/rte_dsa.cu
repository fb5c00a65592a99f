// Diffusion synthetic acceleration (Eq. DSA / Eq. diffusion-correction): matrix-free
// modified-interior-penalty (MIP) DG-Q1 diffusion operator and a preconditioned CG that runs
// as one cooperative persistent kernel (all iterations on the device).
//
// Discretisation (the paper defers its "fully consistent" DSA to another work; this is the
// reading used throughout the library): on the DG-Q1 space of the transport solve,
//   a(u,v) = sum_K int D grad u . grad v + sigma_a u v
//          + sum_interior faces [ kappa [[u]][[v]] - {{D d_n u}}[[v]] - [[u]]{{D d_n v}} ]
//          + sum_boundary faces [ kappa u v - 1/2 (D d_n u) v - 1/2 u (D d_n v) ],
// D = 1/(3 sigma_t), kappa = max(1/4, 4 (D^- + D^+)/h) inside, max(1/4, 8 D/h) on the boundary.
//
// With the orthonormal Legendre basis, a face couples only equal tangential modes, so every
// face block is a 2x2 matrix in the normal degree (tensor identity in the tangential one),
// built from the 1D traces r = (1, sqrt3)/sqrt(h) (right end), l = (1, -sqrt3)/sqrt(h) (left
// end) and the derivative d = (0, 2 sqrt3 / h)/sqrt(h):
//   right face of c (c = "-" side): self  kappa r r^T - D_c/2 (r d^T + d r^T)
//                                   nbr  -kappa r l^T - D_n/2 r d^T + D_c/2 d l^T
//   left face of c (c = "+" side):  self  kappa l l^T + D_c/2 (l d^T + d l^T)
//                                   nbr  -kappa l r^T + D_n/2 l d^T - D_c/2 d r^T
// Boundary faces have the self form with the boundary kappa.  The volume term is
// D_c diag(0, 12/h_x^2) (x) I + D_c I (x) diag(0, 12/h_y^2) + sigma_a I.
#include <cooperative_groups.h>
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "rte_internal.cuh"
#include "rte_mg.cuh"

namespace cg = cooperative_groups;

namespace rte {

template <typename T>
struct MipArgsT {
    int nx, ny;
    T hx, hy;
    const T* D;
    const T* sa;
};
using MipArgs = MipArgsT<double>;

// Add the contribution of one face direction for the pair (u0, u1) (normal degree 0, 1).
// side = +1: face at the "+" end of the cell along the axis (c is the "-" side of the face);
// side = -1: face at the "-" end.  un: neighbour pair (ignored when !has_n).
template <typename T>
__device__ __forceinline__ void mip_face(T h, T Dc, T Dn, bool has_n, int side, T u0, T u1, T un0, T un1, T& y0,
                                         T& y1) {
    const T s3 = T(1.7320508075688772935);
    const T sh = T(1) / sqrt(h);
    const T d1 = T(2) * s3 * sh / h;                     // d = (0, d1)
    const T kap = has_n ? fmax(T(0.25), T(4) * (Dc + Dn) / h) : fmax(T(0.25), T(8) * Dc / h);
    // e = r for side +1, l for side -1 ; o = the neighbour's facing trace (l for side +1, r for -1)
    const T e1 = side > 0 ? s3 * sh : -s3 * sh;
    const T e0 = sh;
    const T eu = e0 * u0 + e1 * u1;                      // e . u
    const T du = d1 * u1;                                // d . u
    const T sg = side > 0 ? T(-0.5) : T(0.5);            // sign of the D/2 terms
    // self: kap e (e.u) + sg Dc (e (d.u) + d (e.u))
    y0 += kap * e0 * eu + sg * Dc * e0 * du;
    y1 += kap * e1 * eu + sg * Dc * (e1 * du + d1 * eu);
    if (has_n) {
        const T o1 = -e1;                                // neighbour's trace on this face
        const T ou = e0 * un0 + o1 * un1;                // o . un
        const T dun = d1 * un1;                          // d . un
        // nbr: -kap e (o.un) + sg Dn e (d.un) - sg Dc d (o.un)
        y0 += -kap * e0 * ou + sg * Dn * e0 * dun;
        y1 += -kap * e1 * ou + sg * Dn * e1 * dun - sg * Dc * d1 * ou;
    }
}

// y = (A x)_c for one cell with own coefficients xo[4]; x supplies the neighbours' values
// (not read when self_only, which gives the diagonal block alone).
template <typename T>
__device__ __forceinline__ void mip_cell(const MipArgsT<T>& m, int c, const T xo[4], const T* __restrict__ x, T y[4],
                                         bool self_only) {
    const int ix = c % m.nx, iy = c / m.nx;
    const T Dc = m.D[c];
    const T xc0 = xo[0], xc1 = xo[1], xc2 = xo[2], xc3 = xo[3];
    const T kx = T(12) * Dc / (m.hx * m.hx), ky = T(12) * Dc / (m.hy * m.hy);
    const T sa = m.sa[c];
    y[0] = sa * xc0;
    y[1] = (sa + kx) * xc1;
    y[2] = (sa + ky) * xc2;
    y[3] = (sa + kx + ky) * xc3;
    // x faces: pairs over the x degree i for each y mode j = 0 (DOFs 0,1) and j = 1 (DOFs 2,3)
    {
        const bool hr = ix + 1 < m.nx, hl = ix > 0;
        const int cr = c + 1, cl = c - 1;
        const T Dr = hr ? m.D[cr] : T(0), Dl = hl ? m.D[cl] : T(0);
        T r0 = 0, r1 = 0, r2 = 0, r3 = 0, l0 = 0, l1 = 0, l2 = 0, l3 = 0;
        if (hr && !self_only) { r0 = x[4 * cr]; r1 = x[4 * cr + 1]; r2 = x[4 * cr + 2]; r3 = x[4 * cr + 3]; }
        if (hl && !self_only) { l0 = x[4 * cl]; l1 = x[4 * cl + 1]; l2 = x[4 * cl + 2]; l3 = x[4 * cl + 3]; }
        mip_face(m.hx, Dc, Dr, hr, +1, xc0, xc1, r0, r1, y[0], y[1]);
        mip_face(m.hx, Dc, Dr, hr, +1, xc2, xc3, r2, r3, y[2], y[3]);
        mip_face(m.hx, Dc, Dl, hl, -1, xc0, xc1, l0, l1, y[0], y[1]);
        mip_face(m.hx, Dc, Dl, hl, -1, xc2, xc3, l2, l3, y[2], y[3]);
    }
    // y faces: pairs over the y degree j for each x mode i = 0 (DOFs 0,2) and i = 1 (DOFs 1,3)
    {
        const bool ht = iy + 1 < m.ny, hb = iy > 0;
        const int ct = c + m.nx, cb = c - m.nx;
        const T Dt = ht ? m.D[ct] : T(0), Db = hb ? m.D[cb] : T(0);
        T t0 = 0, t1 = 0, t2 = 0, t3 = 0, b0 = 0, b1 = 0, b2 = 0, b3 = 0;
        if (ht && !self_only) { t0 = x[4 * ct]; t1 = x[4 * ct + 1]; t2 = x[4 * ct + 2]; t3 = x[4 * ct + 3]; }
        if (hb && !self_only) { b0 = x[4 * cb]; b1 = x[4 * cb + 1]; b2 = x[4 * cb + 2]; b3 = x[4 * cb + 3]; }
        mip_face(m.hy, Dc, Dt, ht, +1, xc0, xc2, t0, t2, y[0], y[2]);
        mip_face(m.hy, Dc, Dt, ht, +1, xc1, xc3, t1, t3, y[1], y[3]);
        mip_face(m.hy, Dc, Db, hb, -1, xc0, xc2, b0, b2, y[0], y[2]);
        mip_face(m.hy, Dc, Db, hb, -1, xc1, xc3, b1, b3, y[1], y[3]);
    }
}

__global__ void dsa_coeff_kernel(int nc, const double* __restrict__ st, const double* __restrict__ ss,
                                 double* __restrict__ D, double* __restrict__ sa) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        D[c] = 1.0 / (3.0 * st[c]);
        sa[c] = st[c] - ss[c];
    }
}

// Inverse of each 4x4 diagonal block (Gauss-Jordan with partial pivoting).
__global__ void dsa_blockinv_kernel(MipArgs m, int nc, double* __restrict__ Minv) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        double A[4][8];
        for (int col = 0; col < 4; ++col) {   // column col = diagonal block applied to e_col
            double xl[4] = {0, 0, 0, 0};
            xl[col] = 1.0;
            double y[4];
            mip_cell<double>(m, c, xl, nullptr, y, true);
            for (int r = 0; r < 4; ++r) A[r][col] = y[r];
        }
        for (int r = 0; r < 4; ++r)
            for (int k = 0; k < 4; ++k) A[r][4 + k] = (r == k) ? 1.0 : 0.0;
        for (int k = 0; k < 4; ++k) {
            int piv = k;
            for (int r = k + 1; r < 4; ++r)
                if (fabs(A[r][k]) > fabs(A[piv][k])) piv = r;
            if (piv != k)
                for (int q = 0; q < 8; ++q) { double t = A[k][q]; A[k][q] = A[piv][q]; A[piv][q] = t; }
            const double inv = 1.0 / A[k][k];
            for (int q = 0; q < 8; ++q) A[k][q] *= inv;
            for (int r = 0; r < 4; ++r) {
                if (r == k) continue;
                const double f = A[r][k];
                for (int q = 0; q < 8; ++q) A[r][q] -= f * A[k][q];
            }
        }
        for (int r = 0; r < 4; ++r)
            for (int k = 0; k < 4; ++k) Minv[16 * (size_t)c + 4 * r + k] = A[r][4 + k];
    }
}

__global__ void dsa_apply_kernel(MipArgs m, int nc, const double* __restrict__ x, double* __restrict__ y) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        double v[4], xo[4] = {x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3]};
        mip_cell<double>(m, c, xo, x, v, false);
        y[4 * c] = v[0]; y[4 * c + 1] = v[1]; y[4 * c + 2] = v[2]; y[4 * c + 3] = v[3];
    }
}

template <typename T>
__global__ void to_t_kernel(long long n, const double* __restrict__ a, T* __restrict__ b) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = (T)a[i];
}

// ---- multigrid setup (probing of the Galerkin vertex operators) ----
__global__ void mg_color_kernel(int nx, int ny, int k, double* __restrict__ e) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nx * ny; v += gridDim.x * blockDim.x)
        e[v] = ((v % nx) % 3 + 3 * ((v / nx) % 3)) == k ? 1.0 : 0.0;
}
__global__ void mg_prolong_dg_kernel(MgArgs M, const double* __restrict__ x, double* __restrict__ z) {
    mg_prolong_dg<double>(M, x, z, true, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}
__global__ void mg_restrict_dg_kernel(MgArgs M, const double* __restrict__ t, double* __restrict__ b) {
    mg_restrict_dg<double, double>(M, t, b, nullptr, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}
__global__ void mg_stencil_kernel(MgLevel F, const double* __restrict__ x, double* __restrict__ y) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < F.nx * F.ny; v += gridDim.x * blockDim.x)
        y[v] = mg_Sx<double>(F, x, v);
}
__global__ void mg_prolong_kernel(MgLevel F, MgLevel C, const double* __restrict__ xC, double* __restrict__ uF) {
    mg_prolong<double>(F, C, xC, uF, true, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}
__global__ void mg_restrict_kernel(MgLevel F, MgLevel C, const double* __restrict__ r, double* __restrict__ bC) {
    mg_restrict<double>(F, C, r, bC, nullptr, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}
// S[d][v] = (A e_color(v+d))[v]: the probe of the colour of neighbour v + d, read at v.
__global__ void mg_fill_kernel(MgLevel Lv, const double* __restrict__ y9) {
    const int N = Lv.nx * Lv.ny;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
        const int i = v % Lv.nx, j = v / Lv.nx;
        double l1 = 0.0;
        for (int d = 0; d < 9; ++d) {
            const int ii = i + d % 3 - 1, jj = j + d / 3 - 1;
            double a = 0.0;
            if (ii >= 0 && ii < Lv.nx && jj >= 0 && jj < Lv.ny) a = y9[(size_t)(ii % 3 + 3 * (jj % 3)) * N + v];
            Lv.S[(size_t)d * N + v] = a;
            l1 += fabs(a);
        }
        Lv.dinv[v] = l1 > 0.0 ? 1.0 / l1 : 0.0;
    }
}
// Explicit inverse of the coarsest stencil operator (N <= kMgCoarseMax) by Gauss-Jordan
// elimination without pivoting (the operator is symmetric positive definite); one block.
__global__ void mg_inverse_kernel(MgLevel C, double* __restrict__ W, double* __restrict__ Ainv) {
    __shared__ double f[kMgCoarseMax];
    const int N = C.nx * C.ny, N2 = 2 * N;
    for (int idx = threadIdx.x; idx < N * N2; idx += blockDim.x) {
        const int r = idx / N2, c = idx % N2;
        double a = 0.0;
        if (c < N) {
            const int di = c % C.nx - r % C.nx, dj = c / C.nx - r / C.nx;
            if (di >= -1 && di <= 1 && dj >= -1 && dj <= 1) a = C.S[(size_t)((di + 1) + 3 * (dj + 1)) * N + r];
        } else {
            a = (c - N == r) ? 1.0 : 0.0;
        }
        W[idx] = a;
    }
    __syncthreads();
    for (int k = 0; k < N; ++k) {
        const double piv = W[(size_t)k * N2 + k];
        __syncthreads();
        for (int c = threadIdx.x; c < N2; c += blockDim.x) W[(size_t)k * N2 + c] /= piv;
        for (int r = threadIdx.x; r < N; r += blockDim.x) f[r] = W[(size_t)r * N2 + k];
        __syncthreads();
        for (int idx = threadIdx.x; idx < N * N2; idx += blockDim.x) {
            const int r = idx / N2, c = idx % N2;
            if (r != k) W[idx] -= f[r] * W[(size_t)k * N2 + c];
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) Ainv[idx] = W[(size_t)(idx / N) * N2 + N + idx % N];
}

static int grid_of(const rte_handle* h, long long n) {
    long long g = (n + 255) / 256;
    return (int)std::max(1ll, std::min(g, (long long)std::max(h->num_sms, 1) * 8));
}

// Build (first call: also size and allocate) the vertex hierarchy and probe its operators.
static int mg_setup(rte_handle* h, const MipArgsT<double>& mip) {
    MgArgs& M = h->mg;
    cudaStream_t st = h->stream;
    if (!h->mg_dev) {
        M.ncx = h->nx;
        M.ncy = h->ny;
        M.g = sqrt(h->hx * h->hy);
        int nx = h->nx + 1, ny = h->ny + 1, L = 0;
        for (;;) {
            M.lv[L].nx = nx;
            M.lv[L].ny = ny;
            const int cx = nx > 2, cy = ny > 2;
            if (nx * ny <= kMgCoarseMax || (!cx && !cy) || L + 1 == kMgMaxLevels) {
                M.lv[L].cx = M.lv[L].cy = 0;
                break;
            }
            M.lv[L].cx = cx;
            M.lv[L].cy = cy;
            nx = cx ? (nx + 1) / 2 : nx;
            ny = cy ? (ny + 1) / 2 : ny;
            ++L;
        }
        M.L = L + 1;
        if (M.lv[L].nx * M.lv[L].ny > kMgCoarseMax) {      // not reachable for meshes below 2^15 cells a side
            M.L = 0;
            return RTE_OK;
        }
        for (int l = 0; l < M.L; ++l) {
            const size_t N = (size_t)M.lv[l].nx * M.lv[l].ny;
            double* blk = nullptr;
            float* blk32 = nullptr;
            RTE_TRY(h->arena.alloc((void**)&blk, sizeof(double) * 13 * N));
            RTE_TRY(h->arena.alloc((void**)&blk32, sizeof(float) * 13 * N));
            M.lv[l].S = blk;
            M.lv[l].dinv = blk + 9 * N;
            M.lv[l].b = blk + 10 * N;
            M.lv[l].x = blk + 11 * N;
            M.lv[l].y = blk + 12 * N;
            M.lv[l].S32 = blk32;
            M.lv[l].dinv32 = blk32 + 9 * N;
            M.lv[l].b32 = blk32 + 10 * N;
            M.lv[l].x32 = blk32 + 11 * N;
            M.lv[l].y32 = blk32 + 12 * N;
        }
        const size_t N0 = (size_t)M.lv[0].nx * M.lv[0].ny, Nc = (size_t)M.lv[M.L - 1].nx * M.lv[M.L - 1].ny;
        // probing vectors [12 N0], Gauss-Jordan work [2 Nc^2], coarsest inverse [Nc^2]
        RTE_TRY(h->arena.alloc((void**)&h->mg_scratch, sizeof(double) * (12 * N0 + 3 * Nc * Nc)));
        M.Ainv = h->mg_scratch + 12 * N0 + 2 * Nc * Nc;
        RTE_TRY(h->arena.alloc((void**)&M.Ainv32, sizeof(float) * Nc * Nc));
        RTE_TRY(h->arena.alloc((void**)&h->mg_dev, sizeof(MgArgs)));
    }
    if (M.L == 0) return RTE_OK;
    M.lb64 = M.lb32 = M.L - 1;
    for (int l = M.L - 1; l >= 1; --l) {      // first level small enough for one block
        const int N = M.lv[l].nx * M.lv[l].ny;
        if (N <= kMgBlockMax64) M.lb64 = l;
        if (N <= kMgBlockMax32) M.lb32 = l;
    }
    const size_t N0 = (size_t)M.lv[0].nx * M.lv[0].ny;
    double* y9 = h->mg_scratch;              // [9 N0]
    double* e = y9 + 9 * N0;                 // [N0]
    double* f1 = e + N0;                     // [N0]
    double* f2 = f1 + N0;                    // [N0]
    // level 0: P^T A P by probing through the DG operator (h->tmp, h->dphi as DG scratch)
    for (int k = 0; k < 9; ++k) {
        mg_color_kernel<<<grid_of(h, N0), 256, 0, st>>>(M.lv[0].nx, M.lv[0].ny, k, e);
        mg_prolong_dg_kernel<<<grid_of(h, h->nc), 256, 0, st>>>(M, e, h->tmp);
        dsa_apply_kernel<<<grid_of(h, h->nc), 256, 0, st>>>(mip, h->nc, h->tmp, h->dphi);
        mg_restrict_dg_kernel<<<grid_of(h, N0), 256, 0, st>>>(M, h->dphi, y9 + k * N0);
    }
    mg_fill_kernel<<<grid_of(h, N0), 256, 0, st>>>(M.lv[0], y9);
    // coarser levels: R A_l P
    for (int l = 0; l + 1 < M.L; ++l) {
        const MgLevel F = M.lv[l], C = M.lv[l + 1];
        const size_t Nf = (size_t)F.nx * F.ny, Ncl = (size_t)C.nx * C.ny;
        for (int k = 0; k < 9; ++k) {
            mg_color_kernel<<<grid_of(h, Ncl), 256, 0, st>>>(C.nx, C.ny, k, e);
            mg_prolong_kernel<<<grid_of(h, Nf), 256, 0, st>>>(F, C, e, f1);
            mg_stencil_kernel<<<grid_of(h, Nf), 256, 0, st>>>(F, f1, f2);
            mg_restrict_kernel<<<grid_of(h, Ncl), 256, 0, st>>>(F, C, f2, y9 + k * Ncl);
        }
        mg_fill_kernel<<<grid_of(h, Ncl), 256, 0, st>>>(C, y9);
    }
    mg_inverse_kernel<<<1, 256, 0, st>>>(M.lv[M.L - 1], h->mg_scratch + 12 * N0, M.Ainv);
    // FP32 copies of the operators for the V-cycle of the FP32 CG
    for (int l = 0; l < M.L; ++l) {
        const long long N = (long long)M.lv[l].nx * M.lv[l].ny;
        to_t_kernel<float><<<grid_of(h, 10 * N), 256, 0, st>>>(10 * N, M.lv[l].S, M.lv[l].S32);   // S and dinv
    }
    {
        const long long Nc = (long long)M.lv[M.L - 1].nx * M.lv[M.L - 1].ny;
        to_t_kernel<float><<<grid_of(h, Nc * Nc), 256, 0, st>>>(Nc * Nc, M.Ainv, M.Ainv32);
    }
    RTE_CUDA_TRY(cudaGetLastError());
    RTE_CUDA_TRY(cudaMemcpyAsync(h->mg_dev, &M, sizeof(MgArgs), cudaMemcpyHostToDevice, st));
    return RTE_OK;
}

// A handle's reduction scratch holds two partial arrays of 4096 doubles (2 per block).
constexpr int kCgMaxGrid = 2048;

template <typename T>
struct CgArgs {
    MipArgsT<T> m;
    int nc;
    const double* b;     // right-hand side (FP64)
    double* x;           // solution (FP64)
    T *xw, *r, *z, *p, *q;
    const T* Minv;
    double* partA;       // [grid * 2]
    double* partB;       // [grid * 2]
    double tol;
    int max_iter;
    int* iters_out;
    const MgArgs* mg;    // two-level preconditioner (device copy) or nullptr for block Jacobi
};

template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sm) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sm[wid * NV + k] = v[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double t = lane < (int)(blockDim.x >> 5) ? sm[lane * NV + k] : 0.0;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            v[k] = t;
        }
    }
    __syncthreads();
}

// Every block sums the per-block partials in the same order: identical results everywhere.
__device__ __forceinline__ void grid_total(const double* part, int nblk, double& s0, double& s1, double* sm) {
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) { a += part[2 * i]; b += part[2 * i + 1]; }
    double v[2] = {a, b};
    block_sum<2>(v, sm);
    if (threadIdx.x == 0) { sm[64] = v[0]; sm[65] = v[1]; }
    __syncthreads();
    s0 = sm[64];
    s1 = sm[65];
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ void apply_minv(const T* __restrict__ Mi, const T r[4], T z[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) z[i] = Mi[4 * i] * r[0] + Mi[4 * i + 1] * r[1] + Mi[4 * i + 2] * r[2] + Mi[4 * i + 3] * r[3];
}

// Preconditioned CG in the arithmetic of T with all inner products accumulated in FP64; one
// cooperative launch runs every iteration.  Preconditioner: block Jacobi on the 4x4 cell
// blocks, plus (a.mg != nullptr) the additive vertex-grid multigrid correction of rte_mg.cuh.
// z = M^{-1} r for the r held in a.r; on return every block's partials of (r.z) are in v[0]
// (block-summed); r must be complete on entry (a grid sync after its last update).
template <typename T, typename Grid>
__device__ __forceinline__ void cg_precond(const CgArgs<T>& a, int Lmax, bool work, bool leader, Grid& grid, int tid,
                                           int nth, bool set_p, double& rz) {
    if (work) {
        for (int c = tid; c < a.nc; c += nth) {
            T rr[4], zz[4];
            for (int k = 0; k < 4; ++k) rr[k] = a.r[4 * c + k];
            apply_minv<T>(a.Minv + 16 * (size_t)c, rr, zz);
            for (int k = 0; k < 4; ++k) a.z[4 * c + k] = zz[k];
        }
        mg_restrict_dg<T, T>(*a.mg, a.r, MgP<T>::b(a.mg->lv[0]), MgP<T>::x(a.mg->lv[0]), tid, nth);
    }
    mg_vcycle<T>(a.mg, Lmax, work, leader, grid, tid, nth);
    if (!work) return;
    const MgArgs& M = *a.mg;
    const int nxv = M.ncx + 1;
    const T q = T(0.25 * M.g), k3 = T(0.57735026918962576451);
    const T* y0 = MgP<T>::y(M.lv[0]);
    rz = 0.0;
    for (int c = tid; c < a.nc; c += nth) {
        const int ix = c % M.ncx, iy = c / M.ncx;
        const int v00 = iy * nxv + ix;
        const T p00 = y0[v00], p10 = y0[v00 + 1], p01 = y0[v00 + nxv], p11 = y0[v00 + nxv + 1];
        const T w[4] = {q * (p00 + p10 + p01 + p11), q * k3 * (-p00 + p10 - p01 + p11),
                        q * k3 * (-p00 - p10 + p01 + p11), q * T(1.0 / 3.0) * (p00 - p10 - p01 + p11)};
        for (int k = 0; k < 4; ++k) {
            const T zk = a.z[4 * c + k] + w[k];
            a.z[4 * c + k] = zk;
            if (set_p) a.p[4 * c + k] = zk;
            rz += (double)a.r[4 * c + k] * zk;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(128) dsa_cg_kernel(CgArgs<T> a) {
    cg::grid_group grid = cg::this_grid();
    __shared__ double sm[80];
    const int nblk = gridDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nth = gridDim.x * blockDim.x;
    const bool mg = a.mg != nullptr;
    double v2[2] = {0.0, 0.0};
    for (int c = tid; c < a.nc; c += nth) {
        T rr[4], zz[4];
        for (int k = 0; k < 4; ++k) { rr[k] = (T)a.b[4 * c + k]; a.xw[4 * c + k] = T(0); a.r[4 * c + k] = rr[k]; }
        for (int k = 0; k < 4; ++k) v2[1] += (double)rr[k] * rr[k];
        if (!mg) {
            apply_minv<T>(a.Minv + 16 * (size_t)c, rr, zz);
            for (int k = 0; k < 4; ++k) {
                a.z[4 * c + k] = zz[k];
                a.p[4 * c + k] = zz[k];
                v2[0] += (double)rr[k] * zz[k];
            }
        }
    }
    if (mg) {
        grid.sync();
        cg_precond<T>(a, sizeof(T) == 4 ? a.mg->lb32 : a.mg->lb64, true, blockIdx.x == 0, grid, tid, nth, true, v2[0]);
    }
    block_sum<2>(v2, sm);
    if (threadIdx.x == 0) { a.partA[2 * blockIdx.x] = v2[0]; a.partA[2 * blockIdx.x + 1] = v2[1]; }
    grid.sync();
    double rz, bb;
    grid_total(a.partA, nblk, rz, bb, sm);
    int it = 0;
    if (bb > 0.0 && rz > 0.0) {
        const double thr = a.tol * a.tol * bb;
        for (it = 1; it <= a.max_iter; ++it) {
            double v1[2] = {0.0, 0.0};
            for (int c = tid; c < a.nc; c += nth) {
                T y[4], po[4] = {a.p[4 * c], a.p[4 * c + 1], a.p[4 * c + 2], a.p[4 * c + 3]};
                mip_cell<T>(a.m, c, po, a.p, y, false);
                for (int k = 0; k < 4; ++k) { a.q[4 * c + k] = y[k]; v1[0] += (double)po[k] * y[k]; }
            }
            block_sum<2>(v1, sm);
            if (threadIdx.x == 0) { a.partB[2 * blockIdx.x] = v1[0]; a.partB[2 * blockIdx.x + 1] = 0.0; }
            grid.sync();
            double pq, dummy;
            grid_total(a.partB, nblk, pq, dummy, sm);
            const T alpha = (T)(rz / pq);
            double v3[2] = {0.0, 0.0};
            for (int c = tid; c < a.nc; c += nth) {
                T rr[4], zz[4];
                for (int k = 0; k < 4; ++k) {
                    a.xw[4 * c + k] += alpha * a.p[4 * c + k];
                    rr[k] = a.r[4 * c + k] - alpha * a.q[4 * c + k];
                    a.r[4 * c + k] = rr[k];
                    v3[1] += (double)rr[k] * rr[k];
                }
                if (!mg) {
                    apply_minv<T>(a.Minv + 16 * (size_t)c, rr, zz);
                    for (int k = 0; k < 4; ++k) {
                        a.z[4 * c + k] = zz[k];
                        v3[0] += (double)rr[k] * zz[k];
                    }
                }
            }
            if (mg) {
                grid.sync();
                cg_precond<T>(a, sizeof(T) == 4 ? a.mg->lb32 : a.mg->lb64, true, blockIdx.x == 0, grid, tid, nth, false,
                              v3[0]);
            }
            block_sum<2>(v3, sm);
            if (threadIdx.x == 0) { a.partA[2 * blockIdx.x] = v3[0]; a.partA[2 * blockIdx.x + 1] = v3[1]; }
            grid.sync();
            double rz_new, rr2;
            grid_total(a.partA, nblk, rz_new, rr2, sm);
            if (rr2 <= thr || !(rr2 == rr2)) break;
            const T beta = (T)(rz_new / rz);
            rz = rz_new;
            for (int c = tid; c < a.nc; c += nth)
                for (int k = 0; k < 4; ++k) a.p[4 * c + k] = a.z[4 * c + k] + beta * a.p[4 * c + k];
            grid.sync();
        }
        if (it > a.max_iter) it = a.max_iter;
    }
    for (int c = tid; c < a.nc; c += nth)
        for (int k = 0; k < 4; ++k) a.x[4 * c + k] = (bb > 0.0 && rz > 0.0) ? (double)a.xw[4 * c + k] : 0.0;
    if (tid == 0) a.iters_out[0] = it;
}


__global__ void dsa_rhs_kernel(int nc, const double* __restrict__ ss, const double* __restrict__ phi_star,
                               const double* __restrict__ phi, double* __restrict__ rhs) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 4 * nc; i += gridDim.x * blockDim.x)
        rhs[i] = ss[i >> 2] * (phi_star[i] - phi[i]);
}

__global__ void axpy_store_kernel(int n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = a[i] + b[i];
}

static MipArgs mip_args(const rte_handle* h) {
    MipArgs m;
    m.nx = h->nx;
    m.ny = h->ny;
    m.hx = h->hx;
    m.hy = h->hy;
    m.D = h->D;
    m.sa = h->sig_a;
    return m;
}

static int elem_grid(const rte_handle* h, long long n) {
    long long g = (n + 255) / 256;
    return (int)std::max(1ll, std::min(g, (long long)std::max(h->num_sms, 1) * 8));
}

template <typename T>
static int cg_grid_for(const rte_handle* h) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dsa_cg_kernel<T>, 128, 0) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
    }
    const int maxg = std::max(1, per_sm) * std::max(1, h->num_sms);
    const int want = (h->nc + 127) / 128;
    return std::max(1, std::min(std::min(maxg, want), kCgMaxGrid));
}

int dsa_prepare(rte_handle* h) {
    const int g = elem_grid(h, h->nc);
    dsa_coeff_kernel<<<g, 256, 0, h->stream>>>(h->nc, h->sig_t, h->sig_s, h->D, h->sig_a);
    dsa_blockinv_kernel<<<g, 256, 0, h->stream>>>(mip_args(h), h->nc, h->Minv);
    RTE_CUDA_TRY(cudaGetLastError());
    if (!h->D32) {
        RTE_TRY(h->arena.alloc((void**)&h->D32, sizeof(float) * h->nc));
        RTE_TRY(h->arena.alloc((void**)&h->sa32, sizeof(float) * h->nc));
        RTE_TRY(h->arena.alloc((void**)&h->Minv32, sizeof(float) * 16 * (size_t)h->nc));
        RTE_TRY(h->arena.alloc((void**)&h->cg_w, sizeof(double) * 5 * (size_t)h->ndof));
    }
    to_t_kernel<float><<<g, 256, 0, h->stream>>>(h->nc, h->D, h->D32);
    to_t_kernel<float><<<g, 256, 0, h->stream>>>(h->nc, h->sig_a, h->sa32);
    to_t_kernel<float><<<g, 256, 0, h->stream>>>(16ll * h->nc, h->Minv, h->Minv32);
    RTE_CUDA_TRY(cudaGetLastError());
    RTE_TRY(mg_setup(h, mip_args(h)));
    if (h->cg_grid == 0) {
        h->cg_grid = cg_grid_for<double>(h);
        h->cg_grid32 = cg_grid_for<float>(h);
    }
    return RTE_OK;
}

int dsa_apply(rte_handle* h, const double* x, double* y, cudaStream_t st) {
    dsa_apply_kernel<<<elem_grid(h, h->nc), 256, 0, st>>>(mip_args(h), h->nc, x, y);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

// Cluster-resident CG: one thread-block cluster (1 to 16 CTAs of kCgBlockThreads threads) runs
// the whole preconditioned CG of one problem, V-cycle included.  Phases are separated by the
// hardware cluster barrier and the inner products are reduced through distributed shared
// memory, so no grid-wide sync is needed: for meshes up to about a hundred thousand cells a
// grid-wide sync costs more than a phase's work.  Clusters of different problems never wait on
// one another, so a launch holds any number of problems (block b of cluster k works on
// problem k).
constexpr int kCgBlockThreads = 1024;
constexpr int kCgClusterMaxCells = 262144;  // cluster schedules are autotuning candidates up to here

// Sum of v over the cluster; every thread gets the total.  sm: [80] doubles of this block,
// slot: which pair of sm[64..69] carries this reduction (rotated so that a slot is rewritten
// only after two further cluster barriers).
template <int NV>
__device__ __forceinline__ void cluster_sum(cg::cluster_group& cl, double (&v)[NV], double* sm, int slot) {
    block_sum<NV>(v, sm);
    double* mine = sm + 64 + 2 * slot;
    if (threadIdx.x == 0)
        for (int k = 0; k < NV; ++k) mine[k] = v[k];
    cl.sync();
    const int nb = (int)cl.num_blocks();
    for (int k = 0; k < NV; ++k) {
        double t = 0.0;
        for (int r = 0; r < nb; ++r) t += cl.map_shared_rank(mine, r)[k];
        v[k] = t;
    }
}

template <typename T>
__global__ void __launch_bounds__(kCgBlockThreads) dsa_cg_cluster_kernel(const CgArgs<T>* __restrict__ args) {
    __shared__ double sm[80];
    cg::cluster_group cl = cg::this_cluster();
    const int cs = (int)cl.num_blocks();
    const CgArgs<T> a = args[blockIdx.x / cs];
    const int tid = (int)cl.block_rank() * blockDim.x + threadIdx.x, nth = cs * blockDim.x;
    const bool mg = a.mg != nullptr;
    int slot = 0;
    auto csync = [&] { cl.sync(); };
    // z = M^{-1} r for the current r (complete), p = z when set_p; returns this thread's r.z part
    auto precond = [&](bool set_p) -> double {
        for (int c = tid; c < a.nc; c += nth) {
            T rr[4], zz[4];
            for (int k = 0; k < 4; ++k) rr[k] = a.r[4 * c + k];
            apply_minv<T>(a.Minv + 16 * (size_t)c, rr, zz);
            for (int k = 0; k < 4; ++k) a.z[4 * c + k] = zz[k];
        }
        if (mg) {
            const MgArgs& M = *a.mg;
            mg_restrict_dg<T, T>(M, a.r, MgP<T>::b(M.lv[0]), MgP<T>::x(M.lv[0]), tid, nth);
            mg_vcycle_group<T>(M, 0, tid, nth, csync);       // starts and ends with a barrier
            const int nxv = M.ncx + 1;
            const T q = T(0.25 * M.g), k3 = T(0.57735026918962576451);
            const T* y0 = MgP<T>::y(M.lv[0]);
            for (int c = tid; c < a.nc; c += nth) {
                const int ix = c % M.ncx, iy = c / M.ncx;
                const int v00 = iy * nxv + ix;
                const T p00 = y0[v00], p10 = y0[v00 + 1], p01 = y0[v00 + nxv], p11 = y0[v00 + nxv + 1];
                a.z[4 * c] += q * (p00 + p10 + p01 + p11);
                a.z[4 * c + 1] += q * k3 * (-p00 + p10 - p01 + p11);
                a.z[4 * c + 2] += q * k3 * (-p00 - p10 + p01 + p11);
                a.z[4 * c + 3] += q * T(1.0 / 3.0) * (p00 - p10 - p01 + p11);
            }
        }
        double rz = 0.0;
        for (int c = tid; c < a.nc; c += nth)
            for (int k = 0; k < 4; ++k) {
                const T zk = a.z[4 * c + k];
                if (set_p) a.p[4 * c + k] = zk;
                rz += (double)a.r[4 * c + k] * zk;
            }
        return rz;
    };
    double v2[2] = {0.0, 0.0};
    for (int c = tid; c < a.nc; c += nth)
        for (int k = 0; k < 4; ++k) {
            const T rk = (T)a.b[4 * c + k];
            a.xw[4 * c + k] = T(0);
            a.r[4 * c + k] = rk;
            v2[1] += (double)rk * rk;
        }
    cl.sync();
    v2[0] = precond(true);
    cluster_sum<2>(cl, v2, sm, slot);
    slot = (slot + 1) % 3;
    double rz = v2[0];
    const double bb = v2[1];
    int it = 0;
    if (bb > 0.0 && rz > 0.0) {
        const double thr = a.tol * a.tol * bb;
        for (it = 1; it <= a.max_iter; ++it) {
            cl.sync();                                         // p complete
            double v1[1] = {0.0};
            for (int c = tid; c < a.nc; c += nth) {
                T y[4], po[4] = {a.p[4 * c], a.p[4 * c + 1], a.p[4 * c + 2], a.p[4 * c + 3]};
                mip_cell<T>(a.m, c, po, a.p, y, false);
                for (int k = 0; k < 4; ++k) { a.q[4 * c + k] = y[k]; v1[0] += (double)po[k] * y[k]; }
            }
            cluster_sum<1>(cl, v1, sm, slot);
            slot = (slot + 1) % 3;
            const T alpha = (T)(rz / v1[0]);
            double v3[2] = {0.0, 0.0};
            for (int c = tid; c < a.nc; c += nth)
                for (int k = 0; k < 4; ++k) {
                    a.xw[4 * c + k] += alpha * a.p[4 * c + k];
                    const T rk = a.r[4 * c + k] - alpha * a.q[4 * c + k];
                    a.r[4 * c + k] = rk;
                    v3[1] += (double)rk * rk;
                }
            cl.sync();                                         // r complete
            v3[0] = precond(false);
            cluster_sum<2>(cl, v3, sm, slot);
            slot = (slot + 1) % 3;
            const double rz_new = v3[0], rr2 = v3[1];
            if (rr2 <= thr || !(rr2 == rr2)) break;
            const T beta = (T)(rz_new / rz);
            rz = rz_new;
            for (int c = tid; c < a.nc; c += nth)
                for (int k = 0; k < 4; ++k) a.p[4 * c + k] = a.z[4 * c + k] + beta * a.p[4 * c + k];
        }
        if (it > a.max_iter) it = a.max_iter;
    }
    for (int c = tid; c < a.nc; c += nth)
        for (int k = 0; k < 4; ++k) a.x[4 * c + k] = (bb > 0.0 && rz > 0.0) ? (double)a.xw[4 * c + k] : 0.0;
    if (tid == 0) a.iters_out[0] = it;
    cl.sync();                                                 // peers' shared memory stays valid
}

// Launch nprob cluster-resident CGs of cs CTAs each (args: DEVICE array of nprob CgArgs).
template <typename T>
static int launch_cg_cluster(const CgArgs<T>* d_args, int nprob, int cs, cudaStream_t st) {
    auto kern = dsa_cg_cluster_kernel<T>;
    // set once per instantiation (a thread-safe function-local static: solves of a batch may run
    // on several host threads)
    static const cudaError_t set_rc = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    RTE_CUDA_TRY(set_rc);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nprob * cs));
    cfg.blockDim = dim3(kCgBlockThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    RTE_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, d_args));
    return RTE_OK;
}

// Largest launchable cluster size (power of two, <= 16) for the cluster CG.
template <typename T>
static int probe_max_cluster_size() {
    int c = 1;
    auto kern = dsa_cg_cluster_kernel<T>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) cudaGetLastError();
    for (int cs = 16; cs >= 2; cs /= 2) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)cs);
        cfg.blockDim = dim3(kCgBlockThreads);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int ncl = 0;
        if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) == cudaSuccess && ncl > 0) { c = cs; break; }
        cudaGetLastError();
    }
    return c;
}

template <typename T>
static int max_cluster_size() {
    static const int c = probe_max_cluster_size<T>();   // thread-safe one-time probe
    return c;
}

template <typename T>
static int launch_cg(rte_handle* h, const double* rhs, double* x, double tol, int max_iter, int grid, cudaStream_t st) {
    CgArgs<T> a;
    if (std::is_same<T, float>::value) {
        MipArgsT<T> m;
        m.nx = h->nx; m.ny = h->ny; m.hx = (T)h->hx; m.hy = (T)h->hy;
        m.D = (const T*)h->D32; m.sa = (const T*)h->sa32;
        a.m = m;
        a.Minv = (const T*)h->Minv32;
    } else {
        MipArgsT<T> m;
        m.nx = h->nx; m.ny = h->ny; m.hx = (T)h->hx; m.hy = (T)h->hy;
        m.D = (const T*)h->D; m.sa = (const T*)h->sig_a;
        a.m = m;
        a.Minv = (const T*)h->Minv;
    }
    a.nc = h->nc;
    a.b = rhs;
    a.x = x;
    T* base = (T*)h->cg_w;
    const size_t n = h->ndof;
    a.xw = base; a.r = base + n; a.z = base + 2 * n; a.p = base + 3 * n; a.q = base + 4 * n;
    a.partA = h->cg_red;
    a.partB = h->cg_red + 4096;
    a.tol = tol;
    a.max_iter = max_iter;
    a.iters_out = h->cg_iters;
    a.mg = h->mg.L > 0 ? h->mg_dev : nullptr;
    if (grid < 0) {                               // cluster-resident schedule of -grid CTAs
        if (!h->cg_args_dev) RTE_TRY(h->arena.alloc(&h->cg_args_dev, sizeof(CgArgs<double>)));
        RTE_CUDA_TRY(cudaMemcpyAsync(h->cg_args_dev, &a, sizeof(CgArgs<T>), cudaMemcpyHostToDevice, st));
        return launch_cg_cluster<T>((const CgArgs<T>*)h->cg_args_dev, 1, -grid, st);
    }
    void* args[] = {&a};
    RTE_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)dsa_cg_kernel<T>, dim3(grid), dim3(128), args, 0, st));
    return RTE_OK;
}

// Autotuner for the CG schedule: a grid-wide synchronisation gets cheaper with fewer blocks while
// the per-block work grows, and on small meshes one block with block barriers beats any grid.
// Time 16 iterations of each candidate (cluster-resident CGs of 1, 2, 4, ... CTAs, then
// cooperative grids of powers of two up to the co-resident maximum) on a right-hand side of
// ones and keep the fastest (a negative grid -cs denotes the cluster-resident kernel with cs
// CTAs).  Runs once per precision.
template <typename T>
static int tune_cg_grid(rte_handle* h, int max_grid, int* best_out, cudaStream_t st) {
    double* b = h->tmp;
    double* x = h->dphi;
    std::vector<double> ones(h->ndof, 1.0);
    RTE_CUDA_TRY(cudaMemcpyAsync(b, ones.data(), sizeof(double) * h->ndof, cudaMemcpyHostToDevice, st));
    cudaEvent_t e0, e1;
    RTE_CUDA_TRY(cudaEventCreate(&e0));
    RTE_CUDA_TRY(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    int best = max_grid;
    // candidates: cluster-resident CGs of 1, 2, ..., max_cluster_size() CTAs (as -cs), then grids
    std::vector<int> cand;
    if (h->nc <= kCgClusterMaxCells)
        for (int cs = 1; cs <= max_cluster_size<T>(); cs *= 2) cand.push_back(-cs);
    for (int grid = 8; ; grid *= 2) {
        cand.push_back(std::min(grid, max_grid));
        if (grid >= max_grid) break;
    }
    for (int gq : cand) {
        float ms_min = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            RTE_CUDA_TRY(cudaEventRecord(e0, st));
            RTE_TRY(launch_cg<T>(h, b, x, 0.0, 16, gq, st));
            RTE_CUDA_TRY(cudaEventRecord(e1, st));
            RTE_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            RTE_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            ms_min = std::min(ms_min, ms);
        }
        if (ms_min < best_ms) { best_ms = ms_min; best = gq; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *best_out = best;
    return RTE_OK;
}

// Tune the CG grid for a precision once (uses h->tmp and h->dphi as scratch: call it before
// either holds live data).
static int dsa_tune(rte_handle* h, int precision, cudaStream_t st) {
    if (h->cg_tuned[precision == RTE_FP32 ? 1 : 0]) return RTE_OK;
    if (precision == RTE_FP32) RTE_TRY(tune_cg_grid<float>(h, h->cg_grid32, &h->cg_grid32, st));
    else RTE_TRY(tune_cg_grid<double>(h, h->cg_grid, &h->cg_grid, st));
    h->cg_tuned[precision == RTE_FP32 ? 1 : 0] = 1;
    return RTE_OK;
}

int dsa_cg_prec(rte_handle* h, const double* rhs, double* x, double tol, int max_iter, int precision, int* iters,
                cudaStream_t st) {
    RTE_PROF_BEGIN(h, RTE_PROF_DSA, st);
    if (precision == RTE_FP32) RTE_TRY(launch_cg<float>(h, rhs, x, tol, max_iter, h->cg_grid32, st));
    else RTE_TRY(launch_cg<double>(h, rhs, x, tol, max_iter, h->cg_grid, st));
    const int rec = h->prof.on ? h->prof.end(RTE_PROF_DSA, st, 0.0, 0.0) : -1;
    if (iters || rec >= 0) {
        RTE_CUDA_TRY(cudaMemcpyAsync(h->h_scalar + 8, h->cg_iters, sizeof(int), cudaMemcpyDeviceToHost, st));
        RTE_CUDA_TRY(cudaStreamSynchronize(st));
        const int it = *reinterpret_cast<int*>(h->h_scalar + 8);
        if (iters) *iters = it;
        if (rec >= 0) {
            // per CG iteration and cell: p, q, x, r, z read/written once (8 vectors x 4 values),
            // D, sigma_a and the 4x4 block inverse; ~260 flops (stencil, block-Jacobi, dots, axpys)
            const double esz = precision == RTE_FP32 ? 4.0 : 8.0;
            h->prof.pending[rec].bytes = (double)it * h->nc * esz * (8 * 4 + 2 + 16);
            h->prof.pending[rec].flops = (double)it * h->nc * 260.0;
        }
    }
    return RTE_OK;
}

int dsa_pretune(rte_handle* h, int precision) { return dsa_tune(h, precision, h->stream); }

int dsa_cg(rte_handle* h, const double* rhs, double* x, double tol, int max_iter, int* iters, cudaStream_t st) {
    return dsa_cg_prec(h, rhs, x, tol, max_iter, RTE_FP64, iters, st);
}

int dsa_correct(rte_handle* h, const rte_opts* o, const double* phi_star, double* phi, int* iters, cudaStream_t st) {
    RTE_TRY(dsa_tune(h, o->dsa_precision, st));
    const int g = elem_grid(h, h->ndof);
    dsa_rhs_kernel<<<g, 256, 0, st>>>(h->nc, h->sig_s, phi_star, phi, h->tmp);
    RTE_CUDA_TRY(cudaGetLastError());
    RTE_TRY(dsa_cg_prec(h, h->tmp, h->dphi, o->dsa_tol, o->dsa_max_iter, o->dsa_precision, iters, st));
    axpy_store_kernel<<<g, 256, 0, st>>>(h->ndof, phi_star, h->dphi, phi);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}


// ---------------------------------------------------------------------------------------------
// Batched CG over independent problems: one cooperative launch in which problem i owns the
// contiguous block range [first_i, first_i + nblk_i).  The grid-wide synchronisations are
// shared, the reductions are per problem (each block sums only its own problem's partials,
// in a fixed order), and a problem that has converged idles until every problem has.
struct CgBatchMap {
    int prob, first, nblk, pad;
};

template <typename T>
__global__ void __launch_bounds__(128) dsa_cg_batch_kernel(const CgArgs<T>* __restrict__ args,
                                                           const CgBatchMap* __restrict__ map, int nprob,
                                                           int max_iter, int mg_levels, int* ndone) {
    cg::grid_group grid = cg::this_grid();
    __shared__ double sm[80];
    const CgBatchMap bm = map[blockIdx.x];
    const CgArgs<T> a = args[bm.prob];
    const int lb = blockIdx.x - bm.first, nblk = bm.nblk;
    const int tid = lb * blockDim.x + threadIdx.x;
    const int nth = nblk * blockDim.x;
    const bool leader = lb == 0 && threadIdx.x == 0;
    const bool mg = a.mg != nullptr;          // this problem's preconditioner (uniform per problem)
    double v2[2] = {0.0, 0.0};
    for (int c = tid; c < a.nc; c += nth) {
        T rr[4], zz[4];
        for (int k = 0; k < 4; ++k) { rr[k] = (T)a.b[4 * c + k]; a.xw[4 * c + k] = T(0); a.r[4 * c + k] = rr[k]; }
        for (int k = 0; k < 4; ++k) v2[1] += (double)rr[k] * rr[k];
        if (!mg) {
            apply_minv<T>(a.Minv + 16 * (size_t)c, rr, zz);
            for (int k = 0; k < 4; ++k) {
                a.z[4 * c + k] = zz[k];
                a.p[4 * c + k] = zz[k];
                v2[0] += (double)rr[k] * zz[k];
            }
        }
    }
    if (mg_levels >= 0) {                     // every block passes the same syncs
        grid.sync();
        cg_precond<T>(a, mg_levels, mg, lb == 0, grid, tid, nth, true, v2[0]);
    }
    block_sum<2>(v2, sm);
    if (threadIdx.x == 0) { a.partA[2 * lb] = v2[0]; a.partA[2 * lb + 1] = v2[1]; }
    grid.sync();
    double rz, bb;
    grid_total(a.partA, nblk, rz, bb, sm);
    const bool started = bb > 0.0 && rz > 0.0;
    bool active = started && a.max_iter > 0;
    if (!active && leader) atomicAdd(ndone, 1);
    const double thr = a.tol * a.tol * bb;
    int it = 0;
    double rz_part = 0.0, rr_part = 0.0;
    for (int k = 1; k <= max_iter; ++k) {
        if (active) {
            double v1[2] = {0.0, 0.0};
            for (int c = tid; c < a.nc; c += nth) {
                T y[4], po[4] = {a.p[4 * c], a.p[4 * c + 1], a.p[4 * c + 2], a.p[4 * c + 3]};
                mip_cell<T>(a.m, c, po, a.p, y, false);
                for (int q = 0; q < 4; ++q) { a.q[4 * c + q] = y[q]; v1[0] += (double)po[q] * y[q]; }
            }
            block_sum<2>(v1, sm);
            if (threadIdx.x == 0) { a.partB[2 * lb] = v1[0]; a.partB[2 * lb + 1] = 0.0; }
        }
        grid.sync();
        if (active) {
            double pq, dummy;
            grid_total(a.partB, nblk, pq, dummy, sm);
            const T alpha = (T)(rz / pq);
            double v3[2] = {0.0, 0.0};
            for (int c = tid; c < a.nc; c += nth) {
                T rr[4], zz[4];
                for (int q = 0; q < 4; ++q) {
                    a.xw[4 * c + q] += alpha * a.p[4 * c + q];
                    rr[q] = a.r[4 * c + q] - alpha * a.q[4 * c + q];
                    a.r[4 * c + q] = rr[q];
                    v3[1] += (double)rr[q] * rr[q];
                }
                if (!mg) {
                    apply_minv<T>(a.Minv + 16 * (size_t)c, rr, zz);
                    for (int q = 0; q < 4; ++q) {
                        a.z[4 * c + q] = zz[q];
                        v3[0] += (double)rr[q] * zz[q];
                    }
                }
            }
            rr_part = v3[1];
            rz_part = v3[0];
        }
        if (mg_levels >= 0) {
            grid.sync();
            cg_precond<T>(a, mg_levels, active && mg, lb == 0, grid, tid, nth, false, rz_part);
        }
        if (active) {
            double v3[2] = {rz_part, rr_part};
            block_sum<2>(v3, sm);
            if (threadIdx.x == 0) { a.partA[2 * lb] = v3[0]; a.partA[2 * lb + 1] = v3[1]; }
        }
        grid.sync();
        if (active) {
            double rz_new, rr2;
            grid_total(a.partA, nblk, rz_new, rr2, sm);
            it = k;
            if (rr2 <= thr || !(rr2 == rr2) || k >= a.max_iter) {
                active = false;
                if (leader) atomicAdd(ndone, 1);
            } else {
                const T beta = (T)(rz_new / rz);
                rz = rz_new;
                for (int c = tid; c < a.nc; c += nth)
                    for (int q = 0; q < 4; ++q) a.p[4 * c + q] = a.z[4 * c + q] + beta * a.p[4 * c + q];
            }
        }
        grid.sync();
        if (*(volatile int*)ndone >= nprob) break;
    }
    for (int c = tid; c < a.nc; c += nth)
        for (int q = 0; q < 4; ++q) a.x[4 * c + q] = started ? (double)a.xw[4 * c + q] : 0.0;
    if (leader) a.iters_out[0] = it;
}

template <typename T>
static CgArgs<T> cg_args(rte_handle* h, const double* rhs, double* x, double tol, int max_iter) {
    CgArgs<T> a;
    MipArgsT<T> m;
    m.nx = h->nx; m.ny = h->ny; m.hx = (T)h->hx; m.hy = (T)h->hy;
    const bool f32 = std::is_same<T, float>::value;
    m.D = f32 ? (const T*)h->D32 : (const T*)h->D;
    m.sa = f32 ? (const T*)h->sa32 : (const T*)h->sig_a;
    a.m = m;
    a.Minv = f32 ? (const T*)h->Minv32 : (const T*)h->Minv;
    a.nc = h->nc;
    a.b = rhs;
    a.x = x;
    T* base = (T*)h->cg_w;
    const size_t n = h->ndof;
    a.xw = base; a.r = base + n; a.z = base + 2 * n; a.p = base + 3 * n; a.q = base + 4 * n;
    a.partA = h->cg_red;
    a.partB = h->cg_red + 4096;
    a.tol = tol;
    a.max_iter = max_iter;
    a.iters_out = h->cg_iters;
    a.mg = h->mg.L > 0 ? h->mg_dev : nullptr;
    return a;
}

// Blocks per problem in proportion to its cell count (at least one, at most kCgMaxGrid, the
// capacity of a handle's partial arrays), total within the co-resident maximum.
static int batch_block_split(rte_handle* const* hs, int n, int max_grid, std::vector<CgBatchMap>& map) {
    long long tot_cells = 0, want = 0;
    for (int i = 0; i < n; ++i) {
        tot_cells += hs[i]->nc;
        want += (hs[i]->nc + 127) / 128;
    }
    const long long G = std::max<long long>(n, std::min<long long>(max_grid, want));
    map.clear();
    for (int i = 0; i < n; ++i) {
        long long nb = std::max(1ll, (G - n) * hs[i]->nc / std::max(1ll, tot_cells) + 1);
        nb = std::min({nb, (long long)(hs[i]->nc + 127) / 128, (long long)kCgMaxGrid});
        nb = std::max(1ll, nb);
        const int first = (int)map.size();
        for (int b = 0; b < nb; ++b) map.push_back(CgBatchMap{i, first, (int)nb, 0});
    }
    return (int)map.size();
}

template <typename T>
static int cg_batch_t(rte_handle* const* hs, int n, const double* const* rhs, double* const* x, double tol, int max_iter,
                      cudaStream_t st) {
    rte_handle* own = hs[0];
    int maxc = 0;
    for (int i = 0; i < n; ++i) maxc = std::max(maxc, hs[i]->nc);
    if (maxc <= kCgClusterMaxCells) {
        // cluster-resident schedule: one cluster per problem (largest problems first), no
        // grid-wide syncs, no waiting between problems (the grid need not be co-resident).
        // Cluster size: about 8192 cells per CTA for the largest problem.
        int cs = 1;
        while (cs < max_cluster_size<T>() && (long long)cs * 8192 < maxc) cs *= 2;
        std::vector<int> order(n);
        for (int i = 0; i < n; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int u, int v) { return hs[u]->nc > hs[v]->nc; });
        std::vector<CgArgs<T>> args(n);
        for (int k = 0; k < n; ++k) args[k] = cg_args<T>(hs[order[k]], rhs[order[k]], x[order[k]], tol, max_iter);
        RTE_TRY(own->arena.grow(&own->batch_buf, &own->batch_cap, sizeof(CgArgs<T>) * n));
        RTE_CUDA_TRY(cudaMemcpyAsync(own->batch_buf, args.data(), sizeof(CgArgs<T>) * n, cudaMemcpyHostToDevice, st));
        return launch_cg_cluster<T>((const CgArgs<T>*)own->batch_buf, n, cs, st);
    }
    int per_sm = 0;
    RTE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dsa_cg_batch_kernel<T>, 128, 0));
    const int max_grid = std::max(1, per_sm) * std::max(1, own->num_sms);
    // problems go in chunks of at most max_grid (one block each at the least)
    for (int s0 = 0; s0 < n; s0 += max_grid) {
        const int m = std::min(n - s0, max_grid);
        std::vector<CgArgs<T>> args(m);
        for (int i = 0; i < m; ++i) args[i] = cg_args<T>(hs[s0 + i], rhs[s0 + i], x[s0 + i], tol, max_iter);
        std::vector<CgBatchMap> map;
        const int grid = batch_block_split(hs + s0, m, max_grid, map);
        const size_t need = sizeof(CgArgs<T>) * m + sizeof(CgBatchMap) * grid + 256;
        RTE_TRY(own->arena.grow(&own->batch_buf, &own->batch_cap, need));
        char* base = (char*)own->batch_buf;
        int* d_ndone = (int*)base;
        CgArgs<T>* d_args = (CgArgs<T>*)(base + 256);
        CgBatchMap* d_map = (CgBatchMap*)(base + 256 + sizeof(CgArgs<T>) * m);
        RTE_CUDA_TRY(cudaMemsetAsync(d_ndone, 0, sizeof(int), st));
        RTE_CUDA_TRY(cudaMemcpyAsync(d_args, args.data(), sizeof(CgArgs<T>) * m, cudaMemcpyHostToDevice, st));
        RTE_CUDA_TRY(cudaMemcpyAsync(d_map, map.data(), sizeof(CgBatchMap) * grid, cudaMemcpyHostToDevice, st));
        int mi = max_iter, nm = m, lmax = 0;
        bool any_mg = false;
        for (int i = 0; i < m; ++i) {
            const MgArgs& Mi = hs[s0 + i]->mg;
            if (Mi.L == 0) continue;
            any_mg = true;
            lmax = std::max(lmax, std::is_same<T, float>::value ? Mi.lb32 : Mi.lb64);
        }
        if (!any_mg) lmax = -1;
        void* kargs[] = {&d_args, &d_map, &nm, &mi, &lmax, &d_ndone};
        RTE_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)dsa_cg_batch_kernel<T>, dim3(grid), dim3(128), kargs, 0, st));
        // the pageable argument vectors are copied before cudaMemcpyAsync returns; the next
        // chunk reuses the device buffer only after this launch (same stream)
    }
    return RTE_OK;
}

// DSA correction for several problems with one batched CG (phi[i] = phi_star[i] + delta_i).
// iters[i] receives problem i's CG iteration count after the call (the call synchronises).
int dsa_correct_batch(rte_handle* const* hs, int n, const rte_opts* o, const double* const* phi_star,
                      double* const* phi, int* iters, cudaStream_t st) {
    if (n <= 0) return RTE_OK;
    rte_handle* own = hs[0];
    std::vector<const double*> rhs(n);
    std::vector<double*> x(n);
    for (int i = 0; i < n; ++i) {
        rte_handle* h = hs[i];
        dsa_rhs_kernel<<<elem_grid(h, h->ndof), 256, 0, st>>>(h->nc, h->sig_s, phi_star[i], phi[i], h->tmp);
        rhs[i] = h->tmp;
        x[i] = h->dphi;
    }
    RTE_CUDA_TRY(cudaGetLastError());
    double bytes = 0.0;
    RTE_PROF_BEGIN(own, RTE_PROF_DSA, st);
    if (o->dsa_precision == RTE_FP32) RTE_TRY(cg_batch_t<float>(hs, n, rhs.data(), x.data(), o->dsa_tol, o->dsa_max_iter, st));
    else RTE_TRY(cg_batch_t<double>(hs, n, rhs.data(), x.data(), o->dsa_tol, o->dsa_max_iter, st));
    const int rec = own->prof.on ? own->prof.end(RTE_PROF_DSA, st, 0.0, 0.0) : -1;
    for (int i = 0; i < n; ++i) {
        rte_handle* h = hs[i];
        axpy_store_kernel<<<elem_grid(h, h->ndof), 256, 0, st>>>(h->ndof, phi_star[i], h->dphi, phi[i]);
        RTE_CUDA_TRY(cudaMemcpyAsync(h->h_scalar + 8, h->cg_iters, sizeof(int), cudaMemcpyDeviceToHost, st));
    }
    RTE_CUDA_TRY(cudaGetLastError());
    RTE_CUDA_TRY(cudaStreamSynchronize(st));
    const double esz = o->dsa_precision == RTE_FP32 ? 4.0 : 8.0;
    double flops = 0.0;
    for (int i = 0; i < n; ++i) {
        const int it = *reinterpret_cast<int*>(hs[i]->h_scalar + 8);
        if (iters) iters[i] = it;
        bytes += (double)it * hs[i]->nc * esz * (8 * 4 + 2 + 16);
        flops += (double)it * hs[i]->nc * 260.0;
    }
    if (rec >= 0) {
        own->prof.pending[rec].bytes = bytes;
        own->prof.pending[rec].flops = flops;
    }
    return RTE_OK;
}

// A kernel of this translation unit (its CUDA library is enumerated by preload_all_kernels).
const void* dsa_kernel_anchor() { return (const void*)dsa_coeff_kernel; }

}  // namespace rte

using namespace rte;

extern "C" int rte_dsa_apply(rte_handle* h, const double* x, double* y) {
    if (!h || !x || !y) return fail(RTE_ERR_ARG, "rte_dsa_apply: null argument");
    return dsa_apply(h, x, y, h->stream);
}

extern "C" int rte_dsa_solve(rte_handle* h, const double* rhs, double* x, double tol, int max_iter, int* iters) {
    if (!h || !rhs || !x || max_iter < 0 || !(tol >= 0)) return fail(RTE_ERR_ARG, "rte_dsa_solve: bad argument");
    if (rhs == h->tmp || x == h->tmp || rhs == h->dphi || x == h->dphi) return fail(RTE_ERR_ARG, "rte_dsa_solve: aliasing");
    RTE_TRY(dsa_tune(h, RTE_FP64, h->stream));
    int it = 0;
    RTE_TRY(dsa_cg(h, rhs, x, tol, max_iter, &it, h->stream));
    if (iters) *iters = it;
    return RTE_OK;
}

// ---------------------------------------------------------------------------------------------
// Allocation-free DSA solve.  Some callers cannot allocate device memory: code that runs while
// another component holds the whole device-memory budget in its own pool, hosts that forbid
// allocation after start-up so that memory use stays fixed, or callers that must not trigger a
// (synchronising) cudaMalloc in the middle of their work.  For them rte_dsa_solve_static runs
// the same preconditioned CG as rte_dsa_solve without a handle: the per-cell coefficients, the
// block inverses, the CG vectors and the reduction partials live in the fixed array below.
// Every GPU that loads this library holds the array (about 5.1 MB) until the process exits.
#define RTE_STATIC_MAX_CELLS 16384
namespace rte {
namespace {
constexpr size_t kStaticPerCell = 38;                 // D, sigma_a, 16 block-inverse, 5 x 4 CG vectors
constexpr size_t kStaticPartials = 4 * 4096;          // two partial arrays of 2 x 4096
constexpr size_t kStaticDoubles = RTE_STATIC_MAX_CELLS * kStaticPerCell + kStaticPartials + 16;
}  // namespace
}  // namespace rte

static __device__ __align__(256) double g_rte_static_scratch[rte::kStaticDoubles];

namespace rte {
namespace {
// Device address of the scratch array in the current device's context.  In host code the
// array's name is only a host-side stand-in, so every call looks the address up (the lookup is
// cheap): a cached address would go stale after cudaDeviceReset or under another context.
// The first lookup on a device also loads this library's device code there.
int static_scratch_address(double** out) {
    void* p = nullptr;
    RTE_CUDA_TRY(cudaGetSymbolAddress(&p, g_rte_static_scratch));
    if (!p) return fail(RTE_ERR_CUDA, "rte_dsa_solve_static: no device address for the scratch array");
    *out = static_cast<double*>(p);
    return RTE_OK;
}
}  // namespace
}  // namespace rte

extern "C" int rte_dsa_solve_static(int nx, int ny, double x0, double x1, double y0, double y1, const double* sig_t,
                                    const double* sig_s, const double* rhs, double* x, double tol, int max_iter,
                                    int* iters, void* stream) {
    using namespace rte;
    if (nx < 1 || ny < 1) return fail(RTE_ERR_ARG, "rte_dsa_solve_static: nx, ny >= 1 required");
    if ((long long)nx * ny > RTE_STATIC_MAX_CELLS)
        return fail(RTE_ERR_ARG, "rte_dsa_solve_static: mesh exceeds the static scratch (at most 16384 cells)");
    if (!sig_t || !sig_s || !rhs || !x) return fail(RTE_ERR_ARG, "rte_dsa_solve_static: null pointer");
    if (!(x1 > x0) || !(y1 > y0) || !(tol >= 0) || max_iter < 0)
        return fail(RTE_ERR_ARG, "rte_dsa_solve_static: empty domain or bad tolerance");
    cudaStream_t st = (cudaStream_t)stream;
    double* base = nullptr;
    RTE_TRY(static_scratch_address(&base));
    const int nc = nx * ny;
    const size_t N = 4 * (size_t)nc;
    MipArgs m;
    m.nx = nx;
    m.ny = ny;
    m.hx = (x1 - x0) / nx;
    m.hy = (y1 - y0) / ny;
    double* D = base;
    double* sa = base + nc;
    double* Minv = base + 2 * (size_t)nc;
    double* vec = base + 18 * (size_t)nc;
    double* part = base + RTE_STATIC_MAX_CELLS * kStaticPerCell;
    int* it_dev = reinterpret_cast<int*>(part + kStaticPartials);
    m.D = D;
    m.sa = sa;
    int dev = 0, sms = 1, per_sm = 1;
    RTE_CUDA_TRY(cudaGetDevice(&dev));
    RTE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    RTE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dsa_cg_kernel<double>, 128, 0));
    const int eg = std::max(1, std::min((nc + 255) / 256, 8 * sms));
    dsa_coeff_kernel<<<eg, 256, 0, st>>>(nc, sig_t, sig_s, D, sa);
    dsa_blockinv_kernel<<<eg, 256, 0, st>>>(m, nc, Minv);
    RTE_CUDA_TRY(cudaGetLastError());
    CgArgs<double> a;
    a.m = m;
    a.nc = nc;
    a.b = rhs;
    a.x = x;
    a.xw = vec;
    a.r = vec + N;
    a.z = vec + 2 * N;
    a.p = vec + 3 * N;
    a.q = vec + 4 * N;
    a.Minv = Minv;
    a.partA = part;
    a.partB = part + 2 * 4096;
    a.tol = tol;
    a.max_iter = max_iter;
    a.iters_out = it_dev;
    a.mg = nullptr;
    const int grid = std::max(1, std::min(std::min(std::max(1, per_sm) * sms, (nc + 127) / 128), 4096));
    void* args[] = {&a};
    RTE_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)dsa_cg_kernel<double>, dim3(grid), dim3(128), args, 0, st));
    if (iters) {
        int hv = 0;
        RTE_CUDA_TRY(cudaMemcpyAsync(&hv, it_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
        RTE_CUDA_TRY(cudaStreamSynchronize(st));
        *iters = hv;
    }
    return RTE_OK;
}
