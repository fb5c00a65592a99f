// Two-level preconditioner for the MIP DG-Q1 diffusion operator A of the DSA step.
//
//   M^{-1} r = B^{-1} r + P V(P^T r)
//
// B: the 4x4 diagonal blocks of A (block Jacobi).  P: the embedding of continuous bilinear
// (vertex-based Q1) functions into the DG-Q1 space.  On continuous functions the MIP jump and
// consistency terms vanish, so P^T A P is the continuous Q1 finite-element diffusion operator
// (with the MIP boundary terms): the smooth, nearly continuous modes that block Jacobi cannot
// damp live there (the additive two-level method of Dobrev, Lazarov, Vassilevski and Zikatanov,
// "Two-level preconditioning of discontinuous Galerkin approximations of second-order elliptic
// equations", 2006).  V is one symmetric geometric multigrid V-cycle on the vertex grids:
//   - Galerkin coarse operators A_{l+1} = R A_l P_l with bilinear P_l and R = P_l^T.  Every
//     operator is a 9-point vertex stencil; its entries are obtained by probing with the nine
//     colours (i mod 3, j mod 3), which separate the nine stencil positions;
//   - two l1-Jacobi sweeps before and after the coarse correction (M = diag of the l1 row
//     norms; 2M - A is positive definite, so the sweeps converge for any SPD stencil);
//   - the coarsest grid (at most kMgCoarseMax vertices) solved with its explicit inverse.
// The V-cycle is a fixed symmetric positive definite operator, so M^{-1} is a valid CG
// preconditioner.  All phases run inside the cooperative CG kernel, separated by grid syncs.
#pragma once

namespace rte {

// The hierarchy's arrays in the arithmetic V of the V-cycle (FP64, or FP32 for the FP32 CG).
template <typename V>
struct MgP;
template <>
struct MgP<double> {
    __device__ __forceinline__ static const double* S(const MgLevel& L) { return L.S; }
    __device__ __forceinline__ static const double* dinv(const MgLevel& L) { return L.dinv; }
    __device__ __forceinline__ static double* b(const MgLevel& L) { return L.b; }
    __device__ __forceinline__ static double* x(const MgLevel& L) { return L.x; }
    __device__ __forceinline__ static double* y(const MgLevel& L) { return L.y; }
    __device__ __forceinline__ static const double* Ainv(const MgArgs& M) { return M.Ainv; }
};
template <>
struct MgP<float> {
    __device__ __forceinline__ static const float* S(const MgLevel& L) { return L.S32; }
    __device__ __forceinline__ static const float* dinv(const MgLevel& L) { return L.dinv32; }
    __device__ __forceinline__ static float* b(const MgLevel& L) { return L.b32; }
    __device__ __forceinline__ static float* x(const MgLevel& L) { return L.x32; }
    __device__ __forceinline__ static float* y(const MgLevel& L) { return L.y32; }
    __device__ __forceinline__ static const float* Ainv(const MgArgs& M) { return M.Ainv32; }
};

// Weight of coarse index I in the prolongation to fine index i along one axis (Nc coarse
// points; fine point 2I coincides with coarse point I; an odd last fine point takes the last
// coarse value).
__host__ __device__ __forceinline__ double mg_w(int i, int I, int Nc, int coarsen) {
    if (!coarsen) return i == I ? 1.0 : 0.0;
    if ((i & 1) == 0) return (i >> 1) == I ? 1.0 : 0.0;
    const int lo = (i - 1) >> 1;
    if (lo + 1 >= Nc) return I == lo ? 1.0 : 0.0;
    return (I == lo || I == lo + 1) ? 0.5 : 0.0;
}

// (P_c^T t_c) at the corner (sx, sy) of cell c, without the factor g / 4.  With s, t the cell's
// coordinates scaled to [-1, 1], the bilinear function with corner values v has Legendre
// coefficients g (a, b / sqrt3, c / sqrt3, d / 3) where a, b, c, d are the corner sums weighted
// by 1, s, t, s t over 4.
template <typename V, typename T>
__device__ __forceinline__ V mg_corner(const T* __restrict__ t, int c, V sx, V sy) {
    const V k3 = V(0.57735026918962576451);
    return (V)t[4 * c] + sx * k3 * (V)t[4 * c + 1] + sy * k3 * (V)t[4 * c + 2] + sx * sy * V(1.0 / 3.0) * (V)t[4 * c + 3];
}

// b = P^T t on the vertex grid of the DG mesh; x = dinv b when x is given (first Jacobi sweep).
template <typename V, typename T>
__device__ __forceinline__ void mg_restrict_dg(const MgArgs& M, const T* __restrict__ t, V* __restrict__ b,
                                               V* __restrict__ x, int tid, int nth) {
    const int nxv = M.ncx + 1, N = nxv * (M.ncy + 1);
    const V q = V(0.25 * M.g);
    const V* dinv = MgP<V>::dinv(M.lv[0]);
    for (int v = tid; v < N; v += nth) {
        const int i = v % nxv, j = v / nxv;
        V s = V(0);
        if (i < M.ncx && j < M.ncy) s += mg_corner<V>(t, j * M.ncx + i, V(-1), V(-1));
        if (i > 0 && j < M.ncy) s += mg_corner<V>(t, j * M.ncx + i - 1, V(1), V(-1));
        if (i < M.ncx && j > 0) s += mg_corner<V>(t, (j - 1) * M.ncx + i, V(-1), V(1));
        if (i > 0 && j > 0) s += mg_corner<V>(t, (j - 1) * M.ncx + i - 1, V(1), V(1));
        s *= q;
        b[v] = s;
        if (x) x[v] = dinv[v] * s;
    }
}

// z = P x (assign) or z += P x on the DG mesh (FP64; used by the probing setup).
template <typename T>
__device__ __forceinline__ void mg_prolong_dg(const MgArgs& M, const double* __restrict__ x, T* __restrict__ z,
                                              bool assign, int tid, int nth) {
    const int nxv = M.ncx + 1, nc = M.ncx * M.ncy;
    const double q = 0.25 * M.g, k3 = 0.57735026918962576451;
    for (int c = tid; c < nc; c += nth) {
        const int ix = c % M.ncx, iy = c / M.ncx;
        const int v00 = iy * nxv + ix;
        const double a = x[v00], b = x[v00 + 1], cc = x[v00 + nxv], d = x[v00 + nxv + 1];
        const double z0 = q * (a + b + cc + d);
        const double z1 = q * k3 * (-a + b - cc + d);
        const double z2 = q * k3 * (-a - b + cc + d);
        const double z3 = q * (1.0 / 3.0) * (a - b - cc + d);
        if (assign) {
            z[4 * c] = (T)z0; z[4 * c + 1] = (T)z1; z[4 * c + 2] = (T)z2; z[4 * c + 3] = (T)z3;
        } else {
            z[4 * c] += (T)z0; z[4 * c + 1] += (T)z1; z[4 * c + 2] += (T)z2; z[4 * c + 3] += (T)z3;
        }
    }
}

// (S x)[v] for the 9-point stencil of level Lv.
template <typename V>
__device__ __forceinline__ V mg_Sx(const MgLevel& Lv, const V* __restrict__ x, int v) {
    const int N = Lv.nx * Lv.ny;
    const V* S = MgP<V>::S(Lv);
    const int i = v % Lv.nx, j = v / Lv.nx;
    V s = V(0);
#pragma unroll
    for (int dj = -1; dj <= 1; ++dj) {
        const int jj = j + dj;
        if (jj < 0 || jj >= Lv.ny) continue;
#pragma unroll
        for (int di = -1; di <= 1; ++di) {
            const int ii = i + di;
            if (ii < 0 || ii >= Lv.nx) continue;
            s = fma(S[(size_t)((di + 1) + 3 * (dj + 1)) * N + v], x[jj * Lv.nx + ii], s);
        }
    }
    return s;
}

// xo = xi + dinv (b - S xi)
template <typename V>
__device__ __forceinline__ void mg_jacobi(const MgLevel& Lv, const V* __restrict__ xi, V* __restrict__ xo, int tid,
                                          int nth) {
    const int N = Lv.nx * Lv.ny;
    const V* dinv = MgP<V>::dinv(Lv);
    const V* b = MgP<V>::b(Lv);
    for (int v = tid; v < N; v += nth) xo[v] = fma(dinv[v], b[v] - mg_Sx<V>(Lv, xi, v), xi[v]);
}

// r = b - S u
template <typename V>
__device__ __forceinline__ void mg_residual(const MgLevel& Lv, const V* __restrict__ u, V* __restrict__ r, int tid,
                                            int nth) {
    const int N = Lv.nx * Lv.ny;
    const V* b = MgP<V>::b(Lv);
    for (int v = tid; v < N; v += nth) r[v] = b[v] - mg_Sx<V>(Lv, u, v);
}

// b_C = R r_F (R = P^T); x_C = dinv_C b_C when x_C is given.
template <typename V>
__device__ __forceinline__ void mg_restrict(const MgLevel& F, const MgLevel& C, const V* __restrict__ r,
                                            V* __restrict__ bC, V* __restrict__ xC, int tid, int nth) {
    const int Nc = C.nx * C.ny;
    const V* dinvC = MgP<V>::dinv(C);
    for (int Vi = tid; Vi < Nc; Vi += nth) {
        const int I = Vi % C.nx, J = Vi / C.nx;
        const int i0 = F.cx ? 2 * I - 1 : I, i1 = F.cx ? 2 * I + 1 : I;
        const int j0 = F.cy ? 2 * J - 1 : J, j1 = F.cy ? 2 * J + 1 : J;
        V s = V(0);
        for (int j = max(j0, 0); j <= min(j1, F.ny - 1); ++j) {
            const V wy = (V)mg_w(j, J, C.ny, F.cy);
            if (wy == V(0)) continue;
            for (int i = max(i0, 0); i <= min(i1, F.nx - 1); ++i) {
                const V wx = (V)mg_w(i, I, C.nx, F.cx);
                if (wx != V(0)) s = fma(wx * wy, r[j * F.nx + i], s);
            }
        }
        bC[Vi] = s;
        if (xC) xC[Vi] = dinvC[Vi] * s;
    }
}

// u_F = P x_C (assign) or u_F += P x_C.
template <typename V>
__device__ __forceinline__ void mg_prolong(const MgLevel& F, const MgLevel& C, const V* __restrict__ xC,
                                           V* __restrict__ uF, bool assign, int tid, int nth) {
    const int N = F.nx * F.ny;
    for (int v = tid; v < N; v += nth) {
        const int i = v % F.nx, j = v / F.nx;
        const int I0 = F.cx ? (i >> 1) : i, I1 = F.cx ? (i >> 1) + 1 : i;
        const int J0 = F.cy ? (j >> 1) : j, J1 = F.cy ? (j >> 1) + 1 : j;
        V s = V(0);
        for (int J = J0; J <= min(J1, C.ny - 1); ++J) {
            const V wy = (V)mg_w(j, J, C.ny, F.cy);
            if (wy == V(0)) continue;
            for (int I = I0; I <= min(I1, C.nx - 1); ++I) {
                const V wx = (V)mg_w(i, I, C.nx, F.cx);
                if (wx != V(0)) s = fma(wx * wy, xC[J * C.nx + I], s);
            }
        }
        uF[v] = assign ? s : uF[v] + s;
    }
}

// y_{L-1} = A_{L-1}^{-1} b_{L-1}
template <typename V>
__device__ __forceinline__ void mg_coarse(const MgArgs& M, int tid, int nth) {
    const MgLevel& C = M.lv[M.L - 1];
    const int N = C.nx * C.ny;
    const V* Ai = MgP<V>::Ainv(M);
    const V* b = MgP<V>::b(C);
    V* y = MgP<V>::y(C);
    for (int i = tid; i < N; i += nth) {
        V s = V(0);
        for (int k = 0; k < N; ++k) s = fma(Ai[(size_t)i * N + k], b[k], s);
        y[i] = s;
    }
}

// Smoothing sweeps before and after each coarse correction (1 or 2).
#ifndef RTE_MG_NU
#define RTE_MG_NU 2
#endif
constexpr int kMgNu = RTE_MG_NU;

// One level's way down: pre-smoothing (x = dinv b, the first sweep, is already formed), the
// residual and its restriction; the iterate ends in y.  Three phases (nu = 2) or two (nu = 1).
template <typename V, typename Sync>
__device__ __forceinline__ void mg_down(const MgLevel* F, const MgLevel* C, int tid, int nth, Sync sync) {
    // F == nullptr: no work on this level for this problem; pass the syncs only
    if (kMgNu == 2) {
        sync();
        if (F) mg_jacobi<V>(*F, MgP<V>::x(*F), MgP<V>::y(*F), tid, nth);      // second pre-sweep: iterate in y
        sync();
        if (F) mg_residual<V>(*F, MgP<V>::y(*F), MgP<V>::x(*F), tid, nth);    // residual in x
        sync();
        if (F) mg_restrict<V>(*F, *C, MgP<V>::x(*F), MgP<V>::b(*C), MgP<V>::x(*C), tid, nth);
    } else {
        sync();
        if (F) mg_residual<V>(*F, MgP<V>::x(*F), MgP<V>::y(*F), tid, nth);    // iterate in x, residual in y
        sync();
        if (F) mg_restrict<V>(*F, *C, MgP<V>::y(*F), MgP<V>::b(*C), MgP<V>::x(*C), tid, nth);
    }
}

// One level's way up: the coarse correction and post-smoothing; the result ends in y.
template <typename V, typename Sync>
__device__ __forceinline__ void mg_up(const MgLevel* F, const MgLevel* C, int tid, int nth, Sync sync) {
    if (kMgNu == 2) {
        sync();
        if (F) mg_prolong<V>(*F, *C, MgP<V>::y(*C), MgP<V>::y(*F), false, tid, nth);
        sync();
        if (F) mg_jacobi<V>(*F, MgP<V>::y(*F), MgP<V>::x(*F), tid, nth);
        sync();
        if (F) mg_jacobi<V>(*F, MgP<V>::x(*F), MgP<V>::y(*F), tid, nth);
    } else {
        sync();
        if (F) mg_prolong<V>(*F, *C, MgP<V>::y(*C), MgP<V>::x(*F), false, tid, nth);
        sync();
        if (F) mg_jacobi<V>(*F, MgP<V>::x(*F), MgP<V>::y(*F), tid, nth);
    }
}

// The part of a V-cycle from level l0 (b and x = dinv b already formed there) down to the
// coarsest grid and back, run by a group of threads (one block, or the blocks of a cluster)
// that synchronises with `sync`: on small levels a grid-wide sync costs more than the whole
// level's work.  Leaves the result in y of level l0.
template <typename V, typename Sync>
__device__ __forceinline__ void mg_vcycle_group(const MgArgs& M, int l0, int tid, int nth, Sync sync) {
    for (int l = l0; l + 1 < M.L; ++l) mg_down<V>(&M.lv[l], &M.lv[l + 1], tid, nth, sync);
    sync();
    mg_coarse<V>(M, tid, nth);
    for (int l = M.L - 2; l >= l0; --l) mg_up<V>(&M.lv[l], &M.lv[l + 1], tid, nth, sync);
    sync();
}

template <typename V>
__device__ __forceinline__ void mg_vcycle_block(const MgArgs& M, int l0) {
    mg_vcycle_group<V>(M, l0, (int)threadIdx.x, (int)blockDim.x, [] { __syncthreads(); });
}

// One V-cycle on lv[0].b with lv[0].x = dinv b (the first pre-smoothing sweep from zero)
// already formed by mg_restrict_dg; the result is left in lv[0].y.  Two l1-Jacobi sweeps before
// and two after each coarse correction (symmetric).  Levels below lb (lb64 / lb32 of the
// hierarchy) run on the whole cooperative grid, 6 grid syncs each; level lb and the coarser
// ones run in one block (leader = that block) between two grid syncs.  (Fusing the residual
// into the restriction and the correction into the first post-sweep saves syncs but multiplies
// the stencil work per point; measured slower at 128 x 128 cells in FP64.)  Every thread of the
// cooperative grid calls it.  The phase schedule is that of an Lmax-level grid part: a problem
// with fewer grid levels (or none: work = false, M may be null) idles through the extra phases,
// so that problems of different sizes in one batched launch pass the same grid syncs.
template <typename V, typename Grid>
__device__ __forceinline__ void mg_vcycle(const MgArgs* M, int Lmax, bool work, bool leader, Grid& grid, int tid,
                                          int nth) {
    const int lb = work ? (sizeof(V) == 4 ? M->lb32 : M->lb64) : 0;
    auto gsync = [&] { grid.sync(); };
    for (int l = 0; l < Lmax; ++l) {
        const bool w = l < lb;
        mg_down<V>(w ? &M->lv[l] : nullptr, w ? &M->lv[l + 1] : nullptr, tid, nth, gsync);
    }
    grid.sync();
    if (work && leader) mg_vcycle_block<V>(*M, lb);
    for (int l = Lmax - 1; l >= 0; --l) {
        const bool w = l < lb;
        mg_up<V>(w ? &M->lv[l] : nullptr, w ? &M->lv[l + 1] : nullptr, tid, nth, gsync);
    }
    grid.sync();
}

}  // namespace rte
