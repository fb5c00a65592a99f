// Full-rank SI-DSA (Sec. 2.2; stop test of Alg. 1) and the discrete-adjoint gradient of a
// linear detector response.  The host loop only launches kernels and reads one scalar per
// outer iteration (the stop test); every arithmetic step runs on the device.
//
// +-Omega_z twins of the CL rule have the same (Omega_x, Omega_y), hence the same upwind
// operator and inflow term in x-y geometry and identical psi_j: the full-rank sweep solves
// each distinct direction once with the summed weight (phi is unchanged).
#include <cuda.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "rte_internal.cuh"

namespace rte {

__global__ void copy_kernel(int n, const double* __restrict__ a, double* __restrict__ b) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = a[i];
}

// Adjoint source d + Sigma_s chi in the sweep precision.
template <typename T>
__global__ void adj_source_kernel(int nc, const double* __restrict__ sig_s, const double* __restrict__ chi,
                                  const double* __restrict__ det, T* __restrict__ S) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 4 * nc; i += gridDim.x * blockDim.x)
        S[i] = (T)fma(sig_s[i >> 2], chi[i], det[i]);
}

// g_t[c] = - sum_a w_a mu_a|_c . psi_a|_c ;  g_s[c] = chi|_c . phi|_c ;  g_q[c] = chi_c,0 sqrt(hx hy)
template <typename T>
__global__ void grad_kernel(int nc, int n, long long stride, const double* __restrict__ wl, const T* __restrict__ psi,
                            const T* __restrict__ mu, const double* __restrict__ chi, const double* __restrict__ phi,
                            double cellint, double* __restrict__ gt, double* __restrict__ gs, double* __restrict__ gq) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        if (gt) {
            double acc = 0.0;
            for (int a = 0; a < n; ++a) {
                const T* p = psi + (long long)a * stride + 4 * (long long)c;
                const T* m = mu + (long long)a * stride + 4 * (long long)c;
                double dot = (double)p[0] * m[0] + (double)p[1] * m[1] + (double)p[2] * m[2] + (double)p[3] * m[3];
                acc = fma(wl[a], dot, acc);
            }
            gt[c] = -acc;
        }
        if (gs) gs[c] = chi[4 * c] * phi[4 * c] + chi[4 * c + 1] * phi[4 * c + 1] + chi[4 * c + 2] * phi[4 * c + 2] +
                        chi[4 * c + 3] * phi[4 * c + 3];
        if (gq) gq[c] = chi[4 * c] * cellint;
    }
}

static int egrid(const rte_handle* h, long long n) {
    long long g = (n + 255) / 256;
    return (int)std::max(1ll, std::min(g, (long long)std::max(h->num_sms, 1) * 8));
}

// Per-ordinate sources of a backward-Euler step (Sec. 3.7), item a = ordinate a:
//   src_a = Sigma_s phi + G + M psi_a^n / dt   (M = identity in the orthonormal basis),
// formed in FP64 and rounded once to the sweep precision.
template <typename T>
__global__ void be_source_kernel(int nc, int n, const double* __restrict__ sig_s, const double* __restrict__ phi,
                                 const double* __restrict__ G, const double* __restrict__ psi_prev, double inv_dt,
                                 T* __restrict__ src) {
    const long long ndof = 4ll * nc, total = ndof * n;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const long long i = k % ndof;
        src[k] = T(fma(sig_s[i >> 2], phi[i], G[i]) + psi_prev[k] * inv_dt);
    }
}

// Low-rank step: F[d] = psi_prev[rep[d]] / dt for the distinct directions, and a flag set when
// psi_prev differs on a +-Omega_z twin pair (pairs[2 t], pairs[2 t + 1]).
__global__ void be_fsrc_kernel(int ndir, long long N, const int* __restrict__ rep, const double* __restrict__ psi_prev,
                               double inv_dt, double* __restrict__ F) {
    const long long total = (long long)ndir * N;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const long long d = k / N, i = k - d * N;
        F[k] = psi_prev[(long long)rep[d] * N + i] * inv_dt;
    }
}

__global__ void twin_mismatch_kernel(int npairs, long long N, const int* __restrict__ pairs,
                                     const double* __restrict__ psi, int* __restrict__ flag) {
    const long long total = (long long)npairs * N;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const long long t = k / N, i = k - t * N;
        if (!(psi[(long long)pairs[2 * t] * N + i] == psi[(long long)pairs[2 * t + 1] * N + i])) atomicOr(flag, 1);
    }
}

template <typename T>
__global__ void to_double_kernel(long long n, const T* __restrict__ a, double* __restrict__ b) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        b[k] = (double)a[k];
}

// Full-rank SI-DSA of one backward-Euler step over every ordinate with the handle's materials
// already shifted (sigma_t + 1/dt): the loop of Alg. 1 with per-ordinate sources.
static int be_loop(rte_handle* h, const rte_opts* o, double inv_dt, const double* psi_prev, double* phi,
                   void* src, void* psi, int* iota, rte_stats* s) {
    const int prec = o->sweep_precision == RTE_FP32 ? RTE_FP32 : RTE_FP64;
    const int M = h->nang;
    cudaStream_t st = h->stream;
    const int g = egrid(h, h->ndof);
    const int gs = egrid(h, (long long)M * h->ndof);
    s->converged = 0;
    for (int n = 1; n <= o->max_outer; ++n) {
        if (prec == RTE_FP32)
            be_source_kernel<float><<<gs, 256, 0, st>>>(h->nc, M, h->sig_s, phi, h->G, psi_prev, inv_dt, (float*)src);
        else
            be_source_kernel<double><<<gs, 256, 0, st>>>(h->nc, M, h->sig_s, phi, h->G, psi_prev, inv_dt, (double*)src);
        RTE_CUDA_TRY(cudaGetLastError());
        RTE_TRY(launch_sweep(h, iota, M, prec, src, h->ndof, 1, 0, psi, st));
        RTE_TRY(launch_phi_reduce(h, iota, h->d_w, M, prec, psi, h->phi_star, st));
        s->total_sweeps += M;
        s->cell_angle_updates += (long long)M * h->nc;
        double diff = 0.0;
        RTE_TRY(max_abs_diff(h, h->phi_star, phi, h->ndof, &diff, st));
        RTE_TRY(check_dep_flag(h, st));
        s->outer_iters = n;
        s->last_diff = diff;
        if (!(diff == diff) || isinf(diff)) return fail(RTE_ERR_NAN, "backward-Euler step: non-finite scalar flux");
        if (diff <= o->eps_si) {
            copy_kernel<<<g, 256, 0, st>>>(h->ndof, h->phi_star, phi);
            RTE_CUDA_TRY(cudaGetLastError());
            s->converged = 1;
            break;
        }
        if (o->use_dsa) {
            int it = 0;
            RTE_TRY(dsa_correct(h, o, h->phi_star, phi, &it, st));
            s->dsa_cg_iters += it;
        } else {
            copy_kernel<<<g, 256, 0, st>>>(h->ndof, h->phi_star, phi);
            RTE_CUDA_TRY(cudaGetLastError());
        }
    }
    RTE_CUDA_TRY(cudaStreamSynchronize(st));
    return RTE_OK;
}

// One SI-DSA iteration loop shared by the forward (reverse = 0) and adjoint (reverse = 1)
// full-rank solves.  Forward source: Sigma_s phi + G (+ inflow); adjoint: det + Sigma_s chi.
static int fr_loop(rte_handle* h, const rte_opts* o, double* phi, const double* det, int reverse, rte_stats* s) {
    const int prec = o->sweep_precision == RTE_FP32 ? RTE_FP32 : RTE_FP64;
    const size_t esz = prec == RTE_FP32 ? sizeof(float) : sizeof(double);
    const int nf = (int)h->fold_rep.size();
    RTE_TRY(ensure_psi_scratch(h, esz * (size_t)nf * h->ndof));
    cudaStream_t st = h->stream;
    const int g = egrid(h, h->ndof);
    s->converged = 0;
    for (int n = 1; n <= o->max_outer; ++n) {
        const bool refine = prec == RTE_FP32 && o->sweep_refine;
        if (!reverse) {
            RTE_TRY(launch_source(h, phi, prec, h->src_w, st));
            if (refine) RTE_TRY(launch_source(h, phi, RTE_FP64, h->src64, st));
        } else if (prec == RTE_FP32) {
            adj_source_kernel<float><<<g, 256, 0, st>>>(h->nc, h->sig_s, phi, det, (float*)h->src_w);
            if (refine) adj_source_kernel<double><<<g, 256, 0, st>>>(h->nc, h->sig_s, phi, det, h->src64);
        } else {
            adj_source_kernel<double><<<g, 256, 0, st>>>(h->nc, h->sig_s, phi, det, (double*)h->src_w);
        }
        RTE_CUDA_TRY(cudaGetLastError());
        void* dpsi = nullptr;
        RTE_TRY(sweep_refined(h, h->d_fold_rep, nf, prec, refine ? 1 : 0, h->src_w, h->src64, reverse ? 0 : 1, reverse,
                              h->psi_w, &dpsi, nullptr, st));
        RTE_TRY(launch_phi_reduce2(h, h->d_fold_w, nf, prec, h->psi_w, dpsi, h->phi_star, st));
        s->total_sweeps += nf * (dpsi ? 2 : 1);
        s->cell_angle_updates += (long long)nf * h->nc * (dpsi ? 2 : 1);
        double diff = 0.0;
        RTE_TRY(max_abs_diff(h, h->phi_star, phi, h->ndof, &diff, st));
        RTE_TRY(check_dep_flag(h, st));
        s->outer_iters = n;
        s->last_diff = diff;
        if (!(diff == diff) || isinf(diff)) return fail(RTE_ERR_NAN, "SI-DSA: non-finite scalar flux");
        if (diff <= o->eps_si) {
            copy_kernel<<<g, 256, 0, st>>>(h->ndof, h->phi_star, phi);
            RTE_CUDA_TRY(cudaGetLastError());
            s->converged = 1;
            break;
        }
        if (o->use_dsa) {
            int it = 0;
            RTE_TRY(dsa_correct(h, o, h->phi_star, phi, &it, st));
            s->dsa_cg_iters += it;
        } else {
            copy_kernel<<<g, 256, 0, st>>>(h->ndof, h->phi_star, phi);
            RTE_CUDA_TRY(cudaGetLastError());
        }
    }
    RTE_CUDA_TRY(cudaStreamSynchronize(st));
    return RTE_OK;
}

// Full-rank SI-DSA over several independent problems in lock step: per outer iteration one
// batched sweep launch covers every unconverged problem's folded ordinates (two with the FP64
// defect correction), one read-back carries every stop test, and one batched cooperative CG
// applies every DSA correction.  A problem leaves the batch when its own stop test passes.
static int fr_batch(rte_handle* const* hs, int nprob, const rte_opts* o, double* const* phi, rte_stats* s) {
    const int prec = o->sweep_precision == RTE_FP32 ? RTE_FP32 : RTE_FP64;
    const size_t esz = prec == RTE_FP32 ? sizeof(float) : sizeof(double);
    const bool refine = prec == RTE_FP32 && o->sweep_refine;
    cudaStream_t st = hs[0]->stream;
    for (int i = 0; i < nprob; ++i) {
        rte_handle* h = hs[i];
        if (h->stream != st) RTE_CUDA_TRY(cudaStreamSynchronize(h->stream));
        const int nf = (int)h->fold_rep.size();
        RTE_TRY(ensure_psi_scratch(h, esz * (size_t)nf * h->ndof));
        if (refine) RTE_TRY(ensure_refine_scratch(h, nf));
        s[i].converged = 0;
    }
    const bool batched = batch_supported(hs, nprob, prec);
    std::vector<int> act(nprob);
    for (int i = 0; i < nprob; ++i) act[i] = i;
    std::vector<rte_handle*> hsub;
    std::vector<const int*> dl;
    std::vector<int> nl;
    std::vector<const void*> srcs;
    std::vector<long long> strides;
    std::vector<void*> outs;
    std::vector<const double*> pstar;
    std::vector<double*> pout;
    std::vector<int> its;
    for (int n = 1; n <= o->max_outer && !act.empty(); ++n) {
        const int m = (int)act.size();
        hsub.resize(m); dl.resize(m); nl.resize(m); srcs.resize(m); strides.assign(m, 0); outs.resize(m);
        for (int k = 0; k < m; ++k) {
            rte_handle* h = hs[act[k]];
            RTE_TRY(launch_source(h, phi[act[k]], prec, h->src_w, st));
            if (refine) RTE_TRY(launch_source(h, phi[act[k]], RTE_FP64, h->src64, st));
            hsub[k] = h;
            dl[k] = h->d_fold_rep;
            nl[k] = (int)h->fold_rep.size();
            srcs[k] = h->src_w;
            outs[k] = h->psi_w;
        }
        if (batched) {
            RTE_TRY(launch_sweep_batch(hsub.data(), m, dl.data(), nl.data(), prec, srcs.data(), strides.data(), 1, 0,
                                       outs.data(), st));
        } else {
            for (int k = 0; k < m; ++k)
                RTE_TRY(launch_sweep(hsub[k], dl[k], nl[k], prec, srcs[k], 0, 1, 0, outs[k], st));
        }
        if (refine) {
            for (int k = 0; k < m; ++k) {
                rte_handle* h = hsub[k];
                RTE_TRY(launch_defect(h, dl[k], nl[k], h->src64, 1, 0, h->psi_w, nullptr, st));
                srcs[k] = h->res_w;
                strides[k] = h->ndof;
                outs[k] = h->dpsi_w;
            }
            if (batched) {
                RTE_TRY(launch_sweep_batch(hsub.data(), m, dl.data(), nl.data(), prec, srcs.data(), strides.data(), 0, 0,
                                           outs.data(), st));
            } else {
                for (int k = 0; k < m; ++k)
                    RTE_TRY(launch_sweep(hsub[k], dl[k], nl[k], prec, srcs[k], strides[k], 0, 0, outs[k], st));
            }
        }
        for (int k = 0; k < m; ++k) {
            rte_handle* h = hsub[k];
            RTE_TRY(launch_phi_reduce2(h, h->d_fold_w, nl[k], prec, h->psi_w, refine ? h->dpsi_w : nullptr, h->phi_star, st));
            RTE_TRY(max_abs_diff_async(h, h->phi_star, phi[act[k]], h->ndof, st));
            RTE_CUDA_TRY(cudaMemcpyAsync(h->h_scalar + 16, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
        }
        RTE_CUDA_TRY(cudaStreamSynchronize(st));
        int timeout = 0;
        for (int k = 0; k < m; ++k) {
            rte_handle* h = hsub[k];
            if (*reinterpret_cast<int*>(h->h_scalar + 16)) {
                RTE_CUDA_TRY(cudaMemsetAsync(h->d_err, 0, sizeof(int), st));
                timeout = 1;
            }
        }
        if (timeout) {
            RTE_CUDA_TRY(cudaStreamSynchronize(st));
            return fail(RTE_ERR_DEP_TIMEOUT, "batched sweep: a band hand-off wait ran out");
        }
        std::vector<int> next;
        pstar.clear(); pout.clear(); hsub.clear();
        for (int k = 0; k < m; ++k) {
            const int i = act[k];
            rte_handle* h = hs[i];
            const double diff = h->h_scalar[0];
            const int mult = refine ? 2 : 1;
            s[i].total_sweeps += nl[k] * mult;
            s[i].cell_angle_updates += (long long)nl[k] * h->nc * mult;
            s[i].outer_iters = n;
            s[i].last_diff = diff;
            if (!(diff == diff) || isinf(diff)) return fail(RTE_ERR_NAN, "batched SI-DSA: non-finite scalar flux");
            if (diff <= o->eps_si) {
                copy_kernel<<<egrid(h, h->ndof), 256, 0, st>>>(h->ndof, h->phi_star, phi[i]);
                s[i].converged = 1;
            } else if (o->use_dsa) {
                next.push_back(i);
                hsub.push_back(h);
                pstar.push_back(h->phi_star);
                pout.push_back(phi[i]);
            } else {
                copy_kernel<<<egrid(h, h->ndof), 256, 0, st>>>(h->ndof, h->phi_star, phi[i]);
                next.push_back(i);
            }
        }
        RTE_CUDA_TRY(cudaGetLastError());
        if (!hsub.empty()) {
            its.assign(hsub.size(), 0);
            RTE_TRY(dsa_correct_batch(hsub.data(), (int)hsub.size(), o, pstar.data(), pout.data(), its.data(), st));
            for (size_t k = 0; k < hsub.size(); ++k) s[next[k]].dsa_cg_iters += its[k];
        }
        act.swap(next);
    }
    RTE_CUDA_TRY(cudaStreamSynchronize(st));
    return RTE_OK;
}

int solve_full_rank(rte_handle* h, const rte_opts* o, double* phi, rte_stats* s) {
    RTE_TRY(fr_loop(h, o, phi, nullptr, 0, s));
    s->final_rank = (int)h->fold_rep.size();
    s->max_rank = s->final_rank;
    return s->converged ? RTE_OK : fail(RTE_ERR_NOT_CONVERGED, "SI-DSA: max_outer reached");
}

}  // namespace rte

using namespace rte;

static int check_opts(const rte_opts* o) {
    if (!o) return fail(RTE_ERR_ARG, "null options");
    if (o->mode != RTE_MODE_FR && o->mode != RTE_MODE_LR) return fail(RTE_ERR_ARG, "bad mode");
    if (o->sweep_precision != RTE_FP32 && o->sweep_precision != RTE_FP64) return fail(RTE_ERR_ARG, "bad precision");
    if (o->basis_precision != RTE_FP64 && o->basis_precision != RTE_DWF32)
        return fail(RTE_ERR_ARG, "basis_precision must be RTE_FP64 or RTE_DWF32");
    if (!(o->eps_si >= 0) || o->max_outer < 1 || o->dsa_max_iter < 0 || !(o->dsa_tol >= 0))
        return fail(RTE_ERR_ARG, "bad tolerances or iteration limits");
    if (o->mode == RTE_MODE_LR && (o->p < 1 || o->p > 64 || o->q < o->p || o->m_max < 0 || o->m_max > 16 ||
                                   o->max_inner < 1))
        return fail(RTE_ERR_ARG, "low-rank options need 1 <= p <= q, p <= 64, 0 <= m_max <= 16");
    if (o->mode == RTE_MODE_LR && (o->tc_projection != 0 && o->tc_projection != 1))
        return fail(RTE_ERR_ARG, "tc_projection must be 0 or 1");
    if (o->mode == RTE_MODE_LR && o->sampling != RTE_SAMPLE_RESIDUAL && o->sampling != RTE_SAMPLE_DEIM)
        return fail(RTE_ERR_ARG, "sampling must be RTE_SAMPLE_RESIDUAL or RTE_SAMPLE_DEIM");
    if (o->mode == RTE_MODE_LR && (o->basis_update < RTE_UPDATE_MGS2A || o->basis_update > RTE_UPDATE_QR))
        return fail(RTE_ERR_ARG, "basis_update must be RTE_UPDATE_MGS2A, RTE_UPDATE_MGSQR or RTE_UPDATE_QR");
    return RTE_OK;
}

extern "C" int rte_si_dsa_solve(rte_handle* h, const rte_opts* o, double* phi, rte_stats* stats) {
    if (!h || !phi) return fail(RTE_ERR_ARG, "rte_si_dsa_solve: null argument");
    RTE_TRY(check_opts(o));
    rte_stats s;
    memset(&s, 0, sizeof(s));
    int rc = o->mode == RTE_MODE_FR ? solve_full_rank(h, o, phi, &s) : solve_low_rank(h, o, phi, &s);
    s.status = rc;
    h->last = s;
    if (stats) *stats = s;
    return rc;
}

extern "C" int rte_get_factors(rte_handle* h, const double** X, const double** S, const double** V, int* rank) {
    if (!h) return fail(RTE_ERR_ARG, "rte_get_factors: null handle");
    if (!h->lr.fX || h->lr.factor_rank <= 0) return fail(RTE_ERR_STATE, "rte_get_factors: no factors (run an LR solve with want_factors = 1)");
    if (X) *X = h->lr.fX;
    if (S) *S = h->lr.fS;
    if (V) *V = h->lr.fV;
    if (rank) *rank = h->lr.factor_rank;
    return RTE_OK;
}

extern "C" int rte_get_lowrank_state(rte_handle* h, int* rank, int* ld, const double** X, const double** Pxm,
                                     const double** Pym, const double** T) {
    if (!h) return fail(RTE_ERR_ARG, "rte_get_lowrank_state: null handle");
    if (!h->lr.X || h->lr.last_rank <= 0)
        return fail(RTE_ERR_STATE, "rte_get_lowrank_state: no low-rank solve has left a basis");
    if (rank) *rank = h->lr.last_rank;
    if (ld) *ld = h->lr.r_cap;
    if (X) *X = h->lr.X;
    if (Pxm) *Pxm = h->lr.Pxm;
    if (Pym) *Pym = h->lr.Pym;
    if (T) *T = h->lr.T;
    return RTE_OK;
}

extern "C" int rte_adjoint_grad(rte_handle* h, const rte_opts* o, const double* phi, const double* det, double* d_sig_t,
                                double* d_sig_s, double* d_q, rte_stats* stats) {
    if (!h || !phi || !det) return fail(RTE_ERR_ARG, "rte_adjoint_grad: null argument");
    RTE_TRY(check_opts(o));
    rte_stats s;
    memset(&s, 0, sizeof(s));
    cudaStream_t st = h->stream;
    const int prec = o->sweep_precision == RTE_FP32 ? RTE_FP32 : RTE_FP64;
    const size_t esz = prec == RTE_FP32 ? sizeof(float) : sizeof(double);
    const int nf = (int)h->fold_rep.size();
    const size_t block = esz * (size_t)nf * h->ndof;
    // chi: adjoint scalar flux by SI-DSA on the transposed system (reversed sweeps, no inflow)
    double* chi = nullptr;
    void* mu = nullptr;
    void* psi = nullptr;
    RTE_TRY(h->arena.alloc((void**)&chi, sizeof(double) * h->ndof));
    RTE_CUDA_TRY(cudaMemsetAsync(chi, 0, sizeof(double) * h->ndof, st));
    RTE_TRY(fr_loop(h, o, chi, det, 1, &s));
    if (!s.converged) return fail(RTE_ERR_NOT_CONVERGED, "adjoint SI-DSA: max_outer reached");
    RTE_TRY(h->arena.alloc(&mu, block));
    RTE_TRY(h->arena.alloc(&psi, block));
    const int g = egrid(h, h->ndof);
    // psi_j from phi (forward sweep), mu_j from d + Sigma_s chi (reversed sweep)
    RTE_TRY(launch_source(h, phi, prec, h->src_w, st));
    RTE_TRY(launch_sweep(h, h->d_fold_rep, nf, prec, h->src_w, 0, 1, 0, psi, st));
    if (prec == RTE_FP32)
        adj_source_kernel<float><<<g, 256, 0, st>>>(h->nc, h->sig_s, chi, det, (float*)h->src_w);
    else
        adj_source_kernel<double><<<g, 256, 0, st>>>(h->nc, h->sig_s, chi, det, (double*)h->src_w);
    RTE_CUDA_TRY(cudaGetLastError());
    RTE_TRY(launch_sweep(h, h->d_fold_rep, nf, prec, h->src_w, 0, 0, 1, mu, st));
    s.total_sweeps += 2 * nf;
    s.cell_angle_updates += 2ll * nf * h->nc;
    const int gc = egrid(h, h->nc);
    const double cellint = sqrt(h->hx * h->hy);
    if (prec == RTE_FP32)
        grad_kernel<float><<<gc, 256, 0, st>>>(h->nc, nf, h->ndof, h->d_fold_w, (const float*)psi, (const float*)mu, chi, phi,
                                               cellint, d_sig_t, d_sig_s, d_q);
    else
        grad_kernel<double><<<gc, 256, 0, st>>>(h->nc, nf, h->ndof, h->d_fold_w, (const double*)psi, (const double*)mu, chi,
                                                phi, cellint, d_sig_t, d_sig_s, d_q);
    RTE_CUDA_TRY(cudaGetLastError());
    RTE_CUDA_TRY(cudaStreamSynchronize(st));
    // the three temporaries go back to the device right away
    for (void* p : {(void*)chi, mu, psi}) {
        auto& v = h->arena.ptrs;
        v.erase(std::remove(v.begin(), v.end(), p), v.end());
        dev_free(p);
    }
    s.status = RTE_OK;
    s.converged = 1;
    if (stats) *stats = s;
    return RTE_OK;
}

// Low-rank SI-DSA of a batch of independent problems (no paper counterpart).  Each problem's
// inner loop is a chain of small dependent launches (a few sweeps of p ordinates, passes over
// an N_x x r basis), which fills a fraction of the GPU.  The problems therefore run
// concurrently: a pool of host threads, each with its own non-blocking stream, takes problems
// largest first and runs the single-problem solve on that stream (its graph-captured inner
// iterations, its per-iteration status read).  Uneven ranks need no lock step: a thread whose
// problem converged takes the next one.  The CG schedules and the p-ordinate sweeps are tuned
// one handle at a time beforehand, so that concurrent work does not disturb their timing.  A graph capture of one
// thread runs while the others wait for their streams or at the batch's gate (BatchGate).
constexpr int kLrBatchThreads = 32;   // host threads (and streams) of a low-rank batch

// Lazy module loading (the CUDA default) loads a kernel at its first launch, and the load
// synchronises the context, which invalidates a stream capture in progress on another host
// thread.  Before the solves of a low-rank batch run on several threads, every kernel of the
// library is loaded into the current context: an anchor kernel of each translation unit gives
// its CUDA library (cuKernelGetLibrary), whose kernels are enumerated and loaded
// (cuKernelGetFunction).  Returns false if the CUDA driver library lacks one of these entry points; the batch
// then runs its solves one after the other on one thread.
static bool preload_all_kernels() {
    static std::mutex mu;
    static std::vector<int> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return false; }
    std::lock_guard<std::mutex> guard(mu);
    if (std::find(done.begin(), done.end(), dev) != done.end()) return true;
    typedef CUresult (*KernelGetLibrary)(CUlibrary*, CUkernel);
    typedef CUresult (*LibraryGetKernelCount)(unsigned int*, CUlibrary);
    typedef CUresult (*LibraryEnumerateKernels)(CUkernel*, unsigned int, CUlibrary);
    typedef CUresult (*KernelGetFunction)(CUfunction*, CUkernel);
    auto entry = [](const char* name, int version) -> void* {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion(name, &p, version, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return p;
    };
    auto get_library = (KernelGetLibrary)entry("cuKernelGetLibrary", 12050);
    auto kernel_count = (LibraryGetKernelCount)entry("cuLibraryGetKernelCount", 12040);
    auto enumerate = (LibraryEnumerateKernels)entry("cuLibraryEnumerateKernels", 12040);
    auto get_function = (KernelGetFunction)entry("cuKernelGetFunction", 12000);
    if (!get_library || !kernel_count || !enumerate || !get_function) return false;
    const void* anchors[] = {(const void*)copy_kernel, sweep_kernel_anchor(), dsa_kernel_anchor(), tc_kernel_anchor(),
                             lowrank_kernel_anchor()};
    for (const void* a : anchors) {
        cudaKernel_t k = nullptr;
        if (cudaGetKernel(&k, a) != cudaSuccess) { cudaGetLastError(); return false; }
        CUlibrary lib = nullptr;
        unsigned int n = 0;
        if (get_library(&lib, (CUkernel)k) != CUDA_SUCCESS || kernel_count(&n, lib) != CUDA_SUCCESS) return false;
        std::vector<CUkernel> ks(n);
        if (n && enumerate(ks.data(), n, lib) != CUDA_SUCCESS) return false;
        for (CUkernel kk : ks) {
            CUfunction f = nullptr;
            if (get_function(&f, kk) != CUDA_SUCCESS) return false;
        }
    }
    done.push_back(dev);
    return true;
}

static int lr_batch(rte_handle* const* hs, int nprob, const rte_opts* o, double* const* phi, rte_stats* s) {
    const int sprec = o->sweep_precision == RTE_FP32 ? RTE_FP32 : RTE_FP64;
    for (int i = 0; i < nprob; ++i) {
        if (o->use_dsa) RTE_TRY(dsa_pretune(hs[i], o->dsa_precision));
        RTE_TRY(sweep_pretune(hs[i], sprec, o->p, 1, hs[i]->stream));
    }
    std::vector<int> order(nprob);
    for (int i = 0; i < nprob; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (long long)hs[a]->ndof * hs[a]->nang > (long long)hs[b]->ndof * hs[b]->nang;
    });
    const unsigned hc = std::max(1u, std::thread::hardware_concurrency());
    const int nthreads = preload_all_kernels() ? std::min({nprob, kLrBatchThreads, (int)hc}) : 1;
    // ordering: each problem's solve starts after the work queued on its handle's stream and
    // that stream waits for the solve's end
    std::vector<cudaEvent_t> ev_in(nprob, nullptr), ev_out(nprob, nullptr);
    std::vector<cudaStream_t> ws(nthreads, nullptr);
    auto cleanup = [&]() {
        for (auto& e : ev_in) if (e) cudaEventDestroy(e);
        for (auto& e : ev_out) if (e) cudaEventDestroy(e);
        for (auto& w : ws) if (w) cudaStreamDestroy(w);
    };
    for (int i = 0; i < nprob; ++i) {
        if (cudaEventCreateWithFlags(&ev_in[i], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev_out[i], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventRecord(ev_in[i], hs[i]->stream) != cudaSuccess) {
            cleanup();
            return fail(RTE_ERR_CUDA, "batched low-rank SI-DSA: event setup failed");
        }
    }
    for (auto& w : ws)
        if (cudaStreamCreateWithFlags(&w, cudaStreamNonBlocking) != cudaSuccess) {
            cleanup();
            return fail(RTE_ERR_CUDA, "batched low-rank SI-DSA: stream creation failed");
        }
    std::atomic<int> next{0};
    std::vector<int> rc(nprob, RTE_OK);
    std::vector<std::string> msg(nprob);
    BatchGate gate;
    auto worker = [&](int t) {
        cudaSetDevice(hs[0]->device);
        tl_gate = nthreads > 1 ? &gate : nullptr;
        for (;;) {
            const int i = next.fetch_add(1);
            if (i >= nprob) break;
            const int k = order[i];
            rte_handle* h = hs[k];
            const cudaStream_t own = h->stream;
            int r = cudaStreamWaitEvent(ws[t], ev_in[k], 0) == cudaSuccess ? RTE_OK : RTE_ERR_CUDA;
            if (r == RTE_OK) {
                h->stream = ws[t];           // the handle is used by this thread alone meanwhile
                if (tl_gate) tl_gate->enter();
                r = solve_low_rank(h, o, phi[k], &s[k]);
                if (tl_gate) tl_gate->leave();
                h->stream = own;
            }
            if (cudaEventRecord(ev_out[k], ws[t]) != cudaSuccess && r == RTE_OK) r = RTE_ERR_CUDA;
            rc[k] = r;
            if (r != RTE_OK) msg[k] = rte_last_error();
        }
        tl_gate = nullptr;
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nthreads; ++t) pool.emplace_back(worker, t);
    worker(0);
    for (auto& th : pool) th.join();
    for (int i = 0; i < nprob; ++i) cudaStreamWaitEvent(hs[i]->stream, ev_out[i], 0);
    for (auto& w : ws) cudaStreamSynchronize(w);
    cleanup();
    // first hard error (a problem that ran out of outer iterations is reported in its stats)
    for (int i = 0; i < nprob; ++i)
        if (rc[i] != RTE_OK && rc[i] != RTE_ERR_NOT_CONVERGED) {
            set_error("batched low-rank SI-DSA, problem " + std::to_string(i) + ": " + msg[i]);
            return rc[i];
        }
    return RTE_OK;
}

extern "C" int rte_si_dsa_solve_batch(rte_handle* const* hs, int nprob, const rte_opts* o, double* const* phi,
                                      rte_stats* stats) {
    if (!hs || nprob < 1 || !phi) return fail(RTE_ERR_ARG, "rte_si_dsa_solve_batch: null argument");
    RTE_TRY(check_opts(o));
    for (int i = 0; i < nprob; ++i) {
        if (!hs[i] || !phi[i]) return fail(RTE_ERR_ARG, "rte_si_dsa_solve_batch: null entry");
        for (int k = 0; k < i; ++k)
            if (hs[k] == hs[i] || phi[k] == phi[i]) return fail(RTE_ERR_ARG, "rte_si_dsa_solve_batch: a handle or phi appears twice");
    }
    std::vector<rte_stats> s(nprob);
    for (auto& x : s) memset(&x, 0, sizeof(x));
    for (int i = 0; i < nprob; ++i)
        if (hs[i]->device != hs[0]->device) return fail(RTE_ERR_ARG, "rte_si_dsa_solve_batch: handles on different devices");
    int rc;
    if (o->mode == RTE_MODE_FR) {
        rc = fr_batch(hs, nprob, o, phi, s.data());
        for (int i = 0; i < nprob; ++i) s[i].final_rank = s[i].max_rank = (int)hs[i]->fold_rep.size();
    } else {
        rc = lr_batch(hs, nprob, o, phi, s.data());
    }
    int all = 1;
    for (int i = 0; i < nprob; ++i) all &= s[i].converged;
    if (rc == RTE_OK && !all) rc = fail(RTE_ERR_NOT_CONVERGED, "batched SI-DSA: max_outer reached for some problem");
    for (int i = 0; i < nprob; ++i) {
        s[i].status = rc;
        hs[i]->last = s[i];
        if (stats) stats[i] = s[i];
    }
    return rc;
}

// The low-rank step (Alg. 1 on the step's steady problem): the time source F of the distinct
// directions, the shifted medium, solve_low_rank with F, psi^{n+1} = X C.
static int be_step_lowrank(rte_handle* h, const rte_opts* o, double inv_dt, const double* psi_prev, double* psi_next,
                           double* phi, rte_stats* stats) {
    rte_stats s;
    memset(&s, 0, sizeof(s));
    cudaStream_t st = h->stream;
    const long long N = h->ndof;
    const int ndir = (int)h->fold_rep.size();
    std::vector<int> pairs;
    for (int j = 0; j < h->nang; ++j)
        if (h->twin[j] > j) { pairs.push_back(j); pairs.push_back(h->twin[j]); }
    double* F = nullptr;
    int* d_pairs = nullptr;
    int* flag = nullptr;
    std::vector<void*> temps;
    auto release = [&]() {
        cudaStreamSynchronize(st);
        for (void* p : temps) {
            auto& v = h->arena.ptrs;
            v.erase(std::remove(v.begin(), v.end(), p), v.end());
            dev_free(p);
        }
    };
    int rc = h->arena.alloc((void**)&F, sizeof(double) * (size_t)ndir * N);
    if (rc == RTE_OK) { temps.push_back(F); rc = h->arena.alloc((void**)&flag, sizeof(int)); }
    if (rc == RTE_OK) { temps.push_back(flag); rc = h->arena.alloc((void**)&d_pairs, sizeof(int) * std::max<size_t>(2, pairs.size())); }
    if (rc == RTE_OK) temps.push_back(d_pairs);
    int mismatch = 0;
    if (rc == RTE_OK) {
        const int npairs = (int)pairs.size() / 2;
        if (cudaMemsetAsync(flag, 0, sizeof(int), st) != cudaSuccess ||
            (npairs && cudaMemcpyAsync(d_pairs, pairs.data(), sizeof(int) * pairs.size(), cudaMemcpyHostToDevice, st) !=
                           cudaSuccess))
            rc = fail(RTE_ERR_CUDA, "rte_be_step: scratch setup");
        if (rc == RTE_OK && npairs)
            twin_mismatch_kernel<<<egrid(h, npairs * N), 256, 0, st>>>(npairs, N, d_pairs, psi_prev, flag);
        if (rc == RTE_OK) be_fsrc_kernel<<<egrid(h, ndir * N), 256, 0, st>>>(ndir, N, h->d_fold_rep, psi_prev, inv_dt, F);
        if (rc == RTE_OK && (cudaGetLastError() != cudaSuccess ||
                             cudaMemcpyAsync(&mismatch, flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                             cudaStreamSynchronize(st) != cudaSuccess))
            rc = fail(RTE_ERR_CUDA, "rte_be_step: time source");
        if (rc == RTE_OK && mismatch)
            rc = fail(RTE_ERR_ARG, "rte_be_step: the low-rank step needs psi_prev equal on +-Omega_z twin pairs");
    }
    if (rc != RTE_OK) { release(); return rc; }
    const std::vector<double> sig_t0 = h->sig_t_h;
    for (double& v : h->sig_t_h) v += inv_dt;
    h->lr.ready = false;
    rc = upload_materials(h);
    if (rc == RTE_OK) rc = solve_low_rank(h, o, phi, &s, F, psi_next);
    h->sig_t_h = sig_t0;
    const int rc2 = upload_materials(h);
    h->lr.ready = false;
    release();
    if (rc == RTE_OK) rc = rc2;
    s.status = rc;
    h->last = s;
    if (stats) *stats = s;
    return rc;
}

extern "C" int rte_be_step(rte_handle* h, const rte_opts* o, double dt, const double* psi_prev, double* psi_next,
                           double* phi, rte_stats* stats) {
    if (!h || !o || !psi_prev || !psi_next || !phi) return fail(RTE_ERR_ARG, "rte_be_step: null argument");
    RTE_TRY(check_opts(o));
    if (!(dt > 0.0) || !isfinite(dt)) return fail(RTE_ERR_ARG, "rte_be_step: need a finite dt > 0");
    if (o->sweep_precision == RTE_FP32 && o->sweep_refine)
        return fail(RTE_ERR_ARG, "rte_be_step: FP32 sweeps without the defect correction (sweep_refine = 0)");
    rte_stats s;
    memset(&s, 0, sizeof(s));
    const int prec = o->sweep_precision == RTE_FP32 ? RTE_FP32 : RTE_FP64;
    const size_t esz = prec == RTE_FP32 ? sizeof(float) : sizeof(double);
    const size_t block = esz * (size_t)h->nang * h->ndof;
    cudaStream_t st = h->stream;
    const double inv_dt = 1.0 / dt;
    if (o->mode == RTE_MODE_LR) return be_step_lowrank(h, o, inv_dt, psi_prev, psi_next, phi, stats);
    void *src = nullptr, *psi = nullptr, *iota = nullptr;
    std::vector<void*> temps;
    auto release = [&]() {
        cudaStreamSynchronize(st);
        for (void* p : temps) {
            auto& v = h->arena.ptrs;
            v.erase(std::remove(v.begin(), v.end(), p), v.end());
            dev_free(p);
        }
    };
    int rc = h->arena.alloc(&src, block);
    if (rc == RTE_OK) { temps.push_back(src); rc = h->arena.alloc(&psi, block); }
    if (rc == RTE_OK) { temps.push_back(psi); rc = h->arena.alloc(&iota, sizeof(int) * (size_t)h->nang); }
    if (rc == RTE_OK) {
        temps.push_back(iota);
        std::vector<int> idx(h->nang);
        for (int j = 0; j < h->nang; ++j) idx[j] = j;
        if (cudaMemcpyAsync(iota, idx.data(), sizeof(int) * h->nang, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = fail(RTE_ERR_CUDA, "rte_be_step: upload of the ordinate list");
    }
    if (rc != RTE_OK) { release(); return rc; }
    // the step's medium: sigma_t + 1/dt in every cell (sweeps, defect-free FP32 copy, DSA)
    const std::vector<double> sig_t0 = h->sig_t_h;
    for (double& v : h->sig_t_h) v += inv_dt;
    rc = upload_materials(h);
    if (rc == RTE_OK) rc = be_loop(h, o, inv_dt, psi_prev, phi, src, psi, (int*)iota, &s);
    if (rc == RTE_OK) {
        const long long n = (long long)h->nang * h->ndof;
        if (prec == RTE_FP32) to_double_kernel<float><<<egrid(h, n), 256, 0, st>>>(n, (const float*)psi, psi_next);
        else to_double_kernel<double><<<egrid(h, n), 256, 0, st>>>(n, (const double*)psi, psi_next);
        if (cudaGetLastError() != cudaSuccess) rc = fail(RTE_ERR_CUDA, "rte_be_step: psi copy");
    }
    // back to the steady problem's medium
    h->sig_t_h = sig_t0;
    const int rc2 = upload_materials(h);
    h->lr.ready = false;
    release();
    if (rc == RTE_OK) rc = rc2;
    if (rc == RTE_OK && !s.converged) rc = fail(RTE_ERR_NOT_CONVERGED, "backward-Euler step: max_outer reached");
    s.status = rc;
    s.final_rank = s.max_rank = h->nang;
    h->last = s;
    if (stats) *stats = s;
    return rc;
}
