// Problem setup: CL quadrature (App. A), source moments and inflow-face vectors of the
// upwind DG-Q1 system (Sec. 2.1, App. B), device upload, and the handle life cycle.
//
// Basis: orthonormal tensor Legendre on each cell, eta_{ij}(x,y) = P_i(x) Q_j(y) with
// P_0 = 1/sqrt(hx), P_1 = sqrt(3) xi / sqrt(hx), xi = 2 (x - xc)/hx (likewise Q_j in y);
// local DOF m = i + 2 j.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "rte_internal.cuh"

namespace rte {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
    set_error(msg);
    return code;
}

std::shared_mutex& alloc_capture_mutex() {
    static std::shared_mutex m;
    return m;
}
thread_local int tl_capture_depth = 0;
thread_local int tl_alloc_depth = 0;

thread_local BatchGate* tl_gate = nullptr;
thread_local int tl_gate_capture_depth = 0;

void BatchGate::enter() {
    std::unique_lock<std::mutex> l(m_);
    cv_.wait(l, [&] { return !capturing_ && waiting_ == 0; });
    ++active_;
}

void BatchGate::leave() {
    std::unique_lock<std::mutex> l(m_);
    if (--active_ == 0) cv_.notify_all();
}

void BatchGate::capture_begin() {
    std::unique_lock<std::mutex> l(m_);
    ++waiting_;
    cv_.wait(l, [&] { return !capturing_ && active_ == 0; });
    --waiting_;
    capturing_ = true;
}

void BatchGate::capture_end() {
    std::unique_lock<std::mutex> l(m_);
    capturing_ = false;
    cv_.notify_all();
}

cudaError_t gate_stream_sync(cudaStream_t st) {
    if (!tl_gate || tl_gate_capture_depth) return cudaStreamSynchronize(st);
    tl_gate->leave();
    const cudaError_t e = cudaStreamSynchronize(st);
    tl_gate->enter();
    return e;
}

int smem_optin(const void* func, size_t bytes) {
    if (bytes <= 48 * 1024) return RTE_OK;
    static std::mutex mu;
    static std::set<std::pair<int, const void*>> done;
    int dev = 0;
    RTE_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> guard(mu);
    if (done.count({dev, func})) return RTE_OK;
    int optin = 0;
    RTE_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    RTE_CUDA_TRY(cudaFuncGetAttributes(&fa, func));
    const int max_dynamic = optin - (int)fa.sharedSizeBytes;     // static shared memory counts too
    if (bytes > (size_t)max_dynamic) return fail(RTE_ERR_ARG, "kernel needs more shared memory than the device offers");
    RTE_CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dynamic));
    done.insert({dev, func});
    return RTE_OK;
}

void dev_free(void* p) {
    if (!p) return;
    AllocLock lk;
    cudaFree(p);
}

cudaError_t pinned_alloc(void** p, size_t n) {
    AllocLock lk;
    return cudaMallocHost(p, n);
}

void pinned_free(void* p) {
    if (!p) return;
    AllocLock lk;
    cudaFreeHost(p);
}

int DeviceArena::alloc(void** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 16;
    AllocLock lk;
    cudaError_t e = cudaMalloc(p, n);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(RTE_ERR_NOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    ptrs.push_back(*p);
    bytes += n;
    return RTE_OK;
}

int DeviceArena::grow(void** buf, size_t* cap, size_t need) {
    if (*buf && *cap >= need) return RTE_OK;
    AllocLock lk;
    if (*buf) {
        // work queued earlier may still read the old block
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return fail(RTE_ERR_CUDA, std::string("grow: ") + cudaGetErrorString(e));
        ptrs.erase(std::remove(ptrs.begin(), ptrs.end(), *buf), ptrs.end());
        dev_free(*buf);
        *buf = nullptr;
        *cap = 0;
    }
    RTE_TRY(alloc(buf, need));
    *cap = need;
    return RTE_OK;
}

void DeviceArena::release_all() {
    AllocLock lk;
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
    bytes = 0;
}

// n-point Gauss-Legendre rule on [-1, 1] by Newton iteration on P_n (nodes mirrored so that
// x_{n-1-k} = -x_k exactly), weights 2 / ((1 - x^2) P_n'(x)^2).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int k = 0; k < (n + 1) / 2; ++k) {
        double z = cos(M_PI * (k + 0.75) / (n + 0.5));   // near the k-th largest root
        double p0 = 1.0, p1 = z, dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            p0 = 1.0;
            p1 = z;                       // P_1
            for (int m = 2; m <= n; ++m) {
                double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
                p0 = p1;
                p1 = p2;
            }                             // p1 = P_n(z), p0 = P_{n-1}(z)
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        p0 = 1.0;
        p1 = z;
        for (int m = 2; m <= n; ++m) {
            double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        double wk = 2.0 / ((1.0 - z * z) * dp * dp);
        x[n - 1 - k] = z;                 // ascending order, mirrored exactly
        x[k] = -z;
        w[k] = w[n - 1 - k] = wk;
    }
    if (n % 2 == 1) x[n / 2] = 0.0;
}

// int_a^b P_i(x) dx for the cell [c0, c0 + h] (closed form).
static inline void moment1d(double a, double b, double c0, double h, double out[2]) {
    double xc = c0 + 0.5 * h;
    double sh = sqrt(h);
    out[0] = (b - a) / sh;
    out[1] = sqrt(3.0) * ((b - xc) * (b - xc) - (a - xc) * (a - xc)) / (h * sh);
}

// int_a^b exp(-al (x - g)^2) dx, from erf or erfc so that the difference keeps its relative
// accuracy in the tails (both arguments of one sign).
static inline double gauss_int(double al, double g, double a, double b) {
    const double s = sqrt(al), u0 = s * (a - g), u1 = s * (b - g);
    double d;
    if (u0 >= 0.0) d = erfc(u0) - erfc(u1);
    else if (u1 <= 0.0) d = erfc(-u1) - erfc(-u0);
    else d = erf(u1) - erf(u0);
    return 0.5 * sqrt(M_PI / al) * d;
}

// Moments of exp(-al (x - g)^2) against the two 1D Legendre modes of the cell [c0, c0 + h]
// (the same normalisation as moment1d): int e P_0 and int e P_1, P_1 ~ 2 (x - xm) / h, with
// int (x - g) e dx = (e(a) - e(b)) / (2 al) in closed form.
static inline void gauss_moment1d(double al, double g, double c0, double h, double out[2]) {
    const double a = c0, b = c0 + h, xm = c0 + 0.5 * h, sh = sqrt(h);
    const double m0 = gauss_int(al, g, a, b);
    const double m1 = (exp(-al * (a - g) * (a - g)) - exp(-al * (b - g) * (b - g))) / (2.0 * al);
    out[0] = m0 / sh;
    out[1] = 2.0 * sqrt(3.0) * (m1 + (g - xm) * m0) / (h * sh);
}

static void source_moments(const rte_handle* h, std::vector<double>& G) {
    G.assign((size_t)h->ndof, 0.0);
    const double cell = sqrt(h->hx * h->hy);
    if (h->has_q)
        for (int c = 0; c < h->nc; ++c) G[4 * (size_t)c] = h->q_h[c] * cell;
    const int nr = (int)(h->rects.size() / 5);
    for (int r = 0; r < nr; ++r) {
        const double* R = &h->rects[5 * r];
        double rx0 = R[0], rx1 = R[1], ry0 = R[2], ry1 = R[3], val = R[4];
        int ia0 = std::max(0, (int)floor((rx0 - h->x0) / h->hx) - 1);
        int ia1 = std::min(h->nx, (int)ceil((rx1 - h->x0) / h->hx) + 1);
        int ib0 = std::max(0, (int)floor((ry0 - h->y0) / h->hy) - 1);
        int ib1 = std::min(h->ny, (int)ceil((ry1 - h->y0) / h->hy) + 1);
        for (int ib = ib0; ib < ib1; ++ib) {
            double cy0 = h->y0 + ib * h->hy;
            double oy0 = std::max(cy0, ry0), oy1 = std::min(cy0 + h->hy, ry1);
            if (oy1 <= oy0) continue;
            double my[2];
            moment1d(oy0, oy1, cy0, h->hy, my);
            for (int ia = ia0; ia < ia1; ++ia) {
                double cx0 = h->x0 + ia * h->hx;
                double ox0 = std::max(cx0, rx0), ox1 = std::min(cx0 + h->hx, rx1);
                if (ox1 <= ox0) continue;
                double mx[2];
                moment1d(ox0, ox1, cx0, h->hx, mx);
                size_t c = (size_t)ib * h->nx + ia;
                for (int j = 0; j < 2; ++j)
                    for (int i = 0; i < 2; ++i) G[4 * c + i + 2 * j] += val * mx[i] * my[j];
            }
        }
    }
    // Gaussian sources amp exp(-al ((x - gx)^2 + (y - gy)^2)): separable, exact per cell
    const int ng = (int)(h->gauss.size() / 4);
    std::vector<double> gxm(2 * (size_t)h->nx), gym(2 * (size_t)h->ny);
    for (int r = 0; r < ng; ++r) {
        const double gx = h->gauss[4 * r], gy = h->gauss[4 * r + 1], al = h->gauss[4 * r + 2],
                     amp = h->gauss[4 * r + 3];
        for (int ia = 0; ia < h->nx; ++ia) gauss_moment1d(al, gx, h->x0 + ia * h->hx, h->hx, &gxm[2 * ia]);
        for (int ib = 0; ib < h->ny; ++ib) gauss_moment1d(al, gy, h->y0 + ib * h->hy, h->hy, &gym[2 * ib]);
        for (int ib = 0; ib < h->ny; ++ib)
            for (int ia = 0; ia < h->nx; ++ia) {
                const size_t c = (size_t)ib * h->nx + ia;
                for (int j = 0; j < 2; ++j)
                    for (int i = 0; i < 2; ++i) G[4 * c + i + 2 * j] += amp * gxm[2 * ia + i] * gym[2 * ib + j];
            }
    }
}

// e_side(k) = int eta_k over the boundary faces of the boundary cells of one side.
static void side_vectors(const rte_handle* h, std::vector<double>& e) {
    e.assign(4 * (size_t)h->ndof, 0.0);
    const double rx = sqrt(h->hy / h->hx), ry = sqrt(h->hx / h->hy), s3 = sqrt(3.0);
    double* eL = &e[0];
    double* eR = &e[(size_t)h->ndof];
    double* eB = &e[2 * (size_t)h->ndof];
    double* eT = &e[3 * (size_t)h->ndof];
    for (int iy = 0; iy < h->ny; ++iy) {
        size_t cl = (size_t)iy * h->nx, cr = cl + h->nx - 1;
        eL[4 * cl] = rx;
        eL[4 * cl + 1] = -s3 * rx;
        eR[4 * cr] = rx;
        eR[4 * cr + 1] = s3 * rx;
    }
    for (int ix = 0; ix < h->nx; ++ix) {
        size_t cb = ix, ct = (size_t)(h->ny - 1) * h->nx + ix;
        eB[4 * cb] = ry;
        eB[4 * cb + 2] = -s3 * ry;
        eT[4 * ct] = ry;
        eT[4 * ct + 2] = s3 * ry;
    }
}

int upload_materials(rte_handle* h) {
    std::vector<float> stf(h->nc), sdw(2 * (size_t)h->nc);
    for (int c = 0; c < h->nc; ++c) {
        stf[c] = (float)h->sig_t_h[c];
        sdw[c] = stf[c];                                              // double-word hi
        sdw[h->nc + c] = (float)(h->sig_t_h[c] - (double)stf[c]);     // and lo
    }
    std::vector<double> G;
    source_moments(h, G);
    RTE_CUDA_TRY(cudaMemcpyAsync(h->sig_t, h->sig_t_h.data(), sizeof(double) * h->nc, cudaMemcpyHostToDevice, h->stream));
    RTE_CUDA_TRY(cudaMemcpyAsync(h->sig_s, h->sig_s_h.data(), sizeof(double) * h->nc, cudaMemcpyHostToDevice, h->stream));
    RTE_CUDA_TRY(cudaMemcpyAsync(h->sig_t_f, stf.data(), sizeof(float) * h->nc, cudaMemcpyHostToDevice, h->stream));
    RTE_CUDA_TRY(cudaMemcpyAsync(h->sig_dw, sdw.data(), sizeof(float) * 2 * h->nc, cudaMemcpyHostToDevice, h->stream));
    RTE_CUDA_TRY(cudaMemcpyAsync(h->G, G.data(), sizeof(double) * h->ndof, cudaMemcpyHostToDevice, h->stream));
    RTE_TRY(dsa_prepare(h));
    RTE_CUDA_TRY(cudaStreamSynchronize(h->stream));   // host vectors above are temporaries
    return RTE_OK;
}

static int check_materials(int nc, const double* st, const double* ss) {
    for (int c = 0; c < nc; ++c) {
        if (!(st[c] > 0.0) || !(ss[c] >= 0.0) || ss[c] > st[c] || !isfinite(st[c]))
            return fail(RTE_ERR_ARG, "materials must satisfy sigma_t > 0 and 0 <= sigma_s <= sigma_t (cell " +
                                         std::to_string(c) + ")");
    }
    return RTE_OK;
}

}  // namespace rte

using namespace rte;

extern "C" {

const char* rte_last_error(void) { return rte::g_last_error.c_str(); }

void rte_default_opts(rte_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->mode = RTE_MODE_FR;
    o->sweep_precision = RTE_FP64;
    o->eps_si = 1e-6;
    o->eps_res = 1e-7;
    o->eps_diff = 1e-7;
    o->eps_svd = 1e-8;
    o->eps_mgs = 1e-10;
    o->eps_break = 1e-12;
    o->dsa_tol = 1e-12;
    o->dsa_max_iter = 20000;
    o->use_dsa = 1;
    o->p = 1;
    o->q = 8;
    o->m_max = 4;
    o->mgs_test = 0;
    o->max_outer = 100;
    o->max_inner = 100000;
    o->truncate = 1;
    o->want_factors = 0;
    o->seed = 20260101ull;
    o->sweep_refine = 1;
}

int rte_setup(const rte_problem* p, void* stream, rte_handle** out) {
    if (!p || !out) return fail(RTE_ERR_ARG, "rte_setup: null argument");
    *out = nullptr;
    if (p->nx < 1 || p->ny < 1 || p->n_theta < 4 || p->n_theta % 4 != 0 || p->n_omz < 1)
        return fail(RTE_ERR_ARG, "rte_setup: need nx, ny >= 1, n_theta a positive multiple of 4, n_omz >= 1");
    if ((long long)p->nx * p->ny > (1ll << 28)) return fail(RTE_ERR_ARG, "rte_setup: mesh too large");
    if (!(p->x1 > p->x0) || !(p->y1 > p->y0)) return fail(RTE_ERR_ARG, "rte_setup: empty domain");
    if (!p->sig_t || !p->sig_s) return fail(RTE_ERR_ARG, "rte_setup: sig_t and sig_s are required");
    if (p->n_rect < 0 || (p->n_rect > 0 && !p->q_rects)) return fail(RTE_ERR_ARG, "rte_setup: bad rectangles");
    if (p->n_gauss < 0 || (p->n_gauss > 0 && !p->q_gauss))
        return fail(RTE_ERR_ARG, "rte_setup: bad Gaussian sources");
    for (int r = 0; r < p->n_gauss; ++r)
        if (!(p->q_gauss[4 * r + 2] > 0.0) || !std::isfinite(p->q_gauss[4 * r + 2]) ||
            !std::isfinite(p->q_gauss[4 * r]) || !std::isfinite(p->q_gauss[4 * r + 1]) ||
            !std::isfinite(p->q_gauss[4 * r + 3]))
            return fail(RTE_ERR_ARG, "rte_setup: Gaussian source needs finite values and a > 0");
    const int nc = p->nx * p->ny;
    RTE_TRY(check_materials(nc, p->sig_t, p->sig_s));

    rte_handle* h = new rte_handle();
    h->nx = p->nx;
    h->ny = p->ny;
    h->nc = nc;
    h->ndof = 4 * nc;
    h->n_theta = p->n_theta;
    h->n_omz = p->n_omz;
    h->nang = p->n_theta * p->n_omz;
    h->x0 = p->x0; h->x1 = p->x1; h->y0 = p->y0; h->y1 = p->y1;
    h->hx = (p->x1 - p->x0) / p->nx;
    h->hy = (p->y1 - p->y0) / p->ny;
    for (int k = 0; k < 4; ++k) h->inflow[k] = p->inflow[k];
    h->stream = (cudaStream_t)stream;
    int dev = 0;
    cudaGetDevice(&dev);
    h->device = dev;
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
    h->sig_t_h.assign(p->sig_t, p->sig_t + nc);
    h->sig_s_h.assign(p->sig_s, p->sig_s + nc);
    h->has_q = p->q_cell != nullptr;
    if (h->has_q) h->q_h.assign(p->q_cell, p->q_cell + nc);
    if (p->n_rect > 0) h->rects.assign(p->q_rects, p->q_rects + 5 * p->n_rect);
    if (p->n_gauss > 0) h->gauss.assign(p->q_gauss, p->q_gauss + 4 * p->n_gauss);

    // CL(N_theta, N_Omega_z) quadrature, App. A
    std::vector<double> z, wz;
    gauss_legendre(h->n_omz, z, wz);
    h->ox.resize(h->nang);
    h->oy.resize(h->nang);
    h->oz.resize(h->nang);
    h->w.resize(h->nang);
    h->twin.resize(h->nang);
    for (int j2 = 0; j2 < h->n_omz; ++j2) {
        double s = sqrt(1.0 - z[j2] * z[j2]);
        for (int j1 = 0; j1 < h->n_theta; ++j1) {
            double th = (2.0 * j1 + 1.0) * M_PI / h->n_theta;
            int j = j2 * h->n_theta + j1;
            h->ox[j] = cos(th) * s;
            h->oy[j] = sin(th) * s;
            h->oz[j] = z[j2];
            h->w[j] = 0.5 * wz[j2] / h->n_theta;
            h->twin[j] = (h->n_omz - 1 - j2) * h->n_theta + j1;
        }
    }
    for (int j = 0; j < h->nang; ++j) {
        if (h->twin[j] >= j) {   // representative: the smaller index of a twin pair
            h->fold_rep.push_back(j);
            h->fold_w.push_back(h->twin[j] == j ? h->w[j] : h->w[j] + h->w[h->twin[j]]);
        }
    }

    int st = RTE_OK;
    auto A = [&](void** ptr, size_t n) { if (st == RTE_OK) st = h->arena.alloc(ptr, n); };
    const size_t nd = (size_t)h->ndof;
    A((void**)&h->sig_t, sizeof(double) * nc);
    A((void**)&h->sig_s, sizeof(double) * nc);
    A((void**)&h->sig_t_f, sizeof(float) * nc);
    A((void**)&h->sig_dw, sizeof(float) * 2 * nc);
    A((void**)&h->b_dw, sizeof(float) * 2 * nd);
    A((void**)&h->G, sizeof(double) * nd);
    A((void**)&h->e_side, sizeof(double) * 4 * nd);
    A((void**)&h->d_ox, sizeof(double) * h->nang);
    A((void**)&h->d_oy, sizeof(double) * h->nang);
    A((void**)&h->d_w, sizeof(double) * h->nang);
    A((void**)&h->d_fold_w, sizeof(double) * h->nang);
    A((void**)&h->d_wlist, sizeof(double) * h->nang);
    A((void**)&h->d_fold_rep, sizeof(int) * h->nang);
    A((void**)&h->d_angles, sizeof(int) * h->nang);
    A((void**)&h->phi_star, sizeof(double) * nd);
    A((void**)&h->dphi, sizeof(double) * nd);
    A((void**)&h->tmp, sizeof(double) * nd);
    A((void**)&h->src_w, sizeof(double) * nd);
    A((void**)&h->src64, sizeof(double) * nd);
    A((void**)&h->red, sizeof(double) * 8192);
    A((void**)&h->D, sizeof(double) * nc);
    A((void**)&h->sig_a, sizeof(double) * nc);
    A((void**)&h->Minv, sizeof(double) * 16 * (size_t)nc);
    A((void**)&h->cg_r, sizeof(double) * nd);
    A((void**)&h->cg_z, sizeof(double) * nd);
    A((void**)&h->cg_p, sizeof(double) * nd);
    A((void**)&h->cg_q, sizeof(double) * nd);
    A((void**)&h->cg_red, sizeof(double) * 8192);
    A((void**)&h->cg_iters, sizeof(int) * 4);
    A((void**)&h->d_err, sizeof(int) * 4);
    A((void**)&h->d_outcols, sizeof(int2) * h->nang);
    if (st != RTE_OK) {
        h->arena.release_all();
        delete h;
        return st;
    }
    if (pinned_alloc((void**)&h->h_angles, sizeof(int) * h->nang) != cudaSuccess ||
        pinned_alloc((void**)&h->h_outcols, sizeof(int2) * h->nang) != cudaSuccess ||
        pinned_alloc((void**)&h->h_wlist, sizeof(double) * h->nang) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_pinned, cudaEventDisableTiming) != cudaSuccess ||
        pinned_alloc((void**)&h->h_scalar, sizeof(double) * 64) != cudaSuccess) {
        cudaGetLastError();
        pinned_free(h->h_angles);
        pinned_free(h->h_outcols);
        pinned_free(h->h_wlist);
        if (h->ev_pinned) cudaEventDestroy(h->ev_pinned);
        h->arena.release_all();
        delete h;
        return fail(RTE_ERR_NOMEM, "rte_setup: pinned host allocation failed");
    }
    std::vector<double> e;
    side_vectors(h, e);
    std::vector<int> rep(h->fold_rep);
    rep.resize(h->nang, 0);
    std::vector<double> fw(h->fold_w);
    fw.resize(h->nang, 0.0);
    auto up = [&](void* dst, const void* src, size_t n) {
        if (st == RTE_OK && cudaMemcpy(dst, src, n, cudaMemcpyHostToDevice) != cudaSuccess)
            st = fail(RTE_ERR_CUDA, "rte_setup: upload failed");
    };
    if (st == RTE_OK && cudaMemset(h->d_err, 0, sizeof(int) * 4) != cudaSuccess) st = fail(RTE_ERR_CUDA, "rte_setup: memset");
    up(h->e_side, e.data(), sizeof(double) * 4 * nd);
    up(h->d_ox, h->ox.data(), sizeof(double) * h->nang);
    up(h->d_oy, h->oy.data(), sizeof(double) * h->nang);
    up(h->d_w, h->w.data(), sizeof(double) * h->nang);
    up(h->d_fold_w, fw.data(), sizeof(double) * h->nang);
    up(h->d_fold_rep, rep.data(), sizeof(int) * h->nang);
    if (st == RTE_OK) st = upload_materials(h);
    if (st != RTE_OK) {
        rte_destroy(h);
        return st;
    }
    *out = h;
    return RTE_OK;
}

int rte_destroy(rte_handle* h) {
    if (!h) return RTE_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    h->arena.release_all();
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->cap_stream2) cudaStreamDestroy(h->cap_stream2);
    if (h->border_stream) cudaStreamDestroy(h->border_stream);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    pinned_free(h->h_angles);
    pinned_free(h->h_outcols);
    pinned_free(h->h_wlist);
    if (h->ev_pinned) cudaEventDestroy(h->ev_pinned);
    pinned_free(h->h_scalar);
    pinned_free(h->lr.host_small);
    pinned_free(h->lr.host_ints);
    delete h;
    return RTE_OK;
}

int rte_set_materials(rte_handle* h, const double* sig_t, const double* sig_s, const double* q_cell) {
    if (!h || !sig_t || !sig_s) return fail(RTE_ERR_ARG, "rte_set_materials: null argument");
    RTE_TRY(check_materials(h->nc, sig_t, sig_s));
    h->sig_t_h.assign(sig_t, sig_t + h->nc);
    h->sig_s_h.assign(sig_s, sig_s + h->nc);
    if (q_cell) {
        h->has_q = true;
        h->q_h.assign(q_cell, q_cell + h->nc);
    }
    h->lr.ready = false;
    return upload_materials(h);
}

int rte_set_wait_limit(rte_handle* h, int spins) {
    if (!h || spins < 0) return fail(RTE_ERR_ARG, "rte_set_wait_limit: null handle or negative limit");
    h->wait_limit = spins == 0 ? (1 << 22) : spins;
    return RTE_OK;
}

int rte_inject_failure(rte_handle* h, int code) {
    if (!h || (code != 0 && code != RTE_ERR_SINGULAR))
        return fail(RTE_ERR_ARG, "rte_inject_failure: null handle or unsupported code");
    h->inject = code;
    return RTE_OK;
}

int rte_get_sizes(const rte_handle* h, int* n_dof, int* n_cells, int* n_angles) {
    if (!h) return fail(RTE_ERR_ARG, "rte_get_sizes: null handle");
    if (n_dof) *n_dof = h->ndof;
    if (n_cells) *n_cells = h->nc;
    if (n_angles) *n_angles = h->nang;
    return RTE_OK;
}

int rte_get_quadrature(const rte_handle* h, double* ox, double* oy, double* oz, double* w) {
    if (!h) return fail(RTE_ERR_ARG, "rte_get_quadrature: null handle");
    for (int j = 0; j < h->nang; ++j) {
        if (ox) ox[j] = h->ox[j];
        if (oy) oy[j] = h->oy[j];
        if (oz) oz[j] = h->oz[j];
        if (w) w[j] = h->w[j];
    }
    return RTE_OK;
}

int rte_get_source(const rte_handle* h, double* G_dev) {
    if (!h || !G_dev) return fail(RTE_ERR_ARG, "rte_get_source: null argument");
    RTE_CUDA_TRY(cudaMemcpyAsync(G_dev, h->G, sizeof(double) * h->ndof, cudaMemcpyDeviceToDevice, h->stream));
    return RTE_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- profiler
namespace rte {

cudaEvent_t Profiler::get_event() {
    if (!free_ev.empty()) {
        cudaEvent_t e = free_ev.back();
        free_ev.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void Profiler::begin(int cls, cudaStream_t st) {
    if (pending.size() > 8192) {
        cudaStreamSynchronize(st);
        flush();
    }
    open_ev = get_event();
    open_cls = cls;
    cudaEventRecord(open_ev, st);
}

int Profiler::end(int cls, cudaStream_t st, double by, double fl) {
    if (open_cls != cls || !open_ev) return -1;
    cudaEvent_t b = get_event();
    cudaEventRecord(b, st);
    pending.push_back(Rec{cls, open_ev, b, by, fl});
    open_ev = nullptr;
    open_cls = -1;
    return (int)pending.size() - 1;
}

void Profiler::flush() {
    for (auto& r : pending) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
            ms[r.cls] += t;
            launches[r.cls] += 1;
            bytes[r.cls] += r.bytes;
            flops[r.cls] += r.flops;
        }
        free_ev.push_back(r.a);
        free_ev.push_back(r.b);
    }
    pending.clear();
    cudaGetLastError();
}

void Profiler::reset() {
    pending.clear();
    for (int k = 0; k < 16; ++k) { ms[k] = 0; bytes[k] = 0; flops[k] = 0; launches[k] = 0; }
}

Profiler::~Profiler() {
    for (auto& r : pending) { free_ev.push_back(r.a); free_ev.push_back(r.b); }
    for (auto e : free_ev) cudaEventDestroy(e);
    if (open_ev) cudaEventDestroy(open_ev);
}

}  // namespace rte

extern "C" int rte_profile_enable(rte_handle* h, int on) {
    if (!h) return rte::fail(RTE_ERR_ARG, "rte_profile_enable: null handle");
    RTE_CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->prof.flush();
    h->prof.reset();
    h->prof.on = on != 0;
    return RTE_OK;
}

extern "C" int rte_profile_read(rte_handle* h, int cls, double* ms, long long* launches, double* bytes, double* flops) {
    if (!h || cls < 0 || cls >= RTE_PROF_NCLASS) return rte::fail(RTE_ERR_ARG, "rte_profile_read: bad argument");
    RTE_CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->prof.flush();
    if (ms) *ms = h->prof.ms[cls];
    if (launches) *launches = h->prof.launches[cls];
    if (bytes) *bytes = h->prof.bytes[cls];
    if (flops) *flops = h->prof.flops[cls];
    return RTE_OK;
}
