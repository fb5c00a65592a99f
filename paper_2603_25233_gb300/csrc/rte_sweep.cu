// Transport sweeps (Sec. 2.2): psi_j = (D_j + Sigma_t)^{-1} b_j for a list of ordinates.
//
// Per cell, in the frame where Omega_x, Omega_y >= 0 (odd Legendre modes flip sign under the
// reflections x -> -x, y -> -y), the upwind DG-Q1 system of Eq. (mat-vec) is
//
//   (sigma_t I + a_x K (x) I + a_y I (x) K) psi = S + a_x (l (x) tau_x) + a_y (tau_y (x) l)
//
// with a_x = |Omega_x|/h_x, a_y = |Omega_y|/h_y, K = [[1, sqrt3], [-sqrt3, 3]] (volume term
// plus outflow face of the orthonormal Legendre basis), l = (1, -sqrt3) (inflow-face trace),
// and tau_x, tau_y the outflow traces of the upwind neighbours (tau = psi_0 + sqrt3 psi_1 per
// tangential mode).  The 4x4 system is solved in closed form by block elimination over the
// y-modes, using K^2 = 4 K - 6 I: M = (alpha I + B)(gamma I + B) + beta^2 I = x I + y K with
// B = a_x K, alpha = sigma + a_y, gamma = sigma + 3 a_y, beta = sqrt3 a_y, and
// M^{-1} = ((x + 4y) I - y K) / (x^2 + 4xy + 6y^2).
//
// Parallel schedule (one warp per ordinate): the mesh is cut into bands of H = min(32, nx)
// rows; lane t owns row t of each band and walks its row in the upwind x order, so at step s
// lane t works on column s - t of band floor(s / nx).  The x-inflow trace stays in registers,
// the y-inflow trace comes from lane t-1 by a shuffle (computed one step earlier), and the
// band above reads the top row of the band below from a shared-memory ring indexed by column.
// A step needs no barrier beyond __syncwarp, and no lane ever waits on another warp.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "rte_internal.cuh"
#include "rte_cell.cuh"
#include "rte_dw.cuh"

namespace rte {

template <typename T>
struct SweepArgs {
    int nx, ny, n;
    T hx, hy, gs;                 // gs = sqrt(hx * hy): ghost-cell mean mode of a unit inflow
    const T* sig_t;
    const T* src;
    long long src_stride;         // elements between the sources of consecutive angles (0 = shared)
    const int* angles;
    const double* ox;
    const double* oy;
    T g[4];                       // inflow left, right, bottom, top
    int add_inflow;
    int reverse;                  // 1: direction -Omega_j (adjoint sweep)
    T* psi;
    long long psi_stride;
    const int* n_dev;             // optional device count of active angles (<= n)
    int spin_limit;               // polls of a band hand-off wait before it gives up
    const int2* outcols;          // optional: item a writes psi columns outcols[a].x and (if >= 0)
                                  // outcols[a].y (the +-Omega_z twin or a repeat: the same psi)
};


template <typename T>
__global__ void __launch_bounds__(128) sweep_warp_kernel(SweepArgs<T> A) {
    pdl_entry();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int a = blockIdx.x * (blockDim.x >> 5) + wib;
    if (a >= A.n || (A.n_dev && a >= *A.n_dev)) return;  // uniform per warp
    T* ring = reinterpret_cast<T*>(smem_raw) + (size_t)wib * 2 * A.nx;
    const int j = A.angles[a];
    double oxd = A.ox[j], oyd = A.oy[j];
    if (A.reverse) { oxd = -oxd; oyd = -oyd; }
    const bool px = oxd >= 0.0, py = oyd >= 0.0;
    const T ax = T(fabs(oxd)) / A.hx, ay = T(fabs(oyd)) / A.hy;
    const T fx = px ? T(1) : T(-1), fy = py ? T(1) : T(-1), fxy = fx * fy;
    const T s3 = T(1.7320508075688772935);
    const T s3ax = s3 * ax, s3ay = s3 * ay;
    T gx = T(0), gy = T(0);
    if (A.add_inflow) {
        gx = (px ? A.g[0] : A.g[1]) * A.gs;
        gy = (py ? A.g[2] : A.g[3]) * A.gs;
    }
    const int nx = A.nx, ny = A.ny;
    const int H = nx < 32 ? nx : 32;
    const int nb = (ny + H - 1) / H;
    const int total = nb * nx;
    const int nsteps = total + H - 1;
    const T* __restrict__ src = A.src + (long long)a * A.src_stride;
    T* __restrict__ psi = nullptr;
    T* __restrict__ psi2 = nullptr;
    if (A.psi) {
        const int2 oc = A.outcols ? A.outcols[a] : make_int2(a, -1);
        psi = A.psi + (long long)oc.x * A.psi_stride;
        if (oc.y >= 0) psi2 = A.psi + (long long)oc.y * A.psi_stride;
    }
    const T* __restrict__ sig_t = A.sig_t;

    T tx0 = T(0), tx1 = T(0), ty0 = T(0), ty1 = T(0);
    int b = 0, xp = 0;                                    // this lane's band and frame column
    for (int s = 0; s < nsteps; ++s) {
        T iy0 = __shfl_up_sync(0xffffffffu, ty0, 1);
        T iy1 = __shfl_up_sync(0xffffffffu, ty1, 1);
        const int rel = s - lane;
        if (lane < H && rel >= 0 && rel < total) {
            const int row = b * H + lane;
            if (row < ny) {
                if (lane == 0) {
                    if (b == 0) { iy0 = gy; iy1 = T(0); }
                    else { iy0 = ring[2 * xp]; iy1 = ring[2 * xp + 1]; }
                }
                if (xp == 0) { tx0 = gx; tx1 = T(0); }
                const int ix = px ? xp : nx - 1 - xp;
                const int iy = py ? row : ny - 1 - row;
                const long long c = (long long)iy * nx + ix;
                T S0, S1, S2, S3;
                load4(src + 4 * c, S0, S1, S2, S3);
                const T sig = sig_t[c];
                S1 *= fx; S2 *= fy; S3 *= fxy;
                const T f0 = fma(ax, tx0, fma(ay, iy0, S0));
                const T f1 = fma(-s3ax, tx0, fma(ay, iy1, S1));
                const T g0 = fma(ax, tx1, fma(-s3ay, iy0, S2));
                const T g1 = fma(-s3ax, tx1, fma(-s3ay, iy1, S3));
                T u0, u1, v0, v1;
                cell_solve<T>(sig, ax, ay, s3, f0, f1, g0, g1, u0, u1, v0, v1);
                tx0 = fma(s3, u1, u0);
                tx1 = fma(s3, v1, v0);
                ty0 = fma(s3, v0, u0);
                ty1 = fma(s3, v1, u1);
                if (psi) store4(psi + 4 * c, u0, fx * u1, fy * v0, fxy * v1);
                if (psi2) store4(psi2 + 4 * c, u0, fx * u1, fy * v0, fxy * v1);
                if (lane == H - 1) { ring[2 * xp] = ty0; ring[2 * xp + 1] = ty1; }
            }
            if (++xp == nx) { xp = 0; ++b; }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------------------------
// Multi-warp sweep: one CTA per ordinate, W warps.  Bands of 32 rows are dealt to the warps
// cyclically (band b -> warp b mod W); inside a band the lane/row schedule is the one above.
// The top-row outflow traces of band b are handed to band b+1 through a per-warp ring in
// shared memory plus a progress counter (columns completed); the consumer's lane 0 waits on
// the counter with a bounded spin (an exhausted wait sets *err and continues, so a kernel
// never hangs; the host turns the flag into RTE_ERR_DEP_TIMEOUT).  The dependence chain only
// points to lower bands, and a ring slot is rewritten only after its consumer has used it
// (the producer's next band depends on the consumer's band through W-1 hand-offs).
// Each lane prefetches its next D-1 cells (source moments and sigma_t) into shared memory
// with cp.async, so global-memory latency stays off the wavefront's critical path.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Prefetch slots, lane-minor so that a warp's accesses to one slot are contiguous (no bank
// conflicts): for each (warp, slot) 32 source quadruples then 32 sigma_t values.  FP32: one
// float4 per lane; FP64: two double2 halves.
template <typename T>
struct Stage;
template <>
struct Stage<float> {
    float4* q;
    float* sig;
    static constexpr size_t bytes_per_cell = 20;
    __device__ __forceinline__ Stage(unsigned char* base, int nslots) {
        q = reinterpret_cast<float4*>(base);
        sig = reinterpret_cast<float*>(q + nslots * 32);
    }
    __device__ __forceinline__ void load(int i, const float* src, const float* sg, long long c) {
        cp_async16(q + i, src + 4 * c);
        cp_async4(sig + i, sg + c);
    }
    __device__ __forceinline__ void read(int i, float& s0, float& s1, float& s2, float& s3, float& st) const {
        const float4 v = q[i];
        s0 = v.x; s1 = v.y; s2 = v.z; s3 = v.w;
        st = sig[i];
    }
};
template <>
struct Stage<double> {
    double2* lo;
    double2* hi;
    double* sig;
    static constexpr size_t bytes_per_cell = 40;
    __device__ __forceinline__ Stage(unsigned char* base, int nslots) {
        lo = reinterpret_cast<double2*>(base);
        hi = lo + nslots * 32;
        sig = reinterpret_cast<double*>(hi + nslots * 32);
    }
    __device__ __forceinline__ void load(int i, const double* src, const double* sg, long long c) {
        cp_async16(lo + i, src + 4 * c);
        cp_async16(hi + i, src + 4 * c + 2);
        cp_async8(sig + i, sg + c);
    }
    __device__ __forceinline__ void read(int i, double& s0, double& s1, double& s2, double& s3, double& st) const {
        const double2 a = lo[i], b = hi[i];
        s0 = a.x; s1 = a.y; s2 = b.x; s3 = b.y;
        st = sig[i];
    }
};

// Output staging of the band kernels: a lane's cells of one row are gathered in shared memory
// kOutCells at a time, and a warp writes the completed row segments (kOutCells x 16 bytes each,
// contiguous in psi) together, instead of 32 scattered 16-byte stores (one per row of the
// anti-diagonal) per step.
constexpr int kOutCells = 4;

// Shared memory of the band kernels: the trace ring [W][2 nx], W progress counters (64 bytes),
// W x D x 32 prefetch slots, W x kOutCells x 32 output cells and a 32-entry segment table per warp.
template <typename T>
__host__ __device__ __forceinline__ size_t band_ring_bytes(int W, int nx) {
    return ((size_t)W * 2 * nx * sizeof(T) + 15) & ~(size_t)15;
}
template <typename T>
__host__ __device__ __forceinline__ size_t band_stage_bytes(int W, int D) {
    return (size_t)W * D * 32 * Stage<T>::bytes_per_cell;
}
template <typename T>
__host__ __device__ __forceinline__ size_t band_smem_bytes(int W, int nx, int D) {
    return band_ring_bytes<T>(W, nx) + 64 + band_stage_bytes<T>(W, D) + (size_t)W * kOutCells * 32 * 4 * sizeof(T) +
           (size_t)W * 32 * sizeof(int2);
}

// one cell's four moments in the output staging buffer
__device__ __forceinline__ void obuf_put(float* o, int i, float a, float b, float c, float d) {
    reinterpret_cast<float4*>(o)[i] = make_float4(a, b, c, d);
}
__device__ __forceinline__ void obuf_put(double* o, int i, double a, double b, double c, double d) {
    reinterpret_cast<double2*>(o)[2 * i] = make_double2(a, b);
    reinterpret_cast<double2*>(o)[2 * i + 1] = make_double2(c, d);
}
__device__ __forceinline__ void obuf_copy(const float* o, int i, float* dst) {
    *reinterpret_cast<float4*>(dst) = reinterpret_cast<const float4*>(o)[i];
}
__device__ __forceinline__ void obuf_copy(const double* o, int i, double* dst) {
    reinterpret_cast<double2*>(dst)[0] = reinterpret_cast<const double2*>(o)[2 * i];
    reinterpret_cast<double2*>(dst)[1] = reinterpret_cast<const double2*>(o)[2 * i + 1];
}

#ifndef RTE_BAND_DEPTH
#define RTE_BAND_DEPTH 4
#endif
constexpr int kBandDepth = RTE_BAND_DEPTH;   // prefetch depth (steps) of the band kernels

// Lane walker over this warp's cells in step order: local band lb, frame column x, linear
// cell index c (advances by +-1 along a row) and whether the lane's row exists in the band.
struct Walk {
    int lb, x, c, valid;
};

__device__ __forceinline__ void walk_band(Walk& wk, int w, int W, int lane, int nx, int ny, bool px, bool py) {
    const int row = (w + wk.lb * W) * 32 + lane;
    wk.valid = row < ny;
    const int iy = py ? row : ny - 1 - row;
    wk.c = iy * nx + (px ? 0 : nx - 1);
}

// Band sweep of angle a of A by the whole block (W = blockDim / 32 warps; warps beyond the
// problem's band count idle).  Shared by the single-problem and the batched kernels.
template <typename T, int D, bool STAGED>
__device__ __forceinline__ void band_sweep_body(const SweepArgs<T>& A, int a, int* err, unsigned char* smem_raw) {
    static_assert((D & (D - 1)) == 0, "D must be a power of two");
    const int W = blockDim.x >> 5;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int nx = A.nx, ny = A.ny;
    T* ring = reinterpret_cast<T*>(smem_raw);                               // [W][2 nx]
    const size_t ring_bytes = band_ring_bytes<T>(W, nx);
    int* prog = reinterpret_cast<int*>(smem_raw + ring_bytes);              // [W <= 16], 64 bytes
    Stage<T> stage(smem_raw + ring_bytes + 64, W * D);
    const int slot0 = w * D * 32 + lane;                                     // slot d: slot0 + 32 d
    // this warp's output cells [kOutCells][32 lanes][4 moments]
    T* obuf = reinterpret_cast<T*>(smem_raw + ring_bytes + 64 + band_stage_bytes<T>(W, D)) +
              (size_t)w * kOutCells * 32 * 4;
    // this warp's table of the row segments completed in a step: (last cell, length | lane << 8)
    int2* segtab = reinterpret_cast<int2*>(smem_raw + ring_bytes + 64 + band_stage_bytes<T>(W, D) +
                                           (size_t)W * kOutCells * 32 * 4 * sizeof(T)) + w * 32;
    const unsigned lanes_below = (1u << lane) - 1u;
    const int seg_grp = lane / kOutCells, seg_j = lane % kOutCells;
    if (threadIdx.x < W) prog[threadIdx.x] = 0;
    __syncthreads();

    const int j = A.angles[a];
    double oxd = A.ox[j], oyd = A.oy[j];
    if (A.reverse) { oxd = -oxd; oyd = -oyd; }
    const bool px = oxd >= 0.0, py = oyd >= 0.0;
    const T ax = T(fabs(oxd)) / A.hx, ay = T(fabs(oyd)) / A.hy;
    const T fx = px ? T(1) : T(-1), fy = py ? T(1) : T(-1), fxy = fx * fy;
    const T s3 = T(1.7320508075688772935);
    const T s3ax = s3 * ax, s3ay = s3 * ay;
    T gx = T(0), gy = T(0);
    if (A.add_inflow) {
        gx = (px ? A.g[0] : A.g[1]) * A.gs;
        gy = (py ? A.g[2] : A.g[3]) * A.gs;
    }
    const int nb = (ny + 31) >> 5;
    const int nbw = w < nb ? (nb - 1 - w) / W + 1 : 0;      // bands owned by this warp
    const int total = nbw * nx;                              // active steps of each lane
    const int dc = px ? 1 : -1;
    const T* __restrict__ src = A.src + (long long)a * A.src_stride;
    const T* __restrict__ sig_t = A.sig_t;
    // the staged variant also serves items with a second output column (outcols); the direct
    // variant keeps a single store per cell (a second, conditional store there measured 33%
    // slower on the single-ordinate sweeps of the low-rank loop)
    T* __restrict__ psi = nullptr;
    T* __restrict__ psi2 = nullptr;
    if (STAGED) {
        if (A.psi) {
            const int2 oc = A.outcols ? A.outcols[a] : make_int2(a, -1);
            psi = A.psi + (long long)oc.x * A.psi_stride;
            if (oc.y >= 0) psi2 = A.psi + (long long)oc.y * A.psi_stride;
        }
    } else {
        psi = A.psi ? A.psi + (long long)a * A.psi_stride : nullptr;
    }
    T* my_ring = ring + (size_t)w * 2 * nx;

    // prefetch walker (D - 1 steps ahead of the compute walker)
    Walk pf{0, 0, 0, 0};
    walk_band(pf, w, W, lane, nx, ny, px, py);
    int kpf = 0;
#pragma unroll
    for (int t = 0; t < D - 1; ++t) {
        if (kpf < total && pf.valid) stage.load(slot0 + 32 * (kpf & (D - 1)), src, sig_t, pf.c);
        cp_commit();
        ++kpf;
        pf.c += dc;
        if (++pf.x == nx) { pf.x = 0; ++pf.lb; walk_band(pf, w, W, lane, nx, ny, px, py); }
    }
    Walk cw{0, 0, 0, 0};
    walk_band(cw, w, W, lane, nx, ny, px, py);
    int band = w;
    T tx0 = T(0), tx1 = T(0), ty0 = T(0), ty1 = T(0);
    // lane 0 of band b waits for the owner of band b - 1 (warp wp) to have completed column x
    // of that band: its progress counter must reach need_base + x + 1
    const int wp = w == 0 ? W - 1 : w - 1;
    const T* rp = ring + (size_t)wp * 2 * nx;
    volatile int* pv = prog + wp;
    int need_base = band > 0 ? ((band - 1) / W) * nx : 0;
    int seen = 0;                                            // lane 0: last progress value read
    int seg_len = 0;                                         // a completed row segment this step:
    int seg_end = 0;                                         // its length and its last cell
    const int nsteps = total + 31;
    for (int s = 0; s < nsteps; ++s) {
        T iy0 = __shfl_up_sync(0xffffffffu, ty0, 1);
        T iy1 = __shfl_up_sync(0xffffffffu, ty1, 1);
        const int k = s - lane;
        if ((unsigned)k < (unsigned)total) {
            if (kpf < total && pf.valid) stage.load(slot0 + 32 * (kpf & (D - 1)), src, sig_t, pf.c);
            cp_commit();
            ++kpf;
            pf.c += dc;
            if (++pf.x == nx) { pf.x = 0; ++pf.lb; walk_band(pf, w, W, lane, nx, ny, px, py); }
            cp_wait<D - 1>();
            const int x = cw.x;
            if (cw.valid) {
                // lane 0 of a band below the first takes its y-inflow from the ring; it waits
                // only when the last progress value it read does not cover column x (the
                // producer publishes every 4 columns, so the wait is rarely entered)
                const bool from_ring = lane == 0 && band > 0;
                if (from_ring && seen < need_base + x + 1) {
                    const int need = need_base + x + 1;
                    int spins = 0;
                    int v = *pv;
                    while (v < need) {
                        if (++spins > A.spin_limit) { atomicExch(err, 1); break; }
                        if (spins > 256) __nanosleep(20);
                        v = *pv;
                    }
                    seen = v;
                    __threadfence_block();
                }
                if (lane == 0) {
                    iy0 = from_ring ? rp[2 * x] : gy;
                    iy1 = from_ring ? rp[2 * x + 1] : T(0);
                }
                if (x == 0) { tx0 = gx; tx1 = T(0); }
                T q0, q1, q2, q3, sig;
                stage.read(slot0 + 32 * (k & (D - 1)), q0, q1, q2, q3, sig);
                const T f0 = fma(ax, tx0, fma(ay, iy0, q0));
                const T f1 = fma(-s3ax, tx0, fma(ay, iy1, fx * q1));
                const T g0 = fma(ax, tx1, fma(-s3ay, iy0, fy * q2));
                const T g1 = fma(-s3ax, tx1, fma(-s3ay, iy1, fxy * q3));
                T u0, u1, v0, v1;
                cell_solve<T>(sig, ax, ay, s3, f0, f1, g0, g1, u0, u1, v0, v1);
                tx0 = fma(s3, u1, u0);
                tx1 = fma(s3, v1, v0);
                ty0 = fma(s3, v0, u0);
                ty1 = fma(s3, v1, u1);
                if (psi) {
                    if (STAGED) {
                        obuf_put(obuf, (x % kOutCells) * 32 + lane, u0, fx * u1, fy * v0, fxy * v1);
                        if (x % kOutCells == kOutCells - 1 || x == nx - 1) {
                            seg_len = x % kOutCells + 1;
                            seg_end = cw.c;
                        }
                    } else {
                        store4(psi + 4 * (long long)cw.c, u0, fx * u1, fy * v0, fxy * v1);
                    }
                }
                if (lane == 31 && band + 1 < nb) {
                    my_ring[2 * x] = ty0;
                    my_ring[2 * x + 1] = ty1;
                    if ((x & 3) == 3 || x == nx - 1) {          // publish every 4 columns
                        __threadfence_block();
                        reinterpret_cast<volatile int*>(prog)[w] = k + 1;
                    }
                }
            }
            cw.c += dc;
            if (++cw.x == nx) {
                cw.x = 0;
                ++cw.lb;
                band += W;
                need_base = ((band - 1) / W) * nx;
                seen = 0;
                walk_band(cw, w, W, lane, nx, ny, px, py);
            }
        }
        if (STAGED && psi) {
            // write the row segments completed this step: each holder enters its segment in the
            // warp's table at its rank among the holders, and lane i copies cell i % kOutCells of
            // entries i / kOutCells, i / kOutCells + 32 / kOutCells, ...; a segment's cells are
            // consecutive in memory.  The warp sync after the table writes also orders this
            // step's output-cell writes before the copies; the one after the copies keeps the
            // next step's writes of cells and table behind them.
            const unsigned m = __ballot_sync(0xffffffffu, seg_len > 0);
            if (m) {
                if (seg_len > 0) segtab[__popc(m & lanes_below)] = make_int2(seg_end, seg_len | (lane << 8));
                __syncwarp();
                const int nseg = __popc(m);
                for (int g = seg_grp; g < nseg; g += 32 / kOutCells) {
                    const int2 e = segtab[g];
                    const int len = e.y & 0xff;
                    if (seg_j < len) {
                        const int src_lane = e.y >> 8;
                        const long long cell = e.x - (len - 1 - seg_j) * dc;
                        obuf_copy(obuf, seg_j * 32 + src_lane, psi + 4 * cell);
                        if (psi2) obuf_copy(obuf, seg_j * 32 + src_lane, psi2 + 4 * cell);
                    }
                }
                seg_len = 0;
                __syncwarp();
            }
        }
    }
    cp_wait<0>();
}

// One block sweeps ordinates blockIdx.x, blockIdx.x + gridDim.x, ... (one per block when the
// grid has n blocks; a persistent grid of fewer blocks takes several in turn).
template <typename T, int D, bool STAGED>
__global__ void __launch_bounds__(512) sweep_band_kernel(SweepArgs<T> A, int* err) {
    pdl_entry();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = A.n_dev ? min(A.n, *A.n_dev) : A.n;
    for (int a = blockIdx.x; a < n; a += gridDim.x) {        // uniform per block
        band_sweep_body<T, D, STAGED>(A, a, err, smem_raw);
        __syncthreads();                                    // the next ordinate reuses shared memory
    }
}

// Batched sweep: block b sweeps angle items[b].y of problem items[b].x (problems of different
// sizes and quadratures in one launch; the block size is that of the problem with most bands).
template <typename T, int D>
__global__ void __launch_bounds__(512) sweep_band_batch_kernel(const SweepArgs<T>* __restrict__ args,
                                                               const int2* __restrict__ items, int* err) {
    pdl_entry();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int2 it = items[blockIdx.x];
    const SweepArgs<T> A = args[it.x];
    band_sweep_body<T, D, true>(A, it.y, err, smem_raw);
}

template <typename T>
__global__ void phi_reduce_kernel(int ndof, int n, const double* __restrict__ wlist, const T* __restrict__ psi,
                                  long long stride, double* __restrict__ phi) {
    pdl_entry();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ndof; i += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int a = 0; a < n; ++a) acc = fma(wlist[a], (double)psi[(long long)a * stride + i], acc);
        phi[i] = acc;
    }
}

template <typename T>
__global__ void source_kernel(int nc, const double* __restrict__ sig_s, const double* __restrict__ phi,
                              const double* __restrict__ G, T* __restrict__ S) {
    pdl_entry();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 4 * nc; i += gridDim.x * blockDim.x)
        S[i] = (T)fma(sig_s[i >> 2], phi[i], G[i]);
}

__global__ void max_abs_diff_partial(int n, const double* __restrict__ a, const double* __restrict__ b,
                                     double* __restrict__ out) {
    pdl_entry();
    __shared__ double sm[32];
    double m = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double d = fabs(a[i] - b[i]);
        m = (d > m || d != d) ? d : m;            // NaN propagates
    }
    for (int o = 16; o > 0; o >>= 1) { double t = __shfl_xor_sync(0xffffffffu, m, o); m = (t > m || t != t) ? t : m; }
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) { double t = __shfl_xor_sync(0xffffffffu, m, o); m = (t > m || t != t) ? t : m; }
        if (threadIdx.x == 0) out[blockIdx.x] = m;
    }
}

__global__ void max_final(int n, const double* __restrict__ part, double* __restrict__ out) {
    pdl_entry();
    __shared__ double sm[32];
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) { double d = part[i]; m = (d > m || d != d) ? d : m; }
    for (int o = 16; o > 0; o >>= 1) { double t = __shfl_xor_sync(0xffffffffu, m, o); m = (t > m || t != t) ? t : m; }
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) { double t = __shfl_xor_sync(0xffffffffu, m, o); m = (t > m || t != t) ? t : m; }
        if (threadIdx.x == 0) out[0] = m;
    }
}

static int grid_for(const rte_handle* h, long long n, int block) {
    long long g = (n + block - 1) / block;
    long long cap = (long long)std::max(h->num_sms, 1) * 8;
    return (int)std::max(1ll, std::min(g, cap));
}

// ---------------------------------------------------------------------------------------------
// Launch configurations of the single-problem sweep and their autotuner (rte_sweep_config).

static long long cfg_key(int precision, bool with_psi, int n) {
    return ((long long)n << 2) | (with_psi ? 2 : 0) | (precision == RTE_FP32 ? 1 : 0);
}

static bool band_mesh(const rte_handle* h) { return h->nx >= 32 && h->ny > 32; }

template <typename T>
static bool band_cfg_valid(const rte_handle* h, int W, int D) {
    const int nb = (h->ny + 31) / 32;
    if (W < 1 || W > 16 || W > nb) return false;
    if (W < nb && h->nx < 32 * W + 4) return false;     // cyclic bands: progress every 4 columns
    if (D != 2 && D != 4 && D != 8) return false;
    return band_smem_bytes<T>(W, h->nx, D) <= 200 * 1024;
}

template <typename T>
static bool warp_cfg_valid(const rte_handle* h, int per_block) {
    if (per_block != 1 && per_block != 2 && per_block != 4) return false;   // launch bound: 128 threads
    return 2 * (size_t)h->nx * sizeof(T) * per_block <= 200 * 1024;
}

template <typename T>
static bool cfg_valid(const rte_handle* h, const rte_sweep_config& c) {
    if (c.kernel == RTE_SWEEP_BAND)
        return band_mesh(h) && (c.angles_per_block == 1 || c.angles_per_block == 2 || c.angles_per_block == 4) &&
               (c.staged == 0 || c.staged == 1) && band_cfg_valid<T>(h, c.warps, c.depth);
    if (c.kernel == RTE_SWEEP_WARP) return warp_cfg_valid<T>(h, c.angles_per_block);
    return false;
}

// The built-in default: every band in flight (at most 16 warps; beyond 16 bands the largest
// cyclic count), depth kBandDepth, staged stores when many ordinates share the launch (2 n >
// number of SMs: throughput) and direct ones for a few (the low-rank inner loop: latency);
// meshes below one band: up to four ordinates per block.
template <typename T>
static rte_sweep_config default_cfg(const rte_handle* h, int n, bool with_psi) {
    rte_sweep_config c = {};
    if (band_mesh(h)) {
        const int nb = (h->ny + 31) / 32;
        const int wrap_max = (h->nx - 4) / 32;
        int W = nb <= 16 ? nb : std::min(16, wrap_max);
        constexpr int D = kBandDepth;
        if (W >= 1 && band_smem_bytes<T>(W, h->nx, D) > 200 * 1024) {
            W = std::min(W, wrap_max);
            while (W > 1 && band_smem_bytes<T>(W, h->nx, D) > 200 * 1024) --W;
        }
        if (W >= 1 && band_cfg_valid<T>(h, W, D)) {
            c.kernel = RTE_SWEEP_BAND;
            c.warps = W;
            c.depth = D;
            c.staged = with_psi && 2 * n > h->num_sms ? 1 : 0;
            c.angles_per_block = 1;
            return c;
        }
    }
    int wpb = 4;
    while (wpb > 1 && !warp_cfg_valid<T>(h, wpb)) wpb >>= 1;
    c.kernel = RTE_SWEEP_WARP;
    c.angles_per_block = wpb;
    return c;
}

template <typename T, int D>
static void (*band_kernel(bool staged))(SweepArgs<T>, int*) {
    return staged ? sweep_band_kernel<T, D, true> : sweep_band_kernel<T, D, false>;
}

template <typename T>
static int launch_cfg(rte_handle* h, const SweepArgs<T>& A, int n, const rte_sweep_config& c, cudaStream_t st) {
    if (c.kernel == RTE_SWEEP_BAND) {
        // deduplicated items (outcols) need the staged variant, which writes both columns
        const bool staged = A.psi && (c.staged || A.outcols);
        void (*kern)(SweepArgs<T>, int*) = c.depth == 2 ? band_kernel<T, 2>(staged)
                                           : c.depth == 8 ? band_kernel<T, 8>(staged)
                                                          : band_kernel<T, 4>(staged);
        const size_t smem = band_smem_bytes<T>(c.warps, h->nx, c.depth);
        RTE_TRY(smem_optin(kern, smem));
        const int apb = std::max(1, c.angles_per_block);
        kern<<<(n + apb - 1) / apb, 32 * c.warps, smem, st>>>(A, h->d_err);
    } else {
        const int wpb = c.angles_per_block;
        const size_t smem = 2 * (size_t)h->nx * sizeof(T) * wpb;
        if (smem > 200 * 1024) return fail(RTE_ERR_ARG, "sweep: nx too large for the shared-memory ring");
        RTE_TRY(smem_optin(sweep_warp_kernel<T>, smem));
        sweep_warp_kernel<T><<<(n + wpb - 1) / wpb, 32 * wpb, smem, st>>>(A);
    }
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

// Time every valid configuration for this launch (one warm launch and two timed ones each, on
// the call's own buffers: a sweep only writes its outputs, so repeating it is harmless) and
// return the fastest.
template <typename T>
static int tune_cfg(rte_handle* h, const SweepArgs<T>& A, int n, cudaStream_t st, rte_sweep_config* best) {
    std::vector<rte_sweep_config> cand;
    if (band_mesh(h)) {
        const int nb = (h->ny + 31) / 32;
        std::vector<int> Ws;
        if (nb <= 16) Ws.push_back(nb);
        for (int W : {16, 8, 4, 2, 1})
            if (W < nb) Ws.push_back(W);
        for (int W : Ws)
            for (int D : {2, 4, 8}) {
                if (!band_cfg_valid<T>(h, W, D)) continue;
                for (int sg = 0; sg <= (A.psi && !A.outcols ? 1 : 0); ++sg)
                    // persistent grids (several ordinates per block) while every SM keeps a block
                    for (int apb : {1, 2, 4})
                        if (apb == 1 || n >= apb * h->num_sms) {
                            rte_sweep_config c = {RTE_SWEEP_BAND, W, D, A.outcols ? 1 : sg, apb, 0.f};
                            cand.push_back(c);
                        }
            }
    }
    if (cand.empty())
        for (int wpb : {1, 2, 4})
            if (warp_cfg_valid<T>(h, wpb)) cand.push_back({RTE_SWEEP_WARP, 0, 0, 0, wpb, 0.f});
    if (cand.empty()) return fail(RTE_ERR_ARG, "sweep: nx too large for the shared-memory ring");
    if (cand.size() == 1) {
        *best = cand[0];
        return RTE_OK;
    }
    cudaEvent_t e0, e1;
    RTE_CUDA_TRY(cudaEventCreate(&e0));
    RTE_CUDA_TRY(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    int rc = RTE_OK;
    for (const rte_sweep_config& c : cand) {
        rc = launch_cfg<T>(h, A, n, c, st);
        if (rc != RTE_OK) break;
        cudaEventRecord(e0, st);
        for (int rep = 0; rep < 2 && rc == RTE_OK; ++rep) rc = launch_cfg<T>(h, A, n, c, st);
        cudaEventRecord(e1, st);
        if (rc != RTE_OK || cudaEventSynchronize(e1) != cudaSuccess) {
            if (rc == RTE_OK) rc = fail(RTE_ERR_CUDA, "sweep autotuner: launch failed");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms *= 0.5f;
        if (ms < best_ms) {
            best_ms = ms;
            *best = c;
            best->ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != RTE_OK) return rc;
    return check_dep_flag(h, st);
}

// The configuration of this launch: the cached one; else, for an uncaptured launch with a host
// ordinate count, the tuned one (cached; the tuner's launches are not profiled); else the default.
template <typename T>
static int choose_cfg(rte_handle* h, const SweepArgs<T>& A, int n, cudaStream_t st, rte_sweep_config* c) {
    const int prec = std::is_same<T, float>::value ? RTE_FP32 : RTE_FP64;
    const long long key = cfg_key(prec, A.psi != nullptr, n);
    auto it = h->sweep_cfg.find(key);
    if (it != h->sweep_cfg.end()) {
        *c = it->second;
        return RTE_OK;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    RTE_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone || A.n_dev) {
        *c = default_cfg<T>(h, n, A.psi != nullptr);
        return RTE_OK;
    }
    RTE_TRY(tune_cfg<T>(h, A, n, st, c));
    h->sweep_cfg[key] = *c;
    return RTE_OK;
}

template <typename T>
static int launch_sweep_t(rte_handle* h, const int* d_angles, int n, const void* src, long long src_stride,
                          int add_inflow, int reverse, void* psi, cudaStream_t st, const int* n_dev,
                          const int2* outcols, int n_out) {
    SweepArgs<T> A;
    A.nx = h->nx;
    A.ny = h->ny;
    A.n = n;
    A.hx = (T)h->hx;
    A.hy = (T)h->hy;
    A.gs = (T)sqrt(h->hx * h->hy);
    A.sig_t = std::is_same<T, float>::value ? (const T*)h->sig_t_f : (const T*)h->sig_t;
    A.src = (const T*)src;
    A.src_stride = src_stride;
    A.angles = d_angles;
    A.ox = h->d_ox;
    A.oy = h->d_oy;
    for (int k = 0; k < 4; ++k) A.g[k] = (T)h->inflow[k];
    A.add_inflow = add_inflow;
    A.reverse = reverse;
    A.psi = (T*)psi;
    A.psi_stride = h->ndof;
    A.n_dev = n_dev;
    A.spin_limit = h->wait_limit;
    A.outcols = outcols;
    rte_sweep_config c;
    RTE_TRY(choose_cfg<T>(h, A, n, st, &c));
    RTE_PROF_BEGIN(h, RTE_PROF_SWEEP, st);
    RTE_TRY(launch_cfg<T>(h, A, n, c, st));
    // algorithmic traffic: psi written once per update, source and sigma_t read once per launch;
    // about 100 flops per cell-angle update (RHS, closed-form 4x4 solve, traces, sign flips)
    RTE_PROF_END(h, RTE_PROF_SWEEP, st,
                 (double)sizeof(T) * ((psi ? 4.0 * n_out : 0.0) * h->nc + 5.0 * h->nc), 100.0 * n * h->nc);
    return RTE_OK;
}

// Tune n-ordinate launches (psi written or not) on scratch buffers (zero source, the distinct
// directions repeated up to n), unless a configuration is cached.
int sweep_pretune(rte_handle* h, int precision, int n, int with_psi, cudaStream_t st) {
    const bool f32 = precision == RTE_FP32;
    if (h->sweep_cfg.count(cfg_key(f32 ? RTE_FP32 : RTE_FP64, with_psi != 0, n))) return RTE_OK;
    const size_t esz = f32 ? sizeof(float) : sizeof(double);
    void* src = nullptr;
    void* psi = nullptr;
    void* ang = nullptr;
    // the distinct directions, repeated cyclically up to n entries
    std::vector<int> hang(n);
    const int nf = std::max(1, (int)h->fold_rep.size());
    for (int k = 0; k < n; ++k) hang[k] = h->fold_rep.empty() ? 0 : h->fold_rep[k % nf];
    int rc = h->arena.alloc(&src, esz * h->ndof);
    if (rc == RTE_OK) rc = h->arena.alloc(&ang, sizeof(int) * (size_t)n);
    if (rc == RTE_OK && with_psi) rc = h->arena.alloc(&psi, esz * h->ndof * (size_t)n);
    if (rc == RTE_OK && (cudaMemsetAsync(src, 0, esz * h->ndof, st) != cudaSuccess ||
                         cudaMemcpyAsync(ang, hang.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, st) != cudaSuccess))
        rc = fail(RTE_ERR_CUDA, "sweep tune: scratch setup");
    if (rc == RTE_OK) {
        rc = f32 ? launch_sweep_t<float>(h, (const int*)ang, n, src, 0, 0, 0, psi, st, nullptr, nullptr, n)
                 : launch_sweep_t<double>(h, (const int*)ang, n, src, 0, 0, 0, psi, st, nullptr, nullptr, n);
    }
    cudaStreamSynchronize(st);
    for (void* p : {src, psi, ang}) {
        if (!p) continue;
        auto& v = h->arena.ptrs;
        v.erase(std::remove(v.begin(), v.end(), p), v.end());
        dev_free(p);
    }
    return rc;
}

int launch_sweep(rte_handle* h, const int* d_angles, int n, int precision, const void* src, long long src_stride,
                 int add_inflow, int reverse, void* psi, cudaStream_t st, const int* n_dev, const int2* outcols,
                 int n_out) {
    if (n <= 0) return RTE_OK;
    if (n_out < 0) n_out = n;
    if (precision == RTE_FP32)
        return launch_sweep_t<float>(h, d_angles, n, src, src_stride, add_inflow, reverse, psi, st, n_dev, outcols,
                                     n_out);
    return launch_sweep_t<double>(h, d_angles, n, src, src_stride, add_inflow, reverse, psi, st, n_dev, outcols, n_out);
}

int launch_phi_reduce(rte_handle* h, const int* /*d_angles*/, const double* d_wlist, int n, int precision,
                      const void* psi, double* phi, cudaStream_t st) {
    const int block = 256;
    const int grid = grid_for(h, h->ndof, block);
    if (precision == RTE_FP32)
        phi_reduce_kernel<float><<<grid, block, 0, st>>>(h->ndof, n, d_wlist, (const float*)psi, h->ndof, phi);
    else
        phi_reduce_kernel<double><<<grid, block, 0, st>>>(h->ndof, n, d_wlist, (const double*)psi, h->ndof, phi);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

int launch_source(rte_handle* h, const double* phi, int precision, void* src, cudaStream_t st) {
    const int block = 256;
    const int grid = grid_for(h, h->ndof, block);
    if (precision == RTE_FP32)
        source_kernel<float><<<grid, block, 0, st>>>(h->nc, h->sig_s, phi, h->G, (float*)src);
    else
        source_kernel<double><<<grid, block, 0, st>>>(h->nc, h->sig_s, phi, h->G, (double*)src);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

int max_abs_diff_async(rte_handle* h, const double* a, const double* b, int n, cudaStream_t st) {
    const int block = 256;
    const int grid = std::min(grid_for(h, n, block), 1024);
    max_abs_diff_partial<<<grid, block, 0, st>>>(n, a, b, h->red);
    max_final<<<1, 256, 0, st>>>(grid, h->red, h->red + 4096);
    RTE_CUDA_TRY(cudaGetLastError());
    RTE_CUDA_TRY(cudaMemcpyAsync(h->h_scalar, h->red + 4096, sizeof(double), cudaMemcpyDeviceToHost, st));
    return RTE_OK;
}

int max_abs_diff(rte_handle* h, const double* a, const double* b, int n, double* host_out, cudaStream_t st) {
    RTE_TRY(max_abs_diff_async(h, a, b, n, st));
    RTE_CUDA_TRY(cudaStreamSynchronize(st));
    *host_out = h->h_scalar[0];
    return RTE_OK;
}


template <typename T>
__global__ void phi_reduce2_kernel(int ndof, int n, const double* __restrict__ wlist, const T* __restrict__ psi,
                                   const T* __restrict__ dpsi, long long stride, double* __restrict__ phi) {
    pdl_entry();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ndof; i += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int a = 0; a < n; ++a) {
            const long long o = (long long)a * stride + i;
            acc = fma(wlist[a], (double)psi[o] + (double)dpsi[o], acc);
        }
        phi[i] = acc;
    }
}

template <typename T>
__global__ void to_double2_kernel(long long n, const T* __restrict__ psi, const T* __restrict__ dpsi,
                                  double* __restrict__ out) {
    pdl_entry();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (double)psi[i] + (dpsi ? (double)dpsi[i] : 0.0);
}

int ensure_refine_scratch(rte_handle* h, int n) {
    const size_t bytes = sizeof(float) * (size_t)std::max(n, 1) * h->ndof;
    if (h->dpsi_cap_bytes < bytes) {
        void *p1 = nullptr, *p2 = nullptr;
        RTE_TRY(h->arena.alloc(&p1, bytes));
        RTE_TRY(h->arena.alloc(&p2, bytes));
        h->dpsi_w = p1;
        h->res_w = p2;
        h->dpsi_cap_bytes = bytes;
    }
    return RTE_OK;
}

// ---- defect of an FP32 sweep in double-word FP32 (rte_dw.cuh).  The defect needs a small
// ABSOLUTE error against |b| (it is the right-hand side of a correction solve), which the cheap
// double-word sum provides even where the terms cancel.

// hi/lo split of an FP64 vector (once per defect launch; the source is shared by the ordinates).
__global__ void dw_split_kernel(int n, const double* __restrict__ v, float* __restrict__ hi, float* __restrict__ lo) {
    pdl_entry();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const DW d = dw_of(v[i]);
        hi[i] = d.h;
        lo[i] = d.l;
    }
}

// r_a = b (+ g_j^bc) - (D_j + Sigma_t) psi_a for FP32 psi, written back in FP32.  The upwind
// operator applied matrix-free.  With s_x = sign(Omega_x), s_y = sign(Omega_y), A = a_x,
// B = s_x sqrt3 a_x, C = 3 a_x, D = a_y, E = s_y sqrt3 a_y, F = 3 a_y, the upwind x-neighbour's
// outflow traces t = (q0 + s_x sqrt3 q1, q2 + s_x sqrt3 q3) and the y-neighbour's
// u = (q0 + s_y sqrt3 q2, q1 + s_y sqrt3 q3) (inflow data on the boundary), the residual of
// cell moments v is
//   r0 = b0 - (sigma + A + D) v0 - B v1 - E v2 + A t0 + D u0
//   r1 = b1 + B v0 - (sigma + C + D) v1 - E v3 - B t0 + D u1
//   r2 = b2 + E v0 - (sigma + A + F) v2 - B v3 + A t1 - E u0
//   r3 = b3 + E v1 + B v2 - (sigma + C + F) v3 - B t1 - E u1
// (D_x^+ = -D_x^{-T} gives the Omega_x < 0 form through s_x).  Every product of an FP32 moment
// with an FP64 coefficient and every partial sum is carried in double-word FP32, so the FP64
// pipe (a small fraction of the FP32 rate on this part) is not used per cell.
__global__ void defect_dw_kernel(int nx, int ny, double hx, double hy, const int* __restrict__ angles,
                                 const double* __restrict__ oxa, const double* __restrict__ oya, int reverse,
                                 int add_inflow, double gL, double gR, double gB, double gT,
                                 const float* __restrict__ sig_hi, const float* __restrict__ sig_lo,
                                 const float* __restrict__ b_hi, const float* __restrict__ b_lo,
                                 const float* __restrict__ psi, long long stride, float* __restrict__ out,
                                 const int* __restrict__ n_dev) {
    pdl_entry();
    const int a = blockIdx.y;
    if (n_dev && a >= *n_dev) return;
    // per-ordinate constants, formed once per block by one thread (FP64 division and square
    // root would otherwise dominate a kernel that handles a few cells per thread)
    struct Cst {
        DW A, D, B, E, AD, CD, AF, CF, sx3, sy3, tin, uin;
        int px, py;
    };
    __shared__ Cst K;
    if (threadIdx.x == 0) {
        const int j = angles[a];
        double ox = oxa[j], oy = oya[j];
        if (reverse) { ox = -ox; oy = -oy; }
        const double s3 = 1.7320508075688772935, gs = sqrt(hx * hy);
        const bool px = ox >= 0.0, py = oy >= 0.0;
        const double A = fabs(ox) / hx, D = fabs(oy) / hy;
        const double sx3 = px ? s3 : -s3, sy3 = py ? s3 : -s3;
        K.A = dw_of(A); K.D = dw_of(D); K.B = dw_of(sx3 * A); K.E = dw_of(sy3 * D);
        K.AD = dw_of(A + D); K.CD = dw_of(3.0 * A + D); K.AF = dw_of(A + 3.0 * D); K.CF = dw_of(3.0 * A + 3.0 * D);
        K.sx3 = dw_of(sx3); K.sy3 = dw_of(sy3);
        K.tin = dw_of(add_inflow ? (px ? gL : gR) * gs : 0.0);
        K.uin = dw_of(add_inflow ? (py ? gB : gT) * gs : 0.0);
        K.px = px; K.py = py;
    }
    __syncthreads();
    const bool px = K.px, py = K.py;
    const DW dA = K.A, dD = K.D, dB = K.B, dE = K.E, dAD = K.AD, dCD = K.CD, dAF = K.AF, dCF = K.CF;
    const DW dsx3 = K.sx3, dsy3 = K.sy3, tin = K.tin, uin = K.uin;
    const int dx = px ? -1 : 1, dyc = py ? -nx : nx;
    const float* v = psi + (long long)a * stride;
    float* r = out + (long long)a * stride;
    const int nc = nx * ny;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        const int ix = c % nx, iy = c / nx;
        float v0, v1, v2, v3;
        load4(v + 4 * (long long)c, v0, v1, v2, v3);
        DW t0 = tin, t1 = DW{0.f, 0.f}, u0 = uin, u1 = DW{0.f, 0.f};
        if (px ? ix > 0 : ix + 1 < nx) {
            float q0, q1, q2, q3;
            load4(v + 4 * (long long)(c + dx), q0, q1, q2, q3);
            t0 = dw_add(DW{q0, 0.f}, dw_mul_f(dsx3, q1));
            t1 = dw_add(DW{q2, 0.f}, dw_mul_f(dsx3, q3));
        }
        if (py ? iy > 0 : iy + 1 < ny) {
            float q0, q1, q2, q3;
            load4(v + 4 * (long long)(c + dyc), q0, q1, q2, q3);
            u0 = dw_add(DW{q0, 0.f}, dw_mul_f(dsy3, q2));
            u1 = dw_add(DW{q1, 0.f}, dw_mul_f(dsy3, q3));
        }
        const DW sg{sig_hi[c], sig_lo[c]};
        const float4 bh = *reinterpret_cast<const float4*>(b_hi + 4 * (long long)c);
        const float4 bl = *reinterpret_cast<const float4*>(b_lo + 4 * (long long)c);
        // r0 = b0 - (sigma + A + D) v0 - B v1 - E v2 + A t0 + D u0
        DW r0 = DW{bh.x, bl.x};
        r0 = dw_add(r0, dw_neg(dw_mul_f(dw_add(sg, dAD), v0)));
        r0 = dw_add(r0, dw_neg(dw_mul_f(dB, v1)));
        r0 = dw_add(r0, dw_neg(dw_mul_f(dE, v2)));
        r0 = dw_add(r0, dw_mul(dA, t0));
        r0 = dw_add(r0, dw_mul(dD, u0));
        // r1 = b1 + B v0 - (sigma + C + D) v1 - E v3 - B t0 + D u1
        DW r1 = DW{bh.y, bl.y};
        r1 = dw_add(r1, dw_mul_f(dB, v0));
        r1 = dw_add(r1, dw_neg(dw_mul_f(dw_add(sg, dCD), v1)));
        r1 = dw_add(r1, dw_neg(dw_mul_f(dE, v3)));
        r1 = dw_add(r1, dw_neg(dw_mul(dB, t0)));
        r1 = dw_add(r1, dw_mul(dD, u1));
        // r2 = b2 + E v0 - (sigma + A + F) v2 - B v3 + A t1 - E u0
        DW r2 = DW{bh.z, bl.z};
        r2 = dw_add(r2, dw_mul_f(dE, v0));
        r2 = dw_add(r2, dw_neg(dw_mul_f(dw_add(sg, dAF), v2)));
        r2 = dw_add(r2, dw_neg(dw_mul_f(dB, v3)));
        r2 = dw_add(r2, dw_mul(dA, t1));
        r2 = dw_add(r2, dw_neg(dw_mul(dE, u0)));
        // r3 = b3 + E v1 + B v2 - (sigma + C + F) v3 - B t1 - E u1
        DW r3 = DW{bh.w, bl.w};
        r3 = dw_add(r3, dw_mul_f(dE, v1));
        r3 = dw_add(r3, dw_mul_f(dB, v2));
        r3 = dw_add(r3, dw_neg(dw_mul_f(dw_add(sg, dCF), v3)));
        r3 = dw_add(r3, dw_neg(dw_mul(dB, t1)));
        r3 = dw_add(r3, dw_neg(dw_mul(dE, u1)));
        store4(r + 4 * (long long)c, __fadd_rn(r0.h, r0.l), __fadd_rn(r1.h, r1.l), __fadd_rn(r2.h, r2.l),
               __fadd_rn(r3.h, r3.l));
    }
}

int launch_defect(rte_handle* h, const int* d_angles, int n, const double* b64, int add_inflow, int reverse,
                  const void* psi, const int* n_dev, cudaStream_t st) {
    dim3 grid((unsigned)std::max(1, std::min((h->nc + 1023) / 1024, 64)), (unsigned)n);
    RTE_PROF_BEGIN(h, RTE_PROF_RESID, st);
    const int g1 = std::max(1, std::min((h->ndof + 255) / 256, 4 * std::max(h->num_sms, 1)));
    dw_split_kernel<<<g1, 256, 0, st>>>(h->ndof, b64, h->b_dw, h->b_dw + h->ndof);
    defect_dw_kernel<<<grid, 256, 0, st>>>(h->nx, h->ny, h->hx, h->hy, d_angles, h->d_ox, h->d_oy, reverse, add_inflow,
                                           h->inflow[0], h->inflow[1], h->inflow[2], h->inflow[3], h->sig_dw,
                                           h->sig_dw + h->nc, h->b_dw, h->b_dw + h->ndof, (const float*)psi, h->ndof,
                                           (float*)h->res_w, n_dev);
    RTE_PROF_END(h, RTE_PROF_RESID, st, (double)n * h->nc * (16.0 + 16.0) + 40.0 * h->nc, 60.0 * n * h->nc);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

int sweep_refined(rte_handle* h, const int* d_angles, int n, int precision, int refine, const void* src,
                  const double* b64, int add_inflow, int reverse, void* psi, void** dpsi_out, const int* n_dev,
                  cudaStream_t st) {
    *dpsi_out = nullptr;
    RTE_TRY(launch_sweep(h, d_angles, n, precision, src, 0, add_inflow, reverse, psi, st, n_dev));
    if (precision != RTE_FP32 || !refine || n <= 0) return RTE_OK;
    RTE_TRY(ensure_refine_scratch(h, n));
    RTE_TRY(launch_defect(h, d_angles, n, b64, add_inflow, reverse, psi, n_dev, st));
    RTE_TRY(launch_sweep(h, d_angles, n, precision, h->res_w, h->ndof, 0, reverse, h->dpsi_w, st, n_dev));
    *dpsi_out = h->dpsi_w;
    return RTE_OK;
}

int launch_phi_reduce2(rte_handle* h, const double* d_wlist, int n, int precision, const void* psi, const void* dpsi,
                       double* phi, cudaStream_t st) {
    if (!dpsi) return launch_phi_reduce(h, nullptr, d_wlist, n, precision, psi, phi, st);
    const int block = 256;
    const int grid = grid_for(h, h->ndof, block);
    phi_reduce2_kernel<float><<<grid, block, 0, st>>>(h->ndof, n, d_wlist, (const float*)psi, (const float*)dpsi,
                                                      h->ndof, phi);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

int launch_to_double2(rte_handle* h, int n, int precision, const void* psi, const void* dpsi, double* out,
                      cudaStream_t st) {
    const long long tot = (long long)n * h->ndof;
    const int grid = grid_for(h, tot, 256);
    if (precision == RTE_FP32)
        to_double2_kernel<float><<<grid, 256, 0, st>>>(tot, (const float*)psi, (const float*)dpsi, out);
    else
        to_double2_kernel<double><<<grid, 256, 0, st>>>(tot, (const double*)psi, (const double*)dpsi, out);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

int check_dep_flag(rte_handle* h, cudaStream_t st) {
    int* hv = reinterpret_cast<int*>(h->h_scalar + 16);
    RTE_CUDA_TRY(cudaMemcpyAsync(hv, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    RTE_CUDA_TRY(cudaStreamSynchronize(st));
    if (*hv) {
        RTE_CUDA_TRY(cudaMemsetAsync(h->d_err, 0, sizeof(int), st));
        return fail(RTE_ERR_DEP_TIMEOUT, "sweep: a band hand-off wait ran out");
    }
    return RTE_OK;
}

int ensure_psi_scratch(rte_handle* h, size_t bytes) {
    if (h->psi_cap_bytes >= bytes) return RTE_OK;
    void* p = nullptr;
    RTE_TRY(h->arena.alloc(&p, bytes));
    h->psi_w = p;          // the previous (smaller) block stays in the arena until rte_destroy
    h->psi_cap_bytes = bytes;
    return RTE_OK;
}

// A kernel of this translation unit (its CUDA library is enumerated by preload_all_kernels).
const void* sweep_kernel_anchor() { return (const void*)source_kernel<double>; }

}  // namespace rte

using namespace rte;

static int sweep_common(rte_handle* h, const int* angles, int n, int precision, const void* src, int src_per_angle,
                        int add_inflow, int reverse, void* psi_out, double* phi_out) {
    if (!h || (n > 0 && (!angles || !src))) return fail(RTE_ERR_ARG, "rte_sweep: null argument");
    if (n < 0 || n > h->nang) return fail(RTE_ERR_ARG, "rte_sweep: n_angles out of range");
    if (precision != RTE_FP32 && precision != RTE_FP64) return fail(RTE_ERR_ARG, "rte_sweep: bad precision");
    if (((uintptr_t)src | (uintptr_t)psi_out | (uintptr_t)phi_out) & 15)
        return fail(RTE_ERR_ARG, "rte_sweep: src, psi_out and phi_out must be 16-byte aligned");
    for (int a = 0; a < n; ++a)
        if (angles[a] < 0 || angles[a] >= h->nang) return fail(RTE_ERR_ARG, "rte_sweep: angle index out of range");
    if (n == 0) {
        if (phi_out) RTE_CUDA_TRY(cudaMemsetAsync(phi_out, 0, sizeof(double) * h->ndof, h->stream));
        return RTE_OK;
    }
    const size_t esz = precision == RTE_FP32 ? sizeof(float) : sizeof(double);
    if (h->pinned_busy) {        // the pinned staging buffers are reused: their last copies must be done
        RTE_CUDA_TRY(cudaEventSynchronize(h->ev_pinned));
        h->pinned_busy = false;
    }
    void* psi = psi_out;
    if (!psi && phi_out) {
        RTE_TRY(ensure_psi_scratch(h, esz * (size_t)n * h->ndof));
        psi = h->psi_w;
    }
    // With a shared source, an ordinate and its +-Omega_z twin (or a repeat of the same ordinate)
    // have the same psi (the S_N system depends on (Omega_x, Omega_y) only): each such pair is
    // solved once and written to both output columns.
    int n_items = n;
    const int2* d_out = nullptr;
    if (!src_per_angle && psi) {
        std::vector<int> first(h->nang, -1);             // open item of each distinct direction
        std::vector<int> item_angle;
        std::vector<int2> oc;
        for (int a = 0; a < n; ++a) {
            const int j = angles[a], key = std::min(j, h->twin[j]);
            if (first[key] >= 0) {
                oc[first[key]].y = a;
                first[key] = -1;
            } else {
                first[key] = (int)oc.size();
                item_angle.push_back(j);
                oc.push_back(make_int2(a, -1));
            }
        }
        n_items = (int)item_angle.size();
        memcpy(h->h_angles, item_angle.data(), sizeof(int) * n_items);
        memcpy(h->h_outcols, oc.data(), sizeof(int2) * n_items);
        RTE_CUDA_TRY(cudaMemcpyAsync(h->d_outcols, h->h_outcols, sizeof(int2) * n_items, cudaMemcpyHostToDevice,
                                     h->stream));
        d_out = h->d_outcols;
    } else {
        memcpy(h->h_angles, angles, sizeof(int) * n);
    }
    RTE_CUDA_TRY(cudaMemcpyAsync(h->d_angles, h->h_angles, sizeof(int) * n_items, cudaMemcpyHostToDevice, h->stream));
    if (phi_out) {               // psi holds the caller's columns in list order: weights by position
        for (int a = 0; a < n; ++a) h->h_wlist[a] = h->w[angles[a]];
        RTE_CUDA_TRY(cudaMemcpyAsync(h->d_wlist, h->h_wlist, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
    }
    RTE_CUDA_TRY(cudaEventRecord(h->ev_pinned, h->stream));
    h->pinned_busy = true;
    RTE_TRY(launch_sweep(h, h->d_angles, n_items, precision, src, src_per_angle ? h->ndof : 0, add_inflow, reverse,
                         psi, h->stream, nullptr, d_out, n));
    if (phi_out) RTE_TRY(launch_phi_reduce(h, h->d_angles, h->d_wlist, n, precision, psi, phi_out, h->stream));
    return check_dep_flag(h, h->stream);
}

extern "C" int rte_sweep(rte_handle* h, const int* angles, int n, int precision, const void* src, int src_per_angle,
                         int add_inflow, void* psi_out, double* phi_out) {
    return sweep_common(h, angles, n, precision, src, src_per_angle, add_inflow, 0, psi_out, phi_out);
}

extern "C" int rte_sweep_adjoint(rte_handle* h, const int* angles, int n, int precision, const void* src,
                                 int src_per_angle, void* mu_out, double* chi_out) {
    return sweep_common(h, angles, n, precision, src, src_per_angle, 0, 1, mu_out, chi_out);
}

// ---------------------------------------------------------------------------------------------
// Batched sweeps over several problems in one launch.
namespace rte {

template <typename T>
static SweepArgs<T> make_args(const rte_handle* h, const int* d_angles, int n, const void* src, long long src_stride,
                              int add_inflow, int reverse, void* psi) {
    SweepArgs<T> A;
    A.nx = h->nx;
    A.ny = h->ny;
    A.n = n;
    A.hx = (T)h->hx;
    A.hy = (T)h->hy;
    A.gs = (T)sqrt(h->hx * h->hy);
    A.sig_t = std::is_same<T, float>::value ? (const T*)h->sig_t_f : (const T*)h->sig_t;
    A.src = (const T*)src;
    A.src_stride = src_stride;
    A.angles = d_angles;
    A.ox = h->d_ox;
    A.oy = h->d_oy;
    for (int k = 0; k < 4; ++k) A.g[k] = (T)h->inflow[k];
    A.add_inflow = add_inflow;
    A.reverse = reverse;
    A.psi = (T*)psi;
    A.psi_stride = h->ndof;
    A.n_dev = nullptr;
    A.spin_limit = h->wait_limit;
    A.outcols = nullptr;
    return A;
}

// The batched kernel gives every band its own warp (block = 32 x the largest band count), so
// band b only ever waits for band b - 1 and the hand-off chain cannot close into a cycle; the
// block size caps the band count at 16 (ny <= 512).
bool batch_supported(rte_handle* const* hs, int nprob, int precision) {
    int W = 1;
    for (int i = 0; i < nprob; ++i) {
        if (hs[i]->ny > 16 * 32) return false;
        W = std::max(W, (hs[i]->ny + 31) / 32);
    }
    // every problem's ring must fit the block's shared memory (the block size is the tallest mesh's)
    for (int i = 0; i < nprob; ++i) {
        const size_t sm = precision == RTE_FP32 ? band_smem_bytes<float>(W, hs[i]->nx, kBandDepth)
                                                : band_smem_bytes<double>(W, hs[i]->nx, kBandDepth);
        if (sm > 200 * 1024) return false;
    }
    return true;
}

// Sweep problem i's n[i] angles (device list d_angles[i]) with source src[i] (stride
// src_stride[i] per angle) into psi[i], all problems in one launch on stream st.
template <typename T>
static int launch_batch_t(rte_handle* const* hs, int nprob, const int* const* d_angles, const int* n,
                          const void* const* src, const long long* src_stride, int add_inflow, int reverse,
                          void* const* psi, cudaStream_t st, rte_handle* owner) {
    std::vector<SweepArgs<T>> args(nprob);
    std::vector<int2> items;
    int W = 1;
    size_t smem = 0;
    constexpr int Dp = kBandDepth;
    for (int i = 0; i < nprob; ++i) {
        args[i] = make_args<T>(hs[i], d_angles[i], n[i], src[i], src_stride[i], add_inflow, reverse, psi[i]);
        W = std::max(W, (hs[i]->ny + 31) / 32);
        for (int a = 0; a < n[i]; ++a) items.push_back(make_int2(i, a));
    }
    // longest sweeps first: blocks are dispatched in index order, so this keeps the long
    // problems off the tail of the launch
    std::stable_sort(items.begin(), items.end(), [&](const int2& u, const int2& v) {
        const long long cu = (long long)(hs[u.x]->nx + 32) * ((hs[u.x]->ny + 31) / 32);
        const long long cv = (long long)(hs[v.x]->nx + 32) * ((hs[v.x]->ny + 31) / 32);
        return cu > cv;
    });
    for (int i = 0; i < nprob; ++i)
        smem = std::max(smem, band_smem_bytes<T>(W, hs[i]->nx, Dp));
    if (items.empty()) return RTE_OK;
    if (smem > 200 * 1024) return fail(RTE_ERR_ARG, "batched sweep: meshes too wide for the shared-memory ring");
    const size_t abytes = (sizeof(SweepArgs<T>) * nprob + 255) & ~(size_t)255;
    RTE_TRY(owner->arena.grow(&owner->sweep_batch_buf, &owner->sweep_batch_cap, abytes + sizeof(int2) * items.size()));
    SweepArgs<T>* d_args = (SweepArgs<T>*)owner->sweep_batch_buf;
    int2* d_items = (int2*)((char*)owner->sweep_batch_buf + abytes);
    RTE_CUDA_TRY(cudaMemcpyAsync(d_args, args.data(), sizeof(SweepArgs<T>) * nprob, cudaMemcpyHostToDevice, st));
    RTE_CUDA_TRY(cudaMemcpyAsync(d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice, st));
    RTE_TRY(smem_optin(sweep_band_batch_kernel<T, Dp>, smem));
    double bytes = 0, fl = 0;
    for (int i = 0; i < nprob; ++i) {
        bytes += (double)sizeof(T) * (4.0 * n[i] * hs[i]->nc + 5.0 * hs[i]->nc);
        fl += 100.0 * n[i] * hs[i]->nc;
    }
    RTE_PROF_BEGIN(owner, RTE_PROF_SWEEP, st);
    sweep_band_batch_kernel<T, Dp><<<(unsigned)items.size(), 32 * W, smem, st>>>(d_args, d_items, owner->d_err);
    RTE_PROF_END(owner, RTE_PROF_SWEEP, st, bytes, fl);
    RTE_CUDA_TRY(cudaGetLastError());
    // the pageable argument vectors are staged before cudaMemcpyAsync returns; a later batch
    // overwrites the device copy only after this launch in stream order
    return RTE_OK;
}

int launch_sweep_batch(rte_handle* const* hs, int nprob, const int* const* d_angles, const int* n, int precision,
                       const void* const* src, const long long* src_stride, int add_inflow, int reverse,
                       void* const* psi, cudaStream_t st) {
    if (precision == RTE_FP32)
        return launch_batch_t<float>(hs, nprob, d_angles, n, src, src_stride, add_inflow, reverse, psi, st, hs[0]);
    return launch_batch_t<double>(hs, nprob, d_angles, n, src, src_stride, add_inflow, reverse, psi, st, hs[0]);
}

}  // namespace rte

extern "C" int rte_sweep_batch(rte_handle* const* hs, int nprob, const int* const* angles, const int* n_angles,
                               int precision, const void* const* src, int add_inflow, void* const* psi_out) {
    using namespace rte;
    if (!hs || nprob < 1 || !angles || !n_angles || !src || !psi_out) return fail(RTE_ERR_ARG, "rte_sweep_batch: null argument");
    if (precision != RTE_FP32 && precision != RTE_FP64) return fail(RTE_ERR_ARG, "rte_sweep_batch: bad precision");
    for (int i = 0; i < nprob; ++i) {
        if (!hs[i] || !src[i] || !psi_out[i] || (!angles[i] && n_angles[i] > 0)) return fail(RTE_ERR_ARG, "rte_sweep_batch: null entry");
        if (n_angles[i] < 0 || n_angles[i] > hs[i]->nang) return fail(RTE_ERR_ARG, "rte_sweep_batch: n_angles out of range");
        if (((uintptr_t)src[i] | (uintptr_t)psi_out[i]) & 15) return fail(RTE_ERR_ARG, "rte_sweep_batch: buffers must be 16-byte aligned");
        for (int a = 0; a < n_angles[i]; ++a)
            if (angles[i][a] < 0 || angles[i][a] >= hs[i]->nang) return fail(RTE_ERR_ARG, "rte_sweep_batch: angle out of range");
    }
    cudaStream_t st = hs[0]->stream;
    if (!batch_supported(hs, nprob, precision)) {
        // meshes outside the batched kernel's shape range: one rte_sweep per problem
        for (int i = 0; i < nprob; ++i)
            RTE_TRY(rte_sweep(hs[i], angles[i], n_angles[i], precision, src[i], 0, add_inflow ? 1 : 0, psi_out[i], nullptr));
        return RTE_OK;
    }
    // earlier work of every handle (which may still read its staged angle list) completes first
    for (int i = 0; i < nprob; ++i)
        if (hs[i]->stream != st) RTE_CUDA_TRY(cudaStreamSynchronize(hs[i]->stream));
    RTE_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<const int*> dl(nprob);
    std::vector<long long> strides(nprob, 0);
    for (int i = 0; i < nprob; ++i) {
        memcpy(hs[i]->h_angles, angles[i], sizeof(int) * n_angles[i]);
        RTE_CUDA_TRY(cudaMemcpyAsync(hs[i]->d_angles, hs[i]->h_angles, sizeof(int) * n_angles[i], cudaMemcpyHostToDevice, st));
        dl[i] = hs[i]->d_angles;
    }
    RTE_TRY(launch_sweep_batch(hs, nprob, dl.data(), n_angles, precision, src, strides.data(), add_inflow ? 1 : 0, 0,
                               psi_out, st));
    return check_dep_flag(hs[0], st);
}

static int sweep_cfg_args(rte_handle* h, int precision, int n, int with_psi, const char* who) {
    if (!h) return fail(RTE_ERR_ARG, std::string(who) + ": null handle");
    if (precision != RTE_FP32 && precision != RTE_FP64) return fail(RTE_ERR_ARG, std::string(who) + ": bad precision");
    if (n < 1 || n > h->nang) return fail(RTE_ERR_ARG, std::string(who) + ": need 1 <= n <= N_Omega");
    if (with_psi != 0 && with_psi != 1) return fail(RTE_ERR_ARG, std::string(who) + ": with_psi must be 0 or 1");
    return RTE_OK;
}

extern "C" int rte_sweep_tune(rte_handle* h, int precision, int n, int with_psi, rte_sweep_config* out) {
    RTE_TRY(sweep_cfg_args(h, precision, n, with_psi, "rte_sweep_tune"));
    h->sweep_cfg.erase(cfg_key(precision, with_psi != 0, n));
    RTE_TRY(sweep_pretune(h, precision, n, with_psi, h->stream));
    if (out) {
        auto it = h->sweep_cfg.find(cfg_key(precision, with_psi != 0, n));
        if (it == h->sweep_cfg.end()) return fail(RTE_ERR_STATE, "rte_sweep_tune: no configuration (profiling on?)");
        *out = it->second;
    }
    return RTE_OK;
}

extern "C" int rte_sweep_set_config(rte_handle* h, int precision, int n, int with_psi, const rte_sweep_config* cfg) {
    RTE_TRY(sweep_cfg_args(h, precision, n, with_psi, "rte_sweep_set_config"));
    const long long key = cfg_key(precision, with_psi != 0, n);
    if (!cfg) {
        h->sweep_cfg.erase(key);
        return RTE_OK;
    }
    const bool ok = precision == RTE_FP32 ? cfg_valid<float>(h, *cfg) : cfg_valid<double>(h, *cfg);
    if (!ok) return fail(RTE_ERR_ARG, "rte_sweep_set_config: configuration not valid for this mesh");
    rte_sweep_config c = *cfg;
    c.ms = 0.f;
    h->sweep_cfg[key] = c;
    return RTE_OK;
}

extern "C" int rte_sweep_get_config(rte_handle* h, int precision, int n, int with_psi, rte_sweep_config* out) {
    RTE_TRY(sweep_cfg_args(h, precision, n, with_psi, "rte_sweep_get_config"));
    if (!out) return fail(RTE_ERR_ARG, "rte_sweep_get_config: null output");
    auto it = h->sweep_cfg.find(cfg_key(precision, with_psi != 0, n));
    if (it != h->sweep_cfg.end()) *out = it->second;
    else *out = precision == RTE_FP32 ? default_cfg<float>(h, n, with_psi != 0) : default_cfg<double>(h, n, with_psi != 0);
    return RTE_OK;
}
