// First projection of the block of swept snapshots onto the spatial basis, X^T Psi (Sec. 3.1,
// step 2; Alg. 2 line "Delta c = X^T psi" of the first pass), on the 5th-generation tensor cores.
//
// Alg. 2 projects every snapshot at least twice.  The first pass only has to remove the bulk of
// the snapshot's component in span(X): whatever error its coefficients carry stays in span(X)
// and is removed by the second pass, which runs in double-word FP32 (about 48 bits) on the CUDA
// cores, and the coefficient of the R column is the exact sum of both passes' coefficients.  So
// the first pass may run at reduced precision; here it runs as a tall-skinny GEMM
//   D[k][v] = sum_i X(i, k) Psi(i, v)      (k < r basis columns, v < 8 snapshots, i < N_x)
// with tcgen05.mma kind::tf32 and FP32 accumulation in tensor memory, in split precision: each
// FP32 operand x is cut into x_hi = x with the low 13 mantissa bits cleared (exactly a TF32
// number) and x_lo = x - x_hi (exact in FP32), and the four products hi*hi + hi*lo + lo*hi +
// lo*lo are accumulated (the split-TF32 scheme of Ootomo and Yokota, 2022).  The products are
// then accurate to about 2^-21 of |x||y| and the sums to FP32 accumulation (a few 1e-7 of the sum
// of absolute products), against about 1e-3 for plain TF32.
//
// The operands come already split: the basis X (its double-word high part) is kept as two FP32
// arrays, X_tf = the TF32 high part and X_lo = the remainder, written when a column is appended,
// and the snapshots likewise when they are formed, so the kernel itself does no arithmetic on
// the CUDA cores.
//
// Work decomposition: CTA (b, m) takes basis columns [128 m, 128 m + 128) and rows
// [rows_per_cta b, rows_per_cta (b + 1)) (split K); its 128 x 16 FP32 accumulator lives in 32
// TMEM columns (snapshot rows past the tensor are the zero fill of the tensor map).  The rows
// stream through a ring of 32-row stages, each holding four TMA tiles (cp.async.bulk.tensor,
// 128-byte swizzle, K-major: a basis column or a snapshot is a row of a tile and 32 consecutive
// FP32 entries of it one 128-byte line): A_tf, A_lo (128 columns) and B_tf, B_lo (16 snapshots).
// Thread 0 (warp 0) is the producer: it waits for a stage's "empty" barrier, then loads it and
// the TMA transaction count completes its "full" barrier.  Thread 32 (warp 1) waits for "full",
// issues the stage's 16 MMAs (4 K-steps of 8 x 4 products) and commits them to "empty".  After
// the last stage it commits to "done"; the epilogue reads the accumulator with tcgen05.ld (warp w
// owns TMEM lanes 32 w .. 32 w + 31 = basis columns) and writes the CTA's partial sums in the
// layout of the CUDA-core X^T V pass, so the same FP64 reduction adds them up.  The CTAs of
// column tile 0 also form each snapshot's partial sum of squares over their rows in double-word
// FP32 (the snapshot norms the basis update needs).  Every barrier wait is bounded: a wait that
// runs out sets *err, the CTA stops issuing work, waits (bounded) for the copies and MMAs it
// issued, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <stdint.h>

#include <algorithm>

#include "rte_internal.cuh"
#include "rte_dw.cuh"

namespace rte {
namespace {

constexpr int kTcM = 128;                 // basis columns per CTA (MMA M)
constexpr int kTcN = 16;                  // snapshot rows of the B tiles (MMA N)
constexpr int kTcK = 32;                  // rows of X per stage: one 128-byte swizzle line of FP32
constexpr int kTcStages = 3;
constexpr int kTcABytes = kTcM * kTcK * 4;              // 16 KB
constexpr int kTcBBytes = kTcN * kTcK * 4;              // 2 KB
constexpr int kTcStageBytes = 2 * kTcABytes + 2 * kTcBBytes;   // A tf | A lo | B tf | B lo
constexpr int kTcSmem = kTcStages * kTcStageBytes + 1024;      // + alignment slack
constexpr int kTcTmemCols = 32;           // smallest allocation; the accumulator uses 16
constexpr long long kTcSpin = 1ll << 22;  // polls of a barrier before a wait gives up

// Instruction descriptor of tcgen05.mma kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32 (bits
// 7-9 and 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kTcIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                              ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major tile with 128-byte swizzle, 8-row groups 1024 bytes
// apart (stride byte offset), leading byte offset unused for this layout (encoded 1), descriptor
// version 1 (bits 46-47), layout type SWIZZLE_128B = 2 (bits 61-63).  Start address in 16-byte
// units; the tile base is 1024-byte aligned, so the base offset field stays 0.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// bounded wait for the phase with the given parity to complete; false when the wait ran out
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (long long it = 0; it < kTcSpin; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(kTcIdesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// stop: the chain's "inner loop finished" flag (nothing to do); rank: the current basis size r.
// part[((b kxtv) + v) rc + k] = sum over rows of CTA b of X(i, k) Psi(i, v0 + v), v < nv <= 8;
// npart[v nblk + b] = sum over the same rows of Psi(i, v0 + v)^2 (column tile 0 only, from the
// double-word snapshots psi2).
struct TcMaps {
    CUtensorMap xt, xl, vt, vl;     // X_tf, X_lo [rc][N]; Psi_tf, Psi_lo [nv_total][N]
};

__global__ void __launch_bounds__(128) xt_tc_kernel(const __grid_constant__ TcMaps maps, int N, int rows_per_cta,
                                                     const int* __restrict__ stop, const int* __restrict__ rank,
                                                     int v0, int nv, double* __restrict__ part, int rc, int kxtv,
                                                     const float2* __restrict__ psi2, double* __restrict__ npart,
                                                     int* err) {
    pdl_entry();
    if (*stop) return;                                                 // uniform over the launch
    const int r = *rank;
    const int m0 = blockIdx.y * kTcM;
    const int row0 = blockIdx.x * rows_per_cta;
    const int rows = min(rows_per_cta, N - row0);
    if (rows <= 0) return;
    if (npart && blockIdx.y == 0) {
        // all nv sums of squares in one pass and one block reduction
        __shared__ double nsum[8][4];
        DW acc[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[v] = DW{0.f, 0.f};
        for (int i = threadIdx.x; i < rows; i += blockDim.x)
#pragma unroll
            for (int v = 0; v < 8; ++v)
                if (v < nv) {
                    const float2 yy = psi2[(long long)(v0 + v) * N + row0 + i];
                    dw_mac(acc[v], DW{yy.x, yy.y}, DW{yy.x, yy.y});
                }
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const DW w = dw_warp_sum(dw_norm(acc[v]));
            if ((threadIdx.x & 31) == 0) nsum[v][threadIdx.x >> 5] = (double)w.h + (double)w.l;
        }
        __syncthreads();
        if (threadIdx.x < nv)
            npart[(long long)threadIdx.x * gridDim.x + blockIdx.x] =
                ((nsum[threadIdx.x][0] + nsum[threadIdx.x][1]) + nsum[threadIdx.x][2]) + nsum[threadIdx.x][3];
    }
    if (m0 >= r) return;                                               // uniform per CTA
    const int ntile = (rows + kTcK - 1) / kTcK;

    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) &
                                                         ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[kTcStages], empty_bar[kTcStages], done_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh, consumed_sh, issued_sh;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(kTcTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&done_bar, 1);
        abort_sh = 0;
        consumed_sh = 0;
        issued_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;
    auto stage_ptr = [&](int s) { return sm + (size_t)s * kTcStageBytes; };

    if (threadIdx.x == 0) {
        // producer: stage s of tile t, after the MMAs of tile t - kTcStages have released it
        int issued = 0;
        for (int t = 0; t < ntile; ++t) {
            const int s = t % kTcStages;
            if (t >= kTcStages && !mbar_wait(&empty_bar[s], (uint32_t)(((t / kTcStages) - 1) & 1))) {
                atomicExch(&abort_sh, 1);
                break;
            }
            if (*(volatile int*)&abort_sh) break;
            unsigned char* p = stage_ptr(s);
            const int x = row0 + t * kTcK;
            mbar_expect_tx(&full_bar[s], 2 * kTcABytes + 2 * kTcBBytes);
            tma_load_2d(p, &maps.xt, x, m0, &full_bar[s]);
            tma_load_2d(p + kTcABytes, &maps.xl, x, m0, &full_bar[s]);
            tma_load_2d(p + 2 * kTcABytes, &maps.vt, x, v0, &full_bar[s]);
            tma_load_2d(p + 2 * kTcABytes + kTcBBytes, &maps.vl, x, v0, &full_bar[s]);
            issued = t + 1;
        }
        issued_sh = issued;
    } else if (threadIdx.x == 32) {
        // MMA issuer
        int consumed = 0;
        for (int t = 0; t < ntile; ++t) {
            const int s = t % kTcStages;
            if (!mbar_wait(&full_bar[s], (uint32_t)((t / kTcStages) & 1))) {
                atomicExch(&abort_sh, 1);
                break;
            }
            consumed = t + 1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            unsigned char* p = stage_ptr(s);
            const uint32_t at = smem_u32(p), al = smem_u32(p + kTcABytes), bt = smem_u32(p + 2 * kTcABytes),
                           bl = smem_u32(p + 2 * kTcABytes + kTcBBytes);
#pragma unroll
            for (int kk = 0; kk < kTcK / 8; ++kk) {          // K = 8 TF32 = 32 bytes per MMA
                const uint32_t off = 32u * kk;
                const uint32_t acc0 = (t > 0 || kk > 0) ? 1u : 0u;
                tc_mma(tmem, sw128_desc(at + off), sw128_desc(bt + off), acc0);
                tc_mma(tmem, sw128_desc(at + off), sw128_desc(bl + off), 1u);
                tc_mma(tmem, sw128_desc(al + off), sw128_desc(bt + off), 1u);
                tc_mma(tmem, sw128_desc(al + off), sw128_desc(bl + off), 1u);
            }
            tc_commit(&empty_bar[s]);
            if (*(volatile int*)&abort_sh) break;
        }
        *(volatile int*)&consumed_sh = consumed;
        tc_commit(&done_bar);                        // every MMA issued above -> done_bar
    }
    const bool ok_done = mbar_wait(&done_bar, 0);
    __syncthreads();
    const bool good = ok_done && !abort_sh && consumed_sh == ntile;
    if (threadIdx.x == 0 && !good) {
        atomicExch(err, 1);
        // copies issued but never waited for (at most kTcStages): let them land before the CTA
        // exits (bounded waits on the phase each one completes)
        for (int t = consumed_sh; t < issued_sh; ++t)
            if (!mbar_wait(&full_bar[t % kTcStages], (uint32_t)((t / kTcStages) & 1))) break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (good) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int k = m0 + 32 * warp + lane;
        if (k < r)
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j < nv) part[((long long)blockIdx.x * kxtv + j) * rc + k] = (double)__uint_as_float(v[j]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
}

// TF32 high part (low 13 mantissa bits cleared) and the exact FP32 remainder of x
__device__ __forceinline__ void tf32_split(float x, float& t, float& l) {
    t = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
    l = __fsub_rn(x, t);
}

__global__ void tc_split_kernel(long long n, const float* __restrict__ x, float* __restrict__ t, float* __restrict__ l) {
    pdl_entry();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        tf32_split(x[i], t[i], l[i]);
}

static PFN_cuTensorMapEncodeTiled_v12000 lookup_encode_fn() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    return nullptr;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = lookup_encode_fn();   // thread-safe, once
    return fn;
}

// 2D FP32 tensor [rows_outer][inner] (inner contiguous) with a box of box_outer x 32 entries,
// 128-byte swizzle, zero fill outside
int encode_2d(CUtensorMap* m, const float* base, long long inner, long long outer, int box_outer) {
    auto fn = encode_fn();
    if (!fn) return fail(RTE_ERR_CUDA, "tensor-core projection: cuTensorMapEncodeTiled unavailable");
    if (((uintptr_t)base & 15) || (inner * 4) % 16)
        return fail(RTE_ERR_ARG, "tensor-core projection: operands must be 16-byte aligned with rows of 4k entries");
    const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    const cuuint64_t strides[1] = {(cuuint64_t)inner * 4};
    const cuuint32_t box[2] = {(cuuint32_t)kTcK, (cuuint32_t)box_outer};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(RTE_ERR_CUDA, "tensor-core projection: tensor map encoding failed");
    return RTE_OK;
}

}  // namespace

// out[v r + k] = sum_b part[((b kxtv) + v) rc + k] in a fixed order (one thread per entry)
__global__ void tc_reduce(const double* __restrict__ part, int nblk, int kxtv, int rc, int r, int nv,
                          double* __restrict__ out) {
    pdl_entry();
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= r * nv) return;
    const int v = e / r, k = e % r;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[((long long)b * kxtv + v) * rc + k];
    out[e] = s;
}

__global__ void tc_set_state(int* st, int r) {
    pdl_entry();
    st[0] = 0;      // stop
    st[1] = r;      // rank
}

int tc_projection_prepare(TcProjection* P, const float* Xt, const float* Xl, int N, int rc, const float* Vt,
                          const float* Vl, int nv_total) {
    TcMaps* m = reinterpret_cast<TcMaps*>(P->maps);
    RTE_TRY(encode_2d(&m->xt, Xt, N, rc, kTcM));
    RTE_TRY(encode_2d(&m->xl, Xl, N, rc, kTcM));
    RTE_TRY(encode_2d(&m->vt, Vt, N, nv_total, kTcN));
    RTE_TRY(encode_2d(&m->vl, Vl, N, nv_total, kTcN));
    RTE_TRY(smem_optin(xt_tc_kernel, kTcSmem));
    P->N = N;
    P->rc = rc;
    P->ready = true;
    return RTE_OK;
}

int tc_projection_launch(const TcProjection* P, int v0, int nv, int rows_per_cta, int nblk, const int* stop,
                         const int* rank, double* part, int kxtv, const float2* psi2, double* npart, int* err,
                         cudaStream_t s) {
    if (!P->ready || nv < 1 || nv > 8 || v0 < 0 || rows_per_cta % kTcK || rows_per_cta < kTcK)
        return fail(RTE_ERR_ARG, "tensor-core projection: bad launch");
    const dim3 grid(nblk, (P->rc + kTcM - 1) / kTcM);
    xt_tc_kernel<<<grid, 128, kTcSmem, s>>>(*reinterpret_cast<const TcMaps*>(P->maps), P->N, rows_per_cta, stop,
                                            rank, v0, nv, part, P->rc, kxtv, psi2, npart, err);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

int tc_split(const float* x, long long n, float* t, float* l, cudaStream_t s) {
    const long long g = std::min((n + 255) / 256, 4096ll);
    tc_split_kernel<<<(int)std::max(1ll, g), 256, 0, s>>>(n, x, t, l);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

// A kernel of this translation unit (its CUDA library is enumerated by preload_all_kernels).
const void* tc_kernel_anchor() { return (const void*)tc_split_kernel; }

}  // namespace rte

using namespace rte;

// Tall-skinny projection on the tensor cores (split TF32, FP32 accumulation) of the handle's DOF
// length: out[v r + k] = sum_i X[k N_x + i] Psi[v N_x + i] (see rte.h).
extern "C" int rte_basis_project(rte_handle* h, const float* X, int r, const float* Psi, int nv, double* out) {
    if (!h || r < 0 || nv < 0 || (r > 0 && nv > 0 && (!X || !Psi || !out)))
        return fail(RTE_ERR_ARG, "rte_basis_project: null argument or negative size");
    if (r == 0 || nv == 0) return RTE_OK;
    if (nv > 8) return fail(RTE_ERR_ARG, "rte_basis_project: at most 8 vectors per call");
    const int N = h->ndof;
    const int rows = 256, nblk = (N + rows - 1) / rows;
    const size_t part_bytes = sizeof(double) * (size_t)nblk * 8 * r;
    const size_t xb = ((sizeof(float) * (size_t)r * N + 255) / 256) * 256;
    const size_t vb = ((sizeof(float) * (size_t)nv * N + 255) / 256) * 256;
    RTE_TRY(h->arena.grow(&h->tc_scratch, &h->tc_scratch_cap, part_bytes + 2 * xb + 2 * vb + 256));
    char* base = static_cast<char*>(h->tc_scratch);
    double* part = reinterpret_cast<double*>(base);
    float* xt = reinterpret_cast<float*>(base + part_bytes);
    float* xl = reinterpret_cast<float*>(base + part_bytes + xb);
    float* vt = reinterpret_cast<float*>(base + part_bytes + 2 * xb);
    float* vl = reinterpret_cast<float*>(base + part_bytes + 2 * xb + vb);
    int* st = reinterpret_cast<int*>(base + part_bytes + 2 * xb + 2 * vb);
    RTE_TRY(tc_split(X, (long long)r * N, xt, xl, h->stream));
    RTE_TRY(tc_split(Psi, (long long)nv * N, vt, vl, h->stream));
    TcProjection P;
    RTE_TRY(tc_projection_prepare(&P, xt, xl, N, r, vt, vl, nv));
    tc_set_state<<<1, 1, 0, h->stream>>>(st, r);
    RTE_TRY(tc_projection_launch(&P, 0, nv, rows, nblk, st, st + 1, part, 8, nullptr, nullptr, h->d_err, h->stream));
    tc_reduce<<<(r * nv + 255) / 256, 256, 0, h->stream>>>(part, nblk, 8, r, r, nv, out);
    RTE_CUDA_TRY(cudaGetLastError());
    return check_dep_flag(h, h->stream);
}
