// Response contraction on the 5th-generation tensor cores (tcgen05) with the
// Poisson likelihood epilogue (Sect. 2.7, 2.8.4; likelihood as in loglike.cu).
//
//   C[row][c] = sum_k (F_t[row][k] ATT_b[k]) R[k][c]
//
// One CTA (128 threads) computes a 128-row x 160-channel tile of C in a TMEM
// accumulator.  Operands are split into BF16 hi + lo parts (a = a_hi + a_lo,
// |a_lo| <= 2^-9 |a|); three MMAs per K step (hi*hi + hi*lo + lo*hi) keep the
// product accurate to ~2^-16 relative, with FP32 accumulation.  A (F_t x ATT)
// is converted and stored by the threads; B (R, pre-split and pre-laid-out
// per tile at ppm_set_response) is copied.  Both live in shared memory in the
// K-major, non-swizzled core-matrix layout (8 rows x 16 bytes per core matrix;
// core matrices 128 B apart along K, KC/8 * 128 B apart along M/N).  Thread 0
// issues the MMAs and commits them to an mbarrier; every wait is bounded and
// a timeout sets an error bit instead of hanging.  The epilogue reads the
// accumulator with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = rows) and
// evaluates the likelihood terms.
#include <cuda_bf16.h>

#include "ppm_internal.cuh"

namespace ppm {
namespace {

constexpr int kTcM = 128;      // rows per CTA (MMA M)
constexpr int kTcN = 160;      // channels per CTA (MMA N: multiple of 16, <= 256)
constexpr int kTcKC = 128;     // K chunk staged in shared memory
constexpr int kTcThreads = 128;
constexpr uint32_t kTmemCols = 256;
constexpr long long kWaitCycles = 4000000000ll;   // ~2 s at the maximum SM clock

// instruction descriptor: D = F32, A = B = BF16, both K-major, N = 160, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                            ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor, no swizzle: LBO = core-matrix stride along
// K, SBO = stride between 8-row groups along M/N (bytes, encoded >> 4)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
           ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        :
        : "r"(d_tmem), "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > kWaitCycles) return false;
    }
}

// ln d! (table, Stirling series beyond it), as in loglike.cu
__device__ __forceinline__ double log_fact(int d, const double *__restrict__ tab)
{
    if (d < kLogFactN) return tab[d];
    const double n = (double)d, r = 1.0 / n, r2 = r * r;
    return n * log(n) - n + 0.5 * log(2.0 * kPI * n) +
           r * (1.0 / 12.0 - r2 * (1.0 / 360.0 - r2 * (1.0 / 1260.0)));
}

__global__ void __launch_bounds__(kTcThreads, 1)
    k_resp_ll_tc(Params p, PlanDev plan, const float *__restrict__ Ft, int total_rows, int nE,
                 const uint4 *__restrict__ Rtc, int n_kc, const float *__restrict__ sigma, int nc,
                 const int *__restrict__ counts, int shared_counts, const float *__restrict__ bkg,
                 double tau, const int *__restrict__ status, const double *__restrict__ lfact,
                 double *__restrict__ row_ll, float *__restrict__ model_counts,
                 unsigned *__restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    // [A_hi | A_lo] (128 x KC bf16 each) [B_hi | B_lo] (160 x KC bf16 each)
    constexpr uint32_t kA = kTcM * kTcKC * 2, kB = kTcN * kTcKC * 2;
    unsigned char *sA = smem, *sB = smem + 2 * kA;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ float att_nh[kTcM];
    __shared__ int s_fail;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row0 = blockIdx.y * kTcM, col0 = blockIdx.x * kTcN;
    const uint32_t bar_a = smem_u32(&bar);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_base)), "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar_a));
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_fail = 0;
    }
    {
        const int row = row0 + tid;
        att_nh[tid] = row < total_rows
                          ? (float)(p.nh_1e20[find_instance_by_row(plan.inst, plan.B, row)] * 1e20)
                          : 0.0f;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;

    uint32_t parity = 0;
    for (int kc = 0; kc < n_kc; ++kc) {
        const int k0 = kc * kTcKC;
        // A: thread handles (row r, 8 consecutive k): FP32 x ATT -> bf16 hi / lo,
        // one 16-byte row of a core matrix each
        for (int idx = tid; idx < kTcM * (kTcKC / 8); idx += kTcThreads) {
            const int r = idx % kTcM, kb = idx / kTcM;
            const int row = row0 + r;
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float v[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = k0 + kb * 8 + 2 * q + h;
                    v[h] = (row < total_rows && k < nE)
                               ? Ft[(size_t)row * nE + k] * expf(-att_nh[r] * sigma[k])
                               : 0.0f;
                }
                const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[0], v[1]);
                const float2 hf = __bfloat1622float2(h2);
                const __nv_bfloat162 l2 = __floats2bfloat162_rn(v[0] - hf.x, v[1] - hf.y);
                hi[q] = *reinterpret_cast<const uint32_t *>(&h2);
                lo[q] = *reinterpret_cast<const uint32_t *>(&l2);
            }
            const uint32_t off = ((r >> 3) * (kTcKC / 8) + kb) * 128 + (r & 7) * 16;
            *reinterpret_cast<uint4 *>(sA + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4 *>(sA + kA + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
        // B: pre-laid-out hi and lo tiles of (column tile, K chunk)
        {
            const uint4 *src = Rtc + ((size_t)blockIdx.x * n_kc + kc) * (2 * kB / 16);
            uint4 *dst = reinterpret_cast<uint4 *>(sB);
            for (int i = tid; i < (int)(2 * kB / 16); i += kTcThreads) dst[i] = src[i];
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
            const uint32_t a_hi = smem_u32(sA), a_lo = a_hi + kA;
            const uint32_t b_hi = smem_u32(sB), b_lo = b_hi + kB;
            const uint32_t lbo = 128, sbo = (kTcKC / 8) * 128;
#pragma unroll 1
            for (int s = 0; s < kTcKC / 16; ++s) {
                const uint32_t o = (uint32_t)s * 256;
                const uint32_t first = (kc == 0 && s == 0) ? 0u : 1u;
                mma_bf16(tmem, smem_desc(a_hi + o, lbo, sbo), smem_desc(b_hi + o, lbo, sbo), first);
                mma_bf16(tmem, smem_desc(a_hi + o, lbo, sbo), smem_desc(b_lo + o, lbo, sbo), 1u);
                mma_bf16(tmem, smem_desc(a_lo + o, lbo, sbo), smem_desc(b_hi + o, lbo, sbo), 1u);
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                :: "r"(bar_a) : "memory");
        }
        if (!mbar_wait(bar_a, parity)) atomicOr(&s_fail, 1);
        parity ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        __syncthreads();
        if (s_fail) break;
    }

    // epilogue: warp w reads TMEM lanes 32w..32w+31 (rows), 32 columns at a time
    double s = 0.0;
    const int r = warp * 32 + lane, row = row0 + r;
    if (!s_fail) {
        int b = 0, crow = row;
        bool ok = false;
        if (row < total_rows) {
            b = find_instance_by_row(plan.inst, plan.B, row);
            crow = shared_counts ? row - plan.inst[b].row0 : row;
            ok = status[b] == 0;
        }
        for (int c0 = 0; c0 < kTcN; c0 += 32) {
            uint32_t v[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
                "%10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, "
                "%26, %27, %28, %29, %30, %31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                  "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                  "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]),
                  "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                  "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
                  "=r"(v[30]), "=r"(v[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < total_rows) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int c = col0 + c0 + j;
                    if (c >= nc) continue;
                    const size_t di = (size_t)crow * nc + c;
                    const double lam =
                        tau * (double)__uint_as_float(v[j]) + (bkg ? (double)bkg[di] : 0.0);
                    if (model_counts) model_counts[(size_t)row * nc + c] = (float)lam;
                    if (!ok) continue;
                    const int d = counts[di];
                    if (lam <= 0.0) {
                        if (d > 0) s += -INFINITY;
                    } else {
                        const double ll = d > 0 ? (double)d * (double)logf((float)lam) : 0.0;
                        s += ll - lam - log_fact(d, lfact);
                    }
                }
            }
        }
    } else if (tid == 0) {
        atomicOr(err, kErrTimeout);
    }
    if (row < total_rows) row_ll[(size_t)row * gridDim.x + blockIdx.x] = s_fail ? 0.0 : s;
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem),
                     "r"(kTmemCols));
}

}  // namespace

int resp_tc_ctiles(int nc) { return (nc + kTcN - 1) / kTcN; }
int resp_tc_kchunks(int nE) { return (nE + kTcKC - 1) / kTcKC; }

// Host-side layout of R for the tensor-core path: for every (column tile,
// K chunk) a block [hi tile | lo tile], each 160 x KC bf16 in the core-matrix
// order of the kernel's shared memory (zero beyond nc / nE).
void resp_tc_layout(const float *R, int nE, int nc, uint16_t *out)
{
    const int nct = resp_tc_ctiles(nc), nkc = resp_tc_kchunks(nE);
    const size_t tile = (size_t)kTcN * kTcKC;
    for (int ct = 0; ct < nct; ++ct)
        for (int kc = 0; kc < nkc; ++kc) {
            uint16_t *hi = out + ((size_t)ct * nkc + kc) * 2 * tile, *lo = hi + tile;
            for (int n = 0; n < kTcN; ++n)
                for (int kk = 0; kk < kTcKC; ++kk) {
                    const int c = ct * kTcN + n, k = kc * kTcKC + kk;
                    const float v = (c < nc && k < nE) ? R[(size_t)k * nc + c] : 0.0f;
                    const __nv_bfloat16 h = __float2bfloat16_rn(v);
                    const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
                    const size_t off = ((size_t)(n >> 3) * (kTcKC / 8) + (kk >> 3)) * 64 +
                                       (n & 7) * 8 + (kk & 7);
                    hi[off] = *reinterpret_cast<const uint16_t *>(&h);
                    lo[off] = *reinterpret_cast<const uint16_t *>(&l);
                }
        }
}

size_t resp_tc_layout_elems(int nE, int nc)
{
    return (size_t)resp_tc_ctiles(nc) * resp_tc_kchunks(nE) * 2 * kTcN * kTcKC;
}

cudaError_t launch_loglike_tc(const Params &p, const PlanDev &plan, const float *Ft,
                              int total_rows, int nE, const uint16_t *Rtc, const float *sigma,
                              int nc, const int *counts, int counts_shared, const float *bkg,
                              double tau, const int *status, const double *lfact,
                              double *row_ll, float *model_counts, unsigned *err, cudaStream_t st)
{
    const size_t smem = (size_t)2 * kTcM * kTcKC * 2 + (size_t)2 * kTcN * kTcKC * 2;
    cudaError_t e = cudaFuncSetAttribute(k_resp_ll_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(resp_tc_ctiles(nc), (total_rows + kTcM - 1) / kTcM);
    k_resp_ll_tc<<<grid, kTcThreads, smem, st>>>(p, plan, Ft, total_rows, nE,
                                                 reinterpret_cast<const uint4 *>(Rtc),
                                                 resp_tc_kchunks(nE), sigma, nc, counts,
                                                 counts_shared, bkg, tau, status, lfact, row_ll,
                                                 model_counts, err);
    return cudaGetLastError();
}

}  // namespace ppm
