// ISM attenuation, response contraction and Poisson log-likelihood
// (Sect. 2.7, 2.8.4; likelihood accumulated on the GPU as in Sect. 6).
//
//   C[row][c] = sum_k F_t[row][k] ATT_b[k] R[k][c],  ATT_b[k] = exp(-N_H,b sigma_k)
//   lambda    = tau C + bkg
//   logL[b]   = sum_{rows of b, c} d ln(lambda) - lambda - ln Gamma(d + 1)
//
// k_resp_ll: 16 x 32 output tile per block; four groups of 128 threads (2 x 2
// outputs each) take every fourth K step of 32 energies (staged through
// shared memory), their partial tiles are added in group order, and the
// first group evaluates the likelihood terms (ln lambda in FP32, sums in
// FP64) and writes one partial sum per (row, column tile).
// k_ll_final adds the partials of each instance in a fixed order.
#include "ppm_internal.cuh"

namespace ppm {
namespace {

constexpr int kTM = 16, kTN = 32, kTK = 32, kGroup = 128, kSplitK = 4, kThreads = kGroup * kSplitK;

// ln Gamma(d + 1) = ln d!: table below kLogFactN (built on the host in FP64),
// Stirling series above it (relative error < 1e-16 for d >= 4096).
__device__ __forceinline__ double log_factorial(int d, const double *__restrict__ tab)
{
    if (d < kLogFactN) return tab[d];
    const double n = (double)d, r = 1.0 / n, r2 = r * r;
    return n * log(n) - n + 0.5 * log(2.0 * kPI * n) +
           r * (1.0 / 12.0 - r2 * (1.0 / 360.0 - r2 * (1.0 / 1260.0)));
}

__global__ void __launch_bounds__(kThreads) k_resp_ll(Params p, PlanDev plan,
                                                const float *__restrict__ Ft, int total_rows,
                                                int nE, const float *__restrict__ R,
                                                const float *__restrict__ sigma, int nc,
                                                const int *__restrict__ counts, int shared_counts,
                                                const float *__restrict__ bkg, double tau,
                                                const int *__restrict__ status,
                                                const double *__restrict__ lfact,
                                                double *__restrict__ row_ll,
                                                float *__restrict__ model_counts)
{
    __shared__ float As[kSplitK][kTK][kTM + 1];
    __shared__ float Bs[kSplitK][kTK][kTN + 1];
    __shared__ float part[kSplitK - 1][kTM][kTN];  // partial tiles of groups 1..3
    __shared__ double red[kTM][17];  // [row][column-pair]
    __shared__ float att_nh[kTM];
    const int row0 = blockIdx.y * kTM, col0 = blockIdx.x * kTN;
    const int grp = threadIdx.x / kGroup, lt = threadIdx.x % kGroup;
    const int tx = lt & 15, ty = lt >> 4;   // 2 x 2 outputs per thread (8 x 16 threads)
    if (threadIdx.x < kTM) {
        const int row = row0 + threadIdx.x;
        att_nh[threadIdx.x] =
            row < total_rows ? (float)(p.nh_1e20[find_instance_by_row(plan.inst, plan.B, row)] * 1e20)
                             : 0.0f;
    }
    __syncthreads();
    float acc[2][2] = {};
    // every group runs the same number of steps (the barriers); steps past
    // nE stage zeros
    const int steps = (nE + kSplitK * kTK - 1) / (kSplitK * kTK);
    for (int st = 0; st < steps; ++st) {
        const int k0 = (st * kSplitK + grp) * kTK;
        for (int i = lt; i < kTM * kTK; i += kGroup) {
            const int rr = i / kTK, kk = i - rr * kTK;
            const int row = row0 + rr, k = k0 + kk;
            As[grp][kk][rr] = (row < total_rows && k < nE)
                                  ? Ft[(size_t)row * nE + k] * expf(-att_nh[rr] * sigma[k])
                                  : 0.0f;
        }
        for (int i = lt; i < kTK * kTN; i += kGroup) {
            const int kk = i / kTN, cc = i - kk * kTN;
            const int k = k0 + kk, c = col0 + cc;
            Bs[grp][kk][cc] = (k < nE && c < nc) ? R[(size_t)k * nc + c] : 0.0f;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < kTK; ++kk) {
            const float a0 = As[grp][kk][ty * 2], a1 = As[grp][kk][ty * 2 + 1];
            const float b0 = Bs[grp][kk][tx * 2], b1 = Bs[grp][kk][tx * 2 + 1];
            acc[0][0] = fmaf(a0, b0, acc[0][0]);
            acc[0][1] = fmaf(a0, b1, acc[0][1]);
            acc[1][0] = fmaf(a1, b0, acc[1][0]);
            acc[1][1] = fmaf(a1, b1, acc[1][1]);
        }
        __syncthreads();
    }
    // partial tiles of groups 1..3 added to group 0's in group order
    if (grp > 0) {
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) part[grp - 1][ty * 2 + i][tx * 2 + j] = acc[i][j];
    }
    __syncthreads();
    if (grp > 0) return;
#pragma unroll
    for (int q = 0; q < kSplitK - 1; ++q)
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) acc[i][j] += part[q][ty * 2 + i][tx * 2 + j];
    // epilogue (first group): likelihood terms in FP64
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int rr = ty * 2 + i, row = row0 + rr;
        double s = 0.0;
        if (row < total_rows) {
            const int b = find_instance_by_row(plan.inst, plan.B, row);
            const int crow = shared_counts ? row - plan.inst[b].row0 : row;
            const bool ok = status[b] == 0;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int c = col0 + tx * 2 + j;
                if (c >= nc) continue;
                const size_t di = (size_t)crow * nc + c;
                const double lam = tau * (double)acc[i][j] + (bkg ? (double)bkg[di] : 0.0);
                const int d = counts[di];
                if (model_counts) model_counts[(size_t)row * nc + c] = (float)lam;
                if (!ok) continue;
                if (lam <= 0.0) {
                    if (d > 0) s += -INFINITY;
                } else {
                    // lambda carries the FP32 rounding of C; ln(lambda) in FP32 adds less
                    const double ll = d > 0 ? (double)d * (double)logf((float)lam) : 0.0;
                    s += ll - lam - log_factorial(d, lfact);
                }
            }
        }
        red[rr][tx] = s;
    }
    // barrier over the first group only (the others have returned)
    asm volatile("bar.sync 1, %0;" ::"r"(kGroup));
    if (threadIdx.x < kTM) {
        const int row = row0 + threadIdx.x;
        double s = 0.0;
        for (int j = 0; j < 16; ++j) s += red[threadIdx.x][j];
        if (row < total_rows) row_ll[(size_t)row * gridDim.x + blockIdx.x] = s;
    }
}

__global__ void k_ll_final(PlanDev plan, const double *__restrict__ row_ll, int n_ctiles,
                           const int *__restrict__ status, double *__restrict__ logL)
{
    const int b = blockIdx.x;
    const InstPlan ip = plan.inst[b];
    __shared__ double red[256];
    double s = 0.0;
    const int n = ip.n_phase * n_ctiles;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += row_ll[(size_t)ip.row0 * n_ctiles + i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) logL[b] = (status[b] == 0) ? red[0] : -INFINITY;
}

}  // namespace

int loglike_ctiles(int nc) { return (nc + kTN - 1) / kTN; }

void launch_ll_final(const PlanDev &plan, const double *row_ll, int n_ctiles, const int *status,
                     double *logL, cudaStream_t st)
{
    k_ll_final<<<plan.B, 256, 0, st>>>(plan, row_ll, n_ctiles, status, logL);
}

cudaError_t launch_loglike(const Params &p, const PlanDev &plan, const float *Ft, int total_rows,
                           int nE, const float *R, const float *sigma, int nc,
                           const int *counts, int counts_shared, const float *bkg, double tau,
                           const int *status, const double *lfact, double *row_ll,
                           float *model_counts, double *logL, cudaStream_t st)
{
    const int ct = loglike_ctiles(nc);
    dim3 grid(ct, (total_rows + kTM - 1) / kTM);
    k_resp_ll<<<grid, kThreads, 0, st>>>(p, plan, Ft, total_rows, nE, R, sigma, nc, counts,
                                    counts_shared, bkg, tau, status, lfact, row_ll, model_counts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_ll_final<<<plan.B, 256, 0, st>>>(plan, row_ll, ct, status, logL);
    return cudaGetLastError();
}

}  // namespace ppm
