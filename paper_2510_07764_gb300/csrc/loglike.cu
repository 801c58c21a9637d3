// ISM attenuation, response contraction and Poisson log-likelihood
// (Sect. 2.7, 2.8.4; likelihood accumulated on the GPU as in Sect. 6).
//
//   C[row][c] = sum_k F_t[row][k] ATT_b[k] R[k][c],  ATT_b[k] = exp(-N_H,b sigma_k)
//   lambda    = tau C + bkg
//   logL[b]   = sum_{rows of b, c} d ln(lambda) - lambda - ln Gamma(d + 1)
//
// k_resp_ll: 64 x 64 output tile per block, K staged through shared memory
// in steps of 32, each thread 4 x 4 outputs; the epilogue evaluates the
// likelihood terms in FP64 and writes one partial sum per (row, column tile).
// k_ll_final adds the partials of each instance in a fixed order.
#include "ppm_internal.cuh"

namespace ppm {
namespace {

constexpr int kTM = 64, kTN = 64, kTK = 32;

__global__ void __launch_bounds__(256) k_resp_ll(Params p, PlanDev plan,
                                                const float *__restrict__ Ft, int total_rows,
                                                int nE, const float *__restrict__ R,
                                                const float *__restrict__ sigma, int nc,
                                                const int *__restrict__ counts, int shared_counts,
                                                const float *__restrict__ bkg, double tau,
                                                const int *__restrict__ status,
                                                double *__restrict__ row_ll,
                                                float *__restrict__ model_counts)
{
    __shared__ float As[kTK][kTM + 4];
    __shared__ float Bs[kTK][kTN + 4];
    __shared__ double red[kTM][17];
    const int row0 = blockIdx.y * kTM, col0 = blockIdx.x * kTN;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4] = {};
    // attenuation depends on the instance of each row
    for (int k0 = 0; k0 < nE; k0 += kTK) {
        for (int i = threadIdx.x; i < kTM * kTK; i += 256) {
            const int rr = i / kTK, kk = i - rr * kTK;
            const int row = row0 + rr, k = k0 + kk;
            float v = 0.0f;
            if (row < total_rows && k < nE) {
                const int b = find_instance_by_row(plan.inst, plan.B, row);
                const float att = expf(-(float)(p.nh_1e20[b] * 1e20) * sigma[k]);
                v = Ft[(size_t)row * nE + k] * att;
            }
            As[kk][rr] = v;
        }
        for (int i = threadIdx.x; i < kTK * kTN; i += 256) {
            const int kk = i / kTN, cc = i - kk * kTN;
            const int k = k0 + kk, c = col0 + cc;
            Bs[kk][cc] = (k < nE && c < nc) ? R[(size_t)k * nc + c] : 0.0f;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < kTK; ++kk) {
            float a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
    // epilogue: likelihood terms in FP64
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int rr = ty * 4 + i, row = row0 + rr;
        double s = 0.0;
        if (row < total_rows) {
            const int b = find_instance_by_row(plan.inst, plan.B, row);
            const int crow = shared_counts ? row - plan.inst[b].row0 : row;
            const bool ok = status[b] == 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = col0 + tx * 4 + j;
                if (c >= nc) continue;
                const size_t di = (size_t)crow * nc + c;
                const double lam = tau * (double)acc[i][j] + (bkg ? (double)bkg[di] : 0.0);
                const int d = counts[di];
                if (model_counts) model_counts[(size_t)row * nc + c] = (float)lam;
                if (!ok) continue;
                if (lam <= 0.0) {
                    if (d > 0) s += -INFINITY;
                } else {
                    s += (double)d * log(lam) - lam - lgamma((double)d + 1.0);
                }
            }
        }
        red[rr][tx] = s;
    }
    __syncthreads();
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

cudaError_t launch_loglike(const Params &p, const PlanDev &plan, const float *Ft, int total_rows,
                           int nE, const float *R, const float *sigma, int nc,
                           const int *counts, int counts_shared, const float *bkg, double tau,
                           const int *status, double *row_ll, float *model_counts,
                           double *logL, cudaStream_t st)
{
    const int ct = (nc + kTN - 1) / kTN;
    dim3 grid(ct, (total_rows + kTM - 1) / kTM);
    k_resp_ll<<<grid, 256, 0, st>>>(p, plan, Ft, total_rows, nE, R, sigma, nc, counts,
                                    counts_shared, bkg, tau, status, row_ll, model_counts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_ll_final<<<plan.B, 256, 0, st>>>(plan, row_ll, ct, status, logL);
    return cudaGetLastError();
}

}  // namespace ppm
