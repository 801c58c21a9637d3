// Reverse mode of the likelihood tail (Sect. 2.7, 2.8.4): ISM attenuation,
// response contraction and Poisson log-likelihood, and the final per-instance
// gradient.
//
//   H[row][c]    = dlogL/dC = tau (d / lambda - 1)          (lambda = tau C + bkg)
//   G[row][k]    = sum_c H[row][c] R[k][c]                   (= dlogL/d(F_t ATT))
//   dlogL/dF_t   = ATT_k G[row][k]
//   Aadj[row][k] = ATT_k G[row][k] / (E_k flux scale)        (adjoint of sum F_p I)
//   per row:       sum_k F_t ATT G            -> D:   F_t scales as D^-2
//                  sum_k F_t ATT sigma_k G    -> N_H: ATT = exp(-N_H sigma)
//
// k_grad_resp: 32 rows x 64 energies per block (256 threads, 2 x 4 outputs
// each), K = channels staged through shared memory in steps of 32, H formed
// while staging.  Row sums are written per (row, energy tile) and added in a
// fixed order by k_grad_final.
#include "ppm_internal.cuh"

namespace ppm {
namespace {

constexpr int kTM = 32, kTN = kGradTN, kTK = 32, kThreads = 256;

__global__ void __launch_bounds__(kThreads)
    k_grad_resp(Params p, PlanDev plan, const float *__restrict__ Ft, int total_rows, int nE,
                int nEpad, const float *__restrict__ invE, const float *__restrict__ R,
                const float *__restrict__ sigma, int nc, const int *__restrict__ counts,
                int shared_counts, const float *__restrict__ bkg, double tau,
                const float *__restrict__ lambda, const int *__restrict__ status,
                float *__restrict__ Aadj, double *__restrict__ row_sums)
{
    __shared__ float Hs[kTK][kTM + 1];
    __shared__ float Rs[kTK][kTN + 1];
    __shared__ double red[kTM][16][2];
    __shared__ int rc[kTM], rok[kTM];
    __shared__ float nh[kTM];
    const int row0 = blockIdx.y * kTM, k0 = blockIdx.x * kTN;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads, 2 rows x 4 k each
    if (threadIdx.x < kTM) {
        const int row = row0 + threadIdx.x;
        int b = 0, crow = 0, ok = 0;
        if (row < total_rows) {
            b = find_instance_by_row(plan.inst, plan.B, row);
            crow = shared_counts ? row - plan.inst[b].row0 : row;
            ok = status[b] == 0;
        }
        rc[threadIdx.x] = crow;
        rok[threadIdx.x] = ok;
        nh[threadIdx.x] = ok ? (float)(p.nh_1e20[b] * 1e20) : 0.0f;
    }
    __syncthreads();
    const float ftau = (float)tau;
    float acc[2][4] = {};
    for (int c0 = 0; c0 < nc; c0 += kTK) {
        for (int i = threadIdx.x; i < kTM * kTK; i += kThreads) {
            const int rr = i / kTK, cc = i - rr * kTK;
            const int row = row0 + rr, c = c0 + cc;
            float h = 0.0f;
            if (row < total_rows && c < nc && rok[rr]) {
                const float lam = lambda[(size_t)row * nc + c];
                const int d = counts[(size_t)rc[rr] * nc + c];
                // lambda = 0 with d = 0 contributes -lambda only; with d > 0 the
                // instance has logL = -inf and its gradient is not defined
                if (lam > 0.0f) h = ftau * ((float)d / lam - 1.0f);
                else h = d == 0 ? -ftau : 0.0f;
            }
            Hs[cc][rr] = h;
        }
        for (int i = threadIdx.x; i < kTK * kTN; i += kThreads) {
            const int kk = i / kTK, cc = i - kk * kTK;  // c fastest: coalesced rows of R
            const int k = k0 + kk, c = c0 + cc;
            Rs[cc][kk] = (k < nE && c < nc) ? R[(size_t)k * nc + c] : 0.0f;
        }
        __syncthreads();
#pragma unroll 8
        for (int cc = 0; cc < kTK; ++cc) {
            const float h0 = Hs[cc][ty * 2], h1 = Hs[cc][ty * 2 + 1];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float r = Rs[cc][tx * 4 + j];
                acc[0][j] = fmaf(h0, r, acc[0][j]);
                acc[1][j] = fmaf(h1, r, acc[1][j]);
            }
        }
        __syncthreads();
    }
    const float sc = (float)(1.0 / kFluxScale);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int rr = ty * 2 + i, row = row0 + rr;
        double sD = 0.0, sN = 0.0;
        if (row < total_rows) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int k = k0 + tx * 4 + j;
                if (k >= nEpad) continue;
                float a = 0.0f;
                if (k < nE && rok[rr]) {
                    const float att = expf(-nh[rr] * sigma[k]);
                    const float g = att * acc[i][j];
                    a = g * invE[k] * sc;
                    const double fg = (double)Ft[(size_t)row * nE + k] * (double)g;
                    sD += fg;
                    sN += fg * (double)sigma[k];
                }
                Aadj[(size_t)row * nEpad + k] = a;
            }
        }
        red[rr][tx][0] = sD;
        red[rr][tx][1] = sN;
    }
    __syncthreads();
    if (threadIdx.x < kTM) {
        const int row = row0 + threadIdx.x;
        double a = 0.0, c = 0.0;
        for (int j = 0; j < 16; ++j) {
            a += red[threadIdx.x][j][0];
            c += red[threadIdx.x][j][1];
        }
        if (row < total_rows) {
            double *o = row_sums + ((size_t)row * gridDim.x + blockIdx.x) * 2;
            o[0] = a;
            o[1] = c;
        }
    }
}

// grad[b] = sum over the instance's rings of the ring contributions, plus the
// closed-form D and N_H terms.  NaN where the instance has no finite logL.
__global__ void k_grad_final(Params p, PlanDev plan, const double *__restrict__ ring_grad,
                             const double *__restrict__ row_sums, int ktiles,
                             const int *__restrict__ status, const double *__restrict__ logL,
                             double *__restrict__ grad)
{
    const int b = blockIdx.x;
    const InstPlan ip = plan.inst[b];
    __shared__ double red[8][kNGrad];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double g[kNGrad];
#pragma unroll
    for (int q = 0; q < kNGrad; ++q) g[q] = 0.0;
    const int n_rings = p.n_spots * ip.n_theta;
    for (int i = threadIdx.x; i < n_rings; i += blockDim.x) {
        const double *rg = ring_grad + (size_t)(ip.ring0 + i) * kRingGrad;
        const int s = i / ip.n_theta;
        g[0] += rg[0];
        g[1] += rg[1];
        g[2] += rg[2];
#pragma unroll
        for (int q = 0; q < 2; ++q)
            if (q == s) {
                g[5 + 4 * q] += rg[3];
                g[6 + 4 * q] += rg[4];
                g[7 + 4 * q] += rg[5];
                g[8 + 4 * q] += rg[6];
            }
    }
    const int nr = ip.n_phase * ktiles;
    for (int i = threadIdx.x; i < nr; i += blockDim.x) {
        const double *rs = row_sums + ((size_t)ip.row0 * ktiles + i) * 2;
        g[3] += rs[0];
        g[4] += rs[1];
    }
#pragma unroll
    for (int q = 0; q < kNGrad; ++q) {
        double v = g[q];
        for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < kNGrad) {
        const int q = threadIdx.x;
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w][q];
        if (q == 3) v *= -2.0 / p.dist_kpc[b];
        if (q == 4) v *= -1e20;
        const bool ok = status[b] == 0 && logL[b] > -INFINITY;
        grad[(size_t)b * kNGrad + q] = ok ? v : NAN;
    }
}

}  // namespace

int grad_ktiles(int nEpad) { return (nEpad + kTN - 1) / kTN; }

cudaError_t launch_grad_resp(const Params &p, const PlanDev &plan, const float *Ft,
                             int total_rows, const EnergyDev &en, const float *R,
                             const float *sigma, int nc, const int *counts, int counts_shared,
                             const float *bkg, double tau, const float *lambda,
                             const int *status, float *Aadj, double *row_sums, cudaStream_t st)
{
    if (total_rows <= 0) return cudaSuccess;
    (void)bkg;  // enters through lambda
    dim3 grid(grad_ktiles(en.nEpad), (total_rows + kTM - 1) / kTM);
    k_grad_resp<<<grid, kThreads, 0, st>>>(p, plan, Ft, total_rows, en.nE, en.nEpad, en.invE, R,
                                           sigma, nc, counts, counts_shared, bkg, tau, lambda,
                                           status, Aadj, row_sums);
    return cudaGetLastError();
}

cudaError_t launch_grad_final(const Params &p, const PlanDev &plan, const double *ring_grad,
                              const double *row_sums, int ktiles, const int *status,
                              const double *logL, double *grad, cudaStream_t st)
{
    k_grad_final<<<plan.B, 256, 0, st>>>(p, plan, ring_grad, row_sums, ktiles, status, logL,
                                         grad);
    return cudaGetLastError();
}

}  // namespace ppm
