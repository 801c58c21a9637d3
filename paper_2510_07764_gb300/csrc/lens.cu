// FP64 light-bending and time-delay tables on the GPU (Sect. 2.3, 2.8.2).
//
// One block per compactness row u: the threads evaluate the bending angle at
// every alpha step of the march in parallel (Eq. salmi_lf, inward rays via the
// periastron of Eq. rho), the block finds where the sequential march would
// stop, differentiates cos(alpha) with respect to cos(psi) by central
// differences along the march and resamples both onto the cos(psi) grid.
// The delay table (Eq. salmi_td, inward composition of Eq. tot_time_delay)
// is evaluated pointwise on the (u, cos alpha) grid.
//
// Quadrature: the integrands of Eqs. salmi_lf / salmi_td vary on the scale
// x ~ |cos alpha| (grazing rays) and x ~ sqrt(q(0)) (periastron near the photon
// sphere), both at the lower end, so [0, 1] is split into panels
// [2^-k-1, 2^-k] (k = 0..24) plus [0, 2^-25], each integrated with 16-point
// Gauss-Legendre (8 points per panel lose ~1e-10 when the periastron of an
// inward ray approaches the photon sphere).
#include "ppm_internal.cuh"

namespace ppm {
namespace {

__constant__ double kGLx[8] = {0.095012509837637441, 0.28160355077925892, 0.45801677765722737, 0.61787624440264377, 0.755404408355003, 0.86563120238783176, 0.9445750230732326, 0.98940093499164994};
__constant__ double kGLw[8] = {0.18945061045506864, 0.18260341504492364, 0.16915651939500265, 0.14959598881657671, 0.12462897125553407, 0.095158511682492605, 0.062253523938647456, 0.027152459411754176};

// kind 0: bending integrand x / sqrt(c^2 + x^2 q); kind 1: delay integrand
// x / (w (1 + w)), w = sqrt(c^2 + x^2 q), q = [2 - x^2 - u(1-x^2)^2/(1-u)] s^2.
__device__ double bend_integral(int kind, double u, double c2, double s2)
{
    const int kPanels = 25;
    double sum = 0.0;
    double a = 0.0, b = ldexp(1.0, -kPanels);
    const double ku = u / (1.0 - u);
    for (int p = 0; p <= kPanels; ++p) {
        double h = 0.5 * (b - a), m = 0.5 * (a + b), s = 0.0;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            double x = (i < 8) ? m - h * kGLx[i] : m + h * kGLx[i - 8];
            double wgt = kGLw[i & 7];
            double y = 1.0 - x * x;
            double q = (2.0 - x * x - ku * y * y) * s2;
            double w = sqrt(c2 + x * x * q);
            s += wgt * ((kind == 0) ? x / w : x / (w * (1.0 + w)));
        }
        sum += h * s;
        a = b;
        b *= 2.0;
    }
    return sum;
}

__device__ double psi_out(double u, double alpha)
{
    double s, c;
    sincos(alpha, &s, &c);
    if (s == 0.0) return 0.0;
    return 2.0 * s / sqrt(1.0 - u) * bend_integral(0, u, c * c, s * s);
}

__device__ double td_out(double u, double alpha)
{
    double s, c;
    sincos(alpha, &s, &c);
    if (s == 0.0) return 0.0;
    return 2.0 * s * s / (1.0 - u) * bend_integral(1, u, c * c, s * s);
}

// periastron ratio (Eq. rho); NaN when the ray is captured
__device__ double periastron(double u, double alpha)
{
    double s = sin(alpha);
    double k = sqrt(3.0 * (1.0 - u));
    double arg = 3.0 * u * k / (2.0 * s);
    if (!(arg <= 1.0)) return nan("");
    return -2.0 * s / k * cos((acos(arg) + 2.0 * kPI) / 3.0);
}

__device__ double psi_any(double u, double alpha)
{
    if (alpha <= 0.5 * kPI) return psi_out(u, alpha);
    double r = periastron(u, alpha);
    if (isnan(r)) return r;
    return 2.0 * psi_out(u / r, 0.5 * kPI) - psi_out(u, kPI - alpha);
}

// c Delta t / R; inward rays: periastron leg in units of R_p = rho R plus the
// radial-delay difference 2[(1 - rho) + u ln((1 - u)/(rho - u))]
__device__ double td_any(double u, double alpha)
{
    if (alpha <= 0.5 * kPI) return td_out(u, alpha);
    double r = periastron(u, alpha);
    if (isnan(r)) return r;
    return 2.0 * r * td_out(u / r, 0.5 * kPI) - td_out(u, kPI - alpha) +
           2.0 * ((1.0 - r) + u * log((1.0 - u) / (r - u)));
}

__device__ __forceinline__ double lin_at(double lo, double hi, int n, int i)
{
    return lo + (hi - lo) * (double)i / (double)(n - 1);
}

__global__ void __launch_bounds__(256) k_lens_march(LensDev L, double dalpha, double *psi_buf,
                                                   double *lists, int j_cap)
{
    const int iu = blockIdx.x;
    const double u = lin_at(L.u_min, L.u_max, L.n_u, iu);
    const double psi_stop = acos(L.cpsi_min);
    double *row = psi_buf + (size_t)iu * j_cap;
    double *cps = lists + (size_t)iu * j_cap * 3;
    double *cal = cps + j_cap;
    double *ld = cal + j_cap;
    __shared__ int s_bad, s_over;
    if (threadIdx.x == 0) { s_bad = j_cap; s_over = j_cap; }
    __syncthreads();
    for (int j = threadIdx.x; j < j_cap; j += blockDim.x) {
        double alpha = j * dalpha;
        double psi = (alpha > kPI) ? nan("") : psi_any(u, alpha);
        row[j] = psi;
        if (isnan(psi) || psi > kPI) atomicMin(&s_bad, j);
        else if (psi > psi_stop) atomicMin(&s_over, j);
    }
    __syncthreads();
    const int n = min(s_bad, s_over == j_cap ? j_cap : s_over + 1);
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        cps[j] = cos(row[j]);
        cal[j] = cos(j * dalpha);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        int a = j > 0 ? j - 1 : j, b = j < n - 1 ? j + 1 : j;
        ld[j] = (b > a) ? (cal[b] - cal[a]) / (cps[b] - cps[a]) : nan("");
    }
    __syncthreads();
    double *Ca = const_cast<double *>(L.Ca) + (size_t)iu * L.n_cpsi;
    double *LF = const_cast<double *>(L.LF) + (size_t)iu * L.n_cpsi;
    for (int ic = threadIdx.x; ic < L.n_cpsi; ic += blockDim.x) {
        double cp = lin_at(L.cpsi_min, L.cpsi_max, L.n_cpsi, ic);
        if (n < 2 || cp < cps[n - 1]) {
            Ca[ic] = nan("");
            LF[ic] = nan("");
            continue;
        }
        int lo = 0, hi = n - 1;  // cps decreasing
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (cps[mid] >= cp) lo = mid; else hi = mid;
        }
        double w = (cp - cps[lo]) / (cps[hi] - cps[lo]);
        Ca[ic] = cal[lo] + w * (cal[hi] - cal[lo]);
        LF[ic] = ld[lo] + w * (ld[hi] - ld[lo]);
    }
}

__global__ void __launch_bounds__(256) k_lens_td(LensDev L)
{
    const int total = L.n_u * L.n_calpha;
    double *TD = const_cast<double *>(L.TD);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        int iu = t / L.n_calpha, ia = t % L.n_calpha;
        double u = lin_at(L.u_min, L.u_max, L.n_u, iu);
        double ca = lin_at(L.ca_min, L.ca_max, L.n_calpha, ia);
        TD[t] = td_any(u, acos(ca));
    }
}

}  // namespace

cudaError_t launch_lens_build(const LensDev &L, double dalpha, double *psi_scratch,
                              double *list_scratch, int j_cap, cudaStream_t st)
{
    k_lens_march<<<L.n_u, 256, 0, st>>>(L, dalpha, psi_scratch, list_scratch, j_cap);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int total = L.n_u * L.n_calpha;
    int blocks = (total + 255) / 256;
    k_lens_td<<<blocks, 256, 0, st>>>(L);
    return cudaGetLastError();
}

}  // namespace ppm
