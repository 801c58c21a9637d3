// Template tangents, FP64 forward mode (derivative of Sect. 2.1-2.6, 2.8.3 with
// respect to M, R_e, inclination, spot colatitude and spot angular radius).
//
// The backward pass does not store the forward geometry: one block per ring
// recomputes the ring set-up and every fine-phase template point with dual
// numbers carrying five tangents, and contracts them with the template
// adjoints written by the backward shift-and-add:
//     dlogL/dtheta += sum_i gF_i dF_i + gZ_i dz_i + gMu_i dmu_i + gPh_i dphi_o,i
// The visibility pattern is taken from the forward template (F == 0 marks an
// invisible point), so both passes use the same piecewise branch.  Adjoints
// of the bridged invisible points are first folded onto their two end
// points, and that of point n_fp onto point 0 (the reverse of the fill).
// Ring-level terms: the element azimuths (spot azimuth and the ring's
// half-width), and the ring's logg and logT through the atmosphere stencil.
#include "ppm_internal.cuh"

namespace ppm {
namespace {

constexpr int ND = 5;  // tangents: M, R_e, incl, colat, zeta
constexpr int kTBlock = 64;  // four blocks per SM at 255 registers: their serial set-ups overlap

struct Dual {
    double v;
    double d[ND];
};

__device__ __forceinline__ Dual dconst(double v)
{
    Dual r;
    r.v = v;
#pragma unroll
    for (int i = 0; i < ND; ++i) r.d[i] = 0.0;
    return r;
}
__device__ __forceinline__ Dual dvar(double v, int dir, double scale = 1.0)
{
    Dual r = dconst(v);
    r.d[dir] = scale;
    return r;
}
__device__ __forceinline__ Dual operator+(const Dual &a, const Dual &b)
{
    Dual r;
    r.v = a.v + b.v;
#pragma unroll
    for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] + b.d[i];
    return r;
}
__device__ __forceinline__ Dual operator-(const Dual &a, const Dual &b)
{
    Dual r;
    r.v = a.v - b.v;
#pragma unroll
    for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] - b.d[i];
    return r;
}
__device__ __forceinline__ Dual operator-(const Dual &a)
{
    Dual r;
    r.v = -a.v;
#pragma unroll
    for (int i = 0; i < ND; ++i) r.d[i] = -a.d[i];
    return r;
}
__device__ __forceinline__ Dual operator*(const Dual &a, const Dual &b)
{
    Dual r;
    r.v = a.v * b.v;
#pragma unroll
    for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}
__device__ __forceinline__ Dual operator/(const Dual &a, const Dual &b)
{
    Dual r;
    const double ib = 1.0 / b.v;
    r.v = a.v * ib;
#pragma unroll
    for (int i = 0; i < ND; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
    return r;
}
__device__ __forceinline__ Dual operator+(const Dual &a, double b)
{
    Dual r = a;
    r.v += b;
    return r;
}
__device__ __forceinline__ Dual operator+(double b, const Dual &a) { return a + b; }
__device__ __forceinline__ Dual operator-(double b, const Dual &a) { return (-a) + b; }
__device__ __forceinline__ Dual operator*(const Dual &a, double b)
{
    Dual r;
    r.v = a.v * b;
#pragma unroll
    for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * b;
    return r;
}
__device__ __forceinline__ Dual operator*(double b, const Dual &a) { return a * b; }
__device__ __forceinline__ Dual operator/(const Dual &a, double b) { return a * (1.0 / b); }
__device__ __forceinline__ Dual operator/(double a, const Dual &b) { return dconst(a) / b; }
// f(a) with f'(a) given
__device__ __forceinline__ Dual chain(const Dual &a, double fv, double fd)
{
    Dual r;
    r.v = fv;
#pragma unroll
    for (int i = 0; i < ND; ++i) r.d[i] = fd * a.d[i];
    return r;
}
__device__ __forceinline__ Dual dsqrt(const Dual &a)
{
    const double s = sqrt(a.v);
    return chain(a, s, s > 0.0 ? 0.5 / s : 0.0);
}
// 1 / sqrt(a) for a > 0, derivative -0.5 a^(-3/2) (no FP64 division)
__device__ __forceinline__ Dual drsqrt(const Dual &a)
{
    const double r = rsqrt(a.v);
    return chain(a, r, -0.5 * r * r * r);
}
// sqrt(a) for a >= 0 through one reciprocal square root (derivative 0 at 0)
__device__ __forceinline__ Dual dsqrt_r(const Dual &a)
{
    if (!(a.v > 0.0)) return chain(a, 0.0, 0.0);
    const double r = rsqrt(a.v);
    return chain(a, a.v * r, 0.5 * r);
}
__device__ __forceinline__ Dual dsin(const Dual &a) { return chain(a, sin(a.v), cos(a.v)); }
__device__ __forceinline__ Dual dcos(const Dual &a) { return chain(a, cos(a.v), -sin(a.v)); }
__device__ __forceinline__ Dual dlog(const Dual &a) { return chain(a, log(a.v), 1.0 / a.v); }
__device__ __forceinline__ Dual dabs(const Dual &a) { return a.v < 0.0 ? -a : a; }

// Bilinear interpolant on a uniform grid and its two partial derivatives.
// The x (compactness) cell ix and weight tx are taken once per ring, and the
// grid scales sx = (nx - 1) / (x1 - x0) and sy likewise are precomputed: no
// FP64 division per point.
struct Bilin {
    double v, dx, dy;
    bool nan;
};
__device__ __forceinline__ Bilin bilin_u(const double *T, int ny, int ix, double tx, double sx,
                                         double y0, double sy, double y)
{
    const double fy = (y - y0) * sy;
    const int iy = min(max((int)floor(fy), 0), ny - 2);
    const double ty = fy - iy;
    const size_t k00 = (size_t)ix * ny + iy, k10 = k00 + ny;
    const double a00 = T[k00], a01 = T[k00 + 1], a10 = T[k10], a11 = T[k10 + 1];
    Bilin b;
    b.nan = isnan(a00) || isnan(a01) || isnan(a10) || isnan(a11);
    b.v = (1.0 - tx) * ((1.0 - ty) * a00 + ty * a01) + tx * ((1.0 - ty) * a10 + ty * a11);
    b.dx = ((1.0 - ty) * (a10 - a00) + ty * (a11 - a01)) * sx;
    b.dy = ((1.0 - tx) * (a01 - a00) + tx * (a11 - a10)) * sy;
    return b;
}

// per-ring constants of the template points' lookups
struct LensU {
    int iu;
    double tu, su, sc, sa, inv_nfp;
};

__device__ __forceinline__ LensU lens_u(const LensDev &L, double u, int n_fp)
{
    LensU U;
    U.su = (L.n_u - 1) / (L.u_max - L.u_min);
    const double fu = (u - L.u_min) * U.su;
    U.iu = min(max((int)floor(fu), 0), L.n_u - 2);
    U.tu = fu - U.iu;
    U.sc = (L.n_cpsi - 1) / (L.cpsi_max - L.cpsi_min);
    U.sa = (L.n_calpha - 1) / (L.ca_max - L.ca_min);
    U.inv_nfp = 1.0 / (double)n_fp;
    return U;
}

__device__ __forceinline__ Dual lift2(const Bilin &b, const Dual &x, const Dual &y)
{
    Dual r;
    r.v = b.v;
#pragma unroll
    for (int i = 0; i < ND; ++i) r.d[i] = b.dx * x.d[i] + b.dy * y.d[i];
    return r;
}

struct RingDual {
    Dual st, ct, R, u, sq1u, cos_eta, sin_eta, beta, gamma, area, dt_obl, sini, cosi, logg, half;
    Dual inv_sq, Rc;  // 1 / sqrt(1 - u), R / c
    double nu, phic;
    int ok;
};

__device__ void ring_setup(const Params &p, int b, int sidx, int r, int n_theta, int n_phi,
                           RingDual &G)
{
    const Dual M = dvar(p.mass_msun[b], 0);
    const Dual GM = M * kGM_SUN;
    const Dual Rs = 2.0 * GM / (kC * kC);
    const Dual Re = dvar(p.radius_km[b] * 1e3, 1, 1e3);
    const double nu = p.spin_hz[b];
    const double D = p.dist_kpc[b] * kKPC_M;
    const Dual Obar = 2.0 * kPI * nu * dsqrt(Re * Re * Re / GM);
    const Dual x = GM / (kC * kC * Re);
    const Dual o2 = p.oblate ? Obar * Obar * (-0.788 + 1.030 * x) : dconst(0.0);
    const Dual g0 = GM / (Re * Re) / dsqrt(1.0 - Rs / Re);
    const Dual tc = dvar(p.colat[sidx], 3), zt = dvar(p.zeta[sidx], 4);
    const Dual lo = (tc.v - zt.v > 0.0) ? tc - zt : dconst(0.0);
    const Dual hi = (tc.v + zt.v < kPI) ? tc + zt : dconst(kPI);
    const Dual dth = (hi - lo) / (double)n_theta;
    const Dual th = lo + (r + 0.5) * dth;
    const Dual dcs = dcos(lo + (double)r * dth) - dcos(lo + (double)(r + 1) * dth);
    const Dual st = dsin(th), ct = dcos(th);
    const Dual num = dcos(zt) - ct * dcos(tc), den = st * dsin(tc);
    Dual half;
    if (den.v <= 0.0) {
        half = dconst(num.v <= 0.0 ? kPI : 0.0);
    } else {
        const Dual q = num / den;
        if (q.v <= -1.0) half = dconst(kPI);
        else if (q.v >= 1.0) half = dconst(0.0);
        else half = chain(q, acos(q.v), -1.0 / sqrt(1.0 - q.v * q.v));
    }
    G.st = st; G.ct = ct; G.half = half;
    const Dual dphi = 2.0 * half / (double)n_phi;
    const Dual R = Re * (1.0 + o2 * ct * ct);
    const Dual u = Rs / R;
    const Dual sq = dsqrt(1.0 - u);
    const Dual f = -2.0 * o2 * Re * ct * st / (R * sq);
    const Dual nf = dsqrt(1.0 + f * f);
    G.R = R; G.u = u; G.sq1u = sq;
    G.inv_sq = 1.0 / sq;
    G.Rc = R * (1.0 / kC);
    G.cos_eta = 1.0 / nf;
    G.sin_eta = f / nf;
    Dual gg = g0;
    if (p.oblate) {
        const Dual O2 = Obar * Obar, O4 = O2 * O2, O6 = O4 * O2;
        const Dual c2 = ct * ct, s2 = st * st;
        const Dual k4 = O4 * (13.47 * x - 27.13 * x * x);
        gg = g0 * (1.0 +
                   s2 * (O2 * (-0.791 + 0.776 * x) + O4 * (-1.315 * x + 2.431 * x * x) +
                         O6 * (-1.172 * x)) +
                   c2 * (O2 * (1.138 - 1.431 * x) + O4 * (0.653 * x - 2.864 * x * x) +
                         O6 * (0.975 * x) - k4) +
                   dabs(ct) * k4);
    }
    G.logg = dlog(gg * 100.0) * (1.0 / log(10.0));
    G.beta = 2.0 * kPI * nu * R * st / (kC * sq);
    G.gamma = 1.0 / dsqrt(1.0 - G.beta * G.beta);
    G.area = R * R * nf * dcs * dphi * (kFluxScale / (D * D));
    G.dt_obl = (Re - R + Rs * dlog((Re - Rs) / (R - Rs))) / kC;
    G.nu = nu;
    const Dual inc = dvar(p.incl_rad[b], 2);
    G.sini = dsin(inc);
    G.cosi = dcos(inc);
    G.phic = p.azim[sidx];
    G.ok = half.v > 0.0;
}

// tangents of (F, z, mu, phi_o) at fine point i, contracted with the adjoints.
// FP64 is scarce on this GPU: the lookups' per-ring parts come from U and
// the per-point divisions are products with reciprocals (results change at
// the level of FP64 rounding).
__device__ __forceinline__ void point_tangent(const RingDual &G, const LensDev &L, const LensU &U,
                                              int i, double gF, double gZ, double gM, double gP,
                                              double *acc)
{
    double sphi, cphi;
    sincospi(2.0 * ((double)i * U.inv_nfp), &sphi, &cphi);
    const Dual cpsi = G.sini * G.st * cphi + G.cosi * G.ct;
    const Bilin bc = bilin_u(L.Ca, L.n_cpsi, U.iu, U.tu, U.su, L.cpsi_min, U.sc, cpsi.v);
    const Bilin bl = bilin_u(L.LF, L.n_cpsi, U.iu, U.tu, U.su, L.cpsi_min, U.sc, cpsi.v);
    if (bc.nan || bl.nan) return;  // cannot happen for a point the forward saw as visible
    const Dual ca = lift2(bc, G.u, cpsi);
    const Dual lf = lift2(bl, G.u, cpsi);
    const Dual sa = dsqrt_r(1.0 - ca * ca);
    const Dual sp2 = 1.0 - cpsi * cpsi;
    // sin(alpha) / sin(psi); its limit sqrt(LF) where sin(psi) < 1e-12
    const Dual ratio = sp2.v > 1e-24 ? sa * drsqrt(sp2) : dsqrt(lf);
    const Dual csig = ca * G.cos_eta + ratio * G.sin_eta * (G.cosi * G.st - G.sini * G.ct * cphi);
    const Dual cxi = -(ratio * G.sini * sphi);
    const Dual den = G.gamma * (1.0 - G.beta * cxi);  // 1 / delta
    const Dual delta = 1.0 / den;
    const Dual mu = delta * csig;
    const Dual F = G.sq1u * delta * delta * delta * mu * lf * G.gamma * G.area;
    const Dual z = den * G.inv_sq;                     // 1 / (delta sqrt(1 - u))
    // time delay: TD bilinear in (u, cos alpha), cos alpha clamped to the table
    Dual cac = ca;
    if (ca.v < L.ca_min) cac = dconst(L.ca_min);
    if (ca.v > L.ca_max) cac = dconst(L.ca_max);
    const Bilin bt = bilin_u(L.TD, L.n_calpha, U.iu, U.tu, U.su, L.ca_min, U.sa, cac.v);
    const Dual td = lift2(bt, G.u, cac);
    const Dual dt = G.Rc * td + G.dt_obl;
#pragma unroll
    for (int d = 0; d < ND; ++d)
        acc[d] += gF * F.d[d] + gZ * z.d[d] + gM * mu.d[d] + gP * G.nu * dt.d[d];
}

__global__ void __launch_bounds__(kTBlock) k_template_bwd(Params p, PlanDev plan, LensDev L,
                                                          AtmDev A, const RingRec *__restrict__ recs,
                                                          const float *__restrict__ tmpl,
                                                          const int *__restrict__ status,
                                                          const float *__restrict__ ringadj,
                                                          double *__restrict__ ring_grad)
{
    const int g = blockIdx.x;
    const int b = find_instance_by_ring(plan.inst, plan.B, g);
    const InstPlan ip = plan.inst[b];
    const int local = g - ip.ring0;
    const int spot = local / ip.n_theta, r = local % ip.n_theta;
    const int sidx = b * p.n_spots + spot;
    const int n_fp = plan.n_fp;
    const int tid = threadIdx.x;
    double *out = ring_grad + (size_t)g * kRingGrad;

    __shared__ double adj[4][kMaxFp + 1];  // folded gF, gZ, gMu, gPh
    __shared__ unsigned char vis[kMaxFp + 1];
    __shared__ RingDual G;
    __shared__ double red[kTBlock / 32][ND];
    __shared__ int s_lo, s_hi;

    const RingRec rec = recs[g];
    if (!rec.visible || status[b] != 0) {
        if (tid < kRingGrad) out[tid] = 0.0;
        return;
    }
    const float *ra = ringadj + (size_t)g * (4 * (n_fp + 1) + kRingAdjTail);
    const float *tF = tmpl + (size_t)g * 4 * (n_fp + 1) + (n_fp + 1);
    if (tid == 0) {
        ring_setup(p, b, sidx, r, ip.n_theta, ip.n_phi, G);
        s_lo = n_fp;
        s_hi = -1;
    }
    for (int i = tid; i <= n_fp; i += blockDim.x) {
#pragma unroll
        for (int q = 0; q < 4; ++q) adj[q][i] = (double)ra[q * (n_fp + 1) + i];
        vis[i] = tF[i] != 0.0f;
    }
    __syncthreads();
    for (int i = tid; i < n_fp; i += blockDim.x)
        if (!vis[i]) {
            atomicMin(&s_lo, i);
            atomicMax(&s_hi, i);
        }
    __syncthreads();
    // reverse of the fill: bridged points feed z and phi_o of their ends,
    // with weights (c - i) / (c - a) and (i - a) / (c - a); every thread sums
    // its share and the block adds the shares in a fixed order
    {
        double f[4] = {0.0, 0.0, 0.0, 0.0};  // to a: z, phi_o; to c: z, phi_o
        if (s_lo <= s_hi) {
            const int a = s_lo - 1, c = s_hi + 1;
            for (int i = s_lo + tid; i <= s_hi; i += blockDim.x) {
                const double t = (double)(i - a) / (double)(c - a);
                f[0] += (1.0 - t) * adj[1][i];
                f[1] += (1.0 - t) * adj[3][i];
                f[2] += t * adj[1][i];
                f[3] += t * adj[3][i];
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            double v = f[q];
            for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if ((tid & 31) == 0) red[tid >> 5][q] = v;
        }
    }
    __syncthreads();
    if (tid == 0) {
        if (s_lo <= s_hi) {
            const int a = s_lo - 1, c = s_hi + 1;
            double t[4] = {0.0, 0.0, 0.0, 0.0};
            for (int w = 0; w < kTBlock / 32; ++w)
                for (int q = 0; q < 4; ++q) t[q] += red[w][q];
            adj[1][a] += t[0];
            adj[3][a] += t[1];
            adj[1][c] += t[2];
            adj[3][c] += t[3];
        }
        // point n_fp is a copy of point 0
        for (int q = 0; q < 4; ++q) adj[q][0] += adj[q][n_fp];
    }
    __syncthreads();
    double acc[ND] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (G.ok) {
        const LensU U = lens_u(L, G.u.v, n_fp);
        for (int i = tid; i < n_fp; i += blockDim.x)
            if (vis[i]) point_tangent(G, L, U, i, adj[0][i], adj[1][i], adj[2][i], adj[3][i], acc);
    }
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        double v = acc[d];
        for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0) red[tid >> 5][d] = v;
    }
    __syncthreads();
    if (tid == 0) {
        double t[ND];
        for (int d = 0; d < ND; ++d) {
            t[d] = 0.0;
            for (int w = 0; w < kTBlock / 32; ++w) t[d] += red[w][d];
        }
        const float *tail = ra + 4 * (n_fp + 1);
        const double sgs = tail[0], sgss = tail[1], gT = tail[2], gG = tail[3], s_ref = tail[4];
        double gazim = 0.0, glogT = 0.0;
        if (G.ok) {
            // element azimuths s_m = (phic - half + (m + 1/2) 2 half / n_phi) / 2 pi
            gazim = sgs / (2.0 * kPI);
            const double ghalf = (2.0 * kPI * sgss + (2.0 * kPI * s_ref - G.phic) * sgs) /
                                 (2.0 * kPI * G.half.v);
            for (int d = 0; d < ND; ++d) t[d] += ghalf * G.half.d[d];
        }
        if (p.emission == 1) {
            // the tail carries dlogL/dlogT and dlogL/dlogg of the ring (the
            // stencil-weight derivatives, zero where clamped, are in the slabs)
            glogT = gT;
            for (int d = 0; d < ND; ++d) t[d] += gG * G.logg.d[d];
        } else {
            // blackbody: the tail carries dlogL/dkT; kT = k_B 10^logT
            glogT = gT * (double)rec.kT * log(10.0);
        }
        out[0] = t[0];
        out[1] = t[1];
        out[2] = t[2];
        out[3] = t[3];
        out[4] = gazim;
        out[5] = t[4];
        out[6] = glogT;
        out[7] = 0.0;
    }
}

}  // namespace

cudaError_t launch_template_bwd(const Params &p, const PlanDev &plan, const LensDev &L,
                                const AtmDev &A, const RingRec *recs, const float *tmpl,
                                const int *status, const float *ringadj, double *ring_grad,
                                cudaStream_t st)
{
    if (plan.total_rings <= 0) return cudaSuccess;
    k_template_bwd<<<plan.total_rings, kTBlock, 0, st>>>(p, plan, L, A, recs, tmpl, status,
                                                          ringadj, ring_grad);
    return cudaGetLastError();
}

}  // namespace ppm
