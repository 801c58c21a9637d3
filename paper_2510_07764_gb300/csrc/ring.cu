// Per-ring setup and pseudo-patch template, FP64 (Sect. 2.1-2.6, 2.8.3).
//
// One block per ring of one spot of one instance:
//   - star shape, slope, gravity and surface speed at the ring colatitude
//     (Eqs. Rtheta, Omega_c_def, def_f, the g(theta) fit of Sect. 2.2, the
//     beta of Sect. 2.4);
//   - the template F, z, phi_o, mu at the n_fp + 1 fine phases (the five
//     steps of Sect. 2.8.3: cos psi, lens lookup, Eq. sigma_relation,
//     visibility, Doppler factor and aberration, flux of Sect. 2.5) and the
//     invisible-segment fill;
//   - the list of active elements of the ring (mask caps removed), compacted;
//   - the ring's atmosphere cell in (logT, logg);
//   - the instance's range status: compactness, temperature or gravity outside
//     the tables, invalid geometry, or a non-finite parameter it uses.
// Every visibility and masking decision is taken in FP64, as in the oracle;
// the template is then stored in FP32 for the shift-and-add kernel.
#include "ppm_internal.cuh"

namespace ppm {
namespace {

constexpr unsigned kFullMask = 0xffffffffu;

struct RingGeo {
    double theta, st, ct, half, dphi, R, u, sq1u, cos_eta, sin_eta, logg, beta, gamma;
    double area, dt_obl, nu, sini, cosi, phic, mask_c, mask_ct, mask_st, mask_phi;
    double phi0, cap_c, cap_ct, cap_st;  // HEALPix mesh: first azimuth, emitter cap
    // per-ring parts of the template points: the lens tables' u cell and
    // weight, 1 / sqrt(1 - u), R / c
    double tu, inv_sq, Rc;
    int iu, ok, has_mask, n_el;
};

// The u (compactness) part of the bilinear lens lookups, the same for every
// template point of a ring: cell iu and weight tu.
__device__ __forceinline__ void lens_u(const LensDev &L, double u, int *iu, double *tu)
{
    const double fu = (u - L.u_min) / (L.u_max - L.u_min) * (L.n_u - 1);
    *iu = min(max((int)floor(fu), 0), L.n_u - 2);
    *tu = fu - *iu;
}

// C_alpha and LF at (u, cpsi), bilinear; the u cell and weight come from
// lens_u, the cpsi position is (cpsi - cpsi_min) * sc with
// sc = (n_cpsi - 1) / (cpsi_max - cpsi_min).  False where a corner is invalid.
__device__ bool lens_lookup_u(const LensDev &L, int iu, double tu, double cpsi, double sc,
                              double *ca, double *lf)
{
    double fc = (cpsi - L.cpsi_min) * sc;
    int ic = min(max((int)floor(fc), 0), L.n_cpsi - 2);
    double tc = fc - ic;
    size_t k00 = (size_t)iu * L.n_cpsi + ic, k10 = k00 + L.n_cpsi;
    double a00 = L.Ca[k00], a01 = L.Ca[k00 + 1], a10 = L.Ca[k10], a11 = L.Ca[k10 + 1];
    if (isnan(a00) || isnan(a01) || isnan(a10) || isnan(a11)) return false;
    double d00 = L.LF[k00], d01 = L.LF[k00 + 1], d10 = L.LF[k10], d11 = L.LF[k10 + 1];
    *ca = (1.0 - tu) * ((1.0 - tc) * a00 + tc * a01) + tu * ((1.0 - tc) * a10 + tc * a11);
    *lf = (1.0 - tu) * ((1.0 - tc) * d00 + tc * d01) + tu * ((1.0 - tc) * d10 + tc * d11);
    return true;
}

// TD at (u, ca), bilinear, ca clamped to its grid; sc = (n_calpha - 1) /
// (ca_max - ca_min)
__device__ double td_lookup_u(const LensDev &L, int iu, double tu, double ca, double sc)
{
    ca = fmin(fmax(ca, L.ca_min), L.ca_max);
    double fc = (ca - L.ca_min) * sc;
    int ic = min(max((int)floor(fc), 0), L.n_calpha - 2);
    double tc = fc - ic;
    size_t k00 = (size_t)iu * L.n_calpha + ic, k10 = k00 + L.n_calpha;
    return (1.0 - tu) * ((1.0 - tc) * L.TD[k00] + tc * L.TD[k00 + 1]) +
           tu * ((1.0 - tc) * L.TD[k10] + tc * L.TD[k10 + 1]);
}

// Stencil of one table axis at q (FP64): first node, taps, weights and their
// derivatives with respect to q.  rule 0: linear; 1: cubic Lagrange on the
// centred four nodes, linear where they would leave the grid; 2: cubic on
// four nodes moved inside the grid (one-sided at the edges).  q is clamped
// to the grid first (the clamped end has zero derivative).
__device__ int axis_stencil(const double *x, int n, double q, int rule, int *taps, float *w,
                            float *dw)
{
    bool clamped = false;
    if (q <= x[0]) { q = x[0]; clamped = true; }
    if (q >= x[n - 1]) { q = x[n - 1]; clamped = true; }
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (x[mid] <= q) lo = mid; else hi = mid;
    }
    if (lo > n - 2) lo = n - 2;
    int s0 = -1;
    if (rule == 1 && lo >= 1 && lo + 2 <= n - 1) s0 = lo - 1;
    if (rule == 2 && n >= 4) s0 = min(max(lo - 1, 0), n - 4);
    for (int a = 0; a < 4; ++a) w[a] = dw[a] = 0.0f;
    if (s0 < 0) {
        const double h = x[lo + 1] - x[lo];
        const double t = (q - x[lo]) / h;
        w[0] = (float)(1.0 - t);
        w[1] = (float)t;
        dw[0] = clamped ? 0.0f : (float)(-1.0 / h);
        dw[1] = clamped ? 0.0f : (float)(1.0 / h);
        *taps = 2;
        return lo;
    }
    for (int a = 0; a < 4; ++a) {
        double den = 1.0, prod = 1.0, der = 0.0;
        for (int b = 0; b < 4; ++b) {
            if (b == a) continue;
            den *= x[s0 + a] - x[s0 + b];
            der = der * (q - x[s0 + b]) + prod;
            prod *= q - x[s0 + b];
        }
        w[a] = (float)(prod / den);
        dw[a] = clamped ? 0.0f : (float)(der / den);
    }
    *taps = 4;
    return s0;
}

// ring-order index of the first pixel of HEALPix ring i (1-based), N = N_side
__device__ __forceinline__ long long healpix_first_pixel(int N, int i)
{
    const long long n = N;
    if (i < N) return 2LL * i * (i - 1);
    if (i <= 3 * N) return 2LL * n * (n - 1) + (long long)(i - N) * 4 * n;
    const long long k = 4LL * N - i;
    return 12LL * n * n - 2 * k * (k + 1);
}

// 128 threads per ring: at about 100 registers a thread four ring blocks fit
// on an SM, so that one block's FP64 set-up overlaps the others' points
constexpr int kRingThreads = 128;

__global__ void __launch_bounds__(kRingThreads, 4) k_ring(Params p, PlanDev plan, LensDev L, AtmDev A,
                                             RingRec *recs, float *tmpl, float *elems,
                                             int *status, unsigned *err,
                                             unsigned long long *triples, int nE, float2 *elemx)
{
    const int g = blockIdx.x;
    const int b = find_instance_by_ring(plan.inst, plan.B, g);
    const InstPlan ip = plan.inst[b];
    const int local = g - ip.ring0;
    const int spot = local / ip.n_theta, r = local % ip.n_theta;
    const int sidx = b * p.n_spots + spot;
    const int n_fp = plan.n_fp;

    __shared__ double sF[kMaxFp + 1], sZ[kMaxFp + 1], sPh[kMaxFp + 1], sMu[kMaxFp + 1];
    __shared__ RingGeo G;
    __shared__ int s_inv_min, s_inv_max, s_vis0, s_base, s_wsum[8], s_cmin, s_cmax;
    const bool use_map = p.logT_map != nullptr;  // (HEALPix mesh only)

    // Ring set-up by warp 0.  Every lane computes the same scalars; the
    // independent sines and cosines are evaluated in one lane-parallel
    // sincos (lane k takes argument k) and the two logarithms in one
    // lane-parallel log10, since an FP64 warp instruction costs the same with
    // one active lane as with 32.  Lane 0 writes the shared record.
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const double GM = p.mass_msun[b] * kGM_SUN;
        const double Rs = 2.0 * GM / (kC * kC);
        const double Re = p.radius_km[b] * 1e3;
        const double nu = p.spin_hz[b];
        const double D = p.dist_kpc[b] * kKPC_M;
        const double Obar = 2.0 * kPI * nu * sqrt(Re * Re * Re / GM);
        const double x = GM / (kC * kC * Re);
        const double o2 = p.oblate ? Obar * Obar * (-0.788 + 1.030 * x) : 0.0;
        const double g0 = GM / (Re * Re) / sqrt(1.0 - Rs / Re);
        const double tc = p.colat[sidx], zt = p.zeta[sidx];
        const double mz = p.mask_zeta[sidx];
        double th, dth = 0.0, lo = 0.0, z = 0.0;
        int n_el = ip.n_phi;
        double phi0 = 0.0, dphi_hp = 0.0;
        if (plan.grid == 1) {
            // HEALPix ring r + 1 of N_side = (rings + 1) / 4 (Gorski et al. 2005):
            // z, pixel count and first azimuth; every pixel has solid angle pi/(3 N^2)
            const int N = (ip.n_theta + 1) / 4, i = r + 1;
            const double NN = (double)N;
            if (i < N || i > 3 * N) {
                const int ipl = i < N ? i : 4 * N - i;
                const double zz = 1.0 - (double)ipl * ipl / (3.0 * NN * NN);
                z = i < N ? zz : -zz;
                n_el = 4 * ipl;
                phi0 = 0.25 * kPI / ipl;
            } else {
                z = 4.0 / 3.0 - 2.0 * i / (3.0 * NN);
                n_el = 4 * N;
                phi0 = 0.5 * kPI / NN * (1.0 - 0.5 * ((i - N + 1) % 2));
            }
            th = acos(z);
            dphi_hp = 2.0 * kPI / n_el;
        } else {
            // ring of the spot's bounding grid
            lo = fmax(tc - zt, 0.0);
            const double hi = fmin(tc + zt, kPI);
            dth = (hi - lo) / ip.n_theta;
            th = lo + (r + 0.5) * dth;
        }
        // lane-parallel sines and cosines
        double arg = 0.0;
        arg = lane == 0 ? th : arg;
        arg = lane == 1 ? lo + r * dth : arg;
        arg = lane == 2 ? lo + (r + 1) * dth : arg;
        arg = lane == 3 ? tc : arg;
        arg = lane == 4 ? zt : arg;
        arg = lane == 5 ? p.incl_rad[b] : arg;
        arg = lane == 6 ? p.mask_colat[sidx] : arg;
        arg = lane == 7 ? mz : arg;
        double sv, cv;
        sincos(arg, &sv, &cv);
        const double st = __shfl_sync(kFullMask, sv, 0), ct = __shfl_sync(kFullMask, cv, 0);
        const double c_lo = __shfl_sync(kFullMask, cv, 1), c_hi = __shfl_sync(kFullMask, cv, 2);
        const double s_tc = __shfl_sync(kFullMask, sv, 3), c_tc = __shfl_sync(kFullMask, cv, 3);
        const double c_zt = __shfl_sync(kFullMask, cv, 4);
        const double sini = __shfl_sync(kFullMask, sv, 5), cosi = __shfl_sync(kFullMask, cv, 5);
        const double s_mc = __shfl_sync(kFullMask, sv, 6), c_mc = __shfl_sync(kFullMask, cv, 6);
        const double c_mz = __shfl_sync(kFullMask, cv, 7);
        double dcos, half, dphi;
        if (plan.grid == 1) {
            dphi = dphi_hp;
            dcos = (kPI / (3.0 * ((ip.n_theta + 1) / 4) * ((ip.n_theta + 1) / 4))) / dphi;
            // rings that cannot reach the emitter cap hold no pixel of the spot;
            // with a temperature map every ring is a candidate
            half = (use_map || fabs(th - tc) <= zt + 1e-12) ? kPI : 0.0;
        } else {
            dcos = c_lo - c_hi;
            const double num = c_zt - ct * c_tc, den = st * s_tc;
            if (den <= 0.0) half = num <= 0.0 ? kPI : 0.0;
            else half = acos(fmin(fmax(num / den, -1.0), 1.0));
            dphi = 2.0 * half / ip.n_phi;
        }
        // shape, slope, gravity, speed
        const double R = Re * (1.0 + o2 * ct * ct);
        const double u = Rs / R;
        const double sq = sqrt(1.0 - u);
        const double f = -2.0 * o2 * Re * ct * st / (R * sq);
        const double sf = sqrt(1.0 + f * f);
        double gg = g0;
        if (p.oblate) {
            const double O2 = Obar * Obar, O4 = O2 * O2, O6 = O4 * O2;
            const double c2 = ct * ct, s2 = st * st;
            gg = g0 * (1.0 +
                       s2 * (O2 * (-0.791 + 0.776 * x) + O4 * (-1.315 * x + 2.431 * x * x) +
                             O6 * (-1.172 * x)) +
                       c2 * (O2 * (1.138 - 1.431 * x) + O4 * (0.653 * x - 2.864 * x * x) +
                             O6 * (0.975 * x) - O4 * (13.47 * x - 27.13 * x * x)) +
                       fabs(ct) * O4 * (13.47 * x - 27.13 * x * x));
        }
        // lane-parallel log10: lane 0 the surface gravity, lane 1 the oblate delay ratio
        const double lv = log10(lane == 1 ? (Re - Rs) / (R - Rs) : gg * 100.0);
        const double logg = __shfl_sync(kFullMask, lv, 0);
        const double lnr = __shfl_sync(kFullMask, lv, 1) * 2.302585092994045684;
        const double beta = 2.0 * kPI * nu * R * st / (kC * sq);
        const double area = R * R * sf * dcos * dphi / (D * D) * kFluxScale;
        if (lane == 0) {
            G.theta = th; G.st = st; G.ct = ct; G.half = half;
            G.n_el = n_el; G.dphi = dphi; G.phi0 = phi0;
            G.cap_c = c_zt; G.cap_ct = c_tc; G.cap_st = s_tc;
            G.R = R; G.u = u; G.sq1u = sq;
            lens_u(L, u, &G.iu, &G.tu);
            G.inv_sq = 1.0 / sq;
            G.Rc = R / kC;
            G.cos_eta = 1.0 / sf;
            G.sin_eta = f / sf;
            G.logg = logg;
            G.beta = beta;
            G.gamma = 1.0 / sqrt(1.0 - beta * beta);
            G.area = area;
            G.dt_obl = (Re - R + Rs * lnr) / kC;
            G.nu = nu;
            G.sini = sini; G.cosi = cosi;
            G.phic = p.azim[sidx];
            G.has_mask = mz > 0.0;
            G.mask_c = G.has_mask ? c_mz : 2.0;
            G.mask_ct = c_mc;
            G.mask_st = s_mc;
            G.mask_phi = p.mask_azim[sidx];
            // range checks (per-instance status)
            bool in_range = u >= L.u_min && u <= L.u_max && D > 0.0 && nu >= 0.0 &&
                            beta < 1.0 && Re > Rs && p.incl_rad[b] >= 0.0 &&
                            p.incl_rad[b] <= kPI && isfinite(area);
            if (!use_map) in_range = in_range && zt > 0.0 && zt <= kPI && tc >= 0.0 && tc <= kPI;
            // inputs that no comparison above reaches: a NaN or infinite value
            // flags the instance instead of running through its profile (a
            // mask needs finite geometry; mask_zeta <= 0, even -inf, is no mask)
            in_range = in_range && isfinite(p.nh_1e20[b]);
            if (!use_map)
                in_range = in_range && isfinite(G.phic) && isfinite(p.logT[sidx]) && !isnan(mz) &&
                           (!(mz > 0.0) || (isfinite(mz) && isfinite(p.mask_colat[sidx]) &&
                                            isfinite(G.mask_phi)));
            if (p.emission == 1) {
                in_range = in_range && logg >= A.logg[0] && logg <= A.logg[A.ng - 1];
                if (!use_map) {
                    const double lt = p.logT[sidx];
                    in_range = in_range && lt >= A.logT[0] && lt <= A.logT[A.nT - 1];
                }
            }
            if (!in_range) atomicMax(&status[b], (int)PPM_ERANGE);
            G.ok = in_range && half > 0.0;
            s_inv_min = n_fp;
            s_inv_max = 0;
            s_vis0 = 0;
            s_cmin = 1 << 30;
            s_cmax = -1;
        }
    }
    __syncthreads();

    const size_t tbase = (size_t)g * 4 * (n_fp + 1);
    if (G.ok) {
        const LensDev Lc = L;
        // FP64 is scarce on this GPU: the per-ring parts of the lookups are
        // hoisted and the per-point divisions become products with
        // reciprocals taken once (results change at the level of FP64 rounding)
        const int iu = G.iu;
        const double tu = G.tu;
        const double sc_c = (Lc.n_cpsi - 1) / (Lc.cpsi_max - Lc.cpsi_min);
        const double sc_a = (Lc.n_calpha - 1) / (Lc.ca_max - Lc.ca_min);
        const double inv_nfp = 1.0 / (double)n_fp;
        for (int i = threadIdx.x; i < n_fp; i += blockDim.x) {
            const double x = (double)i * inv_nfp;  // i / n_fp
            double sphi, cphi;
            sincospi(2.0 * x, &sphi, &cphi);
            // step 2: cos psi
            const double cpsi = G.sini * G.st * cphi + G.cosi * G.ct;
            bool vis = false;
            double ca, lf;
            // step 3: lens table; beyond its cos psi range the point is invisible
            if (cpsi >= Lc.cpsi_min && lens_lookup_u(Lc, iu, tu, cpsi, sc_c, &ca, &lf)) {
                const double sa = sqrt(fmax(0.0, 1.0 - ca * ca));
                const double sp2 = fmax(0.0, 1.0 - cpsi * cpsi);
                // sin(alpha) / sin(psi); its limit sqrt(LF) where sin(psi) < 1e-12
                const double ratio = sp2 > 1e-24 ? sa * rsqrt(sp2) : sqrt(lf);
                // step 4: Eq. sigma_relation
                const double csig = ca * G.cos_eta +
                                    ratio * G.sin_eta * (G.cosi * G.st - G.sini * G.ct * cphi);
                // step 5
                if (csig >= 0.0) {
                    vis = true;
                    const double cxi = -ratio * G.sini * sphi;
                    const double den = G.gamma * (1.0 - G.beta * cxi);  // 1 / delta
                    const double delta = 1.0 / den;
                    const double mu = delta * csig;
                    sF[i] = G.sq1u * delta * delta * delta * mu * lf * G.gamma * G.area;
                    sZ[i] = den * G.inv_sq;                             // 1 / (delta sqrt(1-u))
                    const double dt = G.Rc * td_lookup_u(Lc, iu, tu, ca, sc_a) + G.dt_obl;
                    sPh[i] = x + G.nu * dt;
                    sMu[i] = mu;
                }
            }
            if (!vis) {
                atomicMin(&s_inv_min, i);
                atomicMax(&s_inv_max, i);
                sF[i] = 0.0; sZ[i] = 0.0; sPh[i] = 0.0; sMu[i] = 0.0;
            }
            if (i == 0) s_vis0 = vis;
        }
        __syncthreads();
        const bool vis0 = s_vis0;
        // point n_fp is point 0 one rotation later (it closes the fill interval)
        if (vis0 && threadIdx.x == 0) {
            sF[n_fp] = sF[0]; sZ[n_fp] = sZ[0]; sMu[n_fp] = sMu[0]; sPh[n_fp] = sPh[0] + 1.0;
        }
        __syncthreads();
        if (vis0) {
            const int a = s_inv_min - 1, c = s_inv_max + 1;
            for (int i = threadIdx.x; i < n_fp; i += blockDim.x) {
                if (s_inv_min <= s_inv_max && i >= s_inv_min && i <= s_inv_max) {
                    const double t = (double)(i - a) / (double)(c - a);
                    sZ[i] = sZ[a] + (sZ[c] - sZ[a]) * t;
                    sPh[i] = sPh[a] + (sPh[c] - sPh[a]) * t;
                }
            }
        }
        __syncthreads();
        if (vis0) {
            float *tp = tmpl + tbase;
            for (int i = threadIdx.x; i <= n_fp; i += blockDim.x) {
                tp[i] = (float)sPh[i];
                tp[(n_fp + 1) + i] = (float)sF[i];
                tp[2 * (n_fp + 1) + i] = (float)sZ[i];
                tp[3 * (n_fp + 1) + i] = (float)sMu[i];
                if (i < n_fp && !(sPh[i + 1] > sPh[i])) atomicOr(err, kErrPhaseOrder);
            }
        }
    }

    // active elements, compacted (FP64 mask test, as in the oracle)
    int n_active = 0;
    if (G.ok) {
        float *ep = elems + (size_t)ip.elem0 + (size_t)local * ip.n_phi;
        float2 *xp = use_map ? elemx + (size_t)ip.elem0 + (size_t)local * ip.n_phi : nullptr;
        const long long pix_first =
            use_map ? (long long)ip.pix0 + healpix_first_pixel((ip.n_theta + 1) / 4, r + 1) : 0;
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (threadIdx.x == 0) s_base = 0;
        __syncthreads();
        for (int m0 = 0; m0 < G.n_el; m0 += blockDim.x) {
            const int m = m0 + threadIdx.x;
            bool act = false;
            double phia = 0.0;
            float2 xv = make_float2(0.0f, 0.0f);
            if (m < G.n_el && use_map) {
                // temperature map: the pixel's own log T; dark where not finite or <= 0
                phia = G.phi0 + m * G.dphi;
                const double lt = p.logT_map[pix_first + m];
                act = isfinite(lt) && lt > 0.0;
                if (act && p.emission == 1) {
                    if (lt < A.logT[0] || lt > A.logT[A.nT - 1]) {
                        atomicMax(&status[b], (int)PPM_ERANGE);
                        act = false;
                    } else {
                        int taps;
                        float w[4], dw[4];
                        const int c = axis_stencil(A.logT, A.nT, lt, 0, &taps, w, dw);
                        xv = make_float2(w[1], __int_as_float(c));
                        atomicMin(&s_cmin, c);
                        atomicMax(&s_cmax, c);
                    }
                } else if (act) {
                    xv = make_float2((float)(kKB_KEVK * pow(10.0, lt)), 0.0f);
                }
            } else if (m < G.n_el) {
                if (plan.grid == 1) {
                    // mesh pixel: inside the emitter cap (FP64, as in the oracle)
                    phia = G.phi0 + m * G.dphi;
                    act = G.ct * G.cap_ct + G.st * G.cap_st * cos(phia - G.phic) >= G.cap_c;
                } else {
                    phia = G.phic - G.half + (m + 0.5) * G.dphi;
                    act = true;
                }
                if (act && G.has_mask) {
                    const double cd = G.ct * G.mask_ct + G.st * G.mask_st * cos(phia - G.mask_phi);
                    act = !(cd > G.mask_c);
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, act);
            if (lane == 0) s_wsum[wid] = __popc(bal);
            __syncthreads();
            int off = s_base;
            for (int w = 0; w < wid; ++w) off += s_wsum[w];
            if (act) {
                const int slot = off + __popc(bal & ((1u << lane) - 1u));
                PPM_CHECK(slot < ip.n_phi, plan.err);
                ep[slot] = (float)(phia / (2.0 * kPI));
                if (use_map) xp[slot] = xv;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                int tot = 0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += s_wsum[w];
                s_base += tot;
            }
            __syncthreads();
        }
        n_active = s_base;
    }

    // the (logT, logg) stencils, one axis per lane of warp 0: linear for D,
    // cubic for C, one-sided cubic for A and B; the logg stencil of a map is
    // linear (its logT cells come from the pixels)
    __shared__ int s_sti[2], s_stt[2];
    __shared__ float s_stw[2][4], s_stdw[2][4];
    const double lt = p.logT[sidx];
    if (threadIdx.x < 2 && p.emission == 1) {
        const bool gax = threadIdx.x == 1;
        const int rule = (gax && use_map) ? 0
                         : (A.strategy == kInterpD ? 0 : (A.strategy == kInterpC ? 1 : 2));
        int taps;
        float w[4], dw[4];
        const int i0 = axis_stencil(gax ? A.logg : A.logT, gax ? A.ng : A.nT, gax ? G.logg : lt,
                                    rule, &taps, w, dw);
        s_sti[threadIdx.x] = i0;
        s_stt[threadIdx.x] = taps;
        for (int a = 0; a < 4; ++a) {
            s_stw[threadIdx.x][a] = w[a];
            s_stdw[threadIdx.x][a] = dw[a];
        }
    }
    if (threadIdx.x < 32) __syncwarp();
    if (threadIdx.x == 0) {
        RingRec rec;
        rec.visible = (G.ok && s_vis0 && n_active > 0) ? 1 : 0;
        rec.n_active = n_active;
        rec.iT = 0; rec.ig = 0; rec.tT = 0; rec.tg = 0;
        for (int a = 0; a < 4; ++a) rec.wT[a] = rec.wg[a] = rec.dwT[a] = rec.dwg[a] = 0.0f;
        rec.kT = (float)(kKB_KEVK * exp(lt * 2.302585092994045684));
        if (p.emission == 1) {
            rec.iT = s_sti[0]; rec.tT = s_stt[0];
            rec.ig = s_sti[1]; rec.tg = s_stt[1];
            for (int a = 0; a < 4; ++a) {
                rec.wT[a] = s_stw[0][a]; rec.dwT[a] = s_stdw[0][a];
                rec.wg[a] = s_stw[1][a]; rec.dwg[a] = s_stdw[1][a];
            }
        }
        rec.map = use_map ? 1 : 0;
        if (use_map && p.emission == 1) {
            // the logT cells used by the ring's pixels
            rec.iT = s_cmax >= 0 ? s_cmin : 0;
            rec.tT = s_cmax >= 0 ? s_cmax - s_cmin + 1 : 0;
        }
        recs[g] = rec;
        if (triples && rec.visible)
            atomicAdd(triples, (unsigned long long)n_active * ip.n_phase * ip.n_sub * nE);
    }
}

}  // namespace

cudaError_t launch_ring(const Params &p, const PlanDev &plan, const LensDev &L, const AtmDev &A,
                        RingRec *recs, float *tmpl, float *elems, int *status, unsigned *err,
                        unsigned long long *triples, int nE, cudaStream_t st, float2 *elemx)
{
    if (plan.total_rings <= 0) return cudaSuccess;
    k_ring<<<plan.total_rings, kRingThreads, 0, st>>>(p, plan, L, A, recs, tmpl, elems, status, err,
                                             triples, nE, elemx);
    return cudaGetLastError();
}

}  // namespace ppm
