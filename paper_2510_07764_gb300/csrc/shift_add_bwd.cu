// Adjoint of the shift-and-add with atmosphere interpolation (reverse mode of
// Eq. add_Ft and of the Sect. 4 interpolation), FP32.
//
// Input: A[row][k] = dlogL/dF_t[row][k] / (E_k * flux scale), i.e. the adjoint
// of every contribution F_p I(z_p E_k, mu_p) (F_p in template units).
// One block per ring, all output phases.  For every (element, phase) pair the
// block accumulates, over the energies,
//     sF  = sum_k A_k I_k                 -> dlogL/dF_p
//     sZ  = sum_k A_k dI/dt_k             -> dlogL/dz_p  (t = table position in ln E)
//     sMu = sum_k A_k dI/dmu_k            -> dlogL/dmu_p
//     sT  = sum_k A_k dI/dlogT_k          -> dlogL/dlogT of the ring
//     sG  = sum_k A_k dI/dlogg_k          -> dlogL/dlogg of the ring
// from four sliding interval cubics (intensity, mu-derivative weights, and the
// slab's derivatives with respect to logT and logg, staged alongside it
// from the derivatives of the ring's stencil weights), then scatters them onto
// the ring's template adjoints through the linear phase interpolation,
// including the dependence of the interpolation weight on phi_o and on the
// element azimuth.  The per-ring record (floats):
//     gF[n_fp+1] gZ[n_fp+1] gMu[n_fp+1] gPh[n_fp+1] | sum gs | sum gs*(s - s_ref) | gT | gg
//     | s_ref | 0 0 0
// where gs is the adjoint of an element's azimuth / 2 pi and the second
// tail sum is taken about s_ref (the ring's first active element), which
// keeps it free of cancellation for narrow azimuth spans.
#include "ppm_internal.cuh"

namespace ppm {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kBwdBlock = 512;
// node-major walk: zero adjoints before energy 0 and past the last energy,
// and table rows past the slab that slots beyond their last interval read
constexpr int kApadLead = 2, kApadTail = 16, kBwdMargin = 3;

// floats of a warp's adjoint row: (position, adjoint) pairs, or the padded
// adjoints of the node-major walk
__host__ __device__ constexpr int arow_len(int nEpad) { return 2 * nEpad + kApadLead + kApadTail; }

struct BLayout {
    int tmpl, elems, munodes, pk, E3, arow, adj, red, slab, slabT, slabG, total;
    int det;  // 1: one adjoint copy per warp, added in a fixed order (bitwise reproducible)
};

__device__ __forceinline__ float dot4(const float *__restrict__ q, float w0, float w1, float w2,
                                      float w3)
{
    return fmaf(w3, q[3], fmaf(w2, q[2], fmaf(w1, q[1], w0 * q[0])));
}

struct Cubic {
    float c0, c1, c2, c3, W2, W3;  // power basis of the current interval + nodes q+1, q+2
};

__device__ __forceinline__ void cubic_set(Cubic &C, float a, float b, float c, float d)
{
    C.c0 = b;
    C.c2 = fmaf(0.5f, a + c, -b);
    C.c3 = fmaf(d - a, 1.0f / 6.0f, 0.5f * (b - c));
    C.c1 = fmaf(c - a, 0.5f, -C.c3);
    C.W2 = c;
    C.W3 = d;
}

__device__ __forceinline__ float horner(const Cubic &C, float t)
{
    return fmaf(t, fmaf(t, fmaf(t, C.c3, C.c2), C.c1), C.c0);
}

// the same for two interleaved cubics (packed FP32 pair arithmetic)
struct Cubic2 {
    float2 c0, c1, c2, c3, W2, W3;
};

__device__ __forceinline__ void cubic2_set(Cubic2 &C, float2 a, float2 b, float2 c, float2 d)
{
    const float2 h = make_float2(0.5f, 0.5f), s6 = make_float2(1.0f / 6.0f, 1.0f / 6.0f);
    C.c0 = b;
    C.c2 = __ffma2_rn(h, __fadd2_rn(a, c), make_float2(-b.x, -b.y));
    C.c3 = __ffma2_rn(__fadd2_rn(d, make_float2(-a.x, -a.y)), s6,
                      __fmul2_rn(h, __fadd2_rn(b, make_float2(-c.x, -c.y))));
    C.c1 = __ffma2_rn(__fadd2_rn(c, make_float2(-a.x, -a.y)), h, make_float2(-C.c3.x, -C.c3.y));
    C.W2 = c;
    C.W3 = d;
}

__device__ __forceinline__ void cubic2_shift(Cubic2 &C, float2 d)
{
    cubic2_set(C, C.c0, C.W2, C.W3, d);
}

__device__ __forceinline__ float2 horner2(const Cubic2 &C, float2 t)
{
    return __ffma2_rn(t, __ffma2_rn(t, __ffma2_rn(t, C.c3, C.c2), C.c1), C.c0);
}

__device__ __forceinline__ float2 horner2(float2 k0, float2 k1, float2 k2, float2 k3, float2 t)
{
    return __ffma2_rn(t, __ffma2_rn(t, __ffma2_rn(t, k3, k2), k1), k0);
}

// state of one (element, phase) pair in the backward pass
struct PairB {
    bool on;
    float Fp, zp, w, dphi, dF, dZ, dM;  // interpolation weight, phi_o step, template differences
    int i;                              // template interval
    float w0, w1, w2, w3;               // mu weights (not scaled by F_p)
    float v0, v1, v2, v3;               // their mu derivatives
    int s0;
    float lz;
};

template <bool ATM>
__device__ __forceinline__ PairB pair_bwd(bool on, float s, float phi_out, const float *ph,
                                          const float *mun, int n_fp, int top, const AtmDev &A,
                                          float inv_dlnE)
{
    PairB P;
    P.on = false;
    P.Fp = P.zp = P.w = P.dphi = P.dF = P.dZ = P.dM = 0.0f;
    P.i = 0;
    P.w0 = P.w1 = P.w2 = P.w3 = P.v0 = P.v1 = P.v2 = P.v3 = 0.0f;
    P.s0 = 0;
    P.lz = 0.0f;
    if (!on) return P;
    const float *F = ph + (n_fp + 1), *Z = F + (n_fp + 1), *M = Z + (n_fp + 1);
    const float x = phi_out + s + 1.0f - ph[0];
    const float phip = x - floorf(x) + ph[0];
    int lo = 0;
    for (int step = top; step > 0; step >>= 1) {
        const int c = lo + step;
        if (c <= n_fp - 1 && ph[c] <= phip) lo = c;
    }
    const float dphi = ph[lo + 1] - ph[lo];
    float w = (phip - ph[lo]) / dphi;
    const bool wclamp = !(w >= 0.0f && w <= 1.0f);
    w = fminf(fmaxf(w, 0.0f), 1.0f);
    const float Fp = fmaf(F[lo + 1] - F[lo], w, F[lo]);
    const float zp = fmaf(Z[lo + 1] - Z[lo], w, Z[lo]);
    const float mp = fmaf(M[lo + 1] - M[lo], w, M[lo]);
    if (!(Fp != 0.0f && zp > 0.0f && zp < 1e30f)) return P;
    P.on = true;
    P.Fp = Fp;
    P.zp = zp;
    P.i = lo;
    P.w = w;
    P.dphi = wclamp ? 0.0f : dphi;  // zero marks a clamped weight (no phase derivative)
    P.dF = F[lo + 1] - F[lo];
    P.dZ = Z[lo + 1] - Z[lo];
    P.dM = M[lo + 1] - M[lo];
    if (!ATM) return P;
    const int nmu = A.nmu;
    const bool mclamp = !(mp > mun[0] && mp < mun[nmu - 1]);
    const float mu = fminf(fmaxf(mp, mun[0]), mun[nmu - 1]);
    int i = 0;
    for (int step = 64; step > 0; step >>= 1) {
        const int c = i + step;
        if (c <= nmu - 2 && mun[c] <= mu) i = c;
    }
    float wv[4] = {0.f, 0.f, 0.f, 0.f}, dv[4] = {0.f, 0.f, 0.f, 0.f};
    int s0;
    const bool onesided = A.strategy == kInterpA || A.strategy == kInterpB;
    if (onesided || (i >= 1 && i + 2 <= nmu - 1 && i >= A.n_protect - 1)) {
        s0 = onesided ? min(max(i - 1, 0), nmu - 4) : i - 1;
        float x4[4] = {mun[s0], mun[s0 + 1], mun[s0 + 2], mun[s0 + 3]};
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            float den = 1.0f, prod = 1.0f, der = 0.0f;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                if (b == a) continue;
                den *= (x4[a] - x4[b]);
                // d/dmu prod_{b != a} (mu - x_b): product rule
                der = der * (mu - x4[b]) + prod;
                prod *= (mu - x4[b]);
            }
            wv[a] = prod / den;
            dv[a] = der / den;
        }
    } else {
        s0 = min(max(i - 1, 0), nmu - 4);
        const float h = mun[i + 1] - mun[i];
        const float t = (mu - mun[i]) / h;
        const int o = i - s0;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            wv[a] = (a == o) ? 1.0f - t : ((a == o + 1) ? t : 0.0f);
            dv[a] = (a == o) ? -1.0f / h : ((a == o + 1) ? 1.0f / h : 0.0f);
        }
    }
    if (mclamp) dv[0] = dv[1] = dv[2] = dv[3] = 0.0f;
    P.w0 = wv[0]; P.w1 = wv[1]; P.w2 = wv[2]; P.w3 = wv[3];
    P.v0 = dv[0]; P.v1 = dv[1]; P.v2 = dv[2]; P.v3 = dv[3];
    P.s0 = s0;
    P.lz = logf(zp) * inv_dlnE;
    return P;
}

struct Quint {
    float I, dI, Im, It, Ig;
};

// general evaluation at table position p (edges / clamping), all five values
__device__ __noinline__ Quint bwd_general(const PairB &P, const float *S, const float *ST,
                                          const float *SG, int Pm, int nE_t, float p,
                                          bool onesided)
{
    Quint Q;
    int q0, qn;
    bool cubic = false, clamp = false;
    float t = 0.0f;
    if (p <= 0.0f) { q0 = 0; clamp = true; }
    else if (p >= (float)(nE_t - 1)) { q0 = nE_t - 1; clamp = true; }
    else {
        const float q = floorf(p);
        q0 = (int)q;
        t = p - q;
        cubic = q0 >= 1 && q0 + 2 <= nE_t - 1;
        if (onesided && !cubic) {
            // cubic on the four nodes s..s+3 inside the grid (strategies A, B):
            // Lagrange basis at x = p - s and its derivative
            const int s = min(max(q0 - 1, 0), nE_t - 4);
            const float x = p - (float)s;
            const float l[4] = {-(x - 1.0f) * (x - 2.0f) * (x - 3.0f) * (1.0f / 6.0f),
                                x * (x - 2.0f) * (x - 3.0f) * 0.5f,
                                -x * (x - 1.0f) * (x - 3.0f) * 0.5f,
                                x * (x - 1.0f) * (x - 2.0f) * (1.0f / 6.0f)};
            const float dl[4] = {
                -((x - 2.0f) * (x - 3.0f) + (x - 1.0f) * (x - 3.0f) + (x - 1.0f) * (x - 2.0f)) *
                    (1.0f / 6.0f),
                ((x - 2.0f) * (x - 3.0f) + x * (x - 3.0f) + x * (x - 2.0f)) * 0.5f,
                -((x - 1.0f) * (x - 3.0f) + x * (x - 3.0f) + x * (x - 1.0f)) * 0.5f,
                ((x - 1.0f) * (x - 2.0f) + x * (x - 2.0f) + x * (x - 1.0f)) * (1.0f / 6.0f)};
            Q.I = Q.dI = Q.Im = Q.It = Q.Ig = 0.0f;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const float *r = S + (s + a) * Pm + P.s0;
                const float yi = dot4(r, P.w0, P.w1, P.w2, P.w3);
                Q.I = fmaf(l[a], yi, Q.I);
                Q.dI = fmaf(dl[a], yi, Q.dI);
                Q.Im = fmaf(l[a], dot4(r, P.v0, P.v1, P.v2, P.v3), Q.Im);
                Q.It = fmaf(l[a], dot4(ST + (s + a) * Pm + P.s0, P.w0, P.w1, P.w2, P.w3), Q.It);
                Q.Ig = fmaf(l[a], dot4(SG + (s + a) * Pm + P.s0, P.w0, P.w1, P.w2, P.w3), Q.Ig);
            }
            return Q;
        }
    }
    qn = q0;
    auto node = [&](const float *B, int n, float a0, float a1, float a2, float a3) {
        return dot4(B + n * Pm + P.s0, a0, a1, a2, a3);
    };
    if (clamp) {
        Q.I = node(S, qn, P.w0, P.w1, P.w2, P.w3);
        Q.Im = node(S, qn, P.v0, P.v1, P.v2, P.v3);
        Q.It = node(ST, qn, P.w0, P.w1, P.w2, P.w3);
        Q.Ig = node(SG, qn, P.w0, P.w1, P.w2, P.w3);
        Q.dI = 0.0f;
        return Q;
    }
    if (cubic) {
        Cubic c[4];
        const float *B[4] = {S, S, ST, SG};
#pragma unroll
        for (int z = 0; z < 4; ++z) {
            const bool der = (z == 1);
            const float a0 = der ? P.v0 : P.w0, a1 = der ? P.v1 : P.w1;
            const float a2 = der ? P.v2 : P.w2, a3 = der ? P.v3 : P.w3;
            cubic_set(c[z], node(B[z], q0 - 1, a0, a1, a2, a3), node(B[z], q0, a0, a1, a2, a3),
                      node(B[z], q0 + 1, a0, a1, a2, a3), node(B[z], q0 + 2, a0, a1, a2, a3));
        }
        Q.I = horner(c[0], t);
        Q.dI = fmaf(t, fmaf(t, 3.0f * c[0].c3, 2.0f * c[0].c2), c[0].c1);
        Q.Im = horner(c[1], t);
        Q.It = horner(c[2], t);
        Q.Ig = horner(c[3], t);
        return Q;
    }
    const float b0 = node(S, q0, P.w0, P.w1, P.w2, P.w3), b1 = node(S, q0 + 1, P.w0, P.w1, P.w2, P.w3);
    Q.I = fmaf(t, b1 - b0, b0);
    Q.dI = b1 - b0;
    const float m0 = node(S, q0, P.v0, P.v1, P.v2, P.v3), m1 = node(S, q0 + 1, P.v0, P.v1, P.v2, P.v3);
    Q.Im = fmaf(t, m1 - m0, m0);
    const float t0 = node(ST, q0, P.w0, P.w1, P.w2, P.w3), t1 = node(ST, q0 + 1, P.w0, P.w1, P.w2, P.w3);
    Q.It = fmaf(t, t1 - t0, t0);
    const float g0 = node(SG, q0, P.w0, P.w1, P.w2, P.w3), g1 = node(SG, q0 + 1, P.w0, P.w1, P.w2, P.w3);
    Q.Ig = fmaf(t, g1 - g0, g0);
    return Q;
}

template <int EMIS, bool CLIP, bool NODES>
__global__ void __launch_bounds__(kBwdBlock, 1)
    k_shift_add_bwd(Params p, PlanDev plan, AtmDev A, EnergyDev en, BLayout lay,
                    const RingRec *__restrict__ recs, const float *__restrict__ tmpl,
                    const float *__restrict__ elems, const int *__restrict__ status,
                    const float *__restrict__ Aadj, float *__restrict__ ringadj)
{
    extern __shared__ float sm[];
    const int ring = blockIdx.x;
    const int b = find_instance_by_ring(plan.inst, plan.B, ring);
    const InstPlan ip = plan.inst[b];
    const int n_fp = plan.n_fp;
    const int nE = en.nE, nEpad = en.nEpad;
    const int rec_len = 4 * (n_fp + 1) + kRingAdjTail;
    float *out = ringadj + (size_t)ring * rec_len;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const RingRec rec = recs[ring];
    if (!rec.visible || status[b] != 0) {
        for (int i = tid; i < rec_len; i += blockDim.x) out[i] = 0.0f;
        return;
    }
    // template adjoints gF | gZ | gMu | gPh: one copy per warp in the
    // reproducible mode (lanes add in a fixed order, copies are summed in warp
    // order at the end), else one copy updated with shared-memory atomics
    const int alen = 4 * (n_fp + 1);
    const int ncopy = lay.det ? kBwdBlock / 32 : 1;
    float *adj = sm + lay.adj;
    float *red = sm + lay.red;  // 4 ring sums per warp
    for (int i = tid; i < ncopy * alen; i += blockDim.x) adj[i] = 0.0f;
    {
        const float *tsrc = tmpl + (size_t)ring * 4 * (n_fp + 1);
        for (int i = tid; i < 4 * (n_fp + 1); i += blockDim.x) sm[lay.tmpl + i] = tsrc[i];
        const float *esrc = elems + (size_t)ip.elem0 + (size_t)(ring - ip.ring0) * ip.n_phi;
        for (int i = tid; i < rec.n_active; i += blockDim.x) sm[lay.elems + i] = esrc[i];
        for (int i = tid; i < nEpad; i += blockDim.x) {
            sm[lay.pk + i] = EMIS == 1 ? en.pk[i] : en.E[i];
            if (EMIS == 0) sm[lay.E3 + i] = en.E3[i];
        }
        if (EMIS == 1) {
            for (int i = tid; i < A.nmu; i += blockDim.x) sm[lay.munodes + i] = A.mu[i];
            const int plane = A.nmu * A.nE;
            const float *I0 = A.I + ((size_t)rec.iT * A.ng + rec.ig) * plane;
            const int Pm = A.nmu_pad;
            for (int idx = tid; idx < plane; idx += blockDim.x) {
                // the forward slab (the forward's stencil weights) and its
                // derivatives with respect to logT and logg
                float v = 0.0f, vT = 0.0f, vG = 0.0f;
                const RingRec *rp = recs + ring;  // stencil weights (read in place)
                for (int a = 0; a < rec.tT; ++a)
                    for (int c = 0; c < rec.tg; ++c) {
                        const float I = __ldg(I0 + ((size_t)a * A.ng + c) * plane + idx);
                        v = fmaf(rp->wT[a] * rp->wg[c], I, v);
                        vT = fmaf(rp->dwT[a] * rp->wg[c], I, vT);
                        vG = fmaf(rp->wT[a] * rp->dwg[c], I, vG);
                    }
                const int m = idx / A.nE, n = idx - m * A.nE;
                const int o = n * Pm + m;
                sm[lay.slab + o] = v;
                sm[lay.slabT + o] = vT;
                sm[lay.slabG + o] = vG;
            }
            if (NODES)
                for (int i = tid; i < kBwdMargin * Pm; i += blockDim.x) {
                    sm[lay.slab + A.nE * Pm + i] = 0.0f;
                    sm[lay.slabT + A.nE * Pm + i] = 0.0f;
                    sm[lay.slabG + A.nE * Pm + i] = 0.0f;
                }
        }
    }
    __syncthreads();

    int top = 1;
    while (top * 2 <= n_fp) top *= 2;
    // point samples q = 0 .. n_phase n_sub - 1 at (q - (S - 1)/2) / (n_phase S);
    // each carries 1/S of its output phase's adjoint
    const float inv_nphase = 1.0f / (float)(ip.n_phase * ip.n_sub);
    const float q_half = 0.5f * (float)(ip.n_sub - 1);
    const float inv_sub = 1.0f / (float)ip.n_sub;
    const int n_q = ip.n_phase * ip.n_sub;
    const float inv_dlnE = EMIS == 1 ? (float)(1.0 / A.dlnE) : 0.0f;
    const int Pm = A.nmu_pad;
    const int offT = lay.slabT - lay.slab, offG = lay.slabG - lay.slab;
    const float *ph = sm + lay.tmpl;
    const float *mun = sm + lay.munodes;
    const float *sel = sm + lay.elems;
    const float *S = sm + lay.slab;
    const float *spk = sm + lay.pk;  // table positions (atmosphere) or energies (blackbody)
    const float *sE3 = sm + lay.E3;
    // (table position or energy, adjoint) pairs; the node-major walk keeps the
    // padded adjoints apad instead
    float *arow = sm + lay.arow + warp * arow_len(nEpad);
    float *apad = arow;
    const float2 *parow = reinterpret_cast<const float2 *>(arow);
    const float d = en.step;
    const float pk0 = spk[0], pkl = spk[nE - 1];
    const float lz_safe = 1.25f - pk0;
    const bool sliding = en.sliding != 0;
    const bool onesided = A.strategy == kInterpA || A.strategy == kInterpB;
    const int n_act = rec.n_active;
    const float s_ref = sel[0];
    const float inv_kT = 1.0f / rec.kT;
    const float Kbb = (float)(2.0 / (kH_KEVS * kH_KEVS * kH_KEVS * kC_CM * kC_CM));
    float *adjw = adj + (lay.det ? warp * alen : 0);
    float *gF = adjw, *gZ = adjw + (n_fp + 1), *gM = adjw + 2 * (n_fp + 1), *gP = adjw + 3 * (n_fp + 1);
    float lane_gs = 0.0f, lane_gss = 0.0f, lane_T = 0.0f, lane_G = 0.0f;

    for (int j = warp; j < n_q; j += kBwdBlock / 32) {
        const float *asrc = Aadj + (size_t)(ip.row0 + j / ip.n_sub) * nEpad;
        if (NODES) {
            // apad[kApadLead + k] = A_k, zero outside 0 <= k < nE
            for (int i = lane; i < nE + kApadLead + kApadTail; i += 32) {
                const int k = i - kApadLead;
                apad[i] = (k >= 0 && k < nE) ? asrc[k] * inv_sub : 0.0f;
            }
        } else {
            for (int k = lane; k < nEpad; k += 32) {
                arow[2 * k] = spk[k];
                arow[2 * k + 1] = asrc[k] * inv_sub;
            }
        }
        __syncwarp();
        const float phi_out = ((float)j - q_half) * inv_nphase;
        for (int g0 = 0; g0 < n_act; g0 += 32) {
            const int m = g0 + lane;
            const bool on = m < n_act;
            const float s = on ? sel[m] : 0.0f;
            const PairB P = pair_bwd<EMIS == 1>(on, s, phi_out, ph, mun, n_fp, top, A, inv_dlnE);
            float gFp = 0.f, gzp = 0.f, gmp = 0.f;
            if constexpr (EMIS == 1) {
                const bool fast = P.on && sliding && (pk0 + P.lz >= 1.0f) &&
                                  (pkl + P.lz < (float)(A.nE - 2));
                const bool anyslow = __any_sync(kFull, P.on && !fast);
                float sF = 0.f, sZ = 0.f, sMu = 0.f, sT = 0.f, sG = 0.f;
                if (sliding && !anyslow && NODES) {
                    // node-major walk (energy grid uniform in ln E, step d of
                    // 0.34-0.498 node): every lane moves one table interval per
                    // iteration and takes the two or three energies in it; the
                    // adjoints of virtual energies (before 0, past nE - 1) are
                    // the zeros padding apad.  Strategy B forms the interval
                    // cubics from half-scaled nodes (see cubic_half2), packed as
                    // (I, I_mu) and (I_T, I_g); the others use node weights
                    // and a deferred mu contraction (below).
                    const float lz = fast ? P.lz : lz_safe;
                    const float hw0 = fast ? 0.5f * P.w0 : 0.f, hw1 = fast ? 0.5f * P.w1 : 0.f;
                    const float hw2 = fast ? 0.5f * P.w2 : 0.f, hw3 = fast ? 0.5f * P.w3 : 0.f;
                    const float hv0 = fast ? 0.5f * P.v0 : 0.f, hv1 = fast ? 0.5f * P.v1 : 0.f;
                    const float hv2 = fast ? 0.5f * P.v2 : 0.f, hv3 = fast ? 0.5f * P.v3 : 0.f;
                    const float2 WI0 = make_float2(hw0, hv0), WI1 = make_float2(hw1, hv1);
                    const float2 WI2 = make_float2(hw2, hv2), WI3 = make_float2(hw3, hv3);
                    const float2 WT0 = make_float2(hw0, hw0), WT1 = make_float2(hw1, hw1);
                    const float2 WT2 = make_float2(hw2, hw2), WT3 = make_float2(hw3, hw3);
                    const float x0 = pk0 + lz;
                    const float n0 = floorf(x0);
                    const float f = x0 - n0;
                    int mv = (int)(f * en.inv_step);
                    float t = fmaf(-(float)mv, d, f);
                    if (t >= d) { t -= d; ++mv; }
                    if (t < 0.0f) { t += d; --mv; }
                    int kidx = kApadLead - mv;  // apad index of the energy at t
                    const int i0 = (int)n0;
                    const int s0 = fast ? P.s0 : 0;
                    const float *sp = S + (i0 + 2) * Pm + s0;
                    PPM_CHECK(i0 >= 1 && i0 + 2 <= A.nE - 1 && s0 + 3 < A.nmu, plan.err);
                    auto nodeIM = [&](const float *r) {
                        float2 y = __fmul2_rn(WI0, make_float2(r[0], r[0]));
                        y = __ffma2_rn(WI1, make_float2(r[1], r[1]), y);
                        y = __ffma2_rn(WI2, make_float2(r[2], r[2]), y);
                        return __ffma2_rn(WI3, make_float2(r[3], r[3]), y);
                    };
                    auto nodeTG = [&](const float *r) {
                        const float *rt = r + offT, *rg = r + offG;
                        float2 y = __fmul2_rn(WT0, make_float2(rt[0], rg[0]));
                        y = __ffma2_rn(WT1, make_float2(rt[1], rg[1]), y);
                        y = __ffma2_rn(WT2, make_float2(rt[2], rg[2]), y);
                        return __ffma2_rn(WT3, make_float2(rt[3], rg[3]), y);
                    };
                    int nit = __reduce_max_sync(kFull, (int)floorf(pkl + lz) - i0 + 1) + 1;
                    float2 sFM = make_float2(0.f, 0.f), sTG = make_float2(0.f, 0.f);
                    float sZa = 0.f;
                    if constexpr (CLIP) {
                        // strategy B: the clip decision needs each energy's
                        // intensity, so the interval cubics are evaluated
                        float2 ia = nodeIM(sp - 2 * Pm), ib = nodeIM(sp - Pm), ic = nodeIM(sp);
                        float2 ga = nodeTG(sp - 2 * Pm), gb = nodeTG(sp - Pm), gc = nodeTG(sp);
                        float2 I0, I1, I2, I3, G0, G1, G2, G3;
                        cubic_half2(nodeIM(sp - 3 * Pm), ia, ib, ic, I0, I1, I2, I3);
                        cubic_half2(nodeTG(sp - 3 * Pm), ga, gb, gc, G0, G1, G2, G3);
                        // one energy at position te with adjoint ae
                        auto eval = [&](float te, float ae) {
                            const float2 tt = make_float2(te, te);
                            const float2 vIM = horner2(I0, I1, I2, I3, tt);
                            const float2 vTG = horner2(G0, G1, G2, G3, tt);
                            // max(I, 0) passes no derivative where I <= 0
                            const float a1 = vIM.x > 0.0f ? ae : 0.0f;
                            const float2 ak = make_float2(a1, a1);
                            sFM = __ffma2_rn(ak, vIM, sFM);
                            sTG = __ffma2_rn(ak, vTG, sTG);
                            const float dIdt =
                                fmaf(te, fmaf(te, 3.0f * I3.x, 2.0f * I2.x), I1.x);
                            sZa = fmaf(a1, dIdt, sZa);
                        };
                        // one interval with half nodes (xa, xb, xc) = n, n+1, n+2 of
                        // both pairs; leaves xa = node n + 3 and the next coefficients
                        auto interval = [&](float2 &ja, float2 &jb, float2 &jc, float2 &ka,
                                            float2 &kb, float2 &kc) {
                            const float t2 = t + d, t3 = t2 + d;
                            const float a1 = apad[kidx], a2 = apad[kidx + 1],
                                        a3r = apad[kidx + 2];
                            const bool th = t3 < 1.0f;
                            eval(t, a1);
                            eval(t2, a2);
                            eval(t3, th ? a3r : 0.0f);
                            kidx += th ? 3 : 2;
                            t = (th ? t3 + d : t3) - 1.0f;
                            // node n + 3 (past the last interval: margin rows, zero adjoints)
                            sp += Pm;
                            PPM_CHECK(sp + 3 < S + (A.nE + kBwdMargin) * Pm, plan.err);
                            const float2 yI = nodeIM(sp), yG = nodeTG(sp);
                            cubic_half2(ja, jb, jc, yI, I0, I1, I2, I3);
                            cubic_half2(ka, kb, kc, yG, G0, G1, G2, G3);
                            ja = yI;
                            ka = yG;
                        };
                        for (int n3 = nit / 3; n3 > 0; --n3) {
                            interval(ia, ib, ic, ga, gb, gc);
                            interval(ib, ic, ia, gb, gc, ga);
                            interval(ic, ia, ib, gc, ga, gb);
                        }
                        const int rem = nit % 3;
                        if (rem > 0) interval(ia, ib, ic, ga, gb, gc);
                        if (rem > 1) interval(ib, ic, ia, gb, gc, ga);
                    } else {
                        // No cubic is formed.  The sums over an interval's energies,
                        //   sum_k a_k p(t_k) and sum_k a_k p'(t_k),
                        // are linear in the interval's four node values y_{n-1..n+2},
                        // with weights from the adjoint-weighted moments
                        // m_j = sum_k a_k t_k^j (j = 0..3) through the constant map
                        // from the 4-point cubic's nodes to its power basis
                        // (c0 = y1, c1 = -y0/3 - y1/2 + y2 - y3/6,
                        // c2 = y0/2 - y1 + y2/2, c3 = (y3 - y0)/6 + (y1 - y2)/2);
                        // W and D below are twice those weights.  A node's weights
                        // are summed over the four intervals that use it; when it
                        // leaves the window its total weights multiply its raw
                        // slab rows (all four mu rows of the stencil), and the
                        // element's mu weights contract the accumulated rows once
                        // at the end: the intensity and its mu derivative share
                        // the accumulation.
                        float2 P0 = make_float2(0.f, 0.f), P1 = P0, P2 = P0, P3 = P0;
                        float2 V0 = P0, V1 = P0, V2 = P0, V3 = P0;  // (sum W S, sum D S) per mu row
                        float2 U0 = P0, U1 = P0, U2 = P0, U3 = P0;  // (sum W S_T, sum W S_G)
                        const float *sq = sp - 3 * Pm;              // row of node n - 1
                        // node with total weights X = (W, D) at row r leaves the window
                        auto retire = [&](const float *r, float2 X) {
                            const float *rt = r + offT, *rg = r + offG;
                            const float2 XW = make_float2(X.x, X.x);
                            V0 = __ffma2_rn(X, make_float2(r[0], r[0]), V0);
                            V1 = __ffma2_rn(X, make_float2(r[1], r[1]), V1);
                            V2 = __ffma2_rn(X, make_float2(r[2], r[2]), V2);
                            V3 = __ffma2_rn(X, make_float2(r[3], r[3]), V3);
                            U0 = __ffma2_rn(XW, make_float2(rt[0], rg[0]), U0);
                            U1 = __ffma2_rn(XW, make_float2(rt[1], rg[1]), U1);
                            U2 = __ffma2_rn(XW, make_float2(rt[2], rg[2]), U2);
                            U3 = __ffma2_rn(XW, make_float2(rt[3], rg[3]), U3);
                        };
                        // interval n: partial weights (X0..X3) of nodes n - 1 .. n + 2;
                        // node n - 1 retires and X0 restarts as node n + 3
                        auto interval = [&](float2 &X0, float2 &X1, float2 &X2, float2 &X3) {
                            const float t2 = t + d, t3 = t2 + d;
                            const float a1 = apad[kidx], a2 = apad[kidx + 1],
                                        a3r = apad[kidx + 2];
                            const bool th = t3 < 1.0f;
                            const float a3 = th ? a3r : 0.0f;
                            const float b1 = a1 * (t * t), b2 = a2 * (t2 * t2), b3 = a3 * (t3 * t3);
                            const float m0 = a1 + a2 + a3;
                            const float m1 = fmaf(a1, t, fmaf(a2, t2, a3 * t3));
                            const float m2 = b1 + b2 + b3;
                            const float m3 = fmaf(b1, t, fmaf(b2, t2, b3 * t3));
                            X0 = __fadd2_rn(X0, make_float2(fmaf(m1, -2.0f / 3.0f, fmaf(m3, -1.0f / 3.0f, m2)),
                                                            fmaf(m0, -2.0f / 3.0f, fmaf(m1, 2.0f, -m2))));
                            X1 = __fadd2_rn(X1, make_float2(fmaf(m0 - m2, 2.0f, m3 - m1),
                                                            fmaf(m2, 3.0f, fmaf(m1, -4.0f, -m0))));
                            X2 = __fadd2_rn(X2, make_float2(fmaf(m1, 2.0f, m2 - m3),
                                                            fmaf(m0 + m1, 2.0f, -3.0f * m2)));
                            X3 = __fadd2_rn(X3, make_float2((m3 - m1) * (1.0f / 3.0f),
                                                            fmaf(m0, -1.0f / 3.0f, m2)));
                            kidx += th ? 3 : 2;
                            t = (th ? t3 + d : t3) - 1.0f;
                            PPM_CHECK(sq >= S && sq + 3 < S + (A.nE + kBwdMargin) * Pm, plan.err);
                            retire(sq, X0);
                            sq += Pm;
                            X0 = make_float2(0.f, 0.f);
                        };
                        for (int n4 = nit / 4; n4 > 0; --n4) {
                            interval(P0, P1, P2, P3);
                            interval(P1, P2, P3, P0);
                            interval(P2, P3, P0, P1);
                            interval(P3, P0, P1, P2);
                        }
                        const int rem = nit % 4;
                        // the last three nodes of the window retire after the walk
                        if (rem == 0) {
                            retire(sq, P0); retire(sq + Pm, P1); retire(sq + 2 * Pm, P2);
                        } else if (rem == 1) {
                            interval(P0, P1, P2, P3);
                            retire(sq, P1); retire(sq + Pm, P2); retire(sq + 2 * Pm, P3);
                        } else if (rem == 2) {
                            interval(P0, P1, P2, P3);
                            interval(P1, P2, P3, P0);
                            retire(sq, P2); retire(sq + Pm, P3); retire(sq + 2 * Pm, P0);
                        } else {
                            interval(P0, P1, P2, P3);
                            interval(P1, P2, P3, P0);
                            interval(P2, P3, P0, P1);
                            retire(sq, P3); retire(sq + Pm, P0); retire(sq + 2 * Pm, P1);
                        }
                        // contract the accumulated mu rows with the element's mu
                        // weights (halved: W and D are twice the weights)
                        const float hw0 = fast ? 0.5f * P.w0 : 0.f, hw1 = fast ? 0.5f * P.w1 : 0.f;
                        const float hw2 = fast ? 0.5f * P.w2 : 0.f, hw3 = fast ? 0.5f * P.w3 : 0.f;
                        const float hv0 = fast ? 0.5f * P.v0 : 0.f, hv1 = fast ? 0.5f * P.v1 : 0.f;
                        const float hv2 = fast ? 0.5f * P.v2 : 0.f, hv3 = fast ? 0.5f * P.v3 : 0.f;
                        sFM = make_float2(fmaf(hw0, V0.x, fmaf(hw1, V1.x, fmaf(hw2, V2.x, hw3 * V3.x))),
                                          fmaf(hv0, V0.x, fmaf(hv1, V1.x, fmaf(hv2, V2.x, hv3 * V3.x))));
                        sTG = make_float2(fmaf(hw0, U0.x, fmaf(hw1, U1.x, fmaf(hw2, U2.x, hw3 * U3.x))),
                                          fmaf(hw0, U0.y, fmaf(hw1, U1.y, fmaf(hw2, U2.y, hw3 * U3.y))));
                        sZa = fmaf(hw0, V0.y, fmaf(hw1, V1.y, fmaf(hw2, V2.y, hw3 * V3.y)));
                    }
                    sF = sFM.x;
                    sMu = sFM.y;
                    sT = sTG.x;
                    sG = sTG.y;
                    sZ = sZa;
                } else if (sliding && !anyslow) {
                    // lanes without a pair run the window with zero weights
                    const float lz = fast ? P.lz : lz_safe;
                    const float a0 = fast ? P.w0 : 0.f, a1 = fast ? P.w1 : 0.f;
                    const float a2 = fast ? P.w2 : 0.f, a3 = fast ? P.w3 : 0.f;
                    const float b0 = fast ? P.v0 : 0.f, b1 = fast ? P.v1 : 0.f;
                    const float b2 = fast ? P.v2 : 0.f, b3 = fast ? P.v3 : 0.f;
                    const float q = floorf(pk0 + lz);
                    float off = lz - q;
                    const float *sp = S + ((int)q + 2) * Pm + P.s0;
                    PPM_CHECK(sp - 3 * Pm >= S && sp + 3 < S + A.nE * Pm, plan.err);
                    // (I, I_mu) and (I_T, I_g) as packed pairs: one FFMA2 chain each
                    auto nodeIM = [&](const float *r) {
                        return make_float2(dot4(r, a0, a1, a2, a3), dot4(r, b0, b1, b2, b3));
                    };
                    auto nodeTG = [&](const float *r) {
                        return make_float2(dot4(r + offT, a0, a1, a2, a3), dot4(r + offG, a0, a1, a2, a3));
                    };
                    Cubic2 cIM, cTG;
                    cubic2_set(cIM, nodeIM(sp - 3 * Pm), nodeIM(sp - 2 * Pm), nodeIM(sp - Pm), nodeIM(sp));
                    cubic2_set(cTG, nodeTG(sp - 3 * Pm), nodeTG(sp - 2 * Pm), nodeTG(sp - Pm), nodeTG(sp));
                    float d1 = 2.0f * cIM.c2.x, d2 = 3.0f * cIM.c3.x;  // dI/dt coefficients
                    float2 sFM = make_float2(0.f, 0.f), sTG = make_float2(0.f, 0.f);
                    float sZa = 0.f;
                    const float2 *pa = parow;
#pragma unroll 2
                    for (int k = 0; k < nE; ++k) {
                        const float2 pka = pa[k];  // (table position, adjoint)
                        float t = pka.x + off;
                        if (t >= 1.0f) {
                            sp += Pm;
                            PPM_CHECK(sp + 3 < S + A.nE * Pm, plan.err);
                            cubic2_shift(cIM, nodeIM(sp));
                            cubic2_shift(cTG, nodeTG(sp));
                            d1 = 2.0f * cIM.c2.x;
                            d2 = 3.0f * cIM.c3.x;
                            off -= 1.0f;
                            t -= 1.0f;
                        }
                        const float2 tt = make_float2(t, t);
                        const float2 vIM = horner2(cIM, tt), vTG = horner2(cTG, tt);
                        // strategy B: max(I, 0) passes no derivative where I <= 0
                        const float a1 = CLIP ? (vIM.x > 0.0f ? pka.y : 0.0f) : pka.y;
                        const float2 ak = make_float2(a1, a1);
                        sFM = __ffma2_rn(ak, vIM, sFM);
                        sTG = __ffma2_rn(ak, vTG, sTG);
                        sZa = fmaf(a1, fmaf(t, fmaf(t, d2, d1), cIM.c1.x), sZa);
                    }
                    sF = sFM.x;
                    sMu = sFM.y;
                    sT = sTG.x;
                    sG = sTG.y;
                    sZ = sZa;
                } else if (P.on) {
                    for (int k = 0; k < nE; ++k) {
                        const Quint Q = bwd_general(P, S, S + offT, S + offG, Pm, A.nE,
                                                    spk[k] + P.lz, onesided);
                        // the adjoint row holds padded adjoints in the node-major kernel
                        const float ar = NODES ? apad[kApadLead + k] : parow[k].y;
                        const float ak = CLIP ? (Q.I > 0.0f ? ar : 0.0f) : ar;
                        sF = fmaf(ak, Q.I, sF);
                        sZ = fmaf(ak, Q.dI, sZ);
                        sMu = fmaf(ak, Q.Im, sMu);
                        sT = fmaf(ak, Q.It, sT);
                        sG = fmaf(ak, Q.Ig, sG);
                    }
                }
                if (P.on) {
                    gFp = sF;
                    gzp = P.Fp * sZ * inv_dlnE / P.zp;
                    gmp = P.Fp * sMu;
                    lane_T = fmaf(P.Fp, sT, lane_T);
                    lane_G = fmaf(P.Fp, sG, lane_G);
                }
            } else {
                // analytic isotropic blackbody: C_k = F_p K z^3 E^3 / expm1(x), x = z E / kT;
                // dC/dz = C (3 - r) / z and dC/dkT = C r / kT with r = x e^x / expm1(x)
                if (__any_sync(kFull, P.on) && P.on) {
                    const float bz = Kbb * P.zp * P.zp * P.zp, az = P.zp * inv_kT;
                    float sF = 0.f, sR = 0.f;
                    for (int k = 0; k < nE; ++k) {
                        const float x = az * spk[k];
                        const float em = expm1f(x);
                        const float I0 = bz * sE3[k] / em;
                        const float r = x * (1.0f + 1.0f / em);
                        const float ak = parow[k].y;
                        sF = fmaf(ak, I0, sF);
                        sR = fmaf(ak, I0 * r, sR);
                    }
                    gFp = sF;
                    gzp = P.Fp * (3.0f * sF - sR) / P.zp;
                    lane_T = fmaf(P.Fp, sR * inv_kT, lane_T);
                }
            }
            // the pair's contributions to the template adjoints at points i, i + 1
            float vF0 = 0.f, vF1 = 0.f, vZ0 = 0.f, vZ1 = 0.f, vM0 = 0.f, vM1 = 0.f;
            float vP0 = 0.f, vP1 = 0.f;
            if (P.on) {
                PPM_CHECK(P.i >= 0 && P.i + 1 <= n_fp, plan.err);
                const float w = P.w, u = 1.0f - w;
                vF0 = gFp * u; vF1 = gFp * w;
                vZ0 = gzp * u; vZ1 = gzp * w;
                vM0 = gmp * u; vM1 = gmp * w;
                if (P.dphi > 0.0f) {
                    // phi_p = phi_out + s (mod 1); w = (phi_p - phi_o[i]) / (phi_o[i+1] - phi_o[i])
                    const float gw = gFp * P.dF + gzp * P.dZ + gmp * P.dM;
                    const float gwd = gw / P.dphi;
                    vP0 = gwd * (w - 1.0f);
                    vP1 = -gwd * w;
                    lane_gs += gwd;
                    lane_gss = fmaf(gwd, s - s_ref, lane_gss);
                }
            }
            if (lay.det) {
                // lanes in increasing order into the warp's own copy
                unsigned todo = __ballot_sync(kFull, P.on);
                while (todo) {
                    const int l = __ffs(todo) - 1;
                    todo &= todo - 1;
                    if (lane == l) {
                        gF[P.i] += vF0; gF[P.i + 1] += vF1;
                        gZ[P.i] += vZ0; gZ[P.i + 1] += vZ1;
                        gM[P.i] += vM0; gM[P.i + 1] += vM1;
                        gP[P.i] += vP0; gP[P.i + 1] += vP1;
                    }
                    __syncwarp();
                }
            } else if (P.on) {
                atomicAdd(&gF[P.i], vF0);
                atomicAdd(&gF[P.i + 1], vF1);
                atomicAdd(&gZ[P.i], vZ0);
                atomicAdd(&gZ[P.i + 1], vZ1);
                if (EMIS == 1) {
                    atomicAdd(&gM[P.i], vM0);
                    atomicAdd(&gM[P.i + 1], vM1);
                }
                if (P.dphi > 0.0f) {
                    atomicAdd(&gP[P.i], vP0);
                    atomicAdd(&gP[P.i + 1], vP1);
                }
            }
        }
        __syncwarp();
    }
    // ring sums
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        lane_gs += __shfl_xor_sync(kFull, lane_gs, o);
        lane_gss += __shfl_xor_sync(kFull, lane_gss, o);
        lane_T += __shfl_xor_sync(kFull, lane_T, o);
        lane_G += __shfl_xor_sync(kFull, lane_G, o);
    }
    if (lane == 0) {
        red[4 * warp + 0] = lane_gs;
        red[4 * warp + 1] = lane_gss;
        red[4 * warp + 2] = lane_T;
        red[4 * warp + 3] = lane_G;
    }
    __syncthreads();
    for (int i = tid; i < alen; i += blockDim.x) {
        float v = adj[i];
        for (int c = 1; c < ncopy; ++c) v += adj[c * alen + i];
        out[i] = v;
    }
    if (tid < kRingAdjTail) {
        float v = tid == 4 ? s_ref : 0.0f;
        if (tid < 4) {
            v = 0.0f;
            for (int w = 0; w < kBwdBlock / 32; ++w) v += red[4 * w + tid];
        }
        out[alen + tid] = v;
    }
}

struct BwdSizes {
    BLayout lay;
    size_t bytes;
};

BwdSizes bwd_layout(int emission, const PlanDev &plan, const AtmDev &A, const EnergyDev &en,
                    int n_phi_max, bool det = false)
{
    BwdSizes z;
    BLayout &lay = z.lay;
    int off = 0;
    auto take = [&](int n) { int o = off; off += (n + 3) & ~3; return o; };
    const int slab = emission == 1 ? (A.nE + (en.step > 0.0f ? kBwdMargin : 0)) * A.nmu_pad : 0;
    lay.tmpl = take(4 * (plan.n_fp + 1));
    lay.elems = take(n_phi_max);
    lay.munodes = take(emission == 1 ? A.nmu : 0);
    lay.pk = take(en.nEpad);
    lay.E3 = take(emission == 1 ? 0 : en.nEpad);
    lay.arow = take((kBwdBlock / 32) * arow_len(en.nEpad));
    lay.adj = take((det ? kBwdBlock / 32 : 1) * 4 * (plan.n_fp + 1));
    lay.red = take(4 * (kBwdBlock / 32));
    lay.slab = take(slab);
    lay.slabT = take(slab);
    lay.slabG = take(slab);
    lay.total = off;
    lay.det = det ? 1 : 0;
    z.bytes = (size_t)off * sizeof(float);
    return z;
}

}  // namespace

size_t shift_add_bwd_smem_bytes(int emission, const PlanDev &plan, const AtmDev &A,
                                const EnergyDev &en, int n_phi_max)
{
    return bwd_layout(emission, plan, A, en, n_phi_max).bytes;
}

cudaError_t launch_shift_add_bwd(const Params &p, const PlanDev &plan, const AtmDev &A,
                                 const EnergyDev &en, const RingRec *recs, const float *tmpl,
                                 const float *elems, const int *status, const float *Aadj,
                                 float *ringadj, int n_phi_max, cudaStream_t st,
                                 size_t smem_limit)
{
    if (plan.total_rings <= 0) return cudaSuccess;
    // the reproducible mode when its per-warp adjoint copies fit in shared memory
    BwdSizes z = bwd_layout(p.emission, plan, A, en, n_phi_max, true);
    if (z.bytes > smem_limit) z = bwd_layout(p.emission, plan, A, en, n_phi_max, false);
    cudaError_t e;
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)z.bytes);
        if (r != cudaSuccess) return r;
        kern<<<plan.total_rings, kBwdBlock, z.bytes, st>>>(p, plan, A, en, z.lay, recs, tmpl,
                                                           elems, status, Aadj, ringadj);
        return cudaSuccess;
    };
    // node-major walk on uniform energy grids (as the forward)
    const bool nodes = p.emission == 1 && en.sliding && en.step > 0.0f;
    const bool clip = A.strategy == kInterpB;
    if (p.emission == 0) e = go(k_shift_add_bwd<0, false, false>);
    else if (nodes && clip) e = go(k_shift_add_bwd<1, true, true>);
    else if (nodes) e = go(k_shift_add_bwd<1, false, true>);
    else if (clip) e = go(k_shift_add_bwd<1, true, false>);
    else e = go(k_shift_add_bwd<1, false, false>);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace ppm
