// Shift-and-add with atmosphere interpolation, FP32 (Sect. 2.8.3, Eq. add_Ft;
// Sect. 4 mixed-order interpolation).
//
// Work item = (instance, spot, ring range, tile of `pt` output phases).  Per
// ring the block stages in shared memory:
//   - the ring's template (phi_o, F, z, mu at n_fp + 1 fine phases),
//   - the compacted azimuths of its active elements,
//   - the atmosphere slab I[E][mu] of the ring, already interpolated
//     linearly in (logT, logg) (transposed: mu fastest, so the four mu rows
//     of a stencil are four consecutive words).
// Each warp owns one output phase at a time; its lanes are 32 elements of
// the ring (neighbouring elements see nearly the same redshift and emission
// angle, so their table reads are broadcast-friendly).  Three walks through
// the observed energies:
//   - moment walk (the default for spots; atm_group_moments): per group of
//     64 elements with a ln z spread below 0.45 table node, the moments
//     sum_p eps_p^j u_p of the elements' node values are contracted once
//     per table node from column weights over the group's mu stencils; each
//     energy evaluates one combined cubic, and energies within the group's
//     spread of a node add exact difference terms for the elements on the
//     far side (listed, then handled eight at a time); other groups take
//     one of the two walks below.
// In those two, each element's mu stencil is contracted once per table
// energy node (4 FMA) and the cubic in ln E of the current node interval is
// kept as power-basis coefficients in registers (packed FP32 pairs of
// elements):
//   - node-major (energy grids uniform in ln E with 0.34-0.498 table node
//     per step): every element of the warp moves one table interval per
//     iteration and evaluates the two or three energies inside it; the
//     values go through a per-warp shared-memory ring and are summed into
//     the phase row in blocks of eight energies (atm_group_nodes);
//   - energy walk (other grids): one observed energy per step for all
//     elements, an interval change per element where its position crosses
//     a node; after each chunk of 16 energies the accumulators are
//     transposed across the warp with 16 shuffles so lane l owns energy l
//     (atm_group).
// No atomics: each item writes its tile to a partial buffer that a second
// kernel sums in a fixed order.
#include <algorithm>

#include "ppm_internal.cuh"

namespace ppm {
namespace {

constexpr unsigned kFull = 0xffffffffu;

struct Layout {
    int tmpl, elems, slab, munodes, pk, E, E3, fblk, ring, total;  // offsets in floats
};

__device__ __forceinline__ float contract4(const float *__restrict__ s, int off, float w0,
                                           float w1, float w2, float w3)
{
    return fmaf(w3, s[off + 3], fmaf(w2, s[off + 2], fmaf(w1, s[off + 1], w0 * s[off])));
}

// 16 accumulators per lane -> lanes l and l ^ 16 receive the warp sum of
// accumulator l & 15
__device__ __forceinline__ float transpose_reduce16(float (&acc)[kEC], int lane)
{
#pragma unroll
    for (int off = 8; off >= 1; off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < off; ++i) {
            const float send = upper ? acc[i] : acc[i + off];
            const float keep = upper ? acc[i + off] : acc[i];
            acc[i] = keep + __shfl_xor_sync(kFull, send, off);
        }
    }
    return acc[0] + __shfl_xor_sync(kFull, acc[0], 16);
}

// 8 accumulators per lane -> lanes l, l ^ 8, l ^ 16, l ^ 24 receive the warp
// sum of accumulator l & 7
__device__ __forceinline__ float transpose_reduce8(float (&acc)[8], int lane)
{
#pragma unroll
    for (int off = 4; off >= 1; off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < off; ++i) {
            const float send = upper ? acc[i] : acc[i + off];
            const float keep = upper ? acc[i + off] : acc[i];
            acc[i] = keep + __shfl_xor_sync(kFull, send, off);
        }
    }
    const float t = acc[0] + __shfl_xor_sync(kFull, acc[0], 8);
    return t + __shfl_xor_sync(kFull, t, 16);
}

// Template value at observed phase phip (linear in the interval of phi_o
// that holds it: the last lo <= n_fp - 1 with phi_o[lo] <= phip, else 0).
// The fine phases are nearly uniform over one cycle (phi_o = fine phase plus
// a slowly varying time delay), so the search starts at the uniform guess
// and moves by single steps.
__device__ __forceinline__ void template_at(const float *__restrict__ ph, int n_fp, int top,
                                            float phip, float &Fp, float &zp, float &mp)
{
    (void)top;
    const float *F = ph + (n_fp + 1), *Z = F + (n_fp + 1), *M = Z + (n_fp + 1);
    int lo = min(max((int)((phip - ph[0]) * (float)n_fp), 0), n_fp - 1);
    while (lo > 0 && ph[lo] > phip) --lo;
    while (lo + 1 <= n_fp - 1 && ph[lo + 1] <= phip) ++lo;
    float w = (phip - ph[lo]) / (ph[lo + 1] - ph[lo]);
    w = fminf(fmaxf(w, 0.0f), 1.0f);
    Fp = fmaf(F[lo + 1] - F[lo], w, F[lo]);
    zp = fmaf(Z[lo + 1] - Z[lo], w, Z[lo]);
    mp = fmaf(M[lo + 1] - M[lo], w, M[lo]);
}

// Interpolation weights of one (element, output phase) pair.
struct PairW {
    float w0, w1, w2, w3;  // mu stencil weights times F_p
    int s0;                // first mu row of the stencil
    float lz;              // ln(z_p) / dlnE_table
    bool on;               // contributes (active element, visible phase)
};

template <bool ONESIDED>
__device__ __forceinline__ PairW pair_weights(bool on, float s, float phi_out, const float *ph,
                                              const float *mun, int n_fp, int top,
                                              const AtmDev &A, float inv_dlnE)
{
    PairW P;
    P.w0 = P.w1 = P.w2 = P.w3 = 0.0f;
    P.s0 = 0;
    P.lz = 0.0f;
    P.on = false;
    if (!on) return P;
    const float x = phi_out + s + 1.0f - ph[0];
    const float phip = x - floorf(x) + ph[0];
    float Fp, zp, mp;
    template_at(ph, n_fp, top, phip, Fp, zp, mp);
    if (!(Fp != 0.0f && zp > 0.0f && zp < 1e30f)) return P;
    const int nmu = A.nmu;
    // mu: clamp, interval (the last i <= nmu - 2 with mu_i <= mu: from the
    // bin's entry by single steps), mixed-order weights (Sect. 4)
    const float mu = fminf(fmaxf(mp, mun[0]), mun[nmu - 1]);
    int i = __ldg(A.mu_idx + min(max((int)((mu - mun[0]) * A.mu_bin), 0), kMuBins - 1));
    while (i > 0 && mun[i] > mu) --i;
    while (i + 1 <= nmu - 2 && mun[i + 1] <= mu) ++i;
    float w[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    int s0;
    // A, B (ONESIDED): cubic on four nodes moved inside the grid; C, D:
    // centred cubic, linear on the protected small-mu intervals and at the edges
    if (ONESIDED || (i >= 1 && i + 2 <= nmu - 1 && i >= A.n_protect - 1)) {
        s0 = ONESIDED ? min(max(i - 1, 0), nmu - 4) : i - 1;
        const float x0 = mun[s0], x1 = mun[s0 + 1], x2 = mun[s0 + 2], x3 = mun[s0 + 3];
        const float4 rd = __ldg(A.mu_rden + s0);  // reciprocal Lagrange denominators
        const float d0 = mu - x0, d1 = mu - x1, d2 = mu - x2, d3 = mu - x3;
        w[0] = d1 * d2 * d3 * rd.x;
        w[1] = d0 * d2 * d3 * rd.y;
        w[2] = d0 * d1 * d3 * rd.z;
        w[3] = d0 * d1 * d2 * rd.w;
    } else {
        s0 = min(max(i - 1, 0), nmu - 4);
        const float t = (mu - mun[i]) * __ldg(A.mu_rlin + i);
        const int o = i - s0;
#pragma unroll
        for (int a = 0; a < 4; ++a) w[a] = (a == o) ? 1.0f - t : ((a == o + 1) ? t : 0.0f);
    }
    P.w0 = w[0] * Fp; P.w1 = w[1] * Fp; P.w2 = w[2] * Fp; P.w3 = w[3] * Fp;
    P.s0 = s0;
    P.lz = logf(zp) * inv_dlnE;
    P.on = true;
    return P;
}

// general evaluation (table edges / clamping) of the contracted spectrum at p
__device__ __noinline__ float eval_general(const PairW &P, const float *slab, int Pm, int nE_t,
                                           float p, bool onesided)
{
    if (p <= 0.0f) return contract4(slab, P.s0, P.w0, P.w1, P.w2, P.w3);
    if (p >= (float)(nE_t - 1))
        return contract4(slab, (nE_t - 1) * Pm + P.s0, P.w0, P.w1, P.w2, P.w3);
    const float q = floorf(p);
    const int qi = (int)q;
    const float t = p - q;
    if (onesided && !(qi >= 1 && qi + 2 <= nE_t - 1)) {
        // cubic on the four nodes s..s+3 inside the grid, evaluated at x = p - s
        const int s = min(max(qi - 1, 0), nE_t - 4);
        const float x = p - (float)s;
        float y[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) y[a] = contract4(slab, (s + a) * Pm + P.s0, P.w0, P.w1, P.w2, P.w3);
        // Lagrange basis on the nodes 0, 1, 2, 3
        const float l0 = -(x - 1.0f) * (x - 2.0f) * (x - 3.0f) * (1.0f / 6.0f);
        const float l1 = x * (x - 2.0f) * (x - 3.0f) * 0.5f;
        const float l2 = -x * (x - 1.0f) * (x - 3.0f) * 0.5f;
        const float l3 = x * (x - 1.0f) * (x - 2.0f) * (1.0f / 6.0f);
        return l0 * y[0] + l1 * y[1] + l2 * y[2] + l3 * y[3];
    }
    if (qi >= 1 && qi + 2 <= nE_t - 1) {
        const float a = contract4(slab, (qi - 1) * Pm + P.s0, P.w0, P.w1, P.w2, P.w3);
        const float b = contract4(slab, qi * Pm + P.s0, P.w0, P.w1, P.w2, P.w3);
        const float c = contract4(slab, (qi + 1) * Pm + P.s0, P.w0, P.w1, P.w2, P.w3);
        const float d = contract4(slab, (qi + 2) * Pm + P.s0, P.w0, P.w1, P.w2, P.w3);
        const float c2 = fmaf(0.5f, a + c, -b);
        const float c3 = fmaf(d - a, 1.0f / 6.0f, 0.5f * (b - c));
        const float c1 = fmaf(c - a, 0.5f, -c3);
        return fmaf(t, fmaf(t, fmaf(t, c3, c2), c1), b);
    }
    const float b = contract4(slab, qi * Pm + P.s0, P.w0, P.w1, P.w2, P.w3);
    const float c = contract4(slab, (qi + 1) * Pm + P.s0, P.w0, P.w1, P.w2, P.w3);
    return fmaf(t, c - b, b);
}

// weights of a pair for the slow path (kept out of line: it is rarely taken)
template <bool ONESIDED>
__device__ __noinline__ PairW pair_weights_slow(float s, float phi_out, const float *ph,
                                                const float *mun, int n_fp, int top,
                                                const AtmDev &A, float inv_dlnE)
{
    return pair_weights<ONESIDED>(true, s, phi_out, ph, mun, n_fp, top, A, inv_dlnE);
}

// dot product of a mu stencil row with its weights (four consecutive words)
__device__ __forceinline__ float dot4(const float *__restrict__ q, float w0, float w1, float w2,
                                      float w3)
{
    return fmaf(w3, q[3], fmaf(w2, q[2], fmaf(w1, q[1], w0 * q[0])));
}

// Slab of a (logT, logg) stencil with tT x tg taps (4 x 4 for the cubic
// strategies A, B, C), transposed to [E][mu]; kept out of line (per ring).
__device__ __noinline__ void stage_slab_stencil(const AtmDev &A, const RingRec *rp,
                                                const float *I0, int plane, int Pm, float *slab,
                                                int tid, int nt)
{
    const int tT = rp->tT, tg = rp->tg;
    for (int idx = tid; idx < plane; idx += nt) {
        float v = 0.0f;
        for (int a = 0; a < tT; ++a)
            for (int c = 0; c < tg; ++c)
                v = fmaf(rp->wT[a] * rp->wg[c], __ldg(I0 + ((size_t)a * A.ng + c) * plane + idx), v);
        const int m = idx / A.nE, n = idx - m * A.nE;
        slab[n * Pm + m] = v;
    }
}

// Slab of a 4 x 4 (logT, logg) stencil (the cubic strategies A, B, C) with
// the 16 plane weights in registers and two words' 16 loads in flight per
// thread; same sums as stage_slab_stencil, kept out of line (per ring).
__device__ __noinline__ void stage_slab_4x4(const AtmDev &A, const RingRec *rp, const float *I0,
                                            int plane, int Pm, float *slab, int tid, int nt)
{
    float wv[16];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) wv[4 * a + c] = rp->wT[a] * rp->wg[c];
    const size_t ps = (size_t)plane;
    const size_t gs = (size_t)A.ng * plane;
    constexpr int U = 2;
    for (int base = tid; base < plane; base += U * nt) {
        float v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + u * nt;
            float acc = 0.0f;
            if (idx < plane) {
                float x[16];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c) x[4 * a + c] = __ldg(I0 + a * gs + c * ps + idx);
#pragma unroll
                for (int q = 0; q < 16; ++q) acc = fmaf(wv[q], x[q], acc);
            }
            v[u] = acc;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + u * nt;
            if (idx < plane) {
                const int m = idx / A.nE, n = idx - m * A.nE;
                slab[n * Pm + m] = v[u];
            }
        }
    }
}

// component e & 1 of a packed pair
#define PPM_C(v, e) (((e) & 1) ? (v)[(e) >> 1].y : (v)[(e) >> 1].x)

// One group of 64 NP elements (lanes x 2 NP slots) at one output phase.
// Slot e of a lane is element g0 + lane + 32 e; slots (2p, 2p+1) are packed
// into float2 registers so the position update, the Horner evaluation and
// the slot sum run as paired FP32 instructions (FADD2/FFMA2).  Interval
// shifts stay per slot: a slot's 32 lanes are neighbouring elements and
// shift together, so the branch is nearly warp-uniform.
// MODE: 0 = centred stencils with the linear rules (strategies C, D);
// 1 = one-sided cubic stencils (A); 2 = one-sided and clipped at zero (B)
template <int NP, int MODE>
__device__ __forceinline__ void atm_group(int g0, int n_act, int lane, float phi_out,
                                          const float *sel, const float *ph, const float *mun,
                                          const float *slab, int Pm, int n_fp, int top,
                                          const AtmDev &A, float inv_dlnE, const float *spk,
                                          int nch, bool sliding, float pk0, float pkl,
                                          float lz_safe, float *frow, unsigned *errp)
{
    constexpr int NS = 2 * NP;
    constexpr bool ONESIDED = MODE != 0, CLIP = MODE == 2;
    float2 w0[NP], w1[NP], w2[NP], w3[NP], c0[NP], c1[NP], c2[NP], c3[NP], W2[NP], W3[NP], off[NP];
    const float *sp[NS];
    bool slow[NS];
    const float nEm2 = (float)(A.nE - 2);
#pragma unroll
    for (int e = 0; e < NS; ++e) {
        const int m = g0 + lane + 32 * e;
        const PairW P = pair_weights<ONESIDED>(m < n_act, m < n_act ? sel[m] : 0.0f, phi_out, ph,
                                               mun, n_fp, top, A, inv_dlnE);
        const bool fast = P.on && sliding && (pk0 + P.lz >= 1.0f) && (pkl + P.lz < nEm2);
        slow[e] = P.on && !fast;
        // lanes outside the sliding window run it with zero weights
        const float lz = fast ? P.lz : lz_safe;
        const float q = floorf(pk0 + lz);
        const float a0 = fast ? P.w0 : 0.0f, a1 = fast ? P.w1 : 0.0f;
        const float a2 = fast ? P.w2 : 0.0f, a3 = fast ? P.w3 : 0.0f;
        PPM_C(w0, e) = a0; PPM_C(w1, e) = a1; PPM_C(w2, e) = a2; PPM_C(w3, e) = a3;
        PPM_C(off, e) = lz - q;
        sp[e] = slab + ((int)q + 2) * Pm + P.s0;
        PPM_CHECK(sp[e] - 3 * Pm >= slab && sp[e] + 3 < slab + A.nE * Pm && P.s0 + 3 < A.nmu,
                  errp);
        const float na = dot4(sp[e] - 3 * Pm, a0, a1, a2, a3);
        const float nb = dot4(sp[e] - 2 * Pm, a0, a1, a2, a3);
        const float nc = dot4(sp[e] - Pm, a0, a1, a2, a3);
        const float nd = dot4(sp[e], a0, a1, a2, a3);
        PPM_C(c0, e) = nb;
        PPM_C(c2, e) = fmaf(0.5f, na + nc, -nb);
        PPM_C(c3, e) = fmaf(nd - na, 1.0f / 6.0f, 0.5f * (nb - nc));
        PPM_C(c1, e) = fmaf(nc - na, 0.5f, -PPM_C(c3, e));
        PPM_C(W2, e) = nc;
        PPM_C(W3, e) = nd;
    }
    bool anyslow = false;
#pragma unroll
    for (int e = 0; e < NS; ++e) anyslow |= slow[e];
    anyslow = __any_sync(kFull, anyslow);

    for (int c = 0; c < nch; ++c) {
        float acc[kEC];
        const float *pkc = spk + c * kEC;
#pragma unroll
        for (int s = 0; s < kEC; ++s) acc[s] = 0.0f;
        // the window walk is only in bounds when the host enabled sliding
        if (sliding) {
#pragma unroll
        for (int s = 0; s < kEC; ++s) {
            const float pk = pkc[s];
            float2 t[NP];
#pragma unroll
            for (int p = 0; p < NP; ++p) t[p] = __fadd2_rn(make_float2(pk, pk), off[p]);
#pragma unroll
            for (int e = 0; e < NS; ++e) {
                if (PPM_C(t, e) >= 1.0f) {
                    sp[e] += Pm;
                    PPM_CHECK(sp[e] + 3 < slab + A.nE * Pm, errp);
                    const float d = dot4(sp[e], PPM_C(w0, e), PPM_C(w1, e), PPM_C(w2, e),
                                         PPM_C(w3, e));
                    const float a = PPM_C(c0, e), b = PPM_C(W2, e), cc = PPM_C(W3, e);
                    PPM_C(c0, e) = b;
                    PPM_C(c2, e) = fmaf(0.5f, a + cc, -b);
                    const float k3 = fmaf(d - a, 1.0f / 6.0f, 0.5f * (b - cc));
                    PPM_C(c3, e) = k3;
                    PPM_C(c1, e) = fmaf(cc - a, 0.5f, -k3);
                    PPM_C(W2, e) = cc;
                    PPM_C(W3, e) = d;
                    PPM_C(off, e) -= 1.0f;
                    PPM_C(t, e) -= 1.0f;
                }
            }
            float2 v[NP];
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                v[p] = __ffma2_rn(t[p], __ffma2_rn(t[p], __ffma2_rn(t[p], c3[p], c2[p]), c1[p]),
                                  c0[p]);
                // strategy B: F_p >= 0, so clipping F_p I clips I
                if (CLIP) v[p] = make_float2(fmaxf(v[p].x, 0.0f), fmaxf(v[p].y, 0.0f));
            }
            if (NP == 2) {
                const float2 u = __fadd2_rn(v[0], v[NP - 1]);
                acc[s] = u.x + u.y;
            } else {
                acc[s] = v[0].x + v[0].y;
            }
        }
        }
        if (anyslow) {
#pragma unroll
            for (int e = 0; e < NS; ++e) {
                if (slow[e]) {
                    const int m = g0 + lane + 32 * e;
                    const PairW P = pair_weights_slow<ONESIDED>(sel[m], phi_out, ph, mun, n_fp, top,
                                                                A, inv_dlnE);
#pragma unroll
                    for (int k = 0; k < kEC; ++k) {
                        const float v = eval_general(P, slab, Pm, A.nE, pkc[k] + P.lz, ONESIDED);
                        acc[k] += CLIP ? fmaxf(v, 0.0f) : v;
                    }
                }
            }
        }
        const float tot = transpose_reduce16(acc, lane);
        if (lane < kEC) frow[c * kEC + lane] += tot;
    }
}
#undef PPM_C

// ---------------------------------------------------------------------------
// Node-major walk (energy grids uniform in ln E with a step d of 1/3 to 1/2
// table node; en.step > 0).  Two elements per lane, packed in float2 (slot
// 0: element g0 + lane, slot 1: g0 + lane + 32).  Each iteration moves every
// slot one table interval up in ln E: it evaluates the interval's cubic at
// the observed energies inside it (positions t and t + d always, t + 2d when
// it is below 1), then contracts the next node and rebuilds the power-basis
// coefficients.  Every slot does the same work in every iteration, so the
// interval change is no longer a divergent branch.
//
// After i iterations a slot has passed ceil((i - f) / d) energies (f its
// fractional start), so two slots differ by at most three energies.  Each
// slot stores its values in its own column of a ring of 16 energy rows
// (row = energy mod 16); once every slot of the warp has passed a block of
// 8 energies the warp sums the block's rows (fixed order) into the phase
// row.  A slot starts with up to two virtual energies below energy 0 in its
// first interval and may run up to five past the last one: their rows are
// rewritten by real energies before they are summed, or have been summed
// already, or lie beyond nE.
// ---------------------------------------------------------------------------
constexpr int kRingRows = 16;
constexpr int kRingBlock = 8;
constexpr int kRingWarpBytes = kRingRows * 64 * 4;  // 64 columns of FP32 per row
constexpr int kSlabMargin = 3;  // rows past the table read by slots past their last interval

// the node-major walk applies (atmosphere emission, uniform energy step)
static bool node_walk(const Params &p, const EnergyDev &en)
{
    return p.emission == 1 && en.sliding && en.step > 0.0f;
}

// the moment walk applies (the host asked for it; spot emission from the
// table with an interpolant linear in the table values)
static bool moment_walk(const Params &p, const AtmDev &A, const EnergyDev &en)
{
    return p.emission == 1 && !p.logT_map && en.moments && en.sliding && A.strategy != kInterpB;
}

// rings of the block's warps plus the slack that aligns them to 4096 bytes
static int ring_floats(int warps = kSABlock / 32) { return (warps * kRingWarpBytes + 4096) / 4; }

__device__ __forceinline__ void ring_put(unsigned kk, unsigned colbase, float v)
{
    // row (kk >> 8) & 15 of the ring; colbase has no bits in 0xF00
    asm volatile("st.shared.f32 [%0], %1;" ::"r"((kk & 0xF00u) | colbase), "f"(v));
}

template <bool CLIP>
__device__ __forceinline__ float2 horner2(float2 t, float2 k0, float2 k1, float2 k2, float2 k3)
{
    float2 v = __ffma2_rn(t, __ffma2_rn(t, __ffma2_rn(t, k3, k2), k1), k0);
    // strategy B: F_p >= 0, so clipping F_p I clips I
    if (CLIP) v = make_float2(fmaxf(v.x, 0.0f), fmaxf(v.y, 0.0f));
    return v;
}

// 16 bytes of the ring at shared address a.  The ring is only touched by
// these volatile loads and ring_put's volatile stores, which keep their
// program order; __syncwarp orders the lanes.
__device__ __forceinline__ float4 ring_get4(unsigned a)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(a));
    return v;
}

// MAP: temperature-map elements of one logT cell; a node is contracted
// against the cell's two slabs (slab: lower logT node, slab2: upper) with
// the mu weights scaled by 1 - w and w, w = wcell[m] the element's own
// weight of the upper node.
template <int MODE, bool MAP = false>
__device__ __forceinline__ void atm_group_nodes(int g0, int n_act, int lane, float phi_out,
                                                const float *sel, const float *ph,
                                                const float *mun, const float *slab, int Pm,
                                                int n_fp, int top, const AtmDev &A,
                                                float inv_dlnE, const float *spk, int nE,
                                                int nch, float d, float inv_d, float pk0,
                                                float pkl, float lz_safe, unsigned ring,
                                                float *frow, unsigned *errp,
                                                const float *slab2 = nullptr,
                                                const float *wcell = nullptr)
{
    constexpr bool ONESIDED = MODE != 0, CLIP = MODE == 2;
    const float nEm2 = (float)(A.nE - 2);
    float tv[2], wv[2][4], wb[2][4], uv[2][4];
    unsigned kkv[2];
    int ofv[2], nit = 0;
    bool slow[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int m = g0 + lane + 32 * e;
        const PairW P = pair_weights<ONESIDED>(m < n_act, m < n_act ? sel[m] : 0.0f, phi_out, ph,
                                               mun, n_fp, top, A, inv_dlnE);
        const bool fast = P.on && (pk0 + P.lz >= 1.0f) && (pkl + P.lz < nEm2);
        slow[e] = P.on && !fast;
        // slots outside the window run the walk with zero weights
        const float lz = fast ? P.lz : lz_safe;
        const float x0 = pk0 + lz;
        const float n0 = floorf(x0);
        const float f = x0 - n0;
        // virtual energies -mv .. -1 put the walk's start t in [0, d)
        int mv = (int)(f * inv_d);
        float t = fmaf(-(float)mv, d, f);
        if (t >= d) { t -= d; ++mv; }
        if (t < 0.0f) { t += d; --mv; }
        tv[e] = t;
        kkv[e] = (unsigned)(-mv) << 8;
        const int i0 = (int)n0;
        nit = max(nit, (int)floorf(pkl + lz) - i0 + 1);
        const int s0 = fast ? P.s0 : 0;
        ofv[e] = (i0 + 2) * Pm + s0;
        // half weights: the walk carries u = y / 2 (see cubic_half2)
        const float wT = MAP ? (m < n_act ? wcell[m] : 0.0f) : 0.0f;
        const float fa = MAP ? 1.0f - wT : 1.0f;
        wv[e][0] = fast ? 0.5f * P.w0 * fa : 0.0f;
        wv[e][1] = fast ? 0.5f * P.w1 * fa : 0.0f;
        wv[e][2] = fast ? 0.5f * P.w2 * fa : 0.0f;
        wv[e][3] = fast ? 0.5f * P.w3 * fa : 0.0f;
        wb[e][0] = (MAP && fast) ? 0.5f * P.w0 * wT : 0.0f;
        wb[e][1] = (MAP && fast) ? 0.5f * P.w1 * wT : 0.0f;
        wb[e][2] = (MAP && fast) ? 0.5f * P.w2 * wT : 0.0f;
        wb[e][3] = (MAP && fast) ? 0.5f * P.w3 * wT : 0.0f;
        PPM_CHECK(i0 >= 1 && i0 + 2 <= A.nE - 1 && s0 + 3 < A.nmu, errp);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uv[e][q] = dot4(slab + (i0 - 1 + q) * Pm + s0, wv[e][0], wv[e][1], wv[e][2], wv[e][3]);
            if (MAP)
                uv[e][q] += dot4(slab2 + (i0 - 1 + q) * Pm + s0, wb[e][0], wb[e][1], wb[e][2],
                                 wb[e][3]);
        }
    }
    // one iteration more than the intervals of the last energy: the walk's
    // positions are accumulated and may cross the last node slightly late
    nit = __reduce_max_sync(kFull, nit) + 1;
    const float2 W0 = make_float2(wv[0][0], wv[1][0]), W1 = make_float2(wv[0][1], wv[1][1]);
    const float2 W2 = make_float2(wv[0][2], wv[1][2]), W3 = make_float2(wv[0][3], wv[1][3]);
    const float2 B0 = make_float2(wb[0][0], wb[1][0]), B1 = make_float2(wb[0][1], wb[1][1]);
    const float2 B2 = make_float2(wb[0][2], wb[1][2]), B3 = make_float2(wb[0][3], wb[1][3]);
    float2 a = make_float2(uv[0][1], uv[1][1]);
    float2 b = make_float2(uv[0][2], uv[1][2]);
    float2 c = make_float2(uv[0][3], uv[1][3]);
    float2 K0, K1, K2, K3;
    cubic_half2(make_float2(uv[0][0], uv[1][0]), a, b, c, K0, K1, K2, K3);
    float2 t = make_float2(tv[0], tv[1]);
    const float2 d2 = make_float2(d, d), m1 = make_float2(-1.0f, -1.0f);
    unsigned kk0 = kkv[0], kk1 = kkv[1];
    int of0 = ofv[0], of1 = ofv[1];
    const unsigned cb0 = ring + 4u * lane, cb1 = ring + 128u + 4u * lane;
    // lane (row rr = lane >> 2, quarter q = lane & 3) of a block sum adds the
    // float4 columns q + 4 ((i + rr) & 3), i = 0 .. 3 (no bank conflicts)
    const int rr = lane >> 2, qq = lane & 3;
    unsigned fa[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) fa[i] = ring + 256u * rr + 16u * (qq + 4 * ((i + rr) & 3));
    int r0 = 0;                       // first energy of the ring block not yet summed
    int lim = kRingBlock << 8;        // (r0 + 8) << 8

    // sum energies r0 .. r0 + 7 (rows r0 & 15 ..) into the phase row
    auto flush = [&]() {
        __syncwarp();
        float4 v[4];
        // rows 8-15 for odd blocks (fa[i] < ring + 2048, so the OR adds)
        const unsigned hi = ((unsigned)r0 & 8u) << 8;
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = ring_get4(fa[i] | hi);
        float2 s01 = __fadd2_rn(__fadd2_rn(make_float2(v[0].x, v[0].y), make_float2(v[0].z, v[0].w)),
                                __fadd2_rn(make_float2(v[1].x, v[1].y), make_float2(v[1].z, v[1].w)));
        float2 s23 = __fadd2_rn(__fadd2_rn(make_float2(v[2].x, v[2].y), make_float2(v[2].z, v[2].w)),
                                __fadd2_rn(make_float2(v[3].x, v[3].y), make_float2(v[3].z, v[3].w)));
        s01 = __fadd2_rn(s01, s23);
        float tot = s01.x + s01.y;
        tot += __shfl_xor_sync(kFull, tot, 1);
        tot += __shfl_xor_sync(kFull, tot, 2);
        const int k = r0 + rr;
        if (qq == 0 && k < nE) frow[k] += tot;
        __syncwarp();
        r0 += kRingBlock;
        lim += kRingBlock << 8;
    };

    // one interval: A0, A1, A2 = half values of nodes n, n + 1, n + 2 and
    // K0..K3 the interval's coefficients.  Leaves A0 = node n + 3 and K0..K3
    // of interval n + 1, so the next call takes (A1, A2, A0).
    auto interval = [&](float2 &A0, float2 &A1, float2 &A2) {
        // node n + 3, loaded first so the loads overlap the evaluations (slots
        // past their last interval read the margin rows; those values only
        // reach virtual energies)
        of0 += Pm;
        of1 += Pm;
        PPM_CHECK(of0 + 3 < (A.nE + kSlabMargin) * Pm && of1 + 3 < (A.nE + kSlabMargin) * Pm,
                  errp);
        const float *q0 = slab + of0, *q1 = slab + of1;
        const float2 r0v = make_float2(q0[0], q1[0]), r1v = make_float2(q0[1], q1[1]);
        const float2 r2v = make_float2(q0[2], q1[2]), r3v = make_float2(q0[3], q1[3]);
        float2 s0v, s1v, s2v, s3v;
        if (MAP) {
            const float *p0 = slab2 + of0, *p1 = slab2 + of1;
            s0v = make_float2(p0[0], p1[0]);
            s1v = make_float2(p0[1], p1[1]);
            s2v = make_float2(p0[2], p1[2]);
            s3v = make_float2(p0[3], p1[3]);
        }
        const float2 t2 = __fadd2_rn(t, d2);
        const float2 t3 = __fadd2_rn(t2, d2);
        const float2 v1 = horner2<CLIP>(t, K0, K1, K2, K3);
        const float2 v2 = horner2<CLIP>(t2, K0, K1, K2, K3);
        const float2 v3 = horner2<CLIP>(t3, K0, K1, K2, K3);
        const bool th0 = t3.x < 1.0f, th1 = t3.y < 1.0f;
        const unsigned k3a = kk0 + 512u, k3b = kk1 + 512u;
        ring_put(kk0, cb0, v1.x);
        ring_put(kk1, cb1, v1.y);
        ring_put(kk0 + 256u, cb0, v2.x);
        ring_put(kk1 + 256u, cb1, v2.y);
        if (th0) ring_put(k3a, cb0, v3.x);
        if (th1) ring_put(k3b, cb1, v3.y);
        kk0 = th0 ? k3a + 256u : k3a;
        kk1 = th1 ? k3b + 256u : k3b;
        t = __fadd2_rn(t3, m1);
        if (th0) t.x += d;
        if (th1) t.y += d;
        float2 y = __fmul2_rn(W0, r0v);
        y = __ffma2_rn(W1, r1v, y);
        y = __ffma2_rn(W2, r2v, y);
        y = __ffma2_rn(W3, r3v, y);
        if (MAP) {
            y = __ffma2_rn(B0, s0v, y);
            y = __ffma2_rn(B1, s1v, y);
            y = __ffma2_rn(B2, s2v, y);
            y = __ffma2_rn(B3, s3v, y);
        }
        cubic_half2(A0, A1, A2, y, K0, K1, K2, K3);
        A0 = y;
    };
    // Checked every second interval: when a check finds the slowest slot
    // below r0 + 8, the next two intervals write at most energy r0 + 15
    // (slots differ by three, an interval adds three), inside the ring, and
    // leave the slowest slot below r0 + 16, so one block sum per check keeps
    // up.  kk may start "negative" (virtual energies): compare as signed.
    auto passed = [&]() {
        if (__all_sync(kFull, min((int)kk0, (int)kk1) >= lim)) flush();
    };
    // six intervals per trip (the node roles rotate with period three), then
    // the remainder
    for (int n6 = nit / 6; n6 > 0; --n6) {
        interval(a, b, c);
        interval(b, c, a);
        passed();
        interval(c, a, b);
        interval(a, b, c);
        passed();
        interval(b, c, a);
        interval(c, a, b);
        passed();
    }
    const int rem = nit % 6;
    if (rem > 0) {
        interval(a, b, c);
        if (rem > 1) {
            interval(b, c, a);
            passed();
            if (rem > 2) {
                interval(c, a, b);
                if (rem > 3) {
                    interval(a, b, c);
                    passed();
                    if (rem > 4) interval(b, c, a);
                }
            }
        }
    }
    while (r0 < nE) flush();

    // elements whose window leaves the table interior: general evaluation
    // per chunk of 16 energies, summed across the warp like the energy walk
    if (__any_sync(kFull, slow[0] || slow[1])) {
        for (int cc = 0; cc < nch; ++cc) {
            float acc[kEC];
#pragma unroll
            for (int s = 0; s < kEC; ++s) acc[s] = 0.0f;
            const float *pkc = spk + cc * kEC;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                if (slow[e]) {
                    const int m = g0 + lane + 32 * e;
                    const PairW P = pair_weights_slow<ONESIDED>(sel[m], phi_out, ph, mun, n_fp,
                                                                top, A, inv_dlnE);
                    if (MAP) {
                        const float wT = wcell[m];
                        PairW Pa = P, Pb = P;
                        Pa.w0 *= 1.0f - wT; Pa.w1 *= 1.0f - wT; Pa.w2 *= 1.0f - wT; Pa.w3 *= 1.0f - wT;
                        Pb.w0 *= wT; Pb.w1 *= wT; Pb.w2 *= wT; Pb.w3 *= wT;
#pragma unroll
                        for (int k = 0; k < kEC; ++k) {
                            const float pp = pkc[k] + P.lz;
                            acc[k] += eval_general(Pa, slab, Pm, A.nE, pp, false) +
                                      eval_general(Pb, slab2, Pm, A.nE, pp, false);
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < kEC; ++k) {
                            const float v = eval_general(P, slab, Pm, A.nE, pkc[k] + P.lz, ONESIDED);
                            acc[k] += CLIP ? fmaxf(v, 0.0f) : v;
                        }
                    }
                }
            }
            const float tot = transpose_reduce16(acc, lane);
            if (lane < kEC) frow[cc * kEC + lane] += tot;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Moment walk (atmosphere spots; every interpolation strategy whose value is
// linear in the table values, i.e. all but the clipped one).  The 64 slots
// of a group sit at positions X_p + (pk_k - pk_0) in table nodes (X_p =
// pk_0 + ln z_p / dlnE).  With a reference position ref (the midpoint of the
// group's extreme X_p) and a group spread below kMomSpread node, slot p is
// X_p = ref + eps_p with |eps_p| < kMomSpread / 2, and its node values are
// indexed relative to N0 = floor(ref).  On the reference interval r of an
// energy (its reference position N0 + r + tau, tau in [0, 1)) the cubic of
// slot p at tau + eps_p expands in powers of tau with coefficients linear in
// eps_p^j u_p, so the group's sum needs only the four moments
//   M_j[m] = sum_p eps_p^j u_p[m],   u_p[m] = sum_i w_pi S[N0 + m][s_p + i]
// of each relative node m (S the staged slab, w_pi the mu stencil weights
// times F_p).  The slots of a group are neighbouring elements whose
// stencils cover a few mu columns, so M_j[m] = sum_c Omega_j[c] S[N0 + m][c]
// with the column weights Omega_j summed once per group: the walk is one
// short dot product per node and moment instead of one stencil per slot and
// node.  From M_j[r - 1 .. r + 2] each reference interval gets one combined
// cubic in tau, exact for every slot whose own position tau + eps_p stays in
// [0, 1); a slot that crossed into the next (previous) interval adds the
// difference of the two cubics, the fourth difference of its node values on
// r - 1 .. r + 3 times t (t - 1) (t - 2) / 6 at t = tau + eps_p (on r - 2 ..
// r + 2 times -(t + 1) t (t - 1) / 6).  Energies that can need such terms
// lie within max |eps| of a node, a fraction of about the spread.  Groups
// with a wider spread, or stencils over more than kMomCells columns, are
// left to the node-major walk (uniform grids) or the energy walk.
// ---------------------------------------------------------------------------
constexpr int kMomLead = 2;         // zero rows below the table (relative node -2)
constexpr int kMomCells = 32;       // mu columns of one group's stencils
constexpr float kMomSpread = 0.45f; // widest ln z spread of a group, in table nodes
constexpr int kMomBatch = 8;        // candidate energies whose difference terms run together
constexpr int kCandCap = 4 * (kMomCells + 4);  // candidates listed per group
// per warp, three regions:
//   R0: moments, then combined cubics, of the group's relative nodes
//       [nmom] float4; afterwards the fourth-difference rows and positions of
//       a batch of candidates [kMomBatch][ncol] + [kMomBatch];
//   R1: column weights [kMomCells + 4] float4; afterwards the list of
//       candidate energies [kCandCap];
//   R2: a small batch area [2 kMomCells] + [kMomBatch] (a full list is
//       emptied during the pass over the energies, while R0 still holds
//       the cubics)
__host__ __device__ inline int mom_r0_floats(int nmom)
{
    const int a = 4 * nmom, b = kMomBatch * kMomCells + kMomBatch;
    return a > b ? a : b;
}
__host__ __device__ inline int mom_warp_floats(int nmom)
{
    return mom_r0_floats(nmom) + 4 * (kMomCells + 4) + 2 * kMomCells + kMomBatch;
}
// bytes per warp of the moment kernel's buffers: the moment buffers and the
// node-major walk's ring share them (a group takes one walk or the other),
// in 4096-byte aligned slots
__host__ __device__ inline int mom_slot_bytes(int nmom)
{
    const int b = 4 * mom_warp_floats(nmom);
    return ((b > kRingWarpBytes ? b : kRingWarpBytes) + 4095) / 4096 * 4096;
}

// power-basis coefficients of the cubic through y0..y3 at -1, 0, 1, 2
__device__ __forceinline__ float4 cubic_coefs(float y0, float y1, float y2, float y3)
{
    const float c2 = fmaf(0.5f, y0 + y2, -y1);
    const float c3 = fmaf(y3 - y0, 1.0f / 6.0f, 0.5f * (y1 - y2));
    const float c1 = fmaf(y2 - y0, 0.5f, -c3);
    return make_float4(y1, c1, c2, c3);
}

__device__ __forceinline__ float4 f4fma(float4 a, float s, float4 c)
{
    return make_float4(fmaf(a.x, s, c.x), fmaf(a.y, s, c.y), fmaf(a.z, s, c.z), fmaf(a.w, s, c.w));
}

// combined cubic of a reference interval from the moments of its four
// nodes m[0..3] (relative nodes r - 1 .. r + 2): sum_j c_j(M_j) (tau + eps)^j
// collected by powers of tau
__device__ __forceinline__ float4 combined_cubic(const float4 *m)
{
    const float4 m0 = m[0], m1 = m[1], m2 = m[2], m3 = m[3];
    const float4 a = cubic_coefs(m0.x, m1.x, m2.x, m3.x);   // of M_0
    const float4 b = cubic_coefs(m0.y, m1.y, m2.y, m3.y);   // of M_1
    const float4 c2 = cubic_coefs(m0.z, m1.z, m2.z, m3.z);  // of M_2
    const float4 c3 = cubic_coefs(m0.w, m1.w, m2.w, m3.w);  // of M_3
    return make_float4(a.x + b.y + c2.z + c3.w, fmaf(3.0f, c2.w, fmaf(2.0f, b.z, a.y)),
                       fmaf(3.0f, b.w, a.z), a.w);
}

// weight of stencil entry d (0..3) of a slot, 0 outside
__device__ __forceinline__ float stencil_w(int d, float w0, float w1, float w2, float w3)
{
    float w = d == 0 ? w0 : 0.0f;
    w = d == 1 ? w1 : w;
    w = d == 2 ? w2 : w;
    return d == 3 ? w3 : w;
}

// One group of 64 slots (as atm_group_nodes) by the moment walk; returns
// false, having written nothing, when the group is too wide for it.
template <int MODE>
__device__ __forceinline__ bool atm_group_moments(int g0, int n_act, int lane, float phi_out,
                                                  const float *sel, const float *ph,
                                                  const float *mun, const float *slab, int Pm,
                                                  int n_fp, int top, const AtmDev &A,
                                                  float inv_dlnE, const float *spk, int nE,
                                                  int nch, float pk0, float pkl, int nmom,
                                                  float *wbuf, float *frow, unsigned *errp)
{
    static_assert(MODE != 2, "the clipped interpolant is not linear in the table values");
    constexpr bool ONESIDED = MODE != 0;
    const float nEm2 = (float)(A.nE - 2);
    float X[2], wv[2][4];
    int s0v[2];
    bool fast[2], slow[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int m = g0 + lane + 32 * e;
        const PairW P = pair_weights<ONESIDED>(m < n_act, m < n_act ? sel[m] : 0.0f, phi_out, ph,
                                               mun, n_fp, top, A, inv_dlnE);
        fast[e] = P.on && (pk0 + P.lz >= 1.0f) && (pkl + P.lz < nEm2);
        slow[e] = P.on && !fast[e];
        X[e] = pk0 + P.lz;
        wv[e][0] = fast[e] ? P.w0 : 0.0f;
        wv[e][1] = fast[e] ? P.w1 : 0.0f;
        wv[e][2] = fast[e] ? P.w2 : 0.0f;
        wv[e][3] = fast[e] ? P.w3 : 0.0f;
        s0v[e] = fast[e] ? P.s0 : 0;
    }
    // extreme positions and stencil columns of the group's slots inside the window
    float xmax = fmaxf(fast[0] ? X[0] : -INFINITY, fast[1] ? X[1] : -INFINITY);
    float xmin = fminf(fast[0] ? X[0] : INFINITY, fast[1] ? X[1] : INFINITY);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        xmax = fmaxf(xmax, __shfl_xor_sync(kFull, xmax, o));
        xmin = fminf(xmin, __shfl_xor_sync(kFull, xmin, o));
    }
    const int cmin = __reduce_min_sync(kFull, min(fast[0] ? s0v[0] : INT_MAX, fast[1] ? s0v[1] : INT_MAX));
    const int cmax = __reduce_max_sync(kFull, max(fast[0] ? s0v[0] : INT_MIN, fast[1] ? s0v[1] : INT_MIN));
    const int ncol = cmax - cmin + 4;
    if (xmax >= xmin) {  // some slot of the group is inside the window (warp-uniform)
        const float ref = 0.5f * (xmax + xmin);
        const float nf = floorf(ref);
        const float dref = ref - nf;
        const int N0 = (int)nf;
        const int rmax = (int)floorf(dref + (pkl - pk0));
        PPM_CHECK(rmax + 6 <= nmom, errp);
        if (!(xmax - xmin < kMomSpread) || ncol > kMomCells || rmax + 6 > nmom) return false;
        // |X_p - ref| <= spread / 2 < 1/2: every slot has a_p = 0 and the
        // extreme eps are those of the extreme slots
        const float emax = xmax - ref, emin = xmin - ref;
        const float ev[2] = {fast[0] ? X[0] - ref : 0.0f, fast[1] ? X[1] - ref : 0.0f};
        const int r0f = mom_r0_floats(nmom);
        float4 *Mv = reinterpret_cast<float4 *>(wbuf);                  // R0: [nmom]
        float4 *Om = reinterpret_cast<float4 *>(wbuf + r0f);            // R1: [kMomCells + 4]
        float *Dp = wbuf + r0f + 4 * (kMomCells + 4);                  // R2: [2 kMomCells + kMomBatch]
        int cell0[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) cell0[e] = fast[e] ? s0v[e] - cmin : 0;  // zero weights outside
        const float2 E1 = make_float2(ev[0], ev[1]);
        const float2 E2 = __fmul2_rn(E1, E1);
        const float2 E3 = __fmul2_rn(E2, E1);
        const float2 W0 = make_float2(wv[0][0], wv[1][0]), W1 = make_float2(wv[0][1], wv[1][1]);
        const float2 W2 = make_float2(wv[0][2], wv[1][2]), W3 = make_float2(wv[0][3], wv[1][3]);

        // column weights Omega_j, four columns per pass, summed over the
        // slots in a fixed order (slot sums, then the warp transpose-reduction)
        for (int cb = 0; cb < ncol; cb += 4) {
            float acc[kEC];
#pragma unroll
            for (int qi = 0; qi < 4; ++qi) {
                const int q = cb + qi;
                const float2 W = make_float2(
                    stencil_w(q - cell0[0], wv[0][0], wv[0][1], wv[0][2], wv[0][3]),
                    stencil_w(q - cell0[1], wv[1][0], wv[1][1], wv[1][2], wv[1][3]));
                const float2 v1 = __fmul2_rn(W, E1), v2 = __fmul2_rn(W, E2), v3 = __fmul2_rn(W, E3);
                acc[4 * qi + 0] = W.x + W.y;
                acc[4 * qi + 1] = v1.x + v1.y;
                acc[4 * qi + 2] = v2.x + v2.y;
                acc[4 * qi + 3] = v3.x + v3.y;
            }
            const float tot = transpose_reduce16(acc, lane);
            if (lane < kEC) reinterpret_cast<float *>(Om)[4 * cb + lane] = tot;
        }
        __syncwarp();

        // moments of relative nodes m = -2 .. rmax + 3 (index m + 2), two
        // nodes per lane (m and m + 32): lanes read 32 consecutive rows of
        // one column (odd row pitch: no bank conflicts) and the column
        // weights by broadcast
        const float *sbase = slab + N0 * Pm + cmin;
        for (int m0 = -2; m0 <= rmax + 3; m0 += 64) {
            const int ma = m0 + lane, mb = ma + 32;
            if (ma <= rmax + 3) {
                const bool inb = mb <= rmax + 3;
                float4 acc_a = make_float4(0.0f, 0.0f, 0.0f, 0.0f), acc_b = acc_a;
                const float *ra = sbase + ma * Pm;
                const float *rb = inb ? ra + 32 * Pm : ra;
                PPM_CHECK(N0 + ma >= -kMomLead && N0 + (inb ? mb : ma) < A.nE + kSlabMargin, errp);
#pragma unroll 4
                for (int q = 0; q < ncol; ++q) {
                    const float4 om = Om[q];
                    acc_a = f4fma(om, ra[q], acc_a);
                    acc_b = f4fma(om, rb[q], acc_b);
                }
                Mv[ma + 2] = acc_a;
                if (inb) Mv[mb + 2] = acc_b;
            }
        }
        __syncwarp();
        // combined cubic of reference interval r (moments of nodes r - 1 .. r + 2,
        // indices r + 1 .. r + 4), written in place at index r + 1, two
        // intervals per lane: a pass reads indices up to 67 past its first
        // and writes 64, which later passes no longer read
        for (int r0 = 0; r0 <= rmax; r0 += 64) {
            const int ra = r0 + lane, rb = ra + 32;
            const float4 Pa = ra <= rmax ? combined_cubic(Mv + ra + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 Pb = rb <= rmax ? combined_cubic(Mv + rb + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
            __syncwarp();
            if (ra <= rmax) Mv[ra + 1] = Pa;
            if (rb <= rmax) Mv[rb + 1] = Pb;
            __syncwarp();
        }

        // energies: one per lane, the combined cubic at tau.  Energies
        // within the group's spread of a node (candidates) also need the
        // difference terms of slots on the far side of the node: they are
        // listed, and their terms are added kMomBatch at a time after the
        // last pass (R0 is free then: the cubics are spent), or during the
        // passes when the list is full (in R2).  A candidate within emax of
        // the node above (tau + emax >= 1) has slots only past that node
        // (|eps| < 1/2 keeps tau + eps > 0), one within -emin of the node
        // below only slots before it, so each needs one row of fourth
        // differences of the group's columns, on relative nodes r - 1 .. r + 3
        // or r - 2 .. r + 2; the terms of a batch are reduced by one
        // transposition and added in candidate order.
        int *clist = reinterpret_cast<int *>(Om);  // R1 (the column weights are spent)
        int nc = 0;
        const float inv_ncol = 1.0f / (float)ncol;
        auto flush = [&](float *Drow, float *tauc, int nbmax) {
            for (int cb = 0; cb < nc; cb += nbmax) {
                const int nb = min(nbmax, nc - cb);
#pragma unroll 2
                for (int q = lane; q < nb * ncol; q += 32) {
                    const int ci = (int)(((float)q + 0.5f) * inv_ncol);
                    const int col = q - ci * ncol;
                    const int kc = clist[cb + ci];
                    const float y = dref + (spk[kc] - pk0);
                    const float rf = floorf(y);
                    const float tau = y - rf;
                    const int base = (int)rf - (tau + emax >= 1.0f ? 1 : 2);
                    const float *c = sbase + base * Pm + col;
                    Drow[ci * ncol + col] =
                        fmaf(6.0f, c[2 * Pm], fmaf(-4.0f, c[Pm] + c[3 * Pm], c[0] + c[4 * Pm]));
                    if (col == 0) tauc[ci] = tau;
                }
                __syncwarp();
                float acc[kMomBatch];
#pragma unroll
                for (int ci = 0; ci < kMomBatch; ++ci) {
                    acc[ci] = 0.0f;
                    if (ci < nb) {
                        // both slots packed, without data-dependent branches
                        // (the candidates interleave): a slot on the near
                        // side gets g = 0, one outside the window has zero
                        // weights.  Past the node above, 6 g = t (t - 1) (t - 2)
                        // = t (t (t - 3) + 2); before the node below,
                        // 6 g = -(t + 1) t (t - 1) = t (1 - t^2)
                        const float tb = tauc[ci];
                        const float2 te = __fadd2_rn(make_float2(tb, tb), E1);
                        const float *D0 = Drow + ci * ncol;
                        const float *Da = D0 + cell0[0], *Db = D0 + cell0[1];
                        float2 dv = __fmul2_rn(W0, make_float2(Da[0], Db[0]));
                        dv = __ffma2_rn(W1, make_float2(Da[1], Db[1]), dv);
                        dv = __ffma2_rn(W2, make_float2(Da[2], Db[2]), dv);
                        dv = __ffma2_rn(W3, make_float2(Da[3], Db[3]), dv);
                        float2 g;
                        if (tb + emax >= 1.0f) {  // warp-uniform
                            const float2 p = __fmul2_rn(te, __ffma2_rn(te, __fadd2_rn(te, make_float2(-3.0f, -3.0f)),
                                                                        make_float2(2.0f, 2.0f)));
                            g = make_float2(te.x >= 1.0f ? p.x : 0.0f, te.y >= 1.0f ? p.y : 0.0f);
                        } else {
                            const float2 p = __fmul2_rn(te, __ffma2_rn(__fmul2_rn(te, make_float2(-1.0f, -1.0f)), te,
                                                                        make_float2(1.0f, 1.0f)));
                            g = make_float2(te.x < 0.0f ? p.x : 0.0f, te.y < 0.0f ? p.y : 0.0f);
                        }
                        const float2 c = __fmul2_rn(g, dv);
                        acc[ci] = c.x + c.y;
                    }
                }
                const float tot = transpose_reduce8(acc, lane) * (1.0f / 6.0f);
                if (lane < nb) frow[clist[cb + lane]] += tot;
                __syncwarp();
            }
            nc = 0;
        };
        for (int k0 = 0; k0 < nE; k0 += 32) {
            const int k = k0 + lane;
            const bool in = k < nE;
            float tau = 0.0f;
            if (in) {
                const float y = dref + (spk[k] - pk0);
                const float rf = floorf(y);
                tau = y - rf;
                const float4 Pv = Mv[(int)rf + 1];
                frow[k] += fmaf(tau, fmaf(tau, fmaf(tau, Pv.w, Pv.z), Pv.y), Pv.x);
            }
            const unsigned cand = __ballot_sync(kFull, in && (tau + emax >= 1.0f || tau + emin < 0.0f));
            if (nc + __popc(cand) > kCandCap) {  // the list is full: its terms now, in R2
                __syncwarp();
                flush(Dp, Dp + 2 * kMomCells, min(kMomBatch, 2 * kMomCells / ncol));
            }
            if (cand & (1u << lane)) clist[nc + __popc(cand & ((1u << lane) - 1u))] = k;
            nc += __popc(cand);
        }
        __syncwarp();
        flush(wbuf, wbuf + kMomBatch * kMomCells, kMomBatch);  // R0: the cubics are spent
        __syncwarp();
    }

    // slots whose window leaves the table interior: general evaluation per
    // chunk of 16 energies, summed across the warp like the energy walk
    if (__any_sync(kFull, slow[0] || slow[1])) {
        for (int cc = 0; cc < nch; ++cc) {
            float acc[kEC];
#pragma unroll
            for (int s = 0; s < kEC; ++s) acc[s] = 0.0f;
            const float *pkc = spk + cc * kEC;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                if (slow[e]) {
                    const int m = g0 + lane + 32 * e;
                    const PairW P = pair_weights_slow<ONESIDED>(sel[m], phi_out, ph, mun, n_fp,
                                                                top, A, inv_dlnE);
#pragma unroll
                    for (int k = 0; k < kEC; ++k)
                        acc[k] += eval_general(P, slab, Pm, A.nE, pkc[k] + P.lz, ONESIDED);
                }
            }
            const float tot = transpose_reduce16(acc, lane);
            if (lane < kEC) frow[cc * kEC + lane] += tot;
        }
        __syncwarp();
    }
    return true;
}

// the walks a group of the moment kernel falls back to (out of line: rare)
template <int MODE>
__device__ __noinline__ void group_nodes_fallback(int g0, int n_act, int lane, float phi_out,
                                                  const float *sel, const float *ph,
                                                  const float *mun, const float *slab, int Pm,
                                                  int n_fp, int top, const AtmDev &A,
                                                  float inv_dlnE, const float *spk, int nE,
                                                  int nch, float d, float inv_d, float pk0,
                                                  float pkl, float lz_safe, unsigned ring,
                                                  float *frow, unsigned *errp)
{
    atm_group_nodes<MODE>(g0, n_act, lane, phi_out, sel, ph, mun, slab, Pm, n_fp, top, A,
                          inv_dlnE, spk, nE, nch, d, inv_d, pk0, pkl, lz_safe, ring, frow, errp);
}

template <int MODE>
__device__ __noinline__ void group_energy_fallback(int g0, int n_act, int lane, float phi_out,
                                                   const float *sel, const float *ph,
                                                   const float *mun, const float *slab, int Pm,
                                                   int n_fp, int top, const AtmDev &A,
                                                   float inv_dlnE, const float *spk, int nch,
                                                   float pk0, float pkl, float lz_safe,
                                                   float *frow, unsigned *errp)
{
    atm_group<1, MODE>(g0, n_act, lane, phi_out, sel, ph, mun, slab, Pm, n_fp, top, A, inv_dlnE,
                       spk, nch, true, pk0, pkl, lz_safe, frow, errp);
}

// WALK: 0 = energy walk, 1 = node-major walk, 2 = moment walk; NT threads
template <int EMIS, int MODE, int WALK, int NT = kSABlock>
__global__ void __launch_bounds__(NT, NT > kSABlock ? 1 : 2)
    k_shift_add(Params p, PlanDev plan, AtmDev A, EnergyDev en, Layout lay,
                const RingRec *__restrict__ recs, const float *__restrict__ tmpl,
                const float *__restrict__ elems, const int *__restrict__ status,
                float *__restrict__ partials)
{
    extern __shared__ float sm[];
    __shared__ int s_next;
    if (WALK == 1)  // rows past the table that the node-major walk may read
        for (int i = threadIdx.x; i < kSlabMargin * A.nmu_pad; i += blockDim.x)
            sm[lay.slab + A.nE * A.nmu_pad + i] = 0.0f;
    if (WALK == 2) {  // rows below and past the table that the moment walk may read
        for (int i = threadIdx.x; i < kMomLead * A.nmu_pad; i += blockDim.x)
            sm[lay.slab - kMomLead * A.nmu_pad + i] = 0.0f;
        for (int i = threadIdx.x; i < kSlabMargin * A.nmu_pad; i += blockDim.x)
            sm[lay.slab + A.nE * A.nmu_pad + i] = 0.0f;
    }
    // static schedule: block b runs item order[b]; persistent schedule
    // (plan.queue): blocks take the next entry of the order from a counter
    for (int slot = blockIdx.x;;) {
    if (plan.queue) {
        __syncthreads();  // the previous item's tile has been written out
        if (threadIdx.x == 0) s_next = atomicAdd(plan.queue, 1);
        __syncthreads();
        slot = s_next;
        if (slot >= plan.n_items) break;
    }
    const int item_id = plan.order ? plan.order[slot] : slot;
    const Item it = plan.items[item_id];
    const InstPlan ip = plan.inst[it.b];
    const int n_fp = plan.n_fp;
    const int pt = plan.pt;
    const int nEpad = en.nEpad;
    const int nch = nEpad / kEC;
    float *Fblk = sm + lay.fblk;
    float *spk = sm + lay.pk;
    float *sE = sm + lay.E;
    float *sE3 = sm + lay.E3;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (int i = tid; i < pt * nEpad; i += blockDim.x) Fblk[i] = 0.0f;
    for (int i = tid; i < nEpad; i += blockDim.x) {
        spk[i] = en.pk[i];
        sE[i] = en.E[i];
        sE3[i] = en.E3[i];
    }
    if (EMIS == 1)
        for (int i = tid; i < A.nmu; i += blockDim.x) sm[lay.munodes + i] = A.mu[i];

    int top = 1;
    while (top * 2 <= n_fp) top *= 2;
    // point sample q of the instance: phase (q - (S - 1)/2) / (n_phase S)
    const float inv_nphase = 1.0f / (float)(ip.n_phase * ip.n_sub);
    const float q_half = 0.5f * (float)(ip.n_sub - 1);
    const float inv_dlnE = (EMIS == 1) ? (float)(1.0 / A.dlnE) : 0.0f;
    const int Pm = A.nmu_pad;
    const bool inst_ok = status[it.b] == 0;
    // this warp's ring (node-major walk; in the moment kernel the slot that
    // the moment buffers and the fallback's ring share): 4096-byte aligned
    // shared address
    unsigned ring_w = 0;
    float *wbuf = nullptr;
    if (WALK != 0) {
        const unsigned slot = WALK == 2 ? (unsigned)mom_slot_bytes(en.nmom) : (unsigned)kRingWarpBytes;
        const unsigned s0 = (unsigned)__cvta_generic_to_shared(sm);
        ring_w = ((s0 + 4u * (unsigned)lay.ring + 4095u) & ~4095u) + (unsigned)warp * slot;
        wbuf = sm + (ring_w - s0) / 4u;
    }

    for (int r = it.r0; r < it.r1 && inst_ok; ++r) {
        const int ring = ip.ring0 + it.spot * ip.n_theta + r;
        // the scalar fields of the ring record (its weight arrays are read in place)
        const RingRec *rp = recs + ring;
        struct { int visible, n_active, iT, ig, tT, tg; float kT; } rec = {
            rp->visible, rp->n_active, rp->iT, rp->ig, rp->tT, rp->tg, rp->kT};
        if (!rec.visible) continue;
        __syncthreads();  // previous ring finished with the staged data
        {
            const float *tsrc = tmpl + (size_t)ring * 4 * (n_fp + 1);
            for (int i = tid; i < 4 * (n_fp + 1); i += blockDim.x) sm[lay.tmpl + i] = tsrc[i];
            const float *esrc = elems + (size_t)ip.elem0 + (size_t)(ring - ip.ring0) * ip.n_phi;
            PPM_CHECK(rec.n_active <= ip.n_phi && ring < plan.total_rings, plan.err);
            for (int i = tid; i < rec.n_active; i += blockDim.x) sm[lay.elems + i] = esrc[i];
            if (EMIS == 1) {
                const int plane = A.nmu * A.nE;
                const float *I0 = A.I + ((size_t)rec.iT * A.ng + rec.ig) * plane;
                PPM_CHECK(rec.iT >= 0 && rec.iT + rec.tT <= A.nT && rec.ig >= 0 &&
                              rec.ig + rec.tg <= A.ng,
                          plan.err);
                const bool lin2 = rec.tT == 2 && rec.tg == 2;
                const float w00 = rp->wT[0] * rp->wg[0], w01 = rp->wT[0] * rp->wg[1];
                const float w10 = rp->wT[1] * rp->wg[0], w11 = rp->wT[1] * rp->wg[1];
                const float *I01 = I0 + plane;
                const float *I10 = I0 + (size_t)A.ng * plane;
                const float *I11 = I10 + plane;
                float *slab = sm + lay.slab;
                constexpr int U = 4;  // loads in flight per thread
                if (lin2) {
                    // (logT, logg) bilinear (strategy D): four planes
                    for (int base = tid; base < plane; base += U * NT) {
                        float v[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const int idx = base + u * NT;
                            v[u] = 0.0f;
                            if (idx < plane)
                                v[u] = w00 * __ldg(I0 + idx) + w01 * __ldg(I01 + idx) +
                                       w10 * __ldg(I10 + idx) + w11 * __ldg(I11 + idx);
                        }
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const int idx = base + u * NT;
                            if (idx < plane) {
                                const int m = idx / A.nE, n = idx - m * A.nE;
                                slab[n * Pm + m] = v[u];
                            }
                        }
                    }
                } else if (rec.tT == 4 && rec.tg == 4) {
                    stage_slab_4x4(A, rp, I0, plane, Pm, slab, tid, NT);
                } else {
                    stage_slab_stencil(A, rp, I0, plane, Pm, slab, tid, NT);
                }
            }
        }
        __syncthreads();

        const int n_act = rec.n_active;
        const float *sel = sm + lay.elems;
        const float *slab = sm + lay.slab;
        const float *ph = sm + lay.tmpl;
        const float *mun = sm + lay.munodes;
        const float pk0 = spk[0], pkl = spk[en.nE - 1];
        const float lz_safe = 1.25f - pk0;
        const bool sliding = en.sliding != 0;

        for (int jl = warp; jl < it.nj; jl += NT / 32) {
            const float phi_out = ((float)(it.j0 + jl) - q_half) * inv_nphase;
            if constexpr (EMIS == 1 && WALK == 2) {
                float *frow = Fblk + jl * nEpad;
                for (int g0 = 0; g0 < n_act; g0 += 64) {
                    if (atm_group_moments<MODE>(g0, n_act, lane, phi_out, sel, ph, mun, slab, Pm,
                                                n_fp, top, A, inv_dlnE, spk, en.nE, nch, pk0, pkl,
                                                en.nmom, wbuf, frow, plan.err))
                        continue;
                    // too wide for the moment walk
                    __syncwarp();
                    if (en.step > 0.0f)
                        group_nodes_fallback<MODE>(g0, n_act, lane, phi_out, sel, ph, mun, slab, Pm,
                                                   n_fp, top, A, inv_dlnE, spk, en.nE, nch,
                                                   en.step, en.inv_step, pk0, pkl, lz_safe,
                                                   ring_w, frow, plan.err);
                    else
                        group_energy_fallback<MODE>(g0, n_act, lane, phi_out, sel, ph, mun, slab,
                                                    Pm, n_fp, top, A, inv_dlnE, spk, nch, pk0,
                                                    pkl, lz_safe, frow, plan.err);
                    __syncwarp();
                }
                continue;
            } else if constexpr (EMIS == 1 && WALK == 1) {
                for (int g0 = 0; g0 < n_act; g0 += 64)
                    atm_group_nodes<MODE>(g0, n_act, lane, phi_out, sel, ph, mun, slab, Pm, n_fp,
                                          top, A, inv_dlnE, spk, en.nE, nch, en.step,
                                          en.inv_step, pk0, pkl, lz_safe, ring_w,
                                          Fblk + jl * nEpad, plan.err);
                continue;
            } else if constexpr (EMIS == 1) {
                for (int g0 = 0; g0 < n_act;) {
                    if (n_act - g0 > 64) {
                        atm_group<2, MODE>(g0, n_act, lane, phi_out, sel, ph, mun, slab, Pm, n_fp, top,
                                     A, inv_dlnE, spk, nch, sliding, pk0, pkl, lz_safe,
                                     Fblk + jl * nEpad, plan.err);
                        g0 += 128;
                    } else {
                        atm_group<1, MODE>(g0, n_act, lane, phi_out, sel, ph, mun, slab, Pm, n_fp, top,
                                     A, inv_dlnE, spk, nch, sliding, pk0, pkl, lz_safe,
                                     Fblk + jl * nEpad, plan.err);
                        g0 += 64;
                    }
                }
                continue;
            } else {
            for (int g0 = 0; g0 < n_act; g0 += 128) {
                {
                    // analytic isotropic blackbody: I(z E) = K z^3 E^3 / expm1(z E / kT); the
                    // 1/E of Eq. add_Ft is applied with the flux scale in the reduction
                    const float K = (float)(2.0 / (kH_KEVS * kH_KEVS * kH_KEVS * kC_CM * kC_CM));
                    const float inv_kT = 1.0f / rec.kT;
                    float az[4], bz[4];
                    bool anyon[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int m = g0 + lane + 32 * e;
                        az[e] = 1.0f;
                        bz[e] = 0.0f;
                        if (m < n_act) {
                            const float x = phi_out + sel[m] + 1.0f - ph[0];
                            const float phip = x - floorf(x) + ph[0];
                            float Fp, zp, mp;
                            template_at(ph, n_fp, top, phip, Fp, zp, mp);
                            if (Fp != 0.0f && zp > 0.0f && zp < 1e30f) {
                                az[e] = zp * inv_kT;
                                bz[e] = Fp * K * zp * zp * zp;
                            }
                        }
                        anyon[e] = __any_sync(kFull, bz[e] != 0.0f);
                    }
                    for (int c = 0; c < nch; ++c) {
                        float acc[kEC];
#pragma unroll
                        for (int s = 0; s < kEC; ++s) acc[s] = 0.0f;
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            if (!anyon[e]) continue;
#pragma unroll
                            for (int s = 0; s < kEC; ++s) {
                                const int k = c * kEC + s;
                                acc[s] += bz[e] * sE3[k] / expm1f(az[e] * sE[k]);
                            }
                        }
                        const float tot = transpose_reduce16(acc, lane);
                        if (lane < kEC) Fblk[jl * nEpad + c * kEC + lane] += tot;
                    }
                }
            }
            }
        }
    }
    __syncthreads();
    float *dst = partials + (size_t)item_id * pt * nEpad;
    for (int i = tid; i < it.nj * nEpad; i += blockDim.x) dst[i] = Fblk[i];
    if (!plan.queue) break;
    }
}

// ---------------------------------------------------------------------------
// Full-surface temperature maps (Sect. 2.6): every element has its own logT.
// For each logT cell used by a ring the two logg-interpolated table planes of
// the cell are staged and an element's spectrum is (1 - w) I_lo + w I_hi with
// its own weight w, i.e. each node is contracted against both planes with the
// mu weights scaled by (1 - w) and w.  The node-major walk (two element slots
// per lane, the map form of atm_group_nodes) runs in NT = 512-thread blocks
// where the two slabs and sixteen rings fit in shared memory: one block per SM
// then keeps 16 warps resident, as two blocks of the spot kernel do.  The
// energy walk takes one element per lane (scalar code).  The analytic
// blackbody uses each element's kT.  Same items, partial tiles and reduction
// as k_shift_add.
// ---------------------------------------------------------------------------
struct MapLayout {
    int tmpl, elems, cs, cw, munodes, slab, slab2, pk, E, E3, fblk, ring, total;
};

template <int EMIS, bool NODES, int NT = kSABlock>
__global__ void __launch_bounds__(NT, 1)
    k_shift_add_map(Params p, PlanDev plan, AtmDev A, EnergyDev en, MapLayout lay,
                    const RingRec *__restrict__ recs, const float *__restrict__ tmpl,
                    const float *__restrict__ elems, const float2 *__restrict__ elemx,
                    const int *__restrict__ status, float *__restrict__ partials)
{
    extern __shared__ float sm[];
    __shared__ int s_wsum[NT / 32], s_cnt;
    if (NODES)  // rows past the table that the node-major walk may read
        for (int i = threadIdx.x; i < kSlabMargin * A.nmu_pad; i += blockDim.x) {
            sm[lay.slab + A.nE * A.nmu_pad + i] = 0.0f;
            sm[lay.slab2 + A.nE * A.nmu_pad + i] = 0.0f;
        }
    // work slot: item, and part (0: each ring's first logT cell, 1: its
    // other cells; one part for the analytic blackbody)
    const int parts = plan.parts, part = (int)blockIdx.x % parts;
    const int item_id = plan.order ? plan.order[blockIdx.x / parts] : (int)blockIdx.x / parts;
    const int slot = item_id * parts + part;
    const Item it = plan.items[item_id];
    const InstPlan ip = plan.inst[it.b];
    const int n_fp = plan.n_fp, pt = plan.pt, nEpad = en.nEpad, nE = en.nE;
    const int nch = nEpad / kEC;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {
        // a slot without work writes no partial tile (the reduction skips it)
        bool work = false;
        if (status[it.b] == 0)
            for (int r = it.r0; r < it.r1 && !work; ++r) {
                const RingRec *rq = recs + ip.ring0 + it.spot * ip.n_theta + r;
                work = rq->visible && (part == 0 || (EMIS == 1 && rq->tT > 1));
            }
        if (!work) {
            if (tid == 0 && plan.used) plan.used[slot] = 0;
            return;
        }
    }
    float *Fblk = sm + lay.fblk;
    float *spk = sm + lay.pk, *sE = sm + lay.E, *sE3 = sm + lay.E3;
    float *cs = sm + lay.cs, *cw = sm + lay.cw;
    for (int i = tid; i < pt * nEpad; i += blockDim.x) Fblk[i] = 0.0f;
    for (int i = tid; i < nEpad; i += blockDim.x) {
        spk[i] = en.pk[i];
        sE[i] = en.E[i];
        sE3[i] = en.E3[i];
    }
    if (EMIS == 1)
        for (int i = tid; i < A.nmu; i += blockDim.x) sm[lay.munodes + i] = A.mu[i];
    int top = 1;
    while (top * 2 <= n_fp) top *= 2;
    const float inv_nphase = 1.0f / (float)(ip.n_phase * ip.n_sub);
    const float q_half = 0.5f * (float)(ip.n_sub - 1);
    const float inv_dlnE = (EMIS == 1) ? (float)(1.0 / A.dlnE) : 0.0f;
    const int Pm = A.nmu_pad;
    const bool inst_ok = status[it.b] == 0;
    const float *ph = sm + lay.tmpl;
    const float *mun = sm + lay.munodes;
    const float *S0 = sm + lay.slab, *S1 = sm + lay.slab2;
    const float pk0 = spk[0], pkl = spk[nE - 1];
    const float lz_safe = 1.25f - pk0;
    const bool sliding = en.sliding != 0;
    // this warp's ring (node-major walk): 4096-byte aligned shared address
    unsigned ring_w = 0;
    if (NODES)
        ring_w = (((unsigned)__cvta_generic_to_shared(sm + lay.ring) + 4095u) & ~4095u) +
                 (unsigned)(warp * kRingWarpBytes);

    for (int r = it.r0; r < it.r1 && inst_ok; ++r) {
        const int ring = ip.ring0 + it.spot * ip.n_theta + r;
        const RingRec *rp = recs + ring;
        if (!rp->visible) continue;
        const int n_act = rp->n_active;
        const size_t e0 = (size_t)ip.elem0 + (size_t)(ring - ip.ring0) * ip.n_phi;
        __syncthreads();
        for (int i = tid; i < 4 * (n_fp + 1); i += blockDim.x)
            sm[lay.tmpl + i] = tmpl[(size_t)ring * 4 * (n_fp + 1) + i];
        // this slot's cells of the ring: the first, or the others
        const int c_lo = EMIS == 1 ? rp->iT : 0, c_n = EMIS == 1 ? rp->tT : 1;
        const int c_a = part == 0 ? c_lo : c_lo + 1, c_b = part == 0 ? c_lo + 1 : c_lo + c_n;
        for (int cell = c_a; cell < c_b; ++cell) {
            __syncthreads();  // previous cell (or ring) done with the staged data
            if (EMIS == 1) {
                // the cell's two logT planes, interpolated linearly in logg
                const int plane = A.nmu * A.nE;
                const float wg0 = rp->wg[0], wg1 = rp->wg[1];
                const float *Ia = A.I + ((size_t)cell * A.ng + rp->ig) * plane;
                const float *Ib = Ia + (size_t)A.ng * plane;
                for (int idx = tid; idx < plane; idx += blockDim.x) {
                    const int m = idx / A.nE, n = idx - m * A.nE;
                    sm[lay.slab + n * Pm + m] = wg0 * __ldg(Ia + idx) + wg1 * __ldg(Ia + plane + idx);
                    sm[lay.slab2 + n * Pm + m] = wg0 * __ldg(Ib + idx) + wg1 * __ldg(Ib + plane + idx);
                }
            }
            // the ring's elements in this cell, in ring order (stable compaction)
            if (tid == 0) s_cnt = 0;
            __syncthreads();
            for (int m0 = 0; m0 < n_act; m0 += blockDim.x) {
                const int m = m0 + tid;
                bool in = false;
                float2 x = make_float2(0.0f, 0.0f);
                if (m < n_act) {
                    x = elemx[e0 + m];
                    in = EMIS == 1 ? __float_as_int(x.y) == cell : true;
                }
                const unsigned bal = __ballot_sync(kFull, in);
                if (lane == 0) s_wsum[warp] = __popc(bal);
                __syncthreads();
                int off = s_cnt;
                for (int w = 0; w < warp; ++w) off += s_wsum[w];
                if (in) {
                    const int slot = off + __popc(bal & ((1u << lane) - 1u));
                    cs[slot] = elems[e0 + m];
                    cw[slot] = x.x;
                }
                __syncthreads();
                if (tid == 0) {
                    int tot = 0;
                    for (int w = 0; w < NT / 32; ++w) tot += s_wsum[w];
                    s_cnt += tot;
                }
                __syncthreads();
            }
            const int cnt = s_cnt;
            for (int jl = warp; jl < it.nj; jl += NT / 32) {
                const float phi_out = ((float)(it.j0 + jl) - q_half) * inv_nphase;
                float *frow = Fblk + jl * nEpad;
                if constexpr (EMIS == 1 && NODES) {
                    for (int g0 = 0; g0 < cnt; g0 += 64)
                        atm_group_nodes<0, true>(g0, cnt, lane, phi_out, cs, ph, mun, S0, Pm, n_fp,
                                                 top, A, inv_dlnE, spk, nE, nch, en.step,
                                                 en.inv_step, pk0, pkl, lz_safe, ring_w, frow,
                                                 plan.err, S1, cw);
                    continue;
                }
                for (int g0 = 0; g0 < cnt; g0 += 32) {
                    const int m = g0 + lane;
                    const bool on = m < cnt;
                    if (EMIS == 1) {
                        const PairW P = pair_weights<false>(on, on ? cs[m] : 0.0f, phi_out, ph,
                                                            mun, n_fp, top, A, inv_dlnE);
                        const float wT = on ? cw[m] : 0.0f;
                        PairW Pa = P, Pb = P;
                        Pa.w0 *= 1.0f - wT; Pa.w1 *= 1.0f - wT; Pa.w2 *= 1.0f - wT; Pa.w3 *= 1.0f - wT;
                        Pb.w0 *= wT; Pb.w1 *= wT; Pb.w2 *= wT; Pb.w3 *= wT;
                        const bool fast = P.on && sliding && (pk0 + P.lz >= 1.0f) &&
                                          (pkl + P.lz < (float)(A.nE - 2));
                        const bool slow = P.on && !fast;
                        const float lz = fast ? P.lz : lz_safe;
                        const float a0 = fast ? Pa.w0 : 0.f, a1 = fast ? Pa.w1 : 0.f;
                        const float a2 = fast ? Pa.w2 : 0.f, a3 = fast ? Pa.w3 : 0.f;
                        const float b0 = fast ? Pb.w0 : 0.f, b1 = fast ? Pb.w1 : 0.f;
                        const float b2 = fast ? Pb.w2 : 0.f, b3 = fast ? Pb.w3 : 0.f;
                        const float q = floorf(pk0 + lz);
                        float off = lz - q;
                        int n = (int)q + 2;  // last node of the window
                        auto node = [&](int nn) {
                            const int o = nn * Pm + P.s0;
                            return dot4(S0 + o, a0, a1, a2, a3) + dot4(S1 + o, b0, b1, b2, b3);
                        };
                        float y0 = node(n - 3), y1 = node(n - 2), y2 = node(n - 1), y3 = node(n);
                        float c0 = y1, c2 = fmaf(0.5f, y0 + y2, -y1);
                        float c3 = fmaf(y3 - y0, 1.0f / 6.0f, 0.5f * (y1 - y2));
                        float c1 = fmaf(y2 - y0, 0.5f, -c3);
                        float W2 = y2, W3 = y3;
                        for (int c = 0; c < nch; ++c) {
                            float acc[kEC];
#pragma unroll
                            for (int k = 0; k < kEC; ++k) acc[k] = 0.0f;
                            if (sliding) {
#pragma unroll
                                for (int k = 0; k < kEC; ++k) {
                                    float t = spk[c * kEC + k] + off;
                                    if (t >= 1.0f) {
                                        ++n;
                                        const float d = node(n), a = c0, bb = W2, cc = W3;
                                        c0 = bb;
                                        c2 = fmaf(0.5f, a + cc, -bb);
                                        c3 = fmaf(d - a, 1.0f / 6.0f, 0.5f * (bb - cc));
                                        c1 = fmaf(cc - a, 0.5f, -c3);
                                        W2 = cc;
                                        W3 = d;
                                        off -= 1.0f;
                                        t -= 1.0f;
                                    }
                                    acc[k] = fmaf(t, fmaf(t, fmaf(t, c3, c2), c1), c0);
                                }
                            }
                            if (__any_sync(kFull, slow) && slow) {
                                for (int k = 0; k < kEC; ++k) {
                                    const float pp = spk[c * kEC + k] + P.lz;
                                    acc[k] += eval_general(Pa, S0, Pm, A.nE, pp, false) +
                                              eval_general(Pb, S1, Pm, A.nE, pp, false);
                                }
                            }
                            const float tot = transpose_reduce16(acc, lane);
                            if (lane < kEC) frow[c * kEC + lane] += tot;
                        }
                    } else {
                        // analytic blackbody with the element's own kT
                        const float K = (float)(2.0 / (kH_KEVS * kH_KEVS * kH_KEVS * kC_CM * kC_CM));
                        float az = 1.0f, bz = 0.0f;
                        if (on) {
                            const float x = phi_out + cs[m] + 1.0f - ph[0];
                            const float phip = x - floorf(x) + ph[0];
                            float Fp, zp, mp;
                            template_at(ph, n_fp, top, phip, Fp, zp, mp);
                            if (Fp != 0.0f && zp > 0.0f && zp < 1e30f) {
                                az = zp / cw[m];
                                bz = Fp * K * zp * zp * zp;
                            }
                        }
                        for (int c = 0; c < nch; ++c) {
                            float acc[kEC];
#pragma unroll
                            for (int k = 0; k < kEC; ++k) {
                                const int kk = c * kEC + k;
                                acc[k] = bz != 0.0f ? bz * sE3[kk] / expm1f(az * sE[kk]) : 0.0f;
                            }
                            const float tot = transpose_reduce16(acc, lane);
                            if (lane < kEC) frow[c * kEC + lane] += tot;
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    float *dst = partials + (size_t)slot * pt * nEpad;
    for (int i = tid; i < it.nj * nEpad; i += blockDim.x) dst[i] = Fblk[i];
    if (tid == 0 && plan.used) plan.used[slot] = 1;
}

MapLayout map_layout(const Params &p, const PlanDev &plan, const AtmDev &A, const EnergyDev &en,
                     int n_phi_max, int nt)
{
    MapLayout lay;
    int off = 0;
    auto take = [&](int n) { int o = off; off += (n + 3) & ~3; return o; };
    const bool nodes = node_walk(p, en);
    const int slab = p.emission == 1 ? (A.nE + (nodes ? kSlabMargin : 0)) * A.nmu_pad : 0;
    lay.tmpl = take(4 * (plan.n_fp + 1));
    lay.elems = 0;
    lay.cs = take(n_phi_max);
    lay.cw = take(n_phi_max);
    lay.munodes = take(p.emission == 1 ? A.nmu : 0);
    lay.slab = take(slab);
    lay.slab2 = take(slab);
    lay.pk = take(en.nEpad);
    lay.E = take(en.nEpad);
    lay.E3 = take(en.nEpad);
    lay.fblk = take(plan.pt * en.nEpad);
    lay.ring = take(nodes ? ring_floats(nt / 32) : 0);
    lay.total = off;
    return lay;
}

// F_t[row][k] = (sum over the work items of (instance, phase tile)) / E_k.
// One block per (row, 128-energy chunk): warp w sums items w, w+8, ... with
// float4 loads, then the 8 warp sums are added in warp order (fixed order, so
// the result does not depend on scheduling).
__global__ void __launch_bounds__(256) k_reduce(PlanDev plan, EnergyDev en,
                                               const float *__restrict__ partials,
                                               const int *__restrict__ status, int total_rows,
                                               float *__restrict__ Ft)
{
    __shared__ float4 red[8][32];
    const int nE = en.nE, nEpad = en.nEpad;
    const int pt = plan.pt;
    const int row = blockIdx.x;
    const int k4 = blockIdx.y * 32 + (threadIdx.x & 31);   // float4 index along energy
    const int warp = threadIdx.x >> 5;
    const int b = find_instance_by_row(plan.inst, plan.B, row);
    const InstPlan ip = plan.inst[b];
    // output phase j gathers its n_sub point samples (rows of one tile)
    const int q0 = (row - ip.row0) * ip.n_sub;
    const int tile = q0 / pt, jl0 = q0 - tile * pt;
    const int2 rng = plan.tile_items[ip.tile0 + tile];
    PPM_CHECK(tile < ip.tiles && rng.x >= 0 && rng.y <= plan.n_items && jl0 + ip.n_sub <= pt,
              plan.err);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    const size_t stride4 = (size_t)pt * nEpad / 4;
    const int n_sub = ip.n_sub;
    if (plan.parts > 1) {
        // several work slots per item (temperature maps): warp w adds the
        // written slots w, w + 8, ... of the tile's items, reading 32 flags
        // per ballot (every lane takes part; the loop bounds are the warp's)
        // and the set ones in increasing slot order
        const bool kin = 4 * k4 < nEpad;
        const float4 *base = reinterpret_cast<const float4 *>(partials + (size_t)jl0 * nEpad) + k4;
        const int lane = threadIdx.x & 31;
        const int s0 = rng.x * plan.parts + warp, s1 = rng.y * plan.parts;
        for (int c = s0; c < s1; c += 8 * 32) {
            const int ql = c + 8 * lane;
            unsigned set = __ballot_sync(0xffffffffu, ql < s1 && plan.used[ql] != 0);
            while (set) {
                const int q = c + 8 * (__ffs(set) - 1);
                set &= set - 1;
                for (int sub = 0; sub < n_sub && kin; ++sub) {
                    const float4 a = base[(size_t)q * stride4 + (size_t)sub * nEpad / 4];
                    acc.x += a.x; acc.y += a.y; acc.z += a.z; acc.w += a.w;
                }
            }
        }
    } else if (4 * k4 < nEpad) {
        const float4 *base = reinterpret_cast<const float4 *>(partials + (size_t)jl0 * nEpad) + k4;
        int i = rng.x + warp;
        for (; i + 8 < rng.y; i += 16) {
            const float4 a = base[(size_t)i * stride4], c = base[(size_t)(i + 8) * stride4];
            acc.x += a.x; acc.y += a.y; acc.z += a.z; acc.w += a.w;
            acc.x += c.x; acc.y += c.y; acc.z += c.z; acc.w += c.w;
        }
        if (i < rng.y) {
            const float4 a = base[(size_t)i * stride4];
            acc.x += a.x; acc.y += a.y; acc.z += a.z; acc.w += a.w;
        }
        // further point samples of the same output phase (phase_sub > 1)
        for (int sub = 1; sub < n_sub; ++sub) {
            const float4 *bs = base + (size_t)sub * nEpad / 4;
            for (int q = rng.x + warp; q < rng.y; q += 8) {
                const float4 a = bs[(size_t)q * stride4];
                acc.x += a.x; acc.y += a.y; acc.z += a.z; acc.w += a.w;
            }
        }
    }
    red[warp][threadIdx.x & 31] = acc;
    __syncthreads();
    if (warp == 0 && 4 * k4 < nEpad) {
        float4 s = red[0][threadIdx.x];
        for (int w = 1; w < 8; ++w) {
            const float4 v = red[w][threadIdx.x];
            s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
        }
        const float sc = (float)(1.0 / kFluxScale) / (float)ip.n_sub;
        const bool ok = status[b] == 0;
        const float vals[4] = {s.x, s.y, s.z, s.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = 4 * k4 + q;
            if (k < nE) Ft[(size_t)row * nE + k] = ok ? vals[q] * en.invE[k] * sc : 0.0f;
        }
    }
}

}  // namespace

namespace {

// walk, block size and shared-memory layout of the spot kernel: the moment
// walk where it applies and its per-warp buffers fit the opt-in limit, else
// the node-major walk (or the energy walk)
struct SpotConfig {
    Layout lay;
    int walk, nt;
};

SpotConfig spot_config(const Params &p, const PlanDev &plan, const AtmDev &A, const EnergyDev &en,
                       int n_phi_max, size_t smem_optin)
{
    auto layout = [&](int walk, int nt) {
        Layout lay;
        int off = 0;
        auto take = [&](int n) { int o = off; off += (n + 3) & ~3; return o; };
        lay.tmpl = take(4 * (plan.n_fp + 1));
        lay.elems = take(n_phi_max);
        lay.munodes = take(p.emission == 1 ? A.nmu : 0);
        take(walk == 2 ? kMomLead * A.nmu_pad : 0);  // zero rows below the slab
        const int margin = walk != 0 ? kSlabMargin : 0;
        lay.slab = take(p.emission == 1 ? (A.nE + margin) * A.nmu_pad : 0);
        lay.pk = take(en.nEpad);
        lay.E = take(en.nEpad);
        lay.E3 = take(en.nEpad);
        lay.fblk = take(plan.pt * en.nEpad);
        lay.ring = take(walk == 2 ? ((nt / 32) * mom_slot_bytes(en.nmom) + 4096) / 4
                                  : (walk == 1 ? ring_floats(nt / 32) : 0));
        lay.total = off;
        return lay;
    };
    SpotConfig c;
    if (moment_walk(p, A, en)) {
        c.walk = 2;
        c.nt = kSABlock;
        c.lay = layout(2, kSABlock);
        if ((size_t)c.lay.total * sizeof(float) + 64 <= smem_optin) return c;
    }
    c.walk = node_walk(p, en) ? 1 : 0;
    c.nt = kSABlock;
    c.lay = layout(c.walk, kSABlock);
    return c;
}

}  // namespace

size_t shift_add_smem_bytes(const Params &p, const PlanDev &plan, const AtmDev &A,
                            const EnergyDev &en, int n_phi_max, size_t smem_optin)
{
    // the 256-thread map layout is the minimum; 512 threads are taken only where they fit
    if (p.logT_map)
        return (size_t)map_layout(p, plan, A, en, n_phi_max, kSABlock).total * sizeof(float);
    return (size_t)spot_config(p, plan, A, en, n_phi_max, smem_optin).lay.total * sizeof(float);
}

cudaError_t launch_shift_add(const Params &p, const PlanDev &plan, const AtmDev &A,
                             const EnergyDev &en, const RingRec *recs, const float *tmpl,
                             const float *elems, const int *status, float *partials,
                             int n_phi_max, cudaStream_t st, int grid_blocks,
                             const float2 *elemx, size_t smem_optin)
{
    if (plan.n_items <= 0) return cudaSuccess;
    if (p.logT_map) {
        // temperature maps: one block per item (the static schedule)
        auto go = [&](auto kern, int nt) -> cudaError_t {
            const MapLayout lay = map_layout(p, plan, A, en, n_phi_max, nt);
            const size_t bytes = (size_t)lay.total * sizeof(float);
            cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)bytes);
            if (r != cudaSuccess) return r;
            kern<<<plan.n_items * plan.parts, nt, bytes, st>>>(p, plan, A, en, lay, recs, tmpl,
                                                               elems, elemx, status, partials);
            return cudaGetLastError();
        };
        if (p.emission == 0) return go(k_shift_add_map<0, false>, kSABlock);
        if (!node_walk(p, en)) return go(k_shift_add_map<1, false>, kSABlock);
        // 512 threads where the layout (with sixteen rings) fits the opt-in limit
        const size_t wide = (size_t)map_layout(p, plan, A, en, n_phi_max, 512).total * sizeof(float);
        const size_t stat = (512 / 32 + 1) * sizeof(int);
        if (wide + stat <= smem_optin) return go(k_shift_add_map<1, true, 512>, 512);
        return go(k_shift_add_map<1, true>, kSABlock);
    }
    const SpotConfig cfg = spot_config(p, plan, A, en, n_phi_max, smem_optin);
    // persistent schedule: the queue counter must start at zero on the stream;
    // grid_blocks counts 256-thread blocks (two per SM)
    if (plan.queue) {
        cudaError_t e0 = cudaMemsetAsync(plan.queue, 0, sizeof(int), st);
        if (e0 != cudaSuccess) return e0;
        grid_blocks = grid_blocks * kSABlock / cfg.nt;
        grid_blocks = std::max(1, std::min(grid_blocks, plan.n_items));
    } else {
        grid_blocks = plan.n_items;
    }
    const Layout lay = cfg.lay;
    const size_t bytes = (size_t)lay.total * sizeof(float);
    cudaError_t e;
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)bytes);
        if (r != cudaSuccess) return r;
        kern<<<grid_blocks, cfg.nt, bytes, st>>>(p, plan, A, en, lay, recs, tmpl, elems, status,
                                                 partials);
        return cudaSuccess;
    };
    const int walk = cfg.walk;
    if (p.emission == 0) e = go(k_shift_add<0, 0, 0>);
    else if (walk == 2 && A.strategy == kInterpA) e = go(k_shift_add<1, 1, 2>);
    else if (walk == 2) e = go(k_shift_add<1, 0, 2>);
    else if (walk == 1 && A.strategy == kInterpA) e = go(k_shift_add<1, 1, 1>);
    else if (walk == 1 && A.strategy == kInterpB) e = go(k_shift_add<1, 2, 1>);
    else if (walk == 1) e = go(k_shift_add<1, 0, 1>);
    else if (A.strategy == kInterpA) e = go(k_shift_add<1, 1, 0>);
    else if (A.strategy == kInterpB) e = go(k_shift_add<1, 2, 0>);
    else e = go(k_shift_add<1, 0, 0>);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_reduce(const PlanDev &plan, const EnergyDev &en, const float *partials,
                          const int *status, int total_rows, float *Ft, cudaStream_t st)
{
    if (total_rows <= 0) return cudaSuccess;
    dim3 grid(total_rows, (en.nEpad / 4 + 31) / 32);
    k_reduce<<<grid, 256, 0, st>>>(plan, en, partials, status, total_rows, Ft);
    return cudaGetLastError();
}

}  // namespace ppm
