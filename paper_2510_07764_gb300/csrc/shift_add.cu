// Shift-and-add with atmosphere interpolation, FP32 (Sect. 2.8.3, Eq. add_Ft;
// Sect. 4 mixed-order interpolation).
//
// Work item = (instance, spot, ring range, tile of kPT output phases).  Per
// ring the block stages in shared memory:
//   - the ring's template (phi_o, F, z, mu at n_fp + 1 fine phases),
//   - the compacted azimuths of its active elements,
//   - the atmosphere slab I[E][mu] of the ring, already interpolated
//     linearly in (logT, logg) (transposed: mu fastest, so the four mu rows
//     of a stencil are four consecutive words).
// Each warp owns one output phase at a time; its lanes are 32 elements of
// the ring (neighbouring elements see nearly the same redshift and emission
// angle, so their table reads are broadcast-friendly and their stencil
// shifts coincide).  A lane holds four elements and 32 energy accumulators:
// for each element the mu stencil is contracted once per table energy node
// (4 FMA) and the cubic in ln E is evaluated per observed energy from a
// sliding window of four contracted nodes kept in registers (Newton form:
// 3 FMA + 3 adds per energy).  After each chunk of 32 energies the 32
// accumulators are transposed across the warp with 31 shuffles so lane l
// owns energy l, and added to the block's phase x energy tile.  No atomics:
// each item writes its tile to a partial buffer that a second kernel sums
// in a fixed order.
#include "ppm_internal.cuh"

namespace ppm {
namespace {

constexpr unsigned kFull = 0xffffffffu;

struct Layout {
    int tmpl, elems, slab, munodes, pk, E, E2, fblk, total;  // offsets in floats
};

__device__ __forceinline__ float contract4(const float *__restrict__ s, int off, float w0,
                                           float w1, float w2, float w3)
{
    return fmaf(w3, s[off + 3], fmaf(w2, s[off + 2], fmaf(w1, s[off + 1], w0 * s[off])));
}

// 32 accumulators per lane -> lane l receives the warp sum of accumulator l
__device__ __forceinline__ float transpose_reduce(float (&acc)[kEC], int lane)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < off; ++i) {
            const float send = upper ? acc[i] : acc[i + off];
            const float keep = upper ? acc[i + off] : acc[i];
            acc[i] = keep + __shfl_xor_sync(kFull, send, off);
        }
    }
    return acc[0];
}

// Template value at observed phase phip (linear, lower-bound search on phi_o).
__device__ __forceinline__ void template_at(const float *__restrict__ ph,
                                            const float *__restrict__ F,
                                            const float *__restrict__ Z,
                                            const float *__restrict__ M, int n_fp, int top,
                                            float phip, float &Fp, float &zp, float &mp)
{
    int lo = 0;
    for (int step = top; step > 0; step >>= 1) {
        const int c = lo + step;
        if (c <= n_fp - 1 && ph[c] <= phip) lo = c;
    }
    float w = (phip - ph[lo]) / (ph[lo + 1] - ph[lo]);
    w = fminf(fmaxf(w, 0.0f), 1.0f);
    Fp = fmaf(F[lo + 1] - F[lo], w, F[lo]);
    zp = fmaf(Z[lo + 1] - Z[lo], w, Z[lo]);
    mp = fmaf(M[lo + 1] - M[lo], w, M[lo]);
}

// State of one (element, output phase) pair in the atmosphere path.
struct PairA {
    float w0, w1, w2, w3;  // mu stencil weights times F_p
    int s0;                // first mu row of the stencil
    float lz;              // ln(z_p) / dlnE_table
    int mode;              // 0 off, 1 sliding window, 2 general (table edges)
    int nb;                // smem offset of node q+2 (row) + s0
    float q, qn, W1, W2, W3, d1, d2, d3;
};

__device__ __forceinline__ void pair_setup_atm(PairA &P, bool on, float s, float phi_out,
                                               const float *sm, const Layout &lay, int n_fp,
                                               int top, const AtmDev &A,
                                               const EnergyDev &en, float inv_dlnE,
                                               float pk0, float pkl, float lz_safe)
{
    const float *ph = sm + lay.tmpl;
    const float *Fa = ph + (n_fp + 1);
    const float *Za = Fa + (n_fp + 1);
    const float *Ma = Za + (n_fp + 1);
    const float *mun = sm + lay.munodes;
    const int nmu = A.nmu;
    P.w0 = P.w1 = P.w2 = P.w3 = 0.0f;
    P.s0 = 0;
    P.lz = lz_safe;
    P.mode = 0;
    if (on) {
        const float x = phi_out + s + 1.0f - ph[0];
        const float phip = x - floorf(x) + ph[0];
        float Fp, zp, mp;
        template_at(ph, Fa, Za, Ma, n_fp, top, phip, Fp, zp, mp);
        if (Fp != 0.0f && zp > 0.0f && zp < 1e30f) {
            // mu: clamp, interval, mixed-order weights (Sect. 4)
            const float mu = fminf(fmaxf(mp, mun[0]), mun[nmu - 1]);
            int i = 0;
            for (int step = 64; step > 0; step >>= 1) {
                const int c = i + step;
                if (c <= nmu - 2 && mun[c] <= mu) i = c;
            }
            float w[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            int s0;
            if (i >= 1 && i + 2 <= nmu - 1 && i >= A.n_protect - 1) {
                s0 = i - 1;
                const float x0 = mun[s0], x1 = mun[s0 + 1], x2 = mun[s0 + 2], x3 = mun[s0 + 3];
                w[0] = (mu - x1) * (mu - x2) * (mu - x3) / ((x0 - x1) * (x0 - x2) * (x0 - x3));
                w[1] = (mu - x0) * (mu - x2) * (mu - x3) / ((x1 - x0) * (x1 - x2) * (x1 - x3));
                w[2] = (mu - x0) * (mu - x1) * (mu - x3) / ((x2 - x0) * (x2 - x1) * (x2 - x3));
                w[3] = (mu - x0) * (mu - x1) * (mu - x2) / ((x3 - x0) * (x3 - x1) * (x3 - x2));
            } else {
                s0 = min(max(i - 1, 0), nmu - 4);
                const float t = (mu - mun[i]) / (mun[i + 1] - mun[i]);
                const int o = i - s0;
#pragma unroll
                for (int a = 0; a < 4; ++a) w[a] = (a == o) ? 1.0f - t : ((a == o + 1) ? t : 0.0f);
            }
            P.w0 = w[0] * Fp; P.w1 = w[1] * Fp; P.w2 = w[2] * Fp; P.w3 = w[3] * Fp;
            P.s0 = s0;
            const float lz = logf(zp) * inv_dlnE;
            const bool fast = en.sliding && (pk0 + lz >= 1.0f) && (pkl + lz < (float)(A.nE - 2));
            P.mode = fast ? 1 : 2;
            P.lz = lz;
        }
    }
}

__device__ __forceinline__ void sliding_init(PairA &P, const float *slab, int Pm, float pk0,
                                             float lz_safe)
{
    const float lz = (P.mode == 1) ? P.lz : lz_safe;
    const float q = floorf(pk0 + lz);
    const int qi = (int)q;
    P.nb = (qi + 2) * Pm + P.s0;
    const float Wm = contract4(slab, P.nb - 3 * Pm, P.w0, P.w1, P.w2, P.w3);
    P.W1 = contract4(slab, P.nb - 2 * Pm, P.w0, P.w1, P.w2, P.w3);
    P.W2 = contract4(slab, P.nb - Pm, P.w0, P.w1, P.w2, P.w3);
    P.W3 = contract4(slab, P.nb, P.w0, P.w1, P.w2, P.w3);
    P.d1 = P.W2 - P.W1;
    P.d2 = 0.5f * (Wm + P.W2) - P.W1;
    P.d3 = ((P.W3 - Wm) + 3.0f * (P.W1 - P.W2)) * (1.0f / 6.0f);
    P.q = q;
    P.qn = q + 1.0f;
}

// general evaluation (table edges / clamping) of the contracted spectrum at p
__device__ __noinline__ float eval_general(const PairA &P, const float *slab, int Pm,
                                              int nE_t, float p)
{
    if (p <= 0.0f) return contract4(slab, P.s0, P.w0, P.w1, P.w2, P.w3);
    if (p >= (float)(nE_t - 1))
        return contract4(slab, (nE_t - 1) * Pm + P.s0, P.w0, P.w1, P.w2, P.w3);
    const float q = floorf(p);
    const int qi = (int)q;
    const float t = p - q;
    if (qi >= 1 && qi + 2 <= nE_t - 1) {
        const float a = contract4(slab, (qi - 1) * Pm + P.s0, P.w0, P.w1, P.w2, P.w3);
        const float b = contract4(slab, qi * Pm + P.s0, P.w0, P.w1, P.w2, P.w3);
        const float c = contract4(slab, (qi + 1) * Pm + P.s0, P.w0, P.w1, P.w2, P.w3);
        const float d = contract4(slab, (qi + 2) * Pm + P.s0, P.w0, P.w1, P.w2, P.w3);
        const float d1 = c - b, d2 = 0.5f * (a + c) - b;
        const float d3 = ((d - a) + 3.0f * (b - c)) * (1.0f / 6.0f);
        return b + t * (d1 + (t - 1.0f) * (d2 + (t + 1.0f) * d3));
    }
    const float b = contract4(slab, qi * Pm + P.s0, P.w0, P.w1, P.w2, P.w3);
    const float c = contract4(slab, (qi + 1) * Pm + P.s0, P.w0, P.w1, P.w2, P.w3);
    return fmaf(t, c - b, b);
}

template <int EMIS>
__global__ void __launch_bounds__(kSABlock, 2)
    k_shift_add(Params p, PlanDev plan, AtmDev A, EnergyDev en, Layout lay,
                const RingRec *__restrict__ recs, const float *__restrict__ tmpl,
                const float *__restrict__ elems, const int *__restrict__ status,
                float *__restrict__ partials)
{
    extern __shared__ float sm[];
    const Item it = plan.items[blockIdx.x];
    const InstPlan ip = plan.inst[it.b];
    const int n_fp = plan.n_fp;
    const int nEpad = en.nEpad;
    const int nch = nEpad / kEC;
    float *Fblk = sm + lay.fblk;
    float *spk = sm + lay.pk;
    float *sE = sm + lay.E;
    float *sE2 = sm + lay.E2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (int i = tid; i < kPT * nEpad; i += blockDim.x) Fblk[i] = 0.0f;
    for (int i = tid; i < nEpad; i += blockDim.x) {
        spk[i] = en.pk[i];
        sE[i] = en.E[i];
        sE2[i] = en.E2[i];
    }
    if (EMIS == 1)
        for (int i = tid; i < A.nmu; i += blockDim.x) sm[lay.munodes + i] = A.mu[i];

    int top = 1;
    while (top * 2 <= n_fp) top *= 2;
    const float inv_nphase = 1.0f / (float)ip.n_phase;
    const float inv_dlnE = (EMIS == 1) ? (float)(1.0 / A.dlnE) : 0.0f;
    const int Pm = A.nmu_pad;
    const bool inst_ok = status[it.b] == 0;

    for (int r = it.r0; r < it.r1 && inst_ok; ++r) {
        const int ring = ip.ring0 + it.spot * ip.n_theta + r;
        const RingRec rec = recs[ring];
        if (!rec.visible) continue;
        __syncthreads();  // previous ring finished with the staged data
        {
            const float *tsrc = tmpl + (size_t)ring * 4 * (n_fp + 1);
            for (int i = tid; i < 4 * (n_fp + 1); i += blockDim.x) sm[lay.tmpl + i] = tsrc[i];
            const float *esrc = elems + (size_t)ip.elem0 + (size_t)(ring - ip.ring0) * ip.n_phi;
            for (int i = tid; i < rec.n_active; i += blockDim.x) sm[lay.elems + i] = esrc[i];
            if (EMIS == 1) {
                const size_t plane = (size_t)A.nmu * A.nE;
                const float *I00 = A.I + ((size_t)rec.iT * A.ng + rec.ig) * plane;
                const float *I01 = I00 + plane;
                const float *I10 = I00 + (size_t)A.ng * plane;
                const float *I11 = I10 + plane;
                const float wT = rec.wT, wg = rec.wg;
                const float w00 = (1.0f - wT) * (1.0f - wg), w01 = (1.0f - wT) * wg;
                const float w10 = wT * (1.0f - wg), w11 = wT * wg;
                float *slab = sm + lay.slab;
                for (int idx = tid; idx < (int)plane; idx += blockDim.x) {
                    const int m = idx / A.nE, n = idx - m * A.nE;
                    const float v = w00 * __ldg(I00 + idx) + w01 * __ldg(I01 + idx) +
                                    w10 * __ldg(I10 + idx) + w11 * __ldg(I11 + idx);
                    slab[n * Pm + m] = v;
                }
            }
        }
        __syncthreads();

        const int n_act = rec.n_active;
        const float *sel = sm + lay.elems;
        const float *slab = sm + lay.slab;
        const float pk0 = spk[0], pkl = spk[en.nE - 1];
        const float lz_safe = 1.25f - pk0;

        for (int jl = warp; jl < it.nj; jl += kSABlock / 32) {
            const float phi_out = (float)(it.j0 + jl) * inv_nphase;
            for (int g0 = 0; g0 < n_act; g0 += 128) {
                if (EMIS == 1) {
                    PairA P[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int m = g0 + lane + 32 * e;
                        pair_setup_atm(P[e], m < n_act, m < n_act ? sel[m] : 0.0f, phi_out, sm,
                                       lay, n_fp, top, A, en, inv_dlnE, pk0, pkl, lz_safe);
                    }
                    bool anyfast[4], anyslow[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        anyfast[e] = __any_sync(kFull, P[e].mode == 1);
                        anyslow[e] = __any_sync(kFull, P[e].mode == 2);
                        if (anyfast[e]) sliding_init(P[e], slab, Pm, pk0, lz_safe);
                    }
                    for (int c = 0; c < nch; ++c) {
                        float acc[kEC];
#pragma unroll
                        for (int s = 0; s < kEC; ++s) acc[s] = 0.0f;
                        const float *pkc = spk + c * kEC;
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            if (anyfast[e]) {
                            // sliding window (lanes not in sliding mode add zero here)
                            const float lz = (P[e].mode == 1) ? P[e].lz : lz_safe;
                            const float sw = (P[e].mode == 1) ? 1.0f : 0.0f;
#pragma unroll
                            for (int s = 0; s < kEC; ++s) {
                                const float pv = pkc[s] + lz;
                                if (pv >= P[e].qn) {
                                    P[e].nb += Pm;
                                    const float nv = contract4(slab, P[e].nb, P[e].w0, P[e].w1,
                                                               P[e].w2, P[e].w3);
                                    const float a = P[e].W1;
                                    P[e].W1 = P[e].W2;
                                    P[e].W2 = P[e].W3;
                                    P[e].W3 = nv;
                                    P[e].d1 = P[e].W2 - P[e].W1;
                                    P[e].d2 = 0.5f * (a + P[e].W2) - P[e].W1;
                                    P[e].d3 = ((P[e].W3 - a) + 3.0f * (P[e].W1 - P[e].W2)) *
                                              (1.0f / 6.0f);
                                    P[e].q = P[e].qn;
                                    P[e].qn += 1.0f;
                                }
                                const float t = pv - P[e].q;
                                const float v = fmaf(t, fmaf(pv - P[e].qn,
                                                             fmaf(t + 1.0f, P[e].d3, P[e].d2),
                                                             P[e].d1),
                                                     P[e].W1);
                                acc[s] = fmaf(sw, v, acc[s]);
                            }
                            }
                            if (anyslow[e] && P[e].mode == 2) {
#pragma unroll
                                for (int s = 0; s < kEC; ++s)
                                    acc[s] += eval_general(P[e], slab, Pm, A.nE, pkc[s] + P[e].lz);
                            }
                        }
                        const float tot = transpose_reduce(acc, lane);
                        Fblk[jl * nEpad + c * kEC + lane] += tot;
                    }
                } else {
                    // analytic isotropic blackbody: I(E')/E = K z^3 E^2 / expm1(z E / kT)
                    const float K = (float)(2.0 / (kH_KEVS * kH_KEVS * kH_KEVS * kC_CM * kC_CM));
                    const float inv_kT = 1.0f / rec.kT;
                    const float *ph = sm + lay.tmpl;
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
                            template_at(ph, ph + (n_fp + 1), ph + 2 * (n_fp + 1),
                                        ph + 3 * (n_fp + 1), n_fp, top, phip, Fp, zp, mp);
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
                                acc[s] += bz[e] * sE2[k] / expm1f(az[e] * sE[k]);
                            }
                        }
                        const float tot = transpose_reduce(acc, lane);
                        Fblk[jl * nEpad + c * kEC + lane] += tot;
                    }
                }
            }
        }
    }
    __syncthreads();
    float *dst = partials + (size_t)blockIdx.x * kPT * nEpad;
    for (int i = tid; i < it.nj * nEpad; i += blockDim.x) dst[i] = Fblk[i];
}

__global__ void k_reduce(PlanDev plan, EnergyDev en, const float *__restrict__ partials,
                         const int *__restrict__ status, int total_rows, float *__restrict__ Ft)
{
    const int nE = en.nE, nEpad = en.nEpad;
    const size_t total = (size_t)total_rows * nE;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const int row = (int)(t / nE), k = (int)(t - (size_t)row * nE);
        const int b = find_instance_by_row(plan.inst, plan.B, row);
        const InstPlan ip = plan.inst[b];
        const int j = row - ip.row0;
        const int tile = j / kPT, jl = j - tile * kPT;
        const int2 rng = plan.tile_items[ip.tile0 + tile];
        float s = 0.0f;
        for (int i = rng.x; i < rng.y; ++i) s += partials[((size_t)i * kPT + jl) * nEpad + k];
        Ft[t] = (status[b] == 0) ? s * en.invE[k] * (float)(1.0 / kFluxScale) : 0.0f;
    }
}

}  // namespace

cudaError_t launch_shift_add(const Params &p, const PlanDev &plan, const AtmDev &A,
                             const EnergyDev &en, const RingRec *recs, const float *tmpl,
                             const float *elems, const int *status, float *partials,
                             int n_phi_max, cudaStream_t st)
{
    if (plan.n_items <= 0) return cudaSuccess;
    Layout lay;
    int off = 0;
    auto take = [&](int n) { int o = off; off += (n + 3) & ~3; return o; };
    lay.tmpl = take(4 * (plan.n_fp + 1));
    lay.elems = take(n_phi_max);
    lay.munodes = take(p.emission == 1 ? A.nmu : 0);
    lay.slab = take(p.emission == 1 ? A.nE * A.nmu_pad : 0);
    lay.pk = take(en.nEpad);
    lay.E = take(en.nEpad);
    lay.E2 = take(en.nEpad);
    lay.fblk = take(kPT * en.nEpad);
    lay.total = off;
    const size_t bytes = (size_t)off * sizeof(float);
    cudaError_t e;
    if (p.emission == 1) {
        e = cudaFuncSetAttribute(k_shift_add<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bytes);
        if (e != cudaSuccess) return e;
        k_shift_add<1><<<plan.n_items, kSABlock, bytes, st>>>(p, plan, A, en, lay, recs, tmpl,
                                                              elems, status, partials);
    } else {
        e = cudaFuncSetAttribute(k_shift_add<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bytes);
        if (e != cudaSuccess) return e;
        k_shift_add<0><<<plan.n_items, kSABlock, bytes, st>>>(p, plan, A, en, lay, recs, tmpl,
                                                              elems, status, partials);
    }
    return cudaGetLastError();
}

cudaError_t launch_reduce(const PlanDev &plan, const EnergyDev &en, const float *partials,
                          const int *status, int total_rows, float *Ft, cudaStream_t st)
{
    const size_t total = (size_t)total_rows * en.nE;
    if (total == 0) return cudaSuccess;
    const int blocks = (int)std::min<size_t>((total + 255) / 256, 65535);
    k_reduce<<<blocks, 256, 0, st>>>(plan, en, partials, status, total_rows, Ft);
    return cudaGetLastError();
}

}  // namespace ppm
