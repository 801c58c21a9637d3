// C ABI of libppm.so: contexts, tables, planning, workspace and launches.
#include <algorithm>
#include <cstdarg>
#include <cstdlib>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ppm_internal.cuh"

using namespace ppm;

namespace {

struct DevBuf {
    void *p = nullptr;
    size_t n = 0;
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    // grow-only; the caller must make sure the old contents are no longer in use
    cudaError_t ensure(size_t bytes)
    {
        if (bytes <= n && p) return cudaSuccess;
        release();
        size_t want = std::max<size_t>(bytes + bytes / 4, 256);
        cudaError_t e = cudaMalloc(&p, want);
        if (e != cudaSuccess) { p = nullptr; return e; }
        n = want;
        return cudaSuccess;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

struct HostPlan {
    int pt = kPT;
    std::vector<InstPlan> inst;
    std::vector<Item> items;
    std::vector<int2> tiles;
    std::vector<int> order;
    int total_rings = 0, total_rows = 0, n_phi_max = 0;
    size_t total_elems = 0;
};

struct DeviceGuard {
    int prev = -1, dev;
    explicit DeviceGuard(int d) : dev(d)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    }
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

struct ppm_ctx {
    int device = 0;
    int sm_count = 0;
    size_t smem_optin = 0;
    std::string err;
    // lens
    bool lens_ready = false;
    ppm_lens_spec lens{};
    DevBuf d_Ca, d_LF, d_TD;
    // atmosphere
    bool atm_ready = false;
    int nT = 0, ng = 0, nmu = 0, nEt = 0, n_protect = 0, nmu_pad = 0;
    int interp = kInterpD;  // interpolation strategy (Sect. 4)
    double lnE0_t = 0.0, dlnE_t = 0.0;
    DevBuf d_I, d_logT, d_logg, d_mu;
    DevBuf d_mu_aux;   // mu bin index, reciprocal Lagrange denominators, reciprocal spacings
    float mu_bin = 0.0f;
    // energies
    std::vector<double> E;
    DevBuf d_E, d_E3, d_pk, d_invE;
    bool energy_dirty = true;
    int nEpad = 0, sliding = 0;
    float walk_step = 0.0f;  // uniform pk step (node-major walk) or 0
    // response
    int nc = 0;
    DevBuf d_R, d_sigma, d_Rtc;  // d_Rtc: R split into bf16 hi/lo tiles for the tensor cores
    // work decomposition of the shift-and-add (ppm_set_tiles / ppm_autotune)
    int tile_pt = 0;          // output phases per item: 0 = automatic, 16 or 32
    int tile_waves = 16;      // target waves of 2 blocks per SM (sets the ring-group size)
    int tile_persistent = 0;  // 1: persistent blocks take items from a queue
    int tile_walk = 0;        // 0: moment walk, else node-major walk, where they apply;
                              // 1: energy walk; 2: node-major walk where it applies
    int *d_queue = nullptr;
    // plan
    std::vector<int> plan_key;
    int plan_grid = 0;
    HostPlan plan;
    DevBuf d_plan;
    void *h_pinned = nullptr;
    size_t h_pinned_n = 0;
    cudaEvent_t plan_ev = nullptr;
    // workspace
    DevBuf ws;
    unsigned *d_err = nullptr;
    double *d_lfact = nullptr;  // ln d! for d < kLogFactN
    // stage timing
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    struct Pending { int stage; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    ppm_timing acc{};
    unsigned long long *d_triples = nullptr;
};

namespace {
// NVTX names of the timed stages (ranges around their launches, visible to
// Nsight tools; no-ops without a tool attached)
const char *const kStageName[] = {"ppm ring template", "ppm shift-and-add", "ppm reduce",
                                  "ppm response + logL", "ppm response adjoint",
                                  "ppm backward shift-and-add", "ppm template tangents"};

// an NVTX range for the lifetime of one API call
struct NvtxCall {
    explicit NvtxCall(const char *name) { nvtxRangePushA(name); }
    ~NvtxCall() { nvtxRangePop(); }
};

// records an event pair around one stage when timing is enabled
struct StageTimer {
    ppm_ctx *c;
    int stage;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    bool open = true;
    StageTimer(ppm_ctx *c_, int stage_, cudaStream_t st_) : c(c_), stage(stage_), st(st_)
    {
        nvtxRangePushA(kStageName[stage]);
        if (!c->timing) return;
        a = take();
        if (a) cudaEventRecord(a, st);
    }
    cudaEvent_t take()
    {
        if (!c->ev_pool.empty()) {
            cudaEvent_t e = c->ev_pool.back();
            c->ev_pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        return e;
    }
    ~StageTimer()
    {
        if (open) nvtxRangePop();
    }
    void done(int kernels)
    {
        if (open) nvtxRangePop();
        open = false;
        if (!c->timing) return;
        c->acc.launches += kernels;
        if (!a) return;
        cudaEvent_t b = take();
        if (!b) { c->ev_pool.push_back(a); return; }
        cudaEventRecord(b, st);
        c->pending.push_back({stage, a, b});
    }
};
}  // namespace

static ppm_status fail(ppm_ctx *c, ppm_status s, const char *fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

static ppm_status cuda_fail(ppm_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, e == cudaErrorMemoryAllocation ? PPM_ENOMEM : PPM_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define PPM_CUDA(call, what)                                  \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

extern "C" {

ppm_status ppm_create(ppm_ctx **out, int device)
{
    if (!out) return PPM_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return PPM_EINVAL;
    ppm_ctx *ctx = new ppm_ctx();
    ctx->device = device;
    DeviceGuard g(device);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete ctx;
        return PPM_ECUDA;
    }
    ctx->sm_count = prop.multiProcessorCount;
    ctx->smem_optin = prop.sharedMemPerBlockOptin;
    {
        std::vector<double> lf(kLogFactN);
        for (int d = 0; d < kLogFactN; ++d) lf[d] = std::lgamma((double)d + 1.0);
        if (cudaMalloc(&ctx->d_lfact, kLogFactN * sizeof(double)) != cudaSuccess ||
            cudaMemcpy(ctx->d_lfact, lf.data(), kLogFactN * sizeof(double),
                       cudaMemcpyHostToDevice) != cudaSuccess) {
            ppm_destroy(ctx);
            return PPM_ENOMEM;
        }
    }
    if (cudaMalloc(&ctx->d_queue, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&ctx->d_err, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(ctx->d_err, 0, sizeof(unsigned)) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->plan_ev, cudaEventDisableTiming) != cudaSuccess) {
        ppm_destroy(ctx);
        return PPM_ENOMEM;
    }
    *out = ctx;
    return PPM_OK;
}

void ppm_destroy(ppm_ctx *ctx)
{
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    for (DevBuf *b : {&ctx->d_Ca, &ctx->d_LF, &ctx->d_TD, &ctx->d_I, &ctx->d_logT, &ctx->d_logg,
                      &ctx->d_mu, &ctx->d_mu_aux, &ctx->d_E, &ctx->d_E3, &ctx->d_pk, &ctx->d_invE, &ctx->d_R,
                      &ctx->d_sigma, &ctx->d_Rtc, &ctx->d_plan, &ctx->ws})
        b->release();
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->d_queue) cudaFree(ctx->d_queue);
    if (ctx->d_lfact) cudaFree(ctx->d_lfact);
    if (ctx->d_triples) cudaFree(ctx->d_triples);
    for (auto &pd : ctx->pending) ctx->ev_pool.push_back(pd.a), ctx->ev_pool.push_back(pd.b);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    if (ctx->plan_ev) cudaEventDestroy(ctx->plan_ev);
    delete ctx;
}

const char *ppm_last_error(const ppm_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

// ---------------------------------------------------------------------------
// lens tables
// ---------------------------------------------------------------------------
ppm_status ppm_build_lens(ppm_ctx *ctx, const ppm_lens_spec *s, void *stream)
{
    if (!ctx || !s) return fail(ctx, PPM_EINVAL, "null argument");
    if (s->n_u < 2 || s->n_cpsi < 2 || s->n_calpha < 2 || s->n_u > 8192 || s->n_cpsi > 65536 ||
        s->n_calpha > 65536)
        return fail(ctx, PPM_EINVAL, "lens grid sizes must be in [2, 8192/65536]");
    if (!(s->u_min >= 0.0 && s->u_min < s->u_max && s->u_max < 2.0 / 3.0))
        return fail(ctx, PPM_EINVAL, "need 0 <= u_min < u_max < 2/3");
    if (!(s->cpsi_min >= -1.0 && s->cpsi_min < s->cpsi_max && s->cpsi_max == 1.0))
        return fail(ctx, PPM_EINVAL, "need -1 <= cpsi_min < cpsi_max = 1");
    if (!(s->calpha_min >= -1.0 && s->calpha_min < s->calpha_max && s->calpha_max <= 1.0))
        return fail(ctx, PPM_EINVAL, "need -1 <= calpha_min < calpha_max <= 1");
    if (!(s->dalpha >= kPI / 16384.0 && s->dalpha <= 0.05))
        return fail(ctx, PPM_EINVAL, "need pi/16384 <= dalpha <= 0.05");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    PPM_CUDA(cudaStreamSynchronize(st), "sync before lens build");
    const size_t ncp = (size_t)s->n_u * s->n_cpsi, nca = (size_t)s->n_u * s->n_calpha;
    PPM_CUDA(ctx->d_Ca.ensure(ncp * 8), "alloc Ca");
    PPM_CUDA(ctx->d_LF.ensure(ncp * 8), "alloc LF");
    PPM_CUDA(ctx->d_TD.ensure(nca * 8), "alloc TD");
    const int j_cap = (int)std::floor(kPI / s->dalpha) + 2;
    DevBuf scratch;
    PPM_CUDA(scratch.ensure((size_t)s->n_u * j_cap * 4 * sizeof(double)), "alloc lens scratch");
    LensDev L;
    L.u_min = s->u_min; L.u_max = s->u_max; L.n_u = s->n_u;
    L.cpsi_min = s->cpsi_min; L.cpsi_max = s->cpsi_max; L.n_cpsi = s->n_cpsi;
    L.ca_min = s->calpha_min; L.ca_max = s->calpha_max; L.n_calpha = s->n_calpha;
    L.Ca = ctx->d_Ca.as<double>(); L.LF = ctx->d_LF.as<double>(); L.TD = ctx->d_TD.as<double>();
    double *psi = scratch.as<double>();
    cudaError_t e = launch_lens_build(L, s->dalpha, psi, psi + (size_t)s->n_u * j_cap, j_cap, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    scratch.release();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lens build");
    ctx->lens = *s;
    ctx->lens_ready = true;
    return PPM_OK;
}

ppm_status ppm_get_lens(ppm_ctx *ctx, double *Ca, double *LF, double *TD)
{
    if (!ctx) return PPM_EINVAL;
    if (!ctx->lens_ready) return fail(ctx, PPM_EINVAL, "lens tables not built");
    DeviceGuard g(ctx->device);
    const size_t ncp = (size_t)ctx->lens.n_u * ctx->lens.n_cpsi;
    const size_t nca = (size_t)ctx->lens.n_u * ctx->lens.n_calpha;
    PPM_CUDA(cudaDeviceSynchronize(), "sync");
    if (Ca) PPM_CUDA(cudaMemcpy(Ca, ctx->d_Ca.p, ncp * 8, cudaMemcpyDeviceToHost), "copy Ca");
    if (LF) PPM_CUDA(cudaMemcpy(LF, ctx->d_LF.p, ncp * 8, cudaMemcpyDeviceToHost), "copy LF");
    if (TD) PPM_CUDA(cudaMemcpy(TD, ctx->d_TD.p, nca * 8, cudaMemcpyDeviceToHost), "copy TD");
    return PPM_OK;
}

// ---------------------------------------------------------------------------
// atmosphere, energies, response
// ---------------------------------------------------------------------------
static bool increasing(const double *x, int n)
{
    for (int i = 0; i + 1 < n; ++i)
        if (!(x[i + 1] > x[i]) || !std::isfinite(x[i])) return false;
    return std::isfinite(x[n - 1]);
}

ppm_status ppm_set_atmosphere(ppm_ctx *ctx, const float *I, const double *logT, int nT,
                              const double *logg, int ng, const double *mu, int nmu,
                              const double *lnE, int nE, int n_protect)
{
    if (!ctx || !I || !logT || !logg || !mu || !lnE) return fail(ctx, PPM_EINVAL, "null argument");
    if (nT < 2 || ng < 2 || nmu < 4 || nmu > 128 || nE < 4 || nE > 512)
        return fail(ctx, PPM_EINVAL, "atmosphere sizes out of range");
    if (n_protect < 2 || n_protect > nmu) return fail(ctx, PPM_EINVAL, "bad n_protect");
    if (!increasing(logT, nT) || !increasing(logg, ng) || !increasing(mu, nmu) ||
        !increasing(lnE, nE))
        return fail(ctx, PPM_EINVAL, "table axes must be strictly increasing");
    const double d = (lnE[nE - 1] - lnE[0]) / (nE - 1);
    for (int i = 0; i < nE; ++i)
        if (std::fabs(lnE[i] - (lnE[0] + i * d)) > 1e-9 * std::fabs(lnE[nE - 1] - lnE[0]))
            return fail(ctx, PPM_EINVAL, "ln E axis must be uniformly spaced");
    const int pad = nmu | 1;
    if ((size_t)nE * pad * 4 > 160 * 1024)
        return fail(ctx, PPM_EINVAL, "atmosphere slab (nE x nmu) exceeds 160 KB of shared memory");
    DeviceGuard g(ctx->device);
    PPM_CUDA(cudaDeviceSynchronize(), "sync");
    const size_t n = (size_t)nT * ng * nmu * nE;
    PPM_CUDA(ctx->d_I.ensure(n * 4), "alloc table");
    PPM_CUDA(ctx->d_logT.ensure(nT * 8), "alloc");
    PPM_CUDA(ctx->d_logg.ensure(ng * 8), "alloc");
    PPM_CUDA(ctx->d_mu.ensure(nmu * 4), "alloc");
    PPM_CUDA(cudaMemcpy(ctx->d_I.p, I, n * 4, cudaMemcpyHostToDevice), "copy table");
    PPM_CUDA(cudaMemcpy(ctx->d_logT.p, logT, nT * 8, cudaMemcpyHostToDevice), "copy");
    PPM_CUDA(cudaMemcpy(ctx->d_logg.p, logg, ng * 8, cudaMemcpyHostToDevice), "copy");
    std::vector<float> muf(mu, mu + nmu);
    PPM_CUDA(cudaMemcpy(ctx->d_mu.p, muf.data(), nmu * 4, cudaMemcpyHostToDevice), "copy");
    {
        // lookups of the FP32 mu nodes: bin -> an interval near the bin's
        // start (the kernels correct it by linear steps to the exact
        // interval), Lagrange and linear reciprocal denominators
        const double m0 = muf[0], m1 = muf[nmu - 1];
        const double bin = kMuBins / (m1 - m0);
        std::vector<int> idx(kMuBins);
        for (int b = 0; b < kMuBins; ++b) {
            const double edge = m0 + b / bin;
            int c = 0;
            while (c + 1 <= nmu - 2 && (double)muf[c + 1] <= edge) ++c;
            idx[b] = c;
        }
        std::vector<float> rden(4 * (size_t)nmu, 0.0f), rlin(nmu, 0.0f);
        for (int s0 = 0; s0 + 3 < nmu; ++s0)
            for (int a = 0; a < 4; ++a) {
                double den = 1.0;
                for (int b2 = 0; b2 < 4; ++b2)
                    if (b2 != a) den *= (double)muf[s0 + a] - (double)muf[s0 + b2];
                rden[4 * s0 + a] = (float)(1.0 / den);
            }
        for (int i = 0; i + 1 < nmu; ++i) rlin[i] = (float)(1.0 / ((double)muf[i + 1] - muf[i]));
        const size_t o_rden = kMuBins * sizeof(int), o_rlin = o_rden + rden.size() * 4;
        PPM_CUDA(ctx->d_mu_aux.ensure(o_rlin + rlin.size() * 4), "alloc");
        char *base = ctx->d_mu_aux.as<char>();
        PPM_CUDA(cudaMemcpy(base, idx.data(), kMuBins * sizeof(int), cudaMemcpyHostToDevice), "copy");
        PPM_CUDA(cudaMemcpy(base + o_rden, rden.data(), rden.size() * 4, cudaMemcpyHostToDevice),
                 "copy");
        PPM_CUDA(cudaMemcpy(base + o_rlin, rlin.data(), rlin.size() * 4, cudaMemcpyHostToDevice),
                 "copy");
        ctx->mu_bin = (float)bin;
    }
    ctx->nT = nT; ctx->ng = ng; ctx->nmu = nmu; ctx->nEt = nE; ctx->n_protect = n_protect;
    ctx->nmu_pad = pad; ctx->lnE0_t = lnE[0]; ctx->dlnE_t = d;
    ctx->atm_ready = true;
    ctx->energy_dirty = true;
    return PPM_OK;
}

ppm_status ppm_set_interpolation(ppm_ctx *ctx, int strategy)
{
    if (!ctx) return PPM_EINVAL;
    if (strategy < PPM_INTERP_MIXED || strategy > PPM_INTERP_CUBIC_LINEAR_EDGES)
        return fail(ctx, PPM_EINVAL, "unknown interpolation strategy %d", strategy);
    ctx->interp = strategy;
    return PPM_OK;
}

ppm_status ppm_set_energies(ppm_ctx *ctx, const double *E_keV, int nE)
{
    if (!ctx || !E_keV) return fail(ctx, PPM_EINVAL, "null argument");
    if (nE < 1 || nE > 1024) return fail(ctx, PPM_EINVAL, "need 1 <= nE <= 1024");
    for (int i = 0; i < nE; ++i)
        if (!(E_keV[i] > 0.0) || !std::isfinite(E_keV[i]) || (i && !(E_keV[i] > E_keV[i - 1])))
            return fail(ctx, PPM_EINVAL, "energies must be positive and strictly increasing");
    if (ctx->nc && (int)ctx->E.size() != nE) ctx->nc = 0;  // response no longer matches
    ctx->E.assign(E_keV, E_keV + nE);
    ctx->energy_dirty = true;
    return PPM_OK;
}

ppm_status ppm_set_response(ppm_ctx *ctx, const float *R, int nE, int nc, const float *sigma)
{
    if (!ctx || !R || !sigma) return fail(ctx, PPM_EINVAL, "null argument");
    if (nE != (int)ctx->E.size() || nE < 1) return fail(ctx, PPM_EINVAL, "response nE must match the energy grid");
    if (nc < 1 || nc > 4096) return fail(ctx, PPM_EINVAL, "need 1 <= nc <= 4096");
    DeviceGuard g(ctx->device);
    PPM_CUDA(cudaDeviceSynchronize(), "sync");
    PPM_CUDA(ctx->d_R.ensure((size_t)nE * nc * 4), "alloc R");
    PPM_CUDA(ctx->d_sigma.ensure((size_t)nE * 4), "alloc sigma");
    PPM_CUDA(cudaMemcpy(ctx->d_R.p, R, (size_t)nE * nc * 4, cudaMemcpyHostToDevice), "copy R");
    PPM_CUDA(cudaMemcpy(ctx->d_sigma.p, sigma, (size_t)nE * 4, cudaMemcpyHostToDevice), "copy sigma");
    {
        std::vector<uint16_t> tc(resp_tc_layout_elems(nE, nc));
        resp_tc_layout(R, nE, nc, tc.data());
        PPM_CUDA(ctx->d_Rtc.ensure(tc.size() * 2), "alloc tensor-core response");
        PPM_CUDA(cudaMemcpy(ctx->d_Rtc.p, tc.data(), tc.size() * 2, cudaMemcpyHostToDevice),
                 "copy tensor-core response");
    }
    ctx->nc = nc;
    return PPM_OK;
}

// Down-sampling matrix row block: DS[i][e] for the model grid x[0..n) and one
// detector bin [a, b].  The basis function of node i is the piecewise-linear
// hat on x, continued as a constant beyond the two ends.  Closed-form
// integrals of the linear pieces; adds into ds[i].
static void ds_bin(const double *x, int n, double a, double b, double *ds)
{
    if (!(b > a)) return;
    if (n == 1) { ds[0] += b - a; return; }
    if (a < x[0]) ds[0] += std::min(b, x[0]) - a;
    if (b > x[n - 1]) ds[n - 1] += b - std::max(a, x[n - 1]);
    const double lo = std::max(a, x[0]), hi = std::min(b, x[n - 1]);
    if (!(hi > lo)) return;
    int j = (int)(std::upper_bound(x, x + n, lo) - x) - 1;
    j = std::min(std::max(j, 0), n - 2);
    for (; j < n - 1 && x[j] < hi; ++j) {
        const double x0 = std::max(lo, x[j]), x1 = std::min(hi, x[j + 1]);
        if (!(x1 > x0)) continue;
        const double h = x[j + 1] - x[j];
        const double r0 = x[j + 1] - x0, r1 = x[j + 1] - x1;   // distances to the right node
        const double l0 = x0 - x[j], l1 = x1 - x[j];           // distances to the left node
        ds[j] += (r0 * r0 - r1 * r1) / (2.0 * h);
        ds[j + 1] += (l1 * l1 - l0 * l0) / (2.0 * h);
    }
}

ppm_status ppm_set_response_fine(ppm_ctx *ctx, const double *E_lo, const double *E_hi, int Ne,
                                 const float *Rf, int nc, const float *sigma)
{
    if (!ctx || !E_lo || !E_hi || !Rf || !sigma) return fail(ctx, PPM_EINVAL, "null argument");
    const int nE = (int)ctx->E.size();
    if (nE < 1) return fail(ctx, PPM_EINVAL, "energy grid not set");
    if (Ne < 1 || Ne > (1 << 20)) return fail(ctx, PPM_EINVAL, "need 1 <= Ne <= 1048576");
    if (nc < 1 || nc > 4096) return fail(ctx, PPM_EINVAL, "need 1 <= nc <= 4096");
    for (int e = 0; e < Ne; ++e)
        if (!(E_hi[e] > E_lo[e]) || !std::isfinite(E_lo[e]) || !std::isfinite(E_hi[e]))
            return fail(ctx, PPM_EINVAL, "detector bin %d: need finite E_lo < E_hi", e);
    std::vector<double> R((size_t)nE * nc, 0.0), ds(nE);
    for (int e = 0; e < Ne; ++e) {
        std::fill(ds.begin(), ds.end(), 0.0);
        ds_bin(ctx->E.data(), nE, E_lo[e], E_hi[e], ds.data());
        const float *rf = Rf + (size_t)e * nc;
        for (int i = 0; i < nE; ++i) {
            if (ds[i] == 0.0) continue;
            double *r = R.data() + (size_t)i * nc;
            for (int c = 0; c < nc; ++c) r[c] += ds[i] * (double)rf[c];
        }
    }
    std::vector<float> Rs(R.size());
    for (size_t q = 0; q < R.size(); ++q) Rs[q] = (float)R[q];
    return ppm_set_response(ctx, Rs.data(), nE, nc, sigma);
}

// ---------------------------------------------------------------------------
// planning and launch
// ---------------------------------------------------------------------------
// Position of observed energy k on the table's ln E axis, in nodes.
static float pk_of(const ppm_ctx *ctx, int k)
{
    return ctx->atm_ready ? (float)((std::log(ctx->E[k]) - ctx->lnE0_t) / ctx->dlnE_t) : 0.0f;
}

// The energy walk may slide along the table (consecutive pk differ by less
// than one node and the grid spans less than the table's interior).
static int sliding_of(const ppm_ctx *ctx)
{
    const int nE = (int)ctx->E.size();
    if (!ctx->atm_ready || nE < 1) return 0;
    for (int k = 0; k + 1 < nE; ++k)
        if (!((double)pk_of(ctx, k + 1) - pk_of(ctx, k) < 0.999)) return 0;
    return ((double)pk_of(ctx, nE - 1) - pk_of(ctx, 0) < ctx->nEt - 3.5) ? 1 : 0;
}

// Step of pk when the walk slides, pk is uniform to 1e-4 node and the step
// lies in [0.34, 0.498], so that every table interval holds two or three
// observed energies (the node-major walk of the shift-and-add); 0 otherwise.
static float walk_step_of(const ppm_ctx *ctx)
{
    const int nE = (int)ctx->E.size();
    if (nE < 2 || !sliding_of(ctx)) return 0.0f;
    const double p0 = pk_of(ctx, 0);
    const double d = ((double)pk_of(ctx, nE - 1) - p0) / (nE - 1);
    if (!(d >= 0.34 && d <= 0.498)) return 0.0f;
    for (int k = 0; k < nE; ++k)
        if (!(std::fabs((double)pk_of(ctx, k) - (p0 + k * d)) <= 1e-4)) return 0.0f;
    return (float)d;
}

// the node-major walk applies to the atmosphere shift-and-add of this call
// (spots and temperature maps, forward and backward; the forward spot kernel
// takes the moment walk instead where that applies)
static bool node_walk_on(const ppm_ctx *ctx, const ppm_params *p, float step)
{
    return p->emission == 1 && ctx->tile_walk != 1 && step > 0.0f;
}

// the forward atmosphere shift-and-add of this call takes the moment walk:
// spot emission, an interpolant linear in the table's node values (every
// strategy but the clipped one), energies inside the table
static bool moment_walk_on(const ppm_ctx *ctx, const ppm_params *p)
{
    return p->emission == 1 && ctx->tile_walk == 0 && !p->logT_map && ctx->interp != kInterpB &&
           sliding_of(ctx);
}

// relative table nodes of a moment-walk group: the observed energies' span
// in table nodes plus the stencil margins
static int moment_rows(const ppm_ctx *ctx)
{
    const int nE = (int)ctx->E.size();
    if (nE < 1) return 8;
    return (int)std::ceil((double)pk_of(ctx, nE - 1) - (double)pk_of(ctx, 0)) + 8;
}

static ppm_status refresh_energies(ppm_ctx *ctx)
{
    if (!ctx->energy_dirty) return PPM_OK;
    const int nE = (int)ctx->E.size();
    const int nEpad = (nE + kEC - 1) / kEC * kEC;
    std::vector<float> E(nEpad), E3(nEpad), pk(nEpad), invE(nEpad);
    for (int k = 0; k < nEpad; ++k) {
        const double e = ctx->E[std::min(k, nE - 1)];
        E[k] = (float)e;
        E3[k] = (float)(e * e * e);
        invE[k] = (float)(1.0 / e);
        pk[k] = pk_of(ctx, std::min(k, nE - 1));
    }
    const int sliding = sliding_of(ctx);
    DeviceGuard g(ctx->device);
    PPM_CUDA(cudaDeviceSynchronize(), "sync");
    for (DevBuf *b : {&ctx->d_E, &ctx->d_E3, &ctx->d_pk, &ctx->d_invE})
        PPM_CUDA(b->ensure((size_t)nEpad * 4), "alloc energies");
    PPM_CUDA(cudaMemcpy(ctx->d_E.p, E.data(), nEpad * 4, cudaMemcpyHostToDevice), "copy");
    PPM_CUDA(cudaMemcpy(ctx->d_E3.p, E3.data(), nEpad * 4, cudaMemcpyHostToDevice), "copy");
    PPM_CUDA(cudaMemcpy(ctx->d_pk.p, pk.data(), nEpad * 4, cudaMemcpyHostToDevice), "copy");
    PPM_CUDA(cudaMemcpy(ctx->d_invE.p, invE.data(), nEpad * 4, cudaMemcpyHostToDevice), "copy");
    ctx->nEpad = nEpad;
    ctx->sliding = sliding;
    ctx->walk_step = walk_step_of(ctx);
    ctx->energy_dirty = false;
    return PPM_OK;
}

// rings per spot and element slots per ring of instance b
static int rings_per_spot(const ppm_res *res, int b)
{
    return res->grid == PPM_GRID_HEALPIX ? 4 * res->n_theta[b] - 1 : res->n_theta[b];
}
static int slots_per_ring(const ppm_res *res, int b)
{
    return res->grid == PPM_GRID_HEALPIX ? 4 * res->n_theta[b] : res->n_phi[b];
}

static ppm_status check_params(ppm_ctx *ctx, const ppm_params *p, const ppm_res *res)
{
    if (!p || !res) return fail(ctx, PPM_EINVAL, "null params or res");
    if (p->B < 1 || p->B > (1 << 22)) return fail(ctx, PPM_EINVAL, "need 1 <= B <= 4194304");
    if (p->n_spots < 1 || p->n_spots > 2) return fail(ctx, PPM_EINVAL, "n_spots must be 1 or 2");
    if (p->oblate != 0 && p->oblate != 1) return fail(ctx, PPM_EINVAL, "oblate must be 0 or 1");
    if (p->emission != 0 && p->emission != 1) return fail(ctx, PPM_EINVAL, "emission must be 0 or 1");
    const void *ptrs[] = {p->mass_msun, p->radius_km, p->spin_hz, p->incl_rad, p->dist_kpc,
                          p->nh_1e20, p->colat, p->azim, p->zeta, p->logT,
                          p->mask_colat, p->mask_azim, p->mask_zeta};
    for (const void *q : ptrs)
        if (!q) return fail(ctx, PPM_EINVAL, "null parameter array");
    if (p->logT_map) {
        if (res && res->grid != PPM_GRID_HEALPIX)
            return fail(ctx, PPM_EINVAL, "a temperature map needs grid = PPM_GRID_HEALPIX");
        if (p->n_spots != 1) return fail(ctx, PPM_EINVAL, "a temperature map needs n_spots = 1");
        if (p->emission == 1 && ctx->interp != kInterpD)
            return fail(ctx, PPM_EINVAL,
                        "a temperature map needs the default interpolation strategy");
    }
    if (!res->n_theta || !res->n_phi || !res->n_phase)
        return fail(ctx, PPM_EINVAL, "null resolution array");
    if (res->n_fp < 8 || res->n_fp > kMaxFp) return fail(ctx, PPM_EINVAL, "need 8 <= n_fp <= 1024");
    if (res->grid != PPM_GRID_SPOT && res->grid != PPM_GRID_HEALPIX)
        return fail(ctx, PPM_EINVAL, "grid must be PPM_GRID_SPOT or PPM_GRID_HEALPIX");
    if (!(res->phase_sub == 1 || res->phase_sub == 2 || res->phase_sub == 4 ||
          res->phase_sub == 8 || res->phase_sub == 16))
        return fail(ctx, PPM_EINVAL, "phase_sub must be 1, 2, 4, 8 or 16");
    for (int b = 0; b < p->B; ++b) {
        if (res->grid == PPM_GRID_HEALPIX) {
            if (res->n_theta[b] < 1 || res->n_theta[b] > 1024 || res->n_phase[b] < 1 ||
                res->n_phase[b] > 4096)
                return fail(ctx, PPM_EINVAL, "instance %d: need 1 <= N_side <= 1024", b);
            continue;
        }
        if (res->n_theta[b] < 1 || res->n_theta[b] > 4096 || res->n_phi[b] < 1 ||
            res->n_phi[b] > 4096 || res->n_phase[b] < 1 || res->n_phase[b] > 4096)
            return fail(ctx, PPM_EINVAL, "instance %d: resolution out of range", b);
    }
    if (!ctx->lens_ready) return fail(ctx, PPM_EINVAL, "lens tables not built");
    if (ctx->E.empty()) return fail(ctx, PPM_EINVAL, "energy grid not set");
    if (p->emission == 1 && !ctx->atm_ready) return fail(ctx, PPM_EINVAL, "atmosphere table not set");
    return PPM_OK;
}

static ppm_status make_plan(ppm_ctx *ctx, const ppm_params *p, const ppm_res *res,
                            cudaStream_t st)
{
    const int B = p->B;
    std::vector<int> key;
    key.reserve(3 * B + 4);
    key.push_back(B);
    key.push_back(p->n_spots);
    key.push_back(res->n_fp);
    key.push_back(ctx->sm_count);
    key.push_back((int)ctx->E.size());
    key.push_back(ctx->tile_pt);
    key.push_back(ctx->tile_waves);
    key.push_back(res->grid);
    key.push_back(res->phase_sub);
    key.push_back(p->logT_map ? 1 : 0);
    const bool node = node_walk_on(ctx, p, ctx->walk_step) || moment_walk_on(ctx, p);
    key.push_back(node ? 1 : 0);
    for (int b = 0; b < B; ++b) {
        key.push_back(res->n_theta[b]);
        key.push_back(res->n_phi[b]);
        key.push_back(res->n_phase[b]);
    }
    if (key == ctx->plan_key && ctx->d_plan.p) return PPM_OK;

    HostPlan hp;
    // phase tile: 32 output phases per item, 16 when that leaves fewer than
    // eight waves of blocks (finer items shorten the last wave)
    auto ring_tiles = [&](int pt) {
        long long T = 0;
        for (int b = 0; b < B; ++b)
            T += (long long)p->n_spots * rings_per_spot(res, b) *
                 ((res->n_phase[b] * res->phase_sub + pt - 1) / pt);
        return T;
    };
    // (16 with the node-major walk, whose ring buffers leave room for two
    // blocks per SM only with 16-phase tiles)
    int pt = (node || ring_tiles(kPT) < (long long)ctx->sm_count * 16) ? 16 : kPT;
    if (ctx->tile_pt == 16 || ctx->tile_pt == 32) pt = ctx->tile_pt;
    if (const char *env = getenv("PPM_PHASE_TILE")) {
        const int v = atoi(env);
        if (v == 16 || v == 32) pt = v;
    }
    hp.pt = pt;
    // ring groups sized by work (elements x phases x energies), aiming at
    // tile_waves (default 16) waves of 2 blocks per SM; instances of very
    // different resolution then give items of comparable cost
    const double nE = (double)ctx->E.size();
    double total = 0.0;
    for (int b = 0; b < B; ++b)
        total += (double)p->n_spots * rings_per_spot(res, b) * slots_per_ring(res, b) *
                 res->n_phase[b] * res->phase_sub * nE;
    const double target =
        std::max(1.0, total / ((double)ctx->sm_count * 2.0 * (double)ctx->tile_waves));
    hp.inst.resize(B);
    long long pix = 0;  // temperature-map offset (HEALPix: 12 N^2 pixels per instance)
    for (int b = 0; b < B; ++b) {
        InstPlan &ip = hp.inst[b];
        ip.n_theta = rings_per_spot(res, b);
        ip.n_phi = slots_per_ring(res, b);
        ip.n_phase = res->n_phase[b];
        ip.n_sub = res->phase_sub;
        ip.pix0 = (int)pix;
        if (res->grid == PPM_GRID_HEALPIX) pix += 12LL * res->n_theta[b] * res->n_theta[b];
        const int nq = ip.n_phase * ip.n_sub;  // point samples (pt is a multiple of n_sub)
        ip.ring0 = hp.total_rings;
        ip.elem0 = (int)hp.total_elems;
        ip.row0 = hp.total_rows;
        ip.tiles = (nq + pt - 1) / pt;
        ip.tile0 = (int)hp.tiles.size();
        hp.total_rings += p->n_spots * ip.n_theta;
        hp.total_elems += (size_t)p->n_spots * ip.n_theta * ip.n_phi;
        hp.total_rows += ip.n_phase;
        hp.n_phi_max = std::max(hp.n_phi_max, ip.n_phi);
        const double ring_cost = (double)ip.n_phi * std::min(pt, nq) * nE;
        const int gb = (int)std::min<double>(ip.n_theta, std::max(1.0, std::floor(target / ring_cost)));
        for (int t = 0; t < ip.tiles; ++t) {
            const int begin = (int)hp.items.size();
            for (int s = 0; s < p->n_spots; ++s)
                for (int r0 = 0; r0 < ip.n_theta; r0 += gb) {
                    Item it;
                    it.b = b; it.spot = s; it.r0 = r0; it.r1 = std::min(r0 + gb, ip.n_theta);
                    it.j0 = t * pt; it.nj = std::min(pt, nq - t * pt);
                    hp.items.push_back(it);
                }
            hp.tiles.push_back(make_int2(begin, (int)hp.items.size()));
        }
    }
    if (hp.total_elems > (size_t)INT32_MAX || pix > (long long)INT32_MAX)
        return fail(ctx, PPM_EINVAL, "problem too large");
    // launch order: largest items first (longest-processing-time heuristic)
    hp.order.resize(hp.items.size());
    {
        std::vector<std::pair<double, int>> c(hp.items.size());
        for (size_t i = 0; i < hp.items.size(); ++i) {
            const Item &it = hp.items[i];
            c[i] = {-(double)(it.r1 - it.r0) * hp.inst[it.b].n_phi * it.nj, (int)i};
        }
        std::stable_sort(c.begin(), c.end());
        for (size_t i = 0; i < c.size(); ++i) hp.order[i] = c[i].second;
    }
    const size_t b_inst = align256(hp.inst.size() * sizeof(InstPlan));
    const size_t b_items = align256(hp.items.size() * sizeof(Item));
    const size_t b_tiles = align256(hp.tiles.size() * sizeof(int2));
    const size_t b_order = align256(hp.order.size() * sizeof(int));
    const size_t bytes = b_inst + b_items + b_tiles + b_order;
    // the pinned staging buffer may still feed the previous upload
    PPM_CUDA(cudaEventSynchronize(ctx->plan_ev), "plan event");
    if (ctx->h_pinned_n < bytes) {
        if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
        ctx->h_pinned = nullptr;
        ctx->h_pinned_n = 0;
        PPM_CUDA(cudaMallocHost(&ctx->h_pinned, bytes), "pinned plan buffer");
        ctx->h_pinned_n = bytes;
    }
    char *h = static_cast<char *>(ctx->h_pinned);
    memcpy(h, hp.inst.data(), hp.inst.size() * sizeof(InstPlan));
    memcpy(h + b_inst, hp.items.data(), hp.items.size() * sizeof(Item));
    memcpy(h + b_inst + b_items, hp.tiles.data(), hp.tiles.size() * sizeof(int2));
    memcpy(h + b_inst + b_items + b_tiles, hp.order.data(), hp.order.size() * sizeof(int));
    if (ctx->d_plan.n < bytes) {
        PPM_CUDA(cudaDeviceSynchronize(), "sync");
        PPM_CUDA(ctx->d_plan.ensure(bytes), "alloc plan");
    }
    PPM_CUDA(cudaMemcpyAsync(ctx->d_plan.p, h, bytes, cudaMemcpyHostToDevice, st), "upload plan");
    PPM_CUDA(cudaEventRecord(ctx->plan_ev, st), "plan event");
    ctx->plan = std::move(hp);
    ctx->plan_key = std::move(key);
    ctx->plan_grid = res->grid;
    return PPM_OK;
}

namespace {
struct Work {
    int *status;
    RingRec *recs;
    float *tmpl, *elems, *partials, *Ft;
    float2 *elemx;  // temperature maps only
    double *row_ll;
    // gradient only
    float *lambda, *Aadj, *ringadj;
    double *ring_grad, *row_sums;
    int *used;  // temperature maps: which work slots wrote a partial tile
};
}  // namespace

static ppm_status ensure_workspace(ppm_ctx *ctx, const ppm_params *p, int n_fp, bool need_ft,
                                   bool grad, Work *w)
{
    const HostPlan &hp = ctx->plan;
    const int ct = ctx->nc ? loglike_ctiles(ctx->nc) : 1;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += align256(bytes); return o; };
    const size_t o_status = take((size_t)p->B * sizeof(int));
    const size_t o_recs = take((size_t)hp.total_rings * sizeof(RingRec));
    const size_t o_tmpl = take((size_t)hp.total_rings * 4 * (n_fp + 1) * sizeof(float));
    const size_t o_elems = take(hp.total_elems * sizeof(float));
    const size_t o_elemx = take(p->logT_map ? hp.total_elems * sizeof(float2) : 0);
    const size_t parts = p->logT_map ? 2 : 1;
    const size_t o_part = take(parts * hp.items.size() * hp.pt * ctx->nEpad * sizeof(float));
    const size_t o_used = take(parts > 1 ? parts * hp.items.size() * sizeof(int) : 0);
    const size_t o_ft = take(need_ft ? (size_t)hp.total_rows * ctx->E.size() * sizeof(float) : 0);
    const size_t o_ll = take(need_ft ? (size_t)hp.total_rows * ct * sizeof(double) : 0);
    const size_t rows = grad ? (size_t)hp.total_rows : 0, rings = grad ? hp.total_rings : 0;
    const size_t o_lam = take(rows * ctx->nc * sizeof(float));
    const size_t o_aadj = take(rows * ctx->nEpad * sizeof(float));
    const size_t o_radj = take(rings * (4 * (n_fp + 1) + kRingAdjTail) * sizeof(float));
    const size_t o_rgrad = take(rings * kRingGrad * sizeof(double));
    const size_t o_rsum = take(rows * grad_ktiles(ctx->nEpad) * 2 * sizeof(double));
    if (off > ctx->ws.n) {
        PPM_CUDA(cudaDeviceSynchronize(), "sync");
        PPM_CUDA(ctx->ws.ensure(off), "alloc workspace");
    }
    char *base = ctx->ws.as<char>();
    w->status = reinterpret_cast<int *>(base + o_status);
    w->recs = reinterpret_cast<RingRec *>(base + o_recs);
    w->tmpl = reinterpret_cast<float *>(base + o_tmpl);
    w->elems = reinterpret_cast<float *>(base + o_elems);
    w->elemx = p->logT_map ? reinterpret_cast<float2 *>(base + o_elemx) : nullptr;
    w->partials = reinterpret_cast<float *>(base + o_part);
    w->used = parts > 1 ? reinterpret_cast<int *>(base + o_used) : nullptr;
    w->Ft = reinterpret_cast<float *>(base + o_ft);
    w->row_ll = reinterpret_cast<double *>(base + o_ll);
    w->lambda = reinterpret_cast<float *>(base + o_lam);
    w->Aadj = reinterpret_cast<float *>(base + o_aadj);
    w->ringadj = reinterpret_cast<float *>(base + o_radj);
    w->ring_grad = reinterpret_cast<double *>(base + o_rgrad);
    w->row_sums = reinterpret_cast<double *>(base + o_rsum);
    return PPM_OK;
}

// the mu lookups of the table (AtmDev.mu_idx, mu_rden, mu_rlin, mu_bin)
static void set_mu_lookups(const ppm_ctx *ctx, AtmDev *A)
{
    const char *base = ctx->d_mu_aux.as<char>();
    const size_t o_rden = kMuBins * sizeof(int);
    if (!base) {  // no atmosphere table
        A->mu_idx = nullptr; A->mu_rden = nullptr; A->mu_rlin = nullptr; A->mu_bin = 0.0f;
        return;
    }
    A->mu_idx = reinterpret_cast<const int *>(base);
    A->mu_rden = reinterpret_cast<const float4 *>(base + o_rden);
    A->mu_rlin = reinterpret_cast<const float *>(base + o_rden + 16 * (size_t)ctx->nmu);
    A->mu_bin = ctx->mu_bin;
}

static void fill_devs(ppm_ctx *ctx, const ppm_params *p, int n_fp, Params *P, PlanDev *plan,
                      LensDev *L, AtmDev *A, EnergyDev *en)
{
    P->B = p->B; P->n_spots = p->n_spots; P->oblate = p->oblate; P->emission = p->emission;
    P->mass_msun = p->mass_msun; P->radius_km = p->radius_km; P->spin_hz = p->spin_hz;
    P->incl_rad = p->incl_rad; P->dist_kpc = p->dist_kpc; P->nh_1e20 = p->nh_1e20;
    P->colat = p->colat; P->azim = p->azim; P->zeta = p->zeta; P->logT = p->logT;
    P->mask_colat = p->mask_colat; P->mask_azim = p->mask_azim; P->mask_zeta = p->mask_zeta;
    P->logT_map = p->logT_map;
    const HostPlan &hp = ctx->plan;
    const size_t b_inst = align256(hp.inst.size() * sizeof(InstPlan));
    const size_t b_items = align256(hp.items.size() * sizeof(Item));
    char *d = ctx->d_plan.as<char>();
    plan->B = p->B; plan->n_fp = n_fp; plan->n_items = (int)hp.items.size(); plan->pt = hp.pt;
    plan->grid = ctx->plan_grid;
    plan->total_rings = hp.total_rings;
    plan->inst = reinterpret_cast<const InstPlan *>(d);
    plan->items = reinterpret_cast<const Item *>(d + b_inst);
    plan->tile_items = reinterpret_cast<const int2 *>(d + b_inst + b_items);
    plan->order = reinterpret_cast<const int *>(
        d + b_inst + b_items + align256(hp.tiles.size() * sizeof(int2)));
    plan->queue = ctx->tile_persistent ? ctx->d_queue : nullptr;
    plan->err = ctx->d_err;
    plan->parts = 1;
    plan->used = nullptr;
    const ppm_lens_spec &s = ctx->lens;
    L->u_min = s.u_min; L->u_max = s.u_max; L->n_u = s.n_u;
    L->cpsi_min = s.cpsi_min; L->cpsi_max = s.cpsi_max; L->n_cpsi = s.n_cpsi;
    L->ca_min = s.calpha_min; L->ca_max = s.calpha_max; L->n_calpha = s.n_calpha;
    L->Ca = ctx->d_Ca.as<double>(); L->LF = ctx->d_LF.as<double>(); L->TD = ctx->d_TD.as<double>();
    A->nT = ctx->nT; A->ng = ctx->ng; A->nmu = ctx->nmu; A->nE = ctx->nEt;
    A->n_protect = ctx->n_protect; A->nmu_pad = ctx->nmu_pad; A->strategy = ctx->interp;
    A->I = ctx->d_I.as<float>(); A->logT = ctx->d_logT.as<double>();
    A->logg = ctx->d_logg.as<double>(); A->mu = ctx->d_mu.as<float>();
    set_mu_lookups(ctx, A);
    A->lnE0 = ctx->lnE0_t; A->dlnE = ctx->dlnE_t;
    en->nE = (int)ctx->E.size(); en->nEpad = ctx->nEpad;
    en->E = ctx->d_E.as<float>(); en->E3 = ctx->d_E3.as<float>();
    en->pk = ctx->d_pk.as<float>(); en->invE = ctx->d_invE.as<float>();
    en->sliding = ctx->sliding;
    en->step = node_walk_on(ctx, p, ctx->walk_step) ? ctx->walk_step : 0.0f;
    en->inv_step = en->step > 0.0f ? 1.0f / en->step : 0.0f;
    en->moments = moment_walk_on(ctx, p) ? 1 : 0;
    en->nmom = moment_rows(ctx);
}

static ppm_status run_profile(ppm_ctx *ctx, const ppm_params *p, const ppm_res *res, float *Ft,
                              bool internal_ft, cudaStream_t st, Work *w, bool grad = false)
{
    ppm_status s = check_params(ctx, p, res);
    if (s != PPM_OK) return s;
    if ((s = refresh_energies(ctx)) != PPM_OK) return s;
    if ((s = make_plan(ctx, p, res, st)) != PPM_OK) return s;
    if ((s = ensure_workspace(ctx, p, res->n_fp, internal_ft, grad, w)) != PPM_OK) return s;
    Params P;
    PlanDev plan;
    LensDev L;
    AtmDev A;
    EnergyDev en;
    fill_devs(ctx, p, res->n_fp, &P, &plan, &L, &A, &en);
    plan.parts = p->logT_map ? 2 : 1;
    plan.used = w->used;
    // shared-memory budget of the shift-and-add kernel
    const size_t smem = shift_add_smem_bytes(P, plan, A, en, ctx->plan.n_phi_max, ctx->smem_optin);
    if (smem > ctx->smem_optin)
        return fail(ctx, PPM_EINVAL, "shared memory need %zu B exceeds %zu B (n_phi, nE too large)",
                    smem, ctx->smem_optin);
    if (internal_ft) Ft = w->Ft;
    PPM_CUDA(cudaMemsetAsync(w->status, 0, sizeof(int) * p->B, st), "memset status");
    {
        StageTimer t(ctx, 0, st);
        PPM_CUDA(launch_ring(P, plan, L, A, w->recs, w->tmpl, w->elems, w->status, ctx->d_err,
                             ctx->timing ? ctx->d_triples : nullptr, (int)ctx->E.size(), st,
                             w->elemx),
                 "ring kernel");
        t.done(1);
    }
    {
        StageTimer t(ctx, 1, st);
        PPM_CUDA(launch_shift_add(P, plan, A, en, w->recs, w->tmpl, w->elems, w->status,
                                  w->partials, ctx->plan.n_phi_max, st, 2 * ctx->sm_count,
                                  w->elemx, ctx->smem_optin),
                 "shift-and-add kernel");
        t.done(1);
    }
    {
        StageTimer t(ctx, 2, st);
        PPM_CUDA(launch_reduce(plan, en, w->partials, w->status, ctx->plan.total_rows, Ft, st),
                 "reduce kernel");
        t.done(1);
    }
    if (ctx->timing) ctx->acc.calls += 1;
    return PPM_OK;
}

ppm_status ppm_profile(ppm_ctx *ctx, const ppm_params *p, const ppm_res *res, float *Ft,
                       int *inst_status, void *stream)
{
    NvtxCall nvtx_("ppm_profile");
    if (!ctx) return PPM_EINVAL;
    if (!Ft) return fail(ctx, PPM_EINVAL, "null Ft");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    Work w;
    ppm_status s = run_profile(ctx, p, res, Ft, false, st, &w);
    if (s != PPM_OK) return s;
    if (inst_status)
        PPM_CUDA(cudaMemcpyAsync(inst_status, w.status, sizeof(int) * p->B,
                                 cudaMemcpyDeviceToDevice, st),
                 "copy status");
    ctx->err.clear();
    return PPM_OK;
}

static ppm_status check_loglike_args(ppm_ctx *ctx, const ppm_params *p, const ppm_res *res,
                                     const int *counts, int counts_shared, double tau,
                                     const double *logL)
{
    if (!counts || !logL) return fail(ctx, PPM_EINVAL, "null counts or logL");
    if (!ctx->nc) return fail(ctx, PPM_EINVAL, "response not set");
    if (!(tau > 0.0) || !std::isfinite(tau)) return fail(ctx, PPM_EINVAL, "tau must be positive");
    if (p && res && counts_shared && p->B > 0 && res->n_phase)
        for (int b = 1; b < p->B; ++b)
            if (res->n_phase[b] != res->n_phase[0])
                return fail(ctx, PPM_EINVAL, "shared counts need equal n_phase");
    return PPM_OK;
}

// response contraction + likelihood of the profile in w.Ft
static ppm_status run_loglike(ppm_ctx *ctx, const ppm_params *p, const ppm_res *res,
                              const int *counts, int counts_shared, const float *bkg, double tau,
                              double *logL, float *model_counts, cudaStream_t st, const Work &w)
{
    Params P;
    PlanDev plan;
    LensDev L;
    AtmDev A;
    EnergyDev en;
    fill_devs(ctx, p, res->n_fp, &P, &plan, &L, &A, &en);
    // tensor cores for large row counts (batches); the FP32 tile kernel
    // has lower latency for a few hundred rows
    bool use_tc = ctx->plan.total_rows >= 512;
    if (const char *env = getenv("PPM_RESP_TC")) use_tc = atoi(env) != 0;
    StageTimer t(ctx, 3, st);
    if (use_tc) {
        PPM_CUDA(launch_loglike_tc(P, plan, w.Ft, ctx->plan.total_rows, (int)ctx->E.size(),
                                   ctx->d_Rtc.as<uint16_t>(), ctx->d_sigma.as<float>(), ctx->nc,
                                   counts, counts_shared, bkg, tau, w.status, ctx->d_lfact,
                                   w.row_ll, model_counts, ctx->d_err, st),
                 "tensor-core likelihood kernel");
        launch_ll_final(plan, w.row_ll, resp_tc_ctiles(ctx->nc), w.status, logL, st);
        PPM_CUDA(cudaGetLastError(), "likelihood reduction");
    } else {
        PPM_CUDA(launch_loglike(P, plan, w.Ft, ctx->plan.total_rows, (int)ctx->E.size(),
                                ctx->d_R.as<float>(), ctx->d_sigma.as<float>(), ctx->nc, counts,
                                counts_shared, bkg, tau, w.status, ctx->d_lfact, w.row_ll,
                                model_counts, logL, st),
                 "likelihood kernels");
    }
    t.done(2);
    return PPM_OK;
}

ppm_status ppm_loglike(ppm_ctx *ctx, const ppm_params *p, const ppm_res *res, const int *counts,
                       int counts_shared, const float *bkg, double tau, double *logL,
                       float *model_counts, int *inst_status, void *stream)
{
    NvtxCall nvtx_("ppm_loglike");
    if (!ctx) return PPM_EINVAL;
    ppm_status s = check_loglike_args(ctx, p, res, counts, counts_shared, tau, logL);
    if (s != PPM_OK) return s;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    Work w;
    if ((s = run_profile(ctx, p, res, nullptr, true, st, &w)) != PPM_OK) return s;
    if ((s = run_loglike(ctx, p, res, counts, counts_shared, bkg, tau, logL, model_counts, st,
                         w)) != PPM_OK)
        return s;
    if (inst_status)
        PPM_CUDA(cudaMemcpyAsync(inst_status, w.status, sizeof(int) * p->B,
                                 cudaMemcpyDeviceToDevice, st),
                 "copy status");
    ctx->err.clear();
    return PPM_OK;
}

ppm_status ppm_loglike_grad(ppm_ctx *ctx, const ppm_params *p, const ppm_res *res,
                            const int *counts, int counts_shared, const float *bkg, double tau,
                            double *logL, double *grad, int *inst_status, void *stream)
{
    NvtxCall nvtx_("ppm_loglike_grad");
    if (!ctx) return PPM_EINVAL;
    ppm_status s = check_loglike_args(ctx, p, res, counts, counts_shared, tau, logL);
    if (s != PPM_OK) return s;
    if (!grad) return fail(ctx, PPM_EINVAL, "null grad");
    if (res && res->grid != PPM_GRID_SPOT)
        return fail(ctx, PPM_EINVAL, "the gradient needs the spot grid (PPM_GRID_SPOT)");
    if (p && p->logT_map)
        return fail(ctx, PPM_EINVAL, "the gradient does not support temperature maps");
    if ((s = check_params(ctx, p, res)) != PPM_OK) return s;
    if ((s = refresh_energies(ctx)) != PPM_OK) return s;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    {
        // the backward shift-and-add holds the slab and its two cell-weight
        // derivatives; check its shared memory before any work is enqueued
        PlanDev pd{};
        pd.n_fp = res->n_fp;
        AtmDev A{};
        A.nmu = ctx->nmu;
        A.nE = ctx->nEt;
        A.nmu_pad = ctx->nmu_pad;
        EnergyDev en{};
        en.nEpad = ctx->nEpad;
        int n_phi_max = 0;
        for (int b = 0; b < p->B; ++b) n_phi_max = std::max(n_phi_max, res->n_phi[b]);
        const size_t need = shift_add_bwd_smem_bytes(p->emission, pd, A, en, n_phi_max);
        if (need > ctx->smem_optin)
            return fail(ctx, PPM_EINVAL,
                        "gradient needs %zu B of shared memory per block (three nE x nmu "
                        "slabs); the device allows %zu B",
                        need, ctx->smem_optin);
    }
    Work w;
    if ((s = run_profile(ctx, p, res, nullptr, true, st, &w, true)) != PPM_OK) return s;
    if ((s = run_loglike(ctx, p, res, counts, counts_shared, bkg, tau, logL, w.lambda, st, w)) !=
        PPM_OK)
        return s;
    Params P;
    PlanDev plan;
    LensDev L;
    AtmDev A;
    EnergyDev en;
    fill_devs(ctx, p, res->n_fp, &P, &plan, &L, &A, &en);
    const HostPlan &hp = ctx->plan;
    {
        StageTimer t(ctx, 4, st);
        PPM_CUDA(launch_grad_resp(P, plan, w.Ft, hp.total_rows, en, ctx->d_R.as<float>(),
                                  ctx->d_sigma.as<float>(), ctx->nc, counts, counts_shared, bkg,
                                  tau, w.lambda, w.status, w.Aadj, w.row_sums, st),
                 "response adjoint kernel");
        t.done(1);
    }
    {
        StageTimer t(ctx, 5, st);
        PPM_CUDA(launch_shift_add_bwd(P, plan, A, en, w.recs, w.tmpl, w.elems, w.status, w.Aadj,
                                      w.ringadj, hp.n_phi_max, st, ctx->smem_optin),
                 "backward shift-and-add kernel");
        t.done(1);
    }
    {
        StageTimer t(ctx, 6, st);
        PPM_CUDA(launch_template_bwd(P, plan, L, A, w.recs, w.tmpl, w.status, w.ringadj,
                                     w.ring_grad, st),
                 "template tangent kernel");
        PPM_CUDA(launch_grad_final(P, plan, w.ring_grad, w.row_sums, grad_ktiles(en.nEpad),
                                   w.status, logL, grad, st),
                 "gradient reduction kernel");
        t.done(2);
    }
    if (inst_status)
        PPM_CUDA(cudaMemcpyAsync(inst_status, w.status, sizeof(int) * p->B,
                                 cudaMemcpyDeviceToDevice, st),
                 "copy status");
    ctx->err.clear();
    return PPM_OK;
}

ppm_status ppm_set_tiles(ppm_ctx *ctx, const ppm_tiles *t)
{
    if (!ctx || !t) return fail(ctx, PPM_EINVAL, "null argument");
    if (!(t->phase_tile == 0 || t->phase_tile == 16 || t->phase_tile == 32))
        return fail(ctx, PPM_EINVAL, "phase_tile must be 0, 16 or 32");
    if (t->waves < 1 || t->waves > 256) return fail(ctx, PPM_EINVAL, "waves must be in [1, 256]");
    if (t->persistent != 0 && t->persistent != 1)
        return fail(ctx, PPM_EINVAL, "persistent must be 0 or 1");
    if (t->walk < 0 || t->walk > 2) return fail(ctx, PPM_EINVAL, "walk must be 0, 1 or 2");
    ctx->tile_pt = t->phase_tile;
    ctx->tile_waves = t->waves;
    ctx->tile_persistent = t->persistent;
    ctx->tile_walk = t->walk;
    return PPM_OK;
}

ppm_status ppm_get_tiles(ppm_ctx *ctx, ppm_tiles *t)
{
    if (!ctx || !t) return fail(ctx, PPM_EINVAL, "null argument");
    t->phase_tile = ctx->tile_pt;
    t->waves = ctx->tile_waves;
    t->persistent = ctx->tile_persistent;
    t->walk = ctx->tile_walk;
    t->ms = 0.0;
    return PPM_OK;
}

ppm_status ppm_autotune(ppm_ctx *ctx, const ppm_params *p, const ppm_res *res, void *stream,
                        ppm_tiles *best)
{
    if (!ctx) return PPM_EINVAL;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const bool timing = ctx->timing;
    ctx->timing = false;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PPM_CUDA(cudaEventCreate(&e0), "event");
    PPM_CUDA(cudaEventCreate(&e1), "event");
    ppm_tiles cur{ctx->tile_pt, ctx->tile_waves, ctx->tile_persistent, ctx->tile_walk, 0.0};
    ppm_tiles top = cur;
    top.ms = INFINITY;
    ppm_status s = PPM_OK;
    const int pts[] = {16, 32}, waves[] = {8, 16, 32, 64}, pers[] = {0, 1};
    for (int a : pts)
        for (int wv : waves)
            for (int q : pers) {
                if (s != PPM_OK) break;
                ctx->tile_pt = a;
                ctx->tile_waves = wv;
                ctx->tile_persistent = q;
                Work w;
                // one untimed pass (plan, workspace), then one timed pass
                for (int rep = 0; rep < 2 && s == PPM_OK; ++rep) {
                    if (rep == 1 && cudaEventRecord(e0, st) != cudaSuccess) s = PPM_ECUDA;
                    if (s == PPM_OK) s = run_profile(ctx, p, res, nullptr, true, st, &w);
                    if (rep == 1 && s == PPM_OK && cudaEventRecord(e1, st) != cudaSuccess)
                        s = PPM_ECUDA;
                }
                if (s != PPM_OK) break;
                float ms = 0.0f;
                if (cudaEventSynchronize(e1) != cudaSuccess ||
                    cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                    s = fail(ctx, PPM_ECUDA, "autotune timing failed");
                    break;
                }
                if (ms < top.ms) top = ppm_tiles{a, wv, q, ctx->tile_walk, (double)ms};
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->timing = timing;
    if (s != PPM_OK) {
        ctx->tile_pt = cur.phase_tile;
        ctx->tile_waves = cur.waves;
        ctx->tile_persistent = cur.persistent;
        return s;
    }
    ctx->tile_pt = top.phase_tile;
    ctx->tile_waves = top.waves;
    ctx->tile_persistent = top.persistent;
    if (best) *best = top;
    ctx->err.clear();
    return PPM_OK;
}

ppm_status ppm_set_timing(ppm_ctx *ctx, int enable)
{
    if (!ctx) return PPM_EINVAL;
    DeviceGuard g(ctx->device);
    if (!ctx->d_triples) PPM_CUDA(cudaMalloc(&ctx->d_triples, sizeof(unsigned long long)), "alloc");
    PPM_CUDA(cudaDeviceSynchronize(), "sync");
    PPM_CUDA(cudaMemset(ctx->d_triples, 0, sizeof(unsigned long long)), "memset");
    for (auto &pd : ctx->pending) ctx->ev_pool.push_back(pd.a), ctx->ev_pool.push_back(pd.b);
    ctx->pending.clear();
    ctx->acc = ppm_timing{};
    ctx->timing = enable != 0;
    return PPM_OK;
}

ppm_status ppm_get_timing(ppm_ctx *ctx, ppm_timing *out)
{
    if (!ctx || !out) return fail(ctx, PPM_EINVAL, "null argument");
    DeviceGuard g(ctx->device);
    for (auto &pd : ctx->pending) {
        PPM_CUDA(cudaEventSynchronize(pd.b), "timing event");
        float ms = 0.0f;
        PPM_CUDA(cudaEventElapsedTime(&ms, pd.a, pd.b), "elapsed");
        double *slot[] = {&ctx->acc.ms_ring,         &ctx->acc.ms_shift_add,
                          &ctx->acc.ms_reduce,       &ctx->acc.ms_loglike,
                          &ctx->acc.ms_grad_resp,    &ctx->acc.ms_shift_add_bwd,
                          &ctx->acc.ms_template_bwd};
        *slot[pd.stage] += ms;
        ctx->ev_pool.push_back(pd.a);
        ctx->ev_pool.push_back(pd.b);
    }
    ctx->pending.clear();
    unsigned long long tr = 0;
    if (ctx->d_triples)
        PPM_CUDA(cudaMemcpy(&tr, ctx->d_triples, sizeof(tr), cudaMemcpyDeviceToHost), "read");
    ctx->acc.triples = (double)tr;
    *out = ctx->acc;
    return PPM_OK;
}

ppm_status ppm_sync(ppm_ctx *ctx, void *stream, double timeout_s)
{
    if (!ctx) return PPM_EINVAL;
    if (!(timeout_s > 0.0)) return fail(ctx, PPM_EINVAL, "timeout must be positive");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(st);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return cuda_fail(ctx, e, "stream");
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > timeout_s) return fail(ctx, PPM_ETIMEOUT, "stream not complete after %.3f s", el);
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    unsigned bits = 0;
    PPM_CUDA(cudaMemcpy(&bits, ctx->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost), "read error word");
    if (bits) {
        PPM_CUDA(cudaMemset(ctx->d_err, 0, sizeof(unsigned)), "clear error word");
        return fail(ctx, PPM_ENOTREADY, "device invariant failed (bits 0x%x%s%s%s)", bits,
                    (bits & kErrPhaseOrder) ? ": template observed phases not increasing" : "",
                    (bits & kErrTimeout) ? ": a bounded in-kernel wait timed out" : "",
                    (bits & kErrBounds) ? ": an index check failed" : "");
    }
    return PPM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free forward profile.
//
// Every per-call buffer of ppm_profile (plan, energy arrays, status, ring
// records, templates, element lists, partial sums) is carved out of one
// file-scope device array of fixed size instead of the context's growable
// workspace, and the host-side plan is assembled in a fixed static host
// buffer, so the call allocates neither device nor host memory.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocDeviceBytes = size_t(64) << 20;  // per device, held until exit
constexpr size_t kNoAllocHostBytes = size_t(1) << 20;     // host staging of plan + energies
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocDeviceBytes];

alignas(256) unsigned char g_noalloc_host[kNoAllocHostBytes];
void *g_noalloc_dev[kNoAllocMaxDevices];   // device address of the array, per device

// Sizes of one allocation-free plan (no containers: counts only).
struct NoAllocPlan {
    int pt, n_items, n_tiles, total_rings, total_rows, n_phi_max, nEpad;
    double target;  // work per item that sets the ring-group width
    long long widen;  // ring groups widened by this factor to fit the array
    size_t total_elems;
    size_t o_inst, o_items, o_tiles, host_bytes;        // host staging layout
    size_t o_E, o_E3, o_pk, o_invE;                     // (also mirrored on the device)
    size_t o_status, o_recs, o_tmpl, o_elems, o_part, device_bytes;
};

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// ring-group width of instance b: the rule of ppm_profile's plan (groups of
// about `target` element x phase x energy work per item), times L->widen
int noalloc_group(const ppm_ctx *ctx, const ppm_res *res, int b, const NoAllocPlan *L)
{
    const int nr = rings_per_spot(res, b);
    const int nq = res->n_phase[b] * res->phase_sub;
    const double ring_cost = (double)slots_per_ring(res, b) * std::min(L->pt, nq) *
                             (double)ctx->E.size();
    const double gb = std::max(1.0, std::floor(L->target / ring_cost));
    return (int)std::min<double>(nr, gb * (double)L->widen);
}

void noalloc_sizes(const ppm_ctx *ctx, const ppm_params *p, const ppm_res *res, NoAllocPlan *L)
{
    const int pt = L->pt;
    L->n_items = L->n_tiles = L->total_rings = L->total_rows = L->n_phi_max = 0;
    L->total_elems = 0;
    for (int b = 0; b < p->B; ++b) {
        const int nr = rings_per_spot(res, b), ns = slots_per_ring(res, b);
        const int tiles = (res->n_phase[b] * res->phase_sub + pt - 1) / pt;
        const int gb = noalloc_group(ctx, res, b, L);
        const int groups = (nr + gb - 1) / gb;
        L->n_tiles += tiles;
        L->n_items += tiles * p->n_spots * groups;
        L->total_rings += p->n_spots * nr;
        L->total_rows += res->n_phase[b];
        L->total_elems += (size_t)p->n_spots * nr * ns;
        L->n_phi_max = std::max(L->n_phi_max, ns);
    }
    const int nE = (int)ctx->E.size();
    L->nEpad = (nE + kEC - 1) / kEC * kEC;
    size_t o = 0;
    L->o_inst = o; o += a256((size_t)p->B * sizeof(InstPlan));
    L->o_items = o; o += a256((size_t)L->n_items * sizeof(Item));
    L->o_tiles = o; o += a256((size_t)L->n_tiles * sizeof(int2));
    L->o_E = o; o += a256((size_t)L->nEpad * sizeof(float));
    L->o_E3 = o; o += a256((size_t)L->nEpad * sizeof(float));
    L->o_pk = o; o += a256((size_t)L->nEpad * sizeof(float));
    L->o_invE = o; o += a256((size_t)L->nEpad * sizeof(float));
    L->host_bytes = o;
    L->o_status = o; o += a256((size_t)p->B * sizeof(int));
    L->o_recs = o; o += a256((size_t)L->total_rings * sizeof(RingRec));
    L->o_tmpl = o; o += a256((size_t)L->total_rings * 4 * (res->n_fp + 1) * sizeof(float));
    L->o_elems = o; o += a256(L->total_elems * sizeof(float));
    L->o_part = o; o += a256((size_t)L->n_items * pt * L->nEpad * sizeof(float));
    L->device_bytes = o;
}

}  // namespace

extern "C" ppm_status ppm_profile_noalloc(ppm_ctx *ctx, const ppm_params *p, const ppm_res *res,
                                          float *Ft, int *inst_status, void *stream)
{
    if (!ctx) return PPM_EINVAL;
    if (!Ft) return fail(ctx, PPM_EINVAL, "null Ft");
    ppm_status s = check_params(ctx, p, res);
    if (s != PPM_OK) return s;
    if (p->logT_map)
        return fail(ctx, PPM_EINVAL, "ppm_profile_noalloc does not support temperature maps");
    if (ctx->device < 0 || ctx->device >= kNoAllocMaxDevices)
        return fail(ctx, PPM_EINVAL, "device index beyond %d", kNoAllocMaxDevices);
    DeviceGuard guard(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    // the plan is uploaded from a static host buffer that the next call
    // rewrites: a stream being captured is refused before anything is enqueued
    {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        const cudaError_t e = cudaStreamIsCapturing(st, &cs);
        if (e != cudaSuccess) cudaGetLastError();
        if (e != cudaSuccess || cs != cudaStreamCaptureStatusNone)
            return fail(ctx, PPM_EINVAL,
                        "ppm_profile_noalloc refuses a stream that is being captured");
    }
    // one-time set-up on this device (the current device is ctx->device here)
    if (!g_noalloc_dev[ctx->device]) {
        void *ptr = nullptr;
        PPM_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch), "scratch symbol address");
        g_noalloc_dev[ctx->device] = ptr;
    }
    unsigned char *dev = static_cast<unsigned char *>(g_noalloc_dev[ctx->device]);

    // plan: ppm_profile's phase tile and ring-group rules with the context's
    // tile settings (so that the items, and hence the sums, are the same as
    // ppm_profile's), the ring groups widened by 2, 4, ... only when the
    // per-call buffers would not fit the fixed device array; no persistent
    // queue, items launched in plan order
    long long T32 = 0;
    int max_theta = 1;
    double total = 0.0;
    for (int b = 0; b < p->B; ++b) {
        T32 += (long long)p->n_spots * rings_per_spot(res, b) *
               ((res->n_phase[b] * res->phase_sub + kPT - 1) / kPT);
        max_theta = std::max(max_theta, rings_per_spot(res, b));
        total += (double)p->n_spots * rings_per_spot(res, b) * slots_per_ring(res, b) *
                 res->n_phase[b] * res->phase_sub * (double)ctx->E.size();
    }
    const float step = walk_step_of(ctx);
    int pt = (node_walk_on(ctx, p, step) || moment_walk_on(ctx, p) ||
              T32 < (long long)ctx->sm_count * 16) ? 16 : kPT;
    if (ctx->tile_pt == 16 || ctx->tile_pt == 32) pt = ctx->tile_pt;
    if (const char *env = getenv("PPM_PHASE_TILE")) {
        const int v = atoi(env);
        if (v == 16 || v == 32) pt = v;
    }
    NoAllocPlan L;
    L.pt = pt;
    L.target = std::max(1.0, total / ((double)ctx->sm_count * 2.0 * (double)ctx->tile_waves));
    for (L.widen = 1;; L.widen *= 2) {
        noalloc_sizes(ctx, p, res, &L);
        if (L.device_bytes <= kNoAllocDeviceBytes || L.widen >= max_theta) break;
    }
    if (L.device_bytes > kNoAllocDeviceBytes)
        return fail(ctx, PPM_EINVAL,
                    "problem needs %zu bytes of scratch; ppm_profile_noalloc is limited to %zu",
                    L.device_bytes, kNoAllocDeviceBytes);
    if (L.host_bytes > kNoAllocHostBytes)
        return fail(ctx, PPM_EINVAL, "plan needs %zu bytes of host staging; limit %zu",
                    L.host_bytes, kNoAllocHostBytes);

    // host staging: instance table, items, tile ranges, energy arrays
    unsigned char *h = g_noalloc_host;
    InstPlan *hi = reinterpret_cast<InstPlan *>(h + L.o_inst);
    Item *hit = reinterpret_cast<Item *>(h + L.o_items);
    int2 *ht = reinterpret_cast<int2 *>(h + L.o_tiles);
    int rings = 0, rows = 0, items = 0, tiles = 0;
    size_t elems = 0;
    for (int b = 0; b < p->B; ++b) {
        InstPlan &ip = hi[b];
        ip.n_theta = rings_per_spot(res, b);
        ip.n_phi = slots_per_ring(res, b);
        ip.n_phase = res->n_phase[b];
        ip.pix0 = 0;
        ip.n_sub = res->phase_sub;
        const int nq = ip.n_phase * ip.n_sub;
        ip.ring0 = rings;
        ip.elem0 = (int)elems;
        ip.row0 = rows;
        ip.tiles = (nq + pt - 1) / pt;
        ip.tile0 = tiles;
        rings += p->n_spots * ip.n_theta;
        elems += (size_t)p->n_spots * ip.n_theta * ip.n_phi;
        rows += ip.n_phase;
        const int gb = noalloc_group(ctx, res, b, &L);
        for (int t = 0; t < ip.tiles; ++t) {
            const int begin = items;
            for (int sp = 0; sp < p->n_spots; ++sp)
                for (int r0 = 0; r0 < ip.n_theta; r0 += gb) {
                    Item &it = hit[items++];
                    it.b = b; it.spot = sp; it.r0 = r0; it.r1 = std::min(r0 + gb, ip.n_theta);
                    it.j0 = t * pt; it.nj = std::min(pt, nq - t * pt);
                }
            ht[tiles++] = make_int2(begin, items);
        }
    }
    if (elems > (size_t)INT32_MAX) return fail(ctx, PPM_EINVAL, "problem too large");
    const int nE = (int)ctx->E.size();
    float *hE = reinterpret_cast<float *>(h + L.o_E), *hE3 = reinterpret_cast<float *>(h + L.o_E3);
    float *hpk = reinterpret_cast<float *>(h + L.o_pk);
    float *hinv = reinterpret_cast<float *>(h + L.o_invE);
    for (int k = 0; k < L.nEpad; ++k) {
        const double e = ctx->E[std::min(k, nE - 1)];
        hE[k] = (float)e;
        hE3[k] = (float)(e * e * e);
        hinv[k] = (float)(1.0 / e);
        hpk[k] = pk_of(ctx, std::min(k, nE - 1));
    }
    const int sliding = sliding_of(ctx);

    Params P;
    P.B = p->B; P.n_spots = p->n_spots; P.oblate = p->oblate; P.emission = p->emission;
    P.mass_msun = p->mass_msun; P.radius_km = p->radius_km; P.spin_hz = p->spin_hz;
    P.incl_rad = p->incl_rad; P.dist_kpc = p->dist_kpc; P.nh_1e20 = p->nh_1e20;
    P.colat = p->colat; P.azim = p->azim; P.zeta = p->zeta; P.logT = p->logT;
    P.mask_colat = p->mask_colat; P.mask_azim = p->mask_azim; P.mask_zeta = p->mask_zeta;
    P.logT_map = nullptr;
    PlanDev plan;
    plan.B = p->B; plan.n_fp = res->n_fp; plan.n_items = L.n_items; plan.grid = res->grid;
    plan.total_rings = L.total_rings; plan.pt = L.pt;
    plan.inst = reinterpret_cast<const InstPlan *>(dev + L.o_inst);
    plan.items = reinterpret_cast<const Item *>(dev + L.o_items);
    plan.tile_items = reinterpret_cast<const int2 *>(dev + L.o_tiles);
    plan.order = nullptr;
    plan.queue = nullptr;
    plan.err = ctx->d_err;
    plan.parts = 1;
    plan.used = nullptr;
    const ppm_lens_spec &ls = ctx->lens;
    LensDev Ld;
    Ld.u_min = ls.u_min; Ld.u_max = ls.u_max; Ld.n_u = ls.n_u;
    Ld.cpsi_min = ls.cpsi_min; Ld.cpsi_max = ls.cpsi_max; Ld.n_cpsi = ls.n_cpsi;
    Ld.ca_min = ls.calpha_min; Ld.ca_max = ls.calpha_max; Ld.n_calpha = ls.n_calpha;
    Ld.Ca = ctx->d_Ca.as<double>(); Ld.LF = ctx->d_LF.as<double>(); Ld.TD = ctx->d_TD.as<double>();
    AtmDev A;
    A.nT = ctx->nT; A.ng = ctx->ng; A.nmu = ctx->nmu; A.nE = ctx->nEt;
    A.n_protect = ctx->n_protect; A.nmu_pad = ctx->nmu_pad; A.strategy = ctx->interp;
    A.I = ctx->d_I.as<float>(); A.logT = ctx->d_logT.as<double>();
    A.logg = ctx->d_logg.as<double>(); A.mu = ctx->d_mu.as<float>();
    set_mu_lookups(ctx, &A);
    A.lnE0 = ctx->lnE0_t; A.dlnE = ctx->dlnE_t;
    EnergyDev en;
    en.nE = nE; en.nEpad = L.nEpad; en.sliding = sliding;
    en.step = node_walk_on(ctx, p, step) ? step : 0.0f;
    en.inv_step = en.step > 0.0f ? 1.0f / en.step : 0.0f;
    en.moments = moment_walk_on(ctx, p) ? 1 : 0;
    en.nmom = moment_rows(ctx);
    en.E = reinterpret_cast<const float *>(dev + L.o_E);
    en.E3 = reinterpret_cast<const float *>(dev + L.o_E3);
    en.pk = reinterpret_cast<const float *>(dev + L.o_pk);
    en.invE = reinterpret_cast<const float *>(dev + L.o_invE);
    const size_t smem_need = shift_add_smem_bytes(P, plan, A, en, L.n_phi_max, ctx->smem_optin);
    if (smem_need > ctx->smem_optin)
        return fail(ctx, PPM_EINVAL, "shared memory need %zu B exceeds %zu B", smem_need,
                    ctx->smem_optin);
    int *status = reinterpret_cast<int *>(dev + L.o_status);
    RingRec *recs = reinterpret_cast<RingRec *>(dev + L.o_recs);
    float *tmpl = reinterpret_cast<float *>(dev + L.o_tmpl);
    float *el = reinterpret_cast<float *>(dev + L.o_elems);
    float *part = reinterpret_cast<float *>(dev + L.o_part);
    // pageable source: the copy has consumed the staging buffer when it
    // returns, which can mean waiting for the work already queued on st
    PPM_CUDA(cudaMemcpyAsync(dev, h, L.host_bytes, cudaMemcpyHostToDevice, st), "upload plan");
    // the array keeps the previous call's contents: status must start at zero
    PPM_CUDA(cudaMemsetAsync(dev + L.o_status, 0, sizeof(int) * p->B, st), "clear status");
    PPM_CUDA(launch_ring(P, plan, Ld, A, recs, tmpl, el, status, ctx->d_err, nullptr, nE, st),
             "ring kernel");
    PPM_CUDA(launch_shift_add(P, plan, A, en, recs, tmpl, el, status, part, L.n_phi_max, st, 0,
                              nullptr, ctx->smem_optin),
             "shift-and-add kernel");
    PPM_CUDA(launch_reduce(plan, en, part, status, L.total_rows, Ft, st), "reduce kernel");
    if (inst_status)
        PPM_CUDA(cudaMemcpyAsync(inst_status, status, sizeof(int) * p->B,
                                 cudaMemcpyDeviceToDevice, st),
                 "copy status");
    ctx->err.clear();
    return PPM_OK;
}
