// Internal declarations shared by the CUDA translation units of libppm.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ppm.h"

namespace ppm {

// ---- physical constants (CODATA 2018, IAU 2015 nominal GM_sun) -----------
constexpr double kGM_SUN = 1.32712440018e20;      // m^3 s^-2
constexpr double kC = 299792458.0;                // m s^-1
constexpr double kC_CM = 29979245800.0;           // cm s^-1
constexpr double kH_KEVS = 4.135667696e-18;       // keV s
constexpr double kKB_KEVK = 8.617333262e-8;       // keV K^-1
constexpr double kKPC_M = 3.0856775814913673e19;  // m
constexpr double kPI = 3.141592653589793238462643383279502884;

// Template fluxes are stored as F * kFluxScale so that the FP32 hot loop
// stays in the normal range for element areas down to ~1e-9 sr (R/D ~ 1e-15).
constexpr double kFluxScale = 1e30;

// Shift-and-add tiling: at most kPT output phases per work item (the plan
// picks 16 or 32), kEC energies per register chunk.
constexpr int kPT = 32;
constexpr int kEC = 16;
constexpr int kMaxFp = 1024;
constexpr int kSABlock = 256;

// device-side invariant failure bits (ctx error word)
enum : unsigned {
    kErrPhaseOrder = 1u,  // template observed phases not increasing
    kErrPlan = 2u,        // inconsistent plan (should not happen)
    kErrTimeout = 4u,     // a bounded wait inside a kernel gave up
    kErrBounds = 8u,      // an index check of the bounds-checked build failed
};

// Bounds-checked build (-DPPM_BOUNDS_CHECK, build(check=True)): table, slab
// and template gathers verify their indices and set kErrBounds in the
// context's error word (reported by ppm_sync); the ordinary build compiles
// the checks away.
#ifdef PPM_BOUNDS_CHECK
#define PPM_CHECK(cond, errp)                                   \
    do {                                                        \
        if (!(cond) && (errp)) atomicOr((errp), ppm::kErrBounds); \
    } while (0)
#else
#define PPM_CHECK(cond, errp) ((void)0)
#endif

struct LensDev {
    double u_min, u_max;
    int n_u;
    double cpsi_min, cpsi_max;
    int n_cpsi;
    double ca_min, ca_max;
    int n_calpha;
    const double *Ca, *LF, *TD;
};

// Interpolation strategies of Sect. 4 (PPM_INTERP_* in ppm.h):
//   D (0) the method's mixed scheme: linear in logT, logg; cubic in mu and
//         ln E, linear at the edges and on the protected small-mu intervals;
//   A (1) cubic in all four axes, one-sided four-node stencils at the edges;
//   B (2) A with negative interpolants clipped to zero;
//   C (3) cubic in all four axes with D's linear edge / protected-zone rules.
enum : int { kInterpD = 0, kInterpA = 1, kInterpB = 2, kInterpC = 3 };

struct AtmDev {
    int nT, ng, nmu, nE, n_protect, nmu_pad;
    int strategy;            // kInterp*
    const float *I;          // [nT][ng][nmu][nE]
    const double *logT;      // [nT]
    const double *logg;      // [ng]
    const float *mu;         // [nmu]
    double lnE0, dlnE;       // uniform ln E axis
    // mu lookups: mu_idx[b] an interval near the start of bin b of kMuBins
    // equal bins over [mu_0, mu_last] (mu_bin = kMuBins / (mu_last - mu_0));
    // mu_rden[s] the reciprocal denominators of the four Lagrange weights on
    // nodes s .. s + 3; mu_rlin[i] = 1 / (mu_{i+1} - mu_i)
    const int *mu_idx;
    const float4 *mu_rden;
    const float *mu_rlin;
    float mu_bin;
};
constexpr int kMuBins = 1024;

// Per-instance plan entry (host-built).
struct InstPlan {
    int n_theta, n_phi, n_phase;
    int n_sub;   // point samples per output phase (the items run n_phase * n_sub of them)
    int pix0;    // first pixel of the instance in the temperature map (HEALPix ring order)
    int ring0;   // first global ring index
    int elem0;   // first element slot (rings of this instance use n_phi slots each)
    int row0;    // first F_t row
    int tile0;   // first entry in the tile-range table
    int tiles;   // ceil(n_phase * n_sub / pt)
};

// One shift-and-add work item: rings [r0, r1) of one spot, phases [j0, j0+nj).
struct Item {
    int b, spot, r0, r1, j0, nj;
};

// Per-ring record written by the ring kernel.
struct RingRec {
    int visible;    // 1 if the ring contributes
    int n_active;   // active elements (compacted at the front of the slots)
    int iT, ig;     // first (logT, logg) node of the ring's interpolation stencil
    int tT, tg;     // stencil taps along logT and logg (2 linear, 4 cubic)
    float kT;       // keV (blackbody emission)
    int map;        // 1: per-element temperatures (map); iT .. iT + tT - 1 are the logT cells used
    float wT[4], wg[4];    // stencil weights
    float dwT[4], dwg[4];  // their derivatives d/dlogT, d/dlogg (0 where clamped)
};

struct Params {
    int B, n_spots, oblate, emission;
    const double *mass_msun, *radius_km, *spin_hz, *incl_rad, *dist_kpc, *nh_1e20;
    const double *colat, *azim, *zeta, *logT;
    const double *mask_colat, *mask_azim, *mask_zeta;
    const double *logT_map;   // per-pixel log10 T (HEALPix ring order) or null
};

struct PlanDev {
    int B, n_fp, n_items, total_rings;
    int grid;  // PPM_GRID_SPOT or PPM_GRID_HEALPIX (InstPlan.n_theta = 4 N_side - 1 rings)
    int pt;  // output phases per work item
    const InstPlan *inst;
    const Item *items;
    const int2 *tile_items;  // [sum tiles] item range of (instance, tile)
    const int *order;        // launch order of the items (largest first); null = identity
    int *queue;              // persistent schedule: next-entry counter (null = one block per item)
    unsigned *err;           // device error word (kErr* bits)
    // work slots per item: 1, or 2 for temperature maps (slot 0: each ring's
    // first logT cell, slot 1: its other cells), each with its own partial
    // tile; used[slot] (null with one slot) says whether the slot's block
    // wrote its partial tile (it writes nothing when it has no work)
    int parts;
    int *used;
};

// Energy-side arrays (device).
struct EnergyDev {
    int nE, nEpad;
    const float *E;      // [nEpad] keV (padded with the last value)
    const float *E3;     // [nEpad] E^3
    const float *pk;     // [nEpad] (ln E - lnE0_table) / dlnE_table
    const float *invE;   // [nEpad] 1/E
    int sliding;         // consecutive pk differ by < 1 (one node shift per step)
    float step;          // > 0: pk is uniform with this step (1/3 .. 1/2), node-major walk
    float inv_step;      // 1 / step
    int moments;         // 1: the forward shift-and-add takes the moment walk
    int nmom;            // moment walk: relative table nodes per group (pk span + 8)
};

// ---- launchers (defined in the .cu files) --------------------------------
cudaError_t launch_lens_build(const LensDev &L, double dalpha, double *psi_scratch,
                              double *list_scratch, int j_cap, cudaStream_t st);

// elemx: per element (weight of the upper logT node or kT, logT cell as int
// bits) for temperature maps; may be null without a map
cudaError_t launch_ring(const Params &p, const PlanDev &plan, const LensDev &L,
                        const AtmDev &A, RingRec *recs, float *tmpl, float *elems,
                        int *status, unsigned *err, unsigned long long *triples, int nE,
                        cudaStream_t st, float2 *elemx = nullptr);

size_t shift_add_smem_bytes(const Params &p, const PlanDev &plan, const AtmDev &A,
                            const EnergyDev &en, int n_phi_max, size_t smem_optin);
// grid_blocks: resident blocks of the persistent schedule (ignored without plan.queue);
// smem_optin: the device's opt-in shared memory per block (0: temperature maps
// take 256-thread blocks)
cudaError_t launch_shift_add(const Params &p, const PlanDev &plan, const AtmDev &A,
                             const EnergyDev &en, const RingRec *recs, const float *tmpl,
                             const float *elems, const int *status, float *partials,
                             int n_phi_max, cudaStream_t st, int grid_blocks = 0,
                             const float2 *elemx = nullptr, size_t smem_optin = 0);

cudaError_t launch_reduce(const PlanDev &plan, const EnergyDev &en, const float *partials,
                          const int *status, int total_rows, float *Ft, cudaStream_t st);

constexpr int kLogFactN = 4096;  // ln d! table size

int loglike_ctiles(int nc);
cudaError_t launch_loglike(const Params &p, const PlanDev &plan, const float *Ft,
                           int total_rows, int nE, const float *R, const float *sigma,
                           int nc, const int *counts, int counts_shared, const float *bkg,
                           double tau, const int *status, const double *lfact, double *row_ll,
                           float *model_counts, double *logL, cudaStream_t st);

void launch_ll_final(const PlanDev &plan, const double *row_ll, int n_ctiles, const int *status,
                     double *logL, cudaStream_t st);

// tensor-core response contraction (resp_tc.cu)
int resp_tc_ctiles(int nc);
int resp_tc_kchunks(int nE);
size_t resp_tc_layout_elems(int nE, int nc);
void resp_tc_layout(const float *R, int nE, int nc, uint16_t *out);
cudaError_t launch_loglike_tc(const Params &p, const PlanDev &plan, const float *Ft,
                              int total_rows, int nE, const uint16_t *Rtc, const float *sigma,
                              int nc, const int *counts, int counts_shared, const float *bkg,
                              double tau, const int *status, const double *lfact,
                              double *row_ll, float *model_counts, unsigned *err, cudaStream_t st);

// ---- gradient (ppm_loglike_grad) ------------------------------------------
constexpr int kNGrad = 13;        // M, R_e, incl, D, N_H, (colat, azim, zeta, logT) x 2 spots
constexpr int kRingAdjTail = 8;   // ring sums after the 4 (n_fp + 1) template adjoints
constexpr int kRingGrad = 8;      // per ring: M, R_e, incl, colat, azim, zeta, logT, 0
constexpr int kGradTN = 64;       // energies per block of the response-adjoint kernel

size_t shift_add_bwd_smem_bytes(int emission, const PlanDev &plan, const AtmDev &A,
                                const EnergyDev &en, int n_phi_max);
cudaError_t launch_shift_add_bwd(const Params &p, const PlanDev &plan, const AtmDev &A,
                                 const EnergyDev &en, const RingRec *recs, const float *tmpl,
                                 const float *elems, const int *status, const float *Aadj,
                                 float *ringadj, int n_phi_max, cudaStream_t st,
                                 size_t smem_limit);
cudaError_t launch_template_bwd(const Params &p, const PlanDev &plan, const LensDev &L,
                                const AtmDev &A, const RingRec *recs, const float *tmpl,
                                const int *status, const float *ringadj, double *ring_grad,
                                cudaStream_t st);
int grad_ktiles(int nEpad);
cudaError_t launch_grad_resp(const Params &p, const PlanDev &plan, const float *Ft,
                             int total_rows, const EnergyDev &en, const float *R,
                             const float *sigma, int nc, const int *counts, int counts_shared,
                             const float *bkg, double tau, const float *lambda,
                             const int *status, float *Aadj, double *row_sums, cudaStream_t st);
cudaError_t launch_grad_final(const Params &p, const PlanDev &plan, const double *ring_grad,
                              const double *row_sums, int ktiles, const int *status,
                              const double *logL, double *grad, cudaStream_t st);

// Power basis of the 4-point cubic on the interval between nodes n and n + 1
// from half-scaled node values u_i = y_i / 2 of nodes n - 1 .. n + 2:
// p(t) = c0 + t (k1 + t (k2 + t k3)), c0 = y_n = 2 u1, k2 = u0 + u2 - 2 u1,
// k3 = (u3 - u0) / 3 + u1 - u2, k1 = u2 - u0 - k3 (the centred cubic
// Lagrange interpolant on a uniform grid; no negated operands).
__device__ __forceinline__ void cubic_half2(float2 u0, float2 u1, float2 u2, float2 u3,
                                            float2 &c0, float2 &k1, float2 &k2, float2 &k3)
{
    const float2 m1 = make_float2(-1.0f, -1.0f), m2 = make_float2(-2.0f, -2.0f);
    const float2 p3 = make_float2(1.0f / 3.0f, 1.0f / 3.0f);
    const float2 m3 = make_float2(-1.0f / 3.0f, -1.0f / 3.0f);
    k2 = __ffma2_rn(u1, m2, __fadd2_rn(u0, u2));
    k3 = __ffma2_rn(u3, p3, __ffma2_rn(u0, m3, __ffma2_rn(u2, m1, u1)));
    k1 = __ffma2_rn(k3, m1, __ffma2_rn(u0, m1, u2));
    c0 = __fadd2_rn(u1, u1);
}

// row -> instance lookup (binary search over InstPlan.row0)
__device__ __forceinline__ int find_instance_by_row(const InstPlan *ip, int B, int row)
{
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (ip[mid].row0 <= row) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int find_instance_by_ring(const InstPlan *ip, int B, int ring)
{
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (ip[mid].ring0 <= ring) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace ppm
