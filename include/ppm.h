/*
 * ppm.h -- C ABI of the GB300 pulse-profile likelihood library (libppm.so).
 *
 * The library evaluates the energy-resolved X-ray pulse-profile forward model
 * of Zhou & Huang, "GPU-accelerated X-ray pulse profile modeling"
 * (arXiv 2510.07764), and its Poisson likelihood, entirely in CUDA kernels
 * for sm_103a:
 *
 *   parameters --(light bending, Doppler, atmosphere, shift-and-add)--> F_t
 *   F_t --(ISM attenuation, response contraction)--> expected counts
 *   expected counts, data --> Poisson log-likelihood
 *
 * Conventions
 * -----------
 * - Every entry point returns a ppm_status; nothing throws across the ABI.
 *   On error ppm_last_error() returns a message for the last failed call on
 *   that context (one message per context; see the thread-safety rule below).
 * - "device" pointers are CUDA global-memory pointers on the context's device;
 *   "host" pointers are ordinary process memory.  The caller owns every
 *   pointer it passes; the library never frees caller memory and keeps no
 *   pointer to it after the call returns (table setters copy their inputs).
 * - `stream` is a cudaStream_t (NULL = the legacy default stream).  Compute
 *   calls enqueue work on that stream and return without waiting; outputs are
 *   valid once the stream has completed (see ppm_sync).
 * - Argument errors are detected on the host before any work is enqueued and
 *   return PPM_EINVAL.  Per-instance physics range errors (compactness outside
 *   the lens table, temperature or gravity outside the atmosphere table, a
 *   NaN or infinite parameter value the instance uses) are reported through
 *   `inst_status` and do not fail the call.
 * - Angles are radians, masses solar masses, radii km, distances kpc,
 *   energies keV, hydrogen columns 1e20 cm^-2, temperatures log10(T / K).
 * - A context is not thread-safe: calls on one context must be serialised
 *   (they may use different streams; the context's workspace is reused, so
 *   two compute calls on one context must not overlap on the GPU).
 * - CUDA graphs: once a context has run a problem of the same resolution
 *   (its plan, workspace and kernel attributes are then settled),
 *   ppm_profile, ppm_loglike and ppm_loglike_grad enqueue only kernels and
 *   asynchronous copies and can be captured; a replay reads the parameters,
 *   counts and background again from the same device arrays.  A later call
 *   that grows the workspace invalidates earlier captures.
 */
#ifndef PPM_H
#define PPM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PPM_OK = 0,
    PPM_EINVAL = 1,    /* bad argument, missing table, unsupported size */
    PPM_ERANGE = 2,    /* per-instance: parameters outside the tables or not finite */
    PPM_ENOMEM = 3,    /* device or pinned-host allocation failed */
    PPM_ECUDA = 4,     /* a CUDA runtime call failed */
    PPM_ETIMEOUT = 5,  /* ppm_sync gave up waiting */
    PPM_ENOTREADY = 6  /* a device-side invariant failed (see ppm_sync) */
} ppm_status;

typedef struct ppm_ctx ppm_ctx;

/* Create a context on CUDA device `device`.  The context owns the lens,
 * atmosphere, energy and response tables and a workspace that grows on first
 * use of a larger problem (no allocation on later calls of the same size). */
ppm_status ppm_create(ppm_ctx **out, int device);

/* Destroy a context and free everything it owns.  NULL is ignored. */
void ppm_destroy(ppm_ctx *ctx);

/* Message describing the last failed call on this context ("" if none). */
const char *ppm_last_error(const ppm_ctx *ctx);

/* ------------------------------------------------------------------------
 * Light-bending tables (Sect. 2.3 and 2.8.2 of the paper; grids: Eq.
 * grids_def; bending: Eqs. salmi_lf and rho; delays: Eqs. salmi_td and
 * tot_time_delay).
 *
 * Builds, in FP64 on the GPU, three tables on linear grids:
 *   C_alpha[u][cos psi]  cos(alpha) of the ray that reaches the observer,
 *   LF[u][cos psi]       lensing factor d cos(alpha) / d cos(psi),
 *   TD[u][cos alpha]     c Delta t / R (the run-time delay is
 *                        (R/c) TD + delta t(R), Eq. delta_t_oblate).
 * The alpha march uses steps of `dalpha` (the paper: pi/2048) and stops when
 * psi exceeds arccos(cpsi_min), when the ray is captured, or when psi would
 * pass pi; grid cells beyond the march are marked invalid (treated as
 * invisible).  Requires n_u, n_cpsi, n_calpha >= 2, 0 <= u_min < u_max < 2/3,
 * -1 <= cpsi_min < cpsi_max <= 1, -1 <= calpha_min < calpha_max <= 1,
 * pi/16384 <= dalpha <= 0.05, cpsi_max = 1.  The call waits for `stream`,
 * builds the tables on it and blocks until they are complete.
 * ------------------------------------------------------------------------ */
typedef struct {
    double u_min, u_max;
    int n_u;
    double cpsi_min, cpsi_max;
    int n_cpsi;
    double calpha_min, calpha_max;
    int n_calpha;
    double dalpha;
} ppm_lens_spec;

ppm_status ppm_build_lens(ppm_ctx *ctx, const ppm_lens_spec *spec, void *stream);

/* Copy the lens tables to host arrays (row-major [n_u][n_cpsi] for Ca and LF,
 * [n_u][n_calpha] for TD; invalid cells are NaN).  Any pointer may be NULL.
 * Blocks until the tables are built. */
ppm_status ppm_get_lens(ppm_ctx *ctx, double *Ca, double *LF, double *TD);

/* ------------------------------------------------------------------------
 * Atmosphere interpolation strategy (Sect. 4, the four schemes compared on
 * the paper's two interpolation tests).  Applies to every later call of the
 * context; the default is PPM_INTERP_MIXED.
 *   PPM_INTERP_MIXED        the method's scheme: linear in logT and logg,
 *                           cubic Lagrange in mu and ln E, linear where the
 *                           centred four-node stencil would leave the grid
 *                           and on the protected small-mu intervals;
 *   PPM_INTERP_CUBIC        cubic Lagrange in all four axes, the stencil moved
 *                           inside the grid at the edges (one-sided);
 *   PPM_INTERP_CUBIC_CLIP   as PPM_INTERP_CUBIC, negative interpolants set to 0;
 *   PPM_INTERP_CUBIC_LINEAR_EDGES  cubic in all four axes with the linear
 *                           edge and protected-zone rules of the method.
 * Returns PPM_EINVAL for any other value.
 * ------------------------------------------------------------------------ */
enum {
    PPM_INTERP_MIXED = 0,
    PPM_INTERP_CUBIC = 1,
    PPM_INTERP_CUBIC_CLIP = 2,
    PPM_INTERP_CUBIC_LINEAR_EDGES = 3
};
ppm_status ppm_set_interpolation(ppm_ctx *ctx, int strategy);

/* ------------------------------------------------------------------------
 * Atmosphere table (Sect. 2.5 and 4): specific intensity I(E', mu; T, g) in
 * keV cm^-2 s^-1 keV^-1 sr^-1, host array I[nT][ng][nmu][nE] (float32,
 * linear intensity), with node positions logT[nT], logg[ng] (uniform grids),
 * mu[nmu] (increasing, any spacing) and lnE[nE] (natural log of keV, uniform
 * spacing).  Interpolation is mixed order: linear in logT and logg, cubic
 * Lagrange in mu and ln E, linear on the intervals among the first
 * `n_protect` (>= 2) small-mu nodes and wherever the four-node stencil would
 * leave the grid; queries outside the mu and E ranges clamp to the edge node.
 * Limits: nmu <= 128, nE <= 512, nmu >= 4, nE >= 4, nT, ng >= 2.
 * The table is copied; the call is synchronous.
 * ------------------------------------------------------------------------ */
ppm_status ppm_set_atmosphere(ppm_ctx *ctx, const float *I,
                              const double *logT, int nT, const double *logg, int ng,
                              const double *mu, int nmu, const double *lnE, int nE,
                              int n_protect);

/* Model (observed) energy grid E_keV[nE] (host, strictly increasing,
 * 1 <= nE <= 1024).  Copied; synchronous.  Resets any response matrix whose
 * energy count differs. */
ppm_status ppm_set_energies(ppm_ctx *ctx, const double *E_keV, int nE);

/* Response on the model energy grid (Sect. 2.7, 2.8.4): R[nE][nc] host
 * row-major float32 (effective area x redistribution x energy width, so
 * that counts/s = F_t diag(ATT) R), and the ISM cross-section sigma_ism[nE]
 * in cm^2 (ATT_k = exp(-N_H sigma_k)).  nE must equal the energy grid size;
 * 1 <= nc <= 4096.  Copied; synchronous. */
ppm_status ppm_set_response(ppm_ctx *ctx, const float *R, int nE, int nc,
                            const float *sigma_ism);

/* Response from a fine detector grid (Sect. 2.7, the down-sampling matrix
 * DS and Eq. RSP): Ne detector energy bins [E_lo[e], E_hi[e]] (host, keV,
 * E_lo < E_hi), the fine response Rf[Ne][nc] (host row-major float32:
 * effective area x redistribution, per bin) and sigma_ism[nE] on the model
 * grid.  The library builds, in FP64 on the host,
 *   DS[i][e] = integral over [E_lo[e], E_hi[e]] of the piecewise-linear
 *              interpolant on the model grid that is 1 at E_i and 0 at the
 *              other nodes (constant beyond the grid ends),
 *   R[i][c]  = sum_e DS[i][e] Rf[e][c],
 * and installs R as ppm_set_response does (the attenuation ATT_i stays a
 * per-instance factor applied at run time).  1 <= Ne <= 1<<20; nE is the
 * model grid size set by ppm_set_energies.  Copied; synchronous. */
ppm_status ppm_set_response_fine(ppm_ctx *ctx, const double *E_lo, const double *E_hi, int Ne,
                                 const float *Rf, int nc, const float *sigma);

/* ------------------------------------------------------------------------
 * Parameter vectors: structure of arrays of DEVICE pointers, B instances.
 * Per instance (length B): mass_msun, radius_km (equatorial), spin_hz,
 * incl_rad, dist_kpc, nh_1e20.  Per instance and spot (length B * n_spots,
 * index b * n_spots + s): colat, azim, zeta (angular radius), logT, and a
 * masking cap mask_colat, mask_azim, mask_zeta (mask_zeta <= 0: no mask).
 * An element of a spot is active when its centre is not inside the mask cap
 * (a concentric mask makes a ring, an offset one a crescent).
 * oblate: 0 = Schwarzschild+Doppler sphere, 1 = oblate Schwarzschild.
 * emission: 0 = isotropic blackbody (analytic), 1 = atmosphere table.
 * ------------------------------------------------------------------------ */
typedef struct {
    int B;
    int n_spots;   /* 1 or 2 */
    int oblate;
    int emission;
    const double *mass_msun, *radius_km, *spin_hz, *incl_rad, *dist_kpc, *nh_1e20;
    const double *colat, *azim, *zeta, *logT;
    const double *mask_colat, *mask_azim, *mask_zeta;
    /* Full-surface temperature map (Sect. 2.6), or NULL: DEVICE log10 T_eff per
     * HEALPix pixel in ring order, 12 N_side(b)^2 values per instance,
     * instances concatenated.  Needs grid = PPM_GRID_HEALPIX, n_spots = 1 and
     * the default interpolation strategy; a pixel with a non-finite or
     * non-positive value emits nothing, the spot parameters (colat, azim,
     * zeta, logT, masks) are not used.  Not differentiated (ppm_loglike_grad
     * and ppm_profile_noalloc reject it). */
    const double *logT_map;
} ppm_params;

/* Per-instance resolution: HOST arrays of length B, and the surface grid.
 * grid = PPM_GRID_SPOT: each spot is covered by n_theta rings uniform in
 * colatitude over its angular extent, each ring by n_phi elements uniform
 * over the spot's azimuthal width (1 <= n_theta <= 4096, 1 <= n_phi <= 4096).
 * grid = PPM_GRID_HEALPIX (Sect. 2.6): the whole surface is the HEALPix mesh
 * with N_side = n_theta[b] (1 <= N_side <= 1024; 4 N_side - 1 rings of up
 * to 4 N_side equal-area pixels, n_phi ignored); a spot is the set of pixels
 * whose centres lie within zeta of its centre and outside its mask.  The
 * mesh does not move with the spot, so spot geometry enters only through
 * which pixels are selected (ppm_loglike_grad rejects this grid).
 * n_phase output phases j / n_phase (1 <= n_phase <= 4096).  n_fp fine
 * template phases per ring (8 <= n_fp <= 1024; the paper uses 192). */
enum { PPM_GRID_SPOT = 0, PPM_GRID_HEALPIX = 1 };
typedef struct {
    const int *n_theta, *n_phi, *n_phase;
    int n_fp;
    int grid;   /* PPM_GRID_SPOT or PPM_GRID_HEALPIX */
    int phase_sub;  /* 1, 2, 4, 8 or 16 point samples per output phase bin: bin j is
                       the mean of samples at (j + (q + 1/2)/S - 1/2) / n_phase; 1 = the
                       point sample j / n_phase (Sect. 2.8.3) */
} ppm_res;

/* ------------------------------------------------------------------------
 * Forward profile (Sect. 2.8.3, Eq. add_Ft; flux formula of Sect. 2.5 / App.
 * C).  Writes the photon number flux F_t (photons cm^-2 s^-1 keV^-1) to the
 * DEVICE array Ft, float32, rows of instance b at row offset
 * sum_{b' < b} n_phase[b'], each row nE energies.  inst_status (DEVICE int
 * [B], may be NULL) receives PPM_OK or PPM_ERANGE per instance; rows of an
 * out-of-range instance are zero.  Requires ppm_build_lens, ppm_set_energies
 * and, for emission = 1, ppm_set_atmosphere.
 * ------------------------------------------------------------------------ */
ppm_status ppm_profile(ppm_ctx *ctx, const ppm_params *p, const ppm_res *res,
                       float *Ft, int *inst_status, void *stream);

/* ------------------------------------------------------------------------
 * Allocation-free forward profile.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate GPU memory at evaluation
 * time -- for example a sampler that has already handed the rest of the
 * device memory to its own pool, or one that cannot afford the
 * device-wide synchronisation that cudaMalloc/cudaFree imply while other
 * work is in flight.  It computes what ppm_profile computes, with the same
 * kernels and buffer layouts and a plan built by ppm_profile's phase-tile and
 * ring-group rules under the context's tile settings (no persistent queue;
 * items in plan order), so that its output equals ppm_profile's bit for bit
 * unless its ring groups had to be widened (below).  It takes every per-call
 * buffer from a fixed 64 MiB array in the library's device memory, which
 * every GPU that loads the library holds until the process exits, and builds
 * its plan in a fixed 1 MiB host buffer: it calls no cudaMalloc, cudaFree or
 * other allocating routine.  The context's tables must already be set by the
 * usual setters.  Temperature maps are not supported (PPM_EINVAL).
 *
 * - Problems whose per-call buffers exceed 64 MiB with ppm_profile's ring
 *   groups are retried with groups 2, 4, ... times wider (the sums are then
 *   grouped differently, equal to rounding); problems that exceed it even
 *   with one group per spot, or whose plan exceeds 1 MiB of host staging,
 *   return PPM_EINVAL with a message; nothing is enqueued.  (The default
 *   two-spot 128x128 workload with 128 phases and 256 energies fits.)
 * - The plan is copied from the fixed host buffer with a pageable
 *   cudaMemcpyAsync, which returns only once the buffer has been consumed:
 *   the call can therefore wait on the host for the work already queued on
 *   `stream`.  A stream that is being captured is refused with PPM_EINVAL
 *   before anything is enqueued.
 * - The first call on a device looks up the array's device address on that
 *   device; make that first call before any stream capture.
 * - All calls in the process share the one array per device, which keeps the
 *   previous call's contents (the status words are cleared at every call).
 *   Calls that overlap on the GPU -- two streams, two contexts on one device,
 *   or two host threads -- race on it; serialise them.
 * ------------------------------------------------------------------------ */
ppm_status ppm_profile_noalloc(ppm_ctx *ctx, const ppm_params *p, const ppm_res *res,
                               float *Ft, int *inst_status, void *stream);

/* ------------------------------------------------------------------------
 * Poisson log-likelihood (Sect. 2.7, 2.8.4; the paper states the likelihood
 * only through -2 Delta ln L ~ chi^2, Eq. chi2_def context, and its GPU-side
 * accumulation in Sect. 6): the profile of ppm_profile, attenuated,
 * contracted with the response, lambda = tau * C + bkg, and
 *   logL[b] = sum_{j,c} d ln(lambda) - lambda - ln Gamma(d + 1)
 * accumulated in FP64 (lambda = 0 contributes 0 if d = 0, -inf otherwise).
 * counts: DEVICE int32 [rows][nc] with the row layout of Ft, or, if
 * counts_shared != 0, one [n_phase][nc] block used by every instance (all
 * instances must then have the same n_phase).  bkg: DEVICE float32 with the
 * layout of counts, or NULL.  logL: DEVICE double [B].  model_counts: DEVICE
 * float32 [rows][nc] receiving lambda, or NULL.  Out-of-range instances get
 * logL = -inf and PPM_ERANGE in inst_status.
 * ------------------------------------------------------------------------ */
ppm_status ppm_loglike(ppm_ctx *ctx, const ppm_params *p, const ppm_res *res,
                       const int *counts, int counts_shared, const float *bkg,
                       double tau, double *logL, float *model_counts,
                       int *inst_status, void *stream);

/* ------------------------------------------------------------------------
 * Log-likelihood and its gradient (reverse mode of Sect. 2.8.3 Eq. add_Ft,
 * the Sect. 4 interpolation, Sect. 2.7 attenuation and the response; the
 * paper motivates gradients only through the inference of Sect. 6 and gives
 * no adjoint, so this entry point has no direct counterpart in it).
 * Arguments as ppm_loglike, plus
 *   grad: DEVICE double [B][13], d logL[b] / d theta in the order
 *         M (M_sun), R_e (km), inclination (rad), D (kpc), N_H (1e20 cm^-2),
 *         then colatitude (rad), azimuth (rad), angular radius zeta (rad),
 *         log10 T for spot 1 and for spot 2 (zeros for a missing spot 2).
 * The gradient is that of the piecewise-smooth model the forward pass
 * evaluates: branch decisions (visibility of template points, active
 * elements, interpolation intervals, clamps) are held fixed; quantities
 * clamped at a table edge contribute no derivative.  Spin and the mask
 * parameters are not differentiated.  Instances with inst_status != 0 or
 * logL = -inf get NaN gradients.  Needs emission 1 (atmosphere table) or 0
 * (analytic blackbody), and shared memory for three nE x nmu slabs
 * (PPM_EINVAL otherwise).  Runs the forward pass first (logL is written as
 * by ppm_loglike), then the backward kernels, on `stream`.
 * ------------------------------------------------------------------------ */
ppm_status ppm_loglike_grad(ppm_ctx *ctx, const ppm_params *p, const ppm_res *res,
                            const int *counts, int counts_shared, const float *bkg,
                            double tau, double *logL, double *grad,
                            int *inst_status, void *stream);

/* ------------------------------------------------------------------------
 * Work decomposition of the shift-and-add and its autotuner (no counterpart
 * in the paper, whose GPU design assigns one ring per SM, Sect. 2.9).
 * A work item is (instance, spot, ring group, tile of phase_tile output
 * phases); ring groups are sized so that the whole call makes about
 * `waves` waves of two blocks per SM; items run largest first, either one
 * block per item (persistent = 0) or as a queue drained by two resident
 * blocks per SM (persistent = 1).  phase_tile = 0 picks 16 or 32 from the
 * problem size.  walk selects how a warp steps through the energies with
 * the atmosphere table:
 *   - 1: the energy walk (one observed energy per iteration, interval
 *     changes per element), everywhere;
 *   - 2: the node-major walk wherever the observed energy grid is uniform in
 *     ln E with a step of 0.34 to 0.498 table nodes (every table interval
 *     then holds two or three observed energies; one interval per iteration
 *     for all elements of a warp), the energy walk elsewhere;
 *   - 0 (default): as 2, except that the forward shift-and-add of spots takes
 *     the moment walk wherever the observed energies step by less than one
 *     table node and the interpolation strategy is not B: per group of 64
 *     elements whose ln z spread is below 0.45 table node and whose mu
 *     stencils span at most 32 columns, the moments sum_p eps_p^j u_p of the
 *     node values (eps_p the element's offset from the group's reference
 *     position, j = 0..3) are contracted once per table node from column
 *     weights, and each energy evaluates one combined cubic, plus exact
 *     difference terms for elements on the other side of a node; other
 *     groups take the node-major walk (uniform grids) or the energy walk.
 * All walks evaluate the same interpolants; they differ in the order of the
 * FP32 sums (and, for the node-major walk, in positions accumulated along
 * the grid).  With the node-major or moment walk, phase_tile = 0 picks 16
 * (their shared-memory buffers leave room for two blocks per SM only with
 * 16-phase tiles).  The backward pass of ppm_loglike_grad takes the
 * node-major walk under 0 and 2.  The setting applies to later calls of the
 * context.
 *
 * ppm_autotune runs the forward profile of (p, res) once per candidate
 * (phase_tile 16/32 x waves 8/16/32/64 x persistent 0/1, one untimed and one
 * timed pass each, synchronising `stream`), keeps the fastest, and returns
 * it in *best (ms = its time; walk is left as set).  Results do not depend
 * on the choice (the partial sums are added in a fixed order).
 * ------------------------------------------------------------------------ */
typedef struct {
    int phase_tile;   /* 0 (automatic), 16 or 32 */
    int waves;        /* 1 .. 256, default 16 */
    int persistent;   /* 0 or 1 */
    int walk;         /* 0 (moment, else node-major, where they apply), 1 (energy walk)
                         or 2 (node-major where it applies) */
    double ms;        /* ppm_autotune: time of the chosen candidate */
} ppm_tiles;

ppm_status ppm_set_tiles(ppm_ctx *ctx, const ppm_tiles *t);
ppm_status ppm_get_tiles(ppm_ctx *ctx, ppm_tiles *t);
ppm_status ppm_autotune(ppm_ctx *ctx, const ppm_params *p, const ppm_res *res, void *stream,
                        ppm_tiles *best);

/* ------------------------------------------------------------------------
 * Stage timing (no counterpart in the paper; tracing support).  When enabled,
 * every compute call records CUDA events around its stages on the call's
 * stream and counts its kernel launches and the (active element, output
 * phase, energy) triples its shift-and-add evaluates.  ppm_get_timing waits
 * for the recorded events and returns the totals accumulated since
 * ppm_set_timing; ppm_set_timing(ctx, enable) resets the totals.
 * ------------------------------------------------------------------------ */
typedef struct {
    double ms_ring;        /* per-ring setup + template kernel */
    double ms_shift_add;   /* shift-and-add + atmosphere interpolation kernel */
    double ms_reduce;      /* partial-sum reduction kernel */
    double ms_loglike;     /* response contraction + likelihood kernels */
    double ms_grad_resp;   /* gradient: response / likelihood adjoint kernel */
    double ms_shift_add_bwd; /* gradient: backward shift-and-add kernel */
    double ms_template_bwd;  /* gradient: template tangents + final reduction */
    long long calls;       /* compute calls timed */
    long long launches;    /* kernels launched by those calls */
    double triples;        /* element x phase x energy triples evaluated */
} ppm_timing;

ppm_status ppm_set_timing(ppm_ctx *ctx, int enable);
ppm_status ppm_get_timing(ppm_ctx *ctx, ppm_timing *out);

/* FP32 FMA throughput of device `device` in TFLOP/s (no counterpart in the
 * paper; measurement support for the FP32 roofline of the shift-and-add):
 * 8 independent FMA chains per thread, scalar FFMA (paired = 0) or packed
 * FFMA2 (paired = 1), 8 blocks of 256 threads per SM, timed with CUDA events
 * on `stream` (synchronised).  Allocates and frees 16 KB of device memory. */
ppm_status ppm_fp32_peak(int device, int paired, void *stream, double *tflops);

/* Wait for `stream` with a bounded host-side poll (timeout_s > 0), then report
 * any device-side invariant failure recorded since the last ppm_sync
 * (PPM_ENOTREADY, with a message) and clear it.  Returns PPM_ETIMEOUT if the
 * stream has not completed within timeout_s seconds. */
ppm_status ppm_sync(ppm_ctx *ctx, void *stream, double timeout_s);

#ifdef __cplusplus
}
#endif
#endif /* PPM_H */
