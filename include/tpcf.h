/*
 * tpcf.h -- C ABI of the GB300 (sm_103a) binned harmonic 3PCF estimator.
 *
 * The estimator is that of arXiv:2408.16847, section 3.1: for every pivot i
 * (HEALPix pixel or catalogue point) with weight w_i != 0 and every other point j
 * whose angular separation theta_ij falls in radial bin k = [theta_k, theta_{k+1}),
 *
 *     a_m^k(i) = sum_j w_j d_j exp(-i m phi_ij)          (eq. Xm.binned, unnormalised;
 *                                                         phi_ij = position angle of j
 *                                                         about i, from local north
 *                                                         through east)
 *     S_m(k1,k2) = sum_i w_i d_i a_m^{k1}(i) conj(a_m^{k2}(i))      (eqs. zetamEst,
 *                                                                     zetamEst2)
 *     D(k1,k2)   = sum_i w_i W^{k1}(i) W^{k2}(i),  W^k(i) = sum_j w_j Theta_k(ij)
 *     zeta_m     = S_m / D                 (normalisation by the same estimator run
 *                                           with d = 1 and m = 0; zeta = 0 where D = 0)
 *
 * for m = 0..m_max.  Bins are decided by chord length against 2 sin(theta_e / 2);
 * the j = k self term of the outer product is kept, as in the paper (section 3.4),
 * unless TPCF_SELF_PAIRS_SUBTRACT is set.
 *
 * Conventions common to every call:
 *  - Device buffers ("d_" prefix) are allocated and owned by the caller; the plan
 *    owns its internal tables and scratch.  Host buffers carry an "h_" prefix.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *    Calls enqueue work on it and return; they do not synchronise unless stated.
 *  - Calls never abort: they return a tpcf_status.  Errors found on the device are
 *    latched in the plan's device status word and reported by tpcf_plan_sync()
 *    (and by tpcf_run_host, which synchronises).
 *  - d_delta and d_w are float32, one value per point (RING pixel order for maps,
 *    catalogue order for catalogues).  w = 0 marks a masked point: it is neither a
 *    pivot nor a neighbour.
 *  - zeta / dL_dzeta layout: double[(m_max+1)][K][K][2] (re, im), row-major.
 *    norm layout: double[K][K].
 *  - A plan is not thread-safe; calls on one plan must be serialised by the caller
 *    (the same stream, or external synchronisation).
 */
#ifndef TPCF_H
#define TPCF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tpcf_plan_s* tpcf_plan;
typedef struct tpcf_batch_s* tpcf_batch;

typedef enum {
    TPCF_OK = 0,
    TPCF_ERR_INVALID_ARG = 1, /* a pointer, size, range or flag is not acceptable   */
    TPCF_ERR_CUDA = 2,        /* a CUDA runtime call failed (message: tpcf_last_error) */
    TPCF_ERR_OOM = 3,         /* device allocation failed; nothing leaked           */
    TPCF_ERR_TIMEOUT = 4,     /* a bounded device wait gave up                      */
    TPCF_ERR_UNSUPPORTED = 5, /* valid request the library does not implement      */
    TPCF_ERR_DEVICE = 6       /* a kernel latched an error (bad table / index)      */
} tpcf_status;

/* Plan flags. */
#define TPCF_SELF_PAIRS_KEEP 0u      /* keep the j = k term (the paper's estimator) */
#define TPCF_SELF_PAIRS_SUBTRACT 1u  /* remove it from S_m(k,k) and from D(k,k)     */
#define TPCF_CONTRACT_FP32 0u        /* sum over pivots on the FP32 pipe            */
#define TPCF_CONTRACT_TC 2u          /* sum over pivots on the tensor cores (split
                                        TF32x3 operands, FP32 accumulate): map plans,
                                        tpcf_forward only; catalogue plans, batches and
                                        tpcf_forward_noalloc return UNSUPPORTED     */
/* Normalisation.  The default divides by the weight triple sum of the same pivots:
 * zeta_m = S_m / D with D(k1,k2) = sum_i w_i W^{k1}(i) W^{k2}(i).  The two flags below
 * instead normalise each pivot's moments before the sum over pivots (Sec. 3.1): the
 * prefactor of eq. Xm.binned divides a_m^k(i) by the weight of all the pivot's
 * neighbours, sum_k W^k(i) (PIVOT_TOTAL); the binning figure's caption averages over
 * the points of each bin, a_m^k(i) / W^k(i) (BIN_MEAN).  With X^k(i) the normalised
 * moments (0 where the divisor is 0),
 *   zeta_m(k1,k2) = sum_i w_i d_i X_m^{k1}(i) conj(X_m^{k2}(i)) / sum_i w_i,
 * and d_norm holds sum_i w_i in every entry.  For tpcf_forward (map and catalogue
 * plans) and tpcf_forward_noalloc; with TPCF_SELF_PAIRS_SUBTRACT or TPCF_CONTRACT_TC
 * the plan is not created (UNSUPPORTED); tpcf_backward, batches and
 * tpcf_forward_multi return UNSUPPORTED, and tpcf_plan_autotune tunes the forward
 * only.  At most one of the two flags (else INVALID_ARG). */
#define TPCF_NORM_BIN_MEAN 4u
#define TPCF_NORM_PIVOT_TOTAL 8u

#define TPCF_MAX_BINS 32
#define TPCF_MAX_M 16

/* Angular bins: nbins edges theta_edges_rad[0..nbins] (radians, strictly increasing,
 * theta_edges_rad[0] > 0, theta_edges_rad[nbins] < pi/2), multipoles 0..m_max
 * (0 <= m_max <= TPCF_MAX_M), flags as above.  Copied by the plan. */
typedef struct {
    int32_t nbins;
    const double* theta_edges_rad; /* host pointer */
    int32_t m_max;
    uint32_t flags;
} tpcf_bins;

/* Human-readable name of a status; the pointer is static. */
const char* tpcf_status_string(tpcf_status s);
/* Text of the last CUDA error seen by this thread (static storage). */
const char* tpcf_last_error(void);

/*
 * Map plan for a full-sky HEALPix RING map of resolution nside (1 <= nside <= 8192),
 * 12 nside^2 pixels (Gorski et al. 2005, the pixelisation of the paper's maps,
 * section 3.3).  Builds, on the device and on `stream`, the ring geometry in FP64
 * and the per-ring-pair bin thresholds used by the exact ring-range neighbour
 * search.  On failure *out is left NULL and nothing is leaked.
 */
tpcf_status tpcf_plan_create_map(tpcf_plan* out, int64_t nside, const tpcf_bins* bins, void* stream);

/*
 * Catalogue plan over n points given as unit vectors d_xyz (device, double[n][3],
 * used as given), for point catalogues: the estimator of section 3.1 applies to any
 * sample on the sphere.  Sorts the points, on the device and on `stream`, into a
 * sphere grid of colatitude bands cut into longitude sectors (about 32 points per
 * cell on average); each pivot's neighbours are then read from the cells that the
 * cap of radius theta_max around its tile of 32 pivots overlaps, and binned exactly
 * (fp32 chord from hi/lo coordinates, FP64 decision within 2e-6 of an edge).  The
 * plan keeps its own sorted copy: d_xyz may be freed once the call has returned.
 * Forward calls take d_delta / d_w in the caller's point order, and pivot ranges are
 * ranges of caller indices.  1 <= n <= 2^31 - 1, else TPCF_ERR_INVALID_ARG.
 */
tpcf_status tpcf_plan_create_catalog(tpcf_plan* out, const double* d_xyz, int64_t n,
                                     const tpcf_bins* bins, void* stream);

/*
 * zeta = d_sums / (scale * d_norm), per entry, 0 where the denominator is 0: the last
 * step of an estimate whose sums and normalisation come from different runs.  The
 * edge-corrected catalogue estimate (data with delta = 1, randoms with
 * delta = -alpha, alpha = sum w_data / n_randoms) takes the raw sums S of the union
 * and the norm D of a delta = 1 run over the randoms, with scale = alpha^3.
 * d_sums and d_zeta use the zeta layout, d_norm the norm layout (device, caller
 * owned).  Errors: INVALID_ARG for NULL, nbins / m_max out of range, scale not > 0.
 */
tpcf_status tpcf_normalize(const double* d_sums, const double* d_norm, double scale, int32_t nbins,
                           int32_t m_max, double* d_zeta, void* stream);

/*
 * m-coupling (edge) correction of a data-minus-randoms estimate: masks and survey
 * geometry couple the multipoles (the paper leaves this for later work; Sec. 3.1 gives
 * the harmonic decomposition it acts on).  For a bin pair the estimate is the ratio
 * zeta(phi) = N(phi) / R(phi) of the triplet-angle densities of the D - R field and of
 * the randoms; in harmonic space, with X_{-n} = conj(X_n) and
 * zeta(phi) = sum_m z_m e^{i m phi},
 *     S_m = sum_{m'=-M..M} z_{m'} scale R_{m-m'},    m = -M..M,
 * which is solved per (k1, k2) by Gaussian elimination with partial pivoting (FP64)
 * for z_m, m = 0..m_max.  d_sums: the raw sums S of the D - R run, (m_max+1) x K x K
 * x {re, im} doubles (the zeta layout); d_rsums: the raw sums of the randoms' delta = 1
 * run at multipoles 0..2 m_max, (2 m_max+1) x K x K x {re, im}; scale: alpha^3 as in
 * tpcf_normalize; d_zeta: (m_max+1) x K x K x {re, im} (device, caller owned).  With
 * no coupling (R_n = 0 for n != 0) the result is tpcf_normalize's.  R_0(k1, k2) = 0
 * gives 0; a singular system gives NaN entries.  Errors: INVALID_ARG for NULL,
 * nbins or m_max out of range (m_max <= TPCF_MAX_M), scale not > 0.
 */
tpcf_status tpcf_edge_correct(const double* d_sums, const double* d_rsums, double scale, int32_t nbins,
                              int32_t m_max, double* d_zeta, void* stream);

/* Number of points (pixels) of the plan; -1 if plan is NULL. */
int64_t tpcf_plan_npoints(tpcf_plan plan);

/* Number of CUDA kernels the plan's calls have enqueued so far (plan creation
 * excluded); -1 if plan is NULL.  Lets a caller count launches in a timed region. */
int64_t tpcf_plan_kernel_launches(tpcf_plan plan);

/*
 * Forward estimator over the pivots with index in [pivot_begin, pivot_end)
 * (pivot_begin = 0, pivot_end = npoints for all).  Neighbours are always taken
 * from every point.  Writes d_zeta, d_norm (D) and, if d_sums != NULL, the raw
 * sums S (same layout as zeta).  An empty pivot range writes zeros.
 */
tpcf_status tpcf_forward(tpcf_plan plan, const float* d_delta, const float* d_w,
                         int64_t pivot_begin, int64_t pivot_end, double* d_zeta, double* d_norm,
                         double* d_sums, void* stream);

/*
 * Forward with shared neighbour lists, the fast approximate mode of Sec. 3.2 (pivots
 * very close to one another share one neighbour list).  Each ring's pixels are cut into
 * runs of `group` consecutive pixels (the last run of a ring shorter), and every pivot
 * of a run takes the moments of the run's middle pixel rho, neighbours and angles both:
 *   S_m(k1,k2) = sum_i w_i d_i a_m^{k1}(rho(i)) conj(a_m^{k2}(rho(i))),
 *   D(k1,k2)   = sum_i w_i W^{k1}(rho(i)) W^{k2}(rho(i)),   zeta = S / D,
 * over the pivots in [pivot_begin, pivot_end); the moments of rho (eq. Xm.binned) take
 * every other pixel in the bins, the run's own members included.  The pair work drops
 * by about `group`; the pivots move by at most (group - 1) / 2 ring pixels.  group = 1
 * is tpcf_forward.  Map plans without TPCF_CONTRACT_TC, TPCF_SELF_PAIRS_SUBTRACT or a
 * per-pivot normalisation (else UNSUPPORTED); 1 <= group <= 4096 (else INVALID_ARG).
 * A call with a new group size builds that tile list (host to device copy, a few MB at
 * most) and synchronises `stream`; the plan keeps the list of the last group size.
 * Outputs as tpcf_forward.
 */
tpcf_status tpcf_forward_grouped(tpcf_plan plan, const float* d_delta, const float* d_w, int32_t group,
                                 int64_t pivot_begin, int64_t pivot_end, double* d_zeta, double* d_norm,
                                 double* d_sums, void* stream);

/*
 * Multi-field forward (end of Sec. 2, after eq. ubEstimator): three fields A, B, C on
 * the points of one plan (e.g. tomographic bins), each with its own weights.  With
 * the moments a^k(i; F), W^k(i; F) of eq. Xm.binned taken over field F, and summed over
 * the cyclic permutations (P, X, Y) of (A, B, C):
 *   S_m(k1,k2) = sum_(P,X,Y) sum_i w^P_i P_i a_m^{k1}(i; X) conj(a_m^{k2}(i; Y)),
 *   D(k1,k2)   = sum_(P,X,Y) sum_i w^P_i W^{k1}(i; X) W^{k2}(i; Y),
 *   zeta_m = S_m / D (the same normalisation as tpcf_forward; zeta = 0 where D = 0),
 * over the pivots in [pivot_begin, pivot_end).  With A = B = C this is the single-field
 * estimate.  The sums are full K x K matrices (not Hermitian when the fields differ):
 * d_zeta and d_sums (optional) (m_max+1) x K x K x {re, im} doubles, d_norm K x K.
 * Map and catalogue plans (the fields indexed like the plan's pixels or points) with
 * the FP32 contraction, self pairs kept and the default normalisation (else
 * TPCF_ERR_UNSUPPORTED, also when the three fields' tile moments do not fit in shared
 * memory).  The first call allocates the plan's buffers for fields B and C (2 x 8
 * bytes per point).
 */
tpcf_status tpcf_forward_multi(tpcf_plan plan, const float* d_delta_a, const float* d_w_a,
                               const float* d_delta_b, const float* d_w_b, const float* d_delta_c,
                               const float* d_w_c, int64_t pivot_begin, int64_t pivot_end, double* d_zeta,
                               double* d_norm, double* d_sums, void* stream);

/*
 * The forward above for callers that cannot allocate device memory: programs that
 * hand all device memory to their own pool allocator at start-up, hot loops that
 * must not enter the CUDA allocator (cudaMalloc/cudaFree can synchronise the
 * device), embedders with strict device-memory accounting.  The paper has no
 * counterpart: this is a library service.
 *
 * Same inputs, outputs and pivot range as tpcf_forward (no raw sums).  The call
 * allocates nothing: it reads d_delta and d_w directly and keeps its partial sums
 * in a fixed 16 MiB __device__ array.  The plan is created beforehand (plan creation
 * does allocate), and tpcf_plan_create_map also places that array on its device and
 * looks its address up, so the 16 MiB are taken during set-up and held until the
 * process exits.  If that look-up failed there, the first call on the device retries
 * it; such a first call should come before any stream capture.  The largest plan the
 * ABI allows (32 bins, m_max 16) needs 148 KB per CTA slot; the call runs as many
 * CTAs as there are slots in the array.  All calls share the array and each call
 * clears what must start at zero; calls whose GPU work overlaps (other streams,
 * host threads or plans at the same time) race on it and must be serialised.
 * Map plans without self-pair subtraction only (else TPCF_ERR_UNSUPPORTED); a plan
 * whose per-CTA partial sums (2 (m_max+1) K(K+1)/2 + K(K+1)/2 + 2K doubles) do not
 * fit is rejected with TPCF_ERR_INVALID_ARG and a message in tpcf_last_error().
 */
tpcf_status tpcf_forward_noalloc(tpcf_plan plan, const float* d_delta, const float* d_w,
                                 int64_t pivot_begin, int64_t pivot_end, double* d_zeta, double* d_norm,
                                 void* stream);

/*
 * Adjoint: d_grad[p] = dL/d(delta_p) for a real loss L of zeta over the same pivot
 * range, given d_dL_dzeta = dL/dRe(zeta) + i dL/dIm(zeta) (zeta layout) and the
 * normalisation d_norm from the matching forward.  Recomputes the moments a_m^k
 * instead of storing them.  With TPCF_SELF_PAIRS_SUBTRACT the derivative of the
 * subtracted diagonal is included (map plans; catalogue plans with self-pair
 * subtraction return TPCF_ERR_UNSUPPORTED).  d_grad (float[npoints], caller order for
 * catalogues) is overwritten.
 */
tpcf_status tpcf_backward(tpcf_plan plan, const float* d_delta, const float* d_w,
                          int64_t pivot_begin, int64_t pivot_end, const double* d_norm,
                          const double* d_dL_dzeta, float* d_grad, void* stream);

/*
 * Exact number of in-bin ordered pairs (i, j) whose pivot i lies in
 * [pivot_begin, pivot_end) and has w_i != 0, whatever w_j (the units of the
 * throughput figure).  d_counts (device, int64[3]) receives: the total, the pairs
 * visited as mirror images (equatorial-belt symmetry), the pairs visited singly
 * (catalogue plans visit every pair singly).
 */
tpcf_status tpcf_count_pairs(tpcf_plan plan, const float* d_w, int64_t pivot_begin, int64_t pivot_end,
                             int64_t* d_counts, void* stream);

/*
 * Autotuner of the map pair kernels' launch configuration (the paper has no GPU
 * design; this picks the tile-processing shape on the device at hand).  Times the
 * forward (passes bit 0) and/or the adjoint (bit 1) of the plan on a sample of pivots
 * of the caller's field for every candidate -- register variant sized for 3 or 2
 * resident CTAs per SM, CTAs per SM launched, rings summed in registers between
 * shared-memory flushes, and for the forward the tile layout (32 consecutive pivots,
 * or four runs of 8 a quarter turn apart whose lanes share the position angles on
 * rings with another pixel count) -- and keeps the fastest in the plan.  With both passes and
 * the environment variable TPCF_AUTOTUNE_CACHE naming a file, the result is appended
 * there, keyed by device, nside, bins and flags; a later autotune call or
 * tpcf_plan_create_map with the same key takes it from the file without measuring.
 * Results do not depend on the configuration beyond summation order.  Allocates and
 * frees temporaries (a gradient buffer of npoints floats for the adjoint);
 * synchronises `stream`.  Map plans without TPCF_CONTRACT_TC only (else
 * TPCF_ERR_UNSUPPORTED).
 */
tpcf_status tpcf_plan_autotune(tpcf_plan plan, const float* d_delta, const float* d_w, int32_t passes,
                               void* stream);
/* The plan's launch configuration: host int32[7] = forward (variant, CTAs per SM,
 * flush rings, tile layout: 0 consecutive pivots, 1 quarter-turn runs), adjoint
 * (variant, CTAs per SM, flush rings). */
tpcf_status tpcf_plan_launch_config(tpcf_plan plan, int32_t* config7);
/* Sets it (same layout); TPCF_ERR_INVALID_ARG for a configuration that does not fit. */
tpcf_status tpcf_plan_set_launch_config(tpcf_plan plan, const int32_t* config7);

/*
 * Halo of a pixel range, for splitting the adjoint across devices (map plans): the
 * smallest pixel range [*halo_begin, *halo_end) (whole HEALPix rings, RING order)
 * that holds every pivot with a neighbour in [begin, end) (a neighbour lies within
 * the outer bin edge, Sec. 3.1).  The adjoint restricted to the halo pivots is then
 * exact on [begin, end), so a device that owns that slice of dL/d(delta) needs no
 * contribution from the others.  An empty range gives an empty halo.  Host
 * outputs; reads two entries of the plan's ring table (synchronous).  Catalogue
 * plans: TPCF_ERR_UNSUPPORTED (their caller order has no spatial slices).
 */
tpcf_status tpcf_plan_halo(tpcf_plan plan, int64_t begin, int64_t end, int64_t* halo_begin, int64_t* halo_end);

/*
 * End-to-end call on HOST buffers: copies h_delta and h_w to the device, runs the
 * forward over all pivots and, if h_dL_dzeta != NULL, the adjoint, and copies
 * zeta, norm and (if h_grad != NULL) the gradient back.  Uses device staging
 * buffers owned by the plan (allocated on first use).  Synchronises `stream`.
 */
tpcf_status tpcf_run_host(tpcf_plan plan, const float* h_delta, const float* h_w,
                          const double* h_dL_dzeta, double* h_zeta, double* h_norm,
                          float* h_grad, void* stream);

/*
 * Batched execution (Sec. 3 estimator, for n independent maps): n map plans of any
 * mix of nside, bins and m_max, each with its own inputs and outputs, run as one
 * short launch sequence whose length does not depend on n.  One persistent pair
 * kernel per distinct (m_max, self-pair mode) runs the forward tiles of all its
 * plans from a shared work queue; the small per-entry kernels take every plan in
 * one launch.  When d_dL_dzeta != NULL the batch also runs the adjoint (every
 * d_dL_dzeta[i] and d_grad[i] must then be set; not with self-pair subtraction).
 *
 * tpcf_batch_create validates the arguments, synchronises the plans' last streams
 * and records the sequence into a CUDA graph: the pointers are baked in, so the
 * buffers and plans must outlive the batch.  A plan may appear once per batch, and
 * its batch and its single calls must not run concurrently (they share the plan's
 * scratch).  Arrays: plans, d_delta, d_w (float32[npix] each), d_zeta
 * (double[(m_max+1) K K 2]), d_norm (double[K K]), d_dL_dzeta (same shape as
 * zeta), d_grad (float[npix], overwritten): host arrays of n device pointers.
 * Errors: INVALID_ARG (NULL, n outside [1, 256], duplicate plan), UNSUPPORTED
 * (catalogue plan, adjoint with self-pair subtraction), CUDA/OOM.
 *
 * tpcf_batch_launch replays the graph on `stream` (asynchronous; tpcf_plan_sync on
 * any member reports device errors).  tpcf_batch_kernel_launches gives the kernels
 * of one replay.  tpcf_batch_destroy synchronises and frees (NULL is a no-op).
 */
tpcf_status tpcf_batch_create(tpcf_batch* out, const tpcf_plan* plans, int32_t n,
                              const float* const* d_delta, const float* const* d_w,
                              double* const* d_zeta, double* const* d_norm,
                              const double* const* d_dL_dzeta, float* const* d_grad,
                              void* stream);
tpcf_status tpcf_batch_launch(tpcf_batch batch, void* stream);
int64_t tpcf_batch_kernel_launches(tpcf_batch batch);
void tpcf_batch_destroy(tpcf_batch batch);

/* Convenience: create, launch once and destroy a batch. */
tpcf_status tpcf_forward_batched(const tpcf_plan* plans, int32_t n, const float* const* d_delta,
                                 const float* const* d_w, double* const* d_zeta,
                                 double* const* d_norm, const double* const* d_dL_dzeta,
                                 float* const* d_grad, void* stream);

/* Synchronise the plan's last stream and return any latched device error. */
tpcf_status tpcf_plan_sync(tpcf_plan plan);

/* Free everything the plan owns (synchronises with its pending work). NULL is a no-op. */
void tpcf_plan_destroy(tpcf_plan plan);

/*
 * FP32-pipe throughput of the current device, measured (no counterpart in the paper; the
 * denominator of the pair kernels' roofline): tflops[0] with scalar FMAs, tflops[1] with
 * packed two-lane FMAs (f32x2), each the best of three timed launches of 8 x SMs CTAs.
 * Host output double[2]; synchronises `stream`; allocates a small temporary.
 */
tpcf_status tpcf_probe_fp32_peak(double* tflops, void* stream);

/*
 * Test hooks for the error paths (no counterpart in the paper).
 * tpcf_test_fail_allocation(n): the n-th device allocation the library attempts from
 * now on fails as if the device were out of memory (the calls above then return
 * TPCF_ERR_OOM); n <= 0 disarms.  tpcf_test_live_allocations(): the number of device
 * allocations the library holds (plans, batches, staging), so that a test can check
 * that a failed call leaked nothing.
 */
void tpcf_test_fail_allocation(int64_t n);
int64_t tpcf_test_live_allocations(void);

#ifdef __cplusplus
}
#endif

#endif /* TPCF_H */
