/*
 * smart.h -- C ABI of the B300 (sm_103a) spherical shear-based aperture-mass
 * library (SMART, arXiv 2609.11181).
 *
 * The problem (Sect. 2-3 of the paper): for every output HEALPix pixel
 * centre theta_0, sum over the galaxies (brute force, Sect. 3.1 / 3.4) or
 * the binned shear pixels (pixel-based, Sect. 3.2) that lie within the
 * aperture radius theta_ap; rotate each shear into tangential and cross
 * components with the spherical position angle (Sect. 2.3, Eq. 4),
 * weight by the filter Q, and normalise by the mean weight density inside
 * the aperture (the summed approach, Sect. 2.4).  Outputs per centre:
 * M_ap^E, M_ap^B (Eq. 7), the noise variance (Eq. 8), the weight
 * sum and the member count.
 *
 * Conventions shared by every call
 *  - Array arguments are DEVICE pointers owned by the caller unless a
 *    parameter says "host".  The caller keeps inputs alive until
 *    smart_sync() returns.
 *  - Calls run asynchronously on the context's CUDA stream (the stream
 *    given to smart_create, 0 = legacy default stream) and return at once.
 *    The map calls (smart_map_*), smart_bin_galaxies and smart_set_binned*
 *    never wait for the GPU: errors that only the device can see (invalid
 *    galaxy coordinates, a full guard-band list) are reported by the next
 *    smart_sync.  smart_sync waits with its own deadline.  The set-up calls
 *    that size tables from device results -- smart_set_targets (the ring
 *    tables of every map kind are built there), smart_batch_create -- and
 *    smart_last_fp64_decisions wait for the stream, polling, at most the
 *    context's wait limit (smart_set_wait_limit, default 600 s); past it
 *    they return SMART_E_TIMEOUT (or -1).  smart_timing_read waits with the
 *    deadline it is given; the MLP parameter, scaler and state copies wait
 *    for their handle's stream (smart_mlp_sync takes a deadline).
 *  - The library owns only its internal scratch (sorted catalogue, offsets,
 *    ring tables, binned maps it made itself) and frees it in
 *    smart_destroy().
 *  - No call aborts, traps or throws.  Errors come back as a smart_status;
 *    smart_last_error() gives a one-line description.  Argument errors are
 *    detected on the host before anything is launched.
 *  - Sizes are int64.  nside values must be powers of two in [1, 8192].
 *  - Angles: ra/dec in degrees (float64); theta_ap in arcmin.  The shear
 *    components e1, e2 are given in the local (East = +RA, North = +Dec)
 *    basis; a positive tangential component means alignment perpendicular
 *    to the direction of the aperture centre.
 *  - Pixel indices are RING-scheme indices (Gorski et al. 2005, Sect. 3).
 */
#ifndef SMART_H
#define SMART_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SMART_OK = 0,
    SMART_E_ARG = 1,        /* invalid argument (detected on the host)       */
    SMART_E_NOMEM = 2,      /* device allocation failed                       */
    SMART_E_CUDA = 3,       /* a CUDA runtime call or kernel launch failed   */
    SMART_E_STATE = 4,      /* call order violated (e.g. map before data)    */
    SMART_E_TIMEOUT = 5,    /* smart_sync deadline passed                    */
    SMART_E_OVERFLOW = 6,   /* a size exceeds an internal limit              */
    SMART_E_INTERNAL = 7
} smart_status;

typedef enum {
    SMART_FILTER_POLY = 1,      /* Schneider (1996): Q = 6/pi x^2 (1 - x^2) / theta_ap^2      */
    SMART_FILTER_SCHIRMER = 2,  /* Schirmer et al. (2007): Q = tanh(x/xc)/(x/xc) /
                                   (1 + e^(6-150x) + e^(-47+50x)) / theta_ap^2               */
    SMART_FILTER_JARVIS = 3     /* Jarvis et al. (2004), Gaussian-type, scale s = xc:
                                   Q = (x/s)^2 exp(-x^2 / (2 s^2)) / (4 pi s^2) / theta_ap^2,
                                   truncated at x = 1 (the aperture radius)                  */
} smart_filter_kind;

typedef struct {
    int kind;                   /* smart_filter_kind                          */
    double xc;                  /* Schirmer core (default 0.15) or Jarvis scale
                                   in units of theta_ap (default 0.25); ignored
                                   by the polynomial filter                   */
} smart_filter;

/* Output buffers, one entry per target pixel (device pointers; any may be
   NULL to skip that output). */
typedef struct {
    double *sum_w;      /* f64 [n]: sum of weights in the aperture (Sect. 2.4)     */
    float *map_e;       /* f32 [n]: M_ap^E, summed normalisation (Eq. 7)          */
    float *map_b;       /* f32 [n]: M_ap^B                                          */
    float *var;         /* f32 [n]: sigma_ap^2 (Eq. 8 with weights)          */
    int64_t *count;     /* i64 [n]: galaxies in the aperture (brute force) or
                                    galaxies in the member pixels (pixel mode)    */
    int32_t *members;   /* i32 [n]: aperture members = (centre, point) pairs summed:
                                    galaxies (brute force) or pixels, empty or
                                    not, whose centre is inside (pixel mode)      */
} smart_maps;

typedef struct smart_ctx smart_ctx;

/*
 * Create a context for maps on the RING grid at nside_out with aperture
 * radius theta_ap_arcmin (0 < theta_ap <= 60 deg) and the given filter.
 * nside_bin is the grid that galaxies are sorted / binned on (Sect. 3.2,
 * 3.4).  cuda_stream is a cudaStream_t (may be NULL).  On success *out
 * holds the new context; on failure *out is NULL.
 */
smart_status smart_create(int nside_out, const smart_filter *filter,
                          double theta_ap_arcmin, int nside_bin,
                          void *cuda_stream, smart_ctx **out);

/* Release every device buffer the context owns.  NULL is a no-op. */
void smart_destroy(smart_ctx *ctx);

/* Block until the context's stream is idle, polling with the given deadline
   in seconds (<= 0: wait forever).  Returns SMART_E_TIMEOUT if the deadline
   passes (the work keeps running), SMART_E_CUDA if an asynchronous error
   surfaced. */
smart_status smart_sync(smart_ctx *ctx, double timeout_s);

/* One-line description of the last error on this context ("" if none). */
const char *smart_last_error(const smart_ctx *ctx);

/*
 * Target (output) pixels: n RING indices at nside_out, int64, device
 * pointer.  They must be sorted ascending and unique (SMART_E_ARG if not).
 * The array is copied; the caller may free it after smart_sync.  This call
 * also builds every table the maps need for these targets (ring pairs and
 * Toeplitz tables once per context; target tiles, the pixel map's ring
 * classes and general-target list, the brute-force target groups), so it
 * waits for the stream, at most the wait limit (SMART_E_TIMEOUT after it);
 * the map calls then only enqueue kernels.
 */
smart_status smart_set_targets(smart_ctx *ctx, const int64_t *ring_pix, int64_t n);

/* Wait limit (seconds, >= 0; 0 = none) of the set-up calls' waits on this
   context (smart_set_targets, smart_last_fp64_decisions).  Default 600.
   SMART_E_ARG for a negative value.  Host only. */
smart_status smart_set_wait_limit(smart_ctx *ctx, double seconds);

/*
 * Sect. 3.4 steps 1-3 and Sect. 3.2 step 2: assign each galaxy its RING
 * pixel at nside_bin (bit-exact with the FP64 definition), stable-sort the
 * catalogue by pixel with a GPU LSD radix sort, build the offset table
 * (first galaxy of each pixel) and the per-pixel sums
 *   G1 = sum w e1, G2 = sum w e2, W = sum w, S2 = sum w^2 (e1^2 + e2^2),
 *   n = count
 * in float32, accumulated in sorted order.  ra/dec: f64 degrees; e1, e2,
 * w: f32; all device pointers of n entries.  w may be NULL (all weights 1).
 * Replaces any binned map given earlier with smart_set_binned.  Does not
 * wait: galaxies with non-finite ra/dec or |dec| > 90 are sorted after every
 * pixel and left out of the catalogue and the binned map (they belong to no
 * pixel), and the next smart_sync returns SMART_E_ARG with their number.
 */
smart_status smart_bin_galaxies(smart_ctx *ctx, const double *ra_deg,
                                const double *dec_deg, const float *e1,
                                const float *e2, const float *w, int64_t n);

/*
 * Give per-pixel sums directly (full-sky RING arrays at nside_bin, 12
 * nside_bin^2 entries each, device pointers).  Same meaning as the sums of
 * smart_bin_galaxies.  The arrays are copied (asynchronously, on the
 * context's stream) into the library's packed layout; call again after
 * changing them.  Pixel-based maps only.
 */
smart_status smart_set_binned(smart_ctx *ctx, const float *G1, const float *G2,
                              const float *W, const float *S2, const int32_t *n_p);

/*
 * The binned input of a footprint: only the pixels the caller has, as runs
 * of consecutive RING pixels (a cap gives one or two runs per ring).  px
 * (float4 per pixel: G1, G2, S2, W, 16-byte aligned) and n_p hold the runs'
 * pixels back to back, n_compact of each; runs holds n_runs triples
 * (first RING pixel, length, position of the run's first pixel in px / n_p),
 * int64.  All device pointers.  The pixels are copied into the context's own
 * full-sky map; every other pixel is zero when the map was just made, when it
 * held other data (smart_bin_galaxies, smart_set_binned) or when clear != 0,
 * and otherwise keeps the value of the last call.  A caller whose footprint's
 * data stay zero outside the runs thus ships only the runs: the maps equal
 * those of the full-sky input bit for bit.  A run that does not fit the map
 * or the compact arrays is skipped and the next smart_sync returns
 * SMART_E_ARG.  Asynchronous; SMART_E_ARG for bad pointers or sizes.
 */
smart_status smart_set_binned_runs(smart_ctx *ctx, const float *px, const int32_t *n_p, const int64_t *runs,
                                   int64_t n_runs, int64_t n_compact, int clear);

/*
 * Same input in the library's native layout: px holds 4 floats per pixel
 * (G1, G2, S2, W) -- note S2 before W -- for the 12 nside_bin^2 RING pixels
 * (device pointer, 16-byte aligned), n_p the counts.  Both arrays are
 * borrowed, not copied: they are read by every later map call, so keep them
 * alive and unchanged until then.  smart_set_binned copies its arrays into
 * this layout instead.
 */
smart_status smart_set_binned_packed(smart_ctx *ctx, const float *px, const int32_t *n_p);

/*
 * Brute-force map at galaxy positions (Sect. 3.1 steps 1-5; neighbours
 * found through the sorted catalogue of Sect. 3.4).  Requires
 * smart_bin_galaxies and smart_set_targets.  Membership is s^2 <= T with
 * s the chord between unit vectors and T = 4 sin^2(theta_ap/2), decided
 * exactly as in float64.
 */
smart_status smart_map_bruteforce(smart_ctx *ctx, const smart_maps *out);

/*
 * Pixel-based map (Sect. 3.2 steps 3-5): filter and rotation evaluated at
 * the centres of the binned pixels whose centres are inside the aperture.
 * Requires binned data (smart_bin_galaxies or smart_set_binned) and
 * smart_set_targets.
 */
smart_status smart_map_pixel(smart_ctx *ctx, const smart_maps *out);

/*
 * Pixel-based map with each bin pixel placed at its galaxies' barycentre
 * (Sect. 3.3, sphS_pixB).  Needs smart_bin_galaxies.  Every bin pixel that
 * holds galaxies becomes one point at the w-weighted mean of its galaxies'
 * unit vectors (float64, normalised) carrying the pixel's sums G1, G2, W,
 * S2; points are members when their barycentre lies within theta_ap of the
 * target (float64 decision near the edge, as for galaxies), and the sums are
 * normalised like the other maps.  out->count = galaxies in member pixels,
 * out->members = member pixels.  The records are built once per catalogue.
 */
smart_status smart_map_barycentre(smart_ctx *ctx, const smart_maps *out);

/*
 * Cartesian (projected) shear-based aperture mass at galaxy positions,
 * projS_pos (Sect. 2.2; algorithm of Sect. 5.2.1 steps 1-4), over the
 * catalogue of smart_bin_galaxies and the targets of smart_set_targets:
 *  1. galaxies go to the plane tangent at the reference point (ra_c, dec_c)
 *     (degrees) by the gnomonic projection of Sect. 2.2.1; their shear is
 *     rotated so that its orientation stays relative to the local North
 *     (Sect. 2.2.2); galaxies more than 90 degrees from the reference point
 *     have no image and are left out;
 *  2. the targets' pixel centres go to the same plane;
 *  3. per target, every galaxy whose plane distance is <= theta_ap is a
 *     member; Q is evaluated at the plane distance (same filter kinds as the
 *     spherical maps), gamma_+ / gamma_x from the bearing in the plane;
 *  4. the summed normalisation with A = pi theta_ap^2, the aperture's area
 *     in the plane: M = A S / sum_w, sigma^2 = A^2 V / (2 sum_w^2).
 * Membership is decided like the float64 definition (float32 outside a
 * guard band, float64 inside it), so counts are exact.  Outputs as for
 * smart_map_bruteforce (count = members = galaxies in the plane aperture);
 * a target with no image gets zeros.  SMART_E_STATE without a catalogue or
 * with the averaged normalisation (only the summed form is implemented),
 * SMART_E_ARG for a bad reference point.  Asynchronous on the context
 * stream; the catalogue must stay unchanged until it completes.
 */
smart_status smart_map_projected(smart_ctx *ctx, double ra_c_deg, double dec_c_deg, const smart_maps *out);

/*
 * Equal-area annulus statistics of two maps of this context's targets about
 * a reference point (Sect. 5.2.2): with d the angular distance of a target's
 * pixel centre from (ra_ref, dec_ref) (degrees), annulus k of nbins holds
 * the targets with 1 - cos d in [k, k + 1) (1 - cos rmax_rad) / nbins --
 * annuli of equal area out to rmax_rad (radians, in (0, pi]).  Per annulus:
 * count[k] (int64), and the mean and population standard deviation of
 * eps = (m_x - m_ref) / sigma(m_ref) (Eq. 12), sigma(m_ref) being the
 * population standard deviation of m_ref over all the targets.  m_x, m_ref:
 * float32 [n_targets], device; count, mean, sd: device arrays of nbins (any
 * may be NULL).  Targets beyond rmax_rad are not binned.  Sums are float64
 * atomics (order-dependent in the last bits).  Asynchronous on the context
 * stream.  SMART_E_ARG for nbins outside [1, 2^20] or bad angles.
 */
smart_status smart_annulus_stats(smart_ctx *ctx, double ra_ref_deg, double dec_ref_deg, double rmax_rad,
                                 const float *m_x, const float *m_ref, int nbins, int64_t *count,
                                 double *mean, double *sd);

/*
 * Normalisation of the maps of a context (Sect. 2.4).
 * SMART_NORM_SUMMED (default): M = A S / sum_w with A the aperture area,
 *   sigma^2 = A^2 V / (2 sum_w^2) (the paper's default form).
 * SMART_NORM_AVERAGED: each bin pixel's shear is normalised by that pixel's
 *   own weight W and multiplied by the pixel area A_pix (galaxies carry
 *   w A_pix / W of their bin pixel): M = sum Q gamma+ A_pix / W,
 *   sigma^2 = 1/2 sum Q^2 S2 (A_pix / W)^2; sum_w stays the aperture's weight
 *   and must be requested.  Applies to smart_map_pixel, smart_map_barycentre
 *   and smart_map_bruteforce; batches reject contexts in this mode.
 */
typedef enum { SMART_NORM_SUMMED = 0, SMART_NORM_AVERAGED = 1 } smart_norm;
smart_status smart_set_normalisation(smart_ctx *ctx, int mode);


/* ---- batched pixel-based maps ----------------------------------------- */

typedef struct smart_batch smart_batch;

/*
 * Many pixel-based maps (Sect. 3.2) as one persistent launch.  Each map is a
 * context prepared for smart_map_pixel (targets and binned data set, all
 * contexts with the same filter kind); outs[m] receives map m (its device
 * buffers must stay valid for the life of the batch).  The work of all maps
 * is split into items (tiles of an output ring, chunks of targets) ordered
 * longest first and claimed dynamically by resident CTAs.  With autotune != 0
 * a few launch shapes are timed on this batch (the maps are computed while
 * tuning) and the fastest is kept; the launch is then captured in a CUDA
 * graph on cuda_stream.  Binned inputs are read when the graph runs, so
 * borrowed (packed) maps may change between runs.  Returns SMART_E_ARG for
 * mixed filter kinds.  A NULL stream means a private stream of the batch
 * (graphs cannot be captured on the legacy default stream); it orders itself
 * against the legacy default stream.
 */
smart_status smart_batch_create(smart_ctx *const *ctxs, const smart_maps *outs, int n_maps, int autotune,
                                void *cuda_stream, smart_batch **out);

/* Launch the captured graph on the batch stream (asynchronous). */
smart_status smart_batch_run(smart_batch *batch);

/* Launch shape chosen (resident CTAs per SM, item order) and the tuned time. */
smart_status smart_batch_info(const smart_batch *batch, int *ctas_per_sm, int *longest_first,
                              int64_t *n_items, double *tuned_ms);

/* Last error of a batch; with NULL, why this thread's last smart_batch_create failed. */
const char *smart_batch_last_error(const smart_batch *batch);

/* Waits for the batch stream, then frees the batch (not the contexts). */
void smart_batch_destroy(smart_batch *batch);

/* One-shot: create (no autotune), run once, destroy.  Synchronous. */
smart_status smart_map_batched(smart_ctx *const *ctxs, const smart_maps *outs, int n_maps);

/* ---- geometry utilities (Sect. 3, HEALPix RING; stateless) ---------- */

/* pix[k] = RING pixel at nside of (ra_deg[k], dec_deg[k]); bit-exact with
   the float64 definition.  Device pointers; stream may be NULL. */
smart_status smart_ang2pix(int nside, const double *ra_deg, const double *dec_deg,
                           int64_t n, int64_t *pix, void *cuda_stream);

/* vec[3k..3k+2] = unit vector of the centre of RING pixel pix[k] (f64). */
smart_status smart_pix2vec(int nside, const int64_t *pix, int64_t n, double *vec,
                           void *cuda_stream);

/* Host helper: the chord^2 threshold T = 4 sin^2(theta_ap/2) the library
   uses for theta_ap given in arcmin. */
double smart_chord2(double theta_ap_arcmin);

/* ---- inspection (tests, diagnostics) ------------------------------- */

/*
 * Copy the sorted catalogue out: perm[i] = input index of the galaxy at
 * sorted position i, pix[i] = its pixel (both n entries), offsets[p] =
 * sorted position of the first galaxy of pixel p (12 nside_bin^2 + 1
 * entries).  Device pointers; any may be NULL.
 */
smart_status smart_get_catalog(smart_ctx *ctx, int64_t *perm, int64_t *pix, int64_t *offsets);

/* Copy the binned map out (full-sky arrays at nside_bin). */
smart_status smart_get_binned(smart_ctx *ctx, float *G1, float *G2, float *W,
                              float *S2, int32_t *n_p);

/* Number of member tests that fell inside the float32 guard band and were
   decided in float64 by the last map call (host value; waits for the
   stream at most the wait limit; -1 on a timeout or error). */
int64_t smart_last_fp64_decisions(smart_ctx *ctx);

/* ---- kernel timing (diagnostics; not part of the method) ------------ */

/* Kernels and phases whose launches can be timed. */
typedef enum {
    SMART_KT_PIXEL_TOEPLITZ = 0,   /* pixel mode, rings of equal-length ring pairs */
    SMART_KT_PIXEL_GENERAL = 1,    /* pixel mode, the other targets */
    SMART_KT_GALAXY = 2,           /* brute force, main kernel */
    SMART_KT_GALAXY_BAND = 3,      /* brute force, float64 decisions of guard-band pairs */
    SMART_KT_GALAXY_FINALISE = 4,  /* brute force, normalisation */
    SMART_KT_BIN_KEYS = 5,         /* smart_bin_galaxies: pixel keys (ang2pix) */
    SMART_KT_BIN_SORT = 6,         /* smart_bin_galaxies: every radix pass */
    SMART_KT_BIN_RECORDS = 7,      /* smart_bin_galaxies: permuted galaxy records */
    SMART_KT_BIN_PIXEL_SUMS = 8,   /* smart_bin_galaxies: per-pixel sums */
    SMART_KT_BARY_BUILD = 9,       /* smart_map_barycentre: barycentre records (once per catalogue) */
    SMART_KT_BARY_MAP = 10,        /* smart_map_barycentre: main kernel */
    SMART_KT_PIXEL_BAND = 11,      /* pixel mode, float64 decisions of the general kernel's guard-band pairs */
    SMART_KT_PROJ_RECORDS = 12,    /* smart_map_projected: plane positions and rotated shears */
    SMART_KT_PROJ_MAP = 13,        /* smart_map_projected: main kernel */
    SMART_KT_PROJ_BAND = 14,       /* smart_map_projected: float64 decisions of guard-band pairs */
    SMART_KT_COUNT = 15
} smart_kernel_id;

/*
 * enable != 0: start a fresh timing record; from now on every launch of the
 * kernels above made through this context is bracketed by two CUDA events
 * recorded on the context stream.  enable == 0: stop and discard the record.
 * Events are created on first use (cudaEventCreate) and reused.
 */
smart_status smart_timing_enable(smart_ctx *ctx, int enable);

/*
 * Number of recorded launches of `kernel` and their summed duration in ms
 * (host outputs).  Waits for the recorded events, polling with a deadline of
 * timeout_s seconds (<= 0: no deadline); SMART_E_TIMEOUT if it passes.
 */
smart_status smart_timing_read(smart_ctx *ctx, int kernel, int64_t *launches, double *total_ms,
                               double timeout_s);

/*
 * Positions (into the target array) of the targets that the last pixel map
 * sent to the general kernel; the others went to the Toeplitz kernel.
 * *n_gen (host) receives their number; idx (device, int32, capacity cap)
 * receives the positions unless NULL.  The lists are built by
 * smart_set_targets; SMART_E_STATE for an empty target set or after a
 * smart_set_targets that failed.  Asynchronous on the context stream.
 */
smart_status smart_get_general_targets(smart_ctx *ctx, int32_t *idx, int64_t cap, int64_t *n_gen);

/*
 * The general kernel's mirror pairs (a design of this library; the paper has
 * no counterpart).  Every HEALPix ring is symmetric about the meridians
 * phi = m pi/4, so a general target whose mirror image about one of them is
 * a target as well shares each pair's geometry with it: such pairs are
 * found once per target set (meridians 0, pi/2, pi/4, 3 pi/4 in that order,
 * each target in at most one pair) and run in one thread each.  *n_pairs and
 * *n_single (host) receive the number of pairs and of general targets left
 * unpaired (n_gen = 2 n_pairs + n_single); pairs (device, int32, capacity
 * cap pairs) receives the pairs' target positions as (lower, image) unless
 * NULL.  Built by smart_set_targets; SMART_E_STATE for an empty target set
 * or after a smart_set_targets that failed.
 * Asynchronous on the context stream.
 */
smart_status smart_get_general_pairs(smart_ctx *ctx, int32_t *pairs, int64_t cap, int64_t *n_pairs,
                                     int64_t *n_single);

/*
 * FMA throughput probe (diagnostics; the paper has no counterpart).  Enqueues
 * one kernel of ctas_per_sm (1..8) CTAs of 256 threads per SM on the stream;
 * every thread runs iters x 128 fused multiply-add instructions in eight
 * independent chains, in float32 (bits = 32), float64 (bits = 64) or on
 * float32 pairs, two FMAs per packed instruction (bits = 32 |
 * SMART_PROBE_PACKED; sm_100 and later).  *flops (host)
 * receives the kernel's floating-point operations (an FMA counts 2); the
 * caller times the launch with events on the same stream and divides.
 * Returns at once; SMART_E_ARG for bad arguments, SMART_E_CUDA on a launch
 * failure.  Allocates nothing.
 */
enum { SMART_PROBE_PACKED = 0x100 };
smart_status smart_fma_probe(int bits, int64_t iters, int ctas_per_sm, void *cuda_stream, double *flops);

/*
 * Testing aid (no counterpart in the paper).  In the pixel map, a target of
 * the general kernel with pairs inside the float32 guard band takes a slot
 * whose float64 decisions a follow-up kernel makes; a target that finds no
 * free slot makes them itself, with the same code.  n_slots > 0 caps the
 * slots at n_slots so that tests can run that second path; 0 restores the
 * default (65536 + n_general / 8).  SMART_E_ARG for n_slots < 0.  Host only.
 */
smart_status smart_set_band_slot_limit(smart_ctx *ctx, int64_t n_slots);

/* ---- learned residual correction of the pixel-based map ------------ */

/*
 * The galaxy-level map (Sect. 3.1) and the pixel-based map (Sect. 3.2)
 * differ because the second moves every galaxy to its pixel centre.  A small
 * network predicts the per-pixel difference M_bf^E - M_pix^E from four
 * features of the pixel-based map; the corrected map is written to a
 * separate array and the plain map stays the fallback.  The paper prescribes
 * no such network: features, architecture (4 -> 64 -> 64 -> 1, SiLU), loss
 * (mean squared error on the standardised target) and optimiser (Adam,
 * beta1 0.9, beta2 0.999, eps 1e-8) are this library's.
 *
 * Feature row of a target (float32, 4 values):
 *   [0] M_pix^E   [1] sum of weights   [2] variance of the galaxy counts
 *   n_p over the K bin pixels whose centre lies in the aperture,
 *   sum n_p^2 / K - (sum n_p / K)^2   [3] z of the target pixel centre.
 *
 * Parameter vector (float32 master copy, SMART_MLP_NPARAMS values):
 *   W1 [64][4], b1 [64], W2 [64][64], b2 [64], w3 [64], b3, W[out][in].
 * SMART_MLP_BF16: the three weight matrices are used as their bfloat16
 * roundings (biases float32); the 64 x 64 products run on bf16 tensor cores
 * with float32 accumulation, the first hidden activation and the gradient at
 * the second pre-activation are rounded to bfloat16 as tensor-core operands.
 * SMART_MLP_FP32: every value and product in float32 (a checking mode).
 *
 * All array arguments are device pointers owned by the caller unless marked
 * (host).  Calls run on the handle's stream; those marked "syncs" wait for
 * it.  Errors: SMART_E_ARG bad argument, SMART_E_STATE no parameters yet,
 * SMART_E_NOMEM, SMART_E_CUDA; smart_mlp_last_error tells which.
 */
#define SMART_MLP_FEATURES 4
#define SMART_MLP_NPARAMS 4545

typedef enum { SMART_MLP_BF16 = 0, SMART_MLP_FP32 = 1 } smart_mlp_precision;
typedef struct smart_mlp smart_mlp;

/*
 * Features (and training targets) of ctx's targets.  pixel_map: the output
 * of smart_map_pixel on ctx with map_e, sum_w, count and members set.
 * brute_map (may be NULL): the output of smart_map_bruteforce for the same
 * targets, map_e and sum_w set.  feat: out [n][4].  target: out [n],
 * brute_map->map_e - pixel_map->map_e (needs brute_map; may be NULL).
 * valid: out [n] (may be NULL), 1 where the pixel-based (and galaxy-level)
 * weight sum is positive.  sum_n2: out [n] (may be NULL), sum of n_p^2 over
 * the aperture's bin pixels.  Membership is that of the map kernels, so the
 * count moments are exact integers.
 */
smart_status smart_mlp_features(smart_ctx *ctx, const smart_maps *pixel_map, const smart_maps *brute_map,
                                float *feat, float *target, uint8_t *valid, int64_t *sum_n2);

smart_status smart_mlp_create(int precision, void *cuda_stream, smart_mlp **out);
void smart_mlp_destroy(smart_mlp *h);
const char *smart_mlp_last_error(const smart_mlp *h);
/* Bounded wait for the handle's stream (timeout_s <= 0: no deadline). */
smart_status smart_mlp_sync(smart_mlp *h, double timeout_s);

/* Load (host) float32 parameters; resets the Adam moments and step count. Syncs. */
smart_status smart_mlp_set_params(smart_mlp *h, const float *params);
/* Copy the float32 master parameters to params (host). Syncs. */
smart_status smart_mlp_get_params(smart_mlp *h, float *params);

/* Standardisation (host, 10 doubles): mean[4], sd[4] of the features, mean
   and sd of the target; sd > 0. */
smart_status smart_mlp_set_scaler(smart_mlp *h, const double *scaler);
smart_status smart_mlp_get_scaler(smart_mlp *h, double *scaler);
/* Fit the standardisation to rows `rows` (int32 [n]; NULL = rows 0..n-1) of
   feat [.][4] and target: float64 mean and population sd, deterministic.  Syncs. */
smart_status smart_mlp_fit_scaler(smart_mlp *h, const float *feat, const float *target, const int32_t *rows,
                                  int64_t n);

/*
 * Gradient of the mean squared error over the minibatch idx[0..batch)
 * (int32 rows of feat/target; NULL = rows 0..batch-1) with respect to the
 * parameters.  grad_out (may be NULL): out [SMART_MLP_NPARAMS + 1]; the last
 * value is the sum of squared errors over the batch.  Deterministic (fixed
 * reduction order).
 */
smart_status smart_mlp_gradient(smart_mlp *h, const float *feat, const float *target, const int32_t *idx,
                                int64_t batch, float *grad_out);
/* Gradient as above, then one Adam step with learning rate lr; loss_out
   (may be NULL): out [1], the batch's mean squared error. */
smart_status smart_mlp_train_step(smart_mlp *h, const float *feat, const float *target, const int32_t *idx,
                                  int64_t batch, float lr, float *loss_out);
/* Adam steps taken since the parameters were set (host value). */
int64_t smart_mlp_step(const smart_mlp *h);

/*
 * Corrected map: map_out[i] = map_plain[i] + sd_t * net(feat_i) + mean_t.
 * Where a feature is not finite, the weight sum is not positive or a
 * standardised feature lies beyond +-8, map_out[i] = map_plain[i] and
 * n_fallback (may be NULL, device counter, not cleared here) is incremented.
 * correction (may be NULL): out, the added value (0 at fallbacks).
 * map_out must not alias map_plain.
 */
smart_status smart_mlp_infer(smart_mlp *h, const float *feat, const float *map_plain, int64_t n,
                             float *map_out, float *correction, unsigned long long *n_fallback);

/*
 * Checkpoint: parameters, Adam moments, step count and standardisation in
 * a flat byte buffer (host).  get_state with buf NULL only reports the size.
 * set_state rejects a buffer of another size, version or precision.  Sync.
 */
smart_status smart_mlp_get_state(smart_mlp *h, void *buf, int64_t cap, int64_t *size);
smart_status smart_mlp_set_state(smart_mlp *h, const void *buf, int64_t size);

/* ---- catalogue sort without device allocation ---------------------- */

/*
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot call cudaMalloc or cudaFree when they need a sort: code that
 * runs inside a fixed device-memory budget handed out by its own pool, host
 * threads that must not take the device-wide synchronisation those calls
 * imply, and runtimes that forbid allocation inside their scheduling
 * regions.  It computes the same sort as smart_bin_galaxies without a
 * context: the pixel key of every galaxy (RING, nside), a stable radix sort
 * by key, and the offsets of each pixel's run.
 *
 *   nside    power of two in [1, 8192]
 *   ra, dec  n galaxy positions in degrees (device, f64)
 *   n        0 <= n <= 1048576 (2^20); larger n returns SMART_E_OVERFLOW
 *   pix      out, n entries (device): pixel of the galaxy at sorted position i
 *   perm     out, n entries (device): input index of that galaxy
 *   offsets  out, 12 nside^2 + 1 entries (device): sorted position of the
 *            first galaxy of pixel p; offsets[12 nside^2] = valid galaxies.
 *   stream   cudaStream_t (NULL = legacy default stream)
 *
 * Galaxies with non-finite ra/dec or |dec| > 90 get the key 12 nside^2 and
 * sort after every pixel; they are not reported as an error here.
 *
 * The call allocates nothing.  Its working memory is one fixed array of
 * about 10.5 MB in the library's own device data, held by every GPU that
 * loads the library until the process exits.  The first call on each device
 * looks up that array's device address with that device current; make that
 * first call before any stream capture.  The address is kept for the life of
 * the process: after cudaDeviceReset (or a reset of the primary context) it
 * is stale, and the entry point must not be called again in that process.  All calls share the array, and it
 * keeps the last call's contents: calls that overlap on the GPU (on two
 * streams, or from two host threads, without ordering between them) race and
 * give wrong results.  The work is enqueued on the stream and the call
 * returns without waiting; SMART_E_ARG / SMART_E_OVERFLOW are returned
 * before anything is enqueued, SMART_E_CUDA on a launch or look-up failure.
 */
smart_status smart_sort_catalog_noalloc(int nside, const double *ra, const double *dec,
                                        int64_t n, uint32_t *pix, uint32_t *perm,
                                        int32_t *offsets, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SMART_H */
