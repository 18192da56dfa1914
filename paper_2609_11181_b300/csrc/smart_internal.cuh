// smart_internal.cuh -- device helpers and the context of the SMART library.
//
// Float64 on the device is kept to what must be exact: HEALPix indices and
// pixel centres, the ring-pair constants of the aperture kernels, the rare
// guard-band re-decisions of aperture membership, and the final division by
// the weight sum.  Everything per pair runs in float32.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <unordered_set>
#include <utility>
#include <vector>

#include "../../include/smart.h"

#define SMART_PI 3.14159265358979323846

namespace smart {

// ---------------------------------------------------------------------------
// Float64 sine/cosine with a fixed operation sequence.
//
// Exact reduction to a signed remainder of at most half a quadrant (exact by
// Sterbenz's lemma), then the Maclaurin series of sin (to t^19) and cos (to
// t^20) by Horner's rule with fused multiply-adds.  Every operation is an
// explicit round-to-nearest intrinsic so that the result does not depend on
// compiler contraction; pixel centres therefore agree bit for bit with any
// other implementation of the same sequence.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void series_sincos(double t, double &s, double &c) {
    const double t2 = __dmul_rn(t, t);
    double ps = -1.0 / 121645100408832000.0;
    ps = __fma_rn(ps, t2, 1.0 / 355687428096000.0);
    ps = __fma_rn(ps, t2, -1.0 / 1307674368000.0);
    ps = __fma_rn(ps, t2, 1.0 / 6227020800.0);
    ps = __fma_rn(ps, t2, -1.0 / 39916800.0);
    ps = __fma_rn(ps, t2, 1.0 / 362880.0);
    ps = __fma_rn(ps, t2, -1.0 / 5040.0);
    ps = __fma_rn(ps, t2, 1.0 / 120.0);
    ps = __fma_rn(ps, t2, -1.0 / 6.0);
    s = __fma_rn(__dmul_rn(t, t2), ps, t);
    double pc = 1.0 / 2432902008176640000.0;
    pc = __fma_rn(pc, t2, -1.0 / 6402373705728000.0);
    pc = __fma_rn(pc, t2, 1.0 / 20922789888000.0);
    pc = __fma_rn(pc, t2, -1.0 / 87178291200.0);
    pc = __fma_rn(pc, t2, 1.0 / 479001600.0);
    pc = __fma_rn(pc, t2, -1.0 / 3628800.0);
    pc = __fma_rn(pc, t2, 1.0 / 40320.0);
    pc = __fma_rn(pc, t2, -1.0 / 720.0);
    pc = __fma_rn(pc, t2, 1.0 / 24.0);
    pc = __fma_rn(pc, t2, -0.5);
    c = __fma_rn(t2, pc, 1.0);
}

__device__ __forceinline__ void quadrant(double q, double s, double c, double &so, double &co) {
    double qm = fmod(q, 4.0);
    if (qm < 0.0) qm = __dadd_rn(qm, 4.0);
    const int k = (int)qm;
    if (k == 0) { so = s; co = c; }
    else if (k == 1) { so = c; co = -s; }
    else if (k == 2) { so = -s; co = -c; }
    else { so = -c; co = s; }
}

// angle in degrees
__device__ __forceinline__ void sincos_deg64(double x, double &s, double &c) {
    const double q = rint(__ddiv_rn(x, 90.0));
    const double y = __dadd_rn(x, -__dmul_rn(q, 90.0));
    const double t = __dmul_rn(y, SMART_PI / 180.0);
    double ss, cc;
    series_sincos(t, ss, cc);
    quadrant(q, ss, cc, s, c);
}

// angle in quarter turns (angle = f * pi / 2)
__device__ __forceinline__ void sincos_quarter64(double f, double &s, double &c) {
    const double q = rint(f);
    const double y = __dadd_rn(f, -q);
    const double t = __dmul_rn(y, SMART_PI / 2.0);
    double ss, cc;
    series_sincos(t, ss, cc);
    quadrant(q, ss, cc, s, c);
}

// ---------------------------------------------------------------------------
// HEALPix RING scheme (Gorski et al. 2005).  Rings i = 1 .. 4N-1 from the
// north pole.  Polar rings i < N hold 4i pixels at z = 1 - i^2/(3N^2),
// azimuth (j + 1/2) * (pi/2)/i; equatorial rings N <= i <= 3N hold 4N pixels
// at z = (4N - 2i)/(3N), azimuth (j + 1/2 or j) * (pi/2)/N (half-pixel
// shift when i - N is even); southern rings mirror the northern ones.
// ---------------------------------------------------------------------------
struct RingPix {
    int ring;      // 1 .. 4N-1
    int j;         // index within the ring
};

__device__ __forceinline__ int64_t isqrt64(int64_t v) {
    int64_t r = (int64_t)__dsqrt_rn((double)v);
    while (r * r > v) --r;
    while ((r + 1) * (r + 1) <= v) ++r;
    return r;
}

__host__ __device__ __forceinline__ int64_t npix_of(int64_t N) { return 12 * N * N; }

__device__ __forceinline__ RingPix pix_to_ring(int64_t N, int64_t pix) {
    const int64_t ncap = 2 * N * (N - 1);
    const int64_t npix = 12 * N * N;
    RingPix r;
    if (pix < ncap) {
        const int64_t i = (1 + isqrt64(1 + 2 * pix)) >> 1;
        r.ring = (int)i;
        r.j = (int)(pix - 2 * i * (i - 1));
    } else if (pix < npix - ncap) {
        // nside is a power of two: the division by the ring length 4N is a shift
        const int64_t ip = pix - ncap;
        const int l = __ffsll((long long)N) + 1;      // log2(4N)
        r.ring = (int)((ip >> l) + N);
        r.j = (int)(ip & ((4 * N) - 1));
    } else {
        const int64_t ip = npix - pix;
        const int64_t is = (1 + isqrt64(2 * ip - 1)) >> 1;
        r.ring = (int)(4 * N - is);
        r.j = (int)(pix - (npix - 2 * is * (is + 1)));
    }
    return r;
}

struct RingGeom {
    int64_t start;  // first pixel
    int nr;         // pixels in the ring
    int shifted;    // 1: azimuth offset of half a pixel
    double z, rho;  // cos and sin of the colatitude
};

// z and rho from the ring index: exact integer forms, one rounding each
__device__ __forceinline__ RingGeom ring_geom(int64_t N, int64_t i) {
    RingGeom g;
    const int64_t npix = 12 * N * N;
    const double d3n2 = (double)(3 * N * N);
    if (i < N) {
        g.start = 2 * i * (i - 1);
        g.nr = (int)(4 * i);
        g.shifted = 1;
        g.z = __dadd_rn(1.0, -__ddiv_rn((double)(i * i), d3n2));
        g.rho = __ddiv_rn(__dmul_rn((double)i, __dsqrt_rn((double)(6 * N * N - i * i))), d3n2);
    } else if (i <= 3 * N) {
        g.start = 2 * N * (N - 1) + (i - N) * 4 * N;
        g.nr = (int)(4 * N);
        g.shifted = ((i - N) & 1) == 0;
        g.z = __ddiv_rn((double)(4 * N - 2 * i), (double)(3 * N));
        g.rho = __ddiv_rn(__dsqrt_rn((double)((2 * i - N) * (7 * N - 2 * i))), (double)(3 * N));
    } else {
        const int64_t is = 4 * N - i;
        g.start = npix - 2 * is * (is + 1);
        g.nr = (int)(4 * is);
        g.shifted = 1;
        g.z = -__dadd_rn(1.0, -__ddiv_rn((double)(is * is), d3n2));
        g.rho = __ddiv_rn(__dmul_rn((double)is, __dsqrt_rn((double)(6 * N * N - is * is))), d3n2);
    }
    return g;
}

// azimuth of pixel j of a ring, in quarter turns
__device__ __forceinline__ double ring_phi_quarter(int64_t N, int64_t i, int64_t j) {
    if (i < N) return __ddiv_rn((double)(2 * j + 1), (double)(2 * i));
    if (i <= 3 * N) {
        if (((i - N) & 1) == 0) return __ddiv_rn((double)(2 * j + 1), (double)(2 * N));
        return __ddiv_rn((double)j, (double)N);
    }
    const int64_t is = 4 * N - i;
    return __ddiv_rn((double)(2 * j + 1), (double)(2 * is));
}

__device__ __forceinline__ void pix2vec64(int64_t N, int64_t pix, double &x, double &y, double &z) {
    const RingPix rp = pix_to_ring(N, pix);
    const RingGeom g = ring_geom(N, rp.ring);
    double s, c;
    sincos_quarter64(ring_phi_quarter(N, rp.ring, rp.j), s, c);
    x = __dmul_rn(g.rho, c);
    y = __dmul_rn(g.rho, s);
    z = g.z;
}

__device__ __forceinline__ void radec2vec64(double ra, double dec, double &x, double &y, double &z) {
    double sa, ca, sd, cd;
    sincos_deg64(ra, sa, ca);
    sincos_deg64(dec, sd, cd);
    x = __dmul_rn(cd, ca);
    y = __dmul_rn(cd, sa);
    z = sd;
}

// RING pixel of (ra, dec) in degrees
__device__ __forceinline__ int64_t ang2pix64(int64_t N, double ra, double dec) {
    const int64_t npix = 12 * N * N;
    const int64_t ncap = 2 * N * (N - 1);
    double sd, cd;
    sincos_deg64(dec, sd, cd);
    const double z = sd, sth = cd;
    double a = fmod(ra, 360.0);
    if (a < 0.0) a = __dadd_rn(a, 360.0);
    double tt = __ddiv_rn(a, 90.0);
    if (tt >= 4.0) tt = __dadd_rn(tt, -4.0);
    const double za = fabs(z);
    const double dN = (double)N;
    if (za <= 2.0 / 3.0) {
        const double t1 = __dmul_rn(dN, __dadd_rn(0.5, tt));
        const double t2 = __dmul_rn(__dmul_rn(dN, z), 0.75);
        const int64_t jp = (int64_t)floor(__dadd_rn(t1, -t2));
        const int64_t jm = (int64_t)floor(__dadd_rn(t1, t2));
        const int64_t ir = N + 1 + jp - jm;
        const int64_t kshift = 1 - (ir & 1);
        int64_t ip = (jp + jm - N + kshift + 1) / 2;
        ip = ((ip % (4 * N)) + 4 * N) % (4 * N);
        return ncap + (ir - 1) * 4 * N + ip;
    } else {
        const double tp = __dadd_rn(tt, -floor(tt));
        const double tmp = __dmul_rn(__dmul_rn(dN, sth), __dsqrt_rn(__ddiv_rn(3.0, __dadd_rn(1.0, za))));
        const int64_t jp = (int64_t)floor(__dmul_rn(tp, tmp));
        const int64_t jm = (int64_t)floor(__dmul_rn(__dadd_rn(1.0, -tp), tmp));
        const int64_t ir = jp + jm + 1;
        int64_t ip = (int64_t)floor(__dmul_rn(tt, (double)ir));
        ip = ((ip % (4 * ir)) + 4 * ir) % (4 * ir);
        if (z > 0.0) return 2 * ir * (ir - 1) + ip;
        return npix - 2 * ir * (ir + 1) + ip;
    }
}

// exact membership as in the float64 definition: chord^2 from unit vectors,
// summed in the order (dx^2 + dy^2) + dz^2 with no contraction
__device__ __forceinline__ bool member64(double x0, double y0, double z0,
                                        double x1, double y1, double z1, double T) {
    const double dx = __dadd_rn(x1, -x0);
    const double dy = __dadd_rn(y1, -y0);
    const double dz = __dadd_rn(z1, -z0);
    const double s2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return s2 <= T;
}

// ---------------------------------------------------------------------------
// Ring-pair table.  For every output ring i0 and every bin ring i whose
// colatitude is within theta_disc of i0's, the constants that make the
// per-pair geometry a few float32 operations (see aperture.cu):
//   s^2 = A + B h,  y = C + D h,  x = -rho0 sin u,  h = sin^2(u/2),
// with u the azimuth difference and (x, y) the direction from the point to
// the centre in the point's (East, North) tangent basis.
// ---------------------------------------------------------------------------
struct __align__(16) RingPair {
    int start;      // first pixel of the bin ring
    int nr;         // pixels in the bin ring
    int flags;      // bit0: shifted bin ring, bit1: wide (slow trig), bit2: whole ring
    int ring;       // bin ring index
    float A, B, C, D;
    float dphi;     // 2 pi / nr (rad per bin pixel)
    float hw;       // half window in bin pixels (margin included)
    float mrho0;    // -rho0
    float dlat;     // latitude(i0) - latitude(i), rad (galaxy offsets are relative to it)
    float rho0, z0; // output ring constants (float32)
    float hw_in;    // half window of certain members: |offset| <= hw_in gives
                    // s^2 <= T_disc (1 - 1e-5) (negative: none)
    float pad1;
};
static_assert(sizeof(RingPair) == 64, "RingPair layout");

enum { RP_SHIFTED = 1, RP_WIDE = 2, RP_WHOLE = 4 };

// bits of the device status word read back by smart_sync
enum { SMART_STATUS_BAND_OVERFLOW = 1, SMART_STATUS_INVALID_COORDS = 2, SMART_STATUS_BAD_RUNS = 4 };

// Per ring pair of the pixel-mode table: where its per-offset geometry sits
// in the Toeplitz pool (off = -1: not a Toeplitz pair), the candidate
// offsets [dlo, dlo + ncand), the run [da, da + L) of certain members
// (relative to dlo) and up to three offsets inside the float32 guard band.
struct ToeInfo {
    int off, dlo, da, L, namb, amb0, amb1, amb2;
};

}  // namespace smart

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
struct smart_ctx {
    int nside_out = 0, nside_bin = 0;
    int filter_kind = 0;
    double xc = 0.15;
    double theta_ap = 0;       // rad
    double T = 0;              // 4 sin^2(theta_ap/2)
    double area = 0;           // 2 pi (1 - cos theta_ap)
    cudaStream_t stream = nullptr;
    std::string err;
    double wait_limit_s = 600.0;     // deadline of the waits inside set-up calls
    int64_t *host_rb = nullptr;      // pinned host slots for the set-up calls' read-backs (16)
    std::unordered_set<void *> async_bufs;   // buffers from the stream-ordered allocator

    // targets
    int64_t *targets = nullptr;
    int64_t n_targets = 0, cap_targets = 0;

    // ring-pair tables (pixel mode: theta_ap; brute force: theta_ap + pixel radius)
    smart::RingPair *rp_pix = nullptr;
    smart::RingPair *rp_gal = nullptr;
    int *rp_pix_cnt = nullptr, *rp_gal_cnt = nullptr;
    int kmax_pix = 0, kmax_gal = 0;

    // binned maps, one float4 (G1, G2, S2, W) per pixel plus an int32 count:
    // owned (smart_bin_galaxies, smart_set_binned) or borrowed (smart_set_binned_packed)
    const float4 *PX = nullptr;
    const int32_t *NP = nullptr;
    float4 *own_px = nullptr;        // npix
    int32_t *own_np = nullptr;       // npix + 1
    bool have_binned = false;
    bool binned_from_catalog = false;   // the catalogue offsets are then the count prefix
    bool binned_from_runs = false;      // own map written by smart_set_binned_runs (zero outside the runs)

    // sorted catalogue
    int64_t n_gal = 0, cap_gal = 0;
    bool have_catalog = false;
    uint32_t *keys = nullptr, *keys_alt = nullptr;   // pixel per galaxy
    uint32_t *vals = nullptr, *vals_alt = nullptr;   // input index
    int32_t *offsets = nullptr;                      // npix_bin + 1
    float4 *rec_geo = nullptr;                       // (ddec, dphi, z, rho)
    float4 *rec_shear = nullptr;                     // (w e1, w e2, w, w^2 |e|^2)
    double2 *rec_radec = nullptr;                    // (ra, dec) degrees, for exact re-decisions
    uint32_t *hist = nullptr;
    int64_t cap_hist = 0;
    int32_t *hist_scan = nullptr;
    int64_t cap_hist_scan = 0;
    double *ring_lat = nullptr;                      // latitude (deg) of each bin ring
    int *d_invalid = nullptr;
    int64_t *scan_tmp = nullptr;
    int64_t cap_scan = 0;

    // pixel-mode launch state
    int64_t *tiles = nullptr;                        // first target of each tile (+ end)
    int64_t cap_tiles = 0, n_tiles = 0;
    int32_t *tile_flag = nullptr;
    int64_t cap_tile_flag = 0;
    float4 *qtab = nullptr;                          // filter table (Schirmer)
    int32_t *np_prefix = nullptr;                    // prefix of per-pixel counts (smart_set_binned input)
    int64_t cap_np_prefix = 0;
    int *d_work = nullptr;                           // tile counter of persistent launches
    smart::ToeInfo *toe_info = nullptr;              // Toeplitz tables of the pixel-mode ring pairs
    float4 *toe_geo = nullptr;
    int toe_max_run = 0;                             // longest Toeplitz candidate run of the tables
    unsigned char *toe_ring = nullptr;               // per output ring: all ring pairs Toeplitz
    int32_t *gen_list = nullptr;                     // targets handled by the general kernel
    int64_t cap_gen_list = 0, n_gen = 0;
    int2 *gen_work = nullptr;                        // its work: mirror pairs (target, image), then singles (target, -1)
    int64_t cap_gen_work = 0, n_work = 0, n_work_pairs = 0;
    int64_t targets_version = 0, gen_version = -1;
    int64_t *gal_tiles = nullptr;                    // brute force: groups of up to 4 targets
    int64_t cap_gal_tiles = 0, n_gal_tiles = 0, gal_tiles_version = -1;
    double *raw = nullptr;                           // brute force raw sums + counts
    int64_t cap_raw = 0;
    void *band = nullptr;                            // guard-band pairs awaiting float64 decisions
    int64_t cap_band = 0;
    unsigned long long *d_band_count = nullptr;
    int *d_status = nullptr;                         // device status word
    int num_sms = 148;

    // barycentre form of the pixel map (Sect. 3.3): one record per bin pixel
    // holding galaxies, in the layout of the galaxy records
    int64_t catalog_version = 0, bary_version = -1;
    int32_t *bary_off = nullptr;                     // npix + 1: record of each pixel (prefix of n_p > 0)
    int64_t cap_bary_off = 0;
    float4 *bary_geo = nullptr, *bary_sh = nullptr;
    uint32_t *bary_keys = nullptr;
    int32_t *bary_cnt = nullptr;                     // galaxies of the record's pixel
    double *bary_vec = nullptr;                      // float64 unit vector, 3 per record
    int64_t n_bary = 0, cap_bary = 0;
    int norm = SMART_NORM_SUMMED;                    // normalisation of the maps (Sect. 2.4)
    float4 *avg_buf = nullptr;                       // inputs scaled for the averaged form
    int64_t cap_avg = 0;
    double *bary_wr = nullptr;                       // w r of every galaxy (build scratch)
    int64_t cap_bary_wr = 0;
    int32_t *raw_m = nullptr;                        // member records per target
    int64_t cap_raw_m = 0;
    void *gen_band = nullptr;                        // general kernel: guard-band slots
    int64_t cap_gen_band = 0;
    unsigned long long *d_gen_count = nullptr;       // general kernel: slots claimed
    int64_t cap_gen_count = 0;
    int64_t band_slot_limit = 0;                     // > 0: cap on those slots (testing aid)

    // Cartesian (projected) estimator (Sect. 2.2, Sect. 5.2.1): the plane of
    // the last projection, plane records of the sorted galaxies and targets
    double *proj_plane = nullptr;                    // 9 doubles: c, e_c, n_c
    float4 *proj_xy = nullptr, *proj_sh = nullptr;   // per galaxy: (x hi, y hi, x lo, y lo), rotated shear
    int64_t cap_proj = 0, cap_proj_sh = 0;
    float4 *proj_txy = nullptr;                      // per target: (x hi, y hi, x lo, y lo); NaN: no image
    int64_t cap_proj_t = 0;
    float4 *qtab_plane = nullptr;                    // filter table on the plane distance (tabulated filters)
    double *annulus_buf = nullptr;                   // annulus sums
    int64_t cap_annulus = 0;

    // diagnostics
    unsigned long long *d_fp64_count = nullptr;
    bool timing = false;                             // record events around each kernel launch
    std::vector<cudaEvent_t> ev_pool;                // created on demand, reused after a reset
    size_t ev_used = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> tlog[SMART_KT_COUNT];
};

namespace smart {

smart_status fail(smart_ctx *ctx, smart_status st, const std::string &msg);
smart_status check_cuda(smart_ctx *ctx, cudaError_t e, const char *what);
smart_status ensure_alloc(smart_ctx *ctx, void **p, int64_t &cap, int64_t need, size_t elem, const char *what);
// wait for the context stream, polling, at most ctx->wait_limit_s seconds
// (SMART_E_TIMEOUT after that); used by the set-up calls only
smart_status wait_stream(smart_ctx *ctx, const char *what);

// geometry.cu
smart_status build_ring_pairs(smart_ctx *ctx, double theta_disc, RingPair **out, int **cnt, int *kmax);
double max_pixrad(int nside);

// binning.cu
// out[0..n_out) = exclusive prefix sums of in[0..n_in), inputs past n_in read as 0
smart_status exclusive_scan_i32(smart_ctx *ctx, const int32_t *in, int32_t *out, int64_t n_in, int64_t n_out);

// aperture_pixel.cu
smart_status build_tiles(smart_ctx *ctx);
struct MapArgs;
smart_status prepare_pixel(smart_ctx *c, const smart_maps *out, MapArgs &a);
smart_status launch_count_prefix(smart_ctx *c);
// filter table on the chord (spherical maps) or on the plane distance
// (projected map) of the tabulated filters; no-op for the polynomial filter
smart_status build_filter_table(smart_ctx *c, bool plane, float4 **tab);
smart_status build_tiles_log2(smart_ctx *ctx, int log2_slots, int64_t **tiles, int64_t *cap, int64_t *n_tiles);
// every table the maps need for the current targets (pixel mode and brute
// force), built in smart_set_targets so that the map calls never wait
smart_status prepare_tables(smart_ctx *c);
constexpr int GAL_GROUP_LOG2 = 2;    // brute force and projected: groups of 4 targets per warp

// context.cu
smart_status ensure_own_binned_map(smart_ctx *ctx);

// normalise.cu (averaged normalisation): scaled inputs in ctx->avg_buf, and
// the rescale of the summed-form outputs
smart_status averaged_pixel_input(smart_ctx *c, const float4 *px, const float4 **out);
smart_status averaged_record_input(smart_ctx *c, const float4 *sh, const uint32_t *keys, const float4 *px, int64_t n,
                                   const float4 **out);
smart_status averaged_rescale(smart_ctx *c, const smart_maps *out);

// Brackets one kernel launch with events on the context stream while timing
// is enabled (smart_timing_enable); does nothing otherwise.
class KernelTimer {
  public:
    KernelTimer(smart_ctx *c, int id);
    ~KernelTimer();
  private:
    smart_ctx *c_;
    int id_;
    cudaEvent_t start_ = nullptr;
};

}  // namespace smart
