// aperture_common.cuh -- shared pieces of the aperture-mass kernels.
//
// Per pair (target centre r0, point p) the geometry is reduced to float32
// operations on constants of the ring pair (output ring of r0, bin ring of
// p), computed once in float64 (geometry.cu):
//   u   = azimuth of p - azimuth of r0       (from exact integer lattice offsets)
//   h   = sin^2(u/2)
//   s^2 = A + B h                            chord^2 between r0 and p
//   x   = -rho0 sin u,  y = C + D h          direction p -> r0 in p's (East, North) basis
//   x^2 + y^2 = sin^2 d,  cos 2psi = (y^2 - x^2)/sin^2 d,  sin 2psi = -2xy/sin^2 d
// (the paper's tan psi of Sect. 2.3 equals -x/y; no atan2 is needed).
// Membership s^2 <= T is decided in float32 outside a guard band of relative
// width 4e-6 around T, and inside it by the float64 definition (unit
// vectors from the same series sine/cosine as the float64 reference), so
// member sets and counts are exact.
#pragma once

#include "smart_internal.cuh"

namespace smart {

constexpr int QTAB_BINS = 1024;      // filter table: cubic pieces on the chord s / s_ap in [0, 1]

struct FilterArgs {
    float inv_ap;      // 1 / theta_ap
    float inv_ap2;     // 1 / theta_ap^2
    float qnorm;       // poly: 6 / (pi theta_ap^2)
    float tab_scale;   // QTAB_BINS / sqrt(T): chord -> table coordinate
    const float4 *qtab;  // QTAB_BINS cubic pieces of Q as a function of the chord (table filters)
};

struct MapArgs {
    const int64_t *targets;
    int64_t n;
    int64_t N0, N1;
    const RingPair *table;
    const int *counts;
    int kmax;
    float Tlo, Thi;          // guard band around T (float32)
    double T, area;
    FilterArgs f;
    // pixel-mode inputs: (G1, G2, S2, W) per pixel and the galaxy count
    const float4 *PX;
    const int32_t *NP;
    const int32_t *NPRE;     // exclusive prefix of NP over RING order (npix + 1)
    // tiles of targets (pixel mode): first target of each tile, n_tiles + 1 entries
    const int64_t *tiles;
    int64_t n_tiles;
    const ToeInfo *toe;      // Toeplitz info per ring pair (pixel mode)
    const float4 *toe_geo;   // per-offset (a, b, -b, c) of the Toeplitz ring pairs
    const unsigned char *toe_ring;  // 1: every ring pair of this output ring is Toeplitz
    const int32_t *gen_list;        // targets of the other rings (general kernel)
    int64_t n_gen;
    const int2 *gen_work;           // general kernel's work: n_pairs (target, mirror image), then (target, -1)
    int64_t n_work, n_pairs;
    int *work;               // tile counter of the persistent launch
    // brute-force inputs
    const int32_t *offsets;
    const float4 *geo, *shear;
    const double2 *radec;
    const uint32_t *keys;    // pixel of each sorted galaxy
    double *raw;             // brute force: per target raw sums (SE, SB, SV, SW), float64
    int32_t *raw_n;          // per target member count
    void *band;              // guard-band pair list
    int64_t band_cap;
    unsigned long long *band_count;
    // outputs
    double *sum_w;
    float *map_e, *map_b, *var;
    int64_t *count;
    int32_t *members;
    unsigned long long *fp64_count;
    int *status;             // device status word (SMART_STATUS_* bits)
    float pixrad;            // largest angular radius of a bin pixel (rad)
};

// great-circle separation^2 from the chord^2: d^2 = sum_n 2 s^(2n) / (n^2 C(2n,n))
__device__ __forceinline__ float sep2_from_chord2(float s2) {
    if (s2 > 0.05f) {
        const float d = 2.0f * asinf(0.5f * sqrtf(s2));
        return d * d;
    }
    return s2 * fmaf(s2, fmaf(s2, fmaf(s2, fmaf(s2, 1.0f / 3150.0f, 1.0f / 560.0f), 1.0f / 90.0f), 1.0f / 12.0f), 1.0f);
}

// square root to within a couple of ulps (the hardware approximation; exact
// for 0): a table coordinate, not a result
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Q from the cubic table, indexed by the chord s = sqrt(s2) (uniform bins of
// s / s_ap; Q is smooth in s because the separation d(s) is)
__device__ __forceinline__ float qtab_eval(const float4 *tab, float s2, float scale) {
    const float f = sqrt_approx(s2) * scale;
    const int i = min((int)f, QTAB_BINS - 1);
    const float t = f - (float)i;
    const float4 c = tab[i];
    return fmaf(fmaf(fmaf(c.w, t, c.z), t, c.y), t, c.x);
}

// the same for a member pair (s2 below T, so the index stays below
// QTAB_BINS: no clamp)
__device__ __forceinline__ float qtab_eval_member(const float4 *tab, float s2, float scale) {
    const float f = sqrt_approx(s2) * scale;
    const int i = (int)f;
    const float t = f - (float)i;
    const float4 c = tab[i];
    return fmaf(fmaf(fmaf(c.w, t, c.z), t, c.y), t, c.x);
}

// Q(d) from the chord^2.  Polynomial filter in closed form; the tabulated
// filters (Schirmer, Jarvis) through their cubic table (tab: a shared-memory
// or global copy).  KIND == SMART_FILTER_SCHIRMER stands for every tabulated
// filter: the table, not the template, carries the filter.
template <int KIND>
__device__ __forceinline__ float filter_Q(const FilterArgs &f, const float4 *tab, float s2) {
    if (KIND == SMART_FILTER_POLY) {
        const float X2 = sep2_from_chord2(s2) * f.inv_ap2;
        return f.qnorm * X2 * (1.0f - X2);
    } else {
        return qtab_eval(tab, s2, f.tab_scale);
    }
}

// sin u and sin^2(u/2): 2-term series for |u| <= 0.05 (relative truncation
// below 6e-8, under float32 rounding), 4-term for |u| <= 0.45 (below 5e-9),
// longer series beyond
__device__ __forceinline__ void sin_hav_narrow(float u, float &sinu, float &h) {
    const float u2 = u * u;
    sinu = u * fmaf(u2, -1.0f / 6.0f, 1.0f);
    h = u2 * fmaf(u2, -1.0f / 48.0f, 0.25f);
}

__device__ __forceinline__ void sin_hav_small(float u, float &sinu, float &h) {
    const float u2 = u * u;
    sinu = u * fmaf(u2, fmaf(u2, fmaf(u2, -1.0f / 5040.0f, 1.0f / 120.0f), -1.0f / 6.0f), 1.0f);
    h = u2 * fmaf(u2, fmaf(u2, fmaf(u2, -1.0f / 80640.0f, 1.0f / 1440.0f), -1.0f / 48.0f), 0.25f);
}

// |u| <= pi: sine and cosine of v = u/2 in [-pi/2, pi/2] from their
// Maclaurin series (to v^15 and v^16; truncation below 1e-10)
__device__ __forceinline__ void sin_hav_wide(float u, float &sinu, float &h) {
    const float v = 0.5f * u, v2 = v * v;
    float ps = fmaf(v2, -1.0f / 1307674368000.0f, 1.0f / 6227020800.0f);
    ps = fmaf(v2, ps, -1.0f / 39916800.0f);
    ps = fmaf(v2, ps, 1.0f / 362880.0f);
    ps = fmaf(v2, ps, -1.0f / 5040.0f);
    ps = fmaf(v2, ps, 1.0f / 120.0f);
    ps = fmaf(v2, ps, -1.0f / 6.0f);
    const float sh = fmaf(v * v2, ps, v);
    float pc = fmaf(v2, 1.0f / 20922789888000.0f, -1.0f / 87178291200.0f);
    pc = fmaf(v2, pc, 1.0f / 479001600.0f);
    pc = fmaf(v2, pc, -1.0f / 3628800.0f);
    pc = fmaf(v2, pc, 1.0f / 40320.0f);
    pc = fmaf(v2, pc, -1.0f / 720.0f);
    pc = fmaf(v2, pc, 1.0f / 24.0f);
    pc = fmaf(v2, pc, -0.5f);
    const float ch = fmaf(v2, pc, 1.0f);
    sinu = 2.0f * sh * ch;
    h = sh * sh;
}

__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

struct TargetRing {
    int i0, j0, q0, s0, nr0;
};

__device__ __forceinline__ TargetRing target_ring(int64_t N0, int64_t pix) {
    const RingPix rp = pix_to_ring(N0, pix);
    TargetRing t;
    t.i0 = rp.ring;
    t.j0 = rp.j;
    if (rp.ring < N0) {
        t.q0 = rp.ring;
        t.s0 = 1;
    } else if (rp.ring <= 3 * N0) {
        t.q0 = (int)N0;
        t.s0 = ((rp.ring - N0) & 1) == 0 ? 1 : 0;
    } else {
        t.q0 = (int)(4 * N0 - rp.ring);
        t.s0 = 1;
    }
    t.nr0 = 4 * t.q0;
    return t;
}

// target position on the bin ring's azimuth lattice: X = (2 j0 + s0) q / (2 q0)
// split as Xi + Xf with Xi integer and 0 <= Xf < 1 (exact integer arithmetic)
__device__ __forceinline__ void lattice_position(const TargetRing &t, int q, int &Xi, float &Xf) {
    if (q == t.q0) {
        Xi = t.j0;
        Xf = 0.5f * (float)t.s0;
    } else {
        // num < 2^31 for nside <= 8192: (2 j0 + s0) <= 2^16, q <= 2^13
        const int num = (2 * t.j0 + t.s0) * q;
        const int den = 2 * t.q0;
        const int qi = num / den;
        Xi = qi;
        Xf = (float)(num - qi * den) / (float)den;
    }
}

// The same lattice position with the division by 2 q0 done by a
// multiply-high (set up once per target): m = floor((2^32 - 1) / den) + 1
// overestimates 1 / den by less than 2^-32, so for num < 2^31 the estimate
// is the quotient or one more, fixed by the sign of the remainder.
struct LatticeDiv {
    uint32_t den, m;
    float inv;
};

__device__ __forceinline__ LatticeDiv lattice_div(const TargetRing &t) {
    LatticeDiv d;
    d.den = 2u * (uint32_t)t.q0;
    d.m = (uint32_t)(0xFFFFFFFFull / d.den) + 1u;
    d.inv = 1.0f / (float)d.den;
    return d;
}

__device__ __forceinline__ void lattice_position(const TargetRing &t, const LatticeDiv &d, int q, int &Xi,
                                                 float &Xf) {
    if (q == t.q0) {
        Xi = t.j0;
        Xf = 0.5f * (float)t.s0;
        return;
    }
    const uint32_t num = (uint32_t)((2 * t.j0 + t.s0) * q);     // < 2^30 for nside <= 8192
    uint32_t qi = __umulhi(num, d.m);
    int rem = (int)(num - qi * d.den);
    if (rem < 0) {
        qi -= 1u;
        rem += (int)d.den;
    }
    Xi = (int)qi;
    Xf = (float)rem * d.inv;
}

__device__ __forceinline__ void window(const RingPair &R, float fr, int &kl, int &kh) {
    if (R.flags & RP_WHOLE) {
        kl = (int)floorf(-0.5f * (float)R.nr - fr) + 1;
        kh = kl + R.nr - 1;
    } else {
        kl = (int)ceilf(-fr - R.hw);
        kh = (int)floorf(-fr + R.hw);
    }
}

// summed normalisation (Sect. 2.4): nbar = SW / A, M = S / nbar,
// sigma^2 = SV / (2 nbar^2).  The compensated weight sum is carried to
// float64 (its reported value); the ratio A / SW is then applied in float32.
__device__ __forceinline__ void finalise(const MapArgs &a, int64_t t, float se, float cse, float sb, float csb,
                                         float sv, float csv, float sw, float csw, int64_t cnt, int nmem) {
    const double SW = (double)sw - (double)csw;
    float me = 0.f, mb = 0.f, vv = 0.f;
    if (SW > 0.0) {
        const float r = (float)a.area / (float)SW;       // 1 / nbar
        me = (se - cse) * r;
        mb = (sb - csb) * r;
        vv = 0.5f * (sv - csv) * r * r;
    }
    if (a.sum_w) a.sum_w[t] = SW;
    if (a.map_e) a.map_e[t] = me;
    if (a.map_b) a.map_b[t] = mb;
    if (a.var) a.var[t] = vv;
    if (a.count) a.count[t] = cnt;
    if (a.members) a.members[t] = nmem;
}

FilterArgs make_filter(const smart_ctx *c);
smart_status ensure_filter_table(smart_ctx *c);
smart_status common_args(smart_ctx *c, const smart_maps *out, MapArgs &a);

}  // namespace smart
