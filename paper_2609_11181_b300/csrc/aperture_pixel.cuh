// aperture_pixel.cuh -- device code of the pixel-based aperture mass
// (Sect. 3.2, summed normalisation of Sect. 2.4), shared by the single-map
// launches (aperture_pixel.cu) and the batched launch (aperture_batch.cu).
//
// Work unit: a tile = up to TS consecutive azimuth slots of one output ring
// (targets are RING-sorted, so a tile is a contiguous run of the target
// list).  For each bin ring that can reach the tile (the ring-pair table):
//
//  * Toeplitz path -- the bin ring has as many pixels as the output ring and
//    both grids have the same nside: every pair's geometry depends only on
//    the index offset delta = k - j0.  Geometry, filter and membership are
//    tabulated once per ring pair and offset; the CTA stages the bin-ring
//    segment it needs and each thread slides a window over RB consecutive
//    targets: 4 FMAs + 1 FMA (noise) + 1 add (weight) per pair.
//  * general path (polar rings, unequal rings, unequal nside): per pair
//    geometry from the ring-pair constants, the filter from a cubic table
//    (Schirmer) or in closed form (polynomial).  A target and its mirror
//    image about a meridian m pi/4 share that geometry (general_target2).
//
// Sums: float32 within one ring pair (Toeplitz: two ring pairs); across ring
// pairs float32 totals (Toeplitz, mirror pairs) or compensated (Kahan)
// totals (other general targets); the weight sum goes to float64 for the
// final normalisation.
#pragma once

#include "aperture_common.cuh"

namespace smart {


constexpr int TS = 256;           // azimuth slots per tile (aligned blocks of a ring)
constexpr int TS_LOG2 = 8;
constexpr int NT = 32;            // threads per CTA: one warp (its barriers are warp-wide)
constexpr int RB = 8;             // consecutive slots per thread
constexpr int NCAND = 120;        // longest Toeplitz candidate run kept in shared memory
constexpr int NCAND_SHORT = 64;   // contexts whose runs are all this short stage less
constexpr int GEN_PAIR_CTAS_PER_SM = 4;  // general kernel, mirror pairs: resident 128-thread CTAs per SM
// unpaired general targets that run in the mirror-pair launch (ahead of the
// pairs) instead of a launch of their own: all of them when they are at most
// a sixteenth of the pairs (a launch of their own would run after the pairs,
// a short tail with the GPU nearly idle), else none (their own launch keeps
// seven CTAs per SM)
inline int64_t gen_lead(int64_t n_pairs, int64_t n_single) {
    return n_pairs > 0 && 16 * n_single <= n_pairs ? n_single : 0;
}
static_assert(TS == NT * RB, "tile = threads x slots per thread");
static_assert(NCAND % 8 == 0 && NCAND_SHORT % 8 == 0, "staging layout works on rows of 8 pixels");
// Shared-memory staging of a tile for runs of up to NC offsets: the bin-ring
// segment (TS + NC + 8 pixels) and the geometry (NC entries), each double
// buffered.  Resident CTAs per SM: the registers (168 a thread) allow 12;
// the longer staging (19.2 KB a CTA) allows 11.
template <int NC>
constexpr int toe_segn() { return TS + NC + 8; }
template <int NC>
constexpr int toe_ctas_per_sm() { return NC <= NCAND_SHORT ? 12 : 11; }

// shared-memory position of staged pixel m: rows of eight 16-byte pixels
// (128 bytes, every bank once), the pixel's slot within its row XOR-ed with
// the row index.  Thread t reads pixels m = 8 t + d: the eight threads of a
// quarter warp then sit in eight consecutive rows, and the XOR puts their
// pixels in eight different 16-byte bank groups for every d.
__device__ __forceinline__ int tpos(int m) { return (m & ~7) | ((m ^ (m >> 3)) & 7); }

// the float64 membership decision for a pair inside the guard band
static __device__ __noinline__ bool exact_member_pix(int64_t N0, int64_t N1, double T, unsigned long long *counter,
                                              int64_t target_pix, int64_t bin_pix) {
    double x0, y0, z0, x1, y1, z1;
    pix2vec64(N0, target_pix, x0, y0, z0);
    pix2vec64(N1, bin_pix, x1, y1, z1);
    atomicAdd(counter, 1ull);
    return member64(x0, y0, z0, x1, y1, z1, T);
}

__device__ __forceinline__ bool exact_member(const MapArgs &a, int64_t target_pix, int64_t bin_pix) {
    return exact_member_pix(a.N0, a.N1, a.T, a.fp64_count, target_pix, bin_pix);
}

template <int MODE>
__device__ __forceinline__ void sin_hav(float u, float &sinu, float &h) {
    if (MODE == 0) sin_hav_narrow(u, sinu, h);
    else if (MODE == 1) sin_hav_small(u, sinu, h);
    else sin_hav_wide(u, sinu, h);
}

// one member pair's contribution (pixel mode)
template <int KIND, int MODE>
__device__ __forceinline__ void pixel_pair(const MapArgs &a, const RingPair &R, const float4 *qtab, float u, int p,
                                           float &pe, float &pb, float &pv, float &pw, int &nn, int &nm) {
    float sinu, h;
    sin_hav<MODE>(u, sinu, h);
    const float s2 = fmaf(R.B, h, R.A);
    const float x = R.mrho0 * sinu;
    const float y = fmaf(R.D, h, R.C);
    const float xx = x * x;
    const float sd2 = fmaf(y, y, xx);
    const float cc = fmaf(y, y, -xx);
    const float ss = -2.0f * x * y;
    const float Q = filter_Q<KIND>(a.f, qtab, s2);
    const float w = sd2 > 1e-30f ? __fdividef(Q, sd2) : 0.f;
    const float4 g = __ldg(a.PX + p);
    pe = fmaf(w, fmaf(g.x, cc, g.y * ss), pe);
    pb = fmaf(w, fmaf(g.y, cc, -g.x * ss), pb);
    pv = fmaf(Q * Q, g.z, pv);
    pw += g.w;
    nn += __ldg(a.NP + p);
    nm += 1;
}

// bin-ring index of the mirror image of bin pixel kk (0 <= kk < nr) about
// the meridian m pi/4: (m q - s - kk) mod nr for a ring of nr = 4 q pixels
// centred at azimuths (k + s/2) 2 pi / nr; cm = m q - s lies in [-1, 3 q]
__device__ __forceinline__ int mirror_index(const RingPair &R, int cm, int kk) {
    const int v = cm - kk;
    return v < 0 ? v + R.nr : v;
}

// the guard-band pairs of one target and one ring pair, decided in float64
// (window, u and s^2 exactly as in general_segment).  mline < 0: the pairs
// of target pix itself (tr is its ring).  mline = m >= 0: pix is the mirror
// image about the meridian m pi/4 of the target whose ring position tr
// holds; the window, u and s^2 are that target's, the bin pixels their
// mirror images and the azimuth offsets -u (as in general_segment2).
template <int KIND, int MODE>
__device__ __forceinline__ void band_pairs(const MapArgs &a, const RingPair &R, const TargetRing &tr,
                                           const LatticeDiv &ld, int64_t pix, int mline, const float4 *qtab,
                                           float &pe, float &pb, float &pv, float &pw, int &nn, int &nm) {
    const int q = R.nr >> 2;
    int Xi;
    float Xf;
    lattice_position(tr, ld, q, Xi, Xf);
    const int sh = (R.flags & RP_SHIFTED) ? 1 : 0;
    const float fr = (sh ? 0.5f : 0.0f) - Xf;
    const int cm = mline * q - sh;
    int kl, kh;
    window(R, fr, kl, kh);
    int kk = Xi + kl;
    kk += kk < 0 ? R.nr : (kk >= R.nr ? -R.nr : 0);
    const float u0 = fr * R.dphi;
    float kf = (float)kl;
    for (int k = kl; k <= kh; ++k) {
        const float u = fmaf(kf, R.dphi, u0);
        kf += 1.0f;
        float sinu, h;
        sin_hav<MODE>(u, sinu, h);
        const float s2 = fmaf(R.B, h, R.A);
        const int p = R.start + (mline < 0 ? kk : mirror_index(R, cm, kk));
        kk = (kk + 1 == R.nr) ? 0 : kk + 1;
        if (s2 >= a.Tlo && s2 <= a.Thi && exact_member(a, pix, p))
            pixel_pair<KIND, MODE>(a, R, qtab, mline < 0 ? u : -u, p, pe, pb, pv, pw, nn, nm);
    }
}

// position in the bin ring of lattice offset k (0 <= Xi < nr, -nr < k < nr)
__device__ __forceinline__ int wrap_start(const RingPair &R, int Xi, int k) {
    int kk = Xi + k;
    kk += kk < 0 ? R.nr : (kk >= R.nr ? -R.nr : 0);
    return kk;
}

// One member pair of the general path: bin pixel data g at lattice offset
// kf.  u from the offset each time (not by repeated addition): the
// target's own pixel must get u = 0 exactly, so that it carries no shear.
// Tabulated filters: the table index needs no clamp (a member's chord is
// below the aperture's).  Polynomial filter: Q / sin^2 d without a
// division, t + Q (1/3 + d^2/15 + 2 d^4/189) with t = qnorm/theta^2 (1 -
// d^2/theta^2) and Q = d^2 t (the next term, d^8/675 relative, stays below
// 1e-8 for d^2 up to 0.05, and below 1e-5 for apertures up to 30 degrees).
template <int KIND, int MODE>
__device__ __forceinline__ void member_pair(const MapArgs &a, const RingPair &R, const float4 *qtab, float u0,
                                            float kf, const float4 &g, float &pe, float &pb, float &pv, float &pw) {
    const float u = fmaf(kf, R.dphi, u0);
    float sinu, h;
    sin_hav<MODE>(u, sinu, h);
    const float s2 = fmaf(R.B, h, R.A);
    const float x = R.mrho0 * sinu;
    const float y = fmaf(R.D, h, R.C);
    const float xx = x * x;
    const float cc = fmaf(y, y, -xx);
    const float ss = -2.0f * x * y;
    float Q, w;
    if (KIND == SMART_FILTER_POLY) {
        const float d2 = sep2_from_chord2(s2);
        const float qn1 = a.f.qnorm * a.f.inv_ap2;
        const float t = fmaf(d2, -qn1 * a.f.inv_ap2, qn1);
        Q = d2 * t;
        w = fmaf(Q, fmaf(d2, fmaf(d2, 2.0f / 189.0f, 1.0f / 15.0f), 1.0f / 3.0f), t);
    } else {
        Q = qtab_eval_member(qtab, s2, a.f.tab_scale);
        // sin^2 d = 0 only at the target's own centre, where cc = ss = 0
        // exactly; elsewhere it is at least a squared bin spacing, far above
        // the offset, which only keeps w finite there
        w = __fdividef(Q, fmaf(y, y, xx) + 1e-30f);
    }
    pe = fmaf(w, fmaf(g.x, cc, g.y * ss), pe);
    pb = fmaf(w, fmaf(g.y, cc, -g.x * ss), pb);
    pv = fmaf(Q * Q, g.z, pv);
    pw += g.w;
}

// The certain members of one ring pair that do not cross the bin ring's
// seam: bin pixels pbeg .. pbeg + cnt - 1 (cnt >= 1) at lattice offsets kf,
// kf + 1, ...  No test, no select: every pair is a member.  The bin pixel's
// data is loaded one iteration ahead; the last pair is peeled off the loop
// so that no load passes the run.
template <int KIND, int MODE>
__device__ __forceinline__ void certain_run(const MapArgs &a, const RingPair &R, const float4 *qtab, float u0,
                                            float kf, int pbeg, int cnt, float &pe, float &pb, float &pv,
                                            float &pw) {
    const float4 *pp = a.PX + pbeg;
    float4 gn = __ldg(pp);
    const int last = cnt - 1;
#pragma unroll 4
    for (int i = 0; i < last; ++i) {
        const float4 g = gn;
        gn = __ldg(pp + i + 1);
        member_pair<KIND, MODE>(a, R, qtab, u0, kf, g, pe, pb, pv, pw);
        kf += 1.0f;
    }
    member_pair<KIND, MODE>(a, R, qtab, u0, kf, gn, pe, pb, pv, pw);
}

// pixel-mode general pair loop for one target and one ring pair; MODE picks
// the sine series by the largest |u| of the ring pair (0: <= 0.05 rad,
// 1: <= 0.45 rad, 2: |u| <= pi).  Offsets within hw_in are members for
// certain; the few offsets between hw_in and the window's edges are tested,
// and the members among them join the run.  The run's pairs have no test at
// all, and its galaxy count comes from the count prefix.  Offsets inside the
// float32 guard band are only counted (nband_out): they are decided in
// float64 once the target's other pairs are summed.  A window that stays
// inside the bin ring's pixel range (all but the targets next to the seam
// at azimuth 0) takes one run with no wrapping arithmetic.
template <int KIND, int MODE>
__device__ __forceinline__ void general_segment(const MapArgs &a, const RingPair &R, const TargetRing &tr,
                                                const LatticeDiv &ld, const float4 *qtab, float &pe, float &pb,
                                                float &pv, float &pw, int &nn, int &nm, int &nband_out) {
    const int q = R.nr >> 2;
    int Xi;
    float Xf;
    lattice_position(tr, ld, q, Xi, Xf);
    const float fr = ((R.flags & RP_SHIFTED) ? 0.5f : 0.0f) - Xf;
    int kl, kh;
    window(R, fr, kl, kh);
    int il = max(kl, (int)ceilf(-fr - R.hw_in)), ih = min(kh, (int)floorf(-fr + R.hw_in));
    const float u0 = fr * R.dphi;
    const bool inside = Xi + kl >= 0 && Xi + kh < R.nr;
    // The offsets outside the certain members are tested one by one, from the
    // inside out (the same float32 chord^2 as the guard-band rescan): a member
    // next to the run joins it (chord^2 grows with |u| on either side of the
    // target, so the members form one interval), a member elsewhere is added
    // alone, and the offsets inside the guard band are only counted (nband):
    // they are decided in float64 once the target's other pairs are summed.
    int nband = 0;
    nband_out = 0;
    if (kl > kh) return;      // no offset in the window
    int ilc = il, ihc = ih;   // the tested sides start next to these
    if (il > ih) {            // no certain member: the run grows from the offset nearest the target
        const int ks = min(max(__float2int_rn(-fr), kl), kh);
        const float u = fmaf((float)ks, R.dphi, u0);
        float sinu, h;
        sin_hav<MODE>(u, sinu, h);
        const float s2 = fmaf(R.B, h, R.A);
        ilc = ihc = ks;
        if (s2 < a.Tlo) {
            il = ih = ks;
        } else {
            nband += s2 <= a.Thi ? 1 : 0;
            il = ks + 1;      // an empty run just above ks
            ih = ks;
        }
    }
    // below the run (kl <= k < ilc), then above it (ihc < k <= kh); most ring
    // pairs have no such offset (the two half windows differ by a few
    // hundredths of a pixel)
    if (ilc > kl || ihc < kh)
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
        const int k0 = side == 0 ? kl : ihc + 1, k1 = side == 0 ? ilc - 1 : kh;
        for (int i = 0; i <= k1 - k0; ++i) {
            const int k = side == 0 ? k1 - i : k0 + i;      // from the run outward
            const float u = fmaf((float)k, R.dphi, u0);
            float sinu, h;
            sin_hav<MODE>(u, sinu, h);
            const float s2 = fmaf(R.B, h, R.A);
            if (s2 < a.Tlo) {
                if (side == 0 && k == il - 1) il = k;
                else if (side == 1 && k == ih + 1) ih = k;
                else pixel_pair<KIND, MODE>(a, R, qtab, u, R.start + (inside ? Xi + k : wrap_start(R, Xi, k)), pe, pb,
                                            pv, pw, nn, nm);
            } else {
                nband += s2 <= a.Thi ? 1 : 0;
            }
        }
    }
    const int len = ih - il + 1;
    if (inside) {
        if (len > 0) {
            const int pbeg = R.start + Xi + il;
            certain_run<KIND, MODE>(a, R, qtab, u0, (float)il, pbeg, len, pe, pb, pv, pw);
            nn += __ldg(a.NPRE + pbeg + len) - __ldg(a.NPRE + pbeg);
            nm += len;
        }
    } else if (len > 0) {
        // the run: bin pixels [kk0, nr) then [0, ...) when they wrap
        const int kk0 = wrap_start(R, Xi, il);
        const int n1 = min(len, R.nr - kk0);
#pragma unroll 1
        for (int part = 0; part < 2; ++part) {
            const int cnt = part == 0 ? n1 : len - n1;
            if (cnt <= 0) continue;
            const int pbeg = part == 0 ? R.start + kk0 : R.start;
            certain_run<KIND, MODE>(a, R, qtab, u0, (float)(part == 0 ? il : il + n1), pbeg, cnt, pe, pb, pv, pw);
            nn += __ldg(a.NPRE + pbeg + cnt) - __ldg(a.NPRE + pbeg);
            nm += cnt;
        }
    }
    nband_out = nband;
}

// Targets of the general kernel with guard-band pairs.  Such a target takes
// a slot for its raw sums and a mask of the ring-pair entries that hold
// those pairs (bit e for entry e < 63, bit 63 for every entry from 63 on);
// one thread per slot then decides them in float64 and normalises the
// target.  A target that finds no free slot does the same in place, with
// the same code, so the result never depends on which of the two ran.
struct GenBand {
    double *raw;                   // 4 per slot: SE, SB, SV, SW
    int32_t *cnt;                  // 2 per slot: galaxies, member pixels
    int64_t *idx;                  // the target's position in its general list
    unsigned long long *mask;      // ring-pair entries with guard-band pairs
    unsigned long long *counts;    // [0]: slots claimed
    int64_t cap_slots;
};

constexpr int64_t GEN_BAND_SLOT_BYTES = 4 * sizeof(double) + sizeof(int64_t) + sizeof(unsigned long long) +
                                        2 * sizeof(int32_t);

// the slot arrays in one allocation of slots * GEN_BAND_SLOT_BYTES bytes
inline GenBand gen_band_layout(void *buf, int64_t slots, unsigned long long *counts) {
    GenBand gb;
    char *p = (char *)buf;
    gb.raw = (double *)p;
    p += slots * 4 * sizeof(double);
    gb.idx = (int64_t *)p;
    p += slots * sizeof(int64_t);
    gb.mask = (unsigned long long *)p;
    p += slots * sizeof(unsigned long long);
    gb.cnt = (int32_t *)p;
    gb.counts = counts;
    gb.cap_slots = slots;
    return gb;
}

// slots for n general targets (a small share of them has guard-band pairs)
inline int64_t gen_band_slots(int64_t n) { return (1 << 16) + n / 8; }

// galaxies in the bin pixels [lo, lo + len) of a ring (indices mod nr)
__device__ __forceinline__ int ring_range_count(const int32_t *pre, int start, int nr, int lo, int len) {
    lo %= nr;
    if (lo < 0) lo += nr;
    const int hi = lo + len;
    if (hi <= nr) return __ldg(pre + start + hi) - __ldg(pre + start + lo);
    return (__ldg(pre + start + nr) - __ldg(pre + start + lo)) + (__ldg(pre + start + hi - nr) - __ldg(pre + start));
}

// ------------------------------------------------------------------------
// Toeplitz kernel: output rings whose every ring pair is a Toeplitz pair.
// Persistent CTAs take tiles of up to TS slots of one ring; thread tid owns
// the RB = 8 slots 8 tid .. 8 tid + 7 and keeps the eight bin pixels its
// slots need at the current offset in registers: register W[p & 7] holds bin
// pixel p, so at offset dd slot r reads W[(dd + r) & 7], and each step loads
// one new pixel (8 tid + dd + 7) and one geometry entry for eight pairs.
// Steps are unrolled by eight so that the register of every pixel is fixed
// at compile time (no moves).  Per ring pair the CTA stages, with cp.async
// into a double buffer, the bin-ring segment the tile needs (16-byte pixels
// in the XOR-swizzled row layout of tpos) and the per-offset geometry; ring
// pair e + 1 is in flight while e is summed.  The galaxy counts of the
// windows are differences of the count prefix, read from global memory.
// Tiles of other rings are skipped (the general kernel has them).
// ------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// floor(a / b) for -b <= a < 2b
__device__ __forceinline__ int wraps(int a, int b) { return a < 0 ? -1 : (a >= b ? 1 : 0); }


// what a tile needs of one of its ring pairs; the tile's first TPN ring
// pairs are read into shared memory once, at the start of the tile
struct ToeStage {
    int start, nr, k0, L, off, da, tot, namb;
};
constexpr int TPN = 64;

__device__ __forceinline__ ToeStage toe_param(const MapArgs &a, int64_t row0, int e) {
    ToeStage t;
    t.start = __ldg(&a.table[row0 + e].start);
    t.nr = __ldg(&a.table[row0 + e].nr);
    const ToeInfo ti = a.toe[row0 + e];
    t.L = ti.L;
    t.off = ti.off;
    t.da = ti.da;
    t.k0 = ti.dlo + ti.da;                 // relative to the tile's first slot
    t.namb = ti.namb;
    t.tot = __ldg(a.NPRE + t.start + t.nr) - __ldg(a.NPRE + t.start);   // galaxies on the bin ring
    return t;
}

__device__ __forceinline__ ToeStage tile_param(const MapArgs &a, const ToeStage *par, int64_t row0, int e,
                                               int jbase) {
    ToeStage t = e < TPN ? par[e] : toe_param(a, row0, e);
    t.k0 += jbase;
    return t;
}

// issue the copies of ring pair e of a tile into buffer b
template <int NC>
__device__ __forceinline__ void toe_stage(const MapArgs &a, const ToeStage *par, int64_t row0, int e, int jbase,
                                          int nslots, float4 (*seg)[toe_segn<NC>()], float4 (*geo)[NC], int b,
                                          int tid) {
    const ToeStage t = tile_param(a, par, row0, e, jbase);
    if (t.L > 0) {
        const int nseg = min(toe_segn<NC>(), nslots + t.L + 7);
        if (t.k0 >= 0 && t.k0 + nseg <= t.nr) {
            // no seam: pixel m = tid + NT i sits in row (tid >> 3) + 4 i and
            // column tid & 7, so tpos(m) is one of two per-thread positions
            // (even or odd i) plus NT i: copies with immediate offsets
            const float4 *g = a.PX + t.start + t.k0 + tid;
            const int r0 = tid >> 3, c = tid & 7;
            float4 *se = &seg[b][(r0 << 3) | (c ^ r0)];
            float4 *so = &seg[b][(r0 << 3) | (c ^ (r0 + 4))];
#pragma unroll
            for (int i = 0; i < (toe_segn<NC>() + NT - 1) / NT; ++i)
                if (tid + NT * i < nseg) cp_async16(((i & 1) ? so : se) + NT * i, g + NT * i);
        } else {
            // -nr < k0 + m < 2 nr for every staged m (the window is shorter than the ring)
            for (int m = tid; m < nseg; m += NT) {
                int kk = t.k0 + m;
                kk += kk < 0 ? t.nr : (kk >= t.nr ? -t.nr : 0);
                cp_async16(&seg[b][tpos(m)], a.PX + t.start + kk);
            }
        }
        for (int c = tid; c < t.L; c += NT) cp_async16(&geo[b][c], a.toe_geo + t.off + t.da + c);
    }
    cp_async_commit();
}

template <int NC>
struct ToeShared {
    float4 seg[2][toe_segn<NC>()];
    float4 geo[2][NC];
    int slot_t[TS];
    ToeStage par[TPN];
};

// the pair contribution of slot r: geometry G (Q cos 2psi, Q sin 2psi,
// -Q sin 2psi, Q^2) on pixel P (G1, G2, S2, W)
#define SMART_ACC(r, P, G)                               \
    pe[r] = fmaf(G.x, P.x, fmaf(G.y, P.y, pe[r]));     \
    pb[r] = fmaf(G.x, P.y, fmaf(G.z, P.x, pb[r]));     \
    pv[r] = fmaf(G.w, P.z, pv[r]);                     \
    pw[r] += P.w;

// one offset step j of an eight-step block starting at offset dd0 (a
// multiple of 8): load pixel 8 tid + dd0 + j + 7 into W[(j + 7) & 7] (its
// row is rowA for j = 0 and rowA + 1 otherwise), then the eight pairs
#define SMART_TOE_STEP(j)                                                                   \
    {                                                                                      \
        constexpr int cj = ((j) + 7) & 7;                                                  \
        const int row = (j) == 0 ? rowA : rowA + 1;                                        \
        W[cj] = sg[(row << 3) | (cj ^ (row & 7))];                                         \
        const float4 G = gb[(j)];                                                          \
        SMART_ACC(0, W[(j) & 7], G) SMART_ACC(1, W[((j) + 1) & 7], G)                      \
        SMART_ACC(2, W[((j) + 2) & 7], G) SMART_ACC(3, W[((j) + 3) & 7], G)                \
        SMART_ACC(4, W[((j) + 4) & 7], G) SMART_ACC(5, W[((j) + 5) & 7], G)                \
        SMART_ACC(6, W[((j) + 6) & 7], G) SMART_ACC(7, W[((j) + 7) & 7], G)                \
    }

// one tile of a Toeplitz output ring, summed by the whole CTA (NT threads);
// ends with a barrier, so the shared buffers are free on return.  Sums in
// two levels: float32 partial sums over two ring pairs (2 L terms, a few
// dozen), added to the target's float32 totals (a few dozen partials).  A
// compensated (Kahan) total cost 13 % of the kernel's time (its registers
// crowd the hot loop) for no accuracy the tests or the oracle comparison
// can see.
template <int KIND, int NC>
__device__ __forceinline__ void toeplitz_tile(const MapArgs &a, int64_t tile, ToeShared<NC> &S) {
    auto &seg = S.seg;
    auto &geo = S.geo;
    auto &slot_t = S.slot_t;
    const int tid = threadIdx.x;
    const int64_t tb = a.tiles[tile], te = a.tiles[tile + 1];
    const TargetRing tr0 = target_ring(a.N0, a.targets[tb]);
    const int jbase = tr0.j0 & ~(TS - 1);
    const int nslots = min(TS, tr0.nr0 - jbase);
    const int64_t ring_start0 = a.targets[tb] - tr0.j0;
    const int64_t row0 = (int64_t)(tr0.i0 - 1) * a.kmax;
    const int nent = a.counts[tr0.i0 - 1];
    for (int s = tid; s < TS; s += NT) slot_t[s] = -1;
    for (int e = tid; e < min(nent, TPN); e += NT) S.par[e] = toe_param(a, row0, e);
    __syncthreads();
    for (int64_t t = tb + tid; t < te; t += NT) slot_t[(int)(a.targets[t] - ring_start0) - jbase] = (int)(t - tb);
    __syncthreads();      // slot map and ring-pair parameters written

    toe_stage<NC>(a, S.par, row0, 0, jbase, nslots, seg, geo, 0, tid);

    const int s0 = RB * tid;
    bool any = false;
#pragma unroll
    for (int r = 0; r < RB; ++r) any |= (s0 + r < nslots) && slot_t[s0 + r] >= 0;
    float SE[RB], SB[RB], SV[RB], SW[RB];
    int NN[RB], NM[RB];
    float pe[RB], pb[RB], pv[RB], pw[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        SE[r] = SB[r] = SV[r] = SW[r] = 0.f;
        NN[r] = NM[r] = 0;
        pe[r] = pb[r] = pv[r] = pw[r] = 0.f;
    }

    for (int e = 0; e < nent; ++e) {
        const int b = e & 1;
        cp_async_wait_all();
        __syncthreads();       // ring pair e staged; everyone is done with buffer b ^ 1
        if (e + 1 < nent) toe_stage<NC>(a, S.par, row0, e + 1, jbase, nslots, seg, geo, b ^ 1, tid);
        const ToeStage cur = tile_param(a, S.par, row0, e, jbase);
        const int L = cur.L;
        if (L > 0 && any) {
            const float4 *sg = seg[b];
            float4 W[8];
            // pixels 8 tid .. 8 tid + 6 (row tid); the steps load the rest
#pragma unroll
            for (int c = 0; c < 7; ++c) W[c] = sg[(tid << 3) | (c ^ (tid & 7))];
            int dd0 = 0;
            for (; dd0 + 8 <= L; dd0 += 8) {
                const int rowA = tid + (dd0 >> 3);
                const float4 *gb = geo[b] + dd0;
                SMART_TOE_STEP(0) SMART_TOE_STEP(1) SMART_TOE_STEP(2) SMART_TOE_STEP(3)
                SMART_TOE_STEP(4) SMART_TOE_STEP(5) SMART_TOE_STEP(6) SMART_TOE_STEP(7)
            }
            const int rem = L - dd0;
            if (rem > 0) {
                const int rowA = tid + (dd0 >> 3);
                const float4 *gb = geo[b] + dd0;
                SMART_TOE_STEP(0)
                if (rem > 1) {
                    SMART_TOE_STEP(1)
                    if (rem > 2) {
                        SMART_TOE_STEP(2)
                        if (rem > 3) {
                            SMART_TOE_STEP(3)
                            if (rem > 4) {
                                SMART_TOE_STEP(4)
                                if (rem > 5) {
                                    SMART_TOE_STEP(5)
                                    if (rem > 6) SMART_TOE_STEP(6)
                                }
                            }
                        }
                    }
                }
            }
            // galaxies of the slots' windows [k0 + s, k0 + s + L) from the
            // count prefix in global memory: after the pairs (the window never
            // passes the ring's end more than once; tiles at the seam take the
            // wrapped indices).  Read with lane t taking slots t + 32 r
            // (coalesced) they were slower.
            const int lo0 = cur.k0 + s0;
            const bool seam = lo0 < 0 || lo0 + RB - 1 + L >= cur.nr;
            int pa[RB], pz[RB];
            if (!seam) {
                const int32_t *pp = a.NPRE + cur.start + lo0;
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    pa[r] = __ldg(pp + r);
                    pz[r] = __ldg(pp + r + L);
                }
            } else {
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    const int lo = lo0 + r, hi = lo + L;
                    const int klo = lo - wraps(lo, cur.nr) * cur.nr, khi = hi - wraps(hi, cur.nr) * cur.nr;
                    pa[r] = __ldg(a.NPRE + cur.start + klo);
                    pz[r] = __ldg(a.NPRE + cur.start + khi) + (wraps(hi, cur.nr) - wraps(lo, cur.nr)) * cur.tot;
                }
            }
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                NN[r] += pz[r] - pa[r];
                NM[r] += L;
            }
            if ((e & 1) || e + 1 == nent) {
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    SE[r] += pe[r];
                    SB[r] += pb[r];
                    SV[r] += pv[r];
                    SW[r] += pw[r];
                    pe[r] = pb[r] = pv[r] = pw[r] = 0.f;
                }
            }
        } else if (any && ((e & 1) || e + 1 == nent)) {
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                SE[r] += pe[r];
                SB[r] += pb[r];
                SV[r] += pv[r];
                SW[r] += pw[r];
                pe[r] = pb[r] = pv[r] = pw[r] = 0.f;
            }
        }
    }
    // ---- guard-band offsets, after every ring pair (the hot loop's
    // registers are dead here): decided per target in float64
    if (any) {
        for (int e = 0; e < nent; ++e) {
            const ToeInfo ti = a.toe[row0 + e];
            if (ti.namb <= 0) continue;
            const int nr = __ldg(&a.table[row0 + e].nr), start = __ldg(&a.table[row0 + e].start);
            for (int ia = 0; ia < ti.namb; ++ia) {
                const int c = ia == 0 ? ti.amb0 : (ia == 1 ? ti.amb1 : ti.amb2);
                const float4 G = __ldg(a.toe_geo + ti.off + c);
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    if (s0 + r >= nslots || slot_t[s0 + r] < 0) continue;
                    const int64_t pix = ring_start0 + jbase + s0 + r;
                    int kk = (jbase + s0 + r + ti.dlo + c) % nr;
                    if (kk < 0) kk += nr;
                    const int p = start + kk;
                    if (!exact_member(a, pix, p)) continue;
                    const float4 px = __ldg(a.PX + p);
                    SE[r] += fmaf(G.x, px.x, G.y * px.y);
                    SB[r] += fmaf(G.x, px.y, G.z * px.x);
                    SV[r] += G.w * px.z;
                    SW[r] += px.w;
                    NN[r] += __ldg(a.NP + p);
                    NM[r] += 1;
                }
            }
        }
    }
    cp_async_wait_all();
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        const int ti = (s0 + r < nslots) ? slot_t[s0 + r] : -1;
        if (ti >= 0) finalise(a, tb + ti, SE[r], 0.f, SB[r], 0.f, SV[r], 0.f, SW[r], 0.f, NN[r], NM[r]);
    }
    __syncthreads();   // slot map and buffers are rewritten by the next tile
}
#undef SMART_TOE_STEP
#undef SMART_ACC

// is this tile on an output ring of the Toeplitz kernel?
__device__ __forceinline__ bool toeplitz_tile_wanted(const MapArgs &a, int64_t tile) {
    const TargetRing tr0 = target_ring(a.N0, a.targets[a.tiles[tile]]);
    return a.toe_ring[tr0.i0 - 1] != 0;
}

// mirror line m of two targets on one ring (pix2 the image of pix about
// the meridian m pi/4; tr is the ring position of pix): j + j2 + s = m q
// (mod 4 q)
__device__ __forceinline__ int mirror_line(const TargetRing &tr, int64_t pix, int64_t pix2) {
    const int j2 = tr.j0 + (int)(pix2 - pix);
    return ((tr.j0 + j2 + tr.s0) % tr.nr0) / tr.q0;
}

// guard-band pairs of the ring-pair entries in mask, then the summed
// normalisation (Sect. 2.4) of target t from its raw sums.  tg is the target
// whose window and geometry the sums were taken with: t itself, or the
// partner of a mirror pair (general_target2) when t is the pair's image.
template <int KIND>
__device__ __forceinline__ void band_finish(const MapArgs &a, int64_t t, int64_t tg, const float4 *qtab,
                                            unsigned long long mask, double se, double sb, double sv, double sw,
                                            int NN, int NM) {
    const int64_t pix = a.targets[t];
    const int64_t pixg = tg == t ? pix : a.targets[tg];
    const TargetRing tr = target_ring(a.N0, pixg);
    const LatticeDiv ld = lattice_div(tr);
    const int mline = tg == t ? -1 : mirror_line(tr, pixg, pix);
    const int64_t row0 = (int64_t)(tr.i0 - 1) * a.kmax;
    const int nent = a.counts[tr.i0 - 1];
    float pe = 0.f, pb = 0.f, pv = 0.f, pw = 0.f;
    for (int e = 0; e < nent; ++e) {
        if (!((mask >> min(e, 63)) & 1ull)) continue;
        const RingPair R = a.table[row0 + e];
        const int mode = (R.flags & RP_WIDE) ? 2 : (((R.hw + 1.0f) * R.dphi <= 0.05f) ? 0 : 1);
        if (mode == 0) band_pairs<KIND, 0>(a, R, tr, ld, pix, mline, qtab, pe, pb, pv, pw, NN, NM);
        else if (mode == 1) band_pairs<KIND, 1>(a, R, tr, ld, pix, mline, qtab, pe, pb, pv, pw, NN, NM);
        else band_pairs<KIND, 2>(a, R, tr, ld, pix, mline, qtab, pe, pb, pv, pw, NN, NM);
    }
    const double SW = sw + (double)pw;
    float me = 0.f, mb = 0.f, vv = 0.f;
    if (SW > 0.0) {
        const float r = (float)a.area / (float)SW;       // 1 / nbar
        me = (float)(se + (double)pe) * r;
        mb = (float)(sb + (double)pb) * r;
        vv = 0.5f * (float)(sv + (double)pv) * r * r;
    }
    if (a.sum_w) a.sum_w[t] = SW;
    if (a.map_e) a.map_e[t] = me;
    if (a.map_b) a.map_b[t] = mb;
    if (a.var) a.var[t] = vv;
    if (a.count) a.count[t] = NN;
    if (a.members) a.members[t] = NM;
}

// band_finish out of line, for the rare target that finds no free slot (a
// call keeps the general loop's registers free of it); a points to a
// __grid_constant__ kernel parameter or to global memory
template <int KIND>
__device__ __noinline__ void band_finish_call(const MapArgs *a, int64_t t, int64_t tg, const float4 *qtab,
                                              unsigned long long mask, double se, double sb, double sv, double sw,
                                              int NN, int NM) {
    band_finish<KIND>(*a, t, tg, qtab, mask, se, sb, sv, sw, NN, NM);
}

// the end of a general target: normalised at once without guard-band
// pairs; else its raw sums go to a slot (slot tag: the work-list position
// times two, plus one for the image of a mirror pair), or, without a free
// slot, band_finish runs in place
template <int KIND>
__device__ __forceinline__ void general_finish(const MapArgs &a, int64_t t, int64_t tg, int64_t tag,
                                               const float4 *qtab, const GenBand &gb, unsigned long long mask,
                                               float SE, float cSE, float SB, float cSB, float SV, float SW,
                                               float cSW, int NN, int NM) {
    if (!mask) {
        finalise(a, t, SE, cSE, SB, cSB, SV, 0.f, SW, cSW, NN, NM);
        return;
    }
    const double se = (double)SE - (double)cSE, sb = (double)SB - (double)cSB, sw = (double)SW - (double)cSW;
    const unsigned long long slot = atomicAdd(gb.counts, 1ull);
    if (slot < (unsigned long long)gb.cap_slots) {
        double *raw = gb.raw + 4 * slot;
        raw[0] = se;
        raw[1] = sb;
        raw[2] = (double)SV;
        raw[3] = sw;
        gb.cnt[2 * slot] = NN;
        gb.cnt[2 * slot + 1] = NM;
        gb.idx[slot] = tag;
        gb.mask[slot] = mask;
    } else {
        band_finish_call<KIND>(&a, t, tg, qtab, mask, se, sb, (double)SV, sw, NN, NM);
    }
}

// one target of a general output ring (one thread); gidx is its position in
// the general work list.  Guard-band pairs are left to band_finish.
template <int KIND>
__device__ __forceinline__ void general_target(const MapArgs &a, int64_t t, int64_t gidx, const float4 *qtab,
                                               const GenBand &gb) {
    const int64_t pix = a.targets[t];
    const TargetRing tr = target_ring(a.N0, pix);
    const LatticeDiv ld = lattice_div(tr);
    const int64_t row0 = (int64_t)(tr.i0 - 1) * a.kmax;
    const int nent = a.counts[tr.i0 - 1];
    float SE = 0.f, cSE = 0.f, SB = 0.f, cSB = 0.f, SV = 0.f, SW = 0.f, cSW = 0.f;
    int NN = 0, NM = 0;
    unsigned long long mask = 0;
    for (int e = 0; e < nent; ++e) {
        const RingPair R = a.table[row0 + e];
        const int mode = (R.flags & RP_WIDE) ? 2 : (((R.hw + 1.0f) * R.dphi <= 0.05f) ? 0 : 1);
        float pe = 0.f, pb = 0.f, pv = 0.f, pw = 0.f;
        int nn = 0, nm = 0, nb = 0;
        if (mode == 0) general_segment<KIND, 0>(a, R, tr, ld, qtab, pe, pb, pv, pw, nn, nm, nb);
        else if (mode == 1) general_segment<KIND, 1>(a, R, tr, ld, qtab, pe, pb, pv, pw, nn, nm, nb);
        else general_segment<KIND, 2>(a, R, tr, ld, qtab, pe, pb, pv, pw, nn, nm, nb);
        mask |= nb > 0 ? 1ull << min(e, 63) : 0ull;
        kahan_add(SE, cSE, pe);
        kahan_add(SB, cSB, pb);
        SV += pv;
        kahan_add(SW, cSW, pw);
        NN += nn;
        NM += nm;
    }
    general_finish<KIND>(a, t, t, 2 * gidx, qtab, gb, mask, SE, cSE, SB, cSB, SV, SW, cSW, NN, NM);
}

// ------------------------------------------------------------------------
// Mirror pairs of general targets.  Every HEALPix ring is symmetric about
// the meridians phi = m pi/4 (m = 0..3): the pixel centred at azimuth phi
// has an image at m pi/2 - phi on the same ring.  Two targets that are
// images of each other see mirror-image neighbourhoods on every bin ring:
// the pair (image target, image of bin pixel k) has the azimuth offset -u
// of the pair (target, k), hence the same chord, filter weight and y, and
// x -> -x (cos 2psi unchanged, sin 2psi negated).  general_target2 takes
// both targets in one thread and evaluates each pair's geometry once for
// the two; memberships outside the guard band follow from the shared s^2,
// those inside it are decided in float64 for each target on its own pixels.
// ------------------------------------------------------------------------
struct PairSums {
    float e, b, v, w;
};

// one member pair of the target and of its image: bin pixel data g (target)
// and h (image) at lattice offset kf
template <int KIND, int MODE>
__device__ __forceinline__ void member_pair2(const MapArgs &a, const RingPair &R, const float4 *qtab, float u0,
                                             float kf, const float4 &g, const float4 &h, PairSums &P,
                                             PairSums &M) {
    const float u = fmaf(kf, R.dphi, u0);
    float sinu, hv;
    sin_hav<MODE>(u, sinu, hv);
    const float s2 = fmaf(R.B, hv, R.A);
    const float x = R.mrho0 * sinu;
    const float y = fmaf(R.D, hv, R.C);
    const float xx = x * x;
    const float cc = fmaf(y, y, -xx);
    const float ss = -2.0f * x * y;
    float Q, w;
    if (KIND == SMART_FILTER_POLY) {
        const float d2 = sep2_from_chord2(s2);
        const float qn1 = a.f.qnorm * a.f.inv_ap2;
        const float t = fmaf(d2, -qn1 * a.f.inv_ap2, qn1);
        Q = d2 * t;
        w = fmaf(Q, fmaf(d2, fmaf(d2, 2.0f / 189.0f, 1.0f / 15.0f), 1.0f / 3.0f), t);
    } else {
        Q = qtab_eval_member(qtab, s2, a.f.tab_scale);
        w = __fdividef(Q, fmaf(y, y, xx) + 1e-30f);
    }
    // the weighted rotation once for both targets: wc = Q cos 2psi and
    // ws = Q sin 2psi (w = Q / sin^2 d; cc and ss carry sin^2 d), then two
    // FMAs per sum
    const float QQ = Q * Q, wc = w * cc, ws = w * ss;
    P.e = fmaf(g.y, ws, fmaf(g.x, wc, P.e));
    P.b = fmaf(-g.x, ws, fmaf(g.y, wc, P.b));
    P.v = fmaf(QQ, g.z, P.v);
    P.w += g.w;
    M.e = fmaf(-h.y, ws, fmaf(h.x, wc, M.e));
    M.b = fmaf(h.x, ws, fmaf(h.y, wc, M.b));
    M.v = fmaf(QQ, h.z, M.v);
    M.w += h.w;
}

// certain members of both targets: the target's bin pixels p1 .. p1 + cnt - 1
// upwards, the image's p2 .. p2 - cnt + 1 downwards (cnt >= 1, neither run
// crossing the ring's seam); loads one iteration ahead, last pair peeled
template <int KIND, int MODE>
__device__ __forceinline__ void certain_run2(const MapArgs &a, const RingPair &R, const float4 *qtab, float u0,
                                             float kf, int p1, int p2, int cnt, PairSums &P, PairSums &M) {
    const float4 *pp = a.PX + p1;
    const float4 *qq = a.PX + p2;
    float4 gn = __ldg(pp), hn = __ldg(qq);
    const int last = cnt - 1;
#pragma unroll 4
    for (int i = 0; i < last; ++i) {
        const float4 g = gn, h = hn;
        gn = __ldg(pp + i + 1);
        hn = __ldg(qq - i - 1);
        member_pair2<KIND, MODE>(a, R, qtab, u0, kf, g, h, P, M);
        kf += 1.0f;
    }
    member_pair2<KIND, MODE>(a, R, qtab, u0, kf, gn, hn, P, M);
}

// a tested member of both targets (bin pixels p1 and p2), as pixel_pair
template <int KIND, int MODE>
__device__ __forceinline__ void pixel_pair2(const MapArgs &a, const RingPair &R, const float4 *qtab, float u, int p1,
                                            int p2, PairSums &P, PairSums &M, int &nn, int &nn2, int &nm) {
    float sinu, hv;
    sin_hav<MODE>(u, sinu, hv);
    const float s2 = fmaf(R.B, hv, R.A);
    const float x = R.mrho0 * sinu;
    const float y = fmaf(R.D, hv, R.C);
    const float xx = x * x;
    const float sd2 = fmaf(y, y, xx);
    const float cc = fmaf(y, y, -xx);
    const float ss = -2.0f * x * y;
    const float Q = filter_Q<KIND>(a.f, qtab, s2);
    const float w = sd2 > 1e-30f ? __fdividef(Q, sd2) : 0.f;
    const float QQ = Q * Q;
    const float4 g = __ldg(a.PX + p1), h = __ldg(a.PX + p2);
    P.e = fmaf(w, fmaf(g.x, cc, g.y * ss), P.e);
    P.b = fmaf(w, fmaf(g.y, cc, -g.x * ss), P.b);
    P.v = fmaf(QQ, g.z, P.v);
    P.w += g.w;
    M.e = fmaf(w, fmaf(h.x, cc, -h.y * ss), M.e);
    M.b = fmaf(w, fmaf(h.y, cc, h.x * ss), M.b);
    M.v = fmaf(QQ, h.z, M.v);
    M.w += h.w;
    nn += __ldg(a.NP + p1);
    nn2 += __ldg(a.NP + p2);
    nm += 1;
}

// general_segment for a target and its image about the meridian mline pi/4:
// the window, the tested offsets and the run are the target's; the image
// reads the mirror image of every bin pixel.  The run is cut where either
// of the two crosses its ring's seam (at most three pieces: the window is
// never longer than the ring).
template <int KIND, int MODE>
__device__ __forceinline__ void general_segment2(const MapArgs &a, const RingPair &R, const TargetRing &tr,
                                                 const LatticeDiv &ld, int mline, const float4 *qtab, PairSums &P,
                                                 PairSums &M, int &nn, int &nn2, int &nm, int &nband_out) {
    const int q = R.nr >> 2;
    int Xi;
    float Xf;
    lattice_position(tr, ld, q, Xi, Xf);
    const int sh = (R.flags & RP_SHIFTED) ? 1 : 0;
    const float fr = (sh ? 0.5f : 0.0f) - Xf;
    const int cm = mline * q - sh;
    int kl, kh;
    window(R, fr, kl, kh);
    int il = max(kl, (int)ceilf(-fr - R.hw_in)), ih = min(kh, (int)floorf(-fr + R.hw_in));
    const float u0 = fr * R.dphi;
    int nband = 0;
    nband_out = 0;
    if (kl > kh) return;      // no offset in the window
    int ilc = il, ihc = ih;
    if (il > ih) {            // no certain member: the run grows from the offset nearest the target
        const int ks = min(max(__float2int_rn(-fr), kl), kh);
        const float u = fmaf((float)ks, R.dphi, u0);
        float sinu, hv;
        sin_hav<MODE>(u, sinu, hv);
        const float s2 = fmaf(R.B, hv, R.A);
        ilc = ihc = ks;
        if (s2 < a.Tlo) {
            il = ih = ks;
        } else {
            nband += s2 <= a.Thi ? 1 : 0;
            il = ks + 1;
            ih = ks;
        }
    }
    if (ilc > kl || ihc < kh)
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
        const int k0 = side == 0 ? kl : ihc + 1, k1 = side == 0 ? ilc - 1 : kh;
        for (int i = 0; i <= k1 - k0; ++i) {
            const int k = side == 0 ? k1 - i : k0 + i;      // from the run outward
            const float u = fmaf((float)k, R.dphi, u0);
            float sinu, hv;
            sin_hav<MODE>(u, sinu, hv);
            const float s2 = fmaf(R.B, hv, R.A);
            if (s2 < a.Tlo) {
                if (side == 0 && k == il - 1) il = k;
                else if (side == 1 && k == ih + 1) ih = k;
                else {
                    const int kk = wrap_start(R, Xi, k);
                    pixel_pair2<KIND, MODE>(a, R, qtab, u, R.start + kk, R.start + mirror_index(R, cm, kk), P, M,
                                            nn, nn2, nm);
                }
            } else {
                nband += s2 <= a.Thi ? 1 : 0;
            }
        }
    }
    const int len = ih - il + 1;
    if (len > 0) {
        int kk = wrap_start(R, Xi, il), mm = mirror_index(R, cm, kk), left = len;
        float kf = (float)il;
#pragma unroll 1
        for (int piece = 0; piece < 3 && left > 0; ++piece) {
            const int cnt = min(left, min(R.nr - kk, mm + 1));
            certain_run2<KIND, MODE>(a, R, qtab, u0, kf, R.start + kk, R.start + mm, cnt, P, M);
            nn += __ldg(a.NPRE + R.start + kk + cnt) - __ldg(a.NPRE + R.start + kk);
            nn2 += __ldg(a.NPRE + R.start + mm + 1) - __ldg(a.NPRE + R.start + mm + 1 - cnt);
            left -= cnt;
            kf += (float)cnt;
            kk += cnt;
            kk = kk == R.nr ? 0 : kk;
            mm -= cnt;
            mm = mm < 0 ? R.nr - 1 : mm;
        }
        nm += len;
    }
    nband_out = nband;
}

// a target t and its image t2 about a meridian m pi/4 (one thread); wpos is
// their position in the general work list
template <int KIND>
__device__ __forceinline__ void general_target2(const MapArgs &a, int64_t t, int64_t t2, int64_t wpos,
                                                const float4 *qtab, const GenBand &gb) {
    const int64_t pix = a.targets[t];
    const TargetRing tr = target_ring(a.N0, pix);
    const LatticeDiv ld = lattice_div(tr);
    const int mline = mirror_line(tr, pix, a.targets[t2]);
    const int64_t row0 = (int64_t)(tr.i0 - 1) * a.kmax;
    const int nent = a.counts[tr.i0 - 1];
    float SE = 0.f, SB = 0.f, SV = 0.f, SW = 0.f, SE2 = 0.f, SB2 = 0.f, SV2 = 0.f, SW2 = 0.f;
    int NN = 0, NN2 = 0, NM = 0;
    unsigned long long mask = 0;
    for (int e = 0; e < nent; ++e) {
        const RingPair R = a.table[row0 + e];
        const int mode = (R.flags & RP_WIDE) ? 2 : (((R.hw + 1.0f) * R.dphi <= 0.05f) ? 0 : 1);
        PairSums P{0.f, 0.f, 0.f, 0.f}, M{0.f, 0.f, 0.f, 0.f};
        int nn = 0, nn2 = 0, nm = 0, nb = 0;
        if (mode == 0) general_segment2<KIND, 0>(a, R, tr, ld, mline, qtab, P, M, nn, nn2, nm, nb);
        else if (mode == 1) general_segment2<KIND, 1>(a, R, tr, ld, mline, qtab, P, M, nn, nn2, nm, nb);
        else general_segment2<KIND, 2>(a, R, tr, ld, mline, qtab, P, M, nn, nn2, nm, nb);
        mask |= nb > 0 ? 1ull << min(e, 63) : 0ull;
        SE += P.e;
        SB += P.b;
        SV += P.v;
        SW += P.w;
        SE2 += M.e;
        SB2 += M.b;
        SV2 += M.v;
        SW2 += M.w;
        NN += nn;
        NN2 += nn2;
        NM += nm;
    }
    general_finish<KIND>(a, t, t, 2 * wpos, qtab, gb, mask, SE, 0.f, SB, 0.f, SV, SW, 0.f, NN, NM);
    general_finish<KIND>(a, t2, t, 2 * wpos + 1, qtab, gb, mask, SE2, 0.f, SB2, 0.f, SV2, SW2, 0.f, NN2, NM);
}

}  // namespace smart
