// aperture_galaxy.cu -- brute-force aperture mass at galaxy positions
// (Sect. 3.1 steps 1-5), neighbours found through the catalogue sorted by
// HEALPix pixel (Sect. 3.4).
//
// Work unit: one warp per group of up to GT consecutive targets of one
// output ring.  For every bin ring that can hold members (the ring-pair
// table built for theta_ap plus the largest pixel radius) the galaxies of
// the union of the targets' pixel windows are one contiguous range of the
// sorted catalogue (two when the window wraps).  The lanes walk that range
// with stride 32 -- coalesced 16-byte loads -- and each galaxy record is
// used for all GT targets; sums are reduced across the warp with shuffles
// at the end.
//
// Per galaxy the record holds float32 offsets from its pixel centre
// (latitude in rad, azimuth in bin-pixel units), z = sin(dec), rho =
// cos(dec), and (w e1, w e2, w, w^2 |e|^2).  With dl = lat(target) -
// lat(galaxy) and u the azimuth difference:
//   s^2 = 4 sin^2(dl/2) + 4 rho0 rho sin^2(u/2),
//   x = -rho0 sin u,  y = sin(dl) + 2 z rho0 sin^2(u/2).
#include <math.h>

#include <algorithm>

#include "aperture_common.cuh"

namespace smart {

constexpr int GT_LOG2 = GAL_GROUP_LOG2;
constexpr int GT = 1 << GT_LOG2;   // targets per warp
constexpr int GW = 8;              // warps per CTA

struct GalRing {
    int start, nr;
    float dphi, B0, D0, mrho0, dlat, fr_shift;
    int small;         // |dl| and |u| stay below 0.45 rad: series; else float sincos
};

__device__ __forceinline__ GalRing gal_ring(const RingPair &Rp) {
    GalRing R;
    R.start = Rp.start;
    R.nr = Rp.nr;
    R.dphi = Rp.dphi;
    R.B0 = 4.0f * Rp.rho0;
    R.D0 = 2.0f * Rp.rho0;
    R.mrho0 = Rp.mrho0;
    R.dlat = Rp.dlat;
    R.fr_shift = (Rp.flags & RP_SHIFTED) ? 0.5f : 0.0f;
    R.small = !(Rp.flags & RP_WIDE);
    return R;
}

// galaxy-only part of the pair geometry; frg = the galaxy's azimuth on the
// bin-ring lattice minus its pixel index kg.  MODE 0: |dl| <= 0.05 rad, two
// series terms (truncation below 6e-8 relative); otherwise as below.
template <int MODE>
__device__ __forceinline__ void gal_setup_m(const GalRing &R, const float4 &geo, float &A, float &B, float &C,
                                            float &D, float &frg) {
    const float dl = R.dlat - geo.x;
    if (MODE == 0) {
        const float d2 = dl * dl;
        A = d2 * fmaf(d2, -1.0f / 12.0f, 1.0f);
        C = dl * fmaf(d2, -1.0f / 6.0f, 1.0f);
    } else if (MODE == 1) {
        const float d2 = dl * dl;
        A = d2 * fmaf(d2, fmaf(d2, 1.0f / 360.0f, -1.0f / 12.0f), 1.0f);
        C = dl * fmaf(d2, fmaf(d2, 1.0f / 120.0f, -1.0f / 6.0f), 1.0f);
    } else {
        float sdh, cdh;
        sincosf(0.5f * dl, &sdh, &cdh);
        A = 4.0f * sdh * sdh;
        C = 2.0f * sdh * cdh;
    }
    B = R.B0 * geo.w;
    D = R.D0 * geo.z;
    frg = geo.y + R.fr_shift;
}

__device__ __forceinline__ void gal_setup(const GalRing &R, const float4 &geo, float &A, float &B, float &C,
                                          float &D, float &frg) {
    const float dl = R.dlat - geo.x;
    if (R.small) {
        const float d2 = dl * dl;
        A = d2 * fmaf(d2, fmaf(d2, 1.0f / 360.0f, -1.0f / 12.0f), 1.0f);
        C = dl * fmaf(d2, fmaf(d2, 1.0f / 120.0f, -1.0f / 6.0f), 1.0f);
    } else {
        float sdh, cdh;
        sincosf(0.5f * dl, &sdh, &cdh);
        A = 4.0f * sdh * sdh;
        C = 2.0f * sdh * cdh;
    }
    B = R.B0 * geo.w;
    D = R.D0 * geo.z;
    frg = geo.y + R.fr_shift;
}

// azimuth difference (rad) of a galaxy (pixel kg, fractional lattice offset
// frg) from a target at lattice position Xi + Xf: the integer part is taken
// exactly first, so the float32 difference keeps full relative precision
__device__ __forceinline__ float gal_u(const GalRing &R, int kg, float frg, int Xi, float Xf) {
    int dk = kg - Xi;
    const int half = R.nr >> 1;
    dk += dk > half ? -R.nr : (dk < -half ? R.nr : 0);
    return ((float)dk + (frg - Xf)) * R.dphi;
}

// one member pair's contribution
template <int KIND>
__device__ __forceinline__ void gal_member(const FilterArgs &f, const GalRing &R, float u, float A, float B, float C,
                                           float D, const float4 &sh, float &pe, float &pb, float &pv, float &pw) {
    float sinu, h;
    if (R.small) sin_hav_small(u, sinu, h);
    else sin_hav_wide(u, sinu, h);
    const float s2 = fmaf(B, h, A);
    const float x = R.mrho0 * sinu;
    const float y = fmaf(D, h, C);
    const float xx = x * x;
    const float sd2 = fmaf(y, y, xx);
    const float cc = fmaf(y, y, -xx);
    const float ss = -2.0f * x * y;
    const float Q = filter_Q<KIND>(f, f.qtab, s2);
    const float w = sd2 > 1e-30f ? __fdividef(Q, sd2) : 0.f;
    pe = fmaf(w, fmaf(sh.x, cc, sh.y * ss), pe);
    pb = fmaf(w, fmaf(sh.y, cc, -sh.x * ss), pb);
    pv = fmaf(Q * Q, sh.w, pv);
    pw += sh.z;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Extra inputs of the barycentre form (Sect. 3.3): the records are bin
// pixels placed at their barycentres; cnt = galaxies of each record's pixel,
// vec = the float64 barycentre (3 per record), raw_m = member records per target.
struct BaryArgs {
    const int32_t *cnt;
    const double *vec;
    int32_t *raw_m;
};

// A pair inside the float32 guard band, set aside for the float64 decision.
struct BandPair {
    int64_t target;     // index into the target list
    int32_t galaxy;     // sorted catalogue position
    int32_t entry;      // ring-pair entry of the target's output ring
};

// azimuth offset of a galaxy from a target in bin pixels; a wide ring pair
// (the union window may span most of the ring) wraps it into [-nr/2, nr/2]
template <int MODE>
__device__ __forceinline__ float gal_du(float Gp, float Tr, const GalRing &R) {
    float d = Gp - Tr;
    if (MODE == 2) {
        const float nr = (float)R.nr, half = 0.5f * (float)R.nr;
        d = d > half ? d - nr : (d < -half ? d + nr : d);
    }
    return d;
}

// great-circle separation^2 from the chord^2 for chords below 0.05 (two
// series terms: truncation below 4e-5 of the next term's 1e-8)
__device__ __forceinline__ float sep2_short(float s2) { return s2 * fmaf(s2, 1.0f / 12.0f, 1.0f); }

// The galaxies of one ring pair's union window for the warp's targets: lanes
// stride over the contiguous galaxy runs; each galaxy record serves every
// target.  The azimuth offset of a galaxy from a target is formed from
// small exact numbers: the galaxy's pixel position within the union window
// (an integer below the window length) plus its offset inside the pixel,
// minus the target's lattice position relative to the window start, so its
// float32 rounding stays below 3e-7 of the window's half width -- far inside
// the guard band.  The per-target body has no branch (non-members add zeros
// through a 0/1 factor); a galaxy whose chord^2 to any target lies inside the
// guard band takes one rare branch to the float64 list.  Targets past the
// group's end sit far away (never members).  MODE picks the series: 0 when
// every |u| and |dl| of the ring pair stays below 0.05 rad and theta_ap
// below 0.03 rad, 1 when they stay below 0.45, 2 beyond.
template <int KIND, int MODE, bool BARY>
__device__ __forceinline__ void gal_segment(const MapArgs &a, const BaryArgs &ba, const RingPair &Rp, const GalRing &R,
                                            int e, int lane, int64_t tb, const float (&Tr)[GT],
                                            const float (&onf)[GT], int lo, int len,
                                            float (&pe)[GT], float (&pb)[GT], float (&pv)[GT], float (&pw)[GT],
                                            float (&nf)[GT], int (&nn)[GT], int (&nm)[GT]) {
    // a generous pre-filter for the guard band; the exact test follows.  The
    // band (8e-6 T) is 67 to 134 float32 ulps of T wide; the pre-filter's
    // half width is a quarter larger than the band's, far above the rounding
    // of Tmid and of |s2 - Tmid| (half an ulp each), so that no pair at an
    // edge of the band slips past both the member test and the band list
    const float Tmid = 0.5f * (a.Tlo + a.Thi), Thw = 0.5f * (a.Thi - a.Tlo) * 1.25f;
    const float qn1 = a.f.qnorm * a.f.inv_ap2, qn2 = qn1 * a.f.inv_ap2;
    const int n1 = min(len, Rp.nr - lo);
#pragma unroll 1
    for (int part = 0; part < 2; ++part) {
        const int pa = part == 0 ? lo : 0;
        const int pn = part == 0 ? n1 : len - n1;
        if (pn <= 0) continue;
        const int g0 = __ldg(a.offsets + R.start + pa);
        const int g1 = __ldg(a.offsets + R.start + pa + pn);
        // union-window position of pixel kg: kg - lo (part 0) or kg + n1 (part 1)
        const int kshift = part == 0 ? -(R.start + lo) : n1 - R.start;
#pragma unroll 1
        for (int g = g0 + lane; g < g1; g += 32) {
            const float4 geo = __ldg(a.geo + g);
            const float4 sh = __ldg(a.shear + g);
            const int krel = (int)__ldg(a.keys + g) + kshift;
            const int cnt = BARY ? __ldg(ba.cnt + g) : 1;
            float A, B, C, D, frg;
            gal_setup_m<MODE>(R, geo, A, B, C, D, frg);
            const float Gp = (float)krel + frg;          // galaxy on the window's lattice
            const float g1x2 = 2.0f * sh.x, g2m2 = -2.0f * sh.y;
            float dmin = 3.0e38f;
#pragma unroll
            for (int r = 0; r < GT; ++r) {
                const float u = gal_du<MODE>(Gp, Tr[r], R) * R.dphi;
                float sinu, h;
                if (MODE == 0) sin_hav_narrow(u, sinu, h);
                else if (MODE == 1) sin_hav_small(u, sinu, h);
                else sin_hav_wide(u, sinu, h);
                const float s2 = fmaf(B, h, A);
                const float m = s2 < a.Tlo ? onf[r] : 0.0f;
                dmin = fminf(dmin, fabsf(s2 - Tmid));
                const float x = R.mrho0 * sinu;
                const float y = fmaf(D, h, C);
                const float xx = x * x;
                const float cc = fmaf(y, y, -xx);
                const float xy = x * y;
                // wq = m Q (m: the 0/1 member factor), w = m Q / sin^2 d; the
                // shear terms take -2xy through the galaxy's (2 g1, -2 g2)
                float w, wq;
                if (KIND == SMART_FILTER_POLY) {
                    // polynomial filter, no division: with t = qnorm/theta^2
                    // (1 - d^2/theta^2), Q = d^2 t and Q / sin^2 d = t d^2 / sin^2 d
                    // = t + Q (1/3 + d^2/15 + 2 d^4/189 + ...); MODE 0 (members
                    // within theta_ap <= 0.03) keeps the first term, the rest
                    // lies below float32 rounding
                    const float d2 = MODE == 0 ? sep2_short(s2) : sep2_from_chord2(s2);
                    const float tm = m * fmaf(d2, -qn2, qn1);
                    wq = d2 * tm;
                    const float F = MODE == 0 ? (1.0f / 3.0f)
                                              : fmaf(d2, fmaf(d2, 2.0f / 189.0f, 1.0f / 15.0f), 1.0f / 3.0f);
                    w = fmaf(wq, F, tm);
                } else {
                    wq = m * filter_Q<KIND>(a.f, a.f.qtab, s2);
                    // sin^2 d = 0 only for a galaxy at the target's centre, where cc = xy = 0
                    w = __fdividef(wq, fmaf(y, y, xx) + 1e-30f);
                }
                pe[r] = fmaf(w, fmaf(sh.x, cc, g2m2 * xy), pe[r]);
                pb[r] = fmaf(w, fmaf(sh.y, cc, g1x2 * xy), pb[r]);
                pv[r] = fmaf(wq * wq, sh.w, pv[r]);           // m Q^2 = (m Q)^2
                pw[r] = fmaf(m, sh.z, pw[r]);
                if (BARY) {
                    nn[r] += m != 0.f ? cnt : 0;
                    nm[r] += m != 0.f ? 1 : 0;
                } else {
                    nf[r] += m;
                }
            }
            if (dmin <= Thw) {         // rare: one branch per galaxy, not per pair
                for (int r = 0; r < GT; ++r) {
                    const float u = gal_du<MODE>(Gp, Tr[r], R) * R.dphi;
                    float sinu, h;
                    if (MODE == 0) sin_hav_narrow(u, sinu, h);
                    else if (MODE == 1) sin_hav_small(u, sinu, h);
                    else sin_hav_wide(u, sinu, h);
                    const float s2 = fmaf(B, h, A);
                    if (onf[r] == 0.0f || s2 < a.Tlo || s2 > a.Thi) continue;
                    const unsigned long long slot = atomicAdd(a.band_count, 1ull);
                    if (slot < (unsigned long long)a.band_cap) {
                        BandPair bp;
                        bp.target = tb + r;
                        bp.galaxy = g;
                        bp.entry = e;
                        reinterpret_cast<BandPair *>(a.band)[slot] = bp;
                    }
                }
            }
        }
    }
}

template <int KIND, bool BARY>
__global__ void __launch_bounds__(32 * GW, 2) k_map_galaxy(const MapArgs a, const BaryArgs ba) {
    const int lane = threadIdx.x & 31;
    const int64_t tile = (int64_t)blockIdx.x * GW + (threadIdx.x >> 5);
    if (tile >= a.n_tiles) return;
    const int64_t tb = a.tiles[tile], te = a.tiles[tile + 1];
    const int nt = (int)(te - tb);
    const TargetRing tr0 = target_ring(a.N0, a.targets[tb]);
    const int64_t ring_start0 = a.targets[tb] - tr0.j0;
    int j0[GT];
    bool on[GT];
    float onf[GT];
    const int jlast = (int)(a.targets[tb + nt - 1] - ring_start0);
#pragma unroll
    for (int r = 0; r < GT; ++r) {
        on[r] = r < nt;
        onf[r] = on[r] ? 1.0f : 0.0f;
        j0[r] = on[r] ? (int)(a.targets[tb + r] - ring_start0) : jlast;
    }
    float SE[GT], SB[GT], SV[GT], SW[GT];
    int NN[GT], NM[GT];
#pragma unroll
    for (int r = 0; r < GT; ++r) {
        SE[r] = SB[r] = SV[r] = SW[r] = 0.f;
        NN[r] = NM[r] = 0;
    }
    const int64_t row0 = (int64_t)(tr0.i0 - 1) * a.kmax;
    const int nent = a.counts[tr0.i0 - 1];
    const LatticeDiv ld = lattice_div(tr0);
    for (int e = 0; e < nent; ++e) {
        const RingPair Rp = a.table[row0 + e];
        const GalRing R = gal_ring(Rp);
        const int q = Rp.nr >> 2;
        // every target's lattice position and window; their union in unwrapped pixels
        int Xi[GT];
        float Xf[GT];
        int ulo = INT32_MAX, uhi = INT32_MIN;
#pragma unroll
        for (int r = 0; r < GT; ++r) {
            TargetRing t = tr0;
            t.j0 = j0[r];
            lattice_position(t, ld, q, Xi[r], Xf[r]);
            if (on[r]) {
                int kl, kh;
                window(Rp, R.fr_shift - Xf[r], kl, kh);
                ulo = min(ulo, Xi[r] + kl);
                uhi = max(uhi, Xi[r] + kh);
            }
        }
        if (uhi - ulo + 1 > Rp.nr) {          // whole ring
            ulo = 0;
            uhi = Rp.nr - 1;
        }
        float pe[GT], pb[GT], pv[GT], pw[GT], nf[GT];
        int nn[GT], nm[GT];
        // targets on the union window's lattice; a slot past the group's end
        // repeats the last target, and its 0/1 factor is 0
        float Tr[GT];
#pragma unroll
        for (int r = 0; r < GT; ++r) {
            pe[r] = pb[r] = pv[r] = pw[r] = nf[r] = 0.f;
            nn[r] = nm[r] = 0;
            Tr[r] = (float)(Xi[r] - ulo) + Xf[r];
        }
        // pixel range [ulo, uhi] -> at most two runs of ring pixels
        // ulo lies in (-nr, 2 nr): one correction brings it into [0, nr)
        const int lo = ulo < 0 ? ulo + Rp.nr : (ulo >= Rp.nr ? ulo - Rp.nr : ulo);
        const int len = uhi - ulo + 1;
        // series by the largest |u| (window plus one pixel) and |dl| (ring
        // offset plus a bin pixel's half extent) of the ring pair
        // (MODE 0 also needs theta_ap <= 0.03 rad: its polynomial-filter weight
        // keeps one term of the d^2 / sin^2 d series, d^4/15 < 6e-8 beyond)
        const int mode = (Rp.flags & RP_WIDE) ? 2
                         : ((float)(len + 2) * Rp.dphi <= 0.05f && fabsf(Rp.dlat) + a.pixrad <= 0.05f &&
                            a.T <= 9e-4) ? 0 : 1;
        if (mode == 0) gal_segment<KIND, 0, BARY>(a, ba, Rp, R, e, lane, tb, Tr, onf, lo, len, pe, pb, pv, pw, nf, nn, nm);
        else if (mode == 1) gal_segment<KIND, 1, BARY>(a, ba, Rp, R, e, lane, tb, Tr, onf, lo, len, pe, pb, pv, pw, nf, nn, nm);
        else gal_segment<KIND, 2, BARY>(a, ba, Rp, R, e, lane, tb, Tr, onf, lo, len, pe, pb, pv, pw, nf, nn, nm);
#pragma unroll
        for (int r = 0; r < GT; ++r) {
            SE[r] += pe[r];
            SB[r] += pb[r];
            SV[r] += pv[r];
            SW[r] += pw[r];
            NN[r] += BARY ? nn[r] : (int)nf[r];
            NM[r] += nm[r];
        }
    }
    // warp reduction of the per-lane sums (per lane: float32 partial sums per
    // ring pair, added to float32 totals);
    // raw sums go to float64 scratch, normalised after the guard-band pairs
#pragma unroll
    for (int r = 0; r < GT; ++r) {
        const float se = warp_sum(SE[r]);
        const float sb = warp_sum(SB[r]);
        const float sv = warp_sum(SV[r]);
        const float sw = warp_sum(SW[r]);
        const int n = warp_sum_i(NN[r]);
        const int m = BARY ? warp_sum_i(NM[r]) : 0;
        if (lane == r && on[r]) {
            double *raw = a.raw + 4 * (tb + r);
            raw[0] = se;
            raw[1] = sb;
            raw[2] = sv;
            raw[3] = sw;
            a.raw_n[tb + r] = n;
            if (BARY) ba.raw_m[tb + r] = m;
        }
    }
}

// the guard-band pairs: float64 decision, then the float32 contribution is
// added to the target's raw sums
template <int KIND, bool BARY>
__global__ void k_galaxy_band(const MapArgs a, const BaryArgs ba) {
    const unsigned long long nall = *a.band_count;
    if (nall > (unsigned long long)a.band_cap && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(a.status, SMART_STATUS_BAND_OVERFLOW);
    const unsigned long long nb = min(nall, (unsigned long long)a.band_cap);
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < nb;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const BandPair bp = reinterpret_cast<const BandPair *>(a.band)[i];
        const int64_t pix = a.targets[bp.target];
        double x0, y0, z0, x1, y1, z1;
        pix2vec64(a.N0, pix, x0, y0, z0);
        if (BARY) {
            x1 = ba.vec[3 * (int64_t)bp.galaxy];
            y1 = ba.vec[3 * (int64_t)bp.galaxy + 1];
            z1 = ba.vec[3 * (int64_t)bp.galaxy + 2];
        } else {
            const double2 rd = a.radec[bp.galaxy];
            radec2vec64(rd.x, rd.y, x1, y1, z1);
        }
        atomicAdd(a.fp64_count, 1ull);
        if (!member64(x0, y0, z0, x1, y1, z1, a.T)) continue;
        const TargetRing tr = target_ring(a.N0, pix);
        const RingPair Rp = a.table[(int64_t)(tr.i0 - 1) * a.kmax + bp.entry];
        const GalRing R = gal_ring(Rp);
        int Xi;
        float Xf;
        lattice_position(tr, Rp.nr >> 2, Xi, Xf);
        const float4 geo = a.geo[bp.galaxy];
        const float4 sh = a.shear[bp.galaxy];
        float A, B, C, D, frg;
        gal_setup(R, geo, A, B, C, D, frg);
        float pe = 0.f, pb = 0.f, pv = 0.f, pw = 0.f;
        gal_member<KIND>(a.f, R, gal_u(R, (int)a.keys[bp.galaxy] - R.start, frg, Xi, Xf), A, B, C, D, sh, pe, pb, pv,
                         pw);
        double *raw = a.raw + 4 * bp.target;
        atomicAdd(raw + 0, (double)pe);
        atomicAdd(raw + 1, (double)pb);
        atomicAdd(raw + 2, (double)pv);
        atomicAdd(raw + 3, (double)pw);
        atomicAdd(a.raw_n + bp.target, BARY ? ba.cnt[bp.galaxy] : 1);
        if (BARY) atomicAdd(ba.raw_m + bp.target, 1);
    }
}

// summed normalisation (Sect. 2.4) from the float64 raw sums
__global__ void k_galaxy_finalise(const MapArgs a, const int32_t *__restrict__ raw_m) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < a.n; t += (int64_t)gridDim.x * blockDim.x) {
        const double *raw = a.raw + 4 * t;
        const int n = a.raw_n[t];
        const double SW = raw[3];
        float me = 0.f, mb = 0.f, vv = 0.f;
        if (SW > 0.0) {
            const float r = (float)a.area / (float)SW;
            me = (float)raw[0] * r;
            mb = (float)raw[1] * r;
            vv = 0.5f * (float)raw[2] * r * r;
        }
        if (a.sum_w) a.sum_w[t] = SW;
        if (a.map_e) a.map_e[t] = me;
        if (a.map_b) a.map_b[t] = mb;
        if (a.var) a.var[t] = vv;
        if (a.count) a.count[t] = n;
        if (a.members) a.members[t] = raw_m ? raw_m[t] : n;
    }
}

}  // namespace smart

using namespace smart;

// ------------------------------------------------------------------------
// barycentre records (Sect. 3.3), built once per catalogue: record r of bin
// pixel p (r = prefix of the non-empty pixels) holds the float64 unit vector
// of the w-weighted mean of the pixel's galaxies (products w r, then a sum
// in catalogue order one addition at a time, then normalised), its float32
// offsets from the pixel centre in the galaxy-record layout, the pixel sums
// and the galaxy count.
// ------------------------------------------------------------------------
__global__ void k_bary_flags(const int32_t *__restrict__ np, int64_t npix, int32_t *__restrict__ flag) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x)
        flag[p] = np[p] > 0 ? 1 : 0;
}

// per pixel with galaxies: its record index, key, count and sums
__global__ void k_bary_keys(int64_t npix, const int32_t *__restrict__ boff, const float4 *__restrict__ px,
                            const int32_t *__restrict__ np, float4 *__restrict__ sh, uint32_t *__restrict__ keys,
                            int32_t *__restrict__ cnt) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
        if (np[p] == 0) continue;
        const int32_t r = boff[p];
        const float4 q = px[p];                        // (G1, G2, S2, W)
        sh[r] = make_float4(q.x, q.y, q.w, q.z);       // record layout (w e1, w e2, w, w^2 |e|^2)
        keys[r] = (uint32_t)p;
        cnt[r] = np[p];
    }
}

// w r of every galaxy (float64, one thread per galaxy)
__global__ void k_bary_wr(int64_t n, const double2 *__restrict__ radec, const float4 *__restrict__ rec_sh,
                          double *__restrict__ wr) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const double2 rd = radec[k];
        double x, y, z;
        radec2vec64(rd.x, rd.y, x, y, z);
        const double w = (double)rec_sh[k].z;
        wr[3 * k] = __dmul_rn(w, x);
        wr[3 * k + 1] = __dmul_rn(w, y);
        wr[3 * k + 2] = __dmul_rn(w, z);
    }
}

// one thread per record: the pixel's w r added in catalogue order (one
// addition at a time), normalised; the unit vector and the float32 offsets
// from the pixel centre are written
__global__ void k_bary_vec(int64_t N, const int32_t *__restrict__ nrec_dev, const uint32_t *__restrict__ keys,
                           const int32_t *__restrict__ off, const double *__restrict__ wr,
                           const double *__restrict__ lat_deg, float4 *__restrict__ geo, double *__restrict__ vec) {
    const int64_t nrec = *nrec_dev;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrec; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = keys[r];
        const int32_t a = off[p], b = off[p + 1];
        double sx = 0.0, sy = 0.0, sz = 0.0;
        for (int32_t k = a; k < b; ++k) {
            sx = __dadd_rn(sx, wr[3 * (int64_t)k]);
            sy = __dadd_rn(sy, wr[3 * (int64_t)k + 1]);
            sz = __dadd_rn(sz, wr[3 * (int64_t)k + 2]);
        }
        const double nrm = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(sx, sx), __dmul_rn(sy, sy)), __dmul_rn(sz, sz)));
        const double vx = __ddiv_rn(sx, nrm), vy = __ddiv_rn(sy, nrm), vz = __ddiv_rn(sz, nrm);
        vec[3 * r] = vx;
        vec[3 * r + 1] = vy;
        vec[3 * r + 2] = vz;
        const double rho = sqrt(vx * vx + vy * vy);
        const double dec = atan2(vz, rho) * (180.0 / SMART_PI);
        const double ra = atan2(vy, vx) * (180.0 / SMART_PI);
        const RingPix rp = pix_to_ring(N, p);
        const double cphi = 90.0 * ring_phi_quarter(N, rp.ring, rp.j);
        double da = fmod(ra - cphi, 360.0);
        if (da > 180.0) da -= 360.0;
        if (da <= -180.0) da += 360.0;
        const RingGeom rg = ring_geom(N, rp.ring);
        geo[r] = make_float4((float)((dec - lat_deg[rp.ring]) * (SMART_PI / 180.0)), (float)(da * (double)rg.nr / 360.0),
                             (float)vz, (float)rho);
    }
}

static smart_status build_barycentres(smart_ctx *c) {
    const int64_t N = c->nside_bin;
    const int64_t npix = npix_of(N);
    cudaStream_t s = c->stream;
    smart_status st = ensure_alloc(c, (void **)&c->bary_off, c->cap_bary_off, npix + 1, sizeof(int32_t), "barycentre offsets");
    if (st != SMART_OK) return st;
    // the non-empty flags go to the count-prefix buffer, which a map binned
    // from the catalogue does not use (its prefix is the catalogue offsets)
    st = ensure_alloc(c, (void **)&c->np_prefix, c->cap_np_prefix, npix + 1, sizeof(int32_t), "count prefix");
    if (st != SMART_OK) return st;
    const unsigned g = (unsigned)std::min<int64_t>((npix + 255) / 256, (int64_t)c->num_sms * 32);
    {
        KernelTimer timer(c, SMART_KT_BARY_BUILD);
        k_bary_flags<<<g, 256, 0, s>>>(c->own_np, npix, c->np_prefix);
        if ((st = check_cuda(c, cudaGetLastError(), "k_bary_flags")) != SMART_OK) return st;
        if ((st = exclusive_scan_i32(c, c->np_prefix, c->bary_off, npix, npix + 1)) != SMART_OK) return st;
    }
    // records: one per pixel holding galaxies, at most one per galaxy; sized
    // by that bound so that the count need not be read back (the kernels
    // take it from bary_off[npix] on the device)
    const int64_t need = std::max<int64_t>(std::min<int64_t>(c->n_gal, npix), 1);
    if (need > c->cap_bary) {
        void **bufs[] = {(void **)&c->bary_geo, (void **)&c->bary_sh, (void **)&c->bary_keys, (void **)&c->bary_cnt,
                         (void **)&c->bary_vec};
        const size_t elem[] = {sizeof(float4), sizeof(float4), sizeof(uint32_t), sizeof(int32_t), 3 * sizeof(double)};
        for (int k = 0; k < 5; ++k) {
            int64_t have = *bufs[k] ? c->cap_bary : 0;
            if ((st = ensure_alloc(c, bufs[k], have, need, elem[k], "barycentre records")) != SMART_OK) {
                c->cap_bary = 0;
                return st;
            }
        }
        c->cap_bary = need;
    }
    c->n_bary = need;          // an upper bound of the records
    if (c->n_gal > 0) {
        // w r of every galaxy: float64 scratch of 24 bytes per galaxy
        st = ensure_alloc(c, (void **)&c->bary_wr, c->cap_bary_wr, 3 * c->n_gal, sizeof(double), "barycentre scratch");
        if (st != SMART_OK) return st;
        KernelTimer timer(c, SMART_KT_BARY_BUILD);
        k_bary_keys<<<g, 256, 0, s>>>(npix, c->bary_off, c->own_px, c->own_np, c->bary_sh, c->bary_keys, c->bary_cnt);
        const unsigned gw = (unsigned)std::min<int64_t>((c->n_gal + 255) / 256, (int64_t)c->num_sms * 32);
        k_bary_wr<<<gw, 256, 0, s>>>(c->n_gal, c->rec_radec, c->rec_shear, c->bary_wr);
        const unsigned gv = (unsigned)std::min<int64_t>((need + 127) / 128, (int64_t)c->num_sms * 32);
        k_bary_vec<<<gv, 128, 0, s>>>(N, c->bary_off + npix, c->bary_keys, c->offsets, c->bary_wr, c->ring_lat,
                                      c->bary_geo, c->bary_vec);
    }
    if ((st = check_cuda(c, cudaGetLastError(), "barycentre records")) != SMART_OK) return st;
    c->bary_version = c->catalog_version;
    return SMART_OK;
}

// brute force over galaxy records, or over barycentre records
static smart_status map_records(smart_ctx *c, const smart_maps *out, bool bary) {
    if (!c->have_catalog)
        return fail(c, SMART_E_STATE, bary ? "smart_map_barycentre: no catalogue (smart_bin_galaxies first)"
                                           : "smart_map_bruteforce: no catalogue (smart_bin_galaxies first)");
    MapArgs a{};
    smart_status st = common_args(c, out, a);
    if (st != SMART_OK) return st;
    if (bary && c->bary_version != c->catalog_version) {
        st = build_barycentres(c);
        if (st != SMART_OK) return st;
    }
    if (!c->rp_gal) {
        // galaxies and barycentres lie within one bin-pixel radius of their pixel centre
        const double th = c->theta_ap + max_pixrad(c->nside_bin) * 1.01 + 1e-9;
        st = build_ring_pairs(c, th, &c->rp_gal, &c->rp_gal_cnt, &c->kmax_gal);
        if (st != SMART_OK) return st;
    }
    if (c->gal_tiles_version != c->targets_version) {
        st = build_tiles_log2(c, GT_LOG2, &c->gal_tiles, &c->cap_gal_tiles, &c->n_gal_tiles);
        if (st != SMART_OK) return st;
        c->gal_tiles_version = c->targets_version;
    }
    const int64_t n = c->n_targets;
    st = ensure_alloc(c, (void **)&c->raw, c->cap_raw, 5 * n + 1, sizeof(double), "raw sums");
    if (st != SMART_OK) return st;
    const int64_t band_cap = std::max<int64_t>(1 << 20, 16 * n);
    st = ensure_alloc(c, (void **)&c->band, c->cap_band, band_cap, sizeof(BandPair), "guard-band list");
    if (st != SMART_OK) return st;
    BaryArgs ba{};
    if (bary) {
        st = ensure_alloc(c, (void **)&c->raw_m, c->cap_raw_m, n + 1, sizeof(int32_t), "member records");
        if (st != SMART_OK) return st;
        ba.cnt = c->bary_cnt;
        ba.vec = c->bary_vec;
        ba.raw_m = c->raw_m;
    }
    a.table = c->rp_gal;
    a.counts = c->rp_gal_cnt;
    a.kmax = c->kmax_gal;
    a.pixrad = (float)(max_pixrad(c->nside_bin) * 1.01);
    a.offsets = bary ? c->bary_off : c->offsets;
    a.geo = bary ? c->bary_geo : c->rec_geo;
    a.shear = bary ? c->bary_sh : c->rec_shear;
    a.radec = bary ? nullptr : c->rec_radec;
    a.keys = bary ? c->bary_keys : c->keys;
    a.tiles = c->gal_tiles;
    a.n_tiles = c->n_gal_tiles;
    a.raw = c->raw;
    a.raw_n = reinterpret_cast<int32_t *>(c->raw + 4 * n);
    a.band = c->band;
    a.band_cap = c->cap_band;
    a.band_count = c->d_band_count;
    cudaMemsetAsync(c->d_fp64_count, 0, sizeof(unsigned long long), c->stream);
    cudaMemsetAsync(c->d_band_count, 0, sizeof(unsigned long long), c->stream);
    if (n == 0) return SMART_OK;
    const bool averaged = c->norm == SMART_NORM_AVERAGED;
    if (averaged) {
        // galaxy records take the W of their bin pixel, pixel records their own
        st = bary ? averaged_record_input(c, c->bary_sh, nullptr, nullptr, c->n_bary, &a.shear)
                  : averaged_record_input(c, c->rec_shear, c->keys, c->own_px, c->n_gal, &a.shear);
        if (st != SMART_OK) return st;
    }
    const unsigned blocks = (unsigned)((a.n_tiles + GW - 1) / GW);
    const bool poly = c->filter_kind == SMART_FILTER_POLY;
    if (bary) {
        KernelTimer timer(c, SMART_KT_BARY_MAP);
        if (poly) k_map_galaxy<SMART_FILTER_POLY, true><<<blocks, 32 * GW, 0, c->stream>>>(a, ba);
        else k_map_galaxy<SMART_FILTER_SCHIRMER, true><<<blocks, 32 * GW, 0, c->stream>>>(a, ba);
    } else {
        KernelTimer timer(c, SMART_KT_GALAXY);
        if (poly) k_map_galaxy<SMART_FILTER_POLY, false><<<blocks, 32 * GW, 0, c->stream>>>(a, ba);
        else k_map_galaxy<SMART_FILTER_SCHIRMER, false><<<blocks, 32 * GW, 0, c->stream>>>(a, ba);
    }
    {
        KernelTimer timer(c, SMART_KT_GALAXY_BAND);
        const unsigned gb = (unsigned)c->num_sms;
        if (bary) {
            if (poly) k_galaxy_band<SMART_FILTER_POLY, true><<<gb, 256, 0, c->stream>>>(a, ba);
            else k_galaxy_band<SMART_FILTER_SCHIRMER, true><<<gb, 256, 0, c->stream>>>(a, ba);
        } else {
            if (poly) k_galaxy_band<SMART_FILTER_POLY, false><<<gb, 256, 0, c->stream>>>(a, ba);
            else k_galaxy_band<SMART_FILTER_SCHIRMER, false><<<gb, 256, 0, c->stream>>>(a, ba);
        }
    }
    const unsigned fb = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)c->num_sms * 16);
    {
        KernelTimer timer(c, SMART_KT_GALAXY_FINALISE);
        k_galaxy_finalise<<<fb, 256, 0, c->stream>>>(a, bary ? c->raw_m : nullptr);
    }
    st = check_cuda(c, cudaGetLastError(), bary ? "barycentre launches" : "brute-force launches");
    if (st == SMART_OK && averaged) st = averaged_rescale(c, out);
    return st;
}

extern "C" smart_status smart_map_bruteforce(smart_ctx *c, const smart_maps *out) {
    if (!c) return SMART_E_ARG;
    return map_records(c, out, false);
}

extern "C" smart_status smart_map_barycentre(smart_ctx *c, const smart_maps *out) {
    if (!c) return SMART_E_ARG;
    return map_records(c, out, true);
}
