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
//    (Schirmer) or in closed form (polynomial).
//
// Sums: float32 within one ring pair, compensated (Kahan) across ring pairs;
// the weight sum goes to float64 for the final normalisation.
#pragma once

#include "aperture_common.cuh"

namespace smart {


constexpr int TS = 512;           // azimuth slots per tile (aligned blocks of a ring)
constexpr int TS_LOG2 = 9;
constexpr int NT = 128;           // threads per CTA
constexpr int RB = 4;             // consecutive slots per thread
constexpr int NCAND = 120;        // longest Toeplitz candidate run kept in shared memory
constexpr int SEGN = TS + NCAND + 8;
static_assert(SEGN % 32 == 0, "staging layout works on blocks of 32");

static_assert(TS == NT * RB, "tile = threads x slots per thread");

// shared-memory position of staged pixel m: 4 x 8 transposition inside each
// block of 32, so that lanes reading m = 4 l + c hit 8 distinct 16-byte
// bank groups in every quarter warp
__device__ __forceinline__ int tpos(int m) { return (m & ~31) | ((m & 3) << 3) | ((m >> 2) & 7); }
__device__ __forceinline__ int tpos_inv(int q) { return (q & ~31) | ((q & 7) << 2) | ((q >> 3) & 3); }
__device__ __forceinline__ int qbase(int Q) { return Q + 3 * (Q & ~7); }   // tpos(4Q)

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

// pixel-mode general pair loop for one target and one ring pair; MODE picks
// the sine series by the largest |u| of the ring pair (0: <= 0.05 rad,
// 1: <= 0.45 rad, 2: |u| <= pi).  Pairs inside the float32 guard band are
// only counted in the loop, which keeps its body free of branches; when
// there are any (rarely), the window is scanned again and they are decided
// in float64 after the loop.
template <int KIND, int MODE>
__device__ __forceinline__ void general_segment(const MapArgs &a, const RingPair &R, const TargetRing &tr,
                                                const LatticeDiv &ld, int64_t pix, const float4 *qtab, float &pe,
                                                float &pb, float &pv, float &pw, int &nn, int &nm) {
    const int q = R.nr >> 2;
    int Xi;
    float Xf;
    lattice_position(tr, ld, q, Xi, Xf);
    const float fr = ((R.flags & RP_SHIFTED) ? 0.5f : 0.0f) - Xf;
    int kl, kh;
    window(R, fr, kl, kh);
    // 0 <= Xi < nr and kl > -nr: one correction brings the start into [0, nr)
    int kk0 = Xi + kl;
    kk0 += kk0 < 0 ? R.nr : (kk0 >= R.nr ? -R.nr : 0);
    const float u0 = fr * R.dphi;
    int nband = 0;          // pairs inside the float32 guard band
    // the window's pixels are [kk0, nr) then [0, rest) when it wraps
    const int len = kh - kl + 1;
    const int n1 = min(len, R.nr - kk0);
#pragma unroll 1
    for (int part = 0; part < 2; ++part) {
        const int cnt = part == 0 ? n1 : len - n1;
        if (cnt <= 0) continue;
        const int pbeg = part == 0 ? R.start + kk0 : R.start;
        const int plast = pbeg + cnt - 1;
        float kf = (float)(part == 0 ? kl : kl + n1);
        // the bin pixel's data is loaded one iteration ahead (the load of the
        // last pixel is repeated, never past the run)
        float4 gn = __ldg(a.PX + pbeg);
        // the strict members of a run are contiguous (s^2 grows with |u|): their
        // number and the last one give the galaxy count from the count prefix
        int nrun = 0, last = -1;
        // branch-free body (non-members add zeros), so that consecutive pairs
        // can interleave; guard-band pairs take the rare branch
#pragma unroll 2
        for (int i = 0; i < cnt; ++i) {
            const int p = pbeg + i;
            const float4 g = gn;
            gn = __ldg(a.PX + min(p + 1, plast));
            const float u = fmaf(kf, R.dphi, u0);
            kf += 1.0f;
            float sinu, h;
            sin_hav<MODE>(u, sinu, h);
            const float s2 = fmaf(R.B, h, R.A);
            const bool in = s2 < a.Tlo;
            nband += (!in && s2 <= a.Thi) ? 1 : 0;
            const float x = R.mrho0 * sinu;
            const float y = fmaf(R.D, h, R.C);
            const float xx = x * x;
            const float sd2 = fmaf(y, y, xx);
            const float cc = fmaf(y, y, -xx);
            const float ss = -2.0f * x * y;
            const float Q = filter_Q<KIND>(a.f, qtab, s2);
            const float w = (in && sd2 > 1e-30f) ? __fdividef(Q, sd2) : 0.f;
            pe = fmaf(w, fmaf(g.x, cc, g.y * ss), pe);
            pb = fmaf(w, fmaf(g.y, cc, -g.x * ss), pb);
            pv = fmaf(in ? Q * Q : 0.f, g.z, pv);
            pw += in ? g.w : 0.f;
            nrun += in ? 1 : 0;
            last = in ? i : last;
        }
        if (nrun > 0) {
            nn += __ldg(a.NPRE + pbeg + last + 1) - __ldg(a.NPRE + pbeg + last + 1 - nrun);
            nm += nrun;
        }
    }
    if (nband > 0) {
        // rare: the guard-band pairs, found again and decided in float64 (u and
        // s^2 are recomputed exactly as in the loop)
        int kk = kk0;
        float kf = (float)kl;
        for (int k = kl; k <= kh; ++k) {
            const float u = fmaf(kf, R.dphi, u0);
            kf += 1.0f;
            float sinu, h;
            sin_hav<MODE>(u, sinu, h);
            const float s2 = fmaf(R.B, h, R.A);
            const int p = R.start + kk;
            kk = (kk + 1 == R.nr) ? 0 : kk + 1;
            if (s2 >= a.Tlo && s2 <= a.Thi && exact_member(a, pix, p))
                pixel_pair<KIND, MODE>(a, R, qtab, u, p, pe, pb, pv, pw, nn, nm);
        }
    }
}

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
// the slots 4 tid .. 4 tid + 3 and slides a window of staged pixels over
// them.  Per ring pair the CTA stages, with cp.async into a double buffer,
// the bin-ring segment the tile needs (16-byte pixels in the transposed
// layout), the per-offset geometry of the ring pair and the prefix counts
// of the segment; ring pair e + 1 is in flight while e is summed.  Tiles
// of other rings are skipped (the general kernel has them).
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

constexpr int PREN = SEGN + 8;
constexpr int PREQ = PREN / 4;        // prefix counts in 4 planes: m -> (m & 3) * PREQ + (m >> 2)
static_assert(PREN % 4 == 0, "prefix planes");

__device__ __forceinline__ int ppos(int m) { return (m & 3) * PREQ + (m >> 2); }

struct ToeStage {
    int start, nr, k0, L, off;
};

// issue the copies of ring pair e of a tile into buffer b
__device__ __forceinline__ ToeStage toe_stage(const MapArgs &a, int64_t row0, int e, int jbase, int nslots,
                                              float4 (*seg)[SEGN], float4 (*geo)[NCAND], int (*pre)[PREN], int b,
                                              int tid) {
    ToeStage t;
    t.start = __ldg(&a.table[row0 + e].start);
    t.nr = __ldg(&a.table[row0 + e].nr);
    const ToeInfo ti = a.toe[row0 + e];
    t.L = ti.L;
    t.off = ti.off;
    t.k0 = jbase + ti.dlo + ti.da;
    if (t.L > 0) {
        const int nseg = min(SEGN, nslots + t.L + 3);
        const int nseg32 = (nseg + 31) & ~31;
        // -nr < k0 + m < 2 nr for every staged m (the window is shorter than the ring)
        for (int q = tid; q < nseg32; q += NT) {        // shared-memory positions in order
            const int m = tpos_inv(q);
            if (m >= nseg) continue;
            int kk = t.k0 + m;
            kk += kk < 0 ? t.nr : (kk >= t.nr ? -t.nr : 0);
            cp_async16(&seg[b][q], a.PX + t.start + kk);
        }
        for (int c = tid; c < t.L; c += NT) cp_async16(&geo[b][c], a.toe_geo + ti.off + ti.da + c);
        const int npre = min(PREN, nslots + t.L + 1);
        for (int m = tid; m < npre; m += NT) {
            int kk = t.k0 + m;
            kk += kk < 0 ? t.nr : (kk >= t.nr ? -t.nr : 0);
            cp_async4(&pre[b][ppos(m)], a.NPRE + t.start + kk);
        }
    }
    cp_async_commit();
    return t;
}

struct ToeShared {
    float4 seg[2][SEGN];
    float4 geo[2][NCAND];
    int pre[2][PREN];
    int slot_t[TS];
};

// one tile of a Toeplitz output ring, summed by the whole CTA (NT threads);
// ends with a barrier, so the shared buffers are free on return
template <int KIND>
__device__ __forceinline__ void toeplitz_tile(const MapArgs &a, int64_t tile, ToeShared &S) {
    auto &seg = S.seg;
    auto &geo = S.geo;
    auto &pre = S.pre;
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
    __syncthreads();
    for (int64_t t = tb + tid; t < te; t += NT) slot_t[(int)(a.targets[t] - ring_start0) - jbase] = (int)(t - tb);

    ToeStage cur = toe_stage(a, row0, 0, jbase, nslots, seg, geo, pre, 0, tid);
    __syncthreads();      // slot map written

    const int s0 = RB * tid;
    int tix[RB];
    bool any = false;
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        tix[r] = (s0 + r < nslots) ? slot_t[s0 + r] : -1;
        any |= tix[r] >= 0;
    }
    float SE[RB], cSE[RB], SB[RB], cSB[RB], SV[RB], SW[RB], cSW[RB];
    int NN[RB], NM[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        SE[r] = cSE[r] = SB[r] = cSB[r] = SV[r] = SW[r] = cSW[r] = 0.f;
        NN[r] = NM[r] = 0;
    }

    for (int e = 0; e < nent; ++e) {
        const int b = e & 1;
        cp_async_wait_all();
        __syncthreads();       // ring pair e staged; everyone is done with buffer b ^ 1
        ToeStage nxt;
        if (e + 1 < nent) nxt = toe_stage(a, row0, e + 1, jbase, nslots, seg, geo, pre, b ^ 1, tid);
        const int L = cur.L;
        if (L > 0 && any) {
            float pe[RB], pb[RB], pv[RB], pw[RB];
#pragma unroll
            for (int r = 0; r < RB; ++r) pe[r] = pb[r] = pv[r] = pw[r] = 0.f;
            const float4 *g = geo[b];
            const float4 *sg = seg[b];
            // slot s0 + r uses staged pixel s0 + r + dd for dd in [0, L)
            float4 P0 = sg[tpos(s0)], P1 = sg[tpos(s0 + 1)], P2 = sg[tpos(s0 + 2)];
            const int L4 = L & ~3;
#define SMART_ACC(r, P, G)                        \
pe[r] = fmaf(G.x, P.x, fmaf(G.y, P.y, pe[r])); \
pb[r] = fmaf(G.x, P.y, fmaf(G.z, P.x, pb[r])); \
pv[r] = fmaf(G.w, P.z, pv[r]);                 \
pw[r] += P.w;
            for (int dd = 0; dd < L4; dd += 4) {
                // pixels s0 + dd + 3 .. s0 + dd + 6: quad tid + dd/4 (lane 3), quad + 1 (lanes 0..2)
                const int Q = tid + (dd >> 2);
                const int b0 = qbase(Q), b1 = qbase(Q + 1);
                {
                    const float4 P3 = sg[b0 + 24];
                    const float4 G = g[dd];
                    SMART_ACC(0, P0, G) SMART_ACC(1, P1, G) SMART_ACC(2, P2, G) SMART_ACC(3, P3, G)
                    P0 = P3;
                }
                {
                    const float4 P4 = sg[b1];
                    const float4 G = g[dd + 1];
                    SMART_ACC(0, P1, G) SMART_ACC(1, P2, G) SMART_ACC(2, P0, G) SMART_ACC(3, P4, G)
                    P1 = P4;
                }
                {
                    const float4 P5 = sg[b1 + 8];
                    const float4 G = g[dd + 2];
                    SMART_ACC(0, P2, G) SMART_ACC(1, P0, G) SMART_ACC(2, P1, G) SMART_ACC(3, P5, G)
                    P2 = P5;
                }
                {
                    const float4 P6 = sg[b1 + 16];
                    const float4 G = g[dd + 3];
                    SMART_ACC(0, P0, G) SMART_ACC(1, P1, G) SMART_ACC(2, P2, G) SMART_ACC(3, P6, G)
                    // window for the next block: pixels s0 + dd + 4, + 5, + 6
                    P0 = P1;
                    P1 = P2;
                    P2 = P6;
                }
            }
            for (int dd = L4; dd < L; ++dd) {
                const float4 P3 = sg[tpos(s0 + dd + 3)];
                const float4 G = g[dd];
                SMART_ACC(0, P0, G) SMART_ACC(1, P1, G) SMART_ACC(2, P2, G) SMART_ACC(3, P3, G)
                P0 = P1;
                P1 = P2;
                P2 = P3;
            }
#undef SMART_ACC
            // galaxies in [k0 + s, k0 + s + L) from the staged prefix, with the
            // ring total added for every pass over the ring's end
            const int ring_tot = __ldg(a.NPRE + cur.start + cur.nr) - __ldg(a.NPRE + cur.start);
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                if (tix[r] < 0) continue;
                kahan_add(SE[r], cSE[r], pe[r]);
                kahan_add(SB[r], cSB[r], pb[r]);
                SV[r] += pv[r];
                kahan_add(SW[r], cSW[r], pw[r]);
                NM[r] += L;
                const int lo = cur.k0 + s0 + r;
                NN[r] += pre[b][ppos(s0 + r + L)] - pre[b][ppos(s0 + r)] +
                         (wraps(lo + L, cur.nr) - wraps(lo, cur.nr)) * ring_tot;
            }
        }
        // ---- guard-band offsets: decided per target in float64
        if (any && cur.off >= 0) {
            const ToeInfo ti = a.toe[row0 + e];
            for (int ia = 0; ia < ti.namb; ++ia) {
                const int c = ia == 0 ? ti.amb0 : (ia == 1 ? ti.amb1 : ti.amb2);
                const float4 G = __ldg(a.toe_geo + ti.off + c);
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    if (tix[r] < 0) continue;
                    const int64_t pix = ring_start0 + jbase + s0 + r;
                    int kk = (jbase + s0 + r + ti.dlo + c) % cur.nr;
                    if (kk < 0) kk += cur.nr;
                    const int p = cur.start + kk;
                    if (!exact_member(a, pix, p)) continue;
                    const float4 px = __ldg(a.PX + p);
                    kahan_add(SE[r], cSE[r], fmaf(G.x, px.x, G.y * px.y));
                    kahan_add(SB[r], cSB[r], fmaf(G.x, px.y, G.z * px.x));
                    SV[r] += G.w * px.z;
                    kahan_add(SW[r], cSW[r], px.w);
                    NN[r] += __ldg(a.NP + p);
                    NM[r] += 1;
                }
            }
        }
        cur = nxt;
    }
    cp_async_wait_all();
#pragma unroll
    for (int r = 0; r < RB; ++r)
        if (tix[r] >= 0)
            finalise(a, tb + tix[r], SE[r], cSE[r], SB[r], cSB[r], SV[r], 0.f, SW[r], cSW[r], NN[r], NM[r]);
    __syncthreads();   // slot map and buffers are rewritten by the next tile
}

// is this tile on an output ring of the Toeplitz kernel?
__device__ __forceinline__ bool toeplitz_tile_wanted(const MapArgs &a, int64_t tile) {
    const TargetRing tr0 = target_ring(a.N0, a.targets[a.tiles[tile]]);
    return a.toe_ring[tr0.i0 - 1] != 0;
}

// one target of a general output ring (one thread)
template <int KIND>
__device__ __forceinline__ void general_target(const MapArgs &a, int64_t t, const float4 *qtab) {
    const int64_t pix = a.targets[t];
    const TargetRing tr = target_ring(a.N0, pix);
    const LatticeDiv ld = lattice_div(tr);
    const int64_t row0 = (int64_t)(tr.i0 - 1) * a.kmax;
    const int nent = a.counts[tr.i0 - 1];
    float SE = 0.f, cSE = 0.f, SB = 0.f, cSB = 0.f, SV = 0.f, SW = 0.f, cSW = 0.f;
    int NN = 0, NM = 0;
    for (int e = 0; e < nent; ++e) {
        const RingPair R = a.table[row0 + e];
        const int mode = (R.flags & RP_WIDE) ? 2 : (((R.hw + 1.0f) * R.dphi <= 0.05f) ? 0 : 1);
        float pe = 0.f, pb = 0.f, pv = 0.f, pw = 0.f;
        int nn = 0, nm = 0;
        if (mode == 0) general_segment<KIND, 0>(a, R, tr, ld, pix, qtab, pe, pb, pv, pw, nn, nm);
        else if (mode == 1) general_segment<KIND, 1>(a, R, tr, ld, pix, qtab, pe, pb, pv, pw, nn, nm);
        else general_segment<KIND, 2>(a, R, tr, ld, pix, qtab, pe, pb, pv, pw, nn, nm);
        kahan_add(SE, cSE, pe);
        kahan_add(SB, cSB, pb);
        SV += pv;
        kahan_add(SW, cSW, pw);
        NN += nn;
        NM += nm;
    }
    finalise(a, t, SE, cSE, SB, cSB, SV, 0.f, SW, cSW, NN, NM);
}

}  // namespace smart
