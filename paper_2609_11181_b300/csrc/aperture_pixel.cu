// aperture_pixel.cu -- pixel-based aperture mass (Sect. 3.2, summed
// normalisation of Sect. 2.4) as one persistent, ring-tiled launch.
//
// Work unit: a tile = up to TS consecutive azimuth slots of one output ring
// (targets are RING-sorted, so a tile is a contiguous run of the target
// list).  For each bin ring that can reach the tile (the ring-pair table):
//
//  * Toeplitz path -- the bin ring has as many pixels as the output ring and
//    both grids have the same nside: every pair's geometry depends only on
//    the index offset delta = k - j0.  The CTA evaluates geometry, filter and
//    membership once per delta into a shared table, stages the bin-ring
//    segment the tile needs into shared memory, and each thread slides a
//    window over RB consecutive targets: 4 FMAs + 1 FMA (noise) + 1 add
//    (weight) per pair.
//  * general path (polar rings, unequal rings, unequal nside): per pair
//    geometry from the ring-pair constants, the filter from a shared cubic
//    table (Schirmer) or in closed form (polynomial).
//
// Sums: float32 within one ring pair, compensated (Kahan) across ring pairs;
// the weight sum goes to float64 for the final normalisation.
#include <math.h>

#include <algorithm>

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
__device__ __noinline__ bool exact_member_pix(int64_t N0, int64_t N1, double T, unsigned long long *counter,
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
// set aside (a ring segment crosses the band edge at most twice) and
// decided in float64 after the loop, which keeps the float64 code out of
// the hot loop.
template <int KIND, int MODE>
__device__ __forceinline__ void general_segment(const MapArgs &a, const RingPair &R, const TargetRing &tr,
                                                int64_t pix, const float4 *qtab, float &pe, float &pb, float &pv,
                                                float &pw, int &nn, int &nm) {
    const int q = R.nr >> 2;
    int Xi;
    float Xf;
    lattice_position(tr, q, Xi, Xf);
    const float fr = ((R.flags & RP_SHIFTED) ? 0.5f : 0.0f) - Xf;
    int kl, kh;
    window(R, fr, kl, kh);
    int kk0 = (Xi + kl) % R.nr;
    if (kk0 < 0) kk0 += R.nr;
    const float u0 = fr * R.dphi;
    int def0 = -1, def1 = -1, ndef = 0;
    float ud0 = 0.f, ud1 = 0.f;
    // the window's pixels are [kk0, nr) then [0, rest) when it wraps
    const int len = kh - kl + 1;
    const int n1 = min(len, R.nr - kk0);
#pragma unroll 1
    for (int part = 0; part < 2; ++part) {
        const int cnt = part == 0 ? n1 : len - n1;
        const int pbeg = part == 0 ? R.start + kk0 : R.start;
        float kf = (float)(part == 0 ? kl : kl + n1);
#pragma unroll 1
        for (int i = 0; i < cnt; ++i) {
            const float u = fmaf(kf, R.dphi, u0);
            kf += 1.0f;
            float sinu, h;
            sin_hav<MODE>(u, sinu, h);
            const float s2 = fmaf(R.B, h, R.A);
            const int p = pbeg + i;
            if (s2 >= a.Tlo) {
                if (s2 <= a.Thi) {
                    if (ndef == 0) {
                        def0 = p;
                        ud0 = u;
                    } else {
                        def1 = p;
                        ud1 = u;
                    }
                    ++ndef;
                }
                continue;
            }
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
    }
    if (ndef > 2) {
        // cannot happen for HEALPix spacings; redo the guard-band pairs one by one
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
        return;
    }
    if (ndef >= 1 && exact_member(a, pix, def0)) pixel_pair<KIND, MODE>(a, R, qtab, ud0, def0, pe, pb, pv, pw, nn, nm);
    if (ndef >= 2 && exact_member(a, pix, def1)) pixel_pair<KIND, MODE>(a, R, qtab, ud1, def1, pe, pb, pv, pw, nn, nm);
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
// Toeplitz tables: for every ring pair whose bin ring has as many pixels as
// the output ring (same nside), the pair geometry depends only on the index
// offset delta.  One warp per ring pair evaluates geometry, filter and the
// float32 membership class of every candidate offset once, for all tiles of
// the output ring.
// ------------------------------------------------------------------------
__device__ __forceinline__ bool toe_candidates(int64_t N0, int64_t N1, const RingPair &R, int nr0, int s0, int &dlo,
                                               int &ncand, float &fr0) {
    fr0 = ((R.flags & RP_SHIFTED) ? 0.5f : 0.0f) - 0.5f * (float)s0;
    dlo = (int)ceilf(-fr0 - R.hw);
    const int dhi = (int)floorf(-fr0 + R.hw);
    ncand = dhi - dlo + 1;
    return N0 == N1 && R.nr == nr0 && !(R.flags & RP_WIDE) && ncand >= 1 && ncand <= NCAND;
}

__device__ __forceinline__ void output_ring_shape(int64_t N0, int64_t i0, int &nr0, int &s0) {
    if (i0 < N0) {
        nr0 = (int)(4 * i0);
        s0 = 1;
    } else if (i0 <= 3 * N0) {
        nr0 = (int)(4 * N0);
        s0 = ((i0 - N0) & 1) == 0 ? 1 : 0;
    } else {
        nr0 = (int)(4 * (4 * N0 - i0));
        s0 = 1;
    }
}

__global__ void k_toe_count(const MapArgs a, int64_t nring, int32_t *__restrict__ cnt) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nring * a.kmax) return;
    const int64_t i0 = 1 + idx / a.kmax;
    const int e = (int)(idx % a.kmax);
    int c = 0;
    if (e < a.counts[i0 - 1]) {
        int nr0, s0, dlo, ncand;
        float fr0;
        output_ring_shape(a.N0, i0, nr0, s0);
        if (toe_candidates(a.N0, a.N1, a.table[idx], nr0, s0, dlo, ncand, fr0)) c = ncand;
    }
    cnt[idx] = c;
}

template <int KIND>
__global__ void k_toe_fill(const MapArgs a, int64_t nring, const int32_t *__restrict__ off,
                           ToeInfo *__restrict__ info, float4 *__restrict__ pool) {
    const int64_t idx = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (idx >= nring * a.kmax) return;
    const int64_t i0 = 1 + idx / a.kmax;
    const int e = (int)(idx % a.kmax);
    ToeInfo ti;
    ti.off = -1;
    ti.dlo = ti.da = ti.L = ti.namb = 0;
    ti.amb0 = ti.amb1 = ti.amb2 = 0;
    int nr0, s0, dlo = 0, ncand = 0;
    float fr0 = 0.f;
    output_ring_shape(a.N0, i0, nr0, s0);
    const bool ok = e < a.counts[i0 - 1] && toe_candidates(a.N0, a.N1, a.table[idx], nr0, s0, dlo, ncand, fr0);
    if (ok) {
        const RingPair R = a.table[idx];
        const int base = off[idx];
        const bool narrow = (R.hw + 1.0f) * R.dphi <= 0.05f;
        int da = -1, db = -1, namb = 0, amb[3] = {0, 0, 0};
        for (int c0 = 0; c0 < ncand; c0 += 32) {
            const int c = c0 + lane;
            int k = 0;
            float4 gv = make_float4(0.f, 0.f, 0.f, 0.f);
            if (c < ncand) {
                const float u = ((float)(dlo + c) + fr0) * R.dphi;
                float sinu, h;
                if (narrow) sin_hav_narrow(u, sinu, h);
                else sin_hav_small(u, sinu, h);
                const float s2 = fmaf(R.B, h, R.A);
                k = s2 < a.Tlo ? 1 : (s2 > a.Thi ? 0 : 2);
                if (k) {
                    const float x = R.mrho0 * sinu;
                    const float y = fmaf(R.D, h, R.C);
                    const float xx = x * x;
                    const float sd2 = fmaf(y, y, xx);
                    const float Q = filter_Q<KIND>(a.f, a.f.qtab, s2);
                    const float w = sd2 > 1e-30f ? Q / sd2 : 0.f;
                    const float ga = w * fmaf(y, y, -xx);
                    const float gb = w * (-2.0f * x * y);
                    gv = make_float4(ga, gb, -gb, Q * Q);
                }
                pool[base + c] = gv;
            }
            const unsigned m1 = __ballot_sync(0xffffffffu, k == 1);
            unsigned m2 = __ballot_sync(0xffffffffu, k == 2);
            if (m1) {
                if (da < 0) da = c0 + __ffs(m1) - 1;
                db = c0 + 31 - __clz(m1);
            }
            while (m2) {
                const int b = __ffs(m2) - 1;
                m2 &= m2 - 1;
                if (namb < 3) amb[namb] = c0 + b;
                ++namb;
            }
        }
        if (namb <= 3) {
            ti.off = base;
            ti.dlo = dlo;
            ti.da = da < 0 ? 0 : da;
            ti.L = da < 0 ? 0 : db - da + 1;
            ti.namb = namb;
            ti.amb0 = amb[0];
            ti.amb1 = amb[1];
            ti.amb2 = amb[2];
        }
    }
    if (lane == 0) info[idx] = ti;
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

template <int KIND>
__global__ void __launch_bounds__(NT, 4) k_pixel_toeplitz(const MapArgs a) {
    __shared__ __align__(16) float4 seg[2][SEGN];
    __shared__ __align__(16) float4 geo[2][NCAND];
    __shared__ int pre[2][PREN];
    __shared__ int slot_t[TS];
    __shared__ int s_tile;

    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_tile = atomicAdd(a.work, 1);
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= a.n_tiles) break;
        const int64_t tb = a.tiles[tile], te = a.tiles[tile + 1];
        const TargetRing tr0 = target_ring(a.N0, a.targets[tb]);
        if (!a.toe_ring[tr0.i0 - 1]) {
            __syncthreads();
            continue;
        }
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
        __syncthreads();   // slot map, buffers and s_tile are rewritten by the next tile
    }
}

// ------------------------------------------------------------------------
// General kernel: one thread per target of the other rings; consecutive
// threads hold consecutive targets, so bin pixels are read coalesced.
// ------------------------------------------------------------------------
template <int KIND>
__global__ void __launch_bounds__(128, 6) k_pixel_general(const MapArgs a) {
    __shared__ float4 qtab[KIND == SMART_FILTER_POLY ? 1 : QTAB_BINS];
    if (KIND != SMART_FILTER_POLY) {
        for (int i = threadIdx.x; i < QTAB_BINS; i += blockDim.x) qtab[i] = a.f.qtab[i];
        __syncthreads();
    }
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= a.n_gen) return;
    const int64_t t = a.gen_list[idx];
    const int64_t pix = a.targets[t];
    const TargetRing tr = target_ring(a.N0, pix);
    const int64_t row0 = (int64_t)(tr.i0 - 1) * a.kmax;
    const int nent = a.counts[tr.i0 - 1];
    float SE = 0.f, cSE = 0.f, SB = 0.f, cSB = 0.f, SV = 0.f, SW = 0.f, cSW = 0.f;
    int NN = 0, NM = 0;
    for (int e = 0; e < nent; ++e) {
        const RingPair R = a.table[row0 + e];
        const int mode = (R.flags & RP_WIDE) ? 2 : (((R.hw + 1.0f) * R.dphi <= 0.05f) ? 0 : 1);
        float pe = 0.f, pb = 0.f, pv = 0.f, pw = 0.f;
        int nn = 0, nm = 0;
        if (mode == 0) general_segment<KIND, 0>(a, R, tr, pix, qtab, pe, pb, pv, pw, nn, nm);
        else if (mode == 1) general_segment<KIND, 1>(a, R, tr, pix, qtab, pe, pb, pv, pw, nn, nm);
        else general_segment<KIND, 2>(a, R, tr, pix, qtab, pe, pb, pv, pw, nn, nm);
        kahan_add(SE, cSE, pe);
        kahan_add(SB, cSB, pb);
        SV += pv;
        kahan_add(SW, cSW, pw);
        NN += nn;
        NM += nm;
    }
    finalise(a, t, SE, cSE, SB, cSB, SV, 0.f, SW, cSW, NN, NM);
}

// ------------------------------------------------------------------------
// ring classes and the general kernel's target list (built once per
// target set and table)
// ------------------------------------------------------------------------
__global__ void k_toe_rings(const MapArgs a, int64_t nring, unsigned char *__restrict__ toe_ring) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nring) return;
    const int nent = a.counts[i];
    bool all = nent > 0;
    for (int e = 0; e < nent && all; ++e) all = a.toe[i * a.kmax + e].off >= 0;
    toe_ring[i] = all ? 1 : 0;
}

__global__ void k_gen_flags(const int64_t *__restrict__ t, int64_t n, int64_t N0,
                            const unsigned char *__restrict__ toe_ring, int32_t *__restrict__ flag) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        flag[k] = toe_ring[pix_to_ring(N0, t[k]).ring - 1] ? 0 : 1;
}

__global__ void k_gen_scatter(const int32_t *__restrict__ flag, const int32_t *__restrict__ idx, int64_t n,
                              int32_t *__restrict__ list) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        if (flag[k]) list[idx[k]] = (int32_t)k;
}

// ------------------------------------------------------------------------
// tile list of a sorted target list: a new tile starts where the ring or
// the aligned block of TS azimuth slots changes
// ------------------------------------------------------------------------
__global__ void k_tile_flags(const int64_t *__restrict__ t, int64_t n, int64_t N0, int log2_slots,
                             int32_t *__restrict__ flag) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const RingPix a = pix_to_ring(N0, t[k]);
        int f = 1;
        if (k > 0) {
            const RingPix b = pix_to_ring(N0, t[k - 1]);
            f = (a.ring != b.ring) || ((a.j >> log2_slots) != (b.j >> log2_slots));
        }
        flag[k] = f;
    }
}

__global__ void k_tile_scatter(const int32_t *__restrict__ flag, const int32_t *__restrict__ idx, int64_t n,
                               int64_t *__restrict__ tiles) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        if (flag[k]) tiles[idx[k]] = k;
        if (k == n - 1) tiles[idx[k] + flag[k]] = n;
    }
}

smart_status build_tiles_log2(smart_ctx *c, int log2_slots, int64_t **tiles, int64_t *cap, int64_t *n_tiles) {
    const int64_t n = c->n_targets;
    *n_tiles = 0;
    if (n == 0) return SMART_OK;
    smart_status st = ensure_alloc(c, (void **)&c->tile_flag, c->cap_tile_flag, 2 * n + 1, sizeof(int32_t), "tile flags");
    if (st != SMART_OK) return st;
    int32_t *flag = c->tile_flag, *idx = c->tile_flag + n;
    const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 148 * 32);
    k_tile_flags<<<blocks, 256, 0, c->stream>>>(c->targets, n, c->nside_out, log2_slots, flag);
    st = exclusive_scan_i32(c, flag, idx, n, n);
    if (st != SMART_OK) return st;
    int32_t last[2] = {0, 0};
    cudaMemcpyAsync(&last[0], idx + n - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(&last[1], flag + n - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    st = check_cuda(c, cudaStreamSynchronize(c->stream), "tile count");
    if (st != SMART_OK) return st;
    const int64_t nt = (int64_t)last[0] + last[1];
    st = ensure_alloc(c, (void **)tiles, *cap, nt + 1, sizeof(int64_t), "tiles");
    if (st != SMART_OK) return st;
    k_tile_scatter<<<blocks, 256, 0, c->stream>>>(flag, idx, n, *tiles);
    *n_tiles = nt;
    return check_cuda(c, cudaGetLastError(), "tile scatter");
}

smart_status build_tiles(smart_ctx *c) { return build_tiles_log2(c, TS_LOG2, &c->tiles, &c->cap_tiles, &c->n_tiles); }

// ------------------------------------------------------------------------
// Schirmer filter table: cubic Hermite pieces of Q on QTAB_BINS uniform bins
// of the chord s in [0, s_ap] (s_ap^2 = T), from float64 values and
// analytic derivatives; d = 2 asin(s/2), x = d / theta_ap,
// Q = q(x) / theta_ap^2
// ------------------------------------------------------------------------
__device__ double schirmer_q(double x, double xc, double *dq) {
    const double r = x / xc;
    double th, dth;
    if (r < 1e-4) {
        th = 1.0 - r * r / 3.0;
        dth = -2.0 * r / 3.0 / xc;
    } else {
        const double t = tanh(r);
        th = t / r;
        dth = (r * (1.0 - t * t) - t) / (r * r) / xc;
    }
    const double e1 = exp(6.0 - 150.0 * x), e2 = exp(-47.0 + 50.0 * x);
    const double g = 1.0 / (1.0 + e1 + e2);
    const double dg = -g * g * (-150.0 * e1 + 50.0 * e2);
    *dq = dth * g + th * dg;
    return th * g;
}

// Q and dQ/ds at chord s
__device__ double schirmer_Q_of_chord(double s, double xc, double theta_ap, double *dQ) {
    const double half = 0.5 * s;
    const double d = 2.0 * asin(half);
    const double dd = 1.0 / sqrt(1.0 - half * half);          // d d / d s
    double dq;
    const double q = schirmer_q(d / theta_ap, xc, &dq);
    const double n = 1.0 / (theta_ap * theta_ap);
    *dQ = n * dq * dd / theta_ap;
    return n * q;
}

__global__ void k_filter_table(double xc, double theta_ap, double sap, float4 *__restrict__ tab) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= QTAB_BINS) return;
    const double h = sap / QTAB_BINS;
    double d0, d1;
    const double q0 = schirmer_Q_of_chord(i * h, xc, theta_ap, &d0);
    const double q1 = schirmer_Q_of_chord((i + 1) * h, xc, theta_ap, &d1);
    d0 *= h;
    d1 *= h;
    // Hermite cubic on t in [0, 1]: q0 + d0 t + c2 t^2 + c3 t^3
    const double c2 = 3.0 * (q1 - q0) - 2.0 * d0 - d1;
    const double c3 = 2.0 * (q0 - q1) + d0 + d1;
    tab[i] = make_float4((float)q0, (float)d0, (float)c2, (float)c3);
}

smart_status ensure_filter_table(smart_ctx *c) {
    if (c->filter_kind == SMART_FILTER_POLY || c->qtab) return SMART_OK;
    if (cudaMalloc(&c->qtab, QTAB_BINS * sizeof(float4)) != cudaSuccess) return fail(c, SMART_E_NOMEM, "cudaMalloc(filter table) failed");
    k_filter_table<<<(QTAB_BINS + 127) / 128, 128, 0, c->stream>>>(c->xc, c->theta_ap, sqrt(c->T), c->qtab);
    return check_cuda(c, cudaGetLastError(), "k_filter_table");
}

// Toeplitz tables for every ring pair of the pixel-mode table (once per context)
static smart_status build_toeplitz(smart_ctx *c, const MapArgs &a) {
    const int64_t nring = 4 * (int64_t)c->nside_out - 1;
    const int64_t nidx = nring * a.kmax;
    int32_t *cnt = nullptr, *off = nullptr;
    if (cudaMalloc(&cnt, (size_t)(2 * nidx + 1) * sizeof(int32_t)) != cudaSuccess) return fail(c, SMART_E_NOMEM, "cudaMalloc(toeplitz counts) failed");
    off = cnt + nidx;
    k_toe_count<<<(unsigned)((nidx + 255) / 256), 256, 0, c->stream>>>(a, nring, cnt);
    smart_status st = exclusive_scan_i32(c, cnt, off, nidx, nidx + 1);
    int32_t total = 0;
    if (st == SMART_OK) {
        cudaMemcpyAsync(&total, off + nidx, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
        st = check_cuda(c, cudaStreamSynchronize(c->stream), "toeplitz table size");
    }
    if (st == SMART_OK && cudaMalloc(&c->toe_info, (size_t)nidx * sizeof(ToeInfo)) != cudaSuccess)
        st = fail(c, SMART_E_NOMEM, "cudaMalloc(toeplitz info) failed");
    if (st == SMART_OK && cudaMalloc(&c->toe_geo, (size_t)std::max<int32_t>(total, 1) * sizeof(float4)) != cudaSuccess)
        st = fail(c, SMART_E_NOMEM, "cudaMalloc(toeplitz geometry) failed");
    if (st == SMART_OK) {
        const unsigned blocks = (unsigned)((nidx * 32 + 255) / 256);
        if (c->filter_kind == SMART_FILTER_POLY) k_toe_fill<SMART_FILTER_POLY><<<blocks, 256, 0, c->stream>>>(a, nring, off, c->toe_info, c->toe_geo);
        else k_toe_fill<SMART_FILTER_SCHIRMER><<<blocks, 256, 0, c->stream>>>(a, nring, off, c->toe_info, c->toe_geo);
        st = check_cuda(c, cudaGetLastError(), "k_toe_fill");
    }
    if (st == SMART_OK) st = check_cuda(c, cudaStreamSynchronize(c->stream), "toeplitz build");
    cudaFree(cnt);
    return st;
}

// which output rings go to the Toeplitz kernel, and the list of targets for
// the general kernel (once per target set)
static smart_status build_ring_classes(smart_ctx *c, const MapArgs &a) {
    const int64_t nring = 4 * (int64_t)c->nside_out - 1;
    const int64_t n = c->n_targets;
    smart_status st = SMART_OK;
    if (!c->toe_ring && cudaMalloc(&c->toe_ring, (size_t)nring) != cudaSuccess)
        return fail(c, SMART_E_NOMEM, "cudaMalloc(ring classes) failed");
    k_toe_rings<<<(unsigned)((nring + 127) / 128), 128, 0, c->stream>>>(a, nring, c->toe_ring);
    st = ensure_alloc(c, (void **)&c->tile_flag, c->cap_tile_flag, 2 * n + 1, sizeof(int32_t), "target flags");
    if (st != SMART_OK) return st;
    int32_t *flag = c->tile_flag, *idx = c->tile_flag + n;
    const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 148 * 32);
    k_gen_flags<<<blocks, 256, 0, c->stream>>>(c->targets, n, c->nside_out, c->toe_ring, flag);
    st = exclusive_scan_i32(c, flag, idx, n, n);
    if (st != SMART_OK) return st;
    int32_t last[2] = {0, 0};
    cudaMemcpyAsync(&last[0], idx + n - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(&last[1], flag + n - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    st = check_cuda(c, cudaStreamSynchronize(c->stream), "general target count");
    if (st != SMART_OK) return st;
    const int64_t ng = (int64_t)last[0] + last[1];
    st = ensure_alloc(c, (void **)&c->gen_list, c->cap_gen_list, ng, sizeof(int32_t), "general target list");
    if (st != SMART_OK) return st;
    k_gen_scatter<<<blocks, 256, 0, c->stream>>>(flag, idx, n, c->gen_list);
    st = check_cuda(c, cudaGetLastError(), "general target list");
    if (st != SMART_OK) return st;
    c->n_gen = ng;
    c->gen_version = c->targets_version;
    return SMART_OK;
}

FilterArgs make_filter(const smart_ctx *c) {
    FilterArgs f;
    f.inv_ap = (float)(1.0 / c->theta_ap);
    f.inv_ap2 = (float)(1.0 / (c->theta_ap * c->theta_ap));
    f.qnorm = (float)(6.0 / SMART_PI / (c->theta_ap * c->theta_ap));
    f.tab_scale = (float)(QTAB_BINS / sqrt(c->T));
    f.qtab = c->qtab;
    return f;
}

smart_status common_args(smart_ctx *c, const smart_maps *out, MapArgs &a) {
    if (!out) return fail(c, SMART_E_ARG, "null output struct");
    smart_status st = ensure_filter_table(c);
    if (st != SMART_OK) return st;
    a.targets = c->targets;
    a.n = c->n_targets;
    a.N0 = c->nside_out;
    a.N1 = c->nside_bin;
    a.T = c->T;
    a.area = c->area;
    a.Tlo = (float)(c->T * (1.0 - 4e-6));
    a.Thi = (float)(c->T * (1.0 + 4e-6));
    a.f = make_filter(c);
    a.sum_w = out->sum_w;
    a.map_e = out->map_e;
    a.map_b = out->map_b;
    a.var = out->var;
    a.count = out->count;
    a.members = out->members;
    a.fp64_count = c->d_fp64_count;
    a.status = c->d_status;
    return SMART_OK;
}

}  // namespace smart

using namespace smart;

extern "C" smart_status smart_map_pixel(smart_ctx *c, const smart_maps *out) {
    if (!c) return SMART_E_ARG;
    if (!c->have_binned) return fail(c, SMART_E_STATE, "smart_map_pixel: no binned data (smart_bin_galaxies or smart_set_binned first)");
    MapArgs a{};
    smart_status st = common_args(c, out, a);
    if (st != SMART_OK) return st;
    if (!c->rp_pix) {
        st = build_ring_pairs(c, c->theta_ap, &c->rp_pix, &c->rp_pix_cnt, &c->kmax_pix);
        if (st != SMART_OK) return st;
    }
    const int64_t npix = npix_of(c->nside_bin);
    if (c->binned_from_catalog && c->have_catalog) {
        a.NPRE = c->offsets;                 // the catalogue offsets are the count prefix
    } else {
        st = ensure_alloc(c, (void **)&c->np_prefix, c->cap_np_prefix, npix + 1, sizeof(int32_t), "count prefix");
        if (st != SMART_OK) return st;
        st = exclusive_scan_i32(c, c->NP, c->np_prefix, npix, npix + 1);
        if (st != SMART_OK) return st;
        a.NPRE = c->np_prefix;
    }
    a.table = c->rp_pix;
    a.counts = c->rp_pix_cnt;
    a.kmax = c->kmax_pix;
    if (!c->toe_info) {
        st = build_toeplitz(c, a);
        if (st != SMART_OK) return st;
    }
    a.toe = c->toe_info;
    a.toe_geo = c->toe_geo;
    a.PX = c->PX;
    a.NP = c->NP;
    a.tiles = c->tiles;
    a.n_tiles = c->n_tiles;
    a.work = c->d_work;
    cudaMemsetAsync(c->d_fp64_count, 0, sizeof(unsigned long long), c->stream);
    cudaMemsetAsync(c->d_work, 0, sizeof(int), c->stream);
    if (a.n == 0) return SMART_OK;
    if (c->gen_version != c->targets_version) {
        st = build_ring_classes(c, a);
        if (st != SMART_OK) return st;
    }
    a.toe_ring = c->toe_ring;
    a.gen_list = c->gen_list;
    a.n_gen = c->n_gen;
    if (c->n_gen < a.n) {
        const unsigned grid = (unsigned)std::min<int64_t>(a.n_tiles, (int64_t)c->num_sms * 4);
        if (c->filter_kind == SMART_FILTER_POLY) k_pixel_toeplitz<SMART_FILTER_POLY><<<grid, NT, 0, c->stream>>>(a);
        else k_pixel_toeplitz<SMART_FILTER_SCHIRMER><<<grid, NT, 0, c->stream>>>(a);
        st = check_cuda(c, cudaGetLastError(), "k_pixel_toeplitz launch");
        if (st != SMART_OK) return st;
    }
    if (c->n_gen > 0) {
        const unsigned grid = (unsigned)((c->n_gen + 127) / 128);
        if (c->filter_kind == SMART_FILTER_POLY) k_pixel_general<SMART_FILTER_POLY><<<grid, 128, 0, c->stream>>>(a);
        else k_pixel_general<SMART_FILTER_SCHIRMER><<<grid, 128, 0, c->stream>>>(a);
        st = check_cuda(c, cudaGetLastError(), "k_pixel_general launch");
    }
    return st;
}
