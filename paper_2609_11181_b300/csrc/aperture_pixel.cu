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
__device__ __forceinline__ int qbase(int Q) { return Q + 3 * (Q & ~7); }   // tpos(4Q)

// the float64 membership decision for a pair inside the guard band
__device__ __noinline__ bool exact_member(const MapArgs &a, int64_t target_pix, int64_t bin_pix) {
    double x0, y0, z0, x1, y1, z1;
    pix2vec64(a.N0, target_pix, x0, y0, z0);
    pix2vec64(a.N1, bin_pix, x1, y1, z1);
    atomicAdd(a.fp64_count, 1ull);
    return member64(x0, y0, z0, x1, y1, z1, a.T);
}

// pixel-mode general pair loop for one target and one ring pair
template <int KIND>
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
    int kk = (Xi + kl) % R.nr;
    if (kk < 0) kk += R.nr;
    const int mode = (R.flags & RP_WIDE) ? 2 : (((R.hw + 1.0f) * R.dphi <= 0.05f) ? 0 : 1);
    const float u0 = fr * R.dphi;
    float kf = (float)kl;
    for (int k = kl; k <= kh; ++k) {
        const float u = fmaf(kf, R.dphi, u0);
        kf += 1.0f;
        float sinu, h;
        if (mode == 0) sin_hav_narrow(u, sinu, h);
        else if (mode == 1) sin_hav_small(u, sinu, h);
        else sin_hav_wide(u, sinu, h);
        const float s2 = fmaf(R.B, h, R.A);
        const int p = R.start + kk;
        kk = (kk + 1 == R.nr) ? 0 : kk + 1;
        if (s2 > a.Thi) continue;
        if (s2 >= a.Tlo && !exact_member(a, pix, p)) continue;
        const float x = R.mrho0 * sinu;
        const float y = fmaf(R.D, h, R.C);
        const float xx = x * x;
        const float sd2 = fmaf(y, y, xx);
        const float cc = fmaf(y, y, -xx);
        const float ss = -2.0f * x * y;
        const float Q = filter_Q<KIND>(a.f, qtab, s2);
        const float w = sd2 > 1e-30f ? __fdividef(Q, sd2) : 0.f;
        const float g1 = __ldg(a.G1 + p), g2 = __ldg(a.G2 + p);
        pe = fmaf(w, fmaf(g1, cc, g2 * ss), pe);
        pb = fmaf(w, fmaf(g2, cc, -g1 * ss), pb);
        pv = fmaf(Q * Q, __ldg(a.S2 + p), pv);
        pw += __ldg(a.W + p);
        nn += __ldg(a.NP + p);
        nm += 1;
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

template <int KIND>
__global__ void __launch_bounds__(NT, 4) k_map_pixel_tiled(const MapArgs a) {
    __shared__ float4 seg[SEGN];
    __shared__ float4 geo[NCAND];                       // (a, b, -b, c) per candidate offset
    __shared__ float4 qtab[KIND == SMART_FILTER_POLY ? 1 : QTAB_BINS];
    __shared__ int slot_t[TS];
    __shared__ signed char cls[NCAND];
    __shared__ int s_tile, s_da, s_db, s_namb, s_amb[8];
    __shared__ float gpart[4][RB][NT];                  // general-path partial sums per slot
    __shared__ int gcount[2][RB][NT];

    const int tid = threadIdx.x;
    if (KIND != SMART_FILTER_POLY)
        for (int i = tid; i < QTAB_BINS; i += NT) qtab[i] = a.f.qtab[i];

    for (;;) {
        if (tid == 0) s_tile = atomicAdd(a.work, 1);
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= a.n_tiles) break;
        const int64_t tb = a.tiles[tile], te = a.tiles[tile + 1];
        const TargetRing tr0 = target_ring(a.N0, a.targets[tb]);
        const int jbase = tr0.j0 & ~(TS - 1);
        const int nslots = min(TS, tr0.nr0 - jbase);
        const int64_t ring_start0 = a.targets[tb] - tr0.j0;
        for (int s = tid; s < TS; s += NT) slot_t[s] = -1;
        __syncthreads();
        for (int64_t t = tb + tid; t < te; t += NT) slot_t[(int)(a.targets[t] - ring_start0) - jbase] = (int)(t - tb);
        __syncthreads();

        const int s0 = RB * tid;
        int tix[RB];
        bool any = false;
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            tix[r] = (s0 + r < nslots) ? slot_t[s0 + r] : -1;
            any |= tix[r] >= 0;
        }
        float SE[RB], cSE[RB], SB[RB], cSB[RB], SV[RB], cSV[RB], SW[RB], cSW[RB];
        int NN[RB], NM[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            SE[r] = cSE[r] = SB[r] = cSB[r] = SV[r] = cSV[r] = SW[r] = cSW[r] = 0.f;
            NN[r] = NM[r] = 0;
        }

        const RingPair *row = a.table + (int64_t)(tr0.i0 - 1) * a.kmax;
        const int nent = a.counts[tr0.i0 - 1];
        for (int e = 0; e < nent; ++e) {
            const RingPair R = row[e];
            const float off_bin = (R.flags & RP_SHIFTED) ? 0.5f : 0.0f;
            const float fr0 = off_bin - 0.5f * (float)tr0.s0;
            const int dlo = (int)ceilf(-fr0 - R.hw);
            const int dhi = (int)floorf(-fr0 + R.hw);
            const int ncand = dhi - dlo + 1;
            const bool toe = (a.N0 == a.N1) && (R.nr == tr0.nr0) && !(R.flags & RP_WIDE) && ncand >= 1 &&
                             ncand <= NCAND;
            if (toe) {
                // ---- geometry, filter and membership per offset delta
                const bool narrow = (R.hw + 1.0f) * R.dphi <= 0.05f;
                for (int c = tid; c < ncand; c += NT) {
                    const float u = ((float)(dlo + c) + fr0) * R.dphi;
                    float sinu, h;
                    if (narrow) sin_hav_narrow(u, sinu, h);
                    else sin_hav_small(u, sinu, h);
                    const float s2 = fmaf(R.B, h, R.A);
                    const signed char k = s2 < a.Tlo ? 1 : (s2 > a.Thi ? 0 : 2);
                    cls[c] = k;
                    float4 gv = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (k) {
                        const float x = R.mrho0 * sinu;
                        const float y = fmaf(R.D, h, R.C);
                        const float xx = x * x;
                        const float sd2 = fmaf(y, y, xx);
                        const float Q = filter_Q<KIND>(a.f, qtab, s2);
                        const float w = sd2 > 1e-30f ? Q / sd2 : 0.f;
                        const float ga = w * fmaf(y, y, -xx);
                        const float gb = w * (-2.0f * x * y);
                        gv = make_float4(ga, gb, -gb, Q * Q);
                    }
                    geo[c] = gv;
                }
                __syncthreads();
                if (tid == 0) {
                    int da = -1, db = -2, na = 0;
                    for (int c = 0; c < ncand; ++c) {
                        if (cls[c] == 1) {
                            if (da < 0) da = c;
                            db = c;
                        } else if (cls[c] == 2 && na < 8) {
                            s_amb[na++] = c;
                        }
                    }
                    s_da = da;
                    s_db = db;
                    s_namb = na;
                }
                __syncthreads();
                const int da = s_da, L = s_db - s_da + 1;
                if (L > 0) {
                    // ---- stage the bin-ring segment: m -> bin pixel jbase + dlo + da + m
                    const int nseg = min(SEGN, nslots + L + 3);
                    const int k0 = jbase + dlo + da;
                    for (int m = tid; m < nseg; m += NT) {
                        int kk = (k0 + m) % R.nr;
                        if (kk < 0) kk += R.nr;
                        const int p = R.start + kk;
                        seg[tpos(m)] = make_float4(__ldg(a.G1 + p), __ldg(a.G2 + p), __ldg(a.S2 + p), __ldg(a.W + p));
                    }
                    __syncthreads();
                    if (any) {
                        float pe[RB], pb[RB], pv[RB], pw[RB];
#pragma unroll
                        for (int r = 0; r < RB; ++r) pe[r] = pb[r] = pv[r] = pw[r] = 0.f;
                        const float4 *g = geo + da;
                        // slot s0 + r uses staged pixel s0 + r + dd for dd in [0, L)
                        float4 P0 = seg[tpos(s0)], P1 = seg[tpos(s0 + 1)], P2 = seg[tpos(s0 + 2)];
                        const int L4 = L & ~3;
                        for (int dd = 0; dd < L4; dd += 4) {
                            // pixels s0 + dd + 3 .. s0 + dd + 6: quad tid + dd/4 (lane 3), quad + 1 (lanes 0..2)
                            const int Q = tid + (dd >> 2);
                            const int b0 = qbase(Q), b1 = qbase(Q + 1);
                            const float4 P3 = seg[b0 + 24];
                            const float4 P4 = seg[b1];
                            const float4 P5 = seg[b1 + 8];
                            const float4 P6 = seg[b1 + 16];
                            const float4 *gg = g + dd;
#define SMART_ACC(r, P, G)                        \
    pe[r] = fmaf(G.x, P.x, fmaf(G.y, P.y, pe[r])); \
    pb[r] = fmaf(G.x, P.y, fmaf(G.z, P.x, pb[r])); \
    pv[r] = fmaf(G.w, P.z, pv[r]);                 \
    pw[r] += P.w;
                            {
                                const float4 G = gg[0];
                                SMART_ACC(0, P0, G) SMART_ACC(1, P1, G) SMART_ACC(2, P2, G) SMART_ACC(3, P3, G)
                            }
                            {
                                const float4 G = gg[1];
                                SMART_ACC(0, P1, G) SMART_ACC(1, P2, G) SMART_ACC(2, P3, G) SMART_ACC(3, P4, G)
                            }
                            {
                                const float4 G = gg[2];
                                SMART_ACC(0, P2, G) SMART_ACC(1, P3, G) SMART_ACC(2, P4, G) SMART_ACC(3, P5, G)
                            }
                            {
                                const float4 G = gg[3];
                                SMART_ACC(0, P3, G) SMART_ACC(1, P4, G) SMART_ACC(2, P5, G) SMART_ACC(3, P6, G)
                            }
                            P0 = P4;
                            P1 = P5;
                            P2 = P6;
                        }
                        for (int dd = L4; dd < L; ++dd) {
                            const float4 P3 = seg[tpos(s0 + dd + 3)];
                            const float4 G = g[dd];
                            SMART_ACC(0, P0, G) SMART_ACC(1, P1, G) SMART_ACC(2, P2, G) SMART_ACC(3, P3, G)
                            P0 = P1;
                            P1 = P2;
                            P2 = P3;
                        }
#undef SMART_ACC
#pragma unroll
                        for (int r = 0; r < RB; ++r) {
                            if (tix[r] < 0) continue;
                            kahan_add(SE[r], cSE[r], pe[r]);
                            kahan_add(SB[r], cSB[r], pb[r]);
                            kahan_add(SV[r], cSV[r], pv[r]);
                            kahan_add(SW[r], cSW[r], pw[r]);
                            NM[r] += L;
                            NN[r] += ring_range_count(a.NPRE, R.start, R.nr, jbase + s0 + r + dlo + da, L);
                        }
                    }
                }
                // ---- guard-band offsets: decided per target in float64
                const int namb = s_namb;
                if (any && namb > 0) {
                    for (int ia = 0; ia < namb; ++ia) {
                        const int c = s_amb[ia];
                        const float4 G = geo[c];
#pragma unroll
                        for (int r = 0; r < RB; ++r) {
                            if (tix[r] < 0) continue;
                            const int64_t pix = ring_start0 + jbase + s0 + r;
                            int kk = (jbase + s0 + r + dlo + c) % R.nr;
                            if (kk < 0) kk += R.nr;
                            const int p = R.start + kk;
                            if (!exact_member(a, pix, p)) continue;
                            const float g1 = __ldg(a.G1 + p), g2 = __ldg(a.G2 + p);
                            kahan_add(SE[r], cSE[r], fmaf(G.x, g1, G.y * g2));
                            kahan_add(SB[r], cSB[r], fmaf(G.x, g2, G.z * g1));
                            kahan_add(SV[r], cSV[r], G.w * __ldg(a.S2 + p));
                            kahan_add(SW[r], cSW[r], __ldg(a.W + p));
                            NN[r] += __ldg(a.NP + p);
                            NM[r] += 1;
                        }
                    }
                }
                __syncthreads();   // shared tables are rewritten by the next ring pair
            } else if (any) {
                // ---- general path: each target on its own; partial sums go
                // through shared memory so the slot loop needs no register indexing
#pragma unroll 1
                for (int r = 0; r < RB; ++r) {
                    float pe = 0.f, pb = 0.f, pv = 0.f, pw = 0.f;
                    int nn = 0, nm = 0;
                    const int s = s0 + r;
                    if (s < nslots && slot_t[s] >= 0) {
                        TargetRing tr = tr0;
                        tr.j0 = jbase + s;
                        general_segment<KIND>(a, R, tr, ring_start0 + tr.j0, qtab, pe, pb, pv, pw, nn, nm);
                    }
                    gpart[0][r][tid] = pe;
                    gpart[1][r][tid] = pb;
                    gpart[2][r][tid] = pv;
                    gpart[3][r][tid] = pw;
                    gcount[0][r][tid] = nn;
                    gcount[1][r][tid] = nm;
                }
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    kahan_add(SE[r], cSE[r], gpart[0][r][tid]);
                    kahan_add(SB[r], cSB[r], gpart[1][r][tid]);
                    kahan_add(SV[r], cSV[r], gpart[2][r][tid]);
                    kahan_add(SW[r], cSW[r], gpart[3][r][tid]);
                    NN[r] += gcount[0][r][tid];
                    NM[r] += gcount[1][r][tid];
                }
            }
        }
#pragma unroll
        for (int r = 0; r < RB; ++r)
            if (tix[r] >= 0)
                finalise(a, tb + tix[r], SE[r], cSE[r], SB[r], cSB[r], SV[r], cSV[r], SW[r], cSW[r], NN[r], NM[r]);
        __syncthreads();   // slot map and s_tile are rewritten by the next tile
    }
}

// ------------------------------------------------------------------------
// tile list of a sorted target list: a new tile starts where the ring or
// the aligned block of TS azimuth slots changes
// ------------------------------------------------------------------------
__global__ void k_tile_flags(const int64_t *__restrict__ t, int64_t n, int64_t N0, int32_t *__restrict__ flag) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const RingPix a = pix_to_ring(N0, t[k]);
        int f = 1;
        if (k > 0) {
            const RingPix b = pix_to_ring(N0, t[k - 1]);
            f = (a.ring != b.ring) || ((a.j >> TS_LOG2) != (b.j >> TS_LOG2));
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

smart_status build_tiles(smart_ctx *c) {
    const int64_t n = c->n_targets;
    c->n_tiles = 0;
    if (n == 0) return SMART_OK;
    smart_status st = ensure_alloc(c, (void **)&c->tile_flag, c->cap_tile_flag, 2 * n + 1, sizeof(int32_t), "tile flags");
    if (st != SMART_OK) return st;
    int32_t *flag = c->tile_flag, *idx = c->tile_flag + n;
    const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 148 * 32);
    k_tile_flags<<<blocks, 256, 0, c->stream>>>(c->targets, n, c->nside_out, flag);
    st = exclusive_scan_i32(c, flag, idx, n, n);
    if (st != SMART_OK) return st;
    int32_t last[2] = {0, 0};
    cudaMemcpyAsync(&last[0], idx + n - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(&last[1], flag + n - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    st = check_cuda(c, cudaStreamSynchronize(c->stream), "tile count");
    if (st != SMART_OK) return st;
    const int64_t nt = (int64_t)last[0] + last[1];
    st = ensure_alloc(c, (void **)&c->tiles, c->cap_tiles, nt + 1, sizeof(int64_t), "tiles");
    if (st != SMART_OK) return st;
    k_tile_scatter<<<blocks, 256, 0, c->stream>>>(flag, idx, n, c->tiles);
    c->n_tiles = nt;
    return check_cuda(c, cudaGetLastError(), "tile scatter");
}

// ------------------------------------------------------------------------
// Schirmer filter table: cubic Hermite pieces of q(x) on QTAB_BINS bins of
// x in [0, 1], from float64 values and analytic derivatives
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

__global__ void k_filter_table(double xc, float4 *__restrict__ tab) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= QTAB_BINS) return;
    const double h = 1.0 / QTAB_BINS;
    double d0, d1;
    const double q0 = schirmer_q(i * h, xc, &d0);
    const double q1 = schirmer_q((i + 1) * h, xc, &d1);
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
    k_filter_table<<<(QTAB_BINS + 127) / 128, 128, 0, c->stream>>>(c->xc, c->qtab);
    return check_cuda(c, cudaGetLastError(), "k_filter_table");
}

FilterArgs make_filter(const smart_ctx *c) {
    FilterArgs f;
    f.inv_ap = (float)(1.0 / c->theta_ap);
    f.inv_ap2 = (float)(1.0 / (c->theta_ap * c->theta_ap));
    f.qnorm = c->filter_kind == SMART_FILTER_POLY ? (float)(6.0 / SMART_PI / (c->theta_ap * c->theta_ap))
                                                  : (float)(1.0 / (c->theta_ap * c->theta_ap));
    f.inv_xc = (float)(1.0 / c->xc);
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
    if (c->NP == c->own_np && c->have_catalog) {
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
    a.G1 = c->G1;
    a.G2 = c->G2;
    a.W = c->W;
    a.S2 = c->S2;
    a.NP = c->NP;
    a.tiles = c->tiles;
    a.n_tiles = c->n_tiles;
    a.work = c->d_work;
    cudaMemsetAsync(c->d_fp64_count, 0, sizeof(unsigned long long), c->stream);
    cudaMemsetAsync(c->d_work, 0, sizeof(int), c->stream);
    if (a.n == 0) return SMART_OK;
    const int per_sm = 6;
    const unsigned grid = (unsigned)std::min<int64_t>(a.n_tiles, (int64_t)c->num_sms * per_sm);
    if (c->filter_kind == SMART_FILTER_POLY) k_map_pixel_tiled<SMART_FILTER_POLY><<<grid, NT, 0, c->stream>>>(a);
    else k_map_pixel_tiled<SMART_FILTER_SCHIRMER><<<grid, NT, 0, c->stream>>>(a);
    return check_cuda(c, cudaGetLastError(), "k_map_pixel_tiled launch");
}
