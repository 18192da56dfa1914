// aperture_pixel.cu -- pixel-based aperture mass (Sect. 3.2, summed
// normalisation of Sect. 2.4): setup tables and the single-map launches.
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

#include "aperture_pixel.cuh"

namespace smart {

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

__global__ void k_toe_count(const MapArgs a, int64_t nring, int32_t *__restrict__ cnt, int32_t *__restrict__ cmax) {
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
    if (c > 0) atomicMax(cmax, c);
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
// Toeplitz kernel: persistent CTAs over the tile list; tiles of other
// output rings are skipped (the general kernel has them).
// ------------------------------------------------------------------------
template <int KIND, int NC>
__global__ void __launch_bounds__(NT, toe_ctas_per_sm<NC>()) k_pixel_toeplitz(const MapArgs a) {
    __shared__ __align__(16) ToeShared<NC> S;
    __shared__ int s_tile;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(a.work, 1);
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= a.n_tiles) break;
        const bool want = toeplitz_tile_wanted(a, tile);
        __syncthreads();   // s_tile is read by every thread before it is rewritten
        if (want) toeplitz_tile<KIND, NC>(a, tile, S);
    }
}

// ------------------------------------------------------------------------
// General kernel: one thread per target of the other rings, or per mirror
// pair of them (k_pixel_general_pairs); consecutive threads hold consecutive
// targets, so bin pixels are read coalesced.
// ------------------------------------------------------------------------
template <int KIND>
__global__ void __launch_bounds__(128, 7) k_pixel_general(const __grid_constant__ MapArgs a, const GenBand gb) {
    __shared__ float4 qtab[KIND == SMART_FILTER_POLY ? 1 : QTAB_BINS];
    if (KIND != SMART_FILTER_POLY) {
        for (int i = threadIdx.x; i < QTAB_BINS; i += blockDim.x) qtab[i] = a.f.qtab[i];
        __syncthreads();
    }
    const int64_t idx = a.n_pairs + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= a.n_work) return;
    general_target<KIND>(a, a.gen_work[idx].x, idx, qtab, gb);
}

// the mirror pairs; n_lead unpaired targets (all of them when they are few)
// run first, in the leading threads, so that they finish alongside the pairs
// rather than as a launch of their own after them
template <int KIND>
__global__ void __launch_bounds__(128, GEN_PAIR_CTAS_PER_SM) k_pixel_general_pairs(const __grid_constant__ MapArgs a,
                                                                                  const GenBand gb, int64_t n_lead) {
    __shared__ float4 qtab[KIND == SMART_FILTER_POLY ? 1 : QTAB_BINS];
    if (KIND != SMART_FILTER_POLY) {
        for (int i = threadIdx.x; i < QTAB_BINS; i += blockDim.x) qtab[i] = a.f.qtab[i];
        __syncthreads();
    }
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n_lead) {
        const int64_t idx = a.n_pairs + i;
        general_target<KIND>(a, a.gen_work[idx].x, idx, qtab, gb);
        return;
    }
    const int64_t idx = i - n_lead;
    if (idx >= a.n_pairs) return;
    const int2 w = a.gen_work[idx];
    general_target2<KIND>(a, w.x, w.y, idx, qtab, gb);
}

// the general kernel's targets with guard-band pairs, one thread per slot:
// float64 decisions of those pairs, then normalisation
template <int KIND>
__global__ void k_pixel_band(const MapArgs a, const GenBand gb) {
    __shared__ float4 qtab[KIND == SMART_FILTER_POLY ? 1 : QTAB_BINS];
    if (KIND != SMART_FILTER_POLY) {
        for (int i = threadIdx.x; i < QTAB_BINS; i += blockDim.x) qtab[i] = a.f.qtab[i];
        __syncthreads();
    }
    const unsigned long long n = min(*gb.counts, (unsigned long long)gb.cap_slots);
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const double *raw = gb.raw + 4 * i;
        const int64_t tag = gb.idx[i];
        const int2 w = a.gen_work[tag >> 1];
        band_finish<KIND>(a, (tag & 1) ? w.y : w.x, w.x, qtab, gb.mask[i], raw[0], raw[1], raw[2], raw[3],
                          gb.cnt[2 * i], gb.cnt[2 * i + 1]);
    }
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

// position of p in the ascending list t[0 .. n), or -1
template <typename T>
__device__ __forceinline__ int64_t find_sorted(const T *__restrict__ t, int64_t n, T p) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldg(t + mid) < p) lo = mid + 1;
        else hi = mid;
    }
    return lo < n && __ldg(t + lo) == p ? lo : -1;
}

// One round of mirror pairing of the general targets about the meridian
// m pi/4: a target not paired in an earlier round is paired with its image
// on the same ring (general as well: same ring) when the image is a target
// not paired in an earlier round.  pair[g] = (general-list position of the
// partner, round), or (-1, -1).  The image map is an involution, so within a
// round g and its image decide alike and no third target is involved; a
// partner's entry read during the round is either unset or already (g, round).
__global__ void k_gen_pair_round(const int64_t *__restrict__ targets, int64_t n, int64_t N0,
                                 const int32_t *__restrict__ gen_list, int64_t ng, int m, int round,
                                 int2 *__restrict__ pair) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
        if (pair[g].x >= 0) continue;
        const int64_t pix = __ldg(targets + __ldg(gen_list + g));
        const TargetRing tr = target_ring(N0, pix);
        int j2 = (m * tr.q0 - tr.s0 - tr.j0) % tr.nr0;
        j2 += j2 < 0 ? tr.nr0 : 0;
        if (j2 == tr.j0) continue;                   // on the mirror line itself
        const int64_t t2 = find_sorted<int64_t>(targets, n, pix - tr.j0 + j2);
        if (t2 < 0) continue;
        const int64_t g2 = find_sorted<int32_t>(gen_list, ng, (int32_t)t2);
        if (g2 < 0) continue;
        const int2 q = __ldcg(pair + g2);
        if (q.x >= 0 && q.y != round) continue;
        pair[g] = make_int2((int)g2, round);
    }
}

__global__ void k_gen_work_flags(const int2 *__restrict__ pair, int64_t ng, int32_t *__restrict__ f_pair,
                                 int32_t *__restrict__ f_single) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
        const int p = pair[g].x;
        f_pair[g] = p > g ? 1 : 0;
        f_single[g] = p < 0 ? 1 : 0;
    }
}

// the work list: the pairs (lower position first) in list order, then the
// unpaired targets in list order
__global__ void k_gen_work_scatter(const int2 *__restrict__ pair, const int32_t *__restrict__ gen_list, int64_t ng,
                                   const int32_t *__restrict__ i_pair, const int32_t *__restrict__ i_single,
                                   int64_t n_pairs, int2 *__restrict__ work) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
        const int p = pair[g].x;
        if (p > g) work[i_pair[g]] = make_int2(gen_list[g], gen_list[p]);
        else if (p < 0) work[n_pairs + i_single[g]] = make_int2(gen_list[g], -1);
    }
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
    int32_t *last = reinterpret_cast<int32_t *>(c->host_rb);
    cudaMemcpyAsync(&last[0], idx + n - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(&last[1], flag + n - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    st = wait_stream(c, "tile count");
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

// Jarvis et al. (2004) Gaussian-type filter with scale s (units of theta_ap):
// q = (x/s)^2 exp(-x^2 / (2 s^2)) / (4 pi s^2), and dq/dx
__device__ double jarvis_q(double x, double s, double *dq) {
    const double s2 = s * s;
    const double e = exp(-0.5 * x * x / s2) / (4.0 * SMART_PI * s2);
    *dq = e * (2.0 * x / s2 - x * x * x / (s2 * s2));
    return e * x * x / s2;
}

// Q and dQ/ds at chord s of a tabulated filter (Schirmer or Jarvis)
__device__ double table_Q_of_chord(int kind, double s, double xc, double theta_ap, double *dQ) {
    const double half = 0.5 * s;
    const double d = 2.0 * asin(half);
    const double dd = 1.0 / sqrt(1.0 - half * half);          // d d / d s
    double dq;
    const double q = kind == SMART_FILTER_JARVIS ? jarvis_q(d / theta_ap, xc, &dq) : schirmer_q(d / theta_ap, xc, &dq);
    const double n = 1.0 / (theta_ap * theta_ap);
    *dQ = n * dq * dd / theta_ap;
    return n * q;
}

// Q and dQ/dr at plane distance r (Cartesian estimator: Q of the distance itself)
__device__ double table_Q_of_plane(int kind, double r, double xc, double theta_ap, double *dQ) {
    double dq;
    const double q = kind == SMART_FILTER_JARVIS ? jarvis_q(r / theta_ap, xc, &dq) : schirmer_q(r / theta_ap, xc, &dq);
    const double n = 1.0 / (theta_ap * theta_ap);
    *dQ = n * dq / theta_ap;
    return n * q;
}

// cubic pieces of Q on [0, sap] in QTAB_BINS uniform bins of the chord
// (plane = 0, sap = chord of theta_ap) or of the plane distance (plane = 1,
// sap = theta_ap)
__global__ void k_filter_table(int kind, double xc, double theta_ap, double sap, int plane, float4 *__restrict__ tab) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= QTAB_BINS) return;
    const double h = sap / QTAB_BINS;
    double d0, d1;
    const double q0 = plane ? table_Q_of_plane(kind, i * h, xc, theta_ap, &d0)
                            : table_Q_of_chord(kind, i * h, xc, theta_ap, &d0);
    const double q1 = plane ? table_Q_of_plane(kind, (i + 1) * h, xc, theta_ap, &d1)
                            : table_Q_of_chord(kind, (i + 1) * h, xc, theta_ap, &d1);
    d0 *= h;
    d1 *= h;
    // Hermite cubic on t in [0, 1]: q0 + d0 t + c2 t^2 + c3 t^3
    const double c2 = 3.0 * (q1 - q0) - 2.0 * d0 - d1;
    const double c3 = 2.0 * (q0 - q1) + d0 + d1;
    tab[i] = make_float4((float)q0, (float)d0, (float)c2, (float)c3);
}

smart_status build_filter_table(smart_ctx *c, bool plane, float4 **tab) {
    if (c->filter_kind == SMART_FILTER_POLY || *tab) return SMART_OK;
    if (cudaMalloc(tab, QTAB_BINS * sizeof(float4)) != cudaSuccess) return fail(c, SMART_E_NOMEM, "cudaMalloc(filter table) failed");
    k_filter_table<<<(QTAB_BINS + 127) / 128, 128, 0, c->stream>>>(c->filter_kind, c->xc, c->theta_ap,
                                                                  plane ? c->theta_ap : sqrt(c->T), plane ? 1 : 0,
                                                                  *tab);
    return check_cuda(c, cudaGetLastError(), "k_filter_table");
}

smart_status ensure_filter_table(smart_ctx *c) { return build_filter_table(c, false, &c->qtab); }

// Toeplitz tables for every ring pair of the pixel-mode table (once per context)
static smart_status build_toeplitz(smart_ctx *c, const MapArgs &a) {
    const int64_t nring = 4 * (int64_t)c->nside_out - 1;
    const int64_t nidx = nring * a.kmax;
    int32_t *cnt = nullptr, *off = nullptr, *cmax = nullptr;
    if (cudaMallocAsync(&cnt, (size_t)(2 * nidx + 2) * sizeof(int32_t), c->stream) != cudaSuccess)
        return fail(c, SMART_E_NOMEM, "cudaMallocAsync(toeplitz counts) failed");
    off = cnt + nidx;
    cmax = off + nidx + 1;
    cudaMemsetAsync(cmax, 0, sizeof(int32_t), c->stream);
    k_toe_count<<<(unsigned)((nidx + 255) / 256), 256, 0, c->stream>>>(a, nring, cnt, cmax);
    smart_status st = exclusive_scan_i32(c, cnt, off, nidx, nidx + 1);
    int32_t total = 0;
    if (st == SMART_OK) {
        int32_t *h = reinterpret_cast<int32_t *>(c->host_rb);
        cudaMemcpyAsync(h, off + nidx, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
        cudaMemcpyAsync(h + 1, cmax, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
        st = wait_stream(c, "toeplitz table size");
        total = h[0];
        c->toe_max_run = h[1];
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
    cudaFreeAsync(cnt, c->stream);
    return st;
}

// the general kernel's work list: mirror pairs found in four rounds (the
// meridians 0, pi/2, pi/4, 3 pi/4), then the targets left unpaired
static smart_status build_gen_work(smart_ctx *c, int64_t ng) {
    smart_status st = ensure_alloc(c, (void **)&c->gen_work, c->cap_gen_work, ng, sizeof(int2), "general work list");
    if (st != SMART_OK) return st;
    c->n_work = c->n_work_pairs = 0;
    if (ng == 0) return SMART_OK;
    const size_t words = (size_t)(ng + 1);
    char *scratch = nullptr;
    if (cudaMallocAsync((void **)&scratch, words * (sizeof(int2) + 4 * sizeof(int32_t)), c->stream) != cudaSuccess)
        return fail(c, SMART_E_NOMEM, "cudaMallocAsync(mirror pairs) failed");
    int2 *pair = (int2 *)scratch;
    int32_t *f_pair = (int32_t *)(pair + words), *f_single = f_pair + words, *i_pair = f_single + words,
            *i_single = i_pair + words;
    const unsigned blocks = (unsigned)std::min<int64_t>((ng + 255) / 256, 148 * 32);
    st = check_cuda(c, cudaMemsetAsync(pair, 0xFF, (size_t)ng * sizeof(int2), c->stream), "mirror pairs");
    const int lines[4] = {0, 2, 1, 3};
    for (int r = 0; r < 4 && st == SMART_OK; ++r) {
        k_gen_pair_round<<<blocks, 256, 0, c->stream>>>(c->targets, c->n_targets, c->nside_out, c->gen_list, ng,
                                                         lines[r], r, pair);
        st = check_cuda(c, cudaGetLastError(), "k_gen_pair_round");
    }
    if (st == SMART_OK) {
        k_gen_work_flags<<<blocks, 256, 0, c->stream>>>(pair, ng, f_pair, f_single);
        st = exclusive_scan_i32(c, f_pair, i_pair, ng, ng + 1);
    }
    if (st == SMART_OK) st = exclusive_scan_i32(c, f_single, i_single, ng, ng + 1);
    int32_t *tot = reinterpret_cast<int32_t *>(c->host_rb);
    if (st == SMART_OK) {
        cudaMemcpyAsync(&tot[0], i_pair + ng, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
        cudaMemcpyAsync(&tot[1], i_single + ng, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
        st = wait_stream(c, "general work count");
    }
    if (st == SMART_OK) {
        k_gen_work_scatter<<<blocks, 256, 0, c->stream>>>(pair, c->gen_list, ng, i_pair, i_single, tot[0], c->gen_work);
        st = check_cuda(c, cudaGetLastError(), "general work list");
        c->n_work = (int64_t)tot[0] + tot[1];
        c->n_work_pairs = tot[0];
    }
    cudaFreeAsync(scratch, c->stream);
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
    int32_t *last = reinterpret_cast<int32_t *>(c->host_rb);
    cudaMemcpyAsync(&last[0], idx + n - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(&last[1], flag + n - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    st = wait_stream(c, "general target count");
    if (st != SMART_OK) return st;
    const int64_t ng = (int64_t)last[0] + last[1];
    st = ensure_alloc(c, (void **)&c->gen_list, c->cap_gen_list, ng, sizeof(int32_t), "general target list");
    if (st != SMART_OK) return st;
    k_gen_scatter<<<blocks, 256, 0, c->stream>>>(flag, idx, n, c->gen_list);
    st = check_cuda(c, cudaGetLastError(), "general target list");
    if (st != SMART_OK) return st;
    c->n_gen = ng;
    st = build_gen_work(c, ng);
    if (st != SMART_OK) return st;
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

namespace smart {

// every table of a pixel map (once per context and target set) and the
// launch arguments; the count prefix of a copied binned map is only sized
// here (launch_count_prefix computes it)
smart_status prepare_pixel(smart_ctx *c, const smart_maps *out, MapArgs &a) {
    if (!c->have_binned) return fail(c, SMART_E_STATE, "pixel map: no binned data (smart_bin_galaxies or smart_set_binned first)");
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
        st = ensure_alloc(c, (void **)&c->scan_tmp, c->cap_scan, npix / 1024 + 64, sizeof(int64_t), "scan scratch");
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
    if (a.n > 0 && c->gen_version != c->targets_version) {
        st = build_ring_classes(c, a);
        if (st != SMART_OK) return st;
    }
    a.toe_ring = c->toe_ring;
    a.gen_list = c->gen_list;
    a.n_gen = a.n > 0 ? c->n_gen : 0;
    a.gen_work = c->gen_work;
    a.n_work = a.n > 0 ? c->n_work : 0;
    a.n_pairs = a.n > 0 ? c->n_work_pairs : 0;
    return SMART_OK;
}

smart_status prepare_tables(smart_ctx *c) {
    smart_maps none{};
    MapArgs a{};
    smart_status st = common_args(c, &none, a);
    if (st != SMART_OK) return st;
    // pixel mode: ring pairs and Toeplitz tables (once per context), ring
    // classes and the general kernel's target list (once per target set)
    if (!c->rp_pix && (st = build_ring_pairs(c, c->theta_ap, &c->rp_pix, &c->rp_pix_cnt, &c->kmax_pix)) != SMART_OK)
        return st;
    a.table = c->rp_pix;
    a.counts = c->rp_pix_cnt;
    a.kmax = c->kmax_pix;
    if (!c->toe_info && (st = build_toeplitz(c, a)) != SMART_OK) return st;
    a.toe = c->toe_info;
    a.toe_geo = c->toe_geo;
    if (a.n > 0 && c->gen_version != c->targets_version && (st = build_ring_classes(c, a)) != SMART_OK) return st;
    // brute force and projected maps: ring pairs for theta_ap plus the
    // largest bin-pixel radius (galaxies lie anywhere in their pixel) and
    // groups of targets
    if (!c->rp_gal) {
        const double th = c->theta_ap + max_pixrad(c->nside_bin) * 1.01 + 1e-9;
        if ((st = build_ring_pairs(c, th, &c->rp_gal, &c->rp_gal_cnt, &c->kmax_gal)) != SMART_OK) return st;
    }
    if (c->gal_tiles_version != c->targets_version) {
        if ((st = build_tiles_log2(c, GAL_GROUP_LOG2, &c->gal_tiles, &c->cap_gal_tiles, &c->n_gal_tiles)) != SMART_OK)
            return st;
        c->gal_tiles_version = c->targets_version;
    }
    return SMART_OK;
}

// slots of the general kernel's targets with guard-band pairs (a target
// without a free slot is finished in place); counter reset on the stream
smart_status general_band_buffers(smart_ctx *c, int64_t n_gen, GenBand &gb) {
    const int64_t slots = c->band_slot_limit > 0 ? c->band_slot_limit : gen_band_slots(n_gen);
    smart_status st = ensure_alloc(c, &c->gen_band, c->cap_gen_band, slots, GEN_BAND_SLOT_BYTES, "guard-band slots");
    if (st != SMART_OK) return st;
    st = ensure_alloc(c, (void **)&c->d_gen_count, c->cap_gen_count, 1, sizeof(unsigned long long), "slot counter");
    if (st != SMART_OK) return st;
    gb = gen_band_layout(c->gen_band, slots, c->d_gen_count);
    return check_cuda(c, cudaMemsetAsync(c->d_gen_count, 0, sizeof(unsigned long long), c->stream), "slot counter");
}

smart_status launch_count_prefix(smart_ctx *c) {
    if (c->binned_from_catalog && c->have_catalog) return SMART_OK;
    const int64_t npix = npix_of(c->nside_bin);
    return exclusive_scan_i32(c, c->NP, c->np_prefix, npix, npix + 1);
}

}  // namespace smart

extern "C" smart_status smart_map_pixel(smart_ctx *c, const smart_maps *out) {
    if (!c) return SMART_E_ARG;
    MapArgs a{};
    smart_status st = prepare_pixel(c, out, a);
    if (st != SMART_OK) return st;
    cudaMemsetAsync(c->d_fp64_count, 0, sizeof(unsigned long long), c->stream);
    cudaMemsetAsync(c->d_work, 0, sizeof(int), c->stream);
    st = launch_count_prefix(c);
    if (st != SMART_OK || a.n == 0) return st;
    const bool averaged = c->norm == SMART_NORM_AVERAGED;
    if (averaged && (st = averaged_pixel_input(c, a.PX, &a.PX)) != SMART_OK) return st;
    if (a.n_gen < a.n) {
        // the smaller staging when every Toeplitz run of the tables fits it
        const bool short_runs = c->toe_max_run <= NCAND_SHORT;
        const int cps = short_runs ? toe_ctas_per_sm<NCAND_SHORT>() : toe_ctas_per_sm<NCAND>();
        const unsigned grid = (unsigned)std::min<int64_t>(a.n_tiles, (int64_t)c->num_sms * cps);
        KernelTimer timer(c, SMART_KT_PIXEL_TOEPLITZ);
        const bool poly = c->filter_kind == SMART_FILTER_POLY;
        if (short_runs) {
            if (poly) k_pixel_toeplitz<SMART_FILTER_POLY, NCAND_SHORT><<<grid, NT, 0, c->stream>>>(a);
            else k_pixel_toeplitz<SMART_FILTER_SCHIRMER, NCAND_SHORT><<<grid, NT, 0, c->stream>>>(a);
        } else {
            if (poly) k_pixel_toeplitz<SMART_FILTER_POLY, NCAND><<<grid, NT, 0, c->stream>>>(a);
            else k_pixel_toeplitz<SMART_FILTER_SCHIRMER, NCAND><<<grid, NT, 0, c->stream>>>(a);
        }
        st = check_cuda(c, cudaGetLastError(), "k_pixel_toeplitz launch");
        if (st != SMART_OK) return st;
    }
    if (a.n_gen > 0) {
        GenBand gb{};
        if ((st = general_band_buffers(c, a.n_gen, gb)) != SMART_OK) return st;
        const bool poly = c->filter_kind == SMART_FILTER_POLY;
        {
            KernelTimer timer(c, SMART_KT_PIXEL_GENERAL);
            const int64_t n_single = a.n_work - a.n_pairs, n_lead = gen_lead(a.n_pairs, n_single);
            if (a.n_pairs > 0) {
                const unsigned grid = (unsigned)((a.n_pairs + n_lead + 127) / 128);
                if (poly) k_pixel_general_pairs<SMART_FILTER_POLY><<<grid, 128, 0, c->stream>>>(a, gb, n_lead);
                else k_pixel_general_pairs<SMART_FILTER_SCHIRMER><<<grid, 128, 0, c->stream>>>(a, gb, n_lead);
            }
            if (n_single > n_lead) {
                const unsigned grid = (unsigned)((n_single + 127) / 128);
                if (poly) k_pixel_general<SMART_FILTER_POLY><<<grid, 128, 0, c->stream>>>(a, gb);
                else k_pixel_general<SMART_FILTER_SCHIRMER><<<grid, 128, 0, c->stream>>>(a, gb);
            }
        }
        {
            KernelTimer timer(c, SMART_KT_PIXEL_BAND);
            const unsigned grid = (unsigned)c->num_sms * 4;   // four CTAs per SM (registers allow four)
            if (poly) k_pixel_band<SMART_FILTER_POLY><<<grid, 128, 0, c->stream>>>(a, gb);
            else k_pixel_band<SMART_FILTER_SCHIRMER><<<grid, 128, 0, c->stream>>>(a, gb);
        }
        st = check_cuda(c, cudaGetLastError(), "general kernel launches");
    }
    if (st == SMART_OK && averaged) st = averaged_rescale(c, out);
    return st;
}
