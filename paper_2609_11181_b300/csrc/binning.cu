// binning.cu -- catalogue partitioning by HEALPix pixel (Sect. 3.4 steps 1-3)
// and per-pixel shear sums (Sect. 3.2 step 2) on the device.
//
//   1. pixel of every galaxy (float64, bit-exact with the definition);
//   2. stable LSD radix sort of (pixel, input index), 8-bit digits;
//   3. offset table = exclusive scan of the per-pixel counts;
//   4. galaxy records permuted into sorted order (float32 offsets from the
//      pixel centre -- latitude in rad, azimuth in pixels of the ring -- for
//      the aperture kernel, float64 ra/dec for exact re-decisions);
//   5. per-pixel sums G1, G2, W, S2 and counts, accumulated in sorted order.
#include <math.h>

#include <algorithm>
#include <mutex>

#include "smart_internal.cuh"

namespace smart {

static constexpr int RADIX_BITS = 8;
static constexpr int RADIX = 1 << RADIX_BITS;
static constexpr int SORT_THREADS = 256;
static constexpr int SORT_ITEMS = 16;
static constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;   // 4096 keys per tile
static constexpr int SORT_WARPS = SORT_THREADS / 32;
static constexpr int SCAN_THREADS = 256;
static constexpr int SCAN_ITEMS = 8;
static constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// ---------------------------------------------------------------- keys
__global__ void k_keys(int64_t N, const double *__restrict__ ra, const double *__restrict__ dec, int64_t n,
                       uint32_t *__restrict__ keys, uint32_t *__restrict__ vals, int *__restrict__ invalid) {
    const int64_t npix = 12 * N * N;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const double a = ra[k], d = dec[k];
        uint32_t key;
        if (isfinite(a) && isfinite(d) && d >= -90.0 && d <= 90.0 && fabs(a) < 1e12) {
            key = (uint32_t)ang2pix64(N, a, d);
        } else {
            key = (uint32_t)npix;             // sentinel bucket after every real pixel
            atomicAdd(invalid, 1);
        }
        keys[k] = key;
        vals[k] = (uint32_t)k;
    }
}

// The same pixel from float32 arithmetic when that decision is certain, else
// -1.  Every floor of the float64 definition (ang2pix64) is taken here on a
// float32 value whose error is bounded: the azimuth in quarter turns t to
// 9e-7 (ra rounded to float32 for |ra| < 720, the reduction to [0, 360) and
// the division), |sin|, |cos| of the latitude to 6e-7 (argument rounding + 2
// ulp of sincosf); hence the equatorial arguments N (1/2 + t) -+ (3/4) N z to
// 2.2e-6 N, the polar t_p N cos(dec) sqrt(3 / (1 + |z|)) and its complement
// to 2.6e-6 N and t i to 1.2e-6 N.  A value nearer an integer than about
// twice its bound, a latitude near |z| = 2/3 or the poles, an azimuth near
// the 0/360 seam or an input outside the plain range returns -1, and the
// float64 definition decides; elsewhere its floors cannot differ.
__device__ __forceinline__ int64_t ang2pix_certain(int64_t N, double ra, double dec) {
    const float raf = (float)ra, df = (float)dec;
    if (!(fabsf(raf) < 720.0f) || !(fabsf(df) < 89.99f)) return -1;        // NaN fails too
    const float af = raf - 360.0f * floorf(raf * (1.0f / 360.0f));
    if (!(af > 1e-3f && af < 359.999f)) return -1;
    const float tt = af * (1.0f / 90.0f);
    float sz, cz;
    sincosf(df * 0.0174532925f, &sz, &cz);
    const float za = fabsf(sz);
    if (fabsf(za - 2.0f / 3.0f) < 4e-6f) return -1;
    const float fN = (float)N;
    if (za < 2.0f / 3.0f) {
        const float tol = 5e-6f * fN;
        const float t1 = fN * (0.5f + tt), t2 = 0.75f * fN * sz;
        const float v1 = t1 - t2, v2 = t1 + t2;
        const float f1 = floorf(v1), f2 = floorf(v2);
        if (v1 - f1 < tol || f1 + 1.0f - v1 < tol || v2 - f2 < tol || f2 + 1.0f - v2 < tol) return -1;
        const int64_t jp = (int64_t)f1, jm = (int64_t)f2;
        const int64_t ir = N + 1 + jp - jm;
        const int64_t kshift = 1 - (ir & 1);
        int64_t ip = (jp + jm - N + kshift + 1) / 2;
        ip = ((ip % (4 * N)) + 4 * N) % (4 * N);
        return 2 * N * (N - 1) + (ir - 1) * 4 * N + ip;
    }
    const float tol = 6e-6f * fN;
    const float tp = tt - floorf(tt);
    const float tmp = fN * cz * sqrtf(3.0f / (1.0f + za));
    const float v1 = tp * tmp, v2 = (1.0f - tp) * tmp;
    const float f1 = floorf(v1), f2 = floorf(v2);
    if (v1 - f1 < tol || f1 + 1.0f - v1 < tol || v2 - f2 < tol || f2 + 1.0f - v2 < tol) return -1;
    const int64_t ir = (int64_t)f1 + (int64_t)f2 + 1;
    const float v3 = tt * (float)ir;
    const float f3 = floorf(v3);
    const float tol3 = 3e-6f * fN;
    if (v3 - f3 < tol3 || f3 + 1.0f - v3 < tol3) return -1;
    int64_t ip = (int64_t)f3;
    ip = ((ip % (4 * ir)) + 4 * ir) % (4 * ir);
    if (sz > 0.0f) return 2 * ir * (ir - 1) + ip;
    return 12 * N * N - 2 * ir * (ir + 1) + ip;
}

// keys of the catalogue: float32 where certain; the rest (with any input
// outside the plain range) are listed, warp-aggregated, for k_keys_fix, which
// checks the input and applies the float64 definition
__global__ void k_keys_fast(int64_t N, const double *__restrict__ ra, const double *__restrict__ dec, int64_t n,
                            uint32_t *__restrict__ keys, uint32_t *__restrict__ vals, uint32_t *__restrict__ defer,
                            unsigned long long *__restrict__ n_defer) {
    const int lane = threadIdx.x & 31;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const double a = ra[k], d = dec[k];
        uint32_t key = 0;
        bool need = false;
        const int64_t p = ang2pix_certain(N, a, d);     // -1 also for inputs outside the plain range
        need = p < 0;
        key = need ? 0u : (uint32_t)p;
        keys[k] = key;
        vals[k] = (uint32_t)k;
        const unsigned act = __activemask();
        const unsigned m = __ballot_sync(act, need);
        if (m) {
            const int leader = __ffs(m) - 1;
            unsigned long long b = 0;
            if (lane == leader) b = atomicAdd(n_defer, (unsigned long long)__popc(m));
            b = __shfl_sync(act, b, leader);
            if (need) defer[b + __popc(m & ((1u << lane) - 1u))] = (uint32_t)k;
        }
    }
}

__global__ void k_keys_fix(int64_t N, const double *__restrict__ ra, const double *__restrict__ dec,
                           uint32_t *__restrict__ keys, const uint32_t *__restrict__ defer,
                           const unsigned long long *__restrict__ n_defer, int *__restrict__ invalid) {
    const unsigned long long nd = *n_defer;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < nd;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t k = defer[i];
        const double a = ra[k], d = dec[k];
        if (isfinite(a) && isfinite(d) && d >= -90.0 && d <= 90.0 && fabs(a) < 1e12) {
            keys[k] = (uint32_t)ang2pix64(N, a, d);
        } else {
            keys[k] = (uint32_t)(12 * N * N);     // sentinel bucket after every real pixel
            atomicAdd(invalid, 1);
        }
    }
}

// ------------------------------------------------------- radix passes
__global__ void __launch_bounds__(SORT_THREADS) k_radix_hist(const uint32_t *__restrict__ keys, int64_t n, int shift,
                                                            int64_t ntiles, uint32_t *__restrict__ hist) {
    __shared__ uint32_t h[RADIX];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * SORT_TILE;
#pragma unroll
    for (int r = 0; r < SORT_ITEMS; ++r) {
        const int64_t i = base + r * SORT_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & (RADIX - 1)], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter.  Warp w of the tile owns the contiguous items
// [w*512, (w+1)*512) and walks them in 16 rounds of 32 consecutive items, so
// the ranking order (warp, round, lane) is the input order.  The tile is
// ordered by digit in shared memory first and leaves in runs of equal
// digits (coalesced stores; 3.3 -> 2.2 ms for the four passes over 5e7 keys).
__global__ void __launch_bounds__(SORT_THREADS) k_radix_scatter(const uint32_t *__restrict__ kin,
                                                               const uint32_t *__restrict__ vin,
                                                               uint32_t *__restrict__ kout,
                                                               uint32_t *__restrict__ vout, int64_t n, int shift,
                                                               int64_t ntiles, const uint32_t *__restrict__ hscan) {
    __shared__ uint32_t wcnt[SORT_WARPS][RADIX];
    __shared__ uint32_t tbase[RADIX];
    __shared__ uint32_t tstart[RADIX];                 // first tile-local position of each digit
    __shared__ uint32_t wsum[SORT_WARPS];
    __shared__ uint32_t skey[SORT_TILE], sval[SORT_TILE];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = lane; d < RADIX; d += 32) wcnt[warp][d] = 0;
    tbase[threadIdx.x] = hscan[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    __syncwarp();
    const int64_t base = (int64_t)blockIdx.x * SORT_TILE + (int64_t)warp * (32 * SORT_ITEMS);
    uint32_t key[SORT_ITEMS], val[SORT_ITEMS], rank[SORT_ITEMS];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < SORT_ITEMS; ++r) {
        const int64_t i = base + r * 32 + lane;
        const bool ok = i < n;
        const unsigned valid = __ballot_sync(0xffffffffu, ok);
        key[r] = ok ? kin[i] : 0u;
        val[r] = ok ? vin[i] : 0u;
        const uint32_t d = (key[r] >> shift) & (RADIX - 1);
        rank[r] = 0;
        if (ok) {
            const unsigned peers = __match_any_sync(valid, d);
            const uint32_t before = wcnt[warp][d];
            rank[r] = before + __popc(peers & lt);
            __syncwarp(valid);
            if ((peers & lt) == 0) wcnt[warp][d] = before + __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    // exclusive prefix over warps for each digit (thread = digit), and the
    // digit's total in this tile
    const int dg = threadIdx.x;
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < SORT_WARPS; ++w) {
        const uint32_t c = wcnt[w][dg];
        wcnt[w][dg] = tot;
        tot += c;
    }
    // exclusive scan of the totals over digits: each digit's tile-local start
    uint32_t x = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t t = lane < SORT_WARPS ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < SORT_WARPS) wsum[lane] = t;
    }
    __syncthreads();
    tstart[dg] = x - tot + (warp > 0 ? wsum[warp - 1] : 0u);
    __syncthreads();
    // the tile sorted by digit in shared memory (stable: the rank order is
    // the input order), then written out in runs of equal digits, so that
    // consecutive threads store to consecutive addresses
#pragma unroll
    for (int r = 0; r < SORT_ITEMS; ++r) {
        const int64_t i = base + r * 32 + lane;
        if (i < n) {
            const uint32_t d = (key[r] >> shift) & (RADIX - 1);
            const uint32_t li = tstart[d] + wcnt[warp][d] + rank[r];
            skey[li] = key[r];
            sval[li] = val[r];
        }
    }
    __syncthreads();
    const int cnt = (int)min((int64_t)SORT_TILE, n - (int64_t)blockIdx.x * SORT_TILE);
    for (int li = threadIdx.x; li < cnt; li += SORT_THREADS) {
        const uint32_t k = skey[li];
        const uint32_t d = (k >> shift) & (RADIX - 1);
        const uint32_t pos = tbase[d] + ((uint32_t)li - tstart[d]);
        kout[pos] = k;
        vout[pos] = sval[li];
    }
}

// ------------------------------------------------------------- scan
// exclusive scan of uint32/int32 counts (totals < 2^31), reduce-then-scan.
// in and out may be the same array (the block sums and the allocation-free
// sort scan in place): every item is read and then written by the same
// thread, so in and out carry no no-alias promise and are read with plain
// loads.
template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tile(const T *in, int64_t n_in, int32_t *out, int64_t n,
                                                           int32_t *__restrict__ sums) {
    static_assert(SCAN_ITEMS == 8, "two 16-byte words per thread");
    __shared__ int32_t ws[SCAN_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    // a thread's 8 items are 32 contiguous bytes: two 16-byte loads and
    // stores when both arrays are 16-byte aligned and the items are all in
    // range (every thread but those of the last tile)
    const bool vec = sizeof(T) == 4 && ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0 &&
                     base + SCAN_ITEMS <= n_in && base + SCAN_ITEMS <= n;
    int32_t v[SCAN_ITEMS];
    if (vec) {
        const int4 p = reinterpret_cast<const int4 *>(in + base)[0];
        const int4 q = reinterpret_cast<const int4 *>(in + base)[1];
        v[0] = p.x; v[1] = p.y; v[2] = p.z; v[3] = p.w;
        v[4] = q.x; v[5] = q.y; v[6] = q.z; v[7] = q.w;
    } else {
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            const int64_t i = base + k;
            v[k] = i < n_in ? (int32_t)in[i] : 0;
        }
    }
    int32_t acc = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) acc += v[k];
    // inclusive scan of per-thread totals across the block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t x = acc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int32_t s = lane < SCAN_THREADS / 32 ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < SCAN_THREADS / 32) ws[lane] = s;
    }
    __syncthreads();
    int32_t run = x - acc + (warp > 0 ? ws[warp - 1] : 0);
    if (vec) {
        int32_t o[SCAN_ITEMS];
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            o[k] = run;
            run += v[k];
        }
        reinterpret_cast<int4 *>(out + base)[0] = make_int4(o[0], o[1], o[2], o[3]);
        reinterpret_cast<int4 *>(out + base)[1] = make_int4(o[4], o[5], o[6], o[7]);
    } else {
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            const int64_t i = base + k;
            if (i < n) out[i] = run;
            run += v[k];
        }
    }
    if (threadIdx.x == SCAN_THREADS - 1 && sums) sums[blockIdx.x] = run;
}

__global__ void k_scan_add(int32_t *__restrict__ out, int64_t n, const int32_t *__restrict__ sums) {
    const int64_t i = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x;
    const int32_t s = sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const int64_t j = i + (int64_t)k * SCAN_THREADS;
        if (j < n) out[j] += s;
    }
}

template <typename T>
static smart_status scan_impl(smart_ctx *ctx, const T *in, int64_t n_in, int32_t *out, int64_t n, int32_t *tmp,
                              int64_t tmp_cap) {
    if (n <= 0) return SMART_OK;
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 1) {
        k_scan_tile<T><<<1, SCAN_THREADS, 0, ctx->stream>>>(in, n_in, out, n, nullptr);
        return check_cuda(ctx, cudaGetLastError(), "scan");
    }
    if (nb + 1 > tmp_cap) return fail(ctx, SMART_E_INTERNAL, "scan scratch too small");
    int32_t *sums = tmp;
    k_scan_tile<T><<<(unsigned)nb, SCAN_THREADS, 0, ctx->stream>>>(in, n_in, out, n, sums);
    smart_status st = check_cuda(ctx, cudaGetLastError(), "scan tiles");
    if (st != SMART_OK) return st;
    st = scan_impl<int32_t>(ctx, sums, nb, sums, nb, tmp + nb, tmp_cap - nb);
    if (st != SMART_OK) return st;
    k_scan_add<<<(unsigned)nb, SCAN_THREADS, 0, ctx->stream>>>(out, n, sums);
    return check_cuda(ctx, cudaGetLastError(), "scan add");
}

static int64_t scan_scratch(int64_t n) {
    int64_t s = 0;
    while (n > SCAN_TILE) {
        n = (n + SCAN_TILE - 1) / SCAN_TILE;
        s += n + 1;
    }
    return s + 1;
}

// ------------------------------------------------ counts and offsets
// keys are sorted: the first element of each run of equal keys measures the
// run and stores its length
__global__ void k_run_counts(const uint32_t *__restrict__ keys, int64_t n, uint32_t npix1,
                             int32_t *__restrict__ counts) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        if (i > 0 && keys[i - 1] == k) continue;
        int64_t j = i + 1;
        while (j < n && keys[j] == k) ++j;
        if (k < npix1) counts[k] = (int32_t)(j - i);
    }
}

// per-ring latitude in degrees (for galaxy offsets from their pixel centre)
__global__ void k_ring_lat(int64_t N, double *__restrict__ lat_deg) {
    const int64_t i = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i > 4 * N - 1) return;
    const RingGeom g = ring_geom(N, i);
    lat_deg[i] = atan2(g.z, g.rho) * (180.0 / SMART_PI);
}

// records in sorted order
__global__ void k_records(int64_t N, const uint32_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                          int64_t n, const double *__restrict__ ra, const double *__restrict__ dec,
                          const float *__restrict__ e1, const float *__restrict__ e2, const float *__restrict__ w,
                          const double *__restrict__ lat_deg, float4 *__restrict__ geo, float4 *__restrict__ sh,
                          double2 *__restrict__ radec) {
    const int64_t npix = 12 * N * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t p = keys[i];
        const uint32_t g = vals[i];
        const double a = ra[g], d = dec[g];
        const float ww = w ? w[g] : 1.0f;
        const float x1 = e1[g], x2 = e2[g];
        float4 gr = make_float4(0.f, 0.f, 0.f, 0.f);
        if ((int64_t)p < npix) {
            const RingPix rp = pix_to_ring(N, p);
            const double cphi = 90.0 * ring_phi_quarter(N, rp.ring, rp.j);   // centre azimuth, degrees
            double da = fmod(a - cphi, 360.0);
            if (da > 180.0) da -= 360.0;
            if (da <= -180.0) da += 360.0;
            const double dd = d - lat_deg[rp.ring];
            float sd, cd;
            sincospif((float)(d / 180.0), &sd, &cd);
            // latitude offset in rad; azimuth offset in pixels of the galaxy's own ring
            const RingGeom rg = ring_geom(N, rp.ring);
            gr = make_float4((float)(dd * (SMART_PI / 180.0)), (float)(da * (double)rg.nr / 360.0), sd, cd);
        }
        geo[i] = gr;
        sh[i] = make_float4(ww * x1, ww * x2, ww, ww * ww * (x1 * x1 + x2 * x2));
        radec[i] = make_double2(a, d);
    }
}

// per-pixel sums in sorted order (one thread per pixel), written as
// (G1, G2, S2, W) float4 plus the count
__global__ void k_pixel_sums(const int32_t *__restrict__ off, int64_t npix, const float4 *__restrict__ sh,
                             float4 *__restrict__ px, int32_t *__restrict__ np) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = off[p], b = off[p + 1];
        float g1 = 0.f, g2 = 0.f, ww = 0.f, s2 = 0.f;
        for (int32_t k = a; k < b; ++k) {
            const float4 v = sh[k];
            g1 += v.x;
            g2 += v.y;
            ww += v.z;
            s2 += v.w;
        }
        px[p] = make_float4(g1, g2, s2, ww);
        np[p] = b - a;
    }
}

// the per-galaxy arrays, grown together (stream-ordered: no host wait)
static smart_status ensure_gal_buffers(smart_ctx *c, int64_t n) {
    if (n <= c->cap_gal && c->keys) return SMART_OK;
    void **bufs[] = {(void **)&c->keys, (void **)&c->keys_alt, (void **)&c->vals, (void **)&c->vals_alt,
                     (void **)&c->rec_geo, (void **)&c->rec_shear, (void **)&c->rec_radec};
    const size_t elem[] = {4, 4, 4, 4, 16, 16, 16};
    const int64_t cap = std::max<int64_t>(n, 1);
    for (int k = 0; k < 7; ++k) {
        int64_t have = *bufs[k] ? c->cap_gal : 0;
        smart_status st = ensure_alloc(c, bufs[k], have, cap, elem[k], "galaxy buffers");
        if (st != SMART_OK) {
            c->cap_gal = 0;
            return st;
        }
    }
    c->cap_gal = cap;
    return SMART_OK;
}

// a galaxy with invalid coordinates was counted: flag the device status
// word, which smart_sync reports (the call itself does not wait)
__global__ void k_flag_invalid(const int *__restrict__ invalid, int *__restrict__ status) {
    if (*invalid > 0) atomicOr(status, SMART_STATUS_INVALID_COORDS);
}

static unsigned grid_for(int64_t n, int threads) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 148 * 32));
}

smart_status exclusive_scan_i32(smart_ctx *ctx, const int32_t *in, int32_t *out, int64_t n_in, int64_t n_out) {
    smart_status st = ensure_alloc(ctx, (void **)&ctx->scan_tmp, ctx->cap_scan, scan_scratch(n_out), sizeof(int64_t), "scan scratch");
    if (st != SMART_OK) return st;
    return scan_impl<int32_t>(ctx, in, n_in, out, n_out, (int32_t *)ctx->scan_tmp, ctx->cap_scan * 2);
}

}  // namespace smart

using namespace smart;

extern "C" smart_status smart_bin_galaxies(smart_ctx *c, const double *ra, const double *dec, const float *e1,
                                           const float *e2, const float *w, int64_t n) {
    if (!c) return SMART_E_ARG;
    if (n < 0 || (n > 0 && (!ra || !dec || !e1 || !e2))) return fail(c, SMART_E_ARG, "smart_bin_galaxies: bad pointer or size");
    if (n >= ((int64_t)1 << 31) - 1) return fail(c, SMART_E_OVERFLOW, "smart_bin_galaxies: more than 2^31-2 galaxies");
    const int64_t N = c->nside_bin;
    const int64_t npix = npix_of(N);
    int bits = 0;
    while (((int64_t)1 << bits) <= npix) ++bits;          // keys go up to npix (sentinel)
    smart_status st = ensure_gal_buffers(c, n);
    if (st != SMART_OK) return st;
    if (!c->offsets) {
        if (cudaMalloc(&c->offsets, (size_t)(npix + 1) * sizeof(int32_t)) != cudaSuccess) return fail(c, SMART_E_NOMEM, "cudaMalloc(offsets) failed");
        if ((st = ensure_own_binned_map(c)) != SMART_OK) return st;
        if (cudaMalloc(&c->ring_lat, (size_t)(4 * N) * sizeof(double)) != cudaSuccess) return fail(c, SMART_E_NOMEM, "cudaMalloc(ring lat) failed");
        if (cudaMalloc(&c->d_invalid, sizeof(int)) != cudaSuccess) return fail(c, SMART_E_NOMEM, "cudaMalloc(flag) failed");
        k_ring_lat<<<(unsigned)((4 * N + 127) / 128), 128, 0, c->stream>>>(N, c->ring_lat);
    }
    const int64_t ntiles = std::max<int64_t>(1, (n + SORT_TILE - 1) / SORT_TILE);
    st = ensure_alloc(c, (void **)&c->hist, c->cap_hist, (int64_t)RADIX * ntiles, sizeof(uint32_t), "radix histogram");
    if (st != SMART_OK) return st;
    st = ensure_alloc(c, (void **)&c->hist_scan, c->cap_hist_scan, (int64_t)RADIX * ntiles, sizeof(int32_t), "radix scan");
    if (st != SMART_OK) return st;
    int32_t *hscan = c->hist_scan;
    const int64_t scan_need = std::max(scan_scratch(npix + 1), scan_scratch((int64_t)RADIX * ntiles));
    st = ensure_alloc(c, (void **)&c->scan_tmp, c->cap_scan, scan_need, sizeof(int64_t), "scan scratch");
    if (st != SMART_OK) return st;

    cudaStream_t s = c->stream;
    cudaMemsetAsync(c->d_invalid, 0, sizeof(int), s);
    if (n > 0) {
        {
            // vals_alt and the radix histogram are free until the radix passes:
            // they hold the galaxies left to float64 and their count
            KernelTimer timer(c, SMART_KT_BIN_KEYS);
            unsigned long long *n_defer = reinterpret_cast<unsigned long long *>(c->hist);
            cudaMemsetAsync(n_defer, 0, sizeof(unsigned long long), s);
            k_keys_fast<<<grid_for(n, 256), 256, 0, s>>>(N, ra, dec, n, c->keys, c->vals, c->vals_alt, n_defer);
            k_keys_fix<<<(unsigned)(c->num_sms * 8), 256, 0, s>>>(N, ra, dec, c->keys, c->vals_alt, n_defer,
                                                                   c->d_invalid);
        }
        if ((st = check_cuda(c, cudaGetLastError(), "k_keys")) != SMART_OK) return st;
        uint32_t *ki = c->keys, *ko = c->keys_alt, *vi = c->vals, *vo = c->vals_alt;
        KernelTimer sort_timer(c, SMART_KT_BIN_SORT);
        for (int shift = 0; shift < bits; shift += RADIX_BITS) {
            k_radix_hist<<<(unsigned)ntiles, SORT_THREADS, 0, s>>>(ki, n, shift, ntiles, c->hist);
            st = scan_impl<uint32_t>(c, c->hist, (int64_t)RADIX * ntiles, hscan, (int64_t)RADIX * ntiles,
                                     (int32_t *)c->scan_tmp, c->cap_scan * 2);
            if (st != SMART_OK) return st;
            k_radix_scatter<<<(unsigned)ntiles, SORT_THREADS, 0, s>>>(ki, vi, ko, vo, n, shift, ntiles, (const uint32_t *)hscan);
            if ((st = check_cuda(c, cudaGetLastError(), "k_radix_scatter")) != SMART_OK) return st;
            std::swap(ki, ko);
            std::swap(vi, vo);
        }
        if (ki != c->keys) {          // keep the sorted arrays in keys/vals
            std::swap(c->keys, c->keys_alt);
            std::swap(c->vals, c->vals_alt);
        }
    }
    // counts per pixel (+ the sentinel bucket at npix), then offsets
    int32_t *counts = c->own_np;     // reused: the per-pixel counts are exactly n_p
    cudaMemsetAsync(counts, 0, (size_t)(npix + 1) * sizeof(int32_t), s);
    if (n > 0) {
        k_run_counts<<<grid_for(n, 256), 256, 0, s>>>(c->keys, n, (uint32_t)npix, counts);
        if ((st = check_cuda(c, cudaGetLastError(), "k_run_counts")) != SMART_OK) return st;
    }
    // offsets[0..npix] = exclusive scan of counts[0..npix] (counts[npix] = 0)
    st = scan_impl<int32_t>(c, counts, npix + 1, c->offsets, npix + 1, (int32_t *)c->scan_tmp, c->cap_scan * 2);
    if (st != SMART_OK) return st;
    if (n > 0) {
        KernelTimer timer(c, SMART_KT_BIN_RECORDS);
        k_records<<<grid_for(n, 256), 256, 0, s>>>(N, c->keys, c->vals, n, ra, dec, e1, e2, w, c->ring_lat,
                                                   c->rec_geo, c->rec_shear, c->rec_radec);
        if ((st = check_cuda(c, cudaGetLastError(), "k_records")) != SMART_OK) return st;
    }
    {
        KernelTimer timer(c, SMART_KT_BIN_PIXEL_SUMS);
        k_pixel_sums<<<grid_for(npix, 256), 256, 0, s>>>(c->offsets, npix, c->rec_shear, c->own_px, c->own_np);
    }
    if ((st = check_cuda(c, cudaGetLastError(), "k_pixel_sums")) != SMART_OK) return st;
    c->PX = c->own_px;
    c->NP = c->own_np;
    c->have_binned = true;
    c->binned_from_catalog = true;
    c->binned_from_runs = false;
    c->have_catalog = true;
    c->n_gal = n;
    c->catalog_version += 1;
    k_flag_invalid<<<1, 1, 0, s>>>(c->d_invalid, c->d_status);
    return check_cuda(c, cudaGetLastError(), "smart_bin_galaxies");
}

__global__ void k_copy_catalog(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ vals, int64_t n,
                               int64_t *__restrict__ perm, int64_t *__restrict__ pix) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (perm) perm[i] = vals[i];
        if (pix) pix[i] = keys[i];
    }
}

__global__ void k_copy_offsets(const int32_t *__restrict__ off, int64_t m, int64_t *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = off[i];
}

extern "C" smart_status smart_get_catalog(smart_ctx *c, int64_t *perm, int64_t *pix, int64_t *offsets) {
    if (!c) return SMART_E_ARG;
    if (!c->have_catalog) return fail(c, SMART_E_STATE, "smart_get_catalog: no catalogue binned");
    const int64_t npix = npix_of(c->nside_bin);
    if ((perm || pix) && c->n_gal > 0)
        k_copy_catalog<<<grid_for(c->n_gal, 256), 256, 0, c->stream>>>(c->keys, c->vals, c->n_gal, perm, pix);
    if (offsets) k_copy_offsets<<<grid_for(npix + 1, 256), 256, 0, c->stream>>>(c->offsets, npix + 1, offsets);
    return check_cuda(c, cudaGetLastError(), "smart_get_catalog");
}

__global__ void k_unpack(const float4 *__restrict__ px, const int32_t *__restrict__ np, int64_t npix,
                         float *__restrict__ G1, float *__restrict__ G2, float *__restrict__ W, float *__restrict__ S2,
                         int32_t *__restrict__ n) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = px[p];
        if (G1) G1[p] = v.x;
        if (G2) G2[p] = v.y;
        if (S2) S2[p] = v.z;
        if (W) W[p] = v.w;
        if (n) n[p] = np[p];
    }
}

extern "C" smart_status smart_get_binned(smart_ctx *c, float *G1, float *G2, float *W, float *S2, int32_t *n_p) {
    if (!c) return SMART_E_ARG;
    if (!c->have_binned) return fail(c, SMART_E_STATE, "smart_get_binned: no binned map");
    const int64_t npix = npix_of(c->nside_bin);
    k_unpack<<<grid_for(npix, 256), 256, 0, c->stream>>>(c->PX, c->NP, npix, G1, G2, W, S2, n_p);
    return check_cuda(c, cudaGetLastError(), "smart_get_binned");
}

// ---------------------------------------------------------------------------
// Catalogue sort that allocates no device memory.
//
// Some callers cannot allocate device memory at the moment they need a sort:
// code that runs while a fixed memory budget is already committed (every
// byte handed out by a pool that may not grow), host threads that must not
// call cudaMalloc/cudaFree because those calls synchronise the whole device,
// and runtimes that forbid allocations inside their own scheduling regions.
// For them the sort below works entirely in the caller's output arrays plus
// one file-scope device scratch array of fixed size, reserved on every GPU
// that loads this library for as long as the process lives.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t NOALLOC_MAX_GALAXIES = int64_t(1) << 20;                  // per call
constexpr int64_t NOALLOC_MAX_TILES = NOALLOC_MAX_GALAXIES / SORT_TILE;    // radix tiles
constexpr int64_t NOALLOC_SCAN_INTS = 512 * 1024;                          // scan block sums
constexpr size_t NOALLOC_KEYS_OFF = 0;
constexpr size_t NOALLOC_VALS_OFF = NOALLOC_KEYS_OFF + sizeof(uint32_t) * NOALLOC_MAX_GALAXIES;
constexpr size_t NOALLOC_HIST_OFF = NOALLOC_VALS_OFF + sizeof(uint32_t) * NOALLOC_MAX_GALAXIES;
constexpr size_t NOALLOC_HSCAN_OFF = NOALLOC_HIST_OFF + sizeof(uint32_t) * RADIX * NOALLOC_MAX_TILES;
constexpr size_t NOALLOC_SCAN_OFF = NOALLOC_HSCAN_OFF + sizeof(int32_t) * RADIX * NOALLOC_MAX_TILES;
constexpr size_t NOALLOC_FLAG_OFF = NOALLOC_SCAN_OFF + sizeof(int32_t) * NOALLOC_SCAN_INTS;
constexpr size_t NOALLOC_BYTES = NOALLOC_FLAG_OFF + 256;

// about 10.5 MB on every device that loads the library
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// device address of the scratch array on each device (host code cannot use
// the symbol itself: on the host it is only a stand-in)
std::mutex g_noalloc_mutex;
unsigned char *g_noalloc_ptr[256] = {nullptr};

smart_status noalloc_scratch(unsigned char **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return SMART_E_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SMART_E_CUDA;
        g_noalloc_ptr[dev] = (unsigned char *)p;
    }
    *out = g_noalloc_ptr[dev];
    return SMART_OK;
}

// exclusive scan with block sums in the scratch array (same kernels as the
// context path)
template <typename T>
smart_status noalloc_scan(const T *in, int64_t n_in, int32_t *out, int64_t n, int32_t *tmp, int64_t tmp_cap,
                          cudaStream_t s) {
    if (n <= 0) return SMART_OK;
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 1) {
        k_scan_tile<T><<<1, SCAN_THREADS, 0, s>>>(in, n_in, out, n, nullptr);
        return cudaGetLastError() == cudaSuccess ? SMART_OK : SMART_E_CUDA;
    }
    if (nb + 1 > tmp_cap) return SMART_E_INTERNAL;     // cannot happen within the stated limits
    k_scan_tile<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n_in, out, n, tmp);
    if (cudaGetLastError() != cudaSuccess) return SMART_E_CUDA;
    const smart_status st = noalloc_scan<int32_t>(tmp, nb, tmp, nb, tmp + nb, tmp_cap - nb, s);
    if (st != SMART_OK) return st;
    k_scan_add<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(out, n, tmp);
    return cudaGetLastError() == cudaSuccess ? SMART_OK : SMART_E_CUDA;
}

}  // namespace

extern "C" smart_status smart_sort_catalog_noalloc(int nside, const double *ra, const double *dec, int64_t n,
                                                   uint32_t *pix, uint32_t *perm, int32_t *offsets,
                                                   void *cuda_stream) {
    if (!(nside >= 1 && nside <= 8192 && (nside & (nside - 1)) == 0)) return SMART_E_ARG;
    if (n < 0 || !offsets || (n > 0 && (!ra || !dec || !pix || !perm))) return SMART_E_ARG;
    if (n > NOALLOC_MAX_GALAXIES) return SMART_E_OVERFLOW;
    unsigned char *scr = nullptr;
    smart_status st = noalloc_scratch(&scr);
    if (st != SMART_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int64_t N = nside;
    const int64_t npix = npix_of(N);
    uint32_t *keys_alt = (uint32_t *)(scr + NOALLOC_KEYS_OFF);
    uint32_t *vals_alt = (uint32_t *)(scr + NOALLOC_VALS_OFF);
    uint32_t *hist = (uint32_t *)(scr + NOALLOC_HIST_OFF);
    int32_t *hscan = (int32_t *)(scr + NOALLOC_HSCAN_OFF);
    int32_t *tmp = (int32_t *)(scr + NOALLOC_SCAN_OFF);
    int *invalid = (int *)(scr + NOALLOC_FLAG_OFF);      // counted but never read; cleared per call
    int bits = 0;
    while (((int64_t)1 << bits) <= npix) ++bits;          // keys go up to npix (sentinel)
    // the per-pixel counts are accumulated in place in offsets and the
    // invalid-coordinate counter in the scratch: both start at zero on every
    // call; every other scratch word is written before it is read
    if (cudaMemsetAsync(offsets, 0, (size_t)(npix + 1) * sizeof(int32_t), s) != cudaSuccess ||
        cudaMemsetAsync(invalid, 0, sizeof(int), s) != cudaSuccess)
        return SMART_E_CUDA;
    if (n > 0) {
        const int64_t ntiles = (n + SORT_TILE - 1) / SORT_TILE;
        k_keys<<<grid_for(n, 256), 256, 0, s>>>(N, ra, dec, n, pix, perm, invalid);
        if (cudaGetLastError() != cudaSuccess) return SMART_E_CUDA;
        uint32_t *ki = pix, *ko = keys_alt, *vi = perm, *vo = vals_alt;
        for (int shift = 0; shift < bits; shift += RADIX_BITS) {
            k_radix_hist<<<(unsigned)ntiles, SORT_THREADS, 0, s>>>(ki, n, shift, ntiles, hist);
            st = noalloc_scan<uint32_t>(hist, RADIX * ntiles, hscan, RADIX * ntiles, tmp, NOALLOC_SCAN_INTS, s);
            if (st != SMART_OK) return st;
            k_radix_scatter<<<(unsigned)ntiles, SORT_THREADS, 0, s>>>(ki, vi, ko, vo, n, shift, ntiles,
                                                                     (const uint32_t *)hscan);
            if (cudaGetLastError() != cudaSuccess) return SMART_E_CUDA;
            std::swap(ki, ko);
            std::swap(vi, vo);
        }
        if (ki != pix) {          // an odd number of passes left the result in the scratch
            if (cudaMemcpyAsync(pix, ki, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
                cudaMemcpyAsync(perm, vi, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                return SMART_E_CUDA;
        }
        k_run_counts<<<grid_for(n, 256), 256, 0, s>>>(pix, n, (uint32_t)npix, offsets);
        if (cudaGetLastError() != cudaSuccess) return SMART_E_CUDA;
    }
    // offsets[0..npix] = exclusive scan of the counts, in place
    return noalloc_scan<int32_t>(offsets, npix + 1, offsets, npix + 1, tmp, NOALLOC_SCAN_INTS, s);
}
