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

constexpr int GT = 4;              // targets per warp
constexpr int GW = 8;              // warps per CTA
constexpr int GT_LOG2 = 2;

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
// bin-ring lattice minus its pixel index kg
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

// A pair inside the float32 guard band, set aside for the float64 decision.
struct BandPair {
    int64_t target;     // index into the target list
    int32_t galaxy;     // sorted catalogue position
    int32_t entry;      // ring-pair entry of the target's output ring
};

// The galaxies of one ring pair's union window for the warp's targets: lanes
// stride over the contiguous galaxy runs; each galaxy record serves every
// target.  The per-target body has no branch on membership (non-members add
// zeros), so the GT independent chains can interleave; guard-band pairs take
// a rare branch to the float64 list.
template <int KIND, bool SMALL>
__device__ __forceinline__ void gal_segment(const MapArgs &a, const RingPair &Rp, const GalRing &R, int e, int lane,
                                            int64_t tb, const bool (&on)[GT], const int (&Xi)[GT],
                                            const float (&Xf)[GT], int lo, int len, float (&pe)[GT], float (&pb)[GT],
                                            float (&pv)[GT], float (&pw)[GT], int (&nn)[GT]) {
    const int n1 = min(len, Rp.nr - lo);
#pragma unroll 1
    for (int part = 0; part < 2; ++part) {
        const int pa = part == 0 ? lo : 0;
        const int pn = part == 0 ? n1 : len - n1;
        if (pn <= 0) continue;
        const int g0 = __ldg(a.offsets + R.start + pa);
        const int g1 = __ldg(a.offsets + R.start + pa + pn);
#pragma unroll 1
        for (int g = g0 + lane; g < g1; g += 32) {
            const float4 geo = __ldg(a.geo + g);
            const float4 sh = __ldg(a.shear + g);
            const int kg = (int)__ldg(a.keys + g) - R.start;
            float A, B, C, D, frg;
            gal_setup(R, geo, A, B, C, D, frg);
#pragma unroll
            for (int r = 0; r < GT; ++r) {
                const float u = gal_u(R, kg, frg, Xi[r], Xf[r]);
                float sinu, h;
                if (SMALL) sin_hav_small(u, sinu, h);
                else sin_hav_wide(u, sinu, h);
                const float s2 = fmaf(B, h, A);
                const bool in = on[r] && s2 < a.Tlo;
                if (on[r] && !(s2 < a.Tlo) && s2 <= a.Thi) {
                    const unsigned long long slot = atomicAdd(a.band_count, 1ull);
                    if (slot < (unsigned long long)a.band_cap) {
                        BandPair bp;
                        bp.target = tb + r;
                        bp.galaxy = g;
                        bp.entry = e;
                        reinterpret_cast<BandPair *>(a.band)[slot] = bp;
                    }
                }
                const float x = R.mrho0 * sinu;
                const float y = fmaf(D, h, C);
                const float xx = x * x;
                const float sd2 = fmaf(y, y, xx);
                const float cc = fmaf(y, y, -xx);
                const float ss = -2.0f * x * y;
                const float Q = filter_Q<KIND>(a.f, a.f.qtab, s2);
                const float w = (in && sd2 > 1e-30f) ? __fdividef(Q, sd2) : 0.f;
                pe[r] = fmaf(w, fmaf(sh.x, cc, sh.y * ss), pe[r]);
                pb[r] = fmaf(w, fmaf(sh.y, cc, -sh.x * ss), pb[r]);
                pv[r] = fmaf(in ? Q * Q : 0.f, sh.w, pv[r]);
                pw[r] += in ? sh.z : 0.f;
                nn[r] += in ? 1 : 0;
            }
        }
    }
}

template <int KIND>
__global__ void __launch_bounds__(32 * GW, 2) k_map_galaxy(const MapArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t tile = (int64_t)blockIdx.x * GW + (threadIdx.x >> 5);
    if (tile >= a.n_tiles) return;
    const int64_t tb = a.tiles[tile], te = a.tiles[tile + 1];
    const int nt = (int)(te - tb);
    const TargetRing tr0 = target_ring(a.N0, a.targets[tb]);
    const int64_t ring_start0 = a.targets[tb] - tr0.j0;
    int j0[GT];
    bool on[GT];
#pragma unroll
    for (int r = 0; r < GT; ++r) {
        on[r] = r < nt;
        j0[r] = on[r] ? (int)(a.targets[tb + r] - ring_start0) : tr0.j0;
    }
    float SE[GT], cSE[GT], SB[GT], cSB[GT], SV[GT], SW[GT], cSW[GT];
    int NN[GT];
#pragma unroll
    for (int r = 0; r < GT; ++r) {
        SE[r] = cSE[r] = SB[r] = cSB[r] = SV[r] = SW[r] = cSW[r] = 0.f;
        NN[r] = 0;
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
        float pe[GT], pb[GT], pv[GT], pw[GT];
        int nn[GT];
#pragma unroll
        for (int r = 0; r < GT; ++r) {
            pe[r] = pb[r] = pv[r] = pw[r] = 0.f;
            nn[r] = 0;
        }
        // pixel range [ulo, uhi] -> at most two runs of ring pixels
        // ulo lies in (-nr, 2 nr): one correction brings it into [0, nr)
        const int lo = ulo < 0 ? ulo + Rp.nr : (ulo >= Rp.nr ? ulo - Rp.nr : ulo);
        const int len = uhi - ulo + 1;
        if (R.small) gal_segment<KIND, true>(a, Rp, R, e, lane, tb, on, Xi, Xf, lo, len, pe, pb, pv, pw, nn);
        else gal_segment<KIND, false>(a, Rp, R, e, lane, tb, on, Xi, Xf, lo, len, pe, pb, pv, pw, nn);
#pragma unroll
        for (int r = 0; r < GT; ++r) {
            kahan_add(SE[r], cSE[r], pe[r]);
            kahan_add(SB[r], cSB[r], pb[r]);
            SV[r] += pv[r];
            kahan_add(SW[r], cSW[r], pw[r]);
            NN[r] += nn[r];
        }
    }
    // warp reduction of the per-lane sums (compensation folded in first);
    // raw sums go to float64 scratch, normalised after the guard-band pairs
#pragma unroll
    for (int r = 0; r < GT; ++r) {
        const float se = warp_sum(SE[r] - cSE[r]);
        const float sb = warp_sum(SB[r] - cSB[r]);
        const float sv = warp_sum(SV[r]);
        const float sw = warp_sum(SW[r] - cSW[r]);
        const int n = warp_sum_i(NN[r]);
        if (lane == r && on[r]) {
            double *raw = a.raw + 4 * (tb + r);
            raw[0] = se;
            raw[1] = sb;
            raw[2] = sv;
            raw[3] = sw;
            a.raw_n[tb + r] = n;
        }
    }
}

// the guard-band pairs: float64 decision, then the float32 contribution is
// added to the target's raw sums
template <int KIND>
__global__ void k_galaxy_band(const MapArgs a) {
    const unsigned long long nall = *a.band_count;
    if (nall > (unsigned long long)a.band_cap && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(a.status, SMART_STATUS_BAND_OVERFLOW);
    const unsigned long long nb = min(nall, (unsigned long long)a.band_cap);
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < nb;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const BandPair bp = reinterpret_cast<const BandPair *>(a.band)[i];
        const int64_t pix = a.targets[bp.target];
        const double2 rd = a.radec[bp.galaxy];
        double x0, y0, z0, x1, y1, z1;
        pix2vec64(a.N0, pix, x0, y0, z0);
        radec2vec64(rd.x, rd.y, x1, y1, z1);
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
        atomicAdd(a.raw_n + bp.target, 1);
    }
}

// summed normalisation (Sect. 2.4) from the float64 raw sums
__global__ void k_galaxy_finalise(const MapArgs a) {
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
        if (a.members) a.members[t] = n;
    }
}

}  // namespace smart

using namespace smart;

extern "C" smart_status smart_map_bruteforce(smart_ctx *c, const smart_maps *out) {
    if (!c) return SMART_E_ARG;
    if (!c->have_catalog) return fail(c, SMART_E_STATE, "smart_map_bruteforce: no catalogue (smart_bin_galaxies first)");
    MapArgs a{};
    smart_status st = common_args(c, out, a);
    if (st != SMART_OK) return st;
    if (!c->rp_gal) {
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
    a.table = c->rp_gal;
    a.counts = c->rp_gal_cnt;
    a.kmax = c->kmax_gal;
    a.offsets = c->offsets;
    a.geo = c->rec_geo;
    a.shear = c->rec_shear;
    a.radec = c->rec_radec;
    a.keys = c->keys;
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
    const unsigned blocks = (unsigned)((a.n_tiles + GW - 1) / GW);
    {
        KernelTimer timer(c, SMART_KT_GALAXY);
        if (c->filter_kind == SMART_FILTER_POLY) k_map_galaxy<SMART_FILTER_POLY><<<blocks, 32 * GW, 0, c->stream>>>(a);
        else k_map_galaxy<SMART_FILTER_SCHIRMER><<<blocks, 32 * GW, 0, c->stream>>>(a);
    }
    {
        KernelTimer timer(c, SMART_KT_GALAXY_BAND);
        if (c->filter_kind == SMART_FILTER_POLY) k_galaxy_band<SMART_FILTER_POLY><<<(unsigned)c->num_sms, 256, 0, c->stream>>>(a);
        else k_galaxy_band<SMART_FILTER_SCHIRMER><<<(unsigned)c->num_sms, 256, 0, c->stream>>>(a);
    }
    const unsigned fb = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)c->num_sms * 16);
    {
        KernelTimer timer(c, SMART_KT_GALAXY_FINALISE);
        k_galaxy_finalise<<<fb, 256, 0, c->stream>>>(a);
    }
    return check_cuda(c, cudaGetLastError(), "brute-force launches");
}
