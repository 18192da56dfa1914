// aperture.cu -- the aperture-mass kernels (Sect. 3.1 brute force, Sect. 3.2
// pixel-based, summed normalisation of Sect. 2.4).
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
//
// Accumulation: float32 within one bin ring, compensated (Kahan) across
// rings; the weight sum is carried to float64 for the final division.
#include <math.h>

#include <algorithm>

#include "smart_internal.cuh"

namespace smart {

struct FilterArgs {
    float inv_ap;      // 1 / theta_ap
    float inv_ap2;     // 1 / theta_ap^2
    float qnorm;       // poly: 6 / (pi theta_ap^2); Schirmer: 1 / theta_ap^2
    float inv_xc;      // Schirmer 1 / xc
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
    // pixel-mode inputs
    const float *G1, *G2, *W, *S2;
    const int32_t *NP;
    // brute-force inputs
    const int32_t *offsets;
    const float4 *geo, *shear;
    const double2 *radec;
    // outputs
    double *sum_w;
    float *map_e, *map_b, *var;
    int64_t *count;
    int32_t *members;
    unsigned long long *fp64_count;
};

// great-circle separation^2 from the chord^2: d^2 = sum_n 2 s^(2n) / (n^2 C(2n,n))
__device__ __forceinline__ float sep2_from_chord2(float s2) {
    if (s2 > 0.05f) {
        const float d = 2.0f * asinf(0.5f * sqrtf(s2));
        return d * d;
    }
    return s2 * fmaf(s2, fmaf(s2, fmaf(s2, fmaf(s2, 1.0f / 3150.0f, 1.0f / 560.0f), 1.0f / 90.0f), 1.0f / 12.0f), 1.0f);
}

template <int KIND>
__device__ __forceinline__ float filter_Q(const FilterArgs &f, float s2) {
    const float d2 = sep2_from_chord2(s2);
    if (KIND == SMART_FILTER_POLY) {
        const float X2 = d2 * f.inv_ap2;
        return f.qnorm * X2 * (1.0f - X2);
    } else {
        const float x = sqrtf(d2) * f.inv_ap;
        const float r = x * f.inv_xc;
        const float th = r > 1e-3f ? tanhf(r) / r : fmaf(-r * r, 1.0f / 3.0f, 1.0f);
        const float den = 1.0f + expf(fmaf(-150.0f, x, 6.0f)) + expf(fmaf(50.0f, x, -47.0f));
        return f.qnorm * th / den;
    }
}

// sin u and sin^2(u/2) for |u| <= 0.45 (series, relative error < 2e-9)
__device__ __forceinline__ void small_sin_hav(float u, float &sinu, float &h) {
    const float u2 = u * u;
    sinu = u * fmaf(u2, fmaf(u2, fmaf(u2, -1.0f / 5040.0f, 1.0f / 120.0f), -1.0f / 6.0f), 1.0f);
    h = u2 * fmaf(u2, fmaf(u2, fmaf(u2, -1.0f / 80640.0f, 1.0f / 1440.0f), -1.0f / 48.0f), 0.25f);
}

__device__ __forceinline__ void wide_sin_hav(float u, float &sinu, float &h) {
    float sh, ch;
    sincosf(0.5f * u, &sh, &ch);
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
    int i0, j0, q0, s0;
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
    return t;
}

// target position on the bin ring's azimuth lattice: X = (2 j0 + s0) q / (2 q0)
// split as Xi + Xf with Xi integer and 0 <= Xf < 1 (exact integer arithmetic)
__device__ __forceinline__ void lattice_position(const TargetRing &t, int q, int &Xi, float &Xf) {
    if (q == t.q0) {
        Xi = t.j0;
        Xf = 0.5f * (float)t.s0;
    } else {
        const int64_t num = (int64_t)(2 * t.j0 + t.s0) * q;
        const int64_t den = 2 * (int64_t)t.q0;
        const int64_t qi = num / den;
        Xi = (int)qi;
        Xf = (float)(num - qi * den) / (float)den;
    }
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

__device__ __forceinline__ void finalise(const MapArgs &a, int64_t t, float se, float cse, float sb, float csb,
                                         float sv, float csv, float sw, float csw, int64_t cnt, int nmem) {
    const double SW = (double)sw - (double)csw;
    double me = 0.0, mb = 0.0, vv = 0.0;
    if (SW > 0.0) {
        const double nbar = SW / a.area;
        me = ((double)se - (double)cse) / nbar;
        mb = ((double)sb - (double)csb) / nbar;
        vv = ((double)sv - (double)csv) / (2.0 * nbar * nbar);
    }
    if (a.sum_w) a.sum_w[t] = SW;
    if (a.map_e) a.map_e[t] = (float)me;
    if (a.map_b) a.map_b[t] = (float)mb;
    if (a.var) a.var[t] = (float)vv;
    if (a.count) a.count[t] = cnt;
    if (a.members) a.members[t] = nmem;
}

// ------------------------------------------------------------------------
// pixel mode: one thread per target
// ------------------------------------------------------------------------
template <int KIND>
__global__ void __launch_bounds__(128) k_map_pixel(const MapArgs a) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= a.n) return;
    const int64_t pix = a.targets[t];
    const TargetRing tr = target_ring(a.N0, pix);
    const RingPair *row = a.table + (int64_t)(tr.i0 - 1) * a.kmax;
    const int nent = a.counts[tr.i0 - 1];
    float SE = 0.f, cSE = 0.f, SB = 0.f, cSB = 0.f, SV = 0.f, cSV = 0.f, SW = 0.f, cSW = 0.f;
    int64_t NN = 0;
    int NM = 0;
    bool have64 = false;
    double x0 = 0, y0 = 0, z0 = 0;
    for (int e = 0; e < nent; ++e) {
        const RingPair R = row[e];
        const int q = R.nr >> 2;
        int Xi;
        float Xf;
        lattice_position(tr, q, Xi, Xf);
        const float fr = ((R.flags & RP_SHIFTED) ? 0.5f : 0.0f) - Xf;
        int kl, kh;
        window(R, fr, kl, kh);
        float se = 0.f, sb = 0.f, sv = 0.f, sw = 0.f;
        int nn = 0;
        int kk = (Xi + kl) % R.nr;
        if (kk < 0) kk += R.nr;
        const bool wide = (R.flags & RP_WIDE) != 0;
        for (int k = kl; k <= kh; ++k) {
            const float u = ((float)k + fr) * R.dphi;
            float sinu, h;
            if (wide) wide_sin_hav(u, sinu, h);
            else small_sin_hav(u, sinu, h);
            const float s2 = fmaf(R.B, h, R.A);
            const int p = R.start + kk;
            kk = (kk + 1 == R.nr) ? 0 : kk + 1;
            if (s2 > a.Thi) continue;
            if (s2 >= a.Tlo) {
                if (!have64) {
                    pix2vec64(a.N0, pix, x0, y0, z0);
                    have64 = true;
                }
                double x1, y1, z1;
                pix2vec64(a.N1, p, x1, y1, z1);
                atomicAdd(a.fp64_count, 1ull);
                if (!member64(x0, y0, z0, x1, y1, z1, a.T)) continue;
            }
            const float x = R.mrho0 * sinu;
            const float y = fmaf(R.D, h, R.C);
            const float xx = x * x;
            const float sd2 = fmaf(y, y, xx);
            const float cc = fmaf(y, y, -xx);
            const float ss = -2.0f * x * y;
            const float Q = filter_Q<KIND>(a.f, s2);
            const float w = sd2 > 1e-30f ? Q / sd2 : 0.f;
            const float g1 = __ldg(a.G1 + p), g2 = __ldg(a.G2 + p);
            se = fmaf(w, fmaf(g1, cc, g2 * ss), se);
            sb = fmaf(w, fmaf(g2, cc, -g1 * ss), sb);
            sv = fmaf(Q * Q, __ldg(a.S2 + p), sv);
            sw += __ldg(a.W + p);
            nn += __ldg(a.NP + p);
            NM += 1;
        }
        kahan_add(SE, cSE, se);
        kahan_add(SB, cSB, sb);
        kahan_add(SV, cSV, sv);
        kahan_add(SW, cSW, sw);
        NN += nn;
    }
    finalise(a, t, SE, cSE, SB, cSB, SV, cSV, SW, cSW, NN, NM);
}

// ------------------------------------------------------------------------
// brute force over the sorted catalogue: one thread per target
// ------------------------------------------------------------------------
template <int KIND>
__global__ void __launch_bounds__(128) k_map_galaxy(const MapArgs a) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= a.n) return;
    const int64_t pix = a.targets[t];
    const TargetRing tr = target_ring(a.N0, pix);
    const RingPair *row = a.table + (int64_t)(tr.i0 - 1) * a.kmax;
    const int nent = a.counts[tr.i0 - 1];
    float SE = 0.f, cSE = 0.f, SB = 0.f, cSB = 0.f, SV = 0.f, cSV = 0.f, SW = 0.f, cSW = 0.f;
    int64_t NN = 0;
    int NM = 0;
    bool have64 = false;
    double x0 = 0, y0 = 0, z0 = 0;
    for (int e = 0; e < nent; ++e) {
        const RingPair R = row[e];
        const int q = R.nr >> 2;
        int Xi;
        float Xf;
        lattice_position(tr, q, Xi, Xf);
        const float fr = ((R.flags & RP_SHIFTED) ? 0.5f : 0.0f) - Xf;
        int kl, kh;
        window(R, fr, kl, kh);
        float se = 0.f, sb = 0.f, sv = 0.f, sw = 0.f;
        int nn = 0;
        int kk = (Xi + kl) % R.nr;
        if (kk < 0) kk += R.nr;
        const bool wide = (R.flags & RP_WIDE) != 0;
        const float B0 = 4.0f * R.rho0, D0 = 2.0f * R.rho0;
        for (int k = kl; k <= kh; ++k) {
            const float uc = ((float)k + fr) * R.dphi;
            const int p = R.start + kk;
            kk = (kk + 1 == R.nr) ? 0 : kk + 1;
            const int g0 = __ldg(a.offsets + p), g1 = __ldg(a.offsets + p + 1);
            for (int g = g0; g < g1; ++g) {
                const float4 gg = __ldg(a.geo + g);       // (ddec, dphi, z, rho)
                const float u = uc + gg.y;
                const float dl = R.dlat - gg.x;             // lat0 - lat_galaxy
                float sinu, h, A, C;
                if (wide) {
                    wide_sin_hav(u, sinu, h);
                    float sdh, cdh;
                    sincosf(0.5f * dl, &sdh, &cdh);
                    A = 4.0f * sdh * sdh;
                    C = 2.0f * sdh * cdh;
                } else {
                    small_sin_hav(u, sinu, h);
                    const float d2 = dl * dl;
                    A = d2 * fmaf(d2, fmaf(d2, fmaf(d2, -1.0f / 20160.0f, 1.0f / 360.0f), -1.0f / 12.0f), 1.0f);
                    C = dl * fmaf(d2, fmaf(d2, fmaf(d2, -1.0f / 5040.0f, 1.0f / 120.0f), -1.0f / 6.0f), 1.0f);
                }
                const float s2 = fmaf(B0 * gg.w, h, A);
                if (s2 > a.Thi) continue;
                if (s2 >= a.Tlo) {
                    if (!have64) {
                        pix2vec64(a.N0, pix, x0, y0, z0);
                        have64 = true;
                    }
                    const double2 rd = __ldg(a.radec + g);
                    double x1, y1, z1;
                    radec2vec64(rd.x, rd.y, x1, y1, z1);
                    atomicAdd(a.fp64_count, 1ull);
                    if (!member64(x0, y0, z0, x1, y1, z1, a.T)) continue;
                }
                const float x = R.mrho0 * sinu;
                const float y = fmaf(D0 * gg.z, h, C);
                const float xx = x * x;
                const float sd2 = fmaf(y, y, xx);
                const float cc = fmaf(y, y, -xx);
                const float ss = -2.0f * x * y;
                const float Q = filter_Q<KIND>(a.f, s2);
                const float w = sd2 > 1e-30f ? Q / sd2 : 0.f;
                const float4 sh = __ldg(a.shear + g);      // (w e1, w e2, w, w^2 |e|^2)
                se = fmaf(w, fmaf(sh.x, cc, sh.y * ss), se);
                sb = fmaf(w, fmaf(sh.y, cc, -sh.x * ss), sb);
                sv = fmaf(Q * Q, sh.w, sv);
                sw += sh.z;
                nn += 1;
                NM += 1;
            }
        }
        kahan_add(SE, cSE, se);
        kahan_add(SB, cSB, sb);
        kahan_add(SV, cSV, sv);
        kahan_add(SW, cSW, sw);
        NN += nn;
    }
    finalise(a, t, SE, cSE, SB, cSB, SV, cSV, SW, cSW, NN, NM);
}

static FilterArgs make_filter(const smart_ctx *c) {
    FilterArgs f;
    f.inv_ap = (float)(1.0 / c->theta_ap);
    f.inv_ap2 = (float)(1.0 / (c->theta_ap * c->theta_ap));
    f.qnorm = c->filter_kind == SMART_FILTER_POLY ? (float)(6.0 / SMART_PI / (c->theta_ap * c->theta_ap))
                                                  : (float)(1.0 / (c->theta_ap * c->theta_ap));
    f.inv_xc = (float)(1.0 / c->xc);
    return f;
}

static smart_status common_args(smart_ctx *c, const smart_maps *out, MapArgs &a) {
    if (!out) return fail(c, SMART_E_ARG, "null output struct");
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
    a.table = c->rp_pix;
    a.counts = c->rp_pix_cnt;
    a.kmax = c->kmax_pix;
    a.G1 = c->G1;
    a.G2 = c->G2;
    a.W = c->W;
    a.S2 = c->S2;
    a.NP = c->NP;
    cudaMemsetAsync(c->d_fp64_count, 0, sizeof(unsigned long long), c->stream);
    if (a.n == 0) return SMART_OK;
    const unsigned blocks = (unsigned)((a.n + 127) / 128);
    if (c->filter_kind == SMART_FILTER_POLY) k_map_pixel<SMART_FILTER_POLY><<<blocks, 128, 0, c->stream>>>(a);
    else k_map_pixel<SMART_FILTER_SCHIRMER><<<blocks, 128, 0, c->stream>>>(a);
    return check_cuda(c, cudaGetLastError(), "k_map_pixel launch");
}

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
    a.table = c->rp_gal;
    a.counts = c->rp_gal_cnt;
    a.kmax = c->kmax_gal;
    a.offsets = c->offsets;
    a.geo = c->rec_geo;
    a.shear = c->rec_shear;
    a.radec = c->rec_radec;
    cudaMemsetAsync(c->d_fp64_count, 0, sizeof(unsigned long long), c->stream);
    if (a.n == 0) return SMART_OK;
    const unsigned blocks = (unsigned)((a.n + 127) / 128);
    if (c->filter_kind == SMART_FILTER_POLY) k_map_galaxy<SMART_FILTER_POLY><<<blocks, 128, 0, c->stream>>>(a);
    else k_map_galaxy<SMART_FILTER_SCHIRMER><<<blocks, 128, 0, c->stream>>>(a);
    return check_cuda(c, cudaGetLastError(), "k_map_galaxy launch");
}
