// aperture_galaxy.cu -- brute-force aperture mass at galaxy positions
// (Sect. 3.1 steps 1-5), neighbours found through the catalogue sorted by
// HEALPix pixel (Sect. 3.4).  One thread per target; the bin rings that can
// hold members come from the ring-pair table built for theta_ap plus the
// largest pixel radius; each candidate pixel's galaxies are a contiguous
// range of the sorted catalogue.
#include <math.h>

#include <algorithm>

#include "aperture_common.cuh"

namespace smart {

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
                    sin_hav_wide(u, sinu, h);
                    float sdh, cdh;
                    sincosf(0.5f * dl, &sdh, &cdh);
                    A = 4.0f * sdh * sdh;
                    C = 2.0f * sdh * cdh;
                } else {
                    sin_hav_small(u, sinu, h);
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
                const float Q = filter_Q<KIND>(a.f, a.f.qtab, s2);
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
