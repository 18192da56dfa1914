// geometry.cu -- HEALPix RING geometry on the device and the ring-pair table
// of the aperture kernels (Sect. 3 of the paper; Gorski et al. 2005).
#include <math.h>

#include <algorithm>
#include <vector>

#include "smart_internal.cuh"

namespace smart {

__global__ void k_ang2pix(int64_t N, const double *__restrict__ ra, const double *__restrict__ dec,
                          int64_t n, int64_t *__restrict__ pix) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        pix[k] = ang2pix64(N, ra[k], dec[k]);
}

__global__ void k_pix2vec(int64_t N, const int64_t *__restrict__ pix, int64_t n, double *__restrict__ v) {
    const int64_t npix = 12 * N * N;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        double x = nan(""), y = nan(""), z = nan("");
        const int64_t p = pix[k];
        if (p >= 0 && p < npix) pix2vec64(N, p, x, y, z);
        v[3 * k] = x;
        v[3 * k + 1] = y;
        v[3 * k + 2] = z;
    }
}

// colatitude of ring i
__device__ __forceinline__ double ring_colat(int64_t N, int64_t i) {
    const RingGeom g = ring_geom(N, i);
    return atan2(g.rho, g.z);
}

// One thread per output ring i0.  Bin rings whose colatitude lies within
// theta_disc of i0's are the only ones that can hold members: the angular
// distance from any point of ring i0 to any point of ring i is at least the
// colatitude difference.  Each entry gets the float32 constants of the
// ring-pair geometry and the half window (in bin pixels) from the spherical
// law of cosines,  s^2 = A + B sin^2(dphi/2) <= T_disc.
__global__ void k_ring_pairs(int64_t N0, int64_t N1, double theta_disc, double Tdisc, int kmax,
                             RingPair *__restrict__ out, int *__restrict__ cnt, int *__restrict__ overflow) {
    const int64_t i0 = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i0 > 4 * N0 - 1) return;
    const RingGeom g0 = ring_geom(N0, i0);
    const double th0 = atan2(g0.rho, g0.z);
    const double lat0 = atan2(g0.z, g0.rho);
    const double margin = 1e-9;
    // first bin ring with colatitude >= th0 - theta_disc - margin (binary search)
    int64_t lo = 1, hi = 4 * N1 - 1;
    const double tlo = th0 - theta_disc - margin;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (ring_colat(N1, mid) < tlo) lo = mid + 1;
        else hi = mid;
    }
    int c = 0;
    RingPair *row = out + (i0 - 1) * (int64_t)kmax;
    for (int64_t i = lo; i <= 4 * N1 - 1; ++i) {
        const RingGeom g = ring_geom(N1, i);
        const double th = atan2(g.rho, g.z);
        if (th > th0 + theta_disc + margin) break;
        // latitude difference: A = 4 sin^2(dlat/2) and C = sin(dlat) vanish
        // exactly on the target's own ring (no cancellation of rho z0 - z rho0)
        const double dlat = lat0 - atan2(g.z, g.rho);
        const double sh = sin(0.5 * dlat);
        const double A = 4.0 * sh * sh;
        if (A > Tdisc * (1.0 + 1e-9) + 1e-300) continue;   // no azimuth can reach the disc
        const double B = 4.0 * g.rho * g0.rho;
        const double dphi = 2.0 * SMART_PI / (double)g.nr;
        int flags = g.shifted ? RP_SHIFTED : 0;
        double hw, hw_in = -1.0;
        const double sn2 = (Tdisc - A) / B;
        // certain members: s^2 <= T_disc (1 - 1e-5) for every offset within
        // hw_in, after the float32 rounding of the offsets (relative 1e-6 of
        // the window and 1e-3 bin pixels)
        const double sn2_in = (Tdisc * (1.0 - 1e-5) - A) / B;
        if (B > 0.0 && sn2_in >= 1.0) hw_in = (double)g.nr;
        else if (B > 0.0 && sn2_in > 0.0) hw_in = 2.0 * asin(sqrt(sn2_in)) / dphi * (1.0 - 1e-6) - 1e-3;
        if (!(B > 0.0) || sn2 >= 1.0) {
            flags |= RP_WHOLE | RP_WIDE;
            hw = 0.5 * g.nr;
        } else {
            const double half = 2.0 * asin(sqrt(fmax(sn2, 0.0)));
            // margin: float32 rounding of the window and of the per-pair offsets
            // is below 1e-4 bin pixels; pixels just outside are tested anyway
            hw = half / dphi * (1.0 + 1e-5) + 0.01;
            if (2.0 * hw + 1.0 >= (double)g.nr) {
                flags |= RP_WHOLE | RP_WIDE;
                hw = 0.5 * g.nr;
            } else if ((hw + 1.0) * dphi > 0.45 || theta_disc > 0.4) {
                // |u| can pass 0.45 rad (galaxy offsets add up to one bin pixel)
                flags |= RP_WIDE;
            }
        }
        if (c >= kmax) {
            atomicExch(overflow, 1);
            break;
        }
        RingPair e;
        e.start = (int)g.start;
        e.nr = g.nr;
        e.flags = flags;
        e.ring = (int)i;
        e.A = (float)A;
        e.B = (float)B;
        e.C = (float)sin(dlat);
        e.D = (float)(2.0 * g.z * g0.rho);
        e.dphi = (float)dphi;
        e.hw = (float)hw;
        e.mrho0 = (float)(-g0.rho);
        e.dlat = (float)dlat;
        e.rho0 = (float)g0.rho;
        e.z0 = (float)g0.z;
        e.hw_in = (float)hw_in;
        e.pad1 = 0.f;
        row[c++] = e;
    }
    cnt[i0 - 1] = c;
}

// Largest angular distance between a HEALPix pixel centre and any point of
// that pixel: the corner at the polar/equatorial transition (Gorski et al.
// 2005; the same expression as the HEALPix library's max_pixrad).
double max_pixrad(int nside) {
    const double N = (double)nside;
    const double za = 2.0 / 3.0, pa = SMART_PI / (4.0 * N);
    const double t1 = (1.0 - 1.0 / N) * (1.0 - 1.0 / N);
    const double zb = 1.0 - t1 / 3.0, pb = 0.0;
    const double ra = sqrt((1 - za) * (1 + za)), rb = sqrt((1 - zb) * (1 + zb));
    const double ax = ra * cos(pa), ay = ra * sin(pa), bx = rb * cos(pb), by = rb * sin(pb);
    const double dot = ax * bx + ay * by + za * zb;
    const double cx = ay * zb - za * by, cy = za * bx - ax * zb, cz = ax * by - ay * bx;
    return atan2(sqrt(cx * cx + cy * cy + cz * cz), dot);
}

smart_status build_ring_pairs(smart_ctx *ctx, double theta_disc, RingPair **out, int **cnt, int *kmax) {
    const int64_t N0 = ctx->nside_out, N1 = ctx->nside_bin;
    const int64_t nring = 4 * N0 - 1;
    const int k = (int)(3.0 * theta_disc * (double)N1 * 1.02) + 6;
    const double bytes = (double)nring * (double)k * sizeof(RingPair);
    if (bytes > 8.0e9)
        return fail(ctx, SMART_E_OVERFLOW, "ring-pair table would exceed 8 GB: aperture too large for this nside");
    RingPair *t = nullptr;
    int *c = nullptr, *ov = nullptr;
    cudaError_t e = cudaMalloc(&t, (size_t)nring * k * sizeof(RingPair));
    if (e != cudaSuccess) return fail(ctx, SMART_E_NOMEM, "cudaMalloc(ring-pair table) failed");
    e = cudaMalloc(&c, (size_t)nring * sizeof(int) + sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(t);
        return fail(ctx, SMART_E_NOMEM, "cudaMalloc(ring-pair counts) failed");
    }
    ov = c + nring;
    cudaMemsetAsync(ov, 0, sizeof(int), ctx->stream);
    const double Tdisc = (theta_disc == ctx->theta_ap) ? ctx->T : 4.0 * sin(0.5 * theta_disc) * sin(0.5 * theta_disc);
    k_ring_pairs<<<(unsigned)((nring + 127) / 128), 128, 0, ctx->stream>>>(N0, N1, theta_disc, Tdisc, k, t, c, ov);
    smart_status st = check_cuda(ctx, cudaGetLastError(), "k_ring_pairs launch");
    int32_t *hov = reinterpret_cast<int32_t *>(ctx->host_rb);
    if (st == SMART_OK) st = check_cuda(ctx, cudaMemcpyAsync(hov, ov, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "ring-pair overflow flag");
    if (st == SMART_OK) st = wait_stream(ctx, "ring-pair build");
    if (st == SMART_OK && hov[0]) st = fail(ctx, SMART_E_INTERNAL, "ring-pair table row overflow");
    if (st != SMART_OK) {
        cudaFree(t);
        cudaFree(c);
        return st;
    }
    *out = t;
    *cnt = c;
    *kmax = k;
    return SMART_OK;
}

}  // namespace smart

using namespace smart;

static bool nside_ok(int nside) { return nside >= 1 && nside <= 8192 && (nside & (nside - 1)) == 0; }

extern "C" smart_status smart_ang2pix(int nside, const double *ra_deg, const double *dec_deg, int64_t n,
                                      int64_t *pix, void *cuda_stream) {
    if (!nside_ok(nside) || n < 0 || (n > 0 && (!ra_deg || !dec_deg || !pix))) return SMART_E_ARG;
    if (n == 0) return SMART_OK;
    const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 148 * 64);
    k_ang2pix<<<blocks, 256, 0, (cudaStream_t)cuda_stream>>>(nside, ra_deg, dec_deg, n, pix);
    return cudaGetLastError() == cudaSuccess ? SMART_OK : SMART_E_CUDA;
}

extern "C" smart_status smart_pix2vec(int nside, const int64_t *pix, int64_t n, double *vec, void *cuda_stream) {
    if (!nside_ok(nside) || n < 0 || (n > 0 && (!pix || !vec))) return SMART_E_ARG;
    if (n == 0) return SMART_OK;
    const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 148 * 64);
    k_pix2vec<<<blocks, 256, 0, (cudaStream_t)cuda_stream>>>(nside, pix, n, vec);
    return cudaGetLastError() == cudaSuccess ? SMART_OK : SMART_E_CUDA;
}

extern "C" double smart_chord2(double theta_ap_arcmin) {
    const double th = theta_ap_arcmin * SMART_PI / 10800.0;
    const double sh = sin(0.5 * th);
    return 4.0 * sh * sh;
}
