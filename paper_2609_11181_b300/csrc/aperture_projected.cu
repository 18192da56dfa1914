// aperture_projected.cu -- the Cartesian (projected) shear-based aperture
// mass at galaxy positions, projS_pos (Sect. 2.2, Sect. 5.2.1 steps 1-4), and
// equal-area annulus statistics about the projection centre (Sect. 5.2.2).
//
// Step 1 (per call, one thread per sorted galaxy): the galaxy's float64 unit
// vector r goes to the plane tangent at the reference point c (gnomonic
// projection, Sect. 2.2.1): x = (r . e_c) / (r . c), y = (r . n_c) / (r . c),
// with (e_c, n_c) the East and North unit vectors at c -- the printed
// formula's numerators and denominator written as dot products.  Each
// coordinate is stored as a float32 pair (hi, lo) with hi + lo = x to about
// 2^-48 |x|, so that differences of nearby positions keep full float32
// precision anywhere in a wide field.  The shear is rotated with the basis
// (Sect. 2.2.2): its orientation stays relative to the local North, whose
// image direction is the projection's differential applied to the galaxy's
// North unit vector.  Galaxies more than 90 degrees from c have no image.
// Step 2: the targets' pixel centres are projected the same way.
// Steps 3-4 (main kernel): one warp per group of PT consecutive targets of an
// output ring walks the galaxies of the brute-force ring-pair windows (the
// cap of radius theta_ap plus a bin-pixel radius): a member in the plane is
// always within theta_ap on the sphere, since the plane distance of two
// images is at least their great-circle distance (straight segments of the
// plane are images of great-circle arcs and the projection stretches every
// direction by at least 1).  Per pair: (dx, dy) in the plane, member iff
// dx^2 + dy^2 <= theta_ap^2, Q of the plane distance, and
//   gamma_+ = -(g1 cos 2phi + g2 sin 2phi),  gamma_x = g1 sin 2phi - g2 cos 2phi
// with phi the polar angle of (dx, dy) -- the sign convention of the
// spherical sums -- from cos 2phi = (dx^2 - dy^2) / r^2, sin 2phi =
// 2 dx dy / r^2 (no atan2).  Membership is decided in float32 outside a
// guard band of relative width 4e-6 and, inside it, by the float64
// definition in the same order of operations as the float64 reference.
// Sums are normalised with A = pi theta_ap^2, the aperture's plane area.
#include <math.h>

#include <algorithm>

#include "aperture_common.cuh"

namespace smart {
namespace {

constexpr int PT_LOG2 = GAL_GROUP_LOG2;
constexpr int PT = 1 << PT_LOG2;   // targets per warp (the brute-force target groups)
constexpr int PW = 8;              // warps per CTA

// reference point c and its East / North unit vectors
struct Plane {
    double c[3], e[3], n[3];
};

struct ProjArgs {
    const float4 *gxy;       // per sorted galaxy: (x hi, y hi, x lo, y lo)
    const float4 *gsh;       // per sorted galaxy: rotated (w g1, w g2), w, w^2 |e|^2
    const float4 *txy;       // per target: (x hi, y hi, x lo, y lo); NaN: no image
    const double *plane;     // Plane, 9 doubles
    float Tlo, Thi;          // guard band around theta_ap^2 (float32)
    double Tp;               // theta_ap^2 (float64 definition)
    const float4 *qtab;      // filter table on the plane distance (tabulated filters)
    float tab_scale;         // QTAB_BINS / theta_ap
};

struct ProjBandPair {
    int64_t target;
    int32_t galaxy;
    int32_t pad;
};

__device__ __forceinline__ double dot3_rn(double x, double y, double z, const double *b) {
    return __dadd_rn(__dadd_rn(__dmul_rn(x, b[0]), __dmul_rn(y, b[1])), __dmul_rn(z, b[2]));
}

// plane coordinates of a unit vector in the float64 reference's order of
// operations; false when the point has no image
__device__ __forceinline__ bool plane_xy64(const Plane &P, double rx, double ry, double rz, double &x, double &y,
                                           double *X = nullptr, double *Y = nullptr, double *D = nullptr) {
    const double d = dot3_rn(rx, ry, rz, P.c);
    if (!(d > 0.0)) return false;
    const double xe = dot3_rn(rx, ry, rz, P.e), yn = dot3_rn(rx, ry, rz, P.n);
    x = __ddiv_rn(xe, d);
    y = __ddiv_rn(yn, d);
    if (X) {
        *X = xe;
        *Y = yn;
        *D = d;
    }
    return true;
}

__device__ __forceinline__ Plane load_plane(const double *p) {
    Plane P;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        P.c[i] = p[i];
        P.e[i] = p[3 + i];
        P.n[i] = p[6 + i];
    }
    return P;
}

__device__ __forceinline__ float4 split_xy(double x, double y) {
    const float xh = (float)x, yh = (float)y;
    return make_float4(xh, yh, (float)(x - (double)xh), (float)(y - (double)yh));
}

__global__ void k_plane_setup(double ra_c, double dec_c, double *out) {
    double sa, ca, sd, cd;
    sincos_deg64(ra_c, sa, ca);
    sincos_deg64(dec_c, sd, cd);
    out[0] = __dmul_rn(cd, ca);
    out[1] = __dmul_rn(cd, sa);
    out[2] = sd;
    out[3] = -sa;
    out[4] = ca;
    out[5] = 0.0;
    out[6] = -__dmul_rn(sd, ca);
    out[7] = -__dmul_rn(sd, sa);
    out[8] = cd;
}

// The records only need their positions to about 2^-48 (the float32 hi/lo
// pairs) and the shear rotation to float32: the float64 membership
// decisions recompute positions in the reference's order of operations
// (plane_xy64), so the records take cheaper steps -- the quadrant of an
// angle from a product with 1/90 instead of a division (the reduced angle
// may pass 45 degrees by an ulp, where the series is as accurate), one
// reciprocal for both plane coordinates, and the rotation in float32.
__device__ __forceinline__ void sincos_deg64_rec(double x, double &s, double &c) {
    const double q = rint(__dmul_rn(x, 1.0 / 90.0));
    const double y = __dadd_rn(x, -__dmul_rn(q, 90.0));
    double ss, cc;
    series_sincos(__dmul_rn(y, SMART_PI / 180.0), ss, cc);
    const int k = (int)((long long)q & 3);
    if (k == 0) { s = ss; c = cc; }
    else if (k == 1) { s = cc; c = -ss; }
    else if (k == 2) { s = -ss; c = -cc; }
    else { s = -cc; c = ss; }
}

// step 1: plane position and rotated shear of every sorted galaxy
__global__ void k_proj_records(int64_t n, const double2 *__restrict__ radec, const float4 *__restrict__ sh_in,
                               const double *__restrict__ plane, float4 *__restrict__ gxy, float4 *__restrict__ gsh) {
    const Plane P = load_plane(plane);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const double2 rd = radec[k];
        double sa, ca, sd, cd;
        sincos_deg64_rec(rd.x, sa, ca);
        sincos_deg64_rec(rd.y, sd, cd);
        const double rx = cd * ca, ry = cd * sa, rz = sd;
        const double D = rx * P.c[0] + ry * P.c[1] + rz * P.c[2];
        if (!(D > 0.0)) {
            // no image: far outside every aperture, never a member (finite,
            // so that every product of the pair body stays finite)
            gxy[k] = make_float4(1e18f, 1e18f, 0.f, 0.f);
            gsh[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        const double X = rx * P.e[0] + ry * P.e[1] + rz * P.e[2];
        const double Y = rx * P.n[0] + ry * P.n[1] + rz * P.n[2];
        const double iD = 1.0 / D;
        gxy[k] = split_xy(X * iD, Y * iD);
        // image of the local North t = (-sin d cos a, -sin d sin a, cos d),
        // up to the positive factor 1 / D^2
        const double tx = -sd * ca, ty = -sd * sa, tz = cd;
        const double tc = tx * P.c[0] + ty * P.c[1] + tz * P.c[2];
        const double te = tx * P.e[0] + ty * P.e[1] + tz * P.e[2];
        const double tn = tx * P.n[0] + ty * P.n[1] + tz * P.n[2];
        const float Nx = (float)(te * D - X * tc), Ny = (float)(tn * D - Y * tc);
        const float inn = 1.0f / fmaf(Nx, Nx, Ny * Ny);
        const float c2 = (Ny * Ny - Nx * Nx) * inn;              // cos 2 rho
        const float s2 = -2.0f * Nx * Ny * inn;                  // sin 2 rho
        const float4 g = sh_in[k];                                // (w e1, w e2, w, w^2 |e|^2)
        gsh[k] = make_float4(g.x * c2 - g.y * s2, g.x * s2 + g.y * c2, g.z, g.w);
    }
}

// step 2: plane positions of the targets
__global__ void k_proj_targets(int64_t N0, int64_t n, const int64_t *__restrict__ targets,
                               const double *__restrict__ plane, float4 *__restrict__ txy) {
    const Plane P = load_plane(plane);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        double rx, ry, rz, x, y;
        pix2vec64(N0, targets[t], rx, ry, rz);
        txy[t] = plane_xy64(P, rx, ry, rz, x, y) ? split_xy(x, y) : make_float4(NAN, NAN, NAN, NAN);
    }
}

template <int KIND>
__device__ __forceinline__ float plane_Q(const MapArgs &a, const ProjArgs &p, float r2) {
    if (KIND == SMART_FILTER_POLY) {
        const float X2 = r2 * a.f.inv_ap2;
        return a.f.qnorm * X2 * (1.0f - X2);
    } else {
        return qtab_eval(p.qtab, r2, p.tab_scale);
    }
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int warp_sum_n(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// one pair's float32 contribution (in: a member outside the guard band, or a
// guard-band pair the float64 decision admitted)
template <int KIND>
__device__ __forceinline__ void proj_pair(const MapArgs &a, const ProjArgs &p, float dx, float dy, float r2, bool in,
                                          const float4 &sh, float &pe, float &pb, float &pv, float &pw, int &nn) {
    const float c2n = fmaf(dx, dx, -dy * dy);        // r^2 cos 2phi
    const float s2n = 2.0f * dx * dy;                // r^2 sin 2phi
    float Q, w;
    if (KIND == SMART_FILTER_POLY) {
        // Q = qnorm X^2 (1 - X^2) with X^2 = r^2 / theta^2, so Q / r^2 =
        // qnorm/theta^2 (1 - X^2) exactly: no division
        const float qn1 = a.f.qnorm * a.f.inv_ap2;
        const float t = fmaf(r2, -qn1 * a.f.inv_ap2, qn1);
        Q = r2 * t;
        w = in ? t : 0.f;
    } else {
        Q = plane_Q<KIND>(a, p, r2);
        // r2 = 0 only for a galaxy at the target itself: no shear (c2n = s2n = 0)
        w = in ? __fdividef(Q, r2 + 1e-30f) : 0.f;
    }
    pe = fmaf(-w, fmaf(sh.x, c2n, sh.y * s2n), pe);
    pb = fmaf(w, fmaf(sh.x, s2n, -sh.y * c2n), pb);
    pv = fmaf(in ? Q * Q : 0.f, sh.w, pv);
    pw += in ? sh.z : 0.f;
    nn += in ? 1 : 0;
}

template <int KIND>
__global__ void __launch_bounds__(32 * PW, 2) k_map_projected(const MapArgs a, const ProjArgs p) {
    const int lane = threadIdx.x & 31;
    const int64_t tile = (int64_t)blockIdx.x * PW + (threadIdx.x >> 5);
    if (tile >= a.n_tiles) return;
    const int64_t tb = a.tiles[tile], te = a.tiles[tile + 1];
    const int nt = (int)(te - tb);
    const TargetRing tr0 = target_ring(a.N0, a.targets[tb]);
    const int64_t ring_start0 = a.targets[tb] - tr0.j0;
    int j0[PT];
    bool on[PT];
    float4 T[PT];
#pragma unroll
    for (int r = 0; r < PT; ++r) {
        T[r] = r < nt ? __ldg(p.txy + tb + r) : make_float4(NAN, NAN, NAN, NAN);
        on[r] = r < nt && !isnan(T[r].x);
        // a target without an image (or past the group's end) sits far away:
        // its pairs are finite and never members, its sums stay zero
        if (!on[r]) T[r] = make_float4(-1e18f, -1e18f, 0.f, 0.f);
        j0[r] = r < nt ? (int)(a.targets[tb + r] - ring_start0) : tr0.j0;
    }
    float SE[PT], SB[PT], SV[PT], SW[PT];
    int NN[PT];
#pragma unroll
    for (int r = 0; r < PT; ++r) {
        SE[r] = SB[r] = SV[r] = SW[r] = 0.f;
        NN[r] = 0;
    }
    const int64_t row0 = (int64_t)(tr0.i0 - 1) * a.kmax;
    const int nent = a.counts[tr0.i0 - 1];
    const LatticeDiv ld = lattice_div(tr0);
    for (int e = 0; e < nent; ++e) {
        const RingPair Rp = a.table[row0 + e];
        const float fr_shift = (Rp.flags & RP_SHIFTED) ? 0.5f : 0.0f;
        const int q = Rp.nr >> 2;
        // union of the targets' windows in unwrapped bin pixels
        int ulo = INT32_MAX, uhi = INT32_MIN;
#pragma unroll
        for (int r = 0; r < PT; ++r) {
            if (!on[r]) continue;
            TargetRing t = tr0;
            t.j0 = j0[r];
            int Xi;
            float Xf;
            lattice_position(t, ld, q, Xi, Xf);
            int kl, kh;
            window(Rp, fr_shift - Xf, kl, kh);
            ulo = min(ulo, Xi + kl);
            uhi = max(uhi, Xi + kh);
        }
        if (ulo > uhi) continue;              // no target with an image
        if (uhi - ulo + 1 > Rp.nr) {          // whole ring
            ulo = 0;
            uhi = Rp.nr - 1;
        }
        const int lo = ulo < 0 ? ulo + Rp.nr : (ulo >= Rp.nr ? ulo - Rp.nr : ulo);
        const int len = uhi - ulo + 1;
        const int n1 = min(len, Rp.nr - lo);
        float pe[PT], pb[PT], pv[PT], pw[PT];
        int nn[PT];
#pragma unroll
        for (int r = 0; r < PT; ++r) {
            pe[r] = pb[r] = pv[r] = pw[r] = 0.f;
            nn[r] = 0;
        }
#pragma unroll 1
        for (int part = 0; part < 2; ++part) {
            const int pa = part == 0 ? lo : 0;
            const int pn = part == 0 ? n1 : len - n1;
            if (pn <= 0) continue;
            const int g0 = __ldg(a.offsets + Rp.start + pa);
            const int g1 = __ldg(a.offsets + Rp.start + pa + pn);
#pragma unroll 1
            for (int g = g0 + lane; g < g1; g += 32) {
                const float4 xy = __ldg(p.gxy + g);
                const float4 sh = __ldg(p.gsh + g);
                unsigned band = 0;
#pragma unroll
                for (int r = 0; r < PT; ++r) {
                    const float dx = (xy.x - T[r].x) + (xy.z - T[r].z);
                    const float dy = (xy.y - T[r].y) + (xy.w - T[r].w);
                    const float r2 = fmaf(dx, dx, dy * dy);
                    const bool in = on[r] && r2 < p.Tlo;
                    band |= (on[r] && !(r2 < p.Tlo) && r2 <= p.Thi) ? (1u << r) : 0u;
                    proj_pair<KIND>(a, p, dx, dy, r2, in, sh, pe[r], pb[r], pv[r], pw[r], nn[r]);
                }
                if (band) {              // rare: one branch per galaxy
                    for (int r = 0; r < PT; ++r) {
                        if (!(band & (1u << r))) continue;
                        const unsigned long long slot = atomicAdd(a.band_count, 1ull);
                        if (slot < (unsigned long long)a.band_cap) {
                            ProjBandPair bp;
                            bp.target = tb + r;
                            bp.galaxy = g;
                            bp.pad = 0;
                            reinterpret_cast<ProjBandPair *>(a.band)[slot] = bp;
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < PT; ++r) {
            SE[r] += pe[r];
            SB[r] += pb[r];
            SV[r] += pv[r];
            SW[r] += pw[r];
            NN[r] += nn[r];
        }
    }
#pragma unroll
    for (int r = 0; r < PT; ++r) {
        const float se = warp_sum_f(SE[r]);
        const float sb = warp_sum_f(SB[r]);
        const float sv = warp_sum_f(SV[r]);
        const float sw = warp_sum_f(SW[r]);
        const int n = warp_sum_n(NN[r]);
        if (lane == r && r < nt) {
            double *raw = a.raw + 4 * (tb + r);
            raw[0] = se;
            raw[1] = sb;
            raw[2] = sv;
            raw[3] = sw;
            a.raw_n[tb + r] = n;
        }
    }
}

// guard-band pairs: the float64 definition decides, the float32 contribution
// of an admitted pair is added to the target's raw sums
template <int KIND>
__global__ void k_proj_band(const MapArgs a, const ProjArgs p) {
    const unsigned long long nall = *a.band_count;
    if (nall > (unsigned long long)a.band_cap && blockIdx.x == 0 && threadIdx.x == 0)
        atomicOr(a.status, SMART_STATUS_BAND_OVERFLOW);
    const unsigned long long nb = min(nall, (unsigned long long)a.band_cap);
    const Plane P = load_plane(p.plane);
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < nb;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const ProjBandPair bp = reinterpret_cast<const ProjBandPair *>(a.band)[i];
        double rx, ry, rz, x0, y0, xi, yi;
        pix2vec64(a.N0, a.targets[bp.target], rx, ry, rz);
        const bool ok0 = plane_xy64(P, rx, ry, rz, x0, y0);
        const double2 rd = a.radec[bp.galaxy];
        radec2vec64(rd.x, rd.y, rx, ry, rz);
        const bool ok1 = plane_xy64(P, rx, ry, rz, xi, yi);
        atomicAdd(a.fp64_count, 1ull);
        if (!ok0 || !ok1) continue;
        const double dx = __dsub_rn(xi, x0), dy = __dsub_rn(yi, y0);
        if (!(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) <= p.Tp)) continue;
        const float4 T = p.txy[bp.target];
        const float4 xy = p.gxy[bp.galaxy];
        const float fdx = (xy.x - T.x) + (xy.z - T.z);
        const float fdy = (xy.y - T.y) + (xy.w - T.w);
        float pe = 0.f, pb = 0.f, pv = 0.f, pw = 0.f;
        int nn = 0;
        proj_pair<KIND>(a, p, fdx, fdy, fmaf(fdx, fdx, fdy * fdy), true, p.gsh[bp.galaxy], pe, pb, pv, pw, nn);
        double *raw = a.raw + 4 * bp.target;
        atomicAdd(raw + 0, (double)pe);
        atomicAdd(raw + 1, (double)pb);
        atomicAdd(raw + 2, (double)pv);
        atomicAdd(raw + 3, (double)pw);
        atomicAdd(a.raw_n + bp.target, 1);
    }
}

// summed normalisation with the plane area A = pi theta_ap^2 (a.area)
__global__ void k_proj_finalise(const MapArgs a) {
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

// ------------------------------------------------------------------------
// Equal-area annuli about a reference point (Sect. 5.2.2): annulus k of
// nbins holds the targets with 1 - cos d in [k, k + 1) (1 - cos rmax) / nbins,
// d the angular distance from the reference point, 1 - cos d = s^2 / 2 from
// the chord s.  buf: [0..2] the reference point's unit vector, [3] sum m_ref,
// [4] sum m_ref^2 over every target, then per annulus (count, sum of d, sum
// of d^2) with d = m_x - m_ref.
// ------------------------------------------------------------------------
constexpr int ANN_HEAD = 5;

__global__ void k_annulus_ref(double ra, double dec, double *buf) {
    radec2vec64(ra, dec, buf[0], buf[1], buf[2]);
}

__global__ void k_annulus_sums(int64_t N0, int64_t n, const int64_t *__restrict__ targets, double cmax, int nbins,
                               const float *__restrict__ mx, const float *__restrict__ mref, double *__restrict__ buf) {
    const double rx = buf[0], ry = buf[1], rz = buf[2];
    double s1 = 0.0, s2 = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const double m = (double)mref[t];
        s1 += m;
        s2 += m * m;
        double x, y, z;
        pix2vec64(N0, targets[t], x, y, z);
        const double dx = __dsub_rn(x, rx), dy = __dsub_rn(y, ry), dz = __dsub_rn(z, rz);
        const double u = __dmul_rn(0.5, __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
        if (!(u < cmax)) continue;
        int k = (int)floor(__dmul_rn(__ddiv_rn(u, cmax), (double)nbins));
        k = min(k, nbins - 1);
        const double d = (double)mx[t] - m;
        double *b = buf + ANN_HEAD + 3 * k;
        atomicAdd(b, 1.0);
        atomicAdd(b + 1, d);
        atomicAdd(b + 2, d * d);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(buf + 3, s1);
        atomicAdd(buf + 4, s2);
    }
}

__global__ void k_annulus_final(int64_t n, int nbins, const double *__restrict__ buf, int64_t *__restrict__ count,
                                double *__restrict__ mean, double *__restrict__ sd) {
    const double m = n > 0 ? buf[3] / (double)n : 0.0;
    const double var = n > 0 ? buf[4] / (double)n - m * m : 0.0;
    const double sref = sqrt(var > 0.0 ? var : 0.0);
    for (int k = threadIdx.x; k < nbins; k += blockDim.x) {
        const double *b = buf + ANN_HEAD + 3 * k;
        const double c = b[0];
        double mu = 0.0, s = 0.0;
        if (c > 0.0) {
            mu = b[1] / c;
            const double v = b[2] / c - mu * mu;
            s = sqrt(v > 0.0 ? v : 0.0);
        }
        if (count) count[k] = (int64_t)c;
        if (mean) mean[k] = sref > 0.0 ? mu / sref : 0.0;
        if (sd) sd[k] = sref > 0.0 ? s / sref : 0.0;
    }
}

}  // namespace
}  // namespace smart

using namespace smart;

extern "C" smart_status smart_map_projected(smart_ctx *c, double ra_c_deg, double dec_c_deg, const smart_maps *out) {
    if (!c) return SMART_E_ARG;
    if (!(fabs(dec_c_deg) <= 90.0) || !isfinite(ra_c_deg)) return fail(c, SMART_E_ARG, "smart_map_projected: bad reference point");
    if (!c->have_catalog) return fail(c, SMART_E_STATE, "smart_map_projected: no catalogue (smart_bin_galaxies first)");
    if (c->norm != SMART_NORM_SUMMED)
        return fail(c, SMART_E_STATE, "smart_map_projected: only the summed normalisation is implemented");
    MapArgs a{};
    smart_status st = common_args(c, out, a);
    if (st != SMART_OK) return st;
    if ((st = build_filter_table(c, true, &c->qtab_plane)) != SMART_OK) return st;
    if (!c->rp_gal) {
        const double th = c->theta_ap + max_pixrad(c->nside_bin) * 1.01 + 1e-9;
        if ((st = build_ring_pairs(c, th, &c->rp_gal, &c->rp_gal_cnt, &c->kmax_gal)) != SMART_OK) return st;
    }
    if (c->gal_tiles_version != c->targets_version) {
        if ((st = build_tiles_log2(c, PT_LOG2, &c->gal_tiles, &c->cap_gal_tiles, &c->n_gal_tiles)) != SMART_OK) return st;
        c->gal_tiles_version = c->targets_version;
    }
    const int64_t n = c->n_targets, ng = c->n_gal;
    if ((st = ensure_alloc(c, (void **)&c->raw, c->cap_raw, 5 * n + 1, sizeof(double), "raw sums")) != SMART_OK ||
        (st = ensure_alloc(c, (void **)&c->band, c->cap_band, std::max<int64_t>(1 << 20, 16 * n),
                           sizeof(ProjBandPair), "guard-band list")) != SMART_OK ||
        (st = ensure_alloc(c, (void **)&c->proj_xy, c->cap_proj, ng, sizeof(float4), "plane positions")) != SMART_OK ||
        (st = ensure_alloc(c, (void **)&c->proj_sh, c->cap_proj_sh, ng, sizeof(float4), "plane shears")) != SMART_OK ||
        (st = ensure_alloc(c, (void **)&c->proj_txy, c->cap_proj_t, n, sizeof(float4), "target positions")) != SMART_OK)
        return st;
    if (!c->proj_plane && cudaMalloc(&c->proj_plane, 9 * sizeof(double)) != cudaSuccess)
        return fail(c, SMART_E_NOMEM, "cudaMalloc(plane) failed");
    ProjArgs p{};
    p.gxy = c->proj_xy;
    p.gsh = c->proj_sh;
    p.txy = c->proj_txy;
    p.plane = c->proj_plane;
    p.Tp = c->theta_ap * c->theta_ap;
    p.Tlo = (float)(p.Tp * (1.0 - 4e-6));
    p.Thi = (float)(p.Tp * (1.0 + 4e-6));
    p.qtab = c->qtab_plane;
    p.tab_scale = (float)(QTAB_BINS / c->theta_ap);
    a.area = SMART_PI * p.Tp;
    a.table = c->rp_gal;
    a.counts = c->rp_gal_cnt;
    a.kmax = c->kmax_gal;
    a.offsets = c->offsets;
    a.radec = c->rec_radec;
    a.tiles = c->gal_tiles;
    a.n_tiles = c->n_gal_tiles;
    a.raw = c->raw;
    a.raw_n = reinterpret_cast<int32_t *>(c->raw + 4 * n);
    a.band = c->band;
    a.band_cap = c->cap_band;
    a.band_count = c->d_band_count;
    cudaStream_t s = c->stream;
    cudaMemsetAsync(c->d_fp64_count, 0, sizeof(unsigned long long), s);
    cudaMemsetAsync(c->d_band_count, 0, sizeof(unsigned long long), s);
    if (n == 0) return check_cuda(c, cudaGetLastError(), "projected map");
    {
        KernelTimer timer(c, SMART_KT_PROJ_RECORDS);
        k_plane_setup<<<1, 1, 0, s>>>(ra_c_deg, dec_c_deg, c->proj_plane);
        const unsigned gg = (unsigned)std::max<int64_t>(1, std::min<int64_t>((ng + 255) / 256, (int64_t)c->num_sms * 16));
        if (ng > 0) k_proj_records<<<gg, 256, 0, s>>>(ng, c->rec_radec, c->rec_shear, c->proj_plane, c->proj_xy, c->proj_sh);
        const unsigned gt = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)c->num_sms * 16);
        k_proj_targets<<<gt, 256, 0, s>>>(c->nside_out, n, c->targets, c->proj_plane, c->proj_txy);
    }
    if ((st = check_cuda(c, cudaGetLastError(), "projected records")) != SMART_OK) return st;
    const bool poly = c->filter_kind == SMART_FILTER_POLY;
    const unsigned blocks = (unsigned)((a.n_tiles + PW - 1) / PW);
    {
        KernelTimer timer(c, SMART_KT_PROJ_MAP);
        if (poly) k_map_projected<SMART_FILTER_POLY><<<blocks, 32 * PW, 0, s>>>(a, p);
        else k_map_projected<SMART_FILTER_SCHIRMER><<<blocks, 32 * PW, 0, s>>>(a, p);
    }
    {
        KernelTimer timer(c, SMART_KT_PROJ_BAND);
        if (poly) k_proj_band<SMART_FILTER_POLY><<<(unsigned)c->num_sms, 256, 0, s>>>(a, p);
        else k_proj_band<SMART_FILTER_SCHIRMER><<<(unsigned)c->num_sms, 256, 0, s>>>(a, p);
    }
    const unsigned fb = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)c->num_sms * 16);
    k_proj_finalise<<<fb, 256, 0, s>>>(a);
    return check_cuda(c, cudaGetLastError(), "projected map launches");
}

extern "C" smart_status smart_annulus_stats(smart_ctx *c, double ra_ref_deg, double dec_ref_deg, double rmax_rad,
                                            const float *m_x, const float *m_ref, int nbins, int64_t *count,
                                            double *mean, double *sd) {
    if (!c) return SMART_E_ARG;
    if (nbins < 1 || nbins > (1 << 20) || !(rmax_rad > 0.0 && rmax_rad <= SMART_PI) || !(fabs(dec_ref_deg) <= 90.0) ||
        !isfinite(ra_ref_deg) || (c->n_targets > 0 && (!m_x || !m_ref)))
        return fail(c, SMART_E_ARG, "smart_annulus_stats: bad arguments");
    const int64_t nbuf = ANN_HEAD + 3 * (int64_t)nbins;
    smart_status st = ensure_alloc(c, (void **)&c->annulus_buf, c->cap_annulus, nbuf, sizeof(double), "annulus sums");
    if (st != SMART_OK) return st;
    cudaStream_t s = c->stream;
    if ((st = check_cuda(c, cudaMemsetAsync(c->annulus_buf, 0, (size_t)nbuf * sizeof(double), s), "annulus sums")) !=
        SMART_OK)
        return st;
    // 1 - cos rmax: one host libm call, the same double for every target
    const double cmax = 1.0 - cos(rmax_rad);
    k_annulus_ref<<<1, 1, 0, s>>>(ra_ref_deg, dec_ref_deg, c->annulus_buf);
    const int64_t n = c->n_targets;
    if (n > 0) {
        const unsigned g = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)c->num_sms * 8);
        k_annulus_sums<<<g, 256, 0, s>>>(c->nside_out, n, c->targets, cmax, nbins, m_x, m_ref, c->annulus_buf);
    }
    k_annulus_final<<<1, 256, 0, s>>>(n, nbins, c->annulus_buf, count, mean, sd);
    return check_cuda(c, cudaGetLastError(), "annulus statistics");
}
