/*
 * smart_oracle.c -- plain FP64 CPU oracle for the spherical shear-based
 * aperture-mass method (SMART, arXiv 2609.11181).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * definition that the CUDA path is checked against.  Only the test-suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or constant generator with the CUDA library.
 *
 * Everything is evaluated in IEEE binary64, compiled with
 * -ffp-contract=off so that no multiply-add is fused behind our back; the
 * only fused operations are the explicit fma() calls of the sine/cosine
 * series below.
 *
 * Sections of the paper followed (by section / equation):
 *   Sect. 2, Eq. 3, Eq. 4                      tangential / cross shear
 *   Sect. 2, Eq. 5                             the Q filter
 *   Sect. 2.2, Eq. 7, Eq. 8                    discrete sums, noise map
 *   Sect. 2.3, Eq. 10, Eq. 11                  spherical geometry
 *   Sect. 2.4                                  summed normalisation
 *   Sect. 3 (HEALPix, Gorski et al. 2005)      RING pixelisation
 *   Sect. 3.1 steps 1-5                        brute force (sphS_pos)
 *   Sect. 3.2 steps 1-5                        pixel-based (sphS_pix)
 *   Sect. 3.4 steps 1-3                        sorted catalogue + offsets
 *   Sect. 2.2.1, 2.2.2, Sect. 5.2.1 steps 1-4  Cartesian (projected) estimator
 *   Sect. 5.2.2                                equal-area annulus statistics
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* Sine and cosine in binary64.                                        */
/*                                                                     */
/* Method: exact argument reduction to a signed remainder of at most   */
/* half a quadrant (the subtraction is exact by Sterbenz's lemma),     */
/* followed by the Maclaurin series of sin and cos, truncated where    */
/* the next term is below 2^-60 on |t| <= pi/4, evaluated by Horner's  */
/* rule with fused multiply-adds.  Same algorithm is written,          */
/* separately, in the CUDA library, so that pixel centres and the      */
/* membership predicate come out bit-identical on both sides.          */
/* ------------------------------------------------------------------ */
static void series_sincos(double t, double *s, double *c)
{
    double t2 = t * t;
    /* sin t = t + t^3 * (-1/3! + t^2 (1/5! - t^2 (...)))  up to t^19 */
    double ps = -1.0 / 121645100408832000.0;              /* -1/19! */
    ps = fma(ps, t2, 1.0 / 355687428096000.0);            /*  1/17! */
    ps = fma(ps, t2, -1.0 / 1307674368000.0);             /* -1/15! */
    ps = fma(ps, t2, 1.0 / 6227020800.0);                 /*  1/13! */
    ps = fma(ps, t2, -1.0 / 39916800.0);                  /* -1/11! */
    ps = fma(ps, t2, 1.0 / 362880.0);                     /*  1/9!  */
    ps = fma(ps, t2, -1.0 / 5040.0);                      /* -1/7!  */
    ps = fma(ps, t2, 1.0 / 120.0);                        /*  1/5!  */
    ps = fma(ps, t2, -1.0 / 6.0);                         /* -1/3!  */
    *s = fma(t * t2, ps, t);
    /* cos t = 1 + t^2 * (-1/2! + t^2 (1/4! - ...))  up to t^20 */
    double pc = 1.0 / 2432902008176640000.0;              /*  1/20! */
    pc = fma(pc, t2, -1.0 / 6402373705728000.0);          /* -1/18! */
    pc = fma(pc, t2, 1.0 / 20922789888000.0);             /*  1/16! */
    pc = fma(pc, t2, -1.0 / 87178291200.0);               /* -1/14! */
    pc = fma(pc, t2, 1.0 / 479001600.0);                  /*  1/12! */
    pc = fma(pc, t2, -1.0 / 3628800.0);                   /* -1/10! */
    pc = fma(pc, t2, 1.0 / 40320.0);                      /*  1/8!  */
    pc = fma(pc, t2, -1.0 / 720.0);                       /* -1/6!  */
    pc = fma(pc, t2, 1.0 / 24.0);                         /*  1/4!  */
    pc = fma(pc, t2, -0.5);                               /* -1/2!  */
    *c = fma(t2, pc, 1.0);
}

static void quadrant_apply(double q, double s, double c, double *so, double *co)
{
    double qm = fmod(q, 4.0);
    if (qm < 0.0) qm += 4.0;
    int k = (int)qm;
    switch (k) {
    case 0: *so = s;  *co = c;  break;
    case 1: *so = c;  *co = -s; break;
    case 2: *so = -s; *co = -c; break;
    default: *so = -c; *co = s; break;
    }
}

/* angle given in degrees */
void orc_sincos_deg(double x, double *s, double *c)
{
    double q = nearbyint(x / 90.0);
    double y = x - q * 90.0;                 /* exact */
    double t = y * (ORC_PI / 180.0);
    double ss, cc;
    series_sincos(t, &ss, &cc);
    quadrant_apply(q, ss, cc, s, c);
}

/* angle given in quarter turns: angle = f * pi/2 */
void orc_sincos_quarter(double f, double *s, double *c)
{
    double q = nearbyint(f);
    double y = f - q;                        /* exact */
    double t = y * (ORC_PI / 2.0);
    double ss, cc;
    series_sincos(t, &ss, &cc);
    quadrant_apply(q, ss, cc, s, c);
}

/* ------------------------------------------------------------------ */
/* HEALPix RING scheme (Gorski et al. 2005).  Rings i = 1 .. 4N-1 from  */
/* the north pole.  Polar rings (i < N) hold 4i pixels at              */
/* z = 1 - i^2/(3N^2), phi_j = (pi/2i)(j + 1/2), j = 0..4i-1.           */
/* Equatorial rings (N <= i <= 3N) hold 4N pixels at                   */
/* z = (4N - 2i)/(3N), phi_j = (pi/2N)(j + 1/2) when i - N is even,     */
/* phi_j = (pi/2N) j otherwise.  Southern rings mirror the north.      */
/* ------------------------------------------------------------------ */
static int64_t isqrt64(int64_t v)
{
    int64_t r = (int64_t)sqrt((double)v);
    while (r * r > v) --r;
    while ((r + 1) * (r + 1) <= v) ++r;
    return r;
}

/*
 * Geometry of pixel `pix`: ring index (1-based from north), index within
 * the ring, number of pixels in the ring, z, rho = sqrt(1-z^2) and the
 * azimuth in quarter turns (phi / (pi/2)).
 */
void orc_pix_info(int64_t nside, int64_t pix, int64_t *ring, int64_t *jring,
                  int64_t *nring, double *z, double *rho, double *fq)
{
    const int64_t N = nside;
    const int64_t ncap = 2 * N * (N - 1);
    const int64_t npix = 12 * N * N;
    int64_t i, j, nr;
    double zz, rr, f;
    if (pix < ncap) {
        i = (1 + isqrt64(1 + 2 * pix)) >> 1;
        j = pix - 2 * i * (i - 1);
        nr = 4 * i;
        zz = 1.0 - (double)(i * i) / (double)(3 * N * N);
        rr = (double)i * sqrt((double)(6 * N * N - i * i)) / (double)(3 * N * N);
        f = (double)(2 * j + 1) / (double)(2 * i);
    } else if (pix < npix - ncap) {
        int64_t ip = pix - ncap;
        i = ip / (4 * N) + N;
        j = ip % (4 * N);
        nr = 4 * N;
        zz = (double)(4 * N - 2 * i) / (double)(3 * N);
        rr = sqrt((double)((2 * i - N) * (7 * N - 2 * i))) / (double)(3 * N);
        if (((i - N) & 1) == 0) f = (double)(2 * j + 1) / (double)(2 * N);
        else f = (double)j / (double)N;
    } else {
        int64_t ip = npix - pix;
        int64_t is = (1 + isqrt64(2 * ip - 1)) >> 1;   /* ring counted from south */
        j = pix - (npix - 2 * is * (is + 1));
        nr = 4 * is;
        i = 4 * N - is;
        zz = -(1.0 - (double)(is * is) / (double)(3 * N * N));
        rr = (double)is * sqrt((double)(6 * N * N - is * is)) / (double)(3 * N * N);
        f = (double)(2 * j + 1) / (double)(2 * is);
    }
    if (ring) *ring = i;
    if (jring) *jring = j;
    if (nring) *nring = nr;
    if (z) *z = zz;
    if (rho) *rho = rr;
    if (fq) *fq = f;
}

/* unit vector (x, y, z) of the centre of pixel `pix` */
void orc_pix2vec(int64_t nside, int64_t pix, double *v)
{
    double z, rho, f, s, c;
    orc_pix_info(nside, pix, 0, 0, 0, &z, &rho, &f);
    orc_sincos_quarter(f, &s, &c);
    v[0] = rho * c;
    v[1] = rho * s;
    v[2] = z;
}

/* first pixel, pixel count, z and shift flag of ring i (1-based) */
void orc_ring_info(int64_t nside, int64_t i, int64_t *start, int64_t *nr,
                   double *z, int *shifted)
{
    const int64_t N = nside;
    const int64_t npix = 12 * N * N;
    if (i < N) {
        *start = 2 * i * (i - 1);
        *nr = 4 * i;
        *z = 1.0 - (double)(i * i) / (double)(3 * N * N);
        *shifted = 1;
    } else if (i <= 3 * N) {
        *start = 2 * N * (N - 1) + (i - N) * 4 * N;
        *nr = 4 * N;
        *z = (double)(4 * N - 2 * i) / (double)(3 * N);
        *shifted = ((i - N) & 1) == 0;
    } else {
        int64_t is = 4 * N - i;
        *start = npix - 2 * is * (is + 1);
        *nr = 4 * is;
        *z = -(1.0 - (double)(is * is) / (double)(3 * N * N));
        *shifted = 1;
    }
}

/* RING pixel containing the direction (ra, dec) given in degrees */
int64_t orc_ang2pix(int64_t nside, double ra_deg, double dec_deg)
{
    const int64_t N = nside;
    const int64_t npix = 12 * N * N;
    const int64_t ncap = 2 * N * (N - 1);
    double sd, cd;
    orc_sincos_deg(dec_deg, &sd, &cd);
    double z = sd, sth = cd;
    double a = fmod(ra_deg, 360.0);
    if (a < 0.0) a += 360.0;
    double tt = a / 90.0;                    /* phi in quarter turns */
    if (tt >= 4.0) tt -= 4.0;
    double za = fabs(z);
    if (za <= 2.0 / 3.0) {
        double t1 = (double)N * (0.5 + tt);
        double t2 = ((double)N * z) * 0.75;
        int64_t jp = (int64_t)floor(t1 - t2);
        int64_t jm = (int64_t)floor(t1 + t2);
        int64_t ir = N + 1 + jp - jm;        /* 1 .. 2N+1, counted from ring N */
        int64_t kshift = 1 - (ir & 1);
        int64_t ip = (jp + jm - N + kshift + 1) / 2;
        ip = ((ip % (4 * N)) + 4 * N) % (4 * N);
        return ncap + (ir - 1) * 4 * N + ip;
    } else {
        double tp = tt - floor(tt);
        double tmp = ((double)N * sth) * sqrt(3.0 / (1.0 + za));
        int64_t jp = (int64_t)floor(tp * tmp);
        int64_t jm = (int64_t)floor((1.0 - tp) * tmp);
        int64_t ir = jp + jm + 1;            /* ring counted from the nearest pole */
        int64_t ip = (int64_t)floor(tt * (double)ir);
        ip = ((ip % (4 * ir)) + 4 * ir) % (4 * ir);
        if (z > 0.0) return 2 * ir * (ir - 1) + ip;
        return npix - 2 * ir * (ir + 1) + ip;
    }
}

void orc_ang2pix_many(int64_t nside, int64_t n, const double *ra,
                      const double *dec, int64_t *pix)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) pix[k] = orc_ang2pix(nside, ra[k], dec[k]);
}

void orc_pix2vec_many(int64_t nside, int64_t n, const int64_t *pix, double *v)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) orc_pix2vec(nside, pix[k], v + 3 * k);
}

void orc_radec2vec(double ra, double dec, double *v)
{
    double sa, ca, sd, cd;
    orc_sincos_deg(ra, &sa, &ca);
    orc_sincos_deg(dec, &sd, &cd);
    v[0] = cd * ca;
    v[1] = cd * sa;
    v[2] = sd;
}

/* ------------------------------------------------------------------ */
/* Filters.  Q(theta) = q(theta / theta_ap) / theta_ap^2, truncated at  */
/* theta = theta_ap (the membership predicate does the truncation).    */
/*   kind 1: Schneider (1996) polynomial  q = 6/pi x^2 (1 - x^2)        */
/*   kind 2: Schirmer et al. (2007)                                     */
/*           q = tanh(x/xc)/(x/xc) / (1 + e^(6-150x) + e^(-47+50x))     */
/* ------------------------------------------------------------------ */
double orc_filter_q(int kind, double xc, double x)
{
    if (kind == 1) {
        double x2 = x * x;
        return 6.0 / ORC_PI * x2 * (1.0 - x2);
    }
    if (kind == 2) {
        double r = x / xc;
        double th = (r == 0.0) ? 1.0 : tanh(r) / r;
        return th / (1.0 + exp(6.0 - 150.0 * x) + exp(-47.0 + 50.0 * x));
    }
    if (kind == 3) {
        /* Jarvis et al. (2004), Gaussian-type, scale s = xc (in theta_ap units) */
        double s2 = xc * xc;
        return x * x / s2 * exp(-0.5 * x * x / s2) / (4.0 * ORC_PI * s2);
    }
    return 0.0;
}

/* Schneider (1996) compensated U that generates the polynomial Q */
double orc_filter_u_poly(double x)
{
    double x2 = x * x;
    return 9.0 / ORC_PI * (1.0 - x2) * (1.0 / 3.0 - x2);
}

/* ------------------------------------------------------------------ */
/* One aperture term (Sect. 2.3 geometry, Eq. 4).                  */
/* r0: unit vector of the aperture centre; p: unit vector of the point; */
/* ehat, nhat: the point's local East and North unit vectors.           */
/* Returns 1 when the point lies in the aperture (s^2 <= T).            */
/* ------------------------------------------------------------------ */
typedef struct {
    int kind;
    double xc;
    double theta_ap;
    double T;          /* 4 sin^2(theta_ap / 2), the chord^2 threshold */
} orc_cfg;

static int aperture_term(const orc_cfg *cfg, const double *r0, const double *p,
                         const double *ehat, const double *nhat,
                         double *qval, double *c2, double *s2)
{
    double dx = p[0] - r0[0];
    double dy = p[1] - r0[1];
    double dz = p[2] - r0[2];
    double ssq = dx * dx + dy * dy + dz * dz;   /* chord^2, this order */
    if (!(ssq <= cfg->T)) return 0;
    double d = 2.0 * asin(sqrt(ssq) / 2.0);     /* great-circle separation */
    *qval = orc_filter_q(cfg->kind, cfg->xc, d / cfg->theta_ap)
            / (cfg->theta_ap * cfg->theta_ap);
    /* direction from the point towards the centre in the point's tangent
       plane; the paper's tan(psi) equals -x/y (Sect. 2.3) */
    if (ssq == 0.0) {
        /* the point is the centre itself: psi is undefined (Sect. 2.3 gives
           0/0), the point carries no tangential or cross shear */
        *c2 = 0.0;
        *s2 = 0.0;
        return 1;
    }
    double x = ehat[0] * r0[0] + ehat[1] * r0[1] + ehat[2] * r0[2];
    double y = nhat[0] * r0[0] + nhat[1] * r0[1] + nhat[2] * r0[2];
    double den = x * x + y * y;
    if (den == 0.0) {
        /* a point within rounding of the centre: no direction, no shear */
        *c2 = 0.0;
        *s2 = 0.0;
        return 1;
    }
    *c2 = (y * y - x * x) / den;                /* cos 2 psi */
    *s2 = -2.0 * x * y / den;                   /* sin 2 psi */
    return 1;
}

static int cmp_dbl_idx(const void *a, const void *b)
{
    const double *x = (const double *)a, *y = (const double *)b;
    if (x[0] < y[0]) return -1;
    if (x[0] > y[0]) return 1;
    if (x[1] < y[1]) return -1;
    if (x[1] > y[1]) return 1;
    return 0;
}

/*
 * Pixel barycentres (Sect. 3.3): for every pixel holding galaxies, the
 * w-weighted mean of the galaxies' unit vectors, normalised to the sphere
 * (the paper averages RA and Dec; the mean of unit vectors agrees with that
 * to second order in the pixel size and has no RA wrap).  The sum runs over
 * the galaxies in the order of perm (pixel-sorted, input order within a
 * pixel), one product and one addition at a time.  vec[3 p .. 3 p + 2] is
 * written for pixels with galaxies; other entries are left as they are.
 */
void orc_barycentres(int64_t nside, const double *ra, const double *dec, const double *w,
                     const int64_t *perm, const int64_t *offsets, double *vec)
{
    int64_t npix = 12 * nside * nside;
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t p = 0; p < npix; ++p) {
        if (offsets[p + 1] == offsets[p]) continue;
        double sx = 0.0, sy = 0.0, sz = 0.0;
        for (int64_t a = offsets[p]; a < offsets[p + 1]; ++a) {
            int64_t k = perm[a];
            double r[3];
            orc_radec2vec(ra[k], dec[k], r);
            sx = sx + w[k] * r[0];
            sy = sy + w[k] * r[1];
            sz = sz + w[k] * r[2];
        }
        double nrm = sqrt((sx * sx + sy * sy) + sz * sz);
        vec[3 * p] = sx / nrm;
        vec[3 * p + 1] = sy / nrm;
        vec[3 * p + 2] = sz / nrm;
    }
}

/*
 * Aperture sums over weighted points: the barycentre form of the pixel-based
 * map (Sect. 3.3, sphS_pixB).  Point k sits at the unit vector v[3k..] and
 * carries its pixel's sums G1 = sum w e1, G2 = sum w e2, W = sum w,
 * S2 = sum w^2 |e|^2 and galaxy count np[k].  Membership by the point's
 * position (s^2 <= T), as for galaxies:
 *   SE = sum (G1 cos 2psi + G2 sin 2psi) Q,  SB = sum (-G1 sin 2psi + G2 cos 2psi) Q,
 *   SV = sum S2 Q^2,  SW = sum W,  N = sum np,  K = number of member points.
 * The local East / North of a point come from its unit vector.
 */
void orc_aperture_points(int64_t n0, const double *c, int64_t m, const double *v,
                         const double *G1, const double *G2, const double *W,
                         const double *S2, const int64_t *np,
                         int kind, double xc, double theta_ap,
                         double *SE, double *SB, double *SV, double *SW,
                         int64_t *N, int64_t *K)
{
    orc_cfg cfg;
    cfg.kind = kind;
    cfg.xc = xc;
    cfg.theta_ap = theta_ap;
    double sh = sin(0.5 * theta_ap);
    cfg.T = 4.0 * sh * sh;
    double *gv = (double *)malloc(sizeof(double) * 9 * (size_t)(m > 0 ? m : 1));
    double *zi = (double *)malloc(sizeof(double) * 2 * (size_t)(m > 0 ? m : 1));
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < m; ++k) {
        const double *p = v + 3 * k;
        double *g = gv + 9 * k;
        double rho = sqrt(p[0] * p[0] + p[1] * p[1]);
        double ca = rho > 0.0 ? p[0] / rho : 1.0, sa = rho > 0.0 ? p[1] / rho : 0.0;
        g[0] = p[0]; g[1] = p[1]; g[2] = p[2];
        g[3] = -sa;        g[4] = ca;         g[5] = 0.0;      /* East  */
        g[6] = -p[2] * ca; g[7] = -p[2] * sa; g[8] = rho;      /* North */
    }
    for (int64_t k = 0; k < m; ++k) {
        zi[2 * k] = gv[9 * k + 2];
        zi[2 * k + 1] = (double)k;
    }
    qsort(zi, (size_t)m, 2 * sizeof(double), cmp_dbl_idx);
    double band = sqrt(cfg.T) * (1.0 + 1e-9) + 1e-15;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < n0; ++t) {
        const double *r0 = c + 3 * t;
        double zlo = r0[2] - band, zhi = r0[2] + band;
        int64_t lo = 0, hi = m;
        while (lo < hi) {
            int64_t mid = (lo + hi) / 2;
            if (zi[2 * mid] < zlo) lo = mid + 1; else hi = mid;
        }
        double se = 0, sb = 0, sv = 0, sw = 0;
        int64_t cnt = 0, mem = 0;
        for (int64_t q = lo; q < m && zi[2 * q] <= zhi; ++q) {
            int64_t k = (int64_t)zi[2 * q + 1];
            const double *g = gv + 9 * k;
            double qv, c2, s2;
            if (!aperture_term(&cfg, r0, g, g + 3, g + 6, &qv, &c2, &s2)) continue;
            se += (G1[k] * c2 + G2[k] * s2) * qv;
            sb += (-G1[k] * s2 + G2[k] * c2) * qv;
            sv += S2[k] * qv * qv;
            sw += W[k];
            cnt += np[k];
            mem += 1;
        }
        SE[t] = se; SB[t] = sb; SV[t] = sv; SW[t] = sw; N[t] = cnt; K[t] = mem;
    }
    free(gv);
    free(zi);
}

/*
 * Brute force at galaxy positions (Sect. 3.1, sphS_pos), summed form.
 * For each of the n0 centres (unit vectors c, 3 per centre) sum over all
 * galaxies inside the aperture:
 *   SE = sum w e_+ Q,  SB = sum w e_x Q,  SV = sum w^2 |e|^2 Q^2,
 *   SW = sum w,        N  = number of members.
 * Candidates are restricted to |z_i - z_0| <= sqrt(T) (every member
 * satisfies it, because s^2 >= (z_i - z_0)^2) and then tested exactly.
 */
void orc_aperture_galaxies(int64_t n0, const double *c, int64_t n,
                           const double *ra, const double *dec,
                           const double *e1, const double *e2, const double *w,
                           int kind, double xc, double theta_ap,
                           double *SE, double *SB, double *SV, double *SW,
                           int64_t *N)
{
    orc_cfg cfg;
    cfg.kind = kind;
    cfg.xc = xc;
    cfg.theta_ap = theta_ap;
    double sh = sin(0.5 * theta_ap);
    cfg.T = 4.0 * sh * sh;
    double *gv = (double *)malloc(sizeof(double) * 9 * (size_t)(n > 0 ? n : 1));
    double *zi = (double *)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        double sa, ca, sd, cd;
        orc_sincos_deg(ra[k], &sa, &ca);
        orc_sincos_deg(dec[k], &sd, &cd);
        double *g = gv + 9 * k;
        g[0] = cd * ca; g[1] = cd * sa; g[2] = sd;          /* position */
        g[3] = -sa;     g[4] = ca;      g[5] = 0.0;         /* East  */
        g[6] = -sd * ca; g[7] = -sd * sa; g[8] = cd;        /* North */
    }
    for (int64_t k = 0; k < n; ++k) {
        zi[2 * k] = gv[9 * k + 2];
        zi[2 * k + 1] = (double)k;
    }
    qsort(zi, (size_t)n, 2 * sizeof(double), cmp_dbl_idx);
    double band = sqrt(cfg.T) * (1.0 + 1e-9) + 1e-15;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < n0; ++t) {
        const double *r0 = c + 3 * t;
        double zlo = r0[2] - band, zhi = r0[2] + band;
        int64_t lo = 0, hi = n;
        while (lo < hi) {                        /* first z >= zlo */
            int64_t mid = (lo + hi) / 2;
            if (zi[2 * mid] < zlo) lo = mid + 1; else hi = mid;
        }
        double se = 0, sb = 0, sv = 0, sw = 0;
        int64_t cnt = 0;
        for (int64_t m = lo; m < n && zi[2 * m] <= zhi; ++m) {
            int64_t k = (int64_t)zi[2 * m + 1];
            const double *g = gv + 9 * k;
            double q, c2, s2;
            if (!aperture_term(&cfg, r0, g, g + 3, g + 6, &q, &c2, &s2)) continue;
            double gp = e1[k] * c2 + e2[k] * s2;     /* gamma_+ */
            double gx = -e1[k] * s2 + e2[k] * c2;    /* gamma_x */
            se += w[k] * gp * q;
            sb += w[k] * gx * q;
            sv += w[k] * w[k] * (e1[k] * e1[k] + e2[k] * e2[k]) * q * q;
            sw += w[k];
            cnt += 1;
        }
        SE[t] = se; SB[t] = sb; SV[t] = sv; SW[t] = sw; N[t] = cnt;
    }
    free(gv);
    free(zi);
}

/*
 * Pixels of a RING map at `nside` whose centres lie within the aperture
 * around unit vector r0 (the "centre in disc" convention).  The candidate
 * window on each ring follows from the spherical law of cosines with two
 * pixels of margin on each side; every candidate is then tested with the
 * exact predicate s^2 <= T.  Returns the member count; writes at most
 * `cap` indices to out (ascending ring, then ascending azimuth index).
 */
int64_t orc_query_disc(int64_t nside, const double *r0, double T,
                       int64_t *out, int64_t cap)
{
    const int64_t N = nside;
    int64_t count = 0;
    double rho0 = sqrt((1.0 - r0[2]) * (1.0 + r0[2]));
    double band = sqrt(T) * (1.0 + 1e-9) + 1e-15;
    double phi0q = 0.0;                      /* azimuth of r0 in quarter turns */
    if (rho0 > 0.0) {
        phi0q = atan2(r0[1], r0[0]) / (ORC_PI / 2.0);
        if (phi0q < 0.0) phi0q += 4.0;
    }
    for (int64_t i = 1; i <= 4 * N - 1; ++i) {
        int64_t start, nr;
        double z;
        int sh;
        orc_ring_info(N, i, &start, &nr, &z, &sh);
        if (fabs(z - r0[2]) > band) continue;
        double rho = sqrt((1.0 - z) * (1.0 + z));
        /* s^2 = (z - z0)^2 + (rho - rho0)^2 + 4 rho rho0 sin^2(dphi/2) */
        double base = (z - r0[2]) * (z - r0[2]) + (rho - rho0) * (rho - rho0);
        double prod = 4.0 * rho * rho0;
        int whole = 0;
        double half = 0.0;                   /* half window, quarter turns */
        if (prod <= 0.0) {
            whole = 1;
        } else {
            double sn2 = (T - base) / prod;
            if (sn2 >= 1.0) whole = 1;
            else if (sn2 < 0.0) half = 0.0;
            else half = 2.0 * asin(sqrt(sn2)) / (ORC_PI / 2.0);
        }
        int64_t jlo, jhi;
        if (whole) {
            jlo = 0; jhi = nr - 1;
        } else {
            double off = sh ? 0.5 : 0.0;
            double per = (double)nr / 4.0;   /* pixels per quarter turn */
            jlo = (int64_t)floor((phi0q - half) * per - off) - 2;
            jhi = (int64_t)ceil((phi0q + half) * per - off) + 2;
            if (jhi - jlo + 1 >= nr) { jlo = 0; jhi = nr - 1; }
        }
        /* collect the ring's members in ascending azimuth index */
        int64_t first = count;
        for (int64_t jj = jlo; jj <= jhi; ++jj) {
            int64_t j = ((jj % nr) + nr) % nr;
            int64_t pix = start + j;
            double v[3];
            orc_pix2vec(N, pix, v);
            double dx = v[0] - r0[0], dy = v[1] - r0[1], dz = v[2] - r0[2];
            double ssq = dx * dx + dy * dy + dz * dz;
            if (ssq <= T) {
                if (count < cap) out[count] = pix;
                ++count;
            }
        }
        /* the window may wrap: sort this ring's members ascending */
        if (count <= cap) {
            for (int64_t a = first + 1; a < count; ++a) {
                int64_t key = out[a], b = a - 1;
                while (b >= first && out[b] > key) { out[b + 1] = out[b]; --b; }
                out[b + 1] = key;
            }
        }
    }
    return count;
}

/* every pixel tested: the plain definition, used to pin orc_query_disc */
int64_t orc_query_disc_all(int64_t nside, const double *r0, double T,
                           int64_t *out, int64_t cap)
{
    int64_t npix = 12 * nside * nside, count = 0;
    for (int64_t p = 0; p < npix; ++p) {
        double v[3];
        orc_pix2vec(nside, p, v);
        double dx = v[0] - r0[0], dy = v[1] - r0[1], dz = v[2] - r0[2];
        double ssq = dx * dx + dy * dy + dz * dz;
        if (ssq <= T) {
            if (count < cap) out[count] = p;
            ++count;
        }
    }
    return count;
}

/*
 * Pixel-based aperture mass (Sect. 3.2, sphS_pix), summed form.  Input is
 * a full-sky RING map at nside_bin of per-pixel sums
 *   G1 = sum w e1, G2 = sum w e2, W = sum w, S2 = sum w^2 |e|^2, n = count.
 * The filter and the rotation are evaluated at the pixel centres.  Output
 * per centre: SE = sum Q (G1 cos2psi + G2 sin2psi), SB, SV = sum Q^2 S2,
 * SW = sum W, N = sum n.
 */
static double rd(const void *a, int f32, int64_t p)
{
    return f32 ? (double)((const float *)a)[p] : ((const double *)a)[p];
}

static int64_t rn(const void *a, int f32, int64_t p)
{
    return f32 ? (int64_t)((const int32_t *)a)[p] : ((const int64_t *)a)[p];
}

static void aperture_pixels_impl(int64_t n0, const double *c, int64_t nside_bin,
                                 const void *G1, const void *G2, const void *W,
                                 const void *S2, const void *np, int f32,
                                 int kind, double xc, double theta_ap,
                                 double *SE, double *SB, double *SV, double *SW,
                                 int64_t *N, int64_t *NPIX)
{
    orc_cfg cfg;
    cfg.kind = kind;
    cfg.xc = xc;
    cfg.theta_ap = theta_ap;
    double sh = sin(0.5 * theta_ap);
    cfg.T = 4.0 * sh * sh;
    /* generous bound on the member count: disc area / pixel area, doubled,
       plus a full ring's worth for apertures around a pole */
    double area = 2.0 * ORC_PI * cfg.T / 2.0;            /* 2 pi (1 - cos) */
    double apix = 4.0 * ORC_PI / (12.0 * (double)nside_bin * (double)nside_bin);
    int64_t cap = (int64_t)(2.0 * area / apix) + 16 * nside_bin + 64;
#pragma omp parallel
    {
        int64_t *buf = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
#pragma omp for schedule(dynamic, 16)
        for (int64_t t = 0; t < n0; ++t) {
            const double *r0 = c + 3 * t;
            int64_t m = orc_query_disc(nside_bin, r0, cfg.T, buf, cap);
            if (m > cap) m = cap;               /* cannot happen with the bound */
            double se = 0, sb = 0, sv = 0, sw = 0;
            int64_t cnt = 0;
            for (int64_t a = 0; a < m; ++a) {
                int64_t p = buf[a];
                double z, rho, f, sp, cp;
                orc_pix_info(nside_bin, p, 0, 0, 0, &z, &rho, &f);
                orc_sincos_quarter(f, &sp, &cp);
                double v[3] = {rho * cp, rho * sp, z};
                double eh[3] = {-sp, cp, 0.0};
                double nh[3] = {-z * cp, -z * sp, rho};
                double q, c2, s2;
                if (!aperture_term(&cfg, r0, v, eh, nh, &q, &c2, &s2)) continue;
                double g1 = rd(G1, f32, p), g2 = rd(G2, f32, p);
                se += q * (g1 * c2 + g2 * s2);
                sb += q * (-g1 * s2 + g2 * c2);
                sv += q * q * rd(S2, f32, p);
                sw += rd(W, f32, p);
                cnt += rn(np, f32, p);
            }
            SE[t] = se; SB[t] = sb; SV[t] = sv; SW[t] = sw; N[t] = cnt;
            if (NPIX) NPIX[t] = m;
        }
        free(buf);
    }
}

void orc_aperture_pixels(int64_t n0, const double *c, int64_t nside_bin,
                         const double *G1, const double *G2, const double *W,
                         const double *S2, const int64_t *np,
                         int kind, double xc, double theta_ap,
                         double *SE, double *SB, double *SV, double *SW,
                         int64_t *N, int64_t *NPIX)
{
    aperture_pixels_impl(n0, c, nside_bin, G1, G2, W, S2, np, 0, kind, xc, theta_ap,
                         SE, SB, SV, SW, N, NPIX);
}

/* same, reading float32 sums and int32 counts (as the GPU path stores them) */
void orc_aperture_pixels_f32(int64_t n0, const double *c, int64_t nside_bin,
                             const float *G1, const float *G2, const float *W,
                             const float *S2, const int32_t *np,
                             int kind, double xc, double theta_ap,
                             double *SE, double *SB, double *SV, double *SW,
                             int64_t *N, int64_t *NPIX)
{
    aperture_pixels_impl(n0, c, nside_bin, G1, G2, W, S2, np, 1, kind, xc, theta_ap,
                         SE, SB, SV, SW, N, NPIX);
}

/*
 * Summed normalisation (Sect. 2.4 and Sect. 3.1 step 5): the mean density
 * inside the aperture is nbar = SW / A with A = 2 pi (1 - cos theta_ap), the
 * exact cap area.  M_E = SE / nbar, M_B = SB / nbar, sigma^2 = SV/(2 nbar^2)
 * (Eq. 8 with weights).  Centres with SW = 0 get zeros.
 */
void orc_finalise(int64_t n0, double theta_ap, const double *SE,
                  const double *SB, const double *SV, const double *SW,
                  double *ME, double *MB, double *VAR)
{
    double sh = sin(0.5 * theta_ap);
    double A = 4.0 * ORC_PI * sh * sh;
    for (int64_t t = 0; t < n0; ++t) {
        if (SW[t] > 0.0) {
            double nbar = SW[t] / A;
            ME[t] = SE[t] / nbar;
            MB[t] = SB[t] / nbar;
            VAR[t] = SV[t] / (2.0 * nbar * nbar);
        } else {
            ME[t] = 0.0; MB[t] = 0.0; VAR[t] = 0.0;
        }
    }
}

/*
 * Catalogue partitioning (Sect. 3.4 steps 1-3) and binning (Sect. 3.2
 * step 2).  pix[k] = RING pixel of galaxy k at nside_bin; perm = stable
 * order of the galaxies by pixel (ties keep input order), produced by a
 * counting sort; offsets[p] = position in perm of the first galaxy of
 * pixel p (npix + 1 entries).  Per-pixel sums G1, G2, W, S2 and counts n
 * accumulate the galaxies of each pixel in that sorted order.
 */
void orc_bin_catalog(int64_t nside, int64_t n, const double *ra,
                     const double *dec, const double *e1, const double *e2,
                     const double *w, int64_t *pix, int64_t *perm,
                     int64_t *offsets, double *G1, double *G2, double *W,
                     double *S2, int64_t *np)
{
    int64_t npix = 12 * nside * nside;
    orc_ang2pix_many(nside, n, ra, dec, pix);
    memset(offsets, 0, sizeof(int64_t) * (size_t)(npix + 1));
    for (int64_t k = 0; k < n; ++k) offsets[pix[k] + 1] += 1;
    for (int64_t p = 0; p < npix; ++p) offsets[p + 1] += offsets[p];
    int64_t *cursor = (int64_t *)malloc(sizeof(int64_t) * (size_t)(npix > 0 ? npix : 1));
    memcpy(cursor, offsets, sizeof(int64_t) * (size_t)npix);
    for (int64_t k = 0; k < n; ++k) perm[cursor[pix[k]]++] = k;
    free(cursor);
    for (int64_t p = 0; p < npix; ++p) {
        double g1 = 0, g2 = 0, ww = 0, s2 = 0;
        for (int64_t a = offsets[p]; a < offsets[p + 1]; ++a) {
            int64_t k = perm[a];
            g1 += w[k] * e1[k];
            g2 += w[k] * e2[k];
            ww += w[k];
            s2 += w[k] * w[k] * (e1[k] * e1[k] + e2[k] * e2[k]);
        }
        G1[p] = g1; G2[p] = g2; W[p] = ww; S2[p] = s2;
        np[p] = offsets[p + 1] - offsets[p];
    }
}

/* ------------------------------------------------------------------ */
/* Cartesian (projected) shear-based estimator, projS_pos              */
/* (Sect. 2.2, Sect. 5.2.1 steps 1-4).                                */
/*                                                                    */
/* Step 1: galaxy positions go to the plane tangent at the reference  */
/* point c (gnomonic projection, Sect. 2.2.1).  With r the point's     */
/* unit vector and (e_c, n_c) the East and North unit vectors at c,    */
/* the printed numerators and denominator are dot products:            */
/*   cos(d) sin(a - a_c)                         = r . e_c             */
/*   cos(d_c) sin(d) - sin(d_c) cos(d) cos(a-a_c) = r . n_c            */
/*   sin(d) sin(d_c) + cos(d) cos(d_c) cos(a-a_c) = r . c              */
/* so x = (r . e_c) / (r . c), y = (r . n_c) / (r . c), in this order  */
/* of operations: dot products summed ((0 + 1) + 2), then one division.*/
/* Points with r . c <= 0 have no image and are left out.              */
/* The shear is rotated with the basis (Sect. 2.2.2): its orientation  */
/* is kept relative to the local North, whose image direction in the   */
/* plane is the projection's differential applied to the galaxy's      */
/* North unit vector t:  N = ((t.e_c) P - X (t.c), (t.n_c) P - Y (t.c))*/
/* (up to the positive factor 1/P^2), with X, Y, P the three dot       */
/* products above.  If rho is the angle from the plane's +y axis to N  */
/* (counter-clockwise), gamma_plane = gamma e^{2 i rho}.               */
/* Step 2: the target pixel centres go to the same plane.              */
/* Step 3: per pair, separation (dx, dy) = galaxy - target in the      */
/* plane, member iff dx^2 + dy^2 <= theta_ap^2, Q of the plane distance,*/
/* phi = polar angle of (dx, dy); gamma_+ = -Re(gamma e^{-2 i phi}),   */
/* gamma_x = -Im(gamma e^{-2 i phi}) (the same sign convention as the  */
/* spherical sums; a member at the target itself carries no shear).   */
/* Step 4: sums SE, SB, SV, SW, N as in the spherical brute force; the */
/* normalisation is orc_finalise_area with A = pi theta_ap^2, the      */
/* area of the aperture in the plane.                                  */
/* ------------------------------------------------------------------ */
typedef struct {
    double c[3], e[3], n[3];
} orc_plane;

static void plane_setup(double ra_c, double dec_c, orc_plane *pl)
{
    double sa, ca, sd, cd;
    orc_sincos_deg(ra_c, &sa, &ca);
    orc_sincos_deg(dec_c, &sd, &cd);
    pl->c[0] = cd * ca; pl->c[1] = cd * sa; pl->c[2] = sd;
    pl->e[0] = -sa;     pl->e[1] = ca;      pl->e[2] = 0.0;
    pl->n[0] = -sd * ca; pl->n[1] = -sd * sa; pl->n[2] = cd;
}

static double dot3(const double *a, const double *b)
{
    return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2];
}

/* plane coordinates of unit vector r; returns 0 when r has no image */
static int plane_xy(const orc_plane *pl, const double *r, double *x, double *y)
{
    double P = dot3(r, pl->c);
    if (!(P > 0.0)) return 0;
    *x = dot3(r, pl->e) / P;
    *y = dot3(r, pl->n) / P;
    return 1;
}

void orc_project(double ra_c, double dec_c, int64_t n, const double *v, double *xy, int64_t *ok)
{
    orc_plane pl;
    plane_setup(ra_c, dec_c, &pl);
    for (int64_t k = 0; k < n; ++k) {
        double x = 0.0, y = 0.0;
        ok[k] = plane_xy(&pl, v + 3 * k, &x, &y);
        xy[2 * k] = x;
        xy[2 * k + 1] = y;
    }
}

/* the shear of a galaxy at (ra, dec) in the plane's axes (Sect. 2.2.2) */
static void plane_shear(const orc_plane *pl, double ra, double dec, double e1, double e2,
                        double *g1, double *g2)
{
    double sa, ca, sd, cd;
    orc_sincos_deg(ra, &sa, &ca);
    orc_sincos_deg(dec, &sd, &cd);
    double r[3] = {cd * ca, cd * sa, sd};
    double t[3] = {-sd * ca, -sd * sa, cd};          /* local North */
    double P = dot3(r, pl->c), X = dot3(r, pl->e), Y = dot3(r, pl->n);
    double Nx = dot3(t, pl->e) * P - X * dot3(t, pl->c);
    double Ny = dot3(t, pl->n) * P - Y * dot3(t, pl->c);
    double nn = Nx * Nx + Ny * Ny;
    double c2 = (Ny * Ny - Nx * Nx) / nn;            /* cos 2 rho */
    double s2 = -2.0 * Nx * Ny / nn;                 /* sin 2 rho */
    *g1 = e1 * c2 - e2 * s2;
    *g2 = e1 * s2 + e2 * c2;
}

void orc_plane_shear(double ra_c, double dec_c, int64_t n, const double *ra, const double *dec,
                     const double *e1, const double *e2, double *g)
{
    orc_plane pl;
    plane_setup(ra_c, dec_c, &pl);
    for (int64_t k = 0; k < n; ++k) plane_shear(&pl, ra[k], dec[k], e1[k], e2[k], g + 2 * k, g + 2 * k + 1);
}

void orc_aperture_projected(int64_t n0, const double *c, int64_t n,
                            const double *ra, const double *dec,
                            const double *e1, const double *e2, const double *w,
                            double ra_c, double dec_c, int kind, double xc, double theta_ap,
                            double *SE, double *SB, double *SV, double *SW, int64_t *N)
{
    orc_plane pl;
    plane_setup(ra_c, dec_c, &pl);
    double Tp = theta_ap * theta_ap;
    /* per galaxy: unit vector, plane position, plane shear; or no image */
    double *gv = (double *)malloc(sizeof(double) * 7 * (size_t)(n > 0 ? n : 1));
    double *zi = (double *)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        double *g = gv + 7 * k;
        orc_radec2vec(ra[k], dec[k], g);
        g[5] = 0.0;
        if (plane_xy(&pl, g, g + 3, g + 4)) {
            plane_shear(&pl, ra[k], dec[k], e1[k], e2[k], g + 5, g + 6);
        } else {
            g[3] = 0.0; g[4] = 0.0; g[6] = 0.0;
            g[5] = NAN;                                 /* marks "no image" */
        }
    }
    for (int64_t k = 0; k < n; ++k) {
        zi[2 * k] = gv[7 * k + 2];
        zi[2 * k + 1] = (double)k;
    }
    qsort(zi, (size_t)n, 2 * sizeof(double), cmp_dbl_idx);
    /* a member in the plane is within theta_ap on the sphere too (the plane
       distance of two images is at least their great-circle distance), so
       |z - z0| <= theta_ap bounds the candidates */
    double band = theta_ap * (1.0 + 1e-9) + 1e-15;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < n0; ++t) {
        const double *r0 = c + 3 * t;
        double x0, y0;
        double se = 0, sb = 0, sv = 0, sw = 0;
        int64_t cnt = 0;
        if (plane_xy(&pl, r0, &x0, &y0)) {
            double zlo = r0[2] - band, zhi = r0[2] + band;
            int64_t lo = 0, hi = n;
            while (lo < hi) {
                int64_t mid = (lo + hi) / 2;
                if (zi[2 * mid] < zlo) lo = mid + 1; else hi = mid;
            }
            for (int64_t m = lo; m < n && zi[2 * m] <= zhi; ++m) {
                int64_t k = (int64_t)zi[2 * m + 1];
                const double *g = gv + 7 * k;
                if (isnan(g[5])) continue;
                double dx = g[3] - x0, dy = g[4] - y0;
                double q = dx * dx + dy * dy;
                if (!(q <= Tp)) continue;
                double qv = orc_filter_q(kind, xc, sqrt(q) / theta_ap) / Tp;
                double c2 = 0.0, s2 = 0.0;                 /* cos 2 phi, sin 2 phi */
                if (q > 0.0) {
                    c2 = (dx * dx - dy * dy) / q;
                    s2 = 2.0 * dx * dy / q;
                }
                double gp = -(g[5] * c2 + g[6] * s2);      /* gamma_+ */
                double gx = g[5] * s2 - g[6] * c2;         /* gamma_x */
                se += w[k] * gp * qv;
                sb += w[k] * gx * qv;
                sv += w[k] * w[k] * (e1[k] * e1[k] + e2[k] * e2[k]) * qv * qv;
                sw += w[k];
                cnt += 1;
            }
        }
        SE[t] = se; SB[t] = sb; SV[t] = sv; SW[t] = sw; N[t] = cnt;
    }
    free(gv);
    free(zi);
}

/* summed normalisation with a given aperture area A (sr):
   nbar = SW / A, M = S / nbar, sigma^2 = SV / (2 nbar^2) */
void orc_finalise_area(int64_t n0, double A, const double *SE, const double *SB,
                       const double *SV, const double *SW, double *ME, double *MB, double *VAR)
{
    for (int64_t t = 0; t < n0; ++t) {
        if (SW[t] > 0.0) {
            double nbar = SW[t] / A;
            ME[t] = SE[t] / nbar;
            MB[t] = SB[t] / nbar;
            VAR[t] = SV[t] / (2.0 * nbar * nbar);
        } else {
            ME[t] = 0.0; MB[t] = 0.0; VAR[t] = 0.0;
        }
    }
}

/*
 * Equal-area annulus statistics about a reference point (Sect. 5.2.2): the
 * targets (unit vectors c) are binned by their angular distance d from the
 * reference unit vector r_ref into nbins annuli of equal area out to rmax
 * (annulus k holds 1 - cos d in [k, k + 1) (1 - cos rmax) / nbins); per
 * annulus the count, and the mean and population standard deviation of
 * eps = (mx - mref) / sref are returned, where sref is the population
 * standard deviation of mref over all the given targets (Eq. 12).  Targets
 * beyond rmax are ignored; empty annuli give zeros.
 */
void orc_annulus_stats(int64_t n0, const double *c, const double *r_ref, double rmax,
                       const double *mx, const double *mref, int64_t nbins,
                       int64_t *count, double *mean, double *sd)
{
    double m = 0.0;
    for (int64_t t = 0; t < n0; ++t) m += mref[t];
    m /= (double)(n0 > 0 ? n0 : 1);
    double v = 0.0;
    for (int64_t t = 0; t < n0; ++t) v += (mref[t] - m) * (mref[t] - m);
    double sref = sqrt(v / (double)(n0 > 0 ? n0 : 1));
    double cmax = 1.0 - cos(rmax);
    for (int64_t k = 0; k < nbins; ++k) { count[k] = 0; mean[k] = 0.0; sd[k] = 0.0; }
    for (int64_t t = 0; t < n0; ++t) {
        const double *p = c + 3 * t;
        /* 1 - cos d from the chord: 1 - cos d = s^2 / 2 */
        double dx = p[0] - r_ref[0], dy = p[1] - r_ref[1], dz = p[2] - r_ref[2];
        double u = 0.5 * ((dx * dx + dy * dy) + dz * dz);
        if (!(u < cmax)) continue;
        int64_t k = (int64_t)floor(u / cmax * (double)nbins);
        if (k >= nbins) k = nbins - 1;
        double e = (mx[t] - mref[t]) / sref;
        count[k] += 1;
        mean[k] += e;
        sd[k] += e * e;
    }
    for (int64_t k = 0; k < nbins; ++k) {
        if (count[k] == 0) continue;
        double mu = mean[k] / (double)count[k];
        double var = sd[k] / (double)count[k] - mu * mu;
        mean[k] = mu;
        sd[k] = sqrt(var > 0.0 ? var : 0.0);
    }
}
