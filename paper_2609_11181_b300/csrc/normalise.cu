// normalise.cu -- the averaged normalisation (Sect. 2.4).
//
// The summed form divides the aperture sums by the weight in the aperture:
// M = A S / sum w.  The averaged form normalises each bin pixel's shear by
// that pixel's own weight and multiplies by the pixel area, with no aperture
// density: M = sum_p Q gamma+_p A_pix / W_p (galaxies: each carries
// w A_pix / W of its bin pixel).  The map kernels are the same for both: the
// inputs are scaled by f = A_pix / W (shear sums by f, noise sums by f^2,
// weights kept), the kernels run, and their summed-form outputs are turned
// back into the plain sums by the factor sum_w / A.
#include <math.h>

#include <algorithm>

#include "smart_internal.cuh"

namespace smart {

// binned map (G1, G2, S2, W) -> (G1 f, G2 f, S2 f^2, W)
__global__ void k_avg_pixels(int64_t npix, float apix, const float4 *__restrict__ px, float4 *__restrict__ out) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
        const float4 q = px[p];
        const float f = q.w > 0.f ? apix / q.w : 0.f;
        out[p] = make_float4(q.x * f, q.y * f, q.z * f * f, q.w);
    }
}

// records (w e1, w e2, w, w^2 |e|^2) -> scaled by the W of their bin pixel:
// from the binned map (galaxy records) or from the record itself (pixel
// records, whose w is the pixel's W)
__global__ void k_avg_records(int64_t n, float apix, const float4 *__restrict__ sh, const uint32_t *__restrict__ keys,
                              const float4 *__restrict__ px, float4 *__restrict__ out) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const float4 q = sh[k];
        const float W = px ? px[keys[k]].w : q.z;
        const float f = W > 0.f ? apix / W : 0.f;
        out[k] = make_float4(q.x * f, q.y * f, q.z, q.w * f * f);
    }
}

// summed-form outputs (M = A S / sum_w, sigma^2 = A^2 V / (2 sum_w^2)) back to
// the averaged ones (M = S, sigma^2 = V / 2)
__global__ void k_avg_rescale(int64_t n, double area, const double *__restrict__ sum_w, float *__restrict__ me,
                              float *__restrict__ mb, float *__restrict__ var) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const double sw = sum_w[t];
        if (!(sw > 0.0)) continue;
        const float f = (float)(sw / area);
        if (me) me[t] *= f;
        if (mb) mb[t] *= f;
        if (var) var[t] *= f * f;
    }
}

static float pixel_area(const smart_ctx *c) {
    return (float)(4.0 * SMART_PI / (12.0 * (double)c->nside_bin * (double)c->nside_bin));
}

static unsigned grid_of(const smart_ctx *c, int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)c->num_sms * 32));
}

smart_status averaged_pixel_input(smart_ctx *c, const float4 *px, const float4 **out) {
    const int64_t npix = npix_of(c->nside_bin);
    smart_status st = ensure_alloc(c, (void **)&c->avg_buf, c->cap_avg, npix, sizeof(float4), "averaged inputs");
    if (st != SMART_OK) return st;
    k_avg_pixels<<<grid_of(c, npix), 256, 0, c->stream>>>(npix, pixel_area(c), px, c->avg_buf);
    *out = c->avg_buf;
    return check_cuda(c, cudaGetLastError(), "k_avg_pixels");
}

smart_status averaged_record_input(smart_ctx *c, const float4 *sh, const uint32_t *keys, const float4 *px, int64_t n,
                                   const float4 **out) {
    smart_status st = ensure_alloc(c, (void **)&c->avg_buf, c->cap_avg, std::max<int64_t>(n, 1), sizeof(float4),
                                   "averaged inputs");
    if (st != SMART_OK) return st;
    if (n > 0) k_avg_records<<<grid_of(c, n), 256, 0, c->stream>>>(n, pixel_area(c), sh, keys, px, c->avg_buf);
    *out = c->avg_buf;
    return check_cuda(c, cudaGetLastError(), "k_avg_records");
}

smart_status averaged_rescale(smart_ctx *c, const smart_maps *out) {
    const int64_t n = c->n_targets;
    if (n == 0) return SMART_OK;
    if (!out->sum_w) return fail(c, SMART_E_ARG, "averaged normalisation needs the sum_w output");
    k_avg_rescale<<<grid_of(c, n), 256, 0, c->stream>>>(n, c->area, out->sum_w, out->map_e, out->map_b, out->var);
    return check_cuda(c, cudaGetLastError(), "k_avg_rescale");
}

}  // namespace smart

using namespace smart;

extern "C" smart_status smart_set_normalisation(smart_ctx *c, int mode) {
    if (!c) return SMART_E_ARG;
    if (mode != SMART_NORM_SUMMED && mode != SMART_NORM_AVERAGED)
        return fail(c, SMART_E_ARG, "smart_set_normalisation: mode must be SMART_NORM_SUMMED or SMART_NORM_AVERAGED");
    c->norm = mode;
    return SMART_OK;
}
