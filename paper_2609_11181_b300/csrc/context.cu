// context.cu -- lifetime, error reporting and input registration of a SMART
// context (the C ABI declared in include/smart.h).
#include <math.h>

#include <algorithm>
#include <chrono>
#include <thread>

#include "smart_internal.cuh"

namespace smart {

smart_status fail(smart_ctx *ctx, smart_status st, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return st;
}

smart_status check_cuda(smart_ctx *ctx, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return SMART_OK;
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(ctx, e == cudaErrorMemoryAllocation ? SMART_E_NOMEM : SMART_E_CUDA, m);
}

// grow-only device buffer: reallocates when `need` elements exceed `cap`.
// Stream-ordered (cudaFreeAsync / cudaMallocAsync on the context stream), so
// that growing a buffer never makes the host wait: the old buffer is freed
// after the work already queued on the stream, the new one is ready for the
// work queued after it.
smart_status ensure_alloc(smart_ctx *ctx, void **p, int64_t &cap, int64_t need, size_t elem, const char *what) {
    if (need <= cap && *p) return SMART_OK;
    if (*p) {
        if (ctx->async_bufs.erase(*p)) cudaFreeAsync(*p, ctx->stream);
        else {
            cudaStreamSynchronize(ctx->stream);
            cudaFree(*p);
        }
        *p = nullptr;
        cap = 0;
    }
    const int64_t n = need > 0 ? need : 1;
    cudaError_t e = cudaMallocAsync(p, (size_t)n * elem, ctx->stream);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(ctx, SMART_E_NOMEM, std::string("cudaMallocAsync(") + what + ") failed");
    }
    ctx->async_bufs.insert(*p);
    cap = n;
    return SMART_OK;
}

smart_status wait_stream(smart_ctx *ctx, const char *what) {
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(ctx->stream);
        if (e == cudaSuccess) return SMART_OK;
        if (e != cudaErrorNotReady) return check_cuda(ctx, e, what);
        const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (ctx->wait_limit_s > 0 && dt > ctx->wait_limit_s)
            return fail(ctx, SMART_E_TIMEOUT, std::string(what) + ": wait limit passed");
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

}  // namespace smart

using namespace smart;

static bool nside_ok(int nside) { return nside >= 1 && nside <= 8192 && (nside & (nside - 1)) == 0; }

extern "C" smart_status smart_create(int nside_out, const smart_filter *filter, double theta_ap_arcmin,
                                     int nside_bin, void *cuda_stream, smart_ctx **out) {
    if (!out) return SMART_E_ARG;
    *out = nullptr;
    if (!nside_ok(nside_out) || !nside_ok(nside_bin) || !filter) return SMART_E_ARG;
    if (filter->kind != SMART_FILTER_POLY && filter->kind != SMART_FILTER_SCHIRMER && filter->kind != SMART_FILTER_JARVIS)
        return SMART_E_ARG;
    if (filter->kind != SMART_FILTER_POLY && !(filter->xc > 0.0 && filter->xc < 10.0)) return SMART_E_ARG;
    if (!(theta_ap_arcmin > 0.0) || !(theta_ap_arcmin <= 3600.0)) return SMART_E_ARG;
    smart_ctx *c = new (std::nothrow) smart_ctx();
    if (!c) return SMART_E_NOMEM;
    c->nside_out = nside_out;
    c->nside_bin = nside_bin;
    c->filter_kind = filter->kind;
    c->xc = filter->kind == SMART_FILTER_POLY ? 0.15 : filter->xc;
    c->theta_ap = theta_ap_arcmin * SMART_PI / 10800.0;
    c->T = smart_chord2(theta_ap_arcmin);
    c->area = 2.0 * SMART_PI * (0.5 * c->T);     // 2 pi (1 - cos theta_ap) = pi T
    c->stream = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
        c->num_sms = sms;
    if (cudaMalloc(&c->d_fp64_count, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&c->d_band_count, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&c->d_status, sizeof(int)) != cudaSuccess ||
        cudaMemset(c->d_status, 0, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&c->d_work, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&c->host_rb, 16 * sizeof(int64_t)) != cudaSuccess) {
        if (c->d_fp64_count) cudaFree(c->d_fp64_count);
        delete c;
        return SMART_E_NOMEM;
    }
    *out = c;
    return SMART_OK;
}

extern "C" void smart_destroy(smart_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    void *bufs[] = {c->targets, c->rp_pix, c->rp_gal, c->rp_pix_cnt, c->rp_gal_cnt, c->own_px,
                    c->own_np, c->keys, c->keys_alt, c->vals, c->vals_alt, c->offsets, c->rec_geo,
                    c->rec_shear, c->rec_radec, c->hist, c->hist_scan, c->scan_tmp, c->ring_lat, c->d_invalid,
                    c->tiles, c->tile_flag, c->qtab, c->np_prefix, c->d_work, c->toe_info, c->toe_geo,
                    c->toe_ring, c->gen_list, c->gen_work, c->gal_tiles, c->raw, c->band, c->d_band_count,
                    c->d_status, c->d_fp64_count, c->bary_off, c->bary_geo, c->bary_sh, c->bary_keys,
                    c->bary_cnt, c->bary_vec, c->bary_wr, c->raw_m, c->avg_buf, c->gen_band, c->d_gen_count,
                    c->proj_plane, c->proj_xy, c->proj_sh, c->proj_txy, c->qtab_plane, c->annulus_buf};
    for (void *b : bufs) {
        if (!b) continue;
        if (c->async_bufs.count(b)) cudaFreeAsync(b, c->stream);
        else cudaFree(b);
    }
    cudaStreamSynchronize(c->stream);
    if (c->host_rb) cudaFreeHost(c->host_rb);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    delete c;
}

extern "C" const char *smart_last_error(const smart_ctx *c) { return c ? c->err.c_str() : "null context"; }

extern "C" smart_status smart_sync(smart_ctx *c, double timeout_s) {
    if (!c) return SMART_E_ARG;
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(c->stream);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return check_cuda(c, e, "smart_sync");
        if (timeout_s > 0) {
            double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (dt > timeout_s) return fail(c, SMART_E_TIMEOUT, "smart_sync: deadline passed");
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    int status = 0;
    smart_status st = check_cuda(c, cudaMemcpy(&status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost), "smart_sync status");
    if (st != SMART_OK) return st;
    if (status) {
        cudaMemset(c->d_status, 0, sizeof(int));
        if (status & SMART_STATUS_INVALID_COORDS) {
            int inv = 0;
            if (c->d_invalid) cudaMemcpy(&inv, c->d_invalid, sizeof(int), cudaMemcpyDeviceToHost);
            return fail(c, SMART_E_ARG, "smart_bin_galaxies: " + std::to_string(inv) +
                                            " galaxies with non-finite ra/dec or |dec| > 90 (left out of the catalogue)");
        }
        if (status & SMART_STATUS_BAD_RUNS)
            return fail(c, SMART_E_ARG, "smart_set_binned_runs: a run lies outside the map or the compact arrays "
                                        "(those runs were skipped)");
        if (status & SMART_STATUS_BAND_OVERFLOW)
            return fail(c, SMART_E_OVERFLOW, "guard-band pair list overflowed: map incomplete");
        return fail(c, SMART_E_INTERNAL, "device status " + std::to_string(status));
    }
    return SMART_OK;
}

__global__ void k_check_targets(const int64_t *__restrict__ t, int64_t n, int64_t npix, int *__restrict__ bad) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = t[k];
        if (p < 0 || p >= npix || (k > 0 && t[k - 1] >= p)) atomicExch(bad, 1);
    }
}

extern "C" smart_status smart_set_targets(smart_ctx *c, const int64_t *pix, int64_t n) {
    if (!c) return SMART_E_ARG;
    if (n < 0 || (n > 0 && !pix)) return fail(c, SMART_E_ARG, "smart_set_targets: bad pointer or size");
    if (n > ((int64_t)1 << 31)) return fail(c, SMART_E_OVERFLOW, "smart_set_targets: more than 2^31 targets");
    smart_status st = ensure_alloc(c, (void **)&c->targets, c->cap_targets, n, sizeof(int64_t), "targets");
    if (st != SMART_OK) return st;
    c->n_targets = n;
    c->targets_version += 1;
    c->n_tiles = 0;
    if (n == 0) return SMART_OK;
    st = check_cuda(c, cudaMemcpyAsync(c->targets, pix, (size_t)n * sizeof(int64_t), cudaMemcpyDeviceToDevice, c->stream),
                    "copy targets");
    if (st != SMART_OK) return st;
    // validate range and ordering once (read back into pinned memory, a
    // bounded wait)
    int *bad = nullptr;
    if (cudaMallocAsync(&bad, sizeof(int), c->stream) != cudaSuccess) return fail(c, SMART_E_NOMEM, "flag alloc");
    cudaMemsetAsync(bad, 0, sizeof(int), c->stream);
    const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 148 * 16);
    k_check_targets<<<blocks, 256, 0, c->stream>>>(c->targets, n, npix_of(c->nside_out), bad);
    int32_t *hb32 = reinterpret_cast<int32_t *>(c->host_rb);
    cudaMemcpyAsync(hb32, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    cudaFreeAsync(bad, c->stream);
    st = wait_stream(c, "smart_set_targets: validate targets");
    if (st != SMART_OK) return st;
    const int hb = hb32[0];
    if (hb) {
        c->n_targets = 0;
        c->n_tiles = 0;
        return fail(c, SMART_E_ARG, "smart_set_targets: pixels must be unique, ascending and in [0, 12 nside_out^2)");
    }
    st = build_tiles(c);
    if (st != SMART_OK) return st;
    return prepare_tables(c);
}

extern "C" smart_status smart_set_wait_limit(smart_ctx *c, double seconds) {
    if (!c) return SMART_E_ARG;
    if (!(seconds >= 0.0)) return fail(c, SMART_E_ARG, "smart_set_wait_limit: negative limit");
    c->wait_limit_s = seconds;
    return SMART_OK;
}

__global__ void k_pack(const float *__restrict__ G1, const float *__restrict__ G2, const float *__restrict__ W,
                       const float *__restrict__ S2, const int32_t *__restrict__ n_in, int64_t npix,
                       float4 *__restrict__ px, int32_t *__restrict__ n_out) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
        px[p] = make_float4(G1[p], G2[p], S2[p], W[p]);
        n_out[p] = n_in[p];
    }
}

static smart_status ensure_own_binned(smart_ctx *c) {
    const int64_t npix = npix_of(c->nside_bin);
    if (!c->own_px && cudaMalloc(&c->own_px, (size_t)npix * sizeof(float4)) != cudaSuccess)
        return fail(c, SMART_E_NOMEM, "cudaMalloc(binned map) failed");
    if (!c->own_np && cudaMalloc(&c->own_np, (size_t)(npix + 1) * sizeof(int32_t)) != cudaSuccess)
        return fail(c, SMART_E_NOMEM, "cudaMalloc(binned counts) failed");
    return SMART_OK;
}

namespace smart {
smart_status ensure_own_binned_map(smart_ctx *c) { return ensure_own_binned(c); }
}

extern "C" smart_status smart_set_binned(smart_ctx *c, const float *G1, const float *G2, const float *W,
                                         const float *S2, const int32_t *n_p) {
    if (!c) return SMART_E_ARG;
    if (!G1 || !G2 || !W || !S2 || !n_p) return fail(c, SMART_E_ARG, "smart_set_binned: null pointer");
    smart_status st = ensure_own_binned(c);
    if (st != SMART_OK) return st;
    const int64_t npix = npix_of(c->nside_bin);
    const unsigned blocks = (unsigned)std::min<int64_t>((npix + 255) / 256, (int64_t)c->num_sms * 16);
    k_pack<<<blocks, 256, 0, c->stream>>>(G1, G2, W, S2, n_p, npix, c->own_px, c->own_np);
    st = check_cuda(c, cudaGetLastError(), "k_pack");
    if (st != SMART_OK) return st;
    c->PX = c->own_px;
    c->NP = c->own_np;
    c->have_binned = true;
    c->binned_from_catalog = false;
    return SMART_OK;
}

// one block per run: the run's pixels, contiguous in the compact arrays,
// go to their RING positions in the full-sky map.  A run that does not fit
// the map or the compact arrays is skipped and flagged in the status word.
__global__ void k_scatter_runs(const float4 *__restrict__ px, const int32_t *__restrict__ np,
                               const int64_t *__restrict__ runs, int64_t n_runs, int64_t npix, int64_t n_compact,
                               float4 *__restrict__ out_px, int32_t *__restrict__ out_np, int *__restrict__ status) {
    for (int64_t r = blockIdx.x; r < n_runs; r += gridDim.x) {
        const int64_t first = runs[3 * r], len = runs[3 * r + 1], off = runs[3 * r + 2];
        if (first < 0 || len < 0 || first > npix - len || off < 0 || off > n_compact - len) {
            if (threadIdx.x == 0) atomicOr(status, SMART_STATUS_BAD_RUNS);
            continue;
        }
        for (int64_t i = threadIdx.x; i < len; i += blockDim.x) {
            out_px[first + i] = px[off + i];
            out_np[first + i] = np[off + i];
        }
    }
}

extern "C" smart_status smart_set_binned_runs(smart_ctx *c, const float *px, const int32_t *n_p, const int64_t *runs,
                                              int64_t n_runs, int64_t n_compact, int clear) {
    if (!c) return SMART_E_ARG;
    if (n_runs < 0 || n_compact < 0 || (n_runs > 0 && !runs) || (n_compact > 0 && (!px || !n_p)))
        return fail(c, SMART_E_ARG, "smart_set_binned_runs: bad pointer or size");
    if (((uintptr_t)px & 15) != 0) return fail(c, SMART_E_ARG, "smart_set_binned_runs: pixels not 16-byte aligned");
    const bool fresh = !c->own_px || !c->own_np;
    smart_status st = ensure_own_binned(c);
    if (st != SMART_OK) return st;
    const int64_t npix = npix_of(c->nside_bin);
    // the map is cleared when asked, when it was just made, and when it held
    // other data (a catalogue's or a full map's): pixels outside the runs are
    // then zero
    if (clear || fresh || !c->binned_from_runs) {
        if ((st = check_cuda(c, cudaMemsetAsync(c->own_px, 0, (size_t)npix * sizeof(float4), c->stream), "clear map")) !=
                SMART_OK ||
            (st = check_cuda(c, cudaMemsetAsync(c->own_np, 0, (size_t)(npix + 1) * sizeof(int32_t), c->stream),
                             "clear counts")) != SMART_OK)
            return st;
    }
    if (n_runs > 0) {
        const unsigned blocks = (unsigned)std::min<int64_t>(n_runs, (int64_t)c->num_sms * 16);
        k_scatter_runs<<<blocks, 256, 0, c->stream>>>((const float4 *)px, n_p, runs, n_runs, npix, n_compact, c->own_px,
                                                      c->own_np, c->d_status);
        if ((st = check_cuda(c, cudaGetLastError(), "k_scatter_runs")) != SMART_OK) return st;
    }
    c->PX = c->own_px;
    c->NP = c->own_np;
    c->have_binned = true;
    c->binned_from_catalog = false;
    c->binned_from_runs = true;
    return SMART_OK;
}

extern "C" smart_status smart_set_binned_packed(smart_ctx *c, const float *px, const int32_t *n_p) {
    if (!c) return SMART_E_ARG;
    if (!px || !n_p) return fail(c, SMART_E_ARG, "smart_set_binned_packed: null pointer");
    if (((uintptr_t)px & 15) != 0) return fail(c, SMART_E_ARG, "smart_set_binned_packed: map not 16-byte aligned");
    c->PX = (const float4 *)px;
    c->NP = n_p;
    c->have_binned = true;
    c->binned_from_catalog = false;
    c->binned_from_runs = false;
    return SMART_OK;
}

extern "C" int64_t smart_last_fp64_decisions(smart_ctx *c) {
    if (!c) return -1;
    cudaMemcpyAsync(c->host_rb + 8, c->d_fp64_count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream);
    if (wait_stream(c, "smart_last_fp64_decisions") != SMART_OK) return -1;
    return c->host_rb[8];
}

// ------------------------------------------------------------ kernel timing
namespace smart {

static cudaEvent_t timing_event(smart_ctx *c) {
    if (c->ev_used == c->ev_pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        c->ev_pool.push_back(e);
    }
    return c->ev_pool[c->ev_used++];
}

KernelTimer::KernelTimer(smart_ctx *c, int id) : c_(c), id_(id) {
    if (!c_->timing) return;
    start_ = timing_event(c_);
    if (start_) cudaEventRecord(start_, c_->stream);
}

KernelTimer::~KernelTimer() {
    if (!c_->timing || !start_) return;
    cudaEvent_t stop = timing_event(c_);
    if (!stop) return;
    cudaEventRecord(stop, c_->stream);
    c_->tlog[id_].emplace_back(start_, stop);
}

}  // namespace smart

extern "C" smart_status smart_timing_enable(smart_ctx *c, int enable) {
    if (!c) return SMART_E_ARG;
    c->timing = enable != 0;
    c->ev_used = 0;
    for (auto &l : c->tlog) l.clear();
    return SMART_OK;
}

extern "C" smart_status smart_timing_read(smart_ctx *c, int kernel, int64_t *launches, double *total_ms,
                                          double timeout_s) {
    if (!c) return SMART_E_ARG;
    if (kernel < 0 || kernel >= SMART_KT_COUNT || !launches || !total_ms)
        return fail(c, SMART_E_ARG, "smart_timing_read: bad kernel id or null output");
    double sum = 0.0;
    const auto t0 = std::chrono::steady_clock::now();
    for (const auto &pr : c->tlog[kernel]) {
        for (;;) {          // bounded wait for the stop event
            const cudaError_t e = cudaEventQuery(pr.second);
            if (e == cudaSuccess) break;
            if (e != cudaErrorNotReady) return check_cuda(c, e, "smart_timing_read");
            const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (timeout_s > 0 && dt > timeout_s) return fail(c, SMART_E_TIMEOUT, "smart_timing_read: deadline passed");
            std::this_thread::sleep_for(std::chrono::microseconds(50));
        }
        float ms = 0.f;
        smart_status st = check_cuda(c, cudaEventElapsedTime(&ms, pr.first, pr.second), "cudaEventElapsedTime");
        if (st != SMART_OK) return st;
        sum += ms;
    }
    *launches = (int64_t)c->tlog[kernel].size();
    *total_ms = sum;
    return SMART_OK;
}

extern "C" smart_status smart_set_band_slot_limit(smart_ctx *c, int64_t n_slots) {
    if (!c) return SMART_E_ARG;
    if (n_slots < 0) return fail(c, SMART_E_ARG, "smart_set_band_slot_limit: negative limit");
    c->band_slot_limit = n_slots;
    return SMART_OK;
}

extern "C" smart_status smart_get_general_pairs(smart_ctx *c, int32_t *pairs, int64_t cap, int64_t *n_pairs,
                                                int64_t *n_single) {
    if (!c || !n_pairs || !n_single) return SMART_E_ARG;
    if (c->gen_version != c->targets_version)
        return fail(c, SMART_E_STATE, "smart_get_general_pairs: no tables for the current targets");
    *n_pairs = c->n_work_pairs;
    *n_single = c->n_work - c->n_work_pairs;
    if (pairs && c->n_work_pairs > 0) {
        if (cap < c->n_work_pairs) return fail(c, SMART_E_ARG, "smart_get_general_pairs: output too small");
        return check_cuda(c, cudaMemcpyAsync(pairs, c->gen_work, (size_t)c->n_work_pairs * sizeof(int2),
                                             cudaMemcpyDeviceToDevice, c->stream), "smart_get_general_pairs");
    }
    return SMART_OK;
}

extern "C" smart_status smart_get_general_targets(smart_ctx *c, int32_t *idx, int64_t cap, int64_t *n_gen) {
    if (!c || !n_gen) return SMART_E_ARG;
    if (c->gen_version != c->targets_version)
        return fail(c, SMART_E_STATE, "smart_get_general_targets: no tables for the current targets");
    *n_gen = c->n_gen;
    if (idx && c->n_gen > 0) {
        if (cap < c->n_gen) return fail(c, SMART_E_ARG, "smart_get_general_targets: output too small");
        return check_cuda(c, cudaMemcpyAsync(idx, c->gen_list, (size_t)c->n_gen * sizeof(int32_t),
                                             cudaMemcpyDeviceToDevice, c->stream), "smart_get_general_targets");
    }
    return SMART_OK;
}
