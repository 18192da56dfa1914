// aperture_batch.cu -- many pixel-based maps in one persistent launch,
// captured in a CUDA graph (batched form of Sect. 3.2).
//
// Each map keeps its own context (targets, binned map, aperture, tables).
// The batch builds one global work list of the Toeplitz tiles of all maps,
// ordered by estimated cost, longest first, which a persistent kernel claims
// with an atomic counter (maps of very different size and aperture share the
// SMs without tail effects), and one flat list of the general targets of
// all maps (one thread each).  A small autotuner times a few launch shapes
// (resident CTAs per SM, item order) on the real batch and keeps the
// fastest; the launches (and the count prefixes of copied binned maps) are
// then captured once in a CUDA graph and replayed by smart_batch_run.
#include <math.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "aperture_pixel.cuh"

namespace smart {

struct BatchItem {
    int64_t index;     // tile index (Toeplitz) or first position in the general list
    int map;
    int type;          // 0: Toeplitz tile, 1: chunk of general targets
    int count;         // targets in a general chunk
    int pad;
};

// the Toeplitz tiles of every map, claimed longest first by resident CTAs
template <int KIND, int NC>
__global__ void __launch_bounds__(NT, toe_ctas_per_sm<NC>()) k_pixel_batched(const MapArgs *__restrict__ maps,
                                                          const BatchItem *__restrict__ items, int64_t n_items,
                                                          int *__restrict__ work) {
    __shared__ __align__(16) ToeShared<NC> S;
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(work, 1);
        __syncthreads();
        const int64_t item = s_item;
        __syncthreads();   // every thread has read s_item
        if (item >= n_items) break;
        const BatchItem it = items[item];
        toeplitz_tile<KIND, NC>(maps[it.map], it.index, S);
    }
}

// the general targets of every map: one thread per entry (map, target, its
// mirror image or -1, 0) of the list, whose first np entries are the mirror
// pairs of every map and the rest the unpaired targets.  Thread i of the
// pair launch takes entry np + i for i < n_lead (unpaired targets run ahead
// of the pairs, see gen_lead) and entry i - n_lead after that; the unpaired
// launch takes entries lo + i.  The list runs map by map within each part,
// so the filter table of the block's first map is staged in shared memory;
// entries of another map read theirs from global memory.
template <int KIND>
__device__ __forceinline__ void batched_general(const MapArgs *__restrict__ maps, const int4 *__restrict__ list,
                                                int64_t i, bool pair, int64_t first, const GenBand &gb,
                                                float4 *qtab) {
    const int m0 = list[first].x;
    if (KIND != SMART_FILTER_POLY) {
        const float4 *src = maps[m0].f.qtab;
        for (int k = threadIdx.x; k < QTAB_BINS; k += blockDim.x) qtab[k] = src[k];
        __syncthreads();
    }
    if (i < 0) return;
    const int4 e = list[i];
    const MapArgs &a = maps[e.x];
    if (pair) general_target2<KIND>(a, e.y, e.z, i, e.x == m0 ? qtab : a.f.qtab, gb);
    else general_target<KIND>(a, e.y, i, e.x == m0 ? qtab : a.f.qtab, gb);
}

template <int KIND>
__global__ void __launch_bounds__(128, 7) k_pixel_batched_general(const MapArgs *__restrict__ maps,
                                                                  const int4 *__restrict__ list, int64_t lo,
                                                                  int64_t hi, const GenBand gb) {
    __shared__ float4 qtab[KIND == SMART_FILTER_POLY ? 1 : QTAB_BINS];
    const int64_t first = lo + blockIdx.x * (int64_t)blockDim.x, i = first + threadIdx.x;
    batched_general<KIND>(maps, list, i < hi ? i : -1, false, first, gb, qtab);
}

template <int KIND>
__global__ void __launch_bounds__(128, GEN_PAIR_CTAS_PER_SM) k_pixel_batched_general_pairs(
    const MapArgs *__restrict__ maps, const int4 *__restrict__ list, int64_t np, int64_t n_lead, const GenBand gb) {
    __shared__ float4 qtab[KIND == SMART_FILTER_POLY ? 1 : QTAB_BINS];
    const int64_t i0 = blockIdx.x * (int64_t)blockDim.x, i = i0 + threadIdx.x;
    const int64_t first = i0 < n_lead ? np + i0 : i0 - n_lead;
    const int64_t e = i < n_lead ? np + i : (i - n_lead < np ? i - n_lead : -1);
    batched_general<KIND>(maps, list, e, i >= n_lead, first, gb, qtab);
}

// the general targets with guard-band pairs, one thread per slot
template <int KIND>
__global__ void k_pixel_batched_band(const MapArgs *__restrict__ maps, const int4 *__restrict__ list,
                                     const GenBand gb) {
    const unsigned long long n = min(*gb.counts, (unsigned long long)gb.cap_slots);
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const int64_t tag = gb.idx[i];
        const int4 e = list[tag >> 1];
        const MapArgs &a = maps[e.x];
        const double *raw = gb.raw + 4 * i;
        band_finish<KIND>(a, (tag & 1) ? e.z : e.y, e.y, a.f.qtab, gb.mask[i], raw[0], raw[1], raw[2], raw[3],
                          gb.cnt[2 * i], gb.cnt[2 * i + 1]);
    }
}

__global__ void k_tiles_wanted(const MapArgs a, unsigned char *__restrict__ want) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < a.n_tiles; t += (int64_t)gridDim.x * blockDim.x)
        want[t] = toeplitz_tile_wanted(a, t) ? 1 : 0;
}

}  // namespace smart

using namespace smart;

struct smart_batch {
    std::vector<smart_ctx *> ctxs;
    std::vector<MapArgs> args;
    std::vector<BatchItem> by_cost, natural;
    MapArgs *d_maps = nullptr;
    BatchItem *d_items = nullptr;
    int64_t n_items = 0;
    int4 *d_gen = nullptr;           // general work: (map, target, its mirror image or -1, 0)
    int64_t n_gen = 0;               // entries of d_gen
    int64_t n_gen_pairs = 0;         // the first n_gen_pairs of them are mirror pairs
    int64_t n_gen_targets = 0;       // targets they cover
    void *d_band = nullptr;          // slots of general targets with guard-band pairs
    unsigned long long *d_band_count = nullptr;
    GenBand gb{};
    int *d_work = nullptr;
    cudaStream_t stream = nullptr;
    cudaStream_t side = nullptr;     // the general kernel runs here, beside the persistent kernel
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool own_stream = false;
    int kind = 0;
    bool short_runs = true;   // every map's Toeplitz runs fit the smaller staging
    int ctas_per_sm = toe_ctas_per_sm<NCAND_SHORT>();
    int order = 0;            // 0: longest first, 1: natural
    double tuned_ms = 0.0;
    std::string err;
};

// why the last smart_batch_create of this thread failed (the batch is gone)
static thread_local std::string g_create_err;

static smart_status bfail(smart_batch *b, smart_status st, const std::string &m) {
    if (b) b->err = m;
    g_create_err = m;
    return st;
}

// launch the batched kernel (plus the count prefixes) on the batch stream
static smart_status batch_launch(smart_batch *b, int ctas_per_sm, int order) {
    for (size_t m = 0; m < b->ctxs.size(); ++m) {
        smart_ctx *c = b->ctxs[m];
        cudaStream_t keep = c->stream;
        c->stream = b->stream;
        smart_status st = launch_count_prefix(c);
        c->stream = keep;
        if (st != SMART_OK) return bfail(b, st, "count prefix of map " + std::to_string(m) + ": " + c->err);
    }
    if (cudaMemsetAsync(b->d_work, 0, sizeof(int), b->stream) != cudaSuccess)
        return bfail(b, SMART_E_CUDA, "work counter reset failed");
    const int sms = b->ctxs[0]->num_sms;
    // the general targets on the side stream, concurrent with the persistent
    // kernel (fork after the count prefixes, join before the batch ends): the
    // general blocks fill the SMs the persistent kernel's tail leaves idle
    const bool fork = b->n_gen > 0 && b->n_items > 0;
    if (fork) {
        if (cudaEventRecord(b->ev_fork, b->stream) != cudaSuccess ||
            cudaStreamWaitEvent(b->side, b->ev_fork, 0) != cudaSuccess)
            return bfail(b, SMART_E_CUDA, "fork of the general launch failed");
    }
    if (b->n_gen > 0) {
        cudaStream_t gs = fork ? b->side : b->stream;
        if (cudaMemsetAsync(b->d_band_count, 0, sizeof(unsigned long long), gs) != cudaSuccess)
            return bfail(b, SMART_E_CUDA, "slot counter reset failed");
        const int64_t np = b->n_gen_pairs, ng = b->n_gen, n_lead = gen_lead(np, ng - np);
        const unsigned gp = (unsigned)((np + n_lead + 127) / 128), g1 = (unsigned)((ng - np - n_lead + 127) / 128);
        if (b->kind == SMART_FILTER_POLY) {
            if (np > 0)
                k_pixel_batched_general_pairs<SMART_FILTER_POLY><<<gp, 128, 0, gs>>>(b->d_maps, b->d_gen, np, n_lead, b->gb);
            if (ng > np + n_lead)
                k_pixel_batched_general<SMART_FILTER_POLY><<<g1, 128, 0, gs>>>(b->d_maps, b->d_gen, np + n_lead, ng, b->gb);
            k_pixel_batched_band<SMART_FILTER_POLY><<<4 * sms, 128, 0, gs>>>(b->d_maps, b->d_gen, b->gb);
        } else {
            if (np > 0)
                k_pixel_batched_general_pairs<SMART_FILTER_SCHIRMER><<<gp, 128, 0, gs>>>(b->d_maps, b->d_gen, np, n_lead,
                                                                                        b->gb);
            if (ng > np + n_lead)
                k_pixel_batched_general<SMART_FILTER_SCHIRMER><<<g1, 128, 0, gs>>>(b->d_maps, b->d_gen, np + n_lead, ng,
                                                                                  b->gb);
            k_pixel_batched_band<SMART_FILTER_SCHIRMER><<<4 * sms, 128, 0, gs>>>(b->d_maps, b->d_gen, b->gb);
        }
    }
    if (b->n_items > 0) {
        const unsigned grid = (unsigned)std::min<int64_t>(b->n_items, (int64_t)sms * ctas_per_sm);
        const BatchItem *items = b->d_items + (order == 0 ? 0 : b->n_items);
        const bool poly = b->kind == SMART_FILTER_POLY;
        if (b->short_runs) {
            if (poly)
                k_pixel_batched<SMART_FILTER_POLY, NCAND_SHORT><<<grid, NT, 0, b->stream>>>(b->d_maps, items, b->n_items,
                                                                                           b->d_work);
            else
                k_pixel_batched<SMART_FILTER_SCHIRMER, NCAND_SHORT><<<grid, NT, 0, b->stream>>>(b->d_maps, items,
                                                                                               b->n_items, b->d_work);
        } else {
            if (poly)
                k_pixel_batched<SMART_FILTER_POLY, NCAND><<<grid, NT, 0, b->stream>>>(b->d_maps, items, b->n_items,
                                                                                     b->d_work);
            else
                k_pixel_batched<SMART_FILTER_SCHIRMER, NCAND><<<grid, NT, 0, b->stream>>>(b->d_maps, items, b->n_items,
                                                                                         b->d_work);
        }
    }
    if (fork) {
        if (cudaEventRecord(b->ev_join, b->side) != cudaSuccess ||
            cudaStreamWaitEvent(b->stream, b->ev_join, 0) != cudaSuccess)
            return bfail(b, SMART_E_CUDA, "join of the general launch failed");
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bfail(b, SMART_E_CUDA, std::string("k_pixel_batched: ") + cudaGetErrorString(e));
    return SMART_OK;
}

// process-wide memory of tuned launch shapes, keyed by the batch's shape
static std::map<std::string, std::pair<int, int>> &tune_cache() {
    static std::map<std::string, std::pair<int, int>> m;
    return m;
}

extern "C" void smart_batch_destroy(smart_batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->d_maps) cudaFree(b->d_maps);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_gen) cudaFree(b->d_gen);
    if (b->d_work) cudaFree(b->d_work);
    if (b->d_band) cudaFree(b->d_band);
    if (b->d_band_count) cudaFree(b->d_band_count);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    if (b->side) {
        cudaStreamSynchronize(b->side);
        cudaStreamDestroy(b->side);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    delete b;
}

extern "C" smart_status smart_batch_create(smart_ctx *const *ctxs, const smart_maps *outs, int n_maps, int autotune,
                                           void *cuda_stream, smart_batch **out) {
    if (!out) return SMART_E_ARG;
    *out = nullptr;
    if (!ctxs || !outs || n_maps < 1 || n_maps > (1 << 20)) return SMART_E_ARG;
    smart_batch *b = new (std::nothrow) smart_batch();
    if (!b) return SMART_E_NOMEM;
    g_create_err.clear();
    b->stream = (cudaStream_t)cuda_stream;
    if (!b->stream) {
        // graphs cannot be captured on the legacy default stream: use a
        // private blocking stream (it orders itself against the legacy stream)
        if (cudaStreamCreate(&b->stream) != cudaSuccess) {
            delete b;
            return SMART_E_CUDA;
        }
        b->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        bfail(b, SMART_E_CUDA, "side stream or events could not be created");
        smart_batch_destroy(b);
        return SMART_E_CUDA;
    }
    b->kind = ctxs[0] ? ctxs[0]->filter_kind : 0;
    for (int m = 0; m < n_maps; ++m) {
        if (!ctxs[m] || ctxs[m]->filter_kind != b->kind) {
            bfail(b, SMART_E_ARG, "every map of a batch must use the same filter kind");
            smart_batch_destroy(b);
            return SMART_E_ARG;
        }
        if (ctxs[m]->norm != SMART_NORM_SUMMED) {
            bfail(b, SMART_E_ARG, "batches use the summed normalisation");
            smart_batch_destroy(b);
            return SMART_E_ARG;
        }
    }
    b->ctxs.assign(ctxs, ctxs + n_maps);
    b->args.resize(n_maps);
    smart_status st = SMART_OK;
    std::vector<BatchItem> items;
    std::vector<double> cost;
    std::vector<int4> gen, gen_single;
    for (int m = 0; m < n_maps && st == SMART_OK; ++m) {
        smart_ctx *c = ctxs[m];
        cudaStream_t keep = c->stream;
        c->stream = b->stream;
        MapArgs a{};
        st = prepare_pixel(c, &outs[m], a);
        if (st != SMART_OK) {
            b->err = "map " + std::to_string(m) + ": " + c->err;
            c->stream = keep;
            break;
        }
        a.work = nullptr;
        a.fp64_count = c->d_fp64_count;
        b->args[m] = a;
        if (c->toe_max_run > NCAND_SHORT) {
            b->short_runs = false;
            b->ctas_per_sm = toe_ctas_per_sm<NCAND>();
        }
        // the per-pair cost grows with the number of pixels in an aperture
        const double pix_per_ap = 3.0 * c->nside_bin * c->nside_bin / SMART_PI * c->area;
        if (a.n > 0 && a.n_gen < a.n) {
            std::vector<int64_t> tiles(a.n_tiles + 1);
            std::vector<unsigned char> want(a.n_tiles);
            unsigned char *d_want = nullptr;
            if (cudaMalloc(&d_want, (size_t)std::max<int64_t>(a.n_tiles, 1)) != cudaSuccess) {
                st = bfail(b, SMART_E_NOMEM, "cudaMalloc(tile flags) failed");
            } else {
                k_tiles_wanted<<<(unsigned)std::min<int64_t>((a.n_tiles + 255) / 256, 4096), 256, 0, b->stream>>>(a, d_want);
                cudaMemcpyAsync(want.data(), d_want, (size_t)a.n_tiles, cudaMemcpyDeviceToHost, b->stream);
                cudaMemcpyAsync(tiles.data(), a.tiles, (size_t)(a.n_tiles + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, b->stream);
                if (cudaStreamSynchronize(b->stream) != cudaSuccess) st = bfail(b, SMART_E_CUDA, "tile list download failed");
                cudaFree(d_want);
            }
            for (int64_t t = 0; t < a.n_tiles && st == SMART_OK; ++t) {
                if (!want[t]) continue;
                BatchItem it{t, m, 0, 0, 0};
                items.push_back(it);
                cost.push_back((double)(tiles[t + 1] - tiles[t]) * pix_per_ap);
            }
        }
        if (a.n_work > 0 && st == SMART_OK) {
            std::vector<int2> gw(a.n_work);
            cudaMemcpyAsync(gw.data(), a.gen_work, (size_t)a.n_work * sizeof(int2), cudaMemcpyDeviceToHost, b->stream);
            if (cudaStreamSynchronize(b->stream) != cudaSuccess) st = bfail(b, SMART_E_CUDA, "general list download failed");
            for (int64_t g = 0; g < a.n_work && st == SMART_OK; ++g)
                (g < a.n_pairs ? gen : gen_single).push_back(make_int4(m, gw[g].x, gw[g].y, 0));
            b->n_gen_targets += a.n_gen;
        }
        c->stream = keep;
    }
    if (st != SMART_OK) {
        smart_batch_destroy(b);
        return st;
    }
    b->n_items = (int64_t)items.size();
    std::vector<int64_t> idx(items.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int64_t)i;
    std::stable_sort(idx.begin(), idx.end(), [&](int64_t x, int64_t y) { return cost[x] > cost[y]; });
    b->natural = items;
    b->by_cost.resize(items.size());
    for (size_t i = 0; i < idx.size(); ++i) b->by_cost[i] = items[idx[i]];
    const size_t nb = std::max<size_t>(1, items.size());
    b->n_gen_pairs = (int64_t)gen.size();
    gen.insert(gen.end(), gen_single.begin(), gen_single.end());
    b->n_gen = (int64_t)gen.size();
    if (cudaMalloc(&b->d_maps, sizeof(MapArgs) * n_maps) != cudaSuccess ||
        cudaMalloc(&b->d_items, sizeof(BatchItem) * 2 * nb) != cudaSuccess ||
        cudaMalloc(&b->d_gen, sizeof(int4) * std::max<size_t>(1, gen.size())) != cudaSuccess ||
        cudaMalloc(&b->d_work, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&b->d_band, (size_t)(GEN_BAND_SLOT_BYTES * gen_band_slots(b->n_gen_targets))) != cudaSuccess ||
        cudaMalloc(&b->d_band_count, sizeof(unsigned long long)) != cudaSuccess) {
        bfail(b, SMART_E_NOMEM, "cudaMalloc(batch tables) failed");
        smart_batch_destroy(b);
        return SMART_E_NOMEM;
    }
    b->gb = gen_band_layout(b->d_band, gen_band_slots(b->n_gen_targets), b->d_band_count);
    cudaMemcpyAsync(b->d_maps, b->args.data(), sizeof(MapArgs) * n_maps, cudaMemcpyHostToDevice, b->stream);
    if (!gen.empty())
        cudaMemcpyAsync(b->d_gen, gen.data(), sizeof(int4) * gen.size(), cudaMemcpyHostToDevice, b->stream);
    if (!items.empty()) {
        cudaMemcpyAsync(b->d_items, b->by_cost.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice, b->stream);
        cudaMemcpyAsync(b->d_items + items.size(), b->natural.data(), sizeof(BatchItem) * items.size(),
                        cudaMemcpyHostToDevice, b->stream);
    }
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
        bfail(b, SMART_E_CUDA, "batch table upload failed");
        smart_batch_destroy(b);
        return SMART_E_CUDA;
    }

    // ---- autotuner: resident CTAs per SM x item order, timed on this batch
    std::string key = std::to_string(b->kind) + ":" + std::to_string(n_maps) + ":" + std::to_string(b->n_items);
    for (int m = 0; m < std::min(n_maps, 8); ++m) key += ":" + std::to_string(ctxs[m]->nside_bin) + "/" + std::to_string(ctxs[m]->n_targets);
    auto hit = tune_cache().find(key);
    if (hit != tune_cache().end()) {
        b->ctas_per_sm = hit->second.first;
        b->order = hit->second.second;
    } else if (autotune && b->n_items + b->n_gen > 0) {
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        double best = 1e30;
        // resident one-warp CTAs per SM: the register or shared-memory limit, and fewer
        const int cmax = b->short_runs ? toe_ctas_per_sm<NCAND_SHORT>() : toe_ctas_per_sm<NCAND>();
        const int shapes[] = {cmax - 4, cmax - 2, cmax};
        for (int order = 0; order < 2 && st == SMART_OK; ++order) {
            for (int cps : shapes) {
                st = batch_launch(b, cps, order);       // warm
                if (st != SMART_OK) break;
                cudaEventRecord(e0, b->stream);
                st = batch_launch(b, cps, order);
                if (st != SMART_OK) break;
                cudaEventRecord(e1, b->stream);
                if (cudaEventSynchronize(e1) != cudaSuccess) {
                    st = bfail(b, SMART_E_CUDA, "autotune timing failed");
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) {
                    best = ms;
                    b->ctas_per_sm = cps;
                    b->order = order;
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (st != SMART_OK) {
            smart_batch_destroy(b);
            return st;
        }
        b->tuned_ms = best;
        tune_cache()[key] = std::make_pair(b->ctas_per_sm, b->order);
    }

    // ---- capture the launch (count prefixes + batched kernel) in a graph
    cudaError_t ce = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) {
        bfail(b, SMART_E_CUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(ce));
        smart_batch_destroy(b);
        return SMART_E_CUDA;
    }
    st = batch_launch(b, b->ctas_per_sm, b->order);
    cudaGraph_t g = nullptr;
    ce = cudaStreamEndCapture(b->stream, &g);
    if (st != SMART_OK || ce != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        if (st == SMART_OK) bfail(b, SMART_E_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ce));
        smart_batch_destroy(b);
        return st != SMART_OK ? st : SMART_E_CUDA;
    }
    b->graph = g;
    ce = cudaGraphInstantiate(&b->exec, g, 0);
    if (ce != cudaSuccess) {
        bfail(b, SMART_E_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ce));
        smart_batch_destroy(b);
        return SMART_E_CUDA;
    }
    *out = b;
    return SMART_OK;
}

extern "C" smart_status smart_batch_run(smart_batch *b) {
    if (!b || !b->exec) return SMART_E_ARG;
    const cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
    if (e != cudaSuccess) return bfail(b, SMART_E_CUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
    return SMART_OK;
}

extern "C" smart_status smart_batch_info(const smart_batch *b, int *ctas_per_sm, int *longest_first,
                                         int64_t *n_items, double *tuned_ms) {
    if (!b) return SMART_E_ARG;
    if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
    if (longest_first) *longest_first = b->order == 0;
    if (n_items) *n_items = b->n_items;
    if (tuned_ms) *tuned_ms = b->tuned_ms;
    return SMART_OK;
}

extern "C" const char *smart_batch_last_error(const smart_batch *b) {
    return b ? b->err.c_str() : g_create_err.c_str();
}

extern "C" smart_status smart_map_batched(smart_ctx *const *ctxs, const smart_maps *outs, int n_maps) {
    if (!ctxs || n_maps < 1 || !ctxs[0]) return SMART_E_ARG;
    smart_batch *b = nullptr;
    smart_status st = smart_batch_create(ctxs, outs, n_maps, 0, ctxs[0]->stream, &b);
    if (st != SMART_OK) return st;
    st = smart_batch_run(b);
    smart_batch_destroy(b);          // synchronises the stream
    return st;
}
