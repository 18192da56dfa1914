// Learned residual correction of the pixel-based map.
//
// The pixel-based map (Sect. 3.2) moves every galaxy to its pixel centre;
// the galaxy-level map (Sect. 3.1) does not.  A 4 -> 64 -> 64 -> 1 SiLU
// network predicts their per-pixel difference M_bf^E - M_pix^E from four
// features of the pixel-based map: M_pix^E, the weight sum, the variance of
// the galaxy counts over the aperture's pixels, and z of the pixel centre.
// The corrected map is written to a separate array; the plain map is never
// changed and is the per-pixel fallback.
//
// Kernels (all on the caller's stream):
//   k_mlp_features   one thread per target: sum of n_p^2 over the aperture's
//                    pixels with the membership of the map kernels (float32
//                    test outside a guard band, float64 inside), features,
//                    training target and validity flag.
//   k_mlp_grad<TC>   one CTA per 128 samples: forward and backward of the
//                    whole network with the activations in shared memory;
//                    the 64 x 64 products (forward, input gradient, weight
//                    gradient) run on mma.sync m16n8k16 bf16 tensor cores
//                    with float32 accumulation (TC = true), or on float32
//                    CUDA cores (TC = false, the checking mode).  Writes the
//                    CTA's gradient and loss partials.
//   k_mlp_reduce     deterministic sum of the CTA partials (fixed order).
//   k_mlp_adam       Adam on the float32 master copy, refreshes the bf16
//                    weight copy.
//   k_mlp_infer<TC>  forward only; corrected = plain + prediction, or plain
//                    where a feature is not finite or lies outside the
//                    training range.
//   k_moments        deterministic float64 mean / variance of the features
//                    and target (standardisation).
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <chrono>
#include <string>
#include <thread>

#include "smart_internal.cuh"
#include "aperture_common.cuh"
#include "aperture_pixel.cuh"

namespace smart {
namespace mlp {

constexpr int F = SMART_MLP_FEATURES;   // 4
constexpr int H = 64;
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + H * F;
constexpr int OFF_W2 = OFF_B1 + H;
constexpr int OFF_B2 = OFF_W2 + H * H;
constexpr int OFF_W3 = OFF_B2 + H;
constexpr int OFF_B3 = OFF_W3 + H;
constexpr int NP = OFF_B3 + 1;
static_assert(NP == SMART_MLP_NPARAMS, "parameter layout");
constexpr int PSTRIDE = NP + 1;          // partial row: gradient, then the loss sum
constexpr int S = 128;                   // samples per CTA
constexpr int NTH = 256;                 // 8 warps; warp w owns samples [16 w, 16 w + 16)
constexpr int LDH = H + 8;               // bf16 row stride of [S][H] and [H][H] tiles (conflict-free fragments)
constexpr int LDT = S + 8;               // bf16 row stride of [H][S] tiles
constexpr int LDF = H + 4;               // float row stride
constexpr float XMAX = 8.0f;             // standardised features beyond this fall back to the plain map
static_assert(S == 16 * (NTH / 32), "one m16 tile of samples per warp");

struct Scaler {
    float mu[F], isd[F];
    float t_mu, t_sd, t_isd;
};

// shared-memory image of one CTA: weights, a tile of samples and every
// activation the backward pass needs
template <bool TC>
struct Smem;

template <>
struct Smem<true> {
    __nv_bfloat16 W2[H * LDH];     // [n][k]
    __nv_bfloat16 W2T[H * LDH];    // [k][n]
    __nv_bfloat16 H1[S * LDH];     // [r][k]  first hidden activation (mma operand)
    __nv_bfloat16 H1T[H * LDT];    // [k][r]
    __nv_bfloat16 D2[S * LDH];     // [r][n]  gradient at the second pre-activation
    __nv_bfloat16 D2T[H * LDT];    // [n][r]
    float A1[S * LDF];             // first pre-activation, then its gradient
    float A2[S * LDF];             // second pre-activation
    float W1[H * F], b1[H], b2[H], w3[H];
    float X[S * F], T[S], DY[S], M[S];
    float red[4 * H];
    float b3;
};

template <>
struct Smem<false> {
    float W2[H * H];               // [n][k]
    float H1[S * H];               // [r][k]
    float D2[S * H];               // [r][n]
    float A1[S * LDF];
    float A2[S * LDF];
    float W1[H * F], b1[H], b2[H], w3[H];
    float X[S * F], T[S], DY[S], M[S];
    float red[4 * H];
    float b3;
};

// forward-only image (inference): no transposes, no first pre-activation
template <bool TC>
struct SmemInf;

template <>
struct SmemInf<true> {
    __nv_bfloat16 W2[H * LDH];
    __nv_bfloat16 H1[S * LDH];
    float A2[S * LDF];
    float W1[H * F], b1[H], b2[H], w3[H];
    float X[S * F], T[S], DY[S], M[S];
    float b3;
};

template <>
struct SmemInf<false> {
    float W2[H * H];
    float H1[S * H];
    float A2[S * LDF];
    float W1[H * F], b1[H], b2[H], w3[H];
    float X[S * F], T[S], DY[S], M[S];
    float b3;
};

__device__ __forceinline__ float sigmoidf_(float a) { return 1.0f / (1.0f + __expf(-a)); }

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

// D += A (16x16, row) * B (16x8, col); bf16 operands, float32 accumulators
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// A fragment of rows [r0, r0 + 16), columns [k0, k0 + 16) of a row-major bf16 tile
__device__ __forceinline__ void load_a(uint32_t (&a)[4], const __nv_bfloat16 *M, int ld, int r0, int k0, int g, int tg) {
    a[0] = ld32(M + (r0 + g) * ld + k0 + 2 * tg);
    a[1] = ld32(M + (r0 + g + 8) * ld + k0 + 2 * tg);
    a[2] = ld32(M + (r0 + g) * ld + k0 + 8 + 2 * tg);
    a[3] = ld32(M + (r0 + g + 8) * ld + k0 + 8 + 2 * tg);
}

// B fragment (K rows [k0, k0 + 16), N columns [n0, n0 + 8)) from a tile stored
// column by column: Bt[n][k]
__device__ __forceinline__ void load_b(uint32_t &b0, uint32_t &b1, const __nv_bfloat16 *Bt, int ld, int n0, int k0, int g,
                                       int tg) {
    b0 = ld32(Bt + (n0 + g) * ld + k0 + 2 * tg);
    b1 = ld32(Bt + (n0 + g) * ld + k0 + 8 + 2 * tg);
}

template <bool TC, bool TRAIN = true, typename SM = Smem<TC>>
__device__ void load_weights(SM &s, const float *theta, const __nv_bfloat16 *wb) {
    for (int i = threadIdx.x; i < H * F; i += NTH) s.W1[i] = TC ? __bfloat162float(wb[OFF_W1 + i]) : theta[OFF_W1 + i];
    for (int i = threadIdx.x; i < H; i += NTH) {
        s.b1[i] = theta[OFF_B1 + i];
        s.b2[i] = theta[OFF_B2 + i];
        s.w3[i] = TC ? __bfloat162float(wb[OFF_W3 + i]) : theta[OFF_W3 + i];
    }
    if (threadIdx.x == 0) s.b3 = theta[OFF_B3];
    for (int i = threadIdx.x; i < H * H; i += NTH) {
        if constexpr (TC) {
            const int n = i / H, k = i % H;
            const __nv_bfloat16 w = wb[OFF_W2 + i];
            s.W2[n * LDH + k] = w;
            if constexpr (TRAIN) s.W2T[k * LDH + n] = w;
        } else {
            s.W2[i] = theta[OFF_W2 + i];
        }
    }
}

// standardised features (and target) of samples [base, base + S); rows past
// `count` get mask 0.  in_range (optional) marks the samples
// whose raw features are finite, whose weight sum is positive and whose
// standardised features lie within +-XMAX.
template <bool TC, typename SM = Smem<TC>>
__device__ void load_samples(SM &s, const float *feat, const float *target, const int32_t *idx, int64_t base,
                             int64_t count, const Scaler &sc, bool *in_range) {
    for (int r = threadIdx.x; r < S; r += NTH) {
        const int64_t q = base + r;
        float x[F] = {0.f, 0.f, 0.f, 0.f};
        float t = 0.f, m = 0.f;
        bool ok = false;
        if (q < count) {
            const int64_t gi = idx ? (int64_t)idx[q] : q;
            ok = feat[gi * F + 1] > 0.f;
            for (int f = 0; f < F; ++f) {
                const float v = feat[gi * F + f];
                x[f] = (v - sc.mu[f]) * sc.isd[f];
                ok = ok && isfinite(v) && fabsf(x[f]) <= XMAX;
            }
            if (target) t = (target[gi] - sc.t_mu) * sc.t_isd;
            m = 1.f;
        }
        for (int f = 0; f < F; ++f) s.X[r * F + f] = ok || target ? x[f] : 0.f;
        s.T[r] = t;
        s.M[r] = m;
        if (in_range) in_range[r] = ok;
    }
}

// layer 1 and the 64 x 64 layer: A1, H1, A2 (pre-activation incl. bias)
template <bool TC, bool TRAIN = true, typename SM = Smem<TC>>
__device__ void forward_tile(SM &s) {
    for (int e = threadIdx.x; e < S * H; e += NTH) {
        const int r = e / H, n = e % H;
        float a = s.b1[n];
#pragma unroll
        for (int f = 0; f < F; ++f) a = fmaf(s.W1[n * F + f], s.X[r * F + f], a);
        if constexpr (TRAIN) s.A1[r * LDF + n] = a;
        const float h = a * sigmoidf_(a);
        if constexpr (TC) {
            const __nv_bfloat16 hb = __float2bfloat16_rn(h);
            s.H1[r * LDH + n] = hb;
            if constexpr (TRAIN) s.H1T[n * LDT + r] = hb;
        } else {
            s.H1[r * H + n] = h;
        }
    }
    __syncthreads();
    if constexpr (TC) {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tg = lane & 3;
        const int r0 = 16 * warp;
        uint32_t af[4][4];
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) load_a(af[ks], s.H1, LDH, r0, 16 * ks, g, tg);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                uint32_t b0, b1;
                load_b(b0, b1, s.W2, LDH, 8 * nt, 16 * ks, g, tg);
                mma_bf16(c, af[ks], b0, b1);
            }
            const int n0 = 8 * nt + 2 * tg;
            s.A2[(r0 + g) * LDF + n0] = c[0] + s.b2[n0];
            s.A2[(r0 + g) * LDF + n0 + 1] = c[1] + s.b2[n0 + 1];
            s.A2[(r0 + g + 8) * LDF + n0] = c[2] + s.b2[n0];
            s.A2[(r0 + g + 8) * LDF + n0 + 1] = c[3] + s.b2[n0 + 1];
        }
    } else {
        for (int e = threadIdx.x; e < S * H; e += NTH) {
            const int r = e / H, n = e % H;
            float a = 0.f;
            for (int k = 0; k < H; ++k) a = fmaf(s.H1[r * H + k], s.W2[n * H + k], a);
            s.A2[r * LDF + n] = a + s.b2[n];
        }
    }
    __syncthreads();
}

// output of sample r (threads 0..S-1)
template <bool TC>
__device__ __forceinline__ float head(const Smem<TC> &s, int r) {
    float y = s.b3;
    for (int n = 0; n < H; ++n) {
        const float a = s.A2[r * LDF + n];
        y = fmaf(s.w3[n], a * sigmoidf_(a), y);
    }
    return y;
}

struct GradArgs {
    const float *feat, *target;
    const int32_t *idx;
    int64_t batch;
    float inv_batch;
    Scaler sc;
    const float *theta;
    const __nv_bfloat16 *wb;
    float *partial;                  // [gridDim.x][PSTRIDE]
};

template <bool TC>
__global__ void __launch_bounds__(NTH, 1) k_mlp_grad(const GradArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<TC> &s = *reinterpret_cast<Smem<TC> *>(smem_raw);
    const int tid = threadIdx.x;
    load_weights<TC>(s, a.theta, a.wb);
    load_samples<TC>(s, a.feat, a.target, a.idx, (int64_t)blockIdx.x * S, a.batch, a.sc, nullptr);
    __syncthreads();
    forward_tile<TC>(s);

    // loss and output gradient
    if (tid < S) {
        const float d = s.M[tid] * (head<TC>(s, tid) - s.T[tid]);
        s.DY[tid] = 2.0f * d * a.inv_batch;
        s.red[tid] = d * d;
    }
    __syncthreads();
    float *out = a.partial + (int64_t)blockIdx.x * PSTRIDE;
    if (tid == 0) {
        float L = 0.f, gb3 = 0.f;
        for (int r = 0; r < S; ++r) {
            L += s.red[r];
            gb3 += s.DY[r];
        }
        out[NP] = L;
        out[OFF_B3] = gb3;
    }
    __syncthreads();

    // gradient at the second pre-activation; w3 and b2 gradients (column n,
    // quarter q of the samples)
    {
        const int n = tid % H, q = tid / H;
        float gw3 = 0.f, gb2 = 0.f;
        for (int rr = 0; rr < S / 4; ++rr) {
            const int r = q * (S / 4) + rr;
            const float a2 = s.A2[r * LDF + n];
            const float sg = sigmoidf_(a2);
            const float dy = s.DY[r];
            gw3 = fmaf(dy, a2 * sg, gw3);
            const float g2 = dy * s.w3[n] * (sg * (1.0f + a2 * (1.0f - sg)));
            gb2 += g2;
            if constexpr (TC) {
                const __nv_bfloat16 gb = __float2bfloat16_rn(g2);
                s.D2[r * LDH + n] = gb;
                s.D2T[n * LDT + r] = gb;
            } else {
                s.D2[r * H + n] = g2;
            }
        }
        s.red[q * H + n] = gw3;
        __syncthreads();
        if (tid < H) out[OFF_W3 + tid] = ((s.red[tid] + s.red[H + tid]) + s.red[2 * H + tid]) + s.red[3 * H + tid];
        __syncthreads();
        s.red[q * H + n] = gb2;
        __syncthreads();
        if (tid < H) out[OFF_B2 + tid] = ((s.red[tid] + s.red[H + tid]) + s.red[2 * H + tid]) + s.red[3 * H + tid];
    }
    __syncthreads();

    // gradient at the first pre-activation: dA1 = (D2 W2) * silu'(A1), in place of A1
    if constexpr (TC) {
        const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, tg = lane & 3;
        const int r0 = 16 * warp;
        uint32_t af[4][4];
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) load_a(af[ks], s.D2, LDH, r0, 16 * ks, g, tg);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                uint32_t b0, b1;
                load_b(b0, b1, s.W2T, LDH, 8 * nt, 16 * ks, g, tg);
                mma_bf16(c, af[ks], b0, b1);
            }
            const int k0 = 8 * nt + 2 * tg;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int r = r0 + g + (j >> 1) * 8, k = k0 + (j & 1);
                const float a1 = s.A1[r * LDF + k];
                const float sg = sigmoidf_(a1);
                s.A1[r * LDF + k] = c[j] * (sg * (1.0f + a1 * (1.0f - sg)));
            }
        }
    } else {
        for (int e = tid; e < S * H; e += NTH) {
            const int r = e / H, k = e % H;
            float d = 0.f;
            for (int n = 0; n < H; ++n) d = fmaf(s.D2[r * H + n], s.W2[n * H + k], d);
            const float a1 = s.A1[r * LDF + k];
            const float sg = sigmoidf_(a1);
            s.A1[r * LDF + k] = d * (sg * (1.0f + a1 * (1.0f - sg)));
        }
    }
    __syncthreads();

    // weight gradient of the 64 x 64 layer: gW2 = D2^T H1
    if constexpr (TC) {
        const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, tg = lane & 3;
        const int m0 = 16 * (warp >> 1), ntb = 4 * (warp & 1);
        float acc[4][4] = {};
#pragma unroll
        for (int ks = 0; ks < S / 16; ++ks) {
            uint32_t af[4];
            load_a(af, s.D2T, LDT, m0, 16 * ks, g, tg);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                uint32_t b0, b1;
                load_b(b0, b1, s.H1T, LDT, 8 * (ntb + j), 16 * ks, g, tg);
                mma_bf16(acc[j], af, b0, b1);
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k0 = 8 * (ntb + j) + 2 * tg;
            out[OFF_W2 + (m0 + g) * H + k0] = acc[j][0];
            out[OFF_W2 + (m0 + g) * H + k0 + 1] = acc[j][1];
            out[OFF_W2 + (m0 + g + 8) * H + k0] = acc[j][2];
            out[OFF_W2 + (m0 + g + 8) * H + k0 + 1] = acc[j][3];
        }
    } else {
        for (int e = tid; e < H * H; e += NTH) {
            const int n = e / H, k = e % H;
            float acc = 0.f;
            for (int r = 0; r < S; ++r) acc = fmaf(s.D2[r * H + n], s.H1[r * H + k], acc);
            out[OFF_W2 + e] = acc;
        }
    }
    // first layer: gW1[n][f] = sum_r dA1[r][n] X[r][f]; gb1[n] = sum_r dA1[r][n]
    {
        const int n = tid / F, f = tid % F;
        float acc = 0.f;
        for (int r = 0; r < S; ++r) acc = fmaf(s.A1[r * LDF + n], s.X[r * F + f], acc);
        out[OFF_W1 + tid] = acc;
        if (tid < H) {
            float gb = 0.f;
            for (int r = 0; r < S; ++r) gb += s.A1[r * LDF + tid];
            out[OFF_B1 + tid] = gb;
        }
    }
}

__global__ void k_mlp_reduce(const float *__restrict__ partial, int nblocks, float *__restrict__ grad) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= PSTRIDE) return;
    float acc = 0.f;
    for (int b = 0; b < nblocks; ++b) acc += partial[(int64_t)b * PSTRIDE + p];
    grad[p] = acc;
}

__global__ void k_mlp_adam(float *__restrict__ theta, float *__restrict__ m, float *__restrict__ v,
                           const float *__restrict__ grad, __nv_bfloat16 *__restrict__ wb, float lr, float beta1,
                           float beta2, float eps, float bc1, float bc2, float *__restrict__ loss_out,
                           float inv_batch) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0 && loss_out) *loss_out = grad[NP] * inv_batch;
    if (p >= NP) return;
    const float g = grad[p];
    const float mm = beta1 * m[p] + (1.0f - beta1) * g;
    const float vv = beta2 * v[p] + (1.0f - beta2) * g * g;
    m[p] = mm;
    v[p] = vv;
    const float th = theta[p] - lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
    theta[p] = th;
    wb[p] = __float2bfloat16_rn(th);
}

__global__ void k_mlp_copy_bf16(const float *__restrict__ theta, __nv_bfloat16 *__restrict__ wb) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < NP) wb[p] = __float2bfloat16_rn(theta[p]);
}

struct InferArgs {
    const float *feat, *plain;
    int64_t n;
    Scaler sc;
    const float *theta;
    const __nv_bfloat16 *wb;
    float *out, *corr;
    unsigned long long *n_fallback;
};

// persistent: each CTA loads the weights once and walks tiles of S samples;
// the output layer uses two threads per sample (32 columns each)
template <bool TC>
__global__ void __launch_bounds__(NTH) k_mlp_infer(const InferArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemInf<TC> &s = *reinterpret_cast<SmemInf<TC> *>(smem_raw);
    __shared__ bool in_range[S];
    load_weights<TC, false>(s, a.theta, a.wb);
    const int64_t ntiles = (a.n + S - 1) / S;
    const int r = threadIdx.x >> 1, half = threadIdx.x & 1;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        load_samples<TC>(s, a.feat, nullptr, nullptr, tile * S, a.n, a.sc, in_range);
        __syncthreads();
        forward_tile<TC, false>(s);
        float y = 0.f;
        for (int n = half * (H / 2); n < (half + 1) * (H / 2); ++n) {
            const float a2 = s.A2[r * LDF + n];
            y = fmaf(s.w3[n], a2 * sigmoidf_(a2), y);
        }
        y += __shfl_xor_sync(0xffffffffu, y, 1);
        const int64_t q = tile * S + r;
        if (half == 0 && q < a.n) {
            const float plain = a.plain[q];
            float c = 0.f;
            if (in_range[r]) c = fmaf(y + s.b3, a.sc.t_sd, a.sc.t_mu);
            else if (a.n_fallback) atomicAdd(a.n_fallback, 1ull);
            a.out[q] = plain + c;
            if (a.corr) a.corr[q] = c;
        }
        __syncthreads();       // the next tile overwrites the activations
    }
}

// float64 column moments of [feat | target] over rows (deterministic):
// pass 0 sums x, pass 1 sums (x - mean)^2
constexpr int MOM_BLOCKS = 296, MOM_THREADS = 256, MOM_COLS = F + 1;

__global__ void __launch_bounds__(MOM_THREADS) k_moments(const float *__restrict__ feat, const float *__restrict__ target,
                                                         const int32_t *__restrict__ rows, int64_t n,
                                                         const double *__restrict__ mean, double *__restrict__ part) {
    __shared__ double red[MOM_COLS][MOM_THREADS];
    double acc[MOM_COLS] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t i = blockIdx.x * (int64_t)MOM_THREADS + threadIdx.x; i < n; i += (int64_t)MOM_BLOCKS * MOM_THREADS) {
        const int64_t r = rows ? (int64_t)rows[i] : i;
        for (int c = 0; c < MOM_COLS; ++c) {
            const double x = c < F ? (double)feat[r * F + c] : (double)target[r];
            const double d = mean ? x - mean[c] : x;
            acc[c] += mean ? d * d : d;
        }
    }
    for (int c = 0; c < MOM_COLS; ++c) red[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int w = MOM_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < MOM_COLS; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < MOM_COLS) part[blockIdx.x * MOM_COLS + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void k_moments_final(const double *__restrict__ part, int64_t n, double *__restrict__ out) {
    const int c = threadIdx.x;
    if (c >= MOM_COLS) return;
    double s = 0.0;
    for (int b = 0; b < MOM_BLOCKS; ++b) s += part[b * MOM_COLS + c];
    out[c] = n > 0 ? s / (double)n : 0.0;
}

// ------------------------------------------------------------ features
struct FeatArgs {
    MapArgs m;
    const float *px_e;
    const double *px_w;
    const int64_t *px_count;
    const int32_t *px_members;
    const float *bf_e;
    const double *bf_w;
    float *feat, *target;
    uint8_t *valid;
    int64_t *sum_n2;
};

template <int MODE>
__device__ int64_t sum_n2_segment(const MapArgs &a, const RingPair &R, const TargetRing &tr, int64_t pix) {
    const int q = R.nr >> 2;
    int Xi;
    float Xf;
    lattice_position(tr, q, Xi, Xf);
    const float fr = ((R.flags & RP_SHIFTED) ? 0.5f : 0.0f) - Xf;
    int kl, kh;
    window(R, fr, kl, kh);
    int kk = (Xi + kl) % R.nr;
    if (kk < 0) kk += R.nr;
    const float u0 = fr * R.dphi;
    float kf = (float)kl;
    int64_t acc = 0;
    for (int k = kl; k <= kh; ++k) {
        const float u = fmaf(kf, R.dphi, u0);
        kf += 1.0f;
        float sinu, h;
        sin_hav<MODE>(u, sinu, h);
        const float s2 = fmaf(R.B, h, R.A);
        const int p = R.start + kk;
        kk = (kk + 1 == R.nr) ? 0 : kk + 1;
        // the membership of the map kernels: float32 outside the guard band,
        // float64 inside it
        const bool in = s2 < a.Tlo || (s2 <= a.Thi && exact_member(a, pix, p));
        if (in) {
            const int64_t c = a.NP[p];
            acc += c * c;
        }
    }
    return acc;
}

__global__ void k_mlp_features(const FeatArgs fa) {
    const MapArgs &a = fa.m;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < a.n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pix = a.targets[t];
        const TargetRing tr = target_ring(a.N0, pix);
        const int64_t row0 = (int64_t)(tr.i0 - 1) * a.kmax;
        const int nent = a.counts[tr.i0 - 1];
        int64_t n2 = 0;
        for (int e = 0; e < nent; ++e) {
            const RingPair R = a.table[row0 + e];
            const int mode = (R.flags & RP_WIDE) ? 2 : (((R.hw + 1.0f) * R.dphi <= 0.05f) ? 0 : 1);
            if (mode == 0) n2 += sum_n2_segment<0>(a, R, tr, pix);
            else if (mode == 1) n2 += sum_n2_segment<1>(a, R, tr, pix);
            else n2 += sum_n2_segment<2>(a, R, tr, pix);
        }
        double x, y, z;
        pix2vec64(a.N0, pix, x, y, z);
        const int32_t K = fa.px_members[t];
        const double mean_n = K > 0 ? (double)fa.px_count[t] / K : 0.0;
        const double mean_n2 = K > 0 ? (double)n2 / K : 0.0;
        const double sw = fa.px_w[t];
        fa.feat[t * F + 0] = fa.px_e[t];
        fa.feat[t * F + 1] = (float)sw;
        fa.feat[t * F + 2] = (float)(mean_n2 - mean_n * mean_n);
        fa.feat[t * F + 3] = (float)z;
        bool ok = sw > 0.0;
        if (fa.bf_e) {
            if (fa.target) fa.target[t] = fa.bf_e[t] - fa.px_e[t];
            ok = ok && fa.bf_w[t] > 0.0;
        }
        if (fa.valid) fa.valid[t] = ok ? 1 : 0;
        if (fa.sum_n2) fa.sum_n2[t] = n2;
    }
}

}  // namespace mlp
}  // namespace smart

using namespace smart;
using namespace smart::mlp;

// ------------------------------------------------------------ the handle
struct smart_mlp {
    int precision = SMART_MLP_BF16;
    cudaStream_t stream = nullptr;
    std::string err;
    float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;   // float32 [NP] (grad: PSTRIDE)
    __nv_bfloat16 *wb = nullptr;                                         // bf16 copy [NP]
    float *partial = nullptr;
    int64_t cap_partial = 0;                                             // rows
    double *mom = nullptr;                                               // moments scratch
    double scaler[10] = {0, 0, 0, 0, 1, 1, 1, 1, 0, 1};                 // mu[4], sd[4], t_mu, t_sd
    int64_t step = 0;
    bool have_params = false;
};

namespace {

smart_status mfail(smart_mlp *h, smart_status st, const std::string &msg) {
    h->err = msg;
    return st;
}

smart_status mcheck(smart_mlp *h, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return SMART_OK;
    return mfail(h, SMART_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

Scaler make_scaler(const smart_mlp *h) {
    Scaler s;
    for (int f = 0; f < F; ++f) {
        s.mu[f] = (float)h->scaler[f];
        s.isd[f] = (float)(1.0 / h->scaler[4 + f]);
    }
    s.t_mu = (float)h->scaler[8];
    s.t_sd = (float)h->scaler[9];
    s.t_isd = (float)(1.0 / h->scaler[9]);
    return s;
}

template <bool TC>
smart_status launch_grad(smart_mlp *h, const float *feat, const float *target, const int32_t *idx, int64_t batch) {
    const int64_t blocks = (batch + S - 1) / S;
    if (blocks > h->cap_partial) {
        if (h->partial) cudaFree(h->partial);
        h->partial = nullptr;
        const int64_t cap = std::max<int64_t>(blocks, 64);
        if (cudaMalloc(&h->partial, (size_t)cap * PSTRIDE * sizeof(float)) != cudaSuccess)
            return mfail(h, SMART_E_NOMEM, "cudaMalloc(gradient partials) failed");
        h->cap_partial = cap;
    }
    const size_t smem = sizeof(Smem<TC>);
    smart_status st = mcheck(h, cudaFuncSetAttribute(k_mlp_grad<TC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)smem), "smem attribute");
    if (st != SMART_OK) return st;
    GradArgs a;
    a.feat = feat;
    a.target = target;
    a.idx = idx;
    a.batch = batch;
    a.inv_batch = (float)(1.0 / (double)batch);
    a.sc = make_scaler(h);
    a.theta = h->theta;
    a.wb = h->wb;
    a.partial = h->partial;
    k_mlp_grad<TC><<<(unsigned)blocks, NTH, smem, h->stream>>>(a);
    st = mcheck(h, cudaGetLastError(), "k_mlp_grad");
    if (st != SMART_OK) return st;
    k_mlp_reduce<<<(PSTRIDE + 255) / 256, 256, 0, h->stream>>>(h->partial, (int)blocks, h->grad);
    return mcheck(h, cudaGetLastError(), "k_mlp_reduce");
}

smart_status gradient(smart_mlp *h, const float *feat, const float *target, const int32_t *idx, int64_t batch) {
    if (!h->have_params) return mfail(h, SMART_E_STATE, "no parameters (smart_mlp_set_params first)");
    if (batch <= 0 || !feat || !target) return mfail(h, SMART_E_ARG, "bad batch, features or targets");
    if (batch > ((int64_t)1 << 31)) return mfail(h, SMART_E_OVERFLOW, "batch above 2^31 samples");
    return h->precision == SMART_MLP_BF16 ? launch_grad<true>(h, feat, target, idx, batch)
                                          : launch_grad<false>(h, feat, target, idx, batch);
}

constexpr uint32_t STATE_MAGIC = 0x504C4D53u;    // "SMLP"
constexpr uint32_t STATE_VERSION = 1;

int64_t state_size() {
    return 4 + 4 + 4 + 4 + 8 + 10 * 8 + 3 * (int64_t)NP * 4;
}

}  // namespace

extern "C" smart_status smart_mlp_create(int precision, void *cuda_stream, smart_mlp **out) {
    if (!out) return SMART_E_ARG;
    *out = nullptr;
    if (precision != SMART_MLP_BF16 && precision != SMART_MLP_FP32) return SMART_E_ARG;
    smart_mlp *h = new smart_mlp();
    h->precision = precision;
    h->stream = (cudaStream_t)cuda_stream;
    bool ok = cudaMalloc(&h->theta, NP * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&h->m, NP * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&h->v, NP * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&h->grad, PSTRIDE * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&h->wb, NP * sizeof(__nv_bfloat16)) == cudaSuccess &&
              cudaMalloc(&h->mom, (MOM_BLOCKS * MOM_COLS + 2 * MOM_COLS) * sizeof(double)) == cudaSuccess;
    if (!ok) {
        smart_mlp_destroy(h);
        return SMART_E_NOMEM;
    }
    *out = h;
    return SMART_OK;
}

extern "C" void smart_mlp_destroy(smart_mlp *h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    void *bufs[] = {h->theta, h->m, h->v, h->grad, h->wb, h->partial, h->mom};
    for (void *b : bufs)
        if (b) cudaFree(b);
    delete h;
}

extern "C" const char *smart_mlp_last_error(const smart_mlp *h) { return h ? h->err.c_str() : "null handle"; }

extern "C" smart_status smart_mlp_sync(smart_mlp *h, double timeout_s) {
    if (!h) return SMART_E_ARG;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t e = cudaStreamQuery(h->stream);
        if (e == cudaSuccess) return SMART_OK;
        if (e != cudaErrorNotReady) return mcheck(h, e, "smart_mlp_sync");
        const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (timeout_s > 0 && dt > timeout_s) return mfail(h, SMART_E_TIMEOUT, "smart_mlp_sync: deadline passed");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

extern "C" smart_status smart_mlp_set_params(smart_mlp *h, const float *params) {
    if (!h) return SMART_E_ARG;
    if (!params) return mfail(h, SMART_E_ARG, "null parameters");
    smart_status st = mcheck(h, cudaMemcpyAsync(h->theta, params, NP * sizeof(float), cudaMemcpyHostToDevice, h->stream),
                             "copy parameters");
    if (st != SMART_OK) return st;
    cudaMemsetAsync(h->m, 0, NP * sizeof(float), h->stream);
    cudaMemsetAsync(h->v, 0, NP * sizeof(float), h->stream);
    k_mlp_copy_bf16<<<(NP + 255) / 256, 256, 0, h->stream>>>(h->theta, h->wb);
    h->step = 0;
    h->have_params = true;
    st = mcheck(h, cudaGetLastError(), "k_mlp_copy_bf16");
    if (st != SMART_OK) return st;
    return mcheck(h, cudaStreamSynchronize(h->stream), "smart_mlp_set_params");
}

extern "C" smart_status smart_mlp_get_params(smart_mlp *h, float *params) {
    if (!h) return SMART_E_ARG;
    if (!params) return mfail(h, SMART_E_ARG, "null output");
    if (!h->have_params) return mfail(h, SMART_E_STATE, "no parameters");
    smart_status st = mcheck(h, cudaMemcpyAsync(params, h->theta, NP * sizeof(float), cudaMemcpyDeviceToHost, h->stream),
                             "copy parameters");
    if (st != SMART_OK) return st;
    return mcheck(h, cudaStreamSynchronize(h->stream), "smart_mlp_get_params");
}

extern "C" smart_status smart_mlp_set_scaler(smart_mlp *h, const double *scaler) {
    if (!h) return SMART_E_ARG;
    if (!scaler) return mfail(h, SMART_E_ARG, "null scaler");
    for (int i = 0; i < 10; ++i)
        if (!std::isfinite(scaler[i]) || ((i >= 4 && i < 8) || i == 9) && !(scaler[i] > 0.0))
            return mfail(h, SMART_E_ARG, "scaler: non-finite value or non-positive deviation");
    memcpy(h->scaler, scaler, sizeof(h->scaler));
    return SMART_OK;
}

extern "C" smart_status smart_mlp_get_scaler(smart_mlp *h, double *scaler) {
    if (!h || !scaler) return SMART_E_ARG;
    memcpy(scaler, h->scaler, sizeof(h->scaler));
    return SMART_OK;
}

extern "C" smart_status smart_mlp_fit_scaler(smart_mlp *h, const float *feat, const float *target, const int32_t *rows,
                                             int64_t n) {
    if (!h) return SMART_E_ARG;
    if (n <= 0 || !feat || !target) return mfail(h, SMART_E_ARG, "smart_mlp_fit_scaler: empty or null input");
    double *part = h->mom, *mean = h->mom + MOM_BLOCKS * MOM_COLS, *var = mean + MOM_COLS;
    k_moments<<<MOM_BLOCKS, MOM_THREADS, 0, h->stream>>>(feat, target, rows, n, nullptr, part);
    k_moments_final<<<1, 32, 0, h->stream>>>(part, n, mean);
    k_moments<<<MOM_BLOCKS, MOM_THREADS, 0, h->stream>>>(feat, target, rows, n, mean, part);
    k_moments_final<<<1, 32, 0, h->stream>>>(part, n, var);
    smart_status st = mcheck(h, cudaGetLastError(), "moments");
    if (st != SMART_OK) return st;
    double host[2 * MOM_COLS];
    st = mcheck(h, cudaMemcpyAsync(host, mean, sizeof(host), cudaMemcpyDeviceToHost, h->stream), "copy moments");
    if (st != SMART_OK) return st;
    st = mcheck(h, cudaStreamSynchronize(h->stream), "smart_mlp_fit_scaler");
    if (st != SMART_OK) return st;
    for (int c = 0; c < MOM_COLS; ++c) {
        const double sd = sqrt(host[MOM_COLS + c]);
        const double sd_ok = sd > 0.0 && std::isfinite(sd) ? sd : 1.0;
        if (c < F) {
            h->scaler[c] = host[c];
            h->scaler[4 + c] = sd_ok;
        } else {
            h->scaler[8] = host[c];
            h->scaler[9] = sd_ok;
        }
    }
    return SMART_OK;
}

extern "C" smart_status smart_mlp_gradient(smart_mlp *h, const float *feat, const float *target, const int32_t *idx,
                                           int64_t batch, float *grad_out) {
    if (!h) return SMART_E_ARG;
    smart_status st = gradient(h, feat, target, idx, batch);
    if (st != SMART_OK) return st;
    if (grad_out)
        st = mcheck(h, cudaMemcpyAsync(grad_out, h->grad, PSTRIDE * sizeof(float), cudaMemcpyDeviceToDevice, h->stream),
                    "copy gradient");
    return st;
}

extern "C" smart_status smart_mlp_train_step(smart_mlp *h, const float *feat, const float *target, const int32_t *idx,
                                             int64_t batch, float lr, float *loss_out) {
    if (!h) return SMART_E_ARG;
    if (!(lr > 0.f) || !std::isfinite(lr)) return mfail(h, SMART_E_ARG, "learning rate must be positive");
    smart_status st = gradient(h, feat, target, idx, batch);
    if (st != SMART_OK) return st;
    const double b1 = 0.9, b2 = 0.999;
    h->step += 1;
    const double bc1 = 1.0 - pow(b1, (double)h->step), bc2 = 1.0 - pow(b2, (double)h->step);
    k_mlp_adam<<<(NP + 255) / 256, 256, 0, h->stream>>>(h->theta, h->m, h->v, h->grad, h->wb, lr, (float)b1, (float)b2,
                                                        1e-8f, (float)bc1, (float)bc2, loss_out,
                                                        (float)(1.0 / (double)batch));
    return mcheck(h, cudaGetLastError(), "k_mlp_adam");
}

extern "C" smart_status smart_mlp_infer(smart_mlp *h, const float *feat, const float *map_plain, int64_t n,
                                        float *map_out, float *correction, unsigned long long *n_fallback) {
    if (!h) return SMART_E_ARG;
    if (!h->have_params) return mfail(h, SMART_E_STATE, "no parameters");
    if (n < 0 || (n > 0 && (!feat || !map_plain || !map_out))) return mfail(h, SMART_E_ARG, "bad inputs");
    if (n == 0) return SMART_OK;
    InferArgs a;
    a.feat = feat;
    a.plain = map_plain;
    a.n = n;
    a.sc = make_scaler(h);
    a.theta = h->theta;
    a.wb = h->wb;
    a.out = map_out;
    a.corr = correction;
    a.n_fallback = n_fallback;
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t ntiles = (n + S - 1) / S;
    smart_status st;
    if (h->precision == SMART_MLP_BF16) {
        const size_t smem = sizeof(SmemInf<true>);
        st = mcheck(h, cudaFuncSetAttribute(k_mlp_infer<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                    "smem attribute");
        if (st != SMART_OK) return st;
        k_mlp_infer<true><<<(unsigned)std::min<int64_t>(ntiles, (int64_t)sms * 3), NTH, smem, h->stream>>>(a);
    } else {
        const size_t smem = sizeof(SmemInf<false>);
        st = mcheck(h, cudaFuncSetAttribute(k_mlp_infer<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                    "smem attribute");
        if (st != SMART_OK) return st;
        k_mlp_infer<false><<<(unsigned)std::min<int64_t>(ntiles, (int64_t)sms * 2), NTH, smem, h->stream>>>(a);
    }
    return mcheck(h, cudaGetLastError(), "k_mlp_infer");
}

extern "C" smart_status smart_mlp_get_state(smart_mlp *h, void *buf, int64_t cap, int64_t *size) {
    if (!h) return SMART_E_ARG;
    const int64_t need = state_size();
    if (size) *size = need;
    if (!buf) return SMART_OK;
    if (cap < need) return mfail(h, SMART_E_ARG, "state buffer too small");
    if (!h->have_params) return mfail(h, SMART_E_STATE, "no parameters");
    unsigned char *p = (unsigned char *)buf;
    const uint32_t hdr[4] = {STATE_MAGIC, STATE_VERSION, (uint32_t)h->precision, (uint32_t)NP};
    memcpy(p, hdr, sizeof(hdr));
    p += sizeof(hdr);
    memcpy(p, &h->step, 8);
    p += 8;
    memcpy(p, h->scaler, sizeof(h->scaler));
    p += sizeof(h->scaler);
    float *dev[3] = {h->theta, h->m, h->v};
    for (float *d : dev) {
        smart_status st = mcheck(h, cudaMemcpyAsync(p, d, NP * sizeof(float), cudaMemcpyDeviceToHost, h->stream),
                                 "copy state");
        if (st != SMART_OK) return st;
        p += NP * sizeof(float);
    }
    return mcheck(h, cudaStreamSynchronize(h->stream), "smart_mlp_get_state");
}

extern "C" smart_status smart_mlp_set_state(smart_mlp *h, const void *buf, int64_t size) {
    if (!h) return SMART_E_ARG;
    if (!buf || size != state_size()) return mfail(h, SMART_E_ARG, "state: wrong size");
    const unsigned char *p = (const unsigned char *)buf;
    uint32_t hdr[4];
    memcpy(hdr, p, sizeof(hdr));
    if (hdr[0] != STATE_MAGIC || hdr[1] != STATE_VERSION || hdr[3] != (uint32_t)NP)
        return mfail(h, SMART_E_ARG, "state: bad header");
    if (hdr[2] != (uint32_t)h->precision) return mfail(h, SMART_E_ARG, "state: saved with another precision");
    p += sizeof(hdr);
    int64_t step;
    memcpy(&step, p, 8);
    p += 8;
    double sc[10];
    memcpy(sc, p, sizeof(sc));
    p += sizeof(sc);
    smart_status st = smart_mlp_set_scaler(h, sc);
    if (st != SMART_OK) return st;
    float *dev[3] = {h->theta, h->m, h->v};
    for (float *d : dev) {
        st = mcheck(h, cudaMemcpyAsync(d, p, NP * sizeof(float), cudaMemcpyHostToDevice, h->stream), "copy state");
        if (st != SMART_OK) return st;
        p += NP * sizeof(float);
    }
    k_mlp_copy_bf16<<<(NP + 255) / 256, 256, 0, h->stream>>>(h->theta, h->wb);
    st = mcheck(h, cudaGetLastError(), "k_mlp_copy_bf16");
    if (st != SMART_OK) return st;
    h->step = step;
    h->have_params = true;
    return mcheck(h, cudaStreamSynchronize(h->stream), "smart_mlp_set_state");
}

extern "C" int64_t smart_mlp_step(const smart_mlp *h) { return h ? h->step : -1; }

// features of the context's targets from its pixel-based map (and, for
// training, the galaxy-level map of the same targets)
extern "C" smart_status smart_mlp_features(smart_ctx *c, const smart_maps *pixel_map, const smart_maps *brute_map,
                                           float *feat, float *target, uint8_t *valid, int64_t *sum_n2) {
    if (!c) return SMART_E_ARG;
    if (!pixel_map || !feat || !pixel_map->map_e || !pixel_map->sum_w || !pixel_map->count || !pixel_map->members)
        return fail(c, SMART_E_ARG, "smart_mlp_features: pixel map needs map_e, sum_w, count and members");
    if (brute_map && (!brute_map->map_e || !brute_map->sum_w))
        return fail(c, SMART_E_ARG, "smart_mlp_features: galaxy-level map needs map_e and sum_w");
    if (target && !brute_map) return fail(c, SMART_E_ARG, "smart_mlp_features: targets need the galaxy-level map");
    FeatArgs fa{};
    smart_status st = prepare_pixel(c, pixel_map, fa.m);
    if (st != SMART_OK) return st;
    if (fa.m.n == 0) return SMART_OK;
    fa.px_e = pixel_map->map_e;
    fa.px_w = pixel_map->sum_w;
    fa.px_count = pixel_map->count;
    fa.px_members = pixel_map->members;
    fa.bf_e = brute_map ? brute_map->map_e : nullptr;
    fa.bf_w = brute_map ? brute_map->sum_w : nullptr;
    fa.feat = feat;
    fa.target = target;
    fa.valid = valid;
    fa.sum_n2 = sum_n2;
    const unsigned blocks = (unsigned)std::min<int64_t>((fa.m.n + 127) / 128, (int64_t)c->num_sms * 16);
    k_mlp_features<<<blocks, 128, 0, c->stream>>>(fa);
    return check_cuda(c, cudaGetLastError(), "k_mlp_features");
}
