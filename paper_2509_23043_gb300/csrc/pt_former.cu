// IsingFormer inference on GB300 (sm_103a): the decoder-only transformer of arXiv 2509.23043
// (Methods, "IsingFormer architecture and training"; Supplementary S6) that gives the TAPT
// proposals their law q(x | beta) and draws them. See include/pt_former.h for the model.
//
// Layout (row-major, one row per (configuration, position) for scoring, per configuration
// for a sampling step): residual stream h FP32 [M][d]; layer-norm outputs, attention outputs
// and the first FFN map (GELU applied in place) bfloat16, the inputs of the next matrix
// products; query/key/value bfloat16 [M][3d] for the tensor-core attention of the scoring
// pass, FP32 for the streaming kernel and the sampler. The matrix products run on the tensor
// cores (bfloat16 inputs, FP32 accumulation, bias, GELU or residual in the epilogue), through
// this library's tcgen05 kernels (pt_gemm_tc.cu: the first FFN map, and the whole attention of
// the scoring pass) or cuBLASLt as proj_mode and attn_mode say; the rest are the kernels
// below. Sampling keeps a key/value cache [layer][B][N][2d], bfloat16 (FP32 with the streaming
// attention, attn_mode 1).
#include <cublasLt.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/pt_former.h"
#include "pt_device.cuh"
#include "pt_gemm_tc.h"
#include "pt_softmax2.cuh"

namespace {

thread_local std::string g_ferr;

pt_status ffail(pt_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_ferr = buf;
    return s;
}

#define FCK(x)                                                                           \
    do {                                                                                 \
        cudaError_t e_ = (x);                                                            \
        if (e_ != cudaSuccess) return ffail(PT_ECUDA, "%s: %s", #x, cudaGetErrorString(e_)); \
    } while (0)
#define LCK(x)                                                                           \
    do {                                                                                 \
        cublasStatus_t s_ = (x);                                                         \
        if (s_ != CUBLAS_STATUS_SUCCESS) return ffail(PT_ECUDA, "%s: cublas status %d", #x, (int)s_); \
    } while (0)

constexpr int kDH = 64;          // head dimension
constexpr uint32_t kDomSample = 6u;

// ------------------------------------------------------------------------------ kernels
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(pt::kFull, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(pt::kFull, v, o));
    return v;
}

// h[b N + t] = tok_emb[token] + (beta_b W_beta + b_beta) + PE[t]; token = start (2) at t = 0,
// else the token of spin t - 1 (teacher forcing: the configurations scored). One warp per
// row; with y given, the row's layer norm (gain g, bias bt; the first block's, computed as
// layernorm_kernel computes it) is written to y in the same pass, so h is not read back.
template <int D>
__global__ void embed_score_kernel(const int8_t* __restrict__ spins, const float* __restrict__ beta,
                                   const float* __restrict__ tok, const float* __restrict__ wb,
                                   const float* __restrict__ bb, const float* __restrict__ pe,
                                   const float* __restrict__ g, const float* __restrict__ bt,
                                   float* __restrict__ h, __nv_bfloat16* __restrict__ y, size_t M,
                                   int N) {
    const size_t row = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= M) return;
    const int b = (int)(row / N), t = (int)(row - (size_t)b * N);
    const int k = t == 0 ? 2 : (spins[(size_t)b * N + t - 1] > 0 ? 1 : 0);
    const float be = beta[b];
    float v[D / 32];
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < D / 32; ++i) {
        const int c = lane + 32 * i;
        v[i] = tok[k * D + c] + (be * wb[c] + bb[c]) + pe[(size_t)t * D + c];
        h[row * D + c] = v[i];
        s += v[i];
    }
    if (!y) return;
    const float mu = warp_sum(s) / D;
    float q = 0.f;
#pragma unroll
    for (int i = 0; i < D / 32; ++i) {
        v[i] -= mu;
        q += v[i] * v[i];
    }
    const float rstd = rsqrtf(warp_sum(q) / D + 1e-5f);
#pragma unroll
    for (int i = 0; i < D / 32; ++i) {
        const int c = lane + 32 * i;
        y[row * D + c] = __float2bfloat16_rn(v[i] * rstd * g[c] + bt[c]);
    }
}

// one sampling step: h[b] for position t, the token of the spin drawn at t - 1
__global__ void embed_step_kernel(const int8_t* __restrict__ out, const float* __restrict__ beta,
                                  const float* __restrict__ tok, const float* __restrict__ wb,
                                  const float* __restrict__ bb, const float* __restrict__ pe,
                                  float* __restrict__ h, int N, int d, int t) {
    const int b = blockIdx.x;
    const int k = t == 0 ? 2 : (out[(size_t)b * N + t - 1] > 0 ? 1 : 0);
    const float be = beta[b];
    for (int c = threadIdx.x; c < d; c += blockDim.x)
        h[(size_t)b * d + c] = tok[k * d + c] + (be * wb[c] + bb[c]) + pe[(size_t)t * d + c];
}

// layer norm of each row (one warp per row), eps 1e-5, to bfloat16
template <int D>
__global__ void layernorm_kernel(const float* __restrict__ x, const float* __restrict__ g,
                                 const float* __restrict__ bt, __nv_bfloat16* __restrict__ y,
                                 size_t M) {
    const size_t row = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= M) return;
    const float* xr = x + row * D;
    float v[D / 32];
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < D / 32; ++i) {
        v[i] = xr[lane + 32 * i];
        s += v[i];
    }
    const float mu = warp_sum(s) / D;
    float q = 0.f;
#pragma unroll
    for (int i = 0; i < D / 32; ++i) {
        v[i] -= mu;
        q += v[i] * v[i];
    }
    const float rstd = rsqrtf(warp_sum(q) / D + 1e-5f);
#pragma unroll
    for (int i = 0; i < D / 32; ++i) {
        const int c = lane + 32 * i;
        y[row * D + c] = __float2bfloat16_rn(v[i] * rstd * g[c] + bt[c]);
    }
}

// y = GELU(y) = y (1 + erf(y / sqrt 2)) / 2 in place on bfloat16, evaluated in FP32; eight
// values (16 bytes) per access, n8 = n / 8
__device__ __forceinline__ float gelu_erf(float v) {
    return 0.5f * v * (1.f + erff(v * 0.70710678118654752f));
}
__global__ void gelu_kernel(__nv_bfloat16* __restrict__ y, size_t n8) {
    uint4* p = reinterpret_cast<uint4*>(y);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n8; i += (size_t)gridDim.x * blockDim.x) {
        uint4 w = p[i];
        __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&w);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 f = __bfloat1622float2(h[k]);
            h[k] = __floats2bfloat162_rn(gelu_erf(f.x), gelu_erf(f.y));
        }
        p[i] = w;
    }
}

// Causal multi-head attention of the scoring pass: block (query block of 128, head, b); each
// thread one query row, keys streamed through shared memory 64 at a time, softmax kept
// online (running maximum and sum). qkv FP32 [B N][3d]; out bfloat16 [B N][d].
constexpr int kAQ = 128, kAK = 64;
__global__ void __launch_bounds__(kAQ) attention_kernel(const float* __restrict__ qkv,
                                                        __nv_bfloat16* __restrict__ out, int N, int d) {
    __shared__ float Ks[kAK][kDH];
    __shared__ float Vs[kAK][kDH];
    const int hd = blockIdx.y, b = blockIdx.z;
    const int t0 = blockIdx.x * kAQ;
    const int t = t0 + threadIdx.x;
    const size_t ld = 3 * (size_t)d;
    const float* base = qkv + (size_t)b * N * ld;
    float q[kDH], acc[kDH];
    if (t < N) {
#pragma unroll
        for (int c = 0; c < kDH; ++c) {
            q[c] = base[(size_t)t * ld + hd * kDH + c] * 0.125f;      // 1 / sqrt(64)
            acc[c] = 0.f;
        }
    }
    float m = -INFINITY, l = 0.f;
    const int tmax = min(N - 1, t0 + kAQ - 1);
    for (int j0 = 0; j0 <= tmax; j0 += kAK) {
        __syncthreads();
        for (int e = threadIdx.x; e < kAK * kDH; e += kAQ) {
            const int r = e / kDH, c = e - r * kDH;
            const int j = j0 + r;
            Ks[r][c] = j < N ? base[(size_t)j * ld + d + hd * kDH + c] : 0.f;
            Vs[r][c] = j < N ? base[(size_t)j * ld + 2 * d + hd * kDH + c] : 0.f;
        }
        __syncthreads();
        if (t < N) {
            const int jn = min(kAK, t - j0 + 1);
            for (int r = 0; r < jn; ++r) {
                float s = 0.f;
#pragma unroll
                for (int c = 0; c < kDH; ++c) s = fmaf(q[c], Ks[r][c], s);
                const float mn = fmaxf(m, s);
                const float corr = expf(m - mn), p = expf(s - mn);
                l = l * corr + p;
#pragma unroll
                for (int c = 0; c < kDH; ++c) acc[c] = fmaf(p, Vs[r][c], acc[c] * corr);
                m = mn;
            }
        }
    }
    if (t < N) {
        const float inv = 1.f / l;
        __nv_bfloat16* o = out + ((size_t)b * N + t) * d + hd * kDH;
#pragma unroll
        for (int c = 0; c < kDH; ++c) o[c] = __float2bfloat16_rn(acc[c] * inv);
    }
}

// causal softmax of each score row S[bh][i][0..i] (one warp per row), to bfloat16 P with the
// masked entries j > i set to 0 (the next product reads whole rows). Even N <= 64 K2: each
// lane keeps the column pairs 2 (lane + 32 k), k < K2, in registers (one read of the row,
// 8-byte loads, 4-byte stores); causal_softmax_loop_kernel takes any N.
template <int K2>
__global__ void causal_softmax_kernel(const float* __restrict__ S, __nv_bfloat16* __restrict__ P,
                                      size_t rows, int N) {
    const size_t row = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    const int i = (int)(row % N);
    const float2* sr = reinterpret_cast<const float2*>(S + row * N);
    __nv_bfloat162* pr = reinterpret_cast<__nv_bfloat162*>(P + row * N);
    float2 v[K2];
    float mx = -INFINITY;
#pragma unroll
    for (int k = 0; k < K2; ++k) {
        const int j = 2 * (lane + 32 * k);
        v[k] = j <= i ? sr[lane + 32 * k] : make_float2(-INFINITY, -INFINITY);   // j + 1 < N: N even
        if (j + 1 > i) v[k].y = -INFINITY;
        mx = fmaxf(mx, fmaxf(v[k].x, v[k].y));
    }
    mx = warp_max(mx);
    float sum = 0.f;
#pragma unroll
    for (int k = 0; k < K2; ++k) {
        const int j = 2 * (lane + 32 * k);
        v[k].x = j <= i ? expf(v[k].x - mx) : 0.f;
        v[k].y = j + 1 <= i ? expf(v[k].y - mx) : 0.f;
        sum += v[k].x + v[k].y;
    }
    const float inv = 1.f / warp_sum(sum);
#pragma unroll
    for (int k = 0; k < K2; ++k)
        if (2 * (lane + 32 * k) < N) pr[lane + 32 * k] = __floats2bfloat162_rn(v[k].x * inv, v[k].y * inv);
}

__global__ void causal_softmax_loop_kernel(const float* __restrict__ S, __nv_bfloat16* __restrict__ P,
                                      size_t rows, int N) {
    const size_t row = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    const int i = (int)(row % N);
    const float* sr = S + row * N;
    __nv_bfloat16* pr = P + row * N;
    float mx = -INFINITY;
    for (int j = lane; j <= i; j += 32) mx = fmaxf(mx, sr[j]);
    mx = warp_max(mx);
    float sum = 0.f;
    for (int j = lane; j <= i; j += 32) sum += expf(sr[j] - mx);
    const float inv = 1.f / warp_sum(sum);
    for (int j = lane; j < N; j += 32)
        pr[j] = __float2bfloat16_rn(j <= i ? expf(sr[j] - mx) * inv : 0.f);
}

// Attention of the step-t query against the cached keys 0..t: block b, one warp per head. The
// warp first appends step t's key and value of its head to the cache. Each half-warp then takes
// one cached row at a time (64 floats of this head, 256 contiguous bytes, a float4 per lane):
// keys j = 2i + half for the scores, reduced over the half-warp's 16 lanes, then the value rows
// in the same order for the weighted sum, the two halves added at the end. kStepRows rows per
// half-warp are loaded before any is used, so every warp keeps kStepRows x 512 bytes in flight:
// the kernel streams the cache, and its rate is set by the bytes in flight per SM.
constexpr int kStepRows = 8;
__global__ void __launch_bounds__(256) attention_step_kernel(const float* __restrict__ qkv,
                                                             float* __restrict__ cache,
                                                             __nv_bfloat16* __restrict__ out,
                                                             int N, int d, int t) {
    extern __shared__ float sm[];              // per warp: the t + 1 scores, then probabilities
    const int hd = threadIdx.x >> 5, lane = threadIdx.x & 31, b = blockIdx.x;
    const int half = lane >> 4, c4 = 4 * (lane & 15);
    float* ps = sm + hd * N;
    const float* qr = qkv + (size_t)b * 3 * d + hd * kDH;
    float4 q = *reinterpret_cast<const float4*>(qr + c4);
    q.x *= 0.125f; q.y *= 0.125f; q.z *= 0.125f; q.w *= 0.125f;
    // append this step's key (lanes 0-15) and value (lanes 16-31) of head hd as row t
    float* crow = cache + ((size_t)b * N + t) * 2 * d + hd * kDH;
    *reinterpret_cast<float4*>(crow + half * d + c4) =
        *reinterpret_cast<const float4*>(qr + (1 + half) * d + c4);
    __syncwarp();
    const float* kb = cache + (size_t)b * N * 2 * d + hd * kDH + c4;
    const size_t rs = 2 * (size_t)d;           // floats between consecutive cached rows
    const int nk = t + 1;
    float mx = -INFINITY;
    for (int j0 = 0; j0 < nk; j0 += 2 * kStepRows) {
        float s[kStepRows];
#pragma unroll
        for (int u = 0; u < kStepRows; ++u) {
            const int j = j0 + 2 * u + half;
            float4 k = make_float4(0.f, 0.f, 0.f, 0.f);
            if (j < nk) k = *reinterpret_cast<const float4*>(kb + j * rs);
            s[u] = fmaf(q.x, k.x, fmaf(q.y, k.y, fmaf(q.z, k.z, q.w * k.w)));
        }
#pragma unroll
        for (int u = 0; u < kStepRows; ++u) {
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) s[u] += __shfl_xor_sync(0xffffffffu, s[u], o);
            const int j = j0 + 2 * u + half;
            if (j < nk) {
                if ((lane & 15) == 0) ps[j] = s[u];
                mx = fmaxf(mx, s[u]);
            }
        }
    }
    mx = warp_max(mx);
    __syncwarp();
    float sum = 0.f;
    for (int j = lane; j < nk; j += 32) {
        const float p = expf(ps[j] - mx);
        ps[j] = p;
        sum += p;
    }
    sum = warp_sum(sum);
    __syncwarp();
    const float* vb = kb + d;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int j0 = 0; j0 < nk; j0 += 2 * kStepRows) {
        float4 v[kStepRows];
        float p[kStepRows];
#pragma unroll
        for (int u = 0; u < kStepRows; ++u) {
            const int j = j0 + 2 * u + half;
            v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            p[u] = 0.f;
            if (j < nk) {
                v[u] = *reinterpret_cast<const float4*>(vb + j * rs);
                p[u] = ps[j];
            }
        }
#pragma unroll
        for (int u = 0; u < kStepRows; ++u) {
            acc.x = fmaf(p[u], v[u].x, acc.x);
            acc.y = fmaf(p[u], v[u].y, acc.y);
            acc.z = fmaf(p[u], v[u].z, acc.z);
            acc.w = fmaf(p[u], v[u].w, acc.w);
        }
    }
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 16);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 16);
    acc.z += __shfl_xor_sync(0xffffffffu, acc.z, 16);
    acc.w += __shfl_xor_sync(0xffffffffu, acc.w, 16);
    if (half == 0) {
        const float inv = 1.f / sum;
        __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(out + (size_t)b * d + hd * kDH + c4);
        o[0] = __floats2bfloat162_rn(acc.x * inv, acc.y * inv);
        o[1] = __floats2bfloat162_rn(acc.z * inv, acc.w * inv);
    }
}

// the exponential of the fused scoring kernel (pt_softmax2.cuh)
using ptsm::ex2_approx;
using ptsm::kLog2e8;
__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// The sampling step with a bfloat16 cache (attn_mode 0 and 2), in the arithmetic of the fused
// scoring kernel, so that the log q of a sampled configuration is the one scoring gives it:
// query, keys and values rounded to bfloat16; scores s_j = q . k_j in FP32 (unscaled);
// p_j = 2^((s_j - max) log2(e) / 8); the sum of the p_j in FP32; O = sum bf16(p_j) v_j / sum.
// Block b, one warp per head; each quarter-warp reads one cached row of its head at a time (64
// bfloat16 values, 128 contiguous bytes, 16 per lane), kStepRows16 rows per quarter in flight:
// the same bytes per load instruction as the FP32 kernel, for half the bytes per row.
constexpr int kStepRows16 = 8;
__device__ __forceinline__ void bf16x8_to_float(uint4 r, float (&f)[8]) {
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        f[2 * i] = __uint_as_float(w[i] << 16);
        f[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
    }
}
__global__ void __launch_bounds__(256) attention_step16_kernel(const float* __restrict__ qkv,
                                                               __nv_bfloat16* __restrict__ cache,
                                                               __nv_bfloat16* __restrict__ out,
                                                               int N, int d, int t) {
    extern __shared__ float sm[];              // per warp: the t + 1 scores, then bf16(p)
    const int hd = threadIdx.x >> 5, lane = threadIdx.x & 31, b = blockIdx.x;
    const int qtr = lane >> 3, c8 = 8 * (lane & 7);
    float* ps = sm + hd * N;
    const float* qr = qkv + (size_t)b * 3 * d + hd * kDH;
    float q[8];
    {
        const float4 q0 = *reinterpret_cast<const float4*>(qr + c8);
        const float4 q1 = *reinterpret_cast<const float4*>(qr + c8 + 4);
        q[0] = bf16_round(q0.x); q[1] = bf16_round(q0.y); q[2] = bf16_round(q0.z); q[3] = bf16_round(q0.w);
        q[4] = bf16_round(q1.x); q[5] = bf16_round(q1.y); q[6] = bf16_round(q1.z); q[7] = bf16_round(q1.w);
    }
    // append this step's key (lanes 0-7) and value (lanes 8-15) of head hd as row t
    __nv_bfloat16* crow = cache + ((size_t)b * N + t) * 2 * d + hd * kDH;
    if (qtr < 2) {
        const float4 a0 = *reinterpret_cast<const float4*>(qr + (1 + qtr) * d + c8);
        const float4 a1 = *reinterpret_cast<const float4*>(qr + (1 + qtr) * d + c8 + 4);
        const __nv_bfloat162 w0 = __floats2bfloat162_rn(a0.x, a0.y), w1 = __floats2bfloat162_rn(a0.z, a0.w);
        const __nv_bfloat162 w2 = __floats2bfloat162_rn(a1.x, a1.y), w3 = __floats2bfloat162_rn(a1.z, a1.w);
        *reinterpret_cast<uint4*>(crow + qtr * d + c8) =
            make_uint4(*reinterpret_cast<const uint32_t*>(&w0), *reinterpret_cast<const uint32_t*>(&w1),
                       *reinterpret_cast<const uint32_t*>(&w2), *reinterpret_cast<const uint32_t*>(&w3));
    }
    __syncwarp();
    const __nv_bfloat16* kb = cache + (size_t)b * N * 2 * d + hd * kDH + c8;
    const size_t rs = 2 * (size_t)d;           // elements between consecutive cached rows
    const int nk = t + 1;
    float mx = -INFINITY;
    for (int j0 = 0; j0 < nk; j0 += 4 * kStepRows16) {
        uint4 raw[kStepRows16];
#pragma unroll
        for (int u = 0; u < kStepRows16; ++u) {
            const int j = j0 + 4 * u + qtr;
            raw[u] = make_uint4(0u, 0u, 0u, 0u);
            if (j < nk) raw[u] = *reinterpret_cast<const uint4*>(kb + j * rs);
        }
#pragma unroll
        for (int u = 0; u < kStepRows16; ++u) {
            float k[8];
            bf16x8_to_float(raw[u], k);
            float sc = q[7] * k[7];
#pragma unroll
            for (int c = 6; c >= 0; --c) sc = fmaf(q[c], k[c], sc);
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) sc += __shfl_xor_sync(0xffffffffu, sc, o);
            const int j = j0 + 4 * u + qtr;
            if (j < nk) {
                if ((lane & 7) == 0) ps[j] = sc;
                mx = fmaxf(mx, sc);
            }
        }
    }
    mx = warp_max(mx);
    __syncwarp();
    const float off = -mx * kLog2e8;
    float sum = 0.f;
    for (int j = lane; j < nk; j += 32) {
        const float p = ex2_approx(fmaf(ps[j], kLog2e8, off));
        sum += p;
        ps[j] = bf16_round(p);
    }
    sum = warp_sum(sum);
    __syncwarp();
    const __nv_bfloat16* vb = kb + d;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int j0 = 0; j0 < nk; j0 += 4 * kStepRows16) {
        uint4 raw[kStepRows16];
        float p[kStepRows16];
#pragma unroll
        for (int u = 0; u < kStepRows16; ++u) {
            const int j = j0 + 4 * u + qtr;
            raw[u] = make_uint4(0u, 0u, 0u, 0u);
            p[u] = 0.f;
            if (j < nk) {
                raw[u] = *reinterpret_cast<const uint4*>(vb + j * rs);
                p[u] = ps[j];
            }
        }
#pragma unroll
        for (int u = 0; u < kStepRows16; ++u) {
            float v[8];
            bf16x8_to_float(raw[u], v);
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] = fmaf(p[u], v[c], acc[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], 8);
        acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], 16);
    }
    if (qtr == 0) {
        const float inv = 1.f / sum;
        const __nv_bfloat162 w0 = __floats2bfloat162_rn(acc[0] * inv, acc[1] * inv);
        const __nv_bfloat162 w1 = __floats2bfloat162_rn(acc[2] * inv, acc[3] * inv);
        const __nv_bfloat162 w2 = __floats2bfloat162_rn(acc[4] * inv, acc[5] * inv);
        const __nv_bfloat162 w3 = __floats2bfloat162_rn(acc[6] * inv, acc[7] * inv);
        *reinterpret_cast<uint4*>(out + (size_t)b * d + hd * kDH + c8) =
            make_uint4(*reinterpret_cast<const uint32_t*>(&w0), *reinterpret_cast<const uint32_t*>(&w1),
                       *reinterpret_cast<const uint32_t*>(&w2), *reinterpret_cast<const uint32_t*>(&w3));
    }
}

// final layer norm and head of one row (one warp): the two logits and their log-softmax
template <int D>
__device__ __forceinline__ void head_row(const float* xr, const float* g, const float* bt,
                                         const float* wout, const float* bout, int lane,
                                         float& l0, float& l1) {
    float v[D / 32];
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < D / 32; ++i) {
        v[i] = xr[lane + 32 * i];
        s += v[i];
    }
    const float mu = warp_sum(s) / D;
    float q = 0.f;
#pragma unroll
    for (int i = 0; i < D / 32; ++i) {
        v[i] -= mu;
        q += v[i] * v[i];
    }
    const float rstd = rsqrtf(warp_sum(q) / D + 1e-5f);
    float a0 = 0.f, a1 = 0.f;
#pragma unroll
    for (int i = 0; i < D / 32; ++i) {
        const int c = lane + 32 * i;
        const float z = v[i] * rstd * g[c] + bt[c];
        a0 = fmaf(z, wout[2 * c], a0);
        a1 = fmaf(z, wout[2 * c + 1], a1);
    }
    l0 = warp_sum(a0) + bout[0];
    l1 = warp_sum(a1) + bout[1];
}

__device__ __forceinline__ void log_softmax2(float l0, float l1, float& p0, float& p1) {
    const float m = fmaxf(l0, l1);
    const float lse = m + logf(expf(l0 - m) + expf(l1 - m));
    p0 = l0 - lse;
    p1 = l1 - lse;
}

// scoring head: per row the log-probability of the scored spin (and the logits)
template <int D>
__global__ void head_score_kernel(const float* __restrict__ h, const float* __restrict__ g,
                                  const float* __restrict__ bt, const float* __restrict__ wout,
                                  const float* __restrict__ bout, const int8_t* __restrict__ spins,
                                  float* __restrict__ lp, float* __restrict__ logits, size_t M) {
    const size_t row = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= M) return;
    float l0, l1, p0, p1;
    head_row<D>(h + row * D, g, bt, wout, bout, lane, l0, l1);
    log_softmax2(l0, l1, p0, p1);
    if (lane == 0) {
        lp[row] = spins[row] > 0 ? p1 : p0;
        if (logits) {
            logits[2 * row] = l0;
            logits[2 * row + 1] = l1;
        }
    }
}

// log q[b] = sum over positions, in position order (one warp per configuration)
__global__ void sum_rows_kernel(const float* __restrict__ lp, float* __restrict__ logq, int B, int N) {
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (b >= B) return;
    float s = 0.f;
    for (int t = lane; t < N; t += 32) s += lp[(size_t)b * N + t];
    s = warp_sum(s);
    if (lane == 0) logq[b] = s;
}

struct SampleArgs {
    uint64_t seed;
    uint32_t stream;
};

// sampling head of step t: spin t of each configuration (one warp each) drawn from its
// logits (or copied from the prefix), its log-probability added to log q
template <int D>
__global__ void head_sample_kernel(const float* __restrict__ h, const float* __restrict__ g,
                                   const float* __restrict__ bt, const float* __restrict__ wout,
                                   const float* __restrict__ bout, const int8_t* __restrict__ prefix,
                                   int npre, const SampleArgs* __restrict__ sa, int8_t* __restrict__ out,
                                   float* __restrict__ logq, int B, int N, int t) {
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (b >= B) return;
    float l0, l1, p0, p1;
    head_row<D>(h + (size_t)b * D, g, bt, wout, bout, lane, l0, l1);
    log_softmax2(l0, l1, p0, p1);
    if (lane == 0) {
        int8_t s;
        if (t < npre) {
            s = prefix[(size_t)b * npre + t] > 0 ? 1 : -1;
        } else {
            const uint64_t seed = sa->seed;
            const uint4 r = pt::philox(make_uint4((uint32_t)t, (uint32_t)b, kDomSample << 24, sa->stream),
                                       (uint32_t)seed, (uint32_t)(seed >> 32));
            const float u = (float)(r.x >> 8) * 5.9604644775390625e-08f;   // 2^-24
            s = u < expf(p1) ? 1 : -1;
        }
        out[(size_t)b * N + t] = s;
        const float add = s > 0 ? p1 : p0;
        if (logq) logq[b] = (t == 0 ? 0.f : logq[b]) + add;
    }
}

// ------------------------------------------------------------------------------ host side
float bf16_bits_to_float(uint16_t v) {
    uint32_t u = (uint32_t)v << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

struct Layer {
    float *ln1_g, *ln1_b, *b_qkv, *b_o, *ln2_g, *ln2_b, *b_2;
    __nv_bfloat16 *w_qkv, *w_o, *w_1, *w_2;
    __nv_bfloat16 *b_qkv16, *b_1;   // the biases of the products with bfloat16 output
    // the weight matrices transposed ([out][in], K-major), for the tcgen05 products
    __nv_bfloat16 *w_qkvt, *w_ot, *w_1t, *w_2t;
};

struct Act {                       // activation buffers for `rows` rows
    size_t rows = 0;
    float *h = nullptr, *qkv = nullptr, *lp = nullptr;
    __nv_bfloat16 *a = nullptr, *o = nullptr, *g = nullptr;
    // scoring attention on the tensor cores: bfloat16 query/key/value [rows][3d], scores
    // S FP32 and probabilities P bfloat16, both [B][H][N][N]
    size_t att_elems = 0;           // B H N N
    __nv_bfloat16 *qkv16 = nullptr, *P = nullptr;
    float* S = nullptr;
};

}  // namespace

struct pt_former {
    pt_former_config cfg{};
    cudaStream_t stream = nullptr;     // the caller's stream: every call is ordered on it
    cudaStream_t exec = nullptr;       // the stream the launches go to (stream, or cap in capture)
    cudaStream_t cap = nullptr;        // private stream of the sampling graph (capture, replay)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cublasLtHandle_t lt = nullptr;
    void* workspace = nullptr;
    size_t ws_bytes = 32u << 20;
    std::vector<void*> allocs;
    float *tok = nullptr, *wb = nullptr, *bb = nullptr, *pe = nullptr;
    float *lnf_g = nullptr, *lnf_b = nullptr, *wout = nullptr, *bout = nullptr;
    std::vector<Layer> layers;
    Act score, step;
    void* cache = nullptr;         // sampling: [L][B][N][2d], bfloat16 (attn_mode 0, 2) or FP32 (1)
    int cache_B = 0;
    SampleArgs* d_sargs = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::tuple<int, int, const void*, const void*, const void*, const void*> gkey{};
    std::map<std::vector<long long>, cublasLtMatmulAlgo_t> algos;   // by product shape, layout, alignment
    bool proj_tc = false;          // the tcgen05 kernels are set up (proj_mode 0 or 2)
    bool tc_ready = false;         // gemm_tc_setup succeeded
    int num_sms = 0;
    int* d_err = nullptr;          // nonzero once a wait of a tcgen05 kernel ran out
};

namespace {

template <class T>
pt_status dalloc(pt_former* m, T** p, size_t n) {
    void* q = nullptr;
    FCK(cudaMalloc(&q, n * sizeof(T) + 16));
    m->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return PT_OK;
}

pt_status upload_f32(pt_former* m, float** dst, const uint16_t* src, size_t n) {
    std::vector<float> h(n);
    for (size_t i = 0; i < n; ++i) h[i] = bf16_bits_to_float(src[i]);
    pt_status s = dalloc(m, dst, n);
    if (s != PT_OK) return s;
    FCK(cudaMemcpy(*dst, h.data(), n * 4, cudaMemcpyHostToDevice));
    return PT_OK;
}

pt_status upload_bf16(pt_former* m, __nv_bfloat16** dst, const uint16_t* src, size_t n) {
    pt_status s = dalloc(m, dst, n);
    if (s != PT_OK) return s;
    FCK(cudaMemcpy(*dst, src, n * 2, cudaMemcpyHostToDevice));
    return PT_OK;
}

// a row-major [rows][cols] bfloat16 matrix, uploaded transposed ([cols][rows])
pt_status upload_transposed(pt_former* m, __nv_bfloat16** dst, const uint16_t* src, int rows, int cols) {
    std::vector<uint16_t> t((size_t)rows * cols);
    for (int r = 0; r < rows; ++r)
        for (int c = 0; c < cols; ++c) t[(size_t)c * rows + r] = src[(size_t)r * cols + c];
    return upload_bf16(m, dst, t.data(), t.size());
}

void free_act(Act& a) {
    cudaFree(a.h); cudaFree(a.qkv); cudaFree(a.lp);
    cudaFree(a.a); cudaFree(a.o); cudaFree(a.g);
    cudaFree(a.qkv16); cudaFree(a.P); cudaFree(a.S);
    a = Act{};
}

// the unfused tensor-core path keeps one layer's FP32 scores and bfloat16 probabilities (B H N^2
// entries of 6 bytes) when they fit this budget; else the streaming attention kernel runs (the
// fused kernel keeps neither)
constexpr size_t kAttScratchBytes = size_t(2) << 30;

// the scores, the causal softmax and P V in one tcgen05 kernel (no score or probability buffer)
bool attn_fused(const pt_former* m) {
    return m->cfg.attn_mode == 0 && m->tc_ready && attn_tc_supported(m->cfg.n_spins, m->cfg.d_model);
}

pt_status ensure_att(pt_former* m, Act& a, int B) {
    const size_t N = m->cfg.n_spins, H = m->cfg.n_heads, d = m->cfg.d_model;
    const size_t elems = (size_t)B * H * N * N;
    if (a.att_elems >= elems) return PT_OK;
    cudaFree(a.qkv16); cudaFree(a.P); cudaFree(a.S);
    a.qkv16 = a.P = nullptr;
    a.S = nullptr;
    a.att_elems = 0;
    const size_t rows = (size_t)B * N;
    FCK(cudaMalloc(&a.qkv16, rows * 3 * d * 2));
    if (!attn_fused(m)) {
        FCK(cudaMalloc(&a.S, elems * 4));
        FCK(cudaMalloc(&a.P, elems * 2));
    }
    a.att_elems = elems;
    return PT_OK;
}

pt_status ensure_act(pt_former* m, Act& a, size_t rows) {
    if (a.rows >= rows) return PT_OK;
    free_act(a);
    const size_t d = m->cfg.d_model, F = m->cfg.d_ff;
    FCK(cudaMalloc(&a.h, rows * d * 4));
    FCK(cudaMalloc(&a.qkv, rows * 3 * d * 4));
    FCK(cudaMalloc(&a.lp, rows * 4));
    FCK(cudaMalloc(&a.a, rows * d * 2));
    FCK(cudaMalloc(&a.o, rows * d * 2));
    FCK(cudaMalloc(&a.g, rows * F * 2));
    a.rows = rows;
    return PT_OK;
}

// largest power of two (<= 256) dividing every byte offset given: the alignment cuBLASLt may
// assume for a matrix (its base pointer, leading dimension and batch stride in bytes)
long long alignment(std::initializer_list<unsigned long long> bytes) {
    unsigned long long a = 256;
    for (unsigned long long v : bytes)
        while (a > 1 && v % a) a >>= 1;
    return (long long)a;
}

// the algorithm cuBLASLt's heuristic picks for one product description, chosen once per
// key (shape, layouts, output type, alignments) and kept
pt_status pick_algo(pt_former* m, const std::vector<long long>& key, cublasLtMatmulDesc_t op,
                    cublasLtMatrixLayout_t la, cublasLtMatrixLayout_t lb, cublasLtMatrixLayout_t lc,
                    const long long al[3], const cublasLtMatmulAlgo_t** algo) {
    auto it = m->algos.find(key);
    if (it == m->algos.end()) {
        cublasLtMatmulPreference_t pref = nullptr;
        LCK(cublasLtMatmulPreferenceCreate(&pref));
        LCK(cublasLtMatmulPreferenceSetAttribute(pref, CUBLASLT_MATMUL_PREF_MAX_WORKSPACE_BYTES,
                                                 &m->ws_bytes, sizeof m->ws_bytes));
        const uint32_t a0 = (uint32_t)al[0], a1 = (uint32_t)al[1], a2 = (uint32_t)al[2];
        LCK(cublasLtMatmulPreferenceSetAttribute(pref, CUBLASLT_MATMUL_PREF_MIN_ALIGNMENT_A_BYTES, &a0, sizeof a0));
        LCK(cublasLtMatmulPreferenceSetAttribute(pref, CUBLASLT_MATMUL_PREF_MIN_ALIGNMENT_B_BYTES, &a1, sizeof a1));
        LCK(cublasLtMatmulPreferenceSetAttribute(pref, CUBLASLT_MATMUL_PREF_MIN_ALIGNMENT_C_BYTES, &a2, sizeof a2));
        LCK(cublasLtMatmulPreferenceSetAttribute(pref, CUBLASLT_MATMUL_PREF_MIN_ALIGNMENT_D_BYTES, &a2, sizeof a2));
        cublasLtMatmulHeuristicResult_t res{};
        int got = 0;
        const cublasStatus_t st = cublasLtMatmulAlgoGetHeuristic(m->lt, op, la, lb, lc, lc, pref, 1, &res, &got);
        cublasLtMatmulPreferenceDestroy(pref);
        if (st != CUBLAS_STATUS_SUCCESS || got < 1)
            return ffail(PT_ENOTSUP, "no cuBLASLt algorithm for the product %lld x %lld x %lld", key[1], key[2], key[3]);
        it = m->algos.emplace(key, res.algo).first;
    }
    *algo = &it->second;
    return PT_OK;
}

// Y [rows][n] = X [rows][k] (bf16) W [k][n] (bf16) + bias [n] (+ Y when residual), Y FP32
// (bias FP32) or bfloat16 (yt = CUDA_R_16BF, bias bfloat16): column-major Y^T = W^T X^T,
// with W^T as the [n x k] column-major view of row-major W.
pt_status gemm(pt_former* m, void* Y, cudaDataType_t yt, const __nv_bfloat16* X,
               const __nv_bfloat16* W, const void* bias, size_t rows, int n, int k, bool residual) {
    cublasLtMatmulDesc_t op = nullptr;
    cublasLtMatrixLayout_t la = nullptr, lb = nullptr, lc = nullptr;
    const size_t ys = yt == CUDA_R_32F ? 4 : 2;
    LCK(cublasLtMatmulDescCreate(&op, CUBLAS_COMPUTE_32F, CUDA_R_32F));
    const cublasOperation_t nt = CUBLAS_OP_N;
    LCK(cublasLtMatmulDescSetAttribute(op, CUBLASLT_MATMUL_DESC_TRANSA, &nt, sizeof nt));
    LCK(cublasLtMatmulDescSetAttribute(op, CUBLASLT_MATMUL_DESC_TRANSB, &nt, sizeof nt));
    const cublasLtEpilogue_t ep = CUBLASLT_EPILOGUE_BIAS;
    LCK(cublasLtMatmulDescSetAttribute(op, CUBLASLT_MATMUL_DESC_EPILOGUE, &ep, sizeof ep));
    LCK(cublasLtMatmulDescSetAttribute(op, CUBLASLT_MATMUL_DESC_BIAS_POINTER, &bias, sizeof bias));
    LCK(cublasLtMatmulDescSetAttribute(op, CUBLASLT_MATMUL_DESC_BIAS_DATA_TYPE, &yt, sizeof yt));
    LCK(cublasLtMatrixLayoutCreate(&la, CUDA_R_16BF, n, k, n));
    LCK(cublasLtMatrixLayoutCreate(&lb, CUDA_R_16BF, k, (uint64_t)rows, k));
    LCK(cublasLtMatrixLayoutCreate(&lc, yt, n, (uint64_t)rows, n));
    const long long al[3] = {alignment({(unsigned long long)W, 2ull * n}),
                             alignment({(unsigned long long)X, 2ull * k}),
                             alignment({(unsigned long long)Y, ys * n})};
    const std::vector<long long> key = {0, (long long)rows, n, k, residual ? 1 : 0, (long long)yt,
                                        al[0], al[1], al[2]};
    const cublasLtMatmulAlgo_t* algo = nullptr;
    pt_status s = pick_algo(m, key, op, la, lb, lc, al, &algo);
    cublasStatus_t st = CUBLAS_STATUS_SUCCESS;
    if (s == PT_OK) {
        const float one = 1.f, beta = residual ? 1.f : 0.f;
        st = cublasLtMatmul(m->lt, op, &one, W, la, X, lb, &beta, Y, lc, Y, lc, algo, m->workspace,
                            m->ws_bytes, m->exec);
    }
    cublasLtMatrixLayoutDestroy(la);
    cublasLtMatrixLayoutDestroy(lb);
    cublasLtMatrixLayoutDestroy(lc);
    cublasLtMatmulDescDestroy(op);
    if (s != PT_OK) return s;
    if (st != CUBLAS_STATUS_SUCCESS) return ffail(PT_ECUDA, "cublasLtMatmul: status %d", (int)st);
    return PT_OK;
}

// Strided-batched product on the tensor cores, column-major views: C [m][n] (type ct, leading
// dimension ldc, batch stride sc) = alpha op(A) [m][k] op(B) [k][n], bfloat16 operands, FP32
// accumulation, no epilogue.
pt_status gemm_batched(pt_former* m, cublasOperation_t ta, const __nv_bfloat16* A, int lda, long long sa,
                       const __nv_bfloat16* Bm, int ldb, long long sb, void* C, cudaDataType_t ct, int ldc,
                       long long sc, int mm, int nn, int kk, int batch, float alpha) {
    cublasLtMatmulDesc_t op = nullptr;
    cublasLtMatrixLayout_t la = nullptr, lb = nullptr, lc = nullptr;
    const unsigned long long cs = ct == CUDA_R_32F ? 4 : 2;
    LCK(cublasLtMatmulDescCreate(&op, CUBLAS_COMPUTE_32F, CUDA_R_32F));
    const cublasOperation_t nt = CUBLAS_OP_N;
    LCK(cublasLtMatmulDescSetAttribute(op, CUBLASLT_MATMUL_DESC_TRANSA, &ta, sizeof ta));
    LCK(cublasLtMatmulDescSetAttribute(op, CUBLASLT_MATMUL_DESC_TRANSB, &nt, sizeof nt));
    const int arows = ta == CUBLAS_OP_N ? mm : kk, acols = ta == CUBLAS_OP_N ? kk : mm;
    LCK(cublasLtMatrixLayoutCreate(&la, CUDA_R_16BF, arows, acols, lda));
    LCK(cublasLtMatrixLayoutCreate(&lb, CUDA_R_16BF, kk, nn, ldb));
    LCK(cublasLtMatrixLayoutCreate(&lc, ct, mm, nn, ldc));
    for (auto [l, st] : {std::make_pair(la, sa), std::make_pair(lb, sb), std::make_pair(lc, sc)}) {
        LCK(cublasLtMatrixLayoutSetAttribute(l, CUBLASLT_MATRIX_LAYOUT_BATCH_COUNT, &batch, sizeof batch));
        LCK(cublasLtMatrixLayoutSetAttribute(l, CUBLASLT_MATRIX_LAYOUT_STRIDED_BATCH_OFFSET, &st, sizeof st));
    }
    const long long al[3] = {alignment({(unsigned long long)A, 2ull * lda, 2ull * sa}),
                             alignment({(unsigned long long)Bm, 2ull * ldb, 2ull * sb}),
                             alignment({(unsigned long long)C, cs * ldc, cs * sc})};
    const std::vector<long long> key = {1, mm, nn, kk, batch, (long long)ta, lda, sa, ldb, sb, ldc, sc,
                                        (long long)ct, al[0], al[1], al[2]};
    const cublasLtMatmulAlgo_t* algo = nullptr;
    pt_status s = pick_algo(m, key, op, la, lb, lc, al, &algo);
    cublasStatus_t st = CUBLAS_STATUS_SUCCESS;
    if (s == PT_OK) {
        const float zero = 0.f;
        st = cublasLtMatmul(m->lt, op, &alpha, A, la, Bm, lb, &zero, C, lc, C, lc, algo, m->workspace,
                            m->ws_bytes, m->exec);
    }
    cublasLtMatrixLayoutDestroy(la);
    cublasLtMatrixLayoutDestroy(lb);
    cublasLtMatrixLayoutDestroy(lc);
    cublasLtMatmulDescDestroy(op);
    if (s != PT_OK) return s;
    if (st != CUBLAS_STATUS_SUCCESS) return ffail(PT_ECUDA, "batched cublasLtMatmul: status %d", (int)st);
    return PT_OK;
}

pt_status attention_scores_softmax(pt_former* m, Act& x, int B);

// Causal attention of the scoring pass on the tensor cores, reading the heads' columns of the
// bfloat16 [B N][3d] query/key/value in place and writing the head's columns of the [B N][d]
// output. attn_mode 0 with N <= 256: one tcgen05 kernel (scores, softmax and P V on the SM).
// Otherwise per head, batched over the B configurations on cuBLASLt: S = Q K^T / 8 (row-major
// S [N][N] is the column-major S^T = K Q^T), the causal softmax kernel, then O = P V
// (O^T = V^T P^T).
pt_status attention_tc(pt_former* m, Act& x, int B) {
    const int N = m->cfg.n_spins, d = m->cfg.d_model, H = m->cfg.n_heads;
    const int ld = 3 * d;
    const long long cfg_stride = (long long)N * ld;     // one configuration's rows
    const long long nn = (long long)N * N;
    pt_status s = PT_OK;
    if (attn_fused(m)) {
        // scores, causal softmax and P V in one tcgen05 kernel, O written directly
        FCK(attn_tc(x.qkv16, x.o, B, N, H, d, m->num_sms, m->d_err, m->exec));
        return PT_OK;
    }
    s = attention_scores_softmax(m, x, B);
    if (s != PT_OK) return s;
    for (int hd = 0; hd < H && s == PT_OK; ++hd)
        s = gemm_batched(m, CUBLAS_OP_N, x.qkv16 + 2 * d + hd * kDH, ld, cfg_stride, x.P + hd * nn, N, H * nn,
                         x.o + hd * kDH, CUDA_R_16BF, d, (long long)N * d, kDH, N, N, B, 1.f);
    return s;
}

// S = Q K^T / 8 per head as cuBLASLt batched products (FP32), then the causal-softmax kernel
pt_status attention_scores_softmax(pt_former* m, Act& x, int B) {
    const int N = m->cfg.n_spins, d = m->cfg.d_model, H = m->cfg.n_heads;
    const int ld = 3 * d;
    const long long cfg_stride = (long long)N * ld;
    const long long nn = (long long)N * N;
    pt_status s = PT_OK;
    for (int hd = 0; hd < H && s == PT_OK; ++hd)
        s = gemm_batched(m, CUBLAS_OP_T, x.qkv16 + d + hd * kDH, ld, cfg_stride, x.qkv16 + hd * kDH, ld,
                         cfg_stride, x.S + hd * nn, CUDA_R_32F, N, H * nn, N, N, kDH, B, 0.125f);
    if (s != PT_OK) return s;
    const size_t rows = (size_t)B * H * N;
    const unsigned grid = (unsigned)((rows + 7) / 8);
    if (N % 2 == 0 && N <= 64)
        causal_softmax_kernel<1><<<grid, 256, 0, m->exec>>>(x.S, x.P, rows, N);
    else if (N % 2 == 0 && N <= 128)
        causal_softmax_kernel<2><<<grid, 256, 0, m->exec>>>(x.S, x.P, rows, N);
    else if (N % 2 == 0 && N <= 256)
        causal_softmax_kernel<4><<<grid, 256, 0, m->exec>>>(x.S, x.P, rows, N);
    else if (N % 2 == 0 && N <= 512)
        causal_softmax_kernel<8><<<grid, 256, 0, m->exec>>>(x.S, x.P, rows, N);
    else
        causal_softmax_loop_kernel<<<grid, 256, 0, m->exec>>>(x.S, x.P, rows, N);
    FCK(cudaGetLastError());
    return s;
}

template <int D>
void launch_layernorm(const float* x, const float* g, const float* b, __nv_bfloat16* y, size_t M,
                      cudaStream_t s) {
    layernorm_kernel<D><<<(unsigned)((M + 7) / 8), 256, 0, s>>>(x, g, b, y, M);
}

pt_status layernorm(pt_former* m, const float* x, const float* g, const float* b, __nv_bfloat16* y,
                    size_t M) {
    switch (m->cfg.d_model) {
        case 64: launch_layernorm<64>(x, g, b, y, M, m->exec); break;
        case 128: launch_layernorm<128>(x, g, b, y, M, m->exec); break;
        case 256: launch_layernorm<256>(x, g, b, y, M, m->exec); break;
        case 512: launch_layernorm<512>(x, g, b, y, M, m->exec); break;
        default: return ffail(PT_ENOTSUP, "d_model %d", m->cfg.d_model);
    }
    FCK(cudaGetLastError());
    return PT_OK;
}

template <int D>
void launch_head_score(pt_former* m, const float* h, const int8_t* spins, float* lp, float* logits, size_t M) {
    head_score_kernel<D><<<(unsigned)((M + 7) / 8), 256, 0, m->exec>>>(h, m->lnf_g, m->lnf_b, m->wout,
                                                                         m->bout, spins, lp, logits, M);
}
template <int D>
void launch_head_sample(pt_former* m, const int8_t* prefix, int npre, int8_t* out, float* logq, int B, int t) {
    head_sample_kernel<D><<<(B + 7) / 8, 256, 0, m->exec>>>(m->step.h, m->lnf_g, m->lnf_b, m->wout, m->bout,
                                                              prefix, npre, m->d_sargs, out, logq, B,
                                                              m->cfg.n_spins, t);
}

// rows from which proj_mode 0 takes the first FFN map to the tcgen05 kernel: 128 tiles of
// 128 rows, enough to keep the persistent grid busy (sampling steps, one row per
// configuration, stay on cuBLASLt)
constexpr size_t kTcMinRows = 16384;

// one pre-layer-norm block on rows [0, M) of `a` (attention by `attn`; query/key/value to
// the bfloat16 buffer when qkv_bf16, the operand layout of the tensor-core attention). The
// products run on this library's tcgen05 kernels (bias, GELU and residual in their
// epilogues) or on cuBLASLt as proj_mode says (include/pt_former.h). ln1_done: the block's first
// layer norm is already in x.a (written with the embedding).
template <class AttnFn>
pt_status block(pt_former* m, Act& x, size_t M, const Layer& Ly, bool qkv_bf16, bool ln1_done,
                AttnFn attn) {
    const int d = m->cfg.d_model, F = m->cfg.d_ff;
    const bool tc = m->cfg.proj_mode == 2;                        // every suitable projection
    const bool tc_ffn1 = tc || (m->cfg.proj_mode == 0 && M >= kTcMinRows);
    auto tc_gemm = [&](int epi, const __nv_bfloat16* A, const __nv_bfloat16* Wt, const void* b, void* C, int n,
                       int k) -> pt_status {
        FCK(gemm_tc(epi, A, Wt, b, C, (int)M, n, k, m->num_sms, m->d_err, m->exec));
        return PT_OK;
    };
    pt_status s = ln1_done ? PT_OK : layernorm(m, x.h, Ly.ln1_g, Ly.ln1_b, x.a, M);
    if (s == PT_OK) {
        if (qkv_bf16 && tc && gemm_tc_supported(3 * d, d))
            s = tc_gemm(kEpiBias, x.a, Ly.w_qkvt, Ly.b_qkv16, x.qkv16, 3 * d, d);
        else if (qkv_bf16)
            s = gemm(m, x.qkv16, CUDA_R_16BF, x.a, Ly.w_qkv, Ly.b_qkv16, M, 3 * d, d, false);
        else
            s = gemm(m, x.qkv, CUDA_R_32F, x.a, Ly.w_qkv, Ly.b_qkv, M, 3 * d, d, false);
    }
    if (s == PT_OK) s = attn();
    if (s == PT_OK)
        s = tc && gemm_tc_supported(d, d) ? tc_gemm(kEpiResid, x.o, Ly.w_ot, Ly.b_o, x.h, d, d)
                                          : gemm(m, x.h, CUDA_R_32F, x.o, Ly.w_o, Ly.b_o, M, d, d, true);
    if (s == PT_OK) s = layernorm(m, x.h, Ly.ln2_g, Ly.ln2_b, x.a, M);
    if (s == PT_OK && tc_ffn1 && gemm_tc_supported(F, d)) {
        s = tc_gemm(kEpiGelu, x.a, Ly.w_1t, Ly.b_1, x.g, F, d);
    } else if (s == PT_OK) {
        s = gemm(m, x.g, CUDA_R_16BF, x.a, Ly.w_1, Ly.b_1, M, F, d, false);
        if (s == PT_OK) {
            const size_t n8 = M * (size_t)F / 8;       // F is a multiple of 8
            gelu_kernel<<<(unsigned)std::min<size_t>((n8 + 255) / 256, 152 * 16), 256, 0, m->exec>>>(x.g, n8);
            FCK(cudaGetLastError());
        }
    }
    if (s == PT_OK)
        s = tc && gemm_tc_supported(d, F) ? tc_gemm(kEpiResid, x.g, Ly.w_2t, Ly.b_2, x.h, d, F)
                                          : gemm(m, x.h, CUDA_R_32F, x.g, Ly.w_2, Ly.b_2, M, d, F, true);
    return s;
}

// the sampler's key/value cache: bfloat16 unless the scoring attention is the FP32 streaming
// kernel (attn_mode 1), so that sampler and scorer share their arithmetic
bool cache16(const pt_former* m) { return m->cfg.attn_mode != 1; }

pt_status sample_launches(pt_former* m, int B, const float* beta, const int8_t* prefix, int npre,
                          int8_t* out, float* logq) {
    const int N = m->cfg.n_spins, d = m->cfg.d_model, H = m->cfg.n_heads;
    const size_t smem = (size_t)H * N * 4;
    for (int t = 0; t < N; ++t) {
        embed_step_kernel<<<B, 256, 0, m->exec>>>(out, beta, m->tok, m->wb, m->bb, m->pe, m->step.h, N, d, t);
        FCK(cudaGetLastError());
        for (int l = 0; l < m->cfg.n_layers; ++l) {
            const size_t off = (size_t)l * B * N * 2 * d;       // elements
            pt_status s = block(m, m->step, (size_t)B, m->layers[l], false, false, [&]() -> pt_status {
                if (cache16(m))
                    attention_step16_kernel<<<B, 32 * H, smem, m->exec>>>(
                        m->step.qkv, static_cast<__nv_bfloat16*>(m->cache) + off, m->step.o, N, d, t);
                else
                    attention_step_kernel<<<B, 32 * H, smem, m->exec>>>(
                        m->step.qkv, static_cast<float*>(m->cache) + off, m->step.o, N, d, t);
                FCK(cudaGetLastError());
                return PT_OK;
            });
            if (s != PT_OK) return s;
        }
        switch (d) {
            case 64: launch_head_sample<64>(m, prefix, npre, out, logq, B, t); break;
            case 128: launch_head_sample<128>(m, prefix, npre, out, logq, B, t); break;
            case 256: launch_head_sample<256>(m, prefix, npre, out, logq, B, t); break;
            case 512: launch_head_sample<512>(m, prefix, npre, out, logq, B, t); break;
        }
        FCK(cudaGetLastError());
    }
    return PT_OK;
}

}  // namespace

extern "C" {

const char* pt_former_last_error(void) { return g_ferr.c_str(); }

size_t pt_former_param_count(const pt_former_config* c) {
    if (!c) return 0;
    const size_t d = c->d_model, F = c->d_ff;
    const size_t per = 2 * d + 3 * d * d + 3 * d + d * d + d + 2 * d + d * F + F + F * d + d;
    return 3 * d + 2 * d + (size_t)c->n_layers * per + 2 * d + 2 * d + 2;
}

pt_status pt_former_create(pt_former** out, const pt_former_config* cfg, const uint16_t* params,
                           size_t n_params, void* cuda_stream) {
    if (!out || !cfg || !params) return ffail(PT_EINVAL, "NULL argument");
    *out = nullptr;
    const int d = cfg->d_model, F = cfg->d_ff;
    if (cfg->n_spins < 1 || cfg->n_layers < 0 || cfg->n_heads < 1 || d != 64 * cfg->n_heads ||
        (d != 64 && d != 128 && d != 256 && d != 512) || F < 8 || F % 8 != 0 ||
        cfg->attn_mode < 0 || cfg->attn_mode > 2 || cfg->proj_mode < 0 || cfg->proj_mode > 2)
        return ffail(PT_EINVAL, "unsupported shape (d_model must be 64 x n_heads, one of 64..512; d_ff a multiple of 8)");
    if (n_params != pt_former_param_count(cfg))
        return ffail(PT_EINVAL, "%zu parameters given, the shape has %zu", n_params, pt_former_param_count(cfg));
    pt_former* m = new pt_former();
    m->cfg = *cfg;
    m->stream = (cudaStream_t)cuda_stream;
    m->exec = m->stream;
    pt_status s = PT_OK;
    if (cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->ev_out, cudaEventDisableTiming) != cudaSuccess)
        s = ffail(PT_ECUDA, "stream or event creation");
    const uint16_t* p = params;
    auto take = [&](size_t n) { const uint16_t* q = p; p += n; return q; };
    if (cublasLtCreate(&m->lt) != CUBLAS_STATUS_SUCCESS) s = ffail(PT_ECUDA, "cublasLtCreate");
    if (s == PT_OK && cudaMalloc(&m->workspace, m->ws_bytes) != cudaSuccess) s = ffail(PT_ENOMEM, "workspace");
    if (s == PT_OK) s = upload_f32(m, &m->tok, take(3 * (size_t)d), 3 * (size_t)d);
    if (s == PT_OK) s = upload_f32(m, &m->wb, take(d), d);
    if (s == PT_OK) s = upload_f32(m, &m->bb, take(d), d);
    m->layers.resize(cfg->n_layers);
    for (int l = 0; l < cfg->n_layers && s == PT_OK; ++l) {
        Layer& L = m->layers[l];
        s = upload_f32(m, &L.ln1_g, take(d), d);
        if (s == PT_OK) s = upload_f32(m, &L.ln1_b, take(d), d);
        const uint16_t* wq = take(3 * (size_t)d * d);
        if (s == PT_OK) s = upload_bf16(m, &L.w_qkv, wq, 3 * (size_t)d * d);
        if (s == PT_OK) s = upload_transposed(m, &L.w_qkvt, wq, d, 3 * d);
        const uint16_t* bq = take(3 * (size_t)d);
        if (s == PT_OK) s = upload_f32(m, &L.b_qkv, bq, 3 * (size_t)d);
        if (s == PT_OK) s = upload_bf16(m, &L.b_qkv16, bq, 3 * (size_t)d);
        const uint16_t* wo = take((size_t)d * d);
        if (s == PT_OK) s = upload_bf16(m, &L.w_o, wo, (size_t)d * d);
        if (s == PT_OK) s = upload_transposed(m, &L.w_ot, wo, d, d);
        if (s == PT_OK) s = upload_f32(m, &L.b_o, take(d), d);
        if (s == PT_OK) s = upload_f32(m, &L.ln2_g, take(d), d);
        if (s == PT_OK) s = upload_f32(m, &L.ln2_b, take(d), d);
        const uint16_t* w1 = take((size_t)d * F);
        if (s == PT_OK) s = upload_bf16(m, &L.w_1, w1, (size_t)d * F);
        if (s == PT_OK) s = upload_transposed(m, &L.w_1t, w1, d, F);
        if (s == PT_OK) s = upload_bf16(m, &L.b_1, take(F), F);
        const uint16_t* w2 = take((size_t)F * d);
        if (s == PT_OK) s = upload_bf16(m, &L.w_2, w2, (size_t)F * d);
        if (s == PT_OK) s = upload_transposed(m, &L.w_2t, w2, F, d);
        if (s == PT_OK) s = upload_f32(m, &L.b_2, take(d), d);
    }
    if (s == PT_OK) s = upload_f32(m, &m->lnf_g, take(d), d);
    if (s == PT_OK) s = upload_f32(m, &m->lnf_b, take(d), d);
    if (s == PT_OK) s = upload_f32(m, &m->wout, take(2 * (size_t)d), 2 * (size_t)d);
    if (s == PT_OK) s = upload_f32(m, &m->bout, take(2), 2);
    if (s == PT_OK) {
        // positional code PE[t, 2i] = sin(t / 10000^(2i/d)), PE[t, 2i+1] = cos(...), in FP64
        const int N = cfg->n_spins;
        std::vector<float> pe((size_t)N * d);
        for (int t = 0; t < N; ++t)
            for (int i = 0; i < d / 2; ++i) {
                const double ang = t / std::pow(10000.0, 2.0 * i / d);
                pe[(size_t)t * d + 2 * i] = (float)std::sin(ang);
                pe[(size_t)t * d + 2 * i + 1] = (float)std::cos(ang);
            }
        s = dalloc(m, &m->pe, pe.size());
        if (s == PT_OK && cudaMemcpy(m->pe, pe.data(), pe.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
            s = ffail(PT_ECUDA, "positional code upload");
    }
    if (s == PT_OK) s = dalloc(m, &m->d_sargs, 1);
    if (s == PT_OK) s = dalloc(m, &m->d_err, 1);
    if (s == PT_OK && cudaMemset(m->d_err, 0, sizeof(int)) != cudaSuccess) s = ffail(PT_ECUDA, "error flag");
    m->proj_tc = cfg->proj_mode != 1;
    if (s == PT_OK && (m->proj_tc || cfg->attn_mode == 0)) {
        int dev = 0;
        const cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, dev);
        const cudaError_t e2 = e == cudaSuccess ? gemm_tc_setup() : e;
        if (e2 != cudaSuccess || m->num_sms < 1)
            s = ffail(PT_ECUDA, "tcgen05 product set-up: %s", cudaGetErrorString(e2));
        else
            m->tc_ready = true;
    }
    if (s != PT_OK) {
        pt_former_destroy(m);
        return s;
    }
    *out = m;
    return PT_OK;
}

pt_status pt_former_score(pt_former* m, int32_t B, const int8_t* spins, const float* beta,
                          float* logq, float* logits) {
    if (!m || !spins || !beta || !logq) return ffail(PT_EINVAL, "NULL argument");
    if (B < 1) return ffail(PT_EINVAL, "B must be >= 1");
    const int N = m->cfg.n_spins, d = m->cfg.d_model, H = m->cfg.n_heads;
    const size_t M = (size_t)B * N;
    pt_status s = ensure_act(m, m->score, M);
    if (s != PT_OK) return s;
    Act& x = m->score;
    // the embedding, with the first block's layer norm in the same pass
    const bool ln1_fused = m->cfg.n_layers > 0;
    const float* g0 = ln1_fused ? m->layers[0].ln1_g : nullptr;
    const float* b0 = ln1_fused ? m->layers[0].ln1_b : nullptr;
    __nv_bfloat16* y0 = ln1_fused ? x.a : nullptr;
    const unsigned eg = (unsigned)((M + 7) / 8);
    switch (d) {
        case 64: embed_score_kernel<64><<<eg, 256, 0, m->exec>>>(spins, beta, m->tok, m->wb, m->bb, m->pe, g0, b0, x.h, y0, M, N); break;
        case 128: embed_score_kernel<128><<<eg, 256, 0, m->exec>>>(spins, beta, m->tok, m->wb, m->bb, m->pe, g0, b0, x.h, y0, M, N); break;
        case 256: embed_score_kernel<256><<<eg, 256, 0, m->exec>>>(spins, beta, m->tok, m->wb, m->bb, m->pe, g0, b0, x.h, y0, M, N); break;
        case 512: embed_score_kernel<512><<<eg, 256, 0, m->exec>>>(spins, beta, m->tok, m->wb, m->bb, m->pe, g0, b0, x.h, y0, M, N); break;
    }
    FCK(cudaGetLastError());
    // the probabilities (2 bytes per entry), and the FP32 scores unless fused (4 more)
    const bool tc = m->cfg.attn_mode != 1 && (attn_fused(m) || (size_t)B * H * N * N * 6 <= kAttScratchBytes);
    if (tc) {
        s = ensure_att(m, x, B);
        if (s != PT_OK) return s;
    }
    for (int l = 0; l < m->cfg.n_layers && s == PT_OK; ++l) {
        s = block(m, x, M, m->layers[l], tc, l == 0 && ln1_fused, [&]() -> pt_status {
            if (tc) return attention_tc(m, x, B);
            attention_kernel<<<dim3((N + kAQ - 1) / kAQ, H, B), kAQ, 0, m->exec>>>(x.qkv, x.o, N, d);
            FCK(cudaGetLastError());
            return PT_OK;
        });
    }
    if (s != PT_OK) return s;
    switch (d) {
        case 64: launch_head_score<64>(m, x.h, spins, x.lp, logits, M); break;
        case 128: launch_head_score<128>(m, x.h, spins, x.lp, logits, M); break;
        case 256: launch_head_score<256>(m, x.h, spins, x.lp, logits, M); break;
        case 512: launch_head_score<512>(m, x.h, spins, x.lp, logits, M); break;
    }
    FCK(cudaGetLastError());
    sum_rows_kernel<<<(B + 7) / 8, 256, 0, m->exec>>>(x.lp, logq, B, N);
    FCK(cudaGetLastError());
    return PT_OK;
}

pt_status pt_former_sample(pt_former* m, int32_t B, const float* beta, const int8_t* prefix,
                           int32_t n_prefix, uint64_t seed, uint32_t stream_id, int8_t* out,
                           float* logq) {
    if (!m || !beta || !out) return ffail(PT_EINVAL, "NULL argument");
    const int N = m->cfg.n_spins, d = m->cfg.d_model, H = m->cfg.n_heads;
    if (B < 1) return ffail(PT_EINVAL, "B must be >= 1");
    if (n_prefix < 0 || n_prefix > N || (n_prefix > 0 && !prefix))
        return ffail(PT_EINVAL, "n_prefix must be in [0, N], with a prefix array when > 0");
    if ((size_t)H * N * 4 > 48 * 1024)
        return ffail(PT_ENOTSUP, "sampling keeps per-head scores of N = %d positions in shared memory; N too large", N);
    pt_status s = ensure_act(m, m->step, (size_t)B);
    if (s != PT_OK) return s;
    if (m->cache_B < B) {
        if (m->cache) cudaFree(m->cache);
        m->cache = nullptr;
        m->cache_B = 0;
        FCK(cudaMalloc(&m->cache, (size_t)std::max(m->cfg.n_layers, 1) * B * N * 2 * d * (cache16(m) ? 2 : 4)));
        m->cache_B = B;
        if (m->gexec) { cudaGraphExecDestroy(m->gexec); m->gexec = nullptr; }
    }
    const SampleArgs sa{seed, stream_id};
    FCK(cudaMemcpyAsync(m->d_sargs, &sa, sizeof sa, cudaMemcpyHostToDevice, m->stream));
    const auto key = std::make_tuple((int)B, (int)n_prefix, (const void*)beta, (const void*)prefix,
                                     (const void*)out, (const void*)logq);
    if (!m->gexec || m->gkey != key) {
        if (m->gexec) { cudaGraphExecDestroy(m->gexec); m->gexec = nullptr; }
        // the first call of each shape launches directly (which also finds the cuBLASLt
        // algorithms), then captures the same launches on the private stream for later calls
        s = sample_launches(m, B, beta, prefix, n_prefix, out, logq);
        if (s != PT_OK) return s;
        cudaGraph_t g = nullptr;
        m->exec = m->cap;
        cudaError_t e = cudaStreamBeginCapture(m->cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            s = sample_launches(m, B, beta, prefix, n_prefix, out, logq);
            e = cudaStreamEndCapture(m->cap, &g);
        }
        m->exec = m->stream;
        if (s != PT_OK) { if (g) cudaGraphDestroy(g); return s; }
        if (e != cudaSuccess) return ffail(PT_ECUDA, "capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&m->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return ffail(PT_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
        m->gkey = key;
        return PT_OK;            // this call's sample came from the direct launches
    }
    // replay on the private stream, ordered after and before the caller's stream
    FCK(cudaEventRecord(m->ev_in, m->stream));
    FCK(cudaStreamWaitEvent(m->cap, m->ev_in, 0));
    FCK(cudaGraphLaunch(m->gexec, m->cap));
    FCK(cudaEventRecord(m->ev_out, m->cap));
    FCK(cudaStreamWaitEvent(m->stream, m->ev_out, 0));
    return PT_OK;
}

double pt_former_score_gemm_flops(const pt_former* m, int32_t B) {
    if (!m) return 0.0;
    const double M = (double)B * m->cfg.n_spins, d = m->cfg.d_model, F = m->cfg.d_ff;
    return m->cfg.n_layers * 2.0 * M * (d * 3 * d + d * d + d * F + F * d);
}

pt_status pt_former_check(pt_former* m) {
    if (!m) return ffail(PT_EINVAL, "NULL argument");
    FCK(cudaStreamSynchronize(m->stream));
    int e = 0;
    FCK(cudaMemcpy(&e, m->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e != 0) return ffail(PT_ECUDA, "tcgen05 product kernel: a wait ran out (code %d)", e);
    return PT_OK;
}

pt_status pt_former_destroy(pt_former* m) {
    if (!m) return PT_OK;
    if (m->stream) cudaStreamSynchronize(m->stream);
    else cudaDeviceSynchronize();
    if (m->gexec) cudaGraphExecDestroy(m->gexec);
    free_act(m->score);
    free_act(m->step);
    if (m->cache) cudaFree(m->cache);
    for (void* p : m->allocs) cudaFree(p);
    if (m->workspace) cudaFree(m->workspace);
    if (m->lt) cublasLtDestroy(m->lt);
    if (m->cap) { cudaStreamSynchronize(m->cap); cudaStreamDestroy(m->cap); }
    if (m->ev_in) cudaEventDestroy(m->ev_in);
    if (m->ev_out) cudaEventDestroy(m->ev_out);
    delete m;
    return PT_OK;
}

}  // extern "C"
