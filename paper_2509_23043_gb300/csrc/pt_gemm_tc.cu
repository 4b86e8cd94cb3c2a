// Hand-written Blackwell (sm_103a) tcgen05 kernels of the IsingFormer's blocks (Methods,
// "IsingFormer architecture and training"): the fused causal attention of the scoring pass
// (attn_tc_kernel, described where it is defined) and the projections' matrix products with
// fused epilogues:
//
//     kEpiGelu:  C[M][N] = GELU(A[M][K] W[K][N] + b[N])   bfloat16 C and b (first FFN map),
//                GELU(x) = x (1 + erf(x / sqrt 2)) / 2 (erf to 1.5e-7, see gelu_erf2);
//     kEpiBias:  C[M][N] = A W + b                         bfloat16 C and b (query/key/value);
//     kEpiResid: C[M][N] += A W + b                        FP32 C and b (output map and second
//                                                          FFN map into the residual stream).
//
// A and W bfloat16, the products accumulated in FP32 on the tensor cores. W is given
// transposed, Wt[N][K], so both operands are K-major.
//
// Design (one persistent CTA per SM, 576 threads):
//   - warp 0, one thread: TMA producer. Per output tile (128 x 256) and per K block of 64 it
//     loads A [128 x 64] and Wt [256 x 64] into a three-stage shared-memory ring, 128-byte
//     swizzled (cp.async.bulk.tensor, completion counted on the stage's mbarrier);
//   - warp 1: allocates 512 TMEM columns (two FP32 accumulators of 128 lanes x 256 columns);
//     one thread issues tcgen05.mma (kind::f16, M 128, N 256, K 16), four per K block, and
//     commits each stage back to the producer and each finished accumulator to the epilogue;
//   - warps 2..17: the epilogue. Warp w reads TMEM lanes 32 (w mod 4) .. + 31 (rows of the
//     tile) and one quarter of the columns with tcgen05.ld, 32 columns at a time, applies the
//     epilogue in FP32, and passes the results through a 2.5 KB staging buffer of its own in
//     shared memory, so that four lanes write each row's 64 contiguous bytes. With two
//     accumulators the epilogue of one tile overlaps the products of the next.
// Every wait is bounded (2 s of %globaltimer): on a timeout the kernel records a code in
// *err, every role leaves its loop, the producer waits (bounded) for its own copies in
// flight, the MMA thread for its own products, and TMEM is released before the CTA exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "pt_gemm_tc.h"
#include "pt_softmax2.cuh"

namespace tcg {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 3, NUM_ACC = 2;
constexpr int A_BYTES = BM * BK * 2;            // 16 KB
constexpr int B_BYTES = BN * BK * 2;            // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int EPI_WARPS = 16;
constexpr int STG_PITCH = 80;                   // staging row pitch: 64 bytes + 16 of padding
constexpr int STG_BYTES = 32 * STG_PITCH;       // per epilogue warp
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr int TMEM_COLS = NUM_ACC * BN;         // 512
// barriers: full[STAGES], empty[STAGES], tfull[NUM_ACC], tempty[NUM_ACC], done; then the TMEM
// base address and the abort flag
constexpr int BAR_BYTES = 8 * (2 * STAGES + 2 * NUM_ACC + 1) + 8;
constexpr size_t SMEM_BYTES = 1024 + (size_t)STAGES * STAGE_BYTES + BAR_BYTES + (size_t)EPI_WARPS * STG_BYTES;
constexpr unsigned long long WAIT_NS = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void bar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of `bar` with this parity to complete; false if the CTA is aborting or
// the wait ran out (then the CTA aborts, with `code` in *err).
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                         int* err, int code) {
    const unsigned long long t0 = now_ns();
    while (!bar_try(bar, parity)) {
        if (*abort_flag) return false;
        if (now_ns() - t0 > WAIT_NS) {
            *abort_flag = 1;
            atomicCAS(err, 0, code);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major, 128-byte-swizzled bfloat16 tile whose rows
// are 128 bytes (64 elements) and whose 8-row groups are 1024 bytes apart: start address / 16
// (bits 0-13), leading byte offset 16 / 16 (unused by this layout), stride byte offset
// 1024 / 16 (bits 32-45), the fixed 0b001 at bits 46-48, swizzle mode 2 (128 B) at bits 61-63.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and B bfloat16
// (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N / 8 at bits 17-22, M / 16 at bits
// 24-28.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 32 consecutive FP32 columns of the calling warp's 32 TMEM lanes (one lane per thread)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
          "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
          "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Paired FP32 arithmetic (sm_100 and later): one instruction applies an IEEE operation to both
// halves of a 64-bit register pair, each half rounded as the scalar operation rounds it.
__device__ __forceinline__ uint64_t f2(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ uint64_t dup(float c) { return f2(c, c); }
__device__ __forceinline__ void split2(uint64_t v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
constexpr uint64_t kNeg2 = 0x8000000080000000ull;     // both sign bits

// GELU(x) = x (1 + erf(x / sqrt 2)) / 2 of two values, with erf from Abramowitz and Stegun,
// Handbook of Mathematical Functions, formula 7.1.26: for a >= 0,
//     erf(a) = 1 - (a1 t + a2 t^2 + a3 t^3 + a4 t^4 + a5 t^5) exp(-a^2) + eps,  t = 1 / (1 + p a),
//     |eps| <= 1.5e-7,
// with the handbook's p and a1..a5, and erf(-a) = -erf(a). Per value a reciprocal, five
// multiply-adds and an exponential, fewer instructions than erff in an epilogue that is bound
// by issue, with an error far below the bfloat16 rounding of the result (2^-9 relative); the
// multiply-adds run paired, two values per instruction.
__device__ __forceinline__ void gelu_erf2(float& x0, float& x1) {
    const uint64_t a = mul2(f2(fabsf(x0), fabsf(x1)), dup(0.70710678118654752f));
    float d0, d1, a0, a1;
    split2(fma2(dup(0.3275911f), a, dup(1.f)), d0, d1);
    const uint64_t t = f2(__fdividef(1.f, d0), __fdividef(1.f, d1));
    uint64_t poly = fma2(dup(1.061405429f), t, dup(-1.453152027f));
    poly = fma2(poly, t, dup(1.421413741f));
    poly = fma2(poly, t, dup(-0.284496736f));
    poly = fma2(poly, t, dup(0.254829592f));
    poly = mul2(poly, t);
    split2(a, a0, a1);
    float e0, e1;                                                // erf(a) = 1 - poly exp(-a^2)
    split2(fma2(poly ^ kNeg2, f2(__expf(-a0 * a0), __expf(-a1 * a1)), dup(1.f)), e0, e1);
    split2(mul2(mul2(dup(0.5f), f2(x0, x1)), add2(dup(1.f), f2(copysignf(e0, x0), copysignf(e1, x1)))), x0,
           x1);
}

template <int EPI>
__global__ void __launch_bounds__(THREADS, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const void* __restrict__ bias, void* __restrict__ Cv, int M, int N, int K,
                   int* __restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    // 1024-byte alignment of the stage ring (the 128-byte swizzle repeats every 1024 bytes)
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t ring = (raw + 1023u) & ~1023u;
    uint8_t* ring_ptr = smem_raw + (ring - raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(ring_ptr + (size_t)STAGES * STAGE_BYTES);
    const uint32_t bar0 = smem_u32(bars);
    auto full = [&](int s) { return bar0 + 8u * s; };
    auto empty = [&](int s) { return bar0 + 8u * (STAGES + s); };
    auto tfull = [&](int a) { return bar0 + 8u * (2 * STAGES + a); };
    auto tempty = [&](int a) { return bar0 + 8u * (2 * STAGES + NUM_ACC + a); };
    const uint32_t done = bar0 + 8u * (2 * STAGES + 2 * NUM_ACC);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 2 * NUM_ACC + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    uint8_t* staging = ring_ptr + (size_t)STAGES * STAGE_BYTES + BAR_BYTES;
    auto sA = [&](int s) { return ring + (uint32_t)s * STAGE_BYTES; };
    auto sB = [&](int s) { return ring + (uint32_t)s * STAGE_BYTES + A_BYTES; };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m_tiles = (M + BM - 1) / BM, n_tiles = N / BN, tiles = m_tiles * n_tiles;
    const int kblocks = K / BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            bar_init(full(s), 1);
            bar_init(empty(s), 1);
        }
        for (int a = 0; a < NUM_ACC; ++a) {
            bar_init(tfull(a), 1);
            bar_init(tempty(a), 32 * EPI_WARPS);
        }
        bar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // producer; armed: stages loaded but not yet seen released (waited for on abort)
            int stage = 0;
            uint32_t phase = 0, armed = 0, armed_par = 0;
            bool ok = true;
            for (int t = blockIdx.x; ok && t < tiles; t += gridDim.x) {
                const int m0 = (t / n_tiles) * BM, n0 = (t % n_tiles) * BN;
                for (int kb = 0; kb < kblocks; ++kb) {
                    if (!bar_wait(empty(stage), phase ^ 1u, abort_flag, err, 1)) { ok = false; break; }
                    // the stage's previous load has been consumed; arm it again
                    bar_expect_tx(full(stage), STAGE_BYTES);
                    tma_load_2d(sA(stage), &tmA, kb * BK, m0, full(stage));
                    tma_load_2d(sB(stage), &tmB, kb * BK, n0, full(stage));
                    armed |= 1u << stage;
                    armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
                    if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                }
            }
            if (!ok) {
                // let the copies in flight land before the CTA's shared memory goes away (a
                // stage whose load was consumed has completed its phase already)
                for (int s = 0; s < STAGES; ++s)
                    if (armed >> s & 1u) {
                        const unsigned long long t0 = now_ns();
                        while (!bar_try(full(s), armed_par >> s & 1u) && now_ns() - t0 < WAIT_NS) {}
                    }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int stage = 0, acc = 0;
            uint32_t phase = 0, acc_phase = 0;
            bool ok = true;
            for (int t = blockIdx.x; ok && t < tiles; t += gridDim.x) {
                if (!bar_wait(tempty(acc), acc_phase ^ 1u, abort_flag, err, 2)) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(acc * BN);
                for (int kb = 0; kb < kblocks; ++kb) {
                    if (!bar_wait(full(stage), phase, abort_flag, err, 3)) { ok = false; break; }
                    tc_fence_after();
                    const uint64_t ad = sw128_desc(sA(stage)), bd = sw128_desc(sB(stage));
#pragma unroll
                    for (int k = 0; k < BK / 16; ++k)      // K step of 16 = 32 bytes = 2 in the descriptor
                        mma_f16(d, ad + 2u * k, bd + 2u * k, (kb | k) != 0 ? 1u : 0u);
                    mma_commit(empty(stage));
                    if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                mma_commit(tfull(acc));
                if (++acc == NUM_ACC) { acc = 0; acc_phase ^= 1u; }
            }
            // every product issued so far has finished before TMEM is released
            mma_commit(done);
            const unsigned long long t0 = now_ns();
            while (!bar_try(done, 0) && now_ns() - t0 < WAIT_NS) {}
        }
    } else {
        const int q = warp & 3;                   // TMEM lane quarter of this warp
        const int cq = (warp - 2) >> 2;           // column quarter of the tile
        uint8_t* stg = staging + (size_t)(warp - 2) * STG_BYTES;
        const int rr = lane >> 2, part = lane & 3; // staged read-back: row rr + 8 it, 16-byte part
        int acc = 0;
        uint32_t acc_phase = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
            // the warp leaves together: tcgen05.ld below is warp-collective
            const bool ok = bar_wait(tfull(acc), acc_phase, abort_flag, err, 4);
            if (!__all_sync(0xFFFFFFFFu, ok)) break;
            tc_fence_after();
            const int m0 = (t / n_tiles) * BM, n0 = (t % n_tiles) * BN;
            const int row0 = m0 + 32 * q;         // the warp's first row
#pragma unroll 1
            for (int ch = 0; ch < BN / 4 / 32; ++ch) {
                const int c0 = cq * (BN / 4) + ch * 32;
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * BN + c0), v);
                if (EPI == kEpiResid) {
                    // two halves of 16 columns (64 bytes of FP32 per row): stage A W + b,
                    // then four lanes per row add it to the residual row segment
                    const float* bf = static_cast<const float*>(bias) + n0 + c0;
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float4 bb = *reinterpret_cast<const float4*>(bf + 16 * hh + 4 * i);
                            float4 o;
                            o.x = __uint_as_float(v[16 * hh + 4 * i]) + bb.x;
                            o.y = __uint_as_float(v[16 * hh + 4 * i + 1]) + bb.y;
                            o.z = __uint_as_float(v[16 * hh + 4 * i + 2]) + bb.z;
                            o.w = __uint_as_float(v[16 * hh + 4 * i + 3]) + bb.w;
                            *reinterpret_cast<float4*>(stg + lane * STG_PITCH + 16 * i) = o;
                        }
                        __syncwarp();
#pragma unroll
                        for (int it = 0; it < 4; ++it) {
                            const int r = rr + 8 * it, row = row0 + r;
                            if (row < M) {
                                const float4 o = *reinterpret_cast<const float4*>(stg + r * STG_PITCH + 16 * part);
                                float4* dst = reinterpret_cast<float4*>(static_cast<float*>(Cv) + (size_t)row * N +
                                                                        n0 + c0 + 16 * hh + 4 * part);
                                float4 h = *dst;
                                h.x += o.x;
                                h.y += o.y;
                                h.z += o.z;
                                h.w += o.w;
                                *dst = h;
                            }
                        }
                        __syncwarp();
                    }
                } else {
                    const __nv_bfloat162* b2 =
                        reinterpret_cast<const __nv_bfloat162*>(static_cast<const __nv_bfloat16*>(bias) + n0 + c0);
                    uint32_t ow[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const float2 bb = __bfloat1622float2(b2[i]);
                        float x0, x1;
                        split2(add2(f2(__uint_as_float(v[2 * i]), __uint_as_float(v[2 * i + 1])), f2(bb.x, bb.y)),
                               x0, x1);
                        if (EPI == kEpiGelu) gelu_erf2(x0, x1);
                        const __nv_bfloat162 r = __floats2bfloat162_rn(x0, x1);
                        ow[i] = *reinterpret_cast<const uint32_t*>(&r);
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        *reinterpret_cast<uint4*>(stg + lane * STG_PITCH + 16 * i) =
                            make_uint4(ow[4 * i], ow[4 * i + 1], ow[4 * i + 2], ow[4 * i + 3]);
                    __syncwarp();
#pragma unroll
                    for (int it = 0; it < 4; ++it) {
                        const int r = rr + 8 * it, row = row0 + r;
                        if (row < M)
                            *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(Cv) + (size_t)row * N + n0 + c0 +
                                                      8 * part) =
                                *reinterpret_cast<const uint4*>(stg + r * STG_PITCH + 16 * part);
                    }
                    __syncwarp();
                }
            }
            tc_fence_before();
            bar_arrive(tempty(acc));
            if (++acc == NUM_ACC) { acc = 0; acc_phase ^= 1u; }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    }
}

using ptsm::ex2_approx;
using ptsm::kLog2e8;

// Causal attention of the scoring pass for sequences of at most 256 positions, all of it on
// the SM: O[b N + i][64 h ..] = sum_{j <= i} softmax_j(Q_i . K_j / 8) V_j for every configuration
// b and head h, Q, K and V read in place from the bfloat16 [B N][3d] QKV buffer (head h at
// columns 64 h, d + 64 h and 2d + 64 h; head dimension 64), O bfloat16 [B N][d]. One tile per
// (b, h, block of 128 queries):
//   - warp 0, one thread: TMA loads the 128 query rows and the configuration's 256 key and 256
//     value rows (rows past its N belong to the next configuration or are zero fill past the
//     buffer: they fall outside every query's causal range) into one of two stages;
//   - warp 1, one thread: S = Q K^T (one tcgen05.mma group, K 64, N 256) into the tile's TMEM
//     accumulator, so the whole score row of each query is in TMEM; later O = P V (M 128,
//     N 64, K the keys rounded up to 16) into the first 64 columns of the same accumulator,
//     with P from shared memory (K-major) and V from the stage as loaded (rows of 64 values:
//     MN-major, the instruction's transposed-B form). S of the next tile is issued before P V
//     of this one, so the products of one tile overlap the softmax of the other;
//   - warps 2..9: two groups of four, one per accumulator, taking alternate tiles; a thread owns
//     a row. Pass 1 reads its 256 columns 32 at a time and keeps the running maximum and sum of
//     exp; pass 2 writes exp(s - max) (unnormalised, at most 1) in bfloat16 into the 64 KB P
//     buffer in the 128-byte-swizzled K-major layout the tensor core reads (one buffer, used by
//     the tiles in turn); then O / sum is read from TMEM and written out.
// Each exponential is 2^((s - max) log2(e) / 8): one multiply-add and one ex2 per score (the
// base-2 softmax of FlashAttention-2, Dao 2023). Every wait is bounded as in the products above.
constexpr int ATT_EPI_WARPS = 8;
constexpr int ATT_THREADS = 64 + 32 * ATT_EPI_WARPS;
constexpr int ATT_STAGES = 2;
constexpr int ATT_Q_BYTES = BM * 64 * 2;                      // 16 KB
constexpr int ATT_KV_BYTES = BN * 64 * 2;                     // 32 KB each
constexpr int ATT_STAGE_BYTES = ATT_Q_BYTES + 2 * ATT_KV_BYTES;
constexpr int ATT_P_BYTES = BM * BN * 2;                      // 64 KB: four 16 KB chunks of 64 keys
// barriers: full, empty, sfull, ofull, tempty (one per stage or accumulator), pfull, pempty, done;
// then the TMEM base address and the abort flag
constexpr int ATT_NBAR = 5 * 2 + 3;
constexpr int ATT_BAR_BYTES = 8 * ATT_NBAR + 8;
constexpr size_t ATT_SMEM_BYTES = 1024 + (size_t)ATT_STAGES * ATT_STAGE_BYTES + ATT_P_BYTES + ATT_BAR_BYTES;
static_assert(ATT_SMEM_BYTES <= 232448, "over the opt-in shared memory of a block");

// Instruction descriptor of P V: FP32 accumulator, bfloat16 A and B, A K-major, B MN-major
// (bit 16), N = 64, M = 128.
constexpr uint32_t IDESC_PV = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) | ((uint32_t)(64 >> 3) << 17) |
                              ((uint32_t)(BM >> 4) << 24);

// Descriptor of an MN-major, 128-byte-swizzled bfloat16 tile of one 64-element atom along MN
// (rows of 128 bytes, one per K index, as TMA writes them): 8-row K groups 1024 bytes apart.
// The stride between MN atoms is not used at N = 64; both byte offsets are set to 1024.
__device__ __forceinline__ uint64_t sw128_mn_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(1024 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void mma_f16_pv(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(IDESC_PV), "r"(accumulate)
        : "memory");
}

__global__ void __launch_bounds__(ATT_THREADS, 1)
    attn_tc_kernel(const __grid_constant__ CUtensorMap tmQ, const __grid_constant__ CUtensorMap tmK,
                   __nv_bfloat16* __restrict__ O, int B, int N, int H, int d, int* __restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t ring = (raw + 1023u) & ~1023u;
    uint8_t* ring_ptr = smem_raw + (ring - raw);
    const uint32_t pbuf = ring + (uint32_t)ATT_STAGES * ATT_STAGE_BYTES;          // 1024-aligned
    uint8_t* pbuf_ptr = ring_ptr + (size_t)ATT_STAGES * ATT_STAGE_BYTES;
    uint64_t* bars = reinterpret_cast<uint64_t*>(pbuf_ptr + ATT_P_BYTES);
    const uint32_t bar0 = smem_u32(bars);
    auto full = [&](int s) { return bar0 + 8u * s; };
    auto empty = [&](int s) { return bar0 + 8u * (2 + s); };
    auto sfull = [&](int a) { return bar0 + 8u * (4 + a); };
    auto ofull = [&](int a) { return bar0 + 8u * (6 + a); };
    auto tempty = [&](int a) { return bar0 + 8u * (8 + a); };
    const uint32_t pfull = bar0 + 8u * 10, pempty = bar0 + 8u * 11, done = bar0 + 8u * 12;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + ATT_NBAR);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    auto sQ = [&](int s) { return ring + (uint32_t)s * ATT_STAGE_BYTES; };
    auto sK = [&](int s) { return ring + (uint32_t)s * ATT_STAGE_BYTES + ATT_Q_BYTES; };
    auto sV = [&](int s) { return ring + (uint32_t)s * ATT_STAGE_BYTES + ATT_Q_BYTES + ATT_KV_BYTES; };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m_tiles = (N + BM - 1) / BM;
    const int tiles = B * H * m_tiles;
    const int kp16 = (N + 15) >> 4;                   // K16 steps of P V

    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            bar_init(full(s), 1);
            bar_init(empty(s), 1);
            bar_init(sfull(s), 1);
            bar_init(ofull(s), 1);
            bar_init(tempty(s), 32 * ATT_EPI_WARPS / 2);   // one group per accumulator
        }
        bar_init(pfull, 32 * ATT_EPI_WARPS / 2);           // the writing group
        bar_init(pempty, 1);
        bar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t armed = 0, armed_par = 0;
            for (int u = 0;; ++u) {
                const int t = blockIdx.x + u * gridDim.x;
                if (t >= tiles) break;
                const int s = u & 1;
                const uint32_t ph = (uint32_t)(u >> 1) & 1u;
                const int bh = t / m_tiles, mt = t - bh * m_tiles;
                const int b = bh / H, h = bh - b * H;
                if (!bar_wait(empty(s), ph ^ 1u, abort_flag, err, 21)) {
                    for (int k = 0; k < 2; ++k)
                        if (armed >> k & 1u) {
                            const unsigned long long t0 = now_ns();
                            while (!bar_try(full(k), armed_par >> k & 1u) && now_ns() - t0 < WAIT_NS) {}
                        }
                    break;
                }
                bar_expect_tx(full(s), ATT_STAGE_BYTES);
                tma_load_2d(sQ(s), &tmQ, h * 64, b * N + mt * BM, full(s));          // 128 queries
                tma_load_2d(sK(s), &tmK, d + h * 64, b * N, full(s));                // 256 keys
                tma_load_2d(sV(s), &tmK, 2 * d + h * 64, b * N, full(s));            // 256 values
                armed |= 1u << s;
                armed_par = (armed_par & ~(1u << s)) | (ph << s);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int n = 0;                                     // this block's tiles
            while (blockIdx.x + n * gridDim.x < tiles) ++n;
            // S of tile u into accumulator u & 1, once the tile's stage is loaded and the
            // accumulator's previous tile has been read out
            auto issue_s = [&](int u) -> bool {
                const int a = u & 1;
                const uint32_t ph = (uint32_t)(u >> 1) & 1u;
                if (!bar_wait(tempty(a), ph ^ 1u, abort_flag, err, 22)) return false;
                tc_fence_after();
                if (!bar_wait(full(a), ph, abort_flag, err, 23)) return false;
                tc_fence_after();
                const uint64_t qd = sw128_desc(sQ(a)), kd = sw128_desc(sK(a));
#pragma unroll
                for (int k = 0; k < 4; ++k) mma_f16(tmem + (uint32_t)(a * BN), qd + 2u * k, kd + 2u * k, k != 0 ? 1u : 0u);
                mma_commit(sfull(a));
                return true;
            };
            // P V of tile u once its P is in the buffer; then the stage, the P buffer and the
            // result are released
            auto issue_pv = [&](int u) -> bool {
                const int a = u & 1;
                if (!bar_wait(pfull, (uint32_t)u & 1u, abort_flag, err, 24)) return false;
                tc_fence_after();
                for (int k = 0; k < kp16; ++k) {
                    const uint64_t pd = sw128_desc(pbuf + (uint32_t)(k >> 2) * (BM * 128)) + 2u * (uint32_t)(k & 3);
                    const uint64_t vd = sw128_mn_desc(sV(a) + (uint32_t)k * 2048u);
                    mma_f16_pv(tmem + (uint32_t)(a * BN), pd, vd, k != 0 ? 1u : 0u);
                }
                mma_commit(empty(a));
                mma_commit(pempty);
                mma_commit(ofull(a));
                return true;
            };
            bool ok = n == 0 || issue_s(0);
            for (int u = 0; ok && u < n; ++u) {
                if (u + 1 < n) ok = issue_s(u + 1);
                if (ok) ok = issue_pv(u);
            }
            mma_commit(done);
            const unsigned long long t0 = now_ns();
            while (!bar_try(done, 0) && now_ns() - t0 < WAIT_NS) {}
        }
    } else {
        const int q = warp & 3;                   // TMEM lane quarter: rows 32 q .. 32 q + 31
        const int grp = (warp - 2) >> 2;          // accumulator (and tile parity) of this group
        const int row = 32 * q + lane;            // the thread's row of the tile
        const uint32_t tbase = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(grp * BN);
        uint8_t* prow = pbuf_ptr + (size_t)row * 128;
        const int nchp = (kp16 * 16 + 31) / 32;   // chunks of 32 keys that P V reads
        for (int u = grp;; u += 2) {
            const int t = blockIdx.x + u * gridDim.x;
            if (t >= tiles) break;
            const uint32_t ph = (uint32_t)(u >> 1) & 1u;
            // a group's four warps leave together only through these waits: every one of them
            // sees the same phase complete, or every one runs out of time or sees the abort
            if (!__all_sync(0xFFFFFFFFu, bar_wait(sfull(grp), ph, abort_flag, err, 25))) break;
            tc_fence_after();
            const int bh = t / m_tiles, mt = t - bh * m_tiles;
            const int b = bh / H, h = bh - b * H;
            const int i = mt * BM + row;                   // query position
            const int jmax = min(i, N - 1);                // keys 0 .. jmax
            // the warp's last key (its last row's): tcgen05.ld is warp-collective, so every
            // lane runs the same chunks and masks its own keys
            const int jwarp = min(mt * BM + 32 * q + 31, N - 1);
            // pass 1: running maximum (of the raw scores: the scale 1/8 is positive) and sum
            float mx = -INFINITY, sum = 0.f;
#pragma unroll 1
            for (int ch = 0; ch * 32 <= jwarp; ++ch) {
                uint32_t v[32];
                tmem_ld32(tbase + (uint32_t)(32 * ch), v);
                const bool whole = 32 * ch + 31 <= jmax;
                float cm = -INFINITY;
                if (whole) {
#pragma unroll
                    for (int c = 0; c < 32; ++c) cm = fmaxf(cm, __uint_as_float(v[c]));
                } else {
#pragma unroll
                    for (int c = 0; c < 32; ++c)
                        if (32 * ch + c <= jmax) cm = fmaxf(cm, __uint_as_float(v[c]));
                }
                const float nm = fmaxf(mx, cm);
                const float off = -nm * kLog2e8;
                float cs0 = 0.f, cs1 = 0.f;
                if (whole) {
#pragma unroll
                    for (int c = 0; c < 32; c += 2) {
                        cs0 += ex2_approx(fmaf(__uint_as_float(v[c]), kLog2e8, off));
                        cs1 += ex2_approx(fmaf(__uint_as_float(v[c + 1]), kLog2e8, off));
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < 32; ++c)
                        if (32 * ch + c <= jmax) cs0 += ex2_approx(fmaf(__uint_as_float(v[c]), kLog2e8, off));
                }
                sum = sum * ex2_approx((mx - nm) * kLog2e8) + (cs0 + cs1);
                mx = nm;
            }
            const float off = -mx * kLog2e8;
            // the P buffer is free once P V of the previous tile has read it
            if (u > 0 && !__all_sync(0xFFFFFFFFu, bar_wait(pempty, (uint32_t)(u - 1) & 1u, abort_flag, err, 26)))
                break;
            // pass 2: exp(s - max) in bfloat16 into the P buffer (row `row`, keys in chunks of 64:
            // 16-byte unit k of a 128-byte row stored at unit k ^ (row & 7)); zeros past jmax
#pragma unroll 1
            for (int ch = 0; ch < nchp; ++ch) {
                uint32_t v[32];
                tmem_ld32(tbase + (uint32_t)(32 * ch), v);
                const bool whole = 32 * ch + 31 <= jmax;
                uint32_t w[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int c = 2 * e;
                    float p0 = ex2_approx(fmaf(__uint_as_float(v[c]), kLog2e8, off));
                    float p1 = ex2_approx(fmaf(__uint_as_float(v[c + 1]), kLog2e8, off));
                    if (!whole) {
                        p0 = 32 * ch + c <= jmax ? p0 : 0.f;
                        p1 = 32 * ch + c + 1 <= jmax ? p1 : 0.f;
                    }
                    const __nv_bfloat162 r2 = __floats2bfloat162_rn(p0, p1);
                    w[e] = *reinterpret_cast<const uint32_t*>(&r2);
                }
                uint8_t* cbase = prow + (size_t)(ch >> 1) * (BM * 128);
#pragma unroll
                for (int k4 = 0; k4 < 4; ++k4) {
                    const int unit = ((ch & 1) * 4 + k4) ^ (row & 7);
                    *reinterpret_cast<uint4*>(cbase + 16 * unit) =
                        make_uint4(w[4 * k4], w[4 * k4 + 1], w[4 * k4 + 2], w[4 * k4 + 3]);
                }
            }
            // the generic-proxy stores become visible to the tensor core, and the score reads
            // are complete before P V overwrites the accumulator
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc_fence_before();
            bar_arrive(pfull);
            if (!__all_sync(0xFFFFFFFFu, bar_wait(ofull(grp), ph, abort_flag, err, 27))) break;
            tc_fence_after();
            const float inv = 1.f / sum;
            __nv_bfloat16* orow = O + ((size_t)b * N + i) * d + h * 64;
#pragma unroll 1
            for (int hc = 0; hc < 2; ++hc) {
                uint32_t v[32];
                tmem_ld32(tbase + (uint32_t)(32 * hc), v);
                uint32_t w[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const __nv_bfloat162 r2 = __floats2bfloat162_rn(__uint_as_float(v[2 * e]) * inv,
                                                                    __uint_as_float(v[2 * e + 1]) * inv);
                    w[e] = *reinterpret_cast<const uint32_t*>(&r2);
                }
                if (i < N) {
                    uint4* dst = reinterpret_cast<uint4*>(orow + 32 * hc);
#pragma unroll
                    for (int k4 = 0; k4 < 4; ++k4)
                        dst[k4] = make_uint4(w[4 * k4], w[4 * k4 + 1], w[4 * k4 + 2], w[4 * k4 + 3]);
                }
            }
            tc_fence_before();
            bar_arrive(tempty(grp));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    }
}

}  // namespace tcg

namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

bool encode_2d(CUtensorMap* map, const void* base, uint64_t inner, uint64_t outer, uint32_t box_inner,
               uint32_t box_outer) {
    const cuuint64_t dims[2] = {inner, outer};
    const cuuint64_t strides[1] = {inner * 2};
    const cuuint32_t box[2] = {box_inner, box_outer};
    const cuuint32_t estr[2] = {1, 1};
    return g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

cudaError_t gemm_tc_setup() {
    if (!g_encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                              cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(tcg::gemm_tc_kernel<kEpiGelu>, at, (int)tcg::SMEM_BYTES);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(tcg::gemm_tc_kernel<kEpiBias>, at, (int)tcg::SMEM_BYTES);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(tcg::gemm_tc_kernel<kEpiResid>, at, (int)tcg::SMEM_BYTES);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(tcg::attn_tc_kernel, at, (int)tcg::ATT_SMEM_BYTES);
    return e;
}

bool gemm_tc_supported(int N, int K) {
    return N > 0 && K > 0 && N % tcg::BN == 0 && K % tcg::BK == 0;
}

cudaError_t gemm_tc(int epi, const __nv_bfloat16* A, const __nv_bfloat16* Wt, const void* bias, void* C,
                    int M, int N, int K, int num_sms, int* d_err, cudaStream_t stream) {
    if (!g_encode || !gemm_tc_supported(N, K) || M < 1) return cudaErrorInvalidValue;
    if (((uintptr_t)A | (uintptr_t)Wt | (uintptr_t)C | (uintptr_t)bias) & 15u) return cudaErrorMisalignedAddress;
    CUtensorMap ta, tb;
    if (!encode_2d(&ta, A, (uint64_t)K, (uint64_t)M, tcg::BK, tcg::BM) ||
        !encode_2d(&tb, Wt, (uint64_t)K, (uint64_t)N, tcg::BK, tcg::BN))
        return cudaErrorInvalidValue;
    const int tiles = ((M + tcg::BM - 1) / tcg::BM) * (N / tcg::BN);
    const int grid = tiles < num_sms ? tiles : num_sms;
    switch (epi) {
        case kEpiGelu:
            tcg::gemm_tc_kernel<kEpiGelu><<<grid, tcg::THREADS, tcg::SMEM_BYTES, stream>>>(ta, tb, bias, C, M, N, K, d_err);
            break;
        case kEpiBias:
            tcg::gemm_tc_kernel<kEpiBias><<<grid, tcg::THREADS, tcg::SMEM_BYTES, stream>>>(ta, tb, bias, C, M, N, K, d_err);
            break;
        case kEpiResid:
            tcg::gemm_tc_kernel<kEpiResid><<<grid, tcg::THREADS, tcg::SMEM_BYTES, stream>>>(ta, tb, bias, C, M, N, K, d_err);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

bool attn_tc_supported(int N, int d) {
    return N >= 1 && N <= tcg::BN && N % 8 == 0 && d % 64 == 0;
}

cudaError_t attn_tc(const __nv_bfloat16* qkv, __nv_bfloat16* O, int B, int N, int H, int d, int num_sms,
                    int* d_err, cudaStream_t stream) {
    if (!g_encode || !attn_tc_supported(N, d) || B < 1 || H * 64 != d) return cudaErrorInvalidValue;
    if (((uintptr_t)qkv | (uintptr_t)O) & 15u) return cudaErrorMisalignedAddress;
    // two maps over the same buffer: query tiles of 64 columns by 128 rows; key and value
    // tiles of 64 columns by 256 rows
    CUtensorMap tq, tk;
    if (!encode_2d(&tq, qkv, (uint64_t)3 * d, (uint64_t)B * N, tcg::BK, tcg::BM) ||
        !encode_2d(&tk, qkv, (uint64_t)3 * d, (uint64_t)B * N, tcg::BK, tcg::BN))
        return cudaErrorInvalidValue;
    const int tiles = B * H * ((N + tcg::BM - 1) / tcg::BM);
    const int grid = tiles < num_sms ? tiles : num_sms;
    tcg::attn_tc_kernel<<<grid, tcg::ATT_THREADS, tcg::ATT_SMEM_BYTES, stream>>>(tq, tk, O, B, N, H, d, d_err);
    return cudaGetLastError();
}
