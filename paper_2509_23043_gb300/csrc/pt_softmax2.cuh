// The exponential shared by the IsingFormer's attention kernels: exp((s - max) / 8) as
// 2^((s - max) log2(e) / 8), one multiply-add and one ex2 per score (the base-2 softmax of
// FlashAttention-2, Dao 2023). The fused scoring attention (pt_gemm_tc.cu) and the sampler's
// bfloat16 step (pt_former.cu) both use it, so that a sampled configuration's log q is the
// one scoring gives it.
#pragma once

namespace ptsm {

// 2^x by the PTX ex2.approx instruction (an approximation; subnormal results flush to zero).
// The attention tests bound its effect on the probabilities against the library path.
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

constexpr float kLog2e8 = 1.4426950408889634f / 8.f;   // log2(e) / sqrt(64), head dimension 64

}  // namespace ptsm
