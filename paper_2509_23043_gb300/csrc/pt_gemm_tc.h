// Host interface of the hand-written tcgen05 kernels (pt_gemm_tc.cu) of the IsingFormer: the
// projections' products with fused epilogues, and the scoring pass's fused causal attention.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

// epilogues: C = GELU(A W + b) and C = A W + b (bfloat16 C and b), C += A W + b (FP32 C and b)
constexpr int kEpiGelu = 0, kEpiBias = 1, kEpiResid = 2;

// Once per process and device, before the first launch (and before any stream capture): looks
// up cuTensorMapEncodeTiled and sets the kernels' shared-memory limit.
cudaError_t gemm_tc_setup();

// Whether an N x K weight shape suits the kernels: N a multiple of 256, K a multiple of 64.
bool gemm_tc_supported(int N, int K);

// C[M][N] from A[M][K] and W given as Wt[N][K] (both operands K-major, bfloat16) with the
// epilogue `epi`; all device pointers 16-byte aligned, row strides K and N. One persistent
// block per SM (num_sms). A wait that runs out records a nonzero code in *d_err (device
// memory) and the kernel returns.
cudaError_t gemm_tc(int epi, const __nv_bfloat16* A, const __nv_bfloat16* Wt, const void* bias, void* C,
                    int M, int N, int K, int num_sms, int* d_err, cudaStream_t stream);

// Whether the fused attention kernel takes sequences of N positions and model width d:
// N <= 256 (one key tile), N a multiple of 8, d a multiple of 64 (head dimension 64).
bool attn_tc_supported(int N, int d);

// O[b N + i][64 h + c] = sum over j <= i of softmax_j(Q_i . K_j / 8) V_j[c], bfloat16 [B N][d],
// from the bfloat16 query/key/value buffer qkv [B N][3d] (head h: queries at columns 64 h,
// keys at d + 64 h, values at 2d + 64 h; H = d / 64). Scores, softmax and P V stay on the SM.
// One persistent block per SM; a wait that runs out records a nonzero code in *d_err and the
// kernel returns.
cudaError_t attn_tc(const __nv_bfloat16* qkv, __nv_bfloat16* O, int B, int N, int H, int d, int num_sms,
                    int* d_err, cudaStream_t stream);
