/*
 * pt_former.h - C ABI of the GB300 (sm_103a) IsingFormer inference library (libptformer.so):
 * the decoder-only transformer that generates TAPT's global proposals, arXiv 2509.23043
 * (Methods, "IsingFormer architecture and training"; Supplementary S6).
 *
 * The model gives q(x | beta) = prod_t q(x_t | x_<t, beta) over spin configurations x in
 * {-1,+1}^N. Spin -1 is token 0, +1 token 1; input position 0 holds a start token (2), so
 * the output at position t predicts spin t from spins 0 .. t-1. The input of position t is
 * the token embedding plus the inverse-temperature embedding e_beta = W_beta beta + b_beta
 * plus the sinusoidal positional code. Then n_layers pre-layer-norm blocks, each causal
 * masked multi-head self-attention and a GELU (erf form) feed-forward map, a final layer
 * norm and a linear head to two logits. Layer norms use eps = 1e-5.
 *
 * Numerics: weight matrices in bfloat16; each matrix product takes bfloat16 inputs and
 * accumulates in FP32 (tensor cores). The residual stream is FP32; the outputs of the first
 * FFN map (GELU evaluated in FP32 and stored in place) and, for the tensor-core attention,
 * the queries, keys, values and softmax probabilities are stored in bfloat16. Embeddings,
 * layer norms, softmax and the head compute in FP32. The projections run as this library's
 * tcgen05 matrix products or as cuBLASLt products (proj_mode), with the bias (and GELU or the
 * residual add) in the epilogue; the attention's two batched products run on cuBLASLt; every
 * other step runs in this library's kernels.
 *
 * Conventions: every device pointer is caller-owned device memory on the device of the
 * context, read or written in stream order on the context's stream; host pointers are read
 * during the call only. Errors: a pt_status (pt.h) and pt_former_last_error(). A context is
 * not thread safe.
 */
#ifndef PT_FORMER_H
#define PT_FORMER_H
#include <stddef.h>
#include <stdint.h>

#include "pt.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pt_former pt_former;

/* Model shape (the paper's spin-glass and factorization model: d_model 256, 4 heads, 5
 * layers, FFN 1024). n_spins N >= 1 is the sequence length; d_model a multiple of 64 and of
 * n_heads with d_model / n_heads = 64; d_ff a multiple of 8; n_layers >= 0.
 * attn_mode selects the scoring pass's attention: 0 = automatic: when N <= 256 and N is a
 * multiple of 8, the whole attention in one tcgen05 kernel (scores, causal softmax and O = P V
 * on the SM; no score or probability buffer); else as mode 2 while one layer's FP32 scores and
 * bfloat16 probabilities (6 B H N^2 bytes) fit 2 GiB, else the streaming kernel. 1 = always the
 * streaming kernel (FP32, keys and values streamed through shared memory, softmax online).
 * 2 = the scores as batched cuBLASLt products (FP32), a causal-softmax kernel, then O = P V as
 * batched cuBLASLt products.
 * proj_mode selects the projections' matrix products. This library's tcgen05 kernels
 * (TMA-fed, FP32 accumulators in tensor memory, the bias and GELU or the residual add in the
 * epilogue) take projections whose output width is a multiple of 256 and input width a
 * multiple of 64.
 *   0 = automatic: the first FFN map (bias and GELU fused) on the tcgen05 kernel when a call
 *       has at least 16384 rows (B N for scoring); every other product on cuBLASLt, the GELU
 *       in a kernel of its own otherwise;
 *   1 = cuBLASLt products throughout;
 *   2 = the tcgen05 kernels for every projection that suits them (the output map, both FFN
 *       maps, and the query/key/value map of the tensor-core attention), at any row count. */
typedef struct {
    int32_t n_spins;
    int32_t d_model;
    int32_t n_heads;
    int32_t n_layers;
    int32_t d_ff;
    int32_t attn_mode;
    int32_t proj_mode;
} pt_former_config;

/* Number of bfloat16 parameters of a shape: 3d + 2d (embeddings), per layer
 * 2d + 3d^2 + 3d + d^2 + d + 2d + d F + F + F d + d, then 2d + 2d + 2. */
size_t pt_former_param_count(const pt_former_config *cfg);

/* Create a model from host bfloat16 parameters (uint16 bit patterns), in this order, each
 * matrix row-major [in][out] (y = x W + b):
 *   tok_emb [3][d], w_beta [d], b_beta [d],
 *   for each layer: ln1_g [d], ln1_b [d], w_qkv [d][3d] (query, key, value columns),
 *     b_qkv [3d], w_o [d][d], b_o [d], ln2_g [d], ln2_b [d], w_1 [d][F], b_1 [F],
 *     w_2 [F][d], b_2 [d],
 *   lnf_g [d], lnf_b [d], w_out [d][2], b_out [2].
 * n_params must equal pt_former_param_count(cfg). Work on `cuda_stream` (or NULL). */
pt_status pt_former_create(pt_former **out, const pt_former_config *cfg, const uint16_t *params,
                           size_t n_params, void *cuda_stream);

/* Score B configurations (teacher forcing, one pass over all positions): spins int8 [B][N]
 * (+-1, device), beta float [B] (device). Writes log q(x | beta) float [B] (device) and, if
 * logits is not NULL, the logits float [B][N][2] (device; position t's pair scores spin t).
 * This is the Hastings factor an independent Metropolis-Hastings move with a learned q needs
 * (Supplementary S2). Allocates activation buffers for B rows on first use (grown as
 * needed). Stream ordered, no synchronisation. */
pt_status pt_former_score(pt_former *m, int32_t B, const int8_t *spins, const float *beta,
                          float *logq, float *logits);

/* Sample B configurations autoregressively (Supplementary S6), one position after another
 * with a key-value cache: spin t = +1 iff u_{b,t} < q(+1 | spins < t, beta_b), with u the
 * 24-bit uniform (w >> 8) 2^-24 of output word w = 0 of Philox4x32-10 keyed by seed at
 * counter (t, b, 6 << 24, stream), or spin t = prefix[b][t] for t < n_prefix (the clamped
 * product and carry bits of the factorization order). beta float [B], prefix int8
 * [B][n_prefix] or NULL, out int8 [B][N], logq float [B] or NULL; all device. The launches
 * of one (B, n_prefix) are captured in a CUDA graph on first use and replayed afterwards
 * (seed and stream are read from device memory by the kernels). Stream ordered. The
 * key/value cache is bfloat16 with the arithmetic of the fused scoring attention (query, keys
 * and values in bfloat16, unnormalised probabilities rounded to bfloat16 before P V), except
 * with attn_mode 1, where it is FP32 like the streaming attention: log q of a sampled
 * configuration is then the one the scoring pass of the same model gives it, up to summation
 * order (for attn_mode 0 where the fused attention runs, N <= 256 and a multiple of 8; for
 * other N the scoring attention normalises before rounding, a difference of bfloat16 size).
 * PT_ENOTSUP when n_heads x N x 4 bytes (the per-head scores of one configuration, kept in
 * shared memory) exceed 48 KiB. */
pt_status pt_former_sample(pt_former *m, int32_t B, const float *beta, const int8_t *prefix,
                           int32_t n_prefix, uint64_t seed, uint32_t stream_id, int8_t *out,
                           float *logq);

/* Floating-point operations of the matrix products of one scoring pass over B configurations
 * (2 M K N per product, M = B N rows), for roofline accounting. */
double pt_former_score_gemm_flops(const pt_former *m, int32_t B);

/* Wait for the model's stream and report whether a bounded wait inside a tcgen05 product kernel
 * ran out since creation (PT_ECUDA, with the wait's code in the message; the flag stays set).
 * PT_OK otherwise. Synchronises the stream. */
pt_status pt_former_check(pt_former *m);

/* Release the model and its buffers. NULL is allowed. */
pt_status pt_former_destroy(pt_former *m);

/* Message of the last failing call on the calling thread ("" if none). */
const char *pt_former_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
