// Device-side building blocks shared by the lattice (bit-packed) and graph kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pt {

constexpr uint32_t kFull = 0xFFFFFFFFu;

// Random-stream domains: the top byte of counter word 2 (see the kernels for the layout).
constexpr uint32_t kDomInit = 0u, kDomPlane = 1u, kDomWord = 2u, kDomExch = 3u, kDomProp = 4u,
                   kDomCtx = 5u;

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64-bit
// multiplies with xors, key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Global-move decision (Eq. 1 and Eq. 2): accept with min[1, exp(x)] using a
// 32-bit uniform u, i.e. iff x >= 0 or u + 1 <= 2^32 exp(x), decided as in FP64.
// The FP64 exponential is only evaluated near a tie: a float evaluation is within a relative
// 1.7e-6 of 2^32 exp(x) (|x| <= 22.2 rounded to float: 1.4e-6; expf within 2 ulp: 2.4e-7;
// u + 1 and the margin products rounded: 2e-7), so outside a relative margin of 2^-16 the
// float comparison already gives the FP64 decision.
__device__ __forceinline__ bool accept_fp64(double x, uint32_t u) {
    if (x >= 0.0) return true;
    if (x < -22.2) return false;                      // 2^32 exp(x) < 1 <= u + 1
    const float y = expf((float)x) * 4294967296.0f;
    const float a = (float)u + 1.0f;
    if (a < y * (1.0f - 1.52587890625e-05f)) return true;
    if (a > y * (1.0f + 1.52587890625e-05f)) return false;
    return ((double)u + 1.0) <= ldexp(exp(x), 32);
}

// The same decision for x = b * dE (b >= 0 an FP64 inverse-temperature difference or value,
// dE an integer energy difference), the FP64 ratio of Eq. 1 / Eq. 2. x >= 0 is
// read off the signs; otherwise a float product of b and dE (relative error <= 3 * 2^-24 from
// the FP64 product) feeds the float filter, and only near-ties evaluate the FP64 product and
// exponential.
__device__ __forceinline__ bool accept_ratio(double b, float bf, int dE, uint32_t u) {
    if (dE >= 0 || b == 0.0) return true;             // x = b dE >= 0 (incl. -0.0)
    const float xf = bf * (float)dE;
    if (xf < -22.4f) return false;                    // x < -22.2: 2^32 exp(x) < 1 <= u + 1
    if (xf != 0.0f && xf > -22.1f) {
        const float y = expf(xf) * 4294967296.0f;
        const float a = (float)u + 1.0f;
        if (a < y * (1.0f - 1.52587890625e-05f)) return true;
        if (a > y * (1.0f + 1.52587890625e-05f)) return false;
    }
    return accept_fp64(b * (double)dE, u);
}

// bitwise select: bits of a where m is 1, of b where m is 0
__device__ __forceinline__ uint32_t mux(uint32_t m, uint32_t a, uint32_t b) {
    return (m & a) | (~m & b);
}
__device__ __forceinline__ uint32_t maj3(uint32_t a, uint32_t b, uint32_t c) {
    return (a & b) | (a & c) | (b & c);
}

// 32x32 bit transpose across a warp: lane l holds row l (bit b = column b); afterwards lane
// t holds column t (bit l = old bit t of lane l). Five butterfly stages, each a shuffle, a
// per-lane rotate and a bitwise select.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
#pragma unroll
    for (int j = 16; j >= 1; j >>= 1) {
        const uint32_t m = (j == 16) ? 0x0000FFFFu : (j == 8) ? 0x00FF00FFu
                         : (j == 4) ? 0x0F0F0F0Fu : (j == 2) ? 0x33333333u : 0x55555555u;
        const bool upper = (lane & j) != 0;
        const uint32_t y = __shfl_xor_sync(kFull, x, j);
        const uint32_t rot = __funnelshift_l(y, y, upper ? 32 - j : j);
        const uint32_t keep = upper ? ~m : m;
        x = (x & keep) | (rot & ~keep);
    }
    return x;
}

// 32 bits of a bit string S[0..nw) starting at bit position pos (may be out of range:
// bits outside the string read as 0).
__device__ __forceinline__ uint32_t bits_at(const uint32_t* S, int nw, int pos) {
    const int q = pos >> 5;
    const int r = pos & 31;
    const uint32_t lo = (q >= 0 && q < nw) ? S[q] : 0u;
    const uint32_t hi = (q + 1 >= 0 && q + 1 < nw) ? S[q + 1] : 0u;
    return __funnelshift_r(lo, hi, r);
}

// ------------------------------------------------------------------------------------
// Per-instance descriptors (device memory). Pointers are into the context's buffers.
// ------------------------------------------------------------------------------------
struct Counters {
    long long sweeps;   // sweeps done (the sweep index of the next sweep)
    long long n_ex;     // exchange events done
    long long n_prop;   // proposal events done
    long long pad;
};

// Lattice engine: periodic L^3, J = +-1, no field, no clamp, Metropolis or Gibbs. Spins
// bit-packed: word [wb][site], bit b = walker 32*wb + b.
struct LatInst {
    uint32_t iid;
    int32_t L, N, R, W, NW, ncol, P;
    int32_t nit;           // words per thread per colour class at the launch's block size
    int32_t col_off[4];
    uint32_t* spins;       // [W][N] in site order
    const uint4* itab;     // [N] one entry per site, in colour order (item k of colour c is
                           // itab[col_off[c] + k]); in shared memory the spins are stored in
                           // this colour-major order (item k of colour c at col_off[c] + k).
                           // Eight 16-bit fields:
                           //   x.lo  site index
                           //   x.hi  bits 0-5: neighbour d has a lower colour; bit 6: all six
                           //   y,z,w six neighbours (+x,-x,+y,-y,+z,-z): byte offset into
                           //         the shared {word, complement} pairs (8 bytes per site,
                           //         colour-major) of the neighbour's word, or of its
                           //         complement (+4) when the bond is -1
    const uint16_t* pos;   // [N] colour-major position of each site
    uint2* gspins;         // [W][N] {word, complement}, colour-major, in global memory: the
                           // working copy of an instance whose spins and table do not fit
                           // shared memory (the GSP kernels read itab in place); else nullptr
    const int32_t* active; // nonzero: the instance takes part in launches
    int32_t* E;            // [W*32] per walker
    int16_t* sow;          // [W*32] slot of walker (-1: padding lane)
    int16_t* wos;          // [R] walker of slot
    const uint32_t* thr;   // [R][4] Metropolis thresholds for dE = 4, 8, 12 (and 0 pad), or
                           // [R][8] Gibbs thresholds for I = 6 - 2q, q = 0..6 (and 0 pad)
    const double* beta;    // [R]
    const uint8_t* prop;   // [R]
    int32_t* cursor;       // [R]
    const uint32_t* ebits; // [6][NW]: negative-bond bits +x,+y,+z; wrap bits x,y,z
    const uint32_t* pool;  // entry e, slot r at pool + e * pstride + r * NW
    long long pstride;     // words between consecutive pool entries
    Counters* ctr;
    unsigned long long* stats;  // [4][R]: swap acc, swap att, prop acc, prop att
    const long long* lw;   // [R][N] proposal rule 2: log-odds of each slot's proposal law in
                           // units of 2^-32 (site order), or nullptr
};

// The FP64 acceptance exponent of proposal rule 2 (the independent Metropolis-Hastings move,
// Supplementary S2): x = beta_r (E_r - E^T) + (log q(x_r) - log q(x^T)), the log-odds sum d
// in units of 2^-32 (exact: |d| < 2^53). Rounded product, then rounded sum, never fused.
__device__ __forceinline__ double mh_exponent(double beta, int dE, long long d) {
    return __dadd_rn(__dmul_rn(beta, (double)dE), (double)d * 2.3283064365386963e-10);
}

// Lattice kernel flags: pool proposals, contextual proposals
constexpr int kWithPool = 1, kWithContext = 2, kGibbs = 4, kGlobalSpins = 8;

// Kernel modes
enum : int32_t {
    kModeSweeps = 1,     // n sweeps then energies
    kModePropose = 2,    // one proposal event
    kModeExchange = 4,   // one exchange event
    kModeCycles = 8,     // n cycles of Algorithm 1
    kModeEnergy = 16,    // energies only
};

struct RunArgs {
    uint64_t seed;
    int32_t mode;
    int32_t n;
    int32_t M, every, start, stop;
    int32_t update;      // 0 Metropolis, 1 Gibbs (the lattice engine takes it from its template)
    int32_t prule;       // proposal rule: 0 Delta-E-only, 1 always accept, 2 independent MH
    int32_t ctx_log2;    // contextual proposals: a site is kept with probability 2^-ctx_log2
    int32_t ctx_sweeps;  // contextual proposals: refill sweeps
    uint32_t rk0[10];    // Philox round keys of the seed (kernel parameters, so the rounds
    uint32_t rk1[10];    // read them as constant operands)
};

// Philox4x32-10 with precomputed round keys.
__device__ __forceinline__ uint4 philox_rk(uint4 c, const RunArgs& a) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ a.rk0[i], lo1, hi0 ^ c.w ^ a.rk1[i], lo0);
    }
    return c;
}

// 4-byte asynchronous global -> shared copies (cp.async, sm_80 and later).
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ bool proposal_due(long long s, const RunArgs& a) {
    if (a.every <= 0 || s < a.start) return false;
    if (a.stop > 0 && s > a.stop) return false;
    return ((s - a.start) % a.every) == 0;
}

}  // namespace pt
