// Lattice engine: parallel tempering with global proposals (Algorithm 1 of arXiv 2509.23043)
// on periodic L^3 Edwards-Anderson +-J instances with Metropolis local moves.
//
// Layout. The R replicas of an instance are "walkers" packed 32 per uint32 word: word
// [wb][site] holds spin `site` of walkers 32*wb .. 32*wb+31, bit b set iff spin = +1. A
// walker keeps its lane for the whole run; replica exchange permutes the slot <-> walker
// labels (sow / wos) instead of moving spins, which gives the same chain as swapping
// configurations (Eq. P_swap) since the random numbers of a local move are keyed by the walker.
//
// Local move (Methods: local sweeps; Metropolis rule). For a site word s and its six
// neighbour words n_d, the bond d of every walker is unsatisfied iff s ^ n_d ^ Jneg_d; the
// bit-sliced count c of unsatisfied bonds (0..6) gives dE = 12 - 4c. c >= 3 always flips;
// c = 0, 1, 2 flips iff u < T(beta_slot, dE). The comparison runs MSB first over bit planes:
// plane k of the 32 walkers' u is one Philox output word, so planes are only drawn while some
// walker is still undecided (the result is the full 32-bit u < T comparison).
//
// Energy (Algorithm 1: "Compute E(S_r)"). E = 2 U - 3N with U the number of unsatisfied
// bonds. Every bond joins a site to a neighbour of a lower colour exactly once, so U is
// counted, from scratch, in the last sweep of a cycle: each site of colour c > 0 counts its
// bonds to lower-colour neighbours right after its update (its lower neighbours are final).
// Counts are kept as bit-sliced vertical counters and reduced across each warp by bit
// transposes and popcounts.
#include "pt_device.cuh"
#include "pt_layout.h"

namespace pt {

constexpr int KB = 8;  // vertical counter bits: up to 255 bond counts per thread per word

struct LatSmem {
    uint4* tw;
    uint32_t* spins;
    uint32_t* sdesc;
    uint32_t* ebits;
    uint32_t* pbuf;
    int32_t* E;
    int32_t* Eacc;
    uint32_t* st;      // [4][R] statistics of this launch
    int16_t* sow;
    int16_t* wos;
    uint16_t* csites;
};

__device__ __forceinline__ LatSmem carve_lattice(uint8_t* base, const LatInst& I, int nwarps,
                                                 bool with_pool) {
    LatLayout lay = lattice_layout(I.W, I.N, I.NW, I.R, nwarps, with_pool);
    LatSmem S;
    S.tw = reinterpret_cast<uint4*>(base + lay.tw);
    S.spins = reinterpret_cast<uint32_t*>(base + lay.spins);
    S.sdesc = reinterpret_cast<uint32_t*>(base + lay.sdesc);
    S.ebits = reinterpret_cast<uint32_t*>(base + lay.ebits);
    S.pbuf = reinterpret_cast<uint32_t*>(base + lay.pbuf);
    S.E = reinterpret_cast<int32_t*>(base + lay.E);
    S.Eacc = reinterpret_cast<int32_t*>(base + lay.Eacc);
    S.st = reinterpret_cast<uint32_t*>(base + lay.st);
    S.sow = reinterpret_cast<int16_t*>(base + lay.sow);
    S.wos = reinterpret_cast<int16_t*>(base + lay.wos);
    S.csites = reinterpret_cast<uint16_t*>(base + lay.csites);
    return S;
}

// Bit-sliced thresholds of walker block wb: tw[wb*32 + k] = {plane k of T(dE=4), of T(dE=8),
// of T(dE=12)}, lane b taking the thresholds of the slot walker 32 wb + b currently holds.
__device__ void rebuild_thresholds(const LatInst& I, LatSmem& S) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int wb = warp; wb < I.W; wb += nwarps) {
        const int w = wb * 32 + lane;
        const int slot = (w < I.R) ? S.sow[w] : -1;
        uint32_t t4 = 0, t8 = 0, t12 = 0;
        if (slot >= 0) {
            const uint4 t = reinterpret_cast<const uint4*>(I.thr)[slot];
            t4 = t.x; t8 = t.y; t12 = t.z;
        }
        uint4 mine = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll 4
        for (int k = 0; k < 32; ++k) {
            const uint32_t bx = __ballot_sync(kFull, (t4 >> (31 - k)) & 1u);
            const uint32_t by = __ballot_sync(kFull, (t8 >> (31 - k)) & 1u);
            const uint32_t bz = __ballot_sync(kFull, (t12 >> (31 - k)) & 1u);
            if (lane == k) mine = make_uint4(bx, by, bz, 0u);
        }
        S.tw[wb * 32 + lane] = mine;
    }
}

// Add the 3-bit per-walker value (n2 n1 n0) to a bit-sliced counter.
__device__ __forceinline__ void vc_add3(uint32_t (&c)[KB], uint32_t n0, uint32_t n1, uint32_t n2) {
    uint32_t carry = c[0] & n0;
    c[0] ^= n0;
    uint32_t x = c[1];
    c[1] = x ^ n1 ^ carry;
    carry = maj3(x, n1, carry);
    x = c[2];
    c[2] = x ^ n2 ^ carry;
    carry = maj3(x, n2, carry);
#pragma unroll
    for (int j = 3; j < KB; ++j) {
        x = c[j];
        c[j] = x ^ carry;
        carry &= x;
    }
}

// One sweep: colour classes in order, all (site, walker-block) words of a class in parallel.
template <int MAXW>
__device__ __forceinline__ void lattice_sweep(const LatInst& I, LatSmem& S, uint32_t k0,
                                              uint32_t k1, uint32_t sweep_idx, bool flip_on,
                                              bool energy_on, uint32_t (&cnt)[MAXW][KB],
                                              const int (&off)[12]) {
    const int tid = threadIdx.x, T = blockDim.x;
    for (int c = 0; c < I.ncol; ++c) {
        const int base = I.col_off[c];
        const int nc = I.col_off[c + 1] - base;
        const bool acc = energy_on && c > 0;
#pragma unroll
        for (int wb = 0; wb < MAXW; ++wb) {
            if (wb >= I.W) break;
            uint32_t* sp = S.spins + wb * I.N;
            const int rem = I.R - wb * 32;
            const uint32_t vmask = rem >= 32 ? kFull : ((1u << rem) - 1u);
            const uint32_t ctr2 = (kDomPlane << 24) | (uint32_t)wb;
            const uint4* tw = S.tw + wb * 32;
            for (int k = tid; k < nc; k += T) {
                const int site = S.csites[base + k];
                const uint32_t d = S.sdesc[site];
                const uint32_t s = sp[site];
                uint32_t u[6];
#pragma unroll
                for (int dir = 0; dir < 6; ++dir) {
                    const int nb = site + (((d >> (8 + dir)) & 1u) ? off[6 + dir] : off[dir]);
                    u[dir] = s ^ sp[nb] ^ (0u - ((d >> dir) & 1u));
                }
                const uint32_t s1 = u[0] ^ u[1] ^ u[2], c1 = maj3(u[0], u[1], u[2]);
                const uint32_t s2 = u[3] ^ u[4] ^ u[5], c2 = maj3(u[3], u[4], u[5]);
                const uint32_t b0 = s1 ^ s2, t = s1 & s2;
                const uint32_t b1 = c1 ^ c2 ^ t, b2 = maj3(c1, c2, t);
                uint32_t flip = 0;
                if (flip_on) {
                    const uint32_t always = b2 | (b1 & b0);   // c >= 3: dE <= 0
                    uint32_t und = ~always & vmask, lt = 0;
                    for (int qb = 0; qb < 8 && und; ++qb) {
                        const uint4 r = philox(
                            make_uint4((uint32_t)site, sweep_idx, ctr2 | ((uint32_t)qb << 16), I.iid),
                            k0, k1);
                        const uint32_t rw[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const uint4 tt = tw[qb * 4 + j];
                            // c = 0 -> T(12), 1 -> T(8), 2 -> T(4)
                            const uint32_t tk = mux(b1, tt.x, mux(b0, tt.y, tt.z));
                            lt |= und & ~rw[j] & tk;
                            und &= ~(rw[j] ^ tk);
                        }
                    }
                    flip = (always | lt) & vmask;
                    if (flip) sp[site] = s ^ flip;
                }
                if (acc) {
                    uint32_t n0, n1, n2;
                    if (d & (1u << 24)) {
                        // all six neighbours are lower: the new count is 6 - c where flipped
                        n0 = b0;
                        n1 = b1 ^ (flip & ~b0);
                        n2 = b2 ^ (flip & ~(b1 & b0));
                    } else {
                        uint32_t v[6];
#pragma unroll
                        for (int dir = 0; dir < 6; ++dir)
                            v[dir] = (u[dir] ^ flip) & (0u - ((d >> (16 + dir)) & 1u));
                        const uint32_t e1 = v[0] ^ v[1] ^ v[2], f1 = maj3(v[0], v[1], v[2]);
                        const uint32_t e2 = v[3] ^ v[4] ^ v[5], f2 = maj3(v[3], v[4], v[5]);
                        n0 = e1 ^ e2;
                        const uint32_t g = e1 & e2;
                        n1 = f1 ^ f2 ^ g;
                        n2 = maj3(f1, f2, g);
                    }
                    vc_add3(cnt[wb], n0, n1, n2);
                }
            }
        }
        __syncthreads();
    }
}

// Reduce the vertical counters to per-walker energies E = 2U - 3N.
template <int MAXW>
__device__ __forceinline__ void lattice_energy_finalize(const LatInst& I, LatSmem& S,
                                                        uint32_t (&cnt)[MAXW][KB]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int wb = 0; wb < MAXW; ++wb) {
        if (wb >= I.W) break;
        uint32_t acc = 0;
#pragma unroll
        for (int j = 0; j < KB; ++j) {
            if (__any_sync(kFull, cnt[wb][j] != 0u)) {
                const uint32_t tx = warp_transpose32(cnt[wb][j], lane);
                acc += (uint32_t)__popc(tx) << j;
            }
            cnt[wb][j] = 0u;
        }
        if (acc) atomicAdd(&S.Eacc[wb * 32 + lane], (int)acc);
    }
    __syncthreads();
    for (int w = threadIdx.x; w < I.W * 32; w += blockDim.x) {
        S.E[w] = 2 * S.Eacc[w] - 3 * I.N;
        S.Eacc[w] = 0;
    }
    __syncthreads();
}

// One exchange event (Eq. P_swap). Returns (block-uniformly) whether any pair swapped.
__device__ bool lattice_exchange(const LatInst& I, LatSmem& S, uint32_t k0, uint32_t k1,
                                 long long n_ex, int* flag) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const int first = (n_ex & 1) ? 0 : 1;
        bool any = false;
        for (int r = first + 2 * lane; r + 1 < I.R; r += 64) {
            const int wa = S.wos[r], wc = S.wos[r + 1];
            const int dE = S.E[wc] - S.E[wa];
            const double x = (I.beta[r + 1] - I.beta[r]) * (double)dE;
            bool acc = x >= 0.0;
            if (!acc) {
                const uint4 q = philox(make_uint4((uint32_t)r, (uint32_t)n_ex, kDomExch << 24, I.iid),
                                       k0, k1);
                acc = accept_fp64(x, q.x);
            }
            S.st[I.R + r] += 1u;
            if (acc) {
                S.wos[r] = (int16_t)wc;
                S.wos[r + 1] = (int16_t)wa;
                S.sow[wa] = (int16_t)(r + 1);
                S.sow[wc] = (int16_t)r;
                S.st[r] += 1u;
                any = true;
            }
        }
        any = __any_sync(kFull, any);
        if (lane == 0) *flag = any ? 1 : 0;
    }
    __syncthreads();
    return *flag != 0;
}

// One proposal event (Algorithm 1, Eq. P_accept), one warp per proposal-enabled slot.
__device__ void lattice_propose(const LatInst& I, LatSmem& S, uint32_t k0, uint32_t k1,
                                long long n_prop) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int L = I.L, N = I.N, NW = I.NW;
    uint32_t* buf = S.pbuf + warp * NW;
    const int st[3] = {1, L, L * L};
    for (int r = warp; r < I.R; r += nwarps) {
        if (!I.prop[r]) continue;
        const int w = S.wos[r];
        const int c = I.cursor[r];
        const uint32_t* entry = I.pool + (size_t)c * I.pstride + (size_t)r * NW;
        for (int k = lane; k < NW; k += 32) buf[k] = __ldg(entry + k);
        __syncwarp();
        int U = 0;
        for (int k = lane; k < NW; k += 32) {
            const uint32_t vk = (k < NW - 1 || (N & 31) == 0) ? kFull : ((1u << (N & 31)) - 1u);
            const uint32_t sk = buf[k];
#pragma unroll
            for (int dd = 0; dd < 3; ++dd) {
                const uint32_t Wd = S.ebits[(3 + dd) * NW + k];
                const uint32_t A = bits_at(buf, NW, 32 * k + st[dd]);
                const uint32_t B = Wd ? bits_at(buf, NW, 32 * k + st[dd] - L * st[dd]) : 0u;
                const uint32_t nb = (A & ~Wd) | (B & Wd);
                U += __popc((sk ^ nb ^ S.ebits[dd * NW + k]) & vk);
            }
        }
        U = __reduce_add_sync(kFull, U);
        const int ET = 2 * U - 3 * N;
        int acc = 0;
        if (lane == 0) {
            const double x = I.beta[r] * (double)(S.E[w] - ET);
            acc = x >= 0.0;
            if (!acc) {
                const uint4 q = philox(make_uint4((uint32_t)r, (uint32_t)n_prop, kDomProp << 24, I.iid),
                                       k0, k1);
                acc = accept_fp64(x, q.x);
            }
        }
        acc = __shfl_sync(kFull, acc, 0);
        if (acc) {
            uint32_t* sp = S.spins + (w >> 5) * N;
            const uint32_t bit = 1u << (w & 31);
            for (int i = lane; i < N; i += 32) {
                const uint32_t want = (buf[i >> 5] >> (i & 31)) & 1u;
                const uint32_t cur = (sp[i] & bit) ? 1u : 0u;  // only this warp owns this bit
                if (want != cur) atomicXor(&sp[i], bit);
            }
        }
        if (lane == 0) {
            if (acc) S.E[w] = ET;
            I.cursor[r] = (c + 1) % I.P;
            S.st[3 * I.R + r] += 1u;
            if (acc) S.st[2 * I.R + r] += 1u;
        }
        __syncwarp();
    }
}

template <int MAXW>
__global__ void __launch_bounds__(512) lattice_kernel(const LatInst* __restrict__ insts,
                                                       RunArgs a, int with_pool) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int flag;
    const LatInst& I = insts[blockIdx.x];
    const int nwarps = blockDim.x >> 5;
    LatSmem S = carve_lattice(smem, I, nwarps, with_pool != 0);
    const int tid = threadIdx.x, T = blockDim.x;
    const int N = I.N, L = I.L, W = I.W, R = I.R;

    // state in
    for (int i = tid; i < W * N; i += T) S.spins[i] = I.spins[i];
    for (int i = tid; i < N; i += T) { S.sdesc[i] = I.sdesc[i]; S.csites[i] = I.csites[i]; }
    for (int i = tid; i < W * 32; i += T) { S.E[i] = I.E[i]; S.Eacc[i] = 0; S.sow[i] = I.sow[i]; }
    for (int i = tid; i < R; i += T) S.wos[i] = I.wos[i];
    for (int i = tid; i < 4 * R; i += T) S.st[i] = 0u;
    if (with_pool)
        for (int i = tid; i < 6 * I.NW; i += T) S.ebits[i] = I.ebits[i];
    long long sweeps = I.ctr->sweeps, n_ex = I.ctr->n_ex, n_prop = I.ctr->n_prop;
    const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
    const int L2 = L * L, L3 = L2 * L;
    const int off[12] = {1, -1, L, -L, L2, -L2,
                         1 - L, L - 1, L - L2, L2 - L, L2 - L3, L3 - L2};
    __syncthreads();
    rebuild_thresholds(I, S);
    __syncthreads();

    uint32_t cnt[MAXW][KB];
#pragma unroll
    for (int wb = 0; wb < MAXW; ++wb)
#pragma unroll
        for (int j = 0; j < KB; ++j) cnt[wb][j] = 0u;

    if (a.mode & kModeEnergy) {
        lattice_sweep<MAXW>(I, S, k0, k1, (uint32_t)sweeps, false, true, cnt, off);
        lattice_energy_finalize<MAXW>(I, S, cnt);
    }
    if (a.mode & kModeSweeps) {
        for (int k = 0; k < a.n; ++k) {
            lattice_sweep<MAXW>(I, S, k0, k1, (uint32_t)sweeps, true, k == a.n - 1, cnt, off);
            ++sweeps;
        }
        if (a.n > 0) lattice_energy_finalize<MAXW>(I, S, cnt);
    }
    if (a.mode & kModePropose) {
        ++n_prop;
        if (with_pool) lattice_propose(I, S, k0, k1, n_prop);
        __syncthreads();
    }
    if (a.mode & kModeExchange) {
        ++n_ex;
        if (lattice_exchange(I, S, k0, k1, n_ex, &flag)) {
            rebuild_thresholds(I, S);
            __syncthreads();
        }
    }
    if (a.mode & kModeCycles) {
        for (int cyc = 0; cyc < a.n; ++cyc) {
            for (int m = 0; m < a.M; ++m) {
                lattice_sweep<MAXW>(I, S, k0, k1, (uint32_t)sweeps, true, m == a.M - 1, cnt, off);
                ++sweeps;
            }
            lattice_energy_finalize<MAXW>(I, S, cnt);
            if (proposal_due(sweeps, a)) {
                ++n_prop;
                if (with_pool) lattice_propose(I, S, k0, k1, n_prop);
                __syncthreads();
            }
            ++n_ex;
            if (lattice_exchange(I, S, k0, k1, n_ex, &flag)) {
                rebuild_thresholds(I, S);
                __syncthreads();
            }
        }
    }

    // state out
    for (int i = tid; i < W * N; i += T) I.spins[i] = S.spins[i];
    for (int i = tid; i < W * 32; i += T) { I.E[i] = S.E[i]; I.sow[i] = S.sow[i]; }
    for (int i = tid; i < R; i += T) I.wos[i] = S.wos[i];
    for (int i = tid; i < 4 * R; i += T)
        if (S.st[i]) I.stats[i] += S.st[i];
    if (tid == 0) {
        I.ctr->sweeps = sweeps;
        I.ctr->n_ex = n_ex;
        I.ctr->n_prop = n_prop;
    }
}

// Random initial state (Algorithm 1, "Initialize replica states randomly"): word [wb][site]
// is output word 0 of Philox(site, 0, wb, id), i.e. bit b is walker 32 wb + b's spin.
__global__ void lattice_init_kernel(const LatInst* __restrict__ insts, uint64_t seed) {
    const LatInst& I = insts[blockIdx.x];
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int i = threadIdx.x; i < I.W * I.N; i += blockDim.x) {
        const int wb = i / I.N, site = i - wb * I.N;
        const uint4 r = philox(make_uint4((uint32_t)site, 0u, (kDomInit << 24) | (uint32_t)wb, I.iid),
                               k0, k1);
        I.spins[i] = r.x;
    }
}

// Copy slot configurations of a source batch into pool entry `entry` of a destination
// batch (bit strings, site order).
__global__ void lattice_capture_kernel(const LatInst* __restrict__ dst,
                                       const LatInst* __restrict__ src, int entry) {
    const LatInst& D = dst[blockIdx.x];
    const LatInst& Sr = src[blockIdx.x];
    const int N = Sr.N, NW = Sr.NW;
    for (int idx = threadIdx.x; idx < Sr.R * NW; idx += blockDim.x) {
        const int r = idx / NW, k = idx - r * NW;
        const int w = Sr.wos[r];
        const uint32_t* sp = Sr.spins + (w >> 5) * N;
        uint32_t word = 0;
        for (int b = 0; b < 32; ++b) {
            const int i = k * 32 + b;
            if (i < N) word |= ((sp[i] >> (w & 31)) & 1u) << b;
        }
        uint32_t* out = const_cast<uint32_t*>(D.pool) + (size_t)entry * D.pstride + (size_t)r * NW + k;
        *out = word;
    }
}

// Unpack the configurations of one instance in slot order into int8 [R][N].
__global__ void lattice_read_kernel(const LatInst* __restrict__ insts, int inst, int8_t* out) {
    const LatInst& I = insts[inst];
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < I.R * I.N;
         idx += gridDim.x * blockDim.x) {
        const int r = idx / I.N, i = idx - r * I.N;
        const int w = I.wos[r];
        out[idx] = ((I.spins[(w >> 5) * I.N + i] >> (w & 31)) & 1u) ? 1 : -1;
    }
}

// Write one instance's configurations (int8 [R][N], slot order) with walker ids per slot.
__global__ void lattice_write_kernel(const LatInst* __restrict__ insts, int inst,
                                     const int8_t* in, const int32_t* walker) {
    const LatInst& I = insts[inst];
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < I.W * I.N;
         idx += gridDim.x * blockDim.x) {
        const int wb = idx / I.N, i = idx - wb * I.N;
        uint32_t word = 0;
        for (int r = 0; r < I.R; ++r) {
            const int w = walker[r];
            if ((w >> 5) == wb && in[(size_t)r * I.N + i] > 0) word |= 1u << (w & 31);
        }
        I.spins[idx] = word;
    }
}

// ------------------------------------------------------------------------------------
// host-callable launchers
// ------------------------------------------------------------------------------------
cudaError_t launch_lattice(const LatInst* d_insts, int n, int maxW, int threads, size_t smem,
                           const RunArgs& a, int with_pool, cudaStream_t stream) {
    switch (maxW) {
    case 1:
        cudaFuncSetAttribute(lattice_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        lattice_kernel<1><<<n, threads, smem, stream>>>(d_insts, a, with_pool);
        break;
    case 2:
        cudaFuncSetAttribute(lattice_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        lattice_kernel<2><<<n, threads, smem, stream>>>(d_insts, a, with_pool);
        break;
    default:
        cudaFuncSetAttribute(lattice_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        lattice_kernel<4><<<n, threads, smem, stream>>>(d_insts, a, with_pool);
        break;
    }
    return cudaGetLastError();
}

cudaError_t launch_lattice_init(const LatInst* d, int n, uint64_t seed, cudaStream_t s) {
    lattice_init_kernel<<<n, 256, 0, s>>>(d, seed);
    return cudaGetLastError();
}
cudaError_t launch_lattice_capture(const LatInst* dst, const LatInst* src, int n, int entry,
                                   cudaStream_t s) {
    lattice_capture_kernel<<<n, 256, 0, s>>>(dst, src, entry);
    return cudaGetLastError();
}
cudaError_t launch_lattice_read(const LatInst* d, int inst, int8_t* out, int total, cudaStream_t s) {
    lattice_read_kernel<<<(total + 255) / 256, 256, 0, s>>>(d, inst, out);
    return cudaGetLastError();
}
cudaError_t launch_lattice_write(const LatInst* d, int inst, const int8_t* in, const int32_t* walker,
                                 int total, cudaStream_t s) {
    lattice_write_kernel<<<(total + 255) / 256, 256, 0, s>>>(d, inst, in, walker);
    return cudaGetLastError();
}

}  // namespace pt
