// Graph engine: parallel tempering with global proposals (Algorithm 1 of arXiv 2509.23043)
// on general sparse integer-coupled Ising graphs with fields and clamped spins (e.g. the
// invertible multiplier of Supplementary S4), Gibbs (the paper's rule, Methods) or
// Metropolis local moves, colour class by colour class (DSATUR colouring, Methods).
//
// Layout. Spin bytes [N][Rp] (Rp = R rounded up to 8), 1 where the spin is -1 and 0 where
// it is +1: a thread updates eight walkers of one site from one 8-byte load, and a neighbour's
// 8-byte group is directly the eight walkers' [m = -1] flags. A walker keeps its storage
// column; exchange permutes slot <-> walker labels, thresholds are looked up by the walker's
// current slot.
#include "pt_device.cuh"
#include "pt_layout.h"
#include "pt_graph.cuh"

namespace pt {

struct GraphSmem {
    int8_t* spins;
    uint32_t* thr;
    int32_t* rowp;
    int4* smeta;                 // [nfree] {site, row begin, row split, row end}, colour order
    int32_t* adj;
    int32_t* adjJ;
    int32_t* adjp;
    int32_t* h;
    int2* hk;                    // [nfree] colour order
    int32_t* E;
    int32_t* Eacc;
    uint32_t* st;
    int16_t* sow;
    int16_t* wos;
    uint32_t* pbuf;
    uint32_t* pM;
    uint32_t* pe_ab;
    int32_t* pe_J;
    int32_t* ph_i;
    int32_t* ph_h;
};

__device__ __forceinline__ GraphSmem carve_graph(uint8_t* base, const GraphInst& I,
                                                 bool with_pool) {
    GraphLayout l = graph_layout(I.N, I.R, I.Rp, I.NE, I.Imax, I.nfree, I.NW, with_pool,
                                 I.packed != 0, I.nEb, I.nHb);
    GraphSmem S;
    S.spins = reinterpret_cast<int8_t*>(base + l.spins);
    S.thr = reinterpret_cast<uint32_t*>(base + l.thr);
    S.rowp = reinterpret_cast<int32_t*>(base + l.rowp);
    S.smeta = reinterpret_cast<int4*>(base + l.smeta);
    S.adj = reinterpret_cast<int32_t*>(base + l.adj);
    S.adjJ = reinterpret_cast<int32_t*>(base + l.adjJ);
    S.adjp = reinterpret_cast<int32_t*>(base + l.adjp);
    S.h = reinterpret_cast<int32_t*>(base + l.h);
    S.hk = reinterpret_cast<int2*>(base + l.hk);
    S.E = reinterpret_cast<int32_t*>(base + l.E);
    S.Eacc = reinterpret_cast<int32_t*>(base + l.Eacc);
    S.st = reinterpret_cast<uint32_t*>(base + l.st);
    S.sow = reinterpret_cast<int16_t*>(base + l.sow);
    S.wos = reinterpret_cast<int16_t*>(base + l.wos);
    S.pbuf = reinterpret_cast<uint32_t*>(base + l.pbuf);
    S.pM = reinterpret_cast<uint32_t*>(base + l.pM);
    S.pe_ab = reinterpret_cast<uint32_t*>(base + l.pe_ab);
    S.pe_J = reinterpret_cast<int32_t*>(base + l.pe_J);
    S.ph_i = reinterpret_cast<int32_t*>(base + l.ph_i);
    S.ph_h = reinterpret_cast<int32_t*>(base + l.ph_h);
    return S;
}

// four bits to the low bits of four bytes: bit k -> bit 8 k
__device__ __forceinline__ uint32_t spread4(uint32_t x) {
    return (x * 0x00204081u) & 0x01010101u;
}

// the spin (+1 or -1) of walker k of a stored word
__device__ __forceinline__ int sbyte(uint32_t w, int k) {
    return 1 - 2 * (int)((w >> (8 * k)) & 1u);
}

// One sweep: every free site of every colour class, eight walkers per thread. Thread t takes
// the eight walkers of octet t % O (O = Rp / 8) at the sites t / O, t / O + Ts / O, ... of
// each class (Ts, the threads used, a multiple of O), so it keeps one octet for the whole
// sweep and neighbouring lanes read neighbouring 8-byte groups of one row.
// Uniforms: walker w's 32-bit u at (site, sweep) is hi << 16 | lo, hi the 16-bit half
// (w odd: low, even: high) of output word (w & 7) / 2 of Philox(site, sweep, 2 << 24 | w / 8,
// id) and lo the same half of Philox(site, sweep, 2 << 24 | 1 << 16 | w / 8, id). u < thr
// follows from hi alone unless hi equals the high half of thr (probability at most 2^-16 per
// walker), so the second call runs only for a thread that meets such a tie.
// With energy_on (the last sweep of a cycle) each thread adds, for its octet, the energy
// terms of the free sites it updates: -m (h + the bonds to its counted neighbours,
// rowp..rowl), which sum with Eclamp to the exact energy (each bond counted once, at the end
// updated last); graph_energy_finish turns them into E.
// the rare second draw of graph_sweep_t, out of line so that its registers are not reserved
// across the common path
__device__ __noinline__ uint4 philox_cold(uint4 c, uint32_t k0, uint32_t k1) {
    return philox(c, k0, k1);
}

template <bool PACKED, bool GIBBS>
__device__ void graph_sweep_t(const GraphInst& I, GraphSmem& S, const RunArgs& a,
                              uint32_t sweep_idx, bool energy_on) {
    // the instance's scalars in registers: the descriptor lives in global memory, and the
    // shared-memory stores below would otherwise force it to be read again
    const int O = I.Rp >> 3, R = I.R, Imax = I.Imax, ncol = I.ncol;
    const uint32_t iid = I.iid;
    const int tw = 2 * Imax + 1;
    const int Ts = (blockDim.x / O) * O;
    const int tid = threadIdx.x;
    const int oct = tid % O;
    const int s0 = tid / O, sstep = Ts / O;         // the thread's first site, site stride
    uint2* sp = reinterpret_cast<uint2*>(S.spins);
    // the thread's eight walkers: threshold rows of their slots (fixed during a sweep); the
    // walkers beyond R keep their bytes
    int trow[8];
    uint32_t valid = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int w = oct * 8 + j;
        trow[j] = (w < R) ? S.sow[w] * tw + Imax : Imax;
        valid |= (uint32_t)(w < R) << j;
    }
    // byte masks of the valid walkers in the two words
    const uint32_t vbyte[2] = {spread4(valid & 0xFu), spread4(valid >> 4)};
    int e[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int cbeg = I.col_off[0];
    for (int c = 0; c < ncol; ++c) {
        const int base = cbeg;
        cbeg = I.col_off[c + 1];
        const int nc = cbeg - base;
        for (int si = s0; si < nc && tid < Ts; si += sstep) {
            const int4 meta = S.smeta[base + si];
            const int site = meta.x, split = meta.z, end = meta.w;
            // packed rows: bytes of cw / tw_: 128 + the sum of J over the counted / all
            // neighbours whose spin is -1 (tw_ = cw + rw - 128 per byte, exact: every byte stays
            // within 1..255). With sum J m = sum J - 2 sum_{m=-1} J, h + the counted sum is
            // hk.x - 2 byte(cw) and the local field hk.y - 2 byte(tw_).
            // general rows: hg, f the sums themselves.
            uint32_t cw[2], tw_[2];
            int2 kk;
            int hg[PACKED ? 1 : 8], f[PACKED ? 1 : 8];
            if constexpr (PACKED) {
                uint32_t c0 = 0x80808080u, c1 = 0x80808080u, r0 = 0x80808080u, r1 = 0x80808080u;
                // unrolled: the loads of several neighbours are in flight together
#pragma unroll 4
                for (int a2 = meta.y; a2 < split; ++a2) {
                    const uint32_t pk = (uint32_t)S.adjp[a2];
                    const uint32_t J = (uint32_t)(int)(int8_t)(pk & 0xFFu);
                    const uint2 nb = sp[(pk >> 8) + oct];
                    c0 += J * nb.x;
                    c1 += J * nb.y;
                }
#pragma unroll 4
                for (int a2 = split; a2 < end; ++a2) {
                    const uint32_t pk = (uint32_t)S.adjp[a2];
                    const uint32_t J = (uint32_t)(int)(int8_t)(pk & 0xFFu);
                    const uint2 nb = sp[(pk >> 8) + oct];
                    r0 += J * nb.x;
                    r1 += J * nb.y;
                }
                cw[0] = c0;
                cw[1] = c1;
                tw_[0] = c0 + r0 - 0x80808080u;
                tw_[1] = c1 + r1 - 0x80808080u;
                kk = S.hk[base + si];
            } else {
                const int hs = S.h[site];
#pragma unroll
                for (int j = 0; j < 8; ++j) hg[j] = hs;
                for (int a2 = meta.y; a2 < split; ++a2) {
                    const uint2 wd = sp[S.adj[a2] * O + oct];
                    const int J = S.adjJ[a2];
#pragma unroll
                    for (int j = 0; j < 8; ++j) hg[j] += J * sbyte(j < 4 ? wd.x : wd.y, j & 3);
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) f[j] = hg[j];
                for (int a2 = split; a2 < end; ++a2) {
                    const uint2 wd = sp[S.adj[a2] * O + oct];
                    const int J = S.adjJ[a2];
#pragma unroll
                    for (int j = 0; j < 8; ++j) f[j] += J * sbyte(j < 4 ? wd.x : wd.y, j & 3);
                }
            }
            auto field = [&](int j) -> int {
                if constexpr (PACKED) return kk.y - 2 * (int)((tw_[j >> 2] >> (8 * (j & 3))) & 0xFFu);
                else return f[j];
            };
            auto counted = [&](int j) -> int {
                if constexpr (PACKED) return kk.x - 2 * (int)((cw[j >> 2] >> (8 * (j & 3))) & 0xFFu);
                else return hg[j];
            };
            const uint2 own = sp[site * O + oct];
            const uint32_t ob[2] = {own.x, own.y};
            // threshold index of walker j; Metropolis: moves with m I <= 0 are taken outright
            auto index = [&](int j) -> int {
                if constexpr (GIBBS) return trow[j] + field(j);
                else return trow[j] + max(sbyte(ob[j >> 2], j & 3) * field(j), 0);
            };
            uint32_t forced = 0;
            if constexpr (!GIBBS) {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    forced |= (uint32_t)(sbyte(ob[j >> 2], j & 3) * field(j) <= 0) << j;   // dE = 2 m I
                forced &= valid;
            }
            const uint4 rh = philox_rk(make_uint4((uint32_t)site, sweep_idx,
                                                  (kDomWord << 24) | (uint32_t)oct, iid), a);
            const uint32_t hw[4] = {rh.x, rh.y, rh.z, rh.w};
            uint32_t below = 0, tie = 0;   // u < thr on the high halves; undecided there
            // every walker draws, without a branch: a padding walker reads slot 0's row and a
            // forced Metropolis move row + 0, both in the table; their results are masked
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint32_t t = S.thr[index(j)];
                const uint32_t x = (j & 1) ? (hw[j >> 1] << 16) : (hw[j >> 1] & 0xFFFF0000u);
                below |= (uint32_t)(x < t) << j;
                tie |= (uint32_t)(((x ^ t) >> 16) == 0u) << j;
            }
            tie &= valid & ~forced;        // forced moves and padding walkers need no low half
            if (tie) {
                const uint4 rl = philox_cold(make_uint4((uint32_t)site, sweep_idx,
                                                        (kDomWord << 24) | (1u << 16) | (uint32_t)oct, iid),
                                             (uint32_t)a.seed, (uint32_t)(a.seed >> 32));
                const uint32_t lw[4] = {rl.x, rl.y, rl.z, rl.w};
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (!(tie >> j & 1u)) continue;
                    const uint32_t x = (j & 1) ? (hw[j >> 1] << 16) : (hw[j >> 1] & 0xFFFF0000u);
                    const uint32_t lo = (j & 1) ? (lw[j >> 1] & 0xFFFFu) : (lw[j >> 1] >> 16);
                    below = (below & ~(1u << j)) | ((uint32_t)((x | lo) < S.thr[index(j)]) << j);
                }
            }
            // new [m = -1] flags: Gibbs m = +1 iff u < thr; Metropolis flips if forced or u < thr
            uint32_t out[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t nib = ((GIBBS ? ~below : (forced | below)) >> (4 * h)) & 0xFu;
                out[h] = GIBBS ? ((ob[h] & ~vbyte[h]) | (spread4(nib) & vbyte[h]))
                               : (ob[h] ^ (spread4(nib) & vbyte[h]));
            }
            if (energy_on) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int g = counted(j);
                    e[j] += ((out[j >> 2] >> (8 * (j & 3))) & 1u) ? g : -g;
                }
            }
            if (out[0] != ob[0] || out[1] != ob[1]) sp[site * O + oct] = make_uint2(out[0], out[1]);
        }
        if (energy_on && c == ncol - 1 && tid < Ts) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (e[j]) atomicAdd(&S.Eacc[oct * 8 + j], e[j]);
        }
        __syncthreads();
    }
}

// KIND 1: every instance of the launch has packed rows; 0: either kind, chosen per instance
template <int KIND, bool GIBBS>
__device__ __forceinline__ void graph_sweep(const GraphInst& I, GraphSmem& S, const RunArgs& a,
                                            uint32_t sweep_idx, bool energy_on) {
    if constexpr (KIND == 1) {
        graph_sweep_t<true, GIBBS>(I, S, a, sweep_idx, energy_on);
    } else {
        if (I.packed) graph_sweep_t<true, GIBBS>(I, S, a, sweep_idx, energy_on);
        else graph_sweep_t<false, GIBBS>(I, S, a, sweep_idx, energy_on);
    }
}

// E = Eclamp + the terms the last sweep accumulated; clears the accumulators. Ends
// synchronised.
__device__ void graph_energy_finish(const GraphInst& I, GraphSmem& S) {
    for (int w = threadIdx.x; w < I.Rp; w += blockDim.x) {
        S.E[w] = I.Eclamp + S.Eacc[w];
        S.Eacc[w] = 0;
    }
    __syncthreads();
}

// Exact energies of every walker: E = -1/2 sum_i m_i (I_i + h_i), lanes = walkers.
__device__ void graph_energy(const GraphInst& I, GraphSmem& S) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int wb = 0; wb * 32 < I.R; ++wb) {
        const int w = wb * 32 + lane;
        int acc = 0;
        if (w < I.R) {
            for (int site = warp; site < I.N; site += nwarps) {
                const int hs = I.h[site];
                int f = hs;
                if (I.packed) {
                    for (int a = S.rowp[site]; a < S.rowp[site + 1]; ++a) {
                        const uint32_t pk = (uint32_t)S.adjp[a];
                        f += (int)(int8_t)(pk & 0xFFu) * (1 - 2 * (int)S.spins[(pk >> 8) * 8 + w]);
                    }
                } else {
                    for (int a = S.rowp[site]; a < S.rowp[site + 1]; ++a)
                        f += S.adjJ[a] * (1 - 2 * (int)S.spins[S.adj[a] * I.Rp + w]);
                }
                acc += (1 - 2 * (int)S.spins[site * I.Rp + w]) * (f + hs);
            }
            atomicAdd(&S.Eacc[w], acc);
        }
    }
    __syncthreads();
    for (int w = threadIdx.x; w < I.Rp; w += blockDim.x) {
        S.E[w] = -(S.Eacc[w] / 2);
        S.Eacc[w] = 0;
    }
    __syncthreads();
}

__device__ void graph_exchange(const GraphInst& I, GraphSmem& S, uint32_t k0, uint32_t k1,
                               long long n_ex) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const int first = (n_ex & 1) ? 0 : 1;
        for (int r = first + 2 * lane; r + 1 < I.R; r += 64) {
            const int wa = S.wos[r], wc = S.wos[r + 1];
            const int dE = S.E[wc] - S.E[wa];
            const double db = I.beta[r + 1] - I.beta[r];
            bool acc = dE >= 0 || db == 0.0;
            if (!acc) {
                const uint4 q = philox(make_uint4((uint32_t)r, (uint32_t)n_ex, kDomExch << 24, I.iid),
                                       k0, k1);
                acc = accept_ratio(db, (float)db, dE, q.x);
            }
            S.st[I.R + r] += 1u;
            if (acc) {
                S.wos[r] = (int16_t)wc;
                S.wos[r + 1] = (int16_t)wa;
                S.sow[wa] = (int16_t)(r + 1);
                S.sow[wc] = (int16_t)r;
                S.st[r] += 1u;
            }
        }
    }
    __syncthreads();
}

// One proposal event (Eq. 2) for every enabled slot at once.
//  1. All threads stage the current pool entry of every enabled slot, clamps applied.
//  2. Transpose to one word per site and group of 32 slots: bit l of pM[g][i] is spin i of
//     slot 32 g + l's entry (1 = +1).
//  3. Energies: with x = [m_a != m_b] and b = [m_i = +1], E = Kprop + 2 (sum_e J_e x_e -
//     sum_i h_i b_i). A block of 32 edges of one coupling gives one xor word per lane (its
//     edge, bit = slot); a warp transpose turns it into one word per slot (bit = edge), whose
//     popcount times the block's coupling is the slot's share. Sites of one field likewise.
//  4. The decision of each slot, one thread per slot.
//  5. Accepted entries are copied into their walkers' columns.
// Eacc (zero between events) holds the sums, then the decisions, and is cleared again.
__device__ void graph_propose(const GraphInst& I, GraphSmem& S, uint32_t k0, uint32_t k1,
                              long long n_prop, int rule) {
    const int tid = threadIdx.x, T = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nwarps = T >> 5;
    const int N = I.N, NW = I.NW, R = I.R, G = (R + 31) >> 5, N1 = N + 1;
    const int nEb = I.nEb, nB = I.nEb + I.nHb;
    for (int idx = tid; idx < R * NW; idx += T) {
        const int r = idx / NW, k = idx - r * NW;
        if (!I.prop[r]) continue;
        const uint32_t* entry = I.pool + (size_t)I.cursor[r] * I.pstride + (size_t)r * NW;
        S.pbuf[idx] = (__ldg(entry + k) & ~I.cbits[k]) | I.cbits[NW + k];
    }
    __syncthreads();
    for (int gk = warp; gk < G * NW; gk += nwarps) {
        const int g = gk / NW, k = gk - g * NW;
        const int r = 32 * g + lane;
        const uint32_t x = (r < R && I.prop[r]) ? S.pbuf[r * NW + k] : 0u;
        const uint32_t y = warp_transpose32(x, lane);
        const int i = 32 * k + lane;
        if (i < N) S.pM[g * N1 + i] = y;
    }
    if (tid < G) S.pM[tid * N1 + N] = 0u;
    __syncthreads();
    for (int g = 0; g < G; ++g) {
        const uint32_t* M = S.pM + g * N1;
        int acc = 0;
        for (int bk = warp; bk < nB; bk += nwarps) {
            uint32_t x;
            int wgt;
            if (bk < nEb) {
                const uint32_t ab = S.pe_ab[bk * 32 + lane];
                x = M[ab & 0xFFFFu] ^ M[ab >> 16];
                wgt = S.pe_J[bk];
            } else {
                x = M[S.ph_i[(bk - nEb) * 32 + lane]];
                wgt = -S.ph_h[bk - nEb];
            }
            acc += wgt * __popc(warp_transpose32(x, lane));
        }
        const int r = 32 * g + lane;
        if (r < R && acc != 0) atomicAdd(&S.Eacc[r], acc);
    }
    __syncthreads();
    if (rule == 2) {
        // the independent Metropolis-Hastings move (Supplementary S2): one warp per slot sums
        // the Hastings correction log q(x_r) - log q(x^T) over the sites, lane 0 decides (the
        // slot's accept flag replaces its energy count in Eacc; the other slots' counts are
        // read by their own warps first)
        for (int r = warp; r < R; r += nwarps) {
            if (!I.prop[r]) continue;
            const int w = S.wos[r];
            const long long* lw = I.lw + (size_t)r * N;
            const uint32_t* buf = S.pbuf + r * NW;
            long long d = 0;
            for (int i = lane; i < N; i += 32) {
                const long long wi = __ldg(lw + i);
                if (S.spins[i * I.Rp + w] == 0) d += wi;          // current spin +1
                if ((buf[i >> 5] >> (i & 31)) & 1u) d -= wi;      // proposed spin +1
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) d += __shfl_xor_sync(kFull, d, o);
            if (lane == 0) {
                const int ET = I.Kprop + 2 * S.Eacc[r];
                const uint4 q = philox(make_uint4((uint32_t)r, (uint32_t)n_prop, kDomProp << 24, I.iid),
                                       k0, k1);
                const int acc = accept_fp64(mh_exponent(I.beta[r], S.E[w] - ET, d), q.x);
                if (acc) S.E[w] = ET;
                I.cursor[r] = (I.cursor[r] + 1) % I.P;
                S.st[3 * R + r] += 1u;
                if (acc) S.st[2 * R + r] += 1u;
                S.Eacc[r] = acc;
            }
        }
        for (int r = tid; r < R; r += T)
            if (!I.prop[r]) S.Eacc[r] = 0;
    } else
    for (int r = tid; r < R; r += T) {
        int acc = 0;
        if (I.prop[r]) {
            const int ET = I.Kprop + 2 * S.Eacc[r];
            const int w = S.wos[r];
            const int dE = S.E[w] - ET;
            acc = rule == 1 || dE >= 0 || I.beta[r] == 0.0;
            if (!acc) {
                const uint4 q = philox(make_uint4((uint32_t)r, (uint32_t)n_prop, kDomProp << 24, I.iid),
                                       k0, k1);
                acc = accept_ratio(I.beta[r], (float)I.beta[r], dE, q.x);
            }
            if (acc) S.E[w] = ET;
            I.cursor[r] = (I.cursor[r] + 1) % I.P;
            S.st[3 * R + r] += 1u;
            if (acc) S.st[2 * R + r] += 1u;
        }
        S.Eacc[r] = acc;
    }
    __syncthreads();
    for (int r = warp; r < R; r += nwarps) {
        if (!S.Eacc[r]) continue;
        const int w = S.wos[r];
        const uint32_t* buf = S.pbuf + r * NW;
        for (int i = lane; i < N; i += 32)
            S.spins[i * I.Rp + w] = (int8_t)(((buf[i >> 5] >> (i & 31)) & 1u) ^ 1u);
    }
    __syncthreads();
    for (int r = tid; r < R; r += T) S.Eacc[r] = 0;
}

// The fused cycle kernel's body (one block per instance); the kernels below instantiate it.
template <int KIND, bool GIBBS>
__device__ __forceinline__ void graph_body(const GraphInst* __restrict__ insts, const RunArgs& a,
                                           int with_pool) {
    extern __shared__ __align__(16) uint8_t smem[];
    const GraphInst& I = insts[blockIdx.x];
    if (!*I.active) return;
    GraphSmem S = carve_graph(smem, I, with_pool != 0);
    const int tid = threadIdx.x, T = blockDim.x;
    const int N = I.N, R = I.R, Rp = I.Rp;
    {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(I.spins);
        uint32_t* dst = reinterpret_cast<uint32_t*>(S.spins);
        for (int i = tid; i < N * Rp / 4; i += T) dst[i] = src[i];
    }
    const int tw = 2 * I.Imax + 1;
    for (int i = tid; i < R * tw; i += T) S.thr[i] = I.thr[i];
    for (int i = tid; i <= N; i += T) S.rowp[i] = I.rowp[i];
    if (I.packed) {
        for (int i = tid; i < 2 * I.NE; i += T) S.adjp[i] = I.adjp[i];
    } else {
        for (int i = tid; i < 2 * I.NE; i += T) {
            S.adj[i] = I.adj[i];
            S.adjJ[i] = I.adjJ[i];
        }
    }
    for (int i = tid; i < I.nfree; i += T) {
        const int site = I.csites[i];
        S.smeta[i] = make_int4(site, I.rowp[site], I.rowl[site], I.rowp[site + 1]);
        if (I.packed) S.hk[i] = I.hk[site];
    }
    if (!I.packed)
        for (int i = tid; i < N; i += T) S.h[i] = I.h[i];
    if (with_pool) {
        for (int k = tid; k < 32 * I.nEb; k += T) S.pe_ab[k] = I.pe_ab[k];
        for (int k = tid; k < I.nEb; k += T) S.pe_J[k] = I.pe_J[k];
        for (int k = tid; k < 32 * I.nHb; k += T) S.ph_i[k] = I.ph_i[k];
        for (int k = tid; k < I.nHb; k += T) S.ph_h[k] = I.ph_h[k];
    }
    for (int i = tid; i < Rp; i += T) { S.E[i] = I.E[i]; S.Eacc[i] = 0; S.sow[i] = I.sow[i]; }
    for (int i = tid; i < R; i += T) S.wos[i] = I.wos[i];
    for (int i = tid; i < 4 * R; i += T) S.st[i] = 0u;
    long long sweeps = I.ctr->sweeps, n_ex = I.ctr->n_ex, n_prop = I.ctr->n_prop;
    const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
    __syncthreads();

    if (a.mode & kModeEnergy) graph_energy(I, S);
    if (a.mode & kModeSweeps) {
        for (int k = 0; k < a.n; ++k) {
            graph_sweep<KIND, GIBBS>(I, S, a, (uint32_t)sweeps, k == a.n - 1);
            ++sweeps;
        }
        if (a.n > 0) graph_energy_finish(I, S);
    }
    if (a.mode & kModePropose) {
        ++n_prop;
        if (with_pool) graph_propose(I, S, k0, k1, n_prop, a.prule);
        __syncthreads();
    }
    if (a.mode & kModeExchange) {
        ++n_ex;
        graph_exchange(I, S, k0, k1, n_ex);
    }
    if (a.mode & kModeCycles) {
        for (int cyc = 0; cyc < a.n; ++cyc) {
            for (int m = 0; m < a.M; ++m) {
                graph_sweep<KIND, GIBBS>(I, S, a, (uint32_t)sweeps, m == a.M - 1);
                ++sweeps;
            }
            graph_energy_finish(I, S);
            if (proposal_due(sweeps, a)) {
                ++n_prop;
                if (with_pool) graph_propose(I, S, k0, k1, n_prop, a.prule);
                __syncthreads();
            }
            ++n_ex;
            graph_exchange(I, S, k0, k1, n_ex);
        }
    }

    {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(S.spins);
        uint32_t* dst = reinterpret_cast<uint32_t*>(I.spins);
        for (int i = tid; i < N * Rp / 4; i += T) dst[i] = src[i];
    }
    for (int i = tid; i < Rp; i += T) { I.E[i] = S.E[i]; I.sow[i] = S.sow[i]; }
    for (int i = tid; i < R; i += T) I.wos[i] = S.wos[i];
    for (int i = tid; i < 4 * R; i += T)
        if (S.st[i]) I.stats[i] += S.st[i];
    if (tid == 0) {
        I.ctr->sweeps = sweeps;
        I.ctr->n_ex = n_ex;
        I.ctr->n_prop = n_prop;
    }
}

// Launches whose instances all have packed rows: the register cap lets seven blocks of 128
// threads share an SM (the shared-memory limit of the 8x8 multiplier) where the uncapped
// kernel fits four.
template <bool GIBBS>
__global__ void __maxnreg__(72) graph_kernel_packed(const GraphInst* __restrict__ insts, RunArgs a,
                                                    int with_pool) {
    graph_body<1, GIBBS>(insts, a, with_pool);
}

template <bool GIBBS>
__global__ void __launch_bounds__(512) graph_kernel(const GraphInst* __restrict__ insts, RunArgs a,
                                                    int with_pool) {
    graph_body<0, GIBBS>(insts, a, with_pool);
}

// Random initial state: walker w's spin at a free site is bit (w & 31) of output word 0 of
// Philox(site, 0, w >> 5, id); clamped sites take their clamp value.
__global__ void graph_init_kernel(const GraphInst* __restrict__ insts, uint64_t seed) {
    const GraphInst& I = insts[blockIdx.x];
    const int8_t* cl = I.clamp;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int idx = threadIdx.x; idx < I.N * I.Rp; idx += blockDim.x) {
        const int i = idx / I.Rp, w = idx - i * I.Rp;
        int8_t s = -1;
        if (w < I.R) {
            if (cl[i] != 0) {
                s = cl[i];
            } else {
                const uint4 r = philox(make_uint4((uint32_t)i, 0u, (kDomInit << 24) | (uint32_t)(w >> 5),
                                                  I.iid), k0, k1);
                s = ((r.x >> (w & 31)) & 1u) ? 1 : -1;
            }
        }
        I.spins[idx] = (int8_t)(s < 0);
    }
}

__global__ void graph_capture_kernel(const GraphInst* __restrict__ dst,
                                     const GraphInst* __restrict__ src, int entry) {
    const GraphInst& D = dst[blockIdx.x];
    const GraphInst& Sr = src[blockIdx.x];
    const int N = Sr.N, NW = Sr.NW;
    for (int idx = threadIdx.x; idx < Sr.R * NW; idx += blockDim.x) {
        const int r = idx / NW, k = idx - r * NW;
        const int w = Sr.wos[r];
        uint32_t word = 0;
        for (int b = 0; b < 32; ++b) {
            const int i = k * 32 + b;
            if (i < N && Sr.spins[i * Sr.Rp + w] == 0) word |= 1u << b;
        }
        const_cast<uint32_t*>(D.pool)[(size_t)entry * D.pstride + (size_t)r * NW + k] = word;
    }
}

__global__ void graph_read_kernel(const GraphInst* __restrict__ insts, int inst, int8_t* out) {
    const GraphInst& I = insts[inst];
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < I.R * I.N;
         idx += gridDim.x * blockDim.x) {
        const int r = idx / I.N, i = idx - r * I.N;
        out[idx] = (int8_t)(1 - 2 * I.spins[i * I.Rp + I.wos[r]]);
    }
}

__global__ void graph_write_kernel(const GraphInst* __restrict__ insts, int inst,
                                   const int8_t* in, const int32_t* walker) {
    const GraphInst& I = insts[inst];
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < I.R * I.N;
         idx += gridDim.x * blockDim.x) {
        const int r = idx / I.N, i = idx - r * I.N;
        I.spins[i * I.Rp + walker[r]] = (int8_t)(in[idx] < 0);
    }
}

cudaError_t configure_graph_kernels(int smem) {
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(graph_kernel_packed<true>, at, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(graph_kernel_packed<false>, at, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(graph_kernel<true>, at, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(graph_kernel<false>, at, smem);
    return e;
}

// packed_only: every instance of d_insts has packed rows; gibbs: the Gibbs rule (else
// Metropolis)
cudaError_t launch_graph(const GraphInst* d_insts, int n, int threads, size_t smem,
                         const RunArgs& a, int with_pool, bool packed_only, bool gibbs,
                         cudaStream_t stream) {
    if (packed_only && gibbs) graph_kernel_packed<true><<<n, threads, smem, stream>>>(d_insts, a, with_pool);
    else if (packed_only) graph_kernel_packed<false><<<n, threads, smem, stream>>>(d_insts, a, with_pool);
    else if (gibbs) graph_kernel<true><<<n, threads, smem, stream>>>(d_insts, a, with_pool);
    else graph_kernel<false><<<n, threads, smem, stream>>>(d_insts, a, with_pool);
    return cudaGetLastError();
}
cudaError_t launch_graph_init(const GraphInst* d, int n, uint64_t seed, cudaStream_t s) {
    graph_init_kernel<<<n, 256, 0, s>>>(d, seed);
    return cudaGetLastError();
}
cudaError_t launch_graph_capture(const GraphInst* dst, const GraphInst* src, int n, int entry,
                                 cudaStream_t s) {
    graph_capture_kernel<<<n, 256, 0, s>>>(dst, src, entry);
    return cudaGetLastError();
}
cudaError_t launch_graph_read(const GraphInst* d, int inst, int8_t* out, int total, cudaStream_t s) {
    graph_read_kernel<<<(total + 255) / 256, 256, 0, s>>>(d, inst, out);
    return cudaGetLastError();
}
cudaError_t launch_graph_write(const GraphInst* d, int inst, const int8_t* in, const int32_t* walker,
                               int total, cudaStream_t s) {
    graph_write_kernel<<<(total + 255) / 256, 256, 0, s>>>(d, inst, in, walker);
    return cudaGetLastError();
}

}  // namespace pt
