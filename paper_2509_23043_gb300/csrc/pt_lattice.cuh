// Lattice engine: parallel tempering with global proposals (Algorithm 1 of arXiv 2509.23043)
// on periodic L^3 Edwards-Anderson +-J instances with Metropolis or Gibbs local moves.
//
// Layout. The R replicas of an instance are "walkers" packed 32 per uint32 word: word
// [wb][site] holds spin `site` of walkers 32*wb .. 32*wb+31, bit b set iff spin = +1. A
// walker keeps its lane for the whole run; replica exchange permutes the slot <-> walker
// labels (sow / wos) instead of moving spins, which gives the same chain as swapping
// configurations (Eq. 1) since the random numbers of a local move are keyed by the walker.
//
// Local move (Methods: local sweeps). Shared memory holds every spin word next to its
// complement, and the table points a neighbour across a negative bond at the complement, so
// the word read is n_d ^ Jneg_d and the bond d of every walker is unsatisfied iff s differs
// from it; the bit-sliced count c of unsatisfied bonds (0..6) gives dE = 12 - 4c and the local
// field I = s (6 - 2c).
//  - Metropolis: c >= 3 always flips; c = 0, 1, 2 flips iff u < T(beta_slot, dE).
//  - Gibbs (Eq. 5): the new spin is +1 iff u < T_G(beta_slot, I), I = 6 - 2q with the class
//    q = c where s = +1 and 6 - c where s = -1; a mux tree picks the class's threshold plane.
// The comparison runs MSB first over bit planes: plane k of the 32 walkers' u is one Philox
// output word, so planes are only drawn while some walker is still undecided (the result is
// the full 32-bit u < T comparison).
//
// Energy (Algorithm 1, the energy step of a cycle). E = 2 U - 3N with U the number of unsatisfied
// bonds. Every bond joins a site to a neighbour of a lower colour exactly once, so U is
// counted, from scratch, in the last sweep of a cycle: each site of colour c > 0 counts its
// bonds to lower-colour neighbours right after its update (its lower neighbours are final).
// Counts are kept as bit-sliced vertical counters and reduced across each warp by bit
// transposes and popcounts.
//
// Per cycle the block synchronises four times: after each colour class, after the energy
// counts, and after the exchange. Warp 0 decides the exchange pairs, commits the new labels
// and rebuilds the bit-sliced threshold planes while the other warps wait.
#pragma once
#include "pt_device.cuh"
#include "pt_layout.h"

namespace pt {

// KB: vertical counter bits (a template parameter): a thread's count of unsatisfied bonds
// per walker, over its words of the last colour class, must stay below 2^KB.

// Scalars of the instance held in registers for the whole launch.
struct LP {
    uint32_t iid;
    int L, N, R, W, NW, ncol;
    int cb[4];    // colour class c occupies positions cb[c] .. cb[c+1]-1
};

__device__ __forceinline__ LP load_lp(const LatInst& I) {
    LP p;
    p.iid = I.iid; p.L = I.L; p.N = I.N; p.R = I.R; p.W = I.W; p.NW = I.NW; p.ncol = I.ncol;
#pragma unroll
    for (int c = 0; c < 4; ++c) p.cb[c] = I.col_off[c];
    return p;
}

struct LatSmem {
    uint4* tw;         // [W*32] bit-sliced thresholds {T4, T8, T12} per plane (Metropolis), or
                       // [W*32][2] {T(q = 0..3)}, {T(q = 4..6)} (Gibbs)
    uint2* spins;      // [W*N] {spin word, its complement}, colour-major
    uint4* itab;       // [N]
    double* beta;      // [R]
    double* dbeta;     // [R] beta[r+1] - beta[r] in FP64 (0 for the last slot)
    float* fbeta;      // [R] (float) beta[r]
    float* fdbeta;     // [R] (float) dbeta[r]
    uint4* thr;        // [R] {T(4), T(8), T(12), 0}, or [R][2] {T_G(6 - 2q), q = 0..6, 0}
    uint8_t* prop;     // [R]
    uint32_t* ebits;   // [6*NW]   (with pool)
    uint32_t* stage;   // [R*NW]   proposal staging (with pool)
    int32_t* us;       // [R]      unsatisfied-bond counts of the staged proposals
    int32_t* cursor;   // [R]
    int16_t* accr;     // [W*32]   slot whose proposal the walker accepted, -1 none
    int32_t* E;        // [W*32]
    int32_t* Eacc;     // [2][W*32] double-buffered bond counts
    uint32_t* st;      // [4][R]   statistics of this launch
    int16_t* sow;      // [2][W*32] slot of walker, double-buffered
    int16_t* wos;      // [2][W*32] walker of slot, double-buffered
    // contextual proposals only: spins and tw hold one more block (the scratch lanes)
    uint32_t* cm;      // [N]  lanes whose site is kept in this event
    int16_t* cslot;    // [32] slot of scratch lane j (the enabled slots in order)
    int32_t* ccnt;     // [32] bond counts of the scratch lanes
    int32_t* cmisc;    // [2]  number of enabled slots, mask of accepted lanes
};

// GSP: the spins are the instance's global working copy and the table is read in place
template <bool GSP>
__device__ __forceinline__ LatSmem carve_lattice(uint8_t* base, const LatInst& I, int nwarps,
                                                 bool with_pool, bool with_ctx, bool gibbs) {
    const LatLayout l = lattice_layout(I.W, I.N, I.NW, I.R, nwarps, with_pool, with_ctx, gibbs, GSP);
    LatSmem S;
    S.tw = reinterpret_cast<uint4*>(base + l.tw);
    if constexpr (GSP) {
        S.spins = I.gspins;
        S.itab = const_cast<uint4*>(I.itab);
    } else {
        S.spins = reinterpret_cast<uint2*>(base + l.spins);
        S.itab = reinterpret_cast<uint4*>(base + l.itab);
    }
    S.beta = reinterpret_cast<double*>(base + l.beta);
    S.dbeta = reinterpret_cast<double*>(base + l.dbeta);
    S.fbeta = reinterpret_cast<float*>(base + l.fbeta);
    S.fdbeta = reinterpret_cast<float*>(base + l.fdbeta);
    S.thr = reinterpret_cast<uint4*>(base + l.thr);
    S.prop = reinterpret_cast<uint8_t*>(base + l.prop);
    S.ebits = reinterpret_cast<uint32_t*>(base + l.ebits);
    S.stage = reinterpret_cast<uint32_t*>(base + l.stage);
    S.us = reinterpret_cast<int32_t*>(base + l.us);
    S.cursor = reinterpret_cast<int32_t*>(base + l.cursor);
    S.accr = reinterpret_cast<int16_t*>(base + l.accr);
    S.E = reinterpret_cast<int32_t*>(base + l.E);
    S.Eacc = reinterpret_cast<int32_t*>(base + l.Eacc);
    S.st = reinterpret_cast<uint32_t*>(base + l.st);
    S.sow = reinterpret_cast<int16_t*>(base + l.sow);
    S.wos = reinterpret_cast<int16_t*>(base + l.wos);
    S.cm = reinterpret_cast<uint32_t*>(base + l.cm);
    S.cslot = reinterpret_cast<int16_t*>(base + l.cslot);
    S.ccnt = reinterpret_cast<int32_t*>(base + l.ccnt);
    S.cmisc = reinterpret_cast<int32_t*>(base + l.cmisc);
    return S;
}

// Bit-sliced thresholds of every walker block from a slot-of-walker map, by one warp:
// tw[wb*32 + k] = {plane k of T(dE=4), of T(dE=8), of T(dE=12)} over the walkers 32 wb + b.
// Lane b holds its walker's three thresholds; a 32x32 bit transpose of each (bit 31-k of
// lane b -> bit b of lane k) gives the planes, lane k storing plane k.
// Gibbs: the seven thresholds of each walker the same way, as two uint4 per plane.
template <bool GIBBS>
__device__ __forceinline__ void rebuild_planes_warp(const LP& P, LatSmem& S, const int16_t* sow) {
    const int lane = threadIdx.x & 31;
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    for (int wb = 0; wb < P.W; ++wb) {
        const int w = wb * 32 + lane;
        const int slot = (w < P.R) ? sow[w] : -1;
        if constexpr (GIBBS) {
            const uint4 ta = slot >= 0 ? S.thr[2 * slot] : zero;
            const uint4 tb = slot >= 0 ? S.thr[2 * slot + 1] : zero;
            const uint32_t x0 = warp_transpose32(__brev(ta.x), lane);
            const uint32_t x1 = warp_transpose32(__brev(ta.y), lane);
            const uint32_t x2 = warp_transpose32(__brev(ta.z), lane);
            const uint32_t x3 = warp_transpose32(__brev(ta.w), lane);
            const uint32_t x4 = warp_transpose32(__brev(tb.x), lane);
            const uint32_t x5 = warp_transpose32(__brev(tb.y), lane);
            const uint32_t x6 = warp_transpose32(__brev(tb.z), lane);
            S.tw[2 * (wb * 32 + lane)] = make_uint4(x0, x1, x2, x3);
            S.tw[2 * (wb * 32 + lane) + 1] = make_uint4(x4, x5, x6, 0u);
        } else {
            const uint4 t = slot >= 0 ? S.thr[slot] : zero;
            // plane k is bit 31-k: reverse the bits so that the transpose puts plane k in lane k
            const uint32_t x = warp_transpose32(__brev(t.x), lane);
            const uint32_t y = warp_transpose32(__brev(t.y), lane);
            const uint32_t z = warp_transpose32(__brev(t.z), lane);
            S.tw[wb * 32 + lane] = make_uint4(x, y, z, 0u);
        }
    }
}

// Add the 3-bit per-walker value (n2 n1 n0) to a bit-sliced counter.
template <int KB>
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

// Compare four bit planes of u (one Philox output) with the class-selected thresholds.
__device__ __forceinline__ void compare4(const uint4& r, const uint4* tw, uint32_t b0, uint32_t b1,
                                         uint32_t& und, uint32_t& lt) {
    const uint32_t rw[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint4 tt = tw[j];
        // count 0 -> T(dE=12), 1 -> T(8), 2 -> T(4)
        const uint32_t tk = mux(b1, tt.x, mux(b0, tt.y, tt.z));
        lt |= und & ~rw[j] & tk;
        und &= ~(rw[j] ^ tk);
    }
}

// Gibbs: compare four bit planes of u with the thresholds of the walkers' classes q (3 bits
// q0 q1 q2, 0..6), each plane's threshold picked from the seven threshold planes by a mux
// tree. The four planes are compared as one chain: a walker undecided before the block is
// decided "u < T" within it iff g0 | e0 (g1 | e1 (g2 | e2 g3)), with g = ~r & t (u's bit is 0
// where T's is 1) and e = ~(r ^ t) (the bits agree), and stays undecided iff all four e are 1.
// Each step of the chain is one three-input function of (r, t, h), so a block costs 4 + 4 + 1
// logic operations against 3 per plane compared one at a time. Planes are taken from the least
// significant up.
__device__ __forceinline__ uint32_t gibbs_pick(const uint4* tw, int j, uint32_t q0, uint32_t q1,
                                               uint32_t q2) {
    const uint4 ta = tw[2 * j], tb = tw[2 * j + 1];
    const uint32_t a01 = mux(q0, ta.y, ta.x), a23 = mux(q0, ta.w, ta.z);
    const uint32_t a45 = mux(q0, tb.y, tb.x);
    const uint32_t a03 = mux(q1, a23, a01), a46 = mux(q1, tb.z, a45);
    return mux(q2, a46, a03);
}
__device__ __forceinline__ void chain_step(uint32_t r, uint32_t t, uint32_t& h, uint32_t& e) {
    h = (~r & t) | (~(r ^ t) & h);
    e = e & ~(r ^ t);
}
__device__ __forceinline__ void compare4g(const uint4& r, const uint4* tw, uint32_t q0,
                                          uint32_t q1, uint32_t q2, uint32_t& und, uint32_t& lt) {
    const uint32_t t3 = gibbs_pick(tw, 3, q0, q1, q2);
    uint32_t h = ~r.w & t3, e = und & ~(r.w ^ t3);
    chain_step(r.z, gibbs_pick(tw, 2, q0, q1, q2), h, e);
    chain_step(r.y, gibbs_pick(tw, 1, q0, q1, q2), h, e);
    chain_step(r.x, gibbs_pick(tw, 0, q0, q1, q2), h, e);
    lt |= und & h;
    und = e;
}

__device__ __forceinline__ uint32_t nb_word(const uint8_t* base, uint32_t off) {
    return *reinterpret_cast<const uint32_t*>(base + off);
}

// Count of unsatisfied bonds of a site word s, bit-sliced (b2 b1 b0), from the six words
// m_d = n_d ^ Jneg_d its table entry points at (16-bit byte offsets). With u_d = s ^ m_d the
// first adder stage over (u0, u1, u2) has sum s ^ X1 and carry s ^ M1, X1 and M1 being the
// parity and majority of (m0, m1, m2) (a majority commutes with complementing all inputs), so
// s enters only where the two halves meet.
__device__ __forceinline__ void bond_count(const uint8_t* sp, const uint4& it, uint32_t s,
                                           uint32_t (&m)[6], uint32_t& b0, uint32_t& b1,
                                           uint32_t& b2) {
    m[0] = nb_word(sp, it.y & 0xFFFFu);
    m[1] = nb_word(sp, it.y >> 16);
    m[2] = nb_word(sp, it.z & 0xFFFFu);
    m[3] = nb_word(sp, it.z >> 16);
    m[4] = nb_word(sp, it.w & 0xFFFFu);
    m[5] = nb_word(sp, it.w >> 16);
    const uint32_t X1 = m[0] ^ m[1] ^ m[2], M1 = maj3(m[0], m[1], m[2]);
    const uint32_t X2 = m[3] ^ m[4] ^ m[5], M2 = maj3(m[3], m[4], m[5]);
    const uint32_t t = (s ^ X1) & (s ^ X2);        // carry of the two sum bits
    const uint32_t e = M1 ^ M2;                    // the two carries differ
    b0 = X1 ^ X2;
    b1 = e ^ t;
    b2 = mux(e, t, s ^ M1);                        // majority of (s^M1, s^M2, t)
}

// Energy bookkeeping of one updated word: add its new count of unsatisfied bonds to
// lower-colour neighbours to the thread's vertical counter.
template <int KB>
__device__ __forceinline__ void count_lower_bonds(uint32_t (&cnt)[KB], uint32_t flags,
                                                  const uint32_t (&m)[6], uint32_t s_new,
                                                  uint32_t b0, uint32_t b1, uint32_t b2,
                                                  uint32_t flip) {
    uint32_t n0, n1, n2;
    if (flags & 64u) {
        // all six neighbours are lower: the new count is 6 - c where flipped
        n0 = b0;
        n1 = b1 ^ (flip & ~b0);
        n2 = b2 ^ (flip & ~(b1 & b0));
    } else {
        uint32_t v[6];
#pragma unroll
        for (int dir = 0; dir < 6; ++dir)
            v[dir] = (s_new ^ m[dir]) & (0u - ((flags >> dir) & 1u));
        const uint32_t e1 = v[0] ^ v[1] ^ v[2], f1 = maj3(v[0], v[1], v[2]);
        const uint32_t e2 = v[3] ^ v[4] ^ v[5], f2 = maj3(v[3], v[4], v[5]);
        n0 = e1 ^ e2;
        const uint32_t g = e1 & e2;
        n1 = f1 ^ f2 ^ g;
        n2 = maj3(f1, f2, g);
    }
    vc_add3(cnt, n0, n1, n2);
}

// Plane blocks 3..7 of one word, drawn while some walker is undecided (rarely needed), then
// the new word: Gibbs, the comparison bits themselves; Metropolis, the flips.
template <bool GIBBS>
__device__ __forceinline__ uint32_t finish_word(const RunArgs& a, const LP& P, const uint4* tw,
                                                uint32_t site, uint32_t sweep_idx, uint32_t ctr2,
                                                uint32_t s, uint32_t b0, uint32_t c1, uint32_t c2,
                                                uint32_t always, uint32_t vmask, uint32_t und,
                                                uint32_t lt) {
    for (uint32_t qb = 3; qb < 8 && und; ++qb) {
        const uint4 r = philox_rk(make_uint4(site, sweep_idx, ctr2 | (qb << 16), P.iid), a);
        if constexpr (GIBBS) compare4g(r, tw + 8 * qb, b0, c1, c2, und, lt);
        else compare4(r, tw + 4 * qb, b0, c1, und, lt);
    }
    return GIBBS ? (s ^ lt) & vmask : (always | lt) & vmask;
}

// One sweep: colour classes in order, all (site, walker-block) words of a class in parallel.
template <int MAXW, int KB, bool GIBBS>
__device__ __forceinline__ void lattice_sweep(const LP& P, LatSmem& S, const RunArgs& a,
                                              uint32_t sweep_idx, bool flip_on, bool energy_on,
                                              uint32_t (&cnt)[MAXW][KB]) {
    const int tid = threadIdx.x, T = blockDim.x;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (c >= P.ncol) break;
        const int base = P.cb[c];
        const int nc = P.cb[c + 1] - base;
        const bool acc = energy_on && c > 0;
#pragma unroll
        for (int wb = 0; wb < MAXW; ++wb) {
            if (wb >= P.W) break;
            const uint8_t* sp = reinterpret_cast<const uint8_t*>(S.spins + wb * P.N);
            uint2* own_p = S.spins + wb * P.N + base;
            const int rem = P.R - wb * 32;
            const uint32_t vmask = rem >= 32 ? kFull : ((1u << rem) - 1u);
            const uint32_t ctr2 = (kDomPlane << 24) | (uint32_t)wb;
            const uint4* tw = S.tw + wb * 32 * (GIBBS ? 2 : 1);
            for (int k = tid; k < nc; k += T) {
                const uint4 it = S.itab[base + k];
                const uint32_t s = own_p[k].x;
                uint32_t m[6], b0, b1, b2;
                bond_count(sp, it, s, m, b0, b1, b2);
                uint32_t flip = 0;
                if (flip_on) {
                    uint32_t c1, c2 = 0, always = 0, und;
                    if (GIBBS) {
                        // class q: c where s = +1, 6 - c where s = -1 (q0 = c0 either way)
                        c1 = mux(s, b1, ~(b1 ^ b0));
                        c2 = mux(s, b2, ~(b2 | (b1 & b0)));
                        und = vmask;
                    } else {
                        always = b2 | (b1 & b0);              // count >= 3: dE <= 0
                        c1 = b1;
                        und = ~always & vmask;
                    }
                    uint32_t lt = 0;
                    const uint32_t site = it.x & 0xFFFFu;
                    if (und) {
                        // plane blocks 0-2 are almost always needed by some walker of the
                        // warp: drawn together (three independent Philox chains)
                        uint4 r[3];
#pragma unroll
                        for (int b = 0; b < 3; ++b)
                            r[b] = philox_rk(make_uint4(site, sweep_idx, ctr2 | ((uint32_t)b << 16), P.iid), a);
#pragma unroll
                        for (int b = 0; b < 3; ++b) {
                            if constexpr (GIBBS) compare4g(r[b], tw + 8 * b, b0, c1, c2, und, lt);
                            else compare4(r[b], tw + 4 * b, b0, c1, und, lt);
                        }
                    }
                    flip = und ? finish_word<GIBBS>(a, P, tw, site, sweep_idx, ctr2, s, b0, c1, c2, always,
                                                    vmask, und, lt)
                               : (GIBBS ? (s ^ lt) & vmask : (always | lt) & vmask);
                    if (flip) own_p[k] = make_uint2(s ^ flip, ~(s ^ flip));
                }
                if (acc) count_lower_bonds(cnt[wb], it.x >> 16, m, s ^ flip, b0, b1, b2, flip);
            }
        }
        __syncthreads();
    }
}

// Reduce the vertical counters into the bond counts Eacc[p] (per walker); ends synchronised.
// The KB transposes of a walker block are independent and run interleaved.
template <int MAXW, int KB>
__device__ __forceinline__ void lattice_count_reduce(const LP& P, LatSmem& S,
                                                     uint32_t (&cnt)[MAXW][KB], int p) {
    const int lane = threadIdx.x & 31;
    int32_t* acc_out = S.Eacc + p * P.W * 32;
#pragma unroll
    for (int wb = 0; wb < MAXW; ++wb) {
        if (wb >= P.W) break;
        uint32_t tx[KB];
#pragma unroll
        for (int j = 0; j < KB; ++j) tx[j] = warp_transpose32(cnt[wb][j], lane);
        uint32_t acc = 0;
#pragma unroll
        for (int j = 0; j < KB; ++j) {
            acc += (uint32_t)__popc(tx[j]) << j;
            cnt[wb][j] = 0u;
        }
        if (acc) atomicAdd(&acc_out[wb * 32 + lane], (int)acc);
    }
    __syncthreads();
}

// E[w] = 2U - 3N from the counts of buffer p; zero the other buffer for the next cycle.
__device__ __forceinline__ void lattice_store_energies(const LP& P, LatSmem& S, int p) {
    for (int w = threadIdx.x; w < P.W * 32; w += blockDim.x) {
        S.E[w] = 2 * S.Eacc[p * P.W * 32 + w] - 3 * P.N;
        S.Eacc[(p ^ 1) * P.W * 32 + w] = 0;
    }
}

// One exchange event (Eq. 1) on the labels of buffer q with energies E = 2 Ecount - 3N
// (Ecount != nullptr) or S.E: warp 0 decides every pair, writes the new labels to buffer q^1
// and the statistics, and rebuilds the threshold planes from the new slot-of-walker map.
// The caller synchronises afterwards.
template <bool GIBBS>
__device__ void lattice_exchange(const LP& P, LatSmem& S, const RunArgs& a, long long n_ex,
                                 int q, const int32_t* Ecount) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int R = P.R, WR = P.W * 32;
    int16_t* wos_n = S.wos + (q ^ 1) * WR;
    int16_t* sow_n = S.sow + (q ^ 1) * WR;
    if (warp == 0) {
        const int16_t* wos = S.wos + q * WR;
        const int16_t* sow = S.sow + q * WR;
        for (int r = lane; r < R; r += 32) wos_n[r] = wos[r];
        for (int w = lane; w < WR; w += 32) sow_n[w] = sow[w];
        __syncwarp();
        const int first = (n_ex & 1) ? 0 : 1;
        for (int r = first + 2 * lane; r + 1 < R; r += 64) {
            const int wa = wos[r], wc = wos[r + 1];
            const int ea = Ecount ? 2 * Ecount[wa] - 3 * P.N : S.E[wa];
            const int ec = Ecount ? 2 * Ecount[wc] - 3 * P.N : S.E[wc];
            const int dE = ec - ea;
            bool acc = dE >= 0 || S.dbeta[r] == 0.0;
            if (!acc) {
                const uint4 u = philox_rk(make_uint4((uint32_t)r, (uint32_t)n_ex, kDomExch << 24, P.iid), a);
                acc = accept_ratio(S.dbeta[r], S.fdbeta[r], dE, u.x);
            }
            S.st[R + r] += 1u;
            if (acc) {
                S.st[r] += 1u;
                wos_n[r] = (int16_t)wc;
                wos_n[r + 1] = (int16_t)wa;
                sow_n[wa] = (int16_t)(r + 1);
                sow_n[wc] = (int16_t)r;
            }
        }
        __syncwarp();
        rebuild_planes_warp<GIBBS>(P, S, sow_n);
    }
}

// Copy the next pool entry of every proposal-enabled slot into the staging buffer with
// cp.async, at the start of a cycle that ends with a proposal event: the cursors only move at
// events, so the entries are known a cycle ahead and the copy overlaps the sweeps (the pools
// live in device memory, so this hides a DRAM round trip). Each thread waits for its own
// copies in lattice_propose; the barrier there publishes them.
__device__ __forceinline__ void stage_proposals_async(const LatInst& I, LatSmem& S) {
    const int NW = I.NW, R = I.R;
    for (int idx = threadIdx.x; idx < R * NW; idx += blockDim.x) {
        const int r = idx / NW, k = idx - r * NW;
        if (S.prop[r])
            cp_async4(S.stage + idx, I.pool + (size_t)S.cursor[r] * I.pstride + (size_t)r * NW + k);
    }
    cp_async_commit();
}

// One proposal event (Algorithm 1, Eq. 2) with energies in S.E and labels of buffer q.
// `staged`: the entries were prefetched by stage_proposals_async.
// A: stage the next pool entry of every proposal-enabled slot; B: count its unsatisfied
// bonds (funnel shifts along x, y, z with the wrap masks; E^T = 2U - 3N); C: one thread per
// slot decides in FP64 and advances the cursor; D: merge accepted entries into their walkers'
// lanes 32 sites at a time by a warp bit transpose. Ends synchronised.
static __device__ void lattice_propose(const LatInst& I, LatSmem& S, const RunArgs& a,
                                       long long n_prop, int q, bool staged) {
    const int tid = threadIdx.x, T = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nwarps = T >> 5;
    const int L = I.L, N = I.N, NW = I.NW, R = I.R, WR = I.W * 32;
    const int16_t* wos = S.wos + q * WR;
    if (staged) {
        cp_async_wait_all();
    } else {
        for (int idx = tid; idx < R * NW; idx += T) {
            const int r = idx / NW, k = idx - r * NW;
            if (S.prop[r])
                S.stage[idx] = __ldg(I.pool + (size_t)S.cursor[r] * I.pstride + (size_t)r * NW + k);
        }
    }
    for (int r = tid; r < R; r += T) S.us[r] = 0;
    for (int w = tid; w < WR; w += T) S.accr[w] = -1;
    __syncthreads();
    const int st[3] = {1, L, L * L};
    const int total = R * NW;
    for (int base = warp * 32; base < total; base += T) {
        const int idx = base + lane;
        int r = -1, cnt = 0;
        if (idx < total) {
            r = idx / NW;
            const int k = idx - r * NW;
            if (S.prop[r]) {
                const uint32_t* sb = S.stage + r * NW;
                const uint32_t vk = (k < NW - 1 || (N & 31) == 0) ? kFull : ((1u << (N & 31)) - 1u);
                const uint32_t sk = sb[k];
#pragma unroll
                for (int dd = 0; dd < 3; ++dd) {
                    const uint32_t Wd = S.ebits[(3 + dd) * NW + k];
                    const uint32_t A = bits_at(sb, NW, 32 * k + st[dd]);
                    const uint32_t B = Wd ? bits_at(sb, NW, 32 * k + st[dd] - L * st[dd]) : 0u;
                    const uint32_t nb = (A & ~Wd) | (B & Wd);
                    cnt += __popc((sk ^ nb ^ S.ebits[dd * NW + k]) & vk);
                }
            }
        }
        const uint32_t m = __match_any_sync(kFull, r);
        const int v = __reduce_add_sync(m, cnt);
        if (r >= 0 && lane == __ffs(m) - 1 && v) atomicAdd(&S.us[r], v);
    }
    __syncthreads();
    if (a.prule == 2) {
        // the independent Metropolis-Hastings move (Supplementary S2): one warp per slot sums
        // the Hastings correction log q(x_r) - log q(x^T) over the sites, lane 0 decides
        for (int r = warp; r < R; r += nwarps) {
            if (!S.prop[r]) continue;
            const int w = wos[r];
            const uint2* sw = S.spins + (w >> 5) * N;
            const uint32_t bit = (uint32_t)(w & 31);
            const long long* lw = I.lw + (size_t)r * N;
            const uint32_t* sb = S.stage + r * NW;
            long long d = 0;
            for (int i = lane; i < N; i += 32) {
                const long long wi = __ldg(lw + i);
                if ((sw[I.pos[i]].x >> bit) & 1u) d += wi;
                if ((sb[i >> 5] >> (i & 31)) & 1u) d -= wi;
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) d += __shfl_xor_sync(kFull, d, o);
            if (lane == 0) {
                const int ET = 2 * S.us[r] - 3 * N;
                const uint4 u = philox_rk(make_uint4((uint32_t)r, (uint32_t)n_prop, kDomProp << 24, I.iid), a);
                if (accept_fp64(mh_exponent(S.beta[r], S.E[w] - ET, d), u.x)) {
                    S.E[w] = ET;
                    S.accr[w] = (int16_t)r;
                    S.st[2 * R + r] += 1u;
                }
                S.cursor[r] = (S.cursor[r] + 1) % I.P;
                S.st[3 * R + r] += 1u;
            }
        }
    } else {
        for (int r = tid; r < R; r += T) {
            if (!S.prop[r]) continue;
            const int w = wos[r];
            const int ET = 2 * S.us[r] - 3 * N;
            const int dE = S.E[w] - ET;                   // x = beta_r (E_r - E^T)
            bool acc = a.prule == 1 || dE >= 0 || S.beta[r] == 0.0;
            if (!acc) {
                const uint4 u = philox_rk(make_uint4((uint32_t)r, (uint32_t)n_prop, kDomProp << 24, I.iid), a);
                acc = accept_ratio(S.beta[r], S.fbeta[r], dE, u.x);
            }
            if (acc) {
                S.E[w] = ET;
                S.accr[w] = (int16_t)r;
                S.st[2 * R + r] += 1u;
            }
            S.cursor[r] = (S.cursor[r] + 1) % I.P;
            S.st[3 * R + r] += 1u;
        }
    }
    __syncthreads();
    for (int wb = 0; wb < I.W; ++wb) {
        const int w = wb * 32 + lane;
        const int r = (w < R) ? S.accr[w] : -1;
        const uint32_t am = __ballot_sync(kFull, r >= 0);
        if (!am) continue;
        uint2* sp = S.spins + wb * N;
        for (int g = warp; g < NW; g += nwarps) {
            const uint32_t row = r >= 0 ? S.stage[r * NW + g] : 0u;
            const uint32_t col = warp_transpose32(row, lane);
            const int site = 32 * g + lane;
            if (site < N) {
                const int ps = I.pos[site];
                const uint32_t v = (col & am) | (sp[ps].x & ~am);
                sp[ps] = make_uint2(v, ~v);
            }
        }
    }
    __syncthreads();
}

// Threshold planes of the scratch lanes: lane j takes the thresholds of slot cslot[j]; lanes
// beyond the enabled slots get zero thresholds (they are masked out anyway). One warp.
__device__ __forceinline__ void build_context_planes(const LP& P, LatSmem& S) {
    const int lane = threadIdx.x & 31;
    const int slot = lane < S.cmisc[0] ? S.cslot[lane] : -1;
    const uint4 t = slot >= 0 ? S.thr[slot] : make_uint4(0u, 0u, 0u, 0u);
    const uint32_t x = warp_transpose32(__brev(t.x), lane);
    const uint32_t y = warp_transpose32(__brev(t.y), lane);
    const uint32_t z = warp_transpose32(__brev(t.z), lane);
    S.tw[P.W * 32 + lane] = make_uint4(x, y, z, 0u);
}

// One contextual proposal event (Supplementary S3) for every enabled slot at once, with
// energies in S.E and labels of buffer q. Scratch lane j carries the proposal of the j-th
// enabled slot:
//  A: copy each slot's configuration into its lane and draw the kept sites (lane j keeps a
//     site iff bits j of Philox words 0 .. ctx_log2-1 of (site, event, 5 << 24 | 0xFF << 16)
//     are set);
//  B: ctx_sweeps Metropolis sweeps of the scratch block at each lane's slot temperature,
//     kept sites frozen: the walkers' word update with a per-word lane mask, uniforms from the
//     bit planes of Philox(site, (event - 1) ctx_sweeps + k, 5 << 24 | plane block << 16);
//     the last sweep counts the lanes' unsatisfied bonds (E^T = 2U - 3N);
//  C: one thread per enabled slot decides (the uniform as for pool proposals);
//  D: accepted lanes are copied bit by bit into their walkers. Ends synchronised.
template <int KB>
__device__ void lattice_context_propose(const LP& P, LatSmem& S, const RunArgs& a,
                                        long long n_prop, int q) {
    const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31;
    const int N = P.N, W = P.W, WR = W * 32, R = P.R;
    const int16_t* wos = S.wos + q * WR;
    const int nen = S.cmisc[0];
    const uint32_t lanes = nen >= 32 ? kFull : ((1u << nen) - 1u);
    uint2* scr = S.spins + W * N;
    const uint8_t* scr_b = reinterpret_cast<const uint8_t*>(scr);
    // A
    for (int p = tid; p < N; p += T) {
        uint32_t word = 0;
        for (int j = 0; j < nen; ++j) {
            const int w = wos[S.cslot[j]];
            word |= ((S.spins[(w >> 5) * N + p].x >> (w & 31)) & 1u) << j;
        }
        scr[p] = make_uint2(word, ~word);
        const uint32_t site = S.itab[p].x & 0xFFFFu;
        const uint4 r = philox_rk(make_uint4(site, (uint32_t)n_prop, (kDomCtx << 24) | (0xFFu << 16),
                                             P.iid), a);
        uint32_t kept = r.x;
        if (a.ctx_log2 >= 2) kept &= r.y;
        if (a.ctx_log2 >= 3) kept &= r.z;
        S.cm[p] = kept;
    }
    if (tid == 0) S.cmisc[1] = 0;
    __syncthreads();
    // B
    uint32_t cnt[KB];
#pragma unroll
    for (int j = 0; j < KB; ++j) cnt[j] = 0u;
    const uint4* tw = S.tw + W * 32;
    for (int k = 0; k < a.ctx_sweeps; ++k) {
        const uint32_t t = (uint32_t)((n_prop - 1) * a.ctx_sweeps + k);
        const bool last = k == a.ctx_sweeps - 1;
        for (int c = 0; c < P.ncol; ++c) {
            const int base = P.cb[c];
            const int nc = P.cb[c + 1] - base;
            for (int kk = tid; kk < nc; kk += T) {
                const int pp = base + kk;
                const uint4 it = S.itab[pp];
                const uint32_t s = scr[pp].x;
                uint32_t m[6], b0, b1, b2;
                bond_count(scr_b, it, s, m, b0, b1, b2);
                const uint32_t movable = lanes & ~S.cm[pp];
                const uint32_t always = b2 | (b1 & b0);    // count >= 3: dE <= 0
                uint32_t und = ~always & movable, lt = 0;
                const uint32_t site = it.x & 0xFFFFu;
                for (uint32_t qb = 0; qb < 8 && und; ++qb) {
                    const uint4 r = philox_rk(make_uint4(site, t, (kDomCtx << 24) | (qb << 16), P.iid), a);
                    compare4(r, tw + 4 * qb, b0, b1, und, lt);
                }
                const uint32_t flip = (always | lt) & movable;
                if (flip) scr[pp] = make_uint2(s ^ flip, ~(s ^ flip));
                if (last && c > 0) count_lower_bonds(cnt, it.x >> 16, m, s ^ flip, b0, b1, b2, flip);
            }
            __syncthreads();
        }
    }
    {
        uint32_t tx[KB];
#pragma unroll
        for (int j = 0; j < KB; ++j) tx[j] = warp_transpose32(cnt[j], lane);
        uint32_t accu = 0;
#pragma unroll
        for (int j = 0; j < KB; ++j) accu += (uint32_t)__popc(tx[j]) << j;
        if (accu) atomicAdd(&S.ccnt[lane], (int)accu);
    }
    __syncthreads();
    // C (every lane's count is cleared for the next event)
    const int cj = tid < 32 ? S.ccnt[tid] : 0;
    if (tid < 32) S.ccnt[tid] = 0;
    if (tid < nen) {
        const int j = tid, r = S.cslot[j], w = wos[r];
        const int ET = 2 * cj - 3 * N;
        const int dE = S.E[w] - ET;                   // x = beta_r (E_r - E^T)
        bool acc = a.prule == 1 || dE >= 0 || S.beta[r] == 0.0;
        if (!acc) {
            const uint4 u = philox_rk(make_uint4((uint32_t)r, (uint32_t)n_prop, kDomProp << 24, P.iid), a);
            acc = accept_ratio(S.beta[r], S.fbeta[r], dE, u.x);
        }
        S.st[3 * R + r] += 1u;
        if (acc) {
            S.st[2 * R + r] += 1u;
            S.E[w] = ET;
            atomicOr(reinterpret_cast<unsigned*>(&S.cmisc[1]), 1u << j);
        }
    }
    __syncthreads();
    // D
    const uint32_t am = (uint32_t)S.cmisc[1];
    if (am) {
        for (int i = tid; i < W * N; i += T) {
            const int wb = i / N, p = i - wb * N;
            uint32_t word = S.spins[wb * N + p].x;
            const uint32_t src = scr[p].x;
            for (uint32_t rest = am; rest; rest &= rest - 1) {
                const int j = __ffs(rest) - 1;
                const int w = wos[S.cslot[j]];
                if ((w >> 5) != wb) continue;
                const uint32_t b = 1u << (w & 31);
                word = (word & ~b) | (((src >> j) & 1u) << (w & 31));
            }
            S.spins[wb * N + p] = make_uint2(word, ~word);
        }
    }
    __syncthreads();
}

// CTX: built with the contextual-proposal step (a separate instantiation, so the kernels
// without it keep their code and registers).
// GSP: spins and neighbour table in global memory (instances too large for shared memory;
// L2 keeps them resident), a separate instantiation so the others keep shared addressing.
template <int MAXW, int KB, bool CTX, bool GIBBS, bool GSP = false>
__global__ void __launch_bounds__(512) lattice_kernel(const LatInst* __restrict__ insts,
                                                      RunArgs a, int flags) {
    static_assert(!(CTX && GIBBS), "contextual proposals refill with Metropolis sweeps");
    static_assert(!(CTX && GSP), "contextual proposals are built for shared-memory instances");
    extern __shared__ __align__(16) uint8_t smem[];
    const LatInst& I = insts[blockIdx.x];
    if (!*I.active) return;   // a free serving slot: the whole block leaves at once
    const int nwarps = blockDim.x >> 5;
    const bool with_pool = (flags & kWithPool) != 0;
    constexpr bool with_ctx = CTX;
    LatSmem S = carve_lattice<GSP>(smem, I, nwarps, with_pool, with_ctx, GIBBS);
    const int tid = threadIdx.x, T = blockDim.x;
    const LP P = load_lp(I);
    const int N = P.N, W = P.W, R = P.R, WR = W * 32;

    // state in (spins to colour-major order)
    for (int i = tid; i < W * N; i += T) {
        const int wb = i / N, site = i - wb * N;
        const uint32_t v = I.spins[i];
        S.spins[wb * N + I.pos[site]] = make_uint2(v, ~v);
    }
    if constexpr (!GSP)
        for (int i = tid; i < N; i += T) S.itab[i] = I.itab[i];
    for (int i = tid; i < WR; i += T) {
        S.E[i] = I.E[i];
        S.Eacc[i] = 0;
        S.Eacc[WR + i] = 0;
        S.sow[i] = I.sow[i];
        S.wos[i] = i < R ? I.wos[i] : (int16_t)-1;
    }
    for (int i = tid; i < R; i += T) {
        const double b = I.beta[i];
        const double db = (i + 1 < R) ? I.beta[i + 1] - b : 0.0;
        S.beta[i] = b;
        S.dbeta[i] = db;
        S.fbeta[i] = (float)b;
        S.fdbeta[i] = (float)db;
        S.prop[i] = I.prop[i];
    }
    for (int i = tid; i < R * (GIBBS ? 2 : 1); i += T) S.thr[i] = reinterpret_cast<const uint4*>(I.thr)[i];
    for (int i = tid; i < 4 * R; i += T) S.st[i] = 0u;
    if (with_pool) {
        for (int i = tid; i < 6 * I.NW; i += T) S.ebits[i] = I.ebits[i];
        for (int i = tid; i < R; i += T) S.cursor[i] = I.cursor[i];
    }
    if (with_ctx && tid == 0) {
        int nen = 0;
        for (int r = 0; r < R; ++r)
            if (S.prop[r]) S.cslot[nen++] = (int16_t)r;
        S.cmisc[0] = nen;
    }
    if (with_ctx)
        for (int j = tid; j < 32; j += T) S.ccnt[j] = 0;
    long long sweeps = I.ctr->sweeps, n_ex = I.ctr->n_ex, n_prop = I.ctr->n_prop;
    __syncthreads();
    if (tid < 32) {
        rebuild_planes_warp<GIBBS>(P, S, S.sow);
        if constexpr (CTX) build_context_planes(P, S);
    }
    __syncthreads();

    uint32_t cnt[MAXW][KB];
#pragma unroll
    for (int wb = 0; wb < MAXW; ++wb)
#pragma unroll
        for (int j = 0; j < KB; ++j) cnt[wb][j] = 0u;
    int p = 0;   // bond-count buffer of this cycle
    int q = 0;   // label buffer holding the current slot <-> walker maps

    if (a.mode & kModeEnergy) {
        lattice_sweep<MAXW, KB, GIBBS>(P, S, a, (uint32_t)sweeps, false, true, cnt);
        lattice_count_reduce<MAXW, KB>(P, S, cnt, p);
        lattice_store_energies(P, S, p);
        p ^= 1;
        __syncthreads();
    }
    if (a.mode & kModeSweeps) {
        for (int k = 0; k < a.n; ++k) {
            lattice_sweep<MAXW, KB, GIBBS>(P, S, a, (uint32_t)sweeps, true, k == a.n - 1, cnt);
            ++sweeps;
        }
        if (a.n > 0) {
            lattice_count_reduce<MAXW, KB>(P, S, cnt, p);
            lattice_store_energies(P, S, p);
            p ^= 1;
            __syncthreads();
        }
    }
    if (a.mode & kModePropose) {
        ++n_prop;
        if constexpr (CTX) lattice_context_propose<KB>(P, S, a, n_prop, q);
        else if (with_pool) lattice_propose(I, S, a, n_prop, q, false);
    }
    if (a.mode & kModeExchange) {
        ++n_ex;
        lattice_exchange<GIBBS>(P, S, a, n_ex, q, nullptr);
        q ^= 1;
        __syncthreads();
    }
    if (a.mode & kModeCycles) {
        for (int cyc = 0; cyc < a.n; ++cyc) {
            const bool due = proposal_due(sweeps + a.M, a);
            if (!CTX && due && with_pool) stage_proposals_async(I, S);
            for (int m = 0; m < a.M; ++m) {
                lattice_sweep<MAXW, KB, GIBBS>(P, S, a, (uint32_t)sweeps, true, m == a.M - 1, cnt);
                ++sweeps;
            }
            lattice_count_reduce<MAXW, KB>(P, S, cnt, p);
            ++n_ex;
            if (due) {
                lattice_store_energies(P, S, p);
                __syncthreads();
                ++n_prop;
                if constexpr (CTX) lattice_context_propose<KB>(P, S, a, n_prop, q);
                else if (with_pool) lattice_propose(I, S, a, n_prop, q, true);
                lattice_exchange<GIBBS>(P, S, a, n_ex, q, nullptr);
            } else {
                lattice_exchange<GIBBS>(P, S, a, n_ex, q, S.Eacc + p * WR);
                lattice_store_energies(P, S, p);
            }
            p ^= 1;
            q ^= 1;
            __syncthreads();
        }
    }

    // state out (back to site order)
    for (int i = tid; i < W * N; i += T) {
        const int wb = i / N, site = i - wb * N;
        I.spins[i] = S.spins[wb * N + I.pos[site]].x;
    }
    for (int i = tid; i < WR; i += T) {
        I.E[i] = S.E[i];
        I.sow[i] = S.sow[q * WR + i];
    }
    for (int i = tid; i < R; i += T) I.wos[i] = S.wos[q * WR + i];
    for (int i = tid; i < 4 * R; i += T)
        if (S.st[i]) I.stats[i] += S.st[i];
    if (with_pool)
        for (int i = tid; i < R; i += T) I.cursor[i] = S.cursor[i];
    if (tid == 0) {
        I.ctr->sweeps = sweeps;
        I.ctr->n_ex = n_ex;
        I.ctr->n_prop = n_prop;
    }
}

}  // namespace pt
