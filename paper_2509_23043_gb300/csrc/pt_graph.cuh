// Graph engine: the per-instance descriptor and the shared-memory layout of graph_kernel,
// shared by the host (pt_api.cu) and the kernel (pt_graph.cu).
#pragma once
#include "pt_device.cuh"
#include "pt_layout.h"

namespace pt {

// Graph engine: CSR couplings, fields, clamps, Gibbs or Metropolis. Spin bytes [N][Rp], Rp = R rounded up to 8.
struct GraphInst {
    uint32_t iid;
    int32_t N, R, Rp, NW, ncol, P, NE, Imax, nfree;
    int32_t Eclamp;          // energy of the clamped spins: their fields and mutual bonds
    int32_t col_off[33];
    int8_t* spins;           // [N][Rp]: 1 where the spin is -1, 0 where it is +1
    const int8_t* clamp;     // [N]: 0 free, +-1 clamped
    const int32_t* rowp;     // [N+1] CSR row offsets (each edge seen from both ends)
    const int32_t* rowl;     // [N] a free site's row lists first its "counted" neighbours
                             // (clamped or of a lower colour), rowp[i] .. rowl[i]-1
    const int32_t* adj;      // [2 NE] neighbour index
    const int32_t* adjJ;     // [2 NE] coupling
    const int32_t* adjp;     // [2 NE] packed = (neighbour * Rp/8) << 8 | (uint8) coupling, the
                             // neighbour's row in units of eight walkers; used when `packed`
                             // (every |coupling| and every site's sum of them <= 127)
    int32_t packed;
    const int32_t* h;        // [N]
    const int2* hk;          // [N] packed rows only: {h + sum of J over the counted neighbours
                             // + 256, that + sum of J over the others}, the constants of the
                             // biased byte sums (graph_sweep)
    const int32_t* csites;   // [nfree] free sites in colour order
    // proposal energies: E = Kprop + 2 (sum_e J_e [m_a != m_b] - sum_i h_i [m_i = +1]), with
    // the edges and the sites of nonzero field in blocks of 32 of one coupling (field) value,
    // padded with the index N (a zero word)
    int32_t nEb, nHb, Kprop;     // edge blocks, field blocks, sum_i h_i - sum_e J_e
    const uint32_t* pe_ab;   // [32 nEb] a | b << 16
    const int32_t* pe_J;     // [nEb]
    const int32_t* ph_i;     // [32 nHb] site
    const int32_t* ph_h;     // [nHb]
    const uint32_t* cbits;   // [2][NW]: clamped mask, clamp value (+1) bits
    int32_t* E;              // [Rp] per walker
    int16_t* sow;            // [Rp]
    int16_t* wos;            // [R]
    const uint32_t* thr;     // [R][2*Imax+1]
    const double* beta;      // [R]
    const uint8_t* prop;     // [R]
    int32_t* cursor;         // [R]
    const uint32_t* pool;    // entry e, slot r at pool + e * pstride + r * NW
    long long pstride;
    Counters* ctr;
    unsigned long long* stats;
    const int32_t* active;   // nonzero: the instance takes part in launches
    const long long* lw;     // [R][N] proposal rule 2: log-odds of each slot's proposal law in
                             // units of 2^-32 (clamped sites 0), or nullptr
};

struct GraphLayout {
    size_t spins, thr, rowp, smeta, adj, adjJ, adjp, h, hk, E, Eacc, st, sow, wos, pbuf, pM,
        pe_ab, pe_J, ph_i, ph_h, total;
};

// The free sites in colour order as records {site, row begin, row split, row end} (smeta).
// Packed instances keep only the packed rows (adjp) and the per-site constants hk, in colour
// order beside smeta; the others only adj, adjJ and the fields h (by site). With a pool: every slot's staged proposal (bit-packed,
// [R][NW]), the same transposed to one word per site and group of 32 slots ([ceil(R/32)][N+1],
// word N zero), and the proposal-energy blocks.
PT_HD inline GraphLayout graph_layout(int N, int R, int Rp, int NE, int Imax, int nfree, int NW,
                                      bool with_pool, bool packed, int nEb, int nHb) {
    GraphLayout l;
    size_t o = 0;
    l.spins = o;  o = align16(o + (size_t)N * Rp);
    l.thr = o;    o = align16(o + (size_t)R * (2 * Imax + 1) * 4);
    l.rowp = o;   o = align16(o + (size_t)(N + 1) * 4);
    l.smeta = o;  o = align16(o + (size_t)(nfree > 0 ? nfree : 1) * 16);
    l.adj = o;    o = align16(o + (packed ? 0 : (size_t)2 * NE * 4));
    l.adjJ = o;   o = align16(o + (packed ? 0 : (size_t)2 * NE * 4));
    l.adjp = o;   o = align16(o + (packed ? (size_t)2 * NE * 4 : 0));
    l.h = o;      o = align16(o + (packed ? 0 : (size_t)N * 4));
    l.hk = o;     o = align16(o + (packed ? (size_t)(nfree > 0 ? nfree : 1) * 8 : 0));
    l.E = o;      o = align16(o + (size_t)Rp * 4);
    l.Eacc = o;   o = align16(o + (size_t)Rp * 4);
    l.st = o;     o = align16(o + (size_t)4 * R * 4);
    l.sow = o;    o = align16(o + (size_t)Rp * 2);
    l.wos = o;    o = align16(o + (size_t)R * 2);
    const size_t wp = with_pool ? 1 : 0;
    l.pbuf = o;   o = align16(o + wp * R * NW * 4);
    l.pM = o;     o = align16(o + wp * ((R + 31) / 32) * (N + 1) * 4);
    l.pe_ab = o;  o = align16(o + wp * 32 * nEb * 4);
    l.pe_J = o;   o = align16(o + wp * nEb * 4);
    l.ph_i = o;   o = align16(o + wp * 32 * nHb * 4);
    l.ph_h = o;   o = align16(o + wp * nHb * 4);
    l.total = o;
    return l;
}

}  // namespace pt
