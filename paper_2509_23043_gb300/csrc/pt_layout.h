// Shared-memory layouts of the engines' kernels; used by the host to size the launch and by
// the device to carve the buffer, so the two can never disagree.
#pragma once
#include <cstddef>
#include <cstdint>

#ifdef __CUDACC__
#define PT_HD __host__ __device__
#else
#define PT_HD
#endif

namespace pt {

PT_HD inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

struct LatLayout {
    size_t tw, spins, itab, beta, dbeta, fbeta, fdbeta, thr, prop, ebits, stage, us, cursor, accr, E, Eacc, st, sow, wos,
        cm, cslot, ccnt, cmisc, total;
};

// with_ctx (contextual proposals): one more walker block of spins and threshold planes (the
// scratch lanes), the kept-site masks and the per-lane bookkeeping. gibbs: seven thresholds
// per slot instead of three, so two uint4 per slot and per threshold plane. gsp: the spins and
// the neighbour table stay in global memory (instances too large for shared memory).
PT_HD inline LatLayout lattice_layout(int W, int N, int NW, int R, int nwarps, bool with_pool,
                                      bool with_ctx, bool gibbs, bool gsp = false) {
    LatLayout l;
    const size_t WR = (size_t)W * 32;
    const size_t WB = (size_t)W + (with_ctx ? 1 : 0);   // walker blocks held, scratch included
    const size_t TS = gibbs ? 2 : 1;                      // uint4 per plane and per slot
    size_t o = 0;
    l.tw = o;     o = align16(o + WB * 32 * 16 * TS);
    l.spins = o;  o = align16(o + (gsp ? 0 : WB * N * 8));     // word and complement
    l.itab = o;   o = align16(o + (gsp ? 0 : (size_t)N * 16));
    l.beta = o;   o = align16(o + (size_t)R * 8);
    l.dbeta = o;  o = align16(o + (size_t)R * 8);
    l.fbeta = o;  o = align16(o + (size_t)R * 4);
    l.fdbeta = o; o = align16(o + (size_t)R * 4);
    l.thr = o;    o = align16(o + (size_t)R * 16 * TS);
    l.prop = o;   o = align16(o + (size_t)R);
    l.ebits = o;  o = align16(o + (with_pool ? (size_t)6 * NW * 4 : 0));
    l.stage = o;  o = align16(o + (with_pool ? (size_t)R * NW * 4 : 0));
    l.us = o;     o = align16(o + (with_pool ? (size_t)R * 4 : 0));
    l.cursor = o; o = align16(o + (with_pool ? (size_t)R * 4 : 0));
    l.accr = o;   o = align16(o + (with_pool ? WR * 2 : 0));
    l.E = o;      o = align16(o + WR * 4);
    l.Eacc = o;   o = align16(o + 2 * WR * 4);
    l.st = o;     o = align16(o + (size_t)4 * R * 4);
    l.sow = o;    o = align16(o + 2 * WR * 2);
    l.wos = o;    o = align16(o + 2 * WR * 2);
    l.cm = o;     o = align16(o + (with_ctx ? (size_t)N * 4 : 0));
    l.cslot = o;  o = align16(o + (with_ctx ? 32 * 2 : 0));
    l.ccnt = o;   o = align16(o + (with_ctx ? 32 * 4 : 0));
    l.cmisc = o;  o = align16(o + (with_ctx ? 2 * 4 : 0));
    l.total = o;
    return l;
}

}  // namespace pt
