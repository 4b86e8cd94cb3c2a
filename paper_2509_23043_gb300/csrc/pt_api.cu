// Host side of the C ABI declared in include/pt.h: validation, per-instance layouts, graph
// colouring, FP64 threshold tables, device allocation and kernel launches. No step of the
// method's arithmetic on the spins runs here; it all runs in the kernels of pt_lattice.cu
// and pt_graph.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/pt.h"
#include "pt_device.cuh"
#include "pt_layout.h"
#include "pt_graph.cuh"

namespace pt {
cudaError_t launch_lattice(const LatInst*, int, int, int, int, size_t, const RunArgs&, int, cudaStream_t);
cudaError_t launch_lattice_init(const LatInst*, int, uint64_t, cudaStream_t);
cudaError_t launch_lattice_capture(const LatInst*, const LatInst*, int, int, cudaStream_t);
cudaError_t launch_lattice_read(const LatInst*, int, int8_t*, int, cudaStream_t);
cudaError_t launch_lattice_write(const LatInst*, int, const int8_t*, const int32_t*, int, cudaStream_t);
cudaError_t launch_graph(const GraphInst*, int, int, size_t, const RunArgs&, int, bool, bool, cudaStream_t);
cudaError_t launch_graph_init(const GraphInst*, int, uint64_t, cudaStream_t);
cudaError_t launch_graph_capture(const GraphInst*, const GraphInst*, int, int, cudaStream_t);
cudaError_t launch_graph_read(const GraphInst*, int, int8_t*, int, cudaStream_t);
cudaError_t launch_graph_write(const GraphInst*, int, const int8_t*, const int32_t*, int, cudaStream_t);
cudaError_t launch_gather_energies(const int32_t* const*, const int16_t* const*, const int32_t*,
                                   int, int32_t*, cudaStream_t);
}  // namespace pt

using namespace pt;

namespace {

thread_local std::string g_err;

pt_status fail(pt_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) return fail(PT_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// Thresholds: floor(2^32 p) capped at 2^32 - 1, p evaluated in FP64 exactly as written.
uint32_t prob_to_threshold(double p) {
    const double t = std::floor(std::ldexp(p, 32));
    if (t >= 4294967295.0) return 4294967295u;
    if (t <= 0.0) return 0u;
    return (uint32_t)t;
}
uint32_t metropolis_threshold(double beta, int dE) {
    return prob_to_threshold(std::exp(-beta * (double)dE));
}
uint32_t gibbs_threshold(double beta, int I) {
    return prob_to_threshold(0.5 * (1.0 + std::tanh(beta * (double)I)));
}

// Device arena: host image assembled chunk by chunk, then one allocation and one copy.
struct Arena {
    std::vector<uint8_t> host;
    size_t add(const void* p, size_t bytes) {
        const size_t off = (host.size() + 255) & ~size_t(255);
        host.resize(off + bytes);
        if (p && bytes) memcpy(host.data() + off, p, bytes);
        return off;
    }
    size_t zeros(size_t bytes) { return add(nullptr, bytes); }
};

// Colouring of a general graph by DSATUR (Methods, graph coloring): repeatedly colour the
// uncoloured vertex with the most distinct neighbour colours, ties to the larger number of
// distinct neighbours, then the lower index; use the smallest colour absent among its
// neighbours. Runs on the whole interaction graph.
int dsatur(int N, const std::vector<std::vector<int>>& nbr, std::vector<int>& colour) {
    colour.assign(N, -1);
    std::vector<int> deg(N);
    for (int i = 0; i < N; ++i) deg[i] = (int)nbr[i].size();
    std::vector<std::vector<char>> seen(N);
    std::vector<int> sat(N, 0);
    int ncol = 0;
    for (int step = 0; step < N; ++step) {
        int best = -1;
        for (int i = 0; i < N; ++i) {
            if (colour[i] >= 0) continue;
            if (best < 0 || sat[i] > sat[best] || (sat[i] == sat[best] && deg[i] > deg[best])) best = i;
        }
        std::vector<char> used(ncol + 1, 0);
        for (int j : nbr[best])
            if (colour[j] >= 0) used[colour[j]] = 1;
        int c = 0;
        while (c < (int)used.size() && used[c]) ++c;
        colour[best] = c;
        if (c + 1 > ncol) ncol = c + 1;
        for (int j : nbr[best]) {
            if (colour[j] >= 0) continue;
            if ((int)seen[j].size() <= c) seen[j].resize(c + 1, 0);
            if (!seen[j][c]) { seen[j][c] = 1; ++sat[j]; }
        }
    }
    return ncol;
}

// Colour classes of at most `cap` free sites, where the graph allows it. With
// k = max(ncol, ceil(nfree / cap)) colours available, repeatedly take the largest class above
// cap (the lowest colour among equals) and move its highest-index free site that has no free
// neighbour in some other class below cap, to the smallest such class (the lowest colour
// among equals); stop when no class is above cap or no site of it can move. Clamped sites are
// never updated and keep their colours. Empty colours are then dropped, the others keeping
// their order. Returns the number of colours.
int balance_colours(int N, const std::vector<std::vector<int>>& nbr, const std::vector<int8_t>& clamp,
                    std::vector<int>& col, int ncol, int cap) {
    int nfree = 0;
    for (int i = 0; i < N; ++i) nfree += clamp[i] == 0;
    const int k = std::max(ncol, (nfree + cap - 1) / cap);
    std::vector<int> size(k, 0);
    for (int i = 0; i < N; ++i)
        if (clamp[i] == 0) ++size[col[i]];
    for (;;) {
        int c = -1;
        for (int x = 0; x < k; ++x)
            if (size[x] > cap && (c < 0 || size[x] > size[c])) c = x;
        if (c < 0) break;
        bool moved = false;
        for (int i = N - 1; i >= 0 && !moved; --i) {
            if (clamp[i] != 0 || col[i] != c) continue;
            int d = -1;
            for (int y = 0; y < k; ++y) {
                if (y == c || size[y] >= cap) continue;
                bool free_of = true;
                for (int j : nbr[i])
                    if (clamp[j] == 0 && col[j] == y) { free_of = false; break; }
                if (free_of && (d < 0 || size[y] < size[d])) d = y;
            }
            if (d >= 0) {
                col[i] = d;
                --size[c];
                ++size[d];
                moved = true;
            }
        }
        if (!moved) break;
    }
    std::vector<int> used(k, 0), remap(k, -1);
    for (int i = 0; i < N; ++i) used[col[i]] = 1;
    int n = 0;
    for (int x = 0; x < k; ++x)
        if (used[x]) remap[x] = n++;
    for (int i = 0; i < N; ++i) col[i] = remap[col[i]];
    return n;
}

int lattice_colour(int n, int L) {
    const int x = n % L, y = (n / L) % L, z = n / (L * L);
    if (L % 2 == 0) return (x + y + z) % 2;
    const int cx = (x == L - 1) ? 2 : x % 2, cy = (y == L - 1) ? 2 : y % 2, cz = (z == L - 1) ? 2 : z % 2;
    return (cx + cy + cz) % 3;
}

}  // namespace

// A group: instances of one size class, launched together with one block shape on one
// stream; the groups of a context run concurrently.
struct Group {
    std::vector<int> members;
    int T = 128;
    size_t smem = 0;
    int maxW = 1;
    int maxitems = 0;          // largest (colour class x walker blocks) of a member
    bool packed_only = false;  // graph engine: every member has packed rows
    bool gsp = false;          // lattice engine: the members' spins and tables in global memory
    void* d_insts = nullptr;   // LatInst[] or GraphInst[] of the members
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
};

// Arena offsets of one lattice instance's arrays (for slot replacement).
struct LatOff { size_t spins, itab, pos, E, sow, wos, thr, beta, prop, cur, eb, ctr, st, active, lw, gsp; };

struct pt_ctx {
    int engine = 0;           // 0 lattice, 1 graph
    int n = 0;
    pt_config cfg{};
    cudaStream_t stream = nullptr;
    int with_pool = 0;
    int with_ctx = 0;         // contextual proposals (lattice engine)
    int NWmax = 0;
    int uniformN = -1;        // N when all instances share it, else -1
    int optin = 0;            // device limit on dynamic shared memory per block
    int sms = 0;              // streaming multiprocessors of the device
    int device = -1;          // the device current at creation; every call must run with it
    std::vector<int> N, R, W, NW, Rp, L;
    std::vector<size_t> slab_off;  // words, instance offset inside one pool entry
    size_t slab = 0;               // words per pool entry (all instances, all slots)
    uint8_t* arena = nullptr;
    size_t arena_bytes = 0;
    uint32_t* pool = nullptr;
    std::vector<LatInst> lat;
    std::vector<GraphInst> gr;
    std::vector<LatOff> loff;
    std::vector<int> group_of;     // group index of each instance
    std::vector<Group> groups;
    cudaEvent_t fork = nullptr;
    LatInst* d_lat = nullptr;
    GraphInst* d_gr = nullptr;
    int32_t* d_eoff = nullptr;          // [n] offsets of each instance in the energy output
    int32_t** d_Eptr = nullptr;         // [n] per-instance E pointers
    int16_t** d_wosptr = nullptr;       // [n] per-instance wos pointers
    int32_t* d_eout = nullptr;          // [sum R] gather buffer
    int totalR = 0;
    std::vector<int> eoff;
    // CUDA graph of pt_run_cycles_graph (one cycle count at a time)
    cudaStream_t gstream = nullptr;
    cudaEvent_t gev_in = nullptr, gev_out = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int gcycles = -1;
};

namespace pt {
cudaError_t configure_lattice_kernels(int smem);
cudaError_t configure_graph_kernels(int smem);
}  // namespace pt

namespace {

// NVTX range over an entry point, so that a profiler's timeline shows the library's calls
// (header-only NVTX v3: without an attached tool a push and pop cost a few nanoseconds).
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

RunArgs make_args(const pt_ctx* c, int mode, int nn) {
    RunArgs a{};
    a.seed = c->cfg.seed;
    a.mode = mode;
    a.n = nn;
    a.M = c->cfg.sweeps_per_cycle;
    a.every = c->cfg.propose_every;
    a.start = c->cfg.propose_start;
    a.stop = c->cfg.propose_stop;
    a.update = c->cfg.update;
    a.prule = c->cfg.proposal_rule;
    a.ctx_log2 = c->cfg.context_log2;
    a.ctx_sweeps = c->cfg.context_sweeps;
    // Philox round keys: key bumped by the Weyl constants before each round after the first
    uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
    for (int i = 0; i < 10; ++i) {
        a.rk0[i] = k0;
        a.rk1[i] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return a;
}

cudaError_t launch_group(const pt_ctx* c, const Group& g, const void* d_insts, int count,
                         const RunArgs& a, cudaStream_t s) {
    if (c->engine == 0) {
        // a thread's bond count per walker: at most 6 per word it updates in the colour
        // classes that count (the last one for even L, the last two for odd L)
        const int per_thread = (g.maxitems / std::max(g.maxW, 1) + g.T - 1) / g.T;
        const int counting = (c->L[g.members[0]] % 2 == 0) ? 1 : 2;
        const int kb4 = 6 * per_thread * counting < 16 ? 1 : 0;
        const int flags = (c->with_pool ? kWithPool : 0) | (c->with_ctx ? kWithContext : 0) |
                          (c->cfg.update == 1 ? kGibbs : 0) | (g.gsp ? kGlobalSpins : 0);
        return launch_lattice(static_cast<const LatInst*>(d_insts), count, g.maxW, kb4, g.T, g.smem, a,
                              flags, s);
    }
    return launch_graph(static_cast<const GraphInst*>(d_insts), count, g.T, g.smem, a, c->with_pool,
                        g.packed_only, c->cfg.update == 1, s);
}

// Launch one kernel per group on stream s; with several groups they fork from s onto their
// own streams and join back, so they run concurrently (also inside a stream capture).
pt_status launch_on(pt_ctx* c, int mode, int nn, cudaStream_t s) {
    const RunArgs a = make_args(c, mode, nn);
    cudaError_t e = cudaSuccess;
    if (c->groups.size() == 1) {
        const Group& g = c->groups[0];
        e = launch_group(c, g, g.d_insts, (int)g.members.size(), a, s);
    } else {
        e = cudaEventRecord(c->fork, s);
        for (size_t k = 0; e == cudaSuccess && k < c->groups.size(); ++k) {
            const Group& g = c->groups[k];
            e = cudaStreamWaitEvent(g.stream, c->fork, 0);
            if (e == cudaSuccess) e = launch_group(c, g, g.d_insts, (int)g.members.size(), a, g.stream);
            if (e == cudaSuccess) e = cudaEventRecord(g.done, g.stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, g.done, 0);
        }
    }
    if (e != cudaSuccess) return fail(PT_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
    return PT_OK;
}

pt_status launch_run(pt_ctx* c, int mode, int nn) { return launch_on(c, mode, nn, c->stream); }

// One instance alone (initial energies of a replaced slot).
pt_status launch_one(pt_ctx* c, int inst, int mode) {
    const Group& g = c->groups[c->group_of[inst]];
    const void* d = c->engine == 0 ? static_cast<const void*>(c->d_lat + inst)
                                   : static_cast<const void*>(c->d_gr + inst);
    cudaError_t e = launch_group(c, g, d, 1, make_args(c, mode, 0), c->stream);
    if (e != cudaSuccess) return fail(PT_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
    return PT_OK;
}

void drop_graph(pt_ctx* c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    c->gcycles = -1;
}

// The bit-packed lattice engine takes +-1 lattices without field or clamps (either rule).
bool is_lattice_desc(const pt_instance_desc& d) {
    if (d.lattice_L <= 0) return false;
    if (d.h)
        for (int i = 0; i < d.n_spins; ++i)
            if (d.h[i] != 0) return false;
    if (d.clamp)
        for (int i = 0; i < d.n_spins; ++i)
            if (d.clamp[i] != 0) return false;
    for (int e = 0; e < d.n_edges; ++e)
        if (d.edge_J[e] != 1 && d.edge_J[e] != -1) return false;
    return true;
}

pt_status validate(const pt_instance_desc& d, int k) {
    if (d.n_spins <= 0) return fail(PT_EINVAL, "instance %d: n_spins must be > 0", k);
    if (d.n_replicas < 1 || d.n_replicas > 128)
        return fail(PT_EINVAL, "instance %d: n_replicas must be in [1, 128]", k);
    if (!d.beta) return fail(PT_EINVAL, "instance %d: beta is NULL", k);
    for (int r = 0; r < d.n_replicas; ++r) {
        if (!std::isfinite(d.beta[r]) || d.beta[r] < 0.0)
            return fail(PT_EINVAL, "instance %d: beta[%d] must be finite and >= 0", k, r);
        if (r > 0 && !(d.beta[r - 1] <= d.beta[r]))
            return fail(PT_EINVAL, "instance %d: beta must be ascending (hot -> cold)", k);
    }
    if (d.n_edges < 0 || (d.n_edges > 0 && (!d.edge_i || !d.edge_j || !d.edge_J)))
        return fail(PT_EINVAL, "instance %d: bad edge arrays", k);
    for (int e = 0; e < d.n_edges; ++e) {
        if (d.edge_i[e] < 0 || d.edge_i[e] >= d.n_spins || d.edge_j[e] < 0 || d.edge_j[e] >= d.n_spins)
            return fail(PT_EINVAL, "instance %d: edge %d out of range", k, e);
        if (d.edge_i[e] == d.edge_j[e]) return fail(PT_EINVAL, "instance %d: self loop at edge %d", k, e);
    }
    if (d.clamp)
        for (int i = 0; i < d.n_spins; ++i)
            if (d.clamp[i] < -1 || d.clamp[i] > 1)
                return fail(PT_EINVAL, "instance %d: clamp values must be -1, 0 or +1", k);
    if (d.lattice_L > 0) {
        const long long L = d.lattice_L;
        if (L < 2 || L * L * L != d.n_spins)
            return fail(PT_EINVAL, "instance %d: lattice_L must be >= 2 with n_spins = L^3", k);
        if (d.n_edges != 3 * d.n_spins)
            return fail(PT_EINVAL, "instance %d: a lattice needs its 3N bonds", k);
        for (int n = 0; n < d.n_spins; ++n) {
            const int x = n % (int)L, y = (n / (int)L) % (int)L, z = n / (int)(L * L);
            const int nb[3] = {(int)(((x + 1) % L) + L * (y + L * z)), (int)(x + L * (((y + 1) % L) + L * z)),
                               (int)(x + L * (y + L * ((z + 1) % L)))};
            for (int dd = 0; dd < 3; ++dd)
                if (d.edge_i[3 * n + dd] != n || d.edge_j[3 * n + dd] != nb[dd])
                    return fail(PT_EINVAL, "instance %d: lattice bonds not in canonical order (site %d)", k, n);
        }
    }
    return PT_OK;
}

// -------------------------------------------------------------------------------- lattice
// Host image of one lattice instance: colouring, per-site table, bond bit strings,
// thresholds and initial labels.
struct LatHost {
    int L, N, R, W, NW, ncol;
    int col_off[4];
    std::vector<uint32_t> itab, eb, thr;
    std::vector<uint16_t> pos;
    std::vector<int16_t> sow, wos;
    std::vector<uint8_t> prop;
    int maxitems = 0;
};

pt_status lattice_host(const pt_instance_desc& d, LatHost& h, int k, bool gibbs) {
    const int L = d.lattice_L, N = d.n_spins, R = d.n_replicas, W = (R + 31) / 32, NW = (N + 31) / 32;
    if (N > 8192) return fail(PT_ENOTSUP, "instance %d: lattice engine supports N <= 8192 (L <= 20)", k);
    h.L = L; h.N = N; h.R = R; h.W = W; h.NW = NW;
    h.ncol = (L % 2 == 0) ? 2 : 3;
    std::vector<int> col(N);
    for (int i = 0; i < N; ++i) col[i] = lattice_colour(i, L);
    h.eb.assign(6 * (size_t)NW, 0u);
    h.itab.clear();
    h.itab.reserve(4 * (size_t)N);
    const int L2 = L * L;
    // colour-major position of every site (the shared-memory order of the spins)
    h.pos.assign(N, 0);
    {
        int p = 0;
        for (int cc = 0; cc < h.ncol; ++cc)
            for (int i = 0; i < N; ++i)
                if (col[i] == cc) h.pos[i] = (uint16_t)p++;
    }
    h.col_off[0] = 0;
    int filled = 0;
    h.maxitems = 0;
    for (int cc = 0; cc < h.ncol; ++cc) {
        for (int i = 0; i < N; ++i) {
            if (col[i] != cc) continue;
            const int x = i % L, y = (i / L) % L, z = i / L2;
            const int xm = (x + L - 1) % L, ym = (y + L - 1) % L, zm = (z + L - 1) % L;
            const int nbr[6] = {(x + 1) % L + L * (y + L * z), xm + L * (y + L * z),
                                x + L * ((y + 1) % L + L * z), x + L * (ym + L * z),
                                x + L * (y + L * ((z + 1) % L)), x + L * (y + L * zm)};
            // the +d bond of i is edge 3i+d; its -d bond is the +d bond of nbr[2d+1]
            const int Jv[6] = {d.edge_J[3 * i + 0], d.edge_J[3 * nbr[1] + 0], d.edge_J[3 * i + 1],
                               d.edge_J[3 * nbr[3] + 1], d.edge_J[3 * i + 2], d.edge_J[3 * nbr[5] + 2]};
            uint32_t flags = 0;
            int nlow = 0;
            uint32_t e16[6];
            for (int dir = 0; dir < 6; ++dir) {
                if (col[nbr[dir]] < cc) { flags |= 1u << dir; ++nlow; }
                // byte offset of the neighbour's word, or of its complement across a -1 bond
                e16[dir] = (uint32_t)(8 * h.pos[nbr[dir]]) + (Jv[dir] < 0 ? 4u : 0u);
            }
            if (nlow == 6) flags |= 64u;
            h.itab.push_back((uint32_t)i | (flags << 16));
            h.itab.push_back(e16[0] | (e16[1] << 16));
            h.itab.push_back(e16[2] | (e16[3] << 16));
            h.itab.push_back(e16[4] | (e16[5] << 16));
            ++filled;
        }
        h.col_off[cc + 1] = filled;
        h.maxitems = std::max(h.maxitems, (h.col_off[cc + 1] - h.col_off[cc]) * W);
    }
    for (int cc = h.ncol + 1; cc < 4; ++cc) h.col_off[cc] = filled;
    // bit strings of the bonds (for proposal energies): negative +d bonds, wraps
    for (int i = 0; i < N; ++i) {
        const int x = i % L, y = (i / L) % L, z = i / L2;
        const bool wrap[3] = {x == L - 1, y == L - 1, z == L - 1};
        for (int dd = 0; dd < 3; ++dd) {
            if (d.edge_J[3 * i + dd] < 0) h.eb[(size_t)dd * NW + (i >> 5)] |= 1u << (i & 31);
            if (wrap[dd]) h.eb[(size_t)(3 + dd) * NW + (i >> 5)] |= 1u << (i & 31);
        }
    }
    if (gibbs) {
        // class q = 0..6 has the local field I = 6 - 2q (Methods, Eq. 5)
        h.thr.assign(8 * (size_t)R, 0u);
        for (int r = 0; r < R; ++r)
            for (int q = 0; q < 7; ++q) h.thr[8 * r + q] = gibbs_threshold(d.beta[r], 6 - 2 * q);
    } else {
        h.thr.assign(4 * (size_t)R, 0u);
        for (int r = 0; r < R; ++r) {
            h.thr[4 * r + 0] = metropolis_threshold(d.beta[r], 4);
            h.thr[4 * r + 1] = metropolis_threshold(d.beta[r], 8);
            h.thr[4 * r + 2] = metropolis_threshold(d.beta[r], 12);
        }
    }
    h.sow.assign(W * 32, -1);
    h.wos.assign(R, 0);
    for (int r = 0; r < R; ++r) { h.sow[r] = (int16_t)r; h.wos[r] = (int16_t)r; }
    h.prop.assign(R, 0);
    if (d.prop_enabled)
        for (int r = 0; r < R; ++r) h.prop[r] = d.prop_enabled[r] ? 1 : 0;
    return PT_OK;
}

void lattice_fill_inst(LatInst& I, const LatHost& h, uint32_t iid, int P) {
    I.iid = iid; I.L = h.L; I.N = h.N; I.R = h.R; I.W = h.W; I.NW = h.NW; I.ncol = h.ncol; I.P = P;
    for (int cc = 0; cc < 4; ++cc) I.col_off[cc] = h.col_off[cc];
}

// Block shape of a lattice group, unless threads_per_block fixes it: about two words per
// thread per colour class, so that two blocks share an SM; or, when the context holds at most
// half as many instances as the device has SMs (the SMs are not all busy anyway), about one
// word per thread, which shortens each cycle. Capped at 512 threads (and the words per thread
// at 42, the width of the energy counters).
int lattice_auto_threads(int maxitems, bool few) {
    int T = ((maxitems / (few ? 1 : 2) + 31) / 32) * 32;
    return std::max(64, std::min(512, T));
}

pt_status lattice_group_shape(pt_ctx* c, Group& g, int T) {
    if (T % 32 != 0 || T < 32 || T > 512)
        return fail(PT_EINVAL, "lattice engine: threads_per_block must be a multiple of 32 in [32, 512]");
    if ((g.maxitems + T - 1) / T > 42)
        return fail(PT_ENOTSUP, "too many words per thread (%d); raise threads_per_block", (g.maxitems + T - 1) / T);
    size_t smem = 0;
    for (int k : g.members) {
        const LatLayout l = lattice_layout(c->W[k], c->N[k], c->NW[k], c->R[k], T / 32, c->with_pool != 0,
                                           c->with_ctx != 0, c->cfg.update == 1, g.gsp);
        smem = std::max(smem, l.total);
    }
    if (smem > (size_t)c->optin)
        return fail(PT_ENOTSUP, "instance needs %zu B of shared memory (> %d)", smem, c->optin);
    g.T = T;
    g.smem = smem;
    return PT_OK;
}

pt_status build_lattice(pt_ctx* c, const pt_instance_desc* descs) {
    Arena A;
    const int n = c->n;
    c->lat.resize(n);
    c->loff.resize(n);
    std::vector<int> maxitems(n);
    c->with_pool = c->cfg.pool_size > 0 ? 1 : 0;
    c->with_ctx = c->cfg.proposal_source == 1 ? 1 : 0;
    for (int k = 0; k < n; ++k) {
        const pt_instance_desc& d = descs[k];
        LatHost h;
        pt_status st = lattice_host(d, h, k, c->cfg.update == 1);
        if (st != PT_OK) return st;
        c->N[k] = h.N; c->R[k] = h.R; c->W[k] = h.W; c->NW[k] = h.NW; c->Rp[k] = h.W * 32; c->L[k] = h.L;
        maxitems[k] = h.maxitems;
        LatInst& I = c->lat[k];
        memset(&I, 0, sizeof I);
        lattice_fill_inst(I, h, d.instance_id, c->cfg.pool_size);
        LatOff& o = c->loff[k];
        const int32_t one = 1;
        o.spins = A.zeros((size_t)h.W * h.N * 4);
        o.itab = A.add(h.itab.data(), h.itab.size() * 4);
        o.pos = A.add(h.pos.data(), h.pos.size() * 2);
        o.E = A.zeros((size_t)h.W * 32 * 4);
        o.sow = A.add(h.sow.data(), h.sow.size() * 2);
        o.wos = A.add(h.wos.data(), h.wos.size() * 2);
        o.thr = A.add(h.thr.data(), h.thr.size() * 4);
        o.beta = A.add(d.beta, (size_t)h.R * 8);
        o.prop = A.add(h.prop.data(), h.prop.size());
        o.cur = A.zeros((size_t)h.R * 4);
        o.eb = A.add(h.eb.data(), h.eb.size() * 4);
        o.ctr = A.zeros(sizeof(Counters));
        o.st = A.zeros((size_t)4 * h.R * 8);
        o.active = A.add(&one, 4);
        o.lw = c->cfg.proposal_rule == 2 ? A.zeros((size_t)h.R * h.N * 8) : 0;
        // spins and table too large for shared memory: a global working copy of the
        // {word, complement} spins (the kernel reads the table in place)
        const bool gsp = lattice_layout(h.W, h.N, h.NW, h.R, 1, c->with_pool != 0, c->with_ctx != 0,
                                        c->cfg.update == 1).total > (size_t)c->optin;
        if (gsp && c->with_ctx)
            return fail(PT_ENOTSUP, "instance %d: contextual proposals need the instance's spins in "
                                    "shared memory (at most %d bytes)", k, c->optin);
        o.gsp = gsp ? A.zeros((size_t)h.W * h.N * 8) : 0;
        c->slab_off[k] = c->slab;
        c->slab += (size_t)h.R * h.NW;
        c->NWmax = std::max(c->NWmax, h.NW);
    }
    // groups: one per (walker blocks, L)
    c->group_of.assign(n, -1);
    for (int k = 0; k < n; ++k) {
        int gk = -1;
        for (size_t g = 0; g < c->groups.size(); ++g) {
            const int m = c->groups[g].members[0];
            if (c->W[m] == c->W[k] && c->L[m] == c->L[k] && (c->loff[m].gsp != 0) == (c->loff[k].gsp != 0)) {
                gk = (int)g;
                break;
            }
        }
        if (gk < 0) {
            c->groups.emplace_back();
            gk = (int)c->groups.size() - 1;
            c->groups[gk].gsp = c->loff[k].gsp != 0;
        }
        c->groups[gk].members.push_back(k);
        c->group_of[k] = gk;
    }
    for (Group& g : c->groups) {
        for (int k : g.members) {
            g.maxitems = std::max(g.maxitems, maxitems[k]);
            g.maxW = std::max(g.maxW, c->W[k]);
        }
        if (g.maxW > 2) g.maxW = 4;
        const int T = c->cfg.threads_per_block > 0 ? c->cfg.threads_per_block
                                                    : lattice_auto_threads(g.maxitems, 2 * c->n <= c->sms);
        pt_status st = lattice_group_shape(c, g, T);
        if (st != PT_OK) return st;
    }
    CK(configure_lattice_kernels(c->optin));
    c->arena_bytes = A.host.size();
    CK(cudaMallocAsync((void**)&c->arena, A.host.size(), c->stream));
    CK(cudaMemcpyAsync(c->arena, A.host.data(), A.host.size(), cudaMemcpyHostToDevice, c->stream));
    if (c->with_pool) {
        const size_t words = c->slab * (size_t)c->cfg.pool_size;
        CK(cudaMallocAsync((void**)&c->pool, words * 4, c->stream));
        CK(cudaMemsetAsync(c->pool, 0, words * 4, c->stream));
    }
    uint8_t* b = c->arena;
    for (int k = 0; k < n; ++k) {
        LatInst& I = c->lat[k];
        const LatOff& o = c->loff[k];
        I.spins = (uint32_t*)(b + o.spins);
        I.gspins = o.gsp ? (uint2*)(b + o.gsp) : nullptr;
        I.itab = (const uint4*)(b + o.itab);
        I.pos = (const uint16_t*)(b + o.pos);
        I.E = (int32_t*)(b + o.E);
        I.sow = (int16_t*)(b + o.sow);
        I.wos = (int16_t*)(b + o.wos);
        I.thr = (const uint32_t*)(b + o.thr);
        I.beta = (const double*)(b + o.beta);
        I.prop = (const uint8_t*)(b + o.prop);
        I.cursor = (int32_t*)(b + o.cur);
        I.ebits = (const uint32_t*)(b + o.eb);
        I.ctr = (Counters*)(b + o.ctr);
        I.stats = (unsigned long long*)(b + o.st);
        I.active = (const int32_t*)(b + o.active);
        I.lw = c->cfg.proposal_rule == 2 ? (const long long*)(b + o.lw) : nullptr;
        I.pool = c->pool ? c->pool + c->slab_off[k] : nullptr;
        I.pstride = (long long)c->slab;
    }
    CK(cudaMallocAsync((void**)&c->d_lat, sizeof(LatInst) * n, c->stream));
    CK(cudaMemcpyAsync(c->d_lat, c->lat.data(), sizeof(LatInst) * n, cudaMemcpyHostToDevice, c->stream));
    for (Group& g : c->groups) {
        std::vector<LatInst> m;
        for (int k : g.members) m.push_back(c->lat[k]);
        CK(cudaMallocAsync(&g.d_insts, sizeof(LatInst) * m.size(), c->stream));
        CK(cudaMemcpyAsync(g.d_insts, m.data(), sizeof(LatInst) * m.size(), cudaMemcpyHostToDevice, c->stream));
    }
    cudaError_t e = launch_lattice_init(c->d_lat, n, c->cfg.seed, c->stream);
    if (e != cudaSuccess) return fail(PT_ECUDA, "init: %s", cudaGetErrorString(e));
    CK(cudaStreamSynchronize(c->stream));   // host images above must outlive their copies
    return PT_OK;
}

// -------------------------------------------------------------------------------- graph
pt_status build_graph(pt_ctx* c, const pt_instance_desc* descs) {
    Arena A;
    const int n = c->n;
    struct Off { size_t spins, clamp, rowp, rowl, adj, adjJ, adjp, h, hk, cs, pe_ab, pe_J, ph_i, ph_h, cb, E, sow, wos, thr, beta, prop, cur, ctr, st, active, lw; };
    std::vector<Off> o(n);
    c->gr.resize(n);
    size_t maxsmem = 0;
    int T = c->cfg.threads_per_block > 0 ? c->cfg.threads_per_block : 128;
    if (T % 32 != 0 || T < 32 || T > 512) return fail(PT_EINVAL, "graph engine: threads_per_block must be a multiple of 32 in [32, 512]");
    c->with_pool = c->cfg.pool_size > 0 ? 1 : 0;
    for (int k = 0; k < n; ++k) {
        const pt_instance_desc& d = descs[k];
        const int N = d.n_spins, R = d.n_replicas, Rp = (R + 7) & ~7, NW = (N + 31) / 32, NE = d.n_edges;
        if (N > 65535) return fail(PT_ENOTSUP, "instance %d: graph engine supports N <= 65535", k);
        c->N[k] = N; c->R[k] = R; c->W[k] = (R + 31) / 32; c->NW[k] = NW; c->Rp[k] = Rp;
        GraphInst& I = c->gr[k];
        memset(&I, 0, sizeof I);
        I.iid = d.instance_id; I.N = N; I.R = R; I.Rp = Rp; I.NW = NW; I.NE = NE; I.P = c->cfg.pool_size;
        // CSR with both directions of every edge
        std::vector<int32_t> rowp(N + 1, 0), adj(2 * (size_t)NE), adjJ(2 * (size_t)NE), h(N, 0);
        for (int e = 0; e < NE; ++e) { rowp[d.edge_i[e] + 1]++; rowp[d.edge_j[e] + 1]++; }
        for (int i = 0; i < N; ++i) rowp[i + 1] += rowp[i];
        std::vector<int> fill(N, 0);
        for (int e = 0; e < NE; ++e) {
            const int a = d.edge_i[e], bb = d.edge_j[e];
            adj[rowp[a] + fill[a]] = bb; adjJ[rowp[a] + fill[a]] = d.edge_J[e]; fill[a]++;
            adj[rowp[bb] + fill[bb]] = a; adjJ[rowp[bb] + fill[bb]] = d.edge_J[e]; fill[bb]++;
        }
        if (d.h) for (int i = 0; i < N; ++i) h[i] = d.h[i];
        std::vector<int8_t> clamp(N, 0);
        if (d.clamp) for (int i = 0; i < N; ++i) clamp[i] = d.clamp[i];
        // largest |local field|
        long long Imax = 0;
        for (int i = 0; i < N; ++i) {
            long long s = std::llabs((long long)h[i]);
            for (int a = rowp[i]; a < rowp[i + 1]; ++a) s += std::llabs((long long)adjJ[a]);
            Imax = std::max(Imax, s);
        }
        if (Imax > 4096) return fail(PT_ENOTSUP, "instance %d: local fields up to %lld exceed 4096", k, Imax);
        I.Imax = (int)Imax;
        // colouring: lattice colouring when a lattice is given, else DSATUR
        std::vector<int> col(N);
        int ncol;
        if (d.lattice_L > 0) {
            for (int i = 0; i < N; ++i) col[i] = lattice_colour(i, d.lattice_L);
            ncol = (d.lattice_L % 2 == 0) ? 2 : 3;
        } else {
            std::vector<std::vector<int>> nbr(N);
            for (int i = 0; i < N; ++i) {
                for (int a = rowp[i]; a < rowp[i + 1]; ++a) {
                    const int j = adj[a];
                    bool dup = false;
                    for (int x : nbr[i]) if (x == j) { dup = true; break; }
                    if (!dup) nbr[i].push_back(j);
                }
            }
            ncol = dsatur(N, nbr, col);
            if (c->cfg.colour_cap > 0) ncol = balance_colours(N, nbr, clamp, col, ncol, c->cfg.colour_cap);
        }
        if (ncol > 32) return fail(PT_ENOTSUP, "instance %d: colouring needs %d > 32 colours", k, ncol);
        I.ncol = ncol;
        // Energy fused into the last sweep of a cycle: a free site counts, after its update,
        // its field and its bonds to clamped neighbours and to free neighbours of a lower
        // colour (final by then); each free-free bond is counted once, at its higher-colour
        // end. The clamped spins' own terms are the constant Eclamp.
        std::vector<int32_t> rowl(N);
        for (int i = 0; i < N; ++i) {
            int lo = rowp[i];
            if (clamp[i] == 0) {
                for (int a = rowp[i]; a < rowp[i + 1]; ++a) {
                    const int j = adj[a];
                    if (clamp[j] != 0 || col[j] < col[i]) {
                        std::swap(adj[a], adj[lo]);
                        std::swap(adjJ[a], adjJ[lo]);
                        ++lo;
                    }
                }
            }
            rowl[i] = lo;
        }
        // Packed local fields: four walkers' sums of J * [spin = -1] as bytes of one word
        // (biased by 128), valid while every site's sum of |J| is at most 127 (and the row
        // offsets, in units of eight walkers, fit 24 bits).
        bool packed = (long long)N * (Rp / 8) < (1ll << 24);
        for (int i = 0; i < N && packed; ++i) {
            int sa = 0;
            for (int a = rowp[i]; a < rowp[i + 1]; ++a) sa += std::abs(adjJ[a]);
            if (sa > 127) packed = false;
        }
        std::vector<int32_t> adjp(2 * (size_t)NE, 0);
        if (packed)
            for (size_t a = 0; a < adjp.size(); ++a)
                adjp[a] = (int32_t)(((uint32_t)adj[a] * (uint32_t)(Rp / 8)) << 8 | ((uint32_t)adjJ[a] & 0xFFu));
        I.packed = packed ? 1 : 0;
        {
            long long ec = 0;
            for (int i = 0; i < N; ++i) if (clamp[i] != 0) ec -= (long long)h[i] * clamp[i];
            for (int e = 0; e < NE; ++e)
                if (clamp[d.edge_i[e]] != 0 && clamp[d.edge_j[e]] != 0)
                    ec -= (long long)d.edge_J[e] * clamp[d.edge_i[e]] * clamp[d.edge_j[e]];
            I.Eclamp = (int32_t)ec;
        }
        // free sites colour by colour; within a colour by decreasing degree (then index), so
        // the sites one warp updates together loop over similar numbers of neighbours. Sites
        // of one colour share no edge and draw their random numbers by site index, so their
        // order does not change the result.
        std::vector<int32_t> cs;
        I.col_off[0] = 0;
        for (int cc = 0; cc < ncol; ++cc) {
            const size_t first = cs.size();
            for (int i = 0; i < N; ++i)
                if (col[i] == cc && clamp[i] == 0) cs.push_back(i);
            std::stable_sort(cs.begin() + first, cs.end(), [&](int32_t x, int32_t y) {
                return rowp[x + 1] - rowp[x] > rowp[y + 1] - rowp[y];
            });
            I.col_off[cc + 1] = (int)cs.size();
        }
        I.nfree = (int)cs.size();
        std::vector<uint32_t> cb(2 * (size_t)NW, 0u);
        for (int i = 0; i < N; ++i) {
            if (clamp[i] != 0) cb[i >> 5] |= 1u << (i & 31);
            if (clamp[i] > 0) cb[NW + (i >> 5)] |= 1u << (i & 31);
        }
        const int tw = 2 * I.Imax + 1;
        std::vector<uint32_t> thr((size_t)R * tw, 0u);
        for (int r = 0; r < R; ++r)
            for (int v = -I.Imax; v <= I.Imax; ++v)
                thr[(size_t)r * tw + v + I.Imax] = (c->cfg.update == 1)
                    ? gibbs_threshold(d.beta[r], v)
                    : (v > 0 ? metropolis_threshold(d.beta[r], 2 * v) : 0u);
        std::vector<int16_t> sow(Rp, -1), wos(R);
        for (int r = 0; r < R; ++r) { sow[r] = (int16_t)r; wos[r] = (int16_t)r; }
        std::vector<uint8_t> prop(R, 0);
        if (d.prop_enabled) for (int r = 0; r < R; ++r) prop[r] = d.prop_enabled[r] ? 1 : 0;
        o[k].spins = A.zeros((size_t)N * Rp);
        o[k].clamp = A.add(clamp.data(), N);
        o[k].rowp = A.add(rowp.data(), rowp.size() * 4);
        o[k].rowl = A.add(rowl.data(), rowl.size() * 4);
        o[k].adj = A.add(adj.data(), adj.size() * 4);
        o[k].adjJ = A.add(adjJ.data(), adjJ.size() * 4);
        o[k].adjp = A.add(adjp.data(), adjp.size() * 4);
        o[k].h = A.add(h.data(), h.size() * 4);
        {
            std::vector<int32_t> hk(2 * (size_t)N, 0);
            for (int i = 0; i < N; ++i) {
                long long sc = 0, sr = 0;
                for (int a = rowp[i]; a < rowl[i]; ++a) sc += adjJ[a];
                for (int a = rowl[i]; a < rowp[i + 1]; ++a) sr += adjJ[a];
                hk[2 * (size_t)i] = (int32_t)(h[i] + sc + 256);
                hk[2 * (size_t)i + 1] = (int32_t)(h[i] + sc + sr + 256);
            }
            o[k].hk = A.add(hk.data(), hk.size() * 4);
        }
        o[k].cs = A.add(cs.data(), std::max<size_t>(cs.size(), 1) * 4);
        // proposal-energy blocks: edges grouped by coupling, sites of nonzero field by field,
        // each group padded to a multiple of 32 with the index N
        std::vector<uint32_t> pe_ab;
        std::vector<int32_t> pe_J, ph_i, ph_h;
        {
            std::map<int32_t, std::vector<uint32_t>> byJ;
            for (int e = 0; e < NE; ++e)
                byJ[d.edge_J[e]].push_back((uint32_t)d.edge_i[e] | ((uint32_t)d.edge_j[e] << 16));
            std::map<int32_t, std::vector<int32_t>> byh;
            for (int i = 0; i < N; ++i) if (h[i] != 0) byh[h[i]].push_back(i);
            const uint32_t padab = (uint32_t)N | ((uint32_t)N << 16);
            long long K = 0;
            for (auto& [J, v] : byJ) {
                K -= (long long)J * (long long)v.size();
                v.resize((v.size() + 31) / 32 * 32, padab);
                pe_ab.insert(pe_ab.end(), v.begin(), v.end());
                pe_J.insert(pe_J.end(), v.size() / 32, J);
            }
            for (auto& [hv, v] : byh) {
                K += (long long)hv * (long long)v.size();
                v.resize((v.size() + 31) / 32 * 32, N);
                ph_i.insert(ph_i.end(), v.begin(), v.end());
                ph_h.insert(ph_h.end(), v.size() / 32, hv);
            }
            I.nEb = (int)pe_J.size();
            I.nHb = (int)ph_h.size();
            I.Kprop = (int32_t)K;
        }
        o[k].pe_ab = A.add(pe_ab.data(), std::max<size_t>(pe_ab.size(), 1) * 4);
        o[k].pe_J = A.add(pe_J.data(), std::max<size_t>(pe_J.size(), 1) * 4);
        o[k].ph_i = A.add(ph_i.data(), std::max<size_t>(ph_i.size(), 1) * 4);
        o[k].ph_h = A.add(ph_h.data(), std::max<size_t>(ph_h.size(), 1) * 4);
        o[k].cb = A.add(cb.data(), cb.size() * 4);
        o[k].E = A.zeros((size_t)Rp * 4);
        o[k].sow = A.add(sow.data(), sow.size() * 2);
        o[k].wos = A.add(wos.data(), wos.size() * 2);
        o[k].thr = A.add(thr.data(), thr.size() * 4);
        o[k].beta = A.add(d.beta, (size_t)R * 8);
        o[k].prop = A.add(prop.data(), prop.size());
        o[k].cur = A.zeros((size_t)R * 4);
        o[k].ctr = A.zeros(sizeof(Counters));
        o[k].st = A.zeros((size_t)4 * R * 8);
        const int32_t one = 1;
        o[k].active = A.add(&one, 4);
        o[k].lw = c->cfg.proposal_rule == 2 ? A.zeros((size_t)R * N * 8) : 0;
        c->slab_off[k] = c->slab;
        c->slab += (size_t)R * NW;
        c->NWmax = std::max(c->NWmax, NW);
        const GraphLayout l = graph_layout(N, R, Rp, NE, I.Imax, I.nfree, NW, c->with_pool != 0, I.packed != 0, I.nEb, I.nHb);
        maxsmem = std::max(maxsmem, l.total);
    }
    if (maxsmem > (size_t)c->optin)
        return fail(PT_ENOTSUP, "instance needs %zu B of shared memory (> %d)", maxsmem, c->optin);
    c->groups.assign(1, Group{});
    Group& grp = c->groups[0];
    grp.packed_only = true;
    for (int k = 0; k < n; ++k) {
        grp.members.push_back(k);
        grp.packed_only = grp.packed_only && c->gr[k].packed != 0;
    }
    grp.T = T;
    grp.smem = maxsmem;
    c->group_of.assign(n, 0);
    CK(configure_graph_kernels(c->optin));
    c->arena_bytes = A.host.size();
    CK(cudaMallocAsync((void**)&c->arena, A.host.size(), c->stream));
    CK(cudaMemcpyAsync(c->arena, A.host.data(), A.host.size(), cudaMemcpyHostToDevice, c->stream));
    if (c->with_pool) {
        const size_t words = c->slab * (size_t)c->cfg.pool_size;
        CK(cudaMallocAsync((void**)&c->pool, words * 4, c->stream));
        CK(cudaMemsetAsync(c->pool, 0, words * 4, c->stream));
    }
    uint8_t* b = c->arena;
    for (int k = 0; k < n; ++k) {
        GraphInst& I = c->gr[k];
        I.spins = (int8_t*)(b + o[k].spins);
        I.clamp = (const int8_t*)(b + o[k].clamp);
        I.rowp = (const int32_t*)(b + o[k].rowp);
        I.rowl = (const int32_t*)(b + o[k].rowl);
        I.adj = (const int32_t*)(b + o[k].adj);
        I.adjJ = (const int32_t*)(b + o[k].adjJ);
        I.adjp = (const int32_t*)(b + o[k].adjp);
        I.h = (const int32_t*)(b + o[k].h);
        I.hk = (const int2*)(b + o[k].hk);
        I.csites = (const int32_t*)(b + o[k].cs);
        I.pe_ab = (const uint32_t*)(b + o[k].pe_ab);
        I.pe_J = (const int32_t*)(b + o[k].pe_J);
        I.ph_i = (const int32_t*)(b + o[k].ph_i);
        I.ph_h = (const int32_t*)(b + o[k].ph_h);
        I.cbits = (const uint32_t*)(b + o[k].cb);
        I.E = (int32_t*)(b + o[k].E);
        I.sow = (int16_t*)(b + o[k].sow);
        I.wos = (int16_t*)(b + o[k].wos);
        I.thr = (const uint32_t*)(b + o[k].thr);
        I.beta = (const double*)(b + o[k].beta);
        I.prop = (const uint8_t*)(b + o[k].prop);
        I.cursor = (int32_t*)(b + o[k].cur);
        I.ctr = (Counters*)(b + o[k].ctr);
        I.stats = (unsigned long long*)(b + o[k].st);
        I.active = (const int32_t*)(b + o[k].active);
        I.lw = c->cfg.proposal_rule == 2 ? (const long long*)(b + o[k].lw) : nullptr;
        I.pool = c->pool ? c->pool + c->slab_off[k] : nullptr;
        I.pstride = (long long)c->slab;
    }
    CK(cudaMallocAsync((void**)&c->d_gr, sizeof(GraphInst) * n, c->stream));
    CK(cudaMemcpyAsync(c->d_gr, c->gr.data(), sizeof(GraphInst) * n, cudaMemcpyHostToDevice, c->stream));
    grp.d_insts = c->d_gr;   // the group is the whole batch, in instance order
    cudaError_t e = launch_graph_init(c->d_gr, n, c->cfg.seed, c->stream);
    if (e != cudaSuccess) return fail(PT_ECUDA, "init: %s", cudaGetErrorString(e));
    CK(cudaStreamSynchronize(c->stream));
    return PT_OK;
}

void release(pt_ctx* c) {
    if (!c) return;
    cudaStream_t s = c->stream;
    drop_graph(c);
    for (Group& g : c->groups) {
        if (g.d_insts && !(c->engine == 1)) cudaFreeAsync(g.d_insts, s);
        if (g.stream) cudaStreamDestroy(g.stream);
        if (g.done) cudaEventDestroy(g.done);
    }
    if (c->fork) cudaEventDestroy(c->fork);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    if (c->gev_in) cudaEventDestroy(c->gev_in);
    if (c->gev_out) cudaEventDestroy(c->gev_out);
    if (c->arena) cudaFreeAsync(c->arena, s);
    if (c->pool) cudaFreeAsync(c->pool, s);
    if (c->d_lat) cudaFreeAsync(c->d_lat, s);
    if (c->d_gr) cudaFreeAsync(c->d_gr, s);
    if (c->d_eoff) cudaFreeAsync(c->d_eoff, s);
    if (c->d_Eptr) cudaFreeAsync(c->d_Eptr, s);
    if (c->d_wosptr) cudaFreeAsync(c->d_wosptr, s);
    if (c->d_eout) cudaFreeAsync(c->d_eout, s);
    cudaStreamSynchronize(s);
    delete c;
}

// A context's memory and kernels belong to the device that was current at creation; a call
// made with another device current would launch on the wrong device.
pt_status check_ctx(const pt_ctx* c) {
    if (!c) return fail(PT_EINVAL, "ctx is NULL");
    int cur = -1;
    const cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return fail(PT_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (cur != c->device)
        return fail(PT_ESTATE, "the context was created on device %d but device %d is current; "
                    "call cudaSetDevice(%d) first", c->device, cur, c->device);
    return PT_OK;
}

pt_status check_inst(const pt_ctx* c, int inst) {
    const pt_status s = check_ctx(c);
    if (s != PT_OK) return s;
    if (inst < 0 || inst >= c->n) return fail(PT_EINVAL, "instance %d out of range [0, %d)", inst, c->n);
    return PT_OK;
}

Counters* ctr_ptr(const pt_ctx* c, int inst) {
    return c->engine == 0 ? c->lat[inst].ctr : c->gr[inst].ctr;
}
int32_t* cursor_ptr(const pt_ctx* c, int inst) {
    return c->engine == 0 ? c->lat[inst].cursor : c->gr[inst].cursor;
}

}  // namespace

extern "C" {

const char* pt_last_error(void) { return g_err.c_str(); }

// Contextual proposals hold one scratch lane per enabled slot: at most 32 per instance.
pt_status context_slots_ok(const pt_instance_desc& d, int k) {
    int nen = 0;
    if (d.prop_enabled)
        for (int r = 0; r < d.n_replicas; ++r) nen += d.prop_enabled[r] != 0;
    if (nen > 32)
        return fail(PT_ENOTSUP, "instance %d: %d proposal-enabled slots; contextual proposals take at most 32", k, nen);
    return PT_OK;
}

pt_status pt_create_instances(pt_ctx** out, const pt_instance_desc* descs, int32_t n,
                              const pt_config* cfg, void* cuda_stream) {
    const Range range("pt_create_instances");
    if (!out || !descs || !cfg) return fail(PT_EINVAL, "NULL argument");
    *out = nullptr;
    if (n < 1) return fail(PT_EINVAL, "n must be >= 1");
    if (cfg->update != 0 && cfg->update != 1) return fail(PT_EINVAL, "update must be 0 or 1");
    if (cfg->sweeps_per_cycle < 1) return fail(PT_EINVAL, "sweeps_per_cycle must be >= 1");
    if (cfg->pool_size < 0) return fail(PT_EINVAL, "pool_size must be >= 0");
    if (cfg->propose_every < 0) return fail(PT_EINVAL, "propose_every must be >= 0");
    if (cfg->proposal_rule < 0 || cfg->proposal_rule > 2)
        return fail(PT_EINVAL, "proposal_rule must be 0, 1 or 2");
    if (cfg->proposal_rule == 2 && cfg->proposal_source != 0)
        return fail(PT_EINVAL, "proposal_rule 2 needs pool proposals (proposal_source 0)");
    if (cfg->proposal_source != 0 && cfg->proposal_source != 1)
        return fail(PT_EINVAL, "proposal_source must be 0 or 1");
    if (cfg->colour_cap < 0) return fail(PT_EINVAL, "colour_cap must be >= 0");
    if (cfg->proposal_source == 1) {
        if (cfg->context_log2 < 1 || cfg->context_log2 > 3)
            return fail(PT_EINVAL, "context_log2 must be 1, 2 or 3");
        if (cfg->context_sweeps < 1) return fail(PT_EINVAL, "context_sweeps must be >= 1");
        if (cfg->update != 0)
            return fail(PT_ENOTSUP, "contextual proposals are implemented with Metropolis sweeps");
        for (int k = 0; k < n; ++k) {
            if (!is_lattice_desc(descs[k]))
                return fail(PT_ENOTSUP, "instance %d: contextual proposals are implemented for the "
                                        "lattice engine (J = +-1, no field or clamp)", k);
            pt_status s = context_slots_ok(descs[k], k);
            if (s != PT_OK) return s;
        }
    }
    for (int k = 0; k < n; ++k) {
        pt_status s = validate(descs[k], k);
        if (s != PT_OK) return s;
    }
    const bool lat0 = is_lattice_desc(descs[0]);
    for (int k = 1; k < n; ++k)
        if (is_lattice_desc(descs[k]) != lat0)
            return fail(PT_EINVAL, "instance %d: a context holds only lattice-engine or only graph-engine instances", k);
    pt_ctx* c = new (std::nothrow) pt_ctx();
    if (!c) return fail(PT_ENOMEM, "host allocation failed");
    c->engine = lat0 ? 0 : 1;
    c->n = n;
    c->cfg = *cfg;
    c->stream = (cudaStream_t)cuda_stream;
    c->N.resize(n); c->R.resize(n); c->W.resize(n); c->NW.resize(n); c->Rp.resize(n); c->L.resize(n);
    c->slab_off.resize(n);
    {
        int dev = 0;
        cudaError_t e0 = cudaGetDevice(&dev);
        c->device = dev;
        if (e0 == cudaSuccess)
            e0 = cudaDeviceGetAttribute(&c->optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e0 == cudaSuccess)
            e0 = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
        if (e0 != cudaSuccess) { release(c); return fail(PT_ECUDA, "device query: %s", cudaGetErrorString(e0)); }
    }
    for (int k = 0; k < n; ++k) c->L[k] = descs[k].lattice_L;
    pt_status s = lat0 ? build_lattice(c, descs) : build_graph(c, descs);
    if (s != PT_OK) { release(c); return s; }
    {
        cudaError_t e1 = cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming);
        for (Group& g : c->groups) {
            if (c->groups.size() > 1 && e1 == cudaSuccess) {
                e1 = cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking);
                if (e1 == cudaSuccess) e1 = cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming);
            }
        }
        if (e1 != cudaSuccess) { release(c); return fail(PT_ECUDA, "streams: %s", cudaGetErrorString(e1)); }
        s = launch_run(c, kModeEnergy, 0);   // energies of the initial state
        if (s != PT_OK) { release(c); return s; }
    }
    // energy gather tables
    c->eoff.resize(n);
    int tot = 0;
    std::vector<int32_t*> Ep(n);
    std::vector<int16_t*> Wp(n);
    for (int k = 0; k < n; ++k) {
        c->eoff[k] = tot;
        tot += c->R[k];
        Ep[k] = lat0 ? c->lat[k].E : c->gr[k].E;
        Wp[k] = lat0 ? c->lat[k].wos : c->gr[k].wos;
    }
    std::vector<int32_t> eoff_ext(c->eoff);
    eoff_ext.push_back(tot);
    c->totalR = tot;
    int uniform = c->N[0];
    for (int k = 1; k < n; ++k) if (c->N[k] != uniform) uniform = -1;
    c->uniformN = uniform;
    cudaError_t e;
    if ((e = cudaMallocAsync((void**)&c->d_eoff, (n + 1) * 4, c->stream)) != cudaSuccess ||
        (e = cudaMallocAsync((void**)&c->d_Eptr, n * sizeof(void*), c->stream)) != cudaSuccess ||
        (e = cudaMallocAsync((void**)&c->d_wosptr, n * sizeof(void*), c->stream)) != cudaSuccess ||
        (e = cudaMallocAsync((void**)&c->d_eout, (size_t)tot * 4, c->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(c->d_eoff, eoff_ext.data(), (n + 1) * 4, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(c->d_Eptr, Ep.data(), n * sizeof(void*), cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(c->d_wosptr, Wp.data(), n * sizeof(void*), cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess) {
        release(c);
        return fail(PT_ECUDA, "create: %s", cudaGetErrorString(e));
    }
    *out = c;
    return PT_OK;
}

pt_status pt_destroy(pt_ctx* ctx) {
    release(ctx);
    return PT_OK;
}

pt_status pt_set_stream(pt_ctx* ctx, void* s) {
    if (!ctx) return fail(PT_EINVAL, "ctx is NULL");
    ctx->stream = (cudaStream_t)s;
    return PT_OK;
}

pt_status pt_group_info(const pt_ctx* ctx, int32_t group, int32_t info[4]) {
    if (!ctx || !info) return fail(PT_EINVAL, "NULL argument");
    if (group < 0) { info[0] = (int32_t)ctx->groups.size(); return PT_OK; }
    if (group >= (int32_t)ctx->groups.size()) return fail(PT_EINVAL, "group %d out of range", group);
    const Group& g = ctx->groups[group];
    info[0] = (int32_t)g.members.size();
    info[1] = g.T;
    info[2] = (int32_t)g.smem;
    info[3] = g.members[0];
    return PT_OK;
}

pt_status pt_autotune(pt_ctx* ctx, int32_t probe_cycles, int32_t* threads_out) {
    const Range range("pt_autotune");
    { const pt_status cs = check_ctx(ctx); if (cs != PT_OK) return cs; }
    if (probe_cycles < 1) return fail(PT_EINVAL, "probe_cycles must be >= 1");
    drop_graph(ctx);
    uint8_t* snap = nullptr;
    CK(cudaMallocAsync((void**)&snap, ctx->arena_bytes, ctx->stream));
    CK(cudaMemcpyAsync(snap, ctx->arena, ctx->arena_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaError_t e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    pt_status st = PT_OK;
    const RunArgs a = make_args(ctx, kModeCycles, probe_cycles);
    const int cand[] = {64, 96, 128, 192, 256, 384, 512};
    for (size_t gi = 0; gi < ctx->groups.size() && e == cudaSuccess && st == PT_OK; ++gi) {
        Group& g = ctx->groups[gi];
        const Group keep = g;
        float best = 1e30f;
        int bestT = g.T;
        for (int T : cand) {
            if (ctx->engine == 1 && T > 1024) continue;
            Group trial = keep;
            if (ctx->engine == 0) {
                if (lattice_group_shape(ctx, trial, T) != PT_OK) continue;
            } else {
                const GraphInst& I0 = ctx->gr[g.members[0]];
                size_t smem = 0;
                for (int k : g.members) {
                    const GraphInst& I = ctx->gr[k];
                    const GraphLayout l = graph_layout(I.N, I.R, I.Rp, I.NE, I.Imax, I.nfree, I.NW, ctx->with_pool != 0, I.packed != 0, I.nEb, I.nHb);
                    smem = std::max(smem, l.total);
                }
                (void)I0;
                if (smem > (size_t)ctx->optin) continue;
                trial.T = T;
                trial.smem = smem;
            }
            // warm-up then timed probe, each from the snapshot
            for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
                e = cudaMemcpyAsync(ctx->arena, snap, ctx->arena_bytes, cudaMemcpyDeviceToDevice, ctx->stream);
                if (e == cudaSuccess) e = cudaEventRecord(t0, ctx->stream);
                if (e == cudaSuccess) e = launch_group(ctx, trial, trial.d_insts, (int)trial.members.size(), a, ctx->stream);
                if (e == cudaSuccess) e = cudaEventRecord(t1, ctx->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(t1);
            }
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
            if (e == cudaSuccess && ms < best) { best = ms; bestT = T; }
        }
        if (e == cudaSuccess) {
            if (ctx->engine == 0) st = lattice_group_shape(ctx, g, bestT);
            else {
                size_t smem = 0;
                for (int k : g.members) {
                    const GraphInst& I = ctx->gr[k];
                    const GraphLayout l = graph_layout(I.N, I.R, I.Rp, I.NE, I.Imax, I.nfree, I.NW, ctx->with_pool != 0, I.packed != 0, I.nEb, I.nHb);
                    smem = std::max(smem, l.total);
                }
                g.T = bestT;
                g.smem = smem;
            }
        }
        if (threads_out) threads_out[gi] = g.T;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->arena, snap, ctx->arena_bytes, cudaMemcpyDeviceToDevice, ctx->stream);
    cudaFreeAsync(snap, ctx->stream);
    cudaError_t e2 = cudaStreamSynchronize(ctx->stream);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return fail(PT_ECUDA, "autotune: %s", cudaGetErrorString(e));
    return st;
}

pt_status pt_run_cycles_graph(pt_ctx* ctx, int32_t n_cycles) {
    const Range range("pt_run_cycles_graph");
    { const pt_status cs = check_ctx(ctx); if (cs != PT_OK) return cs; }
    if (n_cycles < 1) return fail(PT_EINVAL, "n_cycles must be >= 1");
    cudaError_t e = cudaSuccess;
    if (!ctx->gstream) {
        e = cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->gev_in, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->gev_out, cudaEventDisableTiming);
        if (e != cudaSuccess) return fail(PT_ECUDA, "graph stream: %s", cudaGetErrorString(e));
    }
    if (!ctx->gexec || ctx->gcycles != n_cycles) {
        drop_graph(ctx);
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return fail(PT_ECUDA, "begin capture: %s", cudaGetErrorString(e));
        pt_status st = launch_on(ctx, kModeCycles, n_cycles, ctx->gstream);
        e = cudaStreamEndCapture(ctx->gstream, &graph);
        if (st != PT_OK) { if (graph) cudaGraphDestroy(graph); return st; }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->gexec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail(PT_ECUDA, "graph: %s", cudaGetErrorString(e));
        ctx->gcycles = n_cycles;
    }
    e = cudaEventRecord(ctx->gev_in, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->gstream, ctx->gev_in, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(ctx->gexec, ctx->gstream);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->gev_out, ctx->gstream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->gev_out, 0);
    if (e != cudaSuccess) return fail(PT_ECUDA, "graph launch: %s", cudaGetErrorString(e));
    return PT_OK;
}

pt_status pt_set_active(pt_ctx* ctx, int32_t inst, int32_t active) {
    pt_status s = check_inst(ctx, inst);
    if (s != PT_OK) return s;
    const int32_t v = active ? 1 : 0;
    const int32_t* dst = ctx->engine == 0 ? ctx->lat[inst].active : ctx->gr[inst].active;
    CK(cudaMemcpyAsync(const_cast<int32_t*>(dst), &v, 4, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return PT_OK;
}

pt_status pt_set_instance(pt_ctx* ctx, int32_t inst, const pt_instance_desc* desc) {
    const Range range("pt_set_instance");
    pt_status s = check_inst(ctx, inst);
    if (s != PT_OK) return s;
    if (!desc) return fail(PT_EINVAL, "desc is NULL");
    if (ctx->engine != 0) return fail(PT_ENOTSUP, "slot replacement is implemented for the lattice engine");
    s = validate(*desc, inst);
    if (s != PT_OK) return s;
    if (!is_lattice_desc(*desc)) return fail(PT_EINVAL, "the new instance needs the lattice engine");
    if (ctx->with_ctx) {
        s = context_slots_ok(*desc, inst);
        if (s != PT_OK) return s;
    }
    if (desc->lattice_L != ctx->L[inst] || desc->n_replicas != ctx->R[inst])
        return fail(PT_EINVAL, "slot %d holds L=%d, R=%d; the new instance must have the same shape",
                    inst, ctx->L[inst], ctx->R[inst]);
    LatHost h;
    s = lattice_host(*desc, h, inst, ctx->cfg.update == 1);
    if (s != PT_OK) return s;
    LatInst& I = ctx->lat[inst];
    lattice_fill_inst(I, h, desc->instance_id, ctx->cfg.pool_size);
    const LatOff& o = ctx->loff[inst];
    uint8_t* b = ctx->arena;
    cudaStream_t st = ctx->stream;
    const int32_t one = 1;
    CK(cudaMemcpyAsync(b + o.itab, h.itab.data(), h.itab.size() * 4, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(b + o.sow, h.sow.data(), h.sow.size() * 2, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(b + o.wos, h.wos.data(), h.wos.size() * 2, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(b + o.thr, h.thr.data(), h.thr.size() * 4, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(b + o.beta, desc->beta, (size_t)h.R * 8, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(b + o.prop, h.prop.data(), h.prop.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(b + o.eb, h.eb.data(), h.eb.size() * 4, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(b + o.cur, 0, (size_t)h.R * 4, st));
    CK(cudaMemsetAsync(b + o.ctr, 0, sizeof(Counters), st));
    CK(cudaMemsetAsync(b + o.st, 0, (size_t)4 * h.R * 8, st));
    if (ctx->cfg.proposal_rule == 2) CK(cudaMemsetAsync(b + o.lw, 0, (size_t)h.R * h.N * 8, st));
    CK(cudaMemcpyAsync(b + o.active, &one, 4, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ctx->d_lat + inst, &I, sizeof(LatInst), cudaMemcpyHostToDevice, st));
    {
        const Group& g = ctx->groups[ctx->group_of[inst]];
        int pos = 0;
        while (g.members[pos] != inst) ++pos;
        CK(cudaMemcpyAsync(static_cast<LatInst*>(g.d_insts) + pos, &I, sizeof(LatInst), cudaMemcpyHostToDevice, st));
    }
    cudaError_t e = launch_lattice_init(ctx->d_lat + inst, 1, ctx->cfg.seed, st);
    if (e != cudaSuccess) return fail(PT_ECUDA, "init: %s", cudaGetErrorString(e));
    s = launch_one(ctx, inst, kModeEnergy);
    if (s != PT_OK) return s;
    CK(cudaStreamSynchronize(st));
    return PT_OK;
}

pt_status pt_info(const pt_ctx* ctx, int32_t inst, int32_t info[6]) {
    if (!ctx || !info) return fail(PT_EINVAL, "NULL argument");
    const Group& g = ctx->groups[(inst >= 0 && inst < ctx->n) ? ctx->group_of[inst] : 0];
    info[0] = ctx->n;
    info[1] = ctx->engine;
    info[2] = g.T;
    info[3] = (int32_t)g.smem;
    info[4] = (inst >= 0 && inst < ctx->n) ? ctx->R[inst] : ctx->totalR;
    info[5] = (inst >= 0 && inst < ctx->n) ? ctx->N[inst] : ctx->uniformN;
    return PT_OK;
}

pt_status pt_sweep(pt_ctx* ctx, int32_t n_sweeps) {
    const Range range("pt_sweep");
    { const pt_status cs = check_ctx(ctx); if (cs != PT_OK) return cs; }
    if (n_sweeps < 0) return fail(PT_EINVAL, "n_sweeps must be >= 0");
    if (n_sweeps == 0) return PT_OK;
    return launch_run(ctx, kModeSweeps, n_sweeps);
}

pt_status pt_global_propose(pt_ctx* ctx) {
    const Range range("pt_global_propose");
    { const pt_status cs = check_ctx(ctx); if (cs != PT_OK) return cs; }
    return launch_run(ctx, kModePropose, 0);
}

pt_status pt_exchange(pt_ctx* ctx) {
    const Range range("pt_exchange");
    { const pt_status cs = check_ctx(ctx); if (cs != PT_OK) return cs; }
    return launch_run(ctx, kModeExchange, 0);
}

pt_status pt_run_cycles(pt_ctx* ctx, int32_t n_cycles) {
    const Range range("pt_run_cycles");
    { const pt_status cs = check_ctx(ctx); if (cs != PT_OK) return cs; }
    if (n_cycles < 0) return fail(PT_EINVAL, "n_cycles must be >= 0");
    if (n_cycles == 0) return PT_OK;
    return launch_run(ctx, kModeCycles, n_cycles);
}

pt_status pt_energies_device(pt_ctx* ctx, int32_t* dev_out) {
    if (!dev_out) return fail(PT_EINVAL, "NULL argument");
    { const pt_status cs = check_ctx(ctx); if (cs != PT_OK) return cs; }
    cudaError_t e = launch_gather_energies(ctx->d_Eptr, ctx->d_wosptr, ctx->d_eoff, ctx->n, dev_out, ctx->stream);
    if (e != cudaSuccess) return fail(PT_ECUDA, "gather: %s", cudaGetErrorString(e));
    return PT_OK;
}

pt_status pt_energies(pt_ctx* ctx, int32_t* out) {
    const Range range("pt_energies");
    if (!out) return fail(PT_EINVAL, "NULL argument");
    { const pt_status cs = check_ctx(ctx); if (cs != PT_OK) return cs; }
    pt_status s = pt_energies_device(ctx, ctx->d_eout);
    if (s != PT_OK) return s;
    CK(cudaMemcpyAsync(out, ctx->d_eout, (size_t)ctx->totalR * 4, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return PT_OK;
}

pt_status pt_read_state(pt_ctx* ctx, int32_t inst, int8_t* spins, int32_t* E) {
    const Range range("pt_read_state");
    pt_status s = check_inst(ctx, inst);
    if (s != PT_OK) return s;
    const int R = ctx->R[inst], N = ctx->N[inst];
    if (spins) {
        int8_t* d = nullptr;
        CK(cudaMallocAsync((void**)&d, (size_t)R * N, ctx->stream));
        cudaError_t e = ctx->engine == 0 ? launch_lattice_read(ctx->d_lat, inst, d, R * N, ctx->stream)
                                         : launch_graph_read(ctx->d_gr, inst, d, R * N, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(spins, d, (size_t)R * N, cudaMemcpyDeviceToHost, ctx->stream);
        cudaFreeAsync(d, ctx->stream);
        if (e != cudaSuccess) return fail(PT_ECUDA, "read_state: %s", cudaGetErrorString(e));
    }
    if (E) {
        s = pt_energies_device(ctx, ctx->d_eout);
        if (s != PT_OK) return s;
        CK(cudaMemcpyAsync(E, ctx->d_eout + ctx->eoff[inst], (size_t)R * 4, cudaMemcpyDeviceToHost, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return PT_OK;
}

pt_status pt_read_walkers(pt_ctx* ctx, int32_t inst, int32_t* walker) {
    pt_status s = check_inst(ctx, inst);
    if (s != PT_OK) return s;
    if (!walker) return fail(PT_EINVAL, "walker is NULL");
    const int R = ctx->R[inst];
    std::vector<int16_t> w(R);
    const int16_t* src = ctx->engine == 0 ? ctx->lat[inst].wos : ctx->gr[inst].wos;
    CK(cudaMemcpyAsync(w.data(), src, (size_t)R * 2, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int r = 0; r < R; ++r) walker[r] = w[r];
    return PT_OK;
}

pt_status pt_read_counters(pt_ctx* ctx, int32_t inst, int64_t counters[3], int32_t* cursors) {
    pt_status s = check_inst(ctx, inst);
    if (s != PT_OK) return s;
    Counters h{};
    CK(cudaMemcpyAsync(&h, ctr_ptr(ctx, inst), sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    if (cursors)
        CK(cudaMemcpyAsync(cursors, cursor_ptr(ctx, inst), (size_t)ctx->R[inst] * 4, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (counters) { counters[0] = h.sweeps; counters[1] = h.n_ex; counters[2] = h.n_prop; }
    return PT_OK;
}

pt_status pt_read_stats(pt_ctx* ctx, int32_t inst, int64_t* swap_acc, int64_t* swap_att,
                        int64_t* prop_acc, int64_t* prop_att) {
    pt_status s = check_inst(ctx, inst);
    if (s != PT_OK) return s;
    const int R = ctx->R[inst];
    std::vector<unsigned long long> h(4 * (size_t)R);
    const unsigned long long* src = ctx->engine == 0 ? ctx->lat[inst].stats : ctx->gr[inst].stats;
    CK(cudaMemcpyAsync(h.data(), src, h.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int r = 0; r < R; ++r) {
        if (r + 1 < R) {
            if (swap_acc) swap_acc[r] = (int64_t)h[r];
            if (swap_att) swap_att[r] = (int64_t)h[R + r];
        }
        if (prop_acc) prop_acc[r] = (int64_t)h[2 * R + r];
        if (prop_att) prop_att[r] = (int64_t)h[3 * R + r];
    }
    return PT_OK;
}

pt_status pt_write_state(pt_ctx* ctx, int32_t inst, const int8_t* spins, const int32_t* walker,
                         const int64_t counters[3], const int32_t* cursors) {
    pt_status s = check_inst(ctx, inst);
    if (s != PT_OK) return s;
    if (!spins || !walker || !counters) return fail(PT_EINVAL, "NULL argument");
    const int R = ctx->R[inst], N = ctx->N[inst];
    std::vector<int> seen(R, 0);
    for (int r = 0; r < R; ++r) {
        if (walker[r] < 0 || walker[r] >= R || seen[walker[r]]++) return fail(PT_EINVAL, "walker ids must be a permutation of 0..R-1");
    }
    for (size_t i = 0; i < (size_t)R * N; ++i)
        if (spins[i] != 1 && spins[i] != -1) return fail(PT_EINVAL, "spins must be +-1");
    if (cursors && ctx->cfg.pool_size > 0)
        for (int r = 0; r < R; ++r)
            if (cursors[r] < 0 || cursors[r] >= ctx->cfg.pool_size) return fail(PT_EINVAL, "cursor out of range");
    std::vector<int8_t> hclamp;
    if (ctx->engine == 1) {  // clamped spins must keep their values
        hclamp.resize(N);
        CK(cudaMemcpyAsync(hclamp.data(), ctx->gr[inst].clamp, N, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        for (int r = 0; r < R; ++r)
            for (int i = 0; i < N; ++i)
                if (hclamp[i] != 0 && spins[(size_t)r * N + i] != hclamp[i])
                    return fail(PT_EINVAL, "spin %d of slot %d contradicts its clamp", i, r);
    }
    // walker labels
    const int Wpad = ctx->engine == 0 ? ctx->W[inst] * 32 : ctx->Rp[inst];
    std::vector<int16_t> wos(R), sow(Wpad, -1);
    for (int r = 0; r < R; ++r) { wos[r] = (int16_t)walker[r]; sow[walker[r]] = (int16_t)r; }
    int8_t* d_sp = nullptr;
    int32_t* d_w = nullptr;
    CK(cudaMallocAsync((void**)&d_sp, (size_t)R * N, ctx->stream));
    CK(cudaMallocAsync((void**)&d_w, (size_t)R * 4, ctx->stream));
    CK(cudaMemcpyAsync(d_sp, spins, (size_t)R * N, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(d_w, walker, (size_t)R * 4, cudaMemcpyHostToDevice, ctx->stream));
    Counters h{};
    h.sweeps = counters[0]; h.n_ex = counters[1]; h.n_prop = counters[2];
    cudaError_t e;
    if (ctx->engine == 0) {
        CK(cudaMemcpyAsync(ctx->lat[inst].wos, wos.data(), R * 2, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->lat[inst].sow, sow.data(), Wpad * 2, cudaMemcpyHostToDevice, ctx->stream));
        e = launch_lattice_write(ctx->d_lat, inst, d_sp, d_w, ctx->W[inst] * N, ctx->stream);
    } else {
        CK(cudaMemcpyAsync(ctx->gr[inst].wos, wos.data(), R * 2, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->gr[inst].sow, sow.data(), Wpad * 2, cudaMemcpyHostToDevice, ctx->stream));
        e = launch_graph_write(ctx->d_gr, inst, d_sp, d_w, R * N, ctx->stream);
    }
    if (e != cudaSuccess) return fail(PT_ECUDA, "write_state: %s", cudaGetErrorString(e));
    CK(cudaMemcpyAsync(ctr_ptr(ctx, inst), &h, sizeof h, cudaMemcpyHostToDevice, ctx->stream));
    if (cursors && ctx->cfg.pool_size > 0)
        CK(cudaMemcpyAsync(cursor_ptr(ctx, inst), cursors, (size_t)R * 4, cudaMemcpyHostToDevice, ctx->stream));
    cudaFreeAsync(d_sp, ctx->stream);
    cudaFreeAsync(d_w, ctx->stream);
    CK(cudaStreamSynchronize(ctx->stream));
    // energies of the written state (all instances: the energy pass leaves others unchanged)
    s = launch_run(ctx, kModeEnergy, 0);
    if (s != PT_OK) return s;
    CK(cudaStreamSynchronize(ctx->stream));
    return PT_OK;
}

// Proposal law of one slot's pool for proposal rule 2: the log-odds log(p/(1-p)) of each site,
// rounded to multiples of 2^-32 (the expression the oracle evaluates), clamped sites 0.
pt_status pt_load_proposal_law(pt_ctx* ctx, int32_t inst, int32_t replica, const double* p_plus) {
    const Range range("pt_load_proposal_law");
    pt_status s = check_inst(ctx, inst);
    if (s != PT_OK) return s;
    if (!p_plus) return fail(PT_EINVAL, "p_plus is NULL");
    if (ctx->cfg.proposal_rule != 2) return fail(PT_ESTATE, "the context's proposal_rule is not 2");
    const int R = ctx->R[inst], N = ctx->N[inst];
    if (replica < 0 || replica >= R) return fail(PT_EINVAL, "replica %d out of range [0, %d)", replica, R);
    const int8_t* clamp = nullptr;
    std::vector<int8_t> hclamp;
    if (ctx->engine == 1) {
        hclamp.resize(N);
        CK(cudaMemcpyAsync(hclamp.data(), ctx->gr[inst].clamp, N, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        clamp = hclamp.data();
    }
    std::vector<long long> w(N);
    for (int i = 0; i < N; ++i) {
        const double p = p_plus[i];
        if (!(p > 0.0 && p < 1.0)) return fail(PT_EINVAL, "p_plus[%d] = %g is not in (0, 1)", i, p);
        const double lo = log(p) - log1p(-p);
        w[i] = (clamp && clamp[i] != 0) ? 0 : llround(ldexp(lo, 32));
    }
    const long long* dst = (ctx->engine == 0 ? ctx->lat[inst].lw : ctx->gr[inst].lw) + (size_t)replica * N;
    CK(cudaMemcpyAsync(const_cast<long long*>(dst), w.data(), (size_t)N * 8, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return PT_OK;
}

pt_status pt_load_proposals(pt_ctx* ctx, int32_t inst, int32_t replica, const int8_t* spins,
                            int32_t count, int32_t first) {
    pt_status s = check_inst(ctx, inst);
    if (s != PT_OK) return s;
    const int R = ctx->R[inst], N = ctx->N[inst], NW = ctx->NW[inst], P = ctx->cfg.pool_size;
    if (P <= 0) return fail(PT_ESTATE, "the context was created with pool_size = 0");
    if (replica < 0 || replica >= R) return fail(PT_EINVAL, "replica %d out of range", replica);
    if (count < 0 || first < 0 || first + count > P) return fail(PT_EINVAL, "pool range [%d, %d) exceeds pool_size %d", first, first + count, P);
    if (count == 0) return PT_OK;
    if (!spins) return fail(PT_EINVAL, "spins is NULL");
    std::vector<uint32_t> bits((size_t)count * NW, 0u);
    for (int e = 0; e < count; ++e)
        for (int i = 0; i < N; ++i) {
            const int8_t v = spins[(size_t)e * N + i];
            if (v != 1 && v != -1) return fail(PT_EINVAL, "pool spins must be +-1");
            if (v > 0) bits[(size_t)e * NW + (i >> 5)] |= 1u << (i & 31);
        }
    uint32_t* dst = ctx->pool + ctx->slab_off[inst] + (size_t)replica * NW + (size_t)first * ctx->slab;
    CK(cudaMemcpy2DAsync(dst, ctx->slab * 4, bits.data(), (size_t)NW * 4, (size_t)NW * 4, count,
                         cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return PT_OK;
}

pt_status pt_load_proposals_packed(pt_ctx* ctx, const uint32_t* words, int32_t first, int32_t count) {
    const Range range("pt_load_proposals_packed");
    { const pt_status cs = check_ctx(ctx); if (cs != PT_OK) return cs; }
    const int P = ctx->cfg.pool_size;
    if (P <= 0) return fail(PT_ESTATE, "the context was created with pool_size = 0");
    if (count < 0 || first < 0 || first + count > P) return fail(PT_EINVAL, "pool range [%d, %d) exceeds pool_size %d", first, first + count, P);
    if (count == 0) return PT_OK;
    if (!words) return fail(PT_EINVAL, "words is NULL");
    CK(cudaMemcpyAsync(ctx->pool + (size_t)first * ctx->slab, words, (size_t)count * ctx->slab * 4,
                       cudaMemcpyHostToDevice, ctx->stream));
    return PT_OK;
}

pt_status pt_load_proposals_inst_packed(pt_ctx* ctx, int32_t inst, const uint32_t* words,
                                        int32_t first, int32_t count) {
    pt_status s = check_inst(ctx, inst);
    if (s != PT_OK) return s;
    const int P = ctx->cfg.pool_size;
    if (P <= 0) return fail(PT_ESTATE, "the context was created with pool_size = 0");
    if (count < 0 || first < 0 || first + count > P) return fail(PT_EINVAL, "pool range [%d, %d) exceeds pool_size %d", first, first + count, P);
    if (count == 0) return PT_OK;
    if (!words) return fail(PT_EINVAL, "words is NULL");
    const size_t row = (size_t)ctx->R[inst] * ctx->NW[inst] * 4;
    CK(cudaMemcpy2DAsync(ctx->pool + ctx->slab_off[inst] + (size_t)first * ctx->slab, ctx->slab * 4,
                         words, row, row, count, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return PT_OK;
}

pt_status pt_read_proposals_packed(pt_ctx* ctx, uint32_t* words, int32_t first, int32_t count) {
    { const pt_status cs = check_ctx(ctx); if (cs != PT_OK) return cs; }
    const int P = ctx->cfg.pool_size;
    if (P <= 0) return fail(PT_ESTATE, "the context was created with pool_size = 0");
    if (count < 0 || first < 0 || first + count > P) return fail(PT_EINVAL, "pool range [%d, %d) exceeds pool_size %d", first, first + count, P);
    if (count == 0) return PT_OK;
    if (!words) return fail(PT_EINVAL, "words is NULL");
    CK(cudaMemcpyAsync(words, ctx->pool + (size_t)first * ctx->slab, (size_t)count * ctx->slab * 4,
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return PT_OK;
}

pt_status pt_capture_proposals(pt_ctx* dst, const pt_ctx* src, int32_t entry) {
    const Range range("pt_capture_proposals");
    if (!dst || !src) return fail(PT_EINVAL, "NULL context");
    { const pt_status cs = check_ctx(dst); if (cs != PT_OK) return cs; }
    { const pt_status cs = check_ctx(src); if (cs != PT_OK) return cs; }
    if (dst->engine != src->engine || dst->n != src->n) return fail(PT_EINVAL, "batches differ in shape");
    for (int k = 0; k < dst->n; ++k)
        if (dst->N[k] != src->N[k] || dst->R[k] != src->R[k]) return fail(PT_EINVAL, "instance %d differs in shape", k);
    if (dst->cfg.pool_size <= 0) return fail(PT_ESTATE, "destination has no pool");
    if (entry < 0 || entry >= dst->cfg.pool_size) return fail(PT_EINVAL, "entry out of range");
    cudaError_t e = dst->engine == 0 ? launch_lattice_capture(dst->d_lat, src->d_lat, dst->n, entry, dst->stream)
                                     : launch_graph_capture(dst->d_gr, src->d_gr, dst->n, entry, dst->stream);
    if (e != cudaSuccess) return fail(PT_ECUDA, "capture: %s", cudaGetErrorString(e));
    return PT_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------ gather kernel
namespace pt {
__global__ void gather_energies_kernel(const int32_t* const* E, const int16_t* const* wos,
                                       const int32_t* off, int32_t* out) {
    const int k = blockIdx.x;
    const int R = off[k + 1] - off[k];
    for (int r = threadIdx.x; r < R; r += blockDim.x) out[off[k] + r] = E[k][wos[k][r]];
}
cudaError_t launch_gather_energies(const int32_t* const* E, const int16_t* const* wos,
                                   const int32_t* off, int n, int32_t* out, cudaStream_t s) {
    gather_energies_kernel<<<n, 128, 0, s>>>(E, wos, off, out);
    return cudaGetLastError();
}
}  // namespace pt

// ------------------------------------------------------------------ allocation-free state read
// pt_read_state allocates a temporary device buffer for the unpacked spins on every call.
// pt_read_state_noalloc serves callers that must not allocate device memory in their steady
// state: it unpacks into a fixed file-scope device buffer instead. Host code cannot use the
// array's name as a device address, so the address is looked up with cudaGetSymbolAddress
// once per device and CUDA context, with that device current, and cached. The cache is keyed
// on the current CUDA context as well as the device: after a device reset the runtime builds
// a new context, which loads the library's module afresh, so the address is looked up again.
// The buffer is shared by every call and keeps the last call's contents; the read kernel
// overwrites every byte that is copied out, so nothing has to be cleared first.
namespace {
constexpr size_t kReadScratchBytes = 256 * 1024;
constexpr int kMaxDevices = 64;
}  // namespace

static __device__ __align__(256) int8_t g_read_scratch[kReadScratchBytes];

namespace {
std::mutex g_scratch_mutex;
struct ScratchEntry {
    void* cu_ctx = nullptr;      // the CUDA context the address belongs to
    int8_t* ptr = nullptr;
};
ScratchEntry g_scratch[kMaxDevices];

// cuCtxGetCurrent through the runtime's driver entry-point table, so that the library does not
// link the driver library itself (it must load where no driver is installed).
using CtxGetCurrentFn = int (*)(void**);
CtxGetCurrentFn ctx_get_current() {
    static CtxGetCurrentFn fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<CtxGetCurrentFn>(f);
    }();
    return fn;
}

pt_status scratch_for_current_device(int8_t** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(PT_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(PT_ENOTSUP, "device %d beyond %d", dev, kMaxDevices);
    const CtxGetCurrentFn get = ctx_get_current();
    if (!get) return fail(PT_ECUDA, "cuCtxGetCurrent is not available");
    void* cu_ctx = nullptr;
    if (get(&cu_ctx) != 0) return fail(PT_ECUDA, "cuCtxGetCurrent failed");
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    ScratchEntry& ent = g_scratch[dev];
    if (!cu_ctx || !ent.ptr || ent.cu_ctx != cu_ctx) {
        // the lookup also binds the device's primary context to this thread when none is
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_read_scratch);
        if (e != cudaSuccess || !p)
            return fail(PT_ECUDA, "cudaGetSymbolAddress(read scratch): %s", cudaGetErrorString(e));
        if (!cu_ctx && (get(&cu_ctx) != 0 || !cu_ctx))
            return fail(PT_ECUDA, "no CUDA context is current after the symbol lookup");
        ent.ptr = static_cast<int8_t*>(p);
        ent.cu_ctx = cu_ctx;
    }
    *out = ent.ptr;
    return PT_OK;
}
}  // namespace

extern "C" pt_status pt_read_state_noalloc(pt_ctx* ctx, int32_t inst, int8_t* spins, int32_t* E) {
    pt_status s = check_inst(ctx, inst);
    if (s != PT_OK) return s;
    const int R = ctx->R[inst], N = ctx->N[inst];
    if (spins) {
        if ((size_t)R * (size_t)N > kReadScratchBytes)
            return fail(PT_ENOTSUP, "R*N = %zu exceeds the %zu-byte allocation-free read buffer; "
                        "use pt_read_state", (size_t)R * (size_t)N, kReadScratchBytes);
        int8_t* d = nullptr;
        s = scratch_for_current_device(&d);
        if (s != PT_OK) return s;
        cudaError_t e = ctx->engine == 0 ? launch_lattice_read(ctx->d_lat, inst, d, R * N, ctx->stream)
                                         : launch_graph_read(ctx->d_gr, inst, d, R * N, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(spins, d, (size_t)R * N, cudaMemcpyDeviceToHost, ctx->stream);
        if (e != cudaSuccess) return fail(PT_ECUDA, "read_state_noalloc: %s", cudaGetErrorString(e));
    }
    if (E) {
        s = pt_energies_device(ctx, ctx->d_eout);
        if (s != PT_OK) return s;
        CK(cudaMemcpyAsync(E, ctx->d_eout + ctx->eoff[inst], (size_t)R * 4, cudaMemcpyDeviceToHost, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return PT_OK;
}
