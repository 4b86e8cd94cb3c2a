/*
 * CPU oracle for TAPT (Algorithm 1 of arXiv 2509.23043). TEST INFRASTRUCTURE ONLY:
 * loaded by tests, the smoke check and the benchmark's CPU-baseline leg, never by the
 * product path. Plain sequential loops; no blocking, fusion or reordering beyond what the
 * paper's definitions state. See pt_oracle.h for the readings taken.
 *
 * Random-number counters (Philox4x32-10, key = seed low/high 32 bits). ctr = {c0,c1,c2,c3}:
 *   init        c0 = site,  c1 = 0,      c2 = (0<<24) | (walker>>5),                 c3 = id
 *               spin = +1 iff bit (walker & 31) of output word 0 is set
 *   local move, bit-plane layout (lattice + J=+-1, no field, no clamp; either rule):
 *               c0 = site,  c1 = sweep, c2 = (1<<24) | (k>>2)<<16 | (walker>>5),     c3 = id
 *               u = sum_k bit(walker & 31) of output word (k & 3), times 2^(31-k), k=0..31
 *   local move, word layout (all other instances):
 *               c0 = site,  c1 = sweep, c2 = (2<<24) | (walker>>2),                  c3 = id
 *               u = output word (walker & 3)
 *   exchange    c0 = lower slot r, c1 = exchange event (1-based), c2 = 3<<24,        c3 = id
 *   proposal    c0 = slot r, c1 = proposal event (1-based),       c2 = 4<<24,        c3 = id
 * A walker is a configuration's identity: it is created with slot r = walker r and moves
 * with its configuration when an exchange swaps two configurations. Local-move random
 * numbers follow the walker; thresholds follow the temperature slot.
 */
#include "pt_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ----------------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as      */
/* 1, 2, 3", SC'11): 10 rounds of two 32x32->64 multiplies and xors, key bumped by the  */
/* Weyl constants between rounds.                                                       */
/* ----------------------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void or_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static uint32_t philox_word(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                            uint32_t c3, int word) {
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    or_philox(ctr, key, out);
    return out[word];
}

/* ----------------------------------------------------------------------------------- */
/* Thresholds and the FP64 acceptance rule                                              */
/* ----------------------------------------------------------------------------------- */
static uint32_t prob_to_threshold(double p) {
    double t = floor(ldexp(p, 32));
    if (t >= 4294967295.0) return 4294967295u;
    if (t <= 0.0) return 0u;
    return (uint32_t)t;
}

/* Metropolis (used for dE > 0 only): flip with probability exp(-beta dE). */
uint32_t or_metropolis_threshold(double beta, int32_t dE) {
    return prob_to_threshold(exp(-beta * (double)dE));
}

/* Gibbs / heat bath (Methods): P(m = +1) = (1 + tanh(beta I)) / 2. */
uint32_t or_gibbs_threshold(double beta, int32_t I) {
    return prob_to_threshold(0.5 * (1.0 + tanh(beta * (double)I)));
}

/* min[1, exp(x)] realised with a 32-bit uniform u: accept iff x >= 0 or u+1 <= 2^32 e^x. */
int or_accept(double x, uint32_t u) {
    if (x >= 0.0) return 1;
    return ((double)u + 1.0) <= ldexp(exp(x), 32);
}

/* ----------------------------------------------------------------------------------- */
/* Energy (Supplementary S4)                                                            */
/* ----------------------------------------------------------------------------------- */
int64_t or_energy(int32_t n, int32_t n_edges, const int32_t *ei, const int32_t *ej,
                  const int32_t *eJ, const int32_t *h, const int8_t *spins) {
    int64_t E = 0;
    for (int32_t e = 0; e < n_edges; ++e)
        E -= (int64_t)eJ[e] * spins[ei[e]] * spins[ej[e]];
    if (h)
        for (int32_t i = 0; i < n; ++i) E -= (int64_t)h[i] * spins[i];
    return E;
}

/* ----------------------------------------------------------------------------------- */
/* Instance state                                                                       */
/* ----------------------------------------------------------------------------------- */
struct or_inst {
    uint32_t id;
    int32_t N, L, NE, R;
    int32_t *ei, *ej, *eJ;
    int32_t *h;               /* N, zero when no field */
    int8_t *clamp;            /* N, 0 free */
    double *beta;
    uint8_t *prop;
    int32_t update, M, every, start, stop;
    int32_t rule;             /* proposal rule: 0 Delta-E-only, 1 always accept, 2 independent MH */
    int32_t source;           /* proposal source: 0 pool, 1 contextual */
    int64_t *lw;              /* [R][N] log-odds of each slot's proposal law, units of 2^-32 */
    int32_t ctx_log2, ctx_sweeps;
    uint64_t seed;
    int32_t P;
    /* adjacency: for site i, neighbours adj_j[adj_off[i] .. adj_off[i+1]) with couplings */
    int32_t *adj_off, *adj_j, *adj_J;
    /* colouring */
    int32_t ncol;
    int32_t *colour;
    int bitplane;
    /* state, in slot order */
    int8_t *spins;            /* R*N */
    int32_t *E;               /* R */
    int32_t *walker;          /* R */
    int8_t *pool;             /* R*P*N */
    int32_t *cursor;          /* R */
    int64_t sweeps, n_ex, n_prop;
    int64_t *swap_acc, *swap_att, *prop_acc, *prop_att;
};

static void *xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s ? s : 1); }

/* Lattice colouring: L even -> (x+y+z) mod 2. L odd -> (c(x)+c(y)+c(z)) mod 3 with
 * c(t) = t mod 2 for t < L-1 and c(L-1) = 2, a proper 3-colouring of the odd cycle, so the
 * sum mod 3 properly colours the periodic cube. Colours are independent sets
 * (Methods, "Graph coloring"). */
static int32_t lattice_colour(int32_t n, int32_t L) {
    int32_t x = n % L, y = (n / L) % L, z = n / (L * L);
    if (L % 2 == 0) return (x + y + z) % 2;
    int32_t cx = (x == L - 1) ? 2 : x % 2;
    int32_t cy = (y == L - 1) ? 2 : y % 2;
    int32_t cz = (z == L - 1) ? 2 : z % 2;
    return (cx + cy + cz) % 3;
}

/* DSATUR (Brelaz 1979), Methods "Graph coloring", over the whole interaction graph
 * (clamped sites included, so the colouring does not depend on the clamp values; clamped
 * sites are then simply never updated): repeatedly colour the uncoloured site with the most
 * distinct neighbour colours, ties broken by the larger number of distinct neighbours, then
 * the lower index; give it the smallest colour absent from its neighbours. */
static int32_t dsatur(or_inst *o) {
    int32_t N = o->N;
    int32_t *deg = (int32_t *)xcalloc((size_t)N, sizeof(int32_t));
    for (int32_t i = 0; i < N; ++i) {
        o->colour[i] = -1;
        for (int32_t a = o->adj_off[i]; a < o->adj_off[i + 1]; ++a) {
            int32_t j = o->adj_j[a];
            int dup = 0;  /* count distinct neighbours */
            for (int32_t b = o->adj_off[i]; b < a; ++b)
                if (o->adj_j[b] == j) { dup = 1; break; }
            if (!dup) deg[i]++;
        }
    }
    int32_t ncol = 0;
    uint8_t *used = (uint8_t *)xcalloc((size_t)N + 1, 1);
    for (int32_t step = 0; step < N; ++step) {
        int32_t best = -1, best_sat = -1, best_deg = -1;
        for (int32_t i = 0; i < N; ++i) {
            if (o->colour[i] >= 0) continue;
            memset(used, 0, (size_t)N + 1);
            int32_t sat = 0;
            for (int32_t a = o->adj_off[i]; a < o->adj_off[i + 1]; ++a) {
                int32_t c = o->colour[o->adj_j[a]];
                if (c >= 0 && !used[c]) { used[c] = 1; ++sat; }
            }
            if (sat > best_sat || (sat == best_sat && deg[i] > best_deg)) {
                best = i; best_sat = sat; best_deg = deg[i];
            }
        }
        memset(used, 0, (size_t)N + 1);
        for (int32_t a = o->adj_off[best]; a < o->adj_off[best + 1]; ++a) {
            int32_t c = o->colour[o->adj_j[a]];
            if (c >= 0) used[c] = 1;
        }
        int32_t c = 0;
        while (used[c]) ++c;
        o->colour[best] = c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    free(used);
    free(deg);
    return ncol;
}

void or_destroy(or_inst *o) {
    if (!o) return;
    free(o->ei); free(o->ej); free(o->eJ); free(o->h); free(o->clamp); free(o->beta);
    free(o->prop); free(o->adj_off); free(o->adj_j); free(o->adj_J); free(o->colour);
    free(o->spins); free(o->E); free(o->walker); free(o->pool); free(o->cursor);
    free(o->swap_acc); free(o->swap_att); free(o->prop_acc); free(o->prop_att);
    free(o->lw);
    free(o);
}

static int32_t energy_of(const or_inst *o, const int8_t *s) {
    return (int32_t)or_energy(o->N, o->NE, o->ei, o->ej, o->eJ, o->h, s);
}

static void recompute_energies(or_inst *o) {
    for (int32_t r = 0; r < o->R; ++r) o->E[r] = energy_of(o, o->spins + (size_t)r * o->N);
}

or_inst *or_create(uint32_t instance_id, int32_t n_spins, int32_t lattice_L,
                   int32_t n_edges, const int32_t *ei, const int32_t *ej, const int32_t *eJ,
                   const int32_t *h, const int8_t *clamp,
                   int32_t n_replicas, const double *beta, const uint8_t *prop_enabled,
                   int32_t update, int32_t sweeps_per_cycle, int32_t propose_every,
                   int32_t propose_start, int32_t propose_stop, uint64_t seed,
                   int32_t pool_size, int32_t proposal_rule, int32_t proposal_source,
                   int32_t context_log2, int32_t context_sweeps) {
    if (n_spins <= 0 || n_edges < 0 || n_replicas <= 0 || sweeps_per_cycle <= 0) return NULL;
    if (update != 0 && update != 1) return NULL;
    if (proposal_rule < 0 || proposal_rule > 2) return NULL;
    if (proposal_rule == 2 && proposal_source != 0) return NULL;
    if (proposal_source != 0 && proposal_source != 1) return NULL;
    if (proposal_source == 1 && (context_log2 < 1 || context_log2 > 3 || context_sweeps < 1))
        return NULL;
    if (lattice_L > 0 && lattice_L * lattice_L * lattice_L != n_spins) return NULL;
    for (int32_t e = 0; e < n_edges; ++e)
        if (ei[e] < 0 || ei[e] >= n_spins || ej[e] < 0 || ej[e] >= n_spins || ei[e] == ej[e])
            return NULL;
    for (int32_t r = 0; r + 1 < n_replicas; ++r)
        if (!(beta[r] <= beta[r + 1])) return NULL;
    or_inst *o = (or_inst *)xcalloc(1, sizeof(or_inst));
    o->id = instance_id; o->N = n_spins; o->L = lattice_L; o->NE = n_edges; o->R = n_replicas;
    o->update = update; o->M = sweeps_per_cycle; o->every = propose_every;
    o->start = propose_start; o->stop = propose_stop; o->seed = seed;
    o->rule = proposal_rule;
    o->source = proposal_source; o->ctx_log2 = context_log2; o->ctx_sweeps = context_sweeps;
    o->P = pool_size > 0 ? pool_size : 0;
    o->lw = (int64_t *)xcalloc((size_t)n_replicas * n_spins, 8);
    o->ei = (int32_t *)xcalloc((size_t)n_edges, 4);
    o->ej = (int32_t *)xcalloc((size_t)n_edges, 4);
    o->eJ = (int32_t *)xcalloc((size_t)n_edges, 4);
    if (n_edges) {
        memcpy(o->ei, ei, (size_t)n_edges * 4);
        memcpy(o->ej, ej, (size_t)n_edges * 4);
        memcpy(o->eJ, eJ, (size_t)n_edges * 4);
    }
    o->h = (int32_t *)xcalloc((size_t)n_spins, 4);
    int has_h = 0, has_clamp = 0, unit_J = 1;
    if (h) { memcpy(o->h, h, (size_t)n_spins * 4); for (int32_t i = 0; i < n_spins; ++i) has_h |= (h[i] != 0); }
    o->clamp = (int8_t *)xcalloc((size_t)n_spins, 1);
    if (clamp) {
        for (int32_t i = 0; i < n_spins; ++i) {
            if (clamp[i] != 0 && clamp[i] != 1 && clamp[i] != -1) { or_destroy(o); return NULL; }
            o->clamp[i] = clamp[i];
            has_clamp |= (clamp[i] != 0);
        }
    }
    for (int32_t e = 0; e < n_edges; ++e) unit_J &= (eJ[e] == 1 || eJ[e] == -1);
    o->beta = (double *)xcalloc((size_t)n_replicas, sizeof(double));
    memcpy(o->beta, beta, (size_t)n_replicas * sizeof(double));
    o->prop = (uint8_t *)xcalloc((size_t)n_replicas, 1);
    if (prop_enabled) memcpy(o->prop, prop_enabled, (size_t)n_replicas);
    o->bitplane = (lattice_L > 0 && !has_h && !has_clamp && unit_J);
    if (proposal_source == 1) {
        int32_t n_en = 0;
        for (int32_t r = 0; r < n_replicas; ++r) n_en += o->prop[r] != 0;
        if (!o->bitplane || n_en > 32) { or_destroy(o); return NULL; }
    }

    /* adjacency lists (each edge seen from both ends; parallel edges kept apart) */
    o->adj_off = (int32_t *)xcalloc((size_t)n_spins + 1, 4);
    for (int32_t e = 0; e < n_edges; ++e) { o->adj_off[ei[e] + 1]++; o->adj_off[ej[e] + 1]++; }
    for (int32_t i = 0; i < n_spins; ++i) o->adj_off[i + 1] += o->adj_off[i];
    o->adj_j = (int32_t *)xcalloc((size_t)2 * n_edges, 4);
    o->adj_J = (int32_t *)xcalloc((size_t)2 * n_edges, 4);
    int32_t *fill = (int32_t *)xcalloc((size_t)n_spins, 4);
    for (int32_t e = 0; e < n_edges; ++e) {
        int32_t a = ei[e], b = ej[e];
        o->adj_j[o->adj_off[a] + fill[a]] = b; o->adj_J[o->adj_off[a] + fill[a]] = eJ[e]; fill[a]++;
        o->adj_j[o->adj_off[b] + fill[b]] = a; o->adj_J[o->adj_off[b] + fill[b]] = eJ[e]; fill[b]++;
    }
    free(fill);

    /* colour classes */
    o->colour = (int32_t *)xcalloc((size_t)n_spins, 4);
    if (lattice_L > 0) {
        o->ncol = (lattice_L % 2 == 0) ? 2 : 3;
        for (int32_t i = 0; i < n_spins; ++i) o->colour[i] = lattice_colour(i, lattice_L);
    } else {
        o->ncol = dsatur(o);
    }

    /* state: walker r starts in slot r; spins from the init stream; clamps applied
     * (Algorithm 1, initialisation: uniformly random replicas) */
    o->spins = (int8_t *)xcalloc((size_t)n_replicas * n_spins, 1);
    o->E = (int32_t *)xcalloc((size_t)n_replicas, 4);
    o->walker = (int32_t *)xcalloc((size_t)n_replicas, 4);
    o->cursor = (int32_t *)xcalloc((size_t)n_replicas, 4);
    o->pool = (int8_t *)xcalloc((size_t)n_replicas * (size_t)o->P * n_spins, 1);
    o->swap_acc = (int64_t *)xcalloc((size_t)n_replicas, 8);
    o->swap_att = (int64_t *)xcalloc((size_t)n_replicas, 8);
    o->prop_acc = (int64_t *)xcalloc((size_t)n_replicas, 8);
    o->prop_att = (int64_t *)xcalloc((size_t)n_replicas, 8);
    for (int32_t r = 0; r < n_replicas; ++r) {
        int32_t w = r;
        o->walker[r] = w;
        for (int32_t i = 0; i < n_spins; ++i) {
            int8_t s;
            if (o->clamp[i] != 0) {
                s = o->clamp[i];
            } else {
                uint32_t word = philox_word(seed, (uint32_t)i, 0u, (uint32_t)(w >> 5),
                                            instance_id, 0);
                s = ((word >> (w & 31)) & 1u) ? 1 : -1;
            }
            o->spins[(size_t)r * n_spins + i] = s;
        }
    }
    recompute_energies(o);
    return o;
}

int or_load_pool(or_inst *o, int32_t r, const int8_t *spins, int32_t count, int32_t first) {
    if (r < 0 || r >= o->R || first < 0 || count < 0 || first + count > o->P) return 1;
    memcpy(o->pool + ((size_t)r * o->P + first) * o->N, spins, (size_t)count * o->N);
    return 0;
}

/* The proposal law of slot r's pool (proposal rule 2): the pool entries are independent
 * draws from the product-Bernoulli law q(x) = prod_i p_i^[x_i=+1] (1-p_i)^[x_i=-1]. Its
 * per-site log-odds log(p_i/(1-p_i)) are stored rounded to multiples of 2^-32, so that
 * log q(x) - log q(x') = sum_i ([x_i=+1] - [x'_i=+1]) log-odds_i is an exact integer sum.
 * Clamped sites carry no weight: the current state and the candidate agree on them. */
int or_load_law(or_inst *o, int32_t r, const double *p_plus) {
    if (r < 0 || r >= o->R) return 1;
    for (int32_t i = 0; i < o->N; ++i)
        if (!(p_plus[i] > 0.0 && p_plus[i] < 1.0)) return 1;
    for (int32_t i = 0; i < o->N; ++i) {
        double lo = log(p_plus[i]) - log1p(-p_plus[i]);
        o->lw[(size_t)r * o->N + i] = o->clamp[i] != 0 ? 0 : llround(ldexp(lo, 32));
    }
    return 0;
}

/* sum of slot r's log-odds over the +1 spins of a configuration (units of 2^-32) */
static int64_t law_weight(const or_inst *o, int32_t r, const int8_t *x) {
    int64_t L = 0;
    for (int32_t i = 0; i < o->N; ++i)
        if (x[i] > 0) L += o->lw[(size_t)r * o->N + i];
    return L;
}

/* the 32-bit uniform of one local move */
static uint32_t local_uniform(const or_inst *o, int32_t site, int32_t walker) {
    uint32_t s = (uint32_t)o->sweeps;
    if (o->bitplane) {
        uint32_t u = 0;
        for (int k = 0; k < 32; ++k) {
            uint32_t c2 = (1u << 24) | ((uint32_t)(k >> 2) << 16) | (uint32_t)(walker >> 5);
            uint32_t word = philox_word(o->seed, (uint32_t)site, s, c2, o->id, k & 3);
            u |= ((word >> (walker & 31)) & 1u) << (31 - k);
        }
        return u;
    }
    /* general graphs: two 16-bit halves, u = hi << 16 | lo, each the (walker odd: low, even:
     * high) half of output word (walker & 7) / 2 of Philox(site, sweep, 2 << 24 | part << 16 |
     * walker / 8, id), part 0 for hi and 1 for lo */
    uint32_t c2 = (2u << 24) | (uint32_t)(walker >> 3);
    uint32_t hi = philox_word(o->seed, (uint32_t)site, s, c2, o->id, (walker & 7) >> 1);
    uint32_t lo = philox_word(o->seed, (uint32_t)site, s, c2 | (1u << 16), o->id, (walker & 7) >> 1);
    if (walker & 1) {
        hi &= 0xFFFFu;
        lo &= 0xFFFFu;
    } else {
        hi >>= 16;
        lo >>= 16;
    }
    return (hi << 16) | lo;
}

/* One sweep (Methods, "Local Monte Carlo sweeps"): every free spin of every replica once,
 * colour class by colour class; sites of one class share no edge, so their order is free. */
static void one_sweep(or_inst *o) {
    for (int32_t c = 0; c < o->ncol; ++c) {
        for (int32_t i = 0; i < o->N; ++i) {
            if (o->colour[i] != c || o->clamp[i] != 0) continue;
            for (int32_t r = 0; r < o->R; ++r) {
                int8_t *m = o->spins + (size_t)r * o->N;
                int32_t w = o->walker[r];
                int32_t I = o->h[i];
                for (int32_t a = o->adj_off[i]; a < o->adj_off[i + 1]; ++a)
                    I += o->adj_J[a] * m[o->adj_j[a]];
                if (o->update == 1) {
                    uint32_t u = local_uniform(o, i, w);
                    m[i] = (u < or_gibbs_threshold(o->beta[r], I)) ? 1 : -1;
                } else {
                    int32_t dE = 2 * m[i] * I;
                    if (dE <= 0) {
                        m[i] = (int8_t)-m[i];
                    } else {
                        uint32_t u = local_uniform(o, i, w);
                        if (u < or_metropolis_threshold(o->beta[r], dE)) m[i] = (int8_t)-m[i];
                    }
                }
            }
        }
    }
    o->sweeps++;
}

void or_sweeps(or_inst *o, int32_t n) {
    for (int32_t k = 0; k < n; ++k) one_sweep(o);
    recompute_energies(o);  /* Algorithm 1: exact energy of every replica */
}

/* Contextual proposals (Supplementary S3). The enabled slots, in ascending order, are
 * numbered j = 0, 1, ...; the random numbers of proposal j are bit j of these Philox words:
 *  - site i is kept (clamped) iff bits j of output words 0 .. context_log2-1 of
 *    Philox(i, event, 5 << 24 | 0xFF << 16, id) are all set (probability 2^-context_log2);
 *  - refill sweep t = (event - 1) * context_sweeps + k draws its 32-bit uniform at site i
 *    from the bit planes of Philox(i, t, 5 << 24 | (plane / 4) << 16, id), plane 0 the most
 *    significant bit, as the local moves of the walkers do. */
static uint32_t ctx_uniform(const or_inst *o, int32_t site, uint32_t t, int32_t j) {
    uint32_t u = 0;
    for (int k = 0; k < 32; ++k) {
        uint32_t c2 = (5u << 24) | ((uint32_t)(k >> 2) << 16);
        uint32_t word = philox_word(o->seed, (uint32_t)site, t, c2, o->id, k & 3);
        u |= ((word >> j) & 1u) << (31 - k);
    }
    return u;
}

static void context_candidate(const or_inst *o, int32_t r, int32_t j, int8_t *cand) {
    const int8_t *cur = o->spins + (size_t)r * o->N;
    memcpy(cand, cur, (size_t)o->N);
    uint8_t *kept = (uint8_t *)xcalloc((size_t)o->N, 1);
    for (int32_t i = 0; i < o->N; ++i) {
        int all = 1;
        for (int q = 0; q < o->ctx_log2; ++q) {
            uint32_t word = philox_word(o->seed, (uint32_t)i, (uint32_t)o->n_prop,
                                        (5u << 24) | (0xFFu << 16), o->id, q);
            all &= (int)((word >> j) & 1u);
        }
        kept[i] = (uint8_t)all;
    }
    for (int32_t k = 0; k < o->ctx_sweeps; ++k) {
        uint32_t t = (uint32_t)((o->n_prop - 1) * o->ctx_sweeps + k);
        for (int32_t c = 0; c < o->ncol; ++c) {
            for (int32_t i = 0; i < o->N; ++i) {
                if (o->colour[i] != c || kept[i]) continue;
                int32_t I = o->h[i];
                for (int32_t a = o->adj_off[i]; a < o->adj_off[i + 1]; ++a)
                    I += o->adj_J[a] * cand[o->adj_j[a]];
                int32_t dE = 2 * cand[i] * I;
                if (dE <= 0 || ctx_uniform(o, i, t, j) < or_metropolis_threshold(o->beta[r], dE))
                    cand[i] = (int8_t)-cand[i];
            }
        }
    }
    free(kept);
}

/* Global proposals (Algorithm 1, Eq. 2). */
void or_propose(or_inst *o) {
    o->n_prop++;
    if (o->source == 1) {
        int8_t *cand = (int8_t *)xcalloc((size_t)o->N, 1);
        int32_t j = 0;
        for (int32_t r = 0; r < o->R; ++r) {
            if (!o->prop[r]) continue;
            context_candidate(o, r, j, cand);   /* from the slot's state before this event */
            ++j;
            int32_t ET = energy_of(o, cand);
            double x = o->beta[r] * (double)(o->E[r] - ET);
            uint32_t u = philox_word(o->seed, (uint32_t)r, (uint32_t)o->n_prop, 4u << 24, o->id, 0);
            o->prop_att[r]++;
            if (o->rule == 1 || or_accept(x, u)) {
                memcpy(o->spins + (size_t)r * o->N, cand, (size_t)o->N);
                o->E[r] = ET;
                o->prop_acc[r]++;
            }
        }
        free(cand);
        return;
    }
    if (o->P <= 0) return;
    int8_t *cand = (int8_t *)xcalloc((size_t)o->N, 1);
    for (int32_t r = 0; r < o->R; ++r) {
        if (!o->prop[r]) continue;
        const int8_t *src = o->pool + ((size_t)r * o->P + o->cursor[r]) * o->N;
        for (int32_t i = 0; i < o->N; ++i) cand[i] = o->clamp[i] != 0 ? o->clamp[i] : src[i];
        int32_t ET = energy_of(o, cand);
        /* Eq. 2: x = beta_r (E_r - E^T); rule 2 adds the Hastings correction of the
         * independent proposal, log q(x_r) - log q(x^T) (Supplementary S2, the MH rule) */
        double x = o->beta[r] * (double)(o->E[r] - ET);
        if (o->rule == 2) {
            int64_t dl = law_weight(o, r, o->spins + (size_t)r * o->N) - law_weight(o, r, cand);
            x = x + ldexp((double)dl, -32);
        }
        uint32_t u = philox_word(o->seed, (uint32_t)r, (uint32_t)o->n_prop, 4u << 24, o->id, 0);
        o->prop_att[r]++;
        if (o->rule == 1 || or_accept(x, u)) {
            memcpy(o->spins + (size_t)r * o->N, cand, (size_t)o->N);
            o->E[r] = ET;
            o->prop_acc[r]++;
        }
        o->cursor[r] = (o->cursor[r] + 1) % o->P;
    }
    free(cand);
}

/* Replica exchange (Algorithm 1, Eq. 1): odd events pair slots (0,1),(2,3)...,
 * even events pair (1,2),(3,4)...; a swap exchanges configurations and energies. */
void or_exchange(or_inst *o) {
    o->n_ex++;
    int32_t first = (o->n_ex & 1) ? 0 : 1;
    int8_t *tmp = (int8_t *)xcalloc((size_t)o->N, 1);
    for (int32_t r = first; r + 1 < o->R; r += 2) {
        double x = (o->beta[r + 1] - o->beta[r]) * (double)(o->E[r + 1] - o->E[r]);
        uint32_t u = philox_word(o->seed, (uint32_t)r, (uint32_t)o->n_ex, 3u << 24, o->id, 0);
        o->swap_att[r]++;
        if (or_accept(x, u)) {
            int8_t *a = o->spins + (size_t)r * o->N, *b = o->spins + (size_t)(r + 1) * o->N;
            memcpy(tmp, a, (size_t)o->N); memcpy(a, b, (size_t)o->N); memcpy(b, tmp, (size_t)o->N);
            int32_t t = o->E[r]; o->E[r] = o->E[r + 1]; o->E[r + 1] = t;
            t = o->walker[r]; o->walker[r] = o->walker[r + 1]; o->walker[r + 1] = t;
            o->swap_acc[r]++;
        }
    }
    free(tmp);
}

/* Proposal schedule: after a cycle that ends at sweep count s, propose iff
 * every > 0, s >= start, (stop <= 0 or s <= stop) and (s - start) % every == 0. */
static int proposal_due(const or_inst *o) {
    if (o->every <= 0) return 0;
    int64_t s = o->sweeps;
    if (s < o->start) return 0;
    if (o->stop > 0 && s > o->stop) return 0;
    return ((s - o->start) % o->every) == 0;
}

void or_run_cycles(or_inst *o, int32_t n) {
    for (int32_t c = 0; c < n; ++c) {
        or_sweeps(o, o->M);
        if (proposal_due(o)) or_propose(o);
        or_exchange(o);
    }
}

void or_read(const or_inst *o, int8_t *spins, int32_t *E, int32_t *walker) {
    if (spins) memcpy(spins, o->spins, (size_t)o->R * o->N);
    if (E) memcpy(E, o->E, (size_t)o->R * 4);
    if (walker) memcpy(walker, o->walker, (size_t)o->R * 4);
}

void or_write(or_inst *o, const int8_t *spins, const int32_t *walker) {
    memcpy(o->spins, spins, (size_t)o->R * o->N);
    if (walker) memcpy(o->walker, walker, (size_t)o->R * 4);
    recompute_energies(o);
}

void or_counters(const or_inst *o, int64_t out[3]) {
    out[0] = o->sweeps; out[1] = o->n_ex; out[2] = o->n_prop;
}

void or_set_counters(or_inst *o, const int64_t in[3], const int32_t *cursors) {
    o->sweeps = in[0]; o->n_ex = in[1]; o->n_prop = in[2];
    if (cursors) memcpy(o->cursor, cursors, (size_t)o->R * 4);
}

void or_cursors(const or_inst *o, int32_t *cursors) {
    memcpy(cursors, o->cursor, (size_t)o->R * 4);
}

void or_stats(const or_inst *o, int64_t *swap_acc, int64_t *swap_att,
              int64_t *prop_acc, int64_t *prop_att) {
    for (int32_t r = 0; r < o->R; ++r) {
        if (swap_acc && r + 1 < o->R) swap_acc[r] = o->swap_acc[r];
        if (swap_att && r + 1 < o->R) swap_att[r] = o->swap_att[r];
        if (prop_acc) prop_acc[r] = o->prop_acc[r];
        if (prop_att) prop_att[r] = o->prop_att[r];
    }
}

/* 1 if site i has a free neighbour of colour c */
static int free_neighbour_coloured(const or_inst *o, int32_t i, int32_t c) {
    for (int32_t a = o->adj_off[i]; a < o->adj_off[i + 1]; ++a) {
        int32_t j = o->adj_j[a];
        if (o->clamp[j] == 0 && o->colour[j] == c) return 1;
    }
    return 0;
}

/* Colour classes of at most `cap` free sites (the colour_cap option of the library; general
 * graphs only, a lattice keeps its checkerboard). The DSATUR classes are a proper colouring
 * of the free sites; so is the result, which only moves a site into a class holding none of
 * its free neighbours. With k = max(ncol, ceil(free sites / cap)) colours to use: while some
 * class holds more than cap free sites, take the fullest (the lowest colour among equally
 * full ones) and scan its free sites from the highest index down; the first one that has no
 * free neighbour in some other class holding fewer than cap free sites moves to the least full
 * such class (the lowest colour among equally full ones). Stop when no class is over cap or
 * no site of the fullest can move. Clamped sites keep their colours. Colours left without a
 * site are removed and the others renumbered in order. Returns the number of colours. */
int32_t or_cap_colours(or_inst *o, int32_t cap) {
    if (cap <= 0 || o->L > 0) return o->ncol;
    int32_t nfree = 0;
    for (int32_t i = 0; i < o->N; ++i) nfree += (o->clamp[i] == 0);
    int32_t k = (nfree + cap - 1) / cap;
    if (k < o->ncol) k = o->ncol;
    int32_t *fill = (int32_t *)xcalloc((size_t)k, 4);
    for (int32_t i = 0; i < o->N; ++i)
        if (o->clamp[i] == 0) fill[o->colour[i]]++;
    for (;;) {
        int32_t over = -1;
        for (int32_t c = 0; c < k; ++c)
            if (fill[c] > cap && (over < 0 || fill[c] > fill[over])) over = c;
        if (over < 0) break;
        int32_t moved = 0;
        for (int32_t i = o->N - 1; i >= 0 && !moved; --i) {
            if (o->clamp[i] != 0 || o->colour[i] != over) continue;
            int32_t to = -1;
            for (int32_t c = 0; c < k; ++c) {
                if (c == over || fill[c] >= cap || free_neighbour_coloured(o, i, c)) continue;
                if (to < 0 || fill[c] < fill[to]) to = c;
            }
            if (to >= 0) {
                o->colour[i] = to;
                fill[over]--;
                fill[to]++;
                moved = 1;
            }
        }
        if (!moved) break;
    }
    int32_t *renum = (int32_t *)xcalloc((size_t)k, 4);
    for (int32_t c = 0; c < k; ++c) renum[c] = -1;
    for (int32_t i = 0; i < o->N; ++i) renum[o->colour[i]] = 1;
    int32_t n = 0;
    for (int32_t c = 0; c < k; ++c)
        if (renum[c] > 0) renum[c] = n++;
    for (int32_t i = 0; i < o->N; ++i) o->colour[i] = renum[o->colour[i]];
    free(renum);
    free(fill);
    o->ncol = n;
    return n;
}

int32_t or_colouring(const or_inst *o, int32_t *colour) {
    if (colour) memcpy(colour, o->colour, (size_t)o->N * 4);
    return o->ncol;
}

int32_t or_bitplane(const or_inst *o) { return o->bitplane; }
