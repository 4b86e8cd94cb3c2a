/*
 * Plain, slow, sequential CPU oracle for parallel tempering with global proposals
 * (Transformer-Augmented Parallel Tempering, Algorithm 1 of arXiv 2509.23043).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load this library. The product path (the CUDA library) shares no
 * code with it and never calls it.
 *
 * Every function restates the paper's definition step by step in the paper's order. The
 * readings taken where the paper is silent are the same ones the CUDA library follows:
 *   - spins m in {-1,+1}; E(m) = -sum_edges J m_i m_j - sum_i h_i m_i (Supplementary S4);
 *   - local field I_i = sum_j J_ij m_j + h_i (Methods, Eq. for I_i);
 *   - Gibbs: new m = +1 iff u < T_G(beta, I), T_G = floor(2^32 (1 + tanh(beta I)) / 2)
 *     (Methods, Gibbs update; u uniform 32-bit);
 *   - Metropolis: flip iff dE <= 0 or u < T_M(beta, dE), T_M = floor(2^32 exp(-beta dE));
 *     both thresholds are capped at 2^32 - 1;
 *   - replica exchange with P_swap = min[1, exp(dbeta dE)] (Eq. 1) and global proposal
 *     with P_accept = min[1, exp(beta_r (E_r - E^T))] (Eq. 2): accept iff x >= 0 or
 *     u + 1 <= 2^32 exp(x), evaluated in FP64;
 *   - random numbers from Philox4x32-10 (Salmon et al., SC'11) keyed by the 64-bit seed,
 *     counters as documented in pt_oracle.c.
 *
 * Parity is pinned by the tests under tests/ (Philox known-answer vectors, brute-force
 * Boltzmann distributions, exact transition matrices, closed forms); see each test.
 */
#ifndef PT_ORACLE_H
#define PT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct or_inst or_inst;

/* Philox4x32-10: out = Philox(ctr, key). */
void or_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Local-move thresholds (see header comment). */
uint32_t or_metropolis_threshold(double beta, int32_t dE);
uint32_t or_gibbs_threshold(double beta, int32_t I);
/* Global-move decision: 1 iff accepted. */
int or_accept(double x, uint32_t u);

/* Energy of one configuration (spins +-1). */
int64_t or_energy(int32_t n, int32_t n_edges, const int32_t *ei, const int32_t *ej,
                  const int32_t *eJ, const int32_t *h, const int8_t *spins);

/* Create one instance. Inputs are copied. update: 0 Metropolis, 1 Gibbs.
 * propose_every = 0 disables proposals in or_run_cycles; propose_stop <= 0 means never stop.
 * proposal_rule: 0 = the Delta-E-only rule of Eq. 2; 1 = always accept (the independent
 * Metropolis-Hastings move for proposals drawn exactly from the slot's Boltzmann law, whose
 * correction cancels the Boltzmann ratio; Supplementary S2); 2 = the independent
 * Metropolis-Hastings move min[1, pi(x')q(x) / (pi(x)q(x'))] for pools drawn from a
 * product-Bernoulli law q given per slot by or_load_law (pool proposals only).
 * proposal_source: 0 = the pool; 1 = contextual proposals (Supplementary S3): a copy of the
 * slot's configuration with every spin kept (clamped) with probability 2^-context_log2
 * (1..3) and the others refilled by context_sweeps (>= 1) Metropolis sweeps at the slot's
 * beta. Contextual proposals need the bit-plane lattice case and at most 32 enabled slots.
 * Returns NULL on invalid input. */
or_inst *or_create(uint32_t instance_id, int32_t n_spins, int32_t lattice_L,
                   int32_t n_edges, const int32_t *ei, const int32_t *ej, const int32_t *eJ,
                   const int32_t *h, const int8_t *clamp,
                   int32_t n_replicas, const double *beta, const uint8_t *prop_enabled,
                   int32_t update, int32_t sweeps_per_cycle, int32_t propose_every,
                   int32_t propose_start, int32_t propose_stop, uint64_t seed,
                   int32_t pool_size, int32_t proposal_rule, int32_t proposal_source,
                   int32_t context_log2, int32_t context_sweeps);
void or_destroy(or_inst *o);

/* Proposal law of slot r for proposal_rule 2: p_plus[i] = P(spin i = +1), in (0, 1). Its
 * log-odds are kept rounded to multiples of 2^-32. Returns nonzero on invalid input. */
int or_load_law(or_inst *o, int32_t r, const double *p_plus);

/* Store `count` configurations (+-1) for replica slot r at pool positions first.. */
int or_load_pool(or_inst *o, int32_t r, const int8_t *spins, int32_t count, int32_t first);

/* n local sweeps of every replica, then energies recomputed from scratch. */
void or_sweeps(or_inst *o, int32_t n);
/* One global-proposal event (proposal-enabled replicas only). */
void or_propose(or_inst *o);
/* One replica-exchange event; parity alternates with the event number. */
void or_exchange(or_inst *o);
/* n cycles of Algorithm 1: M sweeps, energies, proposals when scheduled, exchange. */
void or_run_cycles(or_inst *o, int32_t n);

/* Read the state in temperature-slot order: spins [R][N], energies [R], walker ids [R]. */
void or_read(const or_inst *o, int8_t *spins, int32_t *E, int32_t *walker);
/* Overwrite the state (for checkpoint tests): same layout as or_read. */
void or_write(or_inst *o, const int8_t *spins, const int32_t *walker);
/* counters: [sweeps, exchange events, proposal events]. */
void or_counters(const or_inst *o, int64_t out[3]);
void or_set_counters(or_inst *o, const int64_t in[3], const int32_t *cursors);
void or_cursors(const or_inst *o, int32_t *cursors);
/* acceptance statistics: swap accepted/attempted per pair [R-1], proposals per slot [R]. */
void or_stats(const or_inst *o, int64_t *swap_acc, int64_t *swap_att,
              int64_t *prop_acc, int64_t *prop_att);
/* colour of every site (clamped sites included) and the number of colours. */
int32_t or_colouring(const or_inst *o, int32_t *colour);
/* Rebalance the colour classes to at most cap free sites each (general graphs; see the .c
 * file); call before the first sweep. Returns the number of colours. */
int32_t or_cap_colours(or_inst *o, int32_t cap);
/* 1 when the instance uses the bit-plane random layout (lattice, +-1, no field, no clamps;
 * Metropolis or Gibbs), else 0. */
int32_t or_bitplane(const or_inst *o);

#ifdef __cplusplus
}
#endif
#endif
