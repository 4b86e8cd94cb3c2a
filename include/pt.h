/*
 * pt.h - C ABI of the GB300 (sm_103a) library for parallel tempering with global proposals,
 * i.e. Transformer-Augmented Parallel Tempering (TAPT), arXiv 2509.23043, Algorithm 1.
 *
 * The library runs, for a batch of independent Ising instances, the cycle of Algorithm 1:
 * M local sweeps of every replica (colour class by colour class), the exact energy of every
 * replica, the global proposal move on the proposal-enabled replicas, and replica exchange
 * between neighbouring temperatures with alternating parity. Every step runs in CUDA kernels;
 * the host code only validates, lays out and launches.
 *
 * Conventions (shared by every call)
 *  - spins m in {-1,+1}; energy E(m) = -sum_edges J m_i m_j - sum_i h_i m_i (Supplementary
 *    S4, the paper's Ising energy convention); local field I_i = sum_j J_ij m_j + h_i
 *    (Methods, local Monte Carlo sweeps);
 *  - replica (temperature) slots r = 0..R-1 run hot -> cold: beta ascending;
 *  - every output is in slot order, whatever internal relabelling the library uses;
 *  - all host pointers are owned by the caller and are read (or written) during the call
 *    only; nothing keeps a reference to them;
 *  - all device work is ordered on the CUDA stream given at creation (or pt_set_stream);
 *    calls that return host data synchronise that stream;
 *  - errors: every call returns a pt_status; pt_last_error() gives a message for the last
 *    failing call of the calling thread. Nothing is thrown across the ABI. A context is not
 *    thread safe.
 *  - a context belongs to the device that was current when it was created: every call on it
 *    returns PT_ESTATE, with a message naming both devices, when another device is current.
 */
#ifndef PT_H
#define PT_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PT_OK = 0,
    PT_EINVAL = 1,    /* an argument is out of range or inconsistent */
    PT_ENOMEM = 2,    /* a device or host allocation failed */
    PT_ECUDA = 3,     /* a CUDA call failed (message holds its error string) */
    PT_ETIMEOUT = 4,  /* a bounded device-side wait gave up */
    PT_ESTATE = 5,    /* the call is not valid in the context's current state */
    PT_ENOTSUP = 6    /* valid input that this build does not support (e.g. too large) */
} pt_status;

typedef struct pt_ctx pt_ctx;   /* opaque; owns all device memory of a batch */

/* One Ising instance: the energy-function input of Algorithm 1, with its
 * temperature ladder {beta_r} and proposal-enabled set R_prop.
 *  instance_id   caller's identifier; it keys every random stream of the instance, so an
 *                instance evolves identically whatever batch or position it runs in.
 *  n_spins       N >= 1 (lattice engine: N <= 8192; an instance whose spins and neighbour
 *                table do not fit one block's shared memory keeps both in global memory,
 *                except with contextual proposals (PT_ENOTSUP); graph engine: N <= 65535, and
 *                the instance's state and tables must fit in one block's shared memory, else
 *                PT_ENOTSUP).
 *  lattice_L     > 0: a periodic L^3 lattice (N = L^3, L >= 2); the edges must then be the
 *                3N bonds in canonical order: for site n = x + L(y + L z), its +x, +y, +z
 *                bonds, in that order (Methods, benchmark instances: 3D spin glass). The
 *                lattice is coloured (x+y+z) mod 2 for even L and by a 3-colouring for odd L.
 *                0: a general graph, coloured by DSATUR (Methods, graph coloring).
 *  n_edges, edge_i, edge_j, edge_J
 *                undirected couplings J_ij (int32), one per row; parallel edges are summed
 *                by the energy; self loops are rejected.
 *  h             N local fields, or NULL for none.
 *  clamp         N values: 0 free, +1/-1 clamped to that spin; or NULL. Clamped spins are
 *                never updated (Supplementary S4, output bits clamped).
 *  n_replicas    R, 1 <= R <= 128.
 *  beta          R inverse temperatures, ascending, finite, >= 0.
 *  prop_enabled  R flags (nonzero = slot receives global proposals, the set R_prop), or
 *                NULL for none. */
typedef struct {
    uint32_t instance_id;
    int32_t n_spins;
    int32_t lattice_L;
    int32_t n_edges;
    const int32_t *edge_i;
    const int32_t *edge_j;
    const int32_t *edge_J;
    const int32_t *h;
    const int8_t *clamp;
    int32_t n_replicas;
    const double *beta;
    const uint8_t *prop_enabled;
} pt_instance_desc;

/* Run parameters, shared by every instance of a context.
 *  update            0 Metropolis (flip iff dE <= 0 or u < floor(2^32 exp(-beta dE))),
 *                    1 Gibbs / heat bath (m = +1 iff u < floor(2^32 (1 + tanh(beta I)) / 2)),
 *                    the paper's rule (Methods, Eq. for the Gibbs update). u is a 32-bit
 *                    Philox4x32-10 draw; thresholds are computed in FP64, capped at 2^32-1.
 *  sweeps_per_cycle  M of Algorithm 1 (>= 1).
 *  propose_every, propose_start, propose_stop
 *                    proposal schedule of pt_run_cycles: after a cycle that ends at sweep
 *                    count s, a proposal event happens iff propose_every > 0, s >= start,
 *                    (stop <= 0 or s <= stop) and (s - start) % propose_every == 0.
 *                    (Fig. 3: start 100, then every sweep; Fig. S3: stop after 100.)
 *  pool_size         P, proposal-pool capacity per (instance, slot); 0 = no pools.
 *  seed              64-bit key of every random stream.
 *  threads_per_block 0 = automatic choice; else a multiple of 32 in [32, 512].
 *  proposal_rule     acceptance of a global proposal: 0 = the paper's Delta-E-only rule
 *                    min[1, exp(beta_r (E_r - E^T))] (Eq. 2, an optimization heuristic);
 *                    1 = always accept, which is the independent Metropolis-Hastings move
 *                    when the pool entries are exact draws from the slot's Boltzmann law (the
 *                    proposal-probability correction then cancels the Boltzmann ratio;
 *                    Supplementary S2); 2 = the independent Metropolis-Hastings move
 *                    min[1, pi(x') q(x) / (pi(x) q(x'))] (Supplementary S2, the MH rule) for
 *                    pools drawn from a product-Bernoulli law q given per slot by
 *                    pt_load_proposal_law (pool proposals only; a slot whose law was never
 *                    loaded has the uniform law, for which the rule is the Delta-E-only one).
 *                    Other values: PT_EINVAL.
 *  proposal_source   0 = proposals from the pools (pt_load_proposals...); 1 = contextual
 *                    proposals (Supplementary S3), lattice engine with Metropolis sweeps
 *                    (update 0) only: at each event every
 *                    proposal-enabled slot (at most 32 per instance) copies its configuration,
 *                    keeps each site with probability 2^-context_log2 (1, 2 or 3: 50, 25 or
 *                    12.5 %), refills the other sites by context_sweeps (>= 1) Metropolis
 *                    sweeps at its beta, and the result is accepted by proposal_rule. Pools
 *                    are not used. Violations: PT_EINVAL, or PT_ENOTSUP for the graph engine,
 *                    Gibbs sweeps or more than 32 enabled slots.
 *  colour_cap        graph engine, general graphs (lattice_L = 0): 0 = the DSATUR colour
 *                    classes (Methods, graph coloring) as they are; C > 0 = classes of at most
 *                    C free sites where the graph allows it: with k = max(DSATUR's count,
 *                    ceil(free sites / C)) colours available, repeatedly take the largest class
 *                    above C (lowest colour among equals) and move its highest-index free site
 *                    that has no free neighbour in some other class below C to the smallest such
 *                    class (lowest colour among equals), until no class is above C or none of
 *                    its sites can move; clamped sites keep their colours; empty colours are
 *                    dropped, the others keeping their order. Any proper colouring gives a valid
 *                    sweep; C = 32 fills the 32-site passes of a 128-thread block at R <= 32.
 *                    More than 32 colours: PT_ENOTSUP. Negative: PT_EINVAL.
 */
typedef struct {
    int32_t update;
    int32_t sweeps_per_cycle;
    int32_t propose_every;
    int32_t propose_start;
    int32_t propose_stop;
    int32_t pool_size;
    uint64_t seed;
    int32_t threads_per_block;
    int32_t proposal_rule;
    int32_t proposal_source;
    int32_t context_log2;
    int32_t context_sweeps;
    int32_t colour_cap;
} pt_config;

/* Create a batch of n >= 1 instances (all lattices with J = +-1 and no field or clamp, which
 * run on the bit-packed lattice engine under either rule, or all otherwise, which run on the
 * int8 graph engine: one engine per context), allocate its device memory (cudaMallocAsync
 * on `cuda_stream`, a cudaStream_t or NULL for the legacy stream), draw the random initial
 * state of every replica (Algorithm 1, initialisation) and compute
 * its energies. On success *out owns everything; release it with pt_destroy. */
pt_status pt_create_instances(pt_ctx **out, const pt_instance_desc *descs, int32_t n,
                              const pt_config *cfg, void *cuda_stream);

/* Copy `count` configurations (host, int8 +-1, row-major [count][N]) into the proposal pool
 * of instance `inst`, slot `replica`, at positions first .. first+count-1 (< pool_size).
 * These are the pre-generated proposals S^T_r at beta_r of Algorithm 1. */
pt_status pt_load_proposals(pt_ctx *ctx, int32_t inst, int32_t replica, const int8_t *spins,
                            int32_t count, int32_t first);

/* Proposal law of the pool of instance `inst`, slot `replica`, for proposal_rule 2 (no
 * counterpart call in the paper; the law is the q of Supplementary S2's MH rule): the pool
 * entries are independent draws from q(x) = prod_i p_i^[x_i=+1] (1 - p_i)^[x_i=-1], with
 * p_plus[i] = p_i, N doubles in (0, 1) (host, copied during the call). The library keeps the
 * log-odds log(p_i / (1 - p_i)) rounded to multiples of 2^-32, so log q(x) - log q(x') is an
 * exact integer sum; clamped sites carry no weight. At a proposal event the acceptance
 * exponent is x = beta_r (E_r - E^T) + log q(x_r) - log q(x^T), in FP64. PT_ESTATE unless
 * the context was created with proposal_rule 2; PT_EINVAL for a value outside (0, 1).
 * Synchronises. */
pt_status pt_load_proposal_law(pt_ctx *ctx, int32_t inst, int32_t replica, const double *p_plus);

/* Bulk load of bit-packed pool entries for every instance and slot: host words laid out
 * [count][instance][slot][ceil(N_instance/32)] uint32 (bit i%32 of word i/32 set iff spin i
 * is +1), written to pool positions first .. first+count-1. Stream ordered: the host buffer
 * must stay valid (ideally pinned) until the stream reaches the copy. */
pt_status pt_load_proposals_packed(pt_ctx *ctx, const uint32_t *words, int32_t first,
                                   int32_t count);

/* Bulk load of bit-packed pool entries for one instance: host words [count][R][ceil(N/32)]
 * (same bit order as above) written to positions first .. first+count-1 of its slots.
 * Synchronises (the host buffer may be freed on return). */
pt_status pt_load_proposals_inst_packed(pt_ctx *ctx, int32_t inst, const uint32_t *words,
                                        int32_t first, int32_t count);

/* Inverse of pt_load_proposals_packed: copy pool positions first .. first+count-1 of every
 * instance and slot to host words in the same layout. Synchronises. */
pt_status pt_read_proposals_packed(pt_ctx *ctx, uint32_t *words, int32_t first, int32_t count);

/* Copy the current configuration of every slot of every instance of `src` into pool
 * position `entry` of the same instance and slot of `dst` (same batch shape), on the
 * device. Used to build pools from long PT runs of the method itself. */
pt_status pt_capture_proposals(pt_ctx *dst, const pt_ctx *src, int32_t entry);

/* n_sweeps local sweeps of every replica of every instance (Methods: one sweep updates
 * every free spin once), then the exact energy of every replica (the energy step of Algorithm 1). */
pt_status pt_sweep(pt_ctx *ctx, int32_t n_sweeps);

/* One global-proposal event for every instance: for each r in R_prop, take the next pool
 * entry S^T_r (cursor advances by one mod P whether or not it is accepted), overwrite its
 * clamped spins, compute E^T_r exactly, and accept with min[1, exp(beta_r (E_r - E^T_r))]
 * (Eq. 2, evaluated in FP64). Uses the energies of the last sweep. */
pt_status pt_global_propose(pt_ctx *ctx);

/* One replica-exchange event for every instance: event n (1-based) pairs slots (0,1),(2,3)..
 * when n is odd and (1,2),(3,4).. when n is even, and swaps the configurations and energies
 * of a pair with min[1, exp((beta_{r+1}-beta_r)(E_{r+1}-E_r))] (Eq. 1, FP64). */
pt_status pt_exchange(pt_ctx *ctx);

/* n_cycles cycles of Algorithm 1, fused on the device: M sweeps, energies, a proposal event
 * when the schedule says so, an exchange event. */
pt_status pt_run_cycles(pt_ctx *ctx, int32_t n_cycles);

/* Energies of every replica, the output {E_r} of Algorithm 1 (exact integer energies, the
 * energy step of each cycle): host int32 [sum over instances of R], instance by instance,
 * slot order. Synchronises. */
pt_status pt_energies(pt_ctx *ctx, int32_t *out);

/* Same output {E_r} of Algorithm 1, into caller device memory (int32 [sum over instances of
 * R], the same order; stream ordered, no synchronisation). */
pt_status pt_energies_device(pt_ctx *ctx, int32_t *dev_out);

/* State of one instance, the outputs {S_r} and {E_r} of Algorithm 1: spins int8 [R][N]
 * (+-1) and energies int32 [R] in slot order (either may be NULL). Allocates a temporary
 * device buffer for the unpacked spins (stream ordered). Synchronises. */
pt_status pt_read_state(pt_ctx *ctx, int32_t inst, int8_t *spins, int32_t *E);

/* Same result as pt_read_state, for callers that must not allocate device memory while they
 * run: a real-time or latency-bounded host loop that keeps every allocation (and the
 * implicit synchronisation cudaMalloc/cudaFree can cause) out of its steady state, or a
 * process whose device memory is fully budgeted up front. The paper has no counterpart;
 * this is a property of the library only.
 *  - Allocates nothing: the unpacked spins pass through a fixed device buffer of 256 KiB
 *    (a file-scope __device__ array; every GPU that loads the library holds it until exit),
 *    and the energies through the context's own buffer made at creation.
 *  - R * N above 262144 returns PT_ENOTSUP with a message.
 *  - The first call on a device looks up the buffer's device address (once per device and
 *    CUDA context, with the context's device current); make that first call before any
 *    stream capture. After a device reset the runtime creates a new CUDA context, and the
 *    next call looks the address up again.
 *  - All calls share the one buffer, which keeps the last call's contents. Calls are
 *    stream ordered and synchronise, so calls from one thread never overlap; calls from
 *    several host threads at once would race on the buffer and must be serialised by the
 *    caller.
 * spins (int8 [R][N], slot order) and E (int32 [R]) are host buffers, either may be NULL. */
pt_status pt_read_state_noalloc(pt_ctx *ctx, int32_t inst, int8_t *spins, int32_t *E);

/* Walker identity held by each slot (int32 [R]): a configuration keeps its walker id when
 * an exchange moves it to another slot. Synchronises. */
pt_status pt_read_walkers(pt_ctx *ctx, int32_t inst, int32_t *walker);

/* Overwrite the state of one instance (checkpoint restore): spins int8 [R][N] in slot
 * order, the walker id of each slot (a permutation of 0..R-1), the counters
 * {sweeps, exchange events, proposal events} and the pool cursors int32 [R] (may be NULL).
 * Energies are recomputed on the device. */
pt_status pt_write_state(pt_ctx *ctx, int32_t inst, const int8_t *spins,
                         const int32_t *walker, const int64_t counters[3],
                         const int32_t *cursors);

/* Counters {sweeps, exchange events, proposal events} of one instance, and its pool cursors
 * int32 [R] (may be NULL). Synchronises. */
pt_status pt_read_counters(pt_ctx *ctx, int32_t inst, int64_t counters[3], int32_t *cursors);

/* Acceptance counters of one instance (Figs. S5, S6): swaps accepted/attempted per pair
 * (slot r with r+1) int64 [R-1], proposals accepted/attempted per slot int64 [R]. Any may be
 * NULL. Synchronises. */
pt_status pt_read_stats(pt_ctx *ctx, int32_t inst, int64_t *swap_acc, int64_t *swap_att,
                        int64_t *prop_acc, int64_t *prop_att);

/* Batch shape: number of instances, engine (0 bit-packed lattice engine, 1 graph engine),
 * threads per block used, and the instance's R and N (inst may be -1 for batch values only).*/
pt_status pt_info(const pt_ctx *ctx, int32_t inst, int32_t info[6]);

/* Size-class groups: instances of one shape (lattice: same L and walker-block count) are
 * launched together with one block shape; the groups of a context run concurrently, each
 * on its own stream forked from the context's stream. group = -1: info[0] = number of
 * groups. Else info = {members, threads per block, shared-memory bytes, first member}. */
pt_status pt_group_info(const pt_ctx *ctx, int32_t group, int32_t info[4]);

/* Autotune the block size of every group: each candidate runs probe_cycles cycles from a
 * device snapshot of the state, which is restored afterwards (the run is unchanged). The
 * chosen sizes are written to threads_out [groups] (may be NULL). */
pt_status pt_autotune(pt_ctx *ctx, int32_t probe_cycles, int32_t *threads_out);

/* pt_run_cycles through a CUDA graph: the first call for a cycle count captures the launches
 * of every group (fork/join over the group streams) and later calls replay it. Ordered on
 * the context's stream like every other call. */
pt_status pt_run_cycles_graph(pt_ctx *ctx, int32_t n_cycles);

/* Continuous batching support (lattice engine). pt_set_instance replaces the instance in
 * slot `inst` by a new one of the same shape (same L and R): couplings, ladder, proposal
 * set and instance id; its state is redrawn from the new id, its counters, cursors and
 * statistics reset, and the slot activated. pt_set_active(ctx, inst, 0) makes every later
 * launch skip the slot (its state is kept); 1 makes it take part again. */
pt_status pt_set_instance(pt_ctx *ctx, int32_t inst, const pt_instance_desc *desc);
pt_status pt_set_active(pt_ctx *ctx, int32_t inst, int32_t active);

/* Change the stream of all later calls. */
pt_status pt_set_stream(pt_ctx *ctx, void *cuda_stream);

/* Calibration of the integer pipes (no counterpart in the paper): the sustained rate, in
 * operations per second, of independent 32-bit lop3 operations (kind 0, the integer ALU pipe
 * that bounds the lattice sweep) or 32-bit multiply-adds (kind 1, the pipe of Philox's
 * products), measured on the current device by a full-occupancy kernel on the legacy stream;
 * *ms (may be NULL) receives the best launch time. It allocates and frees a small device
 * buffer and synchronises. PT_EINVAL for another kind or a NULL ops_per_s. */
pt_status pt_calibrate_int(int32_t kind, double *ops_per_s, double *ms);

/* Measured shared-memory load bandwidth of the current device, the peak of the lattice
 * kernel's second roofline (its working set lives in shared memory): every warp of 4 blocks
 * of 512 threads per SM reads 32 consecutive 16-byte words per load, without bank conflicts,
 * from a 16 KB buffer. *bytes_per_s receives the bytes loaded per second of the best of three
 * timed launches, *ms (may be NULL) that launch's time. It allocates and frees a small device
 * buffer and synchronises. PT_EINVAL for a NULL bytes_per_s. */
pt_status pt_calibrate_smem(double *bytes_per_s, double *ms);

/* Release all device memory (stream ordered) and the context. NULL is allowed. */
pt_status pt_destroy(pt_ctx *ctx);

/* Message of the last failing call on the calling thread ("" if none). */
const char *pt_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
