/*
 * icmpt.h -- C ABI of the GB300 library for parallel tempering (PT) with
 * isoenergetic cluster moves (ICM) on Ising spin glasses (Zhu, Ochoa,
 * Katzgraber, "Efficient Cluster Algorithm for Spin Glasses in Any Space
 * Dimension").
 *
 * One simulation step of every instance is, in this order (the paper's
 * "Isoenergetic cluster algorithm", steps 1, 2a, 2b, 3):
 *   1  one Metropolis sweep of each of the 2 N_T replicas (checkerboard:
 *      all sites of colour 0, then all of colour 1);
 *   2a at each ICM temperature, if more than N/2 sites have q_i = -1, the
 *      spins of copy 1 are all reversed;
 *   2b at each ICM temperature (T_k <= T_icm), one Houdayer cluster move:
 *      a uniformly chosen site with q_i = s_i^a s_i^b = -1 seeds the
 *      connected component of {i : q_i = -1}, which is flipped in both copies;
 *   3  one PT pass per copy over the neighbouring temperature pairs;
 *   then the observables of "Benchmark model and observables" (energy, site
 *   overlap, link overlap q_l, P(q)) are accumulated when t >= t_meas.
 *
 * H = -sum_<ij> J_ij s_i s_j, each bond once.
 *
 * Conventions for every entry point:
 *  - Return value: ICM_OK (0) or a negative icm_status.  No C++ exception
 *    crosses the ABI.  After an error, icm_last_error(ctx) describes it.
 *  - Handles are opaque and owned by the library; free them with *_destroy.
 *  - Input arrays are read during the call (host arrays are copied into
 *    device memory before the call returns); the caller keeps ownership.
 *  - Output buffers belong to the caller.  Pointers are host pointers unless
 *    ICM_DEVICE_PTR is set in `flags`, in which case they are device
 *    pointers on the context's device (e.g. the data of a CUDA torch tensor).
 *  - Device work is enqueued on the context's stream and is asynchronous;
 *    the read functions and icm_sync wait for it.
 *  - A context is used by one host thread at a time.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = the 64-bit
 * seed, counters keyed by logical coordinates only (never by batch slot or
 * thread), so that every instance's trajectory is a function of
 * (seed, instance id, inputs) alone:
 *   Metropolis update of replica position r = 2k+c at site i, sweep t:
 *       word r&3 of ctr {i, t, r>>2, inst}
 *   ICM seed at temperature k, sweep t:     word 0 of ctr {k, t, 0, 1<<24 | inst}
 *   PT decision, copy c, pair (k,k+1):      word 0 of ctr {k, t, c, 2<<24 | inst}
 */
#ifndef ICMPT_H
#define ICMPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t icm_status;
#define ICM_OK 0
#define ICM_ERR_ARG (-1)      /* invalid argument */
#define ICM_ERR_OOM (-2)      /* device or host allocation failed */
#define ICM_ERR_BUDGET (-3)   /* request does not fit the memory budget */
#define ICM_ERR_CUDA (-4)     /* a CUDA runtime call failed */
#define ICM_ERR_TIMEOUT (-5)  /* a bounded device wait expired */
#define ICM_ERR_STATE (-6)    /* call not valid in the current state */
#define ICM_ERR_UNSUPPORTED (-7) /* size or feature beyond this build's limits */
#define ICM_PENDING 1          /* icm_query / server results: work still running (not an error) */
#define ICM_CANCELLED 2        /* server results: the request was cancelled (not an error) */

/* Lattice kinds ("Results in two and three space dimensions, as well as on
 * the nonplanar chimera topology").
 *   ICM_SQUARE2D : L x L periodic square lattice, site i = x + L y,
 *                  bond b = 2i + d to the +x (d=0) / +y (d=1) neighbour.
 *   ICM_CUBIC3D  : L^3 periodic cubic lattice, site i = x + L(y + L z),
 *                  bond b = 3i + d to the +x / +y / +z neighbour.
 *   ICM_CHIMERA  : C_M, M x M unit cells of K_{4,4}, open boundary,
 *                  site i = 8(rM + c) + 4h + k (shore h, index k).  Bonds:
 *                  in-cell b = 16 cell + 4 k0 + k1 joins (h=0,k0)-(h=1,k1);
 *                  then (r,c,0,k)-(r+1,c,0,k) at b = 16M^2 + 4(rM+c) + k;
 *                  then (r,c,1,k)-(r,c+1,1,k) at
 *                  b = 16M^2 + 4M(M-1) + 4(r(M-1)+c) + k.
 *   ICM_HYPERCUBIC4D : L^4 periodic hypercubic lattice ("any space
 *                  dimension"), site i = x + L(y + L(z + L w)), bond
 *                  b = 4i + d to the +x / +y / +z / +w neighbour.
 * Lattices need an even L >= 2 (the two-colouring); L = 2 keeps the doubled
 * bonds of the torus as separate bonds.  At most 65535 sites.               */
typedef enum { ICM_SQUARE2D = 0, ICM_CUBIC3D = 1, ICM_CHIMERA = 2, ICM_HYPERCUBIC4D = 3 } icm_lattice;

/* Disorder ("the interactions J_ij are selected from a Gaussian distribution
 * with mean zero and variance J^2 = 1"; bimodal disorder in the discussion of
 * degenerate ground states).
 *   ICM_PM_J  : J = +-1, int8 per bond; integer arithmetic, results are
 *               bit-exact functions of the inputs.
 *   ICM_GAUSS : J real, float32 per bond; fp32 arithmetic.
 * Dilution (the introduction's remedy for the cluster move in three
 * dimensions): a coupling of exactly 0 means the bond is absent.  It is no
 * edge of the cluster graph and is not counted in the link overlap, whose
 * normalisation is the number of bonds present (icm_read_bond_counts).  On
 * an instance with an absent bond, a zero-energy Metropolis proposal is
 * accepted with probability 1/2 instead of always: sites of degree 0-2 make
 * the checkerboard sweep with deterministic zero-energy flips non-ergodic.
 * Detection is automatic, per instance.                                  */
typedef enum { ICM_PM_J = 0, ICM_GAUSS = 1 } icm_disorder;

#define ICM_DEVICE_PTR 1u     /* flags: the buffer is a device pointer */

typedef struct icm_ctx icm_ctx;
typedef struct icm_batch icm_batch;

/* Which steps run at sweep t (each applies when t % every == 0; 0 = never). */
typedef struct {
    int32_t icm_every;        /* steps 2a/2b; default 1 */
    int32_t swap_every;       /* step 3; default 1 */
    int32_t enable_2a;        /* step 2a on/off; default 1 */
    int32_t enable_metropolis;/* step 1 on/off (off only for tests); default 1 */
    int64_t t_meas;           /* accumulate observables when t >= t_meas; default 0 */
    int32_t trace;            /* record the last sweep's ICM/PT decisions; default 0 */
    int32_t reserved;
} icm_schedule;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * (NULL = the legacy default stream) on which all work is enqueued.       */
icm_status icm_ctx_create(icm_ctx **out, int32_t device, void *cuda_stream);

/* Device-memory hooks for a context (no counterpart in the paper: a host
 * facility, so that a framework's caching allocator, e.g. PyTorch's, can own
 * the library's device memory).  alloc returns `bytes` of device memory
 * usable on `stream` (NULL on failure); free releases a block that alloc
 * returned, with the same size.  Calls come from the thread that calls the
 * library, never from device work.                                         */
typedef struct {
    void *(*alloc)(size_t bytes, int32_t device, void *stream, void *user);
    void (*free)(void *ptr, size_t bytes, int32_t device, void *stream, void *user);
    void *user;
} icm_allocator;
/* As icm_ctx_create, plus a device-memory budget and allocator.
 *   hbm_budget : bytes of device memory the context's batches may hold at
 *                once (0 = no limit); an allocation past it fails with
 *                ICM_ERR_BUDGET and the call that needed it fails cleanly.
 *   alloc      : NULL = cudaMalloc / cudaFree; else copied into the context
 *                and used for every batch allocation (state, staging,
 *                scratch, tuning snapshots).                               */
icm_status icm_ctx_create_ex(icm_ctx **out, int32_t device, void *cuda_stream, size_t hbm_budget,
                             const icm_allocator *alloc);
/* Device bytes the context's batches hold now, and its budget (0 = none). */
icm_status icm_ctx_memory(const icm_ctx *ctx, size_t *in_use, size_t *budget);
/* Destroys the context and every batch still alive on it (their handles
 * become invalid). */
icm_status icm_ctx_destroy(icm_ctx *ctx);
/* Description of the last error on this context; owned by the context and
 * valid until the next call on it.  Never NULL.                            */
const char *icm_last_error(const icm_ctx *ctx);
/* Wait for all work enqueued on the context's stream. */
icm_status icm_sync(icm_ctx *ctx);
/* Non-blocking: ICM_OK when all work enqueued on the context's stream has
 * finished, ICM_PENDING while some is still running, or an error. */
icm_status icm_query(icm_ctx *ctx);

/* Number of sites N and bonds N_b of a lattice (host only, no device work). */
icm_status icm_lattice_size(int32_t lattice, int32_t L, int32_t *n_sites, int32_t *n_bonds);

/* ---------------------------------------------------------------- batches */

/* Create a batch of n_inst disorder instances of one lattice and disorder
 * kind that share one temperature ladder.
 *   couplings : [n_inst][N_b] in bond order; int8 (+-1, or 0 = absent) for
 *               ICM_PM_J, float32 (0 = absent) for ICM_GAUSS.  NULL = drawn
 *               from `seed` and each instance id (the paper's disorder,
 *               "Benchmark model and observables": J = +-1 with probability
 *               1/2, or Gaussian with mean 0 and variance 1), Philox
 *               domain 3 keyed by instance id and bond index only:
 *                 +-J bond b: the top bit of word b & 3 of counter
 *                   {b >> 2, 0, 0, 3<<24 | id}, 0 -> +1, 1 -> -1;
 *                 Gaussian bond b: words o0, o1 of counter {b, 1, 0, 3<<24 | id},
 *                   J = sqrt(-2 ln u1) cos(2 pi u2) in double, u1 = (o0 + 1) 2^-32,
 *                   u2 = o1 2^-32, rounded to fp32.
 *               icm_read_couplings returns them.
 *   spins     : [n_inst][2 n_T][N] int8 (+1/-1), replica r = 2k + c is copy
 *               c at temperature position k.  NULL = all spins +1.
 *   instance_ids : [n_inst] uint32 < 2^24, the instance's RNG key.
 *               NULL = 0 .. n_inst-1.
 *   T         : [n_T] temperatures, strictly ascending, > 0 (position k = 0
 *               is the lowest temperature); 1 <= n_T <= 32.
 *   T_icm     : steps 2a/2b run at every k with T_k <= T_icm.
 *   seed      : 64-bit Philox key.
 * The schedule starts at its defaults; the sweep counter of every instance
 * starts at 0.  Instances too large for one CTA's shared memory run in the
 * global-resident layout (wider CTAs).  Errors: ICM_ERR_ARG (bad sizes or
 * values), ICM_ERR_UNSUPPORTED (more than 65535 sites), ICM_ERR_OOM,
 * ICM_ERR_CUDA.                                                             */
icm_status icm_batch_create(icm_ctx *ctx, int32_t lattice, int32_t L, int32_t disorder,
                            int32_t n_inst, const void *couplings, const int8_t *spins,
                            const uint32_t *instance_ids, const double *T, int32_t n_T,
                            double T_icm, uint64_t seed, uint32_t flags, icm_batch **out);
/* Free a batch.  ICM_ERR_STATE while a group (icm_group_create*) holds it:
 * the group's captured launches point at the batch's memory, so destroy
 * the group first.                                                       */
icm_status icm_batch_destroy(icm_batch *b);

/* Replace the couplings and/or spins of every instance (either may be NULL
 * to keep it), reset sweep counters to `t0` and clear the observables.
 * Layouts as in icm_batch_create.                                          */
icm_status icm_batch_load(icm_batch *b, const void *couplings, const int8_t *spins,
                          uint32_t t0, uint32_t flags);

/* Replace the temperature ladder (same n_T; ascending, > 0) and T_icm, e.g.
 * between the steps of an annealing schedule: the paper's introduction
 * proposes simulated annealing with cluster moves at every temperature of
 * its schedule as a ground-state heuristic.  Takes effect from the next
 * icm_run_sweeps; the configurations, energies and sweep counters are kept. */
icm_status icm_set_temperatures(icm_batch *b, const double *T, int32_t n_T, double T_icm);

/* Which steps of the simulation step ("Isoenergetic cluster algorithm":
 * 1 Metropolis sweep, 2a copy-1 reversal, 2b cluster move, 3 PT pass; the
 * observables of "Benchmark model and observables") run at each sweep t, see
 * icm_schedule.  The paper runs every step at every sweep (the default);
 * other schedules serve its comparisons (plain PT: icm_every = 0; the
 * Houdayer algorithm: cluster moves at every temperature without 2a) and
 * tests.  Takes effect from the next icm_run_sweeps.  icm_get_schedule
 * returns the batch's current schedule.                                  */
icm_status icm_set_schedule(icm_batch *b, const icm_schedule *s);
icm_status icm_get_schedule(const icm_batch *b, icm_schedule *s);

/* Enqueue n_sweeps simulation steps of every instance, in one kernel launch.
 * One simulation step is the paper's loop of "Isoenergetic cluster
 * algorithm" (steps 1, 2a, 2b, 3, in that order, as listed at the top of
 * this file), followed by the measurement of "Benchmark model and
 * observables" when t >= t_meas; the sweep counter t of each instance
 * advances by one per step.  Asynchronous: returns once the launch is
 * enqueued on the context's stream.  ICM_ERR_STATE if the batch holds
 * refused (invalid) couplings.                                            */
icm_status icm_run_sweeps(icm_batch *b, uint32_t n_sweeps);

/* ---------------------------------------------------------------- reads
 * Every read waits for the batch's outstanding work.                      */

/* Bonds present (coupling != 0) per instance, [n_inst] int32, host memory:
 * N_b for an undiluted instance.  The link overlap of instance i is
 * q_l = 1 - 2 acc_d / (bonds_i * n_meas).  No device work.               */
icm_status icm_read_bond_counts(const icm_batch *b, int32_t *out);
/* Couplings [n_inst][N_b] in bond order, as loaded or drawn: int8 for
 * ICM_PM_J, float32 for ICM_GAUSS (host or device buffer, ICM_DEVICE_PTR). */
icm_status icm_read_couplings(icm_batch *b, void *out, uint32_t flags);
/* Spins [n_inst][2 n_T][N] int8 +-1, site order, replica r = 2k + c. */
icm_status icm_read_spins(icm_batch *b, int8_t *out, uint32_t flags);
/* Energies [n_inst][2 n_T] (double; exact integers for ICM_PM_J). */
icm_status icm_read_energies(icm_batch *b, double *out, uint32_t flags);
/* Sweep counters [n_inst]. */
icm_status icm_read_sweeps(icm_batch *b, uint32_t *out, uint32_t flags);

/* Accumulated observables since the last clear; per temperature k, over the
 * measured sweeps (n_meas[inst] of them):
 *   accE   [n_inst][n_T] double : sum of E_{2k} + E_{2k+1}
 *   acc_n  [n_inst][n_T] int64  : sum of n = #{i : q_i = -1}
 *   acc_q2 [n_inst][n_T] int64  : sum of (N - 2n)^2       (N^2 q^2)
 *   acc_pmin [n_inst][n_T] int64: sum of min(n, N - n)     (N p, Fig. 1)
 *   acc_d  [n_inst][n_T] int64  : sum of #{bonds with q_i q_j = -1}
 *                                 (q_l = 1 - 2 d / N_b)
 *   hist   [n_inst][n_T][N+1] int64 : histogram of n       (P(q))
 *   n_meas [n_inst] int64
 * Any output pointer may be NULL to skip it.                               */
icm_status icm_read_observables(icm_batch *b, double *accE, int64_t *acc_n, int64_t *acc_q2,
                                int64_t *acc_pmin, int64_t *acc_d, int64_t *hist,
                                int64_t *n_meas, uint32_t flags);
/* Overlaps per instance and temperature position k over the measured sweeps,
 * from the accumulators above ("Benchmark model and observables"):
 *   q_mean  [n_inst][n_T] : <q>,   q = 1 - 2n/N = (1/N) sum_i q_i
 *   q2_mean [n_inst][n_T] : <q^2>
 *   ql_mean [n_inst][n_T] : <q_l>, q_l = (1/N_b) sum over the bonds present of q_i q_j
 *   q_hist  [n_inst][n_T][N+1] : counts of n (P(q) at q = 1 - 2n/N)
 * NaN where no sweep was measured.  Host buffers; any may be NULL.  Step 2a
 * flips copy 1 at ICM temperatures, so the sign of q there is folded:
 * compare P(q) symmetrised.                                                */
icm_status icm_read_overlaps(icm_batch *b, double *q_mean, double *q2_mean, double *ql_mean, int64_t *q_hist);
/* Clear the accumulated observables and the cluster-move counters below. */
icm_status icm_clear_observables(icm_batch *b);

/* Counters of the cluster moves (the paper's step 2b) since the last clear,
 * out [n_inst][2] uint64:
 *   out[i][0] : moves, i.e. ICM temperatures at which a cluster was grown
 *               and flipped (n > 0 q = -1 sites after step 2a; a pair with
 *               n = 0 has no seed and no move);
 *   out[i][1] : growth scans, the passes over the sites that grew the
 *               clusters of all pairs (bit-parallel, all pairs of a sweep
 *               at once), summed over sweeps.
 * They give the cluster-move rate and the work of the growth.  Not part of
 * checkpoints.  Host or device buffer (ICM_DEVICE_PTR); waits for the
 * batch's work.                                                           */
icm_status icm_read_icm_stats(icm_batch *b, uint64_t *out, uint32_t flags);

/* Decisions of the last sweep of the last icm_run_sweeps (schedule.trace = 1):
 *   n_pre [n_inst][n_T] int32 : n before step 2a (-1: no ICM at k)
 *   flip2a [n_inst][n_T] int32: step 2a reversed copy 1
 *   seed_site [n_inst][n_T] int32 : seed site (-1: none)
 *   csize [n_inst][n_T] int32 : cluster size
 *   esum_before / esum_after [n_inst][n_T] double : E_a + E_b around 2a/2b;
 *               esum_after is the sum of E_a and E_b each recomputed from
 *               the spins after the move (not the E_b the kernel carries on,
 *               (E_a + E_b)_before - E_a), so it tests that the move is
 *               isoenergetic (exactly for +-J, to fp32 rounding for Gaussian)
 *   swap_acc [n_inst][2][n_T - 1] uint8 : PT decisions per copy
 * Any output pointer may be NULL.                                          */
icm_status icm_read_trace(icm_batch *b, int32_t *n_pre, int32_t *flip2a, int32_t *seed_site,
                          int32_t *csize, double *esum_before, double *esum_after,
                          uint8_t *swap_acc, uint32_t flags);
/* The moved clusters of the last traced sweep: out [n_inst][n_T][N] uint8
 * (host), 1 where site i (site order) belongs to the cluster that step 2b
 * flipped at temperature position k; all 0 at a k without a move.  Needs a
 * run with the schedule's trace flag set (ICM_ERR_STATE otherwise); the
 * trace then keeps 8 N bytes per instance of device memory.               */
icm_status icm_read_cluster_masks(icm_batch *b, uint8_t *out);

/* ---------------------------------------------------------------- serving
 * Continuous batching: a batch is a table of slots.  One slot can be
 * replaced while the others keep their state; free slots are skipped by the
 * kernel; each slot has its own measurement window.                       */

/* Load one instance into `slot`: couplings [N_b] (NULL = drawn from the
 * batch seed and instance_id as in icm_batch_create), spins [2 n_T][N]
 * (NULL = all +1), its RNG instance id; the slot's sweep counter restarts at 0, its
 * observables are cleared, its window starts at t = 0 and it becomes active.
 * The other slots are untouched.                                          */
icm_status icm_batch_set_slot(icm_batch *b, int32_t slot, const void *couplings, const int8_t *spins,
                              uint32_t instance_id, uint32_t flags);
/* Mark a slot active (1) or free (0: the kernel skips it); slot -1 = all. */
icm_status icm_batch_set_active(icm_batch *b, int32_t slot, int32_t active);
/* Clear the slot's observables and accumulate them from sweep t_start on. */
icm_status icm_batch_start_window(icm_batch *b, int32_t slot, int64_t t_start);

/* Thermalization test of one instance over doubling windows [2^(b-1), 2^b)
 * at the lowest temperature ("Benchmark model and observables", Eq. 1 and
 * Eq. 2).  Eq. 1 is an identity of disorder averages, so for one instance
 * the test is the stability of the block means: the newest block's e and
 * q_l agree with the previous block's within eps_e / eps_ql for `need`
 * consecutive blocks.  delta = E(q_l) - e of the newest block is reported.
 * Host only; no device work.                                              */
typedef struct {
    int32_t blocks;       /* windows seen */
    int32_t stable;       /* consecutive windows agreeing with their predecessor */
    double e[3], ql[3];   /* newest first */
    double delta;         /* -(N_b/N)(1 - q_l)/T - e of the newest window */
} icm_therm_state;
typedef struct {
    double eps_e, eps_ql;
    int32_t need;
} icm_therm_criterion;
icm_status icm_therm_update(icm_therm_state *st, const icm_therm_criterion *c, double e, double q_l,
                            double T_min, double bonds_per_site, int32_t *thermalized);

/* ---------------------------------------------------------------- request server
 * Continuous batching of whole runs: each request is one disorder instance
 * (any lattice, size, disorder kind and ladder) to be run to the test above.
 * Requests are grouped into shape classes -- (lattice, L, disorder, ladder,
 * T_icm, seed) -- and each class is one slot-table batch on its own CUDA
 * stream.  icm_server_step, without waiting on the device:
 *   1. admits queued requests, first come first served, into free slots of
 *      idle classes; a new class is created only while the summed size of
 *      the class batches stays within the device-memory budget (otherwise
 *      the request waits);
 *   2. collects every class whose last launch has finished (icm_query),
 *      advances its slots by `quantum` sweeps and tests each window that
 *      ended ([Q, 2Q), [2Q, 4Q), ...): a slot that meets the criterion or
 *      reaches max_sweeps finishes and is freed, the others start their next
 *      window;
 *   3. launches the next quantum of every idle class with active slots.
 * Classes advance independently, so a class of large lattices does not hold
 * back the small ones.  A request's trajectory depends only on its (seed,
 * instance id) and its inputs, never on its slot or on the other requests.
 * One host thread at a time per server.                                    */
typedef struct icm_server icm_server;
typedef struct {
    int32_t slots_per_class;   /* slots of each class batch; default 64 */
    int32_t quantum;           /* sweeps per launch, a power of two; default 64 */
    uint32_t max_sweeps;       /* sweep cap of a request; default 65536 */
    icm_therm_criterion crit;  /* default {0.005, 0.01, 2} */
    uint64_t hbm_budget;       /* bytes of all class batches together; default 8 GiB */
} icm_server_config;
typedef struct {
    int32_t lattice, L, disorder;
    int32_t n_T;
    const double *T;           /* [n_T], strictly ascending, > 0 */
    double T_icm;
    uint64_t seed;
    uint32_t instance_id;      /* < 2^24 */
    const void *couplings;     /* host [N_b] in bond order, int8 or float32 (copied), or NULL =
                                  drawn from seed and instance_id (see icm_batch_create) */
    const int8_t *spins;       /* host [2 n_T][N] +-1, or NULL = all +1 (copied) */
} icm_request;
typedef struct {
    int32_t status;            /* ICM_PENDING (queued or running), ICM_OK (finished) or ICM_CANCELLED */
    int32_t thermalized;       /* 1: met the criterion; 0: stopped at max_sweeps */
    uint32_t sweeps;           /* sweeps run */
    int32_t slot;              /* slot in its class batch, -1 before admission */
    double e, q_l, delta;      /* last window at T_min: energy per spin, link overlap, E(q_l) - e */
    double accE;               /* last window's raw sums at T_min */
    int64_t acc_d, n_meas;
    double t_submit, t_admit, t_done;   /* seconds of the host's monotonic clock */
} icm_result;

/* cfg NULL = the defaults above. */
icm_status icm_server_create(int32_t device, const icm_server_config *cfg, icm_server **out);
/* Frees every class batch and stream (waits for running launches). */
icm_status icm_server_destroy(icm_server *s);
const char *icm_server_last_error(const icm_server *s);
/* Queue a request (its arrays are copied).  ICM_ERR_BUDGET: its class alone
 * exceeds the memory budget; ICM_ERR_ARG: invalid request.                 */
icm_status icm_server_submit(icm_server *s, const icm_request *r, uint64_t *ticket);
/* One pass of admit / collect / launch (never blocks on the device).
 * finished: requests completed in this pass; launched: kernel launches made. */
icm_status icm_server_step(icm_server *s, int32_t *finished, int32_t *launched);
/* State of a ticket; ICM_ERR_ARG for an unknown ticket. */
icm_status icm_server_poll(const icm_server *s, uint64_t ticket, icm_result *out);
/* Cancel a request.  A queued request is dropped at once; a running one is
 * released at its class's next collection (immediately when the class is
 * idle); its result then has status ICM_CANCELLED and the sweeps it ran.
 * ICM_ERR_STATE when the request has already finished or was cancelled. */
icm_status icm_server_cancel(icm_server *s, uint64_t ticket);
/* Requests queued, requests in slots, classes created. */
icm_status icm_server_status(const icm_server *s, int32_t *queued, int32_t *active, int32_t *classes);
/* Class i (creation order): lattice, L, disorder, n_T, CTA width of its
 * batch, slots in use. */
icm_status icm_server_class_info(const icm_server *s, int32_t i, int32_t *lattice, int32_t *L, int32_t *disorder,
                                 int32_t *n_T, int32_t *threads, int32_t *active);
/* The server's clock (seconds, the host's monotonic clock). */
double icm_server_clock(void);

/* Eq. 2 over the batch: the mean over measured (active) instances of
 * E(q_l) - e at temperature position k from the current accumulators, with
 * its standard error over instances.                                      */
icm_status icm_batch_delta(icm_batch *b, int32_t k, double *delta_mean, double *delta_se, int32_t *n_used);

/* Energies of replica configurations, computed without allocating any device
 * memory.  The paper has no counterpart: this is a service for callers that
 * cannot call cudaMalloc at this point -- code that runs inside a memory pool
 * or arena that forbids outside allocations, pipelines that must not hit
 * cudaMalloc's implicit device synchronisation, and hosts that budget every
 * byte of HBM in advance.
 *   couplings : device [n_inst][N_b] in bond order (int8 +-1 or float32);
 *               this entry point does not take diluted +-J couplings (an
 *               int8 0 counts as +1), Gaussian zeros contribute 0
 *   spins     : device [n_inst][n_rep][N] int8 +-1, 1 <= n_rep <= 64
 *   out       : device [n_inst][n_rep] double, H = -sum_<ij> J_ij s_i s_j
 * Work is enqueued on the context's stream, and the call then synchronises
 * that stream: it returns after the work has ended.  Scratch is one fixed
 * 8 MiB array in the library's device image, held by every GPU that loads
 * the library until the process exits.  Requests that need more (geometry
 * tables + n_inst instances of packed spins, expanded couplings and
 * energies) fail with ICM_ERR_UNSUPPORTED and a message.  The first call on
 * a device looks up the array's address (do it before any stream capture);
 * after a cudaDeviceReset of that device the looked-up address is stale, so
 * do not call this entry point on a device that was reset.  All calls share
 * the array: calls that overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  Every scratch byte a
 * call reads is written earlier in that call.                              */
icm_status icm_energies_static(icm_ctx *ctx, int32_t lattice, int32_t L, int32_t disorder, int32_t n_inst,
                               int32_t n_rep, const void *couplings, const int8_t *spins, double *out);

/* ---------------------------------------------------------------- site percolation
 * Largest cluster of occupied sites (Supplemental Material: the relative
 * size s_max of the largest cluster, whose Binder ratio
 * g = (3 - <s_max^4>/<s_max^2>^2)/2 locates the percolation threshold).
 * Clusters are connected through the lattice's bonds (icm_lattice).
 *   masks : [n_masks][N] bytes in site order, nonzero = occupied
 *   smax  : [n_masks] int32, number of sites of the largest cluster
 * Host or device buffers (ICM_DEVICE_PTR).  The call waits for its work.  */
icm_status icm_percolation(icm_ctx *ctx, int32_t lattice, int32_t L, int32_t n_masks, const uint8_t *masks,
                           int32_t *smax, uint32_t flags);
/* The same on random masks drawn on the device: site i of mask m is
 * occupied iff word 0 of Philox4x32-10(ctr {i, m, 0, 5 << 24}, key = seed)
 * is below floor(p 2^32) (p = 1: every site).                             */
icm_status icm_percolation_random(icm_ctx *ctx, int32_t lattice, int32_t L, double p, uint64_t seed,
                                  int32_t n_masks, int32_t *smax, uint32_t flags);

/* ---------------------------------------------------------------- launch shape
 * The threads per CTA of a batch's kernel, a multiple of 32 up to 1024; one
 * CTA runs one instance.  Up to 128 threads the instance lives in shared
 * memory; wider CTAs use the global-resident layout (the only one for
 * instances too large for shared memory).  Gaussian results depend on the
 * width through the summation order of the fp32 energies; +-J results do
 * not.                                                                      */
icm_status icm_batch_set_threads(icm_batch *b, int32_t threads);
/* Time every valid launch shape on `sweeps` sweeps of this batch and keep
 * the fastest: CTA widths 32..128 (shared memory) when the instance fits,
 * and for instances with more than 128 sites per colour also wide CTAs
 * (256, 512, 1024) and thread-block clusters (K = 4, 8 of 256 or 512
 * threads).  best_threads is the CTA width; icm_batch_cluster gives K.  The
 * batch's state (spins, energies, sweep counters, observables) is restored
 * afterwards, so tuning does not advance the chain.  Allocates a temporary
 * snapshot.                                                                */
icm_status icm_batch_autotune(icm_batch *b, uint32_t sweeps, int32_t *best_threads, float *best_ms);

/* A group runs several batches (e.g. one per lattice size of a mixed-size
 * workload) as one CUDA graph: each batch's kernel on its own forked stream,
 * joined back into the context stream.  The graph is captured at creation
 * with the batches' current schedules and launch shapes and `sweeps_per_launch`;
 * icm_group_run replays it.  Create a group after the batches are set up
 * and re-create it after changing a schedule or the threads of a batch.
 * A group holds its batches: icm_batch_destroy refuses a batch of a live
 * group (destroy the group first).                                        */
typedef struct icm_group icm_group;
icm_status icm_group_create(icm_ctx *ctx, icm_batch *const *batches, int32_t n, uint32_t sweeps_per_launch,
                            icm_group **out);
icm_status icm_group_run(icm_group *g, uint32_t n_launches);
icm_status icm_group_destroy(icm_group *g);

/* The shared form of a group: the instances of every batch -- uneven sizes
 * of one disorder kind and one lattice degree, e.g. 3D L = 4..12 -- share
 * one persistent kernel, the fused simulation step of icm_run_sweeps (the
 * paper's "Isoenergetic cluster algorithm", steps 1, 2a, 2b, 3, and the
 * observables), captured as one launch in the group's graph.  One CTA of
 * 896 threads per SM takes the next tile of instances whenever it is free,
 * largest tiles first: a tile of batch c is up to 896 / team_threads[c] instances side by side,
 * each run by its own team of team_threads[c] threads (threads per
 * instance, a divisor of 896 that is a multiple of 32) with its own shared
 * memory and barrier, as many as the SM's shared memory holds.
 *   team_threads : [n] or NULL; an entry <= 0 (or NULL) picks the width that
 *                  keeps the most threads of the CTA busy (the narrower on a
 *                  tie).
 * Every batch must have the same disorder kind, lattice degree and seed
 * (instance ids tell the instances apart), no dilution and no cluster
 * layout; at most 8 batches (ICM_ERR_UNSUPPORTED otherwise).  Arithmetic and
 * random keys are those of icm_run_sweeps, so a +-J instance follows the same
 * chain either way.  Each batch's schedule and slot flags are taken at
 * creation.  The tile list is device memory of the context (its budget).  */
icm_status icm_group_create_shared(icm_ctx *ctx, icm_batch *const *batches, int32_t n, uint32_t sweeps_per_launch,
                                   const int32_t *team_threads, icm_group **out);
/* The launch shape of a group, per batch: threads per instance and
 * instances per tile (the batch's CTA width and 1 for a graph of separate
 * launches); grid, dynamic shared memory per CTA and tiles of the shared
 * kernel (0 for separate launches).  Any pointer may be NULL.             */
icm_status icm_group_info(const icm_group *g, int32_t *team_threads, int32_t *tile, int32_t *grid, int32_t *smem,
                          int32_t *n_items);

/* ---------------------------------------------------------------- checkpoint / resume
 * The state of a batch -- spins, energies, sweep counters, instance ids,
 * observables, slot flags, ladder and schedule -- as one versioned blob.
 * The random numbers are counter-based (Philox keyed by seed, instance,
 * sweep, site), so no generator state is needed: loading a checkpoint into
 * a batch of the same shape and seed and running n more sweeps gives the
 * same result as running on without the checkpoint.
 * icm_save with buf = NULL stores the required size in *len.             */
icm_status icm_save(icm_batch *b, void *buf, size_t *len);
icm_status icm_load(icm_batch *b, const void *buf, size_t len);

/* Thread-block-cluster layout: each instance runs on a cluster of K CTAs
 * (K = 2, 4 or 8; K SMs), each holding 1/K of the sites of each colour in
 * its shared memory and reading its neighbours' words through the cluster's
 * distributed shared memory.  The arithmetic and random keys are those of
 * the one-CTA layouts (the same chain, bit for bit for +-J); a single large
 * instance finishes its sweeps up to K times sooner.  Any lattice kind
 * (2D, 3D, chimera, 4D), diluted or not, with N/2 divisible into K blocks
 * of a multiple of 32 sites.  K = 0 returns to one CTA per instance (CTA
 * width `threads`, as icm_batch_set_threads).  A batch keeps the layout when
 * couplings with absent bonds are loaded (its kernels change).            */
icm_status icm_batch_set_cluster(icm_batch *b, int32_t K, int32_t threads);
icm_status icm_batch_cluster(const icm_batch *b, int32_t *K);

/* How the thread-block-cluster layout finds the clusters of step 2b (the
 * connected component of q = -1 sites that holds the seed, "Reminder:
 * Houdayer cluster algorithm" and step 2b of the isoenergetic cluster
 * move).  mode 1: union-find labelling of the q = -1 sites over the
 * cluster's shared memory, a few pairs at a time (lock-free hooking of
 * roots by compare-and-swap, path halving); mode 0: label propagation, all
 * pairs at once, one bit per pair and site, in rounds of in-place scans
 * until nothing grows; mode -1 (default): the library's choice, label
 * propagation (faster on every size measured: its word operations serve
 * all pairs at once, where union-find works pair by pair).  Both give the
 * same clusters, so the chain is the same bit for bit.
 * Takes effect now on a clustered batch, else at icm_batch_set_cluster.
 * icm_batch_cluster_growth gives the pairs per union-find group (0 = label
 * propagation, or not clustered).  ICM_ERR_ARG for another mode.          */
icm_status icm_batch_set_cluster_growth(icm_batch *b, int32_t mode);
icm_status icm_batch_cluster_growth(const icm_batch *b, int32_t *pairs_per_group);

/* Kernel-level facts for measurement: threads per CTA, CTAs per SM, grid,
 * dynamic shared memory bytes per CTA and kernel launches issued so far.
 * For the thread-block-cluster layout, CTAs per SM is the count when the
 * most clusters are resident (their CTAs over the SMs, rounded up) and the
 * shared memory is that of one CTA of a cluster.                          */

icm_status icm_batch_info(const icm_batch *b, int32_t *threads, int32_t *ctas_per_sm,
                          int32_t *grid, int32_t *smem_bytes, int64_t *launches);

#ifdef __cplusplus
}
#endif
#endif /* ICMPT_H */
