/*
 * kmc.h -- C ABI of libkmc, the GB300 (sm_103a) implementation of the kinetic
 * Monte-Carlo hysteresis step of Tan, Carrey & Respaud, "Magnetic hyperthermia
 * properties of nanoparticles inside lysosomes using kinetic Monte-Carlo
 * simulations" (arXiv:1407.2737).
 *
 * One call of kmc_run advances every nanoparticle (NP) of every lysosome of a
 * context through S steps per field period, each step being the paper's
 * steps i)-viii) of Sec. II.1:
 *   ii)  total field = applied field along z + dipolar field of all other NPs
 *        of the same lysosome (Eq. 1, exact sum, no cutoff);
 *   iii) working plane through the easy axis and the total field, previous
 *        moment projected onto it;
 *   iv)  extrema of the Stoner-Wohlfarth energy (Eq. 2) by a 200-point scan of
 *        dE/dtheta refined by Newton's method;
 *   v)   fall into the minimum whose basin holds the moment;
 *   vi)  Neel-Arrhenius rates from the lower maximum (Eqs. 3-4) and the jump
 *        probability over one step (Eq. 5);
 *   vii) a counter-based Philox4x32-10 draw u decides the jump (u < P);
 * and accumulates each NP's share of the hysteresis area (Sec. III.2.a).
 *
 * Conventions shared by every entry point:
 *   - SI units: positions in m, volumes in m^3, M_S in A/m, K_eff in J/m^3,
 *     T in K, tau0 in s, fields as mu0*H in tesla, energies in J.
 *   - All pointers are HOST pointers. Inputs are owned by the caller and are
 *     copied before the call returns; outputs go to caller buffers of the
 *     stated capacity (in elements).
 *   - Every call returns a kmc_status and never aborts the process;
 *     kmc_last_error() describes the last failure of the calling thread.
 *   - Device memory is allocated by kmc_create and freed by kmc_destroy.
 *   - Work is queued on the context's CUDA stream (a private stream unless
 *     kmc_set_stream gave one); kmc_run returns once the work is queued.
 *     kmc_read, kmc_sync, kmc_debug_step and kmc_save wait for it, and report
 *     KMC_ETIMEOUT if a device-side wait ran out of time.
 *   - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef KMC_H
#define KMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kmc_ctx kmc_ctx; /* opaque, owned by the library */

typedef enum {
  KMC_OK = 0,
  KMC_EINVAL = 1,    /* bad argument (NULL, negative size, non-finite value) */
  KMC_ENOMEM = 2,    /* host or device allocation failed                     */
  KMC_ECUDA = 3,     /* a CUDA runtime call failed (no device, launch error) */
  KMC_ETIMEOUT = 4,  /* a device-side wait gave up; results are not valid    */
  KMC_ESTATE = 5,    /* call out of order (e.g. kmc_read before kmc_run)     */
  KMC_ECAPACITY = 6, /* output buffer too small; *written = elements needed  */
  KMC_EIO = 7        /* checkpoint file could not be read or written         */
} kmc_status;

typedef enum {
  KMC_FP64_PLAIN = 0, /* every step of the path in FP64                      */
  KMC_FP32_MIXED = 1  /* FP32 pair sum with compensated combine, FP32 scan and
                         Newton; FP64 barrier near switching, FP64 rate
                         exponent and probability, FP64 energy accumulation  */
} kmc_precision;

/* One lysosome (Sec. II.1): NPs of one material (M_S, K_eff) at temperature
 * T with attempt time tau0 = 1/nu0 (nu1^0 = nu2^0 = nu0 in Eqs. 3-4). */
typedef struct {
  int32_t n;            /* number of NPs, >= 1                                 */
  const double *pos;    /* [n][3] centres, m; pairwise distinct              */
  const double *axis;   /* [n][3] easy axes, normalised by the library       */
  const double *vol;    /* [n] magnetic volumes, m^3, > 0                    */
  const double *center; /* [3] origin of the float32 frame, m, or NULL for
                           the centroid of pos                               */
  double Ms;            /* A/m, > 0                                          */
  double Keff;          /* J/m^3, >= 0                                       */
  double T;             /* K, >= 0; T = 0 skips steps vi-vii (no jumps)      */
  double tau0;          /* s, > 0                                            */
  double rho;           /* kg/m^3 for the SAR; <= 0 means 5200 (magnetite)   */
} kmc_lysosome;

/* What kmc_read returns (per lysosome `lys` unless stated). */
enum {
  KMC_READ_LOOP_H = 0,    /* [S*(periods-discard)] mu0 H_ext,k (T), recorded steps */
  KMC_READ_LOOP_M = 1,    /* [same] volume-weighted mean m_z after step k (M/M_S)  */
  KMC_READ_NP_ENERGY = 2, /* [n] energy dissipated by each NP per recorded period, J:
                             mu0 M_S V_i sum_k H_ext,k (m_z,k+1 - m_z,k) / periods */
  KMC_READ_AREA = 3,      /* [1] hysteresis area A, J/m^3 per cycle (Sec. III.2.a) */
  KMC_READ_SAR = 4,       /* [1] SAR = A f / rho, W/kg                             */
  KMC_READ_MOMENTS = 5,   /* [n][3] current unit moments                           */
  KMC_READ_COUNTERS = 6,  /* [7] NP-steps of the last run: jumps, near-threshold
                             draws (|u - P| < 1e-9), profiles with one minimum,
                             working planes that needed the fallback, FP32 scans
                             redone in FP64, FP32 barriers recomputed in FP64 near
                             switching, NPs held because their field, barrier or
                             probability was not finite. Readable after a device
                             error (it does not report one)                        */
  KMC_READ_DHDIP = 7,     /* [n] Eq. 6 per NP, T: the dipolar field along z (the
                             applied field's direction) during the step at
                             +mu0 H_max (step 0 of a period) minus that during the
                             step at -mu0 H_max (step S/2, (S-1)/2 for odd S), each
                             from the moments at the start of the step, averaged
                             over the recorded periods; > 0 where the dipolar
                             field is parallel to the applied one (Sec. III.2.b) */
  KMC_READ_POSITIONS = 8, /* [n][3] current NP centres, m (those given to
                             kmc_create until kmc_regenerate moves them)     */
  KMC_READ_AXES = 9,      /* [n][3] current unit easy axes (FP32 contexts: as
                             held in float32)                                */
};

/* Creates a context holding n_lys lysosomes (copied to the device). Moments
 * start along the easy axis with m_z >= 0. The global step counter, which
 * keys the random draws, starts at 0. */
kmc_status kmc_create(const kmc_lysosome *lys, int32_t n_lys, kmc_precision prec,
                      kmc_ctx **out);

/* Queues later work on `cuda_stream` (a cudaStream_t of the current device,
 * not owned; NULL selects the context's private stream). */
kmc_status kmc_set_stream(kmc_ctx *ctx, void *cuda_stream);

/* Runs `periods` periods of the sinusoidal field mu0 H_ext,k = mu0Hmax
 * cos(2 pi k / S) along z (each period starts at +Hmax, Sec. III.1), frequency
 * f, S = steps_per_period steps of t_step = 1/(f S). The first
 * discard_periods periods are not recorded (Sec. III.1 runs two loops and keeps
 * the second). mu0Hmax holds n_amp = n_lys amplitudes, or n_amp = 1 for all.
 * Moments and the global step counter carry over between runs; the loop,
 * energy and counter outputs are those of the latest run. The draw of NP i of
 * lysosome l at global step s is Philox4x32-10 with key (seed low, seed high)
 * and counter (s low, s high, i, l). Lysosomes do not interact, so a batch
 * advances as up to KMC_MAX_CHAINS independent chains of step kernels (sets of
 * whole lysosomes of about equal work; min(n_lys, KMC_MAX_CHAINS) chains when
 * the lysosomes are of one size), joined once per period; each lysosome's
 * results are those it gets alone under the same launch shape, bit for bit. */
#define KMC_MAX_CHAINS 8
kmc_status kmc_run(kmc_ctx *ctx, const double *mu0Hmax, int32_t n_amp, double f,
                   int32_t steps_per_period, int32_t periods, int32_t discard_periods,
                   uint64_t seed);

/* Copies output `what` (KMC_READ_*) of lysosome `lys` into buf[cap]. Sets
 * *written to the number of elements (also on KMC_ECAPACITY). Waits for
 * queued work. The results of a run (loop, energies, area, SAR, Eq. 6) report
 * a device error as kmc_sync does; the state (moments, positions, axes) and
 * the counters are readable after one. */
kmc_status kmc_read(kmc_ctx *ctx, int32_t what, int32_t lys, double *buf, int64_t cap,
                    int64_t *written);

/* Waits for queued work and reports device-side errors: KMC_ETIMEOUT (a
 * staging wait ran out), KMC_ESTATE (an energy profile with more than two
 * minima, or a non-finite dipolar field or barrier, as two NPs at one point
 * give: such an NP keeps its moment for the step and is counted). The error
 * stays set until the next kmc_run or kmc_debug_step. */
kmc_status kmc_sync(kmc_ctx *ctx);

/* Test hook: one step (steps i-vii) of every NP from the moments m_in
 * ([N][3], all lysosomes in order) under applied fields mu0Hext ([n_lys], T,
 * along z), step length t_step and draws keyed by (seed, step). Runs the
 * kernels of kmc_run. The context's moments become m_out. Outputs, each
 * [N]-major and optional (NULL to skip): m_out [N][3]; B_dip [N][3] dipolar
 * field mu0 H_dip (T); dE [N][2] barriers E3 - E_a (current well a) and
 * E3 - E_b (J, 0 with a single minimum); P [N] jump probability; u [N] draw;
 * flags [N] = n_min | jumped << 2 | near-threshold << 3 | fallback plane << 4 |
 * FP32 scan redone in FP64 << 5 | FP32 barrier recomputed in FP64 << 6 |
 * held for a non-finite field or barrier << 7. With the environment variable
 * KMC_DEBUG_RESCAN=1 an FP32 context scans every target again in FP64 (a test
 * of that path, which Eq. 2's profiles never need: its derivative has at most
 * four roots, so FP32 noise at one node cannot raise the count above four). */
kmc_status kmc_debug_step(kmc_ctx *ctx, const double *mu0Hext, double t_step,
                          uint64_t seed, int64_t step, const double *m_in, double *m_out,
                          double *B_dip, double *dE, double *P, double *u,
                          int32_t *flags);

/* Checkpoint: writes the moments and the global step counter to `path`;
 * kmc_load restores them into a context built from the same lysosomes and
 * precision, so that the next kmc_run continues bit for bit. kmc_load
 * refuses, leaving the context as it was: a file that is not a checkpoint or
 * is cut short (KMC_EIO), one of another context (KMC_EINVAL), or one holding
 * a moment that is not a finite unit vector (KMC_EINVAL). */
kmc_status kmc_save(kmc_ctx *ctx, const char *path);
kmc_status kmc_load(kmc_ctx *ctx, const char *path);

/* Total NPs, lysosomes and global step counter of a context. */
kmc_status kmc_info(const kmc_ctx *ctx, int64_t *n_total, int32_t *n_lys,
                    int64_t *global_step);

/* Launch shape of the fused step kernel. warps: warps per block, each taking
 * every warps-th source record of a tile (4, 8 or 16; with replicas per lane
 * pinned, warps = 1, 2 or 4 times the replicas and tile <= 128). tile: source records per
 * shared-memory tile (a power of two, 32..1024; an FP32 record holds two NPs,
 * an FP64 record one). chunk: sources per work item when a lysosome's sources
 * are split over several blocks (0 = never split; else a multiple of 64).
 * All three 0 (or warps = 0) lets the autotuner choose on the next kmc_run or
 * kmc_debug_step. The shape in use is returned through the out pointers (each
 * may be NULL); call with warps = tile = chunk = -1 to only read it. With the
 * environment variable KMC_TUNE_LOG set (and not "0") the autotuner prints
 * every shape it times, the finalists' second timings and its choice on
 * standard error. */
kmc_status kmc_tuning(kmc_ctx *ctx, int32_t warps, int32_t tile, int32_t chunk,
                      int32_t *warps_out, int32_t *tile_out, int32_t *chunk_out);

/* Targets per lane of the FP32 step kernel: 1 (a block takes 32 targets, one
 * per lane), 2 or 3 (64 or 96 targets, two or three per lane, so that each
 * staged source record feeds that many independent chains; FP32 contexts only,
 * KMC_EINVAL on FP64). All give the same bits at the same warps, tile and
 * chunk. In the symmetric pair form (kmc_pair_form) a lane holds 2 or 4
 * targets (one or two cells of 64 NPs per warp); 4 selects that form, and
 * 1 or 3 are refused while it is pinned. 0 (the default) lets the autotuner
 * choose; a pinned value also applies to a shape set by kmc_tuning. The value
 * in use (0 before the first tuning) is returned through tpl_out (may be
 * NULL); tpl = -1 only reads it. */
kmc_status kmc_targets_per_lane(kmc_ctx *ctx, int32_t tpl, int32_t *tpl_out);

/* Replicas per lane of the FP32 step kernel. When the lysosomes come in sets
 * of k identical consecutive ones (the same NPs, axes, volumes, material,
 * temperature, attempt time, density and frame origin; only the random
 * streams, the amplitudes and hence the moments differ: seeds of one sample),
 * a block of k warps (or 2 k, or 4 k) can take 32 targets of all k lysosomes of a set
 * at once: each staged source record's geometry (separation, distance, its
 * powers) is formed once and serves all k, which add only their own moments'
 * terms. Every lysosome's field, and its whole step, are the bits it gets with
 * one target per lane and as many warps at the same tile and chunk; each warp
 * (or group of two or four warps) then runs one lysosome's steps iii-vii. rpl: 0 lets the autotuner choose (the
 * default; it considers k = 2 and 4 where the sets exist), 1 turns replicas
 * off, 2 or 4 pins them (KMC_EINVAL on FP64 contexts, with two or three
 * targets per lane pinned, or unless n_lys is a multiple of rpl and every set
 * of rpl consecutive lysosomes is identical). A pinned value takes warps = rpl,
 * 2 rpl or 4 rpl in kmc_tuning and drops a shape of another kind. The value in use (0 before
 * the first tuning) is returned through rpl_out (may be NULL); rpl = -1 only
 * reads it. */
kmc_status kmc_replicas_per_lane(kmc_ctx *ctx, int32_t rpl, int32_t *rpl_out);

/* Pair form of the FP32 dipolar sum (Eq. 1, Sec. II.1 step ii).
 *   1 ordered: every (target, source) pair is evaluated for its target, by
 *     the step kernels (one launch per step and chain).
 *   2 symmetric: the pair term of Eq. 1 is symmetric in its geometry (the
 *     separation, the distance and its powers are the same for T_ij and
 *     T_ji), so every unordered pair is formed once and serves both NPs. A
 *     lysosome's NPs are cut into cells of 64; the pairs between a row group
 *     of cells (4 or 8 cells: warps x cells per warp) and the cells above it
 *     run in the symmetric field kernel, the pairs inside a row group in the
 *     ordered form; an update kernel then adds the partial sums in a fixed
 *     order and runs steps iii-vii (two launches per step and chain). The
 *     fields differ from the ordered form's by rounding only; results are
 *     deterministic and do not depend on the chaining.
 * form: 0 lets the autotuner choose (the default: it times both forms on
 * FP32 contexts), 1 or 2 pins one (2: KMC_EINVAL on FP64 contexts, with
 * replicas per lane pinned, or with 1 or 3 targets per lane pinned). A pinned
 * symmetric form reads kmc_tuning's warps (4; 8 with 2 targets per lane; 2
 * with 4) and chunk (source NPs per field item, a multiple of 64; 0 = all cells above
 * the row group); its tile is 32. The form in use (0 before the first
 * tuning) is returned through form_out (may be NULL); form = -1 only reads it. */
kmc_status kmc_pair_form(kmc_ctx *ctx, int32_t form, int32_t *form_out);

/* Persistent period of the FP32 one-target-per-lane step (Sec. II.1 steps
 * i-vii, S steps per field period). 2 runs every field period as one
 * cooperative launch: each block keeps its work item for the whole period and
 * a grid-wide barrier separates the steps (the update of Sec. II.2 is
 * synchronous: a step reads only the moments of the step before), in place of
 * one launch per step and chain. The barrier is bounded in time (2 s): a block
 * that never arrives makes the others give up, kmc_sync then returns
 * KMC_ETIMEOUT, and every block leaves the period at a step boundary. It needs
 * every work item's block resident at once; a plan with more items fails with
 * KMC_EINVAL. The results are the bits of the per-step launches at the same
 * warps (4 or 8), tile and chunk. mode: 0 lets the autotuner choose (the
 * default: it times both where the plan fits), 1 off, 2 on (KMC_EINVAL on FP64
 * contexts). The value in use (0 before the first tuning) is returned through
 * mode_out (may be NULL); mode = -1 only reads it. */
kmc_status kmc_persistent(kmc_ctx *ctx, int32_t mode, int32_t *mode_out);

/* Failure-detection test hook of the persistent period: runs 4 steps in which
 * block 0 does not arrive at the grid barrier after step 1, with the barrier's
 * limit cut to 1 ms. The other blocks give up, nothing faults, and the call
 * returns KMC_ETIMEOUT as designed (KMC_ESTATE if the barrier did not run out)
 * and clears the error word. The moments advance by up to two steps.
 * KMC_EINVAL unless the context's shape is the persistent period. */
kmc_status kmc_debug_grid_stall(kmc_ctx *ctx);

/* Update kernel of the symmetric pair form (kmc_pair_form = 2): 1 gives each
 * update item (32 targets of one cell) one warp, which adds the item's forward
 * and reverse partial sums in slot order and runs steps iii-vii alone; 2 gives
 * it a block of four warps, which share the gather (warp w taking slots w,
 * w + 4, ...; the warps then added in order) and run steps iii-vii together.
 * The first is faster where items are many and their slots few (batches of
 * small lysosomes), the second where a target gathers many slots (large
 * lysosomes). The two round the field sums differently, each in a fixed
 * order. mode: 0 lets the autotuner choose (the default), 1 or 2 pins one.
 * The value in use (0 before the first tuning or outside the symmetric
 * form) is returned through mode_out (may be NULL); mode = -1 only reads it. */
kmc_status kmc_sym_update(kmc_ctx *ctx, int32_t mode, int32_t *mode_out);

/* Cluster split of the FP32 one-target-per-lane step kernel. When every
 * target group's sources are split into exactly two parts (kmc_tuning's chunk
 * with one target per lane), the two parts can run as the two CTAs of a
 * thread-block cluster: the second hands its sums to the first through
 * distributed shared memory, and the first adds them in split order and runs
 * steps iii-vii. That replaces the exchange through global memory (stores,
 * fences, an arrival counter) with two cluster barriers; the results are the
 * same bits. mode: 0 lets the autotuner choose (the default: it times both
 * where the plan allows), 1 off, 2 on (KMC_EINVAL on FP64 contexts; a run or
 * debug step whose plan does not split every group in two fails with
 * KMC_EINVAL). The value in use (0 before the first tuning) is returned
 * through mode_out (may be NULL); mode = -1 only reads it. */
kmc_status kmc_cluster_split(kmc_ctx *ctx, int32_t mode, int32_t *mode_out);

/* Fields of one field item and of one update item in kmc_plan_sym's output. */
#define KMC_SYM_FIELDS 8

/* The symmetric form's work decomposition (kmc_pair_form) for lysosomes of
 * n[l] NPs (host arrays), computed on the host with no GPU, for tests and
 * tools. gc: cells (64 NPs) per row group, 4 or 8; src_cells: source cells
 * per field item (0 = all cells above the row group). Lysosomes come largest
 * first (stable); per lysosome its row groups in order, each as its diagonal
 * item and then its source ranges in order. items_out (capacity cap items):
 * lysosome, row group, first and end source cell (-1, -1 for the diagonal
 * item), forward slot, first reverse slot of the lysosome, 0, 0. upd_out
 * (capacity cap_upd): lysosome, first target, targets (<= 32, inside one
 * cell), first forward slot and count (the row group's items), first reverse
 * slot and count (one per row group below the cell), first target minus the
 * row group's first NP. *n_items, *n_upd and *n_rev (reverse slots) receive
 * the counts (also on KMC_ECAPACITY). chain_cut_items and chain_cut_upd
 * (KMC_MAX_CHAINS + 1 int32 each): chain q runs field items
 * chain_cut_items[q] .. chain_cut_items[q + 1] - 1 and the matching update
 * items; *n_chains receives the chain count. Bad arguments: KMC_EINVAL. */
kmc_status kmc_plan_sym(const int32_t *n, int32_t n_lys, int32_t gc, int32_t src_cells,
                        int32_t *items_out, int64_t cap, int64_t *n_items, int32_t *upd_out,
                        int64_t cap_upd, int64_t *n_upd, int64_t *n_rev,
                        int32_t *chain_cut_items, int32_t *chain_cut_upd, int32_t *n_chains);

/* Fields of one work item in kmc_plan_items' output. */
#define KMC_ITEM_FIELDS 8

/* The work decomposition that kmc_run launches for a batch of n_lys lysosomes
 * of n[l] NPs (host arrays), computed on the host with no GPU, for tests and
 * tools. Each step of Sec. II.1 runs one block per work item: a group of
 * 32 * tpl targets of one lysosome (the last group of a lysosome may be
 * smaller) against one contiguous part of that lysosome's source records
 * (pairs of NPs for KMC_FP32_MIXED, single NPs for KMC_FP64_PLAIN). Groups
 * come lysosome by lysosome, largest lysosome first (stable). A group's parts
 * are consecutive items. chunk > 0 splits a group's sources into parts of
 * chunk NPs and, for a single chain spanning several waves of n_sms SMs x
 * blocks_per_sm blocks (n_sms > 0), gives the last groups one part more each
 * until the items fill whole waves; chunk = 0 splits only to even out one
 * device-wide wave of a single chain (n_sms = 0: never).
 * tpl is 1, 2 or 3 (2 and 3 with KMC_FP32_MIXED only); chunk a multiple of 64;
 * n[l] >= 1.
 * items_out (host, capacity cap items): KMC_ITEM_FIELDS int32 per item, in
 * launch order: lysosome, first target, targets, target group, first source
 * record, end source record (exclusive), part index, parts in the group.
 * *n_items receives the item count (also on KMC_ECAPACITY). chain_cut (host,
 * KMC_MAX_CHAINS + 1 int32): chain q runs items chain_cut[q] .. chain_cut[q +
 * 1] - 1 (cut at lysosome boundaries into runs of about equal source records);
 * *n_chains receives the chain count. Bad arguments give KMC_EINVAL. */
kmc_status kmc_plan_items(const int32_t *n, int32_t n_lys, kmc_precision prec, int32_t tpl,
                          int32_t chunk, int32_t blocks_per_sm, int32_t n_sms, int32_t *items_out,
                          int64_t cap, int64_t *n_items, int32_t *chain_cut, int32_t *n_chains);

/* Largest neighbour rank of kmc_local_concentration (the paper uses 20). */
#define KMC_PHI_MAX_N 64

/* Eq. 8 (Sec. III.5): the local volume concentration around each NP of
 * lysosome `lys`, phi_N,i = 3 N V_i / (4 pi r_N^3) with r_N the distance from
 * NP i to its N-th nearest neighbour in the lysosome. Computed on the device
 * over all pairs in FP64; 1 <= N <= min(n - 1, KMC_PHI_MAX_N), else
 * KMC_EINVAL. Writes phi[n] (host buffer of capacity cap; KMC_ECAPACITY and
 * *written = n if too small). Synchronises the context's stream. */
kmc_status kmc_local_concentration(kmc_ctx *ctx, int32_t lys, int32_t N, double *phi,
                                   int64_t cap, int64_t *written);

/* Radial profile of the last run (Sec. III.4, Fig. 8): the NPs of lysosome
 * `lys` binned into n_shells shells of equal thickness R / n_shells about the
 * lysosome's frame origin (kmc_lysosome.center, else the centroid of pos). NP
 * i, at distance r_i from it, goes to shell floor(n_shells r_i / R), the last
 * shell also taking r_i >= R. radius > 0 sets R; radius <= 0 takes the
 * smallest sphere about the origin holding every NP whole,
 * R = max_i (r_i + (3 V_i / 4 pi)^(1/3)). out [n_shells][4] (host, capacity
 * cap): NP count, then volume-weighted means sum V_i x_i / sum V_i over the
 * shell of x = the NP's hysteresis area (J/m^3 per cycle, KMC_READ_NP_ENERGY
 * over V_i), its Delta_Hdip (T, KMC_READ_DHDIP) and its phi_N (Eq. 8; 0 when
 * N = 0); 0 for an empty shell. *radius_used (may be NULL) receives R.
 * KMC_ESTATE before the first kmc_run. */
kmc_status kmc_shell_profile(kmc_ctx *ctx, int32_t lys, double radius, int32_t n_shells,
                             int32_t N, double *out, int64_t cap, int64_t *written,
                             double *radius_used);

/* The Ref. [8] program's mode (Sec. II.3) on the device, for non-interacting
 * NPs: no sampling and no dipolar field. Each NP carries the probability of
 * each energy well; when the applied field (along z) moves the wells, the
 * probability of an old well goes to the new minimum whose basin contains it,
 * and Eqs. 3-5 relax the two occupations towards equilibrium over each step.
 * Arguments as kmc_create (positions are not used) and kmc_run, without a
 * seed; runs in FP64 on the device, one thread per NP. Writes the
 * volume-weighted mean m_z after each recorded step of every lysosome,
 * loop_M [n_lys][S * (periods - discard)] (host buffer of capacity cap;
 * KMC_ECAPACITY and *written = the size needed if too small). Starts from
 * m = +-easy axis with m_z >= 0, like kmc_create. Synchronous. */
kmc_status kmc_mean_run(const kmc_lysosome *lys, int32_t n_lys, const double *mu0Hmax,
                        int32_t n_amp, double f, int32_t steps_per_period, int32_t periods,
                        int32_t discard_periods, double *loop_M, int64_t cap,
                        int64_t *written);

/* What kmc_regenerate redraws (bit mask). */
enum { KMC_REGEN_AXES = 1, KMC_REGEN_POSITIONS = 2 };

/* Sample regeneration between loops (Sec. II.4), on the device: the paper
 * averages loops over fresh easy axes and, around fixed mean positions (the
 * nodes of a cubic lattice), fresh positions. For lysosome `lys` (-1: all):
 *   KMC_REGEN_AXES       easy axes uniform on the sphere;
 *   KMC_REGEN_POSITIONS  position = mean position + rho e, e uniform on the
 *                        sphere, rho uniform on [0, disorder] (m); the mean
 *                        positions are those given to kmc_create;
 * then every moment of the lysosome restarts along its axis with m_z >= 0.
 * Draws: Philox4x32-10, key (seed lo, seed hi), counter (loop, 0x80000000 |
 * sub, NP, lysosome) with sub 0 for the axis and 1, 2 for the displacement;
 * two 53-bit uniforms per call from words (0, 1) and (2, 3) as for the kMC
 * draw; z = 1 - 2 u0 and azimuth 2 pi u1 give a point on the sphere. The
 * result is what kmc_create would build from the drawn axes and positions;
 * the global step counter carries on. A checkpoint (kmc_save) does not hold
 * the geometry: after kmc_load, call kmc_regenerate again with the same
 * arguments. Errors: KMC_EINVAL (lys out of range, bad mask, disorder < 0 or
 * not finite). Synchronises the context's stream. */
kmc_status kmc_regenerate(kmc_ctx *ctx, int32_t lys, int32_t what, double disorder,
                          uint64_t seed, uint32_t loop);

/* Random sequential addition (Sec. II.4; the alternative to the lattice) of
 * the NPs of lysosome `lys` on the device: spheres of `diameter` (m) placed
 * one after another at candidate centres uniform in the ball of radius
 * radius - diameter/2 (m) about the lysosome's centre, each kept iff no kept
 * sphere lies closer than `diameter`, until every NP has a place; NP i takes
 * the i-th kept centre. Candidate c comes from Philox4x32-10, key (seed lo,
 * seed hi), counter (loop, 0x80000000 | sub, c, lys): direction from sub 3 as
 * for the axes, radius (radius - diameter/2) max(u0, u1, u2) from subs 4 and
 * 5. The kept centres are exactly those of the sequential rule, taken batch
 * by batch. Then, as kmc_regenerate does, the NP arrays follow the new
 * positions and the moments restart along the axes. max_candidates (<= 0:
 * 1000 n) bounds the candidates; KMC_ESTATE if they run out (positions left
 * unchanged). *candidates_used (may be NULL) = candidates consumed.
 * KMC_EINVAL unless 0 < diameter < 2 radius. */
kmc_status kmc_regenerate_rsa(kmc_ctx *ctx, int32_t lys, double radius, double diameter,
                              uint64_t seed, uint32_t loop, int64_t max_candidates,
                              int64_t *candidates_used);

/* Failure-detection test hook (FP64 contexts). Launches one step whose every
 * staged copy waits for 16 bytes more than it delivers, so each block's bounded
 * wait runs out (after 1 ms instead of 2 s) and reports through the device
 * error word; no kernel faults, traps or hangs, and the blocks stop before
 * writing any state. Returns what such a stall returns, KMC_ETIMEOUT, then
 * clears the error so the context stays usable (the next kmc_run proceeds as
 * if the call had not been made). KMC_EINVAL on an FP32 context. */
kmc_status kmc_debug_stall(kmc_ctx *ctx);

/* Frees the context and its device memory. NULL-safe. */
void kmc_destroy(kmc_ctx *ctx);

/* Largest NP count kmc_dipolar_field_noalloc accepts. */
#define KMC_NOALLOC_MAX_N 8192

/* The dipolar field of one lysosome, computed like the FP32-mixed pair sum of
 * kmc_run (split source ranges, compensated sums, the same pair term), for
 * callers that cannot call cudaMalloc: code inside another framework's memory
 * pool, processes whose device memory is reserved up front, or libraries
 * handed device pointers by their caller. It allocates nothing: no
 * cudaMalloc, cudaFree or allocating library call. The paper has no
 * counterpart: this entry point exists only for such callers.
 *
 *   n       NPs, 1 .. KMC_NOALLOC_MAX_N (otherwise KMC_ECAPACITY)
 *   pos     DEVICE [n][3] centres, m (8-byte aligned)
 *   m       DEVICE [n][3] unit moments
 *   vol     DEVICE [n] volumes, m^3
 *   Ms      A/m, > 0
 *   center  HOST [3] origin of the float32 frame, m (e.g. the lysosome centre)
 *   length  unit of the float32 frame, m, > 0 (e.g. the NP diameter)
 *   B       DEVICE [n][3] output: mu0 H_dip on every NP, the all-pairs dipolar
 *           field of the other NPs, T
 *   status  DEVICE int32 output, or NULL: KMC_OK, or KMC_ETIMEOUT if a
 *           shared-memory staging wait of this call ran out (about 2 s); the
 *           targets it affected then hold NaN in B
 *   cuda_stream  stream to queue on (NULL: the default stream)
 * All pointers are owned by the caller. pos, m, vol, B and status must be
 * device (or managed) memory of the current device, which the call checks
 * (cudaPointerGetAttributes) before it launches anything. The call only
 * queues work: B and *status are valid once the stream has reached them.
 * Its working memory is one static device array of about 2 MB that every GPU
 * loading the library holds until the process exits. Every call shares that
 * array and leaves its contents behind (the call clears what must start at
 * zero); calls that overlap on the GPU (other streams, other host threads)
 * race on it. The first call on each device, and the first after the
 * device's context changed, looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture. Setting the environment variable
 * KMC_FAULT=noalloc_stall makes every staging wait expect more bytes than
 * its copy delivers and give up after 1 ms (a test of the timeout path; no
 * copy is left unfinished). Errors: KMC_EINVAL (NULL or misaligned pointer, a
 * buffer that is not device memory of the current device, Ms or length not
 * positive, center not finite), KMC_ECAPACITY (n out of range), KMC_ECUDA
 * (launch failed). */
kmc_status kmc_dipolar_field_noalloc(int32_t n, const double *pos, const double *m,
                                     const double *vol, double Ms, const double *center,
                                     double length, double *B, int32_t *status,
                                     void *cuda_stream);

/* Message of the calling thread's last failure ("" if none). */
const char *kmc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* KMC_H */
