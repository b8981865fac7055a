// kmc_types.h -- data shared by the host side (kmc_api.cu) and the kernels
// (kmc_step.cu) of libkmc.
//
// Reduced units used on the device (chosen so that the pair sum of Eq. 1 is
// purely geometric and every quantity is O(0.01..10)):
//   length  : L = diameter of the lysosome's mean NP volume, positions taken
//             relative to the lysosome's frame origin;
//   field   : b = mu0 H / (mu0 M_S);
//   energy  : e = E / (mu0 M_S^2 V), so Eq. 2 reads e = k sin^2 th - b cos(th - phi)
//             with k = K_eff / (mu0 M_S^2);
//   source  : w_j = V_j / (4 pi L^3), so that Eq. 1 reads
//             b_dip,i = sum_{j != i} [3 (mu_j . d) d / r^5 - mu_j / r^3],
//             mu_j = w_j m_j, d = r_j - r_i in units of L.
#pragma once
#include <stddef.h>
#include <stdint.h>

namespace kmc {

struct __align__(32) dbl4 {  // FP64 record: x, y, z and a fourth value
  double x, y, z, w;
};

// FP32 source record: two NPs (even, odd) interleaved so that each 8-byte
// pair of lanes feeds one packed f32x2 instruction. Per NP j: its position,
// t_j = 3 w_j m_j and n_j = -w_j m_j. With d = r_j - r_i and q = 1/|d|, the
// pair term of Eq. 1, w_j (3 (m_j.d) d / |d|^5 - m_j / |d|^3), is then
// q^3 (u d + n_j) with u = (t_j.d) q^2: three multiply-adds per component and
// one sum per component instead of separate sums of the two terms. 80 bytes:
// five 16-byte shared-memory loads, the last 8 bytes padding. n sits before t:
// this order ran 1-4 % faster than t before n (same instructions). A lysosome with
// an odd NP count ends with a padding NP far away (x = y = z = 1e4 L) whose
// moment is zero.
struct __align__(16) SrcPair {
  float x[2], y[2];
  float z[2], nx[2];
  float ny[2], nz[2];
  float tx[2], ty[2];
  float tz[2], pad[2];
};
constexpr int kRecU2 = 5;  // 16-byte words per SrcPair
static_assert(sizeof(SrcPair) == 16 * kRecU2, "SrcPair is five 16-byte words");
// the FP32 pair loops read the words as x|y, z|nx, ny|nz, tx|ty, tz
static_assert(offsetof(SrcPair, z) == 16 && offsetof(SrcPair, nx) == 24 &&
                  offsetof(SrcPair, ny) == 32 && offsetof(SrcPair, nz) == 40 &&
                  offsetof(SrcPair, tx) == 48 && offsetof(SrcPair, ty) == 56 &&
                  offsetof(SrcPair, tz) == 64,
              "SrcPair word order as the pair loops read it");

// Moment part of a source record from w and the unit moment (every writer
// uses this, so that records rebuilt from the state match the ones the step
// wrote, bit for bit).
__host__ __device__ inline void set_source_moment(SrcPair &r, int h, float w, float mx,
                                                  float my, float mz) {
  const float wx = w * mx, wy = w * my, wz = w * mz;
  r.tx[h] = 3.0f * wx;
  r.ty[h] = 3.0f * wy;
  r.tz[h] = 3.0f * wz;
  r.nx[h] = -wx;
  r.ny[h] = -wy;
  r.nz[h] = -wz;
}

constexpr int kGrid = 200;   // scan points of step iv (Sec. II.1)
constexpr int kTargets = 32; // target NPs per work item (one per lane of a warp)
constexpr float kPadCoord = 1e4f;
constexpr double kLoopScale = 4611686018427387904.0;  // 2^62, fixed point of the loop

struct LysDev {
  int32_t off;      // first NP of the lysosome in the flat per-NP arrays
  int32_t n;        // NPs
  int32_t roff;     // first source record (FP32: NP pairs, FP64: NPs)
  int32_t t_zero;   // 1 if T == 0: steps vi-vii skipped
  double k;         // K_eff / (mu0 M_S^2)
  double bmax;      // mu0 H_max / (mu0 M_S), set by each run
  double lognu0t;   // ln(t_step / tau0), set by each run
};

// One work item = one block: 32 targets of lysosome l against the source
// records [j0, j1). A target group whose sources are split over nsplit items
// has its items stored consecutively (split = 0 .. nsplit-1); the last of
// them to finish combines the partial sums and runs steps iii-vii.
struct Item {
  int32_t l;       // lysosome
  int32_t t0;      // first target (index within the lysosome)
  int32_t nt;      // targets, 1..32 (1..64 with two targets per lane)
  int32_t gid;     // target group (index of its arrival counter)
  int32_t j0, j1;  // source records of this item (relative to the lysosome)
  int32_t split;   // index of this item within its group
  int32_t nsplit;  // items in the group
  int32_t off;     // the lysosome's first NP and first source record (its
  int32_t roff;    // LysDev off and roff), so that one load reaches both
};

// Symmetric pair form (FP32-mixed, kmc_field_sym / kmc_update_sym). A
// lysosome's NPs are cut into cells of kCell = 64 (32 source records; the
// records of every lysosome start on a cell boundary and its last cell is
// padded with far-away NPs without moment). A row group g is gc consecutive
// cells (gc = warps x cells per warp). Every unordered pair of NPs is
// evaluated once: pairs between a row group's cells and the cells above it
// (h >= (g + 1) gc) by the symmetric field kernel, which adds T_ij to the
// target's forward sum and T_ji to the source's reverse sum; pairs inside a
// row group by ordered evaluation in the group's diagonal item.
constexpr int kCell = 64;
constexpr int kCellRec = kCell / 2;

struct SymItem {   // one block of kmc_field_sym
  int32_t l;       // lysosome
  int32_t g;       // row group: target cells g gc .. g gc + gc - 1
  int32_t h0, h1;  // source cells [h0, h1); h0 = h1 = -1: the group's diagonal item
  int32_t fwd;     // forward-partial slot of this item
  int32_t rbase;   // first reverse slot of the lysosome
  int32_t pad[2];
};

struct SymUpd {    // one block of kmc_update_sym: up to 32 targets of one cell
  int32_t l, t0, nt;    // lysosome, first target, targets (1..32)
  int32_t fwd0, nfwd;   // forward-partial slots of the target's row group (consecutive)
  int32_t rev0, nrev;   // reverse slots of the targets' cell, one per row group below
  int32_t gt0;          // t0 minus the first target of the row group
};

// First reverse slot of cell h within its lysosome: cell h' holds one slot
// per row group below it, floor(h' / gc) of them.
__host__ __device__ inline int sym_rev_offset(int h, int gc) {
  const int q = h / gc, r = h % gc;
  return gc * q * (q - 1) / 2 + r * q;
}

struct RunState {   // advanced on the device at the end of each field period
  long long step_base;  // global index of step 0 of the current period
  int32_t period;       // period index within the run (< 0: not recorded)
  int32_t pad;
};

struct DebugOut {   // optional per-NP intermediates (device pointers)
  double *bdip;     // [N][3] reduced dipolar field
  double *dE;       // [N][2] reduced barriers
  double *P;        // [N]
  double *u;        // [N]
  int32_t *flags;   // [N]
};

struct StepArgs {
  const Item *items;
  const LysDev *lys;
  const void *pos;          // [N] float4 / dbl4: x, y, z (units of L), w (targets)
  const void *axis;         // [N] float4 / dbl4 unit easy axis
  void *m;                  // [N] float4 / dbl4 unit moments (owner-updated)
  void *src[2];             // source records, ping-pong: FP32 SrcPair, FP64 dbl4 moments
  const void *src_pos;      // FP64 only: [N] dbl4 source positions (static)
  const double *beta;       // [N] mu0 M_S^2 V_i / (k_B T)
  const double *vfrac;      // [N] V_i / sum of V over the lysosome
  double *e_acc;            // [N] sum_k b_k (m_z,k+1 - m_z,k) over recorded steps
  double *dh_acc;           // [N] Eq. 6: sum over recorded periods of b_dip,z at
                            // step 0 (+b_max) minus b_dip,z at step S/2 (-b_max)
  long long *loop_m;        // [n_lys][n_rec] volume-weighted mean m_z in fixed point
                            // (units of 2^-62): integer sums do not depend on the
                            // order in which blocks add, so runs are reproducible
  unsigned long long *counters;  // [n_lys][kCounters] (enum below)
  int32_t *err;             // device error word
  float *partial;           // scratch: [items][12][32] floats of partial sums
  int32_t *arrivals;        // scratch: [groups] arrival counters, zero between launches
  const RunState *rs;
  double cos_k;             // cos(2 pi k / S)
  unsigned long long seed;
  int32_t k_local;          // step within the period
  int32_t S;
  int32_t discard;
  int32_t n_rec;            // recorded steps per lysosome (loop_m stride)
  DebugOut dbg;
  int32_t debug;
  int32_t force_rescan;     // test hook (kmc_debug_step only): every FP32 target is
                            // scanned again in FP64, as a noisy scan would be
  // failure-detection test hook (FP64 kernel): every tile's expected byte
  // count exceeds its copies by stall_tx, so its wait can only run out, after
  // stall_wait_ns; 0 in every production launch
  uint32_t stall_tx;
  int32_t n_items;          // work items of this launch (bounds checks of KMC_DEBUG builds)
  unsigned long long stall_wait_ns;
  int32_t n_lys;            // lysosomes of the context (bounds checks of KMC_DEBUG builds)
  int32_t gc;               // symmetric form: cells per row group
  // symmetric form: the field kernel's items, the update kernel's items and the
  // partial sums between them: forward [slot][6][gc 64] (sum, -error of 3
  // components per target of the row group), reverse [slot][3][64]
  const SymItem *sitems;
  const SymUpd *supd;
  float *sfwd;
  float *srev;
  int32_t n_upd;
  // persistent period kernel (kmc_persist_f32): the cosine of each step of the
  // period (host-computed, as the per-step launches receive it), the grid
  // barrier's counters and its time limit; failure-detection test hook: block
  // stall_block does not arrive at the barrier of step stall_step (-1: none)
  int32_t stall_block;
  const double *cosk;
  uint32_t *gbar;
  unsigned long long barrier_ns;
  int32_t stall_step;
  int32_t pad5;
};

// Ref. [8] mode (kmc_mean.cuh): per lysosome, per work item, arguments.
struct MeanLysDev {
  int32_t off, n;   // first NP, NPs
  int32_t t_zero;   // T = 0: no relaxation (the wells are only followed)
  int32_t pad;
  double k;         // K_eff / (mu0 M_S^2)
  double bmax;      // mu0 H_max / (mu0 M_S)
  double lognu0t;   // ln(t_step / tau0)
};

struct MeanItem {   // 32 NPs of one lysosome, one warp
  int32_t l, t0, nt, pad;
};

struct MeanArgs {
  const MeanItem *items;
  int32_t n_items;
  int32_t S, periods, discard, n_rec;
  const MeanLysDev *lys;
  const dbl4 *axis;      // [N] unit easy axes
  const double *beta;    // [N] mu0 M_S^2 V_i / (k_B T)
  const double *vfrac;   // [N] V_i / sum V over the lysosome
  const double *cos_k;   // [S] cos(2 pi k / S)
  long long *loop;       // [n_lys][n_rec] volume-weighted <m_z>, units of 2^-62
  int32_t *err;
};

// Sample regeneration between loops (kmc_regen.cuh), one lysosome per launch.
// kRegenGiven: positions already written to pos_si (random sequential
// addition); the kernel only brings the NP's other arrays in line with them
enum : int32_t { kRegenAxes = 1, kRegenPositions = 2, kRegenGiven = 4 };

// Random sequential addition on the device, one batch of B candidates
// (candidate indices c0 .. c0 + B - 1). The batch keeps, in candidate order,
// each candidate that clears every sphere kept before it, until n are kept.
constexpr int kRsaMaxConf = 8;  // listed conflicts per candidate; more: checked in full
struct RsaArgs {
  double Rb;                   // radius of the ball of centres, R - d/2, m
  double d2;                   // d^2, m^2
  unsigned long long seed;
  uint32_t loop;
  int32_t lys;
  long long c0;                // first candidate of the batch
  int32_t B;                   // candidates in the batch
  int32_t n;                   // spheres to keep
  int32_t *kept;               // [1] spheres kept so far (updated by the batch)
  long long *used;             // [1] candidates used when the n-th was kept
  double *pos;                 // [n][3] kept centres, m, about the lysosome centre
  float4 *posf;                // [n] the same in FP32 (x, y, z, 0), for the pre-screen
  float d2_lo, d2_hi;          // FP32 squared distances below d2_lo clash and above d2_hi
                               // clear for certain; in between the FP64 test decides
  double *cand;                // [B][3] scratch
  int32_t *clear;              // [B] 1 if the candidate clears the earlier batches' spheres
  int32_t *nconf;              // [B] earlier candidates of the batch closer than d
  int32_t *conf;               // [B][kRsaMaxConf] their indices
};
constexpr int kRsaMaxBatch = 2048;  // candidates per batch at most
struct RegenArgs {
  int32_t off, n, lys, what;
  uint32_t loop;
  int32_t fp32;
  unsigned long long seed;
  double disorder;        // largest displacement, m
  double len, cx, cy, cz; // length unit and frame origin of the lysosome, m
  const double *nodes;    // [N][3] mean positions (those given at creation), m
  void *pos, *axis, *m;   // float4 / dbl4 per NP, as built at creation
  void *pos64;            // FP32 contexts: [N] dbl4 positions in FP64
  double *pos_si;         // [N][3] out: the new positions, m
};

// Error bits written to the device error word.
enum : int32_t {
  kErrTimeout = 1,     // an mbarrier wait gave up
  kErrExtrema = 2,     // more than two minima or maxima (cannot happen for Eq. 2)
  kErrNonFinite = 4,   // a non-finite dipolar field, barrier or probability: the
                       // NP kept its moment (two NPs at one point, e.g. closer
                       // than the float32 frame resolves)
  kErrBounds = 8,      // KMC_DEBUG builds: an index failed its bounds check; the
                       // access was skipped and err[1] holds the check's site
};

// Sites of the KMC_DEBUG bounds checks (err[1] holds the first that failed).
enum : int32_t {
  kSiteItem = 1,       // block index beyond the launch's work items
  kSiteLys = 2,        // item's lysosome beyond the context's
  kSiteTargets = 3,    // item's targets outside its lysosome, or more than a block holds
  kSiteSources = 4,    // item's source records outside its lysosome's
  kSiteSplit = 5,      // item's part index or part count inconsistent
  kSiteTile = 6,       // a staged tile beyond the item's source records or the buffer
  kSiteBracket = 7,    // a bracket's grid node or rank outside the scan's tables
};

#ifdef KMC_DEBUG
// Records a failed check (error bit and, first come, its site).
__device__ __forceinline__ void debug_fail(int32_t *err, int32_t site) {
  atomicOr(err, kErrBounds);
  atomicCAS(err + 1, 0, site);
}
#define KMC_DCHECK(cond, err, site) ((cond) ? true : (kmc::debug_fail((err), (site)), false))
#else
#define KMC_DCHECK(cond, err, site) true
#endif

// Per-lysosome counters of a run, in NP-steps (KMC_READ_COUNTERS).
enum : int32_t {
  kCntJumps = 0,       // moments that jumped (u < P)
  kCntNear = 1,        // draws within 1e-9 of P
  kCntOneMin = 2,      // profiles with a single minimum
  kCntFallback = 3,    // working planes spanned by axis and moment (field along axis)
  kCntRescan = 4,      // FP32 scans redone in FP64 (more than four sign changes)
  kCntPolish = 5,      // FP32 barriers recomputed in FP64 near switching
  kCntNonFinite = 6,   // NPs held because the field or barrier was not finite
  kCounters = 8,       // slots per lysosome (the last is reserved, always 0)
};

// Bits of the test hook's per-NP flags (kmc_debug_step).
enum : int32_t {
  kFlagJumped = 1 << 2,
  kFlagNear = 1 << 3,
  kFlagFallback = 1 << 4,
  kFlagRescan = 1 << 5,
  kFlagPolish = 1 << 6,
  kFlagNonFinite = 1 << 7,
};

}  // namespace kmc
