// kmc_api.cu -- the C ABI of libkmc (include/kmc.h): contexts, device memory,
// work items, the CUDA-graph step loop, the launch-shape autotuner,
// checkpoints and the test hook. All arithmetic of the kMC step itself lives
// in kmc_step.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "kmc.h"
#include "kmc_launch.h"
#include "kmc_local.h"

using kmc::dbl4;
using kmc::Item;
using kmc::LysDev;
using kmc::RunState;
using kmc::SrcPair;
using kmc::StepArgs;

namespace {

constexpr double kMu0 = 4.0e-7 * 3.14159265358979323846;
constexpr double kKB = 1.380649e-23;
constexpr double kPi = 3.14159265358979323846;
// Lysosomes are independent: a run advances up to kMaxChains disjoint sets of
// them as parallel branches of the period graph, each branch one step kernel
// per step, so one set's update phase overlaps the pair sums of the others
// instead of every step ending in a device-wide barrier.
constexpr int kMaxChains = KMC_MAX_CHAINS;

thread_local std::string g_last_error;

kmc_status fail(kmc_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

#define KMC_CUDA(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return fail(KMC_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));       \
  } while (0)

#define KMC_TRY(x)                 \
  do {                             \
    kmc_status s_ = (x);           \
    if (s_ != KMC_OK) return s_;   \
  } while (0)

bool is_finite(double x) { return std::isfinite(x); }

// Host staging bytes for device records (float4, dbl4, SrcPair), allocated on
// a 64-byte boundary so that records can be written and read in place.
template <typename T>
struct RecordAlloc {
  using value_type = T;
  static constexpr std::size_t kAlign = 64;
  RecordAlloc() = default;
  template <typename U>
  RecordAlloc(const RecordAlloc<U> &) {}
  T *allocate(std::size_t n) {
    return static_cast<T *>(::operator new(n * sizeof(T), std::align_val_t(kAlign)));
  }
  void deallocate(T *p, std::size_t) { ::operator delete(p, std::align_val_t(kAlign)); }
  template <typename U>
  bool operator==(const RecordAlloc<U> &) const { return true; }
  template <typename U>
  bool operator!=(const RecordAlloc<U> &) const { return false; }
};
using HostBytes = std::vector<unsigned char, RecordAlloc<unsigned char>>;

// A named range on the host timeline of a profiler (NVTX; no cost without one).
struct Phase {
  explicit Phase(const char *name) { nvtxRangePushA(name); }
  ~Phase() { nvtxRangePop(); }
  Phase(const Phase &) = delete;
  Phase &operator=(const Phase &) = delete;
};

template <typename V>
V make4(double x, double y, double z, double w) {
  V v;
  v.x = static_cast<decltype(v.x)>(x);
  v.y = static_cast<decltype(v.y)>(y);
  v.z = static_cast<decltype(v.z)>(z);
  v.w = static_cast<decltype(v.w)>(w);
  return v;
}

// Source records (FP32: positions, 3 w_i m_i and -w_i m_i; FP64: w_i m_i) of every NP into
// the source buffer of parity par.
__global__ void sources_f32(const float4 *__restrict__ pos, const float4 *__restrict__ m,
                            const int *__restrict__ slot, SrcPair *__restrict__ src, long long n) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const float4 p = pos[i], q = m[i];
  const int s = slot[i];
  SrcPair &r = src[s >> 1];
  r.x[s & 1] = p.x;
  r.y[s & 1] = p.y;
  r.z[s & 1] = p.z;
  kmc::set_source_moment(r, s & 1, p.w, q.x, q.y, q.z);
}

__global__ void sources_f64(const dbl4 *__restrict__ pos, const dbl4 *__restrict__ m,
                            dbl4 *__restrict__ mu, long long n) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const dbl4 p = pos[i], q = m[i];
  dbl4 r;
  r.x = p.w * q.x;
  r.y = p.w * q.y;
  r.z = p.w * q.z;
  r.w = 0.0;
  mu[i] = r;
}

struct Shape {
  int warps = 0, tile = 0, chunk = 0;
  int tpl = 1;  // targets per lane: 2 or 3 run 64- or 96-target groups (FP32 only)
  int rpl = 1;  // replicas per lane: 2 or 4 run replica lysosomes together (FP32, warps =
                // rpl, 2 rpl or 4 rpl: one, two or four warps per replica)
  // symmetric pair form (FP32): cells per warp (1 or 2; tpl = 2 sym, tile = 32,
  // chunk = source NPs per field item, 0 = a whole row); 0 = the ordered kernels
  int sym = 0;
  // cluster split (FP32, one target per lane): 2 = every target group's two
  // source parts run as a two-CTA cluster and exchange their sums through
  // distributed shared memory; 0 = through global memory
  int cl = 0;
  // symmetric form's update kernel: 0 = one warp per update item, 1 = one block
  int supd = 0;
  // 1: the whole field period as one persistent cooperative launch (FP32, one
  // target per lane) with a grid barrier after each step
  int persist = 0;
  bool operator==(const Shape &o) const {
    return warps == o.warps && tile == o.tile && chunk == o.chunk && tpl == o.tpl &&
           rpl == o.rpl && sym == o.sym && cl == o.cl && supd == o.supd && persist == o.persist;
  }
};

struct TuneKey {
  int prec;
  long long N;
  int n_lys, max_n, tpl_mode, rpl_mode, reps;  // reps: replica sets available (bits)
  int form_mode, cl_mode, supd_mode, persist_mode;
  bool operator<(const TuneKey &o) const {
    return std::tie(prec, N, n_lys, max_n, tpl_mode, rpl_mode, reps, form_mode, cl_mode,
                    supd_mode, persist_mode) <
           std::tie(o.prec, o.N, o.n_lys, o.max_n, o.tpl_mode, o.rpl_mode, o.reps, o.form_mode,
                    o.cl_mode, o.supd_mode, o.persist_mode);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, Shape> g_tune_cache;

std::mutex g_init_mu;
std::vector<int> g_init_done;  // per device ordinal

kmc_status ensure_device_init() {
  int dev = 0;
  KMC_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_init_mu);
  if (static_cast<int>(g_init_done.size()) <= dev) g_init_done.resize(dev + 1, 0);
  if (!g_init_done[dev]) {
    KMC_CUDA(kmc::init_device());
    g_init_done[dev] = 1;
  }
  return KMC_OK;
}

}  // namespace

namespace kmc {
// Lets other translation units of the library report through kmc_last_error().
void set_last_error(const char *msg) { g_last_error = msg ? msg : ""; }
}  // namespace kmc

struct kmc_ctx {
  int fp32 = 0;
  int n_lys = 0;
  long long N = 0;
  size_t vbytes = 0;  // sizeof(float4) or sizeof(dbl4)
  std::vector<int> off, n, roff;
  long long n_records = 0;  // source records over all lysosomes
  std::vector<double> Ms, Keff, T, tau0, rho, vsum;
  std::vector<double> vol;  // [N]
  std::vector<LysDev> h_lys;
  // device memory
  LysDev *d_lys = nullptr;
  void *d_pos = nullptr, *d_axis = nullptr, *d_m = nullptr, *d_src[2] = {nullptr, nullptr};
  int *d_slot = nullptr;  // FP32: record * 2 + half of each NP
  double *d_beta = nullptr, *d_vfrac = nullptr, *d_eacc = nullptr;
  double *d_dh = nullptr;     // [N] Eq. 6 accumulator (reduced field)
  void *d_pos64 = nullptr;    // FP32 contexts: [N] dbl4 positions in FP64 (x, y, z, w)
  double *d_phi = nullptr;    // [max n] scratch of kmc_local_concentration
  float4 *d_phif = nullptr;   // [max n] its FP32 copy of the positions
  std::vector<double> len;    // [n_lys] length unit L, m
  std::vector<double> ctr;    // [n_lys][3] frame origin, m
  std::vector<double> pos_si; // [N][3] current positions, m
  double *d_nodes = nullptr;  // [N][3] positions given at creation (mean positions), m
  double *d_possi = nullptr;  // [N][3] positions written by kmc_regenerate, m
  long long *d_loop = nullptr;  // fixed point, units of 2^-62
  unsigned long long *d_cnt = nullptr;
  int32_t *d_err = nullptr;
  RunState *d_rs = nullptr;
  size_t loop_cap = 0;
  // work items for the current shape and their scratch
  Item *d_items = nullptr;
  size_t items_cap = 0;
  int n_items = 0;
  float *d_partial = nullptr;
  size_t partial_cap = 0;  // items
  int32_t *d_arrivals = nullptr;
  size_t arrivals_cap = 0;
  Shape items_shape;  // shape the items were built for
  std::vector<int> chain_cut;  // chain q runs items chain_cut[q] .. chain_cut[q + 1] - 1
  // symmetric form: field and update items, their chains, the partial sums
  kmc::SymItem *d_sitems = nullptr;
  size_t sitems_cap = 0;
  kmc::SymUpd *d_supd = nullptr;
  size_t supd_cap = 0;
  float *d_sfwd = nullptr, *d_srev = nullptr;
  size_t sfwd_cap = 0, srev_cap = 0;  // floats
  int n_sitems = 0, n_supd = 0;
  std::vector<int> sym_cut_items, sym_cut_upd;
  int form_mode = 0;           // pair form: 0 = the autotuner's choice, 1 = ordered, 2 = symmetric
  int cl_mode = 0;             // cluster split: 0 = the autotuner's choice, 1 = off, 2 = on
  int supd_mode = 0;           // symmetric update: 0 = the autotuner's, 1 = warp, 2 = block per item
  int persist_mode = 0;        // persistent period: 0 = the autotuner's choice, 1 = off, 2 = on
  // persistent period: the steps' cosines and the grid barrier's counters
  double *d_cosk = nullptr;
  size_t cosk_cap = 0;
  uint32_t *d_gbar = nullptr;
  int tpl_mode = 0;            // targets per lane: 0 = the autotuner's choice, else 1, 2 or 3
  int rpl_mode = 0;            // replicas per lane: 0 = the autotuner's choice, 1 = off, 2 or 4
  bool rep_ok[5] = {};         // [k]: the lysosomes form sets of k identical consecutive ones
  cudaStream_t chain_st[kMaxChains] = {};  // branches 1.. of the period graph
  cudaEvent_t chain_ev[kMaxChains] = {};   // [0] fork, [q] join of branch q
  // debug outputs, allocated on first use
  double *d_dbg = nullptr;
  int32_t *d_dbg_flags = nullptr;
  cudaStream_t own_stream = nullptr, stream = nullptr;
  long long step_global = 0;
  // latest run
  bool have_run = false;
  int S = 0, periods = 0, discard = 0, n_rec = 0;
  double f = 0.0;
  std::vector<double> Hmax;
  // launch shape and the captured one-period graph
  Shape shape;
  cudaGraphExec_t gexec = nullptr;
  int g_S = -1, g_discard = -1, g_nrec = -1;
  Shape g_shape;
  unsigned long long g_seed = 0;
};

namespace {

template <typename T>
kmc_status dalloc(T **p, size_t bytes) {
  if (cudaMalloc(reinterpret_cast<void **>(p), bytes ? bytes : 16) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(KMC_ENOMEM, "cudaMalloc of %zu bytes failed", bytes);
  }
  return KMC_OK;
}

void drop_graph(kmc_ctx *c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
}

// Work items for source chunk `chunk`, largest lysosomes first; the items of
// a target group are consecutive.
//
// chunk = 0: one item per group of 32 targets. When the groups fit in one
// wave (at most blocks_per_sm per SM) but do not fill the SMs evenly
// (G = q P + r groups on P SMs), the r smallest groups are split into s parts
// each and placed last, so that the blocks, which start in order, give every
// SM q whole groups plus at most one part: the busiest SM then carries
// q + 1/s group-loads instead of q + 1.
std::vector<Item> build_items(const std::vector<int> &np, bool fp32, int chunk,
                              int blocks_per_sm, int n_sms, int *n_groups, int tpl) {
  const int gsize = kmc::kTargets * tpl;  // targets per group
  const int n_lys = static_cast<int>(np.size());
  std::vector<int> order(n_lys);
  for (int l = 0; l < n_lys; ++l) order[l] = l;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return np[x] > np[y]; });
  struct Group {
    int l, t0, nt, nrec;
  };
  std::vector<Group> groups;
  for (int l : order) {
    const int n = np[l];
    const int nrec = fp32 ? (n + 1) / 2 : n;
    for (int t0 = 0; t0 < n; t0 += gsize) groups.push_back({l, t0, std::min(gsize, n - t0), nrec});
  }
  const int G = static_cast<int>(groups.size());
  std::vector<int> parts(G, 1);
  if (chunk > 0) {
    for (int g = 0; g < G; ++g) {
      const int rchunk = fp32 ? chunk / 2 : chunk;
      parts[g] = std::max(1, (groups[g].nrec + rchunk - 1) / rchunk);
    }
    // A single chain over several waves of items: the last wave would hold
    // N mod slots full-size items and leave the other slots idle until they
    // end, since the next step waits for the whole launch. The last groups
    // (placed last, as they come) take one part more each until the items
    // fill whole waves; their smaller items then end the launch.
    const long long slots = static_cast<long long>(n_sms) * blocks_per_sm;
    long long N = 0;
    for (int g = 0; g < G; ++g) N += parts[g];
    if (n_sms > 0 && N > slots && N % slots != 0) {
      long long extra = slots - N % slots;
      for (int round = 0; extra > 0 && round < 64; ++round) {
        bool grew = false;
        for (int g = G - 1; g >= 0 && extra > 0; --g) {
          if (parts[g] >= groups[g].nrec) continue;  // a part holds one record at least
          ++parts[g];
          --extra;
          grew = true;
        }
        if (!grew) break;
      }
    }
  } else if (n_sms > 0 && G >= n_sms) {
    const int q = G / n_sms, r = G % n_sms;
    int best_s = 1;
    double best = 1.0;  // extra load of the busiest SM without splitting
    for (int s = 2; s <= 8 && r > 0; ++s) {
      const int per_sm = (r * s + n_sms - 1) / n_sms;
      if (q + per_sm > blocks_per_sm) break;
      const double load = static_cast<double>(per_sm) / s;
      if (load < best - 1e-9) {
        best = load;
        best_s = s;
      }
    }
    for (int g = G - r; g < G && best_s > 1; ++g)
      parts[g] = std::min(best_s, std::max(1, groups[g].nrec));
  }
  std::vector<Item> items;
  for (int g = 0; g < G; ++g) {
    const Group &gr = groups[g];
    const int S = parts[g];
    for (int s = 0; s < S; ++s) {
      Item it{};
      it.l = gr.l;
      it.t0 = gr.t0;
      it.nt = gr.nt;
      it.gid = g;
      it.j0 = static_cast<int>(static_cast<long long>(s) * gr.nrec / S);
      it.j1 = static_cast<int>(static_cast<long long>(s + 1) * gr.nrec / S);
      it.split = s;
      it.nsplit = S;
      items.push_back(it);
    }
  }
  *n_groups = G;
  return items;
}

// The launch plan of a batch of lysosomes of np[l] NPs: the items in launch
// order, and the cut of that list into chains. Pure host code (no device
// call), so that kmc_plan_items can show it without a GPU.
struct Plan {
  std::vector<Item> items;
  int groups = 0;
  std::vector<int> chain_cut;  // chain q runs items chain_cut[q] .. chain_cut[q + 1] - 1
};

Plan plan_items(const std::vector<int> &np, bool fp32, int chunk, int blocks_per_sm, int n_sms,
                int tpl) {
  Plan p;
  // with several chains the lysosomes' kernels interleave on the SMs, and the
  // split that evens out one device-wide wave does not apply
  const int chains = std::min(static_cast<int>(np.size()), kMaxChains);
  p.items = build_items(np, fp32, chunk, blocks_per_sm, chains > 1 ? 0 : n_sms, &p.groups, tpl);
  // chains: cut the item list (lysosome by lysosome, largest first) at
  // lysosome boundaries into runs of about equal source-record counts
  long long total = 0, acc = 0;
  for (const Item &it : p.items) total += it.j1 - it.j0;
  p.chain_cut.assign(1, 0);
  for (size_t u = 0; u < p.items.size(); ++u) {
    acc += p.items[u].j1 - p.items[u].j0;
    const bool boundary = u + 1 == p.items.size() || p.items[u + 1].l != p.items[u].l;
    const long long q = static_cast<long long>(p.chain_cut.size());
    if (boundary && q < chains && acc * chains >= total * q)
      p.chain_cut.push_back(static_cast<int>(u + 1));
  }
  const int n_items = static_cast<int>(p.items.size());
  if (p.chain_cut.back() != n_items) p.chain_cut.push_back(n_items);
  return p;
}

// The symmetric form's plan (kmc_field_sym, kmc_update_sym) for lysosomes of
// np[l] NPs and row groups of gc cells; src_cells source cells per field item
// (0: the whole range above the group). Lysosomes largest first; per
// lysosome its row groups in order, each as its diagonal item followed by
// its source ranges in order (the forward slots of a row group are
// consecutive); then one update item per 32 targets. Chains are cut at
// lysosome boundaries into runs of about equal pair counts, the field and
// update lists at the same lysosomes.
struct SymPlan {
  std::vector<kmc::SymItem> items;
  std::vector<kmc::SymUpd> upd;
  std::vector<int> cut_items, cut_upd;
  long long n_rev = 0;  // reverse slots (forward slots: one per item)
};

SymPlan plan_sym(const std::vector<int> &np, int gc, int src_cells) {
  SymPlan p;
  const int n_lys = static_cast<int>(np.size());
  std::vector<int> order(n_lys);
  for (int l = 0; l < n_lys; ++l) order[l] = l;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return np[x] > np[y]; });
  const int chains = std::min(n_lys, kMaxChains);
  double total = 0.0, acc = 0.0;
  for (int l = 0; l < n_lys; ++l) total += static_cast<double>(np[l]) * np[l];
  p.cut_items.assign(1, 0);
  p.cut_upd.assign(1, 0);
  for (int oi = 0; oi < n_lys; ++oi) {
    const int l = order[oi], n = np[l];
    const int nc = (n + kmc::kCell - 1) / kmc::kCell, ng = (nc + gc - 1) / gc;
    const int rbase = static_cast<int>(p.n_rev);
    p.n_rev += kmc::sym_rev_offset(nc, gc);
    std::vector<int> g0(ng), gn(ng);
    for (int g = 0; g < ng; ++g) {
      g0[g] = static_cast<int>(p.items.size());
      kmc::SymItem d{};
      d.l = l;
      d.g = g;
      d.h0 = d.h1 = -1;
      d.fwd = g0[g];
      d.rbase = rbase;
      p.items.push_back(d);
      const int step = src_cells > 0 ? src_cells : nc;
      for (int h0 = (g + 1) * gc; h0 < nc; h0 += step) {
        kmc::SymItem it{};
        it.l = l;
        it.g = g;
        it.h0 = h0;
        it.h1 = std::min(nc, h0 + step);
        it.fwd = static_cast<int>(p.items.size());
        it.rbase = rbase;
        p.items.push_back(it);
      }
      gn[g] = static_cast<int>(p.items.size()) - g0[g];
    }
    for (int t0 = 0; t0 < n; t0 += kmc::kTargets) {
      const int h = t0 / kmc::kCell, g = h / gc;
      kmc::SymUpd u{};
      u.l = l;
      u.t0 = t0;
      u.nt = std::min(kmc::kTargets, n - t0);
      u.fwd0 = g0[g];
      u.nfwd = gn[g];
      u.rev0 = rbase + kmc::sym_rev_offset(h, gc);
      u.nrev = h / gc;
      u.gt0 = t0 - g * gc * kmc::kCell;
      p.upd.push_back(u);
    }
    acc += static_cast<double>(n) * n;
    const int q = static_cast<int>(p.cut_items.size());
    if (oi + 1 < n_lys && q < chains && acc * chains >= total * q) {
      p.cut_items.push_back(static_cast<int>(p.items.size()));
      p.cut_upd.push_back(static_cast<int>(p.upd.size()));
    }
  }
  p.cut_items.push_back(static_cast<int>(p.items.size()));
  p.cut_upd.push_back(static_cast<int>(p.upd.size()));
  return p;
}

// Grows a device buffer to hold `need` elements (contents not kept); a failed
// allocation leaves it empty, and a grown buffer drops the captured graph.
template <typename T>
kmc_status grow(kmc_ctx *c, T **p, size_t *cap, size_t need);

kmc_status set_sym_items(kmc_ctx *c, const Shape &sh) {
  const int gc = sh.warps * sh.sym;
  std::vector<int> np(c->n.begin(), c->n.end());
  const SymPlan plan = plan_sym(np, gc, sh.chunk / kmc::kCell);
  KMC_CUDA(cudaStreamSynchronize(c->stream));
  KMC_TRY(grow(c, &c->d_sitems, &c->sitems_cap, plan.items.size()));
  KMC_TRY(grow(c, &c->d_supd, &c->supd_cap, plan.upd.size()));
  KMC_TRY(grow(c, &c->d_sfwd, &c->sfwd_cap,
               plan.items.size() * 3 * static_cast<size_t>(gc) * kmc::kCell));
  KMC_TRY(grow(c, &c->d_srev, &c->srev_cap,
               std::max<size_t>(1, static_cast<size_t>(plan.n_rev) * 3 * kmc::kCell)));
  KMC_CUDA(cudaMemcpy(c->d_sitems, plan.items.data(), sizeof(kmc::SymItem) * plan.items.size(),
                      cudaMemcpyHostToDevice));
  KMC_CUDA(cudaMemcpy(c->d_supd, plan.upd.data(), sizeof(kmc::SymUpd) * plan.upd.size(),
                      cudaMemcpyHostToDevice));
  c->n_sitems = static_cast<int>(plan.items.size());
  c->n_supd = static_cast<int>(plan.upd.size());
  c->sym_cut_items = plan.cut_items;
  c->sym_cut_upd = plan.cut_upd;
  c->items_shape = sh;
  return KMC_OK;
}

template <typename T>
kmc_status grow(kmc_ctx *c, T **p, size_t *cap, size_t need) {
  if (need <= *cap && *p) return KMC_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  KMC_TRY(dalloc(p, sizeof(T) * need));
  *cap = need;
  drop_graph(c);
  return KMC_OK;
}

kmc_status set_items(kmc_ctx *c, const Shape &sh) {
  if (c->items_shape == sh && (sh.sym ? c->d_sitems != nullptr : c->d_items != nullptr))
    return KMC_OK;
  if (sh.sym) {
    c->items_shape = Shape();
    return set_sym_items(c, sh);
  }
  // until the rebuild completes, no shape's items are valid
  c->items_shape = Shape();
  int dev = 0, n_sms = 0, per_sm = 0;
  KMC_CUDA(cudaGetDevice(&dev));
  KMC_CUDA(cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev));
  KMC_CUDA(kmc::step_blocks_per_sm(c->fp32, sh.warps, sh.tile, sh.tpl, &per_sm, sh.rpl));
  // replicas: the plan of the first lysosome of every set, whose items take
  // the set's other lysosomes along (kmc_step_f32_rep)
  std::vector<int> np;
  for (int l = 0; l < c->n_lys; l += sh.rpl) np.push_back(c->n[l]);
  Plan plan = plan_items(np, c->fp32, sh.chunk, per_sm, n_sms, sh.tpl);
  for (Item &it : plan.items) it.l *= sh.rpl;
  if (sh.persist) {  // one cooperative launch: every item's block resident at once
    int per = 0;
    KMC_CUDA(kmc::persist_blocks_per_sm(sh.warps, sh.tile, &per));
    if (static_cast<long long>(plan.items.size()) > static_cast<long long>(per) * n_sms)
      return fail(KMC_EINVAL, "the persistent period needs every work item resident (%zu items, "
                  "%d x %d blocks)", plan.items.size(), per, n_sms);
  }
  if (sh.cl == 2) {  // two-CTA clusters: exactly two parts per group, item 2 g + part
    for (size_t u = 0; u < plan.items.size(); ++u)
      if (plan.items[u].nsplit != 2 || plan.items[u].split != static_cast<int>(u & 1))
        return fail(KMC_EINVAL, "the cluster split needs exactly two source parts per group");
  }
  for (Item &it : plan.items) {
    it.off = c->h_lys[it.l].off;
    it.roff = c->h_lys[it.l].roff;
  }
  const std::vector<Item> &items = plan.items;
  const int groups = plan.groups;
  KMC_CUDA(cudaStreamSynchronize(c->stream));
  // a failed allocation leaves the buffer empty (null, capacity 0), so a
  // later call allocates again instead of using a stale capacity
  if (items.size() > c->items_cap) {
    if (c->d_items) cudaFree(c->d_items);
    c->d_items = nullptr;
    c->items_cap = 0;
    KMC_TRY(dalloc(&c->d_items, sizeof(Item) * items.size()));
    c->items_cap = items.size();
    drop_graph(c);
  }
  bool split = false;
  for (const Item &it : items) split = split || it.nsplit > 1;
  const size_t need_partial = split ? items.size() : 1;
  if (need_partial > c->partial_cap) {
    if (c->d_partial) cudaFree(c->d_partial);
    c->d_partial = nullptr;
    c->partial_cap = 0;
    KMC_TRY(dalloc(&c->d_partial, sizeof(float) * 12 * kmc::kTargets * 2 * need_partial));
    c->partial_cap = need_partial;
    drop_graph(c);
  }
  if (static_cast<size_t>(groups) > c->arrivals_cap) {
    if (c->d_arrivals) cudaFree(c->d_arrivals);
    c->d_arrivals = nullptr;
    c->arrivals_cap = 0;
    KMC_TRY(dalloc(&c->d_arrivals, sizeof(int32_t) * groups));
    c->arrivals_cap = groups;
    drop_graph(c);
  }
  KMC_CUDA(cudaMemcpy(c->d_items, items.data(), sizeof(Item) * items.size(),
                      cudaMemcpyHostToDevice));
  KMC_CUDA(cudaMemset(c->d_arrivals, 0, sizeof(int32_t) * c->arrivals_cap));
  c->n_items = static_cast<int>(items.size());
  c->items_shape = sh;
  c->chain_cut = plan.chain_cut;
  return KMC_OK;
}

StepArgs base_args(kmc_ctx *c) {
  StepArgs a;
  std::memset(&a, 0, sizeof(a));
  a.items = c->d_items;
  a.lys = c->d_lys;
  a.pos = c->d_pos;
  a.axis = c->d_axis;
  a.m = c->d_m;
  a.src[0] = c->d_src[0];
  a.src[1] = c->d_src[1];
  a.src_pos = c->fp32 ? nullptr : c->d_pos;
  a.beta = c->d_beta;
  a.vfrac = c->d_vfrac;
  a.e_acc = c->d_eacc;
  a.dh_acc = c->d_dh;
  a.loop_m = c->d_loop;
  a.counters = c->d_cnt;
  a.err = c->d_err;
  a.partial = c->d_partial;
  a.arrivals = c->d_arrivals;
  a.rs = c->d_rs;
  a.n_items = c->n_items;
  a.n_lys = c->n_lys;
  if (c->shape.sym > 0 && c->items_shape == c->shape) {  // symmetric form: all of its items
    a.n_items = c->n_sitems;
    a.gc = c->shape.warps * c->shape.sym;
  }
  a.sitems = c->d_sitems;
  a.supd = c->d_supd;
  a.sfwd = c->d_sfwd;
  a.srev = c->d_srev;
  a.n_upd = c->n_supd;
  a.cosk = c->d_cosk;
  a.gbar = c->d_gbar;
  a.barrier_ns = 2000000000ull;  // 2 s
  a.stall_block = -1;
  a.stall_step = -1;
  return a;
}

// The persistent period's cosine table for `steps` steps (the values the
// per-step launches of a period graph receive) and its barrier counters.
kmc_status prepare_persist(kmc_ctx *c, int steps) {
  if (!c->d_gbar) KMC_TRY(dalloc(&c->d_gbar, 2 * sizeof(uint32_t)));
  if (static_cast<size_t>(steps) > c->cosk_cap) {
    if (c->d_cosk) cudaFree(c->d_cosk);
    c->d_cosk = nullptr;
    c->cosk_cap = 0;
    KMC_TRY(dalloc(&c->d_cosk, sizeof(double) * steps));
    c->cosk_cap = static_cast<size_t>(steps);
  }
  std::vector<double> cs(static_cast<size_t>(steps));
  for (int k = 0; k < steps; ++k) cs[k] = std::cos(2.0 * kPi * k / steps);
  KMC_CUDA(cudaMemcpyAsync(c->d_cosk, cs.data(), sizeof(double) * cs.size(),
                           cudaMemcpyHostToDevice, c->stream));
  KMC_CUDA(cudaStreamSynchronize(c->stream));
  return KMC_OK;
}

// One persistent launch of `steps` steps (the barrier counters zeroed first).
cudaError_t launch_period(kmc_ctx *c, StepArgs a, const Shape &sh, int steps) {
  a.S = steps;
  a.cosk = c->d_cosk;
  a.gbar = c->d_gbar;
  cudaError_t e = cudaMemsetAsync(c->d_gbar, 0, 2 * sizeof(uint32_t), c->stream);
  if (e == cudaSuccess) e = kmc::launch_persist(a, sh.warps, sh.tile, c->n_items, c->stream);
  return e;
}

// Chains of the current items (the symmetric form has its own cut).
int n_chains_of(const kmc_ctx *c, const Shape &sh) {
  return static_cast<int>(sh.sym ? c->sym_cut_items.size() : c->chain_cut.size()) - 1;
}

// One step of every item of a (all chains, one stream), shape sh.
cudaError_t launch_one_step(const kmc_ctx *c, StepArgs a, const Shape &sh, cudaStream_t st,
                            bool pdl) {
  if (sh.sym) {
    a.sitems = c->d_sitems;
    a.supd = c->d_supd;
    a.n_items = c->n_sitems;
    a.n_upd = c->n_supd;
    a.gc = sh.warps * sh.sym;
    return kmc::launch_sym(a, sh.warps, sh.sym, c->n_sitems, st, pdl, sh.supd);
  }
  return kmc::launch_step(c->fp32, sh.warps, sh.tile, a, c->n_items, st, pdl, sh.tpl, sh.rpl,
                          sh.cl);
}

kmc_status refresh_sources(kmc_ctx *c, int par) {
  const int bs = 256;
  const unsigned nb = static_cast<unsigned>((c->N + bs - 1) / bs);
  if (c->fp32)
    sources_f32<<<nb, bs, 0, c->stream>>>(static_cast<const float4 *>(c->d_pos),
                                          static_cast<const float4 *>(c->d_m), c->d_slot,
                                          static_cast<SrcPair *>(c->d_src[par]), c->N);
  else
    sources_f64<<<nb, bs, 0, c->stream>>>(static_cast<const dbl4 *>(c->d_pos),
                                          static_cast<const dbl4 *>(c->d_m),
                                          static_cast<dbl4 *>(c->d_src[par]), c->N);
  KMC_CUDA(cudaGetLastError());
  return KMC_OK;
}

kmc_status check_device_error(kmc_ctx *c) {
  int32_t ew[2] = {0, 0};
  KMC_CUDA(cudaMemcpyAsync(ew, c->d_err, sizeof(ew), cudaMemcpyDeviceToHost, c->stream));
  KMC_CUDA(cudaStreamSynchronize(c->stream));
  const int32_t e = ew[0];
  if (e & kmc::kErrBounds)
    return fail(KMC_ESTATE, "a bounds check of the debug build failed (site %d); results are "
                "not valid", ew[1]);
  if (e & kmc::kErrTimeout)
    return fail(KMC_ETIMEOUT, "a device-side wait for a shared-memory copy timed out");
  if (e & kmc::kErrExtrema)
    return fail(KMC_ESTATE, "an energy profile had more than two minima or maxima");
  if (e & kmc::kErrNonFinite)
    return fail(KMC_ESTATE,
                "a dipolar field or barrier was not finite (two NPs at one point?); those NPs "
                "kept their moments (KMC_READ_COUNTERS counts them)");
  return KMC_OK;
}

kmc_status upload_lys(kmc_ctx *c) {
  KMC_CUDA(cudaMemcpyAsync(c->d_lys, c->h_lys.data(), sizeof(LysDev) * c->n_lys,
                           cudaMemcpyHostToDevice, c->stream));
  return KMC_OK;
}

int max_tile(int fp32, int warps) {
  // keep at least two blocks' worth of shared memory per SM
  const size_t budget = 100 * 1024;
  int t = 1024;
  while (t > 32 && kmc::step_smem_bytes(fp32, warps, t) > budget) t /= 2;
  return t;
}

bool shape_ok(const kmc_ctx *c, const Shape &s) {
  if (s.supd != 0 && (s.sym == 0 || s.supd != 1)) return false;
  if (s.persist != 0 && (s.persist != 1 || !c->fp32 || s.tpl != 1 || s.rpl != 1 || s.sym != 0 ||
                         s.cl != 0 || (s.warps != 4 && s.warps != 8)))
    return false;
  if (s.sym) {  // symmetric form: (warps, cells per warp) of its field kernel
    if (!c->fp32 || s.rpl != 1 || s.tpl != 2 * s.sym || s.tile != 32) return false;
    if (!((s.warps == 4 && (s.sym == 1 || s.sym == 2)) || (s.warps == 8 && s.sym == 1) ||
          (s.warps == 2 && s.sym == 2)))
      return false;
    return s.chunk >= 0 && s.chunk % kmc::kCell == 0;
  }
  if (s.tpl > 3) return false;
  if (s.cl != 0 && (s.cl != 2 || !c->fp32 || s.tpl != 1 || s.rpl != 1 || s.chunk <= 0))
    return false;
  if (s.rpl > 1) {  // replicas: their kernel has one warp per replica
    if (!c->fp32 || s.tpl != 1 ||
        (s.warps != s.rpl && s.warps != 2 * s.rpl && s.warps != 4 * s.rpl) ||
        !c->rep_ok[s.rpl])
      return false;
    if (s.tile < 32 || s.tile > 128 || (s.tile & (s.tile - 1))) return false;
    return s.chunk >= 0 && s.chunk % 64 == 0;
  }
  if (s.warps != 4 && s.warps != 8 && s.warps != 16) return false;
  if (s.tile < 32 || s.tile > max_tile(c->fp32, s.warps) || (s.tile & (s.tile - 1))) return false;
  if (s.chunk < 0 || (s.chunk % 64) != 0) return false;
  return true;
}

// Captures `steps` step launches of shape sh as a graph: the chains of the
// current items as parallel branches (fork on c->stream, join back onto it),
// the field at phase 2 pi k / steps in launch k. With `period` launch k is
// step k of a run (k_local = k, then the period advance), else a repeat of one
// unrecorded step.
kmc_status capture_steps(kmc_ctx *c, const StepArgs &a, const Shape &sh, int steps, bool period,
                         cudaGraphExec_t *out) {
  Phase phase("kmc_capture");
  *out = nullptr;
  const int n_chains = n_chains_of(c, sh);
  for (int q = 0; q < n_chains; ++q) {
    if (q > 0 && !c->chain_st[q])
      KMC_CUDA(cudaStreamCreateWithFlags(&c->chain_st[q], cudaStreamNonBlocking));
    if (!c->chain_ev[q])
      KMC_CUDA(cudaEventCreateWithFlags(&c->chain_ev[q], cudaEventDisableTiming));
  }
  cudaGraph_t g = nullptr;
  KMC_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t ce = cudaSuccess;
  // fork: branch 0 stays on the capturing stream, branches 1.. wait for it
  if (n_chains > 1) ce = cudaEventRecord(c->chain_ev[0], c->stream);
  for (int q = 1; q < n_chains && ce == cudaSuccess; ++q)
    ce = cudaStreamWaitEvent(c->chain_st[q], c->chain_ev[0], 0);
  const bool split = c->partial_cap >= static_cast<size_t>(c->n_items);
  for (int q = 0; q < n_chains && ce == cudaSuccess; ++q) {
    cudaStream_t st = q == 0 ? c->stream : c->chain_st[q];
    if (sh.sym) {
      StepArgs b = a;
      const int u0 = c->sym_cut_items[q], v0 = c->sym_cut_upd[q];
      b.sitems = c->d_sitems + u0;
      b.n_items = c->sym_cut_items[q + 1] - u0;
      b.supd = c->d_supd + v0;
      b.n_upd = c->sym_cut_upd[q + 1] - v0;
      b.gc = sh.warps * sh.sym;
      for (int k = 0; k < steps && ce == cudaSuccess; ++k) {
        if (period) b.k_local = k;
        b.cos_k = std::cos(2.0 * kPi * k / steps);
        ce = kmc::launch_sym(b, sh.warps, sh.sym, b.n_items, st, true, sh.supd);
      }
      continue;
    }
    const int u0 = c->chain_cut[q];
    StepArgs b = a;
    b.items = c->d_items + u0;
    b.n_items = c->chain_cut[q + 1] - u0;
    // an item's partials: (sum, error) of 3 FP32 or 6 FP64 (two floats each) components
    // per target
    if (split)
      b.partial = c->d_partial +
                  static_cast<size_t>(u0) * (c->fp32 ? 6 : 12) * kmc::kTargets * sh.tpl * sh.rpl;
    for (int k = 0; k < steps && ce == cudaSuccess; ++k) {
      if (period) b.k_local = k;
      b.cos_k = std::cos(2.0 * kPi * k / steps);
      ce = kmc::launch_step(c->fp32, sh.warps, sh.tile, b, c->chain_cut[q + 1] - u0, st, true,
                            sh.tpl, sh.rpl, sh.cl);
    }
  }
  // join, then the period advance
  for (int q = 1; q < n_chains && ce == cudaSuccess; ++q) {
    ce = cudaEventRecord(c->chain_ev[q], c->chain_st[q]);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(c->stream, c->chain_ev[q], 0);
  }
  if (ce == cudaSuccess && period) ce = kmc::launch_advance(c->d_rs, steps, c->stream);
  const cudaError_t ee = cudaStreamEndCapture(c->stream, &g);
  if (ce != cudaSuccess || ee != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return fail(KMC_ECUDA, "graph capture failed: %s",
                cudaGetErrorString(ce != cudaSuccess ? ce : ee));
  }
  const cudaError_t ie = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    *out = nullptr;
    return fail(KMC_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ie));
  }
  return KMC_OK;
}

// Times one candidate shape on the current state (restored by the caller),
// over `scale` times the usual number of steps. Returns milliseconds per step,
// or a negative value on error.
float time_shape(kmc_ctx *c, const Shape &s, int scale = 1) {
  if (set_items(c, s) != KMC_OK) return -1.f;
  StepArgs a = base_args(c);
  a.cos_k = 1.0;
  a.S = 1;
  a.n_rec = 1;
  if (s.persist) {  // a persistent launch of 32 steps, timed twice after one
    constexpr int kSteps = 32;
    if (prepare_persist(c, kSteps) != KMC_OK) return -1.f;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -1.f;
    if (cudaEventCreate(&e1) != cudaSuccess) {
      cudaEventDestroy(e0);
      return -1.f;
    }
    bool ok = launch_period(c, a, s, kSteps) == cudaSuccess;
    if (ok) ok = cudaEventRecord(e0, c->stream) == cudaSuccess;
    for (int r = 0; r < 2 && ok; ++r) ok = launch_period(c, a, s, kSteps) == cudaSuccess;
    if (ok) ok = cudaEventRecord(e1, c->stream) == cudaSuccess;
    if (ok) ok = cudaEventSynchronize(e1) == cudaSuccess;
    float ms = -1.f;
    if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) ms /= 2 * kSteps;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    return ok ? ms : -1.f;
  }
  // several chains share the SMs, so a shape is timed the way a run executes
  // it: a graph of a few steps of every chain
  const bool chained = n_chains_of(c, s) > 1;
  // per step; short steps are timed over more of them, so that the chains
  // reach their steady interleaving (a short graph favours small blocks,
  // which fill and drain the SMs faster at the graph's ends)
  double pairs = 0.0;
  for (int x : c->n) pairs += static_cast<double>(x) * x;
  const int graph_steps = pairs < 2e8 ? 32 : 2;
  cudaGraphExec_t gx = nullptr;
  if (chained && capture_steps(c, a, s, graph_steps, false, &gx) != KMC_OK) return -1.f;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) {
    if (gx) cudaGraphExecDestroy(gx);
    return -1.f;
  }
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    if (gx) cudaGraphExecDestroy(gx);
    return -1.f;
  }
  int k_one = 0;
  auto one = [&]() {
    if (gx) return cudaGraphLaunch(gx, c->stream);
    StepArgs b = a;  // the field sweeps its cycle in 8 launches
    b.cos_k = std::cos(2.0 * kPi * (k_one++ % 8) / 8);
    return launch_one_step(c, b, s, c->stream, true);
  };
  float ms = -1.f;
  bool ok = true;
  for (int r = 0; r < 2 && ok; ++r) ok = one() == cudaSuccess;
  const int reps = (gx ? 2 : 5) * scale;
  if (ok) ok = cudaEventRecord(e0, c->stream) == cudaSuccess;
  for (int r = 0; r < reps && ok; ++r) ok = one() == cudaSuccess;
  if (ok) ok = cudaEventRecord(e1, c->stream) == cudaSuccess;
  if (ok) ok = cudaEventSynchronize(e1) == cudaSuccess;
  if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) ms /= reps * (gx ? graph_steps : 1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (gx) cudaGraphExecDestroy(gx);
  return ok ? ms : -1.f;
}

kmc_status autotune(kmc_ctx *c) {
  Phase phase("kmc_tune");
  int max_n = 0;
  for (int x : c->n) max_n = std::max(max_n, x);
  const TuneKey key{c->fp32, c->N,        c->n_lys,
                    max_n,   c->tpl_mode, c->rpl_mode,
                    (c->rep_ok[2] ? 1 : 0) | (c->rep_ok[4] ? 2 : 0), c->form_mode,
                    c->cl_mode, c->supd_mode, c->persist_mode};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      c->shape = it->second;
      return set_items(c, c->shape);
    }
  }
  // the timed launches advance a scratch copy of the state: save the moments
  HostBytes saved(c->vbytes * c->N);
  KMC_CUDA(cudaMemcpyAsync(saved.data(), c->d_m, saved.size(), cudaMemcpyDeviceToHost, c->stream));
  KMC_CUDA(cudaStreamSynchronize(c->stream));
  RunState rs{c->step_global, -1, 0};
  KMC_CUDA(cudaMemcpyAsync(c->d_rs, &rs, sizeof(rs), cudaMemcpyHostToDevice, c->stream));
  std::vector<LysDev> keep = c->h_lys;
  // the run's field amplitude and rate when known (kmc_run sets them first),
  // else a typical pair
  for (auto &L : c->h_lys) {
    if (L.bmax > 0.0) continue;
    L.bmax = 0.01;
    L.lognu0t = std::log(5e-8 / 1e-10);
  }
  KMC_TRY(upload_lys(c));
  c->h_lys = keep;
  KMC_TRY(refresh_sources(c, static_cast<int>(c->step_global & 1)));
  float best = 1e30f;
  Shape bs;
  // every shape that timed, for the finalists' second look
  std::vector<std::pair<float, Shape>> timed;
  const char *log_env = std::getenv("KMC_TUNE_LOG");
  const bool log = log_env && log_env[0] && std::strcmp(log_env, "0") != 0;
  auto show = [&](const char *what, const Shape &s, float ms) {
    if (!log) return;
    std::fprintf(stderr,
                 "kmc tune %s: warps %d tile %d chunk %d tpl %d rpl %d sym %d cl %d supd %d "
                 "persist %d: %.4f ms per step\n",
                 what, s.warps, s.tile, s.chunk, s.tpl, s.rpl, s.sym, s.cl, s.supd, s.persist, ms);
  };
  auto consider = [&](const Shape &s, float ms) {
    show("shape", s, ms);
    if (!(ms > 0.f)) return;
    timed.emplace_back(ms, s);
    if (ms < best) {
      best = ms;
      bs = s;
    }
  };
  bs.warps = 4;
  bs.tile = 64;
  bs.chunk = 0;
  bs.tpl = c->tpl_mode != 0 ? c->tpl_mode : 1;
  if (c->rpl_mode > 1) {  // pinned replicas: a shape of their kernel
    bs.warps = c->rpl_mode;
    bs.tpl = 1;
    bs.rpl = c->rpl_mode;
  }
  // the ordered kernels run 1..3 targets per lane; 4 is the symmetric form's
  const bool sym_only = c->form_mode == 2 || c->tpl_mode == 4;
  if (sym_only) {
    bs.tile = 32;
    bs.sym = c->tpl_mode == 4 ? 2 : 1;
    bs.tpl = 2 * bs.sym;
  }
  // symmetric form (FP32): (warps, cells per warp), source NPs per field item
  if (c->fp32 && c->form_mode != 1 && c->rpl_mode <= 1 &&
      (c->tpl_mode == 0 || c->tpl_mode == 2 || c->tpl_mode == 4)) {
    const int wc[4][2] = {{2, 2}, {4, 1}, {4, 2}, {8, 1}};
    for (const auto &v : wc) {
      if (c->tpl_mode != 0 && 2 * v[1] != c->tpl_mode) continue;
      const int gc = v[0] * v[1];
      for (int ch : {0, 256, 512, 1024, 2048, 4096}) {
        // a field item of ch source NPs, at least one row group's worth
        if (ch > 0 && (ch >= max_n || ch < gc * kmc::kCell / 2)) continue;
        Shape s;
        s.warps = v[0];
        s.tile = 32;
        s.chunk = ch;
        s.tpl = 2 * v[1];
        s.sym = v[1];
        s.supd = c->supd_mode == 2 ? 1 : 0;
        const float ms = time_shape(c, s);
        consider(s, ms);
      }
    }
    // the symmetric shapes within 3 % of the best with the other update kernel
    // (shapes that tie with one update kernel can part with the other)
    if (bs.sym && c->supd_mode == 0) {
      std::vector<std::pair<float, Shape>> near;
      for (const auto &t : timed)
        if (t.second.sym && t.first <= 1.03f * best) near.push_back(t);
      std::sort(near.begin(), near.end(),
                [](const std::pair<float, Shape> &x, const std::pair<float, Shape> &y) {
                  return x.first < y.first;
                });
      if (near.size() > 4) near.resize(4);
      for (auto &t : near) {
        Shape s = t.second;
        s.supd = 1;
        consider(s, time_shape(c, s));
      }
    }
  }
  const int warps_c[] = {4, 8};
  const int tiles_f32[] = {64, 128, 256, 512};
  const int tiles_f64[] = {32, 64, 128, 128};  // (the FP64 list has three distinct tiles)
  const int chunks[] = {0, 256, 512, 1024, 2048, 4096, 8192};
  // replicas per lane (FP32, sets of identical lysosomes): one or four warps
  // per replica, one target per lane, tiles of 32..128 records per replica
  for (int rpl = 2; rpl <= 4 && c->fp32 && c->tpl_mode <= 1 && !sym_only; rpl += 2) {
    if (!c->rep_ok[rpl] || (c->rpl_mode != 0 && c->rpl_mode != rpl)) continue;
    for (int wpr : {1, 2, 4}) {
      for (int t : {32, 64, 128}) {
        if (2 * t > 2 * std::max(max_n, 64) && t > 32) continue;
        for (int ch : chunks) {
          if (ch > 0 && (ch >= max_n || ch < 2 * t)) continue;
          Shape s;
          s.warps = rpl * wpr;
          s.tile = t;
          s.chunk = ch;
          s.tpl = 1;
          s.rpl = rpl;
          const float ms = time_shape(c, s);
          consider(s, ms);
        }
      }
    }
  }
  for (int w : warps_c) {
    if (c->rpl_mode > 1 || sym_only) break;  // pinned replicas or form: only their shapes
    for (int q = 0; q < (c->fp32 ? 4 : 3); ++q) {
      const int t = c->fp32 ? tiles_f32[q] : tiles_f64[q];
      if (t > max_tile(c->fp32, w)) continue;
      if ((c->fp32 ? 2 : 1) * t > 2 * std::max(max_n, 64) && q > 0) continue;
      for (int ch : chunks) {
        if (ch > 0 && ch >= max_n) continue;
        if (ch > 0 && ch < (c->fp32 ? 2 : 1) * t) continue;
        for (int tpl = 1; tpl <= 3; ++tpl) {
          if (c->tpl_mode != 0 && tpl != c->tpl_mode) continue;
          if (tpl > 1 && !c->fp32) continue;
          Shape s;
          s.warps = w;
          s.tile = t;
          s.chunk = ch;
          s.tpl = tpl;
          if (c->cl_mode != 2 && c->persist_mode != 2) {
            const float ms = time_shape(c, s);
            consider(s, ms);
          }
          // the same shape with each group's two parts as a two-CTA cluster
          // (time_shape fails unless every group has exactly two parts)
          if (c->fp32 && tpl == 1 && ch > 0 && c->cl_mode != 1 && c->persist_mode != 2) {
            Shape sc = s;
            sc.cl = 2;
            const float mc = time_shape(c, sc);
            consider(sc, mc);
          }
          // the same shape as one persistent launch per period (time_shape
          // fails unless every item's block can be resident at once)
          if (c->fp32 && tpl == 1 && c->persist_mode != 1 && c->cl_mode != 2) {
            Shape sp = s;
            sp.persist = 1;
            const float mp = time_shape(c, sp);
            consider(sp, mp);
          }
        }
      }
    }
  }
  // Shapes within a few per cent of the best are timed twice more, in turn,
  // each time over three times the steps, and the one with the lowest of its
  // times wins: one timing of a few milliseconds moves by about a per cent
  // from launch to launch.
  {
    std::vector<std::pair<float, Shape>> fin;
    for (const auto &t : timed)
      if (t.first <= 1.03f * best) fin.push_back(t);
    std::sort(fin.begin(), fin.end(),
              [](const std::pair<float, Shape> &x, const std::pair<float, Shape> &y) {
                return x.first < y.first;
              });
    if (fin.size() > 6) fin.resize(6);
    if (fin.size() > 1) {
      for (int r = 0; r < 2; ++r)
        for (auto &f : fin) {
          const float ms = time_shape(c, f.second, 3);
          show("finalist", f.second, ms);
          if (ms > 0.f && ms < f.first) f.first = ms;
        }
      for (const auto &f : fin)
        if (f.first < best) {
          best = f.first;
          bs = f.second;
        }
    }
  }
  KMC_CUDA(cudaGetLastError());
  KMC_CUDA(cudaMemcpyAsync(c->d_m, saved.data(), saved.size(), cudaMemcpyHostToDevice, c->stream));
  KMC_CUDA(cudaMemsetAsync(c->d_err, 0, 2 * sizeof(int32_t), c->stream));
  KMC_CUDA(cudaStreamSynchronize(c->stream));
  c->shape = bs;
  show("chosen", bs, best);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = bs;
  }
  return set_items(c, bs);
}

kmc_status ensure_shape(kmc_ctx *c) {
  if (c->shape.warps == 0) return autotune(c);
  return set_items(c, c->shape);
}

void free_ctx(kmc_ctx *c) {
  if (!c) return;
  drop_graph(c);
  void *ptrs[] = {c->d_lys,   c->d_pos,    c->d_axis,    c->d_m,        c->d_src[0],
                  c->d_src[1], c->d_slot,  c->d_beta,    c->d_vfrac,    c->d_eacc,
                  c->d_dh,    c->d_pos64,  c->d_phi,     c->d_nodes,    c->d_possi, c->d_phif,
                  c->d_loop,  c->d_cnt,    c->d_err,     c->d_rs,       c->d_items,
                  c->d_partial, c->d_arrivals, c->d_dbg, c->d_dbg_flags, c->d_sitems,
                  c->d_supd,  c->d_sfwd,   c->d_srev,    c->d_cosk,     c->d_gbar};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (int q = 0; q < kMaxChains; ++q) {
    if (c->chain_st[q]) cudaStreamDestroy(c->chain_st[q]);
    if (c->chain_ev[q]) cudaEventDestroy(c->chain_ev[q]);
  }
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  delete c;
}

kmc_status create_device_state(kmc_ctx *c, const HostBytes &h_pos,
                               const HostBytes &h_axis,
                               const HostBytes &h_m,
                               const HostBytes &h_src,
                               const std::vector<int> &h_slot, const std::vector<double> &h_beta,
                               const std::vector<double> &h_vfrac,
                               const std::vector<dbl4> &h_pos64) {
  const long long N = c->N;
  KMC_CUDA(cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking));
  c->stream = c->own_stream;
  const size_t vb = c->vbytes * N;
  KMC_TRY(dalloc(&c->d_lys, sizeof(LysDev) * c->n_lys));
  KMC_TRY(dalloc(&c->d_pos, vb));
  KMC_TRY(dalloc(&c->d_axis, vb));
  KMC_TRY(dalloc(&c->d_m, vb));
  KMC_TRY(dalloc(&c->d_src[0], h_src.size()));
  KMC_TRY(dalloc(&c->d_src[1], h_src.size()));
  if (c->fp32) KMC_TRY(dalloc(&c->d_slot, sizeof(int) * N));
  KMC_TRY(dalloc(&c->d_beta, sizeof(double) * N));
  KMC_TRY(dalloc(&c->d_vfrac, sizeof(double) * N));
  KMC_TRY(dalloc(&c->d_eacc, sizeof(double) * N));
  KMC_TRY(dalloc(&c->d_dh, sizeof(double) * N));
  if (c->fp32) KMC_TRY(dalloc(&c->d_pos64, sizeof(dbl4) * N));
  KMC_TRY(dalloc(&c->d_cnt, sizeof(unsigned long long) * kmc::kCounters * c->n_lys));
  KMC_TRY(dalloc(&c->d_err, 2 * sizeof(int32_t)));  // error bits, failed check site
  KMC_TRY(dalloc(&c->d_rs, sizeof(RunState)));
  KMC_CUDA(cudaMemcpy(c->d_pos, h_pos.data(), vb, cudaMemcpyHostToDevice));
  KMC_CUDA(cudaMemcpy(c->d_axis, h_axis.data(), vb, cudaMemcpyHostToDevice));
  KMC_CUDA(cudaMemcpy(c->d_m, h_m.data(), vb, cudaMemcpyHostToDevice));
  KMC_CUDA(cudaMemcpy(c->d_src[0], h_src.data(), h_src.size(), cudaMemcpyHostToDevice));
  KMC_CUDA(cudaMemcpy(c->d_src[1], h_src.data(), h_src.size(), cudaMemcpyHostToDevice));
  if (c->fp32)
    KMC_CUDA(cudaMemcpy(c->d_slot, h_slot.data(), sizeof(int) * N, cudaMemcpyHostToDevice));
  KMC_CUDA(cudaMemcpy(c->d_beta, h_beta.data(), sizeof(double) * N, cudaMemcpyHostToDevice));
  KMC_CUDA(cudaMemcpy(c->d_vfrac, h_vfrac.data(), sizeof(double) * N, cudaMemcpyHostToDevice));
  KMC_CUDA(cudaMemset(c->d_eacc, 0, sizeof(double) * N));
  KMC_CUDA(cudaMemset(c->d_dh, 0, sizeof(double) * N));
  if (c->fp32)
    KMC_CUDA(cudaMemcpy(c->d_pos64, h_pos64.data(), sizeof(dbl4) * N, cudaMemcpyHostToDevice));
  KMC_CUDA(cudaMemset(c->d_cnt, 0, sizeof(unsigned long long) * kmc::kCounters * c->n_lys));
  KMC_CUDA(cudaMemset(c->d_err, 0, 2 * sizeof(int32_t)));
  KMC_CUDA(cudaMemcpy(c->d_lys, c->h_lys.data(), sizeof(LysDev) * c->n_lys,
                      cudaMemcpyHostToDevice));
  return KMC_OK;
}

// Lysosomes a and b are replicas: the same NPs (positions, axes, volumes,
// compared bit for bit), material, temperature, attempt time, density and
// frame origin; only their random streams (the lysosome index) differ.
bool same_lysosome(const kmc_lysosome &a, const kmc_lysosome &b) {
  if (a.n != b.n || a.Ms != b.Ms || a.Keff != b.Keff || a.T != b.T || a.tau0 != b.tau0)
    return false;
  if ((a.rho > 0 ? a.rho : 5200.0) != (b.rho > 0 ? b.rho : 5200.0)) return false;
  if ((a.center == nullptr) != (b.center == nullptr)) return false;
  if (a.center && std::memcmp(a.center, b.center, 3 * sizeof(double)) != 0) return false;
  const size_t n = static_cast<size_t>(a.n);
  return std::memcmp(a.pos, b.pos, 3 * n * sizeof(double)) == 0 &&
         std::memcmp(a.axis, b.axis, 3 * n * sizeof(double)) == 0 &&
         std::memcmp(a.vol, b.vol, n * sizeof(double)) == 0;
}

// Checks the lysosome descriptions of kmc_create and kmc_mean_run; *N = NPs.
kmc_status validate_lysosomes(const kmc_lysosome *lys, int32_t n_lys, long long *N_out) {
  long long N = 0;
  for (int l = 0; l < n_lys; ++l) {
    const kmc_lysosome &L = lys[l];
    if (L.n < 1) return fail(KMC_EINVAL, "lysosome %d: n = %d", l, L.n);
    if (!L.pos || !L.axis || !L.vol) return fail(KMC_EINVAL, "lysosome %d: NULL array", l);
    if (!(L.Ms > 0) || !is_finite(L.Ms)) return fail(KMC_EINVAL, "lysosome %d: Ms must be > 0", l);
    if (!(L.Keff >= 0) || !is_finite(L.Keff)) return fail(KMC_EINVAL, "lysosome %d: Keff < 0", l);
    if (!(L.T >= 0) || !is_finite(L.T)) return fail(KMC_EINVAL, "lysosome %d: T < 0", l);
    if (!(L.tau0 > 0) || !is_finite(L.tau0)) return fail(KMC_EINVAL, "lysosome %d: tau0 <= 0", l);
    for (int i = 0; i < L.n; ++i) {
      if (!(L.vol[i] > 0) || !is_finite(L.vol[i]))
        return fail(KMC_EINVAL, "lysosome %d NP %d: volume must be > 0", l, i);
      double a2 = 0;
      for (int q = 0; q < 3; ++q) {
        if (!is_finite(L.pos[3 * i + q]) || !is_finite(L.axis[3 * i + q]))
          return fail(KMC_EINVAL, "lysosome %d NP %d: non-finite input", l, i);
        a2 += L.axis[3 * i + q] * L.axis[3 * i + q];
      }
      if (!(a2 > 0)) return fail(KMC_EINVAL, "lysosome %d NP %d: zero easy axis", l, i);
    }
    N += L.n;
    if (N > (1ll << 30)) return fail(KMC_EINVAL, "too many NPs");
  }
  *N_out = N;
  return KMC_OK;
}

}  // namespace

// ===========================================================================
extern "C" {

const char *kmc_last_error(void) { return g_last_error.c_str(); }

kmc_status kmc_create(const kmc_lysosome *lys, int32_t n_lys, kmc_precision prec,
                      kmc_ctx **out) {
  Phase phase("kmc_create");
  g_last_error.clear();
  if (!out) return fail(KMC_EINVAL, "out is NULL");
  *out = nullptr;
  if (!lys || n_lys < 1) return fail(KMC_EINVAL, "need at least one lysosome");
  if (prec != KMC_FP64_PLAIN && prec != KMC_FP32_MIXED)
    return fail(KMC_EINVAL, "unknown precision %d", static_cast<int>(prec));
  long long N = 0;
  KMC_TRY(validate_lysosomes(lys, n_lys, &N));
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return fail(KMC_ECUDA, "no CUDA device available");
  }
  KMC_TRY(ensure_device_init());

  kmc_ctx *c = new (std::nothrow) kmc_ctx();
  if (!c) return fail(KMC_ENOMEM, "host allocation failed");
  c->fp32 = prec == KMC_FP32_MIXED;
  c->n_lys = n_lys;
  c->N = N;
  // sets of k identical consecutive lysosomes (replicas per lane, FP32)
  for (int k = 2; k <= 4; k += 2) {
    bool ok = c->fp32 && n_lys % k == 0;
    for (int l = 0; ok && l < n_lys; ++l)
      if (l % k != 0) ok = same_lysosome(lys[l], lys[l - 1]);
    c->rep_ok[k] = ok;
  }
  c->vbytes = c->fp32 ? sizeof(float4) : sizeof(dbl4);
  // FP32: every lysosome's records start on a cell boundary (kmc::kCellRec
  // records) and its last cell is padded, for the symmetric form
  auto lys_records = [&](int n) -> long long {
    return c->fp32 ? static_cast<long long>((n + kmc::kCell - 1) / kmc::kCell) * kmc::kCellRec : n;
  };
  long long nrec = 0;
  for (int l = 0; l < n_lys; ++l) nrec += lys_records(lys[l].n);
  c->n_records = nrec;
  HostBytes h_pos(c->vbytes * N), h_axis(c->vbytes * N), h_m(c->vbytes * N);
  HostBytes h_src((c->fp32 ? sizeof(SrcPair) : sizeof(dbl4)) * nrec);
  std::vector<int> h_slot(c->fp32 ? N : 0);
  std::vector<double> h_beta(N), h_vfrac(N);
  std::vector<dbl4> h_pos64(c->fp32 ? N : 0);
  c->vol.resize(N);
  c->pos_si.resize(3 * N);
  c->h_lys.resize(n_lys);
  SrcPair *src32 = reinterpret_cast<SrcPair *>(h_src.data());
  dbl4 *src64 = reinterpret_cast<dbl4 *>(h_src.data());
  long long o = 0, r = 0;
  for (int l = 0; l < n_lys; ++l) {
    const kmc_lysosome &L = lys[l];
    c->off.push_back(static_cast<int>(o));
    c->roff.push_back(static_cast<int>(r));
    c->n.push_back(L.n);
    c->Ms.push_back(L.Ms);
    c->Keff.push_back(L.Keff);
    c->T.push_back(L.T);
    c->tau0.push_back(L.tau0);
    c->rho.push_back(L.rho > 0 ? L.rho : 5200.0);
    double vs = 0, cx = 0, cy = 0, cz = 0;
    for (int i = 0; i < L.n; ++i) {
      vs += L.vol[i];
      cx += L.pos[3 * i];
      cy += L.pos[3 * i + 1];
      cz += L.pos[3 * i + 2];
    }
    if (L.center) {
      cx = L.center[0];
      cy = L.center[1];
      cz = L.center[2];
    } else {
      cx /= L.n;
      cy /= L.n;
      cz /= L.n;
    }
    c->vsum.push_back(vs);
    const double len = std::cbrt(6.0 * (vs / L.n) / kPi);  // diameter of the mean volume
    c->len.push_back(len);
    c->ctr.push_back(cx);
    c->ctr.push_back(cy);
    c->ctr.push_back(cz);
    const double w_scale = 1.0 / (4.0 * kPi * len * len * len);
    LysDev &D = c->h_lys[l];
    D.off = static_cast<int>(o);
    D.n = L.n;
    D.roff = static_cast<int>(r);
    D.t_zero = L.T == 0.0;
    D.k = L.Keff / (kMu0 * L.Ms * L.Ms);
    D.bmax = 0.0;
    D.lognu0t = 0.0;
    if (c->fp32) {  // padding NPs up to the end of the last cell: far away, no moment
      for (long long j = L.n; j < 2 * lys_records(L.n); ++j) {
        SrcPair &pad = src32[r + j / 2];
        const int h = static_cast<int>(j & 1);
        pad.x[h] = pad.y[h] = pad.z[h] = kmc::kPadCoord;
        kmc::set_source_moment(pad, h, 0.0f, 0.0f, 0.0f, 0.0f);
        pad.pad[h] = 0.0f;
      }
    }
    for (int i = 0; i < L.n; ++i, ++o) {
      const double *p = &L.pos[3 * i];
      const double *a = &L.axis[3 * i];
      const double an = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
      const double ax = a[0] / an, ay = a[1] / an, az = a[2] / an;
      const double sgn = az >= 0 ? 1.0 : -1.0;  // initial m along the axis, m_z >= 0
      const double x = (p[0] - cx) / len, y = (p[1] - cy) / len, z = (p[2] - cz) / len;
      const double w = L.vol[i] * w_scale;
      c->vol[o] = L.vol[i];
      for (int q = 0; q < 3; ++q) c->pos_si[3 * o + q] = p[q];
      if (c->fp32) h_pos64[o] = make4<dbl4>(x, y, z, w);
      h_beta[o] = L.T > 0 ? kMu0 * L.Ms * L.Ms * L.vol[i] / (kKB * L.T) : 0.0;
      h_vfrac[o] = L.vol[i] / vs;
      if (c->fp32) {
        const float4 pf = make4<float4>(x, y, z, w);
        reinterpret_cast<float4 *>(h_pos.data())[o] = pf;
        const float4 af = make4<float4>(ax, ay, az, 0.0);
        reinterpret_cast<float4 *>(h_axis.data())[o] = af;
        const float4 mf = make4<float4>(sgn * af.x, sgn * af.y, sgn * af.z, 0.0);
        reinterpret_cast<float4 *>(h_m.data())[o] = mf;
        SrcPair &rec = src32[r + i / 2];
        const int h = i & 1;
        rec.x[h] = pf.x;
        rec.y[h] = pf.y;
        rec.z[h] = pf.z;
        kmc::set_source_moment(rec, h, pf.w, mf.x, mf.y, mf.z);
        rec.pad[h] = 0.0f;
        h_slot[o] = static_cast<int>(2 * (r + i / 2) + h);
      } else {
        reinterpret_cast<dbl4 *>(h_pos.data())[o] = make4<dbl4>(x, y, z, w);
        reinterpret_cast<dbl4 *>(h_axis.data())[o] = make4<dbl4>(ax, ay, az, 0.0);
        reinterpret_cast<dbl4 *>(h_m.data())[o] = make4<dbl4>(sgn * ax, sgn * ay, sgn * az, 0.0);
        src64[r + i] = make4<dbl4>(w * sgn * ax, w * sgn * ay, w * sgn * az, 0.0);
      }
    }
    r += lys_records(L.n);
  }
  const kmc_status st =
      create_device_state(c, h_pos, h_axis, h_m, h_src, h_slot, h_beta, h_vfrac, h_pos64);
  if (st != KMC_OK) {
    free_ctx(c);
    return st;
  }
  *out = c;
  return KMC_OK;
}

kmc_status kmc_set_stream(kmc_ctx *c, void *cuda_stream) {
  if (!c) return fail(KMC_EINVAL, "ctx is NULL");
  KMC_CUDA(cudaStreamSynchronize(c->stream));
  c->stream = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : c->own_stream;
  return KMC_OK;
}

kmc_status kmc_plan_sym(const int32_t *n, int32_t n_lys, int32_t gc, int32_t src_cells,
                        int32_t *items_out, int64_t cap, int64_t *n_items, int32_t *upd_out,
                        int64_t cap_upd, int64_t *n_upd, int64_t *n_rev,
                        int32_t *chain_cut_items, int32_t *chain_cut_upd, int32_t *n_chains) {
  if (!n || n_lys < 1 || !n_items || !n_upd || !n_rev || !chain_cut_items || !chain_cut_upd ||
      !n_chains || cap < 0 || cap_upd < 0 || (cap > 0 && !items_out) || (cap_upd > 0 && !upd_out))
    return fail(KMC_EINVAL, "plan: need n[n_lys >= 1], outputs and capacities >= 0");
  if ((gc != 4 && gc != 8) || src_cells < 0)
    return fail(KMC_EINVAL, "plan: gc 4 or 8, src_cells >= 0");
  std::vector<int> np(n, n + n_lys);
  for (int v : np)
    if (v < 1) return fail(KMC_EINVAL, "plan: every lysosome needs an NP");
  const SymPlan p = plan_sym(np, gc, src_cells);
  *n_items = static_cast<int64_t>(p.items.size());
  *n_upd = static_cast<int64_t>(p.upd.size());
  *n_rev = p.n_rev;
  *n_chains = static_cast<int32_t>(p.cut_items.size()) - 1;
  for (size_t q = 0; q < p.cut_items.size(); ++q) {
    chain_cut_items[q] = p.cut_items[q];
    chain_cut_upd[q] = p.cut_upd[q];
  }
  if (*n_items > cap || *n_upd > cap_upd)
    return fail(KMC_ECAPACITY, "plan: %lld field and %lld update items", (long long)*n_items,
                (long long)*n_upd);
  for (size_t u = 0; u < p.items.size(); ++u) {
    const kmc::SymItem &it = p.items[u];
    const int32_t row[KMC_SYM_FIELDS] = {it.l, it.g, it.h0, it.h1, it.fwd, it.rbase, 0, 0};
    std::memcpy(items_out + KMC_SYM_FIELDS * u, row, sizeof(row));
  }
  for (size_t u = 0; u < p.upd.size(); ++u) {
    const kmc::SymUpd &d = p.upd[u];
    const int32_t row[KMC_SYM_FIELDS] = {d.l, d.t0, d.nt, d.fwd0, d.nfwd, d.rev0, d.nrev, d.gt0};
    std::memcpy(upd_out + KMC_SYM_FIELDS * u, row, sizeof(row));
  }
  return KMC_OK;
}

kmc_status kmc_plan_items(const int32_t *n, int32_t n_lys, kmc_precision prec, int32_t tpl,
                          int32_t chunk, int32_t blocks_per_sm, int32_t n_sms, int32_t *items_out,
                          int64_t cap, int64_t *n_items, int32_t *chain_cut, int32_t *n_chains) {
  if (!n || n_lys < 1 || !n_items || !chain_cut || !n_chains || cap < 0 || (cap > 0 && !items_out))
    return fail(KMC_EINVAL, "plan: need n[n_lys >= 1], outputs and cap >= 0");
  if (prec != KMC_FP32_MIXED && prec != KMC_FP64_PLAIN) return fail(KMC_EINVAL, "bad precision");
  const bool fp32 = prec == KMC_FP32_MIXED;
  if (tpl != 1 && !((tpl == 2 || tpl == 3) && fp32))
    return fail(KMC_EINVAL, "targets per lane: 1, or 2 or 3 with KMC_FP32_MIXED");
  if (chunk < 0 || chunk % 64 != 0 || blocks_per_sm < 1 || n_sms < 0)
    return fail(KMC_EINVAL, "plan: chunk a multiple of 64, blocks_per_sm >= 1, n_sms >= 0");
  std::vector<int> np(n, n + n_lys);
  for (int v : np)
    if (v < 1) return fail(KMC_EINVAL, "plan: every lysosome needs an NP");
  const Plan p = plan_items(np, fp32, chunk, blocks_per_sm, n_sms, tpl);
  *n_items = static_cast<int64_t>(p.items.size());
  *n_chains = static_cast<int32_t>(p.chain_cut.size()) - 1;
  for (size_t q = 0; q < p.chain_cut.size(); ++q) chain_cut[q] = p.chain_cut[q];
  if (static_cast<int64_t>(p.items.size()) > cap)
    return fail(KMC_ECAPACITY, "plan: %lld items, capacity %lld",
                static_cast<long long>(p.items.size()), static_cast<long long>(cap));
  for (size_t u = 0; u < p.items.size(); ++u) {
    const Item &it = p.items[u];
    const int32_t f[KMC_ITEM_FIELDS] = {it.l, it.t0, it.nt, it.gid, it.j0, it.j1, it.split, it.nsplit};
    for (int k = 0; k < KMC_ITEM_FIELDS; ++k) items_out[KMC_ITEM_FIELDS * u + k] = f[k];
  }
  return KMC_OK;
}

kmc_status kmc_targets_per_lane(kmc_ctx *c, int32_t tpl, int32_t *tpl_out) {
  if (!c) return fail(KMC_EINVAL, "ctx is NULL");
  if (tpl != -1) {
    if (tpl < 0 || tpl > 4)
      return fail(KMC_EINVAL, "targets per lane: 0 (autotuned), 1, 2, 3 or 4");
    if (tpl > 1 && !c->fp32)
      return fail(KMC_EINVAL, "two or more targets per lane run on FP32 contexts");
    if (tpl > 1 && c->rpl_mode > 1)
      return fail(KMC_EINVAL, "replicas per lane run one target per lane");
    if (c->form_mode == 2 && (tpl == 1 || tpl == 3))
      return fail(KMC_EINVAL, "the symmetric form runs 2 or 4 targets per lane");
    if (c->form_mode == 1 && tpl == 4)
      return fail(KMC_EINVAL, "the ordered kernels run 1, 2 or 3 targets per lane");
    c->tpl_mode = tpl;
    // a pinned choice applies to the shape in use; 0 leaves it to the autotuner
    if (tpl != 0 && c->shape.warps != 0 && c->shape.rpl == 1) {
      Shape s = c->shape;
      s.tpl = tpl;
      if (s.sym) s.sym = tpl / 2;
      if (s.sym == 0 && tpl == 4) s = Shape();
      c->shape = shape_ok(c, s) ? s : Shape();
    }
  }
  if (tpl_out) *tpl_out = c->tpl_mode != 0 ? c->tpl_mode : (c->shape.warps ? c->shape.tpl : 0);
  return KMC_OK;
}

kmc_status kmc_replicas_per_lane(kmc_ctx *c, int32_t rpl, int32_t *rpl_out) {
  if (!c) return fail(KMC_EINVAL, "ctx is NULL");
  if (rpl != -1) {
    if (rpl != 0 && rpl != 1 && rpl != 2 && rpl != 4)
      return fail(KMC_EINVAL, "replicas per lane: 0 (autotuned), 1 (off), 2 or 4");
    if (rpl > 1 && !c->fp32) return fail(KMC_EINVAL, "replicas per lane run on FP32 contexts");
    if (rpl > 1 && !c->rep_ok[rpl])
      return fail(KMC_EINVAL, "the lysosomes do not form sets of %d identical consecutive ones",
                  rpl);
    if (rpl > 1 && c->tpl_mode > 1)
      return fail(KMC_EINVAL, "replicas per lane run one target per lane");
    c->rpl_mode = rpl;
    // a change drops the shape in use: the next run or step tunes, or takes kmc_tuning's
    if (c->shape.warps != 0 && c->shape.rpl != (rpl > 1 ? rpl : 1) && rpl != 0)
      c->shape = Shape();
  }
  if (rpl_out) *rpl_out = c->rpl_mode != 0 ? c->rpl_mode : (c->shape.warps ? c->shape.rpl : 0);
  return KMC_OK;
}

kmc_status kmc_pair_form(kmc_ctx *c, int32_t form, int32_t *form_out) {
  if (!c) return fail(KMC_EINVAL, "ctx is NULL");
  if (form != -1) {
    if (form < 0 || form > 2)
      return fail(KMC_EINVAL, "pair form: 0 (autotuned), 1 (ordered) or 2 (symmetric)");
    if (form == 2 && !c->fp32) return fail(KMC_EINVAL, "the symmetric form runs on FP32 contexts");
    if (form == 2 && c->rpl_mode > 1)
      return fail(KMC_EINVAL, "the symmetric form does not run replicas per lane");
    if (form == 2 && (c->tpl_mode == 1 || c->tpl_mode == 3))
      return fail(KMC_EINVAL, "the symmetric form runs 2 or 4 targets per lane");
    if (form == 1 && c->tpl_mode == 4)
      return fail(KMC_EINVAL, "the ordered kernels run 1, 2 or 3 targets per lane");
    c->form_mode = form;
    // a change drops the shape in use: the next run or step tunes, or takes kmc_tuning's
    if (c->shape.warps != 0 && form != 0 && (c->shape.sym != 0) != (form == 2)) c->shape = Shape();
  }
  if (form_out)
    *form_out = c->form_mode != 0 ? c->form_mode
                                  : (c->shape.warps ? (c->shape.sym ? 2 : 1) : 0);
  return KMC_OK;
}

kmc_status kmc_persistent(kmc_ctx *c, int32_t mode, int32_t *mode_out) {
  if (!c) return fail(KMC_EINVAL, "ctx is NULL");
  if (mode != -1) {
    if (mode < 0 || mode > 2) return fail(KMC_EINVAL, "persistent period: 0 (autotuned), 1 (off), 2 (on)");
    if (mode == 2 && !c->fp32) return fail(KMC_EINVAL, "the persistent period runs on FP32 contexts");
    c->persist_mode = mode;
    if (mode != 0 && c->shape.warps != 0) {
      Shape s = c->shape;
      s.persist = mode == 2 ? 1 : 0;
      c->shape = shape_ok(c, s) ? s : Shape();
    }
  }
  if (mode_out)
    *mode_out = c->persist_mode != 0 ? c->persist_mode
                                     : (c->shape.warps ? (c->shape.persist ? 2 : 1) : 0);
  return KMC_OK;
}

kmc_status kmc_sym_update(kmc_ctx *c, int32_t mode, int32_t *mode_out) {
  if (!c) return fail(KMC_EINVAL, "ctx is NULL");
  if (mode != -1) {
    if (mode < 0 || mode > 2)
      return fail(KMC_EINVAL, "symmetric update: 0 (autotuned), 1 (warp per item), 2 (block)");
    c->supd_mode = mode;
    if (mode != 0 && c->shape.warps != 0 && c->shape.sym != 0) c->shape.supd = mode == 2 ? 1 : 0;
  }
  if (mode_out)
    *mode_out = c->supd_mode != 0 ? c->supd_mode
                                  : (c->shape.warps && c->shape.sym ? 1 + c->shape.supd : 0);
  return KMC_OK;
}

kmc_status kmc_cluster_split(kmc_ctx *c, int32_t mode, int32_t *mode_out) {
  if (!c) return fail(KMC_EINVAL, "ctx is NULL");
  if (mode != -1) {
    if (mode < 0 || mode > 2) return fail(KMC_EINVAL, "cluster split: 0 (autotuned), 1 (off), 2 (on)");
    if (mode == 2 && !c->fp32) return fail(KMC_EINVAL, "the cluster split runs on FP32 contexts");
    c->cl_mode = mode;
    // the shape in use follows a pinned choice
    if (mode != 0 && c->shape.warps != 0 && c->shape.sym == 0 && c->shape.rpl == 1 &&
        c->shape.tpl == 1) {
      Shape s = c->shape;
      s.cl = mode == 2 ? 2 : 0;
      c->shape = shape_ok(c, s) ? s : Shape();
    }
  }
  if (mode_out)
    *mode_out = c->cl_mode != 0 ? c->cl_mode : (c->shape.warps ? (c->shape.cl ? 2 : 1) : 0);
  return KMC_OK;
}

kmc_status kmc_tuning(kmc_ctx *c, int32_t warps, int32_t tile, int32_t chunk,
                      int32_t *warps_out, int32_t *tile_out, int32_t *chunk_out) {
  if (!c) return fail(KMC_EINVAL, "ctx is NULL");
  if (warps == -1 && tile == -1 && chunk == -1) {
    // read only
  } else if (warps == 0) {
    c->shape = Shape();
  } else {
    Shape s;
    s.warps = warps;
    s.tile = tile;
    s.chunk = chunk;
    s.tpl = c->tpl_mode != 0 ? c->tpl_mode : 1;
    s.rpl = c->rpl_mode > 1 ? c->rpl_mode : 1;
    s.cl = (c->cl_mode == 2 && s.tpl == 1 && s.rpl == 1) ? 2 : 0;
    s.persist = (c->persist_mode == 2 && s.tpl == 1 && s.rpl == 1 && s.cl == 0) ? 1 : 0;
    if (c->form_mode == 2 || c->tpl_mode == 4) {  // symmetric form; the tile does not apply
      s.cl = 0;
      s.supd = c->supd_mode == 2 ? 1 : 0;
      s.sym = c->tpl_mode == 4 ? 2 : 1;
      s.tpl = 2 * s.sym;
      s.tile = 32;
      if (!shape_ok(c, s))
        return fail(KMC_EINVAL, "bad symmetric shape: warps 4, 8 with 2 targets per lane or 2 "
                    "with 4, chunk a multiple of 64");
    } else if (!shape_ok(c, s))
      return fail(KMC_EINVAL,
                  s.rpl > 1 ? "bad shape: with %d replicas per lane, warps = %d or four times that, "
                              "tile a power of two in [32, 128], chunk a multiple of 64"
                            : "bad shape: warps in {4, 8, 16}, tile a power of two in [32, %d], "
                              "chunk a multiple of 64",
                  s.rpl > 1 ? s.rpl : max_tile(c->fp32, warps == 4 || warps == 8 || warps == 16 ? warps : 4),
                  s.rpl);
    c->shape = s;
  }
  if (warps_out) *warps_out = c->shape.warps;
  if (tile_out) *tile_out = c->shape.tile;
  if (chunk_out) *chunk_out = c->shape.chunk;
  return KMC_OK;
}

kmc_status kmc_run(kmc_ctx *c, const double *mu0Hmax, int32_t n_amp, double f, int32_t S,
                   int32_t periods, int32_t discard, uint64_t seed) {
  Phase phase("kmc_run");
  if (!c) return fail(KMC_EINVAL, "ctx is NULL");
  if (!mu0Hmax || (n_amp != 1 && n_amp != c->n_lys))
    return fail(KMC_EINVAL, "need 1 or n_lys = %d amplitudes", c->n_lys);
  for (int q = 0; q < n_amp; ++q)
    if (!is_finite(mu0Hmax[q])) return fail(KMC_EINVAL, "non-finite field amplitude");
  if (!(f > 0) || !is_finite(f)) return fail(KMC_EINVAL, "f must be > 0");
  if (S < 1) return fail(KMC_EINVAL, "steps_per_period must be >= 1");
  if (periods < 0 || discard < 0 || discard > periods)
    return fail(KMC_EINVAL, "need 0 <= discard_periods <= periods");
  const long long n_rec = static_cast<long long>(S) * (periods - discard);
  if (n_rec > (1ll << 28)) return fail(KMC_EINVAL, "too many recorded steps");
  const double t_step = 1.0 / (f * S);
  c->Hmax.assign(c->n_lys, 0.0);
  for (int l = 0; l < c->n_lys; ++l) {
    c->Hmax[l] = mu0Hmax[n_amp == 1 ? 0 : l];
    c->h_lys[l].bmax = c->Hmax[l] / (kMu0 * c->Ms[l]);
    c->h_lys[l].lognu0t = std::log(t_step / c->tau0[l]);
  }
  KMC_TRY(ensure_shape(c));  // the tuner times the shapes at this amplitude and rate
  KMC_TRY(upload_lys(c));
  const size_t need = static_cast<size_t>(c->n_lys) * static_cast<size_t>(std::max(n_rec, 1ll));
  if (need > c->loop_cap) {
    KMC_CUDA(cudaStreamSynchronize(c->stream));
    if (c->d_loop) cudaFree(c->d_loop);
    c->d_loop = nullptr;
    c->loop_cap = 0;
    KMC_TRY(dalloc(&c->d_loop, sizeof(long long) * need));
    c->loop_cap = need;
    drop_graph(c);
  }
  KMC_CUDA(cudaMemsetAsync(c->d_loop, 0, sizeof(long long) * need, c->stream));
  KMC_CUDA(cudaMemsetAsync(c->d_eacc, 0, sizeof(double) * c->N, c->stream));
  KMC_CUDA(cudaMemsetAsync(c->d_dh, 0, sizeof(double) * c->N, c->stream));
  KMC_CUDA(cudaMemsetAsync(c->d_cnt, 0, sizeof(unsigned long long) * kmc::kCounters * c->n_lys,
                           c->stream));
  KMC_CUDA(cudaMemsetAsync(c->d_err, 0, 2 * sizeof(int32_t), c->stream));
  if (c->arrivals_cap)
    KMC_CUDA(cudaMemsetAsync(c->d_arrivals, 0, sizeof(int32_t) * c->arrivals_cap, c->stream));
  KMC_TRY(refresh_sources(c, static_cast<int>(c->step_global & 1)));
  RunState rs{c->step_global, 0, 0};
  KMC_CUDA(cudaMemcpyAsync(c->d_rs, &rs, sizeof(rs), cudaMemcpyHostToDevice, c->stream));
  const Shape &sh = c->shape;
  if (sh.persist) {  // one persistent launch per period, then the period advance
    StepArgs a = base_args(c);
    a.seed = seed;
    a.discard = discard;
    a.n_rec = static_cast<int>(std::max(n_rec, 1ll));
    KMC_TRY(prepare_persist(c, S));
    for (int p = 0; p < periods; ++p) {
      KMC_CUDA(launch_period(c, a, sh, S));
      KMC_CUDA(kmc::launch_advance(c->d_rs, S, c->stream));
    }
  }
  // otherwise one field period (S step launches + the period advance) as a CUDA graph
  if (!sh.persist && (!c->gexec || c->g_S != S || c->g_discard != discard || c->g_nrec != n_rec ||
      !(c->g_shape == sh) || c->g_seed != seed)) {
    drop_graph(c);
    StepArgs a = base_args(c);
    a.seed = seed;
    a.S = S;
    a.discard = discard;
    a.n_rec = static_cast<int>(std::max(n_rec, 1ll));
    KMC_TRY(capture_steps(c, a, sh, S, true, &c->gexec));
    c->g_S = S;
    c->g_discard = discard;
    c->g_nrec = static_cast<int>(n_rec);
    c->g_shape = sh;
    c->g_seed = seed;
  }
  for (int p = 0; p < periods && !sh.persist; ++p)
    KMC_CUDA(cudaGraphLaunch(c->gexec, c->stream));
  c->step_global += static_cast<long long>(S) * periods;
  c->have_run = true;
  c->S = S;
  c->periods = periods;
  c->discard = discard;
  c->n_rec = static_cast<int>(n_rec);
  c->f = f;
  return KMC_OK;
}

kmc_status kmc_sync(kmc_ctx *c) {
  Phase phase("kmc_sync");
  if (!c) return fail(KMC_EINVAL, "ctx is NULL");
  return check_device_error(c);
}

kmc_status kmc_read(kmc_ctx *c, int32_t what, int32_t lys, double *buf, int64_t cap,
                    int64_t *written) {
  Phase phase("kmc_read");
  if (!c) return fail(KMC_EINVAL, "ctx is NULL");
  if (written) *written = 0;
  if (lys < 0 || lys >= c->n_lys) return fail(KMC_EINVAL, "lysosome %d out of range", lys);
  if (cap < 0 || (cap > 0 && !buf)) return fail(KMC_EINVAL, "bad output buffer");
  if (what == KMC_READ_COUNTERS || what == KMC_READ_MOMENTS || what == KMC_READ_POSITIONS ||
      what == KMC_READ_AXES) {
    // state, readable after a device error so that the caller can see what
    // happened (kmc_sync reports the error)
    KMC_CUDA(cudaStreamSynchronize(c->stream));
  } else {
    KMC_TRY(check_device_error(c));
  }
  const int n = c->n[lys], o = c->off[lys];
  int64_t need = 0;
  switch (what) {
    case KMC_READ_LOOP_H:
    case KMC_READ_LOOP_M: need = c->n_rec; break;
    case KMC_READ_NP_ENERGY:
    case KMC_READ_DHDIP: need = n; break;
    case KMC_READ_POSITIONS:
    case KMC_READ_AXES: need = 3ll * n; break;
    case KMC_READ_AREA:
    case KMC_READ_SAR: need = 1; break;
    case KMC_READ_MOMENTS: need = 3ll * n; break;
    case KMC_READ_COUNTERS: need = kmc::kCounters - 1; break;
    default: return fail(KMC_EINVAL, "unknown output %d", what);
  }
  if (what != KMC_READ_MOMENTS && what != KMC_READ_POSITIONS && what != KMC_READ_AXES &&
      !c->have_run)
    return fail(KMC_ESTATE, "no run has been made on this context");
  if (written) *written = need;
  if (cap < need) return fail(KMC_ECAPACITY, "output needs %lld elements", (long long)need);
  const int nper = c->periods - c->discard;
  switch (what) {
    case KMC_READ_LOOP_H: {
      int64_t q = 0;
      for (int p = c->discard; p < c->periods; ++p)
        for (int k = 0; k < c->S; ++k) buf[q++] = c->Hmax[lys] * std::cos(2.0 * kPi * k / c->S);
      break;
    }
    case KMC_READ_LOOP_M:
      if (need) {
        std::vector<long long> fx(need);
        KMC_CUDA(cudaMemcpy(fx.data(),
                            c->d_loop + static_cast<size_t>(lys) * std::max(c->n_rec, 1),
                            sizeof(long long) * need, cudaMemcpyDeviceToHost));
        for (int64_t q = 0; q < need; ++q)
          buf[q] = static_cast<double>(fx[q]) / kmc::kLoopScale;
      }
      break;
    case KMC_READ_NP_ENERGY:
    case KMC_READ_AREA:
    case KMC_READ_SAR: {
      std::vector<double> e(n);
      KMC_CUDA(cudaMemcpy(e.data(), c->d_eacc + o, sizeof(double) * n, cudaMemcpyDeviceToHost));
      const double unit = kMu0 * c->Ms[lys] * c->Ms[lys];  // J / m^3 per unit of e_acc
      double tot = 0.0;
      for (int i = 0; i < n; ++i) {
        const double Ei = nper > 0 ? unit * c->vol[o + i] * e[i] / nper : 0.0;
        if (what == KMC_READ_NP_ENERGY) buf[i] = Ei;
        tot += Ei;
      }
      const double area = tot / c->vsum[lys];
      if (what == KMC_READ_AREA) buf[0] = area;
      if (what == KMC_READ_SAR) buf[0] = area * c->f / c->rho[lys];
      break;
    }
    case KMC_READ_POSITIONS:
      for (int64_t q = 0; q < 3ll * n; ++q) buf[q] = c->pos_si[3ll * o + q];
      break;
    case KMC_READ_AXES:
    case KMC_READ_MOMENTS: {
      HostBytes raw(c->vbytes * n);
      const void *src = what == KMC_READ_AXES ? c->d_axis : c->d_m;
      KMC_CUDA(cudaMemcpy(raw.data(), static_cast<const unsigned char *>(src) + c->vbytes * o,
                          raw.size(), cudaMemcpyDeviceToHost));
      for (int i = 0; i < n; ++i) {
        if (c->fp32) {
          const float4 v = reinterpret_cast<float4 *>(raw.data())[i];
          buf[3 * i] = v.x;
          buf[3 * i + 1] = v.y;
          buf[3 * i + 2] = v.z;
        } else {
          const dbl4 v = reinterpret_cast<dbl4 *>(raw.data())[i];
          buf[3 * i] = v.x;
          buf[3 * i + 1] = v.y;
          buf[3 * i + 2] = v.z;
        }
      }
      break;
    }
    case KMC_READ_DHDIP: {
      std::vector<double> d(n);
      KMC_CUDA(cudaMemcpy(d.data(), c->d_dh + o, sizeof(double) * n, cudaMemcpyDeviceToHost));
      const double unit = kMu0 * c->Ms[lys];  // tesla per unit of reduced field
      for (int i = 0; i < n; ++i) buf[i] = nper > 0 ? unit * d[i] / nper : 0.0;
      break;
    }
    case KMC_READ_COUNTERS: {
      unsigned long long cn[kmc::kCounters];
      KMC_CUDA(cudaMemcpy(cn, c->d_cnt + static_cast<long long>(kmc::kCounters) * lys, sizeof(cn),
                          cudaMemcpyDeviceToHost));
      for (int q = 0; q < kmc::kCounters - 1; ++q) buf[q] = static_cast<double>(cn[q]);
      break;
    }
  }
  return KMC_OK;
}

kmc_status kmc_debug_step(kmc_ctx *c, const double *mu0Hext, double t_step, uint64_t seed,
                          int64_t step, const double *m_in, double *m_out, double *B_dip,
                          double *dE, double *P, double *u, int32_t *flags) {
  Phase phase("kmc_debug_step");
  if (!c) return fail(KMC_EINVAL, "ctx is NULL");
  if (!mu0Hext || !m_in) return fail(KMC_EINVAL, "NULL input");
  if (!(t_step > 0) || !is_finite(t_step)) return fail(KMC_EINVAL, "t_step must be > 0");
  if (step < 0) return fail(KMC_EINVAL, "step must be >= 0");
  for (int l = 0; l < c->n_lys; ++l)
    if (!is_finite(mu0Hext[l])) return fail(KMC_EINVAL, "non-finite field");
  for (long long i = 0; i < 3 * c->N; ++i)
    if (!is_finite(m_in[i])) return fail(KMC_EINVAL, "non-finite moment");
  KMC_TRY(ensure_shape(c));
  const long long N = c->N;
  if (!c->d_dbg) {
    KMC_TRY(dalloc(&c->d_dbg, sizeof(double) * N * 7));
    KMC_TRY(dalloc(&c->d_dbg_flags, sizeof(int32_t) * N));
  }
  HostBytes h_m(c->vbytes * N);
  for (long long i = 0; i < N; ++i) {
    if (c->fp32)
      reinterpret_cast<float4 *>(h_m.data())[i] =
          make4<float4>(m_in[3 * i], m_in[3 * i + 1], m_in[3 * i + 2], 0.0);
    else
      reinterpret_cast<dbl4 *>(h_m.data())[i] =
          make4<dbl4>(m_in[3 * i], m_in[3 * i + 1], m_in[3 * i + 2], 0.0);
  }
  KMC_CUDA(cudaStreamSynchronize(c->stream));
  KMC_CUDA(cudaMemcpy(c->d_m, h_m.data(), h_m.size(), cudaMemcpyHostToDevice));
  const int par = static_cast<int>(step & 1);
  KMC_TRY(refresh_sources(c, par));
  for (int l = 0; l < c->n_lys; ++l) {
    c->h_lys[l].bmax = mu0Hext[l] / (kMu0 * c->Ms[l]);
    c->h_lys[l].lognu0t = std::log(t_step / c->tau0[l]);
  }
  KMC_TRY(upload_lys(c));
  RunState rs{step, -1, 0};
  KMC_CUDA(cudaMemcpyAsync(c->d_rs, &rs, sizeof(rs), cudaMemcpyHostToDevice, c->stream));
  KMC_CUDA(cudaMemsetAsync(c->d_err, 0, 2 * sizeof(int32_t), c->stream));
  if (c->arrivals_cap)
    KMC_CUDA(cudaMemsetAsync(c->d_arrivals, 0, sizeof(int32_t) * c->arrivals_cap, c->stream));
  StepArgs a = base_args(c);
  a.seed = seed;
  a.S = 1;
  a.n_rec = 1;
  a.cos_k = 1.0;
  a.debug = 1;
  // test of the FP32 path's FP64 rescan, which valid profiles of Eq. 2 never need
  const char *rescan = std::getenv("KMC_DEBUG_RESCAN");
  a.force_rescan = c->fp32 && rescan && std::strcmp(rescan, "1") == 0;
  a.dbg.bdip = c->d_dbg;
  a.dbg.dE = c->d_dbg + 3 * N;
  a.dbg.P = c->d_dbg + 5 * N;
  a.dbg.u = c->d_dbg + 6 * N;
  a.dbg.flags = c->d_dbg_flags;
  KMC_CUDA(launch_one_step(c, a, c->shape, c->stream, false));
  KMC_TRY(check_device_error(c));
  std::vector<double> h(7 * N);
  std::vector<int32_t> hf(N);
  KMC_CUDA(cudaMemcpy(h.data(), c->d_dbg, sizeof(double) * 7 * N, cudaMemcpyDeviceToHost));
  KMC_CUDA(cudaMemcpy(hf.data(), c->d_dbg_flags, sizeof(int32_t) * N, cudaMemcpyDeviceToHost));
  KMC_CUDA(cudaMemcpy(h_m.data(), c->d_m, h_m.size(), cudaMemcpyDeviceToHost));
  for (int l = 0; l < c->n_lys; ++l) {
    const double Bunit = kMu0 * c->Ms[l];              // T per reduced field unit
    const double Eunit = kMu0 * c->Ms[l] * c->Ms[l];  // J / m^3 per reduced energy unit
    for (int ii = 0; ii < c->n[l]; ++ii) {
      const long long i = c->off[l] + ii;
      if (B_dip)
        for (int q = 0; q < 3; ++q) B_dip[3 * i + q] = Bunit * h[3 * i + q];
      if (dE)
        for (int q = 0; q < 2; ++q) dE[2 * i + q] = Eunit * c->vol[i] * h[3 * N + 2 * i + q];
      if (P) P[i] = h[5 * N + i];
      if (u) u[i] = h[6 * N + i];
      if (flags) flags[i] = hf[i];
      if (m_out) {
        if (c->fp32) {
          const float4 v = reinterpret_cast<float4 *>(h_m.data())[i];
          m_out[3 * i] = v.x;
          m_out[3 * i + 1] = v.y;
          m_out[3 * i + 2] = v.z;
        } else {
          const dbl4 v = reinterpret_cast<dbl4 *>(h_m.data())[i];
          m_out[3 * i] = v.x;
          m_out[3 * i + 1] = v.y;
          m_out[3 * i + 2] = v.z;
        }
      }
    }
  }
  return KMC_OK;
}

// Checkpoint file: magic, version, precision, n_lys, N, global step, NP counts,
// then the raw moment records.
kmc_status kmc_save(kmc_ctx *c, const char *path) {
  if (!c || !path) return fail(KMC_EINVAL, "NULL argument");
  KMC_TRY(check_device_error(c));
  HostBytes raw(c->vbytes * c->N);
  KMC_CUDA(cudaMemcpy(raw.data(), c->d_m, raw.size(), cudaMemcpyDeviceToHost));
  FILE *fp = std::fopen(path, "wb");
  if (!fp) return fail(KMC_EIO, "cannot open %s for writing", path);
  const char magic[8] = {'K', 'M', 'C', 'S', 'T', 'A', 'T', 'E'};
  const int32_t hdr[3] = {1, c->fp32, c->n_lys};
  const int64_t hdr2[2] = {c->N, c->step_global};
  bool ok = std::fwrite(magic, 1, 8, fp) == 8 && std::fwrite(hdr, sizeof(hdr), 1, fp) == 1 &&
            std::fwrite(hdr2, sizeof(hdr2), 1, fp) == 1 &&
            std::fwrite(c->n.data(), sizeof(int), c->n_lys, fp) ==
                static_cast<size_t>(c->n_lys) &&
            std::fwrite(raw.data(), 1, raw.size(), fp) == raw.size();
  ok = (std::fclose(fp) == 0) && ok;
  if (!ok) return fail(KMC_EIO, "short write to %s", path);
  return KMC_OK;
}

kmc_status kmc_load(kmc_ctx *c, const char *path) {
  if (!c || !path) return fail(KMC_EINVAL, "NULL argument");
  FILE *fp = std::fopen(path, "rb");
  if (!fp) return fail(KMC_EIO, "cannot open %s", path);
  char magic[8];
  int32_t hdr[3];
  int64_t hdr2[2];
  bool ok = std::fread(magic, 1, 8, fp) == 8 && std::memcmp(magic, "KMCSTATE", 8) == 0 &&
            std::fread(hdr, sizeof(hdr), 1, fp) == 1 && std::fread(hdr2, sizeof(hdr2), 1, fp) == 1;
  if (!ok || hdr[0] != 1) {
    std::fclose(fp);
    return fail(KMC_EIO, "%s is not a libkmc checkpoint", path);
  }
  if (hdr[1] != c->fp32 || hdr[2] != c->n_lys || hdr2[0] != c->N || hdr2[1] < 0) {
    std::fclose(fp);
    return fail(KMC_EINVAL, "checkpoint does not match this context");
  }
  std::vector<int> nn(c->n_lys);
  HostBytes raw(c->vbytes * c->N);
  ok = std::fread(nn.data(), sizeof(int), c->n_lys, fp) == static_cast<size_t>(c->n_lys) &&
       std::fread(raw.data(), 1, raw.size(), fp) == raw.size();
  std::fclose(fp);
  if (!ok) return fail(KMC_EIO, "truncated checkpoint %s", path);
  if (nn != c->n) return fail(KMC_EINVAL, "checkpoint does not match this context");
  // every moment must be a finite unit vector (a step keeps |m| = 1 to the
  // precision's rounding); anything else is a damaged file, refused before
  // it reaches the device
  for (long long i = 0; i < c->N; ++i) {
    double x, y, z;
    const unsigned char *e = raw.data() + c->vbytes * i;  // copied out: no alignment assumed
    if (c->fp32) {
      float v[3];
      std::memcpy(v, e, sizeof(v));
      x = v[0], y = v[1], z = v[2];
    } else {
      double v[3];
      std::memcpy(v, e, sizeof(v));
      x = v[0], y = v[1], z = v[2];
    }
    const double r2 = x * x + y * y + z * z;
    if (!is_finite(r2) || std::fabs(r2 - 1.0) > 1e-3)
      return fail(KMC_EINVAL, "checkpoint %s: moment %lld is not a finite unit vector", path, i);
  }
  KMC_CUDA(cudaStreamSynchronize(c->stream));
  KMC_CUDA(cudaMemcpy(c->d_m, raw.data(), raw.size(), cudaMemcpyHostToDevice));
  c->step_global = hdr2[1];
  c->have_run = false;
  return KMC_OK;
}

kmc_status kmc_local_concentration(kmc_ctx *c, int32_t lys, int32_t N, double *phi, int64_t cap,
                                   int64_t *written) {
  if (!c) return fail(KMC_EINVAL, "ctx is NULL");
  if (written) *written = 0;
  if (lys < 0 || lys >= c->n_lys) return fail(KMC_EINVAL, "lysosome %d out of range", lys);
  const int n = c->n[lys];
  if (N < 1 || N > n - 1 || N > kmc::kPhiMaxN)
    return fail(KMC_EINVAL, "neighbour rank N = %d outside 1..min(n - 1 = %d, %d)", N, n - 1,
                kmc::kPhiMaxN);
  if (cap < 0 || (cap > 0 && !phi)) return fail(KMC_EINVAL, "bad output buffer");
  if (written) *written = n;
  if (cap < n) return fail(KMC_ECAPACITY, "output needs %d elements", n);
  KMC_TRY(check_device_error(c));
  if (!c->d_phi) {
    int max_n = 0;
    for (int x : c->n) max_n = std::max(max_n, x);
    KMC_TRY(dalloc(&c->d_phi, sizeof(double) * max_n));
  }
  if (!c->d_phif) {
    int max_n = 0;
    for (int x : c->n) max_n = std::max(max_n, x);
    KMC_TRY(dalloc(&c->d_phif, sizeof(float4) * max_n));
  }
  const dbl4 *pos = static_cast<const dbl4 *>(c->fp32 ? c->d_pos64 : c->d_pos) + c->off[lys];
  // largest distance from the frame origin, in units of L (with a little
  // slack for the rounding of the device's frame coordinates)
  double rmax = 0.0;
  for (int i = 0; i < n; ++i) {
    const double *q = &c->pos_si[3ull * (c->off[lys] + i)];
    const double dx = q[0] - c->ctr[3 * lys], dy = q[1] - c->ctr[3 * lys + 1],
                 dz = q[2] - c->ctr[3 * lys + 2];
    rmax = std::max(rmax, std::sqrt(dx * dx + dy * dy + dz * dz));
  }
  rmax = 1.01 * rmax / c->len[lys];
  KMC_CUDA(kmc::launch_local_concentration(pos, n, N, rmax, c->d_phif, c->d_phi, c->stream));
  KMC_CUDA(cudaMemcpyAsync(phi, c->d_phi, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  KMC_CUDA(cudaStreamSynchronize(c->stream));
  return KMC_OK;
}

kmc_status kmc_shell_profile(kmc_ctx *c, int32_t lys, double radius, int32_t n_shells, int32_t N,
                             double *out, int64_t cap, int64_t *written, double *radius_used) {
  if (!c) return fail(KMC_EINVAL, "ctx is NULL");
  if (written) *written = 0;
  if (lys < 0 || lys >= c->n_lys) return fail(KMC_EINVAL, "lysosome %d out of range", lys);
  if (n_shells < 1 || !is_finite(radius)) return fail(KMC_EINVAL, "need n_shells >= 1, finite radius");
  if (cap < 0 || (cap > 0 && !out)) return fail(KMC_EINVAL, "bad output buffer");
  if (!c->have_run) return fail(KMC_ESTATE, "no run has been made on this context");
  const int n = c->n[lys], o = c->off[lys];
  const int64_t need = 4ll * n_shells;
  if (written) *written = need;
  if (cap < need) return fail(KMC_ECAPACITY, "output needs %lld elements", (long long)need);
  std::vector<double> area(n), dh(n), phi(n, 0.0);
  int64_t got = 0;
  KMC_TRY(kmc_read(c, KMC_READ_NP_ENERGY, lys, area.data(), n, &got));
  KMC_TRY(kmc_read(c, KMC_READ_DHDIP, lys, dh.data(), n, &got));
  if (N > 0) KMC_TRY(kmc_local_concentration(c, lys, N, phi.data(), n, &got));
  // per-NP area (J/m^3 per cycle) from the energy per period
  for (int i = 0; i < n; ++i) area[i] /= c->vol[o + i];
  // radii about the frame origin, in the order of operations of the definition
  const double *ctr = &c->ctr[3 * lys];
  std::vector<double> r(n);
  double rmax = 0.0;
  for (int i = 0; i < n; ++i) {
    const double *p = &c->pos_si[3 * (o + i)];
    const double dx = p[0] - ctr[0], dy = p[1] - ctr[1], dz = p[2] - ctr[2];
    const double sq = dx * dx + dy * dy;
    r[i] = std::sqrt(sq + dz * dz);
    const double a = std::cbrt(3.0 * c->vol[o + i] / (4.0 * kPi));
    rmax = std::max(rmax, r[i] + a);
  }
  const double R = radius > 0.0 ? radius : rmax;
  std::vector<double> vs(n_shells, 0.0);
  for (int64_t q = 0; q < need; ++q) out[q] = 0.0;
  for (int i = 0; i < n; ++i) {
    int sh = n_shells - 1;
    if (R > 0.0) {
      const double x = std::floor(static_cast<double>(n_shells) * r[i] / R);
      if (x < static_cast<double>(n_shells - 1)) sh = static_cast<int>(x);
    }
    const double V = c->vol[o + i];
    double *row = out + 4 * sh;
    row[0] += 1.0;
    row[1] += V * area[i];
    row[2] += V * dh[i];
    row[3] += V * phi[i];
    vs[sh] += V;
  }
  for (int sh = 0; sh < n_shells; ++sh)
    if (vs[sh] > 0.0)
      for (int q = 1; q < 4; ++q) out[4 * sh + q] /= vs[sh];
  if (radius_used) *radius_used = R;
  return KMC_OK;
}

kmc_status kmc_mean_run(const kmc_lysosome *lys, int32_t n_lys, const double *mu0Hmax,
                        int32_t n_amp, double f, int32_t S, int32_t periods, int32_t discard,
                        double *loop_M, int64_t cap, int64_t *written) {
  g_last_error.clear();
  if (written) *written = 0;
  if (!lys || n_lys < 1) return fail(KMC_EINVAL, "need at least one lysosome");
  long long N = 0;
  KMC_TRY(validate_lysosomes(lys, n_lys, &N));
  if (!mu0Hmax || (n_amp != 1 && n_amp != n_lys))
    return fail(KMC_EINVAL, "need 1 or n_lys = %d amplitudes", n_lys);
  for (int q = 0; q < n_amp; ++q)
    if (!is_finite(mu0Hmax[q])) return fail(KMC_EINVAL, "non-finite field amplitude");
  if (!(f > 0) || !is_finite(f)) return fail(KMC_EINVAL, "f must be > 0");
  if (S < 1) return fail(KMC_EINVAL, "steps_per_period must be >= 1");
  if (periods < 0 || discard < 0 || discard > periods)
    return fail(KMC_EINVAL, "need 0 <= discard_periods <= periods");
  const long long n_rec = static_cast<long long>(S) * (periods - discard);
  if (n_rec > (1ll << 28)) return fail(KMC_EINVAL, "too many recorded steps");
  if (cap < 0 || (cap > 0 && !loop_M)) return fail(KMC_EINVAL, "bad output buffer");
  const long long need = n_rec * n_lys;
  if (written) *written = need;
  if (cap < need) return fail(KMC_ECAPACITY, "output needs %lld elements", need);
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return fail(KMC_ECUDA, "no CUDA device available");
  }
  KMC_TRY(ensure_device_init());
  const double t_step = 1.0 / (f * S);
  std::vector<kmc::MeanLysDev> hl(n_lys);
  std::vector<kmc::MeanItem> items;
  std::vector<dbl4> axis(N);
  std::vector<double> beta(N), vfrac(N), cosk(S);
  for (int k = 0; k < S; ++k) cosk[k] = std::cos(2.0 * kPi * k / S);
  long long o = 0;
  for (int l = 0; l < n_lys; ++l) {
    const kmc_lysosome &L = lys[l];
    double vs = 0.0;
    for (int i = 0; i < L.n; ++i) vs += L.vol[i];
    kmc::MeanLysDev &D = hl[l];
    D.off = static_cast<int>(o);
    D.n = L.n;
    D.t_zero = L.T == 0.0;
    D.pad = 0;
    D.k = L.Keff / (kMu0 * L.Ms * L.Ms);
    D.bmax = mu0Hmax[n_amp == 1 ? 0 : l] / (kMu0 * L.Ms);
    D.lognu0t = std::log(t_step / L.tau0);
    for (int t0 = 0; t0 < L.n; t0 += kmc::kTargets)
      items.push_back({l, t0, std::min(kmc::kTargets, L.n - t0), 0});
    for (int i = 0; i < L.n; ++i, ++o) {
      const double *a = &L.axis[3 * i];
      const double an = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
      axis[o] = make4<dbl4>(a[0] / an, a[1] / an, a[2] / an, 0.0);
      beta[o] = L.T > 0 ? kMu0 * L.Ms * L.Ms * L.vol[i] / (kKB * L.T) : 0.0;
      vfrac[o] = L.vol[i] / vs;
    }
  }
  // device copies, freed on every path out
  struct Buffers {
    void *p[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaStream_t st = nullptr;
    ~Buffers() {
      if (st) cudaStreamSynchronize(st);
      for (void *q : p)
        if (q) cudaFree(q);
      if (st) cudaStreamDestroy(st);
    }
  } b;
  KMC_CUDA(cudaStreamCreateWithFlags(&b.st, cudaStreamNonBlocking));
  const size_t nl = static_cast<size_t>(std::max(need, 1ll));
  KMC_TRY(dalloc(reinterpret_cast<kmc::MeanLysDev **>(&b.p[0]), sizeof(kmc::MeanLysDev) * n_lys));
  KMC_TRY(dalloc(reinterpret_cast<kmc::MeanItem **>(&b.p[1]), sizeof(kmc::MeanItem) * items.size()));
  KMC_TRY(dalloc(reinterpret_cast<dbl4 **>(&b.p[2]), sizeof(dbl4) * N));
  KMC_TRY(dalloc(reinterpret_cast<double **>(&b.p[3]), sizeof(double) * 2 * N));
  KMC_TRY(dalloc(reinterpret_cast<double **>(&b.p[4]), sizeof(double) * S));
  KMC_TRY(dalloc(reinterpret_cast<long long **>(&b.p[5]), sizeof(long long) * nl));
  KMC_TRY(dalloc(reinterpret_cast<int32_t **>(&b.p[6]), sizeof(int32_t)));
  double *d_bv = static_cast<double *>(b.p[3]);
  KMC_CUDA(cudaMemcpyAsync(b.p[0], hl.data(), sizeof(kmc::MeanLysDev) * n_lys,
                           cudaMemcpyHostToDevice, b.st));
  KMC_CUDA(cudaMemcpyAsync(b.p[1], items.data(), sizeof(kmc::MeanItem) * items.size(),
                           cudaMemcpyHostToDevice, b.st));
  KMC_CUDA(cudaMemcpyAsync(b.p[2], axis.data(), sizeof(dbl4) * N, cudaMemcpyHostToDevice, b.st));
  KMC_CUDA(cudaMemcpyAsync(d_bv, beta.data(), sizeof(double) * N, cudaMemcpyHostToDevice, b.st));
  KMC_CUDA(cudaMemcpyAsync(d_bv + N, vfrac.data(), sizeof(double) * N, cudaMemcpyHostToDevice,
                           b.st));
  KMC_CUDA(cudaMemcpyAsync(b.p[4], cosk.data(), sizeof(double) * S, cudaMemcpyHostToDevice, b.st));
  KMC_CUDA(cudaMemsetAsync(b.p[5], 0, sizeof(long long) * nl, b.st));
  KMC_CUDA(cudaMemsetAsync(b.p[6], 0, sizeof(int32_t), b.st));
  kmc::MeanArgs a;
  a.items = static_cast<const kmc::MeanItem *>(b.p[1]);
  a.n_items = static_cast<int32_t>(items.size());
  a.S = S;
  a.periods = periods;
  a.discard = discard;
  a.n_rec = static_cast<int32_t>(std::max(n_rec, 1ll));
  a.lys = static_cast<const kmc::MeanLysDev *>(b.p[0]);
  a.axis = static_cast<const dbl4 *>(b.p[2]);
  a.beta = d_bv;
  a.vfrac = d_bv + N;
  a.cos_k = static_cast<const double *>(b.p[4]);
  a.loop = static_cast<long long *>(b.p[5]);
  a.err = static_cast<int32_t *>(b.p[6]);
  KMC_CUDA(kmc::launch_mean(a, b.st));
  std::vector<long long> fx(nl);
  int32_t err = 0;
  KMC_CUDA(cudaMemcpyAsync(fx.data(), b.p[5], sizeof(long long) * nl, cudaMemcpyDeviceToHost,
                           b.st));
  KMC_CUDA(cudaMemcpyAsync(&err, b.p[6], sizeof(int32_t), cudaMemcpyDeviceToHost, b.st));
  KMC_CUDA(cudaStreamSynchronize(b.st));
  if (err & kmc::kErrExtrema)
    return fail(KMC_ESTATE, "an energy profile had more than two minima or maxima");
  for (long long q = 0; q < need; ++q) loop_M[q] = static_cast<double>(fx[q]) / kmc::kLoopScale;
  return KMC_OK;
}

kmc_status kmc_regenerate_rsa(kmc_ctx *c, int32_t lys, double radius, double diameter,
                              uint64_t seed, uint32_t loop, int64_t max_candidates,
                              int64_t *candidates_used) {
  if (!c) return fail(KMC_EINVAL, "ctx is NULL");
  if (candidates_used) *candidates_used = 0;
  if (lys < 0 || lys >= c->n_lys) return fail(KMC_EINVAL, "lysosome %d out of range", lys);
  if (!(diameter > 0.0) || !is_finite(diameter) || !is_finite(radius) ||
      !(radius > 0.5 * diameter))
    return fail(KMC_EINVAL, "need 0 < diameter < 2 radius, both finite");
  const int n = c->n[lys];
  const long long cap = max_candidates > 0 ? max_candidates : 1000ll * n;
  KMC_TRY(check_device_error(c));
  if (!c->d_nodes) {  // the mean positions: those given at creation
    KMC_TRY(dalloc(&c->d_nodes, sizeof(double) * 3 * c->N));
    KMC_TRY(dalloc(&c->d_possi, sizeof(double) * 3 * c->N));
    KMC_CUDA(cudaMemcpy(c->d_nodes, c->pos_si.data(), sizeof(double) * 3 * c->N,
                        cudaMemcpyHostToDevice));
    KMC_CUDA(cudaMemcpy(c->d_possi, c->pos_si.data(), sizeof(double) * 3 * c->N,
                        cudaMemcpyHostToDevice));
  }
  // scratch, freed on every return
  const int B = static_cast<int>(
      std::min<long long>(kmc::kRsaMaxBatch, std::max<long long>(256, 2ll * n)));
  struct Scratch {
    void *p[8] = {};
    ~Scratch() {
      for (void *q : p)
        if (q) cudaFree(q);
    }
  } sc;
  KMC_TRY(dalloc(reinterpret_cast<double **>(&sc.p[0]), sizeof(double) * 3 * n));
  KMC_TRY(dalloc(reinterpret_cast<double **>(&sc.p[1]), sizeof(double) * 3 * B));
  KMC_TRY(dalloc(reinterpret_cast<int32_t **>(&sc.p[2]), sizeof(int32_t) * B));
  KMC_TRY(dalloc(reinterpret_cast<int32_t **>(&sc.p[3]), sizeof(int32_t) * B));
  KMC_TRY(dalloc(reinterpret_cast<int32_t **>(&sc.p[4]), sizeof(int32_t) * B * kmc::kRsaMaxConf));
  KMC_TRY(dalloc(reinterpret_cast<int32_t **>(&sc.p[5]), sizeof(int32_t)));
  KMC_TRY(dalloc(reinterpret_cast<long long **>(&sc.p[6]), sizeof(long long)));
  KMC_TRY(dalloc(reinterpret_cast<float4 **>(&sc.p[7]), sizeof(float4) * n));
  KMC_CUDA(cudaMemsetAsync(sc.p[5], 0, sizeof(int32_t), c->stream));
  kmc::RsaArgs a;
  a.Rb = radius - 0.5 * diameter;
  a.d2 = diameter * diameter;
  a.seed = seed;
  a.loop = loop;
  a.lys = lys;
  a.B = B;
  a.n = n;
  a.pos = static_cast<double *>(sc.p[0]);
  a.cand = static_cast<double *>(sc.p[1]);
  a.clear = static_cast<int32_t *>(sc.p[2]);
  a.nconf = static_cast<int32_t *>(sc.p[3]);
  a.conf = static_cast<int32_t *>(sc.p[4]);
  a.kept = static_cast<int32_t *>(sc.p[5]);
  a.used = static_cast<long long *>(sc.p[6]);
  a.posf = static_cast<float4 *>(sc.p[7]);
  // FP32 pre-screen: with centres within Rb of the origin, converting them
  // to FP32 (error <= u Rb per coordinate, u = 2^-24) and forming the squared
  // distance D^2 in FP32 errs by at most 4 sqrt(3) u Rb D + 5 u D^2; the
  // margin 2M = 32 u (Rb d + d^2) is over four times that at D = d, and the
  // error grows more slowly than |D^2 - d^2| away from it
  {
    const double u = 0x1.0p-24;
    const double M = 16.0 * u * (a.Rb * diameter + a.d2);
    a.d2_lo = static_cast<float>(std::max(0.0, a.d2 - 2.0 * M));
    a.d2_hi = static_cast<float>(a.d2 + 2.0 * M);
  }
  int32_t kept = 0;
  long long c0 = 0;
  while (kept < n) {
    if (c0 >= cap)
      return fail(KMC_ESTATE, "random sequential addition placed %d of %d spheres in %lld "
                  "candidates (packing too dense for this radius)", kept, n, cap);
    a.c0 = c0;
    a.B = static_cast<int>(std::min<long long>(B, cap - c0));
    KMC_CUDA(kmc::launch_rsa_batch(a, c->stream));
    KMC_CUDA(cudaMemcpyAsync(&kept, a.kept, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    KMC_CUDA(cudaStreamSynchronize(c->stream));
    c0 += a.B;
  }
  long long used = 0;
  KMC_CUDA(cudaMemcpy(&used, a.used, sizeof(long long), cudaMemcpyDeviceToHost));
  // the kept centres become the lysosome's positions (absolute, m), then the
  // NP arrays follow them and the moments restart along the axes
  std::vector<double> p(3ull * n);
  KMC_CUDA(cudaMemcpy(p.data(), a.pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost));
  const size_t o = 3ull * c->off[lys];
  for (int i = 0; i < n; ++i)
    for (int q = 0; q < 3; ++q) c->pos_si[o + 3 * i + q] = c->ctr[3 * lys + q] + p[3 * i + q];
  KMC_CUDA(cudaMemcpyAsync(c->d_possi + o, c->pos_si.data() + o, sizeof(double) * 3 * n,
                           cudaMemcpyHostToDevice, c->stream));
  kmc::RegenArgs r;
  r.off = c->off[lys];
  r.n = n;
  r.lys = lys;
  r.what = kmc::kRegenGiven;
  r.loop = loop;
  r.fp32 = c->fp32;
  r.seed = seed;
  r.disorder = 0.0;
  r.len = c->len[lys];
  r.cx = c->ctr[3 * lys];
  r.cy = c->ctr[3 * lys + 1];
  r.cz = c->ctr[3 * lys + 2];
  r.nodes = c->d_nodes;
  r.pos = c->d_pos;
  r.axis = c->d_axis;
  r.m = c->d_m;
  r.pos64 = c->d_pos64;
  r.pos_si = c->d_possi;
  KMC_CUDA(kmc::launch_regen(r, c->stream));
  KMC_TRY(refresh_sources(c, 0));
  KMC_TRY(refresh_sources(c, 1));
  KMC_CUDA(cudaStreamSynchronize(c->stream));
  if (candidates_used) *candidates_used = used;
  return KMC_OK;
}

kmc_status kmc_regenerate(kmc_ctx *c, int32_t lys, int32_t what, double disorder, uint64_t seed,
                          uint32_t loop) {
  if (!c) return fail(KMC_EINVAL, "ctx is NULL");
  if (lys < -1 || lys >= c->n_lys) return fail(KMC_EINVAL, "lysosome %d out of range", lys);
  if (what < 1 || what > (KMC_REGEN_AXES | KMC_REGEN_POSITIONS))
    return fail(KMC_EINVAL, "what must combine KMC_REGEN_AXES and KMC_REGEN_POSITIONS");
  if ((what & KMC_REGEN_POSITIONS) && !(disorder >= 0 && is_finite(disorder)))
    return fail(KMC_EINVAL, "disorder must be finite and >= 0");
  KMC_TRY(check_device_error(c));
  if (!c->d_nodes) {  // the mean positions: those given at creation
    KMC_TRY(dalloc(&c->d_nodes, sizeof(double) * 3 * c->N));
    KMC_TRY(dalloc(&c->d_possi, sizeof(double) * 3 * c->N));
    KMC_CUDA(cudaMemcpy(c->d_nodes, c->pos_si.data(), sizeof(double) * 3 * c->N,
                        cudaMemcpyHostToDevice));
    KMC_CUDA(cudaMemcpy(c->d_possi, c->pos_si.data(), sizeof(double) * 3 * c->N,
                        cudaMemcpyHostToDevice));
  }
  const int l0 = lys < 0 ? 0 : lys, l1 = lys < 0 ? c->n_lys : lys + 1;
  for (int l = l0; l < l1; ++l) {
    kmc::RegenArgs a;
    a.off = c->off[l];
    a.n = c->n[l];
    a.lys = l;
    a.what = what;
    a.loop = loop;
    a.fp32 = c->fp32;
    a.seed = seed;
    a.disorder = disorder;
    a.len = c->len[l];
    a.cx = c->ctr[3 * l];
    a.cy = c->ctr[3 * l + 1];
    a.cz = c->ctr[3 * l + 2];
    a.nodes = c->d_nodes;
    a.pos = c->d_pos;
    a.axis = c->d_axis;
    a.m = c->d_m;
    a.pos64 = c->d_pos64;
    a.pos_si = c->d_possi;
    KMC_CUDA(kmc::launch_regen(a, c->stream));
  }
  KMC_TRY(refresh_sources(c, 0));
  KMC_TRY(refresh_sources(c, 1));
  if (what & KMC_REGEN_POSITIONS) {
    const size_t o = 3ull * c->off[l0];
    const size_t cnt = 3ull * (c->off[l1 - 1] + c->n[l1 - 1]) - o;
    KMC_CUDA(cudaMemcpyAsync(c->pos_si.data() + o, c->d_possi + o, sizeof(double) * cnt,
                             cudaMemcpyDeviceToHost, c->stream));
  }
  KMC_CUDA(cudaStreamSynchronize(c->stream));
  return KMC_OK;
}

kmc_status kmc_debug_grid_stall(kmc_ctx *c) {
  if (!c) return fail(KMC_EINVAL, "ctx is NULL");
  KMC_TRY(check_device_error(c));
  KMC_TRY(ensure_shape(c));
  if (!c->shape.persist)
    return fail(KMC_EINVAL, "the grid-stall hook needs the persistent period (kmc_persistent)");
  constexpr int kSteps = 4;
  KMC_TRY(prepare_persist(c, kSteps));
  RunState rs{c->step_global, -1, 0};
  KMC_CUDA(cudaMemcpyAsync(c->d_rs, &rs, sizeof(rs), cudaMemcpyHostToDevice, c->stream));
  if (c->arrivals_cap)
    KMC_CUDA(cudaMemsetAsync(c->d_arrivals, 0, sizeof(int32_t) * c->arrivals_cap, c->stream));
  StepArgs a = base_args(c);
  a.n_rec = 1;
  a.stall_block = 0;  // block 0 does not arrive at the barrier after step 1
  a.stall_step = 1;
  a.barrier_ns = 1000000ull;  // 1 ms
  KMC_CUDA(launch_period(c, a, c->shape, kSteps));
  const kmc_status st = check_device_error(c);  // KMC_ETIMEOUT when the barrier gave up
  // the blocks left the period at a step boundary: clear the flag and the
  // arrival counters; the moments have advanced by up to two steps
  KMC_CUDA(cudaMemsetAsync(c->d_err, 0, 2 * sizeof(int32_t), c->stream));
  if (c->arrivals_cap)
    KMC_CUDA(cudaMemsetAsync(c->d_arrivals, 0, sizeof(int32_t) * c->arrivals_cap, c->stream));
  KMC_CUDA(cudaStreamSynchronize(c->stream));
  return st == KMC_OK ? fail(KMC_ESTATE, "the stalled grid barrier did not run out") : st;
}

kmc_status kmc_debug_stall(kmc_ctx *c) {
  if (!c) return fail(KMC_EINVAL, "ctx is NULL");
  if (c->fp32) return fail(KMC_EINVAL, "the stall hook runs on FP64 contexts");
  KMC_TRY(check_device_error(c));
  KMC_TRY(ensure_shape(c));
  RunState rs{c->step_global, -1, 0};
  KMC_CUDA(cudaMemcpyAsync(c->d_rs, &rs, sizeof(rs), cudaMemcpyHostToDevice, c->stream));
  if (c->arrivals_cap)
    KMC_CUDA(cudaMemsetAsync(c->d_arrivals, 0, sizeof(int32_t) * c->arrivals_cap, c->stream));
  StepArgs a = base_args(c);
  a.S = 1;
  a.n_rec = 1;
  a.cos_k = 1.0;
  a.stall_tx = 16;
  a.stall_wait_ns = 1000000ull;  // 1 ms
  KMC_CUDA(kmc::launch_step(c->fp32, c->shape.warps, c->shape.tile, a, c->n_items, c->stream));
  const kmc_status st = check_device_error(c);  // KMC_ETIMEOUT when the waits ran out
  // the blocks stopped before any write: clear the flag, the context stays usable
  KMC_CUDA(cudaMemsetAsync(c->d_err, 0, 2 * sizeof(int32_t), c->stream));
  if (c->arrivals_cap)
    KMC_CUDA(cudaMemsetAsync(c->d_arrivals, 0, sizeof(int32_t) * c->arrivals_cap, c->stream));
  KMC_CUDA(cudaStreamSynchronize(c->stream));
  return st == KMC_OK ? fail(KMC_ESTATE, "the stalled waits did not run out") : st;
}

kmc_status kmc_info(const kmc_ctx *c, int64_t *n_total, int32_t *n_lys, int64_t *global_step) {
  if (!c) return fail(KMC_EINVAL, "ctx is NULL");
  if (n_total) *n_total = c->N;
  if (n_lys) *n_lys = c->n_lys;
  if (global_step) *global_step = c->step_global;
  return KMC_OK;
}

void kmc_destroy(kmc_ctx *c) {
  Phase phase("kmc_destroy");
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_ctx(c);
}

}  // extern "C"
