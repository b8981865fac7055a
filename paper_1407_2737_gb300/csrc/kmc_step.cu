// kmc_step.cu -- the fused kMC step kernels of libkmc (sm_103a).
//
// One launch = one time step of every NP of every lysosome (Sec. II.1 steps
// i-vii). The update is synchronous (Sec. II.2): every block reads the source
// moments of the start of the step from one ping-pong buffer and writes the
// new ones to the other.
//
// Work item = one block of NW warps: 32 target NPs of one lysosome (64 in the
// two-targets-per-lane kernel) against a contiguous range of that lysosome's
// sources. Sources are staged in shared
// memory, tile by tile, by bulk asynchronous copies (cp.async.bulk, double
// buffered, completion on an mbarrier). Warp w takes every NW-th source record
// of a tile for the same 32 targets (one per lane), so every shared-memory
// load is a broadcast.
//
// FP32-mixed pair term (Eq. 1 in reduced units) on two sources at once with
// packed f32x2 instructions, in the form of SrcPair: d = r_j - r_i;
// r2 = |d|^2; q = rsqrt(r2) per half; u = (t_j . d) q^2 with t_j = 3 w_j m_j;
// b_dip += q^3 (u d + n_j) with n_j = -w_j m_j. That is 18 packed instructions
// and 2 reciprocal square roots for 2 pairs. Each tile's partial sums are
// folded into a compensated (Kahan) running sum; the NW warp sums are combined
// in a fixed order with Neumaier's summation. The FP64-plain kernel sums the
// two terms apart, A += (mu_j . d) q^5 d and B += q^3 mu_j, and forms 3A - B.
//
// When a target group's sources are split over several items, each item writes
// its compensated partial sums to scratch; the last item of the group to arrive
// (arrival counter) adds all partials in split order (deterministic) and runs
// steps iii-vii. The dipolar field never leaves the chip otherwise.
//
// Steps iii-vii are shared by the whole block: warp 0 sets up the working
// plane of each target, all warps scan the 200-point energy-derivative grid
// (lanes over targets, warps over segments of the grid), all threads run
// Newton's method (one root per thread), and warp 0 takes the decision
// (basins, barrier, rates, draw).
#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "kmc_device.cuh"
#include "kmc_pair.cuh"
#include "kmc_launch.h"
#include "kmc_mean.cuh"
#include "kmc_regen.cuh"

namespace kmc {

// ---------------------------------------------------------------------------
// Pair loops over one staged tile. MASK: the tile holds some of the block's
// own targets, so the self term (r2 = 0; distinct NPs are never coincident)
// is dropped. The one-target FP32 loop is a function of its own (not
// inlined) so that its register allocation and schedule do not depend on the
// rest of the kernel (measured: inlined, the loop lost 7 % of its throughput
// when the update code after it changed, and the 8 x 2000-NP workload still
// runs 2.6 % slower with it inlined).

template <bool MASK>
__device__ __noinline__ AccF32 pair_tile_f32(const ulonglong2 *__restrict__ sp, int cnt,
                                              int first, int stride, f2 X, f2 Y, f2 Z) {
  AccF32 acc;
  acc.x = acc.y = acc.z = 0ull;
#pragma unroll 2
  for (int r = first; r < cnt; r += stride) {
    ulonglong2 a, b, c, d;
    f2 e;
    load_record(sp, r, a, b, c, d, e);
    pair_record<MASK>(a, b, c, d, e, X, Y, Z, acc);
  }
  return acc;
}

__device__ __forceinline__ void pair_tile_f64(const dbl4 *__restrict__ sp,
                                              const dbl4 *__restrict__ sm, int cnt, int first,
                                              int stride, double xi, double yi, double zi,
                                              double (&acc)[6]) {
  for (int j = first; j < cnt; j += stride) {
    const dbl4 p = sp[j];
    const dbl4 q = sm[j];
    const double dx = p.x - xi, dy = p.y - yi, dz = p.z - zi;
    const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
    if (r2 > 0.0) {
      const double inv = rsqrt(r2);
      const double inv2 = inv * inv;
      const double inv3 = inv * inv2;
      const double md = fma(q.x, dx, fma(q.y, dy, q.z * dz));
      const double s = md * inv2 * inv3;
      acc[0] = fma(s, dx, acc[0]);
      acc[1] = fma(s, dy, acc[1]);
      acc[2] = fma(s, dz, acc[2]);
      acc[3] = fma(inv3, q.x, acc[3]);
      acc[4] = fma(inv3, q.y, acc[4]);
      acc[5] = fma(inv3, q.z, acc[5]);
    }
  }
}

// ---------------------------------------------------------------------------
// Steps iii-vii, shared by the block.

template <typename R>
struct EpiShared {
  R h[3][kTargets];    // combined dipolar field
  R k2[kTargets], k[kTargets], bc[kTargets], bs[kTargets];  // profile of Eq. 2
  int cnt[kTargets];   // sign changes found by the scan
  // brackets as the scan finds them (any order): left node, derivative at the
  // left and at the right node
  int ju[kTargets][4];
  R du[kTargets][4], duh[kTargets][4];
  // brackets in grid order after Newton: left node, derivative there, root,
  // energy, sin and cos of the root, offset of the root from the left node
  int jq[kTargets][4];
  R dq[kTargets][4];
  R th[kTargets][4], en[kTargets][4], sq[kTargets][4], cq[kTargets][4], off[kTargets][4];
};


// Scan of step iv: lane = target, the 200 nodes cut into max(nw, 4) contiguous
// segments (so that a segment holds at most 50), warp w taking segments w,
// w + nw, ... (MULTI, for nw < 4), else segment w alone (nw >= 4). A first pass
// evaluates de/dth at the segment's nodes and at the node after it (cyclically:
// the cell after node 199 ends at node 0) and keeps only their signs, as a bit
// mask, so that its loads and arithmetic pipeline freely; a second pass visits
// the sign changes (at most four per target) and records each in a free slot of
// its target (shared-memory counter). All lanes of a warp read the same node,
// a shared-memory broadcast.
constexpr int kMaxSeg = 50;

// FP32 sign pass over kPairBatch consecutive nodes j0 + q0 .. (j0 + q0 even):
// two nodes per packed instruction, read as pairs from the split sin and cos
// tables, each node with profile_d1's roundings (s (2k c + b cos phi) +
// (-b sin phi) c; a packed operation rounds each half as the scalar one), so
// the signs are those of the scalar pass. Bit q of the result: node q0 + q.
constexpr int kPairBatch = 14;
__device__ __forceinline__ unsigned long long pair_signs(const GridTables<float> &tab, f2 K2,
                                                         f2 BC, f2 NBS, int j0, int q0) {
  unsigned bits = 0;
#pragma unroll
  for (int u = 0; u < kPairBatch; u += 2) {
    const int j = j0 + q0 + u;  // < kGridPad: the tables repeat the grid past its end
    const f2 s = *reinterpret_cast<const f2 *>(&tab.ss[j]);
    const f2 c = *reinterpret_cast<const f2 *>(&tab.cc[j]);
    const f2 d = fma2(s, fma2(K2, c, BC), mul2(NBS, c));
    float dl, dh;
    upk(d, dl, dh);
    bits |= (static_cast<unsigned>(dl < 0.f) << u) | (static_cast<unsigned>(dh < 0.f) << (u + 1));
  }
  return static_cast<unsigned long long>(bits) << q0;
}

template <typename R, bool MULTI = false>
__device__ __forceinline__ void segment_scan(EpiShared<R> &sm, const GridTables<R> &tab,
                                             int warp, int nw, int lane, int nt) {
  if (lane >= nt) return;
  const R k2 = sm.k2[lane], bc = sm.bc[lane], bs = sm.bs[lane];
  auto d1 = [&](int j) {
    const auto sc = tab.sc[j];
    return profile_d1(k2, bc, bs, sc.x, sc.y);
  };
  // bit q of the mask: de/dth < 0 at node j0 + q (q = len: the next node).
  // Batches of 13 independent evaluations keep about 40 registers in flight: a
  // fully unrolled pass would hold 51 table entries and, inside the step
  // kernel's register budget, the compiler serialises it (measured 4x slower).
  constexpr int kBatch = 13;
  auto batch = [&](int j0, int q0) {
    unsigned bits = 0;
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      int j = j0 + q0 + u;
      j = j < kGrid ? j : j - kGrid;  // q0 + u <= kMaxSeg + kBatch - 1: one wrap at most
      bits |= static_cast<unsigned>(d1(j) < R(0)) << u;
    }
    return static_cast<unsigned long long>(bits) << q0;
  };
  // the sign changes of a segment's mask: each in a free slot of the target
  auto record = [&](int j0, int len, unsigned long long neg) {
    unsigned long long chg = (neg ^ (neg >> 1)) & ((1ull << len) - 1);
    while (chg) {
      const int q = __ffsll(static_cast<long long>(chg)) - 1;
      chg &= chg - 1;
      const int j = j0 + q;
      const int slot = atomicAdd(&sm.cnt[lane], 1);
      if (slot < 4) {
        sm.ju[lane][slot] = j;
        sm.du[lane][slot] = d1(j);
        sm.duh[lane][slot] = d1(j + 1 < kGrid ? j + 1 : 0);
      }
    }
  };
  // FP32 segments that start on an even node take the packed pass
  constexpr bool kPairs = std::is_same<R, float>::value;
  f2 K2 = 0, BC = 0, NBS = 0;
  if constexpr (kPairs) {
    K2 = pk(k2, k2);
    BC = pk(bc, bc);
    NBS = pk(-bs, -bs);
  }
  auto scan = [&](int j0, int len) {
    unsigned long long neg = 0;
    if constexpr (kPairs) {
      if ((j0 & 1) == 0) {
#pragma unroll 1
        for (int q0 = 0; q0 <= len; q0 += kPairBatch) neg |= pair_signs(tab, K2, BC, NBS, j0, q0);
        record(j0, len, neg);
        return;
      }
    }
#pragma unroll 1
    for (int q0 = 0; q0 <= len; q0 += kBatch) neg |= batch(j0, q0);
    record(j0, len, neg);
  };
  if constexpr (MULTI) {
    constexpr int nseg = (kGrid + kMaxSeg - 1) / kMaxSeg, seg = (kGrid + nseg - 1) / nseg;
    static_assert(nseg * seg == kGrid && nseg % 2 == 0 && seg % 2 == 0,
                  "whole segments, in pairs, starting on even nodes");
    if (nw == 2) {
      // two segments per warp, w and w + 2, their batches interleaved (twice
      // the independent evaluations in flight)
      const int ja = warp * seg, jb = (warp + 2) * seg;
      unsigned long long na = 0, nb = 0;
      if constexpr (kPairs) {
#pragma unroll 1
        for (int q0 = 0; q0 <= seg; q0 += kPairBatch) {
          na |= pair_signs(tab, K2, BC, NBS, ja, q0);
          nb |= pair_signs(tab, K2, BC, NBS, jb, q0);
        }
      } else {
#pragma unroll 1
        for (int q0 = 0; q0 <= seg; q0 += kBatch) {
          na |= batch(ja, q0);
          nb |= batch(jb, q0);
        }
      }
      record(ja, seg, na);
      record(jb, seg, nb);
    } else {
#pragma unroll 1
      for (int sg = warp; sg < nseg; sg += nw) scan(sg * seg, seg);
    }
  } else {
    const int seg = (kGrid + nw - 1) / nw;
    const int j0 = warp * seg, len = min(kGrid, j0 + seg) - j0;
    if (len > 0) scan(j0, len);
  }
}

// Scan of step iv by one warp alone (the replica kernel gives each warp its own
// targets): lane = target, the lane walks all 200 nodes in segments of
// kMaxSeg, with the same evaluations as segment_scan (same bits), and keeps its
// own bracket count, so its brackets land in grid order.
template <typename R>
__device__ __forceinline__ void lane_scan(EpiShared<R> &sm, const GridTables<R> &tab, int lane,
                                          int nt) {
  if (lane >= nt) return;
  const R k2 = sm.k2[lane], bc = sm.bc[lane], bs = sm.bs[lane];
  auto d1 = [&](int j) {
    const auto sc = tab.sc[j];
    return profile_d1(k2, bc, bs, sc.x, sc.y);
  };
  constexpr int kBatch = 13;
  auto batch = [&](int j0, int q0) {
    unsigned bits = 0;
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      int j = j0 + q0 + u;
      j = j < kGrid ? j : j - kGrid;
      bits |= static_cast<unsigned>(d1(j) < R(0)) << u;
    }
    return static_cast<unsigned long long>(bits) << q0;
  };
  int cnt = 0;
  auto record = [&](int j0, unsigned long long neg) {
    unsigned long long chg = (neg ^ (neg >> 1)) & ((1ull << kMaxSeg) - 1);
    while (chg) {
      const int q = __ffsll(static_cast<long long>(chg)) - 1;
      chg &= chg - 1;
      const int j = j0 + q;
      if (cnt < 4) {
        sm.ju[lane][cnt] = j;
        sm.du[lane][cnt] = d1(j);
        sm.duh[lane][cnt] = d1(j + 1 < kGrid ? j + 1 : 0);
      }
      ++cnt;
    }
  };
  // segments of kMaxSeg nodes in pairs, the two segments' batches interleaved
  // (twice the independent evaluations in flight); the sign changes are then
  // recorded in grid order
  static_assert(kGrid % (2 * kMaxSeg) == 0 && kMaxSeg % 2 == 0,
                "whole pairs of segments, starting on even nodes");
  constexpr bool kPairs = std::is_same<R, float>::value;  // FP32: the packed pass
  f2 K2 = 0, BC = 0, NBS = 0;
  if constexpr (kPairs) {
    K2 = pk(k2, k2);
    BC = pk(bc, bc);
    NBS = pk(-bs, -bs);
  }
#pragma unroll 1
  for (int j0 = 0; j0 < kGrid; j0 += 2 * kMaxSeg) {
    unsigned long long na = 0, nb = 0;
    if constexpr (kPairs) {
#pragma unroll 1
      for (int q0 = 0; q0 <= kMaxSeg; q0 += kPairBatch) {
        na |= pair_signs(tab, K2, BC, NBS, j0, q0);
        nb |= pair_signs(tab, K2, BC, NBS, j0 + kMaxSeg, q0);
      }
    } else {
#pragma unroll 1
      for (int q0 = 0; q0 <= kMaxSeg; q0 += kBatch) {
        na |= batch(j0, q0);
        nb |= batch(j0 + kMaxSeg, q0);
      }
    }
    record(j0, na);
    record(j0 + kMaxSeg, nb);
  }
  sm.cnt[lane] = cnt;
}

// FP32 rounding can flip the sign of de/dth at a node where it nearly vanishes
// (a near-double root just before a well disappears), which adds two sign
// changes. A target whose FP32 scan counts more than four is scanned again by
// one thread with the profile evaluated in FP64 at every node, and those
// brackets (at most four, in grid order) replace the FP32 ones. Kept out of
// line: inlined, this rarely taken FP64 code cost the pair loop 7 %.
__device__ __noinline__ void rescan_fp64(EpiShared<float> &sm, int t) {
  const double k2 = sm.k2[t], bc = sm.bc[t], bs = sm.bs[t];
  auto d1 = [&](int j) {
    const double2 sc = g_sc_d[j];
    return profile_d1(k2, bc, bs, sc.x, sc.y);
  };
  const double d_first = d1(0);
  double left = d_first;
  int cnt = 0;
  for (int j = 0; j < kGrid; ++j) {
    const double right = (j + 1 < kGrid) ? d1(j + 1) : d_first;
    if ((left < 0.0) != (right < 0.0)) {
      if (cnt < 4) {
        sm.ju[t][cnt] = j;
        sm.du[t][cnt] = static_cast<float>(left);
        sm.duh[t][cnt] = static_cast<float>(right);
      }
      ++cnt;
    }
    left = right;
  }
  sm.cnt[t] = cnt;
}

// Newton refinement of bracket q (of nb) of target t (one thread); the result
// goes to the bracket's rank in grid order.
template <typename R>
__device__ __forceinline__ void refine_bracket(EpiShared<R> &sm, const GridTables<R> &tab, int t,
                                               int q, int nb, int32_t *err) {
  Profile<R> pf;
  pf.k2 = sm.k2[t];
  pf.k = sm.k[t];
  pf.bc = sm.bc[t];
  pf.bs = sm.bs[t];
  const int ju = sm.ju[t][q];
  int rank = 0;
  for (int p = 0; p < nb; ++p) rank += sm.ju[t][p] < ju;
  if (!KMC_DCHECK(ju >= 0 && ju < kGrid && rank >= 0 && rank < 4, err, kSiteBracket)) return;
  const int j = min(max(ju, 0), kGrid - 1);
  const auto sc = tab.sc[j];
  const R h = tab.th[1] - tab.th[0];
  R s, c;
  const R dl = sm.du[t][q];
  const R off = refine_in_cell(pf, sc.x, sc.y, h, dl, sm.duh[t][q], s, c);
  R th = tab.th[j] + off;
  if (th >= Prec<R>::two_pi) th -= Prec<R>::two_pi;
  sm.jq[t][rank] = ju;
  sm.dq[t][rank] = dl;
  sm.th[t][rank] = th;
  sm.off[t][rank] = off;
  sm.sq[t][rank] = s;
  sm.cq[t][rank] = c;
  sm.en[t][rank] = pf.e(s, c);
}

// Per-target values warp 0 keeps in registers between the stages.
template <typename R>
struct TargetState {
  R ax, ay, az, ex, ey, ez, m_a, m_e, th0, mz_old, bmag, cphi, sphi;
  bool degenerate;
};

// Step iii: working plane through the axis a and the total field b.
template <typename R>
__device__ __forceinline__ TargetState<R> setup_plane(R ax, R ay, R az, R mx, R my, R mz,
                                                      R bx, R by, R bz) {
  TargetState<R> s;
  s.ax = ax;
  s.ay = ay;
  s.az = az;
  s.mz_old = mz;
  s.bmag = sqrt(fma(bx, bx, fma(by, by, bz * bz)));
  s.ex = s.ey = s.ez = R(0);
  s.cphi = R(1);
  s.sphi = R(0);
  s.degenerate = true;
  if (s.bmag > R(0)) {
    const R inv = R(1) / s.bmag;
    const R hx = bx * inv, hy = by * inv, hz = bz * inv;
    R cphi = fma(ax, hx, fma(ay, hy, az * hz));
    const R px = fma(-cphi, ax, hx), py = fma(-cphi, ay, hy), pz = fma(-cphi, az, hz);
    const R sp = sqrt(fma(px, px, fma(py, py, pz * pz)));
    if (sp >= Prec<R>::plane_tol) {
      s.ex = px / sp;
      s.ey = py / sp;
      s.ez = pz / sp;
      s.sphi = sp;
      s.degenerate = false;
    } else {
      cphi = (cphi >= R(0)) ? R(1) : R(-1);
    }
    s.cphi = cphi;
  }
  if (s.degenerate) {
    const R ma = fma(mx, ax, fma(my, ay, mz * az));
    R px = fma(-ma, ax, mx), py = fma(-ma, ay, my), pz = fma(-ma, az, mz);
    R sp = sqrt(fma(px, px, fma(py, py, pz * pz)));
    if (sp < Prec<R>::plane_tol) {
      if (fabs(ax) > R(0.9)) {  // a x y-hat
        px = -az;
        py = R(0);
        pz = ax;
      } else {  // a x x-hat
        px = R(0);
        py = az;
        pz = -ay;
      }
      sp = sqrt(fma(px, px, fma(py, py, pz * pz)));
    }
    s.ex = px / sp;
    s.ey = py / sp;
    s.ez = pz / sp;
  }
  s.m_a = fma(mx, ax, fma(my, ay, mz * az));
  s.m_e = fma(mx, s.ex, fma(my, s.ey, mz * s.ez));
  R th0 = atan2(s.m_e, s.m_a);
  if (th0 < R(0)) th0 += Prec<R>::two_pi;
  s.th0 = th0;
  return s;
}

struct Decision {
  double dEa, dEb, P;
  int nmin, flipped, near, bad, polished;
};

// e^x for an exponent x held in FP64: x log2(e) = n + f exactly split into an
// integer n and a fraction f in [0, 1); 2^f in FP32, then scaled by 2^n.
__device__ __forceinline__ float exp_fp64_arg(double x) {
  const double y = x * 1.4426950408889634073599;  // log2(e)
  if (y < -160.0) return 0.0f;
  const double n = floor(y);
  const float r = exp2f(static_cast<float>(y - n));
  return ldexpf(r, static_cast<int>(fmin(n, 200.0)));
}

// Steps v-vii for target t: basins, barrier (FP64 polish near the switching
// field in the mixed path), Eqs. 3-5 in FP64, draw u < P. Returns (sin, cos)
// of the new angle in the plane.
template <typename R, bool MIXED>
__device__ __forceinline__ Decision decide(const EpiShared<R> &sm, int t,
                                           const TargetState<R> &st, double beta,
                                           double lognu0t, bool t_zero, double u, R &s_new,
                                           R &c_new) {
  Decision o;
  o.dEa = o.dEb = o.P = 0.0;
  o.flipped = o.near = o.bad = o.polished = 0;
  int cnt = sm.cnt[t];
  if (cnt > 4 || cnt < 0) {
    o.bad = 1;
    cnt = cnt < 0 ? 0 : 4;
  }
  int nmin = 0, nmax = 0, imin0 = 0, imin1 = 0, imax0 = 0, imax1 = 0;
  for (int q = 0; q < cnt; ++q) {
    if (sm.dq[t][q] < R(0)) {
      if (nmin == 0) imin0 = q; else imin1 = q;
      ++nmin;
    } else {
      if (nmax == 0) imax0 = q; else imax1 = q;
      ++nmax;
    }
  }
  if (nmin > 2 || nmax > 2) {
    o.bad = 1;
    nmin = 1;
  }
  o.nmin = nmin;
  if (nmin == 0) {  // flat profile (K_eff = 0 and no field): keep the projection
    const R nrm = sqrt(fma(st.m_a, st.m_a, st.m_e * st.m_e));
    s_new = (nrm > R(0)) ? st.m_e / nrm : R(0);
    c_new = (nrm > R(0)) ? st.m_a / nrm : R(1);
    return o;
  }
  if (nmin == 1) {
    s_new = sm.sq[t][imin0];
    c_new = sm.cq[t][imin0];
    return o;
  }
  // v) basins: the two maxima split the circle into two arcs
  const R M1 = sm.th[t][imax0], M2 = sm.th[t][imax1];
  const bool arc0 = on_arc<R>(st.th0, M1, M2);
  const bool arcA = on_arc<R>(sm.th[t][imin0], M1, M2);
  const int wa = (arc0 == arcA) ? imin0 : imin1;
  const int wb = (wa == imin0) ? imin1 : imin0;
  const R e3 = fmin(sm.en[t][imax0], sm.en[t][imax1]);
  double dEa = static_cast<double>(e3 - sm.en[t][wa]);
  double dEb = static_cast<double>(e3 - sm.en[t][wb]);
  if (MIXED && fmin(dEa, dEb) < 1e-3 * static_cast<double>(sm.k[t])) {
    // Near the switching field E3 - E_a cancels: the energies of the two wells
    // and of the lower maximum are taken again in FP64 at the FP32 roots (the
    // energy is stationary there, so the root's FP32 error enters squared).
    Profile<double> pd;
    pd.k = static_cast<double>(sm.k[t]);
    pd.k2 = 2.0 * pd.k;
    pd.bc = static_cast<double>(st.bmag) * static_cast<double>(st.cphi);
    pd.bs = static_cast<double>(st.bmag) * static_cast<double>(st.sphi);
    const int i3 = (sm.en[t][imax0] <= sm.en[t][imax1]) ? imax0 : imax1;
    const int qs[3] = {wa, wb, i3};
    double e64[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int q = qs[k];
      const double2 sc = g_sc_d[min(max(sm.jq[t][q], 0), kGrid - 1)];
      double sd, cd;
      Prec<double>::sincos_small(static_cast<double>(sm.off[t][q]), sd, cd);
      e64[k] = pd.e(fma(sc.x, cd, sc.y * sd), fma(sc.y, cd, -sc.x * sd));
    }
    dEa = e64[2] - e64[0];
    dEb = e64[2] - e64[1];
    o.polished = 1;
  }
  o.dEa = dEa;
  o.dEb = dEb;
  int w = wa;
  if (!t_zero) {
    // vi) Eqs. 3-5 with nu t = exp(x), x = ln(nu0 t_step) - beta dE
    double P;
    if constexpr (MIXED) {
      // the exponent x in FP64; e^x = 2^n 2^f with n integral and the
      // fraction f in [0, 1) evaluated in FP32
      const float ea = exp_fp64_arg(lognu0t - beta * dEa);
      const float eb = exp_fp64_arg(lognu0t - beta * dEb);
      const float sum = ea + eb;
      P = (sum > 0.f) ? static_cast<double>((ea / sum) * (-expm1f(-sum))) : 0.0;
    } else {
      const double ea = exp(lognu0t - beta * dEa);
      const double eb = exp(lognu0t - beta * dEb);
      const double sum = ea + eb;
      P = (sum > 0.0) ? (ea / sum) * (-expm1(-sum)) : 0.0;
    }
    o.P = P;
    // vii) jump iff u < P
    o.near = fabs(u - P) < 1e-9;
    if (u < P) {
      o.flipped = 1;
      w = wb;
    }
  }
  s_new = sm.sq[t][w];
  c_new = sm.cq[t][w];
  return o;
}

// Per-target inputs of steps iii-vii that warp 0 loads (and the draw it makes)
// before the pair loop, so that their latency hides behind it. Lanes past the
// last target repeat the last target.
template <typename V>
struct TargetIn {
  V ax4, m4;
  double beta, vfrac, eacc, u;
  int i, il;
};

template <typename V>
__device__ __forceinline__ TargetIn<V> load_target(const StepArgs &a, const LysDev &L,
                                                   const Item &it, long long step, int lane) {
  TargetIn<V> p;
  p.il = it.t0 + min(lane, it.nt - 1);
  p.i = L.off + p.il;
  p.ax4 = static_cast<const V *>(a.axis)[p.i];
  p.m4 = static_cast<const V *>(a.m)[p.i];
  p.beta = a.beta[p.i];
  p.vfrac = a.vfrac[p.i];
  p.eacc = a.e_acc[p.i];
  p.u = kmc_uniform(a.seed, step, p.il, it.l);
  return p;
}

// Steps iii-vii for the block's targets; sm.h holds their dipolar fields and
// warp 0 holds their inputs in tin. V = float4 (mixed) or dbl4 (plain).
//
// WARP: the steps are run by the calling warp alone, on its own update state
// (the replica kernel, where every warp updates another lysosome): its lanes
// scan the whole grid for their targets and each lane refines its own
// brackets. GROUP > 0: they are run by the gid-th group of GROUP warps of the
// block on that group's update state, with named barriers, several groups
// side by side (the replica kernel with several warps per replica, the
// multi-target kernel with its 32-target parts side by side). The results are
// the same bits as the block's.
// Barriers of a block_update that the whole block runs (GROUP = 0:
// __syncthreads), or that a group of GROUP warps runs (warps gid GROUP ..
// gid GROUP + GROUP - 1, named barrier 1 + gid), several groups side by side.
template <int GROUP>
struct UpdateSync {
  static __device__ __forceinline__ void sync(int gid) {
    if constexpr (GROUP == 0) {
      __syncthreads();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(1 + gid), "n"(GROUP * 32) : "memory");
    }
  }
  static __device__ __forceinline__ bool sync_or(int gid, bool p) {
    if constexpr (GROUP == 0) {
      return __syncthreads_or(p) != 0;
    } else {
      uint32_t r;
      asm volatile(
          "{\n\t.reg .pred q, o;\n\t"
          "setp.ne.u32 q, %1, 0;\n\t"
          "bar.red.or.pred o, %2, %3, q;\n\t"
          "selp.u32 %0, 1, 0, o;\n\t}"
          : "=r"(r)
          : "r"(static_cast<uint32_t>(p)), "r"(1 + gid), "n"(GROUP * 32)
          : "memory");
      return r != 0;
    }
  }
};

template <typename V, bool MIXED, bool WARP = false, int GROUP = 0>
__device__ __forceinline__ void block_update(
    const StepArgs &a, const LysDev &L, const Item &it, long long step, int rec,
    const TargetIn<V> &tin,
    EpiShared<typename std::conditional<MIXED, float, double>::type> &sm,
    const GridTables<typename std::conditional<MIXED, float, double>::type> &tab, int gid = 0) {
  using R = typename std::conditional<MIXED, float, double>::type;
  using Sync = UpdateSync<GROUP>;
  // this update's threads: the block, or a group of GROUP warps
  const int gtid = GROUP ? static_cast<int>(threadIdx.x) - gid * GROUP * 32
                         : static_cast<int>(threadIdx.x);
  const int gthreads = GROUP ? GROUP * 32 : static_cast<int>(blockDim.x);
  const int warp = WARP ? 0 : gtid >> 5, lane = threadIdx.x & 31;
  const int nw = WARP ? 1 : gthreads >> 5;
  const int nt = it.nt;
  const double bext = L.bmax * a.cos_k;
  TargetState<R> st;
  V m4 = tin.m4;
  const int i = tin.i, il = tin.il;
  // iii) working planes (warp 0, one target per lane)
  if (warp == 0) {
    st = setup_plane<R>(tin.ax4.x, tin.ax4.y, tin.ax4.z, m4.x, m4.y, m4.z, sm.h[0][lane],
                        sm.h[1][lane], sm.h[2][lane] + static_cast<R>(bext));
    sm.k[lane] = static_cast<R>(L.k);
    sm.k2[lane] = R(2) * static_cast<R>(L.k);
    sm.bc[lane] = st.bmag * st.cphi;
    sm.bs[lane] = st.bmag * st.sphi;
    sm.cnt[lane] = 0;
  }
  bool noisy = false;  // warp 0: this lane's target was scanned again in FP64
  if constexpr (WARP) {
    __syncwarp();
    // iv) scan and Newton, each lane for its own target
    lane_scan<R>(sm, tab, lane, nt);
    if constexpr (MIXED) {
      noisy = lane < nt && (sm.cnt[lane] > 4 || a.force_rescan);
      if (noisy) rescan_fp64(sm, lane);
    }
    if (lane < nt) {
      const int nb = min(sm.cnt[lane], 4);
#pragma unroll 1
      for (int q = 0; q < nb; ++q) refine_bracket<R>(sm, tab, lane, q, nb, a.err);
    }
    __syncwarp();
  } else {
    Sync::sync(gid);
    // iv) scan: lanes over targets, warps over segments of the grid
    segment_scan<R, (GROUP > 0 && GROUP < 4)>(sm, tab, warp, nw, lane, nt);
    Sync::sync(gid);
    if constexpr (MIXED) {
      noisy = warp == 0 && lane < nt && (sm.cnt[lane] > 4 || a.force_rescan);
      if (Sync::sync_or(gid, noisy)) {
        if (noisy) rescan_fp64(sm, lane);
        Sync::sync(gid);
      }
    }
    // iv) Newton: one bracket per thread
    for (int x = gtid; x < 4 * nt; x += gthreads) {
      const int t = x >> 2, q = x & 3;
      const int nb = min(sm.cnt[t], 4);
      if (q < nb) refine_bracket<R>(sm, tab, t, q, nb, a.err);
    }
    Sync::sync(gid);
    if (warp != 0) return;
  }
  // v-vii) decision and outputs (warp 0)
  const bool active = lane < nt;
  const double u = tin.u;
  R s_new, c_new;
  // lanes past the last target repeat the last target (same state as st);
  // only targets < nt have scan results in shared memory
  const Decision r = decide<R, MIXED>(sm, min(lane, nt - 1), st, tin.beta, L.lognu0t,
                                      L.t_zero != 0, u, s_new, c_new);
  // Guard: a non-finite field, barrier or probability (two NPs at one point)
  // leaves the moment as it was; the NP-step is counted and reported.
  const bool finite = isfinite(sm.h[0][lane]) && isfinite(sm.h[1][lane]) &&
                      isfinite(sm.h[2][lane]) && isfinite(r.dEa) && isfinite(r.dEb) &&
                      isfinite(r.P);
  const R mx = finite ? fma(c_new, st.ax, s_new * st.ex) : m4.x;
  const R my = finite ? fma(c_new, st.ay, s_new * st.ey) : m4.y;
  const R mz = finite ? fma(c_new, st.az, s_new * st.ez) : m4.z;
  const bool jumped = finite && r.flipped;
  const int par = static_cast<int>(step & 1);
  if (active) {
    m4.x = mx;
    m4.y = my;
    m4.z = mz;
    static_cast<V *>(a.m)[i] = m4;
    const R w = static_cast<const V *>(a.pos)[i].w;
    if constexpr (MIXED) {
      SrcPair *rec_out = static_cast<SrcPair *>(a.src[par ^ 1]) + L.roff + (il >> 1);
      set_source_moment(*rec_out, il & 1, w, mx, my, mz);
    } else {
      dbl4 mu;
      mu.x = w * mx;
      mu.y = w * my;
      mu.z = w * mz;
      mu.w = 0.0;
      static_cast<dbl4 *>(a.src[par ^ 1])[i] = mu;
    }
    if (rec >= 0)
      a.e_acc[i] = tin.eacc + bext * (static_cast<double>(mz) - static_cast<double>(st.mz_old));
    // Eq. 6: the dipolar field along the applied field at its two extremes
    const bool at_max = a.k_local == 0, at_min = a.k_local == a.S / 2;
    if (rec >= 0 && (at_max || at_min)) {
      const double hz = static_cast<double>(sm.h[2][lane]);
      double d = a.dh_acc[i];
      if (at_max) d += hz;
      if (at_min) d -= hz;
      a.dh_acc[i] = d;
    }
    if (a.debug) {
      a.dbg.bdip[3 * i + 0] = static_cast<double>(sm.h[0][lane]);
      a.dbg.bdip[3 * i + 1] = static_cast<double>(sm.h[1][lane]);
      a.dbg.bdip[3 * i + 2] = static_cast<double>(sm.h[2][lane]);
      a.dbg.dE[2 * i + 0] = r.dEa;
      a.dbg.dE[2 * i + 1] = r.dEb;
      a.dbg.P[i] = r.P;
      a.dbg.u[i] = u;
      a.dbg.flags[i] = r.nmin | (jumped ? kFlagJumped : 0) | (r.near ? kFlagNear : 0) |
                       (st.degenerate ? kFlagFallback : 0) | (noisy ? kFlagRescan : 0) |
                       (r.polished ? kFlagPolish : 0) | (finite ? 0 : kFlagNonFinite);
    }
  }
  // loop record and counters: one atomic each per block
  if (rec >= 0) {
    double c = active ? tin.vfrac * static_cast<double>(mz) : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if (lane == 0)
      atomicAdd(reinterpret_cast<unsigned long long *>(
                    &a.loop_m[static_cast<long long>(it.l) * a.n_rec + rec]),
                static_cast<unsigned long long>(__double2ll_rn(c * kLoopScale)));
  }
  const unsigned fl = __ballot_sync(0xffffffffu, active && jumped);
  const unsigned ne = __ballot_sync(0xffffffffu, active && r.near);
  const unsigned mo = __ballot_sync(0xffffffffu, active && r.nmin == 1);
  const unsigned dg = __ballot_sync(0xffffffffu, active && st.degenerate);
  const unsigned rs = __ballot_sync(0xffffffffu, active && noisy);
  const unsigned po = __ballot_sync(0xffffffffu, active && r.polished);
  const unsigned nf = __ballot_sync(0xffffffffu, active && !finite);
  const unsigned bd = __ballot_sync(0xffffffffu, active && r.bad);
  if (lane == 0) {
    unsigned long long *c = a.counters + static_cast<long long>(kCounters) * it.l;
    if (fl) atomicAdd(c + kCntJumps, static_cast<unsigned long long>(__popc(fl)));
    if (ne) atomicAdd(c + kCntNear, static_cast<unsigned long long>(__popc(ne)));
    if (mo) atomicAdd(c + kCntOneMin, static_cast<unsigned long long>(__popc(mo)));
    if (dg) atomicAdd(c + kCntFallback, static_cast<unsigned long long>(__popc(dg)));
    if (rs) atomicAdd(c + kCntRescan, static_cast<unsigned long long>(__popc(rs)));
    if (po) atomicAdd(c + kCntPolish, static_cast<unsigned long long>(__popc(po)));
    if (nf) {
      atomicAdd(c + kCntNonFinite, static_cast<unsigned long long>(__popc(nf)));
      atomicOr(a.err, kErrNonFinite);
    }
    if (bd) atomicOr(a.err, kErrExtrema);
  }
}

// ---------------------------------------------------------------------------
// Bounded double-buffered staging of source tiles. issue(t) queues tile t on
// mbarrier t & 1; body(buffer, tile) consumes it. Returns false if a copy
// never landed (error word set); the decision is block-uniform.
template <typename Issue, typename Body>
__device__ __forceinline__ bool staged_loop(int ntiles, uint64_t *bar, int32_t *err,
                                            Issue issue, Body body,
                                            unsigned long long limit_ns = 2000000000ull) {
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (ntiles > 0) issue(0);
    if (ntiles > 1) issue(1);
  }
  for (int t = 0; t < ntiles; ++t) {
    const int b = t & 1;
    const bool ok = mbar_wait_bounded(&bar[b], (t >> 1) & 1, err, limit_ns);
    if (ok) body(b, t);
    // every warp is done with buffer b; a failed wait anywhere stops all
    if (!__syncthreads_and(ok)) {
      if (threadIdx.x == 0) drain_copies(bar, t, ntiles, limit_ns);
      __syncthreads();
      return false;
    }
    if (threadIdx.x == 0 && t + 2 < ntiles) {
      proxy_fence_shared();
      issue(t + 2);
    }
  }
  // every phase is complete: the barriers may be initialised again (the
  // persistent kernel stages every step)
  if (threadIdx.x == 0) {
    mbar_inval(&bar[0]);
    mbar_inval(&bar[1]);
  }
  return true;
}

// After the pair loop the staging bytes hold the warp partials and then the
// update state.
template <typename R>
constexpr size_t epi_bytes(int warps) {
  return static_cast<size_t>(warps) * (sizeof(R) == 4 ? 6 : 12) * kTargets * sizeof(float) +
         sizeof(EpiShared<R>) + 64;
}

// Split partials of one FP32 item of 32 targets: (sum, error) of 3 components.
// The buffer is sized for the FP64 kernel's 6 doubles per target.
constexpr int kPartF32 = 6 * kTargets;

// The sums of a split target group for one lane's target: part by part in
// split order, per component the Neumaier sum of the parts' sums and then
// their compensations added. Part q's six floats (three sums, three
// compensations, each 32 lanes wide) start at base + q stride. The loads of
// four parts are issued before any of them is added, so that one L2 round
// trip, not one per part, precedes every four.
__device__ __forceinline__ void combine_split(const float *base, size_t stride, int nsplit,
                                              int lane, float *hi, float *lo) {
  float s[3] = {0.f, 0.f, 0.f}, e[3] = {0.f, 0.f, 0.f};
#pragma unroll 1
  for (int q0 = 0; q0 < nsplit; q0 += 4) {
    float v[4][6];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int k = 0; k < 6; ++k)
        v[u][k] = q0 + u < nsplit ? __ldcg(base + (q0 + u) * stride + k * 32 + lane) : 0.f;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (q0 + u >= nsplit) break;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        neumaier_add(s[c], e[c], v[u][c]);
        e[c] += v[u][3 + c];
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    hi[c] = s[c];
    lo[c] = e[c];
  }
}

// KMC_DEBUG builds: the block's work item lies inside the launch, its
// lysosome and that lysosome's target and source ranges (records of NPs:
// pairs in FP32, single NPs in FP64), and its part index is consistent; a
// failed check skips the block. Release builds compile this to `true`.
__device__ __forceinline__ bool item_in_bounds(const StepArgs &a, int tpl, bool fp32) {
#ifdef KMC_DEBUG
  if (!KMC_DCHECK(static_cast<int>(blockIdx.x) < a.n_items, a.err, kSiteItem)) return false;
  const Item it = a.items[blockIdx.x];
  if (!KMC_DCHECK(it.l >= 0 && it.l < a.n_lys, a.err, kSiteLys)) return false;
  const LysDev L = a.lys[it.l];
  if (!KMC_DCHECK(it.off == L.off && it.roff == L.roff, a.err, kSiteLys)) return false;
  if (!KMC_DCHECK(it.t0 >= 0 && it.nt >= 1 && it.nt <= kTargets * tpl && it.t0 + it.nt <= L.n,
                  a.err, kSiteTargets))
    return false;
  const int nrec = fp32 ? (L.n + 1) / 2 : L.n;
  if (!KMC_DCHECK(it.j0 >= 0 && it.j0 < it.j1 && it.j1 <= nrec, a.err, kSiteSources))
    return false;
  if (!KMC_DCHECK(it.nsplit >= 1 && it.split >= 0 && it.split < it.nsplit && it.gid >= 0 &&
                      static_cast<int>(blockIdx.x) >= it.split,
                  a.err, kSiteSplit))
    return false;
#endif
  return true;
}

// KMC_DEBUG builds: tile t of an item covers records r0 .. r0 + cnt - 1 inside
// the item's range and fits the staging buffer.
__device__ __forceinline__ bool tile_in_bounds(const StepArgs &a, const Item &it, int r0, int cnt,
                                               int tile) {
  return KMC_DCHECK(r0 >= it.j0 && cnt >= 1 && cnt <= tile && r0 + cnt <= it.j1, a.err,
                    kSiteTile);
}

// ---------------------------------------------------------------------------
// FP32-mixed step kernel.
// CL: the two source parts of every target group run as the two CTAs of a
// thread-block cluster (rank = part); part 1 hands its combined sums to part
// 0 through distributed shared memory instead of global memory, fences and an
// arrival counter, and part 0 adds them in split order (the same operations,
// so the same bits) and runs the update. Every thread of both CTAs passes the
// same two cluster barriers, on the failure paths too.
// One step of the block's work item (kmc_step_f32 runs it once per launch,
// kmc_persist_f32 once per step of a field period). PERSIST: the state of the
// previous step is already visible (a grid barrier), so there is no
// programmatic-launch wait. Returns early for items whose group is finished by
// another item.
template <int NW, bool CL, bool PERSIST>
__device__ __forceinline__ void step_f32_item(const StepArgs &a, int tile, unsigned char *smem,
                                              int &s_last, GridTables<float> &tab) {
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  unsigned char *dyn = smem + 16;
  if (!item_in_bounds(a, 1, true) ||
      (CL && !KMC_DCHECK(a.items[blockIdx.x].nsplit == 2 &&
                             static_cast<int>(blockIdx.x & 1) == a.items[blockIdx.x].split,
                         a.err, kSiteSplit))) {
    if constexpr (CL) {
      cluster_sync();
      cluster_sync();
    }
    return;
  }
  const Item it = a.items[blockIdx.x];
  const LysDev L = a.lys[it.l];  // for the update; positions and sources use it.off, it.roff
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // items, lysosome constants and positions do not change during a run
  const float4 pi = static_cast<const float4 *>(a.pos)[it.off + it.t0 + min(lane, it.nt - 1)];
  // The run state changes only between field periods (the period advance, or
  // a copy before a run), never across a programmatic-launch edge: a period's
  // step launches follow one another inside its graph, and the graph starts
  // after the previous one, advance included, has completed. So it is read
  // before the wait, and the first tile's copy follows the wait at once.
  const long long step = a.rs->step_base + a.k_local;
  const int per = a.rs->period;
  if constexpr (!PERSIST) grid_dependency_wait();
  const int rec = (per >= a.discard) ? (per - a.discard) * a.S + a.k_local : -1;
  const int par = static_cast<int>(step & 1);
  const SrcPair *__restrict__ gsrc = static_cast<const SrcPair *>(a.src[par]) + it.roff;

  TargetIn<float4> tin;
  if (warp == 0) tin = load_target<float4>(a, L, it, step, lane);
  const f2 X = pk(pi.x, pi.x), Y = pk(pi.y, pi.y), Z = pk(pi.z, pi.z);
  float s3[3] = {0.f, 0.f, 0.f}, c3[3] = {0.f, 0.f, 0.f};
  const int nrec = it.j1 - it.j0;
  const int ntiles = (nrec + tile - 1) / tile;
  const int own0 = it.t0 >> 1, own1 = (it.t0 + it.nt - 1) >> 1;  // records holding targets
  ulonglong2 *buf = reinterpret_cast<ulonglong2 *>(dyn);          // [2][tile][kRecU2]
  auto issue = [&](int t) {
    const int b = t & 1;
    const int r0 = it.j0 + t * tile;
    const int cnt = min(tile, it.j1 - r0);
    // tile 0 also brings the grid tables (the persistent kernel loads them
    // once), so that no thread waits on them
    const uint32_t tab_bytes =
        (!PERSIST && t == 0) ? sizeof(tab.sc) + sizeof(tab.th) + sizeof(tab.ss) + sizeof(tab.cc) : 0;
    const bool ok = tile_in_bounds(a, it, r0, cnt, tile);  // else no tile: the error is set
    const uint32_t bytes = ok ? static_cast<uint32_t>(cnt) * sizeof(SrcPair) : 0;
    mbar_expect_tx(&bar[b], bytes + tab_bytes);
    if (tab_bytes) {
      bulk_g2s(tab.sc, g_sc_f, sizeof(tab.sc), &bar[b]);
      bulk_g2s(tab.th, g_theta_f, sizeof(tab.th), &bar[b]);
      bulk_g2s(tab.ss, g_ss_f, sizeof(tab.ss), &bar[b]);
      bulk_g2s(tab.cc, g_cc_f, sizeof(tab.cc), &bar[b]);
    }
    if (ok) bulk_g2s(buf + static_cast<size_t>(b) * tile * kRecU2, gsrc + r0, bytes, &bar[b]);
  };
  auto body = [&](int b, int t) {
    const int r0 = it.j0 + t * tile;
    const int cnt = min(tile, it.j1 - r0);
    const bool mask = (r0 <= own1) && (own0 < r0 + cnt);
    const ulonglong2 *sp = buf + static_cast<size_t>(b) * tile * kRecU2;
    const AccF32 acc = mask ? pair_tile_f32<true>(sp, cnt, warp, NW, X, Y, Z)
                            : pair_tile_f32<false>(sp, cnt, warp, NW, X, Y, Z);
    kahan_add(s3[0], c3[0], hsum(acc.x));
    kahan_add(s3[1], c3[1], hsum(acc.y));
    kahan_add(s3[2], c3[2], hsum(acc.z));
  };
  if (!staged_loop(ntiles, bar, a.err, issue, body)) {
    if constexpr (CL) {
      cluster_sync();
      cluster_sync();
    }
    return;
  }

  // cross-warp combine in a fixed order: value = hi + lo per component
  float *wp = reinterpret_cast<float *>(dyn);  // [NW][6][32]
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    wp[(warp * 6 + c) * 32 + lane] = s3[c];
    wp[(warp * 6 + 3 + c) * 32 + lane] = -c3[c];  // Kahan keeps minus the error
  }
  __syncthreads();
  EpiShared<float> &sm =
      *reinterpret_cast<EpiShared<float> *>(dyn + static_cast<size_t>(NW) * 6 * 32 * 4);
  float hi[3], lo[3];
  if (warp == 0) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float s = 0.f, e = 0.f;
      for (int w = 0; w < NW; ++w) {
        neumaier_add(s, e, wp[(w * 6 + c) * 32 + lane]);
        e += wp[(w * 6 + 3 + c) * 32 + lane];
      }
      hi[c] = s;
      lo[c] = e;
    }
    if (!CL && it.nsplit > 1) {
      float *part = a.partial + static_cast<size_t>(blockIdx.x) * kPartF32;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        __stcg(part + c * 32 + lane, hi[c]);
        __stcg(part + (3 + c) * 32 + lane, lo[c]);
      }
    }
  }
  if constexpr (CL) {
    __shared__ float s_xch[6][kTargets];  // part 1's (sum, error) per component
    if (warp == 0 && it.split == 1) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        s_xch[c][lane] = hi[c];
        s_xch[3 + c][lane] = lo[c];
      }
    }
    cluster_sync();
    if (warp == 0 && it.split == 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float s = 0.f, e = 0.f;
        neumaier_add(s, e, hi[c]);
        e += lo[c];
        neumaier_add(s, e, ld_cluster(&s_xch[c][lane], 1));
        e += ld_cluster(&s_xch[3 + c][lane], 1);
        hi[c] = s;
        lo[c] = e;
      }
    }
    cluster_sync();  // part 0 has read part 1's shared memory
    if (it.split != 0) return;
  } else if (it.nsplit > 1) {
    // another item of the group finishes the step
    if (!arrive_last(&a.arrivals[it.gid], it.nsplit, &s_last)) return;
    if (warp == 0) {
      combine_split(a.partial + static_cast<size_t>(blockIdx.x - it.split) * kPartF32, kPartF32,
                    it.nsplit, lane, hi, lo);
      if (lane == 0) a.arrivals[it.gid] = 0;  // ready for the next launch
    }
  }
  if (warp == 0) {
#pragma unroll
    for (int c = 0; c < 3; ++c) sm.h[c][lane] = hi[c] + lo[c];  // compensation added last
  }
  __syncthreads();
  block_update<float4, true>(a, L, it, step, rec, tin, sm, tab);
}

template <int NW, bool CL = false>
__global__ void __launch_bounds__(NW * 32) kmc_step_f32(const StepArgs a, int tile) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_last;
  __shared__ __align__(16) GridTables<float> tab;  // copied in bulk with the first tile
  step_f32_item<NW, CL, false>(a, tile, smem, s_last, tab);
  // the next step's blocks may now be scheduled; triggering earlier lets them
  // take the slots of early-finishing blocks and unbalances the next step
  grid_launch_dependents();
}

// Persistent form of kmc_step_f32 (one target per lane): one cooperative
// launch runs a whole field period. Every block keeps its work item and runs
// steps 0 .. S - 1, with a bounded grid barrier after each step in place of
// the launch boundary; the step is the same code with the same cosine, so the
// results are the bits of the per-step launches. A barrier that times out
// sets KMC_ETIMEOUT in the error word and every block leaves the period.
template <int NW>
__global__ void __launch_bounds__(NW * 32) kmc_persist_f32(const StepArgs a, int tile) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_last;
  __shared__ int s_ok;
  __shared__ GridTables<float> tab;
  __shared__ StepArgs sa;  // a with this step's k_local and cos_k
  tab.load();
  if (threadIdx.x == 0) sa = a;
#pragma unroll 1
  for (int k = 0; k < a.S; ++k) {
    if (threadIdx.x == 0) {
      sa.k_local = k;
      sa.cos_k = a.cosk[k];
    }
    __syncthreads();
    step_f32_item<NW, false, true>(sa, tile, smem, s_last, tab);
    const bool skip = a.stall_block == static_cast<int>(blockIdx.x) && a.stall_step == k;
    if (!grid_barrier(a.gbar, gridDim.x, a.err, a.barrier_ns, skip, &s_ok)) break;
  }
}

// ---------------------------------------------------------------------------
// FP32-mixed step with TPL targets per lane (2 or 3): the block takes a group
// of 32 TPL targets, lane t holding targets t0 + t, t0 + 32 + t, ..., so that
// every staged source record feeds TPL independent chains. Each target's sums
// are formed by the same packed operations over the same records as in
// kmc_step_f32, and the warps and source parts are combined in the same order,
// so the fields, and hence the whole step, are the same bits. The 32-target
// parts of the group then run steps iii-vii with the same update code: side
// by side, each on its own group of warps, when the warps divide evenly among
// the parts (two or more each), else one after the other on the whole block.
template <int TPL>
struct AccF32N {
  AccF32 t[TPL];  // the lane's targets, in order
};

// The loops for two and three targets take their targets' positions as
// separate arguments, each record feeding every target in turn. Unlike the
// one-target loop they are inlined: out of line, the call's argument passing
// held 122 (two targets) and 164 (three) registers where inlined they take 107
// and 128, and the 50 000-NP and 512-lysosome workloads ran 5-6 % faster. The
// two-target loop is unrolled eight times, held at 4 blocks of 4 warps per SM
// (127 registers, no spill): against twice, -1.6 % per step at 8 x 2000 NPs
// and -4.5 % at 50 000 NPs; four times lies between, once was 8 % slower. The
// three-target loop is not unrolled (its three chains suffice).
template <bool MASK>
__device__ __forceinline__ AccF32N<2> pair_tile_f32_2t(const ulonglong2 *__restrict__ sp, int cnt,
                                                       int first, int stride, f2 X0, f2 Y0, f2 Z0,
                                                       f2 X1, f2 Y1, f2 Z1) {
  AccF32N<2> acc;
  acc.t[0].x = acc.t[0].y = acc.t[0].z = 0ull;
  acc.t[1] = acc.t[0];
#pragma unroll 8
  for (int r = first; r < cnt; r += stride) {
    ulonglong2 a, b, c, d;
    f2 e;
    load_record(sp, r, a, b, c, d, e);
    pair_record<MASK>(a, b, c, d, e, X0, Y0, Z0, acc.t[0]);
    pair_record<MASK>(a, b, c, d, e, X1, Y1, Z1, acc.t[1]);
  }
  return acc;
}

template <bool MASK>
__device__ __forceinline__ AccF32N<3> pair_tile_f32_3t(const ulonglong2 *__restrict__ sp, int cnt,
                                                    int first, int stride, f2 X0, f2 Y0, f2 Z0,
                                                    f2 X1, f2 Y1, f2 Z1, f2 X2, f2 Y2, f2 Z2) {
  AccF32N<3> acc;
  acc.t[0].x = acc.t[0].y = acc.t[0].z = 0ull;
  acc.t[1] = acc.t[0];
  acc.t[2] = acc.t[0];
#pragma unroll 1
  for (int r = first; r < cnt; r += stride) {
    ulonglong2 a, b, c, d;
    f2 e;
    load_record(sp, r, a, b, c, d, e);
    pair_record<MASK>(a, b, c, d, e, X0, Y0, Z0, acc.t[0]);
    pair_record<MASK>(a, b, c, d, e, X1, Y1, Z1, acc.t[1]);
    pair_record<MASK>(a, b, c, d, e, X2, Y2, Z2, acc.t[2]);
  }
  return acc;
}

// Warps that update each 32-target part of the multi-target kernel when its
// parts update side by side (two or more warps per part), else 0: the parts
// update in turn on the whole block.
constexpr int tn_group(int warps, int tpl) {
  return (warps % tpl == 0 && warps / tpl >= 2) ? warps / tpl : 0;
}

// Dynamic shared memory of the multi-target kernel after its pair loop: the
// warps' (sum, -error) pairs of every target, then the update state (one per
// part when the parts update side by side).
constexpr size_t epi_bytes_tn(int warps, int tpl) {
  return static_cast<size_t>(warps) * 6 * tpl * kTargets * sizeof(float) +
         (tn_group(warps, tpl) ? tpl : 1) * sizeof(EpiShared<float>) + 64;
}

// Four warps: held at 4 blocks per SM (128 registers).
template <int NW, int TPL>
__global__ void __launch_bounds__(NW * 32, NW == 4 ? 4 : 0)
    kmc_step_f32_tn(const StepArgs a, int tile) {
  static_assert(TPL == 2 || TPL == 3, "two or three targets per lane");
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  unsigned char *dyn = smem + 16;
  __shared__ int s_last;
  // the update's grid tables: two bulk copies on the first tile's barrier
  __shared__ __align__(16) GridTables<float> tab;
  __shared__ float s_hr[TPL - 1][3][kTargets];  // later parts' fields while the first updates
  if (!item_in_bounds(a, TPL, true)) return;
  const Item it = a.items[blockIdx.x];
  const LysDev L = a.lys[it.l];  // for the update; positions and sources use it.off, it.roff
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int ntk[TPL];  // targets of each 32-target part
#pragma unroll
  for (int k = 0; k < TPL; ++k) ntk[k] = min(max(it.nt - k * kTargets, 0), kTargets);
  const float4 *pos = static_cast<const float4 *>(a.pos);
  f2 X[TPL], Y[TPL], Z[TPL];
  {
    const float4 p0 = pos[it.off + it.t0 + min(lane, ntk[0] - 1)];
#pragma unroll
    for (int k = 0; k < TPL; ++k) {
      const float4 p =
          ntk[k] > 0 ? pos[it.off + it.t0 + k * kTargets + min(lane, ntk[k] - 1)] : p0;
      X[k] = pk(p.x, p.x);
      Y[k] = pk(p.y, p.y);
      Z[k] = pk(p.z, p.z);
    }
  }
  // The run state changes only between field periods (the period advance, or
  // a copy before a run), never across a programmatic-launch edge: a period's
  // step launches follow one another inside its graph, and the graph starts
  // after the previous one, advance included, has completed. So it is read
  // before the wait, and the first tile's copy follows the wait at once.
  const long long step = a.rs->step_base + a.k_local;
  const int per = a.rs->period;
  grid_dependency_wait();
  const int rec = (per >= a.discard) ? (per - a.discard) * a.S + a.k_local : -1;
  const int par = static_cast<int>(step & 1);
  const SrcPair *__restrict__ gsrc = static_cast<const SrcPair *>(a.src[par]) + it.roff;

  // the part whose update this warp runs, and whether it leads it (holds the
  // part's inputs and combines its sums)
  constexpr int kGrp = tn_group(NW, TPL);
  const int gk = kGrp ? warp / kGrp : 0;
  const bool lead = kGrp ? (warp % kGrp == 0) : (warp == 0);
  Item h0 = it;
  h0.t0 = it.t0 + gk * kTargets;
  h0.nt = ntk[gk];
  TargetIn<float4> tin;
  if (lead && h0.nt > 0) tin = load_target<float4>(a, L, h0, step, lane);
  float sk[3 * TPL], ck[3 * TPL];  // Kahan sums: target k, component c at 3 k + c
#pragma unroll
  for (int c = 0; c < 3 * TPL; ++c) sk[c] = ck[c] = 0.f;
  const int nrec = it.j1 - it.j0;
  const int ntiles = (nrec + tile - 1) / tile;
  const int own0 = it.t0 >> 1, own1 = (it.t0 + it.nt - 1) >> 1;  // records holding targets
  ulonglong2 *buf = reinterpret_cast<ulonglong2 *>(dyn);          // [2][tile][kRecU2]
  auto issue = [&](int t) {
    const int b = t & 1;
    const int r0 = it.j0 + t * tile;
    const int cnt = min(tile, it.j1 - r0);
    // tile 0 also brings the grid tables, so that no thread waits on them
    const uint32_t tab_bytes =
        t == 0 ? sizeof(tab.sc) + sizeof(tab.th) + sizeof(tab.ss) + sizeof(tab.cc) : 0;
    const bool ok = tile_in_bounds(a, it, r0, cnt, tile);  // else no tile: the error is set
    const uint32_t bytes = ok ? static_cast<uint32_t>(cnt) * sizeof(SrcPair) : 0;
    mbar_expect_tx(&bar[b], bytes + tab_bytes);
    if (tab_bytes) {
      bulk_g2s(tab.sc, g_sc_f, sizeof(tab.sc), &bar[b]);
      bulk_g2s(tab.th, g_theta_f, sizeof(tab.th), &bar[b]);
      bulk_g2s(tab.ss, g_ss_f, sizeof(tab.ss), &bar[b]);
      bulk_g2s(tab.cc, g_cc_f, sizeof(tab.cc), &bar[b]);
    }
    if (ok) bulk_g2s(buf + static_cast<size_t>(b) * tile * kRecU2, gsrc + r0, bytes, &bar[b]);
  };
  auto body = [&](int b, int t) {
    const int r0 = it.j0 + t * tile;
    const int cnt = min(tile, it.j1 - r0);
    const bool mask = (r0 <= own1) && (own0 < r0 + cnt);
    const ulonglong2 *sp = buf + static_cast<size_t>(b) * tile * kRecU2;
    AccF32N<TPL> acc;
    if constexpr (TPL == 2) {
      acc = mask ? pair_tile_f32_2t<true>(sp, cnt, warp, NW, X[0], Y[0], Z[0], X[1], Y[1], Z[1])
                 : pair_tile_f32_2t<false>(sp, cnt, warp, NW, X[0], Y[0], Z[0], X[1], Y[1], Z[1]);
    } else {
      acc = mask ? pair_tile_f32_3t<true>(sp, cnt, warp, NW, X[0], Y[0], Z[0], X[1], Y[1], Z[1],
                                          X[2], Y[2], Z[2])
                 : pair_tile_f32_3t<false>(sp, cnt, warp, NW, X[0], Y[0], Z[0], X[1], Y[1], Z[1],
                                           X[2], Y[2], Z[2]);
    }
#pragma unroll
    for (int k = 0; k < TPL; ++k) {
      kahan_add(sk[3 * k + 0], ck[3 * k + 0], hsum(acc.t[k].x));
      kahan_add(sk[3 * k + 1], ck[3 * k + 1], hsum(acc.t[k].y));
      kahan_add(sk[3 * k + 2], ck[3 * k + 2], hsum(acc.t[k].z));
    }
  };
  if (!staged_loop(ntiles, bar, a.err, issue, body)) return;

  // cross-warp combine in a fixed order, per target as in kmc_step_f32
  constexpr int kW = 6 * TPL;                  // floats per lane and warp
  float *wp = reinterpret_cast<float *>(dyn);  // [NW][6 TPL][32]: 3 TPL sums, then 3 TPL errors
#pragma unroll
  for (int c = 0; c < 3 * TPL; ++c) {
    wp[(warp * kW + c) * 32 + lane] = sk[c];
    wp[(warp * kW + 3 * TPL + c) * 32 + lane] = -ck[c];
  }
  __syncthreads();
  EpiShared<float> *sms =
      reinterpret_cast<EpiShared<float> *>(dyn + static_cast<size_t>(NW) * kW * 32 * 4);
  if constexpr (kGrp > 0) {
    // each part's lead warp combines the part's sums in kmc_step_f32's order;
    // the groups then run steps iii-vii side by side
    EpiShared<float> &sm = sms[gk];
    float hi[3], lo[3];
    if (lead) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float s = 0.f, e = 0.f;
        for (int w = 0; w < NW; ++w) {
          neumaier_add(s, e, wp[(w * kW + 3 * gk + c) * 32 + lane]);
          e += wp[(w * kW + 3 * TPL + 3 * gk + c) * 32 + lane];
        }
        hi[c] = s;
        lo[c] = e;
      }
      if (it.nsplit > 1) {
        float *part = a.partial + (static_cast<size_t>(blockIdx.x) * TPL + gk) * kPartF32;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          __stcg(part + c * 32 + lane, hi[c]);
          __stcg(part + (3 + c) * 32 + lane, lo[c]);
        }
      }
    }
    if (it.nsplit > 1) {
      if (!arrive_last(&a.arrivals[it.gid], it.nsplit, &s_last)) return;
      if (lead) {
        combine_split(a.partial + (static_cast<size_t>(blockIdx.x - it.split) * TPL + gk) * kPartF32,
                      TPL * kPartF32, it.nsplit, lane, hi, lo);
      }
      if (threadIdx.x == 0) a.arrivals[it.gid] = 0;  // ready for the next launch
    }
    if (lead) {
#pragma unroll
      for (int c = 0; c < 3; ++c) sm.h[c][lane] = hi[c] + lo[c];
    }
    if (h0.nt > 0) block_update<float4, true, false, kGrp>(a, L, h0, step, rec, tin, sm, tab, gk);
    grid_launch_dependents();
    return;
  }
  EpiShared<float> &sm = sms[0];
  float hi[3 * TPL], lo[3 * TPL];
  if (warp == 0) {
#pragma unroll
    for (int c = 0; c < 3 * TPL; ++c) {
      float s = 0.f, e = 0.f;
      for (int w = 0; w < NW; ++w) {
        neumaier_add(s, e, wp[(w * kW + c) * 32 + lane]);
        e += wp[(w * kW + 3 * TPL + c) * 32 + lane];
      }
      hi[c] = s;
      lo[c] = e;
    }
    if (it.nsplit > 1) {
      // every part's partials, each laid out as kmc_step_f32's
      float *part = a.partial + static_cast<size_t>(blockIdx.x) * TPL * kPartF32;
#pragma unroll
      for (int k = 0; k < TPL; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          __stcg(part + k * kPartF32 + c * 32 + lane, hi[3 * k + c]);
          __stcg(part + k * kPartF32 + (3 + c) * 32 + lane, lo[3 * k + c]);
        }
    }
  }
  if (it.nsplit > 1) {
    // another item of the group finishes the step
    if (!arrive_last(&a.arrivals[it.gid], it.nsplit, &s_last)) return;
    if (warp == 0) {
      const float *base = a.partial + static_cast<size_t>(blockIdx.x - it.split) * TPL * kPartF32;
#pragma unroll
      for (int k = 0; k < TPL; ++k)
        combine_split(base + k * kPartF32, TPL * kPartF32, it.nsplit, lane, hi + 3 * k, lo + 3 * k);
      if (lane == 0) a.arrivals[it.gid] = 0;  // ready for the next launch
    }
  }
  if (warp == 0) {
    // the first part's field; the others' wait in shared memory
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      sm.h[c][lane] = hi[c] + lo[c];
#pragma unroll
      for (int k = 1; k < TPL; ++k) s_hr[k - 1][c][lane] = hi[3 * k + c] + lo[3 * k + c];
    }
  }
  __syncthreads();
  block_update<float4, true>(a, L, h0, step, rec, tin, sm, tab);
#pragma unroll 1
  for (int k = 1; k < TPL; ++k) {
    if (ntk[k] == 0) break;
    __syncthreads();
    Item hk = it;
    hk.t0 = it.t0 + k * kTargets;
    hk.nt = ntk[k];
    if (warp == 0) {
      tin = load_target<float4>(a, L, hk, step, lane);
#pragma unroll
      for (int c = 0; c < 3; ++c) sm.h[c][lane] = s_hr[k - 1][c][lane];
    }
    __syncthreads();
    block_update<float4, true>(a, L, hk, step, rec, tin, sm, tab);
  }
  grid_launch_dependents();
}

// ---------------------------------------------------------------------------
// FP32-mixed step for RPL replicas: consecutive lysosomes l, l + 1, ..., l +
// RPL - 1 that share their geometry and material (the same NPs, axes and
// volumes; seeds of one sample) and differ only in their random streams,
// amplitudes and moments. The block has RPL warps and takes 32 targets of
// every replica. Each staged record's geometry (d, r^2, rsqrt, q^2, q^3) is
// formed once and serves all replicas, which add only their own terms
// u = (t.d) q^2 and q^3 (u d + n): 8 + 10 RPL packed operations per record and
// target instead of 18 RPL. Every replica's sums are formed by the same
// operations in the same order as in kmc_step_f32 with NW = RPL WPR warps,
// and the first warp of group r (warps r WPR .. r WPR + WPR - 1) combines
// replica r's warp sums and source parts in kmc_step_f32's order, so each
// replica's field, and its whole step, are the bits it gets alone. Group r
// then runs replica r's steps iii-vii (the groups in parallel): one warp by
// itself (WPR = 1), or two or four warps block-cooperatively on named
// barriers (WPR = 2, 4), which keeps the update's latency near that of one
// block.
template <bool MASK, int RPL, int NW>
__device__ __forceinline__ void pair_tile_f32_rep(const ulonglong2 *__restrict__ sp,
                                                  size_t rstride, int cnt, int first, f2 X,
                                                  f2 Y, f2 Z, AccF32 (&acc)[RPL]) {
#pragma unroll 1
  for (int r = first; r < cnt; r += NW) {
    ulonglong2 a0, b0, c0, d0;
    f2 e0;
    load_record(sp, r, a0, b0, c0, d0, e0);
    const f2 dx = sub2(a0.x, X), dy = sub2(a0.y, Y), dz = sub2(b0.x, Z);
    const f2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
    float r2l, r2h;
    upk(r2, r2l, r2h);
    float il = rsqrt_approx(r2l), ih = rsqrt_approx(r2h);
    if (MASK) {
      il = (r2l > 0.0f) ? il : 0.0f;
      ih = (r2h > 0.0f) ? ih : 0.0f;
    }
    const f2 q = pk(il, ih);
    const f2 q2 = mul2(q, q);
    const f2 q3 = mul2(q, q2);
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
      // replica k's moment words of the same record: z | nx, ny | nz, tx | ty, tz | -
      const ulonglong2 *p = sp + k * rstride + kRecU2 * r;
      const ulonglong2 b = p[1], c = p[2], d = p[3];
      const f2 e = reinterpret_cast<const f2 *>(p + 4)[0];
      const f2 u = mul2(fma2(e, dz, fma2(d.y, dy, mul2(d.x, dx))), q2);
      acc[k].x = fma2(q3, fma2(u, dx, b.y), acc[k].x);
      acc[k].y = fma2(q3, fma2(u, dy, c.x), acc[k].y);
      acc[k].z = fma2(q3, fma2(u, dz, c.y), acc[k].z);
    }
  }
}

// Dynamic shared memory of the replica kernel after its pair loop: the warps'
// (sum, -error) pairs of every replica, then every replica's update state.
constexpr size_t epi_bytes_rep(int rpl, int nw) {
  return static_cast<size_t>(nw) * 6 * rpl * kTargets * sizeof(float) +
         static_cast<size_t>(rpl) * sizeof(EpiShared<float>) + 64;
}

template <int RPL, int WPR = 1>
__global__ void __launch_bounds__(RPL * WPR * 32, (RPL == 2 && WPR == 4) ? 2 : 0)
    kmc_step_f32_rep(const StepArgs a, int tile) {
  static_assert(RPL == 2 || RPL == 4, "two or four replicas per lane");
  static_assert(WPR == 1 || WPR == 2 || WPR == 4, "one, two or four warps per replica");
  constexpr int NW = RPL * WPR;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  unsigned char *dyn = smem + 16;
  __shared__ int s_last;
  // the update's grid tables: two bulk copies on the first tile's barrier
  __shared__ __align__(16) GridTables<float> tab;
  if (!item_in_bounds(a, 1, true)) return;
  const Item it = a.items[blockIdx.x];  // it.l: the first replica
  if (!KMC_DCHECK(it.l + RPL <= a.n_lys, a.err, kSiteLys)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rk = WPR == 1 ? warp : warp / WPR;        // the replica this warp's group updates
  const bool lead = WPR == 1 || warp % WPR == 0;      // the group's first warp
  const LysDev Lw = a.lys[it.l + rk];
  const float4 pi = static_cast<const float4 *>(a.pos)[it.off + it.t0 + min(lane, it.nt - 1)];
  int roff[RPL];  // every replica's first source record
#pragma unroll
  for (int k = 0; k < RPL; ++k) roff[k] = a.lys[it.l + k].roff;
  // The run state changes only between field periods, never across a
  // programmatic-launch edge (as in kmc_step_f32): read before the wait.
  const long long step = a.rs->step_base + a.k_local;
  const int per = a.rs->period;
  grid_dependency_wait();
  const int rec = (per >= a.discard) ? (per - a.discard) * a.S + a.k_local : -1;
  const int par = static_cast<int>(step & 1);
  const SrcPair *__restrict__ gsrc = static_cast<const SrcPair *>(a.src[par]);

  Item iw = it;
  iw.l = it.l + rk;
  const TargetIn<float4> tin = load_target<float4>(a, Lw, iw, step, lane);
  const f2 X = pk(pi.x, pi.x), Y = pk(pi.y, pi.y), Z = pk(pi.z, pi.z);
  float sk[3 * RPL], ck[3 * RPL];  // Kahan sums: replica k, component c at 3 k + c
#pragma unroll
  for (int c = 0; c < 3 * RPL; ++c) sk[c] = ck[c] = 0.f;
  const int nrec = it.j1 - it.j0;
  const int ntiles = (nrec + tile - 1) / tile;
  const int own0 = it.t0 >> 1, own1 = (it.t0 + it.nt - 1) >> 1;  // records holding targets
  ulonglong2 *buf = reinterpret_cast<ulonglong2 *>(dyn);  // [2][RPL][tile][kRecU2]
  const size_t rstride = static_cast<size_t>(tile) * kRecU2;
  auto issue = [&](int t) {
    const int b = t & 1;
    const int r0 = it.j0 + t * tile;
    const int cnt = min(tile, it.j1 - r0);
    // tile 0 also brings the grid tables, so that no thread waits on them
    const uint32_t tab_bytes =
        t == 0 ? sizeof(tab.sc) + sizeof(tab.th) + sizeof(tab.ss) + sizeof(tab.cc) : 0;
    const bool ok = tile_in_bounds(a, it, r0, cnt, tile);  // else no tile: the error is set
    const uint32_t bytes = ok ? static_cast<uint32_t>(cnt) * sizeof(SrcPair) : 0;
    mbar_expect_tx(&bar[b], RPL * bytes + tab_bytes);
    if (tab_bytes) {
      bulk_g2s(tab.sc, g_sc_f, sizeof(tab.sc), &bar[b]);
      bulk_g2s(tab.th, g_theta_f, sizeof(tab.th), &bar[b]);
      bulk_g2s(tab.ss, g_ss_f, sizeof(tab.ss), &bar[b]);
      bulk_g2s(tab.cc, g_cc_f, sizeof(tab.cc), &bar[b]);
    }
    if (!ok) return;
#pragma unroll
    for (int k = 0; k < RPL; ++k)
      bulk_g2s(buf + (static_cast<size_t>(b) * RPL + k) * rstride, gsrc + roff[k] + r0, bytes,
               &bar[b]);
  };
  auto body = [&](int b, int t) {
    const int r0 = it.j0 + t * tile;
    const int cnt = min(tile, it.j1 - r0);
    const bool mask = (r0 <= own1) && (own0 < r0 + cnt);
    const ulonglong2 *sp = buf + static_cast<size_t>(b) * RPL * rstride;
    AccF32 acc[RPL];
#pragma unroll
    for (int k = 0; k < RPL; ++k) acc[k].x = acc[k].y = acc[k].z = 0ull;
    if (mask)
      pair_tile_f32_rep<true, RPL, NW>(sp, rstride, cnt, warp, X, Y, Z, acc);
    else
      pair_tile_f32_rep<false, RPL, NW>(sp, rstride, cnt, warp, X, Y, Z, acc);
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
      kahan_add(sk[3 * k + 0], ck[3 * k + 0], hsum(acc[k].x));
      kahan_add(sk[3 * k + 1], ck[3 * k + 1], hsum(acc[k].y));
      kahan_add(sk[3 * k + 2], ck[3 * k + 2], hsum(acc[k].z));
    }
  };
  if (!staged_loop(ntiles, bar, a.err, issue, body)) return;

  // cross-warp combine in kmc_step_f32's order; group k's first warp combines
  // replica k
  constexpr int kW = 6 * RPL;
  float *wp = reinterpret_cast<float *>(dyn);  // [NW][6 RPL][32]: 3 RPL sums, then 3 RPL errors
#pragma unroll
  for (int c = 0; c < 3 * RPL; ++c) {
    wp[(warp * kW + c) * 32 + lane] = sk[c];
    wp[(warp * kW + 3 * RPL + c) * 32 + lane] = -ck[c];
  }
  __syncthreads();
  EpiShared<float> *sms =
      reinterpret_cast<EpiShared<float> *>(dyn + static_cast<size_t>(NW) * kW * 32 * 4);
  EpiShared<float> &sm = sms[rk];
  float hi[3] = {0.f, 0.f, 0.f}, lo[3] = {0.f, 0.f, 0.f};
  if (lead) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float s = 0.f, e = 0.f;
      for (int w = 0; w < NW; ++w) {
        neumaier_add(s, e, wp[(w * kW + 3 * rk + c) * 32 + lane]);
        e += wp[(w * kW + 3 * RPL + 3 * rk + c) * 32 + lane];
      }
      hi[c] = s;
      lo[c] = e;
    }
  }
  if (it.nsplit > 1) {
    // replica k's partials at k kPartF32, each laid out as kmc_step_f32's
    if (lead) {
      float *part = a.partial + (static_cast<size_t>(blockIdx.x) * RPL + rk) * kPartF32;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        __stcg(part + c * 32 + lane, hi[c]);
        __stcg(part + (3 + c) * 32 + lane, lo[c]);
      }
    }
    // another item of the group finishes the step
    if (!arrive_last(&a.arrivals[it.gid], it.nsplit, &s_last)) return;
    if (lead) {
      combine_split(a.partial + (static_cast<size_t>(blockIdx.x - it.split) * RPL + rk) * kPartF32,
                    RPL * kPartF32, it.nsplit, lane, hi, lo);
    }
    __syncthreads();
    if (threadIdx.x == 0) a.arrivals[it.gid] = 0;  // ready for the next launch
  }
  if (lead) {
#pragma unroll
    for (int c = 0; c < 3; ++c) sm.h[c][lane] = hi[c] + lo[c];  // compensation added last
  }
  if constexpr (WPR == 1) {
    __syncwarp();
    block_update<float4, true, true>(a, Lw, iw, step, rec, tin, sm, tab);
  } else {
    block_update<float4, true, false, WPR>(a, Lw, iw, step, rec, tin, sm, tab, rk);
  }
  grid_launch_dependents();
}

// ---------------------------------------------------------------------------
// FP64-plain step kernel (same structure, scalar FP64 pair loop).
template <int NW>
__global__ void __launch_bounds__(NW * 32) kmc_step_f64(const StepArgs a, int tile) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  unsigned char *dyn = smem + 16;
  __shared__ int s_last;
  __shared__ GridTables<double> tab;
  tab.load();
  if (!item_in_bounds(a, 1, false)) return;
  const Item it = a.items[blockIdx.x];
  const LysDev L = a.lys[it.l];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // items, lysosome constants and positions do not change during a run
  const dbl4 pi = static_cast<const dbl4 *>(a.pos)[L.off + it.t0 + min(lane, it.nt - 1)];
  grid_dependency_wait();
  const long long step = a.rs->step_base + a.k_local;
  const int per = a.rs->period;
  const int rec = (per >= a.discard) ? (per - a.discard) * a.S + a.k_local : -1;
  const int par = static_cast<int>(step & 1);
  const dbl4 *__restrict__ gpos = static_cast<const dbl4 *>(a.src_pos) + L.roff;
  const dbl4 *__restrict__ gmu = static_cast<const dbl4 *>(a.src[par]) + L.roff;

  TargetIn<dbl4> tin;
  if (warp == 0) tin = load_target<dbl4>(a, L, it, step, lane);
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  const int nrec = it.j1 - it.j0;
  const int ntiles = (nrec + tile - 1) / tile;
  dbl4 *spos = reinterpret_cast<dbl4 *>(dyn);  // [2][tile]
  dbl4 *smu = spos + 2 * tile;                 // [2][tile]
  auto issue = [&](int t) {
    const int b = t & 1;
    const int r0 = it.j0 + t * tile;
    const int cnt = min(tile, it.j1 - r0);
    if (!tile_in_bounds(a, it, r0, cnt, tile)) {
      mbar_expect_tx(&bar[b], 0);  // no copy: the phase completes, the error is set
      return;
    }
    const uint32_t bytes = static_cast<uint32_t>(cnt) * sizeof(dbl4);
    mbar_expect_tx(&bar[b], 2 * bytes + a.stall_tx);
    bulk_g2s(spos + b * tile, gpos + r0, bytes, &bar[b]);
    bulk_g2s(smu + b * tile, gmu + r0, bytes, &bar[b]);
  };
  auto body = [&](int b, int t) {
    const int r0 = it.j0 + t * tile;
    const int cnt = min(tile, it.j1 - r0);
    pair_tile_f64(spos + b * tile, smu + b * tile, cnt, warp, NW, pi.x, pi.y, pi.z, acc);
  };
  if (!staged_loop(ntiles, bar, a.err, issue, body,
                   a.stall_tx ? a.stall_wait_ns : 2000000000ull))
    return;

  double *wp = reinterpret_cast<double *>(dyn);  // [NW][6][32]
#pragma unroll
  for (int c = 0; c < 6; ++c) wp[(warp * 6 + c) * 32 + lane] = acc[c];
  __syncthreads();
  EpiShared<double> &sm =
      *reinterpret_cast<EpiShared<double> *>(dyn + static_cast<size_t>(NW) * 12 * 32 * 4);
  double tot[6];
  if (warp == 0) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      double s = 0.0;
      for (int w = 0; w < NW; ++w) s += wp[(w * 6 + c) * 32 + lane];
      tot[c] = s;
    }
    if (it.nsplit > 1) {
      double *part =
          reinterpret_cast<double *>(a.partial + static_cast<size_t>(blockIdx.x) * 12 * 32);
#pragma unroll
      for (int c = 0; c < 6; ++c) __stcg(part + c * 32 + lane, tot[c]);
    }
  }
  if (it.nsplit > 1) {
    if (!arrive_last(&a.arrivals[it.gid], it.nsplit, &s_last)) return;
    if (warp == 0) {
      const double *base = reinterpret_cast<const double *>(
          a.partial + static_cast<size_t>(blockIdx.x - it.split) * 12 * 32);
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        double s = 0.0;
        for (int q = 0; q < it.nsplit; ++q) s += __ldcg(base + (q * 6 + c) * 32 + lane);
        tot[c] = s;
      }
      if (lane == 0) a.arrivals[it.gid] = 0;
    }
  }
  if (warp == 0) {
#pragma unroll
    for (int c = 0; c < 3; ++c) sm.h[c][lane] = 3.0 * tot[c] - tot[3 + c];
  }
  __syncthreads();
  block_update<dbl4, false>(a, L, it, step, rec, tin, sm, tab);
  // the next step's blocks may now be scheduled; triggering earlier lets them
  // take the slots of early-finishing blocks and unbalances the next step
  grid_launch_dependents();
}

// Ends a field period on the device: the next period starts S steps later.
__global__ void kmc_advance_kernel(RunState *rs, int S) {
  rs->step_base += S;
  rs->period += 1;
}

// ---------------------------------------------------------------------------
// Symmetric pair form (FP32-mixed). T_ij and T_ji share their geometry (d,
// r^2, the rsqrt and the powers of 1/r), so each unordered pair is formed
// once for both of its ordered pairs.
//
// Field kernel: a block of W warps takes row group g, i.e. W C cells (warp w:
// cells g W C + w C .. + C - 1; lane L holds record L of each, two targets
// per cell), against the source cells [h0, h1) above the group, one staged
// cell at a time. At step s lane L reads record (L + s) mod 32 of the staged
// cell and forms, for each of its 2 C targets, the geometry of its two pairs
// (8 packed operations, two rsqrt), the forward terms into the target's sums
// (10) and the reverse terms into the sums it carries for that record (10).
// The reverse term of target i at source j is q^3 (v d + n_i) with
// v = (t_i . d) q^2 and d = r_j - r_i: -d enters twice. The reverse sums move
// one lane per step (shuffles), so that after 32 steps lane L holds those of
// record L; the W warps' sums of the cell are then added in warp order into
// the cell's reverse slot for row group g. The group's diagonal item
// evaluates the pairs inside the group in the ordered form instead (each
// warp: its targets against every record of the group, the self pair
// masked). Every sum runs in a fixed order, so results do not depend on the
// launch.
//
// Update kernel: each warp takes one update item, 32 targets of one cell: it
// adds, with compensation, the forward partials of the targets' row group
// (diagonal item first, then the source ranges in order) and the reverse
// slots of their cell (row groups in order), then runs steps iii-vii for its
// targets alone (the warp-level path of block_update, whose results are those
// of the block-cooperative one). The update is a separate kernel here, so its
// throughput, not its latency, counts: no warp waits while another sets up
// planes or decides.
constexpr int kSymUpdWarps = 4;

template <int T>
__device__ __forceinline__ void sym_cell(const ulonglong2 *__restrict__ sp, int lane,
                                         const f2 (&X)[T], const f2 (&Y)[T], const f2 (&Z)[T],
                                         const f2 (&TX)[T], const f2 (&TY)[T], const f2 (&TZ)[T],
                                         const f2 (&NX)[T], const f2 (&NY)[T], const f2 (&NZ)[T],
                                         AccF32 (&acc)[T], f2 &rx, f2 &ry, f2 &rz) {
  const int from = (lane + 1) & (kCellRec - 1);
#pragma unroll 2
  for (int s = 0; s < kCellRec; ++s) {
    ulonglong2 a, b, c, d;
    f2 e;
    load_record(sp, (lane + s) & (kCellRec - 1), a, b, c, d, e);
#pragma unroll
    for (int k = 0; k < T; ++k) {
      const f2 dx = sub2(a.x, X[k]), dy = sub2(a.y, Y[k]), dz = sub2(b.x, Z[k]);
      const f2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
      float r2l, r2h;
      upk(r2, r2l, r2h);
      const f2 q = pk(rsqrt_approx(r2l), rsqrt_approx(r2h));
      const f2 q2 = mul2(q, q);
      const f2 q3 = mul2(q, q2);
      const f2 u = mul2(fma2(e, dz, fma2(d.y, dy, mul2(d.x, dx))), q2);
      acc[k].x = fma2(q3, fma2(u, dx, b.y), acc[k].x);
      acc[k].y = fma2(q3, fma2(u, dy, c.x), acc[k].y);
      acc[k].z = fma2(q3, fma2(u, dz, c.y), acc[k].z);
      const f2 v = mul2(fma2(TZ[k], dz, fma2(TY[k], dy, mul2(TX[k], dx))), q2);
      rx = fma2(q3, fma2(v, dx, NX[k]), rx);
      ry = fma2(q3, fma2(v, dy, NY[k]), ry);
      rz = fma2(q3, fma2(v, dz, NZ[k]), rz);
    }
    rx = __shfl_sync(0xffffffffu, rx, from);
    ry = __shfl_sync(0xffffffffu, ry, from);
    rz = __shfl_sync(0xffffffffu, rz, from);
  }
}

// Ordered pairs of the lane's targets with the 32 records of one staged cell
// (diagonal items); MASK drops the self pair.
template <bool MASK, int T>
__device__ __forceinline__ void ordered_cell(const ulonglong2 *__restrict__ sp, const f2 (&X)[T],
                                             const f2 (&Y)[T], const f2 (&Z)[T],
                                             AccF32 (&acc)[T]) {
#pragma unroll 1
  for (int r = 0; r < kCellRec; ++r) {
    ulonglong2 a, b, c, d;
    f2 e;
    load_record(sp, r, a, b, c, d, e);
#pragma unroll
    for (int k = 0; k < T; ++k) pair_record<MASK>(a, b, c, d, e, X[k], Y[k], Z[k], acc[k]);
  }
}

// KMC_DEBUG builds: the block's symmetric item lies inside the launch and its
// lysosome, and its source cells lie above its row group.
__device__ __forceinline__ bool sym_item_in_bounds(const StepArgs &a, int gc) {
#ifdef KMC_DEBUG
  if (!KMC_DCHECK(static_cast<int>(blockIdx.x) < a.n_items, a.err, kSiteItem)) return false;
  const SymItem it = a.sitems[blockIdx.x];
  if (!KMC_DCHECK(it.l >= 0 && it.l < a.n_lys, a.err, kSiteLys)) return false;
  const int nc = (a.lys[it.l].n + kCell - 1) / kCell;
  if (!KMC_DCHECK(it.g >= 0 && it.g * gc < nc && it.fwd >= 0 && it.rbase >= 0, a.err,
                  kSiteTargets))
    return false;
  if (!KMC_DCHECK((it.h0 == -1 && it.h1 == -1) ||
                      (it.h0 >= (it.g + 1) * gc && it.h0 < it.h1 && it.h1 <= nc),
                  a.err, kSiteSources))
    return false;
#endif
  return true;
}

__device__ __forceinline__ bool sym_upd_in_bounds(const StepArgs &a, int gc, int ui) {
#ifdef KMC_DEBUG
  if (!KMC_DCHECK(ui < a.n_upd, a.err, kSiteItem)) return false;
  const SymUpd u = a.supd[ui];
  if (!KMC_DCHECK(u.l >= 0 && u.l < a.n_lys, a.err, kSiteLys)) return false;
  const int n = a.lys[u.l].n;
  if (!KMC_DCHECK(u.t0 >= 0 && u.nt >= 1 && u.nt <= kTargets && u.t0 + u.nt <= n &&
                      (u.t0 % kCell) + u.nt <= kCell && u.gt0 >= 0 &&
                      u.gt0 + u.nt <= gc * kCell,
                  a.err, kSiteTargets))
    return false;
  if (!KMC_DCHECK(u.fwd0 >= 0 && u.nfwd >= 1 && u.rev0 >= 0 && u.nrev >= 0, a.err, kSiteSplit))
    return false;
#endif
  return true;
}

// Dynamic shared memory of the field kernel: two staged cells and the warps'
// reverse sums of two cells, or the whole row group's records (diagonal).
constexpr size_t sym_field_smem(int w, int c) {
  return 16 + ((2 * kCellRec * sizeof(SrcPair) + 2 * static_cast<size_t>(w) * 6 * 32 * 4) >
                       static_cast<size_t>(w) * c * kCellRec * sizeof(SrcPair)
                   ? (2 * kCellRec * sizeof(SrcPair) + 2 * static_cast<size_t>(w) * 6 * 32 * 4)
                   : static_cast<size_t>(w) * c * kCellRec * sizeof(SrcPair));
}

template <int W, int C>
__global__ void __launch_bounds__(W * 32) kmc_field_sym(const StepArgs a, int /*tile*/) {
  constexpr int T = 2 * C;    // targets per lane
  constexpr int GC = W * C;   // cells per row group
  constexpr int GT = GC * kCell;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  unsigned char *dyn = smem + 16;
  if (!sym_item_in_bounds(a, GC)) return;
  const SymItem it = a.sitems[blockIdx.x];
  const LysDev L = a.lys[it.l];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nc = (L.n + kCell - 1) / kCell;
  const int cell0 = it.g * GC + warp * C;  // the warp's first target cell
  grid_dependency_wait();
  const long long step = a.rs->step_base + a.k_local;
  const int par = static_cast<int>(step & 1);
  const SrcPair *__restrict__ gsrc = static_cast<const SrcPair *>(a.src[par]) + L.roff;

  // the lane's targets: record `lane` of each of the warp's cells; cells past
  // the lysosome (a diagonal item's last group) are far away and have no moment
  f2 X[T], Y[T], Z[T], TX[T], TY[T], TZ[T], NX[T], NY[T], NZ[T];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    SrcPair rr;
    if (cell0 + c < nc) {
      rr = gsrc[(cell0 + c) * kCellRec + lane];
    } else {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        rr.x[h] = rr.y[h] = rr.z[h] = -kPadCoord;
        set_source_moment(rr, h, 0.f, 0.f, 0.f, 0.f);
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = 2 * c + h;
      X[k] = pk(rr.x[h], rr.x[h]);
      Y[k] = pk(rr.y[h], rr.y[h]);
      Z[k] = pk(rr.z[h], rr.z[h]);
      TX[k] = pk(rr.tx[h], rr.tx[h]);
      TY[k] = pk(rr.ty[h], rr.ty[h]);
      TZ[k] = pk(rr.tz[h], rr.tz[h]);
      NX[k] = pk(rr.nx[h], rr.nx[h]);
      NY[k] = pk(rr.ny[h], rr.ny[h]);
      NZ[k] = pk(rr.nz[h], rr.nz[h]);
    }
  }
  float s3[T][3], c3[T][3];  // Kahan sums of the forward field, per target
#pragma unroll
  for (int k = 0; k < T; ++k)
#pragma unroll
    for (int q = 0; q < 3; ++q) s3[k][q] = c3[k][q] = 0.f;
  auto fold = [&](const AccF32 (&acc)[T]) {
#pragma unroll
    for (int k = 0; k < T; ++k) {
      kahan_add(s3[k][0], c3[k][0], hsum(acc[k].x));
      kahan_add(s3[k][1], c3[k][1], hsum(acc[k].y));
      kahan_add(s3[k][2], c3[k][2], hsum(acc[k].z));
    }
  };
  ulonglong2 *buf = reinterpret_cast<ulonglong2 *>(dyn);

  if (it.h0 < 0) {
    // diagonal item: the group's records in one copy, ordered pairs
    const int c0 = it.g * GC, ncv = min(GC, nc - c0);
    const uint32_t bytes = static_cast<uint32_t>(ncv) * kCellRec * sizeof(SrcPair);
    if (threadIdx.x == 0) {
      mbar_init(&bar[0], 1);
      mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      mbar_expect_tx(&bar[0], bytes);
      bulk_g2s(buf, gsrc + c0 * kCellRec, bytes, &bar[0]);
    }
    const bool ok = mbar_wait_bounded(&bar[0], 0, a.err);
    if (!__syncthreads_and(ok)) {
      if (threadIdx.x == 0) mbar_wait_quiet(&bar[0], 0, 2000000000ull);
      __syncthreads();
      return;
    }
#pragma unroll 1
    for (int cs = 0; cs < ncv; ++cs) {
      AccF32 acc[T];
#pragma unroll
      for (int k = 0; k < T; ++k) acc[k].x = acc[k].y = acc[k].z = 0ull;
      const ulonglong2 *sp = buf + static_cast<size_t>(cs) * kCellRec * kRecU2;
      if (cs >= warp * C && cs < warp * C + C)
        ordered_cell<true, T>(sp, X, Y, Z, acc);
      else
        ordered_cell<false, T>(sp, X, Y, Z, acc);
      fold(acc);
    }
  } else {
    float *red = reinterpret_cast<float *>(dyn + 2 * kCellRec * sizeof(SrcPair));  // [2][W][6][32]
    auto issue = [&](int t) {
      const int b = t & 1;
      const uint32_t bytes = kCellRec * sizeof(SrcPair);
      mbar_expect_tx(&bar[b], bytes);
      bulk_g2s(buf + static_cast<size_t>(b) * kCellRec * kRecU2, gsrc + (it.h0 + t) * kCellRec,
               bytes, &bar[b]);
    };
    // the warps' reverse sums of cell h0 + t, added in warp order into its
    // slot for this row group: [3][64], component-major
    auto flush_rev = [&](int t) {
      const float *rb = red + (t & 1) * W * 6 * 32;
      float *dst = a.srev + static_cast<size_t>(it.rbase + sym_rev_offset(it.h0 + t, GC) + it.g) *
                                3 * kCell;
      for (int v = threadIdx.x; v < 6 * 32; v += W * 32) {
        const int j = v >> 5, ln = v & 31;
        float r = rb[j * 32 + ln];
#pragma unroll
        for (int w = 1; w < W; ++w) r += rb[(w * 6 + j) * 32 + ln];
        __stcg(dst + (j % 3) * kCell + 2 * ln + j / 3, r);
      }
    };
    auto body = [&](int b, int t) {
      if (t > 0) flush_rev(t - 1);
      AccF32 acc[T];
#pragma unroll
      for (int k = 0; k < T; ++k) acc[k].x = acc[k].y = acc[k].z = 0ull;
      f2 rx = 0ull, ry = 0ull, rz = 0ull;
      sym_cell<T>(buf + static_cast<size_t>(b) * kCellRec * kRecU2, lane, X, Y, Z, TX, TY, TZ, NX,
                  NY, NZ, acc, rx, ry, rz);
      fold(acc);
      float *rw = red + ((t & 1) * W + warp) * 6 * 32;
      float lo, hi;
      upk(rx, lo, hi);
      rw[0 * 32 + lane] = lo;
      rw[3 * 32 + lane] = hi;
      upk(ry, lo, hi);
      rw[1 * 32 + lane] = lo;
      rw[4 * 32 + lane] = hi;
      upk(rz, lo, hi);
      rw[2 * 32 + lane] = lo;
      rw[5 * 32 + lane] = hi;
    };
    const int ncs = it.h1 - it.h0;
    if (!staged_loop(ncs, bar, a.err, issue, body)) return;
    flush_rev(ncs - 1);
  }
  // forward partials of the warp's targets: [3][GT] at the item's slot, each
  // the Kahan sum with its compensation applied (s - c: Kahan keeps minus
  // the error), i.e. the item's sum rounded once to float
  float *fw = a.sfwd + static_cast<size_t>(it.fwd) * 3 * GT;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    if (cell0 + c >= nc) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = 2 * c + h;
      const int gi = (warp * C + c) * kCell + 2 * lane + h;
#pragma unroll
      for (int q = 0; q < 3; ++q) __stcg(fw + q * GT + gi, s3[k][q] - c3[k][q]);
    }
  }
  grid_launch_dependents();
}

template <int GC>
__global__ void __launch_bounds__(kSymUpdWarps * 32) kmc_update_sym(const StepArgs a, int /*tile*/) {
  constexpr int NW = kSymUpdWarps;
  constexpr int GT = GC * kCell;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char *dyn = smem + 16;
  __shared__ GridTables<float> tab;
  tab.load();
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ui = blockIdx.x * NW + warp;  // this warp's update item
  if (ui >= a.n_upd || !sym_upd_in_bounds(a, GC, ui)) return;
  const SymUpd u = a.supd[ui];
  const LysDev L = a.lys[u.l];
  Item it;
  it.l = u.l;
  it.t0 = u.t0;
  it.nt = u.nt;
  it.gid = 0;
  it.j0 = it.j1 = 0;
  it.split = 0;
  it.nsplit = 1;
  grid_dependency_wait();
  const long long step = a.rs->step_base + a.k_local;
  const int per = a.rs->period;
  const int rec = (per >= a.discard) ? (per - a.discard) * a.S + a.k_local : -1;
  const TargetIn<float4> tin = load_target<float4>(a, L, it, step, lane);
  // lanes past the last target repeat it (their results are not written)
  const int tl = min(lane, u.nt - 1);
  const int gi = u.gt0 + tl, ci = (u.t0 + tl) % kCell;
  // the slots in order; each batch's loads are issued before its additions
  float hi[3] = {0.f, 0.f, 0.f}, lo[3] = {0.f, 0.f, 0.f};
  constexpr int kFwdBatch = 8, kRevBatch = 8;
#pragma unroll 1
  for (int s0 = 0; s0 < u.nfwd; s0 += kFwdBatch) {
    float v[kFwdBatch][3];
#pragma unroll
    for (int b = 0; b < kFwdBatch; ++b) {
      const float *p = a.sfwd + static_cast<size_t>(u.fwd0 + min(s0 + b, u.nfwd - 1)) * 3 * GT;
#pragma unroll
      for (int q = 0; q < 3; ++q) v[b][q] = __ldcg(p + q * GT + gi);
    }
#pragma unroll
    for (int b = 0; b < kFwdBatch; ++b) {
      if (s0 + b >= u.nfwd) break;
#pragma unroll
      for (int q = 0; q < 3; ++q) neumaier_add(hi[q], lo[q], v[b][q]);
    }
  }
#pragma unroll 1
  for (int s0 = 0; s0 < u.nrev; s0 += kRevBatch) {
    float v[kRevBatch][3];
#pragma unroll
    for (int b = 0; b < kRevBatch; ++b) {
      const float *p = a.srev + static_cast<size_t>(u.rev0 + min(s0 + b, u.nrev - 1)) * 3 * kCell;
#pragma unroll
      for (int q = 0; q < 3; ++q) v[b][q] = __ldcg(p + q * kCell + ci);
    }
#pragma unroll
    for (int b = 0; b < kRevBatch; ++b) {
      if (s0 + b >= u.nrev) break;
#pragma unroll
      for (int q = 0; q < 3; ++q) neumaier_add(hi[q], lo[q], v[b][q]);
    }
  }
  EpiShared<float> &sm = reinterpret_cast<EpiShared<float> *>(dyn)[warp];
#pragma unroll
  for (int q = 0; q < 3; ++q) sm.h[q][lane] = hi[q] + lo[q];  // compensation added last
  __syncwarp();
  block_update<float4, true, true>(a, L, it, step, rec, tin, sm, tab);
  grid_launch_dependents();
}

// The update kernel with one block per update item (kmc_pair_form's update
// mode 1): the block's four warps share the gather of the item's partial
// slots (warp w takes slots w, w + 4, ..., then the warps are added in order)
// and run steps iii-vii block-cooperatively. Where a target gathers many
// slots (large lysosomes) the shorter gather outweighs the idle warps of the
// block-cooperative update; kmc_update_sym is faster where items are many
// and slots few. The two give different roundings of the field sums, each in
// a fixed order.
template <int GC>
__global__ void __launch_bounds__(kSymUpdWarps * 32)
    kmc_update_sym_block(const StepArgs a, int /*tile*/) {
  constexpr int NW = kSymUpdWarps;
  constexpr int GT = GC * kCell;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char *dyn = smem + 16;
  __shared__ GridTables<float> tab;
  tab.load();
  if (!sym_upd_in_bounds(a, GC, static_cast<int>(blockIdx.x))) return;
  const SymUpd u = a.supd[blockIdx.x];
  const LysDev L = a.lys[u.l];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Item it;
  it.l = u.l;
  it.t0 = u.t0;
  it.nt = u.nt;
  it.gid = 0;
  it.j0 = it.j1 = 0;
  it.split = 0;
  it.nsplit = 1;
  grid_dependency_wait();
  const long long step = a.rs->step_base + a.k_local;
  const int per = a.rs->period;
  const int rec = (per >= a.discard) ? (per - a.discard) * a.S + a.k_local : -1;
  TargetIn<float4> tin;
  if (warp == 0) tin = load_target<float4>(a, L, it, step, lane);
  // lanes past the last target repeat it (their results are not written)
  const int tl = min(lane, u.nt - 1);
  const int gi = u.gt0 + tl, ci = (u.t0 + tl) % kCell;
  float hi[3] = {0.f, 0.f, 0.f}, lo[3] = {0.f, 0.f, 0.f};
#pragma unroll 1
  for (int sl = warp; sl < u.nfwd; sl += NW) {
    const float *p = a.sfwd + static_cast<size_t>(u.fwd0 + sl) * 3 * GT;
#pragma unroll
    for (int q = 0; q < 3; ++q) neumaier_add(hi[q], lo[q], __ldcg(p + q * GT + gi));
  }
#pragma unroll 1
  for (int sl = warp; sl < u.nrev; sl += NW) {
    const float *p = a.srev + static_cast<size_t>(u.rev0 + sl) * 3 * kCell;
#pragma unroll
    for (int q = 0; q < 3; ++q) neumaier_add(hi[q], lo[q], __ldcg(p + q * kCell + ci));
  }
  float *wp = reinterpret_cast<float *>(dyn);  // [NW][6][32]
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    wp[(warp * 6 + q) * 32 + lane] = hi[q];
    wp[(warp * 6 + 3 + q) * 32 + lane] = lo[q];
  }
  __syncthreads();
  EpiShared<float> &sm =
      *reinterpret_cast<EpiShared<float> *>(dyn + static_cast<size_t>(NW) * 6 * 32 * 4);
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      float s = 0.f, e = 0.f;
      for (int w = 0; w < NW; ++w) {
        neumaier_add(s, e, wp[(w * 6 + q) * 32 + lane]);
        e += wp[(w * 6 + 3 + q) * 32 + lane];
      }
      sm.h[q][lane] = s + e;  // compensation added last
    }
  }
  __syncthreads();
  block_update<float4, true>(a, L, it, step, rec, tin, sm, tab);
  grid_launch_dependents();
}

// ---------------------------------------------------------------------------
// Host side of the launches.

size_t step_smem_bytes(int prec_fp32, int warps, int tile, int tpl, int rpl) {
  if (prec_fp32 && rpl > 1) {
    const size_t stage = 2 * static_cast<size_t>(rpl) * tile * sizeof(SrcPair);
    const size_t epi = epi_bytes_rep(rpl, warps);
    return 16 + (stage > epi ? stage : epi);
  }
  const size_t stage = prec_fp32 ? 2 * static_cast<size_t>(tile) * sizeof(SrcPair)
                                 : 4 * static_cast<size_t>(tile) * sizeof(dbl4);
  const size_t epi = !prec_fp32 ? epi_bytes<double>(warps)
                                : (tpl >= 2 ? epi_bytes_tn(warps, tpl) : epi_bytes<float>(warps));
  return 16 + (stage > epi ? stage : epi);
}

// Launches kernel k over n_items blocks; with pdl the launch carries the
// programmatic stream serialisation attribute.
template <typename K>
static cudaError_t launch_items(K kernel, const StepArgs &a, int n_items, int threads,
                                size_t smem, int tile, cudaStream_t st, bool pdl,
                                int cluster = 0) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(n_items));
  cfg.blockDim = dim3(static_cast<unsigned>(threads));
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  int na = 0;
  if (pdl) {
    attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  if (cluster > 1) {
    if (n_items % cluster != 0) return cudaErrorInvalidValue;
    attr[na].id = cudaLaunchAttributeClusterDimension;
    attr[na].val.clusterDim.x = static_cast<unsigned>(cluster);
    attr[na].val.clusterDim.y = 1;
    attr[na].val.clusterDim.z = 1;
    ++na;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, kernel, a, tile);
}

template <int NW>
static cudaError_t launch_f32(const StepArgs &a, int n_items, int tile, cudaStream_t st,
                              bool pdl, int tpl, int cl) {
  if (cl == 2) {
    if (tpl != 1) return cudaErrorInvalidValue;
    return launch_items(kmc_step_f32<NW, true>, a, n_items, NW * 32,
                        step_smem_bytes(1, NW, tile, 1), tile, st, pdl, 2);
  }
  if (cl != 0) return cudaErrorInvalidValue;
  if (tpl == 2)
    return launch_items(kmc_step_f32_tn<NW, 2>, a, n_items, NW * 32,
                        step_smem_bytes(1, NW, tile, 2), tile, st, pdl);
  if (tpl == 3)
    return launch_items(kmc_step_f32_tn<NW, 3>, a, n_items, NW * 32,
                        step_smem_bytes(1, NW, tile, 3), tile, st, pdl);
  if (tpl != 1) return cudaErrorInvalidValue;
  return launch_items(kmc_step_f32<NW>, a, n_items, NW * 32, step_smem_bytes(1, NW, tile, 1), tile,
                      st, pdl);
}
template <int NW>
static cudaError_t launch_f64(const StepArgs &a, int n_items, int tile, cudaStream_t st,
                              bool pdl) {
  return launch_items(kmc_step_f64<NW>, a, n_items, NW * 32, step_smem_bytes(0, NW, tile, 1),
                      tile, st, pdl);
}

cudaError_t launch_step(int prec_fp32, int warps, int tile, const StepArgs &a, int n_items,
                        cudaStream_t st, bool pdl, int tpl, int rpl, int cl) {
  if (n_items <= 0) return cudaSuccess;
  if (cl != 0 && (!prec_fp32 || rpl > 1)) return cudaErrorInvalidValue;
  if (rpl > 1) {
    if (!prec_fp32 || tpl != 1 || (warps != rpl && warps != 2 * rpl && warps != 4 * rpl))
      return cudaErrorInvalidValue;
    const size_t smem = step_smem_bytes(1, warps, tile, 1, rpl);
    const int th = warps * 32;
    if (rpl == 2 && warps == 2)
      return launch_items(kmc_step_f32_rep<2>, a, n_items, th, smem, tile, st, pdl);
    if (rpl == 4 && warps == 4)
      return launch_items(kmc_step_f32_rep<4>, a, n_items, th, smem, tile, st, pdl);
    if (rpl == 2 && warps == 4)
      return launch_items(kmc_step_f32_rep<2, 2>, a, n_items, th, smem, tile, st, pdl);
    if (rpl == 4 && warps == 8)
      return launch_items(kmc_step_f32_rep<4, 2>, a, n_items, th, smem, tile, st, pdl);
    if (rpl == 2 && warps == 8)
      return launch_items(kmc_step_f32_rep<2, 4>, a, n_items, th, smem, tile, st, pdl);
    if (rpl == 4 && warps == 16)
      return launch_items(kmc_step_f32_rep<4, 4>, a, n_items, th, smem, tile, st, pdl);
    return cudaErrorInvalidValue;
  }
  if (prec_fp32) {
    switch (warps) {
      case 4: return launch_f32<4>(a, n_items, tile, st, pdl, tpl, cl);
      case 8: return launch_f32<8>(a, n_items, tile, st, pdl, tpl, cl);
      case 16: return launch_f32<16>(a, n_items, tile, st, pdl, tpl, cl);
      default: return cudaErrorInvalidValue;
    }
  }
  if (tpl != 1) return cudaErrorInvalidValue;
  switch (warps) {
    case 4: return launch_f64<4>(a, n_items, tile, st, pdl);
    case 8: return launch_f64<8>(a, n_items, tile, st, pdl);
    case 16: return launch_f64<16>(a, n_items, tile, st, pdl);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_persist(const StepArgs &a, int warps, int tile, int n_items, cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(n_items));
  cfg.blockDim = dim3(static_cast<unsigned>(warps * 32));
  cfg.dynamicSmemBytes = step_smem_bytes(1, warps, tile, 1);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (warps == 4) return cudaLaunchKernelEx(&cfg, kmc_persist_f32<4>, a, tile);
  if (warps == 8) return cudaLaunchKernelEx(&cfg, kmc_persist_f32<8>, a, tile);
  return cudaErrorInvalidValue;
}

// Symmetric form: the field kernel over n_field items, then the update kernel
// over the a.n_upd target groups, both on st.
template <int W, int C>
static cudaError_t launch_sym_wc(const StepArgs &a, int n_field, cudaStream_t st, bool pdl,
                                 int upd) {
  cudaError_t e = cudaSuccess;
  if (n_field > 0)
    e = launch_items(kmc_field_sym<W, C>, a, n_field, W * 32, sym_field_smem(W, C), 0, st, pdl);
  if (e == cudaSuccess && a.n_upd > 0) {
    if (upd == 1)
      e = launch_items(kmc_update_sym_block<W * C>, a, a.n_upd, kSymUpdWarps * 32,
                       16 + epi_bytes<float>(kSymUpdWarps), 0, st, pdl);
    else
      e = launch_items(kmc_update_sym<W * C>, a, (a.n_upd + kSymUpdWarps - 1) / kSymUpdWarps,
                       kSymUpdWarps * 32, 16 + kSymUpdWarps * sizeof(EpiShared<float>), 0, st,
                       pdl);
  }
  return e;
}

cudaError_t launch_sym(const StepArgs &a, int warps, int cells, int n_field, cudaStream_t st,
                       bool pdl, int upd) {
  if (upd != 0 && upd != 1) return cudaErrorInvalidValue;
  if (warps == 2 && cells == 2) return launch_sym_wc<2, 2>(a, n_field, st, pdl, upd);
  if (warps == 4 && cells == 1) return launch_sym_wc<4, 1>(a, n_field, st, pdl, upd);
  if (warps == 4 && cells == 2) return launch_sym_wc<4, 2>(a, n_field, st, pdl, upd);
  if (warps == 8 && cells == 1) return launch_sym_wc<8, 1>(a, n_field, st, pdl, upd);
  return cudaErrorInvalidValue;
}

size_t sym_smem_bytes(int warps, int cells) { return sym_field_smem(warps, cells); }

template <typename K>
static cudaError_t occupancy(K kernel, int threads, size_t smem, int *blocks) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kernel, threads, smem);
}

cudaError_t persist_blocks_per_sm(int warps, int tile, int *blocks) {
  *blocks = 0;
  const size_t smem = step_smem_bytes(1, warps, tile, 1);
  if (warps == 4) return occupancy(kmc_persist_f32<4>, 128, smem, blocks);
  if (warps == 8) return occupancy(kmc_persist_f32<8>, 256, smem, blocks);
  return cudaErrorInvalidValue;
}

cudaError_t sym_blocks_per_sm(int warps, int cells, int *blocks) {
  *blocks = 0;
  const size_t smem = sym_field_smem(warps, cells);
  if (warps == 2 && cells == 2) return occupancy(kmc_field_sym<2, 2>, 64, smem, blocks);
  if (warps == 4 && cells == 1) return occupancy(kmc_field_sym<4, 1>, 128, smem, blocks);
  if (warps == 4 && cells == 2) return occupancy(kmc_field_sym<4, 2>, 128, smem, blocks);
  if (warps == 8 && cells == 1) return occupancy(kmc_field_sym<8, 1>, 256, smem, blocks);
  return cudaErrorInvalidValue;
}

cudaError_t step_blocks_per_sm(int prec_fp32, int warps, int tile, int tpl, int *blocks,
                               int rpl) {
  *blocks = 0;
  const size_t smem = step_smem_bytes(prec_fp32, warps, tile, tpl, rpl);
  const int th = warps * 32;
  if (prec_fp32 && rpl > 1) {
    if (rpl == 2 && warps == 2) return occupancy(kmc_step_f32_rep<2>, th, smem, blocks);
    if (rpl == 4 && warps == 4) return occupancy(kmc_step_f32_rep<4>, th, smem, blocks);
    if (rpl == 2 && warps == 4) return occupancy(kmc_step_f32_rep<2, 2>, th, smem, blocks);
    if (rpl == 4 && warps == 8) return occupancy(kmc_step_f32_rep<4, 2>, th, smem, blocks);
    if (rpl == 2 && warps == 8) return occupancy(kmc_step_f32_rep<2, 4>, th, smem, blocks);
    if (rpl == 4 && warps == 16) return occupancy(kmc_step_f32_rep<4, 4>, th, smem, blocks);
    return cudaErrorInvalidValue;
  }
  if (prec_fp32 && tpl == 2) {
    switch (warps) {
      case 4: return occupancy(kmc_step_f32_tn<4, 2>, th, smem, blocks);
      case 8: return occupancy(kmc_step_f32_tn<8, 2>, th, smem, blocks);
      case 16: return occupancy(kmc_step_f32_tn<16, 2>, th, smem, blocks);
      default: return cudaErrorInvalidValue;
    }
  }
  if (prec_fp32 && tpl == 3) {
    switch (warps) {
      case 4: return occupancy(kmc_step_f32_tn<4, 3>, th, smem, blocks);
      case 8: return occupancy(kmc_step_f32_tn<8, 3>, th, smem, blocks);
      case 16: return occupancy(kmc_step_f32_tn<16, 3>, th, smem, blocks);
      default: return cudaErrorInvalidValue;
    }
  }
  if (prec_fp32) {
    switch (warps) {
      case 4: return occupancy(kmc_step_f32<4>, th, smem, blocks);
      case 8: return occupancy(kmc_step_f32<8>, th, smem, blocks);
      case 16: return occupancy(kmc_step_f32<16>, th, smem, blocks);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (warps) {
    case 4: return occupancy(kmc_step_f64<4>, th, smem, blocks);
    case 8: return occupancy(kmc_step_f64<8>, th, smem, blocks);
    case 16: return occupancy(kmc_step_f64<16>, th, smem, blocks);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_mean(const MeanArgs &a, cudaStream_t st) {
  if (a.n_items <= 0) return cudaSuccess;
  const int blocks = (a.n_items + kMeanWarps - 1) / kMeanWarps;
  kmc_mean_kernel<<<blocks, kMeanWarps * 32, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_regen(const RegenArgs &a, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  kmc_regen_kernel<<<(a.n + 127) / 128, 128, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_rsa_batch(const RsaArgs &a, cudaStream_t st) {
  if (a.B <= 0) return cudaSuccess;
  rsa_candidates_kernel<<<(a.B + 127) / 128, 128, 0, st>>>(a);
  rsa_check_kernel<<<a.B, 128, 0, st>>>(a);
  rsa_resolve_kernel<<<1, 1024, rsa_resolve_smem(a.B), st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_advance(RunState *rs, int S, cudaStream_t st) {
  kmc_advance_kernel<<<1, 1, 0, st>>>(rs, S);
  return cudaGetLastError();
}

template <typename K>
static cudaError_t allow_smem(K kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(kMaxStepSmem));
}

cudaError_t init_device() {
  float th_f[kGrid];
  float2 sc_f[kGrid];
  double th_d[kGrid];
  double2 sc_d[kGrid];
  const double two_pi = 6.283185307179586476925286766559;
  for (int j = 0; j < kGrid; ++j) {
    th_d[j] = two_pi * (static_cast<double>(j) + 0.5) / static_cast<double>(kGrid);
    sc_d[j] = make_double2(sin(th_d[j]), cos(th_d[j]));
    th_f[j] = static_cast<float>(th_d[j]);
    sc_f[j] = make_float2(static_cast<float>(sc_d[j].x), static_cast<float>(sc_d[j].y));
  }
  float ss_f[kGridPad], cc_f[kGridPad];
  for (int j = 0; j < kGridPad; ++j) {
    ss_f[j] = sc_f[j % kGrid].x;
    cc_f[j] = sc_f[j % kGrid].y;
  }
  cudaError_t e = cudaMemcpyToSymbol(g_theta_f, th_f, sizeof(th_f));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_sc_f, sc_f, sizeof(sc_f));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_ss_f, ss_f, sizeof(ss_f));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_cc_f, cc_f, sizeof(cc_f));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_theta_d, th_d, sizeof(th_d));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_sc_d, sc_d, sizeof(sc_d));

  // kernel attributes are set here, never inside a stream capture
  if (e == cudaSuccess) e = allow_smem(kmc_step_f32<4>);
  if (e == cudaSuccess) e = allow_smem(kmc_step_f32<8>);
  if (e == cudaSuccess) e = allow_smem(kmc_step_f32<16>);
  if (e == cudaSuccess) e = allow_smem(kmc_persist_f32<4>);
  if (e == cudaSuccess) e = allow_smem(kmc_persist_f32<8>);
  if (e == cudaSuccess) e = allow_smem(kmc_step_f32<4, true>);
  if (e == cudaSuccess) e = allow_smem(kmc_step_f32<8, true>);
  if (e == cudaSuccess) e = allow_smem(kmc_step_f32<16, true>);
  if (e == cudaSuccess) e = allow_smem(kmc_step_f32_tn<4, 2>);
  if (e == cudaSuccess) e = allow_smem(kmc_step_f32_tn<8, 2>);
  if (e == cudaSuccess) e = allow_smem(kmc_step_f32_tn<16, 2>);
  if (e == cudaSuccess) e = allow_smem(kmc_step_f32_tn<4, 3>);
  if (e == cudaSuccess) e = allow_smem(kmc_step_f32_tn<8, 3>);
  if (e == cudaSuccess) e = allow_smem(kmc_step_f32_tn<16, 3>);
  if (e == cudaSuccess) e = allow_smem(kmc_step_f32_rep<2>);
  if (e == cudaSuccess) e = allow_smem(kmc_step_f32_rep<4>);
  if (e == cudaSuccess) e = allow_smem(kmc_step_f32_rep<2, 2>);
  if (e == cudaSuccess) e = allow_smem(kmc_step_f32_rep<4, 2>);
  if (e == cudaSuccess) e = allow_smem(kmc_step_f32_rep<2, 4>);
  if (e == cudaSuccess) e = allow_smem(kmc_step_f32_rep<4, 4>);
  if (e == cudaSuccess) e = allow_smem(kmc_field_sym<2, 2>);
  if (e == cudaSuccess) e = allow_smem(kmc_field_sym<4, 1>);
  if (e == cudaSuccess) e = allow_smem(kmc_field_sym<4, 2>);
  if (e == cudaSuccess) e = allow_smem(kmc_field_sym<8, 1>);
  if (e == cudaSuccess) e = allow_smem(kmc_update_sym<4>);
  if (e == cudaSuccess) e = allow_smem(kmc_update_sym<8>);
  if (e == cudaSuccess) e = allow_smem(kmc_update_sym_block<4>);
  if (e == cudaSuccess) e = allow_smem(kmc_update_sym_block<8>);
  if (e == cudaSuccess) e = allow_smem(kmc_step_f64<4>);
  if (e == cudaSuccess) e = allow_smem(kmc_step_f64<8>);
  if (e == cudaSuccess) e = allow_smem(kmc_step_f64<16>);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(rsa_resolve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(rsa_resolve_smem(kRsaMaxBatch)));
  return e;
}

}  // namespace kmc
