// kmc_device.cuh -- device building blocks of the kMC step (sm_103a):
// bulk-copy (TMA) staging with bounded mbarrier waits, the Philox4x32-10
// draw, and the per-NP update of steps iii-vii of Sec. II.1.
#pragma once
#include <stdint.h>

#include "kmc_types.h"

namespace kmc {

// Grid of step iv: theta_j = 2 pi (j + 1/2) / 200 with its sine and cosine,
// written once per device by init_device (kmc_step.cu, the only translation
// unit that includes this header).
__device__ float g_grid_f[3][kGrid];   // theta_j, sin, cos
__device__ double g_grid_d[3][kGrid];

// ---------------------------------------------------------------------------
// Shared-memory staging by bulk asynchronous copies (TMA engine).

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void proxy_fence_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// Bulk copy global -> shared; both addresses 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for phase `parity` of `bar` for at most ~2 s; returns false (and sets
// the error word) if the copy never completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  int32_t *err) {
  for (int i = 0; i < 64; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > 2000000000ull) {
      atomicOr(err, kErrTimeout);
      return false;
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 32x32->64 multiplications with the Philox multipliers; the key advances by
// the Weyl constants after every round.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// 53-bit uniform in [0,1) for (seed, global step, NP within lysosome, lysosome).
__device__ __forceinline__ double kmc_uniform(unsigned long long seed, long long step,
                                              int np, int lys) {
  const unsigned long long s = static_cast<unsigned long long>(step);
  const uint4 w = philox4x32_10(
      make_uint4(static_cast<uint32_t>(s), static_cast<uint32_t>(s >> 32),
                 static_cast<uint32_t>(np), static_cast<uint32_t>(lys)),
      make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32)));
  const unsigned long long bits =
      (static_cast<unsigned long long>(w.x) << 21) ^ static_cast<unsigned long long>(w.y >> 11);
  return static_cast<double>(bits) * 0x1.0p-53;
}

// ---------------------------------------------------------------------------
// Steps iii-vii for one NP, in reduced units (kmc_types.h).

template <typename R>
struct Prec;
template <>
struct Prec<float> {
  static constexpr float two_pi = 6.28318530717958647692f;
  static constexpr float plane_tol = 1e-6f;   // |b x a| below this: plane from m
  static constexpr float newton_tol = 2e-9f;  // absolute, on the offset in a cell
  static constexpr int newton_max = 24;
  __device__ static float theta(int j) { return g_grid_f[0][j]; }
  __device__ static float sn(int j) { return g_grid_f[1][j]; }
  __device__ static float cs(int j) { return g_grid_f[2][j]; }
  // sin and cos of 0 <= d <= 2 pi / 200 by their Taylor series (error < 1e-11)
  __device__ static void sincos_small(float d, float &s, float &c) {
    const float d2 = d * d;
    s = d * fmaf(d2, fmaf(d2, 1.0f / 120.0f, -1.0f / 6.0f), 1.0f);
    c = fmaf(d2, fmaf(d2, 1.0f / 24.0f, -0.5f), 1.0f);
  }
};
template <>
struct Prec<double> {
  static constexpr double two_pi = 6.283185307179586476925286766559;
  static constexpr double plane_tol = 1e-12;
  static constexpr double newton_tol = 1e-14;
  static constexpr int newton_max = 100;
  __device__ static double theta(int j) { return g_grid_d[0][j]; }
  __device__ static double sn(int j) { return g_grid_d[1][j]; }
  __device__ static double cs(int j) { return g_grid_d[2][j]; }
  // Taylor series to d^9 / d^10: truncation below 1e-24 for d <= 2 pi / 200
  __device__ static void sincos_small(double d, double &s, double &c) {
    const double d2 = d * d;
    s = d * fma(d2, fma(d2, fma(d2, fma(d2, 1.0 / 362880.0, -1.0 / 5040.0), 1.0 / 120.0),
                        -1.0 / 6.0),
                1.0);
    c = fma(d2,
            fma(d2, fma(d2, fma(d2, fma(d2, -1.0 / 3628800.0, 1.0 / 40320.0), -1.0 / 720.0),
                        1.0 / 24.0),
                -0.5),
            1.0);
  }
};

// Eq. 2 in a working plane: e = k sin^2 th - b cos(th - phi);
// de/dth = 2k s c + b (s cos phi - c sin phi); d2e = 2k (c^2 - s^2) + b (c cos phi + s sin phi).
template <typename R>
struct Profile {
  R k2;  // 2k
  R k;
  R bc;  // b cos phi
  R bs;  // b sin phi
  __device__ R d1(R s, R c) const { return s * fma(k2, c, bc) - bs * c; }
  __device__ R d2(R s, R c) const { return k2 * (c * c - s * s) + fma(bc, c, bs * s); }
  __device__ R e(R s, R c) const { return k * s * s - fma(bc, c, bs * s); }
};

// Newton's method with bisection fallback for the root of de/dth inside grid
// cell [theta_j, theta_j + h], as offset d from theta_j. dlo = de/dth at theta_j.
template <typename R>
__device__ __forceinline__ R refine_in_cell(const Profile<R> &pf, R S0, R C0, R h, R dlo,
                                            R &s_out, R &c_out) {
  R lo = R(0), hi = h, x = R(0.5) * h;
  for (int it = 0; it < Prec<R>::newton_max; ++it) {
    R sd, cd;
    Prec<R>::sincos_small(x, sd, cd);
    const R s = fma(S0, cd, C0 * sd), c = fma(C0, cd, -S0 * sd);
    const R d = pf.d1(s, c);
    if (d == R(0)) break;
    if ((d < R(0)) == (dlo < R(0))) {
      lo = x;
      dlo = d;
    } else {
      hi = x;
    }
    const R dd = pf.d2(s, c);
    R xn = (dd != R(0)) ? x - d / dd : R(0.5) * (lo + hi);
    if (!(xn > lo && xn < hi)) xn = R(0.5) * (lo + hi);
    const bool done = fabs(xn - x) < Prec<R>::newton_tol || hi - lo < Prec<R>::newton_tol;
    x = xn;
    if (done) break;
  }
  R sd, cd;
  Prec<R>::sincos_small(x, sd, cd);
  s_out = fma(S0, cd, C0 * sd);
  c_out = fma(C0, cd, -S0 * sd);
  return x;
}

// 1 if x lies on the arc running counter-clockwise from just after `from` up
// to and including `to` (all angles in [0, 2 pi)).
template <typename R>
__device__ __forceinline__ bool on_arc(R x, R from, R to) {
  R dx = x - from, dt = to - from;
  if (dx < R(0)) dx += Prec<R>::two_pi;
  if (dt < R(0)) dt += Prec<R>::two_pi;
  return dx > R(0) && dx <= dt;
}

// Element i of a 4-array without dynamic indexing (keeps it in registers).
template <typename T>
__device__ __forceinline__ T sel4(const T (&a)[4], int i) {
  return i == 0 ? a[0] : (i == 1 ? a[1] : (i == 2 ? a[2] : a[3]));
}

struct NPResult {
  double dEa, dEb, P;  // reduced barriers from the current / other well, jump probability
  int nmin, flipped, near, degenerate, bad;
};

// One NP: axis a, previous unit moment m, total reduced field b. On return m
// holds the new unit moment. beta = mu0 M_S^2 V / k_B T, lognu0t = ln(t_step / tau0).
// MIXED: near the switching field (smallest barrier below 2 % of k) the four
// extrema are polished by one FP64 Newton step and their energies taken in
// FP64, so that E3 - E_a does not lose its digits to cancellation.
template <typename R, bool MIXED>
__device__ __forceinline__ NPResult np_update(R ax, R ay, R az, R &mx, R &my, R &mz, R bx, R by,
                                              R bz, R k, double beta, double lognu0t,
                                              bool t_zero, double u) {
  NPResult o;
  o.dEa = o.dEb = o.P = 0.0;
  o.nmin = o.flipped = o.near = o.degenerate = o.bad = 0;
  // iii) working plane through the axis a and the total field b
  const R bmag = sqrt(fma(bx, bx, fma(by, by, bz * bz)));
  R ex = R(0), ey = R(0), ez = R(0), cphi = R(1), sphi = R(0);
  bool degenerate = true;
  if (bmag > R(0)) {
    const R inv = R(1) / bmag;
    const R hx = bx * inv, hy = by * inv, hz = bz * inv;
    cphi = fma(ax, hx, fma(ay, hy, az * hz));
    const R px = fma(-cphi, ax, hx), py = fma(-cphi, ay, hy), pz = fma(-cphi, az, hz);
    const R sp = sqrt(fma(px, px, fma(py, py, pz * pz)));
    if (sp >= Prec<R>::plane_tol) {
      ex = px / sp;
      ey = py / sp;
      ez = pz / sp;
      sphi = sp;
      degenerate = false;
    } else {
      cphi = (cphi >= R(0)) ? R(1) : R(-1);
    }
  }
  if (degenerate) {
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
    ex = px / sp;
    ey = py / sp;
    ez = pz / sp;
  }
  o.degenerate = degenerate;
  const R m_a = fma(mx, ax, fma(my, ay, mz * az));
  const R m_e = fma(mx, ex, fma(my, ey, mz * ez));
  R th0 = atan2(m_e, m_a);
  if (th0 < R(0)) th0 += Prec<R>::two_pi;

  // iv) 200-point scan of de/dth, sign changes refined by Newton
  Profile<R> pf;
  pf.k = k;
  pf.k2 = R(2) * k;
  pf.bc = bmag * cphi;
  pf.bs = bmag * sphi;
  int cnt = 0;
  int jq0 = 0, jq1 = 0, jq2 = 0, jq3 = 0;
  R dq0 = R(0), dq1 = R(0), dq2 = R(0), dq3 = R(0);
  const R dfirst = pf.d1(Prec<R>::sn(0), Prec<R>::cs(0));
  R dprev = dfirst;
  for (int j = 1; j <= kGrid; ++j) {
    const R d = (j < kGrid) ? pf.d1(Prec<R>::sn(j), Prec<R>::cs(j)) : dfirst;
    if ((d < R(0)) != (dprev < R(0))) {
      if (cnt == 0) {
        jq0 = j - 1;
        dq0 = dprev;
      } else if (cnt == 1) {
        jq1 = j - 1;
        dq1 = dprev;
      } else if (cnt == 2) {
        jq2 = j - 1;
        dq2 = dprev;
      } else if (cnt == 3) {
        jq3 = j - 1;
        dq3 = dprev;
      }
      ++cnt;
    }
    dprev = d;
  }
  if (cnt > 4) {
    o.bad = 1;
    cnt = 4;
  }
  R th[4], en[4], sq[4], cq[4];
  bool ismin[4];
  int jq[4] = {jq0, jq1, jq2, jq3};
  R dq[4] = {dq0, dq1, dq2, dq3};
  R off[4];
  const R hcell = Prec<R>::theta(1) - Prec<R>::theta(0);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    th[q] = en[q] = sq[q] = cq[q] = off[q] = R(0);
    ismin[q] = false;
    if (q < cnt) {
      const int j = jq[q];
      R s, c;
      off[q] = refine_in_cell(pf, Prec<R>::sn(j), Prec<R>::cs(j), hcell, dq[q], s, c);
      R t = Prec<R>::theta(j) + off[q];
      if (t >= Prec<R>::two_pi) t -= Prec<R>::two_pi;
      th[q] = t;
      sq[q] = s;
      cq[q] = c;
      en[q] = pf.e(s, c);
      ismin[q] = dq[q] < R(0);
    }
  }
  int nmin = 0, nmax = 0, imin0 = 0, imin1 = 0, imax0 = 0, imax1 = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (q < cnt) {
      if (ismin[q]) {
        if (nmin == 0) imin0 = q; else imin1 = q;
        ++nmin;
      } else {
        if (nmax == 0) imax0 = q; else imax1 = q;
        ++nmax;
      }
    }
  }
  if (nmin > 2 || nmax > 2) {
    o.bad = 1;
    nmin = 1;
  }
  o.nmin = nmin;
  // new angle of the moment, as its sine and cosine in the plane
  R s_new, c_new;
  if (nmin == 0) {  // flat profile (K_eff = 0 and no field): keep the projection
    const R nrm = sqrt(fma(m_a, m_a, m_e * m_e));
    s_new = (nrm > R(0)) ? m_e / nrm : R(0);
    c_new = (nrm > R(0)) ? m_a / nrm : R(1);
  } else if (nmin == 1) {
    s_new = sel4(sq, imin0);
    c_new = sel4(cq, imin0);
  } else {
    // v) basins: the two maxima split the circle into two arcs
    const R M1 = sel4(th, imax0), M2 = sel4(th, imax1);
    const bool arc0 = on_arc<R>(th0, M1, M2);
    const bool arcA = on_arc<R>(sel4(th, imin0), M1, M2);
    const int wa = (arc0 == arcA) ? imin0 : imin1;
    const int wb = (wa == imin0) ? imin1 : imin0;
    const R e3 = fmin(sel4(en, imax0), sel4(en, imax1));
    double dEa = static_cast<double>(e3 - sel4(en, wa));
    double dEb = static_cast<double>(e3 - sel4(en, wb));
    if (MIXED && fmin(dEa, dEb) < 0.02 * static_cast<double>(k)) {
      // FP64 polish: one Newton step from each FP32 root, energies in FP64
      Profile<double> pd;
      pd.k = static_cast<double>(k);
      pd.k2 = 2.0 * pd.k;
      pd.bc = static_cast<double>(bmag) * static_cast<double>(cphi);
      pd.bs = static_cast<double>(bmag) * static_cast<double>(sphi);
      double e64[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = jq[q];
        const double S0 = g_grid_d[1][j], C0 = g_grid_d[2][j];
        double x = static_cast<double>(off[q]), sd, cd;
        Prec<double>::sincos_small(x, sd, cd);
        double s = fma(S0, cd, C0 * sd), c = fma(C0, cd, -S0 * sd);
        const double dd = pd.d2(s, c);
        if (dd != 0.0) x -= pd.d1(s, c) / dd;
        Prec<double>::sincos_small(x, sd, cd);
        s = fma(S0, cd, C0 * sd);
        c = fma(C0, cd, -S0 * sd);
        e64[q] = pd.e(s, c);
      }
      const double e3d = fmin(sel4(e64, imax0), sel4(e64, imax1));
      dEa = e3d - sel4(e64, wa);
      dEb = e3d - sel4(e64, wb);
    }
    o.dEa = dEa;
    o.dEb = dEb;
    int w = wa;
    if (!t_zero) {
      // vi) Eqs. 3-5 with nu t = exp(ln(nu0 t_step) - beta dE)
      const double ea = exp(lognu0t - beta * dEa);
      const double eb = exp(lognu0t - beta * dEb);
      const double sum = ea + eb;
      const double P = (sum > 0.0) ? (ea / sum) * (-expm1(-sum)) : 0.0;
      o.P = P;
      // vii) jump iff u < P
      o.near = fabs(u - P) < 1e-9;
      if (u < P) {
        o.flipped = 1;
        w = wb;
      }
    }
    s_new = sel4(sq, w);
    c_new = sel4(cq, w);
  }
  mx = fma(c_new, ax, s_new * ex);
  my = fma(c_new, ay, s_new * ey);
  mz = fma(c_new, az, s_new * ez);
  return o;
}

}  // namespace kmc
