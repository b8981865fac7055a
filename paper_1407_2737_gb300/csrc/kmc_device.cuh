// kmc_device.cuh -- device building blocks of the kMC step (sm_103a): the
// Philox4x32-10 draw and the per-NP update of steps iii-vii of Sec. II.1
// (the bulk-copy staging is in kmc_stage.cuh).
#pragma once
#include <stdint.h>

#include <type_traits>

#include "kmc_stage.cuh"
#include "kmc_types.h"

namespace kmc {

// Grid of step iv: theta_j = 2 pi (j + 1/2) / 200 and (sin, cos) of it,
// written once per device by init_device (kmc_step.cu, the only translation
// unit that includes this header).
// (16-byte aligned: the FP32 step kernels copy them to shared memory in bulk)
__device__ __align__(16) float g_theta_f[kGrid];
__device__ __align__(16) float2 g_sc_f[kGrid];
// The same sin and cos in two arrays of their own, node j at j mod kGrid for
// j < kGridPad, so that the FP32 scan reads two consecutive nodes as one
// packed pair, past the end of the grid too.
constexpr int kGridPad = kGrid + 16;
__device__ __align__(16) float g_ss_f[kGridPad];
__device__ __align__(16) float g_cc_f[kGridPad];
__device__ double g_theta_d[kGrid];
__device__ double2 g_sc_d[kGrid];

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
  // Newton stops once a step is below newton_tol (absolute, on the offset in
  // a cell of 0.0314 rad). With de/dth and its derivative in FP32 the step
  // itself carries rounding noise of order 1e-8..1e-7 rad, so the tolerance
  // sits above it: a tighter one is never met and every root runs to
  // newton_max. From the secant start the convergence is quadratic, so the
  // root is then within rounding (~1e-7 rad) after 2-3 steps.
  static constexpr float newton_tol = 3e-7f;
  static constexpr int newton_max = 6;
  __device__ static float div(float a, float b) { return __fdividef(a, b); }
  __device__ static float theta(int j) { return g_theta_f[j]; }
  __device__ static float2 sc(int j) { return g_sc_f[j]; }
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
  __device__ static double div(double a, double b) { return a / b; }
  __device__ static double theta(int j) { return g_theta_d[j]; }
  __device__ static double2 sc(int j) { return g_sc_d[j]; }
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

// Copy of the grid of step iv in shared memory, filled by every block at its
// start (the pair loop hides the loads); the scan reads one node per warp
// (a broadcast), Newton one node per thread.
template <typename R>
struct ScanPairs {};
template <>
struct ScanPairs<float> {
  float ss[kGridPad], cc[kGridPad];  // g_ss_f, g_cc_f
};
template <typename R>
struct GridTables : ScanPairs<R> {
  typename std::conditional<std::is_same<R, float>::value, float2, double2>::type sc[kGrid];
  R th[kGrid];
  __device__ void load() {
    for (int j = threadIdx.x; j < kGrid; j += blockDim.x) {
      sc[j] = Prec<R>::sc(j);
      th[j] = Prec<R>::theta(j);
    }
    if constexpr (std::is_same<R, float>::value) {
      for (int j = threadIdx.x; j < kGridPad; j += blockDim.x) {
        this->ss[j] = g_ss_f[j];
        this->cc[j] = g_cc_f[j];
      }
    }
  }
};
static_assert(sizeof(GridTables<float>::sc) % 16 == 0 && sizeof(GridTables<float>::th) % 16 == 0 &&
                  sizeof(ScanPairs<float>::ss) % 16 == 0 && sizeof(ScanPairs<float>) % 16 == 0,
              "the FP32 tables are copied in bulk");

// de/dth of Eq. 2 at (sin, cos) = (s, c): s (2k c + b cos phi) - b sin phi c,
// with its roundings spelled out so that every evaluation at a node gives the
// same bits wherever the compiler places it (the scan tests the sign of values
// that can sit within rounding of zero, and evaluates each node twice).
__device__ __forceinline__ float profile_d1(float k2, float bc, float bs, float s, float c) {
  return __fmaf_rn(s, __fmaf_rn(k2, c, bc), -__fmul_rn(bs, c));
}
__device__ __forceinline__ double profile_d1(double k2, double bc, double bs, double s,
                                             double c) {
  return __fma_rn(s, __fma_rn(k2, c, bc), -__dmul_rn(bs, c));
}

// Eq. 2 in a working plane: e = k sin^2 th - b cos(th - phi);
// de/dth = 2k s c + b (s cos phi - c sin phi); d2e = 2k (c^2 - s^2) + b (c cos phi + s sin phi).
template <typename R>
struct Profile {
  R k2;  // 2k
  R k;
  R bc;  // b cos phi
  R bs;  // b sin phi
  __device__ R d1(R s, R c) const { return profile_d1(k2, bc, bs, s, c); }
  __device__ R d2(R s, R c) const { return k2 * (c * c - s * s) + fma(bc, c, bs * s); }
  __device__ R e(R s, R c) const { return k * s * s - fma(bc, c, bs * s); }
};

// Newton's method with bisection fallback for the root of de/dth inside grid
// cell [theta_j, theta_j + h], as offset d from theta_j. dlo, dhi = de/dth at
// theta_j and theta_j + h (opposite signs); the first iterate is the secant
// point, so that two or three Newton steps reach the root.
template <typename R>
__device__ __forceinline__ R refine_in_cell(const Profile<R> &pf, R S0, R C0, R h, R dlo,
                                            R dhi, R &s_out, R &c_out) {
  R lo = R(0), hi = h;
  R x = (dlo != dhi) ? h * Prec<R>::div(dlo, dlo - dhi) : R(0.5) * h;
  if (!(x > lo && x < hi)) x = R(0.5) * h;
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
    R xn = (dd != R(0)) ? x - Prec<R>::div(d, dd) : R(0.5) * (lo + hi);
    // Converged: the step is below the tolerance. Tested before the bracket
    // safeguard, because a step that rounds to nothing leaves xn on the
    // bracket end that x itself just became, and the safeguard would then
    // bisect away from the root it has found.
    if (fabs(xn - x) < Prec<R>::newton_tol) {
      x = xn;
      break;
    }
    if (!(xn > lo && xn < hi)) xn = R(0.5) * (lo + hi);
    const bool done = hi - lo < Prec<R>::newton_tol;
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

}  // namespace kmc
