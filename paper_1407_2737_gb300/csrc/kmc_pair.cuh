// kmc_pair.cuh -- the FP32 pair term of Eq. 1 on packed f32x2 registers and
// the compensated sums used to add pair terms up. Shared by the step kernels
// (kmc_step.cu) and the no-allocation field (kmc_noalloc.cu), so that the
// two evaluate every pair with the same instructions in the same order.
#pragma once
#include <stdint.h>

#include "kmc_types.h"

namespace kmc {

// ---------------------------------------------------------------------------
// Packed FP32 pairs (f32x2) in 64-bit registers.
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk(float lo, float hi) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk(f2 v, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ float hsum(f2 v) {
  float lo, hi;
  upk(v, lo, hi);
  return lo + hi;
}

__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Kahan step: adds x to (s, c); the exact sum is s - c.
__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// Neumaier step: adds x to (s, c); the exact sum is s + c.
__device__ __forceinline__ void neumaier_add(float &s, float &c, float x) {
  const float t = s + x;
  if (fabsf(s) >= fabsf(x))
    c += (s - t) + x;
  else
    c += (x - t) + s;
  s = t;
}

struct AccF32 {
  f2 x, y, z;  // packed partial sums of the field (even / odd sources)
};

// One source record against the lane's target (X, Y, Z): the pair terms of
// both sources, 18 packed instructions and two rsqrt (see SrcPair).
template <bool MASK>
__device__ __forceinline__ void pair_record(const ulonglong2 &a, const ulonglong2 &b,
                                            const ulonglong2 &c, const ulonglong2 &d, f2 e,
                                            f2 X, f2 Y, f2 Z, AccF32 &acc) {
  const f2 dx = sub2(a.x, X), dy = sub2(a.y, Y), dz = sub2(b.x, Z);
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
  const f2 u = mul2(fma2(e, dz, fma2(d.y, dy, mul2(d.x, dx))), q2);
  acc.x = fma2(q3, fma2(u, dx, b.y), acc.x);
  acc.y = fma2(q3, fma2(u, dy, c.x), acc.y);
  acc.z = fma2(q3, fma2(u, dz, c.y), acc.z);
}

// Record r of a staged tile: x | y, z | nx, ny | nz, tx | ty, tz | padding.
__device__ __forceinline__ void load_record(const ulonglong2 *__restrict__ sp, int r,
                                            ulonglong2 &a, ulonglong2 &b, ulonglong2 &c,
                                            ulonglong2 &d, f2 &e) {
  const ulonglong2 *p = sp + kRecU2 * r;
  a = p[0];
  b = p[1];
  c = p[2];
  d = p[3];
  e = reinterpret_cast<const f2 *>(p + 4)[0];
}

}  // namespace kmc
