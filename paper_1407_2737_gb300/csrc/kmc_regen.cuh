// kmc_regen.cuh -- sample regeneration between loops on the device (Sec. II.4).
// Included only by kmc_step.cu, which owns the Philox generator.
//
// Between loops the paper draws fresh easy axes and, around fixed mean
// positions (the nodes of a cubic lattice), fresh positions. One thread per NP
// draws from Philox4x32-10 with key (seed lo, seed hi) and counter
// (loop, 0x80000000 | sub, NP, lysosome); the top bit of word 1 keeps these
// counters apart from those of the kMC draws, whose word 1 is the high half of
// a step index below 2^31. Two 53-bit uniforms come from each call, made like
// the kMC draw from words (0, 1) and (2, 3).
//   axes (sub 0): uniform on the sphere, z = 1 - 2 u0, azimuth 2 pi u1;
//   positions: node + rho e, e uniform on the sphere from sub 1 and
//     rho = disorder * (first uniform of sub 2), uniform on [0, disorder].
// The NP's arrays are then rewritten as creation builds them (unit axis,
// position in the lysosome's frame, moment along the axis with m_z >= 0).
#pragma once

namespace kmc {

__device__ __forceinline__ void regen_uniforms(unsigned long long seed, uint32_t loop,
                                               uint32_t sub, int np, int lys, double u[2]) {
  const uint4 w = philox4x32_10(
      make_uint4(loop, 0x80000000u | sub, static_cast<uint32_t>(np), static_cast<uint32_t>(lys)),
      make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32)));
  u[0] = static_cast<double>((static_cast<unsigned long long>(w.x) << 21) ^
                             static_cast<unsigned long long>(w.y >> 11)) * 0x1.0p-53;
  u[1] = static_cast<double>((static_cast<unsigned long long>(w.z) << 21) ^
                             static_cast<unsigned long long>(w.w >> 11)) * 0x1.0p-53;
}

__device__ __forceinline__ void sphere_point(const double u[2], double &x, double &y, double &z) {
  z = 1.0 - 2.0 * u[0];
  const double r2 = 1.0 - z * z;
  const double r = r2 > 0.0 ? sqrt(r2) : 0.0;
  double s, c;
  sincos(Prec<double>::two_pi * u[1], &s, &c);
  x = r * c;
  y = r * s;
}

__global__ void kmc_regen_kernel(const RegenArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int g = a.off + i;
  double ax, ay, az;
  if (a.what & kRegenAxes) {
    double u[2];
    regen_uniforms(a.seed, a.loop, 0u, i, a.lys, u);
    sphere_point(u, ax, ay, az);
    const double an = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay)),
                                     __dmul_rn(az, az)));
    ax /= an;
    ay /= an;
    az /= an;
  } else if (a.fp32) {
    const float4 v = static_cast<const float4 *>(a.axis)[g];
    ax = v.x;
    ay = v.y;
    az = v.z;
  } else {
    const dbl4 v = static_cast<const dbl4 *>(a.axis)[g];
    ax = v.x;
    ay = v.y;
    az = v.z;
  }
  if (a.what & kRegenPositions) {
    double u[2], v[2], ex, ey, ez;
    regen_uniforms(a.seed, a.loop, 1u, i, a.lys, u);
    regen_uniforms(a.seed, a.loop, 2u, i, a.lys, v);
    sphere_point(u, ex, ey, ez);
    const double rho = a.disorder * v[0];
    const double px = a.nodes[3 * g] + rho * ex, py = a.nodes[3 * g + 1] + rho * ey,
                 pz = a.nodes[3 * g + 2] + rho * ez;
    a.pos_si[3 * g] = px;
    a.pos_si[3 * g + 1] = py;
    a.pos_si[3 * g + 2] = pz;
    const double x = (px - a.cx) / a.len, y = (py - a.cy) / a.len, z = (pz - a.cz) / a.len;
    if (a.fp32) {
      float4 &p4 = static_cast<float4 *>(a.pos)[g];
      p4 = make_float4(static_cast<float>(x), static_cast<float>(y), static_cast<float>(z), p4.w);
      dbl4 &q4 = static_cast<dbl4 *>(a.pos64)[g];
      q4.x = x;
      q4.y = y;
      q4.z = z;
    } else {
      dbl4 &p4 = static_cast<dbl4 *>(a.pos)[g];
      p4.x = x;
      p4.y = y;
      p4.z = z;
    }
  }
  const double sgn = az >= 0.0 ? 1.0 : -1.0;
  if (a.fp32) {
    const float fx = static_cast<float>(ax), fy = static_cast<float>(ay), fz = static_cast<float>(az);
    if (a.what & kRegenAxes) static_cast<float4 *>(a.axis)[g] = make_float4(fx, fy, fz, 0.0f);
    const float fs = static_cast<float>(sgn);
    static_cast<float4 *>(a.m)[g] = make_float4(fs * fx, fs * fy, fs * fz, 0.0f);
  } else {
    dbl4 v;
    v.w = 0.0;
    if (a.what & kRegenAxes) {
      v.x = ax;
      v.y = ay;
      v.z = az;
      static_cast<dbl4 *>(a.axis)[g] = v;
    }
    v.x = sgn * ax;
    v.y = sgn * ay;
    v.z = sgn * az;
    static_cast<dbl4 *>(a.m)[g] = v;
  }
}

}  // namespace kmc
