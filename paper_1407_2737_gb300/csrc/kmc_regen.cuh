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
//     rho = disorder * (first uniform of sub 2), uniform on [0, disorder];
//   random sequential addition: candidate c (NP slot of the counter = c) is
//     uniform in the ball of centres, direction from sub 3 and radius
//     Rb max(u0, u1, u2) from subs 4 and 5.
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

// Uniform point on the unit sphere. Roundings are spelled out so that no
// product is fused into a subtraction: near the poles 1 - z^2 cancels, and a
// fused form would differ from the plain one by many ulps.
__device__ __forceinline__ void sphere_point(const double u[2], double &x, double &y, double &z) {
  z = __dsub_rn(1.0, __dmul_rn(2.0, u[0]));
  const double r2 = __dsub_rn(1.0, __dmul_rn(z, z));
  const double r = r2 > 0.0 ? sqrt(r2) : 0.0;
  double s, c;
  sincos(__dmul_rn(Prec<double>::two_pi, u[1]), &s, &c);
  x = __dmul_rn(r, c);
  y = __dmul_rn(r, s);
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
  if (a.what & (kRegenPositions | kRegenGiven)) {
    double px, py, pz;
    if (a.what & kRegenPositions) {
      double u[2], v[2], ex, ey, ez;
      regen_uniforms(a.seed, a.loop, 1u, i, a.lys, u);
      regen_uniforms(a.seed, a.loop, 2u, i, a.lys, v);
      sphere_point(u, ex, ey, ez);
      const double rho = __dmul_rn(a.disorder, v[0]);
      px = __dadd_rn(a.nodes[3 * g], __dmul_rn(rho, ex));
      py = __dadd_rn(a.nodes[3 * g + 1], __dmul_rn(rho, ey));
      pz = __dadd_rn(a.nodes[3 * g + 2], __dmul_rn(rho, ez));
      a.pos_si[3 * g] = px;
      a.pos_si[3 * g + 1] = py;
      a.pos_si[3 * g + 2] = pz;
    } else {
      px = a.pos_si[3 * g];
      py = a.pos_si[3 * g + 1];
      pz = a.pos_si[3 * g + 2];
    }
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

// Candidate c of the random sequential addition, about the lysosome centre.
__device__ __forceinline__ void rsa_candidate(double Rb, unsigned long long seed, uint32_t loop,
                                              long long c, int lys, double *p) {
  double u[2], v[2], w[2], ex, ey, ez;
  const int slot = static_cast<int>(static_cast<uint32_t>(c));
  regen_uniforms(seed, loop, 3u, slot, lys, u);
  regen_uniforms(seed, loop, 4u, slot, lys, v);
  regen_uniforms(seed, loop, 5u, slot, lys, w);
  sphere_point(u, ex, ey, ez);
  double x = v[0] > v[1] ? v[0] : v[1];
  if (w[0] > x) x = w[0];
  const double r = __dmul_rn(Rb, x);
  p[0] = __dmul_rn(r, ex);
  p[1] = __dmul_rn(r, ey);
  p[2] = __dmul_rn(r, ez);
}

// Squared distance, rounded as the definition reads it.
__device__ __forceinline__ double rsa_d2(const double *p, const double *q) {
  const double dx = __dsub_rn(p[0], q[0]), dy = __dsub_rn(p[1], q[1]), dz = __dsub_rn(p[2], q[2]);
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

__global__ void rsa_candidates_kernel(const RsaArgs a) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < a.B) rsa_candidate(a.Rb, a.seed, a.loop, a.c0 + k, a.lys, a.cand + 3 * k);
}

// Block k: does candidate k clear every sphere kept by earlier batches, and
// which earlier candidates of this batch lie closer than d. Against the kept
// spheres an FP32 squared distance settles the pair unless it falls within
// the margin [d2_lo, d2_hi] around d^2, which bounds the FP32 error for
// centres inside the ball; there the FP64 test of the definition decides.
__global__ void rsa_check_kernel(const RsaArgs a) {
  __shared__ int s_nconf;
  const int k = blockIdx.x;
  const int kept = *a.kept;
  const double *p = a.cand + 3 * k;
  const float px = static_cast<float>(p[0]), py = static_cast<float>(p[1]),
              pz = static_cast<float>(p[2]);
  bool clash = false;
  for (int j = threadIdx.x; j < kept && !clash; j += blockDim.x) {
    const float4 q = a.posf[j];
    const float dx = px - q.x, dy = py - q.y, dz = pz - q.z;
    const float d2f = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    if (d2f < a.d2_lo)
      clash = true;
    else if (d2f <= a.d2_hi)
      clash = rsa_d2(p, a.pos + 3 * j) < a.d2;
  }
  if (threadIdx.x == 0) s_nconf = 0;
  clash = __syncthreads_or(clash);
  if (!clash) {
    for (int j = threadIdx.x; j < k; j += blockDim.x)
      if (rsa_d2(p, a.cand + 3 * j) < a.d2) {
        const int q = atomicAdd(&s_nconf, 1);
        if (q < kRsaMaxConf) a.conf[k * kRsaMaxConf + q] = j;
      }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a.clear[k] = clash ? 0 : 1;
    a.nconf[k] = s_nconf;
  }
}

// The batch in candidate order: a candidate that cleared the earlier batches
// is kept unless a candidate kept earlier in this batch lies closer than d.
// That is the sequential rule, candidate by candidate. The walk is one thread
// on shared-memory copies (dynamic shared memory: rsa_resolve_smem(B) bytes);
// the kept centres are then copied out by the whole block.
__host__ __device__ constexpr size_t rsa_resolve_smem(int B) {
  return static_cast<size_t>(B) * (3 + kRsaMaxConf) * sizeof(int32_t);
}

__global__ void rsa_resolve_kernel(const RsaArgs a) {
  extern __shared__ int32_t rsa_sm[];
  int32_t *s_clear = rsa_sm, *s_nconf = rsa_sm + a.B, *s_slot = rsa_sm + 2 * a.B;
  int32_t *s_conf = rsa_sm + 3 * a.B;
  __shared__ int32_t s_kept;
  for (int k = threadIdx.x; k < a.B; k += blockDim.x) {
    s_clear[k] = a.clear[k];
    s_nconf[k] = a.nconf[k];
    s_slot[k] = -1;
  }
  for (int q = threadIdx.x; q < a.B * kRsaMaxConf; q += blockDim.x) s_conf[q] = a.conf[q];
  __syncthreads();
  if (threadIdx.x == 0) {
    int kept = *a.kept;
    for (int k = 0; k < a.B && kept < a.n; ++k) {
      bool ok = s_clear[k] != 0;
      if (ok) {
        const int nc = s_nconf[k];
        if (nc <= kRsaMaxConf) {
          for (int q = 0; q < nc && ok; ++q) ok = s_slot[s_conf[k * kRsaMaxConf + q]] < 0;
        } else {
          for (int j = 0; j < k && ok; ++j)
            ok = !(s_slot[j] >= 0 && rsa_d2(a.cand + 3 * k, a.cand + 3 * j) < a.d2);
        }
      }
      if (ok) {
        s_slot[k] = kept;
        if (++kept == a.n) *a.used = a.c0 + k + 1;
      }
    }
    s_kept = kept;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < a.B; k += blockDim.x) {
    const int sl = s_slot[k];
    if (sl >= 0) {
      const double x = a.cand[3 * k], y = a.cand[3 * k + 1], z = a.cand[3 * k + 2];
      a.pos[3 * sl] = x;
      a.pos[3 * sl + 1] = y;
      a.pos[3 * sl + 2] = z;
      a.posf[sl] = make_float4(static_cast<float>(x), static_cast<float>(y),
                               static_cast<float>(z), 0.0f);
    }
  }
  if (threadIdx.x == 0) *a.kept = s_kept;
}

}  // namespace kmc
