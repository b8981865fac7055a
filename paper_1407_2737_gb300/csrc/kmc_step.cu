// kmc_step.cu -- the fused kMC step kernels of libkmc (sm_103a).
//
// One launch = one time step of every NP of every lysosome (Sec. II.1 steps
// i-vii; the update is synchronous, Sec. II.2, so every block reads the
// moments of the start of the step and writes the other ping-pong buffer).
//
// Block = (lysosome l, 32 target NPs), NW warps. The lysosome's sources are
// streamed through shared memory in tiles of TJ NPs by bulk asynchronous
// copies (cp.async.bulk, double-buffered, completion on an mbarrier). Each warp
// takes every NW-th source of a tile for the same 32 targets (one per lane),
// so each shared-memory load is a broadcast. Partial sums of each tile are
// folded into a compensated (Kahan) per-warp sum, the NW warp sums are combined
// with Neumaier's compensated summation, and warp 0 runs steps iii-vii for its
// 32 NPs straight from registers: the dipolar field never goes to memory.
//
// Pair term (Eq. 1 in reduced units), 19 FP32 operations + 1 reciprocal
// square root: d = r_j - r_i; r2 = |d|^2; q = rsqrt(r2); q3 = q^3;
// s = (mu_j . d) q^2 q3; A += s d; B += q3 mu_j; b_dip = 3A - B.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include "kmc_device.cuh"
#include "kmc_launch.h"

namespace kmc {

__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Kahan step: adds x to (s, c).
__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// Neumaier step: adds x to (s, c) where c collects the rounding errors.
__device__ __forceinline__ void neumaier_add(float &s, float &c, float x) {
  const float t = s + x;
  if (fabsf(s) >= fabsf(x))
    c += (s - t) + x;
  else
    c += (x - t) + s;
  s = t;
}

template <typename V>
struct SrcTraits;
template <>
struct SrcTraits<float4> {
  using R = float;
};
template <>
struct SrcTraits<dbl4> {
  using R = double;
};

// ---------------------------------------------------------------------------
// Pair loops over one staged tile. MASK: the tile holds some of the block's
// own targets, so the self term (r2 = 0; distinct NPs are never coincident)
// is dropped.

template <bool MASK>
__device__ __forceinline__ void pair_tile_f32(const float4 *__restrict__ sp,
                                              const float4 *__restrict__ sm, int cnt,
                                              int first, int stride, float xi, float yi,
                                              float zi, float &ax, float &ay, float &az,
                                              float &bx, float &by, float &bz) {
#pragma unroll 4
  for (int j = first; j < cnt; j += stride) {
    const float4 p = sp[j];
    const float4 q = sm[j];
    const float dx = p.x - xi, dy = p.y - yi, dz = p.z - zi;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float inv = rsqrt_approx(r2);
    if (MASK) inv = (r2 > 0.0f) ? inv : 0.0f;
    const float inv2 = inv * inv;
    const float inv3 = inv * inv2;
    const float md = fmaf(q.x, dx, fmaf(q.y, dy, q.z * dz));
    const float s = md * inv2 * inv3;
    ax = fmaf(s, dx, ax);
    ay = fmaf(s, dy, ay);
    az = fmaf(s, dz, az);
    bx = fmaf(inv3, q.x, bx);
    by = fmaf(inv3, q.y, by);
    bz = fmaf(inv3, q.z, bz);
  }
}

__device__ __forceinline__ void pair_tile_f64(const dbl4 *__restrict__ sp,
                                              const dbl4 *__restrict__ sm, int cnt, int first,
                                              int stride, double xi, double yi, double zi,
                                              double &ax, double &ay, double &az, double &bx,
                                              double &by, double &bz) {
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
      ax = fma(s, dx, ax);
      ay = fma(s, dy, ay);
      az = fma(s, dz, az);
      bx = fma(inv3, q.x, bx);
      by = fma(inv3, q.y, by);
      bz = fma(inv3, q.z, bz);
    }
  }
}

// ---------------------------------------------------------------------------
// Per-NP epilogue shared by both precisions: steps iii-vii, outputs, energy,
// loop and counters. Runs in warp 0; lane = target within the block.

template <typename V, bool MIXED>
__device__ __forceinline__ void epilogue(const StepArgs &a, const LysDev &L, int l, int i0,
                                         int nt, int lane, typename SrcTraits<V>::R hx,
                                         typename SrcTraits<V>::R hy,
                                         typename SrcTraits<V>::R hz, long long step,
                                         int rec) {
  using R = typename SrcTraits<V>::R;
  const bool active = lane < nt;
  const int il = i0 + (active ? lane : 0);  // NP index within the lysosome
  const int i = L.off + il;                 // flat NP index
  const double bext = L.bmax * a.cos_k;
  const V ax4 = static_cast<const V *>(a.axis)[i];
  V m4 = static_cast<V *>(a.m)[i];
  const R mz_old = m4.z;
  R mx = m4.x, my = m4.y, mz = m4.z;
  const double u = kmc_uniform(a.seed, step, il, l);
  const NPResult r = np_update<R, MIXED>(ax4.x, ax4.y, ax4.z, mx, my, mz, hx, hy,
                                         hz + static_cast<R>(bext), static_cast<R>(L.k),
                                         a.beta[i], L.lognu0t, L.t_zero != 0, u);
  if (active) {
    m4.x = mx;
    m4.y = my;
    m4.z = mz;
    static_cast<V *>(a.m)[i] = m4;
    const R w = static_cast<const V *>(a.pos)[i].w;
    V mu4;
    mu4.x = w * mx;
    mu4.y = w * my;
    mu4.z = w * mz;
    mu4.w = R(0);
    const int par = static_cast<int>(step & 1);
    static_cast<V *>(a.mu[par ^ 1])[i] = mu4;
    if (rec >= 0)
      a.e_acc[i] += bext * (static_cast<double>(mz) - static_cast<double>(mz_old));
    if (a.debug) {
      a.dbg.bdip[3 * i + 0] = static_cast<double>(hx);
      a.dbg.bdip[3 * i + 1] = static_cast<double>(hy);
      a.dbg.bdip[3 * i + 2] = static_cast<double>(hz);
      a.dbg.dE[2 * i + 0] = r.dEa;
      a.dbg.dE[2 * i + 1] = r.dEb;
      a.dbg.P[i] = r.P;
      a.dbg.u[i] = u;
      a.dbg.flags[i] = r.nmin | (r.flipped << 2) | (r.near << 3) | (r.degenerate << 4);
    }
  }
  // loop record and counters: one atomic per block
  if (rec >= 0) {
    double c = active ? a.vfrac[i] * static_cast<double>(mz) : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if (lane == 0) atomicAdd(&a.loop_m[static_cast<long long>(l) * a.n_rec + rec], c);
  }
  const unsigned fl = __ballot_sync(0xffffffffu, active && r.flipped);
  const unsigned ne = __ballot_sync(0xffffffffu, active && r.near);
  const unsigned mo = __ballot_sync(0xffffffffu, active && r.nmin == 1);
  const unsigned dg = __ballot_sync(0xffffffffu, active && r.degenerate);
  const unsigned bd = __ballot_sync(0xffffffffu, active && r.bad);
  if (lane == 0) {
    unsigned long long *c = a.counters + 4ll * l;
    if (fl) atomicAdd(c + 0, static_cast<unsigned long long>(__popc(fl)));
    if (ne) atomicAdd(c + 1, static_cast<unsigned long long>(__popc(ne)));
    if (mo) atomicAdd(c + 2, static_cast<unsigned long long>(__popc(mo)));
    if (dg) atomicAdd(c + 3, static_cast<unsigned long long>(__popc(dg)));
    if (bd) atomicOr(a.err, kErrExtrema);
  }
}

// ---------------------------------------------------------------------------
// The fused step kernel. V = float4 (FP32-mixed) or dbl4 (FP64-plain).

template <typename V, int NW>
__global__ void __launch_bounds__(NW * 32) kmc_step_kernel(const StepArgs a, int TJ) {
  using R = typename SrcTraits<V>::R;
  constexpr bool MIXED = sizeof(R) == 4;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  V *spos = reinterpret_cast<V *>(smem_raw);  // [2][TJ]
  V *smu = spos + 2 * TJ;                     // [2][TJ]
  R *red = reinterpret_cast<R *>(smu + 2 * TJ);  // [NW][12][32]
  uint64_t *bar = reinterpret_cast<uint64_t *>(red + NW * 12 * 32);  // [2]

  const int4 it = a.items[blockIdx.x];
  const int l = it.x, i0 = it.y, nt = it.z;
  const LysDev L = a.lys[l];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long step = a.rs->step_base + a.k_local;
  const int per = a.rs->period;
  const int rec = (per >= a.discard) ? (per - a.discard) * a.S + a.k_local : -1;
  const int par = static_cast<int>(step & 1);
  const V *__restrict__ gpos = static_cast<const V *>(a.pos) + L.off;
  const V *__restrict__ gmu = static_cast<const V *>(a.mu[par]) + L.off;

  const int ti = i0 + min(lane, nt - 1);
  const V pi = gpos[ti];
  R ax = R(0), ay = R(0), az = R(0), bx = R(0), by = R(0), bz = R(0);
  // compensated per-warp running sums (FP32 path): value and Kahan term
  R sax = R(0), say = R(0), saz = R(0), sbx = R(0), sby = R(0), sbz = R(0);
  R cax = R(0), cay = R(0), caz = R(0), cbx = R(0), cby = R(0), cbz = R(0);

  const int ntiles = (L.n + TJ - 1) / TJ;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
  }
  __syncthreads();
  auto issue = [&](int t) {
    const int b = t & 1;
    const int j0 = t * TJ;
    const int cnt = min(TJ, L.n - j0);
    const uint32_t bytes = static_cast<uint32_t>(cnt) * sizeof(V);
    mbar_expect_tx(&bar[b], 2 * bytes);
    bulk_g2s(spos + b * TJ, gpos + j0, bytes, &bar[b]);
    bulk_g2s(smu + b * TJ, gmu + j0, bytes, &bar[b]);
  };
  if (threadIdx.x == 0) {
    issue(0);
    if (ntiles > 1) issue(1);
  }
  for (int t = 0; t < ntiles; ++t) {
    const int b = t & 1;
    const int j0 = t * TJ;
    const int cnt = min(TJ, L.n - j0);
    const bool ok = mbar_wait_bounded(&bar[b], (t >> 1) & 1, a.err);
    const bool mask = (j0 < i0 + nt) && (i0 < j0 + cnt);
    if (!ok) {
      // the copy never landed: error word set, results invalid
    } else if constexpr (MIXED) {
      float tax = 0.f, tay = 0.f, taz = 0.f, tbx = 0.f, tby = 0.f, tbz = 0.f;
      if (mask)
        pair_tile_f32<true>(spos + b * TJ, smu + b * TJ, cnt, warp, NW, pi.x, pi.y, pi.z, tax,
                            tay, taz, tbx, tby, tbz);
      else
        pair_tile_f32<false>(spos + b * TJ, smu + b * TJ, cnt, warp, NW, pi.x, pi.y, pi.z, tax,
                             tay, taz, tbx, tby, tbz);
      kahan_add(sax, cax, tax);
      kahan_add(say, cay, tay);
      kahan_add(saz, caz, taz);
      kahan_add(sbx, cbx, tbx);
      kahan_add(sby, cby, tby);
      kahan_add(sbz, cbz, tbz);
    } else {
      pair_tile_f64(spos + b * TJ, smu + b * TJ, cnt, warp, NW, pi.x, pi.y, pi.z, ax, ay, az, bx,
                    by, bz);
    }
    // every warp is done with buffer b; a failed wait anywhere stops all
    if (!__syncthreads_and(ok)) return;
    if (threadIdx.x == 0 && t + 2 < ntiles) {
      proxy_fence_shared();
      issue(t + 2);
    }
  }
  if constexpr (MIXED) {
    ax = sax;
    ay = say;
    az = saz;
    bx = sbx;
    by = sby;
    bz = sbz;
  }
  // cross-warp combine through shared memory (fixed order: deterministic)
  R *rw = red + warp * 12 * 32;
  rw[0 * 32 + lane] = ax;
  rw[1 * 32 + lane] = ay;
  rw[2 * 32 + lane] = az;
  rw[3 * 32 + lane] = bx;
  rw[4 * 32 + lane] = by;
  rw[5 * 32 + lane] = bz;
  rw[6 * 32 + lane] = cax;
  rw[7 * 32 + lane] = cay;
  rw[8 * 32 + lane] = caz;
  rw[9 * 32 + lane] = cbx;
  rw[10 * 32 + lane] = cby;
  rw[11 * 32 + lane] = cbz;
  __syncthreads();
  if (warp != 0) return;
  R h[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if constexpr (MIXED) {
      float sa = 0.f, ca = 0.f, sb = 0.f, cb = 0.f;
      for (int w = 0; w < NW; ++w) {
        neumaier_add(sa, ca, red[w * 384 + c * 32 + lane]);
        ca -= red[w * 384 + (6 + c) * 32 + lane];  // Kahan terms hold minus the error
        neumaier_add(sb, cb, red[w * 384 + (3 + c) * 32 + lane]);
        cb -= red[w * 384 + (9 + c) * 32 + lane];
      }
      // b_dip = 3A - B with the compensations added last
      float s = 0.f, cc = 0.f;
      neumaier_add(s, cc, 3.0f * sa);
      neumaier_add(s, cc, -sb);
      neumaier_add(s, cc, 3.0f * ca - cb);
      h[c] = s + cc;
    } else {
      double sa = 0.0, sb = 0.0;
      for (int w = 0; w < NW; ++w) {
        sa += red[w * 384 + c * 32 + lane];
        sb += red[w * 384 + (3 + c) * 32 + lane];
      }
      h[c] = 3.0 * sa - sb;
    }
  }
  epilogue<V, MIXED>(a, L, l, i0, nt, lane, h[0], h[1], h[2], step, rec);
}

// Ends a field period on the device: the next period starts S steps later.
__global__ void kmc_advance_kernel(RunState *rs, int S) {
  rs->step_base += S;
  rs->period += 1;
}

// ---------------------------------------------------------------------------
// Host side of the launches.

size_t step_smem_bytes(int prec_fp32, int warps, int tile) {
  const size_t v = prec_fp32 ? sizeof(float4) : sizeof(dbl4);
  const size_t r = prec_fp32 ? sizeof(float) : sizeof(double);
  return 4 * static_cast<size_t>(tile) * v + static_cast<size_t>(warps) * 12 * 32 * r + 16;
}

template <typename V, int NW>
static cudaError_t launch_t(const StepArgs &a, int n_items, int tile, cudaStream_t st) {
  const size_t smem = step_smem_bytes(sizeof(V) == sizeof(float4), NW, tile);
  kmc_step_kernel<V, NW><<<n_items, NW * 32, smem, st>>>(a, tile);
  return cudaGetLastError();
}

template <typename V, int NW>
static cudaError_t allow_smem() {
  return cudaFuncSetAttribute(kmc_step_kernel<V, NW>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxStepSmem);
}

cudaError_t launch_step(int prec_fp32, int warps, int tile, const StepArgs &a, int n_items,
                        cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  if (prec_fp32) {
    switch (warps) {
      case 4: return launch_t<float4, 4>(a, n_items, tile, st);
      case 8: return launch_t<float4, 8>(a, n_items, tile, st);
      case 16: return launch_t<float4, 16>(a, n_items, tile, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (warps) {
    case 4: return launch_t<dbl4, 4>(a, n_items, tile, st);
    case 8: return launch_t<dbl4, 8>(a, n_items, tile, st);
    case 16: return launch_t<dbl4, 16>(a, n_items, tile, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_advance(RunState *rs, int S, cudaStream_t st) {
  kmc_advance_kernel<<<1, 1, 0, st>>>(rs, S);
  return cudaGetLastError();
}

cudaError_t init_device() {
  float f[3][kGrid];
  double d[3][kGrid];
  const double two_pi = 6.283185307179586476925286766559;
  for (int j = 0; j < kGrid; ++j) {
    d[0][j] = two_pi * (static_cast<double>(j) + 0.5) / static_cast<double>(kGrid);
    d[1][j] = sin(d[0][j]);
    d[2][j] = cos(d[0][j]);
    for (int q = 0; q < 3; ++q) f[q][j] = static_cast<float>(d[q][j]);
  }
  cudaError_t e = cudaMemcpyToSymbol(g_grid_f, f, sizeof(f));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_grid_d, d, sizeof(d));
  // kernel attributes are set here, never inside a stream capture
  if (e == cudaSuccess) e = allow_smem<float4, 4>();
  if (e == cudaSuccess) e = allow_smem<float4, 8>();
  if (e == cudaSuccess) e = allow_smem<float4, 16>();
  if (e == cudaSuccess) e = allow_smem<dbl4, 4>();
  if (e == cudaSuccess) e = allow_smem<dbl4, 8>();
  if (e == cudaSuccess) e = allow_smem<dbl4, 16>();
  return e;
}

}  // namespace kmc
