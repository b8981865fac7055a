// pair_forms.cu -- measures two ways of evaluating the pair terms of Eq. 1
// (the dipolar field of every NP from all others) on one GB300, over source
// tiles resident in shared memory (no staging, no update), so that only the
// arithmetic of the pair loop is timed:
//
//  * ordered pairs, the library's form (kmc_pair.cuh, used by the step
//    kernels): every (target, source) pair is evaluated once for its target;
//    each warp broadcasts one staged record of two sources to its lanes, each
//    lane holding 1, 2 or 3 targets. 18 packed FP32 operations and 2 rsqrt per
//    record and target, i.e. per two ordered pairs.
//  * symmetric pairs by lane rotation (T_ij = T_ji, so the geometry of a pair
//    serves both of its ordered pairs): a warp takes 32 targets against 32
//    sources; at step s lane L meets source (L + s) mod 32, read from shared
//    memory, adds the forward term to its own target's sum and the reverse
//    term to the reverse sum it carries for that source; the reverse sums move
//    one lane per step by warp shuffles, so that after 32 steps lane L holds
//    the complete reverse sum of source L. 28 scalar FP32 operations, 1 rsqrt
//    and 3 shuffles per pair, i.e. per two ordered pairs.
//
// Both forms are first checked against the definition in FP64 on the host.
// Each prints one line: name, ordered pairs per second, the fraction of the
// nominal FP32 peak at 30 flops per ordered pair, and the largest relative
// error of the check. Sources and targets are drawn uniformly in a ball of
// radius 40 (units of the NP diameter, the 50 000-NP lysosome's radius) by a
// fixed-seed generator; the timing does not depend on the values (the loops
// have no data-dependent branches).
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 \
//        --expt-relaxed-constexpr -I<csrc> pair_forms.cu -o pair_forms
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "kmc_pair.cuh"

using namespace kmc;

namespace {

constexpr int kTile = 256;  // source records (two sources each) resident per block
constexpr int kWarps = 4;
constexpr double kBall = 40.0;

// ---------------------------------------------------------------------------
// Ordered pairs: the step kernels' record loop over a resident tile, TPL
// targets per lane, repeated `reps` times.
template <int TPL>
__global__ void __launch_bounds__(kWarps * 32)
    ordered_pairs(const SrcPair *__restrict__ rec, const float4 *__restrict__ tgt, int reps,
                  float *__restrict__ out) {
  __shared__ __align__(16) ulonglong2 sm[kTile * kRecU2];
  const ulonglong2 *g = reinterpret_cast<const ulonglong2 *>(rec);
  for (int i = threadIdx.x; i < kTile * kRecU2; i += blockDim.x) sm[i] = g[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  f2 X[TPL], Y[TPL], Z[TPL];
  AccF32 acc[TPL];
#pragma unroll
  for (int k = 0; k < TPL; ++k) {
    const float4 p = tgt[(blockIdx.x * TPL + k) * 32 + lane];
    X[k] = pk(p.x, p.x);
    Y[k] = pk(p.y, p.y);
    Z[k] = pk(p.z, p.z);
    acc[k].x = acc[k].y = acc[k].z = 0ull;
  }
  for (int rep = 0; rep < reps; ++rep) {
#pragma unroll 1
    for (int r = warp; r < kTile; r += kWarps) {
      ulonglong2 a, b, c, d;
      f2 e;
      load_record(sm, r, a, b, c, d, e);
#pragma unroll
      for (int k = 0; k < TPL; ++k) pair_record<false>(a, b, c, d, e, X[k], Y[k], Z[k], acc[k]);
    }
  }
  // per warp and target: this warp's share of the field (the check adds the warps)
#pragma unroll
  for (int k = 0; k < TPL; ++k) {
    float *o = out + ((static_cast<size_t>(blockIdx.x) * TPL + k) * kWarps + warp) * 32 * 3;
    o[lane * 3 + 0] = hsum(acc[k].x);
    o[lane * 3 + 1] = hsum(acc[k].y);
    o[lane * 3 + 2] = hsum(acc[k].z);
  }
}

// One NP of the symmetric form: position and moment terms t = 3 w m, n = -w m.
struct Np {
  float x, y, z, tx, ty, tz, nx, ny, nz, pad[3];
};

// Symmetric pairs by lane rotation: warp w of block b takes targets
// tgt[(b W + w) 32 + L] against sources src[(b W + w) 32 + L].
__global__ void __launch_bounds__(kWarps * 32)
    symmetric_pairs(const Np *__restrict__ src, const Np *__restrict__ tgt, int reps,
                    float *__restrict__ fwd, float *__restrict__ rev) {
  __shared__ __align__(16) Np sm[kWarps][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t base = (static_cast<size_t>(blockIdx.x) * kWarps + warp) * 32;
  sm[warp][lane] = src[base + lane];
  __syncwarp();
  const Np me = tgt[base + lane];
  float ax = 0.f, ay = 0.f, az = 0.f;  // forward sum of this lane's target
  float rx = 0.f, ry = 0.f, rz = 0.f;  // reverse sum of the source this lane meets
  for (int rep = 0; rep < reps; ++rep) {
#pragma unroll 4
    for (int s = 0; s < 32; ++s) {
      const Np q = sm[warp][(lane + s) & 31];
      const float dx = q.x - me.x, dy = q.y - me.y, dz = q.z - me.z;
      const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
      float i1;
      asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(i1) : "f"(r2));
      const float i2 = i1 * i1, i3 = i1 * i2;
      // forward: the field at the target from the source, q3 (u d + n_j)
      const float uf = fmaf(q.tz, dz, fmaf(q.ty, dy, q.tx * dx)) * i2;
      ax = fmaf(i3, fmaf(uf, dx, q.nx), ax);
      ay = fmaf(i3, fmaf(uf, dy, q.ny), ay);
      az = fmaf(i3, fmaf(uf, dz, q.nz), az);
      // reverse: the field at the source from the target; d changes sign twice
      const float ur = fmaf(me.tz, dz, fmaf(me.ty, dy, me.tx * dx)) * i2;
      rx = fmaf(i3, fmaf(ur, dx, me.nx), rx);
      ry = fmaf(i3, fmaf(ur, dy, me.ny), ry);
      rz = fmaf(i3, fmaf(ur, dz, me.nz), rz);
      // lane L takes the reverse sum of source L + s + 1 from lane L + 1
      rx = __shfl_sync(0xffffffffu, rx, (lane + 1) & 31);
      ry = __shfl_sync(0xffffffffu, ry, (lane + 1) & 31);
      rz = __shfl_sync(0xffffffffu, rz, (lane + 1) & 31);
    }
  }
  fwd[(base + lane) * 3 + 0] = ax;
  fwd[(base + lane) * 3 + 1] = ay;
  fwd[(base + lane) * 3 + 2] = az;
  rev[(base + lane) * 3 + 0] = rx;
  rev[(base + lane) * 3 + 1] = ry;
  rev[(base + lane) * 3 + 2] = rz;
}

// Symmetric pairs on packed records: warp w of block b holds TPL x 32 targets
// (lane L: targets L, 32 + L, ...) and 32 source records (64 sources) of the
// library's layout in shared memory. At step s lane L reads record
// (L + s) mod 32 and forms, per target, the geometry of its two pairs once
// (8 packed operations, 2 rsqrt), the forward terms into the target's sums
// (10) and the reverse terms into the record's two reverse sums (10): 28 packed
// operations per four ordered pairs. The reverse sums (3 packed registers)
// move one lane per step (6 shuffles), so that after 32 steps lane L holds
// record L's. The reverse term of target i at source j is q^3 (v d + n_i)
// with v = (t_i . d) q^2 and d = r_j - r_i, as -d enters it twice.
template <int TPL>
__global__ void __launch_bounds__(kWarps * 32)
    symmetric_packed(const SrcPair *__restrict__ rec, const Np *__restrict__ tgt, int reps,
                     float *__restrict__ fwd, float *__restrict__ rev) {
  __shared__ __align__(16) ulonglong2 sm[kWarps * 32 * kRecU2];
  const ulonglong2 *g =
      reinterpret_cast<const ulonglong2 *>(rec) + static_cast<size_t>(blockIdx.x) * kWarps * 32 * kRecU2;
  for (int i = threadIdx.x; i < kWarps * 32 * kRecU2; i += blockDim.x) sm[i] = g[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const ulonglong2 *my = sm + warp * 32 * kRecU2;
  const size_t tb = (static_cast<size_t>(blockIdx.x) * kWarps + warp) * 32 * TPL;
  f2 X[TPL], Y[TPL], Z[TPL], TX[TPL], TY[TPL], TZ[TPL], NX[TPL], NY[TPL], NZ[TPL];
  AccF32 acc[TPL];
#pragma unroll
  for (int k = 0; k < TPL; ++k) {
    const Np q = tgt[tb + k * 32 + lane];
    X[k] = pk(q.x, q.x);
    Y[k] = pk(q.y, q.y);
    Z[k] = pk(q.z, q.z);
    TX[k] = pk(q.tx, q.tx);
    TY[k] = pk(q.ty, q.ty);
    TZ[k] = pk(q.tz, q.tz);
    NX[k] = pk(q.nx, q.nx);
    NY[k] = pk(q.ny, q.ny);
    NZ[k] = pk(q.nz, q.nz);
    acc[k].x = acc[k].y = acc[k].z = 0ull;
  }
  f2 rx = 0ull, ry = 0ull, rz = 0ull;
  for (int rep = 0; rep < reps; ++rep) {
#pragma unroll 2
    for (int s = 0; s < 32; ++s) {
      ulonglong2 a, b, c, d;
      f2 e;
      load_record(my, (lane + s) & 31, a, b, c, d, e);
#pragma unroll
      for (int k = 0; k < TPL; ++k) {
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
      const int from = (lane + 1) & 31;
      rx = __shfl_sync(0xffffffffu, rx, from);
      ry = __shfl_sync(0xffffffffu, ry, from);
      rz = __shfl_sync(0xffffffffu, rz, from);
    }
  }
#pragma unroll
  for (int k = 0; k < TPL; ++k) {
    float *o = fwd + (tb + k * 32 + lane) * 3;
    o[0] = hsum(acc[k].x);
    o[1] = hsum(acc[k].y);
    o[2] = hsum(acc[k].z);
  }
  // record `lane` of this warp: sources 2 lane and 2 lane + 1
  float *o = rev + ((static_cast<size_t>(blockIdx.x) * kWarps + warp) * 64 + 2 * lane) * 3;
  float lo, hi;
  upk(rx, lo, hi);
  o[0] = lo;
  o[3] = hi;
  upk(ry, lo, hi);
  o[1] = lo;
  o[4] = hi;
  upk(rz, lo, hi);
  o[2] = lo;
  o[5] = hi;
}

// ---------------------------------------------------------------------------
// Host: a fixed-seed generator (64-bit LCG, top 53 bits) and the FP64 definition.
struct Rng {
  uint64_t s;
  double next() {
    s = s * 6364136223846793005ull + 1442695040888963407ull;
    return static_cast<double>(s >> 11) * 0x1.0p-53;
  }
  void ball(double r, double &x, double &y, double &z) {
    do {
      x = (2 * next() - 1) * r;
      y = (2 * next() - 1) * r;
      z = (2 * next() - 1) * r;
    } while (x * x + y * y + z * z > r * r);
  }
};

// Eq. 1 term of source (position p, moment w m) at target t, in the units of
// the loops: w (3 (m.d) d / r^5 - m / r^3), d = p - t.
void term(const double *p, const double *wm, const double *t, double *out) {
  const double d[3] = {p[0] - t[0], p[1] - t[1], p[2] - t[2]};
  const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  const double r = std::sqrt(r2);
  const double md = wm[0] * d[0] + wm[1] * d[1] + wm[2] * d[2];
  for (int c = 0; c < 3; ++c) out[c] += 3.0 * md * d[c] / (r2 * r2 * r) - wm[c] / (r2 * r);
}

double max_rel(const std::vector<double> &ref, const std::vector<float> &got) {
  double num = 0.0, den = 0.0;
  for (size_t i = 0; i < ref.size(); ++i) {
    num = std::fmax(num, std::fabs(ref[i] - static_cast<double>(got[i])));
    den = std::fmax(den, std::fabs(ref[i]));
  }
  return num / den;
}

template <typename L>
double time_launch(L launch, int iters) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  launch();
  cudaDeviceSynchronize();
  cudaEventRecord(e0);
  for (int i = 0; i < iters; ++i) launch();
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms * 1e-3 / iters;
}

#define CHECK(x)                                                                   \
  do {                                                                             \
    const cudaError_t e_ = (x);                                                    \
    if (e_ != cudaSuccess) {                                                       \
      std::fprintf(stderr, "%s: %s\n", #x, cudaGetErrorString(e_));                \
      return 1;                                                                    \
    }                                                                              \
  } while (0)

}  // namespace

int main() {
  int dev = 0, sms = 0, mhz = 0;
  CHECK(cudaGetDevice(&dev));
  CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CHECK(cudaDeviceGetAttribute(&mhz, cudaDevAttrClockRate, dev));
  const double peak = sms * 128.0 * 2.0 * (mhz * 1e3);  // FP32 lanes x 2 flops x clock
  const int blocks = sms * 8, reps = 64;
  const double w = 1.0 / (4.0 * 3.14159265358979323846);  // V / (4 pi L^3) for a unit cube L^3

  Rng rng{12345};
  // ordered form: one tile of records and 3 x 32 targets per block
  std::vector<SrcPair> rec(kTile);
  std::vector<double> srcp(2 * kTile * 3), srcm(2 * kTile * 3);
  for (int r = 0; r < kTile; ++r)
    for (int h = 0; h < 2; ++h) {
      double x, y, z, mx, my, mz;
      rng.ball(kBall, x, y, z);
      rng.ball(1.0, mx, my, mz);
      const double nm = std::sqrt(mx * mx + my * my + mz * mz);
      const int j = 2 * r + h;
      rec[r].x[h] = static_cast<float>(x);
      rec[r].y[h] = static_cast<float>(y);
      rec[r].z[h] = static_cast<float>(z);
      set_source_moment(rec[r], h, static_cast<float>(w), static_cast<float>(mx / nm),
                        static_cast<float>(my / nm), static_cast<float>(mz / nm));
      rec[r].pad[h] = 0.f;
      srcp[3 * j] = rec[r].x[h];
      srcp[3 * j + 1] = rec[r].y[h];
      srcp[3 * j + 2] = rec[r].z[h];
      srcm[3 * j] = -static_cast<double>(rec[r].nx[h]);  // w m as the loop holds it
      srcm[3 * j + 1] = -static_cast<double>(rec[r].ny[h]);
      srcm[3 * j + 2] = -static_cast<double>(rec[r].nz[h]);
    }
  std::vector<float4> tgt(static_cast<size_t>(blocks) * 3 * 32);
  for (auto &t : tgt) {
    double x, y, z;
    rng.ball(kBall, x, y, z);
    t = make_float4(static_cast<float>(x), static_cast<float>(y), static_cast<float>(z), 0.f);
  }
  // symmetric form: 32 sources and 32 targets per warp
  const size_t nsym = static_cast<size_t>(blocks) * kWarps * 32;
  std::vector<Np> ssrc(nsym), stgt(nsym);
  auto make_np = [&](Np &q) {
    double x, y, z, mx, my, mz;
    rng.ball(kBall, x, y, z);
    rng.ball(1.0, mx, my, mz);
    const double nm = std::sqrt(mx * mx + my * my + mz * mz);
    q.x = static_cast<float>(x);
    q.y = static_cast<float>(y);
    q.z = static_cast<float>(z);
    const float wx = static_cast<float>(w * mx / nm), wy = static_cast<float>(w * my / nm),
                wz = static_cast<float>(w * mz / nm);
    q.tx = 3.f * wx;
    q.ty = 3.f * wy;
    q.tz = 3.f * wz;
    q.nx = -wx;
    q.ny = -wy;
    q.nz = -wz;
    q.pad[0] = q.pad[1] = q.pad[2] = 0.f;
  };
  for (auto &q : ssrc) make_np(q);
  for (auto &q : stgt) make_np(q);

  // symmetric packed form: 32 records and up to 2 x 32 targets (Np) per warp
  const size_t nprec = static_cast<size_t>(blocks) * kWarps * 32;
  std::vector<SrcPair> prec(nprec);
  std::vector<Np> ptgt(nprec * 4);
  for (auto &r : prec)
    for (int h = 0; h < 2; ++h) {
      Np q;
      make_np(q);
      r.x[h] = q.x;
      r.y[h] = q.y;
      r.z[h] = q.z;
      r.nx[h] = q.nx;
      r.ny[h] = q.ny;
      r.nz[h] = q.nz;
      r.tx[h] = q.tx;
      r.ty[h] = q.ty;
      r.tz[h] = q.tz;
      r.pad[h] = 0.f;
    }
  for (auto &q : ptgt) make_np(q);
  SrcPair *d_prec = nullptr;
  Np *d_ptgt = nullptr;
  float *d_pfwd = nullptr, *d_prev = nullptr;
  CHECK(cudaMalloc(&d_prec, sizeof(SrcPair) * nprec));
  CHECK(cudaMalloc(&d_ptgt, sizeof(Np) * ptgt.size()));
  CHECK(cudaMalloc(&d_pfwd, sizeof(float) * ptgt.size() * 3));
  CHECK(cudaMalloc(&d_prev, sizeof(float) * nprec * 2 * 3));
  CHECK(cudaMemcpy(d_prec, prec.data(), sizeof(SrcPair) * nprec, cudaMemcpyHostToDevice));
  CHECK(cudaMemcpy(d_ptgt, ptgt.data(), sizeof(Np) * ptgt.size(), cudaMemcpyHostToDevice));

  SrcPair *d_rec = nullptr;
  float4 *d_tgt = nullptr;
  Np *d_ssrc = nullptr, *d_stgt = nullptr;
  float *d_out = nullptr, *d_fwd = nullptr, *d_rev = nullptr;
  CHECK(cudaMalloc(&d_rec, sizeof(SrcPair) * kTile));
  CHECK(cudaMalloc(&d_tgt, sizeof(float4) * tgt.size()));
  CHECK(cudaMalloc(&d_ssrc, sizeof(Np) * nsym));
  CHECK(cudaMalloc(&d_stgt, sizeof(Np) * nsym));
  CHECK(cudaMalloc(&d_out, sizeof(float) * blocks * 3 * kWarps * 32 * 3));
  CHECK(cudaMalloc(&d_fwd, sizeof(float) * nsym * 3));
  CHECK(cudaMalloc(&d_rev, sizeof(float) * nsym * 3));
  CHECK(cudaMemcpy(d_rec, rec.data(), sizeof(SrcPair) * kTile, cudaMemcpyHostToDevice));
  CHECK(cudaMemcpy(d_tgt, tgt.data(), sizeof(float4) * tgt.size(), cudaMemcpyHostToDevice));
  CHECK(cudaMemcpy(d_ssrc, ssrc.data(), sizeof(Np) * nsym, cudaMemcpyHostToDevice));
  CHECK(cudaMemcpy(d_stgt, stgt.data(), sizeof(Np) * nsym, cudaMemcpyHostToDevice));

  // --- checks against the definition (one repetition, block 0 / warp 0) ---
  auto check_ordered = [&](int tpl, auto kernel) -> double {
    kernel<<<1, kWarps * 32>>>(d_rec, d_tgt, 1, d_out);
    if (cudaDeviceSynchronize() != cudaSuccess) return -1.0;
    std::vector<float> raw(static_cast<size_t>(tpl) * kWarps * 32 * 3);
    cudaMemcpy(raw.data(), d_out, sizeof(float) * raw.size(), cudaMemcpyDeviceToHost);
    std::vector<double> ref(static_cast<size_t>(tpl) * 32 * 3, 0.0);
    std::vector<float> got(ref.size(), 0.f);
    for (int k = 0; k < tpl; ++k)
      for (int l = 0; l < 32; ++l) {
        const float4 t = tgt[k * 32 + l];
        const double tp[3] = {t.x, t.y, t.z};
        for (int j = 0; j < 2 * kTile; ++j) term(&srcp[3 * j], &srcm[3 * j], tp, &ref[(k * 32 + l) * 3]);
        for (int wv = 0; wv < kWarps; ++wv)
          for (int c = 0; c < 3; ++c)
            got[(k * 32 + l) * 3 + c] += raw[((k * kWarps + wv) * 32 + l) * 3 + c];
      }
    return max_rel(ref, got);
  };
  double err[4];
  err[1] = check_ordered(1, ordered_pairs<1>);
  err[2] = check_ordered(2, ordered_pairs<2>);
  err[3] = check_ordered(3, ordered_pairs<3>);
  symmetric_pairs<<<1, kWarps * 32>>>(d_ssrc, d_stgt, 1, d_fwd, d_rev);
  CHECK(cudaDeviceSynchronize());
  {
    std::vector<float> f(32 * 3), r(32 * 3);
    cudaMemcpy(f.data(), d_fwd, sizeof(float) * 96, cudaMemcpyDeviceToHost);
    cudaMemcpy(r.data(), d_rev, sizeof(float) * 96, cudaMemcpyDeviceToHost);
    std::vector<double> rf(96, 0.0), rr(96, 0.0);
    for (int i = 0; i < 32; ++i)
      for (int j = 0; j < 32; ++j) {
        const Np &s = ssrc[j], &t = stgt[i];
        const double sp[3] = {s.x, s.y, s.z}, tp[3] = {t.x, t.y, t.z};
        const double sm[3] = {-s.nx, -s.ny, -s.nz}, tm[3] = {-t.nx, -t.ny, -t.nz};
        term(sp, sm, tp, &rf[3 * i]);  // field at target i from source j
        term(tp, tm, sp, &rr[3 * j]);  // field at source j from target i
      }
    std::vector<float> both(f);
    both.insert(both.end(), r.begin(), r.end());
    std::vector<double> rboth(rf);
    rboth.insert(rboth.end(), rr.begin(), rr.end());
    err[0] = max_rel(rboth, both);
  }

  // symmetric packed, TPL = 1 and 2: block 0, warp 0 (32 records, 32 TPL targets)
  double perr[5] = {0, 0, 0, 0, 0};
  auto check_packed = [&](int tpl, auto kernel) -> double {
    kernel<<<1, kWarps * 32>>>(d_prec, d_ptgt, 1, d_pfwd, d_prev);
    if (cudaDeviceSynchronize() != cudaSuccess) return -1.0;
    std::vector<float> f(static_cast<size_t>(tpl) * 32 * 3), r(64 * 3);
    cudaMemcpy(f.data(), d_pfwd, sizeof(float) * f.size(), cudaMemcpyDeviceToHost);
    cudaMemcpy(r.data(), d_prev, sizeof(float) * r.size(), cudaMemcpyDeviceToHost);
    std::vector<double> rf(f.size(), 0.0), rr(r.size(), 0.0);
    for (int i = 0; i < 32 * tpl; ++i)
      for (int j = 0; j < 64; ++j) {
        const SrcPair &R = prec[j / 2];
        const int h = j & 1;
        const Np &t = ptgt[i];
        const double sp[3] = {R.x[h], R.y[h], R.z[h]}, tp[3] = {t.x, t.y, t.z};
        const double smv[3] = {-R.nx[h], -R.ny[h], -R.nz[h]}, tm[3] = {-t.nx, -t.ny, -t.nz};
        term(sp, smv, tp, &rf[3 * i]);  // field at target i from source j
        term(tp, tm, sp, &rr[3 * j]);   // field at source j from target i
      }
    std::vector<float> both(f);
    both.insert(both.end(), r.begin(), r.end());
    std::vector<double> rboth(rf);
    rboth.insert(rboth.end(), rr.begin(), rr.end());
    return max_rel(rboth, both);
  };
  perr[1] = check_packed(1, symmetric_packed<1>);
  perr[2] = check_packed(2, symmetric_packed<2>);
  perr[3] = check_packed(3, symmetric_packed<3>);
  perr[4] = check_packed(4, symmetric_packed<4>);

  // --- timing ---
  auto report = [&](const char *name, double pairs, double t, double e) {
    std::printf("%s %.6e %.6f %.3e\n", name, pairs / t, 30.0 * pairs / t / peak, e);
  };
  const int iters = 20;
  {
    auto L1 = [&] { ordered_pairs<1><<<blocks, kWarps * 32>>>(d_rec, d_tgt, reps, d_out); };
    report("ordered_1_target_per_lane", double(blocks) * 1 * 32 * kTile * 2 * reps,
           time_launch(L1, iters), err[1]);
    auto L2 = [&] { ordered_pairs<2><<<blocks, kWarps * 32>>>(d_rec, d_tgt, reps, d_out); };
    report("ordered_2_targets_per_lane", double(blocks) * 2 * 32 * kTile * 2 * reps,
           time_launch(L2, iters), err[2]);
    auto L3 = [&] { ordered_pairs<3><<<blocks, kWarps * 32>>>(d_rec, d_tgt, reps, d_out); };
    report("ordered_3_targets_per_lane", double(blocks) * 3 * 32 * kTile * 2 * reps,
           time_launch(L3, iters), err[3]);
    auto LS = [&] { symmetric_pairs<<<blocks, kWarps * 32>>>(d_ssrc, d_stgt, reps, d_fwd, d_rev); };
    // each lane and step: one pair in both directions, two ordered pairs
    report("symmetric_lane_rotation", double(nsym) * 32 * reps * 2, time_launch(LS, iters), err[0]);
    // each lane and step: TPL targets x 2 sources, both directions
    auto P1 = [&] { symmetric_packed<1><<<blocks, kWarps * 32>>>(d_prec, d_ptgt, reps, d_pfwd, d_prev); };
    report("symmetric_packed_1_target_per_lane", double(nprec) * 32 * reps * 4, time_launch(P1, iters),
           perr[1]);
    auto P2 = [&] { symmetric_packed<2><<<blocks, kWarps * 32>>>(d_prec, d_ptgt, reps, d_pfwd, d_prev); };
    report("symmetric_packed_2_targets_per_lane", double(nprec) * 32 * reps * 8, time_launch(P2, iters),
           perr[2]);
    auto P3 = [&] { symmetric_packed<3><<<blocks, kWarps * 32>>>(d_prec, d_ptgt, reps, d_pfwd, d_prev); };
    report("symmetric_packed_3_targets_per_lane", double(nprec) * 32 * reps * 12, time_launch(P3, iters),
           perr[3]);
    auto P4 = [&] { symmetric_packed<4><<<blocks, kWarps * 32>>>(d_prec, d_ptgt, reps, d_pfwd, d_prev); };
    report("symmetric_packed_4_targets_per_lane", double(nprec) * 32 * reps * 16, time_launch(P4, iters),
           perr[4]);
  }
  CHECK(cudaGetLastError());
  cudaFree(d_rec);
  cudaFree(d_tgt);
  cudaFree(d_ssrc);
  cudaFree(d_stgt);
  cudaFree(d_out);
  cudaFree(d_fwd);
  cudaFree(d_rev);
  cudaFree(d_prec);
  cudaFree(d_ptgt);
  cudaFree(d_pfwd);
  cudaFree(d_prev);
  return 0;
}
