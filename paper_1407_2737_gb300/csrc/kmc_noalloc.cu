// kmc_noalloc.cu -- kmc_dipolar_field_noalloc: the dipolar-field part of the
// FP32-mixed step kernel (Eq. 1 with split source ranges and compensated sums)
// for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not available or not
// allowed -- inside another framework's memory pool, in a process whose device
// memory is fully reserved up front, or from host code that only receives
// device pointers from its caller. It takes every input and output as a device
// pointer the caller owns and keeps its own working memory (source records,
// per-item partial sums, per-group arrival counters) in one file-scope static
// device array, so that no call allocates or frees anything.
//
// The array is fixed at kNoallocBytes (2.0 MB, for up to KMC_NOALLOC_MAX_N NPs);
// every GPU that loads the library holds it until the process exits. All calls
// share it: calls that overlap on the GPU (different streams, or host threads)
// race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "kmc.h"
#include "kmc_types.h"

namespace kmc {
void set_last_error(const char *msg);  // kmc_api.cu: the message kmc_last_error() returns
}

namespace {

using kmc::SrcPair;

constexpr int kMaxN = KMC_NOALLOC_MAX_N;
constexpr int kMaxRec = kMaxN / 2;
constexpr int kGroups = kMaxN / 32;
constexpr int kChunkRec = 512;                                  // source records per item
constexpr int kMaxSplit = (kMaxRec + kChunkRec - 1) / kChunkRec;
constexpr int kMaxItems = kGroups * kMaxSplit;
constexpr int kTile = 128;                                      // records per staged tile
constexpr int kWarps = 4;
constexpr size_t kRecBytes = sizeof(SrcPair) * kMaxRec;
constexpr size_t kTgtBytes = sizeof(float4) * kMaxN;
constexpr size_t kPartBytes = sizeof(float) * 6 * 32 * kMaxItems;  // (sum, error) x 3
constexpr size_t kCntBytes = sizeof(int) * kGroups;
constexpr size_t kNoallocBytes = kRecBytes + kTgtBytes + kPartBytes + kCntBytes;

// The working memory of every call (see the file comment).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Device address of g_noalloc_scratch, looked up once per device with that
// device current (a host-side use of the symbol itself is not its address).
std::mutex g_mu;
void *g_addr[64] = {};

constexpr double kPi = 3.14159265358979323846;
constexpr double kMu0 = 4.0e-7 * kPi;

thread_local char g_msg[256];

// ---------------------------------------------------------------------------
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
__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}
__device__ __forceinline__ void neumaier_add(float &s, float &c, float x) {
  const float t = s + x;
  if (fabsf(s) >= fabsf(x))
    c += (s - t) + x;
  else
    c += (x - t) + s;
  s = t;
}

// Regions of the scratch array (base = its device address).
__device__ __forceinline__ SrcPair *sc_rec(unsigned char *base) {
  return reinterpret_cast<SrcPair *>(base);
}
__device__ __forceinline__ float4 *sc_tgt(unsigned char *base) {
  return reinterpret_cast<float4 *>(base + kRecBytes);
}
__device__ __forceinline__ float *sc_part(unsigned char *base) {
  return reinterpret_cast<float *>(base + kRecBytes + kTgtBytes);
}
__device__ __forceinline__ int *sc_cnt(unsigned char *base) {
  return reinterpret_cast<int *>(base + kRecBytes + kTgtBytes + kPartBytes);
}

// Positions (units of `length` about `center`) and source moments w m into the
// pair records, targets into float4; the arrival counters start at zero.
__global__ void noalloc_pack(unsigned char *scratch, int n, const double *__restrict__ pos, const double *__restrict__ m,
                             const double *__restrict__ vol, double cx, double cy, double cz,
                             double inv_len, double w_scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kGroups) sc_cnt(scratch)[i] = 0;
  if (i >= n + (n & 1)) return;
  SrcPair &r = sc_rec(scratch)[i >> 1];
  const int h = i & 1;
  r.pad[h] = 0.0f;
  if (i == n) {  // padding NP of an odd count: far away, no moment
    r.x[h] = r.y[h] = r.z[h] = kmc::kPadCoord;
    kmc::set_source_moment(r, h, 0.0f, 0.0f, 0.0f, 0.0f);
    return;
  }
  const float x = static_cast<float>((pos[3 * i] - cx) * inv_len);
  const float y = static_cast<float>((pos[3 * i + 1] - cy) * inv_len);
  const float z = static_cast<float>((pos[3 * i + 2] - cz) * inv_len);
  const float w = static_cast<float>(vol[i] * w_scale);
  r.x[h] = x;
  r.y[h] = y;
  r.z[h] = z;
  kmc::set_source_moment(r, h, w, static_cast<float>(m[3 * i]), static_cast<float>(m[3 * i + 1]),
                         static_cast<float>(m[3 * i + 2]));
  sc_tgt(scratch)[i] = make_float4(x, y, z, w);
}

// The pair terms of Eq. 1 in the form of kmc::SrcPair: per component,
// q^3 (u d + n) with u = (t.d) q^2.
template <bool MASK>
__device__ __forceinline__ void pairs(const ulonglong2 *__restrict__ sp, int cnt, int first,
                                      f2 X, f2 Y, f2 Z, f2 (&acc)[3]) {
#pragma unroll 2
  for (int r = first; r < cnt; r += kWarps) {
    const ulonglong2 *p = sp + kmc::kRecU2 * r;
    const ulonglong2 a = p[0], b = p[1], c = p[2], d = p[3];
    const f2 e = reinterpret_cast<const f2 *>(p + 4)[0];
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
    acc[0] = fma2(q3, fma2(u, dx, b.y), acc[0]);
    acc[1] = fma2(q3, fma2(u, dy, c.x), acc[1]);
    acc[2] = fma2(q3, fma2(u, dz, c.y), acc[2]);
  }
}

// One block = 32 targets x one source range; the last block of a target group
// adds the partial sums in split order and writes mu0 H_dip = bunit * b_dip.
__global__ void __launch_bounds__(kWarps * 32)
    noalloc_field(unsigned char *scratch, int n, int nsplit, double bunit,
                  double *__restrict__ B) {
  __shared__ __align__(128) ulonglong2 buf[2][kTile * kmc::kRecU2];
  __shared__ float wp[kWarps][6][32];
  __shared__ uint64_t bar[2];
  __shared__ int s_last;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = blockIdx.x / nsplit, split = blockIdx.x % nsplit;
  const int t0 = 32 * g, nt = min(32, n - t0);
  const int nrec = (n + 1) / 2;
  const int j0 = static_cast<int>(static_cast<long long>(split) * nrec / nsplit);
  const int j1 = static_cast<int>(static_cast<long long>(split + 1) * nrec / nsplit);
  const int own0 = t0 >> 1, own1 = (t0 + nt - 1) >> 1;
  const float4 p = sc_tgt(scratch)[t0 + min(lane, nt - 1)];
  const f2 X = pk(p.x, p.x), Y = pk(p.y, p.y), Z = pk(p.z, p.z);
  float s3[3] = {0.f, 0.f, 0.f}, c3[3] = {0.f, 0.f, 0.f};
  const SrcPair *src = sc_rec(scratch);
  const int ntiles = (j1 - j0 + kTile - 1) / kTile;
  const uint32_t b0 = static_cast<uint32_t>(__cvta_generic_to_shared(&bar[0]));
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b0 + 8) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int t) {
    const int r0 = j0 + t * kTile;
    const uint32_t bytes = static_cast<uint32_t>(min(kTile, j1 - r0)) * sizeof(SrcPair);
    const uint32_t bb = b0 + 8 * (t & 1);
    const uint32_t dst = static_cast<uint32_t>(__cvta_generic_to_shared(&buf[t & 1][0]));
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bb), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
        "[%3];" ::"r"(dst),
        "l"(src + r0), "r"(bytes), "r"(bb)
        : "memory");
  };
  if (threadIdx.x == 0) {
    issue(0);
    if (ntiles > 1) issue(1);
  }
  for (int t = 0; t < ntiles; ++t) {
    const uint32_t bb = b0 + 8 * (t & 1);
    const uint32_t parity = (t >> 1) & 1;
    // bounded wait (about 2 s); a copy that never lands ends the block
    bool ok = false;
    unsigned long long t_start = 0;
    for (int spin = 0;; ++spin) {
      uint32_t done;
      asm volatile(
          "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
          "selp.b32 %0, 1, 0, p;\n\t}"
          : "=r"(done)
          : "r"(bb), "r"(parity)
          : "memory");
      if (done) {
        ok = true;
        break;
      }
      unsigned long long now;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
      if (spin == 0) t_start = now;
      if (now - t_start > 2000000000ull) break;
    }
    if (ok) {
      const int r0 = j0 + t * kTile, cnt = min(kTile, j1 - r0);
      f2 acc[3] = {0ull, 0ull, 0ull};
      if (r0 <= own1 && own0 < r0 + cnt)
        pairs<true>(buf[t & 1], cnt, warp, X, Y, Z, acc);
      else
        pairs<false>(buf[t & 1], cnt, warp, X, Y, Z, acc);
#pragma unroll
      for (int c = 0; c < 3; ++c) kahan_add(s3[c], c3[c], hsum(acc[c]));
    }
    if (!__syncthreads_and(ok)) return;  // B is left unwritten
    if (threadIdx.x == 0 && t + 2 < ntiles) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(t + 2);
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    wp[warp][c][lane] = s3[c];
    wp[warp][3 + c][lane] = -c3[c];
  }
  __syncthreads();
  float hi[3], lo[3];
  if (warp == 0) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float s = 0.f, e = 0.f;
      for (int w = 0; w < kWarps; ++w) {
        neumaier_add(s, e, wp[w][c][lane]);
        e += wp[w][3 + c][lane];
      }
      hi[c] = s;
      lo[c] = e;
    }
    if (nsplit > 1) {
      float *part = sc_part(scratch) + static_cast<size_t>(blockIdx.x) * 6 * 32;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        __stcg(part + c * 32 + lane, hi[c]);
        __stcg(part + (3 + c) * 32 + lane, lo[c]);
      }
      __threadfence();
    }
  }
  if (nsplit > 1) {
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&sc_cnt(scratch)[g], 1) == nsplit - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (warp == 0) {
      const float *base = sc_part(scratch) + static_cast<size_t>(blockIdx.x - split) * 6 * 32;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float s = 0.f, e = 0.f;
        for (int q = 0; q < nsplit; ++q) {
          neumaier_add(s, e, __ldcg(base + (q * 6 + c) * 32 + lane));
          e += __ldcg(base + (q * 6 + 3 + c) * 32 + lane);
        }
        hi[c] = s;
        lo[c] = e;
      }
      if (lane == 0) sc_cnt(scratch)[g] = 0;
    }
  }
  if (warp == 0 && lane < nt) {
#pragma unroll
    for (int c = 0; c < 3; ++c) B[3 * (t0 + lane) + c] = bunit * static_cast<double>(hi[c] + lo[c]);
  }
}

kmc_status fail(kmc_status s, const char *msg, cudaError_t e = cudaSuccess) {
  if (e != cudaSuccess)
    snprintf(g_msg, sizeof(g_msg), "%s: %s", msg, cudaGetErrorString(e));
  else
    snprintf(g_msg, sizeof(g_msg), "%s", msg);
  kmc::set_last_error(g_msg);
  return s;
}

}  // namespace

extern "C" {

kmc_status kmc_dipolar_field_noalloc(int32_t n, const double *pos, const double *m,
                                     const double *vol, double Ms, const double *center,
                                     double length, double *B, void *cuda_stream) {
  g_msg[0] = '\0';
  kmc::set_last_error(g_msg);
  if (n < 1 || n > kMaxN)
    return fail(KMC_ECAPACITY, "n must be in [1, KMC_NOALLOC_MAX_N = 8192]");
  if (!pos || !m || !vol || !B || !center)
    return fail(KMC_EINVAL, "NULL pointer argument");
  if (!(Ms > 0) || !std::isfinite(Ms) || !(length > 0) || !std::isfinite(length))
    return fail(KMC_EINVAL, "Ms and length must be finite and > 0");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(KMC_ECUDA, "cudaGetDevice failed", e);
  if (dev < 0 || dev >= 64) return fail(KMC_ECUDA, "device ordinal out of range");
  void *addr = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      e = cudaGetSymbolAddress(&g_addr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_addr[dev] = nullptr;
        return fail(KMC_ECUDA, "cudaGetSymbolAddress of the scratch array failed", e);
      }
    }
    addr = g_addr[dev];
  }
  unsigned char *scratch = static_cast<unsigned char *>(addr);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int nrec = (n + 1) / 2;
  const int nsplit = (nrec + kChunkRec - 1) / kChunkRec;
  const int groups = (n + 31) / 32;
  const double inv_len = 1.0 / length;
  const double w_scale = 1.0 / (4.0 * kPi * length * length * length);
  const int packed = n + (n & 1);
  const int threads = packed > kGroups ? packed : kGroups;
  noalloc_pack<<<(threads + 255) / 256, 256, 0, st>>>(scratch, n, pos, m, vol, center[0],
                                                      center[1], center[2], inv_len, w_scale);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(KMC_ECUDA, "packing kernel launch failed", e);
  noalloc_field<<<groups * nsplit, kWarps * 32, 0, st>>>(scratch, n, nsplit, kMu0 * Ms, B);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(KMC_ECUDA, "field kernel launch failed", e);
  return KMC_OK;
}

}  // extern "C"
