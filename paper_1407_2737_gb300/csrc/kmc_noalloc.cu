// kmc_noalloc.cu -- kmc_dipolar_field_noalloc: the dipolar-field part of the
// FP32-mixed step kernel (split source ranges, compensated sums, the pair term
// of kmc_pair.cuh) for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not available or not
// allowed -- inside another framework's memory pool, in a process whose device
// memory is fully reserved up front, or in host code that only receives
// device pointers from its caller. It takes every input and output as a device
// pointer the caller owns and keeps its own working memory (source records,
// per-item partial sums, per-group arrival counters, an error word) in one
// file-scope static device array, so that no call allocates or frees anything.
//
// The array is fixed at kNoallocBytes (about 2 MB, for up to
// KMC_NOALLOC_MAX_N NPs); every GPU that loads the library holds it until the
// process exits. All calls share it: calls that overlap on the GPU (different
// streams, or host threads) race on it and must be serialised by the caller.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "kmc.h"
#include "kmc_pair.cuh"
#include "kmc_stage.cuh"
#include "kmc_types.h"

namespace kmc {
void set_last_error(const char *msg);  // kmc_api.cu: the message kmc_last_error() returns
}

namespace {

using kmc::AccF32;
using kmc::f2;
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
constexpr size_t kErrBytes = 16;                                // the error word, padded
constexpr size_t kNoallocBytes = kRecBytes + kTgtBytes + kPartBytes + kCntBytes + kErrBytes;

// The working memory of every call (see the file comment).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Device address of g_noalloc_scratch in each device's current context. Host
// code cannot use the symbol itself as a device address; the address is
// looked up with that device current and looked up again if the device's
// context has changed (a reset context reloads the module elsewhere).
struct AddrCache {
  unsigned long long ctx_id = 0;
  void *addr = nullptr;
};
std::mutex g_mu;
AddrCache g_addr[64];

constexpr double kPi = 3.14159265358979323846;
constexpr double kMu0 = 4.0e-7 * kPi;

thread_local char g_msg[256];

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
__device__ __forceinline__ int32_t *sc_err(unsigned char *base) {
  return reinterpret_cast<int32_t *>(base + kRecBytes + kTgtBytes + kPartBytes + kCntBytes);
}

// Positions (units of `length` about `center`) and source moments w m into the
// pair records, targets into float4; the arrival counters and the error word
// start at zero.
__global__ void noalloc_pack(unsigned char *scratch, int n, const double *__restrict__ pos,
                             const double *__restrict__ m, const double *__restrict__ vol,
                             double cx, double cy, double cz, double inv_len, double w_scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kGroups) sc_cnt(scratch)[i] = 0;
  if (i == 0) *sc_err(scratch) = 0;
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

// The records of one staged tile taken by this warp (every kWarps-th).
template <bool MASK>
__device__ __forceinline__ AccF32 tile_pairs(const ulonglong2 *__restrict__ sp, int cnt, int first,
                                             f2 X, f2 Y, f2 Z) {
  AccF32 acc;
  acc.x = acc.y = acc.z = 0ull;
#pragma unroll 2
  for (int r = first; r < cnt; r += kWarps) {
    ulonglong2 a, b, c, d;
    f2 e;
    kmc::load_record(sp, r, a, b, c, d, e);
    kmc::pair_record<MASK>(a, b, c, d, e, X, Y, Z, acc);
  }
  return acc;
}

// One block = 32 targets x one source range; the last block of a target group
// adds the partial sums in split order and writes mu0 H_dip = bunit * b_dip.
// A staging wait that runs out (after wait_ns) sets the error word; the
// block's sums become NaN, so that the group's targets get NaN in B, and the
// block still arrives, so that the group completes. stall_tx > 0 (a test of
// that path) makes every tile expect that many bytes more than its copy
// delivers, so that every wait runs out while no copy is left unfinished.
__global__ void __launch_bounds__(kWarps * 32)
    noalloc_field(unsigned char *scratch, int n, int nsplit, double bunit,
                  double *__restrict__ B, uint32_t stall_tx, unsigned long long wait_ns) {
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
  const f2 X = kmc::pk(p.x, p.x), Y = kmc::pk(p.y, p.y), Z = kmc::pk(p.z, p.z);
  float s3[3] = {0.f, 0.f, 0.f}, c3[3] = {0.f, 0.f, 0.f};
  const SrcPair *src = sc_rec(scratch);
  int32_t *err = sc_err(scratch);
  const int ntiles = (j1 - j0 + kTile - 1) / kTile;
  if (threadIdx.x == 0) {
    kmc::mbar_init(&bar[0], 1);
    kmc::mbar_init(&bar[1], 1);
    kmc::mbar_init_fence();
  }
  __syncthreads();
  auto issue = [&](int t) {
    const int r0 = j0 + t * kTile;
    const uint32_t bytes = static_cast<uint32_t>(min(kTile, j1 - r0)) * sizeof(SrcPair);
    kmc::mbar_expect_tx(&bar[t & 1], bytes + stall_tx);
    kmc::bulk_g2s(&buf[t & 1][0], src + r0, bytes, &bar[t & 1]);
  };
  if (threadIdx.x == 0) {
    issue(0);
    if (ntiles > 1) issue(1);
  }
  bool failed = false;
  for (int t = 0; t < ntiles; ++t) {
    const bool ok = kmc::mbar_wait_bounded(&bar[t & 1], (t >> 1) & 1, err, wait_ns);
    if (ok) {
      const int r0 = j0 + t * kTile, cnt = min(kTile, j1 - r0);
      const AccF32 acc = (r0 <= own1 && own0 < r0 + cnt)
                             ? tile_pairs<true>(buf[t & 1], cnt, warp, X, Y, Z)
                             : tile_pairs<false>(buf[t & 1], cnt, warp, X, Y, Z);
      kmc::kahan_add(s3[0], c3[0], kmc::hsum(acc.x));
      kmc::kahan_add(s3[1], c3[1], kmc::hsum(acc.y));
      kmc::kahan_add(s3[2], c3[2], kmc::hsum(acc.z));
    }
    if (!__syncthreads_and(ok)) {
      if (threadIdx.x == 0) kmc::drain_copies(bar, t, ntiles, wait_ns);
      failed = true;
      break;
    }
    if (threadIdx.x == 0 && t + 2 < ntiles) {
      kmc::proxy_fence_shared();
      issue(t + 2);
    }
  }
  if (failed) {
#pragma unroll
    for (int c = 0; c < 3; ++c) s3[c] = __int_as_float(0x7fc00000);  // NaN
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
        kmc::neumaier_add(s, e, wp[w][c][lane]);
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
          kmc::neumaier_add(s, e, __ldcg(base + (q * 6 + c) * 32 + lane));
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

// The call's status for the caller: KMC_OK, or KMC_ETIMEOUT if a wait ran out.
__global__ void noalloc_status(const unsigned char *scratch, int32_t *status) {
  const int32_t e = *reinterpret_cast<const int32_t *>(scratch + kRecBytes + kTgtBytes +
                                                       kPartBytes + kCntBytes);
  *status = (e & kmc::kErrTimeout) ? KMC_ETIMEOUT : KMC_OK;
}

kmc_status fail(kmc_status s, const char *msg, cudaError_t e = cudaSuccess) {
  if (e != cudaSuccess)
    snprintf(g_msg, sizeof(g_msg), "%s: %s", msg, cudaGetErrorString(e));
  else
    snprintf(g_msg, sizeof(g_msg), "%s", msg);
  kmc::set_last_error(g_msg);
  return s;
}

// A caller buffer must be device (or managed) memory of the current device,
// aligned for its element type.
kmc_status check_device_buffer(const void *p, size_t align, int dev, const char *name) {
  if (reinterpret_cast<uintptr_t>(p) % align != 0) {
    snprintf(g_msg, sizeof(g_msg), "%s is not aligned to %zu bytes", name, align);
    kmc::set_last_error(g_msg);
    return KMC_EINVAL;
  }
  cudaPointerAttributes at;
  const cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    snprintf(g_msg, sizeof(g_msg), "%s: cudaPointerGetAttributes failed: %s", name,
             cudaGetErrorString(e));
    kmc::set_last_error(g_msg);
    return KMC_EINVAL;
  }
  if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev) {
    snprintf(g_msg, sizeof(g_msg),
             "%s is not device memory of the current device %d (memory type %d, device %d)",
             name, dev, static_cast<int>(at.type), at.device);
    kmc::set_last_error(g_msg);
    return KMC_EINVAL;
  }
  return KMC_OK;
}

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Identifier of the current CUDA context (0 if it cannot be read).
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_cur = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked = false;
  if (!looked) {
    looked = true;
    cudaDriverEntryPointQueryResult q1, q2;
    void *f1 = nullptr, *f2p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) ==
            cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess)
      get_cur = reinterpret_cast<CtxGetCurrentFn>(f1);
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2p, 12000, cudaEnableDefault, &q2) ==
            cudaSuccess &&
        q2 == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f2p);
    cudaGetLastError();
  }
  if (!get_cur || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_cur(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

}  // namespace

extern "C" {

kmc_status kmc_dipolar_field_noalloc(int32_t n, const double *pos, const double *m,
                                     const double *vol, double Ms, const double *center,
                                     double length, double *B, int32_t *status,
                                     void *cuda_stream) {
  g_msg[0] = '\0';
  kmc::set_last_error(g_msg);
  if (n < 1 || n > kMaxN)
    return fail(KMC_ECAPACITY, "n must be in [1, KMC_NOALLOC_MAX_N = 8192]");
  if (!pos || !m || !vol || !B || !center)
    return fail(KMC_EINVAL, "NULL pointer argument");
  if (!(Ms > 0) || !std::isfinite(Ms) || !(length > 0) || !std::isfinite(length))
    return fail(KMC_EINVAL, "Ms and length must be finite and > 0");
  for (int q = 0; q < 3; ++q)
    if (!std::isfinite(center[q])) return fail(KMC_EINVAL, "center must be finite");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(KMC_ECUDA, "cudaGetDevice failed", e);
  if (dev < 0 || dev >= 64) return fail(KMC_ECUDA, "device ordinal out of range");
  // every caller buffer is checked on the host before anything is launched
  const struct {
    const void *p;
    size_t align;
    const char *name;
  } bufs[] = {{pos, 8, "pos"}, {m, 8, "m"}, {vol, 8, "vol"}, {B, 8, "B"}, {status, 4, "status"}};
  for (const auto &b : bufs) {
    if (!b.p) continue;  // only status may be NULL here
    const kmc_status s = check_device_buffer(b.p, b.align, dev, b.name);
    if (s != KMC_OK) return s;
  }
  void *addr = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    const unsigned long long ctx = current_context_id();
    if (!g_addr[dev].addr || ctx == 0 || ctx != g_addr[dev].ctx_id) {
      void *a = nullptr;
      e = cudaGetSymbolAddress(&a, g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_addr[dev] = AddrCache();
        return fail(KMC_ECUDA, "cudaGetSymbolAddress of the scratch array failed", e);
      }
      g_addr[dev].addr = a;
      g_addr[dev].ctx_id = ctx;
    }
    addr = g_addr[dev].addr;
  }
  // test of the timeout path: every staging wait runs out after 1 ms
  const char *fault = std::getenv("KMC_FAULT");
  const bool stall = fault && std::strcmp(fault, "noalloc_stall") == 0;
  const uint32_t stall_tx = stall ? 16u : 0u;
  const unsigned long long wait_ns = stall ? 1000000ull : 2000000000ull;
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
  noalloc_field<<<groups * nsplit, kWarps * 32, 0, st>>>(scratch, n, nsplit, kMu0 * Ms, B,
                                                         stall_tx, wait_ns);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(KMC_ECUDA, "field kernel launch failed", e);
  if (status) {
    noalloc_status<<<1, 1, 0, st>>>(scratch, status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(KMC_ECUDA, "status kernel launch failed", e);
  }
  return KMC_OK;
}

}  // extern "C"
