// kmc_stage.cuh -- shared-memory staging by bulk asynchronous copies (the
// TMA engine's cp.async.bulk) completing on mbarriers, with waits bounded in
// time: a copy that never lands makes the wait give up and set a device error
// word instead of spinning forever. Used by the step kernels (kmc_step.cu)
// and the no-allocation field (kmc_noalloc.cu).
#pragma once
#include <stdint.h>

#include "kmc_types.h"

namespace kmc {

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

// Ends an mbarrier's use (all its phases complete), so that its memory can
// be initialised again.
__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
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

// Thread-block clusters. cluster_sync(): every thread of every CTA of the
// cluster arrives (release) and waits (acquire); the caller keeps every
// thread of both CTAs on the same sequence of these calls. ld_cluster() reads
// a float of the shared memory of CTA `rank` of the cluster at the address
// that `p` has in the caller's own shared memory.
__device__ __forceinline__ void cluster_sync() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ float ld_cluster(const float *p, uint32_t rank) {
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(smem_addr(p)), "r"(rank));
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(remote) : "memory");
  return v;
}

// Arrival of a block at the counter of its target group once its partial sums
// are stored (by any of its threads, plain or .cg stores): a block barrier, then
// one release-acquire add by thread 0, which publishes with it the stores the
// barrier ordered before it. Every thread learns whether the block arrived
// last (nsplit - 1 arrivals before it); the last block reads the others'
// partials after the second barrier, which orders those reads after the
// acquire. *flag is a shared int.
__device__ __forceinline__ bool arrive_last(int32_t *counter, int nsplit, int *flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], 1;"
                 : "=r"(old)
                 : "l"(counter)
                 : "memory");
    *flag = old == nsplit - 1;
  }
  __syncthreads();
  return *flag != 0;
}

__device__ __forceinline__ unsigned long long global_ns();

// Grid-wide barrier of a cooperative launch (every block resident), bounded in
// time. gbar[0] counts the arrivals at the current generation gbar[1]: the
// last block to arrive resets the count and advances the generation (release);
// the others wait (acquire) for the generation to change, for at most
// limit_ns, or until another block has reported a timeout in the error word.
// The block's stores before the barrier are published by thread 0's
// release-acquire arrival (after a block barrier) and read after the second
// block barrier. Returns, to every thread, false if the barrier was not
// completed. skip: the block does not arrive (failure-detection test hook).
__device__ __forceinline__ bool grid_barrier(uint32_t *gbar, uint32_t nblocks, int32_t *err,
                                             unsigned long long limit_ns, bool skip, int *flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    if (*reinterpret_cast<volatile int32_t *>(err) & kErrTimeout) {
      ok = 0;
    } else {
      uint32_t g;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(gbar + 1) : "memory");
      bool wait = true;
      if (!skip) {
        uint32_t old;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;"
                     : "=r"(old)
                     : "l"(gbar)
                     : "memory");
        if (old == nblocks - 1) {
          asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(gbar) : "memory");
          asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(gbar + 1), "r"(g + 1)
                       : "memory");
          wait = false;
        }
      }
      if (wait) {
        const unsigned long long t0 = global_ns();
        for (;;) {
          uint32_t gn;
          asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(gn) : "l"(gbar + 1) : "memory");
          if (gn != g) break;
          if (*reinterpret_cast<volatile int32_t *>(err) & kErrTimeout) {
            ok = 0;
            break;
          }
          if (global_ns() - t0 > limit_ns) {
            atomicOr(err, kErrTimeout);
            ok = 0;
            break;
          }
        }
      }
    }
    *flag = ok;
  }
  __syncthreads();
  return *flag != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Programmatic dependent launch. A step kernel launched with programmatic
// stream serialisation may start while the previous step is still running;
// grid_dependency_wait() returns once that grid has completed and its memory
// is visible (at once when there is no such dependency), so every read of
// state the previous step writes comes after it. grid_launch_dependents(),
// once every block has called it or exited, lets the next step's grid launch
// while this one drains.
__device__ __forceinline__ void grid_dependency_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ void grid_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Waits for phase `parity` of `bar` for at most limit_ns (2 s); returns false
// (and sets the error word) if the copy never completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int32_t *err,
                                                  unsigned long long limit_ns = 2000000000ull) {
  for (int i = 0; i < 64; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > limit_ns) {
      atomicOr(err, kErrTimeout);
      return false;
    }
  }
  return true;
}

// The same wait without reporting: true once phase `parity` of `bar` has
// completed, false after limit_ns.
__device__ __forceinline__ bool mbar_wait_quiet(uint64_t *bar, uint32_t parity,
                                                unsigned long long limit_ns) {
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}

// After the wait for tile t gave up (double buffering: tile t on barrier
// t & 1, tile t + 1 possibly issued on the other): one thread waits, again
// for at most limit_ns each, for the copies that may still be landing in the
// block's shared memory, so that none lands after the block has ended.
__device__ __forceinline__ void drain_copies(uint64_t *bar, int t, int ntiles,
                                             unsigned long long limit_ns) {
  mbar_wait_quiet(&bar[t & 1], (t >> 1) & 1, limit_ns);
  if (t + 1 < ntiles) mbar_wait_quiet(&bar[(t + 1) & 1], ((t + 1) >> 1) & 1, limit_ns);
}

}  // namespace kmc
