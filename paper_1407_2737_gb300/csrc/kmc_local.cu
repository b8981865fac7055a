// kmc_local.cu -- local volume concentration phi_N (Eq. 8, Sec. III.5) on the
// device: for every NP i of one lysosome, r_N = distance to its N-th nearest
// neighbour and phi_N,i = 3 N V_i / (4 pi r_N^3).
//
// One thread per target NP, all pairs in FP64 (N^2 work, like the dipolar sum
// but run once per geometry). Source positions are staged through shared
// memory tile by tile; each thread keeps the N smallest squared distances seen
// so far in ascending order and inserts a new one only when it is below the
// current N-th (the N-th order statistic does not depend on how ties between
// equal distances are broken). Squared distances are formed as
// (dx^2 + dy^2) + dz^2 without contraction, the order the oracle uses.
#include <cuda_runtime.h>
#include <math.h>

#include "kmc_local.h"

namespace kmc {

namespace {

// one warp per block: many small blocks spread the targets evenly over the SMs
// (50 000 NPs: 46.9 ms against 50.9 ms with 128-thread blocks)
constexpr int kPhiThreads = 32;
constexpr int kPhiTile = 512;

__global__ void __launch_bounds__(kPhiThreads)
    local_concentration_kernel(const dbl4 *__restrict__ pos, int n, int N,
                               double *__restrict__ phi) {
  __shared__ double sx[kPhiTile], sy[kPhiTile], sz[kPhiTile];
  const int i = blockIdx.x * kPhiThreads + threadIdx.x;
  const bool active = i < n;
  const dbl4 p = pos[active ? i : 0];
  double best[kPhiMaxN];
  for (int q = 0; q < N; ++q) best[q] = INFINITY;
  double thr = INFINITY;  // best[N - 1]
  for (int t0 = 0; t0 < n; t0 += kPhiTile) {
    const int cnt = min(kPhiTile, n - t0);
    __syncthreads();
    for (int j = threadIdx.x; j < cnt; j += kPhiThreads) {
      const dbl4 s = pos[t0 + j];
      sx[j] = s.x;
      sy[j] = s.y;
      sz[j] = s.z;
    }
    __syncthreads();
    if (!active) continue;
    for (int j = 0; j < cnt; ++j) {
      const double dx = __dsub_rn(sx[j], p.x);
      const double dy = __dsub_rn(sy[j], p.y);
      const double dz = __dsub_rn(sz[j], p.z);
      const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
      if (d2 < thr && t0 + j != i) {
        int k = N - 1;
        while (k > 0 && best[k - 1] > d2) {
          best[k] = best[k - 1];
          --k;
        }
        best[k] = d2;
        thr = best[N - 1];
      }
    }
  }
  if (active) {
    const double r = sqrt(thr);
    phi[i] = (3.0 * static_cast<double>(N) * p.w) / (r * r * r);
  }
}

}  // namespace

cudaError_t launch_local_concentration(const dbl4 *pos, int n, int N, double *phi,
                                       cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (n + kPhiThreads - 1) / kPhiThreads;
  local_concentration_kernel<<<blocks, kPhiThreads, 0, st>>>(pos, n, N, phi);
  return cudaGetLastError();
}

}  // namespace kmc
