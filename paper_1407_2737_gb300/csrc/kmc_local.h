// kmc_local.h -- host entry of the local-concentration kernel (kmc_local.cu),
// called by the C ABI layer (kmc_api.cu).
#pragma once
#include <cuda_runtime.h>

#include "kmc_types.h"

namespace kmc {

// Largest neighbour rank N of Eq. 8 (the paper uses N = 20).
constexpr int kPhiMaxN = 64;

// phi[i] = 3 N w_i / r_N^3 for the n NPs of pos (one lysosome; x, y, z in units
// of the length L, w = V_i / (4 pi L^3)), with r_N the distance to the N-th
// nearest other NP: Eq. 8 with V_i = 4 pi L^3 w_i. Requires 1 <= N <= n - 1,
// N <= kPhiMaxN. rmax bounds the distance of every position from the origin
// (it sets the margin of the FP32 pre-screen); posf is [n] scratch.
cudaError_t launch_local_concentration(const dbl4 *pos, int n, int N, double rmax,
                                       float4 *posf, double *phi, cudaStream_t st);

}  // namespace kmc
