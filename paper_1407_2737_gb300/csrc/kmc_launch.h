// kmc_launch.h -- host entry points of the step kernels (kmc_step.cu),
// called by the C ABI layer (kmc_api.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "kmc_types.h"

namespace kmc {

// Dynamic shared memory of one block of the fused step kernel (tpl: targets
// per lane, 2 for the FP32 two-target kernel).
size_t step_smem_bytes(int prec_fp32, int warps, int tile, int tpl = 1, int rpl = 1);

// One time step of every work item (lysosome, 32 targets) on stream st.
// warps in {4, 8, 16}; tile = sources per staged tile. With pdl the launch
// may overlap the tail of the previous kernel on st (programmatic dependent
// launch); the kernel waits for that kernel before it reads any state.
// tpl = 2 or 3 (FP32 only): items are 64- or 96-target groups, two or three
// targets per lane. rpl = 2 or 4 (FP32 only, tpl = 1, warps = rpl or 4 rpl):
// each item is 32 targets of rpl replica lysosomes it.l .. it.l + rpl - 1 that
// share their geometry (kmc_step_f32_rep, one or four warps per replica).
// cl = 2 (FP32, one target per lane): every target group has exactly two
// source parts, items 2 g and 2 g + 1, which run as a two-CTA cluster and
// exchange their sums through distributed shared memory; n_items even.
cudaError_t launch_step(int prec_fp32, int warps, int tile, const StepArgs &a, int n_items,
                        cudaStream_t st, bool pdl = false, int tpl = 1, int rpl = 1,
                        int cl = 0);

// Persistent period (FP32, one target per lane, warps 4 or 8): one cooperative
// launch of n_items blocks runs steps 0 .. a.S - 1 with a grid barrier after
// each (a.cosk, a.gbar zeroed before the launch, a.barrier_ns); every block
// must be resident at once (persist_blocks_per_sm x SMs >= n_items).
cudaError_t launch_persist(const StepArgs &a, int warps, int tile, int n_items, cudaStream_t st);
cudaError_t persist_blocks_per_sm(int warps, int tile, int *blocks);

// Symmetric pair form (FP32): one step = kmc_field_sym<warps, cells> over
// a.sitems[0 .. n_field) and then kmc_update_sym over a.supd[0 .. a.n_upd).
// (warps, cells) in {(2, 2), (4, 1), (4, 2), (8, 1)}; row groups of warps x cells
// cells (4 or 8).
// upd: 0 = kmc_update_sym (one warp per update item), 1 = kmc_update_sym_block
// (one block per item).
cudaError_t launch_sym(const StepArgs &a, int warps, int cells, int n_field, cudaStream_t st,
                       bool pdl = false, int upd = 0);
size_t sym_smem_bytes(int warps, int cells);
cudaError_t sym_blocks_per_sm(int warps, int cells, int *blocks);

// Blocks of the step kernel of this shape that fit on one SM at once.
cudaError_t step_blocks_per_sm(int prec_fp32, int warps, int tile, int tpl, int *blocks,
                               int rpl = 1);

// The Ref. [8] mode over all items of a (one warp per item).
cudaError_t launch_mean(const MeanArgs &a, cudaStream_t st);

// Redraws the axes and/or positions of one lysosome (a.off .. a.off + a.n).
cudaError_t launch_regen(const RegenArgs &a, cudaStream_t st);

// One batch of the random sequential addition (RsaArgs): candidates, their
// checks against the kept spheres, then the in-order pass that keeps them.
cudaError_t launch_rsa_batch(const RsaArgs &a, cudaStream_t st);

// Advances the device run state by one field period of S steps.
cudaError_t launch_advance(RunState *rs, int S, cudaStream_t st);

// Once per process and device: writes the scan grid of step iv and sets the
// kernels' shared-memory limit.
cudaError_t init_device();

// Largest dynamic shared memory of one step block.
constexpr size_t kMaxStepSmem = 200 * 1024;

}  // namespace kmc
