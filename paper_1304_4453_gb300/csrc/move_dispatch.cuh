// Cooperative launches of the persistent batch kernels (move_plm.cu,
// move_plp.cu), instantiated per weight kind and gain width.
#pragma once
#include "phase.cuh"

namespace cd {

// Batch kernel of a PLM move phase / a PLP run for a weight kind and gain width.
const void *move_batch_kernel(int wk, bool big);
const void *plp_batch_kernel(int wk, bool big);

// Largest grid of a persistent kernel: every block resident at once
// (required by the team barriers), at most BARRIER_FAN * BARRIER_SUBS blocks.
inline int persistent_grid(const void *kernel) {
    int dev = 0, sms = 0, per_sm = 0;
    CD_CUDA(cudaGetDevice(&dev));
    CD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, PHASE_SMEM));
    if (per_sm < 1) raise(CD_ECUDA, "persistent kernel does not fit on an SM");
    int g = sms * per_sm;
    if (g > BARRIER_FAN * BARRIER_SUBS) g = BARRIER_FAN * BARRIER_SUBS;
    return g;
}

// grid must not exceed persistent_grid(kernel).
inline void launch_batch(const void *kernel, const BatchArgs &b, int grid, cudaStream_t s) {
    void *args[] = {const_cast<BatchArgs *>(&b)};
    CD_CUDA(cudaLaunchCooperativeKernel(kernel, dim3(grid), dim3(kBlock), args, PHASE_SMEM, s));
    note_launch();
}

}  // namespace cd
