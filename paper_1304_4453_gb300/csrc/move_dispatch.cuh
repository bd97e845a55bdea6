// Cooperative launches of the persistent phase kernels (move_plm.cu,
// move_plp.cu), instantiated per weight kind and gain width.
#pragma once
#include "phase.cuh"

namespace cd {

// Runs a whole PLM move phase; a.result receives {sweeps, converged, ...}.
void launch_move_phase(int wk, bool big, const PhaseArgs &a, cudaStream_t s);
// Runs a whole PLP; a.result receives {iterations, converged}.
void launch_plp_run(int wk, bool big, const PhaseArgs &a, cudaStream_t s);

// Grid of a persistent kernel: every block resident at once (required by
// the grid barrier), at most BARRIER_FAN * BARRIER_SUBS blocks.
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

inline void launch_persistent(const void *kernel, const PhaseArgs &a, cudaStream_t s) {
    const int grid = persistent_grid(kernel);
    void *args[] = {const_cast<PhaseArgs *>(&a)};
    CD_CUDA(cudaLaunchCooperativeKernel(kernel, dim3(grid), dim3(kBlock), args, PHASE_SMEM, s));
    note_launch();
}

}  // namespace cd
