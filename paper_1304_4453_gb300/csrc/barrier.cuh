// Team barrier of the persistent kernels (phase.cuh, color.cu): a team is
// `size` consecutive blocks that synchronise through their own GridBarrier.
// Every block of a team must be resident at once (cooperative launch).
//
// The barrier is a generation counter over a two-level arrival tree; a block
// that waits longer than BARRIER_TIMEOUT_NS sets the error flag and every
// block of the team sees the failure, so the kernel can leave cleanly and
// the host can report CD_ETIMEOUT.
#pragma once
#include "common.cuh"

namespace cd {

constexpr unsigned long long BARRIER_TIMEOUT_NS = 20ull * 1000 * 1000 * 1000;

// Two-level arrival tree: block b arrives at sub-counter b / 32; the last
// arrival of a sub-counter arrives at the root; the last root arrival opens
// the next generation.  Every counter is reset by its last arrival before
// the generation changes, so the next barrier starts from zero.
constexpr int BARRIER_FAN = 32;
constexpr int BARRIER_SUBS = 64;           // up to 2048 blocks
struct GridBarrier {
    unsigned int gen;
    int err;
    unsigned int root;
    unsigned int pad;
    unsigned int sub[BARRIER_SUBS];
};

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// A team: `size` consecutive blocks of the grid that work on one graph and
// synchronise through their own barrier.  The colouring kernel, and a batched
// launch that holds a single graph, use the whole grid as one team.
struct Team {
    int32_t rank, size;
    GridBarrier *bar;
};

// Returns false when the barrier failed (timeout here or in another block).
__device__ __forceinline__ bool team_sync(const Team &t, unsigned *s_gen, int *s_ok) {
    GridBarrier *b = t.bar;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned g = *s_gen;
        int ok = 1;
        __threadfence();
        const unsigned sb = (unsigned)t.rank / BARRIER_FAN;
        const unsigned nsub = ((unsigned)t.size + BARRIER_FAN - 1) / BARRIER_FAN;
        const unsigned sub_size = min((unsigned)BARRIER_FAN, (unsigned)t.size - sb * BARRIER_FAN);
        bool opener = false;
        if (atomicAdd(&b->sub[sb], 1u) == sub_size - 1) {
            atomicExch(&b->sub[sb], 0u);
            __threadfence();
            if (atomicAdd(&b->root, 1u) == nsub - 1) {
                atomicExch(&b->root, 0u);
                __threadfence();
                atomicExch(&b->gen, g + 1);
                opener = true;
            }
        }
        if (!opener) {
            const uint64_t t0 = global_ns();
            while (*(volatile unsigned *)&b->gen == g) {
                if (*(volatile int *)&b->err != 0) { ok = 0; break; }
                if (global_ns() - t0 > BARRIER_TIMEOUT_NS) { atomicExch(&b->err, 1); ok = 0; break; }
                __nanosleep(32);
            }
        }
        __threadfence();
        *s_gen = g + 1;
        *s_ok = ok && *(volatile int *)&b->err == 0;
    }
    __syncthreads();
    return *s_ok != 0;
}

}  // namespace cd
