// Graph construction helpers (graph.cu).
#pragma once
#include "common.cuh"

namespace cd {
// Validates an input CSR (host or device pointers; CD_BORROW: device arrays
// read in place) and builds the owned,
// loop-free device graph with self-loop weights, volumes and omega(E).
// Throws Error{CD_EINVAL} on malformed input.
void build_graph(int64_t n, const int64_t *rp, const int32_t *col, const int32_t *w, int mem,
                 cudaStream_t s, OwnedGraph &out);
// Fills vol, W and max degree of a graph whose rp/col/w/self are set.
void finish_graph(OwnedGraph &g, cudaStream_t s, bool borrowed = false);
// Input-form export; returns the entry count (arrays may be null to query).
int64_t export_graph(const GraphView &g, int64_t *rp, int32_t *col, int64_t *w, int mem, cudaStream_t s);
}  // namespace cd
