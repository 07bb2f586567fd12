// adjoint.cuh -- transposed stencil operators and the reverse-time (adjoint)
// half steps of the collocated TMz leapfrog, for gradients of probe objectives.
#pragma once

#include "internal.cuh"
#include "kernels.cuh"

namespace mfd {

// Transpose of the collocated stencil operators, row j listing every (i, w_ij)
// with j in S(x_i): CSR with rows padded to a multiple of 4 entries (padding:
// column j, weight 0) and sorted by column (and operator kind) so that the
// transposed sums are reproducible. Weights per entry: {w^dx, w^dy, w^hv, 0}.
//
// The kernels read the transpose in the sliced layout of the forward streams:
// rows in slices of 32 (one warp), each slice padded to its longest row (in
// chunks of 4 entries); chunk c of row 32 s + l at (off[s] + c) * 32 + l, one
// int4 of columns and one 4-vector per operator (dx, dy, hv weights), so a
// warp's loads of a chunk are contiguous. Padding: column = the row, weight 0.
struct AdjT {
    DevBuf rowptr;  // int64 [n + 1]
    DevBuf col;     // int32 [nnz]
    DevBuf w;       // Vec<T>::V4 [nnz]
    int64_t nnz = 0;
    int64_t n = 0;
    // sliced form
    DevBuf off;     // int64 [slices + 1], in chunks
    DevBuf scol;    // int4 [off[slices] * 32]
    DevBuf sx, sy, sv;  // Vec<T>::V4 [off[slices] * 32]
    int64_t chunks = 0;
};

mfd_status adj_build(mfd_ctx* ctx, const mfd_weights* curl, const mfd_weights* hv, bool fp64, AdjT& out);

struct AdjArgs {
    bool fp64 = false;
    const int64_t* off = nullptr;
    const int4* scol = nullptr;
    const void* sx = nullptr;
    const void* sy = nullptr;
    const void* sv = nullptr;
    int64_t n = 0;
    void* LA = nullptr;  // {lambda_E, lambda_Hx, lambda_Hy, ce} (ce = dt / (eps0 eps_r), 0 at PEC)
    void* LB = nullptr;  // {t, lambda~_Hx, lambda~_Hy, ce}
    double ch = 0, gamma = 0;
    // Ez of the step's two levels: ez + (*slot0 + k) * n (Ez^n) and the level after it
    // (Ez^{n+1}); slot0 lives on the device so that a captured segment replays anywhere
    const void* ez = nullptr;
    const int64_t* slot0 = nullptr;
    int k = 0;
    const double* eps = nullptr;
    double* g_eps = nullptr;
    // the per-step source and probe terms, done by the threads of their nodes
    // inside the passes (see AdjTerms)
    const struct AdjTerms* terms = nullptr;
    float l2_keep = 0.0f;  // fraction of the transposed streams' lines kept in L2 (stream_policy)
};

// Source and probe terms of a backward step, fused into the passes: the thread
// of node j finds its sources (pass 0) or probes (pass 1) through a bit per node
// and a node-sorted list. Pass 0 adds, before the step's own permittivity term,
// g_amp[k] += mu r_k(t_{n+1}) and g_eps[j] += mu amp_k r_k(t_{n+1}) / eps_r for
// every source k at j (mu = lambda_E^{n+1} at j, n = *seg0 + k_step); pass 1 adds
// 2 dt Ez^n(j) to lambda_E^n once per probe at j when n >= min_step.
struct AdjTerms {
    const uint32_t* smask = nullptr;  // bit j: node j holds a source
    const int64_t* snode = nullptr;   // source nodes, ascending (ties in source order)
    const int* sidx = nullptr;        // the source index of each entry of snode
    int nsrc = 0;
    const double* amp = nullptr;
    const double* f0 = nullptr;
    const double* t0 = nullptr;
    double* g_amp = nullptr;
    const uint32_t* pmask = nullptr;  // bit j: node j holds a probe
    const int64_t* pnode = nullptr;   // probe nodes, ascending
    int nprobe = 0;
    const int64_t* seg0 = nullptr;    // first step of the segment (device)
    double dt = 0;
    int64_t min_step = 0;
};

// pass 0: LA -> LB (and the permittivity gradient of this step); pass 1: LB -> LA
cudaError_t adj_pass(const AdjArgs& a, int pass, cudaStream_t s);

// the probe term dJ/dE^n of J = dt sum_n sum_p (Ez_p^n)^2: LA[p].x += 2 dt Ez[p] at every probe
// (the backward steps add it inside pass 1, AdjTerms; this kernel serves the last level),
// Ez = ez + (*slot0 + k) * n (ez itself when slot0 is NULL). With seg0 (device) the term
// belongs to step n = *seg0 + k and is skipped when n < min_step (the state before the first
// recorded step is not an objective term). One thread per probe (atomic adds: two probes on
// one node add in either order).
cudaError_t adj_probe_term(bool fp64, void* LA, const void* ez, const int64_t* probe, int nprobe, double dt,
                           cudaStream_t s, const int64_t* seg0 = nullptr, int k = 0, int64_t min_step = 0,
                           const int64_t* slot0 = nullptr, int64_t n = 0);

// LA = {0, 0, 0, ce} from the state A = {Ez, Hx, Hy, ce}
cudaError_t init_lambda(bool fp64, void* LA, const void* A, int64_t n, cudaStream_t s);

// J += dt sum of squares of `count` probe values (FP64 accumulator)
cudaError_t probe_energy(bool fp64, const void* buf, int64_t count, double dt, double* J, cudaStream_t s);

// dst[i] = Ez of the V4 state (stride 4)
cudaError_t copy_ez(bool fp64, const void* state, void* dst, int64_t n, cudaStream_t s);
// the same into level (*counter - start) of an Ez history (after a step, the counter holds
// the level just reached), so that captured forward steps fill the history anywhere
cudaError_t copy_ez_level(bool fp64, const void* state, void* hist, int64_t n, const int64_t* counter,
                          int64_t start, cudaStream_t s);

}  // namespace mfd
