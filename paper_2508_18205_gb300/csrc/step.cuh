// step.cuh -- launch descriptors shared by the simulation object and the step kernels.
#pragma once

#include "kernels.cuh"

namespace mfd {

// The per-step terms after the E update, done inside the E pass by the thread of
// each node: soft Ricker sources added to Ez (none at held nodes), then the
// probes of the node record Ez; the step counter n (the step n -> n + 1 being
// taken) is read by every block at its start and advanced by the last block to
// finish (a ticket counter), so a step is two launches.
struct PostArgs {
    const uint32_t* smask = nullptr;  // bit i: node i holds a source (null: none)
    const int64_t* snode = nullptr;   // source nodes, ascending (ties in source order)
    const int* sidx = nullptr;        // the source index of each entry of snode
    int nsrc = 0;
    const double* amp = nullptr;
    const double* f0 = nullptr;
    const double* t0 = nullptr;
    const uint8_t* held = nullptr;    // per node: bits of held components (PEC), or null
    unsigned held_bits = 0;           // bits that hold Ez
    const uint32_t* pmask = nullptr;  // bit i: node i holds a probe (null: none)
    const int64_t* pnode = nullptr;   // probe nodes, ascending
    const int* pidx = nullptr;        // the probe index (record column) of each entry of pnode
    int nprobe = 0;
    void* pbuf = nullptr;             // records [rec][nprobe] of the state's real type
    int64_t pcap = 0;
    const int64_t* pstep0 = nullptr;  // step of record 0
    int64_t* counter = nullptr;       // steps taken
    unsigned* done = nullptr;         // blocks of this launch that have finished (0 between launches)
    double dt = 0;
};

__device__ __forceinline__ bool post_bit(const uint32_t* mask, int64_t i) {
    return mask && ((mask[i >> 5] >> (i & 31)) & 1u);
}
__device__ __forceinline__ int post_first(const int64_t* v, int m, int64_t key) {
    int lo = 0, hi = m;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (v[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// the step counter as the launch starts (every thread of the block calls it)
__device__ __forceinline__ int64_t post_step(const PostArgs& pa) {
    __shared__ int64_t n_s;
    if (threadIdx.x == 0) n_s = *pa.counter;
    __syncthreads();
    return n_s;
}

// Ez of node i after its sources (t_{n+1}), recorded at its probes
template <typename T> __device__ __forceinline__ T post_node(const PostArgs& pa, int64_t i, T ez, int64_t n) {
    if (post_bit(pa.smask, i) && !(pa.held && (pa.held[i] & pa.held_bits))) {
        const double t1 = (double)(n + 1) * pa.dt;
        const double pi = 3.14159265358979323846;
        for (int q = post_first(pa.snode, pa.nsrc, i); q < pa.nsrc && pa.snode[q] == i; ++q) {
            const int k = pa.sidx[q];
            double a = pi * pa.f0[k] * (t1 - pa.t0[k]);
            a = a * a;
            ez += (T)(pa.amp[k] * ((1.0 - 2.0 * a) * exp(-a)));
        }
    }
    if (post_bit(pa.pmask, i)) {
        const int64_t rec = n - *pa.pstep0;
        if (rec >= 0 && rec < pa.pcap)
            for (int q = post_first(pa.pnode, pa.nprobe, i); q < pa.nprobe && pa.pnode[q] == i; ++q)
                static_cast<T*>(pa.pbuf)[rec * pa.nprobe + pa.pidx[q]] = ez;
    }
    return ez;
}

// the last block of the launch to finish advances the step counter (every thread of
// the block calls it, after its stores)
__device__ __forceinline__ void post_finish(const PostArgs& pa, int64_t n) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(pa.done, 1u) == gridDim.x - 1) {
            *pa.counter = n + 1;
            *pa.done = 0u;
            __threadfence();
        }
    }
}

template <typename T> struct Both {
    StencilStreams<float> f;
    StencilStreams<double> d;
};

struct Stag2DPtrs {
    const void* ez = nullptr;  // Ez^n (E set)
    void* ezn = nullptr;       // Ez^{n+1}
    const void* h = nullptr;   // {Hx, Hy}^{n-1/2} (H set)
    void* hn = nullptr;        // {Hx, Hy}^{n+1/2}
    const void* ce = nullptr;  // dt / (eps0 eps_r), 0 at PEC
};

// one TMz half-step launch (collocated or staggered)
struct Launch2D {
    bool staggered = false, fp64 = false, comp = false;
    Both<void> hs, es;  // stencil streams of the H pass and the E pass
    Coefs<float> kf;
    Coefs<double> kd;
    int block[2] = {256, 256};  // threads per block of the H pass and the E pass
    void* A = nullptr;  // collocated state {Ez, Hx, Hy, ce}^n
    void* B = nullptr;  // collocated intermediate {E*, Hx', Hy', ce}
    Stag2DPtrs stag;
    PostArgs post;  // sources, probes and the step counter, done by the E pass
};

cudaError_t launch_2d(const Launch2D& L, int pass, cudaStream_t st);
cudaError_t launch_energy_2d(const Launch2D& L, const double* eps_r, int64_t ne, double eta2, double* partial,
                             unsigned grid, cudaStream_t st);

// one 3D half-step launch (collocated)
struct Launch3D {
    bool fp64 = false, comp = false;
    Both<void> s;
    Coefs<float> kf;
    Coefs<double> kd;
    void* F = nullptr;         // per node {Ex, Ey, Ez, ce}^n then {Hx, Hy, Hz, 0}^{n-1/2}
    void* Es = nullptr;        // {E*, ce}
    void* Hn = nullptr;        // {Hx, Hy, Hz, 0}^{n+1/2}
    const uint8_t* wall = nullptr;  // bit a: node on a wall normal to axis a
    int block[2] = {256, 256};      // threads per block of the H pass and the E pass
    PostArgs post;                  // sources, probes and the step counter, done by the E pass
};

cudaError_t launch_3d(const Launch3D& L, int pass, cudaStream_t st);
cudaError_t launch_energy_3d(const Launch3D& L, const double* eps_r, double eta2, double* partial, unsigned grid,
                             cudaStream_t st);

}  // namespace mfd
