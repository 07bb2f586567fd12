// step.cuh -- launch descriptors shared by the simulation object and the step kernels.
#pragma once

#include "kernels.cuh"

namespace mfd {

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
    int lanes[2] = {1, 1};      // collocated, per pass (H, E): lanes per node (1, 2 or 4)
    void* A = nullptr;  // collocated state {Ez, Hx, Hy, ce}^n
    void* B = nullptr;  // collocated intermediate {E*, Hx', Hy', ce}
    Stag2DPtrs stag;
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
};

cudaError_t launch_3d(const Launch3D& L, int pass, cudaStream_t st);
cudaError_t launch_energy_3d(const Launch3D& L, const double* eps_r, double eta2, double* partial, unsigned grid,
                             cudaStream_t st);

// stencil indices the bounds-checked build found out of range in each file's
// kernels since the last call (0 in the default build)
unsigned long long bounds_take_step2d(cudaStream_t s);
unsigned long long bounds_take_step3d(cudaStream_t s);
unsigned long long bounds_take_adjoint(cudaStream_t s);

}  // namespace mfd
