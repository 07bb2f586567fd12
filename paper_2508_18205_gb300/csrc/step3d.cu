// step3d.cu -- fused 3D full-vector half steps (Eq. 2 with the hyperviscosity
// terms of Eqs. 17-18 on every component), collocated:
//   H pass, node i:  H' = H + ch (-curl E + gamma Dv H),  E* = E + ce gamma Dv E
//   E pass, node i:  E' = E* + ce curl H', then every component tangential to
//                    a PEC wall the node sits on is held at 0.
// curl F = (Dy Fz - Dz Fy, Dz Fx - Dx Fz, Dx Fy - Dy Fx).
//
// State: F holds per node the E block {Ex, Ey, Ez, ce} at F[2 i] and the H
// block {Hx, Hy, Hz, 0} at F[2 i + 1]. Every HV entry needs both blocks of its
// neighbour, fetched by one 32-byte gather. The H pass writes E* and H' to
// their own arrays (Es, Hn); the E pass gathers H' and writes both blocks of F.
#include "kernels.cuh"
#include "step.cuh"

namespace mfd {

template <typename T> struct Curl {
    T dyz, dzy, dzx, dxz, dxy, dyx;  // Dy Fz, Dz Fy, Dz Fx, Dx Fz, Dx Fy, Dy Fx
};

// raw index entries of a chunk -> node ids (and image codes when MIR)
template <bool MIR>
__device__ __forceinline__ int4 ids3(int4 raw, int64_t n, uint4& r) {
    if constexpr (MIR) return img_split(raw, n, r);
    r = make_uint4(0u, 0u, 0u, 0u);
    return chk4(raw, n);
}

// VARN: the curl stencil size varies per centre (s.cext holds the chunks of
// each slice); the other instantiations read nc chunks for every node. A
// VARN instantiation with NC chunks is launched only when every slice reads
// at least NC - 1 of them (s.nc0), so only the last chunk is conditional.
template <typename T, int NC, int NV, bool SHARED, bool COMP, bool MIR = false, bool VARN = false>
__device__ __forceinline__ void h3_node(const StencilStreams<T>& s, const typename Vec<T>::V4* __restrict__ F,
                                        int64_t i, Curl<T>& cu, T vh[3], T ve[3]) {
    using V4 = typename Vec<T>::V4;
    using Acc = typename AccSel<T, COMP>::type;
    const int nc = NC ? NC : s.nc;
    const int nv = NV ? NV : s.nv;
    const int64_t slice = i >> 5;
    const int lane = (int)(i & 31);
    // curl chunks of this slice (warp-uniform): fewer than nc when the stencil
    // size varies per centre and no centre of the slice needs the last ones
    const int ncs = VARN ? (int)s.cext[slice] : nc;
    constexpr int G = VARN ? (NC ? NC - 1 : 0) : NC;   // curl chunks every slice reads (NC = 0: none known)
    Acc a_yz, a_zy, a_zx, a_xz, a_xy, a_yx;            // curl sums (compensated when COMP)
    AccPlain<T> hx, hy, hz, ex, ey, ez;                 // hyperviscosity sums (scaled by gamma)
    const V4* px = s.wx + slice * nc * 32 + lane;
    const V4* py = s.wy + slice * nc * 32 + lane;
    const V4* pz = s.wz + slice * nc * 32 + lane;
    const V4* pv = s.wv + slice * nv * 32 + lane;
    auto curl4 = [&](const V4& wx, const V4& wy, const V4& wz, const V4* f) {
        const T* wxa = &wx.x;
        const T* wya = &wy.x;
        const T* wza = &wz.x;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            a_yz.add(wya[q], f[q].z);
            a_zy.add(wza[q], f[q].y);
            a_zx.add(wza[q], f[q].x);
            a_xz.add(wxa[q], f[q].z);
            a_xy.add(wxa[q], f[q].y);
            a_yx.add(wya[q], f[q].x);
        }
    };
    auto hv4 = [&](const V4& wv, const V4* e, const V4* h) {
        const T* wva = &wv.x;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            hx.add(wva[q], h[q].x);
            hy.add(wva[q], h[q].y);
            hz.add(wva[q], h[q].z);
            ex.add(wva[q], e[q].x);
            ey.add(wva[q], e[q].y);
            ez.add(wva[q], e[q].z);
        }
    };
    if constexpr (SHARED) {
        const int ni = (NC && NV) ? (NC > NV ? NC : NV) : s.ni;
        const int4* ip = s.idx_c + slice * ni * 32 + lane;
#pragma unroll
        for (int c = 0; c < ni; ++c) {
            uint4 r;
            const int4 id = ids3<MIR>(ld_stream(ip + c * 32), s.src_c, r);
            V4 e[4], h[4];
            if (c < nv) {
                ld_gather_eh(F + 2 * (int64_t)id.x, e[0], h[0]);
                ld_gather_eh(F + 2 * (int64_t)id.y, e[1], h[1]);
                ld_gather_eh(F + 2 * (int64_t)id.z, e[2], h[2]);
                ld_gather_eh(F + 2 * (int64_t)id.w, e[3], h[3]);
                if constexpr (MIR) {
                    h[0] = img_h3(h[0], r.x);
                    h[1] = img_h3(h[1], r.y);
                    h[2] = img_h3(h[2], r.z);
                    h[3] = img_h3(h[3], r.w);
                }
            } else {
                e[0] = ld_gather(F + 2 * (int64_t)id.x);
                e[1] = ld_gather(F + 2 * (int64_t)id.y);
                e[2] = ld_gather(F + 2 * (int64_t)id.z);
                e[3] = ld_gather(F + 2 * (int64_t)id.w);
            }
            if constexpr (MIR) {
                e[0] = img_e3(e[0], r.x);
                e[1] = img_e3(e[1], r.y);
                e[2] = img_e3(e[2], r.z);
                e[3] = img_e3(e[3], r.w);
            }
            if constexpr (VARN) {
                if (c < nc && (c < G || c < ncs)) curl4(ld_stream(px + c * 32), ld_stream(py + c * 32), ld_stream(pz + c * 32), e);
            } else {
                if (c < nc) curl4(ld_stream(px + c * 32), ld_stream(py + c * 32), ld_stream(pz + c * 32), e);
            }
            if (c < nv) hv4(ld_stream(pv + c * 32), e, h);
        }
    } else {
        const int4* ic = s.idx_c + slice * nc * 32 + lane;
        const int4* iv = s.idx_v + slice * nv * 32 + lane;
#pragma unroll
        for (int c = 0; c < nc; ++c) {
            if (VARN && c >= G && c >= ncs) break;
            uint4 r;
            const int4 id = ids3<MIR>(ld_stream(ic + c * 32), s.src_c, r);
            V4 e[4];
            e[0] = ld_gather(F + 2 * (int64_t)id.x);
            e[1] = ld_gather(F + 2 * (int64_t)id.y);
            e[2] = ld_gather(F + 2 * (int64_t)id.z);
            e[3] = ld_gather(F + 2 * (int64_t)id.w);
            if constexpr (MIR) {
                e[0] = img_e3(e[0], r.x);
                e[1] = img_e3(e[1], r.y);
                e[2] = img_e3(e[2], r.z);
                e[3] = img_e3(e[3], r.w);
            }
            curl4(ld_stream(px + c * 32), ld_stream(py + c * 32), ld_stream(pz + c * 32), e);
        }
#pragma unroll
        for (int c = 0; c < nv; ++c) {
            uint4 r;
            const int4 id = ids3<MIR>(ld_stream(iv + c * 32), s.src_v, r);
            V4 e[4], h[4];
            ld_gather_eh(F + 2 * (int64_t)id.x, e[0], h[0]);
            ld_gather_eh(F + 2 * (int64_t)id.y, e[1], h[1]);
            ld_gather_eh(F + 2 * (int64_t)id.z, e[2], h[2]);
            ld_gather_eh(F + 2 * (int64_t)id.w, e[3], h[3]);
            if constexpr (MIR) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const unsigned rq = q == 0 ? r.x : q == 1 ? r.y : q == 2 ? r.z : r.w;
                    e[q] = img_e3(e[q], rq);
                    h[q] = img_h3(h[q], rq);
                }
            }
            hv4(ld_stream(pv + c * 32), e, h);
        }
    }
    cu.dyz = a_yz.get();
    cu.dzy = a_zy.get();
    cu.dzx = a_zx.get();
    cu.dxz = a_xz.get();
    cu.dxy = a_xy.get();
    cu.dyx = a_yx.get();
    vh[0] = hx.get();
    vh[1] = hy.get();
    vh[2] = hz.get();
    ve[0] = ex.get();
    ve[1] = ey.get();
    ve[2] = ez.get();
}

// The H pass may take up to 128 registers: at 256 threads per block the
// compensated FP32 kernel runs 2 blocks per SM with 32 bytes of spills; caps
// of 80 (3 blocks) and 64 registers (4 blocks) spilled more and were slower.
template <typename T, int NC, int NV, bool SHARED, bool COMP, bool MIR = false, bool VARN = false>
__global__ void __launch_bounds__(512, 1) k_h3(StencilStreams<T> s, Coefs<T> k, const typename Vec<T>::V4* __restrict__ F,
                                            typename Vec<T>::V4* __restrict__ Es,
                                            typename Vec<T>::V4* __restrict__ Hn) {
    using V4 = typename Vec<T>::V4;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    Curl<T> cu;
    T vh[3], ve[3];
    h3_node<T, NC, NV, SHARED, COMP, MIR, VARN>(s, F, i, cu, vh, ve);
    V4 e, h;
    ld_gather_eh(F + 2 * i, e, h);
    V4 ho, eo;
    ho.x = h.x + k.ch * (-(cu.dyz - cu.dzy) + k.gamma * vh[0]);
    ho.y = h.y + k.ch * (-(cu.dzx - cu.dxz) + k.gamma * vh[1]);
    ho.z = h.z + k.ch * (-(cu.dxy - cu.dyx) + k.gamma * vh[2]);
    ho.w = T(0);
    eo.x = e.x + e.w * (k.gamma * ve[0]);
    eo.y = e.y + e.w * (k.gamma * ve[1]);
    eo.z = e.z + e.w * (k.gamma * ve[2]);
    eo.w = e.w;
    st4(Hn + i, ho);
    st4(Es + i, eo);
}

template <typename T, int NC, bool SHARED, bool COMP, bool MIR = false, bool VARN = false>
__global__ void __launch_bounds__(512, 2) k_e3(StencilStreams<T> s, const typename Vec<T>::V4* __restrict__ Hn,
                                            const typename Vec<T>::V4* __restrict__ Es,
                                            const uint8_t* __restrict__ wall, typename Vec<T>::V4* __restrict__ F) {
    using V4 = typename Vec<T>::V4;
    using Acc = typename AccSel<T, COMP>::type;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    const int nc = NC ? NC : s.nc;
    const int ni = SHARED ? s.ni : nc;
    const int64_t slice = i >> 5;
    const int lane = (int)(i & 31);
    const int4* ip = s.idx_c + slice * ni * 32 + lane;
    const V4* px = s.wx + slice * nc * 32 + lane;
    const V4* py = s.wy + slice * nc * 32 + lane;
    const V4* pz = s.wz + slice * nc * 32 + lane;
    const int ncs = VARN ? (int)s.cext[slice] : nc;  // curl chunks of this slice (see h3_node)
    constexpr int G = VARN ? (NC ? NC - 1 : 0) : NC;
    Acc a_yz, a_zy, a_zx, a_xz, a_xy, a_yx;
#pragma unroll
    for (int c = 0; c < nc; ++c) {
        if (VARN && c >= G && c >= ncs) break;
        uint4 r;
        const int4 id = ids3<MIR>(ld_stream(ip + c * 32), s.src_c, r);
        const V4 wx = ld_stream(px + c * 32), wy = ld_stream(py + c * 32), wz = ld_stream(pz + c * 32);
        V4 f[4];
        f[0] = ld_gather(Hn + id.x);
        f[1] = ld_gather(Hn + id.y);
        f[2] = ld_gather(Hn + id.z);
        f[3] = ld_gather(Hn + id.w);
        if constexpr (MIR) {
            f[0] = img_h3(f[0], r.x);
            f[1] = img_h3(f[1], r.y);
            f[2] = img_h3(f[2], r.z);
            f[3] = img_h3(f[3], r.w);
        }
        const T* wxa = &wx.x;
        const T* wya = &wy.x;
        const T* wza = &wz.x;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            a_yz.add(wya[q], f[q].z);
            a_zy.add(wza[q], f[q].y);
            a_zx.add(wza[q], f[q].x);
            a_xz.add(wxa[q], f[q].z);
            a_xy.add(wxa[q], f[q].y);
            a_yx.add(wya[q], f[q].x);
        }
    }
    const V4 e = ld_gather(Es + i);
    const V4 hown = ld_gather(Hn + i);
    V4 o;
    o.x = e.x + e.w * (a_yz.get() - a_zy.get());
    o.y = e.y + e.w * (a_zx.get() - a_xz.get());
    o.z = e.z + e.w * (a_xy.get() - a_yx.get());
    o.w = e.w;
    const unsigned m = wall ? wall[i] : 0u;
    if (m) {
        // component b is tangential to the wall normal to axis a != b
        if (m & 6u) o.x = T(0);
        if (m & 5u) o.y = T(0);
        if (m & 3u) o.z = T(0);
    }
    st_eh(F + 2 * i, o, hown);
}

template <typename T, bool COMP, bool MIR = false, bool VARN = false>
__global__ void __launch_bounds__(256) k_energy3(StencilStreams<T> s, Coefs<T> k, const typename Vec<T>::V4* __restrict__ F,
                                                 const double* __restrict__ eps_r, double eta2,
                                                 double* __restrict__ partial) {
    using V4 = typename Vec<T>::V4;
    __shared__ double red[256];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double u = 0.0;
    if (i < s.n) {
        Curl<T> cu;
        T vh[3], ve[3];
        if (s.idx_v == s.idx_c)
            h3_node<T, 0, 0, true, COMP, MIR, VARN>(s, F, i, cu, vh, ve);
        else
            h3_node<T, 0, 0, false, COMP, MIR, VARN>(s, F, i, cu, vh, ve);
        const V4 e = F[2 * i], h = F[2 * i + 1];
        const double h1[3] = {(double)(h.x + k.ch * (-(cu.dyz - cu.dzy) + k.gamma * vh[0])),
                              (double)(h.y + k.ch * (-(cu.dzx - cu.dxz) + k.gamma * vh[1])),
                              (double)(h.z + k.ch * (-(cu.dxy - cu.dyx) + k.gamma * vh[2]))};
        const double h0[3] = {(double)h.x, (double)h.y, (double)h.z};
        const double ev[3] = {(double)e.x, (double)e.y, (double)e.z};
        for (int a = 0; a < 3; ++a) {
            double av = 0.5 * (h0[a] + h1[a]);
            u += eps_r[i] * ev[a] * ev[a] + eta2 * av * av;
        }
    }
    red[threadIdx.x] = u;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// node sets with mirror walls (MIR): the same kernels with image codes;
// per-centre curl sizes (VARN): each slice reads its own number of curl chunks
template <typename T, bool COMP, bool MIR, bool VARN>
static void launch3_k(const Launch3D& L, const StencilStreams<T>& s, const Coefs<T>& k, int pass, unsigned grid,
                      int block, cudaStream_t st) {
    using V4 = typename Vec<T>::V4;
    const bool shared = s.idx_v == s.idx_c;
    V4* F = static_cast<V4*>(L.F);
    V4* Es = static_cast<V4*>(L.Es);
    V4* Hn = static_cast<V4*>(L.Hn);
    // the specialised chunk counts: n = 40 (and 41..44 next to mirror walls), N_h = 71
    constexpr int NCS = VARN ? 11 : 10;
    const bool spec = s.nc == NCS && (!VARN || s.nc0 >= NCS - 1);
    if (pass == 0) {
        if (shared && spec && s.nv == 18) k_h3<T, NCS, 18, true, COMP, MIR, VARN><<<grid, block, 0, st>>>(s, k, F, Es, Hn);
        else if (shared) k_h3<T, 0, 0, true, COMP, MIR, VARN><<<grid, block, 0, st>>>(s, k, F, Es, Hn);
        else k_h3<T, 0, 0, false, COMP, MIR, VARN><<<grid, block, 0, st>>>(s, k, F, Es, Hn);
    } else {
        if (shared && spec) k_e3<T, NCS, true, COMP, MIR, VARN><<<grid, block, 0, st>>>(s, Hn, Es, L.wall, F);
        else if (shared) k_e3<T, 0, true, COMP, MIR, VARN><<<grid, block, 0, st>>>(s, Hn, Es, L.wall, F);
        else k_e3<T, 0, false, COMP, MIR, VARN><<<grid, block, 0, st>>>(s, Hn, Es, L.wall, F);
    }
}

template <typename T, bool COMP>
static cudaError_t launch3(const Launch3D& L, const StencilStreams<T>& s, const Coefs<T>& k, int pass, cudaStream_t st) {
    const int block = L.block[pass];
    const unsigned grid = (unsigned)((s.n + block - 1) / block);
    if (s.cext) {
        if (s.mirror) launch3_k<T, COMP, true, true>(L, s, k, pass, grid, block, st);
        else launch3_k<T, COMP, false, true>(L, s, k, pass, grid, block, st);
    } else {
        if (s.mirror) launch3_k<T, COMP, true, false>(L, s, k, pass, grid, block, st);
        else launch3_k<T, COMP, false, false>(L, s, k, pass, grid, block, st);
    }
    return cudaGetLastError();
}

cudaError_t launch_3d(const Launch3D& L, int pass, cudaStream_t st) {
    if (L.fp64) return launch3<double, false>(L, L.s.d, L.kd, pass, st);
    if (L.comp) return launch3<float, true>(L, L.s.f, L.kf, pass, st);
    return launch3<float, false>(L, L.s.f, L.kf, pass, st);
}

template <typename T, bool COMP>
static void energy3_k(const StencilStreams<T>& s, const Coefs<T>& k, const void* F, const double* eps_r, double eta2,
                      double* partial, unsigned grid, cudaStream_t st) {
    using V4 = typename Vec<T>::V4;
    const V4* f = static_cast<const V4*>(F);
    if (s.cext) {
        if (s.mirror) k_energy3<T, COMP, true, true><<<grid, 256, 0, st>>>(s, k, f, eps_r, eta2, partial);
        else k_energy3<T, COMP, false, true><<<grid, 256, 0, st>>>(s, k, f, eps_r, eta2, partial);
    } else {
        if (s.mirror) k_energy3<T, COMP, true><<<grid, 256, 0, st>>>(s, k, f, eps_r, eta2, partial);
        else k_energy3<T, COMP><<<grid, 256, 0, st>>>(s, k, f, eps_r, eta2, partial);
    }
}

cudaError_t launch_energy_3d(const Launch3D& L, const double* eps_r, double eta2, double* partial, unsigned grid,
                             cudaStream_t st) {
    if (L.fp64) energy3_k<double, false>(L.s.d, L.kd, L.F, eps_r, eta2, partial, grid, st);
    else if (L.comp) energy3_k<float, true>(L.s.f, L.kf, L.F, eps_r, eta2, partial, grid, st);
    else energy3_k<float, false>(L.s.f, L.kf, L.F, eps_r, eta2, partial, grid, st);
    return cudaGetLastError();
}

unsigned long long bounds_take_step3d(cudaStream_t s) { return bounds_take_local(s); }

}  // namespace mfd
