// step2d.cu -- fused TMz half steps of the stabilised meshless leapfrog (Eq. 19).
//
// Collocated (the paper's method, Sec. 5): one node set, one index stream
// serving the curl stencil (its first n entries) and the HV stencil.
//   H pass, node i:  Hx' = Hx - ch (Dy Ez - gamma Dv Hx)
//                    Hy' = Hy + ch (Dx Ez + gamma Dv Hy)
//                    E*  = Ez + ce gamma Dv Ez           (the E-row HV term uses E^n)
//   E pass, node i:  Ez' = E* + ce (Dx Hy' - Dy Hx')
// Staggered (E and H on two node sets; curl stencils are cross-set, HV own-set):
//   H pass at H nodes: curl of Ez over E neighbours, HV over H neighbours.
//   E pass at E nodes: Ez' = Ez + ce (Dx Hy' - Dy Hx' + gamma Dv Ez), curl over
//   H neighbours, HV over E neighbours.
#include "kernels.cuh"
#include "step.cuh"

namespace mfd {

// ------------------------------------------------------------ collocated

// the TMz blocks of a chunk's four entries; MIR: entries carry image codes and
// the values enter with their parities (kernels.cuh)
template <bool MIR, typename V4>
__device__ __forceinline__ void gather4_tmz(const V4* __restrict__ A, int4 raw, int64_t n, V4& f0, V4& f1, V4& f2,
                                            V4& f3) {
    if constexpr (MIR) {
        uint4 r;
        const int4 id = img_split(raw, n, r);
        f0 = img_tmz(ld_gather(A + id.x), r.x);
        f1 = img_tmz(ld_gather(A + id.y), r.y);
        f2 = img_tmz(ld_gather(A + id.z), r.z);
        f3 = img_tmz(ld_gather(A + id.w), r.w);
    } else {
        const int4 id = chk4(raw, n);
        f0 = ld_gather(A + id.x);
        f1 = ld_gather(A + id.y);
        f2 = ld_gather(A + id.z);
        f3 = ld_gather(A + id.w);
    }
}

// P lanes per node (P = 1, or 4 for problems too small to fill the GPU with one
// thread per node): lane `part` of the node sums chunks part, part + P, ... of the
// row (SHARED layout); the partial sums are merged across the node's lanes by the
// caller (merge_xor), which every lane of the warp must reach.
template <typename T, int NC, int NV, bool SHARED, bool COMP, int P = 1, bool MIR = false>
__device__ __forceinline__ void h_colloc_node(const StencilStreams<T>& s, const typename Vec<T>::V4* __restrict__ A,
                                              int64_t i, T& dxE, T& dyE, T& vx, T& vy, T& ve, bool act = true,
                                              int part = 0) {
    using V4 = typename Vec<T>::V4;
    using Acc = typename AccSel<T, COMP>::type;  // curl sums (compensated when COMP)
    using AccV = AccPlain<T>;                    // hyperviscosity sums (scaled by gamma)
    const int nc = NC ? NC : s.nc;
    const int nv = NV ? NV : s.nv;
    const int64_t slice = i >> 5;
    const int lane = (int)(i & 31);
    const uint64_t pol = stream_policy(s.l2_keep);
    Acc ax, ay;
    AccV hx, hy, he;
    if constexpr (SHARED) {
        const int ni = (NC && NV) ? (NC > NV ? NC : NV) : s.ni;
        const int4* ip = s.idx_c + slice * ni * 32 + lane;
        const V4* px = s.wx + slice * nc * 32 + lane;
        const V4* py = s.wy + slice * nc * 32 + lane;
        const V4* pv = s.wv + slice * nv * 32 + lane;
#pragma unroll
        for (int c = part; c < (act ? ni : 0); c += P) {
            const int4 raw = ld_stream(ip + c * 32, pol);
            V4 wx, wy, wv;
            if (c < nc) {
                wx = ld_stream(px + c * 32, pol);
                wy = ld_stream(py + c * 32, pol);
            }
            if (c < nv) wv = ld_stream(pv + c * 32, pol);
            V4 f0, f1, f2, f3;
            gather4_tmz<MIR>(A, raw, s.src_c, f0, f1, f2, f3);
            if (c < nc) {
                ax.add(wx.x, f0.x); ax.add(wx.y, f1.x); ax.add(wx.z, f2.x); ax.add(wx.w, f3.x);
                ay.add(wy.x, f0.x); ay.add(wy.y, f1.x); ay.add(wy.z, f2.x); ay.add(wy.w, f3.x);
            }
            if (c < nv) {
                hx.add(wv.x, f0.y); hx.add(wv.y, f1.y); hx.add(wv.z, f2.y); hx.add(wv.w, f3.y);
                hy.add(wv.x, f0.z); hy.add(wv.y, f1.z); hy.add(wv.z, f2.z); hy.add(wv.w, f3.z);
                he.add(wv.x, f0.x); he.add(wv.y, f1.x); he.add(wv.z, f2.x); he.add(wv.w, f3.x);
            }
        }
    } else {
        const int4* ic = s.idx_c + slice * nc * 32 + lane;
        const int4* iv = s.idx_v + slice * nv * 32 + lane;
        const V4* px = s.wx + slice * nc * 32 + lane;
        const V4* py = s.wy + slice * nc * 32 + lane;
        const V4* pv = s.wv + slice * nv * 32 + lane;
#pragma unroll
        for (int c = part; c < (act ? nc : 0); c += P) {
            const int4 raw = ld_stream(ic + c * 32, pol);
            const V4 wx = ld_stream(px + c * 32, pol), wy = ld_stream(py + c * 32, pol);
            V4 g0, g1, g2, g3;
            gather4_tmz<MIR>(A, raw, s.src_c, g0, g1, g2, g3);
            const T f0 = g0.x, f1 = g1.x, f2 = g2.x, f3 = g3.x;
            ax.add(wx.x, f0); ax.add(wx.y, f1); ax.add(wx.z, f2); ax.add(wx.w, f3);
            ay.add(wy.x, f0); ay.add(wy.y, f1); ay.add(wy.z, f2); ay.add(wy.w, f3);
        }
#pragma unroll
        for (int c = part; c < (act ? nv : 0); c += P) {
            const int4 raw = ld_stream(iv + c * 32, pol);
            const V4 wv = ld_stream(pv + c * 32, pol);
            V4 f0, f1, f2, f3;
            gather4_tmz<MIR>(A, raw, s.src_v, f0, f1, f2, f3);
            hx.add(wv.x, f0.y); hx.add(wv.y, f1.y); hx.add(wv.z, f2.y); hx.add(wv.w, f3.y);
            hy.add(wv.x, f0.z); hy.add(wv.y, f1.z); hy.add(wv.z, f2.z); hy.add(wv.w, f3.z);
            he.add(wv.x, f0.x); he.add(wv.y, f1.x); he.add(wv.z, f2.x); he.add(wv.w, f3.x);
        }
    }
#pragma unroll
    for (int off = 1; off < P; off <<= 1) {
        ax.merge_xor(off);
        ay.merge_xor(off);
        hx.merge_xor(off);
        hy.merge_xor(off);
        he.merge_xor(off);
    }
    dxE = ax.get();
    dyE = ay.get();
    vx = hx.get();
    vy = hy.get();
    ve = he.get();
}

template <typename T, int NC, int NV, bool SHARED, bool COMP, int P, bool MIR = false>
__global__ void __launch_bounds__(512) k_h_colloc(StencilStreams<T> s, Coefs<T> k,
                                                  const typename Vec<T>::V4* __restrict__ A,
                                                  typename Vec<T>::V4* __restrict__ B) {
    using V4 = typename Vec<T>::V4;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t i = t / P;
    const int part = (int)(t % P);
    if (P == 1 && i >= s.n) return;  // with P > 1 every lane takes part in the merges
    T dxE, dyE, vx, vy, ve;
    h_colloc_node<T, NC, NV, SHARED, COMP, P, MIR>(s, A, i, dxE, dyE, vx, vy, ve, i < s.n, part);
    if (i >= s.n || part != 0) return;
    const V4 me = ld_gather(A + i);
    V4 out;
    out.x = me.x + me.w * (k.gamma * ve);
    out.y = me.y - k.ch * (dyE - k.gamma * vx);
    out.z = me.z + k.ch * (dxE + k.gamma * vy);
    out.w = me.w;
    st4(B + i, out);
}

template <typename T, int NC, bool SHARED, bool COMP, int P, bool MIR = false>
__global__ void __launch_bounds__(512) k_e_colloc(StencilStreams<T> s, const typename Vec<T>::V4* __restrict__ B,
                                                  typename Vec<T>::V4* __restrict__ A) {
    using V4 = typename Vec<T>::V4;
    using Acc = typename AccSel<T, COMP>::type;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t i = t / P;
    const int part = (int)(t % P);
    if (P == 1 && i >= s.n) return;  // with P > 1 every lane takes part in the merges
    const bool act = i < s.n;
    const int nc = NC ? NC : s.nc;
    const int ni = SHARED ? s.ni : nc;
    const int64_t slice = i >> 5;
    const int lane = (int)(i & 31);
    const int4* ip = s.idx_c + slice * ni * 32 + lane;
    const V4* px = s.wx + slice * nc * 32 + lane;
    const V4* py = s.wy + slice * nc * 32 + lane;
    const uint64_t pol = stream_policy(s.l2_keep);
    Acc dxHy, dyHx;
#pragma unroll
    for (int c = part; c < (act ? nc : 0); c += P) {
        const int4 raw = ld_stream(ip + c * 32, pol);
        const V4 wx = ld_stream(px + c * 32, pol), wy = ld_stream(py + c * 32, pol);
        V4 f0, f1, f2, f3;
        gather4_tmz<MIR>(B, raw, s.src_c, f0, f1, f2, f3);
        dxHy.add(wx.x, f0.z); dxHy.add(wx.y, f1.z); dxHy.add(wx.z, f2.z); dxHy.add(wx.w, f3.z);
        dyHx.add(wy.x, f0.y); dyHx.add(wy.y, f1.y); dyHx.add(wy.z, f2.y); dyHx.add(wy.w, f3.y);
    }
#pragma unroll
    for (int off = 1; off < P; off <<= 1) {
        dxHy.merge_xor(off);
        dyHx.merge_xor(off);
    }
    if (!act || part != 0) return;
    const V4 me = ld_gather(B + i);
    V4 out;
    out.x = me.x + me.w * (dxHy.get() - dyHx.get());
    out.y = me.y;
    out.z = me.z;
    out.w = me.w;
    st4(A + i, out);
}

// energy (Eq. 20) of the collocated state at t_n: H averaged with the H
// update computed on the fly; per-block partial sums in FP64
template <typename T, bool COMP, bool MIR = false>
__global__ void __launch_bounds__(256) k_energy_colloc(StencilStreams<T> s, Coefs<T> k,
                                                       const typename Vec<T>::V4* __restrict__ A,
                                                       const double* __restrict__ eps_r, double eta2,
                                                       double* __restrict__ partial) {
    using V4 = typename Vec<T>::V4;
    __shared__ double red[256];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double u = 0.0;
    if (i < s.n) {
        T dxE, dyE, vx, vy, ve;
        if (s.idx_v == s.idx_c)
            h_colloc_node<T, 0, 0, true, COMP, 1, MIR>(s, A, i, dxE, dyE, vx, vy, ve);
        else
            h_colloc_node<T, 0, 0, false, COMP, 1, MIR>(s, A, i, dxE, dyE, vx, vy, ve);
        const V4 me = A[i];
        const double hx1 = (double)(me.y - k.ch * (dyE - k.gamma * vx));
        const double hy1 = (double)(me.z + k.ch * (dxE + k.gamma * vy));
        const double ax = 0.5 * ((double)me.y + hx1), ay = 0.5 * ((double)me.z + hy1);
        u = eps_r[i] * (double)me.x * (double)me.x + eta2 * (ax * ax + ay * ay);
    }
    red[threadIdx.x] = u;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// ------------------------------------------------------------ staggered

template <typename T, int NC, int NV, bool COMP, bool KEEP>
__device__ __forceinline__ void h_stag_node(const StencilStreams<T>& s, const T* __restrict__ Ez,
                                            const typename Vec<T>::V2* __restrict__ H, int64_t i, T& dxE, T& dyE,
                                            T& vx, T& vy) {
    using V4 = typename Vec<T>::V4;
    using V2 = typename Vec<T>::V2;
    using Acc = typename AccSel<T, COMP>::type;
    using AccV = AccPlain<T>;
    const int nc = NC ? NC : s.nc;
    const int nv = NV ? NV : s.nv;
    const int64_t slice = i >> 5;
    const int lane = (int)(i & 31);
    const V4* px = s.wx + slice * nc * 32 + lane;
    const V4* py = s.wy + slice * nc * 32 + lane;
    const V4* pv = s.wv + slice * nv * 32 + lane;
    const uint64_t pol = KEEP ? stream_policy(s.l2_keep) : 0;
    Acc ax, ay;
    AccV hx, hy;
    // HV sums first: their H gathers are the larger share of the pass's loads, and issuing them
    // first measured 4 % faster than curl-first (the sums themselves do not depend on the order)
    for_idx4<NV, KEEP>(nv, slice, lane, s.idx_v, s.q_v, s.qb_v, s.src_v, pol, [&](int c, int4 id) {
        const V4 wv = ld_stream_k<KEEP>(pv + c * 32, pol);
        const V2 f0 = ld_gather(H + id.x), f1 = ld_gather(H + id.y);
        const V2 f2 = ld_gather(H + id.z), f3 = ld_gather(H + id.w);
        hx.add(wv.x, f0.x); hx.add(wv.y, f1.x); hx.add(wv.z, f2.x); hx.add(wv.w, f3.x);
        hy.add(wv.x, f0.y); hy.add(wv.y, f1.y); hy.add(wv.z, f2.y); hy.add(wv.w, f3.y);
    });
    for_idx4<NC, KEEP>(nc, slice, lane, s.idx_c, s.q_c, s.qb_c, s.src_c, pol, [&](int c, int4 id) {
        const V4 wx = ld_stream_k<KEEP>(px + c * 32, pol), wy = ld_stream_k<KEEP>(py + c * 32, pol);
        const T f0 = ld_gather(Ez + id.x), f1 = ld_gather(Ez + id.y);
        const T f2 = ld_gather(Ez + id.z), f3 = ld_gather(Ez + id.w);
        ax.add(wx.x, f0); ax.add(wx.y, f1); ax.add(wx.z, f2); ax.add(wx.w, f3);
        ay.add(wy.x, f0); ay.add(wy.y, f1); ay.add(wy.z, f2); ay.add(wy.w, f3);
    });
    dxE = ax.get();
    dyE = ay.get();
    vx = hx.get();
    vy = hy.get();
}

template <typename T, int NC, int NV, bool COMP, bool KEEP>
__global__ void __launch_bounds__(512) k_h_stag(StencilStreams<T> s, Coefs<T> k, const T* __restrict__ Ez,
                                                const typename Vec<T>::V2* __restrict__ H,
                                                typename Vec<T>::V2* __restrict__ Hn) {
    using V2 = typename Vec<T>::V2;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    T dxE, dyE, vx, vy;
    h_stag_node<T, NC, NV, COMP, KEEP>(s, Ez, H, i, dxE, dyE, vx, vy);
    const V2 me = ld_gather(H + i);
    V2 out;
    out.x = me.x - k.ch * (dyE - k.gamma * vx);
    out.y = me.y + k.ch * (dxE + k.gamma * vy);
    Hn[i] = out;
}

template <typename T, int NC, int NV, bool COMP, bool KEEP>
__global__ void __launch_bounds__(512) k_e_stag(StencilStreams<T> s, Coefs<T> k, const typename Vec<T>::V2* __restrict__ Hn,
                                                const T* __restrict__ Ez, const T* __restrict__ ce,
                                                T* __restrict__ Ezn) {
    using V4 = typename Vec<T>::V4;
    using V2 = typename Vec<T>::V2;
    using Acc = typename AccSel<T, COMP>::type;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    const int nc = NC ? NC : s.nc;
    const int nv = NV ? NV : s.nv;
    const int64_t slice = i >> 5;
    const int lane = (int)(i & 31);
    const V4* px = s.wx + slice * nc * 32 + lane;
    const V4* py = s.wy + slice * nc * 32 + lane;
    const V4* pv = s.wv + slice * nv * 32 + lane;
    const uint64_t pol = KEEP ? stream_policy(s.l2_keep) : 0;
    Acc dxHy, dyHx;
    AccPlain<T> he;
    for_idx4<NC, KEEP>(nc, slice, lane, s.idx_c, s.q_c, s.qb_c, s.src_c, pol, [&](int c, int4 id) {
        const V4 wx = ld_stream_k<KEEP>(px + c * 32, pol), wy = ld_stream_k<KEEP>(py + c * 32, pol);
        const V2 f0 = ld_gather(Hn + id.x), f1 = ld_gather(Hn + id.y);
        const V2 f2 = ld_gather(Hn + id.z), f3 = ld_gather(Hn + id.w);
        dxHy.add(wx.x, f0.y); dxHy.add(wx.y, f1.y); dxHy.add(wx.z, f2.y); dxHy.add(wx.w, f3.y);
        dyHx.add(wy.x, f0.x); dyHx.add(wy.y, f1.x); dyHx.add(wy.z, f2.x); dyHx.add(wy.w, f3.x);
    });
    for_idx4<NV, KEEP>(nv, slice, lane, s.idx_v, s.q_v, s.qb_v, s.src_v, pol, [&](int c, int4 id) {
        const V4 wv = ld_stream_k<KEEP>(pv + c * 32, pol);
        const T f0 = ld_gather(Ez + id.x), f1 = ld_gather(Ez + id.y);
        const T f2 = ld_gather(Ez + id.z), f3 = ld_gather(Ez + id.w);
        he.add(wv.x, f0); he.add(wv.y, f1); he.add(wv.z, f2); he.add(wv.w, f3);
    });
    const T e = ld_gather(Ez + i);
    Ezn[i] = e + ld_gather(ce + i) * (dxHy.get() - dyHx.get() + k.gamma * he.get());
}

template <typename T, bool COMP>
__global__ void __launch_bounds__(256) k_energy_stag(StencilStreams<T> s, Coefs<T> k, const T* __restrict__ Ez,
                                                     const typename Vec<T>::V2* __restrict__ H,
                                                     const double* __restrict__ eps_r, int64_t ne, double eta2,
                                                     double* __restrict__ partial) {
    using V2 = typename Vec<T>::V2;
    __shared__ double red[256];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double u = 0.0;
    if (i < s.n) {
        T dxE, dyE, vx, vy;
        h_stag_node<T, 0, 0, COMP, true>(s, Ez, H, i, dxE, dyE, vx, vy);
        const V2 me = H[i];
        const double hx1 = (double)(me.x - k.ch * (dyE - k.gamma * vx));
        const double hy1 = (double)(me.y + k.ch * (dxE + k.gamma * vy));
        const double ax = 0.5 * ((double)me.x + hx1), ay = 0.5 * ((double)me.y + hy1);
        u = eta2 * (ax * ax + ay * ay);
    }
    if (i < ne) u += eps_r[i] * (double)Ez[i] * (double)Ez[i];
    red[threadIdx.x] = u;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// ------------------------------------------------------------ dispatch

template <typename T, bool COMP, int P>
static cudaError_t launch_colloc_pass_p(int pass, const StencilStreams<T>& s, const Coefs<T>& k, void* A, void* B,
                                        int block, cudaStream_t st) {
    using V4 = typename Vec<T>::V4;
    const bool shared = s.idx_v == s.idx_c;
    const unsigned grid = (unsigned)((s.n * P + block - 1) / block);
    V4* a = static_cast<V4*>(A);
    V4* b = static_cast<V4*>(B);
#define MFD_H(NC, NV)                                                                       \
    if (s.nc == NC && s.nv == NV) {                                                         \
        if (shared) k_h_colloc<T, NC, NV, true, COMP, P><<<grid, block, 0, st>>>(s, k, a, b); \
        else k_h_colloc<T, NC, NV, false, COMP, P><<<grid, block, 0, st>>>(s, k, a, b);       \
        return cudaGetLastError();                                                          \
    }
#define MFD_E(NC)                                                                        \
    if (s.nc == NC) {                                                                    \
        if (shared) k_e_colloc<T, NC, true, COMP, P><<<grid, block, 0, st>>>(s, b, a);     \
        else k_e_colloc<T, NC, false, COMP, P><<<grid, block, 0, st>>>(s, b, a);           \
        return cudaGetLastError();                                                       \
    }
    if (s.mirror) {  // node sets with mirror walls: the generic kernels with image codes
        if (pass == 0) {
            if (shared) k_h_colloc<T, 0, 0, true, COMP, P, true><<<grid, block, 0, st>>>(s, k, a, b);
            else k_h_colloc<T, 0, 0, false, COMP, P, true><<<grid, block, 0, st>>>(s, k, a, b);
        } else {
            if (shared) k_e_colloc<T, 0, true, COMP, P, true><<<grid, block, 0, st>>>(s, b, a);
            else k_e_colloc<T, 0, false, COMP, P, true><<<grid, block, 0, st>>>(s, b, a);
        }
        return cudaGetLastError();
    }
    if (pass == 0) {
        MFD_H(3, 8) MFD_H(5, 8) MFD_H(8, 8) MFD_H(10, 8)
        if (shared) k_h_colloc<T, 0, 0, true, COMP, P><<<grid, block, 0, st>>>(s, k, a, b);
        else k_h_colloc<T, 0, 0, false, COMP, P><<<grid, block, 0, st>>>(s, k, a, b);
    } else {
        MFD_E(3) MFD_E(5) MFD_E(8) MFD_E(10)
        if (shared) k_e_colloc<T, 0, true, COMP, P><<<grid, block, 0, st>>>(s, b, a);
        else k_e_colloc<T, 0, false, COMP, P><<<grid, block, 0, st>>>(s, b, a);
    }
#undef MFD_H
#undef MFD_E
    return cudaGetLastError();
}

// lanes per node: 2, 4 or 8 to put more threads on each node's gathers
template <typename T, bool COMP>
static cudaError_t launch_colloc_pass(int pass, const StencilStreams<T>& s, const Coefs<T>& k, void* A, void* B,
                                      int block, cudaStream_t st, int lanes) {
    if (lanes == 8) return launch_colloc_pass_p<T, COMP, 8>(pass, s, k, A, B, block, st);
    if (lanes == 4) return launch_colloc_pass_p<T, COMP, 4>(pass, s, k, A, B, block, st);
    if (lanes == 2) return launch_colloc_pass_p<T, COMP, 2>(pass, s, k, A, B, block, st);
    return launch_colloc_pass_p<T, COMP, 1>(pass, s, k, A, B, block, st);
}

template <typename T, bool COMP, bool KEEP>
static cudaError_t launch_stag_pass_k(int pass, const StencilStreams<T>& s, const Coefs<T>& k, const Stag2DPtrs& p,
                                      int block, cudaStream_t st) {
    using V2 = typename Vec<T>::V2;
    const unsigned grid = (unsigned)((s.n + block - 1) / block);
    const T* ez = static_cast<const T*>(p.ez);
    T* ezn = static_cast<T*>(p.ezn);
    const V2* h = static_cast<const V2*>(p.h);
    V2* hn = static_cast<V2*>(p.hn);
    const T* ce = static_cast<const T*>(p.ce);
    if (pass == 0) {
        if (s.nc == 8 && s.nv == 15) k_h_stag<T, 8, 15, COMP, KEEP><<<grid, block, 0, st>>>(s, k, ez, h, hn);
        else if (s.nc == 3 && s.nv == 8) k_h_stag<T, 3, 8, COMP, KEEP><<<grid, block, 0, st>>>(s, k, ez, h, hn);
        else k_h_stag<T, 0, 0, COMP, KEEP><<<grid, block, 0, st>>>(s, k, ez, h, hn);
    } else {
        if (s.nc == 8 && s.nv == 15) k_e_stag<T, 8, 15, COMP, KEEP><<<grid, block, 0, st>>>(s, k, hn, ez, ce, ezn);
        else if (s.nc == 3 && s.nv == 8) k_e_stag<T, 3, 8, COMP, KEEP><<<grid, block, 0, st>>>(s, k, hn, ez, ce, ezn);
        else k_e_stag<T, 0, 0, COMP, KEEP><<<grid, block, 0, st>>>(s, k, hn, ez, ce, ezn);
    }
    return cudaGetLastError();
}

// streams kept in L2 (keep > 0) or every line evict_first
template <typename T, bool COMP>
static cudaError_t launch_stag_pass(int pass, const StencilStreams<T>& s, const Coefs<T>& k, const Stag2DPtrs& p,
                                    int block, cudaStream_t st) {
    return s.l2_keep > 0.0f ? launch_stag_pass_k<T, COMP, true>(pass, s, k, p, block, st)
                            : launch_stag_pass_k<T, COMP, false>(pass, s, k, p, block, st);
}

cudaError_t launch_2d(const Launch2D& L, int pass, cudaStream_t st) {
    const int b = L.block[pass];
    if (L.staggered) {
        if (L.fp64) return launch_stag_pass<double, false>(pass, pass == 0 ? L.hs.d : L.es.d, L.kd, L.stag, b, st);
        if (L.comp) return launch_stag_pass<float, true>(pass, pass == 0 ? L.hs.f : L.es.f, L.kf, L.stag, b, st);
        return launch_stag_pass<float, false>(pass, pass == 0 ? L.hs.f : L.es.f, L.kf, L.stag, b, st);
    }
    if (L.fp64) return launch_colloc_pass<double, false>(pass, L.hs.d, L.kd, L.A, L.B, b, st, L.lanes[pass]);
    if (L.comp) return launch_colloc_pass<float, true>(pass, L.hs.f, L.kf, L.A, L.B, b, st, L.lanes[pass]);
    return launch_colloc_pass<float, false>(pass, L.hs.f, L.kf, L.A, L.B, b, st, L.lanes[pass]);
}

cudaError_t launch_energy_2d(const Launch2D& L, const double* eps_r, int64_t ne, double eta2, double* partial,
                             unsigned grid, cudaStream_t st) {
    if (L.staggered) {
        if (L.fp64)
            k_energy_stag<double, false><<<grid, 256, 0, st>>>(L.hs.d, L.kd, (const double*)L.stag.ez,
                                                               (const double2*)L.stag.h, eps_r, ne, eta2, partial);
        else if (L.comp)
            k_energy_stag<float, true><<<grid, 256, 0, st>>>(L.hs.f, L.kf, (const float*)L.stag.ez,
                                                             (const float2*)L.stag.h, eps_r, ne, eta2, partial);
        else
            k_energy_stag<float, false><<<grid, 256, 0, st>>>(L.hs.f, L.kf, (const float*)L.stag.ez,
                                                              (const float2*)L.stag.h, eps_r, ne, eta2, partial);
    } else if (L.hs.f.mirror) {
        if (L.fp64)
            k_energy_colloc<double, false, true><<<grid, 256, 0, st>>>(L.hs.d, L.kd, (const dbl4*)L.A, eps_r, eta2,
                                                                      partial);
        else if (L.comp)
            k_energy_colloc<float, true, true><<<grid, 256, 0, st>>>(L.hs.f, L.kf, (const float4*)L.A, eps_r, eta2,
                                                                    partial);
        else
            k_energy_colloc<float, false, true><<<grid, 256, 0, st>>>(L.hs.f, L.kf, (const float4*)L.A, eps_r, eta2,
                                                                     partial);
    } else {
        if (L.fp64)
            k_energy_colloc<double, false><<<grid, 256, 0, st>>>(L.hs.d, L.kd, (const dbl4*)L.A, eps_r, eta2, partial);
        else if (L.comp)
            k_energy_colloc<float, true><<<grid, 256, 0, st>>>(L.hs.f, L.kf, (const float4*)L.A, eps_r, eta2, partial);
        else
            k_energy_colloc<float, false><<<grid, 256, 0, st>>>(L.hs.f, L.kf, (const float4*)L.A, eps_r, eta2, partial);
    }
    return cudaGetLastError();
}

unsigned long long bounds_take_step2d(cudaStream_t s) { return bounds_take_local(s); }

}  // namespace mfd
