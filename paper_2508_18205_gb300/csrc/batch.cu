// batch.cu -- many independent collocated TMz domains, each with R right-hand
// sides (field vectors sharing the domain's weights), stepped by ONE persistent
// cooperative kernel that runs all the steps (Eq. 19 per domain and per
// right-hand side), captured in a CUDA graph.
//
// Work decomposition: each node is owned by R/4 consecutive lanes, lane q
// holding right-hand sides 4q .. 4q+3, so one 128-bit gather brings four
// right-hand sides of one field of a neighbour; a warp owns 32/(R/4) nodes
// (8 for R = 16) and a block of 8 warps one tile of 8 x 32/(R/4) nodes. Tiles
// never span two domains; the resident blocks walk the tile list round-robin.
// The stencil streams of a warp's nodes are interleaved ([slice of a warp's
// nodes][chunk][node][4 entries]) so the distinct 16-byte stream reads of a
// warp instruction form one contiguous line; the lanes of a node read the
// same address (broadcast).
//
// Phases per step: H pass over all tiles (writes E* and H'), grid barrier,
// E pass over all tiles (writes E', then the block adds its tile's soft
// sources and records its tile's probes), grid barrier. The barrier spins a
// bounded number of times; on time-out it raises an error flag that every
// block checks, all blocks leave the kernel, and the host reports
// MFD_ERR_TIMEOUT.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "internal.cuh"
#include "kernels.cuh"

namespace mfd {

constexpr int BT_THREADS = 256;  // 8 warps; a tile is 8 x (32 / (R / 4)) nodes (64 for R = 16)

struct BDom {
    int64_t node0;   // first global node
    int64_t idx0;    // first int4 of the domain's index stream
    int64_t wc0;     // first float4 of the domain's curl weight streams
    int64_t wv0;     // first float4 of the domain's HV weight stream
    int n, nc, nv, ni;
    float ch;
    double dt;
};

struct BTile {
    int dom;
    int first;  // first local node
};

struct BArgs {
    const BDom* dom;
    const BTile* tile;
    int ntile;
    const int4* idx;
    const float4* wx;
    const float4* wy;
    const float4* wv;
    float* A;   // [node][3][R]: Ez, Hx, Hy
    float* B;   // [node][3][R]: E*, Hx', Hy'
    float* Hs;  // [node][2][R]: H* = H + (dt/mu0) gamma D H of the current H (variants 2, 3)
    const float* ce;
    const float* gam;  // [domain][R]: the hyperviscosity coefficient gamma of every right-hand side
    // sources grouped by tile
    const int* src_start;  // ntile + 1
    const int64_t* src_node;
    const int* src_rhs;
    const double* src_amp;
    const double* src_f0;
    const double* src_t0;
    // probes grouped by tile
    const int* prb_start;  // ntile + 1
    const int64_t* prb_node;
    const int* prb_slot;
    float* prb_buf;  // [rec][slots][R]
    int prb_slots;
    int64_t prb_cap;
    const int64_t* pstep0;
    int64_t* counter;
    int nsteps;
    unsigned int* bar;  // [0] arrivals, [1] generation, [2] error flag
    unsigned long long spin_limit;
    int64_t ntot;  // nodes over all domains (the range of the stencil indices)
};

__device__ __forceinline__ float4 f4_fma(float w, float4 f, float4 a) {
    a.x = fmaf(w, f.x, a.x);
    a.y = fmaf(w, f.y, a.y);
    a.z = fmaf(w, f.z, a.z);
    a.w = fmaf(w, f.w, a.w);
    return a;
}

__device__ __forceinline__ float4 ld_f4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st_f4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

// grid-wide barrier with a bounded wait; returns false once any block timed out
__device__ bool grid_barrier(unsigned int* bar, unsigned long long limit) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* vb = bar;
        const unsigned int gen = vb[1];
        __threadfence();
        const unsigned int arrived = atomicAdd(&bar[0], 1u);
        if (arrived == gridDim.x - 1) {
            bar[0] = 0;
            __threadfence();
            atomicAdd(&bar[1], 1u);
        } else {
            unsigned long long spins = 0;
            while (vb[1] == gen) {
                if (vb[2] != 0u) break;
                if (++spins > limit) {
                    atomicExch(&bar[2], 1u);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok = (vb[2] == 0u);
    }
    __syncthreads();
    return ok != 0;
}

// PF: the stream values of chunk c + 1 are requested before the gathers of
// chunk c (more registers, DRAM latency of the streams hidden in the warp);
// without PF each chunk's streams are loaded when it starts (fewer registers,
// more resident warps hide it). Both give the same sums in the same order.
template <int R, bool PF>
__device__ void h_tile(const BArgs& a, const BTile t) {
    constexpr int LPN = R / 4;         // lanes per node
    constexpr int NPW = 32 / LPN;      // nodes per warp
    const BDom d = a.dom[t.dom];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / LPN, q = lane % LPN;
    const int local = t.first + warp * NPW + g;
    if (local >= d.n) return;
    const int64_t slice = local / NPW;
    const int4* ip = a.idx + d.idx0 + slice * d.ni * NPW + g;
    const float4* px = a.wx + d.wc0 + slice * d.nc * NPW + g;
    const float4* py = a.wy + d.wc0 + slice * d.nc * NPW + g;
    const float4* pv = a.wv + d.wv0 + slice * d.nv * NPW + g;
    float4 dx = {0, 0, 0, 0}, dy = dx, vx = dx, vy = dx, ve = dx;
    const float4 z4 = {0, 0, 0, 0};
    int4 nid = PF ? chk4(ld_stream(ip), a.ntot) : make_int4(0, 0, 0, 0);
    float4 nwx = PF && d.nc > 0 ? ld_stream(px) : z4, nwy = PF && d.nc > 0 ? ld_stream(py) : z4;
    float4 nwv = PF && d.nv > 0 ? ld_stream(pv) : z4;
    for (int c = 0; c < d.ni; ++c) {
        int4 id;
        float4 wx, wy, wv;
        if constexpr (PF) {
            id = nid;
            wx = nwx;
            wy = nwy;
            wv = nwv;
            if (c + 1 < d.ni) {
                nid = chk4(ld_stream(ip + (c + 1) * NPW), a.ntot);
                nwx = c + 1 < d.nc ? ld_stream(px + (c + 1) * NPW) : z4;
                nwy = c + 1 < d.nc ? ld_stream(py + (c + 1) * NPW) : z4;
                nwv = c + 1 < d.nv ? ld_stream(pv + (c + 1) * NPW) : z4;
            }
        } else {
            id = chk4(ld_stream(ip + c * NPW), a.ntot);
            wx = c < d.nc ? ld_stream(px + c * NPW) : z4;
            wy = c < d.nc ? ld_stream(py + c * NPW) : z4;
            wv = c < d.nv ? ld_stream(pv + c * NPW) : z4;
        }
        const int ids[4] = {id.x, id.y, id.z, id.w};
        const float wxs[4] = {wx.x, wx.y, wx.z, wx.w}, wys[4] = {wy.x, wy.y, wy.z, wy.w};
        const float wvs[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float* f = a.A + (int64_t)ids[e] * 3 * R + 4 * q;
            const float4 ez = ld_f4(f), hx = ld_f4(f + R), hy = ld_f4(f + 2 * R);
            dx = f4_fma(wxs[e], ez, dx);
            dy = f4_fma(wys[e], ez, dy);
            vx = f4_fma(wvs[e], hx, vx);
            vy = f4_fma(wvs[e], hy, vy);
            ve = f4_fma(wvs[e], ez, ve);
        }
    }
    const int64_t i = d.node0 + local;
    const float cei = a.ce[i];
    const float* me = a.A + i * 3 * R + 4 * q;
    const float4 ez = ld_f4(me), hx = ld_f4(me + R), hy = ld_f4(me + 2 * R);
    const float4 gm = ld_f4(a.gam + t.dom * R + 4 * q);
    float4 es, hxn, hyn;
    es.x = ez.x + cei * (gm.x * ve.x);
    es.y = ez.y + cei * (gm.y * ve.y);
    es.z = ez.z + cei * (gm.z * ve.z);
    es.w = ez.w + cei * (gm.w * ve.w);
    hxn.x = hx.x - d.ch * (dy.x - gm.x * vx.x);
    hxn.y = hx.y - d.ch * (dy.y - gm.y * vx.y);
    hxn.z = hx.z - d.ch * (dy.z - gm.z * vx.z);
    hxn.w = hx.w - d.ch * (dy.w - gm.w * vx.w);
    hyn.x = hy.x + d.ch * (dx.x + gm.x * vy.x);
    hyn.y = hy.y + d.ch * (dx.y + gm.y * vy.y);
    hyn.z = hy.z + d.ch * (dx.z + gm.z * vy.z);
    hyn.w = hy.w + d.ch * (dx.w + gm.w * vy.w);
    float* out = a.B + i * 3 * R + 4 * q;
    st_f4(out, es);
    st_f4(out + R, hxn);
    st_f4(out + 2 * R, hyn);
}

template <int R, bool PF>
__device__ void e_tile(const BArgs& a, const BTile t) {
    constexpr int LPN = R / 4;
    constexpr int NPW = 32 / LPN;
    const BDom d = a.dom[t.dom];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / LPN, q = lane % LPN;
    const int local = t.first + warp * NPW + g;
    if (local < d.n) {
        const int64_t slice = local / NPW;
        const int4* ip = a.idx + d.idx0 + slice * d.ni * NPW + g;
        const float4* px = a.wx + d.wc0 + slice * d.nc * NPW + g;
        const float4* py = a.wy + d.wc0 + slice * d.nc * NPW + g;
        float4 dxhy = {0, 0, 0, 0}, dyhx = dxhy;
        int4 nid = PF ? chk4(ld_stream(ip), a.ntot) : make_int4(0, 0, 0, 0);
        float4 nwx = PF ? ld_stream(px) : dxhy, nwy = PF ? ld_stream(py) : dxhy;
        for (int c = 0; c < d.nc; ++c) {
            int4 id;
            float4 wx, wy;
            if constexpr (PF) {
                id = nid;
                wx = nwx;
                wy = nwy;
                if (c + 1 < d.nc) {
                    nid = chk4(ld_stream(ip + (c + 1) * NPW), a.ntot);
                    nwx = ld_stream(px + (c + 1) * NPW);
                    nwy = ld_stream(py + (c + 1) * NPW);
                }
            } else {
                id = chk4(ld_stream(ip + c * NPW), a.ntot);
                wx = ld_stream(px + c * NPW);
                wy = ld_stream(py + c * NPW);
            }
            const int ids[4] = {id.x, id.y, id.z, id.w};
            const float wxs[4] = {wx.x, wx.y, wx.z, wx.w}, wys[4] = {wy.x, wy.y, wy.z, wy.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float* f = a.B + (int64_t)ids[e] * 3 * R + 4 * q;
                dxhy = f4_fma(wxs[e], ld_f4(f + 2 * R), dxhy);
                dyhx = f4_fma(wys[e], ld_f4(f + R), dyhx);
            }
        }
        const int64_t i = d.node0 + local;
        const float cei = a.ce[i];
        const float* me = a.B + i * 3 * R + 4 * q;
        const float4 es = ld_f4(me), hx = ld_f4(me + R), hy = ld_f4(me + 2 * R);
        float4 ez;
        ez.x = es.x + cei * (dxhy.x - dyhx.x);
        ez.y = es.y + cei * (dxhy.y - dyhx.y);
        ez.z = es.z + cei * (dxhy.z - dyhx.z);
        ez.w = es.w + cei * (dxhy.w - dyhx.w);
        float* out = a.A + i * 3 * R + 4 * q;
        st_f4(out, ez);
        st_f4(out + R, hx);
        st_f4(out + 2 * R, hy);
    }
}

// Variants 2 and 3 move the hyperviscosity term of the H row (Eq. 19) one pass
// earlier. It depends only on H^{n-1/2}, which the E pass of the step before
// gathers anyway for its curl; so that pass gathers Hx', Hy' over the whole
// index row (the curl stencil is its first n entries, the HV stencil its first
// N_h), writes H* = H' + (dt/mu0) gamma D H' beside the state, and the next H
// pass gathers only Ez (curl and the E row's HV term) and reads its own node's
// H*. A node-step then gathers 3L field rows instead of 3L + 2n (L = max(n, N_h)).
// The same sums in the same order; the HV term is added to H before the curl
// term instead of after, so results agree with variants 0 and 1 to rounding.
template <int R, bool PF>
__device__ void h_tile_s(const BArgs& a, const BTile t) {
    constexpr int LPN = R / 4;
    constexpr int NPW = 32 / LPN;
    const BDom d = a.dom[t.dom];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / LPN, q = lane % LPN;
    const int local = t.first + warp * NPW + g;
    if (local >= d.n) return;
    const int64_t slice = local / NPW;
    const int4* ip = a.idx + d.idx0 + slice * d.ni * NPW + g;
    const float4* px = a.wx + d.wc0 + slice * d.nc * NPW + g;
    const float4* py = a.wy + d.wc0 + slice * d.nc * NPW + g;
    const float4* pv = a.wv + d.wv0 + slice * d.nv * NPW + g;
    float4 dx = {0, 0, 0, 0}, dy = dx, ve = dx;
    const float4 z4 = {0, 0, 0, 0};
    int4 nid = PF ? chk4(ld_stream(ip), a.ntot) : make_int4(0, 0, 0, 0);
    float4 nwx = PF && d.nc > 0 ? ld_stream(px) : z4, nwy = PF && d.nc > 0 ? ld_stream(py) : z4;
    float4 nwv = PF && d.nv > 0 ? ld_stream(pv) : z4;
    for (int c = 0; c < d.ni; ++c) {
        int4 id;
        float4 wx, wy, wv;
        if constexpr (PF) {
            id = nid;
            wx = nwx;
            wy = nwy;
            wv = nwv;
            if (c + 1 < d.ni) {
                nid = chk4(ld_stream(ip + (c + 1) * NPW), a.ntot);
                nwx = c + 1 < d.nc ? ld_stream(px + (c + 1) * NPW) : z4;
                nwy = c + 1 < d.nc ? ld_stream(py + (c + 1) * NPW) : z4;
                nwv = c + 1 < d.nv ? ld_stream(pv + (c + 1) * NPW) : z4;
            }
        } else {
            id = chk4(ld_stream(ip + c * NPW), a.ntot);
            wx = c < d.nc ? ld_stream(px + c * NPW) : z4;
            wy = c < d.nc ? ld_stream(py + c * NPW) : z4;
            wv = c < d.nv ? ld_stream(pv + c * NPW) : z4;
        }
        const int ids[4] = {id.x, id.y, id.z, id.w};
        const float wxs[4] = {wx.x, wx.y, wx.z, wx.w}, wys[4] = {wy.x, wy.y, wy.z, wy.w};
        const float wvs[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float4 ez = ld_f4(a.A + (int64_t)ids[e] * 3 * R + 4 * q);
            dx = f4_fma(wxs[e], ez, dx);
            dy = f4_fma(wys[e], ez, dy);
            ve = f4_fma(wvs[e], ez, ve);
        }
    }
    const int64_t i = d.node0 + local;
    const float cei = a.ce[i];
    const float4 ez = ld_f4(a.A + i * 3 * R + 4 * q);
    const float* hs = a.Hs + i * 2 * R + 4 * q;
    const float4 hx = ld_f4(hs), hy = ld_f4(hs + R);
    const float4 gm = ld_f4(a.gam + t.dom * R + 4 * q);
    float4 es, hxn, hyn;
    es.x = ez.x + cei * (gm.x * ve.x);
    es.y = ez.y + cei * (gm.y * ve.y);
    es.z = ez.z + cei * (gm.z * ve.z);
    es.w = ez.w + cei * (gm.w * ve.w);
    hxn.x = hx.x - d.ch * dy.x;
    hxn.y = hx.y - d.ch * dy.y;
    hxn.z = hx.z - d.ch * dy.z;
    hxn.w = hx.w - d.ch * dy.w;
    hyn.x = hy.x + d.ch * dx.x;
    hyn.y = hy.y + d.ch * dx.y;
    hyn.z = hy.z + d.ch * dx.z;
    hyn.w = hy.w + d.ch * dx.w;
    float* out = a.B + i * 3 * R + 4 * q;
    st_f4(out, es);
    st_f4(out + R, hxn);
    st_f4(out + 2 * R, hyn);
}

// H* of one node from the gathered HV sums: H + ch gamma (D H)
__device__ __forceinline__ float4 hstar(float4 h, float ch, float4 gm, float4 v) {
    h.x = h.x + ch * (gm.x * v.x);
    h.y = h.y + ch * (gm.y * v.y);
    h.z = h.z + ch * (gm.z * v.z);
    h.w = h.w + ch * (gm.w * v.w);
    return h;
}

// E pass of variants 2 and 3 (WRITE_E) and the prologue that makes H* of the
// current state (WRITE_E = false: reads A, writes Hs only)
template <int R, bool PF, bool WRITE_E>
__device__ void e_tile_s(const BArgs& a, const BTile t) {
    constexpr int LPN = R / 4;
    constexpr int NPW = 32 / LPN;
    const BDom d = a.dom[t.dom];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / LPN, q = lane % LPN;
    const int local = t.first + warp * NPW + g;
    if (local >= d.n) return;
    const float* src = WRITE_E ? a.B : a.A;  // H' after the H pass, or the current state
    const int64_t slice = local / NPW;
    const int4* ip = a.idx + d.idx0 + slice * d.ni * NPW + g;
    const float4* px = a.wx + d.wc0 + slice * d.nc * NPW + g;
    const float4* py = a.wy + d.wc0 + slice * d.nc * NPW + g;
    const float4* pv = a.wv + d.wv0 + slice * d.nv * NPW + g;
    const int nch = WRITE_E ? d.ni : d.nv;
    float4 dxhy = {0, 0, 0, 0}, dyhx = dxhy, vx = dxhy, vy = dxhy;
    const float4 z4 = {0, 0, 0, 0};
    int4 nid = PF ? chk4(ld_stream(ip), a.ntot) : make_int4(0, 0, 0, 0);
    float4 nwx = PF && WRITE_E && d.nc > 0 ? ld_stream(px) : z4, nwy = PF && WRITE_E && d.nc > 0 ? ld_stream(py) : z4;
    float4 nwv = PF && d.nv > 0 ? ld_stream(pv) : z4;
    for (int c = 0; c < nch; ++c) {
        int4 id;
        float4 wx, wy, wv;
        if constexpr (PF) {
            id = nid;
            wx = nwx;
            wy = nwy;
            wv = nwv;
            if (c + 1 < nch) {
                nid = chk4(ld_stream(ip + (c + 1) * NPW), a.ntot);
                nwx = WRITE_E && c + 1 < d.nc ? ld_stream(px + (c + 1) * NPW) : z4;
                nwy = WRITE_E && c + 1 < d.nc ? ld_stream(py + (c + 1) * NPW) : z4;
                nwv = c + 1 < d.nv ? ld_stream(pv + (c + 1) * NPW) : z4;
            }
        } else {
            id = chk4(ld_stream(ip + c * NPW), a.ntot);
            wx = WRITE_E && c < d.nc ? ld_stream(px + c * NPW) : z4;
            wy = WRITE_E && c < d.nc ? ld_stream(py + c * NPW) : z4;
            wv = c < d.nv ? ld_stream(pv + c * NPW) : z4;
        }
        const int ids[4] = {id.x, id.y, id.z, id.w};
        const float wxs[4] = {wx.x, wx.y, wx.z, wx.w}, wys[4] = {wy.x, wy.y, wy.z, wy.w};
        const float wvs[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float* f = src + (int64_t)ids[e] * 3 * R + 4 * q;
            const float4 hx = ld_f4(f + R), hy = ld_f4(f + 2 * R);
            if constexpr (WRITE_E) {
                dxhy = f4_fma(wxs[e], hy, dxhy);
                dyhx = f4_fma(wys[e], hx, dyhx);
            }
            vx = f4_fma(wvs[e], hx, vx);
            vy = f4_fma(wvs[e], hy, vy);
        }
    }
    const int64_t i = d.node0 + local;
    const float* me = src + i * 3 * R + 4 * q;
    const float4 hx = ld_f4(me + R), hy = ld_f4(me + 2 * R);
    const float4 gm = ld_f4(a.gam + t.dom * R + 4 * q);
    float* hs = a.Hs + i * 2 * R + 4 * q;
    st_f4(hs, hstar(hx, d.ch, gm, vx));
    st_f4(hs + R, hstar(hy, d.ch, gm, vy));
    if constexpr (WRITE_E) {
        const float cei = a.ce[i];
        const float4 es = ld_f4(me);
        float4 ez;
        ez.x = es.x + cei * (dxhy.x - dyhx.x);
        ez.y = es.y + cei * (dxhy.y - dyhx.y);
        ez.z = es.z + cei * (dxhy.z - dyhx.z);
        ez.w = es.w + cei * (dxhy.w - dyhx.w);
        float* out = a.A + i * 3 * R + 4 * q;
        st_f4(out, ez);
        st_f4(out + R, hx);
        st_f4(out + 2 * R, hy);
    }
}

// H* of the current state for every tile (one block per tile): run before the
// first launch of variants 2 and 3 after the state or gamma changed on the host
template <int R>
__global__ void __launch_bounds__(BT_THREADS) k_bhstar(BArgs a) { e_tile_s<R, false, false>(a, a.tile[blockIdx.x]); }

// variant 0: stream prefetch, three resident blocks of 256 per SM (80
// registers); variant 1: no prefetch, four resident blocks (64 registers);
// variants 2 and 3: the same two with the H row's HV term in the E pass (H*)
template <int R, int V>
__global__ void __launch_bounds__(BT_THREADS, (V & 1) ? 4 : 3) k_batch(BArgs a) {
    constexpr bool PF = (V & 1) == 0;
    constexpr bool HS = V >= 2;
    __shared__ int64_t step0_s;
    if (threadIdx.x == 0) step0_s = *a.counter;
    __syncthreads();
    const int64_t step0 = step0_s;
    const double pi = 3.14159265358979323846;
    for (int s = 0; s < a.nsteps; ++s) {
        for (int k = blockIdx.x; k < a.ntile; k += gridDim.x) {
            if constexpr (HS) h_tile_s<R, PF>(a, a.tile[k]);
            else h_tile<R, PF>(a, a.tile[k]);
        }
        if (!grid_barrier(a.bar, a.spin_limit)) return;
        const int64_t n = step0 + s;  // step n -> n + 1
        for (int k = blockIdx.x; k < a.ntile; k += gridDim.x) {
            const BTile t = a.tile[k];
            if constexpr (HS) e_tile_s<R, PF, true>(a, t);
            else e_tile<R, PF>(a, t);
            __syncthreads();
            const int s0 = a.src_start[k], s1 = a.src_start[k + 1];
            if (s1 > s0) {
                const double t1 = (double)(n + 1) * a.dom[t.dom].dt;
                for (int j = s0 + threadIdx.x; j < s1; j += blockDim.x) {
                    const int64_t node = a.src_node[j];
                    if (a.ce[node] == 0.0f) continue;
                    double x = pi * a.src_f0[j] * (t1 - a.src_t0[j]);
                    x = x * x;
                    const double r = (1.0 - 2.0 * x) * exp(-x);
                    atomicAdd(a.A + node * 3 * R + a.src_rhs[j], (float)(a.src_amp[j] * r));
                }
                __syncthreads();
            }
            const int p0 = a.prb_start[k], p1 = a.prb_start[k + 1];
            if (p1 > p0) {
                const int64_t rec = n - *a.pstep0;
                if (rec >= 0 && rec < a.prb_cap)
                    for (int j = p0 * R + threadIdx.x; j < p1 * R; j += blockDim.x) {
                        const int p = j / R, r = j % R;
                        a.prb_buf[(rec * a.prb_slots + a.prb_slot[p]) * R + r] = a.A[a.prb_node[p] * 3 * R + r];
                    }
            }
            __syncthreads();
        }
        if (!grid_barrier(a.bar, a.spin_limit)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.counter = step0 + a.nsteps;
}

// ---- packing: [slice of NPW nodes][chunk][node][4 entries], global ids / FP32 weights
// Eq. 20 per right-hand side of one domain, with H averaged between the
// half steps: the H half step of the current state is recomputed (not
// written) and U_r = sum_i eps_r,i Ez_i^2 + eta0^2 |(H^{n-1/2} + H^{n+1/2}) / 2|^2,
// eps_r,i = dt / (eps0 ce_i) (PEC nodes hold Ez = 0). One block per tile of the
// domain writes its partial sums (fixed order, so the result is reproducible).
template <int R>
__global__ void __launch_bounds__(BT_THREADS) k_benergy(BArgs a, int dom, int tile0, double eta2, double dt_eps0,
                                                        double* __restrict__ partial) {
    constexpr int LPN = R / 4;
    constexpr int NPW = 32 / LPN;
    constexpr int TN = 8 * NPW;
    __shared__ double acc[TN][R];
    const BTile t = a.tile[tile0 + blockIdx.x];
    const BDom d = a.dom[dom];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / LPN, q = lane % LPN;
    const int slot = warp * NPW + g;
    const int local = t.first + slot;
    double u[4] = {0.0, 0.0, 0.0, 0.0};
    if (local < d.n) {
        const int64_t sl = local / NPW;
        const int4* ip = a.idx + d.idx0 + sl * d.ni * NPW + g;
        const float4* px = a.wx + d.wc0 + sl * d.nc * NPW + g;
        const float4* py = a.wy + d.wc0 + sl * d.nc * NPW + g;
        const float4* pv = a.wv + d.wv0 + sl * d.nv * NPW + g;
        float4 dx = {0, 0, 0, 0}, dy = dx, vx = dx, vy = dx;
        for (int c = 0; c < d.ni; ++c) {
            const int4 id = chk4(ip[c * NPW], a.ntot);
            const int ids[4] = {id.x, id.y, id.z, id.w};
            const float4 wx = c < d.nc ? px[c * NPW] : make_float4(0, 0, 0, 0);
            const float4 wy = c < d.nc ? py[c * NPW] : make_float4(0, 0, 0, 0);
            const float4 wv = c < d.nv ? pv[c * NPW] : make_float4(0, 0, 0, 0);
            const float wxs[4] = {wx.x, wx.y, wx.z, wx.w}, wys[4] = {wy.x, wy.y, wy.z, wy.w};
            const float wvs[4] = {wv.x, wv.y, wv.z, wv.w};
            for (int e = 0; e < 4; ++e) {
                const float* f = a.A + (int64_t)ids[e] * 3 * R + 4 * q;
                const float4 ez = ld_f4(f), hx = ld_f4(f + R), hy = ld_f4(f + 2 * R);
                dx = f4_fma(wxs[e], ez, dx);
                dy = f4_fma(wys[e], ez, dy);
                vx = f4_fma(wvs[e], hx, vx);
                vy = f4_fma(wvs[e], hy, vy);
            }
        }
        const int64_t i = d.node0 + local;
        const float cei = a.ce[i];
        const float* me = a.A + i * 3 * R + 4 * q;
        const float4 ez = ld_f4(me), hx = ld_f4(me + R), hy = ld_f4(me + 2 * R);
        const float4 gm = ld_f4(a.gam + dom * R + 4 * q);
        const float ezs[4] = {ez.x, ez.y, ez.z, ez.w}, hxs[4] = {hx.x, hx.y, hx.z, hx.w};
        const float hys[4] = {hy.x, hy.y, hy.z, hy.w}, gs[4] = {gm.x, gm.y, gm.z, gm.w};
        const float dxs[4] = {dx.x, dx.y, dx.z, dx.w}, dys[4] = {dy.x, dy.y, dy.z, dy.w};
        const float vxs[4] = {vx.x, vx.y, vx.z, vx.w}, vys[4] = {vy.x, vy.y, vy.z, vy.w};
        const double er = cei > 0.0f ? dt_eps0 / (double)cei : 0.0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float hx1 = hxs[k] - d.ch * (dys[k] - gs[k] * vxs[k]);
            const float hy1 = hys[k] + d.ch * (dxs[k] + gs[k] * vys[k]);
            const double ax = 0.5 * ((double)hxs[k] + (double)hx1), ay = 0.5 * ((double)hys[k] + (double)hy1);
            u[k] = er * (double)ezs[k] * (double)ezs[k] + eta2 * (ax * ax + ay * ay);
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[slot][4 * q + k] = u[k];
    __syncthreads();
    if (threadIdx.x < R) {
        double s = 0.0;
        for (int j = 0; j < TN; ++j) s += acc[j][threadIdx.x];
        partial[(int64_t)blockIdx.x * R + threadIdx.x] = s;
    }
}

__global__ void k_benergy_sum(const double* __restrict__ partial, int nblocks, int R, double* __restrict__ u) {
    const int r = threadIdx.x;
    if (r >= R) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partial[(int64_t)b * R + r];
    u[r] = s;
}

// packed entry j of a row comes from stencil entry perm[node * plen + j] (the
// id order of launch_row_perm) when perm is given
__device__ __forceinline__ int bsrc_entry(const uint8_t* perm, int plen, int64_t node, int j) {
    return perm ? (int)perm[node * plen + j] : j;
}

__global__ void k_bpack_idx(const int32_t* __restrict__ src, int stride, int n_use, int64_t N, int chunks, int npw,
                            int64_t node0, const uint8_t* __restrict__ perm, int plen, int32_t* __restrict__ dst,
                            int64_t total) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int q = (int)(e & 3);
    const int64_t r = e >> 2;
    const int g = (int)(r % npw);
    const int64_t r2 = r / npw;
    const int c = (int)(r2 % chunks);
    const int64_t s = r2 / chunks;
    const int64_t node = s * npw + g;
    const int entry = c * 4 + q;
    int32_t v = (int32_t)node0;
    if (node < N) v = (int32_t)(node0 + src[node * stride + bsrc_entry(perm, plen, node, entry < n_use ? entry : 0)]);
    dst[e] = v;
}

__global__ void k_bpack_w(const double* __restrict__ w, int n_use, int64_t N, int chunks, int npw,
                          const uint8_t* __restrict__ perm, int plen, float* __restrict__ dst, int64_t total) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int q = (int)(e & 3);
    const int64_t r = e >> 2;
    const int g = (int)(r % npw);
    const int64_t r2 = r / npw;
    const int c = (int)(r2 % chunks);
    const int64_t s = r2 / chunks;
    const int64_t node = s * npw + g;
    const int entry = c * 4 + q;
    dst[e] = (node < N && entry < n_use) ? (float)w[node * n_use + bsrc_entry(perm, plen, node, entry)] : 0.0f;
}

__global__ void k_bscatter(const double* __restrict__ src, const int64_t* __restrict__ inv, int64_t n, int nrhs_src,
                           int rhs0, float* __restrict__ state, int64_t node0, int comp, int R) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * nrhs_src) return;
    const int64_t u = e / nrhs_src;
    const int r = (int)(e % nrhs_src);
    state[((node0 + inv[u]) * 3 + comp) * R + rhs0 + r] = (float)src[e];
}

__global__ void k_bgather(const float* __restrict__ state, const int64_t* __restrict__ inv, int64_t n, int nrhs_dst,
                          int rhs0, int64_t node0, int comp, int R, double* __restrict__ dst) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * nrhs_dst) return;
    const int64_t u = e / nrhs_dst;
    const int r = (int)(e % nrhs_dst);
    dst[e] = (double)state[((node0 + inv[u]) * 3 + comp) * R + rhs0 + r];
}

__global__ void k_bzero_held(const float* __restrict__ ce, float* __restrict__ state, int64_t node0, int64_t n, int R) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n || ce[node0 + k] != 0.0f) return;
    for (int r = 0; r < R; ++r) state[((node0 + k) * 3) * R + r] = 0.0f;
}

__global__ void k_bmaterials(const double* __restrict__ eps_user, const uint8_t* __restrict__ pec_user,
                             const int64_t* __restrict__ perm, int64_t n, int64_t node0, double dt_eps0,
                             float* __restrict__ ce, float* __restrict__ state, int R) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t u = perm[k];
    const double er = eps_user ? eps_user[u] : 1.0;
    const bool pec = pec_user && pec_user[u];
    ce[node0 + k] = pec ? 0.0f : (float)(dt_eps0 / er);
    if (pec)
        for (int r = 0; r < R; ++r) state[((node0 + k) * 3) * R + r] = 0.0f;
}

}  // namespace mfd

using namespace mfd;

struct BatchDomain {
    const mfd_nodes* nodes = nullptr;
    int64_t node0 = 0;
    int n = 0;
    double dt = 0, eps0 = 0, mu0 = 0;
    std::vector<int64_t> src_node;
    std::vector<int> src_rhs;
    std::vector<double> src_amp, src_f0, src_t0;
    std::vector<int64_t> prb_node;  // device-order local ids
    int prb_slot0 = 0;
    int64_t prb_cap = 0;
};

struct mfd_batch {
    mfd_ctx* ctx = nullptr;
    std::vector<const mfd_weights*> held;  // one reference on every domain's weights
    int R = 16;
    int ndom = 0;
    int64_t ntot = 0;
    std::vector<BatchDomain> dom;
    DevBuf d_dom, d_tile, idx, wx, wy, wv, A, B, ce, gam, counter, pstep0, bar;
    DevBuf src_start, src_node, src_rhs, src_amp, src_f0, src_t0;
    DevBuf prb_start, prb_node, prb_slot, prb_buf;
    int ntile = 0;
    std::vector<BTile> tiles;
    int prb_slots = 0;
    int64_t prb_cap = 0, prb_from = 0;
    int64_t steps = 0;
    int grid = 0;
    int tile_nodes = 64;
    int variant = 0;  // kernel variant (mfd_batch_set_variant, mfd_batch_autotune)
    DevBuf Hs;              // H* of the current state (variants 2, 3), allocated with the first such variant
    bool hs_valid = false;  // H* matches the state and gamma (the kernel keeps it so; host writes clear it)
    unsigned long long spin_limit = 1ull << 25;  // polls with 64 ns naps: a few seconds before giving up
    bool use_graph = true;
    cudaGraphExec_t graph = nullptr;
    int graph_steps = -1;
    bool tables_dirty = true;
    ~mfd_batch() {
        if (graph) cudaGraphExecDestroy(graph);
    }
};

namespace {

template <typename T> mfd_status upload_vec(mfd_ctx* ctx, DevBuf& b, const std::vector<T>& v) {
    MFD_TRY(b.alloc(std::max<size_t>(1, v.size()) * sizeof(T)));
    if (!v.empty()) MFD_CUDA(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
    return MFD_OK;
}

// sources and probes regrouped by tile
mfd_status build_tables(mfd_batch* b) {
    const int nt = b->ntile;
    std::vector<std::vector<int>> srcs(nt);
    std::vector<int64_t> sn;
    std::vector<int> sr;
    std::vector<double> sa, sf, st0;
    struct P {
        int64_t node;
        int slot;
    };
    std::vector<std::vector<P>> prbs(nt);
    // tile of a (domain, local node)
    const int TN = b->tile_nodes;
    std::vector<int> first_tile(b->ndom + 1, 0);
    for (int d = 0, t = 0; d < b->ndom; ++d) {
        first_tile[d] = t;
        t += (b->dom[d].n + TN - 1) / TN;
        first_tile[d + 1] = t;
    }
    std::vector<int> sstart(nt + 1, 0), pstart(nt + 1, 0);
    std::vector<int64_t> sn_t;
    std::vector<std::vector<int>> src_of_tile(nt);
    for (int d = 0; d < b->ndom; ++d) {
        const BatchDomain& D = b->dom[d];
        for (size_t s = 0; s < D.src_node.size(); ++s) {
            const int64_t loc = D.nodes->h_inv[D.src_node[s]];
            const int t = first_tile[d] + (int)(loc / TN);
            src_of_tile[t].push_back((int)sn.size());
            sn.push_back(D.node0 + loc);
            sr.push_back(D.src_rhs[s]);
            sa.push_back(D.src_amp[s]);
            sf.push_back(D.src_f0[s]);
            st0.push_back(D.src_t0[s]);
        }
        for (size_t p = 0; p < D.prb_node.size(); ++p) {
            const int64_t loc = D.prb_node[p];
            const int t = first_tile[d] + (int)(loc / TN);
            prbs[t].push_back({D.node0 + loc, D.prb_slot0 + (int)p});
        }
    }
    std::vector<int64_t> sn2, pn2;
    std::vector<int> sr2, ps2;
    std::vector<double> sa2, sf2, st2;
    for (int t = 0; t < nt; ++t) {
        sstart[t] = (int)sn2.size();
        for (int j : src_of_tile[t]) {
            sn2.push_back(sn[j]);
            sr2.push_back(sr[j]);
            sa2.push_back(sa[j]);
            sf2.push_back(sf[j]);
            st2.push_back(st0[j]);
        }
        pstart[t] = (int)pn2.size();
        for (auto& p : prbs[t]) {
            pn2.push_back(p.node);
            ps2.push_back(p.slot);
        }
    }
    sstart[nt] = (int)sn2.size();
    pstart[nt] = (int)pn2.size();
    mfd_ctx* ctx = b->ctx;
    MFD_TRY(upload_vec(ctx, b->src_start, sstart));
    MFD_TRY(upload_vec(ctx, b->src_node, sn2));
    MFD_TRY(upload_vec(ctx, b->src_rhs, sr2));
    MFD_TRY(upload_vec(ctx, b->src_amp, sa2));
    MFD_TRY(upload_vec(ctx, b->src_f0, sf2));
    MFD_TRY(upload_vec(ctx, b->src_t0, st2));
    MFD_TRY(upload_vec(ctx, b->prb_start, pstart));
    MFD_TRY(upload_vec(ctx, b->prb_node, pn2));
    MFD_TRY(upload_vec(ctx, b->prb_slot, ps2));
    MFD_CUDA(cudaStreamSynchronize(ctx->stream));
    b->tables_dirty = false;
    return MFD_OK;
}

BArgs make_args(mfd_batch* b, int nsteps) {
    BArgs a;
    a.dom = b->d_dom.as<const BDom>();
    a.tile = b->d_tile.as<const BTile>();
    a.ntile = b->ntile;
    a.idx = b->idx.as<const int4>();
    a.wx = b->wx.as<const float4>();
    a.wy = b->wy.as<const float4>();
    a.wv = b->wv.as<const float4>();
    a.A = b->A.as<float>();
    a.B = b->B.as<float>();
    a.Hs = b->Hs.p ? b->Hs.as<float>() : nullptr;
    a.ce = b->ce.as<const float>();
    a.gam = b->gam.as<const float>();
    a.src_start = b->src_start.as<const int>();
    a.src_node = b->src_node.as<const int64_t>();
    a.src_rhs = b->src_rhs.as<const int>();
    a.src_amp = b->src_amp.as<const double>();
    a.src_f0 = b->src_f0.as<const double>();
    a.src_t0 = b->src_t0.as<const double>();
    a.prb_start = b->prb_start.as<const int>();
    a.prb_node = b->prb_node.as<const int64_t>();
    a.prb_slot = b->prb_slot.as<const int>();
    a.prb_buf = b->prb_buf.as<float>();
    a.prb_slots = b->prb_slots;
    a.prb_cap = b->prb_cap;
    a.pstep0 = b->pstep0.as<const int64_t>();
    a.counter = b->counter.as<int64_t>();
    a.nsteps = nsteps;
    a.bar = b->bar.as<unsigned int>();
    a.spin_limit = b->spin_limit;
    a.ntot = b->ntot;
    return a;
}

template <int R> void* kernel_ptr(int variant) {
    switch (variant) {
        case 0: return (void*)k_batch<R, 0>;
        case 1: return (void*)k_batch<R, 1>;
        case 2: return (void*)k_batch<R, 2>;
        default: return (void*)k_batch<R, 3>;
    }
}

void* batch_kernel(int R, int variant) {
    switch (R) {
        case 4: return kernel_ptr<4>(variant);
        case 8: return kernel_ptr<8>(variant);
        case 16: return kernel_ptr<16>(variant);
        default: return kernel_ptr<32>(variant);
    }
}

// the persistent grid of a variant: every block that can be resident on every SM
mfd_status set_variant(mfd_batch* b, int variant) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel(b->R, variant), BT_THREADS, 0);
    if (e != cudaSuccess || per_sm < 1) return fail(MFD_ERR_CUDA, "occupancy query failed");
    if (variant >= 2 && !b->Hs.p) {
        MFD_TRY(b->Hs.alloc((size_t)b->ntot * 2 * b->R * 4));
        b->hs_valid = false;
    }
    b->variant = variant;
    b->grid = std::min(per_sm * b->ctx->sm_count, std::max(1, b->ntile));
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    b->graph_steps = -1;
    return MFD_OK;
}

// H* of the current state before a launch of variant 2 or 3, when the host has
// changed the state or gamma since the last launch (one block per tile)
cudaError_t ensure_hstar(mfd_batch* b) {
    if (b->variant < 2) {  // the launch advances the state without H*
        b->hs_valid = false;
        return cudaSuccess;
    }
    if (b->hs_valid) return cudaSuccess;
    BArgs a = make_args(b, 0);
    const unsigned g = (unsigned)std::max(1, b->ntile);
    cudaStream_t s = b->ctx->stream;
    switch (b->R) {
        case 4: k_bhstar<4><<<g, BT_THREADS, 0, s>>>(a); break;
        case 8: k_bhstar<8><<<g, BT_THREADS, 0, s>>>(a); break;
        case 16: k_bhstar<16><<<g, BT_THREADS, 0, s>>>(a); break;
        default: k_bhstar<32><<<g, BT_THREADS, 0, s>>>(a); break;
    }
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) b->hs_valid = true;
    return e;
}

cudaError_t launch_batch(mfd_batch* b, int nsteps) {
    BArgs a = make_args(b, nsteps);
    void* args[] = {&a};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)b->grid);
    cfg.blockDim = dim3(BT_THREADS);
    cfg.stream = b->ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, batch_kernel(b->R, b->variant), args);
}

}  // namespace

extern "C" {

mfd_status mfd_batch_create(mfd_ctx* ctx, int ndom, const mfd_sim_desc* descs, int nrhs, mfd_batch** out) {
    if (!ctx || !descs || !out || ndom < 1) return fail(MFD_ERR_ARG, "bad arguments");
    *out = nullptr;
    if (nrhs != 4 && nrhs != 8 && nrhs != 16 && nrhs != 32) return fail(MFD_ERR_ARG, "nrhs must be 4, 8, 16 or 32");
    MFD_CUDA(cudaSetDevice(ctx->device));
    mfd_batch* b = new (std::nothrow) mfd_batch();
    if (!b) return fail(MFD_ERR_OOM, "host allocation failed");
    auto bail = [&](mfd_status s) {
        delete b;
        return s;
    };
    b->ctx = ctx;
    b->R = nrhs;
    b->ndom = ndom;
    b->dom.resize(ndom);
    const int NPW = 32 / (nrhs / 4);
    b->tile_nodes = 8 * NPW;
    std::vector<BDom> hd(ndom);
    std::vector<float> gam_h;
    int64_t node0 = 0, idx0 = 0, wc0 = 0, wv0 = 0;
    for (int d = 0; d < ndom; ++d) {
        const mfd_sim_desc& s = descs[d];
        if (s.dim != 2 || s.precision != MFD_FP32) return bail(fail(MFD_ERR_ARG, "batched domains are 2D FP32"));
        if (!s.h_curl || !s.h_hv || s.h_curl != s.e_curl || s.h_hv != s.e_hv)
            return bail(fail(MFD_ERR_ARG, "batched domains are collocated (h_curl == e_curl, h_hv == e_hv)"));
        const mfd_weights* cw = s.h_curl;
        const mfd_weights* hw = s.h_hv;
        if (cw->st != hw->st) return bail(fail(MFD_ERR_ARG, "batched domains need curl and HV weights on one stencil set"));
        if (cw->op == MFD_OP_LAP_POW || hw->op != MFD_OP_LAP_POW) return bail(fail(MFD_ERR_ARG, "weight operators"));
        const mfd_nodes* nd = cw->st->centres;
        if (cw->st->sources != nd || nd->ctx != ctx) return bail(fail(MFD_ERR_ARG, "stencils must be own-set"));
        if (nd->mirror_axes) return bail(fail(MFD_ERR_ARG, "batched domains do not support mirror walls (images)"));
        if (cw->nsz.p || hw->nsz.p)
            return bail(fail(MFD_ERR_ARG, "batched domains take one stencil size per operator"));
        if (!(s.dt > 0) || !(s.eps0 > 0) || !(s.mu0 > 0)) return bail(fail(MFD_ERR_ARG, "dt, eps0, mu0 must be > 0"));
        BatchDomain& D = b->dom[d];
        D.nodes = nd;
        D.node0 = node0;
        D.n = (int)nd->n;
        D.dt = s.dt;
        D.eps0 = s.eps0;
        D.mu0 = s.mu0;
        for (int r = 0; r < nrhs; ++r) gam_h.push_back((float)s.gamma);
        BDom& h = hd[d];
        h.node0 = node0;
        h.n = D.n;
        h.nc = (cw->n_use + 3) / 4;
        h.nv = (hw->n_use + 3) / 4;
        h.ni = std::max(h.nc, h.nv);
        h.ch = (float)(s.dt / s.mu0);
        h.dt = s.dt;
        const int64_t slices = (D.n + NPW - 1) / NPW;
        h.idx0 = idx0;
        h.wc0 = wc0;
        h.wv0 = wv0;
        idx0 += slices * h.ni * NPW;
        wc0 += slices * h.nc * NPW;
        wv0 += slices * h.nv * NPW;
        node0 += D.n;
        for (int t = 0; t < D.n; t += b->tile_nodes) b->tiles.push_back({d, t});
    }
    b->ntot = node0;
    if (node0 > INT32_MAX) return bail(fail(MFD_ERR_ARG, "too many nodes in the batch"));
    b->ntile = (int)b->tiles.size();
    mfd_status st;
    const int R = nrhs;
    if ((st = b->idx.alloc(idx0 * 16)) || (st = b->wx.alloc(wc0 * 16)) || (st = b->wy.alloc(wc0 * 16)) ||
        (st = b->wv.alloc(wv0 * 16)) || (st = b->A.alloc(node0 * 3 * R * 4)) || (st = b->B.alloc(node0 * 3 * R * 4)) ||
        (st = b->ce.alloc(node0 * 4)) || (st = b->counter.alloc(8)) || (st = b->pstep0.alloc(8)) ||
        (st = b->bar.alloc(16)) || (st = upload_vec(ctx, b->d_dom, hd)) || (st = upload_vec(ctx, b->d_tile, b->tiles)) ||
        (st = upload_vec(ctx, b->gam, gam_h)))
        return bail(st);
    cudaStream_t s = ctx->stream;
    cudaMemsetAsync(b->A.p, 0, b->A.bytes, s);
    cudaMemsetAsync(b->B.p, 0, b->B.bytes, s);
    cudaMemsetAsync(b->counter.p, 0, 8, s);
    cudaMemsetAsync(b->pstep0.p, 0, 8, s);
    cudaMemsetAsync(b->bar.p, 0, 16, s);
    cudaError_t e0 = cudaSuccess;
    for (int d = 0; d < ndom; ++d) {
        const mfd_weights* cw = descs[d].h_curl;
        const mfd_weights* hw = descs[d].h_hv;
        const BDom& h = hd[d];
        const int64_t N = h.n;
        const int64_t slices = (N + NPW - 1) / NPW;
        // rows in ascending neighbour id within the shorter stencil and the rest (launch_row_perm)
        const int plen = std::max(cw->n_use, hw->n_use);
        DevBuf perm;
        if (plen <= 255) {
            if ((st = perm.alloc(N * plen))) return bail(st);
            const int m = std::min(cw->n_use, hw->n_use);
            e0 = launch_row_perm(cw->st->idx.as<int32_t>(), cw->st->n, N, m, m, plen, perm.as<uint8_t>(), s);
            if (e0 != cudaSuccess) return bail(fail(MFD_ERR_CUDA, cudaGetErrorString(e0)));
        }
        const uint8_t* pm = perm.p ? perm.as<uint8_t>() : nullptr;
        int64_t tot = slices * h.ni * NPW * 4;
        k_bpack_idx<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(cw->st->idx.as<int32_t>(), cw->st->n, plen, N, h.ni,
                                                                   NPW, h.node0, pm, plen,
                                                                   b->idx.as<int32_t>() + h.idx0 * 4, tot);
        tot = slices * h.nc * NPW * 4;
        k_bpack_w<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(cw->w.as<double>(), cw->n_use, N, h.nc, NPW, pm, plen,
                                                                 b->wx.as<float>() + h.wc0 * 4, tot);
        k_bpack_w<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(cw->w.as<double>() + N * cw->n_use, cw->n_use, N, h.nc,
                                                                 NPW, pm, plen, b->wy.as<float>() + h.wc0 * 4, tot);
        tot = slices * h.nv * NPW * 4;
        k_bpack_w<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(hw->w.as<double>(), hw->n_use, N, h.nv, NPW, pm, plen,
                                                                 b->wv.as<float>() + h.wv0 * 4, tot);
        if (pm) {  // perm is freed at the end of this iteration
            e0 = cudaStreamSynchronize(s);
            if (e0 != cudaSuccess) return bail(fail(MFD_ERR_CUDA, cudaGetErrorString(e0)));
        }
        k_bmaterials<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(nullptr, nullptr, b->dom[d].nodes->perm.as<int64_t>(), N,
                                                                 h.node0, descs[d].dt / descs[d].eps0, b->ce.as<float>(),
                                                                 b->A.as<float>(), R);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bail(fail(MFD_ERR_CUDA, cudaGetErrorString(e)));
    if ((st = set_variant(b, 0))) return bail(st);
    if ((st = b->prb_buf.alloc(16))) return bail(st);
    if ((st = build_tables(b))) return bail(st);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bail(fail(MFD_ERR_CUDA, cudaGetErrorString(e)));
    retain(ctx);
    for (int d = 0; d < ndom; ++d) {
        retain(descs[d].h_curl);
        retain(descs[d].h_hv);
        b->held.push_back(descs[d].h_curl);
        b->held.push_back(descs[d].h_hv);
    }
    *out = b;
    return MFD_OK;
}

mfd_status mfd_batch_set_materials(mfd_batch* b, int dom, const double* eps_r, const uint8_t* pec) {
    if (!b || dom < 0 || dom >= b->ndom) return fail(MFD_ERR_ARG, "bad arguments");
    MFD_CUDA(cudaSetDevice(b->ctx->device));
    const BatchDomain& D = b->dom[dom];
    DevBuf de, dp;
    if (eps_r) {
        for (int i = 0; i < D.n; ++i)
            if (!(eps_r[i] > 0)) return fail(MFD_ERR_ARG, "eps_r must be > 0");
        MFD_TRY(de.alloc(D.n * 8));
        MFD_CUDA(cudaMemcpyAsync(de.p, eps_r, D.n * 8, cudaMemcpyHostToDevice, b->ctx->stream));
    }
    if (pec) {
        MFD_TRY(dp.alloc(D.n));
        MFD_CUDA(cudaMemcpyAsync(dp.p, pec, D.n, cudaMemcpyHostToDevice, b->ctx->stream));
    }
    b->hs_valid = false;
    k_bmaterials<<<(unsigned)((D.n + 255) / 256), 256, 0, b->ctx->stream>>>(
        de.as<double>(), dp.as<uint8_t>(), D.nodes->perm.as<int64_t>(), D.n, D.node0, D.dt / D.eps0, b->ce.as<float>(),
        b->A.as<float>(), b->R);
    MFD_CUDA(cudaGetLastError());
    MFD_CUDA(cudaStreamSynchronize(b->ctx->stream));
    return MFD_OK;
}

static mfd_status batch_field_args(mfd_batch* b, int dom, int comp, int rhs, int* c, int* nr) {
    if (!b || dom < 0 || dom >= b->ndom) return fail(MFD_ERR_ARG, "bad arguments");
    if (comp != MFD_EZ && comp != MFD_HX && comp != MFD_HY) return fail(MFD_ERR_ARG, "TMz has Ez, Hx, Hy only");
    if (rhs < -1 || rhs >= b->R) return fail(MFD_ERR_ARG, "rhs out of range");
    *c = comp == MFD_EZ ? 0 : (comp == MFD_HX ? 1 : 2);
    *nr = rhs < 0 ? b->R : 1;
    return MFD_OK;
}

// caller-order FP64 values (device, n x nr) into the state
static mfd_status batch_scatter(mfd_batch* b, int dom, int comp, int rhs, const double* dsrc) {
    int c, nr;
    MFD_TRY(batch_field_args(b, dom, comp, rhs, &c, &nr));
    b->hs_valid = false;
    const BatchDomain& D = b->dom[dom];
    const int64_t tot = (int64_t)D.n * nr;
    k_bscatter<<<(unsigned)((tot + 255) / 256), 256, 0, b->ctx->stream>>>(
        dsrc, D.nodes->inv.as<int64_t>(), D.n, nr, rhs < 0 ? 0 : rhs, b->A.as<float>(), D.node0, c, b->R);
    MFD_CUDA(cudaGetLastError());
    if (comp == MFD_EZ) {  // PEC nodes (ce == 0) stay at zero
        k_bzero_held<<<(unsigned)((D.n + 255) / 256), 256, 0, b->ctx->stream>>>(b->ce.as<float>(), b->A.as<float>(),
                                                                                D.node0, D.n, b->R);
        MFD_CUDA(cudaGetLastError());
    }
    return MFD_OK;
}

static mfd_status batch_gather(mfd_batch* b, int dom, int comp, int rhs, double* ddst) {
    int c, nr;
    MFD_TRY(batch_field_args(b, dom, comp, rhs, &c, &nr));
    const BatchDomain& D = b->dom[dom];
    const int64_t tot = (int64_t)D.n * nr;
    k_bgather<<<(unsigned)((tot + 255) / 256), 256, 0, b->ctx->stream>>>(
        b->A.as<float>(), D.nodes->inv.as<int64_t>(), D.n, nr, rhs < 0 ? 0 : rhs, D.node0, c, b->R, ddst);
    MFD_CUDA(cudaGetLastError());
    return MFD_OK;
}

mfd_status mfd_batch_set_field(mfd_batch* b, int dom, int comp, int rhs, const double* host) {
    int c, nr;
    if (!host) return fail(MFD_ERR_ARG, "bad arguments");
    MFD_TRY(batch_field_args(b, dom, comp, rhs, &c, &nr));
    MFD_CUDA(cudaSetDevice(b->ctx->device));
    const size_t bytes = (size_t)b->dom[dom].n * nr * 8;
    DevBuf tmp;
    MFD_TRY(tmp.alloc(bytes));
    MFD_CUDA(cudaMemcpyAsync(tmp.p, host, bytes, cudaMemcpyHostToDevice, b->ctx->stream));
    MFD_TRY(batch_scatter(b, dom, comp, rhs, tmp.as<double>()));
    MFD_CUDA(cudaStreamSynchronize(b->ctx->stream));
    return MFD_OK;
}

mfd_status mfd_batch_get_field(mfd_batch* b, int dom, int comp, int rhs, double* host) {
    int c, nr;
    if (!host) return fail(MFD_ERR_ARG, "bad arguments");
    MFD_TRY(batch_field_args(b, dom, comp, rhs, &c, &nr));
    MFD_CUDA(cudaSetDevice(b->ctx->device));
    const size_t bytes = (size_t)b->dom[dom].n * nr * 8;
    DevBuf tmp;
    MFD_TRY(tmp.alloc(bytes));
    MFD_TRY(batch_gather(b, dom, comp, rhs, tmp.as<double>()));
    MFD_CUDA(cudaMemcpyAsync(host, tmp.p, bytes, cudaMemcpyDeviceToHost, b->ctx->stream));
    MFD_CUDA(cudaStreamSynchronize(b->ctx->stream));
    return MFD_OK;
}

mfd_status mfd_batch_set_field_device(mfd_batch* b, int dom, int comp, int rhs, const double* dev, void* stream) {
    int c, nr;
    if (!dev) return fail(MFD_ERR_ARG, "bad arguments");
    MFD_TRY(batch_field_args(b, dom, comp, rhs, &c, &nr));
    MFD_CUDA(cudaSetDevice(b->ctx->device));
    MFD_TRY(order_streams((cudaStream_t)stream, b->ctx->stream));
    MFD_TRY(batch_scatter(b, dom, comp, rhs, dev));
    return order_streams(b->ctx->stream, (cudaStream_t)stream);
}

mfd_status mfd_batch_get_field_device(mfd_batch* b, int dom, int comp, int rhs, double* dev, void* stream) {
    int c, nr;
    if (!dev) return fail(MFD_ERR_ARG, "bad arguments");
    MFD_TRY(batch_field_args(b, dom, comp, rhs, &c, &nr));
    MFD_CUDA(cudaSetDevice(b->ctx->device));
    MFD_TRY(order_streams((cudaStream_t)stream, b->ctx->stream));
    MFD_TRY(batch_gather(b, dom, comp, rhs, dev));
    return order_streams(b->ctx->stream, (cudaStream_t)stream);
}

mfd_status mfd_batch_set_sources(mfd_batch* b, int dom, int count, const int64_t* node, const int32_t* rhs,
                                 const double* amp, const double* f0, const double* t0) {
    if (!b || dom < 0 || dom >= b->ndom || count < 0) return fail(MFD_ERR_ARG, "bad arguments");
    if (count > 0 && (!node || !rhs || !amp || !f0 || !t0)) return fail(MFD_ERR_ARG, "NULL source arrays");
    BatchDomain& D = b->dom[dom];
    for (int s = 0; s < count; ++s) {
        if (node[s] < 0 || node[s] >= D.n) return fail(MFD_ERR_ARG, "source node out of range");
        if (rhs[s] < 0 || rhs[s] >= b->R) return fail(MFD_ERR_ARG, "source rhs out of range");
        if (!(f0[s] > 0)) return fail(MFD_ERR_ARG, "source frequency must be > 0");
    }
    D.src_node.assign(node, node + count);
    D.src_rhs.assign(rhs, rhs + count);
    D.src_amp.assign(amp, amp + count);
    D.src_f0.assign(f0, f0 + count);
    D.src_t0.assign(t0, t0 + count);
    b->tables_dirty = true;
    return MFD_OK;
}

mfd_status mfd_batch_set_probes(mfd_batch* b, int dom, int count, const int64_t* node, int64_t capacity) {
    if (!b || dom < 0 || dom >= b->ndom || count < 0 || capacity < 0) return fail(MFD_ERR_ARG, "bad arguments");
    if (count > 0 && !node) return fail(MFD_ERR_ARG, "NULL probe array");
    BatchDomain& D = b->dom[dom];
    D.prb_node.resize(count);
    for (int p = 0; p < count; ++p) {
        if (node[p] < 0 || node[p] >= D.n) return fail(MFD_ERR_ARG, "probe node out of range");
        D.prb_node[p] = D.nodes->h_inv[node[p]];
    }
    D.prb_cap = capacity;
    // slots are renumbered over all domains; one capacity for the batch (the largest asked)
    int slots = 0;
    int64_t cap = 0;
    for (auto& X : b->dom) {
        X.prb_slot0 = slots;
        slots += (int)X.prb_node.size();
        cap = std::max(cap, X.prb_cap);
    }
    MFD_CUDA(cudaSetDevice(b->ctx->device));
    // the tables are rebuilt before the next launch; until the buffer is in
    // place no probe is recorded
    b->tables_dirty = true;
    b->prb_cap = 0;
    b->prb_slots = 0;
    MFD_TRY(b->prb_buf.alloc(std::max<int64_t>(1, cap * slots) * b->R * 4));
    b->prb_slots = slots;
    b->prb_cap = cap;
    b->prb_from = b->steps;
    MFD_CUDA(cudaMemcpyAsync(b->pstep0.p, &b->prb_from, 8, cudaMemcpyHostToDevice, b->ctx->stream));
    MFD_CUDA(cudaStreamSynchronize(b->ctx->stream));
    b->tables_dirty = true;
    return MFD_OK;
}

mfd_status mfd_batch_step(mfd_batch* b, int64_t nsteps) {
    if (!b || nsteps < 0 || nsteps > INT32_MAX) return fail(MFD_ERR_ARG, "bad arguments");
    if (nsteps == 0) return MFD_OK;
    MFD_CUDA(cudaSetDevice(b->ctx->device));
    if (b->tables_dirty) {
        // the graph points at the tables' arrays: drop it before they are replaced
        if (b->graph) {
            cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
        }
        b->graph_steps = -1;
        MFD_TRY(build_tables(b));
    }
    cudaStream_t s = b->ctx->stream;
    if (b->use_graph && b->graph_steps != (int)nsteps) {
        if (b->graph) {
            cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
        }
        b->graph_steps = -1;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t el = launch_batch(b, (int)nsteps);
            e = cudaStreamEndCapture(s, &g);
            if (el != cudaSuccess) e = el;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e == cudaSuccess) {
            b->graph_steps = (int)nsteps;
        } else {  // capture of the cooperative launch refused: launch it directly from now on
            cudaGetLastError();
            if (b->graph) cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
            b->use_graph = false;
        }
    }
    MFD_CUDA(ensure_hstar(b));
    if (b->use_graph) MFD_CUDA(cudaGraphLaunch(b->graph, s));
    else MFD_CUDA(launch_batch(b, (int)nsteps));
    unsigned int flags[3];
    MFD_CUDA(cudaMemcpyAsync(flags, b->bar.p, sizeof(flags), cudaMemcpyDeviceToHost, s));
    MFD_CUDA(cudaStreamSynchronize(s));
    if (flags[2] != 0u) {
        // every block has left the kernel; the barrier words are cleared for the
        // next launch, the step counters stay where they were and the fields are
        // left part way through the call (the caller sets them again)
        MFD_CUDA(cudaMemsetAsync(b->bar.p, 0, 16, s));
        MFD_CUDA(cudaStreamSynchronize(s));
        b->hs_valid = false;
        return fail(MFD_ERR_TIMEOUT, "a grid barrier of the batched kernel timed out");
    }
    b->steps += nsteps;
    if (const unsigned long long hits = bounds_take_local(s))
        return fail(MFD_ERR_STATE, std::to_string(hits) + " stencil indices out of range (bounds-checked build)");
    return MFD_OK;
}

// checkpoint / resume: buffer A holds every field at step boundaries (B is
// rewritten by the H half step before it is read), then the probe records
static void batch_state_layout(const mfd_batch* b, StateHead* h) {
    state_head_init(h, 2);
    h->ne = b->ntot;
    h->nrhs = b->R;
    h->steps = b->steps;
    h->probe_from = b->prb_from;
    h->nprobe = b->prb_slots;
    int64_t rec = std::min(b->steps - b->prb_from, b->prb_cap);
    h->rec = b->prb_slots > 0 && rec > 0 ? rec : 0;
    h->bytes[0] = (int64_t)b->A.bytes;
}

static size_t batch_state_total(const StateHead& h) {
    return sizeof(StateHead) + (size_t)h.bytes[0] + (size_t)h.rec * h.nprobe * h.nrhs * 4;
}

mfd_status mfd_batch_state_size(const mfd_batch* b, size_t* bytes) {
    if (!b || !bytes) return fail(MFD_ERR_ARG, "NULL argument");
    StateHead h;
    batch_state_layout(b, &h);
    *bytes = batch_state_total(h);
    return MFD_OK;
}

mfd_status mfd_batch_save_state(mfd_batch* b, void* host, size_t bytes) {
    if (!b || !host) return fail(MFD_ERR_ARG, "NULL argument");
    StateHead h;
    batch_state_layout(b, &h);
    if (bytes < batch_state_total(h)) return fail(MFD_ERR_ARG, "state buffer smaller than mfd_batch_state_size");
    MFD_CUDA(cudaSetDevice(b->ctx->device));
    cudaStream_t s = b->ctx->stream;
    char* o = static_cast<char*>(host);
    std::memcpy(o, &h, sizeof(h));
    o += sizeof(h);
    MFD_CUDA(cudaMemcpyAsync(o, b->A.p, (size_t)h.bytes[0], cudaMemcpyDeviceToHost, s));
    o += h.bytes[0];
    if (h.rec) MFD_CUDA(cudaMemcpyAsync(o, b->prb_buf.p, (size_t)h.rec * h.nprobe * h.nrhs * 4, cudaMemcpyDeviceToHost, s));
    MFD_CUDA(cudaStreamSynchronize(s));
    return MFD_OK;
}

mfd_status mfd_batch_load_state(mfd_batch* b, const void* host, size_t bytes) {
    if (!b || !host) return fail(MFD_ERR_ARG, "NULL argument");
    StateHead in, mine;
    MFD_TRY(state_head_check(host, bytes, 2, &in));
    batch_state_layout(b, &mine);
    if (in.ne != mine.ne || in.nrhs != mine.nrhs || in.bytes[0] != mine.bytes[0])
        return fail(MFD_ERR_ARG, "state blob of another batch (node count or right-hand sides differ)");
    if (in.rec > 0 && (in.nprobe != b->prb_slots || in.rec > b->prb_cap))
        return fail(MFD_ERR_ARG, "state blob probe records need the same probes with enough capacity");
    if (bytes < batch_state_total(in)) return fail(MFD_ERR_ARG, "state blob truncated");
    MFD_CUDA(cudaSetDevice(b->ctx->device));
    cudaStream_t s = b->ctx->stream;
    const char* o = static_cast<const char*>(host) + sizeof(in);
    MFD_CUDA(cudaMemcpyAsync(b->A.p, o, (size_t)in.bytes[0], cudaMemcpyHostToDevice, s));
    b->hs_valid = false;
    o += in.bytes[0];
    if (in.rec) MFD_CUDA(cudaMemcpyAsync(b->prb_buf.p, o, (size_t)in.rec * in.nprobe * in.nrhs * 4, cudaMemcpyHostToDevice, s));
    b->steps = in.steps;
    b->prb_from = in.rec > 0 ? in.probe_from : in.steps;
    const int64_t words[2] = {b->steps, b->prb_from};
    MFD_CUDA(cudaMemcpyAsync(b->counter.p, &words[0], 8, cudaMemcpyHostToDevice, s));
    MFD_CUDA(cudaMemcpyAsync(b->pstep0.p, &words[1], 8, cudaMemcpyHostToDevice, s));
    MFD_CUDA(cudaStreamSynchronize(s));
    return MFD_OK;
}

mfd_status mfd_batch_set_variant(mfd_batch* b, int variant) {
    if (!b || variant < 0 || variant > 3) return fail(MFD_ERR_ARG, "variant must be 0, 1, 2 or 3");
    MFD_CUDA(cudaSetDevice(b->ctx->device));
    MFD_TRY(set_variant(b, variant));
    MFD_CUDA(cudaStreamSynchronize(b->ctx->stream));
    return MFD_OK;
}

int mfd_batch_variant(const mfd_batch* b) { return b ? b->variant : -1; }

mfd_status mfd_batch_autotune(mfd_batch* b, int reps, int* chosen, double* ms) {
    if (!b || reps < 1) return fail(MFD_ERR_ARG, "bad arguments");
    MFD_CUDA(cudaSetDevice(b->ctx->device));
    cudaStream_t s = b->ctx->stream;
    // every trial starts from the same state and leaves nothing behind: the fields,
    // the probe records and the step counters are put back after each
    DevBuf saveA, saveP;
    MFD_TRY(saveA.alloc(b->A.bytes));
    MFD_TRY(saveP.alloc(b->prb_buf.bytes));
    MFD_CUDA(cudaMemcpyAsync(saveA.p, b->A.p, b->A.bytes, cudaMemcpyDeviceToDevice, s));
    MFD_CUDA(cudaMemcpyAsync(saveP.p, b->prb_buf.p, b->prb_buf.bytes, cudaMemcpyDeviceToDevice, s));
    const int64_t steps0 = b->steps;
    auto restore = [&]() -> mfd_status {
        MFD_CUDA(cudaMemcpyAsync(b->A.p, saveA.p, b->A.bytes, cudaMemcpyDeviceToDevice, s));
        MFD_CUDA(cudaMemcpyAsync(b->prb_buf.p, saveP.p, b->prb_buf.bytes, cudaMemcpyDeviceToDevice, s));
        MFD_CUDA(cudaMemcpyAsync(b->counter.p, &steps0, 8, cudaMemcpyHostToDevice, s));
        MFD_CUDA(cudaStreamSynchronize(s));
        b->hs_valid = false;
        b->steps = steps0;
        return MFD_OK;
    };
    cudaEvent_t e0, e1;
    MFD_CUDA(cudaEventCreate(&e0));
    MFD_CUDA(cudaEventCreate(&e1));
    struct EvGuard {
        cudaEvent_t a, b;
        ~EvGuard() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } eg{e0, e1};
    const int start_variant = b->variant;
    int best = start_variant;
    float tbest = 1e30f;
    for (int v = 0; v < 4; ++v) {
        MFD_TRY(set_variant(b, v));
        if (b->tables_dirty) MFD_TRY(build_tables(b));
        MFD_CUDA(ensure_hstar(b));
        MFD_CUDA(launch_batch(b, 1));  // first launch of this kernel: loads it
        MFD_CUDA(cudaEventRecord(e0, s));
        MFD_CUDA(launch_batch(b, reps));
        MFD_CUDA(cudaEventRecord(e1, s));
        MFD_CUDA(cudaEventSynchronize(e1));
        float t = 0;
        MFD_CUDA(cudaEventElapsedTime(&t, e0, e1));
        unsigned int flags[3];
        MFD_CUDA(cudaMemcpy(flags, b->bar.p, sizeof(flags), cudaMemcpyDeviceToHost));
        MFD_TRY(restore());
        if (flags[2] != 0u) {
            MFD_CUDA(cudaMemsetAsync(b->bar.p, 0, 16, s));
            MFD_TRY(set_variant(b, start_variant));
            MFD_CUDA(cudaStreamSynchronize(s));
            return fail(MFD_ERR_TIMEOUT, "a grid barrier of the batched kernel timed out during autotuning");
        }
        if (ms) ms[v] = (double)t / reps;
        if (t < tbest) {
            tbest = t;
            best = v;
        }
    }
    MFD_TRY(set_variant(b, best));
    MFD_CUDA(cudaStreamSynchronize(s));
    if (chosen) *chosen = best;
    return MFD_OK;
}

mfd_status mfd_batch_set_spin_limit(mfd_batch* b, uint64_t limit) {
    if (!b) return fail(MFD_ERR_ARG, "bad arguments");
    b->spin_limit = limit;
    if (b->graph) {  // the limit is a kernel argument baked into the captured graph
        MFD_CUDA(cudaSetDevice(b->ctx->device));
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    b->graph_steps = -1;
    return MFD_OK;
}

mfd_status mfd_batch_read_probes(mfd_batch* b, int dom, double* host, int64_t* steps) {
    if (!b || dom < 0 || dom >= b->ndom) return fail(MFD_ERR_ARG, "bad arguments");
    const BatchDomain& D = b->dom[dom];
    int64_t rec = std::min(b->steps - b->prb_from, b->prb_cap);
    if (rec < 0) rec = 0;
    if (steps) *steps = rec;
    const int np = (int)D.prb_node.size();
    if (!host || rec == 0 || np == 0) return MFD_OK;
    MFD_CUDA(cudaSetDevice(b->ctx->device));
    std::vector<float> tmp((size_t)rec * b->prb_slots * b->R);
    MFD_CUDA(cudaMemcpyAsync(tmp.data(), b->prb_buf.p, tmp.size() * 4, cudaMemcpyDeviceToHost, b->ctx->stream));
    MFD_CUDA(cudaStreamSynchronize(b->ctx->stream));
    for (int64_t k = 0; k < rec; ++k)
        for (int p = 0; p < np; ++p)
            for (int r = 0; r < b->R; ++r)
                host[(k * np + p) * b->R + r] = tmp[(k * b->prb_slots + D.prb_slot0 + p) * b->R + r];
    return MFD_OK;
}

mfd_status mfd_batch_set_gamma(mfd_batch* b, int dom, const double* gamma) {
    if (!b || !gamma || dom < 0 || dom >= b->ndom) return fail(MFD_ERR_ARG, "bad arguments");
    std::vector<float> g(b->R);
    for (int r = 0; r < b->R; ++r) {
        if (!std::isfinite(gamma[r])) return fail(MFD_ERR_ARG, "gamma must be finite");
        g[r] = (float)gamma[r];
    }
    b->hs_valid = false;  // H* carries gamma
    MFD_CUDA(cudaSetDevice(b->ctx->device));
    MFD_CUDA(cudaMemcpyAsync(b->gam.as<float>() + (size_t)dom * b->R, g.data(), b->R * 4, cudaMemcpyHostToDevice,
                             b->ctx->stream));
    MFD_CUDA(cudaStreamSynchronize(b->ctx->stream));
    return MFD_OK;
}

mfd_status mfd_batch_energy(mfd_batch* b, int dom, double* u) {
    if (!b || !u || dom < 0 || dom >= b->ndom) return fail(MFD_ERR_ARG, "bad arguments");
    MFD_CUDA(cudaSetDevice(b->ctx->device));
    int tile0 = 0;
    for (int d = 0; d < dom; ++d) tile0 += (b->dom[d].n + b->tile_nodes - 1) / b->tile_nodes;
    const BatchDomain& D = b->dom[dom];
    const int nt = (D.n + b->tile_nodes - 1) / b->tile_nodes;
    const int R = b->R;
    DevBuf part, du;
    MFD_TRY(part.alloc((size_t)nt * R * 8));
    MFD_TRY(du.alloc((size_t)R * 8));
    BArgs a = make_args(b, 0);
    cudaStream_t s = b->ctx->stream;
    const double eta2 = D.mu0 / D.eps0, dt_eps0 = D.dt / D.eps0;
    switch (R) {
        case 4: k_benergy<4><<<nt, BT_THREADS, 0, s>>>(a, dom, tile0, eta2, dt_eps0, part.as<double>()); break;
        case 8: k_benergy<8><<<nt, BT_THREADS, 0, s>>>(a, dom, tile0, eta2, dt_eps0, part.as<double>()); break;
        case 16: k_benergy<16><<<nt, BT_THREADS, 0, s>>>(a, dom, tile0, eta2, dt_eps0, part.as<double>()); break;
        default: k_benergy<32><<<nt, BT_THREADS, 0, s>>>(a, dom, tile0, eta2, dt_eps0, part.as<double>()); break;
    }
    MFD_CUDA(cudaGetLastError());
    k_benergy_sum<<<1, 32, 0, s>>>(part.as<double>(), nt, R, du.as<double>());
    MFD_CUDA(cudaGetLastError());
    MFD_CUDA(cudaMemcpyAsync(u, du.p, R * 8, cudaMemcpyDeviceToHost, s));
    MFD_CUDA(cudaStreamSynchronize(s));
    return MFD_OK;
}

int64_t mfd_batch_nodes(const mfd_batch* b) { return b ? b->ntot : -1; }

int mfd_batch_uses_graph(const mfd_batch* b) { return b && b->use_graph ? 1 : 0; }

void mfd_batch_destroy(mfd_batch* b) {
    if (!b) return;
    mfd_ctx* ctx = b->ctx;
    std::vector<const mfd_weights*> held = b->held;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    delete b;
    for (const mfd_weights* w : held) release(w);
    release(ctx);
}

}  // extern "C"
