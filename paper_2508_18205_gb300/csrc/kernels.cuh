// kernels.cuh -- the fused leapfrog half-step kernels (Eq. 19 and its 3D form).
//
// Layout in HBM (device, Morton order of each node set):
//  * stencil index and weight streams are "sliced": nodes are grouped in
//    slices of 32 (one warp); within a slice, chunk c of 4 consecutive
//    stencil entries of node 32 s + l sits at ((s * C + c) * 32 + l) * 4.
//    A warp's 128-bit loads of one chunk cover 512 contiguous bytes, and a
//    thread owns one node (one node per thread, no reductions). Rows are
//    padded to a multiple of 4 entries with weight 0 and a valid index.
//  * fields are array-of-structures: 2D collocated {Ez, Hx, Hy, ce} per node
//    (one 16-byte gather brings all three fields of a neighbour); staggered
//    {Hx, Hy} on the H set and Ez + ce on the E set; 3D one block per node
//    {Ex, Ey, Ez, ce, Hx, Hy, Hz, 0} (32 bytes in FP32, one gather), with the
//    H half step writing E* and H' to separate {., ., ., ce} / {., ., ., 0}
//    arrays from which the E half step reassembles the block.
//    ce = dt / (eps0 eps_r) of the node, 0 at a PEC node in 2D.
//  * weight and index streams are read with L1::no_allocate so that L1 keeps
//    the gathered fields of the Morton neighbourhood, and with an L2 policy:
//    a fraction `keep` of their lines is marked evict_last, the rest
//    evict_first. The streams are read once per half step, so they should
//    neither push the gathered fields out of L2 nor, when a problem's streams
//    are about the size of L2, evict one another before the next step: the
//    kept fraction then stays in L2 from one step to the next (the host sizes
//    keep from the L2 capacity and the streams' bytes; 0 for large problems).
//  * the staggered step kernels read their indices in a 16-bit form (Q16):
//    per slice and stream two bases {b0, b1 - 32768}; entry u < 32768 is node
//    b0 + u, entry u >= 32768 is node b1 + (u - 32768), so one slice may draw
//    its neighbours from two index windows of 32768 nodes (a Morton seam or a
//    periodic wrap). Chunks hold 8 entries (16 bytes) per lane, laid out like
//    the 32-bit chunks. A slice whose neighbours do not fit two windows has
//    b0 < 0 and its kernels read the 32-bit stream instead (the choice is per
//    warp, so the branch does not diverge).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mfd {

struct __align__(32) dbl4 {
    double x, y, z, w;
};

template <typename T> struct Vec;
template <> struct Vec<float> {
    using V2 = float2;
    using V4 = float4;
};
template <> struct Vec<double> {
    using V2 = double2;
    using V4 = dbl4;
};

// ---- streamed (read once) loads: bypass L1 allocation, L2 policy `pol`
// (stream_policy); the overloads without a policy mark every line evict_first
__device__ __forceinline__ uint64_t stream_policy(float keep) {
    uint64_t p;
    if (keep > 0.0f)
        asm("createpolicy.fractional.L2::evict_last.L2::evict_first.b64 %0, %1;" : "=l"(p) : "f"(fminf(keep, 1.0f)));
    else
        asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ int4 ld_stream(const int4* p, uint64_t pol) {
    int4 v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0,%1,%2,%3}, [%4], %5;"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ uint4 ld_stream(const uint4* p, uint64_t pol) {
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ int2 ld_stream(const int2* p, uint64_t pol) {
    int2 v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.s32 {%0,%1}, [%2], %3;" : "=r"(v.x), "=r"(v.y) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float4 ld_stream(const float4* p, uint64_t pol) {
    float4 v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ dbl4 ld_stream(const dbl4* p, uint64_t pol) {
    dbl4 v;
    const double2* q = reinterpret_cast<const double2*>(p);
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(q), "l"(pol));
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;"
        : "=d"(v.z), "=d"(v.w)
        : "l"(q + 1), "l"(pol));
    return v;
}
template <typename P> __device__ __forceinline__ auto ld_stream(const P* p) { return ld_stream(p, stream_policy(0.0f)); }
// KEEP = false: every line evict_first, the policy made at the load (pol unused); this
// form measured 1-2 % faster in the staggered kernels than one policy register
// carried through the loop. KEEP = true: the policy register `pol`.
template <bool KEEP, typename P> __device__ __forceinline__ auto ld_stream_k(const P* p, uint64_t pol) {
    if constexpr (KEEP) return ld_stream(p, pol);
    else return ld_stream(p);
}

// ---- gathered (reused by neighbours) loads: through L1
__device__ __forceinline__ float4 ld_gather(const float4* p) { return __ldg(p); }
__device__ __forceinline__ dbl4 ld_gather(const dbl4* p) {
    const double2* q = reinterpret_cast<const double2*>(p);
    double2 a = __ldg(q), b = __ldg(q + 1);
    return dbl4{a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ float2 ld_gather(const float2* p) { return __ldg(p); }
__device__ __forceinline__ double2 ld_gather(const double2* p) { return __ldg(p); }
__device__ __forceinline__ float ld_gather(const float* p) { return __ldg(p); }
__device__ __forceinline__ double ld_gather(const double* p) { return __ldg(p); }

// One node of the interleaved 3D state: its E block {Ex, Ey, Ez, ce} followed
// by its H block {Hx, Hy, Hz, 0} (p points at the E block, 32-byte aligned in
// FP32). Both blocks come in one 256-bit load (FP32) or two (FP64), so a
// stencil entry touches one cache line instead of one line per block.
__device__ __forceinline__ void ld_gather_eh(const float4* p, float4& e, float4& h) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(e.x), "=f"(e.y), "=f"(e.z), "=f"(e.w), "=f"(h.x), "=f"(h.y), "=f"(h.z), "=f"(h.w)
        : "l"(p));
}
__device__ __forceinline__ void ld_gather_eh(const dbl4* p, dbl4& e, dbl4& h) {
    asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];"
        : "=d"(e.x), "=d"(e.y), "=d"(e.z), "=d"(e.w)
        : "l"(p));
    asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];"
        : "=d"(h.x), "=d"(h.y), "=d"(h.z), "=d"(h.w)
        : "l"(p + 1));
}

// writes one node's E and H blocks of the interleaved 3D state (one 256-bit
// store in FP32, two in FP64)
__device__ __forceinline__ void st_eh(float4* p, float4 e, float4 h) {
    asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(e.x), "f"(e.y), "f"(e.z),
                 "f"(e.w), "f"(h.x), "f"(h.y), "f"(h.z), "f"(h.w)
                 : "memory");
}
__device__ __forceinline__ void st_eh(dbl4* p, dbl4 e, dbl4 h) {
    asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(p), "d"(e.x), "d"(e.y), "d"(e.z), "d"(e.w)
                 : "memory");
    asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(p + 1), "d"(h.x), "d"(h.y), "d"(h.z), "d"(h.w)
                 : "memory");
}

__device__ __forceinline__ void st4(float4* p, float4 v) { *p = v; }
__device__ __forceinline__ void st4(dbl4* p, dbl4 v) {
    double2* q = reinterpret_cast<double2*>(p);
    q[0] = make_double2(v.x, v.y);
    q[1] = make_double2(v.z, v.w);
}

// ---- stencil-sum accumulators
// The "compensated" option compensates the curl sums, which carry the O(1)
// update of the fields; the hyperviscosity sums are multiplied by gamma
// (1e-5 .. 1e-2) and stay plain FMA sums.
// Plain: fused multiply-add in the working precision.
template <typename T> struct AccPlain {
    T s = T(0);
    __device__ __forceinline__ void add(T w, T f) { s = fma(w, f, s); }
    __device__ __forceinline__ T get() const { return s; }
    // adds the partial sum of the lane `off` lanes away (all lanes of the warp call it)
    __device__ __forceinline__ void merge_xor(int off) { s += __shfl_xor_sync(0xffffffffu, s, off); }
};
// Compensated FP32 dot product (Ogita, Rump, Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 2005, Dot2): the exact product error comes
// from one FMA, the addition error from Knuth's two-sum; both are carried in c.
struct AccComp {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float w, float f) {
        float p = __fmul_rn(w, f);
        float e = __fmaf_rn(w, f, -p);
        float t = __fadd_rn(s, p);
        float z = __fsub_rn(t, s);
        float r = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
        s = t;
        c = __fadd_rn(c, __fadd_rn(r, e));
    }
    __device__ __forceinline__ float get() const { return __fadd_rn(s, c); }
    // adds the compensated partial sum of the lane `off` lanes away: the two
    // leading parts by Knuth's two-sum, the error terms added to c
    __device__ __forceinline__ void merge_xor(int off) {
        const float s2 = __shfl_xor_sync(0xffffffffu, s, off), c2 = __shfl_xor_sync(0xffffffffu, c, off);
        const float t = __fadd_rn(s, s2);
        const float z = __fsub_rn(t, s);
        const float r = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(s2, z));
        s = t;
        c = __fadd_rn(c, __fadd_rn(r, c2));
    }
};
template <typename T, bool COMP> struct AccSel { using type = AccPlain<T>; };
template <> struct AccSel<float, true> { using type = AccComp; };

// ---- kernel arguments
template <typename T> struct StencilStreams {
    const int4* idx_c = nullptr;  // curl index chunks (or the shared index)
    const int4* idx_v = nullptr;  // HV index chunks (== idx_c when shared)
    const uint4* q_c = nullptr;   // Q16 curl index chunks (8 entries), or null
    const uint4* q_v = nullptr;   // Q16 HV index chunks
    const int2* qb_c = nullptr;   // Q16 bases of the curl stream, one pair per slice
    const int2* qb_v = nullptr;   // Q16 bases of the HV stream
    const typename Vec<T>::V4* wx = nullptr;
    const typename Vec<T>::V4* wy = nullptr;
    const typename Vec<T>::V4* wz = nullptr;
    const typename Vec<T>::V4* wv = nullptr;
    int nc = 0, nv = 0, ni = 0;  // chunks per row: curl weights, HV weights, index (shared: max)
    int64_t n = 0;               // nodes
    int64_t src_c = 0, src_v = 0;  // sizes of the node sets the curl and HV indices point into
    bool mirror = false;           // entries carry image codes (PEC walls by images)
    const uint8_t* cext = nullptr;  // curl chunks each 32-node slice reads (per-centre sizes), or null: nc
    int nc0 = 0;                    // with cext: the fewest curl chunks of any slice
    float l2_keep = 0.0f;           // fraction of the stream lines kept in L2 (stream_policy)
};

// ---- bounds-checked build (compiled with -DMFD_BOUNDS_CHECK): every stencil
// index is tested against the size of the node set it points into before a
// kernel gathers through it. An index outside that set is counted in this
// translation unit's device word and replaced by 0, so nothing is read out of
// bounds and nothing traps; the public call that launched the kernel returns
// MFD_ERR_STATE (bounds_take_* on the host). Without the flag the checks
// compile to nothing.
#ifdef MFD_BOUNDS_CHECK
static __device__ unsigned long long g_bounds_hits;
__device__ __forceinline__ int chk_id(int id, int64_t n) {
    if ((unsigned long long)(long long)id >= (unsigned long long)n) {
        atomicAdd(&g_bounds_hits, 1ull);
        return 0;
    }
    return id;
}
#else
__device__ __forceinline__ int chk_id(int id, int64_t) { return id; }
#endif
__device__ __forceinline__ int4 chk4(int4 v, int64_t n) {
    return make_int4(chk_id(v.x, n), chk_id(v.y, n), chk_id(v.z, n), chk_id(v.w, n));
}
// host: indices this translation unit's kernels found out of range since the
// last call (the count is reset); synchronises s in the checked build only
static inline unsigned long long bounds_take_local(cudaStream_t s) {
#ifdef MFD_BOUNDS_CHECK
    unsigned long long v = 0, z = 0;
    if (cudaStreamSynchronize(s) != cudaSuccess) return 0;
    if (cudaMemcpyFromSymbol(&v, g_bounds_hits, sizeof(v)) != cudaSuccess) return 0;
    if (v) cudaMemcpyToSymbol(g_bounds_hits, &z, sizeof(z));
    return v;
#else
    (void)s;
    return 0;
#endif
}

// ---- PEC walls by images: an index entry of a node set with mirror walls
// carries a reflection code r in its top three bits (bit a: the neighbour is the
// mirror image of node `id` across the walls normal to axis a). A perfect
// conductor reflects the tangential E and the normal H with a sign change and
// the normal E and the tangential H without, so a gathered value enters the
// stencil sum with the sign of its parity under r.
constexpr int IMG_SHIFT = 29;
constexpr int IMG_MASK = (1 << IMG_SHIFT) - 1;
__device__ __forceinline__ float flip(float v, unsigned odd) { return __int_as_float(__float_as_int(v) ^ (int)(odd << 31)); }
__device__ __forceinline__ double flip(double v, unsigned odd) {
    return __longlong_as_double(__double_as_longlong(v) ^ (long long)((unsigned long long)odd << 63));
}
// splits raw entries into node ids (bounds-checked against n) and codes
__device__ __forceinline__ int4 img_split(int4 raw, int64_t n, uint4& code) {
    code = make_uint4((unsigned)raw.x >> IMG_SHIFT, (unsigned)raw.y >> IMG_SHIFT, (unsigned)raw.z >> IMG_SHIFT,
                      (unsigned)raw.w >> IMG_SHIFT);
    return chk4(make_int4(raw.x & IMG_MASK, raw.y & IMG_MASK, raw.z & IMG_MASK, raw.w & IMG_MASK), n);
}
// TMz {Ez, Hx, Hy, ce}: Ez is tangential to every wall, Hx normal to the x walls, Hy to the y walls
template <typename V4> __device__ __forceinline__ V4 img_tmz(V4 f, unsigned r) {
    f.x = flip(f.x, __popc(r & 3u) & 1u);
    f.y = flip(f.y, r & 1u);
    f.z = flip(f.z, (r >> 1) & 1u);
    return f;
}
// 3D E block {Ex, Ey, Ez, ce}: E_b is tangential to the walls normal to the other axes
template <typename V4> __device__ __forceinline__ V4 img_e3(V4 f, unsigned r) {
    f.x = flip(f.x, __popc(r & 6u) & 1u);
    f.y = flip(f.y, __popc(r & 5u) & 1u);
    f.z = flip(f.z, __popc(r & 3u) & 1u);
    return f;
}
// 3D H block {Hx, Hy, Hz, 0}: H_b is normal to the walls normal to axis b
template <typename V4> __device__ __forceinline__ V4 img_h3(V4 f, unsigned r) {
    f.x = flip(f.x, r & 1u);
    f.y = flip(f.y, (r >> 1) & 1u);
    f.z = flip(f.z, (r >> 2) & 1u);
    return f;
}

// ---- Q16 index decoding (see the layout notes at the top)
__device__ __forceinline__ int q16_id(unsigned u, int2 b) { return (int)u + ((u & 0x8000u) ? b.y : b.x); }
__device__ __forceinline__ int4 q16_lo(uint4 u, int2 b) {
    return make_int4(q16_id(u.x & 0xffffu, b), q16_id(u.x >> 16, b), q16_id(u.y & 0xffffu, b), q16_id(u.y >> 16, b));
}
__device__ __forceinline__ int4 q16_hi(uint4 u, int2 b) {
    return make_int4(q16_id(u.z & 0xffffu, b), q16_id(u.z >> 16, b), q16_id(u.w & 0xffffu, b), q16_id(u.w >> 16, b));
}

// Calls body(c, id) for the N4 (or n4_rt when N4 == 0) chunks of 4 stencil
// entries of the node in lane `lane` of slice `slice`, taking the indices from
// the Q16 stream when the slice has one and from the 32-bit stream otherwise.
template <int N4, bool KEEP, typename Body>
__device__ __forceinline__ void for_idx4(int n4_rt, int64_t slice, int lane, const int4* __restrict__ idx,
                                         const uint4* __restrict__ q, const int2* __restrict__ qb, int64_t bound,
                                         uint64_t pol, Body&& body) {
    const int n4 = N4 ? N4 : n4_rt;
    const int n8 = (n4 + 1) >> 1;
    const int2 b = q ? ld_stream_k<KEEP>(qb + slice, pol) : make_int2(-1, 0);
    if (b.x >= 0) {
        const uint4* p = q + slice * n8 * 32 + lane;
#pragma unroll
        for (int c8 = 0; c8 < (N4 ? (N4 + 1) / 2 : n8); ++c8) {
            const uint4 u = ld_stream_k<KEEP>(p + c8 * 32, pol);
            body(2 * c8, chk4(q16_lo(u, b), bound));
            if (2 * c8 + 1 < n4) body(2 * c8 + 1, chk4(q16_hi(u, b), bound));
        }
    } else {
        const int4* p = idx + slice * n4 * 32 + lane;
#pragma unroll
        for (int c = 0; c < n4; ++c) body(c, chk4(ld_stream_k<KEEP>(p + c * 32, pol), bound));
    }
}

template <typename T> struct Coefs {
    T ch;     // dt / mu0
    T gamma;  // Eq. 18 coefficient
};

}  // namespace mfd
