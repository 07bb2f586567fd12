// sim.cu -- the stepped simulation behind mfd_sim_* (include/mfd.h): packing of
// weights and stencils into the sliced streams of kernels.cuh, field and
// material upload, soft sources and probes, graph-captured stepping, energy.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "adjoint.cuh"
#include "internal.cuh"
#include "step.cuh"

namespace mfd {

enum Layout { COLLOC2D = 0, STAG2D = 1, COLLOC3D = 2 };

constexpr int GRAPH_STEPS = 32;  // steps per captured graph (even: ping-pong parity returns)

// ------------------------------------------------------------ packing kernels

// sliced layout: element e -> (slice s, chunk c, lane l, entry q)
// packed entry j of row r comes from stencil entry perm[r * plen + j] when a
// permutation is given (see k_row_perm), else from entry j
__device__ __forceinline__ int src_entry(const uint8_t* perm, int plen, int64_t node, int j) {
    return perm ? (int)perm[node * plen + j] : j;
}

__global__ void k_pack_idx(const int32_t* __restrict__ src, int stride, int64_t N, int n_use, int chunks,
                           const uint8_t* __restrict__ perm, int plen, int32_t* __restrict__ dst, int64_t total) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= total) return;
    int q = (int)(e & 3);
    int lane = (int)((e >> 2) & 31);
    int64_t rest = e >> 7;
    int c = (int)(rest % chunks);
    int64_t s = rest / chunks;
    int64_t node = s * 32 + lane;
    int entry = c * 4 + q;
    int32_t v = 0;
    if (node < N) v = src[node * stride + src_entry(perm, plen, node, entry < n_use ? entry : 0)];
    dst[e] = v;
}

template <typename T>
__global__ void k_pack_w(const double* __restrict__ w, int64_t N, int n_use, int chunks,
                         const uint8_t* __restrict__ perm, int plen, T* __restrict__ dst, int64_t total) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= total) return;
    int q = (int)(e & 3);
    int lane = (int)((e >> 2) & 31);
    int64_t rest = e >> 7;
    int c = (int)(rest % chunks);
    int64_t s = rest / chunks;
    int64_t node = s * 32 + lane;
    int entry = c * 4 + q;
    dst[e] = (node < N && entry < n_use) ? (T)w[node * n_use + src_entry(perm, plen, node, entry)] : (T)0;
}


// Q16 bases of one slice (one thread per slice): b0 is the smallest neighbour
// id; b1 the smallest id past b0's window of 32768; the slice is wide (b0 = -1)
// when an id falls outside both windows. Covering the ids with at most two
// windows, each opened at the smallest id not yet covered, succeeds whenever
// any two windows cover them.
__global__ void k_q16_bases(const int32_t* __restrict__ src, int stride, int64_t N, int n_use, int64_t slices,
                            int2* __restrict__ bases, unsigned long long* __restrict__ wide) {
    const int64_t sl = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (sl >= slices) return;
    const int64_t lo = sl * 32, hi = lo + 32 < N ? lo + 32 : N;
    int64_t b0 = INT64_MAX, b1 = INT64_MAX;
    for (int64_t i = lo; i < hi; ++i)
        for (int e = 0; e < n_use; ++e) b0 = min(b0, (int64_t)src[i * stride + e]);
    for (int64_t i = lo; i < hi; ++i)
        for (int e = 0; e < n_use; ++e) {
            const int64_t v = src[i * stride + e];
            if (v > b0 + 32767) b1 = min(b1, v);
        }
    bool ok = true;
    if (b1 != INT64_MAX)
        for (int64_t i = lo; i < hi && ok; ++i)
            for (int e = 0; e < n_use; ++e) {
                const int64_t v = src[i * stride + e];
                if (v > b0 + 32767 && v > b1 + 32767) ok = false;
            }
    if (b1 == INT64_MAX) b1 = b0 + 32768;
    bases[sl] = ok ? make_int2((int)b0, (int)(b1 - 32768)) : make_int2(-1, 0);
    if (!ok) atomicAdd(wide, 1ull);
}

// Q16 entries, laid out as the 32-bit chunks with 8 entries per chunk:
// element e -> (slice s, chunk c, lane l, entry q)
__global__ void k_pack_q16(const int32_t* __restrict__ src, int stride, int64_t N, int n_use, int chunks8,
                           const int2* __restrict__ bases, uint16_t* __restrict__ dst, int64_t total) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int q = (int)(e & 7);
    const int lane = (int)((e >> 3) & 31);
    const int64_t rest = e >> 8;
    const int c = (int)(rest % chunks8);
    const int64_t sl = rest / chunks8;
    const int64_t node = sl * 32 + lane;
    const int entry = c * 8 + q;
    const int2 b = bases[sl];
    unsigned v = 0;
    if (b.x >= 0 && node < N) {
        const int64_t id = src[node * stride + (entry < n_use ? entry : 0)];
        v = id - b.x <= 32767 ? (unsigned)(id - b.x) : (unsigned)(id - b.y);
    }
    dst[e] = (uint16_t)v;
}

template <typename T>
__global__ void k_scatter(const double* __restrict__ src, const int64_t* __restrict__ inv, int64_t n,
                          T* __restrict__ base, int stride, int offset) {
    int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (u >= n) return;
    base[inv[u] * stride + offset] = (T)src[u];
}

template <typename T>
__global__ void k_gather(const T* __restrict__ base, int stride, int offset, const int64_t* __restrict__ inv, int64_t n,
                         double* __restrict__ dst) {
    int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (u >= n) return;
    dst[u] = (double)base[inv[u] * stride + offset];
}

// ce_i = dt / (eps0 eps_r,i) (0 on 2D PEC nodes), eps_r and held masks in device order
template <typename T>
__global__ void k_materials(const double* __restrict__ eps_user, const uint8_t* __restrict__ pec_user,
                            const int64_t* __restrict__ perm, int64_t n, double dt_eps0, bool pec_zeroes_ce,
                            T* __restrict__ ce, int ce_stride, int ce_offset, double* __restrict__ eps_dev,
                            uint8_t* __restrict__ mask_dev) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    int64_t u = perm[k];
    double er = eps_user ? eps_user[u] : 1.0;
    uint8_t m = pec_user ? pec_user[u] : 0;
    eps_dev[k] = er;
    mask_dev[k] = m;
    double c = dt_eps0 / er;
    if (pec_zeroes_ce && m) c = 0.0;
    ce[k * ce_stride + ce_offset] = (T)c;
}

// hold PEC components at zero: 2D Ez (comps 1 = stride offset), 3D tangential components
template <typename T>
__global__ void k_zero_held(T* __restrict__ E, int stride, const uint8_t* __restrict__ mask, int64_t n, bool three_d) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    unsigned m = mask[k];
    if (!m) return;
    if (!three_d) {
        E[k * stride] = T(0);
        return;
    }
    if (m & 6u) E[k * stride + 0] = T(0);
    if (m & 5u) E[k * stride + 1] = T(0);
    if (m & 3u) E[k * stride + 2] = T(0);
}

// soft Ricker sources after the E update, then probes, then the step counter
template <typename T>
__global__ void k_post(T* __restrict__ ez, int ez_stride, const uint8_t* __restrict__ mask, unsigned held_bits,
                       int nsrc, const int64_t* __restrict__ sn, const double* __restrict__ sa,
                       const double* __restrict__ sf, const double* __restrict__ st0, int nprobe,
                       const int64_t* __restrict__ pn, const T* pv, int pv_stride, T* __restrict__ pbuf,
                       int64_t pcap, const int64_t* __restrict__ pstep0, int64_t* __restrict__ counter, double dt) {
    __shared__ int64_t n_s;
    if (threadIdx.x == 0) n_s = *counter;
    __syncthreads();
    const int64_t n = n_s;
    const double t1 = (double)(n + 1) * dt;
    const double pi = 3.14159265358979323846;
    for (int s = threadIdx.x; s < nsrc; s += blockDim.x) {
        const int64_t i = sn[s];
        if (mask && (mask[i] & held_bits)) continue;
        double a = pi * sf[s] * (t1 - st0[s]);
        a = a * a;
        const double r = (1.0 - 2.0 * a) * exp(-a);
        atomicAdd(ez + i * ez_stride, (T)(sa[s] * r));
    }
    __syncthreads();
    if (nprobe > 0) {
        const int64_t rec = n - *pstep0;
        if (rec >= 0 && rec < pcap)
            for (int p = threadIdx.x; p < nprobe; p += blockDim.x) pbuf[rec * nprobe + p] = pv[pn[p] * pv_stride];
    }
    __syncthreads();
    if (threadIdx.x == 0) *counter = n + 1;
}

__global__ void k_sum(const double* __restrict__ partial, int n, double* __restrict__ out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) s += partial[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// probe records (T [rec][np]) after steps stride, 2 stride, ... -> FP64 [nt][np]
template <typename T>
__global__ void k_probe_samples(const T* __restrict__ buf, int np, int stride, int nt, double* __restrict__ out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)nt * np) return;
    const int64_t n = e / np, m = e % np;
    out[e] = (double)buf[((n + 1) * stride - 1) * np + m];  // record of step (n + 1) stride
}

}  // namespace mfd

using namespace mfd;

struct PackedStencil {
    DevBuf idx_c, idx_v, wx, wy, wz, wv;
    DevBuf q_c, q_v, qb_c, qb_v;     // Q16 index streams and bases (staggered layout)
    int64_t wide_c = 0, wide_v = 0;  // slices left on the 32-bit streams
    int nc = 0, nv = 0, ni = 0;
    int64_t n = 0;
    int64_t src_c = 0, src_v = 0;  // sizes of the node sets the curl and HV indices point into
    bool mirror = false;           // entries carry image codes (node set with mirror walls)
    DevBuf cext;                   // uint8 curl chunks per slice when the curl stencil size varies, else empty
    int nc0 = 0;                   // chunks of the smallest curl stencil
};

struct mfd_sim {
    mfd_ctx* ctx = nullptr;
    mfd_sim_desc d{};
    Layout layout = COLLOC2D;
    bool fp64 = false, comp = false;
    size_t rs = 4;  // bytes per real
    const mfd_nodes* eset = nullptr;
    const mfd_nodes* hset = nullptr;
    int64_t ne = 0, nh = 0;
    PackedStencil hp, ep;  // H-pass and E-pass streams (collocated: ep unused)
    DevBuf s0, s1, s2, s3, s4, s5;
    DevBuf eps, mask, counter, pstep0;
    bool has_mask = false;
    DevBuf src_node, src_amp, src_f0, src_t0;
    int nsrc = 0;
    DevBuf probe_node, probe_buf;
    DevBuf stage;  // FP64 staging of host field I/O (mfd_set_field / mfd_get_field), kept between calls
    int nprobe = 0;
    int64_t probe_cap = 0, probe_from = 0;
    DevBuf partial, energy_out;
    int64_t steps = 0;
    int parity = 0;
    cudaGraphExec_t graph = nullptr;
    bool graph_ok = false;
    std::vector<cudaEvent_t> events;
    AdjT adj;
    bool adj_ok = false;
    int64_t adj_sweeps = 0;  // adjoint sweeps run (mfd_grad_backward)
    int block[2] = {256, 256};  // threads per block of the H and E half-step kernels (autotuned)
    int lanes[2] = {0, 0};      // collocated 2D: lanes per node of each pass (0: the size rule; autotuned)
    int probe_comp = MFD_EZ;    // the component the probes record
    bool q16 = true;            // staggered kernels read Q16 indices (mfd_sim_set_index_format)
    double l2_keep_set = -1.0;  // fraction of the stream lines kept in L2; < 0: sized from the L2 (mfd_sim_set_l2_keep)
    int64_t watch_every = 0;    // energy watchdog: check every this many steps (0: off)
    double watch_ratio = 0, watch_u0 = 0;
    ~mfd_sim() {
        if (graph) cudaGraphExecDestroy(graph);
        for (auto e : events) cudaEventDestroy(e);
    }
};

namespace {

mfd_status pack_stream(mfd_ctx* ctx, const mfd_stencils* st, int n_use, int chunks, DevBuf& out,
                       const DevBuf* perm = nullptr, int plen = 0) {
    const int64_t N = st->centres->n;
    const int64_t slices = (N + 31) / 32;
    const int64_t total = slices * chunks * 128;
    MFD_TRY(out.alloc(total * 4));
    const uint8_t* pm = perm && perm->p ? perm->as<uint8_t>() : nullptr;
    k_pack_idx<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(st->idx.as<int32_t>(), st->n, N, n_use,
                                                                         chunks, pm, plen, out.as<int32_t>(), total);
    MFD_CUDA(cudaGetLastError());
    return MFD_OK;
}

mfd_status pack_weights(mfd_ctx* ctx, const mfd_weights* w, int out_index, int chunks, bool fp64, DevBuf& out,
                        const DevBuf* perm = nullptr, int plen = 0) {
    const int64_t N = w->st->centres->n;
    const int64_t slices = (N + 31) / 32;
    const int64_t total = slices * chunks * 128;
    MFD_TRY(out.alloc(total * (fp64 ? 8 : 4)));
    const double* src = w->w.as<double>() + (int64_t)out_index * N * w->n_use;
    const uint8_t* pm = perm && perm->p ? perm->as<uint8_t>() : nullptr;
    unsigned g = (unsigned)((total + 255) / 256);
    if (fp64) k_pack_w<double><<<g, 256, 0, ctx->stream>>>(src, N, w->n_use, chunks, pm, plen, out.as<double>(), total);
    else k_pack_w<float><<<g, 256, 0, ctx->stream>>>(src, N, w->n_use, chunks, pm, plen, out.as<float>(), total);
    MFD_CUDA(cudaGetLastError());
    return MFD_OK;
}

int chunks_of(int n) { return (n + 3) / 4; }

#ifdef MFD_BOUNDS_CHECK
__global__ void k_check_rows(const int32_t* __restrict__ idx, int stride, int64_t N, int n_use, int64_t nsrc) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < N * n_use) chk_id(idx[(e / n_use) * stride + e % n_use] & IMG_MASK, nsrc);
}

void check_rows(mfd_ctx* ctx, const mfd_stencils* st, int n_use) {
    const int64_t total = st->centres->n * n_use;
    k_check_rows<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(st->idx.as<int32_t>(), st->n,
                                                                           st->centres->n, n_use, st->sources->n);
}
#endif

// MFD_ERR_STATE when a kernel of the bounds-checked build met a stencil index
// outside its node set (always MFD_OK in the default build)
mfd_status bounds_status(cudaStream_t s) {
    const unsigned long long hits = bounds_take_local(s) + bounds_take_step2d(s) + bounds_take_step3d(s) +
                                    bounds_take_adjoint(s);
    if (hits) return fail(MFD_ERR_STATE, std::to_string(hits) + " stencil indices out of range (bounds-checked build)");
    return MFD_OK;
}

// a host vector into a new device buffer (at least one element), synchronously
template <typename T> mfd_status upload_host(DevBuf& b, const std::vector<T>& v) {
    MFD_TRY(b.alloc(std::max<size_t>(1, v.size()) * sizeof(T)));
    if (!v.empty()) MFD_CUDA(cudaMemcpy(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return MFD_OK;
}

// Q16 form of one index stream (chunks4 chunks of 4 entries per row)
mfd_status pack_q16(mfd_ctx* ctx, const mfd_stencils* st, int n_use, int chunks4, DevBuf& q, DevBuf& qb,
                    int64_t& wide) {
    const int64_t N = st->centres->n;
    const int64_t slices = (N + 31) / 32;
    const int chunks8 = (chunks4 + 1) / 2;
    const int64_t total = slices * chunks8 * 256;
    MFD_TRY(q.alloc(total * 2));
    MFD_TRY(qb.alloc(slices * sizeof(int2)));
    DevBuf cnt;
    MFD_TRY(cnt.alloc(8));
    MFD_CUDA(cudaMemsetAsync(cnt.p, 0, 8, ctx->stream));
    k_q16_bases<<<(unsigned)((slices + 127) / 128), 128, 0, ctx->stream>>>(st->idx.as<int32_t>(), st->n, N, n_use,
                                                                          slices, qb.as<int2>(),
                                                                          cnt.as<unsigned long long>());
    MFD_CUDA(cudaGetLastError());
    k_pack_q16<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(st->idx.as<int32_t>(), st->n, N, n_use,
                                                                        chunks8, qb.as<int2>(), q.as<uint16_t>(),
                                                                        total);
    MFD_CUDA(cudaGetLastError());
    unsigned long long w = 0;
    MFD_CUDA(cudaMemcpyAsync(&w, cnt.p, 8, cudaMemcpyDeviceToHost, ctx->stream));
    MFD_CUDA(cudaStreamSynchronize(ctx->stream));
    wide = (int64_t)w;
    return MFD_OK;
}

// curl chunks of each 32-node slice: the most any of its centres needs
__global__ void k_slice_chunks(const int32_t* __restrict__ nsz, int64_t N, int64_t slices, uint8_t* __restrict__ out) {
    const int64_t sl = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (sl >= slices) return;
    int c = 0;
    for (int64_t i = sl * 32; i < sl * 32 + 32 && i < N; ++i) c = max(c, (nsz[i] + 3) / 4);
    out[sl] = (uint8_t)c;
}

// packs the curl and HV streams of one pass
mfd_status pack_pass(mfd_ctx* ctx, const mfd_weights* curl, const mfd_weights* hv, int dim, bool fp64, PackedStencil& p) {
    p.n = curl->st->centres->n;
    p.src_c = curl->st->sources->n;
    p.src_v = hv->st->sources->n;
    p.mirror = curl->st->sources->mirror_axes != 0 || hv->st->sources->mirror_axes != 0;
#ifdef MFD_BOUNDS_CHECK
    // pack-time row check: every stencil entry lies in the node set it points into
    check_rows(ctx, curl->st, curl->n_use);
    check_rows(ctx, hv->st, hv->n_use);
#endif
    p.nc = chunks_of(curl->n_use);
    p.nc0 = chunks_of(curl->n_min);
    p.nv = chunks_of(hv->n_use);
    if (curl->nsz.p) {  // per-centre curl sizes: each slice reads the chunks its centres need
        const int64_t slices = (p.n + 31) / 32;
        MFD_TRY(p.cext.alloc(std::max<int64_t>(slices, 1)));
        k_slice_chunks<<<(unsigned)((slices + 127) / 128), 128, 0, ctx->stream>>>(curl->nsz.as<int32_t>(), p.n,
                                                                                   slices, p.cext.as<uint8_t>());
        MFD_CUDA(cudaGetLastError());
    }
    const bool shared = curl->st == hv->st;
    DevBuf perm;
    int plen = 0;
    if (shared) {
        p.ni = std::max(p.nc, p.nv);
        plen = std::max(curl->n_use, hv->n_use);
        if (plen <= 255) {  // rows in ascending id order (launch_row_perm)
            const int64_t N = curl->st->centres->n;
            MFD_TRY(perm.alloc(N * plen));
            // split points: the stencil sizes below plen (the smallest and the largest curl
            // stencil and the HV stencil), so every stencil keeps its entries
            int cut[3] = {curl->n_min, curl->n_use, hv->n_use};
            std::sort(cut, cut + 3);
            MFD_CUDA(launch_row_perm(curl->st->idx.as<int32_t>(), curl->st->n, N, cut[0], cut[1], plen,
                                     perm.as<uint8_t>(), ctx->stream));
        }
        MFD_TRY(pack_stream(ctx, curl->st, plen, p.ni, p.idx_c, &perm, plen));
    } else {
        p.ni = p.nc;
        MFD_TRY(pack_stream(ctx, curl->st, curl->n_use, p.nc, p.idx_c));
        MFD_TRY(pack_stream(ctx, hv->st, hv->n_use, p.nv, p.idx_v));
        if (dim == 2 && curl->st->centres != curl->st->sources) {  // staggered
            MFD_TRY(pack_q16(ctx, curl->st, curl->n_use, p.nc, p.q_c, p.qb_c, p.wide_c));
            MFD_TRY(pack_q16(ctx, hv->st, hv->n_use, p.nv, p.q_v, p.qb_v, p.wide_v));
        }
    }
    MFD_TRY(pack_weights(ctx, curl, 0, p.nc, fp64, p.wx, &perm, plen));
    MFD_TRY(pack_weights(ctx, curl, 1, p.nc, fp64, p.wy, &perm, plen));
    if (dim == 3) MFD_TRY(pack_weights(ctx, curl, 2, p.nc, fp64, p.wz, &perm, plen));
    MFD_TRY(pack_weights(ctx, hv, 0, p.nv, fp64, p.wv, &perm, plen));
    MFD_CUDA(cudaStreamSynchronize(ctx->stream));  // perm is freed on return
    return MFD_OK;
}

template <typename T> StencilStreams<T> streams(const PackedStencil& p, bool q16 = false) {
    StencilStreams<T> s;
    s.idx_c = p.idx_c.as<const int4>();
    s.idx_v = p.idx_v.p ? p.idx_v.as<const int4>() : s.idx_c;
    if (q16 && p.q_c.p && p.q_v.p) {
        s.q_c = p.q_c.as<const uint4>();
        s.q_v = p.q_v.as<const uint4>();
        s.qb_c = p.qb_c.as<const int2>();
        s.qb_v = p.qb_v.as<const int2>();
    }
    s.wx = p.wx.as<const typename Vec<T>::V4>();
    s.wy = p.wy.as<const typename Vec<T>::V4>();
    s.wz = p.wz.p ? p.wz.as<const typename Vec<T>::V4>() : nullptr;
    s.wv = p.wv.as<const typename Vec<T>::V4>();
    s.nc = p.nc;
    s.nv = p.nv;
    s.ni = p.ni;
    s.n = p.n;
    s.src_c = p.src_c;
    s.src_v = p.idx_v.p ? p.src_v : p.src_c;
    s.mirror = p.mirror;
    s.cext = p.cext.p ? p.cext.as<const uint8_t>() : nullptr;
    s.nc0 = p.nc0;
    return s;
}

// the fraction of the stencil streams' cache lines marked evict_last (stream_policy):
// the kept lines fill about 40 % of the L2 (the rest holds the fields and the lines
// in flight; on a two-die part a line read from both dies may be held in both
// halves of the L2). Measured: the 250k-node collocated problem (streams 0.8x the
// L2) ran 10 % faster per step at that fraction while 60 % and more thrashed; the
// 400^2 staggered problem (1.7x) 5 % faster; at 600^2 (3.7x) every kept fraction
// was slower. So below 0.15 (streams above about 2.7 L2 sizes) nothing is kept
// and every line is evict_first.
float keep_for(int64_t stream_bytes, int64_t l2_bytes) {
    if (stream_bytes <= 0 || l2_bytes <= 0) return 0.0f;
    const double k = 0.4 * (double)l2_bytes / (double)stream_bytes;
    return k >= 1.0 ? 1.0f : (k < 0.15 ? 0.0f : (float)k);
}

// bytes of the stencil streams one step reads: the weights and the index form the kernels take
int64_t step_stream_bytes(const mfd_sim* sim) {
    auto one = [&](const PackedStencil& p) {
        int64_t b = (int64_t)(p.wx.bytes + p.wy.bytes + p.wz.bytes + p.wv.bytes);
        if (sim->q16 && p.q_c.p && p.q_v.p) b += (int64_t)(p.q_c.bytes + p.q_v.bytes + p.qb_c.bytes + p.qb_v.bytes);
        else b += (int64_t)(p.idx_c.bytes + p.idx_v.bytes);
        return b;
    };
    return one(sim->hp) + (sim->layout == STAG2D ? one(sim->ep) : 0);
}

float sim_keep(const mfd_sim* sim) {
    if (sim->layout == COLLOC3D) return 0.0f;  // the 3D kernels stream every line evict_first
    if (sim->l2_keep_set >= 0) return (float)sim->l2_keep_set;
    return keep_for(step_stream_bytes(sim), sim->ctx->l2_bytes);
}

Launch2D make2d(mfd_sim* sim, int parity) {
    Launch2D L;
    L.staggered = sim->layout == STAG2D;
    L.fp64 = sim->fp64;
    L.comp = sim->comp;
    L.hs.f = streams<float>(sim->hp, sim->q16);
    L.hs.d = streams<double>(sim->hp, sim->q16);
    if (L.staggered) {
        L.es.f = streams<float>(sim->ep, sim->q16);
        L.es.d = streams<double>(sim->ep, sim->q16);
    }
    const float keep = sim_keep(sim);
    L.hs.f.l2_keep = L.hs.d.l2_keep = L.es.f.l2_keep = L.es.d.l2_keep = keep;
    L.kf.ch = (float)(sim->d.dt / sim->d.mu0);
    L.kf.gamma = (float)sim->d.gamma;
    L.kd.ch = sim->d.dt / sim->d.mu0;
    L.kd.gamma = sim->d.gamma;
    L.block[0] = sim->block[0];
    L.block[1] = sim->block[1];
    // collocated rows shared by both stencils: four lanes per node while one thread per node
    // would occupy less than a quarter of the GPU's threads, unless the autotuner chose
    if (!L.staggered && sim->hp.idx_v.p == nullptr) {
        const int rule = sim->ne * 4 <= (int64_t)sim->ctx->sm_count * 512 ? 4 : 1;
        for (int p = 0; p < 2; ++p) L.lanes[p] = sim->lanes[p] ? sim->lanes[p] : rule;
    }
    if (!L.staggered) {
        L.A = sim->s0.p;
        L.B = sim->s1.p;
    } else {
        DevBuf* E[2] = {&sim->s0, &sim->s1};
        DevBuf* H[2] = {&sim->s2, &sim->s3};
        L.stag.ez = E[parity]->p;
        L.stag.ezn = E[parity ^ 1]->p;
        L.stag.h = H[parity]->p;
        L.stag.hn = H[parity ^ 1]->p;
        L.stag.ce = sim->s4.p;
    }
    return L;
}

Launch3D make3d(mfd_sim* sim, int parity) {
    Launch3D L;
    L.fp64 = sim->fp64;
    L.comp = sim->comp;
    L.s.f = streams<float>(sim->hp);
    L.s.d = streams<double>(sim->hp);
    L.s.f.l2_keep = L.s.d.l2_keep = sim_keep(sim);
    L.kf.ch = (float)(sim->d.dt / sim->d.mu0);
    L.kf.gamma = (float)sim->d.gamma;
    L.kd.ch = sim->d.dt / sim->d.mu0;
    L.kd.gamma = sim->d.gamma;
    L.block[0] = sim->block[0];
    L.block[1] = sim->block[1];
    (void)parity;  // the 3D state is rewritten in place by the E pass
    L.F = sim->s0.p;
    L.Es = sim->s1.p;
    L.Hn = sim->s2.p;
    L.wall = sim->has_mask ? sim->mask.as<const uint8_t>() : nullptr;
    return L;
}

// where Ez of the current state lives: base pointer, stride (reals), byte size of a real
void ez_location(mfd_sim* sim, int parity_after, void** base, int* stride) {
    if (sim->layout == COLLOC2D) {
        *base = sim->s0.p;
        *stride = 4;
    } else if (sim->layout == STAG2D) {
        *base = parity_after ? sim->s1.p : sim->s0.p;
        *stride = 1;
    } else {
        *base = (char*)sim->s0.p + 2 * sim->rs;
        *stride = 8;
    }
}

cudaError_t launch_post(mfd_sim* sim, int parity_after) {
    void* ez;
    int stride;
    ez_location(sim, parity_after, &ez, &stride);
    // the probed component (mfd_set_probe_component): Ez, or another component
    // of the collocated state (H at the half step the leapfrog holds)
    char* pv = static_cast<char*>(ez);
    int pstride = stride;
    if (sim->probe_comp != MFD_EZ) {
        const int off = sim->layout == COLLOC2D ? (sim->probe_comp == MFD_HX ? 1 : 2)
                                                : (sim->probe_comp <= MFD_EZ ? sim->probe_comp : 4 + sim->probe_comp - MFD_HX);
        pv = static_cast<char*>(sim->s0.p) + (size_t)off * sim->rs;
    }
    const uint8_t* mask = sim->has_mask ? sim->mask.as<const uint8_t>() : nullptr;
    unsigned held = sim->layout == COLLOC3D ? 3u : 0xFFu;
    const double dt = sim->d.dt;
    if (sim->fp64)
        k_post<double><<<1, 256, 0, sim->ctx->stream>>>(
            (double*)ez, stride, mask, held, sim->nsrc, sim->src_node.as<int64_t>(), sim->src_amp.as<double>(),
            sim->src_f0.as<double>(), sim->src_t0.as<double>(), sim->nprobe, sim->probe_node.as<int64_t>(),
            (const double*)pv, pstride, sim->probe_buf.as<double>(), sim->probe_cap, sim->pstep0.as<int64_t>(),
            sim->counter.as<int64_t>(), dt);
    else
        k_post<float><<<1, 256, 0, sim->ctx->stream>>>(
            (float*)ez, stride, mask, held, sim->nsrc, sim->src_node.as<int64_t>(), sim->src_amp.as<double>(),
            sim->src_f0.as<double>(), sim->src_t0.as<double>(), sim->nprobe, sim->probe_node.as<int64_t>(),
            (const float*)pv, pstride, sim->probe_buf.as<float>(), sim->probe_cap, sim->pstep0.as<int64_t>(),
            sim->counter.as<int64_t>(), dt);
    return cudaGetLastError();
}

// enqueues one step; events (optional): before H, between H and E, after E
cudaError_t enqueue_step(mfd_sim* sim, cudaEvent_t* ev) {
    cudaStream_t s = sim->ctx->stream;
    cudaError_t e;
    const int p = sim->parity;
    const int pn = (sim->layout == STAG2D) ? (p ^ 1) : p;
    if (ev) cudaEventRecord(ev[0], s);
    if (sim->layout == COLLOC3D) {
        Launch3D L = make3d(sim, p);
        if ((e = launch_3d(L, 0, s)) != cudaSuccess) return e;
        if (ev) cudaEventRecord(ev[1], s);
        if ((e = launch_3d(L, 1, s)) != cudaSuccess) return e;
    } else {
        Launch2D L = make2d(sim, p);
        if ((e = launch_2d(L, 0, s)) != cudaSuccess) return e;
        if (ev) cudaEventRecord(ev[1], s);
        if ((e = launch_2d(L, 1, s)) != cudaSuccess) return e;
    }
    if (ev) cudaEventRecord(ev[2], s);
    if ((e = launch_post(sim, pn)) != cudaSuccess) return e;
    sim->parity = pn;
    sim->steps += 1;
    return cudaSuccess;
}

mfd_status ensure_graph(mfd_sim* sim) {
    if (sim->graph_ok) return MFD_OK;
    if (sim->graph) {
        cudaGraphExecDestroy(sim->graph);
        sim->graph = nullptr;
    }
    cudaStream_t s = sim->ctx->stream;
    const int64_t steps0 = sim->steps;
    const int par0 = sim->parity;
    MFD_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < GRAPH_STEPS && e == cudaSuccess; ++k) e = enqueue_step(sim, nullptr);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s, &g);
    sim->steps = steps0;
    sim->parity = par0;
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(MFD_ERR_CUDA, std::string("graph capture failed: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&sim->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(MFD_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    sim->graph_ok = true;
    return MFD_OK;
}

// the simulation's staging buffer of at least `bytes` (grown, never shrunk): host field
// I/O then allocates and frees nothing per call (cudaFree synchronises the device)
mfd_status staging(mfd_sim* sim, size_t bytes, double** out) {
    if (sim->stage.bytes < bytes) MFD_TRY(sim->stage.alloc(bytes));
    *out = sim->stage.as<double>();
    return MFD_OK;
}

mfd_status upload(mfd_ctx* ctx, DevBuf& dst, const void* host, size_t bytes) {
    MFD_TRY(dst.alloc(bytes));
    if (bytes) MFD_CUDA(cudaMemcpyAsync(dst.p, host, bytes, cudaMemcpyHostToDevice, ctx->stream));
    return MFD_OK;
}

mfd_status check_set(const mfd_weights* curl, const mfd_weights* hv, const mfd_nodes* centres,
                     const mfd_nodes* curl_src) {
    if (!curl || !hv) return fail(MFD_ERR_ARG, "missing weights");
    if (curl->op != MFD_OP_GRAD && curl->op != MFD_OP_GRAD_VFD) return fail(MFD_ERR_ARG, "curl weights must be first derivatives");
    if (hv->op != MFD_OP_LAP_POW) return fail(MFD_ERR_ARG, "hyperviscosity weights must be Delta^alpha");
    if (curl->st->centres != centres || hv->st->centres != centres) return fail(MFD_ERR_ARG, "weights on a different centre set");
    if (hv->st->sources != centres) return fail(MFD_ERR_ARG, "hyperviscosity stencils must be own-set");
    if (curl->st->sources != curl_src) return fail(MFD_ERR_ARG, "curl stencils must take the other field's nodes");
    return MFD_OK;
}

// per-node materials from device arrays in caller order (eps_r: NULL = vacuum;
// pec: NULL = none): the E coefficient dt / (eps0 eps_r) (0 on held nodes),
// eps_r in device order, the held mask, and held components zeroed
mfd_status apply_materials(mfd_sim* sim, const double* de, const uint8_t* dp) {
    mfd_ctx* ctx = sim->ctx;
    const int64_t ne = sim->ne;
    const double dt_eps0 = sim->d.dt / sim->d.eps0;
    void* ce;
    int stride, offset;
    if (sim->layout == STAG2D) {
        ce = sim->s4.p;
        stride = 1;
        offset = 0;
    } else {
        ce = sim->s0.p;
        stride = sim->layout == COLLOC3D ? 8 : 4;
        offset = 3;
    }
    const bool zero_ce = sim->layout != COLLOC3D;
    unsigned g = (unsigned)((ne + 255) / 256);
    if (sim->fp64)
        k_materials<double><<<g, 256, 0, ctx->stream>>>(de, dp, sim->eset->perm.as<int64_t>(), ne, dt_eps0, zero_ce,
                                                        (double*)ce, stride, offset, sim->eps.as<double>(),
                                                        sim->mask.as<uint8_t>());
    else
        k_materials<float><<<g, 256, 0, ctx->stream>>>(de, dp, sim->eset->perm.as<int64_t>(), ne, dt_eps0, zero_ce,
                                                       (float*)ce, stride, offset, sim->eps.as<double>(),
                                                       sim->mask.as<uint8_t>());
    MFD_CUDA(cudaGetLastError());
    sim->has_mask = dp != nullptr;
    sim->graph_ok = false;
    if (sim->has_mask) {
        void* ez;
        int st2;
        ez_location(sim, sim->parity, &ez, &st2);
        void* base = sim->layout == COLLOC3D ? sim->s0.p : ez;
        if (sim->fp64)
            k_zero_held<double><<<g, 256, 0, ctx->stream>>>((double*)base, st2, sim->mask.as<uint8_t>(), ne,
                                                            sim->layout == COLLOC3D);
        else
            k_zero_held<float><<<g, 256, 0, ctx->stream>>>((float*)base, st2, sim->mask.as<uint8_t>(), ne,
                                                           sim->layout == COLLOC3D);
        MFD_CUDA(cudaGetLastError());
    }
    MFD_CUDA(cudaStreamSynchronize(ctx->stream));
    return MFD_OK;
}

}  // namespace

extern "C" {

mfd_status mfd_energy(mfd_sim* sim, double* u);

mfd_status mfd_sim_create(mfd_ctx* ctx, const mfd_sim_desc* desc, mfd_sim** out) {
    if (!ctx || !desc || !out) return fail(MFD_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (desc->dim != 2 && desc->dim != 3) return fail(MFD_ERR_ARG, "dim must be 2 or 3");
    if (desc->precision != MFD_FP32 && desc->precision != MFD_FP64) return fail(MFD_ERR_ARG, "unknown precision");
    if (desc->nrhs != 1) return fail(MFD_ERR_ARG, "mfd_sim steps one right-hand side; use the batched API for more");
    if (!(desc->dt > 0) || !(desc->eps0 > 0) || !(desc->mu0 > 0)) return fail(MFD_ERR_ARG, "dt, eps0, mu0 must be > 0");
    if (!desc->h_curl || !desc->e_curl) return fail(MFD_ERR_ARG, "missing curl weights");
    const mfd_nodes* H = desc->h_curl->st->centres;
    const mfd_nodes* E = desc->e_curl->st->centres;
    MFD_TRY(check_set(desc->h_curl, desc->h_hv, H, E));
    MFD_TRY(check_set(desc->e_curl, desc->e_hv, E, H));
    if (E->ctx != ctx) return fail(MFD_ERR_ARG, "weights belong to another context");
    if (E->dim != desc->dim) return fail(MFD_ERR_ARG, "dim differs from the node sets");
    const bool colloc = (E == H);
    if (colloc && (desc->h_curl != desc->e_curl || desc->h_hv != desc->e_hv))
        return fail(MFD_ERR_ARG, "collocated: h_curl == e_curl and h_hv == e_hv expected");
    if (desc->dim == 3 && !colloc) return fail(MFD_ERR_ARG, "3D supports the collocated layout only");
    if (!colloc && (desc->h_curl->st->sources->mirror_axes || desc->e_curl->st->sources->mirror_axes))
        return fail(MFD_ERR_ARG, "mirror walls (images) are supported in the collocated layout");
    if ((desc->h_hv && desc->h_hv->nsz.p) || (desc->e_hv && desc->e_hv->nsz.p))
        return fail(MFD_ERR_ARG, "hyperviscosity weights take one stencil size");
    if (desc->dim != 3 && (desc->h_curl->nsz.p || desc->e_curl->nsz.p))
        return fail(MFD_ERR_ARG, "per-centre curl stencil sizes are supported in the 3D layout");
    MFD_CUDA(cudaSetDevice(ctx->device));
    mfd_sim* sim = new (std::nothrow) mfd_sim();
    if (!sim) return fail(MFD_ERR_OOM, "host allocation failed");
    sim->ctx = ctx;
    sim->d = *desc;
    sim->fp64 = desc->precision == MFD_FP64;
    sim->comp = !sim->fp64 && desc->compensated;
    sim->rs = sim->fp64 ? 8 : 4;
    sim->eset = E;
    sim->hset = H;
    sim->ne = E->n;
    sim->nh = H->n;
    sim->layout = desc->dim == 3 ? COLLOC3D : (colloc ? COLLOC2D : STAG2D);
    auto bail = [&](mfd_status st) {
        delete sim;
        return st;
    };
    mfd_status st;
    if ((st = pack_pass(ctx, desc->h_curl, desc->h_hv, desc->dim, sim->fp64, sim->hp))) return bail(st);
    if (sim->layout == STAG2D && (st = pack_pass(ctx, desc->e_curl, desc->e_hv, 2, sim->fp64, sim->ep)))
        return bail(st);
    const size_t rs = sim->rs;
    const int64_t ne = sim->ne, nh = sim->nh;
    if (sim->layout == COLLOC2D) {
        if ((st = sim->s0.alloc(ne * 4 * rs)) || (st = sim->s1.alloc(ne * 4 * rs))) return bail(st);
    } else if (sim->layout == STAG2D) {
        if ((st = sim->s0.alloc(ne * rs)) || (st = sim->s1.alloc(ne * rs)) || (st = sim->s2.alloc(nh * 2 * rs)) ||
            (st = sim->s3.alloc(nh * 2 * rs)) || (st = sim->s4.alloc(ne * rs)))
            return bail(st);
    } else {
        // 3D: s0 = interleaved state {E block, H block} per node, s1 = E*, s2 = H'
        if ((st = sim->s0.alloc(ne * 8 * rs)) || (st = sim->s1.alloc(ne * 4 * rs)) || (st = sim->s2.alloc(ne * 4 * rs)))
            return bail(st);
    }
    for (DevBuf* b : {&sim->s0, &sim->s1, &sim->s2, &sim->s3, &sim->s4})
        if (b->p) cudaMemsetAsync(b->p, 0, b->bytes, ctx->stream);
    const int64_t nmax = std::max(ne, nh);
    if ((st = sim->eps.alloc(ne * 8)) || (st = sim->mask.alloc(ne)) || (st = sim->counter.alloc(8)) ||
        (st = sim->pstep0.alloc(8)) || (st = sim->partial.alloc(((nmax + 255) / 256) * 8)) ||
        (st = sim->energy_out.alloc(8)))
        return bail(st);
    cudaMemsetAsync(sim->counter.p, 0, 8, ctx->stream);
    cudaMemsetAsync(sim->pstep0.p, 0, 8, ctx->stream);
    *out = sim;
    st = mfd_set_materials(sim, nullptr, nullptr);
    if (!st) st = bounds_status(ctx->stream);  // pack-time row checks of the bounds-checked build
    if (st) {
        *out = nullptr;
        return bail(st);
    }
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        *out = nullptr;
        delete sim;
        return fail(MFD_ERR_CUDA, cudaGetErrorString(e));
    }
    retain(ctx);
    retain(desc->h_curl);
    retain(desc->h_hv);
    retain(desc->e_curl);
    retain(desc->e_hv);
    return MFD_OK;
}

mfd_status mfd_set_materials(mfd_sim* sim, const double* eps_r, const uint8_t* pec) {
    if (!sim) return fail(MFD_ERR_ARG, "sim is NULL");
    mfd_ctx* ctx = sim->ctx;
    MFD_CUDA(cudaSetDevice(ctx->device));
    const int64_t ne = sim->ne;
    if (eps_r)
        for (int64_t i = 0; i < ne; ++i)
            if (!(eps_r[i] > 0)) return fail(MFD_ERR_ARG, "eps_r must be > 0");
    DevBuf de, dp;
    if (eps_r) MFD_TRY(upload(ctx, de, eps_r, ne * 8));
    if (pec) MFD_TRY(upload(ctx, dp, pec, ne));
    return apply_materials(sim, de.as<double>(), dp.as<uint8_t>());
}

// locates (buffer, stride, offset, node set) of a component in the current state
static mfd_status locate(mfd_sim* sim, int comp, void** base, int* stride, int* offset, const mfd_nodes** set) {
    const bool is_e = comp <= MFD_EZ;
    if (comp < 0 || comp > MFD_HZ) return fail(MFD_ERR_ARG, "unknown component");
    if (sim->layout != COLLOC3D && comp != MFD_EZ && comp != MFD_HX && comp != MFD_HY)
        return fail(MFD_ERR_ARG, "TMz has Ez, Hx, Hy only");
    *set = is_e ? sim->eset : sim->hset;
    const int p = sim->parity;
    if (sim->layout == COLLOC2D) {
        *base = sim->s0.p;
        *stride = 4;
        *offset = comp == MFD_EZ ? 0 : (comp == MFD_HX ? 1 : 2);
    } else if (sim->layout == STAG2D) {
        if (is_e) {
            *base = p ? sim->s1.p : sim->s0.p;
            *stride = 1;
            *offset = 0;
        } else {
            *base = p ? sim->s3.p : sim->s2.p;
            *stride = 2;
            *offset = comp == MFD_HX ? 0 : 1;
        }
    } else {
        *stride = 8;
        *base = sim->s0.p;
        *offset = is_e ? comp - MFD_EX : 4 + comp - MFD_HX;
    }
    return MFD_OK;
}

// scatter of caller-order FP64 values (device) into component comp of the state
static mfd_status scatter_field(mfd_sim* sim, int comp, const double* dsrc) {
    mfd_ctx* ctx = sim->ctx;
    void* base;
    int stride, offset;
    const mfd_nodes* set;
    MFD_TRY(locate(sim, comp, &base, &stride, &offset, &set));
    unsigned g = (unsigned)((set->n + 255) / 256);
    if (sim->fp64)
        k_scatter<double><<<g, 256, 0, ctx->stream>>>(dsrc, set->inv.as<int64_t>(), set->n, (double*)base, stride, offset);
    else
        k_scatter<float><<<g, 256, 0, ctx->stream>>>(dsrc, set->inv.as<int64_t>(), set->n, (float*)base, stride, offset);
    MFD_CUDA(cudaGetLastError());
    if (comp <= MFD_EZ && sim->has_mask) {
        if (sim->fp64)
            k_zero_held<double><<<g, 256, 0, ctx->stream>>>((double*)base + (sim->layout == COLLOC3D ? 0 : offset),
                                                            stride, sim->mask.as<uint8_t>(), set->n, sim->layout == COLLOC3D);
        else
            k_zero_held<float><<<g, 256, 0, ctx->stream>>>((float*)base + (sim->layout == COLLOC3D ? 0 : offset),
                                                           stride, sim->mask.as<uint8_t>(), set->n, sim->layout == COLLOC3D);
        MFD_CUDA(cudaGetLastError());
    }
    if (comp == MFD_EZ) {
        MFD_CUDA(cudaMemsetAsync(sim->counter.p, 0, 8, ctx->stream));
        MFD_CUDA(cudaMemsetAsync(sim->pstep0.p, 0, 8, ctx->stream));
        sim->steps = 0;
        sim->probe_from = 0;
    }
    return MFD_OK;
}

// gather of component comp into caller-order FP64 values (device)
static mfd_status gather_field(mfd_sim* sim, int comp, double* ddst, int64_t* count) {
    mfd_ctx* ctx = sim->ctx;
    void* base;
    int stride, offset;
    const mfd_nodes* set;
    MFD_TRY(locate(sim, comp, &base, &stride, &offset, &set));
    if (count) *count = set->n;
    if (!ddst) return MFD_OK;
    unsigned g = (unsigned)((set->n + 255) / 256);
    if (sim->fp64)
        k_gather<double><<<g, 256, 0, ctx->stream>>>((const double*)base, stride, offset, set->inv.as<int64_t>(), set->n,
                                                     ddst);
    else
        k_gather<float><<<g, 256, 0, ctx->stream>>>((const float*)base, stride, offset, set->inv.as<int64_t>(), set->n,
                                                    ddst);
    MFD_CUDA(cudaGetLastError());
    return MFD_OK;
}

mfd_status mfd_set_field(mfd_sim* sim, int comp, int rhs, const double* host) {
    if (!sim || !host) return fail(MFD_ERR_ARG, "NULL argument");
    if (rhs != 0) return fail(MFD_ERR_ARG, "rhs out of range");
    mfd_ctx* ctx = sim->ctx;
    MFD_CUDA(cudaSetDevice(ctx->device));
    int64_t n = 0;
    MFD_TRY(gather_field(sim, comp, nullptr, &n));
    double* d = nullptr;
    MFD_TRY(staging(sim, (size_t)n * 8, &d));
    MFD_CUDA(cudaMemcpyAsync(d, host, (size_t)n * 8, cudaMemcpyHostToDevice, ctx->stream));
    MFD_TRY(scatter_field(sim, comp, d));
    MFD_CUDA(cudaStreamSynchronize(ctx->stream));
    return MFD_OK;
}

mfd_status mfd_get_field(mfd_sim* sim, int comp, int rhs, double* host) {
    if (!sim || !host) return fail(MFD_ERR_ARG, "NULL argument");
    if (rhs != 0) return fail(MFD_ERR_ARG, "rhs out of range");
    mfd_ctx* ctx = sim->ctx;
    MFD_CUDA(cudaSetDevice(ctx->device));
    int64_t n = 0;
    MFD_TRY(gather_field(sim, comp, nullptr, &n));
    double* d = nullptr;
    MFD_TRY(staging(sim, (size_t)n * 8, &d));
    MFD_TRY(gather_field(sim, comp, d, nullptr));
    MFD_CUDA(cudaMemcpyAsync(host, d, (size_t)n * 8, cudaMemcpyDeviceToHost, ctx->stream));
    MFD_CUDA(cudaStreamSynchronize(ctx->stream));
    return MFD_OK;
}

mfd_status mfd_set_field_device(mfd_sim* sim, int comp, int rhs, const double* dev, void* stream) {
    if (!sim || !dev) return fail(MFD_ERR_ARG, "NULL argument");
    if (rhs != 0) return fail(MFD_ERR_ARG, "rhs out of range");
    mfd_ctx* ctx = sim->ctx;
    MFD_CUDA(cudaSetDevice(ctx->device));
    MFD_TRY(order_streams((cudaStream_t)stream, ctx->stream));  // the values are ready on the caller's stream
    MFD_TRY(scatter_field(sim, comp, dev));
    return order_streams(ctx->stream, (cudaStream_t)stream);    // the caller may reuse dev after this
}

mfd_status mfd_get_field_device(mfd_sim* sim, int comp, int rhs, double* dev, void* stream) {
    if (!sim || !dev) return fail(MFD_ERR_ARG, "NULL argument");
    if (rhs != 0) return fail(MFD_ERR_ARG, "rhs out of range");
    mfd_ctx* ctx = sim->ctx;
    MFD_CUDA(cudaSetDevice(ctx->device));
    MFD_TRY(order_streams((cudaStream_t)stream, ctx->stream));  // the caller is done with dev
    MFD_TRY(gather_field(sim, comp, dev, nullptr));
    return order_streams(ctx->stream, (cudaStream_t)stream);
}

mfd_status mfd_set_sources(mfd_sim* sim, int count, const int64_t* node, const int32_t* rhs, const double* amp,
                           const double* f0, const double* t0) {
    if (!sim || count < 0) return fail(MFD_ERR_ARG, "bad arguments");
    if (count > 0 && (!node || !amp || !f0 || !t0)) return fail(MFD_ERR_ARG, "NULL source arrays");
    mfd_ctx* ctx = sim->ctx;
    MFD_CUDA(cudaSetDevice(ctx->device));
    std::vector<int64_t> dev_node(count);
    for (int s = 0; s < count; ++s) {
        if (node[s] < 0 || node[s] >= sim->ne) return fail(MFD_ERR_ARG, "source node out of range");
        if (rhs && rhs[s] != 0) return fail(MFD_ERR_ARG, "source rhs out of range");
        if (!(f0[s] > 0)) return fail(MFD_ERR_ARG, "source frequency must be > 0");
        dev_node[s] = sim->eset->h_inv[node[s]];
    }
    // the arrays are replaced one by one: until all are in place the
    // simulation has no sources and no graph that points at the old arrays
    sim->nsrc = 0;
    sim->graph_ok = false;
    MFD_TRY(upload(ctx, sim->src_node, dev_node.data(), count * 8));
    MFD_TRY(upload(ctx, sim->src_amp, amp, count * 8));
    MFD_TRY(upload(ctx, sim->src_f0, f0, count * 8));
    MFD_TRY(upload(ctx, sim->src_t0, t0, count * 8));
    sim->nsrc = count;
    sim->graph_ok = false;
    MFD_CUDA(cudaStreamSynchronize(ctx->stream));
    return MFD_OK;
}

mfd_status mfd_set_probes(mfd_sim* sim, int count, const int64_t* node, int64_t capacity) {
    if (!sim || count < 0 || capacity < 0) return fail(MFD_ERR_ARG, "bad arguments");
    if (count > 0 && !node) return fail(MFD_ERR_ARG, "NULL probe array");
    mfd_ctx* ctx = sim->ctx;
    MFD_CUDA(cudaSetDevice(ctx->device));
    std::vector<int64_t> dev_node(count);
    for (int p = 0; p < count; ++p) {
        if (node[p] < 0 || node[p] >= sim->ne) return fail(MFD_ERR_ARG, "probe node out of range");
        dev_node[p] = sim->eset->h_inv[node[p]];
    }
    // as in mfd_set_sources: no probes and no graph until both arrays are in place;
    // arrays large enough for the new probes are kept (no allocation, no device-wide
    // synchronisation by cudaFree)
    sim->nprobe = 0;
    sim->probe_cap = 0;
    sim->graph_ok = false;
    const size_t node_bytes = (size_t)std::max(1, count) * 8;
    const size_t buf_bytes = (size_t)std::max<int64_t>(1, capacity * count) * sim->rs;
    if (sim->probe_node.bytes < node_bytes) MFD_TRY(sim->probe_node.alloc(node_bytes));
    if (count > 0)
        MFD_CUDA(cudaMemcpyAsync(sim->probe_node.p, dev_node.data(), (size_t)count * 8, cudaMemcpyHostToDevice,
                                 ctx->stream));
    if (sim->probe_buf.bytes < buf_bytes) MFD_TRY(sim->probe_buf.alloc(buf_bytes));
    sim->nprobe = count;
    sim->probe_cap = capacity;
    sim->probe_from = sim->steps;
    int64_t from = sim->steps;
    MFD_CUDA(cudaMemcpyAsync(sim->pstep0.p, &from, 8, cudaMemcpyHostToDevice, ctx->stream));
    sim->graph_ok = false;
    MFD_CUDA(cudaStreamSynchronize(ctx->stream));
    return MFD_OK;
}

mfd_status mfd_set_probe_component(mfd_sim* sim, int comp) {
    if (!sim) return fail(MFD_ERR_ARG, "NULL argument");
    const bool ok = comp == MFD_EZ || (sim->layout == COLLOC2D && (comp == MFD_HX || comp == MFD_HY)) ||
                    (sim->layout == COLLOC3D && comp >= MFD_EX && comp <= MFD_HZ);
    if (!ok) return fail(MFD_ERR_ARG, "probed component: Ez, or a component of the collocated layouts");
    sim->probe_comp = comp;
    sim->graph_ok = false;
    return MFD_OK;
}

static mfd_status step_plain(mfd_sim* sim, int64_t nsteps) {
    if (!sim || nsteps < 0) return fail(MFD_ERR_ARG, "bad arguments");
    MFD_CUDA(cudaSetDevice(sim->ctx->device));
    int64_t left = nsteps;
    if (left >= 2 * GRAPH_STEPS) {
        if (sim->parity) {
            MFD_CUDA(enqueue_step(sim, nullptr));
            --left;
        }
        MFD_TRY(ensure_graph(sim));
        while (left >= GRAPH_STEPS) {
            MFD_CUDA(cudaGraphLaunch(sim->graph, sim->ctx->stream));
            sim->steps += GRAPH_STEPS;
            left -= GRAPH_STEPS;
        }
    }
    while (left > 0) {
        MFD_CUDA(enqueue_step(sim, nullptr));
        --left;
    }
    return bounds_status(sim->ctx->stream);
}

mfd_status mfd_step(mfd_sim* sim, int64_t nsteps) {
    if (!sim || nsteps < 0) return fail(MFD_ERR_ARG, "bad arguments");
    if (sim->watch_every <= 0) return step_plain(sim, nsteps);
    for (int64_t done = 0; done < nsteps;) {
        const int64_t k = std::min(sim->watch_every, nsteps - done);
        MFD_TRY(step_plain(sim, k));
        done += k;
        double u = 0;
        MFD_TRY(mfd_energy(sim, &u));
        if (!(u == u) || !(u <= sim->watch_ratio * sim->watch_u0))
            return fail(MFD_ERR_UNSTABLE, "energy watchdog: U = " + std::to_string(u) + " after step " +
                                              std::to_string(sim->steps) + " exceeds " +
                                              std::to_string(sim->watch_ratio) + " x U0 = " +
                                              std::to_string(sim->watch_u0) + " (or is NaN)");
    }
    return MFD_OK;
}

mfd_status mfd_set_watchdog(mfd_sim* sim, int64_t every, double max_ratio) {
    if (!sim || every < 0 || (every > 0 && !(max_ratio > 0))) return fail(MFD_ERR_ARG, "bad arguments");
    sim->watch_every = every;
    sim->watch_ratio = max_ratio;
    if (every > 0) {
        double u = 0;
        MFD_TRY(mfd_energy(sim, &u));
        if (!(u > 0)) return fail(MFD_ERR_STATE, "energy watchdog needs nonzero fields (set them first)");
        sim->watch_u0 = u;
    }
    return MFD_OK;
}

mfd_status mfd_step_timed(mfd_sim* sim, int64_t nsteps, double* ms) {
    if (!sim || nsteps < 0 || !ms) return fail(MFD_ERR_ARG, "bad arguments");
    MFD_CUDA(cudaSetDevice(sim->ctx->device));
    const size_t need = (size_t)nsteps * 3;
    while (sim->events.size() < need) {
        cudaEvent_t e;
        MFD_CUDA(cudaEventCreate(&e));
        sim->events.push_back(e);
    }
    for (int64_t k = 0; k < nsteps; ++k) MFD_CUDA(enqueue_step(sim, &sim->events[3 * k]));
    MFD_CUDA(cudaStreamSynchronize(sim->ctx->stream));
    double h = 0, e = 0;
    for (int64_t k = 0; k < nsteps; ++k) {
        float a = 0, b = 0;
        MFD_CUDA(cudaEventElapsedTime(&a, sim->events[3 * k], sim->events[3 * k + 1]));
        MFD_CUDA(cudaEventElapsedTime(&b, sim->events[3 * k + 1], sim->events[3 * k + 2]));
        h += a;
        e += b;
    }
    ms[0] = h;
    ms[1] = e;
    return bounds_status(sim->ctx->stream);
}

mfd_status mfd_read_probes(mfd_sim* sim, double* host, int64_t* steps) {
    if (!sim) return fail(MFD_ERR_ARG, "sim is NULL");
    mfd_ctx* ctx = sim->ctx;
    MFD_CUDA(cudaSetDevice(ctx->device));
    int64_t rec = std::min(sim->steps - sim->probe_from, sim->probe_cap);
    if (rec < 0) rec = 0;
    if (steps) *steps = rec;
    if (!host || rec == 0 || sim->nprobe == 0) {
        MFD_CUDA(cudaStreamSynchronize(ctx->stream));
        return MFD_OK;
    }
    const int64_t count = rec * sim->nprobe;
    if (sim->fp64) {
        MFD_CUDA(cudaMemcpyAsync(host, sim->probe_buf.p, count * 8, cudaMemcpyDeviceToHost, ctx->stream));
        MFD_CUDA(cudaStreamSynchronize(ctx->stream));
    } else {
        std::vector<float> tmp(count);
        MFD_CUDA(cudaMemcpyAsync(tmp.data(), sim->probe_buf.p, count * 4, cudaMemcpyDeviceToHost, ctx->stream));
        MFD_CUDA(cudaStreamSynchronize(ctx->stream));
        for (int64_t i = 0; i < count; ++i) host[i] = tmp[i];
    }
    return MFD_OK;
}

mfd_status mfd_sim_dispersion(mfd_sim* sim, int stride, int nt, double h_line, double c_ref, int jmax,
                              double* spectrum, int32_t* kidx, double* c, double* err_l1) {
    if (!sim || stride < 1) return fail(MFD_ERR_ARG, "mfd_sim_dispersion: NULL sim or stride < 1");
    const int nx = sim->nprobe;
    MFD_TRY(dispersion_check(nx, nt, h_line, stride * sim->d.dt, jmax));
    const int64_t rec = std::min(sim->steps - sim->probe_from, sim->probe_cap);
    if (rec < (int64_t)nt * stride)
        return fail(MFD_ERR_STATE, "mfd_sim_dispersion: fewer recorded steps than nt * stride");
    mfd_ctx* ctx = sim->ctx;
    MFD_CUDA(cudaSetDevice(ctx->device));
    DevBuf s;
    MFD_TRY(s.alloc((size_t)nx * nt * 8));
    const unsigned g = (unsigned)(((int64_t)nx * nt + 255) / 256);
    if (sim->fp64)
        k_probe_samples<double><<<g, 256, 0, ctx->stream>>>(sim->probe_buf.as<double>(), nx, stride, nt, s.as<double>());
    else
        k_probe_samples<float><<<g, 256, 0, ctx->stream>>>(sim->probe_buf.as<float>(), nx, stride, nt, s.as<double>());
    MFD_CUDA(cudaGetLastError());
    return dispersion_run(ctx, nx, nt, s.as<double>(), h_line, stride * sim->d.dt, c_ref, jmax, spectrum, kidx, c,
                          err_l1);
}

mfd_status mfd_energy(mfd_sim* sim, double* u) {
    if (!sim || !u) return fail(MFD_ERR_ARG, "NULL argument");
    mfd_ctx* ctx = sim->ctx;
    MFD_CUDA(cudaSetDevice(ctx->device));
    const double eta2 = sim->d.mu0 / sim->d.eps0;
    const int64_t nmax = std::max(sim->ne, sim->nh);
    const unsigned grid = (unsigned)((nmax + 255) / 256);
    if (sim->layout == COLLOC3D) {
        MFD_CUDA(launch_energy_3d(make3d(sim, sim->parity), sim->eps.as<double>(), eta2, sim->partial.as<double>(), grid,
                                  ctx->stream));
    } else {
        MFD_CUDA(launch_energy_2d(make2d(sim, sim->parity), sim->eps.as<double>(), sim->ne, eta2,
                                  sim->partial.as<double>(), grid, ctx->stream));
    }
    k_sum<<<1, 256, 0, ctx->stream>>>(sim->partial.as<double>(), (int)grid, sim->energy_out.as<double>());
    MFD_CUDA(cudaGetLastError());
    MFD_CUDA(cudaMemcpyAsync(u, sim->energy_out.p, 8, cudaMemcpyDeviceToHost, ctx->stream));
    MFD_CUDA(cudaStreamSynchronize(ctx->stream));
    return bounds_status(ctx->stream);
}

int64_t mfd_sim_steps(const mfd_sim* sim) { return sim ? sim->steps : -1; }

// checkpoint / resume: the device field buffers as they are (bit-exact), the
// step index and ping-pong parity, and the probe records so far
static void sim_state_layout(const mfd_sim* sim, StateHead* h, DevBuf* const* bufs) {
    state_head_init(h, 1);
    h->layout = (int32_t)sim->layout;
    h->fp64 = sim->fp64 ? 1 : 0;
    h->ne = sim->ne;
    h->nh = sim->nh;
    h->nrhs = 1;
    h->steps = sim->steps;
    h->probe_from = sim->probe_from;
    h->parity = sim->parity;
    h->nprobe = sim->nprobe;
    int64_t rec = std::min(sim->steps - sim->probe_from, sim->probe_cap);
    h->rec = sim->nprobe > 0 && rec > 0 ? rec : 0;
    for (int b = 0; b < 6; ++b) h->bytes[b] = bufs[b]->p ? (int64_t)bufs[b]->bytes : 0;
}

static size_t state_total(const StateHead& h, size_t rs) {
    size_t t = sizeof(StateHead) + (size_t)h.rec * h.nprobe * rs;
    for (int b = 0; b < 6; ++b) t += (size_t)h.bytes[b];
    return t;
}

mfd_status mfd_sim_state_size(const mfd_sim* sim, size_t* bytes) {
    if (!sim || !bytes) return fail(MFD_ERR_ARG, "NULL argument");
    mfd_sim* m = const_cast<mfd_sim*>(sim);
    DevBuf* bufs[6] = {&m->s0, &m->s1, &m->s2, &m->s3, &m->s4, &m->s5};
    StateHead h;
    sim_state_layout(sim, &h, bufs);
    *bytes = state_total(h, sim->rs);
    return MFD_OK;
}

mfd_status mfd_sim_save_state(mfd_sim* sim, void* host, size_t bytes) {
    if (!sim || !host) return fail(MFD_ERR_ARG, "NULL argument");
    DevBuf* bufs[6] = {&sim->s0, &sim->s1, &sim->s2, &sim->s3, &sim->s4, &sim->s5};
    StateHead h;
    sim_state_layout(sim, &h, bufs);
    if (bytes < state_total(h, sim->rs)) return fail(MFD_ERR_ARG, "state buffer smaller than mfd_sim_state_size");
    mfd_ctx* ctx = sim->ctx;
    MFD_CUDA(cudaSetDevice(ctx->device));
    char* o = static_cast<char*>(host);
    std::memcpy(o, &h, sizeof(h));
    o += sizeof(h);
    for (int b = 0; b < 6; ++b) {
        if (!h.bytes[b]) continue;
        MFD_CUDA(cudaMemcpyAsync(o, bufs[b]->p, (size_t)h.bytes[b], cudaMemcpyDeviceToHost, ctx->stream));
        o += h.bytes[b];
    }
    if (h.rec)
        MFD_CUDA(cudaMemcpyAsync(o, sim->probe_buf.p, (size_t)h.rec * h.nprobe * sim->rs, cudaMemcpyDeviceToHost,
                                 ctx->stream));
    MFD_CUDA(cudaStreamSynchronize(ctx->stream));
    return MFD_OK;
}

mfd_status mfd_sim_load_state(mfd_sim* sim, const void* host, size_t bytes) {
    if (!sim || !host) return fail(MFD_ERR_ARG, "NULL argument");
    StateHead in, mine;
    MFD_TRY(state_head_check(host, bytes, 1, &in));
    DevBuf* bufs[6] = {&sim->s0, &sim->s1, &sim->s2, &sim->s3, &sim->s4, &sim->s5};
    sim_state_layout(sim, &mine, bufs);
    if (in.layout != mine.layout || in.fp64 != mine.fp64 || in.ne != mine.ne || in.nh != mine.nh)
        return fail(MFD_ERR_ARG, "state blob of another layout, precision or node count");
    for (int b = 0; b < 6; ++b)
        if (in.bytes[b] != mine.bytes[b]) return fail(MFD_ERR_ARG, "state blob buffers differ from this simulation");
    if (in.rec > 0 && (in.nprobe != sim->nprobe || in.rec > sim->probe_cap))
        return fail(MFD_ERR_ARG, "state blob probe records need the same probes with enough capacity");
    if (bytes < state_total(in, sim->rs)) return fail(MFD_ERR_ARG, "state blob truncated");
    mfd_ctx* ctx = sim->ctx;
    MFD_CUDA(cudaSetDevice(ctx->device));
    const char* o = static_cast<const char*>(host) + sizeof(in);
    for (int b = 0; b < 6; ++b) {
        if (!in.bytes[b]) continue;
        MFD_CUDA(cudaMemcpyAsync(bufs[b]->p, o, (size_t)in.bytes[b], cudaMemcpyHostToDevice, ctx->stream));
        o += in.bytes[b];
    }
    if (in.rec)
        MFD_CUDA(cudaMemcpyAsync(sim->probe_buf.p, o, (size_t)in.rec * in.nprobe * sim->rs, cudaMemcpyHostToDevice,
                                 ctx->stream));
    sim->steps = in.steps;
    sim->parity = in.parity;
    sim->probe_from = in.rec > 0 ? in.probe_from : in.steps;
    const int64_t words[2] = {sim->steps, sim->probe_from};
    MFD_CUDA(cudaMemcpyAsync(sim->counter.p, &words[0], 8, cudaMemcpyHostToDevice, ctx->stream));
    MFD_CUDA(cudaMemcpyAsync(sim->pstep0.p, &words[1], 8, cudaMemcpyHostToDevice, ctx->stream));
    MFD_CUDA(cudaStreamSynchronize(ctx->stream));
    sim->graph_ok = false;
    return MFD_OK;
}

static bool block_ok(int b) { return b == 64 || b == 128 || b == 256 || b == 512; }

mfd_status mfd_sim_set_lanes(mfd_sim* sim, int lanes_h, int lanes_e) {
    if (!sim) return fail(MFD_ERR_ARG, "NULL argument");
    auto ok = [](int l) { return l == 1 || l == 2 || l == 4; };
    if (!ok(lanes_h) || !ok(lanes_e)) return fail(MFD_ERR_ARG, "lanes per node: 1, 2 or 4");
    if (sim->layout != COLLOC2D || sim->hp.idx_v.p != nullptr)
        return fail(MFD_ERR_ARG, "lanes per node apply to the collocated 2D layout with one index row per node");
    sim->lanes[0] = lanes_h;
    sim->lanes[1] = lanes_e;
    sim->graph_ok = false;
    return MFD_OK;
}

mfd_status mfd_sim_launch_config(const mfd_sim* sim, int* block, int* lanes) {
    if (!sim) return fail(MFD_ERR_ARG, "NULL argument");
    const Launch2D L = sim->layout == COLLOC3D ? Launch2D{} : make2d(const_cast<mfd_sim*>(sim), sim->parity);
    for (int p = 0; p < 2; ++p) {
        if (block) block[p] = sim->block[p];
        if (lanes) lanes[p] = sim->layout == COLLOC2D ? L.lanes[p] : 1;
    }
    return MFD_OK;
}

mfd_status mfd_sim_set_blocks(mfd_sim* sim, int block_h, int block_e) {
    if (!sim || !block_ok(block_h) || !block_ok(block_e)) return fail(MFD_ERR_ARG, "block sizes: 64, 128, 256 or 512");
    sim->block[0] = block_h;
    sim->block[1] = block_e;
    sim->graph_ok = false;
    return MFD_OK;
}

mfd_status mfd_sim_set_index_format(mfd_sim* sim, int format) {
    if (!sim || (format != MFD_INDEX_Q16 && format != MFD_INDEX_I32)) return fail(MFD_ERR_ARG, "bad arguments");
    sim->q16 = format == MFD_INDEX_Q16;
    sim->graph_ok = false;
    return MFD_OK;
}

mfd_status mfd_sim_set_l2_keep(mfd_sim* sim, double keep) {
    if (!sim || !(keep <= 1.0) || std::isnan(keep)) return fail(MFD_ERR_ARG, "keep must be <= 1 (negative: automatic)");
    sim->l2_keep_set = keep < 0 ? -1.0 : keep;
    sim->graph_ok = false;  // the fraction is a kernel argument of the captured steps
    return MFD_OK;
}

double mfd_sim_l2_keep(const mfd_sim* sim) { return sim ? (double)sim_keep(sim) : -1.0; }

mfd_status mfd_sim_index_stats(const mfd_sim* sim, int64_t* out) {
    if (!sim || !out) return fail(MFD_ERR_ARG, "NULL argument");
    const PackedStencil* ps[2] = {&sim->hp, &sim->ep};
    for (int p = 0; p < 2; ++p) {
        const PackedStencil& k = *ps[p];
        const bool has = sim->layout == STAG2D && k.q_c.p != nullptr;
        out[3 * p] = has ? (k.n + 31) / 32 : 0;
        out[3 * p + 1] = has ? k.wide_c : 0;
        out[3 * p + 2] = has ? k.wide_v : 0;
    }
    return MFD_OK;
}

mfd_status mfd_sim_autotune(mfd_sim* sim, int reps, int* chosen) {
    if (!sim || reps < 1) return fail(MFD_ERR_ARG, "bad arguments");
    mfd_ctx* ctx = sim->ctx;
    MFD_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    // the timed launches overwrite state buffers: keep a copy and put it back
    DevBuf* bufs[5] = {&sim->s0, &sim->s1, &sim->s2, &sim->s3, &sim->s4};
    DevBuf save[5];
    for (int b = 0; b < 5; ++b)
        if (bufs[b]->p) {
            MFD_TRY(save[b].alloc(bufs[b]->bytes));
            MFD_CUDA(cudaMemcpyAsync(save[b].p, bufs[b]->p, bufs[b]->bytes, cudaMemcpyDeviceToDevice, s));
        }
    cudaEvent_t e0, e1;
    MFD_CUDA(cudaEventCreate(&e0));
    MFD_CUDA(cudaEventCreate(&e1));
    // candidates: threads per block, and (collocated 2D rows shared by both
    // stencils) lanes per node; the sums of a node are split over its lanes, so
    // a choice changes the summation order, not the stencils
    constexpr int NB = 4;
    const int cand[NB] = {64, 128, 256, 512};
    const bool lanes_tuned = sim->layout == COLLOC2D && sim->hp.idx_v.p == nullptr;
    const int lcand[3] = {1, 2, 4};
    const int nl = lanes_tuned ? 3 : 1;
    const Launch2D L0 = sim->layout == COLLOC3D ? Launch2D{} : make2d(sim, sim->parity);
    int best[2] = {sim->block[0], sim->block[1]};
    int bestl[2] = {L0.lanes[0], L0.lanes[1]};
    mfd_status st = MFD_OK;
    for (int pass = 0; pass < 2 && st == MFD_OK; ++pass) {
        float tbest = 1e30f;
        for (int c = 0; c < NB * nl && st == MFD_OK; ++c) {
            int blk[2] = {best[0], best[1]};
            int lan[2] = {bestl[0], bestl[1]};
            blk[pass] = cand[c % NB];
            if (lanes_tuned) lan[pass] = lcand[c / NB];
            cudaError_t e = cudaSuccess;
            auto launch = [&]() {
                if (sim->layout == COLLOC3D) {
                    Launch3D L = make3d(sim, sim->parity);
                    L.block[0] = blk[0];
                    L.block[1] = blk[1];
                    return launch_3d(L, pass, s);
                }
                Launch2D L = make2d(sim, sim->parity);
                L.block[0] = blk[0];
                L.block[1] = blk[1];
                if (lanes_tuned) {
                    L.lanes[0] = lan[0];
                    L.lanes[1] = lan[1];
                }
                return launch_2d(L, pass, s);
            };
            e = launch();
            cudaEventRecord(e0, s);
            for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch();
            cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                st = fail(MFD_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
                break;
            }
            if (ms < tbest) {
                tbest = ms;
                best[pass] = blk[pass];
                bestl[pass] = lan[pass];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int b = 0; b < 5; ++b)
        if (bufs[b]->p) cudaMemcpyAsync(bufs[b]->p, save[b].p, bufs[b]->bytes, cudaMemcpyDeviceToDevice, s);
    MFD_CUDA(cudaStreamSynchronize(s));
    if (st != MFD_OK) return st;
    sim->block[0] = best[0];
    sim->block[1] = best[1];
    if (lanes_tuned) {
        sim->lanes[0] = bestl[0];
        sim->lanes[1] = bestl[1];
    }
    sim->graph_ok = false;
    if (chosen) {
        chosen[0] = best[0];
        chosen[1] = best[1];
    }
    return MFD_OK;
}

}  // extern "C"

// The gradient of the probe objective in two halves (mfd_grad_forward records,
// mfd_grad_backward sweeps); mfd_grad runs both.
struct mfd_tape {
    mfd_sim* sim = nullptr;
    int64_t nsteps = 0, G = 0, nseg = 0, start = 0, end = 0;
    bool whole = false, used = false;
    size_t sbytes = 0;
    double J = 0;
    DevBuf ckpt, fin, hist, Jd;
    std::vector<int64_t> starts, slots;  // host sources of async copies: valid while the tape lives
};

namespace {

template <typename Body>
mfd_status capture_graph(mfd_sim* sim, cudaStream_t s, Body&& body, cudaGraphExec_t* out) {
    const int64_t steps0 = sim->steps;
    MFD_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = body();
    cudaGraph_t gr = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s, &gr);
    sim->steps = steps0;  // the captured steps have not run
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (gr) cudaGraphDestroy(gr);
        cudaGetLastError();
        return fail(MFD_ERR_CUDA, std::string("gradient graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(out, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) return fail(MFD_ERR_CUDA, std::string("gradient graph instantiate: ") + cudaGetErrorString(e));
    return MFD_OK;
}

struct GraphGuard {
    cudaGraphExec_t g = nullptr;
    ~GraphGuard() {
        if (g) cudaGraphExecDestroy(g);
    }
};

__global__ void k_to_caller(const double* __restrict__ v, const int64_t* __restrict__ perm, int64_t n,
                            double* __restrict__ out) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < n) out[perm[k]] = v[k];
}

__global__ void k_count_nonpositive(const double* __restrict__ v, int64_t n, unsigned long long* __restrict__ bad) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < n && !(v[k] > 0.0)) atomicAdd(bad, 1ull);
}

}  // namespace

extern "C" {

mfd_status mfd_grad_forward(mfd_sim* sim, int64_t nsteps, int64_t every, double* J, mfd_tape** out) {
    if (!sim || nsteps < 1 || every < 0 || !J || !out) return fail(MFD_ERR_ARG, "bad arguments");
    *out = nullptr;
    if (sim->layout != COLLOC2D) return fail(MFD_ERR_ARG, "the gradient supports the collocated 2D layout");
    if (sim->hp.mirror) return fail(MFD_ERR_ARG, "the gradient does not support mirror walls (images)");
    if (sim->probe_comp != MFD_EZ) return fail(MFD_ERR_ARG, "the gradient's objective is over Ez probes");
    if (sim->nprobe < 1 || sim->probe_cap < nsteps)
        return fail(MFD_ERR_STATE, "the gradient needs probes with capacity >= nsteps (mfd_set_probes)");
    mfd_ctx* ctx = sim->ctx;
    MFD_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    const bool f64 = sim->fp64;
    const size_t rs = sim->rs;
    const int64_t n = sim->ne;
    if (!sim->adj_ok) {
        MFD_TRY(adj_build(ctx, sim->d.h_curl, sim->d.h_hv, f64, sim->adj));
        sim->adj_ok = true;
    }
    mfd_tape* tp = new (std::nothrow) mfd_tape();
    if (!tp) return fail(MFD_ERR_OOM, "host allocation failed");
    std::unique_ptr<mfd_tape> guard(tp);
    mfd_tape& T = *tp;
    T.sim = sim;
    T.nsteps = nsteps;
    // The step is linear in the fields, so the adjoint needs the forward run only
    // through Ez of every level (the permittivity gradient). With every == 0 that
    // history is kept whole when it fits in a quarter of the free device memory
    // and nothing is recomputed; otherwise (every >= 1, or no room) the full state
    // is checkpointed every `every` (64) steps and each segment is recomputed from
    // its checkpoint in the backward sweep.
    size_t free_b = 0, total_b = 0;
    MFD_CUDA(cudaMemGetInfo(&free_b, &total_b));
    T.whole = every == 0 && (size_t)(nsteps + 1) * n * rs <= free_b / 4;
    if (every == 0) every = 64;
    T.G = T.whole ? 64 : every;  // steps per captured segment
    T.nseg = (nsteps + T.G - 1) / T.G;
    T.sbytes = (size_t)n * 4 * rs;
    if (!T.whole) {
        MFD_TRY(T.ckpt.alloc((size_t)T.nseg * T.sbytes));
        MFD_TRY(T.fin.alloc(T.sbytes));
    }
    MFD_TRY(T.hist.alloc((size_t)((T.whole ? nsteps : every) + 1) * n * rs));
    MFD_TRY(T.Jd.alloc(8));
    const int64_t start = sim->steps;
    T.start = start;
    T.end = start + nsteps;
    // probes record from the first step of this call
    sim->probe_from = start;
    MFD_CUDA(cudaMemcpyAsync(sim->pstep0.p, &T.start, 8, cudaMemcpyHostToDevice, s));
    MFD_CUDA(cudaMemcpyAsync(sim->counter.p, &T.start, 8, cudaMemcpyHostToDevice, s));
    T.starts.resize(T.nseg);
    T.slots.resize(T.nseg);
    for (int64_t g = 0; g < T.nseg; ++g) {
        T.starts[g] = start + g * T.G;
        T.slots[g] = T.whole ? g * T.G : 0;
    }
    if (T.whole) {
        // every step also writes its Ez level into the history (level = counter - start)
        MFD_CUDA(copy_ez(f64, sim->s0.p, T.hist.p, n, s));
        auto fwd = [&](int64_t len) -> cudaError_t {
            cudaError_t e = cudaSuccess;
            for (int64_t k = 0; k < len && e == cudaSuccess; ++k) {
                e = enqueue_step(sim, nullptr);
                if (e == cudaSuccess)
                    e = copy_ez_level(f64, sim->s0.p, T.hist.p, n, sim->counter.as<int64_t>(), start, s);
            }
            return e;
        };
        GraphGuard gfwd;
        for (int64_t g = 0; g < T.nseg; ++g) {
            const int64_t len = std::min(T.G, nsteps - g * T.G);
            if (len == T.G && T.nseg >= 2) {
                if (!gfwd.g) MFD_TRY(capture_graph(sim, s, [&] { return fwd(len); }, &gfwd.g));
                MFD_CUDA(cudaGraphLaunch(gfwd.g, s));
                sim->steps += len;
            } else {
                MFD_CUDA(fwd(len));
            }
        }
    } else {
        // a checkpoint of the full state at the start of every segment
        for (int64_t g = 0; g < T.nseg; ++g) {
            MFD_CUDA(cudaMemcpyAsync((char*)T.ckpt.p + g * T.sbytes, sim->s0.p, T.sbytes, cudaMemcpyDeviceToDevice, s));
            MFD_TRY(mfd_step(sim, std::min(T.G, nsteps - g * T.G)));
        }
        MFD_CUDA(cudaMemcpyAsync(T.fin.p, sim->s0.p, T.sbytes, cudaMemcpyDeviceToDevice, s));
    }
    MFD_CUDA(probe_energy(f64, sim->probe_buf.p, nsteps * sim->nprobe, sim->d.dt, T.Jd.as<double>(), s));
    MFD_CUDA(cudaMemcpyAsync(&T.J, T.Jd.p, 8, cudaMemcpyDeviceToHost, s));
    MFD_CUDA(cudaStreamSynchronize(s));
    *J = T.J;
    MFD_TRY(bounds_status(s));
    *out = guard.release();
    return MFD_OK;
}

mfd_status mfd_grad_backward(mfd_tape* tape, double* g_eps, double* g_amp, int on_device, void* stream) {
    if (!tape || !g_eps) return fail(MFD_ERR_ARG, "bad arguments");
    mfd_tape& T = *tape;
    mfd_sim* sim = T.sim;
    if (T.used) return fail(MFD_ERR_STATE, "this tape's adjoint sweep has run already");
    if (sim->nsrc > 0 && !g_amp) return fail(MFD_ERR_ARG, "g_amp is NULL");
    if (sim->steps != T.end)
        return fail(MFD_ERR_STATE, "the simulation was stepped or reset after mfd_grad_forward");
    mfd_ctx* ctx = sim->ctx;
    MFD_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    const bool f64 = sim->fp64;
    const size_t rs = sim->rs;
    const int64_t n = sim->ne;
    const int64_t nsteps = T.nsteps, start = T.start, G = T.G, nseg = T.nseg;
    const bool whole = T.whole;
    const size_t sbytes = T.sbytes;
    if (on_device) MFD_TRY(order_streams((cudaStream_t)stream, s));  // the caller is done with the outputs
    DevBuf LA, LB, geps, gamp, seg0, slot0, gcall;
    MFD_TRY(LA.alloc(sbytes));
    MFD_TRY(LB.alloc(sbytes));
    MFD_TRY(geps.alloc((size_t)n * 8));
    MFD_TRY(gamp.alloc(std::max(1, sim->nsrc) * 8));
    MFD_TRY(seg0.alloc(8));
    MFD_TRY(slot0.alloc(8));
    MFD_CUDA(cudaMemsetAsync(geps.p, 0, geps.bytes, s));
    MFD_CUDA(cudaMemsetAsync(gamp.p, 0, gamp.bytes, s));
    DevBuf& hist = T.hist;
    // lambda^N: dJ/dE^N at the probes, zero elsewhere
    MFD_CUDA(init_lambda(f64, LA.p, sim->s0.p, n, s));
    // Ez^N: the last level of the whole history, or staged in level 0 of the segment buffer
    void* ezN = whole ? (char*)hist.p + (size_t)nsteps * n * rs : hist.p;
    if (!whole) MFD_CUDA(copy_ez(f64, sim->s0.p, ezN, n, s));
    MFD_CUDA(adj_probe_term(f64, LA.p, ezN, sim->probe_node.as<int64_t>(), sim->nprobe, sim->d.dt, s));
    AdjArgs a;
    a.fp64 = f64;
    a.off = sim->adj.off.as<int64_t>();
    a.scol = sim->adj.scol.as<int4>();
    a.sx = sim->adj.sx.p;
    a.sy = sim->adj.sy.p;
    a.sv = sim->adj.sv.p;
    a.n = n;
    a.LA = LA.p;
    a.LB = LB.p;
    a.ch = sim->d.dt / sim->d.mu0;
    a.gamma = sim->d.gamma;
    a.eps = sim->eps.as<double>();
    a.g_eps = geps.as<double>();
    a.ez = hist.p;
    a.slot0 = slot0.as<int64_t>();
    // both transposed passes of a backward step read the same streams
    a.l2_keep = sim->l2_keep_set >= 0
                    ? (float)sim->l2_keep_set
                    : keep_for((int64_t)(sim->adj.scol.bytes + sim->adj.sx.bytes + sim->adj.sy.bytes + sim->adj.sv.bytes),
                               sim->ctx->l2_bytes);
    // the per-step source and probe terms, fused into the passes: node bits and node-sorted lists
    AdjTerms terms;
    DevBuf d_smask, d_pmask, d_snode, d_sidx, d_pnode;
    {
        const int64_t words = (n + 31) / 32;
        std::vector<int64_t> hs(sim->nsrc), hp(sim->nprobe);
        MFD_CUDA(cudaStreamSynchronize(s));
        if (sim->nsrc) MFD_CUDA(cudaMemcpy(hs.data(), sim->src_node.p, sim->nsrc * 8, cudaMemcpyDeviceToHost));
        MFD_CUDA(cudaMemcpy(hp.data(), sim->probe_node.p, sim->nprobe * 8, cudaMemcpyDeviceToHost));
        std::vector<int> order(sim->nsrc);
        for (int k = 0; k < sim->nsrc; ++k) order[k] = k;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return hs[x] < hs[y]; });
        std::vector<int64_t> sn(sim->nsrc);
        std::vector<uint32_t> sm(words, 0u), pm(words, 0u);
        for (int q = 0; q < sim->nsrc; ++q) {
            sn[q] = hs[order[q]];
            sm[sn[q] >> 5] |= 1u << (sn[q] & 31);
        }
        std::sort(hp.begin(), hp.end());
        for (int64_t v : hp) pm[v >> 5] |= 1u << (v & 31);
        MFD_TRY(upload_host(d_smask, sm));
        MFD_TRY(upload_host(d_pmask, pm));
        MFD_TRY(upload_host(d_snode, sn));
        MFD_TRY(upload_host(d_sidx, order));
        MFD_TRY(upload_host(d_pnode, hp));
        terms.smask = sim->nsrc ? d_smask.as<uint32_t>() : nullptr;
        terms.snode = d_snode.as<int64_t>();
        terms.sidx = d_sidx.as<int>();
        terms.nsrc = sim->nsrc;
        terms.amp = sim->src_amp.as<double>();
        terms.f0 = sim->src_f0.as<double>();
        terms.t0 = sim->src_t0.as<double>();
        terms.g_amp = gamp.as<double>();
        terms.pmask = d_pmask.as<uint32_t>();
        terms.pnode = d_pnode.as<int64_t>();
        terms.nprobe = sim->nprobe;
        terms.seg0 = seg0.as<int64_t>();
        terms.dt = sim->d.dt;
        terms.min_step = start + 1;
    }
    a.terms = &terms;
    // ---- backward over the segments; a full segment is a captured graph replayed
    // for every full segment (the segment's first step and first level live on the
    // device: seg0, slot0)
    auto recompute = [&](int64_t len) -> cudaError_t {
        cudaError_t e = copy_ez(f64, sim->s0.p, hist.p, n, s);
        for (int64_t k = 0; k < len && e == cudaSuccess; ++k) {
            e = enqueue_step(sim, nullptr);
            if (e == cudaSuccess) e = copy_ez(f64, sim->s0.p, (char*)hist.p + (k + 1) * n * rs, n, s);
        }
        return e;
    };
    auto sweep = [&](int64_t len) -> cudaError_t {
        cudaError_t e = cudaSuccess;
        for (int64_t k = len - 1; k >= 0 && e == cudaSuccess; --k) {  // step seg0 + k -> seg0 + k + 1
            // pass 0 adds the step's source terms, pass 1 the probe terms of level seg0 + k (AdjTerms)
            AdjArgs ak = a;
            ak.k = (int)k;
            e = adj_pass(ak, 0, s);
            if (e == cudaSuccess) e = adj_pass(ak, 1, s);
        }
        return e;
    };
    T.used = true;
    GraphGuard grec, gadj;
    for (int64_t g = nseg - 1; g >= 0; --g) {
        const int64_t len = std::min(G, nsteps - g * G);
        MFD_CUDA(cudaMemcpyAsync(seg0.p, &T.starts[g], 8, cudaMemcpyHostToDevice, s));
        MFD_CUDA(cudaMemcpyAsync(slot0.p, &T.slots[g], 8, cudaMemcpyHostToDevice, s));
        const bool graphs = len == G && nseg >= 2;
        if (!whole) {
            MFD_CUDA(cudaMemcpyAsync(sim->s0.p, (char*)T.ckpt.p + g * sbytes, sbytes, cudaMemcpyDeviceToDevice, s));
            MFD_CUDA(cudaMemcpyAsync(sim->counter.p, &T.starts[g], 8, cudaMemcpyHostToDevice, s));
            sim->steps = T.starts[g];
            if (graphs) {
                if (!grec.g) MFD_TRY(capture_graph(sim, s, [&] { return recompute(len); }, &grec.g));
                MFD_CUDA(cudaGraphLaunch(grec.g, s));
            } else {
                MFD_CUDA(recompute(len));
            }
        }
        if (graphs) {
            if (!gadj.g) MFD_TRY(capture_graph(sim, s, [&] { return sweep(len); }, &gadj.g));
            MFD_CUDA(cudaGraphLaunch(gadj.g, s));
        } else {
            MFD_CUDA(sweep(len));
        }
    }
    // leave the simulation where a plain run of nsteps would
    if (!whole) MFD_CUDA(cudaMemcpyAsync(sim->s0.p, T.fin.p, sbytes, cudaMemcpyDeviceToDevice, s));
    MFD_CUDA(cudaMemcpyAsync(sim->counter.p, &T.end, 8, cudaMemcpyHostToDevice, s));
    sim->steps = T.end;
    sim->adj_sweeps += 1;
    if (on_device) {
        const unsigned gr = (unsigned)((n + 255) / 256);
        k_to_caller<<<gr, 256, 0, s>>>(geps.as<double>(), sim->eset->perm.as<int64_t>(), n, g_eps);
        MFD_CUDA(cudaGetLastError());
        if (sim->nsrc > 0) MFD_CUDA(cudaMemcpyAsync(g_amp, gamp.p, sim->nsrc * 8, cudaMemcpyDeviceToDevice, s));
        MFD_TRY(bounds_status(s));
        MFD_TRY(order_streams(s, (cudaStream_t)stream));
        // the temporaries are released at return (cudaFree waits for the queued work)
        return MFD_OK;
    }
    std::vector<double> gd(n);
    MFD_CUDA(cudaMemcpyAsync(gd.data(), geps.p, n * 8, cudaMemcpyDeviceToHost, s));
    if (sim->nsrc > 0) MFD_CUDA(cudaMemcpyAsync(g_amp, gamp.p, sim->nsrc * 8, cudaMemcpyDeviceToHost, s));
    MFD_CUDA(cudaStreamSynchronize(s));
    for (int64_t k = 0; k < n; ++k) g_eps[sim->eset->h_perm[k]] = gd[k];
    return bounds_status(s);
}

void mfd_tape_destroy(mfd_tape* tape) {
    if (!tape) return;
    cudaSetDevice(tape->sim->ctx->device);
    cudaStreamSynchronize(tape->sim->ctx->stream);
    delete tape;
}

mfd_status mfd_grad(mfd_sim* sim, int64_t nsteps, int64_t every, double* J, double* g_eps, double* g_amp) {
    if (!sim || nsteps < 1 || every < 0 || !J || !g_eps) return fail(MFD_ERR_ARG, "bad arguments");
    if (sim->nsrc > 0 && !g_amp) return fail(MFD_ERR_ARG, "g_amp is NULL");
    mfd_tape* tape = nullptr;
    MFD_TRY(mfd_grad_forward(sim, nsteps, every, J, &tape));
    const mfd_status st = mfd_grad_backward(tape, g_eps, g_amp, 0, nullptr);
    mfd_tape_destroy(tape);
    return st;
}

int64_t mfd_sim_adjoint_sweeps(const mfd_sim* sim) { return sim ? sim->adj_sweeps : -1; }

mfd_status mfd_probe_objective(mfd_sim* sim, double* J) {
    if (!sim || !J) return fail(MFD_ERR_ARG, "NULL argument");
    mfd_ctx* ctx = sim->ctx;
    MFD_CUDA(cudaSetDevice(ctx->device));
    int64_t rec = std::min(sim->steps - sim->probe_from, sim->probe_cap);
    if (rec < 0 || sim->nprobe == 0) rec = 0;
    MFD_CUDA(probe_energy(sim->fp64, sim->probe_buf.p, rec * sim->nprobe, sim->d.dt, sim->energy_out.as<double>(),
                          ctx->stream));
    MFD_CUDA(cudaMemcpyAsync(J, sim->energy_out.p, 8, cudaMemcpyDeviceToHost, ctx->stream));
    MFD_CUDA(cudaStreamSynchronize(ctx->stream));
    return MFD_OK;
}

mfd_status mfd_set_materials_device(mfd_sim* sim, const double* eps_r, const uint8_t* pec, void* stream) {
    if (!sim) return fail(MFD_ERR_ARG, "sim is NULL");
    mfd_ctx* ctx = sim->ctx;
    MFD_CUDA(cudaSetDevice(ctx->device));
    MFD_TRY(order_streams((cudaStream_t)stream, ctx->stream));  // the values are ready on the caller's stream
    const int64_t ne = sim->ne;
    const unsigned g = (unsigned)((ne + 255) / 256);
    if (eps_r) {
        DevBuf bad;
        MFD_TRY(bad.alloc(8));
        MFD_CUDA(cudaMemsetAsync(bad.p, 0, 8, ctx->stream));
        k_count_nonpositive<<<g, 256, 0, ctx->stream>>>(eps_r, ne, bad.as<unsigned long long>());
        MFD_CUDA(cudaGetLastError());
        unsigned long long nb = 0;
        MFD_CUDA(cudaMemcpyAsync(&nb, bad.p, 8, cudaMemcpyDeviceToHost, ctx->stream));
        MFD_CUDA(cudaStreamSynchronize(ctx->stream));
        if (nb) return fail(MFD_ERR_ARG, "eps_r must be > 0");
    }
    MFD_TRY(apply_materials(sim, eps_r, pec));
    return order_streams(ctx->stream, (cudaStream_t)stream);
}

mfd_status mfd_set_source_amps_device(mfd_sim* sim, const double* amp, void* stream) {
    if (!sim || (!amp && sim->nsrc > 0)) return fail(MFD_ERR_ARG, "NULL argument");
    mfd_ctx* ctx = sim->ctx;
    MFD_CUDA(cudaSetDevice(ctx->device));
    MFD_TRY(order_streams((cudaStream_t)stream, ctx->stream));
    if (sim->nsrc > 0)
        MFD_CUDA(cudaMemcpyAsync(sim->src_amp.p, amp, sim->nsrc * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    return order_streams(ctx->stream, (cudaStream_t)stream);
}

void mfd_sim_destroy(mfd_sim* sim) {
    if (!sim) return;
    mfd_ctx* ctx = sim->ctx;
    const mfd_weights* w[4] = {sim->d.h_curl, sim->d.h_hv, sim->d.e_curl, sim->d.e_hv};
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    delete sim;
    for (const mfd_weights* x : w) release(x);
    release(ctx);
}

}  // extern "C"
