// adjoint.cu -- the discrete adjoint of the collocated TMz step (Eq. 19).
//
// With K = diag(dt / (eps0 eps_r)) (0 on PEC nodes), Z = diag(1 - pec),
// curl stencil operators Dx, Dy and hyperviscosity operator V, one forward step is
//   H' = H + ch (C_E E + gamma V H),   C_E E = (-Dy E, Dx E)
//   E' = Z [E + K (gamma V E + C_H H') + b],   C_H H = Dx Hy - Dy Hx.
// Its transpose, applied to (lambda_E', lambda_H') = adjoints of (E', H'):
//   mu     = Z lambda_E'
//   l~H    = lambda_H' + C_H^T (K mu)           (x: -Dy^T K mu, y: +Dx^T K mu)
//   t      = mu + gamma V^T (K mu)
//   lambda_H = l~H + ch gamma V^T l~H
//   lambda_E = t + ch C_E^T l~H                  (-Dy^T l~Hx + Dx^T l~Hy)
// and the permittivity gradient of the step, dE'_i/deps_i = -(E'_i - E_i - b_i) / eps_i:
//   g_eps_i += mu_i (-(E'_i - E_i - b_i) / eps_i).
// Every transposed operator is a gather over the transposed (CSR) stencils.
#include <cub/device/device_scan.cuh>

#include <algorithm>

#include "adjoint.cuh"

namespace mfd {

__global__ void k_t_count(const int32_t* __restrict__ idx, int stride, int64_t n, int ne, int64_t* __restrict__ cnt) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * ne) return;
    const int64_t i = e / ne;
    const int k = (int)(e % ne);
    atomicAdd(reinterpret_cast<unsigned long long*>(cnt + idx[i * stride + k]), 1ull);
}

__global__ void k_t_pad(const int64_t* __restrict__ cnt, int64_t n, int64_t* __restrict__ padded) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    padded[j] = (cnt[j] + 3) & ~(int64_t)3;
}

// kind 0: curl entries (k < n_c) with weights (wx, wy) and, when the stencils are
// shared, the HV weight too; kind 1: HV-only entries of a separate HV stencil
template <typename T>
__global__ void k_t_fill(const int32_t* __restrict__ idx, int stride, int64_t n, int ne, const double* __restrict__ wx,
                         const double* __restrict__ wy, int n_c, const double* __restrict__ wv, int n_v,
                         const int64_t* __restrict__ rowptr, unsigned long long* __restrict__ cursor,
                         int32_t* __restrict__ col, typename Vec<T>::V4* __restrict__ w, int kind) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * ne) return;
    const int64_t i = e / ne;
    const int k = (int)(e % ne);
    const int64_t j = idx[i * stride + k];
    const int64_t pos = rowptr[j] + (int64_t)atomicAdd(cursor + j, 1ull);
    typename Vec<T>::V4 v;
    v.x = (kind == 0 && k < n_c) ? (T)wx[i * n_c + k] : T(0);
    v.y = (kind == 0 && k < n_c) ? (T)wy[i * n_c + k] : T(0);
    v.z = (wv && k < n_v) ? (T)wv[i * n_v + k] : T(0);
    v.w = (T)kind;
    col[pos] = (int32_t)i;
    w[pos] = v;
}

// pad the tail of every row (column j, zero weights) and sort each row by (column, kind)
template <typename T>
__global__ void k_t_finish(const int64_t* __restrict__ rowptr, const unsigned long long* __restrict__ cursor, int64_t n,
                           int32_t* __restrict__ col, typename Vec<T>::V4* __restrict__ w) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int64_t b = rowptr[j], e = rowptr[j + 1], filled = b + (int64_t)cursor[j];
    for (int64_t p = filled; p < e; ++p) {
        col[p] = (int32_t)j;
        typename Vec<T>::V4 z;
        z.x = z.y = z.z = T(0);
        z.w = T(2);
        w[p] = z;
    }
    for (int64_t p = b + 1; p < e; ++p) {
        const int32_t c = col[p];
        const typename Vec<T>::V4 v = w[p];
        int64_t q = p - 1;
        while (q >= b && (col[q] > c || (col[q] == c && w[q].w > v.w))) {
            col[q + 1] = col[q];
            w[q + 1] = w[q];
            --q;
        }
        col[q + 1] = c;
        w[q + 1] = v;
    }
    for (int64_t p = b; p < e; ++p) w[p].w = T(0);
}

// chunks of the longest row of every slice of 32 rows
__global__ void k_t_slice_len(const int64_t* __restrict__ rowptr, int64_t n, int64_t* __restrict__ len) {
    const int64_t sl = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (sl >= (n + 31) / 32) return;
    int64_t m = 0;
    for (int64_t j = sl * 32; j < n && j < sl * 32 + 32; ++j) m = max(m, (rowptr[j + 1] - rowptr[j]) / 4);
    len[sl] = m;
}

template <typename T>
__global__ void k_t_slice_fill(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               const typename Vec<T>::V4* __restrict__ w, int64_t n, const int64_t* __restrict__ off,
                               int4* __restrict__ scol, typename Vec<T>::V4* __restrict__ sx,
                               typename Vec<T>::V4* __restrict__ sy, typename Vec<T>::V4* __restrict__ sv) {
    using V4 = typename Vec<T>::V4;
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int64_t sl = j >> 5, lane = j & 31;
    const int64_t nc = off[sl + 1] - off[sl];
    const int64_t b = rowptr[j], len = (rowptr[j + 1] - b) / 4;
    for (int64_t c = 0; c < nc; ++c) {
        const int64_t d = (off[sl] + c) * 32 + lane;
        int4 ci;
        V4 x, y, v;
        if (c < len) {
            const int64_t p = b + 4 * c;
            ci = make_int4(col[p], col[p + 1], col[p + 2], col[p + 3]);
            x.x = w[p].x; x.y = w[p + 1].x; x.z = w[p + 2].x; x.w = w[p + 3].x;
            y.x = w[p].y; y.y = w[p + 1].y; y.z = w[p + 2].y; y.w = w[p + 3].y;
            v.x = w[p].z; v.y = w[p + 1].z; v.z = w[p + 2].z; v.w = w[p + 3].z;
        } else {
            ci = make_int4((int)j, (int)j, (int)j, (int)j);
            x.x = x.y = x.z = x.w = T(0);
            y = x;
            v = x;
        }
        scol[d] = ci;
        sx[d] = x;
        sy[d] = y;
        sv[d] = v;
    }
}

mfd_status adj_build(mfd_ctx* ctx, const mfd_weights* curl, const mfd_weights* hv, bool fp64, AdjT& out) {
    cudaStream_t s = ctx->stream;
    const int64_t n = curl->st->centres->n;
    const bool shared = curl->st == hv->st;
    out.n = n;
    DevBuf cnt, padded, cursor, tmp;
    MFD_TRY(cnt.alloc((n + 1) * 8));
    MFD_TRY(padded.alloc((n + 1) * 8));
    MFD_TRY(cursor.alloc((n + 1) * 8));
    MFD_TRY(out.rowptr.alloc((n + 1) * 8));
    MFD_CUDA(cudaMemsetAsync(cnt.p, 0, (n + 1) * 8, s));
    MFD_CUDA(cudaMemsetAsync(cursor.p, 0, (n + 1) * 8, s));
    MFD_CUDA(cudaMemsetAsync(padded.p, 0, (n + 1) * 8, s));
    const int ne_c = shared ? std::max(curl->n_use, hv->n_use) : curl->n_use;
    auto grid = [](int64_t t) { return (unsigned)((t + 255) / 256); };
    k_t_count<<<grid(n * ne_c), 256, 0, s>>>(curl->st->idx.as<int32_t>(), curl->st->n, n, ne_c, cnt.as<int64_t>());
    if (!shared)
        k_t_count<<<grid(n * hv->n_use), 256, 0, s>>>(hv->st->idx.as<int32_t>(), hv->st->n, n, hv->n_use,
                                                       cnt.as<int64_t>());
    k_t_pad<<<grid(n), 256, 0, s>>>(cnt.as<int64_t>(), n, padded.as<int64_t>());
    MFD_CUDA(cudaGetLastError());
    size_t tb = 0;
    MFD_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tb, padded.as<int64_t>(), out.rowptr.as<int64_t>(), n + 1, s));
    MFD_TRY(tmp.alloc(tb));
    MFD_CUDA(cub::DeviceScan::ExclusiveSum(tmp.p, tb, padded.as<int64_t>(), out.rowptr.as<int64_t>(), n + 1, s));
    int64_t nnz = 0;
    MFD_CUDA(cudaMemcpyAsync(&nnz, out.rowptr.as<int64_t>() + n, 8, cudaMemcpyDeviceToHost, s));
    MFD_CUDA(cudaStreamSynchronize(s));
    out.nnz = nnz;
    const size_t es = fp64 ? 32 : 16;
    MFD_TRY(out.col.alloc(std::max<int64_t>(nnz, 4) * 4));
    MFD_TRY(out.w.alloc(std::max<int64_t>(nnz, 4) * es));
    const double* wx = curl->w.as<double>();
    const double* wy = wx + n * curl->n_use;
    const double* wv = hv->w.as<double>();
#define FILL(T)                                                                                                        \
    k_t_fill<T><<<grid(n * ne_c), 256, 0, s>>>(curl->st->idx.as<int32_t>(), curl->st->n, n, ne_c, wx, wy, curl->n_use, \
                                               shared ? wv : nullptr, hv->n_use, out.rowptr.as<int64_t>(),             \
                                               cursor.as<unsigned long long>(), out.col.as<int32_t>(),                 \
                                               out.w.as<typename Vec<T>::V4>(), 0);                                    \
    if (!shared)                                                                                                       \
        k_t_fill<T><<<grid(n * hv->n_use), 256, 0, s>>>(hv->st->idx.as<int32_t>(), hv->st->n, n, hv->n_use, nullptr,   \
                                                        nullptr, 0, wv, hv->n_use, out.rowptr.as<int64_t>(),           \
                                                        cursor.as<unsigned long long>(), out.col.as<int32_t>(),        \
                                                        out.w.as<typename Vec<T>::V4>(), 1);                           \
    k_t_finish<T><<<grid(n), 256, 0, s>>>(out.rowptr.as<int64_t>(), cursor.as<unsigned long long>(), n,                \
                                          out.col.as<int32_t>(), out.w.as<typename Vec<T>::V4>());
    if (fp64) {
        FILL(double)
    } else {
        FILL(float)
    }
#undef FILL
    MFD_CUDA(cudaGetLastError());
    // the sliced copy the step kernels read
    const int64_t nsl = (n + 31) / 32;
    DevBuf slen;
    MFD_TRY(slen.alloc((nsl + 1) * 8));
    MFD_TRY(out.off.alloc((nsl + 1) * 8));
    MFD_CUDA(cudaMemsetAsync(slen.p, 0, (nsl + 1) * 8, s));
    k_t_slice_len<<<grid(nsl), 256, 0, s>>>(out.rowptr.as<int64_t>(), n, slen.as<int64_t>());
    MFD_CUDA(cudaGetLastError());
    size_t tb2 = 0;
    MFD_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tb2, slen.as<int64_t>(), out.off.as<int64_t>(), nsl + 1, s));
    DevBuf tmp2;
    MFD_TRY(tmp2.alloc(tb2));
    MFD_CUDA(cub::DeviceScan::ExclusiveSum(tmp2.p, tb2, slen.as<int64_t>(), out.off.as<int64_t>(), nsl + 1, s));
    MFD_CUDA(cudaMemcpyAsync(&out.chunks, out.off.as<int64_t>() + nsl, 8, cudaMemcpyDeviceToHost, s));
    MFD_CUDA(cudaStreamSynchronize(s));
    const int64_t ent = std::max<int64_t>(out.chunks, 1) * 32;
    MFD_TRY(out.scol.alloc(ent * 16));
    MFD_TRY(out.sx.alloc(ent * es));
    MFD_TRY(out.sy.alloc(ent * es));
    MFD_TRY(out.sv.alloc(ent * es));
    if (fp64)
        k_t_slice_fill<double><<<grid(n), 256, 0, s>>>(out.rowptr.as<int64_t>(), out.col.as<int32_t>(), out.w.as<dbl4>(), n,
                                                       out.off.as<int64_t>(), out.scol.as<int4>(), out.sx.as<dbl4>(),
                                                       out.sy.as<dbl4>(), out.sv.as<dbl4>());
    else
        k_t_slice_fill<float><<<grid(n), 256, 0, s>>>(out.rowptr.as<int64_t>(), out.col.as<int32_t>(), out.w.as<float4>(), n,
                                                      out.off.as<int64_t>(), out.scol.as<int4>(), out.sx.as<float4>(),
                                                      out.sy.as<float4>(), out.sv.as<float4>());
    MFD_CUDA(cudaGetLastError());
    MFD_CUDA(cudaStreamSynchronize(s));
    out.col.release();  // the kernels read the sliced copy only
    out.w.release();
    return MFD_OK;
}

// first entry of the ascending list v[0 .. m) that is >= key
__device__ __forceinline__ int lower_bound_i64(const int64_t* v, int m, int64_t key) {
    int lo = 0, hi = m;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (v[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ bool has_bit(const uint32_t* mask, int64_t j) {
    return mask && ((mask[j >> 5] >> (j & 31)) & 1u);
}

template <typename T>
__global__ void __launch_bounds__(256) k_adj_a(const int64_t* __restrict__ off, const int4* __restrict__ scol,
                                               const typename Vec<T>::V4* __restrict__ sx,
                                               const typename Vec<T>::V4* __restrict__ sy,
                                               const typename Vec<T>::V4* __restrict__ sv, int64_t n,
                                               const typename Vec<T>::V4* __restrict__ LA,
                                               typename Vec<T>::V4* __restrict__ LB, T gamma,
                                               const T* __restrict__ ez, const int64_t* __restrict__ slot0, int kl,
                                               const double* __restrict__ eps, double* __restrict__ g_eps,
                                               AdjTerms tm, float keep) {
    using V4 = typename Vec<T>::V4;
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    if (has_bit(tm.smask, j)) {
        // the soft-source terms of step n -> n + 1 at node j (mu = lambda_E^{n+1}; a PEC node is
        // held at zero and has no dependence)
        const V4 l = ld_gather(LA + j);
        if (l.w != T(0)) {
            const double mu = (double)l.x;
            const double t1 = (double)(*tm.seg0 + kl + 1) * tm.dt;
            const double pi = 3.14159265358979323846;
            for (int q = lower_bound_i64(tm.snode, tm.nsrc, j); q < tm.nsrc && tm.snode[q] == j; ++q) {
                const int k = tm.sidx[q];
                double x = pi * tm.f0[k] * (t1 - tm.t0[k]);
                x = x * x;
                const double r = (1.0 - 2.0 * x) * exp(-x);
                tm.g_amp[k] += mu * r;
                g_eps[j] += mu * tm.amp[k] * r / eps[j];
            }
        }
    }
    const int64_t sl = j >> 5;
    const int64_t base = off[sl] * 32 + (j & 31);
    const int nc = (int)(off[sl + 1] - off[sl]);
    const uint64_t pol = stream_policy(keep);
    T ax = 0, ay = 0, av = 0;
    for (int c = 0; c < nc; ++c) {
        const int64_t d = base + (int64_t)c * 32;
        const int4 id = chk4(ld_stream(scol + d, pol), n);
        const V4 wx = ld_stream(sx + d, pol), wy = ld_stream(sy + d, pol), wv = ld_stream(sv + d, pol);
        const int ids[4] = {id.x, id.y, id.z, id.w};
        const T* wxs = &wx.x;
        const T* wys = &wy.x;
        const T* wvs = &wv.x;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const V4 l = ld_gather(LA + ids[q]);
            const T km = l.w * l.x;  // K mu (0 on PEC nodes, where ce = 0)
            ax = fma(-wys[q], km, ax);
            ay = fma(wxs[q], km, ay);
            av = fma(wvs[q], km, av);
        }
    }
    const V4 me = ld_gather(LA + j);
    const T mu = me.w == T(0) ? T(0) : me.x;
    V4 o;
    o.x = mu + gamma * av;
    o.y = me.y + ax;
    o.z = me.z + ay;
    o.w = me.w;
    st4(LB + j, o);
    if (me.w != T(0)) {
        const T* e0 = ez + (*slot0 + kl) * n;
        g_eps[j] += (double)mu * (-((double)e0[n + j] - (double)e0[j]) / eps[j]);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_adj_b(const int64_t* __restrict__ off, const int4* __restrict__ scol,
                                               const typename Vec<T>::V4* __restrict__ sx,
                                               const typename Vec<T>::V4* __restrict__ sy,
                                               const typename Vec<T>::V4* __restrict__ sv, int64_t n,
                                               const typename Vec<T>::V4* __restrict__ LB,
                                               typename Vec<T>::V4* __restrict__ LA, T ch, T gamma,
                                               const T* __restrict__ ez, const int64_t* __restrict__ slot0, int kl,
                                               AdjTerms tm, float keep) {
    using V4 = typename Vec<T>::V4;
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int64_t sl = j >> 5;
    const int64_t base = off[sl] * 32 + (j & 31);
    const int nc = (int)(off[sl + 1] - off[sl]);
    const uint64_t pol = stream_policy(keep);
    T vx = 0, vy = 0, cx = 0, cy = 0;
    for (int c = 0; c < nc; ++c) {
        const int64_t d = base + (int64_t)c * 32;
        const int4 id = chk4(ld_stream(scol + d, pol), n);
        const V4 wx = ld_stream(sx + d, pol), wy = ld_stream(sy + d, pol), wv = ld_stream(sv + d, pol);
        const int ids[4] = {id.x, id.y, id.z, id.w};
        const T* wxs = &wx.x;
        const T* wys = &wy.x;
        const T* wvs = &wv.x;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const V4 l = ld_gather(LB + ids[q]);
            vx = fma(wvs[q], l.y, vx);
            vy = fma(wvs[q], l.z, vy);
            cx = fma(wxs[q], l.z, cx);  // Dx^T l~Hy
            cy = fma(wys[q], l.y, cy);  // Dy^T l~Hx
        }
    }
    const V4 me = ld_gather(LB + j);
    V4 o;
    o.x = me.x + ch * (cx - cy);
    o.y = me.y + ch * gamma * vx;
    o.z = me.z + ch * gamma * vy;
    o.w = me.w;
    if (has_bit(tm.pmask, j) && *tm.seg0 + kl >= tm.min_step) {
        // the probe terms dJ/dE^n at node j, n = *seg0 + kl (one per probe on the node)
        const T e = ez[(*slot0 + kl) * n + j];
        for (int q = lower_bound_i64(tm.pnode, tm.nprobe, j); q < tm.nprobe && tm.pnode[q] == j; ++q)
            o.x += (T)(2.0 * tm.dt * (double)e);
    }
    st4(LA + j, o);
}

cudaError_t adj_pass(const AdjArgs& a, int pass, cudaStream_t s) {
    const unsigned g = (unsigned)((a.n + 255) / 256);
    const AdjTerms tm = a.terms ? *a.terms : AdjTerms{};
    if (a.fp64) {
        const dbl4 *x = (const dbl4*)a.sx, *y = (const dbl4*)a.sy, *v = (const dbl4*)a.sv;
        if (pass == 0)
            k_adj_a<double><<<g, 256, 0, s>>>(a.off, a.scol, x, y, v, a.n, (const dbl4*)a.LA, (dbl4*)a.LB, a.gamma,
                                              (const double*)a.ez, a.slot0, a.k, a.eps, a.g_eps, tm, a.l2_keep);
        else
            k_adj_b<double><<<g, 256, 0, s>>>(a.off, a.scol, x, y, v, a.n, (const dbl4*)a.LB, (dbl4*)a.LA, a.ch,
                                              a.gamma, (const double*)a.ez, a.slot0, a.k, tm, a.l2_keep);
    } else {
        const float4 *x = (const float4*)a.sx, *y = (const float4*)a.sy, *v = (const float4*)a.sv;
        if (pass == 0)
            k_adj_a<float><<<g, 256, 0, s>>>(a.off, a.scol, x, y, v, a.n, (const float4*)a.LA, (float4*)a.LB,
                                             (float)a.gamma, (const float*)a.ez, a.slot0, a.k, a.eps, a.g_eps, tm, a.l2_keep);
        else
            k_adj_b<float><<<g, 256, 0, s>>>(a.off, a.scol, x, y, v, a.n, (const float4*)a.LB, (float4*)a.LA,
                                             (float)a.ch, (float)a.gamma, (const float*)a.ez, a.slot0, a.k, tm, a.l2_keep);
    }
    return cudaGetLastError();
}

template <typename T>
__global__ void k_adj_probe(T* __restrict__ LA, const T* __restrict__ ez, const int64_t* __restrict__ probe, int np,
                            double dt, const int64_t* __restrict__ seg0, int k, int64_t min_step,
                            const int64_t* __restrict__ slot0, int64_t n) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    if (seg0 && *seg0 + k < min_step) return;
    const T* e = slot0 ? ez + (*slot0 + k) * n : ez;
    const int64_t i = probe[p];
    atomicAdd(LA + 4 * i, (T)(2.0 * dt * (double)e[i]));  // a node probed twice gets both terms
}

cudaError_t adj_probe_term(bool fp64, void* LA, const void* ez, const int64_t* probe, int nprobe, double dt,
                           cudaStream_t s, const int64_t* seg0, int k, int64_t min_step, const int64_t* slot0,
                           int64_t n) {
    if (nprobe <= 0) return cudaSuccess;
    const unsigned g = (unsigned)((nprobe + 127) / 128);
    if (fp64)
        k_adj_probe<double><<<g, 128, 0, s>>>((double*)LA, (const double*)ez, probe, nprobe, dt, seg0, k, min_step,
                                              slot0, n);
    else
        k_adj_probe<float><<<g, 128, 0, s>>>((float*)LA, (const float*)ez, probe, nprobe, dt, seg0, k, min_step, slot0,
                                             n);
    return cudaGetLastError();
}

template <typename T> __global__ void k_init_lambda(T* __restrict__ LA, const T* __restrict__ A, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    LA[4 * i] = T(0);
    LA[4 * i + 1] = T(0);
    LA[4 * i + 2] = T(0);
    LA[4 * i + 3] = A[4 * i + 3];
}

unsigned long long bounds_take_adjoint(cudaStream_t s) { return bounds_take_local(s); }

cudaError_t init_lambda(bool fp64, void* LA, const void* A, int64_t n, cudaStream_t s) {
    const unsigned g = (unsigned)((n + 255) / 256);
    if (fp64) k_init_lambda<double><<<g, 256, 0, s>>>((double*)LA, (const double*)A, n);
    else k_init_lambda<float><<<g, 256, 0, s>>>((float*)LA, (const float*)A, n);
    return cudaGetLastError();
}

template <typename T>
__global__ void k_sumsq(const T* __restrict__ buf, int64_t count, double dt, double* __restrict__ J) {
    __shared__ double red[256];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < count; i += 256) {
        const double v = (double)buf[i];
        s += v * v;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *J = dt * red[0];
}

cudaError_t probe_energy(bool fp64, const void* buf, int64_t count, double dt, double* J, cudaStream_t s) {
    if (fp64) k_sumsq<double><<<1, 256, 0, s>>>((const double*)buf, count, dt, J);
    else k_sumsq<float><<<1, 256, 0, s>>>((const float*)buf, count, dt, J);
    return cudaGetLastError();
}

template <typename T> __global__ void k_copy_ez(const T* __restrict__ st, T* __restrict__ dst, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = st[4 * i];
}

template <typename T>
__global__ void k_copy_ez_level(const T* __restrict__ st, T* __restrict__ hist, int64_t n,
                                const int64_t* __restrict__ counter, int64_t start) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) hist[(*counter - start) * n + i] = st[4 * i];
}

cudaError_t copy_ez_level(bool fp64, const void* state, void* hist, int64_t n, const int64_t* counter, int64_t start,
                          cudaStream_t s) {
    const unsigned g = (unsigned)((n + 255) / 256);
    if (fp64) k_copy_ez_level<double><<<g, 256, 0, s>>>((const double*)state, (double*)hist, n, counter, start);
    else k_copy_ez_level<float><<<g, 256, 0, s>>>((const float*)state, (float*)hist, n, counter, start);
    return cudaGetLastError();
}

cudaError_t copy_ez(bool fp64, const void* state, void* dst, int64_t n, cudaStream_t s) {
    const unsigned g = (unsigned)((n + 255) / 256);
    if (fp64) k_copy_ez<double><<<g, 256, 0, s>>>((const double*)state, (double*)dst, n);
    else k_copy_ez<float><<<g, 256, 0, s>>>((const float*)state, (float*)dst, n);
    return cudaGetLastError();
}

}  // namespace mfd
