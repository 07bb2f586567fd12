// yee.cu -- the FDTD (Yee) scheme for TMz (Eq. 4, Eq. 5) on a periodic grid:
// the reference the paper compares its meshless method with (Sec. 3, Sec. 6).
//
// One fused kernel per launch (k_yee, below) advances one step, or four when
// there are no sources and probes: a block holds a window of the grid in
// registers and writes the cells whose dependency cone lies inside it. State
// ping-pongs between two buffers so that no block reads what another block of
// the same launch writes. Soft sources and probes follow each one-step launch
// in k_yee_post. Compulsory traffic per cell and launch: Ez, Hx, Hy read once
// and written once (6 reals).
//
// Arithmetic follows Eq. 5 term by term with round-to-nearest operations (no
// contraction), in the oracle's order, so FP64 results are reproducible
// bit for bit.
#include <cmath>
#include <string>
#include <vector>

#include "internal.cuh"

namespace mfd {

__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }

// periodic index of v in [-1, n + tile): one compare when the grid is at least
// one tile wide (BIG), a full reduction otherwise
template <bool BIG> __device__ __forceinline__ int wrap(int v, int n) {
    if (BIG) return v < 0 ? v + n : (v >= n ? v - n : v);
    return ((v % n) + n) % n;
}

// The step kernel, S steps per launch (S > 1, temporal blocking, for runs
// without sources or probes, whose terms sit between the steps). A block holds
// a 32-column by 4 YW_W-row window of the grid in registers: lane c of warp w
// holds column x0 - S + c of rows y0 - S + 4w .. y0 - S + 3 + 4w (YW_W warps;
// S = the steps per launch), Ez and the old Hx, Hy of each. It computes
// H^{n+1/2} and E^{n+1}, then the next half steps up to E^{n+S}: neighbours
// along x come from the adjacent lane by a shuffle, neighbours along y from the
// thread's own registers or, across warps, through one shared row per warp and
// half step. The valid region shrinks by a cell per half step on the sides the
// stencil reads, leaving a (32 - 2S) x (4 YW_W - 2S) tile (window columns and rows
// S .. end - S), written once: 6 reals of DRAM traffic per cell and launch.
// Arithmetic follows Eq. 5 term by term with round-to-nearest operations (no
// contraction), in the oracle's order, so FP64 results are reproducible bit for
// bit and do not depend on the steps per launch.
constexpr int YW_W = 9;  // warps; four window rows each
template <int S> constexpr int yee_tile_x() { return 32 - 2 * S; }
template <int S> constexpr int yee_tile_y() { return 4 * YW_W - 2 * S; }

template <typename T, bool BIG, int S>
__global__ void __launch_bounds__(32 * YW_W) k_yee(int nx, int ny, T ch, T ce, const T* __restrict__ ez,
                                                   const T* __restrict__ hx, const T* __restrict__ hy,
                                                   T* __restrict__ ez_o, T* __restrict__ hx_o,
                                                   T* __restrict__ hy_o) {
    static_assert(S >= 1 && S <= 4, "one to four steps per launch");
    constexpr int TX = yee_tile_x<S>(), TY = yee_tile_y<S>();
    __shared__ T xe[YW_W][32];  // per warp: E^{n+1} of its first row
    __shared__ T xh[YW_W][32];  // per warp: Hx of its last row (H^{n+1/2}, then H^{n+3/2})
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x, w = threadIdx.y;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int gx = wrap<BIG>(x0 - S + lane, nx);
    const int r0 = 4 * w;  // window rows r0 .. r0 + 3
    T e[5], sx[4], sy[4];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int64_t g = (int64_t)wrap<BIG>(y0 - S + r0 + k, ny) * nx + gx;
        e[k] = ez[g];
        if (k < 4) {
            sx[k] = hx[g];
            sy[k] = hy[g];
        }
    }
    const int i = x0 - S + lane;
#pragma unroll
    for (int st = 0; st < S; ++st) {
        // H half step st: valid on window columns st .. 30 - st, rows st .. 34 - st
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const T right = __shfl_down_sync(FULL, e[k], 1);
            sx[k] = rn_sub(sx[k], rn_mul(ch, rn_sub(e[k + 1], e[k])));
            sy[k] = rn_add(sy[k], rn_mul(ch, rn_sub(right, e[k])));
        }
        xh[w][lane] = sx[3];
        __syncthreads();  // also: every warp has read xe of the previous step
        const T below = w > 0 ? xh[w - 1][lane] : sx[0];  // Hx of row r0 - 1 (row 0 is outside the valid region)
        // E half step st: valid on columns st + 1 .. 30 - st, rows st + 1 .. 34 - st; after the
        // last, the tile (columns and rows S .. end - S) is written with its H
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const T left = __shfl_up_sync(FULL, sy[k], 1);
            const T down = k > 0 ? sx[k - 1] : below;
            const T curl = rn_add(rn_sub(rn_sub(sy[k], left), sx[k]), down);
            const T en = rn_add(e[k], rn_mul(ce, curl));
            if (st + 1 < S) {
                e[k] = en;
            } else {
                const int row = r0 + k, j = y0 - S + row;
                if (lane >= S && lane < S + TX && row >= S && row < S + TY && i < nx && j < ny) {
                    const int64_t g = (int64_t)j * nx + i;
                    ez_o[g] = en;
                    hx_o[g] = sx[k];
                    hy_o[g] = sy[k];
                }
            }
        }
        if (st + 1 < S) {
            xe[w][lane] = e[0];
            __syncthreads();  // also: every warp has read xh above
            e[4] = w + 1 < YW_W ? xe[w + 1][lane] : e[3];  // E of row r0 + 4 (row 4 YW_W: outside)
        }
    }
}

// soft Ricker sources after the E update, then probes, then the step counter
template <typename T>
__global__ void k_yee_post(T* __restrict__ ez, int nsrc, const int64_t* __restrict__ sn, const double* __restrict__ sa,
                           const double* __restrict__ sf, const double* __restrict__ st0, int nprobe,
                           const int64_t* __restrict__ pn, T* __restrict__ pbuf, int64_t pcap,
                           const int64_t* __restrict__ pstep0, int64_t* __restrict__ counter, double dt) {
    __shared__ int64_t n_s;
    if (threadIdx.x == 0) n_s = *counter;
    __syncthreads();
    const int64_t n = n_s;
    const double t1 = (double)(n + 1) * dt;
    const double pi = 3.14159265358979323846;
    // sources one after another in the caller's order (two may share a cell)
    if (threadIdx.x == 0)
        for (int s = 0; s < nsrc; ++s) {
            double a = pi * sf[s] * (t1 - st0[s]);
            a = a * a;
            ez[sn[s]] = (T)((double)ez[sn[s]] + sa[s] * ((1.0 - 2.0 * a) * exp(-a)));
        }
    __syncthreads();
    if (nprobe > 0) {
        const int64_t rec = n - *pstep0;
        if (rec >= 0 && rec < pcap)
            for (int p = threadIdx.x; p < nprobe; p += blockDim.x) pbuf[rec * nprobe + p] = ez[pn[p]];
    }
    __syncthreads();
    if (threadIdx.x == 0) *counter = n + 1;
}

template <typename T> __global__ void k_yee_scatter(const double* __restrict__ src, T* __restrict__ dst, int64_t n) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < n) dst[k] = (T)src[k];
}
template <typename T> __global__ void k_yee_gather(const T* __restrict__ src, double* __restrict__ dst, int64_t n) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < n) dst[k] = (double)src[k];
}

}  // namespace mfd

using namespace mfd;

struct mfd_yee {
    mfd_ctx* ctx = nullptr;
    int64_t nx = 0, ny = 0;
    bool fp64 = false;
    size_t rs = 4;
    double dt = 0, ch = 0, ce = 0;
    DevBuf f[2][3];  // ping-pong {Ez, Hx, Hy}
    int cur = 0;
    DevBuf counter, pstep0, src_node, src_amp, src_f0, src_t0, probe_node, probe_buf;
    int nsrc = 0, nprobe = 0;
    int64_t probe_cap = 0, probe_from = 0, steps = 0;
    cudaGraphExec_t graph = nullptr;
    bool graph_ok = false;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    ~mfd_yee() {
        if (graph) cudaGraphExecDestroy(graph);
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
    }
};

namespace {

constexpr int YEE_GRAPH_STEPS = 32;
// steps per launch without sources and probes; YEE_GRAPH_STEPS / YEE_MULTI launches per graph
// must be even (each launch swaps the buffers)
constexpr int YEE_MULTI = 4;  // measured at 8192^2: 2 -> 0.130 ms per step, 4 -> 0.093 ms
static_assert(YEE_GRAPH_STEPS % (2 * YEE_MULTI) == 0, "an even number of launches per graph");

// one launch of k_yee with S steps (S > 1 only without sources and probes)
template <int S> cudaError_t yee_launch(mfd_yee* y) {
    cudaStream_t s = y->ctx->stream;
    const dim3 grid((unsigned)((y->nx + yee_tile_x<S>() - 1) / yee_tile_x<S>()),
                    (unsigned)((y->ny + yee_tile_y<S>() - 1) / yee_tile_y<S>()));
    const dim3 block(32, YW_W);
    const int a = y->cur, b = y->cur ^ 1;
    // one compare per wrap while the window (columns x0-S .. x0-S+31, rows y0-S .. y0-S+4 YW_W)
    // stays within one period of the grid on either side
    const bool big = y->nx >= 32 && y->ny >= 4 * YW_W + 1;
    const int nx = (int)y->nx, ny = (int)y->ny;
    if (y->fp64) {
        const double *e = y->f[a][0].as<double>(), *hx = y->f[a][1].as<double>(), *hy = y->f[a][2].as<double>();
        double *eo = y->f[b][0].as<double>(), *hxo = y->f[b][1].as<double>(), *hyo = y->f[b][2].as<double>();
        if (big) k_yee<double, true, S><<<grid, block, 0, s>>>(nx, ny, y->ch, y->ce, e, hx, hy, eo, hxo, hyo);
        else k_yee<double, false, S><<<grid, block, 0, s>>>(nx, ny, y->ch, y->ce, e, hx, hy, eo, hxo, hyo);
    } else {
        const float *e = y->f[a][0].as<float>(), *hx = y->f[a][1].as<float>(), *hy = y->f[a][2].as<float>();
        float *eo = y->f[b][0].as<float>(), *hxo = y->f[b][1].as<float>(), *hyo = y->f[b][2].as<float>();
        const float ch = (float)y->ch, ce = (float)y->ce;
        if (big) k_yee<float, true, S><<<grid, block, 0, s>>>(nx, ny, ch, ce, e, hx, hy, eo, hxo, hyo);
        else k_yee<float, false, S><<<grid, block, 0, s>>>(nx, ny, ch, ce, e, hx, hy, eo, hxo, hyo);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    y->cur = b;
    return cudaSuccess;
}

// YEE_MULTI steps in one launch; only without sources and probes
cudaError_t yee_enqueue_multi(mfd_yee* y) {
    cudaError_t e = yee_launch<YEE_MULTI>(y);
    if (e == cudaSuccess) y->steps += YEE_MULTI;
    return e;
}

cudaError_t yee_enqueue(mfd_yee* y) {
    cudaStream_t s = y->ctx->stream;
    cudaError_t e = yee_launch<1>(y);
    if (e != cudaSuccess) return e;
    const int b = y->cur;
    if (y->nsrc > 0 || y->nprobe > 0) {
        if (y->fp64)
            k_yee_post<double><<<1, 256, 0, s>>>(y->f[b][0].as<double>(), y->nsrc, y->src_node.as<int64_t>(),
                                                 y->src_amp.as<double>(), y->src_f0.as<double>(), y->src_t0.as<double>(),
                                                 y->nprobe, y->probe_node.as<int64_t>(), y->probe_buf.as<double>(),
                                                 y->probe_cap, y->pstep0.as<int64_t>(), y->counter.as<int64_t>(), y->dt);
        else
            k_yee_post<float><<<1, 256, 0, s>>>(y->f[b][0].as<float>(), y->nsrc, y->src_node.as<int64_t>(),
                                                y->src_amp.as<double>(), y->src_f0.as<double>(), y->src_t0.as<double>(),
                                                y->nprobe, y->probe_node.as<int64_t>(), y->probe_buf.as<float>(),
                                                y->probe_cap, y->pstep0.as<int64_t>(), y->counter.as<int64_t>(), y->dt);
        e = cudaGetLastError();
    }
    y->steps += 1;
    return e;
}

// the device step counter follows the host one when no post kernel runs
mfd_status yee_sync_counter(mfd_yee* y) {
    MFD_CUDA(cudaMemcpyAsync(y->counter.p, &y->steps, 8, cudaMemcpyHostToDevice, y->ctx->stream));
    MFD_CUDA(cudaStreamSynchronize(y->ctx->stream));
    return MFD_OK;
}

mfd_status yee_graph(mfd_yee* y) {
    if (y->graph_ok) return MFD_OK;
    if (y->graph) {
        cudaGraphExecDestroy(y->graph);
        y->graph = nullptr;
    }
    cudaStream_t s = y->ctx->stream;
    const int cur0 = y->cur;
    const int64_t steps0 = y->steps;
    MFD_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    if (y->nsrc == 0 && y->nprobe == 0)
        for (int k = 0; k < YEE_GRAPH_STEPS && e == cudaSuccess; k += YEE_MULTI) e = yee_enqueue_multi(y);
    else
        for (int k = 0; k < YEE_GRAPH_STEPS && e == cudaSuccess; ++k) e = yee_enqueue(y);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s, &g);
    y->cur = cur0;
    y->steps = steps0;
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(MFD_ERR_CUDA, std::string("graph capture failed: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&y->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(MFD_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    y->graph_ok = true;
    return MFD_OK;
}

mfd_status yee_field(mfd_yee* y, int comp, int* k) {
    if (comp == MFD_EZ) *k = 0;
    else if (comp == MFD_HX) *k = 1;
    else if (comp == MFD_HY) *k = 2;
    else return fail(MFD_ERR_ARG, "the Yee TMz grid has Ez, Hx, Hy only");
    return MFD_OK;
}

}  // namespace

extern "C" {

mfd_status mfd_yee_create(mfd_ctx* ctx, int64_t nx, int64_t ny, int precision, double dt, double h, double eps0,
                          double mu0, mfd_yee** out) {
    if (!ctx || !out) return fail(MFD_ERR_ARG, "mfd_yee_create: NULL argument");
    *out = nullptr;
    if (nx < 2 || ny < 2 || nx > INT32_MAX / 2 || ny > 65535LL * yee_tile_y<4>())
        return fail(MFD_ERR_ARG, "mfd_yee_create: need 2 <= nx < 2^30 and 2 <= ny <= " +
                                     std::to_string(65535LL * yee_tile_y<4>()));
    if (!(dt > 0) || !(h > 0) || !(eps0 > 0) || !(mu0 > 0)) return fail(MFD_ERR_ARG, "dt, h, eps0, mu0 must be > 0");
    if (precision != MFD_FP32 && precision != MFD_FP64) return fail(MFD_ERR_ARG, "precision");
    MFD_CUDA(cudaSetDevice(ctx->device));
    mfd_yee* y = new (std::nothrow) mfd_yee();
    if (!y) return fail(MFD_ERR_OOM, "host allocation failed");
    y->ctx = ctx;
    y->nx = nx;
    y->ny = ny;
    y->fp64 = precision == MFD_FP64;
    y->rs = y->fp64 ? 8 : 4;
    y->dt = dt;
    y->ch = dt / (mu0 * h);
    y->ce = dt / (eps0 * h);
    const size_t bytes = (size_t)nx * ny * y->rs;
    mfd_status st = MFD_OK;
    for (int p = 0; p < 2 && st == MFD_OK; ++p)
        for (int k = 0; k < 3 && st == MFD_OK; ++k) st = y->f[p][k].alloc(bytes);
    if (st == MFD_OK) st = y->counter.alloc(8);
    if (st == MFD_OK) st = y->pstep0.alloc(8);
    if (st != MFD_OK) {
        delete y;
        return st;
    }
    for (int p = 0; p < 2; ++p)
        for (int k = 0; k < 3; ++k) cudaMemsetAsync(y->f[p][k].p, 0, bytes, ctx->stream);
    cudaMemsetAsync(y->counter.p, 0, 8, ctx->stream);
    cudaMemsetAsync(y->pstep0.p, 0, 8, ctx->stream);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        delete y;
        return fail(MFD_ERR_CUDA, cudaGetErrorString(e));
    }
    retain(ctx);
    *out = y;
    return MFD_OK;
}

mfd_status mfd_yee_set_field(mfd_yee* y, int comp, const double* host) {
    if (!y || !host) return fail(MFD_ERR_ARG, "NULL argument");
    int k;
    MFD_TRY(yee_field(y, comp, &k));
    MFD_CUDA(cudaSetDevice(y->ctx->device));
    const int64_t n = y->nx * y->ny;
    DevBuf tmp;
    MFD_TRY(tmp.alloc(n * 8));
    cudaStream_t s = y->ctx->stream;
    MFD_CUDA(cudaMemcpyAsync(tmp.p, host, n * 8, cudaMemcpyHostToDevice, s));
    const unsigned g = (unsigned)((n + 255) / 256);
    if (y->fp64) k_yee_scatter<double><<<g, 256, 0, s>>>(tmp.as<double>(), y->f[y->cur][k].as<double>(), n);
    else k_yee_scatter<float><<<g, 256, 0, s>>>(tmp.as<double>(), y->f[y->cur][k].as<float>(), n);
    MFD_CUDA(cudaGetLastError());
    MFD_CUDA(cudaStreamSynchronize(s));
    return MFD_OK;
}

mfd_status mfd_yee_get_field(mfd_yee* y, int comp, double* host) {
    if (!y || !host) return fail(MFD_ERR_ARG, "NULL argument");
    int k;
    MFD_TRY(yee_field(y, comp, &k));
    MFD_CUDA(cudaSetDevice(y->ctx->device));
    const int64_t n = y->nx * y->ny;
    DevBuf tmp;
    MFD_TRY(tmp.alloc(n * 8));
    cudaStream_t s = y->ctx->stream;
    const unsigned g = (unsigned)((n + 255) / 256);
    if (y->fp64) k_yee_gather<double><<<g, 256, 0, s>>>(y->f[y->cur][k].as<double>(), tmp.as<double>(), n);
    else k_yee_gather<float><<<g, 256, 0, s>>>(y->f[y->cur][k].as<float>(), tmp.as<double>(), n);
    MFD_CUDA(cudaGetLastError());
    MFD_CUDA(cudaMemcpyAsync(host, tmp.p, n * 8, cudaMemcpyDeviceToHost, s));
    MFD_CUDA(cudaStreamSynchronize(s));
    return MFD_OK;
}

mfd_status mfd_yee_set_sources(mfd_yee* y, int count, const int64_t* cell, const double* amp, const double* f0,
                               const double* t0) {
    if (!y || count < 0 || (count > 0 && (!cell || !amp || !f0 || !t0))) return fail(MFD_ERR_ARG, "bad arguments");
    for (int s = 0; s < count; ++s) {
        if (cell[s] < 0 || cell[s] >= y->nx * y->ny) return fail(MFD_ERR_ARG, "source cell out of range");
        if (!(f0[s] > 0)) return fail(MFD_ERR_ARG, "source frequency must be > 0");
    }
    MFD_CUDA(cudaSetDevice(y->ctx->device));
    mfd_ctx* ctx = y->ctx;
    auto up = [&](DevBuf& b, const void* p, size_t bytes) -> mfd_status {
        MFD_TRY(b.alloc(bytes));
        if (bytes) MFD_CUDA(cudaMemcpyAsync(b.p, p, bytes, cudaMemcpyHostToDevice, ctx->stream));
        return MFD_OK;
    };
    // no sources and no graph until every array is in place (a failed call
    // leaves a grid without sources, never a count that outlives its arrays)
    y->nsrc = 0;
    y->graph_ok = false;
    MFD_TRY(up(y->src_node, cell, count * 8));
    MFD_TRY(up(y->src_amp, amp, count * 8));
    MFD_TRY(up(y->src_f0, f0, count * 8));
    MFD_TRY(up(y->src_t0, t0, count * 8));
    y->nsrc = count;
    y->graph_ok = false;
    return yee_sync_counter(y);
}

mfd_status mfd_yee_set_probes(mfd_yee* y, int count, const int64_t* cell, int64_t capacity) {
    if (!y || count < 0 || capacity < 0 || (count > 0 && !cell)) return fail(MFD_ERR_ARG, "bad arguments");
    for (int p = 0; p < count; ++p)
        if (cell[p] < 0 || cell[p] >= y->nx * y->ny) return fail(MFD_ERR_ARG, "probe cell out of range");
    MFD_CUDA(cudaSetDevice(y->ctx->device));
    y->nprobe = 0;
    y->probe_cap = 0;
    y->graph_ok = false;
    MFD_TRY(y->probe_node.alloc(std::max(1, count) * 8));
    if (count) MFD_CUDA(cudaMemcpyAsync(y->probe_node.p, cell, count * 8, cudaMemcpyHostToDevice, y->ctx->stream));
    MFD_TRY(y->probe_buf.alloc(std::max<int64_t>(1, capacity * count) * y->rs));
    y->nprobe = count;
    y->probe_cap = capacity;
    y->probe_from = y->steps;
    MFD_CUDA(cudaMemcpyAsync(y->pstep0.p, &y->probe_from, 8, cudaMemcpyHostToDevice, y->ctx->stream));
    y->graph_ok = false;
    return yee_sync_counter(y);
}

mfd_status mfd_yee_step(mfd_yee* y, int64_t nsteps) {
    if (!y || nsteps < 0) return fail(MFD_ERR_ARG, "bad arguments");
    MFD_CUDA(cudaSetDevice(y->ctx->device));
    int64_t left = nsteps;
    if (left >= 2 * YEE_GRAPH_STEPS) {
        if (y->cur != 0) {  // the graph is captured from buffer 0
            MFD_CUDA(yee_enqueue(y));
            --left;
        }
        MFD_TRY(yee_graph(y));
        while (left >= YEE_GRAPH_STEPS) {
            MFD_CUDA(cudaGraphLaunch(y->graph, y->ctx->stream));
            y->steps += YEE_GRAPH_STEPS;  // YEE_GRAPH_STEPS is even: the buffer parity is unchanged
            left -= YEE_GRAPH_STEPS;
        }
    }
    const bool multi = y->nsrc == 0 && y->nprobe == 0;
    while (left > 0) {
        if (multi && left >= YEE_MULTI) {
            MFD_CUDA(yee_enqueue_multi(y));
            left -= YEE_MULTI;
        } else {
            MFD_CUDA(yee_enqueue(y));
            --left;
        }
    }
    return MFD_OK;
}

int mfd_yee_steps_per_launch(const mfd_yee* y) { return y && y->nsrc == 0 && y->nprobe == 0 ? YEE_MULTI : 1; }

mfd_status mfd_yee_step_timed(mfd_yee* y, int64_t nsteps, double* ms) {
    if (!y || nsteps < 0 || !ms) return fail(MFD_ERR_ARG, "bad arguments");
    MFD_CUDA(cudaSetDevice(y->ctx->device));
    cudaStream_t s = y->ctx->stream;
    for (auto& e : y->ev)
        if (!e) MFD_CUDA(cudaEventCreate(&e));
    double tot = 0.0;
    const bool multi = y->nsrc == 0 && y->nprobe == 0;
    for (int64_t k = 0; k < nsteps; k += (multi && k + YEE_MULTI <= nsteps) ? YEE_MULTI : 1) {
        MFD_CUDA(cudaEventRecord(y->ev[0], s));
        if (multi && k + YEE_MULTI <= nsteps) MFD_CUDA(yee_enqueue_multi(y));
        else MFD_CUDA(yee_enqueue(y));
        MFD_CUDA(cudaEventRecord(y->ev[1], s));
        MFD_CUDA(cudaEventSynchronize(y->ev[1]));
        float t = 0.f;
        MFD_CUDA(cudaEventElapsedTime(&t, y->ev[0], y->ev[1]));
        tot += t;
    }
    *ms = tot;
    return MFD_OK;
}

mfd_status mfd_yee_read_probes(mfd_yee* y, double* host, int64_t* steps) {
    if (!y) return fail(MFD_ERR_ARG, "NULL argument");
    MFD_CUDA(cudaSetDevice(y->ctx->device));
    int64_t rec = std::min(y->steps - y->probe_from, y->probe_cap);
    if (rec < 0) rec = 0;
    if (steps) *steps = rec;
    MFD_CUDA(cudaStreamSynchronize(y->ctx->stream));
    if (!host || rec == 0 || y->nprobe == 0) return MFD_OK;
    const int64_t count = rec * y->nprobe;
    if (y->fp64) {
        MFD_CUDA(cudaMemcpy(host, y->probe_buf.p, count * 8, cudaMemcpyDeviceToHost));
    } else {
        std::vector<float> tmp(count);
        MFD_CUDA(cudaMemcpy(tmp.data(), y->probe_buf.p, count * 4, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < count; ++i) host[i] = tmp[i];
    }
    return MFD_OK;
}

void mfd_yee_destroy(mfd_yee* y) {
    if (!y) return;
    mfd_ctx* ctx = y->ctx;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    delete y;
    release(ctx);
}

}  // extern "C"
