// setup.cu -- one-off setup on the GPU: Morton reordering of node sets, grid-hash
// kNN stencils (Sec. 4.1, Eq. 11) and the batched FP64 solve of the local
// PHS + monomial systems (Eq. 9) for RBF-FD (Eq. 13) and RBF-VFD (Eqs. 14-15)
// weights, including the hyperviscosity operator Delta^alpha (Sec. 5.1).
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>

#include "internal.cuh"
#include "kernels.cuh"

namespace mfd {

// ------------------------------------------------------------ helpers

// order-preserving map of doubles onto int64 for atomic min/max
__device__ __forceinline__ long long dbl_key(double x) {
    long long i = __double_as_longlong(x);
    return i >= 0 ? i : (i ^ 0x7FFFFFFFFFFFFFFFLL);
}
static double key_dbl(long long i) {
    long long b = i >= 0 ? i : (i ^ 0x7FFFFFFFFFFFFFFFLL);
    double x;
    memcpy(&x, &b, sizeof(x));
    return x;
}

__global__ void k_bbox(const double* __restrict__ xyz, int64_t n, int dim, long long* lohi) {
    __shared__ long long slo[3][256], shi[3][256];
    long long lo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, hi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int a = 0; a < dim; ++a) {
            long long k = dbl_key(xyz[i * dim + a]);
            lo[a] = min(lo[a], k);
            hi[a] = max(hi[a], k);
        }
    for (int a = 0; a < 3; ++a) {
        slo[a][threadIdx.x] = lo[a];
        shi[a][threadIdx.x] = hi[a];
    }
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int a = 0; a < 3; ++a) {
                slo[a][threadIdx.x] = min(slo[a][threadIdx.x], slo[a][threadIdx.x + s]);
                shi[a][threadIdx.x] = max(shi[a][threadIdx.x], shi[a][threadIdx.x + s]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int a = 0; a < dim; ++a) {
            atomicMin(&lohi[a], slo[a][0]);
            atomicMax(&lohi[3 + a], shi[a][0]);
        }
}

// bounding box of a device coordinate array (host result)
static mfd_status bbox(cudaStream_t s, const double* d_xyz, int64_t n, int dim, double* lo, double* hi) {
    DevBuf buf;
    MFD_TRY(buf.alloc(6 * sizeof(long long)));
    long long init[6] = {LLONG_MAX, LLONG_MAX, LLONG_MAX, LLONG_MIN, LLONG_MIN, LLONG_MIN};
    MFD_CUDA(cudaMemcpyAsync(buf.p, init, sizeof(init), cudaMemcpyHostToDevice, s));
    int blocks = (int)std::min<int64_t>(1024, (n + 255) / 256);
    k_bbox<<<std::max(blocks, 1), 256, 0, s>>>(d_xyz, n, dim, buf.as<long long>());
    MFD_CUDA(cudaGetLastError());
    long long out[6];
    MFD_CUDA(cudaMemcpyAsync(out, buf.p, sizeof(out), cudaMemcpyDeviceToHost, s));
    MFD_CUDA(cudaStreamSynchronize(s));
    for (int a = 0; a < dim; ++a) {
        lo[a] = key_dbl(out[a]);
        hi[a] = key_dbl(out[3 + a]);
    }
    return MFD_OK;
}

// ------------------------------------------------------------ Morton order

__device__ __forceinline__ uint64_t spread2(uint64_t v) {  // 32 bits -> even positions
    v &= 0xFFFFFFFFull;
    v = (v | (v << 16)) & 0x0000FFFF0000FFFFull;
    v = (v | (v << 8)) & 0x00FF00FF00FF00FFull;
    v = (v | (v << 4)) & 0x0F0F0F0F0F0F0F0Full;
    v = (v | (v << 2)) & 0x3333333333333333ull;
    v = (v | (v << 1)) & 0x5555555555555555ull;
    return v;
}
__device__ __forceinline__ uint64_t spread3(uint64_t v) {  // 21 bits -> every third position
    v &= 0x1FFFFFull;
    v = (v | (v << 32)) & 0x1F00000000FFFFull;
    v = (v | (v << 16)) & 0x1F0000FF0000FFull;
    v = (v | (v << 8)) & 0x100F00F00F00F00Full;
    v = (v | (v << 4)) & 0x10C30C30C30C30C3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

// Order of the packed entries of a shared index row: ascending neighbour id
// within [0, m1), [m1, m2) and [m2, L), one thread per row (the split points
// are the stencil sizes below L of the stencils sharing the row, each a prefix
// of it, so each stencil keeps its entries; with per-centre sizes m1 and m2
// are the smallest and largest curl stencil).
// The entries keep their weights (the same permutation packs both), so a
// stencil sum is the same sum in another order. Adjacent centres' neighbour
// sets overlap, so ordering by id lines up the k-th gathers of a warp's
// centres, which then touch fewer cache lines per warp load (on the jittered
// 3D lattice 15 % fewer) in passes bound by the L1 data pipeline.
__global__ void k_row_perm(const int32_t* __restrict__ src, int stride, int64_t N, int m1, int m2, int L,
                           uint8_t* __restrict__ perm) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= N) return;
    const int32_t* s = src + r * stride;
    uint8_t p[255];
    for (int j = 0; j < L; ++j) p[j] = (uint8_t)j;
    const int lo[3] = {0, m1, m2}, hi[3] = {m1, m2, L};
    for (int part = 0; part < 3; ++part)
        for (int j = lo[part] + 1; j < hi[part]; ++j) {
            const uint8_t pj = p[j];
            const int32_t v = s[pj];
            int k = j - 1;
            while (k >= lo[part] && s[p[k]] > v) {
                p[k + 1] = p[k];
                --k;
            }
            p[k + 1] = pj;
        }
    for (int j = 0; j < L; ++j) perm[r * L + j] = p[j];
}

cudaError_t launch_row_perm(const int32_t* idx, int stride, int64_t n, int m1, int m2, int len, uint8_t* perm,
                            cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_row_perm<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(idx, stride, n, m1, m2, len, perm);
    return cudaGetLastError();
}

struct Box {
    double lo[3], scale[3];
};

__global__ void k_morton_keys(const double* __restrict__ xyz, int64_t n, int dim, Box b,
                              uint64_t* __restrict__ keys, int64_t* __restrict__ ids) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t q[3] = {0, 0, 0};
    const double qmax = dim == 2 ? 4294967295.0 : 2097151.0;
    for (int a = 0; a < dim; ++a) {
        double t = (xyz[i * dim + a] - b.lo[a]) * b.scale[a];
        t = fmin(fmax(t, 0.0), 1.0) * qmax;
        q[a] = (uint64_t)t;
    }
    keys[i] = dim == 2 ? (spread2(q[0]) | (spread2(q[1]) << 1))
                       : (spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2));
    ids[i] = i;
}

__global__ void k_permute(const double* __restrict__ xyz_user, const int64_t* __restrict__ perm, int64_t n,
                          int dim, double* __restrict__ xyz_sorted, int64_t* __restrict__ inv) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    int64_t u = perm[k];
    for (int a = 0; a < dim; ++a) xyz_sorted[k * dim + a] = xyz_user[u * dim + a];
    inv[u] = k;
}

mfd_status morton_order(mfd_ctx* ctx, int dim, int64_t n, const double* d_xyz_user, const double* period,
                        double* d_xyz_sorted, int64_t* d_perm, int64_t* d_inv) {
    cudaStream_t s = ctx->stream;
    double lo[3], hi[3];
    MFD_TRY(bbox(s, d_xyz_user, n, dim, lo, hi));
    Box b;
    for (int a = 0; a < 3; ++a) {
        b.lo[a] = 0;
        b.scale[a] = 0;
    }
    for (int a = 0; a < dim; ++a) {
        if (period[a] > 0) {
            lo[a] = 0.0;
            hi[a] = period[a];
        }
        b.lo[a] = lo[a];
        b.scale[a] = hi[a] > lo[a] ? 1.0 / (hi[a] - lo[a]) : 0.0;
    }
    DevBuf keys, keys2, ids;
    MFD_TRY(keys.alloc(n * 8));
    MFD_TRY(keys2.alloc(n * 8));
    MFD_TRY(ids.alloc(n * 8));
    int blocks = (int)((n + 255) / 256);
    k_morton_keys<<<blocks, 256, 0, s>>>(d_xyz_user, n, dim, b, keys.as<uint64_t>(), ids.as<int64_t>());
    MFD_CUDA(cudaGetLastError());
    size_t tmp_bytes = 0;
    MFD_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, keys.as<uint64_t>(), keys2.as<uint64_t>(),
                                             ids.as<int64_t>(), d_perm, (int64_t)n, 0, 64, s));
    DevBuf tmp;
    MFD_TRY(tmp.alloc(tmp_bytes));
    MFD_CUDA(cub::DeviceRadixSort::SortPairs(tmp.p, tmp_bytes, keys.as<uint64_t>(), keys2.as<uint64_t>(),
                                             ids.as<int64_t>(), d_perm, (int64_t)n, 0, 64, s));
    k_permute<<<blocks, 256, 0, s>>>(d_xyz_user, d_perm, n, dim, d_xyz_sorted, d_inv);
    MFD_CUDA(cudaGetLastError());
    MFD_CUDA(cudaStreamSynchronize(s));
    return MFD_OK;
}

// ------------------------------------------------------------ kNN (grid hash)

struct Grid {
    double lo[3], side[3], period[3];
    int64_t nb[3];
    double rmin;  // smallest cell side
};

__device__ __forceinline__ int64_t cell_coord(double x, const Grid& g, int a) {
    int64_t k = (int64_t)floor((x - g.lo[a]) / g.side[a]);
    return k < 0 ? 0 : (k >= g.nb[a] ? g.nb[a] - 1 : k);
}

__global__ void k_cell_count(const double* __restrict__ xyz, int64_t n, int dim, Grid g,
                             int64_t* __restrict__ cell_of, int* __restrict__ count) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t c[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) c[a] = cell_coord(xyz[i * dim + a], g, a);
    int64_t cell = (c[2] * g.nb[1] + c[1]) * g.nb[0] + c[0];
    cell_of[i] = cell;
    atomicAdd(&count[cell], 1);
}

__global__ void k_cell_fill(const int64_t* __restrict__ cell_of, int64_t n, const int* __restrict__ start,
                            int* __restrict__ cursor, int* __restrict__ list) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t cell = cell_of[i];
    int pos = start[cell] + atomicAdd(&cursor[cell], 1);
    list[pos] = (int)i;
}

// squared distance, FP64, left to right, no contraction
__device__ __forceinline__ double sq_dist(int dim, const double* c, const double* x, const double* per) {
    double s = 0.0;
    for (int a = 0; a < dim; ++a) {
        double d = __dsub_rn(x[a], c[a]);
        if (per[a] > 0.0) {
            double hp = 0.5 * per[a];
            if (d > hp) d = __dsub_rn(d, per[a]);
            else if (d < -hp) d = __dadd_rn(d, per[a]);
        }
        s = __dadd_rn(s, __dmul_rn(d, d));
    }
    return s;
}

constexpr int KNN_MAX = 128;

struct KnnArgs {
    const double* xc;
    const double* xs;
    const int64_t* perm_s;  // source device id -> caller id
    const int* start;
    const int* list;
    int64_t nc, ns;
    int dim, n;
    Grid g;
    int32_t* out;
};

// candidate (d2, uid) ordering
__device__ __forceinline__ bool before(double d1, int64_t u1, double d2, int64_t u2) {
    return d1 < d2 || (d1 == d2 && u1 < u2);
}

__global__ void __launch_bounds__(128) k_knn(KnnArgs a) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= a.nc) return;
    double bd[KNN_MAX];
    int64_t bu[KNN_MAX];
    int bs[KNN_MAX];
    const int n = a.n, dim = a.dim;
    double x[3] = {0, 0, 0};
    for (int q = 0; q < dim; ++q) x[q] = a.xc[c * dim + q];
    int64_t c0[3] = {0, 0, 0};
    for (int q = 0; q < dim; ++q) c0[q] = cell_coord(x[q], a.g, q);
    int cnt = 0, worst = 0;
    auto offer = [&](int j) {
        double d2 = sq_dist(dim, x, a.xs + (int64_t)j * dim, a.g.period);
        int64_t u = a.perm_s[j];
        if (cnt < n) {
            bd[cnt] = d2;
            bu[cnt] = u;
            bs[cnt] = j;
            if (cnt == 0 || before(bd[worst], bu[worst], d2, u)) worst = cnt;
            ++cnt;
        } else if (before(d2, u, bd[worst], bu[worst])) {
            bd[worst] = d2;
            bu[worst] = u;
            bs[worst] = j;
            worst = 0;
            for (int k = 1; k < n; ++k)
                if (before(bd[worst], bu[worst], bd[k], bu[k])) worst = k;
        }
    };
    bool brute = false;
    for (int64_t R = 0;; ++R) {
        bool wraps = false, all = true;
        for (int q = 0; q < dim; ++q) {
            if (a.g.period[q] > 0 && 2 * R + 1 > a.g.nb[q]) wraps = true;
            if (a.g.period[q] > 0 || c0[q] - R > 0 || c0[q] + R < a.g.nb[q] - 1) all = false;
        }
        if (wraps) {
            brute = true;
            break;
        }
        const int64_t r1 = dim > 1 ? R : 0, r2 = dim > 2 ? R : 0;
        for (int64_t oz = -r2; oz <= r2; ++oz)
            for (int64_t oy = -r1; oy <= r1; ++oy)
                for (int64_t ox = -R; ox <= R; ++ox) {
                    int64_t m = max(max(ox < 0 ? -ox : ox, oy < 0 ? -oy : oy), oz < 0 ? -oz : oz);
                    if (m != R) continue;
                    int64_t o[3] = {ox, oy, oz}, k[3] = {0, 0, 0};
                    bool skip = false;
                    for (int q = 0; q < dim; ++q) {
                        k[q] = c0[q] + o[q];
                        if (a.g.period[q] > 0) k[q] = ((k[q] % a.g.nb[q]) + a.g.nb[q]) % a.g.nb[q];
                        else if (k[q] < 0 || k[q] >= a.g.nb[q]) skip = true;
                    }
                    if (skip) continue;
                    int64_t cell = (k[2] * a.g.nb[1] + k[1]) * a.g.nb[0] + k[0];
                    for (int p = a.start[cell]; p < a.start[cell + 1]; ++p) offer(a.list[p]);
                }
        double rg = (double)R * a.g.rmin * (1.0 - 1e-12);
        if (all) break;
        if (cnt == n && bd[worst] < rg * rg) break;
    }
    if (brute) {
        cnt = 0;
        worst = 0;
        for (int64_t j = 0; j < a.ns; ++j) offer((int)j);
    }
    // sort the n survivors by (d2, caller id)
    for (int i = 1; i < n; ++i) {
        double d = bd[i];
        int64_t u = bu[i];
        int s = bs[i];
        int k = i - 1;
        while (k >= 0 && before(d, u, bd[k], bu[k])) {
            bd[k + 1] = bd[k];
            bu[k + 1] = bu[k];
            bs[k + 1] = bs[k];
            --k;
        }
        bd[k + 1] = d;
        bu[k + 1] = u;
        bs[k + 1] = s;
    }
    int32_t* o = a.out + c * n;
    for (int i = 0; i < n; ++i) o[i] = bs[i];
}

mfd_status knn_build(const mfd_nodes* centres, const mfd_nodes* sources, int n, int32_t* d_idx) {
    cudaStream_t s = centres->ctx->stream;
    const int dim = sources->dim;
    if (n < 1 || n > KNN_MAX || n > sources->n) return fail(MFD_ERR_ARG, "stencil size out of range");
    if (sources->n > INT32_MAX) return fail(MFD_ERR_ARG, "source set too large for int32 ids");
    Grid g;
    double lo[3], hi[3];
    MFD_TRY(bbox(s, sources->xyz.as<double>(), sources->n, dim, lo, hi));
    double vol = 1.0;
    for (int a = 0; a < dim; ++a) {
        if (sources->period[a] > 0) {
            lo[a] = 0;
            hi[a] = sources->period[a];
        }
        vol *= std::max(hi[a] - lo[a], 1e-300);
    }
    // about one source per cell
    double cs = std::pow(vol / (double)sources->n, 1.0 / dim);
    int64_t ncell = 1;
    g.rmin = 1e300;
    for (int a = 0; a < 3; ++a) {
        g.lo[a] = 0;
        g.side[a] = 1;
        g.nb[a] = 1;
        g.period[a] = 0;
    }
    for (int a = 0; a < dim; ++a) {
        double ext = hi[a] - lo[a];
        int64_t nb = (int64_t)std::floor(ext / cs);
        if (nb < 1) nb = 1;
        if (nb > (1 << 20)) nb = 1 << 20;
        g.lo[a] = lo[a];
        g.nb[a] = nb;
        g.side[a] = ext > 0 ? ext / (double)nb : 1.0;
        g.period[a] = sources->period[a];
        g.rmin = std::min(g.rmin, g.side[a]);
        ncell *= nb;
    }
    DevBuf cell_of, count, start, cursor, list, tmp;
    MFD_TRY(cell_of.alloc(sources->n * 8));
    MFD_TRY(count.alloc((ncell + 1) * 4));
    MFD_TRY(start.alloc((ncell + 1) * 4));
    MFD_TRY(cursor.alloc((ncell + 1) * 4));
    MFD_TRY(list.alloc(sources->n * 4));
    MFD_CUDA(cudaMemsetAsync(count.p, 0, (ncell + 1) * 4, s));
    MFD_CUDA(cudaMemsetAsync(cursor.p, 0, (ncell + 1) * 4, s));
    int blocks = (int)((sources->n + 255) / 256);
    k_cell_count<<<blocks, 256, 0, s>>>(sources->xyz.as<double>(), sources->n, dim, g, cell_of.as<int64_t>(),
                                        count.as<int>());
    MFD_CUDA(cudaGetLastError());
    size_t tb = 0;
    MFD_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tb, count.as<int>(), start.as<int>(), (int64_t)ncell + 1, s));
    MFD_TRY(tmp.alloc(tb));
    MFD_CUDA(cub::DeviceScan::ExclusiveSum(tmp.p, tb, count.as<int>(), start.as<int>(), (int64_t)ncell + 1, s));
    k_cell_fill<<<blocks, 256, 0, s>>>(cell_of.as<int64_t>(), sources->n, start.as<int>(), cursor.as<int>(),
                                       list.as<int>());
    MFD_CUDA(cudaGetLastError());
    KnnArgs a;
    a.xc = centres->xyz.as<double>();
    a.xs = sources->xyz.as<double>();
    a.perm_s = sources->perm.as<int64_t>();
    a.start = start.as<int>();
    a.list = list.as<int>();
    a.nc = centres->n;
    a.ns = sources->n;
    a.dim = dim;
    a.n = n;
    a.g = g;
    a.out = d_idx;
    k_knn<<<(int)((centres->n + 127) / 128), 128, 0, s>>>(a);
    MFD_CUDA(cudaGetLastError());
    MFD_CUDA(cudaStreamSynchronize(s));
    return MFD_OK;
}

// ------------------------------------------------------------ kNN with mirror walls (PEC by images)
//
// The nodes of a set with mirror walls on [0, hi] per mirrored axis and their
// images x_a -> 2 hi - x_a (for every non-empty subset r of those axes, the
// reflection code) form a periodic set of period 2 hi on those axes (a perfect
// conductor as a mirror); a wall node is its own image and is not repeated.
// The kNN runs on the nodes and the images of the nodes within a band D of the
// walls they are reflected across (an image left out lies at least D outside
// the box, so it cannot be among the n nearest of a centre whose n-th nearest is
// closer than D; the band grows until that holds). Entries are then node device
// ids with the code in the top bits. Images are listed after the nodes, by
// (code, node caller id), so ties of equal distance break as in a set that holds
// every image.

__global__ void k_img_radius(const int32_t* __restrict__ idx, int n, int64_t nc, const double* __restrict__ xc,
                             const double* __restrict__ xs, int dim, double p0, double p1, double p2,
                             unsigned long long* __restrict__ worst) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const double per[3] = {p0, p1, p2};
    const double d2 = sq_dist(dim, xc + c * dim, xs + (int64_t)idx[c * n + n - 1] * dim, per);
    atomicMax(worst, (unsigned long long)__double_as_longlong(d2));  // non-negative doubles order as integers
}

__global__ void k_img_map(const int32_t* __restrict__ ext_idx, int64_t total, const int64_t* __restrict__ ext_perm,
                          const int64_t* __restrict__ orig, const uint8_t* __restrict__ code,
                          const int64_t* __restrict__ inv, int32_t* __restrict__ out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int64_t u = ext_perm[ext_idx[e]];  // caller id in the extended set
    out[e] = (int32_t)inv[orig[u]] | (int32_t)((unsigned)code[u] << IMG_SHIFT);
}

mfd_status knn_build_mirror(const mfd_nodes* centres, const mfd_nodes* sources, int n, int32_t* d_idx) {
    mfd_ctx* ctx = sources->ctx;
    cudaStream_t s = ctx->stream;
    const int dim = sources->dim;
    const int64_t N = sources->n;
    const uint32_t axes = sources->mirror_axes;
    if (n < 1 || n > KNN_MAX || n > N) return fail(MFD_ERR_ARG, "stencil size out of range");
    // caller-order coordinates
    std::vector<double> xd((size_t)N * dim), xu((size_t)N * dim);
    MFD_CUDA(cudaMemcpy(xd.data(), sources->xyz.p, xd.size() * 8, cudaMemcpyDeviceToHost));
    for (int64_t k = 0; k < N; ++k)
        for (int a = 0; a < dim; ++a) xu[sources->h_perm[k] * dim + a] = xd[k * dim + a];
    double per[3] = {0, 0, 0}, ext[3] = {0, 0, 0}, vol = 1.0;
    for (int a = 0; a < dim; ++a) {
        double lo = 1e300, hi = -1e300;
        for (int64_t i = 0; i < N; ++i) {
            lo = std::min(lo, xu[i * dim + a]);
            hi = std::max(hi, xu[i * dim + a]);
        }
        per[a] = ((axes >> a) & 1u) ? 2.0 * sources->mirror_hi[a] : sources->period[a];
        ext[a] = ((axes >> a) & 1u) ? sources->mirror_hi[a] : (per[a] > 0 ? per[a] : hi - lo);
        vol *= std::max(ext[a], 1e-300);
    }
    const double h = std::pow(vol / (double)N, 1.0 / dim);
    const double pi = 3.14159265358979323846;
    const double r_est = dim == 2 ? h * std::sqrt(n / pi) : h * std::cbrt(3.0 * n / (4.0 * pi));
    double D = 2.0 * r_est + 2.0 * h;
    const int64_t nc = centres->n;
    for (int attempt = 0; attempt < 6; ++attempt, D *= 2.0) {
        std::vector<double> xe(xu);
        std::vector<int64_t> orig(N);
        std::vector<uint8_t> code(N, 0);
        for (int64_t i = 0; i < N; ++i) orig[i] = i;
        for (uint32_t r = 1; r < (1u << dim); ++r) {
            if (r & ~axes) continue;
            for (int64_t i = 0; i < N; ++i) {
                bool keep = true;
                for (int a = 0; a < dim && keep; ++a) {
                    if (!((r >> a) & 1u)) continue;
                    const double x = xu[i * dim + a], hi = sources->mirror_hi[a];
                    keep = x > 0.0 && x < hi && std::min(x, hi - x) < D;
                }
                if (!keep) continue;
                for (int a = 0; a < dim; ++a) {
                    const double x = xu[i * dim + a];
                    xe.push_back(((r >> a) & 1u) ? 2.0 * sources->mirror_hi[a] - x : x);
                }
                orig.push_back(i);
                code.push_back((uint8_t)r);
            }
        }
        const int64_t ne = (int64_t)orig.size();
        if (ne > INT32_MAX) return fail(MFD_ERR_ARG, "extended node set too large");
        mfd_nodes* exts = nullptr;
        MFD_TRY(mfd_nodes_create(ctx, dim, ne, xe.data(), per, &exts));
        struct Rel {
            mfd_nodes* p;
            ~Rel() { mfd_nodes_destroy(p); }
        } rel{exts};
        DevBuf eidx, dorig, dcode, worst;
        MFD_TRY(eidx.alloc((size_t)nc * n * 4));
        MFD_TRY(knn_build(centres, exts, n, eidx.as<int32_t>()));
        MFD_TRY(worst.alloc(8));
        MFD_CUDA(cudaMemsetAsync(worst.p, 0, 8, s));
        k_img_radius<<<(unsigned)((nc + 255) / 256), 256, 0, s>>>(eidx.as<int32_t>(), n, nc, centres->xyz.as<double>(),
                                                                  exts->xyz.as<double>(), dim, per[0], per[1], per[2],
                                                                  worst.as<unsigned long long>());
        MFD_CUDA(cudaGetLastError());
        unsigned long long wb = 0;
        MFD_CUDA(cudaMemcpyAsync(&wb, worst.p, 8, cudaMemcpyDeviceToHost, s));
        MFD_CUDA(cudaStreamSynchronize(s));
        double w2;
        std::memcpy(&w2, &wb, 8);
        if (!(w2 < D * D)) continue;  // an image outside the band could be closer: widen it
        MFD_TRY(dorig.alloc((size_t)ne * 8));
        MFD_TRY(dcode.alloc((size_t)ne));
        MFD_CUDA(cudaMemcpyAsync(dorig.p, orig.data(), ne * 8, cudaMemcpyHostToDevice, s));
        MFD_CUDA(cudaMemcpyAsync(dcode.p, code.data(), ne, cudaMemcpyHostToDevice, s));
        const int64_t total = nc * n;
        k_img_map<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(eidx.as<int32_t>(), total, exts->perm.as<int64_t>(),
                                                                  dorig.as<int64_t>(), dcode.as<uint8_t>(),
                                                                  sources->inv.as<int64_t>(), d_idx);
        MFD_CUDA(cudaGetLastError());
        MFD_CUDA(cudaStreamSynchronize(s));
        return MFD_OK;
    }
    return fail(MFD_ERR_STATE, "the image band did not cover the stencils");
}

// ------------------------------------------------------------ weights (batched FP64 solve)

constexpr int WS_THREADS = 128;  // threads per system; 256 for systems that leave room for at most three CTAs of 128 per SM
constexpr int WS_MAX_K = 160;
constexpr int WS_MAX_M = 64;

struct WArgs {
    const double* xc;
    const double* xs;
    const int32_t* idx;
    int64_t nc;
    int stride, n_use, dim, phs_k, M, op, alpha, nout;  // n_use: row length of w
    const int32_t* nsz;        // stencil size per centre, or NULL (all n_use)
    double period[3];
    unsigned mirror;           // mirrored axes: an entry with image code r reflects x_a -> 2 mhi_a - x_a, a in r
    double mhi[3];
    double lap_rbf;            // prod_{i<alpha} (k-2i)(k-2i+d-2)
    double delta;
    double* w;                 // [nout][nc][n_use], zero past a centre's own size
    int* status;
};

__constant__ signed char c_exps[WS_MAX_M][3];
__constant__ double c_poly_rhs[WS_MAX_M];  // Delta^alpha p_q at the origin

__device__ __forceinline__ double ipow(double x, int k) {
    double r = 1.0;
    for (int i = 0; i < k; ++i) r *= x;
    return r;
}

__device__ __forceinline__ double mono(const double* z, int q, int dim) {
    double v = 1.0;
    for (int a = 0; a < dim; ++a) v *= ipow(z[a], c_exps[q][a]);
    return v;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_weights(WArgs a) {
    extern __shared__ double sm[];
    const int M = a.M, nout = a.nout, dim = a.dim;
    __shared__ double red[NT];
    __shared__ int redi[NT];
    __shared__ int piv_s;
    const int tid = threadIdx.x;
    for (int64_t c = blockIdx.x; c < a.nc; c += gridDim.x) {
        // this centre's system (the shared memory is sized for the largest)
        const int n = a.nsz ? a.nsz[c] : a.n_use, K = n + M, ld = K + nout;
        double* A = sm;                 // K x ld (augmented)
        double* z = A + K * ld;         // n x 3 scaled offsets
        double* fac = z + 3 * n;        // K elimination factors
        // offsets to the centre, minimum image
        for (int j = tid; j < n; j += NT) {
            const int32_t raw = a.idx[c * a.stride + j];
            const unsigned code = a.mirror ? (unsigned)raw >> IMG_SHIFT : 0u;
            const int32_t sj = a.mirror ? (raw & IMG_MASK) : raw;
            for (int q = 0; q < 3; ++q) {
                double d = 0.0;
                if (q < dim) {
                    double x = a.xs[(int64_t)sj * dim + q];
                    if ((code >> q) & 1u) x = 2.0 * a.mhi[q] - x;
                    d = x - a.xc[c * dim + q];
                    double p = a.period[q];
                    if (p > 0) {
                        if (d > 0.5 * p) d -= p;
                        else if (d < -0.5 * p) d += p;
                    }
                }
                z[j * 3 + q] = d;
            }
        }
        __syncthreads();
        // stencil radius
        double r2 = 0.0;
        for (int j = tid; j < n; j += NT) {
            double t = 0.0;
            for (int q = 0; q < dim; ++q) t += z[j * 3 + q] * z[j * 3 + q];
            r2 = fmax(r2, t);
        }
        red[tid] = r2;
        __syncthreads();
        for (int s = NT / 2; s > 0; s >>= 1) {
            if (tid < s) red[tid] = fmax(red[tid], red[tid + s]);
            __syncthreads();
        }
        const double scale = sqrt(red[0]);
        __syncthreads();
        if (!(scale > 0.0)) {
            if (tid == 0) atomicExch(a.status, MFD_ERR_SINGULAR);
            continue;
        }
        const double inv = 1.0 / scale;
        for (int j = tid; j < 3 * n; j += NT) z[j] *= inv;
        __syncthreads();
        // system matrix [A P; P^T 0] and right-hand sides
        for (int e = tid; e < K * K; e += NT) {
            int i = e / K, j = e % K;
            double v;
            if (i < n && j < n) {
                double t = 0.0;
                for (int q = 0; q < dim; ++q) {
                    double d = z[i * 3 + q] - z[j * 3 + q];
                    t += d * d;
                }
                v = ipow(sqrt(t), a.phs_k);
            } else if (i < n) {
                v = mono(z + i * 3, j - n, dim);
            } else if (j < n) {
                v = mono(z + j * 3, i - n, dim);
            } else {
                v = 0.0;
            }
            A[i * ld + j] = v;
        }
        const double dz = a.delta * inv;
        for (int e = tid; e < K * nout; e += NT) {
            int i = e / nout, o = e % nout;
            double v = 0.0;
            if (i < n) {
                const double* zi = z + i * 3;
                double t = 0.0;
                for (int q = 0; q < dim; ++q) t += zi[q] * zi[q];
                double r = sqrt(t);
                if (a.op == MFD_OP_GRAD) {
                    // d/dx_o of |x - z_i|^k at x = 0: k |z_i|^(k-2) (0 - z_i)_o
                    v = -(double)a.phs_k * ipow(r, a.phs_k - 2) * zi[o];
                } else if (a.op == MFD_OP_LAP_POW) {
                    v = a.lap_rbf * ipow(r, a.phs_k - 2 * a.alpha);
                } else {
                    double tp = 0.0, tm = 0.0;
                    for (int q = 0; q < dim; ++q) {
                        double sh = q == o ? dz : 0.0;
                        double dp = sh - zi[q], dm = -sh - zi[q];
                        tp += dp * dp;
                        tm += dm * dm;
                    }
                    v = (ipow(sqrt(tp), a.phs_k) - ipow(sqrt(tm), a.phs_k)) / (2.0 * dz);
                }
            } else {
                int q = i - n;
                if (a.op == MFD_OP_GRAD) {
                    int deg = c_exps[q][0] + c_exps[q][1] + c_exps[q][2];
                    v = (deg == 1 && c_exps[q][o] == 1) ? 1.0 : 0.0;
                } else if (a.op == MFD_OP_LAP_POW) {
                    v = c_poly_rhs[q];
                } else {
                    double zp[3] = {0, 0, 0}, zm[3] = {0, 0, 0};
                    zp[o] = dz;
                    zm[o] = -dz;
                    v = (mono(zp, q, dim) - mono(zm, q, dim)) / (2.0 * dz);
                }
            }
            A[i * ld + K + o] = v;
        }
        __syncthreads();
        // Gaussian elimination with partial pivoting on the augmented matrix
        bool singular = false;
        for (int p = 0; p < K; ++p) {
            double best = -1.0;
            int bi = p;
            for (int r = p + tid; r < K; r += NT) {
                double v = fabs(A[r * ld + p]);
                if (v > best) {
                    best = v;
                    bi = r;
                }
            }
            red[tid] = best;
            redi[tid] = bi;
            __syncthreads();
            for (int s = NT / 2; s > 0; s >>= 1) {
                if (tid < s) {
                    double o2 = red[tid + s];
                    int oi = redi[tid + s];
                    if (o2 > red[tid] || (o2 == red[tid] && oi < redi[tid])) {
                        red[tid] = o2;
                        redi[tid] = oi;
                    }
                }
                __syncthreads();
            }
            if (tid == 0) piv_s = redi[0];
            const double pv = red[0];
            __syncthreads();
            if (!(pv > 0.0)) {
                singular = true;
                break;
            }
            const int piv = piv_s;
            if (piv != p)
                for (int col = p + tid; col < ld; col += NT) {
                    double t = A[p * ld + col];
                    A[p * ld + col] = A[piv * ld + col];
                    A[piv * ld + col] = t;
                }
            __syncthreads();
            const double d = A[p * ld + p];
            for (int r = p + 1 + tid; r < K; r += NT) fac[r] = A[r * ld + p] / d;
            __syncthreads();
            const int rows = K - p - 1, cols = ld - p - 1;
            for (int e = tid; e < rows * cols; e += NT) {
                int r = p + 1 + e / cols, col = p + 1 + e % cols;
                A[r * ld + col] -= fac[r] * A[p * ld + col];
            }
            __syncthreads();
        }
        if (singular) {
            if (tid == 0) atomicExch(a.status, MFD_ERR_SINGULAR);
            __syncthreads();
            continue;
        }
        // back substitution: warp o solves right-hand side o
        const int warp = tid >> 5, lane = tid & 31;
        if (warp < nout) {
            const int o = warp;
            for (int p = K - 1; p >= 0; --p) {
                double s = 0.0;
                for (int q = p + 1 + lane; q < K; q += 32) s += A[p * ld + q] * A[q * ld + K + o];
                for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
                if (lane == 0) A[p * ld + K + o] = (A[p * ld + K + o] - s) / A[p * ld + p];
                __syncwarp();
            }
        }
        __syncthreads();
        const int l = a.op == MFD_OP_LAP_POW ? 2 * a.alpha : 1;
        const double sl = ipow(inv, l);
        const int rl = a.n_use;
        for (int e = tid; e < rl * nout; e += NT) {
            int o = e / rl, j = e % rl;
            a.w[((int64_t)o * a.nc + c) * rl + j] = j < n ? A[j * ld + K + o] * sl : 0.0;
        }
        __syncthreads();
    }
}

// monomial exponents in graded order and Delta^alpha of each at the origin,
// the latter by applying the Laplacian to the polynomial's coefficient map
static void poly_tables(int dim, int m, int alpha, std::vector<std::array<int, 3>>& ex, std::vector<double>& lap) {
    ex.clear();
    for (int deg = 0; deg <= m; ++deg) {
        if (dim == 2) {
            for (int a = deg; a >= 0; --a) ex.push_back({a, deg - a, 0});
        } else {
            for (int a = deg; a >= 0; --a)
                for (int b = deg - a; b >= 0; --b) ex.push_back({a, b, deg - a - b});
        }
    }
    lap.assign(ex.size(), 0.0);
    for (size_t q = 0; q < ex.size(); ++q) {
        std::map<std::array<int, 3>, double> poly;
        poly[ex[q]] = 1.0;
        for (int it = 0; it < alpha; ++it) {
            std::map<std::array<int, 3>, double> next;
            for (auto& kv : poly)
                for (int ax = 0; ax < dim; ++ax) {
                    int e = kv.first[ax];
                    if (e < 2) continue;
                    auto k2 = kv.first;
                    k2[ax] -= 2;
                    next[k2] += kv.second * e * (e - 1);
                }
            poly.swap(next);
        }
        auto it0 = poly.find({0, 0, 0});
        lap[q] = it0 == poly.end() ? 0.0 : it0->second;
    }
}

mfd_status weights_solve(const mfd_stencils* st, int n_use, const int32_t* d_nsz, int phs_k, int poly_m, int op,
                         int alpha, double delta, double* d_w) {
    const mfd_nodes* cen = st->centres;
    const mfd_nodes* src = st->sources;
    mfd_ctx* ctx = cen->ctx;
    cudaStream_t s = ctx->stream;
    const int dim = cen->dim;
    std::vector<std::array<int, 3>> ex;
    std::vector<double> lap;
    poly_tables(dim, poly_m, op == MFD_OP_LAP_POW ? alpha : 0, ex, lap);
    const int M = (int)ex.size();
    if (M > WS_MAX_M) return fail(MFD_ERR_ARG, "too many monomials");
    const int K = n_use + M;
    if (K > WS_MAX_K) return fail(MFD_ERR_ARG, "local system larger than " + std::to_string(WS_MAX_K));
    signed char h_ex[WS_MAX_M][3] = {};
    double h_rhs[WS_MAX_M] = {};
    for (int q = 0; q < M; ++q) {
        for (int a = 0; a < 3; ++a) h_ex[q][a] = (signed char)ex[q][a];
        h_rhs[q] = lap[q];
    }
    MFD_CUDA(cudaMemcpyToSymbolAsync(c_exps, h_ex, sizeof(h_ex), 0, cudaMemcpyHostToDevice, s));
    MFD_CUDA(cudaMemcpyToSymbolAsync(c_poly_rhs, h_rhs, sizeof(h_rhs), 0, cudaMemcpyHostToDevice, s));
    WArgs a;
    a.xc = cen->xyz.as<double>();
    a.xs = src->xyz.as<double>();
    a.idx = st->idx.as<int32_t>();
    a.nc = cen->n;
    a.stride = st->n;
    a.n_use = n_use;
    a.nsz = d_nsz;
    a.dim = dim;
    a.phs_k = phs_k;
    a.M = M;
    a.op = op;
    a.alpha = alpha;
    a.nout = op == MFD_OP_LAP_POW ? 1 : dim;
    a.mirror = src->mirror_axes;
    for (int q = 0; q < 3; ++q) {
        const bool m = q < dim && ((src->mirror_axes >> q) & 1u);
        a.mhi[q] = m ? src->mirror_hi[q] : 0.0;
        a.period[q] = q < dim ? (m ? 2.0 * src->mirror_hi[q] : src->period[q]) : 0.0;
    }
    double cf = 1.0;
    for (int i = 0; i < alpha; ++i) cf *= (double)(phs_k - 2 * i) * (double)(phs_k - 2 * i + dim - 2);
    a.lap_rbf = cf;
    a.delta = delta;
    a.w = d_w;
    DevBuf status;
    MFD_TRY(status.alloc(sizeof(int)));
    MFD_CUDA(cudaMemsetAsync(status.p, 0, sizeof(int), s));
    a.status = status.as<int>();
    size_t smem = sizeof(double) * ((size_t)K * (K + a.nout) + 3 * n_use + K);
    MFD_CUDA(cudaFuncSetAttribute(k_weights<WS_THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    MFD_CUDA(cudaFuncSetAttribute(k_weights<2 * WS_THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    MFD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_weights<WS_THREADS>, WS_THREADS, smem));
    if (per_sm < 1) return fail(MFD_ERR_ARG, "local system does not fit in shared memory");
    // a system so large that at most three CTAs fit on an SM gets twice the threads (more
    // warps to cover the FP64 latency: 3D systems of 106 unknowns 11 % faster, the 2D HV
    // systems of 85 unknowns 2 %, the same weights; 512 threads were slower)
    const bool wide = per_sm <= 3;
    if (wide) {
        MFD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_weights<2 * WS_THREADS>, 2 * WS_THREADS, smem));
        if (per_sm < 1) return fail(MFD_ERR_ARG, "local system does not fit in shared memory");
    }
    int64_t grid = std::min<int64_t>(cen->n, (int64_t)per_sm * ctx->sm_count * 8);
    if (wide) k_weights<2 * WS_THREADS><<<(int)std::max<int64_t>(grid, 1), 2 * WS_THREADS, smem, s>>>(a);
    else k_weights<WS_THREADS><<<(int)std::max<int64_t>(grid, 1), WS_THREADS, smem, s>>>(a);
    MFD_CUDA(cudaGetLastError());
    int h_status = 0;
    MFD_CUDA(cudaMemcpyAsync(&h_status, status.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    MFD_CUDA(cudaStreamSynchronize(s));
    if (h_status != 0) return fail(MFD_ERR_SINGULAR, "a local weight system was singular");
    return MFD_OK;
}

}  // namespace mfd

// ------------------------------------------------------------ kNN without allocation
//
// mfd_knn_static: the grid-hash kNN above, on caller-provided device arrays,
// with all of its scratch (bounding box, identity ids, cell counts, cell
// starts, fill cursors and the cell lists) in one file-scope device array.
// For callers that must not allocate device memory at all.

namespace mfd {

constexpr size_t KNN_STATIC_BYTES = (size_t)32 << 20;  // 32 MiB, held by every GPU that loads the library

static __device__ __align__(256) unsigned char g_knn_scratch[KNN_STATIC_BYTES];

// device address of g_knn_scratch, looked up once per device with that device current
static std::mutex g_knn_scratch_mu;
static void* g_knn_scratch_ptr[128] = {};

static mfd_status knn_scratch_address(int device, unsigned char** out) {
    if (device < 0 || device >= 128) return fail(MFD_ERR_ARG, "device id out of range");
    std::lock_guard<std::mutex> lock(g_knn_scratch_mu);
    if (g_knn_scratch_ptr[device]) {
        // a context torn down and made again (cudaDeviceReset) reloads the module
        // elsewhere: an address that no longer names device memory of this device
        // is looked up again
        cudaPointerAttributes at;
        const cudaError_t e = cudaPointerGetAttributes(&at, g_knn_scratch_ptr[device]);
        if (e != cudaSuccess || at.type != cudaMemoryTypeDevice || at.device != device) {
            cudaGetLastError();
            g_knn_scratch_ptr[device] = nullptr;
        }
    }
    if (!g_knn_scratch_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_knn_scratch);
        if (e != cudaSuccess || !p)
            return fail(MFD_ERR_CUDA, std::string("cudaGetSymbolAddress(kNN scratch): ") + cudaGetErrorString(e));
        g_knn_scratch_ptr[device] = p;
    }
    *out = static_cast<unsigned char*>(g_knn_scratch_ptr[device]);
    return MFD_OK;
}

__global__ void k_iota64(int64_t* __restrict__ a, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) a[i] = i;
}

__global__ void k_fill_ll(long long* __restrict__ a, long long lo, long long hi) {
    if (threadIdx.x < 3) a[threadIdx.x] = lo;
    else if (threadIdx.x < 6) a[threadIdx.x] = hi;
}

// exclusive prefix sum of n ints by one block (serial over tiles of 1024)
__global__ void __launch_bounds__(1024) k_scan_excl(const int* __restrict__ in, int* __restrict__ out, int64_t n) {
    __shared__ int buf[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const int v = i < n ? in[i] : 0;
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            int t = threadIdx.x >= off ? buf[threadIdx.x - off] : 0;
            __syncthreads();
            buf[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < n) out[i] = carry + buf[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += buf[1023];
        __syncthreads();
    }
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace mfd

extern "C" mfd_status mfd_knn_static(int dim, int64_t nc, const double* centres, int64_t ns, const double* sources,
                                     const double* period, int n, int32_t* idx, void* stream) {
    using namespace mfd;
    if (dim != 2 && dim != 3) return fail(MFD_ERR_ARG, "dim must be 2 or 3");
    if (nc < 0 || ns < 1 || ns > INT32_MAX) return fail(MFD_ERR_ARG, "node counts out of range");
    if (n < 1 || n > KNN_MAX || n > ns) return fail(MFD_ERR_ARG, "stencil size out of range (1..min(128, ns))");
    if (!sources || (nc > 0 && (!centres || !idx))) return fail(MFD_ERR_ARG, "NULL device array");
    double per[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) {
        per[a] = period ? period[a] : 0.0;
        if (per[a] < 0) return fail(MFD_ERR_ARG, "negative period");
    }
    if (nc == 0) return MFD_OK;
    int device = 0;
    MFD_CUDA(cudaGetDevice(&device));
    unsigned char* base = nullptr;
    MFD_TRY(knn_scratch_address(device, &base));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // bounding box of the sources (first 256 bytes of the scratch)
    long long* lohi = reinterpret_cast<long long*>(base);
    k_fill_ll<<<1, 32, 0, s>>>(lohi, LLONG_MAX, LLONG_MIN);
    int bblocks = (int)std::min<int64_t>(1024, (ns + 255) / 256);
    k_bbox<<<std::max(bblocks, 1), 256, 0, s>>>(sources, ns, dim, lohi);
    MFD_CUDA(cudaGetLastError());
    long long hb[6];
    MFD_CUDA(cudaMemcpyAsync(hb, lohi, sizeof(hb), cudaMemcpyDeviceToHost, s));
    MFD_CUDA(cudaStreamSynchronize(s));
    double lo[3], hi[3];
    for (int a = 0; a < dim; ++a) {
        lo[a] = key_dbl(hb[a]);
        hi[a] = key_dbl(hb[3 + a]);
        if (per[a] > 0 && !(lo[a] >= 0.0 && hi[a] < per[a]))
            return fail(MFD_ERR_ARG, "coordinates of a periodic axis must lie in [0, period)");
    }
    // the same cell grid as mfd_stencils_build: about one source per cell
    Grid g;
    double vol = 1.0;
    for (int a = 0; a < dim; ++a) {
        if (per[a] > 0) {
            lo[a] = 0;
            hi[a] = per[a];
        }
        vol *= std::max(hi[a] - lo[a], 1e-300);
    }
    const double cs = std::pow(vol / (double)ns, 1.0 / dim);
    int64_t ncell = 1;
    g.rmin = 1e300;
    for (int a = 0; a < 3; ++a) {
        g.lo[a] = 0;
        g.side[a] = 1;
        g.nb[a] = 1;
        g.period[a] = 0;
    }
    for (int a = 0; a < dim; ++a) {
        double ext = hi[a] - lo[a];
        int64_t nb = (int64_t)std::floor(ext / cs);
        if (nb < 1) nb = 1;
        if (nb > (1 << 20)) nb = 1 << 20;
        g.lo[a] = lo[a];
        g.nb[a] = nb;
        g.side[a] = ext > 0 ? ext / (double)nb : 1.0;
        g.period[a] = per[a];
        g.rmin = std::min(g.rmin, g.side[a]);
        ncell *= nb;
    }
    // scratch layout: [bbox 256 B][ids 8 ns][cell_of 8 ns][list 4 ns][count, start, cursor: 4 (ncell + 1) each]
    const size_t o_ids = 256;
    const size_t o_cell = o_ids + align256(8 * (size_t)ns);
    const size_t o_list = o_cell + align256(8 * (size_t)ns);
    const size_t o_count = o_list + align256(4 * (size_t)ns);
    const size_t o_start = o_count + align256(4 * (size_t)(ncell + 1));
    const size_t o_cursor = o_start + align256(4 * (size_t)(ncell + 1));
    const size_t need = o_cursor + align256(4 * (size_t)(ncell + 1));
    if (need > KNN_STATIC_BYTES)
        return fail(MFD_ERR_ARG, "mfd_knn_static: " + std::to_string(ns) + " sources need " + std::to_string(need) +
                                     " bytes of scratch; the static scratch holds " +
                                     std::to_string(KNN_STATIC_BYTES) + " (about 1M sources)");
    int64_t* ids = reinterpret_cast<int64_t*>(base + o_ids);
    int64_t* cell_of = reinterpret_cast<int64_t*>(base + o_cell);
    int* list = reinterpret_cast<int*>(base + o_list);
    int* count = reinterpret_cast<int*>(base + o_count);
    int* start = reinterpret_cast<int*>(base + o_start);
    int* cursor = reinterpret_cast<int*>(base + o_cursor);
    // counts and cursors must start at zero (the array keeps the previous call's contents)
    MFD_CUDA(cudaMemsetAsync(count, 0, 4 * (size_t)(ncell + 1), s));
    MFD_CUDA(cudaMemsetAsync(cursor, 0, 4 * (size_t)(ncell + 1), s));
    const unsigned sb = (unsigned)((ns + 255) / 256);
    k_iota64<<<sb, 256, 0, s>>>(ids, ns);
    k_cell_count<<<sb, 256, 0, s>>>(sources, ns, dim, g, cell_of, count);
    k_scan_excl<<<1, 1024, 0, s>>>(count, start, ncell + 1);
    k_cell_fill<<<sb, 256, 0, s>>>(cell_of, ns, start, cursor, list);
    KnnArgs a;
    a.xc = centres;
    a.xs = sources;
    a.perm_s = ids;
    a.start = start;
    a.list = list;
    a.nc = nc;
    a.ns = ns;
    a.dim = dim;
    a.n = n;
    a.g = g;
    a.out = idx;
    k_knn<<<(unsigned)((nc + 127) / 128), 128, 0, s>>>(a);
    MFD_CUDA(cudaGetLastError());
    return MFD_OK;
}
