// api.cu -- C ABI: errors, contexts, node sets, stencils and weights (include/mfd.h).
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "internal.cuh"
#include "kernels.cuh"

namespace mfd {

static thread_local std::string g_last_error;

std::atomic<long long> g_alloc_fail_in{-1};

void set_error(const std::string& msg) { g_last_error = msg; }

mfd_status fail(mfd_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

static const char kStateMagic[8] = {'M', 'F', 'D', 'S', 'T', 'A', 'T', 'E'};

void state_head_init(StateHead* h, int32_t kind) {
    std::memset(h, 0, sizeof(*h));
    std::memcpy(h->magic, kStateMagic, 8);
    h->version = kStateVersion;
    h->kind = kind;
}

mfd_status state_head_check(const void* blob, size_t size, int32_t kind, StateHead* out) {
    if (!blob || size < sizeof(StateHead)) return fail(MFD_ERR_ARG, "state blob too small");
    std::memcpy(out, blob, sizeof(StateHead));
    if (std::memcmp(out->magic, kStateMagic, 8) != 0) return fail(MFD_ERR_ARG, "not a state blob");
    if (out->version != kStateVersion) return fail(MFD_ERR_ARG, "state blob of another version");
    if (out->kind != kind) return fail(MFD_ERR_ARG, "state blob of another object kind");
    return MFD_OK;
}

mfd_status order_streams(cudaStream_t from, cudaStream_t to) {
    if (from == to) return MFD_OK;
    cudaEvent_t e;
    MFD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaError_t r = cudaEventRecord(e, from);
    if (r == cudaSuccess) r = cudaStreamWaitEvent(to, e, 0);
    cudaEventDestroy(e);
    if (r != cudaSuccess) return fail(MFD_ERR_CUDA, std::string("stream ordering: ") + cudaGetErrorString(r));
    return MFD_OK;
}

void retain(const mfd_ctx* c) {
    if (c) const_cast<mfd_ctx*>(c)->refs.fetch_add(1);
}
void retain(const mfd_nodes* n) {
    if (n) const_cast<mfd_nodes*>(n)->refs.fetch_add(1);
}
void retain(const mfd_stencils* s) {
    if (s) const_cast<mfd_stencils*>(s)->refs.fetch_add(1);
}
void retain(const mfd_weights* w) {
    if (w) const_cast<mfd_weights*>(w)->refs.fetch_add(1);
}

void release(const mfd_ctx* cc) {
    mfd_ctx* ctx = const_cast<mfd_ctx*>(cc);
    if (!ctx || ctx->refs.fetch_sub(1) != 1) return;
    cudaSetDevice(ctx->device);
    if (ctx->own_stream && ctx->stream) {
        cudaStreamSynchronize(ctx->stream);
        cudaStreamDestroy(ctx->stream);
    }
    delete ctx;
}

void release(const mfd_nodes* cn) {
    mfd_nodes* n = const_cast<mfd_nodes*>(cn);
    if (!n || n->refs.fetch_sub(1) != 1) return;
    mfd_ctx* ctx = n->ctx;
    cudaSetDevice(ctx->device);
    delete n;
    release(ctx);
}

void release(const mfd_stencils* cs) {
    mfd_stencils* s = const_cast<mfd_stencils*>(cs);
    if (!s || s->refs.fetch_sub(1) != 1) return;
    const mfd_nodes* c = s->centres;
    const mfd_nodes* src = s->sources;
    cudaSetDevice(c->ctx->device);
    delete s;
    release(c);
    release(src);
}

void release(const mfd_weights* cw) {
    mfd_weights* w = const_cast<mfd_weights*>(cw);
    if (!w || w->refs.fetch_sub(1) != 1) return;
    const mfd_stencils* st = w->st;
    cudaSetDevice(st->centres->ctx->device);
    delete w;
    release(st);
}

static mfd_status use_device(const mfd_ctx* ctx) {
    MFD_CUDA(cudaSetDevice(ctx->device));
    return MFD_OK;
}

__global__ void k_rows_to_user(const int32_t* __restrict__ idx, const int64_t* __restrict__ inv_c,
                               const int64_t* __restrict__ perm_s, int64_t nc, int n, int64_t* __restrict__ out) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nc * n) return;
    int64_t u = e / n;  // caller centre id
    int j = (int)(e % n);
    const int32_t v = idx[inv_c[u] * n + j];  // an image entry carries its reflection code (kernels.cuh)
    out[e] = perm_s[v & IMG_MASK] + ((int64_t)((unsigned)v >> IMG_SHIFT) << 32);
}

__global__ void k_w_to_user(const double* __restrict__ w, const int64_t* __restrict__ inv_c, int64_t nc, int n,
                            int nout, double* __restrict__ out) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)nout * nc * n) return;
    int64_t o = e / (nc * n);
    int64_t r = e % (nc * n);
    int64_t u = r / n;
    int j = (int)(r % n);
    out[e] = w[(o * nc + inv_c[u]) * n + j];
}

}  // namespace mfd

using namespace mfd;

extern "C" {

const char* mfd_last_error(void) { return g_last_error.c_str(); }

int mfd_version(void) { return 1; }

int mfd_build_flags(void) {
#ifdef MFD_BOUNDS_CHECK
    return MFD_BUILD_BOUNDS_CHECK;
#else
    return 0;
#endif
}

mfd_status mfd_debug_fail_alloc(int64_t after) {
    g_alloc_fail_in.store(after < 0 ? -1 : (long long)after);
    return MFD_OK;
}

int64_t mfd_debug_alloc_pending(void) { return g_alloc_fail_in.load(); }

mfd_status mfd_ctx_create(int device, void* stream, mfd_ctx** out) {
    if (!out) return fail(MFD_ERR_ARG, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    MFD_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(MFD_ERR_ARG, "no such CUDA device");
    MFD_CUDA(cudaSetDevice(device));
    mfd_ctx* c = new (std::nothrow) mfd_ctx();
    if (!c) return fail(MFD_ERR_OOM, "host allocation failed");
    c->device = device;
    if (stream) {
        c->stream = static_cast<cudaStream_t>(stream);
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            return fail(MFD_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
        }
        c->own_stream = true;
    }
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device);
    c->l2_bytes = l2;
    *out = c;
    return MFD_OK;
}

void* mfd_ctx_stream(const mfd_ctx* ctx) { return ctx ? (void*)ctx->stream : nullptr; }

mfd_status mfd_ctx_sync(mfd_ctx* ctx) {
    if (!ctx) return fail(MFD_ERR_ARG, "ctx is NULL");
    MFD_TRY(use_device(ctx));
    MFD_CUDA(cudaStreamSynchronize(ctx->stream));
    return MFD_OK;
}

void mfd_ctx_destroy(mfd_ctx* ctx) { release(ctx); }

mfd_status mfd_nodes_create(mfd_ctx* ctx, int dim, int64_t n, const double* xyz, const double* period,
                            mfd_nodes** out) {
    if (!ctx || !out || !xyz) return fail(MFD_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (dim != 2 && dim != 3) return fail(MFD_ERR_ARG, "dim must be 2 or 3");
    if (n < 1 || n > ((int64_t)1 << 31) - 1) return fail(MFD_ERR_ARG, "node count out of range");
    MFD_TRY(use_device(ctx));
    mfd_nodes* nd = new (std::nothrow) mfd_nodes();
    if (!nd) return fail(MFD_ERR_OOM, "host allocation failed");
    nd->ctx = ctx;
    nd->dim = dim;
    nd->n = n;
    for (int a = 0; a < dim; ++a) {
        nd->period[a] = period ? period[a] : 0.0;
        if (nd->period[a] < 0) {
            delete nd;
            return fail(MFD_ERR_ARG, "negative period");
        }
    }
    DevBuf user;
    mfd_status st;
    if ((st = user.alloc(n * dim * 8)) || (st = nd->xyz.alloc(n * dim * 8)) || (st = nd->perm.alloc(n * 8)) ||
        (st = nd->inv.alloc(n * 8))) {
        delete nd;
        return st;
    }
    cudaError_t e = cudaMemcpyAsync(user.p, xyz, n * dim * 8, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) {
        delete nd;
        return fail(MFD_ERR_CUDA, cudaGetErrorString(e));
    }
    st = morton_order(ctx, dim, n, user.as<double>(), nd->period, nd->xyz.as<double>(), nd->perm.as<int64_t>(),
                      nd->inv.as<int64_t>());
    if (st) {
        delete nd;
        return st;
    }
    nd->h_perm.resize(n);
    nd->h_inv.resize(n);
    cudaMemcpy(nd->h_perm.data(), nd->perm.p, n * 8, cudaMemcpyDeviceToHost);
    e = cudaMemcpy(nd->h_inv.data(), nd->inv.p, n * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        delete nd;
        return fail(MFD_ERR_CUDA, cudaGetErrorString(e));
    }
    retain(ctx);
    *out = nd;
    return MFD_OK;
}

int64_t mfd_nodes_count(const mfd_nodes* nodes) { return nodes ? nodes->n : -1; }

mfd_status mfd_nodes_permutation(const mfd_nodes* nodes, int64_t* perm) {
    if (!nodes || !perm) return fail(MFD_ERR_ARG, "NULL argument");
    memcpy(perm, nodes->h_perm.data(), nodes->n * 8);
    return MFD_OK;
}

void mfd_nodes_destroy(mfd_nodes* nodes) { release(nodes); }

mfd_status mfd_nodes_set_mirror(mfd_nodes* nodes, uint32_t axes, const double* hi) {
    if (!nodes || (axes && !hi)) return fail(MFD_ERR_ARG, "NULL argument");
    const int dim = nodes->dim;
    if (axes & ~((1u << dim) - 1u)) return fail(MFD_ERR_ARG, "mirror axes beyond the dimension");
    if (nodes->n >= ((int64_t)1 << IMG_SHIFT)) return fail(MFD_ERR_ARG, "too many nodes for image codes");
    std::vector<double> x((size_t)nodes->n * dim);
    MFD_TRY(use_device(nodes->ctx));
    MFD_CUDA(cudaMemcpy(x.data(), nodes->xyz.p, x.size() * 8, cudaMemcpyDeviceToHost));
    for (int a = 0; a < dim; ++a) {
        if (!((axes >> a) & 1u)) continue;
        if (nodes->period[a] > 0) return fail(MFD_ERR_ARG, "a mirrored axis cannot be periodic");
        if (!(hi[a] > 0)) return fail(MFD_ERR_ARG, "mirror walls need hi > 0");
        for (int64_t i = 0; i < nodes->n; ++i)
            if (!(x[i * dim + a] > 0.0 && x[i * dim + a] < hi[a]))
                return fail(MFD_ERR_ARG, "nodes must lie strictly between the mirror walls (0 and hi)");
    }
    nodes->mirror_axes = axes;
    for (int a = 0; a < 3; ++a) nodes->mirror_hi[a] = (a < dim && ((axes >> a) & 1u)) ? hi[a] : 0.0;
    return MFD_OK;
}

mfd_status mfd_stencils_build(const mfd_nodes* centres, const mfd_nodes* sources, int n, mfd_stencils** out) {
    if (!centres || !sources || !out) return fail(MFD_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (centres->ctx != sources->ctx) return fail(MFD_ERR_ARG, "node sets belong to different contexts");
    if (centres->dim != sources->dim) return fail(MFD_ERR_ARG, "node sets differ in dimension");
    for (int a = 0; a < centres->dim; ++a)
        if (centres->period[a] != sources->period[a]) return fail(MFD_ERR_ARG, "node sets differ in periods");
    if (n < 1 || n > 128 || n > sources->n) return fail(MFD_ERR_ARG, "stencil size out of range");
    MFD_TRY(use_device(centres->ctx));
    mfd_stencils* s = new (std::nothrow) mfd_stencils();
    if (!s) return fail(MFD_ERR_OOM, "host allocation failed");
    s->centres = centres;
    s->sources = sources;
    s->n = n;
    mfd_status st = s->idx.alloc(centres->n * n * 4);
    if (!st && sources->mirror_axes) {
        if (centres != sources) st = fail(MFD_ERR_ARG, "stencils with mirror walls are own-set (collocated)");
        else st = knn_build_mirror(centres, sources, n, s->idx.as<int32_t>());
    } else if (!st) {
        st = knn_build(centres, sources, n, s->idx.as<int32_t>());
    }
    if (st) {
        delete s;
        return st;
    }
    retain(centres);
    retain(sources);
    *out = s;
    return MFD_OK;
}

mfd_status mfd_stencils_read(const mfd_stencils* st, int64_t* idx) {
    if (!st || !idx) return fail(MFD_ERR_ARG, "NULL argument");
    mfd_ctx* ctx = st->centres->ctx;
    MFD_TRY(use_device(ctx));
    const int64_t total = st->centres->n * st->n;
    DevBuf out;
    MFD_TRY(out.alloc(total * 8));
    k_rows_to_user<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(
        st->idx.as<int32_t>(), st->centres->inv.as<int64_t>(), st->sources->perm.as<int64_t>(), st->centres->n,
        st->n, out.as<int64_t>());
    MFD_CUDA(cudaGetLastError());
    MFD_CUDA(cudaMemcpyAsync(idx, out.p, total * 8, cudaMemcpyDeviceToHost, ctx->stream));
    MFD_CUDA(cudaStreamSynchronize(ctx->stream));
    return MFD_OK;
}

void mfd_stencils_destroy(mfd_stencils* st) { release(st); }

}  // extern "C"

namespace {

__global__ void k_sizes_to_device(const int32_t* __restrict__ user, const int64_t* __restrict__ perm, int64_t n,
                                  int32_t* __restrict__ dev) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < n) dev[k] = user[perm[k]];
}

// mfd_weights_compute(_sized): sizes == NULL for one stencil size n_use
mfd_status weights_create(const mfd_stencils* st, int n_use, const int32_t* sizes, int phs_k, int poly_m, int op,
                          int alpha, double delta, mfd_weights** out) {
    if (!st || !out) return fail(MFD_ERR_ARG, "NULL argument");
    *out = nullptr;
    const int64_t N = st->centres->n;
    int n_min = n_use;
    if (sizes) {
        n_use = 0;
        n_min = INT32_MAX;
        for (int64_t i = 0; i < N; ++i) {
            n_use = std::max(n_use, (int)sizes[i]);
            n_min = std::min(n_min, (int)sizes[i]);
        }
        if (N == 0) n_use = n_min = 1;
        if (n_min < 1) return fail(MFD_ERR_ARG, "a stencil size is below 1");
    }
    if (n_use < 1 || n_use > st->n) return fail(MFD_ERR_ARG, "n_use out of range");
    if (phs_k < 1 || phs_k > 9 || phs_k % 2 == 0) return fail(MFD_ERR_ARG, "phs_k must be odd, 1..9");
    if (poly_m < 0) return fail(MFD_ERR_ARG, "poly_m < 0");
    if (op != MFD_OP_GRAD && op != MFD_OP_LAP_POW && op != MFD_OP_GRAD_VFD) return fail(MFD_ERR_ARG, "unknown op");
    if (op == MFD_OP_LAP_POW && (alpha < 1 || phs_k < 2 * alpha + 1))
        return fail(MFD_ERR_ARG, "Delta^alpha needs alpha >= 1 and phs_k >= 2 alpha + 1");
    if (op == MFD_OP_GRAD_VFD && !(delta > 0)) return fail(MFD_ERR_ARG, "RBF-VFD needs delta > 0");
    MFD_TRY(use_device(st->centres->ctx));
    mfd_weights* w = new (std::nothrow) mfd_weights();
    if (!w) return fail(MFD_ERR_OOM, "host allocation failed");
    w->st = st;
    w->n_use = n_use;
    w->n_min = n_min;
    w->nout = op == MFD_OP_LAP_POW ? 1 : st->centres->dim;
    w->op = op;
    w->phs_k = phs_k;
    w->poly_m = poly_m;
    w->alpha = alpha;
    w->delta = delta;
    mfd_status s = w->w.alloc((size_t)w->nout * N * n_use * 8);
    if (!s && sizes && n_min < n_use) {  // sizes to device order
        DevBuf user;
        s = user.alloc(N * 4);
        if (!s) s = w->nsz.alloc(N * 4);
        if (!s) {
            cudaStream_t cs = st->centres->ctx->stream;
            cudaError_t e = cudaMemcpyAsync(user.p, sizes, N * 4, cudaMemcpyHostToDevice, cs);
            if (e == cudaSuccess) {
                k_sizes_to_device<<<(unsigned)((N + 255) / 256), 256, 0, cs>>>(
                    user.as<int32_t>(), st->centres->perm.as<int64_t>(), N, w->nsz.as<int32_t>());
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
            if (e != cudaSuccess) s = fail(MFD_ERR_CUDA, cudaGetErrorString(e));
        }
    }
    if (!s) s = weights_solve(st, n_use, w->nsz.p ? w->nsz.as<int32_t>() : nullptr, phs_k, poly_m, op, alpha, delta,
                              w->w.as<double>());
    if (s) {
        delete w;
        return s;
    }
    retain(st);
    *out = w;
    return MFD_OK;
}

}  // namespace

extern "C" {

mfd_status mfd_weights_compute(const mfd_stencils* st, int n_use, int phs_k, int poly_m, int op, int alpha,
                               double delta, mfd_weights** out) {
    return weights_create(st, n_use, nullptr, phs_k, poly_m, op, alpha, delta, out);
}

mfd_status mfd_weights_compute_sized(const mfd_stencils* st, const int32_t* n_per_centre, int phs_k, int poly_m,
                                     int op, int alpha, double delta, mfd_weights** out) {
    if (!n_per_centre) return fail(MFD_ERR_ARG, "NULL argument");
    return weights_create(st, 0, n_per_centre, phs_k, poly_m, op, alpha, delta, out);
}

mfd_status mfd_weights_read(const mfd_weights* w, double* host_w) {
    if (!w || !host_w) return fail(MFD_ERR_ARG, "NULL argument");
    const mfd_nodes* c = w->st->centres;
    MFD_TRY(use_device(c->ctx));
    const int64_t total = (int64_t)w->nout * c->n * w->n_use;
    DevBuf out;
    MFD_TRY(out.alloc(total * 8));
    k_w_to_user<<<(unsigned)((total + 255) / 256), 256, 0, c->ctx->stream>>>(
        w->w.as<double>(), c->inv.as<int64_t>(), c->n, w->n_use, w->nout, out.as<double>());
    MFD_CUDA(cudaGetLastError());
    MFD_CUDA(cudaMemcpyAsync(host_w, out.p, total * 8, cudaMemcpyDeviceToHost, c->ctx->stream));
    MFD_CUDA(cudaStreamSynchronize(c->ctx->stream));
    return MFD_OK;
}

void mfd_weights_destroy(mfd_weights* w) { release(w); }

}  // extern "C"
