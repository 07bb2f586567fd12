// internal.cuh -- shared declarations of the CUDA library behind include/mfd.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/mfd.h"

namespace mfd {

// ------------------------------------------------------------ errors

void set_error(const std::string& msg);
mfd_status fail(mfd_status st, const std::string& msg);

#define MFD_CUDA(call)                                                                     \
    do {                                                                                   \
        cudaError_t e__ = (call);                                                          \
        if (e__ != cudaSuccess)                                                            \
            return ::mfd::fail(MFD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e__)); \
    } while (0)

#define MFD_TRY(call)                         \
    do {                                      \
        mfd_status s__ = (call);              \
        if (s__ != MFD_OK) return s__;        \
    } while (0)

// ------------------------------------------------------------ device buffers

// Fault injection for tests (mfd_debug_fail_alloc): the number of device
// allocations that still succeed before one fails; negative = off.
extern std::atomic<long long> g_alloc_fail_in;

// An owning device allocation (cudaMalloc); freed with the object holding it.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    mfd_status alloc(size_t n) {
        release();
        if (n == 0) n = 16;
        if (g_alloc_fail_in.load(std::memory_order_relaxed) >= 0 && g_alloc_fail_in.fetch_sub(1) == 0)
            return fail(MFD_ERR_OOM, std::string("injected allocation failure (") + std::to_string(n) + " bytes)");
        cudaError_t e = cudaMalloc(&p, n);
        if (e != cudaSuccess) {
            p = nullptr;
            return fail(MFD_ERR_OOM, std::string("cudaMalloc(") + std::to_string(n) + "): " + cudaGetErrorString(e));
        }
        bytes = n;
        return MFD_OK;
    }
    template <typename T> T* as() const { return static_cast<T*>(p); }
};

}  // namespace mfd

// ------------------------------------------------------------ objects

// Every object is reference counted: the creator's reference is dropped by its
// *_destroy call, and each object holds one reference on every object it was
// created from, so a context, node set, stencil set or weight set lives as long
// as anything built on it (destruction order does not matter).
struct mfd_ctx {
    std::atomic<int> refs{1};
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int sm_count = 0;
    int64_t l2_bytes = 0;  // L2 cache size of the device
    mfd::DevBuf status;  // device status words (int32[8]) shared by bounded waits
};

struct mfd_nodes {
    std::atomic<int> refs{1};
    mfd_ctx* ctx = nullptr;
    int dim = 2;
    int64_t n = 0;
    double period[3] = {0, 0, 0};
    mfd::DevBuf xyz;   // double [n][dim], device (Morton) order
    mfd::DevBuf perm;  // int64 [n]: device order -> caller id
    mfd::DevBuf inv;   // int64 [n]: caller id -> device order
    std::vector<int64_t> h_perm;
    std::vector<int64_t> h_inv;
    uint32_t mirror_axes = 0;        // PEC walls by images on these axes (mfd_nodes_set_mirror)
    double mirror_hi[3] = {0, 0, 0};  // the walls of mirrored axis a are at 0 and mirror_hi[a]
};

struct mfd_stencils {
    std::atomic<int> refs{1};
    const mfd_nodes* centres = nullptr;
    const mfd_nodes* sources = nullptr;
    int n = 0;
    mfd::DevBuf idx;  // int32 [centres.n][n], source device ids, rows in centre device order
};

struct mfd_weights {
    std::atomic<int> refs{1};
    const mfd_stencils* st = nullptr;
    int n_use = 0;
    int nout = 0;
    int op = 0;
    int phs_k = 0, poly_m = 0, alpha = 0;
    double delta = 0;
    int n_min = 0;    // smallest stencil size of a centre (== n_use unless sizes vary)
    mfd::DevBuf nsz;  // int32 stencil size per centre (device order) when sizes vary, else empty
    mfd::DevBuf w;    // double [nout][centres.n][n_use], centre device order; a row is zero past its centre's size
};

namespace mfd {

// makes `to` wait for the work queued so far on `from` (an event; nothing if equal)
mfd_status order_streams(cudaStream_t from, cudaStream_t to);

// reference counting (see above); release frees the object when the count drops to 0
void retain(const mfd_ctx* c);
void retain(const mfd_nodes* n);
void retain(const mfd_stencils* s);
void retain(const mfd_weights* w);
void release(const mfd_ctx* c);
void release(const mfd_nodes* n);
void release(const mfd_stencils* s);
void release(const mfd_weights* w);

// ------------------------------------------------------------ state blobs

// Header of a checkpoint (mfd_sim_save_state, mfd_batch_save_state): the
// device buffers that hold the fields follow in order, then the probe records.
struct StateHead {
    char magic[8];        // "MFDSTATE"
    int32_t version;      // 1
    int32_t kind;         // 1 simulation, 2 batch
    int32_t layout;       // simulation layout (0 for a batch)
    int32_t fp64;         // 1 for FP64 fields
    int64_t ne, nh, nrhs; // E nodes, H nodes (batch: total nodes, 0), right-hand sides
    int64_t steps;        // step index n of the saved fields (E at t_n, H at t_n - dt/2)
    int64_t probe_from;   // step at which probe recording started
    int32_t parity;       // ping-pong buffer holding the current fields
    int32_t nprobe;       // probes (batch: probe slots over all domains)
    int64_t rec;          // probe records in the blob
    int64_t bytes[6];     // sizes of the device buffers that follow
};
constexpr int32_t kStateVersion = 1;
void state_head_init(StateHead* h, int32_t kind);
// checks magic, version and kind of a blob of `size` bytes
mfd_status state_head_check(const void* blob, size_t size, int32_t kind, StateHead* out);

// ------------------------------------------------------------ setup kernels

mfd_status morton_order(mfd_ctx* ctx, int dim, int64_t n, const double* d_xyz_user,
                        const double* period, double* d_xyz_sorted, int64_t* d_perm, int64_t* d_inv);
mfd_status knn_build(const mfd_nodes* centres, const mfd_nodes* sources, int n, int32_t* d_idx);
// kNN among the nodes of a set with mirror walls and their images (entries carry image codes)
mfd_status knn_build_mirror(const mfd_nodes* centres, const mfd_nodes* sources, int n, int32_t* d_idx);
// n_use: row length (the largest stencil); d_nsz: per-centre sizes (device order) or NULL
mfd_status weights_solve(const mfd_stencils* st, int n_use, const int32_t* d_nsz, int phs_k, int poly_m, int op,
                         int alpha, double delta, double* d_w);
// per row of a shared index array (n rows of `stride` entries, len <= 255 used):
// the order that sorts entries [0, m) and [m, len) by neighbour id (k_row_perm)
// entries sorted by neighbour id within [0, m1), [m1, m2) and [m2, len)
cudaError_t launch_row_perm(const int32_t* idx, int stride, int64_t n, int m1, int m2, int len, uint8_t* perm,
                            cudaStream_t s);

// ------------------------------------------------------------ dispersion (Sec. 6)

mfd_status dispersion_check(int nx, int nt, double h_line, double dt_sample, int jmax);
// d_samples: device FP64 [nt][nx]; outputs are host pointers (each may be NULL)
mfd_status dispersion_run(mfd_ctx* ctx, int nx, int nt, const double* d_samples, double h_line, double dt_sample,
                          double c_ref, int jmax, double* spectrum, int32_t* kidx, double* c, double* err_l1);

}  // namespace mfd
