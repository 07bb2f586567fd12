/*
 * mfd.h -- C ABI of the GB300 meshless (RBF-FD) Maxwell leapfrog library.
 *
 * The method is the meshless generalisation of the FDTD in "An RBF-based
 * method for computational electromagnetics with reduced numerical
 * dispersion" (arXiv 2508.18205): the interleaved leapfrog of the FDTD is kept
 * (Sec. 5), every spatial derivative is a stencil sum D^L f(x_i) =
 * sum_{j in S(x_i)} w_j f(x_j) over the n nearest nodes (Eq. 16, Eq. 11), the
 * weights come from a local polyharmonic-spline + monomial interpolant (Eq. 9;
 * RBF-FD Eq. 13 or RBF-VFD Eqs. 14-15), and a hyperviscosity term
 * gamma Delta^alpha, itself discretised by RBF-FD, stabilises the update
 * (Eqs. 17-19).
 *
 * Conventions (all calls):
 *  - Every call returns mfd_status: MFD_OK (0) or a negative error code; the
 *    message of the last error on the calling thread is mfd_last_error().
 *    No exception and no abort crosses this boundary.
 *  - Host pointers are read or written only during the call (the library
 *    copies what it keeps). Device memory is owned by the library.
 *  - Objects are reference counted: *_destroy drops the caller's reference,
 *    and every object keeps the objects it was created from (context, node
 *    sets, stencils, weights) alive, so handles may be destroyed in any order.
 *  - Node ids at this boundary are always in the caller's order. Internally
 *    the library reorders every node set along a Morton curve.
 *  - Work is queued on the context's CUDA stream; calls that return host data
 *    synchronise that stream. Asynchronous device errors surface as
 *    MFD_ERR_CUDA at the next synchronising call.
 *  - Coordinates and all physical parameters are FP64.
 */
#ifndef MFD_H
#define MFD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int mfd_status;
#define MFD_OK 0
#define MFD_ERR_ARG -1      /* invalid argument (sizes, null pointers, mismatched objects) */
#define MFD_ERR_OOM -2      /* device or host allocation failed */
#define MFD_ERR_CUDA -3     /* a CUDA runtime call failed */
#define MFD_ERR_SINGULAR -4 /* a local weight system (Eq. 9) had an exactly zero pivot */
#define MFD_ERR_UNSTABLE -5 /* the energy watchdog saw growth beyond its bound or a NaN */
#define MFD_ERR_TIMEOUT -6  /* a bounded device-side wait gave up */
#define MFD_ERR_STATE -7    /* call out of order (e.g. stepping before fields are set) */

/* operators for mfd_weights_compute */
#define MFD_OP_GRAD 0     /* d/dx_a, a < dim, by RBF-FD (Eq. 13): dim outputs */
#define MFD_OP_LAP_POW 1  /* Delta^alpha by RBF-FD (Eq. 13, Sec. 5.1): one output */
#define MFD_OP_GRAD_VFD 2 /* d/dx_a by RBF-VFD (Eqs. 14-15) with central differences */

#define MFD_FP32 0
#define MFD_FP64 1

/* field components */
#define MFD_EX 0
#define MFD_EY 1
#define MFD_EZ 2
#define MFD_HX 3
#define MFD_HY 4
#define MFD_HZ 5

typedef struct mfd_ctx mfd_ctx;
typedef struct mfd_nodes mfd_nodes;
typedef struct mfd_stencils mfd_stencils;
typedef struct mfd_weights mfd_weights;
typedef struct mfd_sim mfd_sim;

/* Message of the last failed call on this thread ("" if none). */
const char* mfd_last_error(void);
int mfd_version(void);
/* How this copy of the library was built: MFD_BUILD_BOUNDS_CHECK is set in the
 * bounds-checked debug build (compiled with MFD_BOUNDS_CHECK defined), where
 * every stencil index is tested against the node set it points into before a
 * kernel gathers through it, and where the stencil rows are tested when a
 * simulation packs them. A failed test does not trap: the index is replaced
 * by 0, and the call that ran the kernel returns MFD_ERR_STATE. It is the
 * stand-in for a memory checker, for test runs; the paper has no counterpart. */
#define MFD_BUILD_BOUNDS_CHECK 1
int mfd_build_flags(void);

/* Fault injection for tests of the error paths (the paper has no
 * counterpart): the next `after` device allocations of the library succeed
 * and the one after them fails with MFD_ERR_OOM without calling cudaMalloc;
 * after < 0 turns it off. Process-wide; it fires once. Every object whose
 * creation failed this way has been freed, and objects created before stay
 * valid. Host only. */
mfd_status mfd_debug_fail_alloc(int64_t after);
/* Allocations left before the injected failure fires; -1 when none is pending. */
int64_t mfd_debug_alloc_pending(void);

/* ------------------------------------------------------------- context */

/* Binds the library to CUDA device `device`. stream: a cudaStream_t to
 * queue work on, or NULL for a stream the context creates (non-blocking).
 * A context is used by one host thread at a time. */
mfd_status mfd_ctx_create(int device, void* stream, mfd_ctx** out);
/* The cudaStream_t the context queues its work on (for the caller's events). */
void* mfd_ctx_stream(const mfd_ctx* ctx);
/* Waits for the context's stream; surfaces asynchronous errors as a status. */
mfd_status mfd_ctx_sync(mfd_ctx* ctx);
void mfd_ctx_destroy(mfd_ctx* ctx);

/* --------------------------------------------------------------- nodes */

/* A scattered node set X = {x_i} (Sec. 4, nodes at spacing ~h).
 * xyz: host, n x dim FP64, caller's order. period: host, dim entries; the
 * period along each axis, 0 for a non-periodic axis (coordinates of a
 * periodic axis must lie in [0, period)). dim is 2 or 3; n >= 1.
 * The node set is copied to the device and reordered along a Morton curve of
 * its bounding box (ties by caller id). */
mfd_status mfd_nodes_create(mfd_ctx* ctx, int dim, int64_t n, const double* xyz,
                            const double* period, mfd_nodes** out);
int64_t mfd_nodes_count(const mfd_nodes* nodes);
/* PEC walls by images (a reading: the paper uses periodic boxes only). The
 * walls of each axis a in `axes` (bit a) are the planes x_a = 0 and
 * x_a = hi[a], and every node lies strictly between them (for example at the
 * cell centres of a grid: a node on a mirror plane sees each neighbour and its
 * image at one distance, and a stencil cut through such a pair is lopsided). A perfect conductor acts as a
 * mirror: the tangential E and the normal H change sign under the reflection,
 * the normal E and the tangential H do not, so the box is a periodic box of
 * period 2 hi[a] holding fields of those parities. Stencils built on this set
 * (own-set, mfd_stencils_build) take the n nearest among its nodes and their
 * mirror images x_a -> 2 hi[a] - x_a; an entry
 * that is an image carries its reflection code r (bit a: reflected across the
 * walls normal to axis a), the weights are solved at the image positions, and
 * the step kernels gather an image with the sign of the field's parity. No
 * component needs holding at the walls (pass no PEC flags): the symmetry is
 * the boundary condition. Call before building stencils; axes must not be
 * periodic; fewer than 2^29 nodes. Supported by the collocated 2D and 3D
 * layouts (not the staggered layout, the batch or the gradient: MFD_ERR_ARG).
 * With curl stencils of the fewest nodes the monomials allow (n = 2 M_m),
 * some stencils of the layer next to a wall give the 3D curl a growing mode;
 * a few more nodes in that layer (mfd_weights_compute_sized, e.g. 44 instead
 * of 40) remove it. */
mfd_status mfd_nodes_set_mirror(mfd_nodes* nodes, uint32_t axes, const double* hi);
/* perm (host, n): perm[k] = caller id of the k-th node in device order. */
mfd_status mfd_nodes_permutation(const mfd_nodes* nodes, int64_t* perm);
void mfd_nodes_destroy(mfd_nodes* nodes);

/* ------------------------------------------------------------ stencils */

/* kNN stencils S(x_c) (Sec. 4.1, Eq. 11): for every node of `centres`, the n
 * nodes of `sources` closest to it, sorted by (squared distance, caller id of
 * the source); periodic axes use the minimum image. Squared distances are
 * FP64 sums dx*dx + dy*dy (+ dz*dz) taken left to right without fused
 * multiply-add, so the result is exactly reproducible. centres and sources
 * may be the same object (collocated stencils start with the centre itself)
 * and must share dim and periods. 1 <= n <= min(128, count(sources)). */
mfd_status mfd_stencils_build(const mfd_nodes* centres, const mfd_nodes* sources, int n,
                              mfd_stencils** out);
/* idx (host, count(centres) x n): caller ids of the stencil nodes, rows in
 * the caller's centre order; an image entry of a set with mirror walls
 * (mfd_nodes_set_mirror) is the node's caller id + r * 2^32, r its reflection
 * code. */
mfd_status mfd_stencils_read(const mfd_stencils* st, int64_t* idx);
void mfd_stencils_destroy(mfd_stencils* st);

/* ------------------------------------------------------------- weights */

/* Stencil weights w^L (Eq. 12) on the first n_use entries of each stencil,
 * from the local interpolant with PHS phi(r) = r^phs_k (phs_k odd, 1..9) and
 * all monomials of total degree <= poly_m (Eq. 9). Each centre's system is
 * shifted to x_c, scaled by the stencil radius and solved in FP64 on the GPU.
 *   op = MFD_OP_GRAD     : RBF-FD first derivatives, dim outputs (Eq. 13)
 *   op = MFD_OP_LAP_POW  : RBF-FD Delta^alpha, one output (Sec. 5.1);
 *                          needs phs_k >= 2 alpha + 1
 *   op = MFD_OP_GRAD_VFD : RBF-VFD first derivatives: the central difference
 *                          (s(x_c + delta e_a) - s(x_c - delta e_a)) / (2 delta)
 *                          of the interpolant (Eqs. 14-15); delta > 0.
 * Returns MFD_ERR_SINGULAR if any system had an exactly zero pivot. */
mfd_status mfd_weights_compute(const mfd_stencils* st, int n_use, int phs_k, int poly_m, int op,
                               int alpha, double delta, mfd_weights** out);
/* mfd_weights_compute with a stencil size per centre: centre c takes the first
 * n_per_centre[c] entries of its stencil (host array, caller's centre order,
 * each in 1..n of the stencils object). Rows are max(n_per_centre) long, zero
 * past the centre's own size (mfd_weights_read). A simulation takes such
 * weights as the curl weights of the 3D layout, where each 32-node slice of the
 * packed streams reads only the chunks its centres need; elsewhere (the 2D
 * layouts, hyperviscosity weights, batches) they are refused with MFD_ERR_ARG.
 * The method fixes one n per operator (Sec. 4.1); a larger curl stencil in the
 * layer next to mirror walls keeps the 3D scheme with images stable there. */
mfd_status mfd_weights_compute_sized(const mfd_stencils* st, const int32_t* n_per_centre, int phs_k, int poly_m,
                                     int op, int alpha, double delta, mfd_weights** out);
/* w (host, nout x count(centres) x n_use) in the caller's centre order,
 * entry j of a row being the weight of stencil entry j (mfd_stencils_read). */
mfd_status mfd_weights_read(const mfd_weights* w, double* host_w);
void mfd_weights_destroy(mfd_weights* w);

/* ----------------------------------------------------------- simulation */

/* The stepped problem. The H field lives on the centres of h_curl / h_hv, the
 * E field on the centres of e_curl / e_hv.
 *   collocated (the paper's method, Sec. 5): one node set; h_curl == e_curl
 *     (MFD_OP_GRAD or MFD_OP_GRAD_VFD weights) and h_hv == e_hv
 *     (MFD_OP_LAP_POW). When the curl and HV weights come from one stencils
 *     object (the curl weights on its first n entries) the kernels read one
 *     index array for both.
 *   staggered: an E node set and an H node set; h_curl has H centres and E
 *     sources, e_curl E centres and H sources; h_hv / e_hv are own-set.
 * One step n -> n+1 (Eq. 19; 3D: Eq. 2 with the same terms on every component):
 *   H <- H + dt/mu0 (-curl E^n + gamma D^{Delta^alpha} H)
 *   E <- E + dt/(eps0 eps_r) (curl H^{n+1/2} + gamma D^{Delta^alpha} E^n)
 *   then soft sources add amp r(t_{n+1}) to Ez, PEC components are held at 0,
 *   and probes record Ez^{n+1}.
 * gamma is the coefficient of Eq. 18 (c (-1)^(alpha-1) h^(2 alpha) in the
 * paper's units). nrhs field vectors are stepped with the same weights. */
typedef struct {
    int dim;       /* 2 (TMz: Ez, Hx, Hy) or 3 (Ex..Hz, collocated only) */
    int precision; /* MFD_FP32 or MFD_FP64: fields, weights and arithmetic */
    int nrhs;      /* right-hand sides (>= 1) */
    int compensated; /* FP32 only: 1 = compensated (two-sum) stencil sums */
    double dt, eps0, mu0, gamma;
    const mfd_weights* h_curl;
    const mfd_weights* h_hv;
    const mfd_weights* e_curl;
    const mfd_weights* e_hv;
} mfd_sim_desc;

mfd_status mfd_sim_create(mfd_ctx* ctx, const mfd_sim_desc* desc, mfd_sim** out);
/* eps_r (host, count(E nodes), NULL = vacuum) and pec (host, count(E nodes),
 * NULL = none). 2D: pec[i] != 0 holds Ez_i at 0. 3D: pec[i] bit a set when
 * the node sits on a wall normal to axis a; every E component tangential to
 * such a wall is held at 0. Fields of held components are zeroed now. */
mfd_status mfd_set_materials(mfd_sim* sim, const double* eps_r, const uint8_t* pec);
/* Field component `comp` (MFD_EX..MFD_HZ) of right-hand side `rhs` from host
 * FP64 values in the caller's order of its node set. E is taken at t_n, H at
 * t_n - dt/2 (Eq. 4, Eq. 21). Resets the step counter to 0 when comp == MFD_EZ. */
mfd_status mfd_set_field(mfd_sim* sim, int comp, int rhs, const double* host);
mfd_status mfd_get_field(mfd_sim* sim, int comp, int rhs, double* host);
/* Zero-copy variants of mfd_set_field / mfd_get_field: `dev` is a device
 * pointer (FP64, caller's node order, on the context's device, e.g. a torch
 * CUDA tensor's storage) and `stream` the cudaStream_t on which the caller
 * produces or consumes it (NULL: the legacy default stream). The library's
 * stream waits for the work already queued on `stream` before it reads or
 * writes `dev`, and `stream` waits for the library's copy before anything the
 * caller queues after the call; no host synchronisation. */
mfd_status mfd_set_field_device(mfd_sim* sim, int comp, int rhs, const double* dev, void* stream);
mfd_status mfd_get_field_device(mfd_sim* sim, int comp, int rhs, double* dev, void* stream);
/* Soft Ricker sources (count >= 0): node (E node, caller id), rhs, amplitude,
 * centre frequency f0 and delay t0; r(t) = (1 - 2 a) exp(-a),
 * a = (pi f0 (t - t0))^2, added to Ez after each E update. */
mfd_status mfd_set_sources(mfd_sim* sim, int count, const int64_t* node, const int32_t* rhs,
                           const double* amp, const double* f0, const double* t0);
/* Probes: Ez (or the component of mfd_set_probe_component) at `count` E nodes
 * (caller ids) is recorded after every step for every rhs, for at most
 * `capacity` steps; recording restarts at 0. */
mfd_status mfd_set_probes(mfd_sim* sim, int count, const int64_t* node, int64_t capacity);
/* The component the probes record after each step (MFD_EZ by default): in the
 * collocated layouts also MFD_HX, MFD_HY (2D) or any of MFD_EX..MFD_HZ (3D),
 * H at t_{n+1/2}, the level the leapfrog holds after step n -> n+1; the
 * staggered layout records Ez only (its H lives on the other node set). The
 * gradient calls need Ez probes (MFD_ERR_ARG otherwise). Takes effect from
 * the next step; the recorded series is not cleared. */
mfd_status mfd_set_probe_component(mfd_sim* sim, int comp);
/* Advances nsteps (>= 0) leapfrog steps on the context stream (launches
 * replay a captured CUDA graph for long runs). */
mfd_status mfd_step(mfd_sim* sim, int64_t nsteps);
/* As mfd_step, without graphs: CUDA events bracket every launch of the H
 * and E half-step kernels; ms[0], ms[1] receive their summed device times
 * (synchronises). */
mfd_status mfd_step_timed(mfd_sim* sim, int64_t nsteps, double* ms);
/* Probe series recorded since mfd_set_probes: host (steps x count x nrhs FP64);
 * *steps receives the number of recorded steps. host may be NULL to query. */
mfd_status mfd_read_probes(mfd_sim* sim, double* host, int64_t* steps);
/* Eq. 20 at the current time t_n for every rhs (host, nrhs values):
 * sum_i eps_r,i |E_i|^2 + (mu0/eps0) |H_i|^2 with H averaged between t_n -
 * dt/2 and t_n + dt/2 (the latter computed on the fly). Multiply by the
 * domain measure / node count for the integral of Eq. 20. */
mfd_status mfd_energy(mfd_sim* sim, double* u);
/* Energy watchdog (failure detection for the instability of Sec. 5 / App. A):
 * with every > 0, mfd_step computes Eq. 20 after every `every` steps and
 * returns MFD_ERR_UNSTABLE (with the steps taken so far kept) once the energy
 * exceeds max_ratio times its value at this call, or is NaN. every = 0 turns
 * it off. Needs the fields set (nonzero energy). */
mfd_status mfd_set_watchdog(mfd_sim* sim, int64_t every, double max_ratio);
/* Threads per block of the H and E half-step kernels (64, 128, 256 or 512;
 * 256 by default). */
mfd_status mfd_sim_set_blocks(mfd_sim* sim, int block_h, int block_e);
/* Autotuner: times each half-step kernel on this problem `reps` times with
 * 64, 128, 256 and 512 threads per block and, in the collocated 2D layout with one
 * index row for both stencils, 1, 2 or 4 threads per node (each summing a
 * share of the node's stencil chunks; the shares are added across the node's
 * threads, so the choice changes the order of the stencil sums, not their
 * terms); keeps the fastest for each pass (chosen[0]: H pass, chosen[1]: E
 * pass, threads per block; may be NULL) and restores the fields, so the
 * simulation does not advance. */
mfd_status mfd_sim_autotune(mfd_sim* sim, int reps, int* chosen);
/* Threads per node of the H and E passes (1, 2 or 4) in the collocated 2D
 * layout whose curl and HV stencils share one index row (else MFD_ERR_ARG). */
mfd_status mfd_sim_set_lanes(mfd_sim* sim, int lanes_h, int lanes_e);
/* The launch configuration in use: block[2] threads per block and lanes[2]
 * threads per node of the H and E passes (1 outside the collocated 2D layout;
 * before any autotuning 4 for node sets too small to fill the GPU, else 1).
 * Either may be NULL. */
mfd_status mfd_sim_launch_config(const mfd_sim* sim, int* block, int* lanes);
/* Index format of the staggered step kernels. The stencil sums are the same
 * in both formats (same entries, same order), so the fields are bit-identical.
 *   MFD_INDEX_Q16 (the default): per slice of 32 nodes (one warp) and per
 *     stencil stream, two bases and 16-bit entries (id = b0 + u for
 *     u < 32768, else b1 + u - 32768); a slice whose neighbour ids do not fit
 *     two windows of 32768 ids (rare: Morton seams and periodic wraps) keeps
 *     its 32-bit entries. Halves the index bytes each step reads.
 *   MFD_INDEX_I32: 32-bit entries everywhere.
 * The collocated and 3D layouts always read 32-bit entries. Returns
 * MFD_ERR_ARG for another format. */
#define MFD_INDEX_Q16 0
#define MFD_INDEX_I32 1
mfd_status mfd_sim_set_index_format(mfd_sim* sim, int format);
/* out (host, 6 values) = {slices, slices whose curl stream is 32-bit, slices
 * whose HV stream is 32-bit} of the H pass, then the same of the E pass;
 * zeros when the layout has no Q16 streams (collocated, 3D). */
mfd_status mfd_sim_index_stats(const mfd_sim* sim, int64_t* out);
/* L2 residency of the stencil streams (no counterpart in the paper: a cache
 * policy of this GPU). The step kernels read the index and weight streams once
 * per half step; a fraction `keep` of their cache lines is loaded with the L2
 * policy evict_last and the rest with evict_first. When a problem's streams
 * are about the size of the L2, the kept lines stay in L2 from one step to the
 * next and the rest stream through without evicting them or the gathered
 * fields. By default (keep < 0) the fraction is sized so that the kept lines
 * fill about 40 % of the device's L2 (1 for problems whose streams fit in
 * that, 0 when that fraction is below 0.15: streams larger than about 2.7
 * times the L2 gain nothing from kept lines); keep in [0, 1] fixes it. The adjoint sweep sizes its
 * own fraction from the transposed streams. The 3D kernels mark every line
 * evict_first whatever keep is (their problems are far larger than the L2).
 * Results do not depend on keep (bit-identical fields). MFD_ERR_ARG for
 * keep > 1 or NaN. */
mfd_status mfd_sim_set_l2_keep(mfd_sim* sim, double keep);
/* The fraction the forward step kernels use (0 for the 3D layout, -1 for a NULL sim). */
double mfd_sim_l2_keep(const mfd_sim* sim);
/* Gradient of the probe objective J = dt sum_{n=1..N} sum_p (Ez_p^n)^2
 * (Ez at the probes of mfd_set_probes after each of the next N = nsteps
 * steps) with respect to the relative permittivity of every E node and the
 * amplitude of every source, by the discrete adjoint of the step: the exact
 * transpose of Eq. 19 run backwards in time with transposed stencil gathers.
 * The step is linear in the fields, so the adjoint needs the forward run only
 * through Ez of every level:
 *   every == 0: Ez of all nsteps + 1 levels is kept on the device when it fits
 *     in a quarter of the free device memory (nothing is recomputed), else as
 *     every == 64;
 *   every >= 1: the forward run keeps a full-state checkpoint every `every`
 *     steps and the backward sweep recomputes one segment at a time from its
 *     checkpoint, so device memory grows as nsteps / every states plus
 *     `every` Ez fields.
 * Both give the same gradient up to the order of atomic additions where two
 * sources or two probes share a node. Collocated 2D problems (the staggered
 * layout would need the transposes of its two cross-set curl stencils and
 * two node sets' adjoint states, and the 3D layout six adjoint components; the
 * differentiation workload is collocated 2D, so only it is built); probes must hold
 * >= nsteps steps. g_eps: host, count(E nodes), caller's order; g_amp: host,
 * one per source (may be NULL without sources); *J receives J. The simulation
 * is left after step start + nsteps, with its probes recorded from the start
 * of the call. every < 0 is MFD_ERR_ARG. */
mfd_status mfd_grad(mfd_sim* sim, int64_t nsteps, int64_t every, double* J, double* g_eps, double* g_amp);
/* The gradient of mfd_grad in two halves, for automatic differentiation whose
 * forward pass computes J and whose backward pass comes later, or not at all:
 *   mfd_grad_forward runs the nsteps steps (from the current state, probes as
 *   in mfd_grad) recording what the adjoint needs (the Ez history, or full
 *   checkpoints every `every` steps, as mfd_grad), writes J and returns a tape;
 *   mfd_grad_backward runs the adjoint sweep over the recorded run and writes
 *   g_eps (count(E nodes), caller order) and g_amp (one per source): host
 *   arrays with on_device = 0 (synchronous), or device FP64 arrays with
 *   on_device = 1, ordered after the work queued on `stream` and before what
 *   the caller queues on it afterwards.
 * The sweep uses the simulation's weights, materials and sources: keep them as
 * they were in the forward half, and do not step the simulation in between
 * (MFD_ERR_STATE). A tape sweeps once (MFD_ERR_STATE after); the simulation is
 * left at the end of the recorded run. mfd_tape_destroy frees a tape (before
 * its simulation). mfd_grad is these two calls in turn. */
typedef struct mfd_tape mfd_tape;
mfd_status mfd_grad_forward(mfd_sim* sim, int64_t nsteps, int64_t every, double* J, mfd_tape** tape);
mfd_status mfd_grad_backward(mfd_tape* tape, double* g_eps, double* g_amp, int on_device, void* stream);
void mfd_tape_destroy(mfd_tape* tape);
/* The probe objective J = dt sum_n sum_p (Ez_p^n)^2 over the probe records
 * since mfd_set_probes (Eq. 20's companion objective of the gradient calls),
 * for a forward run that needs no gradient. */
mfd_status mfd_probe_objective(mfd_sim* sim, double* J);
/* Number of adjoint sweeps this simulation has run (mfd_grad, mfd_grad_backward). */
int64_t mfd_sim_adjoint_sweeps(const mfd_sim* sim);
/* Zero-copy variants of the differentiable inputs: eps_r (device FP64,
 * count(E nodes), caller order; NULL = vacuum; values must be > 0, checked on
 * the device: MFD_ERR_ARG) with pec (device uint8 in caller order, NULL = none)
 * as mfd_set_materials; and the amplitudes of the sources already set (device
 * FP64, one per source). Stream ordering as mfd_set_field_device. */
mfd_status mfd_set_materials_device(mfd_sim* sim, const double* eps_r, const uint8_t* pec, void* stream);
mfd_status mfd_set_source_amps_device(mfd_sim* sim, const double* amp, void* stream);
/* Number of steps taken since the last mfd_set_field(MFD_EZ). */
int64_t mfd_sim_steps(const mfd_sim* sim);
/* Checkpoint / resume of a long run (the paper has no counterpart). The state
 * is what the next step reads, as it sits on the device (bit for bit, in the
 * library's internal node order): E at t_n and H at t_n - dt/2 with the
 * layout's ping-pong buffers (in the collocated 2D layout the per-node E
 * coefficient dt / (eps0 eps_r) sits beside the fields and travels with
 * them), the step index n, and the probe records since mfd_set_probes.
 * Weights, materials, sources and the probe nodes are configuration, not
 * state: load into a simulation built the same way (same weights, layout,
 * precision, materials and sources; the same probes with at least the saved
 * records' capacity), and the run continued from the loaded state is
 * bit-identical to the unbroken run. host is a caller buffer (save: at least
 * mfd_sim_state_size bytes; load: `bytes` bytes of a saved state). A blob whose
 * header does not match (kind, version, layout, precision, node counts, buffer
 * sizes, probes) is MFD_ERR_ARG before anything is changed. */
mfd_status mfd_sim_state_size(const mfd_sim* sim, size_t* bytes);
mfd_status mfd_sim_save_state(mfd_sim* sim, void* host, size_t bytes);
mfd_status mfd_sim_load_state(mfd_sim* sim, const void* host, size_t bytes);
void mfd_sim_destroy(mfd_sim* sim);


/* ------------------------------------------------------------- batches */

/* Many independent collocated TMz problems ("domains", Eq. 19 each), every
 * one with nrhs right-hand sides: field vectors stepped with the same weights
 * (for example one per point source). One persistent cooperative kernel runs
 * all the steps of a mfd_batch_step call for every domain and right-hand side,
 * captured in a CUDA graph (with a direct launch as the fallback where the
 * capture is refused). Its phases are separated by grid barriers whose waits
 * are bounded: a barrier that waits too long makes every block leave the
 * kernel and the call return MFD_ERR_TIMEOUT.
 *   descs[d]: one collocated 2D FP32 problem per domain (h_curl == e_curl,
 *   h_hv == e_hv, both on one stencils object of the domain's node set);
 *   domains may differ in size, stencil size and coefficients.
 *   nrhs: 4, 8, 16 or 32.
 * Fields, sources and probes are addressed per domain; node ids are the
 * caller's ids within the domain. rhs = -1 in set/get_field means all
 * right-hand sides at once (host array n x nrhs, right-hand side fastest).
 * Materials: eps_r (NULL = 1) and pec (nonzero holds Ez at 0) per domain. */
typedef struct mfd_batch mfd_batch;
mfd_status mfd_batch_create(mfd_ctx* ctx, int ndom, const mfd_sim_desc* descs, int nrhs, mfd_batch** out);
mfd_status mfd_batch_set_materials(mfd_batch* b, int dom, const double* eps_r, const uint8_t* pec);
mfd_status mfd_batch_set_field(mfd_batch* b, int dom, int comp, int rhs, const double* host);
mfd_status mfd_batch_get_field(mfd_batch* b, int dom, int comp, int rhs, double* host);
/* Zero-copy variants (device FP64 n x nrhs, or n for one rhs; stream ordering
 * as mfd_set_field_device). */
mfd_status mfd_batch_set_field_device(mfd_batch* b, int dom, int comp, int rhs, const double* dev, void* stream);
mfd_status mfd_batch_get_field_device(mfd_batch* b, int dom, int comp, int rhs, double* dev, void* stream);
/* Soft Ricker sources of domain dom (as mfd_set_sources); rhs[s] selects the
 * right-hand side source s drives. */
mfd_status mfd_batch_set_sources(mfd_batch* b, int dom, int count, const int64_t* node, const int32_t* rhs,
                                 const double* amp, const double* f0, const double* t0);
/* Probes of domain dom: Ez of every right-hand side after each step, for at
 * most `capacity` steps (the batch keeps the largest capacity asked). */
mfd_status mfd_batch_set_probes(mfd_batch* b, int dom, int count, const int64_t* node, int64_t capacity);
/* Advances every domain and right-hand side nsteps steps. A grid barrier
 * that waits longer than the spin limit (mfd_batch_set_spin_limit) makes every
 * block leave the kernel: the call returns MFD_ERR_TIMEOUT, the step counter
 * is not advanced and the fields are left part way through the call (set
 * them again before stepping on); the batch stays usable. */
mfd_status mfd_batch_step(mfd_batch* b, int64_t nsteps);
/* Bound of the grid-barrier waits of the batched kernel (failure detection:
 * a persistent kernel never waits without limit on a shared GPU). A waiting
 * block polls the barrier at most `limit` times, napping 64 ns between polls,
 * then raises the error flag that makes every block leave. Default 2^25 (a
 * few seconds). limit = 0 makes any block that has to wait give up at its
 * first poll, which exercises the timeout path. */
mfd_status mfd_batch_set_spin_limit(mfd_batch* b, uint64_t limit);
/* Variant of the batched kernel. Bit 0 selects the stream loads: clear, every
 * warp requests the index and weight streams of the next chunk of four stencil
 * entries while it gathers the current one, three resident blocks of 256
 * threads per SM; set, each chunk's streams are loaded when it starts, and the
 * kernel is limited to the registers of four resident blocks per SM (more warps
 * hide the latency instead). Bit 1 selects where the hyperviscosity term of the
 * H row of Eq. 19 is summed: clear, in the H pass, which gathers Ez, Hx and Hy
 * over the whole index row, while the E pass gathers Hx, Hy over the curl
 * stencil; set, in the E pass of the step before (it depends only on
 * H^{n-1/2}, which that pass gathers for its curl): the E pass gathers Hx, Hy
 * over the whole row and keeps H* = H + (dt/mu0) gamma D H beside the state
 * (8 nrhs bytes per node, allocated when such a variant is first selected),
 * and the H pass gathers only Ez, so a step gathers 3L rows of right-hand sides
 * per node instead of 3L + 2n (L the row length, n the curl stencil). Variants
 * with the same bit 1 give bit-identical results; the two forms agree to
 * rounding (the HV term is added to H before the curl term instead of after).
 * After a host write to the fields, materials or gamma, the next step of a
 * variant 2 or 3 first computes H* of the state (one extra pass). Variants 0-3;
 * MFD_ERR_ARG for another. */
mfd_status mfd_batch_set_variant(mfd_batch* b, int variant);
int mfd_batch_variant(const mfd_batch* b);
/* Autotuner: times `reps` steps of each variant on this batch (one launch
 * each, CUDA events), keeps the fastest, and puts the fields, probe records and
 * step counter back after every trial, so the batch does not advance.
 * chosen (nullable) receives the variant, ms (nullable, 4 values) the
 * milliseconds per step of each. */
mfd_status mfd_batch_autotune(mfd_batch* b, int reps, int* chosen, double* ms);
/* host: steps x count x nrhs FP64; *steps receives the recorded steps. */
mfd_status mfd_batch_read_probes(mfd_batch* b, int dom, double* host, int64_t* steps);
int64_t mfd_batch_nodes(const mfd_batch* b);
/* 1 when mfd_batch_step replays a captured CUDA graph, 0 for direct launches. */
int mfd_batch_uses_graph(const mfd_batch* b);
/* The hyperviscosity coefficient gamma of every right-hand side of domain dom
 * (host, nrhs FP64, finite; replaces the domain's gamma from mfd_batch_create,
 * which all right-hand sides start with). Right-hand sides that differ only in
 * gamma run several values of the coefficient of Eq. 18 in one launch. */
mfd_status mfd_batch_set_gamma(mfd_batch* b, int dom, const double* gamma);
/* Energy of Eq. 20 of every right-hand side of domain dom in its current state
 * (host output, nrhs FP64): sum over nodes of eps_r Ez^2 + eta0^2 |H|^2 with H
 * averaged between t - dt/2 and t + dt/2 (the next H half step is computed,
 * not applied), eta0^2 = mu0 / eps0, as mfd_energy. */
mfd_status mfd_batch_energy(mfd_batch* b, int dom, double* u);
/* Checkpoint / resume of a batch, as mfd_sim_save_state: every domain's and
 * right-hand side's fields at step n (FP32, internal order), n, and the probe
 * records since mfd_batch_set_probes. Load into a batch created from the same
 * domains and nrhs, with the same materials, sources, gammas and probes. */
mfd_status mfd_batch_state_size(const mfd_batch* b, size_t* bytes);
mfd_status mfd_batch_save_state(mfd_batch* b, void* host, size_t bytes);
mfd_status mfd_batch_load_state(mfd_batch* b, const void* host, size_t bytes);
void mfd_batch_destroy(mfd_batch* b);

/* ------------------------------------------------- hyperviscosity search */

/* The coefficient c of gamma = c (-1)^(alpha-1) h^(2 alpha) (Sec. 5.1, with h
 * = 1 in the caller's units) by multisection on log10 c, the search by which
 * the paper picks c (Sec. 5.1, Sec. 6). Reading: the paper names the method
 * (a bisection) but not its criterion; here the answer is the smallest stable
 * c of [10^log10_lo, 10^log10_hi] to the search's resolution, the least
 * dissipative stable choice.
 *   Round r runs ncand (4, 8, 16 or 32) candidates log10 c_k = lo + (hi - lo)
 *   (k + 1) / ncand, k = 0 .. ncand - 1, at once as right-hand sides of one
 *   batched collocated FP32 domain (curl, hv: weights on one own-set stencil
 *   set, as mfd_batch_create; alpha from hv), each from the fields ez, hx, hy
 *   (host, caller order; H at t - dt/2) and the optional materials eps_r /
 *   pec (NULL: vacuum, no PEC), for nsteps steps. Candidate k is stable when
 *   u(t) = U(t) / U(0) (Eq. 20, mfd_batch_energy) stays <= 1 + tol and finite
 *   at every check, taken every check_every steps and after the last step.
 *   The next interval is [c_{k*-1}, c_{k*}] around the first stable candidate
 *   k* (lo kept when k* = 0).
 * Out: *c_out = 10^hi after `rounds` rounds (a stable value); history (host,
 * nullable) [rounds][ncand][3] = (log10 c_k, max u, final u), a round that
 * stops early (every candidate failed) reports its last u. No stable candidate
 * in a round (the upper end must be stable) is MFD_ERR_UNSTABLE with
 * *c_out = NaN and the history up to that round. */
mfd_status mfd_hv_search(mfd_ctx* ctx, const mfd_weights* curl, const mfd_weights* hv, double dt, double eps0,
                         double mu0, const double* eps_r, const uint8_t* pec, const double* ez, const double* hx,
                         const double* hy, double log10_lo, double log10_hi, int ncand, int rounds, int64_t nsteps,
                         int64_t check_every, double tol, double* c_out, double* history);

/* ----------------------------------------------------------- diagnostics */

/* Measured FMA throughput of `device` in GFLOP/s (FP64 and FP32): eight
 * independent FMA chains per thread on every SM, best of five timed launches.
 * The paper has no counterpart; it is the denominator of the FP64 step's ALU
 * roofline. */
mfd_status mfd_fma_peak(int device, double* fp64_gflops, double* fp32_gflops);

/* ------------------------------------------------------- FDTD reference */

/* The FDTD (Yee) scheme for TMz (Eq. 4, Eq. 5), the grid method the paper
 * generalises and compares with (Sec. 3, Sec. 6), on a periodic nx x ny grid
 * of spacing h: Ez[j][i] at (i h, j h) and time n dt, Hx[j][i] at
 * (i h, (j + 1/2) h) and Hy[j][i] at ((i + 1/2) h, j h), both at (n - 1/2) dt.
 * A step is Eq. 5 with S_c / eta0 = dt / (mu0 h) and eta0 S_c = dt / (eps0 h)
 * (stable for S_c <= 1/sqrt(2)), then soft Ricker sources (as mfd_set_sources,
 * cell index j nx + i), then probes. One fused kernel per step (four steps per
 * launch when there are no sources and probes); long runs replay a CUDA graph.
 * FP64 results equal the reference arithmetic of Eq. 5 taken term by term (no
 * fused multiply-add) bit for bit.
 * 2 <= nx < 2^30, 2 <= ny <= 1834980 (65535 rows of blocks of the four-step kernel's
 * 28-row tiles); fields in host arrays are ny x nx FP64. */
typedef struct mfd_yee mfd_yee;
mfd_status mfd_yee_create(mfd_ctx* ctx, int64_t nx, int64_t ny, int precision, double dt, double h, double eps0,
                          double mu0, mfd_yee** out);
/* comp: MFD_EZ, MFD_HX or MFD_HY; host ny x nx FP64. */
mfd_status mfd_yee_set_field(mfd_yee* y, int comp, const double* host);
mfd_status mfd_yee_get_field(mfd_yee* y, int comp, double* host);
mfd_status mfd_yee_set_sources(mfd_yee* y, int count, const int64_t* cell, const double* amp, const double* f0,
                               const double* t0);
/* Ez of `count` cells after each step, for at most `capacity` steps. */
mfd_status mfd_yee_set_probes(mfd_yee* y, int count, const int64_t* cell, int64_t capacity);
mfd_status mfd_yee_step(mfd_yee* y, int64_t nsteps);
/* nsteps steps, each launch bracketed by CUDA events; *ms = the summed launch times. */
mfd_status mfd_yee_step_timed(mfd_yee* y, int64_t nsteps, double* ms);
/* Steps one kernel launch advances: 4 without sources and probes (four steps
 * fused in one launch, a quarter of the DRAM traffic per step; results equal
 * the one-step kernel's bit for bit), else 1. */
int mfd_yee_steps_per_launch(const mfd_yee* y);
/* host: steps x count FP64; *steps receives the recorded steps. */
mfd_status mfd_yee_read_probes(mfd_yee* y, double* host, int64_t* steps);
void mfd_yee_destroy(mfd_yee* y);

/* ------------------------------------------------------------ dispersion */

/* Numerical dispersion of a run (Sec. 6, Eqs. 24-26), computed on the GPU in
 * FP64. Input: Ez sampled at nx equispaced nodes of a line (spacing h_line
 * along it, in the order of increasing position along the propagation
 * direction) at nt instants dt_sample apart: samples[n][m], host, nt x nx.
 *   spectrum |E(k_i, w_j)| = |sum_n sum_m w_n s[n][m] exp(-i k_i x_m)
 *            exp(+i w_j t_n)| with the symmetric Hann window
 *            w_n = 1/2 - 1/2 cos(2 pi n / (nt - 1)) in time (w = 1 if nt == 1),
 *            k_i = 2 pi i / (nx h_line), w_j = 2 pi j / (nt dt_sample), so a
 *            wave travelling along the line appears at positive k and w;
 *   kidx[j] = argmax over 0 <= i < nx of |E(k_i, w_j)| (smallest i on ties);
 *   c[j]    = w_j / k_kidx[j] (Eq. 24): NaN for j = 0, +inf if kidx[j] = 0;
 *   err_l1  = sum over 1 <= j <= jmax of |c[j] - c_ref| (Eqs. 25-26; Eq. 26
 *             starts at j = 0, where w_0 = 0 leaves c undefined).
 * Outputs (host, each may be NULL): spectrum nt x nx (row j), kidx nt int32,
 * c nt, err_l1 one double. 1 <= nx, nt <= 4096; 0 <= jmax < nt. */
mfd_status mfd_dispersion(mfd_ctx* ctx, int nx, int nt, const double* samples, double h_line, double dt_sample,
                          double c_ref, int jmax, double* spectrum, int32_t* kidx, double* c, double* err_l1);
/* The same analysis of a simulation's own probe series, without a host round
 * trip: the probes (mfd_set_probes, in line order) are the nx line nodes and
 * the samples are the records after steps stride, 2 stride, ..., nt stride
 * counted from mfd_set_probes (dt_sample = stride dt). Needs nt * stride
 * recorded steps. */
mfd_status mfd_sim_dispersion(mfd_sim* sim, int stride, int nt, double h_line, double c_ref, int jmax,
                              double* spectrum, int32_t* kidx, double* c, double* err_l1);
/* Phase speed, in h per dt, of the FDTD (Yee) scheme on a square grid with
 * Courant number S = c dt / h at angular frequency omega (omega_dt = omega dt)
 * and propagation angle phi (Eq. 6), on the branch through k = 0; NaN above
 * the grid's cut-off. Host only. */
mfd_status mfd_fdtd_phase_speed(double omega_dt, double courant, double phi, double* c);

/* ------------------------------------------- partition and halo (host only) */

/* Decomposition of the stepped problem over several GPUs, one shard each. The
 * paper runs on one machine and has no decomposition; these calls give the
 * index structures a sharded run needs, with no communication: every stencil
 * sum of Eq. 16 at a node a shard owns reads owned nodes and a halo of nodes
 * owned by other shards, and one exchange of the field just updated (E before
 * the H half step, H before the E half step of Eq. 19) refreshes the halo.
 * These calls run on the host only: they make no CUDA call and work without a
 * GPU. Partitions and halo plans copy what they need and hold no reference on
 * other objects. */
typedef struct mfd_partition mfd_partition;
typedef struct mfd_halo mfd_halo;

/* Cuts the n nodes of a set, taken in `order` (host, n caller ids, a
 * permutation: order[r] = caller id of the r-th node; NULL = caller order;
 * mfd_nodes_permutation gives the library's Morton order), into nshards
 * contiguous ranges: shard s owns positions [floor(s n / nshards),
 * floor((s + 1) n / nshards)), so shard sizes differ by at most one.
 * 1 <= nshards <= 65536; n >= 0. A non-permutation order is MFD_ERR_ARG. */
mfd_status mfd_partition_create(int64_t n, const int64_t* order, int nshards, mfd_partition** out);
/* owner: host, n int32 output: the shard owning each node (caller id). */
mfd_status mfd_partition_owner(const mfd_partition* part, int32_t* owner);
/* The nodes `shard` owns, in partition order: *count is always set; ids
 * (host, *count int64, caller ids) is written when not NULL. */
mfd_status mfd_partition_owned(const mfd_partition* part, int shard, int64_t* count, int64_t* ids);
void mfd_partition_destroy(mfd_partition* part);

/* Halo plan of one source node set (partitioned by `src`) for the nsets
 * stencil sets that read it. Stencil set k has its centres partitioned by
 * centres[k] (a partition with as many nodes as set k has rows; it may be
 * `src` itself for own-set stencils) and ncols[k] entries per row; idx[k] is
 * host int64 [rows][ncols[k]], caller ids into the source set, rows in the
 * caller order of the centres (mfd_stencils_read). The halo of shard s is the
 * set of source nodes that some stencil of a centre s owns references and
 * that another shard owns; it is ordered by owning shard, then by partition
 * order. An entry outside [0, count(src)) is MFD_ERR_ARG. 1 <= nsets <= 16. */
mfd_status mfd_halo_create(const mfd_partition* src, int nsets, const mfd_partition* const* centres,
                           const int* ncols, const int64_t* const* idx, mfd_halo** out);
/* Number of halo nodes of `shard` (*count), optionally their caller ids (ids,
 * host, *count int64, halo order). */
mfd_status mfd_halo_nodes(const mfd_halo* halo, int shard, int64_t* count, int64_t* ids);
/* The source nodes shard `from` sends to shard `to` in each exchange, in the
 * order they take in the receiver's halo (a contiguous block of it): *count is
 * always set (0 when from == to), ids (host, *count int64, caller ids) is
 * written when not NULL. */
mfd_status mfd_halo_send(const mfd_halo* halo, int from, int to, int64_t* count, int64_t* ids);
/* Stencil set k localised to `shard`: local_idx (host int32 [owned centres of
 * shard][ncols[k]], rows in partition order of the centres) holds, for every
 * entry, the local source index: p in [0, owned) for the p-th owned source
 * node (partition order), owned + j for the j-th halo node. A shard that keeps
 * its owned values followed by its halo in one array applies the stencils
 * unchanged on it. */
mfd_status mfd_halo_local_idx(const mfd_halo* halo, int shard, int set, int32_t* local_idx);
void mfd_halo_destroy(mfd_halo* halo);

/* ------------------------------------------------- kNN without allocation */

/* The kNN stencils of mfd_stencils_build, computed on caller-owned device
 * arrays by a call that allocates no device memory at all. (The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc, for example because the host application owns all device memory
 * through its own pool or forbids allocation once it has started.)
 *   centres: device, nc x dim FP64; sources: device, ns x dim FP64, both in
 *   the caller's order; period: host, dim entries (0 = not periodic);
 *   idx: device, nc x n int32 output, the source indices of each stencil
 *   sorted by (squared distance, source index) -- the same stencils, entry
 *   for entry, that mfd_stencils_build + mfd_stencils_read return.
 *   stream: cudaStream_t (NULL = legacy default stream).
 * Source coordinates of a periodic axis must lie in [0, period) (checked on
 * the bounding box: MFD_ERR_ARG otherwise).
 * All scratch lives in one file-scope device array of 32 MiB (enough for
 * about 1,000,000 sources) that every GPU which loads the library holds until
 * the process exits; larger source sets are rejected with MFD_ERR_ARG and a
 * message. Every call shares that array and leaves its contents behind, so two
 * calls that overlap on the GPU (other streams, other host threads) race: the
 * caller must order them. The first call on each device looks up the array's
 * device address with that device current (set-up); make that first call
 * before any stream capture. If the device's context is torn down and made
 * again (cudaDeviceReset), the next call repeats the set-up. The call
 * synchronises `stream` once (to read the
 * bounding box of the sources) and queues the rest asynchronously. */
mfd_status mfd_knn_static(int dim, int64_t nc, const double* centres, int64_t ns, const double* sources,
                          const double* period, int n, int32_t* idx, void* stream);

#ifdef __cplusplus
}
#endif
#endif
