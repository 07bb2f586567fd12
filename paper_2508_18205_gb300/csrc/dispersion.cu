// dispersion.cu -- numerical dispersion of a run (Sec. 6, Eqs. 24-26) and the
// phase speed of the Yee scheme (Eq. 6).
//
// The transform is small (a line of nx <= 4096 nodes, nt <= 4096 instants), so
// it is written as two direct DFT passes in FP64, one block per output row:
//   time pass : A[j][m] = sum_n w_n s[n][m] exp(+2 pi i j n / nt)  (Hann window)
//   space pass: E[j][i] = sum_m A[j][m] exp(-2 pi i i m / nx)
// with the row's twiddle factors staged in shared memory (integer phase
// indices, reduced modulo the period, so no phase error accumulates). A third
// kernel takes the argmax over i of every row and Eq. 24-25; one thread sums
// Eq. 26 in the order j = 1 .. jmax.
#include <cmath>
#include <limits>
#include <string>
#include <vector>

#include "internal.cuh"

namespace mfd {

constexpr int DISP_MAX = 4096;
constexpr int DISP_THREADS = 256;

__global__ void __launch_bounds__(DISP_THREADS) k_disp_time(const double* __restrict__ s, int nx, int nt,
                                                            double2* __restrict__ A) {
    extern __shared__ double2 tw[];  // nt entries: w_n exp(+2 pi i j n / nt)
    const int j = blockIdx.x;
    for (int n = threadIdx.x; n < nt; n += blockDim.x) {
        const double w = nt > 1 ? 0.5 - 0.5 * cospi(2.0 * (double)n / (double)(nt - 1)) : 1.0;
        const int64_t r = ((int64_t)j * n) % nt;
        double sn, cs;
        sincospi(2.0 * (double)r / (double)nt, &sn, &cs);
        tw[n] = make_double2(w * cs, w * sn);
    }
    __syncthreads();
    for (int m = threadIdx.x; m < nx; m += blockDim.x) {
        double re = 0.0, im = 0.0;
        for (int n = 0; n < nt; ++n) {
            const double v = s[(int64_t)n * nx + m];
            re = fma(tw[n].x, v, re);
            im = fma(tw[n].y, v, im);
        }
        A[(int64_t)j * nx + m] = make_double2(re, im);
    }
}

__global__ void __launch_bounds__(DISP_THREADS) k_disp_space(const double2* __restrict__ A, int nx,
                                                             double* __restrict__ spec) {
    extern __shared__ double2 sm[];  // [0, nx): exp(-2 pi i r / nx); [nx, 2 nx): the row of A
    double2* tw = sm;
    double2* row = sm + nx;
    const int j = blockIdx.x;
    for (int r = threadIdx.x; r < nx; r += blockDim.x) {
        double sn, cs;
        sincospi(2.0 * (double)r / (double)nx, &sn, &cs);
        tw[r] = make_double2(cs, -sn);
        row[r] = A[(int64_t)j * nx + r];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        double re = 0.0, im = 0.0;
        int r = 0;  // (i m) mod nx
        for (int m = 0; m < nx; ++m) {
            const double2 a = row[m], t = tw[r];
            re = fma(a.x, t.x, fma(-a.y, t.y, re));
            im = fma(a.x, t.y, fma(a.y, t.x, im));
            r += i;
            if (r >= nx) r -= nx;
        }
        spec[(int64_t)j * nx + i] = sqrt(re * re + im * im);
    }
}

// Eq. 24 per row j: the first i of largest |E|, c_j = w_j / k_i; Eq. 25
__global__ void __launch_bounds__(DISP_THREADS) k_disp_ridge(const double* __restrict__ spec, int nx, int nt,
                                                             double h_line, double dt_sample, double c_ref,
                                                             int32_t* __restrict__ kidx, double* __restrict__ c,
                                                             double* __restrict__ err) {
    __shared__ double bv[DISP_THREADS];
    __shared__ int bi[DISP_THREADS];
    const int j = blockIdx.x;
    double v = -1.0;
    int at = 0;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const double x = spec[(int64_t)j * nx + i];
        if (x > v) {  // strict: the first (smallest) i of a tie within the thread
            v = x;
            at = i;
        }
    }
    bv[threadIdx.x] = v;
    bi[threadIdx.x] = at;
    __syncthreads();
    for (int w = DISP_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            const double ov = bv[threadIdx.x + w];
            const int oi = bi[threadIdx.x + w];
            if (ov > bv[threadIdx.x] || (ov == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
                bv[threadIdx.x] = ov;
                bi[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int i = bi[0];
        double cj;
        if (j == 0)
            cj = nan("");
        else if (i == 0)
            cj = INFINITY;
        else  // (2 pi j / (nt dt)) / (2 pi i / (nx h))
            cj = ((double)j * (double)nx * h_line) / ((double)i * (double)nt * dt_sample);
        kidx[j] = i;
        c[j] = cj;
        err[j] = fabs(cj - c_ref);
    }
}

__global__ void k_disp_l1(const double* __restrict__ err, int jmax, double* __restrict__ out) {
    double s = 0.0;
    for (int j = 1; j <= jmax; ++j) s += err[j];
    *out = s;
}

mfd_status dispersion_run(mfd_ctx* ctx, int nx, int nt, const double* d_samples, double h_line, double dt_sample,
                          double c_ref, int jmax, double* spectrum, int32_t* kidx, double* c, double* err_l1) {
    cudaStream_t st = ctx->stream;
    DevBuf A, spec, ki, cc, err, l1;
    const int64_t cells = (int64_t)nx * nt;
    MFD_TRY(A.alloc(cells * sizeof(double2)));
    MFD_TRY(spec.alloc(cells * 8));
    MFD_TRY(ki.alloc(nt * 4));
    MFD_TRY(cc.alloc(nt * 8));
    MFD_TRY(err.alloc(nt * 8));
    MFD_TRY(l1.alloc(8));
    const size_t sm_t = (size_t)nt * sizeof(double2), sm_x = 2 * (size_t)nx * sizeof(double2);
    MFD_CUDA(cudaFuncSetAttribute(k_disp_time, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_t));
    MFD_CUDA(cudaFuncSetAttribute(k_disp_space, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_x));
    k_disp_time<<<nt, DISP_THREADS, sm_t, st>>>(d_samples, nx, nt, A.as<double2>());
    MFD_CUDA(cudaGetLastError());
    k_disp_space<<<nt, DISP_THREADS, sm_x, st>>>(A.as<double2>(), nx, spec.as<double>());
    MFD_CUDA(cudaGetLastError());
    k_disp_ridge<<<nt, DISP_THREADS, 0, st>>>(spec.as<double>(), nx, nt, h_line, dt_sample, c_ref, ki.as<int32_t>(),
                                             cc.as<double>(), err.as<double>());
    MFD_CUDA(cudaGetLastError());
    k_disp_l1<<<1, 1, 0, st>>>(err.as<double>(), jmax, l1.as<double>());
    MFD_CUDA(cudaGetLastError());
    if (spectrum) MFD_CUDA(cudaMemcpyAsync(spectrum, spec.p, cells * 8, cudaMemcpyDeviceToHost, st));
    if (kidx) MFD_CUDA(cudaMemcpyAsync(kidx, ki.p, nt * 4, cudaMemcpyDeviceToHost, st));
    if (c) MFD_CUDA(cudaMemcpyAsync(c, cc.p, nt * 8, cudaMemcpyDeviceToHost, st));
    if (err_l1) MFD_CUDA(cudaMemcpyAsync(err_l1, l1.p, 8, cudaMemcpyDeviceToHost, st));
    MFD_CUDA(cudaStreamSynchronize(st));
    return MFD_OK;
}

mfd_status dispersion_check(int nx, int nt, double h_line, double dt_sample, int jmax) {
    if (nx < 1 || nt < 1 || nx > DISP_MAX || nt > DISP_MAX)
        return fail(MFD_ERR_ARG, "dispersion: need 1 <= nx, nt <= " + std::to_string(DISP_MAX));
    if (!(h_line > 0) || !(dt_sample > 0)) return fail(MFD_ERR_ARG, "dispersion: h_line and dt_sample must be > 0");
    if (jmax < 0 || jmax >= nt) return fail(MFD_ERR_ARG, "dispersion: need 0 <= jmax < nt");
    return MFD_OK;
}

}  // namespace mfd

extern "C" {

mfd_status mfd_dispersion(mfd_ctx* ctx, int nx, int nt, const double* samples, double h_line, double dt_sample,
                          double c_ref, int jmax, double* spectrum, int32_t* kidx, double* c, double* err_l1) {
    using namespace mfd;
    if (!ctx || !samples) return fail(MFD_ERR_ARG, "mfd_dispersion: NULL argument");
    MFD_TRY(dispersion_check(nx, nt, h_line, dt_sample, jmax));
    MFD_CUDA(cudaSetDevice(ctx->device));
    DevBuf s;
    MFD_TRY(s.alloc((size_t)nx * nt * 8));
    MFD_CUDA(cudaMemcpyAsync(s.p, samples, (size_t)nx * nt * 8, cudaMemcpyHostToDevice, ctx->stream));
    return dispersion_run(ctx, nx, nt, s.as<double>(), h_line, dt_sample, c_ref, jmax, spectrum, kidx, c, err_l1);
}

mfd_status mfd_fdtd_phase_speed(double omega_dt, double courant, double phi, double* c) {
    if (!c || !(courant > 0) || !(omega_dt >= 0)) return mfd::fail(MFD_ERR_ARG, "mfd_fdtd_phase_speed: bad arguments");
    // Eq. 6 with h = dt = 1: g(kh) = sin^2(kh cos(phi)/2) + sin^2(kh sin(phi)/2)
    // rises monotonically from 0 on [0, pi / max(|cos|, |sin|)]; the root of
    // g = sin^2(omega dt / 2) / S^2 on that interval is the wavenumber.
    const double cp = std::cos(phi), sp = std::sin(phi);
    const double target = std::pow(std::sin(0.5 * omega_dt) / courant, 2);
    auto g = [&](double kh) { return std::pow(std::sin(0.5 * kh * cp), 2) + std::pow(std::sin(0.5 * kh * sp), 2); };
    double lo = 0.0, hi = M_PI / std::fmax(std::fabs(cp), std::fabs(sp));
    if (omega_dt == 0.0) {
        *c = std::numeric_limits<double>::quiet_NaN();
        return MFD_OK;
    }
    if (g(hi) < target) {
        *c = std::numeric_limits<double>::quiet_NaN();
        return MFD_OK;
    }
    while (hi - lo > 1e-15 * hi) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        (g(mid) < target ? lo : hi) = mid;
    }
    *c = omega_dt / (0.5 * (lo + hi));
    return MFD_OK;
}

}  // extern "C"
