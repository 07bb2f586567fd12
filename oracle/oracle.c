/*
 * oracle.c -- plain, slow FP64 CPU reference of the meshless RBF leapfrog.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library. It shares
 * no code, header, table or constant with the CUDA library; the two meet only
 * through the seeded inputs of workloads/.
 *
 * What each part follows (paper: "An RBF-based method for computational
 * electromagnetics with reduced numerical dispersion", arXiv 2508.18205):
 *   O-1 stencils  : the n nodes closest to the centre (Sec. 4.1, Eq. 11),
 *                   ordered by (squared distance, node id); periodic axes use
 *                   the minimum image.
 *   O-2 weights   : the local PHS + monomial saddle system of Eq. 9 with the
 *                   operator applied to the basis (RBF-FD, Eq. 13) or a central
 *                   difference of the interpolant at x_c +- delta e (RBF-VFD,
 *                   Eqs. 14-15); hyperviscosity Delta^alpha by RBF-FD (Sec. 5.1).
 *                   Coordinates are shifted to x_c and scaled by the stencil
 *                   radius; the system is solved by Gaussian elimination with
 *                   partial pivoting.
 *   O-3 stepping  : the stabilised interleaved leapfrog of Eq. 19 (TMz) and its
 *                   3D full-vector form (Eq. 2 with the terms of Eqs. 17-18),
 *                   with soft Ricker sources added after the E update, then the
 *                   PEC condition, then the probes.
 *   O-4 energy    : Eq. 20 with H averaged between the two half steps.
 *   O-5 adjoint   : the exact transpose of O-3 (TMz), by scatter loops.
 *
 * Every stencil sum runs sequentially in stencil order in FP64.
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG -1
#define ORC_ERR_SINGULAR -4
#define ORC_ERR_OOM -2

/* ------------------------------------------------------------------ O-1 */

/* minimum-image offset along one axis (period 0 = not periodic) */
static double orc_wrap(double d, double period)
{
    if (period > 0.0) {
        if (d > 0.5 * period) d -= period;
        else if (d < -0.5 * period) d += period;
    }
    return d;
}

static double orc_d2(int dim, const double* c, const double* x, const double* period)
{
    double s = 0.0;
    for (int a = 0; a < dim; ++a) {
        double d = orc_wrap(x[a] - c[a], period[a]);
        double p = d * d;
        s = s + p;
    }
    return s;
}

/* keeps the n best (d2, id) pairs in ascending order; returns new count */
static int orc_insert(int n, int cnt, double* bd, int64_t* bi, double d2, int64_t id)
{
    if (cnt == n) {
        double ld = bd[n - 1];
        int64_t li = bi[n - 1];
        if (d2 > ld || (d2 == ld && id >= li)) return cnt;
        cnt = n - 1;
    }
    int p = cnt;
    while (p > 0 && (bd[p - 1] > d2 || (bd[p - 1] == d2 && bi[p - 1] > id))) {
        bd[p] = bd[p - 1];
        bi[p] = bi[p - 1];
        --p;
    }
    bd[p] = d2;
    bi[p] = id;
    return cnt + 1;
}

/* Brute force: every source node is a candidate for every centre. */
int orc_knn_brute(int dim, int64_t nc, const double* xc, int64_t ns, const double* xs,
                  const double* period, int n, int64_t* idx)
{
    if (dim < 1 || dim > 3 || n < 1 || n > ns) return ORC_ERR_ARG;
    int bad = 0;
#pragma omp parallel
    {
        double* bd = (double*)malloc(sizeof(double) * n);
        int64_t* bi = (int64_t*)malloc(sizeof(int64_t) * n);
        if (!bd || !bi) {
#pragma omp atomic write
            bad = 1;
        } else {
#pragma omp for schedule(static)
            for (int64_t c = 0; c < nc; ++c) {
                int cnt = 0;
                for (int64_t j = 0; j < ns; ++j)
                    cnt = orc_insert(n, cnt, bd, bi, orc_d2(dim, xc + c * dim, xs + j * dim, period), j);
                memcpy(idx + c * n, bi, sizeof(int64_t) * n);
            }
        }
        free(bd);
        free(bi);
    }
    return bad ? ORC_ERR_OOM : ORC_OK;
}

/* Cell list: sources binned in boxes of side >= cs; rings of boxes are added
 * around the centre's box until the n-th distance is below the radius that
 * the visited rings are guaranteed to cover. Falls back to brute force for a
 * centre when a ring would wrap onto itself. */
int orc_knn_cells(int dim, int64_t nc, const double* xc, int64_t ns, const double* xs,
                  const double* period, int n, double cs, int64_t* idx)
{
    if (dim < 1 || dim > 3 || n < 1 || n > ns || !(cs > 0)) return ORC_ERR_ARG;
    double lo[3] = {0, 0, 0}, side[3] = {1, 1, 1};
    int64_t nb[3] = {1, 1, 1};
    for (int a = 0; a < dim; ++a) {
        double mn = xs[a], mx = xs[a];
        for (int64_t j = 0; j < ns; ++j) {
            if (xs[j * dim + a] < mn) mn = xs[j * dim + a];
            if (xs[j * dim + a] > mx) mx = xs[j * dim + a];
        }
        double ext;
        if (period[a] > 0) { lo[a] = 0.0; ext = period[a]; }
        else { lo[a] = mn; ext = mx - mn; }
        nb[a] = (int64_t)floor(ext / cs);
        if (nb[a] < 1) nb[a] = 1;
        side[a] = ext / (double)nb[a];
        if (!(side[a] > 0)) side[a] = cs;
    }
    int64_t ncell = nb[0] * nb[1] * nb[2];
    int64_t* start = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
    int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (size_t)ns);
    int64_t* cellof = (int64_t*)malloc(sizeof(int64_t) * (size_t)ns);
    if (!start || !list || !cellof) { free(start); free(list); free(cellof); return ORC_ERR_OOM; }
    for (int64_t j = 0; j < ns; ++j) {
        int64_t ci[3] = {0, 0, 0};
        for (int a = 0; a < dim; ++a) {
            int64_t k = (int64_t)floor((xs[j * dim + a] - lo[a]) / side[a]);
            if (k < 0) k = 0;
            if (k >= nb[a]) k = nb[a] - 1;
            ci[a] = k;
        }
        cellof[j] = (ci[2] * nb[1] + ci[1]) * nb[0] + ci[0];
        start[cellof[j] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
    {
        int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
        if (!fill) { free(start); free(list); free(cellof); return ORC_ERR_OOM; }
        memcpy(fill, start, sizeof(int64_t) * (size_t)ncell);
        for (int64_t j = 0; j < ns; ++j) list[fill[cellof[j]]++] = j;
        free(fill);
    }
    int bad = 0;
#pragma omp parallel
    {
        double* bd = (double*)malloc(sizeof(double) * n);
        int64_t* bi = (int64_t*)malloc(sizeof(int64_t) * n);
        if (!bd || !bi) {
#pragma omp atomic write
            bad = 1;
        } else {
#pragma omp for schedule(dynamic, 64)
            for (int64_t c = 0; c < nc; ++c) {
                const double* x = xc + c * dim;
                int64_t c0[3] = {0, 0, 0};
                for (int a = 0; a < dim; ++a) {
                    int64_t k = (int64_t)floor((x[a] - lo[a]) / side[a]);
                    if (k < 0) k = 0;
                    if (k >= nb[a]) k = nb[a] - 1;
                    c0[a] = k;
                }
                double smin = side[0];
                for (int a = 1; a < dim; ++a) if (side[a] < smin) smin = side[a];
                int cnt = 0, done = 0, brute = 0;
                for (int64_t R = 0; !done; ++R) {
                    int wraps = 0, all = 1;
                    for (int a = 0; a < dim; ++a) {
                        if (period[a] > 0 && 2 * R + 1 > nb[a]) wraps = 1;
                        if (period[a] > 0 || c0[a] - R > 0 || c0[a] + R < nb[a] - 1) all = 0;
                    }
                    if (wraps) { brute = 1; break; }
                    int64_t r1 = dim > 1 ? R : 0, r2 = dim > 2 ? R : 0;
                    for (int64_t oz = -r2; oz <= r2; ++oz)
                        for (int64_t oy = -r1; oy <= r1; ++oy)
                            for (int64_t ox = -R; ox <= R; ++ox) {
                                int64_t m = llabs(ox);
                                if (llabs(oy) > m) m = llabs(oy);
                                if (llabs(oz) > m) m = llabs(oz);
                                if (m != R) continue;
                                int64_t o[3] = {ox, oy, oz}, k[3] = {0, 0, 0};
                                int skip = 0;
                                for (int a = 0; a < dim; ++a) {
                                    k[a] = c0[a] + o[a];
                                    if (period[a] > 0) k[a] = ((k[a] % nb[a]) + nb[a]) % nb[a];
                                    else if (k[a] < 0 || k[a] >= nb[a]) skip = 1;
                                }
                                if (skip) continue;
                                int64_t cell = (k[2] * nb[1] + k[1]) * nb[0] + k[0];
                                for (int64_t q = start[cell]; q < start[cell + 1]; ++q) {
                                    int64_t j = list[q];
                                    cnt = orc_insert(n, cnt, bd, bi, orc_d2(dim, x, xs + j * dim, period), j);
                                }
                            }
                    double rg = (double)R * smin * (1.0 - 1e-12);
                    if (all) done = 1;
                    else if (cnt == n && bd[n - 1] < rg * rg) done = 1;
                }
                if (brute) {
                    cnt = 0;
                    for (int64_t j = 0; j < ns; ++j)
                        cnt = orc_insert(n, cnt, bd, bi, orc_d2(dim, x, xs + j * dim, period), j);
                }
                memcpy(idx + c * n, bi, sizeof(int64_t) * n);
            }
        }
        free(bd);
        free(bi);
    }
    free(start);
    free(list);
    free(cellof);
    return bad ? ORC_ERR_OOM : ORC_OK;
}

/* ------------------------------------------------------------------ O-2 */

/* monomials of total degree <= m in graded order (1, x, y, x^2, xy, y^2, ...) */
int orc_monomials(int dim, int m, int* e /* out: count x 3 */)
{
    int q = 0;
    for (int deg = 0; deg <= m; ++deg) {
        if (dim == 1) { e[3 * q] = deg; e[3 * q + 1] = 0; e[3 * q + 2] = 0; ++q; continue; }
        for (int a = deg; a >= 0; --a) {
            if (dim == 2) { e[3 * q] = a; e[3 * q + 1] = deg - a; e[3 * q + 2] = 0; ++q; continue; }
            for (int b = deg - a; b >= 0; --b) {
                e[3 * q] = a; e[3 * q + 1] = b; e[3 * q + 2] = deg - a - b; ++q;
            }
        }
    }
    return q;
}

static double orc_ipow(double x, int k)
{
    double r = 1.0;
    for (int i = 0; i < k; ++i) r *= x;
    return r;
}

static double orc_mono(int dim, const int* e, const double* z)
{
    double v = 1.0;
    for (int a = 0; a < dim; ++a) v *= orc_ipow(z[a], e[a]);
    return v;
}

static double orc_norm(int dim, const double* z)
{
    double s = 0.0;
    for (int a = 0; a < dim; ++a) s += z[a] * z[a];
    return sqrt(s);
}

/* phi(r) = r^k with k odd */
static double orc_phs(double r, int k) { return orc_ipow(r, k); }

static double orc_factorial(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

/* Delta^alpha of the monomial with exponents e, at the origin. Nonzero only
 * when e = 2*beta with |beta| = alpha: then alpha!/beta! * prod (2 beta_a)!. */
static double orc_lap_pow_mono0(int dim, const int* e, int alpha)
{
    int tot = 0;
    for (int a = 0; a < dim; ++a) {
        if (e[a] % 2) return 0.0;
        tot += e[a];
    }
    if (tot != 2 * alpha) return 0.0;
    double v = orc_factorial(alpha);
    for (int a = 0; a < dim; ++a) v = v / orc_factorial(e[a] / 2) * orc_factorial(e[a]);
    return v;
}

/* Gaussian elimination with partial pivoting on the K x K row-major matrix A
 * with nr right-hand sides B (K x nr, row-major); B is overwritten by the
 * solution. Returns ORC_ERR_SINGULAR on an exactly zero pivot. */
int orc_gepp(int K, double* A, int nr, double* B)
{
    for (int p = 0; p < K; ++p) {
        int piv = p;
        double best = fabs(A[p * K + p]);
        for (int r = p + 1; r < K; ++r)
            if (fabs(A[r * K + p]) > best) { best = fabs(A[r * K + p]); piv = r; }
        if (best == 0.0) return ORC_ERR_SINGULAR;
        if (piv != p) {
            for (int c = 0; c < K; ++c) { double t = A[p * K + c]; A[p * K + c] = A[piv * K + c]; A[piv * K + c] = t; }
            for (int c = 0; c < nr; ++c) { double t = B[p * nr + c]; B[p * nr + c] = B[piv * nr + c]; B[piv * nr + c] = t; }
        }
        for (int r = p + 1; r < K; ++r) {
            double f = A[r * K + p] / A[p * K + p];
            if (f == 0.0) continue;
            for (int c = p; c < K; ++c) A[r * K + c] -= f * A[p * K + c];
            for (int c = 0; c < nr; ++c) B[r * nr + c] -= f * B[p * nr + c];
        }
    }
    for (int p = K - 1; p >= 0; --p)
        for (int c = 0; c < nr; ++c) {
            double s = B[p * nr + c];
            for (int q = p + 1; q < K; ++q) s -= A[p * K + q] * B[q * nr + c];
            B[p * nr + c] = s / A[p * K + p];
        }
    return ORC_OK;
}

#define ORC_OP_GRAD 0     /* first derivatives, RBF-FD (Eq. 13); dim outputs */
#define ORC_OP_LAP_POW 1  /* Delta^alpha, RBF-FD (Eq. 13); 1 output */
#define ORC_OP_GRAD_VFD 2 /* first derivatives, RBF-VFD central difference (Eqs. 14-15); dim outputs */

/* Weights of one stencil. rel: n x dim offsets x_j - x_c. w: nout x n. */
int orc_stencil_weights(int dim, int n, const double* rel, int phs_k, int poly_m, int op,
                        int alpha, double delta, double* w)
{
    if (dim < 1 || dim > 3 || n < 1 || poly_m < 0 || (phs_k % 2) != 1) return ORC_ERR_ARG;
    if (op == ORC_OP_LAP_POW && (alpha < 1 || phs_k - 2 * alpha < 1)) return ORC_ERR_ARG;
    int e[3 * 128];
    int M = orc_monomials(dim, poly_m, e);
    if (M > 128) return ORC_ERR_ARG;
    int K = n + M;
    int nout = (op == ORC_OP_LAP_POW) ? 1 : dim;
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
        double r = orc_norm(dim, rel + j * dim);
        if (r > s) s = r;
    }
    if (!(s > 0.0)) return ORC_ERR_SINGULAR;
    double* z = (double*)malloc(sizeof(double) * n * dim);
    double* A = (double*)calloc((size_t)K * K, sizeof(double));
    double* B = (double*)calloc((size_t)K * nout, sizeof(double));
    if (!z || !A || !B) { free(z); free(A); free(B); return ORC_ERR_OOM; }
    for (int j = 0; j < n * dim; ++j) z[j] = rel[j] / s;
    /* [A P; P^T 0] of Eq. 9 */
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) {
            double d[3];
            for (int a = 0; a < dim; ++a) d[a] = z[i * dim + a] - z[j * dim + a];
            A[i * K + j] = orc_phs(orc_norm(dim, d), phs_k);
        }
        for (int q = 0; q < M; ++q) {
            double p = orc_mono(dim, e + 3 * q, z + i * dim);
            A[i * K + n + q] = p;
            A[(n + q) * K + i] = p;
        }
    }
    /* right-hand sides: the operator applied to each basis function at x_c (z = 0) */
    double dz = delta / s;
    for (int o = 0; o < nout; ++o) {
        for (int j = 0; j < n; ++j) {
            const double* zj = z + j * dim;
            double r = orc_norm(dim, zj);
            double v = 0.0;
            if (op == ORC_OP_GRAD) {
                /* d/dx_o |x - z_j|^k at x = 0 */
                v = -(double)phs_k * orc_ipow(r, phs_k - 2) * zj[o];
            } else if (op == ORC_OP_LAP_POW) {
                double cf = 1.0;
                for (int i = 0; i < alpha; ++i)
                    cf *= (double)(phs_k - 2 * i) * (double)(phs_k - 2 * i + dim - 2);
                v = cf * orc_ipow(r, phs_k - 2 * alpha);
            } else {
                double pp[3] = {0, 0, 0}, pm[3] = {0, 0, 0};
                for (int a = 0; a < dim; ++a) { pp[a] = -zj[a]; pm[a] = -zj[a]; }
                pp[o] += dz;
                pm[o] -= dz;
                v = (orc_phs(orc_norm(dim, pp), phs_k) - orc_phs(orc_norm(dim, pm), phs_k)) / (2.0 * dz);
            }
            B[j * nout + o] = v;
        }
        for (int q = 0; q < M; ++q) {
            const int* eq = e + 3 * q;
            double v = 0.0;
            if (op == ORC_OP_GRAD) {
                int deg = eq[0] + eq[1] + eq[2];
                v = (deg == 1 && eq[o] == 1) ? 1.0 : 0.0;
            } else if (op == ORC_OP_LAP_POW) {
                v = orc_lap_pow_mono0(dim, eq, alpha);
            } else {
                double zp[3] = {0, 0, 0}, zm[3] = {0, 0, 0};
                zp[o] = dz;
                zm[o] = -dz;
                v = (orc_mono(dim, eq, zp) - orc_mono(dim, eq, zm)) / (2.0 * dz);
            }
            B[(n + q) * nout + o] = v;
        }
    }
    int st = orc_gepp(K, A, nout, B);
    if (st == ORC_OK) {
        int l = (op == ORC_OP_LAP_POW) ? 2 * alpha : 1;
        double sl = orc_ipow(s, l);
        for (int o = 0; o < nout; ++o)
            for (int j = 0; j < n; ++j) w[o * n + j] = B[j * nout + o] / sl;
    }
    free(z);
    free(A);
    free(B);
    return st;
}

/* Weights for every centre. idx: nc x n source ids (first n_use used when
 * stride > n_use). w: nout x nc x n_use. */
int orc_weights(int dim, int64_t nc, const double* xc, const double* xs, const double* period,
                int stride, int n_use, const int64_t* idx, int phs_k, int poly_m, int op,
                int alpha, double delta, double* w)
{
    if (n_use < 1 || n_use > stride) return ORC_ERR_ARG;
    int nout = (op == ORC_OP_LAP_POW) ? 1 : dim;
    int status = ORC_OK;
#pragma omp parallel
    {
        double* rel = (double*)malloc(sizeof(double) * n_use * dim);
        double* wl = (double*)malloc(sizeof(double) * n_use * nout);
#pragma omp for schedule(dynamic, 64)
        for (int64_t c = 0; c < nc; ++c) {
            if (!rel || !wl) continue;
            for (int j = 0; j < n_use; ++j) {
                int64_t s = idx[c * stride + j];
                for (int a = 0; a < dim; ++a)
                    rel[j * dim + a] = orc_wrap(xs[s * dim + a] - xc[c * dim + a], period[a]);
            }
            int st = orc_stencil_weights(dim, n_use, rel, phs_k, poly_m, op, alpha, delta, wl);
            if (st != ORC_OK) {
#pragma omp atomic write
                status = st;
            }
            for (int o = 0; o < nout; ++o)
                for (int j = 0; j < n_use; ++j) w[(o * nc + c) * n_use + j] = wl[o * n_use + j];
        }
        if (!rel || !wl) {
#pragma omp atomic write
            status = ORC_ERR_OOM;
        }
        free(rel);
        free(wl);
    }
    return status;
}

/* OpenMP threads of the parallel loops below: n > 0 sets the count for the
   calls that follow; returns the count in force. */
int orc_threads(int n)
{
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
}

/* ------------------------------------------------------------------ O-3 */

/* Ricker wavelet r(t) = (1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2), tau = t - t0 */
double orc_ricker(double t, double f0, double t0)
{
    const double pi = 3.14159265358979323846;
    double a = pi * f0 * (t - t0);
    a = a * a;
    return (1.0 - 2.0 * a) * exp(-a);
}

/* D f at node i: sum over the stencil in order */
static double orc_apply(int n, const int64_t* idx, const double* w, const double* f)
{
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += w[j] * f[idx[j]];
    return s;
}

/*
 * PEC walls by images: entry j of a stencil may be the mirror image of node
 * idx[j] across the walls normal to the axes of code[j] (bit a). A perfect
 * conductor flips the tangential E and the normal H under the reflection and
 * keeps the normal E and the tangential H, so the gathered value enters with
 * that sign. kind: 0 Ez (TMz, tangential to every wall), 1 Hx, 2 Hy (TMz);
 * 3 + b the 3D E_b, 6 + b the 3D H_b. code == NULL: no images (orc_apply).
 */
static int orc_img_odd(unsigned r, int kind)
{
    unsigned m;
    if (kind == 0) m = r & 3u;
    else if (kind == 1) m = r & 1u;
    else if (kind == 2) m = r & 2u;
    else if (kind < 6) m = r & (7u & ~(1u << (kind - 3)));
    else m = r & (1u << (kind - 6));
    int k = 0;
    for (; m; m >>= 1) k += (int)(m & 1u);
    return k & 1;
}

static double orc_apply_img(int n, const int64_t* idx, const uint8_t* code, const double* w, const double* f,
                            int kind)
{
    if (!code) return orc_apply(n, idx, w, f);
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
        double v = f[idx[j]];
        if (code[j] && orc_img_odd(code[j], kind)) v = -v;
        s += w[j] * v;
    }
    return s;
}

/*
 * TMz leapfrog (Eq. 19) on an H node set and an E node set. The collocated
 * method passes the same set twice (the paper's method); the staggered layout
 * passes two distinct sets.
 *   H nodes: curl stencil into the E set (hc_idx, hc_wx, hc_wy; nhc entries),
 *            hyperviscosity stencil into the H set (hv_idx, hv_w; nhv entries).
 *   E nodes: curl stencil into the H set (ec_*), HV stencil into the E set (ev_*).
 * Step n -> n+1 (global index step0 + k):
 *   Hx <- Hx - dt/mu0 (Dy Ez - gamma Dhv Hx),  Hy <- Hy + dt/mu0 (Dx Ez + gamma Dhv Hy)
 *   Ez <- Ez + dt/(eps0 eps_r) (Dx Hy' - Dy Hx' + gamma Dhv Ez)   (Ez and its HV from step n)
 *   Ez[src] += amp r(t_{n+1}); Ez[pec] = 0; probes record Ez^{n+1}.
 * energy (optional, nsteps values): Eq. 20 at t_n, H averaged over n -+ 1/2.
 */
static int orc_run_tmz_k(int64_t nh, int nhc, const int64_t* hc_idx, const double* hc_wx, const double* hc_wy,
                int nhv, const int64_t* hv_idx, const double* hv_w,
                int64_t ne, int nec, const int64_t* ec_idx, const double* ec_wx, const double* ec_wy,
                int nev, const int64_t* ev_idx, const double* ev_w,
                const double* eps_r, const uint8_t* pec,
                double dt, double eps0, double mu0, double gamma,
                double* ez, double* hx, double* hy, int64_t step0, int64_t nsteps,
                int nsrc, const int64_t* src_node, const double* src_amp, const double* src_f0,
                const double* src_t0, int nprobe, const int64_t* probe_node, double* probe_out,
                double* energy_out,
                          const uint8_t* hc_code, const uint8_t* hv_code, const uint8_t* ec_code,
                          const uint8_t* ev_code)
{
    double* hx1 = (double*)malloc(sizeof(double) * nh);
    double* hy1 = (double*)malloc(sizeof(double) * nh);
    double* ez1 = (double*)malloc(sizeof(double) * ne);
    if (!hx1 || !hy1 || !ez1) { free(hx1); free(hy1); free(ez1); return ORC_ERR_OOM; }
    const double ch = dt / mu0;
    const double eta2 = mu0 / eps0;
    for (int64_t k = 0; k < nsteps; ++k) {
        int64_t n = step0 + k;
        /* H half step: H^{n+1/2} from E^n and H^{n-1/2} */
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < nh; ++i) {
            double dyE = orc_apply_img(nhc, hc_idx + i * nhc, hc_code ? hc_code + i * nhc : 0, hc_wy + i * nhc, ez, 0);
            double dxE = orc_apply_img(nhc, hc_idx + i * nhc, hc_code ? hc_code + i * nhc : 0, hc_wx + i * nhc, ez, 0);
            double vx = orc_apply_img(nhv, hv_idx + i * nhv, hv_code ? hv_code + i * nhv : 0, hv_w + i * nhv, hx, 1);
            double vy = orc_apply_img(nhv, hv_idx + i * nhv, hv_code ? hv_code + i * nhv : 0, hv_w + i * nhv, hy, 2);
            hx1[i] = hx[i] - ch * (dyE - gamma * vx);
            hy1[i] = hy[i] + ch * (dxE + gamma * vy);
        }
        if (energy_out) {
            double u = 0.0;
            for (int64_t i = 0; i < ne; ++i) u += (eps_r ? eps_r[i] : 1.0) * ez[i] * ez[i];
            for (int64_t i = 0; i < nh; ++i) {
                double ax = 0.5 * (hx[i] + hx1[i]);
                double ay = 0.5 * (hy[i] + hy1[i]);
                u += eta2 * (ax * ax + ay * ay);
            }
            energy_out[k] = u;
        }
        /* E half step: E^{n+1} from H^{n+1/2} and E^n */
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < ne; ++i) {
            double dxH = orc_apply_img(nec, ec_idx + i * nec, ec_code ? ec_code + i * nec : 0, ec_wx + i * nec, hy1, 2);
            double dyH = orc_apply_img(nec, ec_idx + i * nec, ec_code ? ec_code + i * nec : 0, ec_wy + i * nec, hx1, 1);
            double ve = orc_apply_img(nev, ev_idx + i * nev, ev_code ? ev_code + i * nev : 0, ev_w + i * nev, ez, 0);
            double er = eps_r ? eps_r[i] : 1.0;
            ez1[i] = ez[i] + dt / (eps0 * er) * (dxH - dyH + gamma * ve);
        }
        double t1 = (double)(n + 1) * dt;
        for (int s = 0; s < nsrc; ++s) ez1[src_node[s]] += src_amp[s] * orc_ricker(t1, src_f0[s], src_t0[s]);
        if (pec)
            for (int64_t i = 0; i < ne; ++i)
                if (pec[i]) ez1[i] = 0.0;
        memcpy(ez, ez1, sizeof(double) * ne);
        memcpy(hx, hx1, sizeof(double) * nh);
        memcpy(hy, hy1, sizeof(double) * nh);
        for (int p = 0; p < nprobe; ++p) probe_out[k * nprobe + p] = ez[probe_node[p]];
    }
    free(hx1);
    free(hy1);
    free(ez1);
    return ORC_OK;
}

int orc_run_tmz(int64_t nh, int nhc, const int64_t* hc_idx, const double* hc_wx, const double* hc_wy,
                int nhv, const int64_t* hv_idx, const double* hv_w,
                int64_t ne, int nec, const int64_t* ec_idx, const double* ec_wx, const double* ec_wy,
                int nev, const int64_t* ev_idx, const double* ev_w,
                const double* eps_r, const uint8_t* pec,
                double dt, double eps0, double mu0, double gamma,
                double* ez, double* hx, double* hy, int64_t step0, int64_t nsteps,
                int nsrc, const int64_t* src_node, const double* src_amp, const double* src_f0,
                const double* src_t0, int nprobe, const int64_t* probe_node, double* probe_out,
                double* energy_out)
{
    return orc_run_tmz_k(nh, nhc, hc_idx, hc_wx, hc_wy, nhv, hv_idx, hv_w, ne, nec, ec_idx, ec_wx, ec_wy, nev,
                         ev_idx, ev_w, eps_r, pec, dt, eps0, mu0, gamma, ez, hx, hy, step0, nsteps, nsrc,
                         src_node, src_amp, src_f0, src_t0, nprobe, probe_node, probe_out, energy_out, 0, 0, 0, 0);
}

/* orc_run_tmz with image codes per stencil entry (PEC walls by images): the
 * code arrays have the shapes of the index arrays; NULL = no images there */
int orc_run_tmz_img(int64_t nh, int nhc, const int64_t* hc_idx, const double* hc_wx, const double* hc_wy,
                int nhv, const int64_t* hv_idx, const double* hv_w,
                int64_t ne, int nec, const int64_t* ec_idx, const double* ec_wx, const double* ec_wy,
                int nev, const int64_t* ev_idx, const double* ev_w,
                const double* eps_r, const uint8_t* pec,
                double dt, double eps0, double mu0, double gamma,
                double* ez, double* hx, double* hy, int64_t step0, int64_t nsteps,
                int nsrc, const int64_t* src_node, const double* src_amp, const double* src_f0,
                const double* src_t0, int nprobe, const int64_t* probe_node, double* probe_out,
                double* energy_out,
                    const uint8_t* hc_code, const uint8_t* hv_code, const uint8_t* ec_code, const uint8_t* ev_code)
{
    return orc_run_tmz_k(nh, nhc, hc_idx, hc_wx, hc_wy, nhv, hv_idx, hv_w, ne, nec, ec_idx, ec_wx, ec_wy, nev,
                         ev_idx, ev_w, eps_r, pec, dt, eps0, mu0, gamma, ez, hx, hy, step0, nsteps, nsrc,
                         src_node, src_amp, src_f0, src_t0, nprobe, probe_node, probe_out, energy_out, hc_code, hv_code, ec_code, ev_code);
}

/*
 * 3D full-vector leapfrog, collocated (Eq. 2 with the hyperviscosity terms of
 * Eqs. 17-18 on every component):
 *   H <- H + dt/mu0 (-curl E + gamma Dhv H)
 *   E <- E + dt/(eps0 eps_r) (curl H' + gamma Dhv E)
 * curl uses the weights (wx, wy, wz) on the curl stencil (nc entries), Dhv the
 * HV stencil (nv entries), both into the same set. After the E update, soft
 * sources add to Ez, then every E component tangential to a wall the node
 * sits on is zeroed (wall mask bit a = wall normal to axis a), then probes
 * record Ez.
 */
static int orc_run_3d_k(int64_t N, int nc, const int64_t* c_idx, const double* wx, const double* wy,
               const double* wz, int nv, const int64_t* v_idx, const double* wv,
               const double* eps_r, const uint8_t* wall_mask,
               double dt, double eps0, double mu0, double gamma,
               double* E /* 3 x N */, double* H /* 3 x N */, int64_t step0, int64_t nsteps,
               int nsrc, const int64_t* src_node, const double* src_amp, const double* src_f0,
               const double* src_t0, int nprobe, const int64_t* probe_node, double* probe_out,
               double* energy_out,
                         const uint8_t* c_code, const uint8_t* v_code)
{
    double* H1 = (double*)malloc(sizeof(double) * 3 * N);
    double* E1 = (double*)malloc(sizeof(double) * 3 * N);
    if (!H1 || !E1) { free(H1); free(E1); return ORC_ERR_OOM; }
    const double ch = dt / mu0;
    const double eta2 = mu0 / eps0;
    double* Ex = E; double* Ey = E + N; double* Ez = E + 2 * N;
    for (int64_t k = 0; k < nsteps; ++k) {
        int64_t n = step0 + k;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < N; ++i) {
            const int64_t* ci = c_idx + i * nc;
            const uint8_t* cc = c_code ? c_code + i * nc : 0;
            double dyEz = orc_apply_img(nc, ci, cc, wy + i * nc, Ez, 5), dzEy = orc_apply_img(nc, ci, cc, wz + i * nc, Ey, 4);
            double dzEx = orc_apply_img(nc, ci, cc, wz + i * nc, Ex, 3), dxEz = orc_apply_img(nc, ci, cc, wx + i * nc, Ez, 5);
            double dxEy = orc_apply_img(nc, ci, cc, wx + i * nc, Ey, 4), dyEx = orc_apply_img(nc, ci, cc, wy + i * nc, Ex, 3);
            double cx = dyEz - dzEy, cy = dzEx - dxEz, cz = dxEy - dyEx;
            const int64_t* vi = v_idx + i * nv;
            for (int a = 0; a < 3; ++a) {
                double vh = orc_apply_img(nv, vi, v_code ? v_code + i * nv : 0, wv + i * nv, H + a * N, 6 + a);
                double c = (a == 0) ? cx : (a == 1) ? cy : cz;
                H1[a * N + i] = H[a * N + i] + ch * (-c + gamma * vh);
            }
        }
        if (energy_out) {
            double u = 0.0;
            for (int64_t i = 0; i < N; ++i) {
                double er = eps_r ? eps_r[i] : 1.0;
                for (int a = 0; a < 3; ++a) {
                    double av = 0.5 * (H[a * N + i] + H1[a * N + i]);
                    u += er * E[a * N + i] * E[a * N + i] + eta2 * av * av;
                }
            }
            energy_out[k] = u;
        }
        double* Hx1 = H1; double* Hy1 = H1 + N; double* Hz1 = H1 + 2 * N;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < N; ++i) {
            const int64_t* ci = c_idx + i * nc;
            const uint8_t* cc = c_code ? c_code + i * nc : 0;
            double dyHz = orc_apply_img(nc, ci, cc, wy + i * nc, Hz1, 8), dzHy = orc_apply_img(nc, ci, cc, wz + i * nc, Hy1, 7);
            double dzHx = orc_apply_img(nc, ci, cc, wz + i * nc, Hx1, 6), dxHz = orc_apply_img(nc, ci, cc, wx + i * nc, Hz1, 8);
            double dxHy = orc_apply_img(nc, ci, cc, wx + i * nc, Hy1, 7), dyHx = orc_apply_img(nc, ci, cc, wy + i * nc, Hx1, 6);
            double cx = dyHz - dzHy, cy = dzHx - dxHz, cz = dxHy - dyHx;
            const int64_t* vi = v_idx + i * nv;
            double er = eps_r ? eps_r[i] : 1.0;
            for (int a = 0; a < 3; ++a) {
                double ve = orc_apply_img(nv, vi, v_code ? v_code + i * nv : 0, wv + i * nv, E + a * N, 3 + a);
                double c = (a == 0) ? cx : (a == 1) ? cy : cz;
                E1[a * N + i] = E[a * N + i] + dt / (eps0 * er) * (c + gamma * ve);
            }
        }
        double t1 = (double)(n + 1) * dt;
        for (int s = 0; s < nsrc; ++s)
            E1[2 * N + src_node[s]] += src_amp[s] * orc_ricker(t1, src_f0[s], src_t0[s]);
        if (wall_mask)
            for (int64_t i = 0; i < N; ++i) {
                unsigned m = wall_mask[i];
                if (!m) continue;
                for (int b = 0; b < 3; ++b)
                    for (int a = 0; a < 3; ++a)
                        if (((m >> a) & 1u) && a != b) E1[b * N + i] = 0.0;
            }
        memcpy(E, E1, sizeof(double) * 3 * N);
        memcpy(H, H1, sizeof(double) * 3 * N);
        for (int p = 0; p < nprobe; ++p) probe_out[k * nprobe + p] = Ez[probe_node[p]];
    }
    free(H1);
    free(E1);
    return ORC_OK;
}

int orc_run_3d(int64_t N, int nc, const int64_t* c_idx, const double* wx, const double* wy,
               const double* wz, int nv, const int64_t* v_idx, const double* wv,
               const double* eps_r, const uint8_t* wall_mask,
               double dt, double eps0, double mu0, double gamma,
               double* E /* 3 x N */, double* H /* 3 x N */, int64_t step0, int64_t nsteps,
               int nsrc, const int64_t* src_node, const double* src_amp, const double* src_f0,
               const double* src_t0, int nprobe, const int64_t* probe_node, double* probe_out,
               double* energy_out)
{
    return orc_run_3d_k(N, nc, c_idx, wx, wy, wz, nv, v_idx, wv, eps_r, wall_mask, dt, eps0, mu0, gamma, E, H, step0,
                        nsteps, nsrc, src_node, src_amp, src_f0, src_t0, nprobe, probe_node, probe_out, energy_out, 0, 0);
}

/* orc_run_3d with image codes per stencil entry (PEC walls by images) */
int orc_run_3d_img(int64_t N, int nc, const int64_t* c_idx, const double* wx, const double* wy,
               const double* wz, int nv, const int64_t* v_idx, const double* wv,
               const double* eps_r, const uint8_t* wall_mask,
               double dt, double eps0, double mu0, double gamma,
               double* E /* 3 x N */, double* H /* 3 x N */, int64_t step0, int64_t nsteps,
               int nsrc, const int64_t* src_node, const double* src_amp, const double* src_f0,
               const double* src_t0, int nprobe, const int64_t* probe_node, double* probe_out,
               double* energy_out,
                   const uint8_t* c_code, const uint8_t* v_code)
{
    return orc_run_3d_k(N, nc, c_idx, wx, wy, wz, nv, v_idx, wv, eps_r, wall_mask, dt, eps0, mu0, gamma, E, H, step0,
                        nsteps, nsrc, src_node, src_amp, src_f0, src_t0, nprobe, probe_node, probe_out, energy_out, c_code, v_code);
}

/* ------------------------------------------------------------------ O-4 */

/* Eq. 20 without the h^2 factor: sum eps_r Ez^2 + eta0^2 |(H_a + H_b)/2|^2 */
double orc_energy_tmz(int64_t ne, const double* ez, const double* eps_r, int64_t nh,
                      const double* hxa, const double* hya, const double* hxb, const double* hyb,
                      double eta0)
{
    double u = 0.0;
    for (int64_t i = 0; i < ne; ++i) u += (eps_r ? eps_r[i] : 1.0) * ez[i] * ez[i];
    for (int64_t i = 0; i < nh; ++i) {
        double ax = 0.5 * (hxa[i] + hxb[i]);
        double ay = 0.5 * (hya[i] + hyb[i]);
        u += eta0 * eta0 * (ax * ax + ay * ay);
    }
    return u;
}

/* ------------------------------------------------------------------ O-5 */

/* out[idx[i][j]] += w[i][j] * v[i]  (the transpose of the stencil operator) */
static void orc_apply_t(int64_t nrow, int n, const int64_t* idx, const double* w, const double* v,
                        double* out)
{
    for (int64_t i = 0; i < nrow; ++i)
        for (int j = 0; j < n; ++j) out[idx[i * n + j]] += w[i * n + j] * v[i];
}

/*
 * One adjoint (transposed) step of the homogeneous TMz map of orc_run_tmz
 * (no sources, no probes). In: lE = lambda_E^{n+1} (ne), lHx, lHy =
 * lambda_H^{n+1} (nh). Out (in place): lambda^n. With K = diag(dt/(eps0 eps_r))
 * and Z = diag(1 - pec):
 *   mu   = Z lE
 *   lH~  = lH + C_H^T K mu          (C_H H = Dx Hy - Dy Hx)
 *   lH   = lH~ + dt/mu0 gamma Dhv^T lH~
 *   lE   = mu + gamma Dhv_E^T (K mu) + dt/mu0 C_E^T lH~   (C_E E = (-Dy E, Dx E))
 */
int orc_adjoint_step_tmz(int64_t nh, int nhc, const int64_t* hc_idx, const double* hc_wx,
                         const double* hc_wy, int nhv, const int64_t* hv_idx, const double* hv_w,
                         int64_t ne, int nec, const int64_t* ec_idx, const double* ec_wx,
                         const double* ec_wy, int nev, const int64_t* ev_idx, const double* ev_w,
                         const double* eps_r, const uint8_t* pec, double dt, double eps0,
                         double mu0, double gamma, double* lE, double* lHx, double* lHy)
{
    const double ch = dt / mu0;
    double* mu = (double*)calloc(ne, sizeof(double));
    double* kmu = (double*)calloc(ne, sizeof(double));
    double* tx = (double*)calloc(nh, sizeof(double));
    double* ty = (double*)calloc(nh, sizeof(double));
    double* ox = (double*)calloc(nh, sizeof(double));
    double* oy = (double*)calloc(nh, sizeof(double));
    double* oe = (double*)calloc(ne, sizeof(double));
    if (!mu || !kmu || !tx || !ty || !ox || !oy || !oe) {
        free(mu); free(kmu); free(tx); free(ty); free(ox); free(oy); free(oe);
        return ORC_ERR_OOM;
    }
    for (int64_t i = 0; i < ne; ++i) {
        mu[i] = (pec && pec[i]) ? 0.0 : lE[i];
        kmu[i] = dt / (eps0 * (eps_r ? eps_r[i] : 1.0)) * mu[i];
    }
    /* lH~ = lH + C_H^T K mu: Hx gets -Dy^T, Hy gets Dx^T */
    for (int64_t i = 0; i < nh; ++i) { tx[i] = lHx[i]; ty[i] = lHy[i]; }
    {
        double* neg = (double*)malloc(sizeof(double) * ne);
        if (!neg) { free(mu); free(kmu); free(tx); free(ty); free(ox); free(oy); free(oe); return ORC_ERR_OOM; }
        for (int64_t i = 0; i < ne; ++i) neg[i] = -kmu[i];
        orc_apply_t(ne, nec, ec_idx, ec_wy, neg, tx);
        orc_apply_t(ne, nec, ec_idx, ec_wx, kmu, ty);
        free(neg);
    }
    /* lH = lH~ + ch gamma Dhv^T lH~ */
    for (int64_t i = 0; i < nh; ++i) { ox[i] = tx[i]; oy[i] = ty[i]; }
    {
        double* sx = (double*)malloc(sizeof(double) * nh);
        double* sy = (double*)malloc(sizeof(double) * nh);
        if (!sx || !sy) { free(sx); free(sy); free(mu); free(kmu); free(tx); free(ty); free(ox); free(oy); free(oe); return ORC_ERR_OOM; }
        for (int64_t i = 0; i < nh; ++i) { sx[i] = ch * gamma * tx[i]; sy[i] = ch * gamma * ty[i]; }
        orc_apply_t(nh, nhv, hv_idx, hv_w, sx, ox);
        orc_apply_t(nh, nhv, hv_idx, hv_w, sy, oy);
        /* lE = mu + gamma Dhv_E^T K mu + ch C_E^T lH~ ; C_E^T(ux,uy) = -Dy^T ux + Dx^T uy */
        for (int64_t i = 0; i < ne; ++i) oe[i] = mu[i];
        double* gk = (double*)malloc(sizeof(double) * ne);
        if (!gk) { free(sx); free(sy); free(mu); free(kmu); free(tx); free(ty); free(ox); free(oy); free(oe); return ORC_ERR_OOM; }
        for (int64_t i = 0; i < ne; ++i) gk[i] = gamma * kmu[i];
        orc_apply_t(ne, nev, ev_idx, ev_w, gk, oe);
        for (int64_t i = 0; i < nh; ++i) { sx[i] = -ch * tx[i]; sy[i] = ch * ty[i]; }
        orc_apply_t(nh, nhc, hc_idx, hc_wy, sx, oe);
        orc_apply_t(nh, nhc, hc_idx, hc_wx, sy, oe);
        free(gk);
        free(sx);
        free(sy);
    }
    memcpy(lE, oe, sizeof(double) * ne);
    memcpy(lHx, ox, sizeof(double) * nh);
    memcpy(lHy, oy, sizeof(double) * nh);
    free(mu); free(kmu); free(tx); free(ty); free(ox); free(oy); free(oe);
    return ORC_OK;
}

/*
 * Gradient of J = dt * sum_{n=1..N} sum_p (Ez_p^n)^2 with respect to eps_r
 * (per E node) and the source amplitudes, for orc_run_tmz over nsteps from
 * step 0. Stores every state (small problems only), then runs the adjoint
 * recursion backwards:
 *   lambda_E^N = dJ/dE^N,  lambda_H^N = 0;
 *   for n = N-1 .. 0: g_eps_i += mu_i * (-(E_i^{n+1} - E_i^n - b_i^{n+1}) / eps_r_i) on
 *   non-PEC nodes, g_amp_k += mu_{node_k} r_k(t_{n+1}), then lambda^n = M^T lambda^{n+1}
 *   plus dJ/dE^n for n >= 1.
 * ez, hx, hy: initial state (not modified). Returns J in *J.
 */
int orc_grad_tmz(int64_t nh, int nhc, const int64_t* hc_idx, const double* hc_wx, const double* hc_wy,
                 int nhv, const int64_t* hv_idx, const double* hv_w,
                 int64_t ne, int nec, const int64_t* ec_idx, const double* ec_wx, const double* ec_wy,
                 int nev, const int64_t* ev_idx, const double* ev_w,
                 const double* eps_r, const uint8_t* pec, double dt, double eps0, double mu0,
                 double gamma, const double* ez0, const double* hx0, const double* hy0, int64_t nsteps,
                 int nsrc, const int64_t* src_node, const double* src_amp, const double* src_f0,
                 const double* src_t0, int nprobe, const int64_t* probe_node,
                 double* J, double* g_eps, double* g_amp)
{
    size_t se = (size_t)ne, sh = (size_t)nh, S = (size_t)nsteps + 1;
    double* Es = (double*)malloc(sizeof(double) * se * S);
    double* Hxs = (double*)malloc(sizeof(double) * sh * S);
    double* Hys = (double*)malloc(sizeof(double) * sh * S);
    double* probes = (double*)malloc(sizeof(double) * (size_t)(nprobe > 0 ? nprobe : 1));
    double* lE = (double*)calloc(se, sizeof(double));
    double* lHx = (double*)calloc(sh, sizeof(double));
    double* lHy = (double*)calloc(sh, sizeof(double));
    if (!Es || !Hxs || !Hys || !probes || !lE || !lHx || !lHy) {
        free(Es); free(Hxs); free(Hys); free(probes); free(lE); free(lHx); free(lHy);
        return ORC_ERR_OOM;
    }
    memcpy(Es, ez0, sizeof(double) * se);
    memcpy(Hxs, hx0, sizeof(double) * sh);
    memcpy(Hys, hy0, sizeof(double) * sh);
    double j = 0.0;
    for (int64_t n = 0; n < nsteps; ++n) {
        memcpy(Es + (n + 1) * se, Es + n * se, sizeof(double) * se);
        memcpy(Hxs + (n + 1) * sh, Hxs + n * sh, sizeof(double) * sh);
        memcpy(Hys + (n + 1) * sh, Hys + n * sh, sizeof(double) * sh);
        int st = orc_run_tmz(nh, nhc, hc_idx, hc_wx, hc_wy, nhv, hv_idx, hv_w, ne, nec, ec_idx, ec_wx,
                             ec_wy, nev, ev_idx, ev_w, eps_r, pec, dt, eps0, mu0, gamma,
                             Es + (n + 1) * se, Hxs + (n + 1) * sh, Hys + (n + 1) * sh, n, 1, nsrc,
                             src_node, src_amp, src_f0, src_t0, nprobe, probe_node, probes, NULL);
        if (st != ORC_OK) { free(Es); free(Hxs); free(Hys); free(probes); free(lE); free(lHx); free(lHy); return st; }
        for (int p = 0; p < nprobe; ++p) j += dt * probes[p] * probes[p];
    }
    *J = j;
    for (int64_t i = 0; i < ne; ++i) g_eps[i] = 0.0;
    for (int s = 0; s < nsrc; ++s) g_amp[s] = 0.0;
    /* lambda_E^N = dJ/dE^N */
    for (int p = 0; p < nprobe; ++p) lE[probe_node[p]] += 2.0 * dt * Es[(size_t)nsteps * se + probe_node[p]];
    for (int64_t n = nsteps - 1; n >= 0; --n) {
        const double* En = Es + n * se;
        const double* E1 = Es + (n + 1) * se;
        double t1 = (double)(n + 1) * dt;
        for (int64_t i = 0; i < ne; ++i) {
            if (pec && pec[i]) continue;
            double b = 0.0;
            for (int s = 0; s < nsrc; ++s)
                if (src_node[s] == i) b += src_amp[s] * orc_ricker(t1, src_f0[s], src_t0[s]);
            double er = eps_r ? eps_r[i] : 1.0;
            g_eps[i] += lE[i] * (-(E1[i] - En[i] - b) / er);
        }
        for (int s = 0; s < nsrc; ++s) {
            if (pec && pec[src_node[s]]) continue;
            g_amp[s] += lE[src_node[s]] * orc_ricker(t1, src_f0[s], src_t0[s]);
        }
        int st = orc_adjoint_step_tmz(nh, nhc, hc_idx, hc_wx, hc_wy, nhv, hv_idx, hv_w, ne, nec, ec_idx,
                                      ec_wx, ec_wy, nev, ev_idx, ev_w, eps_r, pec, dt, eps0, mu0, gamma,
                                      lE, lHx, lHy);
        if (st != ORC_OK) { free(Es); free(Hxs); free(Hys); free(probes); free(lE); free(lHx); free(lHy); return st; }
        if (n >= 1)
            for (int p = 0; p < nprobe; ++p) lE[probe_node[p]] += 2.0 * dt * En[probe_node[p]];
    }
    free(Es); free(Hxs); free(Hys); free(probes); free(lE); free(lHx); free(lHy);
    return ORC_OK;
}

/*
 * One TMz step (Eq. 19) evaluated only at chosen nodes, for checks at sizes
 * where a full oracle step is too slow. State: ez (E set), hx, hy (H set).
 * H subset: nhs node ids (hs_ids) with their stencils; hpos[j] = position of
 * H node j in the subset or -1. E subset: nes node ids (es_ids) with their
 * stencils, whose curl entries must all lie in the H subset. Outputs the new
 * H at the H subset (hx1, hy1: nhs values) and the new Ez at the E subset
 * (ez1: nes values), without sources or PEC.
 */
int orc_tmz_sample_step(int64_t nhs, const int64_t* hs_ids, int nhc, const int64_t* hc_idx,
                        const double* hc_wx, const double* hc_wy, int nhv, const int64_t* hv_idx,
                        const double* hv_w, int64_t nes, const int64_t* es_ids, int nec,
                        const int64_t* ec_idx, const double* ec_wx, const double* ec_wy, int nev,
                        const int64_t* ev_idx, const double* ev_w, const int64_t* hpos,
                        const double* eps_r_es, double dt, double eps0, double mu0, double gamma,
                        const double* ez, const double* hx, const double* hy, double* hx1,
                        double* hy1, double* ez1)
{
    const double ch = dt / mu0;
    for (int64_t k = 0; k < nhs; ++k) {
        int64_t i = hs_ids[k];
        double dyE = orc_apply(nhc, hc_idx + k * nhc, hc_wy + k * nhc, ez);
        double dxE = orc_apply(nhc, hc_idx + k * nhc, hc_wx + k * nhc, ez);
        double vx = orc_apply(nhv, hv_idx + k * nhv, hv_w + k * nhv, hx);
        double vy = orc_apply(nhv, hv_idx + k * nhv, hv_w + k * nhv, hy);
        hx1[k] = hx[i] - ch * (dyE - gamma * vx);
        hy1[k] = hy[i] + ch * (dxE + gamma * vy);
    }
    for (int64_t k = 0; k < nes; ++k) {
        int64_t i = es_ids[k];
        double dxH = 0.0, dyH = 0.0;
        for (int j = 0; j < nec; ++j) {
            int64_t p = hpos[ec_idx[k * nec + j]];
            if (p < 0) return ORC_ERR_ARG;
            dxH += ec_wx[k * nec + j] * hy1[p];
            dyH += ec_wy[k * nec + j] * hx1[p];
        }
        double ve = orc_apply(nev, ev_idx + k * nev, ev_w + k * nev, ez);
        double er = eps_r_es ? eps_r_es[k] : 1.0;
        ez1[k] = ez[i] + dt / (eps0 * er) * (dxH - dyH + gamma * ve);
    }
    return ORC_OK;
}

/*
 * One 3D step (the collocated full-vector form of Eq. 19) evaluated only at
 * chosen nodes. E, H: 3 x N state. H subset: nhs node ids with curl and HV
 * stencils (hs_*); E subset: nes node ids with their stencils (es_*), whose
 * curl entries must lie in the H subset (hpos maps node -> subset position).
 * Outputs H' at the H subset (H1: 3 x nhs) and E' at the E subset (E1: 3 x
 * nes, tangential components zeroed per wall mask), without sources.
 */
int orc_3d_sample_step(int64_t nhs, const int64_t* hs_ids, int nc, const int64_t* hc_idx, const double* hwx,
                       const double* hwy, const double* hwz, int nv, const int64_t* hv_idx, const double* hwv,
                       int64_t nes, const int64_t* es_ids, const int64_t* ec_idx, const double* ewx,
                       const double* ewy, const double* ewz, const int64_t* ev_idx, const double* ewv,
                       const int64_t* hpos, const double* eps_r_es, const uint8_t* wall_es, int64_t N,
                       double dt, double eps0, double mu0, double gamma, const double* E, const double* H,
                       double* H1, double* E1)
{
    const double ch = dt / mu0;
    const double* Ex = E; const double* Ey = E + N; const double* Ez = E + 2 * N;
    for (int64_t k = 0; k < nhs; ++k) {
        int64_t i = hs_ids[k];
        const int64_t* ci = hc_idx + k * nc;
        double dyEz = orc_apply(nc, ci, hwy + k * nc, Ez), dzEy = orc_apply(nc, ci, hwz + k * nc, Ey);
        double dzEx = orc_apply(nc, ci, hwz + k * nc, Ex), dxEz = orc_apply(nc, ci, hwx + k * nc, Ez);
        double dxEy = orc_apply(nc, ci, hwx + k * nc, Ey), dyEx = orc_apply(nc, ci, hwy + k * nc, Ex);
        double c[3] = {dyEz - dzEy, dzEx - dxEz, dxEy - dyEx};
        for (int a = 0; a < 3; ++a) {
            double vh = orc_apply(nv, hv_idx + k * nv, hwv + k * nv, H + a * N);
            H1[a * nhs + k] = H[a * N + i] + ch * (-c[a] + gamma * vh);
        }
    }
    for (int64_t k = 0; k < nes; ++k) {
        int64_t i = es_ids[k];
        double d[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};  /* d[axis][component] of H' */
        for (int j = 0; j < nc; ++j) {
            int64_t p = hpos[ec_idx[k * nc + j]];
            if (p < 0) return ORC_ERR_ARG;
            const double w[3] = {ewx[k * nc + j], ewy[k * nc + j], ewz[k * nc + j]};
            for (int ax = 0; ax < 3; ++ax)
                for (int cmp = 0; cmp < 3; ++cmp) d[ax][cmp] += w[ax] * H1[cmp * nhs + p];
        }
        double c[3] = {d[1][2] - d[2][1], d[2][0] - d[0][2], d[0][1] - d[1][0]};
        double er = eps_r_es ? eps_r_es[k] : 1.0;
        for (int a = 0; a < 3; ++a) {
            double ve = orc_apply(nv, ev_idx + k * nv, ewv + k * nv, E + a * N);
            E1[a * nes + k] = E[a * N + i] + dt / (eps0 * er) * (c[a] + gamma * ve);
        }
        unsigned m = wall_es ? wall_es[k] : 0u;
        for (int b = 0; b < 3; ++b)
            for (int a = 0; a < 3; ++a)
                if (((m >> a) & 1u) && a != b) E1[b * nes + k] = 0.0;
    }
    return ORC_OK;
}

/*
 * FDTD (Yee) scheme for TMz on a periodic nx x ny grid of spacing h (Eq. 4,
 * Eq. 5): Ez[j][i] at (i h, j h) and time n dt; Hx[j][i] at (i h, (j + 1/2) h),
 * Hy[j][i] at ((i + 1/2) h, j h), both at time (n - 1/2) dt. Per step, with
 * ch = dt / (mu0 h) (S_c / eta0 in Eq. 5) and ce = dt / (eps0 h) (eta0 S_c):
 *   Hx[j][i] -= ch (Ez[j+1][i] - Ez[j][i])
 *   Hy[j][i] += ch (Ez[j][i+1] - Ez[j][i])
 *   Ez[j][i] += ce (Hy[j][i] - Hy[j][i-1] - Hx[j][i] + Hx[j-1][i])   (new H)
 * indices wrapping periodically. Then soft Ricker sources add to Ez at
 * t_{n+1} = (n + 1) dt and probes record Ez (cell index j nx + i).
 */
int orc_run_yee(int64_t nx, int64_t ny, double ch, double ce, double dt, double* ez, double* hx, double* hy,
                int64_t step0, int64_t nsteps, int nsrc, const int64_t* src_cell, const double* src_amp,
                const double* src_f0, const double* src_t0, int nprobe, const int64_t* probe_cell,
                double* probe_out)
{
    if (nx < 1 || ny < 1) return ORC_ERR_ARG;
    for (int64_t k = 0; k < nsteps; ++k) {
        int64_t n = step0 + k;
        for (int64_t j = 0; j < ny; ++j) {
            int64_t jp = (j + 1) % ny;
            for (int64_t i = 0; i < nx; ++i) {
                int64_t ip = (i + 1) % nx;
                double e = ez[j * nx + i];
                hx[j * nx + i] -= ch * (ez[jp * nx + i] - e);
                hy[j * nx + i] += ch * (ez[j * nx + ip] - e);
            }
        }
        for (int64_t j = 0; j < ny; ++j) {
            int64_t jm = (j + ny - 1) % ny;
            for (int64_t i = 0; i < nx; ++i) {
                int64_t im = (i + nx - 1) % nx;
                ez[j * nx + i] += ce * (hy[j * nx + i] - hy[j * nx + im] - hx[j * nx + i] + hx[jm * nx + i]);
            }
        }
        double t1 = (double)(n + 1) * dt;
        for (int s = 0; s < nsrc; ++s) ez[src_cell[s]] += src_amp[s] * orc_ricker(t1, src_f0[s], src_t0[s]);
        for (int p = 0; p < nprobe; ++p) probe_out[k * nprobe + p] = ez[probe_cell[p]];
    }
    return ORC_OK;
}
