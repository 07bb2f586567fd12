// hvsearch.cpp -- the hyperviscosity coefficient c of gamma = c (-1)^(alpha-1)
// h^(2 alpha) by multisection (Sec. 5.1: a usable c lies in an interval and is
// found by search; Sec. 6: the search is a bisection).
//
// Every round runs ncand candidates at once as the right-hand sides of one
// batched domain (each right-hand side with its own gamma, all from the same
// initial fields), checks the energy of Eq. 20 every check_every steps, and
// keeps the sub-interval between the last unstable and the first stable
// candidate; a candidate is stable when U(t)/U(0) stays <= 1 + tol (and
// finite) at every check. The candidates of a round are log-spaced with the
// upper end of the interval as the last one. Host orchestration only: the
// stepping and the energies run in the batched kernels.
#include <cmath>
#include <string>
#include <vector>

#include "internal.cuh"

namespace {

struct BatchGuard {
    mfd_batch* b = nullptr;
    ~BatchGuard() {
        if (b) mfd_batch_destroy(b);
    }
};

}  // namespace

extern "C" mfd_status mfd_hv_search(mfd_ctx* ctx, const mfd_weights* curl, const mfd_weights* hv, double dt,
                                    double eps0, double mu0, const double* eps_r, const uint8_t* pec, const double* ez,
                                    const double* hx, const double* hy, double log10_lo, double log10_hi, int ncand,
                                    int rounds, int64_t nsteps, int64_t check_every, double tol, double* c_out,
                                    double* history) {
    using mfd::fail;
    if (!ctx || !curl || !hv || !ez || !hx || !hy || !c_out) return fail(MFD_ERR_ARG, "mfd_hv_search: NULL argument");
    if (ncand != 4 && ncand != 8 && ncand != 16 && ncand != 32)
        return fail(MFD_ERR_ARG, "mfd_hv_search: ncand must be 4, 8, 16 or 32");
    if (rounds < 1 || nsteps < 1 || check_every < 1 || !(tol > 0) || !(log10_lo < log10_hi) ||
        !std::isfinite(log10_lo) || !std::isfinite(log10_hi))
        return fail(MFD_ERR_ARG, "mfd_hv_search: need rounds, nsteps, check_every >= 1, tol > 0, lo < hi");
    if (hv->op != MFD_OP_LAP_POW || hv->alpha < 1) return fail(MFD_ERR_ARG, "mfd_hv_search: hv must be Delta^alpha weights");
    const double sign = (hv->alpha % 2 == 1) ? 1.0 : -1.0;  // (-1)^(alpha - 1)
    const int R = ncand;
    mfd_sim_desc desc = {};
    desc.dim = 2;
    desc.precision = MFD_FP32;
    desc.nrhs = R;
    desc.compensated = 0;
    desc.dt = dt;
    desc.eps0 = eps0;
    desc.mu0 = mu0;
    desc.gamma = sign * std::pow(10.0, log10_hi);
    desc.h_curl = desc.e_curl = curl;
    desc.h_hv = desc.e_hv = hv;
    BatchGuard g;
    MFD_TRY(mfd_batch_create(ctx, 1, &desc, R, &g.b));
    if (eps_r || pec) MFD_TRY(mfd_batch_set_materials(g.b, 0, eps_r, pec));
    const int64_t n = curl->st->centres->n;
    std::vector<double> fe((size_t)n * R), fx((size_t)n * R), fy((size_t)n * R);
    for (int64_t i = 0; i < n; ++i)
        for (int r = 0; r < R; ++r) {
            fe[i * R + r] = ez[i];
            fx[i * R + r] = hx[i];
            fy[i * R + r] = hy[i];
        }
    double lo = log10_lo, hi = log10_hi;
    std::vector<double> lc(R), gam(R), u0(R), u(R), umax(R), uend(R);
    for (int round = 0; round < rounds; ++round) {
        for (int k = 0; k < R; ++k) {
            lc[k] = lo + (hi - lo) * (double)(k + 1) / (double)R;
            gam[k] = sign * std::pow(10.0, lc[k]);
            umax[k] = 1.0;
        }
        MFD_TRY(mfd_batch_set_gamma(g.b, 0, gam.data()));
        MFD_TRY(mfd_batch_set_field(g.b, 0, MFD_EZ, -1, fe.data()));
        MFD_TRY(mfd_batch_set_field(g.b, 0, MFD_HX, -1, fx.data()));
        MFD_TRY(mfd_batch_set_field(g.b, 0, MFD_HY, -1, fy.data()));
        MFD_TRY(mfd_batch_energy(g.b, 0, u0.data()));
        for (int k = 0; k < R; ++k)
            if (!(u0[k] > 0) || !std::isfinite(u0[k]))
                return fail(MFD_ERR_ARG, "mfd_hv_search: the initial fields carry no energy");
        for (int64_t done = 0; done < nsteps;) {
            const int64_t m = std::min(check_every, nsteps - done);
            MFD_TRY(mfd_batch_step(g.b, m));
            done += m;
            MFD_TRY(mfd_batch_energy(g.b, 0, u.data()));
            bool all_out = true;
            for (int k = 0; k < R; ++k) {
                const double r = u[k] / u0[k];
                uend[k] = r;
                if (!(r <= umax[k])) umax[k] = std::isnan(r) ? INFINITY : r;
                all_out = all_out && !(umax[k] <= 1.0 + tol);
            }
            if (all_out) break;  // every candidate has already failed
        }
        int first = -1;
        for (int k = 0; k < R && first < 0; ++k)
            if (umax[k] <= 1.0 + tol) first = k;
        if (history)
            for (int k = 0; k < R; ++k) {
                double* hrow = history + ((size_t)round * R + k) * 3;
                hrow[0] = lc[k];
                hrow[1] = umax[k];
                hrow[2] = uend[k];
            }
        if (first < 0) {
            *c_out = NAN;
            return fail(MFD_ERR_UNSTABLE, "mfd_hv_search: no stable candidate in round " + std::to_string(round) +
                                              " (the upper end of the interval must be stable)");
        }
        hi = lc[first];
        if (first > 0) lo = lc[first - 1];
    }
    *c_out = std::pow(10.0, hi);
    return MFD_OK;
}
