// Maximum likelihood estimation (Section IV-C): the Nelder-Mead simplex over
// log-parameters driving full evaluations of Eq. 2 (or Eq. 3) through the
// library's own geo_loglik.  Host code; every evaluation runs on the device.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <limits>
#include <vector>

#include "../../include/geo.h"

namespace {

constexpr double kInf = std::numeric_limits<double>::infinity();

struct Problem {
    geo_tiles* t;
    const double *x, *y, *z;
    geo_theta theta0;
    const geo_mle_opts* o;
    void* stream;
    int free_idx[3];   // which of (sigma2, beta, nu) are optimised, in that order
    int d;
    int evals = 0, not_spd = 0, error = 0;
    std::vector<double> best_u;
    double best_f = kInf;

    // theta of a point u (logs of the free parameters)
    void unpack(const std::vector<double>& u, double th[3]) const {
        th[0] = theta0.sigma2;
        th[1] = theta0.beta;
        th[2] = theta0.nu;
        for (int a = 0; a < d; ++a) th[free_idx[a]] = exp(u[(size_t)a]);
    }
    // -l at u, +inf when not positive definite; false when the budget is spent
    // or an evaluation failed otherwise (error set)
    bool eval(const std::vector<double>& u, double& f) {
        if (evals >= o->max_evals || error) return false;
        const int k = evals++;
        double th[3];
        unpack(u, th);
        geo_theta q = theta0;
        q.sigma2 = o->profile ? 1.0 : th[0];
        q.beta = th[1];
        q.nu = th[2];
        if (o->journal && o->journal_len && k < *o->journal_len) {   // replay a journaled evaluation
            const double* rec = o->journal + 4 * (size_t)k;
            if (rec[0] != q.sigma2 || rec[1] != q.beta || rec[2] != q.nu) {
                error = -6;   // the journal belongs to another run
                return false;
            }
            f = rec[3];
            if (std::isinf(f)) ++not_spd;
        } else {
            if (!device_eval(q, f)) return false;
            if (o->journal && o->journal_len && k < o->journal_cap) {
                double* rec = o->journal + 4 * (size_t)k;
                rec[0] = q.sigma2;
                rec[1] = q.beta;
                rec[2] = q.nu;
                rec[3] = f;
                *o->journal_len = k + 1;
            }
        }
        if (f < best_f) {
            best_f = f;
            best_u = u;
        }
        return true;
    }
    // -l of one evaluation on the device (+inf when not positive definite)
    bool device_eval(const geo_theta& q, double& f) {
        double out[3];
        int info = 0;
        const int rc = geo_loglik(t, x, y, z, q, out, &info, stream);
        if (rc == GEO_ERR_NOT_SPD) {
            ++not_spd;
            f = kInf;
        } else if (rc != GEO_OK) {
            error = rc;
            return false;
        } else {
            const double n = (double)t->lay.n;
            const double l = o->profile
                                 ? -0.5 * n * log(2.0 * M_PI) - 0.5 * n - 0.5 * n * log(out[2] / n) - 0.5 * out[1]
                                 : out[0];
            f = std::isfinite(l) ? -l : kInf;
        }
        return true;
    }
};

}  // namespace

extern "C" {

int geo_mle_default_opts(geo_mle_opts* o) {
    if (!o) return -1;
    memset(o, 0, sizeof(*o));
    o->max_evals = 60;
    o->profile = 0;
    o->fix_nu = 0;
    o->xtol = 1e-3;
    o->step = 0.1;
    o->lo[0] = 1e-3;
    o->hi[0] = 1e2;
    o->lo[1] = 1e-4;
    o->hi[1] = 2.0;
    o->lo[2] = 0.05;
    o->hi[2] = 3.0;
    return 0;
}

int geo_mle(geo_tiles* t, const double* d_x, const double* d_y, const double* d_z, geo_theta theta0,
            const geo_mle_opts* opts, geo_mle_result* out, void* stream) {
    if (!t) return -1;
    if (!d_x) return -2;
    if (!d_y) return -3;
    if (!d_z) return -4;
    if (!(theta0.sigma2 > 0 && theta0.beta > 0 && theta0.nu > 0 && theta0.nugget >= 0)) return -5;
    if (!opts || opts->max_evals < 1 || !(opts->xtol >= 0) || !(opts->step > 0)) return -6;
    if (opts->journal && (!opts->journal_len || opts->journal_cap < 0 || *opts->journal_len < 0 ||
                          *opts->journal_len > opts->journal_cap))
        return -6;
    for (int a = 0; a < 3; ++a)
        if (!(opts->lo[a] > 0 && opts->lo[a] <= opts->hi[a])) return -6;
    if (!out) return -7;
    Problem P;
    P.t = t;
    P.x = d_x;
    P.y = d_y;
    P.z = d_z;
    P.theta0 = theta0;
    P.o = opts;
    P.stream = stream;
    P.d = 0;
    if (!opts->profile) P.free_idx[P.d++] = 0;
    P.free_idx[P.d++] = 1;
    if (!opts->fix_nu) P.free_idx[P.d++] = 2;
    const int d = P.d;
    std::vector<double> lo((size_t)d), hi((size_t)d), u0((size_t)d);
    const double th0[3] = {theta0.sigma2, theta0.beta, theta0.nu};
    for (int a = 0; a < d; ++a) {
        lo[(size_t)a] = log(opts->lo[P.free_idx[a]]);
        hi[(size_t)a] = log(opts->hi[P.free_idx[a]]);
        u0[(size_t)a] = log(th0[P.free_idx[a]]);
    }
    auto clamp = [&](std::vector<double> u) {
        for (int a = 0; a < d; ++a) u[(size_t)a] = std::min(std::max(u[(size_t)a], lo[(size_t)a]), hi[(size_t)a]);
        return u;
    };
    // vertex i > 0: u0 + step e_(i-1)
    std::vector<std::vector<double>> V;
    std::vector<double> F;
    for (int i = 0; i <= d; ++i) {
        std::vector<double> u = u0;
        if (i > 0) u[(size_t)(i - 1)] += opts->step;
        u = clamp(u);
        double f;
        if (!P.eval(u, f)) break;
        V.push_back(u);
        F.push_back(f);
    }
    int iters = 0;
    while ((int)V.size() == d + 1) {
        // order by f, ties by current position (stable)
        std::vector<int> ord((size_t)d + 1);
        for (int i = 0; i <= d; ++i) ord[(size_t)i] = i;
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return F[(size_t)a] < F[(size_t)b]; });
        std::vector<std::vector<double>> V2;
        std::vector<double> F2;
        for (int i : ord) {
            V2.push_back(V[(size_t)i]);
            F2.push_back(F[(size_t)i]);
        }
        V.swap(V2);
        F.swap(F2);
        double size = 0.0;
        for (int i = 1; i <= d; ++i)
            for (int a = 0; a < d; ++a) size = std::max(size, fabs(V[(size_t)i][(size_t)a] - V[0][(size_t)a]));
        if (size <= opts->xtol) break;
        std::vector<double> c((size_t)d, 0.0);
        for (int i = 0; i < d; ++i)
            for (int a = 0; a < d; ++a) c[(size_t)a] += V[(size_t)i][(size_t)a];
        for (int a = 0; a < d; ++a) c[(size_t)a] /= (double)d;
        const std::vector<double> w = V[(size_t)d];
        auto along = [&](const std::vector<double>& from, const std::vector<double>& dir_to, double s) {
            // from + s (dir_to - from), clamped
            std::vector<double> u((size_t)d);
            for (int a = 0; a < d; ++a)
                u[(size_t)a] = from[(size_t)a] + s * (dir_to[(size_t)a] - from[(size_t)a]);
            return clamp(u);
        };
        const std::vector<double> r = along(c, w, -1.0);   // c + (c - w)
        double fr;
        if (!P.eval(r, fr)) break;
        if (fr < F[0]) {
            const std::vector<double> e = along(c, w, -2.0);   // c + 2 (c - w)
            double fe;
            if (!P.eval(e, fe)) break;
            if (fe < fr) {
                V[(size_t)d] = e;
                F[(size_t)d] = fe;
            } else {
                V[(size_t)d] = r;
                F[(size_t)d] = fr;
            }
            ++iters;
            continue;
        }
        if (fr < F[(size_t)d - 1]) {
            V[(size_t)d] = r;
            F[(size_t)d] = fr;
            ++iters;
            continue;
        }
        if (fr < F[(size_t)d]) {
            const std::vector<double> oc = along(c, r, 0.5);
            double fo;
            if (!P.eval(oc, fo)) break;
            if (fo <= fr) {
                V[(size_t)d] = oc;
                F[(size_t)d] = fo;
                ++iters;
                continue;
            }
        } else {
            const std::vector<double> ic = along(c, w, 0.5);
            double fi;
            if (!P.eval(ic, fi)) break;
            if (fi < F[(size_t)d]) {
                V[(size_t)d] = ic;
                F[(size_t)d] = fi;
                ++iters;
                continue;
            }
        }
        bool complete = true;   // shrink towards the best vertex
        for (int i = 1; i <= d; ++i) {
            V[(size_t)i] = along(V[0], V[(size_t)i], 0.5);
            double fv;
            if (!P.eval(V[(size_t)i], fv)) {
                V.resize((size_t)i);
                complete = false;
                break;
            }
            F[(size_t)i] = fv;
        }
        if (complete) ++iters;
    }
    if (P.error) return P.error;
    if (P.best_u.empty()) return GEO_ERR_NOT_SPD;   // no evaluation was positive definite
    double th[3];
    P.unpack(P.best_u, th);
    geo_mle_result R;
    memset(&R, 0, sizeof(R));
    R.theta = theta0;
    R.theta.sigma2 = th[0];
    R.theta.beta = th[1];
    R.theta.nu = th[2];
    R.loglik = -P.best_f;
    R.evals = P.evals;
    R.iterations = iters;
    R.not_spd = P.not_spd;
    if (opts->profile) {
        // theta1 = Z' S~^-1 Z / n at the optimum (one more evaluation, not counted)
        geo_theta q = theta0;
        q.sigma2 = 1.0;
        q.beta = th[1];
        q.nu = th[2];
        double o3[3];
        int info = 0;
        const int rc = geo_loglik(t, d_x, d_y, d_z, q, o3, &info, stream);
        if (rc != GEO_OK) return rc;
        R.theta.sigma2 = o3[2] / (double)t->lay.n;
    }
    *out = R;
    return GEO_OK;
}

}  // extern "C"
