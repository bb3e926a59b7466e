// Host FP64 calibration of the relaxation mechanisms (Sec. 3.1-3.2).
//
// Target: alpha(f) = alpha0 f^y (Eq. power_law_attenuation), Kramers-Kronig
// phase velocity (Eq. kk_relation), model wavenumber of Eq.
// dispersion_relations with gamma_i of Eq. gamma1, normalised complex
// objective of Sec. 3.2, adaptive Nelder-Mead over the Table 2 variables and
// a sweep over the real/imaginary weight w.
//
// Conventions (documented readings): the target is w/c(w) - i alpha(w) so
// that attenuation = -Im k_pred; y within 1e-6 of 1 uses the logarithmic
// limit of the Kramers-Kronig relation; log scale is log10; the tolerance
// bounds both the simplex spread in x and in f; the weight is selected on
// the closed-form NRMSE of -Im k_pred.
#include "fw_internal.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <numeric>
#include <thread>
#include <vector>

namespace fwgb {

namespace {
using cd = std::complex<double>;
constexpr double kPi = 3.14159265358979323846;
// valid range of the power-law exponent (abstract, Sec. 3.1)
constexpr double kYMin = 0.4, kYMax = 2.0;

double db_per_neper() { return 20.0 / std::log(10.0); }

struct Band {
    std::vector<double> f, om, alpha, inv_c;
    std::vector<cd> k;          // target wavenumber
    double range_re = 0, range_im = 0;
};

// Power-law attenuation alpha0 f^y in Np/m (Eq. power_law_attenuation) and
// the reciprocal phase velocity of its Kramers-Kronig pair (Eq. kk_relation)
// at frequency f [Hz], with 1/c(2 pi f_ref) = 1/c0; |y - 1| < 1e-6 takes the
// logarithmic limit of the relation.
void power_law_target(double alpha0, double y, double c0, double f_ref, double f, double *alpha, double *inv_c)
{
    const double a0p = alpha0 * 100.0 / db_per_neper() / std::pow(2.0 * kPi * 1e6, y);
    const double w0 = 2.0 * kPi * f_ref, om = 2.0 * kPi * f;
    *alpha = alpha0 * std::pow(f / 1e6, y) * 100.0 / db_per_neper();
    if (std::fabs(y - 1.0) < 1e-6)
        *inv_c = 1.0 / c0 - (2.0 / kPi) * a0p * std::log(om / w0);
    else
        *inv_c = 1.0 / c0 + a0p * std::tan(kPi * y / 2.0) * (std::pow(om, y - 1.0) - std::pow(w0, y - 1.0));
}

Band make_band(double alpha0, double y, const fw_fit_opts &o)
{
    Band b;
    const int n = o.n_freq;
    const double l0 = std::log10(o.f_min), l1 = std::log10(o.f_max);
    b.f.resize(n); b.om.resize(n); b.alpha.resize(n); b.inv_c.resize(n); b.k.resize(n);
    for (int j = 0; j < n; ++j) {
        double f = n > 1 ? std::pow(10.0, l0 + (l1 - l0) * j / (n - 1)) : o.f_min;
        double om = 2.0 * kPi * f;
        double al, ic;
        power_law_target(alpha0, y, o.c0, o.f_ref, f, &al, &ic);
        b.f[j] = f; b.om[j] = om; b.alpha[j] = al; b.inv_c[j] = ic;
        b.k[j] = cd(om * ic, -al);
    }
    auto re_mm = std::minmax_element(b.k.begin(), b.k.end(), [](cd a, cd c) { return a.real() < c.real(); });
    auto im_mm = std::minmax_element(b.k.begin(), b.k.end(), [](cd a, cd c) { return a.imag() < c.imag(); });
    b.range_re = re_mm.second->real() - re_mm.first->real();
    b.range_im = im_mm.second->imag() - im_mm.first->imag();
    return b;
}

// theta layout (Table 2): [kappa1, kappa2, then per mechanism
// log10 d1, log10 d2, log10 alpha1, log10 alpha2]
fw_relax_params params_from_theta(const double *th, int n)
{
    fw_relax_params p{};
    p.n_mech = n;
    p.kappa1 = th[0];
    p.kappa2 = th[1];
    for (int m = 0; m < n; ++m) {
        p.d1[m] = std::pow(10.0, th[2 + 4 * m + 0]);
        p.d2[m] = std::pow(10.0, th[2 + 4 * m + 1]);
        p.alpha1[m] = std::pow(10.0, th[2 + 4 * m + 2]);
        p.alpha2[m] = std::pow(10.0, th[2 + 4 * m + 3]);
    }
    return p;
}

// Eq. dispersion_relations / gamma1 at angular frequency om for speed c.
cd model_k(const fw_relax_params &p, double om, double c)
{
    cd g1 = 0.0, g2 = 0.0;
    const cd iw(0.0, om);
    for (int m = 0; m < p.n_mech; ++m) {
        g1 += (p.d1[m] / (p.kappa1 * p.kappa1)) / (p.d1[m] / p.kappa1 + p.alpha1[m] + iw);
        g2 += (p.d2[m] / (p.kappa2 * p.kappa2)) / (p.d2[m] / p.kappa2 + p.alpha2[m] + iw);
    }
    cd s = 1.0 / (p.kappa1 * p.kappa2) - g1 / p.kappa2 - g2 / p.kappa1 + g1 * g2;
    return (om / c) / std::sqrt(s);
}

// model_k in real arithmetic, for the objective's inner loop (the same
// quantities, without the library's guarded complex division and square
// root, whose care is not needed here: every pole has a > 0 and om > 0):
//   gamma_i = sum_m e_m / (a_m + i om) = sum_m e_m (a_m - i om) / (a_m^2 + om^2),
//   e_m = d_m / kappa_i^2, a_m = d_m / kappa_i + alpha_m;
//   s = 1/(kappa1 kappa2) - gamma1/kappa2 - gamma2/kappa1 + gamma1 gamma2;
//   k = (om/c) / sqrt(s) = (om/c) conj(sqrt(s)) / |s|, principal square root.
struct PoleSet {
    int n;
    double e1[FW_MAX_MECH], a1[FW_MAX_MECH], e2[FW_MAX_MECH], a2[FW_MAX_MECH];
    double k1, k2, inv_k1k2;
    explicit PoleSet(const fw_relax_params &p) : n(p.n_mech), k1(p.kappa1), k2(p.kappa2)
    {
        inv_k1k2 = 1.0 / (p.kappa1 * p.kappa2);
        for (int m = 0; m < n; ++m) {
            e1[m] = p.d1[m] / (p.kappa1 * p.kappa1);
            a1[m] = p.d1[m] / p.kappa1 + p.alpha1[m];
            e2[m] = p.d2[m] / (p.kappa2 * p.kappa2);
            a2[m] = p.d2[m] / p.kappa2 + p.alpha2[m];
        }
    }
    void k(double om, double c, double &kr, double &ki) const
    {
        double g1r = 0, g1i = 0, g2r = 0, g2i = 0;
        const double om2 = om * om;
        for (int m = 0; m < n; ++m) {
            const double q1 = e1[m] / (a1[m] * a1[m] + om2), q2 = e2[m] / (a2[m] * a2[m] + om2);
            g1r += q1 * a1[m];
            g1i -= q1 * om;
            g2r += q2 * a2[m];
            g2i -= q2 * om;
        }
        const double sr = inv_k1k2 - g1r / k2 - g2r / k1 + (g1r * g2r - g1i * g2i);
        const double si = -g1i / k2 - g2i / k1 + (g1r * g2i + g1i * g2r);
        const double r = std::sqrt(sr * sr + si * si);
        double qr, qi;                                   // sqrt(s), real part >= 0
        if (sr >= 0.0) {
            qr = std::sqrt(0.5 * (r + sr));
            qi = si / (2.0 * qr);
        } else {
            qi = std::copysign(std::sqrt(0.5 * (r - sr)), si);
            qr = si / (2.0 * qi);
        }
        const double f = om / (c * r);
        kr = f * qr;
        ki = -f * qi;
    }
};

struct Objective {
    const Band *b;
    double w, c0;
    int n_mech;
    double operator()(const double *th) const
    {
        const PoleSet ps(params_from_theta(th, n_mech));
        const size_t n = b->k.size();
        double acc = 0.0;
        for (size_t j = 0; j < n; ++j) {
            double kr, ki;
            ps.k(b->om[j], c0, kr, ki);
            double dr = (1.0 - w) * (b->k[j].real() - kr) / b->range_re;
            double di = w * (b->k[j].imag() - ki) / b->range_im;
            acc += dr * dr + di * di;
        }
        return acc / double(n);
    }
};

double obj_thunk(const double *x, void *ctx) { return (*static_cast<const Objective *>(ctx))(x); }

void accuracy(const fw_relax_params &p, const Band &b, double c0, double *nrmse, double *disp)
{
    double se = 0.0, sd = 0.0, amin = b.alpha[0], amax = b.alpha[0];
    for (size_t j = 0; j < b.f.size(); ++j) {
        cd kp = model_k(p, b.om[j], c0);
        double e = -kp.imag() - b.alpha[j];
        se += e * e;
        double cm = b.om[j] / kp.real(), ct = 1.0 / b.inv_c[j];
        sd += (cm - ct) * (cm - ct);
        amin = std::min(amin, b.alpha[j]);
        amax = std::max(amax, b.alpha[j]);
    }
    *nrmse = std::sqrt(se / double(b.f.size())) / (amax - amin);
    *disp = std::sqrt(sd / double(b.f.size()));
}

bool opts_ok(const fw_fit_opts &o)
{
    if (!(o.f_min > 0 && o.f_max > o.f_min) || o.n_freq < 2 || o.n_w < 1 || o.n_w > FW_MAX_W) return false;
    if (o.maxiter < 1 || !(o.f_ref > 0) || !(o.c0 > 0)) return false;
    for (int i = 0; i < o.n_w; ++i)
        if (!(o.w[i] > 0.0 && o.w[i] < 1.0)) return false;
    return true;
}

}  // namespace

int nelder_mead(int n, double *x, const double *lo, const double *hi,
                double (*f)(const double *, void *), void *ctx, int maxiter,
                double xatol, double fatol, double *fmin, int *n_iter, int *n_eval)
{
    if (n < 1 || !x || !f) return FW_ERR_ARG;
    const double rho = 1.0, chi = 1.0 + 2.0 / n, psi = 0.75 - 1.0 / (2.0 * n), sigma = 1.0 - 1.0 / n;
    auto clip = [&](double *v) {
        if (!lo) return;
        for (int j = 0; j < n; ++j) v[j] = std::min(std::max(v[j], lo[j]), hi[j]);
    };
    std::vector<double> sim((n + 1) * n), fs(n + 1);
    int evals = 0;
    auto F = [&](const double *v) { ++evals; return f(v, ctx); };
    std::vector<double> x0(x, x + n);
    clip(x0.data());
    for (int j = 0; j < n; ++j) sim[j] = x0[j];
    for (int k = 0; k < n; ++k) {
        double *v = &sim[(k + 1) * n];
        for (int j = 0; j < n; ++j) v[j] = x0[j];
        v[k] = v[k] != 0.0 ? 1.05 * v[k] : 0.00025;
    }
    if (lo) {   // a starting vertex above a bound is mirrored about it
        for (int i = 0; i <= n; ++i)
            for (int j = 0; j < n; ++j) {
                double &v = sim[i * n + j];
                if (v > hi[j]) v = 2.0 * hi[j] - v;
                v = std::min(std::max(v, lo[j]), hi[j]);
            }
    }
    for (int i = 0; i <= n; ++i) fs[i] = F(&sim[i * n]);
    std::vector<int> ord(n + 1);
    std::vector<double> tmp_s((n + 1) * n), tmp_f(n + 1);
    auto sort_simplex = [&]() {
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return fs[a] < fs[b]; });
        for (int i = 0; i <= n; ++i) {
            tmp_f[i] = fs[ord[i]];
            std::copy(&sim[ord[i] * n], &sim[ord[i] * n] + n, &tmp_s[i * n]);
        }
        sim.swap(tmp_s);
        fs.swap(tmp_f);
    };
    sort_simplex();
    std::vector<double> xbar(n), xr(n), xe(n), xc(n);
    int it = 1;
    while (it < maxiter) {
        double sx = 0.0, sf = 0.0;
        for (int i = 1; i <= n; ++i) {
            for (int j = 0; j < n; ++j) sx = std::max(sx, std::fabs(sim[i * n + j] - sim[j]));
            sf = std::max(sf, std::fabs(fs[0] - fs[i]));
        }
        if (sx <= xatol && sf <= fatol) break;
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int i = 0; i < n; ++i) s += sim[i * n + j];
            xbar[j] = s / n;
        }
        const double *xw = &sim[n * n];
        for (int j = 0; j < n; ++j) xr[j] = (1.0 + rho) * xbar[j] - rho * xw[j];
        clip(xr.data());
        double fr = F(xr.data());
        bool shrink = false;
        double *last = &sim[n * n];
        if (fr < fs[0]) {
            for (int j = 0; j < n; ++j) xe[j] = (1.0 + rho * chi) * xbar[j] - rho * chi * xw[j];
            clip(xe.data());
            double fe = F(xe.data());
            if (fe < fr) { std::copy(xe.begin(), xe.end(), last); fs[n] = fe; }
            else { std::copy(xr.begin(), xr.end(), last); fs[n] = fr; }
        } else if (fr < fs[n - 1]) {
            std::copy(xr.begin(), xr.end(), last);
            fs[n] = fr;
        } else if (fr < fs[n]) {
            for (int j = 0; j < n; ++j) xc[j] = (1.0 + psi * rho) * xbar[j] - psi * rho * xw[j];
            clip(xc.data());
            double fc = F(xc.data());
            if (fc <= fr) { std::copy(xc.begin(), xc.end(), last); fs[n] = fc; }
            else shrink = true;
        } else {
            for (int j = 0; j < n; ++j) xc[j] = (1.0 - psi) * xbar[j] + psi * xw[j];
            clip(xc.data());
            double fc = F(xc.data());
            if (fc < fs[n]) { std::copy(xc.begin(), xc.end(), last); fs[n] = fc; }
            else shrink = true;
        }
        if (shrink) {
            for (int i = 1; i <= n; ++i) {
                double *v = &sim[i * n];
                for (int j = 0; j < n; ++j) v[j] = sim[j] + sigma * (v[j] - sim[j]);
                clip(v);
                fs[i] = F(v);
            }
        }
        sort_simplex();
        ++it;
    }
    std::copy(&sim[0], &sim[0] + n, x);
    if (fmin) *fmin = fs[0];
    if (n_iter) *n_iter = it;
    if (n_eval) *n_eval = evals;
    return FW_OK;
}

void default_opts(fw_fit_opts *o)
{
    *o = fw_fit_opts{};
    o->f_min = 1e6;
    o->f_max = 20e6;
    o->n_freq = 200;
    o->n_w = 5;
    const double w[5] = {0.1, 0.3, 0.5, 0.7, 0.9};
    for (int i = 0; i < 5; ++i) o->w[i] = w[i];
    o->maxiter = 50000;
    o->xatol = 1e-25;
    o->fatol = 1e-25;
    o->f_ref = 1e6;
    o->c0 = 1540.0;
    o->n_threads = 0;
}

fw_relax_params lossless_params(int n)
{
    fw_relax_params p{};
    p.n_mech = n;
    p.kappa1 = p.kappa2 = 1.0;
    for (int m = 0; m < n; ++m) {
        p.d1[m] = p.d2[m] = 0.0;
        p.alpha1[m] = p.alpha2[m] = 1e9;
    }
    return p;
}

// One Nelder-Mead run for weight index wi.
FitJob run_weight(double alpha0, double y, int n_mech, const fw_fit_opts &o, int wi)
{
    FitJob r{};
    Band b = make_band(alpha0, y, o);
    Objective obj{&b, o.w[wi], o.c0, n_mech};
    const int n = 2 + 4 * n_mech;
    std::vector<double> th(n), lo(n), hi(n);
    th[0] = th[1] = 1.0;
    lo[0] = lo[1] = 0.98;
    hi[0] = hi[1] = 1.0;
    for (int m = 0; m < n_mech; ++m) {
        const double init[4] = {6.0, 6.0, 9.0, 9.0}, l[4] = {2.0, 2.0, 5.0, 5.0}, h[4] = {10.0, 10.0, 12.0, 12.0};
        for (int k = 0; k < 4; ++k) {
            th[2 + 4 * m + k] = init[k];
            lo[2 + 4 * m + k] = l[k];
            hi[2 + 4 * m + k] = h[k];
        }
    }
    double J = 0.0;
    int it = 0, ne = 0;
    nelder_mead(n, th.data(), lo.data(), hi.data(), obj_thunk, &obj, o.maxiter, o.xatol, o.fatol, &J, &it, &ne);
    r.p = params_from_theta(th.data(), n_mech);
    r.J = J;
    r.w = o.w[wi];
    r.n_iter = it;
    r.n_eval = ne;
    accuracy(r.p, b, o.c0, &r.nrmse, &r.disp);
    return r;
}

// Select among weight results: lowest NRMSE, then dispersion, then order.
void select_fit(const std::vector<FitJob> &res, fw_relax_params *out, fw_fit_report *rep)
{
    size_t best = 0;
    for (size_t i = 1; i < res.size(); ++i) {
        if (res[i].nrmse < res[best].nrmse ||
            (res[i].nrmse == res[best].nrmse && res[i].disp < res[best].disp))
            best = i;
    }
    *out = res[best].p;
    if (rep) {
        rep->J = res[best].J;
        rep->w = res[best].w;
        rep->nrmse = res[best].nrmse;
        rep->disp_rmse = res[best].disp;
        rep->failed = (res[best].nrmse > 0.10 || res[best].disp > 5.0) ? 1 : 0;
        rep->n_iter = res[best].n_iter;
        rep->n_eval = res[best].n_eval;
    }
}

void parallel_for(int n_jobs, int n_threads, const std::function<void(int)> &fn)
{
    if (n_threads <= 0) n_threads = (int)std::max(1u, std::thread::hardware_concurrency());
    n_threads = std::min(n_threads, n_jobs);
    if (n_threads <= 1) {
        for (int i = 0; i < n_jobs; ++i) fn(i);
        return;
    }
    std::atomic<int> next{0};
    std::vector<std::thread> pool;
    for (int t = 0; t < n_threads; ++t)
        pool.emplace_back([&]() {
            for (int i = next++; i < n_jobs; i = next++) fn(i);
        });
    for (auto &th : pool) th.join();
}

int fit_check(double alpha0, double y, int n_mech, const fw_fit_opts &o)
{
    // the valid range of the power law, y in [0.4, 2.0] (abstract, Sec. 3.1);
    // y does not enter a lossless (alpha0 = 0) calibration
    if (n_mech < 1 || n_mech > FW_MAX_MECH || !(alpha0 >= 0.0)) return FW_ERR_ARG;
    if (alpha0 > 0.0 && !(y >= kYMin && y <= kYMax)) return FW_ERR_ARG;
    if (!opts_ok(o)) return FW_ERR_ARG;
    return FW_OK;
}

}  // namespace fwgb

using namespace fwgb;

extern "C" {

void fw_fit_default_opts(fw_fit_opts *opts)
{
    if (opts) default_opts(opts);
}

int fw_fit_relaxation(double alpha0, double y, int n_mech, const fw_fit_opts *opts,
                      fw_relax_params *out, fw_fit_report *rep)
{
    fw_fit_opts o;
    if (opts) o = *opts; else default_opts(&o);
    if (!out) return FW_ERR_ARG;
    int rc = fit_check(alpha0, y, n_mech, o);
    if (rc) return rc;
    if (alpha0 == 0.0) {
        *out = lossless_params(n_mech);
        if (rep) *rep = fw_fit_report{};
        return FW_OK;
    }
    std::vector<FitJob> res(o.n_w);
    parallel_for(o.n_w, o.n_threads, [&](int i) { res[i] = run_weight(alpha0, y, n_mech, o, i); });
    select_fit(res, out, rep);
    return FW_OK;
}

int fw_fit_objective(double alpha0, double y, double w, const fw_fit_opts *opts,
                     const double *theta, int n_mech, double *J)
{
    fw_fit_opts o;
    if (opts) o = *opts; else default_opts(&o);
    if (!theta || !J || !(w > 0 && w < 1)) return FW_ERR_ARG;
    int rc = fit_check(alpha0, y, n_mech, o);
    if (rc) return rc;
    if (!(alpha0 > 0.0)) return FW_ERR_ARG;
    Band b = make_band(alpha0, y, o);
    Objective obj{&b, w, o.c0, n_mech};
    *J = obj(theta);
    return FW_OK;
}

int fw_fit_targets(double alpha0, double y, double c0, double f_ref, const double *f_hz, int n,
                   double *alpha, double *c_phase)
{
    if (!f_hz || n < 0 || (n > 0 && (!alpha || !c_phase)) || !(alpha0 >= 0.0) || !(c0 > 0.0) || !(f_ref > 0.0))
        return FW_ERR_ARG;
    if (alpha0 > 0.0 && !(y >= kYMin && y <= kYMax)) return FW_ERR_ARG;
    for (int j = 0; j < n; ++j)
        if (!(f_hz[j] > 0.0)) return FW_ERR_ARG;
    for (int j = 0; j < n; ++j) {
        double ic;
        power_law_target(alpha0, y, c0, f_ref, f_hz[j], &alpha[j], &ic);
        c_phase[j] = 1.0 / ic;
    }
    return FW_OK;
}

int fw_model_wavenumber(const fw_relax_params *p, double c, const double *f_hz, int n,
                        double *k_re, double *k_im)
{
    if (!p || !f_hz || !k_re || !k_im || n < 0 || !(c > 0) || p->n_mech < 1 || p->n_mech > FW_MAX_MECH)
        return FW_ERR_ARG;
    for (int j = 0; j < n; ++j) {
        cd k = model_k(*p, 2.0 * kPi * f_hz[j], c);
        k_re[j] = k.real();
        k_im[j] = k.imag();
    }
    return FW_OK;
}

int fw_nelder_mead(int n, double *x, const double *lo, const double *hi,
                   double (*f)(const double *, void *), void *ctx, int maxiter, double xatol,
                   double fatol, double *fmin, int *n_iter, int *n_eval)
{
    if ((lo == nullptr) != (hi == nullptr)) return FW_ERR_ARG;
    return nelder_mead(n, x, lo, hi, f, ctx, maxiter, xatol, fatol, fmin, n_iter, n_eval);
}

}  // extern "C"
