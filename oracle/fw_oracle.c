/*
 * FP64 reference time stepper -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the CPU-baseline leg of the bench may
 * load this library.  It shares no code with the CUDA product path.
 *
 * It integrates the stretched pressure-velocity system of the paper, Sec. 2.1:
 *
 *   grad_1 p + rho dv/dt = 0                                  (Eq. wave1)
 *   div_2 v + kappa dp/dt = 0       (kappa = 1/K = compressibility, Eq. wave2)
 *
 * with every spatial derivative stretched as
 *
 *   d/dx~ = (1/kappa_xi) d/dx + sum_nu psi_xi^nu              (Eq. relaxation4)
 *   psi^n = b psi^(n-1) + a (d/dx)^(n-1/2)                    (Eq. relaxation_psi)
 *
 * in the paper's form: one memory variable per mechanism AND per direction on
 * both the gradient (i = 1) and the divergence (i = 2) side, with per-voxel
 * coefficient arrays a, b (Eqs. relaxation_a, relaxation_b are evaluated by
 * the Python side, oracle/medium.py).  The absorbing boundary is one more
 * mechanism of the same form per direction (the C-PML of Sec. 2.1).
 *
 * Discretisation (Sec. 3.3): staggered grid, p at integer points and times,
 * v_d at half points along d and half times; first derivatives of 2M = 8th
 * order with the Taylor staggered coefficients; second-order leapfrog in time.
 * Optionally (Sec. 3.3: 2M-th order in space, fourth order in time, after Tan
 * & Huang, J. Comput. Phys. 276 (2014)) every first derivative takes the
 * time-space stencil of that method instead: with per-point coefficients
 * a_m, b (chosen by the caller from the point's r = c dt / dx, see
 * oracle/medium.py),
 *   D f = (1/dx) [ sum_m a_m (f(+m) - f(-m+1)) along d
 *                + b sum over the other axes e and s = +-1 of the two-point
 *                  difference along d of f shifted by s along e ],
 * the coefficients of a velocity point being those of its cell (the lower
 * neighbour), like its relaxation class.
 * Time index of Eq. relaxation_psi, taken literally: the memory variable
 * lives half a step away from the derivative that drives it, so the
 * derivative g computed in a half step is the midpoint input that advances
 * psi across that half step (psi_new = b psi_old + a g), and the stretched
 * derivative at the time of g uses the mean (psi_old + psi_new)/2.  This is
 * the exact one-step integral of the Debye memory kernel with a midpoint
 * input, second-order accurate in dt.  Values outside the grid are zero unless the
 * axis is periodic.  Nonlinearity: the pressure update uses dt*(K + 2 beta p)
 * with p at the old time.
 *
 * Time step `it` (0-based): v^(it+1/2) from p^it, p^(it+1) from v^(it+1/2),
 * then p[src] += gain * wave[it] and, if it % decim == 0, trace[it/decim] =
 * p[rcv].
 */
#include <stddef.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads the loops below use (1 when built without OpenMP). */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

#define ORC_MAXMECH 4

typedef struct {
    int ndim;                 /* 2 or 3 */
    int n[3];                 /* points along x (fastest), y, z; n[2] = 1 in 2D */
    int periodic[3];          /* per-axis periodic flag (used by the pin tests) */
    int nmech;                /* tissue mechanisms, 0..4 */
    double dx;                /* grid step [m] */
    const double *kdt;        /* K*dt at p points */
    const double *b2dt;       /* 2*beta*dt at p points, or NULL */
    const double *dt_rho[3];  /* dt/rho_face at v_d points */
    const double *ik1[3];     /* 1/kappa_1 at v_d points */
    const double *ik2;        /* 1/kappa_2 at p points */
    const double *a1[ORC_MAXMECH][3], *b1[ORC_MAXMECH][3];   /* at v_d points */
    const double *a2[ORC_MAXMECH][3], *b2[ORC_MAXMECH][3];   /* at p points, per d */
    const double *a1p[3], *b1p[3];   /* absorbing mechanism at v_d points, or NULL */
    const double *a2p[3], *b2p[3];   /* absorbing mechanism at p points, or NULL */
    const double *tha[4], *thb;      /* time-space stencil per cell, or NULL (Taylor weights) */
} orc_coeffs;

typedef struct {
    double *p;
    double *v[3];
    double *psi1[ORC_MAXMECH][3];
    double *psi2[ORC_MAXMECH][3];
    double *psi1p[3];         /* may be NULL where a1p[d] is NULL */
    double *psi2p[3];
} orc_state;

/* 8th-order staggered first-derivative weights (Taylor). */
static const double CM[4] = {1225.0 / 1024.0, -245.0 / 3072.0, 49.0 / 5120.0, -5.0 / 7168.0};

static size_t stride(const orc_coeffs *g, int d)
{
    return d == 0 ? 1 : (d == 1 ? (size_t)g->n[0] : (size_t)g->n[0] * g->n[1]);
}

/* Value of field f at coordinate c along axis d, for the point with linear
 * index base and coordinate c0 along d; zero outside the grid unless the
 * axis is periodic. */
static double at(const orc_coeffs *g, const double *f, size_t base, int d, int c0, int c)
{
    int n = g->n[d];
    if (c < 0 || c >= n) {
        if (!g->periodic[d]) return 0.0;
        c = ((c % n) + n) % n;
    }
    return f[base + ((ptrdiff_t)c - c0) * (ptrdiff_t)stride(g, d)];
}

/* Value of f at the point (i0, i1, i2) moved by s along axis e and by t
 * along axis d; zero outside the grid unless the axis is periodic. */
static double at2(const orc_coeffs *g, const double *f, const int *idx, int e, int s, int d, int t)
{
    int c[3] = {idx[0], idx[1], idx[2]};
    c[e] += s;
    c[d] += t;
    for (int ax = 0; ax < 3; ++ax) {
        int n = g->n[ax];
        if (c[ax] < 0 || c[ax] >= n) {
            if (!g->periodic[ax]) return 0.0;
            c[ax] = ((c[ax] % n) + n) % n;
        }
    }
    return f[((size_t)c[2] * g->n[1] + c[1]) * g->n[0] + c[0]];
}

/* Staggered derivative of f along d at the point idx: o = 0 gives the
 * forward derivative (D+, result at c+1/2 from f at integer points), o = -1
 * the backward one (D-, result at c from f at half points j+1/2 stored at j).
 * Taylor weights, or the time-space stencil when the per-cell arrays are set. */
static double stag(const orc_coeffs *g, const double *f, int i0, int i1, int i2, int d, int o)
{
    int idx[3] = {i0, i1, i2};
    int c = idx[d];
    size_t base = ((size_t)i2 * g->n[1] + i1) * g->n[0] + i0;
    double s = 0.0;
    for (int m = 1; m <= 4; ++m) {
        double w = g->thb ? g->tha[m - 1][base] : CM[m - 1];
        s += w * (at(g, f, base, d, c, c + m + o) - at(g, f, base, d, c, c - m + 1 + o));
    }
    if (g->thb) {
        double x = 0.0;
        for (int e = 0; e < g->ndim; ++e) {
            if (e == d) continue;
            for (int sg = -1; sg <= 1; sg += 2)
                x += at2(g, f, idx, e, sg, d, 1 + o) - at2(g, f, idx, e, sg, d, o);
        }
        s += g->thb[base] * x;
    }
    return s / g->dx;
}

/* Forward staggered derivative of p along d, at the v_d point c+1/2. */
static double dplus(const orc_coeffs *g, const double *p, int i0, int i1, int i2, int d)
{
    return stag(g, p, i0, i1, i2, d, 0);
}

/* Backward staggered derivative of v_d along d, at the p point c
 * (v_d[j] sits at j+1/2). */
static double dminus(const orc_coeffs *g, const double *v, int i0, int i1, int i2, int d)
{
    return stag(g, v, i0, i1, i2, d, -1);
}

/* Exposed for the derivative pin tests. */
void orc_dplus(const orc_coeffs *g, const double *p, double *out, int d)
{
    for (int i2 = 0; i2 < g->n[2]; ++i2)
        for (int i1 = 0; i1 < g->n[1]; ++i1)
            for (int i0 = 0; i0 < g->n[0]; ++i0)
                out[((size_t)i2 * g->n[1] + i1) * g->n[0] + i0] = dplus(g, p, i0, i1, i2, d);
}

void orc_dminus(const orc_coeffs *g, const double *v, double *out, int d)
{
    for (int i2 = 0; i2 < g->n[2]; ++i2)
        for (int i1 = 0; i1 < g->n[1]; ++i1)
            for (int i0 = 0; i0 < g->n[0]; ++i0)
                out[((size_t)i2 * g->n[1] + i1) * g->n[0] + i0] = dminus(g, v, i0, i1, i2, d);
}

static void velocity_half_step(const orc_coeffs *g, orc_state *s)
{
    for (int d = 0; d < g->ndim; ++d) {
#pragma omp parallel for collapse(2) schedule(static)
        for (int i2 = 0; i2 < g->n[2]; ++i2)
            for (int i1 = 0; i1 < g->n[1]; ++i1)
                for (int i0 = 0; i0 < g->n[0]; ++i0) {
                    size_t i = ((size_t)i2 * g->n[1] + i1) * g->n[0] + i0;
                    double gd = dplus(g, s->p, i0, i1, i2, d);
                    double st = g->ik1[d][i] * gd;
                    for (int nu = 0; nu < g->nmech; ++nu) {
                        double *psi = s->psi1[nu][d];
                        double old = psi[i];
                        psi[i] = g->b1[nu][d][i] * old + g->a1[nu][d][i] * gd;
                        st += 0.5 * (old + psi[i]);
                    }
                    if (g->a1p[d]) {
                        double *psi = s->psi1p[d];
                        double old = psi[i];
                        psi[i] = g->b1p[d][i] * old + g->a1p[d][i] * gd;
                        st += 0.5 * (old + psi[i]);
                    }
                    s->v[d][i] -= g->dt_rho[d][i] * st;
                }
    }
}

static void pressure_half_step(const orc_coeffs *g, orc_state *s)
{
#pragma omp parallel for collapse(2) schedule(static)
    for (int i2 = 0; i2 < g->n[2]; ++i2)
        for (int i1 = 0; i1 < g->n[1]; ++i1)
            for (int i0 = 0; i0 < g->n[0]; ++i0) {
                size_t i = ((size_t)i2 * g->n[1] + i1) * g->n[0] + i0;
                double acc = 0.0;
                for (int d = 0; d < g->ndim; ++d) {
                    double q = dminus(g, s->v[d], i0, i1, i2, d);
                    double st = g->ik2[i] * q;
                    for (int nu = 0; nu < g->nmech; ++nu) {
                        double *psi = s->psi2[nu][d];
                        double old = psi[i];
                        psi[i] = g->b2[nu][d][i] * old + g->a2[nu][d][i] * q;
                        st += 0.5 * (old + psi[i]);
                    }
                    if (g->a2p[d]) {
                        double *psi = s->psi2p[d];
                        double old = psi[i];
                        psi[i] = g->b2p[d][i] * old + g->a2p[d][i] * q;
                        st += 0.5 * (old + psi[i]);
                    }
                    acc += st;
                }
                double k = g->kdt[i];
                if (g->b2dt) k += g->b2dt[i] * s->p[i];
                s->p[i] -= k * acc;
            }
}

/* Advance n_steps from time index it0.  Sources: linear indices src_idx,
 * per-source gain and waveform row src_wave into waves[n_wave][wave_len].
 * Receivers: traces[r][trace_len], recorded every decim steps.  Returns 0. */
int orc_run(const orc_coeffs *g, orc_state *s, int n_steps, int it0,
            int n_src, const long *src_idx, const double *src_gain, const int *src_wave,
            const double *waves, int wave_len,
            int n_rcv, const long *rcv_idx, double *traces, int trace_len, int decim)
{
    for (int k = 0; k < n_steps; ++k) {
        int it = it0 + k;
        velocity_half_step(g, s);
        pressure_half_step(g, s);
        if (it < wave_len)
            for (int j = 0; j < n_src; ++j)
                s->p[src_idx[j]] += src_gain[j] * waves[(size_t)src_wave[j] * wave_len + it];
        if (n_rcv > 0 && decim > 0 && it % decim == 0 && it / decim < trace_len)
            for (int r = 0; r < n_rcv; ++r)
                traces[(size_t)r * trace_len + it / decim] = s->p[rcv_idx[r]];
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * Adjoint (transpose) of one time step, for gradients (linear system: the
 * nonlinear factor must be off, b2dt == NULL).
 *
 * Written as reverse-mode differentiation of velocity_half_step and
 * pressure_half_step above, statement by statement:
 *   pressure:  acc = sum_d [ ik2 q_d + sum_nu (old + new)/2 + absorbing ],
 *              new = b2 old + a2 q_d,  p' = p - kdt acc,  q_d = D-_d v_d;
 *   velocity:  st = ik1 g + sum_nu (old + new)/2 + absorbing,
 *              new = b1 old + a1 g,  v' = v - dt_rho st,  g = D+_d p.
 * The transpose of the staggered derivative with zero values beyond the grid
 * is minus the other staggered derivative: (D+)^T = -D-, (D-)^T = -D+ (also
 * for periodic axes).
 *
 * f: forward state BEFORE the step; vh: velocity AFTER the step's velocity
 * half step (the v of the state after the step).  l: adjoint of the state
 * after the step on entry, of the state before the step on return (receiver
 * and source terms of the step are applied by the caller first).  dc: the
 * derivatives of every a, b with respect to the per-voxel factor s on the
 * d of the tissue mechanisms.  grad_kdt and grad_s accumulate dL/d(K dt) and
 * dL/ds per voxel.  wq, wg: scratch fields (n points each).  Returns 0, -1
 * when the nonlinear factor is on, or -2 with the time-space stencil. */
typedef struct {
    const double *da1[ORC_MAXMECH][3], *db1[ORC_MAXMECH][3];   /* at v_d points */
    const double *da2[ORC_MAXMECH][3], *db2[ORC_MAXMECH][3];   /* at p points, per d */
} orc_dcoeffs;

int orc_adjoint_step(const orc_coeffs *g, const orc_state *f, double *const *vh, orc_state *l,
                     const orc_dcoeffs *dc, double *grad_kdt, double *grad_s,
                     double *const *wq, double *const *wg)
{
    if (g->b2dt) return -1;
    /* per-point time-space coefficients make (D+)^T differ from -D-: not covered */
    if (g->thb) return -2;
    /* pressure half step, pointwise: adjoints of acc, psi2, and of q_d into wq */
#pragma omp parallel for collapse(2) schedule(static)
    for (int i2 = 0; i2 < g->n[2]; ++i2)
        for (int i1 = 0; i1 < g->n[1]; ++i1)
            for (int i0 = 0; i0 < g->n[0]; ++i0) {
                size_t i = ((size_t)i2 * g->n[1] + i1) * g->n[0] + i0;
                double lam_acc = -g->kdt[i] * l->p[i];
                double acc = 0.0, gs = 0.0;
                for (int d = 0; d < g->ndim; ++d) {
                    double q = dminus(g, vh[d], i0, i1, i2, d);
                    double lq = g->ik2[i] * lam_acc;
                    acc += g->ik2[i] * q;
                    for (int nu = 0; nu < g->nmech; ++nu) {
                        double old = f->psi2[nu][d][i];
                        double nw = g->b2[nu][d][i] * old + g->a2[nu][d][i] * q;
                        acc += 0.5 * (old + nw);
                        double lnew = l->psi2[nu][d][i];
                        lq += g->a2[nu][d][i] * (lnew + 0.5 * lam_acc);
                        gs += (dc->db2[nu][d][i] * old + dc->da2[nu][d][i] * q) * (lnew + 0.5 * lam_acc);
                        l->psi2[nu][d][i] = g->b2[nu][d][i] * lnew + 0.5 * (1.0 + g->b2[nu][d][i]) * lam_acc;
                    }
                    if (g->a2p[d]) {
                        double old = f->psi2p[d][i];
                        double nw = g->b2p[d][i] * old + g->a2p[d][i] * q;
                        acc += 0.5 * (old + nw);
                        double lnew = l->psi2p[d][i];
                        lq += g->a2p[d][i] * (lnew + 0.5 * lam_acc);
                        l->psi2p[d][i] = g->b2p[d][i] * lnew + 0.5 * (1.0 + g->b2p[d][i]) * lam_acc;
                    }
                    wq[d][i] = lq;
                }
                grad_kdt[i] += -acc * l->p[i];
                grad_s[i] += gs;
            }
    /* q_d = D-_d v_d: adjoint of v_d gains (D-)^T wq = -D+ wq */
    for (int d = 0; d < g->ndim; ++d) {
#pragma omp parallel for collapse(2) schedule(static)
        for (int i2 = 0; i2 < g->n[2]; ++i2)
            for (int i1 = 0; i1 < g->n[1]; ++i1)
                for (int i0 = 0; i0 < g->n[0]; ++i0) {
                    size_t i = ((size_t)i2 * g->n[1] + i1) * g->n[0] + i0;
                    l->v[d][i] -= dplus(g, wq[d], i0, i1, i2, d);
                }
    }
    /* velocity half step, pointwise: adjoints of st, psi1, and of g into wg */
    for (int d = 0; d < g->ndim; ++d) {
#pragma omp parallel for collapse(2) schedule(static)
        for (int i2 = 0; i2 < g->n[2]; ++i2)
            for (int i1 = 0; i1 < g->n[1]; ++i1)
                for (int i0 = 0; i0 < g->n[0]; ++i0) {
                    size_t i = ((size_t)i2 * g->n[1] + i1) * g->n[0] + i0;
                    double lam_st = -g->dt_rho[d][i] * l->v[d][i];
                    double gd = dplus(g, f->p, i0, i1, i2, d);
                    double lg = g->ik1[d][i] * lam_st, gs = 0.0;
                    for (int nu = 0; nu < g->nmech; ++nu) {
                        double old = f->psi1[nu][d][i];
                        double lnew = l->psi1[nu][d][i];
                        lg += g->a1[nu][d][i] * (lnew + 0.5 * lam_st);
                        gs += (dc->db1[nu][d][i] * old + dc->da1[nu][d][i] * gd) * (lnew + 0.5 * lam_st);
                        l->psi1[nu][d][i] = g->b1[nu][d][i] * lnew + 0.5 * (1.0 + g->b1[nu][d][i]) * lam_st;
                    }
                    if (g->a1p[d]) {
                        double lnew = l->psi1p[d][i];
                        lg += g->a1p[d][i] * (lnew + 0.5 * lam_st);
                        l->psi1p[d][i] = g->b1p[d][i] * lnew + 0.5 * (1.0 + g->b1p[d][i]) * lam_st;
                    }
                    wg[d][i] = lg;
                    grad_s[i] += gs;
                }
    }
    /* g_d = D+_d p: adjoint of p gains (D+)^T wg = -D- wg */
#pragma omp parallel for collapse(2) schedule(static)
    for (int i2 = 0; i2 < g->n[2]; ++i2)
        for (int i1 = 0; i1 < g->n[1]; ++i1)
            for (int i0 = 0; i0 < g->n[0]; ++i0) {
                size_t i = ((size_t)i2 * g->n[1] + i1) * g->n[0] + i0;
                double s = 0.0;
                for (int d = 0; d < g->ndim; ++d) s += dminus(g, wg[d], i0, i1, i2, d);
                l->p[i] -= s;
            }
    return 0;
}

int orc_version(void) { return 1; }
