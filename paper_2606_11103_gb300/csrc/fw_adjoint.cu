// Gradients of a receiver functional by the discrete adjoint of the time
// step (Sec. 2.1, Sec. 3.3 discretisation), with forward states recomputed
// from checkpoints.
//
// Functional: L = sum_{r,col} G[r][col] trace[r][col].  Parameters:
//  * c(x) through K dt = rho c^2 dt (pressure update and the volume-source
//    gain K dt / dx^D); dt, the absorbing profile and the relaxation sets
//    are held fixed;
//  * alpha0(x) through a per-voxel factor s(x) = alpha0(x) / alpha0_class on
//    every d of the voxel's class (kappa, alpha at the class values), taken
//    at s = 1: dL/dalpha0 = dL/ds / alpha0;
//  * maps of the absorbing layer are inherited from the nearest interior
//    cell: the gradient folds them back onto the cells they came from.
//
// The adjoint of one time step is reverse-mode differentiation of the two
// sweeps of fw_kernels.cuh, in the kernels' own variables (memory variables
// of the divergence side summed over directions, midpoint update folded into
// ceff and hb = (1 + b)/2):
//   pressure: stp = ceff2 div + sum hb2 psi2 + absorbing, psi2' = b2 psi2 + a2 div,
//             p' = p - K dt stp,  div = sum_d D-_d v_d;
//   velocity: st = ceff1 g + sum hb1 psi1 + absorbing, psi1' = b1 psi1 + a1 g,
//             v' = v - dtr st,  g = D+_d p;
// (in the absorbing layer a -> r a and ceff -> 1/kappa + r (ceff - 1/kappa),
// r the tissue ramp of the cell);
// with (D+)^T = -D- and (D-)^T = -D+ for zero values beyond the grid.
// One reverse step is five launches: receiver injection, source-gain
// gradient, pressure adjoint (pointwise, writes the adjoint of q_d), velocity
// adjoint (stencil of that, pointwise, writes the adjoint of g_d), and the
// stencil update of the pressure adjoint.  Gradients accumulate in FP64.
// The linear system only (no nonlinear factor); FP32 and FP64 media.
#include "fw_internal.h"
#include "fw_kernels.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace fwgb {
void *device_alloc(size_t bytes);
void device_free(void *p);
size_t state_image_bytes(const fw_medium *m);
}  // namespace fwgb

using namespace fwgb;

namespace {

constexpr int kDStride = 16;   // derivative table per class: dA1[4], dB1[4], dA2[4], dB2[4]

template <typename R> struct AdjArgs {
    int nx, ny, nz, px, nmech;
    long long plane, vol;
    bool ax_on[3];
    R c1, c2, c3, c4, dt;
    int wabs;          // absorbing width (0: none) and 1 / length of the tissue ramp
    R inv_lr;
    // adjoint state
    R *lp, *lv[3], *lpsi1[kMaxMech][3], *lpsi2[kMaxMech], *lpsi1p[3], *lpsi2p[3];
    // forward state before the step (f) and velocity after it (fv1)
    const R *fp, *fpsi1[kMaxMech][3], *fpsi2[kMaxMech], *fpsi2p[3];
    const R *fv1[3];
    // maps and tables
    const R *kdt, *rho;
    const uint16_t *cls;
    const R *lut, *dlut;
    const R *pdh[3], *pah[3], *pdi[3], *pai[3];   // absorbing profile at half / integer points
    // scratch: adjoints of q_d and of g_d
    R *Q[3], *Gd[3];
    double *gk, *gs;
};

template <typename R> struct Pt {
    int c[3];          // coordinate along each kernel axis
    int n[3];          // axis lengths
    long long st[3];   // strides
};

// One thread per point: x from the block's x range and thread, the other two
// kernel axes from the grid's y and z (no division of a flat index).
template <typename R>
__device__ __forceinline__ bool point(const AdjArgs<R> &A, Pt<R> &p, long long &i)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= A.nx) return false;
    p.c[0] = x;
    p.c[1] = blockIdx.y;
    p.c[2] = blockIdx.z;
    p.n[0] = A.nx; p.n[1] = A.ny; p.n[2] = A.nz;
    p.st[0] = 1; p.st[1] = A.px; p.st[2] = A.plane;
    i = (long long)blockIdx.z * A.plane + (long long)blockIdx.y * A.px + x;
    return true;
}

// forward staggered derivative at c + 1/2: sum_m c_m (f[c+m] - f[c-m+1])
template <typename R>
__device__ __forceinline__ R dplus(const AdjArgs<R> &A, const R *f, long long i, int c, int n, long long st)
{
    auto at = [&](int cc) -> R { return (cc >= 0 && cc < n) ? f[i + (long long)(cc - c) * st] : R(0); };
    return A.c1 * (at(c + 1) - at(c)) + A.c2 * (at(c + 2) - at(c - 1)) + A.c3 * (at(c + 3) - at(c - 2)) +
           A.c4 * (at(c + 4) - at(c - 3));
}

// backward staggered derivative at c of a half-point field: sum_m c_m (f[c+m-1] - f[c-m])
template <typename R>
__device__ __forceinline__ R dminus(const AdjArgs<R> &A, const R *f, long long i, int c, int n, long long st)
{
    auto at = [&](int cc) -> R { return (cc >= 0 && cc < n) ? f[i + (long long)(cc - c) * st] : R(0); };
    return A.c1 * (at(c) - at(c - 1)) + A.c2 * (at(c + 1) - at(c - 2)) + A.c3 * (at(c + 2) - at(c - 3)) +
           A.c4 * (at(c + 3) - at(c - 4));
}

// tissue-mechanism strength of the cell (the forward sweeps' ramp, same arithmetic)
template <typename R>
__device__ __forceinline__ R cell_ramp(const AdjArgs<R> &A, const Pt<R> &P)
{
    if (A.wabs <= 0) return R(1);
    const R s = fmax(fmax(layer_depth<R>(P.c[0], A.nx, A.wabs), layer_depth<R>(P.c[1], A.ny, A.wabs)),
                     layer_depth<R>(P.c[2], A.nz, A.wabs));
    return ramp_of(s, A.inv_lr);
}

template <typename R, int DIM, int NM>
__global__ void k_adj_pres(const AdjArgs<R> A)
{
    Pt<R> P;
    long long i;
    if (!point(A, P, i)) return;
    {
        const R *t = A.lut + (size_t)A.cls[i] * kLutStride;
        const R *dtb = A.dlut + (size_t)A.cls[i] * kDStride;
        R q[3] = {0, 0, 0}, div = 0;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax)
            if (DIM == 3 || ax != 1) {
                q[ax] = dminus(A, A.fv1[ax], i, P.c[ax], P.n[ax], P.st[ax]);
                div += q[ax];
            }
        const R lp = A.lp[i];
        const R lst = -A.kdt[i] * lp;
        // tissue ramp of the absorbing layer: a -> r a (the forward sweep's ce, r div)
        const R r = cell_ramp(A, P);
        const R ce = t[3] + (r - R(1)) * t[kLutDk + 1];   // the forward sweep's ceff
        R stp = div * ce;
        R ldiv = ce * lst;
        // this step's terms in the working precision; the sum over steps in FP64
        // (FP64 arithmetic is slow on this GPU: one addition per point and step)
        R gs = 0;
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            const R old = A.fpsi2[m][i];
            stp += t[kLutH2 + m] * old;
            const R ln = A.lpsi2[m][i];
            ldiv += r * t[kLutA2 + m] * ln;
            gs += (dtb[12 + m] * old + r * dtb[8 + m] * div) * (ln + R(0.5) * lst);
            A.lpsi2[m][i] = t[kLutB2 + m] * ln + t[kLutH2 + m] * lst;
        }
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            if (DIM == 2 && ax == 1) continue;
            R qv = ldiv;
            if (A.pdi[ax]) {
                const R d = A.pdi[ax][P.c[ax]];
                if (d > R(0)) {
                    R a, b;
                    pml_ab(d, A.pai[ax][P.c[ax]], t[1], A.dt, a, b);
                    const R old = A.fpsi2p[ax][i];
                    stp += R(0.5) * (R(1) + b) * old + R(0.5) * a * q[ax];
                    const R ln = A.lpsi2p[ax][i];
                    qv += a * (ln + R(0.5) * lst);
                    A.lpsi2p[ax][i] = b * ln + R(0.5) * (R(1) + b) * lst;
                }
            }
            A.Q[ax][i] = qv;
        }
        A.gk[i] += double(-stp * lp);
        A.gs[i] += double(gs);
    }
}

template <typename R, int DIM, int NM>
__global__ void k_adj_vel(const AdjArgs<R> A)
{
    Pt<R> P;
    long long i;
    if (!point(A, P, i)) return;
    {
        const R *t = A.lut + (size_t)A.cls[i] * kLutStride;
        const R *dtb = A.dlut + (size_t)A.cls[i] * kDStride;
        const R own = A.rho[i];
        const R r = cell_ramp(A, P);
        const R ce = t[2] + (r - R(1)) * t[kLutDk];
        R gs = 0;   // this step's terms; the sum over steps in FP64
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            if (DIM == 2 && ax == 1) continue;
            const int c = P.c[ax], n = P.n[ax];
            const long long st = P.st[ax];
            const R lv = A.lv[ax][i] - dplus(A, A.Q[ax], i, c, n, st);
            const R nxt = (c + 1 < n) ? A.rho[i + st] : own;
            const R dtr = R(2) * A.dt * fw_rcp(own + nxt);
            const R lst = -dtr * lv;
            const R g = dplus(A, A.fp, i, c, n, st);
            R lg = ce * lst;
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                const R old = A.fpsi1[m][ax][i];
                const R ln = A.lpsi1[m][ax][i];
                lg += r * t[kLutA1 + m] * ln;
                gs += (dtb[4 + m] * old + r * dtb[m] * g) * (ln + R(0.5) * lst);
                A.lpsi1[m][ax][i] = t[kLutB1 + m] * ln + t[kLutH1 + m] * lst;
            }
            if (A.pdh[ax]) {
                const R d = A.pdh[ax][c];
                if (d > R(0)) {
                    R a, b;
                    pml_ab(d, A.pah[ax][c], t[0], A.dt, a, b);
                    const R ln = A.lpsi1p[ax][i];
                    lg += a * (ln + R(0.5) * lst);
                    A.lpsi1p[ax][i] = b * ln + R(0.5) * (R(1) + b) * lst;
                }
            }
            A.Gd[ax][i] = lg;
            A.lv[ax][i] = lv;
        }
        A.gs[i] += double(gs);
    }
}

template <typename R, int DIM, int NM>
__global__ void k_adj_p(const AdjArgs<R> A)
{
    Pt<R> P;
    long long i;
    if (!point(A, P, i)) return;
    {
        R s = 0;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax)
            if (DIM == 3 || ax != 1) s += dminus(A, A.Gd[ax], i, P.c[ax], P.n[ax], P.st[ax]);
        A.lp[i] -= s;
    }
}

template <typename R>
__global__ void k_adj_rcv(R *lp, const long long *idx, const R *G, int n_rcv, int n_col, int col)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n_rcv; r += gridDim.x * blockDim.x)
        lp[idx[r]] += G[(size_t)r * n_col + col];
}

template <typename R>
__global__ void k_adj_src(const R *lp, const long long *idx, const R *waves, const int *wave_of, int wave_len,
                          int it, int n_src, double inv_dxd, double *gk)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_src; s += gridDim.x * blockDim.x)
        gk[idx[s]] += double(waves[(size_t)wave_of[s] * wave_len + it]) * double(lp[idx[s]]) * inv_dxd;
}

// internal gradients -> the user's grid (transpose of the layer inheritance)
template <typename R>
__global__ void k_grad_fold(const double *gk, const double *gs, const R *rho, const R *c, double dt, int nx,
                            int ny, int nz, int px, int w, double *uc, double *us)
{
    const long long n = (long long)nx * ny * nz;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x) {
        const int x = int(j % nx);
        const long long r = j / nx;
        const int y = int(r % ny), z = int(r / ny);
        auto clampw = [w](int cc, int n_) {
            if (w <= 0) return cc;
            int lo = min(w, n_ - 1), hi = max(n_ - 1 - w, 0);
            if (lo > hi) lo = hi = n_ / 2;
            return min(max(cc, lo), hi);
        };
        const int sx = clampw(x, nx), sy = ny > 1 ? clampw(y, ny) : y, sz = clampw(z, nz);
        const long long i = r * px + x;
        const long long t = ((long long)sz * ny + sy) * nx + sx;
        const double gc = gk[i] * 2.0 * double(rho[i]) * double(c[i]) * dt;
        if (gc != 0.0) atomicAdd(&uc[t], gc);
        if (gs[i] != 0.0) atomicAdd(&us[t], gs[i]);
    }
}

template <typename D>
__global__ void k_grad_out(const double *uc, const double *us, const float *a0f, const double *a0d, long long n,
                           D *gc, D *ga)
{
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x) {
        if (gc) gc[j] = D(uc[j]);
        if (ga) {
            double g = us[j];
            if (a0f || a0d) {
                const double a = a0f ? double(a0f[j]) : a0d[j];
                g = a > 0.0 ? g / a : 0.0;
            }
            ga[j] = D(g);
        }
    }
}

// the three adjoint kernels of one reverse step, instantiated per dimension
// and number of mechanisms (their loops unroll)
template <typename R, int DIM, int NM>
void launch_reverse_dn(const AdjArgs<R> &A, dim3 grid, cudaStream_t s)
{
    k_adj_pres<R, DIM, NM><<<grid, 256, 0, s>>>(A);
    k_adj_vel<R, DIM, NM><<<grid, 256, 0, s>>>(A);
    k_adj_p<R, DIM, NM><<<grid, 256, 0, s>>>(A);
}

template <typename R>
void launch_reverse(const AdjArgs<R> &A, int ndim, int nmech, dim3 grid, cudaStream_t s)
{
    if (ndim == 2) {
        switch (nmech) {
        case 1: launch_reverse_dn<R, 2, 1>(A, grid, s); break;
        case 2: launch_reverse_dn<R, 2, 2>(A, grid, s); break;
        case 3: launch_reverse_dn<R, 2, 3>(A, grid, s); break;
        default: launch_reverse_dn<R, 2, 4>(A, grid, s); break;
        }
    } else {
        switch (nmech) {
        case 1: launch_reverse_dn<R, 3, 1>(A, grid, s); break;
        case 2: launch_reverse_dn<R, 3, 2>(A, grid, s); break;
        case 3: launch_reverse_dn<R, 3, 3>(A, grid, s); break;
        default: launch_reverse_dn<R, 3, 4>(A, grid, s); break;
        }
    }
}

int nblocks(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 16); }

struct Buf {
    void *p = nullptr;
    explicit Buf(size_t b) : p(b ? device_alloc(b) : nullptr) {}
    ~Buf() { device_free(p); }
    Buf(const Buf &) = delete;
    Buf &operator=(const Buf &) = delete;
};

#define ADJ_CK(call)                                   \
    do {                                               \
        if ((call) != cudaSuccess) {                   \
            cudaGetLastError();                        \
            return FW_ERR_CUDA;                        \
        }                                              \
    } while (0)

// derivatives of a, b (Eqs. relaxation_a / relaxation_b) with respect to a
// factor s on d, at s = 1:
//   db/ds = -(d dt / kappa) b,
//   da/ds = d alpha (b - 1) / (d + kappa alpha)^2 + d / (kappa (d + kappa alpha)) db/ds
void dab(double d, double al, double ka, double dt, double &da, double &db)
{
    const double b = std::exp(-(d / ka + al) * dt);
    db = -(d * dt / ka) * b;
    da = d * al * (b - 1.0) / ((d + ka * al) * (d + ka * al)) + d / (ka * (d + ka * al)) * db;
}

template <typename R>
int gradient_impl(fw_medium *m, int n_steps, int K, const void *G, const void *alpha0, void *grad_c, void *grad_a,
                  int as_f64, cudaStream_t s)
{
    const size_t vol = m->vol, n_user = (size_t)m->NX * m->NY * m->NZ;
    const size_t SB = state_image_bytes(m);
    const int n_ck = (n_steps + K - 1) / K;
    const int seg_len = std::min(K, n_steps);
    char *slab = static_cast<char *>(m->slab);
    auto off = [slab](const void *p) { return (size_t)(static_cast<const char *>(p) - slab); };

    Buf lam(SB), ck((size_t)n_ck * SB), seg((size_t)(seg_len + 1) * SB), fin(SB);
    Buf scratch(6 * vol * sizeof(R)), gacc(2 * vol * sizeof(double)), uacc(2 * n_user * sizeof(double));
    const size_t nG = (size_t)m->n_rcv * m->n_rec;
    Buf dG(nG * sizeof(R)), dA0(alpha0 ? n_user * (as_f64 ? 8 : 4) : 0);
    Buf dlut((size_t)m->n_classes * kDStride * sizeof(R));
    if (!lam.p || !ck.p || !seg.p || !fin.p || !scratch.p || !gacc.p || !uacc.p || (nG && !dG.p) ||
        (alpha0 && !dA0.p) || !dlut.p)
        return FW_ERR_NOMEM;
    ADJ_CK(cudaMemsetAsync(lam.p, 0, SB, s));
    ADJ_CK(cudaMemsetAsync(scratch.p, 0, 6 * vol * sizeof(R), s));
    ADJ_CK(cudaMemsetAsync(gacc.p, 0, 2 * vol * sizeof(double), s));
    ADJ_CK(cudaMemsetAsync(uacc.p, 0, 2 * n_user * sizeof(double), s));
    // receiver weights in the field type
    if (nG) {
        if (as_f64 == (sizeof(R) == 8)) {
            ADJ_CK(cudaMemcpyAsync(dG.p, G, nG * sizeof(R), cudaMemcpyDefault, s));
        } else {
            std::vector<R> h(nG);
            if (as_f64) {
                std::vector<double> t(nG);
                ADJ_CK(cudaMemcpy(t.data(), G, nG * 8, cudaMemcpyDefault));
                for (size_t k = 0; k < nG; ++k) h[k] = R(t[k]);
            } else {
                std::vector<float> t(nG);
                ADJ_CK(cudaMemcpy(t.data(), G, nG * 4, cudaMemcpyDefault));
                for (size_t k = 0; k < nG; ++k) h[k] = R(t[k]);
            }
            ADJ_CK(cudaMemcpyAsync(dG.p, h.data(), nG * sizeof(R), cudaMemcpyHostToDevice, s));
            ADJ_CK(cudaStreamSynchronize(s));
        }
    }
    if (alpha0) ADJ_CK(cudaMemcpyAsync(dA0.p, alpha0, n_user * (as_f64 ? 8 : 4), cudaMemcpyDefault, s));
    {
        std::vector<R> h((size_t)m->n_classes * kDStride, R(0));
        for (int c = 0; c < m->n_classes; ++c) {
            const fw_relax_params &p = m->classes[c];
            for (int k = 0; k < p.n_mech; ++k) {
                double da, db;
                dab(p.d1[k], p.alpha1[k], p.kappa1, m->dt, da, db);
                h[(size_t)c * kDStride + k] = R(da);
                h[(size_t)c * kDStride + 4 + k] = R(db);
                dab(p.d2[k], p.alpha2[k], p.kappa2, m->dt, da, db);
                h[(size_t)c * kDStride + 8 + k] = R(da);
                h[(size_t)c * kDStride + 12 + k] = R(db);
            }
        }
        ADJ_CK(cudaMemcpyAsync(dlut.p, h.data(), h.size() * sizeof(R), cudaMemcpyHostToDevice, s));
        ADJ_CK(cudaStreamSynchronize(s));
    }

    // ---- forward run with checkpoints ----
    const long long it0 = m->step;
    for (int k = 0; k < n_ck; ++k) {
        ADJ_CK(cudaMemcpyAsync(static_cast<char *>(ck.p) + (size_t)k * SB, slab, SB, cudaMemcpyDeviceToDevice, s));
        int rc = fw_run(m, std::min(K, n_steps - k * K), s);
        if (rc) return rc;
    }
    ADJ_CK(cudaMemcpyAsync(fin.p, slab, SB, cudaMemcpyDeviceToDevice, s));

    // ---- kernel arguments (pointers into images are set per step) ----
    AdjArgs<R> A{};
    A.nx = m->NX; A.ny = m->NY; A.nz = m->NZ; A.px = m->px; A.nmech = m->nmech;
    A.plane = (long long)m->plane;
    A.vol = (long long)vol;
    const double cm[4] = {1225.0 / 1024.0, -245.0 / 3072.0, 49.0 / 5120.0, -5.0 / 7168.0};
    A.c1 = R(cm[0] / m->dx); A.c2 = R(cm[1] / m->dx); A.c3 = R(cm[2] / m->dx); A.c4 = R(cm[3] / m->dx);
    A.dt = R(m->dt);
    A.wabs = m->wabs;
    A.inv_lr = m->wabs > 0 ? R(1) / R(m->g.transition > 0 ? m->g.transition : 0.5 * m->g.pml) : R(0);
    char *L = static_cast<char *>(lam.p);
    A.lp = reinterpret_cast<R *>(L + off(m->p));
    for (int ax = 0; ax < 3; ++ax) {
        A.ax_on[ax] = m->v[ax] != nullptr;
        A.lv[ax] = m->v[ax] ? reinterpret_cast<R *>(L + off(m->v[ax])) : nullptr;
        A.lpsi1p[ax] = m->psi1p[ax] ? reinterpret_cast<R *>(L + off(m->psi1p[ax])) : nullptr;
        A.lpsi2p[ax] = m->psi2p[ax] ? reinterpret_cast<R *>(L + off(m->psi2p[ax])) : nullptr;
        for (int k = 0; k < m->nmech; ++k)
            A.lpsi1[k][ax] = m->psi1[k][ax] ? reinterpret_cast<R *>(L + off(m->psi1[k][ax])) : nullptr;
        const bool layer = m->psi1p[ax] != nullptr;
        A.pdh[ax] = layer ? static_cast<const R *>(m->prof[ax][0]) : nullptr;
        A.pah[ax] = layer ? static_cast<const R *>(m->prof[ax][1]) : nullptr;
        A.pdi[ax] = layer ? static_cast<const R *>(m->prof[ax][2]) : nullptr;
        A.pai[ax] = layer ? static_cast<const R *>(m->prof[ax][3]) : nullptr;
        A.Q[ax] = static_cast<R *>(scratch.p) + ax * vol;
        A.Gd[ax] = static_cast<R *>(scratch.p) + (3 + ax) * vol;
    }
    for (int k = 0; k < m->nmech; ++k) A.lpsi2[k] = reinterpret_cast<R *>(L + off(m->psi2[k]));
    A.kdt = static_cast<const R *>(m->kdt);
    A.rho = static_cast<const R *>(m->rho);
    A.cls = m->cls;
    A.lut = static_cast<const R *>(m->lut);
    A.dlut = static_cast<const R *>(dlut.p);
    A.gk = static_cast<double *>(gacc.p);
    A.gs = static_cast<double *>(gacc.p) + vol;
    auto image = [&](int k) { return static_cast<const char *>(seg.p) + (size_t)k * SB; };
    const dim3 pgrid((unsigned)((m->NX + 255) / 256), (unsigned)m->NY, (unsigned)m->NZ);   // one thread per point
    const double inv_dxd = 1.0 / std::pow(m->dx, m->ndim);

    // ---- reverse sweep, one checkpoint segment at a time ----
    for (int si = n_ck - 1; si >= 0; --si) {
        const int k0 = si * K, k1 = std::min(n_steps, k0 + K);
        ADJ_CK(cudaMemcpyAsync(slab, static_cast<char *>(ck.p) + (size_t)si * SB, SB, cudaMemcpyDeviceToDevice, s));
        m->step = it0 + k0;
        ADJ_CK(cudaMemcpyAsync(seg.p, slab, SB, cudaMemcpyDeviceToDevice, s));
        for (int k = k0; k < k1; ++k) {
            int rc = fw_run(m, 1, s);
            if (rc) return rc;
            ADJ_CK(cudaMemcpyAsync(static_cast<char *>(seg.p) + (size_t)(k - k0 + 1) * SB, slab, SB,
                                   cudaMemcpyDeviceToDevice, s));
        }
        for (int k = k1 - 1; k >= k0; --k) {
            const long long it = it0 + k;
            if (m->n_rcv > 0 && it % m->decim == 0 && it / m->decim < m->n_rec)
                k_adj_rcv<R><<<(m->n_rcv + 255) / 256, 256, 0, s>>>(A.lp, m->rcv_idx, static_cast<const R *>(dG.p),
                                                                   m->n_rcv, m->n_rec, (int)(it / m->decim));
            if (m->n_src > 0 && it < m->wave_len)
                k_adj_src<R><<<(m->n_src + 255) / 256, 256, 0, s>>>(A.lp, m->src_idx, static_cast<const R *>(m->waves),
                                                                   m->wave_of, m->wave_len, (int)it, m->n_src,
                                                                   inv_dxd, A.gk);
            const char *F = image(k - k0), *F1 = image(k - k0 + 1);
            A.fp = reinterpret_cast<const R *>(F + off(m->p));
            for (int ax = 0; ax < 3; ++ax) {
                A.fv1[ax] = m->v[ax] ? reinterpret_cast<const R *>(F1 + off(m->v[ax])) : nullptr;
                A.fpsi2p[ax] = m->psi2p[ax] ? reinterpret_cast<const R *>(F + off(m->psi2p[ax])) : nullptr;
                for (int q = 0; q < m->nmech; ++q)
                    A.fpsi1[q][ax] = m->psi1[q][ax] ? reinterpret_cast<const R *>(F + off(m->psi1[q][ax])) : nullptr;
            }
            for (int q = 0; q < m->nmech; ++q) A.fpsi2[q] = reinterpret_cast<const R *>(F + off(m->psi2[q]));
            launch_reverse<R>(A, m->ndim, m->nmech, pgrid, s);
        }
        ADJ_CK(cudaGetLastError());
    }
    // leave the medium at the end of the forward run
    ADJ_CK(cudaMemcpyAsync(slab, fin.p, SB, cudaMemcpyDeviceToDevice, s));
    m->step = it0 + n_steps;

    // ---- fold onto the user's grid and convert ----
    double *uc = static_cast<double *>(uacc.p), *us = uc + n_user;
    k_grad_fold<R><<<nblocks((long long)n_user), 256, 0, s>>>(A.gk, A.gs, A.rho, static_cast<const R *>(m->cdev),
                                                            m->dt, m->NX, m->NY, m->NZ, m->px, m->wabs, uc, us);
    ADJ_CK(cudaGetLastError());
    Buf out(2 * n_user * (as_f64 ? 8 : 4));
    if (!out.p) return FW_ERR_NOMEM;
    const float *a0f = alpha0 && !as_f64 ? static_cast<const float *>(dA0.p) : nullptr;
    const double *a0d = alpha0 && as_f64 ? static_cast<const double *>(dA0.p) : nullptr;
    if (as_f64) {
        double *o = static_cast<double *>(out.p);
        k_grad_out<double><<<nblocks((long long)n_user), 256, 0, s>>>(uc, us, a0f, a0d, (long long)n_user,
                                                                    grad_c ? o : nullptr, grad_a ? o + n_user : nullptr);
    } else {
        float *o = static_cast<float *>(out.p);
        k_grad_out<float><<<nblocks((long long)n_user), 256, 0, s>>>(uc, us, a0f, a0d, (long long)n_user,
                                                                   grad_c ? o : nullptr, grad_a ? o + n_user : nullptr);
    }
    ADJ_CK(cudaGetLastError());
    const size_t eb = as_f64 ? 8 : 4;
    if (grad_c) ADJ_CK(cudaMemcpyAsync(grad_c, out.p, n_user * eb, cudaMemcpyDefault, s));
    if (grad_a)
        ADJ_CK(cudaMemcpyAsync(grad_a, static_cast<char *>(out.p) + n_user * eb, n_user * eb, cudaMemcpyDefault, s));
    ADJ_CK(cudaStreamSynchronize(s));
    m->last_stream = s;
    return FW_OK;
}

}  // namespace

extern "C" int fw_gradient(fw_medium *m, int n_steps, int checkpoint_every, const void *G, const void *alpha0,
                           void *grad_c, void *grad_alpha0, int as_f64, void *stream)
{
    if (!m || n_steps < 1 || (m->n_rcv > 0 && !G)) return FW_ERR_ARG;
    if (m->sticky) return m->sticky;
    if (m->nonlinear) return FW_ERR_UNSUPPORTED;
    if (m->time_order == 4) return FW_ERR_UNSUPPORTED;   // the transpose of the per-cell time-space weights is not built
    if (m->storage != FW_STORE_F32 && m->storage != FW_STORE_F64) return FW_ERR_UNSUPPORTED;
    if (m->NY > 65535 || m->NZ > 65535) return FW_ERR_UNSUPPORTED;   // launch grid's y and z limits
    int K = checkpoint_every > 0 ? checkpoint_every : std::max(1, (int)std::lround(std::sqrt((double)n_steps)));
    K = std::min(K, n_steps);
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaStreamSynchronize(m->last_stream) != cudaSuccess) {
        cudaGetLastError();
        return FW_ERR_CUDA;
    }
    return m->storage == FW_STORE_F64 ? gradient_impl<double>(m, n_steps, K, G, alpha0, grad_c, grad_alpha0, as_f64, s)
                                      : gradient_impl<float>(m, n_steps, K, G, alpha0, grad_c, grad_alpha0, as_f64, s);
}
