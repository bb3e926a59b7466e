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
// A reverse step is receiver injection and the source-gain gradient, then the
// pressure adjoint (pointwise; gives the adjoint of q_d), the velocity adjoint
// (a stencil of that, pointwise; gives the adjoint of g_d) and the stencil
// update of the pressure adjoint: one tiled kernel in 2D, three kernels in 3D.
// Gradients accumulate in FP64.
// The linear system only (no nonlinear factor); FP32 and FP64 media.
#include "fw_internal.h"
#include "fw_kernels.cuh"

#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

namespace fwgb {
void *device_alloc(size_t bytes);
void device_free(void *p);
size_t state_image_bytes(const fw_medium *m);
cudaError_t image_step_f32(const fw_medium *m, const StepImages &im, const int *zero, int it, cudaStream_t s);
cudaError_t image_step_f64(const fw_medium *m, const StepImages &im, const int *zero, int it, cudaStream_t s);
}  // namespace fwgb

using namespace fwgb;

namespace {

constexpr int kDStride = 16;   // derivative table per class: dA1[4], dB1[4], dA2[4], dB2[4]

// adjoint state: p, v_d, the memory variables of both sides and of the absorbing layer
template <typename R> struct AdjState {
    R *lp, *lv[3], *lpsi1[kMaxMech][3], *lpsi2[kMaxMech], *lpsi1p[3], *lpsi2p[3];
};

template <typename R> struct AdjArgs {
    int nx, ny, nz, px, nmech;
    long long plane, vol;
    bool ax_on[3];
    R c1, c2, c3, c4, dt;
    int wabs;          // absorbing width (0: none) and 1 / length of the tissue ramp
    R inv_lr;
    // adjoint state after the step (read) and before it (written; the same buffer
    // for the three-kernel form, the other buffer of a pair for the one-kernel form)
    AdjState<R> in, out;
    // forward state before the step (f) and velocity after it (fv1)
    const R *fp, *fpsi1[kMaxMech][3], *fpsi2[kMaxMech], *fpsi2p[3];
    const R *fv1[3];
    // maps and tables
    const R *kdt, *rho;
    const uint16_t *cls;
    const R *lut, *dlut;
    const R *pdh[3], *pah[3], *pdi[3], *pai[3];   // absorbing profile at half / integer points
    // scratch of the three-kernel form: adjoints of q_d and of g_d
    R *Q[3], *Gd[3];
    double *gk, *gs;
};

template <typename R> struct Pt {
    int c[3];          // coordinate along each kernel axis
    int n[3];          // axis lengths
    long long st[3];   // strides
};

template <typename R>
__device__ __forceinline__ Pt<R> make_pt(const AdjArgs<R> &A, int x, int y, int z)
{
    Pt<R> p;
    p.c[0] = x; p.c[1] = y; p.c[2] = z;
    p.n[0] = A.nx; p.n[1] = A.ny; p.n[2] = A.nz;
    p.st[0] = 1; p.st[1] = A.px; p.st[2] = A.plane;
    return p;
}

// One thread per point: x from the block's x range and thread, the other two
// kernel axes from the grid's y and z (no division of a flat index).
template <typename R>
__device__ __forceinline__ bool point(const AdjArgs<R> &A, Pt<R> &p, long long &i)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= A.nx) return false;
    p = make_pt(A, x, (int)blockIdx.y, (int)blockIdx.z);
    i = (long long)blockIdx.z * A.plane + (long long)blockIdx.y * A.px + x;
    return true;
}

// forward staggered derivative at c + 1/2: sum_m c_m (f[c+m] - f[c-m+1])
template <typename R>
__device__ __forceinline__ R dplus(const AdjArgs<R> &A, const R *f, long long i, int c, int n, long long st)
{
    auto at = [&](int cc) -> R { return (cc >= 0 && cc < n) ? __ldg(f + i + (long long)(cc - c) * st) : R(0); };
    return A.c1 * (at(c + 1) - at(c)) + A.c2 * (at(c + 2) - at(c - 1)) + A.c3 * (at(c + 3) - at(c - 2)) +
           A.c4 * (at(c + 4) - at(c - 3));
}

// backward staggered derivative at c of a half-point field: sum_m c_m (f[c+m-1] - f[c-m])
template <typename R>
__device__ __forceinline__ R dminus(const AdjArgs<R> &A, const R *f, long long i, int c, int n, long long st)
{
    auto at = [&](int cc) -> R { return (cc >= 0 && cc < n) ? __ldg(f + i + (long long)(cc - c) * st) : R(0); };
    return A.c1 * (at(c) - at(c - 1)) + A.c2 * (at(c + 1) - at(c - 2)) + A.c3 * (at(c + 2) - at(c - 3)) +
           A.c4 * (at(c + 3) - at(c - 4));
}

// the same two differences of a run of values in shared memory (f[k] at the point + k,
// zero beyond the grid already stored)
template <typename R>
__device__ __forceinline__ R dplus_s(const AdjArgs<R> &A, const R *f, int st)
{
    return A.c1 * (f[st] - f[0]) + A.c2 * (f[2 * st] - f[-st]) + A.c3 * (f[3 * st] - f[-2 * st]) +
           A.c4 * (f[4 * st] - f[-3 * st]);
}

template <typename R>
__device__ __forceinline__ R dminus_s(const AdjArgs<R> &A, const R *f, int st)
{
    return A.c1 * (f[0] - f[-st]) + A.c2 * (f[st] - f[-2 * st]) + A.c3 * (f[2 * st] - f[-3 * st]) +
           A.c4 * (f[3 * st] - f[-4 * st]);
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

// Pressure adjoint at an in-grid point i: the adjoints of q_d (Qv).  FULL also
// takes the gradient terms of the step (gs, gk) and writes the memory
// variables before the step; without FULL only the adjoint state is read
// (the halo of the one-kernel form).
template <typename R, int DIM, int NM, bool FULL>
__device__ __forceinline__ void pres_point(const AdjArgs<R> &A, const Pt<R> &P, long long i, R (&Qv)[3], R &gs,
                                           double &gk)
{
    const int cl = __ldg(A.cls + i);
    const R *t = A.lut + (size_t)cl * kLutStride;
    const R *dtb = A.dlut + (size_t)cl * kDStride;
    R q[3] = {0, 0, 0}, div = 0;
    if (FULL) {
#pragma unroll
        for (int ax = 0; ax < 3; ++ax)
            if (DIM == 3 || ax != 1) {
                q[ax] = dminus(A, A.fv1[ax], i, P.c[ax], P.n[ax], P.st[ax]);
                div += q[ax];
            }
    }
    const R lp = __ldg(A.in.lp + i);
    const R lst = -__ldg(A.kdt + i) * lp;
    // tissue ramp of the absorbing layer: a -> r a (the forward sweep's ce, r div)
    const R r = cell_ramp(A, P);
    const R ce = __ldg(t + 3) + (r - R(1)) * __ldg(t + kLutDk + 1);   // the forward sweep's ceff
    R stp = div * ce;
    R ldiv = ce * lst;
    // this step's terms in the working precision; the sum over steps in FP64
    // (FP64 arithmetic is slow on this GPU: one addition per point and step)
    gs = 0;
#pragma unroll
    for (int m = 0; m < NM; ++m) {
        const R ln = __ldg(A.in.lpsi2[m] + i);
        ldiv += r * __ldg(t + kLutA2 + m) * ln;
        if (FULL) {
            const R old = __ldg(A.fpsi2[m] + i);
            stp += __ldg(t + kLutH2 + m) * old;
            gs += (__ldg(dtb + 12 + m) * old + r * __ldg(dtb + 8 + m) * div) * (ln + R(0.5) * lst);
            A.out.lpsi2[m][i] = __ldg(t + kLutB2 + m) * ln + __ldg(t + kLutH2 + m) * lst;
        }
    }
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        if (DIM == 2 && ax == 1) continue;
        R qv = ldiv;
        if (A.pdi[ax]) {
            const R d = __ldg(A.pdi[ax] + P.c[ax]);
            if (d > R(0)) {
                R a, b;
                pml_ab(d, __ldg(A.pai[ax] + P.c[ax]), __ldg(t + 1), A.dt, a, b);
                const R ln = __ldg(A.in.lpsi2p[ax] + i);
                qv += a * (ln + R(0.5) * lst);
                if (FULL) {
                    const R old = __ldg(A.fpsi2p[ax] + i);
                    stp += R(0.5) * (R(1) + b) * old + R(0.5) * a * q[ax];
                    A.out.lpsi2p[ax][i] = b * ln + R(0.5) * (R(1) + b) * lst;
                }
            }
        }
        Qv[ax] = qv;
    }
    gk = FULL ? double(-stp * lp) : 0.0;
}

// Velocity adjoint along axis ax at an in-grid point i, given dq = D+ of the
// adjoint of q_ax there: returns the adjoint of g_ax.  FULL also adds the
// gradient terms to gs and writes v_ax and the memory variables before the
// step.
template <typename R, int NM, bool FULL, int ax>
__device__ __forceinline__ R vel_point(const AdjArgs<R> &A, const Pt<R> &P, long long i, R dq, R &gs)
{
    const int cl = __ldg(A.cls + i);
    const R *t = A.lut + (size_t)cl * kLutStride;
    const R *dtb = A.dlut + (size_t)cl * kDStride;
    const R own = __ldg(A.rho + i);
    const R r = cell_ramp(A, P);
    const R ce = __ldg(t + 2) + (r - R(1)) * __ldg(t + kLutDk);
    const int c = P.c[ax], n = P.n[ax];
    const long long st = P.st[ax];
    const R lv = __ldg(A.in.lv[ax] + i) - dq;
    const R nxt = (c + 1 < n) ? __ldg(A.rho + i + st) : own;
    const R dtr = R(2) * A.dt * fw_rcp(own + nxt);
    const R lst = -dtr * lv;
    const R g = FULL ? dplus(A, A.fp, i, c, n, st) : R(0);
    R lg = ce * lst;
#pragma unroll
    for (int m = 0; m < NM; ++m) {
        const R ln = __ldg(A.in.lpsi1[m][ax] + i);
        lg += r * __ldg(t + kLutA1 + m) * ln;
        if (FULL) {
            const R old = __ldg(A.fpsi1[m][ax] + i);
            gs += (__ldg(dtb + 4 + m) * old + r * __ldg(dtb + m) * g) * (ln + R(0.5) * lst);
            A.out.lpsi1[m][ax][i] = __ldg(t + kLutB1 + m) * ln + __ldg(t + kLutH1 + m) * lst;
        }
    }
    if (A.pdh[ax]) {
        const R d = __ldg(A.pdh[ax] + c);
        if (d > R(0)) {
            R a, b;
            pml_ab(d, __ldg(A.pah[ax] + c), __ldg(t), A.dt, a, b);
            const R ln = __ldg(A.in.lpsi1p[ax] + i);
            lg += a * (ln + R(0.5) * lst);
            if (FULL) A.out.lpsi1p[ax][i] = b * ln + R(0.5) * (R(1) + b) * lst;
        }
    }
    if (FULL) A.out.lv[ax][i] = lv;
    return lg;
}

// ---- three-kernel form (3D): adjoints of q_d and g_d through global scratch ----

template <typename R, int DIM, int NM>
__global__ void k_adj_pres(const AdjArgs<R> A)
{
    Pt<R> P;
    long long i;
    if (!point(A, P, i)) return;
    R Qv[3], gs;
    double gk;
    pres_point<R, DIM, NM, true>(A, P, i, Qv, gs, gk);
#pragma unroll
    for (int ax = 0; ax < 3; ++ax)
        if (DIM == 3 || ax != 1) A.Q[ax][i] = Qv[ax];
    A.gk[i] += gk;
    A.gs[i] += double(gs);
}

template <typename R, int DIM, int NM>
__global__ void k_adj_vel(const AdjArgs<R> A)
{
    Pt<R> P;
    long long i;
    if (!point(A, P, i)) return;
    R gs = 0;   // this step's terms; the sum over steps in FP64
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        if (DIM == 2 && ax == 1) continue;
        const R dq = dplus(A, A.Q[ax], i, P.c[ax], P.n[ax], P.st[ax]);
        A.Gd[ax][i] = ax == 0   ? vel_point<R, NM, true, 0>(A, P, i, dq, gs)
                      : ax == 1 ? vel_point<R, NM, true, 1>(A, P, i, dq, gs)
                                : vel_point<R, NM, true, 2>(A, P, i, dq, gs);
    }
    A.gs[i] += double(gs);
}

template <typename R, int DIM, int NM>
__global__ void k_adj_p(const AdjArgs<R> A)
{
    Pt<R> P;
    long long i;
    if (!point(A, P, i)) return;
    R s = 0;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax)
        if (DIM == 3 || ax != 1) s += dminus(A, A.Gd[ax], i, P.c[ax], P.n[ax], P.st[ax]);
    A.out.lp[i] = A.in.lp[i] - s;
}

// Transpose of the step's injection and recording (k_io), in one launch:
// threads [0, n_src) add the adjoint of the receiver on the source's cell
// (if any and if col >= 0) to the pressure adjoint there and take the
// source-gain gradient of step it (it < wave_len) from it; threads
// [n_src, n_src + n_rcv) add the adjoints of the other receivers (col >= 0).
template <typename R>
__global__ void k_adj_io(R *lp, const long long *src_idx, const R *waves, const int *wave_of, int wave_len, int it,
                         int n_src, const int *src_rcv, const long long *rcv_idx, const int *rcv_src, const R *G,
                         int n_rcv, int n_col, int col, double inv_dxd, double *gk)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_src) {
        const long long k = src_idx[t];
        const int r = col >= 0 ? src_rcv[t] : -1;
        R l = lp[k];
        if (r >= 0) {
            l += G[(size_t)r * n_col + col];
            lp[k] = l;
        }
        if (it < wave_len) gk[k] += double(waves[(size_t)wave_of[t] * wave_len + it]) * double(l) * inv_dxd;
    } else if (col >= 0 && t < n_src + n_rcv) {
        const int r = t - n_src;
        if (rcv_src[r] >= 0) return;     // added by the thread of the source on its cell
        lp[rcv_idx[r]] += G[(size_t)r * n_col + col];
    }
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

// ---- one-kernel form (2D): the whole reverse step per tile ----
//
// A CTA owns a TX x TZ tile of the (x, z) grid.  The adjoints of q_d and g_d
// stay in shared memory over the tile and the halo their two stencils need
// along their own axis: g_d on 4 points before and 3 after the tile (the
// backward difference of the last update), q_d on 7 before and 7 after (the
// forward difference that gives g_d there).  Each CTA recomputes its halo from
// the adjoint state after the step, which it reads from one buffer while it
// writes the state before the step to the other (a neighbour still reads the
// old values).
// tuning overrides: FWGB_ADJ_TX / FWGB_ADJ_TZ (tile), FWGB_ADJ_THREADS
#ifndef FWGB_ADJ_THREADS
#define FWGB_ADJ_THREADS 256
#endif
#ifndef FWGB_ADJ_TX
#define FWGB_ADJ_TX 32
#endif
#ifndef FWGB_ADJ_TZ
#define FWGB_ADJ_TZ 32
#endif
constexpr int kAdjThreads = FWGB_ADJ_THREADS;

template <int TX, int TZ> struct AdjTile {
    static constexpr int QXW = TX + 14, QZH = TZ + 14;   // q_x rows, q_z columns
    static constexpr int GXW = TX + 7, GZH = TZ + 7;     // g_x rows, g_z columns
    static constexpr int FPW = TX + 7, FPH = TZ + 7;     // forward p: columns x0-3 .., rows z0-3 ..
    static constexpr int n_qx = TZ * QXW, n_qz = QZH * TX, n_gx = TZ * GXW, n_gz = GZH * TX;
    static constexpr int n_fp = FPH * FPW, n_v0 = TZ * (TX + 7), n_v2 = (TZ + 7) * TX;
    static constexpr int elems = n_qx + n_qz + n_gx + n_gz + n_fp + n_v0 + n_v2;
    static constexpr int NI = TX * TZ / kAdjThreads;     // tile points per thread
    static_assert(TX * TZ % kAdjThreads == 0, "tile points split evenly over the threads");
};

// ---- one-kernel form (2D) ----
// tissue-mechanism strength of the cell (x, z) (cell_ramp of a 2D grid)
template <typename R>
__device__ __forceinline__ R ramp2(const AdjArgs<R> &A, int x, int z)
{
    const R s = fmax(layer_depth<R>(x, A.nx, A.wabs), layer_depth<R>(z, A.nz, A.wabs));
    return ramp_of(s, A.inv_lr);
}

// Pressure adjoint at an in-grid point i = (x, z) of class table t / dtb and
// tissue strength r: the adjoints of q_x and q_z (Qx, Qz; the halo needs one
// of them, ONLY = 0 or 2).  FULL: qx, qz are the forward D- differences of
// v after the step at the point; takes this step's gradient terms (gs, gk)
// and writes the memory variables before the step.  PLAIN: no absorbing
// layer within reach of the tile (r = 1, no layer memory).
template <typename R, int NM, bool FULL, bool PLAIN, int ONLY = -1>
__device__ __forceinline__ void pres2(const AdjArgs<R> &A, int x, int z, long long i, const R *t, const R *dtb, R r,
                                      R qx, R qz, R &Qx, R &Qz, R &gs, double &gk)
{
    const R div = qx + qz;
    const R lp = __ldg(A.in.lp + i);
    const R lst = -__ldg(A.kdt + i) * lp;
    const R ce = PLAIN ? __ldg(t + 3) : __ldg(t + 3) + (r - R(1)) * __ldg(t + kLutDk + 1);
    R stp = div * ce;
    R ldiv = ce * lst;
    gs = 0;
#pragma unroll
    for (int m = 0; m < NM; ++m) {
        const R ln = __ldg(A.in.lpsi2[m] + i);
        ldiv += (PLAIN ? R(1) : r) * __ldg(t + kLutA2 + m) * ln;
        if (FULL) {
            const R old = __ldg(A.fpsi2[m] + i);
            const R h = __ldg(t + kLutH2 + m);
            stp += h * old;
            gs += (__ldg(dtb + 12 + m) * old + (PLAIN ? R(1) : r) * __ldg(dtb + 8 + m) * div) * (ln + R(0.5) * lst);
            A.out.lpsi2[m][i] = __ldg(t + kLutB2 + m) * ln + h * lst;
        }
    }
    Qx = Qz = ldiv;
    if (!PLAIN) {
#pragma unroll
        for (int ax = 0; ax < 3; ax += 2) {
            if (ONLY >= 0 && ax != ONLY) continue;
            if (!A.pdi[ax]) continue;
            const int c = ax == 0 ? x : z;
            const R d = __ldg(A.pdi[ax] + c);
            if (d > R(0)) {
                R a, b;
                pml_ab(d, __ldg(A.pai[ax] + c), __ldg(t + 1), A.dt, a, b);
                const R ln = __ldg(A.in.lpsi2p[ax] + i);
                (ax == 0 ? Qx : Qz) += a * (ln + R(0.5) * lst);
                if (FULL) {
                    const R old = __ldg(A.fpsi2p[ax] + i);
                    stp += R(0.5) * (R(1) + b) * old + R(0.5) * a * (ax == 0 ? qx : qz);
                    A.out.lpsi2p[ax][i] = b * ln + R(0.5) * (R(1) + b) * lst;
                }
            }
        }
    }
    gk = FULL ? double(-stp * lp) : 0.0;
}

// Velocity adjoint along axis ax (0 or 2) at an in-grid point i, coordinate c
// of n along ax, stride st: given dq = D+ of the adjoint of q_ax there,
// returns the adjoint of g_ax.  FULL: g is the forward D+ difference of p
// before the step; adds the gradient terms to gs and writes v_ax and the
// memory variables before the step.
template <typename R, int NM, bool FULL, bool PLAIN, int ax>
__device__ __forceinline__ R vel2(const AdjArgs<R> &A, int c, int n, long long st, long long i, const R *t,
                                  const R *dtb, R r, R dq, R g, R &gs)
{
    const R own = __ldg(A.rho + i);
    const R ce = PLAIN ? __ldg(t + 2) : __ldg(t + 2) + (r - R(1)) * __ldg(t + kLutDk);
    const R lv = __ldg(A.in.lv[ax] + i) - dq;
    const R nxt = (c + 1 < n) ? __ldg(A.rho + i + st) : own;
    const R dtr = R(2) * A.dt * fw_rcp(own + nxt);
    const R lst = -dtr * lv;
    R lg = ce * lst;
#pragma unroll
    for (int m = 0; m < NM; ++m) {
        const R ln = __ldg(A.in.lpsi1[m][ax] + i);
        lg += (PLAIN ? R(1) : r) * __ldg(t + kLutA1 + m) * ln;
        if (FULL) {
            const R old = __ldg(A.fpsi1[m][ax] + i);
            gs += (__ldg(dtb + 4 + m) * old + (PLAIN ? R(1) : r) * __ldg(dtb + m) * g) * (ln + R(0.5) * lst);
            A.out.lpsi1[m][ax][i] = __ldg(t + kLutB1 + m) * ln + __ldg(t + kLutH1 + m) * lst;
        }
    }
    if (!PLAIN && A.pdh[ax]) {
        const R d = __ldg(A.pdh[ax] + c);
        if (d > R(0)) {
            R a, b;
            pml_ab(d, __ldg(A.pah[ax] + c), __ldg(t), A.dt, a, b);
            const R ln = __ldg(A.in.lpsi1p[ax] + i);
            lg += a * (ln + R(0.5) * lst);
            if (FULL) A.out.lpsi1p[ax][i] = b * ln + R(0.5) * (R(1) + b) * lst;
        }
    }
    if (FULL) A.out.lv[ax][i] = lv;
    return lg;
}

#ifndef FWGB_ADJ_PREFETCH
#define FWGB_ADJ_PREFETCH 2   // 0: none, 1: both sides at the start, 2: velocity side after the tile's q_d
#endif

// Bulk prefetch into L2 of the elements [xa, xb) of row z of a field, clamped
// to the row (rows are 128-byte aligned, so the 16-byte rounding stays inside).
template <typename R, typename T>
__device__ __forceinline__ void prefetch_row(const AdjArgs<R> &A, const T *f, int z, int xa, int xb)
{
    xa = max(xa, 0);
    xb = min(xb, A.px);
    if (!f || z < 0 || z >= A.nz || xa >= xb) return;
    const size_t b = __cvta_generic_to_global(f + (long long)z * A.plane + xa) & ~size_t(15);
    const size_t e = (__cvta_generic_to_global(f + (long long)z * A.plane + xb) + 15) & ~size_t(15);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(b), "r"((unsigned)(e - b)) : "memory");
}

// The fields one side of the reverse step reads on a tile (side 0: pressure
// adjoint, side 1: velocity adjoint), field f of that side: its pointer and
// whether it is read on the q_d halo box (else on the tile with a 4-point
// stencil halo).
template <typename R, int NM>
__device__ __forceinline__ int side_fields(int side) { return side == 0 ? 6 + 2 * NM : 5 + 4 * NM; }

template <typename R, int NM>
__device__ __forceinline__ void side_field(const AdjArgs<R> &A, int side, int f, const void *&p, int &es, bool &box)
{
    es = sizeof(R);
    box = true;
    if (side == 0) {
        if (f == 0) p = A.in.lp;
        else if (f == 1) p = A.kdt;
        else if (f == 2) { p = A.cls; es = 2; }
        else if (f < 3 + NM) p = A.in.lpsi2[f - 3];
        else {
            box = false;
            f -= 3 + NM;
            if (f == 0) p = A.fv1[0];
            else if (f == 1) p = A.fv1[2];
            else if (f == 2) { p = A.gk; es = 8; }
            else p = A.fpsi2[f - 3];
        }
    } else {
        if (f == 0) p = A.in.lv[0];
        else if (f == 1) p = A.in.lv[2];
        else if (f == 2) p = A.rho;
        else if (f < 3 + NM) p = A.in.lpsi1[f - 3][0];
        else if (f < 3 + 2 * NM) p = A.in.lpsi1[f - 3 - NM][2];
        else {
            box = false;
            f -= 3 + 2 * NM;
            if (f == 0) p = A.fp;
            else if (f == 1) { p = A.gs; es = 8; }
            else if (f < 2 + NM) p = A.fpsi1[f - 2][0];
            else p = A.fpsi1[f - 2 - NM][2];
        }
    }
}

template <typename R, int NM, int TX, int TZ>
__device__ __forceinline__ void prefetch_side(const AdjArgs<R> &A, int side, int x0, int z0)
{
    constexpr int ROWS = TZ + 14;
    const int n = side_fields<R, NM>(side) * ROWS;
    for (int j = threadIdx.x; j < n; j += kAdjThreads) {
        const int f = j / ROWS, r = j % ROWS;
        const void *p;
        int es;
        bool box;
        side_field<R, NM>(A, side, f, p, es, box);
        const int h = box ? 7 : 4;
        if (r >= TZ + 2 * h) continue;
        const int z = z0 - h + r, xa = x0 - h, xb = x0 + TX + h;
        if (es == 2) prefetch_row(A, static_cast<const uint16_t *>(p), z, xa, xb);
        else if (es == 4) prefetch_row(A, static_cast<const float *>(p), z, xa, xb);
        else prefetch_row(A, static_cast<const double *>(p), z, xa, xb);
    }
}

// The reverse step on one TX x TZ tile: the pressure adjoint on the tile and
// on the q_d halo (7 points either side along d), the velocity adjoint on the
// tile and on the g_d halo (4 before, 3 after), then the update of the
// pressure adjoint on the tile.  The forward fields whose differences the
// step takes (p before the step, v after it) are staged in shared memory
// with their halos, zero beyond the grid.
template <typename R, int NM, int TX, int TZ, bool PLAIN>
__device__ __forceinline__ void step2_tile(const AdjArgs<R> &A, unsigned char *smem, int x0, int z0)
{
    using T = AdjTile<TX, TZ>;
    R *sQx = reinterpret_cast<R *>(smem);
    R *sQz = sQx + T::n_qx;
    R *sGx = sQz + T::n_qz;
    R *sGz = sGx + T::n_gx;
    R *sFP = sGz + T::n_gz;   // p before the step: rows z0-3 .. z0+TZ+3, columns x0-3 .. x0+TX+3
    R *sV0 = sFP + T::n_fp;   // v_x after it: rows z0 .. z0+TZ-1, columns x0-4 .. x0+TX+2
    R *sV2 = sV0 + T::n_v0;   // v_z after it: rows z0-4 .. z0+TZ+2, columns x0 .. x0+TX-1
    const int tid = threadIdx.x;
    auto inside = [&](int x, int z) { return x >= 0 && x < A.nx && z >= 0 && z < A.nz; };
    auto at = [&](int x, int z) { return (long long)z * A.plane + x; };
    auto tab = [&](int cl) { return A.lut + (size_t)cl * kLutStride; };
    auto dtab = [&](int cl) { return A.dlut + (size_t)cl * kDStride; };

    for (int j = tid; j < T::n_fp; j += kAdjThreads) {
        const int x = x0 - 3 + j % T::FPW, z = z0 - 3 + j / T::FPW;
        sFP[j] = inside(x, z) ? __ldg(A.fp + at(x, z)) : R(0);
    }
    for (int j = tid; j < T::n_v0; j += kAdjThreads) {
        const int x = x0 - 4 + j % (TX + 7), z = z0 + j / (TX + 7);
        sV0[j] = inside(x, z) ? __ldg(A.fv1[0] + at(x, z)) : R(0);
    }
    for (int j = tid; j < T::n_v2; j += kAdjThreads) {
        const int x = x0 + j % TX, z = z0 - 4 + j / TX;
        sV2[j] = inside(x, z) ? __ldg(A.fv1[2] + at(x, z)) : R(0);
    }
    __syncthreads();

    R gsum[T::NI], rk[T::NI];
    int clk[T::NI];
    // q_d: the tile (full pressure adjoint), then the wings
#pragma unroll
    for (int k = 0; k < T::NI; ++k) {
        const int j = tid + k * kAdjThreads, lx = j % TX, lz = j / TX, x = x0 + lx, z = z0 + lz;
        R Qx = 0, Qz = 0;
        gsum[k] = 0;
        clk[k] = 0;
        rk[k] = R(1);
        if (inside(x, z)) {
            const long long i = at(x, z);
            const int cl = __ldg(A.cls + i);
            const R r = PLAIN ? R(1) : ramp2(A, x, z);
            clk[k] = cl;
            rk[k] = r;
            const R qx = dminus_s(A, &sV0[lz * (TX + 7) + lx + 4], 1);
            const R qz = dminus_s(A, &sV2[(lz + 4) * TX + lx], TX);
            double gk;
            pres2<R, NM, true, PLAIN>(A, x, z, i, tab(cl), dtab(cl), r, qx, qz, Qx, Qz, gsum[k], gk);
            A.gk[i] += gk;
        }
        sQx[lz * T::QXW + lx + 7] = Qx;
        sQz[(lz + 7) * TX + lx] = Qz;
    }
    if (FWGB_ADJ_PREFETCH == 2) prefetch_side<R, NM, TX, TZ>(A, 1, x0, z0);
    for (int j = tid; j < 14 * (TZ + TX); j += kAdjThreads) {
        int lx, lz;
        const bool along_x = j < 14 * TZ;
        if (along_x) {       // q_x: 7 points either side of each tile row
            const int w = j % 14;
            lz = j / 14;
            lx = w < 7 ? w - 7 : TX + w - 7;
        } else {             // q_z: 7 rows above and below the tile
            const int jj = j - 14 * TZ, w = jj / TX;
            lx = jj % TX;
            lz = w < 7 ? w - 7 : TZ + w - 7;
        }
        const int x = x0 + lx, z = z0 + lz;
        R Qx = 0, Qz = 0;
        if (inside(x, z)) {
            const long long i = at(x, z);
            const int cl = __ldg(A.cls + i);
            const R r = PLAIN ? R(1) : ramp2(A, x, z);
            R gs;
            double gk;
            if (along_x) pres2<R, NM, false, PLAIN, 0>(A, x, z, i, tab(cl), dtab(cl), r, R(0), R(0), Qx, Qz, gs, gk);
            else pres2<R, NM, false, PLAIN, 2>(A, x, z, i, tab(cl), dtab(cl), r, R(0), R(0), Qx, Qz, gs, gk);
        }
        if (along_x) sQx[lz * T::QXW + lx + 7] = Qx;
        else sQz[(lz + 7) * TX + lx] = Qz;
    }
    __syncthreads();

    // g_d: the tile (full velocity adjoint along both axes), then the wings
#pragma unroll
    for (int k = 0; k < T::NI; ++k) {
        const int j = tid + k * kAdjThreads, lx = j % TX, lz = j / TX, x = x0 + lx, z = z0 + lz;
        R gx = 0, gz = 0;
        if (inside(x, z)) {
            const long long i = at(x, z);
            const R *t = tab(clk[k]), *dtb = dtab(clk[k]);
            const R *fp = &sFP[(lz + 3) * T::FPW + lx + 3];
            gx = vel2<R, NM, true, PLAIN, 0>(A, x, A.nx, 1, i, t, dtb, rk[k], dplus_s(A, &sQx[lz * T::QXW + lx + 7], 1),
                                             dplus_s(A, fp, 1), gsum[k]);
            gz = vel2<R, NM, true, PLAIN, 2>(A, z, A.nz, A.plane, i, t, dtb, rk[k],
                                             dplus_s(A, &sQz[(lz + 7) * TX + lx], TX), dplus_s(A, fp, T::FPW), gsum[k]);
        }
        sGx[lz * T::GXW + lx + 4] = gx;
        sGz[(lz + 4) * TX + lx] = gz;
    }
    for (int j = tid; j < 7 * (TZ + TX); j += kAdjThreads) {
        int lx, lz;
        const bool along_x = j < 7 * TZ;
        if (along_x) {       // g_x: 4 points before and 3 after each tile row
            const int w = j % 7;
            lz = j / 7;
            lx = w < 4 ? w - 4 : TX + w - 4;
        } else {             // g_z: 4 rows above and 3 below the tile
            const int jj = j - 7 * TZ, w = jj / TX;
            lx = jj % TX;
            lz = w < 4 ? w - 4 : TZ + w - 4;
        }
        const int x = x0 + lx, z = z0 + lz;
        R g = 0, unused = 0;
        if (inside(x, z)) {
            const long long i = at(x, z);
            const int cl = __ldg(A.cls + i);
            const R r = PLAIN ? R(1) : ramp2(A, x, z);
            g = along_x ? vel2<R, NM, false, PLAIN, 0>(A, x, A.nx, 1, i, tab(cl), dtab(cl), r,
                                                       dplus_s(A, &sQx[lz * T::QXW + lx + 7], 1), R(0), unused)
                        : vel2<R, NM, false, PLAIN, 2>(A, z, A.nz, A.plane, i, tab(cl), dtab(cl), r,
                                                       dplus_s(A, &sQz[(lz + 7) * TX + lx], TX), R(0), unused);
        }
        if (along_x) sGx[lz * T::GXW + lx + 4] = g;
        else sGz[(lz + 4) * TX + lx] = g;
    }
    __syncthreads();

    // p: the backward differences of g_d on the tile
#pragma unroll
    for (int k = 0; k < T::NI; ++k) {
        const int j = tid + k * kAdjThreads, lx = j % TX, lz = j / TX, x = x0 + lx, z = z0 + lz;
        if (!inside(x, z)) continue;
        const R s = dminus_s(A, &sGx[lz * T::GXW + lx + 4], 1) + dminus_s(A, &sGz[(lz + 4) * TX + lx], TX);
        const long long i = at(x, z);
        A.out.lp[i] = __ldg(A.in.lp + i) - s;
        A.gs[i] += double(gsum[k]);
    }
}

// Tiles whose reads (the q_d halo reaches 7 cells, one more for the velocity
// adjoint's neighbouring density) stay clear of the absorbing layer take the
// PLAIN instance: no layer memory, tissue strength 1.  Registers are held
// to four CTAs per SM (64 per thread) in FP32, two in FP64.
template <typename R, int NM, int TX, int TZ>
__global__ void __launch_bounds__(kAdjThreads, sizeof(R) == 4 ? 4 : 2) k_adj_step2(const AdjArgs<R> A)
{
    extern __shared__ __align__(16) unsigned char adj_smem[];
    const int x0 = blockIdx.x * TX, z0 = blockIdx.y * TZ;
    if (FWGB_ADJ_PREFETCH >= 1) prefetch_side<R, NM, TX, TZ>(A, 0, x0, z0);
    if (FWGB_ADJ_PREFETCH == 1) prefetch_side<R, NM, TX, TZ>(A, 1, x0, z0);
    constexpr int h = 8;
    const bool plain = A.wabs <= 0 || (x0 - h >= A.wabs && x0 + TX + h <= A.nx - A.wabs && z0 - h >= A.wabs &&
                                       z0 + TZ + h <= A.nz - A.wabs);
    if (plain) step2_tile<R, NM, TX, TZ, true>(A, adj_smem, x0, z0);
    else step2_tile<R, NM, TX, TZ, false>(A, adj_smem, x0, z0);
}

constexpr int kAdjTX = FWGB_ADJ_TX, kAdjTZ = FWGB_ADJ_TZ;

template <typename R, int NM>
cudaError_t launch_step2_n(const AdjArgs<R> &A, cudaStream_t s, bool setup)
{
    using T = AdjTile<kAdjTX, kAdjTZ>;
    const size_t smem = (size_t)T::elems * sizeof(R);
    if (setup) return cudaFuncSetAttribute(k_adj_step2<R, NM, kAdjTX, kAdjTZ>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const dim3 grid((unsigned)((A.nx + kAdjTX - 1) / kAdjTX), (unsigned)((A.nz + kAdjTZ - 1) / kAdjTZ));
    k_adj_step2<R, NM, kAdjTX, kAdjTZ><<<grid, kAdjThreads, smem, s>>>(A);
    return cudaGetLastError();
}

// the reverse step's kernels: one in 2D, three in 3D; instantiated per
// dimension and number of mechanisms (their loops unroll).  With setup, only
// the one-kernel form's shared-memory opt-in.
template <typename R, int NM>
cudaError_t launch_reverse_n(const AdjArgs<R> &A, int ndim, dim3 grid, cudaStream_t s, bool setup)
{
    if (ndim == 2) return launch_step2_n<R, NM>(A, s, setup);
    if (setup) return cudaSuccess;
    k_adj_pres<R, 3, NM><<<grid, 256, 0, s>>>(A);
    k_adj_vel<R, 3, NM><<<grid, 256, 0, s>>>(A);
    k_adj_p<R, 3, NM><<<grid, 256, 0, s>>>(A);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_reverse(const AdjArgs<R> &A, int ndim, int nmech, dim3 grid, cudaStream_t s, bool setup = false)
{
    switch (nmech) {
    case 1: return launch_reverse_n<R, 1>(A, ndim, grid, s, setup);
    case 2: return launch_reverse_n<R, 2>(A, ndim, grid, s, setup);
    case 3: return launch_reverse_n<R, 3>(A, ndim, grid, s, setup);
    default: return launch_reverse_n<R, 4>(A, ndim, grid, s, setup);
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

// The recomputation's side stream and the events between it and the caller's
// stream; on every way out, both streams finish before the buffers go.
struct SideStream {
    cudaStream_t main = nullptr, side = nullptr;
    std::vector<cudaEvent_t> ev;
    SideStream() = default;
    SideStream(const SideStream &) = delete;
    SideStream &operator=(const SideStream &) = delete;
    ~SideStream()
    {
        if (side) {
            cudaStreamSynchronize(side);
            cudaStreamDestroy(side);
        }
        if (main) cudaStreamSynchronize(main);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
};

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

    // 2D: one kernel per reverse step, reading the adjoint state from one of a
    // pair of buffers and writing the other; 3D: three kernels in place, with
    // the adjoints of q_d and g_d in global scratch.
    const bool one_kernel = m->ndim == 2;
    // segment images: the states after steps k0 .. k1-2 of a segment (the state
    // before it is its checkpoint, the state after it the next checkpoint)
    Buf lam(SB), lam2(one_kernel ? SB : 0), ck((size_t)n_ck * SB), fin(SB);
    Buf seg0((size_t)std::max(seg_len - 1, 1) * SB), seg1(n_ck > 1 ? (size_t)std::max(seg_len - 1, 1) * SB : 0);
    Buf scratch(one_kernel ? 0 : 6 * vol * sizeof(R)), gacc(2 * vol * sizeof(double)),
        uacc(2 * n_user * sizeof(double));
    const size_t nG = (size_t)m->n_rcv * m->n_rec;
    Buf dG(nG * sizeof(R)), dA0(alpha0 ? n_user * (as_f64 ? 8 : 4) : 0);
    Buf dlut((size_t)m->n_classes * kDStride * sizeof(R)), zero(256);   // zero: step counter of the image steps
    if (!lam.p || (one_kernel && !lam2.p) || !ck.p || !seg0.p || (n_ck > 1 && !seg1.p) || !fin.p || (!one_kernel && !scratch.p) || !gacc.p ||
        !uacc.p || (nG && !dG.p) || (alpha0 && !dA0.p) || !dlut.p || !zero.p)
        return FW_ERR_NOMEM;
    ADJ_CK(cudaMemsetAsync(zero.p, 0, 256, s));
    ADJ_CK(cudaMemsetAsync(lam.p, 0, SB, s));
    if (one_kernel) ADJ_CK(cudaMemsetAsync(lam2.p, 0, SB, s));
    else ADJ_CK(cudaMemsetAsync(scratch.p, 0, 6 * vol * sizeof(R), s));
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
    // the adjoint state's fields at the medium's offsets inside a state-sized buffer
    auto state_in = [&](void *buf) {
        char *L = static_cast<char *>(buf);
        AdjState<R> S{};
        S.lp = reinterpret_cast<R *>(L + off(m->p));
        for (int ax = 0; ax < 3; ++ax) {
            S.lv[ax] = m->v[ax] ? reinterpret_cast<R *>(L + off(m->v[ax])) : nullptr;
            S.lpsi1p[ax] = m->psi1p[ax] ? reinterpret_cast<R *>(L + off(m->psi1p[ax])) : nullptr;
            S.lpsi2p[ax] = m->psi2p[ax] ? reinterpret_cast<R *>(L + off(m->psi2p[ax])) : nullptr;
            for (int k = 0; k < m->nmech; ++k)
                S.lpsi1[k][ax] = m->psi1[k][ax] ? reinterpret_cast<R *>(L + off(m->psi1[k][ax])) : nullptr;
        }
        for (int k = 0; k < m->nmech; ++k) S.lpsi2[k] = reinterpret_cast<R *>(L + off(m->psi2[k]));
        return S;
    };
    A.in = state_in(lam.p);
    A.out = one_kernel ? state_in(lam2.p) : A.in;
    for (int ax = 0; ax < 3; ++ax) {
        A.ax_on[ax] = m->v[ax] != nullptr;
        const bool layer = m->psi1p[ax] != nullptr;
        A.pdh[ax] = layer ? static_cast<const R *>(m->prof[ax][0]) : nullptr;
        A.pah[ax] = layer ? static_cast<const R *>(m->prof[ax][1]) : nullptr;
        A.pdi[ax] = layer ? static_cast<const R *>(m->prof[ax][2]) : nullptr;
        A.pai[ax] = layer ? static_cast<const R *>(m->prof[ax][3]) : nullptr;
        A.Q[ax] = one_kernel ? nullptr : static_cast<R *>(scratch.p) + ax * vol;
        A.Gd[ax] = one_kernel ? nullptr : static_cast<R *>(scratch.p) + (3 + ax) * vol;
    }
    A.kdt = static_cast<const R *>(m->kdt);
    A.rho = static_cast<const R *>(m->rho);
    A.cls = m->cls;
    A.lut = static_cast<const R *>(m->lut);
    A.dlut = static_cast<const R *>(dlut.p);
    A.gk = static_cast<double *>(gacc.p);
    A.gs = static_cast<double *>(gacc.p) + vol;
    const dim3 pgrid((unsigned)((m->NX + 255) / 256), (unsigned)m->NY, (unsigned)m->NZ);   // one thread per point
    const double inv_dxd = 1.0 / std::pow(m->dx, m->ndim);
    ADJ_CK(launch_reverse<R>(A, m->ndim, m->nmech, pgrid, s, true));

    // ---- reverse sweep, one checkpoint segment at a time ----
    // The recomputation of segment si - 1 (a side stream, into the other of two
    // image buffers) runs beside the adjoint of segment si: the adjoint reads
    // only the images and the medium's maps, never the medium's state.
    SideStream ss;
    ss.main = s;
    ADJ_CK(cudaStreamCreateWithFlags(&ss.side, cudaStreamNonBlocking));
    cudaEvent_t ev_start, rec_done[2], rev_done[2], side_done;
    for (cudaEvent_t *e : {&ev_start, &rec_done[0], &rec_done[1], &rev_done[0], &rev_done[1], &side_done}) {
        ADJ_CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
        ss.ev.push_back(*e);
    }
    bool rev_recorded[2] = {false, false};
    char *segs[2] = {static_cast<char *>(seg0.p), static_cast<char *>(seg1.p)};
    // images after steps k0 .. k1-2 of segment si into segs[si & 1]: each step
    // reads the image before it (the checkpoint first) and writes the next
    // (the image step takes memory variables in the state type: FP32 or FP64
    // storage, the only ones fw_gradient accepts)
    auto recompute = [&](int si) -> int {
        const int k0 = si * K, k1 = std::min(n_steps, k0 + K);
        const char *rd = static_cast<const char *>(ck.p) + (size_t)si * SB;
        for (int k = k0; k < k1 - 1; ++k) {
            char *wr = segs[si & 1] + (size_t)(k - k0) * SB;
            const StepImages im{rd, (long long)(wr - rd)};
            const int itk = (int)(it0 + k);
            if ((sizeof(R) == 8 ? image_step_f64(m, im, static_cast<const int *>(zero.p), itk, ss.side)
                                : image_step_f32(m, im, static_cast<const int *>(zero.p), itk, ss.side)) != cudaSuccess)
                return FW_ERR_CUDA;
            rd = wr;
        }
        return FW_OK;
    };
    ADJ_CK(cudaEventRecord(ev_start, s));   // the forward run and the checkpoints
    ADJ_CK(cudaStreamWaitEvent(ss.side, ev_start, 0));
    {
        int rc = recompute(n_ck - 1);
        if (rc) return rc;
    }
    ADJ_CK(cudaEventRecord(rec_done[(n_ck - 1) & 1], ss.side));
    for (int si = n_ck - 1; si >= 0; --si) {
        const int k0 = si * K, k1 = std::min(n_steps, k0 + K);
        ADJ_CK(cudaStreamWaitEvent(s, rec_done[si & 1], 0));
        if (si >= 1) {
            // segs[(si - 1) & 1] was last read by the adjoint of segment si + 1
            if (rev_recorded[(si + 1) & 1]) ADJ_CK(cudaStreamWaitEvent(ss.side, rev_done[(si + 1) & 1], 0));
            int rc = recompute(si - 1);
            if (rc) return rc;
            ADJ_CK(cudaEventRecord(rec_done[(si - 1) & 1], ss.side));
        }
        const char *ck_si = static_cast<const char *>(ck.p) + (size_t)si * SB;
        // image j of the segment: the state after step k0 + j - 1
        auto image = [&](int j) -> const char * {
            if (j == 0) return ck_si;
            if (j == k1 - k0) return si + 1 < n_ck ? ck_si + SB : static_cast<const char *>(fin.p);
            return segs[si & 1] + (size_t)(j - 1) * SB;
        };
        for (int k = k1 - 1; k >= k0; --k) {
            const long long it = it0 + k;
            const int col = (m->n_rcv > 0 && it % m->decim == 0 && it / m->decim < m->n_rec) ? (int)(it / m->decim) : -1;
            if (col >= 0 || (m->n_src > 0 && it < m->wave_len)) {
                const int n_io = m->n_src + (col >= 0 ? m->n_rcv : 0);
                k_adj_io<R><<<(n_io + 255) / 256, 256, 0, s>>>(A.in.lp, m->src_idx, static_cast<const R *>(m->waves),
                                                               m->wave_of, m->wave_len, (int)it, m->n_src, m->src_rcv,
                                                               m->rcv_idx, m->rcv_src, static_cast<const R *>(dG.p),
                                                               m->n_rcv, m->n_rec, col, inv_dxd, A.gk);
            }
            const char *F = image(k - k0), *F1 = image(k - k0 + 1);
            A.fp = reinterpret_cast<const R *>(F + off(m->p));
            for (int ax = 0; ax < 3; ++ax) {
                A.fv1[ax] = m->v[ax] ? reinterpret_cast<const R *>(F1 + off(m->v[ax])) : nullptr;
                A.fpsi2p[ax] = m->psi2p[ax] ? reinterpret_cast<const R *>(F + off(m->psi2p[ax])) : nullptr;
                for (int q = 0; q < m->nmech; ++q)
                    A.fpsi1[q][ax] = m->psi1[q][ax] ? reinterpret_cast<const R *>(F + off(m->psi1[q][ax])) : nullptr;
            }
            for (int q = 0; q < m->nmech; ++q) A.fpsi2[q] = reinterpret_cast<const R *>(F + off(m->psi2[q]));
            ADJ_CK(launch_reverse<R>(A, m->ndim, m->nmech, pgrid, s));
            if (one_kernel) std::swap(A.in, A.out);
        }
        ADJ_CK(cudaEventRecord(rev_done[si & 1], s));
        rev_recorded[si & 1] = true;
        ADJ_CK(cudaGetLastError());
    }
    ADJ_CK(cudaEventRecord(side_done, ss.side));
    ADJ_CK(cudaStreamWaitEvent(s, side_done, 0));
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
