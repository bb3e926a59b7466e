// Host side of the C ABI: medium construction (maps, classes, absorbing
// layer, coefficient tables), sources/receivers, stepping, I/O, checkpoint.
#include "fw_internal.h"
#include "fw_kernels.cuh"

#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

namespace fwgb {
cudaError_t sweeps_f32(const fw_medium *m, cudaStream_t s, int which);
cudaError_t sweeps_bf16(const fw_medium *m, cudaStream_t s, int which);
cudaError_t sweeps_f16(const fw_medium *m, cudaStream_t s, int which);
cudaError_t sweeps_f64(const fw_medium *m, cudaStream_t s, int which);
cudaError_t io_f32(const fw_medium *m, int j, cudaStream_t s);
cudaError_t io_f64(const fw_medium *m, int j, cudaStream_t s);
void noalloc_prepare();
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
bool vel_maps_f32(EncodeTiledFn encode, fw_medium *m);
bool vel_maps_bf16(EncodeTiledFn encode, fw_medium *m);
bool vel_maps_f16(EncodeTiledFn encode, fw_medium *m);
}  // namespace fwgb

using namespace fwgb;

#define FW_CK(call)                                   \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return FW_ERR_CUDA;    \
    } while (0)

namespace {

cudaError_t launch_sweep(const fw_medium *m, cudaStream_t s, int which);

// ---- allocator --------------------------------------------------------------
std::mutex g_alloc_mu;
void *(*g_alloc)(size_t, void *) = nullptr;
void (*g_free)(void *, void *) = nullptr;
void *g_alloc_ctx = nullptr;

// a per-thread allocator (the serving runtime's device arena) takes
// precedence over the process-wide hook
struct ThreadHook {
    void *(*alloc)(size_t, void *) = nullptr;
    void (*release)(void *, void *) = nullptr;
    void *ctx = nullptr;
};
thread_local ThreadHook t_hook;

void *dev_alloc(size_t bytes)
{
    if (bytes == 0) bytes = 256;
    if (t_hook.alloc) return t_hook.alloc(bytes, t_hook.ctx);
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    if (g_alloc) return g_alloc(bytes, g_alloc_ctx);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(void *p)
{
    if (!p) return;
    if (t_hook.release) {
        t_hook.release(p, t_hook.ctx);
        return;
    }
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    if (g_free) g_free(p, g_alloc_ctx);
    else cudaFree(p);
}

// RAII device buffer for temporaries
struct DevBuf {
    void *p = nullptr;
    explicit DevBuf(size_t b) : p(b ? dev_alloc(b) : nullptr) {}
    ~DevBuf() { dev_free(p); }
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// 8th-order staggered weights: sum |c_m| sets the leapfrog stability limit
double stencil_abs_sum()
{
    return 1225.0 / 1024.0 + 245.0 / 3072.0 + 49.0 / 5120.0 + 5.0 / 7168.0;
}

// ---- tensor maps for TMA staging ----------------------------------------------
// The driver's tensor-map encoder, looked up once through the runtime (no
// link against the driver library).  Null where it is not available.
EncodeTiledFn tensor_map_encoder()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Tensor maps of the 3D velocity sweep's streams; the sweep falls back to
// per-thread cp.async staging where they cannot be built (or when the
// environment sets FWGB_NO_TMA=1, for measurement).
void setup_tma(fw_medium *m)
{
    m->tma = false;
    if (m->ndim != 3 || m->storage == FW_STORE_F64) return;
    if (const char *e = std::getenv("FWGB_NO_TMA"))
        if (*e && *e != '0') return;
    EncodeTiledFn enc = tensor_map_encoder();
    if (!enc) return;
    switch (m->storage) {
    case FW_STORE_F32: m->tma = vel_maps_f32(enc, m); break;
    case FW_STORE_BF16: m->tma = vel_maps_bf16(enc, m); break;
    case FW_STORE_F16: m->tma = vel_maps_f16(enc, m); break;
    default: break;
    }
}

// ---- time-space stencil (Sec. 3.3, after Tan & Huang 2014) -----------------
// Weights of the first derivative along d: a_m on the on-axis differences
// f(+m) - f(-m+1), b on the two-point differences at the -+1 neighbours across
// each of the other D-1 axes.  With r = c dt/dx, b = r^2/24 and the a_m solve
//     sum_m (2m-1)^(2j-1) a_m = r^(2j-2) - 2 (D-1) b,   j = 1..4,
// the conditions under which the leapfrog's plane-wave relation matches
// omega = c|k| along the axes to order k^7 and across them at k_d k_e^2.
// The right side is a polynomial in r^2, so is every a_m:
// a_m = sum_n ts[m][n] r^(2n); ts is found by solving the 4x4 system for the
// four coefficient vectors of that polynomial.
void time_space_polynomials(int ndim, double ts[4][4])
{
    double rhs[4][4] = {};          // rhs[n][j]: coefficient of r^(2n) in row j
    for (int j = 0; j < 4; ++j) {
        rhs[0][j] = j == 0 ? 1.0 : 0.0;
        rhs[1][j] = (j == 1 ? 1.0 : 0.0) - 2.0 * (ndim - 1) / 24.0;
        rhs[2][j] = j == 2 ? 1.0 : 0.0;
        rhs[3][j] = j == 3 ? 1.0 : 0.0;
    }
    for (int n = 0; n < 4; ++n) {
        double A[4][5];
        for (int j = 0; j < 4; ++j) {
            for (int mm = 0; mm < 4; ++mm) A[j][mm] = std::pow(2.0 * mm + 1.0, 2 * j + 1);
            A[j][4] = rhs[n][j];
        }
        for (int col = 0; col < 4; ++col) {        // Gauss-Jordan with partial pivoting
            int piv = col;
            for (int r = col + 1; r < 4; ++r)
                if (std::fabs(A[r][col]) > std::fabs(A[piv][col])) piv = r;
            for (int c = 0; c < 5; ++c) std::swap(A[col][c], A[piv][c]);
            for (int r = 0; r < 4; ++r) {
                if (r == col) continue;
                const double f = A[r][col] / A[col][col];
                for (int c = col; c < 5; ++c) A[r][c] -= f * A[col][c];
            }
        }
        for (int mm = 0; mm < 4; ++mm) ts[mm][n] = A[mm][4] / A[mm][mm];
    }
}

// Largest |amplification| factor r_eff * |K(theta)| dx/2 of the lossless
// time-space scheme over a grid of phase advances theta in [0, pi]^D, for the
// weights of Courant number r (the scheme is stable where it is <= 1).
double time_space_amplification(int ndim, const double ts[4][4], double r, double r_eff)
{
    const double kPi = 3.14159265358979323846;
    const double r2 = r * r, b = r2 / 24.0;
    double a[4];
    for (int mm = 0; mm < 4; ++mm) a[mm] = ((ts[mm][3] * r2 + ts[mm][2]) * r2 + ts[mm][1]) * r2 + ts[mm][0];
    const int nt = 33;
    double worst = 0.0;
    const int n2 = ndim == 3 ? nt : 1;
    for (int i = 0; i < nt; ++i)
        for (int j = 0; j < nt; ++j)
            for (int l = 0; l < n2; ++l) {
                const double th[3] = {kPi * i / (nt - 1), kPi * j / (nt - 1), ndim == 3 ? kPi * l / (nt - 1) : 0.0};
                double ss = 0.0;
                for (int d = 0; d < ndim; ++d) {
                    double s = 0.0;
                    for (int mm = 0; mm < 4; ++mm) s += a[mm] * std::sin((2 * mm + 1) * th[d] / 2.0);
                    double cr = 0.0;
                    for (int e = 0; e < ndim; ++e)
                        if (e != d) cr += 2.0 * std::cos(th[e]);
                    s += b * std::sin(th[d] / 2.0) * cr;
                    ss += s * s;
                }
                worst = std::max(worst, r_eff * std::sqrt(ss));
            }
    return worst;
}

// ---- device helpers for construction ---------------------------------------

// Gather an unpadded user map [NZ][NY][NX] (float) into the padded layout,
// replacing the absorbing layer of every axis by the nearest interior value.
template <typename T, typename S>
__global__ void k_gather_inherit(T *dst, const S *src, int nx, int ny, int nz, int px, int w)
{
    const long long n = (long long)nx * ny * nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        int x = int(i % nx);
        long long r = i / nx;
        int y = int(r % ny);
        int z = int(r / ny);
        auto clampw = [w](int c, int n_) {
            if (w <= 0) return c;
            int lo = min(w, n_ - 1), hi = max(n_ - 1 - w, 0);
            if (lo > hi) lo = hi = n_ / 2;
            return min(max(c, lo), hi);
        };
        int sx = clampw(x, nx), sy = (ny > 1) ? clampw(y, ny) : y, sz = clampw(z, nz);
        dst[((long long)z * ny + y) * px + x] = T(src[((long long)sz * ny + sy) * nx + sx]);
    }
}

template <typename T>
__global__ void k_kdt(T *kdt, const T *rho, const T *c, T *b2dt, const T *beta, double dt, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double r = double(rho[i]), cc = double(c[i]);
        kdt[i] = T(r * cc * cc * dt);
        if (b2dt) b2dt[i] = T(2.0 * double(beta[i]) * dt);
    }
}

// max of c and of c/sqrt(kappa1 kappa2) over the padded map (padding is 0)
template <typename T>
__global__ void k_cmax(const T *c, const uint16_t *cls, const double *ceff_scale, size_t n,
                       unsigned int *out)
{
    float m0 = 0.f, m1 = 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float cc = float(c[i]);
        m0 = fmaxf(m0, cc);
        m1 = fmaxf(m1, float(double(cc) * ceff_scale[cls[i]]));
    }
    for (int o = 16; o > 0; o >>= 1) {
        m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, o));
        m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, __float_as_uint(m0));
        atomicMax(out + 1, __float_as_uint(m1));
    }
}

// dense <-> padded copies for field I/O (element type conversion included)
template <typename S, typename D>
__global__ void k_unpad(D *dst, const S *src, int nx, int ny, int nz, int px, double scale)
{
    const long long n = (long long)nx * ny * nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        int x = int(i % nx);
        long long r = i / nx;
        dst[i] = D(double(src[r * px + x]) * scale);
    }
}

template <typename S, typename D>
__global__ void k_pad(D *dst, const S *src, int nx, int ny, int nz, int px, double scale)
{
    const long long n = (long long)nx * ny * nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        int x = int(i % nx);
        long long r = i / nx;
        dst[r * px + x] = D(double(src[i]) * scale);
    }
}

__global__ void k_scale_half(__half *a, size_t n, float f)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        a[i] = __float2half_rn(__half2float(a[i]) * f);
}

template <typename T>
__global__ void k_src_gain(T *gain, const long long *idx, const T *kdt, double inv_dxd, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) gain[i] = T(double(kdt[idx[i]]) * inv_dxd);
}

int grid_blocks(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 152 * 16); }

// ---- absorbing-layer profile (host, FP64) ------------------------------------
// depth s [cells] of the point (i + off) into the layer of width w on an axis
// of n points; layer profile: quadratic ramp to 0.1 d_max over the transition
// cells, then 0.1 -> 1 quadratic over the absorbing cells;
// alpha = pi f0 (1 - s / w); d_max = -3 c_max ln(R0) / (2 L_B dx).
void profile(int n, int w, int lt, int lb, double off, double dmax, double f0,
             std::vector<double> &d, std::vector<double> &al)
{
    d.assign(n, 0.0);
    al.assign(n, 0.0);
    if (w <= 0) return;
    for (int i = 0; i < n; ++i) {
        double x = i + off;
        double s = std::max(0.0, std::max((w - 0.5) - x, x - (n - w - 0.5)));
        double dd;
        if (lt > 0)
            dd = s <= lt ? 0.1 * dmax * (s / lt) * (s / lt) : dmax * (0.1 + 0.9 * ((s - lt) / lb) * ((s - lt) / lb));
        else
            dd = dmax * (s / lb) * (s / lb);
        d[i] = s > 0.0 ? dd : 0.0;
        al[i] = 3.14159265358979323846 * f0 * (1.0 - s / w);
    }
}

// ---- layout -----------------------------------------------------------------
struct Layout {
    size_t off_state_end = 0;   // [0, off_state_end): state + counters (checkpoint image)
    size_t total = 0;
    size_t p, v[3], psi1[FW_MAX_MECH][3], psi2[FW_MAX_MECH], psi1p[3], psi2p[3], it, mon;
    size_t kdt, rho, b2dt, cls, lut, cdev, prof[3][4];
};

struct Dims {
    int ndim, NX, NY, NZ, px, es, eps, wabs, nmech;
    size_t plane, vol;
    bool nl;
};

int axis_len(const Dims &d, int ax) { return ax == 0 ? d.NX : (ax == 1 ? d.NY : d.NZ); }
bool axis_on(const Dims &d, int ax) { return !(d.ndim == 2 && ax == 1); }

Layout make_layout(const Dims &d, int n_classes)
{
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o = align_up(o + bytes, 256);
        return r;
    };
    const size_t sv = d.vol * d.es, spv = d.vol * d.eps;
    L.p = take(sv);
    for (int ax = 0; ax < 3; ++ax) L.v[ax] = axis_on(d, ax) ? take(sv) : 0;
    for (int m = 0; m < d.nmech; ++m)
        for (int ax = 0; ax < 3; ++ax) L.psi1[m][ax] = axis_on(d, ax) ? take(spv) : 0;
    for (int m = 0; m < d.nmech; ++m) L.psi2[m] = take(spv);
    for (int ax = 0; ax < 3; ++ax) {
        L.psi1p[ax] = (axis_on(d, ax) && d.wabs > 0) ? take(sv) : 0;
        L.psi2p[ax] = (axis_on(d, ax) && d.wabs > 0) ? take(sv) : 0;
    }
    L.it = take(sizeof(int) * 64);
    L.mon = take(sizeof(Monitor));
    L.off_state_end = o;
    L.kdt = take(sv);
    L.rho = take(sv);
    L.b2dt = d.nl ? take(sv) : 0;
    L.cls = take(d.vol * sizeof(uint16_t));
    L.cdev = take(sv);
    L.lut = take((size_t)std::max(n_classes, 1) * kLutStride * d.es);
    for (int ax = 0; ax < 3; ++ax)
        for (int k = 0; k < 4; ++k) L.prof[ax][k] = take((size_t)axis_len(d, ax) * d.es + 64);
    L.total = o;
    return L;
}

int make_dims(const fw_grid *g, int n_mech, int storage, bool nl, Dims *d)
{
    if (!g || (g->ndim != 2 && g->ndim != 3)) return FW_ERR_ARG;
    if (n_mech < 1 || n_mech > FW_MAX_MECH) return FW_ERR_ARG;
    if (storage < FW_STORE_F32 || storage > FW_STORE_F64) return FW_ERR_ARG;
    if (g->nx < 1 || g->ny < 1 || g->nz < 1 || !(g->dx > 0)) return FW_ERR_ARG;
    if (g->ndim == 2 && g->nz != 1) return FW_ERR_ARG;
    if (g->pml < 0 || g->transition < 0 || (g->transition > 0 && g->pml == 0)) return FW_ERR_ARG;
    if (g->layer_relax != 0 && g->layer_relax != 1) return FW_ERR_ARG;
    if (g->time_order != 0 && g->time_order != 2 && g->time_order != 4) return FW_ERR_ARG;
    d->ndim = g->ndim;
    d->NX = g->nx;
    d->NY = g->ndim == 3 ? g->ny : 1;
    d->NZ = g->ndim == 3 ? g->nz : g->ny;
    d->px = (int)align_up(g->nx, 32);
    d->plane = (size_t)d->px * d->NY;
    d->vol = d->plane * d->NZ;
    d->es = storage == FW_STORE_F64 ? 8 : 4;
    d->eps = storage == FW_STORE_F64 ? 8 : (storage == FW_STORE_F32 ? 4 : 2);
    d->wabs = g->pml + g->transition;
    d->nmech = n_mech;
    d->nl = nl;
    for (int ax = 0; ax < 3; ++ax)
        if (axis_on(*d, ax) && axis_len(*d, ax) > 1 && 2 * d->wabs >= axis_len(*d, ax)) return FW_ERR_ARG;
    return FW_OK;
}

// per-class coefficient table for the run's dt (Eqs. relaxation_a/b), with
// the midpoint memory-variable update folded in (ceff, hb); sc1 and sc2 scale
// the stored memory variables of the gradient and divergence sides (binary16
// storage).
std::vector<double> build_lut(const std::vector<fw_relax_params> &cl, double dt, double sc1, double sc2)
{
    std::vector<double> t(cl.size() * kLutStride, 0.0);
    for (size_t c = 0; c < cl.size(); ++c) {
        const fw_relax_params &p = cl[c];
        double *e = &t[c * kLutStride];
        e[0] = p.kappa1;
        e[1] = p.kappa2;
        double sa1 = 0.0, sa2 = 0.0;   // sum a/2 per stretch
        for (int m = 0; m < p.n_mech; ++m) {
            double b1 = std::exp(-(p.d1[m] / p.kappa1 + p.alpha1[m]) * dt);
            double a1 = p.d1[m] / (p.kappa1 * (p.d1[m] + p.kappa1 * p.alpha1[m])) * (b1 - 1.0);
            double b2 = std::exp(-(p.d2[m] / p.kappa2 + p.alpha2[m]) * dt);
            double a2 = p.d2[m] / (p.kappa2 * (p.d2[m] + p.kappa2 * p.alpha2[m])) * (b2 - 1.0);
            sa1 += 0.5 * a1;
            sa2 += 0.5 * a2;
            e[kLutA1 + m] = a1 * sc1;
            e[kLutB1 + m] = b1;
            e[kLutH1 + m] = 0.5 * (1.0 + b1) / sc1;
            e[kLutA2 + m] = a2 * sc2;
            e[kLutB2 + m] = b2;
            e[kLutH2 + m] = 0.5 * (1.0 + b2) / sc2;
        }
        e[2] = 1.0 / p.kappa1 + sa1;
        e[3] = 1.0 / p.kappa2 + sa2;
        e[kLutDk] = sa1;
        e[kLutDk + 1] = sa2;
    }
    return t;
}

// Stored value of a memory variable = psi * scale.  binary16 storage keeps
// psi in scaled units so that the memory variables of the expected fields
// stay in the normal range of the format: the gradient side psi1 (Pa/m) is
// stored as a pressure difference per cell in units of the reference
// pressure p_ref (psi1 dx / p_ref), the divergence side psi2 (1/s) as the
// same with the reference impedance rho c = 1.54e6 kg/(m^2 s)
// (psi2 dx Z / p_ref).  p_ref follows the sources (fw_set_sources: 1/100 of
// the largest pressure increment one step of the sources adds, about 1/100
// of the emitted amplitude; 10 Pa before any source).  Other storages use 1.
double psi_scale_of(const fw_medium *m, int side)
{
    if (m->storage != FW_STORE_F16) return 1.0;
    const double pref = m->psi_pref, zref = 1000.0 * 1540.0;
    return side == 1 ? m->dx / pref : m->dx * zref / pref;
}

template <typename T> std::vector<T> cast_vec(const std::vector<double> &v)
{
    return std::vector<T>(v.begin(), v.end());
}

int upload_doubles(fw_medium *m, void *dst, const std::vector<double> &v, cudaStream_t s)
{
    if (m->es == 8) {
        FW_CK(cudaMemcpyAsync(dst, v.data(), v.size() * 8, cudaMemcpyHostToDevice, s));
        FW_CK(cudaStreamSynchronize(s));
    } else {
        std::vector<float> f = cast_vec<float>(v);
        FW_CK(cudaMemcpyAsync(dst, f.data(), f.size() * 4, cudaMemcpyHostToDevice, s));
        FW_CK(cudaStreamSynchronize(s));
    }
    return FW_OK;
}

// Upload a user map (host or device, dense float) into the padded layout with
// absorbing-layer inheritance (inherit = false: a plain copy, the caller's
// values kept inside the layer).  T is the device element type.
template <typename T, typename S>
int upload_map(const fw_medium *m, T *dst, const S *src, cudaStream_t s, bool inherit = true)
{
    const size_t n = (size_t)m->NX * m->NY * m->NZ;
    const S *dsrc = src;
    DevBuf stage(is_device_ptr(src) ? 0 : n * sizeof(S));
    if (!is_device_ptr(src)) {
        if (!stage.p) return FW_ERR_NOMEM;
        FW_CK(cudaMemcpyAsync(stage.p, src, n * sizeof(S), cudaMemcpyDefault, s));
        dsrc = static_cast<const S *>(stage.p);
    }
    k_gather_inherit<T, S><<<grid_blocks(n), 256, 0, s>>>(dst, dsrc, m->NX, m->NY, m->NZ, m->px,
                                                          inherit ? m->wabs : 0);
    FW_CK(cudaGetLastError());
    FW_CK(cudaStreamSynchronize(s));
    return FW_OK;
}

int check_map_positive(const float *h, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!(h[i] > 0.0f) || !std::isfinite(h[i])) return FW_ERR_ARG;
    return FW_OK;
}

int fetch_host(const float *src, size_t n, std::vector<float> &out)
{
    out.resize(n);
    FW_CK(cudaMemcpy(out.data(), src, n * sizeof(float), cudaMemcpyDefault));
    return FW_OK;
}

// cached graphs bake kernel arguments (buffers, counts): drop them whenever
// those change
void drop_graphs(fw_medium *m)
{
    for (auto &kv : m->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    m->graphs.clear();
}

void release(fw_medium *m)
{
    if (!m) return;
    drop_graphs(m);
    if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
    dev_free(m->src_buf);
    dev_free(m->rcv_buf);
    dev_free(m->slab);
    delete m;
}

cudaError_t launch_sweep(const fw_medium *m, cudaStream_t s, int which)
{
    switch (m->storage) {
    case FW_STORE_F32: return sweeps_f32(m, s, which);
    case FW_STORE_BF16: return sweeps_bf16(m, s, which);
    case FW_STORE_F16: return sweeps_f16(m, s, which);
    default: return sweeps_f64(m, s, which);
    }
}

cudaError_t launch_io_any(const fw_medium *m, int j, cudaStream_t s)
{
    return m->storage == FW_STORE_F64 ? io_f64(m, j, s) : io_f32(m, j, s);
}

cudaError_t launch_step(const fw_medium *m, int j, cudaStream_t s)
{
    cudaError_t e = launch_sweep(m, s, 3);
    if (e != cudaSuccess) return e;
    return launch_io_any(m, j, s);
}

int enqueue_steps(fw_medium *m, int n, cudaStream_t s)
{
    for (int j = 0; j < n; ++j) FW_CK(launch_step(m, j, s));
    k_advance<<<1, 1, 0, s>>>(m->d_it, n);
    FW_CK(cudaGetLastError());
    return FW_OK;
}

// pointer of field (which, idx) and its element kind: 0 state, 1 psi
int field_ptr(fw_medium *m, int which, int idx, void **ptr, int *kind)
{
    const int nd = m->ndim;
    auto ax_of = [nd](int d) { return d == 0 ? 0 : (nd == 3 ? d : 2); };
    *kind = 0;
    switch (which) {
    case FW_FIELD_P: *ptr = m->p; return idx == 0 ? FW_OK : FW_ERR_ARG;
    case FW_FIELD_V:
        if (idx < 0 || idx >= nd) return FW_ERR_ARG;
        *ptr = m->v[ax_of(idx)];
        return FW_OK;
    case FW_FIELD_PSI1:
        if (idx < 0 || idx >= nd * m->nmech) return FW_ERR_ARG;
        *ptr = m->psi1[idx / nd][ax_of(idx % nd)];
        *kind = 1;
        return FW_OK;
    case FW_FIELD_PSI2:
        if (idx < 0 || idx >= m->nmech) return FW_ERR_ARG;
        *ptr = m->psi2[idx];
        *kind = 1;
        return FW_OK;
    case FW_FIELD_PSI1P:
    case FW_FIELD_PSI2P:
        if (idx < 0 || idx >= nd || m->wabs == 0) return FW_ERR_ARG;
        *ptr = which == FW_FIELD_PSI1P ? m->psi1p[ax_of(idx)] : m->psi2p[ax_of(idx)];
        return FW_OK;
    default: return FW_ERR_ARG;
    }
}

template <typename D>
cudaError_t unpad_any(const fw_medium *m, void *src, int kind, D *dst, double scale, cudaStream_t s)
{
    const size_t n = (size_t)m->NX * m->NY * m->NZ;
    int nb = grid_blocks(n);
    if (kind == 0 || m->storage == FW_STORE_F32 || m->storage == FW_STORE_F64) {
        if (m->es == 8) k_unpad<double, D><<<nb, 256, 0, s>>>(dst, (const double *)src, m->NX, m->NY, m->NZ, m->px, scale);
        else k_unpad<float, D><<<nb, 256, 0, s>>>(dst, (const float *)src, m->NX, m->NY, m->NZ, m->px, scale);
    } else if (m->storage == FW_STORE_BF16) {
        k_unpad<__nv_bfloat16, D><<<nb, 256, 0, s>>>(dst, (const __nv_bfloat16 *)src, m->NX, m->NY, m->NZ, m->px, scale);
    } else {
        k_unpad<__half, D><<<nb, 256, 0, s>>>(dst, (const __half *)src, m->NX, m->NY, m->NZ, m->px, scale);
    }
    return cudaGetLastError();
}

template <typename S>
cudaError_t pad_any(const fw_medium *m, void *dst, int kind, const S *src, double scale, cudaStream_t s)
{
    const size_t n = (size_t)m->NX * m->NY * m->NZ;
    int nb = grid_blocks(n);
    if (kind == 0 || m->storage == FW_STORE_F32 || m->storage == FW_STORE_F64) {
        if (m->es == 8) k_pad<S, double><<<nb, 256, 0, s>>>((double *)dst, src, m->NX, m->NY, m->NZ, m->px, scale);
        else k_pad<S, float><<<nb, 256, 0, s>>>((float *)dst, src, m->NX, m->NY, m->NZ, m->px, scale);
    } else if (m->storage == FW_STORE_BF16) {
        k_pad<S, __nv_bfloat16><<<nb, 256, 0, s>>>((__nv_bfloat16 *)dst, src, m->NX, m->NY, m->NZ, m->px, scale);
    } else {
        k_pad<S, __half><<<nb, 256, 0, s>>>((__half *)dst, src, m->NX, m->NY, m->NZ, m->px, scale);
    }
    return cudaGetLastError();
}

// C-order mask over the user grid -> padded linear indices (kernel layout)
std::vector<long long> mask_to_index(const fw_medium *m, const uint8_t *mask)
{
    std::vector<long long> out;
    const size_t n = (size_t)m->NX * m->NY * m->NZ;
    for (size_t i = 0; i < n; ++i)
        if (mask[i]) {
            size_t x = i % m->NX, r = i / m->NX;
            out.push_back((long long)(r * m->px + x));
        }
    return out;
}

int choose_zseg(const fw_medium *m)
{
    // tuning override: FWGB_ZSEG planes per CTA (8..1024)
    if (const char *e = std::getenv("FWGB_ZSEG")) {
        int z = std::atoi(e);
        if (z >= 8 && z <= 1024) return z;
    }
    // 16 planes per CTA measured best on the 512^3 workload (L2 sharing of
    // the halo planes between concurrently resident CTAs); at least 8 waves
    // of CTAs over the 152 SMs
    const int tw = m->ndim == 3 ? (m->es == 8 ? 64 : 128) : 256;
    const int by = m->ndim == 3 ? 8 : 1;
    long long tiles = (long long)((m->NX + tw - 1) / tw) * ((m->NY + by - 1) / by);
    int z = 16;
    while (z > 8 && tiles * ((m->NZ + z - 1) / z) < 152LL * 8) z /= 2;
    return z;
}

int create_common(const fw_grid *g, const float *c, const float *rho, const float *beta,
                  const uint16_t *class_idx, const std::vector<fw_relax_params> &classes, int storage,
                  cudaStream_t s, fw_medium **out)
{
    if (!out || !c || !rho || !class_idx || classes.empty()) return FW_ERR_ARG;
    *out = nullptr;
    const int nm = classes[0].n_mech;
    for (auto &p : classes) {
        if (p.n_mech != nm) return FW_ERR_ARG;
        if (!(p.kappa1 > 0 && p.kappa2 > 0)) return FW_ERR_ARG;
        for (int i = 0; i < nm; ++i)
            if (!(p.d1[i] >= 0 && p.d2[i] >= 0 && p.alpha1[i] > 0 && p.alpha2[i] > 0)) return FW_ERR_ARG;
    }
    if (classes.size() > 65535) return FW_ERR_ARG;
    Dims d{};
    int rc = make_dims(g, nm, storage, beta != nullptr, &d);
    if (rc) return rc;
    const size_t n = (size_t)d.NX * d.NY * d.NZ;
    double c_min = 0.0;
    // argument checks on the host copies
    {
        std::vector<float> hc, hr;
        if ((rc = fetch_host(c, n, hc)) || (rc = fetch_host(rho, n, hr))) return rc;
        if (check_map_positive(hc.data(), n) || check_map_positive(hr.data(), n)) return FW_ERR_ARG;
        c_min = *std::min_element(hc.begin(), hc.end());
        std::vector<uint16_t> hk(n);
        FW_CK(cudaMemcpy(hk.data(), class_idx, n * sizeof(uint16_t), cudaMemcpyDefault));
        for (size_t i = 0; i < n; ++i)
            if (hk[i] >= classes.size()) return FW_ERR_ARG;
    }
    fw_medium *m = new (std::nothrow) fw_medium();
    if (!m) return FW_ERR_NOMEM;
    m->g = *g;
    m->ndim = d.ndim;
    m->nmech = nm;
    m->storage = storage;
    m->nonlinear = d.nl;
    m->NX = d.NX; m->NY = d.NY; m->NZ = d.NZ;
    m->px = d.px;
    m->plane = d.plane;
    m->vol = d.vol;
    m->es = d.es;
    m->eps = d.eps;
    m->dx = g->dx;
    m->wabs = d.wabs;
    m->n_classes = (int)classes.size();
    m->classes = classes;
    m->time_order = g->time_order == 4 ? 4 : 2;
    if (m->time_order == 4) time_space_polynomials(d.ndim, m->ts_a);
    Layout L = make_layout(d, m->n_classes);
    m->slab = dev_alloc(L.total);
    m->slab_bytes = L.total;
    if (!m->slab) { release(m); return FW_ERR_NOMEM; }
    char *base = static_cast<char *>(m->slab);
    auto at = [base](size_t off) { return static_cast<void *>(base + off); };
    if (cudaMemsetAsync(m->slab, 0, L.total, s) != cudaSuccess) { release(m); return FW_ERR_CUDA; }
    m->p = at(L.p);
    for (int ax = 0; ax < 3; ++ax) {
        if (axis_on(d, ax)) {
            m->v[ax] = at(L.v[ax]);
            for (int k = 0; k < nm; ++k) m->psi1[k][ax] = at(L.psi1[k][ax]);
            if (d.wabs > 0) { m->psi1p[ax] = at(L.psi1p[ax]); m->psi2p[ax] = at(L.psi2p[ax]); }
        }
        for (int k = 0; k < 4; ++k) m->prof[ax][k] = at(L.prof[ax][k]);
    }
    for (int k = 0; k < nm; ++k) m->psi2[k] = at(L.psi2[k]);
    m->d_it = static_cast<int *>(at(L.it));
    m->mon = static_cast<Monitor *>(at(L.mon));
    m->kdt = at(L.kdt);
    m->rho = at(L.rho);
    m->b2dt = d.nl ? at(L.b2dt) : nullptr;
    m->cls = static_cast<uint16_t *>(at(L.cls));
    m->lut = at(L.lut);
    m->cdev = at(L.cdev);
    m->zseg = choose_zseg(m);
    setup_tma(m);
    // maps into the padded layout with inheritance
    if (d.es == 8) {
        if ((rc = upload_map(m, (double *)m->cdev, c, s)) || (rc = upload_map(m, (double *)m->rho, rho, s))) { release(m); return rc; }
    } else {
        if ((rc = upload_map(m, (float *)m->cdev, c, s)) || (rc = upload_map(m, (float *)m->rho, rho, s))) { release(m); return rc; }
    }
    if ((rc = upload_map(m, m->cls, class_idx, s, g->layer_relax == 0))) { release(m); return rc; }
    // c_max and c_eff,max = max c / sqrt(kappa1 kappa2)
    {
        std::vector<double> sc(classes.size());
        for (size_t i = 0; i < classes.size(); ++i) sc[i] = 1.0 / std::sqrt(classes[i].kappa1 * classes[i].kappa2);
        DevBuf dsc(sc.size() * sizeof(double)), dmx(2 * sizeof(unsigned int));
        if (!dsc.p || !dmx.p) { release(m); return FW_ERR_NOMEM; }
        // stream-ordered uploads: the kernel below runs on s, which need not
        // wait for the legacy stream
        if (cudaMemcpyAsync(dsc.p, sc.data(), sc.size() * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemsetAsync(dmx.p, 0, 8, s) != cudaSuccess) { release(m); return FW_ERR_CUDA; }
        if (d.es == 8) k_cmax<double><<<grid_blocks(d.vol), 256, 0, s>>>((const double *)m->cdev, m->cls, (const double *)dsc.p, d.vol, (unsigned *)dmx.p);
        else k_cmax<float><<<grid_blocks(d.vol), 256, 0, s>>>((const float *)m->cdev, m->cls, (const double *)dsc.p, d.vol, (unsigned *)dmx.p);
        unsigned hm[2];
        if (cudaStreamSynchronize(s) != cudaSuccess ||
            cudaMemcpy(hm, dmx.p, 8, cudaMemcpyDeviceToHost) != cudaSuccess) { release(m); return FW_ERR_CUDA; }
        float f0v, f1v;
        std::memcpy(&f0v, &hm[0], 4);
        std::memcpy(&f1v, &hm[1], 4);
        m->c_max = f0v;
        m->ceff_max = f1v;
    }
    if (g->dt > 0) m->dt = g->dt;
    else if (g->cfl > 0) m->dt = g->cfl * g->dx / m->ceff_max;
    else { release(m); return FW_ERR_ARG; }
    if (m->time_order == 2) {
        const double limit = 1.0 / (std::sqrt((double)d.ndim) * stencil_abs_sum());
        if (m->ceff_max * m->dt / g->dx > limit * (1.0 + 1e-9)) { release(m); return FW_ERR_ARG; }
    } else {
        // weights of the slowest and of the fastest cell with the fastest
        // effective speed: the amplification falls with r at its maximum
        // (theta = pi in every direction), so the two ends bound the map
        const double re = m->ceff_max * m->dt / g->dx;
        for (double cc : {c_min, m->c_max})
            if (time_space_amplification(d.ndim, m->ts_a, cc * m->dt / g->dx, re) > 1.0 + 1e-9) {
                release(m);
                return FW_ERR_ARG;
            }
    }
    // K dt and 2 beta dt
    {
        DevBuf bt(d.nl ? d.vol * d.es : 0);
        if (d.nl) {
            if (!bt.p) { release(m); return FW_ERR_NOMEM; }
            if (d.es == 8) rc = upload_map(m, (double *)bt.p, beta, s);
            else rc = upload_map(m, (float *)bt.p, beta, s);
            if (rc) { release(m); return rc; }
        }
        if (d.es == 8)
            k_kdt<double><<<grid_blocks(d.vol), 256, 0, s>>>((double *)m->kdt, (const double *)m->rho, (const double *)m->cdev,
                                                           (double *)m->b2dt, (const double *)bt.p, m->dt, d.vol);
        else
            k_kdt<float><<<grid_blocks(d.vol), 256, 0, s>>>((float *)m->kdt, (const float *)m->rho, (const float *)m->cdev,
                                                          (float *)m->b2dt, (const float *)bt.p, m->dt, d.vol);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) { release(m); return FW_ERR_CUDA; }
    }
    // class table and absorbing profiles
    if ((rc = upload_doubles(m, m->lut, build_lut(classes, m->dt, psi_scale_of(m, 1), psi_scale_of(m, 2)), s))) { release(m); return rc; }
    {
        const double r0 = g->pml_r0 > 0 ? g->pml_r0 : 1e-5;
        const double dmax = g->pml > 0 ? -3.0 * m->c_max * std::log(r0) / (2.0 * g->pml * g->dx) : 0.0;
        for (int ax = 0; ax < 3; ++ax) {
            const int nax = axis_len(d, ax);
            const int w = (axis_on(d, ax) && nax > 1) ? d.wabs : 0;
            std::vector<double> pd, pa;
            profile(nax, w, g->transition, g->pml, 0.5, dmax, g->f0, pd, pa);
            if ((rc = upload_doubles(m, m->prof[ax][0], pd, s)) || (rc = upload_doubles(m, m->prof[ax][1], pa, s))) { release(m); return rc; }
            profile(nax, w, g->transition, g->pml, 0.0, dmax, g->f0, pd, pa);
            if ((rc = upload_doubles(m, m->prof[ax][2], pd, s)) || (rc = upload_doubles(m, m->prof[ax][3], pa, s))) { release(m); return rc; }
        }
    }
    if (cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking) != cudaSuccess) { release(m); return FW_ERR_CUDA; }
    if (launch_sweep(m, s, 4) != cudaSuccess) { release(m); return FW_ERR_CUDA; }
    if (cudaStreamSynchronize(s) != cudaSuccess) { release(m); return FW_ERR_CUDA; }
    noalloc_prepare();
    m->last_stream = s;
    *out = m;
    return FW_OK;
}

// binary16 memory variables: move the pressure reference to 1/100 of the
// largest per-step source increment max|gain| max|waveform|, rescaling what
// the memory variables hold and the class table's scaled coefficients.
int set_psi_reference(fw_medium *m, const float *waveforms, size_t wl)
{
    std::vector<float> w(wl), gain(m->n_src);
    FW_CK(cudaMemcpy(w.data(), waveforms, wl * sizeof(float), cudaMemcpyDefault));
    FW_CK(cudaMemcpy(gain.data(), m->src_gain, gain.size() * sizeof(float), cudaMemcpyDeviceToHost));
    double wmax = 0.0, gmax = 0.0;
    for (float x : w) wmax = std::max(wmax, (double)std::fabs(x));
    for (float x : gain) gmax = std::max(gmax, (double)std::fabs(x));
    const double pref = wmax * gmax / 100.0;
    if (!(pref > 1e-30 && pref < 1e30) || pref == m->psi_pref) return FW_OK;
    const float f = (float)(m->psi_pref / pref);     // stored ~ 1/p_ref
    cudaStream_t s = m->last_stream;
    for (int k = 0; k < m->nmech; ++k) {
        for (int ax = 0; ax < 3; ++ax)
            if (m->psi1[k][ax]) k_scale_half<<<grid_blocks(m->vol), 256, 0, s>>>((__half *)m->psi1[k][ax], m->vol, f);
        k_scale_half<<<grid_blocks(m->vol), 256, 0, s>>>((__half *)m->psi2[k], m->vol, f);
    }
    FW_CK(cudaGetLastError());
    m->psi_pref = pref;
    int rc = upload_doubles(m, m->lut, build_lut(m->classes, m->dt, psi_scale_of(m, 1), psi_scale_of(m, 2)), s);
    if (rc) return rc;
    FW_CK(cudaStreamSynchronize(s));
    return FW_OK;
}

}  // namespace

namespace fwgb {
// device memory through the installed allocator, and the size of the state
// image (the checkpoint image without the step counter), for the adjoint
void *device_alloc(size_t bytes) { return dev_alloc(bytes); }
void set_thread_allocator(void *(*alloc)(size_t, void *), void (*release)(void *, void *), void *ctx)
{
    t_hook.alloc = alloc;
    t_hook.release = release;
    t_hook.ctx = ctx;
}
void device_free(void *p) { dev_free(p); }
size_t state_image_bytes(const fw_medium *m)
{
    Dims d{m->ndim, m->NX, m->NY, m->NZ, m->px, m->es, m->eps, m->wabs, m->nmech, m->plane, m->vol, m->nonlinear};
    return make_layout(d, m->n_classes).off_state_end;
}
}  // namespace fwgb

namespace fwgb {
// field pointer, element kind and read-back scale, for the staging-array read
int field_lookup(fw_medium *m, int which, int idx, void **ptr, int *kind, double *read_scale)
{
    int rc = field_ptr(m, which, idx, ptr, kind);
    if (rc) return rc;
    *read_scale = *kind == 1 ? 1.0 / psi_scale_of(m, which == FW_FIELD_PSI1 ? 1 : 2) : 1.0;
    return FW_OK;
}
}  // namespace fwgb

// ============================================================================
extern "C" {

int fw_version(void) { return 100; }

const char *fw_strerror(int code)
{
    switch (code) {
    case FW_OK: return "ok";
    case FW_ERR_ARG: return "invalid argument";
    case FW_ERR_CUDA: return "CUDA runtime error";
    case FW_ERR_NOMEM: return "out of memory";
    case FW_ERR_UNSTABLE: return "non-finite pressure (unstable run)";
    case FW_ERR_STATE: return "invalid state for this call";
    case FW_ERR_UNSUPPORTED: return "unsupported combination";
    case FW_ERR_SIZE: return "size above a fixed limit of the call";
    default: return "unknown error";
    }
}

void fw_set_allocator(void *(*alloc)(size_t, void *), void (*release_fn)(void *, void *), void *ctx)
{
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    if (alloc && release_fn) {
        g_alloc = alloc;
        g_free = release_fn;
        g_alloc_ctx = ctx;
    } else {
        g_alloc = nullptr;
        g_free = nullptr;
        g_alloc_ctx = nullptr;
    }
}

int fw_medium_bytes(const fw_grid *g, int n_mech, int storage, int nonlinear, size_t *bytes)
{
    if (!bytes) return FW_ERR_ARG;
    Dims d{};
    int rc = make_dims(g, n_mech, storage, nonlinear != 0, &d);
    if (rc) return rc;
    *bytes = make_layout(d, 65535).total;
    return FW_OK;
}

int fw_create_medium_classes(const fw_grid *g, const float *c, const float *rho, const float *beta,
                             const uint16_t *class_idx, const fw_relax_params *classes, int n_classes,
                             int storage, void *stream, fw_medium **out)
{
    if (!classes || n_classes < 1 || n_classes > 65535) return FW_ERR_ARG;
    std::vector<fw_relax_params> cl(classes, classes + n_classes);
    return create_common(g, c, rho, beta, class_idx, cl, storage, (cudaStream_t)stream, out);
}

int fw_create_medium(const fw_grid *g, const float *c, const float *rho, const float *beta,
                     const float *alpha0, const float *y, int n_mech, int storage,
                     const fw_fit_opts *opts, void *stream, fw_medium **out)
{
    if (!g || !c || !alpha0 || !y || !out) return FW_ERR_ARG;
    Dims d{};
    int rc = make_dims(g, n_mech, storage, beta != nullptr, &d);
    if (rc) return rc;
    const size_t n = (size_t)d.NX * d.NY * d.NZ;
    std::vector<float> ha, hy, hc;
    if ((rc = fetch_host(alpha0, n, ha)) || (rc = fetch_host(y, n, hy)) || (rc = fetch_host(c, n, hc))) return rc;
    // classes = distinct (alpha0, y) pairs, in order of first appearance
    std::unordered_map<unsigned long long, int> key;
    std::vector<uint16_t> idx(n);
    std::vector<std::pair<float, float>> pairs;
    std::vector<double> csum;
    std::vector<size_t> ccount;
    for (size_t i = 0; i < n; ++i) {
        if (!(ha[i] >= 0.0f) || !std::isfinite(ha[i])) return FW_ERR_ARG;
        if (ha[i] > 0.0f && !(hy[i] >= 0.4f && hy[i] <= 2.0f)) return FW_ERR_ARG;   // valid y range (abstract, Sec. 3.1)
        float yy = ha[i] > 0.0f ? hy[i] : 0.0f;
        unsigned int ua, uy;
        std::memcpy(&ua, &ha[i], 4);
        std::memcpy(&uy, &yy, 4);
        unsigned long long k = ((unsigned long long)ua << 32) | uy;
        auto it = key.find(k);
        int ci;
        if (it == key.end()) {
            if (pairs.size() >= 65535) return FW_ERR_ARG;
            ci = (int)pairs.size();
            key.emplace(k, ci);
            pairs.emplace_back(ha[i], yy);
            csum.push_back(0.0);
            ccount.push_back(0);
        } else {
            ci = it->second;
        }
        idx[i] = (uint16_t)ci;
        csum[ci] += hc[i];
        ccount[ci] += 1;
    }
    fw_fit_opts base;
    if (opts) base = *opts; else default_opts(&base);
    const bool own_c0 = !(opts && opts->c0 > 0);
    std::vector<fw_relax_params> classes(pairs.size());
    // one job per (class, weight); results selected per class
    const int nw = base.n_w;
    std::vector<FitJob> jobs(pairs.size() * nw);
    std::vector<fw_fit_opts> copts(pairs.size(), base);
    for (size_t ci = 0; ci < pairs.size(); ++ci) {
        if (own_c0) copts[ci].c0 = csum[ci] / double(ccount[ci]);
        if (pairs[ci].first > 0.0f && (rc = fit_check(pairs[ci].first, pairs[ci].second, n_mech, copts[ci]))) return rc;
    }
    parallel_for((int)jobs.size(), base.n_threads, [&](int j) {
        const int ci = j / nw, wi = j % nw;
        if (pairs[ci].first > 0.0f) jobs[j] = run_weight(pairs[ci].first, pairs[ci].second, n_mech, copts[ci], wi);
    });
    for (size_t ci = 0; ci < pairs.size(); ++ci) {
        if (pairs[ci].first == 0.0f) {
            classes[ci] = lossless_params(n_mech);
        } else {
            std::vector<FitJob> r(jobs.begin() + ci * nw, jobs.begin() + (ci + 1) * nw);
            select_fit(r, &classes[ci], nullptr);
        }
    }
    return create_common(g, c, rho, beta, idx.data(), classes, storage, (cudaStream_t)stream, out);
}

// Source/receiver pairs on one cell: the combined injection-and-recording
// kernel lets the source's thread record the receiver there (after the
// injection), so no two threads touch one cell.  Both lists are sorted.
static int upload_io_map(fw_medium *m, cudaStream_t s)
{
    const std::vector<long long> &a = m->h_src_idx, &b = m->h_rcv_idx;
    std::vector<int> sr(a.size(), -1), rs(b.size(), -1);
    for (size_t i = 0, j = 0; i < a.size() && j < b.size();) {
        if (a[i] < b[j]) ++i;
        else if (b[j] < a[i]) ++j;
        else {
            sr[i] = (int)j;
            rs[j] = (int)i;
            ++i;
            ++j;
        }
    }
    if (m->src_rcv && !sr.empty()) FW_CK(cudaMemcpyAsync(m->src_rcv, sr.data(), sr.size() * 4, cudaMemcpyHostToDevice, s));
    if (m->rcv_src && !rs.empty()) FW_CK(cudaMemcpyAsync(m->rcv_src, rs.data(), rs.size() * 4, cudaMemcpyHostToDevice, s));
    FW_CK(cudaStreamSynchronize(s));
    return FW_OK;
}

int fw_set_sources(fw_medium *m, const uint8_t *mask, const float *waveforms, int n_wave, int n_steps,
                   const int32_t *wave_of_src)
{
    if (!m || !mask || (n_wave > 0 && !waveforms) || n_wave < 0 || n_steps < 0) return FW_ERR_ARG;
    std::vector<long long> idx = mask_to_index(m, mask);
    const int ns = (int)idx.size();
    std::vector<int> wof(ns);
    if (ns > 0) {
        if (n_wave < 1 || n_steps < 1) return FW_ERR_ARG;
        for (int i = 0; i < ns; ++i) {
            int w = wave_of_src ? wave_of_src[i] : (n_wave == 1 ? 0 : i);
            if (w < 0 || w >= n_wave) return FW_ERR_ARG;
            wof[i] = w;
        }
        if (!wave_of_src && n_wave != 1 && n_wave != ns) return FW_ERR_ARG;
    }
    cudaStream_t s = m->last_stream;
    FW_CK(cudaStreamSynchronize(s));
    drop_graphs(m);
    dev_free(m->src_buf);
    m->src_buf = nullptr;
    m->src_rcv = nullptr;
    m->n_src = 0;
    m->h_src_idx.clear();
    // receivers stop pointing at the old sources before anything can fail
    if (int rc = upload_io_map(m, s)) return rc;
    if (ns == 0) return FW_OK;
    const size_t wl = (size_t)n_wave * n_steps;
    const size_t o_idx = 0, o_gain = align_up(ns * 8, 256), o_wof = o_gain + align_up((size_t)ns * m->es, 256),
                 o_map = o_wof + align_up((size_t)ns * 4, 256), o_wave = o_map + align_up((size_t)ns * 4, 256),
                 total = o_wave + align_up(wl * m->es, 256);
    m->src_buf = dev_alloc(total);
    if (!m->src_buf) return FW_ERR_NOMEM;
    char *b = static_cast<char *>(m->src_buf);
    m->src_idx = reinterpret_cast<long long *>(b + o_idx);
    m->src_gain = b + o_gain;
    m->wave_of = reinterpret_cast<int *>(b + o_wof);
    m->src_rcv = reinterpret_cast<int *>(b + o_map);
    m->waves = b + o_wave;
    // every upload is ordered on the medium's stream and complete before
    // return: later work on any other (non-blocking) stream reads these
    // arrays without waiting for the legacy stream
    std::vector<double> w64;
    FW_CK(cudaMemcpyAsync(m->src_idx, idx.data(), ns * 8, cudaMemcpyHostToDevice, s));
    FW_CK(cudaMemcpyAsync(m->wave_of, wof.data(), ns * 4, cudaMemcpyHostToDevice, s));
    if (m->es == 8) {
        w64.assign(waveforms, waveforms + wl);
        FW_CK(cudaMemcpyAsync(m->waves, w64.data(), wl * 8, cudaMemcpyHostToDevice, s));
    } else {
        FW_CK(cudaMemcpyAsync(m->waves, waveforms, wl * 4, cudaMemcpyDefault, s));
    }
    const double inv = 1.0 / std::pow(m->dx, m->ndim);
    if (m->es == 8) k_src_gain<double><<<(ns + 255) / 256, 256, 0, s>>>((double *)m->src_gain, m->src_idx, (const double *)m->kdt, inv, ns);
    else k_src_gain<float><<<(ns + 255) / 256, 256, 0, s>>>((float *)m->src_gain, m->src_idx, (const float *)m->kdt, inv, ns);
    FW_CK(cudaGetLastError());
    FW_CK(cudaStreamSynchronize(s));
    m->n_src = ns;
    m->n_wave = n_wave;
    m->wave_len = n_steps;
    m->h_src_idx = std::move(idx);
    if (int rc = upload_io_map(m, s)) return rc;
    if (m->storage == FW_STORE_F16) return set_psi_reference(m, waveforms, wl);
    return FW_OK;
}

int fw_set_receivers(fw_medium *m, const uint8_t *mask, int decim, int n_steps)
{
    if (!m || !mask || decim < 1 || n_steps < 0) return FW_ERR_ARG;
    std::vector<long long> idx = mask_to_index(m, mask);
    cudaStream_t s = m->last_stream;
    FW_CK(cudaStreamSynchronize(s));
    drop_graphs(m);
    dev_free(m->rcv_buf);
    m->rcv_buf = nullptr;
    m->rcv_src = nullptr;
    m->n_rcv = 0;
    m->n_rec = 0;
    m->h_rcv_idx.clear();
    // sources stop pointing at the old receivers before anything can fail
    if (int rc = upload_io_map(m, s)) return rc;
    const int nr = (int)idx.size();
    if (nr == 0) return FW_OK;
    const int nrec = (n_steps + decim - 1) / decim;
    const size_t o_map = align_up((size_t)nr * 8, 256), o_tr = o_map + align_up((size_t)nr * 4, 256),
                 total = o_tr + align_up((size_t)nr * std::max(nrec, 1) * m->es, 256);
    m->rcv_buf = dev_alloc(total);
    if (!m->rcv_buf) return FW_ERR_NOMEM;
    char *b = static_cast<char *>(m->rcv_buf);
    m->rcv_idx = reinterpret_cast<long long *>(b);
    m->rcv_src = reinterpret_cast<int *>(b + o_map);
    m->traces = b + o_tr;
    // ordered on the medium's stream and complete before return (see fw_set_sources)
    FW_CK(cudaMemcpyAsync(m->rcv_idx, idx.data(), nr * 8, cudaMemcpyHostToDevice, s));
    FW_CK(cudaMemsetAsync(m->traces, 0, (size_t)nr * std::max(nrec, 1) * m->es, s));
    FW_CK(cudaStreamSynchronize(s));
    m->n_rcv = nr;
    m->n_rec = nrec;
    m->decim = decim;
    m->h_rcv_idx = std::move(idx);
    return upload_io_map(m, s);
}

int fw_step(fw_medium *m, int n_steps, void *stream)
{
    if (!m || n_steps < 0) return FW_ERR_ARG;
    if (m->sticky) return m->sticky;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = enqueue_steps(m, n_steps, s);
    if (rc) return rc;
    m->step += n_steps;
    m->last_stream = s;
    return FW_OK;
}

int fw_run(fw_medium *m, int n_steps, void *stream)
{
    if (!m || n_steps < 0) return FW_ERR_ARG;
    if (m->sticky) return m->sticky;
    cudaStream_t s = (cudaStream_t)stream;
    const int chunk = 32;
    int done = 0;
    if (n_steps >= chunk) {
        Graph &gr = m->graphs[chunk];
        if (!gr.exec) {
            FW_CK(cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal));
            int rc = enqueue_steps(m, chunk, m->cap_stream);
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamEndCapture(m->cap_stream, &graph);
            if (rc || e != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                cudaGetLastError();
                return rc ? rc : FW_ERR_CUDA;
            }
            gr.graph = graph;
            FW_CK(cudaGraphInstantiate(&gr.exec, graph, 0));
        }
        for (; done + chunk <= n_steps; done += chunk) FW_CK(cudaGraphLaunch(gr.exec, s));
    }
    if (done < n_steps) {
        int rc = enqueue_steps(m, n_steps - done, s);
        if (rc) return rc;
    }
    m->step += n_steps;
    m->last_stream = s;
    return FW_OK;
}

int fw_step_timed(fw_medium *m, int n_steps, void *stream, double *ms_velocity, double *ms_pressure,
                  double *ms_io, double *ms_total, int *n_launches)
{
    if (!m || n_steps < 0) return FW_ERR_ARG;
    if (m->sticky) return m->sticky;
    cudaStream_t s = (cudaStream_t)stream;
    // all events exist before the first is recorded, so host-side creation
    // never shows up as device time
    std::vector<cudaEvent_t> ev(3 * (size_t)n_steps + 1, nullptr);
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            for (auto &x : ev) if (x) cudaEventDestroy(x);
            return FW_ERR_CUDA;
        }
    int rc = FW_OK;
    int launches = 0;
    for (int j = 0; j < n_steps && rc == FW_OK; ++j) {
        if (cudaEventRecord(ev[3 * j], s) != cudaSuccess || launch_sweep(m, s, 1) != cudaSuccess ||
            cudaEventRecord(ev[3 * j + 1], s) != cudaSuccess || launch_sweep(m, s, 2) != cudaSuccess ||
            cudaEventRecord(ev[3 * j + 2], s) != cudaSuccess || launch_io_any(m, j, s) != cudaSuccess)
            rc = FW_ERR_CUDA;
        launches += 2 + (m->n_src + m->n_rcv > 0);
    }
    if (rc == FW_OK) {
        k_advance<<<1, 1, 0, s>>>(m->d_it, n_steps);
        launches += 1;
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(ev[3 * (size_t)n_steps], s) != cudaSuccess ||
            cudaEventSynchronize(ev[3 * (size_t)n_steps]) != cudaSuccess)
            rc = FW_ERR_CUDA;
    }
    double tv = 0, tp = 0, ti = 0;
    float tot = 0;
    for (int j = 0; j < n_steps && rc == FW_OK; ++j) {
        float a = 0, b = 0, c = 0;
        cudaEventElapsedTime(&a, ev[3 * j], ev[3 * j + 1]);
        cudaEventElapsedTime(&b, ev[3 * j + 1], ev[3 * j + 2]);
        cudaEventElapsedTime(&c, ev[3 * j + 2], ev[3 * j + 3]);
        tv += a; tp += b; ti += c;
    }
    if (rc == FW_OK && n_steps > 0) cudaEventElapsedTime(&tot, ev[0], ev[3 * (size_t)n_steps]);
    for (auto &e : ev) cudaEventDestroy(e);
    if (rc) return rc;
    if (ms_velocity) *ms_velocity = tv;
    if (ms_pressure) *ms_pressure = tp;
    if (ms_io) *ms_io = ti;
    if (ms_total) *ms_total = tot;
    if (n_launches) *n_launches = launches;
    m->step += n_steps;
    m->last_stream = s;
    return FW_OK;
}

int fw_set_waveform_samples(fw_medium *m, int it0, int n, const float *samples, void *stream)
{
    if (!m || !samples || it0 < 0 || n < 0 || (m->n_src > 0 && it0 + n > m->wave_len)) return FW_ERR_ARG;
    if (m->n_src == 0 || n == 0) return FW_OK;
    if (m->es != 4) return FW_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    FW_CK(cudaMemcpy2DAsync(static_cast<float *>(m->waves) + it0, (size_t)m->wave_len * 4, samples, (size_t)n * 4,
                            (size_t)n * 4, m->n_wave, cudaMemcpyDefault, s));
    return FW_OK;
}

int fw_read_receivers_range(fw_medium *m, int col0, int ncol, void *dst, void *stream)
{
    if (!m || !dst || col0 < 0 || ncol < 0 || col0 + ncol > m->n_rec) return FW_ERR_ARG;
    if (m->n_rcv == 0 || ncol == 0) return FW_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t eb = m->es;
    FW_CK(cudaMemcpy2DAsync(dst, (size_t)ncol * eb, static_cast<char *>(m->traces) + col0 * eb,
                            (size_t)m->n_rec * eb, (size_t)ncol * eb, m->n_rcv, cudaMemcpyDefault, s));
    return FW_OK;
}

int fw_read_field(fw_medium *m, int which, int idx, void *dst, int as_f64, void *stream)
{
    if (!m || !dst) return FW_ERR_ARG;
    void *src;
    int kind;
    int rc = field_ptr(m, which, idx, &src, &kind);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)m->NX * m->NY * m->NZ;
    const size_t eb = as_f64 ? 8 : 4;
    const double scale = kind == 1 ? 1.0 / psi_scale_of(m, which == FW_FIELD_PSI1 ? 1 : 2) : 1.0;
    DevBuf tmp(n * eb);
    if (!tmp.p) return FW_ERR_NOMEM;
    if (as_f64) FW_CK(unpad_any<double>(m, src, kind, (double *)tmp.p, scale, s));
    else FW_CK(unpad_any<float>(m, src, kind, (float *)tmp.p, scale, s));
    FW_CK(cudaMemcpyAsync(dst, tmp.p, n * eb, cudaMemcpyDefault, s));
    FW_CK(cudaStreamSynchronize(s));
    return FW_OK;
}

int fw_write_field(fw_medium *m, int which, int idx, const void *src, int as_f64, void *stream)
{
    if (!m || !src) return FW_ERR_ARG;
    void *dst;
    int kind;
    int rc = field_ptr(m, which, idx, &dst, &kind);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)m->NX * m->NY * m->NZ;
    const size_t eb = as_f64 ? 8 : 4;
    const double scale = kind == 1 ? psi_scale_of(m, which == FW_FIELD_PSI1 ? 1 : 2) : 1.0;
    DevBuf tmp(n * eb);
    if (!tmp.p) return FW_ERR_NOMEM;
    FW_CK(cudaMemcpyAsync(tmp.p, src, n * eb, cudaMemcpyDefault, s));
    if (as_f64) FW_CK(pad_any<double>(m, dst, kind, (const double *)tmp.p, scale, s));
    else FW_CK(pad_any<float>(m, dst, kind, (const float *)tmp.p, scale, s));
    FW_CK(cudaStreamSynchronize(s));
    return FW_OK;
}

int fw_read_receivers(fw_medium *m, void *dst, int as_f64, void *stream)
{
    if (!m || !dst) return FW_ERR_ARG;
    if (m->n_rcv == 0) return FW_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)m->n_rcv * m->n_rec;
    const size_t eb = as_f64 ? 8 : 4;
    if ((size_t)m->es == eb) {
        FW_CK(cudaMemcpyAsync(dst, m->traces, n * eb, cudaMemcpyDefault, s));
    } else {
        DevBuf tmp(n * eb);
        if (!tmp.p) return FW_ERR_NOMEM;
        if (as_f64) k_unpad<float, double><<<grid_blocks(n), 256, 0, s>>>((double *)tmp.p, (const float *)m->traces, (int)n, 1, 1, (int)n, 1.0);
        else k_unpad<double, float><<<grid_blocks(n), 256, 0, s>>>((float *)tmp.p, (const double *)m->traces, (int)n, 1, 1, (int)n, 1.0);
        FW_CK(cudaGetLastError());
        FW_CK(cudaMemcpyAsync(dst, tmp.p, n * eb, cudaMemcpyDefault, s));
        FW_CK(cudaStreamSynchronize(s));
    }
    FW_CK(cudaStreamSynchronize(s));
    return FW_OK;
}

int fw_state_bytes(fw_medium *m, size_t *bytes)
{
    if (!m || !bytes) return FW_ERR_ARG;
    Dims d{m->ndim, m->NX, m->NY, m->NZ, m->px, m->es, m->eps, m->wabs, m->nmech, m->plane, m->vol, m->nonlinear};
    *bytes = make_layout(d, m->n_classes).off_state_end + sizeof(long long);
    return FW_OK;
}

int fw_save_state(fw_medium *m, void *dst, void *stream)
{
    size_t nb;
    if (!dst || fw_state_bytes(m, &nb)) return FW_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    FW_CK(cudaStreamSynchronize(m->last_stream));
    FW_CK(cudaMemcpyAsync(dst, m->slab, nb - sizeof(long long), cudaMemcpyDefault, s));
    FW_CK(cudaMemcpyAsync(static_cast<char *>(dst) + nb - sizeof(long long), &m->step, sizeof(long long),
                          cudaMemcpyDefault, s));
    FW_CK(cudaStreamSynchronize(s));
    return FW_OK;
}

int fw_load_state(fw_medium *m, const void *src, void *stream)
{
    size_t nb;
    if (!src || fw_state_bytes(m, &nb)) return FW_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    FW_CK(cudaStreamSynchronize(m->last_stream));
    FW_CK(cudaMemcpyAsync(m->slab, src, nb - sizeof(long long), cudaMemcpyDefault, s));
    long long st = 0;
    FW_CK(cudaMemcpyAsync(&st, static_cast<const char *>(src) + nb - sizeof(long long), sizeof(long long),
                          cudaMemcpyDefault, s));
    FW_CK(cudaStreamSynchronize(s));
    m->step = st;
    m->sticky = 0;
    return FW_OK;
}

int fw_status(fw_medium *m, float *max_abs_p)
{
    if (!m) return FW_ERR_ARG;
    FW_CK(cudaStreamSynchronize(m->last_stream));
    Monitor h{};
    FW_CK(cudaMemcpy(&h, m->mon, sizeof(Monitor), cudaMemcpyDeviceToHost));
    if (max_abs_p) std::memcpy(max_abs_p, &h.max_bits, 4);
    if (h.nonfinite) m->sticky = FW_ERR_UNSTABLE;
    if (h.bad_index) m->sticky = FW_ERR_STATE;
    return m->sticky;
}

int fw_medium_get_info(fw_medium *m, fw_medium_info *info)
{
    if (!m || !info) return FW_ERR_ARG;
    *info = fw_medium_info{};
    info->ndim = m->ndim;
    info->nx = m->g.nx;
    info->ny = m->g.ny;
    info->nz = m->g.nz;
    info->n_mech = m->nmech;
    info->storage = m->storage;
    info->n_classes = m->n_classes;
    info->nonlinear = m->nonlinear ? 1 : 0;
    info->dx = m->dx;
    info->dt = m->dt;
    info->c_max = m->c_max;
    info->ceff_max = m->ceff_max;
    info->device_bytes = m->slab_bytes;
    info->step = m->step;
    info->n_src = m->n_src;
    info->n_rcv = m->n_rcv;
    info->n_rec = m->n_rec;
    info->time_order = m->time_order;
    return FW_OK;
}

void fw_destroy_medium(fw_medium *m)
{
    if (!m) return;
    cudaStreamSynchronize(m->last_stream);
    release(m);
}

}  // extern "C"
