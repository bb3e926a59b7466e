// Fused staggered-grid FDTD kernels for sm_103a (Sec. 2.1, Sec. 3.3).
//
// One time step is two z-marching sweeps over the grid:
//   velocity sweep : g_d = D+_d p (8th order), memory variables of the
//                    gradient side, absorbing-layer mechanism, v_d update;
//   pressure sweep : q_d = D-_d v_d, memory variables of the divergence side
//                    (summed over directions, exact because their
//                    coefficients do not depend on d), absorbing-layer
//                    mechanism per direction, p update (with the optional
//                    nonlinear factor), stability monitor.
// Every field is read once and written once per sweep from HBM: each thread
// owns 4 consecutive x points of one (x, y) column and walks the depth axis;
// the depth-direction taps come from a register queue of 8 planes, the x and
// y taps from a double-buffered shared-memory plane tile with halos.  The
// next plane of every stream is staged in shared memory while the current
// one is computed: by TMA tile copies completed on an mbarrier in the 3D
// FP32-state instances (one thread issues one box per stream), by per-thread
// cp.async copies otherwise.  Stores are 128-bit (FP32) and coalesced.
//
// Memory-variable update (Eq. relaxation_psi, midpoint time index): with the
// derivative g of the current half step, psi_new = b psi_old + a g, and the
// stretched derivative is g/kappa + sum (psi_old + psi_new)/2
//   = g * ceff + sum hb * psi_old,   ceff = 1/kappa + sum a/2,  hb = (1+b)/2,
// with a, b of Eqs. relaxation_a/b from the class table.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fw_internal.h"

namespace fwgb {

constexpr int kMaxMech = FW_MAX_MECH;

// ---------------------------------------------------------------------------
// 4-element vector access in the storage type S, arithmetic in R

template <typename S> struct Io;

template <> struct Io<float> {
    template <typename R> static __device__ __forceinline__ void ld(const float *p, R (&v)[4])
    {
        float4 t = __ldcs(reinterpret_cast<const float4 *>(p));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
    template <typename R> static __device__ __forceinline__ void ldg(const float *p, R (&v)[4])
    {
        float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
    template <typename R> static __device__ __forceinline__ void st(float *p, const R (&v)[4])
    {
        __stcs(reinterpret_cast<float4 *>(p), make_float4(float(v[0]), float(v[1]), float(v[2]), float(v[3])));
    }
    static __device__ __forceinline__ float ld1(const float *p) { return *p; }
    static __device__ __forceinline__ void st1(float *p, float v) { *p = v; }
};

template <> struct Io<double> {
    template <typename R> static __device__ __forceinline__ void ld(const double *p, R (&v)[4])
    {
        double2 a = __ldcs(reinterpret_cast<const double2 *>(p));
        double2 b = __ldcs(reinterpret_cast<const double2 *>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    template <typename R> static __device__ __forceinline__ void ldg(const double *p, R (&v)[4])
    {
        double2 a = __ldg(reinterpret_cast<const double2 *>(p));
        double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    template <typename R> static __device__ __forceinline__ void st(double *p, const R (&v)[4])
    {
        __stcs(reinterpret_cast<double2 *>(p), make_double2(v[0], v[1]));
        __stcs(reinterpret_cast<double2 *>(p) + 1, make_double2(v[2], v[3]));
    }
    static __device__ __forceinline__ double ld1(const double *p) { return *p; }
    static __device__ __forceinline__ void st1(double *p, double v) { *p = v; }
};

template <> struct Io<__nv_bfloat16> {
    template <typename R> static __device__ __forceinline__ void ld(const __nv_bfloat16 *p, R (&v)[4])
    {
        uint2 t = __ldcs(reinterpret_cast<const uint2 *>(p));
        float2 a = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&t.x));
        float2 b = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&t.y));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    template <typename R> static __device__ __forceinline__ void st(__nv_bfloat16 *p, const R (&v)[4])
    {
        __nv_bfloat162 a = __floats2bfloat162_rn(float(v[0]), float(v[1]));
        __nv_bfloat162 b = __floats2bfloat162_rn(float(v[2]), float(v[3]));
        uint2 t;
        t.x = *reinterpret_cast<unsigned int *>(&a);
        t.y = *reinterpret_cast<unsigned int *>(&b);
        __stcs(reinterpret_cast<uint2 *>(p), t);
    }
};

template <> struct Io<__half> {
    template <typename R> static __device__ __forceinline__ void ld(const __half *p, R (&v)[4])
    {
        uint2 t = __ldcs(reinterpret_cast<const uint2 *>(p));
        float2 a = __half22float2(*reinterpret_cast<__half2 *>(&t.x));
        float2 b = __half22float2(*reinterpret_cast<__half2 *>(&t.y));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    template <typename R> static __device__ __forceinline__ void st(__half *p, const R (&v)[4])
    {
        __half2 a = __floats2half2_rn(float(v[0]), float(v[1]));
        __half2 b = __floats2half2_rn(float(v[2]), float(v[3]));
        uint2 t;
        t.x = *reinterpret_cast<unsigned int *>(&a);
        t.y = *reinterpret_cast<unsigned int *>(&b);
        __stcs(reinterpret_cast<uint2 *>(p), t);
    }
};

template <typename R> __device__ __forceinline__ void lut4(const R *lut, int c, int off, R (&v)[4]);
template <> __device__ __forceinline__ void lut4<float>(const float *lut, int c, int off, float (&v)[4])
{
    float4 t = __ldg(reinterpret_cast<const float4 *>(lut + (size_t)c * kLutStride + off));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
template <> __device__ __forceinline__ void lut4<double>(const double *lut, int c, int off, double (&v)[4])
{
    const double2 *q = reinterpret_cast<const double2 *>(lut + (size_t)c * kLutStride + off);
    double2 a = __ldg(q), b = __ldg(q + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

__device__ __forceinline__ float fw_exp(float x) { return expf(x); }
__device__ __forceinline__ float fw_rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double fw_rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ double fw_exp(double x) { return exp(x); }

// Absorbing-layer mechanism coefficients (Eqs. relaxation_a/b with the
// profile d, alpha at this point and the point's tissue kappa).
template <typename R>
__device__ __forceinline__ void pml_ab(R d, R al, R kappa, R dt, R &a, R &b)
{
    b = fw_exp(-(d / kappa + al) * dt);
    a = d / (kappa * (d + kappa * al)) * (b - R(1));
}

// ---------------------------------------------------------------------------
// asynchronous global -> shared copies (cp.async, zero fill when !ok)

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

template <int BYTES>
__device__ __forceinline__ void cp_async(void *sdst, const void *gsrc, bool ok)
{
    const unsigned d = smem_u32(sdst);
    const int n = ok ? BYTES : 0;
    if (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc), "r"(n) : "memory");
    else if (BYTES == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(gsrc), "r"(n) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(gsrc), "r"(n) : "memory");
}

__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N> __device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// copy the 4 consecutive elements of type S at gsrc (16 or 8 bytes, or two
// 16-byte pieces for double)
template <typename S>
__device__ __forceinline__ void cp_async4(S *sdst, const S *gsrc, bool ok)
{
    if (sizeof(S) == 4) cp_async<16>(sdst, gsrc, ok);
    else if (sizeof(S) == 2) cp_async<8>(sdst, gsrc, ok);
    else { cp_async<16>(sdst, gsrc, ok); cp_async<16>(sdst + 2, gsrc + 2, ok); }
}

// ---------------------------------------------------------------------------
// tensor-memory-access (TMA) tile copies completed on an mbarrier

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make the barrier initialisation visible to the asynchronous (copy) proxy
__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Wait for the phase `parity` of bar with a bound on the number of polls;
// false when the bound was reached (the caller records a timeout).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity)
{
    for (unsigned it = 0; it < (1u << 22); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// order this thread's earlier generic-proxy accesses of shared memory before
// later asynchronous-proxy writes to it (a buffer refilled by TMA)
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// 3D tiled copy of the box at (x, y, z) of the tensor described by map into
// shared memory at dst (128-byte aligned); x * element size is a multiple of
// 16 bytes; elements outside the tensor read as zero
__device__ __forceinline__ void tma_load_3d(void *dst, const TensorMapBlob *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_u32(dst)),
                 "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
                 : "memory");
}

// 4 consecutive elements of type S from shared memory, as R
template <typename S> struct Sm;
template <> struct Sm<float> {
    template <typename R> static __device__ __forceinline__ void ld(const float *p, R (&v)[4])
    {
        float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
};
template <> struct Sm<double> {
    template <typename R> static __device__ __forceinline__ void ld(const double *p, R (&v)[4])
    {
        double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
};
template <> struct Sm<__nv_bfloat16> {
    template <typename R> static __device__ __forceinline__ void ld(const __nv_bfloat16 *p, R (&v)[4])
    {
        uint2 t = *reinterpret_cast<const uint2 *>(p);
        float2 a = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&t.x));
        float2 b = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&t.y));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
};
template <> struct Sm<__half> {
    template <typename R> static __device__ __forceinline__ void ld(const __half *p, R (&v)[4])
    {
        uint2 t = *reinterpret_cast<const uint2 *>(p);
        float2 a = __half22float2(*reinterpret_cast<__half2 *>(&t.x));
        float2 b = __half22float2(*reinterpret_cast<__half2 *>(&t.y));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
};

// ---------------------------------------------------------------------------
// launch parameters

template <typename R> struct Geo {
    int nx, ny, nz;      // kernel axes (ny = 1 in 2D)
    int px;              // row pitch (elements), multiple of 32
    long long plane;     // px * ny
    int zseg;            // depth planes per CTA
    int wabs;            // absorbing width in cells (0: none)
    R c1, c2, c3, c4;    // stencil weights / dx
    R dt;
    R lr;                // length [cells] of the tissue-mechanism ramp in the layer
    // time-space stencil (Sec. 3.3, Tan & Huang 2014): per-cell weights
    // a_m = sum_n ta[m][n] r2^n (divided by dx) and cross weight b = r2 tb,
    // r2 = (c dt / dx)^2 = (K dt) r2s / rho
    R ta[4][4];
    R tb, r2s;
};

// Tissue mechanisms in the absorbing layer (two-stage layer, Sec. 4.6 /
// Sec. 5.4): the strength of every tissue mechanism of a cell at depth s
// into the layer (cells, largest over the axes, at the cell centre) is
// r = 1 - (s/L_r)^2 for s < L_r, 0 beyond, at a fixed relaxation rate:
// a -> r a, b unchanged, so ceff -> 1/kappa + r (ceff - 1/kappa).
template <typename R>
__device__ __forceinline__ R layer_depth(int c, int n, int w)
{
    if (n <= 1 || w <= 0) return R(0);
    return fmax(R(0), fmax(R(w) - R(0.5) - R(c), R(c) - (R(n - w) - R(0.5))));
}

template <typename R>
__device__ __forceinline__ R ramp_of(R s, R inv_lr)   // s >= 0; exactly 1 at s = 0
{
    const R q = fmin(s * inv_lr, R(1));
    return R(1) - q * q;
}

template <typename R, typename SS, typename SP> struct VelArgs {
    Geo<R> g;
    const SS *p;
    SS *v[3];
    SP *psi[kMaxMech][3];
    SS *psip[3];                 // absorbing mechanism memory per axis, or null
    const SS *rho;
    const uint16_t *cls;
    const R *lut;
    const R *pd[3], *pa[3];      // absorbing profile at half points per axis
    const SS *kdt;               // K dt per voxel (time-space stencil only)
    Monitor *mon;                // failure record (a staged-copy wait that gave up)
    long long wofs;              // bytes from each state array read to where it is written
                                 // (0: in place; per-thread staging only)
    VelMaps maps;                // tensor maps of the staged streams (TMA staging only)
};

template <typename R, typename SS, typename SP> struct PresArgs {
    Geo<R> g;
    SS *p;
    const SS *v[3];
    SP *psi[kMaxMech];
    SS *psip[3];
    const SS *kdt;               // K dt per voxel
    const SS *b2dt;              // 2 beta dt per voxel, or null (linear)
    const uint16_t *cls;
    const R *lut;
    const R *pd[3], *pa[3];      // absorbing profile at integer points per axis
    Monitor *mon;
    const SS *rho;               // density per voxel (time-space stencil only)
    long long wofs;              // as VelArgs::wofs
    PresMaps maps;               // tensor maps of the staged streams (TMA staging only)
};

// Where a sweep stores a state array it read at p: wofs bytes further on for
// a step from one state image into another (the adjoint's recomputation),
// p itself for the in-place step.
template <typename T> __device__ __forceinline__ T *wr_at(T *p, long long wofs)
{
    return reinterpret_cast<T *>(reinterpret_cast<char *>(p) + wofs);
}

template <typename SS, typename R>
__device__ __forceinline__ void ld4_or_zero(const SS *base, bool ok, R (&v)[4])
{
    if (ok) Io<SS>::ldg(base, v);
    else v[0] = v[1] = v[2] = v[3] = R(0);
}

// ---------------------------------------------------------------------------
// shared-memory layout of the sweeps (dynamic shared memory)
//
// Each sweep keeps two stages: while plane k is computed from stage k&1,
// cp.async copies of plane k+1 fill stage (k+1)&1, so one plane of every
// stream is always in flight.  A stage holds, per stream, the CTA tile
// [BY][4*BX] in the storage type; the derivative tiles (with halos) are
// double-buffered by plane parity as well.

template <typename R, typename SS, typename SP, int DIM, int NM, int BX, int BY, bool TS = false, bool TMA = false>
struct VelSmem {
    static constexpr int TW = 4 * BX, SW = TW + 8, SH = DIM == 3 ? BY + 7 : BY, RO = DIM == 3 ? 3 : 0;
    // per-axis tiles: one slot per axis of the grid (2D: x in slot 0, depth in slot 1)
    static constexpr int NAX = DIM == 3 ? 3 : 2;
    static __host__ __device__ constexpr int slot(int ax) { return DIM == 3 ? ax : (ax == 2 ? 1 : ax); }
    static constexpr size_t TILE = (size_t)BY * TW;
    // per stage (bytes, 16-aligned pieces)
    static constexpr size_t o_v = 0;
    static constexpr size_t o_psi = o_v + NAX * TILE * sizeof(SS);
    static constexpr size_t o_pn = o_psi + (size_t)NM * NAX * TILE * sizeof(SP);
    static constexpr size_t o_rn = o_pn + TILE * sizeof(SS);
    static constexpr size_t o_cls = o_rn + TILE * sizeof(SS);
    static constexpr size_t o_pml = o_cls + (TILE * 2 + 15) / 16 * 16;     // absorbing-layer psi per axis
    static constexpr size_t o_kv = o_pml + NAX * TILE * sizeof(SS);        // K dt of plane k (time-space only)
    static constexpr size_t stage = (o_kv + (TS ? TILE * sizeof(SS) : 0) + 127) / 128 * 128;
    // derivative tiles of p (x/y halos) and rho (+1 halos), two each; every
    // buffer starts on 128 bytes (TMA destinations)
    static constexpr size_t sp_stride = ((size_t)SH * SW * sizeof(R) + 127) / 128 * 128;
    static constexpr size_t sr_stride = ((size_t)(BY + 1) * (TW + 4) * sizeof(R) + 127) / 128 * 128;
    static constexpr size_t o_sp = 2 * stage;
    static constexpr size_t o_sr = o_sp + 2 * sp_stride;
    // two mbarriers (TMA staging) in the padding after the second rho tile,
    // which its copies do not reach: the layout's size is that of the
    // cp.async variant, so both fit the same number of CTAs per SM
    static constexpr size_t o_bar = o_sr + sr_stride + ((size_t)(BY + 1) * (TW + 4) * sizeof(R) + 7) / 8 * 8;
    static_assert(o_bar + 16 <= o_sr + 2 * sr_stride, "no room for the barriers in the rho tile padding");
    static constexpr size_t bytes = o_sr + 2 * sr_stride;
    // bytes the TMA copies of one plane deliver (completion count of its barrier)
    static constexpr unsigned tma_bytes =
        (unsigned)(((size_t)SH * SW + (size_t)(BY + 1) * (TW + 4)) * sizeof(SS) +
                   TILE * (5 + (TS ? 1 : 0)) * sizeof(SS) + (size_t)NM * NAX * TILE * sizeof(SP) + TILE * 2);
};

template <typename R, typename SS, typename SP, int DIM, int NM, int BX, int BY, bool TS = false, bool TMA = false>
struct PresSmem {
    static constexpr int TW = 4 * BX, SWX = TW + 8, SHY = DIM == 3 ? BY + 7 : 1;
    static constexpr int NAX = DIM == 3 ? 3 : 2;   // absorbing-layer tiles: one slot per axis of the grid
    static __host__ __device__ constexpr int slot(int ax) { return DIM == 3 ? ax : (ax == 2 ? 1 : ax); }
    static constexpr size_t TILE = (size_t)BY * TW;
    static constexpr size_t o_qn = 0;
    static constexpr size_t o_p = o_qn + TILE * sizeof(SS);
    static constexpr size_t o_kd = o_p + TILE * sizeof(SS);
    static constexpr size_t o_bd = o_kd + TILE * sizeof(SS);
    static constexpr size_t o_psi = o_bd + TILE * sizeof(SS);
    static constexpr size_t o_cls = o_psi + (size_t)NM * TILE * sizeof(SP);
    static constexpr size_t o_pml = o_cls + (TILE * 2 + 15) / 16 * 16;
    static constexpr size_t o_rh = o_pml + NAX * TILE * sizeof(SS);        // rho of plane k (time-space only)
    static constexpr size_t stage = (o_rh + (TS ? TILE * sizeof(SS) : 0) + 127) / 128 * 128;
    // v_x (x halo) and v_y (y halo) tiles, two each, on 128-byte boundaries
    // (the time-space stencil with TMA staging uses the rings below instead)
    static constexpr bool RINGS = TS && TMA;
    static constexpr size_t svx_stride = RINGS ? 0 : ((size_t)BY * SWX * sizeof(R) + 127) / 128 * 128;
    static constexpr size_t svy_stride = RINGS ? 0 : ((size_t)SHY * TW * sizeof(R) + 127) / 128 * 128;
    static constexpr size_t o_svx = 2 * stage;
    static constexpr size_t o_svy = o_svx + 2 * svx_stride;
    // time-space stencil, TMA staging: rings of four planes (k-1, k, k+1 in
    // use, k+2 landing) of v_x, v_y, v_z with x halos of 4 columns and y
    // halos of 1 row (v_x, v_z: rows y-1 .. y+BY) or 4 below / 3 above (v_y)
    static constexpr int RXH = BY + 2, RYH = BY + 7;
    static constexpr size_t rx_stride = RINGS ? ((size_t)RXH * SWX * sizeof(R) + 127) / 128 * 128 : 0;
    static constexpr size_t ry_stride = RINGS ? ((size_t)RYH * SWX * sizeof(R) + 127) / 128 * 128 : 0;
    static constexpr size_t o_rx = o_svy + 2 * svy_stride;
    static constexpr size_t o_ry = o_rx + 4 * rx_stride;
    static constexpr size_t o_rz = o_ry + 4 * ry_stride;
    static constexpr unsigned ring_bytes = (unsigned)(((size_t)2 * RXH + RYH) * SWX * sizeof(SS));
    static constexpr size_t o_bar = o_rz + 4 * rx_stride;                   // mbarriers (TMA staging)
    static constexpr size_t bytes = o_bar + (TMA ? (RINGS ? 48 : 16) : 0);
};

// ---------------------------------------------------------------------------
// velocity sweep

// TMA staging of plane k (3D): one thread arms the stage's barrier with the
// byte count and issues one tile copy per stream; the copies of the p tile
// (x/y halos and corners included) and of the rho tile (+1 halos) land in
// the derivative buffers of parity k&1
template <typename R, typename SS, typename SP, int NM, int BX, int BY, bool TS>
__device__ __forceinline__ void vel_issue_tma(const VelArgs<R, SS, SP> &A, unsigned char *sm, int k, int xb, int yb)
{
    using L = VelSmem<R, SS, SP, 3, NM, BX, BY, TS, true>;
    unsigned char *st = sm + (k & 1) * L::stage;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + L::o_bar) + (k & 1);
    fence_proxy_async_smem();
    mbar_expect_tx(bar, L::tma_bytes);
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        tma_load_3d(st + L::o_v + L::slot(ax) * L::TILE * sizeof(SS), &A.maps.v[ax], xb, yb, k, bar);
#pragma unroll
        for (int m = 0; m < NM; ++m)
            tma_load_3d(st + L::o_psi + (m * L::NAX + L::slot(ax)) * L::TILE * sizeof(SP), &A.maps.psi[m][ax], xb, yb, k, bar);
    }
    tma_load_3d(st + L::o_pn, &A.maps.p_own, xb, yb, k + 4, bar);
    tma_load_3d(st + L::o_rn, &A.maps.rho_own, xb, yb, k + 1, bar);
    tma_load_3d(st + L::o_cls, &A.maps.cls, xb, yb, k, bar);
    if (TS) tma_load_3d(st + L::o_kv, &A.maps.kdt, xb, yb, k, bar);
    tma_load_3d(sm + L::o_sp + (k & 1) * L::sp_stride, &A.maps.p_halo, xb - 4, yb - L::RO, k, bar);
    tma_load_3d(sm + L::o_sr + (k & 1) * L::sr_stride, &A.maps.rho_halo, xb, yb, k, bar);
}

template <typename R, typename SS, typename SP, int DIM, int NM, int BX, int BY, bool TS, bool TMA>
__device__ __forceinline__ void vel_issue(const VelArgs<R, SS, SP> &A, unsigned char *sm, int k, int x0, int y,
                                          int xb, int yb, long long row, bool hd)
{
    using L = VelSmem<R, SS, SP, DIM, NM, BX, BY, TS, TMA>;
    const Geo<R> &G = A.g;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const long long pk = (long long)k * G.plane;
    unsigned char *st = sm + (k & 1) * L::stage;
    const int e0 = ty * L::TW + 4 * tx;       // this thread's element offset in a stage tile
    if (TMA) {
        if (tx == 0 && ty == 0) vel_issue_tma<R, SS, SP, NM, BX, BY, TS>(A, sm, k, xb, yb);
        // absorbing-layer memory: per thread, where this thread needs it
        if (G.wabs > 0 && hd) {
            const bool in[3] = {x0 < G.wabs || x0 + 3 >= G.nx - G.wabs, y < G.wabs || y >= G.ny - G.wabs,
                                k < G.wabs || k >= G.nz - G.wabs};
#pragma unroll
            for (int ax = 0; ax < 3; ++ax)
                if (in[ax]) cp_async4(reinterpret_cast<SS *>(st + L::o_pml) + L::slot(ax) * L::TILE + e0, A.psip[ax] + pk + row, true);
        }
        return;
    }
    const SS *gz = A.p;                       // any valid address for zero-fill copies
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        if (DIM == 2 && ax == 1) continue;
        cp_async4(reinterpret_cast<SS *>(st + L::o_v) + L::slot(ax) * L::TILE + e0, hd ? A.v[ax] + pk + row : gz, hd);
#pragma unroll
        for (int m = 0; m < NM; ++m)
            cp_async4(reinterpret_cast<SP *>(st + L::o_psi) + (m * L::NAX + L::slot(ax)) * L::TILE + e0,
                      hd ? A.psi[m][ax] + pk + row : reinterpret_cast<const SP *>(gz), hd);
    }
    {
        const bool ok = hd && k + 4 < G.nz;
        cp_async4(reinterpret_cast<SS *>(st + L::o_pn) + e0, ok ? A.p + pk + 4 * G.plane + row : gz, ok);
        const bool okr = hd && k + 1 < G.nz;
        cp_async4(reinterpret_cast<SS *>(st + L::o_rn) + e0, okr ? A.rho + pk + G.plane + row : gz, okr);
        cp_async<8>(reinterpret_cast<uint16_t *>(st + L::o_cls) + e0, hd ? (const void *)(A.cls + pk + row) : (const void *)gz, hd);
        if (TS) cp_async4(reinterpret_cast<SS *>(st + L::o_kv) + e0, hd ? A.kdt + pk + row : gz, hd);
    }
    if (G.wabs > 0 && hd) {                   // absorbing-layer memory where this thread needs it
        const bool in[3] = {x0 < G.wabs || x0 + 3 >= G.nx - G.wabs, DIM == 3 && (y < G.wabs || y >= G.ny - G.wabs),
                            k < G.wabs || k >= G.nz - G.wabs};
#pragma unroll
        for (int ax = 0; ax < 3; ++ax)
            if (in[ax]) cp_async4(reinterpret_cast<SS *>(st + L::o_pml) + L::slot(ax) * L::TILE + e0, A.psip[ax] + pk + row, true);
    }
    // halos of plane k straight into the derivative tiles of parity k&1
    R *sp = reinterpret_cast<R *>(sm + L::o_sp + (k & 1) * L::sp_stride);
    R *sr = reinterpret_cast<R *>(sm + L::o_sr + (k & 1) * L::sr_stride);
    if (tx == 0) {
        const bool ok = y < G.ny && x0 - 4 >= 0;
        cp_async4(reinterpret_cast<SS *>(sp + (L::RO + ty) * L::SW), ok ? A.p + pk + (long long)y * G.px + (x0 - 4) : gz, ok);
    }
    if (tx == BX - 1) {
        const bool ok = y < G.ny && x0 + 4 < G.px;
        cp_async4(reinterpret_cast<SS *>(sp + (L::RO + ty) * L::SW + L::TW + 4),
                  ok ? A.p + pk + (long long)y * G.px + (x0 + 4) : gz, ok);
        const bool okr = y < G.ny && xb + L::TW < G.nx;
        cp_async<sizeof(SS)>(reinterpret_cast<SS *>(sr + ty * (L::TW + 4) + L::TW),
                             okr ? A.rho + pk + (long long)y * G.px + xb + L::TW : gz, okr);
    }
    if (DIM == 3) {
        for (int r = ty; r < 7; r += BY) {      // 3 halo rows below the tile, 4 above
            const int yy = r < 3 ? yb - 3 + r : yb + BY + (r - 3);
            const int hrow = r < 3 ? r : BY + 3 + (r - 3);
            const bool ok = yy >= 0 && yy < G.ny && x0 < G.px;
            cp_async4(reinterpret_cast<SS *>(sp + hrow * L::SW + 4 + 4 * tx), ok ? A.p + pk + (long long)yy * G.px + x0 : gz, ok);
        }
    }
    if (DIM == 3 && ty == 0) {
        const bool ok = yb + BY < G.ny && x0 < G.px;
        cp_async4(reinterpret_cast<SS *>(sr + BY * (L::TW + 4) + 4 * tx), ok ? A.rho + pk + (long long)(yb + BY) * G.px + x0 : gz, ok);
    }
    // time-space stencil: the x halos of the nearest halo row on either side
    // of the tile (the cross terms reach the corner cells of rows y -+ 1)
    if (TS && DIM == 3 && ty < 2 && (tx == 0 || tx == BX - 1)) {
        const int yy = ty == 0 ? yb - 1 : yb + BY;
        const int hrow = ty == 0 ? L::RO - 1 : L::RO + BY;
        const int xc = tx == 0 ? x0 - 4 : x0 + 4;
        const bool ok = yy >= 0 && yy < G.ny && xc >= 0 && xc < G.px;
        cp_async4(reinterpret_cast<SS *>(sp + hrow * L::SW + (tx == 0 ? 0 : L::TW + 4)),
                  ok ? A.p + pk + (long long)yy * G.px + xc : gz, ok);
    }
}

// scalar / 4-vector read-only loads of a field that the running sweep does
// not write, zero outside the grid (ok false)
template <typename SS, typename R>
__device__ __forceinline__ R ldz1(const SS *p, bool ok)
{
    return ok ? R(__ldg(p)) : R(0);
}

// Courant-number dependent weights of the time-space stencil for one cell:
// a[m] = sum_n ta[m][n] r2^n (Horner), b = r2 tb
template <typename R>
__device__ __forceinline__ void ts_weights(const Geo<R> &G, R r2, R (&a)[4], R &b)
{
#pragma unroll
    for (int m = 0; m < 4; ++m) a[m] = ((G.ta[m][3] * r2 + G.ta[m][2]) * r2 + G.ta[m][1]) * r2 + G.ta[m][0];
    b = r2 * G.tb;
}

// Gradient of p at the three faces of this thread's four cells with the
// time-space stencil (Sec. 3.3, after Tan & Huang 2014): per cell the
// on-axis weights a_m(r) and the cross weight b(r), r^2 = (K dt) dt /
// (rho dx^2); the cross term along d is the sum, over the other axes e and
// s = -+1, of the two-point difference along d at the neighbour s along e.
// Plane k (with x/y halos and the corners of rows y -+ 1) comes from the
// tile sp, the own columns of planes k -+ 1 from the register queue q, and
// the few values of planes k -+ 1 off this thread's columns from the
// read-only cache (p is not written by this sweep).
template <typename R, typename SS, typename SP, int DIM, int NM, int BX, int BY>
__device__ __forceinline__ void vel_gradient_ts(const VelArgs<R, SS, SP> &A, const unsigned char *st, const R *sp0,
                                                const R (&q)[8][4], const R (&rho)[4], int k, int x0, int y,
                                                int e0, R (&g)[3][4])
{
    using L = VelSmem<R, SS, SP, DIM, NM, BX, BY, true>;
    constexpr int SW = L::SW, RO = L::RO;
    const Geo<R> &G = A.g;
    const int tx = threadIdx.x, ty = threadIdx.y;
    R kd[4];
    Sm<SS>::ld(reinterpret_cast<const SS *>(st + L::o_kv) + e0, kd);
    // row y of plane k, columns x0-4 .. x0+7
    R w[12];
    {
        const R *s = sp0 + (RO + ty) * SW + 4 * tx;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            R a4[4];
            Sm<R>::ld(s + 4 * q, a4);
#pragma unroll
            for (int i = 0; i < 4; ++i) w[4 * q + i] = a4[i];
        }
    }
    const long long rowk = (long long)y * G.px;
    const bool okm = k >= 1, okp = k + 1 < G.nz;
    // column x0+4 of planes k-1, k+1 and column x0-1 of plane k+1 (row y)
    const R pm4 = ldz1<SS, R>(A.p + (long long)(k - 1) * G.plane + rowk + x0 + 4, okm && x0 + 4 < G.px);
    const R pp4 = ldz1<SS, R>(A.p + (long long)(k + 1) * G.plane + rowk + x0 + 4, okp && x0 + 4 < G.px);
    const R ppm1 = ldz1<SS, R>(A.p + (long long)(k + 1) * G.plane + rowk + x0 - 1, okp && x0 >= 1);
    R X[3][4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const R qm1 = e < 3 ? q[2][e + 1] : pm4, qp1 = e < 3 ? q[4][e + 1] : pp4;
        const R pl = e > 0 ? q[4][e - 1] : ppm1;          // plane k+1, column x-1
        X[0][e] = (qm1 - q[2][e]) + (qp1 - q[4][e]);
        X[2][e] = (pl - w[e + 3]) + (qp1 - w[e + 5]);
        X[1][e] = R(0);
    }
    if (DIM == 3) {
        R um[5], up[6];                                   // rows y-1 (x0..x0+4), y+1 (x0-1..x0+4) of plane k
        {
            const R *s = sp0 + (RO + ty - 1) * SW + 4 + 4 * tx;
            R a4[4];
            Sm<R>::ld(s, a4);
#pragma unroll
            for (int i = 0; i < 4; ++i) um[i] = a4[i];
            um[4] = s[4];
            const R *t = sp0 + (RO + ty + 1) * SW + 4 + 4 * tx;
            Sm<R>::ld(t, a4);
#pragma unroll
            for (int i = 0; i < 4; ++i) up[i + 1] = a4[i];
            up[0] = t[-1];
            up[5] = t[4];
        }
        R a1m[4], a1p[4], am1p[4];                        // rows y+1 of planes k-1, k+1; row y-1 of plane k+1
        const bool oy1 = y + 1 < G.ny, oym = y >= 1;
        ld4_or_zero(A.p + (long long)(k - 1) * G.plane + rowk + G.px + x0, okm && oy1, a1m);
        ld4_or_zero(A.p + (long long)(k + 1) * G.plane + rowk + G.px + x0, okp && oy1, a1p);
        ld4_or_zero(A.p + (long long)(k + 1) * G.plane + rowk - G.px + x0, okp && oym, am1p);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            X[0][e] += (um[e + 1] - um[e]) + (up[e + 2] - up[e + 1]);
            X[1][e] = (up[e] - w[e + 3]) + (up[e + 2] - w[e + 5]) + (a1m[e] - q[2][e]) + (a1p[e] - q[4][e]);
            X[2][e] += (am1p[e] - um[e]) + (a1p[e] - up[e + 1]);
        }
    }
    // y taps: rows y-3 .. y+4 of plane k, this thread's four columns
    R cy[8][4];
    if (DIM == 3)
#pragma unroll
        for (int r = 0; r < 8; ++r) Sm<R>::ld(sp0 + (RO + ty - 3 + r) * SW + 4 + 4 * tx, cy[r]);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const bool live = x0 + e < G.nx;
        const R r2 = live ? kd[e] * G.r2s * fw_rcp(rho[e]) : R(0);
        R a[4], b;
        ts_weights(G, r2, a, b);
        g[0][e] = a[0] * (w[e + 5] - w[e + 4]) + a[1] * (w[e + 6] - w[e + 3]) + a[2] * (w[e + 7] - w[e + 2]) +
                  a[3] * (w[e + 8] - w[e + 1]) + b * X[0][e];
        if (DIM == 3)
            g[1][e] = a[0] * (cy[4][e] - cy[3][e]) + a[1] * (cy[5][e] - cy[2][e]) + a[2] * (cy[6][e] - cy[1][e]) +
                      a[3] * (cy[7][e] - cy[0][e]) + b * X[1][e];
        g[2][e] = a[0] * (q[4][e] - q[3][e]) + a[1] * (q[5][e] - q[2][e]) + a[2] * (q[6][e] - q[1][e]) +
                  a[3] * (q[7][e] - q[0][e]) + b * X[2][e];
    }
}

// 3D: 32-bit memory variables fill shared memory at two CTAs per SM, 16-bit
// ones fit three (registers are held to the matching share)
template <typename R, typename SS, typename SP, int DIM, int NM, int BX, int BY, bool TS, bool TMA>
__global__ void __launch_bounds__(BX *BY, DIM == 3 ? ((BY < 8 && sizeof(SP) == 2 && !TS) ? 3 : 2) : 1)
k_velocity(const __grid_constant__ VelArgs<R, SS, SP> A)
{
    static_assert(!TMA || DIM == 3, "TMA staging is built for the 3D sweep");
    using L = VelSmem<R, SS, SP, DIM, NM, BX, BY, TS, TMA>;
    constexpr int TW = L::TW, SW = L::SW, RO = L::RO;
    static_assert(sizeof(SS) == sizeof(R), "state is stored in the arithmetic type");
    extern __shared__ __align__(128) unsigned char smem[];

    const Geo<R> &G = A.g;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int xb = blockIdx.x * TW, yb = blockIdx.y * BY;
    const int x0 = xb + 4 * tx, y = yb + ty;
    const int z0 = blockIdx.z * G.zseg;
    const int z1 = min(G.nz, z0 + G.zseg);
    const bool hd = (x0 < G.nx) && (y < G.ny);
    const long long row = (long long)y * G.px + x0;
    const int e0 = ty * TW + 4 * tx;

    R q[8][4];      // p of own columns, planes k-3 .. k+4
    R rq[2][4];     // rho of own columns, planes k, k+1
#pragma unroll
    for (int j = 0; j < 7; ++j) {
        const int kk = z0 - 3 + j;
        ld4_or_zero(A.p + kk * G.plane + row, hd && kk >= 0 && kk < G.nz, q[j]);
    }
    ld4_or_zero(A.rho + z0 * G.plane + row, hd && z0 < G.nz, rq[0]);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L::o_bar);
    if (TMA) {
        if (tx == 0 && ty == 0) {
            mbar_init(bars, 1);
            mbar_init(bars + 1, 1);
            mbar_fence_init();
        }
        __syncthreads();
    }
    bool timed_out = false;
    if (z0 < z1) vel_issue<R, SS, SP, DIM, NM, BX, BY, TS, TMA>(A, smem, z0, x0, y, xb, yb, row, hd);
    cp_commit();
    // absorbing-layer profile of this thread's x and y positions (fixed over the march)
    const bool pml_x = G.wabs > 0 && (x0 < G.wabs || x0 + 3 >= G.nx - G.wabs);
    const bool pml_y = DIM == 3 && G.wabs > 0 && (y < G.wabs || y >= G.ny - G.wabs);
    R pdx[4] = {0, 0, 0, 0}, pax[4] = {0, 0, 0, 0}, pdy = 0, pay = 0;
    if (pml_x && hd)
#pragma unroll
        for (int e = 0; e < 4; ++e) { pdx[e] = A.pd[0][x0 + e]; pax[e] = A.pa[0][x0 + e]; }
    if (pml_y && hd) { pdy = A.pd[1][y]; pay = A.pa[1][y]; }
    // layer depths of this thread's cells along x and y (fixed over the march)
    R sxy[4] = {R(0), R(0), R(0), R(0)};
    const R inv_lr = G.wabs > 0 ? R(1) / G.lr : R(0);
    if ((pml_x || pml_y) && hd)
#pragma unroll
        for (int e = 0; e < 4; ++e) sxy[e] = fmax(layer_depth<R>(x0 + e, G.nx, G.wabs), layer_depth<R>(y, G.ny, G.wabs));
    // class coefficients of the last class seen (classes rarely change along a column)
    int ccls = -1;
    R hdr[4], A1[4], B1[4], H1[4], dk1 = R(0);   // dk1 = ceff1 - 1/kappa1 (sum a1/2) of the cached class
    // absorbing-mechanism coefficients along x and y of the four cells: fixed
    // positions, so they change only with the cells' classes (their kappa)
    R pxa[4], pxb[4], pya[4], pyb[4];
    uint2 pkey = make_uint2(0xffffffffu, 0xffffffffu);

    for (int k = z0; k < z1; ++k) {
        const long long pk = (long long)k * G.plane;
        const int buf = k & 1;
        unsigned char *st = smem + buf * L::stage;
        R(*sp)[SW] = reinterpret_cast<R(*)[SW]>(smem + L::o_sp + buf * L::sp_stride);
        R(*sr)[TW + 4] = reinterpret_cast<R(*)[TW + 4]>(smem + L::o_sr + buf * L::sr_stride);
        __syncthreads();                           // iteration k-1 is done with stage/tiles (k+1)&1
        if (!TMA) {                                // centre of the tiles from registers (TMA copies them)
            R *dst = &sp[RO + ty][4 + 4 * tx];
            dst[0] = q[3][0]; dst[1] = q[3][1]; dst[2] = q[3][2]; dst[3] = q[3][3];
            R *r = &sr[ty][4 * tx];
            r[0] = rq[0][0]; r[1] = rq[0][1]; r[2] = rq[0][2]; r[3] = rq[0][3];
        }
        if (k + 1 < z1) vel_issue<R, SS, SP, DIM, NM, BX, BY, TS, TMA>(A, smem, k + 1, x0, y, xb, yb, row, hd);
        cp_commit();
        const bool pml_z = G.wabs > 0 && (k < G.wabs || k >= G.nz - G.wabs);
        R pdz = 0, paz = 0;
        if (pml_z) { pdz = A.pd[2][k]; paz = A.pa[2][k]; }
        cp_wait<1>();                              // this thread's copies of plane k have landed
        // bounded wait for the TMA copies of plane k; after a timeout the
        // thread stops waiting (the sweep then ends quickly, its result
        // flagged on the monitor)
        if (TMA && !timed_out && !mbar_wait_bounded(bars + buf, (unsigned)((k - z0) >> 1) & 1u)) timed_out = true;
        // cp.async staging: everyone's copies and tile centres visible to all.
        // TMA staging: every thread has waited on the barrier itself and
        // reads only its own cp.async copies (absorbing layer), so no barrier
        if (!TMA) __syncthreads();
        Sm<SS>::ld(reinterpret_cast<const SS *>(st + L::o_pn) + e0, q[7]);
        Sm<SS>::ld(reinterpret_cast<const SS *>(st + L::o_rn) + e0, rq[1]);
        if (hd) {
            R g[3][4];
            if (TS) {
                vel_gradient_ts<R, SS, SP, DIM, NM, BX, BY>(A, st, &sp[0][0], q, rq[0], k, x0, y, e0, g);
            } else {
            {
                R w[12];
                const R *s = &sp[RO + ty][4 * tx];
#pragma unroll
                for (int i = 0; i < 12; ++i) w[i] = s[i];
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    g[0][e] = G.c1 * (w[e + 5] - w[e + 4]) + G.c2 * (w[e + 6] - w[e + 3]) +
                              G.c3 * (w[e + 7] - w[e + 2]) + G.c4 * (w[e + 8] - w[e + 1]);
            }
            if (DIM == 3) {
                R c[8][4];
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const R *s = &sp[ty + r][4 + 4 * tx];
                    c[r][0] = s[0]; c[r][1] = s[1]; c[r][2] = s[2]; c[r][3] = s[3];
                }
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    g[1][e] = G.c1 * (c[4][e] - c[3][e]) + G.c2 * (c[5][e] - c[2][e]) +
                              G.c3 * (c[6][e] - c[1][e]) + G.c4 * (c[7][e] - c[0][e]);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e)
                g[2][e] = G.c1 * (q[4][e] - q[3][e]) + G.c2 * (q[5][e] - q[2][e]) +
                          G.c3 * (q[6][e] - q[1][e]) + G.c4 * (q[7][e] - q[0][e]);
            }
            R dtr[3][4];
            {
                const R *r0 = &sr[ty][4 * tx];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const R own = r0[e];
                    const R nxr = (x0 + e + 1 < G.nx) ? r0[e + 1] : own;
                    dtr[0][e] = R(2) * G.dt * fw_rcp(own + nxr);
                    if (DIM == 3) {
                        const R nyr = (y + 1 < G.ny) ? sr[ty + 1][4 * tx + e] : own;
                        dtr[1][e] = R(2) * G.dt * fw_rcp(own + nyr);
                    }
                    const R nzr = (k + 1 < G.nz) ? rq[1][e] : own;
                    dtr[2][e] = R(2) * G.dt * fw_rcp(own + nzr);
                }
            }
            const uint2 cl = *reinterpret_cast<const uint2 *>(reinterpret_cast<const uint16_t *>(st + L::o_cls) + e0);
            const uint16_t cls4[4] = {(uint16_t)(cl.x & 0xffffu), (uint16_t)(cl.x >> 16),
                                      (uint16_t)(cl.y & 0xffffu), (uint16_t)(cl.y >> 16)};
            // tissue-mechanism strength of the four cells (1 outside the layer)
            R rr[4] = {R(1), R(1), R(1), R(1)};
            if (pml_x || pml_y || pml_z) {
                const R sz = layer_depth<R>(k, G.nz, G.wabs);
#pragma unroll
                for (int e = 0; e < 4; ++e) rr[e] = ramp_of(fmax(sxy[e], sz), inv_lr);
            }
            if ((pml_x || pml_y) && (cl.x != pkey.x || cl.y != pkey.y)) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const R kap = __ldg(A.lut + (size_t)cls4[e] * kLutStride);   // kappa1
                    if (pml_x) pml_ab(pdx[e], pax[e], kap, G.dt, pxa[e], pxb[e]);
                    if (pml_y) pml_ab(pdy, pay, kap, G.dt, pya[e], pyb[e]);
                }
                pkey = cl;
            }
            // one direction at a time: its v and psi come from the stage
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                if (DIM == 2 && ax == 1) continue;
                R vv[4], ps[NM][4];
                Sm<SS>::ld(reinterpret_cast<const SS *>(st + L::o_v) + L::slot(ax) * L::TILE + e0, vv);
#pragma unroll
                for (int m = 0; m < NM; ++m)
                    Sm<SP>::ld(reinterpret_cast<const SP *>(st + L::o_psi) + (m * L::NAX + L::slot(ax)) * L::TILE + e0, ps[m]);
                const bool pml_here = ax == 0 ? pml_x : (ax == 1 ? pml_y : pml_z);
                R pp[4];
                if (pml_here) Sm<SS>::ld(reinterpret_cast<const SS *>(st + L::o_pml) + L::slot(ax) * L::TILE + e0, pp);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int c = cls4[e];
                    if (c != ccls) {
                        lut4(A.lut, c, 0, hdr);
                        lut4(A.lut, c, kLutA1, A1);
                        lut4(A.lut, c, kLutB1, B1);
                        lut4(A.lut, c, kLutH1, H1);
                        dk1 = __ldg(A.lut + (size_t)c * kLutStride + kLutDk);
                        ccls = c;
                    }
                    // a dead lane (x >= nx) gets drive 0, so its memory variables stay exactly 0
                    const bool live = x0 + e < G.nx;
                    const R gd = live ? g[ax][e] : R(0);
                    // ramped cell: ceff = 1/kappa + r sum a/2 (exact at r = 1), drive r g
                    const R ce = hdr[2] + (rr[e] - R(1)) * dk1;
                    const R rg = rr[e] * gd;
                    R stv = gd * ce;
#pragma unroll
                    for (int m = 0; m < NM; ++m) {
                        const R po = ps[m][e];
                        stv += H1[m] * po;
                        ps[m][e] = B1[m] * po + A1[m] * rg;
                    }
                    if (pml_here) {
                        const R d = ax == 0 ? pdx[e] : (ax == 1 ? pdy : pdz);
                        if (d > R(0) && live) {
                            R a, b;
                            if (ax == 0) { a = pxa[e]; b = pxb[e]; }
                            else if (ax == 1) { a = pya[e]; b = pyb[e]; }
                            else pml_ab(d, paz, hdr[0], G.dt, a, b);
                            const R po = pp[e];
                            stv += R(0.5) * (R(1) + b) * po + R(0.5) * a * gd;
                            pp[e] = b * po + a * gd;
                        }
                    }
                    vv[e] = live ? vv[e] - dtr[ax][e] * stv : R(0);
                }
                Io<SS>::st(wr_at(A.v[ax] + pk + row, TMA ? 0LL : A.wofs), vv);
#pragma unroll
                for (int m = 0; m < NM; ++m) Io<SP>::st(wr_at(A.psi[m][ax] + pk + row, TMA ? 0LL : A.wofs), ps[m]);
                if (pml_here) Io<SS>::st(wr_at(A.psip[ax] + pk + row, TMA ? 0LL : A.wofs), pp);
            }
        }
#pragma unroll
        for (int j = 0; j < 7; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) q[j][e] = q[j + 1][e];
#pragma unroll
        for (int e = 0; e < 4; ++e) rq[0][e] = rq[1][e];
    }
    cp_wait<0>();
    if (TMA && timed_out) {
        // record the failure; give the copies of the last two planes one more
        // bounded chance to land before the CTA's shared memory is released
        atomicExch(&A.mon->timeout, 1);
        for (int k = max(z0, z1 - 2); k < z1; ++k) mbar_wait_bounded(bars + (k & 1), (unsigned)((k - z0) >> 1) & 1u);
    }
}

// ---------------------------------------------------------------------------
// pressure sweep

// TMA staging of plane k of the pressure sweep (3D): one thread arms the
// stage's barrier and issues one tile copy per stream; v_x (x halo) and v_y
// (y halo) land in the tiles of parity k&1
template <typename R, typename SS, typename SP, int NM, int BX, int BY, bool NL, bool TS>
__device__ __forceinline__ void pres_issue_tma(const PresArgs<R, SS, SP> &A, unsigned char *sm, int k, int xb, int yb)
{
    using L = PresSmem<R, SS, SP, 3, NM, BX, BY, TS, true>;
    constexpr unsigned bytes = (unsigned)((L::RINGS ? 0 : ((size_t)BY * L::SWX + (size_t)L::SHY * L::TW) * sizeof(SS)) +
                                          L::TILE * (3 + (NL ? 1 : 0) + (TS ? 1 : 0)) * sizeof(SS) +
                                          (size_t)NM * L::TILE * sizeof(SP) + L::TILE * 2);
    unsigned char *st = sm + (k & 1) * L::stage;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + L::o_bar) + (k & 1);
    fence_proxy_async_smem();
    mbar_expect_tx(bar, bytes);
    tma_load_3d(st + L::o_qn, &A.maps.vz_own, xb, yb, k + 3, bar);
    tma_load_3d(st + L::o_p, &A.maps.p_own, xb, yb, k, bar);
    tma_load_3d(st + L::o_kd, &A.maps.kdt, xb, yb, k, bar);
    if (NL) tma_load_3d(st + L::o_bd, &A.maps.b2dt, xb, yb, k, bar);
    if (TS) tma_load_3d(st + L::o_rh, &A.maps.rho_own, xb, yb, k, bar);
#pragma unroll
    for (int m = 0; m < NM; ++m) tma_load_3d(st + L::o_psi + m * L::TILE * sizeof(SP), &A.maps.psi[m], xb, yb, k, bar);
    tma_load_3d(st + L::o_cls, &A.maps.cls, xb, yb, k, bar);
    if (!L::RINGS) {
        tma_load_3d(sm + L::o_svx + (k & 1) * L::svx_stride, &A.maps.vx_halo, xb - 4, yb, k, bar);
        tma_load_3d(sm + L::o_svy + (k & 1) * L::svy_stride, &A.maps.vy_halo, xb, yb - 4, k, bar);
    }
}

// Time-space stencil with TMA staging: plane k of the v rings (slot k&3,
// barrier 2 + (k&3)); planes outside the grid read as zero
template <typename R, typename SS, typename SP, int NM, int BX, int BY>
__device__ __forceinline__ void pres_issue_rings(const PresArgs<R, SS, SP> &A, unsigned char *sm, int k, int xb, int yb)
{
    using L = PresSmem<R, SS, SP, 3, NM, BX, BY, true, true>;
    const int s = k & 3;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + L::o_bar) + 2 + s;
    fence_proxy_async_smem();
    mbar_expect_tx(bar, L::ring_bytes);
    tma_load_3d(sm + L::o_rx + s * L::rx_stride, &A.maps.vx_ring, xb - 4, yb - 1, k, bar);
    tma_load_3d(sm + L::o_ry + s * L::ry_stride, &A.maps.vy_ring, xb - 4, yb - 4, k, bar);
    tma_load_3d(sm + L::o_rz + s * L::rx_stride, &A.maps.vz_ring, xb - 4, yb - 1, k, bar);
}

// q_d = D-_d v_d with the time-space stencil from the rings (see
// pres_divergence_ts for the stencil): ring slots of planes k-1, k, k+1 hold
// v_x and v_z with rows y-1 .. y+BY and v_y with rows y-4 .. y+BY+2, all
// with 4 columns of x halo; the depth taps of v_z come from the register
// queue qz (planes k-4 .. k+3)
template <typename R, typename SS, typename SP, int NM, int BX, int BY>
__device__ __forceinline__ void pres_divergence_ts_rings(const PresArgs<R, SS, SP> &A, const unsigned char *st,
                                                         const unsigned char *sm, const R (&qz)[8][4], const R (&kd)[4],
                                                         int k, int x0, int e0, R (&qd)[3][4])
{
    using L = PresSmem<R, SS, SP, 3, NM, BX, BY, true, true>;
    constexpr int SW = L::SWX;
    const Geo<R> &G = A.g;
    const int tx = threadIdx.x, ty = threadIdx.y;
    auto rx = [&](int kk) { return reinterpret_cast<const R *>(sm + L::o_rx + (kk & 3) * L::rx_stride); };
    auto ry = [&](int kk) { return reinterpret_cast<const R *>(sm + L::o_ry + (kk & 3) * L::ry_stride); };
    auto rz = [&](int kk) { return reinterpret_cast<const R *>(sm + L::o_rz + (kk & 3) * L::rx_stride); };
    const int c0 = 4 + 4 * tx;                     // column of x0 in the ring tiles (a multiple of 4)
    const int rX = ty + 1, rY = ty + 4;            // row of y in the v_x / v_z and in the v_y tiles
    // eight values at columns c0-4 .. c0+3 of row r of tile t (two 16-byte loads)
    auto row8 = [&](const R *t, int r, R (&o)[8]) {
        R a4[4], b4[4];
        Sm<R>::ld(t + r * SW + c0 - 4, a4);
        Sm<R>::ld(t + r * SW + c0, b4);
#pragma unroll
        for (int i = 0; i < 4; ++i) { o[i] = a4[i]; o[i + 4] = b4[i]; }
    };
    R X[3][4], t8[8];
    // v_x: two-point x differences at x (v(x) - v(x-1)) of rows y -+ 1 (plane k) and of planes k -+ 1 (row y)
    {
        const R *xs[4] = {rx(k), rx(k), rx(k - 1), rx(k + 1)};
        const int rs[4] = {rX - 1, rX + 1, rX, rX};
#pragma unroll
        for (int e = 0; e < 4; ++e) X[0][e] = R(0);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            row8(xs[j], rs[j], t8);
#pragma unroll
            for (int e = 0; e < 4; ++e) X[0][e] += t8[e + 4] - t8[e + 3];
        }
    }
    // v_y: two-point y differences at y (v(y) - v(y-1)) at columns x -+ 1 (plane k) and of planes k -+ 1
    {
        const R *yk = ry(k);
        R u0[4], u1[4];
        Sm<R>::ld(yk + rY * SW + c0, u0);
        Sm<R>::ld(yk + (rY - 1) * SW + c0, u1);
        const R l0 = yk[rY * SW + c0 - 1], l1 = yk[(rY - 1) * SW + c0 - 1];
        const R g0 = yk[rY * SW + c0 + 4], g1 = yk[(rY - 1) * SW + c0 + 4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const R am = e > 0 ? u0[e - 1] - u1[e - 1] : l0 - l1;
            const R ap = e < 3 ? u0[e + 1] - u1[e + 1] : g0 - g1;
            X[1][e] = am + ap;
        }
#pragma unroll
        for (int s = -1; s <= 1; s += 2) {
            const R *yp = ry(k + s);
            Sm<R>::ld(yp + rY * SW + c0, u0);
            Sm<R>::ld(yp + (rY - 1) * SW + c0, u1);
#pragma unroll
            for (int e = 0; e < 4; ++e) X[1][e] += u0[e] - u1[e];
        }
    }
    // v_z: two-point depth differences (plane k minus k-1) at x -+ 1 (row y) and at y -+ 1
    {
        const R *zk = rz(k), *zm = rz(k - 1);
        R d[6];                                    // columns c0-1 .. c0+4 of row y, plane k minus plane k-1
        {
            R a4[4], b4[4];
            Sm<R>::ld(zk + rX * SW + c0, a4);
            Sm<R>::ld(zm + rX * SW + c0, b4);
#pragma unroll
            for (int e = 0; e < 4; ++e) d[e + 1] = a4[e] - b4[e];
            d[0] = zk[rX * SW + c0 - 1] - zm[rX * SW + c0 - 1];
            d[5] = zk[rX * SW + c0 + 4] - zm[rX * SW + c0 + 4];
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) X[2][e] = d[e] + d[e + 2];
#pragma unroll
        for (int s = -1; s <= 1; s += 2) {
            R a4[4], b4[4];
            Sm<R>::ld(zk + (rX + s) * SW + c0, a4);
            Sm<R>::ld(zm + (rX + s) * SW + c0, b4);
#pragma unroll
            for (int e = 0; e < 4; ++e) X[2][e] += a4[e] - b4[e];
        }
    }
    // on-axis x: columns c0-4 .. c0+7 of row y, plane k
    R w[12];
    {
        const R *xk = rx(k);
        R a4[4];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            Sm<R>::ld(xk + rX * SW + c0 - 4 + 4 * q, a4);
#pragma unroll
            for (int i = 0; i < 4; ++i) w[4 * q + i] = a4[i];
        }
    }
    // on-axis y: rows y-4 .. y+3 of plane k, this thread's four columns
    R cy[8][4];
    {
        const R *yk = ry(k);
#pragma unroll
        for (int r = 0; r < 8; ++r) Sm<R>::ld(yk + (rY - 4 + r) * SW + c0, cy[r]);
    }
    R rh[4];
    Sm<SS>::ld(reinterpret_cast<const SS *>(st + L::o_rh) + e0, rh);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const bool live = x0 + e < G.nx;
        const R r2 = live ? kd[e] * G.r2s * fw_rcp(rh[e]) : R(0);
        R a[4], b;
        ts_weights(G, r2, a, b);
        qd[0][e] = a[0] * (w[e + 4] - w[e + 3]) + a[1] * (w[e + 5] - w[e + 2]) + a[2] * (w[e + 6] - w[e + 1]) +
                   a[3] * (w[e + 7] - w[e + 0]) + b * X[0][e];
        qd[1][e] = a[0] * (cy[4][e] - cy[3][e]) + a[1] * (cy[5][e] - cy[2][e]) + a[2] * (cy[6][e] - cy[1][e]) +
                   a[3] * (cy[7][e] - cy[0][e]) + b * X[1][e];
        qd[2][e] = a[0] * (qz[4][e] - qz[3][e]) + a[1] * (qz[5][e] - qz[2][e]) + a[2] * (qz[6][e] - qz[1][e]) +
                   a[3] * (qz[7][e] - qz[0][e]) + b * X[2][e];
    }
}

template <typename R, typename SS, typename SP, int DIM, int NM, int BX, int BY, bool NL, bool TS, bool TMA>
__device__ __forceinline__ void pres_issue(const PresArgs<R, SS, SP> &A, unsigned char *sm, int k, int x0, int y,
                                           int yb, long long row, bool hd)
{
    using L = PresSmem<R, SS, SP, DIM, NM, BX, BY, TS, TMA>;
    const Geo<R> &G = A.g;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const long long pk = (long long)k * G.plane;
    unsigned char *st = sm + (k & 1) * L::stage;
    const int e0 = ty * L::TW + 4 * tx;
    if (TMA) {
        if (tx == 0 && ty == 0) pres_issue_tma<R, SS, SP, NM, BX, BY, NL, TS>(A, sm, k, x0, yb);
        // absorbing-layer memory: per thread, where this thread needs it
        if (G.wabs > 0 && hd) {
            const bool in[3] = {x0 < G.wabs || x0 + 3 >= G.nx - G.wabs, y < G.wabs || y >= G.ny - G.wabs,
                                k < G.wabs || k >= G.nz - G.wabs};
#pragma unroll
            for (int ax = 0; ax < 3; ++ax)
                if (in[ax]) cp_async4(reinterpret_cast<SS *>(st + L::o_pml) + L::slot(ax) * L::TILE + e0, A.psip[ax] + pk + row, true);
        }
        return;
    }
    const SS *gz = A.p;
    {
        const bool ok = hd && k + 3 < G.nz;
        cp_async4(reinterpret_cast<SS *>(st + L::o_qn) + e0, ok ? A.v[2] + pk + 3 * G.plane + row : gz, ok);
    }
    cp_async4(reinterpret_cast<SS *>(st + L::o_p) + e0, hd ? A.p + pk + row : gz, hd);
    cp_async4(reinterpret_cast<SS *>(st + L::o_kd) + e0, hd ? A.kdt + pk + row : gz, hd);
    if (NL) cp_async4(reinterpret_cast<SS *>(st + L::o_bd) + e0, hd ? A.b2dt + pk + row : gz, hd);
    if (TS) cp_async4(reinterpret_cast<SS *>(st + L::o_rh) + e0, hd ? A.rho + pk + row : gz, hd);
#pragma unroll
    for (int m = 0; m < NM; ++m)
        cp_async4(reinterpret_cast<SP *>(st + L::o_psi) + m * L::TILE + e0,
                  hd ? A.psi[m] + pk + row : reinterpret_cast<const SP *>(gz), hd);
    cp_async<8>(reinterpret_cast<uint16_t *>(st + L::o_cls) + e0, hd ? (const void *)(A.cls + pk + row) : (const void *)gz, hd);
    if (G.wabs > 0 && hd) {
        const bool in[3] = {x0 < G.wabs || x0 + 3 >= G.nx - G.wabs, DIM == 3 && (y < G.wabs || y >= G.ny - G.wabs),
                            k < G.wabs || k >= G.nz - G.wabs};
#pragma unroll
        for (int ax = 0; ax < 3; ++ax)
            if (in[ax]) cp_async4(reinterpret_cast<SS *>(st + L::o_pml) + L::slot(ax) * L::TILE + e0, A.psip[ax] + pk + row, true);
    }
    // v_x (with x halo) and v_y (with y halo) of plane k straight into the tiles
    R *svx = reinterpret_cast<R *>(sm + L::o_svx + (k & 1) * L::svx_stride);
    cp_async4(reinterpret_cast<SS *>(svx + ty * L::SWX + 4 + 4 * tx), hd ? A.v[0] + pk + row : gz, hd);
    if (tx == 0) {
        const bool ok = y < G.ny && x0 - 4 >= 0;
        cp_async4(reinterpret_cast<SS *>(svx + ty * L::SWX), ok ? A.v[0] + pk + (long long)y * G.px + (x0 - 4) : gz, ok);
    }
    if (tx == BX - 1) {
        const bool ok = y < G.ny && x0 + 4 < G.px;
        cp_async4(reinterpret_cast<SS *>(svx + ty * L::SWX + L::TW + 4), ok ? A.v[0] + pk + (long long)y * G.px + (x0 + 4) : gz, ok);
    }
    if (DIM == 3) {
        R *svy = reinterpret_cast<R *>(sm + L::o_svy + (k & 1) * L::svy_stride);
        cp_async4(reinterpret_cast<SS *>(svy + (4 + ty) * L::TW + 4 * tx), hd ? A.v[1] + pk + row : gz, hd);
        for (int r = ty; r < 7; r += BY) {      // 4 halo rows below the tile, 3 above
            const int yy = r < 4 ? yb - 4 + r : yb + BY + (r - 4);
            const int hrow = r < 4 ? r : BY + 4 + (r - 4);
            const bool ok = yy >= 0 && yy < G.ny && x0 < G.px;
            cp_async4(reinterpret_cast<SS *>(svy + hrow * L::TW + 4 * tx), ok ? A.v[1] + pk + (long long)yy * G.px + x0 : gz, ok);
        }
    }
}

// Divergence terms q_d = D-_d v_d at this thread's four cells with the
// time-space stencil (Sec. 3.3, after Tan & Huang 2014), the counterpart of
// vel_gradient_ts: per-cell weights from r^2 = (K dt) dt / (rho dx^2); the
// cross term along d sums, over the other axes e and s = -+1, the two-point
// difference v_d(i) - v_d(i-1) along d at the neighbour s along e.  v_x of
// plane k comes from the tile svx (x halo), v_y from svy (y halo), v_z from
// the register queue; the values of the neighbour rows and planes from the
// read-only cache (v is not written by this sweep).
template <typename R, typename SS, typename SP, int DIM, int NM, int BX, int BY>
__device__ __forceinline__ void pres_divergence_ts(const PresArgs<R, SS, SP> &A, const unsigned char *st,
                                                   const R *svx0, const R *svy0, const R (&qz)[8][4],
                                                   const R (&kd)[4], int k, int x0, int y, int e0, R (&qd)[3][4])
{
    using L = PresSmem<R, SS, SP, DIM, NM, BX, BY, true>;
    constexpr int TW = L::TW, SWX = L::SWX;
    const Geo<R> &G = A.g;
    const int tx = threadIdx.x, ty = threadIdx.y;
    R rh[4];
    Sm<SS>::ld(reinterpret_cast<const SS *>(st + L::o_rh) + e0, rh);
    const long long rowk = (long long)y * G.px;
    const bool okm = k >= 1, okp = k + 1 < G.nz, oxl = x0 >= 1;
    // five values x0-1 .. x0+3 of field f in row rr of plane kk
    auto five = [&](const SS *f, int kk, long long rr, bool ok, R (&o)[5]) {
        R t[4];
        ld4_or_zero(f + (long long)kk * G.plane + rr + x0, ok, t);
        o[0] = ldz1<SS, R>(f + (long long)kk * G.plane + rr + x0 - 1, ok && oxl);
#pragma unroll
        for (int i = 0; i < 4; ++i) o[i + 1] = t[i];
    };
    R w[12];
    {
        const R *s = svx0 + ty * SWX + 4 * tx;
#pragma unroll
        for (int i = 0; i < 12; ++i) w[i] = s[i];
    }
    R X[3][4];
    {   // v_x: planes k -+ 1 of row y; rows y -+ 1 of plane k (3D)
        R m[5], p[5];
        five(A.v[0], k - 1, rowk, okm, m);
        five(A.v[0], k + 1, rowk, okp, p);
#pragma unroll
        for (int e = 0; e < 4; ++e) X[0][e] = (m[e + 1] - m[e]) + (p[e + 1] - p[e]);
        if (DIM == 3) {
            five(A.v[0], k, rowk - G.px, y >= 1, m);
            five(A.v[0], k, rowk + G.px, y + 1 < G.ny, p);
#pragma unroll
            for (int e = 0; e < 4; ++e) X[0][e] += (m[e + 1] - m[e]) + (p[e + 1] - p[e]);
        }
    }
    {   // v_z: columns x -+ 1 of planes k, k-1 (own columns from the queue); rows y -+ 1 (3D)
        const R l0 = ldz1<SS, R>(A.v[2] + (long long)k * G.plane + rowk + x0 - 1, oxl);
        const R l1 = ldz1<SS, R>(A.v[2] + (long long)(k - 1) * G.plane + rowk + x0 - 1, oxl && okm);
        const R r0 = ldz1<SS, R>(A.v[2] + (long long)k * G.plane + rowk + x0 + 4, x0 + 4 < G.px);
        const R r1 = ldz1<SS, R>(A.v[2] + (long long)(k - 1) * G.plane + rowk + x0 + 4, x0 + 4 < G.px && okm);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const R a0 = e > 0 ? qz[4][e - 1] : l0, a1 = e > 0 ? qz[3][e - 1] : l1;
            const R b0 = e < 3 ? qz[4][e + 1] : r0, b1 = e < 3 ? qz[3][e + 1] : r1;
            X[2][e] = (a0 - a1) + (b0 - b1);
        }
        if (DIM == 3) {
            R m0[4], m1[4], p0[4], p1[4];
            ld4_or_zero(A.v[2] + (long long)k * G.plane + rowk - G.px + x0, y >= 1, m0);
            ld4_or_zero(A.v[2] + (long long)(k - 1) * G.plane + rowk - G.px + x0, y >= 1 && okm, m1);
            ld4_or_zero(A.v[2] + (long long)k * G.plane + rowk + G.px + x0, y + 1 < G.ny, p0);
            ld4_or_zero(A.v[2] + (long long)(k - 1) * G.plane + rowk + G.px + x0, y + 1 < G.ny && okm, p1);
#pragma unroll
            for (int e = 0; e < 4; ++e) X[2][e] += (m0[e] - m1[e]) + (p0[e] - p1[e]);
        }
    }
    if (DIM == 3) {   // v_y: columns x -+ 1 of rows y, y-1 (tile svy, ends from the cache); planes k -+ 1
        const R *c0 = svy0 + (4 + ty) * TW, *c1 = svy0 + (3 + ty) * TW;
        const R l0 = tx > 0 ? c0[4 * tx - 1] : ldz1<SS, R>(A.v[1] + (long long)k * G.plane + rowk + x0 - 1, oxl);
        const R l1 = tx > 0 ? c1[4 * tx - 1]
                            : ldz1<SS, R>(A.v[1] + (long long)k * G.plane + rowk - G.px + x0 - 1, oxl && y >= 1);
        const R r0 = tx < BX - 1 ? c0[4 * tx + 4]
                                 : ldz1<SS, R>(A.v[1] + (long long)k * G.plane + rowk + x0 + 4, x0 + 4 < G.px);
        const R r1 = tx < BX - 1 ? c1[4 * tx + 4]
                                 : ldz1<SS, R>(A.v[1] + (long long)k * G.plane + rowk - G.px + x0 + 4,
                                               x0 + 4 < G.px && y >= 1);
        R m0[4], m1[4], p0[4], p1[4];
        ld4_or_zero(A.v[1] + (long long)(k - 1) * G.plane + rowk + x0, okm, m0);
        ld4_or_zero(A.v[1] + (long long)(k - 1) * G.plane + rowk - G.px + x0, okm && y >= 1, m1);
        ld4_or_zero(A.v[1] + (long long)(k + 1) * G.plane + rowk + x0, okp, p0);
        ld4_or_zero(A.v[1] + (long long)(k + 1) * G.plane + rowk - G.px + x0, okp && y >= 1, p1);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const R a0 = e > 0 ? c0[4 * tx + e - 1] : l0, a1 = e > 0 ? c1[4 * tx + e - 1] : l1;
            const R b0 = e < 3 ? c0[4 * tx + e + 1] : r0, b1 = e < 3 ? c1[4 * tx + e + 1] : r1;
            X[1][e] = (a0 - a1) + (b0 - b1) + (m0[e] - m1[e]) + (p0[e] - p1[e]);
        }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const bool live = x0 + e < G.nx;
        const R r2 = live ? kd[e] * G.r2s * fw_rcp(rh[e]) : R(0);
        R a[4], b;
        ts_weights(G, r2, a, b);
        qd[0][e] = a[0] * (w[e + 4] - w[e + 3]) + a[1] * (w[e + 5] - w[e + 2]) + a[2] * (w[e + 6] - w[e + 1]) +
                   a[3] * (w[e + 7] - w[e + 0]) + b * X[0][e];
        if (DIM == 3) {
            const R *c = svy0 + 4 * tx + e;
            qd[1][e] = a[0] * (c[(4 + ty) * TW] - c[(3 + ty) * TW]) + a[1] * (c[(5 + ty) * TW] - c[(2 + ty) * TW]) +
                       a[2] * (c[(6 + ty) * TW] - c[(1 + ty) * TW]) + a[3] * (c[(7 + ty) * TW] - c[(0 + ty) * TW]) +
                       b * X[1][e];
        }
        qd[2][e] = a[0] * (qz[4][e] - qz[3][e]) + a[1] * (qz[5][e] - qz[2][e]) + a[2] * (qz[6][e] - qz[1][e]) +
                   a[3] * (qz[7][e] - qz[0][e]) + b * X[2][e];
    }
}

template <typename R, typename SS, typename SP, int DIM, int NM, int BX, int BY, bool NL, bool TS, bool TMA>
__global__ void __launch_bounds__(BX *BY, DIM == 3 ? ((BY < 8 && !TS) ? 3 : 2) : 1)
k_pressure(const __grid_constant__ PresArgs<R, SS, SP> A)
{
    static_assert(!TMA || DIM == 3, "TMA staging is built for the 3D sweep");
    using L = PresSmem<R, SS, SP, DIM, NM, BX, BY, TS, TMA>;
    constexpr int TW = L::TW, SWX = L::SWX, SHY = L::SHY;
    extern __shared__ __align__(128) unsigned char smem[];

    const Geo<R> &G = A.g;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int xb = blockIdx.x * TW, yb = blockIdx.y * BY;
    const int x0 = xb + 4 * tx, y = yb + ty;
    const int z0 = blockIdx.z * G.zseg;
    const int z1 = min(G.nz, z0 + G.zseg);
    const bool hd = (x0 < G.nx) && (y < G.ny);
    const long long row = (long long)y * G.px + x0;
    const int e0 = ty * TW + 4 * tx;

    R qz[8][4];     // vz of own columns, planes k-4 .. k+3
#pragma unroll
    for (int j = 0; j < 7; ++j) {
        const int kk = z0 - 4 + j;
        ld4_or_zero(A.v[2] + kk * G.plane + row, hd && kk >= 0 && kk < G.nz, qz[j]);
    }
    R pmax = R(0);
    bool bad = false;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L::o_bar);
    if (TMA) {
        if (tx == 0 && ty == 0) {
            for (int b = 0; b < (L::RINGS ? 6 : 2); ++b) mbar_init(bars + b, 1);
            mbar_fence_init();
        }
        __syncthreads();
    }
    if constexpr (L::RINGS) {   // v rings of planes z0-1 .. z0+1 (later planes two ahead, in the loop)
        if (tx == 0 && ty == 0 && z0 < z1)
            for (int kk = z0 - 1; kk <= z0 + 1; ++kk) pres_issue_rings<R, SS, SP, NM, BX, BY>(A, smem, kk, xb, yb);
    }
    // phase parity of the ring barrier of plane kk (first used by plane z0 - 1)
    auto ring_parity = [&](int kk) { return (unsigned)((kk - z0 + 1) >> 2) & 1u; };
    bool timed_out = false;
    if (z0 < z1) pres_issue<R, SS, SP, DIM, NM, BX, BY, NL, TS, TMA>(A, smem, z0, x0, y, yb, row, hd);
    cp_commit();
    const bool pml_x = G.wabs > 0 && (x0 < G.wabs || x0 + 3 >= G.nx - G.wabs);
    const bool pml_y = DIM == 3 && G.wabs > 0 && (y < G.wabs || y >= G.ny - G.wabs);
    R pdx[4] = {0, 0, 0, 0}, pax[4] = {0, 0, 0, 0}, pdy = 0, pay = 0;
    if (pml_x && hd)
#pragma unroll
        for (int e = 0; e < 4; ++e) { pdx[e] = A.pd[0][x0 + e]; pax[e] = A.pa[0][x0 + e]; }
    if (pml_y && hd) { pdy = A.pd[1][y]; pay = A.pa[1][y]; }
    R sxy[4] = {R(0), R(0), R(0), R(0)};
    const R inv_lr = G.wabs > 0 ? R(1) / G.lr : R(0);
    if ((pml_x || pml_y) && hd)
#pragma unroll
        for (int e = 0; e < 4; ++e) sxy[e] = fmax(layer_depth<R>(x0 + e, G.nx, G.wabs), layer_depth<R>(y, G.ny, G.wabs));
    int ccls = -1;
    R hdr[4], A2[4], B2[4], H2[4], dk2 = R(0);   // dk2 = ceff2 - 1/kappa2 (sum a2/2) of the cached class
    // absorbing-mechanism coefficients along x and y, recomputed only when the cells' classes change
    R pxa[4], pxb[4], pya[4], pyb[4];
    uint2 pkey = make_uint2(0xffffffffu, 0xffffffffu);
    for (int k = z0; k < z1; ++k) {
        const long long pk = (long long)k * G.plane;
        const int buf = k & 1;
        unsigned char *st = smem + buf * L::stage;
        const R(*svx)[SWX] = reinterpret_cast<const R(*)[SWX]>(smem + L::o_svx + buf * L::svx_stride);
        const R(*svy)[TW] = reinterpret_cast<const R(*)[TW]>(smem + L::o_svy + buf * L::svy_stride);
        __syncthreads();                           // iteration k-1 is done with stage/tiles (k+1)&1
        if constexpr (L::RINGS) {                  // ring slot of plane k-2 is free: plane k+2 into it
            if (tx == 0 && ty == 0 && k + 2 <= z1) pres_issue_rings<R, SS, SP, NM, BX, BY>(A, smem, k + 2, xb, yb);
        }
        if (k + 1 < z1) pres_issue<R, SS, SP, DIM, NM, BX, BY, NL, TS, TMA>(A, smem, k + 1, x0, y, yb, row, hd);
        cp_commit();
        const bool pml_z = G.wabs > 0 && (k < G.wabs || k >= G.nz - G.wabs);
        R pdz = 0, paz = 0;
        if (pml_z) { pdz = A.pd[2][k]; paz = A.pa[2][k]; }
        cp_wait<1>();
        // bounded wait for the TMA copies of plane k (see the velocity sweep);
        // with TMA staging each thread has waited itself: no barrier needed
        if (TMA && !timed_out && !mbar_wait_bounded(bars + buf, (unsigned)((k - z0) >> 1) & 1u)) timed_out = true;
        if constexpr (L::RINGS) {                  // v rings of planes k-1, k (earlier waits) and k+1
            for (int kk = k == z0 ? z0 - 1 : k + 1; kk <= k + 1 && !timed_out; ++kk)
                if (!mbar_wait_bounded(bars + 2 + (kk & 3), ring_parity(kk))) timed_out = true;
        }
        if (!TMA) __syncthreads();
        Sm<SS>::ld(reinterpret_cast<const SS *>(st + L::o_qn) + e0, qz[7]);
        if (hd) {
            R qd[3][4];
            R pv[4], kd[4], bd[4], ps[NM][4];
            Sm<SS>::ld(reinterpret_cast<const SS *>(st + L::o_kd) + e0, kd);
            if constexpr (L::RINGS) {
                pres_divergence_ts_rings<R, SS, SP, NM, BX, BY>(A, st, smem, qz, kd, k, x0, e0, qd);
            } else if (TS) {
                pres_divergence_ts<R, SS, SP, DIM, NM, BX, BY>(A, st, &svx[0][0], &svy[0][0], qz, kd, k, x0, y, e0, qd);
            } else {
            {
                R w[12];
                const R *s = &svx[ty][4 * tx];
#pragma unroll
                for (int i = 0; i < 12; ++i) w[i] = s[i];
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    qd[0][e] = G.c1 * (w[e + 4] - w[e + 3]) + G.c2 * (w[e + 5] - w[e + 2]) +
                               G.c3 * (w[e + 6] - w[e + 1]) + G.c4 * (w[e + 7] - w[e + 0]);
            }
            if (DIM == 3) {
                R c[8][4];
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const R *s = &svy[ty + r][4 * tx];
                    c[r][0] = s[0]; c[r][1] = s[1]; c[r][2] = s[2]; c[r][3] = s[3];
                }
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    qd[1][e] = G.c1 * (c[4][e] - c[3][e]) + G.c2 * (c[5][e] - c[2][e]) +
                               G.c3 * (c[6][e] - c[1][e]) + G.c4 * (c[7][e] - c[0][e]);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e)
                qd[2][e] = G.c1 * (qz[4][e] - qz[3][e]) + G.c2 * (qz[5][e] - qz[2][e]) +
                           G.c3 * (qz[6][e] - qz[1][e]) + G.c4 * (qz[7][e] - qz[0][e]);
            }
            Sm<SS>::ld(reinterpret_cast<const SS *>(st + L::o_p) + e0, pv);
            if (NL) Sm<SS>::ld(reinterpret_cast<const SS *>(st + L::o_bd) + e0, bd);
#pragma unroll
            for (int m = 0; m < NM; ++m) Sm<SP>::ld(reinterpret_cast<const SP *>(st + L::o_psi) + m * L::TILE + e0, ps[m]);
            const uint2 cl = *reinterpret_cast<const uint2 *>(reinterpret_cast<const uint16_t *>(st + L::o_cls) + e0);
            const uint16_t cls4[4] = {(uint16_t)(cl.x & 0xffffu), (uint16_t)(cl.x >> 16),
                                      (uint16_t)(cl.y & 0xffffu), (uint16_t)(cl.y >> 16)};
            R pp[3][4];
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                const bool pml_here = ax == 0 ? pml_x : (ax == 1 ? pml_y : pml_z);
                if (pml_here) Sm<SS>::ld(reinterpret_cast<const SS *>(st + L::o_pml) + L::slot(ax) * L::TILE + e0, pp[ax]);
            }
            R rr[4] = {R(1), R(1), R(1), R(1)};
            if (pml_x || pml_y || pml_z) {
                const R sz = layer_depth<R>(k, G.nz, G.wabs);
#pragma unroll
                for (int e = 0; e < 4; ++e) rr[e] = ramp_of(fmax(sxy[e], sz), inv_lr);
            }
            if ((pml_x || pml_y) && (cl.x != pkey.x || cl.y != pkey.y)) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const R kap = __ldg(A.lut + (size_t)cls4[e] * kLutStride + 1);   // kappa2
                    if (pml_x) pml_ab(pdx[e], pax[e], kap, G.dt, pxa[e], pxb[e]);
                    if (pml_y) pml_ab(pdy, pay, kap, G.dt, pya[e], pyb[e]);
                }
                pkey = cl;
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c = cls4[e];
                if (c != ccls) {
                    lut4(A.lut, c, 0, hdr);
                    lut4(A.lut, c, kLutA2, A2);
                    lut4(A.lut, c, kLutB2, B2);
                    lut4(A.lut, c, kLutH2, H2);
                    dk2 = __ldg(A.lut + (size_t)c * kLutStride + kLutDk + 1);
                    ccls = c;
                }
                const bool live = x0 + e < G.nx;
                R div = qd[0][e] + qd[2][e];
                if (DIM == 3) div += qd[1][e];
                div = live ? div : R(0);       // dead lane: memory variables stay exactly 0
                const R ce = hdr[3] + (rr[e] - R(1)) * dk2;   // exact at r = 1
                const R rdiv = rr[e] * div;
                R stp = div * ce;
#pragma unroll
                for (int m = 0; m < NM; ++m) {
                    const R po = ps[m][e];
                    stp += H2[m] * po;
                    ps[m][e] = B2[m] * po + A2[m] * rdiv;
                }
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    if (DIM == 2 && ax == 1) continue;
                    const bool pml_here = ax == 0 ? pml_x : (ax == 1 ? pml_y : pml_z);
                    if (!pml_here) continue;
                    const R d = ax == 0 ? pdx[e] : (ax == 1 ? pdy : pdz);
                    if (d > R(0) && live) {
                        R a, b;
                        if (ax == 0) { a = pxa[e]; b = pxb[e]; }
                        else if (ax == 1) { a = pya[e]; b = pyb[e]; }
                        else pml_ab(d, paz, hdr[1], G.dt, a, b);
                        const R po = pp[ax][e];
                        stp += R(0.5) * (R(1) + b) * po + R(0.5) * a * qd[ax][e];
                        pp[ax][e] = b * po + a * qd[ax][e];
                    }
                }
                R fac = kd[e];
                if (NL) fac += bd[e] * pv[e];
                const R pn = live ? pv[e] - fac * stp : R(0);
                pv[e] = pn;
                const R ap = fabs(pn);
                bad |= !(ap <= R(3.0e38));
                pmax = fmax(pmax, ap);
            }
            Io<SS>::st(wr_at(A.p + pk + row, TMA ? 0LL : A.wofs), pv);
#pragma unroll
            for (int m = 0; m < NM; ++m) Io<SP>::st(wr_at(A.psi[m] + pk + row, TMA ? 0LL : A.wofs), ps[m]);
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                const bool pml_here = ax == 0 ? pml_x : (ax == 1 ? pml_y : pml_z);
                if (pml_here) Io<SS>::st(wr_at(A.psip[ax] + pk + row, TMA ? 0LL : A.wofs), pp[ax]);
            }
        }
#pragma unroll
        for (int j = 0; j < 7; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) qz[j][e] = qz[j + 1][e];
    }
    cp_wait<0>();
    if (TMA && timed_out) {
        atomicExch(&A.mon->timeout, 1);
        for (int k = max(z0, z1 - 2); k < z1; ++k) mbar_wait_bounded(bars + (k & 1), (unsigned)((k - z0) >> 1) & 1u);
        if constexpr (L::RINGS)
            for (int kk = max(z0 - 1, z1 - 3); kk <= z1; ++kk) mbar_wait_bounded(bars + 2 + (kk & 3), ring_parity(kk));
    }
    // ---- stability monitor: one atomic per warp ----
    float m = bad ? 0.0f : (float)fmin(pmax, R(3.0e38));
    unsigned any_bad = __ballot_sync(0xffffffffu, bad);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x + threadIdx.y * BX) % 32 == 0) {
        if (m > 0.0f) atomicMax(&A.mon->max_bits, __float_as_uint(m));
        if (any_bad) atomicExch(&A.mon->nonfinite, 1);
    }
}

// ---------------------------------------------------------------------------
// sources, receivers, step counter

template <typename SS, typename R>
__global__ void k_sources(SS *p, const long long *idx, const R *gain, const int *wave_of,
                          const R *waves, int wave_len, int n_src, const int *d_it, int j, long long vol,
                          Monitor *mon)
{
    const int it = *d_it + j;
    if (it >= wave_len) return;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_src; s += gridDim.x * blockDim.x) {
        const long long k = idx[s];
        if (it < 0 || k < 0 || k >= vol) {     // never for a consistent medium: record, skip
            atomicExch(&mon->bad_index, 1);
            continue;
        }
        p[k] = SS(R(p[k]) + gain[s] * waves[(size_t)wave_of[s] * wave_len + it]);
    }
}

// Injection and recording of step it = *d_it + j in one launch: threads
// [0, n_src) inject the sources (and record the receiver on a source's cell,
// src_rcv, after the injection); threads [n_src, n_src + n_rcv) record the
// other receivers.  No two threads touch one cell.
template <typename SS, typename R>
__global__ void k_io(SS *p, const long long *src_idx, const R *gain, const int *wave_of, const R *waves,
                     int wave_len, int n_src, const int *src_rcv, const long long *rcv_idx, const int *rcv_src,
                     SS *traces, int n_rcv, int n_rec, int decim, const int *d_it, int j, long long vol,
                     Monitor *mon)
{
    const int it = *d_it + j;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (it < 0) {
        if (t == 0) atomicExch(&mon->bad_index, 1);
        return;
    }
    const bool rec = n_rcv > 0 && it % decim == 0 && it / decim < n_rec;
    const size_t col = rec ? (size_t)(it / decim) : 0;
    if (t < n_src) {
        const long long k = src_idx[t];
        if (k < 0 || k >= vol) {     // never for a consistent medium: record, skip
            atomicExch(&mon->bad_index, 1);
            return;
        }
        const int r = rec ? src_rcv[t] : -1;
        if (it < wave_len) {
            const SS v = SS(R(p[k]) + gain[t] * waves[(size_t)wave_of[t] * wave_len + it]);
            p[k] = v;
            if (r >= 0) traces[(size_t)r * n_rec + col] = v;
        } else if (r >= 0) {
            traces[(size_t)r * n_rec + col] = p[k];
        }
    } else if (rec && t < n_src + n_rcv) {
        const int r = t - n_src;
        if (rcv_src[r] >= 0) return;     // recorded by the thread of the source on its cell
        const long long k = rcv_idx[r];
        if (k < 0 || k >= vol) {
            atomicExch(&mon->bad_index, 1);
            return;
        }
        traces[(size_t)r * n_rec + col] = p[k];
    }
}

__global__ void k_advance(int *d_it, int n);

}  // namespace fwgb
