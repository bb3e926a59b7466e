// Launch helpers: build kernel arguments from a medium and dispatch the
// template instance for (dimension, mechanisms, nonlinearity).  Included by
// one translation unit per storage type so that they compile in parallel.
#pragma once

#include "fw_kernels.cuh"

#include <cuda.h>

namespace fwgb {

// rows of the 3D CTA tiles (tuning knobs, measured best): the velocity sweep
// runs two 128x4 CTAs per SM, the pressure sweep three 128x4 CTAs per SM
#ifndef FWGB_VEL3_BY
#define FWGB_VEL3_BY 4
#endif
#ifndef FWGB_PRES3_BY
#define FWGB_PRES3_BY 4
#endif
template <typename R> struct Tile3 {
    static constexpr int BX = sizeof(R) == 8 ? 16 : 32, BYV = FWGB_VEL3_BY, BYP = FWGB_PRES3_BY;
};
template <typename R> struct Tile2 { static constexpr int BX = 64, BYV = 1, BYP = 1; };

template <typename R> Geo<R> make_geo(const fw_medium *m)
{
    Geo<R> g{};
    g.nx = m->NX;
    g.ny = m->NY;
    g.nz = m->NZ;
    g.px = m->px;
    g.plane = (long long)m->plane;
    g.zseg = m->zseg;
    g.wabs = m->wabs;
    // 8th-order staggered weights (Taylor) divided by dx
    const double cm[4] = {1225.0 / 1024.0, -245.0 / 3072.0, 49.0 / 5120.0, -5.0 / 7168.0};
    g.c1 = R(cm[0] / m->dx);
    g.c2 = R(cm[1] / m->dx);
    g.c3 = R(cm[2] / m->dx);
    g.c4 = R(cm[3] / m->dx);
    g.dt = R(m->dt);
    g.lr = R(m->g.transition > 0 ? m->g.transition : 0.5 * m->g.pml);
    for (int i = 0; i < 4; ++i)
        for (int n = 0; n < 4; ++n) g.ta[i][n] = R(m->ts_a[i][n] / m->dx);
    g.tb = R(1.0 / (24.0 * m->dx));
    g.r2s = R(m->dt / (m->dx * m->dx));
    return g;
}

// Tensor maps of the streams the 3D velocity sweep stages by TMA: every
// array is addressed as a 3D tensor (px, NY, NZ) with the medium's pitches;
// boxes are the CTA tile (TW x BY) or its halo boxes (p: (TW+8) x (BY+7)
// from (xb-4, yb-3); rho: (TW+4) x (BY+1) from (xb, yb)).  Elements outside
// the tensor read as zero.  encode is the driver's tensor-map encoder.
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

template <typename T> constexpr CUtensorMapDataType map_type();
template <> constexpr CUtensorMapDataType map_type<float>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT32; }
template <> constexpr CUtensorMapDataType map_type<__nv_bfloat16>() { return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; }
template <> constexpr CUtensorMapDataType map_type<__half>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT16; }
template <> constexpr CUtensorMapDataType map_type<uint16_t>() { return CU_TENSOR_MAP_DATA_TYPE_UINT16; }

template <typename T>
bool encode_map(EncodeTiledFn encode, TensorMapBlob *out, const fw_medium *m, const void *base, unsigned bx,
                unsigned by)
{
    const cuuint64_t dims[3] = {(cuuint64_t)m->px, (cuuint64_t)m->NY, (cuuint64_t)m->NZ};
    const cuuint64_t strides[2] = {(cuuint64_t)m->px * sizeof(T), (cuuint64_t)m->plane * sizeof(T)};
    const cuuint32_t box[3] = {bx, by, 1}, estr[3] = {1, 1, 1};
    return encode(reinterpret_cast<CUtensorMap *>(out), map_type<T>(), 3, const_cast<void *>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename R, typename SS, typename SP>
bool build_vel_maps_t(EncodeTiledFn encode, fw_medium *m)
{
    if constexpr (sizeof(R) != 4) {
        return false;
    } else {
        constexpr int TW = 4 * Tile3<R>::BX, BY = Tile3<R>::BYV;
        VelMaps &v = m->vel_maps;
        bool ok = encode_map<SS>(encode, &v.p_halo, m, m->p, TW + 8, BY + 7) &&
                  encode_map<SS>(encode, &v.p_own, m, m->p, TW, BY) &&
                  encode_map<SS>(encode, &v.rho_halo, m, m->rho, TW + 4, BY + 1) &&
                  encode_map<SS>(encode, &v.rho_own, m, m->rho, TW, BY) &&
                  encode_map<uint16_t>(encode, &v.cls, m, m->cls, TW, BY) &&
                  encode_map<SS>(encode, &v.kdt, m, m->kdt, TW, BY);
        for (int ax = 0; ax < 3 && ok; ++ax) {
            ok = encode_map<SS>(encode, &v.v[ax], m, m->v[ax], TW, BY);
            for (int n = 0; n < m->nmech && ok; ++n) ok = encode_map<SP>(encode, &v.psi[n][ax], m, m->psi1[n][ax], TW, BY);
        }
        // pressure sweep: v_x box with 4 columns either side, v_y box with
        // 4 rows below and 3 above
        constexpr int BP = Tile3<R>::BYP;
        PresMaps &q = m->pres_maps;
        ok = ok && encode_map<SS>(encode, &q.vz_own, m, m->v[2], TW, BP) &&
             encode_map<SS>(encode, &q.vx_halo, m, m->v[0], TW + 8, BP) &&
             encode_map<SS>(encode, &q.vy_halo, m, m->v[1], TW, BP + 7) &&
             encode_map<SS>(encode, &q.p_own, m, m->p, TW, BP) && encode_map<SS>(encode, &q.kdt, m, m->kdt, TW, BP) &&
             encode_map<uint16_t>(encode, &q.cls, m, m->cls, TW, BP) &&
             encode_map<SS>(encode, &q.rho_own, m, m->rho, TW, BP) &&
             (!m->nonlinear || encode_map<SS>(encode, &q.b2dt, m, m->b2dt, TW, BP));
        for (int n = 0; n < m->nmech && ok; ++n) ok = encode_map<SP>(encode, &q.psi[n], m, m->psi2[n], TW, BP);
        if (m->time_order == 4)       // the time-space stencil's rings of v planes
            ok = ok && encode_map<SS>(encode, &q.vx_ring, m, m->v[0], TW + 8, BP + 2) &&
                 encode_map<SS>(encode, &q.vy_ring, m, m->v[1], TW + 8, BP + 7) &&
                 encode_map<SS>(encode, &q.vz_ring, m, m->v[2], TW + 8, BP + 2);
        return ok;
    }
}

// which: bit 0 = velocity sweep, bit 1 = pressure sweep, bit 2 = only opt the
// instances into their dynamic shared memory (done once at medium creation,
// outside any stream capture).  im (may be null): a step from one state
// image into another (StepImages) instead of the in-place step of the
// medium's own state.
template <typename R, typename SS, typename SP, int DIM, int NM, bool TS>
cudaError_t launch_dn(const fw_medium *m, cudaStream_t s, int which, const StepImages *im)
{
    constexpr int BX = DIM == 3 ? Tile3<R>::BX : Tile2<R>::BX;
    constexpr int BYV = DIM == 3 ? Tile3<R>::BYV : Tile2<R>::BYV;
    constexpr int BYP = DIM == 3 ? Tile3<R>::BYP : Tile2<R>::BYP;
    // the 3D FP32-state velocity sweep stages its streams by TMA when the
    // medium holds tensor maps for them (the cp.async instance otherwise)
    constexpr bool CAN_TMA = DIM == 3 && sizeof(R) == 4;
    using LV = VelSmem<R, SS, SP, DIM, NM, BX, BYV, TS>;
    using LVT = VelSmem<R, SS, SP, DIM, NM, BX, BYV, TS, CAN_TMA>;
    using LP = PresSmem<R, SS, SP, DIM, NM, BX, BYP, TS>;
    using LPT = PresSmem<R, SS, SP, DIM, NM, BX, BYP, TS, CAN_TMA>;
    if (which & 4) {
        cudaError_t e = cudaFuncSetAttribute(k_velocity<R, SS, SP, DIM, NM, BX, BYV, TS, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LV::bytes);
        if constexpr (CAN_TMA)
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_velocity<R, SS, SP, DIM, NM, BX, BYV, TS, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LVT::bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_pressure<R, SS, SP, DIM, NM, BX, BYP, true, TS, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LP::bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_pressure<R, SS, SP, DIM, NM, BX, BYP, false, TS, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LP::bytes);
        if constexpr (CAN_TMA) {
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_pressure<R, SS, SP, DIM, NM, BX, BYP, true, TS, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LPT::bytes);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_pressure<R, SS, SP, DIM, NM, BX, BYP, false, TS, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LPT::bytes);
        }
        return e;
    }
    const Geo<R> g = make_geo<R>(m);
    const int gx = (m->NX + 4 * BX - 1) / (4 * BX), gz = (m->NZ + m->zseg - 1) / m->zseg;
    // a state array of the medium, or the same array in the image read (rd)
    // or written (nw) by an image step
    const char *slab = static_cast<const char *>(m->slab);
    auto rd = [&](void *a) -> void * {
        return (a && im) ? const_cast<char *>(im->rd) + (static_cast<const char *>(a) - slab) : a;
    };
    auto nw = [&](void *a) -> void * { return (a && im) ? static_cast<char *>(rd(a)) + im->wofs : a; };
    const long long wofs = im ? im->wofs : 0;
    const bool tma = m->tma && !im;   // tensor maps address the medium's own arrays

    VelArgs<R, SS, SP> va{};
    va.g = g;
    va.p = static_cast<const SS *>(rd(m->p));
    va.wofs = wofs;
    for (int ax = 0; ax < 3; ++ax) {
        va.v[ax] = static_cast<SS *>(rd(m->v[ax]));
        va.psip[ax] = static_cast<SS *>(rd(m->psi1p[ax]));
        va.pd[ax] = static_cast<const R *>(m->prof[ax][0]);
        va.pa[ax] = static_cast<const R *>(m->prof[ax][1]);
        for (int n = 0; n < NM; ++n) va.psi[n][ax] = static_cast<SP *>(rd(m->psi1[n][ax]));
    }
    va.rho = static_cast<const SS *>(m->rho);
    va.cls = m->cls;
    va.lut = static_cast<const R *>(m->lut);
    va.kdt = static_cast<const SS *>(m->kdt);
    va.mon = m->mon;
    if (which & 1) {
        const dim3 gv(gx, (m->NY + BYV - 1) / BYV, gz), bv(BX, BYV);
        bool done = false;
        if constexpr (CAN_TMA) {
            if (tma) {
                va.maps = m->vel_maps;
                k_velocity<R, SS, SP, DIM, NM, BX, BYV, TS, true><<<gv, bv, LVT::bytes, s>>>(va);
                done = true;
            }
        }
        if (!done) k_velocity<R, SS, SP, DIM, NM, BX, BYV, TS, false><<<gv, bv, LV::bytes, s>>>(va);
    }
    if (!(which & 2)) return cudaGetLastError();

    PresArgs<R, SS, SP> pa{};
    pa.g = g;
    pa.p = static_cast<SS *>(rd(m->p));
    pa.wofs = wofs;
    for (int ax = 0; ax < 3; ++ax) {
        pa.v[ax] = static_cast<const SS *>(nw(m->v[ax]));   // this step's velocity
        pa.psip[ax] = static_cast<SS *>(rd(m->psi2p[ax]));
        pa.pd[ax] = static_cast<const R *>(m->prof[ax][2]);
        pa.pa[ax] = static_cast<const R *>(m->prof[ax][3]);
    }
    for (int n = 0; n < NM; ++n) pa.psi[n] = static_cast<SP *>(rd(m->psi2[n]));
    pa.kdt = static_cast<const SS *>(m->kdt);
    pa.b2dt = static_cast<const SS *>(m->b2dt);
    pa.cls = m->cls;
    pa.lut = static_cast<const R *>(m->lut);
    pa.mon = m->mon;
    pa.rho = static_cast<const SS *>(m->rho);
    const dim3 gp(gx, (m->NY + BYP - 1) / BYP, gz), bp(BX, BYP);
    if constexpr (CAN_TMA) {
        if (tma) {
            pa.maps = m->pres_maps;
            if (m->nonlinear)
                k_pressure<R, SS, SP, DIM, NM, BX, BYP, true, TS, true><<<gp, bp, LPT::bytes, s>>>(pa);
            else
                k_pressure<R, SS, SP, DIM, NM, BX, BYP, false, TS, true><<<gp, bp, LPT::bytes, s>>>(pa);
            return cudaGetLastError();
        }
    }
    if (m->nonlinear)
        k_pressure<R, SS, SP, DIM, NM, BX, BYP, true, TS, false><<<gp, bp, LP::bytes, s>>>(pa);
    else
        k_pressure<R, SS, SP, DIM, NM, BX, BYP, false, TS, false><<<gp, bp, LP::bytes, s>>>(pa);
    return cudaGetLastError();
}

template <typename R, typename SS, typename SP, bool TS>
cudaError_t launch_ts(const fw_medium *m, cudaStream_t s, int which, const StepImages *im)
{
    const bool d3 = m->ndim == 3;
    switch (m->nmech) {
    case 1: return d3 ? launch_dn<R, SS, SP, 3, 1, TS>(m, s, which, im) : launch_dn<R, SS, SP, 2, 1, TS>(m, s, which, im);
    case 2: return d3 ? launch_dn<R, SS, SP, 3, 2, TS>(m, s, which, im) : launch_dn<R, SS, SP, 2, 2, TS>(m, s, which, im);
    case 3: return d3 ? launch_dn<R, SS, SP, 3, 3, TS>(m, s, which, im) : launch_dn<R, SS, SP, 2, 3, TS>(m, s, which, im);
    case 4: return d3 ? launch_dn<R, SS, SP, 3, 4, TS>(m, s, which, im) : launch_dn<R, SS, SP, 2, 4, TS>(m, s, which, im);
    default: return cudaErrorInvalidValue;
    }
}

// leapfrog instances, or those of the time-space stencil (time_order 4)
template <typename R, typename SS, typename SP>
cudaError_t launch_sweeps(const fw_medium *m, cudaStream_t s, int which, const StepImages *im = nullptr)
{
    return m->time_order == 4 ? launch_ts<R, SS, SP, true>(m, s, which, im)
                              : launch_ts<R, SS, SP, false>(m, s, which, im);
}

// One leapfrog step from the state image at im.rd into the one at
// im.rd + im.wofs (both laid out as the medium's state), sources included at
// step it (absolute); receivers are not recorded and the images' step
// counters are not used.  For the adjoint's recomputation: no copy of the
// state per step, the medium's own state untouched.
template <typename R, typename SS>
cudaError_t launch_image_step(const fw_medium *m, const StepImages &im, const int *zero, int it, cudaStream_t s)
{
    cudaError_t e = launch_sweeps<R, SS, SS>(m, s, 3, &im);
    if (e != cudaSuccess || m->n_src <= 0) return e;
    SS *p = reinterpret_cast<SS *>(const_cast<char *>(im.rd) + im.wofs +
                                   (static_cast<const char *>(m->p) - static_cast<const char *>(m->slab)));
    k_sources<SS, R><<<(m->n_src + 255) / 256, 256, 0, s>>>(p, m->src_idx, static_cast<const R *>(m->src_gain),
                                                           m->wave_of, static_cast<const R *>(m->waves),
                                                           m->wave_len, m->n_src, zero, it, (long long)m->vol,
                                                           m->mon);
    return cudaGetLastError();
}

template <typename R, typename SS>
cudaError_t launch_io(const fw_medium *m, int j, cudaStream_t s)
{
    const int n = m->n_src + m->n_rcv;
    if (n <= 0) return cudaSuccess;
    k_io<SS, R><<<(n + 255) / 256, 256, 0, s>>>(static_cast<SS *>(m->p), m->src_idx,
                                                 static_cast<const R *>(m->src_gain), m->wave_of,
                                                 static_cast<const R *>(m->waves), m->wave_len, m->n_src, m->src_rcv,
                                                 m->rcv_idx, m->rcv_src, static_cast<SS *>(m->traces), m->n_rcv,
                                                 m->n_rec, m->decim, m->d_it, j, (long long)m->vol, m->mon);
    return cudaGetLastError();
}

}  // namespace fwgb
