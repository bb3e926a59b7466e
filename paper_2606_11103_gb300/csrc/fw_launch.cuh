// Launch helpers: build kernel arguments from a medium and dispatch the
// template instance for (dimension, mechanisms, nonlinearity).  Included by
// one translation unit per storage type so that they compile in parallel.
#pragma once

#include "fw_kernels.cuh"

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

// which: bit 0 = velocity sweep, bit 1 = pressure sweep, bit 2 = only opt the
// instances into their dynamic shared memory (done once at medium creation,
// outside any stream capture)
template <typename R, typename SS, typename SP, int DIM, int NM, bool TS>
cudaError_t launch_dn(const fw_medium *m, cudaStream_t s, int which)
{
    constexpr int BX = DIM == 3 ? Tile3<R>::BX : Tile2<R>::BX;
    constexpr int BYV = DIM == 3 ? Tile3<R>::BYV : Tile2<R>::BYV;
    constexpr int BYP = DIM == 3 ? Tile3<R>::BYP : Tile2<R>::BYP;
    using LV = VelSmem<R, SS, SP, DIM, NM, BX, BYV, TS>;
    using LP = PresSmem<R, SS, SP, DIM, NM, BX, BYP, TS>;
    if (which & 4) {
        cudaError_t e = cudaFuncSetAttribute(k_velocity<R, SS, SP, DIM, NM, BX, BYV, TS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LV::bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_pressure<R, SS, SP, DIM, NM, BX, BYP, true, TS>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LP::bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_pressure<R, SS, SP, DIM, NM, BX, BYP, false, TS>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LP::bytes);
        return e;
    }
    const Geo<R> g = make_geo<R>(m);
    const int gx = (m->NX + 4 * BX - 1) / (4 * BX), gz = (m->NZ + m->zseg - 1) / m->zseg;

    VelArgs<R, SS, SP> va{};
    va.g = g;
    va.p = static_cast<const SS *>(m->p);
    for (int ax = 0; ax < 3; ++ax) {
        va.v[ax] = static_cast<SS *>(m->v[ax]);
        va.psip[ax] = static_cast<SS *>(m->psi1p[ax]);
        va.pd[ax] = static_cast<const R *>(m->prof[ax][0]);
        va.pa[ax] = static_cast<const R *>(m->prof[ax][1]);
        for (int n = 0; n < NM; ++n) va.psi[n][ax] = static_cast<SP *>(m->psi1[n][ax]);
    }
    va.rho = static_cast<const SS *>(m->rho);
    va.cls = m->cls;
    va.lut = static_cast<const R *>(m->lut);
    va.kdt = static_cast<const SS *>(m->kdt);
    if (which & 1)
        k_velocity<R, SS, SP, DIM, NM, BX, BYV, TS><<<dim3(gx, (m->NY + BYV - 1) / BYV, gz), dim3(BX, BYV), LV::bytes, s>>>(va);
    if (!(which & 2)) return cudaGetLastError();

    PresArgs<R, SS, SP> pa{};
    pa.g = g;
    pa.p = static_cast<SS *>(m->p);
    for (int ax = 0; ax < 3; ++ax) {
        pa.v[ax] = static_cast<const SS *>(m->v[ax]);
        pa.psip[ax] = static_cast<SS *>(m->psi2p[ax]);
        pa.pd[ax] = static_cast<const R *>(m->prof[ax][2]);
        pa.pa[ax] = static_cast<const R *>(m->prof[ax][3]);
    }
    for (int n = 0; n < NM; ++n) pa.psi[n] = static_cast<SP *>(m->psi2[n]);
    pa.kdt = static_cast<const SS *>(m->kdt);
    pa.b2dt = static_cast<const SS *>(m->b2dt);
    pa.cls = m->cls;
    pa.lut = static_cast<const R *>(m->lut);
    pa.mon = m->mon;
    pa.rho = static_cast<const SS *>(m->rho);
    const dim3 gp(gx, (m->NY + BYP - 1) / BYP, gz), bp(BX, BYP);
    if (m->nonlinear)
        k_pressure<R, SS, SP, DIM, NM, BX, BYP, true, TS><<<gp, bp, LP::bytes, s>>>(pa);
    else
        k_pressure<R, SS, SP, DIM, NM, BX, BYP, false, TS><<<gp, bp, LP::bytes, s>>>(pa);
    return cudaGetLastError();
}

template <typename R, typename SS, typename SP, bool TS>
cudaError_t launch_ts(const fw_medium *m, cudaStream_t s, int which)
{
    const bool d3 = m->ndim == 3;
    switch (m->nmech) {
    case 1: return d3 ? launch_dn<R, SS, SP, 3, 1, TS>(m, s, which) : launch_dn<R, SS, SP, 2, 1, TS>(m, s, which);
    case 2: return d3 ? launch_dn<R, SS, SP, 3, 2, TS>(m, s, which) : launch_dn<R, SS, SP, 2, 2, TS>(m, s, which);
    case 3: return d3 ? launch_dn<R, SS, SP, 3, 3, TS>(m, s, which) : launch_dn<R, SS, SP, 2, 3, TS>(m, s, which);
    case 4: return d3 ? launch_dn<R, SS, SP, 3, 4, TS>(m, s, which) : launch_dn<R, SS, SP, 2, 4, TS>(m, s, which);
    default: return cudaErrorInvalidValue;
    }
}

// leapfrog instances, or those of the time-space stencil (time_order 4)
template <typename R, typename SS, typename SP>
cudaError_t launch_sweeps(const fw_medium *m, cudaStream_t s, int which)
{
    return m->time_order == 4 ? launch_ts<R, SS, SP, true>(m, s, which) : launch_ts<R, SS, SP, false>(m, s, which);
}

template <typename R, typename SS>
cudaError_t launch_io(const fw_medium *m, int j, cudaStream_t s)
{
    if (m->n_src > 0) {
        int nb = (m->n_src + 255) / 256;
        k_sources<SS, R><<<nb, 256, 0, s>>>(static_cast<SS *>(m->p), m->src_idx,
                                            static_cast<const R *>(m->src_gain), m->wave_of,
                                            static_cast<const R *>(m->waves), m->wave_len, m->n_src,
                                            m->d_it, j, (long long)m->vol, m->mon);
    }
    if (m->n_rcv > 0) {
        int nb = (m->n_rcv + 255) / 256;
        k_receivers<SS><<<nb, 256, 0, s>>>(static_cast<const SS *>(m->p), m->rcv_idx,
                                           static_cast<SS *>(m->traces), m->n_rcv, m->n_rec,
                                           m->decim, m->d_it, j, (long long)m->vol, m->mon);
    }
    return cudaGetLastError();
}

}  // namespace fwgb
