// Internal declarations shared by the library's translation units.
#pragma once

#include "../../include/fullwave_gb.h"

#include <atomic>
#include <functional>
#include <map>
#include <vector>

#include <cuda_runtime.h>

namespace fwgb {

// ---- calibration (fw_fit.cpp) ----------------------------------------------
struct FitJob {
    fw_relax_params p;
    double J, w, nrmse, disp;
    int n_iter, n_eval;
};
void default_opts(fw_fit_opts *o);
fw_relax_params lossless_params(int n);
FitJob run_weight(double alpha0, double y, int n_mech, const fw_fit_opts &o, int wi);
void select_fit(const std::vector<FitJob> &res, fw_relax_params *out, fw_fit_report *rep);
void parallel_for(int n_jobs, int n_threads, const std::function<void(int)> &fn);
int fit_check(double alpha0, double y, int n_mech, const fw_fit_opts &o);
int nelder_mead(int n, double *x, const double *lo, const double *hi,
                double (*f)(const double *, void *), void *ctx, int maxiter,
                double xatol, double fatol, double *fmin, int *n_iter, int *n_eval);

// ---- device layout ---------------------------------------------------------
constexpr int kLutStride = 32;   // values per class in the coefficient table
// table block offsets (in values): 0 kappa1, 1 kappa2, 2 ceff1, 3 ceff2,
// 4.. a1[4], 8.. b1[4], 12.. hb1[4], 16.. a2[4], 20.. b2[4], 24.. hb2[4],
// 28 sum a1/2, 29 sum a2/2 (= ceff - 1/kappa, the part the layer ramp scales)
constexpr int kLutA1 = 4, kLutB1 = 8, kLutH1 = 12, kLutA2 = 16, kLutB2 = 20, kLutH2 = 24, kLutDk = 28;

struct Monitor {
    unsigned int max_bits;   // bits of max |p| (non-negative float)
    int nonfinite;
    int bad_index;           // a source/receiver index or step counter out of range (skipped)
    int timeout;             // a bounded wait of a sweep on its staged copies gave up
};

// Tensor-map descriptors of the staged streams of the 3D velocity sweep
// (opaque 128-byte driver objects, built on the host at medium creation):
// p with its x/y halo box and p own box, v_d, psi1[m][d], rho with its +1
// halo box and rho own box, the class index and K dt.
struct alignas(64) TensorMapBlob {
    unsigned char bytes[128];
};
struct VelMaps {
    TensorMapBlob p_halo, p_own, v[3], psi[FW_MAX_MECH][3], rho_halo, rho_own, cls, kdt;
};
// ... and of the 3D pressure sweep: v_z own box (planes ahead), v_x with its
// x halo, v_y with its y halo, p, K dt, 2 beta dt, psi2[m], the class index,
// rho (time-space stencil)
struct PresMaps {
    TensorMapBlob vz_own, vx_halo, vy_halo, p_own, kdt, b2dt, psi[FW_MAX_MECH], cls, rho_own;
    TensorMapBlob vx_ring, vy_ring, vz_ring;   // time-space stencil: v boxes with x and y halos
};

// A step between two state images (buffers laid out as the medium's state):
// every state array is read at its offset in the image at rd and written at
// the same offset in the image wofs bytes further on; maps and tables stay
// the medium's.
struct StepImages {
    const char *rd;
    long long wofs;
};

struct Graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

}  // namespace fwgb

struct fw_medium {
    fw_grid g{};
    int ndim = 0, nmech = 0, storage = 0;
    bool nonlinear = false;
    int NX = 0, NY = 0, NZ = 0;     // kernel axes: x, y (1 in 2D), depth
    int px = 0;                      // row pitch in elements
    size_t plane = 0, vol = 0;       // elements per plane / per array (padded)
    int es = 4, eps = 4;             // element bytes of state and of psi
    double dt = 0, dx = 0, c_max = 0, ceff_max = 0;
    int n_classes = 0;
    int wabs = 0;                    // transition + absorbing cells
    // device memory
    void *slab = nullptr;
    size_t slab_bytes = 0;
    void *p = nullptr, *v[3] = {}, *psi1[FW_MAX_MECH][3] = {}, *psi2[FW_MAX_MECH] = {};
    void *psi1p[3] = {}, *psi2p[3] = {};
    void *kdt = nullptr, *rho = nullptr, *b2dt = nullptr, *lut = nullptr;
    void *cdev = nullptr;            // c map (kept for the class coefficient rebuilds)
    uint16_t *cls = nullptr;
    void *prof[3][4] = {};           // per kernel axis: d, alpha at half points; d, alpha at integer points
    int *d_it = nullptr;
    fwgb::Monitor *mon = nullptr;
    std::vector<fw_relax_params> classes;
    // sources / receivers
    void *src_buf = nullptr, *rcv_buf = nullptr;
    long long *src_idx = nullptr, *rcv_idx = nullptr;
    void *src_gain = nullptr, *waves = nullptr, *traces = nullptr;
    int *wave_of = nullptr;
    int n_src = 0, n_wave = 0, wave_len = 0;
    int n_rcv = 0, n_rec = 0, decim = 1;
    // cells that hold both a source and a receiver: per source the receiver
    // there (or -1), per receiver the source there (or -1); host copies of
    // both index lists to rebuild them
    int *src_rcv = nullptr, *rcv_src = nullptr;
    std::vector<long long> h_src_idx, h_rcv_idx;
    // bookkeeping
    long long step = 0;
    int sticky = 0;
    cudaStream_t last_stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    std::map<int, fwgb::Graph> graphs;
    int zseg = 32;
    double psi_pref = 10.0;          // pressure reference [Pa] of binary16 memory variables
    int time_order = 2;              // 2: leapfrog; 4: time-space stencil (Sec. 3.3)
    double ts_a[4][4] = {};          // time-space weights a_m = sum_n ts_a[m][n] r^(2n)
    bool tma = false;                // 3D sweeps staged by tensor-memory-access copies
    fwgb::VelMaps vel_maps{};
    fwgb::PresMaps pres_maps{};
};
