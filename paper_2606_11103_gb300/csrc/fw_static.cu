// Field read-back that allocates no device memory.
//
// fw_read_field() stages the unpadded copy of a field in a device buffer it
// allocates for the call.  Some callers cannot allocate device memory at that
// point: a process whose device memory is owned by another framework's
// caching allocator (the whole pool handed out), a real-time loop whose
// memory budget is fixed up front, or code that must not synchronise the
// device (cudaMalloc/cudaFree can).  fw_read_field_noalloc() serves them: it
// stages through one file-scope device array of fixed size instead.
#include "fw_internal.h"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>

namespace fwgb {
int field_lookup(fw_medium *m, int which, int idx, void **ptr, int *kind, double *read_scale);
}  // namespace fwgb

namespace {

// The staging array: FW_NOALLOC_MAX_BYTES bytes on every device that loads
// the library, held until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_stage[FW_NOALLOC_MAX_BYTES];

// Device address of g_noalloc_stage per device.  In host code the symbol is a
// host-side stand-in, not a device address, so it is looked up once per
// device with cudaGetSymbolAddress while that device is current.
constexpr int kMaxDevices = 64;
std::mutex g_stage_mu;
void *g_stage_addr[kMaxDevices] = {};

int stage_address(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return FW_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return FW_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_stage_mu);
    if (!g_stage_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_stage) != cudaSuccess || !p) {
            cudaGetLastError();
            return FW_ERR_CUDA;
        }
        g_stage_addr[dev] = p;
    }
    *out = g_stage_addr[dev];
    return FW_OK;
}

// padded field (row pitch px) -> dense C order, same arithmetic as the
// allocating read: value * scale in double, then rounded to D
template <typename S, typename D>
__global__ void k_unpad_to_stage(D *dst, const S *src, int nx, long long n, int px, double scale)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / nx;
        const int x = int(i - r * nx);
        dst[i] = D(double(src[r * px + x]) * scale);
    }
}

template <typename D>
cudaError_t unpad(const fw_medium *m, const void *src, int kind, D *dst, double scale, cudaStream_t s)
{
    const long long n = (long long)m->NX * m->NY * m->NZ;
    const int nb = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
    if (kind == 0 || m->storage == FW_STORE_F32 || m->storage == FW_STORE_F64) {
        if (m->es == 8)
            k_unpad_to_stage<double, D><<<nb, 256, 0, s>>>(dst, (const double *)src, m->NX, n, m->px, scale);
        else
            k_unpad_to_stage<float, D><<<nb, 256, 0, s>>>(dst, (const float *)src, m->NX, n, m->px, scale);
    } else if (m->storage == FW_STORE_BF16) {
        k_unpad_to_stage<__nv_bfloat16, D><<<nb, 256, 0, s>>>(dst, (const __nv_bfloat16 *)src, m->NX, n, m->px, scale);
    } else {
        k_unpad_to_stage<__half, D><<<nb, 256, 0, s>>>(dst, (const __half *)src, m->NX, n, m->px, scale);
    }
    return cudaGetLastError();
}

}  // namespace

namespace fwgb {
// Called by every medium creation with the medium's device current: the
// address lookup loads this file's module on the device (CUDA loads modules
// lazily, at their first use), so the staging array is resident from the
// first medium on, before a caller hands the rest of device memory to a
// pool.  A failure here is not the medium's: the read reports it.
void noalloc_prepare()
{
    void *p = nullptr;
    if (stage_address(&p) != FW_OK) cudaGetLastError();
}
}  // namespace fwgb

extern "C" int fw_read_field_noalloc(fw_medium *m, int which, int idx, void *dst, int as_f64, void *stream)
{
    if (!m || !dst) return FW_ERR_ARG;
    void *src = nullptr;
    int kind = 0;
    double scale = 1.0;
    int rc = fwgb::field_lookup(m, which, idx, &src, &kind, &scale);
    if (rc) return rc;
    const size_t n = (size_t)m->NX * m->NY * m->NZ;
    const size_t bytes = n * (as_f64 ? 8 : 4);
    if (bytes > (size_t)FW_NOALLOC_MAX_BYTES) return FW_ERR_SIZE;
    void *stage = nullptr;
    if ((rc = stage_address(&stage))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // every staged element is written before it is copied out: nothing in the
    // array has to start at zero
    cudaError_t e = as_f64 ? unpad<double>(m, src, kind, static_cast<double *>(stage), scale, s)
                           : unpad<float>(m, src, kind, static_cast<float *>(stage), scale, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, stage, bytes, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return FW_ERR_CUDA;
    }
    return FW_OK;
}
