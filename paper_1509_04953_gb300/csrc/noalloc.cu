// Allocation-free variant of evp_stress_residual, for callers that cannot allocate device
// memory themselves: typically a plug-in or library component whose host application owns
// every device allocation (its own pool, its own accounting) and does not let components call
// cudaMalloc, or a caller with no allocator of its own at hand. evp_stress_residual needs a
// small caller-owned scratch buffer for its per-block partial sums; this entry point uses a
// fixed array that lives in the library's own device memory instead.
#include <cuda.h>
#include <mutex>

#include "../../include/evp.h"
#include "kernels.h"

namespace {

// Partial sums of the z pass, one double per CTA: fft_z_blocks(n) <= 256 * (128/4) = 8192
// for n <= 256 in any precision. Every GPU that loads the library holds this array until exit.
constexpr int kMaxPartials = 8192;
static __device__ __align__(256) double g_resid_partials[kMaxPartials];

// Host code cannot use g_resid_partials as a device address: the name is only a host-side
// stand-in. The device address is looked up once per device, with that device current, and
// cached together with the id of the context it belongs to. A device reset (or any other way
// the context is destroyed and re-created) gives the new context a new id, so the next call
// looks the address up again instead of using a stale one.
constexpr int kMaxDevices = 64;
struct Slot {
    unsigned long long ctx_id;   // 0: no context id known (the address is looked up on every call)
    double *ptr;
};
Slot g_slot[kMaxDevices] = {};
std::mutex g_mu;

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Id of the context current on this thread, through the driver entry points the runtime hands
// out (the library does not link libcuda itself); 0 when there is none or the driver lacks them.
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
            get_id = reinterpret_cast<CtxGetIdFn>(f2);
        }
        looked_up = true;
    }
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

int partials_for_current_device(double **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return EVP_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    unsigned long long id = current_context_id();
    Slot &s = g_slot[dev];
    if (id == 0 || s.ptr == nullptr || s.ctx_id != id) {
        void *p = nullptr;
        // also makes the device's primary context current on this thread if none was
        if (cudaGetSymbolAddress(&p, g_resid_partials) != cudaSuccess || p == nullptr) return EVP_ERR_CUDA;
        s.ptr = static_cast<double *>(p);
        s.ctx_id = current_context_id();
    }
    *out = s.ptr;
    return EVP_OK;
}

}  // namespace

extern "C" int evp_stress_residual_noalloc(int n, int precision, const void *sig_dev, void *spec_dev, double *out_dev,
                                           void *cuda_stream) {
    const bool pow2 = n >= 4 && n <= 256 && (n & (n - 1)) == 0;
    if (!pow2 || !sig_dev || !spec_dev || !out_dev) return EVP_ERR_ARG;
    if (precision < EVP_FP64 || precision > EVP_MIXED_FAST) return EVP_ERR_ARG;
    const int dbl = precision == EVP_FP64;
    const int nparts = evp::fft_z_blocks(n, dbl);
    if (nparts > kMaxPartials) return EVP_ERR_ARG;   // larger than the fixed scratch array
    double *part = nullptr;
    const int rc = partials_for_current_device(&part);
    if (rc != EVP_OK) return rc;
    // Every slot the reduction reads is written by this call's z pass first, so the array needs
    // no clearing; it keeps whatever the last call left in it.
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e;
    if (dbl) {
        e = evp::fft_xy_r2c<double>((const double *)sig_dev, spec_dev, n, 6, s);
        if (e == cudaSuccess) e = evp::fft_z<double>(spec_dev, n, 6, evp::Z_FWD_RESID, 0, 0, part, out_dev, s);
    } else {
        e = evp::fft_xy_r2c<float>((const float *)sig_dev, spec_dev, n, 6, s);
        if (e == cudaSuccess) e = evp::fft_z<float>(spec_dev, n, 6, evp::Z_FWD_RESID, 0, 0, part, out_dev, s);
    }
    if (e == cudaSuccess) e = evp::reduce_partials(part, nparts, 1, out_dev + 6, s);
    return e == cudaSuccess ? EVP_OK : EVP_ERR_CUDA;
}
