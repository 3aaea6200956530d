// Allocation-free variant of evp_stress_residual, for callers that cannot allocate device
// memory themselves: code running where cudaMalloc is unavailable or forbidden (for instance
// inside a host callback, a signal-safe or real-time section, or a plug-in whose host
// application owns every device allocation), or a caller with no allocator of its own at hand.
// evp_stress_residual needs a small caller-owned scratch buffer for its per-block partial sums;
// this entry point uses a fixed array that lives in the library's own device memory instead.
#include <mutex>

#include "../../include/evp.h"
#include "kernels.h"

namespace {

// Partial sums of the z pass, one double per CTA: fft_z_blocks(n) <= 256 * (128/4) = 8192
// for n <= 256 in any precision. Every GPU that loads the library holds this array until exit.
constexpr int kMaxPartials = 8192;
static __device__ __align__(256) double g_resid_partials[kMaxPartials];

// Host code cannot use g_resid_partials as a device address: the name is only a host-side
// stand-in. The device address is looked up once per device, with that device current.
constexpr int kMaxDevices = 64;
double *g_dev_ptr[kMaxDevices] = {};
std::mutex g_mu;

int partials_for_current_device(double **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return EVP_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_resid_partials) != cudaSuccess || p == nullptr) return EVP_ERR_CUDA;
        g_dev_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_dev_ptr[dev];
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
        e = evp::fft_x_r2c<double>((const double *)sig_dev, spec_dev, n, 6, s);
        if (e == cudaSuccess) e = evp::fft_y<double>(spec_dev, n, 6, 0, s);
        if (e == cudaSuccess) e = evp::fft_z<double>(spec_dev, n, 6, evp::Z_FWD_RESID, 0, 0, part, out_dev, s);
    } else {
        e = evp::fft_x_r2c<float>((const float *)sig_dev, spec_dev, n, 6, s);
        if (e == cudaSuccess) e = evp::fft_y<float>(spec_dev, n, 6, 0, s);
        if (e == cudaSuccess) e = evp::fft_z<float>(spec_dev, n, 6, evp::Z_FWD_RESID, 0, 0, part, out_dev, s);
    }
    if (e == cudaSuccess) e = evp::reduce_partials(part, nparts, 1, out_dev + 6, s);
    return e == cudaSuccess ? EVP_OK : EVP_ERR_CUDA;
}
