// Fixed-point control of the basic scheme, on the device (Sec. 2.1 iteration with the mixed boundary
// conditions). After an iteration's z pass has written its partial sums, one block sums them (in a fixed
// order) into sum |xi.sigma_hat|^2; its first thread turns that and the mean stress into err_eq and
// err_bc, decides convergence and computes the correction dE_k of the macroscopic strain on the
// stress-controlled components. The correction goes into the zero-frequency term of the Green-operator
// output, which the z pass leaves at zero; after the z pass's own inverse transform that term is the
// (ky, kx) = (0, 0) entry of every z plane, so the inverse y and x transforms add it to every voxel's
// strain. The host queues iterations in batches and reads this block once per batch; once `done` is set,
// the kernels of the iterations still queued return at once.
#pragma once
#include <cstdint>

#include "../../include/evp.h"
#include "common.cuh"

namespace evp {

struct FpCtl {
    int done, it, conv, status, nmax, nfail;
    unsigned ticket;    // z-pass blocks finished in this iteration (the last one runs the control)
    int pad;
    double err_eq, err_bc;
    double dE[6];
    double tol_loc;     // local-solve tolerance of the next iteration (see evp_config.newton_adapt)
    float tol_loc_f;
};

struct FpCtlParams {
    double N3, tau0, tol, a, b, det, mu0, ntol, eta;
    int max_iter;
};

// What the z pass needs to run the control in its last block (ctl == nullptr: no control).
struct ZCtl {
    FpCtl *ctl;
    int32_t *flags;         // flags[0] failed local solves, flags[1] max local iterations, flags[10] the local
                            // solve's work-list count, flags[11] its pass 1's two-step count (both reset here for
                            // the next iteration)
    double *scal;           // scal[0..5] mean stress (written by the z pass), scal[6] residual sum
    FpCtlParams p;
};

// Every thread of one block calls this with the iteration's nparts partial sums.
template <typename T>
__device__ __forceinline__ void fp_control_block(const ZCtl &z, const double *__restrict__ part, int nparts,
                                                 typename CT<T>::type *__restrict__ spec, long fstride, int n) {
    __shared__ double red[32];
    __shared__ double corr[6];
    __shared__ double meanv[6];
    __shared__ int iv[4];
    __shared__ int go;
    FpCtl *c = z.ctl;
    const FpCtlParams &p = z.p;
    // operands of the decision fetched by separate threads, alongside the reduction
    if (threadIdx.x < 6) meanv[threadIdx.x] = z.scal[threadIdx.x];
    else if (threadIdx.x == 32) iv[0] = c->it;
    else if (threadIdx.x == 33) iv[1] = c->nmax;
    else if (threadIdx.x == 34) iv[2] = z.flags[0];
    else if (threadIdx.x == 35) iv[3] = z.flags[1];
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += part[i];
    s = block_sum(s, red);   // its barriers also publish meanv and iv
    if (threadIdx.x == 0) {
        go = 0;
        z.scal[6] = s;
        z.flags[10] = 0;   // the next iteration's first local-solve pass counts its work list from zero,
        z.flags[11] = 0;   // and its voxels accepted after two steps
        const int it = iv[0] + 1;
        c->it = it;
        c->nmax = max(iv[1], iv[3]);
        double mean[6], mn = 0.0, mu_n = 0.0;
        for (int i = 0; i < 6; ++i) {
            mean[i] = meanv[i];
            mn += mean[i] * mean[i];
            if (i != 2) mu_n += mean[i] * mean[i];
        }
        const double den = fmax(sqrt(mn), p.tau0);
        const double err_eq = sqrt(s) / (p.N3 * den);
        const double err_bc = sqrt(fmax(mu_n, 0.0)) / den;
        c->err_eq = err_eq;
        c->err_bc = err_bc;
        if (iv[2] != 0) {
            c->nfail = iv[2];
            c->status = EVP_ERR_NEWTON;
            c->done = 1;
        } else if (!isfinite(err_eq) || !isfinite(err_bc)) {
            c->status = EVP_ERR_NONFINITE;
            c->done = 1;
        } else if (err_eq <= p.tol && err_bc <= p.tol) {
            c->conv = 1;
            c->done = 1;
        } else if (it >= p.max_iter) {
            c->done = 1;
        } else {
            double dEk[6] = {0, 0, 0, 0, 0, 0};
            dEk[0] = (p.a * (-mean[0]) - p.b * (-mean[1])) / p.det;
            dEk[1] = (-p.b * (-mean[0]) + p.a * (-mean[1])) / p.det;
            for (int i = 3; i < 6; ++i) dEk[i] = -mean[i] / (2.0 * p.mu0);
            for (int i = 0; i < 6; ++i) {
                c->dE[i] += dEk[i];
                corr[i] = dEk[i] * p.N3;   // the inverse transforms are unnormalised; x_c2r scales by 1/N^3
            }
            if (p.eta > 0.0) {
                const double tl = fmax(p.ntol, p.eta * fmax(err_eq, err_bc));
                c->tol_loc = tl;
                c->tol_loc_f = (float)tl;
            }
            go = 1;
        }
    }
    __syncthreads();
    if (!go) return;
    const long zstride = fstride / n;
    for (int t = threadIdx.x; t < 6 * n; t += blockDim.x) {
        const int f = t / n, zz = t - f * n;
        auto &e = spec[f * fstride + zz * zstride];
        e.x += (T)corr[f];
    }
}

}  // namespace evp
