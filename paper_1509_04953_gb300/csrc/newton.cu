// Per-voxel crystal-plasticity kernels (Sec. 2.1 Eqs. HookeLaw / PlasticRate, Sec. 2.2 flow rule
// and density evolution read as a power law with Kocks-Mecking hardening).
//
// Local problem: find sigma with r(sigma) = S:sigma + dt sum_a m^a gdot^a(sigma) - eps_tr = 0,
// gdot^a = gdot0 |tau^a/tau_c|^n sign(tau^a), tau^a = m^a:sigma. This is the implicit Euler
// stress update of Eq. HookeLaw multiplied by the compliance S = C^-1; its Jacobian
// K = S + dt sum_a (n gdot0 |x^a|^(n-1)/tau_c) m^a (x) m^a is symmetric positive definite, so the
// 6x6 Newton system is solved by an LDL^T factorisation, and r is the gradient of a convex potential Phi used
// for Armijo backtracking. eps_tr = eps^{t+dt} - eps_p^t is carried directly (the "trial" elastic
// strain), which keeps FP32 fields accurate when the total strain is large.
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"
#include "local.cuh"

namespace evp {

namespace {

constexpr int kThreads = 128;

// Local-solve statistics, summed over the block before they touch the shared counters (the same-address
// atomics of every warp of a two-million-voxel launch serialise in L2): flags[0] += failed voxels,
// flags[1] = max(local iterations); 64-bit flags[4..5] += iterations (6x6 solves), [6..7] += residual
// evaluations, [8..9] += tangent refreshes. Every thread of the block calls it once.
__device__ __forceinline__ void block_solve_stats(int fail, int maxit, int it, int ev, int rf, int *flags) {
    __shared__ int sh[kThreads / 32][5];
    int f = fail, mx = maxit, sit = it, sev = ev, srf = rf;
    for (int o = 16; o > 0; o >>= 1) {
        f += __shfl_xor_sync(0xffffffffu, f, o);
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        sit += __shfl_xor_sync(0xffffffffu, sit, o);
        sev += __shfl_xor_sync(0xffffffffu, sev, o);
        srf += __shfl_xor_sync(0xffffffffu, srf, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sh[w][0] = f; sh[w][1] = mx; sh[w][2] = sit; sh[w][3] = sev; sh[w][4] = srf;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int tf = 0, tm = 0;
        unsigned long long ti = 0, te = 0, tr = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            tf += sh[k][0]; tm = max(tm, sh[k][1]);
            ti += (unsigned)sh[k][2]; te += (unsigned)sh[k][3]; tr += (unsigned)sh[k][4];
        }
        if (tf) atomicAdd(flags, tf);
        if (tm) atomicMax(flags + 1, tm);
        if (ti) atomicAdd(reinterpret_cast<unsigned long long *>(flags + 4), ti);
        if (te) atomicAdd(reinterpret_cast<unsigned long long *>(flags + 6), te);
        if (tr) atomicAdd(reinterpret_cast<unsigned long long *>(flags + 8), tr);
    }
}

// Damped Newton on one voxel. Returns the iteration count (> 0) or minus it on failure.
// H: the power law's tau_c (TA) or the Ma-Roters flow data (FlowMR<TA>, Sec. 2.2).
template <typename TA, typename TS, typename H>
__device__ int newton_voxel(const TA Sp[21], const TA *__restrict__ M, const TA etr[6], const H &hf, TA sg[6],
                            const MatConst &mc, TA tol, int maxit, TA ls_free, int &nevals) {
    const TA tauc = flow_ref(hf);
    const TA inv_tc = drcp(tauc);
    Eval<TA> e;
    evaluate(Sp, M, etr, hf, inv_tc, sg, mc, e);
    nevals = 1;
    for (int it = 1; it <= maxit; ++it) {
        TA d[6];
        if (!ldl_solve<TS, TA>(e.K, e.r, d)) return -it;
        TA rd = (TA)0, dn = (TA)0, sn = (TA)0;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            rd += e.r[i] * d[i];
            dn += d[i] * d[i];
            sn += sg[i] * sg[i];
        }
        dn = dsqrt(dn);
        const TA scale = dsqrt(sn) + tauc;
        if (dn <= tol * scale) {
            // The full step is below the stopping tolerance (and far below the line-search
            // threshold), so it is taken and the iteration ends without evaluating the new point.
#pragma unroll
            for (int i = 0; i < 6; ++i) sg[i] -= d[i];
            return it;
        }
        const TA phi0 = e.phi;
        TA s = (TA)1, st[6];
        bool ok = false;
        for (int h = 0; h < 60; ++h) {
#pragma unroll
            for (int i = 0; i < 6; ++i) st[i] = sg[i] - s * d[i];
            evaluate(Sp, M, etr, hf, inv_tc, st, mc, e);
            ++nevals;
            if (e.phi <= phi0 - (TA)1e-4 * s * rd || s * dn <= ls_free * scale) {
                ok = true;
                break;
            }
            s *= (TA)0.5;
        }
        if (!ok) return -it;
#pragma unroll
        for (int i = 0; i < 6; ++i) sg[i] = st[i];
        if (s * dn <= tol * scale) return it;
    }
    return -maxit;
}

template <typename TA, typename TS, bool MR = false>
__global__ void __launch_bounds__(kThreads) k_newton(long N3, const TA *__restrict__ epst, const TA *__restrict__ tauc,
                                                    const int32_t *__restrict__ g0, TA *__restrict__ sig,
                                                    const TA *__restrict__ Stab, const TA *__restrict__ Mtab, MatConst mc,
                                                    TA tol, int maxit, TA ls_free, int *__restrict__ flags, const int *__restrict__ skip,
    const TA *__restrict__ tol_dev, MRPtr<TA> mrp) {
    pdl_wait();
    pdl_trigger();
    if (skip != nullptr && *skip) return;   // the fixed point has converged
    if (tol_dev != nullptr) tol = *tol_dev;   // local tolerance set on the device for this iteration
    const long v = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = v < N3;
    int r = 1, nev = 0;
    if (valid) {
        const int g = g0[v];
        TA Sp[21];
        load_compliance(Stab + 36 * (long)g, Sp);
        TA etr[6], sg[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            etr[c] = epst[c * N3 + v];
            sg[c] = sig[c * N3 + v];
        }
        if constexpr (MR)
            r = newton_voxel<TA, TS>(Sp, Mtab + 72 * (long)g, etr, FlowMR<TA>{mrp.tpi, N3, v, tauc[v]}, sg, mc,
                                     tol, maxit, ls_free, nev);
        else
            r = newton_voxel<TA, TS>(Sp, Mtab + 72 * (long)g, etr, tauc[v], sg, mc, tol, maxit, ls_free, nev);
#pragma unroll
        for (int c = 0; c < 6; ++c) sig[c * N3 + v] = sg[c];
    }
    const int its = valid ? (r < 0 ? -r : r) : 0;
    block_solve_stats(valid && r < 0, its, its, nev, 0, flags);
}

// FP64 path: Newton on the FP64 residual with an FP32 tangent and FP32 6x6 solve. Each step is a
// slightly inexact Newton step (relative tangent error ~1e-7), so the iteration contracts at least
// ~1e-6 per step near the solution and stops on the same step-size test; Armijo backtracking on
// the FP64 potential keeps it globally convergent.
__device__ int newton_voxel_df(const double Sp[21], const double *__restrict__ M, const float Spf[21],
                               const float *__restrict__ Mf, const double etr[6], double tauc, double sg[6],
                               const MatConst &mc, double tol, int maxit, double ls_free, int &nevals) {
    const double inv_tc = drcp(tauc);
    EvalDF e;
    evaluate_df(Sp, M, Spf, Mf, etr, tauc, inv_tc, sg, mc, e);
    nevals = 1;
    for (int it = 1; it <= maxit; ++it) {
        float rf[6], df[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) rf[i] = (float)e.r[i];
        if (!ldl_solve<float, float>(e.K, rf, df)) return -it;
        double d[6], rd = 0.0, dn = 0.0, sn = 0.0;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            d[i] = (double)df[i];
            rd += e.r[i] * d[i];
            dn += d[i] * d[i];
            sn += sg[i] * sg[i];
        }
        dn = dsqrt(dn);
        const double scale = dsqrt(sn) + tauc;
        if (dn <= tol * scale && rd >= 0.0) {
#pragma unroll
            for (int i = 0; i < 6; ++i) sg[i] -= d[i];
            return it;
        }
        const double phi0 = e.phi;
        double s = 1.0, st[6];
        bool ok = false;
        for (int h = 0; h < 60; ++h) {
#pragma unroll
            for (int i = 0; i < 6; ++i) st[i] = sg[i] - s * d[i];
            evaluate_df(Sp, M, Spf, Mf, etr, tauc, inv_tc, st, mc, e);
            ++nevals;
            if (e.phi <= phi0 - 1e-4 * s * rd || s * dn <= ls_free * scale) {
                ok = true;
                break;
            }
            s *= 0.5;
        }
        if (!ok) return -it;
#pragma unroll
        for (int i = 0; i < 6; ++i) sg[i] = st[i];
        if (s * dn <= tol * scale) return it;
    }
    return -maxit;
}

__global__ void __launch_bounds__(kThreads) k_newton_df(long N3, const double *__restrict__ epst,
                                                       const double *__restrict__ tauc, const int32_t *__restrict__ g0,
                                                       double *__restrict__ sig, const double *__restrict__ Stab,
                                                       const double *__restrict__ Mtab, const float *__restrict__ Stabf,
                                                       const float *__restrict__ Mtabf, MatConst mc, double tol,
                                                       int maxit, int *__restrict__ flags, const int *__restrict__ skip,
    const double *__restrict__ tol_dev) {
    pdl_wait();
    pdl_trigger();
    if (skip != nullptr && *skip) return;   // the fixed point has converged
    if (tol_dev != nullptr) tol = *tol_dev;   // local tolerance set on the device for this iteration
    const long v = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = v < N3;
    int r = 1, nev = 0;
    if (valid) {
        const int g = g0[v];
        double Sp[21];
        float Spf[21];
        load_compliance(Stab + 36 * (long)g, Sp);
        load_compliance(Stabf + 36 * (long)g, Spf);
        double etr[6], sg[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            etr[c] = epst[c * N3 + v];
            sg[c] = sig[c * N3 + v];
        }
        r = newton_voxel_df(Sp, Mtab + 72 * (long)g, Spf, Mtabf + 72 * (long)g, etr, tauc[v], sg, mc, tol, maxit,
                            1e-6, nev);
#pragma unroll
        for (int c = 0; c < 6; ++c) sig[c * N3 + v] = sg[c];
    }
    const int its = valid ? (r < 0 ? -r : r) : 0;
    block_solve_stats(valid && r < 0, its, its, nev, 0, flags);
}

// Local solve with Jacobian reuse (chord Newton): the LDL^T factors of the tangent are stored per
// voxel and reused across fixed-point iterations; a step costs one residual evaluation and two
// triangular solves. The factors are refreshed (full tangent + factorisation at the current point)
// on request (first fixed-point iteration of an increment), when a step contracts by less than
// 4x, or after a backtracking line search. The local problem is still solved to the same
// tolerance, so the result matches the exact-Newton one to that tolerance.
//
// The factorisation runs in TF and the factors are stored and applied in TS. On the FP32-field path
// TF = double and TS = float: an FP32 factorisation of this tangent loses the small (elastic) pivots
// to cancellation once a few slip systems are far into the power law, while FP64 factors rounded to
// FP32 afterwards are a componentwise perturbation and keep the Newton direction within about 1e-4
// relative even there, so the reused step runs on the FP32 pipe and reads half the bytes.
template <typename TA, typename TS, typename TF, typename H>
__device__ int chord_voxel(const TA Sp[21], const TA *__restrict__ M, const TA etr[6], const H &hf, TA sg[6],
                           const MatConst &mc, TA tol, int maxit, TA ls_free, TS F[21], bool refresh, int &nevals,
                           int &nref) {
    const TA tauc = flow_ref(hf);
    const TA inv_tc = drcp(tauc);
    EvalR<TA> e;
    evaluate_r(Sp, M, etr, hf, inv_tc, sg, mc, e);
    nevals = 1;
    nref = 0;
    TA prev_step = (TA)-1;
    bool fresh = false;
    for (int it = 1; it <= maxit; ++it) {
        if (refresh) {
            Eval<TA> full;
            evaluate(Sp, M, etr, hf, inv_tc, sg, mc, full);
            ++nevals;
            TF Ff[21];
            if (!ldl_factor<TF, TA>(full.K, Ff)) return -it;
#pragma unroll
            for (int q = 0; q < 21; ++q) F[q] = (TS)Ff[q];
            ++nref;
            refresh = false;
            fresh = true;
        }
        TA d[6];
        ldl_apply<TS, TA>(F, e.r, d);
        TA rd = (TA)0, dn = (TA)0, sn = (TA)0;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            rd += e.r[i] * d[i];
            dn += d[i] * d[i];
            sn += sg[i] * sg[i];
        }
        dn = dsqrt(dn);
        const TA scale = dsqrt(sn) + tauc;
        if (dn <= tol * scale && rd >= (TA)0) {
#pragma unroll
            for (int i = 0; i < 6; ++i) sg[i] -= d[i];
            return it;
        }
        if (!fresh && (rd <= (TA)0 || (prev_step > (TA)0 && dn > (TA)0.25 * prev_step))) {
            refresh = true;   // stale tangent: refactor at this point and redo the step
            continue;
        }
        const TA phi0 = e.phi;
        TA s = (TA)1, st[6];
        bool ok = false;
        for (int h = 0; h < 60; ++h) {
#pragma unroll
            for (int i = 0; i < 6; ++i) st[i] = sg[i] - s * d[i];
            evaluate_r(Sp, M, etr, hf, inv_tc, st, mc, e);
            ++nevals;
            if (e.phi <= phi0 - (TA)1e-4 * s * rd || s * dn <= ls_free * scale) {
                ok = true;
                break;
            }
            s *= (TA)0.5;
        }
        if (!ok) return -it;
#pragma unroll
        for (int i = 0; i < 6; ++i) sg[i] = st[i];
        if (s * dn <= tol * scale) return it;
        if (s < (TA)1) refresh = true;
        prev_step = s * dn;
        fresh = false;
    }
    return -maxit;
}

template <typename TA, typename TS, typename TF, bool MR = false>
__global__ void __launch_bounds__(kThreads, sizeof(TA) == 4 ? 3 : 2) k_newton_chord(long N3, const TA *__restrict__ epst, const TA *__restrict__ tauc,
                                                          const int32_t *__restrict__ g0, TA *__restrict__ sig,
                                                          const TA *__restrict__ Stab, const TA *__restrict__ Mtab,
                                                          TS *__restrict__ fac, MatConst mc, TA tol, int maxit,
                                                          TA ls_free, int force_refresh, int *__restrict__ flags, const int *__restrict__ skip,
    const TA *__restrict__ tol_dev, MRPtr<TA> mrp) {
    pdl_wait();
    pdl_trigger();
    if (skip != nullptr && *skip) return;   // the fixed point has converged
    if (tol_dev != nullptr) tol = *tol_dev;   // local tolerance set on the device for this iteration
    const long v = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = v < N3;
    int r = 1, nev = 0, nref = 0;
    if (valid) {
        const int g = g0[v];
        TA Sp[21];
        load_compliance(Stab + 36 * (long)g, Sp);
        TA etr[6], sg[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            etr[c] = epst[c * N3 + v];
            sg[c] = sig[c * N3 + v];
        }
        TS F[21];
        if (!force_refresh) {
            load_factors(fac, N3, v, F);
        }
        if constexpr (MR)
            r = chord_voxel<TA, TS, TF>(Sp, Mtab + 72 * (long)g, etr, FlowMR<TA>{mrp.tpi, N3, v, tauc[v]}, sg,
                                        mc, tol, maxit, ls_free, F, force_refresh != 0, nev, nref);
        else
            r = chord_voxel<TA, TS, TF>(Sp, Mtab + 72 * (long)g, etr, tauc[v], sg, mc, tol, maxit, ls_free, F,
                                        force_refresh != 0, nev, nref);
#pragma unroll
        for (int c = 0; c < 6; ++c) sig[c * N3 + v] = sg[c];
        if (nref) {
            store_factors(fac, N3, v, F);
        }
    }
    const int its = valid ? (r < 0 ? -r : r) : 0;
    block_solve_stats(valid && r < 0, its, its, nev, nref, flags);
}

// Tangent reuse in two passes. Most voxels accept the first chord step once the fixed point has
// settled, while a few need line searches or a refreshed tangent; in one kernel the warps holding
// those few run their long loops with most lanes idle. Pass 1 takes the first step for every voxel
// and stores it where it is accepted; the others are appended to a work list (warp-aggregated,
// order immaterial: each voxel's computation is independent and deterministic). Pass 2 runs the
// full chord iteration on the listed voxels only, from their unchanged state, so every result is
// bitwise the one the single-kernel iteration gives.
// TWO: also the chord iteration's next two moves (below); its registers cost one CTA per SM on the FP32 path.
template <typename TA, typename TS, bool MR = false, bool TWO = true>
__global__ void __launch_bounds__(kThreads, sizeof(TA) == 4 ? (TWO ? 7 : 8) : 1) k_chord_first(long N3, const TA *__restrict__ epst,
                                                         const TA *__restrict__ tauc, const int32_t *__restrict__ g0,
                                                         TA *__restrict__ sig, const TA *__restrict__ Stab,
                                                         const TA *__restrict__ Mtab, const TS *__restrict__ fac,
                                                         MatConst mc, TA tol, TA ls_free, int *__restrict__ flags,
                                                         int32_t *__restrict__ wl, const int *__restrict__ skip,
    const TA *__restrict__ tol_dev, MRPtr<TA> mrp) {
    pdl_wait();
    pdl_trigger();
    if (skip != nullptr && *skip) return;   // the fixed point has converged
    if (tol_dev != nullptr) tol = *tol_dev;   // local tolerance set on the device for this iteration
    const long v = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = v < N3;
    bool done = false, two = false;
    // the stored factors are needed only after the residual: their copies start first, into this thread's slots
    // of shared memory, and run under the other loads and the evaluation
    __shared__ __align__(16) TS fsh[factor_words<TS>() * kThreads];
    if (valid) prefetch_factors(fac, N3, v, fsh);
    if (valid) {
        const int g = g0[v];
        TA Sp[21];
        load_compliance(Stab + 36 * (long)g, Sp);
        TA etr[6], sg[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            etr[c] = epst[c * N3 + v];
            sg[c] = sig[c * N3 + v];
        }
        const TA tc = tauc[v];
        EvalR<TA> e;
        if constexpr (MR)
            evaluate_r<TA, 6>(Sp, Mtab + 72 * (long)g, etr, FlowMR<TA>{mrp.tpi, N3, v, tc}, (TA)0, sg, mc, e);
        else
            evaluate_r<TA, 6>(Sp, Mtab + 72 * (long)g, etr, tc, drcp(tc), sg, mc, e);
        TS F[21];
        prefetched_factors(fsh, F);
        TA d[6];
        ldl_apply<TS, TA>(F, e.r, d);
        TA rd = (TA)0, dn = (TA)0, sn = (TA)0;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            rd += e.r[i] * d[i];
            dn += d[i] * d[i];
            sn += sg[i] * sg[i];
        }
        dn = dsqrt(dn);
        const TA scale = dsqrt(sn) + tc;
        if (dn <= tol * scale && rd >= (TA)0) {   // the acceptance test of chord_voxel
#pragma unroll
            for (int c = 0; c < 6; ++c) sig[c * N3 + v] = sg[c] - d[c];
            done = true;
        } else if (TWO && rd > (TA)0) {
            // chord_voxel's next moves while they stay on its common path, with its operations in its order: the
            // full step of the line search (s = 1) passes the sufficient-decrease test, and the chord step from
            // there passes the acceptance test. Anything else goes to pass 2, which starts over from the
            // unchanged state, so every voxel still ends bitwise where the single-kernel iteration puts it.
            // The grain's compliance and the factors are fetched again (from L1 and shared memory) rather than held
            // in registers through the first step.
            const TA s1 = (TA)1, phi0 = e.phi;
            TA st[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) st[i] = sg[i] - s1 * d[i];
            asm volatile("" ::: "memory");
            TA Sp2[21];
            load_compliance(Stab + 36 * (long)g, Sp2);
            if constexpr (MR)
                evaluate_r<TA>(Sp2, Mtab + 72 * (long)g, etr, FlowMR<TA>{mrp.tpi, N3, v, tc}, (TA)0, st, mc, e);
            else
                evaluate_r<TA>(Sp2, Mtab + 72 * (long)g, etr, tc, drcp(tc), st, mc, e);
            if (e.phi <= phi0 - (TA)1e-4 * s1 * rd || s1 * dn <= ls_free * scale) {
                prefetched_factors(fsh, F);
                ldl_apply<TS, TA>(F, e.r, d);
                TA rd2 = (TA)0, dn2 = (TA)0, sn2 = (TA)0;
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    rd2 += e.r[i] * d[i];
                    dn2 += d[i] * d[i];
                    sn2 += st[i] * st[i];
                }
                dn2 = dsqrt(dn2);
                if (dn2 <= tol * (dsqrt(sn2) + tc) && rd2 >= (TA)0) {
#pragma unroll
                    for (int c = 0; c < 6; ++c) sig[c * N3 + v] = st[c] - d[c];
                    done = true;
                    two = true;
                }
            }
        }
    }
    const unsigned todo = __ballot_sync(0xffffffffu, valid && !done);
    const unsigned twos = __ballot_sync(0xffffffffu, two);
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0 && todo) base = atomicAdd(flags + 10, __popc(todo));
    if (lane == 0 && twos) atomicAdd(flags + 11, __popc(twos));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (valid && !done) wl[base + __popc(todo & ((1u << lane) - 1u))] = (int32_t)v;
    // the accepted voxels are counted by pass 2: N3 - listed with one evaluation and one solve each, plus one more
    // of each for the flags[11] voxels accepted after two steps
}

template <typename TA, typename TS, typename TF, bool MR = false>
__global__ void __launch_bounds__(kThreads, sizeof(TA) == 4 ? 3 : 2) k_chord_rest(
    long N3, const TA *__restrict__ epst, const TA *__restrict__ tauc, const int32_t *__restrict__ g0,
    TA *__restrict__ sig, const TA *__restrict__ Stab, const TA *__restrict__ Mtab, TS *__restrict__ fac, MatConst mc,
    TA tol, int maxit, TA ls_free, int *__restrict__ flags, const int32_t *__restrict__ wl, const int *__restrict__ skip,
    const TA *__restrict__ tol_dev, MRPtr<TA> mrp) {
    pdl_wait();
    pdl_trigger();
    if (skip != nullptr && *skip) return;   // the fixed point has converged
    if (tol_dev != nullptr) tol = *tol_dev;   // local tolerance set on the device for this iteration
    const int count = *(volatile const int *)(flags + 10);
    if (blockIdx.x == 0 && threadIdx.x == 0 && N3 - count > 0) {   // pass 1 accepted the others in one or two steps
        const int twos = *(volatile const int *)(flags + 11);
        atomicMax(flags + 1, twos > 0 ? 2 : 1);
        atomicAdd(reinterpret_cast<unsigned long long *>(flags + 4), (unsigned long long)(N3 - count + twos));
        atomicAdd(reinterpret_cast<unsigned long long *>(flags + 6), (unsigned long long)(N3 - count + twos));
    }
    const long stride = (long)gridDim.x * blockDim.x;
    int t_fail = 0, t_mx = 0, t_it = 0, t_ev = 0, t_rf = 0;
    for (long w0 = (long)blockIdx.x * blockDim.x; w0 < count; w0 += stride) {   // block-uniform trip count
        const long w = w0 + threadIdx.x;
        const bool valid = w < count;
        int r = 1, nev = 0, nref = 0;
        if (valid) {
            const long v = wl[w];
            const int g = g0[v];
            TA Sp[21];
            load_compliance(Stab + 36 * (long)g, Sp);
            TA etr[6], sg[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                etr[c] = epst[c * N3 + v];
                sg[c] = sig[c * N3 + v];
            }
            TS F[21];
            load_factors(fac, N3, v, F);
            if constexpr (MR)
                r = chord_voxel<TA, TS, TF>(Sp, Mtab + 72 * (long)g, etr, FlowMR<TA>{mrp.tpi, N3, v, tauc[v]},
                                            sg, mc, tol, maxit, ls_free, F, false, nev, nref);
            else
                r = chord_voxel<TA, TS, TF>(Sp, Mtab + 72 * (long)g, etr, tauc[v], sg, mc, tol, maxit, ls_free, F, false,
                                            nev, nref);
#pragma unroll
            for (int c = 0; c < 6; ++c) sig[c * N3 + v] = sg[c];
            if (nref) {
                store_factors(fac, N3, v, F);
            }
        }
        if (valid) {
            const int it = r < 0 ? -r : r;
            t_fail += r < 0;
            t_mx = max(t_mx, it);
            t_it += it;
            t_ev += nev;
            t_rf += nref;
        }
    }
    block_solve_stats(t_fail, t_mx, t_it, t_ev, t_rf, flags);
}

// Augmented-Lagrangian local step (the solver the paper names, Sec. 2.1, after Michel et al.):
// with C0 the reference stiffness and S0 = C0^-1, per voxel
//   eps_tr' = S0 lam + eps_tr              (trial strain of the local problem)
//   solve (S + S0) sigma + dt sum m gdot(sigma) = eps_tr'     -> sigma   (Sal = S + S0 per grain)
//   e_tr = eps_tr' - S0 sigma              (local strain, minus eps_p^t)
//   lam  = lam + C0 (eps_tr - e_tr)
//   p    = lam - C0 (e_tr - eps_e^t)       (minus the polarisation; the z pass returns -Gamma0 p)
// init = 1 is the start of an increment: sigma from the plain implicit update at eps_tr (S instead of
// Sal, no lam term), then lam = sigma and e_tr = eps_tr. Partial sums per block: |eps_tr - e_tr|^2,
// |C0 (eps_tr - e_tr)|^2, the six components of lam and the six of sigma.
// Error-free transformations on FP32 (Knuth's two-sum; the rounding error of a product by fma): an
// FP32 result plus the float that it rounded away, exactly.
__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod_f(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = fmaf(a, b, -p);
}

// C0 x for the isotropic reference stiffness (Lame constants l0, m0), component i of Mandel x.
template <typename T> __device__ __forceinline__ T iso_apply_c0(T l0, T m0, const T x[6], int i) {
    const T tr = x[0] + x[1] + x[2];
    return (T)2 * m0 * x[i] + (i < 3 ? l0 * tr : (T)0);
}

// NV per-thread values summed over the block into part[0..NV): warp sums in the value type (a
// five-level pairwise tree), then the warp sums in FP64. On the FP32 path this keeps the FP64 pipe
// out of the per-voxel work; the result stays within a few FP32 roundings of the exact block sum.
template <int NV, typename T> __device__ __forceinline__ void block_sums(const T (&v)[NV], double *sh, double *part) {
    T w[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        w[q] = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w[q] += __shfl_xor_sync(0xffffffffu, w[q], o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) sh[wid * NV + q] = (double)w[q];
    __syncthreads();
    if (threadIdx.x < NV) {
        double t = 0.0;
        for (int k = 0; k < nw; ++k) t += sh[k * NV + threadIdx.x];
        part[threadIdx.x] = t;
    }
}

// The warp's sums of NV per-thread values (a five-level pairwise tree in the value type), added in FP64 by
// lane 0 to row[0..NV) (one row per warp: no other warp touches it, so no barrier).
template <int NV, typename T> __device__ __forceinline__ void warp_accumulate(const T (&v)[NV], double *row) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        T w = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if ((threadIdx.x & 31) == 0) row[q] += (double)w;
    }
}

template <typename TA, typename TS, typename TF, bool MR = false>
__global__ void __launch_bounds__(kThreads, sizeof(TA) == 4 ? 3 : 2) k_al_local(long N3, const TA *__restrict__ epst, const TA *__restrict__ epse,
                                                      const TA *__restrict__ tauc, const int32_t *__restrict__ g0,
                                                      TA *__restrict__ sig, TA *__restrict__ lam, TA *__restrict__ pout,
                                                      const TA *__restrict__ Stab, const TA *__restrict__ Sal,
                                                      const TA *__restrict__ Mtab, MatConst mc, TA l0, TA m0, TA sa,
                                                      TA sb, TA sa_lo, TA sb_lo, double sad, double sbd, TA tol,
                                                      int maxit, TA ls_free, int init,
                                                      int *__restrict__ flags, double *__restrict__ part,
                                                      TS *__restrict__ fac, int refresh, MRPtr<TA> mrp) {
    constexpr int NV = 14;
    // grid-stride over tiles of blockDim voxels (block-uniform trip count): the block's warps run their tiles
    // without waiting for one another; each warp sums its tile's values and lane 0 adds them, in FP64, to the
    // warp's row of acc; the rows are summed once, at the end
    __shared__ double acc[(kThreads / 32) * NV];
    for (int i = threadIdx.x; i < (kThreads / 32) * NV; i += blockDim.x) acc[i] = 0.0;
    __syncthreads();
    int t_fail = 0, t_mx = 0, t_it = 0, t_ev = 0;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long v0 = (long)blockIdx.x * blockDim.x; v0 < N3; v0 += stride) {
    const long v = v0 + threadIdx.x;
    const bool valid = v < N3;
    int r = 1, nev = 0;
    TA sums[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) sums[q] = (TA)0;
    if (valid) {
        const int g = g0[v];
        TA Sp[21];
        load_compliance((init ? Stab : Sal) + 36 * (long)g, Sp);
        // isotropic S0 = C0^-1 = sa I - sb J (Mandel), sa = 1/(2 m0), sb = l0 / (2 m0 (3 l0 + 2 m0))
        TA et[6], lm[6], ee[6], etr[6], sg[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            et[c] = epst[c * N3 + v];
            lm[c] = init ? (TA)0 : lam[c * N3 + v];
            ee[c] = epse[c * N3 + v];
            sg[c] = sig[c * N3 + v];
        }
        const TA ltr = lm[0] + lm[1] + lm[2];
#pragma unroll
        for (int c = 0; c < 6; ++c) etr[c] = et[c] + sa * lm[c] - (c < 3 ? sb * ltr : (TA)0);
        if (fac) {   // tangent reuse: factors refreshed on request or when a step stalls
            TS F[21];
            if (!refresh) {
                load_factors(fac, N3, v, F);
            }
            int nref = 0;
            if constexpr (MR)
                r = chord_voxel<TA, TS, TF>(Sp, Mtab + 72 * (long)g, etr, FlowMR<TA>{mrp.tpi, N3, v, tauc[v]},
                                            sg, mc, tol, maxit, ls_free, F, refresh != 0, nev, nref);
            else
                r = chord_voxel<TA, TS, TF>(Sp, Mtab + 72 * (long)g, etr, tauc[v], sg, mc, tol, maxit, ls_free, F,
                                            refresh != 0, nev, nref);
            if (nref) {
                store_factors(fac, N3, v, F);
            }
        } else {
            if constexpr (MR)
                r = newton_voxel<TA, TF>(Sp, Mtab + 72 * (long)g, etr, FlowMR<TA>{mrp.tpi, N3, v, tauc[v]}, sg,
                                         mc, tol, maxit, ls_free, nev);
            else
                r = newton_voxel<TA, TF>(Sp, Mtab + 72 * (long)g, etr, tauc[v], sg, mc, tol, maxit, ls_free, nev);
        }
        // local strain e_tr = eps_tr' - S0 sigma and the gap d = eps_tr - e_tr to about twice the field
        // precision: near convergence eps_tr and e_tr agree to many digits, and forming them in plain FP32
        // leaves rounding noise in d (hence in the multiplier update) that keeps the iteration from
        // settling. FP64 does it on the FP64 path; the FP32 path uses error-free transformations on the
        // FP32 pipe (the FP64 pipe issues 1/64 as fast).
        TA el[6], d[6], de[6];
        if constexpr (sizeof(TA) == 4) {
            float t1, e1, th, e2;
            two_sum_f(sg[0], sg[1], t1, e1);
            two_sum_f(t1, sg[2], th, e2);
            const float tl = __fadd_rn(e1, e2);   // tr(sigma) = th + tl
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                sig[c * N3 + v] = sg[c];
                if (init) {
                    el[c] = et[c];
                    d[c] = 0.f;
                } else {
                    float p, pe;
                    two_prod_f(sa, sg[c], p, pe);
                    pe = fmaf(sa_lo, sg[c], pe);   // S0 sigma (shear part) = p + pe
                    float sh = p, sl = pe;
                    if (c < 3) {
                        float q, qe, se;
                        two_prod_f(sb, th, q, qe);
                        qe = fmaf(sb, tl, fmaf(sb_lo, th, qe));   // sb tr = q + qe
                        two_sum_f(p, -q, sh, se);
                        sl = __fadd_rn(se, __fsub_rn(pe, qe));
                    }
                    float u, ue, w, we;
                    two_sum_f(etr[c], -sh, u, ue);            // e_tr = u + ul
                    const float ul = __fsub_rn(ue, sl);
                    two_sum_f(et[c], -u, w, we);              // d = eps_tr - e_tr
                    d[c] = __fadd_rn(w, __fsub_rn(we, ul));
                    el[c] = __fadd_rn(u, ul);
                }
                de[c] = el[c] - ee[c];
            }
        } else {
            double s6[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) s6[c] = (double)sg[c];
            const double str = s6[0] + s6[1] + s6[2];
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                sig[c * N3 + v] = sg[c];
                const double eld = init ? (double)et[c] : (double)etr[c] - (sad * s6[c] - (c < 3 ? sbd * str : 0.0));
                d[c] = (TA)((double)et[c] - eld);
                el[c] = (TA)eld;
                de[c] = el[c] - ee[c];
            }
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const TA dl = iso_apply_c0(l0, m0, d, c);
            const TA nl = init ? sg[c] : lm[c] + dl;
            lam[c * N3 + v] = nl;
            pout[c * N3 + v] = nl - iso_apply_c0(l0, m0, de, c);
            sums[0] += d[c] * d[c];
            sums[1] += dl * dl;
            sums[2 + c] = nl;
            sums[8 + c] = sg[c];
        }
    }
    if (valid) {
        const int its = r < 0 ? -r : r;
        t_fail += r < 0;
        t_mx = max(t_mx, its);
        t_it += its;
        t_ev += nev;
    }
    warp_accumulate<NV>(sums, acc + (threadIdx.x >> 5) * NV);
    }
    // flags as in k_newton
    // (its barrier follows every warp's last acc update, so acc is complete after it)
    block_solve_stats(t_fail, t_mx, t_it, t_ev, 0, flags);
    if (threadIdx.x < NV) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += acc[k * NV + threadIdx.x];
        part[NV * (long)blockIdx.x + threadIdx.x] = t;
    }
}

// Start of an increment: tau_c from the densities at t (frozen over the increment) and the
// predictor eps_tr = eps_e^t + (r * deps_prev  |  dE).
template <typename TA>
__global__ void __launch_bounds__(256) k_predictor(long N3, const TA *__restrict__ epse, const TA *__restrict__ deps,
                                                  const TA *__restrict__ rho, TA *__restrict__ epst, TA *__restrict__ tauc,
                                                  MatConst mc, TA r, int use_field, TA d0, TA d1, TA d2, TA d3, TA d4,
                                                  TA d5) {
    const long v = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N3) return;
    // all loads first; arithmetic in the field precision (the FP32 path keeps the FP64 pipe out)
    TA rr[12], ee[6], dd[6];
#pragma unroll
    for (int a = 0; a < 12; ++a) rr[a] = rho[a * N3 + v];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        ee[c] = epse[c * N3 + v];
        dd[c] = use_field ? deps[c * N3 + v] : (TA)0;
    }
    TA rf = (TA)0;
#pragma unroll
    for (int a = 0; a < 12; ++a) rf += rr[a];
    tauc[v] = (TA)mc.tau0 + (TA)mc.alpha_mu_b * sqrt(rf);
    const TA dE[6] = {d0, d1, d2, d3, d4, d5};
#pragma unroll
    for (int c = 0; c < 6; ++c) epst[c * N3 + v] = ee[c] + (use_field ? r * dd[c] : dE[c]);
}

// Error-free sum of two floats (Knuth's two-sum): s + e equals a + b exactly.
__device__ __forceinline__ void two_sum_k(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// k = sum of the 12 densities as a double. FP64 fields: summed in FP64. FP32 fields: summed as an unevaluated
// float pair (two-sum per term, the rounding errors added in float) and converted once: the result is within a few
// units of 2^-48 of the exact sum of the FP32 densities (the FP64 running sum is exact for them too, or nearly),
// with 2 FP64-pipe operations instead of 24 on a pipe that runs at 1/64 of the FP32 rate.
__device__ __forceinline__ double density_total(const double r[12]) {
    double kk = 0.0;
#pragma unroll
    for (int a = 0; a < 12; ++a) kk += r[a];
    return kk;
}
__device__ __forceinline__ double density_total(const float r[12]) {
    float hi = r[0], lo = 0.f;
#pragma unroll
    for (int a = 1; a < 12; ++a) {
        float s, e;
        two_sum_k(hi, r[a], s, e);
        hi = s;
        lo = __fadd_rn(lo, e);
    }
    return (double)hi + (double)lo;
}

// After convergence (a7): advance eps_p, eps_e, the strain increment and the densities with
// the converged shear rates; k = rho_tot as a double.
template <typename TA>
__global__ void __launch_bounds__(kThreads) k_state_update(long N3, const TA *__restrict__ sig, const TA *__restrict__ tauc,
                                                          const int32_t *__restrict__ g0, const TA *__restrict__ Mtab,
                                                          const TA *__restrict__ epst, TA *__restrict__ epse,
                                                          TA *__restrict__ epsp, TA *__restrict__ deps, TA *__restrict__ rho,
                                                          double *__restrict__ kf, MatConst mc) {
    const long v = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N3) return;
    // every operand is loaded before any arithmetic, so a thread has all its requests in flight at once
    const int g = g0[v];
    TA sg[6], tr[6], eo[6], po[6], r[12];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        sg[c] = sig[c * N3 + v];
        tr[c] = epst[c * N3 + v];
        eo[c] = epse[c * N3 + v];
        po[c] = epsp[c * N3 + v];
    }
#pragma unroll
    for (int a = 0; a < 12; ++a) r[a] = rho[a * N3 + v];
    const TA tcv = tauc[v];
    const TA *M = Mtab + 72 * (long)g;
    const TA inv_tc = (TA)1 / tcv;
    const TA g0r = (TA)mc.gdot0, dt = (TA)mc.dt;
    TA ep[6] = {0, 0, 0, 0, 0, 0};
    TA agd[12];
#pragma unroll
    for (int a = 0; a < 12; ++a) {
        TA m[6], tau = (TA)0;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            m[i] = __ldg(M + 6 * a + i);
            tau += m[i] * sg[i];
        }
        const TA x = tau * inv_tc, ax = fabs(x);
        const TA p10 = pow_nm1(ax, mc) * ax;
        const TA gd = x < (TA)0 ? -g0r * p10 : g0r * p10;
        agd[a] = fabs(gd);
#pragma unroll
        for (int i = 0; i < 6; ++i) ep[i] += m[i] * gd;
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        epsp[c * N3 + v] = po[c] + dt * ep[c];
        deps[c * N3 + v] = tr[c] - eo[c];
        epse[c * N3 + v] = tr[c] - dt * ep[c];
    }
    // Kocks-Mecking update in the field precision
    TA rf = (TA)0;
#pragma unroll
    for (int a = 0; a < 12; ++a) rf += r[a];
    const TA srf = sqrt(rf), k1 = (TA)mc.k1, k2 = (TA)mc.k2;
    TA nr[12];
#pragma unroll
    for (int a = 0; a < 12; ++a) {
        nr[a] = r[a] + dt * (k1 * srf - k2 * r[a]) * agd[a];
        rho[a * N3 + v] = nr[a];
    }
    kf[v] = density_total(nr);
}

template <typename TA>
__global__ void k_total_strain(long N3, const TA *__restrict__ epse, const TA *__restrict__ epsp, TA *__restrict__ eps) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 6 * N3) eps[i] = epse[i] + epsp[i];
}

template <typename TA> TA ls_free_of() { return sizeof(TA) == 4 ? (TA)1e-3 : (TA)1e-6; }

}  // namespace

// Each launcher runs the power-law kernels, or their Ma-Roters instantiations when mrp.tpi is set.
template <typename TA, typename F> cudaError_t by_law(MRPtr<TA> mrp, F &&go) {
    if (mrp.tpi) go(std::true_type{});
    else go(std::false_type{});
    return cudaGetLastError();
}

template <typename TA>
cudaError_t newton_field(long N3, const TA *epst, const TA *tauc, const int32_t *g0, TA *sig, const TA *Stab,
                         const TA *Mtab, MatConst mc, double tol, int maxit, int solve_fp64, int *flags,
                         cudaStream_t s, const int *skip, const TA *tol_dev, MRPtr<TA> mrp) {
    const int blocks = (int)((N3 + kThreads - 1) / kThreads);
    return by_law(mrp, [&](auto law) {
        constexpr bool MR = decltype(law)::value;
        if (solve_fp64)
            k_newton<TA, double, MR><<<blocks, kThreads, 0, s>>>(N3, epst, tauc, g0, sig, Stab, Mtab, mc, (TA)tol,
                                                                 maxit, ls_free_of<TA>(), flags, skip, tol_dev, mrp);
        else
            k_newton<TA, TA, MR><<<blocks, kThreads, 0, s>>>(N3, epst, tauc, g0, sig, Stab, Mtab, mc, (TA)tol, maxit,
                                                             ls_free_of<TA>(), flags, skip, tol_dev, mrp);
    });
}

template <typename TA>
cudaError_t newton_chord_field(long N3, const TA *epst, const TA *tauc, const int32_t *g0, TA *sig, const TA *Stab,
                               const TA *Mtab, void *fac, MatConst mc, double tol, int maxit, int solve_fp64,
                               int force_refresh, int *flags, int32_t *wl, int nsm, cudaStream_t s, const int *skip,
                               const TA *tol_dev, MRPtr<TA> mrp, int two_step) {
    const int blocks = (int)((N3 + kThreads - 1) / kThreads);
    if (!force_refresh && wl) {
        // flags[10] counts the listed voxels; pass 2 reads it on the device (no host round trip). Inside the
        // fixed-point loop (skip set) the kernels run as one programmatic-launch chain: the count starts at zero
        // from the increment's flag reset and is reset by each iteration's control block (fpctl.cuh), so no
        // memset breaks the chain; outside it the count is reset here.
        const bool pdl = skip != nullptr;
        if (!pdl) {
            cudaError_t e = cudaMemsetAsync(flags + 10, 0, 2 * sizeof(int), s);
            if (e != cudaSuccess) return e;
        }
        const int rb = std::min(blocks, nsm * (sizeof(TA) == 4 ? 3 : 2));
        cudaError_t err = cudaSuccess;
        by_law(mrp, [&](auto law) {
            constexpr bool MR = decltype(law)::value;
            if (two_step)
                err = launch_k(pdl, k_chord_first<TA, TA, MR, true>, dim3(blocks), dim3(kThreads), 0, s, N3, epst, tauc,
                               g0, sig, Stab, Mtab, (const TA *)fac, mc, (TA)tol, ls_free_of<TA>(), flags, wl, skip,
                               tol_dev, mrp);
            else
                err = launch_k(pdl, k_chord_first<TA, TA, MR, false>, dim3(blocks), dim3(kThreads), 0, s, N3, epst,
                               tauc, g0, sig, Stab, Mtab, (const TA *)fac, mc, (TA)tol, ls_free_of<TA>(), flags, wl,
                               skip, tol_dev, mrp);
            if (err != cudaSuccess) return;
            if (solve_fp64)
                err = launch_k(pdl, k_chord_rest<TA, TA, double, MR>, dim3(rb), dim3(kThreads), 0, s, N3, epst, tauc,
                               g0, sig, Stab, Mtab, (TA *)fac, mc, (TA)tol, maxit, ls_free_of<TA>(), flags,
                               (const int32_t *)wl, skip, tol_dev, mrp);
            else
                err = launch_k(pdl, k_chord_rest<TA, TA, TA, MR>, dim3(rb), dim3(kThreads), 0, s, N3, epst, tauc, g0,
                               sig, Stab, Mtab, (TA *)fac, mc, (TA)tol, maxit, ls_free_of<TA>(), flags,
                               (const int32_t *)wl, skip, tol_dev, mrp);
        });
        return err != cudaSuccess ? err : cudaGetLastError();
    }
    // factors stored in the field precision; factorised in FP64 unless the FP32 solve is asked for
    return by_law(mrp, [&](auto law) {
        constexpr bool MR = decltype(law)::value;
        if (solve_fp64)
            k_newton_chord<TA, TA, double, MR><<<blocks, kThreads, 0, s>>>(N3, epst, tauc, g0, sig, Stab, Mtab,
                                                                           (TA *)fac, mc, (TA)tol, maxit,
                                                                           ls_free_of<TA>(), force_refresh, flags,
                                                                           skip, tol_dev, mrp);
        else
            k_newton_chord<TA, TA, TA, MR><<<blocks, kThreads, 0, s>>>(N3, epst, tauc, g0, sig, Stab, Mtab, (TA *)fac,
                                                                       mc, (TA)tol, maxit, ls_free_of<TA>(),
                                                                       force_refresh, flags, skip, tol_dev, mrp);
    });
}

int al_blocks(long N3) { return (int)((N3 + kThreads - 1) / kThreads); }
int al_grid(long N3, int nsm, int tsize) { return std::min(al_blocks(N3), std::max(nsm, 1) * (tsize == 4 ? 3 : 2)); }

cudaError_t newton_field_df(long N3, const double *epst, const double *tauc, const int32_t *g0, double *sig,
                            const double *Stab, const double *Mtab, const float *Stabf, const float *Mtabf,
                            MatConst mc, double tol, int maxit, int *flags, cudaStream_t s, const int *skip,
                            const double *tol_dev) {
    const int blocks = (int)((N3 + kThreads - 1) / kThreads);
    k_newton_df<<<blocks, kThreads, 0, s>>>(N3, epst, tauc, g0, sig, Stab, Mtab, Stabf, Mtabf, mc, tol, maxit, flags,
                                            skip, tol_dev);
    return cudaGetLastError();
}

template <typename TA>
cudaError_t al_local(long N3, const TA *epst, const TA *epse, const TA *tauc, const int32_t *g0, TA *sig, TA *lam, TA *p,
                     const TA *Stab, const TA *Sal, const TA *Mtab, MatConst mc, double lam0, double mu0, double tol,
                     int maxit, int solve_fp64, int init, int *flags, double *part, void *fac, int refresh,
                     cudaStream_t s, int nsm, MRPtr<TA> mrp) {
    const int blocks = al_grid(N3, nsm, (int)sizeof(TA));
    const double sad = 1.0 / (2.0 * mu0), sbd = lam0 / (2.0 * mu0 * (3.0 * lam0 + 2.0 * mu0));
    const TA sa = (TA)sad, sb = (TA)sbd;
    const TA sa_lo = (TA)(sad - (double)sa), sb_lo = (TA)(sbd - (double)sb);   // S0 = (sa + sa_lo) I - (sb + sb_lo) J
    return by_law(mrp, [&](auto law) {
        constexpr bool MR = decltype(law)::value;
        if (solve_fp64)
            k_al_local<TA, TA, double, MR><<<blocks, kThreads, 0, s>>>(N3, epst, epse, tauc, g0, sig, lam, p, Stab, Sal,
                                                                       Mtab, mc, (TA)lam0, (TA)mu0, sa, sb, sa_lo,
                                                                       sb_lo, sad, sbd, (TA)tol, maxit,
                                                                       ls_free_of<TA>(), init, flags, part, (TA *)fac,
                                                                       refresh, mrp);
        else
            k_al_local<TA, TA, TA, MR><<<blocks, kThreads, 0, s>>>(N3, epst, epse, tauc, g0, sig, lam, p, Stab, Sal,
                                                                   Mtab, mc, (TA)lam0, (TA)mu0, sa, sb, sa_lo, sb_lo,
                                                                   sad, sbd, (TA)tol, maxit, ls_free_of<TA>(), init,
                                                                   flags, part, (TA *)fac, refresh, mrp);
    });
}

template <typename TA>
cudaError_t predictor(long N3, const TA *epse, const TA *deps, const TA *rho, TA *epst, TA *tauc, MatConst mc,
                      double r, const double *dE6, int use_field, cudaStream_t s) {
    const int blocks = (int)((N3 + 255) / 256);
    // the extrapolation ratio and the uniform guess rounded to the field precision once, here
    k_predictor<TA><<<blocks, 256, 0, s>>>(N3, epse, deps, rho, epst, tauc, mc, (TA)r, use_field, (TA)dE6[0],
                                           (TA)dE6[1], (TA)dE6[2], (TA)dE6[3], (TA)dE6[4], (TA)dE6[5]);
    return cudaGetLastError();
}

template <typename TA>
cudaError_t state_update(long N3, const TA *sig, const TA *tauc, const int32_t *g0, const TA *Mtab, TA *epst,
                         TA *epse, TA *epsp, TA *deps, TA *rho, double *k, MatConst mc, cudaStream_t s) {
    const int blocks = (int)((N3 + kThreads - 1) / kThreads);
    k_state_update<TA><<<blocks, kThreads, 0, s>>>(N3, sig, tauc, g0, Mtab, epst, epse, epsp, deps, rho, k, mc);
    return cudaGetLastError();
}

template <typename TA> cudaError_t total_strain(long N3, const TA *epse, const TA *epsp, TA *eps, cudaStream_t s) {
    const long n = 6 * N3;
    k_total_strain<TA><<<(int)((n + 255) / 256), 256, 0, s>>>(N3, epse, epsp, eps);
    return cudaGetLastError();
}

#define EVP_INST(TA)                                                                                              \
    template cudaError_t newton_field<TA>(long, const TA *, const TA *, const int32_t *, TA *, const TA *,        \
                                          const TA *, MatConst, double, int, int, int *, cudaStream_t,           \
                                          const int *, const TA *, MRPtr<TA>);                                   \
    template cudaError_t newton_chord_field<TA>(long, const TA *, const TA *, const int32_t *, TA *, const TA *,  \
                                                const TA *, void *, MatConst, double, int, int, int, int *,       \
                                                int32_t *, int, cudaStream_t, const int *, const TA *, MRPtr<TA>, int); \
    template cudaError_t al_local<TA>(long, const TA *, const TA *, const TA *, const int32_t *, TA *, TA *, TA *, \
                                      const TA *, const TA *, const TA *, MatConst, double, double, double, int, int, \
                                      int, int *, double *, void *, int, cudaStream_t, int, MRPtr<TA>);           \
    template cudaError_t predictor<TA>(long, const TA *, const TA *, const TA *, TA *, TA *, MatConst, double,    \
                                       const double *, int, cudaStream_t);                                        \
    template cudaError_t state_update<TA>(long, const TA *, const TA *, const int32_t *, const TA *, TA *, TA *,  \
                                          TA *, TA *, TA *, double *, MatConst, cudaStream_t);                    \
    template cudaError_t total_strain<TA>(long, const TA *, const TA *, TA *, cudaStream_t);
EVP_INST(float)
EVP_INST(double)
#undef EVP_INST

}  // namespace evp
