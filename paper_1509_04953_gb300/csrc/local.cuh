// Per-voxel constitutive routines shared by the forward Newton and the adjoint kernels
// (Sec. 2.1 Eqs. HookeLaw / PlasticRate with the power-law flow rule, and with the Ma-Roters flow rule of
// Sec. 2.2 Eq. FlowRule).
#pragma once
#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace evp {

template <typename T> __device__ __forceinline__ T dsqrt(T x) { return sqrt(x); }
__device__ __forceinline__ double dsqrt(double x) { return __dsqrt_rn(x); }
template <typename T> __device__ __forceinline__ T drcp(T x) { return (T)1 / x; }
__device__ __forceinline__ double drcp(double x) { return __drcp_rn(x); }

// |x|^(n-1) for the power law; fast path for small integer n (exponentiation by squaring).
template <typename T> __device__ __forceinline__ T pow_nm1(T ax, const MatConst &mc) {
    if (mc.n_int == 10) {
        // the workloads' exponent: |x|^9 = |x| ((|x|^2)^2)^2, the very products the bit loop below forms for
        // e = 9 (its first factor 1 * |x| is exact), in 4 multiplications instead of 18 operations
        const T b2 = ax * ax, b4 = b2 * b2, b8 = b4 * b4;
        return ax * b8;
    }
    if (mc.n_int > 0) {
        // branch-free: the same products in the same order as the bit loop, over all six bits of
        // e <= 63 (selects instead of branches, so independent slip systems can be interleaved)
        const int e = mc.n_int - 1;
        T r = (T)1, b = ax;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            r = ((e >> k) & 1) ? r * b : r;
            b = b * b;
        }
        return r;
    }
    return ax > (T)0 ? (T)pow((double)ax, mc.n - 1.0) : (T)0;
}

// Flow-rule constants in the arithmetic precision.
template <typename TA> __device__ __forceinline__ void flow_consts(const MatConst &mc, TA &dt, TA &g0, TA &nn) {
    if constexpr (sizeof(TA) == 4) { dt = mc.dt_f; g0 = mc.gdot0_f; nn = mc.n_f; }
    else { dt = mc.dt; g0 = mc.gdot0; nn = mc.n; }
}

// Packed lower-triangular index of (i, j), j <= i.
__host__ __device__ constexpr int pk(int i, int j) { return i * (i + 1) / 2 + j; }

// Per-grain tables: compliance rows (36 words) and Schmid vectors (12 x 6 words) per grain, each grain
// starting on a 16-byte boundary (144 g / 288 g bytes in FP32, twice that in FP64). They are read with
// 16-byte vector loads; the load instructions, not the bytes (the tables sit in L1), are what a
// per-voxel kernel issuing one load per word runs short of.
template <typename TA> __device__ __forceinline__ void load_compliance(const TA *__restrict__ S, TA Sp[21]) {
    TA full[36];
    if constexpr (sizeof(TA) == 4) {
        const float4 *S4 = reinterpret_cast<const float4 *>(S);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float4 t = __ldg(S4 + k);
            full[4 * k] = t.x; full[4 * k + 1] = t.y; full[4 * k + 2] = t.z; full[4 * k + 3] = t.w;
        }
    } else {
        const double2 *S2 = reinterpret_cast<const double2 *>(S);
#pragma unroll
        for (int k = 0; k < 18; ++k) {
            const double2 t = __ldg(S2 + k);
            full[2 * k] = t.x; full[2 * k + 1] = t.y;
        }
    }
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) Sp[i * (i + 1) / 2 + j] = full[6 * i + j];
}
// Schmid vectors of slip systems 2p and 2p+1 (12 consecutive words, 16-byte aligned).
template <typename TA> __device__ __forceinline__ void load_slip_pair(const TA *__restrict__ M, int p, TA m[12]) {
    if constexpr (sizeof(TA) == 4) {
        const float4 *M4 = reinterpret_cast<const float4 *>(M + 12 * p);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float4 t = __ldg(M4 + k);
            m[4 * k] = t.x; m[4 * k + 1] = t.y; m[4 * k + 2] = t.z; m[4 * k + 3] = t.w;
        }
    } else {
        const double2 *M2 = reinterpret_cast<const double2 *>(M + 12 * p);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const double2 t = __ldg(M2 + k);
            m[2 * k] = t.x; m[2 * k + 1] = t.y;
        }
    }
}

// Stored tangent factors (21 words per voxel): 16-byte vector planes, then one scalar plane for the last word.
// FP32: planes 0-4 are float4 (words 4k..4k+3), plane 5 is float (word 20); FP64: planes 0-9 are double2 (words
// 2k, 2k+1), plane 10 is double (word 20). Each plane holds N3 voxels, so a voxel's factors come in 5 (10)
// coalesced vector loads and one scalar load, with no padding words.
template <typename TS> __host__ __device__ constexpr int factor_words() { return 21; }
template <typename TS> __device__ __forceinline__ void load_factors(const TS *__restrict__ fac, long N3, long v, TS F[21]) {
    if constexpr (sizeof(TS) == 4) {
        const float4 *f4 = reinterpret_cast<const float4 *>(fac);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const float4 t = f4[k * N3 + v];
            F[4 * k] = t.x; F[4 * k + 1] = t.y; F[4 * k + 2] = t.z; F[4 * k + 3] = t.w;
        }
        F[20] = fac[20 * N3 + v];
    } else {
        const double2 *f2 = reinterpret_cast<const double2 *>(fac);
#pragma unroll
        for (int k = 0; k < 10; ++k) {
            const double2 t = f2[k * N3 + v];
            F[2 * k] = t.x; F[2 * k + 1] = t.y;
        }
        F[20] = fac[20 * N3 + v];
    }
}
template <typename TS> __device__ __forceinline__ void store_factors(TS *__restrict__ fac, long N3, long v, const TS F[21]) {
    if constexpr (sizeof(TS) == 4) {
        float4 *f4 = reinterpret_cast<float4 *>(fac);
#pragma unroll
        for (int k = 0; k < 5; ++k) f4[k * N3 + v] = make_float4(F[4 * k], F[4 * k + 1], F[4 * k + 2], F[4 * k + 3]);
    } else {
        double2 *f2 = reinterpret_cast<double2 *>(fac);
#pragma unroll
        for (int k = 0; k < 10; ++k) f2[k * N3 + v] = make_double2(F[2 * k], F[2 * k + 1]);
    }
    fac[20 * N3 + v] = F[20];
}

// The same factors staged through shared memory: prefetch_factors starts asynchronous copies of this thread's 21
// words into its own slots (plane-major, blockDim.x threads per plane: the vector planes, then the scalar plane),
// prefetched_factors waits for this thread's copies and reads them. Only the issuing thread reads its slots, so no
// barrier is needed.
template <typename TS> __device__ __forceinline__ void prefetch_factors(const TS *__restrict__ fac, long N3, long v, TS *sh) {
    const int t = threadIdx.x, nt = blockDim.x;
    constexpr int W = sizeof(TS) == 4 ? 4 : 2, P = 20 / W;   // words per vector, vector planes
#pragma unroll
    for (int k = 0; k < P; ++k) {
        const unsigned sa = (unsigned)__cvta_generic_to_shared(sh + (k * nt + t) * W);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(fac + (k * N3 + v) * W) : "memory");
    }
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sh + P * nt * W + t);
    if constexpr (sizeof(TS) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(fac + 20 * N3 + v) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(fac + 20 * N3 + v) : "memory");
}
template <typename TS> __device__ __forceinline__ void prefetched_factors(const TS *sh, TS F[21]) {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    const int t = threadIdx.x, nt = blockDim.x;
    constexpr int W = sizeof(TS) == 4 ? 4 : 2, P = 20 / W;
    if constexpr (sizeof(TS) == 4) {
        const float4 *s4 = reinterpret_cast<const float4 *>(sh);
#pragma unroll
        for (int k = 0; k < P; ++k) {
            const float4 q = s4[k * nt + t];
            F[4 * k] = q.x; F[4 * k + 1] = q.y; F[4 * k + 2] = q.z; F[4 * k + 3] = q.w;
        }
    } else {
        const double2 *s2 = reinterpret_cast<const double2 *>(sh);
#pragma unroll
        for (int k = 0; k < P; ++k) {
            const double2 q = s2[k * nt + t];
            F[2 * k] = q.x; F[2 * k + 1] = q.y;
        }
    }
    F[20] = sh[P * nt * W + t];
}

template <typename TA> struct Eval {
    TA r[6];
    TA K[21];
    TA phi;
};

template <typename TA>
__device__ __forceinline__ void evaluate(const TA Sp[21], const TA *__restrict__ M, const TA etr[6], TA tauc, TA inv_tc,
                                         const TA sg[6], const MatConst &mc, Eval<TA> &e) {
    TA dt, g0, nn;
    flow_consts(mc, dt, g0, nn);
    TA phi = (TA)0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        TA acc = (TA)0;
#pragma unroll
        for (int j = 0; j < 6; ++j) acc += Sp[i >= j ? pk(i, j) : pk(j, i)] * sg[j];
        e.r[i] = acc - etr[i];
        phi += sg[i] * ((TA)0.5 * acc - etr[i]);
    }
#pragma unroll
    for (int q = 0; q < 21; ++q) e.K[q] = Sp[q];
    const TA cphi = dt * g0 * tauc / (nn + (TA)1);
    const TA cslope = dt * nn * g0 * inv_tc;
#pragma unroll 1
    for (int p = 0; p < 6; ++p) {
      TA mm[12];
      load_slip_pair(M, p, mm);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const TA *m = mm + 6 * h;
        TA tau = (TA)0;
#pragma unroll
        for (int i = 0; i < 6; ++i) tau += m[i] * sg[i];
        const TA x = tau * inv_tc;
        const TA ax = fabs(x);
        const TA p9 = pow_nm1(ax, mc);       // |x|^(n-1)
        const TA p10 = p9 * ax;              // |x|^n
        const TA gd = x < (TA)0 ? -g0 * p10 : g0 * p10;
        const TA slope = cslope * p9;
        TA sm[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            e.r[i] += dt * gd * m[i];
            sm[i] = slope * m[i];
        }
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int j = 0; j <= i; ++j) e.K[pk(i, j)] += sm[i] * m[j];
        phi += cphi * p10 * ax;
      }
    }
    e.phi = phi;
}


// ---- Ma-Roters flow rule (Sec. 2.2, Eq. FlowRule) ----
// gdot = A sinh((|tau| - tau_pass) / tau_cut) sign(tau) above the passing stress, A = ga tau_pass; its
// derivative A cosh(.) / tau_cut and the convex potential A tau_cut (cosh(.) - 1) (zero below). With
// u = expm1(x) and w = 1/(1+u) = exp(-x): sinh x = u (1+w)/2 and cosh x - 1 = u (1-w)/2, free of
// cancellation for small x; an overflowing x gives infinities that the line search rejects.
template <typename TA> struct FlowMR {
    const TA *__restrict__ tpi;   // (tau_pass, 1 / tau_cut) pairs, 12 x N3 (layout of MRPtr)
    long N3, v;
    TA tref;                      // stopping scale: min_a tau_pass^a
};
template <typename TA> __device__ __forceinline__ TA flow_ref(TA tauc) { return tauc; }
template <typename TA> __device__ __forceinline__ TA flow_ref(const FlowMR<TA> &f) { return f.tref; }
__device__ __forceinline__ float dexpm1(float x) { return expm1f(x); }
// 1/x rounded to nearest (FP32 reciprocal instruction with its IEEE fix-up) / FP64 division
__device__ __forceinline__ float rcp_fast(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_fast(double x) { return 1.0 / x; }
__device__ __forceinline__ double dexpm1(double x) { return expm1(x); }
template <typename TA> __device__ __forceinline__ TA mr_ga(const MatConst &mc) {
    if constexpr (sizeof(TA) == 4) return mc.mr_ga_f;
    else return mc.mr_ga;
}
template <typename TA>
__device__ __forceinline__ void mr_flow(TA tau, TA tp, TA itc, TA ga, TA &gd, TA &slope, TA &psi) {
    const TA x = (fabs(tau) - tp) * itc;
    if (x > (TA)0) {
        const TA u = dexpm1(x), w = rcp_fast(u + (TA)1), A = ga * tp;
        const TA sh = (TA)0.5 * u * ((TA)1 + w), chm1 = (TA)0.5 * u * ((TA)1 - w);
        gd = tau < (TA)0 ? -A * sh : A * sh;
        slope = A * ((TA)1 + chm1) * itc;
        psi = A * chm1 * rcp_fast(itc);   // the potential only steers the line search
    } else {
        gd = (TA)0; slope = (TA)0; psi = (TA)0;
    }
}
template <typename TA> __device__ __forceinline__ void mr_sys(const FlowMR<TA> &f, int a, TA &tp, TA &itc) {
    if constexpr (sizeof(TA) == 4) {
        const float2 t = __ldg(reinterpret_cast<const float2 *>(f.tpi) + (long)a * f.N3 + f.v);
        tp = t.x; itc = t.y;
    } else {
        const double2 t = __ldg(reinterpret_cast<const double2 *>(f.tpi) + (long)a * f.N3 + f.v);
        tp = t.x; itc = t.y;
    }
}

template <typename TA>
__device__ __forceinline__ void evaluate(const TA Sp[21], const TA *__restrict__ M, const TA etr[6], const FlowMR<TA> &f,
                                         TA, const TA sg[6], const MatConst &mc, Eval<TA> &e) {
    TA dt, g0, nn;
    flow_consts(mc, dt, g0, nn);
    const TA ga = mr_ga<TA>(mc);
    TA phi = (TA)0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        TA acc = (TA)0;
#pragma unroll
        for (int j = 0; j < 6; ++j) acc += Sp[i >= j ? pk(i, j) : pk(j, i)] * sg[j];
        e.r[i] = acc - etr[i];
        phi += sg[i] * ((TA)0.5 * acc - etr[i]);
    }
#pragma unroll
    for (int q = 0; q < 21; ++q) e.K[q] = Sp[q];
#pragma unroll 1
    for (int p = 0; p < 6; ++p) {
      TA mm[12];
      load_slip_pair(M, p, mm);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const TA *m = mm + 6 * h;
        TA tau = (TA)0;
#pragma unroll
        for (int i = 0; i < 6; ++i) tau += m[i] * sg[i];
        TA tp, itc, gd, slope, psi;
        mr_sys(f, 2 * p + h, tp, itc);
        mr_flow(tau, tp, itc, ga, gd, slope, psi);
        TA sm[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            e.r[i] += dt * gd * m[i];
            sm[i] = dt * slope * m[i];
        }
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int j = 0; j <= i; ++j) e.K[pk(i, j)] += sm[i] * m[j];
        phi += dt * psi;
      }
    }
    e.phi = phi;
}

// Reciprocal: FP32 division for float; for double an FP32 seed refined by two Newton steps
// r <- r (2 - x r) (each doubles the correct bits: 24 -> 48 -> full precision).
__device__ __forceinline__ float rcp_s(float x) { return 1.0f / x; }
__device__ __forceinline__ double rcp_s(double x) {
    double r = (double)(1.0f / (float)x);
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}

// LDL^T solve of K d = r (K packed lower, SPD; no square roots). L is unit lower, D diagonal.
// Returns false if a pivot is not positive.
template <typename TS, typename TA> __device__ __forceinline__ bool ldl_solve(const TA Kin[21], const TA rin[6], TA dout[6]) {
    TS L[21], invD[6], w[6];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        TS dj = (TS)Kin[pk(j, j)];
#pragma unroll
        for (int k = 0; k < j; ++k) {
            w[k] = L[pk(j, k)] * L[pk(k, k)];   // L_jk D_k (L[kk] holds D_k)
            dj -= w[k] * L[pk(j, k)];
        }
        ok = ok && (dj > (TS)0);
        dj = dj > (TS)0 ? dj : (TS)1;
        L[pk(j, j)] = dj;
        invD[j] = rcp_s(dj);
#pragma unroll
        for (int i = j + 1; i < 6; ++i) {
            TS t = (TS)Kin[pk(i, j)];
#pragma unroll
            for (int k = 0; k < j; ++k) t -= L[pk(i, k)] * w[k];
            L[pk(i, j)] = t * invD[j];
        }
    }
    TS y[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        TS t = (TS)rin[i];
#pragma unroll
        for (int k = 0; k < i; ++k) t -= L[pk(i, k)] * y[k];
        y[i] = t;
    }
#pragma unroll
    for (int i = 5; i >= 0; --i) {
        TS t = y[i] * invD[i];
#pragma unroll
        for (int k = i + 1; k < 6; ++k) t -= L[pk(k, i)] * y[k];
        y[i] = t;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) dout[i] = (TA)y[i];
    return ok;
}


// Residual and potential only (no tangent): the cost of a chord step.
template <typename TA> struct EvalR {
    TA r[6];
    TA phi;
};
// UNROLL: slip-system pairs unrolled per loop trip (6 = fully, letting the table loads run ahead of
// the arithmetic where registers allow).
template <typename TA, int UNROLL = 1>
__device__ __forceinline__ void evaluate_r(const TA Sp[21], const TA *__restrict__ M, const TA etr[6], TA tauc, TA inv_tc,
                                           const TA sg[6], const MatConst &mc, EvalR<TA> &e) {
    TA dt, g0, nn;
    flow_consts(mc, dt, g0, nn);
    TA phi = (TA)0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        TA acc = (TA)0;
#pragma unroll
        for (int j = 0; j < 6; ++j) acc += Sp[i >= j ? pk(i, j) : pk(j, i)] * sg[j];
        e.r[i] = acc - etr[i];
        phi += sg[i] * ((TA)0.5 * acc - etr[i]);
    }
    const TA cphi = dt * g0 * tauc / (nn + (TA)1);
#pragma unroll UNROLL
    for (int p = 0; p < 6; ++p) {
        TA mm[12];
        load_slip_pair(M, p, mm);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const TA *m = mm + 6 * h;
            TA tau = (TA)0;
#pragma unroll
            for (int i = 0; i < 6; ++i) tau += m[i] * sg[i];
            const TA x = tau * inv_tc, ax = fabs(x);
            const TA p10 = pow_nm1(ax, mc) * ax;
            const TA gd = x < (TA)0 ? -g0 * p10 : g0 * p10;
            const TA dg = dt * gd;
#pragma unroll
            for (int i = 0; i < 6; ++i) e.r[i] += dg * m[i];
            phi += cphi * p10 * ax;
        }
    }
    e.phi = phi;
}


template <typename TA, int UNROLL = 1>
__device__ __forceinline__ void evaluate_r(const TA Sp[21], const TA *__restrict__ M, const TA etr[6],
                                           const FlowMR<TA> &f, TA, const TA sg[6], const MatConst &mc, EvalR<TA> &e) {
    TA dt, g0, nn;
    flow_consts(mc, dt, g0, nn);
    const TA ga = mr_ga<TA>(mc);
    TA phi = (TA)0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        TA acc = (TA)0;
#pragma unroll
        for (int j = 0; j < 6; ++j) acc += Sp[i >= j ? pk(i, j) : pk(j, i)] * sg[j];
        e.r[i] = acc - etr[i];
        phi += sg[i] * ((TA)0.5 * acc - etr[i]);
    }
#pragma unroll UNROLL
    for (int p = 0; p < 6; ++p) {
        TA mm[12];
        load_slip_pair(M, p, mm);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const TA *m = mm + 6 * h;
            TA tau = (TA)0;
#pragma unroll
            for (int i = 0; i < 6; ++i) tau += m[i] * sg[i];
            TA tp, itc, gd, slope, psi;
            mr_sys(f, 2 * p + h, tp, itc);
            mr_flow(tau, tp, itc, ga, gd, slope, psi);
            const TA dg = dt * gd;
#pragma unroll
            for (int i = 0; i < 6; ++i) e.r[i] += dg * m[i];
            phi += dt * psi;
        }
    }
    e.phi = phi;
}

// LDL^T factorisation kept for reuse: F[0..14] = strict lower L (row-major by packed index, diagonal
// slots skipped), F[15..20] = 1/D. Returns false if a pivot is not positive.
template <typename TS, typename TA> __device__ __forceinline__ bool ldl_factor(const TA Kin[21], TS F[21]) {
    TS L[21], invD[6], w[6];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        TS dj = (TS)Kin[pk(j, j)];
#pragma unroll
        for (int k = 0; k < j; ++k) {
            w[k] = L[pk(j, k)] * L[pk(k, k)];
            dj -= w[k] * L[pk(j, k)];
        }
        ok = ok && (dj > (TS)0);
        dj = dj > (TS)0 ? dj : (TS)1;
        L[pk(j, j)] = dj;
        invD[j] = rcp_s(dj);
#pragma unroll
        for (int i = j + 1; i < 6; ++i) {
            TS t = (TS)Kin[pk(i, j)];
#pragma unroll
            for (int k = 0; k < j; ++k) t -= L[pk(i, k)] * w[k];
            L[pk(i, j)] = t * invD[j];
        }
    }
    int q = 0;
#pragma unroll
    for (int i = 1; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < i; ++j) F[q++] = L[pk(i, j)];
#pragma unroll
    for (int j = 0; j < 6; ++j) F[15 + j] = invD[j];
    return ok;
}

template <typename TS, typename TA> __device__ __forceinline__ void ldl_apply(const TS F[21], const TA rin[6], TA dout[6]) {
    // strict-lower index of (i, j), j < i: i(i-1)/2 + j
    TS y[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        TS t = (TS)rin[i];
#pragma unroll
        for (int k = 0; k < i; ++k) t -= F[i * (i - 1) / 2 + k] * y[k];
        y[i] = t;
    }
#pragma unroll
    for (int i = 5; i >= 0; --i) {
        TS t = y[i] * F[15 + i];
#pragma unroll
        for (int k = i + 1; k < 6; ++k) t -= F[k * (k - 1) / 2 + i] * y[k];
        y[i] = t;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) dout[i] = (TA)y[i];
}

// FP64 residual and potential with the tangent assembled in FP32 (the tangent only steers the
// iteration; the converged stress is fixed by the FP64 residual). Sf / Mf are FP32 copies of the
// per-grain compliance and Schmid tables.
struct EvalDF {
    double r[6];
    float K[21];
    double phi;
};
__device__ __forceinline__ void evaluate_df(const double Sp[21], const double *__restrict__ M, const float Spf[21],
                                            const float *__restrict__ Mf, const double etr[6], double tauc,
                                            double inv_tc, const double sg[6], const MatConst &mc, EvalDF &e) {
    const double dt = mc.dt, g0 = mc.gdot0, nn = mc.n;
    double phi = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        double acc = 0.0;
#pragma unroll
        for (int j = 0; j < 6; ++j) acc += Sp[i >= j ? pk(i, j) : pk(j, i)] * sg[j];
        e.r[i] = acc - etr[i];
        phi += sg[i] * (0.5 * acc - etr[i]);
    }
#pragma unroll
    for (int q = 0; q < 21; ++q) e.K[q] = Spf[q];
    const double cphi = dt * g0 * tauc / (nn + 1.0);
    const float cslope = (float)(dt * nn * g0 * inv_tc);
#pragma unroll 1
    for (int p = 0; p < 6; ++p) {
      double mm[12];
      float mmf[12];
      load_slip_pair(M, p, mm);
      load_slip_pair(Mf, p, mmf);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const double *m = mm + 6 * h;
        const float *mf = mmf + 6 * h;
        double tau = 0.0;
#pragma unroll
        for (int i = 0; i < 6; ++i) tau += m[i] * sg[i];
        const double x = tau * inv_tc, ax = fabs(x);
        const double p9 = pow_nm1(ax, mc);
        const double p10 = p9 * ax;
        const double dg = x < 0.0 ? -dt * g0 * p10 : dt * g0 * p10;
#pragma unroll
        for (int i = 0; i < 6; ++i) e.r[i] += dg * m[i];
        phi += cphi * p10 * ax;
        const float slope = cslope * (float)p9;
        float sm[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) sm[i] = slope * mf[i];
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int j = 0; j <= i; ++j) e.K[pk(i, j)] += sm[i] * mf[j];
      }
    }
    e.phi = phi;
}

}  // namespace evp
