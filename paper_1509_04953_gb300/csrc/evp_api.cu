// C ABI of libevp_gb300 (declared in include/evp.h): handle, workspace layout, increment driver,
// nucleation and phase-field entry points, field I/O. All device work is enqueued on the
// handle's stream; the library never allocates device memory.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "../../include/evp.h"
#include "common.cuh"
#include "fpctl.cuh"
#include "kernels.h"

using namespace evp;

struct evp_handle {
    evp_config cfg;
    evp_params p;
    int n, G, K, prec;
    long N3;
    long H;          // half-spectrum points per field
    int dbl;         // 1: fields are double
    size_t tsz;      // sizeof(field type)
    cudaStream_t st;
    char *ws;
    size_t ws_bytes;
    // fields
    void *sig, *sigk, *epse, *epst, *epsp, *deps, *rho, *tauc, *eta, *eta2, *spec, *Stab, *Mtab, *fac, *Sal, *lam, *pal;
    float *Stabf, *Mtabf;
    double *k, *kappa, *partials, *scal;
    int32_t *g0, *g, *gprev, *draws, *ids, *ids2, *flags, *blk_counts, *blk_off, *count, *wlist;
    int nsm;
    int r, npf;      // phase-field grid: r = 1 (the mechanics grid) or 2 (refined), npf = r n points per edge
    long N3pf;
    int32_t *gpf;    // argmax id per PF point (= g when r = 1)
    uint8_t *rmax, *rmax2;   // per-row slot bounds of (ids, eta) and (ids2, eta2), for the tiled PF step
    long rmax_bytes;
    double *kpf;     // rho_tot on the PF grid (= k when r = 1)
    int fac_valid;   // stored tangent factors hold a factorisation (of some earlier state) for every voxel
    uint32_t *bitmap;
    int bitmap_words, max_ids, npartials;
    // macroscopic state (host)
    double E[6], dE_prev[6];
    int have_prev, next_id;
    uint64_t seed;
    MatConst mc;
    PFConst pc;
    // adjoint recording
    char *adj;
    size_t adj_bytes;
    int adj_T, adj_c, adj_t;
    double *adj_dE33, *adj_dt, *adj_E, *adj_dEp;
    int *adj_hp;
    // instrumentation
    int64_t launches;
    int64_t newton_solves, newton_evals, newton_refreshes;
    uint32_t prof;   // profiled kernel classes (bit mask)
    double prof_ms[EVP_NCLASS];
    int64_t prof_n[EVP_NCLASS];
    struct Pend { int cls; cudaEvent_t a, b; };
    static constexpr int kMaxPend = 512;   // bracketed launches awaiting collection (several queued iterations)
    Pend pend[kMaxPend];
    int npend;
    cudaEvent_t pool[2 * kMaxPend];
    int npool;
    void *ctl;   // device fixed-point control block (FpCtl)
    // Ma-Roters law (cfg.law == EVP_LAW_MR): rho holds rho_SSD; signed GND components gs, ge and the accumulated
    // rho_GND (12 x N3 each); frozen tau_pass and 1/tau_cut (12 x N3 each, tauc = min tau_pass); shear rates
    // and (sigma_vm, gdot_vm) of the last increment; sample-frame d and t per grain; constants; l_eff
    int mr;
    void *gs, *ge, *gnd, *tpi, *gdm, *aux, *vec;
    MRConst mrc;
    double leff;
    char err[512];
    ~evp_handle() {
        std::free(adj_dE33); std::free(adj_dt); std::free(adj_E); std::free(adj_dEp); std::free(adj_hp);
        for (int i = 0; i < npend; ++i) { cudaEventDestroy(pend[i].a); cudaEventDestroy(pend[i].b); }
        for (int i = 0; i < npool; ++i) cudaEventDestroy(pool[i]);
    }
};

namespace {

int fail(evp_handle *h, int code, const char *fmt, ...) {
    if (h) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(h->err, sizeof h->err, fmt, ap);
        va_end(ap);
    }
    return code;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return fail(h, EVP_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

cudaEvent_t ev_get(evp_handle *h) {
    if (h->npool > 0) return h->pool[--h->npool];
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
void ev_put(evp_handle *h, cudaEvent_t e) {
    if (!e) return;
    if (h->npool < 2 * evp_handle::kMaxPend) h->pool[h->npool++] = e;
    else cudaEventDestroy(e);
}
// Accumulate the device time of every bracketed launch whose events have completed.
void prof_collect(evp_handle *h) {
    int keep = 0;
    for (int i = 0; i < h->npend; ++i) {
        auto &q = h->pend[i];
        float ms = 0.f;
        if (cudaEventQuery(q.b) == cudaSuccess && cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) {
            h->prof_ms[q.cls] += ms;
            h->prof_n[q.cls] += 1;
            ev_put(h, q.a);
            ev_put(h, q.b);
        } else {
            h->pend[keep++] = q;
        }
    }
    h->npend = keep;
}
struct ProfScope {
    evp_handle *h;
    int cls;
    cudaEvent_t a = nullptr;
    ProfScope(evp_handle *h_, int c, int nk) : h(h_), cls(c) {
        h->launches += nk;
        if (h->prof & (1u << c)) {
            if (h->npend >= evp_handle::kMaxPend) {
                cudaStreamSynchronize(h->st);
                prof_collect(h);
            }
            a = ev_get(h);
            if (a) cudaEventRecord(a, h->st);
        }
    }
    ~ProfScope() {
        if (!a) return;
        cudaEvent_t b = ev_get(h);
        if (!b) { ev_put(h, a); return; }
        cudaEventRecord(b, h->st);
        h->pend[h->npend++] = {cls, a, b};
    }
};
#define PROF(cls, nk) ProfScope prof_scope(h, (cls), (nk))

bool pow2(int n) { return n >= 4 && n <= 256 && (n & (n - 1)) == 0; }

int check_cfg(const evp_config *c, char *why, size_t wl) {
    if (!c) return snprintf(why, wl, "config is NULL"), EVP_ERR_ARG;
    if (!pow2(c->n)) return snprintf(why, wl, "n=%d must be a power of two in [4,256]", c->n), EVP_ERR_ARG;
    if (c->grains < 1) return snprintf(why, wl, "grains=%d must be >= 1", c->grains), EVP_ERR_ARG;
    if (c->kmax < 1 || c->kmax > 8) return snprintf(why, wl, "kmax=%d must be in [1,8]", c->kmax), EVP_ERR_ARG;
    if (c->precision < EVP_FP64 || c->precision > EVP_MIXED_FAST)
        return snprintf(why, wl, "unknown precision %d", c->precision), EVP_ERR_ARG;
    if (c->max_iter < 1 || c->newton_max < 1) return snprintf(why, wl, "iteration caps must be >= 1"), EVP_ERR_ARG;
    if (!(c->tol >= 0.0) || !(c->newton_tol > 0.0)) return snprintf(why, wl, "tolerances must be >= 0"), EVP_ERR_ARG;
    if (c->max_ids != 0 && c->max_ids < c->grains) return snprintf(why, wl, "max_ids < grains"), EVP_ERR_ARG;
    if (c->scheme != EVP_SCHEME_BASIC && c->scheme != EVP_SCHEME_AL)
        return snprintf(why, wl, "unknown scheme %d", c->scheme), EVP_ERR_ARG;
    if (c->scheme == EVP_SCHEME_AL && !(c->al_scale >= 1.0))
        return snprintf(why, wl, "al_scale must be >= 1"), EVP_ERR_ARG;
    if (!(c->newton_adapt >= 0.0)) return snprintf(why, wl, "newton_adapt must be >= 0"), EVP_ERR_ARG;
    if (c->pf_refine < 0 || c->pf_refine > 2) return snprintf(why, wl, "pf_refine must be 0, 1 or 2"), EVP_ERR_ARG;
    if (c->law != EVP_LAW_POWER && c->law != EVP_LAW_MR) return snprintf(why, wl, "unknown law %d", c->law), EVP_ERR_ARG;
    if (!(c->ref_scale == 0.0 || (c->ref_scale >= 0.5 && c->ref_scale <= 4.0)))
        return snprintf(why, wl, "ref_scale must be 0 or in [0.5, 4]"), EVP_ERR_ARG;
    if (c->law == EVP_LAW_MR && c->newton_mode == EVP_NEWTON_F32_TANGENT)
        return snprintf(why, wl, "EVP_NEWTON_F32_TANGENT covers the power law only"), EVP_ERR_ARG;
    if (c->newton_mode != EVP_NEWTON_EXACT && c->newton_mode != EVP_NEWTON_REUSE &&
        !(c->newton_mode == EVP_NEWTON_F32_TANGENT && c->precision == EVP_FP64))
        return snprintf(why, wl, "newton_mode %d is not available for precision %d", c->newton_mode, c->precision),
               EVP_ERR_ARG;
    return EVP_OK;
}

// Walk the workspace in a fixed order; assigns pointers when h != nullptr. 256-byte aligned.
size_t layout(const evp_config *c, evp_handle *h, char *base) {
    const long n = c->n, N3 = n * n * n, H = n * n * (n / 2 + 1);
    const size_t T = c->precision == EVP_FP64 ? 8 : 4;
    const int K = c->kmax, G = c->grains;
    const long max_ids = c->max_ids ? c->max_ids : (long)G + 8 * N3;
    const int nb = nucleate_blocks(N3);
    const int r = c->pf_refine == 2 ? 2 : 1;
    const long M3 = (long)r * n * r * n * r * n;   // phase-field points
    const int npart = std::max(std::max(fft_z_blocks((int)n, T == 8), 2 * pf_stat_blocks(M3) + 1), 14 * al_blocks(N3));
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        off = (off + 255) & ~(size_t)255;
        char *p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    char *sig = take(6 * N3 * T), *sigk = take(6 * N3 * T), *epse = take(6 * N3 * T), *epst = take(6 * N3 * T);
    char *epsp = take(6 * N3 * T), *deps = take(6 * N3 * T), *rho = take(12 * N3 * T), *tauc = take(N3 * T);
    char *eta = take(K * M3 * T), *eta2 = take(K * M3 * T), *spec = take(6 * H * 2 * T);
    char *Stab = take(36 * (size_t)G * T), *Mtab = take(72 * (size_t)G * T);
    // stored tangent factors: 21 words per voxel, in planes of 16-byte vectors and one scalar plane
    char *fac = take(c->newton_mode == EVP_NEWTON_REUSE ? 21 * N3 * T : 0);
    char *wlist = take(c->newton_mode == EVP_NEWTON_REUSE ? 4 * N3 : 0);      // voxels left for the second pass
    const bool al = c->scheme == EVP_SCHEME_AL;
    char *Sal = take(al ? 36 * (size_t)G * T : 0), *lam = take(al ? 6 * N3 * T : 0), *pal = take(al ? 6 * N3 * T : 0);
    const bool f32t = c->newton_mode == EVP_NEWTON_F32_TANGENT;
    char *Stabf = take(f32t ? 36 * (size_t)G * 4 : 0), *Mtabf = take(f32t ? 72 * (size_t)G * 4 : 0);
    char *k = take(N3 * 8), *kappa = take(N3 * 8);
    char *g0 = take(N3 * 4), *g = take(N3 * 4), *gprev = take(N3 * 4), *draws = take(N3 * 4);
    char *ids = take(K * M3 * 4), *ids2 = take(K * M3 * 4);
    char *gpf = take(r == 2 ? M3 * 4 : 0), *kpf = take(r == 2 ? M3 * 8 : 0);
    const long rb = pf_row_bounds_bytes(r * (int)n);
    char *rmax = take(rb), *rmax2 = take(rb);
    char *partials = take(sizeof(double) * npart), *scal = take(sizeof(double) * 64);
    char *flags = take(sizeof(int32_t) * 16);
    char *ctl = take(256);   // FpCtl
    char *blk_counts = take(sizeof(int32_t) * nb);
    char *blk_off = take(sizeof(int32_t) * nb + N3);   // offsets, then one mark byte per voxel
    char *count = take(sizeof(int32_t) * 4);
    const long words = (max_ids + 31) / 32;
    char *bitmap = take(sizeof(uint32_t) * words);
    const bool mr = c->law == EVP_LAW_MR;
    char *gnd3 = take(mr ? 36 * N3 * T : 0);   // rho_GNDs, rho_GNDet, rho_GND: one block (field EVP_F_GND)
    char *gs = gnd3, *ge = mr ? gnd3 + 12 * N3 * T : nullptr, *gnd = mr ? gnd3 + 24 * N3 * T : nullptr;
    char *tpi = take(mr ? 24 * N3 * T : 0), *gdm = take(mr ? 12 * N3 * T : 0);
    char *aux = take(mr ? 2 * N3 * T : 0), *vec = take(mr ? 72 * (size_t)G * T : 0);
    if (h) {
        h->mr = mr ? 1 : 0;
        h->gs = gs; h->ge = ge; h->gnd = gnd; h->tpi = tpi; h->gdm = gdm; h->aux = aux; h->vec = vec;
        h->sig = sig; h->sigk = sigk; h->epse = epse; h->epst = epst; h->epsp = epsp; h->deps = deps;
        h->rho = rho; h->tauc = tauc; h->eta = eta; h->eta2 = eta2; h->spec = spec; h->Stab = Stab; h->Mtab = Mtab;
        h->fac = fac;
        h->wlist = (int32_t *)wlist;
        h->Stabf = (float *)Stabf;
        h->Mtabf = (float *)Mtabf;
        h->Sal = Sal;
        h->lam = lam;
        h->pal = pal;
        h->k = (double *)k; h->kappa = (double *)kappa; h->g0 = (int32_t *)g0; h->g = (int32_t *)g;
        h->gprev = (int32_t *)gprev; h->draws = (int32_t *)draws; h->ids = (int32_t *)ids; h->ids2 = (int32_t *)ids2;
        h->partials = (double *)partials; h->scal = (double *)scal; h->flags = (int32_t *)flags;
        h->ctl = ctl;
        h->blk_counts = (int32_t *)blk_counts; h->blk_off = (int32_t *)blk_off; h->count = (int32_t *)count;
        h->bitmap = (uint32_t *)bitmap; h->bitmap_words = (int)words; h->max_ids = (int)max_ids;
        h->npartials = npart;
        h->r = r;
        h->npf = r * (int)n;
        h->N3pf = M3;
        h->gpf = r == 2 ? (int32_t *)gpf : h->g;
        h->rmax = (uint8_t *)rmax;
        h->rmax2 = (uint8_t *)rmax2;
        h->rmax_bytes = rb;
        h->kpf = r == 2 ? (double *)kpf : h->k;
    }
    return (off + 255) & ~(size_t)255;
}

// ---- per-grain tables (sample frame), built on the host in the field precision ----
const double kN4[4][3] = {{1, 1, 1}, {-1, 1, 1}, {1, -1, 1}, {1, 1, -1}};
const double kD4[4][3][3] = {{{0, 1, -1}, {1, 0, -1}, {1, -1, 0}},
                             {{0, 1, -1}, {1, 0, 1}, {1, 1, 0}},
                             {{0, 1, 1}, {1, 0, -1}, {1, 1, 0}},
                             {{0, 1, 1}, {1, 0, 1}, {1, -1, 0}}};
const int kMi[6] = {0, 1, 2, 1, 0, 0}, kMj[6] = {0, 1, 2, 2, 2, 1};

void tensor_to_mandel(const double T[3][3], double v[6]) {
    const double r2 = std::sqrt(2.0);
    for (int I = 0; I < 6; ++I) v[I] = (I < 3 ? 1.0 : r2) * T[kMi[I]][kMj[I]];
}

// 6x6 matrix Q with mandel(R A R^T) = Q mandel(A) for symmetric A.
void mandel_rotation(const double R[3][3], double Q[6][6]) {
    const double r2 = std::sqrt(2.0);
    for (int J = 0; J < 6; ++J) {
        double B[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        const int i = kMi[J], j = kMj[J];
        if (J < 3) B[i][j] = 1.0;
        else { B[i][j] = 1.0 / r2; B[j][i] = 1.0 / r2; }
        double RB[3][3], RBR[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                RB[a][b] = 0;
                for (int c = 0; c < 3; ++c) RB[a][b] += R[a][c] * B[c][b];
            }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                RBR[a][b] = 0;
                for (int c = 0; c < 3; ++c) RBR[a][b] += RB[a][c] * R[b][c];
            }
        double col[6];
        tensor_to_mandel(RBR, col);
        for (int I = 0; I < 6; ++I) Q[I][J] = col[I];
    }
}

template <typename T> void build_tables(const evp_params *p, int G, const double *quat, T *S, T *M) {
    const double den = (p->C11 - p->C12) * (p->C11 + 2.0 * p->C12);
    double Sc[6][6] = {};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Sc[i][j] = i == j ? (p->C11 + p->C12) / den : -p->C12 / den;
    for (int i = 3; i < 6; ++i) Sc[i][i] = 1.0 / (2.0 * p->C44);
    double mc[12][6];
    for (int pl = 0; pl < 4; ++pl)
        for (int d = 0; d < 3; ++d) {
            double nn[3], dd[3], Tm[3][3];
            for (int c = 0; c < 3; ++c) {
                nn[c] = kN4[pl][c] / std::sqrt(3.0);
                dd[c] = kD4[pl][d][c] / std::sqrt(2.0);
            }
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) Tm[a][b] = 0.5 * (dd[a] * nn[b] + dd[b] * nn[a]);
            tensor_to_mandel(Tm, mc[3 * pl + d]);
        }
    for (int g = 0; g < G; ++g) {
        const double *q = quat + 4 * g;
        const double qn = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        const double w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
        const double R[3][3] = {{1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
                                {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
                                {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
        double Q[6][6];
        mandel_rotation(R, Q);
        double QS[6][6];
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) {
                QS[i][j] = 0;
                for (int k = 0; k < 6; ++k) QS[i][j] += Q[i][k] * Sc[k][j];
            }
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) {
                double a = 0;
                for (int k = 0; k < 6; ++k) a += QS[i][k] * Q[j][k];
                S[36 * (size_t)g + 6 * i + j] = (T)a;
            }
        for (int a = 0; a < 12; ++a)
            for (int i = 0; i < 6; ++i) {
                double v = 0;
                for (int k = 0; k < 6; ++k) v += Q[i][k] * mc[a][k];
                M[72 * (size_t)g + 6 * a + i] = (T)v;
            }
    }
}

double voigt_mu(const evp_params *p) { return (p->C11 - p->C12 + 3.0 * p->C44) / 5.0; }
double voigt_lam(const evp_params *p) { return (p->C11 + 4.0 * p->C12 - 2.0 * p->C44) / 5.0; }

size_t field_bytes(const evp_handle *h, uint32_t bit) {
    const size_t N3 = (size_t)h->N3, T = h->tsz, K = (size_t)h->K;
    switch (bit) {
        case EVP_F_SIG: case EVP_F_EPS: case EVP_F_EPSP: case EVP_F_EPSE: case EVP_F_DEPS: return 6 * N3 * T;
        case EVP_F_RHO: return 12 * N3 * T;
        case EVP_F_K: case EVP_F_KAPPA: return N3 * 8;
        case EVP_F_GRAIN: case EVP_F_G0: case EVP_F_DRAWS: return N3 * 4;
        case EVP_F_IDS: return K * (size_t)h->N3pf * 4;
        case EVP_F_ETA: return K * (size_t)h->N3pf * T;
        case EVP_F_GRAIN_PF: return (size_t)h->N3pf * 4;
        case EVP_F_GND: return h->mr ? 36 * N3 * T : 0;
        default: return 0;
    }
}

void *field_ptr(evp_handle *h, uint32_t bit) {
    switch (bit) {
        case EVP_F_SIG: return h->sig;
        case EVP_F_EPSP: return h->epsp;
        case EVP_F_EPSE: return h->epse;
        case EVP_F_DEPS: return h->deps;
        case EVP_F_RHO: return h->rho;
        case EVP_F_K: return h->k;
        case EVP_F_KAPPA: return h->kappa;
        case EVP_F_GRAIN: return h->g;
        case EVP_F_G0: return h->g0;
        case EVP_F_DRAWS: return h->draws;
        case EVP_F_IDS: return h->ids;
        case EVP_F_ETA: return h->eta;
        case EVP_F_GRAIN_PF: return h->gpf;
        case EVP_F_GND: return h->gs;
        default: return nullptr;
    }
}


// ---- Ma-Roters law: host-built constants and thin launch wrappers ----
constexpr double kBoltzmann = 1.380649e-23;   // J/K (exact SI value)

// |cos| / |sin| tables of the slip geometry (crystal frame; the angles do not depend on the orientation),
// the scalar groups of the law, and the per-grain sample-frame d and t (72 words per grain).
template <typename T> void mr_setup(evp_handle *h, const evp_params *p, const double *quat, T *vec) {
    MRConst &c = h->mrc;
    double nn[12][3], dd[12][3], tt[12][3];
    for (int pl = 0; pl < 4; ++pl)
        for (int d = 0; d < 3; ++d)
            for (int q = 0; q < 3; ++q) {
                nn[3 * pl + d][q] = kN4[pl][q] / std::sqrt(3.0);
                dd[3 * pl + d][q] = kD4[pl][d][q] / std::sqrt(2.0);
            }
    for (int a = 0; a < 12; ++a) {
        tt[a][0] = nn[a][1] * dd[a][2] - nn[a][2] * dd[a][1];
        tt[a][1] = nn[a][2] * dd[a][0] - nn[a][0] * dd[a][2];
        tt[a][2] = nn[a][0] * dd[a][1] - nn[a][1] * dd[a][0];
    }
    for (int a = 0; a < 12; ++a)
        for (int b = 0; b < 12; ++b) {
            const double ct = std::fabs(nn[a][0] * tt[b][0] + nn[a][1] * tt[b][1] + nn[a][2] * tt[b][2]);
            const double cd = std::fabs(nn[a][0] * dd[b][0] + nn[a][1] * dd[b][1] + nn[a][2] * dd[b][2]);
            const double v4[4] = {ct, cd, std::sqrt(std::fmax(0.0, 1.0 - ct * ct)), std::sqrt(std::fmax(0.0, 1.0 - cd * cd))};
            for (int k = 0; k < 4; ++k) {
                c.tab[k * 144 + 12 * a + b] = v4[k];
                c.tabf[k * 144 + 12 * a + b] = (float)v4[k];
            }
        }
    const double kT = kBoltzmann * p->T, mu = voigt_mu(p), muPa = 1e6 * mu, b = p->b;
    MRScal<double> &d = c.d;
    d.tp_c = p->c1 * mu * b;
    d.tcut_c = 1e-6 * p->Q_slip / (p->c2 * p->c3 * b * b);
    d.rm_c = 2.0 * kT / (p->c1 * p->c2 * p->c3 * muPa * b * b * b);
    d.dd_c = std::sqrt(3.0) * mu * b / (16.0 * M_PI * (1.0 - p->poisson));
    d.climb_c = p->c7 * std::exp(-p->Q_bulk / kT) * 1e6 / kT;
    d.c4 = p->c4; d.c5 = p->c5; d.c6 = p->c6; d.c8 = p->c8;
    d.inv_b = 1.0 / b;
    d.dt = 1.0;
    d.soften = p->s_soften;
    // prefactor A = 2 k_B T nu_D sqrt(rho_P) exp(-Q_slip/k_B T) / (c1 c3 mu b^2) per unit tau_pass = tp_c sqrt(rho_P)
    h->mc.mr_ga = 2.0 * kT * p->nu_D * std::exp(-p->Q_slip / kT) / (p->c1 * p->c3 * muPa * b * b) / d.tp_c;
    for (int g = 0; g < h->G; ++g) {
        const double *q = quat + 4 * g;
        const double qn = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        const double w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
        const double R[3][3] = {{1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
                                {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
                                {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
        for (int a = 0; a < 12; ++a)
            for (int i = 0; i < 3; ++i) {
                vec[72 * (size_t)g + 3 * a + i] = (T)(R[i][0] * dd[a][0] + R[i][1] * dd[a][1] + R[i][2] * dd[a][2]);
                vec[72 * (size_t)g + 36 + 3 * a + i] = (T)(R[i][0] * tt[a][0] + R[i][1] * tt[a][1] + R[i][2] * tt[a][2]);
            }
    }
}
void mr_set_fp32(MRConst &c) {
    const MRScal<double> &d = c.d;
    c.f = MRScal<float>{(float)d.tp_c, (float)d.tcut_c, (float)d.rm_c, (float)d.dd_c, (float)d.climb_c, (float)d.c4,
                        (float)d.c5, (float)d.c6, (float)d.c8, (float)d.inv_b, (float)d.dt, (float)d.soften};
}

cudaError_t mr_refresh_k(evp_handle *h) {
    if (h->dbl)
        return mr_soften<double>(h->N3, 0, nullptr, nullptr, 0, (const double *)h->rho, (double *)h->gs, (double *)h->ge,
                                 (double *)h->gnd, h->k, h->mrc, h->st);
    return mr_soften<float>(h->N3, 0, nullptr, nullptr, 0, (const float *)h->rho, (float *)h->gs, (float *)h->ge,
                            (float *)h->gnd, h->k, h->mrc, h->st);
}
cudaError_t mr_soften_sel(evp_handle *h, int mode, int lo) {
    if (h->dbl)
        return mr_soften<double>(h->N3, mode, h->gprev, h->g, lo, (const double *)h->rho, (double *)h->gs,
                                 (double *)h->ge, (double *)h->gnd, h->k, h->mrc, h->st);
    return mr_soften<float>(h->N3, mode, h->gprev, h->g, lo, (const float *)h->rho, (float *)h->gs, (float *)h->ge,
                            (float *)h->gnd, h->k, h->mrc, h->st);
}
template <typename TA> MRPtr<TA> mr_ptr(const evp_handle *h) {
    return h->mr ? MRPtr<TA>{(const TA *)h->tpi} : MRPtr<TA>{nullptr};
}
// von Mises equivalent of a Mandel strain, sqrt(2/3 e:e) of its deviator (Eq. L0evolution's eps_vm)
double vm_strain(const double e[6]) {
    const double m = (e[0] + e[1] + e[2]) / 3.0;
    const double ee = (e[0] - m) * (e[0] - m) + (e[1] - m) * (e[1] - m) + (e[2] - m) * (e[2] - m) + e[3] * e[3] +
                      e[4] * e[4] + e[5] * e[5];
    return std::sqrt(ee / 1.5);
}

// Augmented-Lagrangian iterations of one increment (after the predictor): see k_al_local.
// Returns a status; fills the iteration count, residuals, mean stress and the macro strain increment.
static_assert(sizeof(FpCtl) <= 256, "FpCtl must fit its workspace slot");
constexpr int kFpBatch = 16;   // iterations queued between host reads of the control block
constexpr int kTwoStepIters = 40;   // iterations of an increment whose first local-solve pass takes two chord steps
const double kZero6[6] = {0, 0, 0, 0, 0, 0};

// The x and y passes of the fixed point's transforms, forward and inverse: one launch each where the (field, z)
// plane fits shared memory (timed as classes 1 and 5), else the two passes (classes 1, 2 and 4, 5).
int xy_launches(const evp_handle *h) { return fft_xy_fused(h->n, h->dbl) ? 1 : 2; }
template <typename T> cudaError_t fwd_xy(evp_handle *h, const T *in, const int *skip = nullptr) {
    if (fft_xy_fused(h->n, h->dbl)) {
        PROF(1, 1);
        return fft_xy_r2c<T>(in, h->spec, h->n, 6, h->st, skip);
    }
    {
        PROF(1, 1);
        const cudaError_t e = fft_x_r2c<T>(in, h->spec, h->n, 6, h->st, skip);
        if (e != cudaSuccess) return e;
    }
    PROF(2, 1);
    return fft_y<T>(h->spec, h->n, 6, 0, h->st, skip);
}
template <typename T>
cudaError_t inv_xy(evp_handle *h, T *out, T scale, const double *add6, const T *base, const int *skip = nullptr) {
    if (fft_xy_fused(h->n, h->dbl)) {
        PROF(5, 1);
        return fft_xy_c2r<T>(h->spec, out, h->n, 6, scale, add6, h->st, base, skip);
    }
    {
        PROF(4, 1);
        const cudaError_t e = fft_y<T>(h->spec, h->n, 6, 1, h->st, skip);
        if (e != cudaSuccess) return e;
    }
    PROF(5, 1);
    return fft_x_c2r<T>(h->spec, out, h->n, 6, scale, add6, h->st, base, skip);
}

template <typename TA>
int al_loop(evp_handle *h, MatConst mc, double *dE, int *it_out, int *conv_out, int *nmax_out, double *err_eq,
            double *err_bc, double *mean_sig) {
    const long N3 = h->N3;
    const int n = h->n;
    const double muV = h->mc.mu0, lamV = h->mc.lam0;
    const double mu0 = muV / h->cfg.al_scale, lam0 = (lamV + 2.0 * muV / 3.0) - 2.0 * mu0 / 3.0;
    const double a = lam0 + 2.0 * mu0, b = lam0, det = a * a - b * b;
    const int solve64 = h->prec != EVP_MIXED_FAST;
    const int nb = al_grid(N3, h->nsm, (int)sizeof(TA));
    double hs[14];
    int32_t hf[2];
    int nmax = 0, conv = 0, it;
    double ecmp = 0, elam = 0, ebc = 0;
    void *fac = h->cfg.newton_mode == EVP_NEWTON_REUSE ? h->fac : nullptr;
    // local tolerance: newton_tol, or with newton_adapt = eta > 0 loosened to max(newton_tol, eta err) while the
    // iteration is far from converged (err = the larger of the compatibility and multiplier residuals of the
    // previous iteration, 1e-2 before the first), as in the basic scheme
    const double ntol = h->cfg.newton_tol, eta = h->cfg.newton_adapt;
    double tol_loc = eta > 0.0 ? std::fmax(ntol, eta * 1e-2) : ntol;
    auto local = [&](int init, int refresh) -> int {
        { PROF(0, 1);
          CK(al_local<TA>(N3, (const TA *)h->epst, (const TA *)h->epse, (const TA *)h->tauc, h->g0, (TA *)h->sigk,
                          (TA *)h->lam, (TA *)h->pal, (const TA *)h->Stab, (const TA *)h->Sal, (const TA *)h->Mtab, mc,
                          lam0, mu0, tol_loc, h->cfg.newton_max, solve64, init, h->flags, h->partials, fac,
                          refresh, h->st, h->nsm, mr_ptr<TA>(h))); }
        { PROF(6, 1); CK(reduce_partials(h->partials, nb, 14, h->scal + 24, h->st)); }
        CK(cudaMemcpyAsync(hs, h->scal + 24, sizeof hs, cudaMemcpyDeviceToHost, h->st));
        CK(cudaMemcpyAsync(hf, h->flags, sizeof hf, cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        if (h->prof) prof_collect(h);
        nmax = hf[1] > nmax ? hf[1] : nmax;
        if (hf[0] != 0) return fail(h, EVP_ERR_NEWTON, "local Newton failed in %d voxels", hf[0]);
        return EVP_OK;
    };
    int rc = local(1, 1);
    if (rc) { *it_out = 0; *nmax_out = nmax; return rc; }
    for (it = 1; it <= h->cfg.max_iter; ++it) {
        // macroscopic strain on the stress-controlled components from <lam>
        const double m0 = hs[2] / (double)N3, m1 = hs[3] / (double)N3;
        double dEk[6] = {0, 0, 0, 0, 0, 0};
        dEk[0] = (a * (-m0) - b * (-m1)) / det;
        dEk[1] = (-b * (-m0) + a * (-m1)) / det;
        for (int i = 3; i < 6; ++i) dEk[i] = -(hs[2 + i] / (double)N3) / (2.0 * mu0);
        for (int i = 0; i < 6; ++i) dE[i] += dEk[i];
        // compatibility: eps_tr = eps_e^t + dE + Gamma0 * (C0 de - lam)
        CK(fwd_xy<TA>(h, (const TA *)h->pal));
        { PROF(3, 1); CK(fft_z<TA>(h->spec, n, 6, Z_FWD_GAMMA_INV, lam0, mu0, nullptr, nullptr, h->st)); }
        CK(inv_xy<TA>(h, (TA *)h->epst, (TA)(1.0 / (double)N3), dE, (const TA *)h->epse));
        rc = local(0, it == 1);
        if (rc) break;
        double En = 0.0, mn = 0.0, mu_n = 0.0;
        for (int i = 0; i < 6; ++i) {
            const double Ei = h->E[i] + dE[i], mi = hs[2 + i] / (double)N3;
            En += Ei * Ei;
            mn += mi * mi;
            if (i != 2) mu_n += mi * mi;
        }
        const double den = std::fmax(std::sqrt(mn), h->p.tau0);
        ecmp = std::sqrt(hs[0] / (double)N3) / std::fmax(std::sqrt(En), 1e-6);
        elam = std::sqrt(hs[1] / (double)N3) / den;
        ebc = std::sqrt(mu_n) / den;
        if (!std::isfinite(ecmp) || !std::isfinite(elam)) { rc = fail(h, EVP_ERR_NONFINITE, "non-finite AL residual"); break; }
        if (ecmp <= h->cfg.tol && elam <= h->cfg.tol && ebc <= h->cfg.tol && tol_loc <= ntol) { conv = 1; break; }
        if (eta > 0.0) tol_loc = std::fmax(ntol, eta * std::fmax(ecmp, elam));
    }
    if (it > h->cfg.max_iter) it = h->cfg.max_iter;
    *it_out = it;
    *conv_out = conv;
    *nmax_out = nmax;
    *err_eq = elam;
    *err_bc = ebc;
    for (int i = 0; i < 6; ++i) mean_sig[i] = hs[8 + i] / (double)N3;
    return rc;
}
}  // namespace

extern "C" {

int evp_workspace_bytes(const evp_config *cfg, size_t *bytes) {
    char why[256];
    const int rc = check_cfg(cfg, why, sizeof why);
    if (rc) return rc;
    if (!bytes) return EVP_ERR_ARG;
    *bytes = layout(cfg, nullptr, nullptr);
    return EVP_OK;
}

const char *evp_last_error(const evp_handle *h) { return h ? h->err : "no handle"; }

void evp_destroy(evp_handle *h) { delete h; }

int evp_init(evp_handle **out, const evp_config *cfg, const evp_params *p, const int32_t *grain_id, const double *quat,
             uint64_t seed, void *workspace, size_t workspace_bytes, void *cuda_stream) {
    if (!out) return EVP_ERR_ARG;
    *out = nullptr;
    evp_handle *h = new (std::nothrow) evp_handle();
    if (!h) return EVP_ERR_OOM;
    *out = h;
    const int rc = check_cfg(cfg, h->err, sizeof h->err);
    if (rc) return rc;
    if (!p || !grain_id || !quat || !workspace) return fail(h, EVP_ERR_ARG, "NULL argument to evp_init");
    if (((uintptr_t)workspace & 255) != 0) return fail(h, EVP_ERR_ARG, "workspace must be 256-byte aligned");
    h->cfg = *cfg;
    h->p = *p;
    h->n = cfg->n;
    h->G = cfg->grains;
    h->K = cfg->kmax;
    h->prec = cfg->precision;
    h->N3 = (long)h->n * h->n * h->n;
    h->H = (long)h->n * h->n * (h->n / 2 + 1);
    h->dbl = h->prec == EVP_FP64;
    h->tsz = h->dbl ? 8 : 4;
    h->st = (cudaStream_t)cuda_stream;
    const size_t need = layout(cfg, nullptr, nullptr);
    if (workspace_bytes < need)
        return fail(h, EVP_ERR_OOM, "workspace has %zu bytes, needs %zu", workspace_bytes, need);
    h->ws = (char *)workspace;
    h->ws_bytes = workspace_bytes;
    layout(cfg, h, h->ws);
    for (long v = 0; v < h->N3; ++v)
        if (grain_id[v] < 0 || grain_id[v] >= h->G)
            return fail(h, EVP_ERR_ARG, "grain_id[%ld]=%d outside [0,%d)", v, grain_id[v], h->G);
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || h->nsm < 1)
            return fail(h, EVP_ERR_CUDA, "cannot query the device");
    }
    h->seed = seed;
    h->next_id = h->G;
    h->have_prev = 0;
    for (int i = 0; i < 6; ++i) h->E[i] = h->dE_prev[i] = 0.0;
    const double mu = voigt_mu(p), lam = voigt_lam(p);
    h->mc.gdot0 = p->gdot0;
    h->mc.n = p->n;
    h->mc.dt = 1.0;
    h->mc.tau0 = p->tau0;
    h->mc.alpha_mu_b = p->alpha * mu * p->b;
    h->mc.k1 = p->k1;
    h->mc.k2 = p->k2;
    h->mc.lam0 = lam;
    h->mc.mu0 = mu;
    h->mc.n_int = (p->n >= 1.0 && p->n <= 64.0 && p->n == std::floor(p->n)) ? (int)p->n : 0;
    h->mc.set_fp32();
    h->pc.m = 6.0 / p->l_gb;
    h->pc.kappa = 0.75 * p->l_gb;
    h->pc.gam = 1.5;
    h->pc.L_dt = p->L_dt;
    h->pc.Escale = p->zeta * (mu * 1e6) * p->b * p->b * (p->dx / h->r) / p->omega_gb;   // lengths in PF spacings
    h->pc.drop = p->eta_drop;
    h->pc.G = h->G;
    h->pc.K = h->K;
    h->pc.set_fp32();
    h->leff = p->dx;   // Eq. L0evolution starts from the grid size l0
    if (h->mr) {
        const size_t vb = 72 * (size_t)h->G * h->tsz;
        void *hv = std::malloc(vb);
        if (!hv) return fail(h, EVP_ERR_OOM, "host allocation");
        if (h->dbl) mr_setup<double>(h, p, quat, (double *)hv);
        else mr_setup<float>(h, p, quat, (float *)hv);
        mr_set_fp32(h->mrc);
        h->mc.set_fp32();
        cudaError_t ea = cudaMemcpyAsync(h->vec, hv, vb, cudaMemcpyHostToDevice, h->st);
        cudaError_t eb = cudaStreamSynchronize(h->st);
        std::free(hv);
        CK(ea);
        CK(eb);
    }
    // tables
    {
        const size_t G = (size_t)h->G;
        void *hS = std::malloc(36 * G * h->tsz), *hM = std::malloc(72 * G * h->tsz);
        if (!hS || !hM) { std::free(hS); std::free(hM); return fail(h, EVP_ERR_OOM, "host allocation"); }
        if (h->dbl) build_tables<double>(p, h->G, quat, (double *)hS, (double *)hM);
        else build_tables<float>(p, h->G, quat, (float *)hS, (float *)hM);
        if (cfg->scheme == EVP_SCHEME_AL) {
            // S + S0 with S0 the compliance of the AL reference medium (Voigt bulk, shear mu/al_scale)
            void *hA = std::malloc(36 * G * h->tsz);
            if (!hA) { std::free(hS); std::free(hM); return fail(h, EVP_ERR_OOM, "host allocation"); }
            const double mu0 = mu / cfg->al_scale, lam0 = (lam + 2.0 * mu / 3.0) - 2.0 * mu0 / 3.0;
            const double sa = 1.0 / (2.0 * mu0), sb = lam0 / (2.0 * mu0 * (3.0 * lam0 + 2.0 * mu0));
            for (size_t gg = 0; gg < G; ++gg)
                for (int i = 0; i < 6; ++i)
                    for (int j = 0; j < 6; ++j) {
                        const double s0 = (i == j ? sa : 0.0) - (i < 3 && j < 3 ? sb : 0.0);
                        if (h->dbl) ((double *)hA)[36 * gg + 6 * i + j] = ((double *)hS)[36 * gg + 6 * i + j] + s0;
                        else ((float *)hA)[36 * gg + 6 * i + j] = (float)((double)((float *)hS)[36 * gg + 6 * i + j] + s0);
                    }
            cudaError_t ea = cudaMemcpyAsync(h->Sal, hA, 36 * G * h->tsz, cudaMemcpyHostToDevice, h->st);
            cudaError_t eb = cudaStreamSynchronize(h->st);
            std::free(hA);
            CK(ea);
            CK(eb);
        }
        if (cfg->newton_mode == EVP_NEWTON_F32_TANGENT) {
            float *fS = (float *)std::malloc(36 * G * 4), *fM = (float *)std::malloc(72 * G * 4);
            if (!fS || !fM) { std::free(fS); std::free(fM); std::free(hS); std::free(hM); return fail(h, EVP_ERR_OOM, "host allocation"); }
            for (size_t i = 0; i < 36 * G; ++i) fS[i] = (float)((double *)hS)[i];
            for (size_t i = 0; i < 72 * G; ++i) fM[i] = (float)((double *)hM)[i];
            cudaError_t ea = cudaMemcpyAsync(h->Stabf, fS, 36 * G * 4, cudaMemcpyHostToDevice, h->st);
            cudaError_t eb = cudaMemcpyAsync(h->Mtabf, fM, 72 * G * 4, cudaMemcpyHostToDevice, h->st);
            cudaError_t ec = cudaStreamSynchronize(h->st);
            std::free(fS);
            std::free(fM);
            CK(ea);
            CK(eb);
            CK(ec);
        }
        cudaError_t e1 = cudaMemcpyAsync(h->Stab, hS, 36 * G * h->tsz, cudaMemcpyHostToDevice, h->st);
        cudaError_t e2 = cudaMemcpyAsync(h->Mtab, hM, 72 * G * h->tsz, cudaMemcpyHostToDevice, h->st);
        cudaError_t e3 = cudaStreamSynchronize(h->st);
        std::free(hS);
        std::free(hM);
        CK(e1);
        CK(e2);
        CK(e3);
    }
    CK(cudaMemcpyAsync(h->g0, grain_id, sizeof(int32_t) * h->N3, cudaMemcpyHostToDevice, h->st));
    const size_t fb = 6 * (size_t)h->N3 * h->tsz;
    CK(cudaMemsetAsync(h->sig, 0, fb, h->st));
    CK(cudaMemsetAsync(h->epse, 0, fb, h->st));
    CK(cudaMemsetAsync(h->epsp, 0, fb, h->st));
    CK(cudaMemsetAsync(h->deps, 0, fb, h->st));
    if (h->dbl)
        CK(drx_init<double>(h->N3, h->g0, (double *)h->rho, h->k, h->kappa, h->g, h->draws, nullptr, nullptr, h->K,
                            p->rho0, p->kc, p->q, seed, h->st));
    else
        CK(drx_init<float>(h->N3, h->g0, (float *)h->rho, h->k, h->kappa, h->g, h->draws, nullptr, nullptr, h->K,
                           p->rho0, p->kc, p->q, seed, h->st));
    if (h->mr) {   // rho = rho_SSD(0); no GND yet; k = sum of mobile, SSD and GND densities
        CK(cudaMemsetAsync(h->gs, 0, 36 * (size_t)h->N3 * h->tsz, h->st));
        CK(mr_refresh_k(h));
    }
    CK(pf_init(h->n, h->r, h->K, h->g0, h->ids, h->eta, h->ids2, h->eta2, h->dbl, h->gpf, h->st));
    if (h->rmax_bytes) {   // one entry per point in (ids, eta), none in (ids2, eta2)
        CK(cudaMemsetAsync(h->rmax, 1, h->rmax_bytes, h->st));
        CK(cudaMemsetAsync(h->rmax2, 0, h->rmax_bytes, h->st));
    }
    if (h->r == 2) CK(pf_interp(h->n, h->k, h->kpf, h->st));
    CK(cudaStreamSynchronize(h->st));
    return EVP_OK;
}

int evp_set_profiling(evp_handle *h, int on) {
    if (!h) return EVP_ERR_ARG;
    h->prof = on ? (1u << EVP_NCLASS) - 1u : 0u;
    return EVP_OK;
}

int evp_set_profiling_mask(evp_handle *h, uint32_t mask) {
    if (!h) return EVP_ERR_ARG;
    h->prof = mask & ((1u << EVP_NCLASS) - 1u);
    return EVP_OK;
}

int evp_kernel_times(evp_handle *h, double *ms, int64_t *launches, int reset) {
    if (!h) return EVP_ERR_ARG;
    CK(cudaStreamSynchronize(h->st));
    prof_collect(h);
    for (int i = 0; i < EVP_NCLASS; ++i) {
        if (ms) ms[i] = h->prof_ms[i];
        if (launches) launches[i] = h->prof_n[i];
        if (reset) { h->prof_ms[i] = 0.0; h->prof_n[i] = 0; }
    }
    return EVP_OK;
}

int evp_launch_count(const evp_handle *h, int64_t *launches) {
    if (!h || !launches) return EVP_ERR_ARG;
    *launches = h->launches;
    return EVP_OK;
}

int evp_newton_refreshes(const evp_handle *h, int64_t *refreshes) {
    if (!h || !refreshes) return EVP_ERR_ARG;
    *refreshes = h->newton_refreshes;
    return EVP_OK;
}

int evp_newton_counts(const evp_handle *h, int64_t *solves, int64_t *evals) {
    if (!h) return EVP_ERR_ARG;
    if (solves) *solves = h->newton_solves;
    if (evals) *evals = h->newton_evals;
    return EVP_OK;
}

int evp_set_solver(evp_handle *h, double tol, int max_iter, int allow_unconverged) {
    if (!h || max_iter < 1 || !(tol >= 0.0)) return fail(h, EVP_ERR_ARG, "bad solver controls");
    h->cfg.tol = tol;
    h->cfg.max_iter = max_iter;
    h->cfg.allow_unconverged = allow_unconverged;
    return EVP_OK;
}

int evp_increment(evp_handle *h, double dE33, double dt, evp_stats *out) {
    if (!h) return EVP_ERR_ARG;
    if (!(dt > 0.0) || !std::isfinite(dE33)) return fail(h, EVP_ERR_ARG, "dt must be > 0 and dE33 finite");
    const long N3 = h->N3;
    const int n = h->n;
    MatConst mc = h->mc;
    mc.dt = dt;
    mc.set_fp32();
    const double lam0 = mc.lam0, mu0 = mc.mu0;
    // predictor
    double dE[6];
    int use_field = 0;
    double r = 0.0;
    if (h->cfg.predictor && h->have_prev && h->dE_prev[2] != 0.0) {
        r = dE33 / h->dE_prev[2];
        for (int i = 0; i < 6; ++i) dE[i] = r * h->dE_prev[i];
        dE[2] = dE33;
        use_field = 1;
    } else {
        const double nu0 = lam0 / (2.0 * (lam0 + mu0));
        const double g[6] = {-nu0 * dE33, -nu0 * dE33, dE33, 0, 0, 0};
        for (int i = 0; i < 6; ++i) dE[i] = g[i];
    }
    const size_t fb = 6 * (size_t)N3 * h->tsz;
    CK(cudaMemcpyAsync(h->sigk, h->sig, fb, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemsetAsync(h->flags, 0, sizeof(int32_t) * 16, h->st));
    {
        PROF(7, 1);
        if (h->dbl)
            CK(predictor<double>(N3, (double *)h->epse, (double *)h->deps, (double *)h->rho, (double *)h->epst,
                                 (double *)h->tauc, mc, r, dE, use_field, h->st));
        else
            CK(predictor<float>(N3, (float *)h->epse, (float *)h->deps, (float *)h->rho, (float *)h->epst,
                                (float *)h->tauc, mc, r, dE, use_field, h->st));
    }
    if (h->mr) {   // frozen Ma-Roters hardening of the increment; tauc becomes the stopping scale
        PROF(7, 1);
        if (h->dbl)
            CK(mr_harden<double>(N3, (const double *)h->rho, (const double *)h->gs, (const double *)h->ge,
                                 (double *)h->tpi, (double *)h->tauc, h->mrc, h->st));
        else
            CK(mr_harden<float>(N3, (const float *)h->rho, (const float *)h->gs, (const float *)h->ge, (float *)h->tpi,
                                (float *)h->tauc, h->mrc, h->st));
    }
    // reference medium of the basic scheme (Green operator, mixed-BC correction): Voigt, or the shear modulus
    // mu_Voigt / ref_scale with the Voigt bulk modulus (the predictor above keeps the Voigt medium)
    const double rs = h->cfg.ref_scale > 0.0 ? h->cfg.ref_scale : 1.0;
    const double mu0r = rs == 1.0 ? mu0 : mu0 / rs;
    const double lam0r = rs == 1.0 ? lam0 : lam0 + 2.0 * mu0 / 3.0 - 2.0 * mu0r / 3.0;
    // mixed-BC correction: (C0_uu)^-1 on u = {11, 22, 23, 13, 12}
    const double a = lam0r + 2.0 * mu0r, b = lam0r, det = a * a - b * b;
    const int solve64 = h->prec != EVP_MIXED_FAST;
    const double ntol = h->cfg.newton_tol;
    int status = EVP_OK, it = 0, conv = 0, nmax = 0;
    double err_eq = 0, err_bc = 0, mean[6] = {0, 0, 0, 0, 0, 0};
    const int zb = fft_z_blocks(n, h->dbl);
    double hs[8];
    int64_t hcount[3] = {0, 0, 0};
    const int reuse = h->cfg.newton_mode == EVP_NEWTON_REUSE;
    // refactor every voxel's tangent at the first iteration unless valid factors are stored; always while
    // an adjoint is recorded or swept, so that a recomputed increment repeats the recorded one exactly
    const bool fresh = !h->fac_valid || h->adj != nullptr;
    if (h->cfg.scheme == EVP_SCHEME_AL) {
        status = h->dbl ? al_loop<double>(h, mc, dE, &it, &conv, &nmax, &err_eq, &err_bc, mean)
                        : al_loop<float>(h, mc, dE, &it, &conv, &nmax, &err_eq, &err_bc, mean);
        it = it < 1 ? 1 : it;
    } else {
        // iterations are queued in batches; the device control (the z pass's last CTA, fpctl.cuh) decides when to stop
        FpCtl hc{};
        for (int i = 0; i < 6; ++i) hc.dE[i] = dE[i];
        const bool adapt = h->cfg.newton_adapt > 0.0;
        hc.tol_loc = adapt ? std::fmax(ntol, h->cfg.newton_adapt * 1e-2) : ntol;   // before the first residual
        hc.tol_loc_f = (float)hc.tol_loc;
        FpCtl *dc = (FpCtl *)h->ctl;
        const int *skip = &dc->done;
        const double *tl64 = adapt ? &dc->tol_loc : nullptr;
        const float *tl32 = adapt ? &dc->tol_loc_f : nullptr;
        CK(cudaMemcpyAsync(dc, &hc, sizeof hc, cudaMemcpyHostToDevice, h->st));
        const double inv = 1.0 / (double)N3;
        ZCtl zc;   // the z pass's last block runs the control (see fpctl.cuh)
        zc.ctl = dc;
        zc.flags = h->flags;
        zc.scal = h->scal;
        zc.p.N3 = (double)N3; zc.p.tau0 = h->p.tau0; zc.p.tol = h->cfg.tol; zc.p.a = a; zc.p.b = b; zc.p.det = det;
        zc.p.mu0 = mu0r; zc.p.ntol = ntol; zc.p.eta = h->cfg.newton_adapt; zc.p.max_iter = h->cfg.max_iter;
        int queued = 0;
        while (true) {
            const int nb = std::min(kFpBatch, h->cfg.max_iter - queued);
            for (int q = 0; q < nb; ++q) {
                const int first = queued + q == 0 && fresh;
                // the first pass takes two chord steps in the early iterations of an increment, where many voxels
                // need them; later a single step keeps it at one more CTA per SM
                const int two = queued + q < kTwoStepIters;
                if (h->dbl) {
                  { PROF(0, 1);
                    if (h->cfg.newton_mode == EVP_NEWTON_F32_TANGENT)
                        CK(newton_field_df(N3, (double *)h->epst, (double *)h->tauc, h->g0, (double *)h->sigk,
                                           (double *)h->Stab, (double *)h->Mtab, h->Stabf, h->Mtabf, mc, ntol,
                                           h->cfg.newton_max, h->flags, h->st, skip, tl64));
                    else if (reuse)
                        CK(newton_chord_field<double>(N3, (double *)h->epst, (double *)h->tauc, h->g0, (double *)h->sigk,
                                                      (double *)h->Stab, (double *)h->Mtab, h->fac, mc, ntol,
                                                      h->cfg.newton_max, 1, first, h->flags, h->wlist, h->nsm, h->st,
                                                      skip, tl64, mr_ptr<double>(h), two));
                    else
                        CK(newton_field<double>(N3, (double *)h->epst, (double *)h->tauc, h->g0, (double *)h->sigk,
                                                (double *)h->Stab, (double *)h->Mtab, mc, ntol, h->cfg.newton_max, 1,
                                                h->flags, h->st, skip, tl64, mr_ptr<double>(h))); }
                  CK(fwd_xy<double>(h, (const double *)h->sigk, skip));
                  { PROF(3, 1);
                    CK(fft_z<double>(h->spec, n, 6, Z_FWD_GAMMA_INV, lam0r, mu0r, h->partials, h->scal, h->st, skip,
                                     &zc)); }
                } else {
                  { PROF(0, 1);
                    if (reuse)
                        CK(newton_chord_field<float>(N3, (float *)h->epst, (float *)h->tauc, h->g0, (float *)h->sigk,
                                                     (float *)h->Stab, (float *)h->Mtab, h->fac, mc, ntol,
                                                     h->cfg.newton_max, solve64, first, h->flags, h->wlist, h->nsm,
                                                     h->st, skip, tl32, mr_ptr<float>(h), two));
                    else
                        CK(newton_field<float>(N3, (float *)h->epst, (float *)h->tauc, h->g0, (float *)h->sigk,
                                               (float *)h->Stab, (float *)h->Mtab, mc, ntol, h->cfg.newton_max, solve64,
                                               h->flags, h->st, skip, tl32, mr_ptr<float>(h))); }
                  CK(fwd_xy<float>(h, (const float *)h->sigk, skip));
                  { PROF(3, 1);
                    CK(fft_z<float>(h->spec, n, 6, Z_FWD_GAMMA_INV, lam0r, mu0r, h->partials, h->scal, h->st, skip,
                                    &zc)); }
                }
                // the strain correction arrives through the zero-frequency term: no offsets here
                if (h->dbl) {
                    CK(inv_xy<double>(h, (double *)h->epst, inv, kZero6, nullptr, skip));
                } else {
                    CK(inv_xy<float>(h, (float *)h->epst, (float)inv, kZero6, nullptr, skip));
                }
            }
            queued += nb;
            CK(cudaMemcpyAsync(&hc, dc, sizeof hc, cudaMemcpyDeviceToHost, h->st));
            CK(cudaMemcpyAsync(hs, h->scal, sizeof(double) * 7, cudaMemcpyDeviceToHost, h->st));
            CK(cudaStreamSynchronize(h->st));
            if (h->prof) prof_collect(h);
            if (hc.done || queued >= h->cfg.max_iter) break;
        }
        it = hc.it;
        conv = hc.conv;
        nmax = hc.nmax;
        err_eq = hc.err_eq;
        err_bc = hc.err_bc;
        for (int i = 0; i < 6; ++i) {
            dE[i] = hc.dE[i];
            mean[i] = hs[i];
        }
        if (hc.status == EVP_ERR_NEWTON)
            status = fail(h, EVP_ERR_NEWTON, "local Newton failed in %d voxels at iteration %d", hc.nfail, it);
        else if (hc.status == EVP_ERR_NONFINITE)
            status = fail(h, EVP_ERR_NONFINITE, "non-finite residual at iteration %d", it);
    }
    if (it > h->cfg.max_iter) it = h->cfg.max_iter;
    // after a first increment without a local failure every voxel holds factors of an SPD tangent; later
    // increments start from them (stale factors only cost chord steps: a step that does not contract
    // refreshes them)
    if (reuse && h->cfg.scheme == EVP_SCHEME_BASIC) h->fac_valid = status == EVP_OK ? 1 : 0;
    CK(cudaMemcpyAsync(hcount, h->flags + 4, sizeof hcount, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    h->newton_solves += hcount[0];
    h->newton_evals += hcount[1];
    h->newton_refreshes += reuse ? hcount[2] : hcount[0];
    if (status == EVP_OK && !conv) {
        if (h->cfg.allow_unconverged) status = EVP_WARN_UNCONVERGED;
        else status = fail(h, EVP_ERR_FIXEDPOINT, "fixed point not converged in %d iterations (err_eq %.3e, err_bc %.3e)",
                           it, err_eq, err_bc);
    }
    if (out) {
        out->iterations = it;
        out->newton_max_iters = nmax;
        out->status = status;
        out->err_eq = err_eq;
        out->err_bc = err_bc;
        for (int i = 0; i < 6; ++i) {
            out->sig_mean[i] = mean[i];
            out->E[i] = h->E[i] + dE[i];
        }
    }
    if (status < 0) return status;
    if (h->mr) {
        PROF(8, 3);
        MRConst &c = h->mrc;
        c.d.dt = dt;
        c.f.dt = (float)dt;
        if (h->dbl) {
            CK(mr_rates<double>(N3, (const double *)h->sigk, (const double *)h->tpi, h->g0,
                                (const double *)h->Mtab, (const double *)h->epst, (double *)h->epse, (double *)h->epsp,
                                (double *)h->deps, (double *)h->gdm, (double *)h->aux, mc, h->st));
            CK(mr_update<double>(n, h->g, h->g0, (const double *)h->gdm, (const double *)h->aux, (const double *)h->sigk,
                                 (const double *)h->Mtab, (const double *)h->vec, (double *)h->rho, (double *)h->gs,
                                 (double *)h->ge, (double *)h->gnd, h->k, c, h->leff, h->st));
        } else {
            CK(mr_rates<float>(N3, (const float *)h->sigk, (const float *)h->tpi, h->g0,
                               (const float *)h->Mtab, (const float *)h->epst, (float *)h->epse, (float *)h->epsp,
                               (float *)h->deps, (float *)h->gdm, (float *)h->aux, mc, h->st));
            CK(mr_update<float>(n, h->g, h->g0, (const float *)h->gdm, (const float *)h->aux, (const float *)h->sigk,
                                (const float *)h->Mtab, (const float *)h->vec, (float *)h->rho, (float *)h->gs,
                                (float *)h->ge, (float *)h->gnd, h->k, c, h->leff, h->st));
        }
    } else {
    PROF(8, 1);
    if (h->dbl)
        CK(state_update<double>(N3, (double *)h->sigk, (double *)h->tauc, h->g0, (double *)h->Mtab, (double *)h->epst,
                                (double *)h->epse, (double *)h->epsp, (double *)h->deps, (double *)h->rho, h->k, mc,
                                h->st));
    else
        CK(state_update<float>(N3, (float *)h->sigk, (float *)h->tauc, h->g0, (float *)h->Mtab, (float *)h->epst,
                               (float *)h->epse, (float *)h->epsp, (float *)h->deps, (float *)h->rho, h->k, mc, h->st));
    }
    void *t = h->sig;
    h->sig = h->sigk;
    h->sigk = t;
    for (int i = 0; i < 6; ++i) {
        h->E[i] += dE[i];
        h->dE_prev[i] = dE[i];
    }
    // Eq. L0evolution after the increment's GND rates, with the von Mises strain of the macroscopic strain
    if (h->mr) h->leff *= 1.0 + vm_strain(h->E) / h->p.xi;
    h->have_prev = 1;
    CK(cudaStreamSynchronize(h->st));
    if (h->prof) prof_collect(h);
    return status;
}

int drx_nucleate(evp_handle *h, uint64_t step, int32_t *n_new) {
    (void)step;
    if (!h || !n_new) return fail(h, EVP_ERR_ARG, "NULL argument to drx_nucleate");
    const double kc_new = h->p.s_nucl * h->p.kc;
    { PROF(9, h->mr ? 4 : 3);
    // the power law softens its single density family in the nucleation kernel; the Ma-Roters law softens the
    // GND densities of the fresh nuclei (ids >= next_id) afterwards and keeps rho_SSD (Eq. UpdateGND)
    if (h->dbl)
        CK(nucleate<double>(h->n, h->r, h->K, h->g, h->k, h->kappa, h->mr ? nullptr : (double *)h->rho, h->draws,
                            h->ids, (double *)h->eta, h->gpf, h->blk_counts, h->blk_off, h->count, h->next_id,
                            h->p.s_soften, kc_new, h->p.q, h->seed, h->st));
    else
        CK(nucleate<float>(h->n, h->r, h->K, h->g, h->k, h->kappa, h->mr ? nullptr : (float *)h->rho, h->draws,
                           h->ids, (float *)h->eta, h->gpf, h->blk_counts, h->blk_off, h->count, h->next_id,
                           h->p.s_soften, kc_new, h->p.q, h->seed, h->st));
    if (h->mr) CK(mr_soften_sel(h, 1, h->next_id));
    }
    int32_t c = 0;
    CK(cudaMemcpyAsync(&c, h->count, sizeof c, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (h->prof) prof_collect(h);
    *n_new = c;
    if ((long)h->next_id + c > (long)h->max_ids)
        return fail(h, EVP_ERR_OOM, "grain-id space of %d exhausted", h->max_ids);
    h->next_id += c;
    return EVP_OK;
}

int pf_step(evp_handle *h, int nsteps, pf_stats *out) {
    if (!h || nsteps < 0) return fail(h, EVP_ERR_ARG, "bad pf_step arguments");
    const long N3 = h->N3;
    CK(cudaMemcpyAsync(h->gprev, h->g, sizeof(int32_t) * N3, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemsetAsync(h->flags + 2, 0, sizeof(int32_t), h->st));
    if (h->r == 2) { PROF(10, 1); CK(pf_interp(h->n, h->k, h->kpf, h->st)); }   // driving force on the PF grid
    for (int s = 0; s < nsteps; ++s) {
        PROF(10, 1);
        if (h->dbl)
            CK(pf_one_step<double>(h->npf, h->ids, (double *)h->eta, h->ids2, (double *)h->eta2, h->gpf, h->kpf,
                                   h->pc, h->flags + 2, h->rmax, h->rmax2, h->st));
        else
            CK(pf_one_step<float>(h->npf, h->ids, (float *)h->eta, h->ids2, (float *)h->eta2, h->gpf, h->kpf, h->pc,
                                  h->flags + 2, h->rmax, h->rmax2, h->st));
        int32_t *ti = h->ids; h->ids = h->ids2; h->ids2 = ti;
        void *te = h->eta; h->eta = h->eta2; h->eta2 = te;
        uint8_t *tr = h->rmax; h->rmax = h->rmax2; h->rmax2 = tr;
    }
    if (h->r == 2 && nsteps > 0) {   // grain ids of the mechanics grid from the PF children
        PROF(11, 1);
        if (h->dbl) CK(pf_restrict<double>(h->n, h->K, h->ids, (const double *)h->eta, h->g, h->st));
        else CK(pf_restrict<float>(h->n, h->K, h->ids, (const float *)h->eta, h->g, h->st));
    }
    { PROF(11, 1);
    if (h->mr) CK(mr_soften_sel(h, 2, h->G));
    else if (h->dbl) CK(pf_soften<double>(N3, h->gprev, h->g, (double *)h->rho, h->k, h->G, h->p.s_soften, h->st));
    else CK(pf_soften<float>(N3, h->gprev, h->g, (float *)h->rho, h->k, h->G, h->p.s_soften, h->st));
    }
    if (h->r == 2) { PROF(11, 1); CK(pf_interp(h->n, h->k, h->kpf, h->st)); }   // softened densities
    int32_t ovf = 0;
    if (out) {
        const int nb = pf_stat_blocks(h->N3pf);
        // every id in use is below next_id: only those words of the id bitmap are cleared and counted
        const int words = std::min(h->bitmap_words, (h->next_id + 31) / 32);
        { PROF(12, 3);
        if (h->dbl)
            CK(pf_stats_launch<double>(h->npf, h->ids, (double *)h->eta, h->gpf, h->kpf, h->pc, h->bitmap, words,
                                       h->partials, h->st));
        else
            CK(pf_stats_launch<float>(h->npf, h->ids, (float *)h->eta, h->gpf, h->kpf, h->pc, h->bitmap, words,
                                      h->partials, h->st));
        CK(reduce_partials(h->partials, nb, 2, h->scal + 8, h->st));
        }
        double hs[2], ng = 0;
        CK(cudaMemcpyAsync(hs, h->scal + 8, sizeof hs, cudaMemcpyDeviceToHost, h->st));
        CK(cudaMemcpyAsync(&ng, h->partials + 2 * (long)nb, sizeof ng, cudaMemcpyDeviceToHost, h->st));
        CK(cudaMemcpyAsync(&ovf, h->flags + 2, sizeof ovf, cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        if (h->prof) prof_collect(h);
        out->F_tot = hs[0];
        out->X_rex = hs[1] / (double)h->N3pf;
        out->n_grains = (int)ng;
        out->overflow = ovf;
    } else {
        CK(cudaMemcpyAsync(&ovf, h->flags + 2, sizeof ovf, cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        if (h->prof) prof_collect(h);
    }
    return ovf > 0 ? EVP_WARN_OVERFLOW : EVP_OK;
}

int evp_fields_bytes(const evp_handle *h, uint32_t mask, size_t *bytes) {
    if (!h || !bytes) return EVP_ERR_ARG;
    if (mask == 0 || (mask >> 15) != 0) return EVP_ERR_ARG;
    if ((mask & EVP_F_GND) && !h->mr) return EVP_ERR_ARG;   // GND densities exist under the Ma-Roters law only
    size_t tot = 0;
    for (uint32_t bit = 1; bit <= EVP_F_GND; bit <<= 1)
        if (mask & bit) tot += field_bytes(h, bit);
    *bytes = tot;
    return EVP_OK;
}

int get_fields(evp_handle *h, uint32_t mask, void *dst, size_t bytes, int dst_is_device) {
    size_t need = 0;
    if (!h || !dst) return fail(h, EVP_ERR_ARG, "NULL argument to get_fields");
    if (evp_fields_bytes(h, mask, &need) != EVP_OK) return fail(h, EVP_ERR_ARG, "bad field mask 0x%x", mask);
    if (bytes != need) return fail(h, EVP_ERR_ARG, "get_fields: %zu bytes given, %zu expected", bytes, need);
    const cudaMemcpyKind kind = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    size_t off = 0;
    for (uint32_t bit = 1; bit <= EVP_F_GND; bit <<= 1) {
        if (!(mask & bit)) continue;
        const size_t fb = field_bytes(h, bit);
        const void *src = field_ptr(h, bit);
        if (bit == EVP_F_EPS) {
            if (h->dbl) CK(total_strain<double>(h->N3, (double *)h->epse, (double *)h->epsp, (double *)h->spec, h->st));
            else CK(total_strain<float>(h->N3, (float *)h->epse, (float *)h->epsp, (float *)h->spec, h->st));
            src = h->spec;
        }
        CK(cudaMemcpyAsync((char *)dst + off, src, fb, kind, h->st));
        off += fb;
    }
    CK(cudaStreamSynchronize(h->st));
    return EVP_OK;
}

int set_fields(evp_handle *h, uint32_t mask, const void *src, size_t bytes, int src_is_device) {
    size_t need = 0;
    if (!h || !src) return fail(h, EVP_ERR_ARG, "NULL argument to set_fields");
    if (mask & (EVP_F_EPS | EVP_F_G0 | EVP_F_GRAIN_PF))
        return fail(h, EVP_ERR_ARG, "EVP_F_EPS, EVP_F_G0 and EVP_F_GRAIN_PF cannot be set");
    if (evp_fields_bytes(h, mask, &need) != EVP_OK) return fail(h, EVP_ERR_ARG, "bad field mask 0x%x", mask);
    if (bytes != need) return fail(h, EVP_ERR_ARG, "set_fields: %zu bytes given, %zu expected", bytes, need);
    const cudaMemcpyKind kind = src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    size_t off = 0;
    for (uint32_t bit = 1; bit <= EVP_F_GND; bit <<= 1) {
        if (!(mask & bit)) continue;
        const size_t fb = field_bytes(h, bit);
        CK(cudaMemcpyAsync(field_ptr(h, bit), (const char *)src + off, fb, kind, h->st));
        off += fb;
    }
    if ((mask & EVP_F_IDS) && h->rmax_bytes)   // arbitrary active sets: every slot may be in use
        CK(cudaMemsetAsync(h->rmax, h->K, h->rmax_bytes, h->st));
    if (mask & (EVP_F_RHO | EVP_F_GND)) {
        if (h->mr) CK(mr_refresh_k(h));
        else if (h->dbl) CK(refresh_k<double>(h->N3, (double *)h->rho, h->k, h->st));
        else CK(refresh_k<float>(h->N3, (float *)h->rho, h->k, h->st));
        if (h->r == 2) CK(pf_interp(h->n, h->k, h->kpf, h->st));
    }
    CK(cudaStreamSynchronize(h->st));
    return EVP_OK;
}

int evp_get_scalars(const evp_handle *h, double *E6, double *dE_prev6, int *have_prev, int *next_id) {
    if (!h) return EVP_ERR_ARG;
    for (int i = 0; i < 6; ++i) {
        if (E6) E6[i] = h->E[i];
        if (dE_prev6) dE_prev6[i] = h->dE_prev[i];
    }
    if (have_prev) *have_prev = h->have_prev;
    if (next_id) *next_id = h->next_id;
    return EVP_OK;
}

int evp_set_scalars(evp_handle *h, const double *E6, const double *dE_prev6, int have_prev, int next_id) {
    if (!h || next_id < h->G || next_id > h->max_ids) return fail(h, EVP_ERR_ARG, "bad scalars");
    for (int i = 0; i < 6; ++i) {
        if (E6) h->E[i] = E6[i];
        if (dE_prev6) h->dE_prev[i] = dE_prev6[i];
    }
    h->have_prev = have_prev;
    h->next_id = next_id;
    return EVP_OK;
}

int evp_get_leff(const evp_handle *h, double *leff) {
    if (!h || !leff) return EVP_ERR_ARG;
    *leff = h->leff;
    return EVP_OK;
}

int evp_set_leff(evp_handle *h, double leff) {
    if (!h || !(leff > 0.0) || !std::isfinite(leff)) return fail(h, EVP_ERR_ARG, "l_eff must be positive and finite");
    h->leff = leff;
    return EVP_OK;
}

int evp_voronoi(int n, int grains, const int64_t *seeds_dev, int32_t *ids_dev, void *cuda_stream) {
    if (!pow2(n) || grains < 1 || !seeds_dev || !ids_dev) return EVP_ERR_ARG;
    const cudaError_t e = voronoi(n, grains, seeds_dev, ids_dev, (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? EVP_OK : EVP_ERR_CUDA;
}

int evp_rfft3d(int n, int precision, int nfields, const void *in_dev, void *out_dev, void *cuda_stream) {
    if (!pow2(n) || nfields < 1 || nfields > 6 || !in_dev || !out_dev) return EVP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e;
    if (precision == EVP_FP64) {
        e = fft_xy_r2c<double>((const double *)in_dev, out_dev, n, nfields, s);
        if (e == cudaSuccess) e = fft_z<double>(out_dev, n, nfields, Z_FWD, 0, 0, nullptr, nullptr, s);
    } else {
        e = fft_xy_r2c<float>((const float *)in_dev, out_dev, n, nfields, s);
        if (e == cudaSuccess) e = fft_z<float>(out_dev, n, nfields, Z_FWD, 0, 0, nullptr, nullptr, s);
    }
    return e == cudaSuccess ? EVP_OK : EVP_ERR_CUDA;
}

int evp_irfft3d(int n, int precision, int nfields, void *in_dev, void *out_dev, void *cuda_stream) {
    if (!pow2(n) || nfields < 1 || nfields > 6 || !in_dev || !out_dev) return EVP_ERR_ARG;
    if (((uintptr_t)in_dev | (uintptr_t)out_dev) & 15) return EVP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e;
    if (precision == EVP_FP64) {
        e = fft_z<double>(in_dev, n, nfields, Z_INV, 0, 0, nullptr, nullptr, s);
        if (e == cudaSuccess) e = fft_xy_c2r<double>(in_dev, (double *)out_dev, n, nfields, 1.0, nullptr, s);
    } else {
        e = fft_z<float>(in_dev, n, nfields, Z_INV, 0, 0, nullptr, nullptr, s);
        if (e == cudaSuccess) e = fft_xy_c2r<float>(in_dev, (float *)out_dev, n, nfields, 1.0f, nullptr, s);
    }
    return e == cudaSuccess ? EVP_OK : EVP_ERR_CUDA;
}

}  // extern "C"

// ---- differentiation: checkpointed discrete adjoint ----
namespace {

struct AdjLayout {
    size_t slot, tape_rho, tape_sig, lam_ep, lam_rho, Ct, sbar, a, eb, taub, part, total;
    int nseg;
};

AdjLayout adj_layout(const evp_config *c, int T, int ck) {
    const size_t N3 = (size_t)c->n * c->n * c->n;
    const size_t ts = c->precision == EVP_FP64 ? 8 : 4;
    AdjLayout L{};
    L.nseg = (T + ck - 1) / ck;
    size_t off = 0;
    auto take = [&](size_t b) { off = (off + 255) & ~(size_t)255; size_t o = off; off += b; return o; };
    L.slot = take((size_t)(L.nseg + 1) * 36 * N3 * ts);
    L.tape_rho = take((size_t)ck * 12 * N3 * ts);
    L.tape_sig = take((size_t)ck * 6 * N3 * ts);
    L.lam_ep = take(6 * N3 * ts);
    L.lam_rho = take(12 * N3 * ts);
    L.Ct = take(21 * N3 * ts);
    L.sbar = take(6 * N3 * ts);
    L.a = take(6 * N3 * ts);
    L.eb = take(6 * N3 * ts);
    L.taub = take(N3 * ts);
    L.part = take(sizeof(double) * 4 * (size_t)adj_blocks((long)N3));
    L.total = (off + 255) & ~(size_t)255;
    return L;
}

// state slot: sig, epse, epsp, deps (6 each), rho (12) -- everything an increment reads
int save_slot(evp_handle *h, char *slot, int k) {
    const size_t f6 = 6 * (size_t)h->N3 * h->tsz;
    CK(cudaMemcpyAsync(slot, h->sig, f6, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(slot + f6, h->epse, f6, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(slot + 2 * f6, h->epsp, f6, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(slot + 3 * f6, h->deps, f6, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(slot + 4 * f6, h->rho, 2 * f6, cudaMemcpyDeviceToDevice, h->st));
    for (int i = 0; i < 6; ++i) {
        h->adj_E[6 * k + i] = h->E[i];
        h->adj_dEp[6 * k + i] = h->dE_prev[i];
    }
    h->adj_hp[k] = h->have_prev;
    return EVP_OK;
}

int load_slot(evp_handle *h, const char *slot, int k) {
    const size_t f6 = 6 * (size_t)h->N3 * h->tsz;
    CK(cudaMemcpyAsync(h->sig, slot, f6, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(h->epse, slot + f6, f6, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(h->epsp, slot + 2 * f6, f6, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(h->deps, slot + 3 * f6, f6, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(h->rho, slot + 4 * f6, 2 * f6, cudaMemcpyDeviceToDevice, h->st));
    if (h->dbl) CK(refresh_k<double>(h->N3, (double *)h->rho, h->k, h->st));
    else CK(refresh_k<float>(h->N3, (float *)h->rho, h->k, h->st));
    for (int i = 0; i < 6; ++i) {
        h->E[i] = h->adj_E[6 * k + i];
        h->dE_prev[i] = h->adj_dEp[6 * k + i];
    }
    h->have_prev = h->adj_hp[k];
    return EVP_OK;
}

template <typename TA>
int adjoint_sweep(evp_handle *h, const AdjLayout &L, const double *gbar, double *grad, double tol, int max_iter) {
    const long N3 = h->N3;
    const int n = h->n, T = h->adj_t, ck = h->adj_c;
    const size_t ts = h->tsz;
    char *base = h->adj;
    const size_t slot_b = 36 * (size_t)N3 * ts;
    TA *tape_rho = (TA *)(base + L.tape_rho), *tape_sig = (TA *)(base + L.tape_sig);
    TA *lam_ep = (TA *)(base + L.lam_ep), *lam_rho = (TA *)(base + L.lam_rho), *Ct = (TA *)(base + L.Ct);
    TA *sbar = (TA *)(base + L.sbar), *aa = (TA *)(base + L.a), *eb = (TA *)(base + L.eb), *taub = (TA *)(base + L.taub);
    double *part = (double *)(base + L.part);
    const int nb = adj_blocks(N3);
    const int nseg = (T + ck - 1) / ck;
    const double lam0 = h->mc.lam0, mu0 = h->mc.mu0;
    const double aa_ = lam0 + 2.0 * mu0, bb_ = lam0, det = aa_ * aa_ - bb_ * bb_;
    const int zb = fft_z_blocks(n, h->dbl);
    double gk1 = 0, gk2 = 0, gt0 = 0, gn = 0;
    int rc = save_slot(h, base + L.slot + (size_t)nseg * slot_b, nseg);
    if (rc) return rc;
    CK(cudaMemsetAsync(lam_ep, 0, 6 * (size_t)N3 * ts, h->st));
    CK(cudaMemsetAsync(lam_rho, 0, 12 * (size_t)N3 * ts, h->st));
    for (int seg = nseg - 1; seg >= 0; --seg) {
        const int s0 = seg * ck, s1 = std::min(s0 + ck, T);
        rc = load_slot(h, base + L.slot + (size_t)seg * slot_b, seg);
        if (rc) return rc;
        for (int t = s0; t < s1; ++t) {   // recompute the segment, keeping rho^{t-1} and sigma^t
            CK(cudaMemcpyAsync(tape_rho + (size_t)(t - s0) * 12 * N3, h->rho, 12 * (size_t)N3 * ts,
                               cudaMemcpyDeviceToDevice, h->st));
            rc = evp_increment(h, h->adj_dE33[t], h->adj_dt[t], nullptr);
            if (rc < 0) return rc;
            CK(cudaMemcpyAsync(tape_sig + (size_t)(t - s0) * 6 * N3, h->sig, 6 * (size_t)N3 * ts,
                               cudaMemcpyDeviceToDevice, h->st));
        }
        for (int t = s1 - 1; t >= s0; --t) {
            MatConst mc = h->mc;
            mc.dt = h->adj_dt[t];
            mc.set_fp32();
            const TA *rp = tape_rho + (size_t)(t - s0) * 12 * N3, *sg = tape_sig + (size_t)(t - s0) * 6 * N3;
            CK(adj_prep<TA>(N3, h->g0, (const TA *)h->Stab, (const TA *)h->Mtab, rp, sg, lam_ep, lam_rho, Ct, sbar, aa,
                            taub, mc, gbar + 6 * (size_t)t, part, h->st));
            CK(reduce_partials(part, nb, 4, h->scal + 16, h->st));
            double r4[4];
            CK(cudaMemcpyAsync(r4, h->scal + 16, sizeof r4, cudaMemcpyDeviceToHost, h->st));
            CK(cudaStreamSynchronize(h->st));
            gk1 += r4[0];
            gk2 += r4[1];
            gn += r4[2];
            const double rms = std::sqrt(r4[3] / (double)N3);
            CK(cudaMemsetAsync(eb, 0, 6 * (size_t)N3 * ts, h->st));
            if (rms > 0.0) {
                int it;
                double err = 0.0;
                for (it = 1; it <= max_iter; ++it) {
                    CK(adj_tau<TA>(N3, Ct, eb, aa, (TA *)h->sigk, h->st));
                    CK(fft_xy_r2c<TA>((const TA *)h->sigk, h->spec, n, 6, h->st));
                    CK(fft_z<TA>(h->spec, n, 6, Z_FWD_GAMMA_INV, lam0, mu0, h->partials, h->scal, h->st));
                    CK(reduce_partials(h->partials, zb, 1, h->scal + 6, h->st));
                    double hs[7];
                    CK(cudaMemcpyAsync(hs, h->scal, sizeof hs, cudaMemcpyDeviceToHost, h->st));
                    CK(cudaStreamSynchronize(h->st));
                    h->launches += 3 + xy_launches(h);
                    double mu_n = 0.0;
                    for (int i = 0; i < 6; ++i)
                        if (i != 2) mu_n += hs[i] * hs[i];
                    err = std::sqrt(hs[6]) / ((double)N3 * rms) + std::sqrt(mu_n) / rms;
                    if (!std::isfinite(err)) return fail(h, EVP_ERR_NONFINITE, "non-finite adjoint residual");
                    if (err <= tol) break;
                    double dEk[6] = {0, 0, 0, 0, 0, 0};
                    dEk[0] = (aa_ * (-hs[0]) - bb_ * (-hs[1])) / det;
                    dEk[1] = (-bb_ * (-hs[0]) + aa_ * (-hs[1])) / det;
                    for (int i = 3; i < 6; ++i) dEk[i] = -hs[i] / (2.0 * mu0);
                    CK(fft_xy_c2r<TA>(h->spec, eb, n, 6, (TA)(1.0 / (double)N3), dEk, h->st));
                    h->launches += xy_launches(h);
                }
                if (it > max_iter)
                    return fail(h, EVP_ERR_FIXEDPOINT, "adjoint fixed point not converged at increment %d (err %.3e)", t,
                                err);
            }
            CK(adj_finish<TA>(N3, h->g0, (const TA *)h->Mtab, rp, sg, Ct, sbar, eb, taub, lam_ep, lam_rho, mc, part,
                              h->st));
            CK(reduce_partials(part, nb, 2, h->scal + 16, h->st));
            double r2[2];
            CK(cudaMemcpyAsync(r2, h->scal + 16, sizeof r2, cudaMemcpyDeviceToHost, h->st));
            CK(cudaStreamSynchronize(h->st));
            h->launches += 4;
            gt0 += r2[0];
            gn += r2[1];
        }
    }
    rc = load_slot(h, base + L.slot + (size_t)nseg * slot_b, nseg);
    if (rc) return rc;
    CK(cudaStreamSynchronize(h->st));
    grad[0] = gk1;
    grad[1] = gk2;
    grad[2] = gt0;
    grad[3] = gn;
    return EVP_OK;
}

}  // namespace

extern "C" {

int evp_adjoint_workspace_bytes(const evp_config *cfg, int n_increments, int checkpoint_every, size_t *bytes) {
    char why[256];
    if (check_cfg(cfg, why, sizeof why) != EVP_OK || n_increments < 1 || checkpoint_every < 1 || !bytes)
        return EVP_ERR_ARG;
    *bytes = adj_layout(cfg, n_increments, checkpoint_every).total;
    return EVP_OK;
}

int evp_adjoint_begin(evp_handle *h, void *adj_ws, size_t bytes, int n_increments, int checkpoint_every) {
    if (!h || !adj_ws || n_increments < 1 || checkpoint_every < 1) return fail(h, EVP_ERR_ARG, "bad adjoint arguments");
    if (((uintptr_t)adj_ws & 255) != 0) return fail(h, EVP_ERR_ARG, "adjoint workspace must be 256-byte aligned");
    if (h->mr) return fail(h, EVP_ERR_ARG, "the adjoint covers the power law with Kocks-Mecking hardening only");
    const AdjLayout L = adj_layout(&h->cfg, n_increments, checkpoint_every);
    if (bytes < L.total) return fail(h, EVP_ERR_OOM, "adjoint workspace has %zu bytes, needs %zu", bytes, L.total);
    std::free(h->adj_dE33); std::free(h->adj_dt); std::free(h->adj_E); std::free(h->adj_dEp); std::free(h->adj_hp);
    h->adj_dE33 = (double *)std::malloc(sizeof(double) * n_increments);
    h->adj_dt = (double *)std::malloc(sizeof(double) * n_increments);
    h->adj_E = (double *)std::malloc(sizeof(double) * 6 * (L.nseg + 1));
    h->adj_dEp = (double *)std::malloc(sizeof(double) * 6 * (L.nseg + 1));
    h->adj_hp = (int *)std::malloc(sizeof(int) * (L.nseg + 1));
    if (!h->adj_dE33 || !h->adj_dt || !h->adj_E || !h->adj_dEp || !h->adj_hp) return fail(h, EVP_ERR_OOM, "host allocation");
    h->adj = (char *)adj_ws;
    h->adj_bytes = bytes;
    h->adj_T = n_increments;
    h->adj_c = checkpoint_every;
    h->adj_t = 0;
    const int rc = save_slot(h, h->adj + L.slot, 0);
    if (rc) return rc;
    CK(cudaStreamSynchronize(h->st));
    return EVP_OK;
}

int evp_adjoint_step(evp_handle *h, double dE33, double dt, evp_stats *out) {
    if (!h || !h->adj) return fail(h, EVP_ERR_ARG, "evp_adjoint_begin was not called");
    if (h->adj_t >= h->adj_T) return fail(h, EVP_ERR_ARG, "more than %d recorded increments", h->adj_T);
    const int rc = evp_increment(h, dE33, dt, out);
    if (rc < 0) return rc;
    h->adj_dE33[h->adj_t] = dE33;
    h->adj_dt[h->adj_t] = dt;
    h->adj_t += 1;
    if (h->adj_t % h->adj_c == 0 && h->adj_t < h->adj_T) {
        const AdjLayout L = adj_layout(&h->cfg, h->adj_T, h->adj_c);
        const int k = h->adj_t / h->adj_c;
        const int r2 = save_slot(h, h->adj + L.slot + (size_t)k * 36 * h->N3 * h->tsz, k);
        if (r2) return r2;
    }
    return rc;
}

int evp_adjoint_end(evp_handle *h, const double *gbar, double *grad, double tol, int max_iter) {
    if (!h || !h->adj || !gbar || !grad || max_iter < 1 || !(tol > 0.0))
        return fail(h, EVP_ERR_ARG, "bad evp_adjoint_end arguments");
    if (h->adj_t < 1) return fail(h, EVP_ERR_ARG, "no recorded increments");
    const AdjLayout L = adj_layout(&h->cfg, h->adj_T, h->adj_c);
    return h->dbl ? adjoint_sweep<double>(h, L, gbar, grad, tol, max_iter)
                  : adjoint_sweep<float>(h, L, gbar, grad, tol, max_iter);
}

}  // extern "C"

extern "C" {
int evp_residual_scratch_bytes(int n, int precision, size_t *bytes) {
    if (!pow2(n) || !bytes || precision < EVP_FP64 || precision > EVP_MIXED_FAST) return EVP_ERR_ARG;
    *bytes = sizeof(double) * (size_t)fft_z_blocks(n, precision == EVP_FP64);
    return EVP_OK;
}

int evp_stress_residual(int n, int precision, const void *sig_dev, void *spec_dev, void *scratch_dev,
                        double *out_dev, void *cuda_stream) {
    if (!pow2(n) || !sig_dev || !spec_dev || !scratch_dev || !out_dev) return EVP_ERR_ARG;
    if (precision < EVP_FP64 || precision > EVP_MIXED_FAST) return EVP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int dbl = precision == EVP_FP64;
    double *part = (double *)scratch_dev;
    cudaError_t e;
    if (dbl) {
        e = fft_xy_r2c<double>((const double *)sig_dev, spec_dev, n, 6, s);
        if (e == cudaSuccess) e = fft_z<double>(spec_dev, n, 6, Z_FWD_RESID, 0, 0, part, out_dev, s);
    } else {
        e = fft_xy_r2c<float>((const float *)sig_dev, spec_dev, n, 6, s);
        if (e == cudaSuccess) e = fft_z<float>(spec_dev, n, 6, Z_FWD_RESID, 0, 0, part, out_dev, s);
    }
    if (e == cudaSuccess) e = reduce_partials(part, fft_z_blocks(n, dbl), 1, out_dev + 6, s);
    return e == cudaSuccess ? EVP_OK : EVP_ERR_CUDA;
}

}  // extern "C"
