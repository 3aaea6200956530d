// Active-set multi-grain Allen-Cahn step (Sec. 2.4, Eqs. TotalFreeEnergy, GBEnergyDensity,
// StoredEnergyDensity, PFGoverning; sparse storage after the cited Gruber / Vedantam technique).
//
// Grid-nondimensional form (lengths dx, energies omega_gb/dx, time dx^2/(M omega_gb)):
//   m = 6/l, kappa = 3l/4, gamma = 3/2,  E' = zeta mu b^2 rho_tot dx / omega_gb
//   eta_i <- eta_i - L dt [ m (eta_i^3 - eta_i + 2 gamma eta_i (S2 - eta_i^2)) - kappa lap(eta_i)
//                            + (i deformed: 2E' eta_i R/S^2 | i recrystallised: -2E' eta_i D/S^2) ]
// with S2 = D + R the local sum of eta^2 over deformed (D, ids < G) and recrystallised (R)
// grains and a periodic 7-point Laplacian. Each voxel stores up to K (id, eta) pairs sorted by
// id (-1 = empty). Candidates at a voxel are the ids present there or at its six neighbours;
// values below `drop` are discarded, the K largest kept (ties to the smaller id) and the grain
// id is the argmax. This file is compiled without FMA contraction so that, in FP64, each value
// is rounded exactly as the plain formula above prescribes.
#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace evp {

namespace {

constexpr int KM = 8;   // compile-time capacity of the active set (runtime K <= KM)
constexpr int kPF = 128;

struct Nbr {
    long q[7];   // self, x-, x+, y-, y+, z-, z+
};

// n is a power of two (checked at init): coordinates and periodic wraps by masks and shifts
__device__ __forceinline__ Nbr neighbours(int n, long v) {
    const int lg = __ffs(n) - 1;
    const long msk = n - 1;
    const int x = (int)(v & msk), y = (int)((v >> lg) & msk), z = (int)(v >> (2 * lg));
    const long nn = (long)n * n;
    Nbr b;
    b.q[0] = v;
    b.q[1] = v - x + ((x - 1) & msk);
    b.q[2] = v - x + ((x + 1) & msk);
    b.q[3] = v + (long)(((y - 1) & msk) - y) * n;
    b.q[4] = v + (long)(((y + 1) & msk) - y) * n;
    b.q[5] = v + (long)(((z - 1) & msk) - z) * nn;
    b.q[6] = v + (long)(((z + 1) & msk) - z) * nn;
    return b;
}

constexpr int kEmpty = 0x7fffffff;

// Asynchronous global -> shared copy of B bytes (cp.async; completion by commit / wait groups).
template <int B> __device__ __forceinline__ void cp_async(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (B == 4) asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}


template <typename T>
__global__ void __launch_bounds__(kPF) k_pf(int n, const int32_t *__restrict__ ids, const T *__restrict__ eta,
                                           int32_t *__restrict__ ids2, T *__restrict__ eta2, int32_t *__restrict__ gout,
                                           const double *__restrict__ kf, PFConst pc, int32_t *__restrict__ overflow) {
    const long N3 = (long)n * n * n;
    const long v = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N3) return;
    const int K = pc.K, G = pc.G;
    const Nbr nb = neighbours(n, v);
    T m, kap, gam, Ldt, drop;   // in the field precision (no FP64 conversions on the FP32 path)
    if constexpr (sizeof(T) == 4) { m = pc.m_f; kap = pc.kappa_f; gam = pc.gam_f; Ldt = pc.L_dt_f; drop = pc.drop_f; }
    else { m = pc.m; kap = pc.kappa; gam = pc.gam; Ldt = pc.L_dt; drop = pc.drop; }
    // local sums over the voxel's own list, ascending id
    T S2 = (T)0, D = (T)0, R = (T)0;
    for (int j = 0; j < K; ++j) {
        const int id = ids[j * N3 + v];
        if (id < 0) break;
        const T e = eta[j * N3 + v];
        S2 += e * e;
        if (id < G) D += e * e;
        else R += e * e;
    }
    const T Ep = (T)(pc.Escale * kf[v]);
    const T Ssum = D + R;
    // merge the seven sorted lists
    int head[7], pos[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        pos[q] = 0;
        const int id = ids[nb.q[q]];
        head[q] = id < 0 ? kEmpty : id;
    }
    // Kept entries in ascending id order (the merge yields candidates in that order): append; past K,
    // drop the worst (smallest value, the larger id among equal values), which leaves the top K by
    // (value desc, id asc) -- the same set a full sort would keep -- still in id order.
    int kid[KM + 1];
    T ke[KM + 1];
#pragma unroll
    for (int j = 0; j <= KM; ++j) {
        kid[j] = kEmpty;
        ke[j] = (T)0;
    }
    int cnt = 0;
    int best_id = kEmpty, kbest_id = kEmpty;
    T best = (T)-INFINITY, kbest = (T)-INFINITY;
    bool ovf = false;
    for (int guard = 0; guard < 7 * KM; ++guard) {
        int c = head[0];
#pragma unroll
        for (int q = 1; q < 7; ++q) c = min(c, head[q]);
        if (c == kEmpty) break;
        T e[7];
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            e[q] = (T)0;
            if (head[q] == c) {
                e[q] = eta[pos[q] * N3 + nb.q[q]];
                ++pos[q];
                int nx = kEmpty;
                if (pos[q] < K) {
                    const int id = ids[pos[q] * N3 + nb.q[q]];
                    nx = id < 0 ? kEmpty : id;
                }
                head[q] = nx;
            }
        }
        const T e0 = e[0];
        const T lap = e[1] + e[2] + e[3] + e[4] + e[5] + e[6] - (T)6 * e0;
        const T df0 = m * (e0 * e0 * e0 - e0 + (T)2 * gam * e0 * (S2 - e0 * e0));
        T ddef = (T)0;
        if (Ssum > (T)1e-12) ddef = (c < G) ? (T)2 * Ep * e0 * R / (Ssum * Ssum) : -(T)2 * Ep * e0 * D / (Ssum * Ssum);
        const T en = e0 - Ldt * (df0 - kap * lap + ddef);
        if (en > best) { best = en; best_id = c; }
        if (en >= drop) {
            if (en > kbest) { kbest = en; kbest_id = c; }   // ascending ids: a tie keeps the smaller id
#pragma unroll
            for (int j = 0; j <= KM; ++j)
                if (j == cnt) { kid[j] = c; ke[j] = en; }
            ++cnt;
            if (cnt > K) {   // over capacity: remove the worst entry
                ovf = true;
                int wj = 0, wid = kid[0];
                T wv = ke[0];
#pragma unroll
                for (int j = 1; j <= KM; ++j)
                    if (j < cnt && (ke[j] < wv || (ke[j] == wv && kid[j] > wid))) { wj = j; wv = ke[j]; wid = kid[j]; }
#pragma unroll
                for (int j = 0; j < KM; ++j)
                    if (j >= wj) { kid[j] = kid[j + 1]; ke[j] = ke[j + 1]; }
                kid[KM] = kEmpty;
                ke[KM] = (T)0;
                cnt = K;
            }
        }
    }
    if (cnt == 0 && best_id != kEmpty) {   // nothing above the drop threshold: keep the largest
        kid[0] = best_id;
        ke[0] = best;
        cnt = 1;
        kbest_id = best_id;
    }
    gout[v] = kbest_id;
    // Write the kept entries; then clear the slots the destination still holds from its previous use
    // (every buffer keeps -1 / 0 beyond its entries, so those are the only stale ones).
#pragma unroll
    for (int j = 0; j < KM; ++j)
        if (j < cnt) {
            ids2[j * N3 + v] = kid[j];
            eta2[j * N3 + v] = ke[j];
        }
    for (int j = cnt; j < K; ++j) {
        if (ids2[j * N3 + v] < 0) break;
        ids2[j * N3 + v] = -1;
        eta2[j * N3 + v] = (T)0;
    }
    if (ovf) atomicAdd(overflow, 1);
}

// ---- tiled PF step (grids of 32 points per edge and more) ----
// The same update as k_pf, voxel by voxel and in the same arithmetic order (so FP64 results are bitwise the
// same), organised for the SM. A CTA owns a 32 x 8 column tile and marches through kZC planes of z. The active
// sets of the planes z-1, z, z+1 (interior) and the x/y halo of plane z are staged in shared memory by cp.async,
// as (id, eta) pairs with a -1 id after each list's last staged slot, so the seven-list merge reads one pair per
// step and needs no slot-count checks. Which slots to stage comes from a per-row bound: rmax[s] >= the number of
// entries of every point of the 32-point row segment s = (z n + y) (n / 32) + x / 32, so every staged load is
// independent of the others. Each step writes the exact bound of the rows it produced and clears, in the
// destination, the slots between a point's new count and the destination's previous bound, which keeps every
// list -1 / 0 terminated over all K slots (the layout every other reader of the active sets assumes).
// Three plane buffers and one halo buffer keep the FP32 tile at 61 KB, so three CTAs share an SM and cover each
// other's staging waits.
constexpr int kTX = 32, kTY = 8, kZC = 16;
constexpr int kPlane = kTX * kTY;             // interior points of one plane tile
constexpr int kHalo = 2 * kTX + 2 * kTY;      // rows y0-1, y0+8 and columns x0-1, x0+32 of the centre plane
constexpr int kTileThreads = kTX * kTY;
constexpr int kSlots = KM + 1;                // KM slots and the terminating -1

template <typename T> struct alignas(2 * sizeof(T) > 8 ? 16 : 8) PFPair {
    int32_t id;
    T e;
};

template <typename T>
struct PFTile {
    // element index space: 3 interior plane buffers [buf][slot][point], then the halo [slot][halo point]
    PFPair<T> pr[3 * kSlots * kPlane + kSlots * kHalo];
    uint8_t rin[(kZC + 2) * (kTY + 2)];   // bounds of the current buffer: planes z0-1..z0+kZC, rows y0-1..y0+8
    uint8_t rxl[kZC * kTY], rxr[kZC * kTY];   // bounds of the left / right neighbour segments, planes z0.., rows y0..
    uint8_t rdst[kZC * kTY];              // previous bounds of the destination rows
};

__device__ __forceinline__ int tile_int_index(int buf, int j, int p) { return (buf * kSlots + j) * kPlane + p; }
__device__ __forceinline__ int tile_halo_index(int j, int hp) { return 3 * kSlots * kPlane + j * kHalo + hp; }

// Issue the asynchronous copies of one point's slots [0, R) into the tile (element index base, slot stride) and
// write the terminating -1 at slot R (R <= K <= KM: global memory also holds -1 there when R < K).
template <typename T>
__device__ __forceinline__ void stage_point(PFTile<T> &tb, int base, int stride, int R, int K,
                                            const int32_t *__restrict__ ids, const T *__restrict__ eta, long N3,
                                            long v) {
    R = min(R, K);   // a bound never exceeds K; the clamp keeps every access inside the K slot planes regardless
#pragma unroll
    for (int j = 0; j < KM; ++j)
        if (j < R) {
            cp_async<4>(&tb.pr[base + j * stride].id, ids + j * N3 + v);
            cp_async<sizeof(T)>(&tb.pr[base + j * stride].e, eta + j * N3 + v);
        }
    tb.pr[base + R * stride].id = -1;
}

template <typename T>
__global__ void __launch_bounds__(kTileThreads, sizeof(T) == 4 ? 3 : 1)
k_pf_tile(int n, const int32_t *__restrict__ ids, const T *__restrict__ eta, int32_t *__restrict__ ids2,
          T *__restrict__ eta2, int32_t *__restrict__ gout, const double *__restrict__ kf, PFConst pc,
          int32_t *__restrict__ overflow, const uint8_t *__restrict__ rcur, uint8_t *__restrict__ rdst) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PFTile<T> &tb = *reinterpret_cast<PFTile<T> *>(smem_raw);
    const long N3 = (long)n * n * n;
    const int msk = n - 1, nseg = n / kTX;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int xs = blockIdx.x, x0 = xs * kTX, y0 = blockIdx.y * kTY, z0 = blockIdx.z * kZC;
    const int K = pc.K, G = pc.G;
    auto seg = [&](int z, int y, int s) { return ((long)z * n + y) * nseg + s; };
    // row bounds of the chunk
    for (int t = threadIdx.x; t < (kZC + 2) * (kTY + 2); t += kTileThreads) {
        const int pz = t / (kTY + 2), ry = t % (kTY + 2);
        tb.rin[t] = rcur[seg((z0 - 1 + pz) & msk, (y0 - 1 + ry) & msk, xs)];
    }
    for (int t = threadIdx.x; t < kZC * kTY; t += kTileThreads) {
        const int pz = t / kTY, ry = t % kTY;
        tb.rxl[t] = rcur[seg(z0 + pz, y0 + ry, (xs + nseg - 1) % nseg)];
        tb.rxr[t] = rcur[seg(z0 + pz, y0 + ry, (xs + 1) % nseg)];
        tb.rdst[t] = rdst[seg(z0 + pz, y0 + ry, xs)];
    }
    __syncthreads();
    const int p = ty * kTX + tx;
    // plane index pp = 0 .. kZC+1 holds z = z0 - 1 + pp in interior buffer pp % 3
    auto stage_plane = [&](int pp) {
        const int z = (z0 - 1 + pp) & msk;
        const long v = ((long)z * n + (y0 + ty)) * n + x0 + tx;
        stage_point(tb, tile_int_index(pp % 3, 0, p), kPlane, tb.rin[pp * (kTY + 2) + ty + 1], K, ids, eta, N3, v);
    };
    // halo of centre plane i (z = z0 + i)
    auto stage_halo = [&](int i) {
        const int t = threadIdx.x;
        if (t >= kHalo) return;
        const int z = z0 + i;
        int x, y, R;
        if (t < kTX) { x = x0 + t; y = (y0 - 1) & msk; R = tb.rin[(i + 1) * (kTY + 2)]; }
        else if (t < 2 * kTX) { x = x0 + t - kTX; y = (y0 + kTY) & msk; R = tb.rin[(i + 1) * (kTY + 2) + kTY + 1]; }
        else if (t < 2 * kTX + kTY) { x = (x0 - 1) & msk; y = y0 + t - 2 * kTX; R = tb.rxl[i * kTY + t - 2 * kTX]; }
        else { x = (x0 + kTX) & msk; y = y0 + t - 2 * kTX - kTY; R = tb.rxr[i * kTY + t - 2 * kTX - kTY]; }
        const long v = ((long)z * n + y) * n + x;
        stage_point(tb, tile_halo_index(0, t), kHalo, R, K, ids, eta, N3, v);
    };
    stage_plane(0);
    stage_plane(1);
    stage_plane(2);
    stage_halo(0);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();

    T m, kap, gam, Ldt, drop;   // in the field precision (no FP64 conversions on the FP32 path)
    if constexpr (sizeof(T) == 4) { m = pc.m_f; kap = pc.kappa_f; gam = pc.gam_f; Ldt = pc.L_dt_f; drop = pc.drop_f; }
    else { m = pc.m; kap = pc.kappa; gam = pc.gam; Ldt = pc.L_dt; drop = pc.drop; }

    for (int i = 0; i < kZC; ++i) {
        const int z = z0 + i;
        const long v = ((long)z * n + (y0 + ty)) * n + x0 + tx;
        const double kv = kf[v];
        // the seven lists: self, x-, x+, y-, y+, z-, z+ -- element index of the current slot, slot stride
        // (kPlane, or kHalo where the bit of `halo` is set)
        const int c = (i + 1) % 3;
        int at[7];
        at[0] = tile_int_index(c, 0, p);
        unsigned halo = 0;
        if (tx > 0) at[1] = at[0] - 1; else { at[1] = tile_halo_index(0, 2 * kTX + ty); halo |= 2u; }
        if (tx < kTX - 1) at[2] = at[0] + 1; else { at[2] = tile_halo_index(0, 2 * kTX + kTY + ty); halo |= 4u; }
        if (ty > 0) at[3] = at[0] - kTX; else { at[3] = tile_halo_index(0, tx); halo |= 8u; }
        if (ty < kTY - 1) at[4] = at[0] + kTX; else { at[4] = tile_halo_index(0, kTX + tx); halo |= 16u; }
        at[5] = tile_int_index(i % 3, 0, p);
        at[6] = tile_int_index((i + 2) % 3, 0, p);

        // local sums over the voxel's own list, ascending id (the list ends at a -1)
        T S2 = (T)0, D = (T)0, R = (T)0;
        for (int j = 0; j < kSlots; ++j) {
            const PFPair<T> pj = tb.pr[at[0] + j * kPlane];
            if (pj.id < 0) break;
            S2 += pj.e * pj.e;
            if (pj.id < G) D += pj.e * pj.e;
            else R += pj.e * pj.e;
        }
        const T Ep = (T)(pc.Escale * kv);
        const T Ssum = D + R;
        int head[7];
        T cur[7];
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            const PFPair<T> pq = tb.pr[at[q]];
            head[q] = pq.id < 0 ? kEmpty : pq.id;
            cur[q] = pq.e;
        }
        int kid[KM + 1];
        T ke[KM + 1];
#pragma unroll
        for (int j = 0; j <= KM; ++j) {
            kid[j] = kEmpty;
            ke[j] = (T)0;
        }
        int cnt = 0;
        int best_id = kEmpty, kbest_id = kEmpty;
        T best = (T)-INFINITY, kbest = (T)-INFINITY;
        bool ovf = false;
        for (int guard = 0; guard < 7 * KM; ++guard) {
            int cid = head[0];
#pragma unroll
            for (int q = 1; q < 7; ++q) cid = min(cid, head[q]);
            if (cid == kEmpty) break;
            T e[7];
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                const bool hit = head[q] == cid;
                e[q] = hit ? cur[q] : (T)0;
                if (hit) {   // advance list q to its next pair (a -1 id ends it)
                    at[q] += (halo >> q) & 1u ? kHalo : kPlane;
                    const PFPair<T> pq = tb.pr[at[q]];
                    head[q] = pq.id < 0 ? kEmpty : pq.id;
                    cur[q] = pq.e;
                }
            }
            const T e0 = e[0];
            const T lap = e[1] + e[2] + e[3] + e[4] + e[5] + e[6] - (T)6 * e0;
            const T df0 = m * (e0 * e0 * e0 - e0 + (T)2 * gam * e0 * (S2 - e0 * e0));
            T ddef = (T)0;
            if (Ssum > (T)1e-12)
                ddef = (cid < G) ? (T)2 * Ep * e0 * R / (Ssum * Ssum) : -(T)2 * Ep * e0 * D / (Ssum * Ssum);
            const T en = e0 - Ldt * (df0 - kap * lap + ddef);
            if (en > best) { best = en; best_id = cid; }
            if (en >= drop) {
                if (en > kbest) { kbest = en; kbest_id = cid; }   // ascending ids: a tie keeps the smaller id
#pragma unroll
                for (int j = 0; j <= KM; ++j)
                    if (j == cnt) { kid[j] = cid; ke[j] = en; }
                ++cnt;
                if (cnt > K) {   // over capacity: remove the worst entry (smallest value, larger id among equals)
                    ovf = true;
                    int wj = 0, wid = kid[0];
                    T wv = ke[0];
#pragma unroll
                    for (int j = 1; j <= KM; ++j)
                        if (j < cnt && (ke[j] < wv || (ke[j] == wv && kid[j] > wid))) { wj = j; wv = ke[j]; wid = kid[j]; }
#pragma unroll
                    for (int j = 0; j < KM; ++j)
                        if (j >= wj) { kid[j] = kid[j + 1]; ke[j] = ke[j + 1]; }
                    kid[KM] = kEmpty;
                    ke[KM] = (T)0;
                    cnt = K;
                }
            }
        }
        if (cnt == 0 && best_id != kEmpty) {   // nothing above the drop threshold: keep the largest
            kid[0] = best_id;
            ke[0] = best;
            cnt = 1;
            kbest_id = best_id;
        }
        gout[v] = kbest_id;
        // kept entries, then the slots up to the destination's previous bound cleared (beyond it they are empty)
        const int rd = min((int)tb.rdst[i * kTY + ty], K);
#pragma unroll
        for (int j = 0; j < KM; ++j) {
            if (j < cnt) {
                ids2[j * N3 + v] = kid[j];
                eta2[j * N3 + v] = ke[j];
            } else if (j < rd) {
                ids2[j * N3 + v] = -1;
                eta2[j * N3 + v] = (T)0;
            }
        }
        const int rowmax = __reduce_max_sync(0xffffffffu, (unsigned)cnt);
        if (tx == 0) rdst[seg(z, y0 + ty, xs)] = (uint8_t)rowmax;
        const unsigned ob = __ballot_sync(0xffffffffu, ovf);
        if (tx == 0 && ob) atomicAdd(overflow, __popc(ob));
        __syncthreads();   // every thread is done with plane z - 1 and with this halo
        if (i + 1 < kZC) {
            stage_plane(i + 3);   // into the buffer plane z - 1 held
            stage_halo(i + 1);
            asm volatile("cp.async.commit_group;\n" ::: "memory");
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
            __syncthreads();
        }
    }
}

template <typename T>
__global__ void k_pf_soften(long N3, const int32_t *__restrict__ gprev, const int32_t *__restrict__ g, T *__restrict__ rho,
                            double *__restrict__ kf, int G, double s) {
    const long v = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N3) return;
    if (!(gprev[v] < G && g[v] >= G)) return;
    double kk = 0.0;
    for (int a = 0; a < 12; ++a) {
        const T r = (T)(s * (double)rho[a * N3 + v]);
        rho[a * N3 + v] = r;
        kk += (double)r;
    }
    kf[v] = kk;
}

// Per-voxel discrete free energy (bulk + forward-difference gradient + stored energy) and
// recrystallised count, summed per block in FP64; distinct grain ids marked in a bitmap.
template <typename T>
__global__ void __launch_bounds__(256) k_pf_stats(int n, const int32_t *__restrict__ ids, const T *__restrict__ eta,
                                                 const int32_t *__restrict__ g, const double *__restrict__ kf, PFConst pc,
                                                 uint32_t *__restrict__ bitmap, int bitmap_words, double *__restrict__ part) {
    __shared__ double red[32];
    const long N3 = (long)n * n * n;
    const long v = (long)blockIdx.x * blockDim.x + threadIdx.x;
    double F = 0.0, rex = 0.0;
    if (v < N3) {
        const int K = pc.K, G = pc.G;
        const int gi = g[v];
        if (gi >= G) rex = 1.0;
        // one atomic per distinct id of the warp, and none once the bit is set: neighbouring voxels share
        // their ids, and same-address atomics from every voxel serialise
        const bool ok = gi >= 0 && (gi >> 5) < bitmap_words;
        const unsigned peers = __match_any_sync(__activemask(), ok ? gi : -1);
        if (ok && (threadIdx.x & 31) == __ffs(peers) - 1) {
            uint32_t *word = bitmap + (gi >> 5);
            const uint32_t bit = 1u << (gi & 31);
            if (!(*(volatile uint32_t *)word & bit)) atomicOr(word, bit);
        }
        // per-voxel terms in the field precision (the FP32 path keeps the FP64 pipe out), sums in FP64
        using A = T;
        const A gam = sizeof(T) == 4 ? (A)pc.gam_f : (A)pc.gam;
        A f0 = (A)0.25, S2 = (A)0, D = (A)0;
        for (int j = 0; j < K; ++j) {
            const int id = ids[j * N3 + v];
            if (id < 0) break;
            const A e = eta[j * N3 + v];
            f0 += e * e * e * e / (A)4 - e * e / (A)2;
            S2 += e * e;
            if (id < G) D += e * e;
            for (int i2 = j + 1; i2 < K; ++i2) {
                if (ids[i2 * N3 + v] < 0) break;
                const A e2 = eta[i2 * N3 + v];
                f0 += gam * e * e * e2 * e2;
            }
        }
        const A fdef = S2 > (A)1e-12 ? (A)(pc.Escale * kf[v]) * D / S2 : (A)0;
        const Nbr nb = neighbours(n, v);
        A grad = (A)0;
        for (int d = 2; d <= 6; d += 2) {   // x+, y+, z+
            const long w = nb.q[d];
            int pa = 0, pb = 0;
            for (int guard = 0; guard < 2 * KM; ++guard) {
                const int ia = pa < K ? ids[pa * N3 + v] : -1;
                const int ib = pb < K ? ids[pb * N3 + w] : -1;
                const int ca = ia < 0 ? kEmpty : ia, cb = ib < 0 ? kEmpty : ib;
                if (ca == kEmpty && cb == kEmpty) break;
                A ea = (A)0, eb = (A)0;
                if (ca <= cb) { ea = eta[pa * N3 + v]; ++pa; }
                if (cb <= ca) { eb = eta[pb * N3 + w]; ++pb; }
                grad += (eb - ea) * (eb - ea);
            }
        }
        F = (double)((sizeof(T) == 4 ? (A)pc.m_f : (A)pc.m) * f0 +
                     (A)0.5 * (sizeof(T) == 4 ? (A)pc.kappa_f : (A)pc.kappa) * grad + fdef);
    }
    const double sF = block_sum(F, red);
    const double sR = block_sum(rex, red);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sF;
        part[2 * blockIdx.x + 1] = sR;
    }
}

__global__ void k_popc(const uint32_t *__restrict__ bitmap, int words, double *__restrict__ out_slot) {
    __shared__ double red[32];
    double c = 0.0;
    for (int i = threadIdx.x; i < words; i += blockDim.x) c += (double)__popc(bitmap[i]);
    const double s = block_sum(c, red);
    if (threadIdx.x == 0) *out_slot = s;
}

// Deterministic sum of partials [nparts][nvals] -> out[nvals]: one block per column, fixed order.
__global__ void k_reduce(const double *__restrict__ part, int nparts, int nvals, double *__restrict__ out,
                         const int *__restrict__ skip) {
    if (skip != nullptr && *skip) return;
    __shared__ double red[32];
    const int c = blockIdx.x;
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += part[(long)i * nvals + c];
    s = block_sum(s, red);
    if (threadIdx.x == 0) out[c] = s;
}

// ---- 2:1 phase-field grid (Sec. 2.4) ----
// Both grids are cell-centred and periodic: voxel i spans [i, i+1), PF cell I spans [I/2, (I+1)/2).
// Along each axis a PF centre lies between its parent voxel's centre (weight 3/4) and the neighbour on
// its side (weight 1/4). PF point w = X + 2n (Y + 2n Z).
__device__ __forceinline__ void interp_axis(int I, int n, int (&idx)[2], double (&wt)[2]) {
    const int i = I >> 1;
    if ((I & 1) == 0) { idx[0] = (i + n - 1) % n; idx[1] = i; wt[0] = 0.25; wt[1] = 0.75; }
    else { idx[0] = i; idx[1] = (i + 1) % n; wt[0] = 0.75; wt[1] = 0.25; }
}

// kpf = trilinear interpolation of k (rho_tot); the eight terms in (z, y, x) order, weights (wz wy) wx
__global__ void k_interp_k(int n, const double *__restrict__ k, double *__restrict__ kpf) {
    const int m = 2 * n;
    const long M3 = (long)m * m * m;
    const long w = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= M3) return;
    const int X = (int)(w % m), Y = (int)((w / m) % m), Z = (int)(w / ((long)m * m));
    int ix[2], iy[2], iz[2];
    double wx[2], wy[2], wz[2];
    interp_axis(X, n, ix, wx);
    interp_axis(Y, n, iy, wy);
    interp_axis(Z, n, iz, wz);
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < 2; ++c)
                acc += (wz[a] * wy[b]) * wx[c] * k[ix[c] + (long)n * (iy[b] + (long)n * iz[a])];
    kpf[w] = acc;
}

// A voxel's grain id from its eight PF children c = dx + 2 dy + 4 dz: the id with the largest sum of
// order parameters over the children (summed in c order), ties to the smaller id. The children's
// lists are sorted by id, so the eight are merged in ascending id order.
template <typename T>
__global__ void k_restrict(int n, int K, const int32_t *__restrict__ ids, const T *__restrict__ eta,
                           int32_t *__restrict__ g) {
    const long N3 = (long)n * n * n;
    const long v = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N3) return;
    const int m = 2 * n;
    const long M3 = (long)m * m * m;
    const int x = (int)(v % n), y = (int)((v / n) % n), z = (int)(v / ((long)n * n));
    long ch[8];
    int pos[8], head[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        ch[c] = (2 * x + (c & 1)) + (long)m * ((2 * y + ((c >> 1) & 1)) + (long)m * (2 * z + (c >> 2)));
        pos[c] = 0;
        const int id = ids[ch[c]];
        head[c] = id < 0 ? kEmpty : id;
    }
    int best = -1;
    double bsum = 0.0;
    for (int guard = 0; guard < 8 * KM; ++guard) {
        int cmin = head[0];
#pragma unroll
        for (int c = 1; c < 8; ++c) cmin = min(cmin, head[c]);
        if (cmin == kEmpty) break;
        double sum = 0.0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            if (head[c] == cmin) {
                sum += (double)eta[pos[c] * M3 + ch[c]];
                ++pos[c];
                int nx = kEmpty;
                if (pos[c] < K) {
                    const int id = ids[pos[c] * M3 + ch[c]];
                    nx = id < 0 ? kEmpty : id;
                }
                head[c] = nx;
            }
        }
        if (best < 0 || sum > bsum) { best = cmin; bsum = sum; }   // ascending ids: a tie keeps the smaller
    }
    g[v] = best;
}

// initial active sets on the PF grid: one order parameter 1 of the parent voxel's grain
__global__ void k_pf_init(int n, int r, int K, const int32_t *__restrict__ g0, int32_t *__restrict__ ids,
                          void *__restrict__ eta, int32_t *__restrict__ ids2, void *__restrict__ eta2, int eta_double,
                          int32_t *__restrict__ gpf) {
    const int m = r * n;
    const long M3 = (long)m * m * m;
    const long w = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= M3) return;
    const int X = (int)(w % m), Y = (int)((w / m) % m), Z = (int)(w / ((long)m * m));
    const int gi = g0[X / r + (long)n * (Y / r + (long)n * (Z / r))];
    for (int j = 0; j < K; ++j) {
        ids[j * M3 + w] = j == 0 ? gi : -1;
        ids2[j * M3 + w] = -1;   // the step's destination: empty (it only rewrites slots in use)
        if (eta_double) {
            static_cast<double *>(eta)[j * M3 + w] = j == 0 ? 1.0 : 0.0;
            static_cast<double *>(eta2)[j * M3 + w] = 0.0;
        } else {
            static_cast<float *>(eta)[j * M3 + w] = j == 0 ? 1.f : 0.f;
            static_cast<float *>(eta2)[j * M3 + w] = 0.f;
        }
    }
    gpf[w] = gi;
}

}  // namespace

long pf_row_bounds_bytes(int n) { return n >= kTX ? (long)n * n * (n / kTX) : 0; }

template <typename T>
cudaError_t pf_one_step(int n, const int32_t *ids, const T *eta, int32_t *ids2, T *eta2, int32_t *g, const double *k,
                        PFConst pc, int32_t *overflow, const uint8_t *rcur, uint8_t *rdst, cudaStream_t s) {
    const long N3 = (long)n * n * n;
    if (pc.K > KM || pc.K < 1) return cudaErrorInvalidValue;
    if (n >= kTX && rcur != nullptr && rdst != nullptr) {
        // set on every launch (a host-side call of about a microsecond): the attribute belongs to the current
        // device, so a process that drives several GPUs needs it on each
        const int sm = (int)sizeof(PFTile<T>);
        const cudaError_t e = cudaFuncSetAttribute(k_pf_tile<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e != cudaSuccess) return e;
        const dim3 grid(n / kTX, n / kTY, n / kZC);
        k_pf_tile<T><<<grid, kTileThreads, sm, s>>>(n, ids, eta, ids2, eta2, g, k, pc, overflow, rcur, rdst);
    } else {
        k_pf<T><<<(int)((N3 + kPF - 1) / kPF), kPF, 0, s>>>(n, ids, eta, ids2, eta2, g, k, pc, overflow);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t pf_soften(long N3, const int32_t *gprev, const int32_t *g, T *rho, double *k, int G, double s_soften,
                      cudaStream_t s) {
    k_pf_soften<T><<<(int)((N3 + 255) / 256), 256, 0, s>>>(N3, gprev, g, rho, k, G, s_soften);
    return cudaGetLastError();
}

int pf_stat_blocks(long N3) { return (int)((N3 + 255) / 256); }

template <typename T>
cudaError_t pf_stats_launch(int n, const int32_t *ids, const T *eta, const int32_t *g, const double *k, PFConst pc,
                     uint32_t *bitmap, int bitmap_words, double *partials, cudaStream_t s) {
    const long N3 = (long)n * n * n;
    const int nb = pf_stat_blocks(N3);
    cudaError_t e = cudaMemsetAsync(bitmap, 0, sizeof(uint32_t) * (size_t)bitmap_words, s);
    if (e != cudaSuccess) return e;
    k_pf_stats<T><<<nb, 256, 0, s>>>(n, ids, eta, g, k, pc, bitmap, bitmap_words, partials);
    // partials layout: [nb][2] energies / rex counts, then one slot for the distinct-id count
    k_popc<<<1, 1024, 0, s>>>(bitmap, bitmap_words, partials + 2 * (long)nb);
    return cudaGetLastError();
}

cudaError_t reduce_partials(const double *partials, int nparts, int nvals, double *out, cudaStream_t s,
                            const int *skip) {
    k_reduce<<<nvals, 1024, 0, s>>>(partials, nparts, nvals, out, skip);
    return cudaGetLastError();
}

cudaError_t pf_interp(int n, const double *k, double *kpf, cudaStream_t s) {
    const long M3 = 8L * n * n * n;
    k_interp_k<<<(int)((M3 + 255) / 256), 256, 0, s>>>(n, k, kpf);
    return cudaGetLastError();
}

template <typename T>
cudaError_t pf_restrict(int n, int K, const int32_t *ids, const T *eta, int32_t *g, cudaStream_t s) {
    if (K > KM || K < 1) return cudaErrorInvalidValue;
    const long N3 = (long)n * n * n;
    k_restrict<T><<<(int)((N3 + 127) / 128), 128, 0, s>>>(n, K, ids, eta, g);
    return cudaGetLastError();
}

cudaError_t pf_init(int n, int r, int K, const int32_t *g0, int32_t *ids, void *eta, int32_t *ids2, void *eta2,
                    int eta_double, int32_t *gpf, cudaStream_t s) {
    const long M3 = (long)r * n * r * n * r * n;
    k_pf_init<<<(int)((M3 + 255) / 256), 256, 0, s>>>(n, r, K, g0, ids, eta, ids2, eta2, eta_double, gpf);
    return cudaGetLastError();
}

template cudaError_t pf_restrict<float>(int, int, const int32_t *, const float *, int32_t *, cudaStream_t);
template cudaError_t pf_restrict<double>(int, int, const int32_t *, const double *, int32_t *, cudaStream_t);
template cudaError_t pf_one_step<float>(int, const int32_t *, const float *, int32_t *, float *, int32_t *,
                                        const double *, PFConst, int32_t *, const uint8_t *, uint8_t *, cudaStream_t);
template cudaError_t pf_one_step<double>(int, const int32_t *, const double *, int32_t *, double *, int32_t *,
                                         const double *, PFConst, int32_t *, const uint8_t *, uint8_t *, cudaStream_t);
template cudaError_t pf_soften<float>(long, const int32_t *, const int32_t *, float *, double *, int, double, cudaStream_t);
template cudaError_t pf_soften<double>(long, const int32_t *, const int32_t *, double *, double *, int, double, cudaStream_t);
template cudaError_t pf_stats_launch<float>(int, const int32_t *, const float *, const int32_t *, const double *, PFConst,
                                     uint32_t *, int, double *, cudaStream_t);
template cudaError_t pf_stats_launch<double>(int, const int32_t *, const double *, const int32_t *, const double *, PFConst,
                                      uint32_t *, int, double *, cudaStream_t);

}  // namespace evp
