// Field solver of the scattered field (Eqs. MAmper, MFaraday; Yee stagger), sm_103a:
// `k_yee` (1D), `k_yee2r` (2D tiles, below) and `k_yee3s` (3D columns streamed along z).
//
// 1D: one work item = one tile of TX x TY x TZ points (compile-time shape).  The tile's box
// (x: 4 points of halo on each side, y/z: 2) of E, B at step n (buffer set p) and of
// J^{n+1/2} (J_p) arrives by two TMA loads.  In shared memory:
//   A. B^{n+1/2} = B^n - (dt/2) curl E^n             (forward differences, in place)
//   B. E^{n+1}   = E^n + dt (curl B^{n+1/2} - J)      (backward differences, into the J slots)
//      except on faces, where
//   C. first-order Mur: E^{n+1}(0) = E^n(1) + (dt-dx)/(dt+dx) (E^{n+1}(1) - E^n(0)), applied along
//      the lowest face axis of the point, points on fewer faces first;
//   D. B^{n+1}   = B^{n+1/2} - (dt/2) curl E^{n+1}    on the tile, points a component does
//      not have (outside [0, n] / [0, n-1]) forced to zero.
// Tiles whose box touches no face (most of them) skip the face tests and phase C.
// The tile of E^{n+1}, B^{n+1} leaves by one TMA store into buffer set 1-p, and J_{1-p}
// (the next step's deposit target) is cleared on the tile.  No CTA writes what another
// reads in the same launch.
#include <cuda_runtime.h>

#include <algorithm>

#include "beam.cuh"
#include "sff_common.cuh"
#include "sff_kernels.h"

namespace sff {

// bitmask of the axes on whose faces E component c at global point g lies
template <int D>
__device__ __forceinline__ int face_axes(const SimDev& S, int c, const int g[3])
{
    int m = 0;
#pragma unroll
    for (int d = 0; d < D; ++d)
        if (d != c && (g[d] == 0 || g[d] == S.n[d])) m |= 1 << d;
    return m;
}

// does field component comp (0..5: Ex..Bz) have a point at global index g?
template <int D>
__device__ __forceinline__ bool has_point(const SimDev& S, int comp, const int g[3])
{
    const int c = comp % 3;
    const bool isE = comp < 3;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const bool stag = isE ? (d == c) : (d != c);
        const int hi = stag ? S.n[d] - 1 : S.n[d];
        if (g[d] < 0 || g[d] > hi) return false;
    }
    return true;
}

// ONE: the launch is one simulation whose descriptor `one` is a kernel parameter (its
// fields come from the constant bank and its tensor maps are used from parameter space,
// with no acquire); otherwise the descriptors are read from the device array `sims`.
template <int D, typename R, int TX, int TY, int TZ, bool ONE>
__device__ __forceinline__ void yee_body(const SimDev* __restrict__ sims, const SimDev& one,
                                         const Work* __restrict__ work, int nwork, int* __restrict__ counter)
{
    constexpr int HX = 4, HY = D > 1 ? 2 : 0, HZ = D > 2 ? 2 : 0;
    constexpr int EX = TX + 2 * HX, EY = TY + 2 * HY, EZ = TZ + 2 * HZ;
    constexpr int SY = EX, SZ = EX * EY, BV = EX * EY * EZ, TV = TX * TY * TZ;
    constexpr size_t JOFF = round128(6 * BV * sizeof(R));
    constexpr size_t BOXB = round128(JOFF + 3 * BV * sizeof(R));   // one box buffer
    constexpr size_t OOFF = 2 * BOXB;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_item;
    const int tid = threadIdx.x;
    constexpr int NT = 256;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    unsigned phases = 0;     // mbarrier phase per buffer
    R* Out = reinterpret_cast<R*>(smem_raw + OOFF);    // [6][TZ][TY][TX]
    // Two box buffers: while a block computes one tile, the TMA loads of its next tile (taken
    // from the work counter one tile ahead) land in the other.
    auto fetch = [&]() {
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        return it;
    };
    auto tile_lo = [&](const SimDev& S, int tile, int lo[3]) {
        int t = tile;
        lo[0] = (t % S.nyt[0]) * TX;
        t /= S.nyt[0];
        lo[1] = lo[2] = 0;
        if constexpr (D > 1) {
            lo[1] = (t % S.nyt[1]) * TY;
            t /= S.nyt[1];
        }
        if constexpr (D > 2) lo[2] = t * TZ;
    };
    int acq_sim = -1;         // thread 0: the simulation whose tensor maps it has acquired
    auto issue = [&](int it, int b) {
        if (tid != 0) return;
        const Work w = work[it];
        const SimDev& S = ONE ? one : sims[w.sim];
        int l[3];
        tile_lo(S, w.tile, l);
        const int o[3] = {l[0] - HX + GX, D > 1 ? l[1] - HY + G : 0, D > 2 ? l[2] - HZ + G : 0};
        const int p = S.st->parity;
        // one acquire per simulation and block (the maps were written before the launch)
        if (!ONE && w.sim != acq_sim) {
            tensormap_acquire(&S.tm_yin);
            tensormap_acquire(&S.tm_yj);
            tensormap_acquire(&S.tm_yout);
            acq_sim = w.sim;
        }
        unsigned char* box = smem_raw + b * BOXB;
        mbar_arrive_expect_tx(&bars[b], (unsigned)(9 * BV * sizeof(R)));
        tma_load_box<D>(box, &S.tm_yin, o, comp_eb(p), &bars[b]);
        tma_load_box<D>(box + JOFF, &S.tm_yj, o, comp_j(p), &bars[b]);
    };
    int item = fetch();
    if (item < nwork) issue(item, 0);
    int buf = 0;
    while (item < nwork) {
        const int next = fetch();
        if (next < nwork) issue(next, buf ^ 1);
        R* In = reinterpret_cast<R*>(smem_raw + buf * BOXB);        // [6][EZ][EY][EX]: Ex Ey Ez Bx By Bz
        R* Jn = reinterpret_cast<R*>(smem_raw + buf * BOXB + JOFF); // [3][EZ][EY][EX]: J, then E^{n+1}
        R* Ex = In;
        R* Ey = In + BV;
        R* Ez = In + 2 * BV;
        R* Bx = In + 3 * BV;
        R* By = In + 4 * BV;
        R* Bz = In + 5 * BV;
        R* Nx = Jn;
        R* Ny = Jn + BV;
        R* Nz = Jn + 2 * BV;
        const Work wk = work[item];
        const SimDev& S = ONE ? one : sims[wk.sim];
        DevState* st = S.st;
        const int par = st->parity;
        int lo[3];
        tile_lo(S, wk.tile, lo);
        // the box reaches global points lo - h .. lo - h + E - 1; phases use 1 .. E - 2
        bool interior = true;
        {
            const int h[3] = {HX, HY, HZ};
            const int e[3] = {EX, EY, EZ};
#pragma unroll
            for (int d = 0; d < D; ++d)
                if (lo[d] - h[d] + 1 <= 0 || lo[d] - h[d] + e[d] - 2 >= S.n[d]) interior = false;
        }
        const YeeC<R>& yc = yee_of<R>(S);
        const R cdt = yc.cdt, hc = yc.hc, dt = yc.dt, km = yc.km;
        const bool ok = mbar_wait_bounded(&bars[buf], (phases >> buf) & 1u);
        phases ^= 1u << buf;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(&st->status, (unsigned)FLAG_TIMEOUT);
                // let the loads still in flight (this tile's, and the next one's) land
                if (!ok) mbar_wait_bounded(&bars[buf], ((phases >> buf) & 1u) ^ 1u);
                if (next < nwork) mbar_wait_bounded(&bars[buf ^ 1], (phases >> (buf ^ 1)) & 1u);
                bulk_wait0();
            }
            return;
        }

        // A. B^{n+1/2} in place, points 0 .. E-2 on every resolved axis
        for (int i = tid; i < BV; i += NT) {
            const int lx = i % EX, ly = (i / EX) % EY, lz = i / SZ;
            if (lx >= EX - 1) continue;
            if (D > 1 && ly >= EY - 1) continue;
            if (D > 2 && lz >= EZ - 1) continue;
            const R dEz_dy = D > 1 ? Ez[i + SY] - Ez[i] : R(0);
            const R dEx_dy = D > 1 ? Ex[i + SY] - Ex[i] : R(0);
            const R dEy_dz = D > 2 ? Ey[i + SZ] - Ey[i] : R(0);
            const R dEx_dz = D > 2 ? Ex[i + SZ] - Ex[i] : R(0);
            const R dEz_dx = Ez[i + 1] - Ez[i];
            const R dEy_dx = Ey[i + 1] - Ey[i];
            Bx[i] -= hc * (dEz_dy - dEy_dz);
            By[i] -= hc * (dEx_dz - dEz_dx);
            Bz[i] -= hc * (dEy_dx - dEx_dy);
        }
        __syncthreads();

        // B. E^{n+1} into the J slots at points 1 .. E-2 on every resolved axis, off the faces
        for (int i = tid; i < BV; i += NT) {
            const int lx = i % EX, ly = (i / EX) % EY, lz = i / SZ;
            if (lx < 1 || lx >= EX - 1) continue;
            if (D > 1 && (ly < 1 || ly >= EY - 1)) continue;
            if (D > 2 && (lz < 1 || lz >= EZ - 1)) continue;
            const R dBz_dy = D > 1 ? Bz[i] - Bz[i - SY] : R(0);
            const R dBx_dy = D > 1 ? Bx[i] - Bx[i - SY] : R(0);
            const R dBy_dz = D > 2 ? By[i] - By[i - SZ] : R(0);
            const R dBx_dz = D > 2 ? Bx[i] - Bx[i - SZ] : R(0);
            const R dBz_dx = Bz[i] - Bz[i - 1];
            const R dBy_dx = By[i] - By[i - 1];
            const R ex = Ex[i] + cdt * (dBz_dy - dBy_dz) - dt * Nx[i];
            const R ey = Ey[i] + cdt * (dBx_dz - dBz_dx) - dt * Ny[i];
            const R ez = Ez[i] + cdt * (dBy_dx - dBx_dy) - dt * Nz[i];
            if (interior) {
                Nx[i] = ex;
                Ny[i] = ey;
                Nz[i] = ez;
            } else {
                const int g[3] = {lo[0] - HX + lx, lo[1] - HY + ly, lo[2] - HZ + lz};
                if (!face_axes<D>(S, 0, g)) Nx[i] = ex;
                if (!face_axes<D>(S, 1, g)) Ny[i] = ey;
                if (!face_axes<D>(S, 2, g)) Nz[i] = ez;
            }
        }
        __syncthreads();

        // C. Mur faces (tiles touching a face only): one face first, then edges, then corners
        if (!interior) {
            const int es[3] = {1, SY, SZ};
            const int e[3] = {EX, EY, EZ};
            for (int pass = 1; pass <= D; ++pass) {
                for (int i = tid; i < BV; i += NT) {
                    const int l[3] = {i % EX, (i / EX) % EY, i / SZ};
                    if (l[0] < 1 || l[0] >= EX - 1) continue;
                    if (D > 1 && (l[1] < 1 || l[1] >= EY - 1)) continue;
                    if (D > 2 && (l[2] < 1 || l[2] >= EZ - 1)) continue;
                    const int g[3] = {lo[0] - HX + l[0], lo[1] - HY + l[1], lo[2] - HZ + l[2]};
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const int m = face_axes<D>(S, c, g);
                        if (!m || __popc(m) != pass) continue;
                        const int a = __ffs(m) - 1;
                        const int dir = (g[a] == 0) ? 1 : -1;
                        const int ln = l[a] + dir;
                        if (ln < 1 || ln >= e[a] - 1) continue;
                        const int nb = i + dir * es[a];
                        const R* Eo = In + c * BV;
                        R* En = Jn + c * BV;
                        if constexpr (D == 1) {
                            if (S.tf && g[0] == 0) {
                                // total-field run: the condition acts on E - E_inc, so the
                                // plane wave (nodes x = 0 and dx, times t^n and t^{n+1}) enters
                                R inc[2][2];
                                const BeamC<R>& bcs = beam_of<R>(S);
#pragma unroll
                                for (int k = 0; k < 2; ++k) {
                                    const PhaseRef<R> pr = phase_ref<R>(S, (double)(st->step + k) * S.dt, 0);
#pragma unroll
                                    for (int node = 0; node < 2; ++node) {
                                        const int cc[3] = {node, 0, 0};
                                        const R oo[3] = {R(0), R(0), R(0)};
                                        R Ei[3], Bi[3];
                                        incident_at<1, R>(S, bcs, pr, cc, oo, Ei, Bi);
                                        inc[k][node] = Ei[c];
                                    }
                                }
                                En[i] = inc[1][0] + (Eo[nb] - inc[0][1]) +
                                        km * ((En[nb] - inc[1][1]) - (Eo[i] - inc[0][0]));
                                continue;
                            }
                        }
                        En[i] = Eo[nb] + km * (En[nb] - Eo[i]);
                    }
                }
                __syncthreads();
            }
        }

        // D. E^{n+1}, B^{n+1} on the tile
        for (int k = tid; k < TV; k += NT) {
            const int t0 = k % TX, t1 = (k / TX) % TY, t2 = k / (TX * TY);
            const int i = (t0 + HX) + (t1 + HY) * SY + (t2 + HZ) * SZ;
            const R dNz_dy = D > 1 ? Nz[i + SY] - Nz[i] : R(0);
            const R dNx_dy = D > 1 ? Nx[i + SY] - Nx[i] : R(0);
            const R dNy_dz = D > 2 ? Ny[i + SZ] - Ny[i] : R(0);
            const R dNx_dz = D > 2 ? Nx[i + SZ] - Nx[i] : R(0);
            const R dNz_dx = Nz[i + 1] - Nz[i];
            const R dNy_dx = Ny[i + 1] - Ny[i];
            const R v[6] = {Nx[i], Ny[i], Nz[i], Bx[i] - hc * (dNz_dy - dNy_dz), By[i] - hc * (dNx_dz - dNz_dx),
                            Bz[i] - hc * (dNy_dx - dNx_dy)};
            if (interior) {
#pragma unroll
                for (int c = 0; c < 6; ++c) Out[c * TV + k] = v[c];
            } else {
                const int g[3] = {lo[0] + t0, lo[1] + t1, lo[2] + t2};
#pragma unroll
                for (int c = 0; c < 6; ++c) Out[c * TV + k] = has_point<D>(S, c, g) ? v[c] : R(0);
            }
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            const int oc[3] = {lo[0] + GX, D > 1 ? lo[1] + G : 0, D > 2 ? lo[2] + G : 0};
            tma_store_box<D>(&S.tm_yout, oc, comp_eb(1 - par), Out);
            bulk_commit();
        }
        // clear J_{1-p} on the tile (the next step deposits into it)
        {
            R* Fg = reinterpret_cast<R*>(S.F);
            const long long jb = (long long)comp_j(1 - par) * S.sc;
            for (int k = tid; k < 3 * TV; k += NT) {
                const int c = k / TV, r = k - c * TV;
                const int t0 = r % TX, t1 = (r / TX) % TY, t2 = r / (TX * TY);
                Fg[jb + c * S.sc + (long long)(D > 2 ? lo[2] + t2 + G : 0) * S.sz +
                   (long long)(D > 1 ? lo[1] + t1 + G : 0) * S.sy + (lo[0] + t0 + GX)] = R(0);
            }
        }
        if (tid == 0) bulk_wait_read0();
        // this buffer was written by the phases above; the TMA load of the tile after next
        // reuses it (generic-proxy writes before async-proxy writes to the same memory)
        fence_proxy_async_smem();
        __syncthreads();
        item = next;
        buf ^= 1;
    }
    if (tid == 0) bulk_wait0();
}

template <int D, typename R, int TX, int TY, int TZ>
__global__ void __launch_bounds__(256) k_yee(const SimDev* __restrict__ sims, const Work* __restrict__ work,
                                             int nwork, int* __restrict__ counter)
{
    yee_body<D, R, TX, TY, TZ, false>(sims, *sims, work, nwork, counter);
}

template <int D, typename R, int TX, int TY, int TZ>
__global__ void __launch_bounds__(256) k_yee1(const __grid_constant__ SimDev one, const Work* __restrict__ work,
                                              int nwork, int* __restrict__ counter)
{
    yee_body<D, R, TX, TY, TZ, true>(nullptr, one, work, nwork, counter);
}

// ---------------------------------------------------------------------------------
// 2D: one tile of PX x PY points per work item; its box (x: 4 points of halo on each side,
// y: 2 below and 2 above) of E, B and J_p arrives by two TMA loads into one of two
// buffers (the next tile's loads are in flight while this one is updated).  Phases, each
// on the thread's own point of the box (fixed for the launch):
//   A: Bh = B^{n+1/2}  for x in [x0-2, x0+PX], y in [y0-2, y0+PY]   (forward differences)
//   B: N  = E^{n+1}    for x in [x0-1, x0+PX], y in [y0-1, y0+PY]   (backward differences),
//      with the first-order Mur condition on the x / y faces evaluated from the inward
//      neighbour's E^{n+1} by the face point's own thread (for E_z on a corner, the
//      neighbour's neighbour too), so no extra passes or barriers
//   D: B^{n+1} on the tile from Bh and N (forward differences); E^{n+1}, B^{n+1} leave by
//      one TMA store and J_{1-p} is cleared; a tile that ends at x = n_x (y = n_y) also
//      writes that node line with plain stores (no work item holds only the node line).
// Warp w < AH holds box row w, x = 4 .. PX+3 (32 consecutive words: no bank conflicts);
// the last warps hold the rest of the Bh range (x = 2, 3 and PX+4).
// ---------------------------------------------------------------------------------
template <typename R, int PY, int NT, bool ONE>
__device__ __forceinline__ void yee2r_body(const SimDev* __restrict__ sims, const SimDev& one,
                                           const Work* __restrict__ work, int nwork, int* __restrict__ counter)
{
    constexpr int PX = 32;
    constexpr int BX = PX + 8, BY = PY + 4, BV = BX * BY, TV = PX * PY;
    constexpr size_t JOFF = round128(6 * BV * sizeof(R));
    constexpr size_t BOXB = round128(JOFF + 3 * BV * sizeof(R));   // one box buffer
    constexpr size_t HOFF = 2 * BOXB;                              // Bh [3][BV]
    constexpr size_t NOFF = HOFF + round128(3 * BV * sizeof(R));   // N  [3][BV]
    constexpr size_t OOFF = NOFF + round128(3 * BV * sizeof(R));   // Out [6][PY][PX]
    constexpr int AH = PY + 3;                   // Bh rows 0 .. PY+2
    constexpr int NE = 3 * PY + 8;               // Bh points off the core rows
    static_assert(NT == 32 * (AH + (NE + 31) / 32), "one warp per row of 32 points, plus the rest");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_item;
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    unsigned phases = 0;     // mbarrier phase per buffer
    R* Hb = reinterpret_cast<R*>(smem_raw + HOFF);
    R* Nb = reinterpret_cast<R*>(smem_raw + NOFF);
    R* Out = reinterpret_cast<R*>(smem_raw + OOFF);
    // the thread's point: box index, output slot, whether it is in the N range
    int pi, po;
    bool pN;
    {
        const int w = tid >> 5, lane = tid & 31;
        int lx = 4 + lane, ly = w;
        bool has = true;
        if (w >= AH) {
            const int e = lane + 32 * (w - AH);
            has = e < NE;
            if (e < PY + 2) {
                lx = 2;
                ly = 1 + e;
            } else if (e < 2 * PY + 5) {
                lx = 3;
                ly = e - (PY + 2);
            } else {
                lx = PX + 4;
                ly = e - (2 * PY + 5);
            }
        }
        pi = has ? lx + BX * ly : -1;
        pN = has && lx >= 3 && ly >= 1;
        po = (has && lx >= 4 && lx < PX + 4 && ly >= 2 && ly < PY + 2) ? (lx - 4) + PX * (ly - 2) : -1;
    }
    auto fetch = [&]() {
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        return it;
    };
    int acq_sim = -1;         // thread 0: the simulation whose tensor maps it has acquired
    auto issue = [&](int it, int b) {
        if (tid != 0) return;
        const Work w = work[it];
        const SimDev& S = ONE ? one : sims[w.sim];
        const int t = w.tile;
        const int o[3] = {(t % S.nyt[0]) * PX - 4 + GX, (t / S.nyt[0]) * PY - 2 + G, 0};
        const int p = S.st->parity;
        if (!ONE && w.sim != acq_sim) {
            tensormap_acquire(&S.tm_yin);
            tensormap_acquire(&S.tm_yj);
            tensormap_acquire(&S.tm_yout);
            acq_sim = w.sim;
        }
        unsigned char* box = smem_raw + b * BOXB;
        mbar_arrive_expect_tx(&bars[b], (unsigned)(9 * BV * sizeof(R)));
        tma_load_box<2>(box, &S.tm_yin, o, comp_eb(p), &bars[b]);
        tma_load_box<2>(box + JOFF, &S.tm_yj, o, comp_j(p), &bars[b]);
    };
    int item = fetch();
    if (item < nwork) issue(item, 0);
    int buf = 0;
    while (item < nwork) {
        const int next = fetch();
        if (next < nwork) issue(next, buf ^ 1);
        const R* I0 = reinterpret_cast<const R*>(smem_raw + buf * BOXB);           // Ex Ey Ez Bx By Bz
        const R* J0 = reinterpret_cast<const R*>(smem_raw + buf * BOXB + JOFF);    // Jx Jy Jz
        const Work wk = work[item];
        const SimDev& S = ONE ? one : sims[wk.sim];
        DevState* st = S.st;
        const int par = st->parity;
        const int n0 = S.n[0], n1 = S.n[1];
        const int x0 = (wk.tile % S.nyt[0]) * PX, y0 = (wk.tile / S.nyt[0]) * PY;
        const bool interior = x0 > 0 && x0 + PX < n0 && y0 > 0 && y0 + PY < n1;
        const bool xend = x0 + PX == n0, yend = y0 + PY == n1;
        const YeeC<R>& yc = yee_of<R>(S);
        const R cdt = yc.cdt, hc = yc.hc, dt = yc.dt, km = yc.km;
        // the point's faces and validity (bits as in the 3D kernel), and whether it is an
        // output on the node line past the tile
        unsigned f = 0;
        if (pi >= 0) {
            const int gx = x0 - 4 + pi % BX, gy = y0 - 2 + pi / BX;
            const bool past = (xend && gx == n0 && gy >= y0 && gy <= y0 + PY - (yend ? 0 : 1)) ||
                              (yend && gy == n1 && gx >= x0 && gx <= x0 + PX - (xend ? 0 : 1));
            f = (gx == 0 || gx == n0 ? 1u : 0u) | (gy == 0 || gy == n1 ? 2u : 0u) |
                (gx >= 0 && gx <= n0 - 1 ? 4u : 0u) | (gx >= 0 && gx <= n0 ? 8u : 0u) |
                (gy >= 0 && gy <= n1 - 1 ? 16u : 0u) | (gy >= 0 && gy <= n1 ? 32u : 0u) |
                (gx == 0 ? 64u : 0u) | (gy == 0 ? 128u : 0u) | (past ? 256u : 0u);
        }
        const bool ok = mbar_wait_bounded(&bars[buf], (phases >> buf) & 1u);
        phases ^= 1u << buf;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(&st->status, (unsigned)FLAG_TIMEOUT);
                // let the loads still in flight (this tile's, and the next one's) land
                if (!ok) mbar_wait_bounded(&bars[buf], ((phases >> buf) & 1u) ^ 1u);
                if (next < nwork) mbar_wait_bounded(&bars[buf ^ 1], (phases >> (buf ^ 1)) & 1u);
                bulk_wait0();
            }
            return;
        }
        // A: B^{n+1/2} on the Bh range
        if (pi >= 0) {
            const int i = pi;
            const R dEz_dy = I0[2 * BV + i + BX] - I0[2 * BV + i];
            const R dEx_dy = I0[i + BX] - I0[i];
            const R dEz_dx = I0[2 * BV + i + 1] - I0[2 * BV + i];
            const R dEy_dx = I0[BV + i + 1] - I0[BV + i];
            Hb[i] = I0[3 * BV + i] - hc * (dEz_dy - R(0));
            Hb[BV + i] = I0[4 * BV + i] - hc * (R(0) - dEz_dx);
            Hb[2 * BV + i] = I0[5 * BV + i] - hc * (dEy_dx - dEx_dy);
        }
        __syncthreads();
        // B: E^{n+1} on the N range, the Mur condition on the faces
        if (pN) {
            const int i = pi;
            auto enew = [&](int c, int j) -> R {
                if (c == 0) return I0[j] + cdt * ((Hb[2 * BV + j] - Hb[2 * BV + j - BX]) - R(0)) - dt * J0[j];
                if (c == 1) return I0[BV + j] + cdt * (R(0) - (Hb[2 * BV + j] - Hb[2 * BV + j - 1])) - dt * J0[BV + j];
                return I0[2 * BV + j] + cdt * ((Hb[BV + j] - Hb[BV + j - 1]) - (Hb[j] - Hb[j - BX])) - dt * J0[2 * BV + j];
            };
            auto mur = [&](int c, int j, int nb, R en_nb) -> R { return I0[c * BV + nb] + km * (en_nb - I0[c * BV + j]); };
            const bool fx = f & 1u, fy = f & 2u;
            if (interior || (!fx && !fy)) {
                Nb[i] = enew(0, i);
                Nb[BV + i] = enew(1, i);
                Nb[2 * BV + i] = enew(2, i);
            } else {
                const int sx = (f & 64u) ? 1 : -1, sy = (f & 128u) ? BX : -BX;
                Nb[i] = fy ? mur(0, i, i + sy, enew(0, i + sy)) : enew(0, i);
                Nb[BV + i] = fx ? mur(1, i, i + sx, enew(1, i + sx)) : enew(1, i);
                R vz;
                if (fx && fy) {
                    const int nb = i + sx;
                    vz = mur(2, i, nb, mur(2, nb, nb + sy, enew(2, nb + sy)));
                } else if (fx) {
                    vz = mur(2, i, i + sx, enew(2, i + sx));
                } else {
                    vz = mur(2, i, i + sy, enew(2, i + sy));
                }
                Nb[2 * BV + i] = vz;
            }
        }
        // the previous tile's store has read the output buffer that D rewrites
        if (tid == 0) bulk_wait_read0();
        __syncthreads();
        // D: E^{n+1}, B^{n+1} on the tile (and the node line past it)
        if (pi >= 0 && (po >= 0 || (f & 256u))) {
            const int i = pi;
            const R dNz_dy = Nb[2 * BV + i + BX] - Nb[2 * BV + i];
            const R dNx_dy = Nb[i + BX] - Nb[i];
            const R dNz_dx = Nb[2 * BV + i + 1] - Nb[2 * BV + i];
            const R dNy_dx = Nb[BV + i + 1] - Nb[BV + i];
            R v[6] = {Nb[i], Nb[BV + i], Nb[2 * BV + i], Hb[i] - hc * (dNz_dy - R(0)),
                      Hb[BV + i] - hc * (R(0) - dNz_dx), Hb[2 * BV + i] - hc * (dNy_dx - dNx_dy)};
            if (!interior) {
                const bool xs = f & 4u, xn = f & 8u, ys = f & 16u, yn = f & 32u;
                if (!(xs && yn)) v[0] = R(0);
                if (!(xn && ys)) v[1] = R(0);
                if (!(xn && yn)) v[2] = R(0);
                if (!(xn && ys)) v[3] = R(0);
                if (!(xs && yn)) v[4] = R(0);
                if (!(xs && ys)) v[5] = R(0);
            }
            const int gx = x0 - 4 + i % BX, gy = y0 - 2 + i / BX;
            R* jp = reinterpret_cast<R*>(S.F) + (long long)comp_j(1 - par) * S.sc + (long long)(gy + G) * S.sy + (gx + GX);
            if (po >= 0) {
#pragma unroll
                for (int c = 0; c < 6; ++c) Out[c * TV + po] = v[c];
            } else {
                R* ep = jp + (long long)(comp_eb(1 - par) - comp_j(1 - par)) * S.sc;
#pragma unroll
                for (int c = 0; c < 6; ++c) ep[c * S.sc] = v[c];
            }
            // clear J_{1-p} (the next step deposits into it)
            jp[0] = R(0);
            jp[S.sc] = R(0);
            jp[2 * S.sc] = R(0);
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            const int oc[3] = {x0 + GX, y0 + G, 0};
            tma_store_box<2>(&S.tm_yout, oc, comp_eb(1 - par), Out);
            bulk_commit();
        }
        // this box buffer takes the tile after next: its reads above are behind the barrier
        item = next;
        buf ^= 1;
    }
    if (tid == 0) bulk_wait0();
}

template <typename R, int PY, int NT>
__global__ void __launch_bounds__(NT, 2) k_yee2r(const SimDev* __restrict__ sims, const Work* __restrict__ work,
                                                 int nwork, int* __restrict__ counter)
{
    yee2r_body<R, PY, NT, false>(sims, *sims, work, nwork, counter);
}

template <typename R, int PY, int NT>
__global__ void __launch_bounds__(NT, 2) k_yee2r1(const __grid_constant__ SimDev one, const Work* __restrict__ work,
                                                  int nwork, int* __restrict__ counter)
{
    yee2r_body<R, PY, NT, true>(nullptr, one, work, nwork, counter);
}

// ---------------------------------------------------------------------------------
// 3D: a work item is a column of PX x PY points (x, y) over a segment [z0, z1) of planes.
// The column marches along z; plane k of E, B and J_p (box x: 4 points of halo on each
// side, y: 2 below and 1 above) arrives by TMA into a ring of NS stages.  With
//   A(k): Bh = B^{n+1/2} on plane k     (forward differences; planes k, k+1)
//   B(k): N  = E^{n+1}   on plane k     (backward differences; Bh of planes k, k-1), the
//         Mur condition on its x / y faces from the inward neighbour's E^{n+1} evaluated
//         by the face point's own thread; on the z faces (planes 0, n_z) separate passes
//         (plane 0 once N(1) exists)
//   D(k): B^{n+1} on plane k from Bh(k), N(k), N(k+1); E^{n+1}, B^{n+1} of plane k leave
//         by one TMA store (double-buffered) and J_{1-p} of plane k is cleared; a column
//         that ends at x = n_x (y = n_y) also writes that node plane with plain stores,
// iteration q runs A(q+1) together with D(q-1), then B(q+1): two barriers per plane.
// Bh is kept for x in [x0-2, x0+PX], y in [y0-2, y0+PY] and planes from z0-1; N for x in
// [x0-1, x0+PX], y in [y0-1, y0+PY] and planes from z0: one more point than the outputs need
// on the low side in x and y, so that every face point's Mur neighbour (one point inwards)
// is on hand.
// ---------------------------------------------------------------------------------
template <typename R, int PX, int PY, int NS, int NT, bool ONE>
__device__ __forceinline__ void yee3s_body(const SimDev* __restrict__ sims, const SimDev& one,
                                           const Work* __restrict__ work, int nwork, int* __restrict__ counter)
{
    constexpr int TV = PX * PY;
    constexpr int BX = PX + 8, BY = PY + 4, BV = BX * BY;
    constexpr size_t STAGE = round128(9 * BV * sizeof(R));
    constexpr size_t JOFF = round128(6 * BV * sizeof(R));
    constexpr size_t HOFF = NS * STAGE;
    constexpr size_t NOFF = HOFF + round128(9 * BV * sizeof(R));
    constexpr size_t OOFF = NOFF + round128(6 * BV * sizeof(R));
    constexpr int AH = PY + 3;                   // Bh range: box x 2 .. PX+4, y 0 .. PY+2
    constexpr int NW = PX + 2, NH = PY + 2;      // N range:  box x 3 .. PX+4, y 1 .. PY+2
    constexpr int NE = 3 * PY + 8;               // Bh points off the core rows (see below)
    constexpr int NR = 1;                        // Bh points per thread
    static_assert(PX == 32 && NT == 32 * (AH + (NE + 31) / 32), "one warp per row of 32 points, plus the rest");
    static_assert((NS & (NS - 1)) == 0, "a ring of a power-of-two number of stages");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bars[NS];
    __shared__ int s_item;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int k = 0; k < NS; ++k) mbar_init(&bars[k], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto In = [&](int stage) { return reinterpret_cast<R*>(smem_raw + stage * STAGE); };   // [9][BY][BX]
    R* Hr = reinterpret_cast<R*>(smem_raw + HOFF);     // [3][3][BY][BX]  Bh ring
    R* Nr = reinterpret_cast<R*>(smem_raw + NOFF);     // [2][3][BY][BX]  N ring
    R* Outb = reinterpret_cast<R*>(smem_raw + OOFF);   // [2][6][PY][PX]
    // Every phase of a plane works on the thread's own point of the Bh range: Bh on all of
    // them, N on those in the N range, the outputs (box x 4 .. PX+3, y 2 .. PY+1) on those in
    // the tile.  Warp w < AH holds row y = w, x = 4 .. 35 (32 consecutive box points: no bank
    // conflicts in any phase); the last warp holds the rest of the range, x = 2 (y >= 1: Bh
    // at (2, 0) feeds nothing), x = 3 and x = PX+4.  Box indices and output slots are fixed
    // for the launch.
    int pidx[NR], pout[NR];
    bool pN[NR];
    {
        const int w = tid >> 5, lane = tid & 31;
        int lx = 4 + lane, ly = w;
        bool has = true;
        if (w >= AH) {
            const int e = lane + 32 * (w - AH);
            has = e < NE;
            if (e < PY + 2) {
                lx = 2;
                ly = 1 + e;
            } else if (e < 2 * PY + 5) {
                lx = 3;
                ly = e - (PY + 2);
            } else {
                lx = PX + 4;
                ly = e - (2 * PY + 5);
            }
        }
        pidx[0] = has ? lx + BX * ly : -1;
        pN[0] = has && lx >= 3 && ly >= 1;
        pout[0] = (has && lx >= 4 && lx < PX + 4 && ly >= 2 && ly < PY + 2) ? (lx - 4) + PX * (ly - 2) : -1;
    }
    uint32_t ph = 0;      // mbarrier phase of each stage
    int oslot = 0;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= nwork) break;
        const Work wk = work[item];
        const SimDev& S = ONE ? one : sims[wk.sim];
        DevState* st = S.st;
        const int par = st->parity;
        const int n0 = S.n[0], n1 = S.n[1], n2 = S.n[2];
        int t = wk.tile;
        const int cx = t % S.nyt[0];
        t /= S.nyt[0];
        const int cy = t % S.nyt[1];
        const int cz = t / S.nyt[1];
        const int x0 = cx * PX, y0 = cy * PY;
        const int z0 = cz * S.yt[2];
        const int z1 = min(z0 + S.yt[2], n2 + 1);
        // planes loaded: from z0-1 (Bh(z0-1) enters N(z0)) to z1+1 (E(z1+1) enters Bh(z1))
        const int pa = z0 - 1, plast = z1 + 1;
        const bool col_int = x0 > 0 && x0 + PX < n0 && y0 > 0 && y0 + PY < n1;
        const YeeC<R>& yc = yee_of<R>(S);
        const R cdt = yc.cdt, hc = yc.hc, dt = yc.dt, km = yc.km;
        const long long sz = S.sz, sc = S.sc;
        // per point of the column: bit 0 x on a face (0 or n_x), 1 y on a face, 2 x in
        // [0, n_x - 1], 3 x in [0, n_x], 4 y in [0, n_y - 1], 5 y in [0, n_y], 6 x = 0,
        // 7 y = 0, 8 an output past the tile: the column ends at x = n_x (y = n_y) and no
        // column starts there, so this one also writes the node plane x = n_x (y = n_y);
        // and the point's J_{1-p} (cleared for the next step's deposit) on plane -G
        const bool xend = x0 + PX == n0, yend = y0 + PY == n1;
        unsigned pm[NR];
        R* jrow[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int gx = x0 - 4 + pidx[r] % BX, gy = y0 - 2 + pidx[r] / BX;
            const bool past = (xend && gx == n0 && gy >= y0 && gy <= y0 + PY - (yend ? 0 : 1)) ||
                              (yend && gy == n1 && gx >= x0 && gx <= x0 + PX - (xend ? 0 : 1));
            pm[r] = (gx == 0 || gx == n0 ? 1u : 0u) | (gy == 0 || gy == n1 ? 2u : 0u) |
                    (gx >= 0 && gx <= n0 - 1 ? 4u : 0u) | (gx >= 0 && gx <= n0 ? 8u : 0u) |
                    (gy >= 0 && gy <= n1 - 1 ? 16u : 0u) | (gy >= 0 && gy <= n1 ? 32u : 0u) |
                    (gx == 0 ? 64u : 0u) | (gy == 0 ? 128u : 0u) | (past ? 256u : 0u);
            jrow[r] = reinterpret_cast<R*>(S.F) + (long long)comp_j(1 - par) * sc + (long long)(gy + G) * S.sy +
                      (gx + GX);
        }
        auto stage_of = [&](int p) { return (p - pa) & (NS - 1); };
        auto Hs = [&](int p) { return Hr + ((p - pa) % 3) * 3 * BV; };
        auto Ns = [&](int p) { return Nr + ((p - pa) & 1) * 3 * BV; };
        auto issue = [&](int p) {
            const int sgi = stage_of(p);
            const int org[3] = {x0 - 4 + GX, y0 - 2 + G, p + G};
            mbar_arrive_expect_tx(&bars[sgi], (unsigned)(9 * BV * sizeof(R)));
            tma_load_box<3>(In(sgi), &S.tm_yin, org, comp_eb(par), &bars[sgi]);
            tma_load_box<3>(reinterpret_cast<unsigned char*>(In(sgi)) + JOFF, &S.tm_yj, org, comp_j(par), &bars[sgi]);
        };
        if (tid == 0) {
            if (!ONE) {
                tensormap_acquire(&S.tm_yin);
                tensormap_acquire(&S.tm_yj);
                tensormap_acquire(&S.tm_yout);
            }
            for (int p = pa; p <= min(pa + NS - 1, plast); ++p) issue(p);
        }
        int pissued = min(pa + NS - 1, plast);
        int pw = pa - 1;      // last plane waited for
        // Mur faces of plane m (every point of the N range on a face, fewer faces first).
        // Off the z faces only the lines x = 0, n_x and y = 0, n_y of the column are visited
        // (a point on two lines is written twice, with the same value).
        auto mur_plane = [&](int m) {
            const R* Im = In(stage_of(m));
            R* Nm = Ns(m);
            int fx[2], fy[2], nfx = 0, nfy = 0;
            if (4 - x0 >= 3) fx[nfx++] = 4 - x0;
            if (S.n[0] - x0 + 4 <= PX + 4) fx[nfx++] = S.n[0] - x0 + 4;
            if (2 - y0 >= 1) fy[nfy++] = 2 - y0;
            if (S.n[1] - y0 + 2 <= PY + 2) fy[nfy++] = S.n[1] - y0 + 2;
            const bool zf = m == 0 || m == S.n[2];
            const int npass = (nfx > 0) + (nfy > 0) + (zf ? 1 : 0);
            const int ncand = zf ? NW * NH : nfx * NH + nfy * NW;
            for (int pass = 1; pass <= npass; ++pass) {
                for (int k = tid; k < ncand; k += NT) {
                    int lx, ly;
                    if (zf) {
                        lx = 3 + k % NW;
                        ly = 1 + k / NW;
                    } else if (k < nfx * NH) {
                        lx = fx[k / NH];
                        ly = 1 + k % NH;
                    } else {
                        const int r = k - nfx * NH;
                        ly = fy[r / NW];
                        lx = 3 + r % NW;
                    }
                    const int i = lx + BX * ly;
                    const int g[3] = {x0 - 4 + lx, y0 - 2 + ly, m};
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const int fm = face_axes<3>(S, c, g);
                        if (!fm || __popc(fm) != pass) continue;
                        const int a = __ffs(fm) - 1;
                        const int dir = (g[a] == 0) ? 1 : -1;
                        R eo_nb, en_nb;
                        if (a < 2) {
                            const int nb = i + dir * (a == 0 ? 1 : BX);
                            eo_nb = Im[c * BV + nb];
                            en_nb = Nm[c * BV + nb];
                        } else {
                            eo_nb = In(stage_of(m + dir))[c * BV + i];
                            en_nb = Ns(m + dir)[c * BV + i];
                        }
                        Nm[c * BV + i] = eo_nb + km * (en_nb - Im[c * BV + i]);
                    }
                }
                __syncthreads();
            }
        };


        bool failed = false;
        for (int q = z0 - 2; q <= z1; ++q) {
            // Plane q was last read in the previous iteration unless this one's z-face passes
            // read it (B(n_z) reads E(n_z - 1), the plane-0 faces E(0)): otherwise its stage
            // takes plane q+NS as soon as this iteration's first barrier has passed
            const bool early = q + 1 != n2 && q + 1 != 1;
            bool ok = true;
            while (pw < min(q + 2, plast)) {
                ++pw;
                const int sgi = stage_of(pw);
                ok = ok && mbar_wait_bounded(&bars[sgi], (ph >> sgi) & 1u);
                ph ^= 1u << sgi;
            }
            // S1: A(q+1) and D(q-1) on the thread's points
            const bool doA = q + 1 <= z1, doD = q - 1 >= z0;
            if (doA || doD) {
                const int m = q - 1;
                const R* I0 = In(stage_of(q + 1));
                const R* I1 = In(stage_of(q + 2));
                R* Ha = doA ? Hs(q + 1) : Hr;
                const R* H0 = doD ? Hs(m) : Hr;
                const R* N0 = Ns(m + 2);
                const R* N1 = Ns(m + 1);
                R* Out = Outb + oslot * 6 * TV;
                // every output point of the plane has all six components
                const bool zint = col_int && m >= 1 && m <= n2 - 1;
                const bool zs = m >= 0 && m <= n2 - 1, zn = m >= 0 && m <= n2;
                const long long zoff = (long long)(m + G) * sz;
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const int i = pidx[r];
                    if (i < 0) continue;
                    if (doD && (pout[r] >= 0 || (pm[r] & 256u))) {
                        const R dNz_dy = N0[2 * BV + i + BX] - N0[2 * BV + i];
                        const R dNx_dy = N0[i + BX] - N0[i];
                        const R dNy_dz = N1[BV + i] - N0[BV + i];
                        const R dNx_dz = N1[i] - N0[i];
                        const R dNz_dx = N0[2 * BV + i + 1] - N0[2 * BV + i];
                        const R dNy_dx = N0[BV + i + 1] - N0[BV + i];
                        R v[6] = {N0[i], N0[BV + i], N0[2 * BV + i], H0[i] - hc * (dNz_dy - dNy_dz),
                                  H0[BV + i] - hc * (dNx_dz - dNz_dx), H0[2 * BV + i] - hc * (dNy_dx - dNx_dy)};
                        if (!zint) {
                            const unsigned b = pm[r];
                            const bool xs = b & 4u, xn = b & 8u, ys = b & 16u, yn = b & 32u;
                            if (!(xs && yn && zn)) v[0] = R(0);
                            if (!(xn && ys && zn)) v[1] = R(0);
                            if (!(xn && yn && zs)) v[2] = R(0);
                            if (!(xn && ys && zs)) v[3] = R(0);
                            if (!(xs && yn && zs)) v[4] = R(0);
                            if (!(xs && ys && zn)) v[5] = R(0);
                        }
                        const int u = pout[r];
                        R* jp = jrow[r] + zoff;
                        if (u >= 0) {
#pragma unroll
                            for (int c = 0; c < 6; ++c) Out[c * TV + u] = v[c];
                        } else {
                            // past the tile (node plane x = n_x / y = n_y): plain stores
                            R* ep = jp + (long long)(comp_eb(1 - par) - comp_j(1 - par)) * sc;
#pragma unroll
                            for (int c = 0; c < 6; ++c) ep[c * sc] = v[c];
                        }
                        // clear J_{1-p} on plane m (the next step deposits into it)
                        jp[0] = R(0);
                        jp[sc] = R(0);
                        jp[2 * sc] = R(0);
                    }
                    if (doA) {
                        const R dEz_dy = I0[2 * BV + i + BX] - I0[2 * BV + i];
                        const R dEx_dy = I0[i + BX] - I0[i];
                        const R dEy_dz = I1[BV + i] - I0[BV + i];
                        const R dEx_dz = I1[i] - I0[i];
                        const R dEz_dx = I0[2 * BV + i + 1] - I0[2 * BV + i];
                        const R dEy_dx = I0[BV + i + 1] - I0[BV + i];
                        Ha[i] = I0[3 * BV + i] - hc * (dEz_dy - dEy_dz);
                        Ha[BV + i] = I0[4 * BV + i] - hc * (dEx_dz - dEz_dx);
                        Ha[2 * BV + i] = I0[5 * BV + i] - hc * (dEy_dx - dEx_dy);
                    }
                }
            }
            if (doD) fence_proxy_async_smem();
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            if (early && q >= pa && q + NS <= plast) {
                if (tid == 0) issue(q + NS);
                pissued = q + NS;
            }
            if (doD) {
                if (tid == 0) {
                    const int oc[3] = {x0 + GX, y0 + G, q - 1 + G};
                    tma_store_box<3>(&S.tm_yout, oc, comp_eb(1 - par), Outb + oslot * 6 * TV);
                    bulk_commit();
                }
                oslot ^= 1;
            }
            // S2: B(q+1) on the thread's points of the N range, with the Mur condition on the
            // x and y faces; on the z faces the passes of mur_plane follow
            const int b = q + 1;
            if (b >= z0 && b <= z1) {
                const bool fz = b == 0 || b == n2;
                const bool faces = !col_int || fz;
                const R* I0 = In(stage_of(b));
                const R* J0 = I0 + JOFF / sizeof(R);
                const R* Hc = Hs(b);
                const R* Hp = Hs(b + 2);      // plane b-1 (a ring of three)
                R* Nc = Ns(b);
                // E^{n+1} component c at box point j (backward differences of Bh)
                auto enew = [&](int c, int j) -> R {
                    if (c == 0) {
                        const R dBz_dy = Hc[2 * BV + j] - Hc[2 * BV + j - BX];
                        const R dBy_dz = Hc[BV + j] - Hp[BV + j];
                        return I0[j] + cdt * (dBz_dy - dBy_dz) - dt * J0[j];
                    } else if (c == 1) {
                        const R dBx_dz = Hc[j] - Hp[j];
                        const R dBz_dx = Hc[2 * BV + j] - Hc[2 * BV + j - 1];
                        return I0[BV + j] + cdt * (dBx_dz - dBz_dx) - dt * J0[BV + j];
                    }
                    const R dBy_dx = Hc[BV + j] - Hc[BV + j - 1];
                    const R dBx_dy = Hc[j] - Hc[j - BX];
                    return I0[2 * BV + j] + cdt * (dBy_dx - dBx_dy) - dt * J0[2 * BV + j];
                };
                // first-order Mur at face point j of component c from the inward neighbour nb
                // (E^n from the stage, E^{n+1} of the neighbour given)
                auto mur = [&](int c, int j, int nb, R en_nb) -> R {
                    return I0[c * BV + nb] + km * (en_nb - I0[c * BV + j]);
                };
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    if (!pN[r]) continue;
                    const int i = pidx[r];
                    const R ex = enew(0, i), ey = enew(1, i), ez = enew(2, i);
                    const unsigned f = pm[r];
                    const bool fx = f & 1u, fy = f & 2u;
                    if (!faces || (!fx && !fy && !fz)) {
                        Nc[i] = ex;
                        Nc[BV + i] = ey;
                        Nc[2 * BV + i] = ez;
                    } else if (fz) {
                        // z faces: every face point is left to mur_plane
                        if (!(fy || fz)) Nc[i] = ex;
                        if (!(fx || fz)) Nc[BV + i] = ey;
                        if (!(fx || fy)) Nc[2 * BV + i] = ez;
                    } else {
                        // x / y faces (points on fewer faces first, along the lowest face axis:
                        // Ez on an x-y edge takes its x neighbour's value on the y face)
                        const int sx = (f & 64u) ? 1 : -1, sy = (f & 128u) ? BX : -BX;
                        Nc[i] = fy ? mur(0, i, i + sy, enew(0, i + sy)) : ex;
                        Nc[BV + i] = fx ? mur(1, i, i + sx, enew(1, i + sx)) : ey;
                        R vz = ez;
                        if (fx && fy) {
                            const int nb = i + sx;
                            vz = mur(2, i, nb, mur(2, nb, nb + sy, enew(2, nb + sy)));
                        } else if (fx) {
                            vz = mur(2, i, i + sx, enew(2, i + sx));
                        } else if (fy) {
                            vz = mur(2, i, i + sy, enew(2, i + sy));
                        }
                        Nc[2 * BV + i] = vz;
                    }
                }
                // the store of two planes back has read its buffer (reused by the next D)
                if (tid == 0) bulk_wait_read1();
                __syncthreads();
                if (fz && b != 0) mur_plane(b);
                if (b == 1 && z0 <= 1) mur_plane(0);
            } else {
                if (tid == 0) bulk_wait_read1();
                __syncthreads();
            }
            // (z faces) plane q is no longer read: its stage takes plane q+NS
            if (!early && q >= pa && q + NS <= plast) {
                if (tid == 0) issue(q + NS);
                pissued = q + NS;
            }
        }
        if (failed) {
            if (tid == 0) {
                atomicOr(&st->status, (unsigned)FLAG_TIMEOUT);
                // let the loads still in flight land before the block exits
                while (pw < pissued) {
                    ++pw;
                    const int sgi = stage_of(pw);
                    mbar_wait_bounded(&bars[sgi], (ph >> sgi) & 1u);
                    ph ^= 1u << sgi;
                }
                bulk_wait0();
            }
            return;
        }
    }
    if (tid == 0) bulk_wait0();
}

template <typename R, int PX, int PY, int NS, int NT>
__global__ void __launch_bounds__(NT) k_yee3s(const SimDev* __restrict__ sims, const Work* __restrict__ work,
                                              int nwork, int* __restrict__ counter)
{
    yee3s_body<R, PX, PY, NS, NT, false>(sims, *sims, work, nwork, counter);
}

template <typename R, int PX, int PY, int NS, int NT>
__global__ void __launch_bounds__(NT) k_yee3s1(const __grid_constant__ SimDev one, const Work* __restrict__ work,
                                               int nwork, int* __restrict__ counter)
{
    yee3s_body<R, PX, PY, NS, NT, true>(nullptr, one, work, nwork, counter);
}

// 1D field-solver tiles (must match the host's tile choice)
template <int D>
struct YeeTile;
template <>
struct YeeTile<1> {
    static constexpr int X = 128, Y = 1, Z = 1;
};

template <int D, typename R>
static void yee_t(const Group& g, cudaStream_t s)
{
    if constexpr (D == 3) {
        if (g.one)
            k_yee3s1<R, Y3_PX, Y3_PY, Y3_NS, Y3_NT>
                <<<g.yee_grid, Y3_NT, g.yee_smem, s>>>(*g.one, g.ywork, g.nywork, g.counters + 2);
        else
            k_yee3s<R, Y3_PX, Y3_PY, Y3_NS, Y3_NT>
                <<<g.yee_grid, Y3_NT, g.yee_smem, s>>>(g.sims, g.ywork, g.nywork, g.counters + 2);
    } else if constexpr (D == 2) {
        if (g.one)
            k_yee2r1<R, Y2_PY, Y2_NT><<<g.yee_grid, Y2_NT, g.yee_smem, s>>>(*g.one, g.ywork, g.nywork, g.counters + 2);
        else
            k_yee2r<R, Y2_PY, Y2_NT><<<g.yee_grid, Y2_NT, g.yee_smem, s>>>(g.sims, g.ywork, g.nywork, g.counters + 2);
    } else {
        if (g.one)
            k_yee1<D, R, YeeTile<D>::X, YeeTile<D>::Y, YeeTile<D>::Z>
                <<<g.yee_grid, 256, g.yee_smem, s>>>(*g.one, g.ywork, g.nywork, g.counters + 2);
        else
            k_yee<D, R, YeeTile<D>::X, YeeTile<D>::Y, YeeTile<D>::Z>
                <<<g.yee_grid, 256, g.yee_smem, s>>>(g.sims, g.ywork, g.nywork, g.counters + 2);
    }
}

template <int D, typename R>
static void attr_yee(size_t smem, int* out)
{
    // both forms of the kernel get the shared-memory size; the occupancy (which sizes the
    // grid) is the lower of the two
    if constexpr (D == 3) {
        auto k = k_yee3s<R, Y3_PX, Y3_PY, Y3_NS, Y3_NT>;
        auto k1 = k_yee3s1<R, Y3_PX, Y3_PY, Y3_NS, Y3_NT>;
        int b1 = 0;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k, Y3_NT, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k1, Y3_NT, smem);
        *out = std::min(*out, b1);
    } else if constexpr (D == 2) {
        auto k = k_yee2r<R, Y2_PY, Y2_NT>;
        auto k1 = k_yee2r1<R, Y2_PY, Y2_NT>;
        int b1 = 0;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k, Y2_NT, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k1, Y2_NT, smem);
        *out = std::min(*out, b1);
    } else {
        auto k = k_yee<D, R, YeeTile<D>::X, YeeTile<D>::Y, YeeTile<D>::Z>;
        auto k1 = k_yee1<D, R, YeeTile<D>::X, YeeTile<D>::Y, YeeTile<D>::Z>;
        int b1 = 0;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k, 256, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k1, 256, smem);
        *out = std::min(*out, b1);
    }
}

#define SFF_DISPATCH2(dim, prec, FN, ...)                       \
    do {                                                        \
        if ((prec) == 0) {                                      \
            if ((dim) == 1) FN<1, double>(__VA_ARGS__);         \
            else if ((dim) == 2) FN<2, double>(__VA_ARGS__);    \
            else FN<3, double>(__VA_ARGS__);                    \
        } else {                                                \
            if ((dim) == 1) FN<1, float>(__VA_ARGS__);          \
            else if ((dim) == 2) FN<2, float>(__VA_ARGS__);     \
            else FN<3, float>(__VA_ARGS__);                     \
        }                                                       \
    } while (0)

void launch_yee(const Group& g, cudaStream_t s) { SFF_DISPATCH2(g.dim, g.prec, yee_t, g, s); }

int prepare_yee(int dim, int prec, size_t smem)
{
    int b = 0;
    SFF_DISPATCH2(dim, prec, attr_yee, smem, &b);
    return b;
}

}  // namespace sff
