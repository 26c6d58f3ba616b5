// Field solver of the scattered field (Eqs. MAmper, MFaraday; Yee stagger), sm_103a.
//
// One work item = one tile of the grid.  The tile's box (x: 4 points of halo below and
// above, y/z: 2) of E, B at step n (buffer set p) and of J^{n+1/2} (J_p) arrives by two
// TMA loads.  In shared memory:
//   A. B^{n+1/2} = B^n - (dt/2) curl E^n             (forward differences, in place)
//   B. E^{n+1}   = E^n + dt (curl B^{n+1/2} - J)      (backward differences, into the J slots)
//      except on faces, where
//   C. first-order Mur: E^{n+1}(0) = E^n(1) + (dt-dx)/(dt+dx) (E^{n+1}(1) - E^n(0)), applied along
//      the lowest face axis of the point, points on fewer faces first;
//   D. B^{n+1}   = B^{n+1/2} - (dt/2) curl E^{n+1}    on the tile, points a component does
//      not have (outside [0, n] / [0, n-1]) forced to zero.
// The tile of E^{n+1}, B^{n+1} leaves by one TMA store into buffer set 1-p, and J_{1-p}
// (the next step's deposit target) is cleared on the tile.  No CTA writes what another
// reads in the same launch.
#include <cuda_runtime.h>

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

template <int D, typename R>
__global__ void __launch_bounds__(256) k_yee(const SimDev* __restrict__ sims, const Work* __restrict__ work,
                                             int nwork, int* __restrict__ counter)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_item;
    const int tid = threadIdx.x, nth = blockDim.x;
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    unsigned phase = 0;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= nwork) break;
        const Work wk = work[item];
        const SimDev& S = sims[wk.sim];
        DevState* st = S.st;
        const int par = st->parity;

        int tc[3] = {0, 0, 0};
        {
            int t = wk.tile;
            tc[0] = t % S.nyt[0];
            t /= S.nyt[0];
            if constexpr (D > 1) {
                tc[1] = t % S.nyt[1];
                t /= S.nyt[1];
            }
            if constexpr (D > 2) tc[2] = t;
        }
        const int T[3] = {S.yt[0], D > 1 ? S.yt[1] : 1, D > 2 ? S.yt[2] : 1};
        const int lo[3] = {tc[0] * T[0], tc[1] * T[1], tc[2] * T[2]};
        const int hx[3] = {4, D > 1 ? 2 : 0, D > 2 ? 2 : 0};
        const int e[3] = {S.yb[0], D > 1 ? S.yb[1] : 1, D > 2 ? S.yb[2] : 1};
        const int sx = 1, sy = e[0], sz = e[0] * e[1];
        const int bvol = e[0] * e[1] * e[2];
        const int tvol = T[0] * T[1] * T[2];
        const size_t joff = round128(6 * bvol * sizeof(R));
        const size_t ooff = round128(joff + 3 * bvol * sizeof(R));
        R* In = reinterpret_cast<R*>(smem_raw);                 // [6][e_z][e_y][e_x]: Ex Ey Ez Bx By Bz
        R* Jn = reinterpret_cast<R*>(smem_raw + joff);          // [3][e_z][e_y][e_x]: J, then E^{n+1}
        R* Out = reinterpret_cast<R*>(smem_raw + ooff);         // [6][T_z][T_y][T_x]
        const int org[3] = {lo[0] - hx[0] + G, D > 1 ? lo[1] - hx[1] + G : 0, D > 2 ? lo[2] - hx[2] + G : 0};
        if (tid == 0) {
            tensormap_acquire(&S.tm_yin);
            tensormap_acquire(&S.tm_yj);
            tensormap_acquire(&S.tm_yout);
            mbar_arrive_expect_tx(&bar, (unsigned)(9 * bvol * sizeof(R)));
            tma_load_box<D>(In, &S.tm_yin, org, comp_eb(par), &bar);
            tma_load_box<D>(Jn, &S.tm_yj, org, comp_j(par), &bar);
        }
        const bool ok = mbar_wait_bounded(&bar, phase);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(&st->status, (unsigned)FLAG_TIMEOUT);
                mbar_wait_bounded(&bar, phase ^ 1u);
                bulk_wait0();
            }
            return;
        }
        R* Ex = In;
        R* Ey = In + bvol;
        R* Ez = In + 2 * bvol;
        R* Bx = In + 3 * bvol;
        R* By = In + 4 * bvol;
        R* Bz = In + 5 * bvol;
        R* Nx = Jn;              // J on entry, E^{n+1} after phase B
        R* Ny = Jn + bvol;
        R* Nz = Jn + 2 * bvol;
        const R cdt = R(S.dt * S.inv_dx);
        const R hc = R(0.5) * cdt;
        const R dt = R(S.dt);
        const R km = R((S.dt - S.dx) / (S.dt + S.dx));

        // A. B^{n+1/2} in place
        for (int i = tid; i < bvol; i += nth) {
            const int lx = i % e[0], ly = (i / e[0]) % e[1], lz = i / sz;
            if (lx >= e[0] - 1) continue;
            if (D > 1 && ly >= e[1] - 1) continue;
            if (D > 2 && lz >= e[2] - 1) continue;
            const R dEz_dy = D > 1 ? Ez[i + sy] - Ez[i] : R(0);
            const R dEx_dy = D > 1 ? Ex[i + sy] - Ex[i] : R(0);
            const R dEy_dz = D > 2 ? Ey[i + sz] - Ey[i] : R(0);
            const R dEx_dz = D > 2 ? Ex[i + sz] - Ex[i] : R(0);
            const R dEz_dx = Ez[i + sx] - Ez[i];
            const R dEy_dx = Ey[i + sx] - Ey[i];
            Bx[i] -= hc * (dEz_dy - dEy_dz);
            By[i] -= hc * (dEx_dz - dEz_dx);
            Bz[i] -= hc * (dEy_dx - dEx_dy);
        }
        __syncthreads();

        // B. E^{n+1} into the J slots at points 1..e-2 on every resolved axis, off the faces
        for (int i = tid; i < bvol; i += nth) {
            const int l[3] = {i % e[0], (i / e[0]) % e[1], i / sz};
            if (l[0] < 1 || l[0] >= e[0] - 1) continue;
            if (D > 1 && (l[1] < 1 || l[1] >= e[1] - 1)) continue;
            if (D > 2 && (l[2] < 1 || l[2] >= e[2] - 1)) continue;
            const int g[3] = {lo[0] - hx[0] + l[0], lo[1] - hx[1] + l[1], lo[2] - hx[2] + l[2]};
            const R dBz_dy = D > 1 ? Bz[i] - Bz[i - sy] : R(0);
            const R dBx_dy = D > 1 ? Bx[i] - Bx[i - sy] : R(0);
            const R dBy_dz = D > 2 ? By[i] - By[i - sz] : R(0);
            const R dBx_dz = D > 2 ? Bx[i] - Bx[i - sz] : R(0);
            const R dBz_dx = Bz[i] - Bz[i - sx];
            const R dBy_dx = By[i] - By[i - sx];
            if (!face_axes<D>(S, 0, g)) Nx[i] = Ex[i] + cdt * (dBz_dy - dBy_dz) - dt * Nx[i];
            if (!face_axes<D>(S, 1, g)) Ny[i] = Ey[i] + cdt * (dBx_dz - dBz_dx) - dt * Ny[i];
            if (!face_axes<D>(S, 2, g)) Nz[i] = Ez[i] + cdt * (dBy_dx - dBx_dy) - dt * Nz[i];
        }
        __syncthreads();

        // C. Mur faces, points on one face first, then edges, then corners
        const int es[3] = {sx, sy, sz};
        for (int pass = 1; pass <= D; ++pass) {
            for (int i = tid; i < bvol; i += nth) {
                const int l[3] = {i % e[0], (i / e[0]) % e[1], i / sz};
                if (l[0] < 1 || l[0] >= e[0] - 1) continue;
                if (D > 1 && (l[1] < 1 || l[1] >= e[1] - 1)) continue;
                if (D > 2 && (l[2] < 1 || l[2] >= e[2] - 1)) continue;
                const int g[3] = {lo[0] - hx[0] + l[0], lo[1] - hx[1] + l[1], lo[2] - hx[2] + l[2]};
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int m = face_axes<D>(S, c, g);
                    if (!m || __popc(m) != pass) continue;
                    const int a = __ffs(m) - 1;
                    const int dir = (g[a] == 0) ? 1 : -1;
                    const int ln = l[a] + dir;
                    if (ln < 1 || ln >= e[a] - 1) continue;
                    const int nb = i + dir * es[a];
                    const R* Eo = In + c * bvol;
                    R* En = Jn + c * bvol;
                    En[i] = Eo[nb] + km * (En[nb] - Eo[i]);
                }
            }
            __syncthreads();
        }

        // D. E^{n+1}, B^{n+1} on the tile
        for (int k = tid; k < tvol; k += nth) {
            const int t0 = k % T[0], t1 = (k / T[0]) % T[1], t2 = k / (T[0] * T[1]);
            const int i = (t0 + hx[0]) + (t1 + hx[1]) * sy + (t2 + hx[2]) * sz;
            const int g[3] = {lo[0] + t0, lo[1] + t1, lo[2] + t2};
            const R dNz_dy = D > 1 ? Nz[i + sy] - Nz[i] : R(0);
            const R dNx_dy = D > 1 ? Nx[i + sy] - Nx[i] : R(0);
            const R dNy_dz = D > 2 ? Ny[i + sz] - Ny[i] : R(0);
            const R dNx_dz = D > 2 ? Nx[i + sz] - Nx[i] : R(0);
            const R dNz_dx = Nz[i + sx] - Nz[i];
            const R dNy_dx = Ny[i + sx] - Ny[i];
            const R v[6] = {Nx[i], Ny[i], Nz[i], Bx[i] - hc * (dNz_dy - dNy_dz), By[i] - hc * (dNx_dz - dNz_dx),
                            Bz[i] - hc * (dNy_dx - dNx_dy)};
#pragma unroll
            for (int c = 0; c < 6; ++c) Out[c * tvol + k] = has_point<D>(S, c, g) ? v[c] : R(0);
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            const int oc[3] = {lo[0] + G, D > 1 ? lo[1] + G : 0, D > 2 ? lo[2] + G : 0};
            tma_store_box<D>(&S.tm_yout, oc, comp_eb(1 - par), Out);
            bulk_commit();
        }
        // clear J_{1-p} on the tile (the next step deposits into it)
        {
            R* Fg = reinterpret_cast<R*>(S.F);
            const long long jb = (long long)comp_j(1 - par) * S.sc;
            for (int k = tid; k < 3 * tvol; k += nth) {
                const int c = k / tvol, r = k - c * tvol;
                const int t0 = r % T[0], t1 = (r / T[0]) % T[1], t2 = r / (T[0] * T[1]);
                Fg[jb + c * S.sc + (long long)(D > 2 ? lo[2] + t2 + G : 0) * S.sz +
                   (long long)(D > 1 ? lo[1] + t1 + G : 0) * S.sy + (lo[0] + t0 + G)] = R(0);
            }
        }
        if (tid == 0) bulk_wait_read0();
        __syncthreads();
    }
    if (tid == 0) bulk_wait0();
}

template <int D, typename R>
static void yee_t(const Group& g, cudaStream_t s)
{
    k_yee<D, R><<<g.yee_grid, 256, g.yee_smem, s>>>(g.sims, g.ywork, g.nywork, g.counters + 2);
}

template <int D, typename R>
static void attr_yee(size_t smem, int* out)
{
    cudaFuncSetAttribute(k_yee<D, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_yee<D, R>, 256, smem);
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
