// Particle kernels of the scattered-field PIC step (sm_103a):
//   k_push     gather + incident field + Boris + move + Esirkepov deposit, one particle tile
//              per work item: the tile's field box arrives by one TMA load, the current is
//              accumulated in shared memory and leaves by one TMA reduce-add (FP32) or one
//              atomic per nonzero cell (FP64); every particle is written into its
//              destination tile's slots of the other buffer set (warp-aggregated slot
//              reservation); destination-tile and frame counts are histogrammed in shared
//              memory first (one global atomic per neighbour tile);
//   k_scan_lb / k_scan   tile scan: counts and work items of the set just written, slots
//              of the other set for the next push (counts + frame counts);
//   k_cellcount, k_cellscan, k_scatter   the opt-in cell sort: on its steps the push
//              writes in place and these place each tile's particles in cell order;
//   k_step_end step counter, particle count and buffer parity, and the next step's work
//              item numbering (k_prefix does the latter alone when needed).
// Set-up kernels generate the seeded slab, sort arbitrary particle sets by tile and set the
// first slots.
#include <cuda_runtime.h>

#include <algorithm>

#include "beam.cuh"
#include "sff_common.cuh"
#include "sff_kernels.h"

namespace sff {

template <typename R>
__device__ __forceinline__ void shape2(R d, R w[3])
{
    const R a = R(0.5) - d, b = R(0.5) + d;
    w[0] = R(0.5) * a * a;
    w[1] = R(0.75) - d * d;
    w[2] = R(0.5) * b * b;
}

template <int D>
__device__ __forceinline__ void decode_cell(const SimDev& S, unsigned cl, int c[3])
{
    c[0] = (int)(cl & ((1u << S.cb[0]) - 1u));
    c[1] = 0;
    c[2] = 0;
    if constexpr (D > 1) c[1] = (int)((cl >> S.cb[0]) & ((1u << S.cb[1]) - 1u));
    if constexpr (D > 2) c[2] = (int)(cl >> (S.cb[0] + S.cb[1]));
}

template <int D>
__device__ __forceinline__ unsigned encode_cell(const SimDev& S, const int c[3])
{
    unsigned v = (unsigned)c[0];
    if constexpr (D > 1) v |= (unsigned)c[1] << S.cb[0];
    if constexpr (D > 2) v |= (unsigned)c[2] << (S.cb[0] + S.cb[1]);
    return v;
}

template <int D>
__device__ __forceinline__ int tile_of(const SimDev& S, const int c[3])
{
    int t = c[0] / S.pt[0];
    if constexpr (D > 1) t += S.npt[0] * (c[1] / S.pt[1]);
    if constexpr (D > 2) t += S.npt[0] * S.npt[1] * (c[2] / S.pt[2]);
    return t;
}

// order-2 interpolation from a shared-memory box [bz][by][bx]
template <int D, typename R>
__device__ __forceinline__ R interp(const R* f, int bx, int bxy, const int b0, const int b1, const int b2,
                                    const R* w0, const R* w1, const R* w2)
{
    if constexpr (D == 1) {
        return w0[0] * f[b0] + w0[1] * f[b0 + 1] + w0[2] * f[b0 + 2];
    } else if constexpr (D == 2) {
        R v = R(0);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const R* r = f + (b1 + j) * bx + b0;
            v += w1[j] * (w0[0] * r[0] + w0[1] * r[1] + w0[2] * r[2]);
        }
        return v;
    } else {
        R v = R(0);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            R vk = R(0);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const R* r = f + (b2 + k) * bxy + (b1 + j) * bx + b0;
                vk += w1[j] * (w0[0] * r[0] + w0[1] * r[1] + w0[2] * r[2]);
            }
            v += w2[k] * vk;
        }
        return v;
    }
}

// Current accumulation in the work item's shared-memory box.  FP32: 32-bit fixed point with
// the scale q = 2^29 / (max(N, 256) w_max) of the item (N particles): a contribution of one
// particle to one node is bounded by w |v| <= w_max (Esirkepov's partial sums of the shape
// change are at most the move in cells, v dt/dx, times dx/dt; the transverse weights are
// averages of shapes in [0, 1]; |v| < c = 1), so |c q| <= 2^21 and no node's sum leaves
// 2^29.  Each contribution is rounded to the nearest integer by one FMA with 1.5 * 2^23 (the
// sum lands in [2^23, 2^24), where the float spacing is 1: its low bits are the rounded
// integer, exact for |c q| < 2^22) and added with the native shared-memory integer add (the
// FP32 add is a compare-and-swap loop with a round trip per attempt); zero contributions are
// added too (no test).  The box is turned back into FP32 before its TMA reduce-add; each
// contribution's rounding is at most 2^-30 max(N, 256) w_max.  FP64 keeps double sums.
__device__ __forceinline__ void jdep(float* a, float v, float q)
{
    const float f = fmaf(v, q, 12582912.0f);
    atomicAdd(reinterpret_cast<int*>(a), __float_as_int(f) - 0x4B400000);
}
__device__ __forceinline__ void jdep(double* a, double v, double)
{
    if (v != 0.0) atomicAdd(a, v);
}
constexpr float JQ_RANGE = 536870912.0f;   // 2^29

// Global chunk k of a launch group -> simulation, tile and particle slots.  Chunks are
// numbered per simulation by the tile scan (ctile / crange) and across the group by gprefix.
struct ChunkRef {
    int sim, tile, p0, p1;
};

__device__ __forceinline__ ChunkRef chunk_of(const SimDev* __restrict__ sims, int nsims, const int* __restrict__ gprefix,
                                             int k)
{
    int lo = 0, hi = nsims;   // largest s with gprefix[s] <= k
    while (hi - lo > 1) {
        const int m = (lo + hi) >> 1;
        if (gprefix[m] <= k) lo = m; else hi = m;
    }
    const SimDev& S = sims[lo];
    const int par = S.st->parity;
    const int j = k - gprefix[lo];
    const int2 pr = S.crange[par][j];
    ChunkRef r;
    r.sim = lo;
    r.tile = S.ctile[par][j];
    r.p0 = pr.x;
    r.p1 = pr.y;
    return r;
}

// Reserve destination slots for a warp's particles (tile < 0: nothing to place); every lane of
// the warp must call it.
__device__ __forceinline__ int warp_reserve(int tile, int* cursors)
{
    const unsigned peers = __match_any_sync(0xffffffffu, tile);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    const int rank = __popc(peers & ((1u << lane) - 1u));
    int base = 0;
    if (tile >= 0 && lane == leader) base = atomicAdd(&cursors[tile], __popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    return base + rank;
}

// ---- momentum updates; h = q dt / 2 (q = -1, m = 1, c = 1) ----------------------------

// Boris: electric half kick, rotation about B by 2 atan(|h B|/gamma^-), electric half kick.
template <typename R>
__device__ __forceinline__ void boris_update(R u[3], const R E[3], const R B[3], R h)
{
    R um[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) um[d] = u[d] + h * E[d];
    const R tf = h * m_rsqrt(R(1) + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);   // h / gamma^-
    const R tv[3] = {tf * B[0], tf * B[1], tf * B[2]};
    const R t2 = tv[0] * tv[0] + tv[1] * tv[1] + tv[2] * tv[2];
    const R sf = R(2) / (R(1) + t2);
    const R up[3] = {um[0] + (um[1] * tv[2] - um[2] * tv[1]), um[1] + (um[2] * tv[0] - um[0] * tv[2]),
                     um[2] + (um[0] * tv[1] - um[1] * tv[0])};
    const R sv[3] = {sf * tv[0], sf * tv[1], sf * tv[2]};
    u[0] = um[0] + (up[1] * sv[2] - up[2] * sv[1]) + h * E[0];
    u[1] = um[1] + (up[2] * sv[0] - up[0] * sv[2]) + h * E[1];
    u[2] = um[2] + (up[0] * sv[1] - up[1] * sv[0]) + h * E[2];
}

// Implicit-midpoint rotation shared by the Vay and Higuera-Cary schemes: with tau = h B,
// gamma^2 is the positive root of g^4 - sigma g^2 - (tau^2 + (w.tau)^2) = 0,
// sigma = 1 + w^2 - tau^2 (taken in the form without cancellation for either sign of
// sigma), t = tau/gamma and the result solves v - v x t = w: v = (w + (w.t) t + w x t)/(1 + t^2).
template <typename R>
__device__ __forceinline__ void midpoint_rotation(const R w[3], const R B[3], R h, R v[3])
{
    const R tau[3] = {h * B[0], h * B[1], h * B[2]};
    const R t2 = tau[0] * tau[0] + tau[1] * tau[1] + tau[2] * tau[2];
    const R ws = w[0] * tau[0] + w[1] * tau[1] + w[2] * tau[2];
    const R sigma = R(1) + w[0] * w[0] + w[1] * w[1] + w[2] * w[2] - t2;
    const R K = t2 + ws * ws;
    const R Dq = m_sqrt(sigma * sigma + R(4) * K);
    const R g2 = sigma >= R(0) ? R(0.5) * (sigma + Dq) : R(2) * K / (Dq - sigma);
    const R ig = R(1) / m_sqrt(g2);
    const R t[3] = {tau[0] * ig, tau[1] * ig, tau[2] * ig};
    const R tt = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    const R wt = w[0] * t[0] + w[1] * t[1] + w[2] * t[2];
    const R sf = R(1) / (R(1) + tt);
    v[0] = sf * (w[0] + wt * t[0] + (w[1] * t[2] - w[2] * t[1]));
    v[1] = sf * (w[1] + wt * t[1] + (w[2] * t[0] - w[0] * t[2]));
    v[2] = sf * (w[2] + wt * t[2] + (w[0] * t[1] - w[1] * t[0]));
}

// Vay (2008): kick by E + v x B with the old velocity, a second electric half kick, then the
// implicit-midpoint rotation with the gamma of the new momentum.
template <typename R>
__device__ __forceinline__ void vay_update(R u[3], const R E[3], const R B[3], R h)
{
    const R ig0 = R(1) / m_sqrt(R(1) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const R v[3] = {u[0] * ig0, u[1] * ig0, u[2] * ig0};
    const R w[3] = {u[0] + h * (R(2) * E[0] + (v[1] * B[2] - v[2] * B[1])),
                    u[1] + h * (R(2) * E[1] + (v[2] * B[0] - v[0] * B[2])),
                    u[2] + h * (R(2) * E[2] + (v[0] * B[1] - v[1] * B[0]))};
    midpoint_rotation<R>(w, B, h, u);
}

// Higuera-Cary (2017): electric half kick to u^-, implicit-midpoint rotation to the
// mid-rotation momentum ubar (gamma of ubar), u^+ = 2 ubar - u^-, electric half kick.
template <typename R>
__device__ __forceinline__ void higuera_cary_update(R u[3], const R E[3], const R B[3], R h)
{
    const R um[3] = {u[0] + h * E[0], u[1] + h * E[1], u[2] + h * E[2]};
    R ub[3];
    midpoint_rotation<R>(um, B, h, ub);
#pragma unroll
    for (int d = 0; d < 3; ++d) u[d] = R(2) * ub[d] - um[d] + h * E[d];
}

// Frame count of a particle that lands in cell cn of the tile at offset rel (-1, 0, 1 per
// axis) from the work item's tile T0: every neighbour of that tile whose one-cell frame
// holds cn (cn on the tile's first cell along an axis: the neighbour below; on its last:
// the neighbour above; and their combinations along several axes) gets one count, in a
// shared-memory histogram over tile offsets -2..2 per axis from the work item's tile.
// Tiles are at least two cells wide, so a cell is first or last along an axis, not both.
template <int D>
__device__ __forceinline__ void frame_count(const SimDev& S, const int cn[3], const int T0[3], const int rel[3],
                                            int* s_frame)
{
    int f[3] = {0, 0, 0}, base = 0;
    bool any = false;
    constexpr int W[3] = {1, 5, 25};
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const int l = cn[d] - (T0[d] + rel[d] * S.pt[d]);
        f[d] = l == 0 ? -1 : (l == S.pt[d] - 1 ? 1 : 0);
        any = any || f[d] != 0;
        base += (rel[d] + 2) * W[d];
    }
    if (!any) return;
#pragma unroll
    for (int m = 1; m < (1 << D); ++m) {
        int idx = base;
        bool ok = true;
#pragma unroll
        for (int d = 0; d < D; ++d)
            if ((m >> d) & 1) {
                ok = ok && f[d] != 0;
                idx += f[d] * W[d];
            }
        if (ok) atomicAdd(&s_frame[idx], 1);
    }
}

// Threads of a push block and blocks per SM the registers are budgeted for.  The 3D FP32
// push shares its 101 KB box (16x8x4 tiles) among 512 threads at 64 registers: two blocks
// keep 32 warps per SM busy instead of 16 with 256-thread blocks at 128 registers.
template <int D, typename R>
__host__ __device__ constexpr int push_threads()
{
    return (D == 3 && sizeof(R) == 4) ? 512 : 256;
}
template <int D, typename R>
__host__ __device__ constexpr int push_min_blocks()
{
    return sizeof(R) == 8 ? 1 : (D <= 2 ? 4 : 2);
}

// Chunk k of a single simulation (its chunks are numbered from gprefix[0]).
__device__ __forceinline__ ChunkRef chunk_of_one(const SimDev& S, const int* __restrict__ gprefix, int k)
{
    const int par = S.st->parity;
    const int j = k - gprefix[0];
    const int2 pr = S.crange[par][j];
    ChunkRef r;
    r.sim = 0;
    r.tile = S.ctile[par][j];
    r.p0 = pr.x;
    r.p1 = pr.y;
    return r;
}

// The push of a launch group (see k_push / k_push1 below).  ONE: the group is one simulation
// whose descriptor `one` is a kernel parameter (constant bank: its fields cost no load
// instruction, and the tensor maps are used from parameter space); otherwise the
// descriptors of the group's simulations are read from the device array `sims`.
// `sorting`: this step's re-sort orders the tiles by cell; then the simulations that have a
// cell sort are pushed in place (k_scatter places them) and the others straight into the
// other buffer set like every step.
template <int D, typename R, bool ONE>
__device__ __forceinline__ void push_body(const SimDev* __restrict__ sims, const SimDev& one, int nsims,
                                          const int* __restrict__ gprefix, int* __restrict__ counter, int sorting)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_item;
    __shared__ int s_hist[27];
    constexpr int NFR = D == 1 ? 5 : (D == 2 ? 25 : 125);
    __shared__ int s_frame[NFR];
    __shared__ PhaseRef<R> s_pref;
    const int tid = threadIdx.x, nth = blockDim.x;
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    unsigned phase = 0;
    int acq_sim = -1;         // thread 0: the simulation whose tensor maps it has acquired
    for (;;) {
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= gprefix[nsims]) break;
        const ChunkRef ck = ONE ? chunk_of_one(one, gprefix, item) : chunk_of(sims, nsims, gprefix, item);
        const SimDev& S = ONE ? one : sims[ck.sim];
        DevState* st = S.st;
        const int par = st->parity, np = 1 - par;
        const int p0 = ck.p0, p1 = ck.p1;
        const bool direct = !(sorting && S.ccnt != nullptr);

        int tc[3] = {0, 0, 0};
        {
            int t = ck.tile;
            tc[0] = t % S.npt[0];
            t /= S.npt[0];
            if constexpr (D > 1) {
                tc[1] = t % S.npt[1];
                t /= S.npt[1];
            }
            if constexpr (D > 2) tc[2] = t;
        }
        const int T0[3] = {tc[0] * S.pt[0], tc[1] * S.pt[1], tc[2] * S.pt[2]};
        const int bx = S.pb[0], by = D > 1 ? S.pb[1] : 1, bz = D > 2 ? S.pb[2] : 1;
        const int bxy = bx * by, bvol = bxy * bz;
        R* Fs = reinterpret_cast<R*>(smem_raw);   // [6][bz][by][bx]: Ex Ey Ez Bx By Bz at step n
        R* Js = reinterpret_cast<R*>(smem_raw + round128(6 * bvol * sizeof(R)));   // [3][bz][by][bx]
        // box: x nodes [T0-4, T0+pt+4), y/z nodes [T0-2, T0+pt+3); array index = node + GX (x), + G (y, z)
        const int org[3] = {T0[0] - 4 + GX, D > 1 ? T0[1] - 2 + G : 0, D > 2 ? T0[2] - 2 + G : 0};
        if (tid == 0) {
            // the maps were written to device memory before the launch: one acquire per
            // simulation and block orders that write before this thread's TMA uses
            if (!ONE && ck.sim != acq_sim) {
                tensormap_acquire(&S.tm_pf);
                tensormap_acquire(&S.tm_pj);
                acq_sim = ck.sim;
            }
            mbar_arrive_expect_tx(&bar, (unsigned)(6 * bvol * sizeof(R)));
            tma_load_box<D>(Fs, &S.tm_pf, org, S.incgrid ? COMP_TOTAL : comp_eb(par), &bar);
            // double-precision phase reference of this tile, once per tile
            s_pref = phase_ref<R>(S, (double)st->step * S.dt, T0[0]);
        }
        for (int i = tid; i < 3 * bvol; i += nth) Js[i] = R(0);
        if (tid < 27) s_hist[tid] = 0;
        for (int i = tid; i < NFR; i += nth) s_frame[i] = 0;
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

        const BeamC<R>& bc = beam_of<R>(S);
        const PhaseRef<R>& pref = s_pref;     // read from shared memory where used (no registers held)
        // fixed-point scale of this item's current (FP32; unused in FP64)
        const float wmax = st->wmax;
        const R jq = (sizeof(R) == 4 && wmax > 0.f) ? R(JQ_RANGE / ((float)max(p1 - p0, 256) * wmax)) : R(0);
        const R dtdx = bc.dtdx;
        const R jfac = bc.jfac;                     // -q dx/dt, q = -1
        const R hq = bc.hq;                         // q dt / 2
        const int hx[3] = {4, 2, 2};                // box halo below the tile per axis

        // Rounds of nth particles (256 or 512).  With P particles per cell (1, 2, 4 or 8) sitting next to
        // each other after the sort, lane l of warp w takes particle P l + (w mod P) of the
        // round's (w div P)-th group of 32 P: the 32 lanes of a warp then sit in 32
        // consecutive cells, so the same stencil node of the deposit and the gather is a
        // different shared-memory word (mostly a different bank) in every lane.
        const int P = S.lane_p, wq = tid >> 5;
        int q = (tid & 31) * P + (wq & (P - 1)) + 32 * P * (wq / P);
        if (S.pt[0] == 16 && P <= 4) {
            // 16-cell tile rows: a warp's 32 cells span two rows.  The box row pitch is 24
            // words, so rows two apart start 16 banks apart: the warp's groups take rows
            // (r, r + 2) of the round instead of (r, r + 1), and its two half-warps hit
            // disjoint banks.
            const int g = wq / P, l = tid & 31;
            const int row = ((g >> 1) << 2) + (g & 1) + ((l >> 4) << 1);
            q = (row * 16 + (l & 15)) * P + (wq & (P - 1));
        }
        for (int rb = p0; rb < p1; rb += nth) {
            const int p = rb + q;
            // what the placement below needs: new cell (DEAD: removed or no particle),
            // destination tile, offsets, momentum, weight
            unsigned ncl = DEAD;
            int tdst = -1;
            R on[3] = {R(0), R(0), R(0)}, u[3] = {R(0), R(0), R(0)}, wt = R(0);
            if (p < p1) {
                const unsigned cl = S.cell[par][p];
                int c[3];
                decode_cell<D>(S, cl, c);
                R o[3] = {R(0), R(0), R(0)};
#pragma unroll
                for (int d = 0; d < D; ++d) o[d] = reinterpret_cast<const R*>(S.off[par][d])[p];

                // ---- incident field at (x^n, t^n) (in a total-field run, or when it was
                // evaluated on the grid, it is in the gathered field already).  Evaluated
                // before the gather, and the momentum and weight loaded after it: fewer values
                // live across the closed form, the most register-hungry part of the push ----
                R Ei[3] = {R(0), R(0), R(0)}, Bi[3] = {R(0), R(0), R(0)};
                if (!S.tf && !S.incgrid) incident_at<D, R>(S, bc, pref, c, o, Ei, Bi);

                // ---- gather of the scattered field (order-2 shapes on the Yee stagger) ----
                R Wp[3][3], Wd[3][3];
                int lp[3] = {0, 0, 0}, ld[3] = {0, 0, 0};
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    if (d < D) {
                        const int h = o[d] >= R(0.5);
                        shape2(o[d] - R(h), Wp[d]);
                        lp[d] = c[d] + h - 1 - T0[d] + hx[d];
                        shape2(o[d] - R(0.5), Wd[d]);
                        ld[d] = c[d] - 1 - T0[d] + hx[d];
                    } else {
                        Wp[d][0] = Wd[d][0] = R(1);
                        Wp[d][1] = Wd[d][1] = Wp[d][2] = Wd[d][2] = R(0);
                    }
                }
#pragma unroll
                for (int d = 0; d < 3; ++d) u[d] = reinterpret_cast<const R*>(S.mom[par][d])[p];
                wt = reinterpret_cast<const R*>(S.wgt[par])[p];
                R E[3], B[3];
                E[0] = Ei[0] + interp<D, R>(Fs + 0 * bvol, bx, bxy, ld[0], lp[1], lp[2], Wd[0], Wp[1], Wp[2]);
                E[1] = Ei[1] + interp<D, R>(Fs + 1 * bvol, bx, bxy, lp[0], ld[1], lp[2], Wp[0], Wd[1], Wp[2]);
                E[2] = Ei[2] + interp<D, R>(Fs + 2 * bvol, bx, bxy, lp[0], lp[1], ld[2], Wp[0], Wp[1], Wd[2]);
                B[0] = Bi[0] + interp<D, R>(Fs + 3 * bvol, bx, bxy, lp[0], ld[1], ld[2], Wp[0], Wd[1], Wd[2]);
                B[1] = Bi[1] + interp<D, R>(Fs + 4 * bvol, bx, bxy, ld[0], lp[1], ld[2], Wd[0], Wp[1], Wd[2]);
                B[2] = Bi[2] + interp<D, R>(Fs + 5 * bvol, bx, bxy, ld[0], ld[1], lp[2], Wd[0], Wd[1], Wp[2]);

                // ---- momentum update, charge -1, mass 1 (u^{n-1/2} -> u^{n+1/2}) ----
                if (S.pusher == 1) vay_update<R>(u, E, B, hq);
                else if (S.pusher == 2) higuera_cary_update<R>(u, E, B, hq);
                else boris_update<R>(u, E, B, hq);
                const R ig = m_rsqrt(R(1) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);   // 1 / gamma
                const R v[3] = {u[0] * ig, u[1] * ig, u[2] * ig};

                // ---- Esirkepov deposition of the move ----
                // Per axis the old shape covers the old nearest node and its two neighbours; the
                // new shape is shifted by sh in {-1, 0, 1} nodes (|move| < 1 cell), so both fit a
                // window of four nodes starting one below the old support when sh = -1 and at it
                // otherwise.  S0 / DS: old shape / shape change on that window.  Along the
                // current's own axis the window's last partial sum is the total charge change,
                // zero: one node fewer carries that component.  When no lane of the warp changes
                // its nearest node along an axis (sh = 0 everywhere: most steps of most
                // electrons), the window's fourth node is zero for every lane and the loops stop
                // at three nodes on that axis (a warp-uniform bound).
                R S0[3][4], DS[3][4];
                int jw[3] = {0, 0, 0};
                R mv[3] = {R(0), R(0), R(0)};
                bool cross[3] = {false, false, false};
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    mv[d] = dtdx * v[d];
                    const int h0 = o[d] >= R(0.5);
                    const R d0 = o[d] - R(h0);
                    const R r1 = d0 + mv[d];
                    const int sh = (int)m_floor(r1 + R(0.5));
                    const R d1 = r1 - R(sh);
                    R w0[3], w1[3];
                    shape2(d0, w0);
                    shape2(d1, w1);
                    const bool lo = sh < 0, hi = sh > 0;
                    cross[d] = sh != 0;
                    const R o0[4] = {lo ? R(0) : w0[0], lo ? w0[0] : w0[1], lo ? w0[1] : w0[2], lo ? w0[2] : R(0)};
                    const R n1[4] = {hi ? R(0) : w1[0], hi ? w1[0] : w1[1], hi ? w1[1] : w1[2], hi ? w1[2] : R(0)};
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        S0[d][m] = o0[m];
                        DS[d][m] = n1[m] - o0[m];
                    }
                    jw[d] = c[d] + h0 - (lo ? 2 : 1) - T0[d] + hx[d];
                }
                // ---- move: carry the offset into the cell index; removal near the faces.
                // Done before the deposit's loops below, so that across them only the new cell,
                // offsets and destination stay live (not the old cell, offsets and move) ----
                int cn[3] = {c[0], c[1], c[2]};
                bool dead = false;
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    const R x = o[d] + mv[d];
                    const R fl = m_floor(x);
                    R r = x - fl;
                    int k = (int)fl;
                    if (r >= R(1)) {
                        r -= R(1);
                        k += 1;
                    }
                    cn[d] = c[d] + k;
                    on[d] = r;
                    if (cn[d] < S.margin || cn[d] >= S.n[d] - S.margin) dead = true;
                }
                if (dead) {
                    const int slot = atomicAdd(&st->n_exits, 1);
                    if (slot < S.max_exits) {
                        double* e = S.exits + (long long)slot * EXIT_DOUBLES;
                        e[0] = (double)u[0];
                        e[1] = (double)u[1];
                        e[2] = (double)u[2];
                        e[3] = (double)wt;
                        e[4] = (double)S.pid[par][p];
                        e[5] = (double)st->step;
                    } else {
                        atomicOr(&st->status, (unsigned)FLAG_EXIT_OVERFLOW);
                    }
                } else {
                    // destination tile relative to this one (a move is under one cell per axis)
                    int hidx = 0, mul = 1, tg = 0, tmul = 1;
                    int rel[3] = {0, 0, 0};
#pragma unroll
                    for (int d = 0; d < D; ++d) {
                        rel[d] = cn[d] < T0[d] ? -1 : (cn[d] >= T0[d] + S.pt[d] ? 1 : 0);
                        hidx += (rel[d] + 1) * mul;
                        mul *= 3;
                        tg += (tc[d] + rel[d]) * tmul;
                        tmul *= S.npt[d];
                    }
                    atomicAdd(&s_hist[hidx], 1);
                    frame_count<D>(S, cn, T0, rel, s_frame);
                    ncl = encode_cell<D>(S, cn);
                    tdst = tg;
                }
                if (!direct) {
                    S.cell[par][p] = ncl;
#pragma unroll
                    for (int d = 0; d < D; ++d) reinterpret_cast<R*>(S.off[par][d])[p] = on[d];
#pragma unroll
                    for (int d = 0; d < 3; ++d) reinterpret_cast<R*>(S.mom[par][d])[p] = u[d];
                }
                // ---- the deposit on the windows set up above ----
                // window width per axis over the lanes running here (each lane's own vote is in
                // its mask, so its width covers its own window whatever the warp's convergence)
                const unsigned am = __activemask();
                int nw[3] = {4, 4, 4};
#pragma unroll
                for (int d = 0; d < D; ++d) nw[d] = __any_sync(am, cross[d]) ? 4 : 3;
                R* Jx = Js;
                R* Jy = Js + bvol;
                R* Jz = Js + 2 * bvol;
                const R cw = jfac * wt;
                const R third = R(1) / R(3);
                if constexpr (D == 1) {
                    R acc = R(0);
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        if (a >= nw[0] - 1) break;
                        acc += cw * DS[0][a];
                        jdep(&Jx[jw[0] + a], acc, jq);
                    }
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        if (a >= nw[0]) break;
                        const R f = S0[0][a] + R(0.5) * DS[0][a];
                        jdep(&Jy[jw[0] + a], -wt * v[1] * f, jq);
                        jdep(&Jz[jw[0] + a], -wt * v[2] * f, jq);
                    }
                } else if constexpr (D == 2) {
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        if (b >= nw[1]) break;
                        const R fy = S0[1][b] + R(0.5) * DS[1][b];
                        R acc = R(0);
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            if (a >= nw[0] - 1) break;
                            acc += cw * DS[0][a] * fy;
                            jdep(&Jx[(jw[1] + b) * bx + jw[0] + a], acc, jq);
                        }
                    }
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        if (a >= nw[0]) break;
                        const R fx = S0[0][a] + R(0.5) * DS[0][a];
                        R acc = R(0);
#pragma unroll
                        for (int b = 0; b < 3; ++b) {
                            if (b >= nw[1] - 1) break;
                            acc += cw * DS[1][b] * fx;
                            jdep(&Jy[(jw[1] + b) * bx + jw[0] + a], acc, jq);
                        }
                    }
                    const R qv = -wt * v[2];
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        if (b >= nw[1]) break;
#pragma unroll
                        for (int a = 0; a < 4; ++a) {
                            if (a >= nw[0]) break;
                            const R wz = S0[0][a] * S0[1][b] + R(0.5) * DS[0][a] * S0[1][b] +
                                         R(0.5) * S0[0][a] * DS[1][b] + third * DS[0][a] * DS[1][b];
                            jdep(&Jz[(jw[1] + b) * bx + jw[0] + a], qv * wz, jq);
                        }
                    }
                } else {
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) {
                        if (cc >= nw[2]) break;
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            if (b >= nw[1]) break;
                            const R fyz = S0[1][b] * S0[2][cc] + R(0.5) * DS[1][b] * S0[2][cc] +
                                          R(0.5) * S0[1][b] * DS[2][cc] + third * DS[1][b] * DS[2][cc];
                            R acc = R(0);
#pragma unroll
                            for (int a = 0; a < 3; ++a) {
                                if (a >= nw[0] - 1) break;
                                acc += cw * DS[0][a] * fyz;
                                jdep(&Jx[(jw[2] + cc) * bxy + (jw[1] + b) * bx + jw[0] + a], acc, jq);
                            }
                        }
                    }
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) {
                        if (cc >= nw[2]) break;
#pragma unroll
                        for (int a = 0; a < 4; ++a) {
                            if (a >= nw[0]) break;
                            const R fxz = S0[0][a] * S0[2][cc] + R(0.5) * DS[0][a] * S0[2][cc] +
                                          R(0.5) * S0[0][a] * DS[2][cc] + third * DS[0][a] * DS[2][cc];
                            R acc = R(0);
#pragma unroll
                            for (int b = 0; b < 3; ++b) {
                                if (b >= nw[1] - 1) break;
                                acc += cw * DS[1][b] * fxz;
                                jdep(&Jy[(jw[2] + cc) * bxy + (jw[1] + b) * bx + jw[0] + a], acc, jq);
                            }
                        }
                    }
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        if (b >= nw[1]) break;
#pragma unroll
                        for (int a = 0; a < 4; ++a) {
                            if (a >= nw[0]) break;
                            const R fxy = S0[0][a] * S0[1][b] + R(0.5) * DS[0][a] * S0[1][b] +
                                          R(0.5) * S0[0][a] * DS[1][b] + third * DS[0][a] * DS[1][b];
                            R acc = R(0);
#pragma unroll
                            for (int cc = 0; cc < 3; ++cc) {
                                if (cc >= nw[2] - 1) break;
                                acc += cw * DS[2][cc] * fxy;
                                jdep(&Jz[(jw[2] + cc) * bxy + (jw[1] + b) * bx + jw[0] + a], acc, jq);
                            }
                        }
                    }
                }

            }
            // ---- placement into the destination tile's slots of the other buffer set (all
            // lanes of the warp take part in the reservation) ----
            if (direct) {
                const int slot = warp_reserve(tdst, S.tcur);
                if (tdst >= 0) {
                    const long long q0 = S.toff[np][tdst];
                    if (slot < S.toff[np][tdst + 1] - q0) {
                        const long long qd = q0 + slot;
                        S.cell[np][qd] = ncl;
#pragma unroll
                        for (int d = 0; d < D; ++d) reinterpret_cast<R*>(S.off[np][d])[qd] = on[d];
#pragma unroll
                        for (int d = 0; d < 3; ++d) reinterpret_cast<R*>(S.mom[np][d])[qd] = u[d];
                        reinterpret_cast<R*>(S.wgt[np])[qd] = wt;
                        S.pid[np][qd] = S.pid[par][p];
                    } else {
                        atomicOr(&st->status, (unsigned)FLAG_CAPACITY);   // cannot happen: the slack bounds the arrivals
                    }
                }
            }
        }
        __syncthreads();

        // ---- current flush and destination-tile counts ----
        if constexpr (sizeof(R) == 4) {
            // fixed point back to FP32, in place
            const float inv = (float)max(p1 - p0, 256) * wmax * (1.0f / JQ_RANGE);
            int* Jq = reinterpret_cast<int*>(Js);
            for (int i = tid; i < 3 * bvol; i += nth) Jq[i] = __float_as_int(__int2float_rn(Jq[i]) * inv);
            __syncthreads();
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0) {
                tma_reduce_add_box<D>(&S.tm_pj, org, comp_j(par), Js);
                bulk_commit();
            }
        } else {
            R* Fg = reinterpret_cast<R*>(S.F);
            const long long jbase = (long long)comp_j(par) * S.sc;
            for (int i = tid; i < 3 * bvol; i += nth) {
                const R val = Js[i];
                if (val != R(0)) {
                    const int comp = i / bvol, rem = i - comp * bvol;
                    const int lz = rem / bxy, rxy = rem - lz * bxy, ly = rxy / bx, lx = rxy - ly * bx;
                    atomicAdd(&Fg[jbase + comp * S.sc + (long long)(org[2] + lz) * S.sz +
                                  (long long)(org[1] + ly) * S.sy + (org[0] + lx)],
                              val);
                }
            }
        }
        constexpr int NH = D == 1 ? 3 : (D == 2 ? 9 : 27);
        if (tid < NH && s_hist[tid] > 0) {
            int h = tid, nt = 0, mul = 1;
#pragma unroll
            for (int d = 0; d < D; ++d) {
                nt += (tc[d] + (h % 3) - 1) * mul;
                h /= 3;
                mul *= S.npt[d];
            }
            atomicAdd(&S.tcnt[nt], s_hist[tid]);
        }
        for (int i = tid; i < NFR; i += nth) {
            const int v = s_frame[i];
            if (v > 0) {
                int h = i, nt = 0, mul = 1;
                bool in = true;
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    const int tcd = tc[d] + h % 5 - 2;
                    h /= 5;
                    in = in && tcd >= 0 && tcd < S.npt[d];
                    nt += tcd * mul;
                    mul *= S.npt[d];
                }
                if (in) atomicAdd(&S.fcnt[nt], v);
            }
        }
        if constexpr (sizeof(R) == 4) {
            if (tid == 0) bulk_wait_read0();
        }
        __syncthreads();
    }
    if (tid == 0) bulk_wait0();
}

template <int D, typename R>
__global__ void __launch_bounds__(push_threads<D, R>(), push_min_blocks<D, R>())
    k_push(const SimDev* __restrict__ sims, int nsims, const int* __restrict__ gprefix, int* __restrict__ counter,
           int sorting)
{
    push_body<D, R, false>(sims, *sims, nsims, gprefix, counter, sorting);
}

// one simulation: the descriptor by value in the kernel's parameters
template <int D, typename R>
__global__ void __launch_bounds__(push_threads<D, R>(), push_min_blocks<D, R>())
    k_push1(const __grid_constant__ SimDev one, const int* __restrict__ gprefix, int* __restrict__ counter, int sorting)
{
    push_body<D, R, true>(nullptr, one, 1, gprefix, counter, sorting);
}

// Block-wide exclusive scan of one int per thread (blockDim a multiple of 32, <= 1024).
__device__ __forceinline__ int block_exclusive_scan(int v, int* s_warp)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = lane < nw ? s_warp[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    const int r = x - v + (wid > 0 ? s_warp[wid - 1] : 0);
    __syncthreads();
    return r;
}

// Chunks of tile t of buffer set q holding c particles from slot base: ctile / crange
// entries from chunk index rc on.
__device__ __forceinline__ void write_chunks(const SimDev& S, int q, int t, int base, int c, int rc)
{
    const int nc = (c + S.chunk - 1) / S.chunk;
    for (int k = 0; k < nc; ++k) {
        S.ctile[q][rc + k] = t;
        const int a = base + k * S.chunk;
        S.crange[q][rc + k] = make_int2(a, min(a + S.chunk, base + c));
    }
}

// Tile scan of one simulation after a push into buffer set q (one block of 1024 threads):
// per tile the particles now in set q (tcnt) and its frame count (fcnt) give
//   set q:      tnum, the chunk offsets coff and the chunk map (ctile, crange) over the
//               slots toff[q] set by the previous scan;
//   set 1 - q:  toff = exclusive scan of tcnt + fcnt, the slots of the next step's push;
// the particle total goes to n_next; the counts, cursors and frame counts are cleared.
// `compact` (set-up): toff[q] = exclusive scan of tcnt first (no slack: the particles are
// then placed there by the caller) and set 1 - q is left alone.
__device__ void scan_counts(const SimDev& S, int q, bool compact)
{
    __shared__ int s_warp[32];
    const int n = S.nptiles;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int per = (n + nth - 1) / nth;
    const int i0 = min(n, tid * per), i1 = min(n, i0 + per);
    int lp = 0, lc = 0, lk = 0;
    for (int i = i0; i < i1; ++i) {
        const int c = S.tcnt[i];
        lp += c;
        lc += (c + S.chunk - 1) / S.chunk;
        lk += c + S.fcnt[i];
    }
    int rp = block_exclusive_scan(lp, s_warp);
    int rc = block_exclusive_scan(lc, s_warp);
    int rk = block_exclusive_scan(lk, s_warp);
    if (tid == nth - 1) atomicAdd(&S.st->n_next, rp + lp);
    for (int i = i0; i < i1; ++i) {
        const int c = S.tcnt[i];
        if (compact) S.toff[q][i] = rp;
        const int base = compact ? rp : S.toff[q][i];
        S.tnum[q][i] = c;
        S.coff[q][i] = rc;
        write_chunks(S, q, i, base, c, rc);
        if (!compact) S.toff[1 - q][i] = rk;
        rp += c;
        rc += (c + S.chunk - 1) / S.chunk;
        rk += c + S.fcnt[i];
        S.tcnt[i] = 0;
        S.tcur[i] = 0;
        S.fcnt[i] = 0;
    }
    if (tid == nth - 1) {
        if (compact) S.toff[q][n] = rp;
        else S.toff[1 - q][n] = rk;
        S.coff[q][n] = rc;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(1024) k_scan(const SimDev* __restrict__ sims)
{
    const SimDev& S = sims[blockIdx.x];
    scan_counts(S, 1 - S.st->parity, false);
}

// set-up: counts of the particles about to be placed into set q
__global__ void __launch_bounds__(1024) k_scan_one(const SimDev* __restrict__ sim, int q)
{
    scan_counts(*sim, q, true);
}

// set-up, after the particles sit in set q: frame counts of every particle ...
template <int D>
__global__ void k_frame_linear(const SimDev* __restrict__ sim, int q, long long n)
{
    const SimDev& S = *sim;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const unsigned cl = S.cell[q][p];
        if (cl == DEAD) continue;
        int c[3];
        decode_cell<D>(S, cl, c);
        int tc[3] = {0, 0, 0}, T[3] = {0, 0, 0};
#pragma unroll
        for (int d = 0; d < D; ++d) {
            tc[d] = c[d] / S.pt[d];
            T[d] = tc[d] * S.pt[d];
        }
        // every neighbour tile whose one-cell frame holds c
        constexpr int NF = D == 1 ? 3 : (D == 2 ? 9 : 27);
        for (int k = 0; k < NF; ++k) {
            int r = k, nt = 0, mul = 1;
            bool ok = true, nz = false;
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const int f = r % 3 - 1;
                r /= 3;
                const int l = c[d] - T[d];
                ok = ok && (f == 0 || (f < 0 ? l == 0 : l == S.pt[d] - 1));
                const int tcd = tc[d] + f;
                ok = ok && tcd >= 0 && tcd < S.npt[d];
                nz = nz || f != 0;
                nt += tcd * mul;
                mul *= S.npt[d];
            }
            if (ok && nz) atomicAdd(&S.fcnt[nt], 1);
        }
    }
}

// ... then the slots of set 1 - q: exclusive scan of tnum[q] + fcnt (one block)
__global__ void __launch_bounds__(1024) k_next_slots(const SimDev* __restrict__ sim, int q)
{
    const SimDev& S = *sim;
    __shared__ int s_warp[32];
    const int n = S.nptiles;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int per = (n + nth - 1) / nth;
    const int i0 = min(n, tid * per), i1 = min(n, i0 + per);
    int lk = 0;
    for (int i = i0; i < i1; ++i) lk += S.tnum[q][i] + S.fcnt[i];
    int rk = block_exclusive_scan(lk, s_warp);
    for (int i = i0; i < i1; ++i) {
        S.toff[1 - q][i] = rk;
        rk += S.tnum[q][i] + S.fcnt[i];
        S.fcnt[i] = 0;
    }
    if (tid == nth - 1) S.toff[1 - q][n] = rk;
}

// Tile scan of one simulation over several blocks (decoupled look-back): block b (in the
// order blocks start, from a ticket) scans tiles [4096 b, 4096 (b + 1)), publishes its
// aggregate, then adds the totals of the blocks before it -- each published as
// (status << 62) | (slots << 31) | chunks, status 1 aggregate, 2 inclusive prefix --
// waiting (bounded) only on blocks that started earlier.  A wait that gives up flags a
// timeout and takes prefix 0, which keeps every offset inside the particle arrays.
// Outputs as scan_counts (not compact).
__global__ void __launch_bounds__(1024) k_scan_lb(const SimDev* __restrict__ sims)
{
    const SimDev& S = sims[0];
    __shared__ int s_warp[32];
    __shared__ int s_cnt[4096];
    __shared__ int s_tk, s_tc, s_pk, s_pc;
    __shared__ int s_b;
    const int tid = threadIdx.x;
    if (tid == 0) s_b = atomicAdd(S.scanticket, 1);
    __syncthreads();
    const int b = s_b, n = S.nptiles, base = b * 4096;
    const int q = 1 - S.st->parity;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = base + k * 1024 + tid;
        s_cnt[k * 1024 + tid] = i < n ? S.tcnt[i] : 0;
    }
    __syncthreads();
    int c4[4], f4[4], lp = 0, lc = 0, lk = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = base + tid * 4 + k;
        c4[k] = s_cnt[tid * 4 + k];
        f4[k] = i < n ? S.fcnt[i] : 0;
        lp += c4[k];
        lc += (c4[k] + S.chunk - 1) / S.chunk;
        lk += c4[k] + f4[k];
    }
    int rp = block_exclusive_scan(lp, s_warp);
    int rc = block_exclusive_scan(lc, s_warp);
    int rk = block_exclusive_scan(lk, s_warp);
    if (tid == 1023) {
        s_tk = rk + lk;
        s_tc = rc + lc;
        atomicAdd(&S.st->n_next, rp + lp);
    }
    __syncthreads();
    if (tid == 0) {
        unsigned long long* fl = S.scanflags;
        const unsigned long long agg = ((unsigned long long)s_tk << 31) | (unsigned long long)s_tc;
        long long pk = 0, pc = 0;
        // a held block (test aid) publishes nothing: the blocks after it wait out their bound
        const bool publish = b != S.scan_hold;
        if (b == 0) {
            if (publish) atomicExch(&fl[0], (2ull << 62) | agg);
        } else {
            if (publish) atomicExch(&fl[b], (1ull << 62) | agg);
            bool ok = true;
            const int limit = S.scan_spins;
            for (int j = b - 1; j >= 0; --j) {
                unsigned long long f = 0;
                int spins = 0;
                do {
                    f = *reinterpret_cast<volatile unsigned long long*>(&fl[j]);
                } while ((f >> 62) == 0 && ++spins < limit);
                if ((f >> 62) == 0) {
                    ok = false;
                    break;
                }
                pk += (long long)((f >> 31) & 0x7FFFFFFFull);
                pc += (long long)(f & 0x7FFFFFFFull);
                if ((f >> 62) == 2) break;
            }
            if (!ok) {
                atomicOr(&S.st->status, (unsigned)FLAG_TIMEOUT);
                pk = pc = 0;
            }
            if (publish)
                atomicExch(&fl[b], (2ull << 62) | ((unsigned long long)(pk + s_tk) << 31) |
                                       (unsigned long long)(pc + s_tc));
        }
        s_pk = (int)pk;
        s_pc = (int)pc;
    }
    __syncthreads();
    rk += s_pk;
    rc += s_pc;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = base + tid * 4 + k;
        if (i >= n) break;
        const int c = c4[k];
        S.tnum[q][i] = c;
        S.coff[q][i] = rc;
        write_chunks(S, q, i, S.toff[q][i], c, rc);
        S.toff[1 - q][i] = rk;
        rc += (c + S.chunk - 1) / S.chunk;
        rk += c + f4[k];
        S.tcnt[i] = 0;
        S.tcur[i] = 0;
        S.fcnt[i] = 0;
        if (i == n - 1) {
            S.toff[1 - q][n] = rk;
            S.coff[q][n] = rc;
        }
    }
}

// First node of every step: number the chunks of the group's simulations and reset the
// work counters (and the multi-block scan's flags of a single simulation).
__global__ void __launch_bounds__(1024) k_prefix(const SimDev* __restrict__ sims, int nsims, int* __restrict__ gprefix,
                                                 int* __restrict__ counters)
{
    __shared__ int s_warp[32];
    const int tid = threadIdx.x, nth = blockDim.x;
    const int per = (nsims + nth - 1) / nth;
    const int i0 = min(nsims, tid * per), i1 = min(nsims, i0 + per);
    int l = 0;
    for (int i = i0; i < i1; ++i) l += sims[i].coff[sims[i].st->parity][sims[i].nptiles];
    int r = block_exclusive_scan(l, s_warp);
    for (int i = i0; i < i1; ++i) {
        gprefix[i] = r;
        r += sims[i].coff[sims[i].st->parity][sims[i].nptiles];
    }
    if (tid == nth - 1) gprefix[nsims] = r;
    if (tid < 4) counters[tid] = 0;
    if (nsims == 1) {
        const SimDev& S = sims[0];
        for (int j = tid; j < S.nscanblk; j += nth) S.scanflags[j] = 0ull;
        if (tid == 0) *S.scanticket = 0;
    }
}

template <int D, typename R>
__device__ __forceinline__ void copy_particle(const SimDev& S, int from, long long p, int to, long long q)
{
    S.cell[to][q] = S.cell[from][p];
#pragma unroll
    for (int d = 0; d < D; ++d)
        reinterpret_cast<R*>(S.off[to][d])[q] = reinterpret_cast<const R*>(S.off[from][d])[p];
#pragma unroll
    for (int d = 0; d < 3; ++d)
        reinterpret_cast<R*>(S.mom[to][d])[q] = reinterpret_cast<const R*>(S.mom[from][d])[p];
    reinterpret_cast<R*>(S.wgt[to])[q] = reinterpret_cast<const R*>(S.wgt[from])[p];
    S.pid[to][q] = S.pid[from][p];
}


// Cell of c as an index of the tile-major cell arrays: tile * tvol + the cell's rank
// within its tile, x fastest (the order the seeded slab is placed in).
template <int D>
__device__ __forceinline__ int cell_key(const SimDev& S, const int c[3], int* tile)
{
    int t = 0, r = 0;
    const int q0 = c[0] / S.pt[0];
    t = q0;
    r = c[0] - q0 * S.pt[0];
    if constexpr (D > 1) {
        const int q1 = c[1] / S.pt[1];
        t += S.npt[0] * q1;
        r += S.pt[0] * (c[1] - q1 * S.pt[1]);
    }
    if constexpr (D > 2) {
        const int q2 = c[2] / S.pt[2];
        t += S.npt[0] * S.npt[1] * q2;
        r += S.pt[0] * S.pt[1] * (c[2] - q2 * S.pt[2]);
    }
    *tile = t;
    return t * S.tvol + r;
}

constexpr int SCATTER_NP = 2;

// Cell-sort scatter of one chunk per work item (simulations with a cell sort, pushed in
// place this step): each warp reserves destination slots with one atomic per distinct cell
// among its lanes (lanes of one cell write consecutive slots), after the cell's offset
// within its tile, so that every tile of the other buffer set comes out ordered by cell.
template <int D, typename R>
__global__ void __launch_bounds__(256) k_scatter(const SimDev* __restrict__ sims, int nsims,
                                                 const int* __restrict__ gprefix, int* __restrict__ counter)
{
    __shared__ int s_item;
    const int tid = threadIdx.x, nth = blockDim.x;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= gprefix[nsims]) break;
        const ChunkRef ck = chunk_of(sims, nsims, gprefix, item);
        const SimDev& S = sims[ck.sim];
        if (S.ccur == nullptr) continue;     // placed by the push
        const int par = S.st->parity, np = 1 - par;
        // SCATTER_NP particles per thread and round, all their loads issued before the slot
        // reservations (more loads in flight per thread)
        for (int base = ck.p0; base < ck.p1; base += SCATTER_NP * nth) {
            unsigned cl[SCATTER_NP], id[SCATTER_NP];
            R of[SCATTER_NP][D], mo[SCATTER_NP][3], wv[SCATTER_NP];
#pragma unroll
            for (int k = 0; k < SCATTER_NP; ++k) {
                const int p = base + k * nth + tid;
                cl[k] = DEAD;
                if (p < ck.p1) {
                    cl[k] = S.cell[par][p];
#pragma unroll
                    for (int d = 0; d < D; ++d) of[k][d] = reinterpret_cast<const R*>(S.off[par][d])[p];
#pragma unroll
                    for (int d = 0; d < 3; ++d) mo[k][d] = reinterpret_cast<const R*>(S.mom[par][d])[p];
                    wv[k] = reinterpret_cast<const R*>(S.wgt[par])[p];
                    id[k] = S.pid[par][p];
                }
            }
#pragma unroll
            for (int k = 0; k < SCATTER_NP; ++k) {
                int t = -1, key = -1;
                if (cl[k] != DEAD) {
                    int c[3];
                    decode_cell<D>(S, cl[k], c);
                    key = cell_key<D>(S, c, &t);
                }
                const int slot = warp_reserve(key, S.ccur);
                if (t >= 0) {
                    const long long q = (long long)S.toff[np][t] + slot;
                    S.cell[np][q] = cl[k];
#pragma unroll
                    for (int d = 0; d < D; ++d) reinterpret_cast<R*>(S.off[np][d])[q] = of[k][d];
#pragma unroll
                    for (int d = 0; d < 3; ++d) reinterpret_cast<R*>(S.mom[np][d])[q] = mo[k][d];
                    reinterpret_cast<R*>(S.wgt[np])[q] = wv[k];
                    S.pid[np][q] = id[k];
                }
            }
        }
    }
}

// Cell sort, first pass: per-cell counts of the pushed particles (buffer set `parity`, new
// cells), one atomic per distinct cell among a warp's lanes.
template <int D>
__global__ void __launch_bounds__(256) k_cellcount(const SimDev* __restrict__ sims, int nsims,
                                                   const int* __restrict__ gprefix, int* __restrict__ counter)
{
    __shared__ int s_item;
    const int tid = threadIdx.x, nth = blockDim.x;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= gprefix[nsims]) break;
        const ChunkRef ck = chunk_of(sims, nsims, gprefix, item);
        const SimDev& S = sims[ck.sim];
        if (S.ccnt == nullptr) continue;
        const int par = S.st->parity;
        for (int base = ck.p0; base < ck.p1; base += nth) {
            const int p = base + tid;
            int key = -1;
            if (p < ck.p1) {
                const unsigned cl = S.cell[par][p];
                if (cl != DEAD) {
                    int c[3], t;
                    decode_cell<D>(S, cl, c);
                    key = cell_key<D>(S, c, &t);
                }
            }
            const unsigned peers = __match_any_sync(0xffffffffu, key);
            if (key >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&S.ccnt[key], __popc(peers));
        }
    }
}

// Cell sort, second pass: per tile (blocks stride over the tiles of simulation blockIdx.y),
// exclusive scan of the cell counts into the write cursors; the counts are cleared for the
// next sort.
__global__ void __launch_bounds__(256) k_cellscan(const SimDev* __restrict__ sims)
{
    const SimDev& S = sims[blockIdx.y];
    if (S.ccnt == nullptr) return;
    __shared__ int s_warp[32];
    __shared__ int s_total;
    const int tid = threadIdx.x, tv = S.tvol;
    for (int t = blockIdx.x; t < S.nptiles; t += gridDim.x) {
        const long long base = (long long)t * tv;
        int carry = 0;
        for (int i0 = 0; i0 < tv; i0 += 4 * 256) {
            int v[4], sum = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int i = i0 + 4 * tid + k;
                v[k] = i < tv ? S.ccnt[base + i] : 0;
                sum += v[k];
            }
            int run = carry + block_exclusive_scan(sum, s_warp);
            if (tid == 255) s_total = run + sum;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int i = i0 + 4 * tid + k;
                if (i < tv) {
                    S.ccur[base + i] = run;
                    S.ccnt[base + i] = 0;
                }
                run += v[k];
            }
            __syncthreads();
            carry = s_total;
            __syncthreads();
        }
    }
}

// Last node of every step: step counter, particle count and buffer parity of every
// simulation of the group, then the next step's chunk numbering and work counters (what
// k_prefix does), so that a step of the same group needs no k_prefix of its own.
__global__ void __launch_bounds__(1024) k_step_end(const SimDev* __restrict__ sims, int nsims,
                                                   int* __restrict__ gprefix, int* __restrict__ counters)
{
    __shared__ int s_warp[32];
    const int tid = threadIdx.x, nth = blockDim.x;
    const int per = (nsims + nth - 1) / nth;
    const int i0 = min(nsims, tid * per), i1 = min(nsims, i0 + per);
    int l = 0;
    for (int i = i0; i < i1; ++i) {
        const SimDev& S = sims[i];
        DevState* st = S.st;
        const int np = 1 - st->parity;
        st->n_alive = st->n_next;
        st->n_next = 0;
        st->parity = np;
        st->step += 1;
        l += S.coff[np][S.nptiles];
    }
    int r = block_exclusive_scan(l, s_warp);
    for (int i = i0; i < i1; ++i) {
        gprefix[i] = r;
        r += sims[i].coff[sims[i].st->parity][sims[i].nptiles];   // the parity this thread just set
    }
    if (tid == nth - 1) gprefix[nsims] = r;
    if (tid < 4) counters[tid] = 0;
    if (nsims == 1) {
        const SimDev& S = sims[0];
        for (int j = tid; j < S.nscanblk; j += nth) S.scanflags[j] = 0ull;
        if (tid == 0) *S.scanticket = 0;
    }
}

// Incident field on the Yee nodes (the prescribed-field route): one block per row segment of
// 256 x-nodes (blockIdx.x = row * segs + segment) of one simulation (blockIdx.y); each node evaluates the closed form once per distinct
// half-cell offset pattern of the staggered components (2^dim patterns, 2 in 1D, 4 in 2D,
// 6 used in 3D) and writes total = scattered + incident into components COMP_TOTAL..+5.
template <int D, typename R>
__global__ void __launch_bounds__(256) k_incident_grid(const SimDev* __restrict__ sims, int segs)
{
    const SimDev& S = sims[blockIdx.y];
    if (!S.incgrid) return;
    const int ext0 = S.n[0] + 1, ext1 = D > 1 ? S.n[1] + 1 : 1, ext2 = D > 2 ? S.n[2] + 1 : 1;
    const int row = blockIdx.x / segs, x0 = (blockIdx.x % segs) * 256;
    if (row >= ext1 * ext2 || x0 >= ext0) return;
    __shared__ PhaseRef<R> s_pr;
    const DevState* st = S.st;
    if (threadIdx.x == 0) s_pr = phase_ref<R>(S, (double)st->step * S.dt, x0);
    __syncthreads();
    const int x = x0 + threadIdx.x;
    if (x >= ext0) return;
    const int y = row % ext1, z = row / ext1;
    const PhaseRef<R> pr = s_pr;
    const BeamC<R>& bc = beam_of<R>(S);
    R* F = reinterpret_cast<R*>(S.F);
    const long long base = (long long)(D > 2 ? z + G : 0) * S.sz + (long long)(D > 1 ? y + G : 0) * S.sy + (x + GX);
    const long long eb = (long long)comp_eb(st->parity) * S.sc;
    const long long tb = (long long)COMP_TOTAL * S.sc;
    const int c[3] = {x, y, z};
#pragma unroll
    for (int m = 0; m < (1 << D); ++m) {
        // components whose stagger pattern is m: E_q half a cell along axis q, B_q along the others
        int mask = 0;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            int pat = 0;
#pragma unroll
            for (int d = 0; d < D; ++d)
                if (q < 3 ? d == q : d != q - 3) pat |= 1 << d;
            if (pat == m) mask |= 1 << q;
        }
        if (!mask) continue;
        const R o[3] = {(m & 1) ? R(0.5) : R(0), (m & 2) ? R(0.5) : R(0), (m & 4) ? R(0.5) : R(0)};
        R Ei[3], Bi[3];
        incident_at<D, R>(S, bc, pr, c, o, Ei, Bi);
#pragma unroll
        for (int q = 0; q < 6; ++q)
            if (mask & (1 << q)) F[tb + q * S.sc + base] = F[eb + q * S.sc + base] + (q < 3 ? Ei[q] : Bi[q - 3]);
    }
}

// ---- set-up ----------------------------------------------------------------------
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed, unsigned long long k)
{
    // SplitMix64 (Steele, Lea & Flood 2014): k-th output of the stream seeded with `seed`
    unsigned long long z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Seeded slab into buffer set 1, linear order; counts per tile.
template <int D, typename R>
__global__ void k_gen_slab(const SimDev* __restrict__ sim, long long n, int ppc, int lo0, int lo1, int lo2, int n0,
                           int n1, unsigned long long seed, double weight)
{
    const SimDev& S = *sim;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const long long cellp = p / ppc;
        const int lo[3] = {lo0, lo1, lo2};
        const long long rel[3] = {cellp % n0, (cellp / n0) % n1, cellp / ((long long)n0 * n1)};
        int c[3] = {0, 0, 0};
        double x0 = 0.0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            c[d] = lo[d] + (int)rel[d];
            const unsigned long long r = splitmix64(seed, 3ull * (unsigned long long)p + d);
            const double offd = (double)(r >> 40) * (1.0 / 16777216.0);
            reinterpret_cast<R*>(S.off[1][d])[p] = R(offd);
            if (d == 0) x0 = ((double)c[0] + offd) * S.dx;
        }
        // density profile along x (Sec. 3.1's super-Gaussian) at the initial position
        double f = 1.0;
        if (S.profile == 1)
            f = x0 <= S.prof_cut ? 0.0 : exp2(-pow(fabs(2.0 * (x0 - S.prof_x0) / S.prof_fwhm), (double)S.prof_order));
#pragma unroll
        for (int d = 0; d < 3; ++d) reinterpret_cast<R*>(S.mom[1][d])[p] = R(0);
        reinterpret_cast<R*>(S.wgt[1])[p] = R(weight * f);
        S.pid[1][p] = (unsigned)p;
        S.cell[1][p] = encode_cell<D>(S, c);
        atomicAdd(&S.tcnt[tile_of<D>(S, c)], 1);
    }
}

template <int D>
__global__ void k_count_linear(const SimDev* __restrict__ sim, long long n)
{
    const SimDev& S = *sim;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        int c[3];
        decode_cell<D>(S, S.cell[1][p], c);
        atomicAdd(&S.tcnt[tile_of<D>(S, c)], 1);
    }
}

// Set 1 (linear) -> set 0 (sorted by tile); toff[0] already scanned.
template <int D, typename R>
__global__ void k_sort_linear(const SimDev* __restrict__ sim, long long n)
{
    const SimDev& S = *sim;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long nround = (n + stride - 1) / stride * stride;   // uniform trip count per warp
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < nround; p += stride) {
        int t = -1;
        if (p < n) {
            int c[3];
            decode_cell<D>(S, S.cell[1][p], c);
            t = tile_of<D>(S, c);
        }
        const int slot = warp_reserve(t, S.tcur);
        if (t >= 0) copy_particle<D, R>(S, 1, p, 0, (long long)S.toff[0][t] + slot);
    }
}

// Seeded slab, set 1 (generation order: ppc particles per slab cell, x fastest) -> set 0,
// placed directly in cell order within each tile: a particle of cell c goes to
// toff[tile] + (rank of c among the tile's slab cells, x fastest) ppc + (its index in c).
template <int D, typename R>
__global__ void k_place_slab(const SimDev* __restrict__ sim, long long n, int ppc, int lo0, int lo1, int lo2,
                             int hi0, int hi1, int hi2)
{
    const SimDev& S = *sim;
    const int slo[3] = {lo0, lo1, lo2}, shi[3] = {hi0, hi1, hi2};
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        int c[3];
        decode_cell<D>(S, S.cell[1][p], c);
        const int t = tile_of<D>(S, c);
        long long rank = 0, width = 1;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int a = max(slo[d], (c[d] / S.pt[d]) * S.pt[d]);
            const int b = min(shi[d], (c[d] / S.pt[d] + 1) * S.pt[d]);
            rank += (c[d] - a) * width;
            width *= (b - a);
        }
        copy_particle<D, R>(S, 1, p, 0, (long long)S.toff[0][t] + rank * ppc + (p % ppc));
    }
}

// ---- host launch wrappers ------------------------------------------------------------
template <int D, typename R>
static void push_t(const Group& g, bool sorting, cudaStream_t s)
{
    if (g.one)
        k_push1<D, R><<<g.push_grid, push_threads<D, R>(), g.push_smem, s>>>(*g.one, g.gprefix, g.counters + 0,
                                                                              sorting ? 1 : 0);
    else
        k_push<D, R><<<g.push_grid, push_threads<D, R>(), g.push_smem, s>>>(g.sims, g.nsims, g.gprefix,
                                                                             g.counters + 0, sorting ? 1 : 0);
}
template <int D, typename R>
static void cellsort_t(const Group& g, cudaStream_t s)
{
    k_cellcount<D><<<g.scatter_grid, 256, 0, s>>>(g.sims, g.nsims, g.gprefix, g.counters + 3);
    k_cellscan<<<dim3((unsigned)g.cellscan_grid, (unsigned)g.nsims), 256, 0, s>>>(g.sims);
    k_scatter<D, R><<<g.scatter_grid, 256, 0, s>>>(g.sims, g.nsims, g.gprefix, g.counters + 1);
}

#define SFF_DISPATCH(dim, prec, FN, ...)                                 \
    do {                                                                 \
        if ((prec) == 0) {                                               \
            if ((dim) == 1) FN<1, double>(__VA_ARGS__);                  \
            else if ((dim) == 2) FN<2, double>(__VA_ARGS__);             \
            else FN<3, double>(__VA_ARGS__);                             \
        } else {                                                         \
            if ((dim) == 1) FN<1, float>(__VA_ARGS__);                   \
            else if ((dim) == 2) FN<2, float>(__VA_ARGS__);              \
            else FN<3, float>(__VA_ARGS__);                              \
        }                                                                \
    } while (0)

void launch_push(const Group& g, bool sorting, cudaStream_t s) { SFF_DISPATCH(g.dim, g.prec, push_t, g, sorting, s); }
void launch_cell_sort(const Group& g, cudaStream_t s) { SFF_DISPATCH(g.dim, g.prec, cellsort_t, g, s); }
void launch_scan(const Group& g, cudaStream_t s)
{
    // a single simulation scans its tiles over several blocks; a batch, one block per member
    if (g.nsims == 1) k_scan_lb<<<g.scan_blocks, 1024, 0, s>>>(g.sims);
    else k_scan<<<g.nsims, 1024, 0, s>>>(g.sims);
}
void launch_prefix(const Group& g, cudaStream_t s) { k_prefix<<<1, 1024, 0, s>>>(g.sims, g.nsims, g.gprefix, g.counters); }
void launch_step_end(const Group& g, cudaStream_t s)
{
    k_step_end<<<1, 1024, 0, s>>>(g.sims, g.nsims, g.gprefix, g.counters);
}

template <int D, typename R>
static void incgrid_t(const Group& g, cudaStream_t s)
{
    const dim3 grid((unsigned)g.inc_segs * (unsigned)g.inc_rows, g.nsims);
    k_incident_grid<D, R><<<grid, 256, 0, s>>>(g.sims, g.inc_segs);
}

void launch_incident_grid(const Group& g, cudaStream_t s)
{
    if (!g.inc_any) return;
    if (g.prec == 0) {
        if (g.dim == 1) incgrid_t<1, double>(g, s);
        else if (g.dim == 2) incgrid_t<2, double>(g, s);
        else incgrid_t<3, double>(g, s);
    } else {
        if (g.dim == 1) incgrid_t<1, float>(g, s);
        else if (g.dim == 2) incgrid_t<2, float>(g, s);
        else incgrid_t<3, float>(g, s);
    }
}
void launch_scan_one(const SimDev* sim, int q, cudaStream_t s) { k_scan_one<<<1, 1024, 0, s>>>(sim, q); }

template <int D, typename R>
static void frame_t(const SimDev* sim, int q, long long n, cudaStream_t s)
{
    const int grid = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, (long long)device_sms() * 16));
    if (n > 0) k_frame_linear<D><<<grid, 256, 0, s>>>(sim, q, n);
    k_next_slots<<<1, 1024, 0, s>>>(sim, q);
}
void launch_next_slots(const SimDev* sim, int dim, int prec, int q, long long n, cudaStream_t s)
{
    SFF_DISPATCH(dim, prec, frame_t, sim, q, n, s);
}

template <int D, typename R>
static void gen_t(const SimDev* sim, long long n, int ppc, const int lo[3], const int sn[3], unsigned long long seed,
                  double w, cudaStream_t s)
{
    const int grid = (int)std::min<long long>((n + 255) / 256, (long long)device_sms() * 16);
    if (n > 0) k_gen_slab<D, R><<<grid, 256, 0, s>>>(sim, n, ppc, lo[0], lo[1], lo[2], sn[0], sn[1], seed, w);
}
void launch_gen_slab(const SimDev* sim, int dim, int prec, long long n, int ppc, const int slab_lo[3],
                     const int slab_n[3], unsigned long long seed, double weight, cudaStream_t s)
{
    SFF_DISPATCH(dim, prec, gen_t, sim, n, ppc, slab_lo, slab_n, seed, weight, s);
}

template <int D, typename R>
static void count_t(const SimDev* sim, long long n, cudaStream_t s)
{
    const int grid = (int)std::min<long long>((n + 255) / 256, (long long)device_sms() * 16);
    if (n > 0) k_count_linear<D><<<grid, 256, 0, s>>>(sim, n);
}
void launch_count_linear(const SimDev* sim, int dim, int prec, long long n, cudaStream_t s)
{
    SFF_DISPATCH(dim, prec, count_t, sim, n, s);
}

template <int D, typename R>
static void sortlin_t(const SimDev* sim, long long n, cudaStream_t s)
{
    const int grid = (int)std::min<long long>((n + 255) / 256, (long long)device_sms() * 16);
    if (n > 0) k_sort_linear<D, R><<<grid, 256, 0, s>>>(sim, n);
}
template <int D, typename R>
static void place_t(const SimDev* sim, long long n, int ppc, const int lo[3], const int hi[3], cudaStream_t s)
{
    const int grid = (int)std::min<long long>((n + 255) / 256, (long long)device_sms() * 16);
    if (n > 0) k_place_slab<D, R><<<grid, 256, 0, s>>>(sim, n, ppc, lo[0], lo[1], lo[2], hi[0], hi[1], hi[2]);
}
void launch_place_slab(const SimDev* sim, int dim, int prec, long long n, int ppc, const int lo[3], const int hi[3],
                       cudaStream_t s)
{
    SFF_DISPATCH(dim, prec, place_t, sim, n, ppc, lo, hi, s);
}

void launch_sort_linear(const SimDev* sim, int dim, int prec, long long n, cudaStream_t s)
{
    SFF_DISPATCH(dim, prec, sortlin_t, sim, n, s);
}

template <int D, typename R>
static void attr_push(size_t smem, int* out)
{
    cudaFuncSetAttribute(k_push<D, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_push1<D, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int a = 0, b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_push<D, R>, push_threads<D, R>(), smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_push1<D, R>, push_threads<D, R>(), smem);
    *out = std::min(a, b);
}
int prepare_push(int dim, int prec, size_t smem)
{
    int b = 0;
    SFF_DISPATCH(dim, prec, attr_push, smem, &b);
    return b;
}

template <int D, typename R>
static void attr_scatter(int* out)
{
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_scatter<D, R>, 256, 0);
}
int scatter_blocks_per_sm(int dim, int prec)
{
    int b = 0;
    SFF_DISPATCH(dim, prec, attr_scatter, &b);
    return b;
}

}  // namespace sff
