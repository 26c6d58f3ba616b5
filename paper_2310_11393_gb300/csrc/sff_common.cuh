// Internal definitions shared by the kernels and the C-ABI of the GB300 (sm_103a)
// scattered-field PIC library: per-simulation device descriptor, grid layout,
// inline-PTX wrappers for mbarrier / TMA (cp.async.bulk.tensor) and a small
// complex type.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sff {

// Ghost points stored below (and at least this many above) every resolved axis.
// Four keeps every TMA box start on the x axis a multiple of four elements.
constexpr int G = 4;
// ghost width along x: a multiple of 8, so that a tile starting on a multiple of 32 points
// starts on a 32-byte sector (whole-sector stores of the field solver)
constexpr int GX = 8;
constexpr int NCOMP = 9;           // Ex Ey Ez Bx By Bz Jx Jy Jz
constexpr unsigned DEAD = 0xFFFFFFFFu;
constexpr int EXIT_DOUBLES = 6;    // u[3], w, id, step

enum Beam { BEAM_NONE = 0, BEAM_PLANE = 1, BEAM_LP = 2, BEAM_RP = 3, BEAM_UNIFORM = 4, BEAM_GAUSS2D = 5 };
enum Flag { FLAG_TIMEOUT = 1u, FLAG_CFL = 2u, FLAG_EXIT_OVERFLOW = 4u, FLAG_CAPACITY = 8u };

// Device-updated state of one simulation.
struct DevState {
    long long step;       // steps taken; time = step * dt
    int parity;           // which particle buffer set is current
    int n_alive;
    int n_exits;          // exit records claimed (may exceed capacity; then FLAG_EXIT_OVERFLOW)
    unsigned status;
    int n_next;           // particles placed by the running step (summed by the tile scan)
    float wmax;           // largest |weight| of the particles: the scale of the FP32 push's
                          // fixed-point current (set by pic_init and pic_set_particles; kept
                          // here, not in SimDev, so that batch copies of SimDev see updates)
    long long pad[4];
};

// Incident-field constants in the working precision R, computed on the host at set-up.
template <typename R>
struct BeamC {
    int beam, envelope;
    R a, inv_a, two_a, s, inv_s, sp1, sp2, k, phi0, ring2;   // ring2 = delta^4: series when |u|^2 < delta^4
    R a0, dur, inv_dur, t_c;                                  // plane wave
    R dxr;                                                    // cell size
    R eu[3], bu[3];
    // push constants: q dt/2 (q = -1), dt/dx, -q dx/dt, focus offset within its cell per axis
    R hq, dtdx, jfac, frf[3];
    // 2D Gaussian beam: w0, 1/z_R, 1/w0^2, carrier phase offset (phi0 - t_focus) mod 2 pi
    R gw0, ginv_zr, ginv_w02, cph;
};

// Field-solver constants in the working precision R, computed on the host at set-up.
template <typename R>
struct YeeC {
    R cdt;   // dt/dx
    R hc;    // dt/(2 dx)
    R dt;
    R km;    // (dt - dx)/(dt + dx), first-order Mur
};

// Everything a kernel needs to know about one simulation.  Lives in device memory
// (an array of these serves a batch); tensor maps must stay 64-byte aligned.
struct alignas(128) SimDev {
    CUtensorMap tm_pf;        // push box, field comps 0..5 (load)
    CUtensorMap tm_pj;        // push box, current comps 6..8 (reduce-add, FP32)
    CUtensorMap tm_yin;       // field-solver box, E and B comps (load)
    CUtensorMap tm_yj;        // field-solver box, J comps (load)
    CUtensorMap tm_yout;      // field-solver tile, E and B comps (store)

    int dim, prec, beam, envelope;
    int n[3];                 // cells per axis (1 on unresolved axes)
    int na[3];                // allocated points per axis (1 on unresolved axes)
    long long sy, sz, sc;     // element strides of y, z and component
    int pt[3], npt[3];        // particle tile (cells) and tiles per axis
    int nptiles;
    int pb[3];                // particle box extent per axis
    int yt[3], nyt[3];        // field-solver tile and tiles per axis
    int nytiles;
    int yb[3];                // field-solver box extent per axis
    int cb[3];                // bits of each cell coordinate in the packed cell index
    int margin;
    int pusher;               // 0 Boris, 1 Vay, 2 Higuera-Cary
    int tf;                   // total-field run: incident wave injected at x = 0, not at particles
    int incgrid;              // incident field on the grid (components COMP_TOTAL..+5 hold the total)
    double dx, dt, inv_dx;
    // incident field
    double a0, duration, phi0, t_focus, a, s, psi0, w0;
    // slab density profile (PIC_PROFILE_*)
    int profile, prof_order;
    double prof_x0, prof_fwhm, prof_cut;
    double focus[3];
    double e_unif[3], b_unif[3];
    int icf[3];               // focus = (icf + frf) * dx per axis
    float frf[3];
    // device buffers
    void* F;                  // fields: [9][na_z][na_y][na_x], element (0,0,0) is a ghost corner
    // Particle buffer sets: tile t of set q owns slots [toff[q][t], toff[q][t+1]) and holds
    // its tnum[q][t] particles in the first of them; the slack after them bounds exactly
    // the particles one step can bring in (those within one cell outside the tile).
    unsigned* cell[2];        // packed cell index per particle (DEAD = removed)
    void* off[2][3];          // in-cell offset in [0,1) per resolved axis
    void* mom[2][3];          // momentum gamma*v
    void* wgt[2];
    unsigned* pid[2];
    int* toff[2];             // first slot of each tile [nptiles + 1] of each buffer set
    int* tnum[2];             // particles of each tile [nptiles] of each buffer set
    int* coff[2];             // chunk offsets [nptiles + 1]: tile t owns chunks coff[t] .. coff[t+1]-1
    int* ctile[2];            // chunk -> tile map [max_chunks]
    int2* crange[2];          // chunk -> particle slots [p0, p1) [max_chunks]
    int chunk;                // particles per chunk (the unit of work of push and scatter)
    int lane_p;               // push lane stride: particles per cell rounded down to 1, 2, 4 or 8
    int max_chunks;
    int* tcnt;                // per-tile counts of the next step
    int* tcur;                // per-tile write cursors of the push
    int* fcnt;                // per-tile frame counts of the next step: particles within one
                              // cell outside the tile (the most that can enter it in a step)
    int* ccnt;                // cell sort: per-cell counts [nptiles][tvol] (tile-major, x fastest
                              // within a tile), zero between sorts; NULL without cell sort
    int* ccur;                // cell sort: per-cell write cursors (offsets within the tile)
    int tvol;                 // cells per particle tile
    unsigned long long* scanflags;   // multi-block tile scan: per block status | particles | chunks
    int* scanticket;          // multi-block tile scan: block order ticket
    int nscanblk;             // blocks of the multi-block tile scan (tiles / 4096, rounded up)
    int scan_spins;           // polls of a predecessor's flag before the look-back gives up
    int scan_hold;            // test aid: this scan block publishes nothing (-1: none)
    double* exits;            // [max_exits][EXIT_DOUBLES]
    long long max_exits;
    long long cap;            // slots per buffer set (frame factor x particle capacity)
    DevState* st;
    double* rho_ion;          // [na_z][na_y][na_x] ion charge density (diagnostics)
    double* scratch;          // diagnostics scratch: charge density, same layout
    BeamC<float> bcf;         // incident-field constants for the FP32 kernels
    BeamC<double> bcd;        // ... and the FP64 kernels
    YeeC<float> ycf;          // field-solver constants, FP32 and FP64
    YeeC<double> ycd;
};

template <typename R>
__device__ __forceinline__ const YeeC<R>& yee_of(const SimDev& S)
{
    if constexpr (sizeof(R) == 4) return S.ycf;
    else return S.ycd;
}

template <typename R>
__device__ __forceinline__ const BeamC<R>& beam_of(const SimDev& S)
{
    if constexpr (sizeof(R) == 4) return S.bcf;
    else return S.bcd;
}

struct Work {
    int sim;
    int tile;
};


// ---------------------------------------------------------------------------------
// inline PTX: shared-memory addresses, mbarrier, TMA
// ---------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// smem sub-buffers used by TMA start on 128-byte boundaries
__host__ __device__ constexpr size_t round128(size_t b) { return (b + 127) & ~size_t(127); }

// acquire a tensor map that was written to global memory before the launch
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap* tm)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(tm))
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase: gives up after ~2^31 SM clocks (about one
// second at 2 GHz) or 2^22 polls, whichever comes first.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity)
{
    long long t0 = clock64();
    for (int i = 0; i < (1 << 22); ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > (1ll << 31)) break;
    }
    return false;
}

// TMA tiled loads into shared memory, completion counted on `bar`.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int c0, int c1, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int c0, int c1, int c2, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* tm, int c0, int c1, int c2, int c3,
                                            uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

// TMA element-wise add of a shared-memory box into global memory (performed at L2).
__device__ __forceinline__ void tma_reduce_add_2d(const CUtensorMap* tm, int c0, int c1, const void* src)
{
    asm volatile("cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(tm)),
                 "r"(c0), "r"(c1), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void tma_reduce_add_3d(const CUtensorMap* tm, int c0, int c1, int c2, const void* src)
{
    asm volatile("cp.reduce.async.bulk.tensor.3d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                     reinterpret_cast<uint64_t>(tm)),
                 "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void tma_reduce_add_4d(const CUtensorMap* tm, int c0, int c1, int c2, int c3,
                                                  const void* src)
{
    asm volatile(
        "cp.reduce.async.bulk.tensor.4d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(
            reinterpret_cast<uint64_t>(tm)),
        "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(src))
        : "memory");
}

// TMA tiled stores from shared memory.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* tm, int c0, int c1, const void* src)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(tm)),
                 "r"(c0), "r"(c1), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* tm, int c0, int c1, int c2, const void* src)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                     reinterpret_cast<uint64_t>(tm)),
                 "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* tm, int c0, int c1, int c2, int c3, const void* src)
{
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(
                     reinterpret_cast<uint64_t>(tm)),
                 "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(src))
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// L2 prefetch of a tensor box (no shared memory, no completion to wait for).
__device__ __forceinline__ void tma_prefetch_4d(const CUtensorMap* tm, int c0, int c1, int c2, int c3)
{
    asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];" ::"l"(
                     reinterpret_cast<uint64_t>(tm)),
                 "r"(c0), "r"(c1), "r"(c2), "r"(c3)
                 : "memory");
}

// Box load / reduce / store dispatch on the tensor rank (dim + 1: x, [y, [z,]] component).
template <int D>
__device__ __forceinline__ void tma_load_box(void* dst, const CUtensorMap* tm, const int c[3], int comp, uint64_t* bar)
{
    if constexpr (D == 1) tma_load_2d(dst, tm, c[0], comp, bar);
    else if constexpr (D == 2) tma_load_3d(dst, tm, c[0], c[1], comp, bar);
    else tma_load_4d(dst, tm, c[0], c[1], c[2], comp, bar);
}
template <int D>
__device__ __forceinline__ void tma_reduce_add_box(const CUtensorMap* tm, const int c[3], int comp, const void* src)
{
    if constexpr (D == 1) tma_reduce_add_2d(tm, c[0], comp, src);
    else if constexpr (D == 2) tma_reduce_add_3d(tm, c[0], c[1], comp, src);
    else tma_reduce_add_4d(tm, c[0], c[1], c[2], comp, src);
}
template <int D>
__device__ __forceinline__ void tma_store_box(const CUtensorMap* tm, const int c[3], int comp, const void* src)
{
    if constexpr (D == 1) tma_store_2d(tm, c[0], comp, src);
    else if constexpr (D == 2) tma_store_3d(tm, c[0], c[1], comp, src);
    else tma_store_4d(tm, c[0], c[1], c[2], comp, src);
}

// ---------------------------------------------------------------------------------
// complex arithmetic in precision R
// ---------------------------------------------------------------------------------
template <typename R>
struct Cx {
    R x, y;
};
template <typename R>
__device__ __forceinline__ Cx<R> operator+(Cx<R> a, Cx<R> b) { return {a.x + b.x, a.y + b.y}; }
template <typename R>
__device__ __forceinline__ Cx<R> operator-(Cx<R> a, Cx<R> b) { return {a.x - b.x, a.y - b.y}; }
template <typename R>
__device__ __forceinline__ Cx<R> operator-(Cx<R> a) { return {-a.x, -a.y}; }
template <typename R>
__device__ __forceinline__ Cx<R> operator*(Cx<R> a, Cx<R> b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
template <typename R>
__device__ __forceinline__ Cx<R> operator*(R s, Cx<R> a) { return {s * a.x, s * a.y}; }
template <typename R>
__device__ __forceinline__ Cx<R> cinv(Cx<R> b)
{
    R d = R(1) / (b.x * b.x + b.y * b.y);
    return {b.x * d, -b.y * d};
}
template <typename R>
__device__ __forceinline__ Cx<R> operator/(Cx<R> a, Cx<R> b) { return a * cinv(b); }

// math overloads (call CUDA's own functions)
__device__ __forceinline__ float m_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double m_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float m_hypot(float x, float y) { return hypotf(x, y); }
__device__ __forceinline__ double m_hypot(double x, double y) { return hypot(x, y); }
__device__ __forceinline__ float m_log1p(float x) { return log1pf(x); }
__device__ __forceinline__ double m_log1p(double x) { return log1p(x); }
__device__ __forceinline__ float m_exp(float x) { return expf(x); }
__device__ __forceinline__ double m_exp(double x) { return exp(x); }
__device__ __forceinline__ float m_exp2(float x) { return exp2f(x); }
__device__ __forceinline__ double m_exp2(double x) { return exp2(x); }
__device__ __forceinline__ float m_atan2(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double m_atan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ void m_sincos(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void m_sincos(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ float m_sin(float x) { return sinf(x); }
__device__ __forceinline__ double m_sin(double x) { return sin(x); }
__device__ __forceinline__ float m_sinpi(float x) { return sinpif(x); }
__device__ __forceinline__ double m_sinpi(double x) { return sinpi(x); }
__device__ __forceinline__ float m_atan(float x) { return atanf(x); }
__device__ __forceinline__ double m_atan(double x) { return atan(x); }
__device__ __forceinline__ float m_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double m_rsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float m_floor(float x) { return floorf(x); }
__device__ __forceinline__ double m_floor(double x) { return floor(x); }
__device__ __forceinline__ float m_abs(float x) { return fabsf(x); }
__device__ __forceinline__ double m_abs(double x) { return fabs(x); }

template <typename R>
__device__ __forceinline__ Cx<R> csqrt_(Cx<R> z)
{
    R m = m_hypot(z.x, z.y);
    if (z.x >= R(0)) {
        R t = m_sqrt((m + z.x) * R(0.5));
        return {t, t > R(0) ? z.y / (R(2) * t) : R(0)};
    }
    R t = m_sqrt((m - z.x) * R(0.5));
    return {m_abs(z.y) / (R(2) * t), z.y < R(0) ? -t : t};
}

}  // namespace sff
