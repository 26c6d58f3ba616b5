// C-ABI of the GB300 scattered-field PIC library (include/pic.h): configuration
// checks and pulse-parameter derivation on the host, device state in one arena from
// the caller's allocator, TMA tensor maps, the seeded slab, the step as a CUDA graph,
// diagnostics, explicit state I/O and batched stepping of many simulations.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/pic.h"
#include "beam.cuh"
#include "sff_common.cuh"
#include "sff_kernels.h"
#include "sim_internal.h"

using namespace sff;

// Runs body(i0, i1) over [0, n) split into contiguous ranges on up to 16 host threads, at
// least per_min items each (one thread when n is small); returns when all are done.
template <typename F>
static void host_parallel(long long n, long long per_min, F body)
{
    int nt = (int)std::min<long long>(16, std::max<long long>(1, n / per_min));
    const unsigned hc = std::thread::hardware_concurrency();
    if (hc > 0) nt = std::min<int>(nt, (int)hc);
    if (nt <= 1) {
        body(0LL, n);
        return;
    }
    std::vector<std::thread> th;
    const long long chunk = (n + nt - 1) / nt;
    for (int k = 0; k < nt; ++k) {
        const long long i0 = k * chunk, i1 = std::min(n, i0 + chunk);
        if (i0 < i1) th.emplace_back([=] { body(i0, i1); });
    }
    for (auto& t : th) t.join();
}

long long new_group_id()
{
    static std::atomic<long long> next{1};
    return next.fetch_add(1);
}

namespace {

thread_local std::string g_thread_err;

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// ---- pulse parameters, host side -------------------------------------------------
// Complex on-axis field at the focus (xi = eta = zeta = 0, R = i) with Psi_0 = 1:
// LP E_x = (2 Phi_u - Phi_DD + 2i Phi_uD)/a^3, RP E_z = (2 Phi_u - 4 Phi_uu - Phi_DD)/a^3,
// Phi_* from Eq. (phasor) with g^(n) of Eq. (poisson_dstr) at tau_+ = tau + 2ia, tau_- = tau.
using cd = std::complex<double>;

void poisson3_h(double a, double s, cd tau, cd& g0, cd& g1, cd& g2)
{
    const cd w = 1.0 - cd(0, 1) * tau / s;
    g0 = std::exp(-(s + 1.0) * std::log(w));
    const cd q = cd(0, a) / (s * w);
    g1 = (s + 1.0) * g0 * q;
    g2 = (s + 2.0) * g1 * q;
}

double focal_env_h(int beam, double a, double s, double tau)
{
    cd g0p, g1p, g2p, g0m, g1m, g2m;
    poisson3_h(a, s, cd(tau, 2.0 * a), g0p, g1p, g2p);
    poisson3_h(a, s, cd(tau, 0.0), g0m, g1m, g2m);
    const cd G0m = g0p - g0m, G1p = g1p + g1m, G1m = g1p - g1m, G2p = g2p + g2m, G2m = g2p - g2m;
    const cd iR(0, -1), iR2 = iR * iR, iR3 = iR2 * iR;
    const cd Pu = 0.5 * (G1p * iR2 - G0m * iR3);
    const cd Puu = 0.25 * (G2m * iR3 - 3.0 * G1p * iR2 * iR2 + 3.0 * G0m * iR3 * iR2);
    const cd PuD = 0.5 * (G2p * iR2 - G1m * iR3);
    const cd PDD = G2m * iR;
    const cd e = beam == PIC_BEAM_LP ? (2.0 * Pu - PDD + 2.0 * cd(0, 1) * PuD) : (2.0 * Pu - 4.0 * Puu - PDD);
    return std::abs(e) / (a * a * a);
}

double focal_peak_h(int beam, double a, double s, double* tpk)
{
    const int n = 400;
    const double lo = -2.0 * s, hi = 2.0 * s;
    double best = -1.0, tb = 0.0;
    for (int i = 0; i <= n; ++i) {
        const double t = lo + (hi - lo) * i / n;
        const double v = focal_env_h(beam, a, s, t);
        if (v > best) {
            best = v;
            tb = t;
        }
    }
    const double h = (hi - lo) / n;
    double l = tb - h, r = tb + h;
    const double gr = 0.5 * (std::sqrt(5.0) - 1.0);
    double c1 = r - gr * (r - l), c2 = l + gr * (r - l);
    double f1 = focal_env_h(beam, a, s, c1), f2 = focal_env_h(beam, a, s, c2);
    for (int it = 0; it < 200 && (r - l) > 1e-13 * (1.0 + std::fabs(tb)); ++it) {
        if (f1 > f2) {
            r = c2; c2 = c1; f2 = f1; c1 = r - gr * (r - l); f1 = focal_env_h(beam, a, s, c1);
        } else {
            l = c1; c1 = c2; f1 = f2; c2 = l + gr * (r - l); f2 = focal_env_h(beam, a, s, c2);
        }
    }
    *tpk = 0.5 * (l + r);
    return focal_env_h(beam, a, s, *tpk);
}

double focal_fwhm_h(int beam, double a, double s)
{
    double tpk;
    const double half = 0.5 * focal_peak_h(beam, a, s, &tpk);
    double ends[2];
    for (int side = 0; side < 2; ++side) {
        const double dir = side ? -1.0 : 1.0;
        double l = tpk, r = tpk + dir * 60.0 * s;
        for (int it = 0; it < 300; ++it) {
            const double m = 0.5 * (l + r);
            if (focal_env_h(beam, a, s, m) > half) l = m; else r = m;
            if (std::fabs(r - l) < 1e-13 * (1.0 + std::fabs(m))) break;
        }
        ends[side] = 0.5 * (l + r);
    }
    return ends[0] - ends[1];
}

double s_from_duration_h(int beam, double a, double dur)
{
    double lo = 1.0, hi = 1.0e4;
    for (int it = 0; it < 200; ++it) {
        const double m = 0.5 * (lo + hi);
        if (focal_fwhm_h(beam, a, m) < dur) lo = m; else hi = m;
        if (hi - lo < 1e-12 * m) break;
    }
    return 0.5 * (lo + hi);
}

int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }
int bits_for(int n)
{
    int b = 0;
    while ((1ll << b) < n) ++b;
    return b;
}

}  // namespace

namespace {

pic_status fail(pic_sim* s, pic_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (s) s->err = buf;
    g_thread_err = buf;
    return st;
}

#define CU_CHECK(sim, call)                                                                              \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) return fail(sim, PIC_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

struct Layout {
    int dim, es, ncomp;
    int n[3], na[3], pt[3], npt[3], pb[3], yt[3], nyt[3], yb[3], yo[3];
    long long sy, sz, sc, natot;
    int nptiles, nytiles;
    long long cap, max_exits, nslab;
    long long slots;            // slots per particle buffer set: frame factor x cap
    int chunk, max_chunks;
    int tvol, sort_every;       // cells per particle tile; steps between cell sorts (0: none)
    size_t push_smem, yee_smem;
    size_t bytes;
};

pic_status validate(const pic_config* c, pic_sim* s)
{
    if (!c) return fail(s, PIC_EINVAL, "config is NULL");
    if (c->dim < 1 || c->dim > 3) return fail(s, PIC_EINVAL, "dim must be 1, 2 or 3 (got %d)", c->dim);
    for (int d = 0; d < c->dim; ++d)
        if (c->n[d] < 16 || c->n[d] > (1 << 20))
            return fail(s, PIC_EINVAL, "n[%d] = %d outside [16, 2^20]", d, c->n[d]);
    if (!(c->dx > 0)) return fail(s, PIC_EINVAL, "dx must be > 0");
    if (c->precision != PIC_FP64 && c->precision != PIC_FP32) return fail(s, PIC_EINVAL, "unknown precision");
    if (c->beam < PIC_BEAM_NONE || c->beam > PIC_BEAM_GAUSS2D) return fail(s, PIC_EINVAL, "unknown beam %d", c->beam);
    if (c->beam == PIC_BEAM_GAUSS2D) {
        if (c->dim != 2) return fail(s, PIC_EINVAL, "the 2D Gaussian beam needs dim == 2");
        if (!(c->w0 > 0) || !(c->duration > 0))
            return fail(s, PIC_EINVAL, "the 2D Gaussian beam needs w0 > 0 and duration > 0");
    }
    if (c->incident_grid != 0 && c->incident_grid != 1) return fail(s, PIC_EINVAL, "incident_grid must be 0 or 1");
    if (c->tf_mode != 0 && (c->tf_mode != 1 || c->dim != 1 || c->beam != PIC_BEAM_PLANE))
        return fail(s, PIC_EINVAL, "tf_mode = 1 needs dim == 1 and the plane wave");
    if (c->profile < PIC_PROFILE_UNIFORM || c->profile > PIC_PROFILE_SUPERGAUSS)
        return fail(s, PIC_EINVAL, "unknown profile %d", c->profile);
    if (c->profile == PIC_PROFILE_SUPERGAUSS && (!(c->prof_fwhm > 0) || c->prof_order < 1 || c->prof_order > 64))
        return fail(s, PIC_EINVAL, "super-Gaussian profile needs prof_fwhm > 0 and 1 <= prof_order <= 64");
    if ((c->beam == PIC_BEAM_LP || c->beam == PIC_BEAM_RP)) {
        if (c->dim < 2) return fail(s, PIC_EINVAL, "LP/RP beams need dim >= 2");
        if (!(c->a_param > 0 || c->w0 > 0)) return fail(s, PIC_EINVAL, "LP/RP beams need w0 > 0 or a_param > 0");
        if (!(c->s_param > 0 || c->duration > 0))
            return fail(s, PIC_EINVAL, "LP/RP beams need duration > 0 or s_param > 0");
        if (!(c->psi0 > 0 || c->a0 > 0)) return fail(s, PIC_EINVAL, "LP/RP beams need a0 > 0 or psi0 > 0");
    }
    if (c->beam == PIC_BEAM_PLANE && !(c->duration > 0)) return fail(s, PIC_EINVAL, "plane wave needs duration > 0");
    const double dt = c->dt > 0 ? c->dt : c->cfl * c->dx / std::sqrt((double)c->dim);
    if (!(dt > 0) || dt >= c->dx / std::sqrt((double)c->dim))
        return fail(s, PIC_EINVAL, "dt = %g violates the CFL bound dx/sqrt(dim) = %g", dt, c->dx / std::sqrt((double)c->dim));
    const int margin = c->remove_margin > 0 ? c->remove_margin : 3;
    if (margin < 3) return fail(s, PIC_EINVAL, "remove_margin must be >= 3");
    if (c->ppc < 0) return fail(s, PIC_EINVAL, "ppc < 0");
    if (c->ppc > 0) {
        for (int d = 0; d < c->dim; ++d)
            if (c->slab_lo[d] < margin || c->slab_hi[d] > c->n[d] - margin || c->slab_hi[d] <= c->slab_lo[d])
                return fail(s, PIC_EINVAL, "slab [%d,%d) on axis %d must lie in [%d, %d)", c->slab_lo[d], c->slab_hi[d],
                            d, margin, c->n[d] - margin);
        if (!(c->n_e >= 0)) return fail(s, PIC_EINVAL, "n_e < 0");
    }
    for (int d = 0; d < c->dim; ++d)
        if (c->tile[d] < 0 || (c->tile[d] > 0 && (c->tile[d] < 2 || c->tile[d] > 248 || (d == 0 && c->tile[d] % 4))))
            return fail(s, PIC_EINVAL, "tile[%d] = %d invalid (2..248 cells, x a multiple of 4)", d, c->tile[d]);
    if (c->chunk < 0 || (c->chunk > 0 && (c->chunk % 256 || c->chunk > 16384)))
        return fail(s, PIC_EINVAL, "chunk = %d invalid (a multiple of 256, <= 16384)", c->chunk);
    if (c->autotune_steps < 0) return fail(s, PIC_EINVAL, "autotune_steps must be >= 0");
    if (c->pusher < PIC_PUSHER_BORIS || c->pusher > PIC_PUSHER_HC)
        return fail(s, PIC_EINVAL, "unknown pusher %d", c->pusher);
    int bits = 0;
    for (int d = 0; d < c->dim; ++d) bits += bits_for(c->n[d]);
    if (bits > 31) return fail(s, PIC_EINVAL, "grid too large for the packed cell index");
    return PIC_OK;
}

// Tile choice (the autotuner's defaults; `tile` in the config overrides the particle tile).
void choose_tiles(const pic_config* c, int pt[3], int yt[3])
{
    const bool fp64 = c->precision == PIC_FP64;
    // field-solver tiles are fixed per dimension: k_yee is compiled for exactly these shapes
    if (c->dim == 1) {
        pt[0] = 32; yt[0] = 128;
    } else if (c->dim == 2) {
        pt[0] = 16; pt[1] = 16; yt[0] = Y2_PX; yt[1] = Y2_PY;
    } else {
        // columns of Y3_PX x Y3_PY marching along z in segments: at least ~600 work items
        // (a few per resident block on a full GPU), segments of at most 64 planes
        pt[0] = 8; pt[1] = 8; pt[2] = 8;
        yt[0] = Y3_PX; yt[1] = Y3_PY;
        const long long ncol = (long long)ceil_div(c->n[0] + 1, Y3_PX) * ceil_div(c->n[1] + 1, Y3_PY);
        const int nz = c->n[2] + 1;
        int nseg = std::max<int>(ceil_div(nz, 64), (int)std::min<long long>(nz, (600 + ncol - 1) / ncol));
        nseg = std::min(nseg, std::max(1, nz / 8));
        yt[2] = ceil_div(nz, nseg);
    }
    for (int d = c->dim; d < 3; ++d) pt[d] = yt[d] = 1;
    for (int d = 0; d < c->dim; ++d)
        if (c->tile[d] > 0) pt[d] = c->tile[d];
}

Layout make_layout(const pic_config* c)
{
    Layout L{};
    L.dim = c->dim;
    L.es = c->precision == PIC_FP64 ? 8 : 4;
    L.ncomp = c->incident_grid ? NFCOMP_INC : NFCOMP;
    choose_tiles(c, L.pt, L.yt);
    for (int d = 0; d < 3; ++d) {
        if (d < c->dim) {
            const int N = c->n[d];
            L.n[d] = N;
            L.npt[d] = ceil_div(N, L.pt[d]);
            L.nyt[d] = ceil_div(N + 1, L.yt[d]);
            L.pb[d] = d == 0 ? L.pt[d] + 8 : L.pt[d] + 5;
            L.yb[d] = d == 0 ? L.yt[d] + 8 : L.yt[d] + 4;
            L.yo[d] = L.yt[d];
            if (c->dim == 3 && d == 2) L.yb[d] = L.yo[d] = 1;     // one plane per load / store
            long long need = N + 1 + 2 * (d == 0 ? GX : G);
            if (d == 0) {
                // boxes reach 4 points past the last tile; rows start on 128 bytes
                need = std::max<long long>(need, (long long)L.npt[d] * L.pt[d] + 4 + GX);
                need = std::max<long long>(need, (long long)L.nyt[d] * L.yt[d] + 4 + GX);
                const int al = 128 / L.es;
                need = (need + al - 1) / al * al;
            } else {
                need = std::max<long long>(need, (long long)L.npt[d] * L.pt[d] + 7);
                need = std::max<long long>(need, (long long)L.nyt[d] * L.yt[d] + 6);
            }
            L.na[d] = (int)need;
        } else {
            L.n[d] = 1; L.na[d] = 1; L.npt[d] = 1; L.nyt[d] = 1; L.pb[d] = 1; L.yb[d] = 1; L.yo[d] = 1;
            L.pt[d] = 1; L.yt[d] = 1;
        }
    }
    L.sy = L.na[0];
    L.sz = (long long)L.na[0] * L.na[1];
    L.sc = L.sz * L.na[2];
    L.natot = L.sc;
    L.nptiles = L.npt[0] * L.npt[1] * L.npt[2];
    L.nytiles = L.nyt[0] * L.nyt[1] * L.nyt[2];
    L.nslab = 0;
    if (c->ppc > 0) {
        L.nslab = c->ppc;
        for (int d = 0; d < c->dim; ++d) L.nslab *= (c->slab_hi[d] - c->slab_lo[d]);
    }
    L.cap = c->max_particles > 0 ? c->max_particles : std::max<long long>(L.nslab, 1);
    L.max_exits = c->max_exits > 0 ? c->max_exits : L.cap;
    L.chunk = c->chunk > 0 ? c->chunk : 2048;
    L.max_chunks = (int)(L.nptiles + (L.cap + L.chunk - 1) / L.chunk + 1);
    // Every tile keeps slack for the particles within one cell outside it, the only ones a
    // step can bring in (a move is under one cell per axis).  With tiles at least two cells
    // wide a particle lies in the frames of at most 2^dim - 1 other tiles, so 2^dim slots
    // per particle hold every tile's particles and slack.
    L.slots = (1LL << c->dim) * L.cap;
    L.tvol = L.pt[0] * L.pt[1] * L.pt[2];
    // the cell-sort arrays are indexed by int: a tiled grid of 2^31 cells or more sorts by
    // tile only (an explicit request is rejected)
    const long long tcells = (long long)L.nptiles * L.tvol;
    L.sort_every = std::max(0, c->sort_every);
    if (tcells >= (1LL << 31)) L.sort_every = 0;
    const long long pbv = (long long)L.pb[0] * L.pb[1] * L.pb[2];
    const long long ybv = (long long)L.yb[0] * L.yb[1] * L.yb[2];
    const long long ytv = (long long)L.yt[0] * L.yt[1] * L.yt[2];
    L.push_smem = round128((size_t)(6 * pbv * L.es)) + (size_t)(3 * pbv * L.es);
    L.yee_smem = c->dim == 3 ? yee3_smem(L.es)
                 : c->dim == 2 ? yee2_smem(L.es)
                               : 2 * round128(round128((size_t)(6 * ybv * L.es)) + (size_t)(3 * ybv * L.es)) +
                                     (size_t)(6 * ytv * L.es);      // two box buffers + the output tile
    size_t b = 0;
    b += align256(sizeof(SimDev)) + align256(sizeof(DevState));
    b += align256((size_t)L.ncomp * L.natot * L.es);
    const size_t per = 4 + (size_t)(c->dim + 4) * L.es + 4;
    for (int q = 0; q < 2; ++q) {
        b += align256(L.slots * 4) * 2;                                // cell, id
        b += align256(L.slots * L.es) * (size_t)(c->dim + 4);          // off, mom, w
    }
    (void)per;
    b += 4 * align256((size_t)(L.nptiles + 1) * 4) + 5 * align256((size_t)L.nptiles * 4);   // + tnum, fcnt
    b += align256((size_t)((L.nptiles + 4095) / 4096) * 8) + align256(4);
    b += 2 * align256((size_t)L.max_chunks * 4) + 2 * align256((size_t)L.max_chunks * 8);   // ctile, crange
    if (L.sort_every > 0) b += 2 * align256((size_t)tcells * 4);
    b += align256((size_t)L.max_exits * EXIT_DOUBLES * 8);
    b += 2 * align256((size_t)L.natot * 8);
    b += align256((size_t)L.nytiles * sizeof(Work));
    b += align256(64) + align256(64) + align256(8 * 8) + align256(8);
    L.bytes = b;
    return L;
}

pic_status derive(const pic_config* c, pic_params* out, pic_sim* s)
{
    pic_status st = validate(c, s);
    if (st != PIC_OK) return st;
    pic_params p{};
    p.dt = c->dt > 0 ? c->dt : c->cfl * c->dx / std::sqrt((double)c->dim);
    if (c->beam == PIC_BEAM_LP || c->beam == PIC_BEAM_RP) {
        double a = c->a_param, sp = c->s_param, psi0 = c->psi0;
        if (!(a > 0)) {
            const double h = 1.0 + 0.5 * c->w0 * c->w0;     // k^2 w0^2 = 2(sqrt(1 + (ka)^2) - 1)
            a = std::sqrt(h * h - 1.0);
        }
        if (!(sp > 0)) sp = s_from_duration_h(c->beam, a, c->duration);
        if (!(psi0 > 0)) {
            double tpk;
            psi0 = c->a0 / focal_peak_h(c->beam, a, sp, &tpk);
        }
        p.a = a; p.s = sp; p.psi0 = psi0;
    }
    Layout L = make_layout(c);
    if (L.slots >= (1LL << 31))
        return fail(s, PIC_EINVAL, "particle capacity %lld x frame factor exceeds 2^31 slots", L.cap);
    p.n_particles = L.nslab;
    p.device_bytes = (int64_t)L.bytes;
    for (int d = 0; d < 3; ++d) {
        p.tile[d] = L.pt[d];
        p.yee_tile[d] = L.yt[d];
    }
    p.chunk = L.chunk;
    p.sort_every = L.sort_every;
    if (c->sort_every > 0 && L.sort_every == 0)
        return fail(s, PIC_EINVAL, "sort_every > 0 needs fewer than 2^31 cells in the tiled grid");
    *out = p;
    return PIC_OK;
}

typedef CUresult (*PFN_encodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

PFN_encodeTiled get_encode()
{
    static PFN_encodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_encodeTiled>(p);
    });
    return fn;
}

pic_status make_map(pic_sim* s, CUtensorMap* m, const Layout& L, const int box[3], int ncomp)
{
    PFN_encodeTiled enc = get_encode();
    if (!enc) return fail(s, PIC_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const int r = L.dim + 1;
    cuuint64_t gdim[4], gstr[3];
    cuuint32_t bdim[4], estr[4] = {1, 1, 1, 1};
    for (int d = 0; d < L.dim; ++d) {
        gdim[d] = (cuuint64_t)L.na[d];
        bdim[d] = (cuuint32_t)box[d];
    }
    gdim[L.dim] = L.ncomp;
    bdim[L.dim] = (cuuint32_t)ncomp;
    const long long strides[3] = {L.sy, L.sz, L.sc};
    int k = 0;
    for (int d = 1; d < L.dim; ++d) gstr[k++] = (cuuint64_t)strides[d - 1] * L.es;
    gstr[k++] = (cuuint64_t)L.sc * L.es;
    const CUresult cr =
        enc(m, L.es == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)r, s->h.F, gdim,
            gstr, bdim, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return fail(s, PIC_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
    return PIC_OK;
}

void* dev_alloc(pic_sim* s, size_t bytes)
{
    if (s->use_cuda_malloc) {
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
        return p;
    }
    return s->alloc.alloc(bytes, s->alloc.ctx);
}

void dev_free(pic_sim* s, void* p)
{
    if (!p) return;
    if (s->use_cuda_malloc) cudaFree(p);
    else s->alloc.free(p, s->alloc.ctx);
}

// One step as a CUDA graph; `sorted`: the variant whose particles are placed by cell.
// After the push the graph forks: the tile scan (with, in the sorted variant, the cell-sort
// placement) and the field solve touch disjoint data and run concurrently; the step end
// joins them and numbers the next step's chunks (the graph starts at the push: see
// ensure_prefix).
pic_status capture_step(pic_sim* s, bool sorted, GraphBundle* out)
{
    cudaStream_t cs = s->cap_stream, cs2 = s->cap_stream2;
    CU_CHECK(s, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    launch_incident_grid(s->grp, cs);
    launch_push(s->grp, sorted, cs);
    cudaError_t e = cudaEventRecord(s->ev_fork, cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs2, s->ev_fork, 0);
    if (e == cudaSuccess) {
        launch_yee(s->grp, cs2);
        e = cudaEventRecord(s->ev_join, cs2);
    }
    launch_scan(s->grp, cs);
    if (sorted) launch_cell_sort(s->grp, cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, s->ev_join, 0);
    launch_step_end(s->grp, cs);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = ec;
    if (e != cudaSuccess && g) {
        cudaGraphDestroy(g);
        g = nullptr;
    }
    if (e != cudaSuccess) return fail(s, PIC_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    out->graph = g;
    e = cudaGraphInstantiate(&out->exec, g, 0);
    if (e != cudaSuccess) return fail(s, PIC_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    return PIC_OK;
}

// Before a step of the single-simulation group: number the chunks unless the last step of
// this group did (k_step_end) and nothing changed the layout since.
void ensure_prefix(pic_sim* s, cudaStream_t st)
{
    if (s->prefix_group == s->own_group_id) return;
    launch_prefix(s->grp, st);
    s->prefix_group = s->own_group_id;
}

// true when the next step is a cell-sort step (advances the per-sim step count)
bool next_is_sort(pic_sim* s)
{
    if (s->sort_every <= 0) return false;
    if (++s->since_sort < s->sort_every) return false;
    s->since_sort = 0;
    return true;
}

pic_status read_state(pic_sim* s, DevState* out, cudaStream_t st)
{
    CU_CHECK(s, cudaMemcpyAsync(out, s->h.st, sizeof(DevState), cudaMemcpyDeviceToHost, st));
    CU_CHECK(s, cudaStreamSynchronize(st));
    return PIC_OK;
}

pic_status write_state(pic_sim* s, const DevState& v, cudaStream_t st)
{
    CU_CHECK(s, cudaMemcpyAsync(s->h.st, &v, sizeof(DevState), cudaMemcpyHostToDevice, st));
    CU_CHECK(s, cudaStreamSynchronize(st));
    return PIC_OK;
}

// ion background rho_ion = -rho_e of the present particles (step 0)
pic_status compute_rho_ion(pic_sim* s, cudaStream_t st)
{
    DevState ds;
    pic_status r = read_state(s, &ds, st);
    if (r != PIC_OK) return r;
    // immobile ions co-located with the electrons: rho_ion = -rho_e, deposited in place
    CU_CHECK(s, cudaMemsetAsync(s->h.rho_ion, 0, sizeof(double) * s->nalloc_tot, st));
    launch_charge(s->d, s->cfg.dim, s->cfg.precision, s->h.cap, s->h.rho_ion, st, -1.0);
    CU_CHECK(s, cudaGetLastError());
    CU_CHECK(s, cudaStreamSynchronize(st));
    return PIC_OK;
}

// sort the n particles sitting linearly in buffer set 1 into set 0
pic_status sort_linear_into_set0(pic_sim* s, long long n, cudaStream_t st)
{
    DevState ds;
    pic_status r = read_state(s, &ds, st);
    if (r != PIC_OK) return r;
    if (ds.parity == 1) {
        // the particles land in set 0: move E, B to set 0, keep the last current in J_1, clear J_0
        char* F = (char*)s->h.F;
        const size_t comp = (size_t)s->nalloc_tot * s->es;
        CU_CHECK(s, cudaMemcpyAsync(F + comp_eb(0) * comp, F + comp_eb(1) * comp, 6 * comp, cudaMemcpyDeviceToDevice, st));
        CU_CHECK(s, cudaMemcpyAsync(F + comp_j(1) * comp, F + comp_j(0) * comp, 3 * comp, cudaMemcpyDeviceToDevice, st));
        CU_CHECK(s, cudaMemsetAsync(F + comp_j(0) * comp, 0, 3 * comp, st));
    }
    ds.parity = 1;
    r = write_state(s, ds, st);
    if (r != PIC_OK) return r;
    CU_CHECK(s, cudaMemsetAsync(s->h.tcnt, 0, sizeof(int) * s->h.nptiles, st));
    CU_CHECK(s, cudaMemsetAsync(s->h.fcnt, 0, sizeof(int) * s->h.nptiles, st));
    CU_CHECK(s, cudaMemsetAsync(s->h.cell[0], 0xFF, (size_t)s->h.cap * 4, st));
    CU_CHECK(s, cudaMemsetAsync(s->h.cell[1] + n, 0xFF, (size_t)(s->h.cap - n) * 4, st));
    launch_count_linear(s->d, s->cfg.dim, s->cfg.precision, n, st);
    launch_scan_one(s->d, 0, st);
    launch_sort_linear(s->d, s->cfg.dim, s->cfg.precision, n, st);
    CU_CHECK(s, cudaMemsetAsync(s->h.tcur, 0, sizeof(int) * s->h.nptiles, st));
    launch_next_slots(s->d, s->cfg.dim, s->cfg.precision, 0, n, st);
    CU_CHECK(s, cudaGetLastError());
    ds.parity = 0;
    ds.n_alive = (int)n;
    ds.n_next = 0;
    return write_state(s, ds, st);
}

}  // namespace

// =====================================================================================
// C-ABI
// =====================================================================================
extern "C" {

pic_status pic_derive_params(const pic_config* cfg, pic_params* out)
{
    if (!out) return fail(nullptr, PIC_EINVAL, "out is NULL");
    return derive(cfg, out, nullptr);
}

const char* pic_last_error(const pic_sim* sim)
{
    if (sim) return sim->err.c_str();
    return g_thread_err.c_str();
}

pic_status pic_init(const pic_config* cfg_in, const pic_allocator* alloc, void* stream, pic_sim** out)
{
    if (!out) return fail(nullptr, PIC_EINVAL, "out is NULL");
    *out = nullptr;
    pic_params prm;
    pic_status r = derive(cfg_in, &prm, nullptr);
    if (r != PIC_OK) return r;
    pic_config tuned = *cfg_in;
    if (cfg_in->autotune_steps > 0) {
        tuned.autotune_steps = 0;
        if ((r = pic_autotune(&tuned, cfg_in->autotune_steps, stream, nullptr)) != PIC_OK) return r;
        if ((r = derive(&tuned, &prm, nullptr)) != PIC_OK) return r;
    }
    const pic_config* cfg = &tuned;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(nullptr, PIC_ENODEV, "no CUDA device");
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return fail(nullptr, PIC_ENODEV, "no CUDA device");
    if (prop.major * 10 + prop.minor < 100)
        return fail(nullptr, PIC_ENODEV, "device %s (sm_%d%d) is not a Blackwell GPU", prop.name, prop.major, prop.minor);

    pic_sim* s = new pic_sim();
    s->cfg = *cfg;
    s->own_group_id = new_group_id();
    s->prm = prm;
    s->device = dev;
    if (alloc && alloc->alloc && alloc->free) {
        s->alloc = *alloc;
        s->use_cuda_malloc = false;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const Layout L = make_layout(cfg);
    s->es = L.es;
    s->nalloc_tot = L.natot;
    s->arena.size = L.bytes;
    s->arena.base = (char*)dev_alloc(s, L.bytes);
    if (!s->arena.base) {
        delete s;
        return fail(nullptr, PIC_ENOMEM, "device allocation of %zu bytes failed", L.bytes);
    }
    Arena& A = s->arena;
    SimDev& h = s->h;
    memset(&h, 0, sizeof h);
    s->d = (SimDev*)A.take(sizeof(SimDev));
    h.st = (DevState*)A.take(sizeof(DevState));
    h.F = A.take((size_t)L.ncomp * L.natot * L.es);
    for (int q = 0; q < 2; ++q) {
        h.cell[q] = (unsigned*)A.take(L.slots * 4);
        h.pid[q] = (unsigned*)A.take(L.slots * 4);
        for (int d = 0; d < cfg->dim; ++d) h.off[q][d] = A.take(L.slots * L.es);
        for (int d = 0; d < 3; ++d) h.mom[q][d] = A.take(L.slots * L.es);
        h.wgt[q] = A.take(L.slots * L.es);
    }
    h.toff[0] = (int*)A.take((size_t)(L.nptiles + 1) * 4);
    h.toff[1] = (int*)A.take((size_t)(L.nptiles + 1) * 4);
    h.coff[0] = (int*)A.take((size_t)(L.nptiles + 1) * 4);
    h.coff[1] = (int*)A.take((size_t)(L.nptiles + 1) * 4);
    h.ctile[0] = (int*)A.take((size_t)L.max_chunks * 4);
    h.ctile[1] = (int*)A.take((size_t)L.max_chunks * 4);
    h.crange[0] = (int2*)A.take((size_t)L.max_chunks * 8);
    h.crange[1] = (int2*)A.take((size_t)L.max_chunks * 8);
    h.tnum[0] = (int*)A.take((size_t)L.nptiles * 4);
    h.tnum[1] = (int*)A.take((size_t)L.nptiles * 4);
    h.fcnt = (int*)A.take((size_t)L.nptiles * 4);
    h.chunk = L.chunk;
    h.lane_p = 8;
    if (cfg->ppc > 0)
        for (h.lane_p = 1; h.lane_p * 2 <= std::min(cfg->ppc, 8);) h.lane_p *= 2;
    h.max_chunks = L.max_chunks;
    h.tcnt = (int*)A.take((size_t)L.nptiles * 4);
    h.tcur = (int*)A.take((size_t)L.nptiles * 4);
    h.tvol = L.tvol;
    if (L.sort_every > 0) {
        h.ccnt = (int*)A.take((size_t)L.nptiles * L.tvol * 4);
        h.ccur = (int*)A.take((size_t)L.nptiles * L.tvol * 4);
    }
    s->sort_every = L.sort_every;
    s->pcap = L.cap;
    h.nscanblk = (L.nptiles + 4095) / 4096;
    h.scan_spins = 1 << 22;      // about a second of polls of a predecessor's flag
    h.scan_hold = -1;
    h.scanflags = (unsigned long long*)A.take((size_t)h.nscanblk * 8);
    h.scanticket = (int*)A.take(4);
    h.exits = (double*)A.take((size_t)L.max_exits * EXIT_DOUBLES * 8);
    h.rho_ion = (double*)A.take((size_t)L.natot * 8);
    h.scratch = (double*)A.take((size_t)L.natot * 8);
    s->d_ywork = (Work*)A.take((size_t)L.nytiles * sizeof(Work));
    s->d_gprefix = (int*)A.take(64);
    s->d_counters = (int*)A.take(64);
    s->d_acc = (double*)A.take(64);
    s->d_bits = (unsigned long long*)A.take(8);
    if (!s->d_bits) {
        pic_destroy(s);
        return fail(nullptr, PIC_ENOMEM, "arena layout overflow");
    }
    // descriptor
    h.dim = cfg->dim;
    h.prec = cfg->precision;
    h.beam = cfg->beam;
    h.envelope = cfg->envelope;
    for (int d = 0; d < 3; ++d) {
        h.n[d] = L.n[d]; h.na[d] = L.na[d]; h.pt[d] = L.pt[d]; h.npt[d] = L.npt[d]; h.pb[d] = L.pb[d];
        h.yt[d] = L.yt[d]; h.nyt[d] = L.nyt[d]; h.yb[d] = L.yb[d];
        h.cb[d] = d < cfg->dim ? bits_for(cfg->n[d]) : 0;
        h.focus[d] = cfg->focus[d];
        h.e_unif[d] = cfg->e_unif[d];
        h.b_unif[d] = cfg->b_unif[d];
        const double fc = cfg->focus[d] / cfg->dx;
        h.icf[d] = (int)std::floor(fc);
        h.frf[d] = (float)(fc - std::floor(fc));
    }
    h.sy = L.sy; h.sz = L.sz; h.sc = L.sc;
    h.nptiles = L.nptiles;
    h.nytiles = L.nytiles;
    h.margin = cfg->remove_margin > 0 ? cfg->remove_margin : 3;
    h.pusher = cfg->pusher;
    h.tf = cfg->tf_mode;
    h.incgrid = cfg->incident_grid && cfg->beam != PIC_BEAM_NONE && !cfg->tf_mode;
    h.dx = cfg->dx;
    h.dt = prm.dt;
    h.inv_dx = 1.0 / cfg->dx;
    h.a0 = cfg->a0;
    h.w0 = cfg->w0;
    h.profile = cfg->profile;
    h.prof_order = cfg->prof_order;
    h.prof_x0 = cfg->prof_x0;
    h.prof_fwhm = cfg->prof_fwhm;
    h.prof_cut = cfg->prof_cut;
    h.duration = cfg->duration;
    h.phi0 = cfg->phi0;
    h.t_focus = cfg->t_focus;
    h.a = prm.a;
    h.s = prm.s;
    h.psi0 = prm.psi0;
    h.max_exits = L.max_exits;
    h.cap = L.slots;
    h.bcf = make_beam_consts<float>(h);
    h.bcd = make_beam_consts<double>(h);
    h.ycf = {(float)(prm.dt / cfg->dx), (float)(0.5 * prm.dt / cfg->dx), (float)prm.dt,
             (float)((prm.dt - cfg->dx) / (prm.dt + cfg->dx))};
    h.ycd = {prm.dt / cfg->dx, 0.5 * prm.dt / cfg->dx, prm.dt, (prm.dt - cfg->dx) / (prm.dt + cfg->dx)};
    // tensor maps (every box extent must stay within TMA's 256 elements per dimension)
    for (int d = 0; d < 3; ++d)
        if (L.pb[d] > 256 || L.yb[d] > 256) {
            fail(s, PIC_EINVAL, "tile too large: box extent %d/%d on axis %d exceeds 256", L.pb[d], L.yb[d], d);
            std::string m = s->err;
            pic_destroy(s);
            return fail(nullptr, PIC_EINVAL, "%s", m.c_str());
        }
    if ((r = make_map(s, &h.tm_pf, L, L.pb, 6)) != PIC_OK ||
        (r = make_map(s, &h.tm_pj, L, L.pb, 3)) != PIC_OK ||
        (r = make_map(s, &h.tm_yin, L, L.yb, 6)) != PIC_OK ||
        (r = make_map(s, &h.tm_yj, L, L.yb, 3)) != PIC_OK ||
        (r = make_map(s, &h.tm_yout, L, L.yo, 6)) != PIC_OK) {
        std::string m = s->err;
        pic_destroy(s);
        return fail(nullptr, r, "%s", m.c_str());
    }
    auto cleanup = [&](pic_status code) {
        std::string m = s->err;
        pic_destroy(s);
        return fail(nullptr, code, "%s", m.c_str());
    };
#define INIT_CHECK(call)                                                                              \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) {                                                                      \
            fail(s, PIC_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));                       \
            return cleanup(PIC_ECUDA);                                                                \
        }                                                                                             \
    } while (0)
    INIT_CHECK(cudaMemsetAsync(h.F, 0, (size_t)L.ncomp * L.natot * L.es, st));
    INIT_CHECK(cudaMemsetAsync(h.toff[0], 0, (size_t)(L.nptiles + 1) * 4, st));
    INIT_CHECK(cudaMemsetAsync(h.toff[1], 0, (size_t)(L.nptiles + 1) * 4, st));
    INIT_CHECK(cudaMemsetAsync(h.coff[0], 0, (size_t)(L.nptiles + 1) * 4, st));
    INIT_CHECK(cudaMemsetAsync(h.coff[1], 0, (size_t)(L.nptiles + 1) * 4, st));
    INIT_CHECK(cudaMemsetAsync(h.tcnt, 0, (size_t)L.nptiles * 4, st));
    INIT_CHECK(cudaMemsetAsync(h.tcur, 0, (size_t)L.nptiles * 4, st));
    INIT_CHECK(cudaMemsetAsync(h.fcnt, 0, (size_t)L.nptiles * 4, st));
    INIT_CHECK(cudaMemsetAsync(h.tnum[0], 0, (size_t)L.nptiles * 4, st));
    INIT_CHECK(cudaMemsetAsync(h.tnum[1], 0, (size_t)L.nptiles * 4, st));
    for (int q = 0; q < 2; ++q) INIT_CHECK(cudaMemsetAsync(h.cell[q], 0xFF, (size_t)L.slots * 4, st));   // DEAD
    if (h.ccnt) INIT_CHECK(cudaMemsetAsync(h.ccnt, 0, (size_t)L.nptiles * L.tvol * 4, st));
    INIT_CHECK(cudaMemsetAsync(h.scanflags, 0, (size_t)h.nscanblk * 8, st));
    INIT_CHECK(cudaMemsetAsync(h.scanticket, 0, 4, st));
    INIT_CHECK(cudaMemsetAsync(s->d_counters, 0, 64, st));
    INIT_CHECK(cudaMemsetAsync(h.rho_ion, 0, (size_t)L.natot * 8, st));
    DevState ds{};
    ds.parity = 1;
    // the slab's weights are n_e f(x)/ppc with f <= 1 (rounded up: every FP32 weight is below)
    ds.wmax = cfg->ppc > 0 ? std::nextafter((float)(cfg->n_e / cfg->ppc), INFINITY) : 0.f;
    INIT_CHECK(cudaMemcpyAsync(h.st, &ds, sizeof ds, cudaMemcpyHostToDevice, st));
    INIT_CHECK(cudaMemcpyAsync(s->d, &h, sizeof h, cudaMemcpyHostToDevice, st));
    // work lists of the single-simulation group
    {
        std::vector<Work> yw;
        for (int i = 0; i < L.nytiles; ++i)
            if (yee_tile_active(h, cfg->dim, i)) yw.push_back({0, i});
        s->nywork = (int)yw.size();
        INIT_CHECK(cudaMemcpyAsync(s->d_ywork, yw.data(), yw.size() * sizeof(Work), cudaMemcpyHostToDevice, st));
        INIT_CHECK(cudaMemsetAsync(s->d_gprefix, 0, 64, st));
        INIT_CHECK(cudaStreamSynchronize(st));
    }
    // seeded slab: linear into set 1, then sorted into set 0
    if (L.nslab > 0) {
        int lo[3] = {0, 0, 0}, sn[3] = {1, 1, 1};
        for (int d = 0; d < cfg->dim; ++d) {
            lo[d] = cfg->slab_lo[d];
            sn[d] = cfg->slab_hi[d] - cfg->slab_lo[d];
        }
        launch_gen_slab(s->d, cfg->dim, cfg->precision, L.nslab, cfg->ppc, lo, sn, cfg->seed,
                        cfg->n_e / cfg->ppc, st);
        INIT_CHECK(cudaGetLastError());
        launch_scan_one(s->d, 0, st);
        int hi[3] = {1, 1, 1};
        for (int d = 0; d < cfg->dim; ++d) hi[d] = cfg->slab_hi[d];
        launch_place_slab(s->d, cfg->dim, cfg->precision, L.nslab, cfg->ppc, lo, hi, st);
        INIT_CHECK(cudaGetLastError());
    }
    // the first push's destination slots (set 1): tile counts plus frame counts
    launch_next_slots(s->d, cfg->dim, cfg->precision, 0, L.nslab, st);
    INIT_CHECK(cudaGetLastError());
    ds.parity = 0;
    ds.n_alive = (int)L.nslab;
    INIT_CHECK(cudaMemcpyAsync(h.st, &ds, sizeof ds, cudaMemcpyHostToDevice, st));
    INIT_CHECK(cudaStreamSynchronize(st));
    if ((r = compute_rho_ion(s, st)) != PIC_OK) return cleanup(r);

    // launch group and step graph
    const int nsm = prop.multiProcessorCount;
    Group& g = s->grp;
    g.sims = s->d;
    g.one = &s->h;       // the same descriptor, by value for the push (final from here on)
    g.gprefix = s->d_gprefix;
    g.ywork = s->d_ywork;
    g.nywork = s->nywork;
    g.nsims = 1;
    g.counters = s->d_counters;
    g.dim = cfg->dim;
    g.prec = cfg->precision;
    g.push_smem = L.push_smem;
    g.yee_smem = L.yee_smem;
    if (L.push_smem > (size_t)prop.sharedMemPerBlockOptin || L.yee_smem > (size_t)prop.sharedMemPerBlockOptin) {
        fail(s, PIC_EINVAL, "tile needs %zu/%zu bytes of shared memory (max %zu)", L.push_smem, L.yee_smem,
             (size_t)prop.sharedMemPerBlockOptin);
        return cleanup(PIC_EINVAL);
    }
    const int bp = std::max(1, prepare_push(cfg->dim, cfg->precision, L.push_smem));
    const int by = std::max(1, prepare_yee(cfg->dim, cfg->precision, L.yee_smem));
    const int bs = std::max(1, scatter_blocks_per_sm(cfg->dim, cfg->precision));
    g.inc_any = h.incgrid;
    g.scan_blocks = h.nscanblk;
    g.cellscan_grid = std::max(1, std::min(L.nptiles, 8 * nsm));
    g.inc_segs = (cfg->n[0] + 1 + 255) / 256;
    g.inc_rows = (cfg->dim > 1 ? cfg->n[1] + 1 : 1) * (cfg->dim > 2 ? cfg->n[2] + 1 : 1);
    g.push_grid = std::max(1, std::min(L.max_chunks, bp * nsm));
    g.yee_grid = std::max(1, std::min(s->nywork, by * nsm));
    g.scatter_grid = std::max(1, std::min(L.max_chunks, bs * nsm));
    INIT_CHECK(cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking));
    INIT_CHECK(cudaStreamCreateWithFlags(&s->cap_stream2, cudaStreamNonBlocking));
    INIT_CHECK(cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming));
    INIT_CHECK(cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming));
    if ((r = capture_step(s, false, &s->step_graph)) != PIC_OK) return cleanup(r);
    if (s->sort_every > 0 && (r = capture_step(s, true, &s->sort_graph)) != PIC_OK) return cleanup(r);
#undef INIT_CHECK
    *out = s;
    return PIC_OK;
}

pic_status pic_step(pic_sim* s, int n_steps, void* stream)
{
    if (!s) return fail(nullptr, PIC_EINVAL, "sim is NULL");
    if (n_steps < 0) return fail(s, PIC_EINVAL, "n_steps < 0");
    cudaStream_t st = (cudaStream_t)stream;
    if (n_steps > 0) ensure_prefix(s, st);
    for (int i = 0; i < n_steps; ++i)
        CU_CHECK(s, cudaGraphLaunch(next_is_sort(s) ? s->sort_graph.exec : s->step_graph.exec, st));
    return PIC_OK;
}

pic_status pic_profile_step(pic_sim* s, int n_steps, void* stream, double* seconds)
{
    if (!s || !seconds || n_steps < 0) return fail(s, PIC_EINVAL, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t ev[6];
    for (int i = 0; i < 6; ++i) CU_CHECK(s, cudaEventCreate(&ev[i]));
    for (int i = 0; i < 5; ++i) seconds[i] = 0.0;
    pic_status r = PIC_OK;
    if (n_steps > 0) ensure_prefix(s, st);
    for (int k = 0; k < n_steps && r == PIC_OK; ++k) {
        const bool sorted = next_is_sort(s);
        cudaEventRecord(ev[0], st);
        launch_incident_grid(s->grp, st);
        launch_push(s->grp, sorted, st);
        cudaEventRecord(ev[1], st);
        launch_scan(s->grp, st);
        cudaEventRecord(ev[2], st);
        if (sorted) launch_cell_sort(s->grp, st);
        cudaEventRecord(ev[3], st);
        launch_yee(s->grp, st);
        cudaEventRecord(ev[4], st);
        launch_step_end(s->grp, st);
        cudaEventRecord(ev[5], st);
        cudaError_t e = cudaEventSynchronize(ev[5]);
        if (e != cudaSuccess) {
            r = fail(s, PIC_ECUDA, "profiled step failed: %s", cudaGetErrorString(e));
            break;
        }
        for (int i = 0; i < 5; ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
            seconds[i] += 1e-3 * ms;
        }
    }
    for (int i = 0; i < 6; ++i) cudaEventDestroy(ev[i]);
    return r;
}

pic_status pic_destroy(pic_sim* s)
{
    if (!s) return PIC_OK;
    cudaDeviceSynchronize();
    batch_forget(s);
    if (s->step_graph.exec) cudaGraphExecDestroy(s->step_graph.exec);
    if (s->step_graph.graph) cudaGraphDestroy(s->step_graph.graph);
    if (s->sort_graph.exec) cudaGraphExecDestroy(s->sort_graph.exec);
    if (s->sort_graph.graph) cudaGraphDestroy(s->sort_graph.graph);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    if (s->cap_stream2) cudaStreamDestroy(s->cap_stream2);
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    if (s->ev_join) cudaEventDestroy(s->ev_join);
    dev_free(s, s->arena.base);
    delete s;
    return PIC_OK;
}

pic_status pic_info_get(pic_sim* s, pic_info* out, void* stream)
{
    if (!s || !out) return fail(s, PIC_EINVAL, "NULL argument");
    DevState ds;
    pic_status r = read_state(s, &ds, (cudaStream_t)stream);
    if (r != PIC_OK) return r;
    out->step = ds.step;
    out->time = ds.step * s->prm.dt;
    out->n_alive = ds.n_alive;
    out->n_exits = std::min<long long>(ds.n_exits, s->h.max_exits);
    out->status = ds.status;
    out->params = s->prm;
    return PIC_OK;
}

pic_status pic_set_step(pic_sim* s, int64_t step, void* stream)
{
    if (!s || step < 0) return fail(s, PIC_EINVAL, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    DevState ds;
    pic_status r = read_state(s, &ds, st);
    if (r != PIC_OK) return r;
    ds.step = step;
    return write_state(s, ds, st);
}

pic_status pic_test_hold_scan(pic_sim* s, int block, int spins)
{
    if (!s || spins < 1) return fail(s, PIC_EINVAL, "bad argument");
    s->h.scan_hold = block;
    s->h.scan_spins = spins;
    // the two fields of the device descriptor (read by every later launch of the step graph)
    const size_t o = offsetof(SimDev, scan_spins);
    static_assert(offsetof(SimDev, scan_hold) == offsetof(SimDev, scan_spins) + sizeof(int), "layout");
    CU_CHECK(s, cudaMemcpy(reinterpret_cast<char*>(s->d) + o, reinterpret_cast<const char*>(&s->h) + o, 2 * sizeof(int),
                           cudaMemcpyHostToDevice));
    return PIC_OK;
}

pic_status pic_set_particles(pic_sim* s, int64_t n, const double* x, const double* u, const double* w,
                             const int64_t* id, void* stream)
{
    if (!s) return fail(nullptr, PIC_EINVAL, "sim is NULL");
    if (n < 0 || n > s->pcap) return fail(s, PIC_ECAPACITY, "%lld particles exceed the capacity %lld", (long long)n,
                                          (long long)s->pcap);
    if (n > 0 && (!x || !u || !w || !id)) return fail(s, PIC_EINVAL, "NULL particle array");
    cudaStream_t st = (cudaStream_t)stream;
    const int D = s->cfg.dim, es = s->es;
    // host copies in the device layout (left uninitialised: every byte is written below)
    std::unique_ptr<unsigned[]> cell(new unsigned[n > 0 ? n : 1]), pid(new unsigned[n > 0 ? n : 1]);
    std::unique_ptr<char[]> off(new char[(size_t)D * n * es + 1]), mom(new char[(size_t)3 * n * es + 1]),
        wt(new char[(size_t)n * es + 1]);
    // converted on several host threads; each range reports its first invalid particle
    const int nb = 16;
    std::vector<long long> bad(nb, -1);
    std::vector<double> wmx(nb, 0.0);       // largest |weight| of each range
    std::atomic<int> slot{0}, wslot{0};
    host_parallel(n, 1 << 16, [&](long long p0, long long p1) {
        long long first = -1;
        double wm_r = 0.0;
        for (long long p = p0; p < p1 && first < 0; ++p) {
            wm_r = std::max(wm_r, std::fabs(w[p]));
            int c[3] = {0, 0, 0};
            for (int d = 0; d < D; ++d) {
                const double X = x[3 * p + d] / s->cfg.dx;
                const double fl = std::floor(X);
                c[d] = (int)fl;
                if (!(X >= s->h.margin) || !(X < s->h.n[d] - s->h.margin)) first = p;
                double o = X - fl;
                if (es == 4) {
                    float of = (float)o;
                    if (of >= 1.0f) of = std::nextafter(1.0f, 0.0f);
                    memcpy(&off[((size_t)d * n + p) * 4], &of, 4);
                } else {
                    memcpy(&off[((size_t)d * n + p) * 8], &o, 8);
                }
            }
            if (id[p] < 0 || id[p] >= (1ll << 31)) first = p;
            unsigned v = (unsigned)c[0];
            if (D > 1) v |= (unsigned)c[1] << s->h.cb[0];
            if (D > 2) v |= (unsigned)c[2] << (s->h.cb[0] + s->h.cb[1]);
            cell[p] = v;
            pid[p] = (unsigned)id[p];
            for (int d = 0; d < 3; ++d) {
                if (es == 4) {
                    float f = (float)u[3 * p + d];
                    memcpy(&mom[((size_t)d * n + p) * 4], &f, 4);
                } else {
                    memcpy(&mom[((size_t)d * n + p) * 8], &u[3 * p + d], 8);
                }
            }
            if (es == 4) {
                float f = (float)w[p];
                memcpy(&wt[(size_t)p * 4], &f, 4);
            } else {
                memcpy(&wt[(size_t)p * 8], &w[p], 8);
            }
        }
        if (first >= 0) {
            const int k = slot.fetch_add(1);
            if (k < nb) bad[k] = first;
        }
        const int kw = wslot.fetch_add(1);
        if (kw < nb) wmx[kw] = wm_r;
    });
    long long first_bad = -1;
    for (long long b : bad)
        if (b >= 0 && (first_bad < 0 || b < first_bad)) first_bad = b;
    if (first_bad >= 0) {
        const long long p = first_bad;
        if (id[p] < 0 || id[p] >= (1ll << 31)) {
            for (int d = 0; d < D; ++d) {
                const double X = x[3 * p + d] / s->cfg.dx;
                if (!(X >= s->h.margin) || !(X < s->h.n[d] - s->h.margin)) break;
                if (d == D - 1) return fail(s, PIC_EINVAL, "particle id out of range");
            }
        }
        for (int d = 0; d < D; ++d) {
            const double X = x[3 * p + d] / s->cfg.dx;
            if (!(X >= s->h.margin) || !(X < s->h.n[d] - s->h.margin))
                return fail(s, PIC_EINVAL, "particle %lld at %g cells on axis %d is outside [%d, %d)", p, X, d,
                            s->h.margin, s->h.n[d] - s->h.margin);
        }
        return fail(s, PIC_EINVAL, "particle id out of range");
    }
    if (n > 0) {
        CU_CHECK(s, cudaMemcpyAsync(s->h.cell[1], cell.get(), n * 4, cudaMemcpyHostToDevice, st));
        CU_CHECK(s, cudaMemcpyAsync(s->h.pid[1], pid.get(), n * 4, cudaMemcpyHostToDevice, st));
        for (int d = 0; d < D; ++d)
            CU_CHECK(s, cudaMemcpyAsync(s->h.off[1][d], &off[(size_t)d * n * es], n * es, cudaMemcpyHostToDevice, st));
        for (int d = 0; d < 3; ++d)
            CU_CHECK(s, cudaMemcpyAsync(s->h.mom[1][d], &mom[(size_t)d * n * es], n * es, cudaMemcpyHostToDevice, st));
        CU_CHECK(s, cudaMemcpyAsync(s->h.wgt[1], wt.get(), n * es, cudaMemcpyHostToDevice, st));
        // the host copies are released on return: the copies must have read them
        CU_CHECK(s, cudaStreamSynchronize(st));
    }
    s->prefix_group = 0;   // a new layout: the next step numbers its chunks first
    pic_status r = sort_linear_into_set0(s, n, st);
    if (r != PIC_OK) return r;
    // fields live in the set matching parity 0 now; keep the present field values
    DevState ds;
    if ((r = read_state(s, &ds, st)) != PIC_OK) return r;
    {
        // largest |weight| (rounded up in FP32): the scale of the FP32 push's fixed-point current
        double wm = 0.0;
        for (double v : wmx) wm = std::max(wm, v);
        ds.wmax = wm > 0 ? std::nextafter((float)wm, INFINITY) : 0.f;
        if ((r = write_state(s, ds, st)) != PIC_OK) return r;
    }
    if (ds.step == 0) return compute_rho_ion(s, st);
    return PIC_OK;
}

pic_status pic_set_fields(pic_sim* s, const double* fields, void* stream)
{
    if (!s || !fields) return fail(s, PIC_EINVAL, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    DevState ds;
    pic_status r = read_state(s, &ds, st);
    if (r != PIC_OK) return r;
    const int D = s->cfg.dim;
    const int ext[3] = {s->h.n[0] + 1, D > 1 ? s->h.n[1] + 1 : 1, D > 2 ? s->h.n[2] + 1 : 1};
    const long long ne = (long long)ext[0] * ext[1] * ext[2];
    // the device layout of E, B (zero at the points a component does not have and in the
    // ghost region), zero-filled on several host threads
    const size_t nbuf = (size_t)6 * s->nalloc_tot * s->es;
    std::unique_ptr<char[]> buf(new char[nbuf]);
    host_parallel((long long)((nbuf + 4095) / 4096), 1 << 10, [&](long long b0, long long b1) {
        const size_t a = (size_t)b0 * 4096, e = std::min(nbuf, (size_t)b1 * 4096);
        memset(buf.get() + a, 0, e - a);
    });
    // rows (comp, k, j) of the host array converted on up to 16 host threads
    const long long nrows = 6LL * ext[2] * ext[1];
    host_parallel(nrows, 256, [&](long long r0, long long r1) {
        for (long long r = r0; r < r1; ++r) {
            const int j = (int)(r % ext[1]), k = (int)((r / ext[1]) % ext[2]), comp = (int)(r / ((long long)ext[1] * ext[2]));
            const int c = comp % 3;
            for (int i = 0; i < ext[0]; ++i) {
                const int g[3] = {i, j, k};
                bool has = true;
                for (int d = 0; d < D; ++d) {
                    const bool stag = comp < 3 ? (d == c) : (d != c);
                    if (stag && g[d] > s->h.n[d] - 1) has = false;
                }
                if (!has) continue;
                const double v = fields[comp * ne + ((long long)k * ext[1] + j) * ext[0] + i];
                const long long o = comp * s->nalloc_tot + (long long)(D > 2 ? k + G : 0) * s->h.sz +
                                    (long long)(D > 1 ? j + G : 0) * s->h.sy + (i + GX);
                if (s->es == 4) {
                    float f = (float)v;
                    memcpy(&buf[o * 4], &f, 4);
                } else {
                    memcpy(&buf[o * 8], &v, 8);
                }
            }
        }
    });
    char* F = (char*)s->h.F;
    CU_CHECK(s, cudaMemcpyAsync(F + (size_t)comp_eb(ds.parity) * s->nalloc_tot * s->es, buf.get(), nbuf,
                                cudaMemcpyHostToDevice, st));
    CU_CHECK(s, cudaStreamSynchronize(st));
    return PIC_OK;
}

pic_status pic_diag(pic_sim* s, int kind, void* host_out, size_t bytes, void* stream)
{
    if (!s || !host_out) return fail(s, PIC_EINVAL, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    DevState ds;
    pic_status r = read_state(s, &ds, st);
    if (r != PIC_OK) return r;
    if (ds.status & FLAG_TIMEOUT) return fail(s, PIC_ETIMEOUT, "a device wait timed out (status 0x%x)", ds.status);
    if (ds.status & FLAG_CAPACITY)
        return fail(s, PIC_ECAPACITY, "a particle found no slot in its destination tile (status 0x%x)", ds.status);
    const int D = s->cfg.dim;
    const long long nex = std::min<long long>(ds.n_exits, s->h.max_exits);
    double vol = 1.0;
    for (int d = 0; d < D; ++d) vol *= s->cfg.dx;
    switch (kind) {
    case PIC_DIAG_ENERGIES: {
        if (bytes < 8 * sizeof(double)) return fail(s, PIC_ECAPACITY, "ENERGIES needs 64 bytes");
        CU_CHECK(s, cudaMemsetAsync(s->d_acc, 0, 4 * sizeof(double), st));
        launch_energy_fields(s->d, D, s->cfg.precision, s->h.n, s->d_acc, st);
        launch_energy_particles(s->d, D, s->cfg.precision, s->h.cap, nex, s->d_acc, st);
        CU_CHECK(s, cudaGetLastError());
        double acc[4];
        CU_CHECK(s, cudaMemcpyAsync(acc, s->d_acc, sizeof acc, cudaMemcpyDeviceToHost, st));
        CU_CHECK(s, cudaStreamSynchronize(st));
        double* o = (double*)host_out;
        for (int i = 0; i < 4; ++i) o[i] = acc[i] * vol;
        o[4] = (double)ds.n_alive;
        o[5] = (double)nex;
        o[6] = (double)ds.step;
        o[7] = ds.step * s->prm.dt;
        for (int i = 0; i < 4; ++i)
            if (!std::isfinite(o[i])) return fail(s, PIC_ENAN, "energy %d is not finite", i);
        return PIC_OK;
    }
    case PIC_DIAG_GAUSS: {
        if (bytes < sizeof(double)) return fail(s, PIC_ECAPACITY, "GAUSS needs 8 bytes");
        CU_CHECK(s, cudaMemsetAsync(s->h.scratch, 0, sizeof(double) * s->nalloc_tot, st));
        CU_CHECK(s, cudaMemsetAsync(s->d_bits, 0, 8, st));
        launch_charge(s->d, D, s->cfg.precision, s->h.cap, s->h.scratch, st);
        launch_gauss(s->d, D, s->cfg.precision, s->h.n, s->h.scratch, s->d_bits, st);
        CU_CHECK(s, cudaGetLastError());
        unsigned long long bits;
        CU_CHECK(s, cudaMemcpyAsync(&bits, s->d_bits, 8, cudaMemcpyDeviceToHost, st));
        CU_CHECK(s, cudaStreamSynchronize(st));
        double v;
        memcpy(&v, &bits, 8);
        *(double*)host_out = v;
        return PIC_OK;
    }
    case PIC_DIAG_PARTICLES: {
        const long long n = ds.n_alive;
        if (bytes < (size_t)n * 8 * sizeof(double)) return fail(s, PIC_ECAPACITY, "PARTICLES needs %lld bytes", n * 64);
        const int q = ds.parity, es = s->es, nt = s->h.nptiles;
        // the tiles' occupied slots of the current set, in tile order
        std::vector<int> toff(nt + 1), tnum(nt);
        CU_CHECK(s, cudaMemcpyAsync(toff.data(), s->h.toff[q], (nt + 1) * 4, cudaMemcpyDeviceToHost, st));
        CU_CHECK(s, cudaMemcpyAsync(tnum.data(), s->h.tnum[q], nt * 4, cudaMemcpyDeviceToHost, st));
        CU_CHECK(s, cudaStreamSynchronize(st));
        const long long nu = std::min<long long>(toff[nt], s->h.cap);
        long long tot = 0;
        for (int t = 0; t < nt; ++t) tot += tnum[t];
        if (tot != n) return fail(s, PIC_ECUDA, "tile counts (%lld) disagree with the particle count (%lld)", tot, n);
        // host copies (left uninitialised: the copies fill them)
        std::unique_ptr<unsigned[]> cell(new unsigned[nu + 1]), pid(new unsigned[nu + 1]);
        std::unique_ptr<char[]> off(new char[(size_t)D * nu * es + 1]), mom(new char[(size_t)3 * nu * es + 1]),
            wt(new char[(size_t)nu * es + 1]);
        if (nu > 0) {
            CU_CHECK(s, cudaMemcpyAsync(cell.get(), s->h.cell[q], nu * 4, cudaMemcpyDeviceToHost, st));
            CU_CHECK(s, cudaMemcpyAsync(pid.get(), s->h.pid[q], nu * 4, cudaMemcpyDeviceToHost, st));
            for (int d = 0; d < D; ++d)
                CU_CHECK(s, cudaMemcpyAsync(&off[(size_t)d * nu * es], s->h.off[q][d], nu * es, cudaMemcpyDeviceToHost, st));
            for (int d = 0; d < 3; ++d)
                CU_CHECK(s, cudaMemcpyAsync(&mom[(size_t)d * nu * es], s->h.mom[q][d], nu * es, cudaMemcpyDeviceToHost, st));
            CU_CHECK(s, cudaMemcpyAsync(wt.get(), s->h.wgt[q], nu * es, cudaMemcpyDeviceToHost, st));
        }
        CU_CHECK(s, cudaStreamSynchronize(st));
        auto rd = [&](const char* v, size_t idx) {
            if (es == 4) {
                float f;
                memcpy(&f, v + idx * 4, 4);
                return (double)f;
            }
            double xv;
            memcpy(&xv, v + idx * 8, 8);
            return xv;
        };
        // record k of the output = the tiles' particles in tile order; tiles converted on
        // several host threads from their first record index
        std::vector<long long> first(nt + 1, 0);
        for (int t = 0; t < nt; ++t)
            first[t + 1] = first[t] + std::max<long long>(0, std::min<long long>((long long)toff[t] + tnum[t], nu) - toff[t]);
        if (first[nt] != n) return fail(s, PIC_ECUDA, "tile slots hold %lld particles, expected %lld", first[nt], n);
        double* o = (double*)host_out;
        host_parallel(nt, std::max<long long>(1, (1 << 16) * (long long)nt / std::max<long long>(n, 1)),
                      [&](long long t0, long long t1) {
            for (long long t = t0; t < t1; ++t) {
                long long k = first[t];
                const long long p1 = std::min<long long>((long long)toff[t] + tnum[t], nu);
                for (long long p = toff[t]; p < p1; ++p, ++k) {
                    const unsigned cl = cell[p];
                    int c[3];
                    c[0] = (int)(cl & ((1u << s->h.cb[0]) - 1u));
                    c[1] = D > 1 ? (int)((cl >> s->h.cb[0]) & ((1u << s->h.cb[1]) - 1u)) : 0;
                    c[2] = D > 2 ? (int)(cl >> (s->h.cb[0] + s->h.cb[1])) : 0;
                    for (int d = 0; d < 3; ++d)
                        o[8 * k + d] = d < D ? ((double)c[d] + rd(off.get(), (size_t)d * nu + p)) * s->cfg.dx : 0.0;
                    for (int d = 0; d < 3; ++d) o[8 * k + 3 + d] = rd(mom.get(), (size_t)d * nu + p);
                    o[8 * k + 6] = rd(wt.get(), p);
                    o[8 * k + 7] = (double)pid[p];
                }
            }
        });
        return PIC_OK;
    }
    case PIC_DIAG_EXITS: {
        if (bytes < (size_t)nex * EXIT_DOUBLES * 8) return fail(s, PIC_ECAPACITY, "EXITS needs %lld bytes", nex * 48);
        if (nex > 0)
            CU_CHECK(s, cudaMemcpyAsync(host_out, s->h.exits, nex * EXIT_DOUBLES * 8, cudaMemcpyDeviceToHost, st));
        CU_CHECK(s, cudaStreamSynchronize(st));
        return PIC_OK;
    }
    case PIC_DIAG_FIELDS: {
        const int ext[3] = {s->h.n[0] + 1, D > 1 ? s->h.n[1] + 1 : 1, D > 2 ? s->h.n[2] + 1 : 1};
        const long long ne = (long long)ext[0] * ext[1] * ext[2];
        if (bytes < (size_t)9 * ne * 8) return fail(s, PIC_ECAPACITY, "FIELDS needs %lld bytes", 9 * ne * 8);
        const int es = s->es;
        std::vector<char> eb((size_t)6 * s->nalloc_tot * es), jb((size_t)3 * s->nalloc_tot * es);
        const char* F = (const char*)s->h.F;
        CU_CHECK(s, cudaMemcpyAsync(eb.data(), F + (size_t)comp_eb(ds.parity) * s->nalloc_tot * es, eb.size(),
                                    cudaMemcpyDeviceToHost, st));
        // the current deposited by the last step sits in J of the other set
        CU_CHECK(s, cudaMemcpyAsync(jb.data(), F + (size_t)comp_j(1 - ds.parity) * s->nalloc_tot * es, jb.size(),
                                    cudaMemcpyDeviceToHost, st));
        CU_CHECK(s, cudaStreamSynchronize(st));
        double* o = (double*)host_out;
        // rows (comp, k, j) of the host array converted on up to 16 host threads
        const long long nrows = 9LL * ext[2] * ext[1];
        host_parallel(nrows, 256, [&](long long r0, long long r1) {
            for (long long r = r0; r < r1; ++r) {
                const int j = (int)(r % ext[1]), k = (int)((r / ext[1]) % ext[2]);
                const int comp = (int)(r / ((long long)ext[1] * ext[2]));
                const std::vector<char>& src = comp < 6 ? eb : jb;
                const int sc = comp < 6 ? comp : comp - 6;
                const int c = comp % 3;
                for (int i = 0; i < ext[0]; ++i) {
                    const int g[3] = {i, j, k};
                    bool has = true;
                    for (int d = 0; d < D; ++d) {
                        const bool stag = (comp < 3 || comp >= 6) ? (d == c) : (d != c);
                        if (stag && g[d] > s->h.n[d] - 1) has = false;
                    }
                    double v = 0.0;
                    if (has) {
                        const long long idx = sc * s->nalloc_tot + (long long)(D > 2 ? k + G : 0) * s->h.sz +
                                              (long long)(D > 1 ? j + G : 0) * s->h.sy + (i + GX);
                        if (es == 4) {
                            float f;
                            memcpy(&f, &src[idx * 4], 4);
                            v = f;
                        } else {
                            memcpy(&v, &src[idx * 8], 8);
                        }
                    }
                    o[comp * ne + ((long long)k * ext[1] + j) * ext[0] + i] = v;
                }
            }
        });
        return PIC_OK;
    }
    default:
        return fail(s, PIC_EINVAL, "unknown diagnostic kind %d", kind);
    }
}

pic_status pic_histogram(pic_sim* s, int n_e, double e_max, int n_a, double* host_out, void* stream)
{
    if (!s || !host_out || n_e <= 0 || n_a <= 0 || !(e_max > 0)) return fail(s, PIC_EINVAL, "bad argument");
    int prev = -1;
    CU_CHECK(s, cudaGetDevice(&prev));
    if (prev != s->device) CU_CHECK(s, cudaSetDevice(s->device));
    struct Restore {
        int d, now;
        ~Restore()
        {
            if (d >= 0 && d != now) cudaSetDevice(d);
        }
    } restore{prev, s->device};
    cudaStream_t st = (cudaStream_t)stream;
    DevState ds;
    pic_status r = read_state(s, &ds, st);
    if (r != PIC_OK) return r;
    if (ds.status & FLAG_TIMEOUT) return fail(s, PIC_ETIMEOUT, "a device wait timed out (status 0x%x)", ds.status);
    if (ds.status & FLAG_CAPACITY)
        return fail(s, PIC_ECAPACITY, "a particle found no slot in its destination tile (status 0x%x)", ds.status);
    const size_t nb = (size_t)n_e * n_a;
    if (nb > (size_t)s->nalloc_tot) return fail(s, PIC_ECAPACITY, "too many bins");
    CU_CHECK(s, cudaMemsetAsync(s->h.scratch, 0, nb * 8, st));
    launch_histogram(s->d, s->cfg.dim, s->cfg.precision, s->h.cap, std::min<long long>(ds.n_exits, s->h.max_exits),
                     n_e, e_max, n_a, s->h.scratch, st);
    CU_CHECK(s, cudaGetLastError());
    CU_CHECK(s, cudaMemcpyAsync(host_out, s->h.scratch, nb * 8, cudaMemcpyDeviceToHost, st));
    CU_CHECK(s, cudaStreamSynchronize(st));
    return PIC_OK;
}

pic_status pic_eval_incident(pic_sim* s, int64_t n, const double* pts, double* out, void* stream)
{
    if (!s || n < 0 || (n > 0 && (!pts || !out))) return fail(s, PIC_EINVAL, "bad argument");
    if (n == 0) return PIC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    // a diagnostic entry point: temporary device buffers for the points and the results
    double* dp = nullptr;
    CU_CHECK(s, cudaMalloc(&dp, (size_t)n * 10 * sizeof(double)));
    double* dout = dp + 4 * n;
    cudaError_t e = cudaMemcpyAsync(dp, pts, (size_t)n * 4 * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        launch_eval_incident(s->d, s->cfg.dim, s->cfg.precision, n, dp, dout, st);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, (size_t)n * 6 * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(dp);
    if (e != cudaSuccess) return fail(s, PIC_ECUDA, "incident-field evaluation failed: %s", cudaGetErrorString(e));
    return PIC_OK;
}

}  // extern "C"
