// Diagnostics kernels (off the stepping loop): charge density, Gauss-law residual,
// field and kinetic energies (Sec. 3.1, Eqs. L2_t and L2_t_cross use these integrals),
// energy-angle histograms (Sec. 4.2: angle measured from the propagation axis) and a
// point evaluator of the incident field.  Accumulation is in double precision.
#include <cuda_runtime.h>

#include <algorithm>

#include <mutex>

#include "beam.cuh"
#include "sff_common.cuh"
#include "sff_kernels.h"
#include "sim_internal.h"

namespace sff {

template <int D>
__device__ __forceinline__ void decode_cell_d(const SimDev& S, unsigned cl, int c[3])
{
    c[0] = (int)(cl & ((1u << S.cb[0]) - 1u));
    c[1] = 0;
    c[2] = 0;
    if constexpr (D > 1) c[1] = (int)((cl >> S.cb[0]) & ((1u << S.cb[1]) - 1u));
    if constexpr (D > 2) c[2] = (int)(cl >> (S.cb[0] + S.cb[1]));
}

// Slot p of buffer set par holds a particle: slots after a tile's particles hold DEAD or
// stale records of earlier steps, whose cell puts them outside their tile's occupied slots.
template <int D>
__device__ __forceinline__ bool slot_live(const SimDev& S, int par, long long p)
{
    const unsigned cl = S.cell[par][p];
    if (cl == DEAD) return false;
    int c[3];
    decode_cell_d<D>(S, cl, c);
    int t = 0, mul = 1;
    for (int d = 0; d < D; ++d) {
        if (c[d] >= S.n[d]) return false;
        t += (c[d] / S.pt[d]) * mul;
        mul *= S.npt[d];
    }
    return (unsigned long long)(p - S.toff[par][t]) < (unsigned long long)S.tnum[par][t];
}

// end of the occupied slot range of buffer set par (n: slots of a set)
__device__ __forceinline__ long long slots_used(const SimDev& S, int par, long long n)
{
    return min(n, (long long)S.toff[par][S.nptiles]);
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// charge density scale * rho_e, rho_e = -sum w S(x - x_node), added on the primal nodes
// (array coordinates); n: slots of a buffer set (as for the other particle diagnostics)
template <int D, typename R>
__global__ void k_charge(const SimDev* __restrict__ sim, long long n, double* __restrict__ rho, double scale)
{
    const SimDev& S = *sim;
    const int par = S.st->parity;
    const long long nu = slots_used(S, par, n);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < nu;
         p += (long long)gridDim.x * blockDim.x) {
        if (!slot_live<D>(S, par, p)) continue;
        int c[3];
        decode_cell_d<D>(S, S.cell[par][p], c);
        double w[3][3];
        int lo[3] = {0, 0, 0};
        for (int d = 0; d < 3; ++d) {
            if (d < D) {
                const double o = (double)reinterpret_cast<const R*>(S.off[par][d])[p];
                const int h = o >= 0.5;
                const double dl = o - h;
                w[d][0] = 0.5 * (0.5 - dl) * (0.5 - dl);
                w[d][1] = 0.75 - dl * dl;
                w[d][2] = 0.5 * (0.5 + dl) * (0.5 + dl);
                lo[d] = c[d] + h - 1 + (d == 0 ? GX : G);
            } else {
                w[d][0] = 1.0;
                w[d][1] = w[d][2] = 0.0;
            }
        }
        const double q = -scale * (double)reinterpret_cast<const R*>(S.wgt[par])[p];
        const int nk = D > 2 ? 3 : 1, nj = D > 1 ? 3 : 1;
        for (int k = 0; k < nk; ++k)
            for (int j = 0; j < nj; ++j)
                for (int i = 0; i < 3; ++i)
                    atomicAdd(&rho[(long long)(lo[2] + k) * S.sz + (long long)(lo[1] + j) * S.sy + lo[0] + i],
                              q * w[0][i] * w[1][j] * w[2][k]);
    }
}

// max |div E - rho - rho_ion| over interior primal nodes; result as ordered bits
template <int D, typename R>
__global__ void k_gauss(const SimDev* __restrict__ sim, const double* __restrict__ rho, int n0, int n1, int n2,
                        unsigned long long* __restrict__ out)
{
    const SimDev& S = *sim;
    const R* F = reinterpret_cast<const R*>(S.F);
    const long long eb = (long long)comp_eb(S.st->parity) * S.sc;
    const long long total = (long long)n0 * n1 * n2;   // interior extents
    double worst = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k % n0) + 1;
        const int j = D > 1 ? (int)((k / n0) % n1) + 1 : 0;
        const int l = D > 2 ? (int)(k / ((long long)n0 * n1)) + 1 : 0;
        const long long o = (long long)(D > 2 ? l + G : 0) * S.sz + (long long)(D > 1 ? j + G : 0) * S.sy + (i + GX);
        double div = ((double)F[eb + o] - (double)F[eb + o - 1]) * S.inv_dx;
        if (D > 1) div += ((double)F[eb + S.sc + o] - (double)F[eb + S.sc + o - S.sy]) * S.inv_dx;
        if (D > 2) div += ((double)F[eb + 2 * S.sc + o] - (double)F[eb + 2 * S.sc + o - S.sz]) * S.inv_dx;
        const double r = fabs(div - rho[o] - S.rho_ion[o]);
        worst = fmax(worst, r);
    }
    for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(worst));
}

// 1/2 sum F^2 dx^dim over the points each component has: [0] scattered, [1] scattered + incident
template <int D, typename R>
__global__ void k_energy_fields(const SimDev* __restrict__ sim, int m0, int m1, int m2, double* __restrict__ acc)
{
    const SimDev& S = *sim;
    const R* F = reinterpret_cast<const R*>(S.F);
    const int par = S.st->parity;
    const long long eb = (long long)comp_eb(par) * S.sc;
    const double t = (double)S.st->step * S.dt;
    const BeamC<R>& bc = beam_of<R>(S);
    const long long total = (long long)m0 * m1 * m2;   // extents n+1 on resolved axes
    double es = 0.0, et = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const int g[3] = {(int)(k % m0), (int)((k / m0) % m1), (int)(k / ((long long)m0 * m1))};
        const long long o = (long long)(D > 2 ? g[2] + G : 0) * S.sz + (long long)(D > 1 ? g[1] + G : 0) * S.sy +
                            (g[0] + GX);
        for (int comp = 0; comp < 6; ++comp) {
            const int c = comp % 3;
            bool has = true;
            int cc[3] = {g[0], g[1], g[2]};
            R oo[3] = {R(0), R(0), R(0)};
            for (int d = 0; d < D; ++d) {
                const bool stag = comp < 3 ? (d == c) : (d != c);
                if (stag) {
                    if (g[d] > S.n[d] - 1) has = false;
                    oo[d] = R(0.5);
                }
            }
            if (!has) continue;
            const double f = (double)F[eb + comp * S.sc + o];
            es += 0.5 * f * f;
            double inc = 0.0;
            if (S.beam != BEAM_NONE && !S.tf) {
                R Ei[3], Bi[3];
                const PhaseRef<R> pr = phase_ref<R>(S, t, cc[0]);
                incident_at<D, R>(S, bc, pr, cc, oo, Ei, Bi);
                inc = comp < 3 ? (double)Ei[c] : (double)Bi[c];
            }
            et += 0.5 * (f + inc) * (f + inc);
        }
    }
    es = warp_sum(es);
    et = warp_sum(et);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&acc[0], es);
        atomicAdd(&acc[1], et);
    }
}

// [2] sum w (gamma - 1) of electrons in the box, [3] of exit records (times dx^dim on the host)
template <int D, typename R>
__global__ void k_energy_particles(const SimDev* __restrict__ sim, long long n, long long nex, double* __restrict__ acc)
{
    const SimDev& S = *sim;
    const int par = S.st->parity;
    double ka = 0.0, ke = 0.0;
    const long long nu = slots_used(S, par, n);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < nu;
         p += (long long)gridDim.x * blockDim.x) {
        if (!slot_live<D>(S, par, p)) continue;
        double u2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            const double u = (double)reinterpret_cast<const R*>(S.mom[par][d])[p];
            u2 += u * u;
        }
        ka += (double)reinterpret_cast<const R*>(S.wgt[par])[p] * (sqrt(1.0 + u2) - 1.0);
    }
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < nex;
         p += (long long)gridDim.x * blockDim.x) {
        const double* e = S.exits + p * EXIT_DOUBLES;
        ke += e[3] * (sqrt(1.0 + e[0] * e[0] + e[1] * e[1] + e[2] * e[2]) - 1.0);
    }
    ka = warp_sum(ka);
    ke = warp_sum(ke);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&acc[2], ka);
        atomicAdd(&acc[3], ke);
    }
}

__device__ __forceinline__ void hist_add(double* bins, double ux, double uy, double uz, double w, int n_e, double e_max,
                                         int n_a)
{
    const double u2 = ux * ux + uy * uy + uz * uz;
    const double ek = sqrt(1.0 + u2) - 1.0;
    if (!(ek < e_max) || ek < 0.0) return;
    const double ang = atan2(sqrt(uy * uy + uz * uz), ux);   // from the +x (propagation) axis
    int ie = (int)(ek / e_max * n_e);
    int ia = (int)(ang / 3.14159265358979323846 * n_a);
    ie = min(max(ie, 0), n_e - 1);
    ia = min(max(ia, 0), n_a - 1);
    atomicAdd(&bins[(long long)ie * n_a + ia], w);
}

template <int D, typename R>
__global__ void k_histogram(const SimDev* __restrict__ sim, long long n, long long nex, int n_e, double e_max, int n_a,
                            double* __restrict__ bins)
{
    const SimDev& S = *sim;
    const int par = S.st->parity;
    const long long nu = slots_used(S, par, n);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < nu;
         p += (long long)gridDim.x * blockDim.x) {
        if (!slot_live<D>(S, par, p)) continue;
        hist_add(bins, (double)reinterpret_cast<const R*>(S.mom[par][0])[p],
                 (double)reinterpret_cast<const R*>(S.mom[par][1])[p],
                 (double)reinterpret_cast<const R*>(S.mom[par][2])[p], (double)reinterpret_cast<const R*>(S.wgt[par])[p],
                 n_e, e_max, n_a);
    }
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < nex;
         p += (long long)gridDim.x * blockDim.x) {
        const double* e = S.exits + p * EXIT_DOUBLES;
        hist_add(bins, e[0], e[1], e[2], e[3], n_e, e_max, n_a);
    }
}

// incident field at arbitrary points (x, y, z, t), grid coordinates
template <int D, typename R>
__global__ void k_eval_incident(const SimDev* __restrict__ sim, long long n, const double* __restrict__ pts,
                                double* __restrict__ out)
{
    const SimDev& S = *sim;
    const BeamC<R>& bc = beam_of<R>(S);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        int c[3] = {0, 0, 0};
        R o[3] = {R(0), R(0), R(0)};
        for (int d = 0; d < D; ++d) {
            const double X = pts[4 * p + d] * S.inv_dx;
            const double fl = floor(X);
            c[d] = (int)fl;
            o[d] = R(X - fl);
        }
        R E[3], B[3];
        const PhaseRef<R> pr = phase_ref<R>(S, pts[4 * p + 3], c[0]);
        incident_at<D, R>(S, bc, pr, c, o, E, B);
        for (int d = 0; d < 3; ++d) {
            out[6 * p + d] = (double)E[d];
            out[6 * p + 3 + d] = (double)B[d];
        }
    }
}

// ---- host wrappers ----
static int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, (long long)device_sms() * 8)); }

#define SFF_DISPATCH3(dim, prec, FN, ...)                       \
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

template <int D, typename R>
static void charge_t(const SimDev* sim, long long n, double* rho, double scale, cudaStream_t s)
{
    if (n > 0) k_charge<D, R><<<grid_for(n), 256, 0, s>>>(sim, n, rho, scale);
}
void launch_charge(const SimDev* sim, int dim, int prec, long long n_slots, double* rho, cudaStream_t s, double scale)
{
    SFF_DISPATCH3(dim, prec, charge_t, sim, n_slots, rho, scale, s);
}

template <int D, typename R>
static void gauss_t(const SimDev* sim, const double* rho, const int n[3], unsigned long long* out, cudaStream_t s)
{
    const int n0 = n[0] - 1, n1 = D > 1 ? n[1] - 1 : 1, n2 = D > 2 ? n[2] - 1 : 1;
    const long long tot = (long long)n0 * n1 * n2;
    k_gauss<D, R><<<grid_for(tot), 256, 0, s>>>(sim, rho, n0, n1, n2, out);
}
void launch_gauss(const SimDev* sim, int dim, int prec, const int n[3], const double* rho, unsigned long long* out_bits,
                  cudaStream_t s)
{
    SFF_DISPATCH3(dim, prec, gauss_t, sim, rho, n, out_bits, s);
}

template <int D, typename R>
static void efield_t(const SimDev* sim, const int n[3], double* acc, cudaStream_t s)
{
    const int m0 = n[0] + 1, m1 = D > 1 ? n[1] + 1 : 1, m2 = D > 2 ? n[2] + 1 : 1;
    const long long tot = (long long)m0 * m1 * m2;
    k_energy_fields<D, R><<<grid_for(tot), 256, 0, s>>>(sim, m0, m1, m2, acc);
}
void launch_energy_fields(const SimDev* sim, int dim, int prec, const int n[3], double* acc2, cudaStream_t s)
{
    SFF_DISPATCH3(dim, prec, efield_t, sim, n, acc2, s);
}

template <int D, typename R>
static void epart_t(const SimDev* sim, long long n, long long nex, double* acc, cudaStream_t s)
{
    k_energy_particles<D, R><<<grid_for(std::max(n, nex)), 256, 0, s>>>(sim, n, nex, acc);
}
void launch_energy_particles(const SimDev* sim, int dim, int prec, long long n_alive, long long n_exits, double* acc2,
                             cudaStream_t s)
{
    SFF_DISPATCH3(dim, prec, epart_t, sim, n_alive, n_exits, acc2, s);
}

template <int D, typename R>
static void hist_t(const SimDev* sim, long long n, long long nex, int n_e, double e_max, int n_a, double* bins,
                   cudaStream_t s)
{
    k_histogram<D, R><<<grid_for(std::max(n, nex)), 256, 0, s>>>(sim, n, nex, n_e, e_max, n_a, bins);
}
void launch_histogram(const SimDev* sim, int dim, int prec, long long n_alive, long long n_exits, int n_e,
                      double e_max, int n_a, double* bins, cudaStream_t s)
{
    SFF_DISPATCH3(dim, prec, hist_t, sim, n_alive, n_exits, n_e, e_max, n_a, bins, s);
}

template <int D, typename R>
static void evalinc_t(const SimDev* sim, long long n, const double* pts, double* out, cudaStream_t s)
{
    if (n > 0) k_eval_incident<D, R><<<grid_for(n), 256, 0, s>>>(sim, n, pts, out);
}
void launch_eval_incident(const SimDev* sim, int dim, int prec, long long n, const double* pts, double* out,
                          cudaStream_t s)
{
    SFF_DISPATCH3(dim, prec, evalinc_t, sim, n, pts, out, s);
}

}  // namespace sff

// ---- histogram with statically allocated bins (pic_histogram_static) ------------------------
// The bins live in this file-scope array, so the call path allocates nothing.  Host code only
// ever passes the array's device address, looked up once per device.
static __device__ __align__(256) double g_hist_bins[PIC_HIST_STATIC_MAX_BINS];

namespace {
std::mutex g_hist_mu;
double* g_hist_addr[64] = {nullptr};   // device address of g_hist_bins per device ordinal
}  // namespace

namespace {
// Makes `dev` the calling thread's current device for the guard's lifetime.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        ok = prev == dev || cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (ok && prev >= 0) cudaSetDevice(prev);
    }
};
}  // namespace

extern "C" pic_status pic_histogram_static(pic_sim* s, int n_e, double e_max, int n_a, double* host_out, void* stream)
{
    if (!s || !host_out || n_e <= 0 || n_a <= 0 || !(e_max > 0)) return PIC_EINVAL;
    if ((long long)n_e * n_a > PIC_HIST_STATIC_MAX_BINS) {
        s->err = "pic_histogram_static: n_e * n_a exceeds PIC_HIST_STATIC_MAX_BINS (16384)";
        return PIC_EINVAL;
    }
    // the simulation's device is current for the look-up and every launch below
    const int dev = s->device;
    DeviceGuard guard(dev);
    if (!guard.ok || dev < 0 || dev >= 64) {
        s->err = "pic_histogram_static: cannot make the simulation's device current";
        return PIC_ENODEV;
    }
    double* bins = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_hist_mu);
        if (!g_hist_addr[dev]) {
            // set-up, once per device, with that device current
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_hist_bins);
            if (e != cudaSuccess) {
                s->err = std::string("pic_histogram_static: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
                return PIC_ECUDA;
            }
            g_hist_addr[dev] = static_cast<double*>(p);
        }
        bins = g_hist_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    sff::DevState ds;
    cudaError_t e = cudaMemcpyAsync(&ds, s->h.st, sizeof(sff::DevState), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        s->err = std::string("pic_histogram_static: ") + cudaGetErrorString(e);
        return PIC_ECUDA;
    }
    // the device status word, as pic_diag reads it
    if (ds.status & sff::FLAG_TIMEOUT) {
        s->err = "pic_histogram_static: a device wait timed out";
        return PIC_ETIMEOUT;
    }
    if (ds.status & sff::FLAG_CAPACITY) {
        s->err = "pic_histogram_static: a particle found no slot in its destination tile";
        return PIC_ECAPACITY;
    }
    const size_t nb = (size_t)n_e * n_a;
    e = cudaMemsetAsync(bins, 0, nb * sizeof(double), st);
    if (e == cudaSuccess) {
        sff::launch_histogram(s->d, s->cfg.dim, s->cfg.precision, s->h.cap,
                              std::min<long long>(ds.n_exits, s->h.max_exits), n_e, e_max, n_a, bins, st);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, bins, nb * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        s->err = std::string("pic_histogram_static: ") + cudaGetErrorString(e);
        return PIC_ECUDA;
    }
    return PIC_OK;
}
