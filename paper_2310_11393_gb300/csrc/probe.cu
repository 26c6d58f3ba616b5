// Pipe-rate probes (no counterpart in the paper: measurement aids for the roofline of the
// fused push, whose transcendental-heavy closed form is bound by arithmetic issue rather
// than by HBM).  Each probe keeps every SM busy with independent dependency chains of one
// instruction kind and times them with CUDA events; the SM clock during the probe is
// measured from clock64() against the same events.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "../../include/pic.h"
#include "sff_kernels.h"

namespace sff {

int device_sms()
{
    static std::mutex mu;
    static std::vector<int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    std::lock_guard<std::mutex> lk(mu);
    if ((int)cache.size() <= dev) cache.resize(dev + 1, 0);
    if (cache[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 1;
        cache[dev] = n;
    }
    return cache[dev];
}

}  // namespace sff

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int CHAINS = 8;   // independent chains per thread: enough to cover the pipe latency

// FP32 fused multiply-add chains: a <- a * m + c (|m| < 1 keeps every chain bounded).
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_ffma(int iters, float m, float c, float* sink,
                                                               long long* cycles)
{
    float a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = (float)(threadIdx.x + k);
    const long long t0 = clock64();
#pragma unroll 16
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[k]) : "f"(m), "f"(c));
    }
    const long long t1 = clock64();
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
    if (s == -1.0f) sink[0] = s;   // never true: keeps the chains alive
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_dfma(int iters, double m, double c, double* sink,
                                                               long long* cycles)
{
    double a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = (double)(threadIdx.x + k);
    const long long t0 = clock64();
#pragma unroll 16
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(a[k]) : "d"(m), "d"(c));
    }
    const long long t1 = clock64();
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
    if (s == -1.0) sink[0] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// Special-function unit: the approximate sine, a <- sin.approx(a) + c.
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_mufu(int iters, float c, float* sink, long long* cycles)
{
    float a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = 0.1f * (float)k;
    const long long t0 = clock64();
#pragma unroll 16
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) {
            float y;
            asm volatile("sin.approx.f32 %0, %1;" : "=f"(y) : "f"(a[k]));
            a[k] = y + c;
        }
    }
    const long long t1 = clock64();
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
    if (s == -1.0f) sink[0] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

struct Timing {
    double seconds = 0, cycles = 0;
};

template <typename L>
static cudaError_t timed(cudaStream_t st, L launch, int reps, Timing* out, long long* d_cyc, int nblk)
{
    cudaEvent_t e0, e1;
    cudaError_t err = cudaEventCreate(&e0);
    if (err != cudaSuccess) return err;
    err = cudaEventCreate(&e1);
    if (err != cudaSuccess) {
        cudaEventDestroy(e0);
        return err;
    }
    launch();   // warm-up (clocks, instruction cache)
    float best = -1;
    double cyc = 0;
    std::vector<long long> h(nblk);
    for (int r = 0; r < reps && err == cudaSuccess; ++r) {
        cudaEventRecord(e0, st);
        launch();
        cudaEventRecord(e1, st);
        err = cudaEventSynchronize(e1);
        if (err != cudaSuccess) break;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        err = cudaMemcpy(h.data(), d_cyc, sizeof(long long) * nblk, cudaMemcpyDeviceToHost);
        if (best < 0 || ms < best) {
            best = ms;
            cyc = (double)*std::max_element(h.begin(), h.end());
        }
    }
    if (err == cudaSuccess) err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    out->seconds = best * 1e-3;
    out->cycles = cyc;
    return err;
}

}  // namespace

extern "C" pic_status pic_probe_peaks(pic_peaks* out, void* stream)
{
    if (!out) return PIC_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return PIC_ENODEV;
    cudaStream_t st = (cudaStream_t)stream;
    const int sms = sff::device_sms();
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_ffma, PROBE_THREADS, 0);
    per_sm = std::max(1, std::min(per_sm, 8));
    const int nblk = sms * per_sm;
    const double threads = (double)nblk * PROBE_THREADS;
    float* sink = nullptr;
    long long* cyc = nullptr;
    if (cudaMalloc(&sink, 64) != cudaSuccess) return PIC_ENOMEM;
    if (cudaMalloc(&cyc, sizeof(long long) * nblk) != cudaSuccess) {
        cudaFree(sink);
        return PIC_ENOMEM;
    }
    Timing tf, td, tm;
    const int it32 = 1 << 19, it64 = 1 << 14, itmu = 1 << 16;   // 30-60 ms each on a GB300
    cudaError_t e = timed(st, [&] { k_probe_ffma<<<nblk, PROBE_THREADS, 0, st>>>(it32, 0.999999f, 1e-6f, sink, cyc); },
                          3, &tf, cyc, nblk);
    if (e == cudaSuccess)
        e = timed(st, [&] { k_probe_dfma<<<nblk, PROBE_THREADS, 0, st>>>(it64, 0.999999, 1e-6, (double*)sink, cyc); },
                  3, &td, cyc, nblk);
    if (e == cudaSuccess)
        e = timed(st, [&] { k_probe_mufu<<<nblk, PROBE_THREADS, 0, st>>>(itmu, 1e-3f, sink, cyc); }, 3, &tm, cyc, nblk);
    cudaFree(sink);
    cudaFree(cyc);
    if (e != cudaSuccess) return PIC_ECUDA;
    out->sms = sms;
    out->fp32_tflops = threads * it32 * CHAINS * 2.0 / tf.seconds * 1e-12;
    out->fp64_tflops = threads * it64 * CHAINS * 2.0 / td.seconds * 1e-12;
    out->sfu_gops = threads * itmu * CHAINS / tm.seconds * 1e-9;
    out->sm_clock_mhz = tf.cycles / tf.seconds * 1e-6;
    out->fp32_flop_per_clk_sm = out->fp32_tflops * 1e12 / (out->sm_clock_mhz * 1e6) / sms;
    return PIC_OK;
}
