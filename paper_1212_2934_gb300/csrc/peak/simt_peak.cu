// SIMT arithmetic peaks of the current GPU, measured (libffpeak.so).
//
// The Barnes-Hut traversal and the all-pairs kernel are bound by plain FP32 (or
// FP64) arithmetic, not by tensor cores or memory, so their roofline is the rate
// at which the SMs retire fused multiply-adds.  These kernels measure that rate
// directly: every thread runs kChains independent FMA chains (enough
// independent work to cover the pipeline latency) for a fixed number of
// rounds, on a grid of several blocks per SM, timed with CUDA events.  Three
// forms: scalar FP32 fma, the paired FP32 fma that operates on two floats at
// once, and FP64 fma.  Each block also reads its SM clock counter and the
// global nanosecond timer at start and end, so the call reports the SM clock
// the arithmetic actually ran at.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <typename T>
struct Fma;

template <>
struct Fma<float> {
    static constexpr int kFlops = 2;
    __device__ __forceinline__ static float op(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    __device__ __forceinline__ static float init(int i) { return 1.0f + 1e-7f * (float)i; }
    __device__ __forceinline__ static double sum(float a) { return (double)a; }
};

template <>
struct Fma<float2> {
    static constexpr int kFlops = 4;
    __device__ __forceinline__ static float2 op(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
    __device__ __forceinline__ static float2 init(int i) { return make_float2(1.0f + 1e-7f * (float)i, 1.0f - 1e-7f * (float)i); }
    __device__ __forceinline__ static double sum(float2 a) { return (double)a.x + (double)a.y; }
};

template <>
struct Fma<double> {
    static constexpr int kFlops = 2;
    __device__ __forceinline__ static double op(double a, double b, double c) { return __fma_rn(a, b, c); }
    __device__ __forceinline__ static double init(int i) { return 1.0 + 1e-15 * (double)i; }
    __device__ __forceinline__ static double sum(double a) { return a; }
};

// b and c come from the caller so that no chain can be folded at compile time;
// with b slightly below one the chains stay finite for any round count.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T b, T c, int rounds, double* sink,
                                                         unsigned long long* clk)
{
    const uint64_t t0 = global_ns();
    const long long c0 = clock64();
    T a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = Fma<T>::init(i + threadIdx.x);
    for (int r = 0; r < rounds; ++r) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = Fma<T>::op(a[i], b, c);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += Fma<T>::sum(a[i]);
    // never true for the values used; keeps the chains live
    if (s == -1.0) sink[blockIdx.x] = s;
    if (threadIdx.x == 0) {
        const long long c1 = clock64();
        const uint64_t t1 = global_ns();
        atomicAdd(&clk[0], (unsigned long long)(c1 - c0));
        atomicAdd(&clk[1], (unsigned long long)(t1 - t0));
    }
}

template <typename T>
int run(T b, T c, int device, double* tflops, double* ms_out, double* sm_mhz)
{
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return (int)e;
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains<T>, kThreads, 0);
    if (per_sm < 1) per_sm = 1;
    const int blocks = nsm * per_sm;
    double* sink = nullptr;
    unsigned long long* clk = nullptr;
    if ((e = cudaMalloc(&sink, sizeof(double) * blocks)) != cudaSuccess) return (int)e;
    if ((e = cudaMalloc(&clk, 2 * sizeof(unsigned long long))) != cudaSuccess) {
        cudaFree(sink);
        return (int)e;
    }
    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    // size the run to about 200 ms from a short calibration launch
    int rounds = 256;
    float ms = 0.0f;
    for (int attempt = 0; attempt < 4; ++attempt) {
        cudaMemset(clk, 0, 2 * sizeof(unsigned long long));
        cudaEventRecord(ev0);
        k_fma_chains<T><<<blocks, kThreads>>>(b, c, rounds, sink, clk);
        cudaEventRecord(ev1);
        cudaEventSynchronize(ev1);
        cudaEventElapsedTime(&ms, ev0, ev1);
        if (ms > 100.0f || attempt == 3) break;
        const double scale = 200.0 / (ms > 0.01f ? ms : 0.01f);
        const double next = rounds * (scale > 64.0 ? 64.0 : scale);
        rounds = next > 1e7 ? 10000000 : (int)next;
    }
    // best of three timed launches at that size
    double best = 1e30;
    unsigned long long hclk[2] = {0, 0};
    for (int rep = 0; rep < 3; ++rep) {
        cudaMemset(clk, 0, 2 * sizeof(unsigned long long));
        cudaEventRecord(ev0);
        k_fma_chains<T><<<blocks, kThreads>>>(b, c, rounds, sink, clk);
        cudaEventRecord(ev1);
        cudaEventSynchronize(ev1);
        cudaEventElapsedTime(&ms, ev0, ev1);
        if (ms < best) {
            best = ms;
            cudaMemcpy(hclk, clk, sizeof(hclk), cudaMemcpyDeviceToHost);
        }
    }
    e = cudaGetLastError();
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    cudaFree(sink);
    cudaFree(clk);
    if (e != cudaSuccess) return (int)e;
    const double flops = (double)blocks * kThreads * (double)rounds * 8.0 * kChains * Fma<T>::kFlops;
    *tflops = flops / (best * 1e-3) / 1e12;
    *ms_out = best;
    *sm_mhz = hclk[1] > 0 ? (double)hclk[0] / (double)hclk[1] * 1e3 : 0.0;
    return 0;
}

}  // namespace

extern "C" {

// kind 0: FP32 fma, 1: paired FP32 fma (two floats per instruction), 2: FP64 fma.
// Returns 0 or a cudaError_t code; tflops: achieved rate; ms: the timed
// launch; sm_mhz: the SM clock during it (clock counter over the ns timer,
// averaged over blocks).
int ffp_simt_peak(int kind, int device, double* tflops, double* ms, double* sm_mhz)
{
    if (!tflops || !ms || !sm_mhz) return -1;
    switch (kind) {
        case 0: return run<float>(0.9999999f, 1e-7f, device, tflops, ms, sm_mhz);
        case 1: return run<float2>(make_float2(0.9999999f, 0.9999998f), make_float2(1e-7f, 2e-7f),
                                   device, tflops, ms, sm_mhz);
        case 2: return run<double>(0.999999999999, 1e-15, device, tflops, ms, sm_mhz);
        default: return -1;
    }
}

}  // extern "C"
