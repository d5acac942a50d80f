// grpic_peaks.cu -- measured arithmetic ceilings of the device, the
// denominators of the ALU rooflines of the push kernels.
//
// Each probe launches one full-occupancy grid (8 blocks of 256 threads per
// SM) in which every thread runs 8 independent chains of fused multiply-adds
// x <- x a + b, unrolled 16 times per loop trip, so that the chains' latency
// is hidden and loop bookkeeping is ~2 % of the issued instructions.  The rate
// is the best of five timed launches after one warm-up launch, timed with CUDA
// events on the caller's stream.  The paper has no counterpart: this is
// measurement infrastructure.
#include "grpic_internal.cuh"

namespace grpic {
namespace {

constexpr int PEAK_THREADS = 256, PEAK_BLOCKS_PER_SM = 8, PEAK_CHAINS = 8, PEAK_UNROLL = 16;

template <typename T>
__global__ void __launch_bounds__(PEAK_THREADS) fma_peak_kernel(T a, T b, int trips, T *sink)
{
    T x[PEAK_CHAINS];
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) x[k] = (T)(threadIdx.x + k) * T(1e-3);
    for (int t = 0; t < trips; ++t) {
#pragma unroll
        for (int u = 0; u < PEAK_UNROLL; ++u) {
#pragma unroll
            for (int k = 0; k < PEAK_CHAINS; ++k) x[k] = fma(x[k], a, b);
        }
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) s += x[k];
    if (s == T(-12345.678)) *sink = s;  // never true for the inputs used; keeps the chains live
}

// packed FP32: one instruction performs the FMA on both halves of a float2
__global__ void __launch_bounds__(PEAK_THREADS) ffma2_peak_kernel(float2 a, float2 b, int trips, float *sink)
{
    float2 x[PEAK_CHAINS];
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) x[k] = make_float2(((int)threadIdx.x + k) * 1e-3f, ((int)threadIdx.x - k) * 1e-3f);
    for (int t = 0; t < trips; ++t) {
#pragma unroll
        for (int u = 0; u < PEAK_UNROLL; ++u) {
#pragma unroll
            for (int k = 0; k < PEAK_CHAINS; ++k) x[k] = __ffma2_rn(x[k], a, b);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) s += x[k].x + x[k].y;
    if (s == -12345.678f) *sink = s;
}

}  // namespace
}  // namespace grpic

using namespace grpic;

extern "C" grpic_status grpic_alu_peak(int32_t kind, double out[3], void *stream)
{
    if (!out || kind < 0 || kind > 2) return GRPIC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GRPIC_ECUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
        return GRPIC_ECUDA;
    const int blocks = nsm * PEAK_BLOCKS_PER_SM;
    // trips per launch: ~4e11 FP32 flop, ~1e10 FP64 flop (a few ms each)
    const int trips = kind == 1 ? 80 : 5000;
    const double fma_per_launch = (double)blocks * PEAK_THREADS * PEAK_CHAINS * PEAK_UNROLL * trips;
    const double flop_per_fma = kind == 2 ? 4.0 : 2.0;   // a packed FMA is two FMAs
    double *sink = nullptr;
    if (cudaMalloc(&sink, sizeof(double)) != cudaSuccess) return GRPIC_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 0.0f;
    cudaError_t err = cudaSuccess;
    for (int rep = 0; rep < 6 && err == cudaSuccess; ++rep) {
        cudaEventRecord(e0, s);
        if (kind == 0)
            fma_peak_kernel<float><<<blocks, PEAK_THREADS, 0, s>>>(0.999f, 1e-4f, trips, (float *)sink);
        else if (kind == 1)
            fma_peak_kernel<double><<<blocks, PEAK_THREADS, 0, s>>>(0.999, 1e-4, trips, sink);
        else
            ffma2_peak_kernel<<<blocks, PEAK_THREADS, 0, s>>>(make_float2(0.999f, 0.998f), make_float2(1e-4f, 2e-4f),
                                                               trips, (float *)sink);
        cudaEventRecord(e1, s);
        err = cudaEventSynchronize(e1);
        if (err == cudaSuccess) err = cudaGetLastError();
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.0f || ms < best)) best = ms;  // launch 0 warms up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (err != cudaSuccess || best <= 0.0f) return GRPIC_ECUDA;
    out[0] = fma_per_launch * flop_per_fma / (best * 1e-3);             // flop/s
    out[1] = fma_per_launch / 32.0 / (best * 1e-3);                     // FMA warp-instructions/s
    out[2] = nsm;
    return GRPIC_OK;
}
