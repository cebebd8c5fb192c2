// peaks.cu -- calibration kernels for the roofline denominators (mfa_measure_peaks): the
// FP32 FMA rate of the whole chip in scalar and packed FP32x2 form, and the rate at which
// the L2 serves random 32-byte gathers (the access pattern of a decode of random points).
// They are measurement infrastructure for the renderer and decoder, not part of the method.
//
// FMA kernels: every thread runs kChains independent FMA chains (enough to cover the FMA
// latency with a full SM of warps), grid = 8 CTAs of 256 threads per SM.  Gather kernel:
// each thread reads kGatherIters 32-byte entries at hashed positions of a buffer that fits
// in L2 (so DRAM is not involved after the first touch) and folds them into one value it
// stores, so no load can be dropped.  Each is timed with CUDA events around one launch
// after a warm-up launch, on the calling thread's bound stream.
#include <cstdint>

#include "bspline.cuh"
#include "host.cuh"

using namespace mfa;

namespace {

constexpr int kThreadsPerCta = 256;
constexpr int kCtasPerSm = 8;
constexpr int kChains = 8;
constexpr int kFmaIters = 16384;
constexpr int kGatherIters = 256;
constexpr size_t kGatherBytes = 32u << 20;   // 32 MiB: resident in the 129 MB L2

__global__ void __launch_bounds__(kThreadsPerCta) k_fma_peak(float* out, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = static_cast<float>(threadIdx.x + c);
    for (int i = 0; i < kFmaIters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678f) out[blockIdx.x] = s;   // keeps the chains live; practically never true
}

__global__ void __launch_bounds__(kThreadsPerCta) k_fma2_peak(float* out, float a, float b)
{
    f2 x[kChains / 2];
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) x[c] = pk2(static_cast<float>(threadIdx.x + c), static_cast<float>(c));
    const f2 a2 = pk2(a, a), b2 = pk2(b, b);
    for (int i = 0; i < kFmaIters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains / 2; ++c) x[c] = fma2(x[c], a2, b2);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) s += hsum2(x[c]);
    if (s == 12345.678f) out[blockIdx.x] = s;
}

__device__ __forceinline__ uint32_t hash32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// n_entries is a power of two; entry e is the 32 bytes at buf + 32 e.
__global__ void __launch_bounds__(kThreadsPerCta) k_l2_gather_peak(const float* __restrict__ buf, uint32_t mask,
                                                                   unsigned long long* out)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long acc = 0;
    for (int i = 0; i < kGatherIters; ++i) {
        const uint32_t e = hash32(tid * kGatherIters + i) & mask;
        unsigned long long v0, v1, v2, v3;
        asm volatile("ld.global.nc.v4.b64 {%0, %1, %2, %3}, [%4];"
                     : "=l"(v0), "=l"(v1), "=l"(v2), "=l"(v3)
                     : "l"(buf + 8ull * e));
        acc ^= v0 ^ v1 ^ v2 ^ v3;
    }
    out[tid] = acc;
}

}  // namespace

extern "C" int mfa_measure_peaks(mfa_peaks* out)
{
    if (!out) return fail(MFA_ERR_ARG, "out is NULL");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
    cudaStream_t st = current_stream();
    const int ctas = sms * kCtasPerSm;
    const uint32_t entries = static_cast<uint32_t>(kGatherBytes / 32);
    const long long gather_threads = static_cast<long long>(ctas) * kThreadsPerCta;

    float* scratch = nullptr;               // FMA sink (never written in practice)
    float* buf = nullptr;                   // gather source
    unsigned long long* sink = nullptr;     // one value per gather thread
    cudaEvent_t a = nullptr, b = nullptr;
    float ms[3] = { 0, 0, 0 };
    e = cudaMalloc(&scratch, sizeof(float) * ctas);
    if (e == cudaSuccess) e = cudaMalloc(&buf, kGatherBytes);
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(unsigned long long) * gather_threads);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0x3c, kGatherBytes, st);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // warm-up, then the timed launch
            if (rep == 1) e = cudaEventRecord(a, st);
            if (k == 0) k_fma_peak<<<ctas, kThreadsPerCta, 0, st>>>(scratch, 0.999f, 0.001f);
            if (k == 1) k_fma2_peak<<<ctas, kThreadsPerCta, 0, st>>>(scratch, 0.999f, 0.001f);
            if (k == 2) k_l2_gather_peak<<<ctas, kThreadsPerCta, 0, st>>>(buf, entries - 1, sink);
            if (e == cudaSuccess) e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[k], a, b);
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (scratch) cudaFree(scratch);
    if (buf) cudaFree(buf);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) return cuda_fail(e, "peak kernels");
    const double fma_flops = 2.0 * kChains * kFmaIters * static_cast<double>(ctas) * kThreadsPerCta;
    out->fp32_tflops = fma_flops / (ms[0] * 1e-3) / 1e12;
    out->fp32x2_tflops = fma_flops / (ms[1] * 1e-3) / 1e12;
    out->l2_gather_gbs = 32.0 * kGatherIters * static_cast<double>(gather_threads) / (ms[2] * 1e-3) / 1e9;
    out->sm_count = sms;
    out->fma_clock_mhz = out->fp32_tflops * 1e12 / (2.0 * 128.0 * sms) / 1e6;
    return MFA_OK;
}
