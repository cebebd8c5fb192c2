// query.cu -- value+gradient queries at arbitrary points (decode; Sec. III-B, the query of
// Fig. 8 in Sec. V-D.3) and the knot-span search on its own.
//
// One thread per point, grid-stride.  Per point: clamp to [0,1], locate the three spans,
// evaluate the span-local basis and derivatives, contract the (p+1)^3 support.  Models with
// uniform knots and one degree take the cardinal path (span from floor((n-p) u) checked
// against the knots, interior spans without records).  Points are read as three scalar FP32 loads (12 B, coalesced
// across the warp), values and gradients written as scalar stores; for random points the
// control-point gathers hit L2 (the window array of a 128^3 FP32 model is 32 MiB).
#include "bspline.cuh"

namespace mfa {
namespace {

// CARD: the model is on the cardinal path (uniform knots, degree Q-1 on every axis), so the
// span comes from floor((n - p) u) with one exact check against the knots (cardinal_span)
// and interior spans need no record.  Random points make the kernel
// wait on L2 gathers, so occupancy matters more than registers: 4 blocks of 256 per SM
// (64 registers) measure 9 % faster than the 3 that 76 registers allow (0.566 against
// 0.622 ms for 2^24 points on the 128^3 degree-3 FP32 model); degree 4 keeps 3 (64
// registers would spill).  GRAD false (no gradient output) leaves the derivative weights
// and sums unused, so the compiler drops them: a value-only query.
template <int Q, int STORAGE, bool CARD, bool GRAD>
__global__ void __launch_bounds__(256, Q <= 4 ? 4 : 3)
    k_decode(ModelDev M, const float* __restrict__ pts, long long n, float* __restrict__ val, float* __restrict__ grad)
{
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        // points and results stream through once: evict-first loads and stores keep them from
        // pushing the window array out of L2
        const float u = clamp01(__ldcs(pts + 3 * i + 0));
        const float v = clamp01(__ldcs(pts + 3 * i + 1));
        const float w = clamp01(__ldcs(pts + 3 * i + 2));
        float4 r;
        if constexpr (CARD) {
            r = query_cardinal<Q, STORAGE>(M, u, v, w);
        } else {
            const int sx = locate_span(M.ax[0], u);
            const int sy = locate_span(M.ax[1], v);
            const int sz = locate_span(M.ax[2], w);
            r = query2<Q, STORAGE>(M, u, v, w, sx, sy, sz);
        }
        __stcs(val + i, r.x);
        if (GRAD && grad) {
            __stcs(grad + 3 * i + 0, r.y);
            __stcs(grad + 3 * i + 1, r.z);
            __stcs(grad + 3 * i + 2, r.w);
        }
    }
}

// The knot spans k_decode<..., CARD, ...> takes for each point: cardinal_span on the
// cardinal path (the same call query_cardinal makes), locate_span otherwise.
template <bool CARD>
__global__ void __launch_bounds__(256) k_spans(ModelDev M, const float* __restrict__ pts, long long n,
                                               int* __restrict__ spans)
{
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float u = clamp01(__ldg(pts + 3 * i + a));
            if constexpr (CARD)
                spans[3 * i + a] = cardinal_span(M.ax[a], u, cardinal_coord(M.ax[a], u)) + M.ax[a].p;
            else
                spans[3 * i + a] = locate_span(M.ax[a], u);
        }
    }
}

int grid_for(long long n, int threads)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (n + threads - 1) / threads;
    const long long cap = static_cast<long long>(sms) * 32;   // enough resident blocks to fill every SM
    return static_cast<int>(want < cap ? (want > 0 ? want : 1) : cap);
}

template <int Q, bool CARD, bool GRAD>
cudaError_t decode_qcg(const ModelDev& m, const float* pts, long long n, float* val, float* grad, cudaStream_t st)
{
    const int blocks = grid_for(n, 256);
    switch (m.storage) {
    case 1: k_decode<Q, 1, CARD, GRAD><<<blocks, 256, 0, st>>>(m, pts, n, val, grad); break;
    case 2: k_decode<Q, 2, CARD, GRAD><<<blocks, 256, 0, st>>>(m, pts, n, val, grad); break;
    case 3: k_decode<Q, 3, CARD, GRAD><<<blocks, 256, 0, st>>>(m, pts, n, val, grad); break;
    case 4: k_decode<Q, 4, CARD, GRAD><<<blocks, 256, 0, st>>>(m, pts, n, val, grad); break;
    case 5: k_decode<Q, 5, CARD, GRAD><<<blocks, 256, 0, st>>>(m, pts, n, val, grad); break;
    case 6: k_decode<Q, 6, CARD, GRAD><<<blocks, 256, 0, st>>>(m, pts, n, val, grad); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int Q, bool CARD>
cudaError_t decode_qc(const ModelDev& m, const float* pts, long long n, float* val, float* grad, cudaStream_t st)
{
    return grad ? decode_qcg<Q, CARD, true>(m, pts, n, val, grad, st)
                : decode_qcg<Q, CARD, false>(m, pts, n, val, grad, st);
}

template <int Q>
cudaError_t decode_q(const ModelDev& m, const float* pts, long long n, float* val, float* grad, cudaStream_t st)
{
    return m.cardinal ? decode_qc<Q, true>(m, pts, n, val, grad, st) : decode_qc<Q, false>(m, pts, n, val, grad, st);
}

}  // namespace

cudaError_t launch_decode(const ModelDev& m, const float* pts, long long n, float* val, float* grad,
                          cudaStream_t stream)
{
    if (n <= 0) return cudaSuccess;
    switch (m.q) {
    case 2: return decode_q<2>(m, pts, n, val, grad, stream);
    case 3: return decode_q<3>(m, pts, n, val, grad, stream);
    case 4: return decode_q<4>(m, pts, n, val, grad, stream);
    case 5: return decode_q<5>(m, pts, n, val, grad, stream);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_spans(const ModelDev& m, const float* pts, long long n, int* spans, cudaStream_t stream)
{
    if (n <= 0) return cudaSuccess;
    if (m.cardinal)
        k_spans<true><<<grid_for(n, 256), 256, 0, stream>>>(m, pts, n, spans);
    else
        k_spans<false><<<grid_for(n, 256), 256, 0, stream>>>(m, pts, n, spans);
    return cudaGetLastError();
}

}  // namespace mfa
