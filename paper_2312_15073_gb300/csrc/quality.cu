// quality.cu -- the ground truth and the scores of the render-quality comparison
// (Sec. V-D.3, Table II): a direct render of the closed-form Marschner-Lobb signal
// (Sec. V-A.1, Eq. 1) through the same rays, samples, transfer function, shading and
// compositing as the MFA render (mfa_render_ml), and MSE / PSNR / SSIM between two
// rendered images (mfa_image_compare).
//
// Signal: F(x, y, z) = (1 - sin(pi z / 2) + alpha (1 + rho(r))) / (2 (1 + alpha)),
// rho(r) = cos(2 pi f_M cos(pi r / 2)), r = sqrt(x^2 + y^2), on [-1, 1]^3, which the unit
// box maps onto by x = 2u - 1; the gradient with respect to (u, v, w) is twice the one with
// respect to (x, y, z), with rho'(r) x / r continued to the axis by sin(pi r / 2) / r ->
// pi / 2.  FP32 with sincospif (the arguments in units of pi, so no large-argument
// reduction), one thread per pixel.
//
// Metrics (the images are premultiplied RGBA over black): R, G, B clamped to [0, 1] and
// scaled by 255, alpha ignored; MSE over pixels and the three channels, PSNR =
// 10 log10(255^2 / MSE); SSIM with the standard constants of Wang et al. (IEEE TIP 2004):
// an 11 x 11 Gaussian window (sigma 1.5, weights summing to 1), C1 = (0.01 * 255)^2,
// C2 = (0.03 * 255)^2, averaged over the window positions inside the image and the three
// channels.  Window sums and all reductions in FP64, in a fixed order (per-block partial
// sums, then one block adds them), so a result does not depend on timing.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "raycast.cuh"

namespace mfa {
namespace {

constexpr int kMlThreads = 128;
constexpr float kPi = 3.14159265358979323846f;

// {F, dF/du, dF/dv, dF/dw} of the signal at the unit-box point (u, v, w)
__device__ __forceinline__ float4 ml_query(float fm, float alpha, float inv_den, float u, float v, float w)
{
    const float x = fmaf(2.0f, u, -1.0f), y = fmaf(2.0f, v, -1.0f), z = fmaf(2.0f, w, -1.0f);
    const float r = sqrtf(fmaf(x, x, y * y));
    float s_r, c_r, s_rho, c_rho, s_z, c_z;
    sincospif(0.5f * r, &s_r, &c_r);              // sin, cos (pi r / 2)
    sincospif(2.0f * fm * c_r, &s_rho, &c_rho);   // sin, cos (2 pi f_M cos(pi r / 2)); c_rho = rho
    sincospif(0.5f * z, &s_z, &c_z);              // sin, cos (pi z / 2)
    const float sinc = r > 0.0f ? s_r / r : 0.5f * kPi;
    const float g_r = 2.0f * alpha * (kPi * kPi) * fm * s_rho * sinc * inv_den;   // 2 alpha rho'(r) / r / den
    return make_float4((1.0f - s_z + alpha * (1.0f + c_rho)) * inv_den, g_r * x, g_r * y, -kPi * c_z * inv_den);
}

__global__ void __launch_bounds__(kMlThreads) k_render_ml(const __grid_constant__ RenderParams P, float fm,
                                                          float alpha, int shape)
{
    __shared__ float4 tf[kTfSmem];
    stage_tf(tf, P.tf, P.s.tf_n);
    __syncthreads();

    int col, row;
    tile_pixel(tile_shape(shape), blockIdx.x, blockIdx.y, threadIdx.x, col, row);
    unsigned long long count = 0;
    if (col < P.s.width && row < P.s.height) {
        float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        float o[3], d[3], t0, t1;
        if (ray_box(P.s, col, row, o, d, t0, t1)) {
            const int ns = P.s.n_samples;
            const float dt = (t1 - t0) / static_cast<float>(ns);
            const float inv_den = 1.0f / (2.0f * (1.0f + alpha));
            const ShadeParams S = shade_params(P.s, d);
            int k = 0;
            while (k < ns) {
                const float t = fmaf(static_cast<float>(k) + 0.5f, dt, t0);
                const float4 q = ml_query(fm, alpha, inv_den, fmaf(t, d[0], o[0]), fmaf(t, d[1], o[1]),
                                          fmaf(t, d[2], o[2]));
                const float4 c = sample_colour(tf, S, q);
                const float wgt = (1.0f - acc.w) * c.w;
                acc.x = fmaf(wgt, c.x, acc.x);
                acc.y = fmaf(wgt, c.y, acc.y);
                acc.z = fmaf(wgt, c.z, acc.z);
                acc.w += wgt;
                ++k;
                if (acc.w >= P.s.ert_alpha) break;
            }
            count = static_cast<unsigned>(k);
        }
        P.s.out[static_cast<long long>(row) * P.s.width + col] = acc;
    }
    if (P.s.samples_out) add_count(P.s.samples_out, count);
}

// ---------------------------------------------------------------------------------------
// image metrics
// ---------------------------------------------------------------------------------------

constexpr int kWin = 11;                  // SSIM window side
constexpr int kHalo = kWin - 1;
constexpr int kTile = 16;                 // SSIM positions per block side
constexpr int kTileIn = kTile + kHalo;    // input pixels per block side
constexpr int kRedThreads = 256;
constexpr int kMaxPartials = 2048;

struct SsimWeights {
    double w[kWin * kWin];
};

__device__ __forceinline__ double display(float x) { return 255.0 * static_cast<double>(clamp01(x)); }

// block-wide sum of one double per thread (fixed order); the result is valid in thread 0
template <int THREADS>
__device__ __forceinline__ double block_sum(double v, double* sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < THREADS / 32; ++i) s += sh[i];
    __syncthreads();
    return s;
}

// partial[b] = sum over the pixels of block b's grid-stride share of the squared RGB errors
__global__ void __launch_bounds__(kRedThreads) k_sq_err(const float4* __restrict__ a, const float4* __restrict__ b,
                                                        long long n, double* __restrict__ partial)
{
    __shared__ double sh[kRedThreads / 32];
    double s = 0.0;
    for (long long i = blockIdx.x * static_cast<long long>(kRedThreads) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * kRedThreads) {
        const float4 x = a[i], y = b[i];
        const double dr = display(x.x) - display(y.x), dg = display(x.y) - display(y.y),
                     db = display(x.z) - display(y.z);
        s += dr * dr + dg * dg + db * db;
    }
    s = block_sum<kRedThreads>(s, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// partial[b] = sum of SSIM over the three channels at the window positions of block b's
// tiles (tile t covers positions [16 tx, 16 tx + 16) x [16 ty, 16 ty + 16) of the
// (W - 10) x (H - 10) positions; blocks take tiles in a grid-stride loop).
__global__ void __launch_bounds__(kTile * kTile) k_ssim(const float4* __restrict__ a, const float4* __restrict__ b,
                                                       int W, int H, const __grid_constant__ SsimWeights K,
                                                       double* __restrict__ partial)
{
    __shared__ double xa[3][kTileIn][kTileIn];
    __shared__ double xb[3][kTileIn][kTileIn];
    __shared__ double sh[kTile * kTile / 32];
    const int PW = W - kHalo, PH = H - kHalo;               // window positions per row / column
    const int tiles_x = (PW + kTile - 1) / kTile, tiles = tiles_x * ((PH + kTile - 1) / kTile);
    const double C1 = (0.01 * 255.0) * (0.01 * 255.0), C2 = (0.03 * 255.0) * (0.03 * 255.0);
    const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
    double s = 0.0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int x0 = (t % tiles_x) * kTile, y0 = (t / tiles_x) * kTile;
        __syncthreads();   // the previous tile's reads are done
        for (int e = threadIdx.x; e < kTileIn * kTileIn; e += kTile * kTile) {
            const int ex = e % kTileIn, ey = e / kTileIn;
            const int gx = min(x0 + ex, W - 1), gy = min(y0 + ey, H - 1);   // clamped rows feed no counted position
            const long long g = static_cast<long long>(gy) * W + gx;
            const float4 pa = a[g], pb = b[g];
            xa[0][ey][ex] = display(pa.x);
            xa[1][ey][ex] = display(pa.y);
            xa[2][ey][ex] = display(pa.z);
            xb[0][ey][ex] = display(pb.x);
            xb[1][ey][ex] = display(pb.y);
            xb[2][ey][ex] = display(pb.z);
        }
        __syncthreads();
        if (x0 + tx < PW && y0 + ty < PH) {
#pragma unroll 1
            for (int c = 0; c < 3; ++c) {
                double ma = 0.0, mb = 0.0, saa = 0.0, sbb = 0.0, sab = 0.0;
                for (int dy = 0; dy < kWin; ++dy) {
#pragma unroll
                    for (int dx = 0; dx < kWin; ++dx) {
                        const double w = K.w[dy * kWin + dx];
                        const double va = xa[c][ty + dy][tx + dx], vb = xb[c][ty + dy][tx + dx];
                        ma = fma(w, va, ma);
                        mb = fma(w, vb, mb);
                        saa = fma(w, va * va, saa);
                        sbb = fma(w, vb * vb, sbb);
                        sab = fma(w, va * vb, sab);
                    }
                }
                const double va = saa - ma * ma, vb = sbb - mb * mb, cov = sab - ma * mb;
                s += ((2.0 * ma * mb + C1) * (2.0 * cov + C2)) / ((ma * ma + mb * mb + C1) * (va + vb + C2));
            }
        }
    }
    s = block_sum<kTile * kTile>(s, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// out[0] = sum of partial[0..n) in a fixed order
__global__ void __launch_bounds__(kRedThreads) k_sum_partials(const double* __restrict__ partial, int n,
                                                              double* __restrict__ out)
{
    __shared__ double sh[kRedThreads / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += kRedThreads) s += partial[i];
    s = block_sum<kRedThreads>(s, sh);
    if (threadIdx.x == 0) out[0] = s;
}

int sm_count()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

}  // namespace
}  // namespace mfa

#include "host.cuh"

using namespace mfa;

extern "C" int mfa_render_ml(const mfa_ml_signal* sig, const mfa_camera* cam, const mfa_transfer_fn* tf, int width,
                             int height, int n_samples, float* rgba_out, const mfa_render_opts* opts)
{
    if (!sig) return fail(MFA_ERR_ARG, "signal must be non-NULL");
    if (!(sig->f_m >= 0.0 && sig->f_m <= 1e6) || !(sig->alpha >= 0.0 && sig->alpha <= 1e6))
        return fail(MFA_ERR_ARG, "f_m and alpha must be finite and >= 0");
    const int shape = opts ? opts->tile_shape : 0;
    if (shape < 0 || shape >= kTileShapes) return fail(MFA_ERR_ARG, "tile_shape %d outside 0..%d", shape, kTileShapes - 1);
    RenderParams P;
    if (int rc = setup_view(cam, tf, width, height, n_samples, rgba_out, opts ? opts->samples_out : nullptr, 0.0f, 1.0f,
                            1e-6, P.s, P.tf))
        return rc;
    const TileShape T = tile_shape(shape);
    dim3 grid((width + T.tw - 1) / T.tw, (height + T.th - 1) / T.th);
    k_render_ml<<<grid, kMlThreads, 0, current_stream()>>>(P, static_cast<float>(sig->f_m),
                                                            static_cast<float>(sig->alpha), shape);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MFA_OK : cuda_fail(e, "Marschner-Lobb render launch");
}

extern "C" int mfa_image_compare(const float* rgba_test, const float* rgba_ref, int width, int height,
                                 mfa_image_quality* out)
{
    if (!rgba_test || !rgba_ref || !out) return fail(MFA_ERR_ARG, "images and out must be non-NULL");
    if ((reinterpret_cast<uintptr_t>(rgba_test) | reinterpret_cast<uintptr_t>(rgba_ref)) & 15)
        return fail(MFA_ERR_ARG, "images must be 16-byte aligned");
    if (width < kWin || height < kWin || width > 32768 || height > 32768)
        return fail(MFA_ERR_ARG, "image size %dx%d outside %d..32768", width, height, kWin);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t pool;
    cudaError_t e = staging_pool(dev, &pool);
    if (e != cudaSuccess) return cuda_fail(e, "staging pool");
    cudaStream_t st = current_stream();

    const long long n = static_cast<long long>(width) * height;
    const int sms = sm_count();
    const int b_err = static_cast<int>(std::min<long long>((n + kRedThreads - 1) / kRedThreads, std::min(8 * sms, kMaxPartials)));
    const int PW = width - kHalo, PH = height - kHalo;
    const long long tiles = static_cast<long long>((PW + kTile - 1) / kTile) * ((PH + kTile - 1) / kTile);
    const int b_ssim = static_cast<int>(std::min<long long>(tiles, std::min(4 * sms, kMaxPartials)));

    double* d = nullptr;   // partials (err | ssim) | 2 sums
    e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&d), sizeof(double) * (b_err + b_ssim + 2), pool, st);
    if (e != cudaSuccess) return cuda_fail(e, "staging memory");
    SsimWeights K;
    {
        double sum = 0.0;
        for (int i = 0; i < kWin * kWin; ++i) {
            const double ky = i / kWin - (kWin - 1) / 2, kx = i % kWin - (kWin - 1) / 2;
            K.w[i] = std::exp(-(kx * kx + ky * ky) / (2.0 * 1.5 * 1.5));
            sum += K.w[i];
        }
        for (double& w : K.w) w /= sum;
    }
    const float4* A = reinterpret_cast<const float4*>(rgba_test);
    const float4* B = reinterpret_cast<const float4*>(rgba_ref);
    k_sq_err<<<b_err, kRedThreads, 0, st>>>(A, B, n, d);
    k_ssim<<<b_ssim, kTile * kTile, 0, st>>>(A, B, width, height, K, d + b_err);
    k_sum_partials<<<1, kRedThreads, 0, st>>>(d, b_err, d + b_err + b_ssim);
    k_sum_partials<<<1, kRedThreads, 0, st>>>(d + b_err, b_ssim, d + b_err + b_ssim + 1);
    e = cudaGetLastError();
    double sums[2] = { 0.0, 0.0 };
    if (e == cudaSuccess) e = cudaMemcpyAsync(sums, d + b_err + b_ssim, sizeof sums, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(d, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "image metrics");
    out->mse = sums[0] / (3.0 * static_cast<double>(n));
    out->psnr_db = out->mse > 0.0 ? 10.0 * std::log10(255.0 * 255.0 / out->mse) : INFINITY;
    out->ssim = sums[1] / (3.0 * static_cast<double>(PW) * PH);
    return MFA_OK;
}
