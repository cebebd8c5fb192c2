// render.cu -- MFA-VV ray casting (Sec. IV-A.4): one ray per pixel, a value+gradient MFA
// query per sample, 1-D transfer function and Phong shading (Sec. IV-B), front-to-back
// over compositing with early ray termination, one 16-byte store per pixel.
//
// Launch shape: one CTA of 128 threads per 16x8 pixel tile; each warp covers an 8x4
// sub-tile so that its 32 rays are close together and their samples share knot spans
// and control-point rows (broadcast loads in L1).  The hardware block scheduler hands
// tiles to SMs as earlier ones finish, which balances the uneven ray lengths that early
// termination creates.  The transfer-function table travels in the kernel parameters
// and is copied into shared memory once per CTA.
#include "bspline.cuh"

namespace mfa {
namespace {

constexpr int kTileW = 16, kTileH = 8, kThreads = kTileW * kTileH;

template <int Q, int STORAGE>
__global__ void __launch_bounds__(kThreads) k_render(ModelDev M, const __grid_constant__ RenderParams P)
{
    __shared__ float4 tf[kTfMax];
    for (int i = threadIdx.x; i < P.tf_n; i += kThreads) tf[i] = P.tf[i];
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int col = blockIdx.x * kTileW + (warp & 1) * 8 + (lane & 7);
    const int row = blockIdx.y * kTileH + (warp >> 1) * 4 + (lane >> 3);
    unsigned long long count = 0;

    if (col < P.width && row < P.height) {
        // ---- ray through the pixel centre (row 0 at the top)
        const float sx = fmaf(static_cast<float>(2 * col + 1), P.inv_w, -1.0f);
        const float sy = fmaf(static_cast<float>(-(2 * row + 1)), P.inv_h, 1.0f);
        float o[3], d[3];
        if (P.projection == 0) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                o[a] = fmaf(sy, P.uy[a], fmaf(sx, P.rx[a], P.eye[a]));
                d[a] = P.fwd[a];
            }
        } else {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                o[a] = P.eye[a];
                d[a] = fmaf(sy, P.uy[a], fmaf(sx, P.rx[a], P.fwd[a]));
            }
            const float inv = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            d[0] *= inv;
            d[1] *= inv;
            d[2] *= inv;
        }
        // ---- slab clip against [0,1]^3, t >= 0
        float t0 = 0.0f, t1 = INFINITY;
        bool hit = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (d[a] != 0.0f) {
                const float inv = 1.0f / d[a];
                float ta = -o[a] * inv, tb = (1.0f - o[a]) * inv;
                if (ta > tb) { const float t = ta; ta = tb; tb = t; }
                t0 = fmaxf(t0, ta);
                t1 = fminf(t1, tb);
            } else if (o[a] < 0.0f || o[a] > 1.0f) {
                hit = false;
            }
        }
        float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);   // premultiplied rgb, alpha
        if (hit && t0 < t1) {
            const float dt = (t1 - t0) / static_cast<float>(P.n_samples);
            const float tscale = static_cast<float>(P.tf_n - 1);
            const float lx = -d[0], ly = -d[1], lz = -d[2];     // headlight: L = V = -d
            int sx_ = -1, sy_ = -1, sz_ = -1;
            for (int k = 0; k < P.n_samples; ++k) {
                const float t = fmaf(static_cast<float>(k) + 0.5f, dt, t0);
                const float u = clamp01(fmaf(t, d[0], o[0]));
                const float v = clamp01(fmaf(t, d[1], o[1]));
                const float w = clamp01(fmaf(t, d[2], o[2]));
                sx_ = (k == 0) ? locate_span(M.ax[0], u) : walk_span(M.ax[0], u, sx_);
                sy_ = (k == 0) ? locate_span(M.ax[1], v) : walk_span(M.ax[1], v, sy_);
                sz_ = (k == 0) ? locate_span(M.ax[2], w) : walk_span(M.ax[2], w, sz_);
                const float4 q = query<Q, STORAGE>(M, u, v, w, sx_, sy_, sz_);
                ++count;
                // ---- transfer function: linear interpolation between table rows
                float tt = clamp01((q.x - P.vmin) * P.inv_range);
                float4 c;
                if (P.tf_n > 1) {
                    const float xx = tt * tscale;
                    const int i0 = min(static_cast<int>(xx), P.tf_n - 2);
                    const float wt = xx - static_cast<float>(i0);
                    const float4 c0 = tf[i0], c1 = tf[i0 + 1];
                    c.x = fmaf(wt, c1.x - c0.x, c0.x);
                    c.y = fmaf(wt, c1.y - c0.y, c0.y);
                    c.z = fmaf(wt, c1.z - c0.z, c0.z);
                    c.w = fmaf(wt, c1.w - c0.w, c0.w);
                } else {
                    c = tf[0];
                }
                // ---- Phong with a headlight, two-sided
                if (P.shading) {
                    const float g2 = q.y * q.y + q.z * q.z + q.w * q.w;
                    float factor, spec = 0.0f;
                    if (g2 <= P.gtiny2) {
                        factor = P.ka + P.kd;
                    } else {
                        const float ndl = fabsf(q.y * lx + q.z * ly + q.w * lz) * rsqrtf(g2);
                        const float rv = 2.0f * ndl * ndl - 1.0f;     // R.V with V = L
                        spec = rv > 0.0f ? __powf(rv, P.shininess) : 0.0f;
                        factor = fmaf(P.kd, ndl, P.ka);
                    }
                    c.x = clamp01(fmaf(c.x, factor, P.ks * spec));
                    c.y = clamp01(fmaf(c.y, factor, P.ks * spec));
                    c.z = clamp01(fmaf(c.z, factor, P.ks * spec));
                }
                // ---- front-to-back over
                const float wgt = (1.0f - acc.w) * c.w;
                acc.x = fmaf(wgt, c.x, acc.x);
                acc.y = fmaf(wgt, c.y, acc.y);
                acc.z = fmaf(wgt, c.z, acc.z);
                acc.w += wgt;
                if (acc.w >= P.ert_alpha) break;
            }
        }
        P.out[static_cast<long long>(row) * P.width + col] = acc;
    }

    if (P.samples_out) {
        unsigned long long c = count;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
        if (lane == 0 && c) atomicAdd(P.samples_out, c);
    }
}

template <int Q>
cudaError_t render_q(const ModelDev& m, const RenderParams& rp, cudaStream_t st)
{
    dim3 grid((rp.width + kTileW - 1) / kTileW, (rp.height + kTileH - 1) / kTileH);
    switch (m.storage) {
    case 1: k_render<Q, 1><<<grid, kThreads, 0, st>>>(m, rp); break;
    case 2: k_render<Q, 2><<<grid, kThreads, 0, st>>>(m, rp); break;
    case 3: k_render<Q, 3><<<grid, kThreads, 0, st>>>(m, rp); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_render(const ModelDev& m, const RenderParams& rp, cudaStream_t stream)
{
    switch (m.q) {
    case 2: return render_q<2>(m, rp, stream);
    case 3: return render_q<3>(m, rp, stream);
    case 4: return render_q<4>(m, rp, stream);
    case 5: return render_q<5>(m, rp, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace mfa
