// render.cu -- MFA-VV ray casting (Sec. IV-A.4): one ray per pixel, a value+gradient MFA
// query per sample, 1-D transfer function and Phong shading (Sec. IV-B), front-to-back
// over compositing with early ray termination, one 16-byte store per pixel.
//
// Launch shape: one CTA of 128 threads per 16x8 pixel tile; each warp covers an 8x4
// sub-tile so that its 32 rays are close together and their samples share knot spans
// and control-point rows.  The hardware block scheduler hands tiles to SMs as earlier
// ones finish, which balances the uneven ray lengths that early termination creates.
// The transfer-function table travels in the kernel parameters and is copied into
// shared memory once per CTA.
//
// The query is L1-bandwidth bound when every sample reloads its span records (3 x 80 B
// at degree 3) and its support rows (16 x 16 B): L1 returns 128 B per clock per SM to
// the registers.  Along one ray each axis keeps the same knot span for several
// consecutive samples, so each axis's span bounds and record stay in registers and only
// the lanes whose span changed reload it.  With the loads thinned out the kernel is
// bound by FP32 issue (about 285 FFMA of about 450 instructions per sample).
//   variant 2 (default): records cached, scalar arithmetic
//   variant 1:           records cached, packed FP32x2 arithmetic
//   variant 3:           nothing cached, scalar arithmetic
// Packed FP32x2 halves the FMA instructions issued but each one holds the FMA pipe for
// two cycles, and pairing the y-pass adds lane work, so on GB300 it measures 2-6 % slower
// than the scalar form on the 128^3 degree-3 frame (ncu: math-pipe-throttle stalls).
// Variant 3 re-reads every record per sample and is L1 bound.
#include "bspline.cuh"

namespace mfa {
namespace {

constexpr int kTileW = 16, kTileH = 8, kThreads = kTileW * kTileH;
// 4 resident CTAs per SM caps the kernel at 128 registers: the span records of three axes
// stay in registers without spills and 16 warps per SM hide the L1 latency.  Measured on
// the 128^3 degree-3 frame: cap 128 -> 6.33 ms, cap 168 (3 CTAs) -> 7.01 ms, cap 96 (5
// CTAs, spills) -> 10.4 ms.
constexpr int kMinBlocks = 4;

// Per-axis state of a ray: current span and its record (which carries the span's FP32
// bounds [lo, hi) in rec[2], rec[3]: a coordinate u lies in the span iff lo <= u < hi).
template <int Q>
struct AxisCache {
    int s;
    float rec[rec_stride(Q)];
};

// Brings the cache to the span of u.  Along a ray the span moves by at most one step
// between samples in the common case, so the next record is loaded directly and the
// search only runs when u left that span too (or on the first sample).
template <int Q>
__device__ __forceinline__ void axis_update(const AxisDev& A, AxisCache<Q>& C, float u)
{
    if (C.s >= 0 && u >= C.rec[2] && u < C.rec[3]) return;
    int s = C.s < 0 ? locate_span(A, u) : C.s + (u >= C.rec[3] ? 1 : -1);
    load_record<Q>(A, s, C.rec);
    if (u < C.rec[2] || u >= C.rec[3]) {
        s = walk_span(A, u, s);
        load_record<Q>(A, s, C.rec);
    }
    C.s = s;
}

// MODE = variant (see above); MINB = minimum resident CTAs per SM (register cap)
template <int Q, int STORAGE, int MODE, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k_render(ModelDev M, const __grid_constant__ RenderParams P)
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
            AxisCache<Q> cx, cy, cz;
            cx.s = cy.s = cz.s = -1;
            int sx_ = -1, sy_ = -1, sz_ = -1;
            for (int k = 0; k < P.n_samples; ++k) {
                const float t = fmaf(static_cast<float>(k) + 0.5f, dt, t0);
                const float u = clamp01(fmaf(t, d[0], o[0]));
                const float v = clamp01(fmaf(t, d[1], o[1]));
                const float w = clamp01(fmaf(t, d[2], o[2]));
                float4 q;
                if constexpr (MODE == 3) {
                    sx_ = (k == 0) ? locate_span(M.ax[0], u) : walk_span(M.ax[0], u, sx_);
                    sy_ = (k == 0) ? locate_span(M.ax[1], v) : walk_span(M.ax[1], v, sy_);
                    sz_ = (k == 0) ? locate_span(M.ax[2], w) : walk_span(M.ax[2], w, sz_);
                    q = query<Q, STORAGE>(M, u, v, w, sx_, sy_, sz_);
                } else {
                    axis_update<Q>(M.ax[0], cx, u);
                    axis_update<Q>(M.ax[1], cy, v);
                    axis_update<Q>(M.ax[2], cz, w);
                    const int i0 = cx.s - M.ax[0].p, j0 = cy.s - M.ax[1].p, k0 = cz.s - M.ax[2].p;
                    if constexpr (MODE == 1) {
                        q = query2_rec<Q, STORAGE>(M, cx.rec, cy.rec, cz.rec, u, v, w, i0, j0, k0);
                    } else {
                        float Nx[Q], Dx[Q], Ny[Q], Dy[Q], Nz[Q], Dz[Q];
                        record_basis<Q>(cx.rec, u, Nx, Dx);
                        record_basis<Q>(cy.rec, v, Ny, Dy);
                        record_basis<Q>(cz.rec, w, Nz, Dz);
                        q = contract<Q, STORAGE>(M, i0, j0, k0, Nx, Dx, Ny, Dy, Nz, Dz);
                        q.y *= cx.rec[1];
                        q.z *= cy.rec[1];
                        q.w *= cz.rec[1];
                    }
                }
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

template <int Q, int STORAGE>
cudaError_t render_qs(const ModelDev& m, const RenderParams& rp, int variant, cudaStream_t st)
{
    dim3 grid((rp.width + kTileW - 1) / kTileW, (rp.height + kTileH - 1) / kTileH);
    switch (variant) {
    case 0:
    case 2: k_render<Q, STORAGE, 2, kMinBlocks><<<grid, kThreads, 0, st>>>(m, rp); break;
    case 1: k_render<Q, STORAGE, 1, kMinBlocks><<<grid, kThreads, 0, st>>>(m, rp); break;
    default: k_render<Q, STORAGE, 3, kMinBlocks><<<grid, kThreads, 0, st>>>(m, rp); break;
    }
    return cudaGetLastError();
}

template <int Q>
cudaError_t render_q(const ModelDev& m, const RenderParams& rp, int variant, cudaStream_t st)
{
    switch (m.storage) {
    case 1: return render_qs<Q, 1>(m, rp, variant, st);
    case 2: return render_qs<Q, 2>(m, rp, variant, st);
    case 3: return render_qs<Q, 3>(m, rp, variant, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_render(const ModelDev& m, const RenderParams& rp, int variant, cudaStream_t stream)
{
    switch (m.q) {
    case 2: return render_q<2>(m, rp, variant, stream);
    case 3: return render_q<3>(m, rp, variant, stream);
    case 4: return render_q<4>(m, rp, variant, stream);
    case 5: return render_q<5>(m, rp, variant, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace mfa
