// render.cu -- MFA-VV ray casting (Sec. IV-A.4): one ray per pixel, a value+gradient MFA
// query per sample, 1-D transfer function and Phong shading (Sec. IV-B), front-to-back
// over compositing with early ray termination, one 16-byte store per pixel.
//
// Work decomposition: CTAs of 128 threads each render one ray tile; the 32 lanes of a warp
// cover a compact block of pixels (8x4 by default) so that their samples share knot spans
// and control-point rows.  Two launch forms share the per-pixel code:
//   * k_render: one image, one CTA per tile, the hardware block scheduler hands tiles to
//     SMs as earlier ones finish (balancing the uneven ray lengths early termination
//     creates); scalars and the transfer-function table travel as kernel arguments.
//   * k_render_batch: many images of many models in persistent launches, one kernel per
//     (degree class, storage type, cardinal or record path) group.  Each CTA draws tile
//     indices from its group's device counter in the work table until the group is
//     exhausted, and loads the tile's request (model, camera, table) into shared memory
//     when it changes.
//
// Per sample the kernel is bound by FP32 issue and the FMA pipe once the loads are thinned
// out: along one ray each axis keeps the same knot span for several consecutive samples,
// so the per-axis span state stays in registers and only the lanes whose span changed
// reload anything, and the (p+1)^3 contraction runs on packed FP32x2 instructions fed
// directly by the layer-pair window layout (bspline.cuh).  Variants (one contraction):
//   variant 6:  uniform knots and one degree (the cardinal path): interior spans share one
//               basis, computed from t without a record; the state per axis is the span
//               index; software-pipelined like 4
//   variant 4:  span records cached in registers, software-pipelined (the query of sample
//               k+1 interleaves with the colour and compositing of sample k)
//   variant 2:  records cached
//   variant 1:  records cached, the z basis evaluated directly as function pairs
//   variant 3:  nothing cached (records re-read per sample)
//   variant 5:  per-warp control-point bricks in shared memory (below)
// The default (variant 0) is 6 where the cardinal path applies, else 4.  ncu launch times
// on the 128^3 degree-3 FP32 frame (1024^2, 1024 samples, Phong): 6: 4.9 ms, 4: 5.6, 1: 5.7,
// 2: 5.8, 5: 6.9, 3: 7.6.
#include "raycast.cuh"

namespace mfa {
namespace {

constexpr int kThreads = 128;
// 4 resident CTAs per SM caps the kernel at 128 registers: the span records of three axes
// stay in registers without spills and 16 warps per SM hide the L1 latency.  Measured on
// the 128^3 degree-3 frame: cap 128 -> 6.33 ms, cap 168 (3 CTAs) -> 7.01 ms, cap 96 (5
// CTAs, spills) -> 10.4 ms.
constexpr int kMinBlocks = 4;
// Degree class 5 (degree 4) off the cardinal path: the span records of three axes and a
// 5x5x5 support do not fit in 128 registers (variant 4 spilled 720 bytes), so those kernels
// take the register budget of three CTAs per SM.
// The cardinal path at degree class 4 keeps the support of the current cell in registers
// (64 values; see march_cardinal) and takes the budget of three CTAs (160 registers, no
// spills): the window is then read once per cell a ray visits, not once per sample, which
// relieves the L1 data pipe that bounded the kernel.  Measured on the 128^3 degree-3
// 1024^2 frame (bitwise the same image): FP32 4.25 ms without the cache at 4 CTAs, 3.83 ms
// with it at 4 CTAs (128 registers, small spills), 3.61 ms at 3 CTAs; FP16 5.55, 5.07,
// 4.84 ms.  Empty-space skipping (variant 7) visits few cells per ray and keeps no cache
// (SKIP): 4 CTAs.  The patch march (variant 8) takes the cardinal budget too (144
// registers); squeezed to four CTAs (124 registers, no spills) it measured 2.96 against
// 2.93 ms.
template <int Q, bool CARD, bool SKIP = false>
constexpr int min_blocks()
{
    if (CARD && Q == 4 && !SKIP) return 3;
    return Q <= 4 || CARD ? kMinBlocks : 3;
}

// The whole ray of pixel (col, row): premultiplied RGBA; `count` += samples evaluated.
// MODE = variant (see above).
template <int Q, int STORAGE, int MODE>
__device__ __forceinline__ float4 march(const ModelDev& M, const RenderScalars& P, const float4* __restrict__ tf,
                                        int col, int row, unsigned long long& count)
{
    float o[3], d[3], t0, t1;
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);   // premultiplied rgb, alpha
    if (!ray_box(P, col, row, o, d, t0, t1)) return acc;

    const int ns = P.n_samples, tf_n = P.tf_n, shading = P.shading;
    const float vmin = P.vmin, inv_range = P.inv_range, ert = P.ert_alpha, gtiny2 = P.gtiny2;
    const float ka = P.ka, kd = P.kd, ks = P.ks, shin = P.shininess;
    const float dt = (t1 - t0) / static_cast<float>(ns);
    const float tscale = static_cast<float>(tf_n - 1);
    const float lx = -d[0], ly = -d[1], lz = -d[2];     // headlight: L = V = -d
    AxisCache<Q> cx, cy, cz;
    cx.s = cy.s = cz.s = -1;
    int sx_ = -1, sy_ = -1, sz_ = -1;
    for (int k = 0; k < ns; ++k) {
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
                float Ny[Q], Dy[Q], Nz[Q], Dz[Q];
                const XIn<Q, STORAGE> X = xin_record<Q, STORAGE>(cx.rec, u);
                record_basis<Q>(cy.rec, v, Ny, Dy);
                record_basis<Q>(cz.rec, w, Nz, Dz);
                q = contract<Q, STORAGE>(M, i0, j0, k0, X, Ny, Dy, Nz, Dz);
                q.y *= cx.rec[1];
                q.z *= cy.rec[1];
                q.w *= cz.rec[1];
            }
        }
        ++count;
        // ---- transfer function: linear interpolation between table rows
        const float tt = clamp01((q.x - vmin) * inv_range);
        float4 c;
        if (tf_n > 1) {
            const float xx = tt * tscale;
            int i0 = min(static_cast<int>(xx), tf_n - 2);
            MFA_DBG_INDEX(P.dbg, i0, tf_n - 1, kDbgTf);   // row i0 and its difference are read
            const float wt = xx - static_cast<float>(i0);
            const float4 c0 = tf[2 * i0], dc = tf[2 * i0 + 1];   // row and difference (stage_tf)
            c.x = fmaf(wt, dc.x, c0.x);
            c.y = fmaf(wt, dc.y, c0.y);
            c.z = fmaf(wt, dc.z, c0.z);
            c.w = fmaf(wt, dc.w, c0.w);
        } else {
            c = tf[0];
        }
        // ---- Phong with a headlight, two-sided
        if (shading) {
            const float g2 = q.y * q.y + q.z * q.z + q.w * q.w;
            float factor, spec = 0.0f;
            if (g2 <= gtiny2) {
                factor = ka + kd;
            } else {
                const float ndl = fabsf(q.y * lx + q.z * ly + q.w * lz) * rsqrtf(g2);
                const float rv = 2.0f * ndl * ndl - 1.0f;     // R.V with V = L
                spec = rv > 0.0f ? __powf(rv, shin) : 0.0f;
                factor = fmaf(kd, ndl, ka);
            }
            c.x = clamp01(fmaf(c.x, factor, ks * spec));
            c.y = clamp01(fmaf(c.y, factor, ks * spec));
            c.z = clamp01(fmaf(c.z, factor, ks * spec));
        }
        // ---- front-to-back over
        const float wgt = (1.0f - acc.w) * c.w;
        acc.x = fmaf(wgt, c.x, acc.x);
        acc.y = fmaf(wgt, c.y, acc.y);
        acc.z = fmaf(wgt, c.z, acc.z);
        acc.w += wgt;
        if (acc.w >= ert) break;
    }
    return acc;
}

// ----------------------------------------------------------------------------------------
// variant 5: control-point bricks in shared memory, per warp
// ----------------------------------------------------------------------------------------
//
// The 32 rays of a warp march through the same region of the model.  The march is cut
// into segments of S sample indices; for each segment the warp computes the bounding box
// of its rays' sample positions (positions are monotone in the sample index, so the
// segment's end points bound it), turns the box into a range of knot spans per axis, and
// copies the stored control points that range needs (rows of the plain array) into a
// kBrick^3 brick of shared memory -- converted to FP32 once, whatever the storage type.  Every sample of the
// segment then reads its 16 support rows from the brick at fixed offsets (no per-sample
// conversion, no 64-bit address arithmetic).  S adapts so the range fits the brick (halved
// when it does not, doubled back after a segment that fits); a segment of one sample that
// still does not fit is evaluated from global memory.
constexpr int kBrick = 8;
constexpr int kBrickFloats4 = kBrick * kBrick * kBrick;   // 8 KB per warp
constexpr int kSegMax = 64;

// Row P[k][j][i..i+3] of the stored control points as FP32 (zero past the ends).
__device__ __forceinline__ float4 raw_row(const ModelDev& M, int i, int j, int k)
{
    const int nx = M.ax[0].n, ny = M.ax[1].n, nz = M.ax[2].n;
    float v[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        v[a] = 0.0f;
        if (i + a < nx && j < ny && k < nz) {
            const long long e = (static_cast<long long>(k) * ny + j) * nx + i + a;
            if (M.raw_storage == 1) {
                v[a] = __ldg(static_cast<const float*>(M.raw) + e);
            } else {
                const unsigned short h = __ldg(static_cast<const unsigned short*>(M.raw) + e);
                v[a] = M.raw_storage == 2 ? __half2float(__ushort_as_half(h))
                                          : __uint_as_float(static_cast<unsigned>(h) << 16);
            }
        }
    }
    return make_float4(v[0], v[1], v[2], v[3]);
}

// Sum-factorised contraction over a support held in a shared-memory brick (rows at fixed
// offsets from `b0`), in scalar FP32 (the y sums in natural order).
template <int Q>
__device__ __forceinline__ float4 contract_brick(const float4* __restrict__ b0, const float (&Nx)[Q], const float (&Dx)[Q],
                                                 const float (&Ny)[Q], const float (&Dy)[Q], const float (&Nz)[Q],
                                                 const float (&Dz)[Q])
{
    float f = 0.0f, fx = 0.0f, fy = 0.0f, fz = 0.0f;
#pragma unroll
    for (int c = 0; c < Q; ++c) {
        float C = 0.0f, Dv = 0.0f, E = 0.0f;
#pragma unroll
        for (int b = 0; b < Q; ++b) {
            const float4 r4 = b0[(c * kBrick + b) * kBrick];
            const float row[4] = { r4.x, r4.y, r4.z, r4.w };
            float A = 0.0f, B = 0.0f;
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                A = fmaf(Nx[a], row[a], A);
                B = fmaf(Dx[a], row[a], B);
            }
            C = fmaf(Ny[b], A, C);
            Dv = fmaf(Dy[b], A, Dv);
            E = fmaf(Ny[b], B, E);
        }
        f = fmaf(Nz[c], C, f);
        fz = fmaf(Dz[c], C, fz);
        fy = fmaf(Nz[c], Dv, fy);
        fx = fmaf(Nz[c], E, fx);
    }
    return make_float4(f, fx, fy, fz);
}

// Warp-collective: every lane of the warp calls it (valid = false for lanes without a pixel).
template <int Q, int STORAGE>
__device__ __forceinline__ float4 march_bricked(const ModelDev& M, const RenderScalars& P, const float4* __restrict__ tf,
                                                int col, int row, bool valid, unsigned long long& count,
                                                float4* __restrict__ brick)
{
    static_assert(Q <= 4, "bricks hold 4-wide windows");
    const unsigned kFull = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    float o[3], d[3], t0, t1;
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    bool live = ray_box(P, col, row, o, d, t0, t1) && valid;

    const int ns = P.n_samples;
    const float ert = P.ert_alpha;
    const float dt = live ? (t1 - t0) / static_cast<float>(ns) : 0.0f;
    const ShadeParams S = shade_params(P, d);
    AxisCache<Q> cx, cy, cz;
    cx.s = cy.s = cz.s = -1;

    auto pos = [&](int k, float (&u)[3]) {
        const float t = fmaf(static_cast<float>(k) + 0.5f, dt, t0);
#pragma unroll
        for (int a = 0; a < 3; ++a) u[a] = clamp01(fmaf(t, d[a], o[a]));
    };

    int k_lo = 0, seg = 16;
    while (__any_sync(kFull, live) && k_lo < ns) {
        const int kb = min(k_lo + seg, ns) - 1;
        float lo[3] = { 2.0f, 2.0f, 2.0f }, hi[3] = { -1.0f, -1.0f, -1.0f };
        if (live) {
            float pa[3], pb[3];
            pos(k_lo, pa);
            pos(kb, pb);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                lo[a] = fminf(pa[a], pb[a]);
                hi[a] = fmaxf(pa[a], pb[a]);
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                lo[a] = fminf(lo[a], __shfl_xor_sync(kFull, lo[a], off));
                hi[a] = fmaxf(hi[a], __shfl_xor_sync(kFull, hi[a], off));
            }
        }
        // knot spans of the box corners: lanes 0..2 the low corner, lanes 3..5 the high one
        int sv = 0;
        if (lane < 6) {
            const int a = lane % 3;
            const float u = lane < 3 ? (a == 0 ? lo[0] : a == 1 ? lo[1] : lo[2]) : (a == 0 ? hi[0] : a == 1 ? hi[1] : hi[2]);
            sv = locate_span(M.ax[a], clamp01(u));
        }
        int org[3], ext[3];
        bool fits = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int slo = __shfl_sync(kFull, sv, a), shi = __shfl_sync(kFull, sv, a + 3);
            org[a] = slo - M.ax[a].p;
            ext[a] = shi - slo + Q;
            fits = fits && ext[a] <= kBrick;
        }
        if (!fits && seg > 1) {
            seg >>= 1;   // retry this segment with fewer samples
            continue;
        }
        if (fits) {
            const int total = ext[0] * ext[1] * ext[2];
            for (int e = lane; e < total; e += 32) {
                const int ex = e % ext[0], r = e / ext[0];
                const int ey = r % ext[1], ez = r / ext[1];
                brick[(ez * kBrick + ey) * kBrick + ex] = raw_row(M, org[0] + ex, org[1] + ey, org[2] + ez);
            }
            __syncwarp();
        }
        if (live) {
            for (int k = k_lo; k <= kb; ++k) {
                float u[3];
                pos(k, u);
                axis_update<Q>(M.ax[0], cx, u[0]);
                axis_update<Q>(M.ax[1], cy, u[1]);
                axis_update<Q>(M.ax[2], cz, u[2]);
                float Nx[Q], Dx[Q], Ny[Q], Dy[Q], Nz[Q], Dz[Q];   // the brick holds control points
                record_basis<Q>(cx.rec, u[0], Nx, Dx);
                record_basis<Q>(cy.rec, u[1], Ny, Dy);
                record_basis<Q>(cz.rec, u[2], Nz, Dz);
                float4 q;
                if (fits) {
                    const int rx = min(max(cx.s - M.ax[0].p - org[0], 0), kBrick - Q);
                    const int ry = min(max(cy.s - M.ax[1].p - org[1], 0), kBrick - Q);
                    const int rz = min(max(cz.s - M.ax[2].p - org[2], 0), kBrick - Q);
                    q = contract_brick<Q>(brick + (rz * kBrick + ry) * kBrick + rx, Nx, Dx, Ny, Dy, Nz, Dz);
                } else {
                    q = contract<Q, STORAGE>(M, cx.s - M.ax[0].p, cy.s - M.ax[1].p, cz.s - M.ax[2].p,
                                             xin_record<Q, STORAGE>(cx.rec, u[0]), Ny, Dy,
                                             Nz, Dz);
                }
                q.y *= cx.rec[1];
                q.z *= cy.rec[1];
                q.w *= cz.rec[1];
                const float4 c = sample_colour(tf, S, q);
                const float wgt = (1.0f - acc.w) * c.w;
                acc.x = fmaf(wgt, c.x, acc.x);
                acc.y = fmaf(wgt, c.y, acc.y);
                acc.z = fmaf(wgt, c.z, acc.z);
                acc.w += wgt;
                ++count;
                if (acc.w >= ert) {
                    live = false;
                    break;
                }
            }
        }
        __syncwarp();   // the brick is rewritten by the next segment
        k_lo = kb + 1;
        if (fits) seg = min(seg * 2, kSegMax);
    }
    return acc;
}

// ----------------------------------------------------------------------------------------
// one image
// ----------------------------------------------------------------------------------------

template <int Q, int STORAGE, int MODE>
__global__ void __launch_bounds__(kThreads, min_blocks<Q, MODE == 6 || MODE == 7 || MODE >= 9, MODE == 7>())
    k_render(ModelDev M, const __grid_constant__ RenderParams P, int shape)
{
    __shared__ float4 tf[kTfSmem];
    stage_tf(tf, P.tf, P.s.tf_n);
    __syncthreads();

    int col, row;
    tile_pixel(tile_shape(shape), blockIdx.x, blockIdx.y, threadIdx.x, col, row);
    unsigned long long count = 0;
    if constexpr (MODE == 5) {
        __shared__ float4 bricks[kThreads / 32][kBrickFloats4];
        const bool valid = col < P.s.width && row < P.s.height;
        const float4 acc = march_bricked<(Q <= 4 ? Q : 4), STORAGE>(M, P.s, tf, valid ? col : 0, valid ? row : 0, valid,
                                                                    count, bricks[threadIdx.x >> 5]);
        if (valid) P.s.out[static_cast<long long>(row) * P.s.width + col] = acc;
    } else if (col < P.s.width && row < P.s.height) {
        float4 acc;
        if constexpr (MODE == 4)
            acc = march_pipelined<Q, STORAGE>(M, P.s, tf, col, row, count);
        else if constexpr (MODE == 6)
            acc = march_cardinal<Q, STORAGE>(M, P.s, tf, col, row, count);
        else if constexpr (MODE == 7)
            acc = march_cardinal<Q, STORAGE, false, true>(M, P.s, tf, col, row, count);
        else if constexpr (MODE == 8)   // variant 7 off the cardinal path
            acc = march_pipelined<Q, STORAGE, false, true>(M, P.s, tf, col, row, count);
        else if constexpr (MODE == 9)   // variant 8: per-cell patches
            acc = march_patch<STORAGE>(M, P.s, tf, col, row, count);
        else if constexpr (MODE == 10)   // variant 8 off the cardinal path
            acc = march_patch_records<STORAGE>(M, P.s, tf, col, row, count);
        else
            acc = march<Q, STORAGE, MODE>(M, P.s, tf, col, row, count);
        P.s.out[static_cast<long long>(row) * P.s.width + col] = acc;
    }
    if (P.s.samples_out) add_count(P.s.samples_out, count);
}

// Variant 7's visibility bits: bit c of the knot-span cell c is set where some value in the
// cell's bound [min, max] of its support's control points maps to a transfer-function row
// pair with non-zero opacity.  The rows a sample of value f reads are i0(f) and i0(f) + 1
// with i0 monotone in f, so the cell's samples read rows i0(min) .. i0(max) + 1; one row
// more on each side covers FP32 rounding of f just outside the bound.  A prefix count of
// the rows with non-zero opacity answers each cell in O(1).  One thread per 32 cells.
__global__ void __launch_bounds__(256) k_cell_visible(ModelDev M, const __grid_constant__ RenderParams P,
                                                      unsigned* __restrict__ bits)
{
    __shared__ int nz[kTfMax + 2];   // nz[r] = rows below r with non-zero alpha
    if (threadIdx.x == 0) {
        int c = 0;
        for (int r = 0; r < P.s.tf_n; ++r) {
            nz[r] = c;
            c += P.tf[r].w != 0.0f;
        }
        nz[P.s.tf_n] = c;
    }
    __syncthreads();
    const long long cells = static_cast<long long>(M.ncx) * M.ncy * M.ncz;
    const long long words = (cells + 31) / 32;
    const float tscale = static_cast<float>(P.s.tf_n - 1);
    const int tf_last = max(P.s.tf_n - 2, 0);
    for (long long w = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; w < words;
         w += static_cast<long long>(gridDim.x) * blockDim.x) {
        unsigned word = 0u;
        for (int b = 0; b < 32; ++b) {
            const long long c = 32 * w + b;
            if (c >= cells) break;
            const float2 r = M.cell[c];
            const float tl = clamp01((r.x - P.s.vmin) * P.s.inv_range), th = clamp01((r.y - P.s.vmin) * P.s.inv_range);
            const int lo = max(min(static_cast<int>(tl * tscale), tf_last) - 1, 0);
            const int hi = min(min(static_cast<int>(th * tscale), tf_last) + 2, P.s.tf_n - 1);
            if (nz[hi + 1] - nz[lo] > 0) word |= 1u << b;
        }
        bits[w] = word;
    }
}

template <int Q, int STORAGE>
cudaError_t render_qs(const ModelDev& m, const RenderParams& rp, int variant, int shape, cudaStream_t st)
{
    const TileShape T = tile_shape(shape);
    dim3 grid((rp.s.width + T.tw - 1) / T.tw, (rp.s.height + T.th - 1) / T.th);
    if constexpr (compact_window(STORAGE)) {
        // the compact layout has the production marches only: the cardinal path where it
        // applies, else variant 4; variant 7 (skipping) needs cell bounds, which compact
        // models do not keep
        if (m.cardinal)
            k_render<Q, STORAGE, 6><<<grid, kThreads, 0, st>>>(m, rp, shape);
        else
            k_render<Q, STORAGE, 4><<<grid, kThreads, 0, st>>>(m, rp, shape);
        return cudaGetLastError();
    } else {
        switch (variant) {
        case 2: k_render<Q, STORAGE, 2><<<grid, kThreads, 0, st>>>(m, rp, shape); break;
        case 1: k_render<Q, STORAGE, 1><<<grid, kThreads, 0, st>>>(m, rp, shape); break;
        case 7:   // empty-space skipping (needs the visibility bits; without them, variant 6 / 4)
            if (m.cardinal && rp.s.cell_vis)
                k_render<Q, STORAGE, 7><<<grid, kThreads, 0, st>>>(m, rp, shape);
            else if (rp.s.cell_vis)
                k_render<Q, STORAGE, 8><<<grid, kThreads, 0, st>>>(m, rp, shape);
            else if (m.cardinal)
                k_render<Q, STORAGE, 6><<<grid, kThreads, 0, st>>>(m, rp, shape);
            else
                k_render<Q, STORAGE, 4><<<grid, kThreads, 0, st>>>(m, rp, shape);
            break;
        case 0:   // default: the patches on a cardinal model that has them (the batch and
                  // serving kernels' choice too), the cardinal path where it applies, else 4
            if constexpr (Q == 4 && STORAGE == 1) {
                if (m.patch && m.cardinal) {
                    k_render<Q, STORAGE, 9><<<grid, kThreads, 0, st>>>(m, rp, shape);
                    break;
                }
            }
            [[fallthrough]];
        case 6:
            if (m.cardinal)
                k_render<Q, STORAGE, 6><<<grid, kThreads, 0, st>>>(m, rp, shape);
            else
                k_render<Q, STORAGE, 4><<<grid, kThreads, 0, st>>>(m, rp, shape);
            break;
        case 4: k_render<Q, STORAGE, 4><<<grid, kThreads, 0, st>>>(m, rp, shape); break;
        case 8:   // per-cell patches (MFA_WINDOW_PATCH models; otherwise the default)
            if constexpr (Q == 4 && STORAGE == 1) {
                if (m.patch) {
                    if (m.cardinal)
                        k_render<Q, STORAGE, 9><<<grid, kThreads, 0, st>>>(m, rp, shape);
                    else
                        k_render<Q, STORAGE, 10><<<grid, kThreads, 0, st>>>(m, rp, shape);
                    break;
                }
            }
            if (m.cardinal)
                k_render<Q, STORAGE, 6><<<grid, kThreads, 0, st>>>(m, rp, shape);
            else
                k_render<Q, STORAGE, 4><<<grid, kThreads, 0, st>>>(m, rp, shape);
            break;
        case 5:
            if constexpr (Q <= 4) {
                k_render<Q, STORAGE, 5><<<grid, kThreads, 0, st>>>(m, rp, shape);
            } else {
                k_render<Q, STORAGE, 4><<<grid, kThreads, 0, st>>>(m, rp, shape);   // bricks hold 4-wide rows
            }
            break;
        default: k_render<Q, STORAGE, 3><<<grid, kThreads, 0, st>>>(m, rp, shape); break;
        }
        return cudaGetLastError();
    }
}

template <int Q>
cudaError_t render_q(const ModelDev& m, const RenderParams& rp, int variant, int shape, cudaStream_t st)
{
    switch (m.storage) {
    case 1: return render_qs<Q, 1>(m, rp, variant, shape, st);
    case 2: return render_qs<Q, 2>(m, rp, variant, shape, st);
    case 3: return render_qs<Q, 3>(m, rp, variant, shape, st);
    case 4: return render_qs<Q, 4>(m, rp, variant, shape, st);
    case 5: return render_qs<Q, 5>(m, rp, variant, shape, st);
    case 6: return render_qs<Q, 6>(m, rp, variant, shape, st);
    default: return cudaErrorInvalidValue;
    }
}

// ----------------------------------------------------------------------------------------
// object-space decomposition: block segments and their over-merge
// ----------------------------------------------------------------------------------------
//
// The paper renders each partitioned block on its own node into a partial image and
// merges the partial images with the associative over (Sec. IV-A.1, IV-A.4, IV-A.5).  On
// one GPU the blocks are the z index of the launch grid: CTA (tile, b) renders, for every
// pixel of its tile, the samples of that pixel's ray that lie in block b (block_range),
// front to back with early termination on the segment's own alpha, into partial image b.
// The merge then composites, per pixel, the non-empty segments nearest first.

constexpr int kMaxSegBlocks = 64;

template <int Q, int STORAGE, int MODE>
__global__ void __launch_bounds__(kThreads, min_blocks<Q, MODE == 6>())
    k_render_segments(ModelDev M, const __grid_constant__ RenderParams P, int shape, int gx, int gy, int gz,
                      float4* __restrict__ partial)
{
    __shared__ float4 tf[kTfSmem];
    stage_tf(tf, P.tf, P.s.tf_n);
    __syncthreads();

    int col, row;
    tile_pixel(tile_shape(shape), blockIdx.x, blockIdx.y, threadIdx.x, col, row);
    const int b = blockIdx.z;
    SegBlock B;
    B.g[0] = gx;
    B.g[1] = gy;
    B.g[2] = gz;
    B.bi[0] = b % gx;
    B.bi[1] = (b / gx) % gy;
    B.bi[2] = b / (gx * gy);
    unsigned long long count = 0;
    if (col < P.s.width && row < P.s.height) {
        float4 acc;
        if constexpr (MODE == 6)
            acc = march_cardinal<Q, STORAGE, true>(M, P.s, tf, col, row, count, &B);
        else
            acc = march_pipelined<Q, STORAGE, true>(M, P.s, tf, col, row, count, &B);
        const long long npix = static_cast<long long>(P.s.width) * P.s.height;
        partial[b * npix + static_cast<long long>(row) * P.s.width + col] = acc;
    }
    if (P.s.samples_out) add_count(P.s.samples_out, count);
}

// One thread per pixel: the non-empty segments of the pixel's ray, ordered by their first
// sample, composited with over into the output image.
__global__ void __launch_bounds__(256) k_merge_segments(const __grid_constant__ RenderScalars S, int gx, int gy,
                                                        int gz, const float4* __restrict__ partial)
{
    const int col = blockIdx.x * 16 + (threadIdx.x & 15), row = blockIdx.y * 16 + (threadIdx.x >> 4);
    if (col >= S.width || row >= S.height) return;
    const long long npix = static_cast<long long>(S.width) * S.height;
    const long long pix = static_cast<long long>(row) * S.width + col;
    float o[3], d[3], t0, t1;
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (ray_box(S, col, row, o, d, t0, t1)) {
        const int ns = S.n_samples;
        const float dt = (t1 - t0) / static_cast<float>(ns);
        int first[kMaxSegBlocks], blk[kMaxSegBlocks], n = 0;
        SegBlock B;
        B.g[0] = gx;
        B.g[1] = gy;
        B.g[2] = gz;
        const int nb = gx * gy * gz;
        for (int b = 0; b < nb; ++b) {
            B.bi[0] = b % gx;
            B.bi[1] = (b / gx) % gy;
            B.bi[2] = b / (gx * gy);
            int kb, ke;
            block_range(B, o, d, t0, dt, ns, kb, ke);
            if (kb >= ke) continue;
            int i = n++;   // insertion by first sample index (segments are disjoint)
            while (i > 0 && first[i - 1] > kb) {
                first[i] = first[i - 1];
                blk[i] = blk[i - 1];
                --i;
            }
            first[i] = kb;
            blk[i] = b;
        }
        for (int i = 0; i < n; ++i) {
            const float4 p = partial[blk[i] * npix + pix];
            const float tr = 1.0f - acc.w;
            acc.x = fmaf(tr, p.x, acc.x);
            acc.y = fmaf(tr, p.y, acc.y);
            acc.z = fmaf(tr, p.z, acc.z);
            acc.w = fmaf(tr, p.w, acc.w);
        }
    }
    S.out[pix] = acc;
}

template <int Q, int STORAGE>
cudaError_t segments_qs(const ModelDev& m, const RenderParams& rp, bool cardinal, int shape, const int g[3],
                        float4* partial, cudaStream_t st)
{
    const TileShape T = tile_shape(shape);
    dim3 grid((rp.s.width + T.tw - 1) / T.tw, (rp.s.height + T.th - 1) / T.th, g[0] * g[1] * g[2]);
    if (cardinal)
        k_render_segments<Q, STORAGE, 6><<<grid, kThreads, 0, st>>>(m, rp, shape, g[0], g[1], g[2], partial);
    else
        k_render_segments<Q, STORAGE, 4><<<grid, kThreads, 0, st>>>(m, rp, shape, g[0], g[1], g[2], partial);
    return cudaGetLastError();
}

template <int Q>
cudaError_t segments_q(const ModelDev& m, const RenderParams& rp, bool cardinal, int shape, const int g[3],
                       float4* partial, cudaStream_t st)
{
    switch (m.storage) {
    case 1: return segments_qs<Q, 1>(m, rp, cardinal, shape, g, partial, st);
    case 2: return segments_qs<Q, 2>(m, rp, cardinal, shape, g, partial, st);
    case 3: return segments_qs<Q, 3>(m, rp, cardinal, shape, g, partial, st);
    case 4: return segments_qs<Q, 4>(m, rp, cardinal, shape, g, partial, st);
    case 5: return segments_qs<Q, 5>(m, rp, cardinal, shape, g, partial, st);
    case 6: return segments_qs<Q, 6>(m, rp, cardinal, shape, g, partial, st);
    default: return cudaErrorInvalidValue;
    }
}

// ----------------------------------------------------------------------------------------
// persistent batch
// ----------------------------------------------------------------------------------------

// The model tables a persistent kernel's march reads: the CTA's shared-memory copy of the
// request, or a copy of it in registers.  The march reads a few of them at every knot-span
// cell a ray enters, and from shared memory each is a dependent shared load on the critical
// path: a one-request batch of the largest serving view (2048^2, 2048 samples) took 35.4 ms
// that way against 31.6 ms from registers (a plain launch, which reads them as constant-bank
// operands, 31.1 ms).  The register copy fits without spills on the cardinal path with FP32
// layer-pair windows at degree classes 2..4; elsewhere it spilled (16 to 650 bytes), so those
// kernels keep reading the shared copy.
template <int Q, int STORAGE, bool CARD, bool PATCH>
__device__ __forceinline__ float4 march_item(const BatchItem& item, const float4* tf, int col, int row,
                                             unsigned long long& count)
{
    if constexpr (PATCH) {   // the group of models with per-cell patches (degree class 4, FP32)
        const ModelDev m = item.m;
        return march_patch<STORAGE>(m, item.s, tf, col, row, count);
    } else if constexpr (!CARD) {
        return march_pipelined<Q, STORAGE>(item.m, item.s, tf, col, row, count);
    } else if constexpr (STORAGE == 1 && Q <= 4) {
        const ModelDev m = item.m;
        return march_cardinal<Q, STORAGE>(m, item.s, tf, col, row, count);
    } else {
        return march_cardinal<Q, STORAGE>(item.m, item.s, tf, col, row, count);
    }
}

// Persistent CTAs over the requests of one (degree, storage) group: draw a tile, find its
// request (tiles of one request are contiguous, so the previous request is checked
// first), stage the request and its table in shared memory when it changes, render,
// repeat until the counter passes the group's last tile.  One kernel per group keeps each
// degree's (and each path's) register allocation free of the others'.  PATCH: the group of
// models with per-cell patches (render variant 8).
template <int Q, int STORAGE, bool CARD, bool PATCH = false>
__global__ void __launch_bounds__(kThreads, min_blocks<Q, CARD>()) k_render_batch(BatchHead* __restrict__ table, int group,
                                                                       int shape)
{
    __shared__ BatchItem item;
    __shared__ float4 tf[kTfSmem];
    __shared__ int s_tile, s_idx;
    BatchHead* head = table + group;
    const BatchItem* items =
        reinterpret_cast<const BatchItem*>(reinterpret_cast<const char*>(table) + head->items_offset);
    const int n_items = head->n_items, total = head->total_tiles;
    const TileShape T = tile_shape(shape);
    int cur = -1;
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = atomicAdd(&head->next_tile, 1);
            int i = cur < 0 ? 0 : cur;
            if (t < total) {
                if (!(items[i].tile_begin <= t && (i + 1 >= n_items || t < items[i + 1].tile_begin))) {
                    int lo = 0, hi = n_items - 1;      // largest i with tile_begin <= t
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) / 2;
                        if (items[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
                    }
                    i = lo;
                }
            }
            s_tile = t;
            s_idx = i;
        }
        __syncthreads();
        const int t = s_tile, i = s_idx;
        if (t >= total) break;
        if (i != cur) {
            const int* src = reinterpret_cast<const int*>(items + i);
            int* dst = reinterpret_cast<int*>(&item);
            for (int e = threadIdx.x; e < static_cast<int>(sizeof(BatchItem) / sizeof(int)); e += kThreads) dst[e] = src[e];
            __syncthreads();
            stage_tf(tf, item.tf, item.s.tf_n);
            cur = i;
            __syncthreads();
        }
        const int local = t - item.tile_begin;
        const int tx = local % item.tiles_x, ty = local / item.tiles_x;
        int col, row;
        tile_pixel(T, tx, ty, threadIdx.x, col, row);
        unsigned long long count = 0;
        if (col < item.s.width && row < item.s.height) {
            const float4 acc = march_item<Q, STORAGE, CARD, PATCH>(item, tf, col, row, count);
            item.s.out[static_cast<long long>(row) * item.s.width + col] = acc;
        }
        if (item.s.samples_out) add_count(item.s.samples_out, count);
        __syncthreads();   // s_tile / s_idx / item are rewritten next round
    }
}

// ----------------------------------------------------------------------------------------
// serving: persistent CTAs over the device work queue
// ----------------------------------------------------------------------------------------
//
// Thread 0 of a CTA walks the active list (most urgent first), skips records of other
// groups and exhausted ones, and claims a tile of the first record that has one (atomicAdd
// on the record's ticket word; the claim is checked against the record's generation and
// tile count, see ServeRecord).  Its next claims go straight to the same record (one atomic
// instead of the walk's chain of dependent loads) until that record runs out or
// kServeRewalk claims have passed.  Records and the list are rewritten by the host while the
// kernel runs, so they are read through L2 (ld.cg), never from a possibly stale L1 line.
// After a tile, the CTA counts it done; the CTA that finishes a record's last tile
// publishes the record's generation to host-mapped memory (system-scope release), which the
// server thread polls.  A CTA that finds nothing to claim exits: no wait anywhere.
__device__ __forceinline__ int item_total(const ServeRecord* recs, int r) { return __ldcg(&recs[r].total_tiles); }

// Tiles a CTA claims from the record it is on before it walks the active list again.
constexpr int kServeRewalk = 8;

template <int Q, int STORAGE, bool CARD, bool PATCH = false>
__global__ void __launch_bounds__(kThreads, min_blocks<Q, CARD>())
    k_serve(ServeRecord* __restrict__ recs, const ServeQueue* __restrict__ queue, unsigned* __restrict__ done,
            int group, int shape)
{
    __shared__ BatchItem item;
    __shared__ float4 tf[kTfSmem];
    __shared__ int s_rec, s_tile, s_gen;
    const TileShape T = tile_shape(shape);
    int cur_rec = -1, cur_gen = -1;
    // thread 0 only: the record it claimed from last, its generation and tile count, and the
    // claims made since the list was last walked
    int last_rec = -1, last_gen = 0, last_total = 0, since_walk = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            int rec = -1, tile = 0, gen = 0;
            // another tile of the same record: one atomic, checked against the claim's
            // generation and the record's tile count already known; the list is walked again
            // after kServeRewalk claims so that newly published urgent requests get tiles soon
            if (last_rec >= 0 && since_walk < kServeRewalk) {
                ServeRecord* R = recs + last_rec;
                const unsigned long long claim = atomicAdd(&R->ticket, 1ull);
                const int g = static_cast<int>(claim >> 32), t = static_cast<int>(claim & 0xFFFFFFFFu);
                if (g != last_gen) {
                    // the record was republished since: a claim of its current generation is
                    // as valid as any (and must not be dropped), so check it as the walk does
                    const int total = __ldcg(&R->total_tiles);
                    if (g == __ldcg(&R->gen) && t < total) {
                        last_gen = g;
                        last_total = total;
                    }
                }
                if (g == last_gen && t < last_total) {
                    rec = last_rec;
                    tile = t;
                    gen = g;
                    ++since_walk;
                }
            }
            const int n = rec >= 0 ? 0 : min(__ldcg(&queue->n_active), kServeMaxActive);
            if (rec < 0) {
                since_walk = 0;
                last_rec = -1;
            }
            for (int a = 0; a < n && rec < 0; ++a) {
                const int r = __ldcg(&queue->active[a]);
                ServeRecord* R = recs + r;
                if (__ldcg(&R->group) != group) continue;
                const int total = __ldcg(&R->total_tiles);
                const unsigned long long seen = __ldcg(&R->ticket);
                if (static_cast<int>(seen >> 32) != __ldcg(&R->gen) || static_cast<int>(seen & 0xFFFFFFFFu) >= total)
                    continue;   // exhausted, or being republished
                const unsigned long long claim = atomicAdd(&R->ticket, 1ull);
                const int g = static_cast<int>(claim >> 32), t = static_cast<int>(claim & 0xFFFFFFFFu);
                const int claim_total = __ldcg(&R->total_tiles);   // of the claim's generation when valid
                if (g == __ldcg(&R->gen) && t < claim_total) {
                    rec = r;
                    tile = t;
                    gen = g;
                    last_rec = r;
                    last_gen = g;
                    last_total = claim_total;
                }
            }
            s_rec = rec;
            s_tile = tile;
            s_gen = gen;
        }
        __syncthreads();
        const int r = s_rec, t = s_tile, g = s_gen;
        if (r < 0) break;
        if (r != cur_rec || g != cur_gen) {
            const int* src = reinterpret_cast<const int*>(&recs[r].item);
            int* dst = reinterpret_cast<int*>(&item);
            for (int e = threadIdx.x; e < static_cast<int>(sizeof(BatchItem) / sizeof(int)); e += kThreads)
                dst[e] = __ldcg(src + e);
            __syncthreads();
            const float4* rows = recs[r].tf;
            for (int e = threadIdx.x; e < item.s.tf_n; e += kThreads) {
                const float4 a = __ldcg(rows + e), b = e + 1 < item.s.tf_n ? __ldcg(rows + e + 1) : a;
                tf[2 * e] = a;
                tf[2 * e + 1] = make_float4(b.x - a.x, b.y - a.y, b.z - a.z, b.w - a.w);
            }
            cur_rec = r;
            cur_gen = g;
            __syncthreads();
        }
        const int tx = t % item.tiles_x, ty = t / item.tiles_x;
        int col, row;
        tile_pixel(T, tx, ty, threadIdx.x, col, row);
        unsigned long long count = 0;
        if (col < item.s.width && row < item.s.height) {
            const float4 acc = march_item<Q, STORAGE, CARD, PATCH>(item, tf, col, row, count);
            item.s.out[static_cast<long long>(row) * item.s.width + col] = acc;
        }
        if (item.s.samples_out) add_count(item.s.samples_out, count);
        __syncthreads();   // every pixel of the tile is written; s_* are rewritten next round
        if (threadIdx.x == 0) {
            __threadfence();
            const int finished = atomicAdd(&recs[r].done_tiles, 1) + 1;
            if (finished == item_total(recs, r)) {
                __threadfence_system();
                asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(done + r), "r"(static_cast<unsigned>(g))
                             : "memory");
            }
        }
    }
}

template <int Q, int STORAGE, bool CARD, bool PATCH = false>
BatchKernel serve_kernel_qs()
{
    BatchKernel k;
    k.fn = reinterpret_cast<const void*>(&k_serve<Q, STORAGE, CARD, PATCH>);
    int blocks = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_serve<Q, STORAGE, CARD, PATCH>, kThreads, 0);
    k.blocks_per_sm = blocks > 0 ? blocks : 1;
    k.threads = kThreads;
    return k;
}

template <int Q, bool CARD>
BatchKernel serve_kernel_qc(int storage)
{
    switch (storage) {
    case 1: return serve_kernel_qs<Q, 1, CARD>();
    case 2: return serve_kernel_qs<Q, 2, CARD>();
    case 3: return serve_kernel_qs<Q, 3, CARD>();
    case 4: return serve_kernel_qs<Q, 4, CARD>();
    case 5: return serve_kernel_qs<Q, 5, CARD>();
    default: return serve_kernel_qs<Q, 6, CARD>();
    }
}

template <int Q, int STORAGE, bool CARD, bool PATCH = false>
BatchKernel batch_kernel_qs()
{
    BatchKernel k;
    k.fn = reinterpret_cast<const void*>(&k_render_batch<Q, STORAGE, CARD, PATCH>);
    int blocks = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_render_batch<Q, STORAGE, CARD, PATCH>, kThreads, 0);
    k.blocks_per_sm = blocks > 0 ? blocks : 1;
    k.threads = kThreads;
    return k;
}

template <int Q, bool CARD>
BatchKernel batch_kernel_qc(int storage)
{
    switch (storage) {
    case 1: return batch_kernel_qs<Q, 1, CARD>();
    case 2: return batch_kernel_qs<Q, 2, CARD>();
    case 3: return batch_kernel_qs<Q, 3, CARD>();
    case 4: return batch_kernel_qs<Q, 4, CARD>();
    case 5: return batch_kernel_qs<Q, 5, CARD>();
    default: return batch_kernel_qs<Q, 6, CARD>();
    }
}

template <int Q>
BatchKernel batch_kernel_q(int storage, int cardinal)
{
    return cardinal ? batch_kernel_qc<Q, true>(storage) : batch_kernel_qc<Q, false>(storage);
}

}  // namespace

int render_tile_dims(int shape, int* tw, int* th)
{
    if (shape < 0 || shape >= kTileShapes) return -1;
    *tw = tile_shape(shape).tw;
    *th = tile_shape(shape).th;
    return 0;
}

cudaError_t launch_cell_visibility(const ModelDev& m, const RenderParams& rp, unsigned* bits, cudaStream_t stream)
{
    const long long words = (static_cast<long long>(m.ncx) * m.ncy * m.ncz + 31) / 32;
    const long long want = (words + 255) / 256;
    k_cell_visible<<<static_cast<int>(want < 2048 ? want : 2048), 256, 0, stream>>>(m, rp, bits);
    return cudaGetLastError();
}

cudaError_t launch_render(const ModelDev& m, const RenderParams& rp, int variant, int shape, cudaStream_t stream)
{
    switch (m.q) {
    case 2: return render_q<2>(m, rp, variant, shape, stream);
    case 3: return render_q<3>(m, rp, variant, shape, stream);
    case 4: return render_q<4>(m, rp, variant, shape, stream);
    case 5: return render_q<5>(m, rp, variant, shape, stream);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_render_segments(const ModelDev& m, const RenderParams& rp, int variant, int shape, const int g[3],
                                   float4* partial, cudaStream_t stream)
{
    if (g[0] * g[1] * g[2] > kMaxSegBlocks) return cudaErrorInvalidValue;
    const bool cardinal = m.cardinal && variant != 4;
    switch (m.q) {
    case 2: return segments_q<2>(m, rp, cardinal, shape, g, partial, stream);
    case 3: return segments_q<3>(m, rp, cardinal, shape, g, partial, stream);
    case 4: return segments_q<4>(m, rp, cardinal, shape, g, partial, stream);
    case 5: return segments_q<5>(m, rp, cardinal, shape, g, partial, stream);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_merge_segments(const RenderScalars& s, const int g[3], const float4* partial, cudaStream_t stream)
{
    if (g[0] * g[1] * g[2] > kMaxSegBlocks) return cudaErrorInvalidValue;
    dim3 grid((s.width + 15) / 16, (s.height + 15) / 16);
    k_merge_segments<<<grid, 256, 0, stream>>>(s, g[0], g[1], g[2], partial);
    return cudaGetLastError();
}

BatchKernel render_serve_kernel(int q, int storage, int cardinal, bool patch)
{
    if (patch) return serve_kernel_qs<4, 1, true, true>();
    switch (q) {
    case 2: return cardinal ? serve_kernel_qc<2, true>(storage) : serve_kernel_qc<2, false>(storage);
    case 3: return cardinal ? serve_kernel_qc<3, true>(storage) : serve_kernel_qc<3, false>(storage);
    case 4: return cardinal ? serve_kernel_qc<4, true>(storage) : serve_kernel_qc<4, false>(storage);
    default: return cardinal ? serve_kernel_qc<5, true>(storage) : serve_kernel_qc<5, false>(storage);
    }
}

BatchKernel render_batch_kernel(int q, int storage, int cardinal, bool patch)
{
    if (patch) return batch_kernel_qs<4, 1, true, true>();
    switch (q) {
    case 2: return batch_kernel_q<2>(storage, cardinal);
    case 3: return batch_kernel_q<3>(storage, cardinal);
    case 4: return batch_kernel_q<4>(storage, cardinal);
    default: return batch_kernel_q<5>(storage, cardinal);
    }
}

}  // namespace mfa
