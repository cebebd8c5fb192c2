// iso.cu -- isosurface rendering through MFA queries (mfa_render_iso): the other
// visualization the paper names for its query interface (Sec. IV-A.4).  One thread per
// pixel: the ray's samples (the volume render's positions) are examined in order until
// f - iso changes sign between two of them.  A sample whose knot-span cell has all the
// control points of its support on one side of iso has that sign without a query (the
// model lies in the convex hull of those control points), and so do the cell's later
// samples: the search steps to the cell's exit; the others take a value-only query (no
// derivative weights).  The crossing is refined by kIsoSteps Newton
// steps on g(t) = f(o + t d) - iso with the analytic derivative g'(t) = grad f . d, kept
// inside the bracket (each step shrinks the bracket to the side where g changes sign and
// falls back to its midpoint when the Newton point leaves it); the hit is shaded like a
// volume sample of value iso (transfer-function colour, Phong with grad f), opaque.
#include "raycast.cuh"

namespace mfa {
namespace {

constexpr int kIsoThreads = 128;
constexpr int kIsoSteps = 8;

// Queries at successive points of one ray, carrying each axis's span state between them.
template <int Q, int STORAGE, bool CARD>
struct RayQuery;

// Cardinal path (uniform knots, one degree): span = floor((n-p) u), interior spans without
// records.
template <int Q, int STORAGE>
struct RayQuery<Q, STORAGE, true> {
    CardAxis c[3];
    float m[3];
    int base;

    __device__ __forceinline__ void init(const ModelDev& M)
    {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            m[a] = static_cast<float>(M.ax[a].n - M.ax[a].p);
            c[a].jf = -INFINITY;
            c[a].j = 0;
            c[a].edge = false;
        }
        base = 0;
    }

    // brings the span state to the point and returns the local coordinates
    __device__ __forceinline__ void locate(const ModelDev& M, float u, float v, float w, float (&t)[3])
    {
        const float x[3] = { u * m[0], v * m[1], w * m[2] };
        bool moved = false;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            t[a] = x[a] - c[a].jf;
            if (!(t[a] >= 0.0f && t[a] < 1.0f)) {
                card_update(M.ax[a], c[a], x[a]);
                t[a] = x[a] - c[a].jf;
                moved = true;
            }
        }
        if (moved) base = (c[2].j * M.nyp + c[1].j) * M.nxp + c[0].j;
    }

    // f - iso at the parameter point (u, v, w) of the unit box, or, where the point's cell
    // bounds the model away from iso, a stand-in of the same sign without a query
    __device__ __forceinline__ float g(const ModelDev& M, float u, float v, float w, float iso, bool& bounded)
    {
        float t[3];
        locate(M, u, v, w, t);
        int ci = (c[2].j * M.ncy + c[1].j) * M.ncx + c[0].j;
        MFA_DBG_INDEX(M.dbg, ci, static_cast<long long>(M.ncx) * M.ncy * M.ncz, kDbgCell);
        const float2 r = M.cell ? __ldg(M.cell + ci) : make_float2(-INFINITY, INFINITY);   // none: query
        bounded = iso < r.x || iso > r.y;
        if (iso < r.x) return r.x - iso;
        if (iso > r.y) return r.y - iso;
        float Ny[Q], Dy[Q], Nz[Q], Dz[Q];   // derivatives unused: dropped by the compiler
        const XIn<Q, STORAGE> X = xin_card<Q, STORAGE>(M.ax[0], c[0], t[0]);
        card_basis<Q>(M.ax[1], c[1], t[1], Ny, Dy);
        card_basis<Q>(M.ax[2], c[2], t[2], Nz, Dz);
        return value_at<Q, STORAGE>(M, base, X, Ny, Nz) * Cardinal<Q>::template val_scale<STORAGE>() - iso;
    }

    // ray parameter at which the ray o + t d leaves the current cell: the cell spans
    // [j/m, (j+1)/m) along each axis of the unit box
    __device__ __forceinline__ float cell_exit(const float (&o)[3], const float (&d)[3]) const
    {
        float te = INFINITY;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (d[a] > 0.0f) te = fminf(te, (static_cast<float>(c[a].j + 1) / m[a] - o[a]) / d[a]);
            else if (d[a] < 0.0f) te = fminf(te, (static_cast<float>(c[a].j) / m[a] - o[a]) / d[a]);
        }
        return te;
    }

    // {f, df/du, df/dv, df/dw} at the parameter point (u, v, w) of the unit box
    __device__ __forceinline__ float4 at(const ModelDev& M, float u, float v, float w)
    {
        float t[3];
        locate(M, u, v, w, t);
        float Ny[Q], Dy[Q], Nz[Q], Dz[Q];
        const XIn<Q, STORAGE> X = xin_card<Q, STORAGE>(M.ax[0], c[0], t[0]);
        card_basis<Q>(M.ax[1], c[1], t[1], Ny, Dy);
        card_basis<Q>(M.ax[2], c[2], t[2], Nz, Dz);
        float4 q = contract_at<Q, STORAGE>(M, base, X, Ny, Dy, Nz, Dz);
        q.x *= Cardinal<Q>::template val_scale<STORAGE>();
        q.y *= m[0] * Cardinal<Q>::template gradx_scale<STORAGE>();
        q.z *= m[1] * Cardinal<Q>::template gradyz_scale<STORAGE>();
        q.w *= m[2] * Cardinal<Q>::template gradyz_scale<STORAGE>();
        return q;
    }
};

// Record path: each axis's span record cached in registers, reloaded when the span changes.
template <int Q, int STORAGE>
struct RayQuery<Q, STORAGE, false> {
    AxisCache<Q> c[3];

    __device__ __forceinline__ void init(const ModelDev&)
    {
#pragma unroll
        for (int a = 0; a < 3; ++a) c[a].s = -1;
    }

    __device__ __forceinline__ float g(const ModelDev& M, float u, float v, float w, float iso, bool& bounded)
    {
        const float x[3] = { clamp01(u), clamp01(v), clamp01(w) };
#pragma unroll
        for (int a = 0; a < 3; ++a) axis_update<Q>(M.ax[a], c[a], x[a]);
        int ci = ((c[2].s - M.ax[2].p) * M.ncy + (c[1].s - M.ax[1].p)) * M.ncx + (c[0].s - M.ax[0].p);
        MFA_DBG_INDEX(M.dbg, ci, static_cast<long long>(M.ncx) * M.ncy * M.ncz, kDbgCell);
        const float2 r = M.cell ? __ldg(M.cell + ci) : make_float2(-INFINITY, INFINITY);   // none: query
        bounded = iso < r.x || iso > r.y;
        if (iso < r.x) return r.x - iso;
        if (iso > r.y) return r.y - iso;
        float Ny[Q], Dy[Q], Nz[Q], Dz[Q];   // derivatives unused: dropped by the compiler
        const XIn<Q, STORAGE> X = xin_record<Q, STORAGE>(c[0].rec, x[0]);
        record_basis<Q>(c[1].rec, x[1], Ny, Dy);
        record_basis<Q>(c[2].rec, x[2], Nz, Dz);
        return value_at<Q, STORAGE>(
                   M, ((c[2].s - M.ax[2].p) * M.nyp + (c[1].s - M.ax[1].p)) * M.nxp + (c[0].s - M.ax[0].p), X, Ny,
                   Nz) -
               iso;
    }

    // ray parameter at which the ray o + t d leaves the current cell: the span records'
    // FP32 bounds [lo, hi) along each axis
    __device__ __forceinline__ float cell_exit(const float (&o)[3], const float (&d)[3]) const
    {
        float te = INFINITY;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (d[a] > 0.0f) te = fminf(te, (c[a].rec[3] - o[a]) / d[a]);
            else if (d[a] < 0.0f) te = fminf(te, (c[a].rec[2] - o[a]) / d[a]);
        }
        return te;
    }

    __device__ __forceinline__ float4 at(const ModelDev& M, float u, float v, float w)
    {
        const float x[3] = { clamp01(u), clamp01(v), clamp01(w) };
#pragma unroll
        for (int a = 0; a < 3; ++a) axis_update<Q>(M.ax[a], c[a], x[a]);
        float Ny[Q], Dy[Q], Nz[Q], Dz[Q];
        const XIn<Q, STORAGE> X = xin_record<Q, STORAGE>(c[0].rec, x[0]);
        record_basis<Q>(c[1].rec, x[1], Ny, Dy);
        record_basis<Q>(c[2].rec, x[2], Nz, Dz);
        float4 q = contract<Q, STORAGE>(M, c[0].s - M.ax[0].p, c[1].s - M.ax[1].p, c[2].s - M.ax[2].p, X, Ny, Dy,
                                        Nz, Dz);
        q.y *= c[0].rec[1];
        q.z *= c[1].rec[1];
        q.w *= c[2].rec[1];
        return q;
    }
};

template <int Q, int STORAGE, bool CARD>
__global__ void __launch_bounds__(kIsoThreads, Q <= 4 ? 4 : 3)
    k_render_iso(ModelDev M, const __grid_constant__ RenderParams P, float iso, float* __restrict__ depth, int shape)
{
    __shared__ float4 tf[kTfSmem];
    stage_tf(tf, P.tf, P.s.tf_n);
    __syncthreads();

    int col, row;
    tile_pixel(tile_shape(shape), blockIdx.x, blockIdx.y, threadIdx.x, col, row);
    unsigned long long count = 0;
    if (col < P.s.width && row < P.s.height) {
        float4 out = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        float hit_t = INFINITY;
        float o[3], d[3], t0, t1;
        if (ray_box(P.s, col, row, o, d, t0, t1)) {
            const int ns = P.s.n_samples;
            const float dt = (t1 - t0) / static_cast<float>(ns);
            RayQuery<Q, STORAGE, CARD> rq;
            rq.init(M);
            auto query = [&](float t) {
                ++count;
                return rq.at(M, fmaf(t, d[0], o[0]), fmaf(t, d[1], o[1]), fmaf(t, d[2], o[2]));
            };
            bool bounded = false;
            auto g_at = [&](float t) {
                ++count;
                return rq.g(M, fmaf(t, d[0], o[0]), fmaf(t, d[1], o[1]), fmaf(t, d[2], o[2]), iso, bounded);
            };
            // first sign change of g = f - iso between consecutive samples
            float ta = 0.0f, ga = 0.0f, tb = 0.0f;
            bool found = false;
            for (int k = 0; k < ns; ++k) {
                const float t = fmaf(static_cast<float>(k) + 0.5f, dt, t0);
                const float g = g_at(t);
                if (g == 0.0f) {
                    ta = tb = t;
                    found = true;
                    break;
                }
                if (k > 0 && ((ga < 0.0f) != (g < 0.0f))) {
                    tb = t;
                    found = true;
                    break;
                }
                ta = t;
                ga = g;
                if (bounded) {
                    // every sample of this cell has g's sign: step to the cell's last sample
                    // but one (a sample of margin against rounding), counting the samples
                    // passed as examined
                    const float kf = (rq.cell_exit(o, d) - t0) / dt - 0.5f;   // samples k' < kf precede the exit
                    const int klast = kf < static_cast<float>(ns) ? static_cast<int>(ceilf(kf)) - 1 : ns - 1;
                    const int kj = klast - 1;
                    if (kj > k) {
                        count += static_cast<unsigned>(kj - k);
                        ta = fmaf(static_cast<float>(kj) + 0.5f, dt, t0);
                        k = kj;
                    }
                }
            }
            if (found) {
                float t = 0.5f * (ta + tb);
                if (ta != tb) {
                    for (int s = 0; s < kIsoSteps; ++s) {
                        const float4 q = query(t);
                        const float g = q.x - iso;
                        if (g == 0.0f) break;
                        if ((g < 0.0f) == (ga < 0.0f)) {
                            ta = t;
                            ga = g;
                        } else {
                            tb = t;
                        }
                        const float dg = q.y * d[0] + q.z * d[1] + q.w * d[2];
                        const float tn = dg != 0.0f ? t - g / dg : NAN;
                        t = (tn >= ta && tn <= tb) ? tn : 0.5f * (ta + tb);
                    }
                }
                const float4 q = query(t);
                const float4 c = sample_colour(tf, shade_params(P.s, d), make_float4(iso, q.y, q.z, q.w));
                out = make_float4(c.x, c.y, c.z, 1.0f);
                hit_t = t;
            }
        }
        const long long pix = static_cast<long long>(row) * P.s.width + col;
        P.s.out[pix] = out;
        if (depth) depth[pix] = hit_t;
    }
    if (P.s.samples_out) add_count(P.s.samples_out, count);
}

template <int Q, int STORAGE>
cudaError_t iso_qs(const ModelDev& m, const RenderParams& rp, float iso, float* depth, int shape, cudaStream_t st)
{
    const TileShape T = tile_shape(shape);
    dim3 grid((rp.s.width + T.tw - 1) / T.tw, (rp.s.height + T.th - 1) / T.th);
    if (m.cardinal)
        k_render_iso<Q, STORAGE, true><<<grid, kIsoThreads, 0, st>>>(m, rp, iso, depth, shape);
    else
        k_render_iso<Q, STORAGE, false><<<grid, kIsoThreads, 0, st>>>(m, rp, iso, depth, shape);
    return cudaGetLastError();
}

template <int Q>
cudaError_t iso_q(const ModelDev& m, const RenderParams& rp, float iso, float* depth, int shape, cudaStream_t st)
{
    switch (m.storage) {
    case 1: return iso_qs<Q, 1>(m, rp, iso, depth, shape, st);
    case 2: return iso_qs<Q, 2>(m, rp, iso, depth, shape, st);
    case 3: return iso_qs<Q, 3>(m, rp, iso, depth, shape, st);
    case 4: return iso_qs<Q, 4>(m, rp, iso, depth, shape, st);
    case 5: return iso_qs<Q, 5>(m, rp, iso, depth, shape, st);
    case 6: return iso_qs<Q, 6>(m, rp, iso, depth, shape, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_render_iso(const ModelDev& m, const RenderParams& rp, float iso, float* depth, int shape,
                              cudaStream_t st)
{
    switch (m.q) {
    case 2: return iso_q<2>(m, rp, iso, depth, shape, st);
    case 3: return iso_q<3>(m, rp, iso, depth, shape, st);
    case 4: return iso_q<4>(m, rp, iso, depth, shape, st);
    case 5: return iso_q<5>(m, rp, iso, depth, shape, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace
}  // namespace mfa

#include "host.cuh"

using namespace mfa;

extern "C" int mfa_render_iso(const mfa_model* m, const mfa_camera* cam, const mfa_transfer_fn* tf, int width,
                              int height, int n_samples, float iso_value, float* rgba_out, float* depth_out,
                              const mfa_render_opts* opts)
{
    if (!(iso_value == iso_value) || iso_value == INFINITY || iso_value == -INFINITY)
        return fail(MFA_ERR_ARG, "iso_value must be finite");
    const int shape = opts ? opts->tile_shape : 0;
    if (shape < 0 || shape >= kTileShapes) return fail(MFA_ERR_ARG, "tile_shape %d outside 0..%d", shape, kTileShapes - 1);
    RenderParams P;
    if (int rc = setup_render(m, cam, tf, width, height, n_samples, rgba_out, opts ? opts->samples_out : nullptr, P.s,
                              P.tf))
        return rc;
    cudaError_t e = launch_render_iso(m->dev, P, iso_value, depth_out, shape, current_stream());
    return e == cudaSuccess ? MFA_OK : cuda_fail(e, "isosurface launch");
}
