// raycast.cuh -- the per-ray machinery shared by the ray-casting kernels (volume rendering
// in render.cu, isosurfaces in iso.cu): ray tiles, pixel-centre rays clipped to the unit
// box (Sec. IV-A.4), the per-axis span state a ray carries along its samples, the colour
// of a sample (transfer function and Phong, Sec. IV-B), the object-space block ranges
// (Sec. IV-A.1), and the two production ray marches -- span records cached in registers
// (variant 4) and the cardinal path for uniform knots (variant 6) -- both software-
// pipelined over samples.
#pragma once

#include "bspline.cuh"

namespace mfa {

// Ray-tile shapes (CTA tile, warp tile).  Shape 0 is the default; the autotuner picks one
// per workload.
struct TileShape {
    int tw, th;   // pixels per CTA tile
    int ww, wh;   // pixels per warp tile (ww * wh = 32)
};
__host__ __device__ constexpr TileShape tile_shape(int s)
{
    return s == 1 ? TileShape{ 32, 4, 8, 4 } : s == 2 ? TileShape{ 8, 16, 4, 8 } : s == 3 ? TileShape{ 16, 8, 16, 2 }
                                                                                         : TileShape{ 16, 8, 8, 4 };
}

// pixel of thread `tid` in tile (tx, ty)
__device__ __forceinline__ void tile_pixel(const TileShape& T, int tx, int ty, int tid, int& col, int& row)
{
    const int warp = tid >> 5, lane = tid & 31;
    const int wpr = T.tw / T.ww;   // warps per tile row
    col = tx * T.tw + (warp % wpr) * T.ww + lane % T.ww;
    row = ty * T.th + (warp / wpr) * T.wh + lane / T.ww;
}

// Ray through the centre of pixel (col, row) (row 0 at the top): origin o, unit direction
// d, and its parameter interval [t0, t1] inside [0,1]^3 (slab clip, t >= 0).  False when
// the ray misses the box.
__device__ __forceinline__ bool ray_box(const RenderScalars& P, int col, int row, float (&o)[3], float (&d)[3],
                                        float& t0, float& t1)
{
    const float sx = fmaf(static_cast<float>(2 * col + 1), P.inv_w, -1.0f);
    const float sy = fmaf(static_cast<float>(-(2 * row + 1)), P.inv_h, 1.0f);
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
    t0 = 0.0f;
    t1 = INFINITY;
    bool hit = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] != 0.0f) {
            const float inv = 1.0f / d[a];
            float ta = -o[a] * inv, tb = (1.0f - o[a]) * inv;
            if (ta > tb) {
                const float t = ta;
                ta = tb;
                tb = t;
            }
            t0 = fmaxf(t0, ta);
            t1 = fminf(t1, tb);
        } else if (o[a] < 0.0f || o[a] > 1.0f) {
            hit = false;
        }
    }
    return hit && t0 < t1;
}

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

// The transfer function in shared memory: row r at tf[2r] and its forward difference
// row r+1 - row r at tf[2r + 1] (zero for the last row), so a lerp is one packed FMA per two
// channels; the difference is the same FP32 subtraction the lerp would make per sample.
// Every thread of the CTA calls it; the caller synchronises before use.
constexpr int kTfSmem = 2 * kTfMax;
__device__ __forceinline__ void stage_tf(float4* __restrict__ tf, const float4* __restrict__ src, int n)
{
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        const float4 a = src[r], b = r + 1 < n ? src[r + 1] : a;
        tf[2 * r] = a;
        tf[2 * r + 1] = make_float4(b.x - a.x, b.y - a.y, b.z - a.z, b.w - a.w);
    }
}

// Colour of one sample, without branches: transfer-function lerp and, when `shading`,
// Phong with a headlight.  The table coordinate is t = (f - vmin)/(vmax - vmin) with f the
// query's value times vscale (the cardinal path's basis scale), folded into one FMA:
// t = f vmul + vadd.
struct ShadeParams {
    float vmul, vadd, tscale, ka, kd, ks, shin, gtiny2, lx, ly, lz;
    int tf_last, shading;
#ifdef MFA_DEBUG
    unsigned* dbg;
#endif
};

__device__ __forceinline__ ShadeParams shade_params(const RenderScalars& P, const float (&d)[3], float vscale = 1.0f)
{
    ShadeParams S;
    S.vmul = P.inv_range * vscale;
    S.vadd = -P.vmin * P.inv_range;
    S.tscale = static_cast<float>(P.tf_n - 1);
    S.tf_last = max(P.tf_n - 2, 0);
    S.shading = P.shading;
    S.ka = P.ka;
    S.kd = P.kd;
    S.ks = P.ks;
    S.shin = P.shininess;
    S.gtiny2 = P.gtiny2;
    S.lx = -d[0];
    S.ly = -d[1];
    S.lz = -d[2];
#ifdef MFA_DEBUG
    S.dbg = P.dbg;
#endif
    return S;
}

__device__ __forceinline__ float4 sample_colour(const float4* __restrict__ tf, const ShadeParams& S, const float4 q)
{
    const float tt = clamp01(fmaf(q.x, S.vmul, S.vadd));
    const float xx = tt * S.tscale;
    int i0 = min(static_cast<int>(xx), S.tf_last);
    MFA_DBG_INDEX(S.dbg, i0, S.tf_last + 1, kDbgTf);   // row i0 and its difference are read
    const float wt = xx - static_cast<float>(i0);
    const float4 c0 = tf[2 * i0], dc = tf[2 * i0 + 1];
    // c = c0 + wt (c1 - c0), two channels per packed instruction
    const f2 w2 = pk2(wt, wt);
    const f2 rg = fma2(w2, pk2(dc.x, dc.y), pk2(c0.x, c0.y)), ba = fma2(w2, pk2(dc.z, dc.w), pk2(c0.z, c0.w));
    float4 c;
    upk2(rg, c.x, c.y);
    upk2(ba, c.z, c.w);
    const float g2 = q.y * q.y + q.z * q.z + q.w * q.w;
    const bool flat = g2 <= S.gtiny2;
    const float ndl = fabsf(q.y * S.lx + q.z * S.ly + q.w * S.lz) * rsqrtf(flat ? 1.0f : g2);
    const float rv = 2.0f * ndl * ndl - 1.0f;   // R.V with V = L
    float spec = rv > 0.0f ? __powf(rv, S.shin) : 0.0f;
    float factor = fmaf(S.kd, ndl, S.ka);
    factor = flat ? S.ka + S.kd : factor;
    spec = flat ? 0.0f : spec;
    const float ksp = S.ks * spec;
    if (S.shading) {
        c.x = clamp01(fmaf(c.x, factor, ksp));
        c.y = clamp01(fmaf(c.y, factor, ksp));
        c.z = clamp01(fmaf(c.z, factor, ksp));
    }
    return c;
}

// One block of the object-space decomposition (mfa_render_segments): the block grid and
// this block's index per axis.  Block (i, j, k) covers [i/g0, (i+1)/g0] x [j/g1, (j+1)/g1]
// x [k/g2, (k+1)/g2] of the unit box.
struct SegBlock {
    int g[3];
    int bi[3];
};

// The split between two neighbouring blocks along a ray: the first sample index at or past
// their common plane (ray parameter tb), clamped to 0..ns.
__device__ __forceinline__ int split_index(float tb, float t0, float dt, int ns)
{
    const float k = ceilf((tb - t0) / dt - 0.5f);
    return !(k >= 0.0f) ? 0 : (k > static_cast<float>(ns) ? ns : static_cast<int>(k));
}

// Sample index range [kb, ke) of block B on the ray (o, d) whose samples sit at
// t0 + (k + 1/2) dt.  Neighbouring blocks evaluate the same expression for their common
// plane, so the ranges of all blocks partition 0..ns-1; a face on the box boundary gives 0
// or ns, and a ray parallel to an axis's planes stays in the slab holding its origin (the
// top slab keeps the coordinate 1).
__device__ __forceinline__ void block_range(const SegBlock& B, const float (&o)[3], const float (&d)[3], float t0,
                                            float dt, int ns, int& kb, int& ke)
{
    int lo_k = 0, hi_k = ns;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float gf = static_cast<float>(B.g[a]);
        const float lo = static_cast<float>(B.bi[a]) / gf, hi = static_cast<float>(B.bi[a] + 1) / gf;
        const bool first = B.bi[a] == 0, last = B.bi[a] == B.g[a] - 1;
        int k_in, k_out;
        if (d[a] > 0.0f) {
            k_in = first ? 0 : split_index((lo - o[a]) / d[a], t0, dt, ns);
            k_out = last ? ns : split_index((hi - o[a]) / d[a], t0, dt, ns);
        } else if (d[a] < 0.0f) {
            k_in = last ? 0 : split_index((hi - o[a]) / d[a], t0, dt, ns);
            k_out = first ? ns : split_index((lo - o[a]) / d[a], t0, dt, ns);
        } else {
            const bool inside = (o[a] >= lo && o[a] < hi) || (last && o[a] == hi);
            k_in = inside ? 0 : ns;
            k_out = inside ? ns : 0;
        }
        lo_k = max(lo_k, k_in);
        hi_k = min(hi_k, k_out);
    }
    kb = lo_k;
    ke = hi_k;
}

// Software-pipelined ray march (variant 4): the query of sample k+1 is issued before the
// colour and compositing of sample k, so the two independent chains interleave in one
// basic block and the transfer-function / shading / compositing latency of one sample
// hides behind the contraction of the next.  The three span checks share one branch.
// The last iteration queries the final sample a second time (its result is not used).
// SEG: march only the samples of one block of the object-space decomposition (seg), with
// early termination on the segment's own alpha.  SKIP: empty-space skipping as in
// march_cardinal (variant 7 on models off the cardinal path).
template <int Q, int STORAGE, bool SEG = false, bool SKIP = false>
__device__ __forceinline__ float4 march_pipelined(const ModelDev& M, const RenderScalars& P,
                                                  const float4* __restrict__ tf, int col, int row,
                                                  unsigned long long& count, const SegBlock* seg = nullptr)
{
    float o[3], d[3], t0, t1;
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (!ray_box(P, col, row, o, d, t0, t1)) return acc;

    const int ns = P.n_samples;
    const float ert = P.ert_alpha;
    const float dt = (t1 - t0) / static_cast<float>(ns);
    int kb = 0, ke = ns;
    if constexpr (SEG) {
        block_range(*seg, o, d, t0, dt, ns, kb, ke);
        if (kb >= ke) return acc;
    }
    const ShadeParams S = shade_params(P, d);
    AxisCache<Q> cx, cy, cz;
    cx.s = cy.s = cz.s = -1;
    bool cell_vis = true;   // SKIP: the current cell may be visible

    auto query_at = [&](int k, bool& vis) -> float4 {
        const float t = fmaf(static_cast<float>(k) + 0.5f, dt, t0);
        const float u = clamp01(fmaf(t, d[0], o[0]));
        const float v = clamp01(fmaf(t, d[1], o[1]));
        const float w = clamp01(fmaf(t, d[2], o[2]));
        const bool ox = !(cx.s >= 0 && u >= cx.rec[2] && u < cx.rec[3]);
        const bool oy = !(cy.s >= 0 && v >= cy.rec[2] && v < cy.rec[3]);
        const bool oz = !(cz.s >= 0 && w >= cz.rec[2] && w < cz.rec[3]);
        if (ox | oy | oz) {
            if (ox) axis_update<Q>(M.ax[0], cx, u);
            if (oy) axis_update<Q>(M.ax[1], cy, v);
            if (oz) axis_update<Q>(M.ax[2], cz, w);
            if constexpr (SKIP) {
                int ci = ((cz.s - M.ax[2].p) * M.ncy + (cy.s - M.ax[1].p)) * M.ncx + (cx.s - M.ax[0].p);
                MFA_DBG_INDEX(P.dbg, ci, static_cast<long long>(M.ncx) * M.ncy * M.ncz, kDbgCell);
                cell_vis = (__ldg(P.cell_vis + (ci >> 5)) >> (ci & 31)) & 1u;
            }
        }
        vis = cell_vis;
        if constexpr (SKIP) {
            if (!cell_vis) return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
        float Ny[Q], Dy[Q], Nz[Q], Dz[Q];
        const XIn<Q, STORAGE> X = xin_record<Q, STORAGE>(cx.rec, u);
        record_basis<Q>(cy.rec, v, Ny, Dy);
        record_basis<Q>(cz.rec, w, Nz, Dz);
        float4 q = contract<Q, STORAGE>(M, cx.s - M.ax[0].p, cy.s - M.ax[1].p, cz.s - M.ax[2].p, X, Ny, Dy, Nz, Dz);
        q.y *= cx.rec[1];
        q.z *= cy.rec[1];
        q.w *= cz.rec[1];
        return q;
    };

    bool v, vn;
    float4 q = query_at(kb, v);
    for (int k = kb; k < ke; ++k) {
        const float4 qn = query_at(min(k + 1, ke - 1), vn);
        if (!SKIP || v) {
            const float4 c = sample_colour(tf, S, q);
            const float wgt = (1.0f - acc.w) * c.w;
            acc.x = fmaf(wgt, c.x, acc.x);
            acc.y = fmaf(wgt, c.y, acc.y);
            acc.z = fmaf(wgt, c.z, acc.z);
            acc.w += wgt;
            ++count;
        }
        if (acc.w >= ert) break;
        q = qn;
        v = vn;
    }
    return acc;
}

// ----------------------------------------------------------------------------------------
// variant 6: uniform knots (cardinal basis)
// ----------------------------------------------------------------------------------------
//
// For a model with clamped uniform knots and degree Q-1 on all three axes (ModelDev::
// cardinal), every span but the p-1 at each end of an axis carries the same basis
// polynomials (cardinal_basis).  The ray is marched in span units x = (n - p) u, so the
// span is j = floor(x) and its local coordinate t = x - j; the per-axis state is the span
// index alone (no record in registers).  For degree classes 2..4 the support itself (its
// window rows) is kept in registers until a span changes, so a ray reads the window once
// per knot-span cell it crosses rather than once per sample (on the 128^3 frame a warp
// reloads at about one sample in four); the sums are the ones contract_at forms from the
// same rows.
// The end spans, whose functions see the repeated end knots, read their record from
// global memory (L1-resident, a few hundred bytes per axis) for each sample.
// Software-pipelined like variant 4.  (The record path, variant 4, keeps no such cache:
// with its three span records also in registers it needs two CTAs' budget or spills, and
// its own workload, the 512x512x256 non-uniform model at 2048 samples, has about one
// sample per cell: measured 25.1 ms without, 25.7 ms with.)
//
// SKIP (variant 7, empty-space skipping): P.cell_vis marks the knot-span cells whose value
// range (the convex hull bound of their support) reaches a transfer-function row of
// non-zero opacity.  A sample in an unmarked cell would composite with alpha exactly 0 and
// change nothing, so it is neither queried nor composited; the image equals variant 6's
// up to FP32 rounding order (the two instantiations may fuse multiply-adds differently)
// and only evaluated samples are counted.
template <int Q, int STORAGE, bool SEG = false, bool SKIP = false>
__device__ __forceinline__ float4 march_cardinal(const ModelDev& M, const RenderScalars& P,
                                                 const float4* __restrict__ tf, int col, int row,
                                                 unsigned long long& count, const SegBlock* seg = nullptr)
{
    float o[3], d[3], t0, t1;
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (!ray_box(P, col, row, o, d, t0, t1)) return acc;

    const int ns = P.n_samples;
    const float ert = P.ert_alpha;
    const float dt = (t1 - t0) / static_cast<float>(ns);
    int kb = 0, ke = ns;
    if constexpr (SEG) {
        block_range(*seg, o, d, t0, dt, ns, kb, ke);
        if (kb >= ke) return acc;
    }
    const ShadeParams S = shade_params(P, d, Cardinal<Q>::template val_scale<STORAGE>());
    float om[3], dm[3], gs[3];   // ray in span units, gradient scale per axis
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float m = static_cast<float>(M.ax[a].n - M.ax[a].p);
        om[a] = o[a] * m;
        dm[a] = d[a] * m;
        gs[a] = m * (a == 0 ? Cardinal<Q>::template gradx_scale<STORAGE>() : Cardinal<Q>::template gradyz_scale<STORAGE>());
    }
    CardAxis cx{ -INFINITY, 0, false }, cy{ -INFINITY, 0, false }, cz{ -INFINITY, 0, false };
    int base = 0;
    bool cell_vis = true;   // SKIP: the current cell may be visible
    // the support of the current cell, in registers (degree classes 2..4; degree class 5's
    // would take 180 registers): consecutive samples in one cell reuse it, so the window is
    // read once per cell a ray visits instead of once per sample.  Not with skipping, whose
    // rays query few of the cells they cross (the registers cost more than they save there).
    constexpr bool CACHE = Q <= 4 && !SKIP;
    SupportRegs<Q> sup;

    auto query_at = [&](int k, bool& vis) -> float4 {
        const float t = fmaf(static_cast<float>(k) + 0.5f, dt, t0);
        const float x = fmaf(t, dm[0], om[0]);
        const float y = fmaf(t, dm[1], om[1]);
        const float z = fmaf(t, dm[2], om[2]);
        float tx = x - cx.jf, ty = y - cy.jf, tz = z - cz.jf;
        const bool ox = !(tx >= 0.0f && tx < 1.0f);
        const bool oy = !(ty >= 0.0f && ty < 1.0f);
        const bool oz = !(tz >= 0.0f && tz < 1.0f);
        if (ox | oy | oz) {
            if (ox) {
                card_update(M.ax[0], cx, x);
                tx = x - cx.jf;
            }
            if (oy) {
                card_update(M.ax[1], cy, y);
                ty = y - cy.jf;
            }
            if (oz) {
                card_update(M.ax[2], cz, z);
                tz = z - cz.jf;
            }
            base = (cz.j * M.nyp + cy.j) * M.nxp + cx.j;
            if constexpr (SKIP) {
                int ci = (cz.j * M.ncy + cy.j) * M.ncx + cx.j;
                MFA_DBG_INDEX(P.dbg, ci, static_cast<long long>(M.ncx) * M.ncy * M.ncz, kDbgCell);
                cell_vis = (__ldg(P.cell_vis + (ci >> 5)) >> (ci & 31)) & 1u;
            }
            if constexpr (CACHE) load_support<Q, STORAGE>(M, base, sup);
        }
        vis = cell_vis;
        if constexpr (SKIP) {
            if (!cell_vis) return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
        float Ny[Q], Dy[Q], Nz[Q], Dz[Q];
        XIn<Q, STORAGE> X;
        if (card_edge<Q, STORAGE>(cx, cy, cz)) {
            X = xin_card<Q, STORAGE>(M.ax[0], cx, tx);
            card_basis<Q>(M.ax[1], cy, ty, Ny, Dy);
            card_basis<Q>(M.ax[2], cz, tz, Nz, Dz);
        } else {
            X = xin_cardinal<Q, STORAGE>(tx);
            cardinal_basis<Q>(ty, Ny, Dy);
            cardinal_basis<Q>(tz, Nz, Dz);
        }
        float4 q;   // value left unscaled (S.vmul)
        if constexpr (CACHE)
            q = contract_support<Q, STORAGE>(sup, X, Ny, Dy, Nz, Dz);
        else
            q = contract_at<Q, STORAGE>(M, base, X, Ny, Dy, Nz, Dz);
        q.y *= gs[0];
        q.z *= gs[1];
        q.w *= gs[2];
        return q;
    };

    bool v, vn;
    float4 q = query_at(kb, v);
    int k = kb;   // next sample to composite
    int evaluated = 0;
    while (k < ke) {
        const float4 qn = query_at(min(k + 1, ke - 1), vn);
        if (!SKIP || v) {
            const float4 c = sample_colour(tf, S, q);
            const float wgt = (1.0f - acc.w) * c.w;
            acc.x = fmaf(wgt, c.x, acc.x);
            acc.y = fmaf(wgt, c.y, acc.y);
            acc.z = fmaf(wgt, c.z, acc.z);
            acc.w += wgt;
            ++evaluated;
        }
        ++k;
        if (acc.w >= ert) break;
        q = qn;
        v = vn;
    }
    count += static_cast<unsigned>(SKIP ? evaluated : k - kb);
    return acc;
}

// ----------------------------------------------------------------------------------------
// variant 8: per-cell polynomial patches (MFA_WINDOW_PATCH models)
// ----------------------------------------------------------------------------------------
//
// On a degree-3 model with uniform knots, the model restricted to knot-span cell (i, j, k) is
// one tricubic polynomial in the cell's local coordinates (t_x, t_y, t_z) in [0,1)^3:
// f = sum c[a][b][c] t_x^a t_y^b t_z^c, whose 64 coefficients ModelDev::patch holds (from the
// span coefficients of each axis, end spans included).  The march is the cardinal one with
// the cell's patch in registers in place of its window rows, and monomials in place of the
// basis: the contraction runs the same packed passes with y weights {1, t, t^2, t^3} and
// derivative weights {0, 1, 2t, 3t^2} (likewise z), and the x-pass is the Horner sweep of
// the power rows.  No span records, no end-span branch and no basis evaluation per sample.
template <int STORAGE>
__device__ __forceinline__ float4 march_patch(const ModelDev& M, const RenderScalars& P,
                                              const float4* __restrict__ tf, int col, int row,
                                              unsigned long long& count)
{
    static_assert(STORAGE == 1, "patches are FP32");
    float o[3], d[3], t0, t1;
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (!ray_box(P, col, row, o, d, t0, t1)) return acc;

    const int ns = P.n_samples;
    const float ert = P.ert_alpha;
    const float dt = (t1 - t0) / static_cast<float>(ns);
    const ShadeParams S = shade_params(P, d, 1.0f);
    float om[3], dm[3], gs[3];   // ray in span units, gradient scale per axis
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float m = static_cast<float>(M.ax[a].n - M.ax[a].p);
        om[a] = o[a] * m;
        dm[a] = d[a] * m;
        gs[a] = m;
    }
    CardAxis cx{ -INFINITY, 0, false }, cy{ -INFINITY, 0, false }, cz{ -INFINITY, 0, false };
    SupportRegs<4> sup;

    auto query_at = [&](int k) -> float4 {
        const float t = fmaf(static_cast<float>(k) + 0.5f, dt, t0);
        const float x = fmaf(t, dm[0], om[0]);
        const float y = fmaf(t, dm[1], om[1]);
        const float z = fmaf(t, dm[2], om[2]);
        float tx = x - cx.jf, ty = y - cy.jf, tz = z - cz.jf;
        const bool ox = !(tx >= 0.0f && tx < 1.0f);
        const bool oy = !(ty >= 0.0f && ty < 1.0f);
        const bool oz = !(tz >= 0.0f && tz < 1.0f);
        if (ox | oy | oz) {
            if (ox) {
                card_update(M.ax[0], cx, x);
                tx = x - cx.jf;
            }
            if (oy) {
                card_update(M.ax[1], cy, y);
                ty = y - cy.jf;
            }
            if (oz) {
                card_update(M.ax[2], cz, z);
                tz = z - cz.jf;
            }
            int cell = (cz.j * M.ncy + cy.j) * M.ncx + cx.j;
            MFA_DBG_INDEX(M.dbg, cell, static_cast<long long>(M.ncx) * M.ncy * M.ncz, kDbgWindow);
            const float* e = M.patch + static_cast<long long>(cell) * 64;
#pragma unroll
            for (int m = 0; m < 2; ++m)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    f2 (&pr)[4] = sup.r[m][b];
                    asm("ld.global.nc.v4.b64 {%0, %1, %2, %3}, [%4];"
                        : "=l"(pr[0].v), "=l"(pr[1].v), "=l"(pr[2].v), "=l"(pr[3].v)
                        : "l"(e + (4 * m + b) * 8));
                }
        }
        const float ty2 = ty * ty, tz2 = tz * tz;
        const float Ny[4] = { 1.0f, ty, ty2, ty2 * ty }, Dy[4] = { 0.0f, 1.0f, 2.0f * ty, 3.0f * ty2 };
        const float Nz[4] = { 1.0f, tz, tz2, tz2 * tz }, Dz[4] = { 0.0f, 1.0f, 2.0f * tz, 3.0f * tz2 };
        float4 q = contract_support<4, STORAGE>(sup, xin_t<4>(tx), Ny, Dy, Nz, Dz);
        q.y *= gs[0];
        q.z *= gs[1];
        q.w *= gs[2];
        return q;
    };

    float4 q = query_at(0);
    int k = 0;
    while (k < ns) {
        const float4 qn = query_at(min(k + 1, ns - 1));
        const float4 c = sample_colour(tf, S, q);
        const float wgt = (1.0f - acc.w) * c.w;
        acc.x = fmaf(wgt, c.x, acc.x);
        acc.y = fmaf(wgt, c.y, acc.y);
        acc.z = fmaf(wgt, c.z, acc.z);
        acc.w += wgt;
        ++k;
        if (acc.w >= ert) break;
        q = qn;
    }
    count += static_cast<unsigned>(k);
    return acc;
}

// Variant 8 on a model with non-uniform knots: the same patch march with each axis's span
// tracked through its records, of which it reads the head only: the span's first knot U_s,
// 1/h and its FP32 bounds [lo, hi).  The cell's local coordinate is t = (u - U_s)/h, the
// coordinate its patch coefficients are in, and d/du = (1/h) d/dt.
struct PatchAxis {
    int s;                  // knot span (p .. n-1), -1 before the first sample
    float u0, ih, lo, hi;   // the record head
};

__device__ __forceinline__ void patch_axis_update(const AxisDev& A, PatchAxis& C, float u)
{
    if (C.s >= 0 && u >= C.lo && u < C.hi) return;
    int s = C.s < 0 ? locate_span(A, u) : walk_span(A, u, C.s);
    int r = s - A.p;
    MFA_DBG_INDEX(A.dbg, r, A.n - A.p, kDbgRecord);
    const float4 h = __ldg(reinterpret_cast<const float4*>(A.rec + static_cast<long long>(r) * rec_stride(4)));
    C.s = s;
    C.u0 = h.x;
    C.ih = h.y;
    C.lo = h.z;
    C.hi = h.w;
}

template <int STORAGE>
__device__ __forceinline__ float4 march_patch_records(const ModelDev& M, const RenderScalars& P,
                                                      const float4* __restrict__ tf, int col, int row,
                                                      unsigned long long& count)
{
    static_assert(STORAGE == 1, "patches are FP32");
    float o[3], d[3], t0, t1;
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (!ray_box(P, col, row, o, d, t0, t1)) return acc;

    const int ns = P.n_samples;
    const float ert = P.ert_alpha;
    const float dt = (t1 - t0) / static_cast<float>(ns);
    const ShadeParams S = shade_params(P, d, 1.0f);
    PatchAxis cx{ -1, 0.0f, 0.0f, 0.0f, 0.0f }, cy = cx, cz = cx;
    SupportRegs<4> sup;

    auto query_at = [&](int k) -> float4 {
        const float t = fmaf(static_cast<float>(k) + 0.5f, dt, t0);
        const float u = clamp01(fmaf(t, d[0], o[0]));
        const float v = clamp01(fmaf(t, d[1], o[1]));
        const float w = clamp01(fmaf(t, d[2], o[2]));
        const bool ox = !(cx.s >= 0 && u >= cx.lo && u < cx.hi);
        const bool oy = !(cy.s >= 0 && v >= cy.lo && v < cy.hi);
        const bool oz = !(cz.s >= 0 && w >= cz.lo && w < cz.hi);
        if (ox | oy | oz) {
            if (ox) patch_axis_update(M.ax[0], cx, u);
            if (oy) patch_axis_update(M.ax[1], cy, v);
            if (oz) patch_axis_update(M.ax[2], cz, w);
            int cell = ((cz.s - 3) * M.ncy + (cy.s - 3)) * M.ncx + (cx.s - 3);
            MFA_DBG_INDEX(M.dbg, cell, static_cast<long long>(M.ncx) * M.ncy * M.ncz, kDbgWindow);
            const float* e = M.patch + static_cast<long long>(cell) * 64;
#pragma unroll
            for (int m = 0; m < 2; ++m)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    f2 (&pr)[4] = sup.r[m][b];
                    asm("ld.global.nc.v4.b64 {%0, %1, %2, %3}, [%4];"
                        : "=l"(pr[0].v), "=l"(pr[1].v), "=l"(pr[2].v), "=l"(pr[3].v)
                        : "l"(e + (4 * m + b) * 8));
                }
        }
        const float tx = (u - cx.u0) * cx.ih, ty = (v - cy.u0) * cy.ih, tz = (w - cz.u0) * cz.ih;
        const float ty2 = ty * ty, tz2 = tz * tz;
        const float Ny[4] = { 1.0f, ty, ty2, ty2 * ty }, Dy[4] = { 0.0f, 1.0f, 2.0f * ty, 3.0f * ty2 };
        const float Nz[4] = { 1.0f, tz, tz2, tz2 * tz }, Dz[4] = { 0.0f, 1.0f, 2.0f * tz, 3.0f * tz2 };
        float4 q = contract_support<4, STORAGE>(sup, xin_t<4>(tx), Ny, Dy, Nz, Dz);
        q.y *= cx.ih;
        q.z *= cy.ih;
        q.w *= cz.ih;
        return q;
    };

    float4 q = query_at(0);
    int k = 0;
    while (k < ns) {
        const float4 qn = query_at(min(k + 1, ns - 1));
        const float4 c = sample_colour(tf, S, q);
        const float wgt = (1.0f - acc.w) * c.w;
        acc.x = fmaf(wgt, c.x, acc.x);
        acc.y = fmaf(wgt, c.y, acc.y);
        acc.z = fmaf(wgt, c.z, acc.z);
        acc.w += wgt;
        ++k;
        if (acc.w >= ert) break;
        q = qn;
    }
    count += static_cast<unsigned>(k);
    return acc;
}

__device__ __forceinline__ void add_count(unsigned long long* dst, unsigned long long count)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) count += __shfl_xor_sync(0xFFFFFFFFu, count, o);
    if ((threadIdx.x & 31) == 0 && count) atomicAdd(dst, count);
}

}  // namespace mfa
