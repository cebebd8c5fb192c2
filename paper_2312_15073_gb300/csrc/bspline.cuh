// bspline.cuh -- device building blocks of one MFA value+gradient query (Sec. III-B,
// Sec. V-D.3): knot-span location per axis, basis values and derivatives on the span,
// and the (p+1)^3 control-point contraction for the value and the three partials.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "mfa_internal.cuh"

namespace mfa {

// Knot span of u (u already clamped to [0,1]): the largest s in [p, n-1] with
// U[s] <= u.  kup holds the knots rounded up to FP32, so the FP32 comparisons below give
// exactly the answer of the FP64 comparisons on the FP32 value of u.  The grid supplies
// a starting span; the two walks fix it up (at most a few steps: G = 4 (n - p) cells).
__device__ __forceinline__ int locate_span(const AxisDev& A, float u)
{
    int g = min(static_cast<int>(u * A.Gf), A.G - 1);
    int s = __ldg(A.grid + g);
    while (s < A.n - 1 && u >= __ldg(A.kup + s + 1)) ++s;
    while (s > A.p && u < __ldg(A.kup + s)) --s;
    return s;
}

// Same, starting from a previous span (a ray's last sample): u moves monotonically along
// an axis, so this is usually zero or one step.
__device__ __forceinline__ int walk_span(const AxisDev& A, float u, int s)
{
    while (s < A.n - 1 && u >= __ldg(A.kup + s + 1)) ++s;
    while (s > A.p && u < __ldg(A.kup + s)) --s;
    return s;
}

// The Q basis functions N_{s-p+r,p} on span s (zero for r > p) and their derivatives
// with respect to the local coordinate t = (u - U_s)/h, by joint Horner evaluation of
// the span's power-basis coefficients.  inv_h receives 1/h (d/du = inv_h d/dt).
template <int Q>
__device__ __forceinline__ void span_basis(const AxisDev& A, int s, float u, float (&N)[Q], float (&D)[Q],
                                           float& inv_h)
{
    constexpr int RS = rec_stride(Q);
    const float4* r4 = reinterpret_cast<const float4*>(A.rec + (s - A.p) * RS);
    float rec[RS];
#pragma unroll
    for (int v = 0; v < RS / 4; ++v) {
        float4 x = __ldg(r4 + v);
        rec[4 * v + 0] = x.x;
        rec[4 * v + 1] = x.y;
        rec[4 * v + 2] = x.z;
        rec[4 * v + 3] = x.w;
    }
    inv_h = rec[1];
    const float t = (u - rec[0]) * inv_h;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float* c = rec + 2 + i * Q;
        float b = c[Q - 1], d = 0.0f;
#pragma unroll
        for (int k = Q - 2; k >= 0; --k) {
            d = fmaf(d, t, b);
            b = fmaf(b, t, c[k]);
        }
        N[i] = b;
        D[i] = d;
    }
}

// One x-row of the support: Q consecutive control points as FP32.
template <int Q, int STORAGE>
__device__ __forceinline__ void load_row(const void* win, int idx, float (&row)[Q]);

template <int Q>
struct RowF32 {
    static __device__ __forceinline__ void load(const void* win, int idx, float (&row)[Q])
    {
        const float4* W = static_cast<const float4*>(win);
        float4 v = __ldg(W + idx);
        float tmp[4] = { v.x, v.y, v.z, v.w };
#pragma unroll
        for (int a = 0; a < Q && a < 4; ++a) row[a] = tmp[a];
        if constexpr (Q == 5) row[4] = __ldg(reinterpret_cast<const float*>(W + idx + 4));
    }
};

template <int Q, bool BF16>
struct Row16 {
    static __device__ __forceinline__ float2 cvt(unsigned int bits)
    {
        if constexpr (BF16) {
            __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&bits);
            return __bfloat1622float2(h);
        } else {
            __half2 h = *reinterpret_cast<__half2*>(&bits);
            return __half22float2(h);
        }
    }
    static __device__ __forceinline__ void load(const void* win, int idx, float (&row)[Q])
    {
        const uint2* W = static_cast<const uint2*>(win);
        uint2 v = __ldg(W + idx);
        float2 lo = cvt(v.x), hi = cvt(v.y);
        float tmp[4] = { lo.x, lo.y, hi.x, hi.y };
#pragma unroll
        for (int a = 0; a < Q && a < 4; ++a) row[a] = tmp[a];
        if constexpr (Q == 5) {
            unsigned int b = __ldg(reinterpret_cast<const unsigned int*>(W + idx + 4));
            row[4] = cvt(b).x;
        }
    }
};

template <int Q, int STORAGE>
struct RowLoader;
template <int Q> struct RowLoader<Q, 1> : RowF32<Q> {};          // MFA_F32
template <int Q> struct RowLoader<Q, 2> : Row16<Q, false> {};    // MFA_F16
template <int Q> struct RowLoader<Q, 3> : Row16<Q, true> {};     // MFA_BF16

// Sum-factorised contraction over the Q^3 support starting at (i0, j0, k0):
//   x-pass  A_jk = sum_i Nx_i P_ijk,  B_jk = sum_i Dx_i P_ijk          (2 Q^3 FMA)
//   y-pass  C_k = sum_j Ny_j A_jk, Dk = sum_j Dy_j A_jk, E_k = sum_j Ny_j B_jk   (3 Q^2)
//   z-pass  f = sum_k Nz_k C_k, f_z = sum Dz_k C_k, f_y = sum Nz_k D_k, f_x = sum Nz_k E_k
// Returns {f, df/dtx, df/dty, df/dtz} (derivatives in the local span coordinates).
template <int Q, int STORAGE>
__device__ __forceinline__ float4 contract(const ModelDev& M, int i0, int j0, int k0, const float (&Nx)[Q],
                                           const float (&Dx)[Q], const float (&Ny)[Q], const float (&Dy)[Q],
                                           const float (&Nz)[Q], const float (&Dz)[Q])
{
    const int plane = M.nxp * M.nyp;
    const int base = (k0 * M.nyp + j0) * M.nxp + i0;
    float f = 0.0f, fx = 0.0f, fy = 0.0f, fz = 0.0f;
#pragma unroll
    for (int c = 0; c < Q; ++c) {
        float C = 0.0f, Dv = 0.0f, E = 0.0f;
#pragma unroll
        for (int b = 0; b < Q; ++b) {
            float row[Q];
            RowLoader<Q, STORAGE>::load(M.win, base + c * plane + b * M.nxp, row);
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

// Full query at a clamped parameter point: value and world gradient (unit-cube domain,
// so the chain-rule factor to world coordinates is 1; 1/h converts d/dt to d/du).
template <int Q, int STORAGE>
__device__ __forceinline__ float4 query(const ModelDev& M, float u, float v, float w, int sx, int sy, int sz)
{
    float Nx[Q], Dx[Q], Ny[Q], Dy[Q], Nz[Q], Dz[Q], hx, hy, hz;
    span_basis<Q>(M.ax[0], sx, u, Nx, Dx, hx);
    span_basis<Q>(M.ax[1], sy, v, Ny, Dy, hy);
    span_basis<Q>(M.ax[2], sz, w, Nz, Dz, hz);
    float4 r = contract<Q, STORAGE>(M, sx - M.ax[0].p, sy - M.ax[1].p, sz - M.ax[2].p, Nx, Dx, Ny, Dy, Nz, Dz);
    r.y *= hx;
    r.z *= hy;
    r.w *= hz;
    return r;
}

__device__ __forceinline__ float clamp01(float x) { return fminf(fmaxf(x, 0.0f), 1.0f); }

}  // namespace mfa
