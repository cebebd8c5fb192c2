// prep.cu -- model preparation kernels (run once per mfa_model_create).
//
// Turns the uploaded FP64 knots and input-dtype control points into the tables the query
// kernels read (layout in mfa_internal.cuh): knots rounded up to FP32, the span-start
// grid, per-span power-basis records, the layer-pair window array in the storage dtype, and
// the min / max / max-abs of the stored control points.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "mfa_internal.cuh"

namespace mfa {
namespace {

// ----------------------------------------------------------------------------------------
// per-axis tables
// ----------------------------------------------------------------------------------------

__global__ void k_knots_up(const double* __restrict__ U, int m, float* __restrict__ kup)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) kup[i] = __double2float_ru(U[i]);
}

// grid[g] = largest s in [p, n-1] with U[s] <= g/G (FP64 binary search)
__global__ void k_span_grid(const double* __restrict__ U, int n, int p, int G, int* __restrict__ grid)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    double x = static_cast<double>(g) / static_cast<double>(G);
    int lo = p, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (U[mid] <= x) lo = mid; else hi = mid - 1;
    }
    grid[g] = lo;
}

__device__ double safe_div(double a, double b) { return b != 0.0 ? a / b : 0.0; }

// One record per span s in [p, n-1]: the Cox-de Boor recursion carried out on polynomials
// in the local coordinate t (u = U_s + h t), in FP64.  Level k holds N_{s-k+r,k}, r=0..k, as
// coefficient vectors; each level multiplies the previous one by the linear factors
// (u - U_i)/(U_{i+k} - U_i) and (U_{i+k+1} - u)/(U_{i+k+1} - U_{i+1}) written in t.
template <int Q>
__global__ void k_span_records(const double* __restrict__ U, int n, int p, float* __restrict__ rec)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n - p) return;
    const int s = p + idx;
    constexpr int RS = rec_stride(Q);
    float* out = rec + idx * RS;
    const double Us = U[s], h = U[s + 1] - U[s];
    double T[Q][Q];       // T[r][k]: coefficient of t^k of the r-th function of the level
    double Tn[Q][Q];
    for (int r = 0; r < Q; ++r)
        for (int k = 0; k < Q; ++k) T[r][k] = 0.0;
    T[0][0] = 1.0;
    for (int lev = 1; lev <= p; ++lev) {
        for (int r = 0; r <= lev; ++r) {
            const int i = s - lev + r;
            // lower = N_{i,lev-1} = T[r-1], upper = N_{i+1,lev-1} = T[r]
            const double da = U[i + lev] - U[i];
            const double a0 = safe_div(Us - U[i], da), a1 = safe_div(h, da);
            const double db = U[i + lev + 1] - U[i + 1];
            const double b0 = safe_div(U[i + lev + 1] - Us, db), b1 = safe_div(-h, db);
            for (int k = 0; k < Q; ++k) {
                double acc = 0.0;
                if (r >= 1) {
                    acc += a0 * T[r - 1][k];
                    if (k >= 1) acc += a1 * T[r - 1][k - 1];
                }
                if (r <= lev - 1) {
                    acc += b0 * T[r][k];
                    if (k >= 1) acc += b1 * T[r][k - 1];
                }
                Tn[r][k] = acc;
            }
        }
        for (int r = 0; r <= lev; ++r)
            for (int k = 0; k < Q; ++k) T[r][k] = Tn[r][k];
    }
    constexpr int QP = qpair(Q);
    out[0] = __double2float_rn(Us);
    out[1] = h > 0.0 ? __double2float_rn(1.0 / h) : 0.0f;
    out[2] = __double2float_ru(Us);
    out[3] = s < n - 1 ? __double2float_ru(U[s + 1]) : INFINITY;
    for (int k = 0; k < Q; ++k)
        for (int r = 0; r < QP; ++r)
            out[kRecHead + k * QP + r] = (r <= p && r < Q) ? __double2float_rn(T[r][k]) : 0.0f;
    for (int e = kRecHead + Q * QP; e < RS; ++e) out[e] = 0.0f;
}

// ----------------------------------------------------------------------------------------
// control points
// ----------------------------------------------------------------------------------------

// Input element -> FP64 (exact for every input type).
__device__ __forceinline__ double load_in(const void* p, int dtype, long long i)
{
    switch (dtype) {
    case 0: return static_cast<const double*>(p)[i];
    case 1: return static_cast<double>(static_cast<const float*>(p)[i]);
    case 2: return static_cast<double>(__half2float(static_cast<const __half*>(p)[i]));
    default: return static_cast<double>(__bfloat162float(static_cast<const __nv_bfloat16*>(p)[i]));
    }
}

// One round-to-nearest-even step from the exact input value to the storage type.
__device__ __forceinline__ unsigned short to16(double x, int storage)
{
    if (storage == 2) return __half_as_ushort(__double2half(x));
    return __bfloat16_as_ushort(__double2bfloat16(x));
}

// The layer-pair window array (layout in mfa_internal.cuh), one entry per thread.
__global__ void k_window(const void* __restrict__ ctrl, int in_dtype, int storage, int nx, int ny, int nz, int q,
                         void* __restrict__ win)
{
    const int nxp = nx + kPad, nyp = ny + kPad, nzp = nz + kPad;
    const long long total = static_cast<long long>(nxp) * nyp * nzp;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int i = static_cast<int>(e % nxp);
        const long long jk = e / nxp;
        const int j = static_cast<int>(jk % nyp);
        const int k = static_cast<int>(jk / nyp);
        // v[2a + r] = P[k + r][j][i + a]; for q == 3 also v[8 + a] = P[k + 2][j][i + a], then zeros
        double v[16];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const int ia = i + a, kr = k + r;
                const double x = (ia < nx && j < ny && kr < nz)
                                     ? load_in(ctrl, in_dtype, (static_cast<long long>(kr) * ny + j) * nx + ia)
                                     : 0.0;
                if (r < 2) v[2 * a + r] = x; else v[8 + a] = x;
            }
            v[12 + a] = 0.0;
        }
        const int nv = window_values(q);
        if (storage == 1) {
            float4* w = static_cast<float4*>(win) + (nv / 4) * e;
            for (int c = 0; c < nv / 4; ++c)
                w[c] = make_float4(__double2float_rn(v[4 * c]), __double2float_rn(v[4 * c + 1]),
                                   __double2float_rn(v[4 * c + 2]), __double2float_rn(v[4 * c + 3]));
        } else {
            uint4* w = static_cast<uint4*>(win) + (nv / 8) * e;
            for (int c = 0; c < nv / 8; ++c) {
                unsigned int b[4];
#pragma unroll
                for (int a = 0; a < 4; ++a)
                    b[a] = static_cast<unsigned>(to16(v[8 * c + 2 * a], storage)) |
                           (static_cast<unsigned>(to16(v[8 * c + 2 * a + 1], storage)) << 16);
                w[c] = make_uint4(b[0], b[1], b[2], b[3]);
            }
        }
    }
}

// {min, max} over the (p_x+1)(p_y+1)(p_z+1) stored control points of each knot-span cell's
// support, read from the window array (element 0 of entry (k, j, i) is P[k][j][i]).
__global__ void k_cell_range(const void* __restrict__ win, int storage, int nv, int px, int py, int pz, int ncx,
                             int ncy, int ncz, int nxp, int nyp, float2* __restrict__ cell)
{
    const long long total = static_cast<long long>(ncx) * ncy * ncz;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int i0 = static_cast<int>(e % ncx);
        const long long jk = e / ncx;
        const int j0 = static_cast<int>(jk % ncy), k0 = static_cast<int>(jk / ncy);
        float mn = INFINITY, mx = -INFINITY;
        for (int c = 0; c <= pz; ++c)
            for (int b = 0; b <= py; ++b)
                for (int a = 0; a <= px; ++a) {
                    const long long w = (static_cast<long long>(k0 + c) * nyp + (j0 + b)) * nxp + (i0 + a);
                    float v;
                    if (storage == 1) {
                        v = static_cast<const float*>(win)[nv * w];
                    } else {
                        const unsigned short h = static_cast<const unsigned short*>(win)[nv * w];
                        v = storage == 2 ? __half2float(__ushort_as_half(h)) : __bfloat162float(__ushort_as_bfloat16(h));
                    }
                    mn = fminf(mn, v);
                    mx = fmaxf(mx, v);
                }
        cell[e] = make_float2(mn, mx);
    }
}

// order-preserving float <-> int map for atomicMin / atomicMax
__device__ __forceinline__ int f2ord(float f)
{
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7FFFFFFF;
}

__global__ void k_stats_init(int* stats)
{
    stats[0] = f2ord(INFINITY);
    stats[1] = f2ord(-INFINITY);
    stats[2] = f2ord(0.0f);
}

// min, max and max |P| over the stored values (first element of each window entry in the
// unpadded region)
__global__ void k_stats(const void* __restrict__ win, int storage, int nx, int ny, int nz, int q,
                        int* __restrict__ stats)
{
    const int nxp = nx + kPad, nyp = ny + kPad;
    const long long nv = window_values(q);
    const long long total = static_cast<long long>(nx) * ny * nz;
    float mn = INFINITY, mx = -INFINITY, ma = 0.0f;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int i = static_cast<int>(e % nx);
        const long long jk = e / nx;
        const int j = static_cast<int>(jk % ny);
        const int k = static_cast<int>(jk / ny);
        const long long w = (static_cast<long long>(k) * nyp + j) * nxp + i;
        float v;
        if (storage == 1) {
            v = static_cast<const float*>(win)[nv * w];
        } else {
            const unsigned short b = static_cast<const unsigned short*>(win)[nv * w];
            v = storage == 2 ? __half2float(__ushort_as_half(b)) : __bfloat162float(__ushort_as_bfloat16(b));
        }
        mn = fminf(mn, v);
        mx = fmaxf(mx, v);
        ma = fmaxf(ma, fabsf(v));
    }
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
        ma = fmaxf(ma, __shfl_xor_sync(0xFFFFFFFFu, ma, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&stats[0], f2ord(mn));
        atomicMax(&stats[1], f2ord(mx));
        atomicMax(&stats[2], f2ord(ma));
    }
}

}  // namespace

cudaError_t launch_prep_axis(const double* d_knots, int n, int p, int q, float* kup, float* rec, int* grid, int G,
                             cudaStream_t stream)
{
    const int m = n + p + 1;
    k_knots_up<<<(m + 255) / 256, 256, 0, stream>>>(d_knots, m, kup);
    k_span_grid<<<(G + 255) / 256, 256, 0, stream>>>(d_knots, n, p, G, grid);
    const int spans = n - p;
    const int blocks = (spans + 127) / 128;
    switch (q) {
    case 2: k_span_records<2><<<blocks, 128, 0, stream>>>(d_knots, n, p, rec); break;
    case 3: k_span_records<3><<<blocks, 128, 0, stream>>>(d_knots, n, p, rec); break;
    case 4: k_span_records<4><<<blocks, 128, 0, stream>>>(d_knots, n, p, rec); break;
    case 5: k_span_records<5><<<blocks, 128, 0, stream>>>(d_knots, n, p, rec); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_prep_window(const void* d_ctrl, int in_dtype, int storage, int nx, int ny, int nz, int q,
                               void* win, cudaStream_t stream)
{
    const long long total = static_cast<long long>(nx + kPad) * (ny + kPad) * (nz + kPad);
    const long long want = (total + 255) / 256;
    const int blocks = static_cast<int>(want < 65536 ? want : 65536);
    k_window<<<blocks, 256, 0, stream>>>(d_ctrl, in_dtype, storage, nx, ny, nz, q, win);
    return cudaGetLastError();
}

cudaError_t launch_prep_cells(const void* win, int storage, int q, const int degree[3], const int nctrl[3],
                              float2* cell, cudaStream_t stream)
{
    const int ncx = nctrl[0] - degree[0], ncy = nctrl[1] - degree[1], ncz = nctrl[2] - degree[2];
    const long long total = static_cast<long long>(ncx) * ncy * ncz;
    const long long want = (total + 255) / 256;
    const int blocks = static_cast<int>(want < 8192 ? want : 8192);
    k_cell_range<<<blocks, 256, 0, stream>>>(win, storage, window_values(q), degree[0], degree[1], degree[2], ncx, ncy,
                                             ncz, nctrl[0] + kPad, nctrl[1] + kPad, cell);
    return cudaGetLastError();
}

cudaError_t launch_prep_stats(const void* win, int storage, int nx, int ny, int nz, int q, int* d_stats,
                              cudaStream_t stream)
{
    k_stats_init<<<1, 1, 0, stream>>>(d_stats);
    const long long total = static_cast<long long>(nx) * ny * nz;
    const long long want = (total + 255) / 256;
    const int blocks = static_cast<int>(want < 4096 ? want : 4096);
    k_stats<<<blocks, 256, 0, stream>>>(win, storage, nx, ny, nz, q, d_stats);
    return cudaGetLastError();
}

}  // namespace mfa
