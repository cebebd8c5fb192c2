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
__global__ void k_span_records(const double* __restrict__ U, int n, int p, float* __restrict__ rec,
                               double* __restrict__ coef64)
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
    // the same coefficients in FP64, [span][k][r] (Q x Q per span), for the power rows
    if (coef64)
        for (int k = 0; k < Q; ++k)
            for (int r = 0; r < Q; ++r) coef64[(static_cast<long long>(idx) * Q + k) * Q + r] = r <= p ? T[r][k] : 0.0;
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

// The stored control points: one round-to-nearest-even step from the exact input value to
// the storage type, into the plain array.
__global__ void k_raw(const void* __restrict__ ctrl, int in_dtype, int storage, long long total, void* __restrict__ raw)
{
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const double x = load_in(ctrl, in_dtype, e);
        if (storage == 1)
            static_cast<float*>(raw)[e] = __double2float_rn(x);
        else
            static_cast<unsigned short*>(raw)[e] = to16(x, storage);
    }
}

// A stored control point as FP64 (exact), zero outside the grid.
__device__ __forceinline__ double raw_at(const void* raw, int storage, int nx, int ny, int nz, int i, int j, int k)
{
    if (i >= nx || j >= ny || k >= nz) return 0.0;
    const long long e = (static_cast<long long>(k) * ny + j) * nx + i;
    if (storage == 1) return static_cast<double>(static_cast<const float*>(raw)[e]);
    const unsigned short h = static_cast<const unsigned short*>(raw)[e];
    return storage == 2 ? static_cast<double>(__half2float(__ushort_as_half(h)))
                        : static_cast<double>(__uint_as_float(static_cast<unsigned>(h) << 16));
}

// The layer-pair window array (layout in mfa_internal.cuh), one entry per thread, from the
// stored control points (raw, of type raw_storage), in window values of type `storage`.
// 16-bit windows copy the stored values bit for bit.  FP32 windows with coef64 (the x
// axis's FP64 span coefficients, [span][c][r]) store each row's power form on its x span
// i: W_c = sum_r c_{c,r} P[i + r], summed in FP64 from the exact stored values and rounded
// once; entries with no span (i >= n_x - p_x) are zero.  Compact windows are built by
// k_window_compact.
__global__ void k_window(const void* __restrict__ raw, int raw_storage, int nx, int ny, int nz, int nxp, int q,
                         const double* __restrict__ coef64, int px, void* __restrict__ win, int storage)
{
    const int nyp = ny + kPad, nzp = nz + kPad;
    const long long total = static_cast<long long>(nxp) * nyp * nzp;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int i = static_cast<int>(e % nxp);
        const long long jk = e / nxp;
        const int j = static_cast<int>(jk % nyp);
        const int k = static_cast<int>(jk / nyp);
        // P[r][a] = P[k + r][j][i + a] for the entry's layers r = 0..2 and columns a = 0..3
        double P[3][4];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int a = 0; a < 4; ++a) P[r][a] = raw_at(raw, raw_storage, nx, ny, nz, i + a, j, k + r);
        if (coef64) {   // power rows of x span i (degree px: coefficients c = 0..px)
            double W[3][4] = {};
            if (i < nx - px) {
                const double* c = coef64 + static_cast<long long>(i) * q * q;
                for (int r = 0; r < 3; ++r)
                    for (int cc = 0; cc <= px; ++cc) {
                        double w = 0.0;
                        for (int a = 0; a <= px; ++a) w += c[cc * q + a] * P[r][a];
                        W[r][cc] = w;
                    }
            }
            for (int r = 0; r < 3; ++r)
                for (int a = 0; a < 4; ++a) P[r][a] = W[r][a];
        }
        // v[2a + r] = row a of layers r = 0, 1; for q == 3 also v[8 + a] = layer 2; then zeros
        double v[16];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            v[2 * a] = P[0][a];
            v[2 * a + 1] = P[1][a];
            v[8 + a] = P[2][a];
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

// The compact window (storage 4..6): per padded x-row of nxp positions (a multiple of the
// stride S), entry e holds the V stored values at positions S e .. S e + V - 1, zero past
// the grid; one thread per value slot.
__global__ void k_window_compact(const void* __restrict__ raw, int raw_storage, int nx, int ny, int nz, int nxp,
                                 int S, int V, void* __restrict__ win, int storage)
{
    const int ne = nxp / S;
    const long long slots = static_cast<long long>(ne) * (ny + kPad) * (nz + kPad) * V;
    for (long long v = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; v < slots;
         v += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int c = static_cast<int>(v % V);
        const long long ent = v / V;
        const int i = static_cast<int>(ent % ne) * S + c;
        const long long jk = ent / ne;
        const int j = static_cast<int>(jk % (ny + kPad)), k = static_cast<int>(jk / (ny + kPad));
        const double x = raw_at(raw, raw_storage, nx, ny, nz, i, j, k);
        if (storage == 4)
            static_cast<float*>(win)[v] = static_cast<float>(x);
        else
            static_cast<unsigned short*>(win)[v] = to16(x, storage - 3);
    }
}

// Per-cell polynomial patches (degree 3): for cell (i, j, k) with support P[k+c][j+b][i+a],
//   coefficient of t_x^qx t_y^qy t_z^qz = sum_{a,b,c} Cx[qx][a] Cy[qy][b] Cz[qz][c] P[k+c][j+b][i+a],
// Cx[q][a] the power coefficient of t^q in the x span's function a (likewise y, z), summed
// axis by axis in FP64 from the exact stored values and rounded once; one thread per cell.
__global__ void k_patches(const void* __restrict__ raw, int raw_storage, int nx, int ny, int nz,
                          const double* __restrict__ cx, const double* __restrict__ cy, const double* __restrict__ cz,
                          float* __restrict__ patch)
{
    const int ncx = nx - 3, ncy = ny - 3, ncz = nz - 3;
    const long long total = static_cast<long long>(ncx) * ncy * ncz;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int i = static_cast<int>(e % ncx);
        const long long jk = e / ncx;
        const int j = static_cast<int>(jk % ncy), k = static_cast<int>(jk / ncy);
        const double* Cx = cx + static_cast<long long>(i) * 16;
        const double* Cy = cy + static_cast<long long>(j) * 16;
        const double* Cz = cz + static_cast<long long>(k) * 16;
        double T[4][4][4];   // T[c][b][qx], then T[c][qy][qx], then T[qz][qy][qx]
        for (int c = 0; c < 4; ++c)
            for (int b = 0; b < 4; ++b) {
                double P[4];
                for (int a = 0; a < 4; ++a) P[a] = raw_at(raw, raw_storage, nx, ny, nz, i + a, j + b, k + c);
                for (int q = 0; q < 4; ++q) {
                    double w = 0.0;
                    for (int a = 0; a < 4; ++a) w += Cx[q * 4 + a] * P[a];
                    T[c][b][q] = w;
                }
            }
        for (int c = 0; c < 4; ++c)
            for (int qx = 0; qx < 4; ++qx) {
                double v[4];
                for (int q = 0; q < 4; ++q) {
                    double w = 0.0;
                    for (int b = 0; b < 4; ++b) w += Cy[q * 4 + b] * T[c][b][qx];
                    v[q] = w;
                }
                for (int q = 0; q < 4; ++q) T[c][q][qx] = v[q];
            }
        for (int qy = 0; qy < 4; ++qy)
            for (int qx = 0; qx < 4; ++qx) {
                double v[4];
                for (int q = 0; q < 4; ++q) {
                    double w = 0.0;
                    for (int c = 0; c < 4; ++c) w += Cz[q * 4 + c] * T[c][qy][qx];
                    v[q] = w;
                }
                for (int q = 0; q < 4; ++q) T[q][qy][qx] = v[q];
            }
        // entry 4m + b: {c[a][b][2m], c[a][b][2m+1]} for a = 0..3 (qz = 2m, 2m+1)
        float* out = patch + e * 64;
        for (int m = 0; m < 2; ++m)
            for (int b = 0; b < 4; ++b)
                for (int a = 0; a < 4; ++a) {
                    out[(4 * m + b) * 8 + 2 * a] = __double2float_rn(T[2 * m][b][a]);
                    out[(4 * m + b) * 8 + 2 * a + 1] = __double2float_rn(T[2 * m + 1][b][a]);
                }
    }
}

// {min, max} over the (p_x+1)(p_y+1)(p_z+1) stored control points of each knot-span cell's
// support, read from the plain array.
__global__ void k_cell_range(const void* __restrict__ raw, int storage, int nx, int ny, int nz, int px, int py, int pz,
                             int ncx, int ncy, int ncz, float2* __restrict__ cell)
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
                    const float v = static_cast<float>(raw_at(raw, storage, nx, ny, nz, i0 + a, j0 + b, k0 + c));
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

// min, max and max |P| over the stored values (the plain array)
__global__ void k_stats(const void* __restrict__ raw, int storage, long long total, int* __restrict__ stats)
{
    float mn = INFINITY, mx = -INFINITY, ma = 0.0f;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        float v;
        if (storage == 1) {
            v = static_cast<const float*>(raw)[e];
        } else {
            const unsigned short b = static_cast<const unsigned short*>(raw)[e];
            v = storage == 2 ? __half2float(__ushort_as_half(b)) : __uint_as_float(static_cast<unsigned>(b) << 16);
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
                             double* coef64, cudaStream_t stream)
{
    const int m = n + p + 1;
    k_knots_up<<<(m + 255) / 256, 256, 0, stream>>>(d_knots, m, kup);
    k_span_grid<<<(G + 255) / 256, 256, 0, stream>>>(d_knots, n, p, G, grid);
    const int spans = n - p;
    const int blocks = (spans + 127) / 128;
    switch (q) {
    case 2: k_span_records<2><<<blocks, 128, 0, stream>>>(d_knots, n, p, rec, coef64); break;
    case 3: k_span_records<3><<<blocks, 128, 0, stream>>>(d_knots, n, p, rec, coef64); break;
    case 4: k_span_records<4><<<blocks, 128, 0, stream>>>(d_knots, n, p, rec, coef64); break;
    case 5: k_span_records<5><<<blocks, 128, 0, stream>>>(d_knots, n, p, rec, coef64); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

static int grid_blocks(long long total, long long cap)
{
    const long long want = (total + 255) / 256;
    return static_cast<int>(want < cap ? (want > 0 ? want : 1) : cap);
}

cudaError_t launch_prep_raw(const void* d_ctrl, int in_dtype, int storage, long long total, void* raw,
                            cudaStream_t stream)
{
    k_raw<<<grid_blocks(total, 65536), 256, 0, stream>>>(d_ctrl, in_dtype, storage, total, raw);
    return cudaGetLastError();
}

cudaError_t launch_prep_window(const void* raw, int raw_storage, int nx, int ny, int nz, int nxp, int q,
                               const double* coef64, int px, void* win, int storage, cudaStream_t stream)
{
    if (compact_window(storage)) {
        const int S = compact_stride(q, storage), V = compact_values(storage);
        const long long slots = static_cast<long long>(nxp) / S * (ny + kPad) * (nz + kPad) * V;
        cudaError_t e = cudaMemsetAsync(static_cast<char*>(win) + slots * (storage == 4 ? 4 : 2), 0,
                                        8 * (storage == 4 ? 4 : 2), stream);   // the spare values
        if (e != cudaSuccess) return e;
        k_window_compact<<<grid_blocks(slots, 65536), 256, 0, stream>>>(raw, raw_storage, nx, ny, nz, nxp, S, V, win,
                                                                        storage);
        return cudaGetLastError();
    }
    const long long total = static_cast<long long>(nxp) * (ny + kPad) * (nz + kPad);
    k_window<<<grid_blocks(total, 65536), 256, 0, stream>>>(raw, raw_storage, nx, ny, nz, nxp, q, coef64, px, win,
                                                            storage);
    return cudaGetLastError();
}

cudaError_t launch_prep_patches(const void* raw, int raw_storage, const int nctrl[3], const double* const coef64[3],
                                float* patch, cudaStream_t stream)
{
    const long long total = static_cast<long long>(nctrl[0] - 3) * (nctrl[1] - 3) * (nctrl[2] - 3);
    k_patches<<<grid_blocks(total, 65536), 128, 0, stream>>>(raw, raw_storage, nctrl[0], nctrl[1], nctrl[2], coef64[0],
                                                             coef64[1], coef64[2], patch);
    return cudaGetLastError();
}

cudaError_t launch_prep_cells(const void* raw, int storage, const int degree[3], const int nctrl[3], float2* cell,
                              cudaStream_t stream)
{
    const int ncx = nctrl[0] - degree[0], ncy = nctrl[1] - degree[1], ncz = nctrl[2] - degree[2];
    const long long total = static_cast<long long>(ncx) * ncy * ncz;
    k_cell_range<<<grid_blocks(total, 8192), 256, 0, stream>>>(raw, storage, nctrl[0], nctrl[1], nctrl[2], degree[0],
                                                              degree[1], degree[2], ncx, ncy, ncz, cell);
    return cudaGetLastError();
}

cudaError_t launch_prep_stats(const void* raw, int storage, long long total, int* d_stats, cudaStream_t stream)
{
    k_stats_init<<<1, 1, 0, stream>>>(d_stats);
    k_stats<<<grid_blocks(total, 4096), 256, 0, stream>>>(raw, storage, total, d_stats);
    return cudaGetLastError();
}

}  // namespace mfa
