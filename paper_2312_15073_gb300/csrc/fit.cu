// fit.cu -- MFA encoding on the GPU (mfa_fit_ctrl, mfa_model_fit, mfa_model_encode): the
// step that builds a model from a regular grid of values before it is rendered (Sec. III-A,
// Sec. IV-A.2).
//
// Least squares.  The data D[k][j][i] sit at the uniform parameters u_i = i/(m_x - 1) (and
// v_j, w_k).  With collocation matrices A_x[i][c] = N_c(u_i) (A_y, A_z likewise) of full
// column rank, the control points minimising sum (f(u_i, v_j, w_k) - D[k][j][i])^2 are
// P = (A_z^+ (x) A_y^+ (x) A_x^+) D: a least-squares solve along each axis for every line;
// the three commute, and run along z, then y, then x (coalesced passes over the large
// arrays first).  Each 1-D solve uses the normal equations: the Gram matrix
// G = A^T A is symmetric positive definite and banded (half-bandwidth p), so a banded
// Cholesky factor L is computed once per axis, and every line solves L L^T x = A^T y by
// forward and back substitution -- one thread per line, FP64 throughout.  The right-hand
// side A^T y is formed on the fly during the forward sweep from the data points each basis
// function covers (a contiguous range of them).
//
// Adaptive encoding.  Starting from p + 1 control points per axis, the model is fitted,
// evaluated at every data point, and while the largest error exceeds err_max a knot is
// inserted on every axis at the middle of each knot span whose data exceed err_max (the
// error projected onto the axis by its maximum over the other two axes); the loop refits
// with the refined knots and stops when the error is within err_max or no axis can take
// another knot (a span holding fewer than two data parameters, or the axis at its
// control-point limit; where the limit would be passed, the leftmost spans come first).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "bspline.cuh"
#include "host.cuh"

using namespace mfa;

namespace {

constexpr int kFitMaxDegree = kMaxDegree;
constexpr int kFitThreads = 128;

// Largest s in [p, n-1] with U[s] <= u (u in [0, 1]; u = 1 gives n - 1).
__device__ __forceinline__ int fit_span(const double* U, int n, int p, double u)
{
    if (u >= U[n]) return n - 1;
    int lo = p, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (U[mid] <= u) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Per data parameter i: its span and the p + 1 non-zero basis values N_{s-p+r}(u_i), by the
// triangular Cox-de Boor recursion (a zero-length knot interval drops its term).
__global__ void k_fit_basis(const double* __restrict__ U, int n, int p, int m, int* __restrict__ span,
                            double* __restrict__ N)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const double u = m > 1 ? static_cast<double>(i) / static_cast<double>(m - 1) : 0.0;
    const int s = fit_span(U, n, p, u);
    double b[kFitMaxDegree + 1], left[kFitMaxDegree + 1], right[kFitMaxDegree + 1];
    b[0] = 1.0;
    for (int k = 1; k <= p; ++k) {
        left[k] = u - U[s + 1 - k];
        right[k] = U[s + k] - u;
        double saved = 0.0;
        for (int r = 0; r < k; ++r) {
            const double den = right[r + 1] + left[k - r];
            const double tmp = den != 0.0 ? b[r] / den : 0.0;
            b[r] = saved + right[r + 1] * tmp;
            saved = left[k - r] * tmp;
        }
        b[k] = saved;
    }
    span[i] = s;
    for (int r = 0; r <= p; ++r) N[static_cast<long long>(i) * (p + 1) + r] = b[r];
}

// Per control point c: the data range [first, last] of its support and its row of the Gram
// matrix's upper band, G[c][d] = sum_i N_c(u_i) N_{c+d}(u_i), d = 0..p.
__global__ void k_fit_gram(const int* __restrict__ span, const double* __restrict__ N, int m, int n, int p,
                           int* __restrict__ first, int* __restrict__ last, double* __restrict__ G)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    int lo = 0, hi = m;   // first i with span[i] >= c (spans do not decrease with i)
    while (lo < hi) {
        const int mid = (lo + hi) / 2;
        if (span[mid] < c) lo = mid + 1; else hi = mid;
    }
    double g[kFitMaxDegree + 1] = { 0.0, 0.0, 0.0, 0.0, 0.0 };
    int i = lo;
    for (; i < m && span[i] <= c + p; ++i) {
        const int r = c - (span[i] - p);   // c's index among the p + 1 functions of u_i
        const double* Ni = N + static_cast<long long>(i) * (p + 1);
        for (int d = 0; d <= p - r; ++d) g[d] += Ni[r] * Ni[r + d];
    }
    first[c] = lo;
    last[c] = i - 1;
    for (int d = 0; d <= p; ++d) G[static_cast<long long>(c) * (p + 1) + d] = g[d];
}

// Banded Cholesky G = L L^T (one thread: O(n p^2) sequential work).  L[c][d] = L(c, c-d);
// Linv[c] = 1 / L(c, c), so that the line solves multiply instead of dividing (an FP64
// divide costs many FP64 operations, and every line would do 2n of them).
// status = 1 if a pivot is not positive (the data do not determine the spline).
__global__ void k_fit_cholesky(const double* __restrict__ G, int n, int p, double* __restrict__ L,
                               double* __restrict__ Linv, int* __restrict__ status)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    *status = 0;
    const int w = p + 1;
    for (int c = 0; c < n; ++c) {
        for (int d = p; d >= 1; --d) {   // L(c, k) for k = c - d, left to right
            const int k = c - d;
            if (k < 0) {
                L[static_cast<long long>(c) * w + d] = 0.0;
                continue;
            }
            double v = G[static_cast<long long>(k) * w + d];   // G(k, c)
            for (int j = c - p; j < k; ++j) {                  // sum L(c, j) L(k, j)
                if (j < 0 || k - j > p) continue;
                v -= L[static_cast<long long>(c) * w + (c - j)] * L[static_cast<long long>(k) * w + (k - j)];
            }
            L[static_cast<long long>(c) * w + d] = v / L[static_cast<long long>(k) * w];
        }
        double v = G[static_cast<long long>(c) * w];
        for (int d = 1; d <= p; ++d) {
            const double l = L[static_cast<long long>(c) * w + d];
            v -= l * l;
        }
        if (!(v > 0.0)) {
            *status = 1;
            return;
        }
        L[static_cast<long long>(c) * w] = sqrt(v);
        Linv[c] = 1.0 / L[static_cast<long long>(c) * w];
    }
}

// One axis pass: for every line, the least-squares solve L L^T x = A^T y.  Line l reads its
// m data at in[base_in + i * in_stride] and writes its n results at
// out[base_out + c * out_stride], with base = (l / inner) * outer + (l % inner) * inner_step
// for input and output alike.  Data point i contributes N[i][r] to function
// c = span[i] - p + r.
template <typename T>
__global__ void __launch_bounds__(kFitThreads)
    k_fit_lines(const T* __restrict__ in, double* __restrict__ out, long long lines, long long inner,
                long long in_outer, long long in_inner, long long in_stride, long long out_outer, long long out_inner,
                long long out_stride, int n, int p, const int* __restrict__ span, const double* __restrict__ N,
                const int* __restrict__ first, const int* __restrict__ last, const double* __restrict__ L,
                const double* __restrict__ Linv)
{
    const long long l = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (l >= lines) return;
    const long long lo = l / inner, li = l % inner;
    const T* y = in + lo * in_outer + li * in_inner;
    double* x = out + lo * out_outer + li * out_inner;
    const int w = p + 1;
    // forward sweep: z_c = (rhs_c - sum_d L(c, c-d) z_{c-d}) / L(c, c), rhs = A^T y
    double h[kFitMaxDegree + 1] = { 0.0, 0.0, 0.0, 0.0, 0.0 };   // h[d] = z_{c-d}, d >= 1
    for (int c = 0; c < n; ++c) {
        double rhs = 0.0;
        for (int i = first[c]; i <= last[c]; ++i)
            rhs = fma(N[static_cast<long long>(i) * w + (c - span[i] + p)], static_cast<double>(y[i * in_stride]), rhs);
        double v = rhs;
        for (int d = 1; d <= p; ++d) v -= L[static_cast<long long>(c) * w + d] * h[d];
        v *= Linv[c];
        for (int d = p; d >= 2; --d) h[d] = h[d - 1];
        h[1] = v;
        x[c * out_stride] = v;
    }
    // back sweep: x_c = (z_c - sum_d L(c+d, c) x_{c+d}) / L(c, c)
    for (int d = 0; d <= p; ++d) h[d] = 0.0;                      // h[d] = x_{c+d}, d >= 1
    for (int c = n - 1; c >= 0; --c) {
        double v = x[c * out_stride];
        for (int d = 1; d <= p && c + d < n; ++d) v -= L[static_cast<long long>(c + d) * w + d] * h[d];
        v *= Linv[c];
        for (int d = p; d >= 2; --d) h[d] = h[d - 1];
        h[1] = v;
        x[c * out_stride] = v;
    }
}

// Errors of a model at every data point: |f(u_i, v_j, w_k) - D[k][j][i]| folded, by
// maximum on the FP32 bit pattern (errors are non-negative), into the per-axis projections
// ex[i], ey[j], ez[k] (zeroed by the caller).  One warp per x-line (j, k) at a time, its
// lanes on consecutive i (coalesced data reads): the line's maximum goes to ey[j] and ez[k]
// with one atomic each after a warp reduction, and ex[i] is gathered per block in shared
// memory (when n_x fits) and flushed once per block, so the global atomics number about
// two per line plus n_x per block instead of three per data point.
constexpr int kErrThreads = 256;
constexpr int kErrShared = 8192;   // ex entries a block gathers in shared memory

template <int Q, int STORAGE, bool CARD>
__global__ void __launch_bounds__(kErrThreads)
    k_fit_error(ModelDev M, const float* __restrict__ D, int mx, int my, int mz, unsigned* __restrict__ ex,
                unsigned* __restrict__ ey, unsigned* __restrict__ ez)
{
    __shared__ unsigned sx[kErrShared];
    const bool shared_x = mx <= kErrShared;
    if (shared_x)
        for (int i = threadIdx.x; i < mx; i += kErrThreads) sx[i] = 0u;
    __syncthreads();
    constexpr int kWarps = kErrThreads / 32;
    const int lane = threadIdx.x & 31;
    const long long lines = static_cast<long long>(my) * mz;
    for (long long L = blockIdx.x * static_cast<long long>(kWarps) + (threadIdx.x >> 5); L < lines;
         L += static_cast<long long>(gridDim.x) * kWarps) {
        const int j = static_cast<int>(L % my), k = static_cast<int>(L / my);
        const float v = my > 1 ? static_cast<float>(static_cast<double>(j) / (my - 1)) : 0.0f;
        const float w = mz > 1 ? static_cast<float>(static_cast<double>(k) / (mz - 1)) : 0.0f;
        const float* line = D + L * mx;
        unsigned lmax = 0u;
        for (int i = lane; i < mx; i += 32) {
            const float u = mx > 1 ? static_cast<float>(static_cast<double>(i) / (mx - 1)) : 0.0f;
            float f;
            if constexpr (CARD) {
                f = query_cardinal<Q, STORAGE>(M, u, v, w).x;
            } else {
                f = query2<Q, STORAGE>(M, u, v, w, locate_span(M.ax[0], u), locate_span(M.ax[1], v),
                                       locate_span(M.ax[2], w)).x;
            }
            const unsigned err = __float_as_uint(fabsf(f - line[i]));
            lmax = max(lmax, err);
            if (shared_x)
                atomicMax(sx + i, err);
            else
                atomicMax(ex + i, err);
        }
        lmax = __reduce_max_sync(0xFFFFFFFFu, lmax);
        if (lane == 0 && lmax) {
            atomicMax(ey + j, lmax);
            atomicMax(ez + k, lmax);
        }
    }
    __syncthreads();
    if (shared_x)
        for (int i = threadIdx.x; i < mx; i += kErrThreads)
            if (sx[i]) atomicMax(ex + i, sx[i]);
}

template <int Q, int STORAGE>
cudaError_t fit_error_qs(const ModelDev& m, const float* D, const int md[3], unsigned* ex, unsigned* ey, unsigned* ez,
                         cudaStream_t st)
{
    const long long lines = static_cast<long long>(md[1]) * md[2];
    const int blocks = static_cast<int>(std::min<long long>((lines + 7) / 8, 152LL * 16));
    if (m.cardinal)
        k_fit_error<Q, STORAGE, true><<<blocks, kErrThreads, 0, st>>>(m, D, md[0], md[1], md[2], ex, ey, ez);
    else
        k_fit_error<Q, STORAGE, false><<<blocks, kErrThreads, 0, st>>>(m, D, md[0], md[1], md[2], ex, ey, ez);
    return cudaGetLastError();
}

template <int Q>
cudaError_t fit_error_q(const ModelDev& m, const float* D, const int md[3], unsigned* ex, unsigned* ey, unsigned* ez,
                        cudaStream_t st)
{
    switch (m.storage) {
    case 1: return fit_error_qs<Q, 1>(m, D, md, ex, ey, ez, st);
    case 2: return fit_error_qs<Q, 2>(m, D, md, ex, ey, ez, st);
    default: return fit_error_qs<Q, 3>(m, D, md, ex, ey, ez, st);
    }
}

cudaError_t launch_fit_error(const ModelDev& m, const float* D, const int md[3], unsigned* ex, unsigned* ey,
                             unsigned* ez, cudaStream_t st)
{
    switch (m.q) {
    case 2: return fit_error_q<2>(m, D, md, ex, ey, ez, st);
    case 3: return fit_error_q<3>(m, D, md, ex, ey, ez, st);
    case 4: return fit_error_q<4>(m, D, md, ex, ey, ez, st);
    default: return fit_error_q<5>(m, D, md, ex, ey, ez, st);
    }
}

// Clamped knots of n control points at degree p: the caller's, or uniform when NULL.
bool fit_knots(const double* given, int n, int p, std::vector<double>& U, int axis)
{
    const int len = n + p + 1;
    U.resize(len);
    for (int i = 0; i < len; ++i)
        U[i] = i <= p ? 0.0 : (i >= n ? 1.0 : static_cast<double>(i - p) / static_cast<double>(n - p));
    if (!given) return true;
    std::memcpy(U.data(), given, sizeof(double) * len);
    for (int i = 0; i <= p; ++i)
        if (U[i] != 0.0 || U[len - 1 - i] != 1.0) return fail(MFA_ERR_ARG, "knots[%d] must be clamped on [0,1]", axis), false;
    for (int i = 1; i < len; ++i)
        if (!(U[i] >= U[i - 1])) return fail(MFA_ERR_ARG, "knots[%d] must not decrease", axis), false;
    return true;
}

// Device work space of one fit: per axis the basis tables and the Cholesky factor, plus the
// two intermediate arrays of the passes; one pool allocation, carved up on the host.
struct FitSpace {
    char* base = nullptr;
    size_t bytes = 0;
};

// Least-squares control points (FP64, device, [n_z][n_y][n_x]) of the data (FP32, device,
// [m_z][m_y][m_x]); knots U per axis on the host.  Synchronises the stream (to read the
// factorisation status).
int fit_device(const int degree[3], const int nctrl[3], const std::vector<double> U[3], const int md[3], const float* D,
               double* ctrl, cudaStream_t st)
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t pool = nullptr;
    cudaError_t e = staging_pool(dev, &pool);
    if (e != cudaSuccess) return cuda_fail(e, "staging pool");
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    size_t off_U[3], off_span[3], off_N[3], off_first[3], off_last[3], off_G[3], off_L[3], off_Linv[3], total = 0;
    for (int a = 0; a < 3; ++a) {
        const int n = nctrl[a], p = degree[a], m = md[a];
        off_U[a] = total;
        total += al(sizeof(double) * U[a].size());
        off_span[a] = total;
        total += al(sizeof(int) * m);
        off_N[a] = total;
        total += al(sizeof(double) * m * (p + 1));
        off_first[a] = total;
        total += al(sizeof(int) * n);
        off_last[a] = total;
        total += al(sizeof(int) * n);
        off_G[a] = total;
        total += al(sizeof(double) * n * (p + 1));
        off_L[a] = total;
        total += al(sizeof(double) * n * (p + 1));
        off_Linv[a] = total;
        total += al(sizeof(double) * n);
    }
    const size_t off_status = total;
    total += 256;
    const size_t off_t1 = total;   // after z: [n_z][m_y][m_x]
    total += al(sizeof(double) * static_cast<size_t>(nctrl[2]) * md[1] * md[0]);
    const size_t off_t2 = total;   // after y: [n_z][n_y][m_x]
    total += al(sizeof(double) * static_cast<size_t>(nctrl[2]) * nctrl[1] * md[0]);
    char* w = nullptr;
    if ((e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&w), total, pool, st)) != cudaSuccess)
        return cuda_fail(e, "fit work space");
    auto P = [&](size_t off) { return w + off; };
    int* status = reinterpret_cast<int*>(P(off_status));
    int bad = 0;
    for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
        const int n = nctrl[a], p = degree[a], m = md[a];
        double* dU = reinterpret_cast<double*>(P(off_U[a]));
        e = cudaMemcpyAsync(dU, U[a].data(), sizeof(double) * U[a].size(), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) break;
        k_fit_basis<<<(m + 127) / 128, 128, 0, st>>>(dU, n, p, m, reinterpret_cast<int*>(P(off_span[a])),
                                                     reinterpret_cast<double*>(P(off_N[a])));
        k_fit_gram<<<(n + 127) / 128, 128, 0, st>>>(reinterpret_cast<int*>(P(off_span[a])),
                                                    reinterpret_cast<double*>(P(off_N[a])), m, n, p,
                                                    reinterpret_cast<int*>(P(off_first[a])),
                                                    reinterpret_cast<int*>(P(off_last[a])),
                                                    reinterpret_cast<double*>(P(off_G[a])));
        k_fit_cholesky<<<1, 1, 0, st>>>(reinterpret_cast<double*>(P(off_G[a])), n, p,
                                        reinterpret_cast<double*>(P(off_L[a])),
                                        reinterpret_cast<double*>(P(off_Linv[a])), status + a);
        e = cudaGetLastError();
    }
    int st_host[3] = { 0, 0, 0 };
    if (e == cudaSuccess) e = cudaMemcpyAsync(st_host, status, sizeof st_host, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (int a = 0; a < 3; ++a) bad |= st_host[a] ? (1 << a) : 0;
    if (e == cudaSuccess && !bad) {
        const int mx = md[0], my = md[1], nx = nctrl[0], ny = nctrl[1], nz = nctrl[2];
        double* t1 = reinterpret_cast<double*>(P(off_t1));
        double* t2 = reinterpret_cast<double*>(P(off_t2));
        auto blocks = [](long long lines) { return static_cast<unsigned>((lines + kFitThreads - 1) / kFitThreads); };
        // The three axis solves commute; they run z, y, x so that the two passes over the
        // large arrays (the data, then the z-reduced data) read and write along the x-fastest
        // index across a warp's threads (coalesced) and only the last, smallest array is read
        // line by line.
        // z: lines (j, i), data stride m_y m_x
        long long lines = static_cast<long long>(my) * mx;
        k_fit_lines<float><<<blocks(lines), kFitThreads, 0, st>>>(
            D, t1, lines, lines, 0, 1, lines, 0, 1, lines, nz, degree[2], reinterpret_cast<int*>(P(off_span[2])),
            reinterpret_cast<double*>(P(off_N[2])), reinterpret_cast<int*>(P(off_first[2])),
            reinterpret_cast<int*>(P(off_last[2])), reinterpret_cast<double*>(P(off_L[2])),
            reinterpret_cast<double*>(P(off_Linv[2])));
        // y: lines (k, i), stride m_x
        lines = static_cast<long long>(nz) * mx;
        k_fit_lines<double><<<blocks(lines), kFitThreads, 0, st>>>(
            t1, t2, lines, mx, static_cast<long long>(my) * mx, 1, mx, static_cast<long long>(ny) * mx, 1, mx, ny,
            degree[1], reinterpret_cast<int*>(P(off_span[1])), reinterpret_cast<double*>(P(off_N[1])),
            reinterpret_cast<int*>(P(off_first[1])), reinterpret_cast<int*>(P(off_last[1])),
            reinterpret_cast<double*>(P(off_L[1])),
            reinterpret_cast<double*>(P(off_Linv[1])));
        // x: lines (k, j), stride 1
        lines = static_cast<long long>(nz) * ny;
        k_fit_lines<double><<<blocks(lines), kFitThreads, 0, st>>>(
            t2, ctrl, lines, 1, mx, 0, 1, nx, 0, 1, nx, degree[0], reinterpret_cast<int*>(P(off_span[0])),
            reinterpret_cast<double*>(P(off_N[0])), reinterpret_cast<int*>(P(off_first[0])),
            reinterpret_cast<int*>(P(off_last[0])), reinterpret_cast<double*>(P(off_L[0])),
            reinterpret_cast<double*>(P(off_Linv[0])));
        e = cudaGetLastError();
    }
    cudaError_t ef = cudaFreeAsync(w, st);
    if (e != cudaSuccess) return cuda_fail(e, "fit");
    if (bad)
        return fail(MFA_ERR_ARG,
                    "the data do not determine the spline on axis %d: a knot span without enough data parameters",
                    bad & 1 ? 0 : (bad & 2 ? 1 : 2));
    if (ef != cudaSuccess) return cuda_fail(ef, "fit work space free");
    return MFA_OK;
}

int check_fit_args(const int degree[3], const int nctrl[3], const int ndata[3], const float* data)
{
    if (!degree || !nctrl || !ndata || !data) return fail(MFA_ERR_ARG, "degree, nctrl, ndata and data must be non-NULL");
    for (int a = 0; a < 3; ++a) {
        if (degree[a] < 1 || degree[a] > kMaxDegree)
            return fail(MFA_ERR_UNSUPPORTED, "degree[%d] = %d outside 1..%d", a, degree[a], kMaxDegree);
        if (nctrl[a] < degree[a] + 1 || nctrl[a] > (1 << 16))
            return fail(MFA_ERR_ARG, "nctrl[%d] = %d must be in degree+1..65536", a, nctrl[a]);
        if (ndata[a] < nctrl[a] || ndata[a] > (1 << 20))
            return fail(MFA_ERR_ARG, "ndata[%d] = %d must be in nctrl..2^20", a, ndata[a]);
    }
    if (static_cast<long long>(ndata[0]) * ndata[1] * ndata[2] > (1LL << 33))
        return fail(MFA_ERR_ARG, "more than 2^33 data points");
    return MFA_OK;
}

// Model of the least-squares fit (FP64 control points in a pool buffer, then model creation
// from device memory with the requested storage).
mfa_model* fit_model(const int degree[3], const int nctrl[3], const std::vector<double> U[3], const int ndata[3],
                     const float* data, mfa_dtype storage, cudaStream_t st)
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t pool = nullptr;
    cudaError_t e = staging_pool(dev, &pool);
    if (e != cudaSuccess) return cuda_fail(e, "staging pool"), nullptr;
    double* ctrl = nullptr;
    const size_t bytes = sizeof(double) * static_cast<size_t>(nctrl[0]) * nctrl[1] * nctrl[2];
    if ((e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&ctrl), bytes, pool, st)) != cudaSuccess)
        return cuda_fail(e, "control points"), nullptr;
    mfa_model* M = nullptr;
    if (fit_device(degree, nctrl, U, ndata, data, ctrl, st) == MFA_OK) {
        const double* kp[3] = { U[0].data(), U[1].data(), U[2].data() };
        M = model_create(degree, nctrl, kp, ctrl, MFA_F64, storage, true);   // synchronous
    }
    cudaFreeAsync(ctrl, st);
    return M;
}

// Largest error and its projections onto the three axes (host copies).
int fit_errors(const mfa_model* M, const int md[3], const float* data, std::vector<float> proj[3], double* emax,
               cudaStream_t st)
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t pool = nullptr;
    cudaError_t e = staging_pool(dev, &pool);
    if (e != cudaSuccess) return cuda_fail(e, "staging pool");
    const size_t cnt = static_cast<size_t>(md[0]) + md[1] + md[2];
    unsigned* d = nullptr;
    if ((e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&d), sizeof(unsigned) * cnt, pool, st)) != cudaSuccess)
        return cuda_fail(e, "error projections");
    std::vector<unsigned> h(cnt);
    e = cudaMemsetAsync(d, 0, sizeof(unsigned) * cnt, st);
    if (e == cudaSuccess) e = launch_fit_error(M->dev, data, md, d, d + md[0], d + md[0] + md[1], st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d, sizeof(unsigned) * cnt, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(d, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "fit errors");
    size_t o = 0;
    *emax = 0.0;
    for (int a = 0; a < 3; ++a) {
        proj[a].resize(md[a]);
        for (int i = 0; i < md[a]; ++i) {
            float f;
            std::memcpy(&f, &h[o + i], sizeof f);
            proj[a][i] = f;
            *emax = std::max(*emax, static_cast<double>(f));
        }
        o += md[a];
    }
    return MFA_OK;
}

}  // namespace

extern "C" {

int mfa_fit_ctrl(const int degree[3], const int nctrl[3], const double* const knots[3], const int ndata[3],
                 const float* data, double* ctrl_out)
{
    if (int rc = check_fit_args(degree, nctrl, ndata, data)) return rc;
    if (!ctrl_out) return fail(MFA_ERR_ARG, "ctrl_out is NULL");
    std::vector<double> U[3];
    for (int a = 0; a < 3; ++a)
        if (!fit_knots(knots ? knots[a] : nullptr, nctrl[a], degree[a], U[a], a)) return MFA_ERR_ARG;
    return fit_device(degree, nctrl, U, ndata, data, ctrl_out, current_stream());
}

mfa_model* mfa_model_fit(const int degree[3], const int nctrl[3], const double* const knots[3], const int ndata[3],
                         const float* data, mfa_dtype storage, double* max_err)
{
    if (check_fit_args(degree, nctrl, ndata, data)) return nullptr;
    if (storage != MFA_F32 && storage != MFA_F16 && storage != MFA_BF16)
        return fail(MFA_ERR_UNSUPPORTED, "storage dtype must be F32, F16 or BF16"), nullptr;
    std::vector<double> U[3];
    for (int a = 0; a < 3; ++a)
        if (!fit_knots(knots ? knots[a] : nullptr, nctrl[a], degree[a], U[a], a)) return nullptr;
    cudaStream_t st = current_stream();
    mfa_model* M = fit_model(degree, nctrl, U, ndata, data, storage, st);
    if (M && max_err) {
        std::vector<float> proj[3];
        if (fit_errors(M, ndata, data, proj, max_err, st) != MFA_OK) {
            mfa_model_destroy(M);
            return nullptr;
        }
    }
    return M;
}

mfa_model* mfa_model_encode(const int degree[3], const int ndata[3], const float* data, mfa_dtype storage,
                            const mfa_encode_config* cfg, mfa_encode_result* result)
{
    if (!cfg) return fail(MFA_ERR_ARG, "cfg is NULL"), nullptr;
    if (!(cfg->err_max >= 0.0)) return fail(MFA_ERR_ARG, "err_max must be >= 0"), nullptr;
    if (cfg->max_iter < 1 || cfg->max_iter > 1000) return fail(MFA_ERR_ARG, "max_iter outside 1..1000"), nullptr;
    int nctrl[3], limit[3];
    for (int a = 0; a < 3; ++a) {
        if (!degree || degree[a] < 1 || degree[a] > kMaxDegree)
            return fail(MFA_ERR_UNSUPPORTED, "degree[%d] outside 1..%d", a, kMaxDegree), nullptr;
        nctrl[a] = degree[a] + 1;
        limit[a] = cfg->max_ctrl[a] > 0 ? cfg->max_ctrl[a] : (ndata ? ndata[a] : 0);
        if (limit[a] < nctrl[a]) return fail(MFA_ERR_ARG, "max_ctrl[%d] below degree + 1", a), nullptr;
    }
    if (check_fit_args(degree, nctrl, ndata, data)) return nullptr;
    if (storage != MFA_F32 && storage != MFA_F16 && storage != MFA_BF16)
        return fail(MFA_ERR_UNSUPPORTED, "storage dtype must be F32, F16 or BF16"), nullptr;
    cudaStream_t st = current_stream();
    std::vector<double> U[3];
    for (int a = 0; a < 3; ++a) fit_knots(nullptr, nctrl[a], degree[a], U[a], a);
    mfa_model* M = nullptr;
    double emax = INFINITY;
    int fits = 0;
    for (int it = 0; it < cfg->max_iter; ++it) {
        if (M) mfa_model_destroy(M);
        M = fit_model(degree, nctrl, U, ndata, data, storage, st);
        if (!M) return nullptr;
        ++fits;
        std::vector<float> proj[3];
        if (fit_errors(M, ndata, data, proj, &emax, st) != MFA_OK) {
            mfa_model_destroy(M);
            return nullptr;
        }
        if (emax <= cfg->err_max) break;
        bool inserted = false;
        for (int a = 0; a < 3; ++a) {
            const int p = degree[a], n = nctrl[a], m = ndata[a];
            std::vector<double> fresh;
            for (int s = p; s < n; ++s) {   // knot spans of this axis
                const double lo = U[a][s], hi = U[a][s + 1];
                int count = 0;
                float worst = 0.0f;
                for (int i = 0; i < m; ++i) {
                    const double u = m > 1 ? static_cast<double>(i) / (m - 1) : 0.0;
                    if (u >= lo && (u < hi || (s == n - 1 && u <= hi))) {
                        ++count;
                        worst = std::max(worst, proj[a][i]);
                    }
                }
                if (count >= 2 && worst > cfg->err_max) fresh.push_back(0.5 * (lo + hi));
            }
            const int room = std::max(limit[a] - n, 0);
            if (static_cast<int>(fresh.size()) > room) fresh.resize(room);
            if (!fresh.empty()) {
                U[a].insert(U[a].end(), fresh.begin(), fresh.end());
                std::sort(U[a].begin(), U[a].end());
                nctrl[a] += static_cast<int>(fresh.size());
                inserted = true;
            }
        }
        if (!inserted) break;
    }
    if (result) {
        result->iterations = fits;
        result->max_err = emax;
        for (int a = 0; a < 3; ++a) result->nctrl[a] = M->nctrl[a];
    }
    return M;
}

}  // extern "C"
