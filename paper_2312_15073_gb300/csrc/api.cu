// api.cu -- the C ABI declared in include/mfa.h: argument checks, model ownership,
// stream binding, error text, and the host-side set-up of each launch.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mfa.h"
#include "host.cuh"

using namespace mfa;

namespace mfa {

namespace {
thread_local std::string g_error;
thread_local cudaStream_t g_stream = nullptr;
}  // namespace

cudaStream_t current_stream() { return g_stream; }

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(e == cudaErrorMemoryAllocation ? MFA_ERR_NOMEM : MFA_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool valid_dtype(int d) { return d >= MFA_F64 && d <= MFA_BF16; }

// The debug word of device `dev` ({flags, count}, zeroed device memory, allocated on first
// use): what kernels of a debug build write bad indices into.  NULL in release builds.
unsigned* debug_word(int dev)
{
#ifdef MFA_DEBUG
    static std::mutex mu;
    static unsigned* words[64] = {};
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> g(mu);
    if (!words[dev]) {
        unsigned* w = nullptr;
        if (cudaMalloc(&w, 2 * sizeof(unsigned)) != cudaSuccess) return nullptr;
        if (cudaMemset(w, 0, 2 * sizeof(unsigned)) != cudaSuccess) {
            cudaFree(w);
            return nullptr;
        }
        words[dev] = w;
    }
    return words[dev];
#else
    (void)dev;
    return nullptr;
#endif
}
size_t dtype_size(int d) { return d == MFA_F64 ? 8 : d == MFA_F32 ? 4 : 2; }

// Checks one knot vector: length n+p+1, non-decreasing, clamped on [0,1] with exactly
// p+1 end knots at each end (the first and last spans are non-empty).
bool check_knots(const double* U, int n, int p, int axis)
{
    const int m = n + p + 1;
    for (int i = 0; i < m; ++i) {
        if (!std::isfinite(U[i])) return fail(MFA_ERR_ARG, "knots[%d][%d] is not finite", axis, i), false;
        if (i > 0 && U[i] < U[i - 1]) return fail(MFA_ERR_ARG, "knots[%d] decrease at %d", axis, i), false;
    }
    for (int i = 0; i <= p; ++i) {
        if (U[i] != 0.0) return fail(MFA_ERR_ARG, "knots[%d]: the first %d knots must be 0", axis, p + 1), false;
        if (U[n + i] != 1.0) return fail(MFA_ERR_ARG, "knots[%d]: the last %d knots must be 1", axis, p + 1), false;
    }
    if (n > p + 1 && !(U[p + 1] > 0.0 && U[n - 1] < 1.0))
        return fail(MFA_ERR_ARG, "knots[%d]: interior knots must lie strictly inside (0,1)", axis), false;
    return true;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

int check_model_device(const mfa_model* m)
{
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != m->device) return fail(MFA_ERR_ARG, "model lives on device %d but device %d is current", m->device, cur);
    return MFA_OK;
}

// Validates the view of one render call (camera, transfer function, sizes, output) and
// fills the kernel's scalars and table.  The field's value range [fmin, fmax] replaces a NaN
// vmin / vmax; gtiny is the gradient norm below which the normal is undefined.
int setup_view(const mfa_camera* cam, const mfa_transfer_fn* tf, int width, int height, int n_samples,
               float* rgba_out, unsigned long long* samples_out, float fmin, float fmax, double gtiny,
               RenderScalars& S, float4* table)
{
    if (!cam || !tf || !rgba_out) return fail(MFA_ERR_ARG, "camera, tf and rgba_out must be non-NULL");
    if (width < 1 || width > 32768 || height < 1 || height > 32768)
        return fail(MFA_ERR_ARG, "image size %dx%d outside 1..32768", width, height);
    if (n_samples < 1 || n_samples > (1 << 20)) return fail(MFA_ERR_ARG, "n_samples = %d outside 1..2^20", n_samples);
    if (tf->n_entries < 1 || tf->n_entries > kTfMax || !tf->rgba)
        return fail(MFA_ERR_ARG, "transfer function needs 1..%d rows and a table", kTfMax);
    if (cam->projection != 0 && cam->projection != 1) return fail(MFA_ERR_ARG, "projection must be 0 or 1");

    // camera frame in FP64, handed to the kernel in FP32
    double f[3], r[3], u[3];
    for (int a = 0; a < 3; ++a) f[a] = cam->target[a] - cam->eye[a];
    double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    if (!(fl > 0.0) || !std::isfinite(fl)) return fail(MFA_ERR_ARG, "camera eye and target coincide");
    for (double& x : f) x /= fl;
    r[0] = f[1] * cam->up[2] - f[2] * cam->up[1];
    r[1] = f[2] * cam->up[0] - f[0] * cam->up[2];
    r[2] = f[0] * cam->up[1] - f[1] * cam->up[0];
    double rl = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    double ul = std::sqrt(cam->up[0] * cam->up[0] + cam->up[1] * cam->up[1] + cam->up[2] * cam->up[2]);
    if (!(rl > 1e-12 * ul) || !std::isfinite(rl)) return fail(MFA_ERR_ARG, "camera up is parallel to the view direction");
    for (double& x : r) x /= rl;
    u[0] = r[1] * f[2] - r[2] * f[1];
    u[1] = r[2] * f[0] - r[0] * f[2];
    u[2] = r[0] * f[1] - r[1] * f[0];
    const double aspect = static_cast<double>(width) / height;
    double sxs, sys;
    if (cam->projection == 0) {
        if (!(cam->ortho_height > 0.0) || !std::isfinite(cam->ortho_height))
            return fail(MFA_ERR_ARG, "ortho_height must be > 0");
        sys = 0.5 * cam->ortho_height;
        sxs = sys * aspect;
    } else {
        if (!(cam->fov_y_deg > 0.0 && cam->fov_y_deg < 180.0)) return fail(MFA_ERR_ARG, "fov_y_deg outside (0,180)");
        sys = std::tan(0.5 * cam->fov_y_deg * M_PI / 180.0);
        sxs = sys * aspect;
    }

    std::memset(&S, 0, sizeof S);
    for (int a = 0; a < 3; ++a) {
        S.eye[a] = static_cast<float>(cam->eye[a]);
        S.fwd[a] = static_cast<float>(f[a]);
        S.rx[a] = static_cast<float>(r[a] * sxs);
        S.uy[a] = static_cast<float>(u[a] * sys);
    }
    S.projection = cam->projection;
    S.width = width;
    S.height = height;
    S.n_samples = n_samples;
    S.inv_w = 1.0f / static_cast<float>(width);
    S.inv_h = 1.0f / static_cast<float>(height);
    const float vmin = std::isnan(tf->vmin) ? fmin : tf->vmin;
    const float vmax = std::isnan(tf->vmax) ? fmax : tf->vmax;
    S.vmin = vmin;
    S.inv_range = vmax > vmin ? static_cast<float>(1.0 / (static_cast<double>(vmax) - vmin)) : 0.0f;
    S.tf_n = tf->n_entries;
    S.shading = tf->shading ? 1 : 0;
    S.ka = tf->ka;
    S.kd = tf->kd;
    S.ks = tf->ks;
    S.shininess = tf->shininess;
    S.ert_alpha = tf->ert_alpha >= 1.0f ? INFINITY : tf->ert_alpha;
    S.gtiny2 = static_cast<float>(gtiny * gtiny);
    int dev = 0;
    cudaGetDevice(&dev);
    S.dbg = debug_word(dev);
    S.samples_out = samples_out;
    S.out = reinterpret_cast<float4*>(rgba_out);
    for (int i = 0; i < tf->n_entries; ++i)
        table[i] = make_float4(tf->rgba[4 * i], tf->rgba[4 * i + 1], tf->rgba[4 * i + 2], tf->rgba[4 * i + 3]);
    return MFA_OK;
}

// Validates one render call of a model and fills the kernel's scalars and table: the model
// (on the current device), then the view with the model's value range and a normal
// threshold of 1e-6 G, G = max(range, max |P|) x the most spans of an axis (a bound on the
// gradient's scale).
int setup_render(const mfa_model* m, const mfa_camera* cam, const mfa_transfer_fn* tf, int width, int height,
                 int n_samples, float* rgba_out, unsigned long long* samples_out, RenderScalars& S, float4* table)
{
    if (!m) return fail(MFA_ERR_ARG, "model, camera, tf and rgba_out must be non-NULL");
    if (int rc = check_model_device(m)) return rc;
    int spans = 0;
    for (int a = 0; a < 3; ++a) spans = std::max(spans, m->nctrl[a] - m->degree[a]);
    const double scale = std::max(static_cast<double>(m->vmax) - m->vmin, static_cast<double>(m->maxabs));
    return setup_view(cam, tf, width, height, n_samples, rgba_out, samples_out, m->vmin, m->vmax, 1e-6 * scale * spans,
                      S, table);
}

}  // namespace mfa

extern "C" {

const char* mfa_last_error(void) { return g_error.c_str(); }

int mfa_set_stream(void* cuda_stream)
{
    g_stream = static_cast<cudaStream_t>(cuda_stream);
    return MFA_OK;
}

int mfa_debug_build(void)
{
#ifdef MFA_DEBUG
    return 1;
#else
    return 0;
#endif
}

int mfa_debug_status(unsigned* flags, unsigned* count)
{
    if (!flags || !count) return fail(MFA_ERR_ARG, "flags and count must be non-NULL");
    *flags = 0;
    *count = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    unsigned* w = debug_word(dev);
    if (!w) return MFA_OK;
    unsigned h[2];
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(h, w, sizeof h, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(w, 0, sizeof h);
    if (e != cudaSuccess) return cuda_fail(e, "debug status");
    *flags = h[0];
    *count = h[1];
    return MFA_OK;
}

void mfa_model_destroy(mfa_model* m)
{
    if (!m) return;
    DeviceGuard g(m->device);
    if (m->d_win) cudaFree(m->d_win);
    if (m->d_patch) cudaFree(m->d_patch);
    if (m->d_tables) cudaFree(m->d_tables);
    delete m;
}

}  // extern "C"

namespace mfa {

mfa_model* model_create(const int degree[3], const int nctrl[3], const double* const knots[3], const void* ctrl,
                        mfa_dtype in_dtype, mfa_dtype storage, bool ctrl_on_device, int window)
{
    g_error.clear();
    if (!degree || !nctrl || !ctrl) return fail(MFA_ERR_ARG, "degree, nctrl and ctrl must be non-NULL"), nullptr;
    if (!valid_dtype(in_dtype)) return fail(MFA_ERR_ARG, "unknown input dtype %d", (int)in_dtype), nullptr;
    if (storage != MFA_F32 && storage != MFA_F16 && storage != MFA_BF16)
        return fail(MFA_ERR_UNSUPPORTED, "storage dtype must be F32, F16 or BF16"), nullptr;
    if (window != MFA_WINDOW_AUTO && window != MFA_WINDOW_F32 && window != MFA_WINDOW_COMPACT &&
        window != MFA_WINDOW_PATCH)
        return fail(MFA_ERR_ARG, "window = %d is not one of the MFA_WINDOW_* choices", window), nullptr;
    const bool compact = window == MFA_WINDOW_COMPACT;
    // window type (ModelDev::storage): layer pairs of FP32 or of the storage type's values, or
    // the compact plain array of the storage type
    const int wstore =
        compact ? storage + 3 : (window == MFA_WINDOW_F32 || window == MFA_WINDOW_PATCH ? MFA_F32 : storage);
    int qmax = 0;
    for (int a = 0; a < 3; ++a) {
        if (degree[a] < 1 || degree[a] > kMaxDegree)
            return fail(MFA_ERR_UNSUPPORTED, "degree[%d] = %d outside 1..%d", a, degree[a], kMaxDegree), nullptr;
        if (nctrl[a] < degree[a] + 1 || nctrl[a] > (1 << 24))
            return fail(MFA_ERR_ARG, "nctrl[%d] = %d must be in degree+1..2^24", a, nctrl[a]), nullptr;
        qmax = degree[a] + 1 > qmax ? degree[a] + 1 : qmax;
    }
    const bool patches = window == MFA_WINDOW_PATCH;
    if (patches && (degree[0] != 3 || degree[1] != 3 || degree[2] != 3))
        return fail(MFA_ERR_UNSUPPORTED, "MFA_WINDOW_PATCH needs degree 3 on every axis"), nullptr;
    // padded sizes: kPad zeros past the end of every axis; compact models round x up to a
    // multiple of their entry stride, so that their rows are whole entries of eight values
    const int cstride = compact_stride(qmax, wstore);
    const long long nxp = compact ? (nctrl[0] + kPad + cstride - 1) / cstride * cstride : nctrl[0] + kPad;
    const long long nyp = nctrl[1] + kPad, nzp = nctrl[2] + kPad;
    if (nxp * nyp * nzp >= (1LL << 31))
        return fail(MFA_ERR_UNSUPPORTED, "model too large: (nx+4)(ny+4)(nz+4) must stay below 2^31"), nullptr;

    // knot vectors (host, FP64): caller's or clamped uniform.  Caller's knots count as
    // uniform (the cardinal path) only when they equal the clamped uniform vector exactly,
    // i/(n-p) correctly rounded to FP64: the exactness of the cardinal path's span (floor of
    // the rounded product (n-p) u, checked only where it lands on an integer) rests on it.
    std::vector<double> U[3];
    bool uniform = true;
    for (int a = 0; a < 3; ++a) {
        const int n = nctrl[a], p = degree[a], m = n + p + 1;
        U[a].resize(m);
        for (int i = 0; i < m; ++i)
            U[a][i] = i <= p ? 0.0 : (i >= n ? 1.0 : static_cast<double>(i - p) / static_cast<double>(n - p));
        if (knots && knots[a]) {
            for (int i = 0; i < m; ++i)
                if (!(knots[a][i] == U[a][i])) uniform = false;
            std::memcpy(U[a].data(), knots[a], sizeof(double) * m);
            if (!check_knots(U[a].data(), n, p, a)) return nullptr;
        }
    }

    mfa_model* M = new mfa_model();
    cudaGetDevice(&M->device);
    for (int a = 0; a < 3; ++a) {
        M->degree[a] = degree[a];
        M->nctrl[a] = nctrl[a];
    }
    M->storage = storage;
    M->uniform = uniform;
    for (int a = 0; a < 3; ++a) M->knots[a] = U[a];
    const int Q = qmax;
    cudaStream_t st = g_stream;

    // one allocation for the three axes' tables: kup | grid | records, each 256-B aligned
    size_t off_kup[3], off_grid[3], off_rec[3], tab = 0;
    int G[3];
    for (int a = 0; a < 3; ++a) {
        const int n = nctrl[a], p = degree[a];
        G[a] = 4 * (n - p);
        off_kup[a] = tab;
        tab = align_up(tab + sizeof(float) * (n + p + 1), 256);
        off_grid[a] = tab;
        tab = align_up(tab + sizeof(int) * G[a], 256);
        off_rec[a] = tab;
        tab = align_up(tab + sizeof(float) * rec_stride(Q) * (n - p), 256);
    }
    const size_t off_cell = tab;   // per knot-span cell {min, max} of its support (not on compact models)
    const size_t ncells =
        compact ? 0 : static_cast<size_t>(nctrl[0] - degree[0]) * (nctrl[1] - degree[1]) * (nctrl[2] - degree[2]);
    tab = align_up(tab + sizeof(float2) * ncells, 256);
    const size_t val_bytes = storage == MFA_F32 ? 4 : 2;
    // a layer-pair entry per padded position, or entries of eight values per cstride positions
    // (compact: eight spare values at the end, which an FP32 row's second load may touch)
    const size_t win_bytes = compact ? (static_cast<size_t>(nxp / cstride * nyp * nzp) * compact_values(wstore) + 8) *
                                           val_bytes
                                     : static_cast<size_t>(nxp * nyp * nzp) * (wstore == MFA_F32 ? 4 : 2) *
                                           window_values(Q);
    const size_t nctrl_total = static_cast<size_t>(nctrl[0]) * nctrl[1] * nctrl[2];
    const size_t raw_bytes = nctrl_total * val_bytes;
    const size_t off_raw = tab;   // the stored control points, plain array (staging only on compact models)
    if (!compact) tab = align_up(tab + raw_bytes, 256);
    const size_t in_bytes = nctrl_total * dtype_size(in_dtype);
    size_t knot_bytes = 0;
    for (int a = 0; a < 3; ++a) knot_bytes += sizeof(double) * U[a].size();
    const bool pow_rows = power_rows(Q, wstore);
    // FP64 power coefficients of the spans, used while building the window (x, for power rows)
    // and the patches (all three axes), [axis][span][k][r]
    size_t coef_off[3], coef_bytes = 0;
    for (int a = 0; a < 3; ++a) {
        coef_off[a] = coef_bytes;
        if ((a == 0 && pow_rows) || patches) coef_bytes += sizeof(double) * Q * Q * (nctrl[a] - degree[a]);
    }

    void* d_stage = nullptr;   // uploaded knots, stats, x coefficients and input control points; freed below
    const size_t stage_raw = compact ? align_up(raw_bytes, 256) : 0;
    const size_t stage_bytes = align_up(knot_bytes, 256) + 256 + align_up(coef_bytes, 256) + stage_raw +
                               (ctrl_on_device ? 0 : in_bytes);
    cudaError_t e;
    auto cleanup = [&](int code, const char* what, cudaError_t err) -> mfa_model* {
        if (err != cudaSuccess) cuda_fail(err, what); else fail(code, "%s", what);
        if (d_stage) cudaFree(d_stage);
        mfa_model_destroy(M);
        return nullptr;
    };
    if ((e = cudaMalloc(&M->d_tables, tab)) != cudaSuccess) return cleanup(0, "cudaMalloc(tables)", e);
    if ((e = cudaMalloc(&M->d_win, win_bytes)) != cudaSuccess) return cleanup(0, "cudaMalloc(window)", e);
    if ((e = cudaMalloc(&d_stage, stage_bytes)) != cudaSuccess) return cleanup(0, "cudaMalloc(staging)", e);

    char* stage = static_cast<char*>(d_stage);
    double* d_knots[3];
    size_t koff = 0;
    for (int a = 0; a < 3; ++a) {
        d_knots[a] = reinterpret_cast<double*>(stage + koff);
        if ((e = cudaMemcpyAsync(d_knots[a], U[a].data(), sizeof(double) * U[a].size(), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
            return cleanup(0, "upload knots", e);
        koff += sizeof(double) * U[a].size();
    }
    int* d_stats = reinterpret_cast<int*>(stage + align_up(knot_bytes, 256));
    double* d_coefs[3];
    for (int a = 0; a < 3; ++a)
        d_coefs[a] = (a == 0 && pow_rows) || patches
                         ? reinterpret_cast<double*>(stage + align_up(knot_bytes, 256) + 256 + coef_off[a])
                         : nullptr;
    double* d_coef = d_coefs[0];
    void* d_in = ctrl_on_device ? const_cast<void*>(ctrl)
                                : stage + align_up(knot_bytes, 256) + 256 + align_up(coef_bytes, 256) + stage_raw;
    if (!ctrl_on_device && (e = cudaMemcpyAsync(d_in, ctrl, in_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cleanup(0, "upload control points", e);

    char* tabs = static_cast<char*>(M->d_tables);
    for (int a = 0; a < 3; ++a) {
        AxisDev& A = M->dev.ax[a];
        A.kup = reinterpret_cast<const float*>(tabs + off_kup[a]);
        A.grid = reinterpret_cast<const int*>(tabs + off_grid[a]);
        A.rec = reinterpret_cast<const float*>(tabs + off_rec[a]);
        A.n = nctrl[a];
        A.p = degree[a];
        A.G = G[a];
        A.Gf = static_cast<float>(G[a]);
        if ((e = launch_prep_axis(d_knots[a], A.n, A.p, Q, const_cast<float*>(A.kup), const_cast<float*>(A.rec),
                                  const_cast<int*>(A.grid), A.G, d_coefs[a], st)) != cudaSuccess)
            return cleanup(0, "span tables", e);
    }
    void* d_raw = compact ? static_cast<void*>(stage + align_up(knot_bytes, 256) + 256 + align_up(coef_bytes, 256))
                          : static_cast<void*>(tabs + off_raw);
    if ((e = launch_prep_raw(d_in, in_dtype, storage, static_cast<long long>(nctrl_total), d_raw, st)) != cudaSuccess)
        return cleanup(0, "stored control points", e);
    if ((e = launch_prep_window(d_raw, storage, nctrl[0], nctrl[1], nctrl[2], static_cast<int>(nxp), Q, d_coef,
                                degree[0], M->d_win, wstore, st)) != cudaSuccess)
        return cleanup(0, "window array", e);
    if ((e = launch_prep_stats(d_raw, storage, static_cast<long long>(nctrl_total), d_stats, st)) != cudaSuccess)
        return cleanup(0, "control-point statistics", e);
    size_t patch_bytes = 0;
    if (patches) {
        patch_bytes = sizeof(float) * 64 * static_cast<size_t>(nctrl[0] - 3) * (nctrl[1] - 3) * (nctrl[2] - 3);
        if ((e = cudaMalloc(&M->d_patch, patch_bytes)) != cudaSuccess) return cleanup(0, "cudaMalloc(patches)", e);
        const double* const cf[3] = { d_coefs[0], d_coefs[1], d_coefs[2] };
        if ((e = launch_prep_patches(d_raw, storage, nctrl, cf, static_cast<float*>(M->d_patch), st)) != cudaSuccess)
            return cleanup(0, "cell patches", e);
    }
    float2* d_cell = compact ? nullptr : reinterpret_cast<float2*>(tabs + off_cell);
    if (!compact && (e = launch_prep_cells(d_raw, storage, degree, nctrl, d_cell, st)) != cudaSuccess)
        return cleanup(0, "cell bounds", e);
    int stats[3];
    if ((e = cudaMemcpyAsync(stats, d_stats, sizeof stats, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cleanup(0, "read statistics", e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cleanup(0, "model preparation", e);
    cudaFree(d_stage);
    d_stage = nullptr;

    auto ord2f = [](int i) {
        int b = i >= 0 ? i : i ^ 0x7FFFFFFF;
        float f;
        std::memcpy(&f, &b, sizeof f);
        return f;
    };
    M->vmin = ord2f(stats[0]);
    M->vmax = ord2f(stats[1]);
    M->maxabs = ord2f(stats[2]);
    M->dev.win = M->d_win;
    M->dev.patch = static_cast<const float*>(M->d_patch);
    M->dev.raw = compact ? nullptr : d_raw;
    M->window = window;
    M->dev.nxp = static_cast<int>(nxp);
    M->dev.nyp = static_cast<int>(nyp);
    M->dev.nzp = static_cast<int>(nzp);
    M->dev.q = Q;
    M->dev.storage = wstore;
    M->dev.raw_storage = storage;
    M->dev.cardinal = uniform && degree[0] == Q - 1 && degree[1] == Q - 1 && degree[2] == Q - 1 ? 1 : 0;
    M->dev.cell = d_cell;
    M->dev.ncx = nctrl[0] - degree[0];
    M->dev.ncy = nctrl[1] - degree[1];
    M->dev.ncz = nctrl[2] - degree[2];
    M->dev.dbg = debug_word(M->device);
    for (int a = 0; a < 3; ++a) M->dev.ax[a].dbg = M->dev.dbg;
    M->bytes = tab + win_bytes + patch_bytes;
    return M;
}

}  // namespace mfa

extern "C" {

mfa_model* mfa_model_create_ex(const int degree[3], const int nctrl[3], const double* const knots[3],
                               const void* ctrl, mfa_dtype in_dtype, mfa_dtype storage)
{
    return model_create(degree, nctrl, knots, ctrl, in_dtype, storage, false, MFA_WINDOW_AUTO);
}

mfa_model* mfa_model_create_opts(const int degree[3], const int nctrl[3], const double* const knots[3],
                                 const void* ctrl, mfa_dtype in_dtype, mfa_dtype storage, int window)
{
    return model_create(degree, nctrl, knots, ctrl, in_dtype, storage, false, window);
}

mfa_model* mfa_model_create(const int degree[3], const int nctrl[3], const double* const knots[3], const void* ctrl,
                            mfa_dtype dtype)
{
    mfa_dtype storage = (dtype == MFA_F16) ? MFA_F16 : (dtype == MFA_BF16) ? MFA_BF16 : MFA_F32;
    return mfa_model_create_ex(degree, nctrl, knots, ctrl, dtype, storage);
}

int mfa_model_get_info(const mfa_model* m, mfa_model_info* info)
{
    if (!m || !info) return fail(MFA_ERR_ARG, "model and info must be non-NULL");
    for (int a = 0; a < 3; ++a) {
        info->degree[a] = m->degree[a];
        info->nctrl[a] = m->nctrl[a];
    }
    info->storage = m->storage;
    info->vmin = m->vmin;
    info->vmax = m->vmax;
    info->device_bytes = m->bytes;
    info->device = m->device;
    info->cardinal = m->dev.cardinal;
    info->window = m->window;
    return MFA_OK;
}

int mfa_decode(const mfa_model* m, const float* pts, long long n, float* val, float* grad)
{
    if (!m) return fail(MFA_ERR_ARG, "model is NULL");
    if (n < 0) return fail(MFA_ERR_ARG, "n = %lld < 0", n);
    if (n == 0) return MFA_OK;
    if (!pts || !val) return fail(MFA_ERR_ARG, "pts and val must be non-NULL");
    if (int rc = check_model_device(m)) return rc;
    cudaError_t e = launch_decode(m->dev, pts, n, val, grad, g_stream);
    return e == cudaSuccess ? MFA_OK : cuda_fail(e, "decode launch");
}

int mfa_locate_spans(const mfa_model* m, const float* pts, long long n, int* spans)
{
    if (!m) return fail(MFA_ERR_ARG, "model is NULL");
    if (n < 0) return fail(MFA_ERR_ARG, "n = %lld < 0", n);
    if (n == 0) return MFA_OK;
    if (!pts || !spans) return fail(MFA_ERR_ARG, "pts and spans must be non-NULL");
    if (int rc = check_model_device(m)) return rc;
    cudaError_t e = launch_spans(m->dev, pts, n, spans, g_stream);
    return e == cudaSuccess ? MFA_OK : cuda_fail(e, "span launch");
}

int mfa_render_ex(const mfa_model* m, const mfa_camera* cam, const mfa_transfer_fn* tf, int width, int height,
                  int n_samples, float* rgba_out, const mfa_render_opts* opts)
{
    int variant = opts ? opts->variant : 0;
    int shape = opts ? opts->tile_shape : 0;
    if (variant < 0 || variant > 8) return fail(MFA_ERR_ARG, "render variant %d outside 0..8", variant);
    if (shape < 0 || shape >= kTileShapes) return fail(MFA_ERR_ARG, "tile_shape %d outside 0..%d", shape, kTileShapes - 1);
    if (opts && opts->use_tuned && m) tuned_lookup(m, width, height, n_samples, &variant, &shape);
    RenderParams P;
    if (int rc = setup_render(m, cam, tf, width, height, n_samples, rgba_out, opts ? opts->samples_out : nullptr, P.s,
                              P.tf))
        return rc;
    cudaStream_t st = current_stream();
    unsigned* bits = nullptr;   // variant 7: per-cell visibility under this transfer function
    cudaError_t e = cudaSuccess;
    if (variant == 7 && !m->dev.cell) variant = 0;   // no cell bounds (compact models): no skipping
    if (variant == 7) {
        cudaMemPool_t pool;
        const size_t words = (static_cast<size_t>(m->dev.ncx) * m->dev.ncy * m->dev.ncz + 31) / 32;
        if ((e = staging_pool(m->device, &pool)) != cudaSuccess) return cuda_fail(e, "staging pool");
        if ((e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&bits), words * sizeof(unsigned), pool, st)) !=
            cudaSuccess)
            return cuda_fail(e, "staging memory");
        e = launch_cell_visibility(m->dev, P, bits, st);
        P.s.cell_vis = bits;
    }
    if (e == cudaSuccess) e = launch_render(m->dev, P, variant, shape, st);
    if (bits) cudaFreeAsync(bits, st);
    return e == cudaSuccess ? MFA_OK : cuda_fail(e, "render launch");
}

int mfa_render(const mfa_model* m, const mfa_camera* cam, const mfa_transfer_fn* tf, int width, int height,
               int n_samples, float* rgba_out)
{
    return mfa_render_ex(m, cam, tf, width, height, n_samples, rgba_out, nullptr);
}

}  // extern "C"
