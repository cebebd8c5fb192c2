// host.cuh -- host-side pieces shared by the C-ABI translation units (api.cu, batch.cu):
// the model object, error reporting, the calling thread's stream and the validation of
// one render call.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/mfa.h"
#include "mfa_internal.cuh"

// The opaque model of the C ABI: host copies of its shape and statistics plus the device
// tables the kernels read.
struct mfa_model {
    int device = 0;
    int degree[3] = { 0, 0, 0 };
    int nctrl[3] = { 0, 0, 0 };
    mfa_dtype storage = MFA_F32;
    float vmin = 0.0f, vmax = 0.0f, maxabs = 0.0f;
    size_t bytes = 0;
    bool uniform = true;        // every axis has clamped uniform knots
    int window = MFA_WINDOW_AUTO;   // the MFA_WINDOW_* choice the model was built with
    std::vector<double> knots[3];   // the FP64 knot vectors (host copy, for mfa_model_save)
    void* d_win = nullptr;      // window array
    void* d_patch = nullptr;    // per-cell polynomial patches (MFA_WINDOW_PATCH models)
    void* d_tables = nullptr;   // kup, grid and records of the three axes, one allocation
    mfa::ModelDev dev{};
};

namespace mfa {

// Records the error text for mfa_last_error() on the calling thread; returns code.
int fail(int code, const char* fmt, ...);
// Same for a CUDA error (MFA_ERR_NOMEM for allocation failures, else MFA_ERR_CUDA).
int cuda_fail(cudaError_t e, const char* what);
// Stream bound with mfa_set_stream on the calling thread.
cudaStream_t current_stream();
// MFA_OK if the model lives on the current device.
int check_model_device(const mfa_model* m);
// Cached autotuner choice for this workload class, if any.
bool tuned_lookup(const mfa_model* m, int w, int h, int ns, int* variant, int* shape);
// Model creation (mfa_model_create_opts) from control points on the host, or, with
// ctrl_on_device, already in device memory of the current device (read, not kept); window
// is one of MFA_WINDOW_*.
mfa_model* model_create(const int degree[3], const int nctrl[3], const double* const knots[3], const void* ctrl,
                        mfa_dtype in_dtype, mfa_dtype storage, bool ctrl_on_device, int window = MFA_WINDOW_AUTO);
// The library's device staging pool on device `dev` (created on first use, memory kept
// cached between calls; allocate and free with the stream-ordered pool calls).
cudaError_t staging_pool(int dev, cudaMemPool_t* out);
// Validates the view of a render call (camera, transfer function, sizes, output) and fills
// the kernel's scalars and table; [fmin, fmax] stands in for a NaN vmin / vmax, gtiny is the
// gradient norm below which the normal is undefined.
int setup_view(const mfa_camera* cam, const mfa_transfer_fn* tf, int width, int height, int n_samples,
               float* rgba_out, unsigned long long* samples_out, float fmin, float fmax, double gtiny,
               RenderScalars& S, float4* table);
// Validates one render call of a model and fills the kernel's scalars and table (tf_n rows).
int setup_render(const mfa_model* m, const mfa_camera* cam, const mfa_transfer_fn* tf, int width, int height,
                 int n_samples, float* rgba_out, unsigned long long* samples_out, RenderScalars& S, float4* table);

}  // namespace mfa
