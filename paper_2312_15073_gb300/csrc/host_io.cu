// host_io.cu -- host-buffer forms of decode and render (mfa_decode_host, mfa_render_host):
// the same computations for callers whose points, values, gradients and images live in
// host memory.
//
// Device staging comes from a memory pool the library owns (one per device, memory kept
// cached between calls), allocated and freed in the order of the bound stream, so a call
// needs no synchronisation of its own and back-to-back calls reuse the same memory.
// Decode cuts the points into chunks and pipelines them over three helper streams of the
// calling thread -- copy-in of chunk c+1 and copy-out of chunk c-1 run beside the kernel
// on chunk c, the two copy directions on their own engines -- forked from and joined back
// to the bound stream with events.  The kernel stream has the device's greatest priority,
// so that a decode issued beside a long render interleaves its chunks with the render's
// tiles and its copies overlap the render, instead of all waiting for the render's end.  Render stages the whole image (its copy-out is small
// next to the kernel).  Both calls are asynchronous on the bound stream like
// cudaMemcpyAsync: the host buffers must stay valid, and are read or written, until that
// stream has been synchronised; page-locked buffers let the copies overlap, pageable ones
// work but the copies serialise.
#include <cstdint>
#include <mutex>

#include "host.cuh"

using namespace mfa;

namespace {

constexpr long long kDecodeChunk = 1LL << 20;   // points per pipelined chunk
constexpr int kMaxDevices = 64;

std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDevices] = {};

}  // namespace

namespace mfa {

cudaError_t staging_pool(int dev, cudaMemPool_t* out)
{
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        cudaError_t e = cudaMemPoolCreate(&p, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = UINT64_MAX;
        e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return e;
        }
        g_pool[dev] = p;
    }
    *out = g_pool[dev];
    return cudaSuccess;
}

}  // namespace mfa

namespace {

// Helper streams and an event ring of the calling thread, for one device.
struct IoStreams {
    static constexpr int kEvents = 64;
    int device = -1;
    cudaStream_t in = nullptr, run = nullptr, out = nullptr;
    cudaEvent_t ev[kEvents] = {};
    int next = 0;

    cudaError_t init(int dev)
    {
        if (device == dev) return cudaSuccess;
        release();
        int least = 0, greatest = 0;
        cudaDeviceGetStreamPriorityRange(&least, &greatest);
        cudaError_t e = cudaStreamCreateWithFlags(&in, cudaStreamNonBlocking);
        // the chunk kernels at the greatest priority: each is dispatched ahead of other
        // work's pending CTAs as soon as its points have arrived, so the copies of the
        // pipeline keep moving beside a long kernel instead of queueing behind it
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&run, cudaStreamNonBlocking, greatest);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&out, cudaStreamNonBlocking);
        for (int i = 0; i < kEvents && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            release();
            return e;
        }
        device = dev;
        return cudaSuccess;
    }
    // An event to record next.  A wait captures the record made before it was enqueued, so
    // reusing an event after 64 further records is safe.
    cudaEvent_t take()
    {
        cudaEvent_t e = ev[next];
        next = (next + 1) % kEvents;
        return e;
    }
    void release()
    {
        for (auto& e : ev)
            if (e) {
                cudaEventDestroy(e);
                e = nullptr;
            }
        for (cudaStream_t* s : { &in, &run, &out })
            if (*s) {
                cudaStreamDestroy(*s);
                *s = nullptr;
            }
        device = -1;
    }
    ~IoStreams() { release(); }
};
thread_local IoStreams t_io;

// e (a failed CUDA call) as the call's result; later calls of the sequence are skipped.
#define IO_TRY(call, what)                              \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

}  // namespace

extern "C" {

int mfa_decode_host(const mfa_model* m, const float* pts, long long n, float* val, float* grad)
{
    if (!m) return fail(MFA_ERR_ARG, "model is NULL");
    if (n < 0) return fail(MFA_ERR_ARG, "n = %lld < 0", n);
    if (n == 0) return MFA_OK;
    if (!pts || !val) return fail(MFA_ERR_ARG, "pts and val must be non-NULL");
    if (n > (1LL << 40)) return fail(MFA_ERR_ARG, "n = %lld too large", n);
    if (int rc = check_model_device(m)) return rc;
    const int dev = m->device;
    if (dev < 0 || dev >= kMaxDevices) return fail(MFA_ERR_UNSUPPORTED, "device %d", dev);
    cudaMemPool_t pool = nullptr;
    IO_TRY(staging_pool(dev, &pool), "staging pool");
    IO_TRY(t_io.init(dev), "helper streams");
    cudaStream_t st = current_stream();

    char* d = nullptr;   // pts | val | grad
    const size_t b_pts = 12ull * n, b_val = 4ull * n, b_grad = grad ? 12ull * n : 0;
    IO_TRY(cudaMallocFromPoolAsync(reinterpret_cast<void**>(&d), b_pts + b_val + b_grad, pool, st), "staging memory");
    float* d_pts = reinterpret_cast<float*>(d);
    float* d_val = reinterpret_cast<float*>(d + b_pts);
    float* d_grad = grad ? reinterpret_cast<float*>(d + b_pts + b_val) : nullptr;

    // fork: the helper streams start after the work already on the bound stream
    const char* what = "fork";
    cudaEvent_t fork = t_io.take();
    cudaError_t e = cudaEventRecord(fork, st);
    for (cudaStream_t s : { t_io.in, t_io.run, t_io.out })
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, fork, 0);

    for (long long c0 = 0; c0 < n && e == cudaSuccess; c0 += kDecodeChunk) {
        const long long cn = n - c0 < kDecodeChunk ? n - c0 : kDecodeChunk;
        cudaEvent_t loaded = t_io.take(), done = t_io.take();
        what = "copy-in";
        e = cudaMemcpyAsync(d_pts + 3 * c0, pts + 3 * c0, 12ull * cn, cudaMemcpyHostToDevice, t_io.in);
        if (e == cudaSuccess) e = cudaEventRecord(loaded, t_io.in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(t_io.run, loaded, 0);
        if (e == cudaSuccess) {
            what = "decode launch";
            e = launch_decode(m->dev, d_pts + 3 * c0, cn, d_val + c0, d_grad ? d_grad + 3 * c0 : nullptr, t_io.run);
        }
        if (e == cudaSuccess) e = cudaEventRecord(done, t_io.run);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(t_io.out, done, 0);
        if (e == cudaSuccess) {
            what = "copy-out";
            e = cudaMemcpyAsync(val + c0, d_val + c0, 4ull * cn, cudaMemcpyDeviceToHost, t_io.out);
        }
        if (e == cudaSuccess && grad)
            e = cudaMemcpyAsync(grad + 3 * c0, d_grad + 3 * c0, 12ull * cn, cudaMemcpyDeviceToHost, t_io.out);
    }

    // join: the bound stream waits for all three helper streams (after a failure too, so
    // that the free is ordered after whatever was enqueued)
    cudaError_t ej = cudaSuccess;
    for (cudaStream_t s : { t_io.in, t_io.run, t_io.out }) {
        cudaEvent_t join = t_io.take();
        if (ej == cudaSuccess) ej = cudaEventRecord(join, s);
        if (ej == cudaSuccess) ej = cudaStreamWaitEvent(st, join, 0);
    }
    cudaError_t ef = cudaFreeAsync(d, st);
    if (e != cudaSuccess) return cuda_fail(e, what);
    if (ej != cudaSuccess) return cuda_fail(ej, "join");
    if (ef != cudaSuccess) return cuda_fail(ef, "staging free");
    return MFA_OK;
}

int mfa_render_host(const mfa_model* m, const mfa_camera* cam, const mfa_transfer_fn* tf, int width, int height,
                    int n_samples, float* rgba_out, const mfa_render_opts* opts)
{
    if (!m) return fail(MFA_ERR_ARG, "model is NULL");
    if (!rgba_out) return fail(MFA_ERR_ARG, "rgba_out is NULL");
    if (width < 1 || height < 1) return fail(MFA_ERR_ARG, "image size %d x %d", width, height);
    if (int rc = check_model_device(m)) return rc;
    const int dev = m->device;
    if (dev < 0 || dev >= kMaxDevices) return fail(MFA_ERR_UNSUPPORTED, "device %d", dev);
    cudaMemPool_t pool = nullptr;
    IO_TRY(staging_pool(dev, &pool), "staging pool");
    cudaStream_t st = current_stream();
    const size_t bytes = 16ull * static_cast<size_t>(width) * static_cast<size_t>(height);
    float* d_img = nullptr;
    IO_TRY(cudaMallocFromPoolAsync(reinterpret_cast<void**>(&d_img), bytes, pool, st), "staging memory");
    int rc = mfa_render_ex(m, cam, tf, width, height, n_samples, d_img, opts);
    if (rc == MFA_OK) {
        cudaError_t e = cudaMemcpyAsync(rgba_out, d_img, bytes, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "copy-out");
    }
    cudaError_t e = cudaFreeAsync(d_img, st);
    if (rc == MFA_OK && e != cudaSuccess) rc = cuda_fail(e, "staging free");
    return rc;
}

}  // extern "C"
