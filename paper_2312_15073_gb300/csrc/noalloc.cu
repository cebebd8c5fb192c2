// noalloc.cu -- mfa_render_batch_static: the batched render for callers that must not
// allocate.
//
// Some callers cannot call cudaMalloc: a process whose own memory pool has already
// reserved the whole device (a new cudaMalloc would fail), or a latency-bound render loop
// that must not take the allocator's implicit synchronisation after start-up.  The other
// batched entry points need a batch context that owns device and pinned host tables; this
// one keeps the work table of one submission (the per-group heads with their tile
// counters, the requests, their transfer-function rows) in a fixed array in the library's
// own device memory and renders with the same persistent kernels.  It calls no
// cudaMalloc, cudaFree, cudaMallocHost or other allocating routine.
//
// The array is a file-scope __device__ variable: every GPU that loads the library holds
// kStaticTableBytes of it until the process exits.  In host code its name is only a
// host-side stand-in, so its device address is fetched once per device with
// cudaGetSymbolAddress (on the first call on that device, with that device current) and
// passed to the kernels.
#include <atomic>
#include <cstring>

#include "host.cuh"

using namespace mfa;

namespace {

constexpr int kStaticMaxRequests = 32;
// heads + 32 items, rounded up to 256 bytes where the table rows start, + 32 full tables
constexpr size_t kStaticTableBytes = 176 * 1024;
constexpr size_t kStaticRowsOffset = (kBatchItemsOffset + sizeof(BatchItem) * kStaticMaxRequests + 255) / 256 * 256;
static_assert(kStaticRowsOffset + sizeof(float4) * kTfMax * kStaticMaxRequests <= kStaticTableBytes,
              "static work table too small");

static __device__ __align__(256) unsigned char g_static_table[kStaticTableBytes];

constexpr int kMaxDevices = 64;
std::atomic<void*> g_table_addr[kMaxDevices];

// Device address of g_static_table on the current device (looked up once per device).
cudaError_t static_table(int dev, void** out)
{
    void* p = g_table_addr[dev].load(std::memory_order_acquire);
    if (!p) {
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_table);
        if (e != cudaSuccess) return e;
        g_table_addr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return cudaSuccess;
}

}  // namespace

extern "C" int mfa_render_batch_static(const mfa_render_request* reqs, int n)
{
    if (n < 0 || n > kStaticMaxRequests)
        return fail(MFA_ERR_ARG, "n = %d: the allocation-free batch takes 0..%d requests", n, kStaticMaxRequests);
    if (n == 0) return MFA_OK;
    if (!reqs) return fail(MFA_ERR_ARG, "reqs is NULL");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "current device");
    if (dev < 0 || dev >= kMaxDevices) return fail(MFA_ERR_UNSUPPORTED, "device ordinal %d >= %d", dev, kMaxDevices);
    // The table is filled by copies from host memory owned by this call and its caller: a
    // graph captured from them would replay copies from memory that is gone, so a capturing
    // stream is refused before anything is enqueued (the capture stays valid).
    cudaStream_t st = current_stream();
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(st, &cap)) != cudaSuccess) return cuda_fail(e, "stream capture status");
    if (cap != cudaStreamCaptureStatusNone)
        return fail(MFA_ERR_UNSUPPORTED, "the allocation-free batch cannot be captured into a CUDA graph");

    // pass 1: validate everything, build every request's item (scalars, model, ray tiles)
    // and count each group's requests and tiles
    int count[kBatchGroups] = {};
    long long tiles[kBatchGroups] = {};
    BatchItem items[kStaticMaxRequests];
    int group_of[kStaticMaxRequests];
    float4 rows[kTfMax];
    int tw, th;
    render_tile_dims(0, &tw, &th);
    for (int r = 0; r < n; ++r) {
        const mfa_render_request& q = reqs[r];
        if (!q.model) return fail(MFA_ERR_ARG, "request %d: model is NULL", r);
        BatchItem& it = items[r];
        std::memset(&it, 0, sizeof it);
        if (int rc = setup_render(q.model, &q.camera, q.tf, q.width, q.height, q.n_samples, q.rgba_out, q.samples_out,
                                  it.s, rows)) {
            fail(rc, "request %d: %s", r, mfa_last_error());
            return rc;
        }
        const ModelDev& md = q.model->dev;
        const int g = batch_group(md.q, md.storage, md.cardinal, md.patch != nullptr && md.cardinal);
        group_of[r] = g;
        it.m = q.model->dev;
        it.tiles_x = (q.width + tw - 1) / tw;
        it.tile_begin = static_cast<int>(tiles[g]);   // tiles of a group follow request order
        ++count[g];
        tiles[g] += static_cast<long long>(it.tiles_x) * ((q.height + th - 1) / th);
        if (tiles[g] > (1LL << 30)) return fail(MFA_ERR_ARG, "batch too large: more than 2^30 ray tiles");
    }

    void* table = nullptr;
    if ((e = static_table(dev, &table)) != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static work table)");
    char* d = static_cast<char*>(table);

    // heads: item offsets by group, tile counters cleared (the array keeps the last call's
    // contents, so everything the kernels read is rewritten here)
    BatchHead heads[kBatchGroups] = {};
    size_t off = kBatchItemsOffset;
    for (int g = 0; g < kBatchGroups; ++g) {
        heads[g].next_tile = 0;
        heads[g].n_items = count[g];
        heads[g].total_tiles = static_cast<int>(tiles[g]);
        heads[g].items_offset = static_cast<int>(off);
        off += sizeof(BatchItem) * count[g];
    }
    const size_t tf_base = (off + 255) / 256 * 256;   // <= kStaticRowsOffset
    if ((e = cudaMemcpyAsync(d, heads, sizeof heads, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "static table heads");

    // pass 2: items (from pass 1) and table rows (the caller's RGBA rows, already laid out
    // as float4), copied from pageable host memory, which cudaMemcpyAsync stages before it
    // returns, so none of it has to outlive the call
    int placed[kBatchGroups] = {};
    for (int r = 0; r < n; ++r) {
        const mfa_render_request& q = reqs[r];
        BatchItem& it = items[r];
        const int g = group_of[r];
        char* tf_dst = d + tf_base + sizeof(float4) * kTfMax * static_cast<size_t>(r);
        it.tf = reinterpret_cast<const float4*>(tf_dst);
        char* item_dst = d + heads[g].items_offset + sizeof(BatchItem) * placed[g]++;
        if ((e = cudaMemcpyAsync(tf_dst, q.tf->rgba, sizeof(float4) * it.s.tf_n, cudaMemcpyHostToDevice, st)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(item_dst, &it, sizeof it, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_fail(e, "static table items");
    }

    // one persistent kernel per group present, in stream order
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int g = 0; g < kBatchGroups; ++g) {
        if (!count[g]) continue;
        const BatchKernel k = render_batch_kernel(batch_group_q(g), batch_group_storage(g), batch_group_cardinal(g),
                                                  batch_group_patch(g));
        BatchHead* tp = static_cast<BatchHead*>(table);
        int group = g, shape = 0;
        void* args[] = { &tp, &group, &shape };
        e = cudaLaunchKernel(k.fn, dim3(sms * k.blocks_per_sm), dim3(k.threads), args, 0, st);
        if (e != cudaSuccess) return cuda_fail(e, "static batch launch");
    }
    return MFA_OK;
}
