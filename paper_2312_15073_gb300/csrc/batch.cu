// batch.cu -- batched rendering through one CUDA-graph launch (the mfa_batch_* calls of
// include/mfa.h).
//
// A submission writes a work table on the host (pinned memory).  Requests are grouped by
// model degree class Q = p_max + 1, window type and knot path; the table holds one
// BatchHead per group (tile counter = 0, item count, tile count, where the items start),
// then each group's BatchItems (model tables, camera frame, transfer-function scalars,
// first tile index), then every request's transfer-function rows.  The graph copies the
// used part of the table to the device and then runs one persistent render kernel per
// group present, the kernels as independent branches so that one group's CTAs fill the
// SMs another group's tail leaves idle; inside a kernel the resident CTAs draw ray tiles
// of all of the group's requests from the head's counter.  Two table slots alternate so
// the host can fill one while the GPU works on the other.
#include <cstring>
#include <map>
#include <vector>

#include "host.cuh"

using namespace mfa;

namespace {

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

struct GraphEntry {
    cudaGraph_t graph = nullptr;      // kept alive: its node handles address the exec's nodes
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t copy = nullptr;   // the table upload, resized per submission
};

}  // namespace

struct mfa_batch {
    int device = 0;
    int cap = 0;
    size_t table_bytes = 0;   // capacity of one slot
    int shape = 0, grid_ctas = 0;
    struct Slot {
        void* h_table = nullptr;
        void* d_table = nullptr;
        cudaEvent_t done = nullptr;
        bool pending = false;
        std::map<unsigned long long, GraphEntry> graphs;   // per set of groups present (bit g = group g)
    } slot[2];
    int next = 0;
};

namespace {

void drop_graphs(mfa_batch* b)
{
    for (auto& s : b->slot) {
        for (auto& kv : s.graphs) {
            cudaGraphExecDestroy(kv.second.exec);
            cudaGraphDestroy(kv.second.graph);
        }
        s.graphs.clear();
    }
}

// Builds the graph for one slot and one set of groups: the table upload, then one
// persistent kernel per group, each depending only on the upload.
cudaError_t build_graph(mfa_batch* b, mfa_batch::Slot& s, unsigned long long mask, GraphEntry* out)
{
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e != cudaSuccess) return e;
    cudaGraphNode_t copy = nullptr;
    e = cudaGraphAddMemcpyNode1D(&copy, graph, nullptr, 0, s.d_table, s.h_table, b->table_bytes,
                                 cudaMemcpyHostToDevice);
    for (int g = 0; g < kBatchGroups && e == cudaSuccess; ++g) {
        if (!(mask & (1ull << g))) continue;
        const BatchKernel k = render_batch_kernel(batch_group_q(g), batch_group_storage(g), batch_group_cardinal(g),
                                                  batch_group_patch(g));
        void* table = s.d_table;
        int group = g, shape = b->shape;
        void* args[] = { &table, &group, &shape };
        cudaKernelNodeParams kp = {};
        kp.func = const_cast<void*>(k.fn);
        kp.gridDim = dim3(b->grid_ctas > 0 ? b->grid_ctas : sms * k.blocks_per_sm);
        kp.blockDim = dim3(k.threads);
        kp.kernelParams = args;
        cudaGraphNode_t node;
        e = cudaGraphAddKernelNode(&node, graph, &copy, 1, &kp);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&out->exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return e;
    }
    out->graph = graph;
    out->copy = copy;
    return e;
}

thread_local mfa_batch* t_batch = nullptr;

}  // namespace

extern "C" {

void mfa_batch_destroy(mfa_batch* b)
{
    if (!b) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    for (auto& s : b->slot)
        if (s.done) cudaEventSynchronize(s.done);
    drop_graphs(b);
    for (auto& s : b->slot) {
        if (s.done) cudaEventDestroy(s.done);
        if (s.h_table) cudaFreeHost(s.h_table);
        if (s.d_table) cudaFree(s.d_table);
    }
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    delete b;
}

mfa_batch* mfa_batch_create(int max_requests)
{
    if (max_requests < 1 || max_requests > 4096)
        return fail(MFA_ERR_ARG, "max_requests = %d outside 1..4096", max_requests), nullptr;
    mfa_batch* b = new mfa_batch();
    cudaGetDevice(&b->device);
    b->cap = max_requests;
    b->table_bytes = align256(kBatchItemsOffset + sizeof(BatchItem) * static_cast<size_t>(max_requests)) +
                     sizeof(float4) * kTfMax * static_cast<size_t>(max_requests);
    cudaError_t e = cudaSuccess;
    for (auto& s : b->slot) {
        if (e == cudaSuccess) e = cudaMallocHost(&s.h_table, b->table_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&s.d_table, b->table_bytes);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        cuda_fail(e, "batch context");
        mfa_batch_destroy(b);
        return nullptr;
    }
    return b;
}

int mfa_batch_configure(mfa_batch* b, int tile_shape, int grid_ctas)
{
    if (!b) return fail(MFA_ERR_ARG, "batch is NULL");
    int tw, th;
    if (render_tile_dims(tile_shape, &tw, &th) != 0)
        return fail(MFA_ERR_ARG, "tile_shape %d outside 0..%d", tile_shape, kTileShapes - 1);
    if (grid_ctas < 0 || grid_ctas > (1 << 20)) return fail(MFA_ERR_ARG, "grid_ctas = %d outside 0..2^20", grid_ctas);
    if (tile_shape == b->shape && grid_ctas == b->grid_ctas) return MFA_OK;
    for (auto& s : b->slot)
        if (s.done) cudaEventSynchronize(s.done);
    drop_graphs(b);
    b->shape = tile_shape;
    b->grid_ctas = grid_ctas;
    return MFA_OK;
}

int mfa_batch_render(mfa_batch* b, const mfa_render_request* reqs, int n)
{
    if (!b) return fail(MFA_ERR_ARG, "batch is NULL");
    if (n < 0 || n > b->cap) return fail(MFA_ERR_ARG, "n = %d outside 0..%d", n, b->cap);
    if (n == 0) return MFA_OK;
    if (!reqs) return fail(MFA_ERR_ARG, "reqs is NULL");
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != b->device) return fail(MFA_ERR_ARG, "batch lives on device %d but device %d is current", b->device, cur);
    int tw, th;
    render_tile_dims(b->shape, &tw, &th);

    // validate every request and build the items before touching the slot
    std::vector<BatchItem> items[kBatchGroups];
    std::vector<int> item_req[kBatchGroups];
    std::vector<float4> rows(static_cast<size_t>(n) * kTfMax);
    long long tiles[kBatchGroups] = {};
    for (int r = 0; r < n; ++r) {
        const mfa_render_request& q = reqs[r];
        if (!q.model) return fail(MFA_ERR_ARG, "request %d: model is NULL", r);
        BatchItem it;
        std::memset(&it, 0, sizeof it);
        if (int rc = setup_render(q.model, &q.camera, q.tf, q.width, q.height, q.n_samples, q.rgba_out, q.samples_out,
                                  it.s, &rows[static_cast<size_t>(r) * kTfMax])) {
            fail(rc, "request %d: %s", r, mfa_last_error());
            return rc;
        }
        const ModelDev& md = q.model->dev;
        const int g = batch_group(md.q, md.storage, md.cardinal, md.patch != nullptr && md.cardinal);
        it.m = q.model->dev;
        it.tiles_x = (q.width + tw - 1) / tw;
        const long long nt = static_cast<long long>(it.tiles_x) * ((q.height + th - 1) / th);
        it.tile_begin = static_cast<int>(tiles[g]);
        tiles[g] += nt;
        if (tiles[g] > (1LL << 30)) return fail(MFA_ERR_ARG, "batch too large: more than 2^30 ray tiles");
        items[g].push_back(it);
        item_req[g].push_back(r);
    }

    mfa_batch::Slot& s = b->slot[b->next];
    if (s.pending) {
        cudaError_t e = cudaEventSynchronize(s.done);   // the GPU is done with this slot's table
        if (e != cudaSuccess) return cuda_fail(e, "waiting for an earlier batch");
        s.pending = false;
    }
    char* h = static_cast<char*>(s.h_table);
    char* d = static_cast<char*>(s.d_table);
    BatchHead heads[kBatchGroups] = {};
    size_t off = kBatchItemsOffset;
    for (int g = 0; g < kBatchGroups; ++g) off += sizeof(BatchItem) * items[g].size();
    size_t tf_off = align256(off), tf_used = 0;
    off = kBatchItemsOffset;
    unsigned long long mask = 0;
    for (int g = 0; g < kBatchGroups; ++g) {
        heads[g].n_items = static_cast<int>(items[g].size());
        heads[g].total_tiles = static_cast<int>(tiles[g]);
        heads[g].items_offset = static_cast<int>(off);
        for (size_t k = 0; k < items[g].size(); ++k) {
            BatchItem& it = items[g][k];
            const int r = item_req[g][k];
            const size_t bytes = sizeof(float4) * it.s.tf_n;
            std::memcpy(h + tf_off + tf_used, &rows[static_cast<size_t>(r) * kTfMax], bytes);
            it.tf = reinterpret_cast<const float4*>(d + tf_off + tf_used);
            tf_used += align256(bytes);
        }
        if (!items[g].empty()) {
            std::memcpy(h + off, items[g].data(), sizeof(BatchItem) * items[g].size());
            off += sizeof(BatchItem) * items[g].size();
            mask |= 1ull << g;
        }
    }
    std::memcpy(h, heads, sizeof heads);
    const size_t used = tf_off + tf_used;

    auto found = s.graphs.find(mask);
    if (found == s.graphs.end()) {
        GraphEntry ge;
        cudaError_t e = build_graph(b, s, mask, &ge);
        if (e != cudaSuccess) return cuda_fail(e, "building the batch graph");
        found = s.graphs.emplace(mask, ge).first;
    }
    cudaError_t e = cudaGraphExecMemcpyNodeSetParams1D(found->second.exec, found->second.copy, s.d_table, s.h_table,
                                                       used, cudaMemcpyHostToDevice);
    cudaStream_t st = current_stream();
    if (e == cudaSuccess) e = cudaGraphLaunch(found->second.exec, st);
    if (e == cudaSuccess) e = cudaEventRecord(s.done, st);
    if (e != cudaSuccess) return cuda_fail(e, "batch launch");
    s.pending = true;
    b->next ^= 1;
    return MFA_OK;
}

int mfa_render_batch(const mfa_render_request* reqs, int n)
{
    if (n < 0 || n > 4096) return fail(MFA_ERR_ARG, "n = %d outside 0..4096", n);
    if (n == 0) return MFA_OK;
    int cur = -1;
    cudaGetDevice(&cur);
    if (!t_batch || t_batch->cap < n || t_batch->device != cur) {
        int cap = 16;
        while (cap < n) cap *= 2;
        mfa_batch* nb = mfa_batch_create(cap);
        if (!nb) return MFA_ERR_CUDA;
        mfa_batch_destroy(t_batch);
        t_batch = nb;
    }
    return mfa_batch_render(t_batch, reqs, n);
}

}  // extern "C"
