// server.cu -- render serving: resident models, camera-view requests admitted by an HBM
// budget, continuously joined onto the running work, p50/p99 latency (the mfa_server_*
// calls of include/mfa.h).
//
// The paper's concern is input latency: every view or transfer-function change re-runs
// the pipeline (Sec. IV-B, Sec. V-C).  A server thread owns a queue of submitted requests.
// A request is admitted when a slot is free and its output image fits in the HBM arena
// (one device allocation of the budget, sub-allocated on the host).  Two ways to run the
// admitted requests:
//   * device work queue (default): the request is published as a record of a ring in
//     device memory and inserted into the active list, which the host keeps ordered by
//     urgency (arrival time, plus the request's work at a configured sample rate when
//     one is given, so that small views go first without overtaking a large one forever).  Persistent
//     kernels (one per degree class, storage type and path) draw ray tiles from the list;
//     the server launches one after each publication (round-robin over a few streams, so
//     that it never waits behind an earlier kernel's last CTAs), and CTAs already running
//     take the new request's tiles at their next claim, so requests join the running batch
//     at tile granularity.  The CTA finishing a request's last tile writes the record's
//     generation to host-mapped memory, which the server thread polls.
//   * stream per request: each admitted request is launched at once as a one-CTA-per-tile
//     render on a stream whose priority grows as its work shrinks; the block scheduler
//     hands freed SMs to the highest-priority pending tiles; completion is stamped by a
//     host callback.
// Latency runs from the request's arrival time (given by the client, or the submit time) to
// the completion stamp.  No device-side wait is involved anywhere; every host wait has a
// timeout.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstddef>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "host.cuh"

using namespace mfa;

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration_cast<duration<double>>(steady_clock::now().time_since_epoch()).count();
}

// First-fit sub-allocator over one device range; host bookkeeping only.
class Arena {
public:
    void init(char* base, size_t bytes)
    {
        base_ = base;
        free_.clear();
        free_[0] = bytes;
        used_ = 0;
    }
    // offset of a block of `bytes` (256-aligned), or -1
    long long alloc(size_t bytes)
    {
        bytes = (bytes + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > bytes) free_[off + bytes] = len - bytes;
                used_ += bytes;
                sizes_[off] = bytes;
                return static_cast<long long>(off);
            }
        }
        return -1;
    }
    void release(size_t off)
    {
        auto s = sizes_.find(off);
        if (s == sizes_.end()) return;
        size_t len = s->second;
        sizes_.erase(s);
        used_ -= len;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + len == next->first) {
            len += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += len;
                return;
            }
        }
        free_[off] = len;
    }
    char* base() const { return base_; }
    size_t used() const { return used_; }

private:
    char* base_ = nullptr;
    std::map<size_t, size_t> free_;    // offset -> length
    std::map<size_t, size_t> sizes_;   // live offset -> length
    size_t used_ = 0;
};

enum TicketState { kQueued = 0, kRunning = 1, kDone = 2, kFailed = 3, kCancelled = 4 };

struct Ticket {
    long long id = 0;
    int state = kQueued;
    int record = -1;                     // device-queue mode: ring record and its generation
    int gen = 0;
    double deadline = 0;                 // device-queue mode: urgency key
    const mfa_model* model = nullptr;
    mfa_camera camera{};
    mfa_transfer_fn tf{};
    std::vector<float> table;            // the request's own copy of the TF rows
    int width = 0, height = 0, n_samples = 0;
    size_t bytes = 0;
    long long offset = -1;               // arena offset of the image once admitted
    double t_arrival = 0, t_admit = 0, t_done = 0;
    int stream = 0;
    mfa_server* server = nullptr;
    int error = 0;
};

}  // namespace

struct mfa_server {
    mfa_server_config cfg{};
    int device = 0;
    void* arena_mem = nullptr;
    Arena arena;
    std::vector<cudaStream_t> streams;   // index 0 = highest priority
    // device-queue mode
    int n_records = 0;
    ServeRecord* d_recs = nullptr;       // ring of records (device)
    ServeRecord* h_recs = nullptr;       // their pinned host images (copy sources)
    ServeQueue* d_queue = nullptr;       // active list (device)
    ServeQueue* h_queue = nullptr;       // pinned staging, kQueueSlots copies used in turn
    cudaEvent_t queue_ev[4] = {};
    int queue_next = 0;
    unsigned* h_done = nullptr;          // host-mapped completion words, one per record
    unsigned* d_done = nullptr;
    std::vector<int> free_records;
    std::vector<int> record_gen;
    std::vector<Ticket*> running;        // published, not yet complete
    cudaStream_t publish = nullptr;      // record and list uploads
    // persistent kernels go round-robin over several streams: a kernel whose last CTAs are
    // still finishing tiles must not hold back the next launch (which would leave the new
    // requests' tiles to those few CTAs)
    static constexpr int kLaunchStreams = 8;
    cudaStream_t launch_stream[kLaunchStreams] = {};
    int launch_next = 0;
    int sms = 0;
    std::mutex mu;
    std::condition_variable cv;          // wakes the scheduler
    std::condition_variable done_cv;     // wakes waiters
    std::deque<Ticket*> queue;
    std::unordered_map<long long, Ticket*> tickets;
    std::vector<Ticket*> cancelled_keep;   // released while queued; freed at destroy
    long long next_id = 1;
    int in_flight = 0;
    bool stop = false;
    std::thread worker;
    mfa_server_stats stats{};
};

namespace {

void CUDART_CB on_done(void* arg)
{
    Ticket* t = static_cast<Ticket*>(arg);
    mfa_server* s = t->server;
    {
        std::lock_guard<std::mutex> g(s->mu);
        t->t_done = now_s();
        t->state = kDone;
        --s->in_flight;
        ++s->stats.completed;
    }
    s->cv.notify_all();
    s->done_cv.notify_all();
}

// Stream for a request: more work -> lower priority (index), log4 buckets.
int stream_for(const mfa_server* s, const Ticket* t)
{
    const double work = static_cast<double>(t->width) * t->height * t->n_samples;
    int lvl = 0;
    for (double w = 1 << 26; w < work && lvl + 1 < static_cast<int>(s->streams.size()); w *= 4.0) ++lvl;
    return lvl;
}

// Launches one admitted request (called with the mutex NOT held).
int launch(mfa_server* s, Ticket* t)
{
    cudaSetDevice(s->device);
    t->tf.rgba = t->table.data();
    mfa_render_opts opts;
    std::memset(&opts, 0, sizeof opts);
    opts.variant = s->cfg.variant;
    opts.tile_shape = s->cfg.tile_shape;
    opts.use_tuned = s->cfg.use_tuned;
    cudaStream_t st = s->streams[t->stream];
    mfa_set_stream(st);
    int rc = mfa_render_ex(t->model, &t->camera, &t->tf, t->width, t->height, t->n_samples,
                           reinterpret_cast<float*>(s->arena.base() + t->offset), &opts);
    if (rc == MFA_OK) {
        cudaError_t e = cudaLaunchHostFunc(st, on_done, t);
        if (e != cudaSuccess) rc = cuda_fail(e, "completion callback");
    }
    return rc;
}

// ---------------------------------------------------------------------------------------
// device work queue
// ---------------------------------------------------------------------------------------

// Fills the host image of record r for ticket t (scalars, model, table rows, tile count)
// and enqueues its upload: the body first, then the ticket word that opens it for claims.
// Returns the request's kernel group, or a negative MFA status.
int publish_record(mfa_server* s, Ticket* t, int r)
{
    ServeRecord& R = s->h_recs[r];
    t->tf.rgba = t->table.data();
    std::memset(&R.item, 0, sizeof R.item);
    int rc = setup_render(t->model, &t->camera, &t->tf, t->width, t->height, t->n_samples,
                          reinterpret_cast<float*>(s->arena.base() + t->offset), nullptr, R.item.s, R.tf);
    if (rc != MFA_OK) return rc;
    int tw, th;
    render_tile_dims(s->cfg.tile_shape, &tw, &th);
    R.item.m = t->model->dev;
    R.item.tiles_x = (t->width + tw - 1) / tw;
    R.item.tile_begin = 0;
    R.item.tf = s->d_recs[r].tf;
    R.gen = t->gen;
    R.total_tiles = R.item.tiles_x * ((t->height + th - 1) / th);
    R.done_tiles = 0;
    const ModelDev& md = t->model->dev;
    R.group = batch_group(md.q, md.storage, md.cardinal, md.patch != nullptr && md.cardinal);
    R.ticket = static_cast<unsigned long long>(static_cast<unsigned>(t->gen)) << 32;
    const size_t body = offsetof(ServeRecord, gen);
    cudaError_t e = cudaMemcpyAsync(reinterpret_cast<char*>(s->d_recs + r) + body, reinterpret_cast<char*>(&R) + body,
                                    sizeof(ServeRecord) - body, cudaMemcpyHostToDevice, s->publish);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&s->d_recs[r].ticket, &R.ticket, sizeof R.ticket, cudaMemcpyHostToDevice, s->publish);
    return e == cudaSuccess ? R.group : cuda_fail(e, "publish request");
}

// Uploads the active list (records most urgent first) through the next staging copy.
cudaError_t publish_list(mfa_server* s, const std::vector<int>& order)
{
    const int slot = s->queue_next;
    s->queue_next = (slot + 1) % 4;
    cudaError_t e = cudaEventSynchronize(s->queue_ev[slot]);   // its previous upload has been read
    if (e != cudaSuccess) return e;
    ServeQueue& Qh = s->h_queue[slot];
    Qh.n_active = static_cast<int>(order.size());
    for (size_t i = 0; i < order.size(); ++i) Qh.active[i] = order[i];
    e = cudaMemcpyAsync(s->d_queue, &Qh, offsetof(ServeQueue, active) + sizeof(int) * order.size(),
                        cudaMemcpyHostToDevice, s->publish);
    if (e == cudaSuccess) e = cudaEventRecord(s->queue_ev[slot], s->publish);
    return e;
}

// Publishes the admitted tickets (records assigned), the new active list, and launches one
// persistent kernel per group involved, each after the uploads.  Called without the mutex.
void publish_wave(mfa_server* s, const std::vector<Ticket*>& admitted, const std::vector<int>& order)
{
    cudaSetDevice(s->device);
    bool groups[kBatchGroups] = {};
    std::vector<Ticket*> failed;
    for (Ticket* t : admitted) {
        const int g = publish_record(s, t, t->record);
        if (g < 0) {
            t->error = g;
            failed.push_back(t);
        } else {
            groups[g] = true;
        }
    }
    cudaError_t e = publish_list(s, order);
    const int slot = (s->queue_next + 3) % 4;   // the event of the list just uploaded
    for (int g = 0; g < kBatchGroups && e == cudaSuccess; ++g) {
        if (!groups[g]) continue;
        const BatchKernel k = render_serve_kernel(batch_group_q(g), batch_group_storage(g), batch_group_cardinal(g),
                                                  batch_group_patch(g));
        ServeRecord* recs = s->d_recs;
        const ServeQueue* q = s->d_queue;
        unsigned* done = s->d_done;
        int group = g, shape = s->cfg.tile_shape;
        void* args[] = { &recs, &q, &done, &group, &shape };
        cudaStream_t st = s->launch_stream[s->launch_next];
        s->launch_next = (s->launch_next + 1) % mfa_server::kLaunchStreams;
        e = cudaStreamWaitEvent(st, s->queue_ev[slot], 0);
        if (e == cudaSuccess) e = cudaLaunchKernel(k.fn, dim3(s->sms * k.blocks_per_sm), dim3(k.threads), args, 0, st);
    }
    if (e != cudaSuccess) {
        cuda_fail(e, "serving launch");
        for (Ticket* t : admitted)
            if (std::find(failed.begin(), failed.end(), t) == failed.end()) {
                t->error = MFA_ERR_CUDA;
                failed.push_back(t);
            }
    }
    if (!failed.empty()) {
        std::lock_guard<std::mutex> g(s->mu);
        for (Ticket* t : failed) {
            t->state = kFailed;
            t->t_done = now_s();
            --s->in_flight;
            ++s->stats.failed;
            s->running.erase(std::remove(s->running.begin(), s->running.end(), t), s->running.end());
            s->free_records.push_back(t->record);
        }
    }
}

// Completions of the device work queue (called with the mutex held): a record whose
// host-mapped word shows its generation is done.  Returns the number completed.
int poll_done(mfa_server* s)
{
    int n = 0;
    for (size_t i = 0; i < s->running.size();) {
        Ticket* t = s->running[i];
        const unsigned w = reinterpret_cast<volatile unsigned*>(s->h_done)[t->record];
        if (w == static_cast<unsigned>(t->gen)) {
            std::atomic_thread_fence(std::memory_order_acquire);
            t->t_done = now_s();
            t->state = kDone;
            --s->in_flight;
            ++s->stats.completed;
            s->free_records.push_back(t->record);
            s->running[i] = s->running.back();
            s->running.pop_back();
            ++n;
        } else {
            ++i;
        }
    }
    return n;
}

// The active list: running records, most urgent (earliest deadline) first.
std::vector<int> active_order(const mfa_server* s)
{
    std::vector<const Ticket*> v(s->running.begin(), s->running.end());
    std::sort(v.begin(), v.end(), [](const Ticket* a, const Ticket* b) {
        return a->deadline < b->deadline || (a->deadline == b->deadline && a->id < b->id);
    });
    std::vector<int> order;
    for (const Ticket* t : v) order.push_back(t->record);
    return order;
}

void worker_main(mfa_server* s)
{
    cudaSetDevice(s->device);
    const bool queue_mode = s->cfg.mode == 0;
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        // admit in arrival order while a slot and arena memory are free
        std::vector<Ticket*> admitted;
        while (!s->queue.empty() && s->in_flight < s->cfg.max_slots) {
            Ticket* t = s->queue.front();
            if (t->state == kCancelled) {
                s->queue.pop_front();
                continue;
            }
            const long long off = s->arena.alloc(t->bytes);
            if (off < 0) break;   // wait for memory
            s->queue.pop_front();
            t->offset = off;
            t->state = kRunning;
            t->t_admit = now_s();
            t->stream = stream_for(s, t);
            if (queue_mode) {
                t->record = s->free_records.back();
                s->free_records.pop_back();
                t->gen = ++s->record_gen[t->record];
                s->running.push_back(t);
            }
            ++s->in_flight;
            s->stats.peak_in_flight = std::max<long long>(s->stats.peak_in_flight, s->in_flight);
            s->stats.peak_arena_bytes = std::max<long long>(s->stats.peak_arena_bytes, static_cast<long long>(s->arena.used()));
            admitted.push_back(t);
        }
        if (!admitted.empty() && queue_mode) {
            const std::vector<int> order = active_order(s);
            lk.unlock();
            publish_wave(s, admitted, order);
            lk.lock();
            s->done_cv.notify_all();
            continue;
        }
        if (!admitted.empty()) {
            lk.unlock();
            for (Ticket* t : admitted) {
                const int rc = launch(s, t);
                if (rc != MFA_OK) {
                    std::lock_guard<std::mutex> g(s->mu);
                    t->state = kFailed;
                    t->error = rc;
                    t->t_done = now_s();
                    --s->in_flight;
                    ++s->stats.failed;
                }
            }
            lk.lock();
            s->done_cv.notify_all();
            continue;
        }
        if (queue_mode && !s->running.empty()) {
            if (poll_done(s) > 0) {
                s->done_cv.notify_all();
                continue;   // freed slots: admit again
            }
            // poll the completions again soon: a short yield (a timed wait sleeps for the
            // timer slack, tens of microseconds, and every request would pay it)
            lk.unlock();
            std::this_thread::yield();
            lk.lock();
            continue;
        }
        s->cv.wait_for(lk, std::chrono::milliseconds(50));
    }
}

}  // namespace

extern "C" {

double mfa_server_now(void) { return now_s(); }

mfa_server* mfa_server_create(const mfa_server_config* cfg)
{
    if (!cfg) return fail(MFA_ERR_ARG, "config is NULL"), nullptr;
    if (cfg->hbm_budget_bytes < 4096) return fail(MFA_ERR_ARG, "hbm_budget_bytes must be >= 4096"), nullptr;
    if (cfg->max_slots < 1 || cfg->max_slots > 4096) return fail(MFA_ERR_ARG, "max_slots outside 1..4096"), nullptr;
    if (cfg->max_queue < 1) return fail(MFA_ERR_ARG, "max_queue must be >= 1"), nullptr;
    if (cfg->priority_levels < 1 || cfg->priority_levels > 8) return fail(MFA_ERR_ARG, "priority_levels outside 1..8"), nullptr;
    if (cfg->variant < 0 || cfg->variant > 8 || cfg->tile_shape < 0 || cfg->tile_shape >= kTileShapes)
        return fail(MFA_ERR_ARG, "variant or tile_shape out of range"), nullptr;
    if (cfg->mode != 0 && cfg->mode != 1) return fail(MFA_ERR_ARG, "mode must be 0 (device queue) or 1"), nullptr;
    if (!(cfg->urgency_rate >= 0)) return fail(MFA_ERR_ARG, "urgency_rate must be >= 0"), nullptr;
    if (cfg->mode == 0 && cfg->max_slots > kServeMaxActive)
        return fail(MFA_ERR_ARG, "the device work queue takes at most %d requests in flight", kServeMaxActive), nullptr;
    mfa_server* s = new mfa_server();
    s->cfg = *cfg;
    cudaGetDevice(&s->device);
    cudaError_t e = cudaMalloc(&s->arena_mem, cfg->hbm_budget_bytes);
    if (e != cudaSuccess) {
        cuda_fail(e, "server arena");
        delete s;
        return nullptr;
    }
    s->arena.init(static_cast<char*>(s->arena_mem), cfg->hbm_budget_bytes);
    if (cfg->mode == 0) {   // device work queue: record ring, active list, completion words
        s->n_records = cfg->max_slots;
        cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
        const size_t rec_bytes = sizeof(ServeRecord) * s->n_records;
        if (e == cudaSuccess) e = cudaMalloc(&s->d_recs, rec_bytes);
        if (e == cudaSuccess) e = cudaMemset(s->d_recs, 0, rec_bytes);
        if (e == cudaSuccess) e = cudaMallocHost(&s->h_recs, rec_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&s->d_queue, sizeof(ServeQueue));
        if (e == cudaSuccess) e = cudaMemset(s->d_queue, 0, sizeof(ServeQueue));
        if (e == cudaSuccess) e = cudaMallocHost(&s->h_queue, 4 * sizeof(ServeQueue));
        if (e == cudaSuccess) e = cudaHostAlloc(&s->h_done, sizeof(unsigned) * s->n_records, cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->d_done), s->h_done, 0);
        for (auto& ev : s->queue_ev)
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->publish, cudaStreamNonBlocking);
        for (auto& st : s->launch_stream)
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            cuda_fail(e, "server work queue");
            mfa_server_destroy(s);
            return nullptr;
        }
        std::memset(s->h_done, 0, sizeof(unsigned) * s->n_records);
        s->record_gen.assign(s->n_records, 0);
        for (int r = s->n_records - 1; r >= 0; --r) s->free_records.push_back(r);
    }
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    const int span = least - greatest;   // greatest is the most negative (highest) priority
    for (int l = 0; l < cfg->priority_levels; ++l) {
        const int prio = cfg->priority_levels == 1 ? least : greatest + (span * l) / (cfg->priority_levels - 1);
        cudaStream_t st;
        cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio);
        s->streams.push_back(st);
    }
    s->worker = std::thread(worker_main, s);
    return s;
}

int mfa_server_submit(mfa_server* s, const mfa_serve_request* req, long long* ticket)
{
    if (!s || !req || !ticket) return fail(MFA_ERR_ARG, "server, request and ticket must be non-NULL");
    if (!req->model || !req->tf || !req->tf->rgba) return fail(MFA_ERR_ARG, "request needs a model and a table");
    if (req->width < 1 || req->width > 32768 || req->height < 1 || req->height > 32768 || req->n_samples < 1 ||
        req->n_samples > (1 << 20) || req->tf->n_entries < 1 || req->tf->n_entries > kTfMax)
        return fail(MFA_ERR_ARG, "request size, samples or table out of range");
    if (req->model->device != s->device) return fail(MFA_ERR_ARG, "model lives on another device");
    const size_t bytes = static_cast<size_t>(req->width) * req->height * 16;
    if (bytes > s->cfg.hbm_budget_bytes)
        return fail(MFA_ERR_NOMEM, "image of %zu bytes exceeds the HBM budget of %zu bytes", bytes,
                    s->cfg.hbm_budget_bytes);
    Ticket* t = new Ticket();
    t->model = req->model;
    t->camera = req->camera;
    t->tf = *req->tf;
    t->table.assign(req->tf->rgba, req->tf->rgba + 4 * req->tf->n_entries);
    t->width = req->width;
    t->height = req->height;
    t->n_samples = req->n_samples;
    t->bytes = bytes;
    t->server = s;
    t->t_arrival = req->arrival_time_s > 0 ? req->arrival_time_s : now_s();
    t->deadline = t->t_arrival;   // urgency key: arrival, plus the work's head start when asked for
    if (s->cfg.urgency_rate > 0)
        t->deadline += static_cast<double>(req->width) * req->height * req->n_samples / s->cfg.urgency_rate;
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (static_cast<int>(s->queue.size()) >= s->cfg.max_queue) {
            ++s->stats.rejected_busy;
            delete t;
            return fail(MFA_ERR_BUSY, "queue full (%d requests waiting)", s->cfg.max_queue);
        }
        t->id = s->next_id++;
        s->tickets[t->id] = t;
        s->queue.push_back(t);
        ++s->stats.submitted;
        *ticket = t->id;
    }
    s->cv.notify_all();
    return MFA_OK;
}

int mfa_server_poll(mfa_server* s, long long ticket, int* state, double* latency_ms)
{
    if (!s) return fail(MFA_ERR_ARG, "server is NULL");
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return fail(MFA_ERR_ARG, "unknown ticket %lld", ticket);
    Ticket* t = it->second;
    if (state) *state = t->state;
    if (latency_ms) *latency_ms = t->state == kDone ? 1e3 * (t->t_done - t->t_arrival) : -1.0;
    return t->state == kFailed ? t->error : MFA_OK;
}

int mfa_server_wait(mfa_server* s, long long ticket, double timeout_ms, double* latency_ms)
{
    if (!s) return fail(MFA_ERR_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return fail(MFA_ERR_ARG, "unknown ticket %lld", ticket);
    Ticket* t = it->second;
    const auto until = std::chrono::steady_clock::now() +
                       std::chrono::microseconds(static_cast<long long>(std::max(0.0, timeout_ms) * 1e3));
    while (t->state == kQueued || t->state == kRunning) {
        if (s->done_cv.wait_until(lk, until) == std::cv_status::timeout &&
            (t->state == kQueued || t->state == kRunning))
            return fail(MFA_ERR_TIMEOUT, "ticket %lld not done after %.3f ms", ticket, timeout_ms);
    }
    if (latency_ms) *latency_ms = t->state == kDone ? 1e3 * (t->t_done - t->t_arrival) : -1.0;
    if (t->state == kFailed) return fail(t->error, "ticket %lld failed", ticket);
    if (t->state == kCancelled) return fail(MFA_ERR_ARG, "ticket %lld was cancelled", ticket);
    return MFA_OK;
}

int mfa_server_result(mfa_server* s, long long ticket, const float** rgba)
{
    if (!s || !rgba) return fail(MFA_ERR_ARG, "server and rgba must be non-NULL");
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return fail(MFA_ERR_ARG, "unknown ticket %lld", ticket);
    if (it->second->state != kDone) return fail(MFA_ERR_BUSY, "ticket %lld not done", ticket);
    *rgba = reinterpret_cast<const float*>(s->arena.base() + it->second->offset);
    return MFA_OK;
}

int mfa_server_copy_result(mfa_server* s, long long ticket, void* dst, size_t dst_bytes)
{
    if (!s || !dst) return fail(MFA_ERR_ARG, "server and dst must be non-NULL");
    const float* src = nullptr;
    size_t bytes = 0;
    {
        std::lock_guard<std::mutex> g(s->mu);
        auto it = s->tickets.find(ticket);
        if (it == s->tickets.end()) return fail(MFA_ERR_ARG, "unknown ticket %lld", ticket);
        if (it->second->state != kDone) return fail(MFA_ERR_BUSY, "ticket %lld not done", ticket);
        src = reinterpret_cast<const float*>(s->arena.base() + it->second->offset);
        bytes = it->second->bytes;
    }
    if (dst_bytes < bytes) return fail(MFA_ERR_ARG, "destination holds %zu bytes, the image needs %zu", dst_bytes, bytes);
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, current_stream());
    return e == cudaSuccess ? MFA_OK : cuda_fail(e, "copy result");
}

int mfa_server_release(mfa_server* s, long long ticket)
{
    if (!s) return fail(MFA_ERR_ARG, "server is NULL");
    {
        std::lock_guard<std::mutex> g(s->mu);
        auto it = s->tickets.find(ticket);
        if (it == s->tickets.end()) return fail(MFA_ERR_ARG, "unknown ticket %lld", ticket);
        Ticket* t = it->second;
        if (t->state == kRunning) return fail(MFA_ERR_BUSY, "ticket %lld still running", ticket);
        if (t->state == kQueued) {
            t->state = kCancelled;   // the scheduler drops it from the queue
            ++s->stats.cancelled;
            s->tickets.erase(it);
            // the queue still points at it: leave it to the scheduler, which skips cancelled
            // tickets; the ticket object is freed at destroy
            s->cancelled_keep.push_back(t);
            return MFA_OK;
        }
        if (t->offset >= 0) s->arena.release(static_cast<size_t>(t->offset));
        s->tickets.erase(it);
        delete t;
    }
    s->cv.notify_all();
    return MFA_OK;
}

int mfa_server_get_stats(mfa_server* s, mfa_server_stats* out)
{
    if (!s || !out) return fail(MFA_ERR_ARG, "server and out must be non-NULL");
    std::lock_guard<std::mutex> g(s->mu);
    *out = s->stats;
    out->in_flight = s->in_flight;
    out->queued = static_cast<long long>(s->queue.size());
    out->arena_bytes_in_use = static_cast<long long>(s->arena.used());
    return MFA_OK;
}

void mfa_server_destroy(mfa_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->device);
    for (cudaStream_t st : s->streams) {
        cudaStreamSynchronize(st);   // callbacks of launched requests have run after this
        cudaStreamDestroy(st);
    }
    for (cudaStream_t st : s->launch_stream)
        if (st) {
            cudaStreamSynchronize(st);   // persistent kernels have drained the queue
            cudaStreamDestroy(st);
        }
    if (s->publish) {
        cudaStreamSynchronize(s->publish);
        cudaStreamDestroy(s->publish);
    }
    for (cudaEvent_t ev : s->queue_ev)
        if (ev) cudaEventDestroy(ev);
    if (s->d_recs) cudaFree(s->d_recs);
    if (s->d_queue) cudaFree(s->d_queue);
    if (s->h_recs) cudaFreeHost(s->h_recs);
    if (s->h_queue) cudaFreeHost(s->h_queue);
    if (s->h_done) cudaFreeHost(s->h_done);
    for (auto& kv : s->tickets) delete kv.second;
    for (Ticket* t : s->cancelled_keep) delete t;
    cudaFree(s->arena_mem);
    delete s;
}

}  // extern "C"
