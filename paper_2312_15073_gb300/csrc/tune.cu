// tune.cu -- the autotuner: picks the render kernel variant and ray-tile shape for a
// workload by timing every candidate on the GPU, and keeps the choices per workload class
// (the mfa_tune_* calls of include/mfa.h).
//
// A workload class is (degree class Q, storage type, image pixels in powers of 4, samples
// per ray in powers of 2, knot layout uniform or not, largest control-point count per axis
// in powers of 2): the relative speed of the candidates depends on how many samples a ray
// spends per knot span and how many knot spans a warp's rays cover (shared-memory bricks
// win when both are small), which these capture.  Timing uses CUDA events on the calling
// thread's stream around `reps` launches after one warm-up launch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

#include "host.cuh"

using namespace mfa;

namespace {

using Key = std::tuple<int, int, int, int, int, int>;

std::mutex g_mu;
std::map<Key, mfa_tune_result> g_cache;
bool g_env_read = false;   // MFA_TUNE_CACHE consulted (first use of the cache)

// Reads the choices in `path` into the cache (g_mu held); returns how many were read, or
// -1 if the file cannot be opened.
int read_cache_file(const char* path)
{
    FILE* f = std::fopen(path, "r");
    if (!f) return -1;
    char line[256];
    int loaded = 0;
    while (std::fgets(line, sizeof line, f)) {
        if (line[0] == '#') continue;
        int q, s, pb, sb, u, nb, v, t;
        float ms;
        if (std::sscanf(line, "%d %d %d %d %d %d %d %d %f", &q, &s, &pb, &sb, &u, &nb, &v, &t, &ms) != 9) continue;
        if (v < 1 || v > 8 || t < 0 || t >= kTileShapes) continue;
        g_cache[Key(q, s, pb, sb, u, nb)] = mfa_tune_result{ v, t, ms };
        ++loaded;
    }
    std::fclose(f);
    return loaded;
}

// Writes the cache to `path` (g_mu held); false if the file cannot be written.
bool write_cache_file(const char* path)
{
    FILE* f = std::fopen(path, "w");
    if (!f) return false;
    std::fprintf(f, "# q storage pixel_bucket sample_bucket uniform size_bucket variant tile_shape ms\n");
    for (const auto& kv : g_cache)
        std::fprintf(f, "%d %d %d %d %d %d %d %d %.6f\n", std::get<0>(kv.first), std::get<1>(kv.first),
                     std::get<2>(kv.first), std::get<3>(kv.first), std::get<4>(kv.first), std::get<5>(kv.first),
                     kv.second.variant, kv.second.tile_shape, kv.second.ms);
    return std::fclose(f) == 0;
}

// The environment's persistent cache: MFA_TUNE_CACHE names a file whose choices are read
// on the first use of the cache (a missing file is an empty cache) and which every tuning
// run rewrites.  (g_mu held.)
const char* env_cache_path()
{
    const char* p = std::getenv("MFA_TUNE_CACHE");
    return p && *p ? p : nullptr;
}
void read_env_cache()
{
    if (g_env_read) return;
    g_env_read = true;
    if (const char* p = env_cache_path()) read_cache_file(p);
}

int log_bucket(double x, double base) { return x <= 1.0 ? 0 : static_cast<int>(std::floor(std::log(x) / std::log(base))); }

Key key_of(const mfa_model* m, int w, int h, int ns)
{
    // uniform knots <=> every axis's first interior knot sits at 1/(n-p) (the library builds
    // them that way when the caller passes NULL); other layouts share one class
    const int nmax = std::max(m->nctrl[0], std::max(m->nctrl[1], m->nctrl[2]));
    return Key(m->dev.q, m->dev.storage, log_bucket(static_cast<double>(w) * h, 4.0),
               log_bucket(ns, 2.0), m->uniform ? 1 : 0, log_bucket(nmax, 2.0));
}

}  // namespace

namespace mfa {

bool tuned_lookup(const mfa_model* m, int w, int h, int ns, int* variant, int* shape)
{
    std::lock_guard<std::mutex> g(g_mu);
    read_env_cache();
    auto it = g_cache.find(key_of(m, w, h, ns));
    if (it == g_cache.end()) return false;
    *variant = it->second.variant;
    *shape = it->second.tile_shape;
    return true;
}

}  // namespace mfa

extern "C" {

int mfa_tune_render(const mfa_model* m, const mfa_camera* cam, const mfa_transfer_fn* tf, int width, int height,
                    int n_samples, float* rgba_out, int reps, mfa_tune_result* best, mfa_tune_result* all, int max_all,
                    int* n_all)
{
    if (!best) return fail(MFA_ERR_ARG, "best is NULL");
    if (reps < 1 || reps > 1000) return fail(MFA_ERR_ARG, "reps = %d outside 1..1000", reps);
    cudaStream_t st = current_stream();
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e != cudaSuccess) return cuda_fail(e, "tuner events");
    mfa_tune_result top{ 0, 0, INFINITY }, top_skip{ 0, 0, INFINITY };   // top: variants 1-6
    int count = 0, rc = MFA_OK;
    // 6 is the cardinal path (cardinal models only), 7 empty-space skipping
    const bool cardinal = m && m->dev.cardinal;
    const bool patch = m && m->dev.patch;
    for (int variant = 1; variant <= 8 && rc == MFA_OK; ++variant) {
        if (variant == 6 && !cardinal) continue;
        if (variant == 8 && !patch) continue;
        for (int shape = 0; shape < kTileShapes && rc == MFA_OK; ++shape) {
            mfa_render_opts o{};
            o.variant = variant;
            o.tile_shape = shape;
            rc = mfa_render_ex(m, cam, tf, width, height, n_samples, rgba_out, &o);   // warm-up (and validation)
            if (rc != MFA_OK) break;
            cudaEventRecord(a, st);
            for (int r = 0; r < reps && rc == MFA_OK; ++r) rc = mfa_render_ex(m, cam, tf, width, height, n_samples, rgba_out, &o);
            cudaEventRecord(b, st);
            if ((e = cudaEventSynchronize(b)) != cudaSuccess) {
                rc = cuda_fail(e, "tuner timing");
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, a, b);
            const mfa_tune_result r{ variant, shape, ms / reps };
            if (all && count < max_all) all[count] = r;
            ++count;
            mfa_tune_result& t = variant == 7 ? top_skip : top;
            if (r.ms < t.ms) t = r;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc != MFA_OK) return rc;
    // variant 7 adds a visibility pass to variant 6's work: it is taken only where it skips
    // enough to be clearly faster (2 %), not on timing noise where nothing is transparent
    if (top_skip.ms < 0.98f * top.ms) top = top_skip;
    if (n_all) *n_all = count;
    *best = top;
    std::lock_guard<std::mutex> g(g_mu);
    read_env_cache();
    g_cache[key_of(m, width, height, n_samples)] = top;
    if (const char* p = env_cache_path())
        if (!write_cache_file(p)) return fail(MFA_ERR_ARG, "cannot write MFA_TUNE_CACHE file %s", p);
    return MFA_OK;
}

int mfa_tune_batch(mfa_batch* batch, const mfa_render_request* reqs, int n, int reps, mfa_tune_result* best)
{
    if (!batch || !best) return fail(MFA_ERR_ARG, "batch and best must be non-NULL");
    if (reps < 1 || reps > 1000) return fail(MFA_ERR_ARG, "reps = %d outside 1..1000", reps);
    cudaStream_t st = current_stream();
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e != cudaSuccess) return cuda_fail(e, "tuner events");
    mfa_tune_result top{ 4, 0, INFINITY };
    int rc = MFA_OK;
    for (int shape = 0; shape < kTileShapes && rc == MFA_OK; ++shape) {
        if ((rc = mfa_batch_configure(batch, shape, 0)) != MFA_OK) break;
        if ((rc = mfa_batch_render(batch, reqs, n)) != MFA_OK) break;   // warm-up, builds the graph
        cudaEventRecord(a, st);
        for (int r = 0; r < reps && rc == MFA_OK; ++r) rc = mfa_batch_render(batch, reqs, n);
        cudaEventRecord(b, st);
        if ((e = cudaEventSynchronize(b)) != cudaSuccess) {
            rc = cuda_fail(e, "tuner timing");
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms / reps < top.ms) top = mfa_tune_result{ 4, shape, ms / reps };
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc != MFA_OK) return rc;
    *best = top;
    return mfa_batch_configure(batch, top.tile_shape, 0);
}

int mfa_tune_lookup(const mfa_model* m, int width, int height, int n_samples, mfa_tune_result* out)
{
    if (!m || !out) return fail(MFA_ERR_ARG, "model and out must be non-NULL");
    std::lock_guard<std::mutex> g(g_mu);
    read_env_cache();
    auto it = g_cache.find(key_of(m, width, height, n_samples));
    if (it == g_cache.end()) return fail(MFA_ERR_ARG, "no tuned choice for this workload class");
    *out = it->second;
    return MFA_OK;
}

int mfa_tune_save(const char* path)
{
    if (!path) return fail(MFA_ERR_ARG, "path is NULL");
    std::lock_guard<std::mutex> g(g_mu);
    read_env_cache();
    return write_cache_file(path) ? MFA_OK : fail(MFA_ERR_ARG, "cannot write %s", path);
}

int mfa_tune_load(const char* path)
{
    if (!path) return fail(MFA_ERR_ARG, "path is NULL");
    std::lock_guard<std::mutex> g(g_mu);
    read_env_cache();
    const int loaded = read_cache_file(path);
    if (loaded < 0) return fail(MFA_ERR_ARG, "cannot read %s", path);
    return loaded > 0 ? MFA_OK : fail(MFA_ERR_ARG, "no tuning entries in %s", path);
}

}  // extern "C"
