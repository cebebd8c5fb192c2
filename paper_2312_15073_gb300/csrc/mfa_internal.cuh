// mfa_internal.cuh -- device-side model description shared by the libmfa translation units.
//
// Data layout in HBM (one model):
//   * window array  W[(n_z+4)][(n_y+4)][(n_x+4)] of layer-pair entries: entry (k, j, i)
//     holds the eight control points P[k+r][j][i+a], a = 0..3, r = 0..1 (zero past the
//     end), interleaved as {P[k][j][i+a], P[k+1][j][i+a]} column pairs: 32 bytes (FP32
//     storage) or 16 bytes (FP16 / BF16).  One aligned 256-bit load then fetches the same
//     x-row of two z-layers of a (p+1)^3 support for p <= 3 (plus 16 bytes for p = 4), and
//     each column pair is a ready operand of a packed FP32x2 FMA that advances both
//     layers.  Costs 8x the plain array.  Degree class Q = 3 (degree <= 2) appends the row
//     of the third layer, P[k+2][j][i..i+3], and pads the entry to 16 values, so that one
//     256-bit and one 128-bit load fetch a whole z-column of a support row (16x the plain
//     array); window_values(Q) is the entry size in values.
//     FP32 models of degree class Q <= 4 store, in place of each row's control points
//     P[.][j][i..i+Q-1], the row's
//     polynomial on x span i in power form, W_c = sum_r c_{c,r} P[.][j][i+r] (c_{c,r} the
//     power-basis coefficients of span i's basis functions in its local coordinate t),
//     computed in FP64 from the stored values and rounded once; rows of entries past the
//     last span are zero.  16-bit models (and degree class 5) store the control points.
//   * raw  the stored control points as a plain [n_z][n_y][n_x] array (storage type): the
//     model's values, read by the statistics, the cell bounds, checkpoints and the bricks.
//   * per axis: kup[n+p+1]  the FP64 knots rounded UP to FP32, so that for an FP32
//     coordinate u, (u >= kup[s]) is exactly (u >= U[s]) in real arithmetic;
//     grid[G]  (G = 4 (n - p)) the span containing g / G, a starting guess for the span
//     search; rec[(n-p) * RS(Q)]  one record per knot span: {U_s, 1/h, lo, hi, c[k][r]}
//     with lo = kup[s], hi = kup[s+1] (+inf for the last span) -- an FP32 coordinate u
//     lies in span s iff lo <= u < hi -- and c[k][r] (k = 0..Q-1, r = 0..QP-1, QP = Q
//     rounded up to even) the power-basis
//     coefficient of t^k of N_{s-p+r,p} on that span, t = (u - U_s)/h, h = U_{s+1} - U_s
//     (computed in FP64, rounded to FP32; zero for r > p).  Power-major order puts the
//     coefficients of functions r and r+1 side by side, so one 64-bit register pair feeds
//     a packed FP32x2 FMA that advances two basis functions at once.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mfa {

constexpr int kMaxDegree = 4;
constexpr int kMaxQ = kMaxDegree + 1;
constexpr int kTfMax = 256;
constexpr int kPad = 4;                 // zero padding added to every axis of the window array

// basis functions per axis rounded up to pairs, and floats per span record for
// Q = p_max + 1: {U_s, 1/h, lo, hi} + Q*QP coefficients, padded to float4
constexpr int kRecHead = 4;
__host__ __device__ constexpr int window_values(int q) { return q == 3 ? 16 : 8; }
__host__ __device__ constexpr int qpair(int q) { return (q + 1) / 2 * 2; }
__host__ __device__ constexpr int rec_stride(int q) { return ((kRecHead + q * qpair(q)) + 3) / 4 * 4; }
// Window types (ModelDev::storage, a kernel template parameter): 1..3 layer-pair windows
// with FP32 / FP16 / BF16 values; 4..6 the compact layout of FP32 / FP16 / BF16 values:
// the zero-padded plain array [n_z+4][n_y+4][nxp] (nxp = n_x+4 rounded up to a multiple of
// the stride S = compact_stride(q, storage)) kept as entries of V = compact_values(storage)
// values, entry e of an x-row holding its values S e .. S e + V - 1, from which the kernels
// gather layer pairs row by row (one 16-byte load per 16-bit row, two per FP32 row): V/S
// times the padded plain array, 1x FP32 and 1.6x FP16 / BF16 at degree 3, instead of 8x.
constexpr int kWindowTypes = 6;
// Compact entries of window type storage (4..6) and degree class q: compact_values values
// each, one every compact_stride positions of a padded x-row.  16-bit types: eight values
// every 9 - q positions, so that a row of q values starting at any of an entry's first
// 9 - q positions lies inside it (one 16-byte load per row, 8 / (9 - q) times the plain
// array).  FP32: four values every four positions, the plain array itself, a row read as
// its entry and the next one (two 16-byte loads); at 1.6x the FP32 values of a 256^3 model
// no longer stay in L2, which costs more than the second load.
__host__ __device__ constexpr int compact_stride(int q, int storage) { return storage == 4 ? 4 : 9 - q; }
__host__ __device__ constexpr int compact_values(int storage) { return storage == 4 ? 4 : 8; }
__host__ __device__ constexpr bool compact_window(int storage) { return storage >= 4; }
__host__ __device__ constexpr int window_value_type(int storage) { return storage >= 4 ? storage - 3 : storage; }

// Whether a model's window rows hold power forms (FP32, degree classes 2..4) rather than
// control points: degree class 5 (degree 4) keeps control points on every storage type,
// since its rows share their fifth column with the next entry, which leaves no room for a
// fifth coefficient of their own.
__host__ __device__ constexpr bool power_rows(int q, int storage) { return storage == 1 && q <= 4; }

// Debug builds (compiled with -DMFA_DEBUG) check every window, span-record, cell and
// transfer-function index before its load.  A bad index sets a bit of the device's debug
// word (dbg[0]), counts itself in dbg[1] and is replaced by 0, so the kernel completes and
// the host reads the word with mfa_debug_status; nothing traps.  Release builds compile the
// checks away (dbg stays NULL).
enum : unsigned { kDbgWindow = 1u, kDbgRecord = 2u, kDbgCell = 4u, kDbgTf = 8u };
#ifdef MFA_DEBUG
__device__ __forceinline__ long long dbg_index(unsigned* dbg, long long i, long long n, unsigned bit)
{
    if (i >= 0 && i < n) return i;
    if (dbg) {
        atomicOr(dbg, bit);
        atomicAdd(dbg + 1, 1u);
    }
    return 0;
}
#define MFA_DBG_INDEX(dbg, i, n, bit) ((i) = static_cast<decltype(i)>(dbg_index((dbg), (i), (n), (bit))))
#else
#define MFA_DBG_INDEX(dbg, i, n, bit) ((void)0)
#endif

struct AxisDev {
    const float* kup;   // n + p + 1 knots rounded up to FP32
    const float* rec;   // n - p span records of rec_stride(Q) floats
    const int* grid;    // G starting spans
    int n, p;           // control points and degree on this axis
    int G;              // grid cells
    float Gf;           // (float)G
    unsigned* dbg;      // debug word (debug builds) or NULL
};

struct ModelDev {
    AxisDev ax[3];
    const void* win;    // window array (see above)
    const float* patch; // per knot-span cell (i, j, k) (x fastest), its 64 polynomial coefficients
                        // c[a][b][c] of t_x^a t_y^b t_z^c (degree 3, FP32) as 8 entries of the
                        // layer-pair layout: entry 4m + b holds {c[a][b][2m], c[a][b][2m+1]},
                        // a = 0..3 (MFA_WINDOW_PATCH models only, else NULL)
    const void* raw;    // the stored control points, plain [n_z][n_y][n_x], of type raw_storage
                        // (NULL on compact models, whose window holds them)
    int nxp, nyp, nzp;  // padded sizes n + kPad
    int q;              // Q = max degree + 1 (kernel template parameter)
    int storage;        // window type (kernel template parameter): 1..3 layer pairs of FP32 / FP16
                        // / BF16 values, 4..6 compact entries of FP32 / FP16 / BF16 values
    int raw_storage;    // mfa_dtype of the stored control points (FP32 windows may hold 16-bit values)
    int cardinal;       // 1: uniform knots and degree Q-1 on all three axes, so interior
                        // spans share the cardinal basis (render variant 6 applies)
    const float2* cell; // per knot-span cell (i, j, k) = (span - p per axis), x fastest:
                        // {min, max} of the stored control points of its support, which
                        // bound the model on the cell (convex hull property); NULL on
                        // compact models (no bounds: every sample is queried)
    int ncx, ncy, ncz;  // cells per axis, n - p
    unsigned* dbg;      // debug word (debug builds) or NULL
};

// Per-image render parameters (camera frame, image size, transfer-function scalars).
struct RenderScalars {
    float eye[3];       // ray origin (perspective) / view centre (orthographic)
    float fwd[3];       // unit view direction
    float rx[3];        // image-plane step for sx in [-1,1]: right * half-width (ortho) or
                        // right * tan(fov/2) * aspect (perspective)
    float uy[3];        // same for sy: up * half-height or up * tan(fov/2)
    int projection;     // 0 ortho, 1 perspective
    int width, height, n_samples;
    float inv_w, inv_h; // 1/width, 1/height
    float vmin, inv_range;   // transfer-function normalisation (inv_range 0 if vmax <= vmin)
    int tf_n;           // table rows
    int shading;
    float ka, kd, ks, shininess;
    float ert_alpha;    // +inf: no early termination
    float gtiny2;       // squared gradient-norm threshold for an undefined normal
    unsigned long long* samples_out;   // optional device counter
    float4* out;        // height * width premultiplied RGBA
    unsigned* dbg;      // debug word (debug builds) or NULL
    const unsigned* cell_vis;   // variant 7: bit c set where knot-span cell c can be visible
                                // under this transfer function (NULL: every cell)
};

// Single-image launch: the scalars and the table travel as kernel arguments (about 4.3 KB).
struct RenderParams {
    RenderScalars s;
    float4 tf[kTfMax];  // non-premultiplied RGBA rows
};

// One request of a batched launch, in the device work table.
struct BatchItem {
    ModelDev m;
    RenderScalars s;
    const float4* tf;   // device copy of the request's table (tf_n rows)
    int tile_begin;     // index of the request's first ray tile in the batch
    int tiles_x;        // ray tiles per image row
    int pad[2];
};

// Device work table of a batch: kBatchGroups heads (one per degree class x storage type)
// at its start, then the items of every group back to back, then the requests'
// transfer-function rows.  A head holds the tile counter its group's persistent CTAs draw
// from, the group's item count and ray-tile count, and where its items start.
struct BatchHead {
    int next_tile;
    int n_items;
    int total_tiles;
    int items_offset;   // bytes from the start of the table
};
// Groups: (record / cardinal path) x window type x (Q = 2..5), and one group of models with
// per-cell patches (cardinal path, degree class 4, FP32 window values).
constexpr int kPatchGroup = 2 * kWindowTypes * 4;
constexpr int kBatchGroups = kPatchGroup + 1;
constexpr int kBatchItemsOffset = 1024;   // heads occupy the first 1024 bytes
static_assert(kBatchGroups * sizeof(BatchHead) <= kBatchItemsOffset, "batch heads overflow");
static_assert(kBatchGroups <= 64, "group sets are 64-bit masks");
__host__ __device__ constexpr int batch_group(int q, int storage, int cardinal, bool patch)
{
    return patch ? kPatchGroup : (cardinal * kWindowTypes + (storage - 1)) * 4 + (q - 2);
}
__host__ __device__ constexpr int batch_group_q(int g) { return g == kPatchGroup ? 4 : g % 4 + 2; }
__host__ __device__ constexpr int batch_group_storage(int g) { return g == kPatchGroup ? 1 : g / 4 % kWindowTypes + 1; }
__host__ __device__ constexpr int batch_group_cardinal(int g) { return g == kPatchGroup ? 1 : g / (4 * kWindowTypes); }
__host__ __device__ constexpr bool batch_group_patch(int g) { return g == kPatchGroup; }

// launchers (defined in the .cu files), all asynchronous on `stream`
cudaError_t launch_prep_axis(const double* d_knots, int n, int p, int q, float* kup, float* rec, int* grid,
                             int G, double* coef64, cudaStream_t stream);
// the stored control points (plain array in the storage type) from the input
cudaError_t launch_prep_raw(const void* d_ctrl, int in_dtype, int storage, long long total, void* raw,
                            cudaStream_t stream);
// the window array from the stored control points (coef64: the x axis's FP64 span
// coefficients for FP32 power rows, NULL for 16-bit rows)
cudaError_t launch_prep_window(const void* raw, int raw_storage, int nx, int ny, int nz, int nxp, int q,
                               const double* coef64, int px, void* win, int storage, cudaStream_t stream);
// The per-cell polynomial patches (degree 3 on every axis; layout at ModelDev::patch) from
// the stored control points and each axis's FP64 span coefficients coef64[a] ([span][k][r]).
cudaError_t launch_prep_patches(const void* raw, int raw_storage, const int nctrl[3], const double* const coef64[3],
                                float* patch, cudaStream_t stream);
cudaError_t launch_prep_cells(const void* raw, int storage, const int degree[3], const int nctrl[3], float2* cell,
                              cudaStream_t stream);
cudaError_t launch_prep_stats(const void* raw, int storage, long long total, int* d_stats, cudaStream_t stream);
cudaError_t launch_decode(const ModelDev& m, const float* pts, long long n, float* val, float* grad,
                          cudaStream_t stream);
cudaError_t launch_spans(const ModelDev& m, const float* pts, long long n, int* spans, cudaStream_t stream);
cudaError_t launch_render(const ModelDev& m, const RenderParams& rp, int variant, int shape, cudaStream_t stream);
// Variant 7's visibility bits (one per knot-span cell, (ncx ncy ncz + 31) / 32 words).
cudaError_t launch_cell_visibility(const ModelDev& m, const RenderParams& rp, unsigned* bits, cudaStream_t stream);
// Object-space decomposition into g[0] x g[1] x g[2] blocks (at most 64): every block's ray
// segments into partial[block][height][width] (the variant picks the cardinal path unless
// it is 4), then their over-merge into s.out.
cudaError_t launch_render_segments(const ModelDev& m, const RenderParams& rp, int variant, int shape, const int g[3],
                                   float4* partial, cudaStream_t stream);
cudaError_t launch_merge_segments(const RenderScalars& s, const int g[3], const float4* partial, cudaStream_t stream);
// The persistent batched render kernel for models of one degree class q, one storage type
// and one path (cardinal or record): arguments (BatchHead* table, int group, int
// tile_shape).  Launch with `threads` threads per CTA and about SMs x blocks_per_sm CTAs.
struct BatchKernel {
    const void* fn;
    int blocks_per_sm;
    int threads;
};
BatchKernel render_batch_kernel(int q, int storage, int cardinal, bool patch);

// Serving work queue (mfa_server_*, device-queue mode).  Each admitted request occupies a
// record of a ring in device memory; a request's ray tiles are claimed by atomicAdd on the
// record's ticket word, whose high half is the record's generation (bumped every time the
// record is reused) and whose low half counts claimed tiles.  A claim is valid when its
// generation is the record's current one and its tile index is below the record's tile
// count; the host rewrites a record only after every tile of its previous generation is
// done, so a valid claim always renders with the data it was published with.  The host
// keeps the list of active records sorted by its priority and rewrites it on every change.
constexpr int kServeMaxActive = 256;
struct ServeRecord {
    unsigned long long ticket;   // (generation << 32) + next tile
    int gen;                     // generation of the data below
    int total_tiles;
    int done_tiles;              // tiles finished (reset to 0 on publication)
    int group;                   // batch_group() of the request's model
    BatchItem item;              // model, camera, table scalars, output (tf points at tf below)
    float4 tf[kTfMax];           // the request's transfer-function rows
};
struct ServeQueue {
    int n_active;
    int pad[3];
    int active[kServeMaxActive];   // record indices, most urgent first
};
// The persistent serving kernel of one (degree class, storage, path) group: arguments
// (ServeRecord* records, const ServeQueue* queue, unsigned* done (host-mapped: done[r] =
// generation once record r's last tile is finished), int group, int tile_shape).  Its CTAs
// claim tiles of the group's active records in list order and exit when none is left.
BatchKernel render_serve_kernel(int q, int storage, int cardinal, bool patch);
// Pixel size of ray-tile shape `shape` (0..kTileShapes-1); -1 if out of range.
int render_tile_dims(int shape, int* tw, int* th);
constexpr int kTileShapes = 4;

}  // namespace mfa
