/*
 * mfa.h -- C ABI of libmfa: MFA value/gradient queries and MFA ray casting on one GPU.
 *
 * The MFA model (Sec. III-A) is a tensor-product B-spline volume: degrees p_x, p_y, p_z,
 * clamped knot vectors U_x, U_y, U_z on [0,1] and control points P_ijk.  Its value
 *     f(u,v,w) = sum_ijk N_{i,p_x}(u) N_{j,p_y}(v) N_{k,p_z}(w) P_ijk
 * and its analytic gradient (Sec. III-B) are the two queries every volume-visualization
 * sample makes (Sec. III-C, Sec. IV-A.4).  MFA-VV ray casting (Sec. IV-A.4) casts one ray
 * per pixel, queries value and gradient at samples along it, maps them through a user
 * transfer function with shading (Sec. IV-B) and combines neighbouring samples with the
 * over operation (Sec. IV-A.4, IV-A.5).
 *
 * Conventions shared by every call
 *  - Parameter domain = world box = the unit cube [0,1]^3, so world gradients equal
 *    parameter gradients.
 *  - Control-point arrays are [n_z][n_y][n_x] with x fastest.
 *  - Every call except mfa_model_create* returns an mfa_status (0 = MFA_OK).  Arguments
 *    are checked on the host before any launch; a rejected call launches nothing and
 *    leaves every output untouched.  mfa_last_error() returns a text for the last failure
 *    on the calling thread.
 *  - Compute calls are asynchronous on the stream bound with mfa_set_stream on the
 *    calling thread (the legacy default stream if none).  Device pointers passed in must
 *    stay valid until that stream has finished the work.  The library never frees or
 *    keeps caller buffers.
 *  - A model lives on the device that was current when it was created; calls that use it
 *    must run with that device current.
 *
 * Thread safety: distinct models may be used from distinct threads.  A model may be
 * read by many concurrent calls; destroying it while a call that uses it is running or
 * queued is the caller's error.
 */
#ifndef MFA_H
#define MFA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { MFA_F64 = 0, MFA_F32 = 1, MFA_F16 = 2, MFA_BF16 = 3 } mfa_dtype;

typedef enum {
    MFA_OK = 0,
    MFA_ERR_ARG = -1,          /* an argument is out of range or inconsistent */
    MFA_ERR_NOMEM = -2,        /* a device or host allocation failed */
    MFA_ERR_CUDA = -3,         /* a CUDA call failed; mfa_last_error() has its text */
    MFA_ERR_TIMEOUT = -4,      /* a bounded wait ran out */
    MFA_ERR_BUSY = -5,         /* no capacity right now; retry later */
    MFA_ERR_UNSUPPORTED = -6   /* valid request this build does not handle */
} mfa_status;

typedef struct mfa_model mfa_model;   /* opaque; owns all of its device memory */

/*
 * Creates an MFA model on the current device (Sec. III-A; the model-fetch step of
 * Sec. IV-A.3 becomes this one upload).
 *   degree[d]  1..4 for d = x, y, z.
 *   nctrl[d]   control points along d, >= degree[d] + 1.
 *   knots      knots[d] is a HOST array of nctrl[d] + degree[d] + 1 FP64 values,
 *              non-decreasing, clamped (the first degree+1 equal 0, the last degree+1
 *              equal 1).  knots == NULL or knots[d] == NULL selects the clamped uniform
 *              vector (interior knots i / (nctrl - degree)); caller's knots equal to
 *              it in FP64 count as uniform (mfa_model_info.cardinal: with one degree on
 *              all axes, the uniform-knot kernels apply).
 *   ctrl       HOST array of nctrl[0]*nctrl[1]*nctrl[2] values of type `dtype`,
 *              [n_z][n_y][n_x], x fastest.  Copied; the caller keeps ownership.
 *   dtype      type of ctrl.  Storage is FP32 for F64/F32 input, FP16 for F16, BF16 for
 *              BF16 (see mfa_model_create_ex to choose).
 * Device memory: the stored control points (a plain array), the padded layer-pair window
 * the kernels read -- about 32 bytes per control point with FP32 window values, 16 with
 * 16-bit ones, twice that when the largest degree is 2 (each entry also carries a third
 * layer's row) -- and 8 bytes per knot-span cell (the {min, max} bounds the isosurface
 * search reads); the product of the padded sizes (n_x+4)(n_y+4)(n_z+4) must stay below
 * 2^31.  FP32 windows of degree <= 3 hold each row's x-span polynomial in power form
 * (computed in FP64 from the stored values, rounded once to FP32).
 * Synchronous: returns after the model is ready.  Returns NULL on error (reason in
 * mfa_last_error()).
 */
mfa_model* mfa_model_create(const int degree[3], const int nctrl[3], const double* const knots[3],
                            const void* ctrl, mfa_dtype dtype);

/* As mfa_model_create, with the storage type chosen: storage_dtype is MFA_F32, MFA_F16 or
 * MFA_BF16.  Input values are rounded ONCE, to nearest even, from in_dtype to storage
 * (FP64 -> BF16 directly, never through FP32).  Basis values and all accumulation stay
 * FP32 whatever the storage type. */
mfa_model* mfa_model_create_ex(const int degree[3], const int nctrl[3], const double* const knots[3],
                               const void* ctrl, mfa_dtype in_dtype, mfa_dtype storage_dtype);

/* The window the kernels read (not a counterpart of anything in the paper: a memory /
 * speed choice of this implementation).  MFA_WINDOW_AUTO: FP32 window values for FP32
 * storage, the 16-bit values themselves for FP16 / BF16 storage (half the window bytes;
 * each value is widened to FP32 per query).  MFA_WINDOW_F32: FP32 window values whatever
 * the storage type -- the stored 16-bit values are widened exactly once, at creation, so
 * a 16-bit model computes the same sums at the speed of an FP32 one, with an FP32 model's
 * window bytes.  MFA_WINDOW_COMPACT: no layer-pair window.  FP32 models keep the zero-
 * padded plain array of their control points ((n_x+4 rounded up to a multiple of 4) x
 * (n_y+4) x (n_z+4) values; a support row is two aligned 16-byte loads); FP16 / BF16
 * models keep it as entries of eight values, one entry every S = 8 - (largest degree)
 * positions of an x-row (8/S times the plain size, 1.6x at degree 3), so that every
 * support row is one aligned 16-byte load.  Slower per query, but a model of 1-2x its
 * plain size instead of 8-16x (for models that would not otherwise fit in L2 or in
 * memory).  Compact models keep no per-cell bounds, so the isosurface search queries every
 * sample and render variant 7 falls back to the default; render variants 1, 2, 3 and 5
 * run as the default too.  MFA_WINDOW_PATCH (degree 3 on every axis; MFA_ERR_UNSUPPORTED
 * otherwise; any knots and storage type): an FP32 window (as
 * MFA_WINDOW_F32), plus per knot-span cell the 64 coefficients of the model's polynomial on
 * that cell in its local coordinates (computed in FP64 from the stored values, rounded once
 * to FP32; 256 bytes per cell, about 7x the window), which render variant 8 -- and, on
 * uniform knots, the default and the batch and serving kernels -- evaluate with monomials
 * instead of basis functions. */
enum { MFA_WINDOW_AUTO = 0, MFA_WINDOW_F32 = 1, MFA_WINDOW_COMPACT = 2, MFA_WINDOW_PATCH = 3 };

/* As mfa_model_create_ex, with the window chosen (MFA_WINDOW_*; MFA_ERR_ARG otherwise). */
mfa_model* mfa_model_create_opts(const int degree[3], const int nctrl[3], const double* const knots[3],
                                 const void* ctrl, mfa_dtype in_dtype, mfa_dtype storage_dtype, int window);

/* Frees the model and its device memory.  NULL is a no-op. */
void mfa_model_destroy(mfa_model* model);

typedef struct {
    int degree[3];
    int nctrl[3];
    mfa_dtype storage;
    float vmin, vmax;          /* min / max of the stored control points */
    size_t device_bytes;       /* device memory the model holds */
    int device;                /* CUDA ordinal the model lives on */
    int cardinal;              /* 1: uniform knots and one degree on all three axes, so
                                  decode and render take the cardinal path (interior
                                  spans share one basis; render variant 6) */
    int window;                /* the MFA_WINDOW_* choice the model was created with */
} mfa_model_info;

/* Fills *info.  MFA_ERR_ARG on NULL arguments. */
int mfa_model_get_info(const mfa_model* model, mfa_model_info* info);

/*
 * Checkpoint (the paper writes each block's model after encoding and reads it back for
 * rendering, Sec. IV-A.2).
 *   mfa_model_get_ctrl: copies the stored control points to host_out (HOST, caller-owned,
 *     n_x n_y n_z values [n_z][n_y][n_x] of the storage type: 4 bytes FP32, 2 bytes FP16 or
 *     BF16 bits); synchronises the bound stream.
 *   mfa_model_save: writes the model to a file (a 64-byte header with the magic "MFAMODL1",
 *     degrees, counts and storage type; the FP64 knots; the stored control points).
 *   mfa_model_load: creates a model from such a file on the current device; its stored
 *     values are bit-identical to the saved model's.  The header, sizes and file length are
 *     checked before any device work; NULL on error (reason in mfa_last_error()).
 * MFA_ERR_ARG for NULL arguments or a file that cannot be written; MFA_ERR_CUDA on a failed
 * CUDA call.
 */
int mfa_model_get_ctrl(const mfa_model* model, void* host_out);
int mfa_model_save(const mfa_model* model, const char* path);
mfa_model* mfa_model_load(const char* path);

/* Binds a CUDA stream (a cudaStream_t passed as void*) for later calls on the calling
 * thread; NULL selects the legacy default stream.  Always MFA_OK. */
int mfa_set_stream(void* cuda_stream);

/*
 * Value and gradient queries at n arbitrary points (Sec. III-B; the query of Fig. 8,
 * Sec. V-D.3).
 *   pts   DEVICE, n * 3 FP32, (x, y, z) per point; coordinates outside [0,1] are clamped
 *         to it and NaN is read as 0.
 *   val   DEVICE, n FP32: f at each point.
 *   grad  DEVICE, n * 3 FP32 (df/dx, df/dy, df/dz) per point, or NULL for values only.
 * n = 0 is a no-op.  MFA_ERR_ARG on NULL model/pts/val with n > 0 or n < 0.
 */
int mfa_decode(const mfa_model* model, const float* pts, long long n, float* val, float* grad);

/*
 * Knot spans of n points, computed by the same device code mfa_decode runs for this model
 * (the span search on general knots; on the uniform-knot path, floor((n - p) u) with its
 * exact check against the knots): spans[3i + d] = the largest s in [degree_d, nctrl_d - 1]
 * with U_d[s] <= u_d after clamping (a coordinate on an interior knot goes to the span on
 * its right; u = 1 goes to the last span).  The comparison is exact against the FP64
 * knots (Sec. III-A, Sec. III-B).
 *   pts    DEVICE, n * 3 FP32.   spans  DEVICE, n * 3 int32.
 */
int mfa_locate_spans(const mfa_model* model, const float* pts, long long n, int* spans);

typedef struct {
    int projection;                  /* 0 orthographic, 1 perspective */
    double eye[3], target[3], up[3]; /* right-handed look-at; up must not be parallel to
                                        target - eye */
    double fov_y_deg;                /* perspective: full vertical field of view, (0, 180) */
    double ortho_height;             /* orthographic: view height (> 0); width = height W/H */
} mfa_camera;

typedef struct {
    int n_entries;        /* rows of the table, 1..256 */
    const float* rgba;    /* HOST, n_entries * 4, non-premultiplied, row i at t = i/(n-1),
                             linear interpolation between rows, clamped at the ends */
    float vmin, vmax;     /* t = (f - vmin)/(vmax - vmin); NaN selects the model's min/max */
    int shading;          /* 0 none; 1 Phong with a headlight, two-sided */
    float ka, kd, ks, shininess;
    float ert_alpha;      /* early ray termination once accumulated alpha >= ert_alpha;
                             >= 1 disables it */
} mfa_transfer_fn;

typedef struct {
    unsigned long long* samples_out;  /* DEVICE counter or NULL: the number of samples
                                         evaluated (after box clipping and early
                                         termination) is ADDED to it */
    int variant;                      /* kernel variant: 0 = library default (8 for a
                                         cardinal model created with MFA_WINDOW_PATCH, 6
                                         for a cardinal model, see mfa_model_info, else
                                         4: the batch and serving kernels' choice too);
                                         1 = span records cached in registers along the
                                         ray, packed FP32x2 arithmetic; 2 = records cached,
                                         scalar FP32; 3 = nothing cached, scalar FP32;
                                         4 = as 2, software-pipelined over samples;
                                         5 = control-point bricks staged per warp in shared
                                         memory as FP32 (degree <= 3 on every axis; otherwise
                                         4); 6 = uniform knots: interior spans evaluate
                                         the one cardinal basis without span records
                                         (cardinal models only; otherwise 4); 7 = 6 (4 off
                                         the cardinal path) with empty-space skipping
                                         (mfa_render_ex and the server only): a
                                         sample whose knot-span cell's value bound maps
                                         only to transfer-function rows of zero opacity is
                                         neither queried nor composited -- the image
                                         equals 6's (4's) up to FP32 rounding order
                                         (which can move an early-termination decision
                                         by one sample: (1 - ert_alpha) x alpha at most),
                                         samples_out counts the evaluated samples; a pass over the cells builds
                                         the per-render visibility bits (one bit per cell,
                                         from the staging pool); 8 = per-cell polynomial
                                         patches (MFA_WINDOW_PATCH models; otherwise the
                                         default): 6 with each knot-span cell's
                                         coefficients in place of its window rows and
                                         monomials in place of the basis; off the
                                         cardinal path the spans come from the records'
                                         bounds (chosen explicitly or by the tuner, not
                                         by default).  Variants 1-6 and 8 differ only in
                                         FP32 rounding order.
                                         MFA_ERR_ARG outside 0..8. */
    int tile_shape;                   /* ray tile: 0 = 16x8 pixels per CTA with 8x4 per warp
                                         (default), 1 = 32x4 / 8x4, 2 = 8x16 / 4x8,
                                         3 = 16x8 / 16x2.  MFA_ERR_ARG outside 0..3. */
    int use_tuned;                    /* nonzero: take variant and tile_shape from the
                                         autotuner's choice for this workload class when
                                         there is one (mfa_tune_render) */
    int reserved[5];                  /* zero */
} mfa_render_opts;

/*
 * MFA-VV ray casting of one image (Sec. IV-A.4).  For the pixel in column c, row r
 * (row 0 at the top) the ray goes through the pixel centre, is clipped to the unit box,
 * and n_samples samples sit at the midpoints of n_samples equal pieces of the clipped
 * segment.  Each sample queries f and grad f, looks f up in the transfer function,
 * shades with grad f if asked, and is composited front to back with the over operation
 * (premultiplied; background transparent black) until ert_alpha is reached.
 *   rgba_out  DEVICE, height * width * 4 FP32, premultiplied RGBA, row-major from the top.
 * width, height in 1..32768; n_samples in 1..1048576.
 */
int mfa_render(const mfa_model* model, const mfa_camera* camera, const mfa_transfer_fn* tf,
               int width, int height, int n_samples, float* rgba_out);

/* mfa_render with options (opts may be NULL). */
int mfa_render_ex(const mfa_model* model, const mfa_camera* camera, const mfa_transfer_fn* tf,
                  int width, int height, int n_samples, float* rgba_out, const mfa_render_opts* opts);

/*
 * The render with the paper's object-space decomposition (Sec. IV-A.1 partitioning into
 * blocks, Sec. IV-A.4 MFA-VV of each block into a partial image, Sec. IV-A.5 compositing of
 * the partial images with the associative over), on one GPU.  The unit box is split into
 * blocks[0] x blocks[1] x blocks[2] equal blocks (1..64 in total).  Every ray keeps the
 * samples of mfa_render; block b renders those of them inside it -- front to back, early
 * termination on the segment's own alpha -- and the partial images are merged per pixel,
 * nearest segment first, into rgba_out (DEVICE, as mfa_render).  With ert_alpha >= 1 the
 * image equals mfa_render's up to FP32 rounding order; with termination each segment may
 * add what lies behind the single-pass stopping point, at most 1 - ert_alpha per channel.
 * opts as mfa_render_ex (may be NULL; variant 0, 4 or 6 only).  Partial images
 * (16 bytes x pixels x blocks) come from the library's staging pool; asynchronous on the
 * bound stream.  MFA_ERR_ARG on a bad block grid, otherwise errors as mfa_render_ex.
 */
int mfa_render_segments(const mfa_model* model, const mfa_camera* camera, const mfa_transfer_fn* tf, int width,
                        int height, int n_samples, const int blocks[3], float* rgba_out,
                        const mfa_render_opts* opts);

/*
 * Isosurface rendering through MFA queries (Sec. IV-A.4 names isosurfaces as the other
 * visualization the query interface serves).  Per pixel, the ray's samples (those of
 * mfa_render) are queried in order until f - iso_value changes sign between two of them;
 * the crossing is refined by 8 Newton steps on g(t) = f(o + t d) - iso_value with the
 * analytic derivative grad f . d, kept inside the bracket (the bracket shrinks to the side
 * where g changes sign; a Newton point outside it is replaced by its midpoint).  The hit is
 * shaded like a volume sample of value iso_value (transfer-function colour, Phong with
 * grad f when tf->shading) and is opaque: rgba_out (DEVICE, as mfa_render) holds
 * (r, g, b, 1), or 0 where the ray has no crossing; depth_out (DEVICE [height][width]
 * FP32, may be NULL) the hit's ray parameter t (distance from the eye for perspective
 * views), +inf on a miss.  A sample whose knot-span cell has every control point of its
 * support on one side of iso_value takes that side's sign without a query (the model lies
 * in their convex hull; the per-cell bounds are built with the model).  opts may be NULL
 * (its tile_shape and samples_out -- samples examined plus refinement queries -- apply).
 * MFA_ERR_ARG for a non-finite iso_value, otherwise errors as mfa_render_ex.
 */
int mfa_render_iso(const mfa_model* model, const mfa_camera* camera, const mfa_transfer_fn* tf, int width,
                   int height, int n_samples, float iso_value, float* rgba_out, float* depth_out,
                   const mfa_render_opts* opts);

/*
 * Ground truth of the render-quality comparison (Sec. V-D.3): the closed-form
 * Marschner-Lobb signal (Sec. V-A.1, Eq. 1)
 *     F(x, y, z) = (1 - sin(pi z / 2) + alpha (1 + rho(r))) / (2 (1 + alpha)),
 *     rho(r) = cos(2 pi f_M cos(pi r / 2)),  r = sqrt(x^2 + y^2),
 * on [-1, 1]^3, which the unit box maps onto by x = 2u - 1 (likewise y, z), rendered with
 * the rays, samples, transfer function, Phong shading (with the analytic gradient with
 * respect to (u, v, w)), over and early termination of mfa_render.  A NaN tf->vmin / vmax
 * means F's range [0, 1]; the normal is undefined where |grad F| <= 1e-6.  Values in FP32.
 * The paper uses f_M = 6, alpha = 0.25.  rgba_out (DEVICE) and opts as mfa_render_iso.
 * MFA_ERR_ARG for a NULL signal, f_m or alpha negative or not finite, otherwise errors as
 * mfa_render_ex.  Asynchronous on the bound stream.
 */
typedef struct {
    double f_m;     /* radial frequency f_M */
    double alpha;   /* weight of the radial term */
} mfa_ml_signal;
int mfa_render_ml(const mfa_ml_signal* signal, const mfa_camera* camera, const mfa_transfer_fn* tf, int width,
                  int height, int n_samples, float* rgba_out, const mfa_render_opts* opts);

/*
 * Image metrics of the render-quality comparison (Table II: MSE, PSNR, SSIM) between two
 * premultiplied RGBA FP32 images of width x height pixels (DEVICE, [height][width][4],
 * 16-byte aligned).  R, G, B are clamped to [0, 1] and scaled by 255 (alpha is ignored);
 *   mse      mean over pixels and the three channels of the squared difference;
 *   psnr_db  10 log10(255^2 / mse), +inf for equal images;
 *   ssim     the structural similarity of Wang et al. (IEEE TIP 2004) with an 11 x 11
 *            Gaussian window (sigma 1.5, weights summing to 1), C1 = (0.01 * 255)^2,
 *            C2 = (0.03 * 255)^2, averaged over the window positions lying inside the
 *            image and over the three channels (symmetric in the two images).
 * Sums in FP64 in a fixed order (the result does not depend on timing).  A few KB of
 * scratch from the library's staging pool; synchronises the bound stream.  MFA_ERR_ARG
 * for NULL or misaligned pointers or a side outside 11..32768; MFA_ERR_CUDA on a failed
 * CUDA call.
 */
typedef struct {
    double mse;
    double psnr_db;
    double ssim;
} mfa_image_quality;
int mfa_image_compare(const float* rgba_test, const float* rgba_ref, int width, int height, mfa_image_quality* out);

/*
 * Host-buffer forms of mfa_decode and mfa_render_ex: the same queries (Sec. III-B, the
 * query of Fig. 8 in Sec. V-D.3) and the same ray casting (Sec. IV-A.4), for data in HOST
 * memory.
 *   mfa_decode_host: pts HOST n * 3 FP32, val HOST n FP32, grad HOST n * 3 FP32 or NULL;
 *   mfa_render_host: rgba_out HOST [height][width][4] FP32; opts as mfa_render_ex (may be
 *   NULL; its samples_out, if set, is still a DEVICE counter).
 * The library stages the data through device memory of its own (a per-device pool kept
 * cached between calls) and, for decode, pipelines copy-in, kernel and copy-out over
 * chunks of 2^21 points on helper streams of the calling thread.  Both calls are
 * asynchronous on the bound stream, like cudaMemcpyAsync: they return once the work is
 * enqueued, and the host buffers must stay valid -- inputs unchanged, outputs unread --
 * until that stream has been synchronised.  Page-locked host buffers let the copies run
 * beside the kernels; pageable ones work, with serialised copies.  Argument errors are
 * reported as by mfa_decode / mfa_render_ex before any work is enqueued; n = 0 is a no-op.
 * The caller keeps ownership of every buffer.
 */
int mfa_decode_host(const mfa_model* model, const float* pts, long long n, float* val, float* grad);
int mfa_render_host(const mfa_model* model, const mfa_camera* camera, const mfa_transfer_fn* tf,
                    int width, int height, int n_samples, float* rgba_out, const mfa_render_opts* opts);

/*
 * Batched rendering: many images of many models in one persistent launch (the paper
 * renders one partition per core, Sec. IV-A.4; on one GPU the unit of parallel work is a
 * ray tile).  A request is one mfa_render call's worth of arguments.
 */
typedef struct {
    const mfa_model* model;
    mfa_camera camera;
    const mfa_transfer_fn* tf;        /* its table is copied when the batch is submitted */
    int width, height, n_samples;     /* as mfa_render */
    float* rgba_out;                  /* DEVICE, height * width * 4 FP32 */
    unsigned long long* samples_out;  /* DEVICE counter or NULL (samples evaluated are added) */
} mfa_render_request;

typedef struct mfa_batch mfa_batch;   /* reusable batch context; owns its work tables */
typedef struct mfa_server mfa_server; /* render server; owns its output arena */

/*
 * Creates a batch context on the current device for up to max_requests (1..4096)
 * requests per submission.  It owns two pinned host work tables and two device work
 * tables (used alternately, so one submission can be in flight while the next is
 * written) and the CUDA graphs it records: each submission is ONE graph launch made of
 * the table upload and one persistent kernel per control-point storage type present.
 * Inside the kernel, CTAs (SMs x resident CTAs) draw ray tiles of all requests from one
 * device counter.  NULL on error.
 */
mfa_batch* mfa_batch_create(int max_requests);

/* Ray-tile shape (as mfa_render_opts.tile_shape) and CTA count (0 = SMs x occupancy)
 * for later submissions; chosen by the autotuner.  MFA_ERR_ARG on bad values. */
int mfa_batch_configure(mfa_batch* batch, int tile_shape, int grid_ctas);

/*
 * Validates the n requests (every check of mfa_render; MFA_ERR_ARG names the first bad
 * request and nothing is launched), writes the work table and launches the batch graph
 * on the stream bound to the calling thread.  Asynchronous; the outputs are complete
 * when that stream reaches this point.  Blocks only if the work table it is about to
 * overwrite still belongs to a submission the GPU has not started (two in flight at
 * most).  All models must live on the batch's device.  n = 0 is a no-op.
 */
int mfa_batch_render(mfa_batch* batch, const mfa_render_request* reqs, int n);

/* Frees the context after the GPU has finished its submissions.  NULL is a no-op. */
void mfa_batch_destroy(mfa_batch* batch);

/* One-shot form: a thread-local batch context sized on demand, then mfa_batch_render. */
int mfa_render_batch(const mfa_render_request* reqs, int n);

/*
 * Autotuner (no counterpart in the paper: it picks this implementation's launch shape).
 * A workload class is (degree class p_max + 1, storage type, image pixels in powers of 4,
 * samples per ray in powers of 2, uniform or other knots, largest control-point count per
 * axis in powers of 2).
 */
typedef struct {
    int variant;      /* as mfa_render_opts.variant */
    int tile_shape;   /* as mfa_render_opts.tile_shape */
    float ms;         /* measured time per launch */
} mfa_tune_result;

/* Times every variant x tile-shape candidate on this render (one warm-up plus `reps`
 * launches each, CUDA events on the bound stream; synchronises it), stores the fastest as
 * the choice for the workload's class and returns it in *best; `all` (may be NULL)
 * receives up to max_all measured candidates, *n_all their count.  Candidates: variants
 * 1-5 and 7, plus 6 for cardinal models and 8 for MFA_WINDOW_PATCH models.  The class does not include the transfer
 * function, so a stored variant 7 (chosen where this render's table is partly
 * transparent) also serves later renders with other tables: same images, at most its
 * visibility pass slower where nothing is transparent; batches run it as 6.  rgba_out is overwritten.  Any render argument error is returned as by mfa_render. */
int mfa_tune_render(const mfa_model* model, const mfa_camera* camera, const mfa_transfer_fn* tf, int width,
                    int height, int n_samples, float* rgba_out, int reps, mfa_tune_result* best,
                    mfa_tune_result* all, int max_all, int* n_all);
/* Times each tile shape for this batch submission and configures the batch with the
 * fastest (*best).  Synchronises the bound stream. */
int mfa_tune_batch(mfa_batch* batch, const mfa_render_request* reqs, int n, int reps, mfa_tune_result* best);
/* The stored choice for a workload's class; MFA_ERR_ARG if there is none. */
int mfa_tune_lookup(const mfa_model* model, int width, int height, int n_samples, mfa_tune_result* out);
/* Writes / reads the stored choices (one text line per class).  With the environment
 * variable MFA_TUNE_CACHE naming a file, the choices in it are read on the first use of the
 * stored choices (a missing file reads as none), and every mfa_tune_render rewrites it. */
int mfa_tune_save(const char* path);
int mfa_tune_load(const char* path);

/*
 * Serving (the paper's input-latency concern, Sec. IV-B and Sec. V-C, on one GPU): a server
 * keeps client-created models resident, takes camera-view requests of any image size, and
 * admits them in arrival order while a slot is free and the output image fits in its HBM
 * arena (hbm_budget_bytes, allocated once at creation).  Admitted requests run in one of
 * two modes:
 *   mode 0 (device work queue): each request is published as a record in device memory and
 *     placed in an active list ordered by urgency (arrival time, plus the request's work at
 *     urgency_rate when that is set); persistent kernels, one per model degree class, storage
 *     type and knot path, draw ray tiles from the list, so a request joins the running
 *     batch at the next tile any CTA claims; completion is flagged by the kernel in
 *     host-mapped memory and polled by the server thread.  Requests of a kernel group other
 *     than the one holding the SMs get SMs as that group's CTAs run out of tiles.
 *   mode 1 (stream per request): each request is launched at once on a stream whose
 *     priority rises as its work (pixels x samples) falls, and small views overtake large
 *     ones on the SMs that free up; completions are stamped by host callbacks.
 * A server thread does the admitting.  No call waits without a bound.
 */
typedef struct {
    size_t hbm_budget_bytes;   /* arena for output images (>= 4096) */
    int max_slots;             /* requests on the GPU at once, 1..4096 (mode 0: 1..256) */
    int max_queue;             /* waiting requests before submit answers MFA_ERR_BUSY, >= 1 */
    int priority_levels;       /* mode 1: streams of distinct priority, 1..8 (1 = one FIFO stream) */
    int variant, tile_shape;   /* render kernel choice (as mfa_render_opts; mode 0 uses the
                                  tile shape and the default kernel of each model) */
    int use_tuned;             /* mode 1, nonzero: the autotuner's choice per request class */
    int mode;                  /* 0 device work queue, 1 stream per request */
    double urgency_rate;       /* mode 0: requests are served in order of arrival time plus
                                  their work (pixels x samples) / urgency_rate seconds, so
                                  small views overtake larger ones that arrived at most their
                                  work's worth earlier; 0 = arrival order */
} mfa_server_config;

typedef struct {
    const mfa_model* model;           /* resident; must outlive the request */
    mfa_camera camera;
    const mfa_transfer_fn* tf;        /* copied at submit */
    int width, height, n_samples;
    double arrival_time_s;            /* mfa_server_now() clock; <= 0 means the submit time */
} mfa_serve_request;

typedef struct {
    long long submitted, completed, failed, rejected_busy, cancelled;
    long long peak_in_flight, peak_arena_bytes;
    long long in_flight, queued, arena_bytes_in_use;
} mfa_server_stats;

enum { MFA_TICKET_QUEUED = 0, MFA_TICKET_RUNNING = 1, MFA_TICKET_DONE = 2, MFA_TICKET_FAILED = 3 };

/* Seconds on the monotonic clock the server stamps latencies with. */
double mfa_server_now(void);
/* Creates a server on the current device (allocates the arena, the streams and the
 * server thread).  NULL on error. */
mfa_server* mfa_server_create(const mfa_server_config* cfg);
/* Queues a request; *ticket identifies it.  MFA_ERR_NOMEM if its image (width*height*16
 * bytes) can never fit the budget, MFA_ERR_BUSY if max_queue requests are waiting,
 * MFA_ERR_ARG on bad arguments; nothing is queued on error. */
int mfa_server_submit(mfa_server* server, const mfa_serve_request* req, long long* ticket);
/* State of a ticket (MFA_TICKET_*) and, once done, its latency from arrival to
 * completion in ms (-1 before). */
int mfa_server_poll(mfa_server* server, long long ticket, int* state, double* latency_ms);
/* Waits up to timeout_ms for the ticket; MFA_ERR_TIMEOUT if it is still queued or
 * running then.  *latency_ms as in mfa_server_poll. */
int mfa_server_wait(mfa_server* server, long long ticket, double timeout_ms, double* latency_ms);
/* DEVICE pointer to a done ticket's premultiplied RGBA image (height * width * 4 FP32),
 * valid until mfa_server_release.  MFA_ERR_BUSY if the ticket is not done. */
int mfa_server_result(mfa_server* server, long long ticket, const float** rgba);
/* Copies a done ticket's image (width*height*16 bytes) to dst (device or host memory,
 * dst_bytes large enough) asynchronously on the calling thread's bound stream. */
int mfa_server_copy_result(mfa_server* server, long long ticket, void* dst, size_t dst_bytes);
/* Returns a done ticket's image memory to the arena (or cancels a queued ticket).
 * MFA_ERR_BUSY while the ticket is on the GPU. */
int mfa_server_release(mfa_server* server, long long ticket);
int mfa_server_get_stats(mfa_server* server, mfa_server_stats* stats);
/* Stops the server thread, waits for requests on the GPU, frees everything. */
void mfa_server_destroy(mfa_server* server);

/*
 * Allocation-free batched render (the paper has no counterpart; this is a deployment
 * variant of mfa_render_batch).  For callers that cannot call cudaMalloc -- for example a
 * process whose memory pool already holds the whole device, or a render loop that must
 * not take the allocator's implicit synchronisation -- this call renders up to 32
 * requests with the same persistent kernels as mfa_batch_render but keeps the work table
 * in a fixed 176 KiB array inside the library's device image instead of allocating one.
 * Every GPU that loads the library holds that array until the process exits.
 *   reqs, n  as mfa_batch_render; n in 0..32, MFA_ERR_ARG beyond (nothing launched).
 * Asynchronous on the bound stream; it makes no allocation (no cudaMalloc, cudaFree or
 * cudaMallocHost).  The work table is filled by host-to-device copies from this call's
 * own memory, so the call cannot be recorded into a CUDA graph: on a stream that is being
 * captured it returns MFA_ERR_UNSUPPORTED and enqueues nothing (the capture stays valid).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; with lazy module loading that first call also loads the
 * library's device code, which places the array and the kernels in device memory, so make
 * it before the caller's own pool reserves the rest of the device.  All calls share the
 * one array, which keeps the previous call's contents (each call rewrites everything the
 * kernels read, tile counters included): calls whose work overlaps on the GPU -- on
 * different streams, or from different threads -- race and must be serialised by the
 * caller.
 */
int mfa_render_batch_static(const mfa_render_request* reqs, int n);

/*
 * MFA encoding (Sec. III-A, Sec. IV-A.2: the model a block is rendered from is fitted to the
 * block's regular grid of values before visualization).  data: DEVICE FP32
 * [ndata[2]][ndata[1]][ndata[0]], x fastest, the values at the uniform parameters
 * u_i = i / (ndata[0] - 1) (likewise v, w).  The fit minimises the sum of squared errors
 * at the data points over the control points (least squares along each axis -- z, y, x; FP64,
 * normal equations with a banded Cholesky factor per axis).  Errors: MFA_ERR_ARG when a
 * knot span holds too few data parameters to determine the spline, ndata[d] < nctrl[d],
 * bad knots (as mfa_model_create); MFA_ERR_UNSUPPORTED for a degree outside 1..4.  All
 * three synchronise the bound stream.
 *   mfa_fit_ctrl:      the fitted control points, DEVICE FP64 [nctrl[2]][nctrl[1]][nctrl[0]].
 *   mfa_model_fit:     a model of the fit with the given storage type; *max_err (may be
 *                      NULL) receives the largest |f - data| over the data points, with f
 *                      evaluated by the model (FP32 arithmetic).
 *   mfa_model_encode:  adaptive encoding: from degree + 1 control points per axis, fit and,
 *                      while the largest error exceeds cfg->err_max, insert a knot at the
 *                      middle of every knot span whose data exceed it (the error projected
 *                      onto each axis by its maximum over the other two), refit; stop when
 *                      the error is within err_max, when no axis can take another knot (a
 *                      span with fewer than two data parameters, or cfg->max_ctrl reached --
 *                      0 means ndata -- leftmost spans first), or after cfg->max_iter fits.
 *                      *result (may be NULL) receives the fits made, the final error and
 *                      control-point counts.
 */
typedef struct {
    double err_max;      /* target largest |f - data| */
    int max_ctrl[3];     /* control-point limit per axis (0: ndata) */
    int max_iter;        /* fits at most, 1..1000 */
} mfa_encode_config;
typedef struct {
    int iterations;      /* fits made */
    double max_err;      /* largest error of the returned model */
    int nctrl[3];        /* its control points per axis */
} mfa_encode_result;
int mfa_fit_ctrl(const int degree[3], const int nctrl[3], const double* const knots[3], const int ndata[3],
                 const float* data, double* ctrl_out);
mfa_model* mfa_model_fit(const int degree[3], const int nctrl[3], const double* const knots[3], const int ndata[3],
                         const float* data, mfa_dtype storage, double* max_err);
mfa_model* mfa_model_encode(const int degree[3], const int ndata[3], const float* data, mfa_dtype storage,
                            const mfa_encode_config* cfg, mfa_encode_result* result);

/*
 * Calibration for the roofline denominators (no counterpart in the paper: measurement
 * infrastructure).  Runs, on the current device and the bound stream, a chip-wide FP32
 * FMA kernel (scalar and packed FP32x2 forms) and a kernel of random 32-byte gathers from
 * a 32 MiB buffer held in L2, each timed with CUDA events after a warm-up launch, and
 * synchronises the stream.  Allocates and frees about 45 MB of device memory.
 * MFA_ERR_ARG on NULL; MFA_ERR_CUDA / MFA_ERR_NOMEM on a failed CUDA call.
 */
typedef struct {
    double fp32_tflops;     /* scalar FFMA rate, 2 flops per FMA */
    double fp32x2_tflops;   /* packed fma.rn.f32x2 rate, 4 flops per instruction */
    double l2_gather_gbs;   /* bytes of random 32-byte entries served per second */
    double fma_clock_mhz;   /* fp32_tflops / (SMs x 128 lanes x 2 flops) */
    int sm_count;
} mfa_peaks;
int mfa_measure_peaks(mfa_peaks* out);

/*
 * Debug builds (libmfa_debug.so, compiled with -DMFA_DEBUG; paper_2312_15073_gb300.build
 * builds it with debug=True) check every control-point window, span-record, cell and
 * transfer-function index on the device before the load.  A bad index is replaced by 0
 * (nothing traps) and recorded in a per-device word: mfa_debug_status waits for the device,
 * returns the flags (1 window, 2 span record, 4 cell bound, 8 transfer function) and the
 * number of bad indices since the last call, and clears them.  Release builds report 0.
 * mfa_debug_build returns 1 in a debug build, else 0.
 */
int mfa_debug_build(void);
int mfa_debug_status(unsigned int* flags, unsigned int* count);

/* Text of the last error on the calling thread ("" if none). */
const char* mfa_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MFA_H */
