/*
 * oracle.c -- plain FP64 CPU oracle for MFA value/gradient queries and MFA ray casting.
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the benchmark's CPU
 * baseline are the only code that may load this library.  It shares no source, header,
 * table or helper with the GPU library; everything here is written out from the
 * definitions it cites, in FP64, one query or one ray at a time, with no blocking,
 * fusion or reordering beyond the definitions themselves.  Threads only split the
 * independent pixels or points among cores.
 *
 * What it computes
 *  - The MFA model (Sec. III-A): a tensor-product B-spline volume given by degrees
 *    p_x, p_y, p_z, clamped knot vectors U_x, U_y, U_z and control points P_ijk
 *    (x fastest in memory).  The paper defines MFA only by citation, so the B-spline
 *    basis is the textbook one: the Cox-de Boor recursion (de Boor, cited in Sec. I),
 *        N_{i,0}(u) = 1 if U_i <= u < U_{i+1}, else 0,
 *        N_{i,k}(u) = (u-U_i)/(U_{i+k}-U_i) N_{i,k-1}(u)
 *                   + (U_{i+k+1}-u)/(U_{i+k+1}-U_{i+1}) N_{i+1,k-1}(u),
 *    with 0/0 := 0, and its analytic first derivative
 *        N'_{i,k}(u) = k/(U_{i+k}-U_i) N_{i,k-1}(u) - k/(U_{i+k+1}-U_{i+1}) N_{i+1,k-1}(u).
 *  - The value query  f(u,v,w) = sum_ijk N_{i,px}(u) N_{j,py}(v) N_{k,pz}(w) P_ijk  and the
 *    gradient, the same sum with one factor replaced by its derivative (Sec. III-B,
 *    "analytical high-order derivatives"; Sec. V-D.3 on the cost of the value and
 *    gradient queries).  Only the p+1 functions that can be non-zero on the knot span of
 *    u enter the sum; the rest are zero by the recursion.  The parameter domain
 *    [0,1]^3 is the world box, so the world gradient equals the parameter gradient.
 *  - MFA-VV ray casting (Sec. IV-A.4): one ray per pixel, samples along the ray, one
 *    value+gradient query per sample, a 1-D transfer function and gradient shading set
 *    by the user (Sec. IV-B), and the over operation between neighbouring samples,
 *    front to back (Sec. IV-A.4, IV-A.5).
 *  - The same ray casting of the closed-form Marschner-Lobb signal (Sec. V-A.1, Eq. 1),
 *    the ground truth of the render-quality comparison (Sec. V-D.3).
 *
 * Readings of what the paper leaves open (also listed in the design notes):
 *  - knots are clamped and span [0,1]; a coordinate on an interior knot belongs to the
 *    span on its right; u = 1 belongs to the last span; queries are clamped to [0,1]
 *    first, and a NaN coordinate is treated as 0;
 *  - ray (col,row) goes through the pixel centre, row 0 at the top; rays start at the
 *    eye (t >= 0) and are clipped to the unit box by the slab method; n_s samples sit at
 *    the midpoints of n_s equal pieces of [t0,t1];
 *  - transfer function: n_entries RGBA rows at t = i/(n-1), linear interpolation,
 *    t = (f - vmin)/(vmax - vmin) clamped to [0,1]; per-sample alpha is the table's
 *    alpha (no opacity correction);
 *  - Phong with a headlight (L = V = -d), two-sided, colour = c (ka + kd |n.L|) +
 *    ks max(0, R.V)^s clamped to [0,1]; where |grad f| <= 1e-6 G, with
 *    G = max(max P - min P, max |P|) * max_d (n_d - p_d) (a bound on the gradient's
 *    scale), the normal is undefined and the factor is ka + kd with no specular;
 *  - front-to-back premultiplied over, C += (1-A) a c, A += (1-A) a, stop once
 *    A >= ert_alpha (ert_alpha >= 1 never stops); output premultiplied RGBA.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXP 8

typedef struct {
    int p[3];            /* degree per axis (x, y, z) */
    int n[3];            /* control points per axis */
    const double* U[3];  /* knot vectors, length n+p+1 each */
    const double* P;     /* control points [n_z][n_y][n_x], x fastest */
} orc_model;

typedef struct {
    int projection;      /* 0 orthographic, 1 perspective */
    double eye[3], target[3], up[3];
    double fov_y_deg;    /* perspective: full vertical field of view */
    double ortho_height; /* orthographic: view height; width = height * W / H */
} orc_camera;

typedef struct {
    int n_entries;       /* rows of the RGBA table */
    const float* rgba;   /* n_entries * 4, non-premultiplied */
    double vmin, vmax;   /* NaN => min / max of the control points */
    int shading;         /* 0 off, 1 Phong */
    double ka, kd, ks, shininess;
    double ert_alpha;    /* stop when accumulated alpha >= this; >= 1 never stops */
} orc_tf;

/* ------------------------------------------------------------------------------------ */
/* B-spline basis                                                                        */
/* ------------------------------------------------------------------------------------ */

/* num/den with 0/0 (and x/0) read as 0: a zero-length knot interval drops the term. */
static double ratio(double num, double den) { return den != 0.0 ? num / den : 0.0; }

/* Knot span of u: the largest s in [p, n-1] with U[s] <= u (so U[s] <= u < U[s+1] for
 * u inside the domain; u at an interior knot goes right; u = U[n] gives n-1).  A plain
 * binary search over the clamped knot vector. */
int orc_find_span(int n, int p, const double* U, double u)
{
    if (u >= U[n]) return n - 1;
    if (u < U[p]) return p;
    int lo = p, hi = n - 1;          /* invariant: U[lo] <= u, answer in [lo, hi] */
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (U[mid] <= u) lo = mid; else hi = mid - 1;
    }
    return lo;
}

/* The p+1 functions N_{s-p..s, p}(u) that can be non-zero on span s, and their first
 * derivatives, from the Cox-de Boor recursion run level by level:
 * T[k][r] holds N_{s-k+r, k}(u), r = 0..k; T[0][0] = N_{s,0}(u) = 1 because u lies in
 * span s.  Functions of level k-1 outside the triangle are zero on span s. */
void orc_basis(int s, double u, int p, const double* U, double* N, double* dN)
{
    double T[ORC_MAXP + 1][ORC_MAXP + 1];
    T[0][0] = 1.0;
    for (int k = 1; k <= p; ++k) {
        for (int r = 0; r <= k; ++r) {
            int i = s - k + r;
            double lower = (r >= 1) ? T[k - 1][r - 1] : 0.0;   /* N_{i,   k-1} */
            double upper = (r <= k - 1) ? T[k - 1][r] : 0.0;   /* N_{i+1, k-1} */
            T[k][r] = ratio(u - U[i], U[i + k] - U[i]) * lower
                    + ratio(U[i + k + 1] - u, U[i + k + 1] - U[i + 1]) * upper;
        }
    }
    for (int r = 0; r <= p; ++r) N[r] = T[p][r];
    if (!dN) return;
    for (int r = 0; r <= p; ++r) {
        if (p == 0) { dN[r] = 0.0; continue; }
        int i = s - p + r;
        double lower = (r >= 1) ? T[p - 1][r - 1] : 0.0;
        double upper = (r <= p - 1) ? T[p - 1][r] : 0.0;
        dN[r] = ratio((double)p, U[i + p] - U[i]) * lower
              - ratio((double)p, U[i + p + 1] - U[i + 1]) * upper;
    }
}

/* N_{i,k}(u) by the textbook recursion over the whole knot vector (exponential cost;
 * tiny models only).  The half-open degree-0 intervals are closed at the right end of
 * the domain, so that u = U_last belongs to the last non-empty interval, matching the
 * span rule above. */
double orc_basis_direct(int i, int k, double u, const double* U, int nknots)
{
    if (k == 0) {
        if (U[i] <= u && u < U[i + 1]) return 1.0;
        if (u == U[nknots - 1]) {
            int last = nknots - 2;
            while (last > 0 && !(U[last] < U[last + 1])) --last;
            return i == last ? 1.0 : 0.0;
        }
        return 0.0;
    }
    return ratio(u - U[i], U[i + k] - U[i]) * orc_basis_direct(i, k - 1, u, U, nknots)
         + ratio(U[i + k + 1] - u, U[i + k + 1] - U[i + 1]) * orc_basis_direct(i + 1, k - 1, u, U, nknots);
}

double orc_basis_direct_deriv(int i, int k, double u, const double* U, int nknots)
{
    if (k == 0) return 0.0;
    return ratio((double)k, U[i + k] - U[i]) * orc_basis_direct(i, k - 1, u, U, nknots)
         - ratio((double)k, U[i + k + 1] - U[i + 1]) * orc_basis_direct(i + 1, k - 1, u, U, nknots);
}

/* ------------------------------------------------------------------------------------ */
/* value + gradient query                                                                */
/* ------------------------------------------------------------------------------------ */

static double clamp_domain(double u, double lo, double hi)
{
    if (!(u >= lo)) return lo;       /* also catches NaN */
    if (u > hi) return hi;
    return u;
}

/* out = {f, df/dx, df/dy, df/dz}; spans (optional) = the knot span per axis. */
void orc_eval(const orc_model* m, const double uvw[3], double out[4], int spans[3])
{
    double N[3][ORC_MAXP + 1], D[3][ORC_MAXP + 1];
    int s[3];
    for (int a = 0; a < 3; ++a) {
        const double* U = m->U[a];
        double u = clamp_domain(uvw[a], U[m->p[a]], U[m->n[a]]);
        s[a] = orc_find_span(m->n[a], m->p[a], U, u);
        orc_basis(s[a], u, m->p[a], U, N[a], D[a]);
        if (spans) spans[a] = s[a];
    }
    const int nx = m->n[0], ny = m->n[1];
    double f = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int c = 0; c <= m->p[2]; ++c) {
        for (int b = 0; b <= m->p[1]; ++b) {
            for (int a = 0; a <= m->p[0]; ++a) {
                long long i = s[0] - m->p[0] + a;
                long long j = s[1] - m->p[1] + b;
                long long k = s[2] - m->p[2] + c;
                double P = m->P[(k * ny + j) * nx + i];
                f  += N[0][a] * N[1][b] * N[2][c] * P;
                gx += D[0][a] * N[1][b] * N[2][c] * P;
                gy += N[0][a] * D[1][b] * N[2][c] * P;
                gz += N[0][a] * N[1][b] * D[2][c] * P;
            }
        }
    }
    /* world box = parameter domain [0,1]^3: the chain-rule factor 1/extent is 1 */
    out[0] = f; out[1] = gx; out[2] = gy; out[3] = gz;
}

/* The same query summed over ALL n_x n_y n_z control points with the full recursion
 * (no span logic at all).  Tiny models only. */
void orc_eval_direct(const orc_model* m, const double uvw[3], double out[4])
{
    const int nx = m->n[0], ny = m->n[1], nz = m->n[2];
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = clamp_domain(uvw[a], m->U[a][m->p[a]], m->U[a][m->n[a]]);
    double f = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int k = 0; k < nz; ++k) {
        int nk = nz + m->p[2] + 1;
        double Nk = orc_basis_direct(k, m->p[2], u[2], m->U[2], nk);
        double Dk = orc_basis_direct_deriv(k, m->p[2], u[2], m->U[2], nk);
        for (int j = 0; j < ny; ++j) {
            int nj = ny + m->p[1] + 1;
            double Nj = orc_basis_direct(j, m->p[1], u[1], m->U[1], nj);
            double Dj = orc_basis_direct_deriv(j, m->p[1], u[1], m->U[1], nj);
            for (int i = 0; i < nx; ++i) {
                int ni = nx + m->p[0] + 1;
                double Ni = orc_basis_direct(i, m->p[0], u[0], m->U[0], ni);
                double Di = orc_basis_direct_deriv(i, m->p[0], u[0], m->U[0], ni);
                double P = m->P[((long long)k * ny + j) * nx + i];
                f  += Ni * Nj * Nk * P;
                gx += Di * Nj * Nk * P;
                gy += Ni * Dj * Nk * P;
                gz += Ni * Nj * Dk * P;
            }
        }
    }
    out[0] = f; out[1] = gx; out[2] = gy; out[3] = gz;
}

/* ------------------------------------------------------------------------------------ */
/* threads                                                                               */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    long long total, chunk;
    long long next;          /* shared work counter */
    void (*body)(void* ctx, long long begin, long long end, long long* counter);
    void* ctx;
} orc_pool;

typedef struct { orc_pool* pool; long long counter; } orc_worker;

static void* orc_worker_main(void* arg)
{
    orc_worker* w = (orc_worker*)arg;
    orc_pool* pool = w->pool;
    for (;;) {
        long long b = __atomic_fetch_add(&pool->next, pool->chunk, __ATOMIC_RELAXED);
        if (b >= pool->total) break;
        long long e = b + pool->chunk < pool->total ? b + pool->chunk : pool->total;
        pool->body(pool->ctx, b, e, &w->counter);
    }
    return NULL;
}

/* Runs body over [0,total) in chunks on nthreads threads; returns the summed counters. */
static long long orc_parallel(long long total, long long chunk, int nthreads,
                              void (*body)(void*, long long, long long, long long*), void* ctx)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 1024) nthreads = 1024;
    orc_pool pool = { total, chunk, 0, body, ctx };
    orc_worker* ws = (orc_worker*)calloc((size_t)nthreads, sizeof(orc_worker));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    int started = 0;
    for (int t = 0; t < nthreads; ++t) {
        ws[t].pool = &pool;
        if (t == 0) continue;                 /* the calling thread is worker 0 */
        if (pthread_create(&th[t], NULL, orc_worker_main, &ws[t]) != 0) break;
        started = t;
    }
    orc_worker_main(&ws[0]);
    long long sum = ws[0].counter;
    for (int t = 1; t <= started; ++t) { pthread_join(th[t], NULL); sum += ws[t].counter; }
    free(ws); free(th);
    return sum;
}

/* ------------------------------------------------------------------------------------ */
/* decode: value + gradient at arbitrary points                                         */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    const orc_model* m;
    const float* pts;   /* n * 3, FP32 inputs; evaluated at their exact FP64 values */
    double* val;        /* n */
    double* grad;       /* n * 3 or NULL */
    int* spans;         /* n * 3 or NULL */
} orc_decode_ctx;

static void orc_decode_body(void* vctx, long long b, long long e, long long* counter)
{
    orc_decode_ctx* c = (orc_decode_ctx*)vctx;
    for (long long i = b; i < e; ++i) {
        double uvw[3] = { (double)c->pts[3 * i], (double)c->pts[3 * i + 1], (double)c->pts[3 * i + 2] };
        double out[4];
        orc_eval(c->m, uvw, out, c->spans ? &c->spans[3 * i] : NULL);
        c->val[i] = out[0];
        if (c->grad) { c->grad[3 * i] = out[1]; c->grad[3 * i + 1] = out[2]; c->grad[3 * i + 2] = out[3]; }
    }
    *counter += e - b;
}

int orc_decode(const orc_model* m, const float* pts, long long n, double* val, double* grad,
               int* spans, int nthreads)
{
    orc_decode_ctx ctx = { m, pts, val, grad, spans };
    orc_parallel(n, 256, nthreads, orc_decode_body, &ctx);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* ray casting                                                                           */
/* ------------------------------------------------------------------------------------ */

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static void normalize3(double a[3]) { double l = sqrt(dot3(a, a)); a[0] /= l; a[1] /= l; a[2] /= l; }

/* Ray through the centre of pixel (col, row); row 0 is the top row.  Right-handed
 * look-at frame: forward = target - eye, right = forward x up, true up = right x forward. */
void orc_ray(const orc_camera* cam, int W, int H, int col, int row, double o[3], double d[3])
{
    double fwd[3] = { cam->target[0] - cam->eye[0], cam->target[1] - cam->eye[1], cam->target[2] - cam->eye[2] };
    normalize3(fwd);
    double right[3], upv[3];
    cross3(fwd, cam->up, right);
    normalize3(right);
    cross3(right, fwd, upv);
    double sx = 2.0 * (col + 0.5) / W - 1.0;
    double sy = 1.0 - 2.0 * (row + 0.5) / H;
    double aspect = (double)W / (double)H;
    if (cam->projection == 0) {
        double hh = 0.5 * cam->ortho_height, hw = hh * aspect;
        for (int a = 0; a < 3; ++a) {
            o[a] = cam->eye[a] + sx * hw * right[a] + sy * hh * upv[a];
            d[a] = fwd[a];
        }
    } else {
        double th = tan(0.5 * cam->fov_y_deg * M_PI / 180.0);
        for (int a = 0; a < 3; ++a) {
            o[a] = cam->eye[a];
            d[a] = fwd[a] + sx * th * aspect * right[a] + sy * th * upv[a];
        }
        normalize3(d);
    }
}

/* Slab method against [0,1]^3 for t >= 0.  Returns 1 and [t0,t1] on a hit (t0 < t1). */
int orc_clip_unit_box(const double o[3], const double d[3], double* t0, double* t1)
{
    double lo = 0.0, hi = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (d[a] != 0.0) {
            double ta = (0.0 - o[a]) / d[a], tb = (1.0 - o[a]) / d[a];
            if (ta > tb) { double t = ta; ta = tb; tb = t; }
            if (ta > lo) lo = ta;
            if (tb < hi) hi = tb;
        } else if (o[a] < 0.0 || o[a] > 1.0) {
            return 0;
        }
    }
    *t0 = lo; *t1 = hi;
    return lo < hi;
}

static void tf_lookup(const orc_tf* tf, double f, double c[4])
{
    double range = tf->vmax - tf->vmin;
    double t = range > 0.0 ? (f - tf->vmin) / range : 0.0;
    if (!(t >= 0.0)) t = 0.0;
    if (t > 1.0) t = 1.0;
    const int N = tf->n_entries;
    if (N == 1) { for (int ch = 0; ch < 4; ++ch) c[ch] = tf->rgba[ch]; return; }
    double x = t * (N - 1);
    int i0 = (int)floor(x);
    if (i0 > N - 2) i0 = N - 2;
    double w = x - i0;
    for (int ch = 0; ch < 4; ++ch)
        c[ch] = (1.0 - w) * (double)tf->rgba[4 * i0 + ch] + w * (double)tf->rgba[4 * (i0 + 1) + ch];
}

static double clamp01(double x) { return x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x); }

void orc_ml_eval(double f_m, double alpha, const double uvw[3], double out[4]);

/* The scalar field a ray samples: an MFA model, or (m == NULL) the closed-form
 * Marschner-Lobb signal with constants f_m and alpha. */
typedef struct {
    const orc_model* m;
    double f_m, alpha;
} orc_field;

static void orc_field_eval(const orc_field* fld, const double x[3], double q[4])
{
    if (fld->m) orc_eval(fld->m, x, q, NULL);
    else orc_ml_eval(fld->f_m, fld->alpha, x, q);
}

/* Colour of the sample at ray parameter t (transfer function, then Phong if enabled). */
static void orc_sample_colour(const orc_field* fld, const orc_tf* tf, const double o[3], const double d[3],
                          double t, double gtiny, double c[4])
{
    double x[3] = { o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2] };
    double q[4];
    orc_field_eval(fld, x, q);
    tf_lookup(tf, q[0], c);
    if (tf->shading) {
        double g[3] = { q[1], q[2], q[3] };
        double gn = sqrt(dot3(g, g));
        double factor, spec = 0.0;
        if (gn <= gtiny) {
            factor = tf->ka + tf->kd;
        } else {
            double n[3] = { g[0] / gn, g[1] / gn, g[2] / gn };
            double L[3] = { -d[0], -d[1], -d[2] };
            double ndl = dot3(n, L);
            if (ndl < 0.0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; ndl = -ndl; }
            double R[3] = { 2.0 * ndl * n[0] - L[0], 2.0 * ndl * n[1] - L[1], 2.0 * ndl * n[2] - L[2] };
            double rv = dot3(R, L);   /* V = L for a headlight */
            spec = rv > 0.0 ? pow(rv, tf->shininess) : 0.0;
            factor = tf->ka + tf->kd * ndl;
        }
        for (int ch = 0; ch < 3; ++ch) c[ch] = clamp01(c[ch] * factor + tf->ks * spec);
    }
}

/* One pixel: returns premultiplied RGBA and the number of samples evaluated. */
static long long orc_render_pixel(const orc_field* fld, const orc_camera* cam, const orc_tf* tf,
                                  int W, int H, int ns, int col, int row, double gtiny, double rgba[4])
{
    double o[3], d[3], t0, t1;
    rgba[0] = rgba[1] = rgba[2] = rgba[3] = 0.0;
    orc_ray(cam, W, H, col, row, o, d);
    if (!orc_clip_unit_box(o, d, &t0, &t1)) return 0;
    const double dt = (t1 - t0) / ns;
    double C[3] = { 0.0, 0.0, 0.0 }, A = 0.0;
    long long count = 0;
    for (int k = 0; k < ns; ++k) {
        double c[4];
        orc_sample_colour(fld, tf, o, d, t0 + (k + 0.5) * dt, gtiny, c);
        ++count;
        double a = c[3];
        for (int ch = 0; ch < 3; ++ch) C[ch] += (1.0 - A) * a * c[ch];
        A += (1.0 - A) * a;
        if (tf->ert_alpha < 1.0 && A >= tf->ert_alpha) break;
    }
    rgba[0] = C[0]; rgba[1] = C[1]; rgba[2] = C[2]; rgba[3] = A;
    return count;
}

typedef struct {
    const orc_field* fld; const orc_camera* cam; const orc_tf* tf;
    int W, H, ns; const long long* pix; double gtiny; double* out;
} orc_render_ctx;

static void orc_render_body(void* vctx, long long b, long long e, long long* counter)
{
    orc_render_ctx* c = (orc_render_ctx*)vctx;
    for (long long i = b; i < e; ++i) {
        long long p = c->pix ? c->pix[i] : i;
        int col = (int)(p % c->W), row = (int)(p / c->W);
        *counter += orc_render_pixel(c->fld, c->cam, c->tf, c->W, c->H, c->ns, col, row, c->gtiny, &c->out[4 * i]);
    }
}

/* Renders the pixels listed in pix (indices row*W + col), or all W*H pixels when pix is
 * NULL, into out (npix * 4 doubles).  Returns the number of samples evaluated. */
/* The transfer function with vmin/vmax filled in from the control points where NaN, and
 * the gradient-norm threshold below which the normal is undefined. */
static void orc_prepare_tf(const orc_model* m, const orc_tf* tf_in, orc_tf* tf_out, double* gtiny_out)
{
    const long long total = (long long)m->n[0] * m->n[1] * m->n[2];
    double pmin = m->P[0], pmax = m->P[0];
    for (long long i = 1; i < total; ++i) {
        if (m->P[i] < pmin) pmin = m->P[i];
        if (m->P[i] > pmax) pmax = m->P[i];
    }
    orc_tf tf = *tf_in;
    if (isnan(tf.vmin)) tf.vmin = pmin;
    if (isnan(tf.vmax)) tf.vmax = pmax;
    int spans = 0;
    for (int a = 0; a < 3; ++a) if (m->n[a] - m->p[a] > spans) spans = m->n[a] - m->p[a];
    double scale = pmax - pmin;
    if (fabs(pmax) > scale) scale = fabs(pmax);
    if (fabs(pmin) > scale) scale = fabs(pmin);
    *tf_out = tf;
    *gtiny_out = 1e-6 * scale * spans;
}

long long orc_render(const orc_model* m, const orc_camera* cam, const orc_tf* tf_in,
                     int W, int H, int ns, const long long* pix, long long npix,
                     double* out, int nthreads)
{
    orc_tf tf;
    double gtiny;
    orc_prepare_tf(m, tf_in, &tf, &gtiny);
    if (!pix) npix = (long long)W * H;
    const orc_field fld = { m, 0.0, 0.0 };
    orc_render_ctx ctx = { &fld, cam, &tf, W, H, ns, pix, gtiny, out };
    return orc_parallel(npix, 16, nthreads, orc_render_body, &ctx);
}

/* ------------------------------------------------------------------------------------ */
/* Object-space decomposition (Sec. IV-A.1, IV-A.4, IV-A.5)                              */
/* ------------------------------------------------------------------------------------ */
/*
 * The volume is split into g[0] x g[1] x g[2] equal blocks of the unit box (block
 * (i, j, k) covers [i/g0, (i+1)/g0] x [j/g1, (j+1)/g1] x [k/g2, (k+1)/g2]).  Each block
 * renders, for every ray, the segment of the ray's samples that lies in it -- front to
 * back, with early termination on the segment's own accumulated alpha -- into a partial
 * image, and the partial images are combined per pixel with the over operation in front-
 * to-back order of the segments (the associativity of over, Sec. IV-A.5).  Sample k of a
 * ray stays where the single-pass render puts it, t_k = t0 + (k + 1/2) dt.  The split
 * between two neighbouring blocks is the sample index
 *     K(t_b) = clamp(ceil((t_b - t0)/dt - 1/2), 0, n_s),
 * t_b the ray parameter at their common plane, so the blocks' index ranges partition
 * 0..n_s-1 (a block face on the box boundary gives 0 or n_s; a ray parallel to an axis's
 * planes stays in the slab holding its origin, the top slab keeping the coordinate 1).
 */
#define ORC_MAX_BLOCKS 512

static int orc_split_index(double tb, double t0, double dt, int ns)
{
    double k = ceil((tb - t0) / dt - 0.5);
    if (!(k >= 0.0)) return 0;
    if (k > ns) return ns;
    return (int)k;
}

/* Sample index range [*kb, *ke) of block bi on the ray (o, d) with samples t0 + (k+1/2) dt. */
void orc_block_range(const int g[3], const int bi[3], const double o[3], const double d[3], double t0, double dt,
                     int ns, int* kb, int* ke)
{
    int lo_k = 0, hi_k = ns;
    for (int a = 0; a < 3; ++a) {
        const double lo = (double)bi[a] / g[a], hi = (double)(bi[a] + 1) / g[a];
        int k_in, k_out;
        if (d[a] > 0.0) {
            k_in = bi[a] == 0 ? 0 : orc_split_index((lo - o[a]) / d[a], t0, dt, ns);
            k_out = bi[a] == g[a] - 1 ? ns : orc_split_index((hi - o[a]) / d[a], t0, dt, ns);
        } else if (d[a] < 0.0) {
            k_in = bi[a] == g[a] - 1 ? 0 : orc_split_index((hi - o[a]) / d[a], t0, dt, ns);
            k_out = bi[a] == 0 ? ns : orc_split_index((lo - o[a]) / d[a], t0, dt, ns);
        } else {
            const int inside = (o[a] >= lo && o[a] < hi) || (bi[a] == g[a] - 1 && o[a] == hi);
            k_in = inside ? 0 : ns;
            k_out = inside ? ns : 0;
        }
        if (k_in > lo_k) lo_k = k_in;
        if (k_out < hi_k) hi_k = k_out;
    }
    *kb = lo_k;
    *ke = hi_k;
}

static long long orc_render_pixel_segments(const orc_model* m, const orc_camera* cam, const orc_tf* tf, int W,
                                           int H, int ns, const int g[3], int col, int row, double gtiny,
                                           double rgba[4])
{
    double o[3], d[3], t0, t1;
    rgba[0] = rgba[1] = rgba[2] = rgba[3] = 0.0;
    orc_ray(cam, W, H, col, row, o, d);
    if (!orc_clip_unit_box(o, d, &t0, &t1)) return 0;
    const double dt = (t1 - t0) / ns;
    const int nb = g[0] * g[1] * g[2];
    const orc_field fld = { m, 0.0, 0.0 };
    int kb[ORC_MAX_BLOCKS], ke[ORC_MAX_BLOCKS], done[ORC_MAX_BLOCKS];
    double part[ORC_MAX_BLOCKS][4];
    long long count = 0;
    for (int b = 0; b < nb; ++b) {
        const int bi[3] = { b % g[0], (b / g[0]) % g[1], b / (g[0] * g[1]) };
        orc_block_range(g, bi, o, d, t0, dt, ns, &kb[b], &ke[b]);
        done[b] = kb[b] >= ke[b];
        double C[3] = { 0.0, 0.0, 0.0 }, A = 0.0;
        for (int k = kb[b]; k < ke[b]; ++k) {   /* the block's segment, front to back */
            double c[4];
            orc_sample_colour(&fld, tf, o, d, t0 + (k + 0.5) * dt, gtiny, c);
            ++count;
            double a = c[3];
            for (int ch = 0; ch < 3; ++ch) C[ch] += (1.0 - A) * a * c[ch];
            A += (1.0 - A) * a;
            if (tf->ert_alpha < 1.0 && A >= tf->ert_alpha) break;
        }
        part[b][0] = C[0]; part[b][1] = C[1]; part[b][2] = C[2]; part[b][3] = A;
    }
    /* over of the partial images, nearest segment first */
    double C[3] = { 0.0, 0.0, 0.0 }, A = 0.0;
    for (;;) {
        int next = -1;
        for (int b = 0; b < nb; ++b)
            if (!done[b] && (next < 0 || kb[b] < kb[next])) next = b;
        if (next < 0) break;
        done[next] = 1;
        for (int ch = 0; ch < 3; ++ch) C[ch] += (1.0 - A) * part[next][ch];
        A += (1.0 - A) * part[next][3];
    }
    rgba[0] = C[0]; rgba[1] = C[1]; rgba[2] = C[2]; rgba[3] = A;
    return count;
}

typedef struct {
    const orc_model* m; const orc_camera* cam; const orc_tf* tf;
    int W, H, ns; const int* g; const long long* pix; double gtiny; double* out;
} orc_segments_ctx;

static void orc_segments_body(void* vctx, long long b, long long e, long long* counter)
{
    orc_segments_ctx* c = (orc_segments_ctx*)vctx;
    for (long long i = b; i < e; ++i) {
        long long p = c->pix ? c->pix[i] : i;
        int col = (int)(p % c->W), row = (int)(p / c->W);
        *counter += orc_render_pixel_segments(c->m, c->cam, c->tf, c->W, c->H, c->ns, c->g, col, row, c->gtiny,
                                              &c->out[4 * i]);
    }
}

/* orc_render with the volume split into g[0] x g[1] x g[2] blocks (at most 512) rendered
 * as separate segments and merged with over.  Returns the samples evaluated, -1 on a bad g. */
long long orc_render_segments(const orc_model* m, const orc_camera* cam, const orc_tf* tf_in, int W, int H, int ns,
                              const int g[3], const long long* pix, long long npix, double* out, int nthreads)
{
    if (g[0] < 1 || g[1] < 1 || g[2] < 1 || (long long)g[0] * g[1] * g[2] > ORC_MAX_BLOCKS) return -1;
    orc_tf tf;
    double gtiny;
    orc_prepare_tf(m, tf_in, &tf, &gtiny);
    if (!pix) npix = (long long)W * H;
    orc_segments_ctx ctx = { m, cam, &tf, W, H, ns, g, pix, gtiny, out };
    return orc_parallel(npix, 16, nthreads, orc_segments_body, &ctx);
}

/* ------------------------------------------------------------------------------------ */
/* Isosurface rendering through MFA queries (Sec. IV-A.4 names isosurface rendering as  */
/* the other visualization the query interface serves)                                    */
/* ------------------------------------------------------------------------------------ */
/*
 * Per ray: the samples of the volume render, t_k = t0 + (k + 1/2) dt, are queried in
 * order; the first k with g(t_{k-1}) and g(t_k) of opposite signs (or g(t_k) = 0), where
 * g(t) = f(o + t d) - iso, brackets the first crossing.  The crossing is refined by
 * ORC_ISO_STEPS Newton steps on g with the analytic derivative g'(t) = grad f . d, started
 * at the bracket's midpoint and kept inside the bracket: each step queries g at t (stopping
 * if it is exactly 0), shrinks the bracket to the side where g changes sign, then takes the
 * Newton point if it lies in the bracket (ends included), else the new midpoint.  The hit is shaded like a volume sample with value iso at
 * that point: the transfer function's colour at iso, Phong with the normal
 * grad f / |grad f| (two-sided headlight), alpha 1.  A ray without a crossing is
 * transparent black.  The count is every query made (samples and refinement steps).
 */
#define ORC_ISO_STEPS 8

static void orc_query_on_ray(const orc_model* m, const double o[3], const double d[3], double t, double q[4])
{
    double x[3] = { o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2] };
    orc_eval(m, x, q, NULL);
}

static long long orc_iso_pixel(const orc_model* m, const orc_camera* cam, const orc_tf* tf, int W, int H, int ns,
                               double iso, int col, int row, double gtiny, double rgba[4], double* depth)
{
    double o[3], d[3], t0, t1;
    rgba[0] = rgba[1] = rgba[2] = rgba[3] = 0.0;
    *depth = INFINITY;
    orc_ray(cam, W, H, col, row, o, d);
    if (!orc_clip_unit_box(o, d, &t0, &t1)) return 0;
    const double dt = (t1 - t0) / ns;
    long long count = 0;
    double q[4], ta = 0.0, ga = 0.0, tb = 0.0;
    int found = 0;
    for (int k = 0; k < ns && !found; ++k) {
        const double t = t0 + (k + 0.5) * dt;
        orc_query_on_ray(m, o, d, t, q);
        ++count;
        const double g = q[0] - iso;
        if (g == 0.0) {
            ta = tb = t;
            ga = 0.0;
            found = 1;
        } else if (k > 0 && ((ga < 0.0) != (g < 0.0))) {
            tb = t;
            found = 1;
        } else {
            ta = t;
            ga = g;
        }
    }
    if (!found) return count;
    double t = 0.5 * (ta + tb);
    if (ta != tb) {
        for (int s = 0; s < ORC_ISO_STEPS; ++s) {
            orc_query_on_ray(m, o, d, t, q);
            ++count;
            const double g = q[0] - iso;
            if (g == 0.0) break;   /* t is the root */
            if ((g < 0.0) == (ga < 0.0)) { ta = t; ga = g; } else { tb = t; }
            const double dg = q[1] * d[0] + q[2] * d[1] + q[3] * d[2];
            const double tn = dg != 0.0 ? t - g / dg : NAN;
            t = (tn >= ta && tn <= tb) ? tn : 0.5 * (ta + tb);
        }
    }
    orc_query_on_ray(m, o, d, t, q);   /* the normal at the hit */
    ++count;
    double c[4];
    tf_lookup(tf, iso, c);
    if (tf->shading) {
        double g[3] = { q[1], q[2], q[3] };
        double gn = sqrt(dot3(g, g));
        double factor, spec = 0.0;
        if (gn <= gtiny) {
            factor = tf->ka + tf->kd;
        } else {
            double n[3] = { g[0] / gn, g[1] / gn, g[2] / gn };
            double L[3] = { -d[0], -d[1], -d[2] };
            double ndl = dot3(n, L);
            if (ndl < 0.0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; ndl = -ndl; }
            double R[3] = { 2.0 * ndl * n[0] - L[0], 2.0 * ndl * n[1] - L[1], 2.0 * ndl * n[2] - L[2] };
            double rv = dot3(R, L);
            spec = rv > 0.0 ? pow(rv, tf->shininess) : 0.0;
            factor = tf->ka + tf->kd * ndl;
        }
        for (int ch = 0; ch < 3; ++ch) c[ch] = clamp01(c[ch] * factor + tf->ks * spec);
    }
    rgba[0] = c[0]; rgba[1] = c[1]; rgba[2] = c[2]; rgba[3] = 1.0;
    *depth = t;
    return count;
}

typedef struct {
    const orc_model* m; const orc_camera* cam; const orc_tf* tf;
    int W, H, ns; double iso; const long long* pix; double gtiny; double* out; double* depth;
} orc_iso_ctx;

static void orc_iso_body(void* vctx, long long b, long long e, long long* counter)
{
    orc_iso_ctx* c = (orc_iso_ctx*)vctx;
    for (long long i = b; i < e; ++i) {
        long long p = c->pix ? c->pix[i] : i;
        int col = (int)(p % c->W), row = (int)(p / c->W);
        *counter += orc_iso_pixel(c->m, c->cam, c->tf, c->W, c->H, c->ns, c->iso, col, row, c->gtiny, &c->out[4 * i],
                                  &c->depth[i]);
    }
}

/* Isosurface image of the pixels listed in pix (or all W*H): premultiplied RGBA in out
 * (npix * 4) and the hit parameter t in depth (npix; +inf where the ray misses).
 * Returns the number of queries made. */
long long orc_render_iso(const orc_model* m, const orc_camera* cam, const orc_tf* tf_in, int W, int H, int ns,
                         double iso, const long long* pix, long long npix, double* out, double* depth, int nthreads)
{
    orc_tf tf;
    double gtiny;
    orc_prepare_tf(m, tf_in, &tf, &gtiny);
    if (!pix) npix = (long long)W * H;
    orc_iso_ctx ctx = { m, cam, &tf, W, H, ns, iso, pix, gtiny, out, depth };
    return orc_parallel(npix, 16, nthreads, orc_iso_body, &ctx);
}

/* ------------------------------------------------------------------------------------ */
/* Ground truth of the Marschner-Lobb workload (Sec. V-A.1, Eq. 1)                        */
/* ------------------------------------------------------------------------------------ */
/*
 * The paper evaluates its renders against the closed-form signal
 *     F(x, y, z) = (1 - sin(pi z / 2) + alpha (1 + rho(r))) / (2 (1 + alpha)),
 *     rho(r) = cos(2 pi f_M cos(pi r / 2)),  r = sqrt(x^2 + y^2),
 * rendered directly (its "ground truth" image, Sec. V-D.3).  Reading: the signal lives on
 * [-1, 1]^3 and the unit parameter box maps onto it by x = 2u - 1 (likewise y, z), so the
 * gradient with respect to (u, v, w) is twice the one with respect to (x, y, z):
 *     dF/dz = -(pi / 2) cos(pi z / 2) / (2 (1 + alpha)),
 *     dF/dx = alpha rho'(r) (x / r) / (2 (1 + alpha)),   likewise dF/dy with y,
 *     rho'(r) = pi^2 f_M sin(2 pi f_M cos(pi r / 2)) sin(pi r / 2),
 * where rho'(r) / r is continued to r = 0 by sin(pi r / 2) / r -> pi / 2.  F spans [0, 1]
 * exactly, which is the transfer function's default value range here; the normal is
 * undefined where |grad F| <= 1e-6 (the field's range times 1e-6).
 */
void orc_ml_eval(double f_m, double alpha, const double uvw[3], double out[4])
{
    const double x = 2.0 * uvw[0] - 1.0, y = 2.0 * uvw[1] - 1.0, z = 2.0 * uvw[2] - 1.0;
    const double r = sqrt(x * x + y * y);
    const double c = cos(M_PI * r / 2.0);
    const double rho = cos(2.0 * M_PI * f_m * c);
    const double den = 2.0 * (1.0 + alpha);
    out[0] = (1.0 - sin(M_PI * z / 2.0) + alpha * (1.0 + rho)) / den;
    const double sinc = r > 0.0 ? sin(M_PI * r / 2.0) / r : M_PI / 2.0;
    const double drho_over_r = M_PI * M_PI * f_m * sin(2.0 * M_PI * f_m * c) * sinc;
    out[1] = 2.0 * alpha * drho_over_r * x / den;
    out[2] = 2.0 * alpha * drho_over_r * y / den;
    out[3] = 2.0 * (-(M_PI / 2.0) * cos(M_PI * z / 2.0)) / den;
}

/* render() of the closed-form signal instead of a model. */
long long orc_render_ml(double f_m, double alpha, const orc_camera* cam, const orc_tf* tf_in, int W, int H, int ns,
                        const long long* pix, long long npix, double* out, int nthreads)
{
    orc_tf tf = *tf_in;
    if (isnan(tf.vmin)) tf.vmin = 0.0;
    if (isnan(tf.vmax)) tf.vmax = 1.0;
    if (!pix) npix = (long long)W * H;
    const orc_field fld = { NULL, f_m, alpha };
    orc_render_ctx ctx = { &fld, cam, &tf, W, H, ns, pix, 1e-6, out };
    return orc_parallel(npix, 16, nthreads, orc_render_body, &ctx);
}
