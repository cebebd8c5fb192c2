// bspline.cuh -- device building blocks of one MFA value+gradient query (Sec. III-B,
// Sec. V-D.3): knot-span location per axis, basis values and derivatives on the span,
// and the (p+1)^3 control-point contraction for the value and the three partials.
//
// Arithmetic is FP32 throughout.  The contraction uses packed FP32x2 instructions
// (`fma.rn.f32x2`, `mul.rn.f32x2` on sm_100+) over pairs of z-layers, which the layer-pair
// window layout delivers as ready operands; this halves the issue slots of the dominant
// loop.  Each lane of a packed op is an ordinary FP32
// round-to-nearest FMA / multiply.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "mfa_internal.cuh"

namespace mfa {

// ----------------------------------------------------------------------------------------
// knot spans
// ----------------------------------------------------------------------------------------

// Knot span of u (u already clamped to [0,1]): the largest s in [p, n-1] with
// U[s] <= u.  kup holds the knots rounded up to FP32, so the FP32 comparisons below give
// exactly the answer of the FP64 comparisons on the FP32 value of u.  The grid supplies
// a starting span; the two walks fix it up (at most a few steps: G = 4 (n - p) cells).
__device__ __forceinline__ int locate_span(const AxisDev& A, float u)
{
    int g = min(static_cast<int>(u * A.Gf), A.G - 1);
    int s = __ldg(A.grid + g);
    while (s < A.n - 1 && u >= __ldg(A.kup + s + 1)) ++s;
    while (s > A.p && u < __ldg(A.kup + s)) --s;
    return s;
}

// Same, starting from a previous span (a ray's last sample): u moves monotonically along
// an axis, so this is usually zero or one step.
__device__ __forceinline__ int walk_span(const AxisDev& A, float u, int s)
{
    while (s < A.n - 1 && u >= __ldg(A.kup + s + 1)) ++s;
    while (s > A.p && u < __ldg(A.kup + s)) --s;
    return s;
}

// ----------------------------------------------------------------------------------------
// packed FP32x2 helpers
// ----------------------------------------------------------------------------------------

struct f2 {
    unsigned long long v;
};

__device__ __forceinline__ f2 pk2(float a, float b)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(f2 x, float& a, float& b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x.v)); }
__device__ __forceinline__ float hsum2(f2 x)
{
    float a, b;
    upk2(x, a, b);
    return a + b;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b)
{
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}

// ----------------------------------------------------------------------------------------
// span records and basis functions
// ----------------------------------------------------------------------------------------

// A span record {U_s, 1/h, lo, hi, c[k][r]} copied into registers.
template <int Q>
__device__ __forceinline__ void load_record(const AxisDev& A, int s, float (&rec)[rec_stride(Q)])
{
    constexpr int RS = rec_stride(Q);
    int r = s - A.p;
    MFA_DBG_INDEX(A.dbg, r, A.n - A.p, kDbgRecord);
    const float4* r4 = reinterpret_cast<const float4*>(A.rec + r * RS);
#pragma unroll
    for (int v = 0; v < RS / 4; ++v) {
        float4 x = __ldg(r4 + v);
        rec[4 * v + 0] = x.x;
        rec[4 * v + 1] = x.y;
        rec[4 * v + 2] = x.z;
        rec[4 * v + 3] = x.w;
    }
}

// The Q basis functions N_{s-p+r,p} on the record's span (zero for r > p) and their
// derivatives with respect to the local coordinate t = (u - U_s)/h (record_basis_t takes t,
// record_basis takes u), by joint Horner
// evaluation of the power-basis coefficients (value b and derivative d together:
// d <- d t + b, b <- b t + c_k).  d/du = (1/h) d/dt = rec[1] d/dt.
template <int Q>
__device__ __forceinline__ void record_basis_t(const float (&rec)[rec_stride(Q)], float t, float (&N)[Q], float (&D)[Q])
{
    constexpr int QP = qpair(Q);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        float b = rec[kRecHead + (Q - 1) * QP + i], d = 0.0f;
#pragma unroll
        for (int k = Q - 2; k >= 0; --k) {
            d = fmaf(d, t, b);
            b = fmaf(b, t, rec[kRecHead + k * QP + i]);
        }
        N[i] = b;
        D[i] = d;
    }
}

template <int Q>
__device__ __forceinline__ void record_basis(const float (&rec)[rec_stride(Q)], float u, float (&N)[Q], float (&D)[Q])
{
    record_basis_t<Q>(rec, (u - rec[0]) * rec[1], N, D);
}

// Packed form: functions (2m, 2m+1) advance together; N2[m] = {N_2m, N_2m+1}, D2 likewise.
template <int Q>
__device__ __forceinline__ void record_basis2(const float (&rec)[rec_stride(Q)], float u, f2 (&N2)[qpair(Q) / 2],
                                              f2 (&D2)[qpair(Q) / 2])
{
    constexpr int QP = qpair(Q);
    const float t = (u - rec[0]) * rec[1];
    const f2 t2 = pk2(t, t);
#pragma unroll
    for (int m = 0; m < QP / 2; ++m) {
        f2 b = pk2(rec[kRecHead + (Q - 1) * QP + 2 * m], rec[kRecHead + (Q - 1) * QP + 2 * m + 1]);
        f2 d = b;                                   // first step of d <- d t + b with d = 0
        b = fma2(b, t2, pk2(rec[kRecHead + (Q - 2) * QP + 2 * m], rec[kRecHead + (Q - 2) * QP + 2 * m + 1]));
#pragma unroll
        for (int k = Q - 3; k >= 0; --k) {
            d = fma2(d, t2, b);
            b = fma2(b, t2, pk2(rec[kRecHead + k * QP + 2 * m], rec[kRecHead + k * QP + 2 * m + 1]));
        }
        N2[m] = b;
        D2[m] = d;
    }
}

// Loads span s's record and evaluates it at u; inv_h receives 1/h.
template <int Q>
__device__ __forceinline__ void span_basis(const AxisDev& A, int s, float u, float (&N)[Q], float (&D)[Q],
                                           float& inv_h)
{
    float rec[rec_stride(Q)];
    load_record<Q>(A, s, rec);
    inv_h = rec[1];
    record_basis<Q>(rec, u, N, D);
}

// ----------------------------------------------------------------------------------------
// uniform knots: the cardinal basis
// ----------------------------------------------------------------------------------------
//
// With uniform knot spacing h, the Cox-de Boor recursion (Sec. III-B) has integer knot
// differences in units of h.  On one span, with local coordinate t in [0,1), the degree-k
// functions r = 0..k that are non-zero there satisfy
//   N^k_r = ((t + k - r) N^{k-1}_{r-1} + (r + 1 - t) N^{k-1}_r) / k,   N^0_0 = 1,
// (out-of-range terms zero) and dN^p_r/dt = N^{p-1}_{r-1} - N^{p-1}_r.  cardinal_basis
// returns the scaled values M = p! N^p and G = (p-1)! dN^p/dt, which drops every division
// from the triangle; the contraction's results are scaled back once per sample.  This holds
// on every span whose 2p surrounding knots are all uniform, i.e. all spans but the p-1 at
// each end of a clamped knot vector.  The y and z weights are always the scaled M and G;
// the x factor is scaled the same way on 16-bit models and exact on FP32 models, whose
// window rows carry the x span's polynomial (power rows, below), hence the per-storage
// scale factors of the value, the x partial and the y / z partials.
__host__ __device__ constexpr float factorial(int k) { return k <= 1 ? 1.0f : k * factorial(k - 1); }
template <int Q>
struct Cardinal {
    static constexpr int p = Q - 1;
    static constexpr float kBasisScale = factorial(p);        // M = kBasisScale N
    static constexpr float kDerivScale = factorial(p - 1);    // G = kDerivScale dN/dt
    template <int STORAGE>
    static constexpr float x_val() { return power_rows(Q, STORAGE) ? 1.0f : factorial(p); }
    template <int STORAGE>
    static constexpr float x_der() { return power_rows(Q, STORAGE) ? 1.0f : factorial(p - 1); }
    template <int STORAGE>
    static constexpr float val_scale() { return 1.0f / (x_val<STORAGE>() * factorial(p) * factorial(p)); }
    template <int STORAGE>
    static constexpr float gradx_scale() { return 1.0f / (x_der<STORAGE>() * factorial(p) * factorial(p)); }
    template <int STORAGE>
    static constexpr float gradyz_scale() { return 1.0f / (x_val<STORAGE>() * factorial(p - 1) * factorial(p)); }
};

template <int Q>
__device__ __forceinline__ void cardinal_basis(float t, float (&M)[Q], float (&G)[Q])
{
    const float s = 1.0f - t;
    if constexpr (Q == 4) {
        // p = 3 written out: M = {s^3, 3t^3 - 6t^2 + 4, 3s^3 - 6s^2 + 4, t^3},
        // G = differences of the quadratic level {s^2, 1 + 2ts, t^2}
        const float t2 = t * t, s2 = s * s;
        M[0] = s2 * s;
        M[1] = fmaf(t2, fmaf(3.0f, t, -6.0f), 4.0f);
        M[2] = fmaf(s2, fmaf(3.0f, s, -6.0f), 4.0f);
        M[3] = t2 * t;
        G[0] = -s2;
        G[1] = t * fmaf(3.0f, t, -4.0f);
        G[2] = s * fmaf(3.0f, t, 1.0f);
        G[3] = t2;
    } else {
        float L[Q];   // level k of the triangle, scaled by k!
        L[0] = 1.0f;
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            if (k == Q - 1) {
                G[0] = -L[0];
#pragma unroll
                for (int r = 1; r < k; ++r) G[r] = L[r - 1] - L[r];
                G[k] = L[k - 1];
            }
            L[k] = t * L[k - 1];
#pragma unroll
            for (int r = k - 1; r >= 1; --r)
                L[r] = fmaf(t + static_cast<float>(k - r), L[r - 1], (static_cast<float>(r + 1) - t) * L[r]);
            L[0] = s * L[0];
        }
#pragma unroll
        for (int r = 0; r < Q; ++r) M[r] = L[r];
    }
}

// ----------------------------------------------------------------------------------------
// control-point layer pairs
// ----------------------------------------------------------------------------------------

// One window entry (k, j, i) as QP column pairs: pr[a] = {P[k][j][i+a], P[k+1][j][i+a]}
// (the same row of two consecutive z-layers side by side, the layout of a packed FP32x2
// operand).  Entries past Q meet zero basis values; they are always inside the
// zero-padded window array.  FP32: one 256-bit load (a 16-byte one for Q = 2; Q = 5 adds
// 16 bytes of entry i + 4).  load_triple (Q = 3) also returns the entry's third-layer row
// r3[a] = P[k+2][j][i+a] (a 128-bit load of the entry's second half).
template <int Q>
struct PairF32 {
    static __device__ __forceinline__ void load(const ModelDev& M, int idx, f2 (&pr)[qpair(Q)])
    {
        const float* e = static_cast<const float*>(M.win) + static_cast<long long>(window_values(Q)) * idx;
        if constexpr (qpair(Q) == 2) {
            asm("ld.global.nc.v2.b64 {%0, %1}, [%2];" : "=l"(pr[0].v), "=l"(pr[1].v) : "l"(e));
        } else {
            asm("ld.global.nc.v4.b64 {%0, %1, %2, %3}, [%4];"
                : "=l"(pr[0].v), "=l"(pr[1].v), "=l"(pr[2].v), "=l"(pr[3].v)
                : "l"(e));
        }
        if constexpr (qpair(Q) == 6)
            asm("ld.global.nc.v2.b64 {%0, %1}, [%2];" : "=l"(pr[4].v), "=l"(pr[5].v) : "l"(e + 32));
    }
    static __device__ __forceinline__ void load_triple(const ModelDev& M, int idx, f2 (&pr)[4], float (&r3)[4])
    {
        static_assert(Q == 3, "third-layer rows exist in degree-class-3 windows only");
        load(M, idx, pr);
        const float* e = static_cast<const float*>(M.win) + static_cast<long long>(window_values(Q)) * idx;
        asm("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
            : "=f"(r3[0]), "=f"(r3[1]), "=f"(r3[2]), "=f"(r3[3])
            : "l"(e + 8));
    }
};

// 16-bit storage: an entry is 16 bytes, one 32-bit word {layer k, layer k+1} per column
// (32 bytes for Q = 3, the third-layer row in the first 8 bytes of the second half).
template <int Q, bool BF16>
struct Pair16 {
    static __device__ __forceinline__ float2 cvt(unsigned int bits)
    {
        if constexpr (BF16) {
            // BF16 is the upper half of an FP32 pattern: the word's high value is the word
            // with its low 16 bits cleared, the low value the word shifted up by 16 (two
            // integer operations, no conversion instruction)
            return make_float2(__uint_as_float(bits << 16), __uint_as_float(bits & 0xFFFF0000u));
        } else {
            __half2 h = *reinterpret_cast<__half2*>(&bits);
            return __half22float2(h);
        }
    }
    static __device__ __forceinline__ f2 cvt2(unsigned int bits)
    {
        const float2 x = cvt(bits);
        return pk2(x.x, x.y);
    }
    static __device__ __forceinline__ void load(const ModelDev& M, int idx, f2 (&pr)[qpair(Q)])
    {
        const unsigned short* e = static_cast<const unsigned short*>(M.win) + static_cast<long long>(window_values(Q)) * idx;
        if constexpr (qpair(Q) == 2) {
            const uint2 w = __ldg(reinterpret_cast<const uint2*>(e));
            pr[0] = cvt2(w.x);
            pr[1] = cvt2(w.y);
        } else {
            const uint4 w = __ldg(reinterpret_cast<const uint4*>(e));
            pr[0] = cvt2(w.x);
            pr[1] = cvt2(w.y);
            pr[2] = cvt2(w.z);
            pr[3] = cvt2(w.w);
        }
        if constexpr (qpair(Q) == 6) {
            const uint2 w = __ldg(reinterpret_cast<const uint2*>(e + 32));
            pr[4] = cvt2(w.x);
            pr[5] = cvt2(w.y);
        }
    }
    static __device__ __forceinline__ void load_triple(const ModelDev& M, int idx, f2 (&pr)[4], float (&r3)[4])
    {
        static_assert(Q == 3, "third-layer rows exist in degree-class-3 windows only");
        load(M, idx, pr);
        const unsigned short* e = static_cast<const unsigned short*>(M.win) + static_cast<long long>(window_values(Q)) * idx;
        const uint2 w = __ldg(reinterpret_cast<const uint2*>(e + 8));
        const float2 lo = cvt(w.x), hi = cvt(w.y);
        r3[0] = lo.x;
        r3[1] = lo.y;
        r3[2] = hi.x;
        r3[3] = hi.y;
    }
};

// The compact layout: the stored values at V / S times the zero-padded plain array, no layer
// pairs, S = compact_stride(Q, type), V = compact_values(type).  Each padded x-row of n_xp
// values (n_xp a multiple of S) is kept as n_xp / S entries of V values, entry e holding the
// row's values S e .. S e + V - 1 (zeros past the row's end).  16-bit types: eight values
// every S = 9 - Q positions (1.6x at degree 3), so the Q values of any support row lie
// inside the entry it starts in: one aligned 16-byte load per row.  FP32: four values every
// four positions (the plain array), a row read as its entry and the next (two aligned
// 16-byte loads, mostly from one 32-byte sector).  Then a select by the row's offset
// s = i mod S in the entry, one step per bit of s.  A window index idx is the position of P[k][j][i] in the
// padded plain array (below 2^31); since rows hold whole entries its entry is idx / S and
// its offset idx mod S, and the layer k+1 lies n_xp n_yp positions further.  Values a
// column pair needs beyond the Q of its row (the padding column of degree classes 3 and 5)
// are zero; they meet zero basis values.
template <int Q, int VT>
struct PairCompact {
    static constexpr int S = compact_stride(Q, VT + 3);
    static constexpr int QP = qpair(Q);
    static __device__ __forceinline__ void entry_of(long long idx, unsigned& e, int& s)
    {
        const unsigned u = static_cast<unsigned>(idx);
        e = u / S;
        s = static_cast<int>(u - e * S);
    }
    // FP32: the row's values v[s .. s + Q - 1] (zero past them) from its entry and the next
    // one (eight values from two aligned 16-byte loads; s <= 3, so s + Q - 1 <= 7)
    static __device__ __forceinline__ void row(const ModelDev& M, long long idx, float (&o)[QP])
    {
        static_assert(S == 4, "FP32 compact entries are four values every four positions");
        unsigned e;
        int s;
        entry_of(idx, e, s);
        const float* p = static_cast<const float*>(M.win) + 4ull * e;
        const float4 v0 = __ldg(reinterpret_cast<const float4*>(p)), v1 = __ldg(reinterpret_cast<const float4*>(p + 4));
        const float v[12] = { v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w, 0.0f, 0.0f, 0.0f, 0.0f };
        // b = v shifted by 2 (s & 2), o = b shifted by 1 (s & 1)
        float b[QP + 1];
#pragma unroll
        for (int x = 0; x <= QP; ++x) b[x] = (s & 2) ? v[x + 2] : v[x];
#pragma unroll
        for (int x = 0; x < QP; ++x) o[x] = x < Q ? ((s & 1) ? b[x + 1] : b[x]) : 0.0f;
    }
    // 16-bit: the row's values as 32-bit words of two, word c = {v[s + 2c], v[s + 2c + 1]},
    // from one 128-bit load: word shifts by the bits 2 and 1 of s, a byte permute by bit 0
    static constexpr int NW = QP / 2;
    static __device__ __forceinline__ void row16(const ModelDev& M, long long idx, unsigned (&o)[NW])
    {
        unsigned e;
        int s;
        entry_of(idx, e, s);
        const uint4 q = __ldg(static_cast<const uint4*>(M.win) + e);
        const unsigned W[4] = { q.x, q.y, q.z, q.w };
        unsigned A[NW + 2], B[NW + 1];
#pragma unroll
        for (int x = 0; x < NW + 2; ++x) {
            const unsigned lo = x < 4 ? W[x] : 0u, hi = x + 2 < 4 ? W[x + 2] : 0u;
            A[x] = (S > 4 && (s & 4)) ? hi : lo;
        }
#pragma unroll
        for (int x = 0; x <= NW; ++x) B[x] = (s & 2) ? A[x + 1] : A[x];
        const unsigned sel = (s & 1) ? 0x5432u : 0x3210u;
#pragma unroll
        for (int c = 0; c < NW; ++c) o[c] = __byte_perm(B[c], B[c + 1], sel);
    }
    static __device__ __forceinline__ f2 cvt2(unsigned bits) { return Pair16<Q, VT == 3>::cvt2(bits); }
    static __device__ __forceinline__ void load(const ModelDev& M, int idx, f2 (&pr)[QP])
    {
        const long long layer = static_cast<long long>(M.nxp) * M.nyp;
        if constexpr (VT == 1) {
            float lo[QP], hi[QP];
            row(M, idx, lo);
            row(M, idx + layer, hi);
#pragma unroll
            for (int a = 0; a < QP; ++a) pr[a] = pk2(lo[a], hi[a]);
        } else {
            unsigned lo[NW], hi[NW];
            row16(M, idx, lo);
            row16(M, idx + layer, hi);
            // column pairs {layer k, layer k+1} as the 16-bit window's words
#pragma unroll
            for (int c = 0; c < NW; ++c) {
                pr[2 * c] = cvt2(__byte_perm(lo[c], hi[c], 0x5410u));
                pr[2 * c + 1] = cvt2(__byte_perm(lo[c], hi[c], 0x7632u));
            }
        }
    }
    static __device__ __forceinline__ void load_triple(const ModelDev& M, int idx, f2 (&pr)[4], float (&r3)[4])
    {
        static_assert(Q == 3, "third-layer rows exist in degree class 3 only");
        load(M, idx, pr);
        const long long layer2 = 2ll * M.nxp * M.nyp;
        if constexpr (VT == 1) {
            row(M, idx + layer2, r3);
        } else {
            unsigned w[NW];
            row16(M, idx + layer2, w);
#pragma unroll
            for (int c = 0; c < NW; ++c) {
                const float2 x = Pair16<Q, VT == 3>::cvt(w[c]);
                r3[2 * c] = x.x;
                r3[2 * c + 1] = x.y;
            }
        }
    }
};

template <int Q, int STORAGE>
struct PairLoader;
template <int Q> struct PairLoader<Q, 1> : PairF32<Q> {};          // MFA_F32 layer pairs
template <int Q> struct PairLoader<Q, 2> : Pair16<Q, false> {};    // MFA_F16 layer pairs
template <int Q> struct PairLoader<Q, 3> : Pair16<Q, true> {};     // MFA_BF16 layer pairs
template <int Q> struct PairLoader<Q, 4> : PairCompact<Q, 1> {};   // compact FP32
template <int Q> struct PairLoader<Q, 5> : PairCompact<Q, 2> {};   // compact FP16
template <int Q> struct PairLoader<Q, 6> : PairCompact<Q, 3> {};   // compact BF16

// ----------------------------------------------------------------------------------------
// the x-pass: power rows (FP32 models) or basis-weighted rows (16-bit models)
// ----------------------------------------------------------------------------------------
//
// On one x span the B-spline restricted to a row of control points is a polynomial in the
// span's local coordinate t: sum_r N_{i+r}(t) P_{i+r} = sum_c W_c t^c with
// W_c = sum_r c_{c,r} P_{i+r}, c_{c,r} the power-basis coefficients of the span's basis
// functions.  FP32 models store W in place of P in each window row (computed in FP64 from
// the stored control points at model creation, then rounded once to FP32; a row is only
// ever read by samples in its own x span), so the x-pass is a Horner evaluation: Q-1
// packed FMAs for the row's value A and Q-2 for dA/dt, against 2Q for the basis-weighted
// sums, and the x basis itself is never evaluated.  16-bit models keep the control points
// (W in 16 bits would add its own rounding to the model) and weight them by the x basis.

// What the x-pass needs: the local coordinate t (power rows) or the x basis values and
// derivatives (control-point rows).  XPk is the same packed for the FP32x2 x-pass, each
// value duplicated into both lanes; contractions pack their input on entry.
template <int Q, bool POW>
struct XInT {
    float n[Q], d[Q];
};
template <int Q>
struct XInT<Q, true> {
    float t;
};
template <int Q, int STORAGE>
using XIn = XInT<Q, power_rows(Q, STORAGE)>;

template <int Q, bool POW>
struct XPk {
    f2 n[Q], d[Q];
};
template <int Q>
struct XPk<Q, true> {
    f2 t;
};

// A = sum_c W_c t^c and B = dA/dt of a window row (both z-layers of the pair at once), by
// one Horner sweep that carries the derivative: d <- d t + a, a <- a t + W_c.
template <int Q>
__device__ __forceinline__ void power_row(const f2 (&w)[qpair(Q)], f2 t, f2& A, f2& B)
{
    if constexpr (Q == 2) {
        A = fma2(w[1], t, w[0]);
        B = w[1];
    } else {
        f2 a = fma2(w[Q - 1], t, w[Q - 2]);
        f2 d = w[Q - 1];
#pragma unroll
        for (int c = Q - 3; c >= 0; --c) {
            d = fma2(d, t, a);
            a = fma2(a, t, w[c]);
        }
        A = a;
        B = d;
    }
}

// The row's value only.
template <int Q>
__device__ __forceinline__ f2 power_row_value(const f2 (&w)[qpair(Q)], f2 t)
{
    f2 a = fma2(w[Q - 1], t, w[Q - 2]);
#pragma unroll
    for (int c = Q - 3; c >= 0; --c) a = fma2(a, t, w[c]);
    return a;
}

// {A, B} of one window row for either kind of row.
template <int Q, int STORAGE>
__device__ __forceinline__ void x_row(const f2 (&pr)[qpair(Q)], const XPk<Q, power_rows(Q, STORAGE)>& X, f2& A,
                                      f2& B)
{
    if constexpr (power_rows(Q, STORAGE)) {
        power_row<Q>(pr, X.t, A, B);
    } else {
        A = mul2(X.n[0], pr[0]);
        B = mul2(X.d[0], pr[0]);
#pragma unroll
        for (int a = 1; a < Q; ++a) {
            A = fma2(X.n[a], pr[a], A);
            B = fma2(X.d[a], pr[a], B);
        }
    }
}

template <int Q, int STORAGE>
__device__ __forceinline__ f2 x_row_value(const f2 (&pr)[qpair(Q)], const XPk<Q, power_rows(Q, STORAGE)>& X)
{
    if constexpr (power_rows(Q, STORAGE)) {
        return power_row_value<Q>(pr, X.t);
    } else {
        f2 A = mul2(X.n[0], pr[0]);
#pragma unroll
        for (int a = 1; a < Q; ++a) A = fma2(X.n[a], pr[a], A);
        return A;
    }
}

__device__ __forceinline__ float lo2(f2 x)
{
    float a, b;
    upk2(x, a, b);
    return a;
}

// The third-layer row of a degree-class-3 entry (plain FP32): its A and B.
template <int STORAGE>
__device__ __forceinline__ void x_row3(const float (&r3)[4], const XPk<3, power_rows(3, STORAGE)>& X, float& A3,
                                       float& B3)
{
    if constexpr (power_rows(3, STORAGE)) {
        const float t = lo2(X.t);
        const float a = fmaf(r3[2], t, r3[1]);
        B3 = fmaf(r3[2], t, a);
        A3 = fmaf(a, t, r3[0]);
    } else {
        A3 = lo2(X.n[0]) * r3[0];
        B3 = lo2(X.d[0]) * r3[0];
#pragma unroll
        for (int a = 1; a < 3; ++a) {
            A3 = fmaf(lo2(X.n[a]), r3[a], A3);
            B3 = fmaf(lo2(X.d[a]), r3[a], B3);
        }
    }
}

template <int STORAGE>
__device__ __forceinline__ float x_row3_value(const float (&r3)[4], const XPk<3, power_rows(3, STORAGE)>& X)
{
    if constexpr (power_rows(3, STORAGE)) {
        const float t = lo2(X.t);
        return fmaf(fmaf(r3[2], t, r3[1]), t, r3[0]);
    } else {
        float A3 = lo2(X.n[0]) * r3[0];
#pragma unroll
        for (int a = 1; a < 3; ++a) A3 = fmaf(lo2(X.n[a]), r3[a], A3);
        return A3;
    }
}

// {X_a, X_a} for every a
template <int Q>
__device__ __forceinline__ void pack_dup(const float (&X)[Q], f2 (&X2)[Q])
{
#pragma unroll
    for (int a = 0; a < Q; ++a) X2[a] = pk2(X[a], X[a]);
}

// {X_2m, X_2m+1} (zero past Q)
template <int Q>
__device__ __forceinline__ void pack_pairs(const float (&X)[Q], f2 (&X2)[qpair(Q) / 2])
{
#pragma unroll
    for (int m = 0; m < qpair(Q) / 2; ++m) X2[m] = pk2(X[2 * m], 2 * m + 1 < Q ? X[2 * m + 1] : 0.0f);
}

// x-pass input from basis values and derivatives (control-point rows) or the local
// coordinate t (power rows).
template <int Q>
__device__ __forceinline__ XInT<Q, false> xin_basis(const float (&N)[Q], const float (&D)[Q])
{
    XInT<Q, false> X;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        X.n[a] = N[a];
        X.d[a] = D[a];
    }
    return X;
}
template <int Q>
__device__ __forceinline__ XInT<Q, true> xin_t(float t)
{
    XInT<Q, true> X;
    X.t = t;
    return X;
}

// The packed form of an x-pass input.
template <int Q, bool POW>
__device__ __forceinline__ XPk<Q, POW> pack_x(const XInT<Q, POW>& X)
{
    XPk<Q, POW> P;
    if constexpr (POW) {
        P.t = pk2(X.t, X.t);
    } else {
        pack_dup<Q>(X.n, P.n);
        pack_dup<Q>(X.d, P.d);
    }
    return P;
}

// x-pass input on a span whose record is in registers, at parameter u: the record's local
// coordinate t = (u - U_s)/h, or the basis by Horner on the record.
template <int Q, int STORAGE>
__device__ __forceinline__ XIn<Q, STORAGE> xin_record(const float (&rec)[rec_stride(Q)], float u)
{
    if constexpr (power_rows(Q, STORAGE)) {
        return xin_t<Q>((u - rec[0]) * rec[1]);
    } else {
        float N[Q], D[Q];
        record_basis<Q>(rec, u, N, D);
        return xin_basis<Q>(N, D);
    }
}

// ----------------------------------------------------------------------------------------
// contraction
// ----------------------------------------------------------------------------------------

// Degree class 3: the support's three z-layers are the pair (k0, k0+1) of each entry, run
// packed as in contract_pairs, and the entry's third-layer row k0+2, run as plain FP32
// FMAs beside it (the same x, y and z sums; no lane multiplies a padding layer).  Weights
// arrive packed as for contract_pairs: nz[0] = {Nz_0, Nz_1}, nz[1] = {Nz_2, 0}.
template <int STORAGE, class Rows>
__device__ __forceinline__ float4 contract_triple_rows(Rows&& rows, const XIn<3, STORAGE>& Xin, const f2 (&ny)[3],
                                                       const f2 (&dy)[3], const f2 (&nz)[2], const f2 (&dz)[2])
{
    const auto X = pack_x(Xin);
    f2 CC, DD, EE;
    float C3, D3, E3;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        f2 pr[4];
        float r3[4];
        rows(b, pr, r3);
        f2 A, B;
        float A3, B3;
        x_row<3, STORAGE>(pr, X, A, B);
        x_row3<STORAGE>(r3, X, A3, B3);
        const float nyb = lo2(ny[b]), dyb = lo2(dy[b]);
        if (b == 0) {
            CC = mul2(ny[0], A);
            DD = mul2(dy[0], A);
            EE = mul2(ny[0], B);
            C3 = nyb * A3;
            D3 = dyb * A3;
            E3 = nyb * B3;
        } else {
            CC = fma2(ny[b], A, CC);
            DD = fma2(dy[b], A, DD);
            EE = fma2(ny[b], B, EE);
            C3 = fmaf(nyb, A3, C3);
            D3 = fmaf(dyb, A3, D3);
            E3 = fmaf(nyb, B3, E3);
        }
    }
    const float nz2 = lo2(nz[1]), dz2 = lo2(dz[1]);
    return make_float4(fmaf(nz2, C3, hsum2(mul2(nz[0], CC))), fmaf(nz2, E3, hsum2(mul2(nz[0], EE))),
                       fmaf(nz2, D3, hsum2(mul2(nz[0], DD))), fmaf(dz2, C3, hsum2(mul2(dz[0], CC))));
}

// Window row b of a degree-class-3 support whose first row is entry `base`: the layer pair
// (k0, k0+1) and the third layer's row.
template <int STORAGE>
__device__ __forceinline__ void window_row3(const ModelDev& M, int base, int b, f2 (&pr)[4], float (&r3)[4])
{
    int idx = base + b * M.nxp;
    MFA_DBG_INDEX(M.dbg, idx, static_cast<long long>(M.nxp) * M.nyp * M.nzp, kDbgWindow);
    PairLoader<3, STORAGE>::load_triple(M, idx, pr, r3);
}

template <int STORAGE>
__device__ __forceinline__ float4 contract_triple(const ModelDev& M, int base, const XIn<3, STORAGE>& Xin,
                                                  const f2 (&ny)[3], const f2 (&dy)[3], const f2 (&nz)[2],
                                                  const f2 (&dz)[2])
{
    return contract_triple_rows<STORAGE>(
        [&](int b, f2 (&pr)[4], float (&r3)[4]) { window_row3<STORAGE>(M, base, b, pr, r3); }, Xin, ny, dy, nz, dz);
}

// Sum-factorised contraction over the Q^3 support whose first row is window entry `base`
// (= (k0 nyp + j0) nxp + i0 for the support origin (i0, j0, k0)):
//   x-pass  A_jk = sum_i Nx_i P_ijk,  B_jk = sum_i Dx_i P_ijk   (x_row: a Horner sweep of the
//           power row, or 2 Q^3 FMA against the x basis)
//   y-pass  C_k = sum_j Ny_j A_jk, D_k = sum_j Dy_j A_jk, E_k = sum_j Ny_j B_jk   (3 Q^2)
//   z-pass  f = sum_k Nz_k C_k, f_z = sum Dz_k C_k, f_y = sum Nz_k D_k, f_x = sum Nz_k E_k
// Returns {f, df/dtx, df/dty, df/dtz} (derivatives in the local span coordinates).
//
// All three passes run on packed FP32x2 values over pairs of z-layers (k, k+1): one
// window entry gives {A_jk, A_j,k+1} (and B likewise), the y-pass turns them into
// {C_k, C_k+1}, {D_k, D_k+1}, {E_k, E_k+1} with weights {Ny_j, Ny_j}, and the z-pass
// accumulates those against {Nz_k, Nz_k+1}; the two halves of each of the four results are
// added once at the end.  ny, dy hold each basis value twice, nz, dz the values of
// functions (2m, 2m+1) (zero past Q).  Each lane is an ordinary FP32 FMA; the z sums add
// their even and odd terms separately before the final addition.
// The layer-pair contraction (Q != 3) over rows supplied by rows(m, b, pr): pr = the
// column pairs of support row b in z-layer pair m.
template <int Q, int STORAGE, class Rows>
__device__ __forceinline__ float4 contract_rows(Rows&& rows, const XIn<Q, STORAGE>& Xin, const f2 (&ny)[Q],
                                                const f2 (&dy)[Q], const f2 (&nz)[qpair(Q) / 2],
                                                const f2 (&dz)[qpair(Q) / 2])
{
    const auto X = pack_x(Xin);
    constexpr int NP = qpair(Q) / 2;
    f2 F, FX, FY, FZ;
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        f2 CC, DD, EE;
#pragma unroll
        for (int b = 0; b < Q; ++b) {
            f2 pr[qpair(Q)];
            rows(m, b, pr);
            f2 A, B;
            x_row<Q, STORAGE>(pr, X, A, B);
            if (b == 0) {
                CC = mul2(ny[0], A);
                DD = mul2(dy[0], A);
                EE = mul2(ny[0], B);
            } else {
                CC = fma2(ny[b], A, CC);
                DD = fma2(dy[b], A, DD);
                EE = fma2(ny[b], B, EE);
            }
        }
        if (m == 0) {
            F = mul2(nz[0], CC);
            FZ = mul2(dz[0], CC);
            FY = mul2(nz[0], DD);
            FX = mul2(nz[0], EE);
        } else {
            F = fma2(nz[m], CC, F);
            FZ = fma2(dz[m], CC, FZ);
            FY = fma2(nz[m], DD, FY);
            FX = fma2(nz[m], EE, FX);
        }
    }
    return make_float4(hsum2(F), hsum2(FX), hsum2(FY), hsum2(FZ));
}

// Window row b of z-layer pair m of the support whose first row is entry `base`.
template <int Q, int STORAGE>
__device__ __forceinline__ void window_row(const ModelDev& M, int base, int m, int b, f2 (&pr)[qpair(Q)])
{
    int idx = base + m * 2 * M.nxp * M.nyp + b * M.nxp;   // Q = 5 also reads entry idx + 1
    MFA_DBG_INDEX(M.dbg, idx, static_cast<long long>(M.nxp) * M.nyp * M.nzp - (qpair(Q) == 6), kDbgWindow);
    PairLoader<Q, STORAGE>::load(M, idx, pr);
}

template <int Q, int STORAGE>
__device__ __forceinline__ float4 contract_pairs(const ModelDev& M, int base, const XIn<Q, STORAGE>& Xin,
                                                 const f2 (&ny)[Q], const f2 (&dy)[Q], const f2 (&nz)[qpair(Q) / 2],
                                                 const f2 (&dz)[qpair(Q) / 2])
{
    if constexpr (Q == 3) {
        return contract_triple<STORAGE>(M, base, Xin, ny, dy, nz, dz);
    } else {
        return contract_rows<Q, STORAGE>(
            [&](int m, int b, f2 (&pr)[qpair(Q)]) { window_row<Q, STORAGE>(M, base, m, b, pr); }, Xin, ny, dy, nz,
            dz);
    }
}

// The support of one query held in registers: the rows contract_pairs would load (for
// degree class 3 the layer pair and the third layer's row of each entry), kept while a
// ray's samples stay in one knot-span cell.
template <int Q>
struct SupportRegs {
    f2 r[qpair(Q) / 2][Q][qpair(Q)];
};
template <>
struct SupportRegs<3> {
    f2 r[3][4];
    float r3[3][4];
};

template <int Q, int STORAGE>
__device__ __forceinline__ void load_support(const ModelDev& M, int base, SupportRegs<Q>& S)
{
    if constexpr (Q == 3) {
#pragma unroll
        for (int b = 0; b < 3; ++b) window_row3<STORAGE>(M, base, b, S.r[b], S.r3[b]);
    } else {
#pragma unroll
        for (int m = 0; m < qpair(Q) / 2; ++m)
#pragma unroll
            for (int b = 0; b < Q; ++b) window_row<Q, STORAGE>(M, base, m, b, S.r[m][b]);
    }
}

// contract_at on a support held in registers: the same sums in the same order.
template <int Q, int STORAGE>
__device__ __forceinline__ float4 contract_support(const SupportRegs<Q>& S, const XIn<Q, STORAGE>& X,
                                                   const float (&Ny)[Q], const float (&Dy)[Q], const float (&Nz)[Q],
                                                   const float (&Dz)[Q])
{
    f2 ny[Q], dy[Q], nz[qpair(Q) / 2], dz[qpair(Q) / 2];
    pack_dup<Q>(Ny, ny);
    pack_dup<Q>(Dy, dy);
    pack_pairs<Q>(Nz, nz);
    pack_pairs<Q>(Dz, dz);
    if constexpr (Q == 3) {
        return contract_triple_rows<STORAGE>(
            [&](int b, f2 (&pr)[4], float (&r3)[4]) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    pr[c] = S.r[b][c];
                    r3[c] = S.r3[b][c];
                }
            },
            X, ny, dy, nz, dz);
    } else {
        return contract_rows<Q, STORAGE>(
            [&](int m, int b, f2 (&pr)[qpair(Q)]) {
#pragma unroll
                for (int c = 0; c < qpair(Q); ++c) pr[c] = S.r[m][b][c];
            },
            X, ny, dy, nz, dz);
    }
}

// Value only: the x-, y- and z-sums of contract_pairs (contract_triple for Q = 3) without
// the derivative sums, in the same order, so f is bit-identical to the value contract_pairs
// returns; rows as for contract_rows / contract_triple_rows.
template <int Q, int STORAGE, class Rows>
__device__ __forceinline__ float contract_value_rows(Rows&& rows, const XIn<Q, STORAGE>& Xin, const f2 (&ny)[Q],
                                                     const f2 (&nz)[qpair(Q) / 2])
{
    const auto X = pack_x(Xin);
    if constexpr (Q == 3) {
        f2 CC;
        float C3;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            f2 pr[4];
            float r3[4];
            rows(b, pr, r3);
            const f2 A = x_row_value<3, STORAGE>(pr, X);
            const float A3 = x_row3_value<STORAGE>(r3, X);
            const float nyb = lo2(ny[b]);
            CC = b == 0 ? mul2(ny[0], A) : fma2(ny[b], A, CC);
            C3 = b == 0 ? nyb * A3 : fmaf(nyb, A3, C3);
        }
        return fmaf(lo2(nz[1]), C3, hsum2(mul2(nz[0], CC)));
    } else {
        constexpr int NP = qpair(Q) / 2;
        f2 F;
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            f2 CC;
#pragma unroll
            for (int b = 0; b < Q; ++b) {
                f2 pr[qpair(Q)];
                rows(m, b, pr);
                const f2 A = x_row_value<Q, STORAGE>(pr, X);
                CC = b == 0 ? mul2(ny[0], A) : fma2(ny[b], A, CC);
            }
            F = m == 0 ? mul2(nz[0], CC) : fma2(nz[m], CC, F);
        }
        return hsum2(F);
    }
}

template <int Q, int STORAGE>
__device__ __forceinline__ float contract_value(const ModelDev& M, int base, const XIn<Q, STORAGE>& Xin,
                                                const f2 (&ny)[Q], const f2 (&nz)[qpair(Q) / 2])
{
    if constexpr (Q == 3)
        return contract_value_rows<3, STORAGE>(
            [&](int b, f2 (&pr)[4], float (&r3)[4]) { window_row3<STORAGE>(M, base, b, pr, r3); }, Xin, ny, nz);
    else
        return contract_value_rows<Q, STORAGE>(
            [&](int m, int b, f2 (&pr)[qpair(Q)]) { window_row<Q, STORAGE>(M, base, m, b, pr); }, Xin, ny, nz);
}

// Contraction from the x-pass input and scalar y / z basis values.
template <int Q, int STORAGE>
__device__ __forceinline__ float4 contract_at(const ModelDev& M, int base, const XIn<Q, STORAGE>& X,
                                              const float (&Ny)[Q], const float (&Dy)[Q], const float (&Nz)[Q],
                                              const float (&Dz)[Q])
{
    f2 ny[Q], dy[Q], nz[qpair(Q) / 2], dz[qpair(Q) / 2];
    pack_dup<Q>(Ny, ny);
    pack_dup<Q>(Dy, dy);
    pack_pairs<Q>(Nz, nz);
    pack_pairs<Q>(Dz, dz);
    return contract_pairs<Q, STORAGE>(M, base, X, ny, dy, nz, dz);
}

// Value only, from the x-pass input and scalar y / z basis values.
template <int Q, int STORAGE>
__device__ __forceinline__ float value_at(const ModelDev& M, int base, const XIn<Q, STORAGE>& X, const float (&Ny)[Q],
                                          const float (&Nz)[Q])
{
    f2 ny[Q], nz[qpair(Q) / 2];
    pack_dup<Q>(Ny, ny);
    pack_pairs<Q>(Nz, nz);
    return contract_value<Q, STORAGE>(M, base, X, ny, nz);
}

// Same, from the support's origin (i0, j0, k0) in the window array.
template <int Q, int STORAGE>
__device__ __forceinline__ float4 contract(const ModelDev& M, int i0, int j0, int k0, const XIn<Q, STORAGE>& X,
                                           const float (&Ny)[Q], const float (&Dy)[Q], const float (&Nz)[Q],
                                           const float (&Dz)[Q])
{
    return contract_at<Q, STORAGE>(M, (k0 * M.nyp + j0) * M.nxp + i0, X, Ny, Dy, Nz, Dz);
}

// Full query at a clamped parameter point: value and world gradient (unit-cube domain,
// so the chain-rule factor to world coordinates is 1; 1/h converts d/dt to d/du).
template <int Q, int STORAGE>
__device__ __forceinline__ float4 query(const ModelDev& M, float u, float v, float w, int sx, int sy, int sz)
{
    float rx[rec_stride(Q)], Ny[Q], Dy[Q], Nz[Q], Dz[Q], hy, hz;
    load_record<Q>(M.ax[0], sx, rx);
    span_basis<Q>(M.ax[1], sy, v, Ny, Dy, hy);
    span_basis<Q>(M.ax[2], sz, w, Nz, Dz, hz);
    float4 r = contract<Q, STORAGE>(M, sx - M.ax[0].p, sy - M.ax[1].p, sz - M.ax[2].p, xin_record<Q, STORAGE>(rx, u),
                                    Ny, Dy, Nz, Dz);
    r.y *= rx[1];
    r.z *= hy;
    r.w *= hz;
    return r;
}

// Query from three records already in registers, the z basis evaluated directly as
// function pairs (record_basis2) for the packed z-pass.
template <int Q, int STORAGE>
__device__ __forceinline__ float4 query2_rec(const ModelDev& M, const float (&rx)[rec_stride(Q)],
                                             const float (&ry)[rec_stride(Q)], const float (&rz)[rec_stride(Q)],
                                             float u, float v, float w, int i0, int j0, int k0)
{
    constexpr int NP = qpair(Q) / 2;
    float Ny[Q], Dy[Q];
    f2 ny[Q], dy[Q], nz[NP], dz[NP];
    const XIn<Q, STORAGE> X = xin_record<Q, STORAGE>(rx, u);
    record_basis<Q>(ry, v, Ny, Dy);
    record_basis2<Q>(rz, w, nz, dz);
    pack_dup<Q>(Ny, ny);
    pack_dup<Q>(Dy, dy);
    float4 r = contract_pairs<Q, STORAGE>(M, (k0 * M.nyp + j0) * M.nxp + i0, X, ny, dy, nz, dz);
    r.y *= rx[1];
    r.z *= ry[1];
    r.w *= rz[1];
    return r;
}

// Same, loading the three records.
template <int Q, int STORAGE>
__device__ __forceinline__ float4 query2(const ModelDev& M, float u, float v, float w, int sx, int sy, int sz)
{
    float rx[rec_stride(Q)], ry[rec_stride(Q)], rz[rec_stride(Q)];
    load_record<Q>(M.ax[0], sx, rx);
    load_record<Q>(M.ax[1], sy, ry);
    load_record<Q>(M.ax[2], sz, rz);
    return query2_rec<Q, STORAGE>(M, rx, ry, rz, u, v, w, sx - M.ax[0].p, sy - M.ax[1].p, sz - M.ax[2].p);
}

// ----------------------------------------------------------------------------------------
// queries on the cardinal path (ModelDev::cardinal: uniform knots, degree Q-1 on every axis)
// ----------------------------------------------------------------------------------------
//
// Coordinates are taken in span units x = (n - p) u.  A query at a given parameter u takes
// the exact span of u (cardinal_span: floor(x) checked against the knots); a ray march,
// whose samples are positioned in span units directly, takes floor(x), the span of its
// position x / (n - p).  Either way the span index j is clamped to 0..n-p-1 and the local
// coordinate is t = x - j (exact in FP32, in [0, 1]).  Spans at least p-1 from both ends use
// cardinal_basis; the p-1 end spans on each side, whose functions see the repeated end
// knots, evaluate their record at the same t (uniform spacing makes the record's local
// coordinate equal to x - j) and rescale to M, G.
struct CardAxis {
    float jf;    // span index as a float: t = x - jf
    int j;       // span index, 0..n-p-1
    bool edge;   // one of the p-1 end spans: evaluate from its record
};

__device__ __forceinline__ void card_set(const AxisDev& A, CardAxis& C, int j)
{
    C.j = j;
    C.jf = static_cast<float>(j);
    C.edge = j < A.p - 1 || j > A.n - 2 * A.p;
}

// Ray marches (span-unit positions x, no parameter u): the span is floor(x), clamped so
// that positions just outside the box take the end spans.
__device__ __forceinline__ void card_update(const AxisDev& A, CardAxis& C, float x)
{
    card_set(A, C, min(max(__float2int_rd(x), 0), A.n - A.p - 1));
}

// Span-unit coordinate of a clamped FP32 parameter u (one FP32 multiply).
__device__ __forceinline__ float cardinal_coord(const AxisDev& A, float u)
{
    return u * static_cast<float>(A.n - A.p);
}

// Knot span of a clamped FP32 parameter u on the cardinal path, as j = s - p: the largest
// s with U_s <= u, exactly as locate_span finds it.  x = cardinal_coord(u) is the product
// (n - p) u correctly rounded to FP32, and rounding is monotone with every integer below
// 2^24 representable, so x > j implies (n - p) u > j and x < j + 1 implies (n - p) u <
// j + 1: floor(x) is the span of the exact product, except when the rounding carried x
// onto the integer j itself from below (u within half an ulp of a knot, e.g. u =
// fl32(0.04) just below the knot 5/125 with x = 5.0).  Only then is u compared with the
// knot, exactly (kup holds the knots rounded up to FP32: u >= kup[s] iff u >= U_s), and
// j moves down one span when u lies below it; the local coordinate x - j is then 1.
// (The exact product's span is the span against the FP64 knots, which on this path are
// exactly i/(n-p) rounded to FP64: no FP32 value lies strictly between i/(n-p) and its
// FP64 rounding.)
__device__ __forceinline__ int cardinal_span(const AxisDev& A, float u, float x)
{
    int j = min(max(__float2int_rd(x), 0), A.n - A.p - 1);
    if (x == static_cast<float>(j) && j > 0 && u < __ldg(A.kup + A.p + j)) --j;
    return j;
}

// Scaled basis (M = p! N, G = (p-1)! dN/dt) on the axis's current span.
template <int Q>
__device__ __forceinline__ void card_basis(const AxisDev& A, const CardAxis& C, float t, float (&N)[Q], float (&D)[Q])
{
    if (C.edge) {
        float rec[rec_stride(Q)];
        load_record<Q>(A, C.j + A.p, rec);
        record_basis_t<Q>(rec, t, N, D);   // uniform spacing: the record's t is x - j too
#pragma unroll
        for (int r = 0; r < Q; ++r) {
            N[r] *= Cardinal<Q>::kBasisScale;
            D[r] *= Cardinal<Q>::kDerivScale;
        }
    } else {
        cardinal_basis<Q>(t, N, D);
    }
}

// x-pass input on the cardinal path at local coordinate t: t itself (power rows, whose
// end spans carry their own polynomials), or the scaled basis of the axis's current span.
template <int Q, int STORAGE>
__device__ __forceinline__ XIn<Q, STORAGE> xin_card(const AxisDev& A, const CardAxis& C, float t)
{
    if constexpr (power_rows(Q, STORAGE)) {
        return xin_t<Q>(t);
    } else {
        float N[Q], D[Q];
        card_basis<Q>(A, C, t, N, D);
        return xin_basis<Q>(N, D);
    }
}

// Same on an interior span (no record).
template <int Q, int STORAGE>
__device__ __forceinline__ XIn<Q, STORAGE> xin_cardinal(float t)
{
    if constexpr (power_rows(Q, STORAGE)) {
        return xin_t<Q>(t);
    } else {
        float N[Q], D[Q];
        cardinal_basis<Q>(t, N, D);
        return xin_basis<Q>(N, D);
    }
}

// Whether any axis needs its end-span record: the x axis only with control-point rows.
template <int Q, int STORAGE>
__device__ __forceinline__ bool card_edge(const CardAxis& cx, const CardAxis& cy, const CardAxis& cz)
{
    return (power_rows(Q, STORAGE) ? false : cx.edge) | cy.edge | cz.edge;
}

// Value and parameter-space gradient at a clamped point on the cardinal path (spans exact,
// as cardinal_span finds them).
template <int Q, int STORAGE>
__device__ __forceinline__ float4 query_cardinal(const ModelDev& M, float u, float v, float w)
{
    const float x = cardinal_coord(M.ax[0], u);
    const float y = cardinal_coord(M.ax[1], v);
    const float z = cardinal_coord(M.ax[2], w);
    CardAxis cx, cy, cz;
    card_set(M.ax[0], cx, cardinal_span(M.ax[0], u, x));
    card_set(M.ax[1], cy, cardinal_span(M.ax[1], v, y));
    card_set(M.ax[2], cz, cardinal_span(M.ax[2], w, z));
    float Ny[Q], Dy[Q], Nz[Q], Dz[Q];
    const XIn<Q, STORAGE> X = xin_card<Q, STORAGE>(M.ax[0], cx, x - cx.jf);
    card_basis<Q>(M.ax[1], cy, y - cy.jf, Ny, Dy);
    card_basis<Q>(M.ax[2], cz, z - cz.jf, Nz, Dz);
    float4 r = contract_at<Q, STORAGE>(M, (cz.j * M.nyp + cy.j) * M.nxp + cx.j, X, Ny, Dy, Nz, Dz);
    r.x *= Cardinal<Q>::template val_scale<STORAGE>();
    r.y *= static_cast<float>(M.ax[0].n - M.ax[0].p) * Cardinal<Q>::template gradx_scale<STORAGE>();
    r.z *= static_cast<float>(M.ax[1].n - M.ax[1].p) * Cardinal<Q>::template gradyz_scale<STORAGE>();
    r.w *= static_cast<float>(M.ax[2].n - M.ax[2].p) * Cardinal<Q>::template gradyz_scale<STORAGE>();
    return r;
}

__device__ __forceinline__ float clamp01(float x) { return fminf(fmaxf(x, 0.0f), 1.0f); }

}  // namespace mfa
