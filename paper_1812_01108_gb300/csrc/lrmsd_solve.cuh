// LRMSD building blocks of Section 4 shared by the LRMSD kernels and the
// fused chain training steps: the 17 shifted moments, the eigen-solve of T(R)
// by the four lanes of a quad, the per-pair state and the residual.
#pragma once

#include "tpl_common.cuh"

namespace tpl {
namespace {

constexpr int kMom = 17;     // sum dx (3), sum dy (3), sum dx dy^T (9), sum |dx|^2, sum |dy|^2
constexpr int kSlot = 20;    // floats per chunk partial (5 float4)
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int checked_atoms(int n, int Nmax) {
    if (n < 0 || n > Nmax) {
        flag_status(TPL_STATUS_BAD_LENGTH);
        n = n < 0 ? 0 : Nmax;
    }
    return n;
}

__device__ __forceinline__ int pair_atoms(const int32_t* num_atoms, int p, int Nmax) {
    return checked_atoms(num_atoms[p], Nmax);
}



// Four consecutive atoms (12 floats, 16-byte aligned) into xyz[4].
__device__ __forceinline__ void load4(const float* __restrict__ p, float3 (&v)[4]) {
    const float4* q = reinterpret_cast<const float4*>(p);
    float4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
    v[0] = make_float3(a.x, a.y, a.z);
    v[1] = make_float3(a.w, b.x, b.y);
    v[2] = make_float3(b.z, b.w, c.x);
    v[3] = make_float3(c.y, c.z, c.w);
}

// Butterfly sum: every lane ends with the same total.
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Fixed-order sum over the four lanes of a quad, (0 + 1) + (2 + 3) in every lane.
template <typename T>
__device__ __forceinline__ T quad_sum(T v, int sub) {
    const T o1 = __shfl_xor_sync(kFull, v, 1);
    const T lo = (sub & 1) ? o1 + v : v + o1;
    const T o2 = __shfl_xor_sync(kFull, lo, 2);
    return (sub & 2) ? o2 + lo : lo + o2;
}

// ---------------------------------------------------------------------------
// Eigen-solve of T(R) (part of K5)
// ---------------------------------------------------------------------------
// Double-float ("double-word") arithmetic on the FP32 pipe: a value is the
// unevaluated sum hi + lo of two floats, |lo| <= ulp(hi) / 2, about 48
// significant bits.  The building blocks are the classical error-free
// transformations -- Knuth's TwoSum, the FMA form of Dekker's TwoProduct,
// Dekker's Fast2Sum -- combined into the double-word sum and product
// analysed by Joldes, Muller and Popescu (ACM TOMS 44 (2017) 1).  The
// round-to-nearest intrinsics keep the compiler from contracting or
// reordering them.  FP64 issues at a small fraction of the FP32 rate on this
// GPU, so the solve uses this form where it needs more than FP32.
// ---------------------------------------------------------------------------
struct DF {
    float hi, lo;
};

// exact a + b (Knuth)
__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return DF{s, e};
}

// exact a + b for |a| >= |b| (Dekker)
__device__ __forceinline__ DF fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}

// exact a * b (FMA)
__device__ __forceinline__ DF two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return DF{p, fmaf(a, b, -p)};
}

__device__ __forceinline__ DF df_add(DF x, DF y) {
    DF s = two_sum(x.hi, y.hi);
    const DF t = two_sum(x.lo, y.lo);
    s = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}

__device__ __forceinline__ DF df_neg(DF x) { return DF{-x.hi, -x.lo}; }
__device__ __forceinline__ DF df_sub(DF x, DF y) { return df_add(x, df_neg(y)); }
__device__ __forceinline__ DF df_twice(DF x) { return DF{__fmul_rn(2.f, x.hi), __fmul_rn(2.f, x.lo)}; }

__device__ __forceinline__ DF df_mul(DF x, DF y) {
    const DF p = two_prod(x.hi, y.hi);
    const float e = fmaf(x.lo, y.lo, fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo)));
    return fast_two_sum(p.hi, e);
}

__device__ __forceinline__ DF df_mul_f(DF x, float y) {
    const DF p = two_prod(x.hi, y);
    return fast_two_sum(p.hi, fmaf(x.lo, y, p.lo));
}

// 1 / sqrt(x) for x > 0: FP32 estimate, one Newton step s (3 - x s^2) / 2 with
// the residual 1 - x s^2 in double-float
__device__ __forceinline__ DF df_rsqrt(DF x) {
    const float s0 = rsqrtf(x.hi);
    const DF e = df_sub(DF{1.f, 0.f}, df_mul_f(df_mul_f(x, s0), s0));
    return fast_two_sum(s0, __fmul_rn(__fmul_rn(0.5f, s0), e.hi));
}

// a + b + c to double-float accuracy
__device__ __forceinline__ DF df_sum3(float a, float b, float c) { return df_add(two_sum(a, b), DF{c, 0.f}); }

__device__ __forceinline__ float df_round(DF x) { return __fadd_rn(x.hi, x.lo); }

// Adjugate of a symmetric 4x4 (float): the same Laplace expansion in FP32,
// used only for the starting eigenvector.
__device__ __forceinline__ float adjugate4f(float a00, float a01, float a02, float a03, float a11,
                                           float a12, float a13, float a22, float a23, float a33,
                                           float (&m)[16]) {
    const float a10 = a01, a20 = a02, a21 = a12, a30 = a03, a31 = a13, a32 = a23;
    const float s0 = a00 * a11 - a10 * a01, s1 = a00 * a12 - a10 * a02, s2 = a00 * a13 - a10 * a03;
    const float s3 = a01 * a12 - a11 * a02, s4 = a01 * a13 - a11 * a03, s5 = a02 * a13 - a12 * a03;
    const float c5 = a22 * a33 - a32 * a23, c4 = a21 * a33 - a31 * a23, c3 = a21 * a32 - a31 * a22;
    const float c2 = a20 * a33 - a30 * a23, c1 = a20 * a32 - a30 * a22, c0 = a20 * a31 - a30 * a21;
    m[0] = a11 * c5 - a12 * c4 + a13 * c3;
    m[4] = -a10 * c5 + a12 * c2 - a13 * c1;
    m[8] = a10 * c4 - a11 * c2 + a13 * c0;
    m[12] = -a10 * c3 + a11 * c1 - a12 * c0;
    m[5] = a00 * c5 - a02 * c2 + a03 * c1;
    m[9] = -a00 * c4 + a01 * c2 - a03 * c0;
    m[13] = a00 * c3 - a01 * c1 + a02 * c0;
    m[10] = a30 * s4 - a31 * s2 + a33 * s0;
    m[14] = -a30 * s3 + a31 * s1 - a32 * s0;
    m[15] = a20 * s3 - a21 * s1 + a22 * s0;
    m[1] = m[4]; m[2] = m[8]; m[3] = m[12]; m[6] = m[9]; m[7] = m[13]; m[11] = m[14];
    return s0 * c5 - s1 * c4 + s2 * c3 + s3 * c2 - s4 * c1 + s5 * c0;
}

// FP32 estimate of the largest eigenpair of T(R) for R scaled to |R|_F = 1
// (T, lambda and the adjugate are O(1); the eigenvectors do not depend on the
// scale): Newton's method on the characteristic polynomial l^4 + c2 l^2 +
// c1 l + c0 (c2 = -2, c1 = -8 det R, c0 = det T) from the upper bound E0/2
// (e0s = E0 |R|^-1), then the column of adj(T - l I) with the largest
// diagonal entry, scaled by it.  jb is that column.
__device__ __forceinline__ void fp32_eigen_estimate(const float (&r)[9], float e0s, float& lam,
                                                    float (&qf)[4], int& jb, float& adj) {
    const float t00 = r[0] + r[4] + r[8], t01 = r[5] - r[7], t02 = r[6] - r[2], t03 = r[1] - r[3];
    const float t11 = r[0] - r[4] - r[8], t12 = r[1] + r[3], t13 = r[2] + r[6];
    const float t22 = -r[0] + r[4] - r[8], t23 = r[5] + r[7], t33 = -r[0] - r[4] + r[8];
    const float detR = r[0] * (r[4] * r[8] - r[5] * r[7]) - r[1] * (r[3] * r[8] - r[5] * r[6]) +
                       r[2] * (r[3] * r[7] - r[4] * r[6]);
    float m[16];
    const float c0 = adjugate4f(t00, t01, t02, t03, t11, t12, t13, t22, t23, t33, m);
    const float c2 = -2.f, c1 = -8.f * detR;
    lam = fminf(2.f, 0.5f * e0s * (1.f + 1e-5f));
    // From above the largest root, Newton's method on a polynomial with real
    // roots only (T is symmetric) decreases monotonically to that root, which
    // is positive (T has trace 0 and is not 0).  Near a double root the FP32
    // polynomial is rounding noise and a step can jump anywhere; a step that
    // would leave (0, lam) ends the iteration instead.
    for (int it = 0; it < 24; ++it) {
        const float l2 = lam * lam;
        const float pv = (l2 + c2) * l2 + c1 * lam + c0;
        const float dp = (4.f * l2 + 2.f * c2) * lam + c1;
        if (!(fabsf(dp) > 0.f)) break;
        const float step = __fdividef(pv, dp);
        const float next = lam - step;
        if (!(next < lam && next > 0.f)) break;
        lam = next;
        if (fabsf(step) <= 1e-6f * fabsf(lam)) break;
    }
    adjugate4f(t00 - lam, t01, t02, t03, t11 - lam, t12, t13, t22 - lam, t23, t33 - lam, m);
    jb = 0;
    float best = m[0];
    qf[0] = m[0]; qf[1] = m[4]; qf[2] = m[8]; qf[3] = m[12];
#pragma unroll
    for (int k = 1; k < 4; ++k)
        if (fabsf(m[5 * k]) > fabsf(best)) {
            best = m[5 * k];
            jb = k;
#pragma unroll
            for (int i = 0; i < 4; ++i) qf[i] = m[4 * i + k];
        }
    adj = fabsf(best);  // of order one for a well separated lambda_max; small near a double one
    if (fabsf(best) > 0.f) {
        const float ib = 1.f / fabsf(best);
#pragma unroll
        for (int i = 0; i < 4; ++i) qf[i] *= ib;
    } else {
        qf[0] = 1.f; qf[1] = qf[2] = qf[3] = 0.f;
        jb = 0;
    }
}

// One rotation of the cyclic Jacobi method on the symmetric 4x4 a (both
// triangles kept), zeroing a[P][Q], with the rotation accumulated into the
// columns of v (Jacobi 1846).  With d = a_qq - a_pp and b = 2 a_pq the
// tangent of the rotation angle is the smaller root of t^2 + 2 (d / b) t - 1
// = 0, t = sgn(d) b / (|d| + sqrt(d^2 + b^2)), which needs no division by the
// small a_pq; cos = 1 / sqrt(1 + t^2), sin = t cos.  The rotation need not
// zero a_pq to the last bit: the eigenvector is refined against the exact T
// afterwards.  An entry below 1e-18 is left alone (T is scaled to O(1), so it
// is rounding noise, and b^2 must not underflow).
template <int P, int Q>
__device__ __forceinline__ void jacobi_rotate(float (&a)[4][4], float (&v)[4][4]) {
    const float apq = a[P][Q];
    if (!(fabsf(apq) > 1e-18f)) return;
    const float d = a[Q][Q] - a[P][P], b = 2.f * apq;
    const float h = fmaf(d, d, b * b);
    const float t = __fdividef(copysignf(1.f, d) * b, fabsf(d) + h * rsqrtf(h));
    const float c = rsqrtf(fmaf(t, t, 1.f)), s = t * c;
    a[P][P] = fmaf(-t, apq, a[P][P]);
    a[Q][Q] = fmaf(t, apq, a[Q][Q]);
    a[P][Q] = a[Q][P] = 0.f;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        if (r == P || r == Q) continue;
        const float g = a[r][P], e = a[r][Q];
        a[r][P] = a[P][r] = c * g - s * e;
        a[r][Q] = a[Q][r] = fmaf(s, g, c * e);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const float g = v[r][P], e = v[r][Q];
        v[r][P] = c * g - s * e;
        v[r][Q] = fmaf(s, g, c * e);
    }
}

constexpr float kSuspectAdj = 5e-2f;  // FP32 adjugate diagonal below which Jacobi takes over
constexpr int kJacobiSweeps = 4;       // most sweeps (six rotations each)
constexpr float kJacobiOff = 1e-7f;    // largest off-diagonal entry that ends the sweeps
constexpr float kRefineRatio = 0.1f;   // largest |correction| along another eigenvector

// y = T q row by row as Dot2 sums (Ogita, Rump and Oishi, SIAM J. Sci.
// Comput. 26 (2005) 1955): T's entries are exact double-floats of the FP32 R,
// each product hi * q split by TwoProduct, the running sum by TwoSum, all
// error terms (and lo * q) carried in a second float.  ys + yc is T q with
// about twice the FP32 precision.
__device__ __forceinline__ void dot2_rows(const DF (&T)[4][4], const float (&q)[4], float (&ys)[4],
                                          float (&yc)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float s = 0.f, c = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const DF p = two_prod(T[i][j].hi, q[j]);
            const DF t = two_sum(s, p.hi);
            s = t.hi;
            c = __fadd_rn(c, __fadd_rn(t.lo, p.lo));
            c = fmaf(T[i][j].lo, q[j], c);
        }
        ys[i] = s;
        yc[i] = c;
    }
}

// Eigen-solve of one pair from the summed moments S by each lane of a quad
// (sub = lane & 3; the four lanes hold the same moments and compute the same
// eigenpair, so no lane waits on another): centre the moments, scale R to
// |R|_F = 1, then
//  1. an FP32 estimate q of the eigenvector of the largest eigenvalue: Newton
//     on the characteristic polynomial and a column of the adjugate of
//     T - lambda I (fp32_eigen_estimate).  Where that column is small (a
//     nearly double lambda_max: collinear or two-fold symmetric clouds, two
//     atoms) the adjugate is rounding noise, and all eigenpairs come from
//     cyclic Jacobi in FP32 instead (two disjoint rotations at a time, at most
//     four sweeps), q the eigenvector of the largest one;
//  2. one refinement of q against the exact T: y = T q by compensated dot
//     products (dot2_rows), mu = q . y, the residual r = y - mu q, and the
//     correction dq with (T - mu I + q q^T) dq = -r, dq orthogonal to q to
//     first order.  On the estimate's path that matrix is well conditioned (its
//     eigenvalues are lambda_i - mu, i > 1, and about 1) and is solved in FP32
//     through its adjugate.  On Jacobi's path dq = sum_i v_i (v_i . r) / (mu -
//     lambda_i) over the other eigenvectors, leaving out a term whose
//     correction would not be small (|v_i . r| >= 0.1 |mu - lambda_i|:
//     lambda_i within rounding of lambda_max, where every vector of the
//     eigenspace is optimal).  The error of q goes from the FP32 solve's to
//     about its square;
//  3. q + dq normalised in double-float and row sub of U(q) (Section 4)
//     formed in double-float and rounded once.
// Only lanes with `store` write the pair's state st: U (9), xc (3), yc (3), 0
// (lanes 0-2 a row of U each, lane 3 the centroids).
__device__ __forceinline__ void quad_eigen_solve(const float (&S)[kSlot], const float (&x0)[3],
                                                 const float (&y0)[3], int n, int sub, int lane,
                                                 bool store, float* __restrict__ st) {
    (void)lane;
    float xc[3] = {0.f, 0.f, 0.f}, yc[3] = {0.f, 0.f, 0.f}, r[9], e0 = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) r[k] = 0.f;
    if (n > 0) {
        const float inv = 1.f / n;
        float mx[3], my[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            mx[a] = S[a] * inv;
            my[a] = S[3 + a] * inv;
            xc[a] = x0[a] + mx[a];
            yc[a] = y0[a] + my[a];
        }
        // centred correlation R_ab = sum x'_a y'_b and E0 = sum |x'|^2 + |y'|^2
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int c = 0; c < 3; ++c) r[3 * a + c] = S[6 + 3 * a + c] - n * mx[a] * my[c];
        e0 = S[15] + S[16] - n * (mx[0] * mx[0] + mx[1] * mx[1] + mx[2] * mx[2] +
                                  my[0] * my[0] + my[1] * my[1] + my[2] * my[2]);
    }
    float fro = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) fro = fmaf(r[k], r[k], fro);
    const bool solve = n > 0 && fro > 0.f;  // else U = I (one atom, or all atoms coincide)
    DF qd[4] = {DF{1.f, 0.f}, DF{0.f, 0.f}, DF{0.f, 0.f}, DF{0.f, 0.f}};
    if (solve) {
        const float sc = rsqrtf(fro);
#pragma unroll
        for (int k = 0; k < 9; ++k) r[k] *= sc;
        // T(R) as exact double-floats of the FP32 entries
        DF T[4][4];
        T[0][0] = df_sum3(r[0], r[4], r[8]);
        T[0][1] = T[1][0] = two_sum(r[5], -r[7]);
        T[0][2] = T[2][0] = two_sum(r[6], -r[2]);
        T[0][3] = T[3][0] = two_sum(r[1], -r[3]);
        T[1][1] = df_sum3(r[0], -r[4], -r[8]);
        T[1][2] = T[2][1] = two_sum(r[1], r[3]);
        T[1][3] = T[3][1] = two_sum(r[2], r[6]);
        T[2][2] = df_sum3(-r[0], r[4], -r[8]);
        T[2][3] = T[3][2] = two_sum(r[5], r[7]);
        T[3][3] = df_sum3(-r[0], -r[4], r[8]);
        float lam, qf[4], adj;
        int jb;
        fp32_eigen_estimate(r, e0 * sc, lam, qf, jb, adj);
        float q[4], dq[4] = {0.f, 0.f, 0.f, 0.f};
        if (adj >= kSuspectAdj) {
            // 1. the adjugate column, normalised
            const float nq = rsqrtf(fmaf(qf[0], qf[0], fmaf(qf[1], qf[1], fmaf(qf[2], qf[2], qf[3] * qf[3]))));
#pragma unroll
            for (int i = 0; i < 4; ++i) q[i] = qf[i] * nq;
            // 2. refinement through (T - mu I + q q^T)
            float ys[4], yr[4];
            dot2_rows(T, q, ys, yr);
            float mu = 0.f;
#pragma unroll
            for (int i = 0; i < 4; ++i) mu = fmaf(q[i], ys[i], mu);
            float res[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) res[i] = fmaf(-mu, q[i], ys[i]) + yr[i];
            float m[16];
            const float det = adjugate4f(
                T[0][0].hi - mu + q[0] * q[0], T[0][1].hi + q[0] * q[1], T[0][2].hi + q[0] * q[2],
                T[0][3].hi + q[0] * q[3], T[1][1].hi - mu + q[1] * q[1], T[1][2].hi + q[1] * q[2],
                T[1][3].hi + q[1] * q[3], T[2][2].hi - mu + q[2] * q[2], T[2][3].hi + q[2] * q[3],
                T[3][3].hi - mu + q[3] * q[3], m);
            // (the adjugate path runs only for a well separated lambda_max, so det
            // is of order one; an exact zero would leave q unrefined)
            const float idet = fabsf(det) > 1e-30f ? -__frcp_rn(det) : 0.f;
#pragma unroll
            for (int i = 0; i < 4; ++i)
                dq[i] = idet * fmaf(m[4 * i], res[0], fmaf(m[4 * i + 1], res[1], fmaf(m[4 * i + 2], res[2], m[4 * i + 3] * res[3])));
        } else {
            // 1. cyclic Jacobi
            float a[4][4], v[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    a[i][j] = T[i][j].hi;
                    v[i][j] = i == j ? 1.f : 0.f;
                }
#pragma unroll 1
            for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
                jacobi_rotate<0, 1>(a, v);
                jacobi_rotate<2, 3>(a, v);
                jacobi_rotate<0, 2>(a, v);
                jacobi_rotate<1, 3>(a, v);
                jacobi_rotate<0, 3>(a, v);
                jacobi_rotate<1, 2>(a, v);
                const float off = fmaxf(fmaxf(fmaxf(fabsf(a[0][1]), fabsf(a[0][2])), fmaxf(fabsf(a[0][3]), fabsf(a[1][2]))),
                                        fmaxf(fabsf(a[1][3]), fabsf(a[2][3])));
                if (off < kJacobiOff) break;
            }
            int kb = 0;
            float best = a[0][0];
#pragma unroll
            for (int i = 1; i < 4; ++i)
                if (a[i][i] > best) {
                    best = a[i][i];
                    kb = i;
                }
#pragma unroll
            for (int i = 0; i < 4; ++i) q[i] = kb == 0 ? v[i][0] : (kb == 1 ? v[i][1] : (kb == 2 ? v[i][2] : v[i][3]));
            // 2. refinement along the other eigenvectors
            float ys[4], yr[4];
            dot2_rows(T, q, ys, yr);
            float mu = 0.f;
#pragma unroll
            for (int i = 0; i < 4; ++i) mu = fmaf(q[i], ys[i], mu);
            float res[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) res[i] = fmaf(-mu, q[i], ys[i]) + yr[i];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (e == kb) continue;
                float w = 0.f;
#pragma unroll
                for (int i = 0; i < 4; ++i) w = fmaf(v[i][e], res[i], w);
                const float den = mu - a[e][e];
                if (fabsf(w) < kRefineRatio * fabsf(den)) {
                    const float coef = __fdividef(w, den);
#pragma unroll
                    for (int i = 0; i < 4; ++i) dq[i] = fmaf(coef, v[i][e], dq[i]);
                }
            }
        }
        // 3. q + dq as double-floats, normalised
        DF nn = DF{0.f, 0.f};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            qd[i] = two_sum(q[i], dq[i]);
            nn = df_add(nn, df_mul(qd[i], qd[i]));
        }
        const DF is = df_rsqrt(nn);
#pragma unroll
        for (int i = 0; i < 4; ++i) qd[i] = df_mul(qd[i], is);
    }
    const DF q0 = qd[0], q1 = qd[1], q2 = qd[2], q3 = qd[3];
    // row sub of U(q) (Section 4), formed in double-float and rounded once
    const DF a = df_mul(q0, q0), bq = df_mul(q1, q1), c = df_mul(q2, q2), d = df_mul(q3, q3);
    DF u0, u1, u2;
    if (sub == 0) {
        u0 = df_sub(df_add(a, bq), df_add(c, d));
        u1 = df_twice(df_sub(df_mul(q1, q2), df_mul(q0, q3)));
        u2 = df_twice(df_add(df_mul(q1, q3), df_mul(q0, q2)));
    } else if (sub == 1) {
        u0 = df_twice(df_add(df_mul(q1, q2), df_mul(q0, q3)));
        u1 = df_sub(df_add(a, c), df_add(bq, d));
        u2 = df_twice(df_sub(df_mul(q2, q3), df_mul(q0, q1)));
    } else {
        u0 = df_twice(df_sub(df_mul(q1, q3), df_mul(q0, q2)));
        u1 = df_twice(df_add(df_mul(q2, q3), df_mul(q0, q1)));
        u2 = df_sub(df_add(a, d), df_add(bq, c));
    }
    if (store) {
        if (sub < 3) {
            st[3 * sub] = df_round(u0);
            st[3 * sub + 1] = df_round(u1);
            st[3 * sub + 2] = df_round(u2);
        } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                st[9 + k] = xc[k];
                st[12 + k] = yc[k];
            }
            st[15] = 0.f;
        }
    }
}

// Quad-lane sum of a pair's nch partials (slot stride kSlot floats): lane
// sub sums partials sub, sub + 4, ... in order, then the fixed-order quad
// sum; L2 loads (the partials are written by other SMs in the same kernel).
__device__ __forceinline__ void quad_sum_partials(const float* __restrict__ part, int nch, int sub,
                                                  float (&S)[kSlot]) {
#pragma unroll
    for (int k = 0; k < kSlot; ++k) S[k] = 0.f;
#pragma unroll 4
    for (int c = sub; c < nch; c += 4) {
        const float4* q = reinterpret_cast<const float4*>(part + (size_t)c * kSlot);
#pragma unroll
        for (int k = 0; k < kSlot / 4; ++k) {
            const float4 v = __ldcg(q + k);
            S[4 * k] += v.x; S[4 * k + 1] += v.y; S[4 * k + 2] += v.z; S[4 * k + 3] += v.w;
        }
    }
#pragma unroll
    for (int k = 0; k < kMom; ++k) S[k] = quad_sum(S[k], sub);
}

__device__ __forceinline__ void first_atoms(const float* __restrict__ x, const float* __restrict__ y, int n,
                                            float (&x0)[3], float (&y0)[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        x0[a] = n > 0 ? x[a] : 0.f;
        y0[a] = n > 0 ? y[a] : 0.f;
    }
}

// U x + loads of the per-pair state
struct PairState {
    float3 u0, u1, u2;  // rows of U
    float3 xc, yc;
    float scale;
};

// The state is written by an earlier kernel: read-only loads, four float4.
__device__ __forceinline__ PairState load_state(const float* st) {
    const float4* q = reinterpret_cast<const float4*>(st);
    const float4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2), d = __ldg(q + 3);
    PairState s;
    s.u0 = make_float3(a.x, a.y, a.z);
    s.u1 = make_float3(a.w, b.x, b.y);
    s.u2 = make_float3(b.z, b.w, c.x);
    s.xc = make_float3(c.y, c.z, c.w);
    s.yc = make_float3(d.x, d.y, d.z);
    s.scale = d.w;
    return s;
}

__device__ __forceinline__ PairState load_state_shared(const float* st) {
    PairState s;
    s.u0 = make_float3(st[0], st[1], st[2]);
    s.u1 = make_float3(st[3], st[4], st[5]);
    s.u2 = make_float3(st[6], st[7], st[8]);
    s.xc = make_float3(st[9], st[10], st[11]);
    s.yc = make_float3(st[12], st[13], st[14]);
    s.scale = 0.f;
    return s;
}

__device__ __forceinline__ float3 residual(const PairState& s, float3 x, float3 y) {
    const float3 xp = f3_sub(x, s.xc), yp = f3_sub(y, s.yc);
    return make_float3(yp.x - f3_dot(s.u0, xp), yp.y - f3_dot(s.u1, xp), yp.z - f3_dot(s.u2, xp));
}

}  // namespace
}  // namespace tpl
