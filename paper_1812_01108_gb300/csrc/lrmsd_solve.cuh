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
constexpr int kRqPasses = 4;          // most Rayleigh-quotient passes of the eigen-solve
constexpr float kNearDouble = 1e-4f;  // |adjugate column|^2 below which another pass runs
constexpr int kPowerSteps = 24;       // power iterations when the adjugate passes fail (double eigenvalue)
constexpr float kEigenResidual2 = 1e-18f;  // |T q - lambda q|^2 above which they run
constexpr float kSuspectAdj = 5e-2f;       // FP32 adjugate diagonal below which the result is checked

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

// ---------------------------------------------------------------------------
// Double-float ("double-word") arithmetic on the FP32 pipe: a value is the
// unevaluated sum hi + lo of two floats, |lo| <= ulp(hi) / 2, about 48
// significant bits.  The building blocks are the classical error-free
// transformations -- Knuth's TwoSum, the FMA form of Dekker's TwoProduct,
// Dekker's Fast2Sum -- combined into the double-word sum, product and
// quotient analysed by Joldes, Muller and Popescu (ACM TOMS 44 (2017) 1).
// The round-to-nearest intrinsics keep the compiler from contracting or
// reordering them.  FP64 issues at a small fraction of the FP32 rate on this
// GPU, so the eigen-solve refines in this form instead.
// ---------------------------------------------------------------------------
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_zero() { return DF{0.f, 0.f}; }

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

// x / y: FP32 quotient, then one correction with the double-float remainder
__device__ __forceinline__ DF df_div(DF x, DF y) {
    const float q1 = __fdiv_rn(x.hi, y.hi);
    const DF r = df_sub(x, df_mul_f(y, q1));
    const float q2 = __fdiv_rn(r.hi, y.hi);
    return fast_two_sum(q1, q2);
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

__device__ __forceinline__ DF df_shfl_xor(DF x, int m) {
    return DF{__shfl_xor_sync(0xffffffffu, x.hi, m), __shfl_xor_sync(0xffffffffu, x.lo, m)};
}
__device__ __forceinline__ DF df_shfl(DF x, int src) {
    return DF{__shfl_sync(0xffffffffu, x.hi, src), __shfl_sync(0xffffffffu, x.lo, src)};
}

__device__ __forceinline__ DF pick4(int i, DF a, DF b, DF c, DF d) {
    return i == 0 ? a : (i == 1 ? b : (i == 2 ? c : d));
}


// Eigen-solve of one pair by the four lanes of a quad (sub = lane & 3), from
// the summed moments S: lane i forms row i of T q for the Rayleigh quotient,
// cofactor (jb, i) of the adjugate row and row i of U, so the dependent
// double-float chain is about a quarter as long; the FP32 estimate runs in
// all four lanes alike.  Every lane of the warp must call it (quad shuffles); only lanes with
// `store` write the pair's state st: U (9), xc (3), yc (3), 0.
__device__ __forceinline__ void quad_eigen_solve(const float (&S)[kSlot], const float (&x0)[3],
                                                 const float (&y0)[3], int n, int sub, int lane,
                                                 bool store, float* __restrict__ st) {
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
    const float sc = solve ? rsqrtf(fro) : 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) r[k] *= sc;
    float lam = 0.f, qf[4] = {1.f, 0.f, 0.f, 0.f};
    int jb = 0;
    float adj = 1.f;
    if (solve) fp32_eigen_estimate(r, e0 * sc, lam, qf, jb, adj);
    const bool suspect = solve && adj < kSuspectAdj;  // a (nearly) double lambda_max
    // ---- refinement in double-float arithmetic (about 48 significant bits),
    // every lane of the warp together from here on
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
    // Rayleigh-quotient passes: lambda = q.T q / q.q at the current estimate,
    // then q = row jb of adj(T - lambda I) (lane sub forms its entry).  One pass
    // is exact to rounding when the largest eigenvalue is well separated (the
    // adjugate column is then of order one, |R|_F being 1).  When it is (nearly)
    // double -- collinear clouds, where any turn about the line fits as well --
    // the FP32 estimate can lean towards the other eigenvectors, and each further
    // pass squares that error; passes repeat while the column stays small.
    // Every lane runs every pass (full-warp shuffles); a quad keeps the pass
    // results only while it still needs them.
    DF qv[4] = {DF{qf[0], 0.f}, DF{qf[1], 0.f}, DF{qf[2], 0.f}, DF{qf[3], 0.f}};
    int jv = jb;
    bool need = true, ok = false;
    const int base = lane & ~3;
    for (int pass = 0; pass < kRqPasses; ++pass) {
        if (!__any_sync(kFull, need)) break;
        DF w = df_zero();
#pragma unroll
        for (int k = 0; k < 4; ++k) w = df_add(w, df_mul(pick4(sub, T[0][k], T[1][k], T[2][k], T[3][k]), qv[k]));
        DF num = df_mul(w, pick4(sub, qv[0], qv[1], qv[2], qv[3]));
        num = df_add(num, df_shfl_xor(num, 1));
        num = df_add(num, df_shfl_xor(num, 2));
        DF den = df_mul(qv[0], qv[0]);
#pragma unroll
        for (int k = 1; k < 4; ++k) den = df_add(den, df_mul(qv[k], qv[k]));
        const DF lam2 = den.hi > 0.f ? df_div(num, den) : df_zero();
        // cofactor (jv, sub) of A = T - lambda I: rows other than jv, columns other than sub
        DF M[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int ri = k < jv ? k : k + 1;
            DF row[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                row[c] = pick4(ri, T[0][c], T[1][c], T[2][c], T[3][c]);
                if (c == ri) row[c] = df_sub(row[c], lam2);
            }
            M[k][0] = sub == 0 ? row[1] : row[0];
            M[k][1] = sub <= 1 ? row[2] : row[1];
            M[k][2] = sub <= 2 ? row[3] : row[2];
        }
        DF qc = df_sub(df_mul(M[0][0], df_sub(df_mul(M[1][1], M[2][2]), df_mul(M[1][2], M[2][1]))),
                       df_mul(M[0][1], df_sub(df_mul(M[1][0], M[2][2]), df_mul(M[1][2], M[2][0]))));
        qc = df_add(qc, df_mul(M[0][2], df_sub(df_mul(M[1][0], M[2][1]), df_mul(M[1][1], M[2][0]))));
        if ((jv + sub) & 1) qc = df_neg(qc);
        DF nn = df_mul(qc, qc);
        nn = df_add(nn, df_shfl_xor(nn, 1));
        nn = df_add(nn, df_shfl_xor(nn, 2));
        const bool ok_p = solve && nn.hi > 0.f;
        const DF qn = ok_p ? df_mul(qc, df_rsqrt(nn)) : df_zero();
        DF qg[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) qg[k] = df_shfl(qn, base + k);
        if (need) {
            ok = ok_p;
#pragma unroll
            for (int k = 0; k < 4; ++k) qv[k] = qg[k];
            need = ok_p && nn.hi < kNearDouble;
            // next cofactor row: the largest entry of the estimate
            jv = 0;
#pragma unroll
            for (int k = 1; k < 4; ++k)
                if (fabsf(qv[k].hi) > fabsf(pick4(jv, qv[0], qv[1], qv[2], qv[3]).hi)) jv = k;
        }
    }
    // The passes stop once the adjugate column is not small, which presumes
    // that lambda was already close to lambda_max.  When the FP32 estimate's
    // eigenvector is rounding noise -- lambda_max exactly double, as for two
    // atoms or collinear atoms (R of rank one) -- the Rayleigh quotient of
    // that noise is not, and the adjugate column is then a mixture of
    // eigenvectors.  So when the FP32 adjugate was small (the sign of a
    // double root) the result is checked by its eigen-residual |T q -
    // (q.T q) q|; a pair that fails the check takes power iterations of
    // T + 2 I (positive definite: |R|_F = 1 bounds the eigenvalues of T by
    // sqrt(3)), which reach the eigenspace of lambda_max at a ratio of at
    // most (lambda_3 + 2) / (lambda_max + 2) per step; any vector of that
    // space is optimal.
    bool redo = false;
    if (__any_sync(kFull, suspect)) {
        DF w = df_zero();
#pragma unroll
        for (int k = 0; k < 4; ++k) w = df_add(w, df_mul(pick4(sub, T[0][k], T[1][k], T[2][k], T[3][k]), qv[k]));
        const DF qs = pick4(sub, qv[0], qv[1], qv[2], qv[3]);
        DF num = df_mul(w, qs);
        num = df_add(num, df_shfl_xor(num, 1));
        num = df_add(num, df_shfl_xor(num, 2));
        const DF r = df_sub(w, df_mul(num, qs));  // q has unit length
        DF rr = df_mul(r, r);
        rr = df_add(rr, df_shfl_xor(rr, 1));
        rr = df_add(rr, df_shfl_xor(rr, 2));
        redo = suspect && (!ok || rr.hi > kEigenResidual2);
    }
    if (__any_sync(kFull, redo)) {
        DF pq[4] = {qv[0], qv[1], qv[2], qv[3]};
        if (!ok) pq[0] = DF{1.f, 0.f}, pq[1] = pq[2] = pq[3] = DF{0.5f, 0.f};
#pragma unroll 1
        for (int it = 0; it < kPowerSteps; ++it) {
            DF w = df_mul_f(pick4(sub, pq[0], pq[1], pq[2], pq[3]), 2.f);
#pragma unroll
            for (int k = 0; k < 4; ++k) w = df_add(w, df_mul(pick4(sub, T[0][k], T[1][k], T[2][k], T[3][k]), pq[k]));
            DF nn = df_mul(w, w);
            nn = df_add(nn, df_shfl_xor(nn, 1));
            nn = df_add(nn, df_shfl_xor(nn, 2));
            const DF wn = nn.hi > 0.f ? df_mul(w, df_rsqrt(nn)) : df_zero();
#pragma unroll
            for (int k = 0; k < 4; ++k) pq[k] = df_shfl(wn, base + k);
        }
        if (redo && (pq[0].hi != 0.f || pq[1].hi != 0.f || pq[2].hi != 0.f || pq[3].hi != 0.f)) {
#pragma unroll
            for (int k = 0; k < 4; ++k) qv[k] = pq[k];
            ok = true;
        }
    }
    DF q0 = qv[0], q1 = qv[1], q2 = qv[2], q3 = qv[3];
    if (!ok) {
        q0 = DF{1.f, 0.f};
        q1 = q2 = q3 = df_zero();
    }
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
