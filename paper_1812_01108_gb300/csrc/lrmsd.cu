// LRMSD of the paper (Section 4) on sm_103a.
//
// Forward, one launch: one CTA per pair (K5 lrmsd_pair_kernel)
//  - moments: the CTA streams both clouds, the moments shifted by the pair's
//    first atom in FP32 -- sum dx, sum dy, sum dx dy^T, sum |dx|^2, sum
//    |dy|^2 (x = target, y = input, as in the paper's R = sum x y^T);
//  - eigen-solve: one quad of warp 0 centres R, estimates the largest
//    eigenpair of the 4x4 matrix T(R) in FP32 (Newton's method on the
//    characteristic polynomial, as in the quaternion-characteristic-polynomial
//    approach of Theobald, Acta Cryst. A61 (2005) 478, then an adjugate
//    column) and refines it in double-float FP32 arithmetic, about 48 bits
//    (Rayleigh quotient of T, adjugate of T - lambda I), then U(q);
//  - residuals: LRMSD^2 = (sum |x'|^2 + |y'|^2 - 2 lambda)/N equals sum |y'_i -
//    U x'_i|^2 / N at the optimum; the residual form has no cancellation, so
//    it is summed in FP32 per thread and in FP64 over the warps.  The clouds
//    were just read by the moments, so this pass reads them from L2;
//  - LRMSD and the gradient scale 1 / (N LRMSD).
// Backward:
//  K6 lrmsd_grad: grad_y_i = w (y'_i - U x'_i) / (N LRMSD).
// Every sum runs in a fixed order, so the results are the same from run to run.
#include <mutex>

#include "kernels.h"
#include "sched.cuh"
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

// Workspace: the per-pair state the backward reads (U row-major, centroid of
// the target, centroid of the input, 1 / (N LRMSD)).
struct WsLayout {
    size_t state, total;
};

__host__ __device__ constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

__host__ __device__ constexpr WsLayout ws_layout(int P, int Nmax) {
    (void)Nmax;
    WsLayout w{};
    w.state = 0;
    w.total = align256((size_t)(P > 0 ? P : 1) * 16 * sizeof(float));
    return w;
}

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

// Eigen-solve of the fused training step: the partials are per tile of `tile`
// residues of chain p (the full-atom forward's tile moments), eight pairs per
// warp.
__global__ void __launch_bounds__(32) lrmsd_solve_tiles_kernel(
    const float* __restrict__ input, const float* __restrict__ target,
    const int32_t* __restrict__ num_atoms, int P, int Nmax, const float* __restrict__ part1,
    int tiles_max, float* __restrict__ state, const int32_t* __restrict__ lengths, int tile, int Lmax) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int sub = gid & 3, lane = threadIdx.x & 31;
    const bool active = (gid >> 2) < P;
    const int p = active ? (gid >> 2) : P - 1;
    const int n = pair_atoms(num_atoms, p, Nmax);
    const int L = min(max(lengths[p], 0), Lmax);
    const int nch = fa_num_tiles(L, tile);
    float x0[3], y0[3];
    first_atoms(target + (size_t)p * Nmax * 3, input + (size_t)p * Nmax * 3, n, x0, y0);
    float S[kSlot];
    quad_sum_partials(part1 + (size_t)p * tiles_max * kSlot, nch, sub, S);
    quad_eigen_solve(S, x0, y0, n, sub, lane, active, state + 16 * (size_t)p);
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

// ---------------------------------------------------------------------------
// K5: the whole forward of a pair in one CTA: moments, eigen-solve by one quad
// of warp 0, residual sum and LRMSD, with block barriers between the steps.
// Two shapes: 256 threads with four groups of four atoms per thread in
// flight (two CTAs per SM) for batches that fit one wave, and a compact one,
// 128 threads with one group (eight CTAs per SM), for larger batches: about
// 1200 pairs are then in flight, their clouds (tens of MB) stay in L2, and
// the residual pass reads them from there instead of from HBM, while other
// CTAs on the SM stream while one CTA's quad solves.
// ---------------------------------------------------------------------------
constexpr int kPNT = 256;
constexpr int kCNT = 128;  // compact shape

template <int NT, int G, int MINB>
__global__ void __launch_bounds__(NT, MINB) lrmsd_pair_kernel(
    const float* __restrict__ input, const float* __restrict__ target,
    const int32_t* __restrict__ num_atoms, int P, int Nmax, float* __restrict__ state,
    float* __restrict__ lrmsd) {
    constexpr int kPNT = NT;
    constexpr int NW = kPNT / 32;
    constexpr int kBatch = 4 * G * kPNT;  // G groups of 4 atoms per thread in flight
    __shared__ float s_mom[NW][kMom + 1];
    __shared__ double s_res[NW];
    __shared__ __align__(16) float s_st[16];
    const int p = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float* x = target + (size_t)p * Nmax * 3;
    const float* y = input + (size_t)p * Nmax * 3;
    // The first batch and the first atoms are read up to Nmax (inside the
    // padded rows) so that their loads do not wait for the atom count.
    float3 sx = make_float3(0.f, 0.f, 0.f), sy = sx;
    if (Nmax > 0) {
        sx = make_float3(__ldg(x), __ldg(x + 1), __ldg(x + 2));
        sy = make_float3(__ldg(y), __ldg(y + 1), __ldg(y + 2));
    }
    const int n = pair_atoms(num_atoms, p, Nmax);
    if (n == 0) sx = sy = make_float3(0.f, 0.f, 0.f);
    float m[kMom];
#pragma unroll
    for (int k = 0; k < kMom; ++k) m[k] = 0.f;
    for (int base = 0; base < (base == 0 ? Nmax : n); base += kBatch) {
        const int bound = base == 0 ? Nmax : n;
        float3 xv[G][4], yv[G][4];
#pragma unroll
        for (int s = 0; s < G; ++s) {
            const int i0 = base + 4 * (threadIdx.x + kPNT * s);
            if (i0 < bound) {
                load4(x + 3 * (size_t)i0, xv[s]);
                load4(y + 3 * (size_t)i0, yv[s]);
            }
        }
#pragma unroll
        for (int s = 0; s < G; ++s) {
            const int i0 = base + 4 * (threadIdx.x + kPNT * s);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (i0 + q < n) {
                    const float3 dx = f3_sub(xv[s][q], sx), dy = f3_sub(yv[s][q], sy);
                    m[0] += dx.x; m[1] += dx.y; m[2] += dx.z;
                    m[3] += dy.x; m[4] += dy.y; m[5] += dy.z;
                    m[6] = fmaf(dx.x, dy.x, m[6]); m[7] = fmaf(dx.x, dy.y, m[7]); m[8] = fmaf(dx.x, dy.z, m[8]);
                    m[9] = fmaf(dx.y, dy.x, m[9]); m[10] = fmaf(dx.y, dy.y, m[10]); m[11] = fmaf(dx.y, dy.z, m[11]);
                    m[12] = fmaf(dx.z, dy.x, m[12]); m[13] = fmaf(dx.z, dy.y, m[13]); m[14] = fmaf(dx.z, dy.z, m[14]);
                    m[15] += f3_dot(dx, dx);
                    m[16] += f3_dot(dy, dy);
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < kMom; ++k) {
        const float v = warp_sum(m[k]);
        if (lane == 0) s_mom[warp][k] = v;
    }
    __syncthreads();
    if (warp == 0) {
        // lane k < kMom sums moment k over the warps (fixed order), then every
        // lane takes all of them
        float v = 0.f;
        if (lane < kMom)
#pragma unroll
            for (int w = 0; w < NW; ++w) v += s_mom[w][lane];
        float S[kSlot];
#pragma unroll
        for (int k = 0; k < kSlot; ++k) S[k] = k < kMom ? __shfl_sync(kFull, v, k) : 0.f;
        const float x0[3] = {sx.x, sx.y, sx.z}, y0[3] = {sy.x, sy.y, sy.z};
        quad_eigen_solve(S, x0, y0, n, lane & 3, lane, lane < 4, s_st);
    }
    __syncthreads();
    const PairState ps = load_state_shared(s_st);
    float acc = 0.f;
    for (int base = 0; base < n; base += kBatch) {
        float3 xv[G][4], yv[G][4];
#pragma unroll
        for (int s = 0; s < G; ++s) {
            const int i0 = base + 4 * (threadIdx.x + kPNT * s);
            if (i0 < n) {
                load4(x + 3 * (size_t)i0, xv[s]);
                load4(y + 3 * (size_t)i0, yv[s]);
            }
        }
#pragma unroll
        for (int s = 0; s < G; ++s) {
            const int i0 = base + 4 * (threadIdx.x + kPNT * s);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (i0 + q < n) {
                    const float3 d = residual(ps, xv[s][q], yv[s][q]);
                    acc += f3_dot(d, d);
                }
        }
    }
    acc = warp_sum(acc);
    if (lane == 0) s_res[warp] = (double)acc;
    __syncthreads();
    if (threadIdx.x < 15) state[16 * (size_t)p + threadIdx.x] = s_st[threadIdx.x];
    if (threadIdx.x == 0) {
        double sum = 0.0;
#pragma unroll
        for (int w = 0; w < NW; ++w) sum += s_res[w];
        float lr, scale;
        lrmsd_from_sum(sum, n, lr, scale);
        state[16 * (size_t)p + 15] = scale;
        lrmsd[p] = lr;
    }
}

// ---------------------------------------------------------------------------
// K6: one CTA per 2048 atoms of a pair (a write stream: large CTAs keep the
// stores of a pair together)
// ---------------------------------------------------------------------------
constexpr int kGNT = 256;
constexpr int kGChunk = kGNT * 8;  // two groups of 4 atoms per thread

__global__ void __launch_bounds__(kGNT) lrmsd_grad_kernel(const float* __restrict__ grad_lrmsd,
                                                          const float* __restrict__ input,
                                                          const float* __restrict__ target,
                                                          const int32_t* __restrict__ num_atoms,
                                                          int P, int Nmax, const float* __restrict__ state,
                                                          float* __restrict__ grad_input, int nch_max) {
    const int p = blockIdx.x / nch_max, c = blockIdx.x % nch_max;
    const int n = pair_atoms(num_atoms, p, Nmax);
    const float* x = target + (size_t)p * Nmax * 3;
    const float* y = input + (size_t)p * Nmax * 3;
    float* gy = grad_input + (size_t)p * Nmax * 3;
    const PairState ps = load_state(state + 16 * (size_t)p);
    const float w = __ldg(grad_lrmsd + p) * ps.scale;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int i0 = c * kGChunk + 4 * (threadIdx.x + kGNT * s);
        if (i0 >= Nmax) continue;
        float g[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) g[k] = 0.f;
        if (i0 < n) {
            float3 xv[4], yv[4];
            load4(x + 3 * (size_t)i0, xv);
            load4(y + 3 * (size_t)i0, yv);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (i0 + q < n) {
                    const float3 r = residual(ps, xv[q], yv[q]);
                    g[3 * q] = w * r.x;
                    g[3 * q + 1] = w * r.y;
                    g[3 * q + 2] = w * r.z;
                }
        }
        float4* o = reinterpret_cast<float4*>(gy + 3 * (size_t)i0);
        o[0] = make_float4(g[0], g[1], g[2], g[3]);
        o[1] = make_float4(g[4], g[5], g[6], g[7]);
        o[2] = make_float4(g[8], g[9], g[10], g[11]);
    }
}

// ---------------------------------------------------------------------------
// K7: plain FP64 per-pair form (one CTA per pair, FP64 block sums, cyclic
// Jacobi on T, LRMSD by the closed form of Section 4).
// ---------------------------------------------------------------------------
constexpr int kRefNT = 128;

template <int V>
__device__ void block_sum64(double (&v)[V], double* s) {
    for (int k = 0; k < V; ++k) s[k * kRefNT + threadIdx.x] = v[k];
    __syncthreads();
    for (int w = kRefNT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < V; ++k) s[k * kRefNT + threadIdx.x] += s[k * kRefNT + threadIdx.x + w];
        __syncthreads();
    }
    for (int k = 0; k < V; ++k) v[k] = s[k * kRefNT];
    __syncthreads();
}

__device__ void jacobi4(double (&A)[4][4], double (&V)[4][4]) {
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) V[i][j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < 4; ++i)
            for (int j = i + 1; j < 4; ++j) off += A[i][j] * A[i][j];
        if (off < 1e-300) break;
        for (int p = 0; p < 3; ++p)
            for (int q = p + 1; q < 4; ++q) {
                if (A[p][q] == 0.0) continue;
                const double th = 0.5 * (A[q][q] - A[p][p]) / A[p][q];
                const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(1.0 + th * th));
                const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                for (int k = 0; k < 4; ++k) {
                    const double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 4; ++k) {
                    const double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 4; ++k) {
                    const double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
    }
}

__global__ void __launch_bounds__(kRefNT) lrmsd_fwd_ref64_kernel(
    const double* __restrict__ input, const double* __restrict__ target,
    const int32_t* __restrict__ num_atoms, int P, int Nmax, double* __restrict__ lrmsd,
    double* __restrict__ state) {
    __shared__ double s[10 * kRefNT];
    __shared__ double s_c[6];
    const int p = blockIdx.x;
    const int n = pair_atoms(num_atoms, p, Nmax);
    const double* x = target + (size_t)p * Nmax * 3;
    const double* y = input + (size_t)p * Nmax * 3;
    double c6[6] = {0, 0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < n; i += kRefNT)
        for (int a = 0; a < 3; ++a) {
            c6[a] += x[3 * i + a];
            c6[3 + a] += y[3 * i + a];
        }
    block_sum64<6>(c6, s);
    if (threadIdx.x == 0)
        for (int k = 0; k < 6; ++k) s_c[k] = n > 0 ? c6[k] / n : 0.0;
    __syncthreads();
    double m[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};  // R (9), E0
    for (int i = threadIdx.x; i < n; i += kRefNT) {
        double xp[3], yp[3];
        for (int a = 0; a < 3; ++a) {
            xp[a] = x[3 * i + a] - s_c[a];
            yp[a] = y[3 * i + a] - s_c[3 + a];
        }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) m[3 * a + b] += xp[a] * yp[b];
        m[9] += xp[0] * xp[0] + xp[1] * xp[1] + xp[2] * xp[2] + yp[0] * yp[0] + yp[1] * yp[1] + yp[2] * yp[2];
    }
    block_sum64<10>(m, s);
    if (threadIdx.x != 0) return;
    double* st = state + 16 * (size_t)p;
    double U[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    double lr = 0.0;
    if (n > 0) {
        const double* R = m;  // R[3a+b]
        double A[4][4] = {
            {R[0] + R[4] + R[8], R[5] - R[7], R[6] - R[2], R[1] - R[3]},
            {R[5] - R[7], R[0] - R[4] - R[8], R[1] + R[3], R[2] + R[6]},
            {R[6] - R[2], R[1] + R[3], -R[0] + R[4] - R[8], R[5] + R[7]},
            {R[1] - R[3], R[2] + R[6], R[5] + R[7], -R[0] - R[4] + R[8]}};
        double V[4][4];
        jacobi4(A, V);
        int best = 0;
        for (int k = 1; k < 4; ++k)
            if (A[k][k] > A[best][best]) best = k;
        const double lam = A[best][best];
        double q[4] = {V[0][best], V[1][best], V[2][best], V[3][best]};
        const double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        for (int k = 0; k < 4; ++k) q[k] /= qn;
        U[0] = q[0] * q[0] + q[1] * q[1] - q[2] * q[2] - q[3] * q[3];
        U[1] = 2 * (q[1] * q[2] - q[0] * q[3]);
        U[2] = 2 * (q[1] * q[3] + q[0] * q[2]);
        U[3] = 2 * (q[1] * q[2] + q[0] * q[3]);
        U[4] = q[0] * q[0] - q[1] * q[1] + q[2] * q[2] - q[3] * q[3];
        U[5] = 2 * (q[2] * q[3] - q[0] * q[1]);
        U[6] = 2 * (q[1] * q[3] - q[0] * q[2]);
        U[7] = 2 * (q[2] * q[3] + q[0] * q[1]);
        U[8] = q[0] * q[0] - q[1] * q[1] - q[2] * q[2] + q[3] * q[3];
        const double rad = (m[9] - 2.0 * lam) / n;
        lr = sqrt(rad > 0.0 ? rad : 0.0);
    }
    for (int k = 0; k < 9; ++k) st[k] = U[k];
    for (int k = 0; k < 6; ++k) st[9 + k] = s_c[k];
    st[15] = lr;
    lrmsd[p] = lr;
}

__global__ void __launch_bounds__(kRefNT) lrmsd_bwd_ref64_kernel(
    const double* __restrict__ grad_lrmsd, const double* __restrict__ input,
    const double* __restrict__ target, const int32_t* __restrict__ num_atoms, int P, int Nmax,
    const double* __restrict__ state, double* __restrict__ grad_input) {
    const int p = blockIdx.x;
    const int n = pair_atoms(num_atoms, p, Nmax);
    const double* st = state + 16 * (size_t)p;
    const double lr = st[15];
    const double w = (n > 0 && lr >= 1e-12) ? grad_lrmsd[p] / (n * lr) : 0.0;
    const double* x = target + (size_t)p * Nmax * 3;
    const double* y = input + (size_t)p * Nmax * 3;
    double* g = grad_input + (size_t)p * Nmax * 3;
    for (int i = threadIdx.x; i < Nmax; i += kRefNT) {
        if (i >= n) {
            g[3 * i] = g[3 * i + 1] = g[3 * i + 2] = 0.0;
            continue;
        }
        const double xp[3] = {x[3 * i] - st[9], x[3 * i + 1] - st[10], x[3 * i + 2] - st[11]};
        for (int a = 0; a < 3; ++a)
            g[3 * i + a] = w * ((y[3 * i + a] - st[12 + a]) -
                                (st[3 * a] * xp[0] + st[3 * a + 1] * xp[1] + st[3 * a + 2] * xp[2]));
    }
}

}  // namespace


size_t lrmsd_ws_bytes(int P, int Nmax) { return ws_layout(P, Nmax).total; }

cudaError_t launch_lrmsd_solve_tiles(const float* input, const float* target, const int32_t* num_atoms,
                                     int P, int Nmax, const float* tile_moments, int tiles_max,
                                     const int32_t* lengths, int tile, int Lmax, float* state,
                                     cudaStream_t s) {
    if (P == 0) return cudaSuccess;
    lrmsd_solve_tiles_kernel<<<(4 * P + 31) / 32, 32, 0, s>>>(input, target, num_atoms, P, Nmax, tile_moments,
                                                             tiles_max, state, lengths, tile, Lmax);
    return cudaGetLastError();
}

const float* lrmsd_state(const void* ws, int P, int Nmax) {
    return reinterpret_cast<const float*>(static_cast<const char*>(ws) + ws_layout(P, Nmax).state);
}

// Shape of the pair kernel: the wide one when the batch fits the GPU in one
// wave of its CTAs, else the compact one.
static bool pair_path(int P) {
    return P <= persistent_grid((const void*)lrmsd_pair_kernel<kPNT, 4, 2>, kPNT, 0);
}

int lrmsd_forward_launches(int P) { return P <= 0 ? 0 : 1; }

cudaError_t launch_lrmsd_forward(const float* input, const float* target, const int32_t* num_atoms,
                                 int P, int Nmax, float* lrmsd, void* ws, cudaStream_t s) {
    if (P == 0) return cudaSuccess;
    float* state = reinterpret_cast<float*>(static_cast<char*>(ws) + ws_layout(P, Nmax).state);
    if (pair_path(P))
        lrmsd_pair_kernel<kPNT, 4, 2><<<P, kPNT, 0, s>>>(input, target, num_atoms, P, Nmax, state, lrmsd);
    else
        lrmsd_pair_kernel<kCNT, 2, 6><<<P, kCNT, 0, s>>>(input, target, num_atoms, P, Nmax, state, lrmsd);
    return cudaGetLastError();
}

cudaError_t launch_lrmsd_backward(const float* grad_lrmsd, const float* input, const float* target,
                                  const int32_t* num_atoms, int P, int Nmax, float* grad_input,
                                  const void* ws, cudaStream_t s) {
    if (P == 0) return cudaSuccess;
    const WsLayout L = ws_layout(P, Nmax);
    const float* state = reinterpret_cast<const float*>(static_cast<const char*>(ws) + L.state);
    const int nch = (Nmax + kGChunk - 1) / kGChunk > 0 ? (Nmax + kGChunk - 1) / kGChunk : 1;
    const unsigned grid = (unsigned)P * (unsigned)nch;  // block = pair * nch + chunk
    lrmsd_grad_kernel<<<grid, kGNT, 0, s>>>(grad_lrmsd, input, target, num_atoms, P, Nmax, state, grad_input,
                                            nch);
    return cudaGetLastError();
}

cudaError_t launch_lrmsd_forward_ref64(const double* input, const double* target,
                                       const int32_t* num_atoms, int P, int Nmax, double* lrmsd,
                                       double* state, cudaStream_t s) {
    if (P == 0) return cudaSuccess;
    lrmsd_fwd_ref64_kernel<<<P, kRefNT, 0, s>>>(input, target, num_atoms, P, Nmax, lrmsd, state);
    return cudaGetLastError();
}

cudaError_t launch_lrmsd_backward_ref64(const double* grad_lrmsd, const double* input,
                                        const double* target, const int32_t* num_atoms, int P,
                                        int Nmax, const double* state, double* grad_input,
                                        cudaStream_t s) {
    if (P == 0) return cudaSuccess;
    lrmsd_bwd_ref64_kernel<<<P, kRefNT, 0, s>>>(grad_lrmsd, input, target, num_atoms, P, Nmax, state,
                                                grad_input);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free LRMSD forward.
//
// Some callers cannot allocate device memory and cannot hand this library a
// workspace either: code running under a framework or runtime whose allocator
// owns all device memory and refuses new allocations once a run is planned, or
// behind an interface that has no argument for scratch memory.  For them the
// forward keeps its scratch in the fixed array below, which lives in the
// library's own device memory: every GPU that loads the library holds
// kNoAllocScratchBytes for it until the process exits.  The caller still owns
// the inputs and the output.
// ---------------------------------------------------------------------------
constexpr int kNoAllocMaxPairs = 4096;
constexpr int kNoAllocMaxAtoms = 8192;
constexpr size_t kNoAllocScratchBytes = ws_layout(kNoAllocMaxPairs, kNoAllocMaxAtoms).total;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the scratch array on the current device.  In host code
// the array's name only stands in for the symbol, so the address is looked up
// with cudaGetSymbolAddress, once per device, with that device current.
static cudaError_t noalloc_scratch_address(void** out) {
    static std::mutex mu;
    static void* addr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        addr[dev] = p;
    }
    *out = addr[dev];
    return cudaSuccess;
}

int lrmsd_noalloc_max_pairs() { return kNoAllocMaxPairs; }
int lrmsd_noalloc_max_atoms() { return kNoAllocMaxAtoms; }
size_t lrmsd_noalloc_scratch_bytes() { return kNoAllocScratchBytes; }

cudaError_t launch_lrmsd_forward_noalloc(const float* input, const float* target,
                                         const int32_t* num_atoms, int P, int Nmax, float* lrmsd,
                                         cudaStream_t s) {
    if (P == 0) return cudaSuccess;
    void* scratch = nullptr;
    cudaError_t e = noalloc_scratch_address(&scratch);
    if (e != cudaSuccess) return e;
    // Nothing in the scratch has to start at zero: every partial that is read
    // is written first in the same call.
    return launch_lrmsd_forward(input, target, num_atoms, P, Nmax, lrmsd, scratch, s);
}

}  // namespace tpl
