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
//    column; cyclic Jacobi where lambda_max is nearly double), refines the
//    eigenvector once against the exact T (compensated products and sums),
//    then U(q);
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
#include "lrmsd_solve.cuh"

namespace tpl {

namespace {

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

// Eigen-solve of the fused training step: the partials are per tile of `tile`
// residues of chain p (the full-atom forward's tile moments), eight pairs per
// warp.
__global__ void __launch_bounds__(32) lrmsd_solve_tiles_kernel(
    const float* __restrict__ input, const float* __restrict__ target,
    const int32_t* __restrict__ num_atoms, int P, int Nmax, const float* __restrict__ part1,
    int tiles_max, float* __restrict__ state, const int32_t* __restrict__ lengths, int tile, int Lmax,
    bool balanced, int min_tiles) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int sub = gid & 3, lane = threadIdx.x & 31;
    const int p = (gid >> 2) < P ? (gid >> 2) : P - 1;
    const int L = min(max(lengths[p], 0), Lmax);
    const int n = num_atoms ? pair_atoms(num_atoms, p, Nmax) : min(3 * L, Nmax);
    const int nch = balanced ? fa_num_tiles(L, tile) : (L > 0 ? (L + tile - 1) / tile : 1);
    const bool active = (gid >> 2) < P && nch >= min_tiles;
    float x0[3], y0[3];
    first_atoms(target + (size_t)p * Nmax * 3, input + (size_t)p * Nmax * 3, n, x0, y0);
    float S[kSlot];
    quad_sum_partials(part1 + (size_t)p * tiles_max * kSlot, nch, sub, S);
    quad_eigen_solve(S, x0, y0, n, sub, lane, active, state + 16 * (size_t)p);
}

// ---------------------------------------------------------------------------
// K5: the whole forward of a pair in one CTA: moments, eigen-solve by one quad
// of one warp, residual sum and LRMSD, with block barriers between the steps.
// The solving warp is the pair index modulo the CTA's warps: the CTAs an SM
// holds then solve on different schedulers.  Two shapes: 256 threads with
// four groups of four atoms per thread in flight (two CTAs per SM) for
// batches that fit one wave, and a compact one, 128 threads with two groups
// (six CTAs per SM), for larger batches: about 900 pairs are then in flight,
// their clouds (tens of MB) stay in L2, and the residual pass reads them from
// there instead of from HBM, while other CTAs on the SM stream while one
// CTA's quad solves.
// ---------------------------------------------------------------------------
constexpr int kPNT = 256;
constexpr int kCNT = 128;  // compact shape

// The residual pass and the state of one pair, by the whole CTA after the
// eigen-solve left U and the centroids in s_st: sum |y'_i - U x'_i|^2 (FP32
// per thread, FP64 over the warps), LRMSD and 1 / (N LRMSD); G groups of four
// atoms per thread in flight.  Ends with the state written (16 floats).
template <int NT, int G>
__device__ __forceinline__ void residual_pass(const float* __restrict__ x, const float* __restrict__ y, int n,
                                              const float* s_st, double* s_res, float* __restrict__ state_p,
                                              float* __restrict__ lrmsd_p) {
    constexpr int NW = NT / 32;
    constexpr int kBatch = 4 * G * NT;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const PairState ps = load_state_shared(s_st);
    float acc = 0.f;
    for (int base = 0; base < n; base += kBatch) {
        float3 xv[G][4], yv[G][4];
#pragma unroll
        for (int s = 0; s < G; ++s) {
            const int i0 = base + 4 * (threadIdx.x + NT * s);
            if (i0 < n) {
                load4(x + 3 * (size_t)i0, xv[s]);
                load4(y + 3 * (size_t)i0, yv[s]);
            }
        }
#pragma unroll
        for (int s = 0; s < G; ++s) {
            const int i0 = base + 4 * (threadIdx.x + NT * s);
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
    if (threadIdx.x < 15) state_p[threadIdx.x] = s_st[threadIdx.x];
    if (threadIdx.x == 0) {
        double sum = 0.0;
#pragma unroll
        for (int w = 0; w < NW; ++w) sum += s_res[w];
        float lr, scale;
        lrmsd_from_sum(sum, n, lr, scale);
        state_p[15] = scale;
        *lrmsd_p = lr;
    }
}

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
    if (warp == (p & (NW - 1))) {  // differs from pair to pair: co-resident CTAs solve on different schedulers
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
    residual_pass<NT, G>(x, y, n, s_st, s_res, state + 16 * (size_t)p, lrmsd + p);
}

// K5p: the LRMSD of the fused full-atom step from the forward's per-tile
// moments (the forward reduced each tile's atoms against the target): one CTA
// per chain; one quad of one warp sums the chain's tile partials in order and
// solves, then the CTA sums the squared residuals over the chain's atoms,
// which the forward has just written and read, so they come from L2.
template <int NT, int G>
__global__ void __launch_bounds__(NT) lrmsd_parts_kernel(
    const float* __restrict__ input, const float* __restrict__ target, const int32_t* __restrict__ num_atoms,
    int P, int Nmax, const float* __restrict__ part1, int tiles_max, const int32_t* __restrict__ lengths,
    int tile, int Lmax, float* __restrict__ state, float* __restrict__ lrmsd) {
    __shared__ double s_res[NT / 32];
    __shared__ __align__(16) float s_st[16];
    const int p = blockIdx.x;
    const int lane = threadIdx.x & 31;
    const float* x = target + (size_t)p * Nmax * 3;
    const float* y = input + (size_t)p * Nmax * 3;
    const int n = pair_atoms(num_atoms, p, Nmax);
    if ((threadIdx.x >> 5) == (p & (NT / 32 - 1))) {  // solves of co-resident CTAs on different schedulers
        const int L = min(max(lengths[p], 0), Lmax);
        float x0[3], y0[3];
        first_atoms(x, y, n, x0, y0);
        float S[kSlot];
        quad_sum_partials(part1 + (size_t)p * tiles_max * kSlot, fa_num_tiles(L, tile), lane & 3, S);
        quad_eigen_solve(S, x0, y0, n, lane & 3, lane, lane < 4, s_st);
    }
    __syncthreads();
    residual_pass<NT, G>(x, y, n, s_st, s_res, state + 16 * (size_t)p, lrmsd + p);
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
                                     cudaStream_t s, bool balanced, int min_tiles) {
    if (P == 0) return cudaSuccess;
    lrmsd_solve_tiles_kernel<<<(4 * P + 31) / 32, 32, 0, s>>>(input, target, num_atoms, P, Nmax, tile_moments,
                                                             tiles_max, state, lengths, tile, Lmax, balanced,
                                                             min_tiles);
    return cudaGetLastError();
}

cudaError_t launch_lrmsd_parts(const float* input, const float* target, const int32_t* num_atoms, int P,
                               int Nmax, const float* tile_moments, int tiles_max, const int32_t* lengths, int tile,
                               int Lmax, float* state, float* lrmsd, cudaStream_t s) {
    if (P == 0) return cudaSuccess;
    lrmsd_parts_kernel<kPNT, 4><<<P, kPNT, 0, s>>>(input, target, num_atoms, P, Nmax, tile_moments, tiles_max,
                                                   lengths, tile, Lmax, state, lrmsd);
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
