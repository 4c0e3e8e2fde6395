// Shared device-side building blocks of the sm_103a kernels: rigid transforms
// in the sparse form of the paper's R(alpha, theta, d), warp/block scans over
// the associative rigid-transform product, and the device status word.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tpl.h"

namespace tpl {

// ---------------------------------------------------------------------------
// Device status word (data-dependent errors, read by tpl_get_status).
// ---------------------------------------------------------------------------
extern __device__ int g_status;

__device__ __forceinline__ void flag_status(int bits) { atomicOr(&g_status, bits); }

// ---------------------------------------------------------------------------
// Rigid transform [Q t; 0 1] with Q stored by columns (c0, c1, c2).
// ---------------------------------------------------------------------------
struct Rigid {
    float3 c0, c1, c2, t;
};

__device__ __forceinline__ Rigid rigid_identity() {
    Rigid r;
    r.c0 = make_float3(1.f, 0.f, 0.f);
    r.c1 = make_float3(0.f, 1.f, 0.f);
    r.c2 = make_float3(0.f, 0.f, 1.f);
    r.t = make_float3(0.f, 0.f, 0.f);
    return r;
}

__device__ __forceinline__ float3 f3_axpy(float a, float3 x, float3 y) {
    return make_float3(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z));
}
__device__ __forceinline__ float3 f3_scale(float a, float3 x) {
    return make_float3(a * x.x, a * x.y, a * x.z);
}
__device__ __forceinline__ float3 f3_add(float3 a, float3 b) {
    return make_float3(a.x + b.x, a.y + b.y, a.z + b.z);
}
__device__ __forceinline__ float3 f3_sub(float3 a, float3 b) {
    return make_float3(a.x - b.x, a.y - b.y, a.z - b.z);
}
__device__ __forceinline__ float3 f3_cross(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float f3_dot(float3 a, float3 b) {
    return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z));
}

// Q v
__device__ __forceinline__ float3 rot_apply(const Rigid& m, float3 v) {
    return f3_axpy(v.z, m.c2, f3_axpy(v.y, m.c1, f3_scale(v.x, m.c0)));
}
// Q v + t  (a point in the frame's coordinates to the parent's)
__device__ __forceinline__ float3 point_apply(const Rigid& m, float3 v) {
    return f3_axpy(v.z, m.c2, f3_axpy(v.y, m.c1, f3_axpy(v.x, m.c0, m.t)));
}

// a * b (apply b first, then a)
__device__ __forceinline__ Rigid rigid_mul(const Rigid& a, const Rigid& b) {
    Rigid r;
    r.c0 = rot_apply(a, b.c0);
    r.c1 = rot_apply(a, b.c1);
    r.c2 = rot_apply(a, b.c2);
    r.t = point_apply(a, b.t);
    return r;
}

// m <- m * R(alpha, theta, d), R from the paper's explicit matrix (Section 3):
// new x axis a = cos(th) c0 - sin(th) c2 (the bond direction), b = sin(th) c0 +
// cos(th) c2, new c1 = sin(al) b + cos(al) c1, new c2 = cos(al) b - sin(al) c1,
// t += d a.  27 FMAs instead of a dense 3x4 product.
__device__ __forceinline__ void rigid_mul_R(Rigid& m, float ca, float sa, float ct, float st,
                                            float d) {
    float3 a = f3_axpy(ct, m.c0, f3_scale(-st, m.c2));
    float3 b = f3_axpy(st, m.c0, f3_scale(ct, m.c2));
    float3 n1 = f3_axpy(sa, b, f3_scale(ca, m.c1));
    float3 n2 = f3_axpy(ca, b, f3_scale(-sa, m.c1));
    m.c0 = a;
    m.c1 = n1;
    m.c2 = n2;
    m.t = f3_axpy(d, a, m.t);
}

// R(alpha, theta, d) itself as a Rigid.
__device__ __forceinline__ Rigid rigid_R(float ca, float sa, float ct, float st, float d) {
    Rigid r;
    r.c0 = make_float3(ct, 0.f, -st);
    r.c1 = make_float3(sa * st, ca, sa * ct);
    r.c2 = make_float3(ca * st, -sa, ca * ct);
    r.t = make_float3(d * ct, 0.f, -d * st);
    return r;
}

// m <- m * R_x(rho)
__device__ __forceinline__ void rigid_mul_Rx(Rigid& m, float cr, float sr) {
    float3 n1 = f3_axpy(cr, m.c1, f3_scale(sr, m.c2));
    float3 n2 = f3_axpy(-sr, m.c1, f3_scale(cr, m.c2));
    m.c1 = n1;
    m.c2 = n2;
}

// Gram-Schmidt on the columns: keeps composed carries on SO(3) in FP32.
__device__ __forceinline__ void rigid_reortho(Rigid& m) {
    float3 c0 = m.c0;
    c0 = f3_scale(rsqrtf(f3_dot(c0, c0)), c0);
    float3 c1 = f3_axpy(-f3_dot(c0, m.c1), c0, m.c1);
    c1 = f3_scale(rsqrtf(f3_dot(c1, c1)), c1);
    m.c0 = c0;
    m.c1 = c1;
    m.c2 = f3_cross(c0, c1);
}

__device__ __forceinline__ Rigid shfl_up_rigid(const Rigid& m, int delta) {
    Rigid r;
    const unsigned full = 0xffffffffu;
    r.c0.x = __shfl_up_sync(full, m.c0.x, delta);
    r.c0.y = __shfl_up_sync(full, m.c0.y, delta);
    r.c0.z = __shfl_up_sync(full, m.c0.z, delta);
    r.c1.x = __shfl_up_sync(full, m.c1.x, delta);
    r.c1.y = __shfl_up_sync(full, m.c1.y, delta);
    r.c1.z = __shfl_up_sync(full, m.c1.z, delta);
    r.c2.x = __shfl_up_sync(full, m.c2.x, delta);
    r.c2.y = __shfl_up_sync(full, m.c2.y, delta);
    r.c2.z = __shfl_up_sync(full, m.c2.z, delta);
    r.t.x = __shfl_up_sync(full, m.t.x, delta);
    r.t.y = __shfl_up_sync(full, m.t.y, delta);
    r.t.z = __shfl_up_sync(full, m.t.z, delta);
    return r;
}

// Shared-memory slot for a Rigid (12 floats).
struct RigidS {
    float v[12];
};
__device__ __forceinline__ void store_rigid(RigidS& s, const Rigid& m) {
    s.v[0] = m.c0.x; s.v[1] = m.c0.y; s.v[2] = m.c0.z;
    s.v[3] = m.c1.x; s.v[4] = m.c1.y; s.v[5] = m.c1.z;
    s.v[6] = m.c2.x; s.v[7] = m.c2.y; s.v[8] = m.c2.z;
    s.v[9] = m.t.x; s.v[10] = m.t.y; s.v[11] = m.t.z;
}
__device__ __forceinline__ Rigid load_rigid(const RigidS& s) {
    Rigid m;
    m.c0 = make_float3(s.v[0], s.v[1], s.v[2]);
    m.c1 = make_float3(s.v[3], s.v[4], s.v[5]);
    m.c2 = make_float3(s.v[6], s.v[7], s.v[8]);
    m.t = make_float3(s.v[9], s.v[10], s.v[11]);
    return m;
}

// ---------------------------------------------------------------------------
// Block-wide exclusive scan of rigid transforms (product in thread order) and
// of an int count.  `s_rig` / `s_cnt` hold NW+1 entries.  On return `excl` is
// x_0 * ... * x_{tid-1}, `cnt_excl` the sum of earlier counts, and `total` /
// `cnt_total` include every thread.  All threads of the CTA must call it (two
// __syncthreads); the caller composes a carry in front.
//
// Every product of warp totals is re-orthonormalised before it is composed
// further: in FP32 the loss of orthogonality of composed rotations, not the
// rounding of the rotation angle, is what drifts along a long chain, and a
// scaled rotation also scales the translations it is later composed with, so
// operands are corrected before use (a correction of the result afterwards
// leaves the translations already built from it).
// ---------------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ void block_scan_rigid_count(const Rigid& x, int cnt, RigidS* s_rig,
                                                       int* s_cnt, Rigid& excl, int& cnt_excl,
                                                       Rigid& total, int& cnt_total) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    Rigid inc = x;
    int cinc = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        Rigid y = shfl_up_rigid(inc, off);
        int cy = __shfl_up_sync(0xffffffffu, cinc, off);
        if (lane >= off) {
            inc = rigid_mul(y, inc);
            cinc += cy;
        }
    }
    if (lane == 31) {
        store_rigid(s_rig[warp], inc);
        s_cnt[warp] = cinc;
    }
    __syncthreads();
    if (warp == 0) {
        Rigid w = (lane < NW) ? load_rigid(s_rig[lane]) : rigid_identity();
        int cw = (lane < NW) ? s_cnt[lane] : 0;
#pragma unroll
        for (int off = 1; off < NW; off <<= 1) {
            Rigid y = shfl_up_rigid(w, off);
            int cy = __shfl_up_sync(0xffffffffu, cw, off);
            if (lane >= off) {
                w = rigid_mul(y, w);
                rigid_reortho(w);
                cw += cy;
            }
        }
        // exclusive warp prefixes, carry folded in; slot NW = total
        Rigid wex = shfl_up_rigid(w, 1);
        int cex = __shfl_up_sync(0xffffffffu, cw, 1);
        if (lane == 0) {
            wex = rigid_identity();
            cex = 0;
        }
        if (lane < NW) {
            store_rigid(s_rig[lane], wex);
            s_cnt[lane] = cex;
        }
        if (lane == NW - 1) {
            store_rigid(s_rig[NW], w);
            s_cnt[NW] = cw;
        }
    }
    __syncthreads();
    Rigid lex = shfl_up_rigid(inc, 1);
    int clex = __shfl_up_sync(0xffffffffu, cinc, 1);
    if (lane == 0) {
        lex = rigid_identity();
        clex = 0;
    }
    excl = rigid_mul(load_rigid(s_rig[warp]), lex);
    cnt_excl = s_cnt[warp] + clex;
    total = load_rigid(s_rig[NW]);
    cnt_total = s_cnt[NW];
}

// ---------------------------------------------------------------------------
// Segmented block-wide exclusive scan of rigid transforms: a thread with
// `head` set starts a new segment (its result is the identity); otherwise the
// result is the product of the earlier threads back to the segment's head.
// Two __syncthreads; s_rig / s_flag hold NW+1 entries.
// ---------------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ Rigid block_seg_scan_rigid(const Rigid& x, bool head, RigidS* s_rig,
                                                      int* s_flag) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    Rigid inc = x;
    int fl = head ? 1 : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const Rigid y = shfl_up_rigid(inc, off);
        const int fy = __shfl_up_sync(0xffffffffu, fl, off);
        if (lane >= off) {
            if (!fl) inc = rigid_mul(y, inc);
            fl |= fy;
        }
    }
    if (lane == 31) {
        store_rigid(s_rig[warp], inc);
        s_flag[warp] = fl;
    }
    __syncthreads();
    if (warp == 0) {
        Rigid w = (lane < NW) ? load_rigid(s_rig[lane]) : rigid_identity();
        int wf = (lane < NW) ? s_flag[lane] : 0;
#pragma unroll
        for (int off = 1; off < NW; off <<= 1) {
            const Rigid y = shfl_up_rigid(w, off);
            const int fy = __shfl_up_sync(0xffffffffu, wf, off);
            if (lane >= off) {
                if (!wf) {
                    w = rigid_mul(y, w);
                    rigid_reortho(w);
                }
                wf |= fy;
            }
        }
        Rigid wex = shfl_up_rigid(w, 1);
        if (lane == 0) wex = rigid_identity();
        if (lane < NW) store_rigid(s_rig[lane], wex);
    }
    __syncthreads();
    Rigid lex = shfl_up_rigid(inc, 1);
    int lexf = __shfl_up_sync(0xffffffffu, fl, 1);
    if (lane == 0) {
        lex = rigid_identity();
        lexf = 0;
    }
    if (head) return rigid_identity();
    return lexf ? lex : rigid_mul(load_rigid(s_rig[warp]), lex);
}

// ---------------------------------------------------------------------------
// Segmented block-wide exclusive scan of ints (same segments as above): the
// sum over the earlier threads back to the segment's head (0 at a head).
// Two __syncthreads; s_val / s_flag hold NW+1 entries.
// ---------------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ int block_seg_scan_count(int x, bool head, int* s_val, int* s_flag) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    int inc = x;
    int fl = head ? 1 : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, off);
        const int fy = __shfl_up_sync(0xffffffffu, fl, off);
        if (lane >= off) {
            if (!fl) inc += y;
            fl |= fy;
        }
    }
    if (lane == 31) {
        s_val[warp] = inc;
        s_flag[warp] = fl;
    }
    __syncthreads();
    if (warp == 0) {
        int w = (lane < NW) ? s_val[lane] : 0;
        int wf = (lane < NW) ? s_flag[lane] : 0;
#pragma unroll
        for (int off = 1; off < NW; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, off);
            const int fy = __shfl_up_sync(0xffffffffu, wf, off);
            if (lane >= off) {
                if (!wf) w += y;
                wf |= fy;
            }
        }
        int wex = __shfl_up_sync(0xffffffffu, w, 1);
        if (lane == 0) wex = 0;
        if (lane < NW) s_val[lane] = wex;
    }
    __syncthreads();
    int lex = __shfl_up_sync(0xffffffffu, inc, 1);
    int lexf = __shfl_up_sync(0xffffffffu, fl, 1);
    if (lane == 0) {
        lex = 0;
        lexf = 0;
    }
    if (head) return 0;
    return lexf ? lex : s_val[warp] + lex;
}

// ---------------------------------------------------------------------------
// Block-wide exclusive REVERSE (suffix) scan of a 6-float sum (r x g, g):
// `after` = sum over threads with a larger index; `total` = sum over all
// threads.  scratch: NW+1 float[6].  Two __syncthreads.
// ---------------------------------------------------------------------------
struct Sum6 {
    float3 c, g;
};
__device__ __forceinline__ Sum6 sum6_zero() {
    Sum6 s;
    s.c = make_float3(0.f, 0.f, 0.f);
    s.g = make_float3(0.f, 0.f, 0.f);
    return s;
}
__device__ __forceinline__ Sum6 sum6_add(const Sum6& a, const Sum6& b) {
    Sum6 s;
    s.c = f3_add(a.c, b.c);
    s.g = f3_add(a.g, b.g);
    return s;
}
__device__ __forceinline__ Sum6 shfl_down_sum6(const Sum6& a, int delta) {
    const unsigned full = 0xffffffffu;
    Sum6 s;
    s.c.x = __shfl_down_sync(full, a.c.x, delta);
    s.c.y = __shfl_down_sync(full, a.c.y, delta);
    s.c.z = __shfl_down_sync(full, a.c.z, delta);
    s.g.x = __shfl_down_sync(full, a.g.x, delta);
    s.g.y = __shfl_down_sync(full, a.g.y, delta);
    s.g.z = __shfl_down_sync(full, a.g.z, delta);
    return s;
}

template <int NT>
__device__ __forceinline__ void block_suffix_sum6(const Sum6& x, float* s6, Sum6& after,
                                                  Sum6& total) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    Sum6 inc = x;  // inclusive suffix within the warp
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        Sum6 y = shfl_down_sum6(inc, off);
        if (lane + off < 32) inc = sum6_add(inc, y);
    }
    if (lane == 0) {
        float* p = s6 + 6 * warp;
        p[0] = inc.c.x; p[1] = inc.c.y; p[2] = inc.c.z;
        p[3] = inc.g.x; p[4] = inc.g.y; p[5] = inc.g.z;
    }
    __syncthreads();
    if (warp == 0) {
        Sum6 w = sum6_zero();
        if (lane < NW) {
            const float* p = s6 + 6 * lane;
            w.c = make_float3(p[0], p[1], p[2]);
            w.g = make_float3(p[3], p[4], p[5]);
        }
#pragma unroll
        for (int off = 1; off < NW; off <<= 1) {
            Sum6 y = shfl_down_sum6(w, off);
            if (lane + off < 32) w = sum6_add(w, y);
        }
        // exclusive suffix of warps: sum over warps > lane
        Sum6 wex = shfl_down_sum6(w, 1);
        if (lane >= NW - 1) wex = sum6_zero();
        __syncwarp();
        if (lane < NW) {
            const Sum6 v = wex;
            float* p = s6 + 6 * lane;
            p[0] = v.c.x; p[1] = v.c.y; p[2] = v.c.z;
            p[3] = v.g.x; p[4] = v.g.y; p[5] = v.g.z;
        }
        if (lane == 0) {
            const Sum6 v = w;
            float* p = s6 + 6 * NW;
            p[0] = v.c.x; p[1] = v.c.y; p[2] = v.c.z;
            p[3] = v.g.x; p[4] = v.g.y; p[5] = v.g.z;
        }
    }
    __syncthreads();
    Sum6 lex = shfl_down_sum6(inc, 1);
    if (lane == 31) lex = sum6_zero();
    const float* p = s6 + 6 * warp;
    Sum6 wv;
    wv.c = make_float3(p[0], p[1], p[2]);
    wv.g = make_float3(p[3], p[4], p[5]);
    after = sum6_add(wv, lex);
    const float* q = s6 + 6 * NW;
    total.c = make_float3(q[0], q[1], q[2]);
    total.g = make_float3(q[3], q[4], q[5]);
}

// Segmented form: a thread with `tail` set ends its segment, so its result
// is zero; otherwise the result sums the later threads up to and including
// the segment's tail.  Two __syncthreads; s6 holds NW+1 float[6], s_flag NW+1.
template <int NT>
__device__ __forceinline__ Sum6 block_seg_suffix_sum6(const Sum6& x, bool tail, float* s6,
                                                      int* s_flag) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    Sum6 inc = x;
    int fl = tail ? 1 : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const Sum6 y = shfl_down_sum6(inc, off);
        const int fy = __shfl_down_sync(0xffffffffu, fl, off);
        if (lane + off < 32) {
            if (!fl) inc = sum6_add(inc, y);
            fl |= fy;
        }
    }
    if (lane == 0) {
        float* p = s6 + 6 * warp;
        p[0] = inc.c.x; p[1] = inc.c.y; p[2] = inc.c.z;
        p[3] = inc.g.x; p[4] = inc.g.y; p[5] = inc.g.z;
        s_flag[warp] = fl;
    }
    __syncthreads();
    if (warp == 0) {
        Sum6 w = sum6_zero();
        int wf = 0;
        if (lane < NW) {
            const float* p = s6 + 6 * lane;
            w.c = make_float3(p[0], p[1], p[2]);
            w.g = make_float3(p[3], p[4], p[5]);
            wf = s_flag[lane];
        }
#pragma unroll
        for (int off = 1; off < NW; off <<= 1) {
            const Sum6 y = shfl_down_sum6(w, off);
            const int fy = __shfl_down_sync(0xffffffffu, wf, off);
            if (lane + off < 32) {
                if (!wf) w = sum6_add(w, y);
                wf |= fy;
            }
        }
        Sum6 wex = shfl_down_sum6(w, 1);  // segment sum starting at the next warp
        if (lane >= NW - 1) wex = sum6_zero();
        __syncwarp();
        if (lane < NW) {
            float* p = s6 + 6 * lane;
            p[0] = wex.c.x; p[1] = wex.c.y; p[2] = wex.c.z;
            p[3] = wex.g.x; p[4] = wex.g.y; p[5] = wex.g.z;
        }
    }
    __syncthreads();
    Sum6 lex = shfl_down_sum6(inc, 1);
    int lexf = __shfl_down_sync(0xffffffffu, fl, 1);
    if (lane == 31) {
        lex = sum6_zero();
        lexf = 0;
    }
    if (tail) return sum6_zero();
    if (lexf) return lex;
    const float* p = s6 + 6 * warp;
    Sum6 wv;
    wv.c = make_float3(p[0], p[1], p[2]);
    wv.g = make_float3(p[3], p[4], p[5]);
    return sum6_add(lex, wv);
}

// LRMSD = sqrt(sum / n) and the gradient factor 1 / (n LRMSD) from the FP64
// residual sum of n atoms.  Both are stored as float, so they are formed in
// FP32 (within an ulp or two of the FP64 forms, without FP64's long sqrt and
// divide sequences).  An LRMSD below 1e-12 has no gradient: factor 0, status
// TPL_STATUS_ZERO_LRMSD.
__device__ __forceinline__ void lrmsd_from_sum(double sum, int n, float& lr, float& scale) {
    lr = 0.f;
    scale = 0.f;
    if (n <= 0) return;
    const float ms = (float)sum / (float)n;
    lr = ms > 0.f ? sqrtf(ms) : 0.f;
    if (lr >= 1e-12f)
        scale = 1.f / ((float)n * lr);
    else
        flag_status(TPL_STATUS_ZERO_LRMSD);
}

// Inputs of an LRMSD gradient formed inside a chain backward (Section 4): for
// chain b, g_i = w_b ((y_i - yc) - U (x_i - xc)) with y the chain's
// coordinates, x the target and w_b = grad_lrmsd[b] / (N LRMSD), from the
// per-pair state of the LRMSD forward (U row-major, xc, yc, 1 / (N LRMSD)).
struct LrmsdGrad {
    const float* target;
    const float* state;
    const float* grad_lrmsd;
    // fused training step: LRMSD per chain out, atoms per chain in
    float* lrmsd_out;
    const int32_t* num_atoms;
};

__device__ __forceinline__ int clamp_length(const int32_t* lengths, int b, int Lmax) {
    int L = lengths[b];
    if (L < 0 || L > Lmax) {
        flag_status(TPL_STATUS_BAD_LENGTH);
        L = L < 0 ? 0 : Lmax;
    }
    return L;
}

}  // namespace tpl
