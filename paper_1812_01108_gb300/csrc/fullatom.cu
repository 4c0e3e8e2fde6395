// Full-atom model of the paper (Section 2) on sm_103a.
//
// Chains are cut into tiles of NT residues (one residue per thread) that
// persistent CTAs take from the schedule's work list; the tiles of a chain
// meet through the aggregate look-back of sched.cuh.
//
// K3 fa_fwd_kernel: the residue-to-residue transform T_j = R_1(phi_j)
// R_3(psi_j) R_4(omega_{j+1}) is scanned across the tile (exclusive prefix =
// M_0 of residue j, the frame of its N, relative to the tile start), together
// with an exclusive scan of the per-residue atom counts (the residue's first
// output atom).  Each thread then builds M_1, M_3 and the side-chain frames
// M_1 R' R(chi_1) R(chi_2) ... and places its atoms r = M_g r0 into a
// shared-memory stage; once the look-back has given the tile's start frame it
// is applied in place and the CTA writes the stage out with 16-byte stores.
// The residue tables live in shared memory.
//
// K4 fa_bwd_coords_kernel / fa_bwd_kernel: Eq. 1 as suffix sums.  For a frame
// with x axis u and origin p, dL/dalpha = u . sum_{k downstream} (r_k - p) x
// g_k.  chi_k gradients are local to the residue (suffix over its side-chain
// groups); phi, psi and omega add the sum over all later residues, a reverse
// suffix scan of (sum r x g, sum g) across the tile plus the suffix of the
// later tiles (look-back, tiles of a chain taken last to first).  Axes and
// origins come from the forward's coordinates (fa_bwd_coords_kernel) or from
// frames recomputed from the angles and the tile-start frames (fa_bwd_kernel).
#include "kernels.h"
#include "sched.cuh"
#include "tables.h"
#include "tpl_common.cuh"

namespace tpl {

namespace {

__device__ __forceinline__ void copy_table(FaTable& dst, const FaTable& src) {
    const int n = sizeof(FaTable) / 4;
    const int* s = reinterpret_cast<const int*>(&src);
    int* d = reinterpret_cast<int*>(&dst);
    for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = s[i];
}

__device__ __forceinline__ int residue_type(const uint8_t* __restrict__ sq, int j, bool valid) {
    if (!valid) return kGlyCode;
    int t = sq[j];
    if (t >= kNumTypes) {
        flag_status(TPL_STATUS_BAD_RESIDUE);
        t = kGlyCode;
    }
    return t;
}

// Residue transform T_j = R(phi) R(psi) R(omega_{j+1}) (the last residue of a
// chain has no R_4).  Returns the sin/cos of phi and psi for reuse.
__device__ __forceinline__ Rigid residue_transform(const FaTable& tab, const float* ang, int Lmax,
                                                   int j, int L, float& sp, float& cp, float& ss,
                                                   float& cs) {
    Rigid A = rigid_identity();
    if (j >= L) return A;
    sincosf(ang[j], &sp, &cp);
    sincosf(ang[Lmax + j], &ss, &cs);
    A = rigid_R(cp, sp, tab.bb.ct[1], tab.bb.st[1], tab.bb.d[1]);
    rigid_mul_R(A, cs, ss, tab.bb.ct[2], tab.bb.st[2], tab.bb.d[2]);
    if (j + 1 < L) {
        float so, co;
        sincosf(ang[2 * Lmax + j + 1], &so, &co);
        rigid_mul_R(A, co, so, tab.bb.ct[0], tab.bb.st[0], tab.bb.d[0]);
    }
    return A;
}

__device__ __forceinline__ void stage_atom(float* stage, int slot, float3 r) {
    stage[3 * slot + 0] = r.x;
    stage[3 * slot + 1] = r.y;
    stage[3 * slot + 2] = r.z;
}

// Copy of the float range [g0, g1) between global memory and a shared buffer
// laid out so that stage[off + i] <-> global[g0 + i], off = g0 mod 4: the
// 16-byte aligned middle moves as float4, the ragged ends as floats.
template <int NT, bool TO_GLOBAL>
__device__ __forceinline__ void copy_range(float* __restrict__ glob, float* __restrict__ stage,
                                           int g0, int g1) {
    if (g1 <= g0) return;
    const int off = g0 & 3;
    const int head = min(g1, (g0 + 3) & ~3);
    const int tail = max(head, g1 & ~3);
    for (int i = g0 + threadIdx.x; i < head; i += NT) {
        if (TO_GLOBAL) glob[i] = stage[off + i - g0];
        else stage[off + i - g0] = __ldg(glob + i);
    }
    for (int q = head / 4 + threadIdx.x; q < tail / 4; q += NT) {
        float4* sp = reinterpret_cast<float4*>(stage + off + 4 * q - g0);
        float4* gp = reinterpret_cast<float4*>(glob) + q;
        if (TO_GLOBAL) *gp = *sp;
        else *sp = __ldg(gp);
    }
    for (int i = tail + threadIdx.x; i < g1; i += NT) {
        if (TO_GLOBAL) glob[i] = stage[off + i - g0];
        else stage[off + i - g0] = __ldg(glob + i);
    }
}

// Store of the float range [g0, g1) from a shared buffer with stage[i - g0] <->
// global[i]: 16-byte aligned global stores, gathered from shared memory.
template <int NT>
__device__ __forceinline__ void store_range(float* __restrict__ glob, const float* __restrict__ stage,
                                            int g0, int g1) {
    if (g1 <= g0) return;
    const int head = min(g1, (g0 + 3) & ~3);
    const int tail = max(head, g1 & ~3);
    for (int i = g0 + threadIdx.x; i < head; i += NT) glob[i] = stage[i - g0];
    for (int q = head / 4 + threadIdx.x; q < tail / 4; q += NT) {
        const float* sp = stage + 4 * q - g0;
        reinterpret_cast<float4*>(glob)[q] = make_float4(sp[0], sp[1], sp[2], sp[3]);
    }
    for (int i = tail + threadIdx.x; i < g1; i += NT) glob[i] = stage[i - g0];
}

// Fetch the 128-byte line at p into L2 (a hint; nothing waits on it).
__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Asynchronous copy (cp.async, no register round trip) of the float range
// [g0, g1) of global memory into stage[off + i - g0], off = g0 mod 4: 16-byte
// copies for the aligned middle, 4-byte copies for the ragged ends.  The caller
// commits and waits (cp_async_wait_all) before a barrier.
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

template <int NT>
__device__ __forceinline__ void async_copy_range(const float* __restrict__ glob, float* __restrict__ stage,
                                                 int g0, int g1) {
    if (g1 <= g0) return;
    const int off = g0 & 3;
    const int head = min(g1, (g0 + 3) & ~3);
    const int tail = max(head, g1 & ~3);
    for (int i = g0 + threadIdx.x; i < head; i += NT) cp_async4(stage + off + i - g0, glob + i);
    for (int q = head / 4 + threadIdx.x; q < tail / 4; q += NT) cp_async16(stage + off + 4 * q - g0, glob + 4 * q);
    for (int i = tail + threadIdx.x; i < g1; i += NT) cp_async4(stage + off + i - g0, glob + i);
}

template <int NT>
__device__ __forceinline__ void zero_range(float* __restrict__ glob, int g0, int g1) {
    if (g1 <= g0) return;
    const int head = min(g1, (g0 + 3) & ~3);
    const int tail = max(head, g1 & ~3);
    for (int i = g0 + threadIdx.x; i < head; i += NT) glob[i] = 0.f;
    for (int q = head / 4 + threadIdx.x; q < tail / 4; q += NT)
        reinterpret_cast<float4*>(glob)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = tail + threadIdx.x; i < g1; i += NT) glob[i] = 0.f;
}

__device__ __forceinline__ bool ws_matches(const ChainWs& ws, int tile, int B, int Lmax) {
    return ws.hdr[kHdrMagic] == kWsMagic && ws.hdr[kHdrTile] == tile && ws.hdr[kHdrB] == B &&
           ws.hdr[kHdrLmax] == Lmax;
}

// ---------------------------------------------------------------------------
// K3: forward.  One tile of NT residues per step of a persistent CTA:
//  1. every angle row and the type of each thread's residue are loaded up
//     front; T_j is built and scanned across the tile with the atom counts,
//     and the tile's aggregate is published for the look-back;
//  2. each thread places its residue's atoms (N, CA, C, O, then the side
//     chain group by group) in tile-local coordinates in the stage;
//  3. the look-back gives the tile's start frame, which is applied to the
//     stage in place (not for a chain's first tile: R_0 = I);
//  4. the stage is written out with 16-byte stores.
// ---------------------------------------------------------------------------
template <int NT>
__host__ __device__ constexpr size_t fa_fwd_smem() {
    return (size_t)(4 + NT * kMaxAtoms * 3) * 4;
}

// CTAs per SM the forward and backward kernels are compiled for (register cap)
template <int NT>
__host__ __device__ constexpr int fa_min_blocks() {
    return NT >= 512 ? 1 : (NT >= 384 ? 2 : (NT >= 256 ? 4 : (NT >= 192 ? 5 : 8)));
}

// The coordinate-reading backward stages two tiles (coordinates and their
// gradients), so shared memory holds fewer of its CTAs per SM.
template <int NT>
__host__ __device__ constexpr int fa_bwd_min_blocks() {
    return NT >= 384 ? 2 : (NT >= 256 ? 4 : (NT >= 192 ? 5 : 8));
}

// LM: also reduce, per tile, the LRMSD moments (Section 4) of the tile's atoms
// against `target`: sum dx, sum dy, sum dx dy^T, sum |dx|^2, sum |dy|^2 with
// dx = x - x_0 (x the target, x_0 its first atom) and dy = y (the chain's
// first atom, N of residue 0, is the origin: R_0 = I).
template <int NT, bool LM>
__global__ void __launch_bounds__(NT, fa_min_blocks<NT>()) fa_fwd_kernel(
    const float* __restrict__ angles, const uint8_t* __restrict__ seq,
    const int32_t* __restrict__ lengths, int Lmax, int Amax, float* __restrict__ coords,
    int32_t* __restrict__ num_atoms, ChainWs ws, const float* __restrict__ target,
    const __grid_constant__ FaTable tab) {
    constexpr int NW = NT / 32;
    __shared__ FaTable s_tab;
    __shared__ RigidS s_rig[NW + 1];
    __shared__ int s_cnt[NW + 1];
    __shared__ int s_v, s_next;
    __shared__ float s_mom[LM ? NW : 1][17];
    extern __shared__ float4 s_dyn[];
    float* stage = reinterpret_cast<float*>(s_dyn);  // tile-local atoms, 3 floats each

    copy_table(s_tab, tab);
    const int ntiles = ws.hdr[kHdrTiles];
    int v = take_tile(ws.hdr + kHdrFwdNext, &s_v);
    while (v < ntiles) {
        const int2 ct = ws.tiles[v];
        const int b = ct.x, t = ct.y;
        const int L = clamp_length(lengths, b, Lmax);
        const int T = L > 0 ? (L + NT - 1) / NT : 1;
        const int slot0 = b * ws.tmax;
        const float* ang = angles + (size_t)b * 7 * Lmax;
        float* out = coords + (size_t)b * Amax * 3;

        const int j = t * NT + threadIdx.x;
        const bool valid = j < L;
        int type = kGlyCode;
        float a_phi = 0.f, a_psi = 0.f, a_om = 0.f, a_chi[kMaxGroups] = {0.f, 0.f, 0.f, 0.f};
        if (valid) {
            // every angle row up front (the chi rows too, used or not), so no
            // load waits inside the side-chain loop
            type = residue_type(seq + (size_t)b * Lmax, j, true);
            a_phi = __ldg(ang + j);
            a_psi = __ldg(ang + Lmax + j);
            if (j + 1 < L) a_om = __ldg(ang + 2 * Lmax + j + 1);
#pragma unroll
            for (int c = 0; c < kMaxGroups; ++c) a_chi[c] = __ldg(ang + (3 + c) * Lmax + j);
        }
        const int nat = valid ? s_tab.n_atoms[type] : 0;
        float sp = 0.f, cp = 1.f, ss = 0.f, cs = 1.f;
        Rigid A = rigid_identity();
        if (valid) {
            sincosf(a_phi, &sp, &cp);
            sincosf(a_psi, &ss, &cs);
            A = rigid_R(cp, sp, s_tab.bb.ct[1], s_tab.bb.st[1], s_tab.bb.d[1]);
            rigid_mul_R(A, cs, ss, s_tab.bb.ct[2], s_tab.bb.st[2], s_tab.bb.d[2]);
            if (j + 1 < L) {
                float so, co;
                sincosf(a_om, &so, &co);
                rigid_mul_R(A, co, so, s_tab.bb.ct[0], s_tab.bb.st[0], s_tab.bb.d[0]);
            }
        }
        Rigid E, Tot;
        int a0, tile_atoms;
        block_scan_rigid_count<NT>(A, nat, s_rig, s_cnt, E, a0, Tot, tile_atoms);
        // publish the tile's aggregate now (successors need it); every warp
        // gathers the prefix later, so no warp waits on another for it
        if (threadIdx.x == NT - 32) publish_prefix_agg(ws, slot0 + t, Tot, tile_atoms);
        // residue atoms in tile-local coordinates (E is relative to the tile start)
        if (valid) {
            float* st = stage + 3 * a0;
            stage_atom(st, 0, E.t);  // N = M_0 0
            Rigid M1 = E;
            rigid_mul_R(M1, cp, sp, s_tab.bb.ct[1], s_tab.bb.st[1], s_tab.bb.d[1]);
            stage_atom(st, 1, M1.t);  // CA = M_1 0
            Rigid M3 = M1;
            rigid_mul_R(M3, cs, ss, s_tab.bb.ct[2], s_tab.bb.st[2], s_tab.bb.d[2]);
            stage_atom(st, 2, M3.t);  // C = M_3 0
            const float4 o = s_tab.o_r0;
            stage_atom(st, 3, point_apply(M3, make_float3(o.x, o.y, o.z)));
            // side-chain groups: S_k = S_{k-1} R(chi_k), S_0 = M_1 R'; atoms r = S_k r0
            Rigid S = M1;
            rigid_mul_Rx(S, s_tab.rp_c, s_tab.rp_s);
            const int ng = s_tab.n_groups[type], nchi = s_tab.n_chi[type];
            int e = 0;
#pragma unroll
            for (int k = 0; k < kMaxGroups; ++k) {
                if (k >= ng) break;
                float sc, cc;
                if (k < nchi) {
                    // chi moves only its own side chain (no error propagates along
                    // the chain): the SFU sine/cosine is accurate enough here
                    __sincosf(a_chi[k], &sc, &cc);
                } else {
                    cc = s_tab.fixchi[type][k].x;
                    sc = s_tab.fixchi[type][k].y;
                }
                const float4 gk = s_tab.grp[type][k];
                rigid_mul_R(S, cc, sc, gk.x, gk.y, gk.z);
                const int end = s_tab.grp_end[type][k];
                for (; e < end; ++e) {
                    const float4 r0 = s_tab.side[type][e];
                    stage_atom(st, (int)r0.w & 15, point_apply(S, make_float3(r0.x, r0.y, r0.z)));
                }
            }
        }
        __syncthreads();
        // frame at the tile start (every warp gathers it), applied in place
        int pc;
        const Rigid P = gather_prefix(ws, slot0, t, pc);
        const int requested = request_tile(ws.hdr + kHdrFwdNext);  // after the last wait of this tile
        if (threadIdx.x == 0) s_next = requested;
        if (threadIdx.x == 0) store_rigid_g(ws.start + 4 * (size_t)(slot0 + t), P, pc, tile_atoms);
        if (valid) ws.ratom[(size_t)b * Lmax + j] = pc + a0;  // the backward reads its atoms directly
        const int end_atom = pc + tile_atoms;
        const int nout = max(0, min(end_atom, Amax) - pc);
        if (t > 0) {  // the chain's first tile starts at the identity frame (R_0 = I)
            for (int a = threadIdx.x; a < nout; a += NT) {
                const float3 r = point_apply(P, make_float3(stage[3 * a], stage[3 * a + 1], stage[3 * a + 2]));
                stage[3 * a] = r.x;
                stage[3 * a + 1] = r.y;
                stage[3 * a + 2] = r.z;
            }
        }
        __syncthreads();
        {
            // the next tile's angle rows and sequence into L2 while this tile is stored
            const int vn = s_next;
            if (vn < ntiles && threadIdx.x < 64) {
                const int2 cn = ws.tiles[vn];
                const int row = threadIdx.x >> 3, part = threadIdx.x & 7;  // 8 rows x 8 parts of NT residues
                const int jn = cn.y * NT + part * (NT / 8);
                if (cn.x >= 0 && jn < Lmax) {
                    const char* base = row < 7 ? reinterpret_cast<const char*>(angles + ((size_t)cn.x * 7 + row) * Lmax + jn)
                                               : reinterpret_cast<const char*>(seq + (size_t)cn.x * Lmax + jn);
                    const int bytes = (row < 7 ? 4 : 1) * min(NT / 8, Lmax - jn);
                    for (int o = 0; o < bytes; o += 128) prefetch_l2(base + o);
                }
            }
        }
        if (end_atom > Amax && threadIdx.x == 0) flag_status(TPL_STATUS_TOO_MANY_ATOMS);
        store_range<NT>(out, stage, 3 * pc, 3 * (pc + nout));
        if (t == T - 1) {
            if (threadIdx.x == 0) num_atoms[b] = end_atom;
            zero_range<NT>(out, 3 * min(end_atom, Amax), 3 * Amax);
        }
        if constexpr (LM) {
            const float* tg = target + (size_t)b * Amax * 3;
            const float3 x0 = make_float3(__ldg(tg), __ldg(tg + 1), __ldg(tg + 2));
            float m[17];
#pragma unroll
            for (int k = 0; k < 17; ++k) m[k] = 0.f;
            for (int a = threadIdx.x; a < nout; a += NT) {
                const float* xa = tg + 3 * (size_t)(pc + a);
                const float3 dx = make_float3(__ldg(xa) - x0.x, __ldg(xa + 1) - x0.y, __ldg(xa + 2) - x0.z);
                const float3 dy = make_float3(stage[3 * a], stage[3 * a + 1], stage[3 * a + 2]);
                m[0] += dx.x; m[1] += dx.y; m[2] += dx.z;
                m[3] += dy.x; m[4] += dy.y; m[5] += dy.z;
                m[6] = fmaf(dx.x, dy.x, m[6]); m[7] = fmaf(dx.x, dy.y, m[7]); m[8] = fmaf(dx.x, dy.z, m[8]);
                m[9] = fmaf(dx.y, dy.x, m[9]); m[10] = fmaf(dx.y, dy.y, m[10]); m[11] = fmaf(dx.y, dy.z, m[11]);
                m[12] = fmaf(dx.z, dy.x, m[12]); m[13] = fmaf(dx.z, dy.y, m[13]); m[14] = fmaf(dx.z, dy.z, m[14]);
                m[15] += f3_dot(dx, dx);
                m[16] += f3_dot(dy, dy);
            }
            // block sum: warp shuffles, then the warp sums in a fixed order
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
            for (int k = 0; k < 17; ++k) {
                float v = m[k];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                m[k] = v;
            }
            if (lane == 0)
#pragma unroll
                for (int k = 0; k < 17; ++k) s_mom[warp][k] = m[k];
            __syncthreads();
            if (threadIdx.x < 17) {
                float v = 0.f;
                for (int w = 0; w < NW; ++w) v += s_mom[w][threadIdx.x];
                ws.tmom[(size_t)(slot0 + t) * 20 + threadIdx.x] = v;
            }
        }
        v = next_tile(requested, &s_v);
    }
}

// Block-wide exclusive scan of an int (tile atom offsets); two __syncthreads.
template <int NT>
__device__ __forceinline__ int block_scan_int(int x, int* s_cnt, int& total) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
    }
    if (lane == 31) s_cnt[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = lane < NW ? s_cnt[lane] : 0;
#pragma unroll
        for (int off = 1; off < NW; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += y;
        }
        if (lane < NW) s_cnt[lane] = w - (lane < NW ? s_cnt[lane] : 0);
        if (lane == NW - 1) s_cnt[NW] = w;
    }
    __syncthreads();
    total = s_cnt[NW];
    return s_cnt[warp] + inc - x;
}

// ---------------------------------------------------------------------------
// K4': backward from the forward's coordinates.  Axes and origins come from
// atom positions (phi: N->CA, psi: CA->C, omega: C_{j-1}->N_j, chi_k: origin of
// group k-1 -> origin of group k); the tile's atoms and their upstream
// gradients are staged in shared memory with 16-byte loads.
// ---------------------------------------------------------------------------

__device__ __forceinline__ float3 unit3(float3 v) { return f3_scale(rsqrtf(f3_dot(v, v)), v); }


// RES (with LR, the fused training step): the LRMSD gradient is formed
// without its 1 / (N LRMSD) factor, each tile also sums its atoms' squared
// residuals |y' - U x'|^2 (Section 4), and the chain's first tile -- taken
// last -- waits for the chain's other tiles, forms LRMSD in FP64 and rescales
// the chain's angle gradients.
template <int NT, bool LR, bool RES>
__global__ void __launch_bounds__(NT, fa_bwd_min_blocks<NT>()) fa_bwd_coords_kernel(
    const uint8_t* __restrict__ seq, const int32_t* __restrict__ lengths, int B, int Lmax, int Amax,
    const float* __restrict__ coords, const float* __restrict__ grad_coords,
    float* __restrict__ grad_angles, ChainWs ws, LrmsdGrad lg, const __grid_constant__ FaTable tab) {
    constexpr int NW = NT / 32;
    __shared__ FaTable s_tab;
    __shared__ float s6[6 * (NW + 1)];
    __shared__ int s_v;
    __shared__ float s_res[NW];
    __shared__ float s_scale;
    extern __shared__ float4 s_dyn[];
    float* st_r = reinterpret_cast<float*>(s_dyn);  // the tile's coordinates

    if (!ws_matches(ws, NT, B, Lmax)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) flag_status(TPL_STATUS_BAD_WORKSPACE);
        for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < (size_t)B * 7 * Lmax; i += (size_t)gridDim.x * NT)
            grad_angles[i] = 0.f;
        return;
    }
    copy_table(s_tab, tab);
    const int ntiles = ws.hdr[kHdrTiles];
    int* counter = ws.bflag + ws.slots;
    int v = take_tile(counter, &s_v);
    while (v < ntiles) {
        const int2 ct = ws.tiles[v];
        const int b = ct.x;
        const int L = clamp_length(lengths, b, Lmax);
        const int T = L > 0 ? (L + NT - 1) / NT : 1;
        const int t = T - 1 - ct.y;  // last tile first
        const int slot0 = b * ws.tmax;
        const uint8_t* sq = seq + (size_t)b * Lmax;
        const float* r_in = coords + (size_t)b * Amax * 3;
        const float* g_in = grad_coords + (size_t)b * Amax * 3;
        float* ga = grad_angles + (size_t)b * 7 * Lmax;

        // the tile's coordinates are staged with coalesced asynchronous copies
        // (the forward recorded the tile's first atom and atom count, and
        // every residue's first atom); each thread reads the gradient or
        // target of its own atoms directly
        const float4 sd = ws.start[4 * (size_t)(slot0 + t) + 3];
        const int pc = __float_as_int(sd.x);
        const int soff = (3 * pc) & 3;
        async_copy_range<NT>(r_in, st_r, 3 * pc, 3 * min(pc + __float_as_int(sd.y), Amax));
        const int j = t * NT + threadIdx.x;
        const bool valid = j < L;
        const int type = residue_type(sq, j, valid);
        const int nat = valid ? s_tab.n_atoms[type] : 0;
        const int a0 = valid ? __ldg(ws.ratom + (size_t)b * Lmax + j) : 0;
        const int ap = (valid && j > 0) ? __ldg(ws.ratom + (size_t)b * Lmax + j - 1) : 0;

        const bool in_range = valid && a0 >= pc && a0 + nat <= Amax && a0 - pc + nat <= NT * kMaxAtoms;
        cp_async_wait_all();
        __syncthreads();
        float res_acc = 0.f;  // RES: this thread's squared residuals
        float gchi[kMaxGroups] = {0.f, 0.f, 0.f, 0.f};
        Sum6 all = sum6_zero(), nsum = sum6_zero(), csum = sum6_zero();
        float3 rN = make_float3(0.f, 0.f, 0.f), rCA = rN, rC = rN, rCprev = rN;
        if (in_range) {
            const float* sr = st_r + soff + 3 * (a0 - pc);
            auto R = [&](int k) { return make_float3(sr[3 * k], sr[3 * k + 1], sr[3 * k + 2]); };
            // the coordinate gradient: read, or formed from the LRMSD state
            const float* sg = LR ? lg.target + ((size_t)b * Amax + a0) * 3 : g_in + 3 * (size_t)a0;
            float3 u0 = make_float3(0.f, 0.f, 0.f), u1 = u0, u2 = u0, xc = u0, yc = u0;
            float w = 0.f;
            if constexpr (LR) {
                const float* st = lg.state + 16 * (size_t)b;
                u0 = make_float3(__ldg(st), __ldg(st + 1), __ldg(st + 2));
                u1 = make_float3(__ldg(st + 3), __ldg(st + 4), __ldg(st + 5));
                u2 = make_float3(__ldg(st + 6), __ldg(st + 7), __ldg(st + 8));
                xc = make_float3(__ldg(st + 9), __ldg(st + 10), __ldg(st + 11));
                yc = make_float3(__ldg(st + 12), __ldg(st + 13), __ldg(st + 14));
                w = __ldg(lg.grad_lrmsd + b) * (RES ? 1.f : __ldg(st + 15));
            }
            auto G = [&](int k) {
                const float3 v = make_float3(__ldg(sg + 3 * k), __ldg(sg + 3 * k + 1), __ldg(sg + 3 * k + 2));
                if constexpr (!LR) return v;
                const float3 xp = f3_sub(v, xc), yp = f3_sub(R(k), yc);
                const float3 r = make_float3(yp.x - f3_dot(u0, xp), yp.y - f3_dot(u1, xp), yp.z - f3_dot(u2, xp));
                if constexpr (RES) res_acc += f3_dot(r, r);
                return f3_scale(w, r);
            };
            auto add = [&](Sum6& s, int k) {
                const float3 g = G(k);
                s.c = f3_add(s.c, f3_cross(R(k), g));
                s.g = f3_add(s.g, g);
            };
            rN = R(0);
            rCA = R(1);
            rC = R(2);
            if (j > 0) {  // C of the previous residue (the tile before holds it for the first)
                const float* pr = ap >= pc ? st_r + soff + 3 * (ap + 2 - pc) : r_in + 3 * (size_t)(ap + 2);
                rCprev = make_float3(pr[0], pr[1], pr[2]);
            }
            add(nsum, 0);
            add(all, 1);
            add(csum, 2);
            add(csum, 3);
            // side chain, entries in decreasing group order: suffix over groups
            const int nchi = s_tab.n_chi[type];
            Sum6 suf = sum6_zero();
            for (int e = nat - 5; e >= 0; --e) {
                const int w = (int)s_tab.side[type][e].w;
                const int grp = w >> 4;
                add(suf, w & 15);
                const bool last_of_group = (e == 0) || (((int)s_tab.side[type][e - 1].w >> 4) != grp);
                if (last_of_group && grp <= nchi) {
                    const int o1 = s_tab.origin[type][grp - 1];
                    const int o0 = grp >= 2 ? s_tab.origin[type][grp - 2] : 1;
                    const float3 p = R(o1);
                    const float val = f3_dot(unit3(f3_sub(p, R(o0))), f3_sub(suf.c, f3_cross(p, suf.g)));
#pragma unroll
                    for (int k = 0; k < kMaxGroups; ++k)
                        if (k == grp - 1) gchi[k] = val;
                }
            }
            all = sum6_add(sum6_add(all, suf), csum);
        }
        const Sum6 own = sum6_add(all, nsum);
        Sum6 after, total;
        block_suffix_sum6<NT>(own, s6, after, total);
        if (threadIdx.x == NT - 32) publish_suffix_agg(ws, slot0 + t, total);
        after = sum6_add(after, gather_suffix(ws, slot0, t, T));  // every warp gathers it
        // after the last wait of this tile (the chain's first tile of a fused
        // step still waits for the chain's other tiles: it asks later)
        int requested = (RES && t == 0) ? 0 : request_tile(counter);
        if (j < Lmax) {
            float gphi = 0.f, gpsi = 0.f, gomg = 0.f;
            if (in_range) {
                Sum6 x = sum6_add(csum, after);
                gpsi = f3_dot(unit3(f3_sub(rC, rCA)), f3_sub(x.c, f3_cross(rC, x.g)));
                x = sum6_add(all, after);
                gphi = f3_dot(unit3(f3_sub(rCA, rN)), f3_sub(x.c, f3_cross(rCA, x.g)));
                if (j > 0) {
                    x = sum6_add(own, after);
                    gomg = f3_dot(unit3(f3_sub(rN, rCprev)), f3_sub(x.c, f3_cross(rN, x.g)));
                }
            }
            ga[j] = gphi;
            ga[Lmax + j] = gpsi;
            ga[2 * Lmax + j] = gomg;
#pragma unroll
            for (int k = 0; k < kMaxGroups; ++k) ga[(3 + k) * Lmax + j] = gchi[k];
        }
        if (t == T - 1) {
            for (int i = min(Lmax, T * NT) + threadIdx.x; i < Lmax; i += NT)
#pragma unroll
                for (int r = 0; r < 7; ++r) ga[r * Lmax + i] = 0.f;
        }
        if constexpr (RES) {
            // this tile's residual sum, then "done" once every thread's
            // gradient writes are in
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) res_acc += __shfl_xor_sync(0xffffffffu, res_acc, o);
            if ((threadIdx.x & 31) == 0) s_res[threadIdx.x >> 5] = res_acc;
            __syncthreads();
            if (threadIdx.x == 0) {
                float tot = 0.f;
                for (int w2 = 0; w2 < NW; ++w2) tot += s_res[w2];
                ws.tres[slot0 + t] = tot;
                __threadfence();
                flag_release(ws.tdone + slot0 + t, 1);
            }
            if (t == 0) {
                // the chain's LRMSD from its tiles' residual sums (fixed order,
                // FP64), then the factor 1 / (N LRMSD) on all its gradients
                if (threadIdx.x == 0) {
                    double sum = 0.0;
                    for (int tp = 0; tp < T; ++tp) {
                        if (tp > 0) wait_flag(ws.tdone + slot0 + tp);
                        sum += (double)__ldcg(ws.tres + slot0 + tp);
                    }
                    const int n = lg.num_atoms[b] < Amax ? lg.num_atoms[b] : Amax;
                    float lr, scale;
                    lrmsd_from_sum(sum, n, lr, scale);
                    lg.lrmsd_out[b] = lr;
                    s_scale = scale;
                }
                __syncthreads();
                const float sc = s_scale;
                for (int i = threadIdx.x; i < 7 * L; i += NT) {
                    float* q = ga + (i / L) * Lmax + (i % L);
                    *q = __ldcg(q) * sc;
                }
                requested = request_tile(counter);
            }
        }
        v = next_tile(requested, &s_v);
    }
}

// ---------------------------------------------------------------------------
// K4: backward (frames recomputed from the angles and the forward's tile
// starts; tiles of a chain taken last to first).
// ---------------------------------------------------------------------------
template <int NT>
__global__ void __launch_bounds__(NT) fa_bwd_kernel(const float* __restrict__ angles,
                                                    const uint8_t* __restrict__ seq,
                                                    const int32_t* __restrict__ lengths, int B,
                                                    int Lmax, int Amax,
                                                    const float* __restrict__ grad_coords,
                                                    float* __restrict__ grad_angles, ChainWs ws,
                                                    const __grid_constant__ FaTable tab) {
    constexpr int NW = NT / 32;
    __shared__ FaTable s_tab;
    __shared__ RigidS s_rig[NW + 1];
    __shared__ int s_cnt[NW + 1];
    __shared__ float s6[6 * (NW + 1)];
    __shared__ int s_v;
    extern __shared__ float4 s_dyn[];
    float* stage = reinterpret_cast<float*>(s_dyn);  // g of the tile's atoms

    if (!ws_matches(ws, NT, B, Lmax)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) flag_status(TPL_STATUS_BAD_WORKSPACE);
        for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < (size_t)B * 7 * Lmax; i += (size_t)gridDim.x * NT)
            grad_angles[i] = 0.f;
        return;
    }
    copy_table(s_tab, tab);
    const int ntiles = ws.hdr[kHdrTiles];
    int* counter = ws.bflag + ws.slots;
    int v = take_tile(counter, &s_v);
    while (v < ntiles) {
        const int2 ct = ws.tiles[v];
        const int b = ct.x;
        const int L = clamp_length(lengths, b, Lmax);
        const int T = L > 0 ? (L + NT - 1) / NT : 1;
        const int t = T - 1 - ct.y;  // last tile first
        const int slot0 = b * ws.tmax;
        const float* ang = angles + (size_t)b * 7 * Lmax;
        const uint8_t* sq = seq + (size_t)b * Lmax;
        const float* g_in = grad_coords + (size_t)b * Amax * 3;
        float* ga = grad_angles + (size_t)b * 7 * Lmax;

        const int j = t * NT + threadIdx.x;
        const bool valid = j < L;
        const int type = residue_type(sq, j, valid);
        float sp = 0.f, cp = 1.f, ss = 0.f, cs = 1.f;
        const Rigid A = residue_transform(s_tab, ang, Lmax, j, L, sp, cp, ss, cs);
        Rigid E, Tot;
        int a0, ctot;
        block_scan_rigid_count<NT>(A, valid ? s_tab.n_atoms[type] : 0, s_rig, s_cnt, E, a0, Tot, ctot);
        int pc;
        E = rigid_mul(load_rigid_prev(ws.start + 4 * (size_t)(slot0 + t), pc), E);
        const int soff = (3 * pc) & 3;
        copy_range<NT, false>(const_cast<float*>(g_in), stage, 3 * pc, 3 * min(pc + ctot, Amax));
        __syncthreads();

        float gchi[kMaxGroups] = {0.f, 0.f, 0.f, 0.f};
        Sum6 all = sum6_zero(), nsum = sum6_zero(), csum = sum6_zero();
        float3 u_phi = make_float3(0.f, 0.f, 0.f), p_phi = u_phi, u_psi = u_phi, p_psi = u_phi;
        const bool in_range = valid && pc + a0 + s_tab.n_atoms[type] <= Amax;
        if (in_range) {
            const float* st = stage + soff + 3 * a0;
            auto gat = [&](int slot) {
                return make_float3(st[3 * slot], st[3 * slot + 1], st[3 * slot + 2]);
            };
            auto add = [](Sum6& s, float3 r, float3 g) {
                s.c = f3_add(s.c, f3_cross(r, g));
                s.g = f3_add(s.g, g);
            };
            add(nsum, E.t, gat(0));
            Rigid M1 = E;
            rigid_mul_R(M1, cp, sp, s_tab.bb.ct[1], s_tab.bb.st[1], s_tab.bb.d[1]);
            u_phi = M1.c0;
            p_phi = M1.t;
            add(all, M1.t, gat(1));
            Rigid M3 = M1;
            rigid_mul_R(M3, cs, ss, s_tab.bb.ct[2], s_tab.bb.st[2], s_tab.bb.d[2]);
            u_psi = M3.c0;
            p_psi = M3.t;
            add(csum, M3.t, gat(2));
            const float4 o = s_tab.o_r0;
            add(csum, point_apply(M3, make_float3(o.x, o.y, o.z)), gat(3));
            Rigid S = M1;
            rigid_mul_Rx(S, s_tab.rp_c, s_tab.rp_s);
            const int ng = s_tab.n_groups[type], nchi = s_tab.n_chi[type];
            float3 gu[kMaxGroups], gp[kMaxGroups];
            Sum6 gs[kMaxGroups];
            int e = 0;
#pragma unroll
            for (int k = 0; k < kMaxGroups; ++k) {
                gs[k] = sum6_zero();
                gu[k] = make_float3(0.f, 0.f, 0.f);
                gp[k] = gu[k];
                if (k < ng) {
                    float sc, cc;
                    if (k < nchi) {
                        sincosf(ang[(3 + k) * Lmax + j], &sc, &cc);
                    } else {
                        cc = s_tab.fixchi[type][k].x;
                        sc = s_tab.fixchi[type][k].y;
                    }
                    const float4 gk = s_tab.grp[type][k];
                    rigid_mul_R(S, cc, sc, gk.x, gk.y, gk.z);
                    gu[k] = S.c0;
                    gp[k] = S.t;
                    const int end = s_tab.grp_end[type][k];
                    for (; e < end; ++e) {
                        const float4 r0 = s_tab.side[type][e];
                        add(gs[k], point_apply(S, make_float3(r0.x, r0.y, r0.z)), gat((int)r0.w & 15));
                    }
                }
            }
            Sum6 suf = sum6_zero();
#pragma unroll
            for (int k = kMaxGroups - 1; k >= 0; --k) {
                suf = sum6_add(suf, gs[k]);
                if (k < nchi) gchi[k] = f3_dot(gu[k], f3_sub(suf.c, f3_cross(gp[k], suf.g)));
            }
            // all = CA + side chain + C + O (N is not downstream of phi)
            all = sum6_add(sum6_add(all, suf), csum);
        }
        const Sum6 own = sum6_add(all, nsum);
        Sum6 after, total;
        block_suffix_sum6<NT>(own, s6, after, total);
        if (threadIdx.x == NT - 32) publish_suffix_agg(ws, slot0 + t, total);
        after = sum6_add(after, gather_suffix(ws, slot0, t, T));  // every warp gathers it
        const int requested = request_tile(counter);  // after the last wait of this tile
        if (j < Lmax) {
            float gphi = 0.f, gpsi = 0.f, gomg = 0.f;
            if (in_range) {
                Sum6 x = sum6_add(csum, after);
                gpsi = f3_dot(u_psi, f3_sub(x.c, f3_cross(p_psi, x.g)));
                x = sum6_add(all, after);
                gphi = f3_dot(u_phi, f3_sub(x.c, f3_cross(p_phi, x.g)));
                if (j > 0) {
                    x = sum6_add(own, after);
                    gomg = f3_dot(E.c0, f3_sub(x.c, f3_cross(E.t, x.g)));
                }
            }
            ga[j] = gphi;
            ga[Lmax + j] = gpsi;
            ga[2 * Lmax + j] = gomg;
#pragma unroll
            for (int k = 0; k < kMaxGroups; ++k) ga[(3 + k) * Lmax + j] = gchi[k];
        }
        if (t == T - 1) {
            for (int i = min(Lmax, T * NT) + threadIdx.x; i < Lmax; i += NT)
#pragma unroll
                for (int r = 0; r < 7; ++r) ga[r * Lmax + i] = 0.f;
        }
        v = next_tile(requested, &s_v);
    }
}

// ---------------------------------------------------------------------------
// K7: plain FP64 per-chain forms (one CTA per chain, thread 0 serial).
// ---------------------------------------------------------------------------
struct Frame64 {
    double m[12];  // dense 3x4 row-major
};

__device__ void f64_identity(Frame64& f) {
    for (int k = 0; k < 12; ++k) f.m[k] = 0.0;
    f.m[0] = f.m[5] = f.m[10] = 1.0;
}

// f <- f * R(alpha, theta, d), R the dense Section 3 matrix
__device__ void f64_mul_R(Frame64& f, double alpha, double ct, double st, double d) {
    double sa, ca;
    sincos(alpha, &sa, &ca);
    const double R[12] = {ct, sa * st, ca * st, d * ct, 0.0, ca, -sa, 0.0, -st, sa * ct, ca * ct, -d * st};
    double N[12];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 4; ++c) {
            double s = (c == 3) ? f.m[4 * r + 3] : 0.0;
            for (int k = 0; k < 3; ++k) s += f.m[4 * r + k] * R[4 * k + c];
            N[4 * r + c] = s;
        }
    for (int k = 0; k < 12; ++k) f.m[k] = N[k];
}

__device__ void f64_mul_Rx(Frame64& f, double c, double s) {
    for (int r = 0; r < 3; ++r) {
        const double a1 = f.m[4 * r + 1], a2 = f.m[4 * r + 2];
        f.m[4 * r + 1] = c * a1 + s * a2;
        f.m[4 * r + 2] = -s * a1 + c * a2;
    }
}

__device__ void f64_point(const Frame64& f, const double* v, double* out) {
    for (int r = 0; r < 3; ++r)
        out[r] = f.m[4 * r] * v[0] + f.m[4 * r + 1] * v[1] + f.m[4 * r + 2] * v[2] + f.m[4 * r + 3];
}

__global__ void fa_fwd_ref64_kernel(const double* __restrict__ angles,
                                    const uint8_t* __restrict__ seq,
                                    const int32_t* __restrict__ lengths, int B, int Lmax, int Amax,
                                    double* __restrict__ coords, int32_t* __restrict__ num_atoms,
                                    const __grid_constant__ FaTableD tab) {
    const int b = blockIdx.x;
    const int L = clamp_length(lengths, b, Lmax);
    const double* ang = angles + (size_t)b * 7 * Lmax;
    const uint8_t* sq = seq + (size_t)b * Lmax;
    double* out = coords + (size_t)b * Amax * 3;
    // total atom count (every thread, for the zero fill)
    int total = 0;
    for (int j = 0; j < L; ++j) total += tab.n_atoms[sq[j] < kNumTypes ? sq[j] : kGlyCode];
    for (int i = 3 * min(total, Amax) + threadIdx.x; i < 3 * Amax; i += blockDim.x) out[i] = 0.0;
    if (threadIdx.x != 0) return;
    Frame64 M0, M1, M3, S[kMaxGroups + 1];
    f64_identity(M0);
    int a = 0;
    for (int j = 0; j < L; ++j) {
        int type = sq[j];
        if (type >= kNumTypes) {
            flag_status(TPL_STATUS_BAD_RESIDUE);
            type = kGlyCode;
        }
        M1 = M0;
        f64_mul_R(M1, ang[j], tab.bb.ct[1], tab.bb.st[1], tab.bb.d[1]);
        M3 = M1;
        f64_mul_R(M3, ang[Lmax + j], tab.bb.ct[2], tab.bb.st[2], tab.bb.d[2]);
        S[0] = M1;
        f64_mul_Rx(S[0], tab.rp_c, tab.rp_s);
        for (int k = 0; k < tab.n_groups[type]; ++k) {
            S[k + 1] = S[k];
            const double chi = (k < tab.n_chi[type]) ? ang[(3 + k) * Lmax + j] : tab.fixchi[type][k];
            f64_mul_R(S[k + 1], chi, tab.grp_ct[type][k], tab.grp_st[type][k], tab.grp_d[type][k]);
        }
        for (int t = 0; t < tab.n_atoms[type]; ++t, ++a) {
            const int g = tab.group[type][t];
            const Frame64& F = g == 0 ? M0 : (g == 1 ? M1 : (g == 2 ? M3 : S[g - 2]));
            if (a < Amax) f64_point(F, tab.r0[type][t], out + 3 * a);
        }
        if (j + 1 < L) {
            M0 = M3;
            f64_mul_R(M0, ang[2 * Lmax + j + 1], tab.bb.ct[0], tab.bb.st[0], tab.bb.d[0]);
        }
    }
    if (a > Amax) flag_status(TPL_STATUS_TOO_MANY_ATOMS);
    num_atoms[b] = a;
}

__device__ void cross_acc(double* acc, const double* r, const double* p, const double* g) {
    const double x = r[0] - p[0], y = r[1] - p[1], z = r[2] - p[2];
    acc[0] += y * g[2] - z * g[1];
    acc[1] += z * g[0] - x * g[2];
    acc[2] += x * g[1] - y * g[0];
}

__device__ double axis_dot(const double* from, const double* to, const double* acc) {
    double u[3] = {to[0] - from[0], to[1] - from[1], to[2] - from[2]};
    const double n = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    return (u[0] * acc[0] + u[1] * acc[1] + u[2] * acc[2]) / n;
}

__global__ void fa_bwd_ref64_kernel(const uint8_t* __restrict__ seq,
                                    const int32_t* __restrict__ lengths, int B, int Lmax, int Amax,
                                    const double* __restrict__ coords,
                                    const double* __restrict__ grad_coords,
                                    double* __restrict__ grad_angles,
                                    const __grid_constant__ FaTableD tab) {
    const int b = blockIdx.x;
    const int L = clamp_length(lengths, b, Lmax);
    const uint8_t* sq = seq + (size_t)b * Lmax;
    double* ga = grad_angles + (size_t)b * 7 * Lmax;
    for (int i = threadIdx.x; i < 7 * Lmax; i += blockDim.x) ga[i] = 0.0;
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double* r = coords + (size_t)b * Amax * 3;
    const double* g = grad_coords + (size_t)b * Amax * 3;
    auto type_of = [&](int j) { return sq[j] < kNumTypes ? (int)sq[j] : kGlyCode; };
    int off = 0;
    for (int j = 0; j < L; ++j) off += tab.n_atoms[type_of(j)];
    if (off > Amax) return;  // flagged by the forward
    // Sc = sum r x g and Sg = sum g over residues after the current one
    double Sc[3] = {0, 0, 0}, Sg[3] = {0, 0, 0};
    for (int j = L - 1; j >= 0; --j) {
        const int type = type_of(j);
        const int n = tab.n_atoms[type];
        off -= n;
        const double* rr = r + 3 * off;
        const double* gg = g + 3 * off;
        // chi_k: atoms of groups >= k about the axis origin(k-1) -> origin(k)
        for (int k = 0; k < tab.n_chi[type]; ++k) {
            const int o1 = tab.origin[type][k];
            const int o0 = (k == 0) ? 1 : tab.origin[type][k - 1];
            double acc[3] = {0, 0, 0};
            for (int t = 0; t < n; ++t)
                if (tab.group[type][t] >= 3 + k) cross_acc(acc, rr + 3 * t, rr + 3 * o1, gg + 3 * t);
            ga[(3 + k) * Lmax + j] = axis_dot(rr + 3 * o0, rr + 3 * o1, acc);
        }
        // Residue sums about the origin: all atoms, and C + O.
        double Ac[3] = {0, 0, 0}, Ag[3] = {0, 0, 0}, Cc[3] = {0, 0, 0}, Cg[3] = {0, 0, 0};
        const double zero[3] = {0, 0, 0};
        for (int t = 0; t < n; ++t) {
            if (t == 0) continue;  // N handled with omega
            cross_acc(Ac, rr + 3 * t, zero, gg + 3 * t);
            for (int c = 0; c < 3; ++c) Ag[c] += gg[3 * t + c];
            if (tab.group[type][t] == 2) {
                cross_acc(Cc, rr + 3 * t, zero, gg + 3 * t);
                for (int c = 0; c < 3; ++c) Cg[c] += gg[3 * t + c];
            }
        }
        auto about = [](const double* c, const double* gsum, const double* p, double* o) {
            o[0] = c[0] - (p[1] * gsum[2] - p[2] * gsum[1]);
            o[1] = c[1] - (p[2] * gsum[0] - p[0] * gsum[2]);
            o[2] = c[2] - (p[0] * gsum[1] - p[1] * gsum[0]);
        };
        double x[3], sc[3], sg[3];
        // psi: C, O and later residues about CA -> C
        for (int c = 0; c < 3; ++c) { sc[c] = Cc[c] + Sc[c]; sg[c] = Cg[c] + Sg[c]; }
        about(sc, sg, rr + 6, x);
        ga[Lmax + j] = axis_dot(rr + 3, rr + 6, x);
        // phi: all but N and later residues about N -> CA
        for (int c = 0; c < 3; ++c) { sc[c] = Ac[c] + Sc[c]; sg[c] = Ag[c] + Sg[c]; }
        about(sc, sg, rr + 3, x);
        ga[j] = axis_dot(rr, rr + 3, x);
        // add N to the residue sums
        cross_acc(Ac, rr, zero, gg);
        for (int c = 0; c < 3; ++c) Ag[c] += gg[c];
        for (int c = 0; c < 3; ++c) { Sc[c] += Ac[c]; Sg[c] += Ag[c]; }
        // omega_j (j >= 1): residues >= j about C_{j-1} -> N_j
        if (j >= 1) {
            const int nprev = tab.n_atoms[type_of(j - 1)];
            const double* cprev = r + 3 * (off - nprev + 2);
            about(Sc, Sg, rr, x);
            ga[2 * Lmax + j] = axis_dot(cprev, rr, x);
        }
    }
}

// The dynamic shared-memory limit is raised once per device and kernel, so no
// attribute call happens during a stream capture after the first launch.
template <typename K>
cudaError_t smem_attr_once(K kernel, int bytes, bool* done_per_device) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (done_per_device[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done_per_device[dev] = true;
    return e;
}

template <int NT, bool LM = false>
cudaError_t fa_fwd_t(const float* angles, const uint8_t* seq, const int32_t* lengths, int Lmax,
                     int Amax, float* coords, int32_t* num_atoms, const ChainWs& ws,
                     cudaStream_t s, const float* target = nullptr) {
    const size_t smem = fa_fwd_smem<NT>();
    static bool done[64] = {false};
    cudaError_t e = smem_attr_once(fa_fwd_kernel<NT, LM>, (int)smem, done);
    if (e != cudaSuccess) return e;
    const int grid = persistent_grid((const void*)fa_fwd_kernel<NT, LM>, NT, smem);
    fa_fwd_kernel<NT, LM><<<grid, NT, smem, s>>>(angles, seq, lengths, Lmax, Amax, coords, num_atoms,
                                                 ws, target, fa_table());
    return cudaGetLastError();
}

template <int NT, bool LR, bool RES = false>
cudaError_t fa_bwd_coords_t(const uint8_t* seq, const int32_t* lengths, int B, int Lmax, int Amax,
                            const float* coords, const float* grad_coords, float* grad_angles,
                            const ChainWs& ws, LrmsdGrad lg, cudaStream_t s) {
    const size_t smem = (size_t)(4 + NT * kMaxAtoms * 3) * sizeof(float);
    static bool done[64] = {false};
    cudaError_t e = smem_attr_once(fa_bwd_coords_kernel<NT, LR, RES>, (int)smem, done);
    if (e != cudaSuccess) return e;
    const int grid = persistent_grid((const void*)fa_bwd_coords_kernel<NT, LR, RES>, NT, smem);
    fa_bwd_coords_kernel<NT, LR, RES><<<grid, NT, smem, s>>>(seq, lengths, B, Lmax, Amax, coords, grad_coords,
                                                                grad_angles, ws, lg, fa_table());
    return cudaGetLastError();
}

template <int NT>
cudaError_t fa_bwd_t(const float* angles, const uint8_t* seq, const int32_t* lengths, int B,
                     int Lmax, int Amax, const float* grad_coords, float* grad_angles,
                     const ChainWs& ws, cudaStream_t s) {
    const size_t smem = (size_t)(4 + NT * kMaxAtoms * 3) * sizeof(float);
    static bool done[64] = {false};
    cudaError_t e = smem_attr_once(fa_bwd_kernel<NT>, (int)smem, done);
    if (e != cudaSuccess) return e;
    const int grid = persistent_grid((const void*)fa_bwd_kernel<NT>, NT, smem);
    fa_bwd_kernel<NT><<<grid, NT, smem, s>>>(angles, seq, lengths, B, Lmax, Amax, grad_coords,
                                             grad_angles, ws, fa_table());
    return cudaGetLastError();
}

}  // namespace

bool fullatom_cfg_supported(int threads) {
    return threads == 64 || threads == 128 || threads == 192 || threads == 256 || threads == 384 ||
           threads == 512;
}

cudaError_t launch_fullatom_forward(const float* angles, const uint8_t* seq,
                                    const int32_t* lengths, int B, int Lmax, int Amax,
                                    float* coords, int32_t* num_atoms, int sched_mode,
                                    void* workspace, LaunchCfg cfg, cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    ChainWs ws;
    chain_ws_layout(workspace, B, Lmax, &ws, true);
    cudaError_t e = launch_schedule(lengths, B, Lmax, cfg.threads, sched_mode, 1, ws, s);
    if (e != cudaSuccess) return e;
    switch (cfg.threads) {
        case 64: return fa_fwd_t<64>(angles, seq, lengths, Lmax, Amax, coords, num_atoms, ws, s);
        case 128: return fa_fwd_t<128>(angles, seq, lengths, Lmax, Amax, coords, num_atoms, ws, s);
        case 192: return fa_fwd_t<192>(angles, seq, lengths, Lmax, Amax, coords, num_atoms, ws, s);
        case 256: return fa_fwd_t<256>(angles, seq, lengths, Lmax, Amax, coords, num_atoms, ws, s);
        case 384: return fa_fwd_t<384>(angles, seq, lengths, Lmax, Amax, coords, num_atoms, ws, s);
        case 512: return fa_fwd_t<512>(angles, seq, lengths, Lmax, Amax, coords, num_atoms, ws, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fullatom_backward(const float* angles, const uint8_t* seq,
                                     const int32_t* lengths, int B, int Lmax, int Amax,
                                     const float* coords, const float* grad_coords,
                                     float* grad_angles, bool from_coords, void* workspace,
                                     LaunchCfg cfg, cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    ChainWs ws;
    chain_ws_layout(workspace, B, Lmax, &ws, true);
    cudaError_t e = reset_backward_flags(ws, s);
    if (e != cudaSuccess) return e;
    if (from_coords) {
        switch (cfg.threads) {
            case 64: return fa_bwd_coords_t<64, false>(seq, lengths, B, Lmax, Amax, coords, grad_coords, grad_angles, ws, LrmsdGrad{}, s);
            case 128: return fa_bwd_coords_t<128, false>(seq, lengths, B, Lmax, Amax, coords, grad_coords, grad_angles, ws, LrmsdGrad{}, s);
            case 192: return fa_bwd_coords_t<192, false>(seq, lengths, B, Lmax, Amax, coords, grad_coords, grad_angles, ws, LrmsdGrad{}, s);
            case 256: return fa_bwd_coords_t<256, false>(seq, lengths, B, Lmax, Amax, coords, grad_coords, grad_angles, ws, LrmsdGrad{}, s);
            case 384: return fa_bwd_coords_t<384, false>(seq, lengths, B, Lmax, Amax, coords, grad_coords, grad_angles, ws, LrmsdGrad{}, s);
            case 512: return fa_bwd_coords_t<512, false>(seq, lengths, B, Lmax, Amax, coords, grad_coords, grad_angles, ws, LrmsdGrad{}, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (cfg.threads) {
        case 64: return fa_bwd_t<64>(angles, seq, lengths, B, Lmax, Amax, grad_coords, grad_angles, ws, s);
        case 128: return fa_bwd_t<128>(angles, seq, lengths, B, Lmax, Amax, grad_coords, grad_angles, ws, s);
        case 192: return fa_bwd_t<192>(angles, seq, lengths, B, Lmax, Amax, grad_coords, grad_angles, ws, s);
        case 256: return fa_bwd_t<256>(angles, seq, lengths, B, Lmax, Amax, grad_coords, grad_angles, ws, s);
        case 384: return fa_bwd_t<384>(angles, seq, lengths, B, Lmax, Amax, grad_coords, grad_angles, ws, s);
        case 512: return fa_bwd_t<512>(angles, seq, lengths, B, Lmax, Amax, grad_coords, grad_angles, ws, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fullatom_forward_ref64(const double* angles, const uint8_t* seq,
                                          const int32_t* lengths, int B, int Lmax, int Amax,
                                          double* coords, int32_t* num_atoms, cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    fa_fwd_ref64_kernel<<<B, 128, 0, s>>>(angles, seq, lengths, B, Lmax, Amax, coords, num_atoms,
                                          fa_table_d());
    return cudaGetLastError();
}

cudaError_t launch_fullatom_backward_lrmsd(const uint8_t* seq, const int32_t* lengths, int B, int Lmax,
                                          int Amax, const float* coords, const float* target,
                                          const float* grad_lrmsd, const float* lrmsd_state,
                                          float* grad_angles, void* workspace, LaunchCfg cfg,
                                          cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    ChainWs ws;
    chain_ws_layout(workspace, B, Lmax, &ws, true);
    cudaError_t e = reset_backward_flags(ws, s);
    if (e != cudaSuccess) return e;
    const LrmsdGrad lg{target, lrmsd_state, grad_lrmsd};
    switch (cfg.threads) {
        case 64: return fa_bwd_coords_t<64, true>(seq, lengths, B, Lmax, Amax, coords, nullptr, grad_angles, ws, lg, s);
        case 128: return fa_bwd_coords_t<128, true>(seq, lengths, B, Lmax, Amax, coords, nullptr, grad_angles, ws, lg, s);
        case 192: return fa_bwd_coords_t<192, true>(seq, lengths, B, Lmax, Amax, coords, nullptr, grad_angles, ws, lg, s);
        case 256: return fa_bwd_coords_t<256, true>(seq, lengths, B, Lmax, Amax, coords, nullptr, grad_angles, ws, lg, s);
        case 384: return fa_bwd_coords_t<384, true>(seq, lengths, B, Lmax, Amax, coords, nullptr, grad_angles, ws, lg, s);
        case 512: return fa_bwd_coords_t<512, true>(seq, lengths, B, Lmax, Amax, coords, nullptr, grad_angles, ws, lg, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fullatom_lrmsd_forward(const float* angles, const uint8_t* seq, const int32_t* lengths,
                                          const float* target, int B, int Lmax, int Amax, float* coords,
                                          int32_t* num_atoms, int sched_mode, void* workspace, LaunchCfg cfg,
                                          cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    ChainWs ws;
    chain_ws_layout(workspace, B, Lmax, &ws, true, true);
    cudaError_t e = launch_schedule(lengths, B, Lmax, cfg.threads, sched_mode, 1, ws, s);
    if (e != cudaSuccess) return e;
    switch (cfg.threads) {
        case 64: e = fa_fwd_t<64, true>(angles, seq, lengths, Lmax, Amax, coords, num_atoms, ws, s, target); break;
        case 128: e = fa_fwd_t<128, true>(angles, seq, lengths, Lmax, Amax, coords, num_atoms, ws, s, target); break;
        case 192: e = fa_fwd_t<192, true>(angles, seq, lengths, Lmax, Amax, coords, num_atoms, ws, s, target); break;
        case 256: e = fa_fwd_t<256, true>(angles, seq, lengths, Lmax, Amax, coords, num_atoms, ws, s, target); break;
        case 384: e = fa_fwd_t<384, true>(angles, seq, lengths, Lmax, Amax, coords, num_atoms, ws, s, target); break;
        case 512: e = fa_fwd_t<512, true>(angles, seq, lengths, Lmax, Amax, coords, num_atoms, ws, s, target); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return launch_lrmsd_solve_tiles(coords, target, num_atoms, B, Amax, ws.tmom, ws.tmax, lengths, cfg.threads,
                                    Lmax, ws.lstate, s);
}

cudaError_t launch_fullatom_lrmsd_backward(const uint8_t* seq, const int32_t* lengths, const float* coords,
                                           const float* target, const float* grad_lrmsd,
                                           const int32_t* num_atoms, float* lrmsd, int B, int Lmax, int Amax,
                                           float* grad_angles, void* workspace, LaunchCfg cfg, cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    ChainWs ws;
    chain_ws_layout(workspace, B, Lmax, &ws, true, true);
    cudaError_t e = reset_backward_flags(ws, s);
    if (e != cudaSuccess) return e;
    LrmsdGrad lg{target, ws.lstate, grad_lrmsd, lrmsd, num_atoms};
    switch (cfg.threads) {
        case 64: return fa_bwd_coords_t<64, true, true>(seq, lengths, B, Lmax, Amax, coords, nullptr, grad_angles, ws, lg, s);
        case 128: return fa_bwd_coords_t<128, true, true>(seq, lengths, B, Lmax, Amax, coords, nullptr, grad_angles, ws, lg, s);
        case 192: return fa_bwd_coords_t<192, true, true>(seq, lengths, B, Lmax, Amax, coords, nullptr, grad_angles, ws, lg, s);
        case 256: return fa_bwd_coords_t<256, true, true>(seq, lengths, B, Lmax, Amax, coords, nullptr, grad_angles, ws, lg, s);
        case 384: return fa_bwd_coords_t<384, true, true>(seq, lengths, B, Lmax, Amax, coords, nullptr, grad_angles, ws, lg, s);
        case 512: return fa_bwd_coords_t<512, true, true>(seq, lengths, B, Lmax, Amax, coords, nullptr, grad_angles, ws, lg, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fullatom_backward_ref64(const double* angles, const uint8_t* seq,
                                           const int32_t* lengths, int B, int Lmax, int Amax,
                                           const double* coords, const double* grad_coords,
                                           double* grad_angles, cudaStream_t s) {
    (void)angles;
    if (B == 0) return cudaSuccess;
    fa_bwd_ref64_kernel<<<B, 128, 0, s>>>(seq, lengths, B, Lmax, Amax, coords, grad_coords,
                                          grad_angles, fa_table_d());
    return cudaGetLastError();
}

}  // namespace tpl
