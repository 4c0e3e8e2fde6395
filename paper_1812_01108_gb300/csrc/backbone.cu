// Backbone model of the paper (Section 3) on sm_103a.
//
// K1 bb_fwd_kernel: persistent CTAs take tiles of NT*K residues from a work
// list.  Each thread owns K consecutive residues (3K transforms: R(omega_j)
// R(phi_j) R(psi_j), R_0 = I), composes them serially in registers, then the
// CTA runs an exclusive parallel prefix scan over the per-thread rigid
// transforms; the frame at the tile start is the product of the earlier
// tiles' aggregates (bounded look-back, re-orthonormalised).  Coordinates are
// staged in shared memory and written with coalesced 16-byte stores.
//
// K2 bb_bwd_kernel: the adjoint of Eq. 2 as a reverse suffix scan.  With u_i
// the x axis of M_i (bond i-1 -> i) and p_i = r_i,
//   dL/dalpha_i = u_i . (sum_{k>=i} r_k x g_k - p_i x sum_{k>=i} g_k),
// which equals the paper's sum_k g_k . (M_{i-1} dR_i M_i^{-1} r_k).  Tiles of a
// chain are taken last to first; the sum over later tiles comes from a
// bounded look-back.  Frames are recomputed from the angles and the forward's
// tile-start frames (RECOMPUTE) or read from the forward's coordinates
// (FROM_COORDS).
#include "kernels.h"
#include "tables.h"
#include "sched.cuh"
#include "tpl_common.cuh"
#include "bulk.cuh"
#include "lrmsd_solve.cuh"

namespace tpl {

namespace {

template <int K>
__device__ __forceinline__ void load_row(const float* __restrict__ row, int j0, int Lmax,
                                         float (&v)[K]) {
    if (j0 < Lmax) {
        if constexpr (K == 4) {
            float4 q = __ldg(reinterpret_cast<const float4*>(row + j0));
            v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
        } else if constexpr (K == 2) {
            float2 q = __ldg(reinterpret_cast<const float2*>(row + j0));
            v[0] = q.x; v[1] = q.y;
        } else {
            v[0] = __ldg(row + j0);
        }
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = 0.f;
    }
}

template <int K>
__device__ __forceinline__ void store_row(float* row, int j0, int Lmax, const float (&v)[K]) {
    if (j0 >= Lmax) return;
    if constexpr (K == 4) {
        *reinterpret_cast<float4*>(row + j0) = make_float4(v[0], v[1], v[2], v[3]);
    } else if constexpr (K == 2) {
        *reinterpret_cast<float2*>(row + j0) = make_float2(v[0], v[1]);
    } else {
        row[j0] = v[0];
    }
}

// 9K consecutive floats (K residues x 3 atoms x xyz) at p, 16/8/4-byte aligned for K = 4/2/1.
template <int K>
__device__ __forceinline__ void load_atoms(const float* __restrict__ p, bool ok, float (&v)[9 * K]) {
    if (!ok) {
#pragma unroll
        for (int i = 0; i < 9 * K; ++i) v[i] = 0.f;
        return;
    }
    if constexpr (K == 4) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            float4 q = __ldg(reinterpret_cast<const float4*>(p) + i);
            v[4 * i] = q.x; v[4 * i + 1] = q.y; v[4 * i + 2] = q.z; v[4 * i + 3] = q.w;
        }
    } else if constexpr (K == 2) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            float2 q = __ldg(reinterpret_cast<const float2*>(p) + i);
            v[2 * i] = q.x; v[2 * i + 1] = q.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) v[i] = __ldg(p + i);
    }
}

template <int K>
__device__ __forceinline__ void store_stage(float* s, const float (&v)[9 * K]) {
    if constexpr (K == 4) {
#pragma unroll
        for (int i = 0; i < 9; ++i)
            reinterpret_cast<float4*>(s)[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    } else if constexpr (K == 2) {
#pragma unroll
        for (int i = 0; i < 9; ++i) reinterpret_cast<float2*>(s)[i] = make_float2(v[2 * i], v[2 * i + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) s[i] = v[i];
    }
}

// Angle row read by the transform placing atom k of a residue: N <- omega (2),
// CA <- phi (0), C <- psi (1).
__device__ __forceinline__ constexpr int row_of(int k) { return k == 0 ? 2 : (k == 1 ? 0 : 1); }

// Product of the 3K transforms of a thread's residues j0 .. j0+K-1 (R_0 = I;
// residues past L are identities) and the local atom positions it places;
// WITH_O: also each residue's carbonyl O, rigid in the frame of C after psi.
template <int K, bool WITH_O = false>
__device__ __forceinline__ Rigid thread_product(const float* __restrict__ ang, int j0, int L, int Lmax,
                                                const BackboneConst& bc, float3 (&pos)[3 * K],
                                                float3* opos = nullptr) {
    float a[3][K];
    load_row<K>(ang, j0, Lmax, a[0]);
    load_row<K>(ang + Lmax, j0, Lmax, a[1]);
    load_row<K>(ang + 2 * Lmax, j0, Lmax, a[2]);
    Rigid A = rigid_identity();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int j = j0 + k;
#pragma unroll
        for (int at = 0; at < 3; ++at) {
            if (j < L && (j > 0 || at > 0)) {
                float s, c;
                sincosf(a[row_of(at)][k], &s, &c);
                rigid_mul_R(A, c, s, bc.ct[at], bc.st[at], bc.d[at]);
            }
            pos[3 * k + at] = A.t;
        }
        if constexpr (WITH_O) opos[k] = point_apply(A, make_float3(bc.o[0], bc.o[1], bc.o[2]));
    }
    if (j0 < L) rigid_reortho(A);  // the scan composes orthonormal operands
    return A;
}

// A thread's K residues of carbonyl O (3K floats from residue j0 of a row of
// [Lmax][3]), zeros past L; 16/8/4-byte stores for K = 4/2/1.
template <int K>
__device__ __forceinline__ void store_o(float* __restrict__ row, int j0, int L, int Lmax, const Rigid& E,
                                        const float3 (&opos)[K]) {
    if (j0 >= Lmax) return;
    float v[3 * K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float3 r = point_apply(E, opos[k]);
        const bool ok = j0 + k < L;
        v[3 * k] = ok ? r.x : 0.f;
        v[3 * k + 1] = ok ? r.y : 0.f;
        v[3 * k + 2] = ok ? r.z : 0.f;
    }
    float* p = row + 3 * (size_t)j0;
    if constexpr (K == 4) {
#pragma unroll
        for (int i = 0; i < 3; ++i)
            reinterpret_cast<float4*>(p)[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    } else if constexpr (K == 2) {
#pragma unroll
        for (int i = 0; i < 3; ++i) reinterpret_cast<float2*>(p)[i] = make_float2(v[2 * i], v[2 * i + 1]);
    } else {
        p[0] = v[0]; p[1] = v[1]; p[2] = v[2];
    }
}

// K floats of O (3K) of a thread's residues, zeros when !ok.
template <int K>
__device__ __forceinline__ void load_o(const float* __restrict__ p, bool ok, float (&v)[3 * K]) {
    if (!ok) {
#pragma unroll
        for (int i = 0; i < 3 * K; ++i) v[i] = 0.f;
        return;
    }
    if constexpr (K == 4) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float4 q = __ldg(reinterpret_cast<const float4*>(p) + i);
            v[4 * i] = q.x; v[4 * i + 1] = q.y; v[4 * i + 2] = q.z; v[4 * i + 3] = q.w;
        }
    } else if constexpr (K == 2) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float2 q = __ldg(reinterpret_cast<const float2*>(p) + i);
            v[2 * i] = q.x; v[2 * i + 1] = q.y;
        }
    } else {
        v[0] = __ldg(p); v[1] = __ldg(p + 1); v[2] = __ldg(p + 2);
    }
}

// ---------------------------------------------------------------------------
// K1: forward.  One tile (NT*K residues) per step of a persistent CTA.
// WITH_O: also the carbonyl O of every residue into o_coords [B][Lmax][3].
// ---------------------------------------------------------------------------
template <int NT, int K, bool WITH_O = false>
__global__ void __launch_bounds__(NT, 768 / NT) bb_fwd_kernel(const float* __restrict__ angles,
                                                    const int32_t* __restrict__ lengths, int Lmax,
                                                    float* __restrict__ coords, ChainWs ws,
                                                    BackboneConst bc, float* __restrict__ o_coords) {
    constexpr int NW = NT / 32;
    constexpr int TILE = NT * K;
    __shared__ RigidS s_rig[NW + 1];
    __shared__ int s_cnt[NW + 1];
    __shared__ int s_v;
    __shared__ __align__(16) float s_out[TILE * 9];
    __shared__ PackS s_pack;

    const int ntiles = ws.hdr[kHdrTiles];
    int v = take_tile(ws.hdr + kHdrFwdNext, &s_v);
    while (v < ntiles) {
        const int2 ct = ws.tiles[v];
        // the previous entry's bulk store has read the stage before it is refilled
        // (the entry's block scan barriers order this before every stage write)
        if (threadIdx.x == 0) bulk_store_wait_read();
        if (ct.x < 0) {
            // a pack of whole short chains: segmented scan, no look-back
            const int m = ct.y;
            load_pack<K>(ws, lengths, Lmax, -1 - ct.x, m, s_pack);
            const int slot = threadIdx.x * K;
            const int ci = pack_member(s_pack, m, slot);
            const int b = ci >= 0 ? s_pack.b[ci] : 0;
            const int L = ci >= 0 ? s_pack.len[ci] : 0;
            const int j0 = ci >= 0 ? slot - s_pack.off[ci] : Lmax;  // Lmax: nothing to load
            float3 pos[3 * K], opos[K];
            const Rigid A = thread_product<K, WITH_O>(angles + (size_t)b * 3 * Lmax, j0, L, Lmax, bc, pos, opos);
            const Rigid E = block_seg_scan_rigid<NT>(A, ci < 0 || j0 == 0, s_rig, s_cnt);
            const int requested = request_tile(ws.hdr + kHdrFwdNext);
            if constexpr (WITH_O) store_o<K>(o_coords + (size_t)b * 3 * Lmax, j0, L, Lmax, E, opos);
            float vv[9 * K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
#pragma unroll
                for (int at = 0; at < 3; ++at) {
                    const float3 r = point_apply(E, pos[3 * k + at]);
                    vv[9 * k + 3 * at + 0] = r.x;
                    vv[9 * k + 3 * at + 1] = r.y;
                    vv[9 * k + 3 * at + 2] = r.z;
                }
            }
            store_stage<K>(s_out + threadIdx.x * 9 * K, vv);
            fence_proxy_async();  // the stage writes, before the bulk store reads them
            __syncthreads();
            // each chain's whole row: its atoms from the stage (16-byte copies when
            // the stage offset allows), the float4 that straddles the end, zeros
            for (int i = 0; i < m; ++i) {
                const int n9 = 9 * s_pack.len[i], o9 = 9 * s_pack.off[i];
                float4* dst = reinterpret_cast<float4*>(coords + (size_t)s_pack.b[i] * 9 * Lmax);
                const int full = n9 >> 2;
                if (full > 0 && ((smem_addr(s_out + o9) | (unsigned)reinterpret_cast<uintptr_t>(dst)) & 15u) == 0u) {
                    // one bulk store (TMA engine) that runs on while the CTA goes on
                    if (threadIdx.x == 0) bulk_store(reinterpret_cast<float*>(dst), s_out + o9, 16u * (unsigned)full);
                } else if ((o9 & 3) == 0) {
                    const float4* src = reinterpret_cast<const float4*>(s_out + o9);
                    for (int q = threadIdx.x; q < full; q += NT) dst[q] = src[q];
                } else {
                    for (int q = threadIdx.x; q < full; q += NT) {
                        const float* e = s_out + o9 + 4 * q;
                        dst[q] = make_float4(e[0], e[1], e[2], e[3]);
                    }
                }
                if ((n9 & 3) && threadIdx.x == 0) {
                    const int e = 4 * full;
                    dst[full] = make_float4(s_out[o9 + e], e + 1 < n9 ? s_out[o9 + e + 1] : 0.f,
                                            e + 2 < n9 ? s_out[o9 + e + 2] : 0.f, 0.f);
                }
                const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
                if (!(ws.flags & TPL_FLAG_PADDING_ZEROED)) {
                    for (int q = ((n9 + 3) >> 2) + threadIdx.x; q < 9 * Lmax / 4; q += NT) dst[q] = z;
                    if constexpr (WITH_O) {  // O rows past the chain's slots
                        float* orow = o_coords + (size_t)s_pack.b[i] * 3 * Lmax;
                        for (int q = 3 * (s_pack.off[i + 1] - s_pack.off[i]) + threadIdx.x; q < 3 * Lmax; q += NT)
                            orow[q] = 0.f;
                    }
                }
            }
            v = next_tile(requested, &s_v);
            continue;
        }
        const int b = ct.x, t = ct.y;
        const int L = clamp_length(lengths, b, Lmax);
        const int T = L > 0 ? (L + TILE - 1) / TILE : 1;
        const int slot0 = b * ws.tmax;
        const float* ang = angles + (size_t)b * 3 * Lmax;
        float* out = coords + (size_t)b * 9 * Lmax;
        const int tile0 = t * TILE;
        const int j0 = tile0 + threadIdx.x * K;
        float3 pos[3 * K], opos[K];
        const Rigid A = thread_product<K, WITH_O>(ang, j0, L, Lmax, bc, pos, opos);
        Rigid E, Tot;
        int ce, ctot;
        block_scan_rigid_count<NT>(A, 0, s_rig, s_cnt, E, ce, Tot, ctot);
        if (threadIdx.x == NT - 32) publish_prefix_agg(ws, slot0 + t, Tot, 0);
        int pc;
        const Rigid P = gather_prefix(ws, slot0, t, pc);  // every warp gathers it
        // the next tile is requested only now: a CTA that holds a tile it has
        // not started never waits, so no wait can chain through held tiles
        const int requested = request_tile(ws.hdr + kHdrFwdNext);
        if (threadIdx.x == 0) store_rigid_g(ws.start + 4 * (size_t)(slot0 + t), P, 0);
        E = rigid_mul(P, E);
        if constexpr (WITH_O) store_o<K>(o_coords + (size_t)b * 3 * Lmax, j0, L, Lmax, E, opos);
        float vv[9 * K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const bool valid = j0 + k < L;
#pragma unroll
            for (int at = 0; at < 3; ++at) {
                const float3 r = point_apply(E, pos[3 * k + at]);
                vv[9 * k + 3 * at + 0] = valid ? r.x : 0.f;
                vv[9 * k + 3 * at + 1] = valid ? r.y : 0.f;
                vv[9 * k + 3 * at + 2] = valid ? r.z : 0.f;
            }
        }
        store_stage<K>(s_out + threadIdx.x * 9 * K, vv);
        fence_proxy_async();  // the stage writes, before the bulk store reads them
        __syncthreads();
        // with the padding kept zero by the caller, the stores stop at the
        // chain's last residue (rounded up to 4 residues: the stage holds
        // zeros past it)
        const int nres = (ws.flags & TPL_FLAG_PADDING_ZEROED) ? min(TILE, (L - tile0 + 3) & ~3)
                                                             : min(TILE, Lmax - tile0);  // multiple of 4
        float* dst = out + 9 * (size_t)tile0;  // 16-byte aligned: tile0 and nres are multiples of 4
        if (nres > 0 && ((smem_addr(s_out) | (unsigned)reinterpret_cast<uintptr_t>(dst)) & 15u) == 0u) {
            if (threadIdx.x == 0) bulk_store(dst, s_out, 36u * (unsigned)nres);  // runs on into the next tile
        } else {
            const float4* src = reinterpret_cast<const float4*>(s_out);
            for (int i = threadIdx.x; i < nres * 9 / 4; i += NT) reinterpret_cast<float4*>(dst)[i] = src[i];
        }
        if (t == T - 1 && !(ws.flags & TPL_FLAG_PADDING_ZEROED)) {  // zero the residues past the last tile
            float4* o4 = reinterpret_cast<float4*>(out);
            for (int i = min(Lmax, T * TILE) * 9 / 4 + threadIdx.x; i < Lmax * 9 / 4; i += NT)
                o4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            if constexpr (WITH_O) {
                float* orow = o_coords + (size_t)b * 3 * Lmax;
                for (int i = 3 * min(Lmax, T * TILE) + threadIdx.x; i < 3 * Lmax; i += NT) orow[i] = 0.f;
            }
        }
        v = next_tile(requested, &s_v);
    }
    if (threadIdx.x == 0) bulk_store_wait_all();  // the last stores are in global memory
}

// Local product of a thread's K residues (no positions), sin/cos cached.
template <int K>
__device__ __forceinline__ Rigid local_product(const float* ang, int j0, int L, int Lmax,
                                               const BackboneConst& bc, float (&sn)[3 * K],
                                               float (&cs)[3 * K]) {
    float a[3][K];
    load_row<K>(ang, j0, Lmax, a[0]);
    load_row<K>(ang + Lmax, j0, Lmax, a[1]);
    load_row<K>(ang + 2 * Lmax, j0, Lmax, a[2]);
    Rigid A = rigid_identity();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int j = j0 + k;
#pragma unroll
        for (int at = 0; at < 3; ++at) {
            sincosf(a[row_of(at)][k], &sn[3 * k + at], &cs[3 * k + at]);
            if (j < L && (j > 0 || at > 0))
                rigid_mul_R(A, cs[3 * k + at], sn[3 * k + at], bc.ct[at], bc.st[at], bc.d[at]);
        }
    }
    if (j0 < L) rigid_reortho(A);  // as in the forward: identical frames
    return A;
}

__device__ __forceinline__ bool ws_matches(const ChainWs& ws, int tile, int B, int Lmax) {
    return ws.hdr[kHdrMagic] == kWsMagic && ws.hdr[kHdrTile] == tile && ws.hdr[kHdrB] == B &&
           ws.hdr[kHdrLmax] == Lmax;
}

// ---------------------------------------------------------------------------
// K2: backward.  Tiles of a chain are taken last to first; frames are rebuilt
// from the angles and the forward's tile-start frames (RECOMPUTE) or read from
// the forward's coordinates (FROM_COORDS).
// ---------------------------------------------------------------------------
// LR (with FROM_COORDS): the coordinate gradient is the LRMSD gradient,
// formed from the coordinates, the target and the LRMSD state.
// RES (with LR, the training step's chains of more than one tile): the LRMSD
// gradient is formed without its 1 / (N LRMSD) factor, each tile also sums
// its atoms' squared residuals, and the chain's first tile -- taken last --
// waits for the chain's other tiles, forms LRMSD (FP64 over the tiles) and
// rescales the chain's angle gradients.  Entries of whole chains are skipped
// (the step kernel has done them).
// WITH_O (not with LR): the carbonyl O atoms are among the moved atoms, O_j
// after C_j (moved by every angle up to psi_j), with gradient grad_o and, for
// FROM_COORDS, positions o_coords ([B][Lmax][3] each).
template <int NT, int K, bool FROM_COORDS, bool LR, bool RES = false, bool WITH_O = false>
__global__ void __launch_bounds__(NT, 512 / NT) bb_bwd_kernel(const float* __restrict__ angles,
                                                    const int32_t* __restrict__ lengths, int B,
                                                    int Lmax, const float* __restrict__ coords,
                                                    const float* __restrict__ grad_coords,
                                                    float* __restrict__ grad_angles, ChainWs ws,
                                                    LrmsdGrad lg, BackboneConst bc,
                                                    const float* __restrict__ o_coords = nullptr,
                                                    const float* __restrict__ grad_o = nullptr) {
    static_assert(FROM_COORDS || !LR, "the LRMSD gradient needs the coordinates");
    static_assert(!(LR && WITH_O), "the LRMSD gradient covers N, CA and C only");
    static_assert(LR || !RES, "the residual sums belong to the LRMSD gradient");
    __shared__ float s_res[NT / 32];
    __shared__ float s_scale;
    constexpr int NW = NT / 32;
    constexpr int TILE = NT * K;
    __shared__ RigidS s_rig[NW + 1];
    __shared__ int s_cnt[NW + 1];
    __shared__ float s6[6 * (NW + 1)];
    __shared__ int s_v;
    __shared__ PackS s_pack;

    const bool ok = ws_matches(ws, TILE, B, Lmax);
    if (!ok) {
        if (blockIdx.x == 0 && threadIdx.x == 0) flag_status(TPL_STATUS_BAD_WORKSPACE);
        for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < (size_t)B * 3 * Lmax; i += (size_t)gridDim.x * NT)
            grad_angles[i] = 0.f;
        return;
    }
    const int ntiles = ws.hdr[kHdrTiles];
    int* counter = ws.bflag + ws.slots;
    int v = take_tile(counter, &s_v);
    while (v < ntiles) {
        const int2 ct = ws.tiles[v];
        // a pack of whole short chains (segmented scans, no look-back) or one
        // tile of a chain, the chain's tiles taken last to first
        const bool pack = ct.x < 0;
        int b, L, j0, t = 0, T = 1, m = 0;
        bool head = false, tail = false;
        if (pack) {
            m = ct.y;
            load_pack<K>(ws, lengths, Lmax, -1 - ct.x, m, s_pack);
            const int slot = threadIdx.x * K;
            const int ci = pack_member(s_pack, m, slot);
            b = ci >= 0 ? s_pack.b[ci] : 0;
            L = ci >= 0 ? s_pack.len[ci] : 0;
            j0 = ci >= 0 ? slot - s_pack.off[ci] : Lmax;  // Lmax: nothing to load or store
            head = ci < 0 || j0 == 0;
            tail = ci < 0 || slot + K >= s_pack.off[ci + 1];
        } else {
            b = ct.x;
            L = clamp_length(lengths, b, Lmax);
            T = L > 0 ? (L + TILE - 1) / TILE : 1;
            t = T - 1 - ct.y;
            j0 = t * TILE + threadIdx.x * K;
        }
        if constexpr (RES) {
            if (pack || T == 1) {  // a whole chain: done by the step kernel
                v = next_tile(request_tile(counter), &s_v);
                continue;
            }
        }
        const int slot0 = b * ws.tmax;
        const float* ang = angles + (size_t)b * 3 * Lmax;
        const float* g_in = grad_coords + (size_t)b * 9 * Lmax;
        float res_acc = 0.f;  // RES: this thread's squared residuals
        int requested = 0;
        float* ga = grad_angles + (size_t)b * 3 * Lmax;

        float g[9 * K];
        if constexpr (LR) {
            float x[9 * K], y[9 * K];
            const size_t o = (size_t)b * 9 * Lmax + 9 * (size_t)min(j0, Lmax - K);
            load_atoms<K>(lg.target + o, j0 < Lmax, x);
            load_atoms<K>(coords + o, j0 < Lmax, y);
            const float* st = lg.state + 16 * (size_t)b;
            const float3 u0 = make_float3(__ldg(st), __ldg(st + 1), __ldg(st + 2));
            const float3 u1 = make_float3(__ldg(st + 3), __ldg(st + 4), __ldg(st + 5));
            const float3 u2 = make_float3(__ldg(st + 6), __ldg(st + 7), __ldg(st + 8));
            const float3 xc = make_float3(__ldg(st + 9), __ldg(st + 10), __ldg(st + 11));
            const float3 yc = make_float3(__ldg(st + 12), __ldg(st + 13), __ldg(st + 14));
            const float w = __ldg(lg.grad_lrmsd + b) * (RES ? 1.f : __ldg(st + 15));
#pragma unroll
            for (int q = 0; q < 3 * K; ++q) {
                const float3 xp = f3_sub(make_float3(x[3 * q], x[3 * q + 1], x[3 * q + 2]), xc);
                const float3 yp = f3_sub(make_float3(y[3 * q], y[3 * q + 1], y[3 * q + 2]), yc);
                const float3 d = make_float3(yp.x - f3_dot(u0, xp), yp.y - f3_dot(u1, xp), yp.z - f3_dot(u2, xp));
                g[3 * q] = w * d.x;
                g[3 * q + 1] = w * d.y;
                g[3 * q + 2] = w * d.z;
                if (RES && j0 + q / 3 < L) res_acc += f3_dot(d, d);
            }
        } else {
            load_atoms<K>(g_in + 9 * (size_t)min(j0, Lmax - K), j0 < Lmax, g);
        }
        float go[WITH_O ? 3 * K : 1];  // the thread's O gradients
        if constexpr (WITH_O) load_o<K>(grad_o + (size_t)b * 3 * Lmax + 3 * (size_t)min(j0, Lmax - K), j0 < Lmax, go);
        Sum6 own = sum6_zero();
        float gr[3][K];
        // (sum r x g, sum g) over the later atoms of the chain, from the block
        // suffix scan and, for a tile, the look-back over the chain's later tiles
        auto later_sums = [&](const Sum6& x) {
            Sum6 after, total;
            if (pack) {
                after = block_seg_suffix_sum6<NT>(x, tail, s6, s_cnt);
            } else {
                block_suffix_sum6<NT>(x, s6, after, total);
                if (threadIdx.x == NT - 32) publish_suffix_agg(ws, slot0 + t, total);
                after = sum6_add(after, gather_suffix(ws, slot0, t, T));  // every warp gathers it
            }
            // after the last wait of this tile (the step's first tile waits
            // once more, at its end, and asks then)
            if (!(RES && t == 0)) requested = request_tile(counter);
            return after;
        };
        if constexpr (!FROM_COORDS) {
            float sn[3 * K], cs[3 * K];
            Rigid A = local_product<K>(ang, j0, L, Lmax, bc, sn, cs);
            Rigid E;
            if (pack) {
                E = block_seg_scan_rigid<NT>(A, head, s_rig, s_cnt);
            } else {
                Rigid Tot;
                int ce, ctot;
                block_scan_rigid_count<NT>(A, 0, s_rig, s_cnt, E, ce, Tot, ctot);
                int pc;
                E = rigid_mul(load_rigid_prev(ws.start + 4 * (size_t)(slot0 + t), pc), E);
            }
            // pass 1: per-thread totals of (r x g, g)
            Rigid M = E;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int j = j0 + k;
                if (j < L) {
#pragma unroll
                    for (int at = 0; at < 3; ++at) {
                        if (j > 0 || at > 0)
                            rigid_mul_R(M, cs[3 * k + at], sn[3 * k + at], bc.ct[at], bc.st[at], bc.d[at]);
                        const float3 gi = make_float3(g[9 * k + 3 * at], g[9 * k + 3 * at + 1], g[9 * k + 3 * at + 2]);
                        own.c = f3_add(own.c, f3_cross(M.t, gi));
                        own.g = f3_add(own.g, gi);
                    }
                    if constexpr (WITH_O) {  // M: the frame of C after psi
                        const float3 ro = point_apply(M, make_float3(bc.o[0], bc.o[1], bc.o[2]));
                        const float3 gi = make_float3(go[3 * k], go[3 * k + 1], go[3 * k + 2]);
                        own.c = f3_add(own.c, f3_cross(ro, gi));
                        own.g = f3_add(own.g, gi);
                    }
                }
            }
            // pass 2: gradients, atoms ascending with S = sum over atoms >= current
            Sum6 S = sum6_add(later_sums(own), own);
            M = E;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int j = j0 + k;
#pragma unroll
                for (int at = 0; at < 3; ++at) {
                    float val = 0.f;
                    if (j < L) {
                        const bool has_angle = (j > 0 || at > 0);
                        if (has_angle)
                            rigid_mul_R(M, cs[3 * k + at], sn[3 * k + at], bc.ct[at], bc.st[at], bc.d[at]);
                        const float3 gi = make_float3(g[9 * k + 3 * at], g[9 * k + 3 * at + 1], g[9 * k + 3 * at + 2]);
                        if (has_angle) val = f3_dot(M.c0, f3_sub(S.c, f3_cross(M.t, S.g)));
                        S.c = f3_sub(S.c, f3_cross(M.t, gi));
                        S.g = f3_sub(S.g, gi);
                    }
                    gr[row_of(at)][k] = val;
                }
                if constexpr (WITH_O) {  // O_j, after C_j
                    if (j < L) {
                        const float3 ro = point_apply(M, make_float3(bc.o[0], bc.o[1], bc.o[2]));
                        const float3 gi = make_float3(go[3 * k], go[3 * k + 1], go[3 * k + 2]);
                        S.c = f3_sub(S.c, f3_cross(ro, gi));
                        S.g = f3_sub(S.g, gi);
                    }
                }
            }
        } else {
            const float* r_in = coords + (size_t)b * 9 * Lmax;
            float r[9 * K];
            load_atoms<K>(r_in + 9 * (size_t)min(j0, Lmax - K), j0 < Lmax, r);
            float3 prev = make_float3(0.f, 0.f, 0.f);
            if (j0 > 0 && j0 < Lmax) prev = make_float3(r_in[9 * j0 - 3], r_in[9 * j0 - 2], r_in[9 * j0 - 1]);
#pragma unroll
            for (int q = 0; q < 3 * K; ++q) {
                if (j0 + q / 3 < L) {
                    const float3 ri = make_float3(r[3 * q], r[3 * q + 1], r[3 * q + 2]);
                    const float3 gi = make_float3(g[3 * q], g[3 * q + 1], g[3 * q + 2]);
                    own.c = f3_add(own.c, f3_cross(ri, gi));
                    own.g = f3_add(own.g, gi);
                }
            }
            float ro[WITH_O ? 3 * K : 1];
            if constexpr (WITH_O) {
                load_o<K>(o_coords + (size_t)b * 3 * Lmax + 3 * (size_t)min(j0, Lmax - K), j0 < Lmax, ro);
#pragma unroll
                for (int k = 0; k < K; ++k)
                    if (j0 + k < L) {
                        const float3 oi = make_float3(ro[3 * k], ro[3 * k + 1], ro[3 * k + 2]);
                        const float3 gi = make_float3(go[3 * k], go[3 * k + 1], go[3 * k + 2]);
                        own.c = f3_add(own.c, f3_cross(oi, gi));
                        own.g = f3_add(own.g, gi);
                    }
            }
            Sum6 S = sum6_add(later_sums(own), own);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int j = j0 + k;
#pragma unroll
                for (int at = 0; at < 3; ++at) {
                    const int q = 3 * k + at;
                    float val = 0.f;
                    const float3 ri = make_float3(r[3 * q], r[3 * q + 1], r[3 * q + 2]);
                    if (j < L) {
                        const float3 gi = make_float3(g[3 * q], g[3 * q + 1], g[3 * q + 2]);
                        if (j > 0 || at > 0) {
                            float3 u = f3_sub(ri, prev);
                            u = f3_scale(rsqrtf(f3_dot(u, u)), u);
                            val = f3_dot(u, f3_sub(S.c, f3_cross(ri, S.g)));
                        }
                        S.c = f3_sub(S.c, f3_cross(ri, gi));
                        S.g = f3_sub(S.g, gi);
                    }
                    prev = ri;
                    gr[row_of(at)][k] = val;
                }
                if constexpr (WITH_O) {  // O_j, after C_j
                    if (j < L) {
                        const float3 oi = make_float3(ro[3 * k], ro[3 * k + 1], ro[3 * k + 2]);
                        const float3 gi = make_float3(go[3 * k], go[3 * k + 1], go[3 * k + 2]);
                        S.c = f3_sub(S.c, f3_cross(oi, gi));
                        S.g = f3_sub(S.g, gi);
                    }
                }
            }
        }
        store_row<K>(ga, j0, Lmax, gr[0]);
        store_row<K>(ga + Lmax, j0, Lmax, gr[1]);
        store_row<K>(ga + 2 * Lmax, j0, Lmax, gr[2]);
        if (ws.flags & TPL_FLAG_PADDING_ZEROED) {
            // the caller keeps the rows past each chain zero
        } else if (pack) {  // rows past each chain's slots
            for (int i = 0; i < m; ++i) {
                float* gi = grad_angles + (size_t)s_pack.b[i] * 3 * Lmax;
                for (int j = s_pack.off[i + 1] - s_pack.off[i] + threadIdx.x; j < Lmax; j += NT) {
                    gi[j] = 0.f;
                    gi[Lmax + j] = 0.f;
                    gi[2 * Lmax + j] = 0.f;
                }
            }
        } else if (t == T - 1) {
            for (int i = min(Lmax, T * TILE) + threadIdx.x; i < Lmax; i += NT) {
                ga[i] = 0.f;
                ga[Lmax + i] = 0.f;
                ga[2 * Lmax + i] = 0.f;
            }
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
                for (int w2 = 0; w2 < NT / 32; ++w2) tot += s_res[w2];
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
                    float lr, scale;
                    lrmsd_from_sum(sum, 3 * L, lr, scale);
                    lg.lrmsd_out[b] = lr;
                    s_scale = scale;
                }
                __syncthreads();
                const float sc = s_scale;
                for (int i = threadIdx.x; i < 3 * L; i += NT) {
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
// K2q: the paper's O(L^2) evaluation of Eq. 2 -- every (angle, atom) term
// summed directly, no suffix scan -- as a GPU comparator for K2.  The angle
// at atom q (q >= 1: omega at N, phi at CA, psi at C) turns the atoms k >= q
// about the unit bond u_q = (r_q - r_{q-1}) / |.| through p_q = r_q, so
//   dL/dalpha_q = sum_{k >= q} g_k . (u_q x (r_k - p_q)) = u_q . sum_{k >= q} (r_k - p_q) x g_k.
// One thread per atom q of a chain (grid y = chain); the CTA stages tiles of
// the chain's coordinates and gradients in shared memory and every thread
// sums the tile's atoms k >= q, like a tiled all-pairs sum.
// ---------------------------------------------------------------------------
constexpr int kQNT = 128;

__global__ void __launch_bounds__(kQNT) bb_bwd_quadratic_kernel(const int32_t* __restrict__ lengths, int Lmax,
                                                              const float* __restrict__ coords,
                                                              const float* __restrict__ grad_coords,
                                                              float* __restrict__ grad_angles) {
    __shared__ float3 s_r[kQNT], s_g[kQNT];
    const int b = blockIdx.y;
    const int L = clamp_length(lengths, b, Lmax);
    const int na = 3 * L;
    const int q0 = blockIdx.x * kQNT, q = q0 + threadIdx.x;
    const float* r_in = coords + (size_t)b * 9 * Lmax;
    const float* g_in = grad_coords + (size_t)b * 9 * Lmax;
    float3 rq = make_float3(0.f, 0.f, 0.f), u = rq;
    if (q < na) {
        rq = make_float3(r_in[3 * q], r_in[3 * q + 1], r_in[3 * q + 2]);
        if (q > 0) {
            u = f3_sub(rq, make_float3(r_in[3 * q - 3], r_in[3 * q - 2], r_in[3 * q - 1]));
            u = f3_scale(rsqrtf(f3_dot(u, u)), u);
        }
    }
    float3 c = make_float3(0.f, 0.f, 0.f);  // sum_{k >= q} (r_k - p_q) x g_k
    for (int k0 = q0; k0 < na; k0 += kQNT) {
        const int k = k0 + threadIdx.x;
        __syncthreads();
        s_r[threadIdx.x] = k < na ? make_float3(r_in[3 * k], r_in[3 * k + 1], r_in[3 * k + 2]) : rq;
        s_g[threadIdx.x] = k < na ? make_float3(g_in[3 * k], g_in[3 * k + 1], g_in[3 * k + 2])
                                  : make_float3(0.f, 0.f, 0.f);
        __syncthreads();
        const int kend = min(kQNT, na - k0);
        for (int t = 0; t < kend; ++t)
            if (k0 + t >= q) c = f3_add(c, f3_cross(f3_sub(s_r[t], rq), s_g[t]));
    }
    if (q < 3 * Lmax) {
        // atom q = 3 j + at carries omega_j (at 0), phi_j (at 1) or psi_j (at 2)
        const int j = q / 3, at = q % 3;
        const float val = (q > 0 && q < na) ? f3_dot(u, c) : 0.f;
        grad_angles[(size_t)b * 3 * Lmax + row_of(at) * Lmax + j] = val;
    }
}

// ---------------------------------------------------------------------------
// K1s: the backbone training step on the LRMSD loss (Section 4 chained into
// Eq. 2): coordinates, LRMSD_b and the gradient of sum_b w_b LRMSD_b with
// respect to the angles.  A work-list entry that holds whole chains (a pack
// of short chains, or a chain of one tile) runs the whole step in its CTA
// with the chains' coordinates and target atoms in shared memory: forward
// scan, the 17 LRMSD moments of each chain, the eigen-solve (one quad of
// warp 0 per chain), the residual sum and LRMSD (FP64 over the threads),
// each atom's gradient w_b (y' - U x') / (N LRMSD), and the segmented suffix
// scan of Eq. 2.  HBM traffic per residue: angles in (12 B), target in (36),
// coordinates out (36), angle gradient out (12).  A tile of a longer chain
// only runs the forward and reduces its tile's moments; the eigen-solve and
// the backward of such chains follow in two more launches.
// ---------------------------------------------------------------------------

// Sums over the threads of each pack member (sid = member index, -1 for none)
// of F values: member i's totals in tot[i * F .. i * F + F).  Segments are
// contiguous thread ranges: a shuffle suffix scan within each warp (lanes of
// equal sid), the head lane of each segment in a warp writes the warp's
// partial, and the partials are added over the warps in order.  Fixed order,
// two barriers.  s_part holds NW * kMaxPack * F values.
template <int NT, int F, typename T>
__device__ __forceinline__ void pack_member_sums(T (&v)[F], int sid, T* s_part, T* tot, int m) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int so = __shfl_down_sync(0xffffffffu, sid, off);
#pragma unroll
        for (int q = 0; q < F; ++q) {
            const T y = __shfl_down_sync(0xffffffffu, v[q], off);
            if (lane + off < 32 && so == sid) v[q] += y;
        }
    }
    const int sp = __shfl_up_sync(0xffffffffu, sid, 1);
    const bool head = sid >= 0 && (lane == 0 || sp != sid);
    T* mine = s_part + (size_t)warp * kMaxPack * F;
    for (int i = lane; i < kMaxPack * F; i += 32) mine[i] = T(0);
    __syncwarp();
    if (head)
#pragma unroll
        for (int q = 0; q < F; ++q) mine[sid * F + q] = v[q];
    __syncthreads();
    for (int i = threadIdx.x; i < m * F; i += NT) {
        T x = T(0);
#pragma unroll
        for (int w = 0; w < NW; ++w) x += s_part[(size_t)w * kMaxPack * F + i];
        tot[i] = x;
    }
    __syncthreads();
}

// Writes each pack member's row of n9 = 9 len floats from the stage (slot
// offsets o9 = 9 off) to `out` rows of 9 Lmax floats, with the zero padding
// past it unless the caller keeps the padding zero.
template <int NT>
__device__ __forceinline__ void store_pack_rows(float* __restrict__ out, const float* s_out, const PackS& pk,
                                                int m, int Lmax, bool write_padding) {
    for (int i = 0; i < m; ++i) {
        const int n9 = 9 * pk.len[i], o9 = 9 * pk.off[i];
        float4* dst = reinterpret_cast<float4*>(out + (size_t)pk.b[i] * 9 * Lmax);
        const int full = n9 >> 2;
        if ((o9 & 3) == 0) {
            const float4* src = reinterpret_cast<const float4*>(s_out + o9);
            for (int q = threadIdx.x; q < full; q += NT) dst[q] = src[q];
        } else {
            for (int q = threadIdx.x; q < full; q += NT) {
                const float* e = s_out + o9 + 4 * q;
                dst[q] = make_float4(e[0], e[1], e[2], e[3]);
            }
        }
        if ((n9 & 3) && threadIdx.x == 0) {
            const int e = 4 * full;
            dst[full] = make_float4(s_out[o9 + e], e + 1 < n9 ? s_out[o9 + e + 1] : 0.f,
                                    e + 2 < n9 ? s_out[o9 + e + 2] : 0.f, 0.f);
        }
        if (write_padding)
            for (int q = ((n9 + 3) >> 2) + threadIdx.x; q < 9 * Lmax / 4; q += NT)
                dst[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// The 17 moments of atoms y (coordinates) against x (target): sum dx, sum dy,
// sum dx dy^T, sum |dx|^2, sum |dy|^2 with dx = x - x0, dy = y (the chain's
// first atom is the origin, R_0 = I).
__device__ __forceinline__ void add_moments(float (&m)[kMom], float3 x, float3 x0, float3 dy) {
    const float3 dx = f3_sub(x, x0);
    m[0] += dx.x; m[1] += dx.y; m[2] += dx.z;
    m[3] += dy.x; m[4] += dy.y; m[5] += dy.z;
    m[6] = fmaf(dx.x, dy.x, m[6]); m[7] = fmaf(dx.x, dy.y, m[7]); m[8] = fmaf(dx.x, dy.z, m[8]);
    m[9] = fmaf(dx.y, dy.x, m[9]); m[10] = fmaf(dx.y, dy.y, m[10]); m[11] = fmaf(dx.y, dy.z, m[11]);
    m[12] = fmaf(dx.z, dy.x, m[12]); m[13] = fmaf(dx.z, dy.y, m[13]); m[14] = fmaf(dx.z, dy.z, m[14]);
    m[15] += f3_dot(dx, dx);
    m[16] += f3_dot(dy, dy);
}

__device__ __forceinline__ float3 ld3(const float* p) { return make_float3(p[0], p[1], p[2]); }

template <int NT, int K>
constexpr int step_min_blocks() { return NT >= 512 ? 1 : (NT >= 256 ? 3 : 4); }

// Dynamic shared memory of K1s: the tile's coordinates (the target atoms are
// read from global memory, each thread its own, and stay in L1 across the
// passes; staging them too would halve the CTAs per SM).
template <int NT, int K>
constexpr size_t step_smem() { return (size_t)9 * NT * K * sizeof(float); }

template <int NT, int K>
__global__ void __launch_bounds__(NT, step_min_blocks<NT, K>()) bb_step_kernel(
    const float* __restrict__ angles, const int32_t* __restrict__ lengths, int Lmax,
    const float* __restrict__ target, const float* __restrict__ grad_lrmsd, float* __restrict__ coords,
    float* __restrict__ lrmsd, float* __restrict__ grad_angles, ChainWs ws, BackboneConst bc) {
    constexpr int NW = NT / 32;
    constexpr int TILE = NT * K;
    __shared__ RigidS s_rig[NW + 1];
    __shared__ int s_cnt[NW + 1];
    __shared__ float s6[6 * (NW + 1)];
    __shared__ int s_v;
    __shared__ PackS s_pack;
    __shared__ float s_part[NW * kMaxPack * kMom];
    __shared__ float s_tot[kMaxPack * kMom];
    __shared__ double s_dpart[NW * kMaxPack];
    __shared__ double s_dtot[kMaxPack];
    __shared__ __align__(16) float s_state[kMaxPack * 16];
    __shared__ float s_w[kMaxPack];
    extern __shared__ float4 s_dyn[];
    float* s_out = reinterpret_cast<float*>(s_dyn);  // [9 TILE] coordinates of the tile
    const bool write_padding = !(ws.flags & TPL_FLAG_PADDING_ZEROED);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    const int ntiles = ws.hdr[kHdrTiles];
    int v = take_tile(ws.hdr + kHdrFwdNext, &s_v);
    while (v < ntiles) {
        const int2 ct = ws.tiles[v];
        int m = 1, T = 1, L = 0, b = 0;
        if (ct.x < 0) {
            m = ct.y;
            load_pack<K>(ws, lengths, Lmax, -1 - ct.x, m, s_pack);
        } else {
            b = ct.x;
            L = clamp_length(lengths, b, Lmax);
            T = L > 0 ? (L + TILE - 1) / TILE : 1;
            if (T == 1) {  // one whole chain: a pack of one
                if (threadIdx.x == 0) {
                    s_pack.b[0] = b;
                    s_pack.len[0] = L;
                    s_pack.off[0] = 0;
                    s_pack.off[1] = (L + K - 1) / K * K;
                }
                __syncthreads();
            }
        }
        if (T == 1) {
            // ---- the whole step for the entry's chains ----
            const int slot = threadIdx.x * K;
            const int ci = pack_member(s_pack, m, slot);
            b = ci >= 0 ? s_pack.b[ci] : 0;
            L = ci >= 0 ? s_pack.len[ci] : 0;
            const int j0 = ci >= 0 ? slot - s_pack.off[ci] : Lmax;  // Lmax: nothing to load or store
            float3 pos[3 * K];
            const Rigid A = thread_product<K>(angles + (size_t)b * 3 * Lmax, j0, L, Lmax, bc, pos);
            const Rigid E = block_seg_scan_rigid<NT>(A, ci < 0 || j0 == 0, s_rig, s_cnt);
            const int requested = request_tile(ws.hdr + kHdrFwdNext);
            {
                float vv[9 * K];
#pragma unroll
                for (int k = 0; k < K; ++k)
#pragma unroll
                    for (int at = 0; at < 3; ++at) {
                        const float3 r = point_apply(E, pos[3 * k + at]);
                        vv[9 * k + 3 * at + 0] = r.x;
                        vv[9 * k + 3 * at + 1] = r.y;
                        vv[9 * k + 3 * at + 2] = r.z;
                    }
                store_stage<K>(s_out + threadIdx.x * 9 * K, vv);
            }
            __syncthreads();
            store_pack_rows<NT>(coords, s_out, s_pack, m, Lmax, write_padding);
            const float* my_r = s_out + 9 * slot;  // this thread's atoms
            const float* tg = target + (size_t)b * 9 * Lmax;  // the chain's target
            const float* my_x = tg + 9 * (size_t)min(j0, Lmax - K);
            const int nres = ci >= 0 ? max(0, min(K, L - j0)) : 0;  // real residues of this thread
            // moments of each chain
            {
                float mom[kMom];
#pragma unroll
                for (int q = 0; q < kMom; ++q) mom[q] = 0.f;
                if (nres > 0) {
                    const float3 x0 = make_float3(__ldg(tg), __ldg(tg + 1), __ldg(tg + 2));
#pragma unroll
                    for (int q = 0; q < 3 * K; ++q)
                        if (q < 3 * nres) add_moments(mom, ld3(my_x + 3 * q), x0, ld3(my_r + 3 * q));
                }
                pack_member_sums<NT, kMom>(mom, ci, s_part, s_tot, m);
            }
            // eigen-solve: member i on lanes 4 i .. 4 i + 3 of warp 0
            if (warp == 0) {
                const int i = lane >> 2;
                const bool active = i < m;
                const int ii = active ? i : 0;
                float S[kSlot];
#pragma unroll
                for (int q = 0; q < kSlot; ++q) S[q] = q < kMom ? s_tot[ii * kMom + q] : 0.f;
                const float* x0p = target + (size_t)s_pack.b[ii] * 9 * Lmax;
                const float* y0p = s_out + 9 * s_pack.off[ii];
                const float x0[3] = {x0p[0], x0p[1], x0p[2]}, y0[3] = {y0p[0], y0p[1], y0p[2]};
                quad_eigen_solve(S, x0, y0, 3 * s_pack.len[ii], lane & 3, lane, active, s_state + 16 * ii);
            }
            __syncthreads();
            // residuals and LRMSD of each chain (FP32 per thread, FP64 over the threads)
            const PairState ps = load_state_shared(s_state + 16 * (ci >= 0 ? ci : 0));
            {
                float acc = 0.f;
#pragma unroll
                for (int q = 0; q < 3 * K; ++q)
                    if (q < 3 * nres) {
                        const float3 d = residual(ps, ld3(my_x + 3 * q), ld3(my_r + 3 * q));
                        acc += f3_dot(d, d);
                    }
                double dv[1] = {(double)acc};
                pack_member_sums<NT, 1>(dv, ci, s_dpart, s_dtot, m);
            }
            if (threadIdx.x < m) {
                const int i = threadIdx.x;
                float lr, scale;
                lrmsd_from_sum(s_dtot[i], 3 * s_pack.len[i], lr, scale);
                lrmsd[s_pack.b[i]] = lr;
                s_w[i] = __ldg(grad_lrmsd + s_pack.b[i]) * scale;
            }
            __syncthreads();
            // each atom's gradient, then the backward of Eq. 2 (segmented suffix scan)
            // (the atom gradients are formed again from shared memory in the
            // walk below rather than kept in registers)
            const float w = ci >= 0 ? s_w[ci] : 0.f;
            Sum6 own = sum6_zero();
#pragma unroll
            for (int q = 0; q < 3 * K; ++q) {
                if (q < 3 * nres) {
                    const float3 ri = ld3(my_r + 3 * q);
                    const float3 gi = f3_scale(w, residual(ps, ld3(my_x + 3 * q), ri));
                    own.c = f3_add(own.c, f3_cross(ri, gi));
                    own.g = f3_add(own.g, gi);
                }
            }
            const bool tail = ci < 0 || slot + K >= s_pack.off[ci + 1];
            Sum6 S = sum6_add(block_seg_suffix_sum6<NT>(own, tail, s6, s_cnt), own);
            float gr[3][K];
            float3 prev = (j0 > 0 && ci >= 0) ? ld3(my_r - 3) : make_float3(0.f, 0.f, 0.f);
#pragma unroll
            for (int k = 0; k < K; ++k) {
#pragma unroll
                for (int at = 0; at < 3; ++at) {
                    const int q = 3 * k + at;
                    float val = 0.f;
                    const float3 ri = ld3(my_r + 3 * q);
                    if (k < nres) {
                        const float3 gi = f3_scale(w, residual(ps, ld3(my_x + 3 * q), ri));
                        if (j0 + k > 0 || at > 0) {
                            float3 u = f3_sub(ri, prev);
                            u = f3_scale(rsqrtf(f3_dot(u, u)), u);
                            val = f3_dot(u, f3_sub(S.c, f3_cross(ri, S.g)));
                        }
                        S.c = f3_sub(S.c, f3_cross(ri, gi));
                        S.g = f3_sub(S.g, gi);
                    }
                    prev = ri;
                    gr[row_of(at)][k] = val;
                }
            }
            float* ga = grad_angles + (size_t)b * 3 * Lmax;
            store_row<K>(ga, j0, Lmax, gr[0]);
            store_row<K>(ga + Lmax, j0, Lmax, gr[1]);
            store_row<K>(ga + 2 * Lmax, j0, Lmax, gr[2]);
            if (write_padding)  // rows past each chain's slots
                for (int i = 0; i < m; ++i) {
                    float* gi = grad_angles + (size_t)s_pack.b[i] * 3 * Lmax;
                    for (int j = s_pack.off[i + 1] - s_pack.off[i] + threadIdx.x; j < Lmax; j += NT) {
                        gi[j] = 0.f;
                        gi[Lmax + j] = 0.f;
                        gi[2 * Lmax + j] = 0.f;
                    }
                }
            v = next_tile(requested, &s_v);
            continue;
        }
        // ---- a tile of a longer chain: forward and the tile's moments ----
        const int t = ct.y;
        const int slot0 = b * ws.tmax;
        float* out = coords + (size_t)b * 9 * Lmax;
        const int tile0 = t * TILE;
        const int j0 = tile0 + threadIdx.x * K;
        float3 pos[3 * K];
        const Rigid A = thread_product<K>(angles + (size_t)b * 3 * Lmax, j0, L, Lmax, bc, pos);
        Rigid E, Tot;
        int ce, ctot;
        block_scan_rigid_count<NT>(A, 0, s_rig, s_cnt, E, ce, Tot, ctot);
        if (threadIdx.x == NT - 32) publish_prefix_agg(ws, slot0 + t, Tot, 0);
        int pc;
        const Rigid P = gather_prefix(ws, slot0, t, pc);  // every warp gathers it
        const int requested = request_tile(ws.hdr + kHdrFwdNext);
        E = rigid_mul(P, E);
        {
            float vv[9 * K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const bool valid = j0 + k < L;
#pragma unroll
                for (int at = 0; at < 3; ++at) {
                    const float3 r = point_apply(E, pos[3 * k + at]);
                    vv[9 * k + 3 * at + 0] = valid ? r.x : 0.f;
                    vv[9 * k + 3 * at + 1] = valid ? r.y : 0.f;
                    vv[9 * k + 3 * at + 2] = valid ? r.z : 0.f;
                }
            }
            store_stage<K>(s_out + threadIdx.x * 9 * K, vv);
        }
        __syncthreads();
        const int nres_out = write_padding ? min(TILE, Lmax - tile0) : min(TILE, (L - tile0 + 3) & ~3);  // multiple of 4
        {
            float4* dst = reinterpret_cast<float4*>(out + 9 * (size_t)tile0);
            const float4* src = reinterpret_cast<const float4*>(s_out);
            for (int i = threadIdx.x; i < nres_out * 9 / 4; i += NT) dst[i] = src[i];
            if (t == T - 1 && write_padding) {  // zero the residues past the last tile
                float4* o4 = reinterpret_cast<float4*>(out);
                for (int i = min(Lmax, T * TILE) * 9 / 4 + threadIdx.x; i < Lmax * 9 / 4; i += NT)
                    o4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        {
            float mom[kMom];
#pragma unroll
            for (int q = 0; q < kMom; ++q) mom[q] = 0.f;
            const int nres = max(0, min(K, L - j0));
            if (nres > 0) {
                const float* tg = target + (size_t)b * 9 * Lmax;
                const float3 x0 = make_float3(__ldg(tg), __ldg(tg + 1), __ldg(tg + 2));
                const float* my_r = s_out + 9 * threadIdx.x * K;
                const float* my_x = tg + 9 * (size_t)j0;
#pragma unroll
                for (int q = 0; q < 3 * K; ++q)
                    if (q < 3 * nres) add_moments(mom, ld3(my_x + 3 * q), x0, ld3(my_r + 3 * q));
            }
            pack_member_sums<NT, kMom>(mom, nres > 0 ? 0 : -1, s_part, s_tot, 1);
            if (threadIdx.x < kMom) ws.tmom[(size_t)(slot0 + t) * kSlot + threadIdx.x] = s_tot[threadIdx.x];
        }
        v = next_tile(requested, &s_v);
    }
}

// ---------------------------------------------------------------------------
// K7: plain FP64 per-chain forms (one CTA per chain, thread 0 serial).
// ---------------------------------------------------------------------------
__global__ void bb_fwd_ref64_kernel(const double* __restrict__ angles,
                                    const int32_t* __restrict__ lengths, int B, int Lmax,
                                    double* __restrict__ coords, BackboneConstD bc) {
    const int b = blockIdx.x;
    const int L = clamp_length(lengths, b, Lmax);
    double* out = coords + (size_t)b * 9 * Lmax;
    for (int i = 9 * L + threadIdx.x; i < 9 * Lmax; i += blockDim.x) out[i] = 0.0;
    if (threadIdx.x != 0) return;
    const double* ang = angles + (size_t)b * 3 * Lmax;
    // M = [Q | t] as a dense 3x4, M <- M R with R the Section 3 matrix
    double M[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};
    for (int j = 0; j < L; ++j)
        for (int at = 0; at < 3; ++at) {
            const int i = 3 * j + at;
            if (i > 0) {
                double sa, ca;
                sincos(ang[row_of(at) * Lmax + j], &sa, &ca);
                const double ct = bc.ct[at], st = bc.st[at], d = bc.d[at];
                const double R[12] = {ct, sa * st, ca * st, d * ct, 0.0, ca, -sa, 0.0,
                                      -st, sa * ct, ca * ct, -d * st};
                double N[12];
                for (int r = 0; r < 3; ++r)
                    for (int c = 0; c < 4; ++c) {
                        double s = (c == 3) ? M[4 * r + 3] : 0.0;
                        for (int k = 0; k < 3; ++k) s += M[4 * r + k] * R[4 * k + c];
                        N[4 * r + c] = s;
                    }
                for (int k = 0; k < 12; ++k) M[k] = N[k];
            }
            out[3 * i + 0] = M[3];
            out[3 * i + 1] = M[7];
            out[3 * i + 2] = M[11];
        }
}

__global__ void bb_bwd_ref64_kernel(const int32_t* __restrict__ lengths, int B, int Lmax,
                                    const double* __restrict__ coords,
                                    const double* __restrict__ grad_coords,
                                    double* __restrict__ grad_angles) {
    const int b = blockIdx.x;
    const int L = clamp_length(lengths, b, Lmax);
    double* ga = grad_angles + (size_t)b * 3 * Lmax;
    for (int i = L + threadIdx.x; i < Lmax; i += blockDim.x) {
        ga[i] = 0.0;
        ga[Lmax + i] = 0.0;
        ga[2 * Lmax + i] = 0.0;
    }
    if (threadIdx.x != 0 || L == 0) return;
    const double* r = coords + (size_t)b * 9 * Lmax;
    const double* g = grad_coords + (size_t)b * 9 * Lmax;
    double Sc[3] = {0, 0, 0}, Sg[3] = {0, 0, 0};
    for (int i = 3 * L - 1; i >= 1; --i) {
        const double* ri = r + 3 * i;
        const double* gi = g + 3 * i;
        Sc[0] += ri[1] * gi[2] - ri[2] * gi[1];
        Sc[1] += ri[2] * gi[0] - ri[0] * gi[2];
        Sc[2] += ri[0] * gi[1] - ri[1] * gi[0];
        Sg[0] += gi[0]; Sg[1] += gi[1]; Sg[2] += gi[2];
        double u[3] = {ri[0] - ri[-3], ri[1] - ri[-2], ri[2] - ri[-1]};
        const double n = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        u[0] /= n; u[1] /= n; u[2] /= n;
        const double w0 = Sc[0] - (ri[1] * Sg[2] - ri[2] * Sg[1]);
        const double w1 = Sc[1] - (ri[2] * Sg[0] - ri[0] * Sg[2]);
        const double w2 = Sc[2] - (ri[0] * Sg[1] - ri[1] * Sg[0]);
        ga[row_of(i % 3) * Lmax + i / 3] = u[0] * w0 + u[1] * w1 + u[2] * w2;
    }
    ga[2 * Lmax + 0] = 0.0;  // omega_0: R_0 = I carries no angle
}

template <int NT, int K>
cudaError_t fwd_t(const float* angles, const int32_t* lengths, int B, int Lmax, float* coords,
                  const ChainWs& ws, cudaStream_t s) {
    const int grid = persistent_grid((const void*)bb_fwd_kernel<NT, K>, NT, 0);
    bb_fwd_kernel<NT, K><<<grid, NT, 0, s>>>(angles, lengths, Lmax, coords, ws, backbone_const(), nullptr);
    return cudaGetLastError();
}

template <int NT, int K>
cudaError_t bwd_t(const float* angles, const int32_t* lengths, int B, int Lmax,
                  const float* coords, const float* grad_coords, float* grad_angles,
                  bool from_coords, const ChainWs& ws, const LrmsdGrad& lg, cudaStream_t s) {
    if (lg.target) {
        const int grid = persistent_grid((const void*)bb_bwd_kernel<NT, K, true, true>, NT, 0);
        bb_bwd_kernel<NT, K, true, true><<<grid, NT, 0, s>>>(angles, lengths, B, Lmax, coords, grad_coords,
                                                              grad_angles, ws, lg, backbone_const());
    } else if (from_coords) {
        const int grid = persistent_grid((const void*)bb_bwd_kernel<NT, K, true, false>, NT, 0);
        bb_bwd_kernel<NT, K, true, false><<<grid, NT, 0, s>>>(angles, lengths, B, Lmax, coords, grad_coords,
                                                               grad_angles, ws, lg, backbone_const());
    } else {
        const int grid = persistent_grid((const void*)bb_bwd_kernel<NT, K, false, false>, NT, 0);
        bb_bwd_kernel<NT, K, false, false><<<grid, NT, 0, s>>>(angles, lengths, B, Lmax, coords, grad_coords,
                                                                grad_angles, ws, lg, backbone_const());
    }
    return cudaGetLastError();
}

template <int NT, int K>
cudaError_t fwd_o_t(const float* angles, const int32_t* lengths, int Lmax, float* coords, float* o_coords,
                    const ChainWs& ws, cudaStream_t s) {
    const int grid = persistent_grid((const void*)bb_fwd_kernel<NT, K, true>, NT, 0);
    bb_fwd_kernel<NT, K, true><<<grid, NT, 0, s>>>(angles, lengths, Lmax, coords, ws, backbone_const(), o_coords);
    return cudaGetLastError();
}

template <int NT, int K>
cudaError_t bwd_o_t(const float* angles, const int32_t* lengths, int B, int Lmax, const float* coords,
                    const float* o_coords, const float* grad_coords, const float* grad_o, float* grad_angles,
                    bool from_coords, const ChainWs& ws, cudaStream_t s) {
    const LrmsdGrad none{nullptr, nullptr, nullptr};
    if (from_coords) {
        const int grid = persistent_grid((const void*)bb_bwd_kernel<NT, K, true, false, false, true>, NT, 0);
        bb_bwd_kernel<NT, K, true, false, false, true><<<grid, NT, 0, s>>>(
            angles, lengths, B, Lmax, coords, grad_coords, grad_angles, ws, none, backbone_const(), o_coords, grad_o);
    } else {
        const int grid = persistent_grid((const void*)bb_bwd_kernel<NT, K, false, false, false, true>, NT, 0);
        bb_bwd_kernel<NT, K, false, false, false, true><<<grid, NT, 0, s>>>(
            angles, lengths, B, Lmax, coords, grad_coords, grad_angles, ws, none, backbone_const(), nullptr, grad_o);
    }
    return cudaGetLastError();
}

template <int NT, int K>
cudaError_t step_t(const float* angles, const int32_t* lengths, int B, int Lmax, const float* target,
                   const float* grad_lrmsd, float* coords, float* lrmsd, float* grad_angles, const ChainWs& ws,
                   cudaStream_t s) {
    constexpr int TILE = NT * K;
    const size_t smem = step_smem<NT, K>();
    static bool done[64] = {false};
    cudaError_t e = smem_attr_once(bb_step_kernel<NT, K>, (int)smem, done);
    if (e != cudaSuccess) return e;
    const int grid = persistent_grid((const void*)bb_step_kernel<NT, K>, NT, smem);
    bb_step_kernel<NT, K><<<grid, NT, smem, s>>>(angles, lengths, Lmax, target, grad_lrmsd, coords, lrmsd,
                                                 grad_angles, ws, backbone_const());
    e = cudaGetLastError();
    if (e != cudaSuccess || Lmax <= TILE) return e;  // every chain was whole: the step is done
    // chains of more than one tile: eigen-solve from the tile moments, then
    // the backward with the residual sums
    e = reset_backward_flags(ws, s);
    if (e != cudaSuccess) return e;
    e = launch_lrmsd_solve_tiles(coords, target, nullptr, B, 3 * Lmax, ws.tmom, ws.tmax, lengths, TILE, Lmax,
                                 ws.lstate, s, false, 2);
    if (e != cudaSuccess) return e;
    const LrmsdGrad lg{target, ws.lstate, grad_lrmsd, lrmsd, nullptr};
    const int bgrid = persistent_grid((const void*)bb_bwd_kernel<NT, K, true, true, true>, NT, 0);
    bb_bwd_kernel<NT, K, true, true, true><<<bgrid, NT, 0, s>>>(angles, lengths, B, Lmax, coords, nullptr,
                                                                grad_angles, ws, lg, backbone_const());
    return cudaGetLastError();
}

}  // namespace

bool backbone_step_cfg_supported(int threads, int k) {
    return (threads == 128 && (k == 2 || k == 4)) || (threads == 256 && (k == 2 || k == 4)) ||
           (threads == 512 && k == 2);
}

bool backbone_o_cfg_supported(int threads, int k) {
    return (threads == 128 && (k == 1 || k == 2 || k == 4)) || (threads == 256 && k == 4);
}

#define TPL_BB_O_DISPATCH(FN, ...)                                            \
    switch (cfg.threads * 8 + cfg.res_per_thread) {                           \
        case 128 * 8 + 1: return FN<128, 1>(__VA_ARGS__);                     \
        case 128 * 8 + 2: return FN<128, 2>(__VA_ARGS__);                     \
        case 128 * 8 + 4: return FN<128, 4>(__VA_ARGS__);                     \
        case 256 * 8 + 4: return FN<256, 4>(__VA_ARGS__);                     \
        default: return cudaErrorInvalidValue;                                \
    }

cudaError_t launch_backbone_forward_o(const float* angles, const int32_t* lengths, int B, int Lmax,
                                      float* coords, float* o_coords, int sched_mode, void* workspace,
                                      LaunchCfg cfg, cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    ChainWs ws;
    chain_ws_layout(workspace, B, Lmax, &ws);
    ws.flags = cfg.flags;
    cudaError_t e = launch_schedule(lengths, B, Lmax, cfg.threads * cfg.res_per_thread, sched_mode,
                                    cfg.res_per_thread, ws, s);
    if (e != cudaSuccess) return e;
    TPL_BB_O_DISPATCH(fwd_o_t, angles, lengths, Lmax, coords, o_coords, ws, s)
}

cudaError_t launch_backbone_backward_o(const float* angles, const int32_t* lengths, int B, int Lmax,
                                       const float* coords, const float* o_coords, const float* grad_coords,
                                       const float* grad_o, float* grad_angles, bool from_coords,
                                       void* workspace, LaunchCfg cfg, cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    ChainWs ws;
    chain_ws_layout(workspace, B, Lmax, &ws);
    ws.flags = cfg.flags;
    cudaError_t e = reset_backward_flags(ws, s);
    if (e != cudaSuccess) return e;
    TPL_BB_O_DISPATCH(bwd_o_t, angles, lengths, B, Lmax, coords, o_coords, grad_coords, grad_o, grad_angles,
                      from_coords, ws, s)
}

cudaError_t launch_backbone_lrmsd_step(const float* angles, const int32_t* lengths, int B, int Lmax,
                                       const float* target, const float* grad_lrmsd, float* coords,
                                       float* lrmsd, float* grad_angles, int sched_mode, void* workspace,
                                       LaunchCfg cfg, cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    ChainWs ws;
    chain_ws_layout(workspace, B, Lmax, &ws, false, true);
    ws.flags = cfg.flags;
    cudaError_t e = launch_schedule(lengths, B, Lmax, cfg.threads * cfg.res_per_thread, sched_mode,
                                    cfg.res_per_thread, ws, s);
    if (e != cudaSuccess) return e;
    switch (cfg.threads * 8 + cfg.res_per_thread) {
        case 128 * 8 + 2: return step_t<128, 2>(angles, lengths, B, Lmax, target, grad_lrmsd, coords, lrmsd, grad_angles, ws, s);
        case 128 * 8 + 4: return step_t<128, 4>(angles, lengths, B, Lmax, target, grad_lrmsd, coords, lrmsd, grad_angles, ws, s);
        case 256 * 8 + 2: return step_t<256, 2>(angles, lengths, B, Lmax, target, grad_lrmsd, coords, lrmsd, grad_angles, ws, s);
        case 256 * 8 + 4: return step_t<256, 4>(angles, lengths, B, Lmax, target, grad_lrmsd, coords, lrmsd, grad_angles, ws, s);
        case 512 * 8 + 2: return step_t<512, 2>(angles, lengths, B, Lmax, target, grad_lrmsd, coords, lrmsd, grad_angles, ws, s);
        default: return cudaErrorInvalidValue;
    }
}

bool backbone_cfg_supported(int threads, int k) {
    return (threads == 64 || threads == 128 || threads == 256 || threads == 512) &&
           (k == 1 || k == 2 || k == 4);
}

#define TPL_BB_DISPATCH(FN, ...)                                              \
    switch (cfg.threads * 8 + cfg.res_per_thread) {                           \
        case 64 * 8 + 1: return FN<64, 1>(__VA_ARGS__);                       \
        case 64 * 8 + 2: return FN<64, 2>(__VA_ARGS__);                       \
        case 64 * 8 + 4: return FN<64, 4>(__VA_ARGS__);                       \
        case 128 * 8 + 1: return FN<128, 1>(__VA_ARGS__);                     \
        case 128 * 8 + 2: return FN<128, 2>(__VA_ARGS__);                     \
        case 128 * 8 + 4: return FN<128, 4>(__VA_ARGS__);                     \
        case 256 * 8 + 1: return FN<256, 1>(__VA_ARGS__);                     \
        case 256 * 8 + 2: return FN<256, 2>(__VA_ARGS__);                     \
        case 256 * 8 + 4: return FN<256, 4>(__VA_ARGS__);                     \
        case 512 * 8 + 1: return FN<512, 1>(__VA_ARGS__);                     \
        case 512 * 8 + 2: return FN<512, 2>(__VA_ARGS__);                     \
        default: return cudaErrorInvalidValue;                                \
    }

cudaError_t launch_backbone_forward(const float* angles, const int32_t* lengths, int B, int Lmax,
                                    float* coords, int sched_mode, void* workspace,
                                    LaunchCfg cfg, cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    ChainWs ws;
    chain_ws_layout(workspace, B, Lmax, &ws);
    ws.flags = cfg.flags;
    cudaError_t e = launch_schedule(lengths, B, Lmax, cfg.threads * cfg.res_per_thread, sched_mode,
                                    cfg.res_per_thread, ws, s);
    if (e != cudaSuccess) return e;
    TPL_BB_DISPATCH(fwd_t, angles, lengths, B, Lmax, coords, ws, s)
}

cudaError_t launch_backbone_backward_quadratic(const int32_t* lengths, int B, int Lmax, const float* coords,
                                              const float* grad_coords, float* grad_angles, cudaStream_t s) {
    if (B == 0 || Lmax == 0) return cudaSuccess;
    const dim3 grid((3 * Lmax + kQNT - 1) / kQNT, B);
    bb_bwd_quadratic_kernel<<<grid, kQNT, 0, s>>>(lengths, Lmax, coords, grad_coords, grad_angles);
    return cudaGetLastError();
}

cudaError_t launch_backbone_backward(const float* angles, const int32_t* lengths, int B, int Lmax,
                                     const float* coords, const float* grad_coords,
                                     float* grad_angles, bool from_coords, void* workspace,
                                     LaunchCfg cfg, cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    ChainWs ws;
    chain_ws_layout(workspace, B, Lmax, &ws);
    ws.flags = cfg.flags;
    cudaError_t e = reset_backward_flags(ws, s);
    if (e != cudaSuccess) return e;
    const LrmsdGrad none{nullptr, nullptr, nullptr};
    TPL_BB_DISPATCH(bwd_t, angles, lengths, B, Lmax, coords, grad_coords, grad_angles, from_coords, ws, none, s)
}

cudaError_t launch_backbone_backward_lrmsd(const float* angles, const int32_t* lengths, int B, int Lmax,
                                           const float* coords, const float* target,
                                           const float* grad_lrmsd, const float* lrmsd_state,
                                           float* grad_angles, void* workspace, LaunchCfg cfg,
                                           cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    ChainWs ws;
    chain_ws_layout(workspace, B, Lmax, &ws);
    ws.flags = cfg.flags;
    cudaError_t e = reset_backward_flags(ws, s);
    if (e != cudaSuccess) return e;
    const LrmsdGrad lg{target, lrmsd_state, grad_lrmsd};
    TPL_BB_DISPATCH(bwd_t, angles, lengths, B, Lmax, coords, nullptr, grad_angles, true, ws, lg, s)
}

cudaError_t launch_backbone_forward_ref64(const double* angles, const int32_t* lengths, int B,
                                          int Lmax, double* coords, cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    bb_fwd_ref64_kernel<<<B, 128, 0, s>>>(angles, lengths, B, Lmax, coords, backbone_const_d());
    return cudaGetLastError();
}

cudaError_t launch_backbone_backward_ref64(const double* angles, const int32_t* lengths, int B,
                                           int Lmax, const double* coords,
                                           const double* grad_coords, double* grad_angles,
                                           cudaStream_t s) {
    (void)angles;
    if (B == 0) return cudaSuccess;
    bb_bwd_ref64_kernel<<<B, 128, 0, s>>>(lengths, B, Lmax, coords, grad_coords, grad_angles);
    return cudaGetLastError();
}

}  // namespace tpl
