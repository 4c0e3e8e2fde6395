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
// output atom).  Once the look-back has given the tile's start frame, each
// thread composes it in, builds M_1, M_3 and the side-chain frames M_1 R'
// R(chi_1) R(chi_2) ... and places the atoms r = M_g r0 into a shared-memory
// stage (with one residue per thread the side chains are built in the order
// of residue types, so that a warp's lanes run the same loops); the stage goes
// out by a bulk store.  The residue tables live in shared memory.
//
// K4 fa_bwd_coords_kernel / fa_bwd_kernel: Eq. 1 as suffix sums.  For a frame
// with x axis u and origin p, dL/dalpha = u . sum_{k downstream} (r_k - p) x
// g_k.  chi_k gradients are local to the residue (suffix over its side-chain
// groups); phi, psi and omega add the sum over all later residues, a reverse
// suffix scan of (sum r x g, sum g) across the tile plus the suffix of the
// later tiles (look-back, tiles of a chain taken last to first).  Axes and
// origins come from the forward's coordinates (fa_bwd_coords_kernel, whose
// side-chain sums run in the order of residue types like the forward's where
// that keeps its CTAs per SM) or
// from frames recomputed from the angles and the tile-start frames
// (fa_bwd_kernel).
#include "kernels.h"
#include "sched.cuh"
#include "tables.h"
#include "tpl_common.cuh"
#include "bulk.cuh"

namespace tpl {

namespace {

__device__ __forceinline__ void copy_table(FaTable& dst, const FaTable& src) {
    const int n = sizeof(FaTable) / 4;
    const int* s = reinterpret_cast<const int*>(&src);
    int* d = reinterpret_cast<int*>(&dst);
    for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = s[i];
}

// The residue table reaches the kernels as a kernel parameter.  Copying its
// 6 KB from parameter space into shared memory serialises on the constant
// cache (several microseconds per CTA), so the first CTA that runs on a device
// also leaves a copy in global memory and sets g_fa_tab_ready; later CTAs copy
// that one with 16-byte loads.  Every launch passes the same table, so a CTA
// that finds the flag unset copies the parameter instead and the result is
// the same either way.
static_assert(sizeof(FaTable) % 16 == 0, "the table is copied in 16-byte pieces");
__device__ FaTable g_fa_tab;
__device__ int g_fa_tab_ready;

__device__ __forceinline__ void load_table(FaTable& dst, const FaTable& param) {
    __shared__ int s_ready;
    if (threadIdx.x == 0) s_ready = flag_acquire(&g_fa_tab_ready);
    __syncthreads();
    constexpr int n4 = (int)(sizeof(FaTable) / 16);
    int4* d = reinterpret_cast<int4*>(&dst);
    if (s_ready) {
        const int4* src = reinterpret_cast<const int4*>(&g_fa_tab);
        for (int i = threadIdx.x; i < n4; i += blockDim.x) d[i] = __ldcg(src + i);
    } else {
        copy_table(dst, param);
        if (blockIdx.x == 0) {
            __syncthreads();
            int4* g = reinterpret_cast<int4*>(&g_fa_tab);
            for (int i = threadIdx.x; i < n4; i += blockDim.x) g[i] = d[i];
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) flag_release(&g_fa_tab_ready, 1);
        }
    }
    __syncthreads();
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

// async_copy_range with the 16-byte aligned middle moved by one bulk copy:
// stage[off + i - g0] <- glob[i], off = g0 mod 4.  Returns whether a bulk copy
// was issued (the same answer in every thread); the caller then waits on `bar`.
template <int NT>
__device__ __forceinline__ bool bulk_copy_range(const float* __restrict__ glob, float* __restrict__ stage, int g0,
                                                int g1, uint64_t* bar) {
    if (g1 <= g0) return false;
    const int off = g0 & 3;
    const int head = min(g1, (g0 + 3) & ~3);
    const int tail = max(head, g1 & ~3);
    for (int i = g0 + threadIdx.x; i < head; i += NT) cp_async4(stage + off + i - g0, glob + i);
    for (int i = tail + threadIdx.x; i < g1; i += NT) cp_async4(stage + off + i - g0, glob + i);
    if (tail <= head) return false;
    float* dst = stage + off + head - g0;  // a multiple of 4 floats from the 16-byte aligned stage
    const float* src = glob + head;        // 16-byte aligned: the row is, and head is a multiple of 4
    const unsigned bytes = 4u * (unsigned)(tail - head);
    if (((smem_addr(dst) | (unsigned)reinterpret_cast<uintptr_t>(src)) & 15u) != 0u) {  // (not expected)
        for (int i = head + threadIdx.x; i < tail; i += NT) cp_async4(stage + off + i - g0, glob + i);
        return false;
    }
    if (threadIdx.x == 0) bulk_load(dst, src, bytes, bar);
    return true;
}

// bulk_copy_range for two arrays of the same layout at the same range (the
// tile's coordinates and their gradient or target), into two stages: both
// aligned middles come in under one barrier phase.
template <int NT>
__device__ __forceinline__ bool bulk_copy_range2(const float* __restrict__ glob1, float* __restrict__ stage1,
                                                 const float* __restrict__ glob2, float* __restrict__ stage2, int g0,
                                                 int g1, uint64_t* bar) {
    if (g1 <= g0) return false;
    const int off = g0 & 3;
    const int head = min(g1, (g0 + 3) & ~3);
    const int tail = max(head, g1 & ~3);
    for (int i = g0 + threadIdx.x; i < head; i += NT) {
        cp_async4(stage1 + off + i - g0, glob1 + i);
        cp_async4(stage2 + off + i - g0, glob2 + i);
    }
    for (int i = tail + threadIdx.x; i < g1; i += NT) {
        cp_async4(stage1 + off + i - g0, glob1 + i);
        cp_async4(stage2 + off + i - g0, glob2 + i);
    }
    if (tail <= head) return false;
    float* dst1 = stage1 + off + head - g0;
    float* dst2 = stage2 + off + head - g0;
    const float* src1 = glob1 + head;
    const float* src2 = glob2 + head;
    if (((smem_addr(dst1) | smem_addr(dst2) | (unsigned)reinterpret_cast<uintptr_t>(src1) |
          (unsigned)reinterpret_cast<uintptr_t>(src2)) & 15u) != 0u) {  // (not expected)
        for (int i = head + threadIdx.x; i < tail; i += NT) {
            cp_async4(stage1 + off + i - g0, glob1 + i);
            cp_async4(stage2 + off + i - g0, glob2 + i);
        }
        return false;
    }
    if (threadIdx.x == 0) bulk_load2(dst1, src1, dst2, src2, 4u * (unsigned)(tail - head), bar);
    return true;
}

// store_range for a stage laid out as stage[off + i - g0] <-> glob[i], off =
// g0 mod 4: the ragged ends by the threads, the 16-byte aligned middle by one
// bulk store (which runs on while the CTA goes on to its next tile).
template <int NT>
__device__ __forceinline__ void bulk_store_range(float* __restrict__ glob, const float* __restrict__ stage, int g0,
                                                 int g1) {
    if (g1 <= g0) return;
    const int off = g0 & 3;
    const int head = min(g1, (g0 + 3) & ~3);
    const int tail = max(head, g1 & ~3);
    for (int i = g0 + threadIdx.x; i < head; i += NT) glob[i] = stage[off + i - g0];
    for (int i = tail + threadIdx.x; i < g1; i += NT) glob[i] = stage[off + i - g0];
    if (tail <= head) return;
    const float* src = stage + off + head - g0;
    float* dst = glob + head;
    if (((smem_addr(src) | (unsigned)reinterpret_cast<uintptr_t>(dst)) & 15u) != 0u) {  // (not expected)
        for (int i = head + threadIdx.x; i < tail; i += NT) glob[i] = stage[off + i - g0];
        return;
    }
    if (threadIdx.x == 0) bulk_store(dst, src, 4u * (unsigned)(tail - head));
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
// Launch shapes.  A CTA has NT threads; each thread owns K consecutive
// residues, so a tile holds at most NT * K - 1 residues (balanced tiles,
// fa_num_tiles).  The stage holds a tile's atoms (12 bytes each) so that the
// forward writes and the backward reads them with coalesced 16-byte accesses;
// it has room for kStageAtoms atoms per residue slot on average.  A residue
// has at most 14 atoms: a tile whose atoms do not fit (a long run of the
// largest types) bypasses the stage and its atoms go to (come from) global
// memory directly.
// ---------------------------------------------------------------------------
constexpr int kStageAtoms = 10;

template <int NT, int K>
__host__ __device__ constexpr int fa_stage_atoms() {
    return NT * K * kStageAtoms;
}
template <int NT, int K>
__host__ __device__ constexpr size_t fa_smem() {
    return (size_t)(4 + 3 * fa_stage_atoms<NT, K>()) * sizeof(float);
}

// The coordinate-reading backward stages a tile's coordinates and, beside
// them, its coordinate gradient (or target); the forward that reduces the
// LRMSD moments stages the tile's target beside its atoms: two stages.
template <int NT, int K>
__host__ __device__ constexpr size_t fa_bwd_smem() {
    return 2 * fa_smem<NT, K>();
}

// CTAs per SM the kernels are compiled for: what shared memory allows (227 KB
// per SM; the residue table and the scan scratch take about 7 KB per CTA),
// capped by a register budget per thread that grows with K.
template <int K>
__host__ __device__ constexpr int fa_reg_budget() {
    return K == 1 ? 80 : (K == 2 ? 96 : 160);
}
// The plain forward with one residue per thread places side chains in the
// order of residue types (fa_fwd_kernel, step 4): a record per residue (frame,
// chi, type, first atom, room: 19 words) and the permutation, NT each.
template <int K, bool LM, bool PACK>
__host__ __device__ constexpr bool fa_fwd_perm() {
    return K == 1 && !LM && !PACK;
}
constexpr int kRecWords = 19;
template <int NT, int K, bool LM, bool PACK>
__host__ __device__ constexpr size_t fa_fwd_smem() {
    return (LM ? fa_bwd_smem<NT, K>() : fa_smem<NT, K>()) +
           (fa_fwd_perm<K, LM, PACK>() ? (size_t)(kRecWords + 1) * NT * sizeof(float) : 0);
}

template <int NT, int K>
__host__ __device__ constexpr int fa_min_blocks_for(size_t smem) {
    return (227 * 1024 / (int)(smem + 7 * 1024)) < (65536 / (NT * fa_reg_budget<K>()))
               ? (227 * 1024 / (int)(smem + 7 * 1024))
               : (65536 / (NT * fa_reg_budget<K>()));
}

// The coordinate-reading backward with one residue per thread also sums side
// chains in the order of residue types: type, first atom and the permutation
// (NT ints each) and each residue's side-chain sums (6 NT floats) -- for the
// shapes whose CTAs per SM that shared memory leaves unchanged (at 256 threads
// it would cost a CTA per SM, and the sort then loses: 365 against 328 us per
// backward at 4096 x 700).
constexpr size_t fa_bwd_perm_bytes(int NT) { return (size_t)9 * NT * sizeof(float); }
template <int NT, int K, bool PACK>
__host__ __device__ constexpr bool fa_bwd_perm() {
    return K == 1 && !PACK &&
           fa_min_blocks_for<NT, K>(fa_bwd_smem<NT, K>() + fa_bwd_perm_bytes(NT)) ==
               fa_min_blocks_for<NT, K>(fa_bwd_smem<NT, K>());
}
template <int NT, int K, bool PACK>
__host__ __device__ constexpr size_t fa_bwd_coords_smem() {
    return fa_bwd_smem<NT, K>() + (fa_bwd_perm<NT, K, PACK>() ? fa_bwd_perm_bytes(NT) : 0);
}

// K consecutive floats (bytes) at p, 4K-byte (K-byte) aligned.
template <int K>
__device__ __forceinline__ void load_k(const float* __restrict__ p, float (&v)[K]) {
    if constexpr (K == 4) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(p));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else if constexpr (K == 2) {
        const float2 q = __ldg(reinterpret_cast<const float2*>(p));
        v[0] = q.x; v[1] = q.y;
    } else {
        v[0] = __ldg(p);
    }
}
template <int K>
__device__ __forceinline__ void load_k(const uint8_t* __restrict__ p, int (&v)[K]) {
    if constexpr (K == 4) {
        const uchar4 q = __ldg(reinterpret_cast<const uchar4*>(p));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else if constexpr (K == 2) {
        const uchar2 q = __ldg(reinterpret_cast<const uchar2*>(p));
        v[0] = q.x; v[1] = q.y;
    } else {
        v[0] = __ldg(p);
    }
}

template <int K>
__device__ __forceinline__ void load_k(const int* __restrict__ p, int (&v)[K]) {
    if constexpr (K == 4) {
        const int4 q = __ldg(reinterpret_cast<const int4*>(p));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else if constexpr (K == 2) {
        const int2 q = __ldg(reinterpret_cast<const int2*>(p));
        v[0] = q.x; v[1] = q.y;
    } else {
        v[0] = __ldg(p);
    }
}

// K consecutive floats (ints) to p, 4K-byte aligned.
template <int K>
__device__ __forceinline__ void store_k(float* p, const float (&v)[K]) {
    if constexpr (K == 4) *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    else if constexpr (K == 2) *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
    else p[0] = v[0];
}
template <int K>
__device__ __forceinline__ void store_k(int* p, const int (&v)[K]) {
    if constexpr (K == 4) *reinterpret_cast<int4*>(p) = make_int4(v[0], v[1], v[2], v[3]);
    else if constexpr (K == 2) *reinterpret_cast<int2*>(p) = make_int2(v[0], v[1]);
    else p[0] = v[0];
}

// The tile-start record of the forward, for the backward: frame at the tile
// start, the tile's first atom and its atom count.
__device__ __forceinline__ void tile_record(const ChainWs& ws, int slot, int& first, int& count) {
    const float4 d = ws.start[4 * (size_t)slot + 3];
    first = __float_as_int(d.x);
    count = __float_as_int(d.y);
}

// Side chain of one residue of type ty from its base frame S = M_1 R': the
// groups S_k = S_{k-1} R(chi_k) (free chi from the angles, fixed ones from the
// table) and every atom r = S_k r0, handed to put(output index, r).
template <typename Put>
__device__ __forceinline__ void side_chain(Rigid S, int ty, float chi0, float chi1, float chi2, float chi3,
                                           const FaTable& tab, Put&& put) {
    const int ng = tab.n_groups[ty], nchi = tab.n_chi[ty];
    const float chi[kMaxGroups] = {chi0, chi1, chi2, chi3};
    int e = 0;
#pragma unroll
    for (int g = 0; g < kMaxGroups; ++g) {
        if (g >= ng) break;
        float sc, cc;
        if (g < nchi) {
            // chi moves only its own side chain (no error propagates along the
            // chain): the SFU sine/cosine is accurate enough here
            __sincosf(chi[g], &sc, &cc);
        } else {
            cc = tab.fixchi[ty][g].x;
            sc = tab.fixchi[ty][g].y;
        }
        const float4 gk = tab.grp[ty][g];
        rigid_mul_R(S, cc, sc, gk.x, gk.y, gk.z);
        const int end = tab.grp_end[ty][g];
        for (; e < end; ++e) {
            const float4 r0 = tab.side[ty][e];
            put((int)r0.w & 15, point_apply(S, make_float3(r0.x, r0.y, r0.z)));
        }
    }
}

// ---------------------------------------------------------------------------
// K3: forward.  One tile per step of a persistent CTA:
//  1. each thread loads the angle rows and types of its K residues (vector
//     loads), builds the residue transforms T_j = R_1(phi_j) R_3(psi_j)
//     R_4(omega_{j+1}) and their product;
//  2. the CTA scans the products and the atom counts (tile-local frame of
//     each thread's first residue, its first atom) and publishes the tile's
//     aggregate for the chain's later tiles;
//  3. one warp gathers the earlier tiles' aggregates (the frame at the tile
//     start; the identity for a chain's first tile, R_0 = I);
//  4. each thread walks its residues in the chain's frame: N = M_0 0, CA =
//     M_1 0, C and O from M_3, the side-chain groups S_0 = M_1 R', S_k =
//     S_{k-1} R(chi_k), placing every atom r = M_g r0 into the stage.  With
//     one residue per thread (PERM) a residue leaves its side-chain record
//     in shared memory instead, a counting sort orders the tile's residues by
//     type, and thread i builds the side chain of the i-th;
//  5. the stage goes out by a bulk store (its ragged ends by the threads).
// The residue tables live in shared memory.
// LM: also reduce, per tile, the LRMSD moments (Section 4) of the tile's atoms
// against `target`: sum dx, sum dy, sum dx dy^T, sum |dx|^2, sum |dy|^2 with
// dx = x - x_0 (x the target, x_0 its first atom) and dy = y (the chain's
// first atom, N of residue 0, is the origin: R_0 = I).  The tile's target rows
// come into a second stage by a bulk copy issued once the tile's first atom is
// known, which runs while the atoms are placed; the moments are summed from
// the two stages.
// ---------------------------------------------------------------------------
// PACK: the work list may hold packs of whole short chains (segmented scans,
// per-chain stores); compiled separately so that tiles of one chain pay nothing.
template <int NT, int K, bool LM, bool PACK>
__global__ void __launch_bounds__(NT, (fa_min_blocks_for<NT, K>(fa_fwd_smem<NT, K, LM, PACK>()))) fa_fwd_kernel(
    const float* __restrict__ angles, const uint8_t* __restrict__ seq,
    const int32_t* __restrict__ lengths, int Lmax, int Amax, float* __restrict__ coords,
    int32_t* __restrict__ num_atoms, ChainWs ws, const float* __restrict__ target,
    const __grid_constant__ FaTable tab) {
    static_assert(!(LM && PACK), "the fused step's schedule has no packs");
    constexpr int NW = NT / 32;
    constexpr int TILE = NT * K;
    constexpr int CAP = fa_stage_atoms<NT, K>();
    __shared__ FaTable s_tab;
    __shared__ RigidS s_rig[NW + 1];
    __shared__ int s_cnt[NW + 1];
    __shared__ int s_v, s_next;
    __shared__ float4 s_start[4];  // tile-start frame and its first atom
    __shared__ float s_mom[LM ? NW : 1][17];
    __shared__ PackS s_pack;                            // a pack of whole short chains
    __shared__ int s_cnt2[NW + 1], s_fl2[NW + 1];
    __shared__ int s_mtot[kMaxPack], s_mbase[kMaxPack + 1];  // atoms per member, stage offsets
    __shared__ __align__(8) uint64_t s_bar;  // LM: completes when the tile's target has landed
    extern __shared__ float4 s_dyn[];
    float* stage = reinterpret_cast<float*>(s_dyn);  // the tile's atoms, 3 floats each
    float* stage_t = stage + fa_smem<NT, K>() / sizeof(float);  // LM: the tile's target, same layout
    constexpr bool PERM = fa_fwd_perm<K, LM, PACK>();
    float* rec = stage + fa_smem<NT, K>() / sizeof(float);  // PERM: word f of residue i at rec[f * NT + i]
    int* perm = reinterpret_cast<int*>(rec + kRecWords * NT);  // PERM: thread of the i-th residue in type order
    __shared__ int s_tcnt[kNumTypes], s_tbase[kNumTypes];

    load_table(s_tab, tab);
    if (LM && threadIdx.x == 0) mbar_init(&s_bar);  // visible after take_tile's barrier
    unsigned bphase = 0;                             // the barrier phase the next target copy completes
    const int ntiles = ws.hdr[kHdrTiles];
    int v = take_tile(ws.hdr + kHdrFwdNext, &s_v);
    while (v < ntiles) {
        const int2 ct = ws.tiles[v];
        if (PERM && threadIdx.x < kNumTypes) s_tcnt[threadIdx.x] = 0;  // used after the scan's barriers
        // a tile of one chain, or (chains per CTA > 1) a pack of whole chains,
        // each in its own slots of K residues, scanned as segments
        const bool pack = PACK && ct.x < 0;
        int m = 0, ci = -1;
        if (pack) {
            m = ct.y;
            if (threadIdx.x < kMaxPack) s_mtot[threadIdx.x] = 0;
            load_pack<K>(ws, lengths, Lmax, -1 - ct.x, m, s_pack);
            ci = pack_member(s_pack, m, threadIdx.x * K);
        }
        const int b = pack ? s_pack.b[ci >= 0 ? ci : 0] : ct.x;
        const int t = pack ? 0 : ct.y;
        const int L = pack ? (ci >= 0 ? s_pack.len[ci] : 0) : clamp_length(lengths, b, Lmax);
        const int T = pack ? 1 : fa_num_tiles(L, TILE);
        const int s0 = pack ? 0 : fa_tile_start(L, T, t), s1 = pack ? L : fa_tile_start(L, T, t + 1);
        const int slot0 = b * ws.tmax;
        const float* ang = angles + (size_t)b * 7 * Lmax;
        float* out = coords + (size_t)b * Amax * 3;
        const int j0 = pack ? (ci >= 0 ? threadIdx.x * K - s_pack.off[ci] : 0) : s0 + threadIdx.x * K;

        // 1. inputs of the thread's residues, every angle row up front
        int type[K];
        float phi[K], psi[K], om[K], chi[kMaxGroups][K];
        float om_next = 0.f;
        if (j0 < s1) {
            load_k<K>(seq + (size_t)b * Lmax + j0, type);
            load_k<K>(ang + j0, phi);
            load_k<K>(ang + Lmax + j0, psi);
            load_k<K>(ang + 2 * Lmax + j0, om);
#pragma unroll
            for (int c = 0; c < kMaxGroups; ++c) load_k<K>(ang + (3 + c) * Lmax + j0, chi[c]);
            if (j0 + K < L) om_next = __ldg(ang + 2 * Lmax + j0 + K);
        }
        float sp[K], cp[K], ss[K], cs[K], so[K], co[K];
        Rigid A = rigid_identity();
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int j = j0 + k;
            sp[k] = ss[k] = so[k] = 0.f;
            cp[k] = cs[k] = co[k] = 1.f;
            if (j < s1) {
                int ty = type[k];
                if (ty >= kNumTypes) {
                    flag_status(TPL_STATUS_BAD_RESIDUE);
                    ty = kGlyCode;
                }
                type[k] = ty;
                cnt += s_tab.n_atoms[ty];
                sincosf(phi[k], &sp[k], &cp[k]);
                sincosf(psi[k], &ss[k], &cs[k]);
                if (k == 0) A = rigid_R(cp[k], sp[k], s_tab.bb.ct[1], s_tab.bb.st[1], s_tab.bb.d[1]);
                else rigid_mul_R(A, cp[k], sp[k], s_tab.bb.ct[1], s_tab.bb.st[1], s_tab.bb.d[1]);
                rigid_mul_R(A, cs[k], ss[k], s_tab.bb.ct[2], s_tab.bb.st[2], s_tab.bb.d[2]);
                if (j + 1 < L) {  // R_4(omega_{j+1}) places the next residue's N
                    sincosf(k + 1 < K ? om[k + 1] : om_next, &so[k], &co[k]);
                    rigid_mul_R(A, co[k], so[k], s_tab.bb.ct[0], s_tab.bb.st[0], s_tab.bb.d[0]);
                }
            }
        }
        if (j0 < s1) rigid_reortho(A);  // the scan composes orthonormal operands

        // 2. tile-local frame of the first residue and its first atom
        Rigid X, Tot;
        int a0, tile_atoms;
        if (pack) {
            // segments: no look-back, each chain starts at R_0 = I and atom 0
            const bool head = ci < 0 || j0 == 0;
            X = block_seg_scan_rigid<NT>(A, head, s_rig, s_cnt);
            a0 = block_seg_scan_count<NT>(cnt, head, s_cnt2, s_fl2);
            if (ci >= 0 && threadIdx.x * K + K >= s_pack.off[ci + 1]) s_mtot[ci] = a0 + cnt;  // the chain's last thread
            if (threadIdx.x == 0) s_next = request_tile(ws.hdr + kHdrFwdNext);
            __syncthreads();
            if (threadIdx.x == 0) {
                int sb = 0;
                for (int i = 0; i < m; ++i) {
                    s_mbase[i] = sb;
                    sb += s_mtot[i];
                }
                s_mbase[m] = sb;
                bulk_store_wait_read();  // the previous tile's stage is read out before it is refilled
            }
            if (threadIdx.x < m)  // the record the backward reads: first atom 0, the chain's atom count
                store_rigid_g(ws.start + 4 * (size_t)s_pack.b[threadIdx.x] * ws.tmax, rigid_identity(), 0,
                              s_mtot[threadIdx.x]);
            __syncthreads();
            tile_atoms = ci >= 0 ? s_mtot[ci] : 0;
        } else {
            block_scan_rigid_count<NT>(A, cnt, s_rig, s_cnt, X, a0, Tot, tile_atoms);
            if (threadIdx.x == NT - 32 && t + 1 < T) publish_prefix_agg(ws, slot0 + t, Tot, tile_atoms);

            // 3. frame at the tile start and its first atom (one warp)
            if (threadIdx.x < 32) {
                int pc = 0;
                const Rigid P = gather_prefix(ws, slot0, t, pc);
                if (threadIdx.x == 0) {
                    s_next = request_tile(ws.hdr + kHdrFwdNext);  // after the last wait of this tile
                    store_rigid_g(s_start, P, pc, tile_atoms);
                    store_rigid_g(ws.start + 4 * (size_t)(slot0 + t), P, pc, tile_atoms);
                    bulk_store_wait_read();  // the previous tile's stage is read out before it is refilled
                }
            }
            __syncthreads();
        }
        int pc = 0;
        const Rigid P = pack ? rigid_identity() : load_rigid_prev(s_start, pc);
        const int requested = s_next;
        const int end_atom = pc + tile_atoms;
        const int nout = max(0, min(end_atom, Amax) - pc);
        // the tile's atoms go through the stage unless they do not fit in it
        // (a pack: every member's atoms, one after the other)
        const bool staged = pack ? s_mbase[m] <= CAP : tile_atoms <= CAP;
        const int sbase = pack && ci >= 0 ? s_mbase[ci] : 0;
        // a tile's stage starts at float (3 pc) mod 4, so that its 16-byte
        // aligned middle maps onto 16-byte aligned global memory (bulk store)
        const int soff = pack ? 0 : (3 * pc) & 3;
        float* dst = staged ? stage + soff + 3 * sbase : out + 3 * (size_t)pc;
        const int lim = staged ? CAP - sbase : Amax - pc;  // tile atoms at or past it are not written
        // LM: the tile's target rows come into their own stage (same layout) by a
        // bulk copy that runs while the atoms are placed
        bool lm_bulk = false;
        if constexpr (LM) {
            if (staged) lm_bulk = bulk_copy_range<NT>(target + (size_t)b * Amax * 3, stage_t, 3 * pc, 3 * (pc + nout), &s_bar);
        }

        // 4. atoms in the chain's frame
        if (j0 < s1) {
            Rigid M0 = t > 0 ? rigid_mul(P, X) : X;
            int a = a0;
            int ra[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int j = j0 + k;
                if (j >= s1) break;
                const int ty = type[k];
                ra[k] = pc + a;
                float* st = dst + 3 * a;
                const int room = lim - a;  // atoms of this residue that may be written
                auto put = [&](int idx, float3 r) {
                    if (idx < room) stage_atom(st, idx, r);
                };
                Rigid M1 = M0;
                rigid_mul_R(M1, cp[k], sp[k], s_tab.bb.ct[1], s_tab.bb.st[1], s_tab.bb.d[1]);
                Rigid M3 = M1;
                rigid_mul_R(M3, cs[k], ss[k], s_tab.bb.ct[2], s_tab.bb.st[2], s_tab.bb.d[2]);
                put(0, M0.t);  // N = M_0 0
                put(1, M1.t);  // CA = M_1 0
                put(2, M3.t);  // C = M_3 0
                if (ty != kBackboneCode) {  // O (a backbone-only residue has none)
                    const float4 o = s_tab.o_r0;
                    put(3, point_apply(M3, make_float3(o.x, o.y, o.z)));
                }
                // side-chain groups: S_k = S_{k-1} R(chi_k), S_0 = M_1 R'; atoms r = S_k r0
                Rigid S = M1;
                rigid_mul_Rx(S, s_tab.rp_c, s_tab.rp_s);
                if constexpr (PERM) {
                    // placed below, in the order of residue types: the record
                    const int i = threadIdx.x;
                    rec[0 * NT + i] = S.c0.x; rec[1 * NT + i] = S.c0.y; rec[2 * NT + i] = S.c0.z;
                    rec[3 * NT + i] = S.c1.x; rec[4 * NT + i] = S.c1.y; rec[5 * NT + i] = S.c1.z;
                    rec[6 * NT + i] = S.c2.x; rec[7 * NT + i] = S.c2.y; rec[8 * NT + i] = S.c2.z;
                    rec[9 * NT + i] = S.t.x; rec[10 * NT + i] = S.t.y; rec[11 * NT + i] = S.t.z;
#pragma unroll
                    for (int g = 0; g < kMaxGroups; ++g) rec[(12 + g) * NT + i] = chi[g][k];
                    rec[17 * NT + i] = __int_as_float(a);
                    rec[18 * NT + i] = __int_as_float(room);
                } else {
                    side_chain(S, ty, chi[0][k], chi[1][k], chi[2][k], chi[3][k], s_tab, put);
                }
                a += s_tab.n_atoms[ty];
                if (k + 1 < K && j + 1 < L) {  // the next residue's frame
                    M0 = M3;
                    rigid_mul_R(M0, co[k], so[k], s_tab.bb.ct[0], s_tab.bb.st[0], s_tab.bb.d[0]);
                }
            }
            // each residue's first atom, which the backward reads its atoms by
            // (a thread's K residues lie in one tile: tile starts are multiples
            // of 4; past the chain's end the entries are unused)
            store_k<K>(ws.ratom + (size_t)b * Lmax + j0, ra);
        }
        if constexpr (PERM) {
            // side chains in the order of residue types, so that the lanes of a
            // warp mostly build the same groups and atoms: a counting sort of the
            // tile's residues by type (the order within a type does not matter:
            // every atom's place is fixed), then thread i takes the i-th residue
            const int my_ty = j0 < s1 ? type[0] : kBackboneCode;  // code 20 and empty slots: no side chain
            const int my_rank = atomicAdd(&s_tcnt[my_ty], 1);
            rec[16 * NT + threadIdx.x] = __int_as_float(my_ty);
            __syncthreads();
            if (threadIdx.x < 32) {
                const int c = threadIdx.x < kNumTypes ? s_tcnt[threadIdx.x] : 0;
                int incl = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if ((int)threadIdx.x >= o) incl += y;
                }
                if (threadIdx.x < kNumTypes) s_tbase[threadIdx.x] = incl - c;
            }
            __syncthreads();
            perm[s_tbase[my_ty] + my_rank] = threadIdx.x;
            __syncthreads();
            const int r = perm[threadIdx.x];
            const int ty = __float_as_int(rec[16 * NT + r]);
            if (s_tab.n_groups[ty] > 0) {
                Rigid S;
                S.c0 = make_float3(rec[0 * NT + r], rec[1 * NT + r], rec[2 * NT + r]);
                S.c1 = make_float3(rec[3 * NT + r], rec[4 * NT + r], rec[5 * NT + r]);
                S.c2 = make_float3(rec[6 * NT + r], rec[7 * NT + r], rec[8 * NT + r]);
                S.t = make_float3(rec[9 * NT + r], rec[10 * NT + r], rec[11 * NT + r]);
                const int ar = __float_as_int(rec[17 * NT + r]), room_r = __float_as_int(rec[18 * NT + r]);
                float* st = dst + 3 * ar;
                auto put = [&](int idx, float3 rr) {
                    if (idx < room_r) stage_atom(st, idx, rr);
                };
                side_chain(S, ty, rec[12 * NT + r], rec[13 * NT + r], rec[14 * NT + r], rec[15 * NT + r], s_tab, put);
            }
        }
        if constexpr (LM) {
            if (staged) cp_async_wait_all();  // the ragged ends of the target rows
            if (lm_bulk) {
                mbar_wait(&s_bar, bphase);
                bphase ^= 1u;
            }
        }
        fence_proxy_async();  // the stage writes, ordered before the bulk store that reads them
        __syncthreads();
        {
            // the next tile's angle rows and sequence into L2 while this tile is stored
            if (requested < ntiles && threadIdx.x < 64) {
                const int2 cn = ws.tiles[requested];
                const int row = threadIdx.x >> 3, part = threadIdx.x & 7;  // 8 rows x 8 parts of the tile
                if (cn.x >= 0) {
                    const int Ln = clamp_length(lengths, cn.x, Lmax);
                    const int Tn = fa_num_tiles(Ln, TILE);
                    const int sn = fa_tile_start(Ln, Tn, cn.y), en = fa_tile_start(Ln, Tn, cn.y + 1);
                    const int per = (en - sn + 7) / 8;
                    const int jn = sn + part * per;
                    if (jn < en) {
                        const char* base = row < 7 ? reinterpret_cast<const char*>(angles + ((size_t)cn.x * 7 + row) * Lmax + jn)
                                                   : reinterpret_cast<const char*>(seq + (size_t)cn.x * Lmax + jn);
                        const int bytes = (row < 7 ? 4 : 1) * min(per, en - jn);
                        for (int o = 0; o < bytes; o += 128) prefetch_l2(base + o);
                    }
                }
            }
        }
        // 5. the stage out
        if (pack) {  // member by member (block-wide loops)
            for (int i = 0; i < m; ++i) {
                const int n = s_mtot[i];
                float* oi = coords + (size_t)s_pack.b[i] * Amax * 3;
                if (staged) store_range<NT>(oi, stage + 3 * s_mbase[i], 0, 3 * min(n, Amax));
                if (threadIdx.x == 0) {
                    num_atoms[s_pack.b[i]] = n;
                    if (n > Amax) flag_status(TPL_STATUS_TOO_MANY_ATOMS);
                }
                if (!(ws.flags & TPL_FLAG_PADDING_ZEROED)) zero_range<NT>(oi, 3 * min(n, Amax), 3 * Amax);
            }
        } else {
            if (end_atom > Amax && threadIdx.x == 0) flag_status(TPL_STATUS_TOO_MANY_ATOMS);
            if (staged) bulk_store_range<NT>(out, stage, 3 * pc, 3 * (pc + nout));
            if (t == T - 1) {
                if (threadIdx.x == 0) num_atoms[b] = end_atom;
                if (!(ws.flags & TPL_FLAG_PADDING_ZEROED)) zero_range<NT>(out, 3 * min(end_atom, Amax), 3 * Amax);
            }
        }
        if constexpr (LM) {  // (never with PACK: the fused step's schedule has no packs)
            const float* tg = target + (size_t)b * Amax * 3;
            const float3 x0 = make_float3(__ldg(tg), __ldg(tg + 1), __ldg(tg + 2));
            // the tile's coordinates: the stage, or (tiles that bypass it) this
            // CTA's own global writes, visible after the barrier above
            const float* ys = staged ? stage + soff : out + 3 * (size_t)pc;
            const float* xs = staged ? stage_t + soff : tg + 3 * (size_t)pc;  // the target: its stage, or global
            float m[17];
#pragma unroll
            for (int q = 0; q < 17; ++q) m[q] = 0.f;
            for (int a = threadIdx.x; a < nout; a += NT) {
                const float3 dx = make_float3(xs[3 * a] - x0.x, xs[3 * a + 1] - x0.y, xs[3 * a + 2] - x0.z);
                const float3 dy = make_float3(ys[3 * a], ys[3 * a + 1], ys[3 * a + 2]);
                m[0] += dx.x; m[1] += dx.y; m[2] += dx.z;
                m[3] += dy.x; m[4] += dy.y; m[5] += dy.z;
                m[6] = fmaf(dx.x, dy.x, m[6]); m[7] = fmaf(dx.x, dy.y, m[7]); m[8] = fmaf(dx.x, dy.z, m[8]);
                m[9] = fmaf(dx.y, dy.x, m[9]); m[10] = fmaf(dx.y, dy.y, m[10]); m[11] = fmaf(dx.y, dy.z, m[11]);
                m[12] = fmaf(dx.z, dy.x, m[12]); m[13] = fmaf(dx.z, dy.y, m[13]); m[14] = fmaf(dx.z, dy.z, m[14]);
                m[15] += f3_dot(dx, dx);
                m[16] += f3_dot(dy, dy);
            }
            fence_proxy_async();  // the target stage's reads, ordered before the next tile's bulk copy
            // block sum: warp shuffles, then the warp sums in a fixed order
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
            for (int q = 0; q < 17; ++q) {
                float x = m[q];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                m[q] = x;
            }
            if (lane == 0)
#pragma unroll
                for (int q = 0; q < 17; ++q) s_mom[warp][q] = m[q];
            __syncthreads();
            if (threadIdx.x < 17) {
                float x = 0.f;
                for (int w = 0; w < NW; ++w) x += s_mom[w][threadIdx.x];
                ws.tmom[(size_t)(slot0 + t) * 20 + threadIdx.x] = x;
            }
        }
        v = next_tile(requested, &s_v);
    }
    if (threadIdx.x == 0) bulk_store_wait_all();  // the last tile's bulk store is in global memory
}


__device__ __forceinline__ float3 unit3(float3 v) { return f3_scale(rsqrtf(f3_dot(v, v)), v); }

// Side-chain part of a residue's backward (Eq. 1): its atoms in decreasing
// group order, the running suffix (sum r x g, sum g) over the groups, and each
// free chi's gradient u . (sum r x g - p x sum g) at the end of its group, into
// gchi[group][k].  Returns the residue's side-chain sums.  Rp(a) and G(a, r)
// give atom a's position and coordinate gradient; add accumulates a Sum6.
template <int K, typename RpF, typename GF, typename AddF>
__device__ __forceinline__ Sum6 side_chain_sums(int ty, int a, int nat, float (&gchi)[kMaxGroups][K], int k,
                                                const FaTable& tab, RpF& Rp, GF& G, AddF& add) {
    const int nchi = tab.n_chi[ty];
    Sum6 suf = sum6_zero();
    for (int e = nat - 5; e >= 0; --e) {
        const int wv = (int)tab.side[ty][e].w;
        const int grp = wv >> 4;
        const float3 r = Rp(a + (wv & 15));
        add(suf, r, G(a + (wv & 15), r));
        const bool last_of_group = (e == 0) || (((int)tab.side[ty][e - 1].w >> 4) != grp);
        if (last_of_group && grp <= nchi) {
            const int o1 = tab.origin[ty][grp - 1];
            const int o0 = grp >= 2 ? tab.origin[ty][grp - 2] : 1;
            const float3 p = Rp(a + o1);
            const float val = f3_dot(unit3(f3_sub(p, Rp(a + o0))), f3_sub(suf.c, f3_cross(p, suf.g)));
#pragma unroll
            for (int c = 0; c < kMaxGroups; ++c)
                if (c == grp - 1) gchi[c][k] = val;
        }
    }
    return suf;
}

// ---------------------------------------------------------------------------
// K4': backward from the forward's coordinates.  For a frame with x axis u and
// origin p, dL/dalpha = u . sum_{k downstream} (r_k - p) x g_k; axes and
// origins come from atom positions (phi: N->CA, psi: CA->C, omega: C_{j-1}->N_j,
// chi_k: origin of group k-1 -> origin of group k).  One tile per step of a
// persistent CTA, the tiles of a chain taken last to first:
//  1. the tile's coordinates and, in a second stage, their gradient (with LR
//     the target) come into shared memory by bulk copies of the TMA engine
//     (the forward recorded each tile's first atom and atom count, and every
//     residue's first atom);
//  2. each thread walks its K residues: every atom's gradient (read, or the
//     LRMSD gradient formed from the coordinates, the target and the LRMSD
//     state), the residue's (sum r x g, sum g), and the chi gradients from the
//     suffix over its side-chain groups;
//  3. a block suffix scan of the threads' sums and one warp's look-back over
//     the chain's later tiles give, for every thread, the sums over all later
//     atoms of the chain;
//  4. each thread walks its residues back, adding each residue's sums, and
//     forms phi, psi and omega from them and from its N, C and O terms.
// ---------------------------------------------------------------------------
template <int NT, int K, bool LR, bool PACK>
__global__ void __launch_bounds__(NT, (fa_min_blocks_for<NT, K>(fa_bwd_coords_smem<NT, K, PACK>()))) fa_bwd_coords_kernel(
    const uint8_t* __restrict__ seq, const int32_t* __restrict__ lengths, int B, int Lmax, int Amax,
    const float* __restrict__ coords, const float* __restrict__ grad_coords,
    float* __restrict__ grad_angles, ChainWs ws, LrmsdGrad lg, const __grid_constant__ FaTable tab) {
    constexpr int NW = NT / 32;
    constexpr int TILE = NT * K;
    constexpr int CAP = fa_stage_atoms<NT, K>();
    __shared__ FaTable s_tab;
    __shared__ float s6[6 * (NW + 1)];
    __shared__ float s_later[6];
    __shared__ int s_v, s_next;
    __shared__ PackS s_pack;  // a pack of whole short chains
    __shared__ int s_fl[NW + 1];
    __shared__ int s_mn[kMaxPack], s_mbase[kMaxPack + 1];  // atoms per member, stage offsets (floats)
    __shared__ __align__(8) uint64_t s_bar;  // completes when a tile's bulk copy has landed
    extern __shared__ float4 s_dyn[];
    float* st_r = reinterpret_cast<float*>(s_dyn);  // the tile's coordinates
    float* st_g = st_r + fa_smem<NT, K>() / sizeof(float);  // their gradient (or target), same layout
    constexpr bool PERM = fa_bwd_perm<NT, K, PACK>();
    int* s_rty = reinterpret_cast<int*>(st_r + 2 * fa_smem<NT, K>() / sizeof(float));  // PERM: residue type
    int* s_ra = s_rty + NT;                                  // PERM: first atom
    int* s_perm = s_ra + NT;                                 // PERM: thread of the i-th residue in type order
    float* s_suf = reinterpret_cast<float*>(s_perm + NT);    // PERM: side-chain sums, word q at q * NT + i
    __shared__ int s_tcnt[kNumTypes], s_tbase[kNumTypes];

    if (!ws_matches(ws, TILE, B, Lmax)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) flag_status(TPL_STATUS_BAD_WORKSPACE);
        for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < (size_t)B * 7 * Lmax; i += (size_t)gridDim.x * NT)
            grad_angles[i] = 0.f;
        return;
    }
    load_table(s_tab, tab);
    if (threadIdx.x == 0) mbar_init(&s_bar);  // visible after take_tile's barrier
    unsigned bphase = 0;                      // the barrier phase the next bulk copy completes
    const int ntiles = ws.hdr[kHdrTiles];
    int* counter = ws.bflag + ws.slots;
    int v = take_tile(counter, &s_v);
    while (v < ntiles) {
        const int2 ct = ws.tiles[v];
        if (PERM && threadIdx.x < kNumTypes) s_tcnt[threadIdx.x] = 0;  // used after the staging barrier
        // a tile of one chain (the chain's tiles taken last to first), or a
        // pack of whole chains in slots of K residues (segmented sums)
        if (ct.x < 0 && !PACK) {
            // a pack, but this backward was not built for packs (the forward
            // ran with another schedule than these options name)
            if (threadIdx.x == 0) flag_status(TPL_STATUS_BAD_WORKSPACE);
            for (int i = 0; i < ct.y; ++i) {
                float* gi = grad_angles + (size_t)ws.order[-1 - ct.x + i] * 7 * Lmax;
                for (int q = threadIdx.x; q < 7 * Lmax; q += NT) gi[q] = 0.f;
            }
            v = next_tile(request_tile(counter), &s_v);
            continue;
        }
        const bool pack = PACK && ct.x < 0;
        int m = 0, ci = -1;
        if (pack) {
            m = ct.y;
            load_pack<K>(ws, lengths, Lmax, -1 - ct.x, m, s_pack);
            ci = pack_member(s_pack, m, threadIdx.x * K);
            if (threadIdx.x == 0) {
                int sb = 0;
                for (int i = 0; i < m; ++i) {
                    int pc_i, n_i;
                    tile_record(ws, s_pack.b[i] * ws.tmax, pc_i, n_i);
                    s_mn[i] = min(n_i, Amax);
                    s_mbase[i] = sb;
                    sb += (3 * s_mn[i] + 3) & ~3;  // each member 16-byte aligned in the stage
                }
                s_mbase[m] = sb;
            }
            __syncthreads();
        }
        const int b = pack ? s_pack.b[ci >= 0 ? ci : 0] : ct.x;
        const int L = pack ? (ci >= 0 ? s_pack.len[ci] : 0) : clamp_length(lengths, b, Lmax);
        const int T = pack ? 1 : fa_num_tiles(L, TILE);
        const int t = pack ? 0 : T - 1 - ct.y;  // last tile first
        const int s0 = pack ? 0 : fa_tile_start(L, T, t), s1 = pack ? L : fa_tile_start(L, T, t + 1);
        const int slot0 = b * ws.tmax;
        const float* r_in = coords + (size_t)b * Amax * 3;
        float* ga = grad_angles + (size_t)b * 7 * Lmax;

        // 1. the tile's coordinates into the stage (unless they do not fit)
        int pc = 0, n = 0;
        if (!pack) tile_record(ws, slot0 + t, pc, n);
        else if (ci >= 0) n = s_mn[ci];
        const int a_end = min(pc + n, Amax);  // the tile's atoms present in the output
        const bool staged = pack ? s_mbase[m] <= 3 * CAP : n <= CAP;
        bool bulk = false;  // the tile's aligned middle comes in by one bulk copy
        if (staged) {
            if (pack) {
                for (int i = 0; i < m; ++i)
                    async_copy_range<NT>(coords + (size_t)s_pack.b[i] * Amax * 3, st_r + s_mbase[i], 0, 3 * s_mn[i]);
            } else {
                const float* g_in = (LR ? lg.target : grad_coords) + (size_t)b * Amax * 3;
                bulk = bulk_copy_range2<NT>(r_in, st_r, g_in, st_g, 3 * pc, 3 * a_end, &s_bar);
            }
        }
        const bool staged_g = staged && !pack;  // G comes from st_g at the coordinates' offsets
        // atom a is at rb[rofs + 3 a]
        const float* rb = staged ? st_r + (pack && ci >= 0 ? s_mbase[ci] : 0) : r_in;
        const int rofs = staged && !pack ? ((3 * pc) & 3) - 3 * pc : 0;
        const int j0 = pack ? (ci >= 0 ? threadIdx.x * K - s_pack.off[ci] : 0) : s0 + threadIdx.x * K;
        int type[K], a0[K];
        if (j0 < s1) {
            load_k<K>(seq + (size_t)b * Lmax + j0, type);
            load_k<K>(ws.ratom + (size_t)b * Lmax + j0, a0);
        }
        int aprev = 0;  // first atom of the residue before the thread's first one
        if (j0 < s1 && j0 > 0) aprev = __ldg(ws.ratom + (size_t)b * Lmax + j0 - 1);
        float3 u0 = make_float3(0.f, 0.f, 0.f), u1 = u0, u2 = u0, xc = u0, yc = u0;
        float w = 0.f;
        if constexpr (LR) {
            const float* st = lg.state + 16 * (size_t)b;
            u0 = make_float3(__ldg(st), __ldg(st + 1), __ldg(st + 2));
            u1 = make_float3(__ldg(st + 3), __ldg(st + 4), __ldg(st + 5));
            u2 = make_float3(__ldg(st + 6), __ldg(st + 7), __ldg(st + 8));
            xc = make_float3(__ldg(st + 9), __ldg(st + 10), __ldg(st + 11));
            yc = make_float3(__ldg(st + 12), __ldg(st + 13), __ldg(st + 14));
            w = __ldg(lg.grad_lrmsd + b) * __ldg(st + 15);
        }
        auto Rp = [&](int a) { return make_float3(rb[rofs + 3 * a], rb[rofs + 3 * a + 1], rb[rofs + 3 * a + 2]); };
        // the coordinate gradient of atom a at position r: read, or formed from
        // the LRMSD state
        auto G = [&](int a, float3 r) {
            float3 v3;
            if (staged_g) {
                v3 = make_float3(st_g[rofs + 3 * a], st_g[rofs + 3 * a + 1], st_g[rofs + 3 * a + 2]);
            } else {
                const float* src = LR ? lg.target + ((size_t)b * Amax + a) * 3 : grad_coords + ((size_t)b * Amax + a) * 3;
                v3 = make_float3(__ldg(src), __ldg(src + 1), __ldg(src + 2));
            }
            if constexpr (!LR) return v3;
            const float3 xp = f3_sub(v3, xc), yp = f3_sub(r, yc);
            const float3 d = make_float3(yp.x - f3_dot(u0, xp), yp.y - f3_dot(u1, xp), yp.z - f3_dot(u2, xp));
            return f3_scale(w, d);
        };
        auto add = [](Sum6& s, float3 r, float3 g) {
            s.c = f3_add(s.c, f3_cross(r, g));
            s.g = f3_add(s.g, g);
        };
        cp_async_wait_all();
        if (bulk) {
            mbar_wait(&s_bar, bphase);
            bphase ^= 1u;
        }
        __syncthreads();

        // 2. residue sums and chi gradients; with up to two residues per thread
        // the N and C, O sums and the axis atoms are kept for step 4, with more
        // they are formed again there
        constexpr bool KEEP = K <= 2;
        Sum6 own[K];
        Sum6 tsum = sum6_zero();
        bool in_range[K];
        float gchi[kMaxGroups][K];
        Sum6 nkeep[KEEP ? K : 1], cokeep[KEEP ? K : 1];
        float3 rkeep[KEEP ? K : 1][3];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int j = j0 + k;
            own[k] = sum6_zero();
            in_range[k] = false;
#pragma unroll
            for (int c = 0; c < kMaxGroups; ++c) gchi[c][k] = 0.f;
            if (j >= s1) continue;
            int ty = type[k];
            if (ty >= kNumTypes) {
                flag_status(TPL_STATUS_BAD_RESIDUE);
                ty = kGlyCode;
            }
            type[k] = ty;
            const int nat = s_tab.n_atoms[ty];
            const int a = a0[k];
            in_range[k] = a >= pc && a + nat <= a_end;
            if (in_range[k]) {
                Sum6 s = sum6_zero();
                if constexpr (KEEP) {
                    Sum6 ns = sum6_zero(), co = sum6_zero(), ca = sum6_zero();
                    const float3 rN = Rp(a), rCA = Rp(a + 1), rC = Rp(a + 2);
                    add(ns, rN, G(a, rN));
                    add(ca, rCA, G(a + 1, rCA));
                    add(co, rC, G(a + 2, rC));
                    if (nat > 3) {  // O (a backbone-only residue has none)
                        const float3 rO = Rp(a + 3);
                        add(co, rO, G(a + 3, rO));
                    }
                    s = sum6_add(sum6_add(ns, ca), co);
                    nkeep[k] = ns;
                    cokeep[k] = co;
                    rkeep[k][0] = rN;
                    rkeep[k][1] = rCA;
                    rkeep[k][2] = rC;
                } else {
#pragma unroll
                    for (int q = 0; q < min(4, nat); ++q) {  // N, CA, C, O
                        const float3 r = Rp(a + q);
                        add(s, r, G(a + q, r));
                    }
                }
                if constexpr (PERM) {
                    own[k] = s;  // the side chain's sums are added after the type-ordered pass
                } else {
                    const Sum6 suf = side_chain_sums(ty, a, nat, gchi, k, s_tab, Rp, G, add);
                    own[k] = sum6_add(s, suf);
                    tsum = sum6_add(tsum, own[k]);
                }
            }
        }
        if constexpr (PERM) {
            // side chains in the order of residue types (as in the forward):
            // thread i takes the i-th residue, writes its chi gradients and hands
            // its side-chain sums back through shared memory
            const int my_ty = (j0 < s1 && in_range[0]) ? type[0] : kBackboneCode;  // code 20: no side chain
            const int my_rank = atomicAdd(&s_tcnt[my_ty], 1);
            s_rty[threadIdx.x] = my_ty;
            s_ra[threadIdx.x] = j0 < s1 ? a0[0] : 0;
            __syncthreads();
            if (threadIdx.x < 32) {
                const int c = threadIdx.x < kNumTypes ? s_tcnt[threadIdx.x] : 0;
                int incl = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if ((int)threadIdx.x >= o) incl += y;
                }
                if (threadIdx.x < kNumTypes) s_tbase[threadIdx.x] = incl - c;
            }
            __syncthreads();
            s_perm[s_tbase[my_ty] + my_rank] = threadIdx.x;
            __syncthreads();
            const int r = s_perm[threadIdx.x];
            const int ty = s_rty[r];
            const int jr = s0 + r;  // the residue (one per thread)
            float gc[kMaxGroups][1] = {{0.f}, {0.f}, {0.f}, {0.f}};
            Sum6 suf = sum6_zero();
            if (ty != kBackboneCode) suf = side_chain_sums(ty, s_ra[r], (int)s_tab.n_atoms[ty], gc, 0, s_tab, Rp, G, add);
            if (jr < s1) {
#pragma unroll
                for (int c = 0; c < kMaxGroups; ++c) ga[(3 + c) * Lmax + jr] = gc[c][0];
            }
            s_suf[0 * NT + r] = suf.c.x; s_suf[1 * NT + r] = suf.c.y; s_suf[2 * NT + r] = suf.c.z;
            s_suf[3 * NT + r] = suf.g.x; s_suf[4 * NT + r] = suf.g.y; s_suf[5 * NT + r] = suf.g.z;
            __syncthreads();
            if (j0 < s1 && in_range[0]) {
                const int i = threadIdx.x;
                Sum6 sc;
                sc.c = make_float3(s_suf[0 * NT + i], s_suf[1 * NT + i], s_suf[2 * NT + i]);
                sc.g = make_float3(s_suf[3 * NT + i], s_suf[4 * NT + i], s_suf[5 * NT + i]);
                own[0] = sum6_add(own[0], sc);
                tsum = own[0];
            }
        }
        // A thread's K residues lie in one tile (tile starts are multiples of 4),
        // except past the chain's end, where the last tile writes zeros anyway.
        if (!PERM && j0 < s1) {
#pragma unroll
            for (int c = 0; c < kMaxGroups; ++c) store_k<K>(ga + (3 + c) * Lmax + j0, gchi[c]);
        }

        // 3. sums over the later threads of the tile and the chain's later tiles
        Sum6 after, total;
        if (pack) {  // within each chain only: tail flags at the chains' last threads
            const bool tail = ci < 0 || threadIdx.x * K + K >= s_pack.off[ci + 1];
            after = block_seg_suffix_sum6<NT>(tsum, tail, s6, s_fl);
            if (threadIdx.x == 0) {
                for (int q = 0; q < 6; ++q) s_later[q] = 0.f;
                s_next = request_tile(counter);
            }
        } else {
            block_suffix_sum6<NT>(tsum, s6, after, total);
            if (threadIdx.x == NT - 32 && t > 0) publish_suffix_agg(ws, slot0 + t, total);
            if (threadIdx.x < 32) {
                const Sum6 later = gather_suffix(ws, slot0, t, T);
                if (threadIdx.x == 0) {
                    s_later[0] = later.c.x; s_later[1] = later.c.y; s_later[2] = later.c.z;
                    s_later[3] = later.g.x; s_later[4] = later.g.y; s_later[5] = later.g.z;
                    s_next = request_tile(counter);  // after the last wait of this tile
                }
            }
        }
        __syncthreads();
        const int requested = s_next;
        Sum6 A;
        A.c = f3_add(after.c, make_float3(s_later[0], s_later[1], s_later[2]));
        A.g = f3_add(after.g, make_float3(s_later[3], s_later[4], s_later[5]));

        // 4. phi, psi, omega, residues last to first
        float gphi[K], gpsi[K], gomg[K];
#pragma unroll
        for (int k = K - 1; k >= 0; --k) {
            const int j = j0 + k;
            gphi[k] = gpsi[k] = gomg[k] = 0.f;
            if (j >= s1) continue;
            if (in_range[k]) {
                const int a = a0[k];
                float3 rN, rCA, rC;
                Sum6 nsum, co;
                if constexpr (KEEP) {
                    rN = rkeep[k][0];
                    rCA = rkeep[k][1];
                    rC = rkeep[k][2];
                    nsum = nkeep[k];
                    co = cokeep[k];
                } else {
                    rN = Rp(a);
                    rCA = Rp(a + 1);
                    rC = Rp(a + 2);
                    nsum = sum6_zero();
                    co = sum6_zero();
                    add(nsum, rN, G(a, rN));
                    add(co, rC, G(a + 2, rC));
                    if (type[k] != kBackboneCode) {  // O
                        const float3 rO = Rp(a + 3);
                        add(co, rO, G(a + 3, rO));
                    }
                }
                Sum6 x = sum6_add(co, A);
                gpsi[k] = f3_dot(unit3(f3_sub(rC, rCA)), f3_sub(x.c, f3_cross(rC, x.g)));
                Sum6 rest;  // every atom of the residue but N, and everything after it
                rest.c = f3_sub(own[k].c, nsum.c);
                rest.g = f3_sub(own[k].g, nsum.g);
                x = sum6_add(rest, A);
                gphi[k] = f3_dot(unit3(f3_sub(rCA, rN)), f3_sub(x.c, f3_cross(rCA, x.g)));
                if (j > 0) {  // C of the previous residue
                    const int ap = (k > 0 ? a0[k - 1] : aprev) + 2;
                    const float3 rCp = (staged && ap >= pc) ? Rp(ap) : make_float3(__ldg(r_in + 3 * (size_t)ap),
                                                                                    __ldg(r_in + 3 * (size_t)ap + 1),
                                                                                    __ldg(r_in + 3 * (size_t)ap + 2));
                    x = sum6_add(own[k], A);
                    gomg[k] = f3_dot(unit3(f3_sub(rN, rCp)), f3_sub(x.c, f3_cross(rN, x.g)));
                }
            }
            A = sum6_add(A, own[k]);
        }
        if (j0 < s1) {
            store_k<K>(ga + j0, gphi);
            store_k<K>(ga + Lmax + j0, gpsi);
            store_k<K>(ga + 2 * Lmax + j0, gomg);
        }
        if (pack) {
            if (!(ws.flags & TPL_FLAG_PADDING_ZEROED))  // rows past each chain's last residue
                for (int i = 0; i < m; ++i) {
                    float* gi = grad_angles + (size_t)s_pack.b[i] * 7 * Lmax;
                    for (int jj = s_pack.len[i] + threadIdx.x; jj < Lmax; jj += NT)
#pragma unroll
                        for (int r = 0; r < 7; ++r) gi[r * Lmax + jj] = 0.f;
                }
        } else if (t == T - 1 && !(ws.flags & TPL_FLAG_PADDING_ZEROED)) {  // rows past the chain's last residue
            for (int i = L + threadIdx.x; i < Lmax; i += NT)
#pragma unroll
                for (int r = 0; r < 7; ++r) ga[r * Lmax + i] = 0.f;
        }
        fence_proxy_async();  // this tile's stage reads, ordered before the next tile's bulk copy
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
    load_table(s_tab, tab);
    const int ntiles = ws.hdr[kHdrTiles];
    int* counter = ws.bflag + ws.slots;
    int v = take_tile(counter, &s_v);
    while (v < ntiles) {
        const int2 ct = ws.tiles[v];
        if (ct.x < 0) {
            // a pack of whole chains (a packed forward): frames are rebuilt per
            // tile of one chain only -- the packed backward reads the coordinates
            if (threadIdx.x == 0) flag_status(TPL_STATUS_BAD_WORKSPACE);
            for (int i = 0; i < ct.y; ++i) {
                float* gi = grad_angles + (size_t)ws.order[-1 - ct.x + i] * 7 * Lmax;
                for (int q = threadIdx.x; q < 7 * Lmax; q += NT) gi[q] = 0.f;
            }
            v = next_tile(request_tile(counter), &s_v);
            continue;
        }
        const int b = ct.x;
        const int L = clamp_length(lengths, b, Lmax);
        const int T = fa_num_tiles(L, NT);
        const int t = T - 1 - ct.y;  // last tile first
        const int s0 = fa_tile_start(L, T, t), s1 = fa_tile_start(L, T, t + 1);
        const int slot0 = b * ws.tmax;
        const float* ang = angles + (size_t)b * 7 * Lmax;
        const uint8_t* sq = seq + (size_t)b * Lmax;
        const float* g_in = grad_coords + (size_t)b * Amax * 3;
        float* ga = grad_angles + (size_t)b * 7 * Lmax;

        const int j = s0 + threadIdx.x;
        const bool valid = j < s1;
        const int type = residue_type(sq, j, valid);
        float sp = 0.f, cp = 1.f, ss = 0.f, cs = 1.f;
        // the forward's frames exactly: the same residue transform, re-orthonormalised
        Rigid A = rigid_identity();
        if (valid) {
            A = residue_transform(s_tab, ang, Lmax, j, L, sp, cp, ss, cs);
            rigid_reortho(A);
        }
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
            if (type != kBackboneCode) {  // O
                const float4 o = s_tab.o_r0;
                add(csum, point_apply(M3, make_float3(o.x, o.y, o.z)), gat(3));
            }
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
        if (valid) {
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
        if (t == T - 1 && !(ws.flags & TPL_FLAG_PADDING_ZEROED)) {  // rows past the chain's last residue
            for (int i = L + threadIdx.x; i < Lmax; i += NT)
#pragma unroll
                for (int r = 0; r < 7; ++r) ga[r * Lmax + i] = 0.f;
        }
        v = next_tile(requested, &s_v);
    }
}

// ---------------------------------------------------------------------------
// K4q: the paper's depth-first form of Eq. 1 as a comparator: each angle's
// derivative sums, over every atom that the angle moves, the lever term
// g_k . (u x (r_k - p)) = u . ((r_k - p) x g_k), from the forward's
// coordinates -- O(L) work per backbone angle, O(L^2) per chain.  One thread
// per (residue, angle): kQRes residues x 7 angles per CTA; the CTA walks the
// chain's atoms from its first residue on in shared-memory tiles.  An angle
// of residue j moves every atom of the later residues (phi, psi, omega) and,
// in residue j: phi and omega all atoms, psi the C and O group, chi_k the
// side-chain groups k and beyond.  Axes and pivots as in K4'.
// ---------------------------------------------------------------------------
constexpr int kQNT = 128;
constexpr int kQRes = kQNT / 7;  // 18 residues, 126 angle slots

__global__ void __launch_bounds__(kQNT) fa_bwd_quadratic_kernel(
    const uint8_t* __restrict__ seq, const int32_t* __restrict__ lengths, int Lmax, int Amax,
    const float* __restrict__ coords, const float* __restrict__ grad_coords, float* __restrict__ grad_angles,
    const __grid_constant__ FaTable tab) {
    __shared__ float3 s_r[kQNT], s_g[kQNT];
    __shared__ int s_first[kQRes + 1];  // first atom of the CTA's residues (and past the last)
    __shared__ int s_red[kQNT / 32];
    const int b = blockIdx.y;
    const int L = clamp_length(lengths, b, Lmax);
    const int j0 = blockIdx.x * kQRes;
    const uint8_t* sq = seq + (size_t)b * Lmax;
    auto type_of = [&](int j) {
        const int c = sq[j];
        if (c >= kNumTypes) {
            flag_status(TPL_STATUS_BAD_RESIDUE);
            return kGlyCode;
        }
        return c;
    };
    // atoms before residue j0 (block sum), then the CTA's residues (thread 0)
    int before = 0;
    for (int j = threadIdx.x; j < min(j0, L); j += kQNT) before += tab.n_atoms[type_of(j)];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) before += __shfl_xor_sync(0xffffffffu, before, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = before;
    __syncthreads();
    if (threadIdx.x == 0) {
        int a = 0;
        for (int w = 0; w < kQNT / 32; ++w) a += s_red[w];
        for (int q = 0; q <= kQRes; ++q) {
            s_first[q] = a;
            if (j0 + q < L) a += tab.n_atoms[type_of(j0 + q)];
        }
    }
    __syncthreads();
    const int a_begin = s_first[0];
    int a_end = 0;  // atoms of the chain
    {
        int rest = 0;
        for (int j = j0 + kQRes + threadIdx.x; j < L; j += kQNT) rest += tab.n_atoms[type_of(j)];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rest += __shfl_xor_sync(0xffffffffu, rest, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = rest;
        __syncthreads();
        for (int w = 0; w < kQNT / 32; ++w) a_end += s_red[w];
        a_end += s_first[kQRes];
    }
    const bool over = a_end > Amax;  // flagged by the forward; nothing is read past Amax
    const int jl = threadIdx.x / 7, ang = threadIdx.x % 7;  // ang: 0 phi, 1 psi, 2 omega, 3.. chi
    const int j = j0 + jl;
    const float* r_in = coords + (size_t)b * Amax * 3;
    const float* g_in = grad_coords + (size_t)b * Amax * 3;
    bool active = jl < kQRes && j < L && !over;
    int ty = kGlyCode, a0 = 0, a1 = 0;
    unsigned groups = 0x7fu;  // rigid groups of residue j the angle moves (bit g: group g)
    float3 u = make_float3(0.f, 0.f, 0.f), p = u;
    if (active) {
        ty = type_of(j);
        a0 = s_first[jl];
        a1 = s_first[jl + 1];
        auto at = [&](int i) { return make_float3(r_in[3 * i], r_in[3 * i + 1], r_in[3 * i + 2]); };
        if (ang == 0) {  // phi: N -> CA, all but N
            p = at(a0 + 1);
            u = f3_sub(p, at(a0));
            groups = 0x7eu;
        } else if (ang == 1) {  // psi: CA -> C, the C and O group
            p = at(a0 + 2);
            u = f3_sub(p, at(a0 + 1));
            groups = 0x04u;
        } else if (ang == 2) {  // omega: C_{j-1} -> N_j (omega_0: R_0 = I, no angle)
            active = j > 0;
            if (active) {
                p = at(a0);
                u = f3_sub(p, at(a0 - tab.n_atoms[type_of(j - 1)] + 2));
            }
        } else {  // chi_k, k = ang - 3: origin of group k-1 (CA for k = 0) -> origin of group k
            const int k = ang - 3;
            active = k < tab.n_chi[ty];
            if (active) {
                p = at(a0 + tab.origin[ty][k]);
                u = f3_sub(p, at(a0 + (k == 0 ? 1 : tab.origin[ty][k - 1])));
                groups = 0x7fu & ~((1u << (3 + k)) - 1u);
            }
        }
        if (active) u = f3_scale(rsqrtf(f3_dot(u, u)), u);
    }
    // chi angles move atoms of their own residue only
    const int a_stop = active ? (ang >= 3 ? a1 : a_end) : 0;
    float3 c = make_float3(0.f, 0.f, 0.f);  // sum over moved atoms of (r_k - p) x g_k
    const int a_last = over ? a_begin : a_end;
    for (int t0 = a_begin; t0 < a_last; t0 += kQNT) {
        const int k = t0 + threadIdx.x;
        __syncthreads();
        s_r[threadIdx.x] = k < a_last ? make_float3(r_in[3 * k], r_in[3 * k + 1], r_in[3 * k + 2])
                                      : make_float3(0.f, 0.f, 0.f);
        s_g[threadIdx.x] = k < a_last ? make_float3(g_in[3 * k], g_in[3 * k + 1], g_in[3 * k + 2])
                                      : make_float3(0.f, 0.f, 0.f);
        __syncthreads();
        const int lo = max(t0, a0), hi = min(t0 + kQNT, a_stop);
        for (int m = lo; m < hi; ++m) {
            // atoms of residue j: only the groups the angle moves
            if (m < a1 && !((groups >> tab.atom_grp[ty][m - a0]) & 1u)) continue;
            c = f3_add(c, f3_cross(f3_sub(s_r[m - t0], p), s_g[m - t0]));
        }
    }
    if (jl < kQRes && j < Lmax)
        grad_angles[(size_t)b * 7 * Lmax + (size_t)ang * Lmax + j] = active ? f3_dot(u, c) : 0.f;
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

template <int NT, int K, bool LM, bool PACK>
cudaError_t fa_fwd_t(const float* angles, const uint8_t* seq, const int32_t* lengths, int Lmax,
                     int Amax, float* coords, int32_t* num_atoms, const ChainWs& ws,
                     cudaStream_t s, const float* target) {
    const size_t smem = fa_fwd_smem<NT, K, LM, PACK>();
    static bool done[64] = {false};
    cudaError_t e = smem_attr_once(fa_fwd_kernel<NT, K, LM, PACK>, (int)smem, done);
    if (e != cudaSuccess) return e;
    const int grid = persistent_grid((const void*)fa_fwd_kernel<NT, K, LM, PACK>, NT, smem);
    fa_fwd_kernel<NT, K, LM, PACK><<<grid, NT, smem, s>>>(angles, seq, lengths, Lmax, Amax, coords, num_atoms,
                                                          ws, target, fa_table());
    return cudaGetLastError();
}

template <int NT, int K, bool LR, bool PACK>
cudaError_t fa_bwd_coords_t(const uint8_t* seq, const int32_t* lengths, int B, int Lmax, int Amax,
                            const float* coords, const float* grad_coords, float* grad_angles,
                            const ChainWs& ws, LrmsdGrad lg, cudaStream_t s) {
    const size_t smem = fa_bwd_coords_smem<NT, K, PACK>();
    static bool done[64] = {false};
    cudaError_t e = smem_attr_once(fa_bwd_coords_kernel<NT, K, LR, PACK>, (int)smem, done);
    if (e != cudaSuccess) return e;
    const int grid = persistent_grid((const void*)fa_bwd_coords_kernel<NT, K, LR, PACK>, NT, smem);
    fa_bwd_coords_kernel<NT, K, LR, PACK><<<grid, NT, smem, s>>>(seq, lengths, B, Lmax, Amax, coords,
                                                                      grad_coords, grad_angles, ws, lg, fa_table());
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

// Launch shapes (threads x residues per thread) of the full-atom kernels.
#define TPL_FA_SHAPES(X) \
    X(128, 1) X(256, 1) X(384, 1) X(128, 2) X(192, 2) X(64, 4) X(192, 4)

bool fullatom_cfg_supported(int threads, int k) {
#define TPL_FA_SUPPORTED(NT, K) \
    if (threads == NT && k == K) return true;
    TPL_FA_SHAPES(TPL_FA_SUPPORTED)
#undef TPL_FA_SUPPORTED
    return false;
}

#define TPL_FA_CASE_FWD(NT, K) case NT * 8 + K: e = fa_fwd_t<NT, K, LMV, PACKV>(angles, seq, lengths, Lmax, Amax, coords, num_atoms, ws, s, target); break;
#define TPL_FA_CASE_BWD(NT, K) case NT * 8 + K: return fa_bwd_coords_t<NT, K, LRV, PACKV>(seq, lengths, B, Lmax, Amax, coords, grad_coords, grad_angles, ws, lg, s);

namespace {

template <bool LMV, bool PACKV>
cudaError_t fa_forward_shape(const float* angles, const uint8_t* seq, const int32_t* lengths, int Lmax, int Amax,
                             float* coords, int32_t* num_atoms, const ChainWs& ws, LaunchCfg cfg, cudaStream_t s,
                             const float* target) {
    cudaError_t e = cudaErrorInvalidValue;
    switch (cfg.threads * 8 + cfg.res_per_thread) {
        TPL_FA_SHAPES(TPL_FA_CASE_FWD)
        default: return cudaErrorInvalidValue;
    }
    return e;
}

template <bool LRV, bool PACKV>
cudaError_t fa_backward_shape(const uint8_t* seq, const int32_t* lengths, int B, int Lmax, int Amax,
                              const float* coords, const float* grad_coords, float* grad_angles,
                              const ChainWs& ws, LrmsdGrad lg, LaunchCfg cfg, cudaStream_t s) {
    switch (cfg.threads * 8 + cfg.res_per_thread) {
        TPL_FA_SHAPES(TPL_FA_CASE_BWD)
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_fullatom_forward(const float* angles, const uint8_t* seq,
                                    const int32_t* lengths, int B, int Lmax, int Amax,
                                    float* coords, int32_t* num_atoms, int sched_mode,
                                    void* workspace, LaunchCfg cfg, cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    ChainWs ws;
    chain_ws_layout(workspace, B, Lmax, &ws, true);
    ws.flags = cfg.flags;
    cudaError_t e = launch_schedule(lengths, B, Lmax, cfg.threads * cfg.res_per_thread, sched_mode,
                                    cfg.res_per_thread, ws, s, true);
    if (e != cudaSuccess) return e;
    if (sched_mode == kSchedPacked)
        return fa_forward_shape<false, true>(angles, seq, lengths, Lmax, Amax, coords, num_atoms, ws, cfg, s, nullptr);
    return fa_forward_shape<false, false>(angles, seq, lengths, Lmax, Amax, coords, num_atoms, ws, cfg, s, nullptr);
}

cudaError_t launch_fullatom_backward(const float* angles, const uint8_t* seq,
                                     const int32_t* lengths, int B, int Lmax, int Amax,
                                     const float* coords, const float* grad_coords,
                                     float* grad_angles, bool from_coords, void* workspace,
                                     LaunchCfg cfg, cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    ChainWs ws;
    chain_ws_layout(workspace, B, Lmax, &ws, true);
    ws.flags = cfg.flags;
    cudaError_t e = reset_backward_flags(ws, s);
    if (e != cudaSuccess) return e;
    if (from_coords && cfg.packed)
        return fa_backward_shape<false, true>(seq, lengths, B, Lmax, Amax, coords, grad_coords, grad_angles,
                                                     ws, LrmsdGrad{}, cfg, s);
    if (from_coords)
        return fa_backward_shape<false, false>(seq, lengths, B, Lmax, Amax, coords, grad_coords, grad_angles,
                                                      ws, LrmsdGrad{}, cfg, s);
    // frames rebuilt from the angles: one residue per thread
    if (cfg.res_per_thread != 1) return cudaErrorInvalidValue;
    switch (cfg.threads) {
        case 128: return fa_bwd_t<128>(angles, seq, lengths, B, Lmax, Amax, grad_coords, grad_angles, ws, s);
        case 256: return fa_bwd_t<256>(angles, seq, lengths, B, Lmax, Amax, grad_coords, grad_angles, ws, s);
        case 384: return fa_bwd_t<384>(angles, seq, lengths, B, Lmax, Amax, grad_coords, grad_angles, ws, s);
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
    ws.flags = cfg.flags;
    cudaError_t e = reset_backward_flags(ws, s);
    if (e != cudaSuccess) return e;
    const LrmsdGrad lg{target, lrmsd_state, grad_lrmsd};
    if (cfg.packed)
        return fa_backward_shape<true, true>(seq, lengths, B, Lmax, Amax, coords, nullptr, grad_angles, ws, lg,
                                                    cfg, s);
    return fa_backward_shape<true, false>(seq, lengths, B, Lmax, Amax, coords, nullptr, grad_angles, ws, lg,
                                                 cfg, s);
}

cudaError_t launch_fullatom_lrmsd_forward(const float* angles, const uint8_t* seq, const int32_t* lengths,
                                          const float* target, int B, int Lmax, int Amax, float* coords,
                                          int32_t* num_atoms, float* lrmsd, int sched_mode, void* workspace,
                                          LaunchCfg cfg, cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    ChainWs ws;
    chain_ws_layout(workspace, B, Lmax, &ws, true, true);
    ws.flags = cfg.flags;
    const int tile = cfg.threads * cfg.res_per_thread;
    cudaError_t e = launch_schedule(lengths, B, Lmax, tile, sched_mode, 1, ws, s, true);
    if (e != cudaSuccess) return e;
    e = fa_forward_shape<true, false>(angles, seq, lengths, Lmax, Amax, coords, num_atoms, ws, cfg, s, target);
    if (e != cudaSuccess) return e;
    return launch_lrmsd_parts(coords, target, num_atoms, B, Amax, ws.tmom, ws.tmax, lengths, tile, Lmax, ws.lstate,
                              lrmsd, s);
}

cudaError_t launch_fullatom_lrmsd_backward(const uint8_t* seq, const int32_t* lengths, const float* coords,
                                           const float* target, const float* grad_lrmsd, int B, int Lmax,
                                           int Amax, float* grad_angles, void* workspace, LaunchCfg cfg,
                                           cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    ChainWs ws;
    chain_ws_layout(workspace, B, Lmax, &ws, true, true);
    ws.flags = cfg.flags;
    cudaError_t e = reset_backward_flags(ws, s);
    if (e != cudaSuccess) return e;
    const LrmsdGrad lg{target, ws.lstate, grad_lrmsd};
    return fa_backward_shape<true, false>(seq, lengths, B, Lmax, Amax, coords, nullptr, grad_angles, ws, lg,
                                                 cfg, s);
}

cudaError_t launch_fullatom_backward_quadratic(const uint8_t* seq, const int32_t* lengths, int B, int Lmax,
                                              int Amax, const float* coords, const float* grad_coords,
                                              float* grad_angles, cudaStream_t s) {
    if (B == 0 || Lmax == 0) return cudaSuccess;
    const dim3 grid((Lmax + kQRes - 1) / kQRes, B);
    fa_bwd_quadratic_kernel<<<grid, kQNT, 0, s>>>(seq, lengths, Lmax, Amax, coords, grad_coords, grad_angles,
                                                  fa_table());
    return cudaGetLastError();
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
