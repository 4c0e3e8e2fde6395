// Tile scheduling shared by the chain kernels (backbone and full atom).
//
// A chain of L residues is cut into tiles of TILE residues.  A schedule kernel
// writes the list of (chain, tile) entries -- chains in batch order, longest
// first, or longest first with the chains of at most one tile packed several
// per entry -- and zeroes the forward flags and work counter.  The chain kernels are persistent: each CTA
// takes the next list entry from an atomic counter, so every tile a CTA waits
// for was taken earlier by a CTA that is running and never waits on a later
// one (no deadlock, whatever order the hardware starts CTAs in).
//
// Cross-tile dependencies use aggregate-only look-back: a tile publishes its
// own aggregate (flag + data), then combines the aggregates of all the tiles
// it depends on in a fixed order.  Nothing waits on a wait, and the rounding
// of the result does not depend on timing (results are deterministic).
//  - forward: prefix of the rigid transforms (and atom counts) of tiles < t;
//    the prefix (frame at the tile start) is stored for the backward;
//  - backward: suffix of the (sum r x g, sum g) of tiles > t, the tiles of a
//    chain taken last-to-first.
// Every wait is bounded: after kSpinLimit polls the kernel sets
// TPL_STATUS_TIMEOUT, takes zero for the missing term and goes on.
#pragma once

#include "tpl_common.cuh"

namespace tpl {

constexpr int kMinTile = 64;          // smallest tile of any launch shape (sizes the workspace)
constexpr int kSpinLimit = 1 << 20;   // polls of one flag before giving up
constexpr int kSpinFast = 64;         // polls back to back before each later poll sleeps 100 ns
constexpr int kWsMagic = 0x54504c31;  // written by the schedule kernel, checked by the backward

// Header words.
enum {
    kHdrTiles = 0,     // number of list entries
    kHdrFwdNext = 1,   // forward work counter
    kHdrTile = 2,      // tile size the schedule was built for
    kHdrMagic = 3,
    kHdrB = 4,
    kHdrLmax = 5,
};

// A list entry is (chain, tile) for a tile of one chain, or, for a pack of
// short chains that share one tile (chains per CTA > 1), (-1 - start, count):
// the chains order[start .. start + count), each a whole chain, in slots
// padded to the granule of the kernel (residues per thread).
constexpr int kMaxPack = 8;

struct ChainWs {
    int* hdr;        // 64 ints
    int2* tiles;     // [B * tmax] list entries
    int* order;      // [B] chains in schedule order (packs index into it)
    int* fflag;      // [B * tmax] forward aggregate flags
    float4* fagg;    // [B * tmax][4] forward aggregate: rigid (12 floats) + atom count
    float4* start;   // [B * tmax][4] frame at the tile start + first atom index
    int* bflag;      // [B * tmax + 4]: backward flags; word B * tmax is the backward work counter
    float4* bagg;    // [B * tmax][2] backward aggregate (c, g)
    int* ratom;      // [B * Lmax] first atom of each residue (full atom only; else null)
    // fused training step only (else null): per tile, the LRMSD moments of its
    // atoms (20 floats), the sum of its squared residuals, a done flag; per
    // chain, the LRMSD state (U, centroids, 1 / (N LRMSD): 16 floats)
    float* tmom;
    float* tres;
    int* tdone;
    float* lstate;
    int tmax;        // tiles per chain for the smallest tile
    int slots;       // B * tmax
    int flags;       // TPL_FLAG_* of the call (set by the launcher)
};

__host__ __device__ inline size_t ws_align(size_t x) { return (x + 255) & ~size_t(255); }

// Tiles per chain the workspace provides: enough for the smallest tile, also
// when a full-atom chain is split into balanced tiles (fa_num_tiles).
__host__ __device__ inline int ws_tmax(int Lmax) {
    int t = (Lmax + kMinTile - 5) / (kMinTile - 4);
    return t < 1 ? 1 : t;
}

// Full-atom tiles are balanced: a chain of L residues becomes T = ceil(L /
// (tile - 4)) tiles of nearly equal length whose starts are multiples of 4
// (so a thread's residues start 16-byte aligned), each at most tile - 1
// residues.  Tile t covers residues [fa_tile_start(L, T, t), fa_tile_start(L,
// T, t + 1)).  An empty chain has one (empty) tile.
__host__ __device__ inline int fa_num_tiles(int L, int tile) {
    return L > 0 ? (L + tile - 5) / (tile - 4) : 1;
}
__host__ __device__ inline int fa_tile_start(int L, int T, int t) {
    return t >= T ? L : (int)(((long long)t * L / T) & ~3LL);
}

// Offsets of the regions; `base` may be null to only size the workspace.
// Whether the output padding is written (flags) is set by the launcher.
__host__ __device__ inline size_t chain_ws_layout(void* base, int B, int Lmax, ChainWs* w,
                                                  bool per_residue = false, bool step = false) {
    const int tmax = ws_tmax(Lmax);
    const size_t slots = (size_t)(B > 0 ? B : 1) * tmax;
    size_t o = 0;
    const size_t hdr = o; o = ws_align(o + 64 * sizeof(int));
    const size_t tiles = o; o = ws_align(o + slots * sizeof(int2));
    const size_t order = o; o = ws_align(o + (size_t)(B > 0 ? B : 1) * sizeof(int));
    const size_t fflag = o; o = ws_align(o + slots * sizeof(int));
    const size_t fagg = o; o = ws_align(o + slots * 4 * sizeof(float4));
    const size_t start = o; o = ws_align(o + slots * 4 * sizeof(float4));
    const size_t bflag = o; o = ws_align(o + (slots + 4) * sizeof(int));
    const size_t bagg = o; o = ws_align(o + slots * 2 * sizeof(float4));
    const size_t ratom = o;
    if (per_residue) o = ws_align(o + (size_t)(B > 0 ? B : 1) * (Lmax > 0 ? Lmax : 1) * sizeof(int));
    const size_t tmom = o;
    if (step) o = ws_align(o + slots * 20 * sizeof(float));
    const size_t tres = o;
    if (step) o = ws_align(o + slots * sizeof(float));
    const size_t tdone = o;
    if (step) o = ws_align(o + slots * sizeof(int));
    const size_t lstate = o;
    if (step) o = ws_align(o + (size_t)(B > 0 ? B : 1) * 16 * sizeof(float));
    if (w) {
        char* c = static_cast<char*>(base);
        w->hdr = reinterpret_cast<int*>(c + hdr);
        w->tiles = reinterpret_cast<int2*>(c + tiles);
        w->order = reinterpret_cast<int*>(c + order);
        w->fflag = reinterpret_cast<int*>(c + fflag);
        w->fagg = reinterpret_cast<float4*>(c + fagg);
        w->start = reinterpret_cast<float4*>(c + start);
        w->bflag = reinterpret_cast<int*>(c + bflag);
        w->bagg = reinterpret_cast<float4*>(c + bagg);
        w->ratom = per_residue ? reinterpret_cast<int*>(c + ratom) : nullptr;
        w->tmom = step ? reinterpret_cast<float*>(c + tmom) : nullptr;
        w->tres = step ? reinterpret_cast<float*>(c + tres) : nullptr;
        w->tdone = step ? reinterpret_cast<int*>(c + tdone) : nullptr;
        w->lstate = step ? reinterpret_cast<float*>(c + lstate) : nullptr;
        w->tmax = tmax;
        w->slots = (int)slots;
        w->flags = 0;
    }
    return o;
}

// ---------------------------------------------------------------------------
// flag publication / acquisition (release / acquire at GPU scope)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void flag_release(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int flag_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bounded wait for a nonzero flag.  Returns false (and flags the status word)
// on timeout.  The first polls run back to back: a short wait (a neighbour
// tile publishing moments later) is the common case, and a sleep requested
// here lasts microseconds on this GPU, far longer than asked.
__device__ __forceinline__ bool wait_flag(const int* p) {
    for (int it = 0; it < kSpinLimit; ++it) {
        if (flag_acquire(p) != 0) return true;
        if (it >= kSpinFast) __nanosleep(100);
    }
    flag_status(TPL_STATUS_TIMEOUT);
    return false;
}

__device__ __forceinline__ void store_rigid_g(float4* dst, const Rigid& m, int cnt, int cnt2 = 0) {
    dst[0] = make_float4(m.c0.x, m.c0.y, m.c0.z, m.c1.x);
    dst[1] = make_float4(m.c1.y, m.c1.z, m.c2.x, m.c2.y);
    dst[2] = make_float4(m.c2.z, m.t.x, m.t.y, m.t.z);
    dst[3] = make_float4(__int_as_float(cnt), __int_as_float(cnt2), 0.f, 0.f);
}

// L2 reads (the data was written by another CTA of this launch).
__device__ __forceinline__ Rigid load_rigid_g(const float4* src, int& cnt) {
    const float4 a = __ldcg(src), b = __ldcg(src + 1), c = __ldcg(src + 2), d = __ldcg(src + 3);
    Rigid m;
    m.c0 = make_float3(a.x, a.y, a.z);
    m.c1 = make_float3(a.w, b.x, b.y);
    m.c2 = make_float3(b.z, b.w, c.x);
    m.t = make_float3(c.y, c.z, c.w);
    cnt = __float_as_int(d.x);
    return m;
}

// Plain reads of data written by an earlier launch (the forward's tile starts).
__device__ __forceinline__ Rigid load_rigid_prev(const float4* src, int& cnt) {
    const float4 a = src[0], b = src[1], c = src[2], d = src[3];
    Rigid m;
    m.c0 = make_float3(a.x, a.y, a.z);
    m.c1 = make_float3(a.w, b.x, b.y);
    m.c2 = make_float3(b.z, b.w, c.x);
    m.t = make_float3(c.y, c.z, c.w);
    cnt = __float_as_int(d.x);
    return m;
}

__device__ __forceinline__ Rigid shfl_down_rigid(const Rigid& m, int delta) {
    Rigid r;
    const unsigned full = 0xffffffffu;
    r.c0.x = __shfl_down_sync(full, m.c0.x, delta);
    r.c0.y = __shfl_down_sync(full, m.c0.y, delta);
    r.c0.z = __shfl_down_sync(full, m.c0.z, delta);
    r.c1.x = __shfl_down_sync(full, m.c1.x, delta);
    r.c1.y = __shfl_down_sync(full, m.c1.y, delta);
    r.c1.z = __shfl_down_sync(full, m.c1.z, delta);
    r.c2.x = __shfl_down_sync(full, m.c2.x, delta);
    r.c2.y = __shfl_down_sync(full, m.c2.y, delta);
    r.c2.z = __shfl_down_sync(full, m.c2.z, delta);
    r.t.x = __shfl_down_sync(full, m.t.x, delta);
    r.t.y = __shfl_down_sync(full, m.t.y, delta);
    r.t.z = __shfl_down_sync(full, m.t.z, delta);
    return r;
}

__device__ __forceinline__ Rigid shfl_rigid(const Rigid& m, int src) {
    Rigid r;
    const unsigned full = 0xffffffffu;
    r.c0.x = __shfl_sync(full, m.c0.x, src);
    r.c0.y = __shfl_sync(full, m.c0.y, src);
    r.c0.z = __shfl_sync(full, m.c0.z, src);
    r.c1.x = __shfl_sync(full, m.c1.x, src);
    r.c1.y = __shfl_sync(full, m.c1.y, src);
    r.c1.z = __shfl_sync(full, m.c1.z, src);
    r.c2.x = __shfl_sync(full, m.c2.x, src);
    r.c2.y = __shfl_sync(full, m.c2.y, src);
    r.c2.z = __shfl_sync(full, m.c2.z, src);
    r.t.x = __shfl_sync(full, m.t.x, src);
    r.t.y = __shfl_sync(full, m.t.y, src);
    r.t.z = __shfl_sync(full, m.t.z, src);
    return r;
}

// Publication of a tile's forward aggregate (one thread).  The release store
// orders the data stores before the flag.
__device__ __forceinline__ void publish_prefix_agg(const ChainWs& ws, int slot, const Rigid& agg,
                                                   int cnt) {
    store_rigid_g(ws.fagg + 4 * (size_t)slot, agg, cnt);
    flag_release(ws.fflag + slot, 1);
}

// Forward look-back, called by all 32 lanes of a warp (every warp that needs
// the result calls it; no cross-warp synchronisation).  Lane l waits for tile
// base + l of each group of 32 predecessors (the waits overlap) and the warp
// folds the aggregates in a fixed tree: the result, in every lane, is
// A_0 A_1 ... A_{t-1} (product in tile order, re-orthonormalised) and the sum
// of their atom counts, identical in every run.
__device__ __forceinline__ Rigid gather_prefix(const ChainWs& ws, int slot0, int t, int& pre_cnt) {
    const int lane = threadIdx.x & 31;
    Rigid acc = rigid_identity();
    int cnt = 0;
    for (int base = 0; base < t; base += 32) {
        const int tp = base + lane;
        Rigid a = rigid_identity();
        int c = 0;
        if (tp < t && wait_flag(ws.fflag + slot0 + tp)) a = load_rigid_g(ws.fagg + 4 * (size_t)(slot0 + tp), c);
        const int n = min(32, t - base);
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            if (off >= n) break;
            const Rigid y = shfl_down_rigid(a, off);
            const int cy = __shfl_down_sync(0xffffffffu, c, off);
            if ((lane & (2 * off - 1)) == 0 && lane + off < n) {
                a = rigid_mul(a, y);
                c += cy;
            }
        }
        acc = rigid_mul(acc, shfl_rigid(a, 0));
        cnt += __shfl_sync(0xffffffffu, c, 0);
    }
    if (t > 0) rigid_reortho(acc);
    pre_cnt = cnt;
    return acc;
}

__device__ __forceinline__ Sum6 load_sum6_g(const float4* s) {
    const float4 a = __ldcg(s), b = __ldcg(s + 1);
    Sum6 v;
    v.c = make_float3(a.x, a.y, a.z);
    v.g = make_float3(a.w, b.x, b.y);
    return v;
}

__device__ __forceinline__ void publish_suffix_agg(const ChainWs& ws, int slot, const Sum6& agg) {
    float4* d = ws.bagg + 2 * (size_t)slot;
    d[0] = make_float4(agg.c.x, agg.c.y, agg.c.z, agg.g.x);
    d[1] = make_float4(agg.g.y, agg.g.z, 0.f, 0.f);
    flag_release(ws.bflag + slot, 1);
}

// Backward look-back, all 32 lanes of a warp: the sum of the totals of tiles
// t+1..T-1 in a fixed tree order, in every lane.
__device__ __forceinline__ Sum6 gather_suffix(const ChainWs& ws, int slot0, int t, int T) {
    const int lane = threadIdx.x & 31;
    Sum6 acc = sum6_zero();
    for (int base = t + 1; base < T; base += 32) {
        const int tp = base + lane;
        Sum6 v = sum6_zero();
        if (tp < T && wait_flag(ws.bflag + slot0 + tp)) v = load_sum6_g(ws.bagg + 2 * (size_t)(slot0 + tp));
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const Sum6 y = shfl_down_sum6(v, off);
            if ((lane & (2 * off - 1)) == 0) v = sum6_add(v, y);
        }
        acc = sum6_add(acc, v);
    }
    Sum6 r;
    r.c = make_float3(__shfl_sync(0xffffffffu, acc.c.x, 0), __shfl_sync(0xffffffffu, acc.c.y, 0),
                      __shfl_sync(0xffffffffu, acc.c.z, 0));
    r.g = make_float3(__shfl_sync(0xffffffffu, acc.g.x, 0), __shfl_sync(0xffffffffu, acc.g.y, 0),
                      __shfl_sync(0xffffffffu, acc.g.z, 0));
    return r;
}

// Chains of a packed list entry, in shared memory: chain id, length and first
// slot (slots of G residues; off[count] = slots used).
struct PackS {
    int b[kMaxPack];
    int len[kMaxPack];
    int off[kMaxPack + 1];
};

// Fills `s` for the pack (start, m) with warp 0; all threads must call it.
template <int G>
__device__ __forceinline__ void load_pack(const ChainWs& ws, const int32_t* lengths, int Lmax,
                                          int start, int m, PackS& s) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int b = 0, L = 0;
        if (lane < m) {
            b = ws.order[start + lane];
            L = clamp_length(lengths, b, Lmax);
        }
        const int lp = (L + G - 1) / G * G;
        int inc = lp;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, off);
            if (lane >= off) inc += y;
        }
        if (lane < m) {
            s.b[lane] = b;
            s.len[lane] = L;
            s.off[lane] = inc - lp;
            if (lane == m - 1) s.off[m] = inc;
        }
    }
    __syncthreads();
}

// Member of the pack whose slots hold residue slot `slot`, or -1 (unused slot).
__device__ __forceinline__ int pack_member(const PackS& s, int m, int slot) {
    int ci = -1;
    for (int i = 0; i < m; ++i)
        if (s.off[i] <= slot && slot < s.off[i + 1]) ci = i;
    return ci;
}

// Work-list entries for a persistent CTA.  take_tile() is called once at the
// start; during a tile thread 0 requests the next entry (request_tile) once its
// warp has finished the tile's look-back, and next_tile() hands it to the CTA
// after the tile's stores.  Between the two the CTA waits on nothing, so a
// tile held but not yet started never delays a tile that waits on it by more
// than one tile's stores: waits cannot chain through held tiles.
__device__ __forceinline__ int take_tile(int* counter, int* s_v) {
    if (threadIdx.x == 0) *s_v = atomicAdd(counter, 1);
    __syncthreads();
    return *s_v;
}
__device__ __forceinline__ int request_tile(int* counter) {
    return threadIdx.x == 0 ? atomicAdd(counter, 1) : 0;
}
__device__ __forceinline__ int next_tile(int requested, int* s_v) {
    __syncthreads();  // everyone is done with this tile's shared data
    if (threadIdx.x == 0) *s_v = requested;
    __syncthreads();
    return *s_v;
}

// Host side: raises a kernel's dynamic shared memory limit once per device
// (not again during a graph capture after the first call).
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

// Host side: schedule kernel (api.cu).
// Chain order of the schedule: batch order, longest first, or longest first
// with the chains of at most one tile packed several per tile (granule =
// residues per thread, the unit a chain's slots are padded to).
enum SchedMode { kSchedBatch = 0, kSchedLongest = 1, kSchedPacked = 2 };
// balanced: full-atom tiles (fa_num_tiles per chain) instead of ceil(L / tile).
cudaError_t launch_schedule(const int32_t* lengths, int B, int Lmax, int tile, int mode, int granule,
                            const ChainWs& ws, cudaStream_t s, bool balanced = false);
cudaError_t reset_backward_flags(const ChainWs& ws, cudaStream_t s);

}  // namespace tpl
