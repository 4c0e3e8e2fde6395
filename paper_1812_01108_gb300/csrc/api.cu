// C ABI of the library (include/tpl.h): argument checks, workspace layout,
// the schedule kernel (work lists of tiles and packed short chains), the
// autotuners and dispatch to the kernels.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/tpl.h"
#include "kernels.h"
#include "sched.cuh"
#include "tables.h"
#include "tpl_common.cuh"

namespace tpl {

__device__ int g_status = 0;

namespace {

thread_local std::string t_last_error;

tpl_status fail(tpl_status code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
tpl_status fail(tpl_status code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_last_error = buf;
    return code;
}

tpl_status ok() {
    t_last_error.clear();
    return TPL_OK;
}

tpl_status cuda_fail(cudaError_t e, const char* where) {
    return fail(TPL_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }


// ---------------------------------------------------------------------------
// K8: the work list.  CTA 0 builds it; the other CTAs of the launch zero the
// forward look-back flags (and the fused step's done flags), which from one
// SM alone would take longer than the sort.
// Chain order: batch order, or longest first by a stable counting sort on 64
// length buckets.  In packed mode a chain of at most one tile goes instead to
// the class m = min(8, tile / slots), the number of such chains that fit one
// tile (slots = length rounded up to the granule); the classes follow the
// long chains, m ascending, and every m consecutive chains of a class form
// one packed entry.  The sort: each warp counts the keys of a contiguous run
// of chains, one scan over (key, warp) gives every warp its first position
// per key, and each warp walks its run again placing its chains (so chains of
// equal key keep batch order).  Then the entries per thread, an exclusive
// scan, and the entries.  The work is issue-bound on one SM: every chain's
// key is computed once and kept in shared memory with its length.
// ---------------------------------------------------------------------------
constexpr int kBuckets = 64;
constexpr int kKeys = kBuckets + kMaxPack;
constexpr int kSchedThreadsSmall = 256;  // batches of at most kSchedSmallB chains
constexpr int kSchedThreads = 1024;
constexpr int kSchedSmallB = 1024;
constexpr int kSchedCache = 16384;  // chains whose length, key and order entry stay in shared memory
constexpr int kZeroPerCta = 4 * kSchedThreadsSmall;  // int4 words zeroed per flag-zeroing CTA and pass

__device__ __forceinline__ int sched_key(int L, int Lmax, int tile, int mode, int granule) {
    if (mode == kSchedPacked && L <= tile) {  // chains per packed tile, 1..kMaxPack
        const int slots = (L + granule - 1) / granule * granule;
        return kBuckets - 1 + (slots == 0 ? kMaxPack : min(kMaxPack, tile / slots));
    }
    const int bucket = Lmax < (1 << 24) ? (L * kBuckets) / (Lmax + 1)
                                        : (int)(((long long)L * kBuckets) / ((long long)Lmax + 1));
    return kBuckets - 1 - bucket;
}

__device__ __forceinline__ int sched_len(const int32_t* lengths, int b, int Lmax) {
    const int L = lengths[b];
    return L < 0 ? 0 : (L > Lmax ? Lmax : L);
}

template <int NTS>
__global__ void __launch_bounds__(NTS) schedule_kernel(const int32_t* __restrict__ lengths,
                                                                 int B, int Lmax, int tile, int mode,
                                                                 int granule, bool balanced, ChainWs ws) {
    if (blockIdx.x > 0) {  // flag zeroing, 16 bytes at a time (the regions are 256-byte aligned)
        const int n = B * ws.tmax;
        const size_t stride = (size_t)(gridDim.x - 1) * NTS;
        const size_t i0 = (size_t)(blockIdx.x - 1) * NTS + threadIdx.x;
        int4* f4 = reinterpret_cast<int4*>(ws.fflag);
        for (size_t i = i0; i < (size_t)n / 4; i += stride) f4[i] = make_int4(0, 0, 0, 0);
        if (i0 < (size_t)(n & 3)) ws.fflag[(n & ~3) + i0] = 0;
        if (ws.tdone) {  // fused training step: the backward's per-tile done flags
            int4* d4 = reinterpret_cast<int4*>(ws.tdone);
            for (size_t i = i0; i < (size_t)n / 4; i += stride) d4[i] = make_int4(0, 0, 0, 0);
            if (i0 < (size_t)(n & 3)) ws.tdone[(n & ~3) + i0] = 0;
        }
        return;
    }
    __shared__ int s_start[kKeys + 1];
    constexpr int kSchedWarps = NTS / 32;
    __shared__ int s_wcnt[kSchedWarps][kKeys];  // per warp: key counts, then next position per key
    __shared__ int s_part[33];
    extern __shared__ int s_cache[];  // [ncache] lengths, [ncache] order entries, [ncache] keys (bytes)
    const int ncache = B < kSchedCache ? B : kSchedCache;
    int* s_len = s_cache;
    int* s_ord = s_cache + ncache;
    unsigned char* s_key = reinterpret_cast<unsigned char*>(s_cache + 2 * ncache);
    int* order = ws.order;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    // four independent loads in flight per thread, then the keys
    for (int b0 = 0; b0 < ncache; b0 += 4 * NTS) {
        int L[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int b = b0 + q * NTS + threadIdx.x;
            L[q] = b < ncache ? sched_len(lengths, b, Lmax) : 0;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int b = b0 + q * NTS + threadIdx.x;
            if (b < ncache) {
                s_len[b] = L[q];
                s_key[b] = (unsigned char)sched_key(L[q], Lmax, tile, mode, granule);
            }
        }
    }
    for (int i = threadIdx.x; i < kSchedWarps * kKeys; i += NTS) (&s_wcnt[0][0])[i] = 0;
    __syncthreads();
    auto len = [&](int b) { return b < ncache ? s_len[b] : sched_len(lengths, b, Lmax); };
    auto key = [&](int b) {
        return b < ncache ? (int)s_key[b] : sched_key(sched_len(lengths, b, Lmax), Lmax, tile, mode, granule);
    };
    auto set_order = [&](int i, int b) {
        order[i] = b;
        if (i < ncache) s_ord[i] = b;
    };
    auto ord = [&](int i) { return i < ncache ? s_ord[i] : order[i]; };
    if (mode != kSchedBatch) {
        // the run of chains of this warp
        const int per_w = (B + kSchedWarps - 1) / kSchedWarps;
        const int w0 = warp * per_w, w1 = min(B, w0 + per_w);
        // 1. key counts of the run: one shared-memory add per distinct key of 32 chains
        for (int c0 = w0; c0 < w1; c0 += 32) {
            const int b = c0 + lane;
            const int k = b < w1 ? key(b) : -1;
            const unsigned peers = __match_any_sync(0xffffffffu, k);
            if (k >= 0 && (peers & lt) == 0) s_wcnt[warp][k] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // 2. per key, exclusive scan over the warps (warp w scans keys w, w + 32, ...)
        for (int k = warp; k < kKeys; k += kSchedWarps) {
            const int c = lane < kSchedWarps ? s_wcnt[lane][k] : 0;
            int inc = c;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, inc, off);
                if (lane >= off) inc += y;
            }
            if (lane < kSchedWarps) s_wcnt[lane][k] = inc - c;
            if (lane == 31) s_start[k] = inc;  // the key's count, scanned below
        }
        __syncthreads();
        if (warp == 0) {  // exclusive scan of the key counts, kKeys <= 128: 4 per lane
            static_assert(kKeys <= 128, "key scan covers 128 keys");
            int c[4], sum = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = 4 * lane + q;
                c[q] = k < kKeys ? s_start[k] : 0;
                sum += c[q];
            }
            int inc = sum;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, inc, off);
                if (lane >= off) inc += y;
            }
            __syncwarp();
            int run = inc - sum;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = 4 * lane + q;
                if (k < kKeys) s_start[k] = run;
                run += c[q];
            }
            if (lane == 31) s_start[kKeys] = inc;
        }
        __syncthreads();
        // 3. positions: key start + this warp's first position within the key
        //    + the chains of the key earlier in the run
        for (int c0 = w0; c0 < w1; c0 += 32) {
            const int b = c0 + lane;
            const int k = b < w1 ? key(b) : -1;
            const unsigned peers = __match_any_sync(0xffffffffu, k);
            if (k >= 0) set_order(s_start[k] + s_wcnt[warp][k] + __popc(peers & lt), b);
            __syncwarp();
            if (k >= 0 && (peers & lt) == 0) s_wcnt[warp][k] += __popc(peers);
            __syncwarp();
        }
    } else {
        for (int b = threadIdx.x; b < B; b += NTS) set_order(b, b);
    }
    __syncthreads();
    // each thread owns a contiguous run of the ordered chains
    const int per = (B + NTS - 1) / NTS;
    const int i0 = threadIdx.x * per, i1 = min(B, i0 + per);
    auto ntiles = [&](int L) {
        if (balanced) return fa_num_tiles(L, tile);
        return L > 0 ? (L + tile - 1) / tile : 1;  // an empty chain still gets one tile (zero fill)
    };
    // entries that start at order position i: a long chain's tiles, or one
    // packed entry at every m-th chain of a class
    auto entries = [&](int i, int b) {
        const int k = key(b);
        if (mode != kSchedPacked || k < kBuckets) return ntiles(len(b));
        return ((i - s_start[k]) % (k - kBuckets + 1)) == 0 ? 1 : 0;
    };
    int mine = 0;
    for (int i = i0; i < i1; ++i) mine += entries(i, ord(i));
    // block-wide exclusive scan of `mine`: warp shuffles, then the warp totals
    int inc = mine;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
    }
    if (lane == 31) s_part[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int w = lane < kSchedWarps ? s_part[lane] : 0;
        int wi = w;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wi, off);
            if (lane >= off) wi += y;
        }
        if (lane < kSchedWarps) s_part[lane] = wi - w;  // exclusive prefix of warp totals
        if (lane == 31) s_part[32] = wi;
    }
    __syncthreads();
    int base = s_part[warp] + inc - mine;
    for (int i = i0; i < i1; ++i) {
        const int b = ord(i);
        const int k = key(b);
        if (mode == kSchedPacked && k >= kBuckets) {
            const int m = k - kBuckets + 1;
            if (((i - s_start[k]) % m) == 0) ws.tiles[base++] = make_int2(-1 - i, min(m, s_start[k + 1] - i));
        } else {
            const int n = ntiles(len(b));
            for (int q = 0; q < n; ++q) ws.tiles[base + q] = make_int2(b, q);
            base += n;
        }
    }
    if (threadIdx.x == 0) {
        ws.hdr[kHdrTiles] = s_part[32];
        ws.hdr[kHdrFwdNext] = 0;
        ws.hdr[kHdrTile] = tile;
        ws.hdr[kHdrMagic] = kWsMagic;
        ws.hdr[kHdrB] = B;
        ws.hdr[kHdrLmax] = Lmax;
    }
}

tpl_opts resolve(const tpl_opts* o) {
    tpl_opts r;
    memset(&r, 0, sizeof(r));
    if (o) r = *o;
    return r;
}

// Schedule mode of a chain call (kSched* of sched.cuh); packing is a
// backbone feature.
int sched_mode(const tpl_opts& o, bool can_pack) {
    switch (o.schedule) {
        case TPL_SCHED_LONGEST_FIRST: return kSchedLongest;
        case TPL_SCHED_BATCH_ORDER: return kSchedBatch;
        case TPL_SCHED_PACKED: return can_pack ? kSchedPacked : kSchedLongest;
        default: return can_pack ? kSchedPacked : kSchedBatch;
    }
}

tpl_status check_opts(const tpl_opts& o) {
    if (o.bwd_mode < TPL_BWD_AUTO || o.bwd_mode > TPL_BWD_FROM_COORDS)
        return fail(TPL_ERR_INVALID_ARG, "bwd_mode %d unknown", o.bwd_mode);
    if (o.schedule < TPL_SCHED_AUTO || o.schedule > TPL_SCHED_PACKED)
        return fail(TPL_ERR_INVALID_ARG, "schedule %d unknown", o.schedule);
    if (o.threads < 0 || o.res_per_thread < 0)
        return fail(TPL_ERR_INVALID_ARG, "negative launch option");
    if (o.flags & ~TPL_FLAG_PADDING_ZEROED) return fail(TPL_ERR_INVALID_ARG, "unknown flags 0x%x", o.flags);
    return TPL_OK;
}

// Backbone defaults: 128 threads x 4 residues (tile 512 residues).
LaunchCfg backbone_cfg(const tpl_opts& o) {
    LaunchCfg c;
    c.threads = o.threads ? o.threads : 128;
    c.res_per_thread = o.res_per_thread ? o.res_per_thread : 4;
    c.flags = o.flags;
    return c;
}

// Full-atom defaults: 384 threads x 1 residue (tiles of up to 383 residues);
// threads without residues per thread take the fewest residues per thread that
// form a supported shape.
LaunchCfg fullatom_cfg(const tpl_opts& o) {
    LaunchCfg c;
    c.threads = o.threads ? o.threads : 384;
    c.res_per_thread = o.res_per_thread ? o.res_per_thread : 1;
    if (o.threads && !o.res_per_thread)
        for (int k : {1, 2, 4})
            if (fullatom_cfg_supported(c.threads, k)) {
                c.res_per_thread = k;
                break;
            }
    c.flags = o.flags;
    c.packed = o.schedule == TPL_SCHED_PACKED;
    return c;
}

bool fullatom_cfg_supported_recompute(const LaunchCfg& c) {
    return c.res_per_thread == 1 && (c.threads == 128 || c.threads == 256 || c.threads == 384);
}

tpl_status check_fullatom_cfg(const LaunchCfg& c) {
    if (!fullatom_cfg_supported(c.threads, c.res_per_thread))
        return fail(TPL_ERR_INVALID_ARG, "unsupported full-atom launch %d threads x %d residues", c.threads,
                    c.res_per_thread);
    return TPL_OK;
}

tpl_status check_chain_args(int B, int Lmax, const void* const* ptrs, int nptr) {
    if (B < 0 || Lmax < 0) return fail(TPL_ERR_INVALID_ARG, "B=%d Lmax=%d must be >= 0", B, Lmax);
    if (Lmax % 4 != 0) return fail(TPL_ERR_BAD_SHAPE, "Lmax=%d must be a multiple of 4", Lmax);
    if (B == 0) return TPL_OK;
    for (int i = 0; i < nptr; ++i) {
        if (!ptrs[i]) return fail(TPL_ERR_INVALID_ARG, "pointer argument %d is NULL", i);
        if (!aligned16(ptrs[i])) return fail(TPL_ERR_MISALIGNED, "pointer argument %d not 16-byte aligned", i);
    }
    return TPL_OK;
}

tpl_status check_ws(void* ws, size_t have, size_t need) {
    if (need == 0) return TPL_OK;
    if (!ws) return fail(TPL_ERR_WORKSPACE, "workspace is NULL (%zu bytes needed)", need);
    if (!aligned16(ws)) return fail(TPL_ERR_MISALIGNED, "workspace not 16-byte aligned");
    if (have < need) return fail(TPL_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", have, need);
    return TPL_OK;
}

}  // namespace

size_t chain_ws_bytes(int B, int Lmax, bool per_residue, bool step) {
    return chain_ws_layout(nullptr, B, Lmax, nullptr, per_residue, step);
}

// One thread waits on `flag` with the chain kernels' bounded wait.
__global__ void selftest_wait_kernel(const int* flag) {
    if (threadIdx.x == 0) wait_flag(flag);
}

// Dynamic shared memory of the sort CTA for n cached chains: lengths and
// order entries (ints), keys (bytes).
static size_t sched_smem(int n) { return (size_t)n * (2 * sizeof(int) + 1); }

cudaError_t launch_schedule(const int32_t* lengths, int B, int Lmax, int tile, int mode, int granule,
                            const ChainWs& ws, cudaStream_t s, bool balanced) {
    // the shared-memory limit is raised once per device (not during a capture after the first call)
    static bool raised[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!raised[dev]) {
        e = cudaFuncSetAttribute(schedule_kernel<kSchedThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sched_smem(kSchedCache));
        if (e != cudaSuccess) return e;
        raised[dev] = true;
    }
    // CTA 0 sorts; the others zero the flags (one pass of kZeroPerCta words each)
    const size_t words = ((size_t)B * ws.tmax + 3) / 4;
    const int zero_ctas = (int)std::min<size_t>(148, (words + kZeroPerCta - 1) / kZeroPerCta);
    // a small batch sorts with fewer threads (fewer warps to synchronise; a few
    // chains per thread either way); its shared memory stays under 48 KB
    if (B <= kSchedSmallB)
        schedule_kernel<kSchedThreadsSmall><<<1 + std::max(zero_ctas, 1), kSchedThreadsSmall, sched_smem(B), s>>>(
            lengths, B, Lmax, tile, mode, granule, balanced, ws);
    else
        schedule_kernel<kSchedThreads><<<1 + std::max(zero_ctas, 1), kSchedThreads,
                                         sched_smem(B < kSchedCache ? B : kSchedCache), s>>>(
            lengths, B, Lmax, tile, mode, granule, balanced, ws);
    return cudaGetLastError();
}

cudaError_t reset_backward_flags(const ChainWs& ws, cudaStream_t s) {
    return cudaMemsetAsync(ws.bflag, 0, (size_t)(ws.slots + 4) * sizeof(int), s);
}

// CTAs of a persistent launch: SMs x resident CTAs per SM, cached per kernel
// and device (the occupancy query is a host-side call, safe during capture).
int persistent_grid(const void* kernel, int threads, size_t smem) {
    struct Entry {
        const void* k;
        int dev, threads;
        size_t smem;
        int grid;
    };
    static std::mutex mu;
    static std::vector<Entry> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    for (const Entry& e : cache)
        if (e.k == kernel && e.dev == dev && e.threads == threads && e.smem == smem) return e.grid;
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        sms = 1;
    cache.push_back(Entry{kernel, dev, threads, smem, per_sm * sms});
    return per_sm * sms;
}

cudaError_t read_and_clear_status(cudaStream_t s, int* out) {
    int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbolAsync(out, g_status, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyToSymbolAsync(g_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

}  // namespace tpl

using namespace tpl;

namespace {

// ---------------------------------------------------------------------------
// Autotuner: times forward + backward for every supported launch shape and
// schedule on the caller's own batch and returns the fastest options.  Each
// candidate's calls are captured once into a CUDA graph (the form a training
// loop replays; launched one by one, the calls rank shapes differently) after
// one direct, untimed pass; the graph is replayed once untimed, then the best
// of `kTuneReps` replays between CUDA events on `stream` counts.
// ---------------------------------------------------------------------------
constexpr int kTuneReps = 5;

template <class Step>
tpl_status tune(const tpl_opts* cands, int n, cudaStream_t s, const Step& step, tpl_opts* best,
                       float* best_ms) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
        return fail(TPL_ERR_INVALID_ARG, "autotune cannot run while the stream is being captured");
    // the candidates run on a stream of the tuner's own (the caller's stream
    // may be the legacy default stream, which cannot be captured), after the
    // work already queued on the caller's stream
    cudaStream_t ts = nullptr;
    if (cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "autotune");
    cudaError_t es = cudaStreamSynchronize(s);
    if (es != cudaSuccess) {
        cudaStreamDestroy(ts);
        return cuda_fail(es, "autotune");
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) {
        cudaStreamDestroy(ts);
        return cuda_fail(cudaGetLastError(), "autotune");
    }
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaStreamDestroy(ts);
        return cuda_fail(cudaGetLastError(), "autotune");
    }
    const tpl_stream tstream = reinterpret_cast<tpl_stream>(ts);
    float best_t = -1.f;
    tpl_status st = TPL_OK;
    for (int c = 0; c < n && st == TPL_OK; ++c) {
        if (step(cands[c], tstream) != TPL_OK) continue;  // a shape this call rejects
        cudaError_t e = cudaStreamSynchronize(ts);
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        if (e == cudaSuccess) e = cudaStreamBeginCapture(ts, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const tpl_status sc = step(cands[c], tstream);
            e = cudaStreamEndCapture(ts, &graph);
            if (sc != TPL_OK) {
                st = sc;
                if (graph) cudaGraphDestroy(graph);
                break;
            }
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        float t_min = -1.f;
        for (int r = -1; r < kTuneReps && e == cudaSuccess; ++r) {
            cudaEventRecord(e0, ts);
            e = cudaGraphLaunch(exec, ts);
            cudaEventRecord(e1, ts);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && r >= 0 && (t_min < 0.f || ms < t_min)) t_min = ms;
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "autotune");
            break;
        }
        if (t_min >= 0.f && (best_t < 0.f || t_min < best_t)) {
            best_t = t_min;
            *best = cands[c];
        }
    }
    cudaStreamSynchronize(ts);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(ts);
    if (st != TPL_OK) return st;
    if (best_t < 0.f) return fail(TPL_ERR_INVALID_ARG, "autotune: no launch shape accepted these arguments");
    if (best_ms) *best_ms = best_t;
    return ok();
}

}  // namespace

extern "C" {

const char* tpl_version(void) { return "0.1.0"; }

const char* tpl_last_error(void) { return t_last_error.c_str(); }

size_t tpl_backbone_workspace_size(int B, int Lmax) { return chain_ws_bytes(B, Lmax, false, false); }

size_t tpl_fullatom_workspace_size(int B, int Lmax) { return chain_ws_bytes(B, Lmax, true, false); }

size_t tpl_backbone_lrmsd_workspace_size(int B, int Lmax) { return chain_ws_bytes(B, Lmax, false, true); }

size_t tpl_lrmsd_workspace_size(int P, int Nmax) {
    if (P <= 0 || Nmax < 0) return 256;
    return lrmsd_ws_bytes(P, Nmax);
}

int tpl_lrmsd_forward_launches(int P) { return lrmsd_forward_launches(P); }

tpl_status tpl_backbone_forward(const float* angles, const int32_t* lengths, int B, int Lmax,
                                float* coords, void* workspace, size_t workspace_bytes,
                                const tpl_opts* opts, tpl_stream stream) {
    tpl_opts o = resolve(opts);
    tpl_status st = check_opts(o);
    if (st) return st;
    const void* ptrs[3] = {angles, lengths, coords};
    if ((st = check_chain_args(B, Lmax, ptrs, 3))) return st;
    if (B == 0) return ok();
    LaunchCfg cfg = backbone_cfg(o);
    if (!backbone_cfg_supported(cfg.threads, cfg.res_per_thread) ||
        (cfg.threads == 512 && cfg.res_per_thread == 4))
        return fail(TPL_ERR_INVALID_ARG, "unsupported backbone launch %d x %d", cfg.threads, cfg.res_per_thread);
    if ((st = check_ws(workspace, workspace_bytes, tpl_backbone_workspace_size(B, Lmax)))) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = launch_backbone_forward(angles, lengths, B, Lmax, coords, sched_mode(o, true),
                                            workspace, cfg, s);
    if (e != cudaSuccess) return cuda_fail(e, "backbone_forward");
    return ok();
}

tpl_status tpl_backbone_backward(const float* angles, const int32_t* lengths, int B, int Lmax,
                                 const float* coords, const float* grad_coords, float* grad_angles,
                                 void* workspace, size_t workspace_bytes, const tpl_opts* opts,
                                 tpl_stream stream) {
    tpl_opts o = resolve(opts);
    tpl_status st = check_opts(o);
    if (st) return st;
    const bool from_coords = o.bwd_mode == TPL_BWD_FROM_COORDS;
    const void* ptrs[5] = {angles, lengths, grad_coords, grad_angles, from_coords ? (const void*)coords : angles};
    if ((st = check_chain_args(B, Lmax, ptrs, 5))) return st;
    if (B == 0) return ok();
    LaunchCfg cfg = backbone_cfg(o);
    if (!backbone_cfg_supported(cfg.threads, cfg.res_per_thread) ||
        (cfg.threads == 512 && cfg.res_per_thread == 4))
        return fail(TPL_ERR_INVALID_ARG, "unsupported backbone launch %d x %d", cfg.threads, cfg.res_per_thread);
    if ((st = check_ws(workspace, workspace_bytes, tpl_backbone_workspace_size(B, Lmax)))) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = launch_backbone_backward(angles, lengths, B, Lmax, coords, grad_coords,
                                             grad_angles, from_coords, workspace, cfg, s);
    if (e != cudaSuccess) return cuda_fail(e, "backbone_backward");
    return ok();
}

tpl_status tpl_backbone_forward_o(const float* angles, const int32_t* lengths, int B, int Lmax, float* coords,
                                  float* o_coords, void* workspace, size_t workspace_bytes, const tpl_opts* opts,
                                  tpl_stream stream) {
    tpl_opts o = resolve(opts);
    tpl_status st = check_opts(o);
    if (st) return st;
    const void* ptrs[4] = {angles, lengths, coords, o_coords};
    if ((st = check_chain_args(B, Lmax, ptrs, 4))) return st;
    if (B == 0) return ok();
    LaunchCfg cfg = backbone_cfg(o);
    if (!backbone_o_cfg_supported(cfg.threads, cfg.res_per_thread))
        return fail(TPL_ERR_INVALID_ARG, "launch %d x %d not supported with the O atoms", cfg.threads,
                    cfg.res_per_thread);
    if ((st = check_ws(workspace, workspace_bytes, tpl_backbone_workspace_size(B, Lmax)))) return st;
    cudaError_t e = launch_backbone_forward_o(angles, lengths, B, Lmax, coords, o_coords, sched_mode(o, true),
                                              workspace, cfg, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "backbone_forward_o");
    return ok();
}

tpl_status tpl_backbone_backward_o(const float* angles, const int32_t* lengths, int B, int Lmax,
                                   const float* coords, const float* o_coords, const float* grad_coords,
                                   const float* grad_o, float* grad_angles, void* workspace, size_t workspace_bytes,
                                   const tpl_opts* opts, tpl_stream stream) {
    tpl_opts o = resolve(opts);
    tpl_status st = check_opts(o);
    if (st) return st;
    const bool from_coords = o.bwd_mode == TPL_BWD_FROM_COORDS;
    const void* ptrs[7] = {angles, lengths, grad_coords, grad_o, grad_angles,
                           from_coords ? (const void*)coords : angles, from_coords ? (const void*)o_coords : angles};
    if ((st = check_chain_args(B, Lmax, ptrs, 7))) return st;
    if (B == 0) return ok();
    LaunchCfg cfg = backbone_cfg(o);
    if (!backbone_o_cfg_supported(cfg.threads, cfg.res_per_thread))
        return fail(TPL_ERR_INVALID_ARG, "launch %d x %d not supported with the O atoms", cfg.threads,
                    cfg.res_per_thread);
    if ((st = check_ws(workspace, workspace_bytes, tpl_backbone_workspace_size(B, Lmax)))) return st;
    cudaError_t e = launch_backbone_backward_o(angles, lengths, B, Lmax, coords, o_coords, grad_coords, grad_o,
                                               grad_angles, from_coords, workspace, cfg,
                                               reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "backbone_backward_o");
    return ok();
}

tpl_status tpl_backbone_backward_quadratic(const int32_t* lengths, int B, int Lmax, const float* coords,
                                           const float* grad_coords, float* grad_angles, tpl_stream stream) {
    const void* ptrs[4] = {lengths, coords, grad_coords, grad_angles};
    tpl_status st = check_chain_args(B, Lmax, ptrs, 4);
    if (st) return st;
    if (B == 0) return ok();
    if (B > 65535) return fail(TPL_ERR_BAD_SHAPE, "B=%d above 65535 chains per call", B);
    cudaError_t e = launch_backbone_backward_quadratic(lengths, B, Lmax, coords, grad_coords, grad_angles,
                                                       reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "backbone_backward_quadratic");
    return ok();
}

tpl_status tpl_fullatom_backward_quadratic(const uint8_t* seq, const int32_t* lengths, int B, int Lmax, int Amax,
                                           const float* coords, const float* grad_coords, float* grad_angles,
                                           tpl_stream stream) {
    const void* ptrs[5] = {seq, lengths, coords, grad_coords, grad_angles};
    tpl_status st = check_chain_args(B, Lmax, ptrs, 5);
    if (st) return st;
    if (Amax < 0 || Amax % 4 != 0) return fail(TPL_ERR_BAD_SHAPE, "Amax=%d must be a multiple of 4", Amax);
    if (B == 0) return ok();
    if (B > 65535) return fail(TPL_ERR_BAD_SHAPE, "B=%d above 65535 chains per call", B);
    cudaError_t e = launch_fullatom_backward_quadratic(seq, lengths, B, Lmax, Amax, coords, grad_coords,
                                                       grad_angles, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "fullatom_backward_quadratic");
    return ok();
}

tpl_status tpl_fullatom_forward(const float* angles, const uint8_t* seq, const int32_t* lengths,
                                int B, int Lmax, int Amax, float* coords, int32_t* num_atoms,
                                void* workspace, size_t workspace_bytes, const tpl_opts* opts,
                                tpl_stream stream) {
    tpl_opts o = resolve(opts);
    tpl_status st = check_opts(o);
    if (st) return st;
    const void* ptrs[5] = {angles, seq, lengths, coords, num_atoms};
    if ((st = check_chain_args(B, Lmax, ptrs, 5))) return st;
    if (Amax < 0 || Amax % 4 != 0) return fail(TPL_ERR_BAD_SHAPE, "Amax=%d must be a multiple of 4", Amax);
    if (B == 0) return ok();
    LaunchCfg cfg = fullatom_cfg(o);
    if ((st = check_fullatom_cfg(cfg))) return st;
    if ((st = check_ws(workspace, workspace_bytes, tpl_fullatom_workspace_size(B, Lmax)))) return st;
    // packed (chains per CTA > 1) only on request, and only for a backward that
    // reads the coordinates (rebuilding frames works per tile of one chain)
    if (o.schedule == TPL_SCHED_PACKED && o.bwd_mode == TPL_BWD_RECOMPUTE)
        return fail(TPL_ERR_INVALID_ARG, "a packed full-atom schedule needs the FROM_COORDS backward");
    const int mode = o.schedule == TPL_SCHED_PACKED ? kSchedPacked : sched_mode(o, false);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = launch_fullatom_forward(angles, seq, lengths, B, Lmax, Amax, coords, num_atoms,
                                            mode, workspace, cfg, s);
    if (e != cudaSuccess) return cuda_fail(e, "fullatom_forward");
    return ok();
}

size_t tpl_fullatom_lrmsd_workspace_size(int B, int Lmax) { return chain_ws_bytes(B, Lmax, true, true); }

tpl_status tpl_fullatom_lrmsd_forward(const float* angles, const uint8_t* seq, const int32_t* lengths, int B,
                                      int Lmax, int Amax, const float* target, float* coords, int32_t* num_atoms,
                                      float* lrmsd, void* workspace, size_t workspace_bytes, const tpl_opts* opts,
                                      tpl_stream stream) {
    tpl_opts o = resolve(opts);
    tpl_status st = check_opts(o);
    if (st) return st;
    const void* ptrs[7] = {angles, seq, lengths, target, coords, num_atoms, lrmsd};
    if ((st = check_chain_args(B, Lmax, ptrs, 7))) return st;
    if (Amax < 0 || Amax % 4 != 0) return fail(TPL_ERR_BAD_SHAPE, "Amax=%d must be a multiple of 4", Amax);
    if (B == 0) return ok();
    LaunchCfg cfg = fullatom_cfg(o);
    if ((st = check_fullatom_cfg(cfg))) return st;
    if ((st = check_ws(workspace, workspace_bytes, tpl_fullatom_lrmsd_workspace_size(B, Lmax)))) return st;
    cudaError_t e = launch_fullatom_lrmsd_forward(angles, seq, lengths, target, B, Lmax, Amax, coords, num_atoms,
                                                  lrmsd, sched_mode(o, false), workspace, cfg,
                                                  reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "fullatom_lrmsd_forward");
    return ok();
}

tpl_status tpl_fullatom_lrmsd_backward(const uint8_t* seq, const int32_t* lengths, int B, int Lmax, int Amax,
                                       const float* coords, const float* target, const float* grad_lrmsd,
                                       float* grad_angles, void* workspace, size_t workspace_bytes,
                                       const tpl_opts* opts, tpl_stream stream) {
    tpl_opts o = resolve(opts);
    tpl_status st = check_opts(o);
    if (st) return st;
    const void* ptrs[6] = {seq, lengths, coords, target, grad_lrmsd, grad_angles};
    if ((st = check_chain_args(B, Lmax, ptrs, 6))) return st;
    if (Amax < 0 || Amax % 4 != 0) return fail(TPL_ERR_BAD_SHAPE, "Amax=%d must be a multiple of 4", Amax);
    if (B == 0) return ok();
    LaunchCfg cfg = fullatom_cfg(o);
    if ((st = check_fullatom_cfg(cfg))) return st;
    if ((st = check_ws(workspace, workspace_bytes, tpl_fullatom_lrmsd_workspace_size(B, Lmax)))) return st;
    cudaError_t e = launch_fullatom_lrmsd_backward(seq, lengths, coords, target, grad_lrmsd, B, Lmax, Amax,
                                                   grad_angles, workspace, cfg, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "fullatom_lrmsd_backward");
    return ok();
}

tpl_status tpl_backbone_lrmsd_step(const float* angles, const int32_t* lengths, int B, int Lmax,
                                   const float* target, const float* grad_lrmsd, float* coords, float* lrmsd,
                                   float* grad_angles, void* workspace, size_t workspace_bytes,
                                   const tpl_opts* opts, tpl_stream stream) {
    tpl_opts o = resolve(opts);
    tpl_status st = check_opts(o);
    if (st) return st;
    const void* ptrs[7] = {angles, lengths, target, grad_lrmsd, coords, lrmsd, grad_angles};
    if ((st = check_chain_args(B, Lmax, ptrs, 7))) return st;
    if (B == 0) return ok();
    if (o.bwd_mode == TPL_BWD_RECOMPUTE)
        return fail(TPL_ERR_INVALID_ARG, "the training step forms its gradient from the coordinates (no RECOMPUTE)");
    LaunchCfg cfg = backbone_cfg(o);
    if (!backbone_step_cfg_supported(cfg.threads, cfg.res_per_thread))
        return fail(TPL_ERR_INVALID_ARG, "launch shape %d threads x %d residues not supported by the training step",
                    cfg.threads, cfg.res_per_thread);
    if ((st = check_ws(workspace, workspace_bytes, tpl_backbone_lrmsd_workspace_size(B, Lmax)))) return st;
    cudaError_t e = launch_backbone_lrmsd_step(angles, lengths, B, Lmax, target, grad_lrmsd, coords, lrmsd,
                                               grad_angles, sched_mode(o, true), workspace, cfg,
                                               reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "backbone_lrmsd_step");
    return ok();
}

tpl_status tpl_backbone_backward_lrmsd(const float* angles, const int32_t* lengths, int B, int Lmax,
                                       const float* coords, const float* target, const float* grad_lrmsd,
                                       const void* lrmsd_workspace, size_t lrmsd_workspace_bytes,
                                       float* grad_angles, void* workspace, size_t workspace_bytes,
                                       const tpl_opts* opts, tpl_stream stream) {
    tpl_opts o = resolve(opts);
    tpl_status st = check_opts(o);
    if (st) return st;
    const void* ptrs[6] = {angles, lengths, coords, target, grad_lrmsd, grad_angles};
    if ((st = check_chain_args(B, Lmax, ptrs, 6))) return st;
    if (B == 0) return ok();
    LaunchCfg cfg = backbone_cfg(o);
    if (!backbone_cfg_supported(cfg.threads, cfg.res_per_thread) ||
        (cfg.threads == 512 && cfg.res_per_thread == 4))
        return fail(TPL_ERR_INVALID_ARG, "unsupported backbone launch %d x %d", cfg.threads, cfg.res_per_thread);
    if ((st = check_ws(workspace, workspace_bytes, tpl_backbone_workspace_size(B, Lmax)))) return st;
    if ((st = check_ws(const_cast<void*>(lrmsd_workspace), lrmsd_workspace_bytes,
                       tpl_lrmsd_workspace_size(B, 3 * Lmax))))
        return st;
    cudaError_t e = launch_backbone_backward_lrmsd(angles, lengths, B, Lmax, coords, target, grad_lrmsd,
                                                   lrmsd_state(lrmsd_workspace, B, 3 * Lmax), grad_angles,
                                                   workspace, cfg, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "backbone_backward_lrmsd");
    return ok();
}

tpl_status tpl_fullatom_backward_lrmsd(const float* angles, const uint8_t* seq, const int32_t* lengths,
                                       int B, int Lmax, int Amax, const float* coords, const float* target,
                                       const float* grad_lrmsd, const void* lrmsd_workspace,
                                       size_t lrmsd_workspace_bytes, float* grad_angles, void* workspace,
                                       size_t workspace_bytes, const tpl_opts* opts, tpl_stream stream) {
    tpl_opts o = resolve(opts);
    tpl_status st = check_opts(o);
    if (st) return st;
    const void* ptrs[7] = {angles, seq, lengths, coords, target, grad_lrmsd, grad_angles};
    if ((st = check_chain_args(B, Lmax, ptrs, 7))) return st;
    if (Amax < 0 || Amax % 4 != 0) return fail(TPL_ERR_BAD_SHAPE, "Amax=%d must be a multiple of 4", Amax);
    if (B == 0) return ok();
    LaunchCfg cfg = fullatom_cfg(o);
    if ((st = check_fullatom_cfg(cfg))) return st;
    if ((st = check_ws(workspace, workspace_bytes, tpl_fullatom_workspace_size(B, Lmax)))) return st;
    if ((st = check_ws(const_cast<void*>(lrmsd_workspace), lrmsd_workspace_bytes, tpl_lrmsd_workspace_size(B, Amax))))
        return st;
    cudaError_t e = launch_fullatom_backward_lrmsd(seq, lengths, B, Lmax, Amax, coords, target, grad_lrmsd,
                                                   lrmsd_state(lrmsd_workspace, B, Amax), grad_angles,
                                                   workspace, cfg, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "fullatom_backward_lrmsd");
    return ok();
}

tpl_status tpl_fullatom_backward(const float* angles, const uint8_t* seq, const int32_t* lengths,
                                 int B, int Lmax, int Amax, const float* coords,
                                 const float* grad_coords, float* grad_angles, void* workspace,
                                 size_t workspace_bytes, const tpl_opts* opts, tpl_stream stream) {
    tpl_opts o = resolve(opts);
    tpl_status st = check_opts(o);
    if (st) return st;
    // AUTO reads the forward's coordinates when they are given
    const bool from_coords = o.bwd_mode == TPL_BWD_FROM_COORDS ||
                             (o.bwd_mode == TPL_BWD_AUTO && coords != nullptr);
    const void* ptrs[6] = {angles, seq, lengths, grad_coords, grad_angles, from_coords ? (const void*)coords : angles};
    if ((st = check_chain_args(B, Lmax, ptrs, 6))) return st;
    if (Amax < 0 || Amax % 4 != 0) return fail(TPL_ERR_BAD_SHAPE, "Amax=%d must be a multiple of 4", Amax);
    if (B == 0) return ok();
    LaunchCfg cfg = fullatom_cfg(o);
    if ((st = check_fullatom_cfg(cfg))) return st;
    if (!from_coords && !fullatom_cfg_supported_recompute(cfg))
        return fail(TPL_ERR_INVALID_ARG,
                    "rebuilding frames from the angles needs one residue per thread and 128, 256 or 384 threads "
                    "(got %d x %d); pass the forward's coordinates", cfg.threads, cfg.res_per_thread);
    if ((st = check_ws(workspace, workspace_bytes, tpl_fullatom_workspace_size(B, Lmax)))) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = launch_fullatom_backward(angles, seq, lengths, B, Lmax, Amax, coords, grad_coords,
                                             grad_angles, from_coords, workspace, cfg, s);
    if (e != cudaSuccess) return cuda_fail(e, "fullatom_backward");
    return ok();
}

static tpl_status check_pair_args(int P, int Nmax, const void* const* ptrs, int nptr) {
    if (P < 0 || Nmax < 0) return fail(TPL_ERR_INVALID_ARG, "P=%d Nmax=%d must be >= 0", P, Nmax);
    if (Nmax % 4 != 0) return fail(TPL_ERR_BAD_SHAPE, "Nmax=%d must be a multiple of 4", Nmax);
    if ((long long)P * ((Nmax + 255) / 256 + 1) > 0x7fffffffLL)
        return fail(TPL_ERR_BAD_SHAPE, "P=%d x Nmax=%d too large for one call", P, Nmax);
    if (P == 0) return TPL_OK;
    for (int i = 0; i < nptr; ++i) {
        if (!ptrs[i]) return fail(TPL_ERR_INVALID_ARG, "pointer argument %d is NULL", i);
        if (!aligned16(ptrs[i])) return fail(TPL_ERR_MISALIGNED, "pointer argument %d not 16-byte aligned", i);
    }
    return TPL_OK;
}

tpl_status tpl_lrmsd_forward(const float* input, const float* target, const int32_t* num_atoms,
                             int P, int Nmax, float* lrmsd, void* workspace, size_t workspace_bytes,
                             tpl_stream stream) {
    const void* ptrs[4] = {input, target, num_atoms, lrmsd};
    tpl_status st = check_pair_args(P, Nmax, ptrs, 4);
    if (st) return st;
    if (P == 0) return ok();
    if ((st = check_ws(workspace, workspace_bytes, tpl_lrmsd_workspace_size(P, Nmax)))) return st;
    cudaError_t e = launch_lrmsd_forward(input, target, num_atoms, P, Nmax, lrmsd, workspace,
                                         reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "lrmsd_forward");
    return ok();
}

tpl_status tpl_lrmsd_backward(const float* grad_lrmsd, const float* input, const float* target,
                              const int32_t* num_atoms, int P, int Nmax, float* grad_input,
                              const void* workspace, size_t workspace_bytes, tpl_stream stream) {
    const void* ptrs[5] = {grad_lrmsd, input, target, num_atoms, grad_input};
    tpl_status st = check_pair_args(P, Nmax, ptrs, 5);
    if (st) return st;
    if (P == 0) return ok();
    if ((st = check_ws(const_cast<void*>(workspace), workspace_bytes, tpl_lrmsd_workspace_size(P, Nmax))))
        return st;
    cudaError_t e = launch_lrmsd_backward(grad_lrmsd, input, target, num_atoms, P, Nmax, grad_input,
                                          workspace, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "lrmsd_backward");
    return ok();
}

tpl_status tpl_lrmsd_forward_noalloc(const float* input, const float* target,
                                     const int32_t* num_atoms, int P, int Nmax, float* lrmsd,
                                     tpl_stream stream) {
    const void* ptrs[4] = {input, target, num_atoms, lrmsd};
    tpl_status st = check_pair_args(P, Nmax, ptrs, 4);
    if (st) return st;
    if (P == 0) return ok();
    if (P > lrmsd_noalloc_max_pairs() || Nmax > lrmsd_noalloc_max_atoms())
        return fail(TPL_ERR_BAD_SHAPE,
                    "P=%d, Nmax=%d exceed the allocation-free limits (P <= %d, Nmax <= %d); "
                    "use tpl_lrmsd_forward with a workspace",
                    P, Nmax, lrmsd_noalloc_max_pairs(), lrmsd_noalloc_max_atoms());
    cudaError_t e = launch_lrmsd_forward_noalloc(input, target, num_atoms, P, Nmax, lrmsd,
                                                 reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "lrmsd_forward_noalloc");
    return ok();
}

// --------------------------------------------------------------------------- FP64 forms
static tpl_status check_ref_args(int B, int Lmax, const void* const* ptrs, int nptr) {
    if (B < 0 || Lmax < 0) return fail(TPL_ERR_INVALID_ARG, "sizes must be >= 0");
    if (B > 2147483647 / 2) return fail(TPL_ERR_BAD_SHAPE, "batch too large");
    if (B == 0) return TPL_OK;
    for (int i = 0; i < nptr; ++i)
        if (!ptrs[i]) return fail(TPL_ERR_INVALID_ARG, "pointer argument %d is NULL", i);
    return TPL_OK;
}

tpl_status tpl_backbone_forward_ref64(const double* angles, const int32_t* lengths, int B, int Lmax,
                                      double* coords, tpl_stream stream) {
    const void* ptrs[3] = {angles, lengths, coords};
    tpl_status st = check_ref_args(B, Lmax, ptrs, 3);
    if (st) return st;
    cudaError_t e = launch_backbone_forward_ref64(angles, lengths, B, Lmax, coords,
                                                  reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ok() : cuda_fail(e, "backbone_forward_ref64");
}

tpl_status tpl_backbone_backward_ref64(const double* angles, const int32_t* lengths, int B,
                                       int Lmax, const double* coords, const double* grad_coords,
                                       double* grad_angles, tpl_stream stream) {
    const void* ptrs[4] = {lengths, coords, grad_coords, grad_angles};
    tpl_status st = check_ref_args(B, Lmax, ptrs, 4);
    if (st) return st;
    cudaError_t e = launch_backbone_backward_ref64(angles, lengths, B, Lmax, coords, grad_coords,
                                                   grad_angles, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ok() : cuda_fail(e, "backbone_backward_ref64");
}

tpl_status tpl_fullatom_forward_ref64(const double* angles, const uint8_t* seq,
                                      const int32_t* lengths, int B, int Lmax, int Amax,
                                      double* coords, int32_t* num_atoms, tpl_stream stream) {
    const void* ptrs[5] = {angles, seq, lengths, coords, num_atoms};
    tpl_status st = check_ref_args(B, Lmax, ptrs, 5);
    if (st) return st;
    if (Amax < 0) return fail(TPL_ERR_INVALID_ARG, "Amax must be >= 0");
    cudaError_t e = launch_fullatom_forward_ref64(angles, seq, lengths, B, Lmax, Amax, coords,
                                                  num_atoms, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ok() : cuda_fail(e, "fullatom_forward_ref64");
}

tpl_status tpl_fullatom_backward_ref64(const double* angles, const uint8_t* seq,
                                       const int32_t* lengths, int B, int Lmax, int Amax,
                                       const double* coords, const double* grad_coords,
                                       double* grad_angles, tpl_stream stream) {
    const void* ptrs[5] = {seq, lengths, coords, grad_coords, grad_angles};
    tpl_status st = check_ref_args(B, Lmax, ptrs, 5);
    if (st) return st;
    if (Amax < 0) return fail(TPL_ERR_INVALID_ARG, "Amax must be >= 0");
    cudaError_t e = launch_fullatom_backward_ref64(angles, seq, lengths, B, Lmax, Amax, coords,
                                                   grad_coords, grad_angles,
                                                   reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ok() : cuda_fail(e, "fullatom_backward_ref64");
}

tpl_status tpl_lrmsd_forward_ref64(const double* input, const double* target,
                                   const int32_t* num_atoms, int P, int Nmax, double* lrmsd,
                                   double* lrmsd_state, tpl_stream stream) {
    const void* ptrs[5] = {input, target, num_atoms, lrmsd, lrmsd_state};
    tpl_status st = check_ref_args(P, Nmax, ptrs, 5);
    if (st) return st;
    cudaError_t e = launch_lrmsd_forward_ref64(input, target, num_atoms, P, Nmax, lrmsd, lrmsd_state,
                                               reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ok() : cuda_fail(e, "lrmsd_forward_ref64");
}

tpl_status tpl_lrmsd_backward_ref64(const double* grad_lrmsd, const double* input,
                                    const double* target, const int32_t* num_atoms, int P,
                                    int Nmax, const double* lrmsd_state, double* grad_input,
                                    tpl_stream stream) {
    const void* ptrs[6] = {grad_lrmsd, input, target, num_atoms, lrmsd_state, grad_input};
    tpl_status st = check_ref_args(P, Nmax, ptrs, 6);
    if (st) return st;
    cudaError_t e = launch_lrmsd_backward_ref64(grad_lrmsd, input, target, num_atoms, P, Nmax,
                                                lrmsd_state, grad_input,
                                                reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ok() : cuda_fail(e, "lrmsd_backward_ref64");
}

// --------------------------------------------------------------------------- host helpers
tpl_status tpl_residue_table(int code, char* three_letter, int* n_atoms, int* n_chi) {
    if (code < 0 || code >= kNumTypes) return fail(TPL_ERR_INVALID_ARG, "residue code %d", code);
    const FaTable& t = fa_table();
    if (three_letter) {
        memcpy(three_letter, residue_three(code), 3);
        three_letter[3] = 0;
    }
    if (n_atoms) *n_atoms = t.n_atoms[code];
    if (n_chi) *n_chi = t.n_chi[code];
    return ok();
}

tpl_status tpl_residue_atom(int code, int idx, char* name, int* group, float* r0) {
    if (code < 0 || code >= kNumTypes) return fail(TPL_ERR_INVALID_ARG, "residue code %d", code);
    const FaTableD& d = fa_table_d();
    if (idx < 0 || idx >= d.n_atoms[code]) return fail(TPL_ERR_INVALID_ARG, "atom index %d", idx);
    if (name) {
        strncpy(name, residue_atom_name(code, idx), 7);
        name[7] = 0;
    }
    if (group) *group = d.group[code][idx];
    if (r0)
        for (int k = 0; k < 3; ++k) r0[k] = (float)d.r0[code][idx][k];
    return ok();
}

int tpl_fullatom_chain_atoms(const uint8_t* seq_host, int length) {
    if (!seq_host || length < 0) return -1;
    const FaTable& t = fa_table();
    int n = 0;
    for (int j = 0; j < length; ++j) {
        if (seq_host[j] >= kNumTypes) return -1;
        n += t.n_atoms[seq_host[j]];
    }
    return n;
}

int tpl_fullatom_max_atoms(const uint8_t* seq_host, const int32_t* lengths_host, int B, int Lmax) {
    if (B < 0 || Lmax < 0 || (B > 0 && (!seq_host || !lengths_host))) return -1;
    int best = 0;
    for (int b = 0; b < B; ++b) {
        const int L = lengths_host[b];
        if (L < 0 || L > Lmax) return -1;
        const int n = tpl_fullatom_chain_atoms(seq_host + (size_t)b * Lmax, L);
        if (n < 0) return -1;
        if (n > best) best = n;
    }
    return best;
}

int backbone_candidates(int bwd_mode, tpl_opts* cands) {
    int n = 0;
    const int threads[4] = {64, 128, 256, 512}, ks[3] = {1, 2, 4}, sch[2] = {TPL_SCHED_PACKED, TPL_SCHED_LONGEST_FIRST};
    for (int si = 0; si < 2; ++si)
        for (int ti = 0; ti < 4; ++ti)
            for (int ki = 0; ki < 3; ++ki) {
                if (!backbone_cfg_supported(threads[ti], ks[ki]) || (threads[ti] == 512 && ks[ki] == 4)) continue;
                tpl_opts o;
                memset(&o, 0, sizeof(o));
                o.bwd_mode = bwd_mode;
                o.threads = threads[ti];
                o.res_per_thread = ks[ki];
                o.schedule = sch[si];
                cands[n++] = o;
            }
    return n;
}

int fullatom_candidates(int bwd_mode, tpl_opts* cands) {
    int n = 0;
    const int shapes[7][2] = {{128, 1}, {256, 1}, {384, 1}, {128, 2}, {192, 2}, {64, 4}, {192, 4}};
    // packed schedules (chains per CTA > 1) need a backward that reads the coordinates
    const int sch[3] = {TPL_SCHED_BATCH_ORDER, TPL_SCHED_LONGEST_FIRST, TPL_SCHED_PACKED};
    const int nsch = bwd_mode == TPL_BWD_RECOMPUTE ? 2 : 3;
    for (int si = 0; si < nsch; ++si)
        for (int ti = 0; ti < 7; ++ti) {
            tpl_opts o;
            memset(&o, 0, sizeof(o));
            o.bwd_mode = bwd_mode;
            o.threads = shapes[ti][0];
            o.res_per_thread = shapes[ti][1];
            o.schedule = sch[si];
            // rebuilding frames from the angles takes one residue per thread
            if (bwd_mode == TPL_BWD_RECOMPUTE && !fullatom_cfg_supported_recompute(LaunchCfg{o.threads, o.res_per_thread}))
                continue;
            cands[n++] = o;
        }
    return n;
}

tpl_status tpl_backbone_autotune(const float* angles, const int32_t* lengths, int B, int Lmax,
                                 float* coords, const float* grad_coords, float* grad_angles,
                                 void* workspace, size_t workspace_bytes, int bwd_mode, tpl_opts* best,
                                 float* best_ms, tpl_stream stream) {
    if (!best) return fail(TPL_ERR_INVALID_ARG, "best is NULL");
    tpl_opts cands[32];
    const int n = backbone_candidates(bwd_mode, cands);
    return tune(cands, n, reinterpret_cast<cudaStream_t>(stream), [&](const tpl_opts& o, tpl_stream ts) {
        tpl_status st = tpl_backbone_forward(angles, lengths, B, Lmax, coords, workspace, workspace_bytes, &o, ts);
        if (st) return st;
        return tpl_backbone_backward(angles, lengths, B, Lmax, coords, grad_coords, grad_angles, workspace,
                                     workspace_bytes, &o, ts);
    }, best, best_ms);
}

tpl_status tpl_backbone_lrmsd_autotune(const float* angles, const int32_t* lengths, int B, int Lmax,
                                       float* coords, const float* target, const int32_t* num_atoms,
                                       const float* grad_lrmsd, float* lrmsd, void* lrmsd_workspace,
                                       size_t lrmsd_workspace_bytes, float* grad_angles, void* workspace,
                                       size_t workspace_bytes, tpl_opts* best, float* best_ms, tpl_stream stream) {
    if (!best) return fail(TPL_ERR_INVALID_ARG, "best is NULL");
    tpl_opts cands[32];
    const int n = backbone_candidates(TPL_BWD_FROM_COORDS, cands);
    return tune(cands, n, reinterpret_cast<cudaStream_t>(stream), [&](const tpl_opts& o, tpl_stream ts) {
        tpl_status st = tpl_backbone_forward(angles, lengths, B, Lmax, coords, workspace, workspace_bytes, &o, ts);
        if (st) return st;
        st = tpl_lrmsd_forward(coords, target, num_atoms, B, 3 * Lmax, lrmsd, lrmsd_workspace, lrmsd_workspace_bytes,
                               ts);
        if (st) return st;
        return tpl_backbone_backward_lrmsd(angles, lengths, B, Lmax, coords, target, grad_lrmsd, lrmsd_workspace,
                                           lrmsd_workspace_bytes, grad_angles, workspace, workspace_bytes, &o,
                                           ts);
    }, best, best_ms);
}

tpl_status tpl_fullatom_autotune(const float* angles, const uint8_t* seq, const int32_t* lengths, int B,
                                 int Lmax, int Amax, float* coords, int32_t* num_atoms,
                                 const float* grad_coords, float* grad_angles, void* workspace,
                                 size_t workspace_bytes, int bwd_mode, tpl_opts* best, float* best_ms,
                                 tpl_stream stream) {
    if (!best) return fail(TPL_ERR_INVALID_ARG, "best is NULL");
    tpl_opts cands[32];
    const int n = fullatom_candidates(bwd_mode, cands);
    return tune(cands, n, reinterpret_cast<cudaStream_t>(stream), [&](const tpl_opts& o, tpl_stream ts) {
        tpl_status st = tpl_fullatom_forward(angles, seq, lengths, B, Lmax, Amax, coords, num_atoms, workspace,
                                             workspace_bytes, &o, ts);
        if (st) return st;
        return tpl_fullatom_backward(angles, seq, lengths, B, Lmax, Amax, coords, grad_coords, grad_angles,
                                     workspace, workspace_bytes, &o, ts);
    }, best, best_ms);
}

tpl_status tpl_fullatom_lrmsd_autotune(const float* angles, const uint8_t* seq, const int32_t* lengths, int B,
                                       int Lmax, int Amax, float* coords, int32_t* num_atoms, const float* target,
                                       const float* grad_lrmsd, float* lrmsd, void* lrmsd_workspace,
                                       size_t lrmsd_workspace_bytes, float* grad_angles, void* workspace,
                                       size_t workspace_bytes, tpl_opts* best, float* best_ms, tpl_stream stream) {
    if (!best) return fail(TPL_ERR_INVALID_ARG, "best is NULL");
    tpl_opts cands[32];
    const int n = fullatom_candidates(TPL_BWD_FROM_COORDS, cands);
    return tune(cands, n, reinterpret_cast<cudaStream_t>(stream), [&](const tpl_opts& o, tpl_stream ts) {
        tpl_status st = tpl_fullatom_forward(angles, seq, lengths, B, Lmax, Amax, coords, num_atoms, workspace,
                                             workspace_bytes, &o, ts);
        if (st) return st;
        st = tpl_lrmsd_forward(coords, target, num_atoms, B, Amax, lrmsd, lrmsd_workspace, lrmsd_workspace_bytes,
                               ts);
        if (st) return st;
        return tpl_fullatom_backward_lrmsd(angles, seq, lengths, B, Lmax, Amax, coords, target, grad_lrmsd,
                                           lrmsd_workspace, lrmsd_workspace_bytes, grad_angles, workspace,
                                           workspace_bytes, &o, ts);
    }, best, best_ms);
}

tpl_status tpl_selftest_wait_timeout(const int* flag, tpl_stream stream) {
    if (!flag || (reinterpret_cast<uintptr_t>(flag) & 3u))
        return fail(TPL_ERR_INVALID_ARG, "flag is NULL or not 4-byte aligned");
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) return fail(TPL_ERR_NO_DEVICE, "no CUDA device");
    selftest_wait_kernel<<<1, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(flag);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ok() : cuda_fail(e, "selftest_wait_timeout");
}

tpl_status tpl_get_status(tpl_stream stream, int* device_status) {
    if (!device_status) return fail(TPL_ERR_INVALID_ARG, "device_status is NULL");
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) return fail(TPL_ERR_NO_DEVICE, "no CUDA device");
    cudaError_t e = read_and_clear_status(reinterpret_cast<cudaStream_t>(stream), device_status);
    return e == cudaSuccess ? ok() : cuda_fail(e, "get_status");
}

}  // extern "C"
