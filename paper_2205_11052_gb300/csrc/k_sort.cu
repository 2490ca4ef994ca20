// Periodic binning: counting sort of the particle store by deposit tile,
// followed by the deposit work list (tile, particle range) build.
//
// The paper has no sort (its nearest step is the particle-to-rank search of
// Section 5.2.1); binning keeps particles grouped by deposit tile so the
// deposit can accumulate each tile in shared memory.
//
// Key of a particle with stencil base (i, j, k), tile T = (Tx, Ty, Tz):
//   key = ti + ntx (tj + nty tk),   (ti, tj, tk) = (i/Tx, j/Ty, k/Tz).
// Between sorts particles drift by a fraction of a cell per step, so a warp
// of consecutive particles mostly shares one tile: its lanes claim one
// contiguous destination range with a single atomic and the scatter writes
// stay coalesced.  (Cell-level keys would send the 32 lanes of a warp to ~32
// different cells after any drift, i.e. 4-byte scattered stores.)
// Passes: histogram (warp-aggregated atomics) -> exclusive scan (in place) ->
// scatter (the scanned offsets serve as cursors; afterwards bins[key] holds
// the end of bin key) -> per-tile ranges -> scan of items per tile -> items.
// Order within a tile is the claim order (not deterministic).
#include <algorithm>

#include "pic_internal.cuh"

namespace pic {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanSeg = kScanThreads * kScanItems;   // 4096 elements per block

__device__ __forceinline__ int tile_key(int32_t c, const Geom &g, int &bad) {
    int i = cell_i(c), j = cell_j(c), k = cell_k(c);
    if (i >= g.n[0] || j >= g.n[1] || k >= g.n[2]) {   // never produced by the kernels
        bad = 1;
        i = j = k = 0;
    }
    // exact division by the tile size through a multiply-high (indices < 2^10)
    const int ti = tile_div(i, g.tdiv[0]), tj = tile_div(j, g.tdiv[1]), tk = tile_div(k, g.tdiv[2]);
    return ti + g.ntile[0] * (tj + g.ntile[1] * tk);
}

// Lanes of a warp whose keys form a contiguous run (consecutive lanes, equal
// keys; binned particles arrive in such runs) share shared-table updates:
// the run's first lane does one update for the whole run.
struct WarpRun {
    int head;   // first lane of this lane's run
    int len;    // its length
};

__device__ __forceinline__ WarpRun warp_run(int key) {
    const int lane = threadIdx.x & 31;
    const int prev = __shfl_up_sync(0xffffffffu, key, 1);
    const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || key != prev);
    const unsigned upto = (lane == 31) ? 0xffffffffu : ((2u << lane) - 1u);
    WarpRun r;
    r.head = 31 - __clz(heads & upto);
    const unsigned after = heads & ~((r.head == 31) ? 0xffffffffu : ((2u << r.head) - 1u));
    r.len = (after ? __ffs(after) - 1 : 32) - r.head;
    return r;
}

// slot of `key` in the shared open-addressing table (inserting it), or -1
// when the table is full
__device__ __forceinline__ int table_slot(int32_t *hkey, int key, int size) {
    int h = (int)(((unsigned)key * 2654435761u) >> 24) & (size - 1);
    for (int probes = 0; probes < size; ++probes) {
        const int k = hkey[h];
        if (k == key) return h;
        if (k == -1) {
            const int prev = atomicCAS(&hkey[h], -1, key);
            if (prev == -1 || prev == key) return h;
        }
        h = (h + 1) & (size - 1);
    }
    return -1;
}

#ifndef PIC_SORT_STAGE
#define PIC_SORT_STAGE 512
#endif
constexpr int kStage = PIC_SORT_STAGE;     // particles per staged slice
constexpr int kHash = 256;                 // slots of the per-slice tile table
constexpr int kPerThread = kStage / 256;   // the staged kernels run 256 threads per block
#ifndef PIC_HIST_STAGE
#define PIC_HIST_STAGE 2048
#endif
constexpr int kHistStage = PIC_HIST_STAGE;   // particles per histogram slice
constexpr int kHistPer = kHistStage / 256;

// ---- bulk asynchronous copies (TMA) into shared memory, mbarrier completion ----

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// bounded wait for the phase of the given parity; false if it gave up
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (int it = 0; it < (1 << 22); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Block-staged scatter.  A block takes kStage consecutive particles into
// shared memory, finds the slice's distinct destination tiles with a small
// shared hash table (a slice comes from one or two tiles plus strays into
// their neighbours, i.e. a few dozen keys), claims one global range per tile
// with one atomic, and writes every tile's particles contiguously, in
// destination order (a slice-local scan of the table's counts gives each
// particle its position in the slice's output runs; thread t then writes the
// t-th particle of those runs, so a warp's stores fall into one or two runs of
// consecutive addresses even when half the slice changes tile).  A slice
// with more distinct tiles than the table holds (the first binning of
// particles in arbitrary order) falls back to per-warp claims.
//
// The slices a block walks are double-buffered: while one is processed, the
// eight arrays of its next slice arrive by bulk asynchronous copies (2 KB
// each, completion counted on an mbarrier); a partial last slice is loaded
// with plain loads.  Every wait is bounded: a copy that never completes
// raises PIC_FLAG_TIMEOUT and the block stops.
constexpr int kArrays = 8;                                   // cell, o[3], v[3], pid
constexpr size_t kBufBytes = (size_t)kStage * 4 * kArrays;   // one staged slice
static_assert(kHash == 256, "the staged scatter scans its table with one thread per slot");
constexpr size_t kStageSmem = 2 * kBufBytes + (size_t)kStage * 4 + (size_t)kHash * 12 +
                              2 * sizeof(uint64_t) + (size_t)kStage * 2;

// the arrays of a set from particle o on
__device__ __forceinline__ ParticleSet offset_set(ParticleSet s, int64_t o) {
    s.cell += o;
    for (int d = 0; d < 3; ++d) {
        s.o[d] += o;
        s.v[d] += o;
    }
    s.pid += o;
    return s;
}

__device__ __forceinline__ const void *src_array(const ParticleSet &s, int a) {
    if (a == 0) return s.cell;
    if (a < 4) return s.o[a - 1];
    if (a < 7) return s.v[a - 4];
    return s.pid;
}

// SortRange: particles [o, o + n) of set ctrl->cur ^ rel move to the same
// range of the other set
struct SortRange {
    int64_t o;
    int rel;
};

__global__ void __launch_bounds__(256) k_scatter_staged(int64_t n, Geom g, Ctrl *ctrl,
                                                         int32_t *bins, int shift, SortRange rg) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint32_t *buf0 = reinterpret_cast<uint32_t *>(smem);
    uint16_t *slid = reinterpret_cast<uint16_t *>(smem + 2 * kBufBytes);    // kStage table slots
    uint16_t *srank = slid + kStage;                                         // kStage ranks
    int32_t *hkey = reinterpret_cast<int32_t *>(srank + kStage);             // kHash keys
    int32_t *hcnt = hkey + kHash;                                            // kHash counts
    int32_t *hbase = hcnt + kHash;                                           // kHash global bases
    uint64_t *bar = reinterpret_cast<uint64_t *>(hbase + kHash);             // 2 mbarriers
    uint16_t *inv = reinterpret_cast<uint16_t *>(bar + 2);                   // kStage positions
    __shared__ int overflow;
    __shared__ int wsum[8];

    const int cur = ctrl->cur ^ rg.rel;
    const ParticleSet src = offset_set(ctrl->sets[cur], rg.o);
    const ParticleSet dst = offset_set(ctrl->sets[1 - cur], rg.o);
    const int64_t nslices = (n + kStage - 1) / kStage;
    int bad = 0;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    // issue the bulk copies of a full slice into buffer b (thread 0)
    auto issue = [&](int64_t sl, int b) {
        uint32_t *bb = buf0 + (size_t)b * kStage * kArrays;
        fence_proxy_async();
        mbar_arrive_expect_tx(&bar[b], (uint32_t)kBufBytes);
        for (int a = 0; a < kArrays; ++a)
            bulk_load(bb + (size_t)a * kStage,
                      static_cast<const uint32_t *>(src_array(src, a)) + sl * kStage,
                      (uint32_t)(kStage * 4), &bar[b]);
    };
    uint32_t phase[2] = {0u, 0u};
    int b = 0;
    int64_t sl = blockIdx.x;
    if (sl < nslices && (sl + 1) * kStage <= n && threadIdx.x == 0) issue(sl, 0);
    for (; sl < nslices; sl += gridDim.x, b ^= 1) {
        const int64_t s0 = sl * kStage;
        const int m = (int)(s0 + kStage <= n ? kStage : n - s0);
        uint32_t *bb = buf0 + (size_t)b * kStage * kArrays;
        int32_t *sc = reinterpret_cast<int32_t *>(bb);
        float *so = reinterpret_cast<float *>(bb + kStage);          // 3 x kStage offsets
        float *sv = reinterpret_cast<float *>(bb + 4 * kStage);      // 3 x kStage velocities
        int32_t *sid = reinterpret_cast<int32_t *>(bb + 7 * kStage); // kStage ids
        for (int h = threadIdx.x; h < kHash; h += blockDim.x) {
            hkey[h] = -1;
            hcnt[h] = 0;
        }
        if (threadIdx.x == 0) overflow = 0;
        if (m == kStage) {
            const bool ok = mbar_wait(&bar[b], phase[b]);
            phase[b] ^= 1u;
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0) atomicOr(&ctrl->flags, PIC_FLAG_TIMEOUT);
                mbar_wait(&bar[b], phase[b] ^ 1u);   // one more bounded wait for the copies
                return;
            }
        } else {
            for (int j = threadIdx.x; j < m; j += blockDim.x) {
                const int64_t p = s0 + j;
                sc[j] = __ldcs(src.cell + p);
                so[j] = __ldcs(src.o[0] + p);
                so[kStage + j] = __ldcs(src.o[1] + p);
                so[2 * kStage + j] = __ldcs(src.o[2] + p);
                sv[j] = __ldcs(src.v[0] + p);
                sv[kStage + j] = __ldcs(src.v[1] + p);
                sv[2 * kStage + j] = __ldcs(src.v[2] + p);
                sid[j] = __ldcs(src.pid + p);
            }
            __syncthreads();
        }
        // the next slice of this block streams into the other buffer meanwhile
        {
            const int64_t nx = sl + gridDim.x;
            if (nx < nslices && (nx + 1) * kStage <= n && threadIdx.x == 0) issue(nx, b ^ 1);
        }
        // slot of each particle's tile in the table and its rank there; the
        // first lane of each run of equal keys in a warp acts for the run
        for (int jb = 0; jb < m; jb += blockDim.x) {
            const int j = jb + threadIdx.x;
            const bool act = j < m;
            const int lane = threadIdx.x & 31;
            const int key = act ? tile_key(sc[j], g, bad) >> shift : -1 - lane;
            const WarpRun r = warp_run(key);
            int h = 0, base = 0;
            if (act && lane == r.head) {
                h = table_slot(hkey, key, kHash);
                if (h >= 0) base = atomicAdd(&hcnt[h], r.len);
            }
            h = __shfl_sync(0xffffffffu, h, r.head);
            base = __shfl_sync(0xffffffffu, base, r.head);
            if (act) {
                if (h < 0) {
                    overflow = 1;
                    slid[j] = 0xffff;
                } else {
                    slid[j] = (uint16_t)h;
                    srank[j] = (uint16_t)(base + (lane - r.head));
                }
            }
        }
        __syncthreads();
        if (overflow) {
            // arbitrary input order: claim per particle (aggregated per warp)
            const int lane = threadIdx.x & 31;
            for (int jb = 0; jb < m; jb += blockDim.x) {
                const int j = jb + threadIdx.x;
                const bool act = j < m;
                const unsigned active = __ballot_sync(0xffffffffu, act);
                if (act) {
                    const int key = tile_key(sc[j], g, bad) >> shift;
                    const unsigned peers = __match_any_sync(active, key);
                    const int leader = __ffs(peers) - 1;
                    int old = 0;
                    if (lane == leader) old = atomicAdd(bins + key, __popc(peers));
                    const int q = __shfl_sync(peers, old, leader) + __popc(peers & ((1u << lane) - 1u));
                    dst.cell[q] = sc[j];
                    dst.o[0][q] = so[j];
                    dst.o[1][q] = so[kStage + j];
                    dst.o[2][q] = so[2 * kStage + j];
                    dst.v[0][q] = sv[j];
                    dst.v[1][q] = sv[kStage + j];
                    dst.v[2][q] = sv[2 * kStage + j];
                    dst.pid[q] = sid[j];
                }
            }
        } else {
            {
                // claim, then turn hcnt into the slots' slice-local offsets
                // (exclusive scan, one thread per slot)
                const int h = threadIdx.x, lane = h & 31, w = h >> 5;
                const int cnt = hcnt[h];
                if (cnt > 0) hbase[h] = atomicAdd(bins + hkey[h], cnt);
                int incl = cnt;
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                if (lane == 31) wsum[w] = incl;
                __syncthreads();
                int before = 0;
                for (int q = 0; q < w; ++q) before += wsum[q];
                hcnt[h] = before + incl - cnt;
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < kPerThread; ++u) {
                const int j = u * 256 + threadIdx.x;
                if (j < m) inv[hcnt[slid[j]] + srank[j]] = (uint16_t)j;
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < kPerThread; ++u) {
                const int t = u * 256 + threadIdx.x;
                if (t < m) {
                    const int j = inv[t];
                    const int q = hbase[slid[j]] + srank[j];
                    dst.cell[q] = sc[j];
                    dst.o[0][q] = so[j];
                    dst.o[1][q] = so[kStage + j];
                    dst.o[2][q] = so[2 * kStage + j];
                    dst.v[0][q] = sv[j];
                    dst.v[1][q] = sv[kStage + j];
                    dst.v[2][q] = sv[2 * kStage + j];
                    dst.pid[q] = sid[j];
                }
            }
        }
        __syncthreads();   // buffer b and the table are free again
    }
    if (bad) atomicOr(&ctrl->flags, PIC_FLAG_BAD_CELL);
}

// Histogram with the same per-slice aggregation: counts of the slice's
// distinct tiles in a shared hash table, one global atomic per tile and
// slice (per-warp aggregated atomics when the table overflows).
__global__ void __launch_bounds__(256) k_histogram_staged(int64_t n, Geom g, Ctrl *ctrl,
                                                           int32_t *bins, int shift, SortRange rg) {
    __shared__ int32_t hkey[kHash];
    __shared__ int32_t hcnt[kHash];
    const ParticleSet ps = offset_set(ctrl->sets[ctrl->cur ^ rg.rel], rg.o);
    const int64_t nslices = (n + kHistStage - 1) / kHistStage;
    int bad = 0;
    for (int64_t sl = blockIdx.x; sl < nslices; sl += gridDim.x) {
        const int64_t s0 = sl * kHistStage;
        const int m = (int)(s0 + kHistStage <= n ? kHistStage : n - s0);
        for (int h = threadIdx.x; h < kHash; h += blockDim.x) {
            hkey[h] = -1;
            hcnt[h] = 0;
        }
        __syncthreads();
        // the slice's cells first (kHistStage / 256 loads in flight per thread)
        int32_t cv[kHistPer];
#pragma unroll
        for (int u = 0; u < kHistPer; ++u) {
            const int j = u * 256 + threadIdx.x;
            cv[u] = j < m ? __ldcs(ps.cell + s0 + j) : 0;
        }
#pragma unroll
        for (int u = 0; u < kHistPer; ++u) {
            const int j = u * 256 + threadIdx.x;
            const bool act = j < m;
            const int lane = threadIdx.x & 31;
            const int key = act ? tile_key(cv[u], g, bad) >> shift : -1 - lane;
            const WarpRun r = warp_run(key);
            if (act && lane == r.head) {
                const int h = table_slot(hkey, key, kHash);
                if (h >= 0) atomicAdd(&hcnt[h], r.len);
                else atomicAdd(bins + key, r.len);   // table full: straight to the grid
            }
        }
        __syncthreads();
        for (int h = threadIdx.x; h < kHash; h += blockDim.x)
            if (hcnt[h] > 0) atomicAdd(bins + hkey[h], hcnt[h]);
        __syncthreads();
    }
    if (bad) atomicOr(&ctrl->flags, PIC_FLAG_BAD_CELL);
}


// ---- exclusive scan of int32 (in place), total written to data[n] -------------

__device__ __forceinline__ int block_exclusive_scan(int val, int *total) {
    __shared__ int warp_tot[kScanThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = val;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int w = (lane < kScanThreads / 32) ? warp_tot[lane] : 0;
        int wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = wi - w;   // exclusive warp offsets
        if (lane == kScanThreads / 32 - 1) *total = wi;
    }
    __syncthreads();
    const int r = warp_tot[wid] + inc - val;
    __syncthreads();
    return r;
}

__global__ void k_scan_reduce(const int32_t *__restrict__ data, int64_t n, int32_t *sums) {
    const int64_t seg0 = (int64_t)blockIdx.x * kScanSeg;
    int s = 0;
    for (int q = 0; q < kScanItems; ++q) {
        const int64_t idx = seg0 + (int64_t)q * kScanThreads + threadIdx.x;
        if (idx < n) s += data[idx];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ int ws[kScanThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) t += ws[w];
        sums[blockIdx.x] = t;
    }
}

// single block: exclusive scan of the nb block sums, total to sums[nb]
__global__ void k_scan_top(int32_t *sums, int nb) {
    __shared__ int tot;
    int carry = 0;
    for (int base = 0; base < nb; base += kScanThreads) {
        const int idx = base + threadIdx.x;
        const int val = idx < nb ? sums[idx] : 0;
        const int ex = block_exclusive_scan(val, &tot);
        if (idx < nb) sums[idx] = carry + ex;
        __syncthreads();
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void k_scan_apply(int32_t *data, int64_t n, const int32_t *sums, int nb) {
    __shared__ int tot;
    const int64_t seg0 = (int64_t)blockIdx.x * kScanSeg;
    const int64_t t0 = seg0 + (int64_t)threadIdx.x * kScanItems;   // contiguous per thread
    int vals[kScanItems];
    int s = 0;
    for (int q = 0; q < kScanItems; ++q) {
        const int64_t idx = t0 + q;
        vals[q] = idx < n ? data[idx] : 0;
        s += vals[q];
    }
    int run = block_exclusive_scan(s, &tot) + sums[blockIdx.x];
    for (int q = 0; q < kScanItems; ++q) {
        const int64_t idx = t0 + q;
        if (idx < n) data[idx] = run;
        run += vals[q];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) data[n] = sums[nb];
}

cudaError_t exclusive_scan_impl(int32_t *data, int64_t n, int32_t *tmp, cudaStream_t st) {
    const int nb = (int)((n + kScanSeg - 1) / kScanSeg);
    if (nb == 0) {
        return cudaMemsetAsync(data, 0, sizeof(int32_t), st);
    }
    k_scan_reduce<<<nb, kScanThreads, 0, st>>>(data, n, tmp);
    k_scan_top<<<1, kScanThreads, 0, st>>>(tmp, nb);
    k_scan_apply<<<nb, kScanThreads, 0, st>>>(data, n, tmp, nb);
    return cudaGetLastError();
}

// ---- work list ----------------------------------------------------------------

__global__ void k_tile_ranges(const int32_t *__restrict__ bin_end, int ntiles, int chunk,
                              int32_t *tile_items, int2 *tile_range) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const int s = (t == 0) ? 0 : bin_end[t - 1];
    const int e = bin_end[t];
    tile_range[t] = make_int2(s, e);
    tile_items[t] = (e - s + chunk - 1) / chunk;
}

__global__ void k_fill_items(int ntiles, int chunk, const int32_t *__restrict__ item_off,
                             const int2 *__restrict__ tile_range, int4 *items, Ctrl *ctrl,
                             int flip) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        ctrl->n_items = item_off[ntiles];
        if (flip) ctrl->cur = 1 - ctrl->cur;    // particles now live in the other set
    }
    if (t >= ntiles) return;
    const int2 r = tile_range[t];
    int o = item_off[t];
    for (int s = r.x; s < r.y; s += chunk) {
        items[o++] = make_int4(t, s, min(r.y, s + chunk), 0);
    }
}

__global__ void k_flip(Ctrl *ctrl) { ctrl->cur = 1 - ctrl->cur; }

}  // namespace

cudaError_t exclusive_scan(int32_t *data, int64_t n, int32_t *tmp, cudaStream_t st) {
    return exclusive_scan_impl(data, n, tmp, st);
}

// per-tile ranges from the bin ends left by a scatter, then the work items
cudaError_t launch_worklist(const int32_t *bin_end, int ntiles, int chunk, int32_t *tile_items,
                            int2 *tile_range, int4 *items, int32_t *scan_tmp, Ctrl *ctrl, int flip,
                            cudaStream_t st) {
    const int T = 256;
    const int tb = (ntiles + T - 1) / T;
    k_tile_ranges<<<tb, T, 0, st>>>(bin_end, ntiles, chunk, tile_items, tile_range);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = exclusive_scan_impl(tile_items, ntiles, scan_tmp, st)) != cudaSuccess) return e;
    k_fill_items<<<tb, T, 0, st>>>(ntiles, chunk, tile_items, tile_range, items, ctrl, flip);
    return cudaGetLastError();
}

// One-time set-up outside any stream capture: the staged scatter's shared memory.
cudaError_t sort_prepare() {
    return cudaFuncSetAttribute(k_scatter_staged, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kStageSmem);
}

// histogram, scan and staged scatter by tile key >> shift (nb keys)
cudaError_t sort_pass(int64_t n, const Geom &g, int shift, int64_t nb, Ctrl *ctrl, int32_t *bins,
                      int32_t *scan_tmp, cudaStream_t st, SortRange rg = SortRange{0, 0}) {
    cudaError_t e = cudaMemsetAsync(bins, 0, sizeof(int32_t) * (size_t)(nb + 1), st);
    if (e != cudaSuccess) return e;
    const int T = 256;
    if (n > 0) {
        const int hblocks = (int)std::min<int64_t>((n + kHistStage - 1) / kHistStage, 152 * 8);
        k_histogram_staged<<<hblocks, T, 0, st>>>(n, g, ctrl, bins, shift, rg);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = exclusive_scan_impl(bins, nb, scan_tmp, st)) != cudaSuccess) return e;
    if (n > 0) {
        // resident blocks per SM as the staging buffer allows (228 KB per SM)
        const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(8, (228 * 1024) / (kStageSmem + 1024)));
        const int sblocks = (int)std::min<int64_t>((n + kStage - 1) / kStage, 152 * per_sm);
        k_scatter_staged<<<sblocks, T, kStageSmem, st>>>(n, g, ctrl, bins, shift, rg);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Shifts of the coarse passes that precede the full-key pass for particles in
// arbitrary order.  Each pass sorts by the next kDigit bits of the tile key
// (most significant first): a 512-particle slice of pass p spans one or two
// buckets of pass p - 1, so it meets at most 2^(kDigit + 1) distinct keys
// (never overflowing the staged table) and writes runs of ~512 / 2^kDigit
// consecutive particles per key.
#ifndef PIC_PRESORT_DIGIT
#define PIC_PRESORT_DIGIT 4
#endif
constexpr int kDigit = PIC_PRESORT_DIGIT;
static_assert(kDigit >= 1 && (2 << kDigit) <= kHash, "presort digit too wide for the table");

int coarse_shifts(int ntiles, int *shifts) {
    int bits = 0;
    while ((1 << bits) < ntiles) ++bits;
    int k = 0;
    for (int sft = bits - kDigit; sft > 0; sft -= kDigit) shifts[k++] = sft;
    return k;
}

int sort_launches(int64_t n, int ntiles, bool presort) {
    int sh[32];
    const int passes = (presort && n > 0) ? coarse_shifts(ntiles, sh) : 0;
    // per coarse pass: histogram, 3 scan, scatter, flip; then the full-key pass
    // (histogram, 3 scan, scatter) and the work list (ranges, 3 scan, fill)
    return passes * 6 + (n > 0 ? 10 : 8);
}

cudaError_t launch_sort(int64_t n, const Geom &g, int chunk, Ctrl *ctrl, int32_t *bins,
                        int64_t nbins, int32_t *scan_tmp, int32_t *tile_items,
                        int2 *tile_range, int4 *items, bool presort, cudaStream_t st) {
    cudaError_t e;
    if (presort && n > 0) {
        const int nt = g.ntile[0] * g.ntile[1] * g.ntile[2];
        int sh[32];
        const int passes = coarse_shifts(nt, sh);
        for (int p = 0; p < passes; ++p) {
            if ((e = sort_pass(n, g, sh[p], ((nt - 1) >> sh[p]) + 1, ctrl, bins, scan_tmp, st)))
                return e;
            k_flip<<<1, 1, 0, st>>>(ctrl);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    if ((e = sort_pass(n, g, 0, nbins, ctrl, bins, scan_tmp, st)) != cudaSuccess) return e;
    const int T = 256;
    const int ntiles = g.ntile[0] * g.ntile[1] * g.ntile[2];
    const int tb = (ntiles + T - 1) / T;
    k_tile_ranges<<<tb, T, 0, st>>>(bins, ntiles, chunk, tile_items, tile_range);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = exclusive_scan_impl(tile_items, ntiles, scan_tmp, st)) != cudaSuccess) return e;
    k_fill_items<<<tb, T, 0, st>>>(ntiles, chunk, tile_items, tile_range, items, ctrl,
                                   n > 0 ? 1 : 0);
    return cudaGetLastError();
}

// Coarse passes and the full-key pass over particles [o, o + n) alone, set
// to set (starting in the current set, which no kernel here changes); the
// range ends in set cur ^ (*passes & 1).  Used while later ranges are still
// being loaded; o must be a multiple of 4 (bulk copies start on 16 bytes).
cudaError_t launch_sort_range(int64_t n, int64_t o, const Geom &g, Ctrl *ctrl, int32_t *bins,
                              int64_t nbins, int32_t *scan_tmp, int *passes, int *kernels,
                              cudaStream_t st) {
    *passes = 0;
    *kernels = 0;
    if (n <= 0) return cudaSuccess;
    if (o % 4 != 0) return cudaErrorInvalidValue;
    const int nt = g.ntile[0] * g.ntile[1] * g.ntile[2];
    int sh[33];
    const int k = coarse_shifts(nt, sh);
    sh[k] = 0;
    cudaError_t e;
    for (int p = 0; p <= k; ++p) {
        const int64_t nb = p < k ? ((nt - 1) >> sh[p]) + 1 : nbins;
        if ((e = sort_pass(n, g, sh[p], nb, ctrl, bins, scan_tmp, st, SortRange{o, p & 1})))
            return e;
        *kernels += 5;
    }
    *passes = k + 1;
    return cudaSuccess;
}

cudaError_t launch_flip(Ctrl *ctrl, cudaStream_t st) {
    k_flip<<<1, 1, 0, st>>>(ctrl);
    return cudaGetLastError();
}

}  // namespace pic
