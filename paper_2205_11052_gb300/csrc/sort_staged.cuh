// Staged counting-sort passes over the particle store: a histogram of bin
// keys and a scatter into the other particle set, both by slices of
// consecutive particles aggregated in a small shared hash table.  The key of
// a particle comes from a functor, key_of(cell, particle index, bad) (called
// for increasing particle indices within a thread), so the
// single-run binning (tile keys) and the batched one (global tile ids of each
// instance) share the kernels.
#pragma once

#include <algorithm>

#include "pic_internal.cuh"
#include "tma.cuh"

namespace pic {

namespace {

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
#define PIC_SORT_STAGE 1024
#endif
constexpr int kStage = PIC_SORT_STAGE;     // particles per staged slice
constexpr int kHash = 256;                 // slots of the per-slice tile table
constexpr int kPerThread = kStage / 256;   // the staged kernels run 256 threads per block
#ifndef PIC_HIST_STAGE
#define PIC_HIST_STAGE 4096
#endif
constexpr int kHistStage = PIC_HIST_STAGE;   // particles per histogram slice
constexpr int kHistPer = kHistStage / 256;

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
// eight arrays of its next slice arrive by bulk asynchronous copies (4 KB
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

template <class Key>
__global__ void __launch_bounds__(256) k_scatter_staged(int64_t n, Key key_param, Ctrl *ctrl,
                                                         int32_t *bins, SortRange rg,
                                                         const int32_t *gate) {
    if (gate && !*gate) return;
    Key key_of = key_param;   // a per-thread copy (functors may cache lookups)
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
            const int key = act ? key_of(sc[j], rg.o + s0 + j, bad) : -1 - lane;
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
                    const int key = key_of(sc[j], rg.o + s0 + j, bad);
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
template <class Key>
__global__ void __launch_bounds__(256) k_histogram_staged(int64_t n, Key key_param, Ctrl *ctrl,
                                                           int32_t *bins, SortRange rg,
                                                           const int32_t *gate) {
    if (gate && !*gate) return;
    Key key_of = key_param;   // a per-thread copy (functors may cache lookups)
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
            const int key = act ? key_of(cv[u], rg.o + s0 + j, bad) : -1 - lane;
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


// One pass by key_of over particles [rg.o, rg.o + n) of set cur ^ rg.rel
// into the same range of the other set; nb keys (bins holds nb + 1 ints).
template <class Key>
cudaError_t staged_pass(int64_t n, const Key &key_of, int64_t nb, Ctrl *ctrl, int32_t *bins,
                        int32_t *scan_tmp, cudaStream_t st, SortRange rg = SortRange{0, 0},
                        const int32_t *gate = nullptr) {
    cudaError_t e = cudaMemsetAsync(bins, 0, sizeof(int32_t) * (size_t)(nb + 1), st);
    if (e != cudaSuccess) return e;
    const int T = 256;
    if (n > 0) {
        const int hblocks = (int)std::min<int64_t>((n + kHistStage - 1) / kHistStage, 152 * 8);
        k_histogram_staged<Key><<<hblocks, T, 0, st>>>(n, key_of, ctrl, bins, rg, gate);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = exclusive_scan(bins, nb, scan_tmp, st, gate)) != cudaSuccess) return e;
    if (n > 0) {
        // resident blocks per SM as the staging buffer allows (228 KB per SM)
        const int per_sm =
            (int)std::max<size_t>(1, std::min<size_t>(8, (228 * 1024) / (kStageSmem + 1024)));
        const int sblocks = (int)std::min<int64_t>((n + kStage - 1) / kStage, 152 * per_sm);
        k_scatter_staged<Key><<<sblocks, T, kStageSmem, st>>>(n, key_of, ctrl, bins, rg, gate);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// the scatter's shared memory (above the default 48 KB); once per device,
// outside any stream capture
template <class Key>
cudaError_t staged_prepare() {
    return cudaFuncSetAttribute(k_scatter_staged<Key>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kStageSmem);
}

}  // namespace

}  // namespace pic
