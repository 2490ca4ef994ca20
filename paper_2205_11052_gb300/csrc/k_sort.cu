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
#include "sort_staged.cuh"

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

// the single run's binning key: the deposit tile, optionally coarsened
struct TileKey {
    Geom g;
    int shift;
    __device__ __forceinline__ int operator()(int32_t c, int64_t, int &bad) const {
        return tile_key(c, g, bad) >> shift;
    }
};

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

__global__ void k_scan_reduce(const int32_t *__restrict__ data, int64_t n, int32_t *sums,
                              const int32_t *gate) {
    if (gate && !*gate) return;
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
__global__ void k_scan_top(int32_t *sums, int nb, const int32_t *gate) {
    if (gate && !*gate) return;
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

__global__ void k_scan_apply(int32_t *data, int64_t n, const int32_t *sums, int nb,
                             const int32_t *gate) {
    if (gate && !*gate) return;
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

cudaError_t exclusive_scan_impl(int32_t *data, int64_t n, int32_t *tmp, cudaStream_t st,
                                const int32_t *gate = nullptr) {
    const int nb = (int)((n + kScanSeg - 1) / kScanSeg);
    if (nb == 0) {
        return cudaMemsetAsync(data, 0, sizeof(int32_t), st);
    }
    k_scan_reduce<<<nb, kScanThreads, 0, st>>>(data, n, tmp, gate);
    k_scan_top<<<1, kScanThreads, 0, st>>>(tmp, nb, gate);
    k_scan_apply<<<nb, kScanThreads, 0, st>>>(data, n, tmp, nb, gate);
    return cudaGetLastError();
}

// ---- work list ----------------------------------------------------------------

__global__ void k_tile_ranges(const int32_t *__restrict__ bin_end, int ntiles, int chunk,
                              int32_t *tile_items, int2 *tile_range, const int32_t *gate) {
    if (gate && !*gate) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const int s = (t == 0) ? 0 : bin_end[t - 1];
    const int e = bin_end[t];
    tile_range[t] = make_int2(s, e);
    tile_items[t] = (e - s + chunk - 1) / chunk;
}

__global__ void k_fill_items(int ntiles, int chunk, const int32_t *__restrict__ item_off,
                             const int2 *__restrict__ tile_range, int4 *items, Ctrl *ctrl,
                             int flip, const int32_t *gate) {
    if (gate && !*gate) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        ctrl->n_items = item_off[ntiles];
        if (flip) ctrl->cur = 1 - ctrl->cur;    // particles now live in the other set
        // a re-binning: every particle is back inside its tile
        ctrl->rebins += 1;
        ctrl->since_sort = 0;
        ctrl->stray_step = 0ull;
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

cudaError_t exclusive_scan(int32_t *data, int64_t n, int32_t *tmp, cudaStream_t st,
                           const int32_t *gate) {
    return exclusive_scan_impl(data, n, tmp, st, gate);
}

namespace {
__global__ void k_rebin_decide(Ctrl *ctrl, long long max_strays, int period) {
    const bool due = (period > 0 && ctrl->since_sort >= period) ||
                     ctrl->stray_step > (unsigned long long)max_strays;
    ctrl->rebin = due ? 1 : 0;
    ctrl->stray_step = 0ull;
}
}  // namespace

cudaError_t launch_rebin_decide(Ctrl *ctrl, long long max_strays, int period, cudaStream_t st) {
    k_rebin_decide<<<1, 1, 0, st>>>(ctrl, max_strays < 0 ? 0 : max_strays, period);
    return cudaGetLastError();
}

// per-tile ranges from the bin ends left by a scatter, then the work items
cudaError_t launch_worklist(const int32_t *bin_end, int ntiles, int chunk, int32_t *tile_items,
                            int2 *tile_range, int4 *items, int32_t *scan_tmp, Ctrl *ctrl, int flip,
                            cudaStream_t st) {
    const int T = 256;
    const int tb = (ntiles + T - 1) / T;
    k_tile_ranges<<<tb, T, 0, st>>>(bin_end, ntiles, chunk, tile_items, tile_range, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = exclusive_scan_impl(tile_items, ntiles, scan_tmp, st)) != cudaSuccess) return e;
    k_fill_items<<<tb, T, 0, st>>>(ntiles, chunk, tile_items, tile_range, items, ctrl, flip,
                                   nullptr);
    return cudaGetLastError();
}

// One-time set-up outside any stream capture: the staged scatter's shared memory.
cudaError_t sort_prepare() {
    return staged_prepare<TileKey>();
}

// histogram, scan and staged scatter by tile key >> shift (nb keys)
cudaError_t sort_pass(int64_t n, const Geom &g, int shift, int64_t nb, Ctrl *ctrl, int32_t *bins,
                      int32_t *scan_tmp, cudaStream_t st, SortRange rg = SortRange{0, 0},
                      const int32_t *gate = nullptr) {
    return staged_pass(n, TileKey{g, shift}, nb, ctrl, bins, scan_tmp, st, rg, gate);
}

// Shifts of the coarse passes that precede the full-key pass for particles in
// arbitrary order.  Each pass sorts by the next kDigit bits of the tile key
// (most significant first): while the buckets of pass p - 1 hold at least a
// slice (kStage particles) each, a slice of pass p spans one or two of them,
// so it meets at most 2^(kDigit + 1) distinct keys (not overflowing the staged
// table) and writes runs of ~kStage / 2^kDigit consecutive particles per key;
// a slice that meets more keys takes the scatter's per-warp fallback.
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
                        int2 *tile_range, int4 *items, bool presort, cudaStream_t st,
                        const int32_t *gate) {
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
    if ((e = sort_pass(n, g, 0, nbins, ctrl, bins, scan_tmp, st, SortRange{0, 0}, gate)) !=
        cudaSuccess)
        return e;
    const int T = 256;
    const int ntiles = g.ntile[0] * g.ntile[1] * g.ntile[2];
    const int tb = (ntiles + T - 1) / T;
    k_tile_ranges<<<tb, T, 0, st>>>(bins, ntiles, chunk, tile_items, tile_range, gate);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = exclusive_scan_impl(tile_items, ntiles, scan_tmp, st, gate)) != cudaSuccess) return e;
    k_fill_items<<<tb, T, 0, st>>>(ntiles, chunk, tile_items, tile_range, items, ctrl,
                                   n > 0 ? 1 : 0, gate);
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

namespace {
// The failure path of the bounded waits, on purpose and without a fault: an
// mbarrier that no thread arrives on and no copy completes is waited for with
// the same bounded wait the staged kernels use; the wait gives up after its
// poll limit, the kernel raises PIC_FLAG_TIMEOUT and returns.  Nothing is in
// flight, so the block can leave at once.
__global__ void k_timeout_selftest(Ctrl *ctrl) {
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    mbar_fence_init();
    if (!mbar_wait(&bar, 0u)) atomicOr(&ctrl->flags, PIC_FLAG_TIMEOUT);
}
}  // namespace

cudaError_t launch_timeout_selftest(Ctrl *ctrl, cudaStream_t st) {
    k_timeout_selftest<<<1, 32, 0, st>>>(ctrl);
    return cudaGetLastError();
}

cudaError_t launch_flip(Ctrl *ctrl, cudaStream_t st) {
    k_flip<<<1, 1, 0, st>>>(ctrl);
    return cudaGetLastError();
}

}  // namespace pic
