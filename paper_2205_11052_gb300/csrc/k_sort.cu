// Periodic binning: counting sort of the particle store by tile-major cell
// index, followed by the deposit work list (tile, particle range) build.
//
// The paper has no sort (its nearest step is the particle-to-rank search of
// Section 5.2.1); binning keeps particles grouped by deposit tile and ordered
// by cell within a tile, so the deposit can accumulate each tile in shared
// memory and aggregate equal cells within a warp.
//
// Key of a particle with stencil base (i, j, k), tile T = (Tx, Ty, Tz):
//   tile id = ti + ntx (tj + nty tk),   (ti, tj, tk) = (i/Tx, j/Ty, k/Tz)
//   key     = tile id * Tx Ty Tz + li + Tx (lj + Ty lk),  (li, ...) = (i mod Tx, ...)
// Passes: histogram (warp-aggregated atomics) -> exclusive scan (in place) ->
// scatter (the scanned offsets serve as cursors; afterwards bins[key] holds
// the end of bin key) -> per-tile ranges -> scan of items per tile -> items.
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
    const int ti = i / g.tile[0], tj = j / g.tile[1], tk = k / g.tile[2];
    const int li = i - ti * g.tile[0], lj = j - tj * g.tile[1], lk = k - tk * g.tile[2];
    const int tid = ti + g.ntile[0] * (tj + g.ntile[1] * tk);
    return tid * g.tvol + li + g.tile[0] * (lj + g.tile[1] * lk);
}

// atomicAdd(&base[key], 1) for every active lane, aggregated over lanes that
// share a key; returns each lane's old value plus its rank among those lanes.
__device__ __forceinline__ int warp_agg_increment(int32_t *base, int key, unsigned active) {
    const int lane = threadIdx.x & 31;
    const unsigned peers = __match_any_sync(active, key);
    const int leader = __ffs(peers) - 1;
    const int rank = __popc(peers & ((1u << lane) - 1u));
    int old = 0;
    if (lane == leader) old = atomicAdd(base + key, __popc(peers));
    old = __shfl_sync(peers, old, leader);
    return old + rank;
}

__global__ void k_histogram(int64_t n, Geom g, Ctrl *ctrl, int32_t *bins) {
    const ParticleSet ps = ctrl->sets[ctrl->cur];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int bad = 0;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t p = base + threadIdx.x;
        const bool act = p < n;
        const unsigned active = __ballot_sync(0xffffffffu, act);
        if (act) {
            const int key = tile_key(ps.cell[p], g, bad);
            warp_agg_increment(bins, key, active);
        }
    }
    if (bad) atomicOr(&ctrl->flags, PIC_FLAG_BAD_CELL);
}

__global__ void k_scatter(int64_t n, Geom g, Ctrl *ctrl, int32_t *bins) {
    const int cur = ctrl->cur;
    const ParticleSet src = ctrl->sets[cur];
    const ParticleSet dst = ctrl->sets[1 - cur];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t p = base + threadIdx.x;
        const bool act = p < n;
        const unsigned active = __ballot_sync(0xffffffffu, act);
        if (act) {
            const int32_t c = src.cell[p];
            int bad = 0;
            const int key = tile_key(c, g, bad);
            const int q = warp_agg_increment(bins, key, active);
            dst.cell[q] = c;
            dst.o[0][q] = src.o[0][p];
            dst.o[1][q] = src.o[1][p];
            dst.o[2][q] = src.o[2][p];
            dst.v[0][q] = src.v[0][p];
            dst.v[1][q] = src.v[1][p];
            dst.v[2][q] = src.v[2][p];
            dst.pid[q] = src.pid[p];
        }
    }
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

cudaError_t exclusive_scan(int32_t *data, int64_t n, int32_t *tmp, cudaStream_t st) {
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

__global__ void k_tile_ranges(const int32_t *__restrict__ bin_end, int ntiles, int tvol,
                              int chunk, int32_t *tile_items, int2 *tile_range) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const int s = (t == 0) ? 0 : bin_end[(int64_t)t * tvol - 1];
    const int e = bin_end[(int64_t)(t + 1) * tvol - 1];
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

}  // namespace

cudaError_t launch_sort(int64_t n, const Geom &g, int chunk, Ctrl *ctrl, int32_t *bins,
                        int64_t nbins, int32_t *scan_tmp, int32_t *tile_items,
                        int2 *tile_range, int4 *items, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(bins, 0, sizeof(int32_t) * (size_t)(nbins + 1), st);
    if (e != cudaSuccess) return e;
    const int T = 256;
    const int blocks = (int)std::min<int64_t>((n + T - 1) / T, 152 * 16);
    if (n > 0) {
        k_histogram<<<blocks, T, 0, st>>>(n, g, ctrl, bins);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = exclusive_scan(bins, nbins, scan_tmp, st)) != cudaSuccess) return e;
    if (n > 0) {
        k_scatter<<<blocks, T, 0, st>>>(n, g, ctrl, bins);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int ntiles = g.ntile[0] * g.ntile[1] * g.ntile[2];
    const int tb = (ntiles + T - 1) / T;
    k_tile_ranges<<<tb, T, 0, st>>>(bins, ntiles, g.tvol, chunk, tile_items, tile_range);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = exclusive_scan(tile_items, ntiles, scan_tmp, st)) != cudaSuccess) return e;
    k_fill_items<<<tb, T, 0, st>>>(ntiles, chunk, tile_items, tile_range, items, ctrl,
                                   n > 0 ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace pic
