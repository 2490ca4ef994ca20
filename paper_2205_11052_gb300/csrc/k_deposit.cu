// Scatter (Section 3.1 step 1 of arXiv 2205.11052) with the cloud-in-cell
// shape on the cell-centred grid of Section 3.2:
//   rho_g = sum_p q_p W(x_g - x_p) / h^3,  W = prod_d (1 - |dx_d| / h_d)_+ .
// A particle with stencil base (i, j, k) and offsets (fx, fy, fz) adds
// q_p / h^3 * w_a(fx) w_b(fy) w_c(fz) to node (i + a, j + b, k + c), a, b, c
// in {0, 1}, with w_0(f) = 1 - f and w_1(f) = f (periodic wrap).
//
// Tiled kernel: each CTA takes a contiguous run of work items (ranges of
// binned particles whose stencil base was inside one tile at the last sort;
// consecutive items share tiles) and accumulates the unscaled weights in a
// shared-memory copy of the tile plus `guard` cells on each side (plus the +1
// stencil layer).  After each item the tile is folded into per-tile sums
// that go to the grid with one global atomic per touched node when the run
// moves to another tile.  Particles that drifted beyond the guard since the
// last sort go straight to the grid with global atomics, so the result never
// depends on the sort cadence.  Each thread loads its next particle before
// depositing the current one.
//
// Two accumulators:
//  * FP32: float shared tile, float global atomics into rho.
//  * fixed point: the particle's 2^20 units split over its eight corners by
//    nested rounding (cic::fixed_split: they sum exactly to 2^20, none is
//    negative), u32 shared atomics (at most 4095 particles per work item, so
//    a slot cannot reach 2^32) and u64
//    global atomics into an integer grid that k_rho_finish scales into rho.
//    Integer addition is associative, so this deposit is deterministic and
//    conserves the particles' total weight exactly.
#include <algorithm>

#include "cic.cuh"

namespace pic {

namespace {

using namespace cic;

// B > 0: every tile box is B slots long on each axis (cic::box_row)
template <bool FIXED, int B>
__global__ void __launch_bounds__(256, PIC_DEP_MIN_BLOCKS) k_deposit_tiles(Geom g, const Ctrl *__restrict__ ctrl,
                                                           const int4 *__restrict__ items,
                                                           float qscale, float *rho,
                                                           unsigned long long *rho64, Ctrl *ctrl_w,
                                                           int sparse_below) {
    extern __shared__ __align__(16) uint32_t acc[];
    const ParticleSet ps = ctrl->sets[ctrl->cur];
    const int n_items = ctrl->n_items;
    unsigned long long strays = 0;
    int bad = 0;
    int it0, it1;
    item_run(items, n_items, it0, it1);
    const int S = tile_of(g, 0).S;
    void *sum = reinterpret_cast<char *>(acc) + sum_offset(S);
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        acc[s] = 0u;
        if (FIXED) reinterpret_cast<unsigned long long *>(sum)[s] = 0ull;
        else reinterpret_cast<float *>(sum)[s] = 0.0f;
    }
    __syncthreads();
    // t: the tile of the dense items (sparse items go straight to the grid)
    int cur_tile = -1;
    Tile t = tile_of(g, 0);
    for (int it = it0; it < it1; ++it) {
        const int4 item = items[it];
        if (item.z - item.y < sparse_below) {
            // few particles: skip the shared tile, add straight to the grid
            for (int p = item.y + threadIdx.x; p < item.z; p += blockDim.x) {
                int i, j, k;
                if (!decode_cell(ps.cell[p], g, i, j, k)) bad = 1;
                const float fx = ps.o[0][p], fy = ps.o[1][p], fz = ps.o[2][p];
                float w[8];
                weights(fx, fy, fz, w);
                deposit_global<FIXED>(rho, rho64, g, i, j, k, w, fx, fy, fz, qscale);
            }
            continue;
        }
        if (item.x != cur_tile) {
            if (cur_tile >= 0) tile_flush_sum<FIXED>(sum, t, g, rho, rho64, qscale);
            cur_tile = item.x;
            t = tile_of(g, item.x);
        }
        int p = item.y + threadIdx.x;
        int32_t nc = 0;
        float nfx = 0.f, nfy = 0.f, nfz = 0.f;
        if (p < item.z) {
            nc = __ldcs(ps.cell + p);
            nfx = __ldcs(ps.o[0] + p);
            nfy = __ldcs(ps.o[1] + p);
            nfz = __ldcs(ps.o[2] + p);
        }
        for (; p < item.z; p += blockDim.x) {
            const int32_t c = nc;
            const float fx = nfx, fy = nfy, fz = nfz;
            const int pn = p + (int)blockDim.x;
            if (pn < item.z) {
                nc = __ldcs(ps.cell + pn);
                nfx = __ldcs(ps.o[0] + pn);
                nfy = __ldcs(ps.o[1] + pn);
                nfz = __ldcs(ps.o[2] + pn);
            }
            int i, j, k;
            if (!decode_cell(c, g, i, j, k)) bad = 1;
            if (!tile_add<FIXED, B>(acc, t, g, i, j, k, fx, fy, fz, rho, rho64, qscale)) ++strays;
        }
        __syncthreads();
        tile_fold<FIXED>(acc, sum, S);
        __syncthreads();
    }
    if (cur_tile >= 0) tile_flush_sum<FIXED>(sum, t, g, rho, rho64, qscale);
    if (bad) atomicOr(&ctrl_w->flags, PIC_FLAG_BAD_CELL);
    if (strays) atomicAdd(&ctrl_w->stray, strays);
}

// integer grid -> charge density, and clear the integer grid for next time;
// two nodes per thread and iteration (16-byte loads and stores of the 8-byte
// words, 8-byte stores of the densities), the odd last node by thread 0
__global__ void __launch_bounds__(256) k_rho_finish(int64_t ng, unsigned long long *__restrict__ rho64,
                                                    float *__restrict__ rho, double scale) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n2 = ng >> 1;
    ulonglong2 *r2 = reinterpret_cast<ulonglong2 *>(rho64);
    float2 *f2 = reinterpret_cast<float2 *>(rho);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n2; q += stride) {
        const ulonglong2 v = __ldcs(r2 + q);
        __stcs(f2 + q, make_float2((float)((double)(long long)v.x * scale),
                                   (float)((double)(long long)v.y * scale)));
        __stcs(r2 + q, make_ulonglong2(0ull, 0ull));
    }
    if ((ng & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        const long long v = (long long)rho64[ng - 1];
        rho[ng - 1] = (float)((double)v * scale);
        rho64[ng - 1] = 0ull;
    }
}

}  // namespace

cudaError_t launch_rho_finish(const Geom &g, unsigned long long *rho64, float *rho, double qscale,
                              cudaStream_t st) {
    const int64_t ng = (int64_t)g.n[0] * g.n[1] * g.n[2];
    const int fb = (int)std::max<int64_t>(1, std::min<int64_t>((ng / 2 + 255) / 256, 152 * 8));
    k_rho_finish<<<fb, 256, 0, st>>>(ng, rho64, rho, qscale / (double)kFixOne);
    return cudaGetLastError();
}

cudaError_t launch_deposit(int64_t n, const Geom &g, const Ctrl *ctrl, const int4 *items,
                           int max_items, double qscale_d, float *rho, unsigned long long *rho64,
                           bool fixed, Ctrl *ctrl_w, int grid_blocks, int sparse_below,
                           cudaStream_t st) {
    (void)n;
    const float qscale = (float)qscale_d;
    const size_t smem = tile_deposit_smem(g);   // item tile + the block's tile sums
    const int blocks = grid_blocks < max_items ? grid_blocks : (max_items > 0 ? max_items : 1);
    cudaError_t e;
    // the default geometry (8^3 tiles, two guard layers) as a constant box
    bool cbox = true;
    for (int d = 0; d < 3; ++d) cbox = cbox && g.tile[d] + 2 * g.guard + 1 == 13;
#define PIC_DT(F, B)                                                                           \
    do {                                                                                       \
        if (smem > 48 * 1024 &&                                                                \
            (e = cudaFuncSetAttribute(k_deposit_tiles<F, B>,                                   \
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,             \
                                      (int)smem)) != cudaSuccess)                              \
            return e;                                                                          \
        k_deposit_tiles<F, B><<<blocks, 256, smem, st>>>(g, ctrl, items, qscale, rho, rho64,   \
                                                         ctrl_w, sparse_below);                \
    } while (0)
    if (fixed) {
        if (cbox) PIC_DT(true, 13);
        else PIC_DT(true, 0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        return launch_rho_finish(g, rho64, rho, qscale_d, st);
    }
    PIC_DT(false, 0);
#undef PIC_DT
    return cudaGetLastError();
}

}  // namespace pic
