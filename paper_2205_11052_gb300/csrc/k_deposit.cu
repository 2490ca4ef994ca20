// Scatter (Section 3.1 step 1 of arXiv 2205.11052) with the cloud-in-cell
// shape on the cell-centred grid of Section 3.2:
//   rho_g = sum_p q_p W(x_g - x_p) / h^3,  W = prod_d (1 - |dx_d| / h_d)_+ .
// A particle with stencil base (i, j, k) and offsets (fx, fy, fz) adds
// q_p / h^3 * w_a(fx) w_b(fy) w_c(fz) to node (i + a, j + b, k + c), a, b, c
// in {0, 1}, with w_0(f) = 1 - f and w_1(f) = f (periodic wrap).
//
// Tiled kernel: one CTA per work item (a range of binned particles whose
// stencil base was inside one tile at the last sort).  The CTA accumulates
// unscaled weights in a shared-memory copy of the tile plus `guard` cells on
// each side (plus the +1 stencil layer), first summing lanes of a warp that
// share a cell (segmented shuffle reduction over the cell-ordered particles),
// and finally adds the tile to rho with one global atomic per touched node.
// Particles that drifted beyond the guard since the last sort go straight to
// rho with global atomics, so the result never depends on the sort cadence.
#include "pic_internal.cuh"

namespace pic {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ bool decode_cell(int32_t c, const Geom &g, int &i, int &j, int &k) {
    i = cell_i(c);
    j = cell_j(c);
    k = cell_k(c);
    if (i >= g.n[0] || j >= g.n[1] || k >= g.n[2]) {
        i = j = k = 0;
        return false;
    }
    return true;
}

// place axis index a (0 <= a < n) relative to tile origin o with guard G:
// returns the slot in [0, T + 2G) or -1 if farther than G cells away
__device__ __forceinline__ int tile_slot(int a, int o, int n, int T, int G) {
    int d = a - o;
    if (d < 0) d += n;
    if (d >= T + G) {
        d -= n;
        if (d < -G) return -1;
    }
    return d + G;
}

__device__ __forceinline__ void deposit_global(float *rho, const Geom &g, int i, int j, int k,
                                               const float w[8], float qscale) {
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int i1 = (i + 1 == nx) ? 0 : i + 1;
    const int j1 = (j + 1 == ny) ? 0 : j + 1;
    const int k1 = (k + 1 == nz) ? 0 : k + 1;
    const int64_t nxy = (int64_t)nx * ny;
    const int64_t r00 = (int64_t)j * nx + k * nxy, r10 = (int64_t)j1 * nx + k * nxy;
    const int64_t r01 = (int64_t)j * nx + k1 * nxy, r11 = (int64_t)j1 * nx + k1 * nxy;
    atomicAdd(rho + r00 + i, w[0] * qscale);
    atomicAdd(rho + r00 + i1, w[1] * qscale);
    atomicAdd(rho + r10 + i, w[2] * qscale);
    atomicAdd(rho + r10 + i1, w[3] * qscale);
    atomicAdd(rho + r01 + i, w[4] * qscale);
    atomicAdd(rho + r01 + i1, w[5] * qscale);
    atomicAdd(rho + r11 + i, w[6] * qscale);
    atomicAdd(rho + r11 + i1, w[7] * qscale);
}

__device__ __forceinline__ void cic_weights(float fx, float fy, float fz, float w[8]) {
    const float x0 = 1.0f - fx, y0 = 1.0f - fy, z0 = 1.0f - fz;
    const float a = y0 * z0, b = fy * z0, c = y0 * fz, d = fy * fz;
    w[0] = x0 * a; w[1] = fx * a;
    w[2] = x0 * b; w[3] = fx * b;
    w[4] = x0 * c; w[5] = fx * c;
    w[6] = x0 * d; w[7] = fx * d;
}

__global__ void __launch_bounds__(256) k_deposit_tiles(Geom g, const Ctrl *ctrl,
                                                        const int4 *__restrict__ items,
                                                        float qscale, float *rho, Ctrl *ctrl_w,
                                                        int sparse_below) {
    extern __shared__ float acc[];
    const ParticleSet ps = ctrl->sets[ctrl->cur];
    const int n_items = ctrl->n_items;
    const int G = g.guard;
    const int S0 = g.tile[0] + 2 * G + 1, S1 = g.tile[1] + 2 * G + 1, S2 = g.tile[2] + 2 * G + 1;
    const int S01 = S0 * S1, S = S01 * S2;
    const int lane = threadIdx.x & 31;
    unsigned long long strays = 0;
    int bad = 0;

    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int4 item = items[it];
        const int tile = item.x;
        const int tx = tile % g.ntile[0];
        const int ty = (tile / g.ntile[0]) % g.ntile[1];
        const int tz = tile / (g.ntile[0] * g.ntile[1]);
        const int ox = tx * g.tile[0], oy = ty * g.tile[1], oz = tz * g.tile[2];

        if (item.z - item.y < sparse_below) {
            // few particles: skip the shared tile, add straight to rho
            for (int p = item.y + threadIdx.x; p < item.z; p += blockDim.x) {
                int i, j, k;
                if (!decode_cell(ps.cell[p], g, i, j, k)) bad = 1;
                float w[8];
                cic_weights(ps.o[0][p], ps.o[1][p], ps.o[2][p], w);
                deposit_global(rho, g, i, j, k, w, qscale);
            }
            continue;
        }

        for (int s = threadIdx.x; s < S; s += blockDim.x) acc[s] = 0.0f;
        __syncthreads();

        for (int base = item.y; base < item.z; base += blockDim.x) {
            const int p = base + threadIdx.x;
            const bool valid = p < item.z;
            int i = 0, j = 0, k = 0, c = 0;
            float w[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            int slot = -1;
            if (valid) {
                c = ps.cell[p];
                if (!decode_cell(c, g, i, j, k)) bad = 1;
                cic_weights(ps.o[0][p], ps.o[1][p], ps.o[2][p], w);
                const int si = tile_slot(i, ox, g.n[0], g.tile[0], G);
                const int sj = tile_slot(j, oy, g.n[1], g.tile[1], G);
                const int sk = tile_slot(k, oz, g.n[2], g.tile[2], G);
                if (si >= 0 && sj >= 0 && sk >= 0) slot = si + S0 * sj + S01 * sk;
            }
            // segmented warp reduction over runs of equal slots (cell order)
            const int key = (slot >= 0) ? slot : -1 - lane;
            const int prev = __shfl_up_sync(kFull, key, 1);
            const bool head = (lane == 0) || (key != prev);
            const unsigned heads = __ballot_sync(kFull, head);
            if (heads != kFull) {
                const unsigned above = heads & ~((2u << lane) - 1u);   // heads after this lane
                const int end = above ? (__ffs(above) - 2) : 31;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float t = __shfl_down_sync(kFull, w[q], o);
                        if (lane + o <= end) w[q] += t;
                    }
                }
            }
            if (valid) {
                if (slot >= 0) {
                    if (head) {
                        atomicAdd(acc + slot, w[0]);
                        atomicAdd(acc + slot + 1, w[1]);
                        atomicAdd(acc + slot + S0, w[2]);
                        atomicAdd(acc + slot + S0 + 1, w[3]);
                        atomicAdd(acc + slot + S01, w[4]);
                        atomicAdd(acc + slot + S01 + 1, w[5]);
                        atomicAdd(acc + slot + S01 + S0, w[6]);
                        atomicAdd(acc + slot + S01 + S0 + 1, w[7]);
                    }
                } else {
                    ++strays;
                    deposit_global(rho, g, i, j, k, w, qscale);
                }
            }
        }
        __syncthreads();

        // flush: one global atomic per touched node of the tile + guard
        for (int s = threadIdx.x; s < S; s += blockDim.x) {
            const float val = acc[s];
            if (val != 0.0f) {
                const int a = s % S0, b = (s / S0) % S1, cc = s / S01;
                int gi = (ox - G + a) % g.n[0];
                int gj = (oy - G + b) % g.n[1];
                int gk = (oz - G + cc) % g.n[2];
                if (gi < 0) gi += g.n[0];
                if (gj < 0) gj += g.n[1];
                if (gk < 0) gk += g.n[2];
                atomicAdd(rho + gi + (int64_t)g.n[0] * (gj + (int64_t)g.n[1] * gk), val * qscale);
            }
        }
        __syncthreads();
    }
    if (bad) atomicOr(&ctrl_w->flags, PIC_FLAG_BAD_CELL);
    if (strays) atomicAdd(&ctrl_w->stray, strays);
}

// Reference-free fallback used before any binning exists and for tests:
// every particle adds its eight weights with global atomics.
__global__ void k_deposit_direct(int64_t n, Geom g, const Ctrl *ctrl, float qscale, float *rho,
                                 Ctrl *ctrl_w) {
    const ParticleSet ps = ctrl->sets[ctrl->cur];
    int bad = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        int i, j, k;
        if (!decode_cell(ps.cell[p], g, i, j, k)) bad = 1;
        float w[8];
        cic_weights(ps.o[0][p], ps.o[1][p], ps.o[2][p], w);
        deposit_global(rho, g, i, j, k, w, qscale);
    }
    if (bad) atomicOr(&ctrl_w->flags, PIC_FLAG_BAD_CELL);
}

}  // namespace

cudaError_t launch_deposit(int64_t n, const Geom &g, const Ctrl *ctrl, const int4 *items,
                           int max_items, float qscale, float *rho, Ctrl *ctrl_w,
                           int grid_blocks, int sparse_below, cudaStream_t st) {
    (void)n;
    const int S = (g.tile[0] + 2 * g.guard + 1) * (g.tile[1] + 2 * g.guard + 1) *
                  (g.tile[2] + 2 * g.guard + 1);
    const size_t smem = sizeof(float) * (size_t)S;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_deposit_tiles,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int blocks = grid_blocks < max_items ? grid_blocks : (max_items > 0 ? max_items : 1);
    k_deposit_tiles<<<blocks, 256, smem, st>>>(g, ctrl, items, qscale, rho, ctrl_w, sparse_below);
    return cudaGetLastError();
}

cudaError_t launch_deposit_direct(int64_t n, const Geom &g, const Ctrl *ctrl, float qscale,
                                  float *rho, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int T = 256;
    const int blocks = (int)((n + T - 1) / T < 152 * 16 ? (n + T - 1) / T : 152 * 16);
    k_deposit_direct<<<blocks, T, 0, st>>>(n, g, ctrl, qscale, rho, const_cast<Ctrl *>(ctrl));
    return cudaGetLastError();
}

}  // namespace pic
