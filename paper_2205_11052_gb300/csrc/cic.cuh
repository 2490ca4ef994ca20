// Device helpers of the cloud-in-cell shape on the cell-centred grid
// (Section 3.2 of arXiv 2205.11052), shared by the deposit, the fused
// push + deposit and the adjoint kernels.
//
// A particle with stencil base (i, j, k) and offsets (fx, fy, fz) in [0, 1)
// has weight w_a(fx) w_b(fy) w_c(fz) on node (i + a, j + b, k + c), a, b, c in
// {0, 1}, with w_0(f) = 1 - f and w_1(f) = f; corners are numbered
// a | b << 1 | c << 2.
#pragma once

#include "pic_internal.cuh"

namespace pic {
namespace cic {

constexpr float kFixScale = 1048576.0f;   // 2^20: fixed-point unit of a weight
constexpr uint32_t kFixOne = 1u << 20;

__device__ __forceinline__ bool decode_cell(int32_t c, const Geom &g, int &i, int &j, int &k) {
    i = cell_i(c);
    j = cell_j(c);
    k = cell_k(c);
    if (i >= g.n[0] || j >= g.n[1] || k >= g.n[2]) {   // never produced by the kernels
        i = j = k = 0;
        return false;
    }
    return true;
}

// place axis index a (0 <= a < n) relative to tile origin o with guard G:
// the slot in [0, T + 2G), or -1 if farther than G cells from the tile
__device__ __forceinline__ int tile_slot(int a, int o, int n, int T, int G) {
    int d = a - o;
    if (d < 0) d += n;
    if (d >= T + G) {
        d -= n;
        if (d < -G) return -1;
    }
    return d + G;
}

__device__ __forceinline__ void weights(float fx, float fy, float fz, float w[8]) {
    const float x0 = 1.0f - fx, y0 = 1.0f - fy, z0 = 1.0f - fz;
    const float a = y0 * z0, b = fy * z0, c = y0 * fz, d = fy * fz;
    w[0] = x0 * a; w[1] = fx * a;
    w[2] = x0 * b; w[3] = fx * b;
    w[4] = x0 * c; w[5] = fx * c;
    w[6] = x0 * d; w[7] = fx * d;
}

// Fixed-point CIC weights by nested splitting: the particle's 2^20 units are
// split between the two x corners, each x share between its two y corners
// and each of those between its two z corners.  A split rounds the upper
// share X f to the nearest integer and gives the lower corner the rest, so
// the eight integers sum to exactly 2^20, none is negative, and each lies
// within 1.5 units of 2^20 times the exact weight.  The rounding is FP32's
// own: X f + 2^23 (one fused multiply-add, X f < 2^23) rounds to an integer
// held in the mantissa bits, and subtracting 2^23 back is exact.
__device__ __forceinline__ void fixed_split(float fx, float fy, float fz, uint32_t q[8]) {
    constexpr float kMagic = 8388608.0f;         // 2^23
    constexpr uint32_t kMagicBits = 0x4B000000u;  // its bit pattern
    const float r = fmaf(kFixScale, fx, kMagic);
    const uint32_t x1 = __float_as_uint(r) - kMagicBits;
    const float x1f = r - kMagic;
    const uint32_t xi[2] = {kFixOne - x1, x1};
    const float xf[2] = {kFixScale - x1f, x1f};
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const float ry = fmaf(xf[a], fy, kMagic);
        const uint32_t y1 = __float_as_uint(ry) - kMagicBits;
        const float y1f = ry - kMagic;
        const uint32_t yi[2] = {xi[a] - y1, y1};
        const float yf[2] = {xf[a] - y1f, y1f};
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const uint32_t z1 = __float_as_uint(fmaf(yf[b], fz, kMagic)) - kMagicBits;
            q[a | b << 1 | 4] = z1;
            q[a | b << 1] = yi[b] - z1;
        }
    }
}

// the eight stencil node indices (periodic)
__device__ __forceinline__ void nodes(const Geom &g, int i, int j, int k, int64_t nd[8]) {
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int i1 = (i + 1 == nx) ? 0 : i + 1;
    const int j1 = (j + 1 == ny) ? 0 : j + 1;
    const int k1 = (k + 1 == nz) ? 0 : k + 1;
    const int64_t nxy = (int64_t)nx * ny;
    const int64_t r00 = (int64_t)j * nx + k * nxy, r10 = (int64_t)j1 * nx + k * nxy;
    const int64_t r01 = (int64_t)j * nx + k1 * nxy, r11 = (int64_t)j1 * nx + k1 * nxy;
    nd[0] = r00 + i; nd[1] = r00 + i1; nd[2] = r10 + i; nd[3] = r10 + i1;
    nd[4] = r01 + i; nd[5] = r01 + i1; nd[6] = r11 + i; nd[7] = r11 + i1;
}

// add one particle's weights straight to the grid (global atomics)
template <bool FIXED>
__device__ __forceinline__ void deposit_global(float *rho, unsigned long long *rho64, const Geom &g,
                                               int i, int j, int k, const float w[8], float fx,
                                               float fy, float fz, float qscale) {
    int64_t nd[8];
    nodes(g, i, j, k, nd);
    if (FIXED) {
        uint32_t q[8];
        fixed_split(fx, fy, fz, q);
#pragma unroll
        for (int c = 0; c < 8; ++c) atomicAdd(rho64 + nd[c], (unsigned long long)q[c]);
    } else {
#pragma unroll
        for (int c = 0; c < 8; ++c) atomicAdd(rho + nd[c], w[c] * qscale);
    }
}

// Shared-memory tile of one work item: (T + 1 + 2G)^3 slots around tile
// origin o; add one particle (or send it to the grid if it left the guard).
struct Tile {
    int ox, oy, oz, S0, S01, S;
    unsigned m0, m01;   // ceil(2^32 / S0), ceil(2^32 / S01): slot -> (a, b, c) by multiply-high
};

// slot s -> its (a, b, c) position in the tile box; exact for s * S01 < 2^32
__host__ __device__ __forceinline__ unsigned mulhi32(unsigned a, unsigned m) {
#ifdef __CUDA_ARCH__
    return __umulhi(a, m);
#else
    return (unsigned)(((unsigned long long)a * m) >> 32);
#endif
}

__host__ __device__ __forceinline__ void tile_pos(const Tile &t, int s, int &a, int &b, int &c) {
    c = (int)mulhi32((unsigned)s, t.m01);
    const int r = s - c * t.S01;
    b = (int)mulhi32((unsigned)r, t.m0);
    a = r - b * t.S0;
}

// o + d folded into [0, n) for d within a few periods of the box
__host__ __device__ __forceinline__ int wrap_index(int v, int n) {
    while (v < 0) v += n;
    while (v >= n) v -= n;
    return v;
}

__host__ __device__ __forceinline__ Tile tile_of(const Geom &g, int tile) {
    Tile t;
    const int tx = tile % g.ntile[0];
    const int ty = (tile / g.ntile[0]) % g.ntile[1];
    const int tz = tile / (g.ntile[0] * g.ntile[1]);
    t.ox = tx * g.tile[0];
    t.oy = ty * g.tile[1];
    t.oz = tz * g.tile[2];
    const int G = g.guard;
    t.S0 = g.tile[0] + 2 * G + 1;
    t.S01 = t.S0 * (g.tile[1] + 2 * G + 1);
    t.S = t.S01 * (g.tile[2] + 2 * G + 1);
    t.m0 = 0xFFFFFFFFu / (unsigned)t.S0 + 1u;
    t.m01 = 0xFFFFFFFFu / (unsigned)t.S01 + 1u;
    return t;
}

// slot of axis index a (0 <= a < n) in the box of the tile with origin o
// grown by G cells on each side: (a - o + G) mod n, valid below T + 2G (on a
// periodic axis shorter than the box, slots alias nodes, which the flush maps
// back to the same node)
__device__ __forceinline__ int box_slot(int a, int o, int n, int G) {
    int s = a - o + G;
    if (s < 0) s += n;
    if (s >= n) s -= n;
    return s;
}

// Box extents: B > 0 says the box is B slots long on every axis (a constant
// of the kernel, so slot offsets become immediates); B = 0 reads them from t.
template <int B>
__device__ __forceinline__ int box_row(const Tile &t) { return B > 0 ? B : t.S0; }
template <int B>
__device__ __forceinline__ int box_plane(const Tile &t) { return B > 0 ? B * B : t.S01; }

// slot s of stencil base (i, j, k) in the box of tile t; true if the whole
// 2x2x2 stencil lies inside the box
template <int B = 0>
__device__ __forceinline__ bool box_base(const Tile &t, const Geom &g, int i, int j, int k, int &s) {
    const int G = g.guard;
    const int si = box_slot(i, t.ox, g.n[0], G);
    const int sj = box_slot(j, t.oy, g.n[1], G);
    const int sk = box_slot(k, t.oz, g.n[2], G);
    s = si + box_row<B>(t) * sj + box_plane<B>(t) * sk;
    if (B > 0)
        return (unsigned)si < (unsigned)(B - 1) && (unsigned)sj < (unsigned)(B - 1) &&
               (unsigned)sk < (unsigned)(B - 1);
    return (unsigned)si < (unsigned)(t.S0 - 1) && (unsigned)sj < (unsigned)(g.tile[1] + 2 * G) &&
           (unsigned)sk < (unsigned)(g.tile[2] + 2 * G);
}

// returns true if the particle went to the shared tile, false if to the grid
template <bool FIXED, int B = 0>
__device__ __forceinline__ bool tile_add(uint32_t *acc, const Tile &t, const Geom &g, int i, int j,
                                         int k, float fx, float fy, float fz, float *rho,
                                         unsigned long long *rho64, float qscale) {
    int s;
    if (box_base<B>(t, g, i, j, k, s)) {
        const int S0 = box_row<B>(t), S01 = box_plane<B>(t);
        const int off[8] = {0, 1, S0, S0 + 1, S01, S01 + 1, S01 + S0, S01 + S0 + 1};
        if (FIXED) {
            uint32_t q[8];
            fixed_split(fx, fy, fz, q);
#pragma unroll
            for (int c = 0; c < 8; ++c) atomicAdd(acc + s + off[c], q[c]);
        } else {
            float w[8];
            weights(fx, fy, fz, w);
            float *accf = reinterpret_cast<float *>(acc);
#pragma unroll
            for (int c = 0; c < 8; ++c) atomicAdd(accf + s + off[c], w[c]);
        }
        return true;
    }
    float w[8];
    weights(fx, fy, fz, w);
    deposit_global<FIXED>(rho, rho64, g, i, j, k, w, fx, fy, fz, qscale);
    return false;
}

// add the shared tile to the grid: one global atomic per touched slot
template <bool FIXED>
__device__ __forceinline__ void tile_flush(const uint32_t *acc, const Tile &t, const Geom &g,
                                           float *rho, unsigned long long *rho64, float qscale) {
    const int G = g.guard;
    for (int s = threadIdx.x; s < t.S; s += blockDim.x) {
        const uint32_t raw = acc[s];
        if (raw != 0u) {
            int a, b, cz;
            tile_pos(t, s, a, b, cz);
            const int gi = wrap_index(t.ox - G + a, g.n[0]);
            const int gj = wrap_index(t.oy - G + b, g.n[1]);
            const int gk = wrap_index(t.oz - G + cz, g.n[2]);
            const int64_t node = gi + (int64_t)g.n[0] * (gj + (int64_t)g.n[1] * gk);
            if (FIXED) atomicAdd(rho64 + node, (unsigned long long)raw);
            else atomicAdd(rho + node, __uint_as_float(raw) * qscale);
        }
    }
}

// Second level of a block's deposit: the block walks a contiguous run of
// work items, folds each item's tile into `sum` (FIXED: 64-bit sums of the
// 32-bit item tiles, which cannot overflow; FP32: float sums) and flushes
// `sum` to the grid only when the run moves to another tile, so the items of
// one densely filled tile cost one set of grid atomics per block instead of
// one per item.  Each slot is touched by one thread in both loops.
template <bool FIXED>
__device__ __forceinline__ void tile_fold(uint32_t *acc, void *sum, int S) {
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        if (FIXED) reinterpret_cast<unsigned long long *>(sum)[s] += acc[s];
        else reinterpret_cast<float *>(sum)[s] += __uint_as_float(acc[s]);
        acc[s] = 0u;
    }
}

template <bool FIXED>
__device__ __forceinline__ void tile_flush_sum(void *sum, const Tile &t, const Geom &g, float *rho,
                                               unsigned long long *rho64, float qscale) {
    const int G = g.guard;
    for (int s = threadIdx.x; s < t.S; s += blockDim.x) {
        unsigned long long q = 0ull;
        float f = 0.0f;
        if (FIXED) {
            q = reinterpret_cast<unsigned long long *>(sum)[s];
            reinterpret_cast<unsigned long long *>(sum)[s] = 0ull;
        } else {
            f = reinterpret_cast<float *>(sum)[s];
            reinterpret_cast<float *>(sum)[s] = 0.0f;
        }
        if (FIXED ? q != 0ull : f != 0.0f) {
            int a, b, cz;
            tile_pos(t, s, a, b, cz);
            const int gi = wrap_index(t.ox - G + a, g.n[0]);
            const int gj = wrap_index(t.oy - G + b, g.n[1]);
            const int gk = wrap_index(t.oz - G + cz, g.n[2]);
            const int64_t node = gi + (int64_t)g.n[0] * (gj + (int64_t)g.n[1] * gk);
            if (FIXED) atomicAdd(rho64 + node, q);
            else atomicAdd(rho + node, f * qscale);
        }
    }
}

// the two shared tiles of a block: 32-bit item tile, then the 8-byte sums
__host__ __device__ __forceinline__ size_t sum_offset(int S) { return ((size_t)S * 4 + 7) & ~(size_t)7; }

// Copy of the field (one float4 per node) on the box of tile t -- the deposit
// tile's slots: the tile, G cells on each side and the +1 stencil layer,
// periodic -- into shared memory, one slot per thread and iteration.
__device__ __forceinline__ void stage_box(float4 *sE, const float4 *__restrict__ E4, const Tile &t,
                                          const Geom &g) {
    const int G = g.guard;
    for (int s = threadIdx.x; s < t.S; s += blockDim.x) {
        int a, b, cz;
        tile_pos(t, s, a, b, cz);
        const int gi = wrap_index(t.ox - G + a, g.n[0]);
        const int gj = wrap_index(t.oy - G + b, g.n[1]);
        const int gk = wrap_index(t.oz - G + cz, g.n[2]);
        sE[s] = __ldg(E4 + gi + (int64_t)g.n[0] * (gj + (int64_t)g.n[1] * gk));
    }
}

// byte offset of a staged box of S slots in the push kernels' shared memory,
// after the item tile and the tile sums
__host__ __device__ __forceinline__ size_t stage_offset(int S) {
    return (sum_offset(S) + 8 * (size_t)S + 15) & ~(size_t)15;
}

}  // namespace cic
}  // namespace pic
