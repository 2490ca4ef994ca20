// The per-particle gather + Boris push + drift of Section 3.1 steps 3-4
// (Eq. momentum_eqn) and Section 3.2 of arXiv 2205.11052, shared by the
// single-run and the batched kernels.
//
// E is interpolated to the particle with the CIC weights of the deposit, the
// velocity is advanced by the Boris rotation (exact solution of
// v1 = v0 + dt (q/m) [e + (v0 + v1)/2 x B]) and the position drifts by a full
// step in cell units, carried into the cell index and wrapped periodically.
#pragma once

#include "cic.cuh"
#include "pic_internal.cuh"

namespace pic {

__device__ __forceinline__ void advance_cells(const Geom &g, float sx, float sy, float sz, int &i,
                                              int &j, int &k, int32_t &c, float &fx, float &fy,
                                              float &fz, int &bad);

// CIC interpolation of the eight corner values (corner bits a | b<<1 | c<<2)
__device__ __forceinline__ void interp_E(const float4 e[8], float fx, float fy, float fz,
                                        float &ex, float &ey, float &ez) {
    const float wx1 = fx, wx0 = 1.0f - fx;
    const float wy1 = fy, wy0 = 1.0f - fy;
    const float wz1 = fz, wz0 = 1.0f - fz;
    const float w00 = wy0 * wz0, w10 = wy1 * wz0, w01 = wy0 * wz1, w11 = wy1 * wz1;
    ex = w00 * (wx0 * e[0].x + wx1 * e[1].x) + w10 * (wx0 * e[2].x + wx1 * e[3].x) +
         w01 * (wx0 * e[4].x + wx1 * e[5].x) + w11 * (wx0 * e[6].x + wx1 * e[7].x);
    ey = w00 * (wx0 * e[0].y + wx1 * e[1].y) + w10 * (wx0 * e[2].y + wx1 * e[3].y) +
         w01 * (wx0 * e[4].y + wx1 * e[5].y) + w11 * (wx0 * e[6].y + wx1 * e[7].y);
    ez = w00 * (wx0 * e[0].z + wx1 * e[1].z) + w10 * (wx0 * e[2].z + wx1 * e[3].z) +
         w01 * (wx0 * e[4].z + wx1 * e[5].z) + w11 * (wx0 * e[6].z + wx1 * e[7].z);
}

// E at the particle from the grid in global memory (periodic stencil)
__device__ __forceinline__ void gather_E_global(const Geom &g, const float4 *__restrict__ E4, int i,
                                                int j, int k, float fx, float fy, float fz,
                                                float &ex, float &ey, float &ez) {
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int i1 = (i + 1 == nx) ? 0 : i + 1;
    const int j1 = (j + 1 == ny) ? 0 : j + 1;
    const int k1 = (k + 1 == nz) ? 0 : k + 1;
    const int nxy = nx * ny;
    const int r00 = j * nx + k * nxy, r10 = j1 * nx + k * nxy;
    const int r01 = j * nx + k1 * nxy, r11 = j1 * nx + k1 * nxy;
    float4 e[8];
    e[0] = __ldg(E4 + r00 + i);
    e[1] = __ldg(E4 + r00 + i1);
    e[2] = __ldg(E4 + r10 + i);
    e[3] = __ldg(E4 + r10 + i1);
    e[4] = __ldg(E4 + r01 + i);
    e[5] = __ldg(E4 + r01 + i1);
    e[6] = __ldg(E4 + r11 + i);
    e[7] = __ldg(E4 + r11 + i1);
    interp_E(e, fx, fy, fz, ex, ey, ez);
}

// E8 holds, per node q, E at q and at its +x neighbour (periodic): 32 bytes,
// so each of the four (y, z) corner rows of the stencil is one aligned
// 256-bit read-only load
__device__ __forceinline__ void ld_pair(const float4 *p, float4 &a, float4 &b) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}

__device__ __forceinline__ void gather_E_pairs(const Geom &g, const float4 *__restrict__ E8, int i,
                                               int j, int k, float fx, float fy, float fz,
                                               float &ex, float &ey, float &ez) {
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int j1 = (j + 1 == ny) ? 0 : j + 1;
    const int k1 = (k + 1 == nz) ? 0 : k + 1;
    const int nxy = nx * ny;
    const int r00 = j * nx + k * nxy + i, r10 = j1 * nx + k * nxy + i;
    const int r01 = j * nx + k1 * nxy + i, r11 = j1 * nx + k1 * nxy + i;
    float4 e[8];
    ld_pair(E8 + 2 * r00, e[0], e[1]);
    ld_pair(E8 + 2 * r10, e[2], e[3]);
    ld_pair(E8 + 2 * r01, e[4], e[5]);
    ld_pair(E8 + 2 * r11, e[6], e[7]);
    interp_E(e, fx, fy, fz, ex, ey, ez);
}

// E at the particle from a copy of the field on a box in shared memory (one
// float4 per slot; s0 is the stencil base's slot, rows S0 slots apart in y,
// planes S01 apart in z)
template <int B = 0>
__device__ __forceinline__ void gather_E_box(const float4 *sE, int s0, int S0r, int S01r, float fx,
                                             float fy, float fz, float &ex, float &ey,
                                             float &ez) {
    const int S0 = B > 0 ? B : S0r, S01 = B > 0 ? B * B : S01r;   // B > 0: a constant box
    float4 e[8];
    e[0] = sE[s0];
    e[1] = sE[s0 + 1];
    e[2] = sE[s0 + S0];
    e[3] = sE[s0 + S0 + 1];
    e[4] = sE[s0 + S01];
    e[5] = sE[s0 + S01 + 1];
    e[6] = sE[s0 + S01 + S0];
    e[7] = sE[s0 + S01 + S0 + 1];
    interp_E(e, fx, fy, fz, ex, ey, ez);
}

// Boris kick with the interpolated field (plus the external quadrupole), then
// a full drift in cell units carried into the cell index and wrapped; (i, j, k)
// is the particle's stencil base before the step and after it
template <bool EXT, bool MAG>
__device__ __forceinline__ void kick_drift(const Geom &g, const PushConst &pc, float ex, float ey,
                                           float ez, int &i, int &j, int &k, int32_t &c, float &fx,
                                           float &fy, float &fz, float &vx, float &vy, float &vz,
                                           int &bad) {
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    if (EXT) {
        // quadrupole about the box centre at x in [0, L): (x - c)/h = i - N/2 +
        // 1/2 + f, wrapped into [-N/2, N/2) (a particle in [0, h/2) has its
        // stencil base on node N-1, i.e. i + 1/2 + f lies in [N, N + 1/2))
        float ux = (float)i - pc.half_n[0] + 0.5f + fx;
        float uy = (float)j - pc.half_n[1] + 0.5f + fy;
        float uz = (float)k - pc.half_n[2] + 0.5f + fz;
        if (ux >= pc.half_n[0]) ux -= (float)nx;
        if (uy >= pc.half_n[1]) uy -= (float)ny;
        if (uz >= pc.half_n[2]) uz -= (float)nz;
        ex += -0.5f * pc.wz2 * (ux * g.h[0]);
        ey += -0.5f * pc.wz2 * (uy * g.h[1]);
        ez += pc.wz2 * (uz * g.h[2]);
    }
    // Boris: half kick, rotation, half kick
    float mx = vx + pc.qm_half_dt * ex;
    float my = vy + pc.qm_half_dt * ey;
    float mz = vz + pc.qm_half_dt * ez;
    if (MAG) {
        const float px = mx + (my * pc.t[2] - mz * pc.t[1]);
        const float py = my + (mz * pc.t[0] - mx * pc.t[2]);
        const float pz = mz + (mx * pc.t[1] - my * pc.t[0]);
        mx += py * pc.s[2] - pz * pc.s[1];
        my += pz * pc.s[0] - px * pc.s[2];
        mz += px * pc.s[1] - py * pc.s[0];
    }
    vx = mx + pc.qm_half_dt * ex;
    vy = my + pc.qm_half_dt * ey;
    vz = mz + pc.qm_half_dt * ez;

    // drift a full step in cell units, carry into the cell index, wrap
    advance_cells(g, fx + pc.dt_over_h[0] * vx, fy + pc.dt_over_h[1] * vy,
                  fz + pc.dt_over_h[2] * vz, i, j, k, c, fx, fy, fz, bad);
}

// New in-cell offsets s (in cell units, relative to the stencil base
// (i, j, k)): carry floor(s) into the cell index, keep the fraction, wrap
// periodically, repack the cell; (i, j, k) become the new stencil base
__device__ __forceinline__ void advance_cells(const Geom &g, float sx, float sy, float sz, int &i,
                                              int &j, int &k, int32_t &c, float &fx, float &fy,
                                              float &fz, int &bad) {
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    float flx = floorf(sx), fly = floorf(sy), flz = floorf(sz);
    fx = sx - flx;
    fy = sy - fly;
    fz = sz - flz;
    if (fx >= 1.0f) { fx = 0.0f; flx += 1.0f; }
    if (fy >= 1.0f) { fy = 0.0f; fly += 1.0f; }
    if (fz >= 1.0f) { fz = 0.0f; flz += 1.0f; }
    if (!(fabsf(flx) < 1.0e6f && fabsf(fly) < 1.0e6f && fabsf(flz) < 1.0e6f)) {
        bad |= PIC_FLAG_NONFINITE;
        flx = fly = flz = 0.0f;
        fx = fy = fz = 0.0f;
    }
    i += (int)flx;
    j += (int)fly;
    k += (int)flz;
    if ((unsigned)i >= (unsigned)nx) { i %= nx; if (i < 0) i += nx; }
    if ((unsigned)j >= (unsigned)ny) { j %= ny; if (j < 0) j += ny; }
    if ((unsigned)k >= (unsigned)nz) { k %= nz; if (k < 0) k += nz; }
    c = pack_cell(i, j, k);
}

// stencil base of a packed cell (flagged and clamped to 0 if out of range)
__device__ __forceinline__ void decode_base(const Geom &g, int32_t c, int &i, int &j, int &k,
                                            int &bad) {
    i = cell_i(c);
    j = cell_j(c);
    k = cell_k(c);
    if (i >= g.n[0] || j >= g.n[1] || k >= g.n[2]) {   // never produced by the kernels
        bad |= PIC_FLAG_BAD_CELL;
        i = j = k = 0;
    }
}

// gather from the grid in global memory + kick + drift
template <bool EXT, bool MAG>
__device__ __forceinline__ void push_one(const Geom &g, const PushConst &pc,
                                         const float4 *__restrict__ E4, int32_t &c, float &fx,
                                         float &fy, float &fz, float &vx, float &vy, float &vz,
                                         int &bad) {
    int i, j, k;
    decode_base(g, c, i, j, k, bad);
    float ex, ey, ez;
    gather_E_global(g, E4, i, j, k, fx, fy, fz, ex, ey, ez);
    kick_drift<EXT, MAG>(g, pc, ex, ey, ez, i, j, k, c, fx, fy, fz, vx, vy, vz, bad);
}

// gather from the x-paired grid + kick + drift; (i, j, k) receives the new
// stencil base (the fields of the new packed cell c)
template <bool EXT, bool MAG>
__device__ __forceinline__ void push_one_pairs(const Geom &g, const PushConst &pc,
                                               const float4 *__restrict__ E8, int32_t &c,
                                               float &fx, float &fy, float &fz, float &vx,
                                               float &vy, float &vz, int &bad, int &i, int &j,
                                               int &k) {
    decode_base(g, c, i, j, k, bad);
    float ex, ey, ez;
    gather_E_pairs(g, E8, i, j, k, fx, fy, fz, ex, ey, ez);
    kick_drift<EXT, MAG>(g, pc, ex, ey, ez, i, j, k, c, fx, fy, fz, vx, vy, vz, bad);
}

template <bool EXT, bool MAG>
__device__ __forceinline__ void push_one_pairs(const Geom &g, const PushConst &pc,
                                               const float4 *__restrict__ E8, int32_t &c,
                                               float &fx, float &fy, float &fz, float &vx,
                                               float &vy, float &vz, int &bad) {
    int i, j, k;
    push_one_pairs<EXT, MAG>(g, pc, E8, c, fx, fy, fz, vx, vy, vz, bad, i, j, k);
}

// Gather + kick + drift with E read from sE, the block's shared-memory copy
// of the box of tile t (cic::stage_box), when the particle's stencil lies in
// that box: eight 16-byte shared loads, a few shared wavefronts per warp
// instead of one L1 wavefront per particle and 32-byte global read.  Other
// particles, and every particle when sE is null, read the x-paired grid E8.
// (i, j, k) receives the new stencil base.
template <bool EXT, bool MAG, int B = 0>
__device__ __forceinline__ void push_one_staged(const Geom &g, const PushConst &pc,
                                                const float4 *__restrict__ E8, const float4 *sE,
                                                const cic::Tile &t, int32_t &c, float &fx,
                                                float &fy, float &fz, float &vx, float &vy,
                                                float &vz, int &bad, int &i, int &j, int &k) {
    decode_base(g, c, i, j, k, bad);
    float ex, ey, ez;
    int s0;
    if (sE != nullptr && cic::box_base<B>(t, g, i, j, k, s0))
        gather_E_box<B>(sE, s0, t.S0, t.S01, fx, fy, fz, ex, ey, ez);
    else
        gather_E_pairs(g, E8, i, j, k, fx, fy, fz, ex, ey, ez);
    kick_drift<EXT, MAG>(g, pc, ex, ey, ez, i, j, k, c, fx, fy, fz, vx, vy, vz, bad);
}

}  // namespace pic
