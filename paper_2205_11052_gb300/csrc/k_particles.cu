// Particle kernels: load/normalise, readback, and the fused gather + push.
//
// Gather + push follows Section 3.1 steps 3-4 (Eq. momentum_eqn) and
// Section 3.2 of arXiv 2205.11052: E is interpolated to the particle with the
// CIC weights of the deposit, the velocity is advanced by the Boris rotation
// (exact solution of v1 = v0 + dt (q/m) [e + (v0 + v1)/2 x B]), and the
// position drifts by a full step, wrapped periodically.  The device keeps the
// drift-kick-drift state (x_{n+1/2}, v_n), so one pass takes x_{n+1/2} to
// x_{n+3/2} = x_{n+1/2} + dt v_{n+1}.
#include <math.h>

#include "pic_internal.cuh"

namespace pic {

namespace {

__device__ __forceinline__ void raise_flag(Ctrl *ctrl, int bit) { atomicOr(&ctrl->flags, bit); }

// ---------------------------------------------------------------------------
// load: FP64 (x_0, v_0) -> x_{1/2} = x_0 + dt/2 v_0 -> (cell, offset, v)
// ---------------------------------------------------------------------------
__global__ void k_load(const double *__restrict__ x, const double *__restrict__ v, int64_t m,
                       int64_t base, Geom g, double ih0, double ih1, double ih2, double dt,
                       Ctrl *ctrl) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= m) return;
    const ParticleSet ps = ctrl->sets[ctrl->cur];
    const double ih[3] = {ih0, ih1, ih2};
    int idx[3];
    float off[3];
    bool ok = true;
    for (int d = 0; d < 3; ++d) {
        double vd = v[3 * p + d];
        double xd = x[3 * p + d] + 0.5 * dt * vd;
        double s = xd * ih[d] - 0.5;      // node g at (g + 1/2) h
        if (!isfinite(s) || !isfinite(vd) || fabs(s) > 4.0e15) {
            ok = false;
            s = 0.0;
        }
        double fl = floor(s);
        double f = s - fl;
        long long il = (long long)fl % g.n[d];
        if (il < 0) il += g.n[d];
        float ff = (float)f;
        if (ff >= 1.0f) {             // rounding to 1.0f moves to the next node
            ff = 0.0f;
            il += 1;
            if (il == g.n[d]) il = 0;
        }
        idx[d] = (int)il;
        off[d] = ff;
        ps.v[d][base + p] = ok ? (float)vd : 0.0f;
    }
    if (!ok) raise_flag(ctrl, PIC_FLAG_NONFINITE);
    ps.cell[base + p] = pack_cell(idx[0], idx[1], idx[2]);
    ps.o[0][base + p] = off[0];
    ps.o[1][base + p] = off[1];
    ps.o[2][base + p] = off[2];
    ps.pid[base + p] = (int32_t)(base + p);
}

__global__ void k_invperm(int64_t n, const Ctrl *ctrl, int32_t *inv) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const ParticleSet ps = ctrl->sets[ctrl->cur];
    inv[ps.pid[p]] = (int32_t)p;
}

// synchronised readback: x_n = x_{n+1/2} - dt/2 v_n, in load order
__global__ void k_unload(int64_t o0, int64_t m, const int32_t *__restrict__ inv, Geom g,
                         double h0, double h1, double h2, double L0, double L1, double L2,
                         double dt, const Ctrl *ctrl, double *__restrict__ x,
                         double *__restrict__ v) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= m) return;
    const ParticleSet ps = ctrl->sets[ctrl->cur];
    int64_t p = inv[o0 + q];
    int32_t c = ps.cell[p];
    const int idx[3] = {cell_i(c), cell_j(c), cell_k(c)};
    const double h[3] = {h0, h1, h2};
    const double L[3] = {L0, L1, L2};
    for (int d = 0; d < 3; ++d) {
        double vd = (double)ps.v[d][p];
        double xd = ((double)idx[d] + 0.5 + (double)ps.o[d][p]) * h[d] - 0.5 * dt * vd;
        xd -= L[d] * floor(xd / L[d]);
        if (xd >= L[d]) xd -= L[d];
        if (xd < 0.0) xd = 0.0;
        x[3 * q + d] = xd;
        v[3 * q + d] = vd;
    }
}

// ---------------------------------------------------------------------------
// fused gather + Boris push + drift + periodic wrap
// ---------------------------------------------------------------------------
template <bool DIAG, bool EXT, bool MAG>
__global__ void __launch_bounds__(256) k_gather_push(int64_t n, Geom g, PushConst pc, Ctrl *ctrl,
                                                      const float4 *__restrict__ E4,
                                                      double *__restrict__ part) {
    const ParticleSet ps = ctrl->sets[ctrl->cur];
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int nxy = nx * ny;
    float a_vx = 0.f, a_vy = 0.f, a_vz = 0.f, a_v2 = 0.f;
    int bad = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        const int32_t c = ps.cell[p];
        int i = cell_i(c), j = cell_j(c), k = cell_k(c);
        if (i >= nx || j >= ny || k >= nz) {   // never produced by the kernels
            bad |= PIC_FLAG_BAD_CELL;
            i = j = k = 0;
        }
        float fx = ps.o[0][p], fy = ps.o[1][p], fz = ps.o[2][p];
        float vx = ps.v[0][p], vy = ps.v[1][p], vz = ps.v[2][p];

        // CIC stencil nodes (periodic)
        const int i1 = (i + 1 == nx) ? 0 : i + 1;
        const int j1 = (j + 1 == ny) ? 0 : j + 1;
        const int k1 = (k + 1 == nz) ? 0 : k + 1;
        const int r00 = j * nx + k * nxy, r10 = j1 * nx + k * nxy;
        const int r01 = j * nx + k1 * nxy, r11 = j1 * nx + k1 * nxy;
        const float4 e000 = __ldg(E4 + r00 + i), e100 = __ldg(E4 + r00 + i1);
        const float4 e010 = __ldg(E4 + r10 + i), e110 = __ldg(E4 + r10 + i1);
        const float4 e001 = __ldg(E4 + r01 + i), e101 = __ldg(E4 + r01 + i1);
        const float4 e011 = __ldg(E4 + r11 + i), e111 = __ldg(E4 + r11 + i1);
        const float wx1 = fx, wx0 = 1.0f - fx;
        const float wy1 = fy, wy0 = 1.0f - fy;
        const float wz1 = fz, wz0 = 1.0f - fz;
        const float w00 = wy0 * wz0, w10 = wy1 * wz0, w01 = wy0 * wz1, w11 = wy1 * wz1;
        float ex = w00 * (wx0 * e000.x + wx1 * e100.x) + w10 * (wx0 * e010.x + wx1 * e110.x) +
                   w01 * (wx0 * e001.x + wx1 * e101.x) + w11 * (wx0 * e011.x + wx1 * e111.x);
        float ey = w00 * (wx0 * e000.y + wx1 * e100.y) + w10 * (wx0 * e010.y + wx1 * e110.y) +
                   w01 * (wx0 * e001.y + wx1 * e101.y) + w11 * (wx0 * e011.y + wx1 * e111.y);
        float ez = w00 * (wx0 * e000.z + wx1 * e100.z) + w10 * (wx0 * e010.z + wx1 * e110.z) +
                   w01 * (wx0 * e001.z + wx1 * e101.z) + w11 * (wx0 * e011.z + wx1 * e111.z);
        if (EXT) {
            // quadrupole about the box centre: (x - c)/h = i - N/2 + 1/2 + f
            const float dx = ((float)i - pc.half_n[0] + 0.5f + fx) * g.h[0];
            const float dy = ((float)j - pc.half_n[1] + 0.5f + fy) * g.h[1];
            const float dz = ((float)k - pc.half_n[2] + 0.5f + fz) * g.h[2];
            ex += -0.5f * pc.wz2 * dx;
            ey += -0.5f * pc.wz2 * dy;
            ez += pc.wz2 * dz;
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
        float sx = fx + pc.dt_over_h[0] * vx;
        float sy = fy + pc.dt_over_h[1] * vy;
        float sz = fz + pc.dt_over_h[2] * vz;
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

        ps.cell[p] = pack_cell(i, j, k);
        ps.o[0][p] = fx;
        ps.o[1][p] = fy;
        ps.o[2][p] = fz;
        ps.v[0][p] = vx;
        ps.v[1][p] = vy;
        ps.v[2][p] = vz;
        if (DIAG) {
            a_vx += vx;
            a_vy += vy;
            a_vz += vz;
            a_v2 += vx * vx + vy * vy + vz * vz;
        }
    }
    if (bad) raise_flag(ctrl, bad);
    if (DIAG) {
        // per-thread FP32 partials (a few particles each) -> FP64 block sum in
        // a fixed order -> one partial per block (deterministic)
        double d[4] = {(double)a_vx, (double)a_vy, (double)a_vz, (double)a_v2};
        __shared__ double red[4][8];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        for (int q = 0; q < 4; ++q) {
            double t = d[q];
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0) red[q][wid] = t;
        }
        __syncthreads();
        if (threadIdx.x < 4) {
            double t = 0.0;
            const int nw = blockDim.x >> 5;
            for (int w = 0; w < nw; ++w) t += red[threadIdx.x][w];
            part[4 * blockIdx.x + threadIdx.x] = t;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->step += 1;
}

}  // namespace

cudaError_t launch_load(const double *x, const double *v, int64_t m, int64_t base, const Geom &g,
                        const double *inv_h_d, double dt, Ctrl *ctrl, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    const int T = 256;
    const int64_t B = (m + T - 1) / T;
    k_load<<<(unsigned)B, T, 0, st>>>(x, v, m, base, g, inv_h_d[0], inv_h_d[1], inv_h_d[2], dt,
                                      ctrl);
    return cudaGetLastError();
}

cudaError_t launch_invperm(int64_t n, Ctrl *ctrl, int32_t *inv, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int T = 256;
    k_invperm<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(n, ctrl, inv);
    return cudaGetLastError();
}

cudaError_t launch_unload(int64_t o0, int64_t m, const int32_t *inv, const Geom &g,
                          const double *h_d, const double *L_d, double dt, const Ctrl *ctrl,
                          double *x, double *v, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    const int T = 256;
    k_unload<<<(unsigned)((m + T - 1) / T), T, 0, st>>>(o0, m, inv, g, h_d[0], h_d[1], h_d[2],
                                                        L_d[0], L_d[1], L_d[2], dt, ctrl, x, v);
    return cudaGetLastError();
}

cudaError_t launch_gather_push(int64_t n, const Geom &g, const PushConst &pc, bool diag,
                               Ctrl *ctrl, const float4 *E4, double *part, int blocks,
                               int threads, cudaStream_t st) {
    const bool ext = pc.wz2 != 0.0f;
    const bool mag = pc.t[0] != 0.0f || pc.t[1] != 0.0f || pc.t[2] != 0.0f;
#define PIC_GP(D, X, M) k_gather_push<D, X, M><<<blocks, threads, 0, st>>>(n, g, pc, ctrl, E4, part)
    if (diag) {
        if (ext) { if (mag) PIC_GP(true, true, true); else PIC_GP(true, true, false); }
        else     { if (mag) PIC_GP(true, false, true); else PIC_GP(true, false, false); }
    } else {
        if (ext) { if (mag) PIC_GP(false, true, true); else PIC_GP(false, true, false); }
        else     { if (mag) PIC_GP(false, false, true); else PIC_GP(false, false, false); }
    }
#undef PIC_GP
    return cudaGetLastError();
}

}  // namespace pic
