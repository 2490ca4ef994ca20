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

#include <algorithm>

#include "cic.cuh"
#include "push.cuh"

namespace pic {

namespace {

__device__ __forceinline__ void raise_flag(Ctrl *ctrl, int bit) { atomicOr(&ctrl->flags, bit); }

// Velocity moments (sum v, sum |v|^2) are summed per thread in FP32 over a
// few particles (one work item's share, or one loop iteration) and then
// added to the thread's FP64 totals, so no FP32 sum runs over more than a
// few dozen terms.
__device__ __forceinline__ void fold_moments(float (&a)[4], double (&d)[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        d[q] += (double)a[q];
        a[q] = 0.f;
    }
}

// ---------------------------------------------------------------------------
// load: FP64 (x_0, v_0) -> x_{1/2} = x_0 + dt/2 v_0 -> (cell, offset, v)
// ---------------------------------------------------------------------------
constexpr int kLoadThreads = 256;

__global__ void __launch_bounds__(kLoadThreads) k_load(const double *__restrict__ x,
                                                      const double *__restrict__ v, int64_t m,
                                                      int64_t base, Geom g, double ih0,
                                                      double ih1, double ih2, double dt,
                                                      Ctrl *ctrl) {
    // the block's 256 (x, y, z) triples of x and of v are read as contiguous
    // runs (every byte once, six independent loads per thread) and staged in
    // shared memory: the source may be host memory read over the chip-to-chip
    // link, where strided 8-byte reads would fetch each line three times
    __shared__ double sx[3 * kLoadThreads], sv[3 * kLoadThreads];
    const ParticleSet ps = ctrl->sets[ctrl->cur];
    const double ih[3] = {ih0, ih1, ih2};
    bool any_bad = false;
    // blocks stride over runs of kLoadThreads particles
    for (int64_t p0 = (int64_t)blockIdx.x * kLoadThreads; p0 < m;
         p0 += (int64_t)gridDim.x * kLoadThreads) {
        const int cnt = (int)(m - p0 < kLoadThreads ? m - p0 : kLoadThreads);
        __syncthreads();   // the previous run's shared values are consumed
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const int j = r * kLoadThreads + threadIdx.x;
            if (j < 3 * cnt) {
                sx[j] = x[3 * p0 + j];
                sv[j] = v[3 * p0 + j];
            }
        }
        __syncthreads();
        if ((int)threadIdx.x >= cnt) continue;
        const int64_t p = p0 + threadIdx.x;
        double xr[3], vr[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            xr[d] = sx[3 * threadIdx.x + d];
            vr[d] = sv[3 * threadIdx.x + d];
        }
        int idx[3];
        float off[3];
        bool ok = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double vd = vr[d];
            double xd = xr[d] + 0.5 * dt * vd;
            double s = xd * ih[d] - 0.5;      // node g at (g + 1/2) h
            // finite v and |s| < 2^52, tested on the exponent fields (FP64
            // instructions are scarce on this GPU; integer ones are not)
            const unsigned es =
                (unsigned)((unsigned long long)__double_as_longlong(s) >> 52) & 0x7ffu;
            const unsigned ev =
                (unsigned)((unsigned long long)__double_as_longlong(vd) >> 52) & 0x7ffu;
            if (es >= 1023u + 52u || ev == 0x7ffu) {
                ok = false;
                s = 0.0;
            }
            double fl = floor(s);
            double f = s - fl;
            long long il = (long long)fl;
            if ((unsigned long long)il >= (unsigned long long)g.n[d]) {   // outside: wrap
                il %= g.n[d];
                if (il < 0) il += g.n[d];
            }
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
        if (!ok) any_bad = true;
        ps.cell[base + p] = pack_cell(idx[0], idx[1], idx[2]);
        ps.o[0][base + p] = off[0];
        ps.o[1][base + p] = off[1];
        ps.o[2][base + p] = off[2];
        ps.pid[base + p] = (int32_t)(base + p);
    }
    if (any_bad) raise_flag(ctrl, PIC_FLAG_NONFINITE);
}

__global__ void k_invperm(int64_t n, const Ctrl *ctrl, int32_t *inv) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const ParticleSet ps = ctrl->sets[ctrl->cur];
    inv[ps.pid[p]] = (int32_t)p;
}

// synchronised readback: x_n = x_{n+1/2} - dt/2 v_n, in load order
__global__ void __launch_bounds__(kLoadThreads) k_unload(int64_t o0, int64_t m,
                                                        const int32_t *__restrict__ inv, Geom g,
                                                        double h0, double h1, double h2,
                                                        double L0, double L1, double L2, double dt,
                                                        const Ctrl *ctrl, double *__restrict__ x,
                                                        double *__restrict__ v) {
    // results are staged in shared memory and written as contiguous runs (the
    // destination may be host memory written over the chip-to-chip link)
    __shared__ double sx[3 * kLoadThreads], sv[3 * kLoadThreads];
    const int64_t q0 = (int64_t)blockIdx.x * kLoadThreads;
    const int cnt = (int)(m - q0 < kLoadThreads ? m - q0 : kLoadThreads);
    if ((int)threadIdx.x < cnt) {
        const ParticleSet ps = ctrl->sets[ctrl->cur];
        const int64_t p = inv[o0 + q0 + threadIdx.x];
        const int32_t c = ps.cell[p];
        const int idx[3] = {cell_i(c), cell_j(c), cell_k(c)};
        const double h[3] = {h0, h1, h2};
        const double L[3] = {L0, L1, L2};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double vd = (double)ps.v[d][p];
            double xd = ((double)idx[d] + 0.5 + (double)ps.o[d][p]) * h[d] - 0.5 * dt * vd;
            if (xd < 0.0 || xd >= L[d]) {   // wrap (the FP64 division only when needed)
                xd -= L[d] * floor(xd / L[d]);
                if (xd >= L[d]) xd -= L[d];
                if (xd < 0.0) xd = 0.0;
            }
            sx[3 * threadIdx.x + d] = xd;
            sv[3 * threadIdx.x + d] = vd;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const int j = r * kLoadThreads + threadIdx.x;
        if (j < 3 * cnt) {
            x[3 * q0 + j] = sx[j];
            v[3 * q0 + j] = sv[j];
        }
    }
}

// ---------------------------------------------------------------------------
// gather + Boris push + drift + periodic wrap (push_one in push.cuh)
//
// Each thread owns groups of 4 consecutive particles: the seven SoA streams
// are read and written as 16-byte vectors with evict-first hints (they are
// touched once per step), while the float4 field is read through the
// read-only path so it stays cached (the whole 128^3 field is 32 MiB).
// ---------------------------------------------------------------------------
template <bool DIAG, bool EXT, bool MAG>
__global__ void __launch_bounds__(256, 3) k_gather_push(int64_t n, Geom g, PushConst pc, Ctrl *ctrl,
                                                      const float4 *__restrict__ E8,
                                                      double *__restrict__ part) {
    const ParticleSet ps = ctrl->sets[ctrl->cur];
    float a_vx = 0.f, a_vy = 0.f, a_vz = 0.f, a_v2 = 0.f;
    double d_v[4] = {0.0, 0.0, 0.0, 0.0};
    int bad = 0;
    const int64_t ngroups = n >> 2;                      // full groups of 4
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < ngroups; q += stride) {
        int4 c = __ldcs(reinterpret_cast<const int4 *>(ps.cell) + q);
        float4 ox = __ldcs(reinterpret_cast<const float4 *>(ps.o[0]) + q);
        float4 oy = __ldcs(reinterpret_cast<const float4 *>(ps.o[1]) + q);
        float4 oz = __ldcs(reinterpret_cast<const float4 *>(ps.o[2]) + q);
        float4 ux = __ldcs(reinterpret_cast<const float4 *>(ps.v[0]) + q);
        float4 uy = __ldcs(reinterpret_cast<const float4 *>(ps.v[1]) + q);
        float4 uz = __ldcs(reinterpret_cast<const float4 *>(ps.v[2]) + q);
        push_one_pairs<EXT, MAG>(g, pc, E8, c.x, ox.x, oy.x, oz.x, ux.x, uy.x, uz.x, bad);
        push_one_pairs<EXT, MAG>(g, pc, E8, c.y, ox.y, oy.y, oz.y, ux.y, uy.y, uz.y, bad);
        push_one_pairs<EXT, MAG>(g, pc, E8, c.z, ox.z, oy.z, oz.z, ux.z, uy.z, uz.z, bad);
        push_one_pairs<EXT, MAG>(g, pc, E8, c.w, ox.w, oy.w, oz.w, ux.w, uy.w, uz.w, bad);
        __stcs(reinterpret_cast<int4 *>(ps.cell) + q, c);
        __stcs(reinterpret_cast<float4 *>(ps.o[0]) + q, ox);
        __stcs(reinterpret_cast<float4 *>(ps.o[1]) + q, oy);
        __stcs(reinterpret_cast<float4 *>(ps.o[2]) + q, oz);
        __stcs(reinterpret_cast<float4 *>(ps.v[0]) + q, ux);
        __stcs(reinterpret_cast<float4 *>(ps.v[1]) + q, uy);
        __stcs(reinterpret_cast<float4 *>(ps.v[2]) + q, uz);
        if (DIAG) {
            a_vx += (ux.x + ux.y) + (ux.z + ux.w);
            a_vy += (uy.x + uy.y) + (uy.z + uy.w);
            a_vz += (uz.x + uz.y) + (uz.z + uz.w);
            a_v2 += (ux.x * ux.x + uy.x * uy.x + uz.x * uz.x) + (ux.y * ux.y + uy.y * uy.y + uz.y * uz.y) +
                    (ux.z * ux.z + uy.z * uy.z + uz.z * uz.z) + (ux.w * ux.w + uy.w * uy.w + uz.w * uz.w);
            d_v[0] += (double)a_vx;
            d_v[1] += (double)a_vy;
            d_v[2] += (double)a_vz;
            d_v[3] += (double)a_v2;
            a_vx = a_vy = a_vz = a_v2 = 0.f;
        }
    }
    // the n mod 4 particles after the last full group: first threads of block 0
    if (blockIdx.x == 0 && threadIdx.x < (n & 3)) {
        const int64_t p = (ngroups << 2) + threadIdx.x;
        int32_t c = ps.cell[p];
        float fx = ps.o[0][p], fy = ps.o[1][p], fz = ps.o[2][p];
        float vx = ps.v[0][p], vy = ps.v[1][p], vz = ps.v[2][p];
        push_one_pairs<EXT, MAG>(g, pc, E8, c, fx, fy, fz, vx, vy, vz, bad);
        ps.cell[p] = c;
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
        // per-thread FP64 totals -> FP64 block sum in a fixed order -> one
        // partial per block (deterministic)
        double d[4] = {d_v[0] + a_vx, d_v[1] + a_vy, d_v[2] + a_vz, d_v[3] + a_v2};
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
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctrl->step += 1;
        ctrl->since_sort += 1;
    }
}


// ---------------------------------------------------------------------------
// fused gather + push + deposit of the new positions (one pass per step)
//
// Scatter of step n+1 needs exactly the positions this push writes, so the
// CTA that pushes a work item's particles also deposits them into the
// item's shared-memory tile (the sort's tile plus guard cells) and flushes
// it at the end: per step the particle store is read and written once (56
// bytes per particle) instead of being read again by a separate deposit.
// ---------------------------------------------------------------------------
// E from the block's shared copy of its tile's box when it holds one (see
// push_one_staged), else from the x-paired grid.
template <bool DIAG, bool EXT, bool MAG, bool FIXED, int B>
__device__ __forceinline__ void pd_one(const Geom &g, const PushConst &pc, const float4 *E8,
                                       const float4 *sE, bool sparse, uint32_t *acc,
                                       const cic::Tile &t, float *rho, unsigned long long *rho64,
                                       float qscale, int32_t &c, float &fx, float &fy, float &fz,
                                       float &vx, float &vy, float &vz, int &bad,
                                       unsigned long long &strays, float (&a)[4]) {
    int i, j, k;
    push_one_staged<EXT, MAG, B>(g, pc, E8, sE, t, c, fx, fy, fz, vx, vy, vz, bad, i, j, k);
    if (sparse) {
        float w[8];
        cic::weights(fx, fy, fz, w);
        cic::deposit_global<FIXED>(rho, rho64, g, i, j, k, w, fx, fy, fz, qscale);
    } else if (!cic::tile_add<FIXED, B>(acc, t, g, i, j, k, fx, fy, fz, rho, rho64, qscale)) {
        ++strays;
    }
    if (DIAG) {
        a[0] += vx;
        a[1] += vy;
        a[2] += vz;
        a[3] += vx * vx + vy * vy + vz * vz;
    }
}

// E4 not null: the block copies its tile's box of E4 to shared memory at
// each change of tile and gathers there (see pd_one).  B > 0: every tile box
// is B slots long on each axis (see cic::box_row).
template <bool DIAG, bool EXT, bool MAG, bool FIXED, int B>
__global__ void __launch_bounds__(PIC_PD_THREADS, PIC_PD_MIN_BLOCKS) k_push_deposit(Geom g, PushConst pc, Ctrl *ctrl,
                                                          const int4 *__restrict__ items,
                                                          const float4 *__restrict__ E4,
                                                          const float4 *__restrict__ E8,
                                                          float *rho, unsigned long long *rho64,
                                                          float qscale, int sparse_below,
                                                          double *__restrict__ part,
                                                          SaveY save) {
    extern __shared__ __align__(16) uint32_t acc[];
    const ParticleSet ps = ctrl->sets[ctrl->cur];
    const int n_items = ctrl->n_items;
    float a[4] = {0.f, 0.f, 0.f, 0.f};
    double dm[4] = {0.0, 0.0, 0.0, 0.0};
    int bad = 0;
    unsigned long long strays = 0;
    // a contiguous run of work items per block (consecutive items share tiles)
    int it0, it1;
    item_run(items, n_items, it0, it1);
    const int S = cic::tile_of(g, 0).S;
    void *sum = reinterpret_cast<char *>(acc) + cic::sum_offset(S);
    float4 *sE = reinterpret_cast<float4 *>(reinterpret_cast<char *>(acc) + cic::stage_offset(S));
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        acc[s] = 0u;
        if (FIXED) reinterpret_cast<unsigned long long *>(sum)[s] = 0ull;
        else reinterpret_cast<float *>(sum)[s] = 0.0f;
    }
    __syncthreads();
    // t: the tile of the dense items (sparse items deposit and gather globally)
    int cur_tile = -1;
    cic::Tile t = cic::tile_of(g, 0);
    for (int it = it0; it < it1; ++it) {
        const int4 item = items[it];
        const bool sparse = item.z - item.y < sparse_below;
        if (!sparse && item.x != cur_tile) {
            if (cur_tile >= 0) cic::tile_flush_sum<FIXED>(sum, t, g, rho, rho64, qscale);
            cur_tile = item.x;
            t = cic::tile_of(g, item.x);
            if (E4 != nullptr) {
                // every read of the previous box ended at the item's last barrier
                cic::stage_box(sE, E4, t, g);
                __syncthreads();
            }
        }
        const float4 *sEi = (E4 != nullptr && !sparse) ? sE : nullptr;
        // one particle per thread and iteration (coalesced 4-byte streams);
        // the next iteration's particle is loaded before this one is pushed
        int p = item.y + threadIdx.x;
        int32_t nc = 0;
        float nfx = 0.f, nfy = 0.f, nfz = 0.f, nvx = 0.f, nvy = 0.f, nvz = 0.f;
        if (p < item.z) {
            nc = __ldcs(ps.cell + p);
            nfx = __ldcs(ps.o[0] + p); nfy = __ldcs(ps.o[1] + p); nfz = __ldcs(ps.o[2] + p);
            nvx = __ldcs(ps.v[0] + p); nvy = __ldcs(ps.v[1] + p); nvz = __ldcs(ps.v[2] + p);
        }
        for (; p < item.z; p += blockDim.x) {
            int32_t c = nc;
            float fx = nfx, fy = nfy, fz = nfz, vx = nvx, vy = nvy, vz = nvz;
            const int pn = p + (int)blockDim.x;
            if (pn < item.z) {
                nc = __ldcs(ps.cell + pn);
                nfx = __ldcs(ps.o[0] + pn); nfy = __ldcs(ps.o[1] + pn); nfz = __ldcs(ps.o[2] + pn);
                nvx = __ldcs(ps.v[0] + pn); nvy = __ldcs(ps.v[1] + pn); nvz = __ldcs(ps.v[2] + pn);
            }
            if (save.cell) {
                __stcs(save.cell + p, c);
                __stcs(save.o[0] + p, fx);
                __stcs(save.o[1] + p, fy);
                __stcs(save.o[2] + p, fz);
                if (save.v[0]) {
                    __stcs(save.v[0] + p, vx);
                    __stcs(save.v[1] + p, vy);
                    __stcs(save.v[2] + p, vz);
                }
            }
            pd_one<DIAG, EXT, MAG, FIXED, B>(g, pc, E8, sEi, sparse, acc, t, rho, rho64, qscale, c,
                                          fx, fy, fz, vx, vy, vz, bad, strays, a);
            __stcs(ps.cell + p, c);
            __stcs(ps.o[0] + p, fx);
            __stcs(ps.o[1] + p, fy);
            __stcs(ps.o[2] + p, fz);
            __stcs(ps.v[0] + p, vx);
            __stcs(ps.v[1] + p, vy);
            __stcs(ps.v[2] + p, vz);
        }
        if (DIAG) fold_moments(a, dm);
        if (!sparse) {
            __syncthreads();
            cic::tile_fold<FIXED>(acc, sum, S);
            __syncthreads();
        }
    }
    if (cur_tile >= 0) cic::tile_flush_sum<FIXED>(sum, t, g, rho, rho64, qscale);
    if (bad) raise_flag(ctrl, bad);
    if (strays) {
        atomicAdd(&ctrl->stray, strays);
        atomicAdd(&ctrl->stray_step, strays);
    }
    if (DIAG) {
        const double *d = dm;
        __shared__ double red[4][PIC_PD_THREADS / 32];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        for (int q = 0; q < 4; ++q) {
            double tt = d[q];
            for (int o = 16; o > 0; o >>= 1) tt += __shfl_down_sync(0xffffffffu, tt, o);
            if (lane == 0) red[q][wid] = tt;
        }
        __syncthreads();
        if (threadIdx.x < 4) {
            double tt = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tt += red[threadIdx.x][w];
            part[4 * blockIdx.x + threadIdx.x] = tt;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctrl->step += 1;
        ctrl->since_sort += 1;
    }
}


}  // namespace

cudaError_t launch_load(const double *x, const double *v, int64_t m, int64_t base, const Geom &g,
                        const double *inv_h_d, double dt, Ctrl *ctrl, cudaStream_t st,
                        int max_blocks) {
    if (m <= 0) return cudaSuccess;
    const int T = kLoadThreads;
    int64_t B = (m + T - 1) / T;
    if (max_blocks > 0) B = std::min<int64_t>(B, max_blocks);
    k_load<<<(unsigned)B, T, 0, st>>>(x, v, m, base, g, inv_h_d[0], inv_h_d[1], inv_h_d[2], dt,
                                      ctrl);
    return cudaGetLastError();
}

// Device-to-device copy of up to 8 arrays in one launch (16-byte vectors; the
// byte tail of each array by the first threads).  Copies inside the arena run
// on the SMs at HBM speed rather than through a copy engine.
__global__ void __launch_bounds__(256) k_copy(CopyList cl) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int a = 0; a < cl.count; ++a) {
        const int64_t n16 = cl.bytes[a] >> 4;
        const uint4 *src = reinterpret_cast<const uint4 *>(cl.src[a]);
        uint4 *dst = reinterpret_cast<uint4 *>(cl.dst[a]);
        for (int64_t q = t0; q < n16; q += stride) dst[q] = src[q];
        const int64_t rem = cl.bytes[a] & 15;
        if (t0 < rem) cl.dst[a][(n16 << 4) + t0] = cl.src[a][(n16 << 4) + t0];
    }
}

cudaError_t launch_copy(const CopyList &cl, cudaStream_t st) {
    int64_t total = 0;
    for (int a = 0; a < cl.count; ++a) {
        if ((reinterpret_cast<uintptr_t>(cl.dst[a]) | reinterpret_cast<uintptr_t>(cl.src[a])) & 15)
            return cudaErrorMisalignedAddress;
        total += cl.bytes[a] >> 4;
    }
    if (total == 0 && cl.count == 0) return cudaSuccess;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 8));
    k_copy<<<blocks, 256, 0, st>>>(cl);
    return cudaGetLastError();
}

__global__ void k_pid_positions(int64_t n, const int32_t *__restrict__ pid, int32_t *pos) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) pos[pid[p]] = (int32_t)p;
}

cudaError_t launch_pid_positions(int64_t n, const int32_t *pid, int32_t *pos, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_pid_positions<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, pid, pos);
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
    const int T = kLoadThreads;
    k_unload<<<(unsigned)((m + T - 1) / T), T, 0, st>>>(o0, m, inv, g, h_d[0], h_d[1], h_d[2],
                                                        L_d[0], L_d[1], L_d[2], dt, ctrl, x, v);
    return cudaGetLastError();
}

cudaError_t launch_gather_push(int64_t n, const Geom &g, const PushConst &pc, bool diag,
                               Ctrl *ctrl, const float4 *E8, double *part, int blocks,
                               int threads, cudaStream_t st) {
    const bool ext = pc.wz2 != 0.0f;
    const bool mag = pc.t[0] != 0.0f || pc.t[1] != 0.0f || pc.t[2] != 0.0f;
#define PIC_GP(D, X, M) k_gather_push<D, X, M><<<blocks, threads, 0, st>>>(n, g, pc, ctrl, E8, part)
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

namespace pic {

// ---------------------------------------------------------------------------
// uniform plasma test (Section 4.4): random displacements instead of the push
// ---------------------------------------------------------------------------

// c-th output (c >= 1) of the SplitMix64 generator seeded with `seed`
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t c) {
    uint64_t z = seed + c * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// displacement along axis d (in cells, in [-1, 1)) of particle pid in step n:
// 2u - 1 with u = the top 24 bits of output ((n 2^32 + pid) 4 + d + 1)
__device__ __forceinline__ float move_cells(uint64_t seed, long long n, int32_t pid, int d) {
    const uint64_t c = (((uint64_t)n << 32) + (uint64_t)(uint32_t)pid) * 4ull + (uint64_t)d + 1ull;
    const uint32_t r = (uint32_t)(splitmix64(seed, c) >> 40);
    return (float)r * (1.0f / 8388608.0f) - 1.0f;   // exact: r < 2^24
}

__device__ __forceinline__ void move_one(const Geom &g, uint64_t seed, long long n, int32_t pid,
                                         int32_t &c, float &fx, float &fy, float &fz, int &bad) {
    int i, j, k;
    decode_base(g, c, i, j, k, bad);
    advance_cells(g, fx + move_cells(seed, n, pid, 0), fy + move_cells(seed, n, pid, 1),
                  fz + move_cells(seed, n, pid, 2), i, j, k, c, fx, fy, fz, bad);
}

template <bool DIAG>
__device__ __forceinline__ void block_moments(const double (&d)[4], double *part) {
    if (!DIAG) return;
    __shared__ double red[4][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int q = 0; q < 4; ++q) {
        double tt = d[q];
        for (int o = 16; o > 0; o >>= 1) tt += __shfl_down_sync(0xffffffffu, tt, o);
        if (lane == 0) red[q][wid] = tt;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double tt = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tt += red[threadIdx.x][w];
        part[4 * blockIdx.x + threadIdx.x] = tt;
    }
}

// the random move of every particle with the deposit of the new positions
// (the work items and shared tiles of k_push_deposit); velocities untouched.
// B > 0: every tile box is B slots long on each axis (see cic::box_row).
template <bool DIAG, bool FIXED, int B>
__global__ void __launch_bounds__(256, PIC_MV_MIN_BLOCKS) k_move_deposit(
    Geom g, uint64_t seed, Ctrl *ctrl, const int4 *__restrict__ items, float *rho,
    unsigned long long *rho64, float qscale, int sparse_below, double *__restrict__ part) {
    extern __shared__ __align__(16) uint32_t acc[];
    const ParticleSet ps = ctrl->sets[ctrl->cur];
    const int n_items = ctrl->n_items;
    const long long n = ctrl->step;   // advanced after this kernel (k_step_inc)
    float a[4] = {0.f, 0.f, 0.f, 0.f};
    double dm[4] = {0.0, 0.0, 0.0, 0.0};
    int bad = 0;
    unsigned long long strays = 0;
    int it0, it1;
    item_run(items, n_items, it0, it1);
    const int S = cic::tile_of(g, 0).S;
    void *sum = reinterpret_cast<char *>(acc) + cic::sum_offset(S);
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        acc[s] = 0u;
        if (FIXED) reinterpret_cast<unsigned long long *>(sum)[s] = 0ull;
        else reinterpret_cast<float *>(sum)[s] = 0.0f;
    }
    __syncthreads();
    // t: the tile of the dense items (sparse items deposit globally)
    int cur_tile = -1;
    cic::Tile t = cic::tile_of(g, 0);
    for (int it = it0; it < it1; ++it) {
        const int4 item = items[it];
        const bool sparse = item.z - item.y < sparse_below;
        if (!sparse && item.x != cur_tile) {
            if (cur_tile >= 0) cic::tile_flush_sum<FIXED>(sum, t, g, rho, rho64, qscale);
            cur_tile = item.x;
            t = cic::tile_of(g, item.x);
        }
        // the next particle's streams are loaded before the current one moves
        int p = item.y + threadIdx.x;
        int32_t nc = 0, npid = 0;
        float nfx = 0.f, nfy = 0.f, nfz = 0.f;
        if (p < item.z) {
            nc = __ldcs(ps.cell + p);
            nfx = __ldcs(ps.o[0] + p); nfy = __ldcs(ps.o[1] + p); nfz = __ldcs(ps.o[2] + p);
            npid = ps.pid[p];
        }
        for (; p < item.z; p += blockDim.x) {
            int32_t c = nc;
            float fx = nfx, fy = nfy, fz = nfz;
            const int32_t pid = npid;
            const int pn = p + (int)blockDim.x;
            if (pn < item.z) {
                nc = __ldcs(ps.cell + pn);
                nfx = __ldcs(ps.o[0] + pn); nfy = __ldcs(ps.o[1] + pn); nfz = __ldcs(ps.o[2] + pn);
                npid = ps.pid[pn];
            }
            move_one(g, seed, n, pid, c, fx, fy, fz, bad);
            const int i = cell_i(c), j = cell_j(c), k = cell_k(c);
            if (sparse) {
                float w[8];
                cic::weights(fx, fy, fz, w);
                cic::deposit_global<FIXED>(rho, rho64, g, i, j, k, w, fx, fy, fz, qscale);
            } else if (!cic::tile_add<FIXED, B>(acc, t, g, i, j, k, fx, fy, fz, rho, rho64, qscale)) {
                ++strays;
            }
            if (DIAG) {
                const float vx = ps.v[0][p], vy = ps.v[1][p], vz = ps.v[2][p];
                a[0] += vx;
                a[1] += vy;
                a[2] += vz;
                a[3] += vx * vx + vy * vy + vz * vz;
            }
            __stcs(ps.cell + p, c);
            __stcs(ps.o[0] + p, fx);
            __stcs(ps.o[1] + p, fy);
            __stcs(ps.o[2] + p, fz);
        }
        if (DIAG) fold_moments(a, dm);
        if (!sparse) {
            __syncthreads();
            cic::tile_fold<FIXED>(acc, sum, S);
            __syncthreads();
        }
    }
    if (cur_tile >= 0) cic::tile_flush_sum<FIXED>(sum, t, g, rho, rho64, qscale);
    if (bad) raise_flag(ctrl, bad);
    if (strays) {
        atomicAdd(&ctrl->stray, strays);
        atomicAdd(&ctrl->stray_step, strays);
    }
    block_moments<DIAG>(dm, part);
}

// the random move alone (split calls: pic_gather_push)
template <bool DIAG>
__global__ void __launch_bounds__(256) k_move(int64_t np, Geom g, uint64_t seed, Ctrl *ctrl,
                                               double *__restrict__ part) {
    const ParticleSet ps = ctrl->sets[ctrl->cur];
    const long long n = ctrl->step;
    float a[4] = {0.f, 0.f, 0.f, 0.f};
    double dm[4] = {0.0, 0.0, 0.0, 0.0};
    int bad = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += stride) {
        int32_t c = ps.cell[p];
        float fx = ps.o[0][p], fy = ps.o[1][p], fz = ps.o[2][p];
        move_one(g, seed, n, ps.pid[p], c, fx, fy, fz, bad);
        ps.cell[p] = c;
        ps.o[0][p] = fx;
        ps.o[1][p] = fy;
        ps.o[2][p] = fz;
        if (DIAG) {
            const float vx = ps.v[0][p], vy = ps.v[1][p], vz = ps.v[2][p];
            a[0] += vx;
            a[1] += vy;
            a[2] += vz;
            a[3] += vx * vx + vy * vy + vz * vz;
            fold_moments(a, dm);
        }
    }
    if (bad) raise_flag(ctrl, bad);
    block_moments<DIAG>(dm, part);
}

__global__ void k_step_inc(Ctrl *ctrl) {
    ctrl->step += 1;
    ctrl->since_sort += 1;
}

// the box edge compiled as a constant into the fixed-point push and move:
// 8^3 tiles with two guard layers (the default geometry)
constexpr int kConstBox = 13;
bool const_box(const Geom &g) {
    for (int d = 0; d < 3; ++d)
        if (g.tile[d] + 2 * g.guard + 1 != kConstBox) return false;
    return true;
}

cudaError_t launch_move(int64_t np, const Geom &g, uint64_t seed, bool diag, bool fixed, bool deposit,
                        Ctrl *ctrl, const int4 *items, int max_items, float *rho,
                        unsigned long long *rho64, double qscale, int sparse_below, double *part,
                        int blocks, cudaStream_t st) {
    const int nb = std::max(1, std::min(blocks, deposit ? max_items : blocks));
    if (deposit) {
        const size_t smem = tile_deposit_smem(g);
        const float qs = (float)qscale;
        const bool cbox = const_box(g);
#define PIC_MV(D, F, B) \
    k_move_deposit<D, F, B><<<nb, 256, smem, st>>>(g, seed, ctrl, items, rho, rho64, qs, sparse_below, part)
        if (diag) {
            if (!fixed) PIC_MV(true, false, 0);
            else if (cbox) PIC_MV(true, true, kConstBox);
            else PIC_MV(true, true, 0);
        } else {
            if (!fixed) PIC_MV(false, false, 0);
            else if (cbox) PIC_MV(false, true, kConstBox);
            else PIC_MV(false, true, 0);
        }
#undef PIC_MV
    } else {
        if (diag) k_move<true><<<nb, 256, 0, st>>>(np, g, seed, ctrl, part);
        else k_move<false><<<nb, 256, 0, st>>>(np, g, seed, ctrl, part);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_step_inc<<<1, 1, 0, st>>>(ctrl);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return (deposit && fixed) ? launch_rho_finish(g, rho64, rho, qscale, st) : cudaSuccess;
}

// item tile + the block's tile sums
size_t tile_deposit_smem(const Geom &g) {
    const cic::Tile t0 = cic::tile_of(g, 0);
    return cic::sum_offset(t0.S) + 8 * (size_t)t0.S;
}
// staged field: the box's float4 slots after the deposit tiles, if
// PIC_PD_MIN_BLOCKS such blocks (plus the kernel's static shared memory and
// the runtime's 1 KiB per block) fit in an SM's 228 KiB
bool push_stages_E(const Geom &g) {
#if PIC_PD_STAGE_E
    const int S = cic::tile_of(g, 0).S;
    const size_t per_block = cic::stage_offset(S) + 16 * (size_t)S + 256 + 1024;
    return per_block * PIC_PD_MIN_BLOCKS <= (size_t)228 * 1024;
#else
    (void)g;
    return false;
#endif
}
size_t push_deposit_smem(const Geom &g) {
    const int S = cic::tile_of(g, 0).S;
    return push_stages_E(g) ? cic::stage_offset(S) + 16 * (size_t)S : tile_deposit_smem(g);
}

// Allow the fused kernels' shared memory (call outside any stream capture)
cudaError_t push_deposit_prepare(const Geom &g) {
    cudaError_t e = cudaSuccess;
    const size_t tsm = tile_deposit_smem(g);
    if (tsm > 48 * 1024) {
#define PIC_MVA(D, F, B)                                                                       \
        if ((e = cudaFuncSetAttribute(k_move_deposit<D, F, B>,                                  \
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm)) != \
            cudaSuccess)                                                                        \
            return e
        PIC_MVA(false, false, 0); PIC_MVA(false, true, 0); PIC_MVA(true, false, 0);
        PIC_MVA(true, true, 0); PIC_MVA(false, true, kConstBox); PIC_MVA(true, true, kConstBox);
#undef PIC_MVA
    }
    const size_t smem = push_deposit_smem(g);
    if (smem <= 48 * 1024) return cudaSuccess;
#define PIC_PDA(D, X, M, F, B)                                                                \
    if ((e = cudaFuncSetAttribute(k_push_deposit<D, X, M, F, B>,                              \
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != \
        cudaSuccess)                                                                          \
        return e
#define PIC_PDA2(D, X, M) \
    PIC_PDA(D, X, M, false, 0); PIC_PDA(D, X, M, true, 0); PIC_PDA(D, X, M, true, kConstBox)
    PIC_PDA2(false, false, false); PIC_PDA2(false, false, true);
    PIC_PDA2(false, true, false);  PIC_PDA2(false, true, true);
    PIC_PDA2(true, false, false);  PIC_PDA2(true, false, true);
    PIC_PDA2(true, true, false);   PIC_PDA2(true, true, true);
#undef PIC_PDA2
#undef PIC_PDA
    return cudaSuccess;
}

cudaError_t launch_push_deposit(const Geom &g, const PushConst &pc, bool diag, bool fixed,
                                Ctrl *ctrl, const int4 *items, int max_items, const float4 *E4,
                                const float4 *E8, float *rho, unsigned long long *rho64,
                                double qscale, int sparse_below, double *part, int blocks,
                                const SaveY &save, cudaStream_t st) {
    const bool ext = pc.wz2 != 0.0f;
    const bool mag = pc.t[0] != 0.0f || pc.t[1] != 0.0f || pc.t[2] != 0.0f;
    const size_t smem = push_deposit_smem(g);
    const float4 *E4s = push_stages_E(g) ? E4 : nullptr;
    const int nb = std::max(1, std::min(blocks, max_items));
    const float qs = (float)qscale;
    cudaError_t e = cudaSuccess;
    const bool cbox = const_box(g);
#define PIC_PD(D, X, M, F, B)                                                                   \
    k_push_deposit<D, X, M, F, B><<<nb, PIC_PD_THREADS, smem, st>>>(g, pc, ctrl, items, E4s, E8, \
                                                                    rho, rho64, qs,             \
                                                                    sparse_below, part, save)
#define PIC_PD_F(D, X, M)                                  \
    do {                                                   \
        if (!fixed) PIC_PD(D, X, M, false, 0);             \
        else if (cbox) PIC_PD(D, X, M, true, kConstBox);   \
        else PIC_PD(D, X, M, true, 0);                     \
    } while (0)
    if (diag) {
        if (ext) { if (mag) PIC_PD_F(true, true, true); else PIC_PD_F(true, true, false); }
        else     { if (mag) PIC_PD_F(true, false, true); else PIC_PD_F(true, false, false); }
    } else {
        if (ext) { if (mag) PIC_PD_F(false, true, true); else PIC_PD_F(false, true, false); }
        else     { if (mag) PIC_PD_F(false, false, true); else PIC_PD_F(false, false, false); }
    }
#undef PIC_PD_F
#undef PIC_PD
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return fixed ? launch_rho_finish(g, rho64, rho, qscale, st) : cudaSuccess;
}

}  // namespace pic
