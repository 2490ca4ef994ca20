// Batched ensembles: many independent PIC runs (different grids, particle
// counts, charges) advanced by one set of launches per phase.
//
// Every instance keeps the scheme of the single-run path (Section 3.1 steps
// 1-4 and Section 3.2 of arXiv 2205.11052); what changes is only where its
// data lives:
//  * particles of instance i occupy [p0_i, p0_i + np_i) of one shared SoA
//    store (binning keys are global tile ids, tile0_i + local tile, which are
//    ordered by instance, so sorting never moves a particle out of its range);
//  * its grids occupy nodes [g0_i, g0_i + ng_i) of the concatenated rho, rho64
//    and E arrays, instances of equal grid size (a size class) adjacent so a
//    batched cuFFT plan covers the class;
//  * a work item (global tile, particle range) names its instance through the
//    tile -> instance table, so one persistent push + deposit launch walks the
//    work of every instance.
#include <algorithm>

#include "batch.cuh"
#include "cic.cuh"
#include "push.cuh"
#include "sort_staged.cuh"

namespace pic {

namespace {

// instance owning particle p: binary search over the particle offsets
__device__ __forceinline__ int inst_of_particle(const long long *__restrict__ p0, int n_inst,
                                                long long p) {
    int lo = 0, hi = n_inst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p0[mid] <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void k_b_load(const double *__restrict__ x, const double *__restrict__ v, int64_t m,
                         int64_t base, const InstDesc *__restrict__ desc,
                         const long long *__restrict__ p0, int n_inst, double dt, Ctrl *ctrl) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= m) return;
    const int64_t p = base + q;
    const InstDesc &D = desc[inst_of_particle(p0, n_inst, p)];
    const ParticleSet ps = ctrl->sets[ctrl->cur];
    int idx[3];
    float off[3];
    bool ok = true;
    for (int d = 0; d < 3; ++d) {
        const double vd = v[3 * q + d];
        double s = (x[3 * q + d] + 0.5 * dt * vd) * D.inv_h_d[d] - 0.5;
        if (!isfinite(s) || !isfinite(vd) || fabs(s) > 4.0e15) {
            ok = false;
            s = 0.0;
        }
        const double fl = floor(s);
        long long il = (long long)fl % D.g.n[d];
        if (il < 0) il += D.g.n[d];
        float ff = (float)(s - fl);
        if (ff >= 1.0f) {
            ff = 0.0f;
            if (++il == D.g.n[d]) il = 0;
        }
        idx[d] = (int)il;
        off[d] = ff;
        ps.v[d][p] = ok ? (float)vd : 0.0f;
    }
    if (!ok) atomicOr(&ctrl->flags, PIC_FLAG_NONFINITE);
    ps.cell[p] = pack_cell(idx[0], idx[1], idx[2]);
    ps.o[0][p] = off[0];
    ps.o[1][p] = off[1];
    ps.o[2][p] = off[2];
    ps.pid[p] = (int32_t)p;
}

__global__ void k_b_unload(int64_t o0, int64_t m, const int32_t *__restrict__ inv,
                           const InstDesc *__restrict__ desc, const long long *__restrict__ p0,
                           int n_inst, double dt, const Ctrl *ctrl, double *__restrict__ x,
                           double *__restrict__ v) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= m) return;
    const ParticleSet ps = ctrl->sets[ctrl->cur];
    const int64_t p = inv[o0 + q];
    const InstDesc &D = desc[inst_of_particle(p0, n_inst, p)];
    const int32_t c = ps.cell[p];
    const int idx[3] = {cell_i(c), cell_j(c), cell_k(c)};
    for (int d = 0; d < 3; ++d) {
        const double vd = (double)ps.v[d][p];
        double xd = ((double)idx[d] + 0.5 + (double)ps.o[d][p]) * D.h_d[d] - 0.5 * dt * vd;
        xd -= D.L_d[d] * floor(xd / D.L_d[d]);
        if (xd >= D.L_d[d]) xd -= D.L_d[d];
        if (xd < 0.0) xd = 0.0;
        x[3 * q + d] = xd;
        v[3 * q + d] = vd;
    }
}

__device__ __forceinline__ int b_key(int32_t c, const InstDesc &D, int &bad) {
    int i = cell_i(c), j = cell_j(c), k = cell_k(c);
    if (i >= D.g.n[0] || j >= D.g.n[1] || k >= D.g.n[2]) {
        bad = 1;
        i = j = k = 0;
    }
    const int ti = tile_div(i, D.g.tdiv[0]), tj = tile_div(j, D.g.tdiv[1]);
    const int tk = tile_div(k, D.g.tdiv[2]);
    return D.tile0 + ti + D.g.ntile[0] * (tj + D.g.ntile[1] * tk);
}

__device__ __forceinline__ void b_slice(int64_t n, int64_t &b0, int64_t &b1) {
    const int64_t per = ((n + gridDim.x - 1) / gridDim.x + blockDim.x - 1) / blockDim.x * blockDim.x;
    b0 = (int64_t)blockIdx.x * per;
    b1 = b0 + per < n ? b0 + per : n;
}

// binning key of particle p: the global tile id of its instance's tile.  A
// thread's copy remembers the particle range of the last instance it looked
// up (a thread meets consecutive particles of one instance), so the binary
// search runs only when p leaves it.
struct BatchKey {
    const InstDesc *desc;
    const long long *p0;
    int n_inst;
    mutable long long lo = 0, hi = 0;
    mutable int inst = 0;
    __device__ __forceinline__ int operator()(int32_t c, int64_t p, int &bad) const {
        if (p < lo || p >= hi) {
            inst = inst_of_particle(p0, n_inst, p);
            lo = p0[inst];
            hi = p0[inst + 1];
        }
        return b_key(c, desc[inst], bad);
    }
};

// Work items (instance tile, particle range) in contiguous runs per block:
// the deposit of the instance's tile and (PUSH) the gather + push before it.
// Each item's tile accumulates in shared memory (u32 fixed point, or FP32
// bits) and is folded into a 64-bit per-tile sum after the item; the sum is
// flushed to the instance's grid when the block moves to another tile, so
// consecutive items of one tile cost one flush.  With DIAG each item leaves
// its FP32 particle moments, summed in FP64 in a fixed order, in part[item].
template <bool PUSH, bool DIAG, bool EXT, bool MAG, bool FIXED>
__global__ void __launch_bounds__(256, PIC_BATCH_PD_MIN_BLOCKS) k_b_push_deposit(
    const InstDesc *__restrict__ desc, const int32_t *__restrict__ tile_inst, Ctrl *ctrl,
    const int4 *__restrict__ items, const float4 *__restrict__ E4, const float4 *__restrict__ E8,
    float *rho, unsigned long long *rho64, int sparse_below, int max_S,
    double *__restrict__ part) {
    extern __shared__ __align__(16) uint32_t acc[];
    __shared__ double red[4][8];
    void *sum = reinterpret_cast<char *>(acc) + cic::sum_offset(max_S);
    float4 *sE = reinterpret_cast<float4 *>(reinterpret_cast<char *>(acc) + cic::stage_offset(max_S));
    const ParticleSet ps = ctrl->sets[ctrl->cur];
    const int n_items = ctrl->n_items;
    int it0, it1;
    item_run(items, n_items, it0, it1);
    for (int s = threadIdx.x; s < max_S; s += blockDim.x) {
        acc[s] = 0u;
        if (FIXED) reinterpret_cast<unsigned long long *>(sum)[s] = 0ull;
        else reinterpret_cast<float *>(sum)[s] = 0.0f;
    }
    __syncthreads();
    int bad = 0;
    int cur_tile = -1;
    const InstDesc *Dc = desc;
    cic::Tile tc{};
    for (int it = it0; it < it1; ++it) {
        const int4 item = items[it];
        const InstDesc &D = desc[tile_inst[item.x]];
        const Geom g = D.g;
        const PushConst pc = D.pc;
        const float4 *Ei = E8 + 2 * D.g0;
        float *rhoi = rho + D.g0;
        unsigned long long *rho64i = rho64 + D.g0;
        const float qscale = D.qscale;
        const bool sparse = item.z - item.y < sparse_below;
        const cic::Tile t = cic::tile_of(g, item.x - D.tile0);
        if (!sparse && item.x != cur_tile) {
            if (cur_tile >= 0)
                cic::tile_flush_sum<FIXED>(sum, tc, Dc->g, rho + Dc->g0, rho64 + Dc->g0, Dc->qscale);
            cur_tile = item.x;
            tc = t;
            Dc = &D;
            if (PUSH && E4 != nullptr) {
                // every read of the previous box ended at the item's last barrier
                cic::stage_box(sE, E4 + D.g0, t, g);
                __syncthreads();
            }
        }
        const float4 *sEi = (PUSH && E4 != nullptr && !sparse) ? sE : nullptr;
        float a[4] = {0.f, 0.f, 0.f, 0.f};
        // the next particle's streams are loaded before the current one is pushed
        int p = item.y + threadIdx.x;
        int32_t nc = 0;
        float nfx = 0.f, nfy = 0.f, nfz = 0.f, nvx = 0.f, nvy = 0.f, nvz = 0.f;
        if (p < item.z) {
            nc = __ldcs(ps.cell + p);
            nfx = __ldcs(ps.o[0] + p); nfy = __ldcs(ps.o[1] + p); nfz = __ldcs(ps.o[2] + p);
            if (PUSH) {
                nvx = __ldcs(ps.v[0] + p); nvy = __ldcs(ps.v[1] + p); nvz = __ldcs(ps.v[2] + p);
            }
        }
        for (; p < item.z; p += blockDim.x) {
            int32_t c = nc;
            float fx = nfx, fy = nfy, fz = nfz;
            const float cvx = nvx, cvy = nvy, cvz = nvz;
            {
                const int pn = p + (int)blockDim.x;
                if (pn < item.z) {
                    nc = __ldcs(ps.cell + pn);
                    nfx = __ldcs(ps.o[0] + pn); nfy = __ldcs(ps.o[1] + pn); nfz = __ldcs(ps.o[2] + pn);
                    if (PUSH) {
                        nvx = __ldcs(ps.v[0] + pn); nvy = __ldcs(ps.v[1] + pn);
                        nvz = __ldcs(ps.v[2] + pn);
                    }
                }
            }
            int i, j, k;
            if (PUSH) {
                float vx = cvx, vy = cvy, vz = cvz;
                push_one_staged<EXT, MAG>(g, pc, Ei, sEi, t, c, fx, fy, fz, vx, vy, vz, bad, i, j,
                                          k);
                __stcs(ps.cell + p, c);
                __stcs(ps.o[0] + p, fx);
                __stcs(ps.o[1] + p, fy);
                __stcs(ps.o[2] + p, fz);
                __stcs(ps.v[0] + p, vx);
                __stcs(ps.v[1] + p, vy);
                __stcs(ps.v[2] + p, vz);
                if (DIAG) {
                    a[0] += vx;
                    a[1] += vy;
                    a[2] += vz;
                    a[3] += vx * vx + vy * vy + vz * vz;
                }
            }
            if (!PUSH && !cic::decode_cell(c, g, i, j, k)) bad |= PIC_FLAG_BAD_CELL;
            if (sparse) {
                float w[8];
                cic::weights(fx, fy, fz, w);
                cic::deposit_global<FIXED>(rhoi, rho64i, g, i, j, k, w, fx, fy, fz, qscale);
            } else {
                cic::tile_add<FIXED>(acc, t, g, i, j, k, fx, fy, fz, rhoi, rho64i, qscale);
            }
        }
        if (!sparse) {
            __syncthreads();
            cic::tile_fold<FIXED>(acc, sum, t.S);
            __syncthreads();
        }
        if (DIAG) {
            const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
            for (int q = 0; q < 4; ++q) {
                double tt = (double)a[q];
                for (int o = 16; o > 0; o >>= 1) tt += __shfl_down_sync(0xffffffffu, tt, o);
                if (lane == 0) red[q][wid] = tt;
            }
            __syncthreads();
            if (threadIdx.x < 4) {
                double tt = 0.0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tt += red[threadIdx.x][w];
                part[4 * (int64_t)it + threadIdx.x] = tt;
            }
            __syncthreads();
        }
    }
    if (cur_tile >= 0)
        cic::tile_flush_sum<FIXED>(sum, tc, Dc->g, rho + Dc->g0, rho64 + Dc->g0, Dc->qscale);
    if (bad) atomicOr(&ctrl->flags, bad);
}

// integer grid -> charge density of each node's instance; clears rho64
__global__ void k_b_rho_finish(int64_t ng, const InstDesc *__restrict__ desc,
                               const long long *__restrict__ g0, int n_inst,
                               unsigned long long *__restrict__ rho64, float *__restrict__ rho) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int inst = 0;
    for (int64_t gidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gidx < ng; gidx += stride) {
        inst = inst_of_particle(g0, n_inst, gidx);
        const double scale = desc[inst].qscale_d * (1.0 / (double)cic::kFixOne);
        rho[gidx] = (float)((double)(long long)rho64[gidx] * scale);
        rho64[gidx] = 0ull;
    }
}

// Green kernel of one size class: m instances with equal grids; instance j of
// the class is desc[first + j], its half spectrum rho_hat[j * nhalf ...]
__global__ void k_b_green(const InstDesc *__restrict__ desc, int first, int m, int64_t nhalf,
                          const float2 *__restrict__ rho_hat, float2 *__restrict__ E_hat,
                          double *__restrict__ modes) {
    const int64_t qq = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (qq >= (int64_t)m * nhalf) return;
    const int j = (int)(qq / nhalf);
    const int64_t q = qq - (int64_t)j * nhalf;
    const InstDesc &D = desc[first + j];
    const int nx = D.g.n[0], ny = D.g.n[1], nz = D.g.n[2], nh = D.g.nh;
    const int a = (int)(q % nh);
    const int64_t r = q / nh;
    const int b = (int)(r % ny);
    const int c = (int)(r / ny);
    const int my = (b <= ny / 2) ? b : b - ny;
    const int mz = (c <= nz / 2) ? c : c - nz;
    const float kx = (float)(D.two_pi_over_L[0] * a), ky = (float)(D.two_pi_over_L[1] * my);
    const float kz = (float)(D.two_pi_over_L[2] * mz);
    const float gx = ((nx & 1) == 0 && a == nx / 2) ? 0.0f : kx;
    const float gy = ((ny & 1) == 0 && b == ny / 2) ? 0.0f : ky;
    const float gz = ((nz & 1) == 0 && c == nz / 2) ? 0.0f : kz;
    float2 ex = make_float2(0.f, 0.f), ey = ex, ez = ex;
    if (q != 0) {
        const float2 rh = rho_hat[qq];
        const float sc = (float)D.inv_ng / (kx * kx + ky * ky + kz * kz);
        ex = make_float2(gx * sc * rh.y, -gx * sc * rh.x);
        ey = make_float2(gy * sc * rh.y, -gy * sc * rh.x);
        ez = make_float2(gz * sc * rh.y, -gz * sc * rh.x);
    }
    const int64_t mh = (int64_t)m * nhalf;
    E_hat[qq] = ex;
    E_hat[qq + mh] = ey;
    E_hat[qq + 2 * mh] = ez;
    if (a == D.mode_idx[0] && b == D.mode_idx[1] && c == D.mode_idx[2]) {
        const float2 mv = (D.mode_comp == 0) ? ex : (D.mode_comp == 1 ? ey : ez);
        modes[2 * (first + j)] = (double)mv.x;
        modes[2 * (first + j) + 1] = D.mode_conj ? -(double)mv.y : (double)mv.y;
    }
}

// field energies and charge of one instance per block, FP64, fixed order
__global__ void __launch_bounds__(256) k_b_diag_field(const InstDesc *__restrict__ desc,
                                                      const float *__restrict__ rho,
                                                      const float4 *__restrict__ E4,
                                                      double *__restrict__ fpart) {
    const InstDesc &D = desc[blockIdx.x];
    const int64_t ng = (int64_t)D.g.n[0] * D.g.n[1] * D.g.n[2];
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t q = threadIdx.x; q < ng; q += blockDim.x) {
        const float4 e = E4[D.g0 + q];
        const double ex = e.x, ey = e.y, ez = e.z;
        s[0] += ex * ex;
        s[1] += ey * ey;
        s[2] += ez * ez;
        s[3] += (double)rho[D.g0 + q];
    }
    __shared__ double red[4][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int q = 0; q < 4; ++q) {
        double t = s[q];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) red[q][wid] = t;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[threadIdx.x][w];
        fpart[4 * blockIdx.x + threadIdx.x] = D.dV * t;
    }
}

// one record per instance: the instance's items are [item_off[tile0],
// item_off[tile0 + ntiles]) of the work list (items follow the tile order)
__global__ void k_b_diag_finalize(const InstDesc *__restrict__ desc, int n_inst,
                                  const int32_t *__restrict__ item_off,
                                  const double *__restrict__ fpart,
                                  const double *__restrict__ ppart,
                                  const double *__restrict__ modes, Ctrl *ctrl, double dt,
                                  pic_diag_t *ring, int ring_cap) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const long long step = ctrl->step;        // advanced by k_b_step_done afterwards
    const long long slot = ctrl->diag_written % ring_cap;
    if (i < n_inst) {
        const InstDesc &D = desc[i];
        double s[4] = {0.0, 0.0, 0.0, 0.0};
        for (int it = item_off[D.tile0]; it < item_off[D.tile0 + D.ntiles]; ++it)
            for (int q = 0; q < 4; ++q) s[q] += ppart[4 * (int64_t)it + q];
        pic_diag_t d;
        d.step = step;
        d.t_field = ((double)step + 0.5) * dt;
        d.Wx = fpart[4 * i];
        d.Wy = fpart[4 * i + 1];
        d.Wz = fpart[4 * i + 2];
        d.Q = fpart[4 * i + 3];
        d.mode_re = modes[2 * i];
        d.mode_im = modes[2 * i + 1];
        d.t = ((double)step + 1.0) * dt;
        d.Px = D.mp * s[0];
        d.Py = D.mp * s[1];
        d.Pz = D.mp * s[2];
        d.K = 0.5 * D.mp * s[3];
        ring[slot * n_inst + i] = d;
    }
}

// planar (Ex, Ey, Ez) of a size class -> interleaved float4 E of its instances
// planar (Ex, Ey, Ez) of a size class -> E4 and the x-paired E8 (E at q and at
// its +x neighbour; instances and rows start at multiples of nx, so the row
// position of q is q mod nx)
__global__ void k_b_pack(int64_t mng, int nx, const float *__restrict__ planar,
                         float4 *__restrict__ E4, float4 *__restrict__ E8) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < mng; q += stride) {
        const int i = (int)(q % nx);
        const int64_t q1 = (i + 1 == nx) ? q - i : q + 1;
        const float4 e = make_float4(planar[q], planar[q + mng], planar[q + 2 * mng], 0.0f);
        E4[q] = e;
        E8[2 * q] = e;
        E8[2 * q + 1] = make_float4(planar[q1], planar[q1 + mng], planar[q1 + 2 * mng], 0.0f);
    }
}

__global__ void k_b_step_done(Ctrl *ctrl, int diag) {
    ctrl->step += 1;
    if (diag) ctrl->diag_written += 1;
}

}  // namespace

cudaError_t launch_b_load(const double *x, const double *v, int64_t m, int64_t base,
                          const InstDesc *desc, const long long *p0, int n_inst, double dt,
                          Ctrl *ctrl, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    k_b_load<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(x, v, m, base, desc, p0, n_inst, dt, ctrl);
    return cudaGetLastError();
}

cudaError_t launch_b_unload(int64_t o0, int64_t m, const int32_t *inv, const InstDesc *desc,
                            const long long *p0, int n_inst, double dt, const Ctrl *ctrl,
                            double *x, double *v, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    k_b_unload<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(o0, m, inv, desc, p0, n_inst, dt, ctrl,
                                                            x, v);
    return cudaGetLastError();
}

cudaError_t launch_b_sort(int64_t n, const InstDesc *desc, const long long *p0, int n_inst,
                          int ntiles, int chunk, Ctrl *ctrl, int32_t *bins, int32_t *scan_tmp,
                          int32_t *tile_items, int2 *tile_range, int4 *items, cudaStream_t st) {
    cudaError_t e = staged_pass(n, BatchKey{desc, p0, n_inst}, ntiles, ctrl, bins, scan_tmp, st);
    if (e != cudaSuccess) return e;
    return launch_worklist(bins, ntiles, chunk, tile_items, tile_range, items, scan_tmp, ctrl,
                           n > 0 ? 1 : 0, st);
}

cudaError_t batch_sort_prepare() { return staged_prepare<BatchKey>(); }

size_t batch_push_smem(int max_S, bool staged) {
    return staged ? cic::stage_offset(max_S) + 16 * (size_t)max_S
                  : cic::sum_offset(max_S) + 8 * (size_t)max_S;
}

bool batch_stages_E(int max_S, int threads) {
#if PIC_PD_STAGE_E
    const int64_t per_sm = std::max(1, PIC_BATCH_PD_MIN_BLOCKS * 256 / std::max(1, threads));
    const size_t per_block = batch_push_smem(max_S, true) + 256 + 1024;
    return (size_t)per_sm * per_block <= (size_t)228 * 1024;
#else
    (void)max_S;
    (void)threads;
    return false;
#endif
}

cudaError_t launch_b_push_deposit(bool push, bool diag, bool ext, bool mag, bool fixed,
                                  const InstDesc *desc, const int32_t *tile_inst, Ctrl *ctrl,
                                  const int4 *items, int blocks, int threads, int max_S,
                                  const float4 *E4, const float4 *E8,
                                  float *rho, unsigned long long *rho64, int sparse_below,
                                  double *part, cudaStream_t st) {
    const size_t smem = batch_push_smem(max_S, E4 != nullptr && push);
    cudaError_t e = cudaSuccess;
#define PIC_BPD(P, D, X, M, F)                                                                  \
    do {                                                                                        \
        auto kern = k_b_push_deposit<P, D, X, M, F>;                                            \
        if (smem > 48 * 1024 &&                                                                 \
            (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,        \
                                      (int)smem)) != cudaSuccess)                               \
            return e;                                                                           \
        kern<<<blocks, threads, smem, st>>>(desc, tile_inst, ctrl, items, push ? E4 : nullptr, \
                                            E8, rho, rho64, sparse_below, max_S, part);         \
    } while (0)
#define PIC_BPD_F(P, D, X, M) \
    do { if (fixed) PIC_BPD(P, D, X, M, true); else PIC_BPD(P, D, X, M, false); } while (0)
#define PIC_BPD_M(P, D, X) \
    do { if (mag) PIC_BPD_F(P, D, X, true); else PIC_BPD_F(P, D, X, false); } while (0)
#define PIC_BPD_X(P, D) \
    do { if (ext) PIC_BPD_M(P, D, true); else PIC_BPD_M(P, D, false); } while (0)
    if (!push) PIC_BPD_F(false, false, false, false);
    else if (diag) PIC_BPD_X(true, true);
    else PIC_BPD_X(true, false);
#undef PIC_BPD_X
#undef PIC_BPD_M
#undef PIC_BPD_F
#undef PIC_BPD
    return cudaGetLastError();
}

cudaError_t launch_b_rho_finish(int64_t ng, const InstDesc *desc, const long long *g0, int n_inst,
                                unsigned long long *rho64, float *rho, cudaStream_t st) {
    const int b = (int)std::max<int64_t>(1, std::min<int64_t>((ng + 255) / 256, 152 * 8));
    k_b_rho_finish<<<b, 256, 0, st>>>(ng, desc, g0, n_inst, rho64, rho);
    return cudaGetLastError();
}

cudaError_t launch_b_green(const InstDesc *desc, int first, int m, int64_t nhalf,
                           const float2 *rho_hat, float2 *E_hat, double *modes, cudaStream_t st) {
    const int64_t tot = (int64_t)m * nhalf;
    if (tot <= 0) return cudaSuccess;
    k_b_green<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(desc, first, m, nhalf, rho_hat, E_hat,
                                                             modes);
    return cudaGetLastError();
}

cudaError_t launch_b_diag(const InstDesc *desc, int n_inst, const float *rho, const float4 *E4,
                          double *fpart, cudaStream_t st) {
    k_b_diag_field<<<n_inst, 256, 0, st>>>(desc, rho, E4, fpart);
    return cudaGetLastError();
}

cudaError_t launch_b_diag_finalize(const InstDesc *desc, int n_inst, const int32_t *item_off,
                                   const double *fpart, const double *ppart, const double *modes,
                                   Ctrl *ctrl, double dt, pic_diag_t *ring, int ring_cap,
                                   cudaStream_t st) {
    k_b_diag_finalize<<<(n_inst + 127) / 128, 128, 0, st>>>(desc, n_inst, item_off, fpart, ppart,
                                                            modes, ctrl, dt, ring, ring_cap);
    return cudaGetLastError();
}

cudaError_t launch_b_pack(int64_t mng, int nx, const float *planar, float4 *E4, float4 *E8,
                          cudaStream_t st) {
    const int b = (int)std::max<int64_t>(1, std::min<int64_t>((mng + 255) / 256, 152 * 8));
    k_b_pack<<<b, 256, 0, st>>>(mng, nx, planar, E4, E8);
    return cudaGetLastError();
}

cudaError_t launch_b_step_done(Ctrl *ctrl, bool diag, cudaStream_t st) {
    k_b_step_done<<<1, 1, 0, st>>>(ctrl, diag ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace pic
