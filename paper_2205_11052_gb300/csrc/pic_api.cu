// C ABI of the GB300 PIC library (declared in include/pic.h): configuration
// validation, arena layout, cuFFT plans and the step driver.  Every device
// operation is a launch of this library's kernels (k_*.cu), a cuFFT execution
// or a memset/memcpy, enqueued on the caller's stream.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "pic_internal.cuh"

using namespace pic;

namespace {

thread_local char g_err[512] = "no error";

int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

#define PIC_CUDA(call)                                                                  \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(PIC_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

#define PIC_CUFFT(call)                                                       \
    do {                                                                      \
        cufftResult r_ = (call);                                              \
        if (r_ != CUFFT_SUCCESS)                                              \
            return fail(PIC_ERR_CUFFT, "%s failed: cufftResult %d", #call, (int)r_); \
    } while (0)

constexpr size_t kAlign = 256;
constexpr int kTimerRing = 64;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Byte offsets of every device buffer inside the caller's arena.
struct Layout {
    size_t ctrl, sets, rho, rho64, rho_hat, E_hat, E4, E8, lrho2, bins, scan_tmp, tile_items, tile_range,
        items, fpart, ppart, ring, inv, stage_x, stage_v, adjE4, ktab, fft, total;
    size_t set_stride;   // bytes of one per-particle array
};

}  // namespace

int pic::record_error(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

// ranges a page-locked host load is split into (each binned on a side stream
// while the next is read over the host link)
constexpr int kLoadRanges = 8;
constexpr int64_t kOverlapMin = 1 << 22;   // particles below which loads are not split

struct pic_ctx {
    pic_grid_t grid;
    pic_species_t sp;
    pic_params_t prm;
    Geom geom;
    double L[3], h[3], inv_h[3], dV;
    int64_t cap, ng, nhalf, nbins, ntiles, max_items, staging;
    int chunk, block, sparse_below, deposit_blocks;
    int mode_idx[3], mode_conj;
    size_t fft_reserve;
    Layout lay;
    // bound state
    bool bound;
    char *arena;
    cudaStream_t st;
    cufftHandle r2c, c2r;     // rho -> rho^ ; 3 x E^ -> E4 (stride 4)
    cufftHandle r2c3, c2r1;   // adjoint: lE4 (stride 4) -> 3 x lE^ ; lrho^ -> lrho
    bool plans;
    ParticleSet hsets[2];     // host copies of the device set descriptors
    // state of the last pic_adjoint_forward
    struct {
        bool ready;
        int n_steps, K, nseg, cur, cur_end;
        double w[3];
        char *buf;
        int64_t step0;
        long long step0_dev;
        double pgrad[4];    // dJ/dB_ext (3), dJ/d(wz2) of the last backward pass
        bool pgrad_ready;
    } adj;
    // phase timers: a ring of event pairs per phase, drained when it wraps
    bool timing;
    bool events_made;
    cudaEvent_t ev[PIC_PHASE_COUNT][kTimerRing][2];
    int64_t ev_count[PIC_PHASE_COUNT];     // pairs recorded since enabling
    int64_t ev_drained[PIC_PHASE_COUNT];   // pairs already summed
    double ms[PIC_PHASE_COUNT];
    int64_t launches;
    // overlapped load: a second stream sorts loaded ranges while the next ones load
    bool side_made;
    cudaStream_t side;
    cudaEvent_t side_ev[kLoadRanges + 1];
    // host mirror of the run
    int64_t np;
    int64_t step;
    int since_sort;
    bool loaded;
    bool rho_current;   // rho holds the deposit of the current positions

    template <class T>
    T *at(size_t off) const { return reinterpret_cast<T *>(arena + off); }
    Ctrl *ctrl() const { return at<Ctrl>(lay.ctrl); }
};

namespace {

bool finite_pos(double x) { return isfinite(x) && x > 0.0; }

// Plan dimensions, slowest first, dropping unit y/z axes (x is the R2C axis).
int fft_dims(const pic_ctx *c, long long *n, long long *nin) {
    int r = 0;
    if (c->grid.n[2] > 1) { n[r] = c->grid.n[2]; nin[r] = c->grid.n[2]; ++r; }
    if (c->grid.n[1] > 1) { n[r] = c->grid.n[1]; nin[r] = c->grid.n[1]; ++r; }
    n[r] = c->grid.n[0];
    nin[r] = c->grid.n[0] / 2 + 1;
    ++r;
    return r;
}

// The four transforms: rho -> rho^ (R2C), 3 x E^ -> E4 (C2R, batch 3, output
// stride 4), lE4 -> 3 x lE^ (R2C, batch 3, input stride 4), lrho^ -> lrho (C2R).
int make_plans(pic_ctx *c, bool estimate_only, size_t *ws_max) {
    long long n[3], nh[3];
    const int rank = fft_dims(c, n, nh);
    cufftHandle p[4] = {0, 0, 0, 0};
    size_t ws[4] = {0, 0, 0, 0};
    cufftResult r = CUFFT_SUCCESS;
    int made = 0;
    for (; made < 4 && r == CUFFT_SUCCESS; ++made) {
        r = cufftCreate(&p[made]);
        if (r != CUFFT_SUCCESS) break;
        cufftSetAutoAllocation(p[made], 0);
    }
    auto plan = [&](int q, long long *inembed, long long istride, long long idist,
                    long long *onembed, long long ostride, long long odist, cufftType t,
                    long long batch) {
        if (estimate_only)
            return cufftGetSizeMany64(p[q], rank, n, inembed, istride, idist, onembed, ostride,
                                      odist, t, batch, &ws[q]);
        return cufftMakePlanMany64(p[q], rank, n, inembed, istride, idist, onembed, ostride, odist,
                                   t, batch, &ws[q]);
    };
    if (r == CUFFT_SUCCESS) r = plan(0, nullptr, 1, 0, nullptr, 1, 0, CUFFT_R2C, 1);
    if (r == CUFFT_SUCCESS) r = plan(1, nh, 1, c->nhalf, n, 4, 1, CUFFT_C2R, 3);
    if (r == CUFFT_SUCCESS) r = plan(2, n, 4, 1, nh, 1, c->nhalf, CUFFT_R2C, 3);
    if (r == CUFFT_SUCCESS) r = plan(3, nullptr, 1, 0, nullptr, 1, 0, CUFFT_C2R, 1);
    if (r != CUFFT_SUCCESS || estimate_only) {
        for (int q = 0; q < made && q < 4; ++q)
            if (p[q]) cufftDestroy(p[q]);
        if (r != CUFFT_SUCCESS) return fail(PIC_ERR_CUFFT, "cuFFT plan setup failed: %d", (int)r);
        *ws_max = std::max(std::max(ws[0], ws[1]), std::max(ws[2], ws[3]));
        return PIC_OK;
    }
    c->r2c = p[0];
    c->c2r = p[1];
    c->r2c3 = p[2];
    c->c2r1 = p[3];
    c->plans = true;
    *ws_max = std::max(std::max(ws[0], ws[1]), std::max(ws[2], ws[3]));
    return PIC_OK;
}

void destroy_plans(pic_ctx *c) {
    if (!c->plans) return;
    cufftDestroy(c->r2c);
    cufftDestroy(c->c2r);
    cufftDestroy(c->r2c3);
    cufftDestroy(c->c2r1);
    c->plans = false;
}

void compute_layout(pic_ctx *c) {
    Layout &L = c->lay;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o += align_up(bytes ? bytes : 1);
        return at;
    };
    const size_t capb = (size_t)std::max<int64_t>(c->cap, 1) * 4;
    L.set_stride = align_up(capb);
    L.ctrl = take(sizeof(Ctrl));
    L.sets = take(2 * 8 * L.set_stride);
    L.rho = take((size_t)c->ng * 4);
    L.rho64 = take((size_t)c->ng * 8);
    L.rho_hat = take((size_t)c->nhalf * 8);
    L.E_hat = take((size_t)c->nhalf * 8 * 3);
    L.E4 = take((size_t)c->ng * 16);
    L.E8 = take((size_t)c->ng * 32);
    L.bins = take((size_t)(c->nbins + 1) * 4);
    const int64_t scan_n = std::max(c->nbins, c->ntiles);
    L.scan_tmp = take((size_t)((scan_n + 4095) / 4096 + 2) * 4);
    L.tile_items = take((size_t)(c->ntiles + 1) * 4);
    L.tile_range = take((size_t)c->ntiles * 8);
    L.items = take((size_t)c->max_items * 16);
    L.fpart = take((size_t)kDiagFieldBlocks * 4 * 8);
    L.ppart = take((size_t)kMaxPushBlocks * 4 * 8);
    L.ring = take((size_t)c->prm.diag_capacity * sizeof(pic_diag_t));
    L.inv = take(capb);
    L.stage_x = take((size_t)c->staging * 24);
    L.stage_v = take((size_t)c->staging * 24);
    L.adjE4 = take((size_t)c->ng * 16);
    L.lrho2 = take((size_t)c->ng * 8);
    L.ktab = take((size_t)(c->geom.nh + c->grid.n[1] + c->grid.n[2]) * 4);
    L.fft = take(c->fft_reserve);
    L.total = o;
}

int check_ready(const pic_ctx *c) {
    if (!c) return fail(PIC_ERR_ARG, "null handle");
    if (!c->bound) return fail(PIC_ERR_STATE, "no workspace bound (call pic_bind_workspace)");
    return PIC_OK;
}

int check_loaded(const pic_ctx *c) {
    int r = check_ready(c);
    if (r) return r;
    if (!c->loaded) return fail(PIC_ERR_STATE, "no particles loaded (call pic_load_particles)");
    return PIC_OK;
}

double qscale_of(const pic_ctx *c) {
    if (c->np <= 0) return 0.0;
    return c->sp.total_charge / (double)c->np / c->dV;
}

double mp_of(const pic_ctx *c) {
    if (c->np <= 0) return 0.0;
    return c->sp.total_charge / (double)c->np / c->sp.q_over_m;
}

// the push kernel takes 4 particles per thread and fits 3 blocks per SM
int push_blocks_of(const pic_ctx *c) {
    const int64_t b = (c->np / 4 + c->block - 1) / c->block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, std::min(kMaxPushBlocks, 152 * 3 * 2)));
}

PushConst push_const(const pic_ctx *c) {
    PushConst pc;
    const double qm = c->sp.q_over_m, dt = c->prm.dt;
    pc.qm_half_dt = (float)(0.5 * dt * qm);
    double t[3], t2 = 0.0;
    for (int d = 0; d < 3; ++d) {
        pc.dt_over_h[d] = (float)(dt * c->inv_h[d]);
        t[d] = 0.5 * dt * qm * c->prm.B_ext[d];
        t2 += t[d] * t[d];
    }
    for (int d = 0; d < 3; ++d) {
        pc.t[d] = (float)t[d];
        pc.s[d] = (float)(2.0 * t[d] / (1.0 + t2));
        pc.half_n[d] = (float)(0.5 * c->grid.n[d]);
    }
    pc.wz2 = (float)c->prm.wz2;
    return pc;
}

// Sum the elapsed time of recorded pairs up to `upto` (exclusive).
int drain_timer(pic_ctx *c, int ph, int64_t upto) {
    for (; c->ev_drained[ph] < upto; ++c->ev_drained[ph]) {
        const int slot = (int)(c->ev_drained[ph] % kTimerRing);
        PIC_CUDA(cudaEventSynchronize(c->ev[ph][slot][1]));
        float t = 0.f;
        PIC_CUDA(cudaEventElapsedTime(&t, c->ev[ph][slot][0], c->ev[ph][slot][1]));
        c->ms[ph] += t;
    }
    return PIC_OK;
}

int timer_begin(pic_ctx *c, int ph) {
    if (!c->timing) return PIC_OK;
    // reuse a slot only after its previous pair has been summed
    int r = drain_timer(c, ph, c->ev_count[ph] - kTimerRing + 1);
    if (r) return r;
    const int slot = (int)(c->ev_count[ph] % kTimerRing);
    PIC_CUDA(cudaEventRecord(c->ev[ph][slot][0], c->st));
    return PIC_OK;
}

int timer_end(pic_ctx *c, int ph, int kernels) {
    c->launches += kernels;
    if (!c->timing) return PIC_OK;
    const int slot = (int)(c->ev_count[ph] % kTimerRing);
    PIC_CUDA(cudaEventRecord(c->ev[ph][slot][1], c->st));
    c->ev_count[ph] += 1;
    return PIC_OK;
}

// presort: the store is in arbitrary order (right after a load)
int do_sort(pic_ctx *c, bool presort = false) {
    int r = timer_begin(c, PIC_PHASE_SORT);
    if (r) return r;
    PIC_CUDA(launch_sort(c->np, c->geom, c->chunk, c->ctrl(), c->at<int32_t>(c->lay.bins),
                         c->nbins, c->at<int32_t>(c->lay.scan_tmp),
                         c->at<int32_t>(c->lay.tile_items), c->at<int2>(c->lay.tile_range),
                         c->at<int4>(c->lay.items), presort, c->st));
    c->since_sort = 0;
    return timer_end(c, PIC_PHASE_SORT, sort_launches(c->np, (int)c->ntiles, presort));
}

// stray-triggered re-binning: the device decides (from the last push's strays
// and the pushes since the last re-binning) and the sort kernels follow the gate
int do_sort_gated(pic_ctx *c) {
    int r = timer_begin(c, PIC_PHASE_SORT);
    if (r) return r;
    const long long max_strays = (long long)floor(c->prm.stray_rebin * (double)c->np);
    PIC_CUDA(launch_rebin_decide(c->ctrl(), max_strays, c->prm.sort_period, c->st));
    PIC_CUDA(launch_sort(c->np, c->geom, c->chunk, c->ctrl(), c->at<int32_t>(c->lay.bins),
                         c->nbins, c->at<int32_t>(c->lay.scan_tmp),
                         c->at<int32_t>(c->lay.tile_items), c->at<int2>(c->lay.tile_range),
                         c->at<int4>(c->lay.items), false, c->st, &c->ctrl()->rebin));
    return timer_end(c, PIC_PHASE_SORT, 1 + sort_launches(c->np, (int)c->ntiles, false));
}

int do_deposit(pic_ctx *c) {
    // the fixed-point path overwrites every node of rho (and re-zeroes the
    // integer grid); the FP32 path accumulates into a cleared rho
    if (!(c->prm.options & PIC_OPT_FIXED_DEPOSIT) || c->np <= 0)
        PIC_CUDA(cudaMemsetAsync(c->at<float>(c->lay.rho), 0, (size_t)c->ng * 4, c->st));
    if (c->np > 0) {
        int r = timer_begin(c, PIC_PHASE_DEPOSIT);
        if (r) return r;
        const bool fixed = (c->prm.options & PIC_OPT_FIXED_DEPOSIT) != 0;
        PIC_CUDA(launch_deposit(c->np, c->geom, c->ctrl(), c->at<int4>(c->lay.items),
                                (int)c->max_items, qscale_of(c), c->at<float>(c->lay.rho),
                                c->at<unsigned long long>(c->lay.rho64), fixed, c->ctrl(),
                                c->deposit_blocks, c->sparse_below, c->st));
        c->rho_current = true;
        return timer_end(c, PIC_PHASE_DEPOSIT, fixed ? 2 : 1);
    }
    c->rho_current = true;
    return PIC_OK;
}

int do_solve(pic_ctx *c) {
    int r = timer_begin(c, PIC_PHASE_SOLVE);
    if (r) return r;
    PIC_CUFFT(cufftExecR2C(c->r2c, c->at<cufftReal>(c->lay.rho), c->at<cufftComplex>(c->lay.rho_hat)));
    PIC_CUDA(launch_green(c->geom, c->at<float>(c->lay.ktab), c->at<float2>(c->lay.rho_hat), c->at<float2>(c->lay.E_hat),
                          c->nhalf, c->mode_idx, c->prm.mode_comp, c->mode_conj, c->ctrl(), c->st));
    PIC_CUFFT(cufftExecC2R(c->c2r, c->at<cufftComplex>(c->lay.E_hat), c->at<cufftReal>(c->lay.E4)));
    PIC_CUDA(launch_pair_E(c->geom, c->at<float4>(c->lay.E4), c->at<float4>(c->lay.E8), c->st));
    return timer_end(c, PIC_PHASE_SOLVE, 2);
}

bool uniform_move(const pic_ctx *c) { return (c->prm.options & PIC_OPT_UNIFORM_MOVE) != 0; }
bool param_grads(const pic_ctx *c) { return (c->prm.options & PIC_OPT_ADJOINT_PARAMS) != 0; }

int do_gather_push(pic_ctx *c, bool diag) {
    int r = timer_begin(c, PIC_PHASE_PUSH);
    if (r) return r;
    if (uniform_move(c) && c->np > 0) {
        PIC_CUDA(launch_move(c->np, c->geom, c->prm.seed, diag, false, false, c->ctrl(), nullptr, 0,
                             nullptr, nullptr, 0.0, 0, c->at<double>(c->lay.ppart),
                             push_blocks_of(c), c->st));
    } else {
        PIC_CUDA(launch_gather_push(c->np, c->geom, push_const(c), diag, c->ctrl(),
                                    c->at<float4>(c->lay.E8), c->at<double>(c->lay.ppart),
                                    push_blocks_of(c), c->block, c->st));
    }
    c->step += 1;
    c->since_sort += 1;
    c->rho_current = false;
    return timer_end(c, PIC_PHASE_PUSH, 1);
}

int do_diag_field(pic_ctx *c) {
    int r = timer_begin(c, PIC_PHASE_DIAG);
    if (r) return r;
    PIC_CUDA(launch_diag_field(c->geom, c->at<float>(c->lay.rho), c->at<float4>(c->lay.E4),
                               c->at<double>(c->lay.fpart), c->st));
    return timer_end(c, PIC_PHASE_DIAG, 1);
}

int do_diag_finalize(pic_ctx *c, int push_blocks) {
    int r = timer_begin(c, PIC_PHASE_DIAG);
    if (r) return r;
    PIC_CUDA(launch_diag_finalize(c->at<double>(c->lay.fpart), c->at<double>(c->lay.ppart),
                                  push_blocks, c->dV, mp_of(c), c->prm.dt, c->ctrl(),
                                  c->at<pic_diag_t>(c->lay.ring), c->prm.diag_capacity, c->st));
    return timer_end(c, PIC_PHASE_DIAG, 1);
}

// waves of resident blocks in the grids of the uniform move + deposit and the
// split-call deposit
#ifndef PIC_MV_WAVES
#define PIC_MV_WAVES 1
#endif
#ifndef PIC_DEP_WAVES
#define PIC_DEP_WAVES 1
#endif

int fused_blocks_of(const pic_ctx *c) {
    const int per = uniform_move(c) ? PIC_MV_MIN_BLOCKS * PIC_MV_WAVES : PIC_PD_MIN_BLOCKS * PIC_PD_WAVES;
    return (int)std::max<int64_t>(1, std::min<int64_t>(c->max_items, std::min(kMaxPushBlocks, 152 * per)));
}

// gather + push + deposit of the new positions in one kernel (pic_step)
int do_push_deposit(pic_ctx *c, bool diag, const SaveY &save = SaveY{}) {
    const bool fixed = (c->prm.options & PIC_OPT_FIXED_DEPOSIT) != 0;
    if (!fixed || c->np <= 0)
        PIC_CUDA(cudaMemsetAsync(c->at<float>(c->lay.rho), 0, (size_t)c->ng * 4, c->st));
    int r = timer_begin(c, PIC_PHASE_PUSH);
    if (r) return r;
    if (c->np > 0 && uniform_move(c)) {
        PIC_CUDA(launch_move(c->np, c->geom, c->prm.seed, diag, fixed, true, c->ctrl(),
                             c->at<int4>(c->lay.items), (int)c->max_items, c->at<float>(c->lay.rho),
                             c->at<unsigned long long>(c->lay.rho64), qscale_of(c),
                             c->sparse_below, c->at<double>(c->lay.ppart), fused_blocks_of(c),
                             c->st));
    } else if (c->np > 0) {
        PIC_CUDA(launch_push_deposit(c->geom, push_const(c), diag, fixed, c->ctrl(),
                                     c->at<int4>(c->lay.items), (int)c->max_items,
                                     c->at<float4>(c->lay.E4), c->at<float4>(c->lay.E8),
                                     c->at<float>(c->lay.rho),
                                     c->at<unsigned long long>(c->lay.rho64), qscale_of(c),
                                     c->sparse_below, c->at<double>(c->lay.ppart),
                                     fused_blocks_of(c), save, c->st));
    } else {
        // nothing to push: the plain kernel still records zero moments and the step
        PIC_CUDA(launch_gather_push(0, c->geom, push_const(c), diag, c->ctrl(),
                                    c->at<float4>(c->lay.E8), c->at<double>(c->lay.ppart), 1,
                                    c->block, c->st));
    }
    c->step += 1;
    c->since_sort += 1;
    c->rho_current = true;
    return timer_end(c, PIC_PHASE_PUSH, c->np > 0 ? (fixed ? 2 : 1) : 1);
}

// ---- adjoint buffer layout (caller-owned device memory) ---------------------
// The forward sweep re-bins the particles at the start of every segment of K
// steps (a checkpoint) and every R steps inside it (R = the re-binning period),
// so the tiled kernels always see tile-ordered particles.  Each re-binning
// starts a new particle order; an "order record" keeps its pid array and work
// items.  Buffer:
//   checkpoints [n_ckpt]: cell, o[3], v[3], pid (order record 0), items, n_items
//   per-step store [K]  : cell, o[3] (and, for parameter gradients, v[3]
//                         before the kick) and E8 of each step of the segment
//                         being reversed
//   order records [nrec - 1]: pid, items, n_items of records 1.. of that segment
//   multiplier backup   : ly[3], lv[3] while a segment is recomputed/permuted
//   parameter gradients : per-block partials of a reverse step and the 10 sums
struct AdjLayout {
    size_t arr, items, ckpt, segy, segE, rec, n_ckpt, off_items, off_nitems;
    size_t off_segy, off_segE, off_rec, off_lam, off_pg, total;
    int R, nrec, ny;   // ny: arrays per stored step (4, or 7 with velocities)
};

AdjLayout adj_layout(const pic_ctx *c, int n_steps, int K) {
    AdjLayout L;
    L.arr = align_up((size_t)std::max<int64_t>(c->cap, 1) * 4);
    L.items = align_up((size_t)c->max_items * 16);
    L.off_items = 8 * L.arr;
    L.off_nitems = L.off_items + L.items;
    L.ckpt = L.off_nitems + kAlign;
    L.ny = param_grads(c) ? 7 : 4;
    L.segy = (size_t)L.ny * L.arr;            // cell, o[3] (, v[3])
    L.segE = align_up((size_t)c->ng * 32);    // x-paired E of one step
    L.rec = L.arr + L.items + kAlign;         // pid, items, n_items
    L.R = std::max(1, std::min(c->prm.sort_period > 0 ? c->prm.sort_period : K, K));
    L.nrec = (K + L.R - 1) / L.R;
    const int nseg = n_steps > 1 ? (n_steps - 1 + K - 1) / K : 0;
    L.n_ckpt = (size_t)std::max(nseg, 1);
    L.off_segy = L.n_ckpt * L.ckpt;
    L.off_segE = L.off_segy + (size_t)K * L.segy;
    L.off_rec = L.off_segE + (size_t)K * L.segE;
    L.off_lam = L.off_rec + (size_t)(L.nrec - 1) * L.rec;
    L.off_pg = L.off_lam + 6 * L.arr;
    L.total = L.off_pg + (param_grads(c) ? align_up(sizeof(double) * kPGradTerms *
                                                    ((size_t)kAdjPushMaxBlocks + 1))
                                         : 0);
    return L;
}

// `count` (<= 8) particle arrays of np 4-byte entries, in one copy kernel
int copy_arrays(pic_ctx *c, char *const dst[], char *const src[], int count) {
    const size_t bytes = (size_t)c->np * 4;
    if (bytes == 0) return PIC_OK;
    CopyList cl{};
    cl.count = count;
    for (int q = 0; q < count; ++q) {
        cl.dst[q] = dst[q];
        cl.src[q] = src[q];
        cl.bytes[q] = (int64_t)bytes;
    }
    PIC_CUDA(launch_copy(cl, c->st));
    return PIC_OK;
}

int copy_bytes(pic_ctx *c, void *dst, const void *src, size_t bytes) {
    if (bytes == 0) return PIC_OK;
    PIC_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, c->st));
    return PIC_OK;
}

void set_arrays(const ParticleSet &s, char *out[8]) {
    out[0] = reinterpret_cast<char *>(s.cell);
    for (int d = 0; d < 3; ++d) {
        out[1 + d] = reinterpret_cast<char *>(s.o[d]);
        out[4 + d] = reinterpret_cast<char *>(s.v[d]);
    }
    out[7] = reinterpret_cast<char *>(s.pid);
}

void buf_arrays(char *base, size_t arr, int count, char *out[]) {
    for (int q = 0; q < count; ++q) out[q] = base + (size_t)q * arr;
}

// order record r of the current segment (r = 0: the segment's checkpoint)
struct OrderRec {
    char *pid, *items, *nitems;
};
OrderRec order_rec(const pic_ctx *c, const AdjLayout &L, int seg, int r) {
    OrderRec o;
    if (r == 0) {
        char *base = c->adj.buf + (size_t)seg * L.ckpt;
        o.pid = base + 7 * L.arr;
        o.items = base + L.off_items;
        o.nitems = base + L.off_nitems;
    } else {
        char *base = c->adj.buf + L.off_rec + (size_t)(r - 1) * L.rec;
        o.pid = base;
        o.items = base + L.arr;
        o.nitems = base + L.arr + L.items;
    }
    return o;
}

// current set's pid and work items -> order record
int adj_record(pic_ctx *c, const AdjLayout &L, int seg, int rec, int cur) {
    const OrderRec o = order_rec(c, L, seg, rec);
    int r;
    if ((r = copy_bytes(c, o.pid, c->hsets[cur].pid, (size_t)c->np * 4)) ||
        (r = copy_bytes(c, o.items, c->at<char>(c->lay.items), (size_t)c->max_items * 16)) ||
        (r = copy_bytes(c, o.nitems, &c->ctrl()->n_items, sizeof(int))))
        return r;
    return PIC_OK;
}

// work items of an order record -> the live work items
int adj_use_items(pic_ctx *c, const AdjLayout &L, int seg, int rec) {
    const OrderRec o = order_rec(c, L, seg, rec);
    int r;
    if ((r = copy_bytes(c, c->at<char>(c->lay.items), o.items, (size_t)c->max_items * 16)) ||
        (r = copy_bytes(c, &c->ctrl()->n_items, o.nitems, sizeof(int))))
        return r;
    return PIC_OK;
}

// checkpoint `seg` <-> the current particle set (with order record 0)
int adj_save(pic_ctx *c, const AdjLayout &L, int seg, int cur) {
    char *dst[8], *src[8];
    buf_arrays(c->adj.buf + (size_t)seg * L.ckpt, L.arr, 7, dst);
    set_arrays(c->hsets[cur], src);
    int r = copy_arrays(c, dst, src, 7);
    return r ? r : adj_record(c, L, seg, 0, cur);
}

int adj_restore(pic_ctx *c, const AdjLayout &L, int seg, int cur) {
    char *dst[8], *src[8];
    buf_arrays(c->adj.buf + (size_t)seg * L.ckpt, L.arr, 8, src);
    set_arrays(c->hsets[cur], dst);
    int r = copy_arrays(c, dst, src, 8);
    return r ? r : adj_use_items(c, L, seg, 0);
}

// The Boris rotation R (row-major) of v' = R v + (dt q/m / 2)(R + I) e, from
// v- -> v- + (v- + v- x t) x s with t = (dt q/m / 2) B, s = 2 t / (1 + |t|^2);
// *mag = 0 (and R = I) without a magnetic field.
void boris_rotation(const pic_ctx *c, int *mag, float R[9]) {
    const double h = 0.5 * c->prm.dt * c->sp.q_over_m;
    const double t[3] = {h * c->prm.B_ext[0], h * c->prm.B_ext[1], h * c->prm.B_ext[2]};
    const double tt = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    const double sc[3] = {2.0 * t[0] / (1.0 + tt), 2.0 * t[1] / (1.0 + tt), 2.0 * t[2] / (1.0 + tt)};
    *mag = tt > 0.0;
    for (int j = 0; j < 3; ++j) {   // column j: the rotation of unit vector e_j
        double v[3] = {0.0, 0.0, 0.0};
        v[j] = 1.0;
        const double p[3] = {v[0] + (v[1] * t[2] - v[2] * t[1]), v[1] + (v[2] * t[0] - v[0] * t[2]),
                             v[2] + (v[0] * t[1] - v[1] * t[0])};
        const double r[3] = {v[0] + (p[1] * sc[2] - p[2] * sc[1]),
                             v[1] + (p[2] * sc[0] - p[0] * sc[2]),
                             v[2] + (p[0] * sc[1] - p[1] * sc[0])};
        for (int i = 0; i < 3; ++i) R[3 * i + j] = (float)r[i];
    }
}

// M[k] (row-major 3 x 3) = dR/dB_k of the Boris rotation R v = v + (v + v x t) x s,
// t = h B (h = dt q/m / 2), s = 2t / (1 + |t|^2): column j is
// h [ (e_j x e_k) x s + (e_j + e_j x t) x (2 / (1 + |t|^2)) (e_k - t_k s) ]
void boris_rotation_derivative(const pic_ctx *c, double M[3][9]) {
    const double h = 0.5 * c->prm.dt * c->sp.q_over_m;
    const double t[3] = {h * c->prm.B_ext[0], h * c->prm.B_ext[1], h * c->prm.B_ext[2]};
    const double D = 1.0 + t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    const double sv[3] = {2.0 * t[0] / D, 2.0 * t[1] / D, 2.0 * t[2] / D};
    auto cross = [](const double a[3], const double b[3], double o[3]) {
        o[0] = a[1] * b[2] - a[2] * b[1];
        o[1] = a[2] * b[0] - a[0] * b[2];
        o[2] = a[0] * b[1] - a[1] * b[0];
    };
    for (int k = 0; k < 3; ++k) {
        double ek[3] = {0.0, 0.0, 0.0};
        ek[k] = 1.0;
        double ds[3];
        for (int d = 0; d < 3; ++d) ds[d] = (2.0 / D) * (ek[d] - t[k] * sv[d]);
        for (int j = 0; j < 3; ++j) {
            double ej[3] = {0.0, 0.0, 0.0};
            ej[j] = 1.0;
            double a[3], b[3], w[3], x[3], wt[3];
            cross(ej, ek, a);
            cross(a, sv, b);               // (e_j x e_k) x s
            cross(ej, t, wt);
            for (int d = 0; d < 3; ++d) w[d] = ej[d] + wt[d];
            cross(w, ds, x);               // (e_j + e_j x t) x ds
            for (int i = 0; i < 3; ++i) M[k][3 * i + j] = h * (b[i] + x[i]);
        }
    }
}

AdjBound step_bound(const AdjBound &ab, int par) {
    AdjBound b = ab;
    b.par = par;
    return b;
}

// field (x-paired) of step `slot` of the segment being reversed
int adj_keep_E(pic_ctx *c, const AdjLayout &L, int slot) {
    CopyList cl{};
    cl.count = 1;
    cl.dst[0] = c->adj.buf + L.off_segE + (size_t)slot * L.segE;
    cl.src[0] = c->at<char>(c->lay.E8);
    cl.bytes[0] = c->ng * 32;
    PIC_CUDA(launch_copy(cl, c->st));
    return PIC_OK;
}

// Re-bin; *cur follows the particles (the sort moves a non-empty store to the
// other set, which is also where the multipliers live: back them up first
// when they are live).
int adj_rebin(pic_ctx *c, int *cur) {
    int r = do_sort(c);
    if (r) return r;
    if (c->np > 0) *cur = 1 - *cur;
    return PIC_OK;
}

// multipliers (ly, lv: o[], v[] of the set that is not current) <-> backup
int adj_lam_backup(pic_ctx *c, const AdjLayout &L, int cur, bool to_backup) {
    const ParticleSet &ls = c->hsets[1 - cur];
    char *lam[6] = {reinterpret_cast<char *>(ls.o[0]), reinterpret_cast<char *>(ls.o[1]),
                    reinterpret_cast<char *>(ls.o[2]), reinterpret_cast<char *>(ls.v[0]),
                    reinterpret_cast<char *>(ls.v[1]), reinterpret_cast<char *>(ls.v[2])};
    char *bk[6];
    buf_arrays(c->adj.buf + L.off_lam, L.arr, 6, bk);
    return to_backup ? copy_arrays(c, bk, lam, 6) : copy_arrays(c, lam, bk, 6);
}

LamOut adj_backup_out(pic_ctx *c, const AdjLayout &L) {
    char *bk[6];
    buf_arrays(c->adj.buf + L.off_lam, L.arr, 6, bk);
    LamOut o;
    for (int d = 0; d < 3; ++d) {
        o.o[d] = reinterpret_cast<float *>(bk[d]);
        o.v[d] = reinterpret_cast<float *>(bk[3 + d]);
    }
    return o;
}

// Multipliers held in the backup in the order given by pid_later -> the live
// multiplier arrays in the order given by pid_earlier (same particles).
int adj_permute_from_backup(pic_ctx *c, const AdjLayout &L, int cur, const int32_t *pid_later,
                            const int32_t *pid_earlier) {
    if (c->np <= 0) return PIC_OK;
    int32_t *pos = c->at<int32_t>(c->lay.inv);
    const ParticleSet &ls = c->hsets[1 - cur];
    char *bk[6];
    buf_arrays(c->adj.buf + L.off_lam, L.arr, 6, bk);
    const float *in_o[3] = {reinterpret_cast<float *>(bk[0]), reinterpret_cast<float *>(bk[1]),
                            reinterpret_cast<float *>(bk[2])};
    const float *in_v[3] = {reinterpret_cast<float *>(bk[3]), reinterpret_cast<float *>(bk[4]),
                            reinterpret_cast<float *>(bk[5])};
    float *out_o[3] = {ls.o[0], ls.o[1], ls.o[2]};
    float *out_v[3] = {ls.v[0], ls.v[1], ls.v[2]};
    PIC_CUDA(launch_pid_positions(c->np, pid_later, pos, c->st));
    PIC_CUDA(launch_adj_reorder(c->np, pos, pid_earlier, in_o, in_v, out_o, out_v, c->st));
    return PIC_OK;
}

// One forward step of a sweep that keeps its trajectory: re-bin when an order
// starts here (recording it), solve, keep E_n, push + deposit keeping y_n.
int adj_keep_step(pic_ctx *c, const AdjLayout &L, int seg, int a0, int n, int *cur) {
    int r;
    if (n > a0 && (n - a0) % L.R == 0) {
        if ((r = adj_rebin(c, cur)) || (r = adj_record(c, L, seg, (n - a0) / L.R, *cur)))
            return r;
    }
    if (!c->rho_current && (r = do_deposit(c))) return r;
    if ((r = do_solve(c)) || (r = adj_keep_E(c, L, n - a0))) return r;
    if (c->np == 0) return do_push_deposit(c, false);
    // y_n is written by the push that reads it
    char *y[7];
    buf_arrays(c->adj.buf + L.off_segy + (size_t)(n - a0) * L.segy, L.arr, L.ny, y);
    SaveY save{};
    save.cell = reinterpret_cast<int32_t *>(y[0]);
    for (int d = 0; d < 3; ++d) save.o[d] = reinterpret_cast<float *>(y[1 + d]);
    if (L.ny == 7)
        for (int d = 0; d < 3; ++d) save.v[d] = reinterpret_cast<float *>(y[4 + d]);
    return do_push_deposit(c, false, save);
}

// the adjoint field solve of step m (par = m & 1: its bound bookkeeping slot)
int adj_solve(pic_ctx *c, int par) {
    PIC_CUFFT(cufftExecR2C(c->r2c3, c->at<cufftReal>(c->lay.adjE4), c->at<cufftComplex>(c->lay.E_hat)));
    PIC_CUDA(launch_green_adj(c->geom, c->L, c->at<float2>(c->lay.E_hat),
                              c->at<float2>(c->lay.rho_hat), c->nhalf, c->st));
    PIC_CUFFT(cufftExecC2R(c->c2r1, c->at<cufftComplex>(c->lay.rho_hat), c->at<cufftReal>(c->lay.rho)));
    PIC_CUDA(launch_adj_pair_rho(c->geom, c->at<float>(c->lay.rho), c->at<float2>(c->lay.lrho2),
                                 c->at<float4>(c->lay.adjE4), c->ctrl(), par, c->st));
    return PIC_OK;
}

// Device address of `bytes` of page-locked host memory mapped into the GPU's
// address space (e.g. from cudaHostAlloc or torch's pin_memory), or nullptr
// when the range is ordinary pageable memory.  Both ends must resolve into
// the same mapping.  On this Grace-coupled part kernels then read and write
// the host buffers directly over the chip-to-chip link instead of staging
// them through copies.
const void *mapped_host(const void *p, size_t bytes) {
#if PIC_ZERO_COPY
    if (!p || bytes == 0) return nullptr;
    cudaPointerAttributes a{}, b{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    const char *last = static_cast<const char *>(p) + bytes - 1;
    if (cudaPointerGetAttributes(&b, last) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer ||
        !b.devicePointer)
        return nullptr;
    if (static_cast<const char *>(b.devicePointer) - static_cast<const char *>(a.devicePointer) !=
        (ptrdiff_t)(bytes - 1))
        return nullptr;
    return a.devicePointer;
#else
    (void)p;
    (void)bytes;
    return nullptr;
#endif
}

// Reset the resettable head of the control block (everything before `cur`).
// a raised device flag as a status: a bounded wait that gave up is reported
// as such, every other flag as PIC_ERR_DEVICE_FLAG
int flag_error(int32_t flags) {
    return (flags & PIC_FLAG_TIMEOUT) ? PIC_ERR_TIMEOUT : PIC_ERR_DEVICE_FLAG;
}

int reset_ctrl(pic_ctx *c) {
    PIC_CUDA(cudaMemsetAsync(c->ctrl(), 0, offsetof(Ctrl, cur), c->st));
    return PIC_OK;
}

}  // namespace

// =============================================================================
// C ABI
// =============================================================================
extern "C" {

const char *pic_last_error(void) { return g_err; }

int pic_create(const pic_grid_t *grid, const pic_species_t *species, const pic_params_t *params,
               pic_handle_t *out) {
    if (!grid || !species || !params || !out) return fail(PIC_ERR_ARG, "null argument");
    *out = nullptr;
    for (int d = 0; d < 3; ++d) {
        if (grid->n[d] < 1 || grid->n[d] > kMaxN)
            return fail(PIC_ERR_ARG, "grid n[%d] = %d outside 1..%d", d, grid->n[d], kMaxN);
        if (!finite_pos(grid->L[d]))
            return fail(PIC_ERR_ARG, "grid L[%d] must be finite and > 0", d);
    }
    if (grid->n[0] < 2) return fail(PIC_ERR_ARG, "grid n[0] must be >= 2 (R2C axis)");
    if (species->n_particles < 0 || species->n_particles > 2147483647LL)
        return fail(PIC_ERR_ARG, "n_particles %lld outside 0..2^31-1",
                    (long long)species->n_particles);
    if (!isfinite(species->q_over_m) || species->q_over_m == 0.0)
        return fail(PIC_ERR_ARG, "q_over_m must be finite and nonzero");
    if (!isfinite(species->total_charge)) return fail(PIC_ERR_ARG, "total_charge must be finite");
    if (!finite_pos(params->dt)) return fail(PIC_ERR_ARG, "dt must be finite and > 0");
    for (int d = 0; d < 3; ++d)
        if (!isfinite(params->B_ext[d])) return fail(PIC_ERR_ARG, "B_ext must be finite");
    if (!isfinite(params->wz2)) return fail(PIC_ERR_ARG, "wz2 must be finite");
    for (int d = 0; d < 3; ++d)
        if (params->tile[d] < 0) return fail(PIC_ERR_ARG, "tile[%d] must be >= 0", d);
    if (params->guard < 0 || params->guard > 8) return fail(PIC_ERR_ARG, "guard outside 0..8");
    if (params->diag_every < 0) return fail(PIC_ERR_ARG, "diag_every must be >= 0");
    if (params->diag_capacity < 0) return fail(PIC_ERR_ARG, "diag_capacity must be >= 0");
    if (params->mode_comp < 0 || params->mode_comp > 2)
        return fail(PIC_ERR_ARG, "mode_comp must be 0, 1 or 2");
    for (int d = 0; d < 3; ++d)
        if (2 * abs(params->mode[d]) > grid->n[d])
            return fail(PIC_ERR_ARG, "mode[%d] = %d beyond the Nyquist index", d, params->mode[d]);
    if (params->block != 0 && (params->block < 32 || params->block > 256 || params->block % 32))
        return fail(PIC_ERR_ARG, "block must be 0 or a multiple of 32 in 32..256");
    if (params->chunk != 0 && (params->chunk < 32 || params->chunk > kMaxChunk))
        return fail(PIC_ERR_ARG, "chunk must be 0 or in 32..%d", kMaxChunk);
    if (params->options & ~(PIC_OPT_FIXED_DEPOSIT | PIC_OPT_UNIFORM_MOVE | PIC_OPT_ADJOINT_PARAMS))
        return fail(PIC_ERR_ARG, "unknown option bits");
    if (!isfinite(params->stray_rebin) || params->stray_rebin < 0.0)
        return fail(PIC_ERR_ARG, "stray_rebin must be finite and >= 0");

    pic_ctx *c = new (std::nothrow) pic_ctx();
    if (!c) return fail(PIC_ERR_ARG, "out of host memory");
    c->grid = *grid;
    c->sp = *species;
    c->prm = *params;
    pic_params_t &p = c->prm;
    if (p.sort_period == 0) p.sort_period = 1;
    if (p.diag_capacity == 0) p.diag_capacity = 1024;
    if (p.guard == 0) p.guard = 2;
    c->block = p.block ? p.block : 256;
    c->chunk = p.chunk ? p.chunk : kMaxChunk;

    Geom &g = c->geom;
    int64_t nt = 1;
    for (int d = 0; d < 3; ++d) {
        g.n[d] = grid->n[d];
        int T = p.tile[d] ? p.tile[d] : 8;
        T = std::min(T, grid->n[d]);
        g.tile[d] = T;
        g.ntile[d] = (grid->n[d] + T - 1) / T;
        nt *= g.ntile[d];
        c->L[d] = grid->L[d];
        c->h[d] = grid->L[d] / grid->n[d];
        c->inv_h[d] = grid->n[d] / grid->L[d];
        g.h[d] = (float)c->h[d];
        g.inv_h[d] = (float)c->inv_h[d];
    }
    g.nh = grid->n[0] / 2 + 1;
    g.guard = p.guard;
    for (int d = 0; d < 3; ++d)
        g.tdiv[d] = g.tile[d] > 1 ? (unsigned)((((uint64_t)1 << 32) + g.tile[d] - 1) / g.tile[d]) : 0u;
    g.tvol = g.tile[0] * g.tile[1] * g.tile[2];
    c->dV = c->h[0] * c->h[1] * c->h[2];
    c->ntiles = nt;
    c->nbins = nt;    // the binning key is the deposit tile
    if (tile_deposit_smem(g) > kMaxSmemPerBlock) {
        delete c;
        return fail(PIC_ERR_ARG, "deposit tile plus guard too large for shared memory "
                                 "(%zu bytes > %d)", tile_deposit_smem(g), kMaxSmemPerBlock);
    }
    if (c->nbins > 2147483647LL - 1) {
        delete c;
        return fail(PIC_ERR_ARG, "too many tiles for this grid");
    }
    c->cap = species->n_particles;
    c->ng = (int64_t)grid->n[0] * grid->n[1] * grid->n[2];
    c->nhalf = (int64_t)g.nh * grid->n[1] * grid->n[2];
    c->max_items = c->ntiles + (c->cap + c->chunk - 1) / c->chunk + 1;
    c->staging = std::max<int64_t>(1, std::min<int64_t>(c->cap, (int64_t)1 << 22));
    c->sparse_below = 64;
    c->deposit_blocks = 152 * PIC_DEP_MIN_BLOCKS * PIC_DEP_WAVES;   // waves of the resident blocks

    int m[3] = {p.mode[0], p.mode[1], p.mode[2]};
    c->mode_conj = 0;
    if (m[0] < 0) {   // use the conjugate of the mirrored mode (real field)
        for (int d = 0; d < 3; ++d) m[d] = -m[d];
        c->mode_conj = 1;
    }
    c->mode_idx[0] = m[0];
    c->mode_idx[1] = ((m[1] % grid->n[1]) + grid->n[1]) % grid->n[1];
    c->mode_idx[2] = ((m[2] % grid->n[2]) + grid->n[2]) % grid->n[2];

    // cuFFT work area: the library's own size query when it works here,
    // never less than a conservative bound
    size_t wmax = 0;
    size_t bound = (size_t)c->nhalf * 8 * 3 + ((size_t)4 << 20);
    if (make_plans(c, true, &wmax) == PIC_OK) bound = std::max(bound, wmax);
    c->fft_reserve = bound;
    compute_layout(c);
    *out = c;
    snprintf(g_err, sizeof(g_err), "no error");
    return PIC_OK;
}

int pic_buffer_sizes(pic_handle_t c, pic_bufsizes_t *out) {
    if (!c || !out) return fail(PIC_ERR_ARG, "null argument");
    out->workspace_bytes = c->lay.total;
    out->workspace_align = kAlign;
    out->particle_capacity = c->cap;
    out->grid_nodes = c->ng;
    out->staging_particles = c->staging;
    return PIC_OK;
}

int pic_bind_workspace(pic_handle_t c, void *arena, size_t bytes, void *stream) {
    if (!c || !arena) return fail(PIC_ERR_ARG, "null argument");
    if ((uintptr_t)arena % kAlign) return fail(PIC_ERR_ARG, "arena not %zu-byte aligned", kAlign);
    if (bytes < c->lay.total)
        return fail(PIC_ERR_CAPACITY, "arena of %zu bytes < required %zu", bytes, c->lay.total);
    destroy_plans(c);
    c->bound = false;
    c->loaded = false;
    c->adj.ready = false;
    c->arena = static_cast<char *>(arena);
    c->st = static_cast<cudaStream_t>(stream);
    size_t wmax = 0;
    int r = make_plans(c, false, &wmax);
    if (r) return r;
    if (wmax > c->fft_reserve) {
        destroy_plans(c);
        return fail(PIC_ERR_CAPACITY, "cuFFT needs %zu work bytes, %zu reserved", wmax,
                    c->fft_reserve);
    }
    void *work = c->arena + c->lay.fft;
    for (cufftHandle p : {c->r2c, c->c2r, c->r2c3, c->c2r1}) {
        PIC_CUFFT(cufftSetWorkArea(p, work));
        PIC_CUFFT(cufftSetStream(p, c->st));
    }

    PIC_CUDA(sort_prepare());
    PIC_CUDA(push_deposit_prepare(c->geom));
    Ctrl h;
    memset(&h, 0, sizeof(h));
    for (int s = 0; s < 2; ++s) {
        char *base = c->arena + c->lay.sets + (size_t)s * 8 * c->lay.set_stride;
        ParticleSet &ps = h.sets[s];
        ps.cell = reinterpret_cast<int32_t *>(base);
        for (int d = 0; d < 3; ++d) {
            ps.o[d] = reinterpret_cast<float *>(base + (size_t)(1 + d) * c->lay.set_stride);
            ps.v[d] = reinterpret_cast<float *>(base + (size_t)(4 + d) * c->lay.set_stride);
        }
        ps.pid = reinterpret_cast<int32_t *>(base + (size_t)7 * c->lay.set_stride);
    }
    c->hsets[0] = h.sets[0];
    c->hsets[1] = h.sets[1];
    PIC_CUDA(cudaMemcpyAsync(c->ctrl(), &h, sizeof(h), cudaMemcpyHostToDevice, c->st));
    std::vector<float> ktab((size_t)(c->geom.nh + c->grid.n[1] + c->grid.n[2]));
    green_table(c->geom, c->L, ktab.data());
    PIC_CUDA(cudaMemcpyAsync(c->at<float>(c->lay.ktab), ktab.data(), ktab.size() * 4,
                             cudaMemcpyHostToDevice, c->st));
    PIC_CUDA(cudaMemsetAsync(c->at<char>(c->lay.E4), 0, (size_t)c->ng * 16, c->st));
    PIC_CUDA(cudaMemsetAsync(c->at<char>(c->lay.rho), 0, (size_t)c->ng * 4, c->st));
    PIC_CUDA(cudaMemsetAsync(c->at<char>(c->lay.rho64), 0, (size_t)c->ng * 8, c->st));
    PIC_CUDA(cudaMemsetAsync(c->at<char>(c->lay.ring), 0,
                             (size_t)c->prm.diag_capacity * sizeof(pic_diag_t), c->st));
    PIC_CUDA(cudaStreamSynchronize(c->st));
    c->bound = true;
    c->np = 0;
    c->step = 0;
    c->since_sort = 0;
    return PIC_OK;
}

int pic_set_stream(pic_handle_t c, void *stream) {
    int r = check_ready(c);
    if (r) return r;
    c->st = static_cast<cudaStream_t>(stream);
    for (cufftHandle p : {c->r2c, c->c2r, c->r2c3, c->c2r1}) PIC_CUFFT(cufftSetStream(p, c->st));
    return PIC_OK;
}

void pic_destroy(pic_handle_t c) {
    if (!c) return;
    destroy_plans(c);
    if (c->side_made) {
        for (cudaEvent_t e : c->side_ev) cudaEventDestroy(e);
        cudaStreamDestroy(c->side);
    }
    if (c->events_made)
        for (int p = 0; p < PIC_PHASE_COUNT; ++p)
            for (int s = 0; s < kTimerRing; ++s)
                for (int e = 0; e < 2; ++e) cudaEventDestroy(c->ev[p][s][e]);
    delete c;
}

namespace {

// coarse passes the first binning of particles in arbitrary order needs
int presort_passes(const pic_ctx *c) {
    return (sort_launches(1, (int)c->ntiles, true) - sort_launches(1, (int)c->ntiles, false)) / 6;
}

int load_overlapped(pic_ctx *c, const double *mx, const double *mv, int64_t n) {
    if (!c->side_made) {
        PIC_CUDA(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
        for (cudaEvent_t &e : c->side_ev) PIC_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        c->side_made = true;
    }
    // ranges of a multiple of 512 particles (bulk copies start on 16 bytes)
    const int64_t per = ((n + kLoadRanges - 1) / kLoadRanges + 511) / 512 * 512;
    int passes = 0;
    for (int k = 0; k < kLoadRanges; ++k) {
        const int64_t o = (int64_t)k * per;
        if (o >= n) break;
        const int64_t m = std::min(per, n - o);
        PIC_CUDA(launch_load(mx + 3 * o, mv + 3 * o, m, o, c->geom, c->inv_h, c->prm.dt, c->ctrl(),
                             c->st, kNumSMs));
        c->launches += 1;
        PIC_CUDA(cudaEventRecord(c->side_ev[k], c->st));
        PIC_CUDA(cudaStreamWaitEvent(c->side, c->side_ev[k], 0));
        int kernels = 0;
        PIC_CUDA(launch_sort_range(m, o, c->geom, c->ctrl(), c->at<int32_t>(c->lay.bins), c->nbins,
                                   c->at<int32_t>(c->lay.scan_tmp), &passes, &kernels, c->side));
        c->launches += kernels;
    }
    PIC_CUDA(cudaEventRecord(c->side_ev[kLoadRanges], c->side));
    PIC_CUDA(cudaStreamWaitEvent(c->st, c->side_ev[kLoadRanges], 0));
    if (passes & 1) {   // the ranges now live in the other set
        PIC_CUDA(launch_flip(c->ctrl(), c->st));
        c->launches += 1;
    }
    return PIC_OK;
}

}  // namespace

int pic_load_particles(pic_handle_t c, const double *x, const double *v, int64_t n,
                       int src_is_device) {
    int r = check_ready(c);
    if (r) return r;
    if (n < 0) return fail(PIC_ERR_ARG, "negative particle count");
    if (n > c->cap) return fail(PIC_ERR_CAPACITY, "%lld particles > capacity %lld",
                                (long long)n, (long long)c->cap);
    if (n > 0 && (!x || !v)) return fail(PIC_ERR_ARG, "null particle array");
    if ((r = reset_ctrl(c))) return r;
    const double *mx = src_is_device ? nullptr
                                     : static_cast<const double *>(mapped_host(x, (size_t)n * 24));
    const double *mv = mx ? static_cast<const double *>(mapped_host(v, (size_t)n * 24)) : nullptr;
    if (src_is_device) {
        PIC_CUDA(launch_load(x, v, n, 0, c->geom, c->inv_h, c->prm.dt, c->ctrl(), c->st));
    } else if (mx && mv && n >= kOverlapMin && presort_passes(c) > 0) {
        // page-locked host arrays, read in place by the load kernel one range
        // at a time on one block per SM (the host link, not the SMs, bounds
        // it); each loaded range is binned on the side stream meanwhile, so
        // the final full-key pass sees tile-ordered runs
        if ((r = load_overlapped(c, mx, mv, n))) return r;
        c->np = n;
        c->step = 0;
        c->loaded = true;
        c->rho_current = false;
        if ((r = do_sort(c))) return r;
        PIC_CUDA(cudaStreamSynchronize(c->st));
        return PIC_OK;
    } else if (mx && mv) {
        // page-locked host arrays: read in place by the load kernel
        PIC_CUDA(launch_load(mx, mv, n, 0, c->geom, c->inv_h, c->prm.dt, c->ctrl(), c->st));
    } else {
        double *sx = c->at<double>(c->lay.stage_x), *sv = c->at<double>(c->lay.stage_v);
        for (int64_t o = 0; o < n; o += c->staging) {
            const int64_t m = std::min<int64_t>(c->staging, n - o);
            PIC_CUDA(cudaMemcpyAsync(sx, x + 3 * o, (size_t)m * 24, cudaMemcpyHostToDevice, c->st));
            PIC_CUDA(cudaMemcpyAsync(sv, v + 3 * o, (size_t)m * 24, cudaMemcpyHostToDevice, c->st));
            PIC_CUDA(launch_load(sx, sv, m, o, c->geom, c->inv_h, c->prm.dt, c->ctrl(), c->st));
        }
    }
    c->np = n;
    c->step = 0;
    c->loaded = true;
    c->rho_current = false;
    if ((r = do_sort(c, true))) return r;
    if (!src_is_device) PIC_CUDA(cudaStreamSynchronize(c->st));
    return PIC_OK;
}

int pic_get_particles(pic_handle_t c, double *x, double *v, int dst_is_device) {
    int r = check_loaded(c);
    if (r) return r;
    if (c->np > 0 && (!x || !v)) return fail(PIC_ERR_ARG, "null output array");
    int32_t *inv = c->at<int32_t>(c->lay.inv);
    PIC_CUDA(launch_invperm(c->np, c->ctrl(), inv, c->st));
    if (dst_is_device) {
        PIC_CUDA(launch_unload(0, c->np, inv, c->geom, c->h, c->L, c->prm.dt, c->ctrl(), x, v, c->st));
        return PIC_OK;
    }
    double *mx = static_cast<double *>(const_cast<void *>(mapped_host(x, (size_t)c->np * 24)));
    double *mv = mx ? static_cast<double *>(const_cast<void *>(mapped_host(v, (size_t)c->np * 24)))
                    : nullptr;
    if (mx && mv) {
        // page-locked host arrays: written in place by the unload kernel
        PIC_CUDA(launch_unload(0, c->np, inv, c->geom, c->h, c->L, c->prm.dt, c->ctrl(), mx, mv,
                               c->st));
        PIC_CUDA(cudaStreamSynchronize(c->st));
        return PIC_OK;
    }
    double *sx = c->at<double>(c->lay.stage_x), *sv = c->at<double>(c->lay.stage_v);
    for (int64_t o = 0; o < c->np; o += c->staging) {
        const int64_t m = std::min<int64_t>(c->staging, c->np - o);
        PIC_CUDA(launch_unload(o, m, inv, c->geom, c->h, c->L, c->prm.dt, c->ctrl(), sx, sv, c->st));
        PIC_CUDA(cudaMemcpyAsync(x + 3 * o, sx, (size_t)m * 24, cudaMemcpyDeviceToHost, c->st));
        PIC_CUDA(cudaMemcpyAsync(v + 3 * o, sv, (size_t)m * 24, cudaMemcpyDeviceToHost, c->st));
    }
    PIC_CUDA(cudaStreamSynchronize(c->st));
    return PIC_OK;
}

int pic_get_field(pic_handle_t c, float *rho, float *E, int dst_is_device) {
    int r = check_ready(c);
    if (r) return r;
    const cudaMemcpyKind k = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (rho) PIC_CUDA(cudaMemcpyAsync(rho, c->at<float>(c->lay.rho), (size_t)c->ng * 4, k, c->st));
    if (E) PIC_CUDA(cudaMemcpyAsync(E, c->at<float>(c->lay.E4), (size_t)c->ng * 16, k, c->st));
    if (!dst_is_device) PIC_CUDA(cudaStreamSynchronize(c->st));
    return PIC_OK;
}

int pic_set_rho(pic_handle_t c, const float *rho, int src_is_device) {
    int r = check_ready(c);
    if (r) return r;
    c->rho_current = false;
    if (!rho) return fail(PIC_ERR_ARG, "null rho");
    const cudaMemcpyKind k = src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    PIC_CUDA(cudaMemcpyAsync(c->at<float>(c->lay.rho), rho, (size_t)c->ng * 4, k, c->st));
    if (!src_is_device) PIC_CUDA(cudaStreamSynchronize(c->st));
    return PIC_OK;
}

int pic_get_counts(pic_handle_t c, int64_t *n_particles, int64_t *step) {
    if (!c) return fail(PIC_ERR_ARG, "null handle");
    if (n_particles) *n_particles = c->np;
    if (step) *step = c->step;
    return PIC_OK;
}

int pic_sort(pic_handle_t c) {
    int r = check_loaded(c);
    if (r) return r;
    return do_sort(c);
}

int pic_deposit(pic_handle_t c) {
    int r = check_loaded(c);
    if (r) return r;
    return do_deposit(c);
}

int pic_field_solve(pic_handle_t c) {
    int r = check_ready(c);
    if (r) return r;
    return do_solve(c);
}

int pic_gather_push(pic_handle_t c) {
    int r = check_loaded(c);
    if (r) return r;
    return do_gather_push(c, false);
}

int pic_step(pic_handle_t c, int n) {
    int r = check_loaded(c);
    if (r) return r;
    if (n < 0) return fail(PIC_ERR_ARG, "negative step count");
    // each step: [re-bin] -> (deposit, only if rho is stale) -> solve ->
    // [field diagnostics, before rho is replaced] -> fused gather + push +
    // deposit of the new positions -> [particle diagnostics]
    for (int s = 0; s < n; ++s) {
        if (c->prm.stray_rebin > 0.0 && c->np > 0) {
            if ((r = do_sort_gated(c))) return r;
        } else if (c->prm.sort_period > 0 && c->since_sort >= c->prm.sort_period) {
            if ((r = do_sort(c))) return r;
        }
        if (!c->rho_current && (r = do_deposit(c))) return r;
        if ((r = do_solve(c))) return r;
        const bool diag = c->prm.diag_every > 0 && ((c->step + 1) % c->prm.diag_every == 0);
        if (diag && (r = do_diag_field(c))) return r;
        if ((r = do_push_deposit(c, diag))) return r;
        if (diag && (r = do_diag_finalize(c, c->np > 0 ? fused_blocks_of(c) : 1))) return r;
    }
    return PIC_OK;
}

int pic_diagnostics(pic_handle_t c, pic_diag_t *out, int max_records, int *n_out) {
    int r = check_ready(c);
    if (r) return r;
    if (n_out) *n_out = 0;
    if (max_records < 0 || (max_records > 0 && !out)) return fail(PIC_ERR_ARG, "bad output buffer");
    PIC_CUDA(cudaStreamSynchronize(c->st));
    Ctrl h;
    PIC_CUDA(cudaMemcpy(&h, c->ctrl(), sizeof(Ctrl), cudaMemcpyDeviceToHost));
    const long long cap = c->prm.diag_capacity;
    const long long have = std::min<long long>(h.diag_written, cap);
    const long long first = h.diag_written - have;     // oldest record kept
    const long long want = std::min<long long>(have, max_records);
    std::vector<pic_diag_t> all((size_t)std::max<long long>(cap, 1));
    if (want > 0) {
        PIC_CUDA(cudaMemcpy(all.data(), c->at<pic_diag_t>(c->lay.ring), (size_t)cap * sizeof(pic_diag_t),
                            cudaMemcpyDeviceToHost));
        for (long long q = 0; q < want; ++q) out[q] = all[(size_t)((first + q) % cap)];
    }
    if (n_out) *n_out = (int)want;
    if (h.flags) return fail(flag_error(h.flags), "device error flags 0x%x", h.flags);
    return PIC_OK;
}

int pic_rebin_stats(pic_handle_t c, int64_t *rebins, int64_t *strays) {
    int r = check_ready(c);
    if (r) return r;
    PIC_CUDA(cudaStreamSynchronize(c->st));
    Ctrl h;
    PIC_CUDA(cudaMemcpy(&h, c->ctrl(), sizeof(Ctrl), cudaMemcpyDeviceToHost));
    if (rebins) *rebins = h.rebins;
    if (strays) *strays = (int64_t)h.stray_step;
    return PIC_OK;
}

int pic_selftest_timeout(pic_handle_t c) {
    int r = check_ready(c);
    if (r) return r;
    PIC_CUDA(launch_timeout_selftest(c->ctrl(), c->st));
    PIC_CUDA(cudaStreamSynchronize(c->st));
    int32_t f = 0;
    PIC_CUDA(cudaMemcpy(&f, c->ctrl(), sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (f & PIC_FLAG_TIMEOUT) return fail(PIC_ERR_TIMEOUT, "bounded device wait gave up (flags 0x%x)", f);
    return fail(PIC_ERR_STATE, "the self-test wait completed, which it must not");
}

int pic_device_flags(pic_handle_t c, int32_t *flags, int clear) {
    int r = check_ready(c);
    if (r) return r;
    PIC_CUDA(cudaStreamSynchronize(c->st));
    int32_t f = 0;
    PIC_CUDA(cudaMemcpy(&f, c->ctrl(), sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (flags) *flags = f;
    if (clear) PIC_CUDA(cudaMemset(c->ctrl(), 0, sizeof(int32_t)));
    return PIC_OK;
}

int pic_adjoint_buffer_bytes(pic_handle_t c, int n_steps, int K, size_t *bytes) {
    if (!c || !bytes) return fail(PIC_ERR_ARG, "null argument");
    if (n_steps < 1 || K < 1) return fail(PIC_ERR_ARG, "n_steps and checkpoint_every must be >= 1");
    *bytes = adj_layout(c, n_steps, K).total;
    return PIC_OK;
}

int pic_adjoint_forward(pic_handle_t c, int n_steps, int K, const double *w, void *buf,
                        size_t bytes, double *J) {
    int r = check_loaded(c);
    if (r) return r;
    if (n_steps < 1 || K < 1) return fail(PIC_ERR_ARG, "n_steps and checkpoint_every must be >= 1");
    if (!w || !buf || !J) return fail(PIC_ERR_ARG, "null argument");
    for (int d = 0; d < 3; ++d)
        if (!isfinite(w[d]) || w[d] < 0.0) return fail(PIC_ERR_ARG, "weights must be finite and >= 0");
    if ((uintptr_t)buf % kAlign) return fail(PIC_ERR_ARG, "adjoint buffer not 256-byte aligned");
    if (uniform_move(c)) return fail(PIC_ERR_ARG, "the uniform-plasma move has no adjoint");
    const AdjLayout L = adj_layout(c, n_steps, K);
    if (bytes < L.total)
        return fail(PIC_ERR_CAPACITY, "adjoint buffer of %zu bytes < required %zu", bytes, L.total);
    PIC_CUDA(cudaStreamSynchronize(c->st));
    int32_t cur = 0;
    PIC_CUDA(cudaMemcpy(&cur, &c->ctrl()->cur, sizeof(cur), cudaMemcpyDeviceToHost));
    PIC_CUDA(cudaMemcpy(&c->adj.step0_dev, &c->ctrl()->step, sizeof(long long), cudaMemcpyDeviceToHost));
    c->adj.ready = false;
    c->adj.n_steps = n_steps;
    c->adj.K = K;
    c->adj.nseg = n_steps > 1 ? (n_steps - 1 + K - 1) / K : 0;
    c->adj.cur = cur;
    c->adj.buf = static_cast<char *>(buf);
    c->adj.step0 = c->step;
    for (int d = 0; d < 3; ++d) c->adj.w[d] = w[d];
    // checkpoint s holds the state at step s K, re-binned so that the
    // segment's tiled kernels (forward and reverse) see tile-ordered particles
    // The last segment's positions, fields and orders are kept as they are
    // computed, so the reverse sweep starts without recomputing it (with
    // K >= n_steps - 1 nothing is recomputed at all).
    const int nck = (int)L.n_ckpt;
    for (int s = 0; s < nck; ++s) {
        if ((r = adj_rebin(c, &cur)) || (r = adj_save(c, L, s, cur))) return r;
        const int a0 = s * K, b0 = std::min(a0 + K, n_steps - 1);
        const bool keep = s == c->adj.nseg - 1;
        for (int n = a0; n < b0; ++n) {
            if (keep) {
                if ((r = adj_keep_step(c, L, s, a0, n, &cur))) return r;
                continue;
            }
            if (n > a0 && (n - a0) % L.R == 0 && (r = adj_rebin(c, &cur))) return r;
            if (!c->rho_current && (r = do_deposit(c))) return r;
            if ((r = do_solve(c)) || (r = do_push_deposit(c, false))) return r;
        }
    }
    c->adj.cur_end = cur;
    if (!c->rho_current && (r = do_deposit(c))) return r;
    if ((r = do_solve(c))) return r;
    PIC_CUDA(launch_diag_field(c->geom, c->at<float>(c->lay.rho), c->at<float4>(c->lay.E4),
                               c->at<double>(c->lay.fpart), c->st));
    PIC_CUDA(launch_objective(c->at<double>(c->lay.fpart), kDiagFieldBlocks, c->dV, c->adj.w,
                              &c->ctrl()->scalar[0], c->st));
    PIC_CUDA(cudaMemcpyAsync(J, &c->ctrl()->scalar[0], sizeof(double), cudaMemcpyDeviceToHost, c->st));
    PIC_CUDA(cudaStreamSynchronize(c->st));
    c->adj.ready = true;
    return PIC_OK;
}

int pic_adjoint_backward(pic_handle_t c, double scale, double *gx, double *gv, int dst_is_device) {
    int r = check_loaded(c);
    if (r) return r;
    if (!c->adj.ready) return fail(PIC_ERR_STATE, "no pic_adjoint_forward to reverse");
    if (c->np > 0 && (!gx || !gv)) return fail(PIC_ERR_ARG, "null output array");
    const AdjLayout L = adj_layout(c, c->adj.n_steps, c->adj.K);
    const int K = c->adj.K;
    int cur = c->adj.cur_end;
    const float qsc = (float)qscale_of(c);
    const float c_kick = (float)(c->prm.dt * c->sp.q_over_m);
    const float dt = (float)c->prm.dt, wz2 = (float)c->prm.wz2;
    const float kb = 2.0f * fabsf(qsc) *
                     (float)std::max(c->inv_h[0], std::max(c->inv_h[1], c->inv_h[2]));
    AdjBound ab{};
    ab.c_abs = fabsf(c_kick);
    ab.dt = dt;
    ab.kb = kb;
    boris_rotation(c, &ab.mag, ab.R);
    float4 *lE4 = c->at<float4>(c->lay.adjE4);
    const float2 *lrho2 = c->at<float2>(c->lay.lrho2);
    const bool pgrad = param_grads(c);
    double *pg_part = reinterpret_cast<double *>(c->adj.buf + L.off_pg);
    double *pg_acc = pg_part + (size_t)kPGradTerms * kAdjPushMaxBlocks;
    c->adj.pgrad_ready = false;
    if (pgrad) PIC_CUDA(cudaMemsetAsync(pg_acc, 0, sizeof(double) * kPGradTerms, c->st));

    // terminal: lE = 2 h^3 w E of the final field, then (dD/dy)^T S^T
    PIC_CUDA(cudaMemsetAsync(c->ctrl()->adj_ly, 0, sizeof(c->ctrl()->adj_ly) * 3, c->st));
    {
        const ParticleSet &cs = c->hsets[cur];
        const float *cyo[3] = {cs.o[0], cs.o[1], cs.o[2]};
        PIC_CUDA(launch_adj_zero(c->np, c->ctrl(), c->st));
        const double seed[3] = {2.0 * c->dV * c->adj.w[0], 2.0 * c->dV * c->adj.w[1],
                                2.0 * c->dV * c->adj.w[2]};
        PIC_CUDA(launch_adj_seed(c->ng, c->at<float4>(c->lay.E4), lE4, seed, c->st));
        const int last = c->adj.n_steps - 1;   // the step whose field J measures
        if ((r = adj_solve(c, last & 1))) return r;
        PIC_CUDA(launch_adj_rho(c->np, c->geom, c->ctrl(), cs.cell, cyo, lrho2, qsc, LamOut{},
                                last & 1, c->st));
    }

    bool backup_ready = false;   // the multipliers already sit in the backup
    for (int s = c->adj.nseg - 1; s >= 0; --s) {
        const int a0 = s * K, b0 = std::min(a0 + K, c->adj.n_steps - 1);
        if (s != c->adj.nseg - 1) {
            // recompute the segment from its checkpoint, keeping each step's
            // positions, field and particle order (the last segment was kept
            // by the forward sweep); the multipliers, in checkpoint s + 1's
            // order, wait in the backup while the re-binning uses their arrays
            if (!backup_ready && (r = adj_lam_backup(c, L, cur, true))) return r;
            backup_ready = false;
            if ((r = adj_restore(c, L, s, cur))) return r;
            c->rho_current = false;
            for (int n = a0; n < b0; ++n)
                if ((r = adj_keep_step(c, L, s, a0, n, &cur))) return r;
            const int32_t *pid_next =
                reinterpret_cast<const int32_t *>(order_rec(c, L, s + 1, 0).pid);
            if ((r = adj_permute_from_backup(c, L, cur, pid_next, c->hsets[cur].pid))) return r;
        }
        // reverse steps.  The deposit term of step n is applied by the reverse
        // push of step n - 1 (rt), or on its own where an order starts.
        int rec = (b0 - 1 - a0) / L.R;
        if (b0 > a0 && (r = adj_use_items(c, L, s, rec))) return r;
        AdjRhoTerm rt{};
        for (int n = b0 - 1; n >= a0; --n) {
            char *y[7];
            buf_arrays(c->adj.buf + L.off_segy + (size_t)(n - a0) * L.segy, L.arr, L.ny, y);
            const int32_t *ycell = reinterpret_cast<const int32_t *>(y[0]);
            const float *yo[3] = {reinterpret_cast<const float *>(y[1]),
                                  reinterpret_cast<const float *>(y[2]),
                                  reinterpret_cast<const float *>(y[3])};
            const float4 *En = reinterpret_cast<const float4 *>(c->adj.buf + L.off_segE +
                                                                (size_t)(n - a0) * L.segE);
            PGrad pg{};
            if (pgrad) {
                for (int d = 0; d < 3; ++d) {
                    pg.yv[d] = reinterpret_cast<const float *>(y[4 + d]);
                    pg.half_n[d] = 0.5f * (float)c->geom.n[d];
                    pg.h[d] = (float)c->h[d];
                }
                pg.part = pg_part;
            }
            PIC_CUDA(launch_adj_push(c->geom, c->ctrl(), c->at<int4>(c->lay.items),
                                     (int)c->max_items, ycell, yo, En, lE4, c_kick, dt, wz2, rt,
                                     step_bound(ab, n & 1), pg, c->ctrl(), c->st));
            if (pgrad) PIC_CUDA(launch_pgrad_acc(pg_part, (int)c->max_items, pg_acc, c->st));
            if ((r = adj_solve(c, n & 1))) return r;
            rt.cell = ycell;
            for (int d = 0; d < 3; ++d) rt.o[d] = yo[d];
            rt.lrho2 = lrho2;
            rt.sx = qsc * (float)c->inv_h[0];
            rt.sy = qsc * (float)c->inv_h[1];
            rt.sz = qsc * (float)c->inv_h[2];
            if (rec > 0 && n == a0 + rec * L.R) {
                // order `rec` began at this step: finish the step in it, then
                // move the multipliers to the order before the re-binning
                PIC_CUDA(launch_adj_rho(c->np, c->geom, c->ctrl(), rt.cell, rt.o, lrho2, qsc,
                                        adj_backup_out(c, L), n & 1, c->st));
                rt = AdjRhoTerm{};
                const int32_t *pid_l = reinterpret_cast<const int32_t *>(order_rec(c, L, s, rec).pid);
                const int32_t *pid_e =
                    reinterpret_cast<const int32_t *>(order_rec(c, L, s, rec - 1).pid);
                if ((r = adj_permute_from_backup(c, L, cur, pid_l, pid_e))) return r;
                --rec;
                if ((r = adj_use_items(c, L, s, rec))) return r;
            }
        }
        if (rt.cell) {
            // the segment's first step; before another segment is recomputed
            // the multipliers go to the backup anyway, so write them there
            const bool to_backup = s > 0 && c->np > 0;
            PIC_CUDA(launch_adj_rho(c->np, c->geom, c->ctrl(), rt.cell, rt.o, lrho2, qsc,
                                    to_backup ? adj_backup_out(c, L) : LamOut{}, a0 & 1, c->st));
            backup_ready = to_backup;
        }
    }

    // The multipliers are now in the order of checkpoint 0: restore it (the
    // state the forward sweep started from, re-binned, with its work items).
    if ((r = adj_restore(c, L, 0, cur))) return r;

    // gradients in load order: dJ/dx0 = ly, dJ/dv0 = lv + dt/2 ly
    int32_t *inv = c->at<int32_t>(c->lay.inv);
    PIC_CUDA(launch_invperm(c->np, c->ctrl(), inv, c->st));
    if (dst_is_device) {
        PIC_CUDA(launch_adj_unload(0, c->np, inv, c->ctrl(), 0.5 * c->prm.dt, scale, gx, gv, c->st));
    } else {
        double *sx = c->at<double>(c->lay.stage_x), *sv = c->at<double>(c->lay.stage_v);
        for (int64_t o = 0; o < c->np; o += c->staging) {
            const int64_t m = std::min<int64_t>(c->staging, c->np - o);
            PIC_CUDA(launch_adj_unload(o, m, inv, c->ctrl(), 0.5 * c->prm.dt, scale, sx, sv, c->st));
            PIC_CUDA(cudaMemcpyAsync(gx + 3 * o, sx, (size_t)m * 24, cudaMemcpyDeviceToHost, c->st));
            PIC_CUDA(cudaMemcpyAsync(gv + 3 * o, sv, (size_t)m * 24, cudaMemcpyDeviceToHost, c->st));
        }
    }
    PIC_CUDA(cudaMemcpyAsync(&c->ctrl()->step, &c->adj.step0_dev, sizeof(long long),
                             cudaMemcpyHostToDevice, c->st));
    c->step = c->adj.step0;
    c->since_sort = 0;
    c->adj.cur_end = cur;
    c->adj.ready = false;
    c->rho_current = false;
    double acc[kPGradTerms];
    if (pgrad)
        PIC_CUDA(cudaMemcpyAsync(acc, pg_acc, sizeof(acc), cudaMemcpyDeviceToHost, c->st));
    PIC_CUDA(cudaStreamSynchronize(c->st));
    if (pgrad) {
        // dJ/dB_k = sum_ij (dR/dB_k)_ij A_ij, A_ij = sum lv_tot_i vm_j over
        // particles and steps; dJ/d(wz2) = sum le . Q
        double M[3][9];
        boris_rotation_derivative(c, M);
        for (int k = 0; k < 3; ++k) {
            double g = 0.0;
            for (int q = 0; q < 9; ++q) g += M[k][q] * acc[q];
            c->adj.pgrad[k] = scale * g;
        }
        c->adj.pgrad[3] = scale * acc[9];
        c->adj.pgrad_ready = true;
    }
    return PIC_OK;
}

int pic_adjoint_param_gradient(pic_handle_t c, double grad[4]) {
    int r = check_ready(c);
    if (r) return r;
    if (!grad) return fail(PIC_ERR_ARG, "null output array");
    if (!param_grads(c)) return fail(PIC_ERR_STATE, "created without PIC_OPT_ADJOINT_PARAMS");
    if (!c->adj.pgrad_ready) return fail(PIC_ERR_STATE, "no pic_adjoint_backward since the last forward");
    for (int q = 0; q < 4; ++q) grad[q] = c->adj.pgrad[q];
    return PIC_OK;
}

int pic_dot_f64(pic_handle_t c, const double *x, const double *y, int64_t n, double *out) {
    int r = check_ready(c);
    if (r) return r;
    if (!out || (n > 0 && (!x || !y)) || n < 0) return fail(PIC_ERR_ARG, "bad argument");
    if (n == 0) {
        *out = 0.0;
        return PIC_OK;
    }
    PIC_CUDA(launch_dot(n, x, y, c->at<double>(c->lay.fpart), kDiagFieldBlocks * 4,
                        &c->ctrl()->scalar[1], c->st));
    PIC_CUDA(cudaMemcpyAsync(out, &c->ctrl()->scalar[1], sizeof(double), cudaMemcpyDeviceToHost, c->st));
    PIC_CUDA(cudaStreamSynchronize(c->st));
    return PIC_OK;
}

int pic_enable_timers(pic_handle_t c, int enable) {
    int r = check_ready(c);
    if (r) return r;
    if (enable && !c->events_made) {
        for (int p = 0; p < PIC_PHASE_COUNT; ++p)
            for (int s = 0; s < kTimerRing; ++s)
                for (int e = 0; e < 2; ++e) PIC_CUDA(cudaEventCreate(&c->ev[p][s][e]));
        c->events_made = true;
    }
    if (c->timing) PIC_CUDA(cudaStreamSynchronize(c->st));
    c->timing = enable != 0;
    for (int p = 0; p < PIC_PHASE_COUNT; ++p) {
        c->ev_count[p] = 0;
        c->ev_drained[p] = 0;
        c->ms[p] = 0.0;
    }
    c->launches = 0;
    return PIC_OK;
}

int pic_read_timers(pic_handle_t c, double *ms, int64_t *calls, int64_t *kernel_launches) {
    int r = check_ready(c);
    if (r) return r;
    for (int p = 0; p < PIC_PHASE_COUNT; ++p) {
        if (c->timing && (r = drain_timer(c, p, c->ev_count[p]))) return r;
        if (ms) ms[p] = c->ms[p];
        if (calls) calls[p] = c->ev_count[p];
    }
    if (kernel_launches) *kernel_launches = c->launches;
    return PIC_OK;
}

}  // extern "C"
