// C ABI of batched ensembles (declared in include/pic.h): many independent
// PIC runs of uneven size advanced by one set of launches per phase.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <vector>

#include "batch.cuh"
#include "cic.cuh"

using namespace pic;

namespace {

#define B_CUDA(call)                                                                         \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return record_error(PIC_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

#define B_CUFFT(call)                                                                          \
    do {                                                                                       \
        cufftResult r_ = (call);                                                               \
        if (r_ != CUFFT_SUCCESS)                                                               \
            return record_error(PIC_ERR_CUFFT, "%s failed: cufftResult %d", #call, (int)r_); \
    } while (0)

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct SizeClass {
    int n[3];
    int first, m;             // internal instances [first, first + m)
    int64_t ng, nhalf;        // per instance
    int64_t g0, h0;           // offsets of the class in the grid / half-spectrum arrays
    cufftHandle r2c, c2r;
};

}  // namespace

struct pic_batch {
    int n_inst;
    pic_params_t prm;
    double qm;
    std::vector<pic_instance_t> inst;     // caller order
    std::vector<int> order;               // internal index -> caller index
    std::vector<int> where;               // caller index -> internal index
    std::vector<InstDesc> desc;           // internal order
    std::vector<long long> p0, g0;        // internal order, with a final total entry
    std::vector<int32_t> tile_inst;
    std::vector<SizeClass> cls;
    int64_t np, ng, nhalf_tot;
    int ntiles, max_items, chunk, sparse_below, fused_blocks, block;
    bool stage_E;   // the push stages each tile's box of E in shared memory
    int max_S;                 // largest tile (plus guard) of any instance, in nodes
    size_t fft_reserve;
    int64_t staging;
    // arena layout
    size_t o_ctrl, o_desc, o_p0, o_g0, o_tinst, o_sets, set_stride, o_rho, o_rho64, o_E4, o_E8, o_rhoh,
        o_Eh, o_Epl, o_bins, o_scan, o_titems, o_trange, o_items, o_fpart, o_ppart, o_modes, o_ring, o_inv,
        o_sx, o_sv, o_fft, total;
    char *arena;
    cudaStream_t st;
    bool bound, loaded, plans, rho_current;
    int64_t step;
    int since_sort;

    template <class T>
    T *at(size_t off) const { return reinterpret_cast<T *>(arena + off); }
    Ctrl *ctrl() const { return at<Ctrl>(o_ctrl); }
};

namespace {

int batch_plans(pic_batch *b, bool estimate, size_t *ws_max) {
    *ws_max = 0;
    for (SizeClass &c : b->cls) {
        long long n[3], nh[3];
        int r = 0;
        if (c.n[2] > 1) { n[r] = c.n[2]; nh[r] = c.n[2]; ++r; }
        if (c.n[1] > 1) { n[r] = c.n[1]; nh[r] = c.n[1]; ++r; }
        n[r] = c.n[0];
        nh[r] = c.n[0] / 2 + 1;
        ++r;
        cufftHandle p1 = 0, p2 = 0;
        B_CUFFT(cufftCreate(&p1));
        cufftResult e = cufftCreate(&p2);
        if (e != CUFFT_SUCCESS) {
            cufftDestroy(p1);
            return record_error(PIC_ERR_CUFFT, "cufftCreate failed: %d", (int)e);
        }
        cufftSetAutoAllocation(p1, 0);
        cufftSetAutoAllocation(p2, 0);
        size_t w1 = 0, w2 = 0;
        if (estimate) {
            e = cufftGetSizeMany64(p1, r, n, nullptr, 1, c.ng, nullptr, 1, c.nhalf, CUFFT_R2C, c.m, &w1);
            if (e == CUFFT_SUCCESS)
                e = cufftGetSizeMany64(p2, r, n, nh, 1, c.nhalf, n, 1, c.ng, CUFFT_C2R, 3 * c.m, &w2);
        } else {
            e = cufftMakePlanMany64(p1, r, n, nullptr, 1, c.ng, nullptr, 1, c.nhalf, CUFFT_R2C, c.m, &w1);
            if (e == CUFFT_SUCCESS)
                e = cufftMakePlanMany64(p2, r, n, nh, 1, c.nhalf, n, 1, c.ng, CUFFT_C2R, 3 * c.m, &w2);
        }
        if (e != CUFFT_SUCCESS || estimate) {
            cufftDestroy(p1);
            cufftDestroy(p2);
            if (e != CUFFT_SUCCESS) return record_error(PIC_ERR_CUFFT, "batched cuFFT plan failed: %d", (int)e);
        } else {
            c.r2c = p1;
            c.c2r = p2;
        }
        *ws_max = std::max(*ws_max, std::max(w1, w2));
    }
    if (!estimate) b->plans = true;
    return PIC_OK;
}

void batch_destroy_plans(pic_batch *b) {
    if (!b->plans) return;
    for (SizeClass &c : b->cls) {
        cufftDestroy(c.r2c);
        cufftDestroy(c.c2r);
    }
    b->plans = false;
}

void batch_layout(pic_batch *b) {
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o += align_up(bytes ? bytes : 1);
        return at;
    };
    const int64_t capn = std::max<int64_t>(b->np, 1);
    b->set_stride = align_up((size_t)capn * 4);
    b->o_ctrl = take(sizeof(Ctrl));
    b->o_desc = take(sizeof(InstDesc) * b->n_inst);
    b->o_p0 = take(sizeof(long long) * (b->n_inst + 1));
    b->o_g0 = take(sizeof(long long) * (b->n_inst + 1));
    b->o_tinst = take(sizeof(int32_t) * b->ntiles);
    b->o_sets = take(2 * 8 * b->set_stride);
    b->o_rho = take((size_t)b->ng * 4);
    b->o_rho64 = take((size_t)b->ng * 8);
    b->o_E4 = take((size_t)b->ng * 16);
    b->o_E8 = take((size_t)b->ng * 32);
    b->o_rhoh = take((size_t)b->nhalf_tot * 8);
    b->o_Eh = take((size_t)b->nhalf_tot * 8 * 3);
    b->o_Epl = take((size_t)b->ng * 4 * 3);
    b->o_bins = take((size_t)(b->ntiles + 1) * 4);
    b->o_scan = take((size_t)((b->ntiles + 4095) / 4096 + 2) * 4);
    b->o_titems = take((size_t)(b->ntiles + 1) * 4);
    b->o_trange = take((size_t)b->ntiles * 8);
    b->o_items = take((size_t)b->max_items * 16);
    b->o_fpart = take((size_t)b->n_inst * 4 * 8);
    b->o_ppart = take((size_t)b->max_items * 4 * 8);
    b->o_modes = take((size_t)b->n_inst * 2 * 8);
    b->o_ring = take((size_t)b->prm.diag_capacity * b->n_inst * sizeof(pic_diag_t));
    b->o_inv = take((size_t)capn * 4);
    b->o_sx = take((size_t)b->staging * 24);
    b->o_sv = take((size_t)b->staging * 24);
    b->o_fft = take(b->fft_reserve);
    b->total = o;
}

int b_ready(const pic_batch *b) {
    if (!b) return record_error(PIC_ERR_ARG, "null batch handle");
    if (!b->bound) return record_error(PIC_ERR_STATE, "no workspace bound (call pic_batch_bind_workspace)");
    return PIC_OK;
}

int b_loaded(const pic_batch *b) {
    int r = b_ready(b);
    if (r) return r;
    if (!b->loaded) return record_error(PIC_ERR_STATE, "no particles loaded (call pic_batch_load_particles)");
    return PIC_OK;
}

bool b_ext(const pic_batch *b) { return b->prm.wz2 != 0.0; }
bool b_mag(const pic_batch *b) {
    return b->prm.B_ext[0] != 0.0 || b->prm.B_ext[1] != 0.0 || b->prm.B_ext[2] != 0.0;
}
bool b_fixed(const pic_batch *b) { return (b->prm.options & PIC_OPT_FIXED_DEPOSIT) != 0; }

int b_deposit_pass(pic_batch *b, bool push, bool diag) {
    if (!b_fixed(b)) B_CUDA(cudaMemsetAsync(b->at<float>(b->o_rho), 0, (size_t)b->ng * 4, b->st));
    B_CUDA(launch_b_push_deposit(push, diag, b_ext(b), b_mag(b), b_fixed(b), b->at<InstDesc>(b->o_desc),
                                 b->at<int32_t>(b->o_tinst), b->ctrl(), b->at<int4>(b->o_items),
                                 b->fused_blocks, b->block, b->max_S,
                                 b->stage_E ? b->at<float4>(b->o_E4) : nullptr,
                                 b->at<float4>(b->o_E8),
                                 b->at<float>(b->o_rho), b->at<unsigned long long>(b->o_rho64),
                                 b->sparse_below, b->at<double>(b->o_ppart), b->st));
    if (b_fixed(b))
        B_CUDA(launch_b_rho_finish(b->ng, b->at<InstDesc>(b->o_desc), b->at<long long>(b->o_g0),
                                   b->n_inst, b->at<unsigned long long>(b->o_rho64),
                                   b->at<float>(b->o_rho), b->st));
    b->rho_current = true;
    return PIC_OK;
}

int b_sort(pic_batch *b) {
    B_CUDA(launch_b_sort(b->np, b->at<InstDesc>(b->o_desc), b->at<long long>(b->o_p0), b->n_inst,
                         b->ntiles, b->chunk, b->ctrl(), b->at<int32_t>(b->o_bins),
                         b->at<int32_t>(b->o_scan), b->at<int32_t>(b->o_titems),
                         b->at<int2>(b->o_trange), b->at<int4>(b->o_items), b->st));
    b->since_sort = 0;
    return PIC_OK;
}

int b_solve(pic_batch *b) {
    float *rho = b->at<float>(b->o_rho);
    float2 *rhoh = b->at<float2>(b->o_rhoh), *Eh = b->at<float2>(b->o_Eh);
    float *E = b->at<float>(b->o_E4);
    for (SizeClass &c : b->cls) {
        B_CUFFT(cufftExecR2C(c.r2c, rho + c.g0, reinterpret_cast<cufftComplex *>(rhoh + c.h0)));
        B_CUDA(launch_b_green(b->at<InstDesc>(b->o_desc), c.first, c.m, c.nhalf, rhoh + c.h0,
                             Eh + 3 * c.h0, b->at<double>(b->o_modes), b->st));
        // 3m inverse transforms into planar (Ex, Ey, Ez) of the class, then interleave
        float *pl = b->at<float>(b->o_Epl) + 3 * c.g0;
        B_CUFFT(cufftExecC2R(c.c2r, reinterpret_cast<cufftComplex *>(Eh + 3 * c.h0), pl));
        B_CUDA(launch_b_pack((int64_t)c.m * c.ng, c.n[0], pl, reinterpret_cast<float4 *>(E) + c.g0,
                             b->at<float4>(b->o_E8) + 2 * c.g0, b->st));
    }
    return PIC_OK;
}

}  // namespace

extern "C" {

int pic_batch_create(const pic_instance_t *inst, int n_inst, double q_over_m,
                     const pic_params_t *params, pic_batch_t *out) {
    if (!inst || !params || !out || n_inst < 1) return record_error(PIC_ERR_ARG, "null argument or no instances");
    *out = nullptr;
    if (!isfinite(q_over_m) || q_over_m == 0.0) return record_error(PIC_ERR_ARG, "q_over_m must be finite and nonzero");
    if (!(isfinite(params->dt) && params->dt > 0.0)) return record_error(PIC_ERR_ARG, "dt must be finite and > 0");
    if (params->chunk != 0 && (params->chunk < 32 || params->chunk > kMaxChunk))
        return record_error(PIC_ERR_ARG, "chunk must be 0 or in 32..%d", kMaxChunk);
    if (params->block != 0 && (params->block < 64 || params->block > 256 || params->block % 32))
        return record_error(PIC_ERR_ARG, "block must be 0 or a multiple of 32 in 64..256");
    if (params->guard < 0 || params->guard > 8) return record_error(PIC_ERR_ARG, "guard outside 0..8");
    if (params->diag_every < 0 || params->diag_capacity < 0) return record_error(PIC_ERR_ARG, "negative diagnostic setting");
    if (params->mode_comp < 0 || params->mode_comp > 2) return record_error(PIC_ERR_ARG, "mode_comp must be 0, 1 or 2");
    if (params->options & ~PIC_OPT_FIXED_DEPOSIT)
        return record_error(PIC_ERR_ARG, "unknown option bits (the uniform-plasma move is not "
                                         "available in ensembles)");
    for (int d = 0; d < 3; ++d)
        if (params->tile[d] < 0 || !isfinite(params->B_ext[d])) return record_error(PIC_ERR_ARG, "bad tile or B_ext");
    if (!isfinite(params->wz2)) return record_error(PIC_ERR_ARG, "wz2 must be finite");
    int64_t np = 0;
    for (int i = 0; i < n_inst; ++i) {
        const pic_instance_t &I = inst[i];
        for (int d = 0; d < 3; ++d) {
            if (I.n[d] < 1 || I.n[d] > kMaxN) return record_error(PIC_ERR_ARG, "instance %d: n[%d] outside 1..%d", i, d, kMaxN);
            if (!(isfinite(I.L[d]) && I.L[d] > 0.0)) return record_error(PIC_ERR_ARG, "instance %d: bad L", i);
            if (2 * abs(params->mode[d]) > I.n[d]) return record_error(PIC_ERR_ARG, "instance %d: mode beyond Nyquist", i);
        }
        if (I.n[0] < 2) return record_error(PIC_ERR_ARG, "instance %d: n[0] must be >= 2", i);
        if (I.n_particles < 0 || !isfinite(I.total_charge)) return record_error(PIC_ERR_ARG, "instance %d: bad particles or charge", i);
        np += I.n_particles;
    }
    if (np > 2147483647LL) return record_error(PIC_ERR_ARG, "more than 2^31-1 particles in total");

    pic_batch *b = new (std::nothrow) pic_batch();
    if (!b) return record_error(PIC_ERR_ARG, "out of host memory");
    b->n_inst = n_inst;
    b->prm = *params;
    if (b->prm.sort_period == 0) b->prm.sort_period = 1;
    if (b->prm.diag_capacity == 0) b->prm.diag_capacity = 256;
    if (b->prm.guard == 0) b->prm.guard = 2;
    b->qm = q_over_m;
    b->inst.assign(inst, inst + n_inst);
    b->chunk = b->prm.chunk ? b->prm.chunk : kMaxChunk;
    b->block = b->prm.block ? b->prm.block : 256;
    b->sparse_below = 64;
    b->np = np;

    // internal order: grouped by grid size (size classes), stable
    std::map<std::vector<int>, std::vector<int>> groups;
    for (int i = 0; i < n_inst; ++i) groups[{inst[i].n[0], inst[i].n[1], inst[i].n[2]}].push_back(i);
    for (auto &kv : groups) {
        SizeClass c;
        c.n[0] = kv.first[0];
        c.n[1] = kv.first[1];
        c.n[2] = kv.first[2];
        c.first = (int)b->order.size();
        c.m = (int)kv.second.size();
        c.ng = (int64_t)c.n[0] * c.n[1] * c.n[2];
        c.nhalf = (int64_t)(c.n[0] / 2 + 1) * c.n[1] * c.n[2];
        b->cls.push_back(c);
        for (int i : kv.second) b->order.push_back(i);
    }
    b->where.assign(n_inst, 0);
    for (int j = 0; j < n_inst; ++j) b->where[b->order[j]] = j;

    const double two_pi = 6.283185307179586476925286766559;
    b->desc.resize(n_inst);
    b->p0.assign(n_inst + 1, 0);
    b->g0.assign(n_inst + 1, 0);
    int64_t g0 = 0, h0 = 0;
    int tile0 = 0;
    int max_S = 1;
    int64_t max_items = 1;
    for (SizeClass &c : b->cls) {
        c.g0 = g0;
        c.h0 = h0;
        for (int j = c.first; j < c.first + c.m; ++j) {
            const pic_instance_t &I = inst[b->order[j]];
            InstDesc D;
            memset(&D, 0, sizeof(D));
            int64_t ntl = 1;
            for (int d = 0; d < 3; ++d) {
                D.g.n[d] = I.n[d];
                D.g.tile[d] = std::min(b->prm.tile[d] ? b->prm.tile[d] : 8, I.n[d]);
                D.g.ntile[d] = (I.n[d] + D.g.tile[d] - 1) / D.g.tile[d];
                ntl *= D.g.ntile[d];
                D.h_d[d] = I.L[d] / I.n[d];
                D.inv_h_d[d] = I.n[d] / I.L[d];
                D.L_d[d] = I.L[d];
                D.two_pi_over_L[d] = two_pi / I.L[d];
                D.g.h[d] = (float)D.h_d[d];
                D.g.inv_h[d] = (float)D.inv_h_d[d];
            }
            D.g.nh = I.n[0] / 2 + 1;
            D.g.guard = b->prm.guard;
            for (int d = 0; d < 3; ++d)
                D.g.tdiv[d] = D.g.tile[d] > 1 ? (unsigned)((((uint64_t)1 << 32) + D.g.tile[d] - 1) / D.g.tile[d]) : 0u;
            D.g.tvol = D.g.tile[0] * D.g.tile[1] * D.g.tile[2];
            // push constants (as in the single-run path)
            const double dt = b->prm.dt;
            double t[3], t2 = 0.0;
            D.pc.qm_half_dt = (float)(0.5 * dt * q_over_m);
            for (int d = 0; d < 3; ++d) {
                D.pc.dt_over_h[d] = (float)(dt * D.inv_h_d[d]);
                t[d] = 0.5 * dt * q_over_m * b->prm.B_ext[d];
                t2 += t[d] * t[d];
            }
            for (int d = 0; d < 3; ++d) {
                D.pc.t[d] = (float)t[d];
                D.pc.s[d] = (float)(2.0 * t[d] / (1.0 + t2));
                D.pc.half_n[d] = (float)(0.5 * I.n[d]);
            }
            D.pc.wz2 = (float)b->prm.wz2;
            D.p0 = b->p0[j];
            D.np = I.n_particles;
            b->p0[j + 1] = b->p0[j] + I.n_particles;
            D.g0 = g0;
            b->g0[j] = g0;
            g0 += c.ng;
            D.tile0 = tile0;
            D.ntiles = (int)ntl;
            for (int64_t q = 0; q < ntl; ++q) b->tile_inst.push_back(j);
            tile0 += (int)ntl;
            D.dV = D.h_d[0] * D.h_d[1] * D.h_d[2];
            const double qp = I.n_particles > 0 ? I.total_charge / (double)I.n_particles : 0.0;
            D.qscale_d = qp / D.dV;
            D.qscale = (float)D.qscale_d;
            D.mp = qp / q_over_m;
            D.inv_ng = 1.0 / (double)c.ng;
            int m[3] = {b->prm.mode[0], b->prm.mode[1], b->prm.mode[2]};
            D.mode_conj = 0;
            if (m[0] < 0) {
                for (int d = 0; d < 3; ++d) m[d] = -m[d];
                D.mode_conj = 1;
            }
            D.mode_idx[0] = m[0];
            D.mode_idx[1] = ((m[1] % I.n[1]) + I.n[1]) % I.n[1];
            D.mode_idx[2] = ((m[2] % I.n[2]) + I.n[2]) % I.n[2];
            D.mode_comp = b->prm.mode_comp;
            const int G = b->prm.guard;
            max_S = std::max(max_S, (D.g.tile[0] + 2 * G + 1) * (D.g.tile[1] + 2 * G + 1) *
                                        (D.g.tile[2] + 2 * G + 1));
            max_items += ntl + (I.n_particles + b->chunk - 1) / b->chunk;
            b->desc[j] = D;
        }
        h0 += (int64_t)c.m * c.nhalf;
    }
    b->g0[n_inst] = g0;
    b->ng = g0;
    b->nhalf_tot = h0;
    b->ntiles = tile0;
    b->max_items = (int)std::min<int64_t>(max_items, 2147483647LL);
    b->max_S = max_S;
    if (batch_push_smem(max_S) > (size_t)kMaxSmemPerBlock) {
        delete b;
        return record_error(PIC_ERR_ARG, "deposit tile plus guard too large for shared memory");
    }
    // two waves of the blocks that fit on an SM (the kernel's register budget
    // is sized for PIC_BATCH_PD_MIN_BLOCKS blocks of 256 threads)
    b->stage_E = batch_stages_E(max_S, b->block);
    const int64_t per_sm = std::max<int64_t>(
        1, std::min<int64_t>((int64_t)PIC_BATCH_PD_MIN_BLOCKS * 256 / b->block,
                             (int64_t)kMaxSmemPerBlock /
                                 std::max<size_t>(1, batch_push_smem(max_S, b->stage_E))));
    b->fused_blocks = (int)std::max<int64_t>(
        1, std::min<int64_t>(b->max_items, (int64_t)kNumSMs * per_sm * 2));
    b->staging = std::max<int64_t>(1, std::min<int64_t>(np, (int64_t)1 << 22));
    size_t ws = 0;
    size_t bound = (size_t)b->nhalf_tot * 8 * 3 + ((size_t)4 << 20);
    if (batch_plans(b, true, &ws) == PIC_OK) bound = std::max(bound, ws);
    b->fft_reserve = bound;
    batch_layout(b);
    *out = b;
    return PIC_OK;
}

int pic_batch_buffer_sizes(pic_batch_t b, pic_bufsizes_t *out) {
    if (!b || !out) return record_error(PIC_ERR_ARG, "null argument");
    out->workspace_bytes = b->total;
    out->workspace_align = kAlign;
    out->particle_capacity = b->np;
    out->grid_nodes = b->ng;
    out->staging_particles = b->staging;
    return PIC_OK;
}

int pic_batch_bind_workspace(pic_batch_t b, void *arena, size_t bytes, void *stream) {
    if (!b || !arena) return record_error(PIC_ERR_ARG, "null argument");
    if ((uintptr_t)arena % kAlign) return record_error(PIC_ERR_ARG, "arena not 256-byte aligned");
    if (bytes < b->total)
        return record_error(PIC_ERR_CAPACITY, "arena of %zu bytes < required %zu", bytes, b->total);
    batch_destroy_plans(b);
    b->bound = b->loaded = false;
    b->arena = static_cast<char *>(arena);
    b->st = static_cast<cudaStream_t>(stream);
    size_t ws = 0;
    int r = batch_plans(b, false, &ws);
    if (r) return r;
    if (ws > b->fft_reserve) {
        batch_destroy_plans(b);
        return record_error(PIC_ERR_CAPACITY, "cuFFT needs %zu work bytes, %zu reserved", ws, b->fft_reserve);
    }
    for (SizeClass &c : b->cls)
        for (cufftHandle p : {c.r2c, c.c2r}) {
            B_CUFFT(cufftSetWorkArea(p, b->arena + b->o_fft));
            B_CUFFT(cufftSetStream(p, b->st));
        }
    B_CUDA(batch_sort_prepare());
    Ctrl h;
    memset(&h, 0, sizeof(h));
    for (int s = 0; s < 2; ++s) {
        char *base = b->arena + b->o_sets + (size_t)s * 8 * b->set_stride;
        h.sets[s].cell = reinterpret_cast<int32_t *>(base);
        for (int d = 0; d < 3; ++d) {
            h.sets[s].o[d] = reinterpret_cast<float *>(base + (size_t)(1 + d) * b->set_stride);
            h.sets[s].v[d] = reinterpret_cast<float *>(base + (size_t)(4 + d) * b->set_stride);
        }
        h.sets[s].pid = reinterpret_cast<int32_t *>(base + (size_t)7 * b->set_stride);
    }
    B_CUDA(cudaMemcpyAsync(b->ctrl(), &h, sizeof(h), cudaMemcpyHostToDevice, b->st));
    B_CUDA(cudaMemcpyAsync(b->at<InstDesc>(b->o_desc), b->desc.data(), sizeof(InstDesc) * b->n_inst,
                           cudaMemcpyHostToDevice, b->st));
    B_CUDA(cudaMemcpyAsync(b->at<long long>(b->o_p0), b->p0.data(), sizeof(long long) * (b->n_inst + 1),
                           cudaMemcpyHostToDevice, b->st));
    B_CUDA(cudaMemcpyAsync(b->at<long long>(b->o_g0), b->g0.data(), sizeof(long long) * (b->n_inst + 1),
                           cudaMemcpyHostToDevice, b->st));
    B_CUDA(cudaMemcpyAsync(b->at<int32_t>(b->o_tinst), b->tile_inst.data(), sizeof(int32_t) * b->ntiles,
                           cudaMemcpyHostToDevice, b->st));
    B_CUDA(cudaMemsetAsync(b->at<char>(b->o_E4), 0, (size_t)b->ng * 16, b->st));
    B_CUDA(cudaMemsetAsync(b->at<char>(b->o_E8), 0, (size_t)b->ng * 32, b->st));
    B_CUDA(cudaMemsetAsync(b->at<char>(b->o_rho), 0, (size_t)b->ng * 4, b->st));
    B_CUDA(cudaMemsetAsync(b->at<char>(b->o_rho64), 0, (size_t)b->ng * 8, b->st));
    B_CUDA(cudaMemsetAsync(b->at<char>(b->o_modes), 0, (size_t)b->n_inst * 16, b->st));
    B_CUDA(cudaStreamSynchronize(b->st));
    b->bound = true;
    return PIC_OK;
}

void pic_batch_destroy(pic_batch_t b) {
    if (!b) return;
    batch_destroy_plans(b);
    delete b;
}

int pic_batch_load_particles(pic_batch_t b, const double *x, const double *v, int src_is_device) {
    int r = b_ready(b);
    if (r) return r;
    if (b->np > 0 && (!x || !v)) return record_error(PIC_ERR_ARG, "null particle array");
    B_CUDA(cudaMemsetAsync(b->ctrl(), 0, offsetof(Ctrl, cur), b->st));
    const InstDesc *desc = b->at<InstDesc>(b->o_desc);
    const long long *p0 = b->at<long long>(b->o_p0);
    double *sx = b->at<double>(b->o_sx), *sv = b->at<double>(b->o_sv);
    int64_t src = 0;   // caller-order offset
    for (int i = 0; i < b->n_inst; ++i) {
        const int j = b->where[i];
        const int64_t n = b->inst[i].n_particles, dst = b->p0[j];
        if (src_is_device) {
            B_CUDA(launch_b_load(x + 3 * src, v + 3 * src, n, dst, desc, p0, b->n_inst, b->prm.dt,
                                 b->ctrl(), b->st));
        } else {
            for (int64_t o = 0; o < n; o += b->staging) {
                const int64_t m = std::min<int64_t>(b->staging, n - o);
                B_CUDA(cudaMemcpyAsync(sx, x + 3 * (src + o), (size_t)m * 24, cudaMemcpyHostToDevice, b->st));
                B_CUDA(cudaMemcpyAsync(sv, v + 3 * (src + o), (size_t)m * 24, cudaMemcpyHostToDevice, b->st));
                B_CUDA(launch_b_load(sx, sv, m, dst + o, desc, p0, b->n_inst, b->prm.dt, b->ctrl(), b->st));
            }
        }
        src += n;
    }
    b->loaded = true;
    b->rho_current = false;
    b->step = 0;
    if ((r = b_sort(b))) return r;
    if (!src_is_device) B_CUDA(cudaStreamSynchronize(b->st));
    return PIC_OK;
}

int pic_batch_step(pic_batch_t b, int n) {
    int r = b_loaded(b);
    if (r) return r;
    if (n < 0) return record_error(PIC_ERR_ARG, "negative step count");
    for (int s = 0; s < n; ++s) {
        if (b->prm.sort_period > 0 && b->since_sort >= b->prm.sort_period && (r = b_sort(b))) return r;
        if (!b->rho_current && (r = b_deposit_pass(b, false, false))) return r;
        if ((r = b_solve(b))) return r;
        const bool diag = b->prm.diag_every > 0 && ((b->step + 1) % b->prm.diag_every == 0);
        if (diag)
            B_CUDA(launch_b_diag(b->at<InstDesc>(b->o_desc), b->n_inst, b->at<float>(b->o_rho),
                                 b->at<float4>(b->o_E4), b->at<double>(b->o_fpart), b->st));
        if ((r = b_deposit_pass(b, true, diag))) return r;
        if (diag)
            B_CUDA(launch_b_diag_finalize(b->at<InstDesc>(b->o_desc), b->n_inst,
                                          b->at<int32_t>(b->o_titems), b->at<double>(b->o_fpart),
                                          b->at<double>(b->o_ppart), b->at<double>(b->o_modes),
                                          b->ctrl(), b->prm.dt, b->at<pic_diag_t>(b->o_ring),
                                          b->prm.diag_capacity, b->st));
        B_CUDA(launch_b_step_done(b->ctrl(), diag, b->st));
        b->step += 1;
        b->since_sort += 1;
    }
    return PIC_OK;
}

int pic_batch_diagnostics(pic_batch_t b, pic_diag_t *out, int max_records, int *n_out) {
    int r = b_ready(b);
    if (r) return r;
    if (n_out) *n_out = 0;
    if (max_records < 0 || (max_records > 0 && !out)) return record_error(PIC_ERR_ARG, "bad output buffer");
    B_CUDA(cudaStreamSynchronize(b->st));
    Ctrl h;
    B_CUDA(cudaMemcpy(&h, b->ctrl(), sizeof(Ctrl), cudaMemcpyDeviceToHost));
    const long long cap = b->prm.diag_capacity;
    const long long have = std::min<long long>(h.diag_written, cap);
    const long long first = h.diag_written - have;
    const long long want = std::min<long long>(have, max_records);
    if (want > 0) {
        std::vector<pic_diag_t> all((size_t)cap * b->n_inst);
        B_CUDA(cudaMemcpy(all.data(), b->at<pic_diag_t>(b->o_ring), all.size() * sizeof(pic_diag_t),
                          cudaMemcpyDeviceToHost));
        for (long long q = 0; q < want; ++q) {
            const size_t slot = (size_t)((first + q) % cap);
            for (int i = 0; i < b->n_inst; ++i)
                out[(size_t)q * b->n_inst + i] = all[slot * b->n_inst + b->where[i]];
        }
    }
    if (n_out) *n_out = (int)want;
    if (h.flags)
        return record_error((h.flags & PIC_FLAG_TIMEOUT) ? PIC_ERR_TIMEOUT : PIC_ERR_DEVICE_FLAG,
                            "device error flags 0x%x", h.flags);
    return PIC_OK;
}

int pic_batch_get_particles(pic_batch_t b, double *x, double *v, int dst_is_device) {
    int r = b_loaded(b);
    if (r) return r;
    if (b->np > 0 && (!x || !v)) return record_error(PIC_ERR_ARG, "null output array");
    int32_t *inv = b->at<int32_t>(b->o_inv);
    B_CUDA(launch_invperm(b->np, b->ctrl(), inv, b->st));
    const InstDesc *desc = b->at<InstDesc>(b->o_desc);
    const long long *p0 = b->at<long long>(b->o_p0);
    double *sx = b->at<double>(b->o_sx), *sv = b->at<double>(b->o_sv);
    int64_t dst = 0;   // caller-order offset
    for (int i = 0; i < b->n_inst; ++i) {
        const int j = b->where[i];
        const int64_t n = b->inst[i].n_particles, src = b->p0[j];
        for (int64_t o = 0; o < n; o += b->staging) {
            const int64_t m = std::min<int64_t>(b->staging, n - o);
            if (dst_is_device) {
                B_CUDA(launch_b_unload(src + o, m, inv, desc, p0, b->n_inst, b->prm.dt, b->ctrl(),
                                       x + 3 * (dst + o), v + 3 * (dst + o), b->st));
            } else {
                B_CUDA(launch_b_unload(src + o, m, inv, desc, p0, b->n_inst, b->prm.dt, b->ctrl(), sx,
                                       sv, b->st));
                B_CUDA(cudaMemcpyAsync(x + 3 * (dst + o), sx, (size_t)m * 24, cudaMemcpyDeviceToHost, b->st));
                B_CUDA(cudaMemcpyAsync(v + 3 * (dst + o), sv, (size_t)m * 24, cudaMemcpyDeviceToHost, b->st));
            }
        }
        dst += n;
    }
    if (!dst_is_device) B_CUDA(cudaStreamSynchronize(b->st));
    return PIC_OK;
}

int pic_batch_set_stream(pic_batch_t b, void *stream) {
    int r = b_ready(b);
    if (r) return r;
    b->st = static_cast<cudaStream_t>(stream);
    for (SizeClass &c : b->cls)
        for (cufftHandle p : {c.r2c, c.c2r}) B_CUFFT(cufftSetStream(p, b->st));
    return PIC_OK;
}

}  // extern "C"
