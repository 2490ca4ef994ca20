// Internal declarations of the GB300 PIC library: device data layout,
// kernel launchers and the handle.  Not part of the C ABI (see pic.h).
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

#include "pic.h"

namespace pic {

// ----------------------------------------------------------------------------
// Particle store: structure of arrays, 32 bytes per particle.
//   cell  packed stencil-base cell (i | j << 10 | k << 20), i.e. the node
//         index of the lower corner of the particle's CIC stencil
//   o[3]  FP32 offset in [0, 1) of the position from that node, in cells
//   v[3]  FP32 velocity
//   pid   load-order index (touched only by the sort and the readback)
// Two sets exist; the sort scatters from the current one into the other and
// flips Ctrl::cur on the device, so captured CUDA graphs stay valid.
// ----------------------------------------------------------------------------
struct ParticleSet {
    int32_t *cell;
    float *o[3];
    float *v[3];
    int32_t *pid;
};

// Device control block (lives in the arena).  Everything before `cur` is
// cleared when particles are loaded.
struct Ctrl {
    int32_t flags;          // PIC_FLAG_* bits, OR-ed by kernels
    int32_t n_items;        // deposit work items built by the last sort
    unsigned long long stray;   // particles deposited outside their tile (stat)
    long long step;         // steps since the last load
    long long diag_written; // diagnostic records written since the load
    double mode[2];         // tracked Fourier coefficient of the last solve
    double scalar[2];       // objective and dot-product results
    // adjoint sweep: bit patterns of non-negative float maxima (atomicMax on
    // the bits orders them), double-buffered by step parity: |ly|, |lv| of
    // the multipliers and |lrho| of the last adjoint solve
    unsigned int adj_ly[2], adj_lv[2], adj_lrho[2];
    // stray-triggered re-binning: strays of the last push (summed by the push
    // kernels, cleared by each re-binning decision and each re-binning), the
    // pushes since the last re-binning, re-binnings since the load, and the
    // gate the decision sets for the sort kernels of the current step
    unsigned long long stray_step;
    long long rebins;
    int32_t since_sort;
    int32_t rebin;
    int32_t cur;            // which ParticleSet holds the particles
    int32_t pad0;
    ParticleSet sets[2];
};

constexpr int kCellBits = 10;
constexpr int kCellMask = (1 << kCellBits) - 1;
constexpr int kMaxN = 1 << kCellBits;      // 1024 nodes per axis

__host__ __device__ __forceinline__ int32_t pack_cell(int i, int j, int k) {
    return i | (j << kCellBits) | (k << (2 * kCellBits));
}
__host__ __device__ __forceinline__ int cell_i(int32_t c) { return c & kCellMask; }
__host__ __device__ __forceinline__ int cell_j(int32_t c) { return (c >> kCellBits) & kCellMask; }
__host__ __device__ __forceinline__ int cell_k(int32_t c) { return (c >> (2 * kCellBits)) & kCellMask; }

// Grid geometry passed by value to kernels.
struct Geom {
    int n[3];          // nodes per axis
    int nh;            // Nx/2 + 1 (R2C innermost length)
    int tile[3];       // deposit tile (cells per axis)
    int ntile[3];      // tiles per axis = ceil(n / tile)
    int guard;         // guard layers around a tile
    int tvol;          // tile[0]*tile[1]*tile[2]
    unsigned tdiv[3];  // ceil(2^32 / tile[d]), 0 for a tile of 1 (see tile_div)
    float h[3];        // cell size
    float inv_h[3];
};

// a / tile[d] for 0 <= a < 1024 by a multiply-high (exact: the rounding of the
// reciprocal adds less than 2^-22 to a quotient whose fraction is <= 1 - 1/1024)
__device__ __forceinline__ int tile_div(int a, unsigned tdiv) {
    return tdiv ? (int)__umulhi((unsigned)a, tdiv) : a;
}

// Per-step push constants (FP32, precomputed on the host in FP64).
struct PushConst {
    float qm_half_dt;      // (q/m) dt / 2
    float dt_over_h[3];    // dt / h_d
    float t[3];            // (q/m) B dt / 2
    float s[3];            // 2 t / (1 + |t|^2)
    float wz2;             // quadrupole strength
    float half_n[3];       // N_d / 2 (box centre in cells)
};

// Diagnostic partial layout: 4 doubles per block.
constexpr int kDiagFieldBlocks = 512;
constexpr int kNumSMs = 152;   // streaming multiprocessors of the GPU (two dies of 76)
constexpr int kMaxPushBlocks = kNumSMs * 8;
constexpr int kMaxSmemPerBlock = 227 * 1024;   // opt-in shared memory per block
// resident blocks per SM the fused push + deposit kernel is compiled for
#ifndef PIC_PD_MIN_BLOCKS
#define PIC_PD_MIN_BLOCKS 3
#endif
// threads per block of the fused push + deposit, and its grid in waves of
// PIC_PD_MIN_BLOCKS blocks per SM
#ifndef PIC_PD_THREADS
#define PIC_PD_THREADS 256
#endif
#ifndef PIC_PD_WAVES
#define PIC_PD_WAVES 1
#endif
// the fused push + deposit gathers E from a shared-memory copy of its tile's
// box when PIC_PD_MIN_BLOCKS blocks with that copy still fit on an SM
#ifndef PIC_PD_STAGE_E
#define PIC_PD_STAGE_E 1
#endif
// resident blocks per SM of the uniform-plasma move + deposit
#ifndef PIC_MV_MIN_BLOCKS
#define PIC_MV_MIN_BLOCKS 4
#endif
// resident blocks per SM of the split-call deposit
#ifndef PIC_DEP_MIN_BLOCKS
#define PIC_DEP_MIN_BLOCKS 4
#endif
// read and write page-locked host particle arrays in place (no staging copies)
#ifndef PIC_ZERO_COPY
#define PIC_ZERO_COPY 1
#endif
// resident blocks per SM the reverse push is compiled for
#ifndef PIC_ADJ_MIN_BLOCKS
#define PIC_ADJ_MIN_BLOCKS 3
#endif
constexpr int kMaxChunk = 4095;   // fixed-point tile slots stay below 2^32

// Set the thread-local message returned by pic_last_error(); returns `code`.
int record_error(int code, const char *fmt, ...);

// The run of work items [it0, it1) of this block.  Items cover the particles
// [0, P) in order; item i costs its particles plus a fixed kItemCost for its
// tile's fold and flush, so the cost before item i is y_i + kItemCost i, and
// the block takes the items that start within its equal share of the total
// (with fewer items than blocks, block b takes item b).
#ifndef PIC_ITEM_COST
#define PIC_ITEM_COST 1024
#endif
constexpr long long kItemCost = PIC_ITEM_COST;
// Called by every thread of the block (it synchronises): the two item
// indices are found by a two-level search in which each thread tests one
// sample per round, so a block start costs a few dependent loads (two while
// n_items <= blockDim^2), not log2(n_items).
__device__ __forceinline__ void item_run(const int4 *__restrict__ items, int n_items, int &it0,
                                         int &it1) {
    if (n_items <= (int)gridDim.x) {
        // at most one item per block: consecutive blocks (spread over the SMs)
        // take consecutive items, however large
        it0 = min((int)blockIdx.x, n_items);
        it1 = min((int)blockIdx.x + 1, n_items);
        return;
    }
    const long long total =
        n_items > 0 ? (long long)items[n_items - 1].z + kItemCost * n_items : 0;
    const long long c0 = total * blockIdx.x / gridDim.x;
    const long long c1 = total * (blockIdx.x + 1) / gridDim.x;
    auto cost = [&](int i) { return (long long)items[i].y + kItemCost * i; };
    // level 1: sample i_t = (t + 1) * step - 1; the first index with cost >= c lies
    // in the step-wide bucket after the last sample below c
    const int nt = (int)blockDim.x;
    const int step = (n_items + nt - 1) / nt;   // >= 1 when n_items > 0
    const int t = (int)threadIdx.x;
    const int si = min((t + 1) * step, n_items) - 1;
    const long long cs = (n_items > 0 && si >= 0) ? cost(si) : 0;
    const int b0 = __syncthreads_count(n_items > 0 && si >= 0 && cs < c0 && (t + 1) * step <= n_items);
    const int b1 = __syncthreads_count(n_items > 0 && si >= 0 && cs < c1 && (t + 1) * step <= n_items);
    // level 2: the first index with cost >= c lies in [b * step, min(n, (b + 1) * step)):
    // count the costs below c there, blockDim at a time
    const int lo0 = b0 * step, lo1 = b1 * step;
    const int hi0 = min(n_items, lo0 + step), hi1 = min(n_items, lo1 + step);
    int r0 = 0, r1 = 0;
    for (int k = 0; k < step; k += nt) {
        const int j0 = lo0 + k + t, j1 = lo1 + k + t;
        r0 += __syncthreads_count(j0 < hi0 && cost(j0) < c0);
        r1 += __syncthreads_count(j1 < hi1 && cost(j1) < c1);
    }
    it0 = min(n_items, lo0 + r0);
    it1 = blockIdx.x + 1 == gridDim.x ? n_items : min(n_items, lo1 + r1);
}

// ----------------------------------------------------------------------------
// kernel launchers (defined in the k_*.cu files); all enqueue on `st`.
// ----------------------------------------------------------------------------
// max_blocks > 0 caps the grid (blocks then stride over the particles)
cudaError_t launch_load(const double *x, const double *v, int64_t m, int64_t base,
                        const Geom &g, const double *inv_h_d, double dt, Ctrl *ctrl,
                        cudaStream_t st, int max_blocks = 0);
cudaError_t launch_invperm(int64_t n, Ctrl *ctrl, int32_t *inv, cudaStream_t st);
cudaError_t launch_unload(int64_t o0, int64_t m, const int32_t *inv, const Geom &g,
                          const double *h_d, const double *L_d, double dt, const Ctrl *ctrl,
                          double *x, double *v, cudaStream_t st);

cudaError_t exclusive_scan(int32_t *data, int64_t n, int32_t *tmp, cudaStream_t st,
                           const int32_t *gate = nullptr);
cudaError_t sort_prepare();   // kernel attributes; call once per device outside capture
cudaError_t launch_worklist(const int32_t *bin_end, int ntiles, int chunk, int32_t *tile_items,
                            int2 *tile_range, int4 *items, int32_t *scan_tmp, Ctrl *ctrl, int flip,
                            cudaStream_t st);
// presort: the particles are in arbitrary order (just loaded); coarse passes
// by tile key >> shift run first so that no slice overflows the staged table
// gate != nullptr: every kernel of the sort returns at once unless *gate is
// nonzero on the device (the stray-triggered re-binning of pic_step)
cudaError_t launch_sort(int64_t n, const Geom &g, int chunk, Ctrl *ctrl, int32_t *bins,
                        int64_t nbins, int32_t *scan_tmp, int32_t *tile_items,
                        int2 *tile_range, int4 *items, bool presort, cudaStream_t st,
                        const int32_t *gate = nullptr);
// ctrl->rebin = (period > 0 and ctrl->since_sort >= period) or
// ctrl->stray_step > max_strays; clears ctrl->stray_step
cudaError_t launch_rebin_decide(Ctrl *ctrl, long long max_strays, int period, cudaStream_t st);
// kernels launch_sort issues
int sort_launches(int64_t n, int ntiles, bool presort);
// coarse passes + full-key pass over particles [o, o + n) of the current set
// (which stays unchanged); the range ends in set cur ^ (*passes & 1)
cudaError_t launch_sort_range(int64_t n, int64_t o, const Geom &g, Ctrl *ctrl, int32_t *bins,
                              int64_t nbins, int32_t *scan_tmp, int *passes, int *kernels,
                              cudaStream_t st);
cudaError_t launch_flip(Ctrl *ctrl, cudaStream_t st);   // ctrl->cur = 1 - ctrl->cur
// one bounded wait that nothing completes: raises PIC_FLAG_TIMEOUT (pic_selftest_timeout)
cudaError_t launch_timeout_selftest(Ctrl *ctrl, cudaStream_t st);

cudaError_t launch_deposit(int64_t n, const Geom &g, const Ctrl *ctrl, const int4 *items,
                           int max_items, double qscale, float *rho, unsigned long long *rho64,
                           bool fixed, Ctrl *ctrl_w, int grid_blocks, int sparse_below,
                           cudaStream_t st);

cudaError_t launch_rho_finish(const Geom &g, unsigned long long *rho64, float *rho, double qscale,
                              cudaStream_t st);
// the uniform-plasma random move (PIC_OPT_UNIFORM_MOVE) of every particle,
// with the deposit of the new positions when `deposit` (then over the work
// items, like launch_push_deposit); advances the device step counter
cudaError_t launch_move(int64_t np, const Geom &g, uint64_t seed, bool diag, bool fixed, bool deposit,
                        Ctrl *ctrl, const int4 *items, int max_items, float *rho,
                        unsigned long long *rho64, double qscale, int sparse_below, double *part,
                        int blocks, cudaStream_t st);
// dynamic shared memory of the fused push + deposit kernel for geometry g,
// whether it stages E in shared memory, and the one-time attribute setting it
// needs above 48 KiB
size_t push_deposit_smem(const Geom &g);
bool push_stages_E(const Geom &g);
size_t tile_deposit_smem(const Geom &g);   // the deposit tiles alone (unstaged kernels)
cudaError_t push_deposit_prepare(const Geom &g);
// Optional copy of the positions a push starts from (cell, o[3]), written by
// the fused kernel as it reads them (the adjoint keeps each step's y).
struct SaveY {
    int32_t *cell;
    float *o[3];
    float *v[3];   // also the velocities before the kick (null: not saved)
};
// E4: the field, one float4 per node; E8: the x-paired field (launch_pair_E),
// 2 float4 per node
cudaError_t launch_push_deposit(const Geom &g, const PushConst &pc, bool diag, bool fixed,
                                Ctrl *ctrl, const int4 *items, int max_items, const float4 *E4,
                                const float4 *E8, float *rho, unsigned long long *rho64, double qscale,
                                int sparse_below, double *part, int blocks, const SaveY &save,
                                cudaStream_t st);
cudaError_t launch_gather_push(int64_t n, const Geom &g, const PushConst &pc, bool diag,
                               Ctrl *ctrl, const float4 *E8, double *part, int blocks,
                               int threads, cudaStream_t st);
// E8[2q] = E4[q], E8[2q + 1] = E4[q + x (periodic)]
cudaError_t launch_pair_E(const Geom &g, const float4 *E4, float4 *E8, cudaStream_t st);

// FP32 wavenumbers of every FFT index per axis (x: nh, y: ny, z: nz entries)
void green_table(const Geom &g, const double *L_d, float *ktab);
cudaError_t launch_green(const Geom &g, const float *ktab, const float2 *rho_hat,
                         float2 *E_hat, int64_t nhalf, const int *mode_idx, int mode_comp,
                         int mode_conj, Ctrl *ctrl, cudaStream_t st);
cudaError_t launch_diag_field(const Geom &g, const float *rho, const float4 *E4,
                              double *part, cudaStream_t st);
cudaError_t launch_diag_finalize(const double *field_part, const double *push_part,
                                 int push_blocks, double dV, double mp, double dt,
                                 Ctrl *ctrl, pic_diag_t *ring, int ring_cap, cudaStream_t st);

// adjoint (k_adjoint.cu)
cudaError_t launch_adj_seed(int64_t ng, const float4 *E4, float4 *lE4, const double *scale3,
                            cudaStream_t st);
// up to 8 device-to-device copies in one launch (pointers 16-byte aligned)
struct CopyList {
    int count;
    char *dst[8];
    const char *src[8];
    int64_t bytes[8];
};
cudaError_t launch_copy(const CopyList &cl, cudaStream_t st);

// The deposit term of the adjoint of one step, (dD/dy)^T lrho evaluated at
// that step's positions (cell, o) and scaled by q/h_d, folded into the
// reverse push of the step before it (cell == nullptr: no such term).
// Per-step constants of the reverse push of step n: the step's parity and the
// constants of the bound on |le| that scales the integer accumulation of
// G^T le (c = dt q/m; kb = 2 max_d |q / h_d| bounds the deposit term per unit
// |lrho|; with B, |le_d| <= (1 + sqrt 3)/2 |c| max|lv_tot|); with mag set, the
// Boris rotation R (row-major) of v' = R v + (c/2)(R + I) e.
struct AdjBound {
    int par;
    float c_abs, dt, kb;
    int mag;
    float R[9];
};
struct AdjRhoTerm {
    const int32_t *cell;
    const float *o[3];
    const float2 *lrho2;   // x-paired lrho (launch_pair_scalar)
    float sx, sy, sz;
};
// Parameter-gradient sums of one reverse step (part == nullptr: off): per
// block, A_ij = sum_p lv_tot_i vm_j (9, row-major) and sum_p le . Q(y_p)
// (Q the quadrupole direction field), from the saved velocities yv before the
// kick; half_n and h give the box centre in cells and the spacing.
struct PGrad {
    const float *yv[3];
    double *part;   // kPGradTerms doubles per block
    float half_n[3], h[3];
};
constexpr int kPGradTerms = 10;
constexpr int kAdjPushMaxBlocks = kNumSMs * PIC_ADJ_MIN_BLOCKS * 2;
cudaError_t launch_adj_push(const Geom &g, const Ctrl *ctrl, const int4 *items, int max_items,
                            const int32_t *ycell, const float *const yo[3], const float4 *E8,
                            float4 *lE4, float c_kick, float dt, float wz2, const AdjRhoTerm &rt,
                            const AdjBound &ab, const PGrad &pg, Ctrl *ctrl_w, cudaStream_t st);
// acc[q] += the fixed-order sum of the kPGradTerms partials of the blocks the
// last launch_adj_push used (max_items caps them as there)
cudaError_t launch_pgrad_acc(const double *part, int max_items, double *acc, cudaStream_t st);
cudaError_t launch_green_adj(const Geom &g, const double *L_d, const float2 *lE_hat,
                             float2 *lrho_hat, int64_t nhalf, cudaStream_t st);
// where k_adj_rho writes the updated multipliers (o[0] == nullptr: in place)
struct LamOut {
    float *o[3];
    float *v[3];
};
cudaError_t launch_adj_rho(int64_t n, const Geom &g, Ctrl *ctrl, const int32_t *ycell,
                           const float *const yo[3], const float2 *lrho2, float qscale,
                           const LamOut &out, int par, cudaStream_t st);
// lrho2[q] = (lrho[q], lrho[q + x (periodic)]); lE4 cleared
cudaError_t launch_adj_pair_rho(const Geom &g, const float *lrho, float2 *lrho2, float4 *lE4,
                                Ctrl *ctrl, int par, cudaStream_t st);
cudaError_t launch_adj_zero(int64_t n, const Ctrl *ctrl, cudaStream_t st);
struct ReorderArgs {
    const float *in_o[3];
    const float *in_v[3];
    float *out_o[3];
    float *out_v[3];
};
cudaError_t launch_adj_reorder(int64_t n, const int32_t *pos, const int32_t *pid_prev,
                               const float *const in_o[3], const float *const in_v[3],
                               float *const out_o[3], float *const out_v[3], cudaStream_t st);
// pos[pid[j]] = j for j < n (the inverse of a particle order)
cudaError_t launch_pid_positions(int64_t n, const int32_t *pid, int32_t *pos, cudaStream_t st);
cudaError_t launch_adj_unload(int64_t o0, int64_t m, const int32_t *inv, const Ctrl *ctrl,
                              double half_dt, double scale, double *gx, double *gv,
                              cudaStream_t st);
cudaError_t launch_objective(const double *fpart, int nb, double dV, const double *w,
                             double *out, cudaStream_t st);
cudaError_t launch_dot(int64_t n, const double *a, const double *b, double *part, int max_part,
                       double *out, cudaStream_t st);

}  // namespace pic
