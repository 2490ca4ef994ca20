// Batched ensembles: per-instance descriptors and the kernel launchers of
// k_batch.cu (internal; the C ABI is in pic.h).
#pragma once

#include "pic_internal.cuh"

namespace pic {

// resident blocks per SM the batched push + deposit kernel is compiled for
#ifndef PIC_BATCH_PD_MIN_BLOCKS
#define PIC_BATCH_PD_MIN_BLOCKS 3
#endif

// One instance of an ensemble (device copy in the batch arena).
struct InstDesc {
    Geom g;                    // grid, tiles, guard (FP32 spacing)
    PushConst pc;              // push constants of this grid
    long long p0, np;          // its particles: [p0, p0 + np) of the shared store
    long long g0;              // its first node in the concatenated grids
    int tile0, ntiles;         // its global tile ids: [tile0, tile0 + ntiles)
    float qscale;              // q_p / h^3
    double qscale_d, mp, dV;   // FP64 copies for the conversions and reductions
    double inv_h_d[3], h_d[3], L_d[3], two_pi_over_L[3];
    double inv_ng;             // 1 / N_g (folded into the Green kernel)
    int mode_idx[3], mode_comp, mode_conj;
};

cudaError_t launch_b_load(const double *x, const double *v, int64_t m, int64_t base,
                          const InstDesc *desc, const long long *p0, int n_inst, double dt,
                          Ctrl *ctrl, cudaStream_t st);
cudaError_t launch_b_unload(int64_t o0, int64_t m, const int32_t *inv, const InstDesc *desc,
                            const long long *p0, int n_inst, double dt, const Ctrl *ctrl,
                            double *x, double *v, cudaStream_t st);
cudaError_t launch_b_sort(int64_t n, const InstDesc *desc, const long long *p0, int n_inst,
                          int ntiles, int chunk, Ctrl *ctrl, int32_t *bins, int32_t *scan_tmp,
                          int32_t *tile_items, int2 *tile_range, int4 *items, cudaStream_t st);
cudaError_t batch_sort_prepare();   // kernel attributes; once per device outside capture
// shared memory of the batched push + deposit: u32 tile slots + 64-bit per-tile sums
// dynamic shared memory of the batched push + deposit for tiles of up to
// max_S slots, without or with (staged) the copy of the field on the box
size_t batch_push_smem(int max_S, bool staged = false);
// whether blocks of `threads` threads stage the field: the resident blocks
// per SM the kernel is sized for still fit with the staged box
bool batch_stages_E(int max_S, int threads);
// E4: the field, one float4 per node (null: no staging); E8: its x-paired copy
cudaError_t launch_b_push_deposit(bool push, bool diag, bool ext, bool mag, bool fixed,
                                  const InstDesc *desc, const int32_t *tile_inst, Ctrl *ctrl,
                                  const int4 *items, int blocks, int threads, int max_S,
                                  const float4 *E4, const float4 *E8,
                                  float *rho, unsigned long long *rho64, int sparse_below,
                                  double *part, cudaStream_t st);
cudaError_t launch_b_rho_finish(int64_t ng, const InstDesc *desc, const long long *g0, int n_inst,
                                unsigned long long *rho64, float *rho, cudaStream_t st);
cudaError_t launch_b_green(const InstDesc *desc, int first, int m, int64_t nhalf,
                           const float2 *rho_hat, float2 *E_hat, double *modes, cudaStream_t st);
cudaError_t launch_b_diag(const InstDesc *desc, int n_inst, const float *rho, const float4 *E4,
                          double *fpart, cudaStream_t st);
cudaError_t launch_b_diag_finalize(const InstDesc *desc, int n_inst, const int32_t *item_off,
                                   const double *fpart, const double *ppart, const double *modes,
                                   Ctrl *ctrl, double dt, pic_diag_t *ring, int ring_cap,
                                   cudaStream_t st);
// planar E of a size class (grids of nx points per row) -> E4 and x-paired E8
cudaError_t launch_b_pack(int64_t mng, int nx, const float *planar, float4 *E4, float4 *E8,
                          cudaStream_t st);
cudaError_t launch_b_step_done(Ctrl *ctrl, bool diag, cudaStream_t st);

}  // namespace pic
