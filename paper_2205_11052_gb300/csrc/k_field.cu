// Field solve (Section 3.1 step 2, Eq. potential; Section 3.2 of
// arXiv 2205.11052) and the FP64 diagnostic reductions.
//
// Around cuFFT's R2C / C2R transforms, k_green maps the charge spectrum to
// the three field spectra:  -Lap(phi) = rho - rho_i (eps0 = 1), E = -grad(phi)
//   E^_d(m) = -i k_d rho^(m) / |k|^2 / N_g,   k_d = 2 pi m_d / L_d,
// with |k|^2 over the continuous wavenumbers (m_d in [-N_d/2, N_d/2)), the
// k = 0 mode (the uniform ion background) set to zero and each axis' Nyquist
// component of the gradient set to zero so E stays real.  The 1/N_g of the
// inverse transform is folded in here.  The C2R writes E interleaved as
// float4 (Ex, Ey, Ez, 0) so the gather reads one 16-byte vector per node.
//
// Diagnostics (figures of Section 4): W_d = h^3 sum_g E_d^2, Q = h^3 sum_g rho,
// accumulated in FP64 per block in a fixed order, then summed by one block.
#include <math.h>

#include "pic_internal.cuh"

namespace pic {

namespace {

// One thread per coefficient of an x-row (a) of the half spectrum; the row
// (b, c) comes from the block's y and z indices, so no index is divided.
// ktab holds the FP32 wavenumbers of every FFT index per axis (x: nh
// entries, then y: ny, then z: nz), rounded once from FP64 on the host.
__global__ void __launch_bounds__(128) k_green(int nx, int ny, int nz, int nh,
                                               const float *__restrict__ ktab, float inv_ng,
                                               const float2 *__restrict__ rho_hat,
                                               float2 *__restrict__ E_hat, int64_t nhalf, int mi,
                                               int mj, int mk, int mode_comp, int mode_conj,
                                               Ctrl *ctrl) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nh) return;
    const int b = blockIdx.y, c = blockIdx.z;
    const int64_t q = ((int64_t)c * ny + b) * nh + a;
    const float kx = ktab[a], ky = ktab[nh + b], kz = ktab[nh + ny + c];
    const float gx = ((nx & 1) == 0 && a == nx / 2) ? 0.0f : kx;
    const float gy = ((ny & 1) == 0 && b == ny / 2) ? 0.0f : ky;
    const float gz = ((nz & 1) == 0 && c == nz / 2) ? 0.0f : kz;
    const float k2 = kx * kx + ky * ky + kz * kz;
    float2 ex = make_float2(0.f, 0.f), ey = ex, ez = ex;
    if (q != 0) {
        const float2 rh = rho_hat[q];
        const float sc = inv_ng / k2;
        // -i * g * rh = g * (rh.y, -rh.x)
        ex = make_float2(gx * sc * rh.y, -gx * sc * rh.x);
        ey = make_float2(gy * sc * rh.y, -gy * sc * rh.x);
        ez = make_float2(gz * sc * rh.y, -gz * sc * rh.x);
    }
    E_hat[q] = ex;
    E_hat[q + nhalf] = ey;
    E_hat[q + 2 * nhalf] = ez;
    if (a == mi && b == mj && c == mk) {
        const float2 m = (mode_comp == 0) ? ex : (mode_comp == 1 ? ey : ez);
        ctrl->mode[0] = (double)m.x;
        ctrl->mode[1] = mode_conj ? -(double)m.y : (double)m.y;
    }
}

// (hi, lo) += a, with the rounding error of the FP32 sum (Knuth's TwoSum,
// exact in round-to-nearest) carried in lo.
__device__ __forceinline__ void ff_add(float &hi, float &lo, float a) {
    const float s = __fadd_rn(hi, a);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(a, bb));
    lo = __fadd_rn(lo, err);
    hi = s;
}

// (hi, lo) += x^2: the product x*x is split exactly into its rounded value
// and the FMA residual x*x - fl(x*x) (an FP32 product of FP32 inputs is exact
// in 48 bits)
__device__ __forceinline__ void ff_add_sq(float &hi, float &lo, float x) {
    const float p = __fmul_rn(x, x);
    const float e = __fmaf_rn(x, x, -p);
    ff_add(hi, lo, p);
    lo = __fadd_rn(lo, e);
}

// Per-block partial sums of Ex^2, Ey^2, Ez^2 and rho.  Each thread keeps FP32
// (hi, lo) pairs whose error is that of ~48-bit arithmetic (FP64 instructions
// run at a small fraction of the FP32 rate on this part); the pairs are
// combined in FP64 across threads and blocks in a fixed order.
__global__ void __launch_bounds__(256) k_diag_field(int64_t ng, const float *__restrict__ rho,
                                                     const float4 *__restrict__ E4, double *part) {
    float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // two nodes per iteration, both loaded before either is summed
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; g + stride < ng; g += 2 * stride) {
        const float4 e = __ldcs(E4 + g), e2 = __ldcs(E4 + g + stride);
        const float r = __ldcs(rho + g), r2 = __ldcs(rho + g + stride);
        ff_add_sq(hi[0], lo[0], e.x);
        ff_add_sq(hi[1], lo[1], e.y);
        ff_add_sq(hi[2], lo[2], e.z);
        ff_add(hi[3], lo[3], r);
        ff_add_sq(hi[0], lo[0], e2.x);
        ff_add_sq(hi[1], lo[1], e2.y);
        ff_add_sq(hi[2], lo[2], e2.z);
        ff_add(hi[3], lo[3], r2);
    }
    if (g < ng) {
        const float4 e = E4[g];
        ff_add_sq(hi[0], lo[0], e.x);
        ff_add_sq(hi[1], lo[1], e.y);
        ff_add_sq(hi[2], lo[2], e.z);
        ff_add(hi[3], lo[3], rho[g]);
    }
    double s[4];
    for (int q = 0; q < 4; ++q) s[q] = (double)hi[q] + (double)lo[q];
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
        part[4 * blockIdx.x + threadIdx.x] = t;
    }
}

__global__ void k_diag_finalize(const double *__restrict__ fpart, int fblocks,
                                const double *__restrict__ ppart, int pblocks, double dV,
                                double mp, double dt, Ctrl *ctrl, pic_diag_t *ring,
                                int ring_cap) {
    // one block of 256 threads: fixed-order partial sums then a fixed tree
    __shared__ double red[8][256];
    double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < fblocks; b += blockDim.x)
        for (int q = 0; q < 4; ++q) s[q] += fpart[4 * b + q];
    for (int b = threadIdx.x; b < pblocks; b += blockDim.x)
        for (int q = 0; q < 4; ++q) s[4 + q] += ppart[4 * b + q];
    for (int q = 0; q < 8; ++q) red[q][threadIdx.x] = s[q];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int q = 0; q < 8; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const long long step = ctrl->step - 1;   // the push already advanced it
        pic_diag_t d;
        d.step = step;
        d.t_field = ((double)step + 0.5) * dt;
        d.Wx = dV * red[0][0];
        d.Wy = dV * red[1][0];
        d.Wz = dV * red[2][0];
        d.Q = dV * red[3][0];
        d.mode_re = ctrl->mode[0];
        d.mode_im = ctrl->mode[1];
        d.t = ((double)step + 1.0) * dt;
        d.Px = mp * red[4][0];
        d.Py = mp * red[5][0];
        d.Pz = mp * red[6][0];
        d.K = 0.5 * mp * red[7][0];
        const long long slot = ctrl->diag_written % ring_cap;
        ring[slot] = d;
        ctrl->diag_written += 1;
    }
}

}  // namespace

// The push kernels read E through 256-bit loads of x-adjacent node pairs:
// E8[2q] = E at node q, E8[2q + 1] = E at its +x neighbour (periodic).
__global__ void k_pair_E(int nx, int64_t ng, const float4 *__restrict__ E4, float4 *__restrict__ E8) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= ng) return;
    const int64_t row = q / nx;
    const int i = (int)(q - row * nx);
    const int64_t q1 = (i + 1 == nx) ? row * nx : q + 1;
    E8[2 * q] = E4[q];
    E8[2 * q + 1] = E4[q1];
}

cudaError_t launch_pair_E(const Geom &g, const float4 *E4, float4 *E8, cudaStream_t st) {
    const int64_t ng = (int64_t)g.n[0] * g.n[1] * g.n[2];
    k_pair_E<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(g.n[0], ng, E4, E8);
    return cudaGetLastError();
}

void green_table(const Geom &g, const double *L_d, float *ktab) {
    const double two_pi = 6.283185307179586476925286766559;
    int o = 0;
    for (int a = 0; a < g.nh; ++a) ktab[o++] = (float)(two_pi / L_d[0] * a);
    for (int b = 0; b < g.n[1]; ++b) {
        const int m = (b <= g.n[1] / 2) ? b : b - g.n[1];
        ktab[o++] = (float)(two_pi / L_d[1] * m);
    }
    for (int c = 0; c < g.n[2]; ++c) {
        const int m = (c <= g.n[2] / 2) ? c : c - g.n[2];
        ktab[o++] = (float)(two_pi / L_d[2] * m);
    }
}

cudaError_t launch_green(const Geom &g, const float *ktab, const float2 *rho_hat, float2 *E_hat,
                         int64_t nhalf, const int *mode_idx, int mode_comp, int mode_conj,
                         Ctrl *ctrl, cudaStream_t st) {
    const double ng = (double)g.n[0] * g.n[1] * g.n[2];
    const int T = 128;
    const dim3 grid((unsigned)((g.nh + T - 1) / T), (unsigned)g.n[1], (unsigned)g.n[2]);
    k_green<<<grid, T, 0, st>>>(g.n[0], g.n[1], g.n[2], g.nh, ktab, (float)(1.0 / ng), rho_hat,
                                E_hat, nhalf, mode_idx[0], mode_idx[1], mode_idx[2], mode_comp,
                                mode_conj, ctrl);
    return cudaGetLastError();
}

cudaError_t launch_diag_field(const Geom &g, const float *rho, const float4 *E4, double *part,
                              cudaStream_t st) {
    const int64_t ng = (int64_t)g.n[0] * g.n[1] * g.n[2];
    k_diag_field<<<kDiagFieldBlocks, 256, 0, st>>>(ng, rho, E4, part);
    return cudaGetLastError();
}

cudaError_t launch_diag_finalize(const double *field_part, const double *push_part,
                                 int push_blocks, double dV, double mp, double dt, Ctrl *ctrl,
                                 pic_diag_t *ring, int ring_cap, cudaStream_t st) {
    k_diag_finalize<<<1, 256, 0, st>>>(field_part, kDiagFieldBlocks, push_part, push_blocks, dV,
                                       mp, dt, ctrl, ring, ring_cap);
    return cudaGetLastError();
}

}  // namespace pic
