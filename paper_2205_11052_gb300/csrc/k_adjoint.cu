// Discrete adjoint of the drift-kick-drift step (not in the paper: the
// gradient of the final field energy with respect to the initial phase space).
//
// On the device state y = x_{n+1/2} (cell + offset) and v = v_n, one forward
// step with B = 0 is (Section 3.1 steps 1-4, Section 3.2 of arXiv 2205.11052)
//   e  = G(y) S D(y) + E_ext(y),   v' = v + c e  (c = dt q/m),   y' = y + dt v'.
// Given the adjoints (ly', lv') of (y', v'), the chain rule gives
//   lv  = lv' + dt ly'                         ; le = c lv
//   ly  = ly' + (dG/dy . E)^T le + Ext^T le     (k_adj_push)
//            + (dD/dy)^T S^T G^T le             (G^T le: deposit of the 3-vector
//                                                 le in k_adj_push; S^T in
//                                                 k_green_adj; (dD/dy)^T in
//                                                 k_adj_rho)
// with D the CIC deposit (rho_g = sum_p q_p W_pg / h^3), G the CIC gather with
// the same weights, and S the spectral field operator whose transpose has the
// conjugate symbol +i k_d / |k|^2 (k = 0 and the Nyquist gradient zeroed).
// The objective J = sum_d w_d h^3 sum_g E_d,g^2 seeds lE = 2 h^3 w E (k_adj_seed).
//
// dW/dy of a CIC weight w_a(fx) w_b(fy) w_c(fz): d w_1 / dx = 1/h, d w_0 / dx = -1/h.
#include <algorithm>

#include "pic_internal.cuh"

namespace pic {

namespace {

__device__ __forceinline__ bool decode(int32_t c, const Geom &g, int &i, int &j, int &k) {
    i = cell_i(c);
    j = cell_j(c);
    k = cell_k(c);
    if (i >= g.n[0] || j >= g.n[1] || k >= g.n[2]) {
        i = j = k = 0;
        return false;
    }
    return true;
}

__device__ __forceinline__ void nodes8(const Geom &g, int i, int j, int k, int64_t nd[8]) {
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

// weights and their gradients for the 8 corners (corner bits a | b<<1 | c<<2)
__device__ __forceinline__ void weights_and_grads(float fx, float fy, float fz, const Geom &g,
                                                  float w[8], float dwx[8], float dwy[8],
                                                  float dwz[8]) {
    const float ax[2] = {1.0f - fx, fx}, ay[2] = {1.0f - fy, fy}, az[2] = {1.0f - fz, fz};
    const float sx[2] = {-g.inv_h[0], g.inv_h[0]};
    const float sy[2] = {-g.inv_h[1], g.inv_h[1]};
    const float sz[2] = {-g.inv_h[2], g.inv_h[2]};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int a = c & 1, b = (c >> 1) & 1, d = (c >> 2) & 1;
        w[c] = ax[a] * ay[b] * az[d];
        dwx[c] = sx[a] * ay[b] * az[d];
        dwy[c] = ax[a] * sy[b] * az[d];
        dwz[c] = ax[a] * ay[b] * sz[d];
    }
}

__device__ __forceinline__ int tile_slot(int a, int o, int n, int T, int G) {
    int d = a - o;
    if (d < 0) d += n;
    if (d >= T + G) {
        d -= n;
        if (d < -G) return -1;
    }
    return d + G;
}

// lE = 2 h^3 w_d E_d  (terminal seed)
__global__ void k_adj_seed(int64_t ng, const float4 *__restrict__ E4, float4 *__restrict__ lE4,
                           float sx, float sy, float sz) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < ng; q += stride) {
        const float4 e = E4[q];
        lE4[q] = make_float4(sx * e.x, sy * e.y, sz * e.z, 0.0f);
    }
}

// reverse push: lv <- lv + dt ly; le = c lv; ly += (dG/dy . E)^T le + Ext^T le;
// lE += G^T le (shared-memory tile per work item, strays with global atomics)
__global__ void __launch_bounds__(256) k_adj_push(Geom g, const Ctrl *__restrict__ ctrl,
                                                   const int4 *__restrict__ items,
                                                   const int32_t *__restrict__ ycell,
                                                   const float *__restrict__ yo0,
                                                   const float *__restrict__ yo1,
                                                   const float *__restrict__ yo2,
                                                   const float4 *__restrict__ E4,
                                                   float4 *__restrict__ lE4, float c_kick,
                                                   float dt, float wz2, Ctrl *ctrl_w) {
    extern __shared__ float acc[];   // 3 * S floats: x, y, z components
    const int cur = ctrl->cur;
    const ParticleSet lam = ctrl->sets[1 - cur];   // ly in o[], lv in v[]
    const int n_items = ctrl->n_items;
    const int G = g.guard;
    const int S0 = g.tile[0] + 2 * G + 1, S1 = g.tile[1] + 2 * G + 1, S2 = g.tile[2] + 2 * G + 1;
    const int S01 = S0 * S1, S = S01 * S2;
    int bad = 0;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int4 item = items[it];
        const int tile = item.x;
        const int tx = tile % g.ntile[0];
        const int ty = (tile / g.ntile[0]) % g.ntile[1];
        const int tz = tile / (g.ntile[0] * g.ntile[1]);
        const int ox = tx * g.tile[0], oy = ty * g.tile[1], oz = tz * g.tile[2];
        for (int s = threadIdx.x; s < 3 * S; s += blockDim.x) acc[s] = 0.0f;
        __syncthreads();
        for (int p = item.y + threadIdx.x; p < item.z; p += blockDim.x) {
            int i, j, k;
            if (!decode(ycell[p], g, i, j, k)) bad = 1;
            float w[8], dwx[8], dwy[8], dwz[8];
            weights_and_grads(yo0[p], yo1[p], yo2[p], g, w, dwx, dwy, dwz);
            int64_t nd[8];
            nodes8(g, i, j, k, nd);
            float ly[3] = {lam.o[0][p], lam.o[1][p], lam.o[2][p]};
            float lv[3] = {lam.v[0][p], lam.v[1][p], lam.v[2][p]};
#pragma unroll
            for (int d = 0; d < 3; ++d) lv[d] += dt * ly[d];
            const float le[3] = {c_kick * lv[0], c_kick * lv[1], c_kick * lv[2]};
            float tx_ = 0.f, ty_ = 0.f, tz_ = 0.f;
#pragma unroll
            for (int cc = 0; cc < 8; ++cc) {
                const float4 e = __ldg(E4 + nd[cc]);
                const float s = le[0] * e.x + le[1] * e.y + le[2] * e.z;
                tx_ += dwx[cc] * s;
                ty_ += dwy[cc] * s;
                tz_ += dwz[cc] * s;
            }
            ly[0] += tx_ - 0.5f * wz2 * le[0];
            ly[1] += ty_ - 0.5f * wz2 * le[1];
            ly[2] += tz_ + wz2 * le[2];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                lam.o[d][p] = ly[d];
                lam.v[d][p] = lv[d];
            }
            // G^T le
            const int si = tile_slot(i, ox, g.n[0], g.tile[0], G);
            const int sj = tile_slot(j, oy, g.n[1], g.tile[1], G);
            const int sk = tile_slot(k, oz, g.n[2], g.tile[2], G);
            if (si >= 0 && sj >= 0 && sk >= 0) {
                const int s = si + S0 * sj + S01 * sk;
                const int off[8] = {0, 1, S0, S0 + 1, S01, S01 + 1, S01 + S0, S01 + S0 + 1};
#pragma unroll
                for (int cc = 0; cc < 8; ++cc) {
                    atomicAdd(acc + s + off[cc], w[cc] * le[0]);
                    atomicAdd(acc + S + s + off[cc], w[cc] * le[1]);
                    atomicAdd(acc + 2 * S + s + off[cc], w[cc] * le[2]);
                }
            } else {
#pragma unroll
                for (int cc = 0; cc < 8; ++cc) {
                    float *dst = reinterpret_cast<float *>(lE4 + nd[cc]);
                    atomicAdd(dst + 0, w[cc] * le[0]);
                    atomicAdd(dst + 1, w[cc] * le[1]);
                    atomicAdd(dst + 2, w[cc] * le[2]);
                }
            }
        }
        __syncthreads();
        for (int s = threadIdx.x; s < S; s += blockDim.x) {
            const float ax = acc[s], ay = acc[S + s], az = acc[2 * S + s];
            if (ax != 0.0f || ay != 0.0f || az != 0.0f) {
                const int a = s % S0, b = (s / S0) % S1, cz = s / S01;
                int gi = (ox - G + a) % g.n[0];
                int gj = (oy - G + b) % g.n[1];
                int gk = (oz - G + cz) % g.n[2];
                if (gi < 0) gi += g.n[0];
                if (gj < 0) gj += g.n[1];
                if (gk < 0) gk += g.n[2];
                float *dst = reinterpret_cast<float *>(
                    lE4 + gi + (int64_t)g.n[0] * (gj + (int64_t)g.n[1] * gk));
                atomicAdd(dst + 0, ax);
                atomicAdd(dst + 1, ay);
                atomicAdd(dst + 2, az);
            }
        }
        __syncthreads();
    }
    if (bad) atomicOr(&ctrl_w->flags, PIC_FLAG_BAD_CELL);
}

// lrho^ = sum_d (+i g_d / |k|^2) lE^_d / N_g   (S^T, with the C2R 1/N_g folded in)
__global__ void k_green_adj(int nx, int ny, int nz, int nh, double tpx, double tpy, double tpz,
                            double inv_ng, const float2 *__restrict__ lE_hat,
                            float2 *__restrict__ lrho_hat, int64_t nhalf) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nhalf) return;
    const int a = (int)(q % nh);
    const int64_t r = q / nh;
    const int b = (int)(r % ny);
    const int c = (int)(r / ny);
    const int my = (b <= ny / 2) ? b : b - ny;
    const int mz = (c <= nz / 2) ? c : c - nz;
    const float kx = (float)(tpx * a), ky = (float)(tpy * my), kz = (float)(tpz * mz);
    const float gx = ((nx & 1) == 0 && a == nx / 2) ? 0.0f : kx;
    const float gy = ((ny & 1) == 0 && b == ny / 2) ? 0.0f : ky;
    const float gz = ((nz & 1) == 0 && c == nz / 2) ? 0.0f : kz;
    float2 out = make_float2(0.f, 0.f);
    if (q != 0) {
        const float k2 = kx * kx + ky * ky + kz * kz;
        const float sc = (float)inv_ng / k2;
        const float2 ex = lE_hat[q], ey = lE_hat[q + nhalf], ez = lE_hat[q + 2 * nhalf];
        // +i g (re + i im) = g (-im + i re)
        const float sr = -(gx * ex.y + gy * ey.y + gz * ez.y);
        const float si = gx * ex.x + gy * ey.x + gz * ez.x;
        out = make_float2(sc * sr, sc * si);
    }
    lrho_hat[q] = out;
}

// ly += (q_p / h^3) sum_corner grad W lrho  ((dD/dy)^T lrho)
__global__ void k_adj_rho(int64_t n, Geom g, const Ctrl *__restrict__ ctrl,
                          const int32_t *__restrict__ ycell, const float *__restrict__ yo0,
                          const float *__restrict__ yo1, const float *__restrict__ yo2,
                          const float *__restrict__ lrho, float qscale) {
    const ParticleSet lam = ctrl->sets[1 - ctrl->cur];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        int i, j, k;
        decode(ycell[p], g, i, j, k);
        float w[8], dwx[8], dwy[8], dwz[8];
        weights_and_grads(yo0[p], yo1[p], yo2[p], g, w, dwx, dwy, dwz);
        int64_t nd[8];
        nodes8(g, i, j, k, nd);
        float tx = 0.f, ty = 0.f, tz = 0.f;
#pragma unroll
        for (int cc = 0; cc < 8; ++cc) {
            const float r = __ldg(lrho + nd[cc]);
            tx += dwx[cc] * r;
            ty += dwy[cc] * r;
            tz += dwz[cc] * r;
        }
        lam.o[0][p] += qscale * tx;
        lam.o[1][p] += qscale * ty;
        lam.o[2][p] += qscale * tz;
    }
}

__global__ void k_adj_zero(int64_t n, const Ctrl *__restrict__ ctrl) {
    const ParticleSet lam = ctrl->sets[1 - ctrl->cur];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            lam.o[d][p] = 0.0f;
            lam.v[d][p] = 0.0f;
        }
    }
}

// dJ/dx0 = ly_0, dJ/dv0 = lv_0 + dt/2 ly_0 (y_0 = x_0 + dt/2 v_0), in load
// order, scaled by the caller's upstream gradient
__global__ void k_adj_unload(int64_t o0, int64_t m, const int32_t *__restrict__ inv,
                             const Ctrl *__restrict__ ctrl, double half_dt, double scale,
                             double *__restrict__ gx, double *__restrict__ gv) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= m) return;
    const ParticleSet lam = ctrl->sets[1 - ctrl->cur];
    const int64_t p = inv[o0 + q];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double ly = lam.o[d][p], lv = lam.v[d][p];
        gx[3 * q + d] = scale * ly;
        gv[3 * q + d] = scale * (lv + half_dt * ly);
    }
}

// J = h^3 sum_d w_d sum_g E_d^2 from the per-block field partials
__global__ void k_objective(const double *__restrict__ fpart, int nb, double dV, double w0,
                            double w1, double w2, double *out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        s += w0 * fpart[4 * b] + w1 * fpart[4 * b + 1] + w2 * fpart[4 * b + 2];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = dV * red[0];
}

// out = sum_i a_i b_i in FP64, fixed order (per-block partials, then one block)
__global__ void k_dot_partials(int64_t n, const double *__restrict__ a,
                               const double *__restrict__ b, double *part) {
    __shared__ double red[256];
    double s = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride)
        s += a[q] * b[q];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_dot_final(const double *__restrict__ part, int nb, double *out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int q = threadIdx.x; q < nb; q += blockDim.x) s += part[q];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

}  // namespace

cudaError_t launch_adj_seed(int64_t ng, const float4 *E4, float4 *lE4, const double *scale3,
                            cudaStream_t st) {
    const int b = (int)std::min<int64_t>((ng + 255) / 256, 152 * 8);
    k_adj_seed<<<b, 256, 0, st>>>(ng, E4, lE4, (float)scale3[0], (float)scale3[1],
                                  (float)scale3[2]);
    return cudaGetLastError();
}

cudaError_t launch_adj_push(const Geom &g, const Ctrl *ctrl, const int4 *items, int max_items,
                            const int32_t *ycell, const float *const yo[3], const float4 *E4,
                            float4 *lE4, float c_kick, float dt, float wz2, Ctrl *ctrl_w,
                            cudaStream_t st) {
    const int S = (g.tile[0] + 2 * g.guard + 1) * (g.tile[1] + 2 * g.guard + 1) *
                  (g.tile[2] + 2 * g.guard + 1);
    const size_t smem = sizeof(float) * 3 * (size_t)S;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_adj_push, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int blocks = std::max(1, std::min(152 * 4, max_items));
    k_adj_push<<<blocks, 256, smem, st>>>(g, ctrl, items, ycell, yo[0], yo[1], yo[2], E4, lE4,
                                          c_kick, dt, wz2, ctrl_w);
    return cudaGetLastError();
}

cudaError_t launch_green_adj(const Geom &g, const double *L_d, const float2 *lE_hat,
                             float2 *lrho_hat, int64_t nhalf, cudaStream_t st) {
    const double two_pi = 6.283185307179586476925286766559;
    const double ng = (double)g.n[0] * g.n[1] * g.n[2];
    k_green_adj<<<(unsigned)((nhalf + 255) / 256), 256, 0, st>>>(
        g.n[0], g.n[1], g.n[2], g.nh, two_pi / L_d[0], two_pi / L_d[1], two_pi / L_d[2], 1.0 / ng,
        lE_hat, lrho_hat, nhalf);
    return cudaGetLastError();
}

cudaError_t launch_adj_rho(int64_t n, const Geom &g, const Ctrl *ctrl, const int32_t *ycell,
                           const float *const yo[3], const float *lrho, float qscale,
                           cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int b = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
    k_adj_rho<<<b, 256, 0, st>>>(n, g, ctrl, ycell, yo[0], yo[1], yo[2], lrho, qscale);
    return cudaGetLastError();
}

cudaError_t launch_adj_zero(int64_t n, const Ctrl *ctrl, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int b = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
    k_adj_zero<<<b, 256, 0, st>>>(n, ctrl);
    return cudaGetLastError();
}

cudaError_t launch_adj_unload(int64_t o0, int64_t m, const int32_t *inv, const Ctrl *ctrl,
                              double half_dt, double scale, double *gx, double *gv,
                              cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    k_adj_unload<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(o0, m, inv, ctrl, half_dt, scale,
                                                              gx, gv);
    return cudaGetLastError();
}

cudaError_t launch_objective(const double *fpart, int nb, double dV, const double *w,
                             double *out, cudaStream_t st) {
    k_objective<<<1, 256, 0, st>>>(fpart, nb, dV, w[0], w[1], w[2], out);
    return cudaGetLastError();
}

cudaError_t launch_dot(int64_t n, const double *a, const double *b, double *part, int max_part,
                       double *out, cudaStream_t st) {
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, max_part));
    k_dot_partials<<<nb, 256, 0, st>>>(n, a, b, part);
    k_dot_final<<<1, 256, 0, st>>>(part, nb, out);
    return cudaGetLastError();
}

}  // namespace pic
