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

#include "cic.cuh"
#include "push.cuh"
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

// warp-reduced maximum of a non-negative float, merged into *dst (float bits)
__device__ __forceinline__ void max_to(unsigned int *dst, float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v > 0.0f) atomicMax(dst, __float_as_uint(v));
}

// the 8 corner nodes of cell (i, j, k), corner bits a | b<<1 | c<<2 (int32:
// grids have at most 2^30 nodes)
__device__ __forceinline__ void corners(int i, int j, int k, int nx, int ny, int nz, int nd[8]) {
    const int i1 = (i + 1 == nx) ? 0 : i + 1;
    const int j1 = (j + 1 == ny) ? 0 : j + 1;
    const int k1 = (k + 1 == nz) ? 0 : k + 1;
    const int r00 = (j + ny * k) * nx, r10 = (j1 + ny * k) * nx;
    const int r01 = (j + ny * k1) * nx, r11 = (j1 + ny * k1) * nx;
    nd[0] = r00 + i; nd[1] = r00 + i1; nd[2] = r10 + i; nd[3] = r10 + i1;
    nd[4] = r01 + i; nd[5] = r01 + i1; nd[6] = r11 + i; nd[7] = r11 + i1;
}

// the 8 corner values of an x-paired scalar grid (v2[q] = (v[q], v[q + x])):
// four aligned 8-byte loads, corner bits a | b<<1 | c<<2
__device__ __forceinline__ void corners_from_pairs(const float2 *__restrict__ v2, int i, int j,
                                                   int k, int nx, int ny, int nz, float sc[8]) {
    const int j1 = (j + 1 == ny) ? 0 : j + 1;
    const int k1 = (k + 1 == nz) ? 0 : k + 1;
    const float2 a = __ldg(v2 + (j + ny * k) * nx + i), b = __ldg(v2 + (j1 + ny * k) * nx + i);
    const float2 c = __ldg(v2 + (j + ny * k1) * nx + i), d = __ldg(v2 + (j1 + ny * k1) * nx + i);
    sc[0] = a.x; sc[1] = a.y; sc[2] = b.x; sc[3] = b.y;
    sc[4] = c.x; sc[5] = c.y; sc[6] = d.x; sc[7] = d.y;
}

// Gradient, with respect to the in-cell offsets (fx, fy, fz), of the CIC
// interpolation sum_abc w_abc s_abc with w_abc = ax_a ay_b az_c
// (ax_0 = 1 - fx, ax_1 = fx): d/dfx = sum_bc ay_b az_c (s_1bc - s_0bc),
// likewise along y and z.  Multiply by 1/h for the gradient in y.
__device__ __forceinline__ void interp_grad(float fx, float fy, float fz, const float sc[8],
                                            float &dx, float &dy, float &dz) {
    const float gx = 1.0f - fx, gy = 1.0f - fy, gz = 1.0f - fz;
    dx = gy * gz * (sc[1] - sc[0]) + fy * gz * (sc[3] - sc[2]) + gy * fz * (sc[5] - sc[4]) +
         fy * fz * (sc[7] - sc[6]);
    dy = gx * gz * (sc[2] - sc[0]) + fx * gz * (sc[3] - sc[1]) + gx * fz * (sc[6] - sc[4]) +
         fx * fz * (sc[7] - sc[5]);
    dz = gx * gy * (sc[4] - sc[0]) + fx * gy * (sc[5] - sc[1]) + gx * fy * (sc[6] - sc[2]) +
         fx * fy * (sc[7] - sc[3]);
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

// reverse push: [ly += (dD/dy)^T lrho of the following step, when given;]
// lv_tot = lv + dt ly; le = c lv_tot, lv <- lv_tot (with B: le = (c/2)(R^T + I)
// lv_tot, lv <- R^T lv_tot); ly += (dG/dy . E)^T le + Ext^T le;
// lE += G^T le (shared-memory tile per work item, strays with global atomics;
// global updates are one 16-byte vector atomic per node).
//
// The gather term is the offset gradient (interp_grad) of the CIC
// interpolation of s_abc = le . E at the 8 corners.
template <bool PG>
__global__ void __launch_bounds__(256, PIC_ADJ_MIN_BLOCKS) k_adj_push(Geom g, const Ctrl *__restrict__ ctrl,
                                                      const int4 *__restrict__ items,
                                                      const int32_t *__restrict__ ycell,
                                                      const float *__restrict__ yo0,
                                                      const float *__restrict__ yo1,
                                                      const float *__restrict__ yo2,
                                                      const float4 *__restrict__ E8,
                                                      float4 *__restrict__ lE4, float c_kick,
                                                      float dt, float wz2, AdjRhoTerm rt,
                                                      AdjBound ab, PGrad pg, Ctrl *ctrl_w) {
    // 3 * S integer accumulators (x, y, z components) in units of 1 / qs
    extern __shared__ int acc[];
    const int cur = ctrl->cur;
    // |le| <= c (|lv| + dt (|ly| + kb |lrho|)) with the maxima left by the
    // kernels that wrote lv, ly and lrho (read slot: the other parity); a node
    // of an item gets at most 4095 contributions w |le| <= |le|, so
    // qs = 2^(30 - e) with 4096 |le|max < 2^e keeps every sum below 2^30
    const int rd = ab.par ^ 1;
    const float m_ly = __uint_as_float(ctrl->adj_ly[rd]);
    const float m_lv = __uint_as_float(ctrl->adj_lv[rd]);
    const float m_rho = rt.cell ? __uint_as_float(ctrl->adj_lrho[rd]) : 0.0f;
    const float m_le = ab.c_abs * (ab.mag ? 1.3660255f : 1.0f) *
                       (m_lv + ab.dt * (m_ly + ab.kb * m_rho));
    float qs = 1073741824.0f;   // 2^30 when every |le| is 0
    int nonfinite = 0;
    if (!(m_le <= 3.0e38f)) {
        nonfinite = 1;
        qs = 1.0f;
    } else if (m_le > 0.0f) {
        int e;
        frexpf(4096.0f * m_le, &e);
        qs = ldexpf(1.0f, max(-120, min(120, 30 - e)));
    }
    const float inv_qs = 1.0f / qs;   // exact: a power of two
    if (blockIdx.x == 0 && threadIdx.x == 0) ctrl_w->adj_lrho[ab.par] = 0u;   // for this step's solve
    float mly = 0.0f, mlv = 0.0f;
    const ParticleSet lam = ctrl->sets[1 - cur];   // ly in o[], lv in v[]
    const int n_items = ctrl->n_items;
    const int G = g.guard;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int S0 = g.tile[0] + 2 * G + 1, S1 = g.tile[1] + 2 * G + 1, S2 = g.tile[2] + 2 * G + 1;
    const int S01 = S0 * S1, S = S01 * S2;
    int bad = 0;
    // PG: sum_p lv_tot_i vm_j (row-major) and sum_p le . Q
    float pa[kPGradTerms];
#pragma unroll
    for (int q = 0; q < kPGradTerms; ++q) pa[q] = 0.0f;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int4 item = items[it];
        const int tile = item.x;
        const int tx = tile % g.ntile[0];
        const int ty = (tile / g.ntile[0]) % g.ntile[1];
        const int tz = tile / (g.ntile[0] * g.ntile[1]);
        const int ox = tx * g.tile[0], oy = ty * g.tile[1], oz = tz * g.tile[2];
        const cic::Tile tb = cic::tile_of(g, tile);
        for (int q = threadIdx.x; q < 3 * S; q += blockDim.x) acc[q] = 0;
        __syncthreads();
        // the next particle's position and multipliers are loaded before the
        // current one is reversed
        int p = item.y + threadIdx.x;
        int32_t nyc = 0;
        float nly0 = 0.f, nly1 = 0.f, nly2 = 0.f, nfx = 0.f, nfy = 0.f, nfz = 0.f;
        float nlv0 = 0.f, nlv1 = 0.f, nlv2 = 0.f;
        if (p < item.z) {
            nyc = ycell[p];
            nly0 = lam.o[0][p]; nly1 = lam.o[1][p]; nly2 = lam.o[2][p];
            nfx = yo0[p]; nfy = yo1[p]; nfz = yo2[p];
            nlv0 = lam.v[0][p]; nlv1 = lam.v[1][p]; nlv2 = lam.v[2][p];
        }
        for (; p < item.z; p += blockDim.x) {
            int i, j, k;
            if (!decode(nyc, g, i, j, k)) bad = 1;
            float ly0 = nly0, ly1 = nly1, ly2 = nly2;
            const float fx = nfx, fy = nfy, fz = nfz;
            const float plv0 = nlv0, plv1 = nlv1, plv2 = nlv2;
            {
                const int pn = p + (int)blockDim.x;
                if (pn < item.z) {
                    nyc = ycell[pn];
                    nly0 = lam.o[0][pn]; nly1 = lam.o[1][pn]; nly2 = lam.o[2][pn];
                    nfx = yo0[pn]; nfy = yo1[pn]; nfz = yo2[pn];
                    nlv0 = lam.v[0][pn]; nlv1 = lam.v[1][pn]; nlv2 = lam.v[2][pn];
                }
            }
            if (rt.cell) {
                // the deposit term (dD/dy)^T lrho of the step after this one
                int ri, rj, rk;
                decode(rt.cell[p], g, ri, rj, rk);
                float rs[8];
                corners_from_pairs(rt.lrho2, ri, rj, rk, nx, ny, nz, rs);
                float rx, ry, rz;
                interp_grad(rt.o[0][p], rt.o[1][p], rt.o[2][p], rs, rx, ry, rz);
                ly0 += rt.sx * rx;
                ly1 += rt.sy * ry;
                ly2 += rt.sz * rz;
            }
            float lv0 = plv0 + dt * ly0;
            float lv1 = plv1 + dt * ly1;
            float lv2 = plv2 + dt * ly2;
            const float lt0 = lv0, lt1 = lv1, lt2 = lv2;   // lv_tot (for PG)
            float le0, le1, le2;
            if (ab.mag) {
                // lv <- R^T lv_tot, le = (c/2)(R^T lv_tot + lv_tot)
                const float r0 = ab.R[0] * lv0 + ab.R[3] * lv1 + ab.R[6] * lv2;
                const float r1 = ab.R[1] * lv0 + ab.R[4] * lv1 + ab.R[7] * lv2;
                const float r2 = ab.R[2] * lv0 + ab.R[5] * lv1 + ab.R[8] * lv2;
                const float hc = 0.5f * c_kick;
                le0 = hc * (r0 + lv0);
                le1 = hc * (r1 + lv1);
                le2 = hc * (r2 + lv2);
                lv0 = r0;
                lv1 = r1;
                lv2 = r2;
            } else {
                le0 = c_kick * lv0;
                le1 = c_kick * lv1;
                le2 = c_kick * lv2;
            }
            int nd[8];
            corners(i, j, k, nx, ny, nz, nd);
            float sc[8];
            float ex = 0.0f, ey = 0.0f, ez = 0.0f;   // E at y (PG)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                float4 e0, e1;
                ld_pair(E8 + 2 * nd[2 * r], e0, e1);
                sc[2 * r] = le0 * e0.x + le1 * e0.y + le2 * e0.z;
                sc[2 * r + 1] = le0 * e1.x + le1 * e1.y + le2 * e1.z;
                if (PG) {
                    // corners 2r, 2r + 1 share the (y, z) factor of their weights
                    const float wyz = ((r & 1) ? fy : 1.0f - fy) * ((r & 2) ? fz : 1.0f - fz);
                    const float w0 = (1.0f - fx) * wyz, w1 = fx * wyz;
                    ex += w0 * e0.x + w1 * e1.x;
                    ey += w0 * e0.y + w1 * e1.y;
                    ez += w0 * e0.z + w1 * e1.z;
                }
            }
            if (PG) {
                // the quadrupole direction Q(y) = (-(x-c)/2, -(y-c)/2, (z-c)) as in
                // the forward kick, vm = v + (c_kick / 2) (e + wz2 Q); sums of
                // lv_tot_i vm_j and le . Q
                float ux = (float)i - pg.half_n[0] + 0.5f + fx;
                float uy = (float)j - pg.half_n[1] + 0.5f + fy;
                float uz = (float)k - pg.half_n[2] + 0.5f + fz;
                if (ux >= pg.half_n[0]) ux -= (float)nx;
                if (uy >= pg.half_n[1]) uy -= (float)ny;
                if (uz >= pg.half_n[2]) uz -= (float)nz;
                const float Q0 = -0.5f * ux * pg.h[0], Q1 = -0.5f * uy * pg.h[1], Q2 = uz * pg.h[2];
                const float hc = 0.5f * c_kick;
                const float vm0 = pg.yv[0][p] + hc * (ex + wz2 * Q0);
                const float vm1 = pg.yv[1][p] + hc * (ey + wz2 * Q1);
                const float vm2 = pg.yv[2][p] + hc * (ez + wz2 * Q2);
                pa[0] += lt0 * vm0; pa[1] += lt0 * vm1; pa[2] += lt0 * vm2;
                pa[3] += lt1 * vm0; pa[4] += lt1 * vm1; pa[5] += lt1 * vm2;
                pa[6] += lt2 * vm0; pa[7] += lt2 * vm1; pa[8] += lt2 * vm2;
                pa[9] += le0 * Q0 + le1 * Q1 + le2 * Q2;
            }
            float dx, dy, dz;
            interp_grad(fx, fy, fz, sc, dx, dy, dz);
            ly0 += g.inv_h[0] * dx - 0.5f * wz2 * le0;
            ly1 += g.inv_h[1] * dy - 0.5f * wz2 * le1;
            ly2 += g.inv_h[2] * dz + wz2 * le2;
            lam.o[0][p] = ly0;
            lam.o[1][p] = ly1;
            lam.o[2][p] = ly2;
            lam.v[0][p] = lv0;
            lam.v[1][p] = lv1;
            lam.v[2][p] = lv2;
            mly = fmaxf(mly, fmaxf(fabsf(ly0), fmaxf(fabsf(ly1), fabsf(ly2))));
            mlv = fmaxf(mlv, fmaxf(fabsf(lv0), fmaxf(fabsf(lv1), fabsf(lv2))));
            // G^T le
            const float gx = 1.0f - fx, gy = 1.0f - fy, gz = 1.0f - fz;
            const float w[8] = {gx * gy * gz, fx * gy * gz, gx * fy * gz, fx * fy * gz,
                                gx * gy * fz, fx * gy * fz, gx * fy * fz, fx * fy * fz};
            const int si = tile_slot(i, ox, nx, g.tile[0], G);
            const int sj = tile_slot(j, oy, ny, g.tile[1], G);
            const int sk = tile_slot(k, oz, nz, g.tile[2], G);
            if (si >= 0 && sj >= 0 && sk >= 0) {
                const int s = si + S0 * sj + S01 * sk;
                const int off[8] = {0, 1, S0, S0 + 1, S01, S01 + 1, S01 + S0, S01 + S0 + 1};
                const float q0 = qs * le0, q1 = qs * le1, q2 = qs * le2;
#pragma unroll
                for (int cc = 0; cc < 8; ++cc) {
                    atomicAdd(acc + s + off[cc], __float2int_rn(w[cc] * q0));
                    atomicAdd(acc + S + s + off[cc], __float2int_rn(w[cc] * q1));
                    atomicAdd(acc + 2 * S + s + off[cc], __float2int_rn(w[cc] * q2));
                }
            } else {
#pragma unroll
                for (int cc = 0; cc < 8; ++cc)
                    atomicAdd(lE4 + nd[cc], make_float4(w[cc] * le0, w[cc] * le1, w[cc] * le2, 0.0f));
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < S; q += blockDim.x) {
            const int ix = acc[q], iy = acc[S + q], iz = acc[2 * S + q];
            if (ix != 0 || iy != 0 || iz != 0) {
                const float ax = (float)ix * inv_qs, ay = (float)iy * inv_qs, az = (float)iz * inv_qs;
                int a, b, cz;
                cic::tile_pos(tb, q, a, b, cz);
                const int gi = cic::wrap_index(ox - G + a, nx);
                const int gj = cic::wrap_index(oy - G + b, ny);
                const int gk = cic::wrap_index(oz - G + cz, nz);
                atomicAdd(lE4 + gi + (int64_t)nx * (gj + (int64_t)ny * gk),
                          make_float4(ax, ay, az, 0.0f));
            }
        }
        __syncthreads();
    }
    max_to(&ctrl_w->adj_ly[ab.par], mly);
    max_to(&ctrl_w->adj_lv[ab.par], mlv);
    if (bad) atomicOr(&ctrl_w->flags, PIC_FLAG_BAD_CELL);
    if (nonfinite) atomicOr(&ctrl_w->flags, PIC_FLAG_NONFINITE);
    if (PG) {
        // block sums in FP64, fixed order: warp shuffles, then the 8 warps
        __shared__ double red[kPGradTerms][8];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int q = 0; q < kPGradTerms; ++q) {
            double t = (double)pa[q];
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0) red[q][wid] = t;
        }
        __syncthreads();
        if (threadIdx.x < kPGradTerms) {
            double t = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[threadIdx.x][q];
            pg.part[(size_t)kPGradTerms * blockIdx.x + threadIdx.x] = t;
        }
    }
}

// acc[q] += sum over blocks of part[b][q]: strided per-thread sums, then a
// fixed tree (one block of 256 threads)
__global__ void k_pgrad_acc(const double *__restrict__ part, int blocks, double *acc) {
    __shared__ double red[kPGradTerms][256];
    double s[kPGradTerms];
    for (int q = 0; q < kPGradTerms; ++q) s[q] = 0.0;
    for (int b = threadIdx.x; b < blocks; b += blockDim.x)
        for (int q = 0; q < kPGradTerms; ++q) s[q] += part[(size_t)kPGradTerms * b + q];
    for (int q = 0; q < kPGradTerms; ++q) red[q][threadIdx.x] = s[q];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int q = 0; q < kPGradTerms; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if ((int)threadIdx.x < kPGradTerms) acc[threadIdx.x] += red[threadIdx.x][0];
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
// (with `out` given, the updated multipliers go there instead of in place:
// ly + term to out.o, lv copied to out.v)
__global__ void k_adj_rho(int64_t n, Geom g, Ctrl *ctrl, const int32_t *__restrict__ ycell,
                          const float *__restrict__ yo0, const float *__restrict__ yo1,
                          const float *__restrict__ yo2, const float2 *__restrict__ lrho2,
                          float qscale, LamOut out, int par) {
    const ParticleSet lam = ctrl->sets[1 - ctrl->cur];
    float mly = 0.0f;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const float sx = qscale * g.inv_h[0], sy = qscale * g.inv_h[1], sz = qscale * g.inv_h[2];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        int i, j, k;
        decode(ycell[p], g, i, j, k);
        float sc[8];
        corners_from_pairs(lrho2, i, j, k, nx, ny, nz, sc);
        float dx, dy, dz;
        interp_grad(yo0[p], yo1[p], yo2[p], sc, dx, dy, dz);
        const float ly0 = lam.o[0][p] + sx * dx, ly1 = lam.o[1][p] + sy * dy;
        const float ly2 = lam.o[2][p] + sz * dz;
        if (out.o[0]) {
            out.o[0][p] = ly0;
            out.o[1][p] = ly1;
            out.o[2][p] = ly2;
            out.v[0][p] = lam.v[0][p];
            out.v[1][p] = lam.v[1][p];
            out.v[2][p] = lam.v[2][p];
        } else {
            lam.o[0][p] = ly0;
            lam.o[1][p] = ly1;
            lam.o[2][p] = ly2;
        }
        mly = fmaxf(mly, fmaxf(fabsf(ly0), fmaxf(fabsf(ly1), fabsf(ly2))));
    }
    max_to(&ctrl->adj_ly[par], mly);
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

// The forward sweep re-bins the particles every few steps, and the
// multipliers of a step are in that step's particle order.  Moving them back
// across a re-binning is a permutation: with pos[pid] the slot of particle
// pid in the later order, slot i of the earlier order (particle
// pid_prev[i]) takes the multipliers from slot pos[pid_prev[i]].
__global__ void k_adj_reorder(int64_t n, const int32_t *__restrict__ pos,
                              const int32_t *__restrict__ pid_prev, ReorderArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t j = pos[pid_prev[i]];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        a.out_o[d][i] = a.in_o[d][j];
        a.out_v[d][i] = a.in_v[d][j];
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
                            const int32_t *ycell, const float *const yo[3], const float4 *E8,
                            float4 *lE4, float c_kick, float dt, float wz2, const AdjRhoTerm &rt,
                            const AdjBound &ab, const PGrad &pg, Ctrl *ctrl_w, cudaStream_t st) {
    const int S = (g.tile[0] + 2 * g.guard + 1) * (g.tile[1] + 2 * g.guard + 1) *
                  (g.tile[2] + 2 * g.guard + 1);
    const size_t smem = sizeof(int) * 3 * (size_t)S;
    const int blocks = std::max(1, std::min(kAdjPushMaxBlocks, max_items));
#define PIC_ADJ(PGV)                                                                            \
    do {                                                                                        \
        if (smem > 48 * 1024) {                                                                 \
            cudaError_t e = cudaFuncSetAttribute(k_adj_push<PGV>,                               \
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                                 (int)smem);                                    \
            if (e != cudaSuccess) return e;                                                     \
        }                                                                                       \
        k_adj_push<PGV><<<blocks, 256, smem, st>>>(g, ctrl, items, ycell, yo[0], yo[1], yo[2],  \
                                                   E8, lE4, c_kick, dt, wz2, rt, ab, pg,        \
                                                   ctrl_w);                                     \
    } while (0)
    if (pg.part) PIC_ADJ(true);
    else PIC_ADJ(false);
#undef PIC_ADJ
    return cudaGetLastError();
}

cudaError_t launch_pgrad_acc(const double *part, int max_items, double *acc, cudaStream_t st) {
    const int blocks = std::max(1, std::min(kAdjPushMaxBlocks, max_items));
    k_pgrad_acc<<<1, 256, 0, st>>>(part, blocks, acc);
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

// lrho2[q] = (lrho[q], lrho[q + x]) (periodic): the x-paired copy read by
// the deposit-term gathers; also clears lE for the next reverse push (its
// transform has been taken by now)
//
// Bound bookkeeping for step m (par = m & 1): the maximum |lrho| goes to
// adj_lrho[par]; adj_ly / adj_lv[par ^ 1], last read by the reverse push of
// step m, are cleared for the push of step m - 1 to fill.
__global__ void k_adj_pair_rho(int nx, int64_t ng, const float *__restrict__ lrho,
                               float2 *__restrict__ lrho2, float4 *__restrict__ lE4, Ctrl *ctrl,
                               int par) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q == 0) {
        ctrl->adj_ly[par ^ 1] = 0u;
        ctrl->adj_lv[par ^ 1] = 0u;
    }
    float m = 0.0f;
    if (q < ng) {
        const int64_t row = q / nx;
        const int i = (int)(q - row * nx);
        const float a = lrho[q];
        lrho2[q] = make_float2(a, lrho[(i + 1 == nx) ? row * nx : q + 1]);
        lE4[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        m = fabsf(a);
    }
    max_to(&ctrl->adj_lrho[par], m);
}

cudaError_t launch_adj_pair_rho(const Geom &g, const float *lrho, float2 *lrho2, float4 *lE4,
                                Ctrl *ctrl, int par, cudaStream_t st) {
    const int64_t ng = (int64_t)g.n[0] * g.n[1] * g.n[2];
    k_adj_pair_rho<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(g.n[0], ng, lrho, lrho2, lE4,
                                                                 ctrl, par);
    return cudaGetLastError();
}

cudaError_t launch_adj_rho(int64_t n, const Geom &g, Ctrl *ctrl, const int32_t *ycell,
                           const float *const yo[3], const float2 *lrho2, float qscale,
                           const LamOut &out, int par, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int b = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
    k_adj_rho<<<b, 256, 0, st>>>(n, g, ctrl, ycell, yo[0], yo[1], yo[2], lrho2, qscale, out, par);
    return cudaGetLastError();
}

cudaError_t launch_adj_zero(int64_t n, const Ctrl *ctrl, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int b = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
    k_adj_zero<<<b, 256, 0, st>>>(n, ctrl);
    return cudaGetLastError();
}

cudaError_t launch_adj_reorder(int64_t n, const int32_t *pos, const int32_t *pid_prev,
                               const float *const in_o[3], const float *const in_v[3],
                               float *const out_o[3], float *const out_v[3], cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    ReorderArgs a;
    for (int d = 0; d < 3; ++d) {
        a.in_o[d] = in_o[d];
        a.in_v[d] = in_v[d];
        a.out_o[d] = out_o[d];
        a.out_v[d] = out_v[d];
    }
    k_adj_reorder<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, pos, pid_prev, a);
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
