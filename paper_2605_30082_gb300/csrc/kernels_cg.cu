// Flexible conjugate gradients preconditioned by one V-cycle (the same iteration as the
// oracle's or_mg_fcg): with z_k = V(r_k),
//     alpha_k = (r_k . z_k) / (d_k . A d_k),  x += alpha_k d_k,  r -= alpha_k A d_k,
//     beta_k+1 = -alpha_k (z_k+1 . A d_k) / (r_k . z_k),  d_k+1 = z_k+1 + beta_k+1 d_k.
// The scalars stay in device memory (slots of `sc`, see mg_internal.cuh): every kernel that
// needs a step length reads the dot products the previous reduction left there, so the
// inner loop never waits on the host.
//
// FP32 kernels work on colour-split finest levels (hx % 4 == 0), the vector kernels on
// 4-float vectors; FP64 kernels on natural-layout arrays.  Reductions use a fixed grid and
// a one-block final sum, so results do not depend on scheduling.
#include "mg_internal.cuh"

namespace mg {

namespace {

constexpr int kThreads = 256;

// block sum of a (and b) in double, fixed order, written to partials[2 * blockIdx.x (+1)]
__device__ __forceinline__ void block_sum_pair(double a, double b, double *partials) {
    __shared__ double sa[32], sb[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sa[warp] = a;
        sb[warp] = b;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        a = lane < nw ? sa[lane] : 0.0;
        b = lane < nw ? sb[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (lane == 0) {
            partials[2 * blockIdx.x] = a;
            partials[2 * blockIdx.x + 1] = b;
        }
    }
}

// sc[slot_a] = sum of partials[2 q], sc[slot_b] = sum of partials[2 q + 1] (slot_b < 0: unused)
__global__ void k_cg_final(const double *__restrict__ partials, int nb, double *sc, int slot_a, int slot_b) {
    __shared__ double sa[256], sb[256];
    double a = 0.0, b = 0.0;
    for (int q = threadIdx.x; q < nb; q += blockDim.x) {
        a += partials[2 * q];
        b += partials[2 * q + 1];
    }
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sa[threadIdx.x] += sa[threadIdx.x + w];
            sb[threadIdx.x] += sb[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sc[slot_a] = sa[0];
        if (slot_b >= 0) sc[slot_b] = sb[0];
    }
}

struct Coef32c {
    const float *s;             // s = 1/rho per cell (s-form) when non-null
    const float *fx, *fy, *fz;  // low-face coefficients otherwise
};

// q = A d on a colour-split level (both colours), partial sums of d . q.
// (A d)_c = ih2 sum_f beta_f (d_c - d_nb), beta_f = (s_c + s_nb) / 2 in the s-form.
// Thread t handles the 4 cells k0..k0+3 of one colour row; the six neighbours of a cell
// of colour c at (k, y, z), x = 2k + p, are the other colour's k + p - 1, k + p in the
// same row and k in the rows y +- 1, z +- 1.
template <bool SFORM>
__global__ void k_cg_apply32(Lay L, float ih2, Coef32c cf, const float *__restrict__ d, float *q, double *partials) {
    const int hx = L.hx, kv = hx >> 2;
    const i64 rows = (i64)L.ny * L.nz;
    const i64 per_col = rows * kv;
    const i64 dy = hx, dz = (i64)L.ny * hx;
    double acc = 0.0;
    for (i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x; t < 2 * per_col; t += (i64)gridDim.x * blockDim.x) {
        const int col = t >= per_col;
        // t < n / 4 < 2^31: 32-bit divisions (64-bit ones cost several times as many instructions)
        const unsigned tt = (unsigned)(t - col * per_col), rowu = tt / (unsigned)kv;
        const i64 row = rowu;
        const int k0 = (int)(tt - rowu * (unsigned)kv) << 2;
        const int y = (int)(rowu % (unsigned)L.ny), z = (int)(rowu / (unsigned)L.ny);
        const int p = (col + y + z) & 1;
        const i64 own = col * L.half + row * hx + k0;
        const i64 opp = (1 - col) * L.half + row * hx + k0;
        const bool hy0 = y > 0, hy1 = y < L.ny - 1, hz0 = z > 0, hz1 = z < L.nz - 1;
        const bool xw0 = (p == 0 && k0 == 0), xw1 = (p == 1 && k0 + 4 == hx);
        auto ld4 = [&](const float *A, i64 off, bool ok, float (&v)[4]) {
            if (ok) {
                const float4 c4 = *reinterpret_cast<const float4 *>(A + off);
                v[0] = c4.x; v[1] = c4.y; v[2] = c4.z; v[3] = c4.w;
            } else {
                v[0] = v[1] = v[2] = v[3] = 0.f;
            }
        };
        // same-row window of the other colour: m[v] = O[k0+v+p-1], n[v] = O[k0+v+p]
        auto window = [&](const float *O, float (&m)[4], float (&nn)[4]) {
            const float4 c4 = *reinterpret_cast<const float4 *>(O + opp);
            if (p) {
                const float e = (k0 + 4 < hx) ? O[opp + 4] : 0.f;
                m[0] = c4.x; m[1] = c4.y; m[2] = c4.z; m[3] = c4.w;
                nn[0] = c4.y; nn[1] = c4.z; nn[2] = c4.w; nn[3] = e;
            } else {
                const float e = (k0 > 0) ? O[opp - 1] : 0.f;
                m[0] = e; m[1] = c4.x; m[2] = c4.y; m[3] = c4.z;
                nn[0] = c4.x; nn[1] = c4.y; nn[2] = c4.z; nn[3] = c4.w;
            }
        };
        float dc[4], dm[4], dp[4], d2[4], d3[4], d4[4], d5[4];
        ld4(d, own, true, dc);
        window(d, dm, dp);
        ld4(d, opp - dy, hy0, d2);
        ld4(d, opp + dy, hy1, d3);
        ld4(d, opp - dz, hz0, d4);
        ld4(d, opp + dz, hz1, d5);
        float w0[4], w1[4], w2[4], w3[4], w4[4], w5[4];
        if (SFORM) {
            float sc[4], sm[4], sp[4], s2[4], s3[4], s4[4], s5[4];
            ld4(cf.s, own, true, sc);
            window(cf.s, sm, sp);
            ld4(cf.s, opp - dy, hy0, s2);
            ld4(cf.s, opp + dy, hy1, s3);
            ld4(cf.s, opp - dz, hz0, s4);
            ld4(cf.s, opp + dz, hz1, s5);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                w0[v] = (v == 0 && xw0) ? 0.f : 0.5f * (sc[v] + sm[v]);
                w1[v] = (v == 3 && xw1) ? 0.f : 0.5f * (sc[v] + sp[v]);
                w2[v] = hy0 ? 0.5f * (sc[v] + s2[v]) : 0.f;
                w3[v] = hy1 ? 0.5f * (sc[v] + s3[v]) : 0.f;
                w4[v] = hz0 ? 0.5f * (sc[v] + s4[v]) : 0.f;
                w5[v] = hz1 ? 0.5f * (sc[v] + s5[v]) : 0.f;
            }
        } else {
            float dummy[4];
            ld4(cf.fx, own, true, w0);      // low x face (0 at the wall)
            window(cf.fx, dummy, w1);       // high x face = the x+1 neighbour's low face
            if (xw1) w1[3] = 0.f;
            ld4(cf.fy, own, true, w2);
            ld4(cf.fy, opp + dy, hy1, w3);
            ld4(cf.fz, own, true, w4);
            ld4(cf.fz, opp + dz, hz1, w5);
            (void)dummy;
        }
        float qv[4];
        float part = 0.f;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            float a = w0[v] * (dc[v] - dm[v]);
            a += w1[v] * (dc[v] - dp[v]);
            a += w2[v] * (dc[v] - d2[v]);
            a += w3[v] * (dc[v] - d3[v]);
            a += w4[v] * (dc[v] - d4[v]);
            a += w5[v] * (dc[v] - d5[v]);
            qv[v] = a * ih2;
            part = fmaf(dc[v], qv[v], part);
        }
        *reinterpret_cast<float4 *>(q + own) = make_float4(qv[0], qv[1], qv[2], qv[3]);
        acc += (double)part;
    }
    block_sum_pair(acc, 0.0, partials);
}

// partial sums of (r . z, z . q), 4 floats per thread step
__global__ void k_cg_dots32(i64 n4, const float4 *__restrict__ r, const float4 *__restrict__ z,
                            const float4 *__restrict__ q, double *partials) {
    double a = 0.0, b = 0.0;
    for (i64 m = (i64)blockIdx.x * blockDim.x + threadIdx.x; m < n4; m += (i64)gridDim.x * blockDim.x) {
        const float4 rv = r[m], zv = z[m], qv = q[m];
        a += (double)(rv.x * zv.x + rv.y * zv.y + rv.z * zv.z + rv.w * zv.w);
        b += (double)(zv.x * qv.x + zv.y * qv.y + zv.z * qv.z + zv.w * qv.w);
    }
    block_sum_pair(a, b, partials);
}

// d = z + beta d with beta = -alpha (z . q_prev) / (r_prev . z_prev); first: d = z
__global__ void k_cg_dir32(i64 n4, const float4 *__restrict__ z, float4 *dv, const double *__restrict__ sc,
                           int first, int rz_prev) {
    const i64 m = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n4) return;
    const float4 zv = z[m];
    if (first) {
        dv[m] = zv;
        return;
    }
    const float beta = (float)(-sc[CG_ALPHA] * sc[CG_ZQ] / sc[rz_prev]);
    float4 v = dv[m];
    v.x = fmaf(beta, v.x, zv.x);
    v.y = fmaf(beta, v.y, zv.y);
    v.z = fmaf(beta, v.z, zv.z);
    v.w = fmaf(beta, v.w, zv.w);
    dv[m] = v;
}

// alpha = (r . z) / (d . A d); x += alpha d, r -= alpha A d; the first thread records alpha
__global__ void k_cg_update32(i64 n4, float4 *x, float4 *r, const float4 *__restrict__ dv,
                              const float4 *__restrict__ q, double *sc, int rz_cur) {
    const i64 m = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    const double alpha_d = sc[rz_cur] / sc[CG_PQ];
    if (m == 0) sc[CG_ALPHA] = alpha_d;
    if (m >= n4) return;
    const float alpha = (float)alpha_d;
    const float4 dd = dv[m], qq = q[m];
    float4 xv = x[m], rv = r[m];
    xv.x = fmaf(alpha, dd.x, xv.x);
    xv.y = fmaf(alpha, dd.y, xv.y);
    xv.z = fmaf(alpha, dd.z, xv.z);
    xv.w = fmaf(alpha, dd.w, xv.w);
    rv.x = fmaf(-alpha, qq.x, rv.x);
    rv.y = fmaf(-alpha, qq.y, rv.y);
    rv.z = fmaf(-alpha, qq.z, rv.z);
    rv.w = fmaf(-alpha, qq.w, rv.w);
    x[m] = xv;
    r[m] = rv;
}

// ---- FP64, natural layout ---------------------------------------------------------------
// q = A d in diagonal form, (A d)_c = ih2 (dg_c d_c - sum_f beta_f d_nb), partials of d . q
__global__ void k_cg_apply64(Dims dm, double ih2, const double *__restrict__ fx, const double *__restrict__ fy,
                             const double *__restrict__ fz, const double *__restrict__ dg,
                             const double *__restrict__ d, double *q, double *partials) {
    double acc = 0.0;
    const int nx = dm.nx, ny = dm.ny, nz = dm.nz;
    const i64 nxy = dm.nxy, rows = (i64)ny * nz;
    for (i64 row = blockIdx.x; row < rows; row += gridDim.x) {
        const int j = (int)(row % ny), k = (int)(row / ny);
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const i64 c = row * nx + i;
            double a = dg[c] * d[c];
            if (i > 0) a = fma(-fx[c], d[c - 1], a);
            if (i < nx - 1) a = fma(-fx[c + 1], d[c + 1], a);
            if (j > 0) a = fma(-fy[c], d[c - nx], a);
            if (j < ny - 1) a = fma(-fy[c + nx], d[c + nx], a);
            if (k > 0) a = fma(-fz[c], d[c - nxy], a);
            if (k < nz - 1) a = fma(-fz[c + nxy], d[c + nxy], a);
            a *= ih2;
            q[c] = a;
            acc = fma(d[c], a, acc);
        }
    }
    block_sum_pair(acc, 0.0, partials);
}

__global__ void k_cg_dots64(i64 n, const double *__restrict__ r, const double *__restrict__ z,
                            const double *__restrict__ q, double *partials) {
    double a = 0.0, b = 0.0;
    for (i64 m = (i64)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (i64)gridDim.x * blockDim.x) {
        const double zv = z[m];
        a = fma(r[m], zv, a);
        b = fma(zv, q[m], b);
    }
    block_sum_pair(a, b, partials);
}

__global__ void k_cg_dir64(i64 n, const double *__restrict__ z, double *dv, const double *__restrict__ sc,
                           int first, int rz_prev) {
    const i64 m = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    if (first) {
        dv[m] = z[m];
        return;
    }
    const double beta = -sc[CG_ALPHA] * sc[CG_ZQ] / sc[rz_prev];
    dv[m] = fma(beta, dv[m], z[m]);
}

// alpha = (r . z) / (d . A d); x += alpha d, r -= alpha A d; partials of |r|^2 (and of sum x)
__global__ void k_cg_update64(i64 n, double *x, double *r, const double *__restrict__ dv,
                              const double *__restrict__ q, double *sc, int rz_cur, double *partials) {
    const double alpha = sc[rz_cur] / sc[CG_PQ];
    if (blockIdx.x == 0 && threadIdx.x == 0) sc[CG_ALPHA] = alpha;
    double rr = 0.0, sx = 0.0;
    for (i64 m = (i64)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (i64)gridDim.x * blockDim.x) {
        const double xv = fma(alpha, dv[m], x[m]);
        const double rv = fma(-alpha, q[m], r[m]);
        x[m] = xv;
        r[m] = rv;
        rr = fma(rv, rv, rr);
        sx += xv;
    }
    block_sum_pair(rr, sx, partials);
}

inline unsigned blocks_for(i64 n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

void launch_cg_apply32(cudaStream_t s, Lay L, double ih2, const float *sinv, const float *fx, const float *fy,
                       const float *fz, const float *d, float *q, double *partials, double *sc) {
    const Coef32c cf{sinv, fx, fy, fz};
    static const int wave_s = wave_blocks((const void *)k_cg_apply32<true>, kThreads);
    static const int wave_n = wave_blocks((const void *)k_cg_apply32<false>, kThreads);
    const int nb = fill_blocks(reduce_blocks(L.n / 4), sinv ? wave_s : wave_n);
    count_launch(2);
    if (sinv) k_cg_apply32<true><<<nb, kThreads, 0, s>>>(L, (float)ih2, cf, d, q, partials);
    else k_cg_apply32<false><<<nb, kThreads, 0, s>>>(L, (float)ih2, cf, d, q, partials);
    k_cg_final<<<1, 256, 0, s>>>(partials, nb, sc, CG_PQ, -1);
}

void launch_cg_dots32(cudaStream_t s, i64 n, const float *r, const float *z, const float *q, double *partials,
                      double *sc, int rz_slot) {
    static const int wave = wave_blocks((const void *)k_cg_dots32, kThreads);
    const int nb = fill_blocks(reduce_blocks(n / 4), wave);
    count_launch(2);
    k_cg_dots32<<<nb, kThreads, 0, s>>>(n / 4, reinterpret_cast<const float4 *>(r),
                                        reinterpret_cast<const float4 *>(z), reinterpret_cast<const float4 *>(q),
                                        partials);
    k_cg_final<<<1, 256, 0, s>>>(partials, nb, sc, rz_slot, CG_ZQ);
}

void launch_cg_dir32(cudaStream_t s, i64 n, const float *z, float *d, const double *sc, bool first, int rz_prev) {
    count_launch();
    k_cg_dir32<<<blocks_for(n / 4), kThreads, 0, s>>>(n / 4, reinterpret_cast<const float4 *>(z),
                                                      reinterpret_cast<float4 *>(d), sc, first ? 1 : 0, rz_prev);
}

void launch_cg_update32(cudaStream_t s, i64 n, float *x, float *r, const float *d, const float *q, double *sc,
                        int rz_cur) {
    count_launch();
    k_cg_update32<<<blocks_for(n / 4), kThreads, 0, s>>>(n / 4, reinterpret_cast<float4 *>(x),
                                                         reinterpret_cast<float4 *>(r),
                                                         reinterpret_cast<const float4 *>(d),
                                                         reinterpret_cast<const float4 *>(q), sc, rz_cur);
}

void launch_cg_apply64(cudaStream_t s, Dims d, double ih2, const double *fx, const double *fy, const double *fz,
                       const double *dg, const double *dv, double *q, double *partials, double *sc) {
    const i64 rows = (i64)d.ny * d.nz;
    static const int wave = wave_blocks((const void *)k_cg_apply64, kThreads);
    int nb = fill_blocks(reduce_blocks(d.n), wave);
    if (nb > rows) nb = (int)rows;
    count_launch(2);
    k_cg_apply64<<<nb, kThreads, 0, s>>>(d, ih2, fx, fy, fz, dg, dv, q, partials);
    k_cg_final<<<1, 256, 0, s>>>(partials, nb, sc, CG_PQ, -1);
}

void launch_cg_dots64(cudaStream_t s, i64 n, const double *r, const double *z, const double *q, double *partials,
                      double *sc, int rz_slot) {
    const int nb = reduce_blocks(n);
    count_launch(2);
    k_cg_dots64<<<nb, kThreads, 0, s>>>(n, r, z, q, partials);
    k_cg_final<<<1, 256, 0, s>>>(partials, nb, sc, rz_slot, CG_ZQ);
}

void launch_cg_dir64(cudaStream_t s, i64 n, const double *z, double *d, const double *sc, bool first, int rz_prev) {
    count_launch();
    k_cg_dir64<<<blocks_for(n), kThreads, 0, s>>>(n, z, d, sc, first ? 1 : 0, rz_prev);
}

void launch_cg_update64(cudaStream_t s, i64 n, double *x, double *r, const double *d, const double *q, double *sc,
                        int rz_cur, double *partials) {
    static const int wave = wave_blocks((const void *)k_cg_update64, kThreads);
    const int nb = fill_blocks(reduce_blocks(n), wave);
    count_launch(2);
    k_cg_update64<<<nb, kThreads, 0, s>>>(n, x, r, d, q, sc, rz_cur, partials);
    k_cg_final<<<1, 256, 0, s>>>(partials, nb, sc, CG_RR, CG_SX);
}

}  // namespace mg
