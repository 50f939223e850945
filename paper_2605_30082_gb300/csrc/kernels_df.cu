// Outer defect-correction kernels of the MG_MIXED_DF mode: the finest-level solution,
// the scaled right-hand side and the FP64 coefficients are carried as pairs of FP32
// numbers (hi, lo) with value hi + lo ("double-float"), about 48 significant bits.
// The residual and the update then run on the FP32 units only; GB300 executes FP64
// at a small fraction of its FP32 rate, while the double-float result is as accurate
// as the residual check at relative tolerance 1e-10 needs.
//
// Error-free transformations (Knuth's TwoSum; Dekker's product, written with an FMA):
//   two_sum(a, b) = (s, e) with s = fl(a + b) and s + e = a + b exactly,
//   two_prod(a, b) = (p, e) with p = fl(a * b) and p + e = a * b exactly.
// A double-float x*y + acc keeps the exact product of the high parts, the cross terms
// hi*lo in FP32, drops lo*lo (2^-48 relative), and renormalises after each addition.
#include "mg_internal.cuh"

namespace mg {

namespace {

constexpr int kThreads = 256;
inline unsigned blocks_for(i64 n) { return (unsigned)((n + kThreads - 1) / kThreads); }

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// acc += x * y for double-float acc, x, y
__device__ __forceinline__ void df_fma(float &ah, float &al, float xh, float xl, float yh, float yl) {
    const float p = xh * yh;
    float e = fmaf(xh, yh, -p);
    e = fmaf(xh, yl, fmaf(xl, yh, e));
    float s, t;
    two_sum(ah, p, s, t);
    t += al + e;
    ah = s + t;
    al = t - (ah - s);
}

__device__ __forceinline__ float df_value(float h, float l) { return h + l; }

__global__ void k_split(i64 n, const double *__restrict__ src, float2 *dst) {
    const i64 m = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    const double v = src[m];
    const float hi = d2f_rn(v);
    dst[m] = make_float2(hi, d2f_rn(v - f2d_exact(hi)));
}

__global__ void k_join(i64 n, const float2 *__restrict__ src, double *dst) {
    const i64 m = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    const float2 v = src[m];
    dst[m] = f2d_exact(v.x) + f2d_exact(v.y);
}

// h^2 r = h^2 b + sum_f beta_f p_nb - d p_c in double-float (b already scaled by h^2);
// one thread per cell pair x = 2k, 2k+1 (even nx); r32 = s32 * h^2 r in the split level-0
// layout; partials: (sum (h^2 r)^2, sum p), FP32 per thread.
__global__ void k_resid_df(Dims d, Lay L, const float2 *__restrict__ fx, const float2 *__restrict__ fy,
                           const float2 *__restrict__ fz, const float2 *__restrict__ dg,
                           const float2 *__restrict__ b, const float2 *__restrict__ p, float *r32, float s32,
                           double *partials) {
    float q = 0.f, sp = 0.f;
    const int nx = d.nx, ny = d.ny, nz = d.nz, hx = nx >> 1;
    const int nxy = nx * ny;
    const int npairs = (int)(d.n >> 1);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < npairs; t += gridDim.x * blockDim.x) {
        const int row = t / hx, k = t - row * hx;
        const int j = row % ny, z = row / ny;
        const int c = row * nx + 2 * k;
        const float4 pc = *reinterpret_cast<const float4 *>(p + c);   // (h0, l0, h1, l1)
        const float4 bb = *reinterpret_cast<const float4 *>(b + c);
        const float4 fxa = *reinterpret_cast<const float4 *>(fx + c);
        const float4 fya = *reinterpret_cast<const float4 *>(fy + c);
        const float4 fza = *reinterpret_cast<const float4 *>(fz + c);
        const float4 dd = *reinterpret_cast<const float4 *>(dg + c);
        float a0h = bb.x, a0l = bb.y, a1h = bb.z, a1l = bb.w;
        if (k > 0) {
            const float2 pm = p[c - 1];
            df_fma(a0h, a0l, fxa.x, fxa.y, pm.x, pm.y);
        }
        df_fma(a0h, a0l, fxa.z, fxa.w, pc.z, pc.w);  // the face between the pair
        df_fma(a1h, a1l, fxa.z, fxa.w, pc.x, pc.y);
        if (k < hx - 1) {
            const float2 f = fx[c + 2], pp = p[c + 2];
            df_fma(a1h, a1l, f.x, f.y, pp.x, pp.y);
        }
        if (j > 0) {
            const float4 pm = *reinterpret_cast<const float4 *>(p + c - nx);
            df_fma(a0h, a0l, fya.x, fya.y, pm.x, pm.y);
            df_fma(a1h, a1l, fya.z, fya.w, pm.z, pm.w);
        }
        if (j < ny - 1) {
            const float4 f = *reinterpret_cast<const float4 *>(fy + c + nx);
            const float4 pp = *reinterpret_cast<const float4 *>(p + c + nx);
            df_fma(a0h, a0l, f.x, f.y, pp.x, pp.y);
            df_fma(a1h, a1l, f.z, f.w, pp.z, pp.w);
        }
        if (z > 0) {
            const float4 pm = *reinterpret_cast<const float4 *>(p + c - nxy);
            df_fma(a0h, a0l, fza.x, fza.y, pm.x, pm.y);
            df_fma(a1h, a1l, fza.z, fza.w, pm.z, pm.w);
        }
        if (z < nz - 1) {
            const float4 f = *reinterpret_cast<const float4 *>(fz + c + nxy);
            const float4 pp = *reinterpret_cast<const float4 *>(p + c + nxy);
            df_fma(a0h, a0l, f.x, f.y, pp.x, pp.y);
            df_fma(a1h, a1l, f.z, f.w, pp.z, pp.w);
        }
        df_fma(a0h, a0l, -dd.x, -dd.y, pc.x, pc.y);
        df_fma(a1h, a1l, -dd.z, -dd.w, pc.z, pc.w);
        const float r0 = df_value(a0h, a0l), r1 = df_value(a1h, a1l);
        if (r32) {
            const int par = (j + z) & 1;
            const i64 base = (i64)row * hx + k;
            r32[par * L.half + base] = r0 * s32;
            r32[(1 - par) * L.half + base] = r1 * s32;
        }
        q = fmaf(r0, r0, q);
        q = fmaf(r1, r1, q);
        sp += pc.x + pc.z;
    }
    // block sum of (q, sp) -> partials[2 * blockIdx.x], fixed order
    __shared__ double sa[32], sb[32];
    double a = q, bsum = sp;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        bsum += __shfl_xor_sync(0xffffffffu, bsum, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sa[warp] = a;
        sb[warp] = bsum;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        a = lane < nw ? sa[lane] : 0.0;
        bsum = lane < nw ? sb[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            bsum += __shfl_xor_sync(0xffffffffu, bsum, o);
        }
        if (lane == 0) {
            partials[2 * blockIdx.x] = a;
            partials[2 * blockIdx.x + 1] = bsum;
        }
    }
}

__global__ void k_final_df(const double *__restrict__ partials, int nb, double *out) {
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
        out[0] = sa[0];
        out[1] = sb[0];
    }
}

// ---- s-form double-float residual (operator set from a density) ------------------------
// With s = 1/rho per cell and beta_f = (s_c + s_nb) / 2,
//   2 h^2 r_c = 2 h^2 b_c + sum_f (s_c + s_nb) (p_nb - p_c),
// which reads 24 B per cell (p, h^2 b, s as double-float pairs) instead of the face form's 48.
// Intermediate pairs stay unnormalised: the high parts of every sum are exact (TwoSum) and
// the low parts collect the errors in FP32, dropping terms of relative size 2^-48.
__device__ __forceinline__ void df_diff(float ah, float al, float bh, float bl, float &dh, float &dl) {
    float e;
    two_sum(ah, -bh, dh, e);
    dl = e + (al - bl);
}
__device__ __forceinline__ void df_sum(float ah, float al, float bh, float bl, float &sh, float &sl) {
    float e;
    two_sum(ah, bh, sh, e);
    sl = e + (al + bl);
}
// (sa + sb) * (pa - pb) for double-float sa, sb, pa, pb; unnormalised product
__device__ __forceinline__ void df_face(float sah, float sal, float sbh, float sbl, float pah, float pal,
                                        float pbh, float pbl, float &fh, float &fl) {
    float bh, bl, dh, dl;
    df_sum(sah, sal, sbh, sbl, bh, bl);
    df_diff(pah, pal, pbh, pbl, dh, dl);
    fh = bh * dh;
    fl = fmaf(bh, dh, -fh);
    fl = fmaf(bh, dl, fmaf(bl, dh, fl));
}
__device__ __forceinline__ void df_acc(float &ah, float &al, float fh, float fl) {
    float s, t;
    two_sum(ah, fh, s, t);
    ah = s;
    al += t + fl;
}

constexpr int kDfsZ = 16;        // planes per tile
constexpr int kDfsThreads = 128;

// One thread per cell pair x = 2k, 2k+1 of a row (even nx); a warp covers 32 pairs of one row
// and each thread marches kDfsZ planes in z, carrying the (z-1, z) face product from the
// previous plane.  Persistent blocks take tiles (row chunk, row, z-chunk) in a fixed order so
// the partial sums do not depend on scheduling.  Outputs as k_resid_df.
__global__ void __launch_bounds__(kDfsThreads, 6)
    k_resid_dfs(Dims d, Lay L, const float2 *__restrict__ s2, const float2 *__restrict__ b, const float2 *__restrict__ p,
                float *r32, float s32, double *partials, int tiles_x, int tiles_y, i64 ntiles) {
    const int nx = d.nx, ny = d.ny, nz = d.nz, hx = nx >> 1;
    const i64 nxy = d.nxy;
    const int vb = blockDim.x, lane = threadIdx.x & 31;
    const float4 f0 = make_float4(0.f, 0.f, 0.f, 0.f);
    auto ld = [](const float2 *A, i64 off) { return *reinterpret_cast<const float4 *>(A + off); };
    double qd = 0.0, spd = 0.0;
    for (i64 t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int tx = (int)(t % tiles_x);
        const i64 rest = t / tiles_x;
        const int yb = (int)(rest % tiles_y), zc = (int)(rest / tiles_y);
        const int kvi = tx * vb + threadIdx.x, yi = yb * blockDim.y + threadIdx.y;
        const bool active = kvi < hx && yi < ny;
        const int k = min(kvi, hx - 1), y = min(yi, ny - 1);
        const bool kl = k > 0, kr = k < hx - 1, hy0 = y > 0, hy1 = y < ny - 1;
        const int z0 = zc * kDfsZ, z1 = min(z0 + kDfsZ, nz);
        i64 c = ((i64)z0 * ny + y) * nx + 2 * k;
        float4 pc = ld(p, c), sc = ld(s2, c);
        // carried (z-1, z) face products of the two cells
        float4 cz = f0;
        if (z0 > 0) {
            const float4 pm = ld(p, c - nxy), sm = ld(s2, c - nxy);
            df_face(sm.x, sm.y, sc.x, sc.y, pc.x, pc.y, pm.x, pm.y, cz.x, cz.y);
            df_face(sm.z, sm.w, sc.z, sc.w, pc.z, pc.w, pm.z, pm.w, cz.z, cz.w);
        }
        float q = 0.f, sp = 0.f;
        for (int z = z0; z < z1; ++z) {
            const bool hz0 = z > 0, hz1 = z < nz - 1;
            float4 pp = f0, sq = f0;
            if (hz1) {
                pp = ld(p, c + nxy);
                sq = ld(s2, c + nxy);
            }
            const float4 bb = ld(b, c);
            float a0h = 2.f * bb.x, a0l = 2.f * bb.y, a1h = 2.f * bb.z, a1l = 2.f * bb.w;
            float fh, fl;
            // faces to z-1: minus the carried products
            if (hz0) {
                df_acc(a0h, a0l, -cz.x, -cz.y);
                df_acc(a1h, a1l, -cz.z, -cz.w);
            }
            // faces to z+1, carried to the next plane
            if (hz1) {
                df_face(sc.x, sc.y, sq.x, sq.y, pp.x, pp.y, pc.x, pc.y, cz.x, cz.y);
                df_face(sc.z, sc.w, sq.z, sq.w, pp.z, pp.w, pc.z, pc.w, cz.z, cz.w);
                df_acc(a0h, a0l, cz.x, cz.y);
                df_acc(a1h, a1l, cz.z, cz.w);
            }
            if (hy0) {
                const float4 pn = ld(p, c - nx), sn = ld(s2, c - nx);
                df_face(sc.x, sc.y, sn.x, sn.y, pn.x, pn.y, pc.x, pc.y, fh, fl);
                df_acc(a0h, a0l, fh, fl);
                df_face(sc.z, sc.w, sn.z, sn.w, pn.z, pn.w, pc.z, pc.w, fh, fl);
                df_acc(a1h, a1l, fh, fl);
            }
            if (hy1) {
                const float4 pn = ld(p, c + nx), sn = ld(s2, c + nx);
                df_face(sc.x, sc.y, sn.x, sn.y, pn.x, pn.y, pc.x, pc.y, fh, fl);
                df_acc(a0h, a0l, fh, fl);
                df_face(sc.z, sc.w, sn.z, sn.w, pn.z, pn.w, pc.z, pc.w, fh, fl);
                df_acc(a1h, a1l, fh, fl);
            }
            // x faces: inside the pair, then x-1 of cell 0 and x+1 of cell 1 (neighbour lanes)
            df_face(sc.x, sc.y, sc.z, sc.w, pc.z, pc.w, pc.x, pc.y, fh, fl);
            df_acc(a0h, a0l, fh, fl);
            df_acc(a1h, a1l, -fh, -fl);
            float plh = __shfl_up_sync(0xffffffffu, pc.z, 1), pll = __shfl_up_sync(0xffffffffu, pc.w, 1);
            float slh = __shfl_up_sync(0xffffffffu, sc.z, 1), sll = __shfl_up_sync(0xffffffffu, sc.w, 1);
            float prh = __shfl_down_sync(0xffffffffu, pc.x, 1), prl = __shfl_down_sync(0xffffffffu, pc.y, 1);
            float srh = __shfl_down_sync(0xffffffffu, sc.x, 1), srl = __shfl_down_sync(0xffffffffu, sc.y, 1);
            if (lane == 0) {
                const float2 pv = kl ? p[c - 1] : make_float2(0.f, 0.f), sv = kl ? s2[c - 1] : make_float2(0.f, 0.f);
                plh = pv.x; pll = pv.y; slh = sv.x; sll = sv.y;
            }
            if (lane == 31) {
                const float2 pv = kr ? p[c + 2] : make_float2(0.f, 0.f), sv = kr ? s2[c + 2] : make_float2(0.f, 0.f);
                prh = pv.x; prl = pv.y; srh = sv.x; srl = sv.y;
            }
            df_face(sc.x, sc.y, slh, sll, plh, pll, pc.x, pc.y, fh, fl);
            if (kl) df_acc(a0h, a0l, fh, fl);
            df_face(sc.z, sc.w, srh, srl, prh, prl, pc.z, pc.w, fh, fl);
            if (kr) df_acc(a1h, a1l, fh, fl);
            const float r0 = 0.5f * (a0h + a0l), r1 = 0.5f * (a1h + a1l);
            if (active) {
                if (r32) {
                    const int par = (y + z) & 1;
                    const i64 base = ((i64)z * ny + y) * hx + k;
                    r32[par * L.half + base] = r0 * s32;
                    r32[(1 - par) * L.half + base] = r1 * s32;
                }
                q = fmaf(r0, r0, q);
                q = fmaf(r1, r1, q);
                sp += pc.x + pc.z;
            }
            pc = pp;
            sc = sq;
            c += nxy;
        }
        qd += (double)q;
        spd += (double)sp;
    }
    // block sum -> partials[2 * blockIdx.x], fixed order
    __shared__ double sa[32], sb[32];
    double a = qd, bsum = spd;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        bsum += __shfl_xor_sync(0xffffffffu, bsum, o);
    }
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int warp = tid >> 5;
    if (lane == 0) {
        sa[warp] = a;
        sb[warp] = bsum;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x * blockDim.y) >> 5;
        a = lane < nw ? sa[lane] : 0.0;
        bsum = lane < nw ? sb[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            bsum += __shfl_xor_sync(0xffffffffu, bsum, o);
        }
        if (lane == 0) {
            partials[2 * blockIdx.x] = a;
            partials[2 * blockIdx.x + 1] = bsum;
        }
    }
}

__device__ __forceinline__ i64 sto(const Lay &L, int x, int y, int z) {
    const i64 row = (i64)z * L.ny + y;
    if (!L.split) return row * L.nx + x;
    return ((x + y + z) & 1) * L.half + row * L.hx + (x >> 1);
}

// p = p + (alpha e - shift) in double-float (e in the level-0 FP32 layout)
__global__ void k_update_df(Dims d, Lay L, float2 *p, const float *__restrict__ e, float alpha, float shift) {
    const i64 m = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= d.n) return;
    const int i = (int)(m % d.nx);
    const i64 row = m / d.nx;
    const float t = fmaf(alpha, e[sto(L, i, (int)(row % d.ny), (int)(row / d.ny))], -shift);
    float2 v = p[m];
    float s, err;
    two_sum(v.x, t, s, err);
    err += v.y;
    const float hi = s + err;
    p[m] = make_float2(hi, err - (hi - s));
}

}  // namespace

void launch_split(cudaStream_t s, i64 n, const double *src, float2 *dst) {
    count_launch();
    k_split<<<blocks_for(n), kThreads, 0, s>>>(n, src, dst);
}

void launch_join(cudaStream_t s, i64 n, const float2 *src, double *dst) {
    count_launch();
    k_join<<<blocks_for(n), kThreads, 0, s>>>(n, src, dst);
}

void launch_resid_df(cudaStream_t s, Dims d, Lay L, const float2 *fx, const float2 *fy, const float2 *fz,
                     const float2 *diag, const float2 *b, const float2 *p, float *r32, float s32,
                     double *partials, double *out) {
    static const int wave = wave_blocks((const void *)k_resid_df, kReduceThreads);
    const int nb = fill_blocks(reduce_blocks(d.n / 2), wave);
    count_launch();
    k_resid_df<<<nb, kReduceThreads, 0, s>>>(d, L, fx, fy, fz, diag, b, p, r32, s32, partials);
    count_launch();
    k_final_df<<<1, 256, 0, s>>>(partials, nb, out);
}

void launch_resid_dfs(cudaStream_t s, Dims d, Lay L, const float2 *s2, const float2 *b, const float2 *p,
                      float *r32, float s32, double *partials, double *out) {
    const int hx = d.nx / 2;
    const int vb = (hx % 64 == 0) ? 64 : 32;
    const dim3 blk(vb, kDfsThreads / vb);
    const int tiles_x = (hx + vb - 1) / vb, tiles_y = (d.ny + (int)blk.y - 1) / (int)blk.y;
    const i64 ntiles = (i64)tiles_x * tiles_y * ((d.nz + kDfsZ - 1) / kDfsZ);
    i64 nb = (i64)device_sms() * 6;
    if (nb > ntiles) nb = ntiles;
    if (nb > reduce_blocks(d.n)) nb = reduce_blocks(d.n);  // the partials buffer holds reduce_blocks(n) pairs
    count_launch();
    k_resid_dfs<<<(unsigned)nb, blk, 0, s>>>(d, L, s2, b, p, r32, s32, partials, tiles_x, tiles_y, ntiles);
    count_launch();
    k_final_df<<<1, 256, 0, s>>>(partials, (int)nb, out);
}

void launch_update_df(cudaStream_t s, Dims d, Lay L, float2 *p, const float *e32, double alpha, double shift) {
    count_launch();
    k_update_df<<<blocks_for(d.n), kThreads, 0, s>>>(d, L, p, e32, (float)alpha, (float)shift);
}

}  // namespace mg
