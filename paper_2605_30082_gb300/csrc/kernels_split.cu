// FP32 V-cycle kernels on colour-split levels.
//
// Storage: an FP32 level with even nx keeps every cell array colour-split: all
// red cells ((x+y+z) even) first, then all black cells, each colour row by row
// with the cell at x stored at k = x >> 1.  Levels with odd nx (possible only on
// the coarsest level) keep the natural layout.  `sto` maps (x, y, z) to the
// storage index in either case.
//
// For a cell of colour c at (k, y, z), x = 2k + p with p = (c + y + z) & 1, the six
// neighbours all have the other colour and sit in the other half at
//   x-1: k + p - 1,   x+1: k + p      (same row)
//   y-1, y+1, z-1, z+1: k             (the rows above, below, before, after)
// so a half sweep reads the other colour with unit-stride, vectorisable loads and
// no shared memory: 4 B of the other colour's x, 8 B of 1/rho (both colours) or
// 12 B of face coefficients, and 4 B of b per updated cell, plus the write.
//
// Coefficients: SFORM uses s = 1/rho per cell and beta_f = (s_c + s_nb)/2 (the
// finest level when the operator came from a density); otherwise the low-face
// arrays fx, fy, fz (beta of the face between a cell and its x-1, y-1, z-1
// neighbour) stored in the same split layout.
//
// Two exact properties of red-black Gauss-Seidel shorten the V-cycle:
//  - after the last pre-smoothing sweep (black last) every black row is solved,
//    so the black residuals are zero and the restriction sums red residuals only;
//  - the first post-smoothing sweep (black first) overwrites every black cell, so
//    the coarse correction only needs to be added to the red cells.
#include "mg_internal.cuh"

namespace mg {

namespace {

constexpr int kThreads = 256;
inline unsigned blocks_for(i64 n) { return (unsigned)((n + kThreads - 1) / kThreads); }

__device__ __forceinline__ i64 sto(const Lay &L, int x, int y, int z) {
    const i64 row = (i64)z * L.ny + y;
    if (!L.split) return row * L.nx + x;
    return ((x + y + z) & 1) * L.half + row * L.hx + (x >> 1);
}

struct Coef32 {
    const float *s;             // SFORM when non-null
    const float *fx, *fy, *fz;  // face form otherwise
};

// ---- generic (scalar, any layout) stencil pieces --------------------------------------
// sum_f beta_f x_nb and sum_f beta_f at cell (x, y, z), SFORM carries a factor 2
__device__ __forceinline__ void stencil_any(const Lay &L, const Coef32 &cf, const float *__restrict__ xv,
                                            int x, int y, int z, float &num, float &den) {
    const i64 c = sto(L, x, y, z);
    const bool hx0 = x > 0, hx1 = x < L.nx - 1, hy0 = y > 0, hy1 = y < L.ny - 1, hz0 = z > 0, hz1 = z < L.nz - 1;
    const i64 n0 = hx0 ? sto(L, x - 1, y, z) : c, n1 = hx1 ? sto(L, x + 1, y, z) : c;
    const i64 n2 = hy0 ? sto(L, x, y - 1, z) : c, n3 = hy1 ? sto(L, x, y + 1, z) : c;
    const i64 n4 = hz0 ? sto(L, x, y, z - 1) : c, n5 = hz1 ? sto(L, x, y, z + 1) : c;
    float w0, w1, w2, w3, w4, w5;
    if (cf.s) {
        const float sc = cf.s[c];
        w0 = hx0 ? sc + cf.s[n0] : 0.f;
        w1 = hx1 ? sc + cf.s[n1] : 0.f;
        w2 = hy0 ? sc + cf.s[n2] : 0.f;
        w3 = hy1 ? sc + cf.s[n3] : 0.f;
        w4 = hz0 ? sc + cf.s[n4] : 0.f;
        w5 = hz1 ? sc + cf.s[n5] : 0.f;
    } else {
        w0 = cf.fx[c];
        w1 = hx1 ? cf.fx[n1] : 0.f;
        w2 = cf.fy[c];
        w3 = hy1 ? cf.fy[n3] : 0.f;
        w4 = cf.fz[c];
        w5 = hz1 ? cf.fz[n5] : 0.f;
    }
    float nm = w0 * xv[n0];
    nm += w1 * xv[n1];
    nm += w2 * xv[n2];
    nm += w3 * xv[n3];
    nm += w4 * xv[n4];
    nm += w5 * xv[n5];
    num = nm;
    den = ((w0 + w1) + (w2 + w3)) + (w4 + w5);
}

// half sweep of colour `col`, one thread per cell of that colour, any layout
__global__ void k_half_any(Lay L, float h2, Coef32 cf, const float *__restrict__ b, float *xv, int col,
                           int from_zero) {
    const int halfw = (L.nx + 1) >> 1;
    const i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    const i64 rows = (i64)L.ny * L.nz;
    if (t >= rows * halfw) return;
    const i64 row = t / halfw;
    const int m = (int)(t - row * halfw);
    const int y = (int)(row % L.ny), z = (int)(row / L.ny);
    const int x = 2 * m + ((col + y + z) & 1);
    if (x >= L.nx) return;
    float num, den;
    stencil_any(L, cf, xv, x, y, z, num, den);
    if (from_zero) num = 0.f;
    const float hh = cf.s ? 2.f * h2 : h2;
    xv[sto(L, x, y, z)] = __fdividef(hh * b[sto(L, x, y, z)] + num, den);
}

struct Upd {
    double *p;      // natural FP64 solution of the finest level (UPDATE 1)
    float2 *p2;     // natural double-float solution of the finest level (UPDATE 2)
    float alpha;    // scale of the correction, rounded to FP32 on the host
    float shift;    // gauge shift, rounded to FP32 on the host (no FP64 conversion on the device)
};

__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// double-float (h, l) + t, renormalised (Knuth's TwoSum on the high parts)
__device__ __forceinline__ void df_add(float &h, float &l, float t) {
    float s, e;
    two_sum_f(h, t, s, e);
    e += l;
    h = s + e;
    l = e - (h - s);
}

// ---- vectorised half sweep on split levels (hx % 4 == 0) ---------------------------------
// one thread updates 4 consecutive cells (k0..k0+3) of colour col in one row.
// UPDATE (last red half sweep of the finest level): instead of storing the 4 new red values,
// add alpha * x - shift for them and for the 4 black values of the same row positions --
// together the 8 consecutive cells x = 2 k0 .. 2 k0 + 7 -- to the solution: the FP64 one
// (UPDATE 1) or the double-float one (UPDATE 2).
// GHOST: a slab of a decomposed level (L.zlo / L.zhi), its ghost planes as z neighbours
template <bool SFORM, bool FROM_ZERO, int UPDATE = 0, bool GHOST = false>
__global__ void k_half_vec(Lay L, float h2, Coef32 cf, const float *__restrict__ b, float *xv, int col,
                           Upd up = Upd{}) {
    const int hx = L.hx, kv = hx >> 2;
    const i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    const i64 rows = (i64)L.ny * L.nz;
    if (t >= rows * kv) return;
    // thread and row indices stay below 2^31 (at most 2e9 cells): 32-bit divisions, several
    // times cheaper than 64-bit ones
    const unsigned tu = (unsigned)t, rowu = tu / (unsigned)kv;
    const i64 row = rowu;
    const int k0 = (int)(tu - rowu * (unsigned)kv) << 2;
    const int y = (int)(rowu % (unsigned)L.ny), z = (int)(rowu / (unsigned)L.ny);
    const int p = (col + y + z) & 1;  // x = 2k + p
    const i64 own = col * L.half + row * hx + k0;
    const i64 opp = (1 - col) * L.half + row * hx + k0;
    const bool hy0 = y > 0, hy1 = y < L.ny - 1;
    const bool hz0 = z > 0 || (GHOST && L.zlo), hz1 = z < L.nz - 1 || (GHOST && L.zhi);
    const i64 dy = hx, dz = (i64)L.ny * hx;
    // same-row other-colour window: xm[v] = O[k0+v+p-1], xp[v] = O[k0+v+p]
    auto window = [&](const float *O, float (&m)[4], float (&q)[4]) {
        const float4 c4 = *reinterpret_cast<const float4 *>(O + opp);
        if (p) {
            const float e = (k0 + 4 < hx) ? O[opp + 4] : 0.f;
            m[0] = c4.x; m[1] = c4.y; m[2] = c4.z; m[3] = c4.w;
            q[0] = c4.y; q[1] = c4.z; q[2] = c4.w; q[3] = e;
        } else {
            const float e = (k0 > 0) ? O[opp - 1] : 0.f;
            m[0] = e; m[1] = c4.x; m[2] = c4.y; m[3] = c4.z;
            q[0] = c4.x; q[1] = c4.y; q[2] = c4.z; q[3] = c4.w;
        }
    };
    auto ld4 = [&](const float *A, i64 off, bool ok, float (&v)[4]) {
        if (ok) {
            const float4 c4 = *reinterpret_cast<const float4 *>(A + off);
            v[0] = c4.x; v[1] = c4.y; v[2] = c4.z; v[3] = c4.w;
        } else {
            v[0] = v[1] = v[2] = v[3] = 0.f;
        }
    };
    // wall masks along x: the first cell of a row has no x-1 when p == 0, the last no x+1 when p == 1
    const bool xw0 = (p == 0 && k0 == 0), xw1 = (p == 1 && k0 + 4 == hx);
    float xm[4], xp[4], ym[4], yp[4], zm[4], zp[4];
    if (!FROM_ZERO) {
        window(xv, xm, xp);
        ld4(xv, opp - dy, hy0, ym);
        ld4(xv, opp + dy, hy1, yp);
        ld4(xv, opp - dz, hz0, zm);
        ld4(xv, opp + dz, hz1, zp);
    }
    float w0[4], w1[4], w2[4], w3[4], w4[4], w5[4];
    if (SFORM) {
        float sc[4], sm_[4], sp_[4], s2[4], s3[4], s4[4], s5[4];
        ld4(cf.s, own, true, sc);
        window(cf.s, sm_, sp_);
        ld4(cf.s, opp - dy, hy0, s2);
        ld4(cf.s, opp + dy, hy1, s3);
        ld4(cf.s, opp - dz, hz0, s4);
        ld4(cf.s, opp + dz, hz1, s5);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            w0[v] = (v == 0 && xw0) ? 0.f : sc[v] + sm_[v];
            w1[v] = (v == 3 && xw1) ? 0.f : sc[v] + sp_[v];
            w2[v] = hy0 ? sc[v] + s2[v] : 0.f;
            w3[v] = hy1 ? sc[v] + s3[v] : 0.f;
            w4[v] = hz0 ? sc[v] + s4[v] : 0.f;
            w5[v] = hz1 ? sc[v] + s5[v] : 0.f;
        }
    } else {
        float d0[4], d1[4];
        ld4(cf.fx, own, true, w0);           // low x face (0 at x = 0)
        window(cf.fx, d0, w1);               // high x face = the x+1 neighbour's low face
        if (xw1) w1[3] = 0.f;
        ld4(cf.fy, own, true, w2);
        ld4(cf.fy, opp + dy, hy1, w3);
        ld4(cf.fz, own, true, w4);
        ld4(cf.fz, opp + dz, hz1, w5);
        (void)d0;
        (void)d1;
    }
    float bb[4];
    ld4(b, own, true, bb);
    const float hh = SFORM ? 2.f * h2 : h2;
    float out[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        float num = 0.f;
        if (!FROM_ZERO) {
            num = w0[v] * xm[v];
            num += w1[v] * xp[v];
            num += w2[v] * ym[v];
            num += w3[v] * yp[v];
            num += w4[v] * zm[v];
            num += w5[v] * zp[v];
        }
        const float den = ((w0[v] + w1[v]) + (w2[v] + w3[v])) + (w4[v] + w5[v]);
        out[v] = __fdividef(hh * bb[v] + num, den);
    }
    if (UPDATE == 0) {
        *reinterpret_cast<float4 *>(xv + own) = make_float4(out[0], out[1], out[2], out[3]);
    } else if (UPDATE == 2) {
        const float4 blk = *reinterpret_cast<const float4 *>(xv + opp);
        const float bk[4] = {blk.x, blk.y, blk.z, blk.w};
        const float al = up.alpha, sh = up.shift;
        float2 *pr = up.p2 + row * L.nx + 2 * k0;
        float4 pvs[4];  // all loads before the first store
#pragma unroll
        for (int v = 0; v < 4; ++v) pvs[v] = *reinterpret_cast<const float4 *>(pr + 2 * v);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            float4 pv = pvs[v];  // (h0, l0, h1, l1)
            const float e0 = p ? bk[v] : out[v], e1 = p ? out[v] : bk[v];
            df_add(pv.x, pv.y, fmaf(al, e0, -sh));
            df_add(pv.z, pv.w, fmaf(al, e1, -sh));
            *reinterpret_cast<float4 *>(pr + 2 * v) = pv;
        }
    } else {
        // red at x = 2k + p, black at x = 2k + 1 - p; same-row black values O[k0..k0+3]
        const float4 blk = *reinterpret_cast<const float4 *>(xv + opp);
        const float bk[4] = {blk.x, blk.y, blk.z, blk.w};
        const float al = up.alpha, sh = up.shift;
        double *pr = up.p + row * L.nx + 2 * k0;
        double2 pvs[4];  // all loads before the first store
#pragma unroll
        for (int v = 0; v < 4; ++v) pvs[v] = *reinterpret_cast<const double2 *>(pr + 2 * v);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const double2 pv = pvs[v];
            const float e0 = p ? bk[v] : out[v], e1 = p ? out[v] : bk[v];  // cells 2(k0+v) and 2(k0+v)+1
            *reinterpret_cast<double2 *>(pr + 2 * v) =
                make_double2(pv.x + f2d_exact(fmaf(al, e0, -sh)), pv.y + f2d_exact(fmaf(al, e1, -sh)));
        }
    }
}

// ---- z-marching vectorised half sweep (split levels, hx % 4 == 0, hx / 4 >= 32) -----------
// A warp covers 32 consecutive 4-cell vectors of one row.  Each thread walks ZC planes in z
// and keeps the other colour's x (and s) of planes z-1, z and z+1 in registers, so each plane
// of the other colour comes from memory once per sweep instead of three times (z-1, z, z+1).
// The same-row window scalars (x at k0-1 and k0+4) come from the neighbouring lanes; the
// lanes at a warp's edge load them.  Lanes past the end of a row, or rows past ny, compute on
// clamped (in-bounds) indices and store nothing; all lanes of a warp share one row and one
// z-range, so the shuffles are always converged.  Arithmetic per cell is that of k_half_vec.
template <bool SFORM, bool FROM_ZERO, int UPDATE, int ZC, bool GHOST = false>
__global__ void __launch_bounds__(64, 12) k_half_z(Lay L, float h2, Coef32 cf, const float *__restrict__ b,
                                                    float *xv, int col, Upd up) {
    const int hx = L.hx, kv = hx >> 2;
    const int kvi = blockIdx.x * blockDim.x + threadIdx.x;
    const int yi = blockIdx.y * blockDim.y + threadIdx.y;
    const bool active = kvi < kv && yi < L.ny;
    const int k0 = min(kvi, kv - 1) << 2;
    const int y = min(yi, L.ny - 1);
    const int z0 = blockIdx.z * ZC, z1 = min(z0 + ZC, L.nz);
    const int lane = threadIdx.x & 31;
    const i64 dy = hx, dz = (i64)L.ny * hx;
    const bool hy0 = y > 0, hy1 = y < L.ny - 1;
    const bool kl = k0 > 0, kr = k0 + 4 < hx;
    i64 opp = (i64)(1 - col) * L.half + ((i64)z0 * L.ny + y) * hx + k0;
    i64 own = (i64)col * L.half + ((i64)z0 * L.ny + y) * hx + k0;
    const float4 f0 = make_float4(0.f, 0.f, 0.f, 0.f);
    auto ld = [](const float *A, i64 off) { return *reinterpret_cast<const float4 *>(A + off); };
    // planes z-1 and z of the other colour (x, and s in SFORM)
    float4 xzm = f0, xzc = f0, szm = f0, szc = f0;
    const bool glo = GHOST && L.zlo, ghi = GHOST && L.zhi;  // a slab's ghost planes are neighbours
    if (!FROM_ZERO) {
        if (z0 > 0 || glo) xzm = ld(xv, opp - dz);
        xzc = ld(xv, opp);
    }
    if (SFORM) {
        if (z0 > 0 || glo) szm = ld(cf.s, opp - dz);
        szc = ld(cf.s, opp);
    }
    const float hh = SFORM ? 2.f * h2 : h2;
    for (int z = z0; z < z1; ++z) {
        const bool hz0 = z > 0 || glo, hz1 = z < L.nz - 1 || ghi;
        const int p = (col + y + z) & 1;  // x = 2k + p
        const bool xw0 = (p == 0 && !kl), xw1 = (p == 1 && !kr);
        float4 xzp = f0, ym = f0, yp = f0;
        if (!FROM_ZERO) {
            if (hz1) xzp = ld(xv, opp + dz);
            if (hy0) ym = ld(xv, opp - dy);
            if (hy1) yp = ld(xv, opp + dy);
        }
        float w0[4], w1[4], w2[4], w3[4], w4[4], w5[4];
        float4 szp = f0;
        if (SFORM) {
            float4 s2 = f0, s3 = f0;
            if (hz1) szp = ld(cf.s, opp + dz);
            if (hy0) s2 = ld(cf.s, opp - dy);
            if (hy1) s3 = ld(cf.s, opp + dy);
            const float4 sc4 = ld(cf.s, own);
            float sl = __shfl_up_sync(0xffffffffu, szc.w, 1), sr = __shfl_down_sync(0xffffffffu, szc.x, 1);
            if (lane == 0) sl = kl ? cf.s[opp - 1] : 0.f;
            if (lane == 31) sr = kr ? cf.s[opp + 4] : 0.f;
            const float so[4] = {szc.x, szc.y, szc.z, szc.w}, sc[4] = {sc4.x, sc4.y, sc4.z, sc4.w};
            const float s2v[4] = {s2.x, s2.y, s2.z, s2.w}, s3v[4] = {s3.x, s3.y, s3.z, s3.w};
            const float s4v[4] = {szm.x, szm.y, szm.z, szm.w}, s5v[4] = {szp.x, szp.y, szp.z, szp.w};
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const float sm = p ? so[v] : (v ? so[v - 1] : sl);
                const float sp = p ? (v < 3 ? so[v + 1] : sr) : so[v];
                w0[v] = (v == 0 && xw0) ? 0.f : sc[v] + sm;
                w1[v] = (v == 3 && xw1) ? 0.f : sc[v] + sp;
                w2[v] = hy0 ? sc[v] + s2v[v] : 0.f;
                w3[v] = hy1 ? sc[v] + s3v[v] : 0.f;
                w4[v] = hz0 ? sc[v] + s4v[v] : 0.f;
                w5[v] = hz1 ? sc[v] + s5v[v] : 0.f;
            }
        } else {
            const float4 fo = ld(cf.fx, opp);  // low x faces of the other colour = high faces of own
            float fr = __shfl_down_sync(0xffffffffu, fo.x, 1);
            if (lane == 31) fr = kr ? cf.fx[opp + 4] : 0.f;
            const float fov[4] = {fo.x, fo.y, fo.z, fo.w};
            const float4 a0 = ld(cf.fx, own), a2 = ld(cf.fy, own), a4 = ld(cf.fz, own);
            const float4 a3 = hy1 ? ld(cf.fy, opp + dy) : f0, a5 = hz1 ? ld(cf.fz, opp + dz) : f0;
            const float a0v[4] = {a0.x, a0.y, a0.z, a0.w}, a2v[4] = {a2.x, a2.y, a2.z, a2.w};
            const float a3v[4] = {a3.x, a3.y, a3.z, a3.w}, a4v[4] = {a4.x, a4.y, a4.z, a4.w};
            const float a5v[4] = {a5.x, a5.y, a5.z, a5.w};
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                w0[v] = a0v[v];
                w1[v] = (v == 3 && xw1) ? 0.f : (p ? (v < 3 ? fov[v + 1] : fr) : fov[v]);
                w2[v] = a2v[v];
                w3[v] = a3v[v];
                w4[v] = a4v[v];
                w5[v] = a5v[v];
            }
        }
        const float4 b4 = ld(b, own);
        const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
        float out[4];
        if (FROM_ZERO) {
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const float den = ((w0[v] + w1[v]) + (w2[v] + w3[v])) + (w4[v] + w5[v]);
                out[v] = __fdividef(hh * bv[v], den);
            }
        } else {
            float xl = __shfl_up_sync(0xffffffffu, xzc.w, 1), xr = __shfl_down_sync(0xffffffffu, xzc.x, 1);
            if (lane == 0) xl = kl ? xv[opp - 1] : 0.f;
            if (lane == 31) xr = kr ? xv[opp + 4] : 0.f;
            const float xo[4] = {xzc.x, xzc.y, xzc.z, xzc.w};
            const float ymv[4] = {ym.x, ym.y, ym.z, ym.w}, ypv[4] = {yp.x, yp.y, yp.z, yp.w};
            const float zmv[4] = {xzm.x, xzm.y, xzm.z, xzm.w}, zpv[4] = {xzp.x, xzp.y, xzp.z, xzp.w};
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const float xm = p ? xo[v] : (v ? xo[v - 1] : xl);
                const float xp = (v == 3 && xw1) ? 0.f : (p ? (v < 3 ? xo[v + 1] : xr) : xo[v]);
                float num = w0[v] * xm;
                num += w1[v] * xp;
                num += w2[v] * ymv[v];
                num += w3[v] * ypv[v];
                num += w4[v] * zmv[v];
                num += w5[v] * zpv[v];
                const float den = ((w0[v] + w1[v]) + (w2[v] + w3[v])) + (w4[v] + w5[v]);
                out[v] = __fdividef(hh * bv[v] + num, den);
            }
        }
        if (active) {
            if (UPDATE == 0) {
                *reinterpret_cast<float4 *>(xv + own) = make_float4(out[0], out[1], out[2], out[3]);
            } else {
                // red at x = 2k + p, black at x = 2k + 1 - p; the black values are xzc
                const float bk[4] = {xzc.x, xzc.y, xzc.z, xzc.w};
                const i64 nat = ((i64)z * L.ny + y) * L.nx + 2 * k0;
                if (UPDATE == 2) {
                    const float al = up.alpha, sh = up.shift;
                    float2 *pr = up.p2 + nat;
                    // all loads before the first store: otherwise the four read-modify-writes
                    // of the same row run one HBM round trip after another
                    float4 pvs[4];
#pragma unroll
                    for (int v = 0; v < 4; ++v) pvs[v] = *reinterpret_cast<const float4 *>(pr + 2 * v);  // (h0, l0, h1, l1)
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        float4 pv = pvs[v];
                        const float e0 = p ? bk[v] : out[v], e1 = p ? out[v] : bk[v];
                        df_add(pv.x, pv.y, fmaf(al, e0, -sh));
                        df_add(pv.z, pv.w, fmaf(al, e1, -sh));
                        *reinterpret_cast<float4 *>(pr + 2 * v) = pv;
                    }
                } else {
                    // FP32 correction alpha e - shift, one FP64 addition per cell
                    const float al = up.alpha, sh = up.shift;
                    double *pr = up.p + nat;
                    double2 pvs[4];  // all loads before the first store (see above)
#pragma unroll
                    for (int v = 0; v < 4; ++v) pvs[v] = *reinterpret_cast<const double2 *>(pr + 2 * v);
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const double2 pv = pvs[v];
                        const float e0 = p ? bk[v] : out[v], e1 = p ? out[v] : bk[v];
                        *reinterpret_cast<double2 *>(pr + 2 * v) =
                            make_double2(pv.x + f2d_exact(fmaf(al, e0, -sh)), pv.y + f2d_exact(fmaf(al, e1, -sh)));
                    }
                }
            }
        }
        xzm = xzc;
        xzc = xzp;
        szm = szc;
        szc = szp;
        own += dz;
        opp += dz;
    }
}

// Staged form of k_half_z for the s-form regular sweep (the finest level's dominant kernel).
// The per-plane loads of a thread (the other colour's rows y -+ 1 and their s, its own s and
// b: six 16-byte vectors) travel by cp.async into a ring of kZsStages planes in shared memory,
// issued kZsStages - 1 planes ahead of the plane being computed.  In flight they hold no
// registers (121 registers for one plane held in registers, 80 here), so 11 blocks fit per SM
// instead of 8, each with two planes of loads under way.  Every thread reads back only its
// own copies: cp.async.wait_group is its only wait (no barrier, no spin), and a slot is
// refilled only after the arithmetic that used it.  The other colour's row y (planes z -+ 1
// and the window) still rolls through registers, the next plane's window scalars of the
// warp's edge lanes too.  Arithmetic as k_half_z: bitwise the same results.
constexpr int kZsStages = 3;
constexpr int kZsFields = 6;  // ym, yp, s2 (= s at y - 1), s3 (y + 1), own s, own b
constexpr size_t kZsSmem = (size_t)kZsStages * kZsFields * 64 * sizeof(float4);

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// 64 threads per block (64 vectors of one row, or 32 of two rows), ZC planes per block
template <int ZC, int MINB, bool GHOST = false>
__global__ void __launch_bounds__(64, MINB) k_half_zs(Lay L, float h2, const float *__restrict__ sv,
                                                       const float *__restrict__ b, float *xv, int col) {
    extern __shared__ float4 stg[];  // [kZsStages][kZsFields][64 threads]
    constexpr int D = kZsStages;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int hx = L.hx, kv = hx >> 2;
    const int kvi = blockIdx.x * blockDim.x + threadIdx.x;
    const int yi = blockIdx.y * blockDim.y + threadIdx.y;
    const bool active = kvi < kv && yi < L.ny;
    const int k0 = min(kvi, kv - 1) << 2;
    const int y = min(yi, L.ny - 1);
    const int z0 = blockIdx.z * ZC, z1 = min(z0 + ZC, L.nz);
    const int lane = threadIdx.x & 31;
    const i64 dy = hx, dz = (i64)L.ny * hx;
    const bool hy0 = y > 0, hy1 = y < L.ny - 1;
    const bool kl = k0 > 0, kr = k0 + 4 < hx;
    const i64 row0 = ((i64)z0 * L.ny + y) * hx + k0;
    const i64 opp0 = (i64)(1 - col) * L.half + row0;
    const i64 own0 = (i64)col * L.half + row0;
    const float4 f0 = make_float4(0.f, 0.f, 0.f, 0.f);
    auto ld = [](const float *A, i64 off) { return *reinterpret_cast<const float4 *>(A + off); };
    auto slot = [&](int st, int f) { return stg + (st * kZsFields + f) * 64 + tid; };
    // plane z0 + t into stage t % D (rows outside the grid are not copied; their slots are
    // never read)
    auto issue = [&](int t) {
        const i64 o = opp0 + (i64)t * dz, w = own0 + (i64)t * dz;
        const int st = t % D;
        if (hy0) {
            cp_async16(slot(st, 0), xv + o - dy);
            cp_async16(slot(st, 2), sv + o - dy);
        }
        if (hy1) {
            cp_async16(slot(st, 1), xv + o + dy);
            cp_async16(slot(st, 3), sv + o + dy);
        }
        cp_async16(slot(st, 4), sv + w);
        cp_async16(slot(st, 5), b + w);
    };
    // the window scalars beyond the warp's edge lanes (lane 0: x - 1, lane 31: x + 4)
    auto scalars = [&](i64 o, float &xl, float &sl, float &xr, float &sr) {
        xl = sl = xr = sr = 0.f;
        if (lane == 0 && kl) {
            xl = xv[o - 1];
            sl = sv[o - 1];
        }
        if (lane == 31 && kr) {
            xr = xv[o + 4];
            sr = sv[o + 4];
        }
    };
    // other colour, row y: planes z-1, z, z+1 (rolling); a slab's ghost planes are neighbours
    const bool glo = GHOST && L.zlo, ghi = GHOST && L.zhi;
    const int zend = L.nz + (ghi ? 1 : 0);  // planes readable above: the ghost plane too
    float4 xzm = (z0 > 0 || glo) ? ld(xv, opp0 - dz) : f0, xzc = ld(xv, opp0);
    float4 szm = (z0 > 0 || glo) ? ld(sv, opp0 - dz) : f0, szc = ld(sv, opp0);
    float4 xzp = z0 + 1 < zend ? ld(xv, opp0 + dz) : f0, szp = z0 + 1 < zend ? ld(sv, opp0 + dz) : f0;
#pragma unroll
    for (int t = 0; t < D - 1; ++t) {
        if (z0 + t < z1) issue(t);
        cp_async_commit();  // one group per plane, empty past the chunk: the counting stays uniform
    }
    float cxl, csl, cxr, csr;
    scalars(opp0, cxl, csl, cxr, csr);
    const float hh = 2.f * h2;
    for (int z = z0; z < z1; ++z) {
        const int t = z - z0;
        if (z + D - 1 < z1) issue(t + D - 1);
        cp_async_commit();
        const i64 opp = opp0 + (i64)t * dz, own = own0 + (i64)t * dz;
        float nxl = 0.f, nsl = 0.f, nxr = 0.f, nsr = 0.f;
        float4 xzpp = f0, szpp = f0;
        if (z + 1 < z1) {
            scalars(opp + dz, nxl, nsl, nxr, nsr);
            if (z + 2 < zend) {
                xzpp = ld(xv, opp + 2 * dz);
                szpp = ld(sv, opp + 2 * dz);
            }
        }
        cp_async_wait<D - 1>();  // all but the D - 1 newest groups done: plane z has landed
        const int st = t % D;
        const float4 cym = hy0 ? *slot(st, 0) : f0, cyp = hy1 ? *slot(st, 1) : f0;
        const float4 cs2 = hy0 ? *slot(st, 2) : f0, cs3 = hy1 ? *slot(st, 3) : f0;
        const float4 csc = *slot(st, 4), cbb = *slot(st, 5);
        const bool hz0 = z > 0 || glo, hz1 = z < L.nz - 1 || ghi;
        const int p = (col + y + z) & 1;  // x = 2k + p
        const bool xw0 = (p == 0 && !kl), xw1 = (p == 1 && !kr);
        float sl = __shfl_up_sync(0xffffffffu, szc.w, 1), sr = __shfl_down_sync(0xffffffffu, szc.x, 1);
        float xl = __shfl_up_sync(0xffffffffu, xzc.w, 1), xr = __shfl_down_sync(0xffffffffu, xzc.x, 1);
        if (lane == 0) {
            sl = csl;
            xl = cxl;
        }
        if (lane == 31) {
            sr = csr;
            xr = cxr;
        }
        const float so[4] = {szc.x, szc.y, szc.z, szc.w}, sc[4] = {csc.x, csc.y, csc.z, csc.w};
        const float s2v[4] = {cs2.x, cs2.y, cs2.z, cs2.w}, s3v[4] = {cs3.x, cs3.y, cs3.z, cs3.w};
        const float s4v[4] = {szm.x, szm.y, szm.z, szm.w}, s5v[4] = {szp.x, szp.y, szp.z, szp.w};
        const float xov[4] = {xzc.x, xzc.y, xzc.z, xzc.w};
        const float ymv[4] = {cym.x, cym.y, cym.z, cym.w}, ypv[4] = {cyp.x, cyp.y, cyp.z, cyp.w};
        const float zmv[4] = {xzm.x, xzm.y, xzm.z, xzm.w}, zpv[4] = {xzp.x, xzp.y, xzp.z, xzp.w};
        const float bv[4] = {cbb.x, cbb.y, cbb.z, cbb.w};
        float out[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const float sm = p ? so[v] : (v ? so[v - 1] : sl);
            const float sp = p ? (v < 3 ? so[v + 1] : sr) : so[v];
            const float w0 = (v == 0 && xw0) ? 0.f : sc[v] + sm;
            const float w1 = (v == 3 && xw1) ? 0.f : sc[v] + sp;
            const float w2 = hy0 ? sc[v] + s2v[v] : 0.f;
            const float w3 = hy1 ? sc[v] + s3v[v] : 0.f;
            const float w4 = hz0 ? sc[v] + s4v[v] : 0.f;
            const float w5 = hz1 ? sc[v] + s5v[v] : 0.f;
            const float xm = p ? xov[v] : (v ? xov[v - 1] : xl);
            const float xp = (v == 3 && xw1) ? 0.f : (p ? (v < 3 ? xov[v + 1] : xr) : xov[v]);
            float num = w0 * xm;
            num += w1 * xp;
            num += w2 * ymv[v];
            num += w3 * ypv[v];
            num += w4 * zmv[v];
            num += w5 * zpv[v];
            const float den = ((w0 + w1) + (w2 + w3)) + (w4 + w5);
            out[v] = __fdividef(hh * bv[v] + num, den);
        }
        if (active) __stcs(reinterpret_cast<float4 *>(xv + own), make_float4(out[0], out[1], out[2], out[3]));  // streaming store
        xzm = xzc;
        xzc = xzp;
        xzp = xzpp;
        szm = szc;
        szc = szp;
        szp = szpp;
        cxl = nxl;
        csl = nsl;
        cxr = nxr;
        csr = nsr;
    }
    cp_async_wait<0>();  // only empty groups can remain; leave none behind
}

// Staged form of k_half_z for the face-form regular sweep (the levels below the finest, whose
// coarsened faces are stored per face, and a finest level loaded from face coefficients).  A
// thread's nine per-plane vectors -- the other colour's x in rows y -+ 1, the other colour's
// low x faces (its cells' high x faces), its own low x, y and z faces, the other colour's low
// y faces in row y + 1 and low z faces in plane z + 1 (its high y and z faces), its own b --
// travel by cp.async into a ring of kZfStages planes in shared memory, one plane ahead of the
// plane being computed, as in k_half_zs; the other colour's row y (planes z -+ 1) rolls
// through registers, the window scalars of the warp's edge lanes are loaded one plane ahead.
// Every thread reads back only its own copies after cp.async.wait_group (no barrier, no spin).
// Arithmetic as k_half_z, in the same order: bitwise the same results.
constexpr int kZfStages = 2;
constexpr int kZfFields = 9;  // ym, yp, fo, own fx, fy, fz, fy at y + 1, fz at z + 1, own b
constexpr size_t kZfSmem = (size_t)kZfStages * kZfFields * 64 * sizeof(float4);

template <int ZC, int MINB>
__global__ void __launch_bounds__(64, MINB) k_half_zf(Lay L, float h2, Coef32 cf, const float *__restrict__ b,
                                                       float *xv, int col) {
    extern __shared__ float4 stg[];  // [kZfStages][kZfFields][64 threads]
    constexpr int D = kZfStages;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int hx = L.hx, kv = hx >> 2;
    const int kvi = blockIdx.x * blockDim.x + threadIdx.x;
    const int yi = blockIdx.y * blockDim.y + threadIdx.y;
    const bool active = kvi < kv && yi < L.ny;
    const int k0 = min(kvi, kv - 1) << 2;
    const int y = min(yi, L.ny - 1);
    const int z0 = blockIdx.z * ZC, z1 = min(z0 + ZC, L.nz);
    const int lane = threadIdx.x & 31;
    const i64 dy = hx, dz = (i64)L.ny * hx;
    const bool hy0 = y > 0, hy1 = y < L.ny - 1;
    const bool kl = k0 > 0, kr = k0 + 4 < hx;
    const i64 row0 = ((i64)z0 * L.ny + y) * hx + k0;
    const i64 opp0 = (i64)(1 - col) * L.half + row0;
    const i64 own0 = (i64)col * L.half + row0;
    const float4 f0 = make_float4(0.f, 0.f, 0.f, 0.f);
    auto ld = [](const float *A, i64 off) { return *reinterpret_cast<const float4 *>(A + off); };
    auto slot = [&](int st, int f) { return stg + (st * kZfFields + f) * 64 + tid; };
    // plane z0 + t into stage t % D (slots whose neighbour is outside the grid are not copied
    // and never read)
    auto issue = [&](int t) {
        const i64 o = opp0 + (i64)t * dz, w = own0 + (i64)t * dz;
        const int st = t % D;
        if (hy0) cp_async16(slot(st, 0), xv + o - dy);
        if (hy1) {
            cp_async16(slot(st, 1), xv + o + dy);
            cp_async16(slot(st, 6), cf.fy + o + dy);
        }
        cp_async16(slot(st, 2), cf.fx + o);
        cp_async16(slot(st, 3), cf.fx + w);
        cp_async16(slot(st, 4), cf.fy + w);
        cp_async16(slot(st, 5), cf.fz + w);
        if (z0 + t < L.nz - 1) cp_async16(slot(st, 7), cf.fz + o + dz);
        cp_async16(slot(st, 8), b + w);
    };
    // the window scalars beyond the warp's edge lanes (lane 0: x at k0 - 1; lane 31: x and the
    // low x face at k0 + 4)
    auto scalars = [&](i64 o, float &xl, float &xr, float &fr) {
        xl = xr = fr = 0.f;
        if (lane == 0 && kl) xl = xv[o - 1];
        if (lane == 31 && kr) {
            xr = xv[o + 4];
            fr = cf.fx[o + 4];
        }
    };
    // other colour, row y: planes z-1, z, z+1 (rolling)
    float4 xzm = z0 > 0 ? ld(xv, opp0 - dz) : f0, xzc = ld(xv, opp0);
    float4 xzp = z0 + 1 < L.nz ? ld(xv, opp0 + dz) : f0;
#pragma unroll
    for (int t = 0; t < D - 1; ++t) {
        if (z0 + t < z1) issue(t);
        cp_async_commit();  // one group per plane, empty past the chunk: the counting stays uniform
    }
    float cxl, cxr, cfr;
    scalars(opp0, cxl, cxr, cfr);
    for (int z = z0; z < z1; ++z) {
        const int t = z - z0;
        if (z + D - 1 < z1) issue(t + D - 1);
        cp_async_commit();
        const i64 opp = opp0 + (i64)t * dz, own = own0 + (i64)t * dz;
        float nxl = 0.f, nxr = 0.f, nfr = 0.f;
        float4 xzpp = f0;
        if (z + 1 < z1) {
            scalars(opp + dz, nxl, nxr, nfr);
            if (z + 2 < L.nz) xzpp = ld(xv, opp + 2 * dz);
        }
        cp_async_wait<D - 1>();  // all but the D - 1 newest groups done: plane z has landed
        const int st = t % D;
        const bool hz1 = z < L.nz - 1;
        const int p = (col + y + z) & 1;  // x = 2k + p
        const bool xw1 = (p == 1 && !kr);
        const float4 ym = hy0 ? *slot(st, 0) : f0, yp = hy1 ? *slot(st, 1) : f0;
        const float4 fo = *slot(st, 2), a0 = *slot(st, 3), a2 = *slot(st, 4), a4 = *slot(st, 5);
        const float4 a3 = hy1 ? *slot(st, 6) : f0, a5 = hz1 ? *slot(st, 7) : f0;
        const float4 b4 = *slot(st, 8);
        float fr = __shfl_down_sync(0xffffffffu, fo.x, 1);
        if (lane == 31) fr = cfr;
        float xl = __shfl_up_sync(0xffffffffu, xzc.w, 1), xr = __shfl_down_sync(0xffffffffu, xzc.x, 1);
        if (lane == 0) xl = cxl;
        if (lane == 31) xr = cxr;
        const float fov[4] = {fo.x, fo.y, fo.z, fo.w};
        const float a0v[4] = {a0.x, a0.y, a0.z, a0.w}, a2v[4] = {a2.x, a2.y, a2.z, a2.w};
        const float a3v[4] = {a3.x, a3.y, a3.z, a3.w}, a4v[4] = {a4.x, a4.y, a4.z, a4.w};
        const float a5v[4] = {a5.x, a5.y, a5.z, a5.w};
        const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
        const float xo[4] = {xzc.x, xzc.y, xzc.z, xzc.w};
        const float ymv[4] = {ym.x, ym.y, ym.z, ym.w}, ypv[4] = {yp.x, yp.y, yp.z, yp.w};
        const float zmv[4] = {xzm.x, xzm.y, xzm.z, xzm.w}, zpv[4] = {xzp.x, xzp.y, xzp.z, xzp.w};
        float out[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const float w0 = a0v[v];
            const float w1 = (v == 3 && xw1) ? 0.f : (p ? (v < 3 ? fov[v + 1] : fr) : fov[v]);
            const float w2 = a2v[v], w3 = a3v[v], w4 = a4v[v], w5 = a5v[v];
            const float xm = p ? xo[v] : (v ? xo[v - 1] : xl);
            const float xp = (v == 3 && xw1) ? 0.f : (p ? (v < 3 ? xo[v + 1] : xr) : xo[v]);
            float num = w0 * xm;
            num += w1 * xp;
            num += w2 * ymv[v];
            num += w3 * ypv[v];
            num += w4 * zmv[v];
            num += w5 * zpv[v];
            const float den = ((w0 + w1) + (w2 + w3)) + (w4 + w5);
            out[v] = __fdividef(h2 * bv[v] + num, den);
        }
        if (active) *reinterpret_cast<float4 *>(xv + own) = make_float4(out[0], out[1], out[2], out[3]);
        xzm = xzc;
        xzc = xzp;
        xzp = xzpp;
        cxl = nxl;
        cxr = nxr;
        cfr = nfr;
    }
    cp_async_wait<0>();  // only empty groups can remain; leave none behind
}

bool half_z_ok(const Lay &L) { return L.split && L.hx % 4 == 0 && L.hx / 4 >= 32; }

// 16 planes per thread where that still gives about 4 waves of 64-thread blocks (12 resident
// per SM, on the device's SM count), else 4
template <bool SFORM, bool FROM_ZERO, int UPDATE, bool GHOST = false>
void run_half_z(cudaStream_t s, const Lay &L, float h2, const Coef32 &cf, const float *b, float *x, int col,
                const Upd &up) {
    const int kv = L.hx / 4;
    const int vb = (kv % 64 == 0) ? 64 : 32;  // lanes per row
    const int ry = 64 / vb;                    // rows per block
    const unsigned gx = (kv + vb - 1) / vb, gy = (L.ny + ry - 1) / ry;
    const dim3 blk(vb, ry);
    const i64 sms = device_sms();
    // a slab's launch runs beside the other slabs' ones: it needs about one wave by itself
    if (SFORM && !FROM_ZERO && UPDATE == 0 && (i64)gx * gy * ((L.nz + 15) / 16) >= (GHOST ? 1 : 4) * sms * 8) {
        // 11 blocks x 18 KB of staging per SM: ask for the largest shared-memory carveout
        static const bool carveout = [] {
            // a preference only: the launch is valid either way
            if (cudaFuncSetAttribute(k_half_zs<16, 11, GHOST>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
                (void)cudaGetLastError();
            return true;
        }();
        (void)carveout;
        k_half_zs<16, 11, GHOST><<<dim3(gx, gy, (L.nz + 15) / 16), blk, kZsSmem, s>>>(L, h2, cf.s, b, x, col);
        return;
    }
    // the face form's regular sweeps, staged, where the grid gives at least four waves of
    // 4-plane blocks (11 blocks x 18 KB of staging per SM, as k_half_zs)
    if (!SFORM && !FROM_ZERO && UPDATE == 0 && !GHOST && (i64)gx * gy * ((L.nz + 3) / 4) >= 4 * sms * 11) {
        static const bool carveout = [] {
            // a preference only: the launch is valid either way
            if (cudaFuncSetAttribute(k_half_zf<4, 11>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
                (void)cudaGetLastError();
            return true;
        }();
        (void)carveout;
        k_half_zf<4, 11><<<dim3(gx, gy, (L.nz + 3) / 4), blk, kZfSmem, s>>>(L, h2, cf, b, x, col);
        return;
    }
    if ((i64)gx * gy * ((L.nz + 15) / 16) >= 4 * sms * 12)
        k_half_z<SFORM, FROM_ZERO, UPDATE, 16, GHOST><<<dim3(gx, gy, (L.nz + 15) / 16), blk, 0, s>>>(L, h2, cf, b, x, col, up);
    else
        k_half_z<SFORM, FROM_ZERO, UPDATE, 4, GHOST><<<dim3(gx, gy, (L.nz + 3) / 4), blk, 0, s>>>(L, h2, cf, b, x, col, up);
}

// ---- vectorised red-only residual + restriction (split fine level, hx % 4 == 0) ----------
// The red children of coarse cell (I, J, K) are the red cells at k = I of the 4 fine rows
// (2J + b, 2K + c); one thread handles coarse cells I0..I0+3 of one coarse row.
constexpr int kRrThreads = 64;

// GHOST: the fine level is a slab (L.zlo / L.zhi) and Lc a view of the whole coarse level
// (its arrays at the slab's first coarse plane, an even one)
template <bool SFORM, bool GHOST = false>
__global__ void __launch_bounds__(kRrThreads, 12) k_rr_red_vec(Lay L, Lay Lc, float ih2, Coef32 cf, const float *__restrict__ b,
                             const float *__restrict__ xv, float *bc) {
    const int hx = L.hx, kv = hx >> 2;
    const i64 T = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    const i64 crows = (i64)Lc.ny * Lc.nz;
    if (T >= crows * kv) return;
    // thread and row indices stay below 2^31 (at most 2e9 cells): 32-bit divisions, several
    // times cheaper than 64-bit ones
    const unsigned Tu = (unsigned)T, crowu = Tu / (unsigned)kv;
    const int k0 = (int)(Tu - crowu * (unsigned)kv) << 2;
    const int J = (int)(crowu % (unsigned)Lc.ny), K = (int)(crowu / (unsigned)Lc.ny);
    const i64 dy = hx, dz = (i64)L.ny * hx;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
        const int y = 2 * J + (ch & 1), z = 2 * K + (ch >> 1);
        const int p = (y + z) & 1;  // red cells of this row sit at x = 2k + p
        const i64 row = (i64)z * L.ny + y;
        const i64 own = row * hx + k0;               // red half
        const i64 opp = L.half + row * hx + k0;      // black half
        const bool hy0 = y > 0, hy1 = y < L.ny - 1;
        const bool hz0 = z > 0 || (GHOST && L.zlo), hz1 = z < L.nz - 1 || (GHOST && L.zhi);
        const bool xw0 = (p == 0 && k0 == 0), xw1 = (p == 1 && k0 + 4 == hx);
        auto window = [&](const float *O, float (&m)[4], float (&q)[4]) {
            const float4 c4 = *reinterpret_cast<const float4 *>(O + opp);
            if (p) {
                const float e = (k0 + 4 < hx) ? O[opp + 4] : 0.f;
                m[0] = c4.x; m[1] = c4.y; m[2] = c4.z; m[3] = c4.w;
                q[0] = c4.y; q[1] = c4.z; q[2] = c4.w; q[3] = e;
            } else {
                const float e = (k0 > 0) ? O[opp - 1] : 0.f;
                m[0] = e; m[1] = c4.x; m[2] = c4.y; m[3] = c4.z;
                q[0] = c4.x; q[1] = c4.y; q[2] = c4.z; q[3] = c4.w;
            }
        };
        auto ld4 = [&](const float *A, i64 off, bool ok, float (&v)[4]) {
            if (ok) {
                const float4 c4 = *reinterpret_cast<const float4 *>(A + off);
                v[0] = c4.x; v[1] = c4.y; v[2] = c4.z; v[3] = c4.w;
            } else {
                v[0] = v[1] = v[2] = v[3] = 0.f;
            }
        };
        float xc[4], xm[4], xp[4], ym[4], yp[4], zm[4], zp[4], bb[4];
        ld4(xv, own, true, xc);
        window(xv, xm, xp);
        ld4(xv, opp - dy, hy0, ym);
        ld4(xv, opp + dy, hy1, yp);
        ld4(xv, opp - dz, hz0, zm);
        ld4(xv, opp + dz, hz1, zp);
        ld4(b, own, true, bb);
        float w0[4], w1[4], w2[4], w3[4], w4[4], w5[4];
        if (SFORM) {
            float sc[4], sm_[4], sp_[4], s2[4], s3[4], s4[4], s5[4];
            ld4(cf.s, own, true, sc);
            window(cf.s, sm_, sp_);
            ld4(cf.s, opp - dy, hy0, s2);
            ld4(cf.s, opp + dy, hy1, s3);
            ld4(cf.s, opp - dz, hz0, s4);
            ld4(cf.s, opp + dz, hz1, s5);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                w0[v] = (v == 0 && xw0) ? 0.f : 0.5f * (sc[v] + sm_[v]);
                w1[v] = (v == 3 && xw1) ? 0.f : 0.5f * (sc[v] + sp_[v]);
                w2[v] = hy0 ? 0.5f * (sc[v] + s2[v]) : 0.f;
                w3[v] = hy1 ? 0.5f * (sc[v] + s3[v]) : 0.f;
                w4[v] = hz0 ? 0.5f * (sc[v] + s4[v]) : 0.f;
                w5[v] = hz1 ? 0.5f * (sc[v] + s5[v]) : 0.f;
            }
        } else {
            float d0[4];
            ld4(cf.fx, own, true, w0);
            window(cf.fx, d0, w1);
            if (xw1) w1[3] = 0.f;
            ld4(cf.fy, own, true, w2);
            ld4(cf.fy, opp + dy, hy1, w3);
            ld4(cf.fz, own, true, w4);
            ld4(cf.fz, opp + dz, hz1, w5);
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            float ax = w0[v] * (xc[v] - xm[v]);
            ax += w1[v] * (xc[v] - xp[v]);
            ax += w2[v] * (xc[v] - ym[v]);
            ax += w3[v] * (xc[v] - yp[v]);
            ax += w4[v] * (xc[v] - zm[v]);
            ax += w5[v] * (xc[v] - zp[v]);
            acc[v] += bb[v] - ax * ih2;
        }
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) bc[sto(Lc, k0 + v, J, K)] = acc[v] * 0.125f;
}

// ---- vectorised red-only prolongation + correction (split fine level, hx % 4 == 0) -------
// one thread adds P ec to 4 consecutive red cells of one fine row
__global__ void k_prolong_red_vec(Lay L, Lay Lc, const float *__restrict__ ec, float *xv, int kind) {
    const int hx = L.hx, kv = hx >> 2;
    const i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    const i64 rows = (i64)L.ny * L.nz;
    if (t >= rows * kv) return;
    // thread and row indices stay below 2^31 (at most 2e9 cells): 32-bit divisions, several
    // times cheaper than 64-bit ones
    const unsigned tu = (unsigned)t, rowu = tu / (unsigned)kv;
    const i64 row = rowu;
    const int k0 = (int)(tu - rowu * (unsigned)kv) << 2;
    const int y = (int)(rowu % (unsigned)L.ny), z = (int)(rowu / (unsigned)L.ny);
    const int p = (y + z) & 1;  // red x = 2k + p, coarse I = k
    const int J = y >> 1, K = z >> 1;
    float out[4];
    float4 x4 = *reinterpret_cast<const float4 *>(xv + row * hx + k0);
    out[0] = x4.x; out[1] = x4.y; out[2] = x4.z; out[3] = x4.w;
    if (kind == MG_PROLONG_CONSTANT) {
#pragma unroll
        for (int v = 0; v < 4; ++v) out[v] += __ldg(ec + sto(Lc, k0 + v, J, K));
    } else {
        int J2 = (y & 1) ? J + 1 : J - 1;
        int K2 = (z & 1) ? K + 1 : K - 1;
        if (J2 < 0 || J2 >= Lc.ny) J2 = J;
        if (K2 < 0 || K2 >= Lc.nz) K2 = K;
        // coarse values at I = k0 - 1 .. k0 + 4 of the four coarse rows
        float c[4][6];
        const int Js[2] = {J, J2}, Ks[2] = {K, K2};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int JJ = Js[r & 1], KK = Ks[r >> 1];
#pragma unroll
            for (int u = 0; u < 6; ++u) {
                int I = k0 - 1 + u;
                if (I < 0) I = 0;
                if (I >= Lc.nx) I = Lc.nx - 1;
                c[r][u] = __ldg(ec + sto(Lc, I, JJ, KK));
            }
        }
        const float w0 = 0.75f, w1 = 0.25f;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int I = k0 + v;
            int I2 = p ? I + 1 : I - 1;
            if (I2 < 0 || I2 >= Lc.nx) I2 = I;
            const int u1 = I + 1 - k0, u2 = I2 + 1 - k0;  // positions in c[][]
            float a = w0 * w0 * w0 * c[0][u1];
            a += w1 * w0 * w0 * c[0][u2];
            a += w0 * w1 * w0 * c[1][u1];
            a += w1 * w1 * w0 * c[1][u2];
            a += w0 * w0 * w1 * c[2][u1];
            a += w1 * w0 * w1 * c[2][u2];
            a += w0 * w1 * w1 * c[3][u1];
            a += w1 * w1 * w1 * c[3][u2];
            out[v] += a;
        }
    }
    *reinterpret_cast<float4 *>(xv + row * hx + k0) = make_float4(out[0], out[1], out[2], out[3]);
}

// ---- separable red-only trilinear prolongation (split fine level, coarse nx % 8 == 0) -----
// One thread takes coarse row (J, K) and I0 = k0 .. k0+7: the 8 red cells k0 .. k0+7 of each of
// the 4 fine rows y = 2J + d, z = 2K + e.  Fine row (d, e) interpolates in y and z first,
//   R_de(I) = 9/16 c(J, K) + 3/16 c(J_d, K) + 3/16 c(J, K_e) + 1/16 c(J_d, K_e)
// with J_d = J - 1 + 2d and K_e = K - 1 + 2e clamped into the grid (the wall mirror), then in x:
// the red cell at k (x = 2k + p, coarse I = k) gains 3/4 R(I) + 1/4 R(I + 2p - 1), clamped.
// Each coarse row supplies I = k0 - 1 .. k0 + 8: two float4 (even and odd I, one per colour
// half) and two scalars.
constexpr int kProlThreads = 64;

// GHOST: the fine level is a slab and Lc a view of the whole coarse level from the slab's first
// coarse plane (Lc.zlo / Lc.zhi: the coarse planes next to the view are the neighbours', read
// where the whole grid would read them instead of the wall's mirror)
template <bool GHOST = false>
__global__ void __launch_bounds__(kProlThreads, 10) k_prolong_red8(Lay L, Lay Lc, const float *__restrict__ ec, float *xv) {
    const int hx = L.hx, kv = hx >> 3;  // 8-cell groups per fine row
    const i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    const i64 crows = (i64)Lc.ny * Lc.nz;
    if (t >= crows * kv) return;
    // thread and row indices stay below 2^31 (at most 2e9 cells): 32-bit divisions, several
    // times cheaper than 64-bit ones
    const unsigned tu = (unsigned)t, crowu = tu / (unsigned)kv;
    const int k0 = (int)(tu - crowu * (unsigned)kv) << 3;
    const int J = (int)(crowu % (unsigned)Lc.ny), K = (int)(crowu / (unsigned)Lc.ny);
    const int hxc = Lc.hx, ncx = Lc.nx;
    const int Js[3] = {max(J - 1, 0), J, min(J + 1, Lc.ny - 1)};
    const int Ks[3] = {(GHOST && Lc.zlo) ? K - 1 : max(K - 1, 0), K, (GHOST && Lc.zhi) ? K + 1 : min(K + 1, Lc.nz - 1)};
    float R[4][10];  // [2e + d][I - k0 + 1]
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int u = 0; u < 10; ++u) R[r][u] = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {      // coarse row J - 1 + a
#pragma unroll
        for (int c = 0; c < 3; ++c) {  // coarse row K - 1 + c
            const int JJ = Js[a], KK = Ks[c];
            const int q = (JJ + KK) & 1;  // colour of coarse I even
            const i64 rowc = (i64)KK * Lc.ny + JJ;
            const float *ev = ec + (i64)q * Lc.half + rowc * hxc;        // even I, position I / 2
            const float *od = ec + (i64)(1 - q) * Lc.half + rowc * hxc;  // odd I
            const float4 e4 = *reinterpret_cast<const float4 *>(ev + (k0 >> 1));
            const float4 o4 = *reinterpret_cast<const float4 *>(od + (k0 >> 1));
            float v[10];
            v[1] = e4.x; v[2] = o4.x; v[3] = e4.y; v[4] = o4.y;
            v[5] = e4.z; v[6] = o4.z; v[7] = e4.w; v[8] = o4.w;
            v[0] = k0 > 0 ? od[(k0 >> 1) - 1] : v[1];          // I = k0 - 1, mirrored at the wall
            v[9] = k0 + 8 < ncx ? ev[(k0 >> 1) + 4] : v[8];    // I = k0 + 8
            // weight of this coarse row in fine row (d, e): y factor (3/4 own, 1/4 neighbour)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
#pragma unroll
                for (int d = 0; d < 2; ++d) {
                    // fine row (d, e) uses coarse rows J and J_d = J - 1 + 2d, K and K_e = K - 1 + 2e
                    const bool ya = (a == 1) || (a == 2 * d);
                    const bool za = (c == 1) || (c == 2 * e);
                    if (!ya || !za) continue;
                    // when J_d was clamped onto J the two y weights land on the same row
                    float wy = (a == 1) ? 0.75f : 0.25f;
                    float wz = (c == 1) ? 0.75f : 0.25f;
                    const float w = wy * wz;
#pragma unroll
                    for (int u = 0; u < 10; ++u) R[2 * e + d][u] = fmaf(w, v[u], R[2 * e + d][u]);
                }
            }
        }
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
#pragma unroll
        for (int d = 0; d < 2; ++d) {
            const int y = 2 * J + d, z = 2 * K + e;
            if (y >= L.ny || z >= L.nz) continue;
            const int p = (d + e) & 1;  // red x = 2k + p
            float *xr = xv + ((i64)z * L.ny + y) * hx + k0;
            float4 a4 = *reinterpret_cast<const float4 *>(xr);
            float4 b4 = *reinterpret_cast<const float4 *>(xr + 4);
            float o[8] = {a4.x, a4.y, a4.z, a4.w, b4.x, b4.y, b4.z, b4.w};
            const float *Rr = R[2 * e + d];
#pragma unroll
            for (int v = 0; v < 8; ++v) o[v] += 0.75f * Rr[v + 1] + 0.25f * (p ? Rr[v + 2] : Rr[v]);
            *reinterpret_cast<float4 *>(xr) = make_float4(o[0], o[1], o[2], o[3]);
            *reinterpret_cast<float4 *>(xr + 4) = make_float4(o[4], o[5], o[6], o[7]);
        }
    }
}

// ---- residual (generic) ------------------------------------------------------------------
// r(x, y, z) = b - A x   (FP32, any layout)
__device__ __forceinline__ float resid_any(const Lay &L, float ih2, const Coef32 &cf, const float *__restrict__ b,
                                           const float *__restrict__ xv, int x, int y, int z) {
    float num, den;
    stencil_any(L, cf, xv, x, y, z, num, den);
    const i64 c = sto(L, x, y, z);
    const float ax = xv[c] * den - num;
    return b[c] - (cf.s ? 0.5f : 1.f) * ax * ih2;
}

__global__ void k_residual_any(Lay L, float ih2, Coef32 cf, const float *__restrict__ b,
                               const float *__restrict__ xv, float *r, int apply_only) {
    const i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L.n) return;
    const int x = (int)(t % L.nx);
    const i64 row = t / L.nx;
    const int y = (int)(row % L.ny), z = (int)(row / L.ny);
    const i64 c = sto(L, x, y, z);
    if (apply_only) {
        float num, den;
        stencil_any(L, cf, xv, x, y, z, num, den);
        r[c] = (cf.s ? 0.5f : 1.f) * (xv[c] * den - num) * ih2;
    } else {
        r[c] = resid_any(L, ih2, cf, b, xv, x, y, z);
    }
}

// coarse b = mean of the children's residuals; red_only: black children contribute 0
// (exact after a black half sweep, which solves every black row)
__global__ void k_resid_restrict_any(Lay L, Lay Lc, float ih2, Coef32 cf, const float *__restrict__ b,
                                     const float *__restrict__ xv, float *bc, int red_only) {
    const i64 T = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (T >= Lc.n) return;
    const int I = (int)(T % Lc.nx);
    const i64 row = T / Lc.nx;
    const int J = (int)(row % Lc.ny), K = (int)(row / Lc.ny);
    float s = 0.f;
    for (int cc = 0; cc < 2; ++cc)
        for (int bb = 0; bb < 2; ++bb)
            for (int aa = 0; aa < 2; ++aa) {
                const int x = 2 * I + aa, y = 2 * J + bb, z = 2 * K + cc;
                if (red_only && ((x + y + z) & 1)) continue;
                s += resid_any(L, ih2, cf, b, xv, x, y, z);
            }
    bc[sto(Lc, I, J, K)] = s * 0.125f;
}

// x += P ec on cells of colour `only_col` (0 red, 1 black) or on all cells (-1)
__global__ void k_prolong_any(Lay L, Lay Lc, const float *__restrict__ ec, float *xv, int kind, int only_col) {
    const i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L.n) return;
    const int x = (int)(t % L.nx);
    const i64 row = t / L.nx;
    const int y = (int)(row % L.ny), z = (int)(row / L.ny);
    if (only_col >= 0 && ((x + y + z) & 1) != only_col) return;
    const int I = x >> 1, J = y >> 1, K = z >> 1;
    float v;
    if (kind == MG_PROLONG_CONSTANT) {
        v = ec[sto(Lc, I, J, K)];
    } else {
        int I2 = (x & 1) ? I + 1 : I - 1;
        int J2 = (y & 1) ? J + 1 : J - 1;
        int K2 = (z & 1) ? K + 1 : K - 1;
        if (I2 < 0 || I2 >= Lc.nx) I2 = I;
        if (J2 < 0 || J2 >= Lc.ny) J2 = J;
        if (K2 < 0 || K2 >= Lc.nz) K2 = K;
        const float w0 = 0.75f, w1 = 0.25f;
        v = w0 * w0 * w0 * ec[sto(Lc, I, J, K)];
        v += w1 * w0 * w0 * ec[sto(Lc, I2, J, K)];
        v += w0 * w1 * w0 * ec[sto(Lc, I, J2, K)];
        v += w1 * w1 * w0 * ec[sto(Lc, I2, J2, K)];
        v += w0 * w0 * w1 * ec[sto(Lc, I, J, K2)];
        v += w1 * w0 * w1 * ec[sto(Lc, I2, J, K2)];
        v += w0 * w1 * w1 * ec[sto(Lc, I, J2, K2)];
        v += w1 * w1 * w1 * ec[sto(Lc, I2, J2, K2)];
    }
    xv[sto(L, x, y, z)] += v;
}

// e = pinv r on the coarsest level (FP64 accumulation), pinv in natural cell order
__global__ void k_coarse_matvec_lay(Lay L, const double *__restrict__ pinv, const float *__restrict__ r, float *e) {
    const int nc = (int)L.n;
    const int row = (int)(((i64)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= nc) return;
    const double *a = pinv + (i64)row * nc;
    double s = 0.0;
    for (int q = lane; q < nc; q += 32) {
        const int x = q % L.nx, y = (q / L.nx) % L.ny, z = q / (L.nx * L.ny);
        s += a[q] * (double)r[sto(L, x, y, z)];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        const int x = row % L.nx, y = (row / L.nx) % L.ny, z = row / (L.nx * L.ny);
        e[sto(L, x, y, z)] = (float)s;
    }
}

// natural <-> level storage
__global__ void k_pack(Lay L, const float *__restrict__ nat, float *st) {
    const i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L.n) return;
    const int x = (int)(t % L.nx);
    const i64 row = t / L.nx;
    st[sto(L, x, (int)(row % L.ny), (int)(row / L.ny))] = nat[t];
}
__global__ void k_unpack(Lay L, const float *__restrict__ st, float *nat) {
    const i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L.n) return;
    const int x = (int)(t % L.nx);
    const i64 row = t / L.nx;
    nat[t] = st[sto(L, x, (int)(row % L.ny), (int)(row / L.ny))];
}
// FP64 natural -> FP32 level storage, rounded to nearest; blocks take rows (grid y, strided)
__global__ void k_pack64(Lay L, const double *__restrict__ nat, float *st) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= L.nx) return;
    const i64 rows = (i64)L.ny * L.nz;
    for (i64 row = blockIdx.y; row < rows; row += gridDim.y) {
        const int y = (int)(row % L.ny), z = (int)(row / L.ny);
        st[sto(L, x, y, z)] = d2f_rn(nat[row * L.nx + x]);
    }
}
// s = 1/rho (FP64, natural): FP32 in the level's layout, and optionally as a pair (hi, lo) of
// FP32 numbers with hi + lo = s to about 2^-48 (natural layout) for the double-float residual
__global__ void k_pack_inv64(Lay L, const double *__restrict__ sinv, float *st, float2 *s2) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= L.nx) return;
    const i64 rows = (i64)L.ny * L.nz;
    for (i64 row = blockIdx.y; row < rows; row += gridDim.y) {
        const int y = (int)(row % L.ny), z = (int)(row / L.ny);
        const i64 t = row * L.nx + x;
        const double v = sinv[t];
        const float hi = d2f_rn(v);
        st[sto(L, x, y, z)] = hi;
        if (s2) s2[t] = make_float2(hi, d2f_rn(v - f2d_exact(hi)));
    }
}

}  // namespace

Lay make_lay(Dims d) {
    Lay L;
    L.nx = d.nx;
    L.ny = d.ny;
    L.nz = d.nz;
    L.n = d.n;
    L.split = (d.nx % 2 == 0);
    L.hx = d.nx / 2;
    L.half = d.n / 2;
    L.zlo = L.zhi = 0;
    return L;
}

// a slab (L.zlo / L.zhi): split layout with hx % 4 == 0 (the decomposed mixed cycle); s-form
// (the finest level) or face form (the face arrays with their ghost plane above)
template <bool SFORM>
void half32_slab(cudaStream_t s, const Lay &L, float h2, const Coef32 &cf, const float *b, float *x, int col,
                 bool from_zero) {
    if (half_z_ok(L)) {
        if (from_zero) run_half_z<SFORM, true, 0, true>(s, L, h2, cf, b, x, col, Upd{});
        else run_half_z<SFORM, false, 0, true>(s, L, h2, cf, b, x, col, Upd{});
        return;
    }
    const i64 work = (i64)L.ny * L.nz * (L.hx / 4);
    if (from_zero) k_half_vec<SFORM, true, 0, true><<<blocks_for(work), kThreads, 0, s>>>(L, h2, cf, b, x, col, Upd{});
    else k_half_vec<SFORM, false, 0, true><<<blocks_for(work), kThreads, 0, s>>>(L, h2, cf, b, x, col, Upd{});
}

void launch_half32_slab(cudaStream_t s, const Lay &L, float h2, const Coef32 &cf, const float *b, float *x, int col,
                        bool from_zero) {
    if (cf.s) half32_slab<true>(s, L, h2, cf, b, x, col, from_zero);
    else half32_slab<false>(s, L, h2, cf, b, x, col, from_zero);
}

void launch_half32(cudaStream_t s, Lay L, double h2, const float *sinv, const float *fx, const float *fy,
                   const float *fz, const float *b, float *x, int col, bool from_zero) {
    Coef32 cf{sinv, fx, fy, fz};
    count_launch();
    if (L.zlo || L.zhi) {
        launch_half32_slab(s, L, (float)h2, cf, b, x, col, from_zero);
        return;
    }
    if (half_z_ok(L)) {
        if (sinv) {
            if (from_zero) run_half_z<true, true, 0>(s, L, (float)h2, cf, b, x, col, Upd{});
            else run_half_z<true, false, 0>(s, L, (float)h2, cf, b, x, col, Upd{});
        } else {
            if (from_zero) run_half_z<false, true, 0>(s, L, (float)h2, cf, b, x, col, Upd{});
            else run_half_z<false, false, 0>(s, L, (float)h2, cf, b, x, col, Upd{});
        }
    } else if (L.split && L.hx % 4 == 0) {
        const i64 work = (i64)L.ny * L.nz * (L.hx / 4);
        if (sinv) {
            if (from_zero) k_half_vec<true, true><<<blocks_for(work), kThreads, 0, s>>>(L, (float)h2, cf, b, x, col);
            else k_half_vec<true, false><<<blocks_for(work), kThreads, 0, s>>>(L, (float)h2, cf, b, x, col);
        } else {
            if (from_zero) k_half_vec<false, true><<<blocks_for(work), kThreads, 0, s>>>(L, (float)h2, cf, b, x, col);
            else k_half_vec<false, false><<<blocks_for(work), kThreads, 0, s>>>(L, (float)h2, cf, b, x, col);
        }
    } else {
        const i64 work = (i64)L.ny * L.nz * ((L.nx + 1) / 2);
        k_half_any<<<blocks_for(work), kThreads, 0, s>>>(L, (float)h2, cf, b, x, col, from_zero ? 1 : 0);
    }
}

bool half32_update_ok(Lay L) { return L.split && L.hx % 4 == 0; }

void launch_half32_update(cudaStream_t s, Lay L, double h2, const float *sinv, const float *fx, const float *fy,
                          const float *fz, const float *b, const float *x, double *p, float2 *p2, double alpha,
                          double shift) {
    Coef32 cf{sinv, fx, fy, fz};
    Upd up{p, p2, (float)alpha, (float)shift};
    count_launch();
    const i64 work = (i64)L.ny * L.nz * (L.hx / 4);
    float *xv = const_cast<float *>(x);  // read only in the UPDATE variants
    if (L.zlo || L.zhi) {  // a slab: s-form, FP64 solution (the decomposed mixed cycle)
        if (half_z_ok(L)) run_half_z<true, false, 1, true>(s, L, (float)h2, cf, b, xv, 0, up);
        else k_half_vec<true, false, 1, true><<<blocks_for(work), kThreads, 0, s>>>(L, (float)h2, cf, b, xv, 0, up);
        return;
    }
    if (half_z_ok(L)) {
        if (p2) {
            if (sinv) run_half_z<true, false, 2>(s, L, (float)h2, cf, b, xv, 0, up);
            else run_half_z<false, false, 2>(s, L, (float)h2, cf, b, xv, 0, up);
        } else {
            if (sinv) run_half_z<true, false, 1>(s, L, (float)h2, cf, b, xv, 0, up);
            else run_half_z<false, false, 1>(s, L, (float)h2, cf, b, xv, 0, up);
        }
        return;
    }
    if (p2) {
        if (sinv) k_half_vec<true, false, 2><<<blocks_for(work), kThreads, 0, s>>>(L, (float)h2, cf, b, xv, 0, up);
        else k_half_vec<false, false, 2><<<blocks_for(work), kThreads, 0, s>>>(L, (float)h2, cf, b, xv, 0, up);
    } else {
        if (sinv) k_half_vec<true, false, 1><<<blocks_for(work), kThreads, 0, s>>>(L, (float)h2, cf, b, xv, 0, up);
        else k_half_vec<false, false, 1><<<blocks_for(work), kThreads, 0, s>>>(L, (float)h2, cf, b, xv, 0, up);
    }
}

void launch_residual32(cudaStream_t s, Lay L, double ih2, const float *sinv, const float *fx, const float *fy,
                       const float *fz, const float *b, const float *x, float *r, bool apply_only) {
    Coef32 cf{sinv, fx, fy, fz};
    count_launch();
    k_residual_any<<<blocks_for(L.n), kThreads, 0, s>>>(L, (float)ih2, cf, b, x, r, apply_only ? 1 : 0);
}

void launch_resid_restrict32(cudaStream_t s, Lay L, Lay Lc, double ih2, const float *sinv, const float *fx,
                             const float *fy, const float *fz, const float *b, const float *x, float *bc,
                             bool red_only) {
    Coef32 cf{sinv, fx, fy, fz};
    count_launch();
    if (red_only && L.split && L.hx % 4 == 0) {
        const i64 work = (i64)Lc.ny * Lc.nz * (L.hx / 4);
        const unsigned nb = (unsigned)((work + kRrThreads - 1) / kRrThreads);
        if ((L.zlo || L.zhi) && sinv) k_rr_red_vec<true, true><<<nb, kRrThreads, 0, s>>>(L, Lc, (float)ih2, cf, b, x, bc);
        else if (L.zlo || L.zhi) k_rr_red_vec<false, true><<<nb, kRrThreads, 0, s>>>(L, Lc, (float)ih2, cf, b, x, bc);
        else if (sinv) k_rr_red_vec<true><<<nb, kRrThreads, 0, s>>>(L, Lc, (float)ih2, cf, b, x, bc);
        else k_rr_red_vec<false><<<nb, kRrThreads, 0, s>>>(L, Lc, (float)ih2, cf, b, x, bc);
        return;
    }
    k_resid_restrict_any<<<blocks_for(Lc.n), kThreads, 0, s>>>(L, Lc, (float)ih2, cf, b, x, bc, red_only ? 1 : 0);
}

void launch_prolong32(cudaStream_t s, Lay L, Lay Lc, const float *ec, float *x, int kind, int only_col) {
    count_launch();
    if (only_col == 0 && kind == MG_PROLONG_TRILINEAR && L.split && Lc.split && Lc.nx % 8 == 0 &&
        2 * Lc.nx == L.nx && 2 * Lc.ny == L.ny && 2 * Lc.nz == L.nz) {
        const i64 work = (i64)Lc.ny * Lc.nz * (L.hx / 8);
        const unsigned nb = (unsigned)((work + kProlThreads - 1) / kProlThreads);
        if (Lc.zlo || Lc.zhi) k_prolong_red8<true><<<nb, kProlThreads, 0, s>>>(L, Lc, ec, x);
        else k_prolong_red8<<<nb, kProlThreads, 0, s>>>(L, Lc, ec, x);
        return;
    }
    if (only_col == 0 && L.split && L.hx % 4 == 0) {
        const i64 work = (i64)L.ny * L.nz * (L.hx / 4);
        k_prolong_red_vec<<<blocks_for(work), kThreads, 0, s>>>(L, Lc, ec, x, kind);
        return;
    }
    k_prolong_any<<<blocks_for(L.n), kThreads, 0, s>>>(L, Lc, ec, x, kind, only_col);
}

void launch_coarse_matvec32(cudaStream_t s, Lay L, const double *pinv, const float *r, float *e) {
    count_launch();
    k_coarse_matvec_lay<<<blocks_for(L.n * 32), kThreads, 0, s>>>(L, pinv, r, e);
}

void launch_pack32(cudaStream_t s, Lay L, const float *nat, float *st) {
    count_launch();
    k_pack<<<blocks_for(L.n), kThreads, 0, s>>>(L, nat, st);
}
void launch_unpack32(cudaStream_t s, Lay L, const float *st, float *nat) {
    count_launch();
    k_unpack<<<blocks_for(L.n), kThreads, 0, s>>>(L, st, nat);
}
void launch_pack64to32(cudaStream_t s, Lay L, const double *nat, float *st) {
    count_launch();
    const i64 rows = (i64)L.ny * L.nz;
    const dim3 grd((unsigned)((L.nx + 127) / 128), (unsigned)(rows < 65535 ? rows : 65535));
    k_pack64<<<grd, 128, 0, s>>>(L, nat, st);
}
void launch_pack_inv_rho(cudaStream_t s, Lay L, const double *sinv, float *st, float2 *s2) {
    count_launch();
    const i64 rows = (i64)L.ny * L.nz;
    const dim3 grd((unsigned)((L.nx + 127) / 128), (unsigned)(rows < 65535 ? rows : 65535));
    k_pack_inv64<<<grd, 128, 0, s>>>(L, sinv, st, s2);
}

}  // namespace mg
