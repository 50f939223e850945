// Fine-level FP64 passes and deterministic reductions: RHS mean and norm,
// the FP64 residual of the outer loop (with its norm, the mean of p and the
// scaled FP32 copy that feeds the inner V-cycle), the solution update, and the
// fused adjoint gradient kernel.
//
// Every reduction runs on a grid whose size depends only on n and the device
// model (one wave of resident blocks at most); each block writes one partial
// (warp shuffles in a fixed pattern), and one block sums the partials in index
// order, so results are bitwise reproducible for the same inputs and device.
#include <cmath>

#include "mg_internal.cuh"

namespace mg {

static unsigned long long g_launches = 0;

void count_launch(int k) { __atomic_fetch_add(&g_launches, (unsigned long long)k, __ATOMIC_RELAXED); }

unsigned long long launches_total() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

int reduce_blocks(i64 n) {
    i64 b = (n + kReduceThreads - 1) / kReduceThreads;
    const i64 cap = 152 * 8;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

int wave_blocks(const void *kernel, int threads) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess ||
        sms < 1 || per_sm < 1) {
        (void)cudaGetLastError();  // the query failed before any launch: keep the full count
        return 1 << 30;
    }
    return sms * per_sm;
}

int fill_blocks(int nb, int wave) {
    // a grid-stride loop over nb > wave blocks runs as one full wave and a partly filled one;
    // with exactly one wave every block does the same share of the work
    return nb > wave ? wave : nb;
}

namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(i64 n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// reduce (a, b) over the block; thread 0 writes them to out[0], out[1]
__device__ __forceinline__ void block_sum2(double a, double b, double *out) {
    __shared__ double sa[32], sb[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sa[warp] = a;
        sb[warp] = b;
    }
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        a = lane < nw ? sa[lane] : 0.0;
        b = lane < nw ? sb[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (lane == 0) {
            out[0] = a;
            out[1] = b;
        }
    }
}

__global__ void k_final(const double *__restrict__ partials, int nb, double *out) {
    double a = 0.0, b = 0.0;
    for (int q = threadIdx.x; q < nb; q += blockDim.x) {
        a += partials[2 * q];
        b += partials[2 * q + 1];
    }
    block_sum2(a, b, out);
}

template <typename T> struct Vec16;
template <> struct Vec16<double> {
    using type = double2;
    static constexpr int n = 2;
    __device__ static void get(const double2 &u, double (&v)[4]) { v[0] = u.x; v[1] = u.y; v[2] = v[3] = 0.0; }
};
template <> struct Vec16<float> {
    using type = float4;
    static constexpr int n = 4;
    __device__ static void get(const float4 &u, double (&v)[4]) { v[0] = u.x; v[1] = u.y; v[2] = u.z; v[3] = u.w; }
};

inline __device__ bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// sums of x and, with SQ, of x^2.  A single 8-byte load in flight per thread leaves HBM at
// about a third of its bandwidth, so a 16-byte-aligned x is read as two 16-byte loads per
// thread and iteration; the elements past the last whole vector (and an unaligned x) take the
// scalar loop.  GB300 issues FP64 additions at a small fraction of its FP32 rate, so the
// gauge sums, which need no squares, take one FP64 addition per element instead of two.
template <typename T, bool SQ>
__global__ void k_sum_sumsq(i64 n, const T *__restrict__ x, double *partials) {
    using V = Vec16<T>;
    double a = 0.0, b = 0.0;
    const i64 tid = (i64)blockIdx.x * blockDim.x + threadIdx.x, nt = (i64)gridDim.x * blockDim.x;
    i64 m0 = 0;
    if (aligned16(x)) {
        const typename V::type *xv = reinterpret_cast<const typename V::type *>(x);
        const i64 nv = n / V::n;
        for (i64 m = tid; m < nv; m += 2 * nt) {
            const typename V::type u0 = xv[m];
            const bool two = m + nt < nv;
            typename V::type u1 = u0;
            if (two) u1 = xv[m + nt];
            double v[4];
            V::get(u0, v);
#pragma unroll
            for (int q = 0; q < V::n; ++q) {
                a += v[q];
                if (SQ) b += v[q] * v[q];
            }
            if (two) {
                V::get(u1, v);
#pragma unroll
                for (int q = 0; q < V::n; ++q) {
                    a += v[q];
                    if (SQ) b += v[q] * v[q];
                }
            }
        }
        m0 = nv * V::n;
    }
    for (i64 m = m0 + tid; m < n; m += nt) {
        double v = (double)x[m];
        a += v;
        if (SQ) b += v * v;
    }
    block_sum2(a, b, partials + 2 * blockIdx.x);
}

// v * 2^m by an integer addition to the IEEE-754 exponent field (binary64: 11 exponent bits
// from bit 52) when v is normal and stays normal, exact like the multiplication; otherwise
// (zero, subnormal, a result leaving the normal range, infinity, NaN) v * s, in a function of
// its own so that the compiler keeps it off the common path.
__device__ __noinline__ double mul_slow(double v, double s) { return v * s; }
__device__ __forceinline__ double mul_pow2(double v, int m, double s) {
    const long long bits = __double_as_longlong(v);
    const int e = (int)((bits >> 52) & 0x7ff);
    if (e >= 1 && e <= 2046 && e + m >= 1 && e + m <= 2046) return __longlong_as_double(bits + ((long long)m << 52));
    return mul_slow(v, s);
}

// b64 = (b - mean(b)) * scale; partials: sum of b64^2.  16-byte loads and stores, two per
// thread and iteration, where b and b64 are 16-byte aligned (as k_sum_sumsq).  With POW2
// (scale = 2^m: 1 in the FP64 mode, h^2 in the mixed modes when h is a power of two) the
// scaling is an exponent addition: two FP64 operations per element instead of three.
template <bool POW2>
__global__ void k_sub_mean(i64 n, const double *__restrict__ b, const double *__restrict__ sum,
                           double scale, int m2, double *b64, double *partials) {
    const double mean = sum[0] / (double)n;
    double q = 0.0;
    auto f = [&](double u) { return POW2 ? mul_pow2(u - mean, m2, scale) : (u - mean) * scale; };
    const i64 tid = (i64)blockIdx.x * blockDim.x + threadIdx.x, nt = (i64)gridDim.x * blockDim.x;
    i64 m0 = 0;
    if (aligned16(b) && aligned16(b64)) {
        const double2 *bv = reinterpret_cast<const double2 *>(b);
        double2 *ov = reinterpret_cast<double2 *>(b64);
        const i64 nv = n / 2;
        for (i64 m = tid; m < nv; m += 2 * nt) {
            const double2 u0 = bv[m];
            const bool two = m + nt < nv;
            double2 u1 = u0;
            if (two) u1 = bv[m + nt];
            const double2 w0 = make_double2(f(u0.x), f(u0.y));
            ov[m] = w0;
            q += w0.x * w0.x;
            q += w0.y * w0.y;
            if (two) {
                const double2 w1 = make_double2(f(u1.x), f(u1.y));
                ov[m + nt] = w1;
                q += w1.x * w1.x;
                q += w1.y * w1.y;
            }
        }
        m0 = nv * 2;
    }
    for (i64 m = m0 + tid; m < n; m += nt) {
        const double v = f(b[m]);
        b64[m] = v;
        q += v * v;
    }
    block_sum2(q, 0.0, partials + 2 * blockIdx.x);
}

__device__ __forceinline__ i64 sto(const Lay &L, int x, int y, int z) {
    const i64 row = (i64)z * L.ny + y;
    if (!L.split) return row * L.nx + x;
    return ((x + y + z) & 1) * L.half + row * L.hx + (x >> 1);
}

// h^2 r = h^2 b - (d p_c - sum_f beta_f p_nb), d = sum_f beta_f: 7 FP64 fused multiply-adds
// per cell when b arrives already scaled by h^2 (SCALED), one more multiply otherwise.
// partials: (sum (h^2 r)^2 and sum p, each accumulated in FP32 per thread); r32 = s32 * h^2 r.
// The FP32 sum of p only steers the per-iteration gauge shift; the exit gauge is exact.
// One thread handles the cell pair x = 2k, 2k+1 of a row (even nx): aligned double2 loads,
// and the pair's red and black r32 values land at index k of the two colour halves.
template <bool SCALED>
__global__ void k_fine_resid_pair(Dims d, Lay L, double h2, const double *__restrict__ fx,
                                  const double *__restrict__ fy, const double *__restrict__ fz,
                                  const double *__restrict__ dg, const double *__restrict__ b,
                                  const double *__restrict__ p, float *r32, float s32, double *partials) {
    float q = 0.f, sp = 0.f;
    const int nx = d.nx, ny = d.ny, nz = d.nz, hx = nx >> 1;
    const int nxy = nx * ny;
    const int npairs = (int)(d.n >> 1);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < npairs; t += gridDim.x * blockDim.x) {
        const int row = t / hx, k = t - row * hx;
        const int j = row % ny, z = row / ny;
        const int c = row * nx + 2 * k;  // cells c (x = 2k) and c + 1
        const double2 pc = *reinterpret_cast<const double2 *>(p + c);
        const double2 bb = *reinterpret_cast<const double2 *>(b + c);
        const double2 fxa = *reinterpret_cast<const double2 *>(fx + c);   // low x faces of both cells
        const double2 fya = *reinterpret_cast<const double2 *>(fy + c);
        const double2 fza = *reinterpret_cast<const double2 *>(fz + c);
        const double2 dd = *reinterpret_cast<const double2 *>(dg + c);
        double a0 = SCALED ? bb.x : h2 * bb.x;
        double a1 = SCALED ? bb.y : h2 * bb.y;
        // x faces: cell 0 low (x-1), shared face (between the pair), cell 1 high (x+2)
        if (k > 0) a0 = fma(fxa.x, p[c - 1], a0);
        a0 = fma(fxa.y, pc.y, a0);
        a1 = fma(fxa.y, pc.x, a1);
        if (k < hx - 1) a1 = fma(fx[c + 2], p[c + 2], a1);
        if (j > 0) {
            const double2 pm = *reinterpret_cast<const double2 *>(p + c - nx);
            a0 = fma(fya.x, pm.x, a0);
            a1 = fma(fya.y, pm.y, a1);
        }
        if (j < ny - 1) {
            const double2 f = *reinterpret_cast<const double2 *>(fy + c + nx);
            const double2 pp = *reinterpret_cast<const double2 *>(p + c + nx);
            a0 = fma(f.x, pp.x, a0);
            a1 = fma(f.y, pp.y, a1);
        }
        if (z > 0) {
            const double2 pm = *reinterpret_cast<const double2 *>(p + c - nxy);
            a0 = fma(fza.x, pm.x, a0);
            a1 = fma(fza.y, pm.y, a1);
        }
        if (z < nz - 1) {
            const double2 f = *reinterpret_cast<const double2 *>(fz + c + nxy);
            const double2 pp = *reinterpret_cast<const double2 *>(p + c + nxy);
            a0 = fma(f.x, pp.x, a0);
            a1 = fma(f.y, pp.y, a1);
        }
        a0 = fma(-dd.x, pc.x, a0);
        a1 = fma(-dd.y, pc.y, a1);
        const float r0 = d2f_trunc(a0), r1 = d2f_trunc(a1);
        if (r32) {
            const int par = (j + z) & 1;  // colour of cell x = 2k
            const i64 base = (i64)row * hx + k;
            r32[par * L.half + base] = r0 * s32;
            r32[(1 - par) * L.half + base] = r1 * s32;
        }
        q = fmaf(r0, r0, q);
        q = fmaf(r1, r1, q);
        sp += d2f_trunc(pc.x) + d2f_trunc(pc.y);
    }
    block_sum2((double)q, (double)sp, partials + 2 * blockIdx.x);
}

// the same residual, one thread per cell (any nx; used when nx is odd)
template <bool SCALED>
__global__ void k_fine_resid_cell(Dims d, Lay L, double h2, const double *__restrict__ fx,
                                  const double *__restrict__ fy, const double *__restrict__ fz,
                                  const double *__restrict__ dg, const double *__restrict__ b,
                                  const double *__restrict__ p, float *r32, float s32, double *partials) {
    float q = 0.f, sp = 0.f;
    const int nx = d.nx, ny = d.ny, nz = d.nz;
    const i64 nxy = d.nxy;
    for (i64 c = (i64)blockIdx.x * blockDim.x + threadIdx.x; c < d.n; c += (i64)gridDim.x * blockDim.x) {
        const int i = (int)(c % nx);
        const i64 row = c / nx;
        const int j = (int)(row % ny), k = (int)(row / ny);
        const double pc = p[c];
        double acc = SCALED ? b[c] : h2 * b[c];
        if (i > 0) acc = fma(fx[c], p[c - 1], acc);
        if (i < nx - 1) acc = fma(fx[c + 1], p[c + 1], acc);
        if (j > 0) acc = fma(fy[c], p[c - nx], acc);
        if (j < ny - 1) acc = fma(fy[c + nx], p[c + nx], acc);
        if (k > 0) acc = fma(fz[c], p[c - nxy], acc);
        if (k < nz - 1) acc = fma(fz[c + nxy], p[c + nxy], acc);
        acc = fma(-dg[c], pc, acc);
        const float rf = d2f_trunc(acc);
        if (r32) r32[sto(L, i, j, k)] = rf * s32;
        q = fmaf(rf, rf, q);
        sp += d2f_trunc(pc);
    }
    block_sum2((double)q, (double)sp, partials + 2 * blockIdx.x);
}

// r = b - ih2 * sum_f beta_f (p_c - p_nb); partials: (sum r^2, sum p)
__global__ void k_fine_residual(Dims d, Lay L, double ih2, const double *__restrict__ fx,
                                const double *__restrict__ fy, const double *__restrict__ fz,
                                const double *__restrict__ b, const double *__restrict__ p,
                                float *r32, double scale, double *partials) {
    double q = 0.0, sp = 0.0;
    for (i64 c = (i64)blockIdx.x * blockDim.x + threadIdx.x; c < d.n; c += (i64)gridDim.x * blockDim.x) {
        int i = (int)(c % d.nx);
        i64 row = c / d.nx;
        int j = (int)(row % d.ny), k = (int)(row / d.ny);
        double pc = p[c];
        double s = 0.0;
        if (i > 0) s += fx[c] * (pc - p[c - 1]);
        if (i < d.nx - 1) s += fx[c + 1] * (pc - p[c + 1]);
        if (j > 0) s += fy[c] * (pc - p[c - d.nx]);
        if (j < d.ny - 1) s += fy[c + d.nx] * (pc - p[c + d.nx]);
        if (k > 0) s += fz[c] * (pc - p[c - d.nxy]);
        if (k < d.nz - 1) s += fz[c + d.nxy] * (pc - p[c + d.nxy]);
        double r = b[c] - s * ih2;
        if (r32) r32[sto(L, i, j, k)] = (float)(r * scale);
        q += r * r;
        sp += pc;
    }
    block_sum2(q, sp, partials + 2 * blockIdx.x);
}

// p = (p - shift) + alpha e: 2 FP64 operations, the FP32 value widened exactly with integer operations
__global__ void k_update(Dims d, Lay L, double *p, const float *__restrict__ e, float alpha, float shift) {
    const i64 m = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= d.n) return;
    const int i = (int)(m % d.nx);
    const i64 row = m / d.nx;
    // the correction alpha e - shift is formed in FP32 (e is an FP32 V-cycle result; the outer
    // loop corrects its rounding), the update itself is one FP64 addition
    const float c = fmaf(alpha, e[sto(L, i, (int)(row % d.ny), (int)(row / d.ny))], -shift);
    p[m] += f2d_exact(c);
}

// n (<= 32) doubles from src, and with esrc one unsigned, into mapped pinned host memory
__global__ void k_readback(const double *__restrict__ src, double *dst, int n, const unsigned *esrc,
                           unsigned *edst) {
    const int t = threadIdx.x;
    if (t < n) dst[t] = src[t];
    if (t == 0 && esrc) *edst = *esrc;
}

__global__ void k_add_const(i64 n, double *p, double c) {
    i64 m = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (m < n) p[m] += c;
}

// dL/dbeta_f = -(lam_L - lam_R)(p_L - p_R) ih2 + sigma csf_f (lam_L - lam_R) ih on the low
// faces of each cell (walls 0); partial sums of beta_f csf_f (lam_L - lam_R) ih (= dL/dsigma,
// one FP64 multiplication and one FMA per face, the factor ih applied once per block).
// Blocks take whole rows (no 64-bit division per cell).  The differences of lambda and p are
// formed in FP64 (they cancel); their product, an FP32 output, is formed in FP32 from the
// differences rounded to nearest.  dL/dsigma is summed in FP64.
__global__ void k_adjoint_grad(Dims d, float ih, float ih2, double ihd, const double *__restrict__ lam,
                               const double *__restrict__ p, const double *__restrict__ fx,
                               const double *__restrict__ fy, const double *__restrict__ fz,
                               const double *__restrict__ csx, const double *__restrict__ csy,
                               const double *__restrict__ csz, float sigma, float *gx, float *gy,
                               float *gz, double *partials) {
    double ds = 0.0;
    const int nx = d.nx, ny = d.ny;
    const i64 nxy = d.nxy, rows = (i64)ny * d.nz;
    for (i64 row = blockIdx.x; row < rows; row += gridDim.x) {
        // rows = ny * nz < 2^31: 32-bit division (a 64-bit one costs several times as many
        // instructions per row)
        const int r32 = (int)row, j = r32 % ny, k = r32 / ny;
        const i64 c0 = row * nx;
        const i64 ax0 = row * (nx + 1);                        // x faces: (nz, ny, nx + 1)
        const i64 ay0 = ((i64)k * (ny + 1) + j) * nx;          // y faces: (nz, ny + 1, nx)
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const i64 c = c0 + i;
            const double lc = lam[c], pc = p[c];
            float g0 = 0.f, g1 = 0.f, g2 = 0.f;
            if (i > 0) {
                const double dl = lam[c - 1] - lc;
                const float dlf = d2f_rn(dl);
                g0 = -dlf * d2f_rn(p[c - 1] - pc) * ih2;
                if (csx) {
                    g0 = fmaf(sigma * d2f_rn(csx[ax0 + i]) * ih, dlf, g0);
                    ds = fma(fx[c] * csx[ax0 + i], dl, ds);
                }
            }
            if (j > 0) {
                const double dl = lam[c - nx] - lc;
                const float dlf = d2f_rn(dl);
                g1 = -dlf * d2f_rn(p[c - nx] - pc) * ih2;
                if (csy) {
                    g1 = fmaf(sigma * d2f_rn(csy[ay0 + i]) * ih, dlf, g1);
                    ds = fma(fy[c] * csy[ay0 + i], dl, ds);
                }
            }
            if (k > 0) {
                const double dl = lam[c - nxy] - lc;
                const float dlf = d2f_rn(dl);
                g2 = -dlf * d2f_rn(p[c - nxy] - pc) * ih2;
                if (csz) {
                    g2 = fmaf(sigma * d2f_rn(csz[c]) * ih, dlf, g2);
                    ds = fma(fz[c] * csz[c], dl, ds);
                }
            }
            if (gx) {
                gx[ax0 + i] = g0;
                gy[ay0 + i] = g1;
                gz[c] = g2;
                if (i == nx - 1) gx[ax0 + nx] = 0.f;
                if (j == ny - 1) gy[ay0 + i + nx] = 0.f;
                if (k == d.nz - 1) gz[c + nxy] = 0.f;
            }
        }
    }
    block_sum2(ds * ihd, 0.0, partials + 2 * blockIdx.x);
}

}  // namespace

template <typename T>
void launch_sum_sumsq(cudaStream_t s, i64 n, const T *x, double *partials, double *out, bool squares) {
    static const int wave_q = wave_blocks((const void *)k_sum_sumsq<T, true>, kReduceThreads);
    static const int wave_s = wave_blocks((const void *)k_sum_sumsq<T, false>, kReduceThreads);
    const int nb = fill_blocks(reduce_blocks(n), squares ? wave_q : wave_s);
    count_launch();
    if (squares) k_sum_sumsq<T, true><<<nb, kReduceThreads, 0, s>>>(n, x, partials);
    else k_sum_sumsq<T, false><<<nb, kReduceThreads, 0, s>>>(n, x, partials);
    count_launch();
    k_final<<<1, kReduceThreads, 0, s>>>(partials, nb, out);
}
template void launch_sum_sumsq<double>(cudaStream_t, i64, const double *, double *, double *, bool);
template void launch_sum_sumsq<float>(cudaStream_t, i64, const float *, double *, double *, bool);

void launch_sub_mean(cudaStream_t s, i64 n, const double *b, const double *sum, double scale, double *b64,
                     double *partials, double *out) {
    static const int wave_p = wave_blocks((const void *)k_sub_mean<true>, kReduceThreads);
    static const int wave_m = wave_blocks((const void *)k_sub_mean<false>, kReduceThreads);
    int e = 0;
    const bool pow2 = std::frexp(scale, &e) == 0.5;  // scale = 2^(e - 1)
    const int nb = fill_blocks(reduce_blocks(n), pow2 ? wave_p : wave_m);
    count_launch();
    if (pow2) k_sub_mean<true><<<nb, kReduceThreads, 0, s>>>(n, b, sum, scale, e - 1, b64, partials);
    else k_sub_mean<false><<<nb, kReduceThreads, 0, s>>>(n, b, sum, scale, 0, b64, partials);
    count_launch();
    k_final<<<1, kReduceThreads, 0, s>>>(partials, nb, out);
}

void launch_fine_residual(cudaStream_t s, Dims d, Lay L, double ih2, const double *fx, const double *fy,
                          const double *fz, const double *b, const double *p, float *r32,
                          double scale, double *partials, double *out) {
    static const int wave = wave_blocks((const void *)k_fine_residual, kReduceThreads);
    const int nb = fill_blocks(reduce_blocks(d.n), wave);
    count_launch();
    k_fine_residual<<<nb, kReduceThreads, 0, s>>>(d, L, ih2, fx, fy, fz, b, p, r32, scale, partials);
    count_launch();
    k_final<<<1, kReduceThreads, 0, s>>>(partials, nb, out);
}

void launch_fine_resid2(cudaStream_t s, Dims d, Lay L, double h2, const double *fx, const double *fy,
                        const double *fz, const double *diag, const double *b, bool b_scaled, const double *p,
                        float *r32, float s32, double *partials, double *out) {
    if (d.nx & 1) {
        static const int wave_ct = wave_blocks((const void *)k_fine_resid_cell<true>, kReduceThreads);
        static const int wave_cf = wave_blocks((const void *)k_fine_resid_cell<false>, kReduceThreads);
        const int nb = fill_blocks(reduce_blocks(d.n), b_scaled ? wave_ct : wave_cf);
        count_launch();
        if (b_scaled) k_fine_resid_cell<true><<<nb, kReduceThreads, 0, s>>>(d, L, h2, fx, fy, fz, diag, b, p, r32, s32, partials);
        else k_fine_resid_cell<false><<<nb, kReduceThreads, 0, s>>>(d, L, h2, fx, fy, fz, diag, b, p, r32, s32, partials);
        count_launch();
        k_final<<<1, kReduceThreads, 0, s>>>(partials, nb, out);
        return;
    }
    static const int wave_pt = wave_blocks((const void *)k_fine_resid_pair<true>, kReduceThreads);
    static const int wave_pf = wave_blocks((const void *)k_fine_resid_pair<false>, kReduceThreads);
    const int nb = fill_blocks(reduce_blocks(d.n / 2), b_scaled ? wave_pt : wave_pf);
    count_launch();
    if (b_scaled) k_fine_resid_pair<true><<<nb, kReduceThreads, 0, s>>>(d, L, h2, fx, fy, fz, diag, b, p, r32, s32, partials);
    else k_fine_resid_pair<false><<<nb, kReduceThreads, 0, s>>>(d, L, h2, fx, fy, fz, diag, b, p, r32, s32, partials);
    count_launch();
    k_final<<<1, kReduceThreads, 0, s>>>(partials, nb, out);
}

void launch_update(cudaStream_t s, Dims d, Lay L, double *p, const float *e32, double alpha, double shift) {
    count_launch();
    k_update<<<blocks_for(d.n), kThreads, 0, s>>>(d, L, p, e32, (float)alpha, (float)shift);
}

void launch_readback(cudaStream_t s, const double *src, double *dst_mapped, int n) {
    count_launch();
    k_readback<<<1, 32, 0, s>>>(src, dst_mapped, n, nullptr, nullptr);
}

void launch_readback_u32(cudaStream_t s, const unsigned *src, unsigned *dst_mapped) {
    count_launch();
    k_readback<<<1, 32, 0, s>>>(nullptr, nullptr, 0, src, dst_mapped);
}

void launch_add_const(cudaStream_t s, i64 n, double *p, double c) {
    count_launch();
    k_add_const<<<blocks_for(n), kThreads, 0, s>>>(n, p, c);
}

void launch_adjoint_grad(cudaStream_t s, Dims d, double h, const double *lam, const double *p,
                         const double *fx, const double *fy, const double *fz, const double *csfx,
                         const double *csfy, const double *csfz, double sigma, float *gx,
                         float *gy, float *gz, double *partials, double *out) {
    static const int wave = wave_blocks((const void *)k_adjoint_grad, kReduceThreads);
    int nb = fill_blocks(reduce_blocks(d.n), wave);
    count_launch();
    const i64 rows = (i64)d.ny * d.nz;
    if (nb > rows) nb = (int)rows;
    k_adjoint_grad<<<nb, kReduceThreads, 0, s>>>(d, (float)(1.0 / h), (float)(1.0 / (h * h)), 1.0 / h, lam, p,
                                                 fx, fy, fz, csfx, csfy, csfz, (float)sigma, gx, gy, gz,
                                                 partials);
    count_launch();
    k_final<<<1, kReduceThreads, 0, s>>>(partials, nb, out);
}

}  // namespace mg
