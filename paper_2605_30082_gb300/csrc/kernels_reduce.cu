// Fine-level FP64 passes and deterministic reductions: RHS mean and norm,
// the FP64 residual of the outer loop (with its norm, the mean of p and the
// scaled FP32 copy that feeds the inner V-cycle), the solution update, and the
// fused adjoint gradient kernel.
//
// Every reduction runs on a grid whose size depends only on n and the device
// model (one wave of resident blocks at most); each block writes one partial
// (warp shuffles in a fixed pattern), and one block sums the partials in index
// order, so results are bitwise reproducible for the same inputs and device.
#include <atomic>
#include <cmath>

#include <nvtx3/nvToolsExt.h>

#include "mg_internal.cuh"

namespace mg {

static unsigned long long g_launches = 0;

void count_launch(int k) { __atomic_fetch_add(&g_launches, (unsigned long long)k, __ATOMIC_RELAXED); }

NvtxRange::NvtxRange(const char *name) { nvtxRangePushA(name); }
NvtxRange::~NvtxRange() { nvtxRangePop(); }

unsigned long long launches_total() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

int device_sms() {
    constexpr int kMaxDev = 64;
    static std::atomic<int> cache[kMaxDev];
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
        (void)cudaGetLastError();
        dev = -1;
    }
    if (dev >= 0 && dev < kMaxDev && (v = cache[dev].load(std::memory_order_relaxed)) > 0) return v;
    if (dev < 0 || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
        (void)cudaGetLastError();
        return 152;  // the query failed: size for GB300 (grid sizes only; results do not depend on it)
    }
    if (dev < kMaxDev) cache[dev].store(v, std::memory_order_relaxed);
    return v;
}

int reduce_blocks(i64 n) {
    i64 b = (n + kReduceThreads - 1) / kReduceThreads;
    const i64 cap = (i64)device_sms() * 8;
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
// GHOST: a slab of a decomposed grid (d.zlo / d.zhi): its ghost planes count as interior
// neighbours; whole-grid levels compile without the two extra tests
template <bool SCALED, bool GHOST>
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
        if (z > 0 || (GHOST && d.zlo)) {
            const double2 pm = *reinterpret_cast<const double2 *>(p + c - nxy);
            a0 = fma(fza.x, pm.x, a0);
            a1 = fma(fza.y, pm.y, a1);
        }
        if (z < nz - 1 || (GHOST && d.zhi)) {
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

// r32 = s32 * (the residual of p = 0) in the level layout, rounded as the residual kernels round
// theirs: the residual of p = 0 is h^2 b~ itself, truncated to FP32, times s32.  A cold-started
// solve takes its first inner right-hand side from here instead of an FP64 residual pass.
__global__ void k_zero_resid32(Dims d, Lay L, const double *__restrict__ b, float s32, float *r32) {
    const i64 c = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.n) return;
    const unsigned cu = (unsigned)c, r = cu / (unsigned)d.nx;  // c < 2^32: 32-bit divisions
    const int i = (int)(cu - r * (unsigned)d.nx), j = (int)(r % (unsigned)d.ny), k = (int)(r / (unsigned)d.ny);
    r32[sto(L, i, j, k)] = d2f_trunc(b[c]) * s32;
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
        if (k > 0 || d.zlo) acc = fma(fz[c], p[c - nxy], acc);  // a slab's ghost planes count as interior
        if (k < nz - 1 || d.zhi) acc = fma(fz[c + nxy], p[c + nxy], acc);
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

// ---- fused gradient without a surface term: no FP64 arithmetic -------------------------
// A double v is split into two floats v ~ hi + lo with integer operations on its IEEE-754
// fields: hi keeps the sign, exponent and top 23 fraction bits (truncation), lo the value of
// the 29 bits dropped, taken to 23 of them (the low 6 are truncated: |v - hi - lo| <= 2^-46 |v|).
// lo is formed exactly as the difference of two floats with the same exponent 2^E (E = e - 1046
// for the double's biased exponent e): (2^E with the dropped bits as its fraction) - 2^E.
// A difference of two doubles is then (hi_a - hi_b) + (lo_a - lo_b) in FP32: the first term is
// exact when a and b are within a factor of two (the cancelling case), otherwise rounded once;
// the result is within about one FP32 unit of the exact difference plus an absolute 2^-45
// max(|a|, |b|) (the pair holds 47 bits of the 53).  For the FP32 face gradients that is far
// below their own rounding wherever a - b is not itself within 2^-20 of a's magnitude.
// |v| below 2^-126 gives 0 (an absolute error under 2^-126); |v| >= 2^128, infinity and NaN
// give hi = +-inf, so that a non-finite input still gives a non-finite gradient.
__device__ __forceinline__ void split_f64(double v, float &hi, float &lo) {
    // branch-free: the FP32 exponent of v is (e - 896) mod 256 = (e & 0xff) ^ 0x80 for the
    // biased FP64 exponent e in [897, 1150]; outside that range selects give 0 or +-inf/NaN
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const unsigned h32 = (unsigned)(u >> 32), l32 = (unsigned)u;
    const unsigned e = (h32 >> 20) & 0x7ffu;
    const unsigned sign = h32 & 0x80000000u;
    unsigned hb = (((h32 << 3) & 0x7ffffff8u) ^ 0x40000000u) | sign | (l32 >> 29);
    if (e - 897u > 253u) hb = e < 897u ? sign : (sign | 0x7f800000u);  // 0, or +-inf (also for NaN)
    hi = __uint_as_float(hb);
    // lo: 2^E with the dropped bits as its fraction, minus 2^E, E = hi's exponent - 23 (e >= 920)
    const unsigned base = (hb & 0xff800000u) - 0x0b800000u;
    const float l = __uint_as_float(base | ((l32 >> 6) & 0x7fffffu)) - __uint_as_float(base);
    lo = (e - 920u <= 230u) ? l : 0.f;
}

// dL/dbeta_f = -(lam_L - lam_R)(p_L - p_R)/h^2 on every interior face, FP32, with the
// differences formed from split_f64 pairs.  Block (32, kGradRows): a warp covers 32 cells of a
// row and marches kGradPlanes planes in z, keeping the previous plane's pairs in registers (the
// z face), taking the x-1 pair from the neighbouring lane (lane 0 loads it) and loading the
// y-1 row (split again; that row was just read by the warp above, so it comes from cache).
constexpr int kGradRows = 8, kGradPlanes = 32;

__global__ void __launch_bounds__(32 * kGradRows) k_adjoint_grad_split(
    int nx, int ny, int nz, float ih2, const double *__restrict__ lam, const double *__restrict__ p,
    float *__restrict__ gx, float *__restrict__ gy, float *__restrict__ gz) {
    const int lane = threadIdx.x;
    const int x = blockIdx.x * 32 + lane;
    const int y = blockIdx.y * kGradRows + threadIdx.y;
    const int z0 = blockIdx.z * kGradPlanes;
    const int z1 = min(z0 + kGradPlanes, nz);
    const bool act = x < nx && y < ny;
    const int nxy = nx * ny;  // < 2^31 (checked by the launcher with nx * ny * (nz + 1))
    float lzh = 0.f, lzl = 0.f, pzh = 0.f, pzl = 0.f;  // plane z - 1
    if (act && z0 > 0) {
        const int c = (z0 - 1) * nxy + y * nx + x;
        split_f64(lam[c], lzh, lzl);
        split_f64(p[c], pzh, pzl);
    }
    for (int z = z0; z < z1; ++z) {
        const int c = z * nxy + y * nx + x;
        float lh = 0.f, ll = 0.f, ph = 0.f, pl = 0.f;
        double lyd = 0.0, pyd = 0.0;
        if (act) {
            const double lc = lam[c], pc = p[c];
            if (y > 0) {
                lyd = lam[c - nx];
                pyd = p[c - nx];
            }
            split_f64(lc, lh, ll);
            split_f64(pc, ph, pl);
        }
        // x - 1 pair from the lane to the left (every lane takes part in the shuffles)
        float lxh = __shfl_up_sync(0xffffffffu, lh, 1), lxl = __shfl_up_sync(0xffffffffu, ll, 1);
        float pxh = __shfl_up_sync(0xffffffffu, ph, 1), pxl = __shfl_up_sync(0xffffffffu, pl, 1);
        if (act) {
            if (lane == 0 && x > 0) {
                split_f64(lam[c - 1], lxh, lxl);
                split_f64(p[c - 1], pxh, pxl);
            }
            float g0 = 0.f, g1 = 0.f, g2 = 0.f;
            if (x > 0) g0 = -((lxh - lh) + (lxl - ll)) * (((pxh - ph) + (pxl - pl)) * ih2);
            if (y > 0) {
                float lyh, lyl, pyh, pyl;
                split_f64(lyd, lyh, lyl);
                split_f64(pyd, pyh, pyl);
                g1 = -((lyh - lh) + (lyl - ll)) * (((pyh - ph) + (pyl - pl)) * ih2);
            }
            if (z > 0) g2 = -((lzh - lh) + (lzl - ll)) * (((pzh - ph) + (pzl - pl)) * ih2);
            const int row = z * ny + y;
            const int ax = row * (nx + 1) + x;          // x faces: (nz, ny, nx + 1)
            const int ay = (z * (ny + 1) + y) * nx + x;  // y faces: (nz, ny + 1, nx)
            __stcs(gx + ax, g0);
            __stcs(gy + ay, g1);
            __stcs(gz + c, g2);
            if (x == nx - 1) gx[ax + 1] = 0.f;
            if (y == ny - 1) gy[ay + nx] = 0.f;
            if (z == nz - 1) gz[c + nxy] = 0.f;
        }
        lzh = lh;
        lzl = ll;
        pzh = ph;
        pzl = pl;
    }
}

// The same for even nx, two cells per thread: 16-byte loads of lam and p (both 16-byte
// aligned, as the ABI requires), each plane's loads issued one plane ahead, and every value
// split once.  Block (32, kGrad2Rows): a warp covers 64 cells of a row, the block a tile of
// 64 cells x kGrad2Rows rows, marching kGrad2Planes planes in z.  Per plane each thread writes
// its pairs into a shared-memory tile (double-buffered by plane parity, one barrier per plane);
// the y-1 row of a warp is the tile row above it, the x-1 cell of a lane the neighbouring
// lane's second cell (shuffle).  The tile's halo -- row y0 - 1 and the cells x0 - 1 of its
// rows, 160 values -- is loaded and split by five warps, one value per lane: warps 0 and 1 lam
// of the halo row, warps 2 and 3 p, warp 4 the halo column (lanes 0-15 lam, 16-31 p).  So no
// lane splits a neighbour's value again, no warp waits on a halo load that was not
// prefetched, and no warp splits more than one value beyond its own cells before the barrier.
constexpr int kGrad2Rows = 16, kGrad2Planes = 32;
static_assert(kGrad2Rows >= 5, "five warps of the block load the halo");

__device__ __forceinline__ float4 split2(double2 v) {
    float4 r;
    split_f64(v.x, r.x, r.y);
    split_f64(v.y, r.z, r.w);
    return r;  // (hi, lo) of cell x, then of cell x + 1
}
// -(la - lb)(pa - pb) ih2 from the split pairs
__device__ __forceinline__ float grad_face(float lah, float lal, float lbh, float lbl, float pah, float pal,
                                           float pbh, float pbl, float ih2) {
    return -((lah - lbh) + (lal - lbl)) * (((pah - pbh) + (pal - pbl)) * ih2);
}

struct GradTile {
    float4 l[2][kGrad2Rows][32], p[2][kGrad2Rows][32];  // pairs of the tile's cells
    float4 yl[2][32], yp[2][32];                          // pairs of the halo row y0 - 1, as the tile
    float2 xl[2][kGrad2Rows], xp[2][kGrad2Rows];          // pair of cell x0 - 1 of each row
};

__global__ void __launch_bounds__(32 * kGrad2Rows) k_adjoint_grad_split2(
    int nx, int ny, int nz, float ih2, const double *__restrict__ lam, const double *__restrict__ p,
    float *__restrict__ gx, float *__restrict__ gy, float *__restrict__ gz) {
    __shared__ GradTile T;
    const int lane = threadIdx.x, ty = threadIdx.y;
    const int x0 = blockIdx.x * 64, y0 = blockIdx.y * kGrad2Rows;
    const int x = x0 + 2 * lane;
    const int y = y0 + ty;
    const int z0 = blockIdx.z * kGrad2Planes;
    const int z1 = min(z0 + kGrad2Planes, nz);
    const bool act = x < nx && y < ny;  // nx even: x + 1 < nx too
    const int nxy = nx * ny;
    // the halo value this thread loads per plane (warps 0-4), as an offset from the plane start
    const int hx = x0 + (ty & 1) * 32 + lane, hy = y0 + (lane & 15);
    const bool hrow = ty < 4 && y0 > 0 && hx < nx;
    const bool hcol = ty == 4 && x0 > 0 && hy < ny;
    const bool hld = hrow || hcol;
    const double *hsrc = (ty == 2 || ty == 3 || (ty == 4 && lane >= 16)) ? p : lam;
    const int hoff = hrow ? (y0 - 1) * nx + hx : (hcol ? hy * nx + x0 - 1 : 0);
    const double2 zero2 = make_double2(0.0, 0.0);
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 lz = zero4, pz = zero4;  // plane z - 1
    if (act && z0 > 0) {
        const int c = (z0 - 1) * nxy + y * nx + x;
        lz = split2(*reinterpret_cast<const double2 *>(lam + c));
        pz = split2(*reinterpret_cast<const double2 *>(p + c));
    }
    // running offsets of this thread's cells, x faces, y faces and halo value in plane z
    int c = z0 * nxy + y * nx + x;
    int ax = (z0 * ny + y) * (nx + 1) + x;  // x faces: (nz, ny, nx + 1), not 8-byte aligned
    int ay = (z0 * (ny + 1) + y) * nx + x;  // y faces: (nz, ny + 1, nx), even
    int hc = z0 * nxy + hoff;
    const int sx = ny * (nx + 1), sy = (ny + 1) * nx;
    double2 Lc = zero2, Pc = zero2;
    double Hc = 0.0;
    if (z0 < z1) {
        if (act) {
            Lc = *reinterpret_cast<const double2 *>(lam + c);
            Pc = *reinterpret_cast<const double2 *>(p + c);
        }
        if (hld) Hc = hsrc[hc];
    }
    for (int z = z0; z < z1; ++z, c += nxy, ax += sx, ay += sy, hc += nxy) {
        const int buf = z & 1;
        double2 Ln = zero2, Pn = zero2;
        double Hn = 0.0;
        if (z + 1 < z1) {
            if (act) {
                Ln = *reinterpret_cast<const double2 *>(lam + c + nxy);
                Pn = *reinterpret_cast<const double2 *>(p + c + nxy);
            }
            if (hld) Hn = hsrc[hc + nxy];
        }
        const float4 l = split2(Lc), q = split2(Pc);
        T.l[buf][ty][lane] = l;
        T.p[buf][ty][lane] = q;
        if (ty < 5) {  // warp-uniform: the halo (zeros where it is not loaded)
            float hh, hl;
            split_f64(Hc, hh, hl);
            const float2 hv = make_float2(hh, hl);
            if (ty < 4) reinterpret_cast<float2 *>(ty < 2 ? T.yl[buf] : T.yp[buf])[(ty & 1) * 32 + lane] = hv;
            else if (lane < 16) T.xl[buf][lane] = hv;
            else T.xp[buf][lane - 16] = hv;
        }
        __syncthreads();  // buffer `buf` was last read two planes ago, before the previous barrier
        const float4 ly = ty > 0 ? T.l[buf][ty - 1][lane] : T.yl[buf][lane];
        const float4 py = ty > 0 ? T.p[buf][ty - 1][lane] : T.yp[buf][lane];
        // cell x - 1: the second cell of the lane to the left; lane 0 takes the halo column
        const float2 hxl = T.xl[buf][ty], hxp = T.xp[buf][ty];
        float lxh = __shfl_up_sync(0xffffffffu, l.z, 1), lxl = __shfl_up_sync(0xffffffffu, l.w, 1);
        float pxh = __shfl_up_sync(0xffffffffu, q.z, 1), pxl = __shfl_up_sync(0xffffffffu, q.w, 1);
        if (lane == 0) {
            lxh = hxl.x;
            lxl = hxl.y;
            pxh = hxp.x;
            pxl = hxp.y;
        }
        if (act) {
            float a0 = 0.f, b0 = 0.f, b1 = 0.f, e0 = 0.f, e1 = 0.f;
            if (x > 0) a0 = grad_face(lxh, lxl, l.x, l.y, pxh, pxl, q.x, q.y, ih2);
            const float a1 = grad_face(l.x, l.y, l.z, l.w, q.x, q.y, q.z, q.w, ih2);
            if (y > 0) {
                b0 = grad_face(ly.x, ly.y, l.x, l.y, py.x, py.y, q.x, q.y, ih2);
                b1 = grad_face(ly.z, ly.w, l.z, l.w, py.z, py.w, q.z, q.w, ih2);
            }
            if (z > 0) {
                e0 = grad_face(lz.x, lz.y, l.x, l.y, pz.x, pz.y, q.x, q.y, ih2);
                e1 = grad_face(lz.z, lz.w, l.z, l.w, pz.z, pz.w, q.z, q.w, ih2);
            }
            __stcs(gx + ax, a0);
            __stcs(gx + ax + 1, a1);
            __stcs(reinterpret_cast<float2 *>(gy + ay), make_float2(b0, b1));
            __stcs(reinterpret_cast<float2 *>(gz + c), make_float2(e0, e1));
            if (x + 2 == nx) gx[ax + 2] = 0.f;
            if (y == ny - 1) *reinterpret_cast<float2 *>(gy + ay + nx) = make_float2(0.f, 0.f);
            if (z == nz - 1) *reinterpret_cast<float2 *>(gz + c + nxy) = make_float2(0.f, 0.f);
        }
        lz = l;
        pz = q;
        Lc = Ln;
        Pc = Pn;
        Hc = Hn;
    }
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
    static const int wave_pt = wave_blocks((const void *)k_fine_resid_pair<true, false>, kReduceThreads);
    static const int wave_pf = wave_blocks((const void *)k_fine_resid_pair<false, false>, kReduceThreads);
    const int nb = fill_blocks(reduce_blocks(d.n / 2), b_scaled ? wave_pt : wave_pf);
    count_launch();
    if (d.zlo || d.zhi) {
        // a slab; its own wave: the ghost tests take more registers, one resident block fewer
        // per SM
        static const int wave_gt = wave_blocks((const void *)k_fine_resid_pair<true, true>, kReduceThreads);
        static const int wave_gf = wave_blocks((const void *)k_fine_resid_pair<false, true>, kReduceThreads);
        const int ng = fill_blocks(reduce_blocks(d.n / 2), b_scaled ? wave_gt : wave_gf);
        if (b_scaled)
            k_fine_resid_pair<true, true><<<ng, kReduceThreads, 0, s>>>(d, L, h2, fx, fy, fz, diag, b, p, r32, s32, partials);
        else
            k_fine_resid_pair<false, true><<<ng, kReduceThreads, 0, s>>>(d, L, h2, fx, fy, fz, diag, b, p, r32, s32, partials);
        count_launch();
        k_final<<<1, kReduceThreads, 0, s>>>(partials, ng, out);
        return;
    }
    if (b_scaled) {
        k_fine_resid_pair<true, false><<<nb, kReduceThreads, 0, s>>>(d, L, h2, fx, fy, fz, diag, b, p, r32, s32, partials);
    } else {
        k_fine_resid_pair<false, false><<<nb, kReduceThreads, 0, s>>>(d, L, h2, fx, fy, fz, diag, b, p, r32, s32, partials);
    }
    count_launch();
    k_final<<<1, kReduceThreads, 0, s>>>(partials, nb, out);
}

void launch_zero_resid32(cudaStream_t s, Dims d, Lay L, const double *b, double scale32, float *r32) {
    count_launch();
    k_zero_resid32<<<blocks_for(d.n), kThreads, 0, s>>>(d, L, b, (float)scale32, r32);
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

inline bool aligned16h(const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; }
inline bool aligned8h(const void *q) { return (reinterpret_cast<uintptr_t>(q) & 7) == 0; }

void launch_adjoint_grad(cudaStream_t s, Dims d, double h, const double *lam, const double *p,
                         const double *fx, const double *fy, const double *fz, const double *csfx,
                         const double *csfy, const double *csfz, double sigma, float *gx,
                         float *gy, float *gz, double *partials, double *out) {
    // without a surface term dL/dsigma is 0 (the caller sets it) and the face gradients need no
    // FP64 arithmetic: the split-FP32 kernel, when the face arrays fit 32-bit indices
    if (!csfx && gx && (i64)(d.nx + 1) * (d.ny + 1) * (d.nz + 1) < (1ll << 31)) {
        count_launch();
        if (d.nx % 2 == 0 && aligned16h(lam) && aligned16h(p) && aligned8h(gy) && aligned8h(gz)) {
            const dim3 grid((d.nx / 2 + 31) / 32, (d.ny + kGrad2Rows - 1) / kGrad2Rows,
                            (d.nz + kGrad2Planes - 1) / kGrad2Planes);
            k_adjoint_grad_split2<<<grid, dim3(32, kGrad2Rows), 0, s>>>(d.nx, d.ny, d.nz, (float)(1.0 / (h * h)),
                                                                        lam, p, gx, gy, gz);
            return;
        }
        const dim3 grid((d.nx + 31) / 32, (d.ny + kGradRows - 1) / kGradRows,
                        (d.nz + kGradPlanes - 1) / kGradPlanes);
        k_adjoint_grad_split<<<grid, dim3(32, kGradRows), 0, s>>>(d.nx, d.ny, d.nz, (float)(1.0 / (h * h)),
                                                                  lam, p, gx, gy, gz);
        return;
    }
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
