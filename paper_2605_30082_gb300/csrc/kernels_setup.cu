// Set-up kernels: density mixing (Eq. (5)), face coefficients, coarsening,
// inverse diagonals, precision copies, CSF faces, RHS assembly and the dense
// coarse-level inverse.  All FP64, one thread per cell (these run once per
// density field, not inside the V-cycle).
#include "mg_internal.cuh"

namespace mg {

namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(i64 n) { return (unsigned)((n + kThreads - 1) / kThreads); }

struct FracArgs {
    const double *f[4];
    double drho[4];  // rho_q - rho_last
    double rho_last;
    int nfrac;
};

// Eq. (5) in the form rho_last + sum_q (rho_q - rho_last) f_q: one FMA per fraction (the
// literal sum_q rho_q f_q + rho_last (1 - sum_q f_q) takes 2 nfrac + 1 FP64 operations, which
// bound this kernel by the FP64 pipe); equal in exact arithmetic, within a few units in the
// last place in FP64
__global__ void k_density(i64 n, FracArgs a, double *rho) {
    i64 m = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    double r = a.rho_last;
    for (int q = 0; q < a.nfrac; ++q) r = fma(a.drho[q], a.f[q][m], r);
    rho[m] = r;
}

// 0 < v <= 1.79e308, tested on the bit pattern (positive doubles order like their bits, NaN and
// infinity lie above the bound, negative values and zero at or below 0): no FP64 comparison
__device__ __forceinline__ bool good_positive(double v) {
    const long long u = __double_as_longlong(v);
    return u > 0 && u <= 0x7fefdcf158adbb99ll;
}

// v / 2 for v = 0 or normal with a normal result (exponent field above 1): one integer subtraction
// from the exponent field instead of an FP64 multiplication; otherwise the multiplication
__device__ __forceinline__ double half_of(double v) {
    const long long u = __double_as_longlong(v);
    const int e = (int)((u >> 52) & 0x7ff);
    if (e > 1 && e < 0x7ff) return __longlong_as_double(u - (1ll << 52));
    return 0.5 * v;
}

// s = 1/rho per cell, validating rho (finite and > 0)
__global__ void k_inv_rho(i64 n, const double *__restrict__ rho, double *sinv, unsigned *err) {
    const i64 m = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    const double r = rho[m];
    if (!good_positive(r)) {
        atomicOr(err, 1u);
        sinv[m] = 1.0;
        return;
    }
    sinv[m] = recip64(r);
}

// beta on the low faces: 1 / harmonic mean of the two densities = (s_L + s_R) / 2; blocks take
// rows (grid y, strided), threads the cells of a row
__global__ void k_faces_from_s(Dims d, const double *__restrict__ sv, double *fx, double *fy, double *fz) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.nx) return;
    const i64 rows = (i64)d.ny * d.nz;
    for (i64 row = blockIdx.y; row < rows; row += gridDim.y) {
        const int j = (int)((unsigned)row % (unsigned)d.ny), k = (int)((unsigned)row / (unsigned)d.ny);  // rows < 2^31
        const i64 c = row * d.nx + i;
        const double sc = sv[c];
        fx[c] = i > 0 ? half_of(sv[c - 1] + sc) : 0.0;
        fy[c] = j > 0 ? half_of(sv[c - d.nx] + sc) : 0.0;
        fz[c] = k > 0 ? half_of(sv[c - d.nxy] + sc) : 0.0;
    }
}

// the same for even nx, two cells per thread: 16-byte loads and stores (the x - 1 value of the
// pair's first cell is one scalar load, from the line the neighbouring lane reads); the same
// additions in the same order as k_faces_from_s, so bitwise the same faces
__global__ void k_faces_from_s2(Dims d, const double *__restrict__ sv, double *fx, double *fy, double *fz) {
    const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= d.nx) return;
    const i64 rows = (i64)d.ny * d.nz;
    auto ld2 = [](const double *q) { return *reinterpret_cast<const double2 *>(q); };
    auto st2 = [](double *q, double a, double b) { *reinterpret_cast<double2 *>(q) = make_double2(a, b); };
    for (i64 row = blockIdx.y; row < rows; row += gridDim.y) {
        const int j = (int)((unsigned)row % (unsigned)d.ny), k = (int)((unsigned)row / (unsigned)d.ny);  // rows < 2^31
        const i64 c = row * d.nx + i;
        const double2 sc = ld2(sv + c);
        const double sl = i > 0 ? sv[c - 1] : 0.0;
        st2(fx + c, i > 0 ? half_of(sl + sc.x) : 0.0, half_of(sc.x + sc.y));
        if (j > 0) {
            const double2 sy = ld2(sv + c - d.nx);
            st2(fy + c, half_of(sy.x + sc.x), half_of(sy.y + sc.y));
        } else {
            st2(fy + c, 0.0, 0.0);
        }
        if (k > 0) {
            const double2 sz = ld2(sv + c - d.nxy);
            st2(fz + c, half_of(sz.x + sc.x), half_of(sz.y + sc.y));
        } else {
            st2(fz + c, 0.0, 0.0);
        }
    }
}

__global__ void k_faces_from_api(Dims d, const double *__restrict__ bx, const double *__restrict__ by,
                                 const double *__restrict__ bz, double *fx, double *fy, double *fz,
                                 unsigned *err) {
    i64 c = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.n) return;
    const unsigned cu_ = (unsigned)c, ru_ = cu_ / (unsigned)d.nx;  // c < 2^32: 32-bit divisions
    int i = (int)(cu_ - ru_ * (unsigned)d.nx);
    int j = (int)(ru_ % (unsigned)d.ny);
    int k = (int)(ru_ / (unsigned)d.ny);
    double vx = 0.0, vy = 0.0, vz = 0.0;
    if (i > 0) vx = bx[((i64)k * d.ny + j) * (d.nx + 1) + i];
    if (j > 0) vy = by[((i64)k * (d.ny + 1) + j) * d.nx + i];
    if (k > 0) vz = bz[c];  // (nz+1, ny, nx): plane k starts at k*nxy
    if ((i > 0 && !good_positive(vx)) || (j > 0 && !good_positive(vy)) ||
        (k > 0 && !good_positive(vz)))
        atomicOr(err, 1u);
    fx[c] = vx;
    fy[c] = vy;
    fz[c] = vz;
}

__global__ void k_faces_to_api(Dims d, const double *__restrict__ fx, const double *__restrict__ fy,
                               const double *__restrict__ fz, double *bx, double *by, double *bz) {
    i64 c = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.n) return;
    const unsigned cu_ = (unsigned)c, ru_ = cu_ / (unsigned)d.nx;  // c < 2^32: 32-bit divisions
    int i = (int)(cu_ - ru_ * (unsigned)d.nx);
    int j = (int)(ru_ % (unsigned)d.ny);
    int k = (int)(ru_ / (unsigned)d.ny);
    i64 ax = ((i64)k * d.ny + j) * (d.nx + 1) + i;
    i64 ay = ((i64)k * (d.ny + 1) + j) * d.nx + i;
    bx[ax] = i > 0 ? fx[c] : 0.0;
    by[ay] = j > 0 ? fy[c] : 0.0;
    bz[c] = k > 0 ? fz[c] : 0.0;
    if (i == d.nx - 1) bx[ax + 1] = 0.0;
    if (j == d.ny - 1) by[ay + d.nx] = 0.0;
    if (k == d.nz - 1) bz[c + d.nxy] = 0.0;
}

__global__ void k_invdiag(Dims d, const double *__restrict__ fx, const double *__restrict__ fy,
                          const double *__restrict__ fz, double *invd64, double *diag) {
    i64 c = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.n) return;
    const unsigned cu_ = (unsigned)c, ru_ = cu_ / (unsigned)d.nx;  // c < 2^32: 32-bit divisions
    int i = (int)(cu_ - ru_ * (unsigned)d.nx);
    int j = (int)(ru_ % (unsigned)d.ny);
    int k = (int)(ru_ / (unsigned)d.ny);
    // order x-, x+, y-, y+, z-, z+ (low faces of i=0 etc. are stored as 0)
    double s = fx[c];
    if (i < d.nx - 1) s += fx[c + 1];
    s += fy[c];
    if (j < d.ny - 1) s += fy[c + d.nx];
    s += fz[c];
    if (k < d.nz - 1 || d.zhi) s += fz[c + d.nxy];  // a slab's face to its ghost plane counts
    if (invd64) invd64[c] = recip64(s);
    if (diag) diag[c] = s;
}

// coarse low face = mean of the 4 fine low faces that tile it
__global__ void k_coarsen(Dims f, Dims cd, const double *__restrict__ ffx,
                          const double *__restrict__ ffy, const double *__restrict__ ffz,
                          double *cfx, double *cfy, double *cfz) {
    i64 C = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (C >= cd.n) return;
    int I = (int)(C % cd.nx);
    int J = (int)((C / cd.nx) % cd.ny);
    int K = (int)(C / cd.nxy);
    i64 base = ((i64)(2 * K) * f.ny + 2 * J) * f.nx + 2 * I;  // child (0,0,0)
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b) sx += ffx[base + c * f.nxy + b * f.nx];
    for (int c = 0; c < 2; ++c)
        for (int a = 0; a < 2; ++a) sy += ffy[base + c * f.nxy + a];
    for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) sz += ffz[base + b * f.nx + a];
    cfx[C] = sx / 4.0;
    cfy[C] = sy / 4.0;
    cfz[C] = sz / 4.0;
}

__global__ void k_to_f32(i64 n, const double *__restrict__ src, float *dst) {
    i64 m = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (m < n) dst[m] = (float)src[m];
}

__global__ void k_csf_faces(Dims d, double ih, const double *__restrict__ f,
                            const double *__restrict__ kap, double *cx, double *cy, double *cz) {
    i64 c = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.n) return;
    const unsigned cu_ = (unsigned)c, ru_ = cu_ / (unsigned)d.nx;  // c < 2^32: 32-bit divisions
    int i = (int)(cu_ - ru_ * (unsigned)d.nx);
    int j = (int)(ru_ % (unsigned)d.ny);
    int k = (int)(ru_ / (unsigned)d.ny);
    i64 ax = ((i64)k * d.ny + j) * (d.nx + 1) + i;
    i64 ay = ((i64)k * (d.ny + 1) + j) * d.nx + i;
    double fc = f[c], kc = kap[c];
    cx[ax] = i > 0 ? 0.5 * (kap[c - 1] + kc) * (fc - f[c - 1]) * ih : 0.0;
    cy[ay] = j > 0 ? 0.5 * (kap[c - d.nx] + kc) * (fc - f[c - d.nx]) * ih : 0.0;
    cz[c] = k > 0 ? 0.5 * (kap[c - d.nxy] + kc) * (fc - f[c - d.nxy]) * ih : 0.0;
    if (i == d.nx - 1) cx[ax + 1] = 0.0;
    if (j == d.ny - 1) cy[ay + d.nx] = 0.0;
    if (k == d.nz - 1) cz[c + d.nxy] = 0.0;
}

// b = b0 + D u + sigma D(beta csf); D over interior faces, (+high - low)/h; terms optional
__global__ void k_rhs(Dims d, double ih, const double *b0, const double *__restrict__ ux,
                      const double *__restrict__ uy, const double *__restrict__ uz,
                      const double *__restrict__ fx, const double *__restrict__ fy,
                      const double *__restrict__ fz, const double *__restrict__ csx,
                      const double *__restrict__ csy, const double *__restrict__ csz, double sigma,
                      double *b) {
    i64 c = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.n) return;
    const unsigned cu_ = (unsigned)c, ru_ = cu_ / (unsigned)d.nx;  // c < 2^32: 32-bit divisions
    int i = (int)(cu_ - ru_ * (unsigned)d.nx);
    int j = (int)(ru_ % (unsigned)d.ny);
    int k = (int)(ru_ / (unsigned)d.ny);
    i64 ax = ((i64)k * d.ny + j) * (d.nx + 1) + i;
    i64 ay = ((i64)k * (d.ny + 1) + j) * d.nx + i;
    double v = b0 ? b0[c] : 0.0;
    if (ux) {
        // (high - low) per axis, wall faces as 0: five FP64 additions and one fused
        // multiply-add per cell
        const double xm = i > 0 ? ux[ax] : 0.0, xp = i < d.nx - 1 ? ux[ax + 1] : 0.0;
        const double ym = j > 0 ? uy[ay] : 0.0, yp = j < d.ny - 1 ? uy[ay + d.nx] : 0.0;
        const double zm = k > 0 ? uz[c] : 0.0, zp = k < d.nz - 1 ? uz[c + d.nxy] : 0.0;
        const double s = ((xp - xm) + (yp - ym)) + (zp - zm);
        v = fma(s, ih, v);
    }
    if (csx) {
        double t = 0.0;
        if (i > 0) t -= fx[c] * csx[ax];
        if (i < d.nx - 1) t += fx[c + 1] * csx[ax + 1];
        if (j > 0) t -= fy[c] * csy[ay];
        if (j < d.ny - 1) t += fy[c + d.nx] * csy[ay + d.nx];
        if (k > 0) t -= fz[c] * csz[c];
        if (k < d.nz - 1) t += fz[c + d.nxy] * csz[c + d.nxy];
        v += sigma * (t * ih);
    }
    b[c] = v;
}

// ---- dense coarse inverse -----------------------------------------------------------
// M (row-major nc x nc) = A_c; one thread per row
__global__ void k_coarse_assemble(Dims d, double ih2, const double *__restrict__ fx,
                                  const double *__restrict__ fy, const double *__restrict__ fz,
                                  double *M) {
    i64 c = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.n) return;
    const unsigned cu_ = (unsigned)c, ru_ = cu_ / (unsigned)d.nx;  // c < 2^32: 32-bit divisions
    int i = (int)(cu_ - ru_ * (unsigned)d.nx);
    int j = (int)(ru_ % (unsigned)d.ny);
    int k = (int)(ru_ / (unsigned)d.ny);
    double *row = M + c * d.n;
    for (i64 q = 0; q < d.n; ++q) row[q] = 0.0;
    double diag = 0.0, v;
    if (i > 0) { v = fx[c] * ih2; row[c - 1] -= v; diag += v; }
    if (i < d.nx - 1) { v = fx[c + 1] * ih2; row[c + 1] -= v; diag += v; }
    if (j > 0) { v = fy[c] * ih2; row[c - d.nx] -= v; diag += v; }
    if (j < d.ny - 1) { v = fy[c + d.nx] * ih2; row[c + d.nx] -= v; diag += v; }
    if (k > 0) { v = fz[c] * ih2; row[c - d.nxy] -= v; diag += v; }
    if (k < d.nz - 1) { v = fz[c + d.nxy] * ih2; row[c + d.nxy] -= v; diag += v; }
    row[c] = diag;
}

// scal[0] = c = mean(diag)/nc; adds c to every entry; scal[1] = 1/M[0][0]
__global__ void k_coarse_shift(int nc, double *M, double *scal) {
    __shared__ double red[1024];
    double t = 0.0;
    for (int q = threadIdx.x; q < nc; q += blockDim.x) t += M[(i64)q * nc + q];
    red[threadIdx.x] = t;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    double cshift = red[0] / nc / nc;
    __syncthreads();
    for (i64 q = threadIdx.x; q < (i64)nc * nc; q += blockDim.x) M[q] += cshift;
    __syncthreads();
    if (threadIdx.x == 0) {
        scal[0] = cshift;
        scal[1] = 1.0 / M[0];
    }
}

// ---- blocked Gauss-Jordan inversion in place (no pivoting: M is symmetric positive definite)
// Block step on the pivot block K = [kb, kb + bs): P^-1 (one block), the row panel
// M[K, J] <- P^-1 M[K, J], the trailing update M[I, J] <- M[I, J] - M[I, K] M[K, J], and the
// column panel M[I, K] <- -M[I, K] P^-1, M[K, K] <- P^-1 (I, J outside K).  The same algebra as
// the element-wise sweeps, BS pivots per step, so n / BS steps of four launches instead of n.
constexpr int GJ_BS = kGjBlock;

// P^-1 of the bs x bs pivot block by element-wise Gauss-Jordan in shared memory; Pinv (bs x bs,
// row-major) written to global scratch.  One block of GJ_BS x GJ_BS threads.
__global__ void k_gj_pivot_inv(int n, int kb, int bs, const double *__restrict__ M, double *Pinv) {
    __shared__ double P[GJ_BS][GJ_BS + 1];
    __shared__ double rps;
    const int tx = threadIdx.x, ty = threadIdx.y;
    if (tx < bs && ty < bs) P[ty][tx] = M[(i64)(kb + ty) * n + kb + tx];
    __syncthreads();
    for (int k = 0; k < bs; ++k) {
        // one FP64 division per pivot (by one thread), not one per thread
        if (tx == 0 && ty == 0) rps = 1.0 / P[k][k];
        __syncthreads();
        double v = 0.0;
        if (tx < bs && ty < bs) {
            const double rp = rps;
            if (ty == k && tx == k) v = rp;
            else if (ty == k) v = P[k][tx] * rp;
            else if (tx == k) v = -P[ty][k] * rp;
            else v = P[ty][tx] - P[ty][k] * (P[k][tx] * rp);
        }
        __syncthreads();
        if (tx < bs && ty < bs) P[ty][tx] = v;
        __syncthreads();
    }
    if (tx < bs && ty < bs) Pinv[ty * GJ_BS + tx] = P[ty][tx];
}

// row panel: for the 32-column tile blockIdx.x (skipping K's columns), M[K, J] <- P^-1 M[K, J]
__global__ void k_gj_row_panel(int n, int kb, int bs, double *M, const double *__restrict__ Pinv) {
    __shared__ double Pi[GJ_BS][GJ_BS + 1], R[GJ_BS][GJ_BS + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int j = blockIdx.x * GJ_BS + tx;
    const bool colok = j < n && (j < kb || j >= kb + bs);
    if (ty < bs && tx < bs) Pi[ty][tx] = Pinv[ty * GJ_BS + tx];
    if (ty < bs) R[ty][tx] = colok ? M[(i64)(kb + ty) * n + j] : 0.0;
    __syncthreads();
    if (ty < bs && colok) {
        double acc = 0.0;
        for (int t = 0; t < bs; ++t) acc = fma(Pi[ty][t], R[t][tx], acc);
        M[(i64)(kb + ty) * n + j] = acc;
    }
}

// trailing update of the 32 x 32 tile (blockIdx.y rows, blockIdx.x columns), rows and columns
// outside K: M[i, j] -= sum_t M[i, kb + t] M[kb + t, j] (the row panel already updated)
__global__ void k_gj_trailing(int n, int kb, int bs, double *M) {
    __shared__ double C[GJ_BS][GJ_BS + 1], R[GJ_BS][GJ_BS + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = blockIdx.y * GJ_BS + ty, j = blockIdx.x * GJ_BS + tx;
    const bool rowok = i < n && (i < kb || i >= kb + bs), colok = j < n && (j < kb || j >= kb + bs);
    // C[ty][t] = M[i, kb + t], R[t][tx] = M[kb + t, j]
    C[ty][tx] = (i < n && tx < bs) ? M[(i64)i * n + kb + tx] : 0.0;
    R[ty][tx] = (ty < bs && j < n) ? M[(i64)(kb + ty) * n + j] : 0.0;
    __syncthreads();
    if (rowok && colok) {
        double acc = M[(i64)i * n + j];
        for (int t = 0; t < bs; ++t) acc = fma(-C[ty][t], R[t][tx], acc);
        M[(i64)i * n + j] = acc;
    }
}

// column panel: M[i, K] <- -M[i, K] P^-1 for rows i outside K; the block of rows holding K
// writes M[K, K] = P^-1
__global__ void k_gj_col_panel(int n, int kb, int bs, double *M, const double *__restrict__ Pinv) {
    __shared__ double Pi[GJ_BS][GJ_BS + 1], C[GJ_BS][GJ_BS + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = blockIdx.x * GJ_BS + ty;
    if (ty < bs && tx < bs) Pi[ty][tx] = Pinv[ty * GJ_BS + tx];
    C[ty][tx] = (i < n && tx < bs) ? M[(i64)i * n + kb + tx] : 0.0;
    __syncthreads();
    if (i < n && tx < bs) {
        if (i >= kb && i < kb + bs) {
            M[(i64)i * n + kb + tx] = Pi[i - kb][tx];
        } else {
            double acc = 0.0;
            for (int t = 0; t < bs; ++t) acc = fma(C[ty][t], Pi[t][tx], acc);
            M[(i64)i * n + kb + tx] = -acc;
        }
    }
}

__global__ void k_pinv_finish(int nc, double *M, const double *__restrict__ scal) {
    i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (i64)nc * nc) return;
    M[e] -= 1.0 / (scal[0] * (double)nc * (double)nc);
}

}  // namespace

void launch_density(cudaStream_t s, i64 n, int nfrac, const double *const *frac,
                    const double *rho_phase, double *rho) {
    FracArgs a;
    a.nfrac = nfrac;
    a.rho_last = rho_phase[nfrac];
    for (int q = 0; q < 4; ++q) {
        a.f[q] = q < nfrac ? frac[q] : nullptr;
        a.drho[q] = q < nfrac ? rho_phase[q] - rho_phase[nfrac] : 0.0;
    }
    count_launch();
    k_density<<<blocks_for(n), kThreads, 0, s>>>(n, a, rho);
}

void launch_faces_from_rho(cudaStream_t s, Dims d, const double *rho, double *sinv, double *fx, double *fy,
                           double *fz, unsigned *err) {
    count_launch(2);
    k_inv_rho<<<blocks_for(d.n), kThreads, 0, s>>>(d.n, rho, sinv, err);
    const i64 rows = (i64)d.ny * d.nz;
    auto a16 = [](const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
    if (d.nx % 2 == 0 && a16(sinv) && a16(fx) && a16(fy) && a16(fz)) {
        const dim3 grd((unsigned)((d.nx / 2 + 127) / 128), (unsigned)(rows < 65535 ? rows : 65535));
        k_faces_from_s2<<<grd, 128, 0, s>>>(d, sinv, fx, fy, fz);
        return;
    }
    const dim3 grd((unsigned)((d.nx + 127) / 128), (unsigned)(rows < 65535 ? rows : 65535));
    k_faces_from_s<<<grd, 128, 0, s>>>(d, sinv, fx, fy, fz);
}

void launch_faces_from_api(cudaStream_t s, Dims d, const double *bx, const double *by,
                           const double *bz, double *fx, double *fy, double *fz, unsigned *err) {
    count_launch();
    k_faces_from_api<<<blocks_for(d.n), kThreads, 0, s>>>(d, bx, by, bz, fx, fy, fz, err);
}

void launch_faces_to_api(cudaStream_t s, Dims d, const double *fx, const double *fy,
                         const double *fz, double *bx, double *by, double *bz) {
    count_launch();
    k_faces_to_api<<<blocks_for(d.n), kThreads, 0, s>>>(d, fx, fy, fz, bx, by, bz);
}

void launch_invdiag(cudaStream_t s, Dims d, const double *fx, const double *fy, const double *fz,
                    double *invd64, double *diag) {
    if (!invd64 && !diag) return;
    count_launch();
    k_invdiag<<<blocks_for(d.n), kThreads, 0, s>>>(d, fx, fy, fz, invd64, diag);
}

void launch_coarsen(cudaStream_t s, Dims fine, const double *ffx, const double *ffy,
                    const double *ffz, double *cfx, double *cfy, double *cfz) {
    Dims cd = make_dims(fine.nx / 2, fine.ny / 2, fine.nz / 2);
    count_launch();
    k_coarsen<<<blocks_for(cd.n), kThreads, 0, s>>>(fine, cd, ffx, ffy, ffz, cfx, cfy, cfz);
}

void launch_to_f32(cudaStream_t s, i64 n, const double *src, float *dst) {
    count_launch();
    k_to_f32<<<blocks_for(n), kThreads, 0, s>>>(n, src, dst);
}

void launch_csf_faces(cudaStream_t s, Dims d, double h, const double *f, const double *kappa,
                      double *cx, double *cy, double *cz) {
    count_launch();
    k_csf_faces<<<blocks_for(d.n), kThreads, 0, s>>>(d, 1.0 / h, f, kappa, cx, cy, cz);
}

void launch_rhs(cudaStream_t s, Dims d, double h, const double *b0, const double *ux, const double *uy,
                const double *uz, const double *fx, const double *fy, const double *fz,
                const double *csfx, const double *csfy, const double *csfz, double sigma,
                double *b) {
    count_launch();
    k_rhs<<<blocks_for(d.n), kThreads, 0, s>>>(d, 1.0 / h, b0, ux, uy, uz, fx, fy, fz, csfx, csfy,
                                               csfz, sigma, b);
}

void launch_coarse_assemble(cudaStream_t s, Dims d, double ih2, const double *fx, const double *fy,
                            const double *fz, double *M, double *scal) {
    count_launch();
    k_coarse_assemble<<<blocks_for(d.n), kThreads, 0, s>>>(d, ih2, fx, fy, fz, M);
    count_launch();
    k_coarse_shift<<<1, 1024, 0, s>>>((int)d.n, M, scal);
}

void launch_gj_blocked(cudaStream_t s, int nc, double *M, double *scratch) {
    const dim3 blk(GJ_BS, GJ_BS);
    const int nt = (nc + GJ_BS - 1) / GJ_BS;
    for (int kb = 0; kb < nc; kb += GJ_BS) {
        const int bs = nc - kb < GJ_BS ? nc - kb : GJ_BS;
        count_launch(4);
        k_gj_pivot_inv<<<1, blk, 0, s>>>(nc, kb, bs, M, scratch);
        k_gj_row_panel<<<nt, blk, 0, s>>>(nc, kb, bs, M, scratch);
        k_gj_trailing<<<dim3(nt, nt), blk, 0, s>>>(nc, kb, bs, M);
        k_gj_col_panel<<<nt, blk, 0, s>>>(nc, kb, bs, M, scratch);
    }
}

void launch_pinv_finish(cudaStream_t s, int nc, double *M, const double *scal) {
    count_launch();
    k_pinv_finish<<<blocks_for((i64)nc * nc), kThreads, 0, s>>>(nc, M, scal);
}

}  // namespace mg
