// The two passes either side of the solve: the velocity correction that closes the
// projection step, and the density adjoint that carries dL/dbeta back to the density
// and the phase fractions.
//
// Velocity correction (paper §2, Eqs. (1)-(2)): with A = -D diag(beta) G and
// A p = D u + sigma D(beta csf), the face velocities
//     u_f <- u_f + beta_f ( (p_R - p_L)/h + sigma csf_f )
// have zero discrete divergence.  Wall faces keep their values (zero-flux faces).
//
// Density adjoint (Eq. (5) and beta_f = (1/rho_L + 1/rho_R)/2):
//     dL/drho_c = -1/(2 rho_c^2) * sum over the interior faces f of c of dL/dbeta_f,
//     dL/df_q   = dL/drho_c * (rho_q - rho_last).
#include <cmath>

#include "mg_internal.cuh"

namespace mg {
namespace {

// v * 2^m (m >= 0) by an integer addition to the IEEE-754 exponent field (binary64: 11 exponent
// bits from bit 52; the sign bit is untouched), exact like the FP64 multiplication it replaces,
// for normal v whose scaled exponent stays below the maximum; otherwise (zero, subnormal,
// overflow, infinity, NaN) the FP64 multiplication, in a function of its own so that the
// compiler cannot evaluate it on the common path.  GB300 issues FP64 arithmetic at a small
// fraction of its FP32 rate, and the velocity correction is bound by it: this takes one FP64
// instruction per face off the pipe when h is a power of two.
__device__ __noinline__ double scale_mul(double v, double s) { return v * s; }
__device__ __forceinline__ double scale_pow2(double v, int m, double s) {
    const long long bits = __double_as_longlong(v);
    const int e = (int)((bits >> 52) & 0x7ff);
    if (e >= 1 && e + m <= 2046) return __longlong_as_double(bits + ((long long)m << 52));
    return scale_mul(v, s);
}

// One block per grid row (j, k) (grid (ny, nz), looping over k beyond the grid), the threads
// across the row; a thread owns the low faces of its cells (x, y, z), so every interior face
// is written exactly once.  FP64 arithmetic: the corrected velocity must keep the divergence
// of the solve's residual, far below FP32 rounding.  Out of place (o* may be u*): with
// COPY_WALLS the threads of the boundary cells also copy the wall faces from u to o.
// A thread takes kBatch (2) cells of its row at a time and loads all their inputs before the
// first store: the output may be the input (in place), so the compiler may not move a later
// cell's loads above an earlier cell's stores, and cell-by-cell the loads of each cell would
// wait a full memory latency.
constexpr int kBatch = 2;

template <bool CSF, bool COPY_WALLS, bool POW2>
__global__ void k_project(Dims d, double ih, int log2ih, double sigma, const double *__restrict__ p,
                          const double *__restrict__ fx, const double *__restrict__ fy,
                          const double *__restrict__ fz, const double *__restrict__ csx,
                          const double *__restrict__ csy, const double *__restrict__ csz, const double *ux,
                          const double *uy, const double *uz, double *ox, double *oy, double *oz) {
    const int nx = d.nx, ny = d.ny, nz = d.nz;
    const int j = blockIdx.x;
    const i64 nxy = d.nxy;
    for (int k = blockIdx.y; k < nz; k += gridDim.y) {
        const i64 row = (i64)k * ny + j;
        const i64 c0 = row * nx;
        const i64 ax0 = row * (nx + 1);                // x faces: (nz, ny, nx + 1)
        const i64 ay0 = ((i64)k * (ny + 1) + j) * nx;  // y faces: (nz, ny + 1, nx)
        const double *pr = p + c0;
        for (int i0 = threadIdx.x; i0 < nx; i0 += kBatch * blockDim.x) {
            double gxv[kBatch], gyv[kBatch], gzv[kBatch], bxv[kBatch], byv[kBatch], bzv[kBatch];
            double uxv[kBatch], uyv[kBatch], uzv[kBatch], cxv[kBatch], cyv[kBatch], czv[kBatch];
#pragma unroll
            for (int m = 0; m < kBatch; ++m) {
                const int i = i0 + m * blockDim.x;
                if (i >= nx) break;
                const i64 c = c0 + i;
                const double pc = pr[i];
                // dp across the low faces (0 where the face is a wall: not written)
                gxv[m] = i > 0 ? pc - pr[i - 1] : 0.0;
                gyv[m] = j > 0 ? pc - pr[i - nx] : 0.0;
                gzv[m] = k > 0 ? pc - p[c - nxy] : 0.0;
                bxv[m] = fx[c];
                byv[m] = fy[c];
                bzv[m] = fz[c];
                uxv[m] = ux[ax0 + i];
                uyv[m] = uy[ay0 + i];
                uzv[m] = uz[c];
                if (CSF) {
                    cxv[m] = csx[ax0 + i];
                    cyv[m] = csy[ay0 + i];
                    czv[m] = csz[c];
                }
            }
#pragma unroll
            for (int m = 0; m < kBatch; ++m) {
                const int i = i0 + m * blockDim.x;
                if (i >= nx) break;
                const i64 c = c0 + i;
                // u + beta (dp / h): with h a power of two as (beta / h) dp, the scaling exact,
                // so one rounding either way (the FMA)
                if (i > 0) {
                    if (CSF) ox[ax0 + i] = fma(bxv[m], fma(sigma, cxv[m], POW2 ? scale_pow2(gxv[m], log2ih, ih) : gxv[m] * ih), uxv[m]);
                    else if (POW2) ox[ax0 + i] = fma(scale_pow2(bxv[m], log2ih, ih), gxv[m], uxv[m]);
                    else ox[ax0 + i] = fma(bxv[m], gxv[m] * ih, uxv[m]);
                }
                if (j > 0) {
                    if (CSF) oy[ay0 + i] = fma(byv[m], fma(sigma, cyv[m], POW2 ? scale_pow2(gyv[m], log2ih, ih) : gyv[m] * ih), uyv[m]);
                    else if (POW2) oy[ay0 + i] = fma(scale_pow2(byv[m], log2ih, ih), gyv[m], uyv[m]);
                    else oy[ay0 + i] = fma(byv[m], gyv[m] * ih, uyv[m]);
                }
                if (k > 0) {
                    if (CSF) oz[c] = fma(bzv[m], fma(sigma, czv[m], POW2 ? scale_pow2(gzv[m], log2ih, ih) : gzv[m] * ih), uzv[m]);
                    else if (POW2) oz[c] = fma(scale_pow2(bzv[m], log2ih, ih), gzv[m], uzv[m]);
                    else oz[c] = fma(bzv[m], gzv[m] * ih, uzv[m]);
                }
                if (COPY_WALLS) {
                    if (i == 0) ox[ax0] = ux[ax0];
                    if (i == nx - 1) ox[ax0 + nx] = ux[ax0 + nx];
                    if (j == 0) oy[ay0 + i] = uyv[m];
                    if (j == ny - 1) oy[ay0 + i + nx] = uy[ay0 + i + nx];
                    if (k == 0) oz[c] = uzv[m];
                    if (k == nz - 1) oz[c + nxy] = uz[c + nxy];
                }
            }
        }
    }
}

// dL/drho and the fraction gradients.  The face gradients are FP32 (as mg_adjoint writes
// them), so the per-cell sum and the factor -1/(2 rho^2) run in FP32 and only the results
// are widened.  A density outside [2^-20, 2^21) takes the FP64 formula instead, so that
// 1/(2 rho^2) and its product with the gradient sum stay far inside the FP32 range.
struct FracOut {
    double *q[4];   // dL/df_q cell arrays (q < nfrac)
    float dr[4];    // rho_q - rho_last
};
__global__ void k_density_grads(Dims d, const double *__restrict__ rho, const float *__restrict__ gx,
                                const float *__restrict__ gy, const float *__restrict__ gz, double *drho,
                                int nfrac, FracOut fo) {
    const int nx = d.nx, ny = d.ny, nz = d.nz;
    const i64 nxy = d.nxy;
    const int j = blockIdx.x;  // grid (ny, nz) as for k_project
    for (int k = blockIdx.y; k < nz; k += gridDim.y) {
        const i64 row = (i64)k * ny + j;
        const i64 c0 = row * nx;
        const i64 ax0 = row * (nx + 1);
        const i64 ay0 = ((i64)k * (ny + 1) + j) * nx;
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const i64 c = c0 + i;
            float g = 0.f;
            if (i > 0) g += gx[ax0 + i];
            if (i < nx - 1) g += gx[ax0 + i + 1];
            if (j > 0) g += gy[ay0 + i];
            if (j < ny - 1) g += gy[ay0 + i + nx];
            if (k > 0) g += gz[c];
            if (k < nz - 1) g += gz[c + nxy];
            const double r = rho[c];
            double dd;
            float d32;
            // 2^-20 <= r < 2^21, tested on the high word (sign 0, biased exponent 1003 .. 1043)
            // so that no FP64 comparison reaches the FP64 pipe
            const unsigned rhi = (unsigned)__double2hiint(r);
            if (rhi >= (1003u << 20) && rhi < (1044u << 20)) {
                const float r32 = d2f_rn(r);
                d32 = -g * __frcp_rn(2.f * r32 * r32);
                dd = f2d_exact(d32);
            } else {
                dd = -(double)g / (2.0 * r * r);
                d32 = d2f_rn(dd);
            }
            drho[c] = dd;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < nfrac) fo.q[q][c] = f2d_exact(d32 * fo.dr[q]);
        }
    }
}

dim3 row_grid(Dims d) { return dim3((unsigned)d.ny, (unsigned)(d.nz < 65535 ? d.nz : 65535)); }

int row_threads(Dims d) { return d.nx >= 256 ? 128 : (d.nx >= 128 ? 128 : (d.nx > 32 ? 64 : 32)); }

}  // namespace

void launch_project(cudaStream_t s, Dims d, double h, const double *p, const double *fx, const double *fy,
                    const double *fz, const double *csfx, const double *csfy, const double *csfz, double sigma,
                    const double *ux, const double *uy, const double *uz, double *ox, double *oy, double *oz) {
    const bool copy = !(ox == ux && oy == uy && oz == uz);
    const double ih = 1.0 / h;
    int ex = 0;
    const int log2ih = (std::frexp(ih, &ex) == 0.5 && ex - 1 >= 0 && ex - 1 < 1000) ? ex - 1 : -1;
    const dim3 nb = row_grid(d);
    const int nt = row_threads(d);
    count_launch();
    if (csfx) {
        if (copy && log2ih >= 0)
            k_project<true, true, true><<<nb, nt, 0, s>>>(d, ih, log2ih, sigma, p, fx, fy, fz, csfx, csfy, csfz, ux,
                                                          uy, uz, ox, oy, oz);
        else if (log2ih >= 0)
            k_project<true, false, true><<<nb, nt, 0, s>>>(d, ih, log2ih, sigma, p, fx, fy, fz, csfx, csfy, csfz, ux,
                                                           uy, uz, ox, oy, oz);
        else if (copy)
            k_project<true, true, false><<<nb, nt, 0, s>>>(d, ih, log2ih, sigma, p, fx, fy, fz, csfx, csfy, csfz, ux,
                                                           uy, uz, ox, oy, oz);
        else
            k_project<true, false, false><<<nb, nt, 0, s>>>(d, ih, log2ih, sigma, p, fx, fy, fz, csfx, csfy, csfz, ux,
                                                            uy, uz, ox, oy, oz);
    } else if (log2ih >= 0) {
        if (copy)
            k_project<false, true, true><<<nb, nt, 0, s>>>(d, ih, log2ih, 0.0, p, fx, fy, fz, nullptr, nullptr,
                                                           nullptr, ux, uy, uz, ox, oy, oz);
        else
            k_project<false, false, true><<<nb, nt, 0, s>>>(d, ih, log2ih, 0.0, p, fx, fy, fz, nullptr, nullptr,
                                                            nullptr, ux, uy, uz, ox, oy, oz);
    } else {
        if (copy)
            k_project<false, true, false><<<nb, nt, 0, s>>>(d, ih, log2ih, 0.0, p, fx, fy, fz, nullptr, nullptr,
                                                            nullptr, ux, uy, uz, ox, oy, oz);
        else
            k_project<false, false, false><<<nb, nt, 0, s>>>(d, ih, log2ih, 0.0, p, fx, fy, fz, nullptr, nullptr,
                                                             nullptr, ux, uy, uz, ox, oy, oz);
    }
}

void launch_density_grads(cudaStream_t s, Dims d, const double *rho, const float *gx, const float *gy,
                          const float *gz, double *drho, int nfrac, const double *rho_phase,
                          double *const *dfrac) {
    FracOut fo;
    for (int q = 0; q < 4; ++q) {
        fo.q[q] = q < nfrac ? dfrac[q] : nullptr;
        fo.dr[q] = q < nfrac ? (float)(rho_phase[q] - rho_phase[nfrac]) : 0.f;
    }
    count_launch();
    k_density_grads<<<row_grid(d), row_threads(d), 0, s>>>(d, rho, gx, gy, gz, drho, nfrac, fo);
}

}  // namespace mg
