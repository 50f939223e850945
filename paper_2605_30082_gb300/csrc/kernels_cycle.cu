// V-cycle kernels of the FP64 path on one level (natural layout): the red-black half sweep,
// operator application, residual, residual + 8:1 restriction, prolongation + correction,
// and the dense coarse solve.  Templated on the element type; the FP32 inner cycle of the
// mixed modes uses the colour-split kernels of kernels_split.cu instead.
//
// Operator (cell-centred, homogeneous Neumann walls):
//   (A x)_c = ih2 * sum_{interior faces f of c} beta_f (x_c - x_nb(f))
// Restriction: coarse b = mean of the 8 children of the fine residual.
// Prolongation: cell-centred trilinear (weights 3/4, 1/4 per axis; at a wall
// the missing coarse neighbour is replaced by the parent) or constant.
#include "mg_internal.cuh"

namespace mg {

namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(i64 n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// (i, j, k) of cell c; cells number at most 2e9 < 2^32, so 32-bit divisions (64-bit ones cost
// several times as many instructions)
__device__ __forceinline__ void cell_ijk(const Dims &d, i64 c, int &i, int &j, int &k) {
    const unsigned cu = (unsigned)c, r = cu / (unsigned)d.nx;
    i = (int)(cu - r * (unsigned)d.nx);
    j = (int)(r % (unsigned)d.ny);
    k = (int)(r / (unsigned)d.ny);
}

// sum_f beta_f x_nb in the order x-, x+, y-, y+, z-, z+
template <typename T>
__device__ __forceinline__ T nb_sum(const Dims &d, int i, int j, int k, i64 c, const Coef<T> &cf,
                                    const T *__restrict__ x) {
    T s = T(0);
    if (i > 0) s += cf.fx[c] * x[c - 1];
    if (i < d.nx - 1) s += cf.fx[c + 1] * x[c + 1];
    if (j > 0) s += cf.fy[c] * x[c - d.nx];
    if (j < d.ny - 1) s += cf.fy[c + d.nx] * x[c + d.nx];
    if (k > 0 || d.zlo) s += cf.fz[c] * x[c - d.nxy];
    if (k < d.nz - 1 || d.zhi) s += cf.fz[c + d.nxy] * x[c + d.nxy];
    return s;
}

// sum_f beta_f (x_c - x_nb), same order
template <typename T>
__device__ __forceinline__ T flux_sum(const Dims &d, int i, int j, int k, i64 c, const Coef<T> &cf,
                                      const T *__restrict__ x) {
    T xc = x[c];
    T s = T(0);
    if (i > 0) s += cf.fx[c] * (xc - x[c - 1]);
    if (i < d.nx - 1) s += cf.fx[c + 1] * (xc - x[c + 1]);
    if (j > 0) s += cf.fy[c] * (xc - x[c - d.nx]);
    if (j < d.ny - 1) s += cf.fy[c + d.nx] * (xc - x[c + d.nx]);
    if (k > 0 || d.zlo) s += cf.fz[c] * (xc - x[c - d.nxy]);
    if (k < d.nz - 1 || d.zhi) s += cf.fz[c + d.nxy] * (xc - x[c + d.nxy]);
    return s;
}

// red-black Gauss-Seidel half sweep of colour q ((i+j+k) % 2 == q), in place:
//   x_c = (h2 b_c + sum_f beta_f x_nb) * invd_c   (invd = 1 / sum_f beta_f)
// one thread per cell of the colour; used by the FP64 V-cycle, whose cost is
// FP64 arithmetic rather than bytes, so it keeps zero redundant work
template <typename T>
__global__ void k_rbgs_half(Dims d, T h2, Coef<T> cf, const T *__restrict__ b, T *x, int colour) {
    const int half = (d.nx + 1) >> 1;
    const i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    const i64 rows = (i64)d.ny * d.nz;
    if (t >= rows * half) return;
    const unsigned tu = (unsigned)t, rowu = tu / (unsigned)half;  // t < 2^31: 32-bit divisions
    const i64 row = rowu;
    const int m = (int)(tu - rowu * (unsigned)half);
    const int j = (int)(rowu % (unsigned)d.ny), k = (int)(rowu / (unsigned)d.ny);
    const int i = 2 * m + ((colour + j + k) & 1);
    if (i >= d.nx) return;
    const i64 c = row * d.nx + i;
    const T num = nb_sum(d, i, j, k, c, cf, x);
    x[c] = (h2 * b[c] + num) * cf.invd[c];
}

template <typename T>
__global__ void k_apply(Dims d, T ih2, Coef<T> cf, const T *__restrict__ x, T *y) {
    i64 c = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.n) return;
    int i, j, k;
    cell_ijk(d, c, i, j, k);
    y[c] = flux_sum(d, i, j, k, c, cf, x) * ih2;
}

template <typename T>
__global__ void k_residual(Dims d, T ih2, Coef<T> cf, const T *__restrict__ b,
                           const T *__restrict__ x, T *r) {
    i64 c = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.n) return;
    int i, j, k;
    cell_ijk(d, c, i, j, k);
    r[c] = b[c] - flux_sum(d, i, j, k, c, cf, x) * ih2;
}

// one thread per coarse cell: mean of the residuals of its 8 children; red_only: the black
// children count as 0 (exact after a black half sweep, which solves every black row)
template <typename T>
__global__ void k_resid_restrict(Dims f, Dims cd, T ih2, Coef<T> cf, const T *__restrict__ b,
                                 const T *__restrict__ x, T *bc, int red_only) {
    i64 C = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (C >= cd.n) return;
    int I, J, K;
    cell_ijk(cd, C, I, J, K);
    T s = T(0);
    for (int cc = 0; cc < 2; ++cc)
        for (int bb = 0; bb < 2; ++bb)
            for (int aa = 0; aa < 2; ++aa) {
                int i = 2 * I + aa, j = 2 * J + bb, k = 2 * K + cc;
                if (red_only && ((i + j + k) & 1)) continue;
                i64 c = ((i64)k * f.ny + j) * f.nx + i;
                s += b[c] - flux_sum(f, i, j, k, c, cf, x) * ih2;
            }
    bc[C] = s / T(8);
}

// e += P ec on the cells of colour only_col (0 red, 1 black) or on all cells (-1)
template <typename T>
__global__ void k_prolong(Dims cd, Dims f, const T *__restrict__ ec, T *e, int kind, int only_col) {
    i64 c = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= f.n) return;
    int i, j, k;
    cell_ijk(f, c, i, j, k);
    if (only_col >= 0 && ((i + j + k) & 1) != only_col) return;
    int I = i >> 1, J = j >> 1, K = k >> 1;
    T v;
    if (kind == MG_PROLONG_CONSTANT) {
        v = ec[((i64)K * cd.ny + J) * cd.nx + I];
    } else {
        int I2 = (i & 1) ? I + 1 : I - 1;
        int J2 = (j & 1) ? J + 1 : J - 1;
        int K2 = (k & 1) ? K + 1 : K - 1;
        if (I2 < 0 || I2 >= cd.nx) I2 = I;
        if (J2 < 0 || J2 >= cd.ny) J2 = J;
        if ((K2 < 0 && !cd.zlo) || (K2 >= cd.nz && !cd.zhi)) K2 = K;  // a slab's ghost plane counts
        const T w[2] = {T(0.75), T(0.25)};
        int Ii[2] = {I, I2}, Jj[2] = {J, J2}, Kk[2] = {K, K2};
        v = T(0);
#pragma unroll
        for (int cc = 0; cc < 2; ++cc)
#pragma unroll
            for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                for (int aa = 0; aa < 2; ++aa)
                    v += w[aa] * w[bb] * w[cc] * ec[((i64)Kk[cc] * cd.ny + Jj[bb]) * cd.nx + Ii[aa]];
    }
    e[c] += v;
}

// e = pinv r, one warp per row, FP64 accumulation
// Red-only residual + restriction in diagonal form on a level with the diagonal d = sum beta:
//   h^2 r_c = h^2 b_c + sum_f beta_f x_nb - d_c x_c   (7 FMA and one multiply per red child),
// coarse b = ih2/8 * (sum over the 4 red children).  Blocks take coarse rows (grid y, strided),
// threads coarse I: no 64-bit division per cell.
__global__ void k_rr_red_diag64(Dims f, Dims cd, double h2, double ih2_8, Coef<double> cf,
                                const double *__restrict__ dg, const double *__restrict__ b,
                                const double *__restrict__ x, double *bc) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= cd.nx) return;
    const i64 crows = (i64)cd.ny * cd.nz;
    for (i64 cr = blockIdx.y; cr < crows; cr += gridDim.y) {
        const int J = (int)(cr % cd.ny), K = (int)(cr / cd.ny);
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = 2 * J + (q & 1), k = 2 * K + (q >> 1);
            const int i = 2 * I + ((j + k) & 1);  // the red child in this fine row
            const i64 c = ((i64)k * f.ny + j) * f.nx + i;
            double a = h2 * b[c];
            if (i > 0) a = fma(cf.fx[c], x[c - 1], a);
            if (i < f.nx - 1) a = fma(cf.fx[c + 1], x[c + 1], a);
            if (j > 0) a = fma(cf.fy[c], x[c - f.nx], a);
            if (j < f.ny - 1) a = fma(cf.fy[c + f.nx], x[c + f.nx], a);
            if (k > 0 || f.zlo) a = fma(cf.fz[c], x[c - f.nxy], a);
            if (k < f.nz - 1 || f.zhi) a = fma(cf.fz[c + f.nxy], x[c + f.nxy], a);
            s += fma(-dg[c], x[c], a);
        }
        bc[(i64)cr * cd.nx + I] = s * ih2_8;
    }
}

// x += P ec on the cells of one colour only; threads take the cells of that colour in a row
// (grid x), blocks strided rows (grid y)
template <typename T>
__global__ void k_prolong_col(Dims cd, Dims f, const T *__restrict__ ec, T *e, int kind, int col) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const i64 rows = (i64)f.ny * f.nz;
    for (i64 row = blockIdx.y; row < rows; row += gridDim.y) {
        const int j = (int)((unsigned)row % (unsigned)f.ny), k = (int)((unsigned)row / (unsigned)f.ny);
        const int i = 2 * m + ((col + j + k) & 1);
        if (i >= f.nx) continue;
        const int I = i >> 1, J = j >> 1, K = k >> 1;
        T v;
        if (kind == MG_PROLONG_CONSTANT) {
            v = ec[((i64)K * cd.ny + J) * cd.nx + I];
        } else {
            int I2 = (i & 1) ? I + 1 : I - 1;
            int J2 = (j & 1) ? J + 1 : J - 1;
            int K2 = (k & 1) ? K + 1 : K - 1;
            if (I2 < 0 || I2 >= cd.nx) I2 = I;
            if (J2 < 0 || J2 >= cd.ny) J2 = J;
            if ((K2 < 0 && !cd.zlo) || (K2 >= cd.nz && !cd.zhi)) K2 = K;  // a slab's ghost plane counts
            const T w[2] = {T(0.75), T(0.25)};
            const int Ii[2] = {I, I2}, Jj[2] = {J, J2}, Kk[2] = {K, K2};
            v = T(0);
#pragma unroll
            for (int cc = 0; cc < 2; ++cc)
#pragma unroll
                for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                    for (int aa = 0; aa < 2; ++aa)
                        v += w[aa] * w[bb] * w[cc] * ec[((i64)Kk[cc] * cd.ny + Jj[bb]) * cd.nx + Ii[aa]];
        }
        e[row * f.nx + i] += v;
    }
}

template <typename T>
__global__ void k_coarse_matvec(int nc, const double *__restrict__ pinv, const T *__restrict__ r,
                                T *e) {
    int row = (int)(((i64)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    int lane = threadIdx.x & 31;
    if (row >= nc) return;
    const double *a = pinv + (i64)row * nc;
    double s = 0.0;
    for (int q = lane; q < nc; q += 32) s += a[q] * (double)r[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) e[row] = (T)s;
}

}  // namespace

void launch_rbgs_half64(cudaStream_t s, Dims d, double h2, Coef<double> c, const double *b, double *p,
                        int colour) {
    const i64 work = (i64)d.ny * d.nz * ((d.nx + 1) / 2);
    count_launch();
    k_rbgs_half<double><<<blocks_for(work), kThreads, 0, s>>>(d, h2, c, b, p, colour);
}

template <typename T>
void launch_apply(cudaStream_t s, Dims d, double ih2, Coef<T> c, const T *x, T *y) {
    count_launch();
    k_apply<T><<<blocks_for(d.n), kThreads, 0, s>>>(d, (T)ih2, c, x, y);
}

template <typename T>
void launch_residual(cudaStream_t s, Dims d, double ih2, Coef<T> c, const T *b, const T *x, T *r) {
    count_launch();
    k_residual<T><<<blocks_for(d.n), kThreads, 0, s>>>(d, (T)ih2, c, b, x, r);
}

template <typename T>
void launch_resid_restrict(cudaStream_t s, Dims fine, double ih2, Coef<T> c, const T *b,
                           const T *x, T *bc, bool red_only) {
    Dims cd = make_dims(fine.nx / 2, fine.ny / 2, fine.nz / 2);
    count_launch();
    k_resid_restrict<T><<<blocks_for(cd.n), kThreads, 0, s>>>(fine, cd, (T)ih2, c, b, x, bc, red_only ? 1 : 0);
}

template <typename T>
void launch_prolong(cudaStream_t s, Dims coarse, const T *ec, T *e, int kind, int only_col) {
    Dims f = make_dims(coarse.nx * 2, coarse.ny * 2, coarse.nz * 2);
    count_launch();
    if (only_col >= 0) {
        const unsigned gx = (unsigned)(((f.nx + 1) / 2 + 127) / 128);
        const i64 rows = (i64)f.ny * f.nz;
        const unsigned gy = (unsigned)(rows < 65535 ? rows : 65535);
        k_prolong_col<T><<<dim3(gx, gy), 128, 0, s>>>(coarse, f, ec, e, kind, only_col);
        return;
    }
    k_prolong<T><<<blocks_for(f.n), kThreads, 0, s>>>(coarse, f, ec, e, kind, only_col);
}

void launch_rr_red_diag64(cudaStream_t s, Dims fine, double h2, Coef<double> c, const double *dg,
                          const double *b, const double *x, double *bc) {
    Dims cd = make_dims(fine.nx / 2, fine.ny / 2, fine.nz / 2);
    count_launch();
    const unsigned gx = (unsigned)((cd.nx + 127) / 128);
    const i64 crows = (i64)cd.ny * cd.nz;
    const unsigned gy = (unsigned)(crows < 65535 ? crows : 65535);
    k_rr_red_diag64<<<dim3(gx, gy), 128, 0, s>>>(fine, cd, h2, 1.0 / (8.0 * h2), c, dg, b, x, bc);
}

template <typename T>
void launch_coarse_matvec(cudaStream_t s, int nc, const double *pinv, const T *r, T *e) {
    i64 threads = (i64)nc * 32;
    count_launch();
    k_coarse_matvec<T><<<blocks_for(threads), kThreads, 0, s>>>(nc, pinv, r, e);
}

#define MG_INSTANTIATE(T)                                                                        \
    template void launch_apply<T>(cudaStream_t, Dims, double, Coef<T>, const T *, T *);          \
    template void launch_residual<T>(cudaStream_t, Dims, double, Coef<T>, const T *, const T *,  \
                                     T *);                                                       \
    template void launch_resid_restrict<T>(cudaStream_t, Dims, double, Coef<T>, const T *,       \
                                           const T *, T *, bool);                                \
    template void launch_prolong<T>(cudaStream_t, Dims, const T *, T *, int, int);               \
    template void launch_coarse_matvec<T>(cudaStream_t, int, const double *, const T *, T *);

MG_INSTANTIATE(double)
MG_INSTANTIATE(float)
#undef MG_INSTANTIATE

}  // namespace mg
