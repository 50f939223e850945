// Unfused V-cycle kernels on one level: the FP64 red-black half sweep,
// operator application, residual, residual + 8:1 restriction, prolongation +
// correction, and the dense coarse solve.  (The FP32 sweeps, with restriction
// or prolongation fused in, are the z-marching passes of kernels_pass.cu.)  Templated on the level's element
// type (double for the FP64 path, float for the inner cycle of MIXED).
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

__device__ __forceinline__ void cell_ijk(const Dims &d, i64 c, int &i, int &j, int &k) {
    i = (int)(c % d.nx);
    i64 r = c / d.nx;
    j = (int)(r % d.ny);
    k = (int)(r / d.ny);
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
    if (k > 0) s += cf.fz[c] * x[c - d.nxy];
    if (k < d.nz - 1) s += cf.fz[c + d.nxy] * x[c + d.nxy];
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
    if (k > 0) s += cf.fz[c] * (xc - x[c - d.nxy]);
    if (k < d.nz - 1) s += cf.fz[c + d.nxy] * (xc - x[c + d.nxy]);
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
    const i64 row = t / half;
    const int m = (int)(t - row * half);
    const int j = (int)(row % d.ny), k = (int)(row / d.ny);
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
        if (K2 < 0 || K2 >= cd.nz) K2 = K;
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
    k_prolong<T><<<blocks_for(f.n), kThreads, 0, s>>>(coarse, f, ec, e, kind, only_col);
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
