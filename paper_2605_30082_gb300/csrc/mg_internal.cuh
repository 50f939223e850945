// Internal declarations of the GB300 multigrid Poisson library (not part of the ABI).
//
// Storage inside the library.  Every per-level array is a cell array of the
// level's shape (nz, ny, nx), x fastest.  Face coefficients are kept as three
// cell arrays of LOW faces: fx[c] is the coefficient of the face between cell
// c and its x-1 neighbour (0 for i = 0, the wall); the high face of c is the
// low face of its x+1 neighbour, or the wall (0) when i = nx-1.  The ABI's
// (n+1)-long face layouts are converted on entry and exit.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mg.h"

namespace mg {

typedef long long i64;

struct Dims {
    int nx, ny, nz;
    i64 nxy, n;
    // z slab of a domain-decomposed level (mg_dd.cu): a ghost plane below (zlo) or above (zhi)
    // the nz own planes holds the neighbouring slab's values, so the faces between slabs count
    // as interior; 0 on every whole-grid level (the walls)
    int zlo, zhi;
};

inline Dims make_dims(int nx, int ny, int nz) {
    Dims d;
    d.nx = nx;
    d.ny = ny;
    d.nz = nz;
    d.nxy = (i64)nx * ny;
    d.n = d.nxy * nz;
    d.zlo = d.zhi = 0;
    return d;
}

// Storage layout of an FP32 level: colour-split (all red cells, then all black, each
// colour row by row, cell x of a row at k = x >> 1) when nx is even, else natural.
// A z slab of a decomposed level (mg_dd.cu, split layout only) keeps a ghost plane below and
// above its nz own planes in each colour half: `half` is then the stride between the two
// halves (nz + 2 planes each), the arrays point at the red half's first own plane, and zlo /
// zhi say whether the ghost below / above holds a neighbour's values (the planes between
// slabs count as interior) or is a wall; the slab starts at an even whole-grid plane, so the
// colour of a cell is the same as on the whole grid.
struct Lay {
    int nx, ny, nz;
    i64 n;
    bool split;
    int hx;     // nx / 2
    i64 half;   // n / 2 (a slab: the colour stride)
    int zlo, zhi;
};
Lay make_lay(Dims d);

template <typename T>
struct Coef {
    const T *fx, *fy, *fz;  // low-face coefficients
    const T *invd;          // 1 / sum of the cell's interior face coefficients (FP64 only)
};

#ifdef __CUDACC__
// ---- IEEE-754 conversions and the FP64 reciprocal, with few FP64-pipe instructions --------
// GB300 runs FP64 arithmetic and FP64<->FP32 conversions at a small fraction of its FP32
// rate, so the hot kernels convert by integer operations on the IEEE-754 fields
// (binary64: 1 sign, 11 exponent (bias 1023), 52 fraction bits; binary32: 1, 8 (bias 127), 23).

// FP64 -> FP32 by truncating the IEEE-754 fields with integer operations (the
// binary64 layout: 1 sign, 11 exponent (bias 1023), 52 fraction bits; binary32:
// 1, 8 (bias 127), 23).  Rounds toward zero; results below the FP32 normal range
// become zero, above it infinity; NaN stays NaN.  Keeps the conversion off the
// FP64 pipe, which GB300 runs at a small fraction of the FP32 rate.
__device__ __forceinline__ float d2f_trunc(double v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const unsigned hi = (unsigned)(u >> 32);
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu);
    const unsigned frac = (unsigned)((u >> 29) & 0x7fffffu);
    if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (frac ? 0x400000u : 0u));
    const int e32 = e - 1023 + 127;
    if (e32 <= 0) return __uint_as_float(sign);
    if (e32 >= 255) return __uint_as_float(sign | 0x7f800000u);
    return __uint_as_float(sign | ((unsigned)e32 << 23) | frac);
}

// FP32 -> FP64 exactly with integer operations (FP32 subnormals become zero)
__device__ __forceinline__ double f2d_exact(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned sign = u & 0x80000000u;
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned m = u & 0x7fffffu;
    if (e == 0) return __hiloint2double((int)sign, 0);
    const unsigned ed = (e == 0xffu) ? 0x7ffu : (e - 127u + 1023u);
    return __hiloint2double((int)(sign | (ed << 20) | (m >> 3)), (int)(m << 29));
}

// FP64 -> FP32 rounded to nearest, ties to even, with integer operations on the IEEE-754
// fields: the 29 dropped fraction bits decide the rounding; a carry out of the fraction
// increments the exponent (up to infinity).  Results below the FP32 normal range become
// (signed) zero; NaN stays NaN.
__device__ __forceinline__ float d2f_rn(double v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const unsigned hi = (unsigned)(u >> 32);
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu);
    const unsigned frac = (unsigned)((u >> 29) & 0x7fffffu);
    if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (((u << 12) != 0ull) ? 0x400000u : 0u));
    const int e32 = e - 1023 + 127;
    if (e32 <= 0) return __uint_as_float(sign);
    if (e32 >= 255) return __uint_as_float(sign | 0x7f800000u);
    const unsigned rest = (unsigned)(u & 0x1fffffffull);  // the 29 dropped bits
    const unsigned up = (rest > 0x10000000u || (rest == 0x10000000u && (frac & 1u))) ? 1u : 0u;
    const unsigned mag = ((unsigned)e32 << 23) + frac + up;  // a carry moves into the exponent
    return __uint_as_float(sign | (mag >= 0x7f800000u ? 0x7f800000u : mag));
}

// 1 / x for positive x.  Seed: the FP32 reciprocal (round to nearest) of x rounded to FP32,
// relative error <= 2^-23; then two Newton-Raphson steps y <- y + y (1 - x y) in FP64, each
// squaring the relative error (2^-46, then below FP64 rounding), so the result is within one
// unit in the last place of 1/x.  Outside [2^-100, 2^100] (where the FP32 seed could leave
// the FP32 range) it divides.
__device__ __forceinline__ double recip64(double x) {
    // the range test on the bit pattern (positive doubles order like their bits): no FP64
    // comparison on the FP64 pipe
    const long long xb = __double_as_longlong(x);
    if (!(xb >= 0x39b0000000000000ll && xb <= 0x4630000000000000ll)) return 1.0 / x;
    double y = f2d_exact(__frcp_rn(d2f_rn(x)));
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}
#endif

// process-wide count of kernel launches (read through mg_kernel_launches)
void count_launch(int k = 1);
unsigned long long launches_total();

// the stream a handle queues its work on, replaced by `s`; returns the previous one (the
// decomposed solver records its cycle, the whole-grid handle's launches included, on a
// private stream)
cudaStream_t swap_handle_stream(mg_handle *h, cudaStream_t s);

// A mixed-precision handle's FP32 level l, for the decomposed mixed cycle (mg_dd.cu), which
// runs the levels from its switch level down on a whole-grid handle: the level's storage layout,
// its right-hand side and iterate arrays, and one FP32 V-cycle of the handle from level l down
// (from x = 0, on that level's b32, into its x32; the handle's options and recorded tail, or,
// `recording` under a stream capture, the tail's launches one by one)
Lay handle_lay32(mg_handle *h, int l);
float *handle_b32(mg_handle *h, int l);
float *handle_x32(mg_handle *h, int l);
void handle_vcycle32(mg_handle *h, int l, bool recording = false);
// the adaptive inner-cycle count of the mixed outer loop: the first, and the next from the
// contraction of the last outer iteration (k cycles from relres rr_prev to rr)
int handle_first_inner();
int handle_next_inner(double rr_prev, double rr, int k, double rtol);

// NVTX range for the lifetime of the object: a profiler attached to the process (Nsight
// Systems, ncu --nvtx) sees each entry point as one named range; without one the calls do
// nothing (header-only NVTX3, which looks up a tool only when one is injected)
struct NvtxRange {
    explicit NvtxRange(const char *name);
    ~NvtxRange();
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// the most blocks a deterministic reduction over n elements uses (its partials buffer holds
// that many pairs); launchers take min(this, one wave of the kernel)
int reduce_blocks(i64 n);
// streaming multiprocessors of the current device (queried once per device; 152 on GB300)
int device_sms();
constexpr int kReduceThreads = 256;
// blocks of one full wave of `kernel` at `threads` threads per block on the current device
// (resident blocks per SM x SMs; 2^30 if the query fails).  Launchers cache it in a function-
// local static: every device a process uses is of the same model.
int wave_blocks(const void *kernel, int threads);
// min(nb, wave): the grid of a grid-stride reduction that needs nb <= reduce_blocks(n) blocks
int fill_blocks(int nb, int wave);

// ---- setup kernels (FP64) -------------------------------------------------------
void launch_density(cudaStream_t s, i64 n, int nfrac, const double *const *frac,
                    const double *rho_phase, double *rho);
// s = 1/rho per cell into `sinv` (validated: err |= 1 on a bad density), then the FP64 low faces
void launch_faces_from_rho(cudaStream_t s, Dims d, const double *rho, double *sinv, double *fx, double *fy,
                           double *fz, unsigned *err);
void launch_faces_from_api(cudaStream_t s, Dims d, const double *bx, const double *by,
                           const double *bz, double *fx, double *fy, double *fz, unsigned *err);
void launch_faces_to_api(cudaStream_t s, Dims d, const double *fx, const double *fy,
                         const double *fz, double *bx, double *by, double *bz);
// 1 / sum of the interior face coefficients of each cell, and (diag non-null) the sum itself
void launch_invdiag(cudaStream_t s, Dims d, const double *fx, const double *fy, const double *fz,
                    double *invd64, double *diag);
void launch_coarsen(cudaStream_t s, Dims fine, const double *ffx, const double *ffy,
                    const double *ffz, double *cfx, double *cfy, double *cfz);
void launch_to_f32(cudaStream_t s, i64 n, const double *src, float *dst);

void launch_csf_faces(cudaStream_t s, Dims d, double h, const double *f, const double *kappa,
                      double *cx, double *cy, double *cz);
void launch_rhs(cudaStream_t s, Dims d, double h, const double *b0, const double *ux, const double *uy,
                const double *uz, const double *fx, const double *fy, const double *fz,
                const double *csfx, const double *csfy, const double *csfz, double sigma,
                double *b);
// dense coarse inverse (Gauss-Jordan on A_c + c 1 1^T, then minus 1/(c n^2))
void launch_coarse_assemble(cudaStream_t s, Dims d, double ih2, const double *fx, const double *fy,
                            const double *fz, double *M, double *scal);
// Gauss-Jordan inversion in place by blocks of kGjBlock pivots (scratch: kGjBlock x kGjBlock
// doubles, the inverse of the current pivot block)
constexpr int kGjBlock = 32;
void launch_gj_blocked(cudaStream_t s, int nc, double *M, double *scratch);
void launch_pinv_finish(cudaStream_t s, int nc, double *M, const double *scal);

// ---- V-cycle kernels --------------------------------------------------------------
// ---- FP32 colour-split level kernels (kernels_split.cu) ----
// half sweep of colour col in place; sinv = 1/rho per cell (beta = (s_L + s_R)/2) when
// non-null, else the low-face arrays; from_zero: the other colour is taken as zero.
// On a slab (L.zlo / L.zhi; see Lay) the V-cycle kernels take its ghost planes as z
// neighbours: split layout with hx % 4 == 0, s-form or face form (fz with its ghost plane
// above: the face to the neighbour above), restriction of red residuals only, trilinear
// prolongation of the red cells from a coarse slab or view (Lc.zlo / Lc.zhi) whose nx is a
// multiple of 8; other cases are not supported on slabs
void launch_half32(cudaStream_t s, Lay L, double h2, const float *sinv, const float *fx, const float *fy,
                   const float *fz, const float *b, float *x, int col, bool from_zero);
// the last red half sweep of the finest level with the outer update fused in: the new red
// values and the black values of the same row positions (x, split, level 0) go straight
// into p = (p - shift) + alpha * x (p natural FP64); x itself is not written.
// Needs a split layout with hx % 4 == 0 (half32_update_ok).
bool half32_update_ok(Lay L);
// p2 non-null: the double-float solution is updated instead of p
void launch_half32_update(cudaStream_t s, Lay L, double h2, const float *sinv, const float *fx, const float *fy,
                          const float *fz, const float *b, const float *x, double *p, float2 *p2, double alpha,
                          double shift);

// ---- fused red-black sweep of the finest level (kernels_fused.cu) ----
// s-form split level with hx % 64 == 0: one sweep, colour c1 first, reading x from X and
// writing both colours to Y (X != Y); from_zero: X is not read (x = 0).  With p non-null the
// second colour's new values and the first colour's go into p = (p - shift) + alpha x (natural
// FP64) instead of Y.  A bounded wait that runs out sets bit 4 of *err.  inject_wait (tests
// only): one block issues no copies for one plane, so that its wait runs out.
bool sweep_fused_ok(Lay L);
void launch_sweep_fused(cudaStream_t s, Lay L, double h2, const float *sinv, const float *b, const float *X,
                        float *Y, int c1, bool from_zero, double *p, double alpha, double shift, unsigned *err,
                        bool inject_wait = false);

// ---- MG_MIXED_DF outer loop (kernels_df.cu): double-float (hi, lo) FP32 pairs ----
void launch_split(cudaStream_t s, i64 n, const double *src, float2 *dst);   // hi = fl32(v), lo = fl32(v - hi)
void launch_join(cudaStream_t s, i64 n, const float2 *src, double *dst);    // v = hi + lo in FP64
// h^2 r = b + sum_f beta_f p_nb - d p_c (b scaled by h^2); out[0] = sum (h^2 r)^2, out[1] = sum p;
// optional r32 = s32 * h^2 r in the split level-0 layout.  Needs even nx.
void launch_resid_df(cudaStream_t s, Dims d, Lay L, const float2 *fx, const float2 *fy, const float2 *fz,
                     const float2 *diag, const float2 *b, const float2 *p, float *r32, float s32,
                     double *partials, double *out);
// s-form double-float residual: s2 = 1/rho as FP32 pairs (natural layout), otherwise as launch_resid_df
void launch_resid_dfs(cudaStream_t s, Dims d, Lay L, const float2 *s2, const float2 *b, const float2 *p,
                      float *r32, float s32, double *partials, double *out);
// ---- flexible CG (kernels_cg.cu) --------------------------------------------------------
// slots of the device scalar array: r . z of the current and of the previous iteration
// alternate between CG_RZ0 and CG_RZ1
enum { CG_RZ0 = 0, CG_PQ = 1, CG_ALPHA = 2, CG_ZQ = 3, CG_RZ1 = 4, CG_RR = 5, CG_SX = 6, CG_NSLOT = 8 };
void launch_cg_apply32(cudaStream_t s, Lay L, double ih2, const float *sinv, const float *fx, const float *fy,
                       const float *fz, const float *d, float *q, double *partials, double *sc);
void launch_cg_dots32(cudaStream_t s, i64 n, const float *r, const float *z, const float *q, double *partials,
                      double *sc, int rz_slot);
void launch_cg_dir32(cudaStream_t s, i64 n, const float *z, float *d, const double *sc, bool first, int rz_prev);
void launch_cg_update32(cudaStream_t s, i64 n, float *x, float *r, const float *d, const float *q, double *sc,
                        int rz_cur);
void launch_cg_apply64(cudaStream_t s, Dims d, double ih2, const double *fx, const double *fy, const double *fz,
                       const double *dg, const double *dv, double *q, double *partials, double *sc);
void launch_cg_dots64(cudaStream_t s, i64 n, const double *r, const double *z, const double *q, double *partials,
                      double *sc, int rz_slot);
void launch_cg_dir64(cudaStream_t s, i64 n, const double *z, double *d, const double *sc, bool first, int rz_prev);
void launch_cg_update64(cudaStream_t s, i64 n, double *x, double *r, const double *d, const double *q, double *sc,
                        int rz_cur, double *partials);

void launch_update_df(cudaStream_t s, Dims d, Lay L, float2 *p, const float *e32, double alpha, double shift);
// r = b - A x (or r = A x when apply_only)
void launch_residual32(cudaStream_t s, Lay L, double ih2, const float *sinv, const float *fx, const float *fy,
                       const float *fz, const float *b, const float *x, float *r, bool apply_only);
// bc = mean of the 8 children's residuals (red_only: black children count as 0)
void launch_resid_restrict32(cudaStream_t s, Lay L, Lay Lc, double ih2, const float *sinv, const float *fx,
                             const float *fy, const float *fz, const float *b, const float *x, float *bc,
                             bool red_only);
// x += P ec on the cells of colour only_col (0 red, 1 black) or all cells (-1)
void launch_prolong32(cudaStream_t s, Lay L, Lay Lc, const float *ec, float *x, int kind, int only_col);
void launch_coarse_matvec32(cudaStream_t s, Lay L, const double *pinv, const float *r, float *e);
void launch_pack32(cudaStream_t s, Lay L, const float *nat, float *st);
void launch_unpack32(cudaStream_t s, Lay L, const float *st, float *nat);
void launch_pack64to32(cudaStream_t s, Lay L, const double *nat, float *st);
// s (FP64, natural) -> FP32 in the level layout, and optionally FP32 pairs (natural)
void launch_pack_inv_rho(cudaStream_t s, Lay L, const double *sinv, float *st, float2 *s2);
// FP64 red-black half sweep of one colour, in place
// FP64 red-only residual + restriction in diagonal form (dg = sum of the cell's face betas)
void launch_rr_red_diag64(cudaStream_t s, Dims fine, double h2, Coef<double> c, const double *dg,
                          const double *b, const double *x, double *bc);
void launch_rbgs_half64(cudaStream_t s, Dims d, double h2, Coef<double> c, const double *b, double *p,
                        int colour);
template <typename T>
void launch_apply(cudaStream_t s, Dims d, double ih2, Coef<T> c, const T *x, T *y);
template <typename T>
void launch_residual(cudaStream_t s, Dims d, double ih2, Coef<T> c, const T *b, const T *x, T *r);
// bc = mean of the 8 children's residuals (red_only: black children count as 0)
template <typename T>
void launch_resid_restrict(cudaStream_t s, Dims fine, double ih2, Coef<T> c, const T *b,
                           const T *x, T *bc, bool red_only);
// e += P ec on the cells of colour only_col (0 red, 1 black) or all cells (-1)
template <typename T>
void launch_prolong(cudaStream_t s, Dims coarse, const T *ec, T *e, int kind, int only_col);
template <typename T>
void launch_coarse_matvec(cudaStream_t s, int nc, const double *pinv, const T *r, T *e);

// ---- reductions, fine-level FP64 passes, adjoint -----------------------------------
// partials: reduce_blocks(n) x 2 doubles; out: 2 doubles (deterministic order)
// scalars for the host: a one-thread-per-value kernel stores n (<= 32) doubles, or one
// unsigned, into mapped pinned host memory (device-side address of a cudaHostAllocMapped
// buffer), so that the host's wait for them never queues behind bulk copies that other
// streams run on the copy engines
void launch_readback(cudaStream_t s, const double *src, double *dst_mapped, int n);
void launch_readback_u32(cudaStream_t s, const unsigned *src, unsigned *dst_mapped);
// out[0] = sum x, out[1] = sum x^2 (0 unless `squares`)
template <typename T>
void launch_sum_sumsq(cudaStream_t s, i64 n, const T *x, double *partials, double *out, bool squares);
// b64 = (b - sum[0]/n) * scale, with the sum of squares of b64 into out[0]
void launch_sub_mean(cudaStream_t s, i64 n, const double *b, const double *sum, double scale, double *b64,
                     double *partials, double *out);
// fine FP64 residual r = b - A p: out[0] = sum r^2, out[1] = sum p; optional r32 = scale * r
// stored in the level-0 FP32 layout L
void launch_fine_residual(cudaStream_t s, Dims d, Lay L, double ih2, const double *fx, const double *fy,
                          const double *fz, const double *b, const double *p, float *r32,
                          double scale, double *partials, double *out);
// fine FP64 residual in diagonal form, h^2 r = h^2 b - (diag p_c - sum_f beta_f p_nb):
// out[0] = sum (h^2 r)^2, out[1] = sum p; optional r32 = s32 * h^2 r in the level-0 layout L.
// On a slab of a decomposed grid (d.zlo or d.zhi, even nx; p with its ghost planes beside the
// own ones, fz with the face to the ghost above) the ghost planes count as interior neighbours,
// and r32 is stored in the slab's layout L (L.half the colour stride)
void launch_fine_resid2(cudaStream_t s, Dims d, Lay L, double h2, const double *fx, const double *fy,
                        const double *fz, const double *diag, const double *b, bool b_scaled, const double *p,
                        float *r32, float s32, double *partials, double *out);
// r32 = (float)(ih2 scale) * trunc_fp32(b): the scaled FP32 residual of p = 0, as the outer
// residual kernels would write it (b = h^2 b~ in the mixed modes)
void launch_zero_resid32(cudaStream_t s, Dims d, Lay L, const double *b, double scale32, float *r32);
// p = p - shift + alpha * e32 (e32 in the level-0 FP32 layout L; shift a host scalar)
void launch_update(cudaStream_t s, Dims d, Lay L, double *p, const float *e32, double alpha, double shift);
void launch_add_const(cudaStream_t s, i64 n, double *p, double c);
void launch_adjoint_grad(cudaStream_t s, Dims d, double h, const double *lam, const double *p,
                         const double *fx, const double *fy, const double *fz, const double *csfx,
                         const double *csfy, const double *csfz, double sigma, float *gx,
                         float *gy, float *gz, double *partials, double *out);

// ---- either side of the solve (kernels_project.cu) --------------------------------------
// o = u + beta (G p + sigma csf) on the interior faces, o = u on the walls (csfx NULL: no
// surface term); o may be u (in place; the walls are then not rewritten)
void launch_project(cudaStream_t s, Dims d, double h, const double *p, const double *fx, const double *fy,
                    const double *fz, const double *csfx, const double *csfy, const double *csfz, double sigma,
                    const double *ux, const double *uy, const double *uz, double *ox, double *oy, double *oz);
// dL/drho from FP32 face gradients, and dL/df_q = dL/drho (rho_q - rho_last) into dfrac[q]
void launch_density_grads(cudaStream_t s, Dims d, const double *rho, const float *gx, const float *gy,
                          const float *gz, double *drho, int nfrac, const double *rho_phase,
                          double *const *dfrac);

}  // namespace mg
