// Domain-decomposed FP64 multigrid solve: z slabs with ghost planes (mg_dd_* in include/mg.h).
//
// The paper's solver runs one MPI rank per domain and names the switch between multigrid
// levels as a cost of its scaling (§4.1, §4.3.2).  This file is that decomposition for the
// FP64 V-cycle of this library, with the ranks held as separate slab buffers on one GPU:
//   - level l is cut into `ranks` slabs of planes[l] planes along z; a slab stores its own
//     planes and one ghost plane below and above for x, and its z faces up to the face to the
//     ghost above, so that the faces between slabs act as interior faces (Dims.zlo / zhi);
//   - every red or black half sweep, and the prolongation, is followed by a halo exchange:
//     each slab's first and last own planes are copied into its neighbours' ghost planes;
//   - the red-only residual + restriction of the last decomposed level writes each slab's
//     coarse planes into one whole-grid array (the gather of the coarse levels onto one rank),
//     where a whole-grid handle runs the rest of the V-cycle through the FP64 components; the
//     prolongation back reads each slab's coarse planes and their neighbours from that array;
//   - the residual norm and the mean of p are sums of per-slab partial sums, added on the
//     host in slab order (the all-reduce).
// Every cell sees the same arithmetic, in the same order, as in the whole-grid FP64 V-cycle,
// so one V-cycle gives bitwise the same result for any number of slabs.  The exchange is a
// device-to-device copy here; between GPUs it would be one send/receive per neighbour.
//
// The mixed-precision solve (precision MG_MIXED) cuts the same levels, as deep as its kernels
// allow: FP32 slabs in the colour-split layout with a ghost plane below and above in each colour
// half (mg::Lay zlo / zhi), s = 1/rho on the finest level and the low faces below it, the FP32
// kernels in their ghost variants, an exchange of the colour just updated after every half
// sweep and after the prolongation, the last cut level's red residuals restricted straight into
// the whole-grid handle's FP32 level (the gather), the rest of the inner V-cycle on that handle,
// and the FP64 outer loop slab by slab (the fused residual kernel over each slab with its p
// ghost planes exchanged first; the norms and sums of p added over the slabs).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "mg_internal.cuh"

namespace {

constexpr int kThreads = 256;

// one slab of one decomposed level
struct Slab {
    mg::Dims d;      // own planes (nz = planes), zlo / zhi when a neighbour exists below / above
    int z0;          // first whole-grid plane of the slab
    double *xe;      // x with a ghost plane below and above: planes + 2 planes
    double *x;       // = xe + nxy, the first own plane
    double *b;       // own planes
    double *fx, *fy; // low faces of the own planes
    double *fze;     // low z faces of the own planes and of the ghost above: planes + 1 planes
    double *invd, *dg;
    // mixed precision: FP32 arrays in the slab layout `lay` (each colour half with a ghost plane
    // below and above; the pointers at the red half's first own plane): x, b, and s = 1/rho on
    // the finest level or the low faces below it (fz with the face to the ghost plane above)
    mg::Lay lay;
    float *x32, *b32, *s32, *fx32, *fy32, *fz32;
};

// The mixed solve's FP32 s = 1/rho of one slab: the whole grid's s (natural FP64) over the
// slab's planes and its ghost planes into the slab's colour-split layout, rounded to nearest as
// the whole-grid pack rounds it; z0 is the slab's first whole-grid plane (even, so colours agree)
__global__ void k_pack_slab_s32(mg::Lay L, int z0, int nz_total, const double *__restrict__ s_whole, float *s32) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= L.nx) return;
    const int rows = L.ny * (L.nz + 2);
    for (int row = blockIdx.y; row < rows; row += gridDim.y) {
        const int y = row % L.ny, z = row / L.ny - 1;  // z = -1 .. nz (the ghost planes)
        const int zg = z0 + z;
        if (zg < 0 || zg >= nz_total) continue;  // beyond a wall: never read
        const double v = s_whole[((mg::i64)zg * L.ny + y) * L.nx + x];
        s32[((x + y + z) & 1) * L.half + ((mg::i64)z * L.ny + y) * L.hx + (x >> 1)] = mg::d2f_rn(v);
    }
}

// The FP32 low faces of one slab of a cut level below the finest: the slab's FP64 faces (own
// planes; for fz also the face to the ghost plane above, `planes` = nz + 1) into its colour-split
// layout, rounded to nearest as the whole-grid pack rounds them
__global__ void k_pack_slab_faces(mg::Lay L, int planes, const double *__restrict__ f, float *f32) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= L.nx) return;
    const int rows = L.ny * planes;
    for (int row = blockIdx.y; row < rows; row += gridDim.y) {
        const int y = row % L.ny, z = row / L.ny;
        f32[((x + y + z) & 1) * L.half + ((mg::i64)z * L.ny + y) * L.hx + (x >> 1)] =
            mg::d2f_rn(f[((mg::i64)z * L.ny + y) * L.nx + x]);
    }
}

// out = (in - c) * scale, the mixed modes' scaled zero-mean right-hand side
__global__ void k_sub_scalar_scale(mg::i64 n, const double *__restrict__ in, double c, double scale, double *out) {
    const mg::i64 m = (mg::i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (m < n) out[m] = (in[m] - c) * scale;
}

__global__ void k_sub_scalar(mg::i64 n, const double *__restrict__ in, double c, double *out) {
    const mg::i64 m = (mg::i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (m < n) out[m] = in[m] - c;
}

// the coarse low z faces of one plane from the 2 x 2 fine faces that tile them
__global__ void k_coarsen_z_plane(mg::Dims f, mg::Dims c, const double *__restrict__ ffz_plane,
                                  double *cfz_plane) {
    const int C = blockIdx.x * blockDim.x + threadIdx.x;
    if (C >= c.nx * c.ny) return;
    const int I = C % c.nx, J = C / c.nx;
    const mg::i64 base = (mg::i64)(2 * J) * f.nx + 2 * I;
    double sz = 0.0;
    for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) sz += ffz_plane[base + b * f.nx + a];
    cfz_plane[C] = sz / 4.0;
}

inline unsigned blocks_for(mg::i64 n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// a CUDA event pair destroyed on every way out of a call
struct EventPair {
    cudaEvent_t e[2] = {nullptr, nullptr};
    ~EventPair() {
        for (cudaEvent_t x : e)
            if (x) cudaEventDestroy(x);
    }
};

}  // namespace

struct mg_dd {
    mg_opts o;
    mg_dd_plan plan;
    cudaStream_t s;
    int P, ndec;
    std::vector<std::vector<Slab>> lv;  // [level < ndec][rank]
    mg_handle *ch;                       // whole grid from the switch level down
    int ch_nlev;
    double *cx[MG_MAX_LEVELS], *cb[MG_MAX_LEVELS];
    double *gfx, *gfy, *gfz, *sinv;      // set-up scratch: whole-grid level-0 low faces, 1/rho
    double *abx, *aby, *abz;             // switch-level faces in the ABI layout
    double *partials, *red;
    unsigned *err;
    std::vector<void *> allocs;
    long long exchanges, halo_bytes;     // per V-cycle
    // one stream per rank: each phase of the cycle (a half sweep, an exchange, the restriction,
    // the prolongation) forks from s onto the ranks' streams and joins back, so the ranks' slabs
    // are worked on concurrently, as on separate GPUs (empty: every rank on s, one after another)
    std::vector<cudaStream_t> rs;
    std::vector<cudaEvent_t> rdone;
    cudaEvent_t fork;
    // the whole V-cycle recorded once as a CUDA graph (fixed buffers and arguments) and replayed
    // by every cycle; null: launched call by call
    cudaGraphExec_t cyc_exec;
    long long cyc_launches;
    cudaGraphExec_t mix_exec[2];  // mixed: inner V-cycle without update, from zero / continuing
    long long mix_launches[2];
    bool cyc_tried;
    int have_op;
    // mixed precision: the whole-grid handle's FP32 level 0 (the switch level), its layout and
    // arrays, gathered into by the slabs' restriction and read by their prolongation
    bool mixed;
    mg::Lay clay;
    float *cb32, *cx32;
    char msg[256];
};

namespace {

int dd_fail(mg_dd *dd, int code, const char *fmt, ...) {
    if (dd) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(dd->msg, sizeof(dd->msg), fmt, ap);
        va_end(ap);
    }
    return code;
}

#define DD_CUDA(dd, call)                                                                        \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return dd_fail((dd), MG_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));  \
    } while (0)

mg::Coef<double> coef(const Slab &S) { return {S.fx, S.fy, S.fze, S.invd}; }

// f(r, stream) for every rank, on the rank's stream after everything queued so far on dd->s;
// dd->s then waits for all of them
template <typename F>
int per_rank(mg_dd *dd, F &&f) {
    if (dd->rs.empty()) {
        for (int r = 0; r < dd->P; ++r) {
            const int rc = f(r, dd->s);
            if (rc) return rc;
        }
        return MG_OK;
    }
    DD_CUDA(dd, cudaEventRecord(dd->fork, dd->s));
    for (int r = 0; r < dd->P; ++r) {
        DD_CUDA(dd, cudaStreamWaitEvent(dd->rs[r], dd->fork, 0));
        const int rc = f(r, dd->rs[r]);
        DD_CUDA(dd, cudaEventRecord(dd->rdone[r], dd->rs[r]));  // joined even after a failed launch
        if (rc) return rc;
    }
    for (int r = 0; r < dd->P; ++r) DD_CUDA(dd, cudaStreamWaitEvent(dd->s, dd->rdone[r], 0));
    return MG_OK;
}

// ghost planes of x on level l from the neighbouring slabs' first / last own planes: each rank
// receives its two planes (the neighbours' planes were finished by the phase before)
int exchange(mg_dd *dd, int l) {
    std::vector<Slab> &R = dd->lv[l];
    const size_t bytes = sizeof(double) * (size_t)R[0].d.nxy;
    return per_rank(dd, [&](int r, cudaStream_t st) -> int {
        if (r > 0)
            DD_CUDA(dd, cudaMemcpyAsync(R[r].xe, R[r - 1].x + (R[r - 1].d.nz - 1) * R[r - 1].d.nxy, bytes,
                                        cudaMemcpyDeviceToDevice, st));
        if (r + 1 < dd->P)
            DD_CUDA(dd, cudaMemcpyAsync(R[r].x + R[r].d.n, R[r + 1].x, bytes, cudaMemcpyDeviceToDevice, st));
        return MG_OK;
    });
}

int smooth(mg_dd *dd, int l, int sweeps, int order) {
    const double h2 = dd->o.h * dd->o.h * (double)(1ll << (2 * l));
    std::vector<Slab> &R = dd->lv[l];
    for (int sw = 0; sw < sweeps; ++sw)
        for (int half = 0; half < 2; ++half) {
            const int col = order ? 1 - half : half;
            int rc = per_rank(dd, [&](int r, cudaStream_t st) -> int {
                mg::launch_rbgs_half64(st, R[r].d, h2, coef(R[r]), R[r].b, R[r].x, col);
                return MG_OK;
            });
            if (rc) return rc;
            rc = exchange(dd, l);
            if (rc) return rc;
        }
    return MG_OK;
}

// the whole-grid V-cycle tail (switch level down to the coarsest) from x = 0, by the FP64
// components of the whole-grid handle
int tail(mg_dd *dd, int k) {
    if (k == dd->ch_nlev - 1) return mg_coarse_solve(dd->ch, MG_F64, dd->cb[k], dd->cx[k]);
    int rc = mg_presmooth_restrict(dd->ch, k, MG_F64, dd->cx[k], dd->cb[k], dd->o.pre, 1, dd->cb[k + 1]);
    if (rc) return rc;
    rc = tail(dd, k + 1);
    if (rc) return rc;
    return mg_prolong_postsmooth(dd->ch, k, MG_F64, dd->cx[k + 1], dd->cx[k], dd->cb[k], dd->o.post);
}

// one V-cycle on decomposed level l (x from zero, or from the slabs' x with valid ghosts)
int vcycle(mg_dd *dd, int l, bool x_zero) {
    std::vector<Slab> &R = dd->lv[l];
    const double h2 = dd->o.h * dd->o.h * (double)(1ll << (2 * l));
    int rc;
    if (x_zero) {
        rc = per_rank(dd, [&](int r, cudaStream_t st) -> int {
            DD_CUDA(dd, cudaMemsetAsync(R[r].xe, 0, sizeof(double) * (size_t)(R[r].d.n + 2 * R[r].d.nxy), st));
            return MG_OK;
        });
        if (rc) return rc;
    }
    rc = smooth(dd, l, dd->o.pre, 0);
    if (rc) return rc;
    const bool last = l + 1 == dd->ndec;
    rc = per_rank(dd, [&](int r, cudaStream_t st) -> int {
        Slab &S = R[r];
        double *bc;
        if (!last) {
            bc = dd->lv[l + 1][r].b;
        } else {
            const mg::i64 cnxy = (mg::i64)(S.d.nx / 2) * (S.d.ny / 2);
            bc = dd->cb[0] + (mg::i64)(S.z0 / 2) * cnxy;
        }
        // after a pre-smoothing sweep (black last) every black residual is zero
        if (dd->o.pre > 0)
            mg::launch_rr_red_diag64(st, S.d, h2, coef(S), S.dg, S.b, S.x, bc);
        else
            mg::launch_resid_restrict<double>(st, S.d, 1.0 / h2, coef(S), S.b, S.x, bc, false);
        return MG_OK;
    });
    if (rc) return rc;
    rc = last ? tail(dd, 0) : vcycle(dd, l + 1, true);
    if (rc) return rc;
    // prolongation: red cells only when a post sweep (black first) follows
    rc = per_rank(dd, [&](int r, cudaStream_t st) -> int {
        Slab &S = R[r];
        mg::Dims cd;
        const double *ec;
        if (!last) {
            cd = dd->lv[l + 1][r].d;
            ec = dd->lv[l + 1][r].x;
        } else {
            cd = mg::make_dims(S.d.nx / 2, S.d.ny / 2, S.d.nz / 2);
            cd.zlo = S.d.zlo;
            cd.zhi = S.d.zhi;
            ec = dd->cx[0] + (mg::i64)(S.z0 / 2) * cd.nxy;  // the neighbours' planes lie beside it
        }
        mg::launch_prolong<double>(st, cd, ec, S.x, dd->o.prolong, dd->o.post > 0 ? 0 : -1);
        return MG_OK;
    });
    if (rc) return rc;
    rc = exchange(dd, l);
    if (rc) return rc;
    return smooth(dd, l, dd->o.post, 1);
}

// ---- the mixed-precision cycle: FP32 slabs of the finest level ------------------------------

// The coarse level of cut level l for slab r, as its restriction and prolongation see it: the
// next cut level's slab, or, below the last cut level, a view of the whole-grid handle's FP32
// level 0 from the slab's first coarse plane (even, so colours agree) with its neighbours' planes
// beside it (the gather and the scatter back)
struct Coarse {
    mg::Lay lay;
    float *b, *x;
};
Coarse coarse_of(const mg_dd *dd, int l, int r) {
    const Slab &S = dd->lv[l][r];
    if (l + 1 < dd->ndec) {
        const Slab &C = dd->lv[l + 1][r];
        return {C.lay, C.b32, C.x32};
    }
    mg::Lay v = dd->clay;
    v.nz = S.d.nz / 2;
    v.n = (mg::i64)v.nx * v.ny * v.nz;
    v.zlo = S.d.zlo;
    v.zhi = S.d.zhi;
    const mg::i64 off = (mg::i64)(S.z0 / 2) * v.ny * v.hx;
    return {v, dd->cb32 + off, dd->cx32 + off};
}

// colour c's first and last own planes of every slab's FP32 x on cut level l into its
// neighbours' ghost planes
int exchange32(mg_dd *dd, int l, int c) {
    std::vector<Slab> &R = dd->lv[l];
    const size_t plane = (size_t)R[0].lay.ny * R[0].lay.hx;
    return per_rank(dd, [&](int r, cudaStream_t st) -> int {
        float *col = R[r].x32 + (size_t)c * R[r].lay.half;
        if (r > 0) {
            const Slab &B = R[r - 1];
            DD_CUDA(dd, cudaMemcpyAsync(col - plane, B.x32 + (size_t)c * B.lay.half + (size_t)(B.lay.nz - 1) * plane,
                                        4 * plane, cudaMemcpyDeviceToDevice, st));
        }
        if (r + 1 < dd->P)
            DD_CUDA(dd, cudaMemcpyAsync(col + (size_t)R[r].lay.nz * plane, R[r + 1].x32 + (size_t)c * R[r + 1].lay.half,
                                        4 * plane, cudaMemcpyDeviceToDevice, st));
        return MG_OK;
    });
}

// h^2 of cut level l (the spacing doubles per level: an exact power-of-two scaling)
double h2_of(const mg_dd *dd, int l) { return dd->o.h * dd->o.h * (double)(1ll << (2 * l)); }

// a half sweep of colour c on every slab of cut level l, then the exchange of that colour
int half_mixed(mg_dd *dd, int l, int c, bool from_zero) {
    std::vector<Slab> &R = dd->lv[l];
    const double h2 = h2_of(dd, l);
    const int rc = per_rank(dd, [&](int r, cudaStream_t st) -> int {
        mg::launch_half32(st, R[r].lay, h2, R[r].s32, R[r].fx32, R[r].fy32, R[r].fz32, R[r].b32, R[r].x32, c, from_zero);
        return MG_OK;
    });
    return rc ? rc : exchange32(dd, l, c);
}

// One FP32 V-cycle from cut level l down, in the order of the whole-grid cycle: from x32 = 0
// (from_zero) or from the slabs' x32; with alpha_shift (finest level), the last red half sweep
// adds alpha x - shift to the slabs' FP64 p instead of storing x32.  `recording`: under a stream
// capture (the whole-grid handle then records its levels launch by launch).
int vcycle_mixed(mg_dd *dd, int l, bool from_zero, const double *alpha_shift, bool recording = false) {
    std::vector<Slab> &R = dd->lv[l];
    const double h2 = h2_of(dd, l);
    int rc;
    for (int sw = 0; sw < dd->o.pre; ++sw) {
        if ((rc = half_mixed(dd, l, 0, from_zero && sw == 0))) return rc;
        if ((rc = half_mixed(dd, l, 1, false))) return rc;
    }
    // the red residuals (every black one is zero after the black sweep), restricted into the
    // coarse right-hand side
    rc = per_rank(dd, [&](int r, cudaStream_t st) -> int {
        const Coarse co = coarse_of(dd, l, r);
        mg::launch_resid_restrict32(st, R[r].lay, co.lay, 1.0 / h2, R[r].s32, R[r].fx32, R[r].fy32, R[r].fz32, R[r].b32,
                                    R[r].x32, co.b, true);
        return MG_OK;
    });
    if (rc) return rc;
    if (l + 1 < dd->ndec) {
        if ((rc = vcycle_mixed(dd, l + 1, true, nullptr, recording))) return rc;
    } else {
        mg::handle_vcycle32(dd->ch, 0, recording);  // the switch level down, on the caller's stream
    }
    // the prolongation back: the red cells of each slab from its coarse planes and those beside
    rc = per_rank(dd, [&](int r, cudaStream_t st) -> int {
        const Coarse co = coarse_of(dd, l, r);
        mg::launch_prolong32(st, R[r].lay, co.lay, co.x, R[r].x32, MG_PROLONG_TRILINEAR, 0);
        return MG_OK;
    });
    if (rc) return rc;
    if ((rc = exchange32(dd, l, 0))) return rc;
    for (int sw = 0; sw < dd->o.post; ++sw) {
        if ((rc = half_mixed(dd, l, 1, false))) return rc;
        if (sw + 1 < dd->o.post || !alpha_shift) {
            if ((rc = half_mixed(dd, l, 0, false))) return rc;
            continue;
        }
        rc = per_rank(dd, [&](int r, cudaStream_t st) -> int {
            mg::launch_half32_update(st, R[r].lay, h2, R[r].s32, nullptr, nullptr, nullptr, R[r].b32, R[r].x32, R[r].x,
                                     nullptr, alpha_shift[0], alpha_shift[1]);
            return MG_OK;
        });
        if (rc) return rc;
    }
    return MG_OK;
}

// Record f() (one cycle) on a private stream, the whole-grid handle's launches included;
// nothing runs.  Returns the instantiated graph, or null where recording is refused (the
// cycles then launch call by call); *launches = the kernels it holds.
template <typename F>
cudaGraphExec_t record_cycle(mg_dd *dd, F &&f, long long *launches) {
    *launches = 0;
    cudaStream_t cap = nullptr;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    // the recording must not see work still queued on the caller's stream
    if (cudaStreamSynchronize(dd->s) != cudaSuccess) {
        cudaGetLastError();
        cudaStreamDestroy(cap);
        return nullptr;
    }
    cudaStream_t saved = dd->s;
    dd->s = cap;
    cudaStream_t saved_ch = mg::swap_handle_stream(dd->ch, cap);
    const unsigned long long l0 = mg::launches_total();
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    int rc = MG_ERR_CUDA;
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        rc = f();
        if (cudaStreamEndCapture(cap, &g) != cudaSuccess) rc = MG_ERR_CUDA;
    }
    const long long n = (long long)(mg::launches_total() - l0);
    mg::count_launch((int)-n);  // recorded, not run
    mg::swap_handle_stream(dd->ch, saved_ch);
    dd->s = saved;
    if (rc == MG_OK && g && cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) exec = nullptr;
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    cudaGetLastError();
    *launches = exec ? n : 0;
    return exec;
}

// The cycles whose buffers and arguments do not depend on the operator, recorded once: the
// FP64 V-cycle; the mixed inner V-cycles without the outer update, from zero and continuing
// (the last cycle of an outer iteration takes that iteration's update scalars: launched).
void build_cycle_graph(mg_dd *dd) {
    dd->cyc_tried = true;
    if (!dd->mixed) {
        dd->cyc_exec = record_cycle(dd, [&] { return vcycle(dd, 0, false); }, &dd->cyc_launches);
        return;
    }
    for (int k = 0; k < 2; ++k)
        dd->mix_exec[k] = record_cycle(dd, [&] { return vcycle_mixed(dd, 0, k == 0, nullptr, true); }, &dd->mix_launches[k]);
}

// one V-cycle of level 0 from the slabs' x: the recorded graph, or call by call
int cycle(mg_dd *dd) {
    if (dd->cyc_exec) {
        DD_CUDA(dd, cudaGraphLaunch(dd->cyc_exec, dd->s));
        mg::count_launch((int)dd->cyc_launches);
        return MG_OK;
    }
    return vcycle(dd, 0, false);
}

// per slab, by the whole grid's fused residual kernel over the slab's own planes (its ghost
// planes as neighbours): sum of (h^2 r)^2 and sum of x; one read-back for all slabs, added in
// slab order (the all-reduce of the two scalars a rank would exchange)
int slab_residual_norms(mg_dd *dd, double *rn2_h4, double *sp) {
    const int P = dd->P;
    const double h2 = dd->o.h * dd->o.h;
    for (int r = 0; r < P; ++r) {
        Slab &S = dd->lv[0][r];
        mg::launch_fine_resid2(dd->s, S.d, mg::make_lay(S.d), h2, S.fx, S.fy, S.fze, S.dg, S.b, false, S.x,
                               nullptr, 0.f, dd->partials, dd->red + 2 * r);
    }
    std::vector<double> h(2 * (size_t)P);
    DD_CUDA(dd, cudaMemcpyAsync(h.data(), dd->red, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, dd->s));
    DD_CUDA(dd, cudaStreamSynchronize(dd->s));
    double q = 0.0, x = 0.0;
    for (int r = 0; r < P; ++r) {
        q += h[2 * r];
        x += h[2 * r + 1];
    }
    *rn2_h4 = q;
    *sp = x;
    return MG_OK;
}

// the sum of the slabs' own planes of x in FP64, added in slab order
int slab_sum_x(mg_dd *dd, double *sum) {
    const int P = dd->P;
    for (int r = 0; r < P; ++r) {
        Slab &S = dd->lv[0][r];
        mg::launch_sum_sumsq<double>(dd->s, S.d.n, S.x, dd->partials, dd->red + 2 * r, false);
    }
    std::vector<double> h(2 * (size_t)P);
    DD_CUDA(dd, cudaMemcpyAsync(h.data(), dd->red, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, dd->s));
    DD_CUDA(dd, cudaStreamSynchronize(dd->s));
    double a = 0.0;
    for (int r = 0; r < P; ++r) a += h[2 * r];
    *sum = a;
    return MG_OK;
}

// the same for one array per slab: sum and sum of squares of the slabs' b
int slab_sums_b(mg_dd *dd, double *sum, double *sumsq) {
    const int P = dd->P;
    for (int r = 0; r < P; ++r) {
        Slab &S = dd->lv[0][r];
        mg::launch_sum_sumsq<double>(dd->s, S.d.n, S.b, dd->partials, dd->red + 2 * r, true);
    }
    std::vector<double> h(2 * (size_t)P);
    DD_CUDA(dd, cudaMemcpyAsync(h.data(), dd->red, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, dd->s));
    DD_CUDA(dd, cudaStreamSynchronize(dd->s));
    double a = 0.0, q = 0.0;
    for (int r = 0; r < P; ++r) {
        a += h[2 * r];
        q += h[2 * r + 1];
    }
    *sum = a;
    *sumsq = q;
    return MG_OK;
}

void *dd_alloc(mg_dd *dd, size_t bytes) {
    void *p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 8) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    dd->allocs.push_back(p);
    return p;
}

// The mixed-precision solve on the slabs, step for step the whole grid's cold-started mixed
// loop: b~ = (b - mean b) h^2; the first inner right-hand side is b~ in FP32 scaled by 1 / |b~|;
// each outer iteration runs `inner` FP32 V-cycles (the last one adding its correction to p), then
// the FP64 residual of every slab, with p's ghost planes exchanged first, which also writes the
// next scaled FP32 right-hand side and the partial sums of r^2 and p; the exact FP64 mean of p is
// removed at exit.
int solve_mixed(mg_dd *dd, const double *b, double *p, mg_stats *st) {
    cudaStream_t s = dd->s;
    EventPair ev;
    DD_CUDA(dd, cudaEventCreate(&ev.e[0]));
    DD_CUDA(dd, cudaEventCreate(&ev.e[1]));
    DD_CUDA(dd, cudaEventRecord(ev.e[0], s));
    const double n = (double)dd->o.nx * dd->o.ny * dd->o.nz;
    const double h2 = dd->o.h * dd->o.h, ih2 = 1.0 / h2;
    std::vector<Slab> &R = dd->lv[0];
    double sb = 0.0;
    for (Slab &S : R) {
        mg::launch_sum_sumsq<double>(s, S.d.n, b + (size_t)S.z0 * S.d.nxy, dd->partials, dd->red, false);
        double hb[2];
        DD_CUDA(dd, cudaMemcpyAsync(hb, dd->red, sizeof(hb), cudaMemcpyDeviceToHost, s));
        DD_CUDA(dd, cudaStreamSynchronize(s));
        sb += hb[0];
    }
    for (Slab &S : R) {
        mg::count_launch();
        k_sub_scalar_scale<<<blocks_for(S.d.n), kThreads, 0, s>>>(S.d.n, b + (size_t)S.z0 * S.d.nxy, sb / n, h2, S.b);
        DD_CUDA(dd, cudaMemsetAsync(S.xe, 0, 8 * (size_t)(S.d.n + 2 * S.d.nxy), s));
    }
    double t, q0;
    int rc = slab_sums_b(dd, &t, &q0);
    if (rc) return rc;
    const double nb = std::sqrt(q0) / h2;
    double hist[MG_HIST_LEN];
    int hn = 0, cycles = 0, outer = 0, status = MG_ERR_NOT_CONVERGED;
    double rr = nb > 0.0 ? 1.0 : 0.0;
    hist[hn++] = rr;
    if (nb == 0.0 || rr <= dd->o.rtol) status = MG_OK;
    const bool adaptive = dd->o.inner_cycles == 0;
    int inner = adaptive ? mg::handle_first_inner() : dd->o.inner_cycles;
    double scale = 1.0 / nb, rn = nb, mu = 0.0;
    if (status == MG_ERR_NOT_CONVERGED)
        for (Slab &S : R) mg::launch_zero_resid32(s, S.d, S.lay, S.b, ih2 * scale, S.b32);
    while (status == MG_ERR_NOT_CONVERGED) {
        if (adaptive && cycles + inner > dd->o.max_cycles) inner = dd->o.max_cycles - cycles;
        if (inner < 1 || cycles + inner > dd->o.max_cycles) break;
        for (int k = 0; k + 1 < inner; ++k) {
            const int g = k == 0 ? 0 : 1;
            if (dd->mix_exec[g]) {
                DD_CUDA(dd, cudaGraphLaunch(dd->mix_exec[g], s));
                mg::count_launch((int)dd->mix_launches[g]);
            } else if ((rc = vcycle_mixed(dd, 0, k == 0, nullptr))) {
                return rc;
            }
        }
        const double as[2] = {1.0 / scale, mu};
        if ((rc = vcycle_mixed(dd, 0, inner == 1, as))) return rc;
        scale = 1.0 / rn;
        if ((rc = exchange(dd, 0))) return rc;  // p's ghost planes
        for (int r = 0; r < dd->P; ++r) {
            Slab &S = R[r];
            mg::launch_fine_resid2(s, S.d, S.lay, h2, S.fx, S.fy, S.fze, S.dg, S.b, true, S.x, S.b32, (float)(ih2 * scale),
                                   dd->partials, dd->red + 2 * r);
        }
        std::vector<double> hs(2 * (size_t)dd->P);
        DD_CUDA(dd, cudaMemcpyAsync(hs.data(), dd->red, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost, s));
        DD_CUDA(dd, cudaStreamSynchronize(s));
        double q = 0.0, sp = 0.0;
        for (int r = 0; r < dd->P; ++r) {
            q += hs[2 * r];
            sp += hs[2 * r + 1];
        }
        rn = std::sqrt(q) * ih2;
        mu = sp / n;
        const double rr_prev = rr;
        rr = rn / nb;
        cycles += inner;
        ++outer;
        if (adaptive) inner = mg::handle_next_inner(rr_prev, rr, inner, dd->o.rtol);
        if (hn < MG_HIST_LEN) hist[hn++] = rr;
        if (!std::isfinite(rr) || rr > 1e12) {
            status = MG_ERR_DIVERGED;
            break;
        }
        if (rr <= dd->o.rtol) status = MG_OK;
    }
    // exact zero-mean gauge at exit (the outer loop shifts by an FP32-accumulated mean)
    if (nb > 0.0) {
        double sx;
        if ((rc = slab_sum_x(dd, &sx))) return rc;
        for (Slab &S : R) mg::launch_add_const(s, S.d.n, S.x, -sx / n);
    }
    for (Slab &S : R)
        DD_CUDA(dd, cudaMemcpyAsync(p + (size_t)S.z0 * S.d.nxy, S.x, 8 * (size_t)S.d.n, cudaMemcpyDeviceToDevice, s));
    DD_CUDA(dd, cudaEventRecord(ev.e[1], s));
    DD_CUDA(dd, cudaEventSynchronize(ev.e[1]));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev.e[0], ev.e[1]);
    DD_CUDA(dd, cudaGetLastError());
    if (st) {
        st->status = status;
        st->cycles = cycles;
        st->outer = outer;
        st->relres = rr;
        for (int k = 0; k < MG_HIST_LEN; ++k) st->relres_hist[k] = k < hn ? hist[k] : 0.0;
        st->ms = ms;
    }
    if (status == MG_ERR_NOT_CONVERGED)
        return dd_fail(dd, status, "not converged: relres %.3e after %d cycles", rr, cycles);
    if (status == MG_ERR_DIVERGED) return dd_fail(dd, status, "diverged: relres %.3e", rr);
    return MG_OK;
}

}  // namespace

extern "C" {

int mg_dd_make_plan(int nx, int ny, int nz, int coarsest, int ranks, int max_decomposed, mg_dd_plan *plan) {
    if (!plan || nx < 1 || ny < 1 || nz < 1 || coarsest < 2 || ranks < 1 || ranks > MG_DD_MAX_RANKS ||
        max_decomposed < 0)
        return MG_ERR_ARG;
    std::memset(plan, 0, sizeof(*plan));
    plan->ranks = ranks;
    // the whole-grid hierarchy (the rule of mg_create)
    int n = 0, x = nx, y = ny, z = nz;
    for (;;) {
        plan->nx[n] = x;
        plan->ny[n] = y;
        plan->nz[n] = z;
        ++n;
        const int mx = x > y ? (x > z ? x : z) : (y > z ? y : z);
        if (x % 2 || y % 2 || z % 2 || mx <= coarsest || n == MG_MAX_LEVELS) break;
        x /= 2;
        y /= 2;
        z /= 2;
    }
    plan->levels = n;
    // level l is cut into slabs while it is not the coarsest, nz_l divides evenly and every
    // slab has an even number (>= 2) of planes, so that its restriction pairs stay inside it
    int s = 0;
    while (s < n - 1 && (max_decomposed == 0 || s < max_decomposed) && plan->nz[s] % ranks == 0 &&
           (plan->nz[s] / ranks) % 2 == 0 && plan->nz[s] / ranks >= 2) {
        plan->planes[s] = plan->nz[s] / ranks;
        ++s;
    }
    plan->switch_level = s;
    return s >= 1 ? MG_OK : MG_ERR_ARG;
}

int mg_dd_create(const mg_opts *o, int ranks, int max_decomposed, void *stream, mg_dd **out) {
    mg::NvtxRange nvtx_("mg_dd_create");
    if (!out) return MG_ERR_ARG;
    *out = nullptr;
    if (!o || o->method != MG_METHOD_VCYCLE || !(o->h > 0.0) || o->pre < 0 || o->post < 0 || o->max_cycles < 0 ||
        o->warm_start)
        return MG_ERR_ARG;
    const bool mixed = o->precision == MG_MIXED;
    if (!mixed && (o->precision != MG_FP64 || o->inner_cycles != 1)) return MG_ERR_ARG;
    // the mixed cycle cuts the finest level only, with the finest level's fast kernels: red-only
    // restriction (pre >= 1), red-only trilinear prolongation (post >= 1) from a coarse level
    // whose rows hold a multiple of 8 cells, and even first coarse planes (slabs of 4k planes)
    if (mixed && (o->inner_cycles < 0 || o->pre < 1 || o->post < 1 || o->prolong != MG_PROLONG_TRILINEAR ||
                  o->nx % 16 != 0 || ranks < 1 || o->nz % (4 * ranks) != 0))
        return MG_ERR_ARG;
    mg_dd *dd = new (std::nothrow) mg_dd();
    if (!dd) return MG_ERR_OOM;
    dd->o = *o;
    dd->mixed = mixed;
    dd->s = static_cast<cudaStream_t>(stream);
    if (mg_dd_make_plan(o->nx, o->ny, o->nz, o->coarsest, ranks, max_decomposed, &dd->plan) != MG_OK) {
        delete dd;
        return MG_ERR_ARG;
    }
    if (mixed) {
        // the mixed cycle's cut levels prolong with the red trilinear kernel (coarse rows of a
        // multiple of 8 cells, so nx_l a multiple of 16) and the last one restricts into a view
        // of the whole coarse level starting at an even plane (slabs of 4k planes)
        const mg_dd_plan &pl = dd->plan;
        int sw = pl.switch_level;
        auto fits = [&](int k) {
            for (int l = 0; l < k; ++l)
                if (pl.nx[l] % 16 != 0) return false;
            return pl.planes[k - 1] % 4 == 0;
        };
        while (sw > 0 && !fits(sw)) --sw;
        if (sw == 0 || mg_dd_make_plan(o->nx, o->ny, o->nz, o->coarsest, ranks, sw, &dd->plan) != MG_OK) {
            delete dd;
            return MG_ERR_ARG;
        }
    }
    dd->P = ranks;
    dd->ndec = dd->plan.switch_level;
    const mg_dd_plan &pl = dd->plan;
    bool ok = true;
    auto A = [&](size_t n_doubles) {
        double *p = static_cast<double *>(dd_alloc(dd, 8 * n_doubles));
        if (!p) ok = false;
        return p;
    };
    dd->lv.resize(dd->ndec);
    for (int l = 0; l < dd->ndec && ok; ++l) {
        dd->lv[l].resize(ranks);
        for (int r = 0; r < ranks && ok; ++r) {
            Slab &S = dd->lv[l][r];
            S.d = mg::make_dims(pl.nx[l], pl.ny[l], pl.planes[l]);
            S.d.zlo = r > 0;
            S.d.zhi = r + 1 < ranks;
            S.z0 = r * pl.planes[l];
            const size_t n = (size_t)S.d.n, nxy = (size_t)S.d.nxy;
            S.xe = A(n + 2 * nxy);
            S.x = S.xe ? S.xe + nxy : nullptr;
            S.b = A(n);
            S.fx = A(n);
            S.fy = A(n);
            S.fze = A(n + nxy);
            S.invd = mixed ? nullptr : A(n);
            S.dg = A(n);
            if (mixed) {  // the FP32 slab layout: each colour half with its two ghost planes
                S.lay = mg::make_lay(S.d);
                S.lay.zlo = S.d.zlo;
                S.lay.zhi = S.d.zhi;
                const size_t plane = (size_t)S.lay.ny * S.lay.hx;
                S.lay.half = (mg::i64)((S.d.nz + 2) * plane);
                auto F = [&]() {
                    float *q = static_cast<float *>(dd_alloc(dd, 4 * 2 * (size_t)S.lay.half));
                    if (!q) ok = false;
                    return q ? q + plane : nullptr;
                };
                S.x32 = F();
                S.b32 = F();
                if (l == 0) {
                    S.s32 = F();
                } else {
                    S.fx32 = F();
                    S.fy32 = F();
                    S.fz32 = F();
                }
            }
        }
    }
    const mg::i64 n0 = (mg::i64)o->nx * o->ny * o->nz;
    dd->gfx = A(n0);
    dd->gfy = A(n0);
    dd->gfz = A(n0);
    dd->sinv = A(n0);
    const int sl = dd->ndec;
    const int snx = pl.nx[sl], sny = pl.ny[sl], snz = pl.nz[sl];
    dd->abx = A((size_t)snz * sny * (snx + 1));
    dd->aby = A((size_t)snz * (sny + 1) * snx);
    dd->abz = A((size_t)(snz + 1) * sny * snx);
    dd->partials = A(2 * (size_t)mg::reduce_blocks(n0));
    dd->red = A(4 * (size_t)MG_DD_MAX_RANKS);
    dd->err = static_cast<unsigned *>(dd_alloc(dd, 256));
    if (!ok || !dd->err) {
        mg_dd_destroy(dd);
        return MG_ERR_OOM;
    }
    // the whole-grid handle for the switch level and below
    mg_opts co = *o;
    co.nx = snx;
    co.ny = sny;
    co.nz = snz;
    co.h = o->h * (double)(1ll << sl);
    co.rtol = 0.0;
    int rc = mg_create(&co, stream, &dd->ch);
    if (rc != MG_OK) {
        mg_dd_destroy(dd);
        return rc;
    }
    dd->ch_nlev = mg_num_levels(dd->ch);
    if (mixed) {  // the slabs gather into, and prolong from, the handle's own FP32 level 0
        dd->clay = mg::handle_lay32(dd->ch, 0);
        dd->cb32 = mg::handle_b32(dd->ch, 0);
        dd->cx32 = mg::handle_x32(dd->ch, 0);
    }
    for (int k = 0; k < dd->ch_nlev && ok && !mixed; ++k) {
        int dims[3];
        mg_level_dims(dd->ch, k, dims);
        const size_t n = (size_t)dims[0] * dims[1] * dims[2];
        dd->cx[k] = A(n);
        dd->cb[k] = A(n);
    }
    if (!ok) {
        mg_dd_destroy(dd);
        return MG_ERR_OOM;
    }
    // halo traffic of one V-cycle: an exchange after every half sweep and after the prolongation
    dd->exchanges = 0;
    dd->halo_bytes = 0;
    for (int l = 0; l < dd->ndec; ++l) {
        // FP64: both colours of a plane; mixed (finest level only): the one colour just updated,
        // FP32 (the outer loop's exchange of p's FP64 planes comes once per outer iteration)
        const long long per = mixed ? 2ll * (ranks - 1) * 4ll * (pl.nx[l] / 2) * pl.ny[l]
                                    : 2ll * (ranks - 1) * 8ll * pl.nx[l] * pl.ny[l];
        const long long k = 2ll * o->pre + 2ll * o->post + 1;
        dd->exchanges += k;
        dd->halo_bytes += k * per;
    }
    // the ranks' streams (without them the ranks run one after another on the caller's stream)
    bool streams = cudaEventCreateWithFlags(&dd->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int r = 0; r < ranks && streams; ++r) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            streams = false;
            break;
        }
        dd->rs.push_back(st);
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            streams = false;
            break;
        }
        dd->rdone.push_back(ev);
    }
    if (!streams) {
        cudaGetLastError();
        for (cudaStream_t st : dd->rs) cudaStreamDestroy(st);
        for (cudaEvent_t ev : dd->rdone) cudaEventDestroy(ev);
        dd->rs.clear();
        dd->rdone.clear();
    }
    *out = dd;
    return MG_OK;
}

int mg_dd_destroy(mg_dd *dd) {
    if (!dd) return MG_OK;
    if (dd->s) cudaStreamSynchronize(dd->s);
    for (cudaStream_t st : dd->rs) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (cudaEvent_t ev : dd->rdone) cudaEventDestroy(ev);
    if (dd->fork) cudaEventDestroy(dd->fork);
    if (dd->cyc_exec) cudaGraphExecDestroy(dd->cyc_exec);
    for (cudaGraphExec_t e : dd->mix_exec)
        if (e) cudaGraphExecDestroy(e);
    if (dd->ch) mg_destroy(dd->ch);
    for (void *p : dd->allocs) cudaFree(p);
    cudaGetLastError();
    delete dd;
    return MG_OK;
}

const char *mg_dd_last_error(const mg_dd *dd) { return dd ? dd->msg : ""; }

int mg_dd_get_plan(const mg_dd *dd, mg_dd_plan *plan) {
    if (!dd || !plan) return MG_ERR_ARG;
    *plan = dd->plan;
    return MG_OK;
}

int mg_dd_traffic(const mg_dd *dd, long long *exchanges, long long *halo_bytes) {
    if (!dd) return MG_ERR_ARG;
    if (exchanges) *exchanges = dd->exchanges;
    if (halo_bytes) *halo_bytes = dd->halo_bytes;
    return MG_OK;
}

int mg_dd_set_density(mg_dd *dd, const double *rho) {
    mg::NvtxRange nvtx_("mg_dd_set_density");
    if (!dd) return MG_ERR_ARG;
    if (!rho) return dd_fail(dd, MG_ERR_ARG, "rho is NULL");
    dd->have_op = 0;
    const mg_dd_plan &pl = dd->plan;
    cudaStream_t s = dd->s;
    mg::Dims g = mg::make_dims(dd->o.nx, dd->o.ny, dd->o.nz);
    DD_CUDA(dd, cudaMemsetAsync(dd->err, 0, sizeof(unsigned), s));
    mg::launch_faces_from_rho(s, g, rho, dd->sinv, dd->gfx, dd->gfy, dd->gfz, dd->err);
    // level 0 slabs: their planes of the whole-grid faces; fze's last plane is the low face of
    // the next slab's first plane (0 above the top slab: the wall)
    for (int r = 0; r < dd->P; ++r) {
        Slab &S = dd->lv[0][r];
        const size_t off = (size_t)S.z0 * S.d.nxy, bytes = 8 * (size_t)S.d.n, pb = 8 * (size_t)S.d.nxy;
        DD_CUDA(dd, cudaMemcpyAsync(S.fx, dd->gfx + off, bytes, cudaMemcpyDeviceToDevice, s));
        DD_CUDA(dd, cudaMemcpyAsync(S.fy, dd->gfy + off, bytes, cudaMemcpyDeviceToDevice, s));
        DD_CUDA(dd, cudaMemcpyAsync(S.fze, dd->gfz + off, bytes, cudaMemcpyDeviceToDevice, s));
        if (S.d.zhi)
            DD_CUDA(dd, cudaMemcpyAsync(S.fze + S.d.n, dd->gfz + off + S.d.n, pb, cudaMemcpyDeviceToDevice, s));
        else
            DD_CUDA(dd, cudaMemsetAsync(S.fze + S.d.n, 0, pb, s));
        if (dd->mixed) {  // s = 1/rho in FP32 over the slab's planes and its ghost planes
            const int rows = S.lay.ny * (S.lay.nz + 2);
            const dim3 grd((unsigned)((S.lay.nx + 127) / 128), (unsigned)(rows < 65535 ? rows : 65535));
            mg::count_launch();
            k_pack_slab_s32<<<grd, 128, 0, s>>>(S.lay, S.z0, dd->o.nz, dd->sinv, S.s32);
        }
    }
    // decomposed levels: diagonal, then the next level's faces slab by slab
    for (int l = 0; l < dd->ndec; ++l) {
        for (int r = 0; r < dd->P; ++r) {
            Slab &S = dd->lv[l][r];
            mg::launch_invdiag(s, S.d, S.fx, S.fy, S.fze, S.invd, S.dg);
            if (dd->mixed && l > 0) {  // the FP32 faces of a cut level below the finest
                const dim3 grd((unsigned)((S.lay.nx + 127) / 128), (unsigned)std::min(S.lay.ny * (S.lay.nz + 1), 65535));
                mg::count_launch(3);
                k_pack_slab_faces<<<grd, 128, 0, s>>>(S.lay, S.lay.nz, S.fx, S.fx32);
                k_pack_slab_faces<<<grd, 128, 0, s>>>(S.lay, S.lay.nz, S.fy, S.fy32);
                k_pack_slab_faces<<<grd, 128, 0, s>>>(S.lay, S.lay.nz + 1, S.fze, S.fz32);
            }
            mg::Dims cd = mg::make_dims(S.d.nx / 2, S.d.ny / 2, S.d.nz / 2);
            if (l + 1 < dd->ndec) {
                Slab &C = dd->lv[l + 1][r];
                mg::launch_coarsen(s, S.d, S.fx, S.fy, S.fze, C.fx, C.fy, C.fze);
                // the face to the ghost above: from the fine faces to the fine ghost above
                mg::count_launch();
                k_coarsen_z_plane<<<blocks_for(cd.nxy), kThreads, 0, s>>>(S.d, cd, S.fze + S.d.n, C.fze + C.d.n);
            } else {
                // the switch level is whole: the slabs' coarse planes side by side
                const mg::i64 off = (mg::i64)(S.z0 / 2) * cd.nxy;
                mg::launch_coarsen(s, S.d, S.fx, S.fy, S.fze, dd->gfx + off, dd->gfy + off, dd->gfz + off);
            }
        }
    }
    DD_CUDA(dd, cudaGetLastError());
    unsigned herr = 0;
    DD_CUDA(dd, cudaMemcpyAsync(&herr, dd->err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    DD_CUDA(dd, cudaStreamSynchronize(s));
    if (herr) return dd_fail(dd, MG_ERR_DENSITY, "density must be finite and > 0 everywhere");
    // the whole-grid handle takes the switch level's faces (ABI layout)
    const int sl = dd->ndec;
    mg::Dims sd = mg::make_dims(pl.nx[sl], pl.ny[sl], pl.nz[sl]);
    mg::launch_faces_to_api(s, sd, dd->gfx, dd->gfy, dd->gfz, dd->abx, dd->aby, dd->abz);
    int rc = mg_set_face_coeffs(dd->ch, dd->abx, dd->aby, dd->abz);
    if (rc) return dd_fail(dd, rc, "switch level: %s", mg_last_error(dd->ch));
    dd->have_op = 1;
    // the cycles' buffers and arguments do not depend on the operator: recorded once
    if (!dd->cyc_tried) build_cycle_graph(dd);
    return MG_OK;
}

int mg_dd_vcycle(mg_dd *dd, const double *b, double *x) {
    mg::NvtxRange nvtx_("mg_dd_vcycle");
    if (!dd) return MG_ERR_ARG;
    if (!b || !x) return dd_fail(dd, MG_ERR_ARG, "null array");
    if (dd->mixed) return dd_fail(dd, MG_ERR_ARG, "mg_dd_vcycle: FP64 decompositions only");
    if (!dd->have_op) return dd_fail(dd, MG_ERR_STATE, "coefficients not set");
    cudaStream_t s = dd->s;
    for (Slab &S : dd->lv[0]) {
        const size_t off = (size_t)S.z0 * S.d.nxy, pb = 8 * (size_t)S.d.nxy;
        DD_CUDA(dd, cudaMemcpyAsync(S.b, b + off, 8 * (size_t)S.d.n, cudaMemcpyDeviceToDevice, s));
        DD_CUDA(dd, cudaMemcpyAsync(S.x, x + off, 8 * (size_t)S.d.n, cudaMemcpyDeviceToDevice, s));
        if (S.d.zlo) DD_CUDA(dd, cudaMemcpyAsync(S.xe, x + off - S.d.nxy, pb, cudaMemcpyDeviceToDevice, s));
        if (S.d.zhi) DD_CUDA(dd, cudaMemcpyAsync(S.x + S.d.n, x + off + S.d.n, pb, cudaMemcpyDeviceToDevice, s));
    }
    int rc = cycle(dd);
    if (rc) return rc;
    for (Slab &S : dd->lv[0])
        DD_CUDA(dd, cudaMemcpyAsync(x + (size_t)S.z0 * S.d.nxy, S.x, 8 * (size_t)S.d.n, cudaMemcpyDeviceToDevice, s));
    DD_CUDA(dd, cudaGetLastError());
    DD_CUDA(dd, cudaStreamSynchronize(s));
    return MG_OK;
}

int mg_dd_solve(mg_dd *dd, const double *b, double *p, mg_stats *st) {
    mg::NvtxRange nvtx_("mg_dd_solve");
    if (!dd) return MG_ERR_ARG;
    if (!b || !p) return dd_fail(dd, MG_ERR_ARG, "null array");
    if (!dd->have_op) return dd_fail(dd, MG_ERR_STATE, "coefficients not set");
    if (dd->mixed) return solve_mixed(dd, b, p, st);
    cudaStream_t s = dd->s;
    EventPair ev;
    DD_CUDA(dd, cudaEventCreate(&ev.e[0]));
    DD_CUDA(dd, cudaEventCreate(&ev.e[1]));
    DD_CUDA(dd, cudaEventRecord(ev.e[0], s));
    const double n = (double)dd->o.nx * dd->o.ny * dd->o.nz;
    // b~ = b - mean(b) slab by slab (the mean from the slabs' partial sums)
    double sb = 0.0;
    for (Slab &S : dd->lv[0]) {
        mg::launch_sum_sumsq<double>(s, S.d.n, b + (size_t)S.z0 * S.d.nxy, dd->partials, dd->red, false);
        double h[2];
        DD_CUDA(dd, cudaMemcpyAsync(h, dd->red, sizeof(h), cudaMemcpyDeviceToHost, s));
        DD_CUDA(dd, cudaStreamSynchronize(s));
        sb += h[0];
    }
    for (Slab &S : dd->lv[0]) {
        mg::count_launch();
        k_sub_scalar<<<blocks_for(S.d.n), kThreads, 0, s>>>(S.d.n, b + (size_t)S.z0 * S.d.nxy, sb / n, S.b);
        DD_CUDA(dd, cudaMemsetAsync(S.xe, 0, 8 * (size_t)(S.d.n + 2 * S.d.nxy), s));
    }
    double t, nb2;
    int rc = slab_sums_b(dd, &t, &nb2);
    if (rc) return rc;
    const double nb = std::sqrt(nb2);
    double hist[MG_HIST_LEN];
    int hn = 0, cycles = 0, status = MG_ERR_NOT_CONVERGED;
    double rr = nb > 0.0 ? 1.0 : 0.0;
    hist[hn++] = rr;
    if (nb == 0.0 || rr <= dd->o.rtol) status = MG_OK;
    const double ih2 = 1.0 / (dd->o.h * dd->o.h);
    while (status == MG_ERR_NOT_CONVERGED && cycles < dd->o.max_cycles) {
        rc = cycle(dd);
        if (rc) return rc;
        double rn2, sp;
        rc = slab_residual_norms(dd, &rn2, &sp);
        if (rc) return rc;
        // zero mean, ghosts included (they hold the neighbours' planes, shifted alike)
        for (Slab &S : dd->lv[0]) mg::launch_add_const(s, S.d.n + 2 * S.d.nxy, S.xe, -sp / n);
        rr = std::sqrt(rn2) * ih2 / nb;
        ++cycles;
        if (hn < MG_HIST_LEN) hist[hn++] = rr;
        if (!std::isfinite(rr) || rr > 1e12) {
            status = MG_ERR_DIVERGED;
            break;
        }
        if (rr <= dd->o.rtol) status = MG_OK;
    }
    // exact zero-mean gauge at exit (the per-cycle shifts use the residual kernel's FP32 sum of x)
    if (nb > 0.0) {
        double sx;
        rc = slab_sum_x(dd, &sx);
        if (rc) return rc;
        for (Slab &S : dd->lv[0]) mg::launch_add_const(s, S.d.n, S.x, -sx / n);
    }
    for (Slab &S : dd->lv[0])
        DD_CUDA(dd, cudaMemcpyAsync(p + (size_t)S.z0 * S.d.nxy, S.x, 8 * (size_t)S.d.n, cudaMemcpyDeviceToDevice, s));
    DD_CUDA(dd, cudaEventRecord(ev.e[1], s));
    DD_CUDA(dd, cudaEventSynchronize(ev.e[1]));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev.e[0], ev.e[1]);
    DD_CUDA(dd, cudaGetLastError());
    if (st) {
        st->status = status;
        st->cycles = cycles;
        st->outer = cycles;
        st->relres = rr;
        for (int q = 0; q < MG_HIST_LEN; ++q) st->relres_hist[q] = q < hn ? hist[q] : 0.0;
        st->ms = ms;
    }
    if (status == MG_ERR_NOT_CONVERGED)
        return dd_fail(dd, status, "not converged: relres %.3e after %d cycles", rr, cycles);
    if (status == MG_ERR_DIVERGED) return dd_fail(dd, status, "diverged: relres %.3e", rr);
    return MG_OK;
}

}  // extern "C"
