// Host side of the C ABI declared in include/mg.h: the handle, its one-arena
// device allocation, the V-cycle driver, the FP64 and mixed-precision outer
// loops, the adjoint, and the component entry points.
//
// Memory: every device buffer of a handle is carved out of one cudaMalloc made
// in mg_create (a pool in the sense of the paper's §4.2: allocation happens
// once, never inside a solve).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <new>

#include "mg_internal.cuh"

namespace mg {
unsigned long long launches_total();
}

using mg::Coef;
using mg::Dims;
using mg::i64;

namespace {

struct Level {
    Dims d;
    mg::Lay lay;  // storage of the FP32 arrays of this level
    double h, h2, ih2;
    double *fx64, *fy64, *fz64, *invd64;
    double *d64;            // level 0: sum of the interior face coefficients (FP64 residual)
    float2 *fx2, *fy2, *fz2, *d2;  // MIXED_DF, level 0: coefficients and diagonal as FP32 pairs
    float2 *s2;                    // MIXED_DF, level 0: 1/rho as FP32 pairs (operator from a density)
    float *fx32, *fy32, *fz32;
    double *x64, *b64;      // FP64 path: iterate and RHS, levels >= 1
    float *x32, *b32;       // MIXED inner cycle, all levels (level 0: e and the scaled r)
    float *s1_32, *s2_32;   // MIXED: scratch of the component entry points, all levels
    float *s32;             // MIXED, level 0: 1/rho per cell (used when the operator came from rho)
    // (every FP32 array of a level is stored in that level's layout `lay`)
};

constexpr int kProfEvents = 8192;

}  // namespace

struct mg_handle {
    mg_opts o;
    cudaStream_t s;
    int nlev;
    Level lv[MG_MAX_LEVELS];
    int nc;
    double *pinv, *gj_tmp, *scal;
    double *bt;        // zero-mean fine RHS (scaled by h^2 in the mixed modes)
    float2 *bt2, *p2;  // MIXED_DF: the RHS and the solution as FP32 pairs
    double *partials;  // reduction partials
    // flexible CG (MG_METHOD_FCG): FP32 finest-level vectors (mixed; r and x are the level's
    // b32 and x32), FP64 vectors (MG_FP64), device scalars
    float *cg_z32, *cg_d32, *cg_q32;
    double *cg_r64, *cg_z64, *cg_d64, *cg_q64;
    double *cg_sc;
    double *red;       // device reduction results (16 doubles)
    double *hred;      // mapped pinned host memory: 16 doubles read back from red (and the CG
                       // scalars), then the error word as an unsigned
    double *hred_dev;  // the device-side address of hred
    unsigned *herr;    // = (unsigned *)(hred + 16), host side
    unsigned *err;     // device error word
    void *arena;
    size_t arena_bytes;
    int have_op;
    int sform0;        // level-0 FP32 kernels use s = 1/rho (operator set from a density)
    int inject;        // pending one-shot test faults (MG_INJECT_* bits, mg_debug_inject)
    cudaEvent_t ev0, ev1;
    // the V-cycle below the finest level, recorded once at mg_create as a CUDA graph (its
    // launches use fixed buffers and parameters) and replayed by every cycle; null: launched
    // kernel by kernel
    cudaGraphExec_t tail_exec;
    long long tail_launches;
    // optional per-class timing of level-0 kernels (events recorded around launches)
    int prof_on;
    cudaEvent_t *pev;
    int pev_used;
    int pev_cls[kProfEvents / 2];
    long long prof_count[MG_PROF_NCLASS];
    double prof_ms[MG_PROF_NCLASS];
    char msg[512];
};

namespace {

int fail(mg_handle *h, int code, const char *fmt, ...) {
    if (h) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(h->msg, sizeof(h->msg), fmt, ap);
        va_end(ap);
    }
    return code;
}

// n device doubles to h->hred[k..k+n) (k = dst - h->hred) by a kernel writing mapped host
// memory, not by a copy-engine transfer; the caller synchronises the stream before reading
#define MG_READBACK(h, s, dst, src, n)                                                          \
    do {                                                                                        \
        mg::launch_readback((s), (src), (h)->hred_dev + ((dst) - (h)->hred), (n));               \
        MG_CUDA((h), cudaGetLastError());                                                       \
    } while (0)
#define MG_READBACK_ERR(h, s)                                                                   \
    do {                                                                                        \
        mg::launch_readback_u32((s), (h)->err, reinterpret_cast<unsigned *>((h)->hred_dev + 16)); \
        MG_CUDA((h), cudaGetLastError());                                                       \
    } while (0)

#define MG_CUDA(h, call)                                                                        \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return fail((h), MG_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                                    \
    } while (0)

int check_launch(mg_handle *h, const char *where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail(h, MG_ERR_CUDA, "kernel launch in %s failed: %s", where, cudaGetErrorString(e));
    return MG_OK;
}

int num_levels(int nx, int ny, int nz, int coarsest) {
    int nl = 1;
    while (nx % 2 == 0 && ny % 2 == 0 && nz % 2 == 0) {
        int mx = nx > ny ? nx : ny;
        mx = mx > nz ? mx : nz;
        if (mx <= coarsest) break;
        nx /= 2;
        ny /= 2;
        nz /= 2;
        ++nl;
    }
    return nl;
}

template <typename T>
Coef<T> coef(const Level &L);
template <>
Coef<double> coef<double>(const Level &L) {
    return Coef<double>{L.fx64, L.fy64, L.fz64, L.invd64};
}
// ---- optional timing of level-0 kernels ------------------------------------------
void prof_begin(mg_handle *h, int cls) {
    if (!h->prof_on || h->pev_used + 2 > kProfEvents) return;
    h->pev_cls[h->pev_used / 2] = cls;
    cudaEventRecord(h->pev[h->pev_used], h->s);
}
void prof_end(mg_handle *h) {
    if (!h->prof_on || h->pev_used + 2 > kProfEvents) return;
    cudaEventRecord(h->pev[h->pev_used + 1], h->s);
    h->pev_used += 2;
}
// called after a stream synchronisation: fold recorded pairs into the totals
void prof_collect(mg_handle *h) {
    if (!h->prof_on) return;
    for (int q = 0; q + 1 < h->pev_used; q += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->pev[q], h->pev[q + 1]) == cudaSuccess) {
            int cls = h->pev_cls[q / 2];
            h->prof_count[cls] += 1;
            h->prof_ms[cls] += ms;
        }
    }
    h->pev_used = 0;
}

// ---- the V-cycle below the finest level as a CUDA graph ------------------------------
// Levels 1 .. coarsest run many short launches (about 60 per cycle at 512^3, most of a few
// microseconds); replaying them as one graph removes the per-launch host cost and most of the
// gaps between them.  The graph is recorded once in mg_create (build_tail_graph) from the
// same functions the cycle calls, so a replay launches the same kernels with the same
// arguments in the same order.
}  // namespace

namespace mg {
cudaStream_t swap_handle_stream(mg_handle *h, cudaStream_t s) {
    cudaStream_t o = h->s;
    h->s = s;
    return o;
}
}  // namespace mg

namespace {

void replay_tail(mg_handle *h) {
    if (cudaGraphLaunch(h->tail_exec, h->s) == cudaSuccess) mg::count_launch((int)h->tail_launches);
    // a failed launch leaves its error for the solve's check_launch
}

// ---- FP64 V-cycle: in-place per-colour half sweeps, standalone transfers --------------
// (FP64 arithmetic, not bytes, bounds these kernels on GB300, so they do no
// redundant work; see the fused FP32 passes below for the bandwidth-bound cycle)
void smooth64(mg_handle *h, int l, double *x, const double *b, int sweeps, int order) {
    Level &L = h->lv[l];
    for (int sw = 0; sw < sweeps; ++sw)
        for (int half = 0; half < 2; ++half) {
            if (l == 0) prof_begin(h, MG_PROF_SMOOTH);
            mg::launch_rbgs_half64(h->s, L.d, L.h2, coef<double>(L), b, x, order ? 1 - half : half);
            if (l == 0) prof_end(h);
        }
}

void presmooth_restrict64(mg_handle *h, int l, const double *b, double *x, double *bc, int sweeps) {
    Level &L = h->lv[l];
    smooth64(h, l, x, b, sweeps, 0);
    if (l == 0) prof_begin(h, MG_PROF_RESID_RESTRICT);
    // after a pre-smoothing sweep (black last) every black residual is zero
    if (sweeps > 0 && L.d64)
        mg::launch_rr_red_diag64(h->s, L.d, L.h2, coef<double>(L), L.d64, b, x, bc);
    else
        mg::launch_resid_restrict<double>(h->s, L.d, L.ih2, coef<double>(L), b, x, bc, sweeps > 0);
    if (l == 0) prof_end(h);
}

void prolong_postsmooth64(mg_handle *h, int l, const double *b, const double *ec, double *x, int sweeps) {
    if (l == 0) prof_begin(h, MG_PROF_PROLONG);
    // the first post sweep (black first) overwrites every black cell: correct the red ones only
    mg::launch_prolong<double>(h->s, h->lv[l + 1].d, ec, x, h->o.prolong, sweeps > 0 ? 0 : -1);
    if (l == 0) prof_end(h);
    smooth64(h, l, x, b, sweeps, 1);
}

// one V-cycle on level l for A x = b, x in place (x_zero: x starts at zero)
void vcycle64(mg_handle *h, int l, const double *b, double *x, bool x_zero) {
    if (l == h->nlev - 1) {
        if (l == 0) prof_begin(h, MG_PROF_COARSE);
        mg::launch_coarse_matvec<double>(h->s, h->nc, h->pinv, b, x);
        if (l == 0) prof_end(h);
        return;
    }
    Level &L = h->lv[l], &C = h->lv[l + 1];
    if (x_zero) cudaMemsetAsync(x, 0, sizeof(double) * (size_t)L.d.n, h->s);
    presmooth_restrict64(h, l, b, x, C.b64, h->o.pre);
    if (l == 0) prof_begin(h, MG_PROF_COARSE_LEVELS);
    if (l == 0 && h->tail_exec) replay_tail(h);
    else vcycle64(h, l + 1, C.b64, C.x64, true);
    if (l == 0) prof_end(h);
    prolong_postsmooth64(h, l, b, C.x64, x, h->o.post);
}

// ---- FP32 V-cycle on colour-split levels ------------------------------------------------
const float *sinv32(mg_handle *h, int l) { return (l == 0 && h->sform0) ? h->lv[0].s32 : nullptr; }

void half32(mg_handle *h, int l, const float *b, float *x, int col, bool from_zero) {
    Level &L = h->lv[l];
    if (l == 0) prof_begin(h, MG_PROF_SMOOTH);
    mg::launch_half32(h->s, L.lay, L.h2, sinv32(h, l), L.fx32, L.fy32, L.fz32, b, x, col, from_zero);
    if (l == 0) prof_end(h);
}

// Fused red-black sweeps (finest level, s-form operator, layout permitting): each sweep reads
// x from one buffer and writes both colours to the other.  The second buffer is the level's
// FP32 x-face array, which the s-form operator leaves unused.
bool fused0(const mg_handle *h, int l) {
    return l == 0 && h->o.fused_sweeps && h->sform0 && mg::sweep_fused_ok(h->lv[0].lay);
}

// one fused sweep X -> Y, colour c1 first; with `p` the outer update replaces the store
void sweep_fused(mg_handle *h, const float *b, const float *X, float *Y, int c1, bool from_zero,
                 double *p = nullptr, double alpha = 0.0, double shift = 0.0) {
    Level &L = h->lv[0];
    prof_begin(h, p ? MG_PROF_UPDATE : MG_PROF_SMOOTH);
    const bool inject = (h->inject & MG_INJECT_FUSED_WAIT) != 0;
    h->inject &= ~MG_INJECT_FUSED_WAIT;
    mg::launch_sweep_fused(h->s, L.lay, L.h2, L.s32, b, X, Y, c1, from_zero, p, alpha, shift, h->err, inject);
    prof_end(h);
}

// `sweeps` red-black sweeps in place; order 0 red first, 1 black first; from_zero: x = 0 on entry
void smooth32(mg_handle *h, int l, const float *b, float *x, int sweeps, int order, bool from_zero) {
    if (fused0(h, l) && sweeps > 0) {
        float *buf[2] = {x, h->lv[0].fx32};
        int sw = 0;
        if (sweeps % 2) {  // one sweep as two half sweeps in place: the fused pairs then end in x
            half32(h, l, b, x, order ? 1 : 0, from_zero);
            half32(h, l, b, x, order ? 0 : 1, false);
            sw = 1;
        }
        for (int i = 0; sw < sweeps; ++sw, ++i)  // an even number: x -> scratch -> x ...
            sweep_fused(h, b, buf[i & 1], buf[(i + 1) & 1], order ? 1 : 0, from_zero && sw == 0);
        return;
    }
    for (int sw = 0; sw < sweeps; ++sw) {
        half32(h, l, b, x, order ? 1 : 0, from_zero && sw == 0);
        half32(h, l, b, x, order ? 0 : 1, false);
    }
}

// x <- pre-smoothing (from zero if from_zero), bc = R(b - A x)
void presmooth_restrict32(mg_handle *h, int l, const float *b, float *x, float *bc, int sweeps, bool from_zero) {
    Level &L = h->lv[l], &C = h->lv[l + 1];
    if (sweeps == 0 && from_zero) cudaMemsetAsync(x, 0, sizeof(float) * (size_t)L.d.n, h->s);
    smooth32(h, l, b, x, sweeps, 0, from_zero);
    if (l == 0) prof_begin(h, MG_PROF_RESID_RESTRICT);
    // after a pre-smoothing sweep (black last) every black residual is zero
    mg::launch_resid_restrict32(h->s, L.lay, C.lay, L.ih2, sinv32(h, l), L.fx32, L.fy32, L.fz32, b, x, bc,
                                sweeps > 0);
    if (l == 0) prof_end(h);
}

// The outer update fused into the last half sweep of the finest level (MIXED)
struct OuterUpdate {
    double *p;     // FP64 solution (MIXED)
    float2 *p2;    // double-float solution (MIXED_DF)
    double alpha, shift;
};

// x <- post-smoothing of x + P ec.  With `up` (finest level, sweeps >= 1), the last (red)
// half sweep adds alpha * x - shift to the FP64 solution instead of storing x.
void prolong_postsmooth32(mg_handle *h, int l, const float *b, const float *ec, float *x, int sweeps,
                          const OuterUpdate *up = nullptr) {
    Level &L = h->lv[l], &C = h->lv[l + 1];
    if (l == 0) prof_begin(h, MG_PROF_PROLONG);
    // the first post sweep (black first) overwrites every black cell: correct the red ones only
    mg::launch_prolong32(h->s, L.lay, C.lay, ec, x, h->o.prolong, sweeps > 0 ? 0 : -1);
    if (l == 0) prof_end(h);
    if (!up) {
        smooth32(h, l, b, x, sweeps, 1, false);
        return;
    }
    if (fused0(h, l) && up->p) {
        // sweeps - 1 fused sweeps alternating between the buffers, then the fused sweep whose
        // second colour goes (with the first) into the FP64 solution
        float *buf[2] = {x, h->lv[0].fx32};
        for (int i = 0; i < sweeps - 1; ++i) sweep_fused(h, b, buf[i & 1], buf[(i + 1) & 1], 1, false);
        sweep_fused(h, b, buf[(sweeps - 1) & 1], buf[sweeps & 1], 1, false, up->p, up->alpha, up->shift);
        return;
    }
    smooth32(h, l, b, x, sweeps - 1, 1, false);
    half32(h, l, b, x, 1, false);
    prof_begin(h, MG_PROF_UPDATE);
    mg::launch_half32_update(h->s, L.lay, L.h2, sinv32(h, l), L.fx32, L.fy32, L.fz32, b, x, up->p, up->p2,
                             up->alpha, up->shift);
    prof_end(h);
}

// one V-cycle on level l for A x = b from x = 0 (or, with from_zero false, from the x passed
// in); result in x (or, with `up` on level 0, added to the FP64 solution by the last half sweep)
void vcycle32(mg_handle *h, int l, const float *b, float *x, const OuterUpdate *up = nullptr,
              bool from_zero = true) {
    Level &L = h->lv[l];
    if (l == h->nlev - 1) {
        if (l == 0) prof_begin(h, MG_PROF_COARSE);
        mg::launch_coarse_matvec32(h->s, L.lay, h->pinv, b, x);
        if (l == 0) prof_end(h);
        return;
    }
    Level &C = h->lv[l + 1];
    presmooth_restrict32(h, l, b, x, C.b32, h->o.pre, from_zero);
    if (l == 0) prof_begin(h, MG_PROF_COARSE_LEVELS);
    if (l == 0 && h->tail_exec) replay_tail(h);
    else vcycle32(h, l + 1, C.b32, C.x32);
    if (l == 0) prof_end(h);
    prolong_postsmooth32(h, l, b, C.x32, x, h->o.post, up);
}

// Record levels 1 .. coarsest of one V-cycle (FP64 or FP32, as the handle's cycle) on a private
// stream under capture; nothing runs.  Without a graph (capture or instantiation refused) the
// cycle launches the kernels itself.
void build_tail_graph(mg_handle *h) {
    h->tail_exec = nullptr;
    h->tail_launches = 0;
    if (h->nlev < 2) return;
    cudaStream_t cap = nullptr;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    cudaStream_t saved = h->s;
    h->s = cap;
    const unsigned long long l0 = mg::launches_total();
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        if (h->o.precision == MG_FP64) vcycle64(h, 1, h->lv[1].b64, h->lv[1].x64, true);
        else vcycle32(h, 1, h->lv[1].b32, h->lv[1].x32);
        ok = cudaStreamEndCapture(cap, &g) == cudaSuccess && g != nullptr;
    }
    const long long n = (long long)(mg::launches_total() - l0);
    mg::count_launch((int)-n);  // recorded, not run
    h->s = saved;
    if (ok && cudaGraphInstantiate(&h->tail_exec, g, 0) != cudaSuccess) h->tail_exec = nullptr;
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    cudaGetLastError();
    h->tail_launches = h->tail_exec ? n : 0;
}

// ---- set-up of the operator hierarchy -------------------------------------------------
int finish_operator(mg_handle *h) {
    cudaStream_t s = h->s;
    for (int l = 0; l + 1 < h->nlev; ++l) {
        Level &F = h->lv[l], &C = h->lv[l + 1];
        mg::launch_coarsen(s, F.d, F.fx64, F.fy64, F.fz64, C.fx64, C.fy64, C.fz64);
    }
    bool mixed = h->o.precision != MG_FP64;
    for (int l = 0; l < h->nlev; ++l) {
        Level &L = h->lv[l];
        mg::launch_invdiag(s, L.d, L.fx64, L.fy64, L.fz64, L.invd64, L.d64);
        if (mixed && !(l == 0 && h->sform0)) {  // the s-form finest level has no FP32 faces
            mg::launch_pack64to32(s, L.lay, L.fx64, L.fx32);
            mg::launch_pack64to32(s, L.lay, L.fy64, L.fy32);
            mg::launch_pack64to32(s, L.lay, L.fz64, L.fz32);
        }
    }
    if (h->o.precision == MG_MIXED_DF) {
        Level &F = h->lv[0];
        mg::launch_split(s, F.d.n, F.fx64, F.fx2);
        mg::launch_split(s, F.d.n, F.fy64, F.fy2);
        mg::launch_split(s, F.d.n, F.fz64, F.fz2);
        mg::launch_split(s, F.d.n, F.d64, F.d2);
    }
    // dense pseudo-inverse of the coarsest operator
    Level &C = h->lv[h->nlev - 1];
    mg::launch_coarse_assemble(s, C.d, C.ih2, C.fx64, C.fy64, C.fz64, h->pinv, h->scal);
    mg::launch_gj_blocked(s, h->nc, h->pinv, h->gj_tmp);  // in place, 32 pivots per step
    mg::launch_pinv_finish(s, h->nc, h->pinv, h->scal);
    prof_end(h);  // MG_PROF_SETUP, begun by the caller
    int st = check_launch(h, "operator set-up");
    if (st) return st;
    MG_READBACK_ERR(h, s);
    MG_CUDA(h, cudaStreamSynchronize(s));
    const unsigned herr = *h->herr;
    if (herr) {
        h->have_op = 0;
        return fail(h, MG_ERR_DENSITY, "density / face coefficients must be finite and > 0");
    }
    h->have_op = 1;
    return MG_OK;
}

// ---- flexible CG preconditioned by one V-cycle ------------------------------------------
// k iterations on the finest FP32 level for A32 x = r from x = 0 (r = the level's b32, the
// scaled outer residual, overwritten by the updated residual; x = the level's x32).  Every
// scalar stays on the device (slots of cg_sc); r . z of the current and the previous
// iteration alternate between two slots.
void inner_fcg32(mg_handle *h, int k) {
    Level &F = h->lv[0];
    cudaStream_t s = h->s;
    const i64 n = F.d.n;
    cudaMemsetAsync(F.x32, 0, sizeof(float) * (size_t)n, s);
    for (int j = 0; j < k; ++j) {
        const int rz_cur = (j & 1) ? mg::CG_RZ1 : mg::CG_RZ0, rz_prev = (j & 1) ? mg::CG_RZ0 : mg::CG_RZ1;
        vcycle32(h, 0, F.b32, h->cg_z32);  // z = V(r)
        mg::launch_cg_dots32(s, n, F.b32, h->cg_z32, h->cg_q32, h->partials, h->cg_sc, rz_cur);
        mg::launch_cg_dir32(s, n, h->cg_z32, h->cg_d32, h->cg_sc, j == 0, rz_prev);
        mg::launch_cg_apply32(s, F.lay, F.ih2, sinv32(h, 0), F.fx32, F.fy32, F.fz32, h->cg_d32, h->cg_q32,
                              h->partials, h->cg_sc);
        mg::launch_cg_update32(s, n, F.x32, F.b32, h->cg_d32, h->cg_q32, h->cg_sc, rz_cur);
    }
}

// ---- adaptive inner cycles (mixed V-cycle iteration, inner_cycles 0) ----------------------
// Each outer iteration costs an FP64 residual (bound by the FP64 pipe) besides its V-cycles;
// running as many V-cycles per outer iteration as the tolerance still needs, and no more,
// spends the fewest residuals without adding V-cycles.  The contraction per V-cycle rho is
// taken from the last outer iteration, and the next iteration runs
//     k = ceil(log(rtol / rr) / log(rho) + margin),   1 <= k <= kMaxAdaptive,
// V-cycles (margin 0.25 of a cycle: a slightly optimistic rho would otherwise cost a whole
// extra outer iteration).  At most 6: the inner cycles work on one FP32-scaled residual; at
// 512^3 five, six, seven and eight cycles per outer residual all contract by 0.50-0.53 per
// cycle, but seven and eight round the cycle count up (28 and 32 forward V-cycles against 24),
// while six needs 24 + 30 V-cycles with 4 + 5 FP64 residuals where five needs 5 + 6.
constexpr int kFirstAdaptive = 6, kMaxAdaptive = 6;

int next_inner(double rr_prev, double rr, int k, double rtol) {
    if (!(rr > 0.0) || !(rr_prev > 0.0) || !(rtol > 0.0) || rr <= rtol) return k;
    double rho = std::pow(rr / rr_prev, 1.0 / k);
    if (!(rho > 0.0)) rho = 0.01;
    if (rho > 0.95) rho = 0.95;
    if (rho < 0.01) rho = 0.01;
    const double m = std::log(rtol / rr) / std::log(rho) + 0.25;
    int kn = (int)std::ceil(m);
    return kn < 1 ? 1 : (kn > kMaxAdaptive ? kMaxAdaptive : kn);
}

// ---- one solve A x = b - mean(b), zero-mean x -------------------------------------------
int solve_impl(mg_handle *h, const double *b, double *p, int warm, mg_stats *st) {
    cudaStream_t s = h->s;
    Level &F = h->lv[0];
    const i64 n = F.d.n;
    int hist_n = 0;
    double hist[MG_HIST_LEN];
    MG_CUDA(h, cudaEventRecord(h->ev0, s));
    // b~ = b - mean(b), |b~|
    // the mixed modes keep b~ scaled by h^2 (what their outer residual kernels consume)
    const bool mixed = h->o.precision != MG_FP64;
    const bool df = h->o.precision == MG_MIXED_DF;
    const double bscale = mixed ? F.h2 : 1.0;
    mg::launch_sum_sumsq<double>(s, n, b, h->partials, h->red, false);
    mg::launch_sub_mean(s, n, b, h->red, bscale, h->bt, h->partials, h->red + 2);
    MG_READBACK(h, s, h->hred, h->red, 4);
    MG_CUDA(h, cudaStreamSynchronize(s));
    int rc = check_launch(h, "rhs preparation");
    if (rc) return rc;
    const double nb = std::sqrt(h->hred[2]) / bscale;
    if (!std::isfinite(nb)) return fail(h, MG_ERR_ARG, "right-hand side is not finite");
    if (df && !(nb < 1e30)) return fail(h, MG_ERR_ARG, "MG_MIXED_DF needs |b - mean b| < 1e30");
    int status = MG_OK;
    int cycles = 0, outer = 0;
    // V-cycles per outer iteration; inner_cycles 0 (mixed V-cycle iteration): chosen per outer
    // iteration from the contraction observed so far (kFirstAdaptive for the first)
    const bool adaptive = mixed && h->o.inner_cycles == 0;
    int inner = mixed ? (adaptive ? kFirstAdaptive : h->o.inner_cycles) : 1;
    const bool fcg = h->o.method == MG_METHOD_FCG;
    double rr = 0.0;
    if (nb == 0.0) {
        MG_CUDA(h, cudaMemsetAsync(p, 0, sizeof(double) * (size_t)n, s));
        hist[hist_n++] = 0.0;
    } else {
        if (warm) {
            mg::launch_sum_sumsq<double>(s, n, p, h->partials, h->red + 4, false);
            MG_READBACK(h, s, h->hred + 4, h->red + 4, 1);
            MG_CUDA(h, cudaStreamSynchronize(s));
            mg::launch_add_const(s, n, p, -h->hred[4] / (double)n);
        } else {
            MG_CUDA(h, cudaMemsetAsync(p, 0, sizeof(double) * (size_t)n, s));
        }
        double scale = 1.0 / nb;  // r32 = scale * r (scale = 1 / previous residual norm)
        const bool fuse = mixed && h->nlev > 1 && h->o.post >= 1 && mg::half32_update_ok(F.lay);
        if (df) {
            mg::launch_split(s, n, h->bt, h->bt2);
            mg::launch_split(s, n, p, h->p2);
        }
        auto residual = [&](bool write32) -> int {
            prof_begin(h, MG_PROF_FINE_RESIDUAL);
            if (df && h->sform0)
                mg::launch_resid_dfs(s, F.d, F.lay, F.s2, h->bt2, h->p2, write32 ? F.b32 : nullptr,
                                     (float)(F.ih2 * scale), h->partials, h->red + 6);
            else if (df)
                mg::launch_resid_df(s, F.d, F.lay, F.fx2, F.fy2, F.fz2, F.d2, h->bt2, h->p2,
                                    write32 ? F.b32 : nullptr, (float)(F.ih2 * scale), h->partials, h->red + 6);
            else
                mg::launch_fine_resid2(s, F.d, F.lay, F.h2, F.fx64, F.fy64, F.fz64, F.d64, h->bt, mixed, p,
                                       write32 ? F.b32 : nullptr, (float)(F.ih2 * scale), h->partials, h->red + 6);
            prof_end(h);
            MG_READBACK(h, s, h->hred + 6, h->red + 6, 2);
            MG_CUDA(h, cudaStreamSynchronize(s));
            prof_collect(h);
            return check_launch(h, "fine residual");
        };
        double rn, mu;
        if (!warm && !df) {
            // p = 0: its residual is b~ itself, of norm nb, and mean(p) = 0; the mixed modes take
            // the scaled FP32 copy the residual kernel would have written (no FP64 pass)
            if (mixed) mg::launch_zero_resid32(s, F.d, F.lay, h->bt, F.ih2 * scale, F.b32);
            rn = nb;
            mu = 0.0;
        } else {
            rc = residual(mixed);
            if (rc) return rc;
            rn = std::sqrt(h->hred[6]) * F.ih2;  // the kernel sums (h^2 r)^2
            mu = h->hred[7] / (double)n;
        }
        rr = rn / nb;
        hist[hist_n++] = rr;
        status = MG_ERR_NOT_CONVERGED;
        if (rr <= h->o.rtol) status = MG_OK;
        if (!mixed && fcg && status == MG_ERR_NOT_CONVERGED) {
            // FP64 flexible CG on A p = b~, preconditioned by one FP64 V-cycle; the stopping
            // test uses the CG-updated residual r, the exit the true residual
            double *r = h->cg_r64, *z = h->cg_z64, *d = h->cg_d64, *q = h->cg_q64;
            mg::launch_residual<double>(s, F.d, F.ih2, coef<double>(F), h->bt, p, r);
            for (int j = 0; j < h->o.max_cycles && status == MG_ERR_NOT_CONVERGED; ++j) {
                const int rz_cur = (j & 1) ? mg::CG_RZ1 : mg::CG_RZ0, rz_prev = (j & 1) ? mg::CG_RZ0 : mg::CG_RZ1;
                vcycle64(h, 0, r, z, true);
                mg::launch_cg_dots64(s, n, r, z, q, h->partials, h->cg_sc, rz_cur);
                mg::launch_cg_dir64(s, n, z, d, h->cg_sc, j == 0, rz_prev);
                mg::launch_cg_apply64(s, F.d, F.ih2, F.fx64, F.fy64, F.fz64, F.d64, d, q, h->partials, h->cg_sc);
                mg::launch_cg_update64(s, n, p, r, d, q, h->cg_sc, rz_cur, h->partials);
                MG_READBACK(h, s, h->hred + 6, h->cg_sc + mg::CG_RR, 1);
                MG_CUDA(h, cudaStreamSynchronize(s));
                rr = std::sqrt(h->hred[6]) / nb;
                cycles = outer = j + 1;
                if (hist_n < MG_HIST_LEN) hist[hist_n++] = rr;
                if (!std::isfinite(rr) || rr > 1e12) {
                    status = MG_ERR_DIVERGED;
                    break;
                }
                if (rr <= h->o.rtol) status = MG_OK;
            }
            // the true residual of the final iterate
            rc = residual(false);
            if (rc) return rc;
            rr = std::sqrt(h->hred[6]) * F.ih2 / nb;
            if (status == MG_OK && rr > h->o.rtol) status = MG_ERR_NOT_CONVERGED;
        }
        for (int it = 1; !(fcg && !mixed) && status == MG_ERR_NOT_CONVERGED; ++it) {
            // the adaptive count shrinks to the cycles left; a fixed count stops before exceeding
            if (adaptive && cycles + inner > h->o.max_cycles) inner = h->o.max_cycles - cycles;
            if (inner < 1 || cycles + inner > h->o.max_cycles) break;
            if (mixed && fcg) {
                // inner_cycles flexible-CG iterations in FP32, then the outer update
                inner_fcg32(h, inner);
                prof_begin(h, MG_PROF_UPDATE);
                if (df) mg::launch_update_df(s, F.d, F.lay, h->p2, F.x32, 1.0 / scale, mu);
                else mg::launch_update(s, F.d, F.lay, p, F.x32, 1.0 / scale, mu);
                prof_end(h);
                scale = 1.0 / rn;
            } else if (mixed) {
                // inner_cycles FP32 V-cycles on the scaled residual: the first from zero, the
                // next ones continuing from the previous correction
                for (int q = 0; q + 1 < inner; ++q) vcycle32(h, 0, F.b32, F.x32, nullptr, q == 0);
                if (fuse) {
                    OuterUpdate up{df ? nullptr : p, df ? h->p2 : nullptr, 1.0 / scale, mu};
                    vcycle32(h, 0, F.b32, F.x32, &up, inner == 1);
                } else {
                    vcycle32(h, 0, F.b32, F.x32, nullptr, inner == 1);
                    prof_begin(h, MG_PROF_UPDATE);
                    if (df) mg::launch_update_df(s, F.d, F.lay, h->p2, F.x32, 1.0 / scale, mu);
                    else mg::launch_update(s, F.d, F.lay, p, F.x32, 1.0 / scale, mu);
                    prof_end(h);
                }
                scale = 1.0 / rn;
            } else {
                vcycle64(h, 0, h->bt, p, false);
            }
            rc = residual(mixed);
            if (rc) return rc;
            rn = std::sqrt(h->hred[6]) * F.ih2;
            if (h->inject & MG_INJECT_DIVERGE) {  // test fault: the read-back norm is lost
                h->inject &= ~MG_INJECT_DIVERGE;
                rn = HUGE_VAL;
            }
            double mu_new = h->hred[7] / (double)n;
            if (!mixed) mg::launch_add_const(s, n, p, -mu_new);  // FP64 path: zero mean each cycle
            mu = mixed ? mu_new : 0.0;
            const double rr_prev = rr;
            rr = rn / nb;
            cycles += inner;
            if (adaptive) inner = next_inner(rr_prev, rr, inner, h->o.rtol);
            outer = it;
            if (hist_n < MG_HIST_LEN) hist[hist_n++] = rr;
            if (!std::isfinite(rr) || rr > 1e12) {
                status = MG_ERR_DIVERGED;
                break;
            }
            if (rr <= h->o.rtol) status = MG_OK;
        }
        if (df) mg::launch_join(s, n, h->p2, p);
        // exact zero-mean gauge at exit (the per-iteration shifts use an FP32 sum)
        mg::launch_sum_sumsq<double>(s, n, p, h->partials, h->red + 12, false);
        MG_READBACK(h, s, h->hred + 12, h->red + 12, 1);
        MG_CUDA(h, cudaStreamSynchronize(s));
        mg::launch_add_const(s, n, p, -h->hred[12] / (double)n);
        (void)mu;
    }
    MG_CUDA(h, cudaEventRecord(h->ev1, s));
    MG_CUDA(h, cudaEventSynchronize(h->ev1));
    rc = check_launch(h, "solve");
    if (rc) return rc;
    if (fused0(h, 0)) {  // a bounded wait of a fused sweep that ran out sets bit 4
        MG_READBACK_ERR(h, s);
        MG_CUDA(h, cudaStreamSynchronize(s));
        const unsigned herr = *h->herr;
        if (herr & 4u) {
            MG_CUDA(h, cudaMemsetAsync(h->err, 0, sizeof(unsigned), s));
            return fail(h, MG_ERR_CUDA, "a fused sweep gave up waiting for its shared-memory copies");
        }
    }
    if (st) {
        st->status = status;
        st->cycles = cycles;
        st->outer = outer;
        st->relres = rr;
        for (int q = 0; q < MG_HIST_LEN; ++q) st->relres_hist[q] = q < hist_n ? hist[q] : 0.0;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, h->ev0, h->ev1);
        st->ms = ms;
    }
    if (status == MG_ERR_NOT_CONVERGED)
        fail(h, status, "not converged: relres %.3e after %d cycles (rtol %.3e)", rr, cycles, h->o.rtol);
    if (status == MG_ERR_DIVERGED) fail(h, status, "diverged: relres %.3e at cycle %d", rr, cycles);
    return status;
}

// smoothing components need the sweep scratch of the handle's own V-cycle precision
int check_cycle_dtype(mg_handle *h, int dtype) {
    if ((dtype == MG_F64) != (h->o.precision == MG_FP64))
        return fail(h, MG_ERR_ARG, "smoothing components run in the handle's V-cycle precision "
                                   "(MG_F64 for MG_FP64 handles, MG_F32 for the mixed modes)");
    return MG_OK;
}

int check_level(mg_handle *h, int level, int dtype, bool need_coarser) {
    if (!h) return MG_ERR_ARG;
    if (level < 0 || level >= h->nlev || (need_coarser && level >= h->nlev - 1))
        return fail(h, MG_ERR_ARG, "level %d out of range (levels: %d)", level, h->nlev);
    if (dtype != MG_F64 && dtype != MG_F32) return fail(h, MG_ERR_ARG, "dtype must be MG_F64 or MG_F32");
    if (dtype == MG_F32 && h->o.precision == MG_FP64)
        return fail(h, MG_ERR_ARG, "MG_F32 components need a mixed-precision handle");
    if (!h->have_op) return fail(h, MG_ERR_STATE, "coefficients not set");
    return MG_OK;
}

}  // namespace

namespace mg {
Lay handle_lay32(mg_handle *h, int l) { return h->lv[l].lay; }
float *handle_b32(mg_handle *h, int l) { return h->lv[l].b32; }
float *handle_x32(mg_handle *h, int l) { return h->lv[l].x32; }
void handle_vcycle32(mg_handle *h, int l, bool recording) {
    // under a stream capture the coarse levels are recorded launch by launch, not as a replay
    // of the handle's own graph
    cudaGraphExec_t tail = h->tail_exec;
    if (recording) h->tail_exec = nullptr;
    vcycle32(h, l, h->lv[l].b32, h->lv[l].x32);
    h->tail_exec = tail;
}
int handle_first_inner() { return kFirstAdaptive; }
int handle_next_inner(double rr_prev, double rr, int k, double rtol) { return next_inner(rr_prev, rr, k, rtol); }
}  // namespace mg

extern "C" {

void mg_default_opts(mg_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->nx = o->ny = o->nz = 32;
    o->h = 1.0 / 32;
    o->precision = MG_FP64;
    o->pre = o->post = 2;
    o->coarsest = 4;
    o->prolong = MG_PROLONG_TRILINEAR;
    o->rtol = 1e-10;
    o->max_cycles = 200;
    o->warm_start = 0;
    o->inner_cycles = 1;
    o->method = MG_METHOD_VCYCLE;
    o->fused_sweeps = 0;
}

int mg_create(const mg_opts *o, void *stream, mg_handle **out) {
    mg::NvtxRange nvtx_("mg_create");
    if (!out) return MG_ERR_ARG;
    *out = nullptr;
    if (!o) return MG_ERR_ARG;
    if (o->nx < 1 || o->ny < 1 || o->nz < 1 || (i64)o->nx * o->ny * o->nz < 2 ||
        (i64)o->nx * o->ny * o->nz > (i64)2000000000 || !(o->h > 0.0) || !std::isfinite(o->h) ||
        (o->precision != MG_FP64 && o->precision != MG_MIXED && o->precision != MG_MIXED_DF) ||
        (o->precision == MG_MIXED_DF && o->nx % 2 != 0) || o->pre < 0 || o->post < 0 ||
        o->pre > 64 || o->post > 64 || o->coarsest < 2 ||
        (o->prolong != MG_PROLONG_TRILINEAR && o->prolong != MG_PROLONG_CONSTANT) || !(o->rtol >= 0.0) ||
        o->max_cycles < 0 || o->inner_cycles < 0 || o->inner_cycles > 8 ||
        (o->precision == MG_FP64 && o->inner_cycles != 1) ||
        (o->inner_cycles == 0 && o->method != MG_METHOD_VCYCLE) ||
        (o->method != MG_METHOD_VCYCLE && o->method != MG_METHOD_FCG) ||
        (o->method == MG_METHOD_FCG && o->precision != MG_FP64 && o->nx % 8 != 0) ||
        (o->fused_sweeps != 0 && o->fused_sweeps != 1))
        return MG_ERR_ARG;
    int nl = num_levels(o->nx, o->ny, o->nz, o->coarsest);
    if (nl > MG_MAX_LEVELS) return MG_ERR_ARG;
    i64 nc = (i64)(o->nx >> (nl - 1)) * (o->ny >> (nl - 1)) * (o->nz >> (nl - 1));
    if (nc > MG_MAX_COARSE) return MG_ERR_ARG;

    mg_handle *h = new (std::nothrow) mg_handle();
    if (!h) return MG_ERR_OOM;
    h->o = *o;
    h->s = (cudaStream_t)stream;
    h->nlev = nl;
    h->nc = (int)nc;
    const bool mixed = o->precision != MG_FP64;
    const bool dfm = o->precision == MG_MIXED_DF;

    // plan the arena: (pointer slot, bytes) pairs, each rounded up to 256 B
    struct Slot {
        void **p;
        size_t bytes;
    };
    Slot slots[16 * MG_MAX_LEVELS + 32];
    int ns = 0;
    auto add = [&](void **p, size_t bytes) { slots[ns++] = Slot{p, (bytes + 255) & ~(size_t)255}; };
    for (int l = 0; l < nl; ++l) {
        Level &L = h->lv[l];
        L.d = mg::make_dims(o->nx >> l, o->ny >> l, o->nz >> l);
        L.lay = mg::make_lay(L.d);
        L.h = std::ldexp(o->h, l);
        L.h2 = L.h * L.h;
        L.ih2 = 1.0 / L.h2;
        size_t n = (size_t)L.d.n;
        add((void **)&L.fx64, 8 * n);
        add((void **)&L.fy64, 8 * n);
        add((void **)&L.fz64, 8 * n);
        if (!mixed) add((void **)&L.invd64, 8 * n);  // only the FP64 smoother divides by the diagonal
        if (l == 0 || !mixed) add((void **)&L.d64, 8 * n);  // FP64 cycle: diagonal-form restriction
        if (mixed) {
            add((void **)&L.fx32, 4 * n);
            add((void **)&L.fy32, 4 * n);
            add((void **)&L.fz32, 4 * n);
            add((void **)&L.x32, 4 * n);
            add((void **)&L.b32, 4 * n);
            add((void **)&L.s1_32, 4 * n);
            add((void **)&L.s2_32, 4 * n);
            if (l == 0) add((void **)&L.s32, 4 * n);
            if (l == 0 && dfm) {
                add((void **)&L.fx2, 8 * n);
                add((void **)&L.fy2, 8 * n);
                add((void **)&L.fz2, 8 * n);
                add((void **)&L.d2, 8 * n);
                add((void **)&L.s2, 8 * n);
            }
        } else if (l > 0) {
            add((void **)&L.x64, 8 * n);
            add((void **)&L.b64, 8 * n);
        }
    }
    add((void **)&h->pinv, 8 * (size_t)nc * nc);
    add((void **)&h->gj_tmp, 8 * (size_t)mg::kGjBlock * mg::kGjBlock);
    add((void **)&h->scal, 8 * 4);
    add((void **)&h->bt, 8 * (size_t)h->lv[0].d.n);
    if (dfm) {
        add((void **)&h->bt2, 8 * (size_t)h->lv[0].d.n);
        add((void **)&h->p2, 8 * (size_t)h->lv[0].d.n);
    }
    add((void **)&h->partials, 16 * (size_t)mg::reduce_blocks(h->lv[0].d.n));
    add((void **)&h->cg_sc, 8 * mg::CG_NSLOT);
    if (o->method == MG_METHOD_FCG) {
        const size_t n0 = (size_t)h->lv[0].d.n;
        if (mixed) {
            add((void **)&h->cg_z32, 4 * n0);
            add((void **)&h->cg_d32, 4 * n0);
            add((void **)&h->cg_q32, 4 * n0);
        } else {
            add((void **)&h->cg_r64, 8 * n0);
            add((void **)&h->cg_z64, 8 * n0);
            add((void **)&h->cg_d64, 8 * n0);
            add((void **)&h->cg_q64, 8 * n0);
        }
    }
    add((void **)&h->red, 8 * 16);
    add((void **)&h->err, 256);
    size_t total = 0;
    for (int q = 0; q < ns; ++q) total += slots[q].bytes;
    cudaError_t e = cudaMalloc(&h->arena, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA;
    }
    h->arena_bytes = total;
    char *cur = (char *)h->arena;
    for (int q = 0; q < ns; ++q) {
        *slots[q].p = cur;
        cur += slots[q].bytes;
    }
    if (cudaHostAlloc((void **)&h->hred, 17 * sizeof(double), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void **)&h->hred_dev, h->hred, 0) != cudaSuccess ||
        cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess) {
        cudaGetLastError();
        if (h->hred) cudaFreeHost(h->hred);
        cudaFree(h->arena);
        delete h;
        return MG_ERR_CUDA;
    }
    h->herr = reinterpret_cast<unsigned *>(h->hred + 16);
    if (cudaMemsetAsync(h->err, 0, 256, h->s) != cudaSuccess) {
        mg_destroy(h);
        return MG_ERR_CUDA;
    }
    build_tail_graph(h);
    h->msg[0] = 0;
    *out = h;
    return MG_OK;
}

int mg_destroy(mg_handle *h) {
    if (!h) return MG_OK;
    cudaStreamSynchronize(h->s);
    if (h->tail_exec) cudaGraphExecDestroy(h->tail_exec);
    if (h->pev) {
        for (int q = 0; q < kProfEvents; ++q) cudaEventDestroy(h->pev[q]);
        delete[] h->pev;
    }
    cudaEventDestroy(h->ev0);
    cudaEventDestroy(h->ev1);
    cudaFreeHost(h->hred);
    cudaFree(h->arena);
    delete h;
    return MG_OK;
}

const char *mg_last_error(const mg_handle *h) { return h ? h->msg : "null handle"; }

int mg_num_levels(const mg_handle *h) { return h ? h->nlev : MG_ERR_ARG; }

int mg_level_dims(const mg_handle *h, int level, int *dims3) {
    if (!h || !dims3 || level < 0 || level >= h->nlev) return MG_ERR_ARG;
    dims3[0] = h->lv[level].d.nx;
    dims3[1] = h->lv[level].d.ny;
    dims3[2] = h->lv[level].d.nz;
    return MG_OK;
}

int mg_density_from_fractions(mg_handle *h, int nfrac, const double *const *frac_dev,
                              const double *rho_phase, double *rho_dev) {
    mg::NvtxRange nvtx_("mg_density_from_fractions");
    if (!h) return MG_ERR_ARG;
    if (nfrac < 1 || nfrac > 4 || !frac_dev || !rho_phase || !rho_dev)
        return fail(h, MG_ERR_ARG, "mg_density_from_fractions: 1..4 fractions and non-null arrays");
    for (int q = 0; q < nfrac; ++q)
        if (!frac_dev[q]) return fail(h, MG_ERR_ARG, "fraction %d is NULL", q);
    prof_begin(h, MG_PROF_DENSITY);
    mg::launch_density(h->s, h->lv[0].d.n, nfrac, frac_dev, rho_phase, rho_dev);
    prof_end(h);
    return check_launch(h, "mg_density_from_fractions");
}

int mg_set_density(mg_handle *h, const double *rho) {
    mg::NvtxRange nvtx_("mg_set_density");
    if (!h) return MG_ERR_ARG;
    if (!rho) return fail(h, MG_ERR_ARG, "rho is NULL");
    h->have_op = 0;
    prof_begin(h, MG_PROF_SETUP);  // ended by finish_operator
    MG_CUDA(h, cudaMemsetAsync(h->err, 0, sizeof(unsigned), h->s));
    Level &F = h->lv[0];
    // s = 1/rho goes through the RHS buffer, which holds nothing between calls
    mg::launch_faces_from_rho(h->s, F.d, rho, h->bt, F.fx64, F.fy64, F.fz64, h->err);
    h->sform0 = h->o.precision != MG_FP64;
    if (h->sform0) mg::launch_pack_inv_rho(h->s, F.lay, h->bt, F.s32, h->o.precision == MG_MIXED_DF ? F.s2 : nullptr);
    return finish_operator(h);
}

int mg_set_face_coeffs(mg_handle *h, const double *bx, const double *by, const double *bz) {
    mg::NvtxRange nvtx_("mg_set_face_coeffs");
    if (!h) return MG_ERR_ARG;
    if (!bx || !by || !bz) return fail(h, MG_ERR_ARG, "face arrays must be non-null");
    h->have_op = 0;
    prof_begin(h, MG_PROF_SETUP);  // ended by finish_operator
    MG_CUDA(h, cudaMemsetAsync(h->err, 0, sizeof(unsigned), h->s));
    Level &F = h->lv[0];
    mg::launch_faces_from_api(h->s, F.d, bx, by, bz, F.fx64, F.fy64, F.fz64, h->err);
    h->sform0 = 0;
    return finish_operator(h);
}

int mg_get_level_faces(mg_handle *h, int level, double *bx, double *by, double *bz) {
    int rc = check_level(h, level, MG_F64, false);
    if (rc) return rc;
    if (!bx || !by || !bz) return fail(h, MG_ERR_ARG, "face arrays must be non-null");
    Level &L = h->lv[level];
    mg::launch_faces_to_api(h->s, L.d, L.fx64, L.fy64, L.fz64, bx, by, bz);
    return check_launch(h, "mg_get_level_faces");
}

int mg_csf_faces(mg_handle *h, const double *f, const double *kappa, double *cx, double *cy,
                 double *cz) {
    mg::NvtxRange nvtx_("mg_csf_faces");
    if (!h) return MG_ERR_ARG;
    if (!f || !kappa || !cx || !cy || !cz) return fail(h, MG_ERR_ARG, "mg_csf_faces: null array");
    mg::launch_csf_faces(h->s, h->lv[0].d, h->o.h, f, kappa, cx, cy, cz);
    return check_launch(h, "mg_csf_faces");
}

int mg_rhs(mg_handle *h, const double *b0, const double *ux, const double *uy, const double *uz,
           const double *csfx, const double *csfy, const double *csfz, double sigma, double *b) {
    mg::NvtxRange nvtx_("mg_rhs");
    if (!h) return MG_ERR_ARG;
    if (!b) return fail(h, MG_ERR_ARG, "mg_rhs: b is NULL");
    bool u = ux || uy || uz;
    if (u && !(ux && uy && uz)) return fail(h, MG_ERR_ARG, "mg_rhs: give all three velocity arrays or none");
    bool csf = csfx || csfy || csfz;
    if (csf && !(csfx && csfy && csfz)) return fail(h, MG_ERR_ARG, "mg_rhs: give all three csf arrays or none");
    if (csf && !h->have_op) return fail(h, MG_ERR_STATE, "mg_rhs: the surface term needs coefficients set");
    if (!std::isfinite(sigma)) return fail(h, MG_ERR_ARG, "mg_rhs: sigma not finite");
    Level &F = h->lv[0];
    prof_begin(h, MG_PROF_RHS);
    mg::launch_rhs(h->s, F.d, h->o.h, b0, u ? ux : nullptr, uy, uz, F.fx64, F.fy64, F.fz64,
                   csf ? csfx : nullptr, csf ? csfy : nullptr, csf ? csfz : nullptr, sigma, b);
    prof_end(h);
    return check_launch(h, "mg_rhs");
}

static bool aligned16(const void *q) { return ((uintptr_t)q & 15u) == 0; }

int mg_solve(mg_handle *h, const double *b, double *p, mg_stats *st) {
    mg::NvtxRange nvtx_("mg_solve");
    if (!h) return MG_ERR_ARG;
    if (!b || !p) return fail(h, MG_ERR_ARG, "mg_solve: null array");
    if (!aligned16(p)) return fail(h, MG_ERR_ARG, "mg_solve: p must be 16-byte aligned");
    if (!h->have_op) return fail(h, MG_ERR_STATE, "mg_solve: coefficients not set");
    h->msg[0] = 0;
    return solve_impl(h, b, p, h->o.warm_start, st);
}

int mg_adjoint(mg_handle *h, const double *w, const double *p, double *lam, float *gbx, float *gby,
               float *gbz, const double *csfx, const double *csfy, const double *csfz, double sigma,
               double *dLdsigma, mg_stats *st) {
    mg::NvtxRange nvtx_("mg_adjoint");
    if (!h) return MG_ERR_ARG;
    if (!w || !p || !lam) return fail(h, MG_ERR_ARG, "mg_adjoint: w, p, lam must be non-null");
    if (!aligned16(lam)) return fail(h, MG_ERR_ARG, "mg_adjoint: lam must be 16-byte aligned");
    bool g = gbx || gby || gbz;
    if (g && !(gbx && gby && gbz)) return fail(h, MG_ERR_ARG, "mg_adjoint: give all three gradients or none");
    bool csf = csfx || csfy || csfz;
    if (csf && !(csfx && csfy && csfz)) return fail(h, MG_ERR_ARG, "mg_adjoint: give all three csf arrays or none");
    if (!h->have_op) return fail(h, MG_ERR_STATE, "mg_adjoint: coefficients not set");
    h->msg[0] = 0;
    int rc = solve_impl(h, w, lam, 0, st);
    if (rc != MG_OK) return rc;
    Level &F = h->lv[0];
    if (g || dLdsigma) {
        prof_begin(h, MG_PROF_ADJOINT_GRAD);
        mg::launch_adjoint_grad(h->s, F.d, h->o.h, lam, p, F.fx64, F.fy64, F.fz64,
                                csf ? csfx : nullptr, csf ? csfy : nullptr, csf ? csfz : nullptr,
                                sigma, gbx, gby, gbz, h->partials, h->red + 8);
        prof_end(h);
        MG_READBACK(h, h->s, h->hred + 8, h->red + 8, 1);
        MG_CUDA(h, cudaStreamSynchronize(h->s));
        prof_collect(h);
        rc = check_launch(h, "adjoint gradient");
        if (rc) return rc;
        if (dLdsigma) *dLdsigma = csf ? h->hred[8] : 0.0;
    }
    return MG_OK;
}

int mg_project(mg_handle *h, const double *p, const double *csfx, const double *csfy, const double *csfz,
               double sigma, const double *ux, const double *uy, const double *uz, double *ox, double *oy,
               double *oz) {
    mg::NvtxRange nvtx_("mg_project");
    if (!h) return MG_ERR_ARG;
    if (!p || !ux || !uy || !uz || !ox || !oy || !oz)
        return fail(h, MG_ERR_ARG, "mg_project: p, u and out arrays must be non-null");
    const int same = (ox == ux) + (oy == uy) + (oz == uz);
    if (same != 0 && same != 3)
        return fail(h, MG_ERR_ARG, "mg_project: out must be all three u arrays (in place) or none of them");
    bool csf = csfx || csfy || csfz;
    if (csf && !(csfx && csfy && csfz)) return fail(h, MG_ERR_ARG, "mg_project: give all three csf arrays or none");
    if (csf && !std::isfinite(sigma)) return fail(h, MG_ERR_ARG, "mg_project: sigma not finite");
    if (!h->have_op) return fail(h, MG_ERR_STATE, "mg_project: coefficients not set");
    Level &F = h->lv[0];
    prof_begin(h, MG_PROF_PROJECT);
    mg::launch_project(h->s, F.d, h->o.h, p, F.fx64, F.fy64, F.fz64, csf ? csfx : nullptr,
                       csf ? csfy : nullptr, csf ? csfz : nullptr, sigma, ux, uy, uz, ox, oy, oz);
    prof_end(h);
    return check_launch(h, "mg_project");
}

int mg_density_grads(mg_handle *h, const double *rho, const float *gbx, const float *gby, const float *gbz,
                     double *drho, int nfrac, const double *rho_phase, double *const *dfrac_dev) {
    mg::NvtxRange nvtx_("mg_density_grads");
    if (!h) return MG_ERR_ARG;
    if (!rho || !gbx || !gby || !gbz || !drho)
        return fail(h, MG_ERR_ARG, "mg_density_grads: rho, gradients and drho must be non-null");
    if (nfrac < 0 || nfrac > 4) return fail(h, MG_ERR_ARG, "mg_density_grads: nfrac must be 0..4");
    if (nfrac > 0) {
        if (!rho_phase || !dfrac_dev)
            return fail(h, MG_ERR_ARG, "mg_density_grads: rho_phase and dfrac_dev needed for nfrac > 0");
        for (int q = 0; q < nfrac; ++q)
            if (!dfrac_dev[q]) return fail(h, MG_ERR_ARG, "mg_density_grads: dfrac %d is NULL", q);
        for (int q = 0; q <= nfrac; ++q)
            if (!std::isfinite(rho_phase[q])) return fail(h, MG_ERR_ARG, "mg_density_grads: rho_phase not finite");
    }
    prof_begin(h, MG_PROF_DENSITY_GRAD);
    mg::launch_density_grads(h->s, h->lv[0].d, rho, gbx, gby, gbz, drho, nfrac, rho_phase, dfrac_dev);
    prof_end(h);
    return check_launch(h, "mg_density_grads");
}

// FP32 components take natural-layout arrays: they are packed into the level's storage
// (scratch s1_32, s2_32, x32 of the level), run through the same kernels the V-cycle
// uses, and unpacked.
int mg_apply(mg_handle *h, int level, int dtype, const void *x, void *y) {
    int rc = check_level(h, level, dtype, false);
    if (rc) return rc;
    if (!x || !y) return fail(h, MG_ERR_ARG, "mg_apply: null array");
    Level &L = h->lv[level];
    if (dtype == MG_F64) {
        mg::launch_apply<double>(h->s, L.d, L.ih2, coef<double>(L), (const double *)x, (double *)y);
    } else {
        mg::launch_pack32(h->s, L.lay, (const float *)x, L.s1_32);
        mg::launch_residual32(h->s, L.lay, L.ih2, sinv32(h, level), L.fx32, L.fy32, L.fz32, nullptr, L.s1_32,
                              L.s2_32, true);
        mg::launch_unpack32(h->s, L.lay, L.s2_32, (float *)y);
    }
    return check_launch(h, "mg_apply");
}

int mg_smooth(mg_handle *h, int level, int dtype, void *x, const void *b, int sweeps, int order) {
    int rc = check_level(h, level, dtype, false);
    if (rc) return rc;
    rc = check_cycle_dtype(h, dtype);
    if (rc) return rc;
    if (!x || !b || sweeps < 0) return fail(h, MG_ERR_ARG, "mg_smooth: bad argument");
    if (sweeps == 0) return MG_OK;
    Level &L = h->lv[level];
    if (dtype == MG_F64) {
        smooth64(h, level, (double *)x, (const double *)b, sweeps, order ? 1 : 0);
    } else {
        mg::launch_pack32(h->s, L.lay, (const float *)x, L.s1_32);
        mg::launch_pack32(h->s, L.lay, (const float *)b, L.s2_32);
        smooth32(h, level, L.s2_32, L.s1_32, sweeps, order ? 1 : 0, false);
        mg::launch_unpack32(h->s, L.lay, L.s1_32, (float *)x);
    }
    return check_launch(h, "mg_smooth");
}

int mg_presmooth_restrict(mg_handle *h, int level, int dtype, void *x, const void *b, int sweeps,
                          int x_is_zero, void *bc) {
    int rc = check_level(h, level, dtype, true);
    if (rc) return rc;
    rc = check_cycle_dtype(h, dtype);
    if (rc) return rc;
    if (!x || !b || !bc || sweeps < 0) return fail(h, MG_ERR_ARG, "mg_presmooth_restrict: bad argument");
    Level &L = h->lv[level], &C = h->lv[level + 1];
    if (dtype == MG_F64) {
        if (x_is_zero) MG_CUDA(h, cudaMemsetAsync(x, 0, 8 * (size_t)L.d.n, h->s));
        presmooth_restrict64(h, level, (const double *)b, (double *)x, (double *)bc, sweeps);
    } else {
        mg::launch_pack32(h->s, L.lay, (const float *)b, L.s2_32);
        if (!x_is_zero) mg::launch_pack32(h->s, L.lay, (const float *)x, L.s1_32);
        presmooth_restrict32(h, level, L.s2_32, L.s1_32, C.s2_32, sweeps, x_is_zero != 0);
        mg::launch_unpack32(h->s, L.lay, L.s1_32, (float *)x);
        mg::launch_unpack32(h->s, C.lay, C.s2_32, (float *)bc);
    }
    return check_launch(h, "mg_presmooth_restrict");
}

int mg_prolong_postsmooth(mg_handle *h, int level, int dtype, const void *ec, void *x, const void *b,
                          int sweeps) {
    int rc = check_level(h, level, dtype, true);
    if (rc) return rc;
    rc = check_cycle_dtype(h, dtype);
    if (rc) return rc;
    if (!x || !b || !ec || sweeps < 0) return fail(h, MG_ERR_ARG, "mg_prolong_postsmooth: bad argument");
    Level &L = h->lv[level], &C = h->lv[level + 1];
    if (dtype == MG_F64) {
        prolong_postsmooth64(h, level, (const double *)b, (const double *)ec, (double *)x, sweeps);
    } else {
        mg::launch_pack32(h->s, L.lay, (const float *)x, L.s1_32);
        mg::launch_pack32(h->s, L.lay, (const float *)b, L.s2_32);
        mg::launch_pack32(h->s, C.lay, (const float *)ec, C.s1_32);
        prolong_postsmooth32(h, level, L.s2_32, C.s1_32, L.s1_32, sweeps);
        mg::launch_unpack32(h->s, L.lay, L.s1_32, (float *)x);
    }
    return check_launch(h, "mg_prolong_postsmooth");
}

int mg_residual(mg_handle *h, int level, int dtype, const void *x, const void *b, void *r,
                double *norm2) {
    int rc = check_level(h, level, dtype, false);
    if (rc) return rc;
    if (!x || !b || !r) return fail(h, MG_ERR_ARG, "mg_residual: null array");
    Level &L = h->lv[level];
    if (dtype == MG_F64) {
        mg::launch_residual<double>(h->s, L.d, L.ih2, coef<double>(L), (const double *)b, (const double *)x, (double *)r);
        if (norm2) mg::launch_sum_sumsq<double>(h->s, L.d.n, (const double *)r, h->partials, h->red + 10, true);
    } else {
        mg::launch_pack32(h->s, L.lay, (const float *)x, L.s1_32);
        mg::launch_pack32(h->s, L.lay, (const float *)b, L.s2_32);
        mg::launch_residual32(h->s, L.lay, L.ih2, sinv32(h, level), L.fx32, L.fy32, L.fz32, L.s2_32, L.s1_32,
                              L.x32, false);
        mg::launch_unpack32(h->s, L.lay, L.x32, (float *)r);
        if (norm2) mg::launch_sum_sumsq<float>(h->s, L.d.n, (const float *)r, h->partials, h->red + 10, true);
    }
    rc = check_launch(h, "mg_residual");
    if (rc) return rc;
    if (norm2) {
        MG_READBACK(h, h->s, h->hred + 10, h->red + 10, 2);
        MG_CUDA(h, cudaStreamSynchronize(h->s));
        *norm2 = std::sqrt(h->hred[11]);
    }
    return MG_OK;
}

int mg_residual_restrict(mg_handle *h, int level, int dtype, const void *x, const void *b, void *bc) {
    int rc = check_level(h, level, dtype, true);
    if (rc) return rc;
    if (!x || !b || !bc) return fail(h, MG_ERR_ARG, "mg_residual_restrict: null array");
    Level &L = h->lv[level], &C = h->lv[level + 1];
    if (dtype == MG_F64) {
        mg::launch_resid_restrict<double>(h->s, L.d, L.ih2, coef<double>(L), (const double *)b, (const double *)x,
                                          (double *)bc, false);
    } else {
        mg::launch_pack32(h->s, L.lay, (const float *)x, L.s1_32);
        mg::launch_pack32(h->s, L.lay, (const float *)b, L.s2_32);
        mg::launch_resid_restrict32(h->s, L.lay, C.lay, L.ih2, sinv32(h, level), L.fx32, L.fy32, L.fz32, L.s2_32,
                                    L.s1_32, C.s2_32, false);
        mg::launch_unpack32(h->s, C.lay, C.s2_32, (float *)bc);
    }
    return check_launch(h, "mg_residual_restrict");
}

int mg_prolong_correct(mg_handle *h, int level, int dtype, const void *ec, void *x) {
    int rc = check_level(h, level, dtype, true);
    if (rc) return rc;
    if (!ec || !x) return fail(h, MG_ERR_ARG, "mg_prolong_correct: null array");
    Level &L = h->lv[level], &C = h->lv[level + 1];
    if (dtype == MG_F64) {
        mg::launch_prolong<double>(h->s, C.d, (const double *)ec, (double *)x, h->o.prolong, -1);
    } else {
        mg::launch_pack32(h->s, L.lay, (const float *)x, L.s1_32);
        mg::launch_pack32(h->s, C.lay, (const float *)ec, C.s1_32);
        mg::launch_prolong32(h->s, L.lay, C.lay, C.s1_32, L.s1_32, h->o.prolong, -1);
        mg::launch_unpack32(h->s, L.lay, L.s1_32, (float *)x);
    }
    return check_launch(h, "mg_prolong_correct");
}

int mg_coarse_solve(mg_handle *h, int dtype, const void *r, void *e) {
    int rc = check_level(h, h ? h->nlev - 1 : 0, dtype, false);
    if (rc) return rc;
    if (!r || !e) return fail(h, MG_ERR_ARG, "mg_coarse_solve: null array");
    Level &L = h->lv[h->nlev - 1];
    if (dtype == MG_F64) {
        mg::launch_coarse_matvec<double>(h->s, h->nc, h->pinv, (const double *)r, (double *)e);
    } else {
        mg::launch_pack32(h->s, L.lay, (const float *)r, L.s1_32);
        mg::launch_coarse_matvec32(h->s, L.lay, h->pinv, L.s1_32, L.s2_32);
        mg::launch_unpack32(h->s, L.lay, L.s2_32, (float *)e);
    }
    return check_launch(h, "mg_coarse_solve");
}

int mg_profile(mg_handle *h, int enable) {
    if (!h) return MG_ERR_ARG;
    MG_CUDA(h, cudaStreamSynchronize(h->s));
    if (enable && !h->pev) {
        h->pev = new (std::nothrow) cudaEvent_t[kProfEvents];
        if (!h->pev) return fail(h, MG_ERR_OOM, "profile events");
        for (int q = 0; q < kProfEvents; ++q) MG_CUDA(h, cudaEventCreate(&h->pev[q]));
    }
    h->prof_on = enable ? 1 : 0;
    h->pev_used = 0;
    for (int c = 0; c < MG_PROF_NCLASS; ++c) {
        h->prof_count[c] = 0;
        h->prof_ms[c] = 0.0;
    }
    return MG_OK;
}

int mg_profile_read(mg_handle *h, int cls, long long *launches, double *ms) {
    if (!h || cls < 0 || cls >= MG_PROF_NCLASS) return MG_ERR_ARG;
    MG_CUDA(h, cudaStreamSynchronize(h->s));
    prof_collect(h);
    if (launches) *launches = h->prof_count[cls];
    if (ms) *ms = h->prof_ms[cls];
    return MG_OK;
}

long long mg_kernel_launches(void) { return (long long)mg::launches_total(); }

int mg_debug_inject(mg_handle *h, int faults) {
    if (!h || (faults & ~(MG_INJECT_FUSED_WAIT | MG_INJECT_DIVERGE))) return MG_ERR_ARG;
    h->inject = faults;
    return MG_OK;
}

}  // extern "C"
