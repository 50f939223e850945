// Fused red-black Gauss-Seidel sweep of the finest FP32 level (colour-split storage,
// coefficients s = 1/rho), staged through shared memory by bulk asynchronous copies.
//
// One sweep updates every cell of the first colour c1 from the old values of the second
// colour c2, then every cell of c2 from the new c1 values.  Two half sweeps stream the
// grid twice (20 B per cell: each reads the other colour, s of both colours and its own
// b, and writes its own colour); the fused sweep streams it once: the old c2 values, s and
// b of both colours are read (10 B per cell) and both colours are written (4 B), 14 B per
// cell.  It reads x from one buffer and writes the new values of both colours to another
// (ping-pong): c1 at a tile's edge is recomputed by every tile that needs it, from old c2
// values that no tile overwrites during the sweep, so tiles never wait for one another.
//
// Tile: TX four-aligned positions k of one colour (2 TX cells of a row) x TY rows, marching
// ZC planes in z.  At step t the tile computes c1 at plane t on rows y0-1 .. y0+TY (one row
// of halo on each side, and the scalar positions k0-1 and k0+TX) and then c2 at plane t-1
// on its own rows, from c1 at planes t-2, t-1, t kept in shared memory.  The arrays of one
// plane that neighbours read (old c2 and s of c2 on rows y0-2 .. y0+TY+1, s of c1 on rows
// y0-1 .. y0+TY; columns k0-4 .. k0+TX+3) form one stage of a ring of kStages = kAhead + 4
// stages: the stage of plane t+1+kAhead is copied in while planes t-2 .. t+1 are in use.
// b, read only at a thread's own cells, goes to registers one plane ahead.  One warp issues
// the copies (cp.async.bulk, one per row and array, completion counted in bytes on the
// stage's mbarrier); every thread waits on the mbarrier of the newest plane before computing.
// Each wait is bounded (about a second): when one runs out the block records an error in the
// device error word (bit 4), waits (bounded again) for the copies it issued and returns;
// blocks that start after that return at once.
//
// The per-cell arithmetic is that of the half-sweep kernels, in the same order, so the fused
// sweep gives bitwise the results of a red and a black half sweep.
#include <cuda_runtime.h>

#include "mg_internal.cuh"

namespace mg {
namespace {

constexpr int TX = 64;               // positions k per tile (one colour)
constexpr int TY = 8;                // rows per tile
constexpr int ZC = 64;               // planes per tile
constexpr int W = TX + 8;            // shared-memory row: k0-4 .. k0+TX+3
constexpr int kAhead = 2;            // planes copied ahead of the newest plane in use
constexpr int kStages = kAhead + 4;  // planes t-2 .. t+1 in use, kAhead in flight
constexpr int R_XO = TY + 4, R_S2 = TY + 4, R_S1 = TY + 2;
constexpr int O_XO = 0, O_S2 = O_XO + R_XO * W, O_S1 = O_S2 + R_S2 * W, STAGE = O_S1 + R_S1 * W;  // floats per stage
constexpr int R_C1 = TY + 2;         // rows of new c1 values kept per plane
constexpr int C1PLANE = R_C1 * W;
constexpr int kThreads = 160;        // 10 rows x 16 vectors of c1; warps 0-3 also do c2
constexpr int kProducerWarp = 4;
constexpr long long kWaitCycles = 1ll << 31;
constexpr size_t kSmemBytes = sizeof(float) * ((size_t)kStages * STAGE + 3 * C1PLANE) + 16 * kStages;
static_assert(kThreads == R_C1 * (TX / 4), "one c1 vector per thread");
static_assert((W * 4) % 16 == 0 && (STAGE * 4) % 16 == 0, "16-byte aligned rows and stages");

struct FUpd {
    double *p;
    float alpha, shift;
};

// ---- mbarrier and bulk-copy primitives (PTX) ------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx_arrive(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait on one phase of a stage's mbarrier: gives up after about 2^31 clock cycles
// (about a second)
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}
// global -> shared bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned),
// completion reported to the mbarrier as transferred bytes
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void *src, unsigned bytes, unsigned bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// ---- one Gauss-Seidel update, the arithmetic of the half-sweep kernels ------------------
// w* are 2 beta of the six faces (0 at walls), x* the neighbours; hh = 2 h^2
__device__ __forceinline__ float gs_update(float w0, float w1, float w2, float w3, float w4, float w5, float xm,
                                           float xp, float ym, float yp, float zm, float zp, float hh, float bb) {
    float num = w0 * xm;
    num += w1 * xp;
    num += w2 * ym;
    num += w3 * yp;
    num += w4 * zm;
    num += w5 * zp;
    const float den = ((w0 + w1) + (w2 + w3)) + (w4 + w5);
    return __fdividef(hh * bb + num, den);
}
__device__ __forceinline__ float gs_from_zero(float w0, float w1, float w2, float w3, float w4, float w5, float hh,
                                              float bb) {
    const float den = ((w0 + w1) + (w2 + w3)) + (w4 + w5);
    return __fdividef(hh * bb, den);
}

__device__ __forceinline__ float4 ld4(const float *a) { return *reinterpret_cast<const float4 *>(a); }
#define F0 make_float4(0.f, 0.f, 0.f, 0.f)

// The same-row window of a 4-vector at smem position e (16-byte aligned): the values at e-1
// and e+4 come from the neighbouring lanes (a warp holds two rows of 16 vectors); the first
// and last lanes of a row read them from the halo columns.  0 beyond the row's ends.
__device__ __forceinline__ void window_ends(const float4 &v4, const float *at, int lane, bool kl, bool kr, float &l,
                                            float &r) {
    l = __shfl_up_sync(0xffffffffu, v4.w, 1);
    r = __shfl_down_sync(0xffffffffu, v4.x, 1);
    if ((lane & 15) == 0) l = kl ? at[-1] : 0.f;
    if ((lane & 15) == 15) r = kr ? at[4] : 0.f;
}

// Four cells of one colour at positions k..k+3 of a row (x = 2k + p): s of the other colour
// in the same row (so4, with the window ends sl, sr), own s (sc4), s of the other colour at
// y-1, y+1, z-1, z+1 (s2..s5), the other colour's x likewise (xo4, xl, xr, ym4, yp4, zm4,
// zp4), own b (b4).  The expressions are those of the half-sweep kernels.
template <bool FROM_ZERO>
__device__ __forceinline__ void vec_update(int p, bool xw0, bool xw1, bool hy0, bool hy1, bool hz0, bool hz1,
                                           const float4 &so4, float sl, float sr, const float4 &sc4,
                                           const float4 &s2, const float4 &s3, const float4 &s4, const float4 &s5,
                                           const float4 &xo4, float xl, float xr, const float4 &ym4,
                                           const float4 &yp4, const float4 &zm4, const float4 &zp4,
                                           const float4 &b4, float hh, float out[4]) {
    const float so[4] = {so4.x, so4.y, so4.z, so4.w}, sc[4] = {sc4.x, sc4.y, sc4.z, sc4.w};
    const float s2v[4] = {s2.x, s2.y, s2.z, s2.w}, s3v[4] = {s3.x, s3.y, s3.z, s3.w};
    const float s4v[4] = {s4.x, s4.y, s4.z, s4.w}, s5v[4] = {s5.x, s5.y, s5.z, s5.w};
    const float xov[4] = {xo4.x, xo4.y, xo4.z, xo4.w};
    const float ymv[4] = {ym4.x, ym4.y, ym4.z, ym4.w}, ypv[4] = {yp4.x, yp4.y, yp4.z, yp4.w};
    const float zmv[4] = {zm4.x, zm4.y, zm4.z, zm4.w}, zpv[4] = {zp4.x, zp4.y, zp4.z, zp4.w};
    const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
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
        if (FROM_ZERO) {
            out[v] = gs_from_zero(w0, w1, w2, w3, w4, w5, hh, bv[v]);
        } else {
            const float xm = p ? xov[v] : (v ? xov[v - 1] : xl);
            const float xp = (v == 3 && xw1) ? 0.f : (p ? (v < 3 ? xov[v + 1] : xr) : xov[v]);
            out[v] = gs_update(w0, w1, w2, w3, w4, w5, xm, xp, ymv[v], ypv[v], zmv[v], zpv[v], hh, bv[v]);
        }
    }
}

struct Geo {
    int hx, ny, nz;
    long long half, dz;  // colour offset, plane stride (ny * hx)
};

// Copies of plane q for the tile (k0, y0) into stage `st` (floats), by one warp; returns
// nothing, arrives on the stage's mbarrier with the exact byte count first.
__device__ __forceinline__ void issue_plane(const Geo &g, int q, int k0, int y0, int c1, bool from_zero,
                                            const float *X, const float *sv, float *stg,
                                            unsigned bar, int lane, bool skip = false) {
    const int c2 = 1 - c1;
    const int ks = k0 - 4 < 0 ? 0 : k0 - 4, ke = k0 + TX + 4 > g.hx ? g.hx : k0 + TX + 4;
    const unsigned rb = (unsigned)(ke - ks) * 4u;
    const int e = ks - (k0 - 4);
    const bool plane_ok = q >= 0 && q < g.nz;
    // row tasks: XO (R_XO), S2 (R_S2), S1 (R_S1)
    constexpr int NT = R_XO + R_S2 + R_S1;
    const float *srcs[2];
    unsigned dsts[2];
    int cnt = 0;
    unsigned mine = 0;
    for (int task = lane; task < NT; task += 32) {
        int r, off, y;
        const float *base;
        if (task < R_XO) {
            r = task; off = O_XO; y = y0 - 2 + r; base = from_zero ? nullptr : X + c2 * g.half;
        } else if (task < R_XO + R_S2) {
            r = task - R_XO; off = O_S2; y = y0 - 2 + r; base = sv + c2 * g.half;
        } else {
            r = task - R_XO - R_S2; off = O_S1; y = y0 - 1 + r; base = sv + c1 * g.half;
        }
        if (!plane_ok || base == nullptr || y < 0 || y >= g.ny) continue;
        srcs[cnt] = base + (long long)q * g.dz + (long long)y * g.hx + ks;
        dsts[cnt] = smem_u32(stg + off + r * W + e);
        ++cnt;
        mine += rb;
    }
    // the expected byte count goes to the mbarrier before any copy can complete
    unsigned total = mine;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
    if (lane == 0) mbar_expect_tx_arrive(bar, total);
    __syncwarp();
    // skip (a test's fault injection): the bytes are expected but no copy is issued, so the
    // stage's phase never completes and its wait runs out, with no copy in flight to the stage
    if (!skip)
        for (int i = 0; i < cnt; ++i) bulk_g2s(dsts[i], srcs[i], rb, bar);
}

template <bool FROM_ZERO, bool UPDATE>
__global__ void __launch_bounds__(kThreads, 3)
    k_sweep_fused(Geo g, float h2, const float *__restrict__ sv, const float *__restrict__ b, const float *X,
                  float *Y, int c1, FUpd up, unsigned *err, int skip_plane) {
    extern __shared__ __align__(16) float sm[];
    float *stages = sm;
    float *c1n = sm + (size_t)kStages * STAGE;  // 3 planes of new c1 values
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(c1n + 3 * C1PLANE);
    __shared__ int abort_flag;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int k0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * ZC;
    const int zend = min(z0 + ZC, g.nz);
    const int c2 = 1 - c1;
    const float hh = 2.f * h2;
    // planes z0-2 .. zend+1 are loaded; plane q uses stage (q - z0 + 2) % kStages
    const int qlo = z0 - 2, qhi = zend + 1;
    auto stage_of = [&](int q) { return (q - qlo) % kStages; };
    auto parity_of = [&](int q) { return (unsigned)(((q - qlo) / kStages) & 1); };
    auto bar_of = [&](int q) { return smem_u32(&bars[stage_of(q)]); };

    if (tid == 0) {
        // a block that already gave up waiting (this launch or an earlier one) stops the rest
        abort_flag = (*(volatile unsigned *)err & 4u) ? 1 : 0;
        for (int s = 0; s < kStages; ++s) mbar_init(smem_u32(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (abort_flag) return;
    if (warp == kProducerWarp)
        for (int q = qlo; q <= min(qlo + kAhead + 1, qhi); ++q)
            issue_plane(g, q, k0, y0, c1, FROM_ZERO, X, sv, stages + (size_t)stage_of(q) * STAGE, bar_of(q), lane);
    int issued = min(qlo + kAhead + 1, qhi);  // newest plane issued
    // fault injection (tests only; -1 otherwise): block (0, 0, 0) skips the copies of plane
    // skip_plane, which it issues inside the loop below
    const int skip_q = (blockIdx.x | blockIdx.y | blockIdx.z) == 0 ? skip_plane : -1000;
    // planes z0-2 and z0-1 are used from the first step on
    bool ok = mbar_wait(bar_of(qlo), parity_of(qlo)) && mbar_wait(bar_of(qlo + 1), parity_of(qlo + 1));

    // c1 task of this thread: row r1 (y0-1+r1), vector v1 (k0+4 v1)
    const int r1 = tid / (TX / 4), v1 = tid % (TX / 4);
    const int y1 = y0 - 1 + r1;
    const int kv1 = k0 + 4 * v1, e1 = 4 + 4 * v1;
    // c1 halo task (threads 0 .. 2 R_C1 - 1): row tid >> 1, k0-1 (even tid) or k0+TX (odd)
    const int rh = tid >> 1, sideh = tid & 1;
    const int yh = y0 - 1 + rh, kh = sideh ? k0 + TX : k0 - 1, eh = sideh ? TX + 4 : 3;
    // c2 task (threads 0 .. 8*16-1): row r2 (y0+r2), vector v2
    const int r2 = tid / (TX / 4), v2 = tid % (TX / 4);
    const int y2 = y0 + r2;
    const int kv2 = k0 + 4 * v2, e2 = 4 + 4 * v2;
    // b is read only at a thread's own cells: it bypasses the stages and is loaded into
    // registers one step ahead (c1 of plane t+1, c2 of plane t, while plane t computes)
    const bool c1row = y1 >= 0 && y1 < g.ny, hrow = tid < 2 * R_C1 && yh >= 0 && yh < g.ny && kh >= 0 && kh < g.hx;
    const bool c2row = tid < TY * (TX / 4) && y2 < g.ny;
    const float *b1p = b + c1 * g.half + (long long)y1 * g.hx + kv1;
    const float *bhp = b + c1 * g.half + (long long)yh * g.hx + kh;
    const float *b2p = b + c2 * g.half + (long long)y2 * g.hx + kv2;
    auto ldb4 = [&](const float *bp, bool row_ok, int q) {
        return (row_ok && q >= 0 && q < g.nz) ? *reinterpret_cast<const float4 *>(bp + (long long)q * g.dz) : F0;
    };
    auto ldb1 = [&](const float *bp, bool row_ok, int q) {
        return (row_ok && q >= 0 && q < g.nz) ? bp[(long long)q * g.dz] : 0.f;
    };
    float4 b1cur = ldb4(b1p, c1row, z0 - 1), b2cur = F0;
    float bhcur = ldb1(bhp, hrow, z0 - 1);

    for (int t = z0 - 1; t <= zend; ++t) {
        // the newest plane in use; the barrier below makes a failed wait everyone's exit
        if (t + 1 <= qhi) ok = ok && mbar_wait(bar_of(t + 1), parity_of(t + 1));
        if (!ok) abort_flag = 1;
        __syncthreads();
        if (abort_flag) break;
        // copies of plane t+1+kAhead into the stage of plane t-3, which the previous step used
        // last (finished by every thread at the barrier above)
        if (issued + 1 <= qhi) {
            const int q = issued + 1;
            if (warp == kProducerWarp)
                issue_plane(g, q, k0, y0, c1, FROM_ZERO, X, sv, stages + (size_t)stage_of(q) * STAGE, bar_of(q),
                            lane, q == skip_q);
            issued = q;
        }
        // b for the next step
        const float4 b1nxt = ldb4(b1p, c1row, t + 1), b2nxt = ldb4(b2p, c2row, t);
        const float bhnxt = ldb1(bhp, hrow, t + 1);
        const float *Sm = stages + (size_t)stage_of(t - 1 >= qlo ? t - 1 : qlo) * STAGE;  // plane t-1
        const float *Sc = stages + (size_t)stage_of(t) * STAGE;                            // plane t
        const float *Sp = stages + (size_t)stage_of(t + 1 <= qhi ? t + 1 : qhi) * STAGE;  // plane t+1
        float *C1c = c1n + (size_t)((t + 3) % 3) * C1PLANE;
        // ---- c1 at plane t, rows y0-1 .. y0+TY (all lanes take part: shuffles) ----
        if (t >= 0 && t < g.nz) {
            const bool hz0 = t > 0, hz1 = t < g.nz - 1;
            {
                const int y = y1;
                const bool hy0 = y > 0, hy1 = y < g.ny - 1;
                const int p = (c1 + y + t) & 1;
                const bool kl = kv1 > 0, kr = kv1 + 4 < g.hx;
                const bool xw0 = (p == 0 && !kl), xw1 = (p == 1 && !kr);
                const int ro = r1 + 1;  // XO / S2 row of y
                const float4 so4 = ld4(Sc + O_S2 + ro * W + e1), sc4 = ld4(Sc + O_S1 + r1 * W + e1);
                const float4 s2 = hy0 ? ld4(Sc + O_S2 + (ro - 1) * W + e1) : F0;
                const float4 s3 = hy1 ? ld4(Sc + O_S2 + (ro + 1) * W + e1) : F0;
                const float4 s4 = hz0 ? ld4(Sm + O_S2 + ro * W + e1) : F0;
                const float4 s5 = hz1 ? ld4(Sp + O_S2 + ro * W + e1) : F0;
                const float4 b4 = b1cur;
                float sl, sr;
                window_ends(so4, Sc + O_S2 + ro * W + e1, lane, kl, kr, sl, sr);
                float4 xo4 = F0, ym4 = F0, yp4 = F0, zm4 = F0, zp4 = F0;
                float xl = 0.f, xr = 0.f;
                if (!FROM_ZERO) {
                    xo4 = ld4(Sc + O_XO + ro * W + e1);
                    if (hy0) ym4 = ld4(Sc + O_XO + (ro - 1) * W + e1);
                    if (hy1) yp4 = ld4(Sc + O_XO + (ro + 1) * W + e1);
                    if (hz0) zm4 = ld4(Sm + O_XO + ro * W + e1);
                    if (hz1) zp4 = ld4(Sp + O_XO + ro * W + e1);
                    window_ends(xo4, Sc + O_XO + ro * W + e1, lane, kl, kr, xl, xr);
                }
                float out[4];
                vec_update<FROM_ZERO>(p, xw0, xw1, hy0, hy1, hz0, hz1, so4, sl, sr, sc4, s2, s3, s4, s5, xo4, xl, xr,
                                      ym4, yp4, zm4, zp4, b4, hh, out);
                if (y >= 0 && y < g.ny) {
                    *reinterpret_cast<float4 *>(C1c + r1 * W + e1) = make_float4(out[0], out[1], out[2], out[3]);
                    if (!UPDATE && r1 >= 1 && r1 <= TY && t >= z0 && t < zend)
                        *reinterpret_cast<float4 *>(Y + c1 * g.half + (long long)t * g.dz + (long long)y * g.hx + kv1) =
                            make_float4(out[0], out[1], out[2], out[3]);
                }
            }
            if (tid < 2 * R_C1 && yh >= 0 && yh < g.ny && kh >= 0 && kh < g.hx) {
                // the scalar positions k0-1 and k0+TX: the same update, one cell
                const int y = yh, k = kh, e = eh;
                const bool hy0 = y > 0, hy1 = y < g.ny - 1;
                const int p = (c1 + y + t) & 1;
                const int ro = rh + 1;
                const float sc = Sc[O_S1 + rh * W + e];
                const bool xw0 = (p == 0 && k == 0), xw1 = (p == 1 && k == g.hx - 1);
                // same-row neighbours of the other colour at k + p - 1 and k + p
                const float sm_ = xw0 ? 0.f : Sc[O_S2 + ro * W + e + p - 1];
                const float sp_ = xw1 ? 0.f : Sc[O_S2 + ro * W + e + p];
                const float w0 = xw0 ? 0.f : sc + sm_;
                const float w1 = xw1 ? 0.f : sc + sp_;
                const float w2 = hy0 ? sc + Sc[O_S2 + (ro - 1) * W + e] : 0.f;
                const float w3 = hy1 ? sc + Sc[O_S2 + (ro + 1) * W + e] : 0.f;
                const float w4 = hz0 ? sc + Sm[O_S2 + ro * W + e] : 0.f;
                const float w5 = hz1 ? sc + Sp[O_S2 + ro * W + e] : 0.f;
                const float bb = bhcur;
                float o;
                if (FROM_ZERO) {
                    o = gs_from_zero(w0, w1, w2, w3, w4, w5, hh, bb);
                } else {
                    const float xm = xw0 ? 0.f : Sc[O_XO + ro * W + e + p - 1];
                    const float xp = xw1 ? 0.f : Sc[O_XO + ro * W + e + p];
                    const float ym = hy0 ? Sc[O_XO + (ro - 1) * W + e] : 0.f;
                    const float yp = hy1 ? Sc[O_XO + (ro + 1) * W + e] : 0.f;
                    const float zm = hz0 ? Sm[O_XO + ro * W + e] : 0.f;
                    const float zp = hz1 ? Sp[O_XO + ro * W + e] : 0.f;
                    o = gs_update(w0, w1, w2, w3, w4, w5, xm, xp, ym, yp, zm, zp, hh, bb);
                }
                C1c[rh * W + e] = o;
            }
        }
        __syncthreads();
        // ---- c2 at plane t-1, rows y0 .. y0+TY-1 (warps 0-3, all lanes take part) ----
        const int z = t - 1;
        if (tid < TY * (TX / 4) && z >= z0 && z < zend) {
            const int y = y2;
            const bool hy0 = y > 0, hy1 = y < g.ny - 1, hz0 = z > 0, hz1 = z < g.nz - 1;
            const int p = (c2 + y + z) & 1;
            const bool kl = kv2 > 0, kr = kv2 + 4 < g.hx;
            const bool xw0 = (p == 0 && !kl), xw1 = (p == 1 && !kr);
            const float *Tm = stages + (size_t)stage_of(z - 1) * STAGE;  // plane z-1 (>= qlo)
            const float *Tc = Sm;                                        // plane z = t-1
            const float *Tp = Sc;                                        // plane z+1 = t
            const float *Cm = c1n + (size_t)((z - 1 + 3) % 3) * C1PLANE;
            const float *Cc = c1n + (size_t)((z + 3) % 3) * C1PLANE;
            const float *Cp = C1c;
            const int rc = r2 + 1;  // C1 / S1 row of y
            const float4 so4 = ld4(Tc + O_S1 + rc * W + e2), sc4 = ld4(Tc + O_S2 + (r2 + 2) * W + e2);
            const float4 s2 = hy0 ? ld4(Tc + O_S1 + (rc - 1) * W + e2) : F0;
            const float4 s3 = hy1 ? ld4(Tc + O_S1 + (rc + 1) * W + e2) : F0;
            const float4 s4 = hz0 ? ld4(Tm + O_S1 + rc * W + e2) : F0;
            const float4 s5 = hz1 ? ld4(Tp + O_S1 + rc * W + e2) : F0;
            const float4 b4 = b2cur;
            const float4 xo4 = ld4(Cc + rc * W + e2);
            const float4 ym4 = hy0 ? ld4(Cc + (rc - 1) * W + e2) : F0;
            const float4 yp4 = hy1 ? ld4(Cc + (rc + 1) * W + e2) : F0;
            const float4 zm4 = hz0 ? ld4(Cm + rc * W + e2) : F0;
            const float4 zp4 = hz1 ? ld4(Cp + rc * W + e2) : F0;
            float sl, sr, xl, xr;
            window_ends(so4, Tc + O_S1 + rc * W + e2, lane, kl, kr, sl, sr);
            window_ends(xo4, Cc + rc * W + e2, lane, kl, kr, xl, xr);
            float out[4];
            vec_update<false>(p, xw0, xw1, hy0, hy1, hz0, hz1, so4, sl, sr, sc4, s2, s3, s4, s5, xo4, xl, xr, ym4,
                              yp4, zm4, zp4, b4, hh, out);
            if (y < g.ny) {
                if (!UPDATE) {
                    *reinterpret_cast<float4 *>(Y + c2 * g.half + (long long)z * g.dz + (long long)y * g.hx + kv2) =
                        make_float4(out[0], out[1], out[2], out[3]);
                } else {
                    // c2 at x = 2k + p, c1 (new, same positions k) at x = 2k + 1 - p
                    const float bk[4] = {xo4.x, xo4.y, xo4.z, xo4.w};
                    double *pr = up.p + ((long long)z * g.ny + y) * (2ll * g.hx) + 2ll * kv2;
                    double2 pvs[4];  // all loads before the first store
#pragma unroll
                    for (int v = 0; v < 4; ++v) pvs[v] = *reinterpret_cast<const double2 *>(pr + 2 * v);
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const double2 pv = pvs[v];
                        const float ea = p ? bk[v] : out[v], eb = p ? out[v] : bk[v];
                        *reinterpret_cast<double2 *>(pr + 2 * v) = make_double2(
                            pv.x + f2d_exact(fmaf(up.alpha, ea, -up.shift)), pv.y + f2d_exact(fmaf(up.alpha, eb, -up.shift)));
                    }
                }
            }
        }
        b1cur = b1nxt;
        b2cur = b2nxt;
        bhcur = bhnxt;
    }
    if (abort_flag) {
        // a wait ran out: record it, then wait (bounded) for every copy this block issued
        if (tid == 0) atomicOr(err, 4u);
        if (tid == 0)  // the copies possibly in flight: the newest plane of each stage
            for (int q = max(qlo, issued - kStages + 1); q <= issued; ++q) mbar_wait(bar_of(q), parity_of(q));
        __syncthreads();
    }
}

}  // namespace

bool sweep_fused_ok(Lay L) { return L.split && L.hx % TX == 0 && L.hx >= TX && L.ny >= 2 && L.nz >= 2; }

size_t sweep_fused_smem() { return kSmemBytes; }

template <bool FZ, bool UPD>
void run_fused(cudaStream_t s, dim3 grid, const Geo &g, float h2, const float *sinv, const float *b, const float *X,
               float *Y, int c1, const FUpd &up, unsigned *err, int skip_plane) {
    // the dynamic shared-memory opt-in is a per-device attribute of the kernel
    static unsigned long long done = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !(done >> dev & 1ull)) {
        cudaFuncSetAttribute(k_sweep_fused<FZ, UPD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
        if (dev >= 0 && dev < 64) done |= 1ull << dev;
    }
    k_sweep_fused<FZ, UPD><<<grid, kThreads, kSmemBytes, s>>>(g, h2, sinv, b, X, Y, c1, up, err, skip_plane);
}

void launch_sweep_fused(cudaStream_t s, Lay L, double h2, const float *sinv, const float *b, const float *X,
                        float *Y, int c1, bool from_zero, double *p, double alpha, double shift, unsigned *err,
                        bool inject_wait) {
    Geo g{L.hx, L.ny, L.nz, (long long)L.half, (long long)L.ny * L.hx};
    // the first plane block (0, 0, 0) issues inside its loop: kAhead + 2 planes past its first (-2)
    const int skip_plane = inject_wait ? kAhead : -1;
    const dim3 grid(L.hx / TX, (L.ny + TY - 1) / TY, (L.nz + ZC - 1) / ZC);
    FUpd up{p, (float)alpha, (float)shift};
    count_launch();
    if (p)
        run_fused<false, true>(s, grid, g, (float)h2, sinv, b, X, Y, c1, up, err, skip_plane);
    else if (from_zero)
        run_fused<true, false>(s, grid, g, (float)h2, sinv, b, X, Y, c1, up, err, skip_plane);
    else
        run_fused<false, false>(s, grid, g, (float)h2, sinv, b, X, Y, c1, up, err, skip_plane);
}

}  // namespace mg
