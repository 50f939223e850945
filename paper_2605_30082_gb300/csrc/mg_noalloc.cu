// Allocation-free dense Neumann solve (mg_dense_solve_noalloc in include/mg.h).
//
// Some callers cannot allocate device memory at the moment they need a
// solve: programs whose device memory is owned by another allocator such as a
// framework's caching allocator (a raw cudaMalloc from inside can fail when
// that pool has reserved the memory, or fragment it), loops held to a fixed
// memory budget, and code that cannot pay for the device-wide synchronisation
// that cudaMalloc and cudaFree may perform.  This entry point serves them: it
// needs no handle and allocates nothing.  Its working memory is one
// file-scope __device__ array, present on every GPU that loads this library
// until the process exits.
//
// Host code may not pass the array's name to a kernel (in host code it names a
// host-side stand-in, not device memory).  The device address is looked up
// once per device with cudaGetSymbolAddress, with that device current, on the
// first call made on that device, and cached.  The call reads its error word
// back and synchronises the caller's stream before it returns.
#include <mutex>

#include "mg_internal.cuh"

namespace {

constexpr int kMaxCells = MG_NOALLOC_MAX_CELLS;
constexpr size_t kPivotDoubles = (size_t)mg::kGjBlock * mg::kGjBlock;
// layout in doubles: M [kMaxCells^2] | W [the inverse of one pivot block of the Gauss-Jordan
// elimination] | fx, fy, fz [kMaxCells each] | scal [4] | error word.  About 2.1 MB in all.
constexpr size_t kScratchDoubles =
    (size_t)kMaxCells * kMaxCells + kPivotDoubles + 3 * (size_t)kMaxCells + 8;

__device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 256;
std::mutex g_mutex;
double *g_scratch_ptr[kMaxDevices];

// device address of the scratch array on the current device (looked up once per device)
int scratch_address(double **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return MG_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return MG_ERR_CUDA;
        }
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return MG_OK;
}

}  // namespace

extern "C" int mg_dense_solve_noalloc(int nx, int ny, int nz, double h, const double *bx,
                                      const double *by, const double *bz, const double *r,
                                      double *e, void *stream) {
    if (nx < 1 || ny < 1 || nz < 1 || !(h > 0.0) || !bx || !by || !bz || !r || !e) return MG_ERR_ARG;
    const long long n = (long long)nx * ny * nz;
    if (n < 2 || n > kMaxCells) return MG_ERR_ARG;  // beyond the fixed scratch: refuse
    double *base = nullptr;
    int rc = scratch_address(&base);
    if (rc != MG_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nc = (int)n;
    double *M = base;
    double *W = M + (size_t)kMaxCells * kMaxCells;
    double *fx = W + kPivotDoubles;
    double *fy = fx + kMaxCells;
    double *fz = fy + kMaxCells;
    double *scal = fz + kMaxCells;
    unsigned *err = reinterpret_cast<unsigned *>(scal + 4);
    mg::Dims d = mg::make_dims(nx, ny, nz);

    // the error word keeps the previous call's value: clear it first
    if (cudaMemsetAsync(err, 0, sizeof(unsigned), s) != cudaSuccess) {
        cudaGetLastError();
        return MG_ERR_CUDA;
    }
    mg::launch_faces_from_api(s, d, bx, by, bz, fx, fy, fz, err);
    // every entry of M, W and scal below is written before it is read
    mg::launch_coarse_assemble(s, d, 1.0 / (h * h), fx, fy, fz, M, scal);
    mg::launch_gj_blocked(s, nc, M, W);  // in place; W holds each pivot block's inverse
    mg::launch_pinv_finish(s, nc, M, scal);
    mg::launch_coarse_matvec<double>(s, nc, M, r, e);
    unsigned herr = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&herr, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return MG_ERR_CUDA;
    }
    return herr ? MG_ERR_DENSITY : MG_OK;
}
