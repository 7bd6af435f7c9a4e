// rafem_pcg_csr_noalloc: the persistent FP64 Jacobi-PCG solver applied to a caller-supplied CSR system, with
// every piece of working memory taken from one fixed array that the library owns for the life of the process.
//
// Some callers cannot allocate device memory at the point where they need a solve: code inside a framework whose
// caching allocator already holds the device's memory (a cudaMalloc there may fail, or force the allocator to
// give back its cache), or a time-critical loop that cannot afford the implicit device synchronisation of
// cudaMalloc/cudaFree. This entry point serves them: it calls no allocation routine of any kind, and the caller
// only passes its own inputs and outputs. The call is synchronous: it waits on its stream after checking the
// input and again after the solve, and reads both results back into host variables.
//
// The working memory (Krylov vectors, diagonal positions, per-tile partial sums, work tiles, solver state and
// the grid-barrier word) lives in the file-scope array g_noalloc_scratch below. Host code cannot use that name
// as an address (it names a host-side stand-in), so the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, and then passed to the kernels. The address is kept for the
// life of the process, so it goes stale if the device is reset (cudaDeviceReset reloads the module).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <mutex>

#include "internal.h"

namespace rafem {
namespace {

constexpr int kMaxRows = RAFEM_NOALLOC_MAX_ROWS;
constexpr int kMaxTiles = 4096;
constexpr int kLanes = 8;  // CSR with 8 lanes per row

constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Byte layout of the scratch array.
constexpr size_t kVecBytes = align256((size_t)kMaxRows * sizeof(double));
constexpr size_t kOffVec = 0;                                           // r, u, w, p, s, dinv
constexpr size_t kOffDiag = kOffVec + 6 * kVecBytes;                    // int32 [kMaxRows]
constexpr size_t kOffPartial = kOffDiag + align256((size_t)kMaxRows * 4);  // double [kPartialQ][kMaxTiles]
constexpr size_t kOffTiles = kOffPartial + align256((size_t)kPartialQ * kMaxTiles * 8);  // int32 [3][kMaxTiles]
constexpr size_t kOffInstTiles = kOffTiles + align256((size_t)3 * kMaxTiles * 4);  // int32 [2]
constexpr size_t kOffFlag = kOffInstTiles + 256;                        // int32 bad-input counter
constexpr size_t kOffInst = kOffFlag + 256;                             // InstState
constexpr size_t kOffBar = kOffInst + align256(sizeof(InstState));      // GridBarrier
constexpr size_t kScratchBytes = kOffBar + align256(sizeof(GridBarrier));
static_assert(kScratchBytes <= RAFEM_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the declared size");

static __device__ __align__(256) unsigned char g_noalloc_scratch[RAFEM_NOALLOC_SCRATCH_BYTES];

struct Carve {
    double* vec[6];
    int32_t* diag;
    double* partial;
    int32_t *tile_r0, *tile_r1, *tile_inst, *inst_t0, *inst_t1;
    int32_t* flag;
    InstState* inst;
    GridBarrier* bar;
};

Carve carve(unsigned char* base) {
    Carve c;
    for (int k = 0; k < 6; ++k) c.vec[k] = reinterpret_cast<double*>(base + kOffVec + k * kVecBytes);
    c.diag = reinterpret_cast<int32_t*>(base + kOffDiag);
    c.partial = reinterpret_cast<double*>(base + kOffPartial);
    c.tile_r0 = reinterpret_cast<int32_t*>(base + kOffTiles);
    c.tile_r1 = c.tile_r0 + kMaxTiles;
    c.tile_inst = c.tile_r1 + kMaxTiles;
    c.inst_t0 = reinterpret_cast<int32_t*>(base + kOffInstTiles);
    c.inst_t1 = c.inst_t0 + 1;
    c.flag = reinterpret_cast<int32_t*>(base + kOffFlag);
    c.inst = reinterpret_cast<InstState*>(base + kOffInst);
    c.bar = reinterpret_cast<GridBarrier*>(base + kOffBar);
    return c;
}

// Checks the CSR arrays (monotone row pointers, columns in range, a stored diagonal in every row), records the
// diagonal positions and builds the work tiles. Counts every bad row into *flag (cleared by the caller first).
__global__ void k_noalloc_prepare(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                  int32_t* __restrict__ diag, int n_tiles, int rows_per_tile, int32_t* tile_r0,
                                  int32_t* tile_r1, int32_t* tile_inst, int32_t* inst_t0, int32_t* inst_t1,
                                  int32_t* flag) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    for (int row = tid; row < n; row += stride) {
        const int s = rp[row], e = rp[row + 1];
        int d = -1;
        bool ok = s <= e && s >= 0;
        for (int k = s; ok && k < e; ++k) {
            const int c = ci[k];
            if (c < 0 || c >= n) ok = false;
            if (c == row) d = k;
        }
        if (!ok || d < 0) {
            atomicAdd(flag, 1);
            d = 0;
        }
        diag[row] = d;
    }
    for (int t = tid; t < n_tiles; t += stride) {
        const long long r0 = (long long)t * rows_per_tile, r1 = r0 + rows_per_tile;
        tile_r0[t] = (int32_t)(r0 < n ? r0 : n);
        tile_r1[t] = (int32_t)(r1 < n ? r1 : n);
        tile_inst[t] = 0;
    }
    if (tid == 0) {
        *inst_t0 = 0;
        *inst_t1 = n_tiles;
    }
}

// Device address of the scratch array, looked up once per device (with that device current).
std::mutex g_mutex;
void* g_addr[128] = {};

cudaError_t scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_addr[dev]);
    return cudaSuccess;
}

int to_status(cudaError_t e) { return e == cudaSuccess ? RAFEM_OK : RAFEM_ERR_CUDA; }

}  // namespace
}  // namespace rafem

using namespace rafem;

extern "C" int rafem_pcg_csr_noalloc(int32_t n_rows, const int32_t* row_ptr, const int32_t* col, const double* vals,
                                     const double* b, double* x, double tol, int32_t max_iter, void* stream,
                                     rafem_step_stats* stats) {
    if (stats) *stats = rafem_step_stats{};
    if (n_rows < 1 || n_rows > kMaxRows || !row_ptr || !col || !vals || !b || !x || !(tol > 0) || max_iter < 1)
        return RAFEM_ERR_BAD_INPUT;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return to_status(e);
    Carve c = carve(base);

    int block = 0;
    const int maxb = krylov_max_blocks(kLanes, RAFEM_PRECISION_FP64, false, &block);
    if (maxb <= 0) return RAFEM_ERR_CUDA;
    const int rows_per_tile = (n_rows + maxb - 1) / maxb;
    const int n_tiles = (n_rows + rows_per_tile - 1) / rows_per_tile;
    if (n_tiles > kMaxTiles) return RAFEM_ERR_INTERNAL;

    // the bad-row counter must start at zero; the solver state and barrier are reset by the solver launch
    if ((e = cudaMemsetAsync(c.flag, 0, sizeof(int32_t), st)) != cudaSuccess) return to_status(e);
    k_noalloc_prepare<<<(n_rows + 255) / 256, 256, 0, st>>>(n_rows, row_ptr, col, c.diag, n_tiles, rows_per_tile,
                                                             c.tile_r0, c.tile_r1, c.tile_inst, c.inst_t0, c.inst_t1,
                                                             c.flag);
    if ((e = cudaGetLastError()) != cudaSuccess) return to_status(e);
    int32_t bad = 0;
    if ((e = cudaMemcpyAsync(&bad, c.flag, sizeof(bad), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return to_status(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return to_status(e);
    if (bad) return RAFEM_ERR_BAD_INPUT;

    SolveArgs a{};
    a.N = n_rows;
    a.rp = row_ptr;
    a.ci = col;
    a.A = vals;
    a.diag = c.diag;
    a.b = b;
    a.x = x;
    a.r = c.vec[0];
    a.u = c.vec[1];
    a.w = c.vec[2];
    a.p = c.vec[3];
    a.s = c.vec[4];
    a.dinv = c.vec[5];
    a.n_tiles = n_tiles;
    a.tile_r0 = c.tile_r0;
    a.tile_r1 = c.tile_r1;
    a.tile_inst = c.tile_inst;
    a.n_inst = 1;
    a.inst_t0 = c.inst_t0;
    a.inst_t1 = c.inst_t1;
    a.inst = c.inst;
    a.partial = c.partial;
    a.bar = c.bar;
    a.tol = tol;
    a.max_iter = max_iter;
    a.spin_limit_ns = kDefaultWaitNs;
    if ((e = launch_krylov(a, kLanes, RAFEM_PRECISION_FP64, false, std::min(n_tiles, maxb), block, st)) != cudaSuccess)
        return to_status(e);
    InstState s;
    GridBarrier g;
    if ((e = cudaMemcpyAsync(&s, c.inst, sizeof(s), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return to_status(e);
    if ((e = cudaMemcpyAsync(&g, c.bar, sizeof(g), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return to_status(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return to_status(e);
    int status = g.err ? g.err : s.status;
    if (stats) {
        stats->status = status;
        stats->iters_V = s.iters;
        stats->relres_V = s.relres;
    }
    return status;
}
