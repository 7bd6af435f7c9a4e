// ILU(0) preconditioner (Sec. II-B: a preconditioner speeds up the Krylov solve): numeric factorisation and the
// standalone application z = (LU)^-1 r. The ILU(0)-PCG solver itself (ilu_ring.cu) streams the factors computed
// here through shared memory.
//
// The factorisation is taken on a symmetric permutation P A P^T whose rows are grouped into levels that never
// depend on each other (greedy colours of the matrix graph, or dependency levels of the original numbering;
// setup.h build_ilu). Each level is a contiguous, 32-aligned range of rows of a SELL-32 layout (the combined
// layout: every row's entries sorted, the diagonal at position dk).
//
// Numeric ILU(0) (once per assembled matrix): the row-by-row IKJ form, one thread per row of a level, levels in
// order (one launch each). Row i reads only rows of earlier levels, which are final. The application runs one
// launch per level: forward levels 0..C-1, then backward levels C-2..0.
#include <cuda_runtime.h>

#include <cmath>

#include "grid_sync.cuh"
#include "internal.h"

namespace rafem {

namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

struct Lay {
    int Np, n_levels;
    const int32_t* lvl;
    const int32_t* sp;
    const int32_t* sc;
    const uint8_t* rlen;
    const uint8_t* dk;
    const int32_t* perm;
};

Lay lay_of(const IluLayout& L) { return Lay{L.Np, L.n_levels, L.lvl, L.sp, L.sc, L.rlen, L.dk, L.perm}; }

// ---- refactorisation ----------------------------------------------------------------------------------------

__global__ void k_ilu_init(long long nnz, const int32_t* __restrict__ pmap, const double* __restrict__ vals,
                           double* __restrict__ Ap, double* __restrict__ F) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nnz; q += (long long)gridDim.x * blockDim.x) {
        const int pm = pmap[q];
        const double v = pm >= 0 ? vals[pm] : (pm == -2 ? 1.0 : 0.0);
        Ap[q] = v;
        F[q] = v;
    }
}

// IKJ ILU(0) of the rows of one level (slices [s0, s1)): for each stored k < i in increasing order
// l_ik = w_k / u_kk, then w_j -= l_ik u_kj for the stored j > k of row k that row i also stores.
__global__ void __launch_bounds__(kThreads) k_ilu_factor(Lay L, double* __restrict__ F, int s0, int s1) {
    const int s = s0 + (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    if (s >= s1) return;
    const int lane = threadIdx.x & 31, row = s * 32 + lane;
    const int len = L.rlen[row], d = L.dk[row], base = L.sp[s];
    for (int k = 0; k < d; ++k) {
        const int pos = base + 32 * k + lane;
        const int c = L.sc[pos];
        const int cl = c & 31, cb = L.sp[c >> 5], cd = L.dk[c], clen = L.rlen[c];
        const double l = F[pos] / F[cb + 32 * cd + cl];
        F[pos] = l;
        int p = k + 1;
        int cp = p < len ? L.sc[base + 32 * p + lane] : 0x7fffffff;
        for (int t = cd + 1; t < clen && p < len; ++t) {
            const int j = L.sc[cb + 32 * t + cl];
            while (cp < j) {
                ++p;
                cp = p < len ? L.sc[base + 32 * p + lane] : 0x7fffffff;
            }
            if (cp == j) F[base + 32 * p + lane] -= l * F[cb + 32 * t + cl];
        }
    }
}

// dinv_i = 1 / u_ii for every padded row (the sweeps multiply instead of dividing: an FP64 division costs about
// ten FP64 operations on a part whose FP64 rate is a small fraction of its FP32 rate)
__global__ void k_ilu_dinv(Lay L, const double* __restrict__ F, double* __restrict__ dinv) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= L.Np) return;
    dinv[row] = 1.0 / F[L.sp[row >> 5] + 32 * L.dk[row] + (row & 31)];
}

// ---- standalone application z = (LU)^-1 r ------------------------------------------------------------------

__global__ void k_ilu_gather(int Np, const int32_t* __restrict__ perm, const double* __restrict__ r,
                             double* __restrict__ rv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < Np) rv[i] = perm[i] >= 0 ? r[perm[i]] : 0.0;
}

__global__ void k_ilu_scatter(int Np, const int32_t* __restrict__ perm, const double* __restrict__ zv,
                              double* __restrict__ z) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < Np && perm[i] >= 0) z[perm[i]] = zv[i];
}

// forward pass of one level: z = rv - L z (lower entries); `last` also divides by the diagonal
__global__ void k_ilu_fwd(Lay L, const double* __restrict__ F, const double* __restrict__ dinv,
                          const double* __restrict__ rv, double* __restrict__ z, int s0, int s1, int last) {
    const int s = s0 + (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    if (s >= s1) return;
    const int lane = threadIdx.x & 31, row = s * 32 + lane, base = L.sp[s], d = L.dk[row];
    double acc = rv[row];
    for (int k = 0; k < d; ++k) {
        const int pos = base + 32 * k + lane;
        acc -= F[pos] * z[L.sc[pos]];
    }
    if (last) acc *= dinv[row];
    z[row] = acc;
}

// backward pass of one level (not the last): z = (z - U z) / u_ii (upper entries)
__global__ void k_ilu_bwd(Lay L, const double* __restrict__ F, const double* __restrict__ dinv, double* __restrict__ z,
                          int s0, int s1) {
    const int s = s0 + (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    if (s >= s1) return;
    const int lane = threadIdx.x & 31, row = s * 32 + lane, base = L.sp[s], d = L.dk[row], len = L.rlen[row];
    double acc = z[row];
    for (int k = d + 1; k < len; ++k) {
        const int pos = base + 32 * k + lane;
        acc -= F[pos] * z[L.sc[pos]];
    }
    z[row] = acc * dinv[row];
}

}  // namespace

cudaError_t launch_ilu_refactor(const IluLayout& L, const double* vals, double* Ap, double* F, double* dinv,
                                cudaStream_t st) {
    k_ilu_init<<<148 * 8, kThreads, 0, st>>>(L.nnz, L.pmap, vals, Ap, F);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const Lay lay = lay_of(L);
    for (int l = 1; l < L.n_levels; ++l) {
        const int s0 = L.h_lvl[l] / 32, s1 = L.h_lvl[l + 1] / 32;
        if (s1 <= s0) continue;
        k_ilu_factor<<<blocks_for(32LL * (s1 - s0)), kThreads, 0, st>>>(lay, F, s0, s1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_ilu_dinv<<<blocks_for(L.Np), kThreads, 0, st>>>(lay, F, dinv);
    return cudaGetLastError();
}

cudaError_t launch_ilu_apply(const IluLayout& L, const double* F, const double* dinv, const double* r, double* z,
                             double* rv, double* zv, cudaStream_t st) {
    const Lay lay = lay_of(L);
    k_ilu_gather<<<blocks_for(L.Np), kThreads, 0, st>>>(L.Np, L.perm, r, rv);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int C = L.n_levels;
    for (int l = 0; l < C; ++l) {
        const int s0 = L.h_lvl[l] / 32, s1 = L.h_lvl[l + 1] / 32;
        if (s1 > s0) k_ilu_fwd<<<blocks_for(32LL * (s1 - s0)), kThreads, 0, st>>>(lay, F, dinv, rv, zv, s0, s1,
                                                                           l == C - 1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    for (int l = C - 2; l >= 0; --l) {
        const int s0 = L.h_lvl[l] / 32, s1 = L.h_lvl[l + 1] / 32;
        if (s1 > s0) k_ilu_bwd<<<blocks_for(32LL * (s1 - s0)), kThreads, 0, st>>>(lay, F, dinv, zv, s0, s1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_ilu_scatter<<<blocks_for(L.Np), kThreads, 0, st>>>(L.Np, L.perm, zv, z);
    return cudaGetLastError();
}

}  // namespace rafem
