// Initial guess by projection onto the recent solutions (an extension of the predictor step of the main loop,
// Sec. II-A: the solution is extrapolated in time before the corrector solves).
//
// With x_n, x_{n-1}, ... the last k solutions (k <= 4) of an SPD system A x = b whose matrix changed since, the
// guess is the A-orthogonal projection of the new solution onto their span:
//     x_0 = D c,   (D^T A D) c = D^T b,
// with D the difference basis d_0 = x_n, d_1 = x_n - x_{n-1}, d_2 = x_n - 2 x_{n-1} + x_{n-2}, d_3 = third
// difference (the same span, much better conditioned than the raw solutions). This minimises the A-norm error
// over the span, which contains every polynomial extrapolation of the same solutions, so the Krylov solve starts
// closer than with the polynomial predictor. Sums run over free rows only (the symmetric lift makes A block
// diagonal with identity Dirichlet rows), and Dirichlet entries are set to their prescribed values.
//
// Four launches per solve, per problem instance of a batch (the solver's work tiles never straddle instances):
//   k_proj_basis:   the basis D at every node, interleaved (one 32-byte sector per node);
//   k_proj_gram:    one pass over A (SELL-32 or CSR) computing A d_i (four FMAs per stored entry: on B300 this
//                   pass is bound by the FP64 pipe), and per chunk the partial sums of G = D^T A D and D^T b;
//   k_proj_solve:   per instance, G scaled to unit diagonal and factorised by Cholesky (the basis shrinks while a
//                   pivot is not positive), c solved;
//   k_proj_combine: x = D c on free rows, history shifted (x_{n-3} <- x_{n-2} <- x_{n-1} <- x_n).
#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"

namespace rafem {

namespace {

constexpr int kThreads = 256;
constexpr int kQ = 14;  // 10 entries of the symmetric 4 x 4 Gram matrix + 4 right-hand sides
constexpr int kChunk = kProjChunk;  // rows per block: tiles are split so that the pass has enough parallelism
constexpr int kBatch = 5;  // interior rows of the Kuhn lattice have 15 entries
constexpr int kSolveThreads = 256;

__device__ __forceinline__ int tri(int i, int l) { return i <= l ? l * (l + 1) / 2 + i : i * (i + 1) / 2 + l; }

// Sums 16 values over the warp by recursive halving: at each of the offsets 16, 8, 4, 2 a lane keeps one half of
// its values and adds the partner's copy of that half, so 16 shuffles replace the 80 of one butterfly per value.
// On return lane l holds the warp total of value l >> 1 (fixed order, deterministic).
__device__ __forceinline__ double warp_sum16(double (&v)[16]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int h = 8; h >= 1; h >>= 1) {
        const bool up = lane & (2 * h);
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const double send = up ? v[i] : v[i + h];
            const double keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 2 * h);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// difference basis at node j from x_n and the history (components i >= k are zero)
__device__ __forceinline__ void basis(const double* x, const double* h1, const double* h2, const double* h3, int k,
                                      int j, double (&d)[4]) {
    const double a = x[j];
    const double b = k > 1 ? h1[j] : 0.0;
    const double c = k > 2 ? h2[j] : 0.0;
    const double e = k > 3 ? h3[j] : 0.0;
    d[0] = a;
    d[1] = k > 1 ? a - b : 0.0;
    d[2] = k > 2 ? a - 2.0 * b + c : 0.0;
    d[3] = k > 3 ? a - 3.0 * b + 3.0 * c - e : 0.0;
}

// Rows of chunk c: chunk c = (tile c / n_sub, part c % n_sub), kChunk rows each (fewer at the tile's end).
__device__ __forceinline__ void chunk_rows(const ProjArgs& a, int c, int& t, int& r0, int& r1) {
    t = c / a.n_sub;
    const int sub = c % a.n_sub;
    r0 = a.tile_r0[t] + sub * kChunk;
    r1 = min(r0 + kChunk, a.tile_r1[t]);
}

// One block per chunk: the basis D at the chunk's nodes, interleaved [node][4] (32 bytes, one sector per node), so
// the gathers of the next pass need no arithmetic.
__global__ void __launch_bounds__(kThreads) k_proj_basis(ProjArgs a) {
    for (int ch = blockIdx.x; ch < a.n_tiles * a.n_sub; ch += gridDim.x) {
        int t, r0, r1;
        chunk_rows(a, ch, t, r0, r1);
        const int k = a.kin[a.tile_inst[t]];
        for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
            double d[4];
            basis(a.x, a.h1, a.h2, a.h3, k, row, d);
            reinterpret_cast<double4*>(a.D)[row] = make_double4(d[0], d[1], d[2], d[3]);
        }
    }
}

// One block per chunk of a tile: A d_i for the chunk's rows, then its partial sums of G and D^T b over free rows.
__global__ void __launch_bounds__(kThreads, 3) k_proj_gram(ProjArgs a) {
    __shared__ double red[kQ][kThreads / 32];
    for (int ch = blockIdx.x; ch < a.n_tiles * a.n_sub; ch += gridDim.x) {
        int t, r0, r1;
        chunk_rows(a, ch, t, r0, r1);
        const int inst = a.tile_inst[t];
        const int k = a.kin[inst];
        double acc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = 0.0;
        if (k > 0) {
            for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
                if (a.bc[row]) continue;
                double y[4] = {0.0, 0.0, 0.0, 0.0};
                int q0, q1, stride;
                if (a.sell) {
                    const int s = row >> 5, base = __ldg(a.rp + s);
                    q0 = base + (row & 31);
                    q1 = __ldg(a.rp + s + 1) + (row & 31);
                    stride = 32;
                } else {
                    q0 = __ldg(a.rp + row);
                    q1 = __ldg(a.rp + row + 1);
                    stride = 1;
                }
                const double2* D = reinterpret_cast<const double2*>(a.D);  // written by the previous launch
                // entries in batches: values and columns first, then the gathers, then the FMAs, so that a row
                // waits for two memory round trips per batch rather than two per entry
                for (int q = q0; q < q1; q += kBatch * stride) {
                    double v[kBatch];
                    int j[kBatch];
#pragma unroll
                    for (int u = 0; u < kBatch; ++u) {
                        const int qq = q + u * stride;
                        const bool ok = qq < q1;
                        v[u] = ok ? __ldg(a.A + qq) : 0.0;
                        j[u] = ok ? (a.ci16 ? row + (int)__ldg(a.ci16 + qq) : __ldg(a.ci + qq)) : row;
                    }
                    double2 lo[kBatch], hi[kBatch];
#pragma unroll
                    for (int u = 0; u < kBatch; ++u) {
                        lo[u] = __ldg(D + 2 * j[u]);
                        hi[u] = __ldg(D + 2 * j[u] + 1);
                    }
#pragma unroll
                    for (int u = 0; u < kBatch; ++u) {
                        y[0] = fma(v[u], lo[u].x, y[0]);
                        y[1] = fma(v[u], lo[u].y, y[1]);
                        y[2] = fma(v[u], hi[u].x, y[2]);
                        y[3] = fma(v[u], hi[u].y, y[3]);
                    }
                }
                const double2 lo = __ldg(D + 2 * row), hi = __ldg(D + 2 * row + 1);
                const double d[4] = {lo.x, lo.y, hi.x, hi.y};
                const double bi = a.b[row];
#pragma unroll
                for (int l = 0; l < 4; ++l) {
#pragma unroll
                    for (int i = 0; i <= l; ++i) acc[l * (l + 1) / 2 + i] = fma(d[i], y[l], acc[l * (l + 1) / 2 + i]);
                    acc[10 + l] = fma(d[l], bi, acc[10 + l]);
                }
            }
        }
        // block reduction (fixed order)
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const double v = warp_sum16(acc);
        if (!(lane & 1) && (lane >> 1) < kQ) red[lane >> 1][warp] = v;
        __syncthreads();
        if (threadIdx.x < kQ) {
            double v = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) v += red[threadIdx.x][w];
            a.partial[(size_t)threadIdx.x * a.n_tiles * a.n_sub + ch] = v;
        }
        __syncthreads();
    }
}

// One block per instance: G and D^T b summed from the chunks' partials (threads stride over the chunks, fixed-order
// reduction), then thread 0 solves: G scaled to unit diagonal, Cholesky, c (0 when there is no history).
__global__ void __launch_bounds__(kSolveThreads) k_proj_solve(ProjArgs a) {
    __shared__ double red[kQ][kSolveThreads / 32];
    const int inst = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k0 = a.kin[inst];
    double G[10], r[4], c[4] = {0.0, 0.0, 0.0, 0.0};
    const int c0 = a.inst_t0[inst] * a.n_sub, c1 = a.inst_t1[inst] * a.n_sub;
    {
        // the 14 quantities of a chunk are loaded together, so their latencies overlap
        double acc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = 0.0;
        const size_t nq = (size_t)a.n_tiles * a.n_sub;
        for (int ch = c0 + threadIdx.x; ch < c1; ch += kSolveThreads) {
#pragma unroll
            for (int q = 0; q < kQ; ++q) acc[q] += a.partial[q * nq + ch];
        }
        const double v = warp_sum16(acc);
        if (!(lane & 1) && (lane >> 1) < kQ) red[lane >> 1][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        double v = 0.0;
        for (int w = 0; w < kSolveThreads / 32; ++w) v += red[q][w];
        if (q < 10) G[q] = v;
        else r[q - 10] = v;
    }
    int k = k0;
    while (k > 0) {
        // scale to unit diagonal, factorise L L^T
        double s[4], L[10];
        bool ok = true;
        for (int i = 0; i < k && ok; ++i) {
            ok = G[tri(i, i)] > 0.0;
            s[i] = ok ? rsqrt(G[tri(i, i)]) : 0.0;
        }
        for (int l = 0; l < k && ok; ++l) {
            for (int i = 0; i <= l && ok; ++i) {
                double v = G[tri(i, l)] * s[i] * s[l];
                for (int m = 0; m < i; ++m) v -= L[tri(m, i)] * L[tri(m, l)];
                if (i == l) {
                    ok = v > 1e-14;
                    L[tri(l, l)] = ok ? sqrt(v) : 0.0;
                } else {
                    L[tri(i, l)] = v / L[tri(i, i)];
                }
            }
        }
        if (ok) {
            double y[4];
            for (int i = 0; i < k; ++i) {
                double v = r[i] * s[i];
                for (int m = 0; m < i; ++m) v -= L[tri(m, i)] * y[m];
                y[i] = v / L[tri(i, i)];
            }
            for (int i = k - 1; i >= 0; --i) {
                double v = y[i];
                for (int m = i + 1; m < k; ++m) v -= L[tri(i, m)] * c[m];
                c[i] = v / L[tri(i, i)];
            }
            for (int i = 0; i < k; ++i) c[i] *= s[i];
            break;
        }
        --k;  // drop the highest difference and try again
    }
    for (int i = 0; i < 4; ++i) a.coef[4 * inst + i] = c[i];
    a.kout[inst] = k;
}

// One block per chunk: x = D c on free rows (when the instance has history); history shifted.
__global__ void __launch_bounds__(kThreads) k_proj_combine(ProjArgs a) {
    for (int ch = blockIdx.x; ch < a.n_tiles * a.n_sub; ch += gridDim.x) {
        int t, r0, r1;
        chunk_rows(a, ch, t, r0, r1);
        const int inst = a.tile_inst[t];
        const int k = a.kout[inst];
        const double c0 = a.coef[4 * inst], c1 = a.coef[4 * inst + 1], c2 = a.coef[4 * inst + 2],
                     c3 = a.coef[4 * inst + 3];
        for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
            const double xn = a.x[row], x1 = a.h1[row], x2 = a.h2[row];
            if (k > 0 && !a.bc[row]) {
                const double4 d = reinterpret_cast<const double4*>(a.D)[row];
                a.x[row] = c0 * d.x + c1 * d.y + c2 * d.z + c3 * d.w;
            }
            a.h3[row] = x2;
            a.h2[row] = x1;
            a.h1[row] = xn;
        }
    }
}

// Solutions available to each instance: min(4, hist - lag) (hist from the step statistics).
__global__ void k_proj_count(ProjArgs a, const int32_t* hist, int lag) {
    const int inst = blockIdx.x * blockDim.x + threadIdx.x;
    if (inst >= a.n_inst) return;
    const int h = *hist - lag;
    a.kin[inst] = h < 0 ? 0 : (h > 4 ? 4 : h);
}

}  // namespace

cudaError_t launch_projection(const ProjArgs& a, const int32_t* hist, int lag, cudaStream_t st) {
    k_proj_count<<<(a.n_inst + 127) / 128, 128, 0, st>>>(a, hist, lag);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long nch = (long long)a.n_tiles * a.n_sub;
    const int grid = (int)(nch < 148 * 32 ? nch : 148 * 32);
    k_proj_basis<<<grid, kThreads, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_proj_gram<<<grid, kThreads, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_proj_solve<<<a.n_inst, kSolveThreads, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_proj_combine<<<grid, kThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace rafem
