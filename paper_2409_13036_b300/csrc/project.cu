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

#include "dw.cuh"
#include "internal.h"

namespace rafem {

namespace {

constexpr int kThreads = 256;
constexpr int kQ = 14;  // 10 entries of the symmetric 4 x 4 Gram matrix + 4 right-hand sides
constexpr int kChunk = kProjChunk;  // rows per block: tiles are split so that the pass has enough parallelism
constexpr int kBatch = 5;  // interior rows of the Kuhn lattice have 15 entries
constexpr int kSolveThreads = 256;
constexpr int kBatchApply = 3;  // double-word apply: fewer live registers, four blocks per SM

__device__ __forceinline__ int tri(int i, int l) { return i <= l ? l * (l + 1) / 2 + i : i * (i + 1) / 2 + l; }

// Arithmetic of the sums: FP64, or double-word (dw.cuh: float pairs on the FP32 pipes, stored as float2).
struct ArithF64 {
    using T = double;
    using S = double;  // storage
    __device__ static T zero() { return 0.0; }
    __device__ static T add(T x, T y) { return x + y; }
    __device__ static T shfl(T v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
    __device__ static T load(const S* p) { return *p; }
    __device__ static void store(S* p, T v) { *p = v; }
    __device__ static double value(T v) { return v; }
};
struct ArithDW {
    using T = dw::df;
    using S = float2;
    __device__ static T zero() { return dw::make(0.0f); }
    __device__ static T add(T x, T y) { return dw::add(x, y); }
    __device__ static T shfl(T v, int o) {
        return {__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
    }
    __device__ static T load(const S* p) { return dw::load(p); }
    __device__ static void store(S* p, T v) { dw::store(p, v); }
    __device__ static double value(T v) { return dw::to_double(v); }
};

// Sums 16 values over the warp by recursive halving: at each of the offsets 16, 8, 4, 2 a lane keeps one half of
// its values and adds the partner's copy of that half, so 16 shuffles replace the 80 of one butterfly per value.
// On return lane l holds the warp total of value l >> 1 (fixed order, deterministic).
template <class Ar>
__device__ __forceinline__ typename Ar::T warp_sum16(typename Ar::T (&v)[16]) {
    using T = typename Ar::T;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int h = 8; h >= 1; h >>= 1) {
        const bool up = lane & (2 * h);
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const T send = up ? v[i] : v[i + h];
            const T keep = up ? v[i + h] : v[i];
            v[i] = Ar::add(keep, Ar::shfl(send, 2 * h));
        }
    }
    return Ar::add(v[0], Ar::shfl(v[0], 1));
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
        const double v = warp_sum16<ArithF64>(acc);
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
template <class Ar>
__global__ void __launch_bounds__(kSolveThreads) k_proj_solve(ProjArgs a) {
    using T = typename Ar::T;
    __shared__ T red[kQ][kSolveThreads / 32];
    const int inst = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k0 = a.kin[inst];
    double G[10], r[4], c[4] = {0.0, 0.0, 0.0, 0.0};
    const int c0 = a.inst_t0[inst] * a.n_sub, c1 = a.inst_t1[inst] * a.n_sub;
    {
        // the 14 quantities of a chunk are loaded together, so their latencies overlap
        T acc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = Ar::zero();
        const size_t nq = (size_t)a.n_tiles * a.n_sub;
        const typename Ar::S* partial = reinterpret_cast<const typename Ar::S*>(a.partial);
        for (int ch = c0 + threadIdx.x; ch < c1; ch += kSolveThreads) {
#pragma unroll
            for (int q = 0; q < kQ; ++q) acc[q] = Ar::add(acc[q], Ar::load(partial + q * nq + ch));
        }
        const T v = warp_sum16<Ar>(acc);
        if (!(lane & 1) && (lane >> 1) < kQ) red[lane >> 1][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        T v = Ar::zero();
        for (int w = 0; w < kSolveThreads / 32; ++w) v = Ar::add(v, red[q][w]);
        if (q < 10) G[q] = Ar::value(v);
        else r[q - 10] = Ar::value(v);
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

// ---- double-word variants of the three passes over the nodes and the matrix (dw.cuh). D holds four float pairs
// per node (32 bytes, as in FP64), the partial sums float pairs; the FP64 matrix values and vectors are split by
// integer operations as they are read, and x = D c is written with one FP64 addition per node.

__device__ __forceinline__ dw::df pair(float a, float b) { return dw::make(a, b); }

// d_0 = x, d_1 = x - h1, d_2 = d_1 - (h1 - h2), d_3 = d_2 - ((h1 - h2) - (h2 - h3)) from the split values
__global__ void __launch_bounds__(kThreads) k_proj_basis_dw(ProjArgs a) {
    float4* D = reinterpret_cast<float4*>(a.D);
    for (int ch = blockIdx.x; ch < a.n_tiles * a.n_sub; ch += gridDim.x) {
        int t, r0, r1;
        chunk_rows(a, ch, t, r0, r1);
        const int k = a.kin[a.tile_inst[t]];
        for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
            const dw::df x = dw::split(a.x[row]);
            const dw::df h1 = k > 1 ? dw::split(a.h1[row]) : dw::make(0.0f);
            const dw::df h2 = k > 2 ? dw::split(a.h2[row]) : dw::make(0.0f);
            const dw::df h3 = k > 3 ? dw::split(a.h3[row]) : dw::make(0.0f);
            const dw::df e1 = dw::sub(x, h1), e2 = dw::sub(h1, h2), e3 = dw::sub(h2, h3);
            const dw::df d1 = k > 1 ? e1 : dw::make(0.0f);
            const dw::df d2 = k > 2 ? dw::sub(e1, e2) : dw::make(0.0f);
            const dw::df d3 = k > 3 ? dw::sub(d2, dw::sub(e2, e3)) : dw::make(0.0f);
            D[2 * row] = make_float4(x.h, x.l, d1.h, d1.l);
            D[2 * row + 1] = make_float4(d2.h, d2.l, d3.h, d3.l);
        }
    }
}

// Y = A D on the free rows of instances with history (four float pairs per node, the layout of D). Kept apart
// from the sums below so that few registers stay live and enough warps hide the gathers' latency.
__global__ void __launch_bounds__(kThreads, 4) k_proj_apply_dw(ProjArgs a) {
    const float4* D = reinterpret_cast<const float4*>(a.D);  // written by the previous launch
    float4* Y = reinterpret_cast<float4*>(a.Y);
    for (int ch = blockIdx.x; ch < a.n_tiles * a.n_sub; ch += gridDim.x) {
        int t, r0, r1;
        chunk_rows(a, ch, t, r0, r1);
        if (a.kin[a.tile_inst[t]] == 0) continue;
        for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
            if (a.bc[row]) continue;
            dw::df y[4] = {dw::make(0.0f), dw::make(0.0f), dw::make(0.0f), dw::make(0.0f)};
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
            for (int q = q0; q < q1; q += kBatchApply * stride) {
                double v[kBatchApply];
                int j[kBatchApply];
#pragma unroll
                for (int u = 0; u < kBatchApply; ++u) {
                    const int qq = q + u * stride;
                    const bool ok = qq < q1;
                    v[u] = ok ? __ldg(a.A + qq) : 0.0;
                    j[u] = ok ? (a.ci16 ? row + (int)__ldg(a.ci16 + qq) : __ldg(a.ci + qq)) : row;
                }
                float4 lo[kBatchApply], hi[kBatchApply];
#pragma unroll
                for (int u = 0; u < kBatchApply; ++u) {
                    lo[u] = __ldg(D + 2 * j[u]);
                    hi[u] = __ldg(D + 2 * j[u] + 1);
                }
#pragma unroll
                for (int u = 0; u < kBatchApply; ++u) {
                    const dw::df av = dw::split(v[u]);
                    dw::dot_acc(y[0], av, pair(lo[u].x, lo[u].y));
                    dw::dot_acc(y[1], av, pair(lo[u].z, lo[u].w));
                    dw::dot_acc(y[2], av, pair(hi[u].x, hi[u].y));
                    dw::dot_acc(y[3], av, pair(hi[u].z, hi[u].w));
                }
            }
#pragma unroll
            for (int l = 0; l < 4; ++l) y[l] = dw::finish(y[l]);
            Y[2 * row] = make_float4(y[0].h, y[0].l, y[1].h, y[1].l);
            Y[2 * row + 1] = make_float4(y[2].h, y[2].l, y[3].h, y[3].l);
        }
    }
}

// Per chunk: the partial sums of G = D^T Y and D^T b over its free rows.
__global__ void __launch_bounds__(kThreads) k_proj_gram_dw(ProjArgs a) {
    __shared__ float2 red[kQ][kThreads / 32];
    const float4* D = reinterpret_cast<const float4*>(a.D);
    const float4* Y = reinterpret_cast<const float4*>(a.Y);
    float2* partial = reinterpret_cast<float2*>(a.partial);
    for (int ch = blockIdx.x; ch < a.n_tiles * a.n_sub; ch += gridDim.x) {
        int t, r0, r1;
        chunk_rows(a, ch, t, r0, r1);
        const int k = a.kin[a.tile_inst[t]];
        dw::df acc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = dw::make(0.0f);
        if (k > 0) {
            for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
                if (a.bc[row]) continue;
                const float4 dlo = __ldg(D + 2 * row), dhi = __ldg(D + 2 * row + 1);
                const float4 ylo = __ldg(Y + 2 * row), yhi = __ldg(Y + 2 * row + 1);
                const dw::df d[4] = {pair(dlo.x, dlo.y), pair(dlo.z, dlo.w), pair(dhi.x, dhi.y), pair(dhi.z, dhi.w)};
                const dw::df y[4] = {pair(ylo.x, ylo.y), pair(ylo.z, ylo.w), pair(yhi.x, yhi.y), pair(yhi.z, yhi.w)};
                const dw::df bi = dw::split(a.b[row]);
#pragma unroll
                for (int l = 0; l < 4; ++l) {
#pragma unroll
                    for (int i = 0; i <= l; ++i) dw::dot_acc(acc[l * (l + 1) / 2 + i], d[i], y[l]);
                    dw::dot_acc(acc[10 + l], d[l], bi);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < kQ; ++q) acc[q] = dw::finish(acc[q]);
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const dw::df v = warp_sum16<ArithDW>(acc);
        if (!(lane & 1) && (lane >> 1) < kQ) red[lane >> 1][warp] = make_float2(v.h, v.l);
        __syncthreads();
        if (threadIdx.x < kQ) {
            dw::df s = dw::make(0.0f);
            for (int w = 0; w < kThreads / 32; ++w) s = dw::add(s, dw::load(&red[threadIdx.x][w]));
            dw::store(partial + (size_t)threadIdx.x * a.n_tiles * a.n_sub + ch, s);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kThreads) k_proj_combine_dw(ProjArgs a) {
    const float4* D = reinterpret_cast<const float4*>(a.D);
    for (int ch = blockIdx.x; ch < a.n_tiles * a.n_sub; ch += gridDim.x) {
        int t, r0, r1;
        chunk_rows(a, ch, t, r0, r1);
        const int inst = a.tile_inst[t];
        const int k = a.kout[inst];
        const dw::df c0 = dw::split(a.coef[4 * inst]), c1 = dw::split(a.coef[4 * inst + 1]),
                     c2 = dw::split(a.coef[4 * inst + 2]), c3 = dw::split(a.coef[4 * inst + 3]);
        for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
            const double xn = a.x[row], x1 = a.h1[row], x2 = a.h2[row];
            if (k > 0 && !a.bc[row]) {
                const float4 lo = D[2 * row], hi = D[2 * row + 1];
                const dw::df s01 = dw::add(dw::mul(c0, pair(lo.x, lo.y)), dw::mul(c1, pair(lo.z, lo.w)));
                const dw::df s23 = dw::add(dw::mul(c2, pair(hi.x, hi.y)), dw::mul(c3, pair(hi.z, hi.w)));
                a.x[row] = dw::to_double(dw::add(s01, s23));
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
    if (a.dw) {
        k_proj_basis_dw<<<grid, kThreads, 0, st>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_proj_apply_dw<<<grid, kThreads, 0, st>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_proj_gram_dw<<<grid, kThreads, 0, st>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_proj_solve<ArithDW><<<a.n_inst, kSolveThreads, 0, st>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_proj_combine_dw<<<grid, kThreads, 0, st>>>(a);
        return cudaGetLastError();
    }
    k_proj_basis<<<grid, kThreads, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_proj_gram<<<grid, kThreads, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_proj_solve<ArithF64><<<a.n_inst, kSolveThreads, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_proj_combine<<<grid, kThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace rafem
