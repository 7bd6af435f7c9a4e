// Initial guess by projection onto the recent solutions (an extension of the predictor step of the main loop,
// Sec. II-A: the solution is extrapolated in time before the corrector solves).
//
// With x_n, x_{n-1}, ... the last k solutions (k <= kProjMax) of an SPD system A x = b whose matrix changed since,
// the guess is the A-orthogonal projection of the new solution onto their span:
//     x_0 = D c,   (D^T A D) c = D^T b,
// with D the difference basis d_0 = x_n, d_1 = x_n - x_{n-1}, d_j = the j-th backward difference (the same span,
// much better conditioned than the raw solutions). This minimises the A-norm error over the span, which contains
// every polynomial extrapolation of the same solutions, so the Krylov solve starts closer than with the
// polynomial predictor. Sums run over free rows only (the symmetric lift makes A block diagonal with identity
// Dirichlet rows), and Dirichlet entries are set to their prescribed values.
//
// No past solution is stored: the backward differences obey d_j(n) = d_{j-1}(n) - d_{j-1}(n-1), so each call
// builds its basis from the current solution and the previous call's basis, which stays in memory (and in the
// differentiation form's checkpoints) as the predictor's history: K - 1 subtractions per node.
//
// Launches per solve, per problem instance of a batch (the solver's work tiles never straddle instances), all
// compiled for the context's basis limit K (2, 4, 6 or 8); with the double-word gather assembly and K = 4 the
// basis is built before the potential's assembly, which accumulates Y = A D itself, and k_proj_apply is skipped:
//   k_proj_count:   one thread: the basis size of every instance;
//   k_proj_basis:   the basis D at every node from the solution and the previous basis (K 8-byte entries each);
//   k_proj_apply:   Y = A D, one pass over A (SELL-32 or CSR), entries in batches;
//   k_proj_gram:    per chunk of rows the partial sums of G = D^T Y and D^T b; with many quantities (K = 6, 8)
//                   two or four warps share a row set, each accumulating a share of them;
//   k_proj_solve:   per instance, G scaled to unit diagonal and factorised by Cholesky (the basis shrinks while a
//                   pivot is not positive), c solved;
//   k_proj_combine: x = D c on free rows.
// Every pass runs in FP64 or in double-word arithmetic (dw.cuh), as the assembly does; the Cholesky is FP64.
#include <cuda_runtime.h>

#include <cmath>

#include "dw.cuh"
#include "internal.h"

namespace rafem {

namespace {

constexpr int kThreads = 256;
constexpr int kChunk = kProjChunk;  // rows per block: tiles are split so that the passes have enough parallelism
constexpr int kSolveThreads = 256;

// Quantities of a basis of K: the Gram entries G[i][l] (i <= l) at l (l + 1) / 2 + i, then (D^T b)[l].
template <int K>
struct Basis {
    static constexpr int kGram = K * (K + 1) / 2;
    static constexpr int kQ = kGram + K;
    static constexpr int kGroups = kQ <= 16 ? 1 : (kQ <= 32 ? 2 : 4);  // warps sharing a row set in the Gram pass
    static constexpr int kPerGroup = (kQ + kGroups - 1) / kGroups;
    static_assert(kPerGroup <= 16, "warp_sum16 reduces at most 16 quantities per thread");
    static_assert(K % 2 == 0 && K <= kProjMax, "even basis sizes up to kProjMax");
};

// Arithmetic of the passes: FP64, or double-word (float pairs on the FP32 pipes, stored as float2).
struct ArithF64 {
    using T = double;
    using S = double;  // 8-byte storage
    __device__ static T zero() { return 0.0; }
    __device__ static T from(double x) { return x; }
    __device__ static double value(T v) { return v; }
    __device__ static T add(T x, T y) { return x + y; }
    __device__ static T sub(T x, T y) { return x - y; }
    __device__ static void dot(T& acc, T x, T y) { acc = fma(x, y, acc); }
    __device__ static T finish(T v) { return v; }
    __device__ static T shfl(T v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
    __device__ static T load(const S* p) { return *p; }
    __device__ static void store(S* p, T v) { *p = v; }
    // two consecutive entries as one 16-byte access
    __device__ static void ldg2(const S* p, T& a, T& b) {
        const double2 v = __ldg(reinterpret_cast<const double2*>(p));
        a = v.x;
        b = v.y;
    }
    __device__ static void ld2(const S* p, T& a, T& b) {
        const double2 v = *reinterpret_cast<const double2*>(p);
        a = v.x;
        b = v.y;
    }
    __device__ static void st2(S* p, T a, T b) { *reinterpret_cast<double2*>(p) = make_double2(a, b); }
};
struct ArithDW {
    using T = dw::df;
    using S = float2;
    __device__ static T zero() { return dw::make(0.0f); }
    __device__ static T from(double x) { return dw::split(x); }
    __device__ static double value(T v) { return dw::to_double(v); }
    __device__ static T add(T x, T y) { return dw::add(x, y); }
    __device__ static T sub(T x, T y) { return dw::sub(x, y); }
    __device__ static void dot(T& acc, T x, T y) { dw::dot_acc(acc, x, y); }
    __device__ static T finish(T v) { return dw::finish(v); }
    __device__ static T shfl(T v, int o) {
        return {__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
    }
    __device__ static T load(const S* p) { return dw::load(p); }
    __device__ static void store(S* p, T v) { dw::store(p, v); }
    __device__ static void ldg2(const S* p, T& a, T& b) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p));
        a = dw::make(v.x, v.y);
        b = dw::make(v.z, v.w);
    }
    __device__ static void ld2(const S* p, T& a, T& b) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        a = dw::make(v.x, v.y);
        b = dw::make(v.z, v.w);
    }
    __device__ static void st2(S* p, T a, T b) { *reinterpret_cast<float4*>(p) = make_float4(a.h, a.l, b.h, b.l); }
};

// Quantity q of a basis of K: (i, l) of G[i][l], or i = -1 and l for (D^T b)[l].
template <int K>
__host__ __device__ constexpr int q_col(int q) {
    if (q >= Basis<K>::kGram) return q - Basis<K>::kGram;
    int l = 0;
    while ((l + 1) * (l + 2) / 2 <= q) ++l;
    return l;
}
template <int K>
__host__ __device__ constexpr int q_row(int q) {
    return q >= Basis<K>::kGram ? -1 : q - q_col<K>(q) * (q_col<K>(q) + 1) / 2;
}

__device__ __forceinline__ int tri(int i, int l) { return i <= l ? l * (l + 1) / 2 + i : i * (i + 1) / 2 + l; }

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

// Rows of chunk c: chunk c = (tile c / n_sub, part c % n_sub), kChunk rows each (fewer at the tile's end).
__device__ __forceinline__ void chunk_rows(const ProjArgs& a, int c, int& t, int& r0, int& r1) {
    t = c / a.n_sub;
    const int sub = c % a.n_sub;
    r0 = a.tile_r0[t] + sub * kChunk;
    r1 = min(r0 + kChunk, a.tile_r1[t]);
}

// One thread: the basis size of every instance, min(kmax, hist - lag) with hist the steps completed since the last
// state reset.
__global__ void k_proj_count(ProjArgs a, const int32_t* hist, int lag) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const int s = *hist - lag;
    const int k = s < 0 ? 0 : (s > a.kmax ? a.kmax : s);
    for (int i = 0; i < a.n_inst; ++i) a.kin[i] = k;
}

// D at the chunk's nodes from the solution and the previous call's basis: d_0 = x, d_j = d_{j-1} - d_{j-1}(old)
// (entries j >= k are 0). In place: every old entry of the row is read before any is written.
template <class Ar, int K>
__global__ void __launch_bounds__(kThreads) k_proj_basis(ProjArgs a) {
    using T = typename Ar::T;
    typename Ar::S* D = reinterpret_cast<typename Ar::S*>(a.D);
    for (int ch = blockIdx.x; ch < a.n_tiles * a.n_sub; ch += gridDim.x) {
        int t, r0, r1;
        chunk_rows(a, ch, t, r0, r1);
        const int k = a.kin[a.tile_inst[t]];
        if (k == 0) continue;
        for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
            typename Ar::S* d = D + (size_t)row * K;
            T old[K];
#pragma unroll
            for (int j = 0; j < K; j += 2) Ar::ld2(d + j, old[j], old[j + 1]);
            T cur = Ar::from(a.x[row]);
            T nw[K];
            nw[0] = cur;
#pragma unroll
            for (int j = 1; j < K; ++j) {
                if (j < k) cur = Ar::sub(cur, old[j - 1]);
                nw[j] = j < k ? cur : Ar::zero();
            }
#pragma unroll
            for (int j = 0; j < K; j += 2) Ar::st2(d + j, nw[j], nw[j + 1]);
        }
    }
}

// Y = A D on the free rows of instances with history, entries in batches of KB (columns and values, then the
// basis gathers, then the arithmetic).
template <class Ar, int K, int KB>
__global__ void __launch_bounds__(kThreads, 3) k_proj_apply(ProjArgs a) {
    using T = typename Ar::T;
    const typename Ar::S* D = reinterpret_cast<const typename Ar::S*>(a.D);  // written by the previous launch
    typename Ar::S* Y = reinterpret_cast<typename Ar::S*>(a.Y);
    for (int ch = blockIdx.x; ch < a.n_tiles * a.n_sub; ch += gridDim.x) {
        int t, r0, r1;
        chunk_rows(a, ch, t, r0, r1);
        const int k = a.kin[a.tile_inst[t]];
        if (k == 0) continue;
        for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
            if (a.bc[row]) continue;
            T y[K];
#pragma unroll
            for (int d = 0; d < K; ++d) y[d] = Ar::zero();
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
            for (int q = q0; q < q1; q += KB * stride) {
                double v[KB];
                int j[KB];
#pragma unroll
                for (int u = 0; u < KB; ++u) {
                    const int qq = q + u * stride;
                    const bool ok = qq < q1;
                    v[u] = ok ? __ldg(a.A + qq) : 0.0;
                    j[u] = ok ? (a.ci16 ? row + (int)__ldg(a.ci16 + qq) : __ldg(a.ci + qq)) : row;
                }
                T dj[KB][K];
#pragma unroll
                for (int u = 0; u < KB; ++u)
#pragma unroll
                    for (int d = 0; d < K; d += 2) Ar::ldg2(D + (size_t)j[u] * K + d, dj[u][d], dj[u][d + 1]);
#pragma unroll
                for (int u = 0; u < KB; ++u) {
                    const T av = Ar::from(v[u]);
#pragma unroll
                    for (int d = 0; d < K; ++d)
                        if (d < k) Ar::dot(y[d], av, dj[u][d]);
                }
            }
            typename Ar::S* yr = Y + (size_t)row * K;
#pragma unroll
            for (int d = 0; d < K; ++d) Ar::store(yr + d, Ar::finish(y[d]));
        }
    }
}

// Quantities G kPerGroup .. G kPerGroup + kPerGroup - 1 of one row into the group's accumulators.
template <class Ar, int K, int G>
__device__ __forceinline__ void gram_row(typename Ar::T (&acc)[16], const typename Ar::T (&d)[K],
                                         const typename Ar::T (&y)[K], typename Ar::T bi) {
    using B = Basis<K>;
#pragma unroll
    for (int j = 0; j < B::kPerGroup; ++j) {
        const int q = G * B::kPerGroup + j;
        if (q < B::kQ) {
            if (q_row<K>(q) >= 0)
                Ar::dot(acc[j], d[q_row<K>(q)], y[q_col<K>(q)]);
            else
                Ar::dot(acc[j], d[q_col<K>(q)], bi);
        }
    }
}

// Per chunk: partial sums of the basis's quantities over its free rows. Warp w of the block takes quantity group
// w % groups for the rows of row set w / groups (32 rows at a time), so a row's D and Y are read by every group
// (the repeats from L1) and every thread holds at most 16 accumulators.
template <class Ar, int K>
__global__ void __launch_bounds__(kThreads) k_proj_gram(ProjArgs a) {
    using T = typename Ar::T;
    using B = Basis<K>;
    constexpr int kSets = kThreads / 32 / B::kGroups;  // row sets per block
    __shared__ typename Ar::S red[B::kQ][kSets];
    const typename Ar::S* D = reinterpret_cast<const typename Ar::S*>(a.D);
    const typename Ar::S* Y = reinterpret_cast<const typename Ar::S*>(a.Y);
    typename Ar::S* partial = reinterpret_cast<typename Ar::S*>(a.partial);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = warp % B::kGroups, set = warp / B::kGroups;
    for (int ch = blockIdx.x; ch < a.n_tiles * a.n_sub; ch += gridDim.x) {
        int t, r0, r1;
        chunk_rows(a, ch, t, r0, r1);
        const int k = a.kin[a.tile_inst[t]];
        T acc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = Ar::zero();
        if (k > 0) {
            for (int row = r0 + set * 32 + lane; row < r1; row += kSets * 32) {
                if (a.bc[row]) continue;
                T d[K], y[K];
#pragma unroll
                for (int e = 0; e < K; e += 2) {
                    Ar::ldg2(D + (size_t)row * K + e, d[e], d[e + 1]);
                    Ar::ldg2(Y + (size_t)row * K + e, y[e], y[e + 1]);
                }
                const T bi = Ar::from(a.b[row]);
                if constexpr (B::kGroups == 1) {
                    gram_row<Ar, K, 0>(acc, d, y, bi);
                } else if constexpr (B::kGroups == 2) {
                    if (g == 0) gram_row<Ar, K, 0>(acc, d, y, bi);
                    else gram_row<Ar, K, 1>(acc, d, y, bi);
                } else {
                    switch (g) {  // warp-uniform
                        case 0: gram_row<Ar, K, 0>(acc, d, y, bi); break;
                        case 1: gram_row<Ar, K, 1>(acc, d, y, bi); break;
                        case 2: gram_row<Ar, K, 2>(acc, d, y, bi); break;
                        default: gram_row<Ar, K, 3>(acc, d, y, bi); break;
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < B::kPerGroup; ++q) acc[q] = Ar::finish(acc[q]);
        const T v = warp_sum16<Ar>(acc);
        const int q = g * B::kPerGroup + (lane >> 1);
        if (!(lane & 1) && (lane >> 1) < B::kPerGroup && q < B::kQ) Ar::store(&red[q][set], v);
        __syncthreads();
        for (int qq = threadIdx.x; qq < B::kQ; qq += blockDim.x) {
            T s = Ar::zero();
            for (int w = 0; w < kSets; ++w) s = Ar::add(s, Ar::load(&red[qq][w]));
            Ar::store(partial + (size_t)qq * a.n_tiles * a.n_sub + ch, s);
        }
        __syncthreads();
    }
}

// One block per instance: every warp sums a share of the quantities over the instance's chunks (lanes stride over
// the chunks, fixed-order reduction), then thread 0 solves: G scaled to unit diagonal, Cholesky, c (0 when there
// is no history).
template <class Ar, int K>
__global__ void __launch_bounds__(kSolveThreads) k_proj_solve(ProjArgs a) {
    using T = typename Ar::T;
    using B = Basis<K>;
    __shared__ double tot[B::kQ];
    const int inst = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k0 = a.kin[inst];
    const int c0 = a.inst_t0[inst] * a.n_sub, c1 = a.inst_t1[inst] * a.n_sub;
    const size_t nq = (size_t)a.n_tiles * a.n_sub;
    const typename Ar::S* partial = reinterpret_cast<const typename Ar::S*>(a.partial);
    for (int q = warp; q < B::kQ; q += kSolveThreads / 32) {
        T v = Ar::zero();
        if (k0 > 0)
            for (int ch = c0 + lane; ch < c1; ch += 32) v = Ar::add(v, Ar::load(partial + q * nq + ch));
#pragma unroll
        for (int o = 16; o; o >>= 1) v = Ar::add(v, Ar::shfl(v, o));
        if (lane == 0) tot[q] = Ar::value(v);
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double c[K];
    for (int i = 0; i < K; ++i) c[i] = 0.0;
    int k = k0;
    while (k > 0) {
        // scale to unit diagonal, factorise L L^T
        double s[K], L[B::kGram];
        bool ok = true;
        for (int i = 0; i < k && ok; ++i) {
            ok = tot[tri(i, i)] > 0.0;
            s[i] = ok ? rsqrt(tot[tri(i, i)]) : 0.0;
        }
        for (int l = 0; l < k && ok; ++l) {
            for (int i = 0; i <= l && ok; ++i) {
                double v = tot[tri(i, l)] * s[i] * s[l];
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
            double y[K];
            for (int i = 0; i < k; ++i) {
                double v = tot[B::kGram + i] * s[i];
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
        for (int i = 0; i < K; ++i) c[i] = 0.0;
        --k;  // drop the highest difference and try again
    }
    for (int i = 0; i < K; ++i) a.coef[kProjMax * inst + i] = c[i];
    a.kout[inst] = k;
}

// One block per chunk: x = D c on free rows (when the instance has history), and the residual of that guess,
// b - A x = b - Y c, for the solver's first residual (0 on Dirichlet rows, where x already holds the prescribed
// value).
template <class Ar, int K>
__global__ void __launch_bounds__(kThreads) k_proj_combine(ProjArgs a) {
    using T = typename Ar::T;
    const typename Ar::S* D = reinterpret_cast<const typename Ar::S*>(a.D);
    const typename Ar::S* Y = reinterpret_cast<const typename Ar::S*>(a.Y);
    for (int ch = blockIdx.x; ch < a.n_tiles * a.n_sub; ch += gridDim.x) {
        int t, r0, r1;
        chunk_rows(a, ch, t, r0, r1);
        const int inst = a.tile_inst[t];
        const int k = a.kout[inst];
        T c[K];
#pragma unroll
        for (int i = 0; i < K; ++i) c[i] = Ar::from(a.coef[kProjMax * inst + i]);
        for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
            if (k > 0 && !a.bc[row]) {
                T s = Ar::zero(), ay = Ar::zero();
#pragma unroll
                for (int d = 0; d < K; d += 2) {
                    T d0, d1, y0, y1;
                    Ar::ldg2(D + (size_t)row * K + d, d0, d1);
                    Ar::ldg2(Y + (size_t)row * K + d, y0, y1);
                    if (d < k) {
                        Ar::dot(s, c[d], d0);
                        Ar::dot(ay, c[d], y0);
                    }
                    if (d + 1 < k) {
                        Ar::dot(s, c[d + 1], d1);
                        Ar::dot(ay, c[d + 1], y1);
                    }
                }
                a.x[row] = Ar::value(Ar::finish(s));
                a.r0[row] = Ar::value(Ar::sub(Ar::from(a.b[row]), Ar::finish(ay)));
            } else if (k > 0) {
                a.r0[row] = 0.0;
            }
        }
    }
}

template <class Ar, int K>
cudaError_t launch_basis(const ProjArgs& a, int grid, cudaStream_t st) {
    k_proj_basis<Ar, K><<<grid, kThreads, 0, st>>>(a);
    return cudaGetLastError();
}

template <class Ar, int K>
cudaError_t launch_rest(const ProjArgs& a, int grid, bool apply, cudaStream_t st) {
    cudaError_t e;
    if (apply) {
        k_proj_apply<Ar, K, K <= 4 ? 3 : 2><<<grid, kThreads, 0, st>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_proj_gram<Ar, K><<<grid, kThreads, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_proj_solve<Ar, K><<<a.n_inst, kSolveThreads, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_proj_combine<Ar, K><<<grid, kThreads, 0, st>>>(a);
    return cudaGetLastError();
}

int grid_of(const ProjArgs& a) {
    const long long nch = (long long)a.n_tiles * a.n_sub;
    return (int)(nch < 148 * 32 ? nch : 148 * 32);
}

template <class Ar>
cudaError_t sized_basis(const ProjArgs& a, cudaStream_t st) {
    const int g = grid_of(a);
    switch (proj_stride(a.kmax)) {
        case 2: return launch_basis<Ar, 2>(a, g, st);
        case 4: return launch_basis<Ar, 4>(a, g, st);
        case 6: return launch_basis<Ar, 6>(a, g, st);
        default: return launch_basis<Ar, 8>(a, g, st);
    }
}

template <class Ar>
cudaError_t sized_rest(const ProjArgs& a, bool apply, cudaStream_t st) {
    const int g = grid_of(a);
    switch (proj_stride(a.kmax)) {
        case 2: return launch_rest<Ar, 2>(a, g, apply, st);
        case 4: return launch_rest<Ar, 4>(a, g, apply, st);
        case 6: return launch_rest<Ar, 6>(a, g, apply, st);
        default: return launch_rest<Ar, 8>(a, g, apply, st);
    }
}

}  // namespace

cudaError_t launch_projection_basis(const ProjArgs& a, const int32_t* hist, int lag, cudaStream_t st) {
    k_proj_count<<<1, 32, 0, st>>>(a, hist, lag);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return a.dw ? sized_basis<ArithDW>(a, st) : sized_basis<ArithF64>(a, st);
}

cudaError_t launch_projection_rest(const ProjArgs& a, bool apply, cudaStream_t st) {
    return a.dw ? sized_rest<ArithDW>(a, apply, st) : sized_rest<ArithF64>(a, apply, st);
}

cudaError_t launch_projection(const ProjArgs& a, const int32_t* hist, int lag, cudaStream_t st) {
    cudaError_t e = launch_projection_basis(a, hist, lag, st);
    if (e != cudaSuccess) return e;
    return launch_projection_rest(a, true, st);
}

}  // namespace rafem
