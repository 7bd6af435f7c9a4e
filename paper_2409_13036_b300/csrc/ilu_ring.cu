// ILU(0)-preconditioned conjugate gradients with the matrix and factor streams staged in shared memory, in FP64 or
// in mixed precision (FP32 inner iterations, FP64 residual refinement). Sec. II-B: CG for symmetric
// positive-definite systems, with a preconditioner to speed up convergence.
//
// The factors are those of P A P^T (ilu.cu refactors them after every assembly, in a combined layout); this
// solver keeps three SELL-32 layouts over the padded level numbering: P A P^T itself, the strictly lower factor L
// (unit diagonal implied) and the strictly upper part of U, with 1 / u_ii apart. Rows of one level never depend on
// each other, so a triangular sweep is one SpMV-like pass per level: the producer warp streams the level's slices
// of L (or U) into the shared-memory ring with bulk copies, and the consumer warps gather z of earlier (later)
// levels from L2 and finish their rows in the pass's epilogue. Where every slice of a layout shares one column
// pattern (lattice-like meshes), only values are streamed.
//
// Block b owns, in every level, the b-th run of spb slices of that level (spb = slices of the level / blocks,
// rounded up), so row-local vectors stay with their block. One persistent cooperative launch per solve:
//   gather:    x, b into the level order; (b, b)                                                  -- barrier --
//   residual:  r = b - A x (FP64 SpMV), level-0 rows z = r; (r, r)                                -- barrier --
//   precondition: forward levels 1..C-1:  z_i = r_i - (L z)_i (the last level also times 1 / u_ii)
//                 backward levels C-2..0: z_i = (z_i - (U z)_i) / u_ii; partial (r, z)    -- a barrier per level --
//   iteration: A: q = A z + beta q,  p = z + beta p, partial (p, q)                 -- barrier: alpha = gamma / delta
//              B: x += alpha p, r -= alpha q, partial (r, r); level-0 rows z = r                 -- barrier --
//              precondition (gamma), beta = gamma / gamma_prev
// In mixed precision the iteration runs on FP32 values, factors and vectors and corrects d (x = x64 + d); it ends
// at inner_tol or once the predicted FP64 residual reaches the target, then x64 += d and the FP64 residual starts
// the next refinement. Every block reduces the per-block sums itself in a fixed order (deterministic); consecutive
// reductions use distinct partial-sum slots. Every wait is bounded.
#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

#include "grid_sync.cuh"
#include "internal.h"
#include "sell_ring.cuh"

namespace rafem {

namespace {

using namespace sell;

enum { P_BB = 0, P_RR64 = 1, P_RR32 = 2, P_GAMMA = 3, P_DELTA = 4, P_RR = 5, P_TRUE = 6, P_SLOTS = 7 };
static_assert(P_SLOTS <= kIluRingSlots, "partial-sum slots");

struct Part {
    const int32_t* sp;
    const int32_t* sc;
    const int32_t* pat_off;
    const int32_t* pat_pool;
};

template <typename VT>
struct Vals {
    const VT* A;      // P A P^T in layout A
    const VT* L;      // strictly lower factor in layout L
    const VT* U;      // strictly upper factor in layout U
    const VT* dinv;   // 1 / u_ii
};

struct Args {
    int Np, n_levels, N;
    const int32_t* lvl;   // [n_levels + 1] first padded row of each level
    const int32_t* perm;  // [Np] original row, -1 dummy
    Part pA, pL, pU;
    Vals<double> v64;
    Vals<float> v32;
    const double* b;      // [N] original order
    double* x;            // [N] original order: initial guess in, solution out
    double *xv, *bv;      // [Np] FP64 solution and right-hand side in the level order
    double *r64;          // [Np] FP64 residual (FP64 mode: the CG residual)
    double *z64, *p64, *q64;
    float *r32, *z32, *p32, *q32, *d32;
    double* partial;      // [kIluRingSlots][grid]
    GridBarrier* bar;
    InstState* inst;
    double tol, inner_tol;
    int max_iter, max_refine;
    long long spin_limit_ns;
};

// Rows of level l owned by this block: [r0, r1), empty when r0 >= r1.
__device__ __forceinline__ void level_rows(const Args& a, int l, int& r0, int& r1) {
    const int l0 = __ldg(a.lvl + l), l1 = __ldg(a.lvl + l + 1);
    const int S = (l1 - l0) >> 5, spb = (S + gridDim.x - 1) / gridDim.x;
    const int s0 = min((int)blockIdx.x * spb, S), s1 = min(s0 + spb, S);
    r0 = l0 + 32 * s0;
    r1 = l0 + 32 * s1;
}

// SpMV over rows [r0, r1) of one layout through the ring: per-entry 32-bit columns, or shared slice patterns.
template <bool PAT, typename VT, class Emit>
__device__ __forceinline__ bool part_spmv(const Args& a, Ring& g, const Part& p, const VT* vals, const VT* xin, int r0,
                                          int r1, const Emit& em) {
    if (r0 >= r1) return __syncthreads_and(1);
    if constexpr (PAT)
        return sell_tile<VT, VT>(a, g, p.sp, SliceCols{p.pat_off, p.pat_pool, a.Np}, vals, xin, r0, r1, em);
    else
        return sell_tile<VT, VT>(a, g, p.sp, EntryCols<int32_t>{p.sc}, vals, xin, r0, r1, em);
}

__device__ __forceinline__ void publish1(double v, double* sm, double* slot) {
    double q[1] = {v};
    block_sum<1>(q, sm);
    if (threadIdx.x == 0) slot[blockIdx.x] = q[0];
}
__device__ __forceinline__ double total(const double* slot, double* s_tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp == 0) {
        double acc = 0.0;
        for (int t = lane; t < (int)gridDim.x; t += 32) acc += __ldcg(slot + t);
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) *s_tot = acc;
    }
    __syncthreads();
    const double v = *s_tot;
    __syncthreads();
    return v;
}

// ---- epilogues -------------------------------------------------------------------------------------------------

// FP64 residual r = b - A x of the current solution; level-0 rows start the forward sweep (z = r; with a single
// level z = r / u_ii). Mixed: r32 = (float) r, d32 = 0.
template <bool MIXED>
struct EmResidual {
    const Args& a;
    bool level0, single;
    double* v;  // [rr64, rr32 (mixed), (r, z) with a single level]
    __device__ __forceinline__ double pre(int row) const { return ldcg(a.bv + row); }
    __device__ __forceinline__ void fin(int row, double ax, double bi) const {
        const double r = bi - ax;
        v[0] = fma(r, r, v[0]);
        if constexpr (MIXED) {
            const float r32 = (float)r;
            a.r32[row] = r32;
            a.d32[row] = 0.0f;
            if (level0) {
                const float z = single ? r32 * ldcg(a.v32.dinv + row) : r32;
                a.z32[row] = z;
                v[2] = fma((double)r32, (double)z, v[2]);
            }
            v[1] = fma((double)r32, (double)r32, v[1]);
        } else {
            a.r64[row] = r;
            if (level0) {
                const double z = single ? r * ldcg(a.v64.dinv + row) : r;
                a.z64[row] = z;
                v[2] = fma(r, z, v[2]);
            }
        }
    }
};

// forward sweep of one level: z = r - L z (the last level also divides by u_ii and adds (r, z))
template <typename VT>
struct EmForward {
    const VT* r;
    VT* z;
    const VT* dinv;
    bool last;
    VT* g;
    __device__ __forceinline__ VT pre(int row) const { return ldcg(r + row); }
    __device__ __forceinline__ void fin(int row, VT lz, VT ri) const {
        VT zi = ri - lz;
        if (last) {
            zi *= ldcg(dinv + row);
            g[0] = fma(ri, zi, g[0]);
        }
        z[row] = zi;
    }
};

// backward sweep of one level: z = (z - U z) / u_ii; (r, z)
template <typename VT>
struct EmBackward {
    const VT* r;
    VT* z;
    const VT* dinv;
    VT* g;
    struct P {
        VT z, r, d;
    };
    __device__ __forceinline__ P pre(int row) const { return P{ldcg(z + row), ldcg(r + row), ldcg(dinv + row)}; }
    __device__ __forceinline__ void fin(int row, VT uz, const P& p) const {
        const VT zi = (p.z - uz) * p.d;
        z[row] = zi;
        g[0] = fma(p.r, zi, g[0]);
    }
};

// phase A: q = A z + beta q, p = z + beta p; (p, q)
template <typename VT>
struct EmDirection {
    const VT* z;
    VT *p, *q;
    VT beta;
    bool first;
    VT* v;
    __device__ __forceinline__ VT pre(int row) const { return ldcg(z + row); }
    __device__ __forceinline__ void fin(int row, VT az, VT zi) const {
        const VT pi = first ? zi : fma(beta, ldcg(p + row), zi);
        const VT qi = first ? az : fma(beta, ldcg(q + row), az);
        p[row] = pi;
        q[row] = qi;
        v[0] = fma(pi, qi, v[0]);
    }
};

template <bool MIXED, bool PAT>
__global__ void __launch_bounds__(kBlock, 1) k_ilu_ring(Args a) {
    RAFEM_RING_SETUP(1)
    using VT = typename std::conditional<MIXED, float, double>::type;
    __shared__ double sm[kSumMax * kBlock];
    __shared__ double s_tot;
    const int C = a.n_levels;
    VT *r, *z, *p, *q;
    Vals<VT> vv;
    if constexpr (MIXED) {
        r = a.r32, z = a.z32, p = a.p32, q = a.q32;
        vv = a.v32;
    } else {
        r = a.r64, z = a.z64, p = a.p64, q = a.q64;
        vv = a.v64;
    }
    double* slot[P_SLOTS];
    for (int k = 0; k < P_SLOTS; ++k) slot[k] = a.partial + (size_t)k * gridDim.x;
    unsigned target = 0;
    bool err = false;
    int iters = 0, refine = 0, status = RAFEM_NOT_CONVERGED;
    double bb = 0.0, rr64 = 0.0, relres = 0.0;

    // gather x, b into the level order; (b, b)
    {
        double v = 0.0;
        for (int l = 0; l < C; ++l) {
            int r0, r1;
            level_rows(a, l, r0, r1);
            for (int row = r0 + threadIdx.x; row < r1; row += kBlock) {
                const int o = __ldg(a.perm + row);
                const double bi = o >= 0 ? a.b[o] : 0.0;
                a.xv[row] = o >= 0 ? a.x[o] : 0.0;
                a.bv[row] = bi;
                v = fma(bi, bi, v);
            }
        }
        publish1(v, sm, slot[P_BB]);
        err = grid_barrier(a.bar, a.spin_limit_ns, target);
        bb = total(slot[P_BB], &s_tot);
    }
    const double bbs = bb > 0.0 ? bb : 1.0;
    const double tol2 = a.tol * a.tol;

    // z = (LU)^-1 r for the levels after the first (level-0 rows already hold z = r); returns (r, z)
    auto precondition = [&](double& gamma) -> bool {
        double g64 = 0.0;
        VT g[1] = {VT(0)};
        for (int l = 1; l < C; ++l) {
            int r0, r1;
            level_rows(a, l, r0, r1);
            const bool ok = part_spmv<PAT>(a, ring, a.pL, vv.L, (const VT*)z, r0, r1,
                                           EmForward<VT>{r, z, vv.dinv, l == C - 1, g});
            if (grid_barrier(a.bar, a.spin_limit_ns, target) || !ok) return false;
        }
        for (int l = C - 2; l >= 0; --l) {
            int r0, r1;
            level_rows(a, l, r0, r1);
            const bool ok =
                part_spmv<PAT>(a, ring, a.pU, vv.U, (const VT*)z, r0, r1, EmBackward<VT>{r, z, vv.dinv, g});
            if (l == 0) {
                g64 = (double)g[0];
                publish1(g64, sm, slot[P_GAMMA]);
            }
            if (grid_barrier(a.bar, a.spin_limit_ns, target) || !ok) return false;
        }
        gamma = total(slot[P_GAMMA], &s_tot);
        return true;
    };

    bool done = err;
    while (!done) {
        // FP64 residual of the current solution (the whole CG residual in FP64 mode)
        double rr32_0 = 0.0, gamma = 0.0;
        {
            double v[3] = {0.0, 0.0, 0.0};
            bool ok = true;
            for (int l = 0; l < C; ++l) {
                int r0, r1;
                level_rows(a, l, r0, r1);
                ok = part_spmv<PAT>(a, ring, a.pA, a.v64.A, (const double*)a.xv, r0, r1,
                                    EmResidual<MIXED>{a, l == 0, C == 1, v}) &&
                     ok;
            }
            publish1(v[0], sm, slot[P_RR64]);
            if (MIXED) publish1(v[1], sm, slot[P_RR32]);
            if (C == 1) publish1(v[2], sm, slot[P_GAMMA]);
            if (grid_barrier(a.bar, a.spin_limit_ns, target) || !ok) {
                err = true;
                break;
            }
            rr64 = total(slot[P_RR64], &s_tot);
            if (MIXED) rr32_0 = total(slot[P_RR32], &s_tot);
            if (C == 1) gamma = total(slot[P_GAMMA], &s_tot);  // (r, z) with a single level
            relres = sqrt(rr64 / bbs);
        }
        if (!(rr64 == rr64)) {
            status = RAFEM_ERR_NONFINITE;
            break;
        }
        if (rr64 <= tol2 * bbs) {
            status = RAFEM_OK;
            break;
        }
        if (iters >= a.max_iter || (MIXED && refine >= a.max_refine)) break;
        if (MIXED) ++refine;
        if (C > 1 && !precondition(gamma)) {
            err = true;
            break;
        }
        // the inner solve's stop on (r, r): FP64 mode the target itself; mixed inner_tol of its start, or the
        // predicted FP64 target (||r64|| times the inner reduction)
        const double thr = MIXED ? fmax(a.inner_tol * a.inner_tol, tol2 * bbs / fmax(rr64, 1e-300)) * rr32_0
                                 : tol2 * bbs;
        bool first = true;
        double beta = 0.0, rr = MIXED ? rr32_0 : rr64;
        while (true) {
            if (!(gamma > 0.0)) {
                // lost positive curvature: FP64 mode stops; mixed keeps the correction found so far
                if (!MIXED) status = gamma == gamma ? RAFEM_ERR_BREAKDOWN : RAFEM_ERR_NONFINITE;
                break;
            }
            // A: q = A z + beta q, p = z + beta p; (p, q)
            double delta;
            {
                VT v[1] = {VT(0)};
                bool ok = true;
                for (int l = 0; l < C; ++l) {
                    int r0, r1;
                    level_rows(a, l, r0, r1);
                    ok = part_spmv<PAT>(a, ring, a.pA, vv.A, (const VT*)z, r0, r1,
                                        EmDirection<VT>{z, p, q, (VT)beta, first, v}) &&
                         ok;
                }
                publish1((double)v[0], sm, slot[P_DELTA]);
                if (grid_barrier(a.bar, a.spin_limit_ns, target) || !ok) {
                    err = true;
                    break;
                }
                delta = total(slot[P_DELTA], &s_tot);
            }
            if (!(delta > 0.0)) {
                if (!MIXED) status = delta == delta ? RAFEM_ERR_BREAKDOWN : RAFEM_ERR_NONFINITE;
                break;
            }
            const VT alpha = (VT)(gamma / delta);
            first = false;
            // B: x (or d) += alpha p, r -= alpha q; (r, r); level-0 rows z = r
            {
                double v = 0.0;
                for (int l = 0; l < C; ++l) {
                    int r0, r1;
                    level_rows(a, l, r0, r1);
                    const bool lev0 = l == 0;
                    for (int row = r0 + threadIdx.x; row < r1; row += kBlock) {
                        const VT pi = ldcg(p + row), qi = ldcg(q + row);
                        if constexpr (MIXED)
                            a.d32[row] = fmaf(alpha, pi, ldcg(a.d32 + row));
                        else
                            a.xv[row] = fma(alpha, pi, ldcg(a.xv + row));
                        const VT ri = fma(-alpha, qi, ldcg(r + row));
                        r[row] = ri;
                        v = fma((double)ri, (double)ri, v);
                        if (lev0) z[row] = C == 1 ? ri * ldcg(vv.dinv + row) : ri;
                    }
                }
                publish1(v, sm, slot[P_RR]);
                if (grid_barrier(a.bar, a.spin_limit_ns, target)) {
                    err = true;
                    break;
                }
                rr = total(slot[P_RR], &s_tot);
            }
            ++iters;
            if (!(rr == rr)) {
                status = RAFEM_ERR_NONFINITE;
                err = false;
                done = true;
                break;
            }
            if (rr <= thr) {
                if (!MIXED) status = RAFEM_OK;
                break;
            }
            if (iters >= a.max_iter) break;
            const double gprev = gamma;
            if (C > 1) {
                if (!precondition(gamma)) {
                    err = true;
                    break;
                }
            } else {
                double g = 0.0;
                int r0, r1;
                level_rows(a, 0, r0, r1);
                for (int row = r0 + threadIdx.x; row < r1; row += kBlock)
                    g = fma((double)ldcg(r + row), (double)ldcg(z + row), g);
                publish1(g, sm, slot[P_GAMMA]);
                if (grid_barrier(a.bar, a.spin_limit_ns, target)) {
                    err = true;
                    break;
                }
                gamma = total(slot[P_GAMMA], &s_tot);
            }
            beta = gamma / gprev;
        }
        if (err || done) break;
        if constexpr (!MIXED) {
            // FP64 mode: one pass; the true residual below gives the reported relative residual
            break;
        } else {
            // x64 += d (row-local), then the next FP64 residual
            for (int l = 0; l < C; ++l) {
                int r0, r1;
                level_rows(a, l, r0, r1);
                for (int row = r0 + threadIdx.x; row < r1; row += kBlock)
                    a.xv[row] = ldcg(a.xv + row) + (double)ldcg(a.d32 + row);
            }
            if (grid_barrier(a.bar, a.spin_limit_ns, target)) {
                err = true;
                break;
            }
        }
    }
    // FP64 mode: true residual of the final x; both modes: x back in the original order
    if (!err) {
        double v = 0.0;
        bool ok = true;
        for (int l = 0; l < C; ++l) {
            int r0, r1;
            level_rows(a, l, r0, r1);
            if (!MIXED) {
                struct EmTrue {
                    const double* bv;
                    double* v;
                    __device__ __forceinline__ double pre(int row) const { return ldcg(bv + row); }
                    __device__ __forceinline__ void fin(int, double ax, double bi) const {
                        const double t = bi - ax;
                        v[0] = fma(t, t, v[0]);
                    }
                };
                ok = part_spmv<PAT>(a, ring, a.pA, a.v64.A, (const double*)a.xv, r0, r1, EmTrue{a.bv, &v}) && ok;
            }
            for (int row = r0 + threadIdx.x; row < r1; row += kBlock) {
                const int o = __ldg(a.perm + row);
                if (o >= 0) a.x[o] = ldcg(a.xv + row);
            }
        }
        if (!MIXED) {
            publish1(v, sm, slot[P_TRUE]);
            if (grid_barrier(a.bar, a.spin_limit_ns, target) || !ok) err = true;
            else relres = sqrt(total(slot[P_TRUE], &s_tot) / bbs);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        InstState st = {};
        st.bb = bb;
        st.rr = rr64;
        st.iters = iters;
        st.refine = refine;
        st.status = err ? (a.bar->err ? a.bar->err : RAFEM_ERR_TIMEOUT) : status;
        st.relres = relres;
        a.inst[0] = st;
    }
}

// factor values of the combined layout -> the three ring layouts (FP64 and, in mixed precision, FP32 copies)
__global__ void k_ilu_split(long long n, const int32_t* __restrict__ src, const double* __restrict__ from,
                            double* __restrict__ to64, float* __restrict__ to32) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int s = src[q];
        const double v = s >= 0 ? from[s] : 0.0;
        if (to64) to64[q] = v;
        if (to32) to32[q] = (float)v;
    }
}

__global__ void k_narrow_vec(int n, const double* __restrict__ in, float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

template <bool MIXED, bool PAT>
void* kernel() {
    return (void*)k_ilu_ring<MIXED, PAT>;
}

void* pick(bool mixed, bool pat) {
    return mixed ? (pat ? kernel<true, true>() : kernel<true, false>())
                 : (pat ? kernel<false, true>() : kernel<false, false>());
}

}  // namespace

int ilu_ring_max_blocks() {
    int dev = 0, sms = 0, per = 1;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    for (bool m : {false, true})
        for (bool pt : {false, true}) {
            int q = 0;
            void* k = pick(m, pt);
            if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kRingBytes) != cudaSuccess)
                return 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, k, kBlock, kRingBytes) != cudaSuccess) return 0;
            per = q < per ? q : per;
        }
    return sms * per;
}

cudaError_t launch_ilu_ring_split(const IluRingDev& d, const double* Ap, const double* F, const double* dinv,
                                  bool mixed, cudaStream_t st) {
    struct Job {
        long long n;
        const int32_t* src;
        const double* from;
        double* to64;
        float* to32;
    } jobs[3] = {{d.nA, d.A.src, Ap, d.A64, mixed ? d.A32 : nullptr},
                 {d.nL, d.L.src, F, d.L64, mixed ? d.L32 : nullptr},
                 {d.nU, d.U.src, F, d.U64, mixed ? d.U32 : nullptr}};
    for (const Job& j : jobs) {
        if (j.n <= 0) continue;
        k_ilu_split<<<148 * 8, 256, 0, st>>>(j.n, j.src, j.from, j.to64, j.to32);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (mixed) {
        k_narrow_vec<<<(d.Np + 255) / 256, 256, 0, st>>>(d.Np, dinv, d.dinv32);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

cudaError_t launch_ilu_ring(const IluRingSolve& s, int grid, cudaStream_t st) {
    const IluRingDev& d = *s.d;
    Args a{};
    a.Np = d.Np;
    a.n_levels = d.n_levels;
    a.N = s.N;
    a.lvl = d.lvl;
    a.perm = d.perm;
    a.pA = Part{d.A.sp, d.A.sc, d.A.pat_off, d.A.pat_pool};
    a.pL = Part{d.L.sp, d.L.sc, d.L.pat_off, d.L.pat_pool};
    a.pU = Part{d.U.sp, d.U.sc, d.U.pat_off, d.U.pat_pool};
    a.v64 = Vals<double>{d.A64, d.L64, d.U64, s.dinv64};
    a.v32 = Vals<float>{d.A32, d.L32, d.U32, d.dinv32};
    a.b = s.b;
    a.x = s.x;
    a.xv = d.xv;
    a.bv = d.bv;
    a.r64 = d.r64;
    a.z64 = d.z64;
    a.p64 = d.p64;
    a.q64 = d.q64;
    a.r32 = d.r32;
    a.z32 = d.z32;
    a.p32 = d.p32;
    a.q32 = d.q32;
    a.d32 = d.d32;
    a.partial = d.partial;
    a.bar = s.bar;
    a.inst = s.inst;
    a.tol = s.tol;
    a.inner_tol = s.inner_tol;
    a.max_iter = s.max_iter;
    a.max_refine = s.max_refine;
    a.spin_limit_ns = s.spin_limit_ns;
    cudaError_t e = cudaMemsetAsync(s.bar, 0, sizeof(GridBarrier), st);
    if (e != cudaSuccess) return e;
    if (s.bar_missing > 0 && (e = launch_barrier_reset(s.bar, s.bar_missing, st)) != cudaSuccess) return e;
    void* params[] = {&a};
    return cudaLaunchCooperativeKernel(pick(s.mixed, d.patterns), dim3(grid), dim3(kBlock), params, kRingBytes, st);
}

}  // namespace rafem
