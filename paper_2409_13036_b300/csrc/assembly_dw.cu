// Row-owner (gather) assembly in double-word arithmetic: the same element and node passes as the FP64 gather
// kernels (potential matrix from sigma(T) of Sec. II-A, Joule source and backward-Euler thermal right-hand side),
// with every operation on the FP32 pipes through dw.cuh. FP64 inputs are split into float pairs by integer
// operations, either once per node per pass (the fields, k_split_fields) or once per context (the element
// constants, k_fill_cval_dw / k_fill_tq), and each FP64 value written costs one FP64 addition. The results agree
// with the FP64 kernels to a few units of 2^-48 relative to the magnitudes summed.
#include <cuda_runtime.h>

#include "dw.cuh"
#include "internal.h"

namespace rafem {

namespace {

constexpr int kThreads = 256;
constexpr int kBatch = 4;  // contributions loaded together (edges of the Kuhn lattice are shared by 4 or 6 tets)
using dw::df;

// The next column's contribution lists are prefetched into L2 while the current column is summed, so that its
// loads do not wait on DRAM (an L2 evict-first policy on these one-time streams and on the matrix stores was
// measured slightly slower).
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

inline int blocks_for(long long n) { return (int)((n + kThreads - 1) / kThreads); }

__global__ void __launch_bounds__(kThreads) k_split_fields(int N, const double* __restrict__ a, float2* __restrict__ a2,
                                                           const double* __restrict__ b, float2* __restrict__ b2,
                                                           const double* __restrict__ c, float2* __restrict__ c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    dw::store(a2 + i, dw::split(a[i]));
    if (b) dw::store(b2 + i, dw::split(b[i]));
    if (c) dw::store(c2 + i, dw::split(c[i]));
}

// sigma(T)/sigma0 = 1 + alpha (T_mean - 37) from the sum of the four nodal temperatures
__device__ __forceinline__ df sigma_factor(df tsum, df alpha) {
    return dw::add_fp(dw::mul(alpha, dw::add_fp(dw::scale(tsum, 0.25f), -37.0f)), 1.0f);
}

__device__ __forceinline__ df sum4(const float2* __restrict__ x, const int (&n)[4]) {
    return dw::add_fast(dw::add_fast(dw::ldg(x + n[0]), dw::ldg(x + n[1])),
                        dw::add_fast(dw::ldg(x + n[2]), dw::ldg(x + n[3])));
}

__global__ void __launch_bounds__(kThreads) k_sigma_factor_dw(int E, const int32_t* __restrict__ nodes,
                                                              const float2* __restrict__ Ts, float2 alpha,
                                                              float2* __restrict__ f) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const size_t Es = (size_t)E;
    int n[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) n[a] = __ldg(nodes + a * Es + e);
    dw::store(f + e, sigma_factor(sum4(Ts, n), dw::make(alpha.x, alpha.y)));
}

// Row i of A_V: off-diagonal a_ij = sum over the elements sharing edge (i, j) of sigma0_e G_e[ab] f_e, diagonal
// = -(sum of the row's off-diagonals) (zero row sums of the stiffness), Dirichlet columns lifted into b_i.
// kY: also (A D)_i for the projection predictor's basis D (4 float pairs per node, entries >= kin[0] zero), from
// the same row of the lifted matrix (lifted columns excluded), so the predictor needs no pass over A.
template <bool kY>
__global__ void __launch_bounds__(kThreads) k_assemble_V_gather_dw(
    int N, const int32_t* __restrict__ sp, const int32_t* __restrict__ sc, const int32_t* __restrict__ diag,
    const int32_t* __restrict__ goff, const int32_t* __restrict__ gcnt, const float2* __restrict__ cval,
    const int32_t* __restrict__ celem, const float2* __restrict__ f, const uint8_t* __restrict__ bc,
    const double* __restrict__ g, double* __restrict__ vals, float* __restrict__ vals32, double* __restrict__ b,
    int row_lift, const float4* __restrict__ D, float4* __restrict__ Y, const int32_t* __restrict__ kin) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= N) return;
    if (bc[row]) {
        b[row] = g[row];
        return;
    }
    const int s = row >> 5, lane = row & 31;
    const int base = __ldg(sp + s), w = (__ldg(sp + s + 1) - base) >> 5, q0 = base >> 5;
    const int dpos = __ldg(diag + row);
    const bool wy = kY && *kin > 0;  // written by the previous launch
    df y[4] = {dw::make(0.0f), dw::make(0.0f), dw::make(0.0f), dw::make(0.0f)};
    df dsum = dw::make(0.0f), lift = dw::make(0.0f);
    int P_next = w > 0 ? __ldg(gcnt + q0) : 0, off_next = w > 0 ? __ldg(goff + q0) : 0;
    for (int k = 0; k < w; ++k) {
        const int pos = base + 32 * k + lane;
        const int P = P_next, off = off_next + lane;
        if (k + 1 < w) {
            P_next = __ldg(gcnt + q0 + k + 1);
            off_next = __ldg(goff + q0 + k + 1);
            for (int m = 0; m < P_next; ++m) {  // in flight while this column's contributions are summed
                prefetch_l2(cval + off_next + lane + 32 * m);
                prefetch_l2(celem + off_next + lane + 32 * m);
            }
        }
        if (P == 0 || pos == dpos) continue;
        const int j = __ldg(sc + pos);
        float4 dj0, dj1;
        if (kY && wy) {  // the column's basis entries, loaded while its contributions are summed
            dj0 = __ldg(D + 2 * j);
            dj1 = __ldg(D + 2 * j + 1);
        }
        df acc = dw::make(0.0f);
        // contributions in batches: coefficients and element ids, then the factor gathers, then the arithmetic,
        // so that a batch costs two memory round trips instead of two per contribution
        for (int m0 = 0; m0 < P; m0 += kBatch) {
            float2 cv[kBatch];
            int ce[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const bool ok = m0 + u < P;
                cv[u] = ok ? __ldg(cval + off + 32 * (m0 + u)) : make_float2(0.0f, 0.0f);
                ce[u] = ok ? __ldg(celem + off + 32 * (m0 + u)) : -1;
            }
            float2 fv[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) fv[u] = ce[u] >= 0 ? __ldg(f + ce[u]) : make_float2(0.0f, 0.0f);
#pragma unroll
            for (int u = 0; u < kBatch; ++u)
                if (ce[u] >= 0) acc = dw::add_fast(acc, dw::mul(dw::make(cv[u].x, cv[u].y), dw::make(fv[u].x, fv[u].y)));
        }
        dsum = dw::add(dsum, acc);
        if (j != row && bc[j] && !row_lift) {
            lift = dw::add(lift, dw::mul(acc, dw::split(g[j])));
        } else {
            vals[pos] = dw::to_double(acc);
            if (vals32) vals32[pos] = acc.h;
            if (kY && wy) {
                dw::dot_acc(y[0], acc, dw::make(dj0.x, dj0.y));
                dw::dot_acc(y[1], acc, dw::make(dj0.z, dj0.w));
                dw::dot_acc(y[2], acc, dw::make(dj1.x, dj1.y));
                dw::dot_acc(y[3], acc, dw::make(dj1.z, dj1.w));
            }
        }
    }
    vals[dpos] = -dw::to_double(dsum);
    if (vals32) vals32[dpos] = -dsum.h;
    b[row] = -dw::to_double(lift);
    if (kY && wy) {
        const df aii = dw::neg(dsum);
        const float4 d0 = __ldg(D + 2 * row), d1 = __ldg(D + 2 * row + 1);
        dw::dot_acc(y[0], aii, dw::make(d0.x, d0.y));
        dw::dot_acc(y[1], aii, dw::make(d0.z, d0.w));
        dw::dot_acc(y[2], aii, dw::make(d1.x, d1.y));
        dw::dot_acc(y[3], aii, dw::make(d1.z, d1.w));
#pragma unroll
        for (int l = 0; l < 4; ++l) y[l] = dw::finish(y[l]);
        Y[2 * row] = make_float4(y[0].h, y[0].l, y[1].h, y[1].l);
        Y[2 * row + 1] = make_float4(y[2].h, y[2].l, y[3].h, y[3].l);
    }
}

// Element pass of the thermal right-hand side: w_e = f_e sum_{a<b} q_ab (V_a - V_b)^2 + m_e sum_a T_old,a with
// q_ab = -sigma0_e G_e[ab] / 4 and m_e = (rho_c/dt) vol_e / 20 (tq). Because the rows of G_e sum to zero,
// V^T G_e V = -sum_{a<b} G_e[ab] (V_a - V_b)^2, so sigma_e V^T G_e V / 4 (the Joule heat Q_e vol_e shared by the
// four vertices) needs only the six edge coefficients and no cancelling squares of potentials.
__global__ void __launch_bounds__(kThreads) k_rhsT_elem_dw(int E, const int32_t* __restrict__ nodes,
                                                           const float2* __restrict__ tq, const float2* __restrict__ Ts,
                                                           const float2* __restrict__ To, const float2* __restrict__ V,
                                                           float2 alpha, float2* __restrict__ w) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const size_t Es = (size_t)E;
    int n[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) n[a] = __ldg(nodes + a * Es + e);
    df v[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) v[a] = dw::ldg(V + n[a]);
    const df to = sum4(To, n);
    const df f = sigma_factor(Ts == To ? to : sum4(Ts, n), dw::make(alpha.x, alpha.y));
    constexpr int pa[6] = {0, 0, 0, 1, 1, 2}, pb[6] = {1, 2, 3, 2, 3, 3};
    df S = dw::make(0.0f);
#pragma unroll
    for (int k = 0; k < 6; ++k)
        S = dw::add_fast(S, dw::mul(dw::ldg(tq + k * Es + e), dw::sqr(dw::add_fast(v[pa[k]], dw::neg(v[pb[k]])))));
    dw::store(w + e, dw::add(dw::mul(f, S), dw::mul(dw::ldg(tq + 6 * Es + e), to)));
}

// Row pass: b_i = bconst_i + mT_i T_old,i + sum_{e containing i} w_e on free rows, g_i on Dirichlet rows.
__global__ void __launch_bounds__(kThreads) k_rhsT_gather_dw(int N, const int32_t* __restrict__ ioff,
                                                             const int32_t* __restrict__ icnt,
                                                             const int32_t* __restrict__ ielem,
                                                             const float2* __restrict__ w,
                                                             const double* __restrict__ mT,
                                                             const double* __restrict__ bconst,
                                                             const float2* __restrict__ To,
                                                             const uint8_t* __restrict__ bc,
                                                             const double* __restrict__ g, double* __restrict__ b) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= N) return;
    if (bc[row]) {
        b[row] = g[row];
        return;
    }
    const int s = row >> 5, lane = row & 31;
    const int off = __ldg(ioff + s) + lane, P = __ldg(icnt + s);
    df acc = dw::make(0.0f);
    for (int m0 = 0; m0 < P; m0 += 2 * kBatch) {
        int v[2 * kBatch];
#pragma unroll
        for (int u = 0; u < 2 * kBatch; ++u) v[u] = m0 + u < P ? __ldg(ielem + off + 32 * (m0 + u)) : -1;
        float2 wv[2 * kBatch];
#pragma unroll
        for (int u = 0; u < 2 * kBatch; ++u) wv[u] = v[u] >= 0 ? __ldg(w + (v[u] >> 2)) : make_float2(0.0f, 0.0f);
#pragma unroll
        for (int u = 0; u < 2 * kBatch; ++u)
            if (v[u] >= 0) dw::sum_acc(acc, dw::make(wv[u].x, wv[u].y));
    }
    acc = dw::finish(acc);
    const df base = dw::add(dw::split(bconst[row]), dw::mul(dw::split(mT[row]), dw::ldg(To + row)));
    b[row] = dw::to_double(dw::add(base, acc));
}

__global__ void k_fill_cval_dw(long long nc, const int32_t* __restrict__ celem, const uint8_t* __restrict__ cg,
                               const double* __restrict__ sigma0, const double* __restrict__ G, long long E,
                               float2* __restrict__ cval) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nc; i += (long long)gridDim.x * blockDim.x) {
        const int gi = cg[i];
        const int e = celem[i];
        dw::store(cval + i, gi == 255 ? dw::make(0.0f) : dw::split(sigma0[e] * G[gi * E + e]));
    }
}

// tq[k][e]: k < 6 the edge coefficients -sigma0_e G_e[ab] / 4 in the order (01, 02, 03, 12, 13, 23) (G entries
// 4..9), k = 6 the lumped mass factor c_mass vol_e / 20
__global__ void __launch_bounds__(kThreads) k_fill_tq(int E, const double* __restrict__ G, const double* __restrict__ vol,
                                                      const double* __restrict__ sigma0, double c_mass,
                                                      float2* __restrict__ tq) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const size_t Es = (size_t)E;
    const double q = -0.25 * sigma0[e];
#pragma unroll
    for (int k = 0; k < 6; ++k) dw::store(tq + k * Es + e, dw::split(q * G[(4 + k) * Es + e]));
    dw::store(tq + 6 * Es + e, dw::split(c_mass * (1.0 / 20.0) * vol[e]));
}

// host-side split of a double parameter into a float pair: the nearest float, then the nearest float to the rest
float2 split_host(double x) {
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
}

}  // namespace

cudaError_t launch_fill_dw(const GatherDw& d, long long nc, const int32_t* celem, const uint8_t* cg,
                           const ElemData& el, double c_mass, cudaStream_t st) {
    if (nc > 0) {
        k_fill_cval_dw<<<148 * 8, kThreads, 0, st>>>(nc, celem, cg, el.sigma0, el.G, (long long)el.E, d.cval);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_fill_tq<<<blocks_for(el.E), kThreads, 0, st>>>(el.E, el.G, el.vol, el.sigma0, c_mass, d.tq);
    return cudaGetLastError();
}

cudaError_t launch_assemble_V_gather_dw(const GatherData& gd, const GatherDw& d, int N, const int32_t* sp,
                                        const int32_t* sc, const int32_t* diag, const ElemData& el, const double* T,
                                        double alpha, const uint8_t* bc, const double* g, double* vals, float* vals32,
                                        double* b, int row_lift, const double* D, double* Y, const int32_t* kin,
                                        cudaStream_t st) {
    k_split_fields<<<blocks_for(N), kThreads, 0, st>>>(N, T, d.Ts, nullptr, nullptr, nullptr, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    float2* f = reinterpret_cast<float2*>(gd.ework);
    k_sigma_factor_dw<<<blocks_for(el.E), kThreads, 0, st>>>(el.E, el.nodes, d.Ts, split_host(alpha), f);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (D)
        k_assemble_V_gather_dw<true><<<blocks_for(N), kThreads, 0, st>>>(
            N, sp, sc, diag, gd.goff, gd.gcnt, d.cval, gd.celem, f, bc, g, vals, vals32, b, row_lift,
            reinterpret_cast<const float4*>(D), reinterpret_cast<float4*>(Y), kin);
    else
        k_assemble_V_gather_dw<false><<<blocks_for(N), kThreads, 0, st>>>(
            N, sp, sc, diag, gd.goff, gd.gcnt, d.cval, gd.celem, f, bc, g, vals, vals32, b, row_lift, nullptr, nullptr,
            nullptr);
    return cudaGetLastError();
}

cudaError_t launch_rhs_T_gather_dw(const GatherData& gd, const GatherDw& d, int N, const ElemData& el,
                                   const double* T_sigma, const double* T_old, const double* V, const uint8_t* bc,
                                   const double* g, const double* bconst, double alpha, double* b, cudaStream_t st) {
    const bool same = T_sigma == T_old;
    k_split_fields<<<blocks_for(N), kThreads, 0, st>>>(N, V, d.V, T_old, d.To, same ? nullptr : T_sigma,
                                                       same ? nullptr : d.Ts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    float2* w = reinterpret_cast<float2*>(gd.ework);
    k_rhsT_elem_dw<<<blocks_for(el.E), kThreads, 0, st>>>(el.E, el.nodes, d.tq, same ? d.To : d.Ts, d.To, d.V,
                                                          split_host(alpha), w);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_rhsT_gather_dw<<<blocks_for(N), kThreads, 0, st>>>(N, gd.ioff, gd.icnt, gd.ielem, w, gd.mT, bconst, d.To, bc, g, b);
    return cudaGetLastError();
}

}  // namespace rafem
