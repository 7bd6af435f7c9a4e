// Row-owner (gather) assembly of the monolithic step's 2 x 2 block Jacobian and residual (the 2N x 2N coupled
// system of Table II, Newton form): the same blocks as the colour scatter of assembly.cu, built in two passes
// without read-modify-write traffic on the matrix.
//   element pass: per (element e, vertex a) the quantities its blocks and residual need,
//       q_ea = { ds_e (G_e V_e)_a,  -sigma_e (G_e V_e)_a / 2,  sigma_e,  -ds_e (V_e^T G_e V_e) / 4 },
//       rt_ea = the thermal residual contribution of e to its vertex a,
//     sigma_e = sigma0_e (1 + alpha (Tbar_e - 37)), ds_e = sigma0_e alpha / 4;
//   row pass: for row i and each off-diagonal entry (i, j), over the elements sharing edge (i, j) with i = vertex
//     a and j = vertex b of e:
//       VV += sigma_e G_e[ab],  VT += q_ea.x,  TV += q_eb.y,  TT += q_ea.w  (+ the constant thermal entry),
//     and the diagonal from the row's incident elements: VV_ii = -(sum of the row's off-diagonal VV) (the rows of
//     G_e sum to zero), VT_ii = sum q_ea.x, TV_ii = sum q_ea.y, TT_ii = constant + sum q_ea.w; the residual
//     R_V,i = sum_e sigma_e (G_e V_e)_a = -2 sum q_ea.y and R_T,i = sum rt_ea. Dirichlet rows become identity
//     rows of their own unknown with residual x_i - g_i; columns are kept (row-only lift).
// Every entry is written exactly once (padding entries as zero), so the matrix and the residual need no clearing.
#include <cuda_runtime.h>

#include "internal.h"

namespace rafem {

namespace {

constexpr int kThreads = 256;
constexpr int kBatch = 4;  // contributions loaded together

inline int blocks_for(long long n) { return (int)((n + kThreads - 1) / kThreads); }

// index of the distinct entry (a, b) of a symmetric 4x4 element matrix in the G layout
__device__ __forceinline__ int gidx(int a, int b) {
    if (a == b) return a;
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return lo == 0 ? 3 + hi : (lo == 1 ? 5 + hi : 9);
}

// per contribution: G_e[a][b] (0 for padding)
__global__ void k_fill_contrib_G(long long nc, const int32_t* __restrict__ celem, const uint8_t* __restrict__ cab,
                                 const double* __restrict__ G, long long E, double* __restrict__ Gc) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nc; i += (long long)gridDim.x * blockDim.x) {
        const int c = cab[i];
        Gc[i] = c == 255 ? 0.0 : G[gidx(c >> 2, c & 3) * E + celem[i]];
    }
}

// The constant thermal block (unlifted): tc_ij = sum_e k_e G_e[ab] + cm vol_e / 20 (1 + [a == b]), cm = rho_c/dt +
// perf; the diagonal from the row's off-diagonal stiffness sums and its incident elements' masses.
__global__ void __launch_bounds__(kThreads) k_coupled_tconst(int N, const int32_t* __restrict__ sp,
                                                             const int32_t* __restrict__ diag, GatherData gd,
                                                             const uint8_t* __restrict__ cab,
                                                             const double* __restrict__ Gc, const double* __restrict__ kk,
                                                             const double* __restrict__ vol, double cm,
                                                             double* __restrict__ tc) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= N) return;
    const int s = row >> 5, lane = row & 31;
    const int base = sp[s], w = (sp[s + 1] - base) >> 5, q0 = base >> 5;
    const int dpos = diag[row];
    const double cmv = cm * (1.0 / 20.0);
    double ksum = 0.0;
    for (int k = 0; k < w; ++k) {
        const int pos = base + 32 * k + lane;
        if (pos == dpos) continue;
        const int P = gd.gcnt[q0 + k], off = gd.goff[q0 + k] + lane;
        double kg = 0.0, m = 0.0;
        for (int j = 0; j < P; ++j) {
            const int i = off + 32 * j;
            if (cab[i] == 255) continue;
            const int e = gd.celem[i];
            kg = fma(kk[e], Gc[i], kg);
            m += vol[e];
        }
        ksum += kg;
        tc[pos] = fma(cmv, m, kg);
    }
    const int off = gd.ioff[s] + lane, P = gd.icnt[s];
    double m = 0.0;
    for (int j = 0; j < P; ++j) {
        const int v = gd.ielem[off + 32 * j];
        if (v >= 0) m += vol[v >> 2];
    }
    tc[dpos] = fma(2.0 * cmv, m, -ksum);
}

__global__ void __launch_bounds__(kThreads) k_coupled_elem(ElemData el, const double* __restrict__ V,
                                                           const double* __restrict__ T,
                                                           const double* __restrict__ To, double alpha, double c_dt,
                                                           double perf, double T_a, double2* __restrict__ q,
                                                           double2* __restrict__ rt) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= el.E) return;
    const size_t E = (size_t)el.E;
    int n[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) n[a] = __ldg(el.nodes + a * E + e);
    double Ge[10];
#pragma unroll
    for (int c = 0; c < 10; ++c) Ge[c] = __ldg(el.G + c * E + e);
    const double sig0 = __ldg(el.sigma0 + e), kk = __ldg(el.k + e), vol = __ldg(el.vol + e);
    double v[4], t[4], to[4], tsum = 0.0, tosum = 0.0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        v[a] = V[n[a]];
        t[a] = T[n[a]];
        to[a] = To[n[a]];
        tsum += t[a];
        tosum += to[a];
    }
    const double sig = sig0 * (1.0 + alpha * (0.25 * tsum - 37.0)), ds = 0.25 * sig0 * alpha;
    double gv[4], gt[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        gv[a] = 0.0;
        gt[a] = 0.0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            gv[a] = fma(Ge[gidx(a, b)], v[b], gv[a]);
            gt[a] = fma(Ge[gidx(a, b)], t[b], gt[a]);
        }
    }
    const double quad = v[0] * gv[0] + v[1] * gv[1] + v[2] * gv[2] + v[3] * gv[3];
    const double mv = vol * (1.0 / 20.0), cm = c_dt + perf, tq = -0.25 * ds * quad;
    const double rconst = -perf * T_a * 0.25 * vol - 0.25 * sig * quad;
    double r[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        q[8 * (size_t)e + 2 * a] = make_double2(ds * gv[a], -0.5 * sig * gv[a]);
        q[8 * (size_t)e + 2 * a + 1] = make_double2(sig, tq);
        r[a] = fma(kk, gt[a], cm * mv * (tsum + t[a])) - c_dt * mv * (tosum + to[a]) + rconst;
    }
    rt[2 * (size_t)e] = make_double2(r[0], r[1]);
    rt[2 * (size_t)e + 1] = make_double2(r[2], r[3]);
}

__global__ void __launch_bounds__(kThreads) k_coupled_gather(
    int N, const int32_t* __restrict__ sp, const int32_t* __restrict__ diag, GatherData gd,
    const uint8_t* __restrict__ cab, const double* __restrict__ Gc, const double* __restrict__ tc,
    const double2* __restrict__ q, const double* __restrict__ rt, const uint8_t* __restrict__ bcV,
    const uint8_t* __restrict__ bcT, const double* __restrict__ gV, const double* __restrict__ gT,
    const double* __restrict__ V, const double* __restrict__ T, double* __restrict__ vals4, double* __restrict__ R) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= N) return;
    const bool dv = bcV[row] != 0, dt = bcT[row] != 0;
    const int s = row >> 5, lane = row & 31;
    const int base = __ldg(sp + s), w = (__ldg(sp + s + 1) - base) >> 5, q0 = base >> 5;
    const int dpos = __ldg(diag + row);
    double dsum = 0.0;
    for (int k = 0; k < w; ++k) {
        const int pos = base + 32 * k + lane;
        if (pos == dpos) continue;
        const int P = __ldg(gd.gcnt + q0 + k), off = __ldg(gd.goff + q0 + k) + lane;
        double vv = 0.0, vt = 0.0, tv = 0.0, tt = 0.0;
        for (int m0 = 0; m0 < P; m0 += kBatch) {
            int c[kBatch], e[kBatch];
            double g[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int i = off + 32 * (m0 + u);
                c[u] = m0 + u < P ? __ldg(cab + i) : 255;
                e[u] = c[u] != 255 ? __ldg(gd.celem + i) : 0;
                g[u] = c[u] != 255 ? __ldg(Gc + i) : 0.0;
            }
            double2 qx[kBatch], qs[kBatch];
            double tb[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                if (c[u] != 255) {
                    const size_t qa = 8 * (size_t)e[u] + 2 * (c[u] >> 2);
                    qx[u] = __ldg(q + qa);
                    qs[u] = __ldg(q + qa + 1);
                    tb[u] = __ldg(&q[8 * (size_t)e[u] + 2 * (c[u] & 3)].y);
                } else {
                    qx[u] = qs[u] = make_double2(0.0, 0.0);
                    tb[u] = 0.0;
                }
            }
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                vv = fma(g[u], qs[u].x, vv);
                vt += qx[u].x;
                tv += tb[u];
                tt += qs[u].y;
            }
        }
        dsum += vv;
        double* o = vals4 + 4 * (size_t)pos;
        o[0] = dv ? 0.0 : vv;
        o[1] = dv ? 0.0 : vt;
        o[2] = dt ? 0.0 : tv;
        o[3] = dt ? 0.0 : __ldg(tc + pos) + tt;
    }
    const int off = __ldg(gd.ioff + s) + lane, P = __ldg(gd.icnt + s);
    double vtd = 0.0, tvd = 0.0, ttd = 0.0, rtd = 0.0;
    for (int m = 0; m < P; ++m) {
        const int v = __ldg(gd.ielem + off + 32 * m);
        if (v < 0) continue;
        const double2 qx = __ldg(q + 2 * (size_t)v);
        vtd += qx.x;
        tvd += qx.y;
        ttd += __ldg(&q[2 * (size_t)v + 1].y);
        rtd += __ldg(rt + v);
    }
    double* o = vals4 + 4 * (size_t)dpos;
    o[0] = dv ? 1.0 : -dsum;
    o[1] = dv ? 0.0 : vtd;
    o[2] = dt ? 0.0 : tvd;
    o[3] = dt ? 1.0 : __ldg(tc + dpos) + ttd;
    R[2 * (size_t)row] = dv ? V[row] - gV[row] : -2.0 * tvd;
    R[2 * (size_t)row + 1] = dt ? T[row] - gT[row] : rtd;
}

}  // namespace

cudaError_t launch_coupled_fill(const CoupledGather& cg, const GatherData& gd, long long nc, int N, const int32_t* sp,
                                const int32_t* diag, const ElemData& el, double cm, bool geometry, cudaStream_t st) {
    if (geometry) {
        k_fill_contrib_G<<<148 * 8, kThreads, 0, st>>>(nc, gd.celem, cg.cab, el.G, el.E, cg.Gc);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_coupled_tconst<<<blocks_for(N), kThreads, 0, st>>>(N, sp, diag, gd, cg.cab, cg.Gc, el.k, el.vol, cm, cg.tc);
    return cudaGetLastError();
}

cudaError_t launch_coupled_gather(const CoupledGather& cg, const GatherData& gd, int N, const int32_t* sp,
                                  const int32_t* diag, const ElemData& el, const double* V, const double* T,
                                  const double* T_old, double alpha, double c_dt, double perf, double T_a,
                                  const uint8_t* bcV, const uint8_t* bcT, const double* gV, const double* gT,
                                  double* vals4, double* R, cudaStream_t st) {
    k_coupled_elem<<<blocks_for(el.E), kThreads, 0, st>>>(el, V, T, T_old, alpha, c_dt, perf, T_a, cg.q,
                                                          reinterpret_cast<double2*>(cg.rt));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_coupled_gather<<<blocks_for(N), kThreads, 0, st>>>(N, sp, diag, gd, cg.cab, cg.Gc, cg.tc, cg.q, cg.rt, bcV, bcT,
                                                         gV, gT, V, T, vals4, R);
    return cudaGetLastError();
}

}  // namespace rafem
