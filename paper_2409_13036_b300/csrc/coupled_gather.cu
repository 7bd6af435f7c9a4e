// Row-owner (gather) assembly of the monolithic step's 2 x 2 block Jacobian and residual (the 2N x 2N coupled
// system of Table II, Newton form): the same blocks as the colour scatter of assembly.cu, built in two passes
// without read-modify-write traffic on the matrix.
//   element pass: per element e a 64-byte record {sigma_e, ds_e, tq_e, 0, (G_e V_e)_0..3} and the parts of the
//     thermal residual that are not the constant thermal matrix times T,
//       rt_ea = -(rho_c/dt) (M_e T_old)_a - perf T_a vol_e / 4 - sigma_e (V_e^T G_e V_e) / 4,  with
//     sigma_e = sigma0_e (1 + alpha (Tbar_e - 37)), ds_e = sigma0_e alpha / 4, tq_e = -ds_e (V_e^T G_e V_e) / 4;
//   row pass: for row i and each off-diagonal entry (i, j), over the elements sharing edge (i, j) with i = vertex
//     a and j = vertex b of e:
//       VV += sigma_e G_e[ab],  VT += ds_e (G_e V_e)_a,  TV += -sigma_e (G_e V_e)_b / 2,  TT += tq_e
//     (+ the constant thermal entry), and the diagonal from the row's incident elements: VV_ii = -(sum of the
//     row's off-diagonal VV) (the rows of G_e sum to zero), VT_ii = sum ds_e (G_e V_e)_a, TV_ii = sum -sigma_e
//     (G_e V_e)_a / 2, TT_ii = constant + sum tq_e; the residual R_V,i = sum_e sigma_e (G_e V_e)_a = -2 TV_ii and
//     R_T,i = sum_j tc_ij T_j + sum rt_ea (tc the constant thermal matrix k G + (rho_c/dt + perf) M, unlifted).
//     Dirichlet rows become identity rows of their own unknown with residual x_i - g_i; columns are kept (row-only
//     lift).
// Every entry is written exactly once (padding entries as zero), so the matrix and the residual need no clearing.
// The records are what the row pass gathers (16 reads of each, from the four rows of its vertices): at 64 bytes
// they stay in L2 between those reads, and the one-time streams (contribution lists, matrix stores) bypass it.
#include <cuda_runtime.h>

#include "internal.h"

namespace rafem {

namespace {

constexpr int kThreads = 256;
constexpr int kBatch = 2;  // contributions loaded together (2 measured faster than 4 and 6)

inline int blocks_for(long long n) { return (int)((n + kThreads - 1) / kThreads); }

// 32 bytes through the read-only path in one access (sm_100 and later); p 32-byte aligned
__device__ __forceinline__ void ldg256(const double* p, double& a, double& b, double& c, double& d) {
    asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];" : "=d"(a), "=d"(b), "=d"(c), "=d"(d) : "l"(p));
}

// x[i] of four registers, i in 0..3
__device__ __forceinline__ double pick4(double x0, double x1, double x2, double x3, int i) {
    return i < 2 ? (i == 0 ? x0 : x1) : (i == 2 ? x2 : x3);
}

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
                                                           double perf, double T_a, double2* __restrict__ rec,
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
    const double sig0 = __ldg(el.sigma0 + e), vol = __ldg(el.vol + e);
    double v[4], to[4], tsum = 0.0, tosum = 0.0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        v[a] = V[n[a]];
        tsum += T[n[a]];
        tosum += To[n[a]];
        to[a] = To[n[a]];
    }
    const double sig = sig0 * (1.0 + alpha * (0.25 * tsum - 37.0)), ds = 0.25 * sig0 * alpha;
    double gv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        gv[a] = 0.0;
#pragma unroll
        for (int b = 0; b < 4; ++b) gv[a] = fma(Ge[gidx(a, b)], v[b], gv[a]);
    }
    const double quad = fma(v[0], gv[0], fma(v[1], gv[1], fma(v[2], gv[2], v[3] * gv[3])));
    // the FP64 pipe bounds this pass: the constant thermal matrix times T is left to the row pass, the mass term
    // -c_dt mv (tosum + to_a) shares its vertex-independent part, and every product folds into an FMA
    const double cdv = c_dt * vol * (1.0 / 20.0), tq = -0.25 * ds * quad;
    const double r0 = fma(-cdv, tosum, fma(-0.25 * sig, quad, -perf * T_a * 0.25 * vol));
    double2* o = rec + 4 * (size_t)e;
    o[0] = make_double2(sig, ds);
    o[1] = make_double2(tq, 0.0);
    o[2] = make_double2(gv[0], gv[1]);
    o[3] = make_double2(gv[2], gv[3]);
    double r[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) r[a] = fma(-cdv, to[a], r0);
    rt[2 * (size_t)e] = make_double2(r[0], r[1]);
    rt[2 * (size_t)e + 1] = make_double2(r[2], r[3]);
}

__global__ void __launch_bounds__(kThreads) k_coupled_gather(
    int N, const int32_t* __restrict__ sp, const int32_t* __restrict__ sc, const int32_t* __restrict__ diag,
    GatherData gd, const uint8_t* __restrict__ cab, const double* __restrict__ Gc, const double* __restrict__ tc,
    const double2* __restrict__ rec, const double* __restrict__ rt, const uint8_t* __restrict__ bcV,
    const uint8_t* __restrict__ bcT, const double* __restrict__ gV, const double* __restrict__ gT,
    const double* __restrict__ V, const double* __restrict__ T, double* __restrict__ vals4, double* __restrict__ R) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= N) return;
    const bool dv = bcV[row] != 0, dt = bcT[row] != 0;
    const int s = row >> 5, lane = row & 31;
    const int base = __ldg(sp + s), w = (__ldg(sp + s + 1) - base) >> 5, q0 = base >> 5;
    const int dpos = __ldg(diag + row);
    double dsum = 0.0, tcT = 0.0;  // tcT: the constant thermal matrix's row times T
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
                c[u] = m0 + u < P ? __ldcs(cab + i) : 255;
                e[u] = c[u] != 255 ? __ldcs(gd.celem + i) : 0;
                g[u] = c[u] != 255 ? __ldcs(Gc + i) : 0.0;
            }
            // each record in two 32-byte accesses: {sigma, ds, tq, 0} and (G V)_0..3
            double sg[kBatch], ds[kBatch], tq[kBatch], ga[kBatch], gb[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                if (c[u] != 255) {
                    const double* r = reinterpret_cast<const double*>(rec + 4 * (size_t)e[u]);
                    double z, g0, g1, g2, g3;
                    ldg256(r, sg[u], ds[u], tq[u], z);
                    ldg256(r + 4, g0, g1, g2, g3);
                    ga[u] = pick4(g0, g1, g2, g3, c[u] >> 2);
                    gb[u] = pick4(g0, g1, g2, g3, c[u] & 3);
                } else {
                    sg[u] = ds[u] = tq[u] = ga[u] = gb[u] = 0.0;
                }
            }
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                vv = fma(g[u], sg[u], vv);
                vt = fma(ds[u], ga[u], vt);
                tv = fma(-0.5 * sg[u], gb[u], tv);
                tt += tq[u];
            }
        }
        dsum += vv;
        const double tcij = __ldcs(tc + pos);
        tcT = fma(tcij, T[__ldcs(sc + pos)], tcT);
        double2* o = reinterpret_cast<double2*>(vals4 + 4 * (size_t)pos);
        __stcs(o, dv ? make_double2(0.0, 0.0) : make_double2(vv, vt));
        __stcs(o + 1, dt ? make_double2(0.0, 0.0) : make_double2(tv, tcij + tt));
    }
    const int off = __ldg(gd.ioff + s) + lane, P = __ldg(gd.icnt + s);
    const double tcii = __ldcs(tc + dpos);
    double vtd = 0.0, tvd = 0.0, ttd = 0.0, rtd = fma(tcii, T[row], tcT);
    for (int m = 0; m < P; ++m) {
        const int v = __ldg(gd.ielem + off + 32 * m);
        if (v < 0) continue;
        const double* r = reinterpret_cast<const double*>(rec + 4 * (size_t)(v >> 2));
        double sg, ds, tq, z, g0, g1, g2, g3;
        ldg256(r, sg, ds, tq, z);
        ldg256(r + 4, g0, g1, g2, g3);
        const double ga = pick4(g0, g1, g2, g3, v & 3);
        vtd = fma(ds, ga, vtd);
        tvd = fma(-0.5 * sg, ga, tvd);
        ttd += tq;
        rtd += __ldcs(rt + v);
    }
    double2* o = reinterpret_cast<double2*>(vals4 + 4 * (size_t)dpos);
    __stcs(o, dv ? make_double2(1.0, 0.0) : make_double2(-dsum, vtd));
    __stcs(o + 1, dt ? make_double2(0.0, 1.0) : make_double2(tvd, tcii + ttd));
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
                                  const int32_t* sc, const int32_t* diag, const ElemData& el, const double* V, const double* T,
                                  const double* T_old, double alpha, double c_dt, double perf, double T_a,
                                  const uint8_t* bcV, const uint8_t* bcT, const double* gV, const double* gT,
                                  double* vals4, double* R, cudaStream_t st) {
    k_coupled_elem<<<blocks_for(el.E), kThreads, 0, st>>>(el, V, T, T_old, alpha, c_dt, perf, T_a, cg.rec,
                                                          reinterpret_cast<double2*>(cg.rt));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_coupled_gather<<<blocks_for(N), kThreads, 0, st>>>(N, sp, sc, diag, gd, cg.cab, cg.Gc, cg.tc, cg.rec, cg.rt, bcV, bcT,
                                                         gV, gT, V, T, vals4, R);
    return cudaGetLastError();
}

}  // namespace rafem
