// Element-level kernels: geometry, colour-partitioned atomic-free assembly with fused Dirichlet lift, thermal
// right-hand side (Joule source + mass term).
//
// Sec. III-A computes each element's equations in one GPU thread and places them in the CSR global matrix
// with threads mapped to disjoint matrix regions so that no two threads race. Here the disjointness comes
// from an element colouring: all elements of one colour share no node, so one launch per colour scatters
// its 16 entries per element with plain loads and stores (no atomics); successive colours are ordered by the
// stream. The Dirichlet lift is folded into the scatter: entries of Dirichlet rows are never written (they
// hold the identity set once at create), entries in Dirichlet columns of free rows move to the right-hand
// side as -A_ij g_j and stay zero in the matrix.
#include <cuda_runtime.h>

#include "internal.h"
#include "setup.h"

namespace rafem {

namespace {

constexpr int kThreads = 256;

// index of the distinct entry (a, b) of a symmetric 4x4 element matrix in the G layout
__device__ __forceinline__ int gidx(int a, int b) {
    if (a == b) return a;
    int lo = a < b ? a : b, hi = a < b ? b : a;
    // (0,1)->4 (0,2)->5 (0,3)->6 (1,2)->7 (1,3)->8 (2,3)->9
    return lo == 0 ? 3 + hi : (lo == 1 ? 5 + hi : 9);
}

__global__ void __launch_bounds__(kThreads) k_geometry(int E, const int32_t* __restrict__ nodes,
                                                       const double* __restrict__ xyz, double* __restrict__ G,
                                                       double* __restrict__ vol) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    double X[4][3];
    for (int a = 0; a < 4; ++a) {
        int n = nodes[(size_t)a * E + e];
        for (int c = 0; c < 3; ++c) X[a][c] = xyz[3 * (size_t)n + c];
    }
    double e1[3], e2[3], e3[3];
    for (int c = 0; c < 3; ++c) {
        e1[c] = X[1][c] - X[0][c];
        e2[c] = X[2][c] - X[0][c];
        e3[c] = X[3][c] - X[0][c];
    }
    // rows of the inverse edge matrix are cross products / det: grad(phi_1) = (e2 x e3)/det, ...
    double c[4][3];
    c[1][0] = e2[1] * e3[2] - e2[2] * e3[1];
    c[1][1] = e2[2] * e3[0] - e2[0] * e3[2];
    c[1][2] = e2[0] * e3[1] - e2[1] * e3[0];
    c[2][0] = e3[1] * e1[2] - e3[2] * e1[1];
    c[2][1] = e3[2] * e1[0] - e3[0] * e1[2];
    c[2][2] = e3[0] * e1[1] - e3[1] * e1[0];
    c[3][0] = e1[1] * e2[2] - e1[2] * e2[1];
    c[3][1] = e1[2] * e2[0] - e1[0] * e2[2];
    c[3][2] = e1[0] * e2[1] - e1[1] * e2[0];
    for (int q = 0; q < 3; ++q) c[0][q] = -(c[1][q] + c[2][q] + c[3][q]);
    double det = e1[0] * c[1][0] + e1[1] * c[1][1] + e1[2] * c[1][2];
    double adet = fabs(det);
    vol[e] = adet / 6.0;
    // vol * grad_a . grad_b = (|det|/6) * (c_a . c_b) / det^2 = c_a . c_b / (6 |det|)
    double s = 1.0 / (6.0 * adet);
    for (int a = 0; a < 4; ++a)
        for (int b = a; b < 4; ++b)
            G[(size_t)gidx(a, b) * E + e] = s * (c[a][0] * c[b][0] + c[a][1] * c[b][1] + c[a][2] * c[b][2]);
}

__global__ void k_init_rhs(int N, const uint8_t* __restrict__ bc, const double* __restrict__ g,
                           const double* __restrict__ base, double* __restrict__ b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    b[i] = bc[i] ? g[i] : (base ? base[i] : 0.0);
}

__global__ void k_set_identity(int N, const uint8_t* __restrict__ bc, const int32_t* __restrict__ diag,
                               double* __restrict__ vals, float* __restrict__ vals32) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N || !bc[i]) return;
    vals[diag[i]] = 1.0;
    if (vals32) vals32[diag[i]] = 1.0f;
}

// MODE 0: potential matrix  sigma(Tbar_e) * G_e
// MODE 1: thermal matrix    k_e * G_e + c_matrix * vol_e/20 * (1 + delta_ab), constant rhs perf*T_a*vol/4
// Memory accesses are batched into three dependent rounds (element data; nodal gathers; previous values of the
// slots to accumulate into) followed by the stores, instead of one read-modify-write chain per entry.
// row_lift = 1 keeps the Dirichlet columns of free rows in the matrix (no right-hand-side lift): the system is
// then nonsymmetric, with the same solution.
template <int MODE>
__global__ void __launch_bounds__(kThreads) k_assemble(ElemData el, int e0, int e1, const double* __restrict__ T,
                                                       const uint8_t* __restrict__ bc, const double* __restrict__ g,
                                                       double coef_a, double coef_b, double* __restrict__ vals,
                                                       float* __restrict__ vals32, double* __restrict__ rhs,
                                                       int row_lift, const int32_t* __restrict__ list) {
    const int ep = e0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (ep >= e1) return;
    const int e = list ? __ldg(list + ep) : ep;  // storage index of the element
    const size_t E = (size_t)el.E;
    // load stage 1: element data
    int n[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) n[a] = __ldg(el.nodes + a * E + e);
    int32_t code[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) code[q] = __ldg(el.slots + q * E + e);
    double Ge[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) Ge[q] = __ldg(el.G + q * E + e);
    const double own = MODE == 0 ? __ldg(el.sigma0 + e) : __ldg(el.k + e);
    const double vol = MODE == 1 ? __ldg(el.vol + e) : 0.0;
    // load stage 2: nodal gathers
    bool d[4];
    double tn[4] = {0.0, 0.0, 0.0, 0.0}, gn[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        d[a] = bc[n[a]] != 0;
        gn[a] = g[n[a]];
        if (MODE == 0) tn[a] = T[n[a]];
    }
    double scale, mdiag = 0.0, moff = 0.0, rhs_const = 0.0;
    if (MODE == 0) {
        const double Tbar = 0.25 * (tn[0] + tn[1] + tn[2] + tn[3]);
        scale = own * (1.0 + coef_a * (Tbar - 37.0));
    } else {
        scale = own;
        moff = coef_a * vol * (1.0 / 20.0);
        mdiag = 2.0 * moff;
        rhs_const = coef_b * vol * 0.25;
    }
    // load stage 3: previous values of the slots this element accumulates into
    double old[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int a = q >> 2, b = q & 3;
        const bool acc = !d[a] && (row_lift || !d[b]) && !(code[q] & SLOT_FIRST);
        old[q] = acc ? vals[code[q] & SLOT_MASK] : 0.0;
    }
    double rold[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) rold[a] = d[a] ? 0.0 : rhs[n[a]];
    // stores
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        if (d[a]) continue;  // Dirichlet row: identity, fixed at create
        double lift = 0.0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int q = a * 4 + b;
            double v = scale * Ge[gidx(a, b)];
            if (MODE == 1) v += (a == b) ? mdiag : moff;
            if (d[b] && !row_lift) {
                lift += v * gn[b];
            } else {
                const int32_t c = code[q];
                const double val = old[q] + v;
                vals[c & SLOT_MASK] = val;
                if (vals32 && (c & SLOT_LAST)) vals32[c & SLOT_MASK] = (float)val;
            }
        }
        if (MODE == 1 || lift != 0.0) rhs[n[a]] = rold[a] + (rhs_const - lift);
    }
}

// Monolithic Newton system of one colour (the 2N x 2N coupled step, unknowns (V_i, T_i) per node): residual
//   R_V = K(sigma(T)) V,   R_T = A_T T - (rho_c/dt) M T_old - perf T_a M 1 - F(V, sigma(T)),
// F_a = sum_e sigma_e V_e^T G_e V_e / 4, sigma_e = sigma0_e (1 + alpha (Tbar_e - 37)), and its Jacobian, one 2 x 2
// block (row-major: V row, T row) per stored entry of the node pattern:
//   dR_V/dV = sigma G,  dR_V/dT_b = ds (G V)_a,  dR_T/dV_b = -sigma (G V)_b / 2,
//   dR_T/dT = k G + (rho_c/dt + perf) M - ds (V^T G V) / 4,   ds = sigma0 alpha / 4.
// Blocks are stored by the slot's first writer and accumulated by the others (colour order); R accumulates
// (zeroed before the first colour). Dirichlet rows are replaced afterwards (k_coupled_dirichlet).
__global__ void __launch_bounds__(kThreads) k_coupled(ElemData el, int e0, int e1, const int32_t* __restrict__ list,
                                                      const double* __restrict__ V, const double* __restrict__ T,
                                                      const double* __restrict__ To, double alpha, double c_dt,
                                                      double perf, double T_a, double* __restrict__ vals4,
                                                      double* __restrict__ R) {
    const int ep = e0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (ep >= e1) return;
    const int e = list ? __ldg(list + ep) : ep;
    const size_t E = (size_t)el.E;
    int n[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) n[a] = __ldg(el.nodes + a * E + e);
    double Ge[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) Ge[q] = __ldg(el.G + q * E + e);
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
    const double mv = vol * (1.0 / 20.0), cm = c_dt + perf;
    double old[16][4];
    int32_t code[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        code[q] = __ldg(el.slots + q * E + e);
        const bool acc = !(code[q] & SLOT_FIRST);
        const size_t pos = 4 * (size_t)(code[q] & SLOT_MASK);
#pragma unroll
        for (int c = 0; c < 4; ++c) old[q][c] = acc ? vals4[pos + c] : 0.0;
    }
    double rv[4], rt[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        rv[a] = R[2 * (size_t)n[a]];
        rt[a] = R[2 * (size_t)n[a] + 1];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int q = a * 4 + b;
            const double g = Ge[gidx(a, b)];
            const size_t pos = 4 * (size_t)(code[q] & SLOT_MASK);
            vals4[pos + 0] = fma(sig, g, old[q][0]);
            vals4[pos + 1] = fma(ds, gv[a], old[q][1]);
            vals4[pos + 2] = fma(-0.5 * sig, gv[b], old[q][2]);
            vals4[pos + 3] = old[q][3] + (fma(kk, g, cm * mv * (a == b ? 2.0 : 1.0)) - 0.25 * ds * quad);
        }
        R[2 * (size_t)n[a]] = fma(sig, gv[a], rv[a]);
        R[2 * (size_t)n[a] + 1] =
            rt[a] + (fma(kk, gt[a], cm * mv * (tsum + t[a])) - c_dt * mv * (tosum + to[a]) - perf * T_a * 0.25 * vol -
                     0.25 * sig * quad);
    }
}

// Dirichlet rows of the monolithic system: the V (T) row of a node with a prescribed potential (temperature)
// becomes the identity row of its own unknown with residual x_i - g_i; columns are kept (row-only lift).
__global__ void k_coupled_dirichlet(int N, int sell, const int32_t* __restrict__ rp, const int32_t* __restrict__ diag,
                                    const uint8_t* __restrict__ bcV, const uint8_t* __restrict__ bcT,
                                    const double* __restrict__ gV, const double* __restrict__ gT,
                                    const double* __restrict__ V, const double* __restrict__ T,
                                    double* __restrict__ vals4, double* __restrict__ R) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const bool dv = bcV[i] != 0, dt = bcT[i] != 0;
    if (!dv && !dt) return;
    int q0, q1, stride;
    if (sell) {
        const int s = i >> 5, base = rp[s];
        q0 = base + (i & 31);
        q1 = base + (rp[s + 1] - base) + (i & 31);
        stride = 32;
    } else {
        q0 = rp[i];
        q1 = rp[i + 1];
        stride = 1;
    }
    for (int q = q0; q < q1; q += stride) {
        if (dv) vals4[4 * (size_t)q + 0] = vals4[4 * (size_t)q + 1] = 0.0;
        if (dt) vals4[4 * (size_t)q + 2] = vals4[4 * (size_t)q + 3] = 0.0;
    }
    const size_t d = 4 * (size_t)diag[i];
    if (dv) {
        vals4[d + 0] = 1.0;
        R[2 * (size_t)i] = V[i] - gV[i];
    }
    if (dt) {
        vals4[d + 3] = 1.0;
        R[2 * (size_t)i + 1] = T[i] - gT[i];
    }
}

// Newton update x <- x - delta (interleaved delta) of the potential and the temperature.
__global__ void k_newton_update(int N, const double* __restrict__ delta, double* __restrict__ V,
                                double* __restrict__ T) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    V[i] -= delta[2 * (size_t)i];
    T[i] -= delta[2 * (size_t)i + 1];
}

// Thermal right-hand side contributions of one element (free rows only):
//   Joule:  Q_e vol_e / 4 with Q_e vol_e = sigma_e * V_e^T G_e V_e   (= sigma_e vol_e |grad V|^2)
//   mass:   (rho_c/dt) (M_e T_old)_a = (rho_c/dt) vol_e/20 (sum_b T_b + T_a)
__global__ void __launch_bounds__(kThreads) k_rhs_T(ElemData el, int e0, int e1, const double* __restrict__ Ts,
                                                    const double* __restrict__ To, const double* __restrict__ V,
                                                    const uint8_t* __restrict__ bc, double alpha, double c_mass,
                                                    double* __restrict__ b) {
    const int e = e0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= e1) return;
    const size_t E = (size_t)el.E;
    int n[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) n[a] = __ldg(el.nodes + a * E + e);
    double Ge[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) Ge[q] = __ldg(el.G + q * E + e);
    const double sig0 = __ldg(el.sigma0 + e), vol = __ldg(el.vol + e);
    double v[4], to[4], ts = 0.0;
    bool d[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        v[a] = V[n[a]];
        to[a] = To[n[a]];
        ts += Ts[n[a]];
        d[a] = bc[n[a]] != 0;
    }
    double bold[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) bold[a] = d[a] ? 0.0 : b[n[a]];
    const double sig = sig0 * (1.0 + alpha * (0.25 * ts - 37.0));
    const double quad = Ge[0] * v[0] * v[0] + Ge[1] * v[1] * v[1] + Ge[2] * v[2] * v[2] + Ge[3] * v[3] * v[3] +
                        2.0 * (Ge[4] * v[0] * v[1] + Ge[5] * v[0] * v[2] + Ge[6] * v[0] * v[3] + Ge[7] * v[1] * v[2] +
                               Ge[8] * v[1] * v[3] + Ge[9] * v[2] * v[3]);
    const double q4 = 0.25 * sig * quad;
    const double mv = c_mass * vol * (1.0 / 20.0);
    const double tsum = to[0] + to[1] + to[2] + to[3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
        if (!d[a]) b[n[a]] = bold[a] + (q4 + mv * (tsum + to[a]));
}

// ---- row-owner ("gather") assembly on the SELL-32 layout --------------------------------------------------
// The potential matrix is K(T) = sum_e f_e (sigma0_e G_e) with f_e = 1 + alpha (Tbar_e - 37). One element pass
// writes f_e; then one thread per row sums, for each off-diagonal entry, the precomputed products
// c = sigma0_e G_e[a][b] of the elements sharing that edge, weighted by f_e. Because every element stiffness
// annihilates constants, K_ii = -sum_{j != i} K_ij, so the diagonal needs no list of its own. The lift is
// row-local: Dirichlet columns move to the right-hand side and stay zero, Dirichlet rows keep the identity.
// Every value is written once, in the slice layout, with no colouring.

__global__ void k_fill_cval(long long nc, const int32_t* __restrict__ celem, const uint8_t* __restrict__ cg,
                            const double* __restrict__ sigma0, const double* __restrict__ G, long long E,
                            double* __restrict__ cval) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nc; i += (long long)gridDim.x * blockDim.x) {
        const int g = cg[i];
        const int e = celem[i];
        cval[i] = g == 255 ? 0.0 : sigma0[e] * G[g * E + e];
    }
}

__global__ void __launch_bounds__(kThreads) k_sigma_factor(int E, const int32_t* __restrict__ nodes,
                                                           const double* __restrict__ T, double alpha,
                                                           double* __restrict__ f) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const size_t Es = (size_t)E;
    double ts = 0.0;
#pragma unroll
    for (int a = 0; a < 4; ++a) ts += T[__ldg(nodes + a * Es + e)];
    f[e] = 1.0 + alpha * (0.25 * ts - 37.0);
}

__global__ void __launch_bounds__(kThreads) k_assemble_V_gather(
    int N, const int32_t* __restrict__ sp, const int32_t* __restrict__ sc, const int32_t* __restrict__ diag,
    const int32_t* __restrict__ goff, const int32_t* __restrict__ gcnt, const double* __restrict__ cval,
    const int32_t* __restrict__ celem, const double* __restrict__ f, const uint8_t* __restrict__ bc,
    const double* __restrict__ g, double* __restrict__ vals, float* __restrict__ vals32, double* __restrict__ b,
    int row_lift) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= N) return;
    if (bc[row]) {
        b[row] = g[row];
        return;
    }
    const int s = row >> 5, lane = row & 31;
    const int base = __ldg(sp + s), w = (__ldg(sp + s + 1) - base) >> 5, q0 = base >> 5;
    const int dpos = __ldg(diag + row);
    double dsum = 0.0, lift = 0.0;
    for (int k = 0; k < w; ++k) {
        const int pos = base + 32 * k + lane;
        const int P = __ldg(gcnt + q0 + k);
        if (P == 0 || pos == dpos) continue;
        const int off = __ldg(goff + q0 + k) + lane;
        double acc = 0.0;
        for (int m = 0; m < P; ++m) acc = fma(__ldg(cval + off + 32 * m), f[__ldg(celem + off + 32 * m)], acc);
        dsum += acc;
        const int j = __ldg(sc + pos);
        if (j != row && bc[j] && !row_lift) {
            lift = fma(acc, g[j], lift);
        } else {
            vals[pos] = acc;
            if (vals32) vals32[pos] = (float)acc;
        }
    }
    vals[dpos] = -dsum;
    if (vals32) vals32[dpos] = (float)(-dsum);
    b[row] = -lift;
}

// Element pass of the thermal right-hand side: w_e = Q_e vol_e / 4 + (rho_c/dt) vol_e/20 * sum_b T_old,b with
// Q_e vol_e = sigma_e V_e^T G_e V_e and sigma_e at T_sigma. The pass is bound by the FP64 pipe (B300 issues FP64
// at a small fraction of its FP32 rate), so the quadratic form is arranged for FMAs (18 operations instead of
// ~30) and the temperature sum is shared when sigma and the mass term use the same field (the lagged step).
__global__ void __launch_bounds__(kThreads) k_rhsT_elem(ElemData el, const double* __restrict__ Ts,
                                                        const double* __restrict__ To, const double* __restrict__ V,
                                                        double alpha, double c20, double* __restrict__ w) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= el.E) return;
    const size_t E = (size_t)el.E;
    int n[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) n[a] = __ldg(el.nodes + a * E + e);
    double Ge[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) Ge[q] = __ldg(el.G + q * E + e);
    const double sig0 = __ldg(el.sigma0 + e), vol = __ldg(el.vol + e);
    double v[4], tsum = 0.0, ts;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        v[a] = V[n[a]];
        tsum += To[n[a]];
    }
    if (Ts == To) {
        ts = tsum;
    } else {
        ts = 0.0;
#pragma unroll
        for (int a = 0; a < 4; ++a) ts += Ts[n[a]];
    }
    const double q4 = 0.25 * (sig0 * fma(alpha, fma(0.25, ts, -37.0), 1.0));
    // v^T G v = sum_a G_aa v_a^2 + 2 sum_{a<b} G_ab v_a v_b
    const double a0 = fma(Ge[4], v[1], fma(Ge[5], v[2], Ge[6] * v[3]));
    const double a1 = fma(Ge[7], v[2], Ge[8] * v[3]);
    const double off = fma(v[0], a0, fma(v[1], a1, v[2] * (Ge[9] * v[3])));
    const double dia = fma(Ge[0] * v[0], v[0], fma(Ge[1] * v[1], v[1], fma(Ge[2] * v[2], v[2], Ge[3] * v[3] * v[3])));
    const double quad = fma(2.0, off, dia);
    w[e] = fma(q4, quad, (c20 * vol) * tsum);
}

// Row pass: b_i = bconst_i + mT_i T_old,i + sum_{e containing i} w_e for free rows, g_i for Dirichlet rows;
// mT_i = (rho_c/dt) sum_e vol_e / 20 (the T_a term of (M_e T_old)_a).
__global__ void __launch_bounds__(kThreads) k_rhsT_gather(int N, const int32_t* __restrict__ ioff,
                                                          const int32_t* __restrict__ icnt,
                                                          const int32_t* __restrict__ ielem,
                                                          const double* __restrict__ w, const double* __restrict__ mT,
                                                          const double* __restrict__ bconst,
                                                          const double* __restrict__ To, const uint8_t* __restrict__ bc,
                                                          const double* __restrict__ g, double* __restrict__ b) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= N) return;
    if (bc[row]) {
        b[row] = g[row];
        return;
    }
    const int s = row >> 5, lane = row & 31;
    const int off = __ldg(ioff + s) + lane, P = __ldg(icnt + s);
    double acc = 0.0;
    for (int m = 0; m < P; ++m) {
        const int v = __ldg(ielem + off + 32 * m);
        if (v >= 0) acc += w[v >> 2];
    }
    b[row] = bconst[row] + mT[row] * To[row] + acc;
}

// mT_i = c_mass * sum_{e containing i} vol_e / 20 (once at create).
__global__ void __launch_bounds__(kThreads) k_node_mass(int N, const int32_t* __restrict__ ioff,
                                                        const int32_t* __restrict__ icnt,
                                                        const int32_t* __restrict__ ielem,
                                                        const double* __restrict__ vol, double c_mass,
                                                        double* __restrict__ mT) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= N) return;
    const int s = row >> 5, lane = row & 31;
    const int off = __ldg(ioff + s) + lane, P = __ldg(icnt + s);
    double acc = 0.0;
    for (int m = 0; m < P; ++m) {
        const int v = __ldg(ielem + off + 32 * m);
        if (v >= 0) acc += vol[v >> 2];
    }
    mT[row] = c_mass * acc * (1.0 / 20.0);
}

__global__ void __launch_bounds__(kThreads) k_spmv64(int N, const int32_t* __restrict__ rp,
                                                     const int32_t* __restrict__ ci, const double* __restrict__ A,
                                                     const double* __restrict__ x, double* __restrict__ y) {
    // 8 lanes per row
    int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    int row = gtid >> 3, lane = gtid & 7;
    if (row >= N) return;
    double acc = 0.0;
    for (int k = rp[row] + lane; k < rp[row + 1]; k += 8) acc = fma(A[k], x[ci[k]], acc);
    unsigned mask = 0xffu << (threadIdx.x & 24);
    for (int o = 4; o; o >>= 1) acc += __shfl_xor_sync(mask, acc, o, 8);
    if (lane == 0) y[row] = acc;
}

__global__ void __launch_bounds__(kThreads) k_spmv64_sell(int N, const int32_t* __restrict__ sp,
                                                          const int32_t* __restrict__ sc,
                                                          const double* __restrict__ A, const double* __restrict__ x,
                                                          double* __restrict__ y) {
    int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= N) return;
    int s = row >> 5, lane = row & 31;
    int base = sp[s], w = (sp[s + 1] - base) >> 5;
    double acc = 0.0;
    for (int k = 0; k < w; ++k) acc = fma(A[base + 32 * k + lane], x[sc[base + 32 * k + lane]], acc);
    y[row] = acc;
}

__global__ void k_max_abs_diff(int N, const double* __restrict__ a, const double* __restrict__ b,
                               unsigned long long* out) {
    double m = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        m = fmax(m, fabs(a[i] - b[i]));
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    // non-negative doubles order like their bit patterns
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

inline unsigned blocks_for(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

cudaError_t launch_geometry(const ElemData& el, const double* xyz, double* G, double* vol, cudaStream_t st) {
    if (el.E == 0) return cudaSuccess;
    k_geometry<<<blocks_for(el.E), kThreads, 0, st>>>(el.E, el.nodes, xyz, G, vol);
    return cudaGetLastError();
}

cudaError_t launch_init_rhs(int N, const uint8_t* bc, const double* g, const double* base, double* b,
                            cudaStream_t st) {
    k_init_rhs<<<blocks_for(N), kThreads, 0, st>>>(N, bc, g, base, b);
    return cudaGetLastError();
}

cudaError_t launch_set_dirichlet_identity(int N, const uint8_t* bc, const int32_t* diag, double* vals,
                                          float* vals32, cudaStream_t st) {
    k_set_identity<<<blocks_for(N), kThreads, 0, st>>>(N, bc, diag, vals, vals32);
    return cudaGetLastError();
}

cudaError_t launch_assemble_V(const ElemData& el, int e0, int e1, const double* T, const uint8_t* bc,
                              const double* g, double alpha, double* vals, float* vals32, double* b, int row_lift,
                              cudaStream_t st) {
    if (e1 <= e0) return cudaSuccess;
    k_assemble<0><<<blocks_for(e1 - e0), kThreads, 0, st>>>(el, e0, e1, T, bc, g, alpha, 0.0, vals, vals32, b,
                                                            row_lift, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_assemble_T(const ElemData& el, int e0, int e1, const uint8_t* bc, const double* g,
                              double c_matrix, double perf_Ta, double* vals, float* vals32, double* bconst,
                              int row_lift, const int32_t* list, cudaStream_t st) {
    if (e1 <= e0) return cudaSuccess;
    k_assemble<1><<<blocks_for(e1 - e0), kThreads, 0, st>>>(el, e0, e1, nullptr, bc, g, c_matrix, perf_Ta, vals,
                                                            vals32, bconst, row_lift, list);
    return cudaGetLastError();
}

cudaError_t launch_rhs_T(const ElemData& el, int e0, int e1, const double* T_sigma, const double* T_old,
                         const double* V, const uint8_t* bc, double alpha, double c_mass, double* b,
                         cudaStream_t st) {
    if (e1 <= e0) return cudaSuccess;
    k_rhs_T<<<blocks_for(e1 - e0), kThreads, 0, st>>>(el, e0, e1, T_sigma, T_old, V, bc, alpha, c_mass, b);
    return cudaGetLastError();
}

cudaError_t launch_spmv64(int N, int sell, const int32_t* rp, const int32_t* ci, const double* A, const double* x,
                          double* y, cudaStream_t st) {
    if (sell)
        k_spmv64_sell<<<blocks_for(N), kThreads, 0, st>>>(N, rp, ci, A, x, y);
    else
        k_spmv64<<<blocks_for(8LL * N), kThreads, 0, st>>>(N, rp, ci, A, x, y);
    return cudaGetLastError();
}

cudaError_t launch_fill_cval(long long nc, const int32_t* celem, const uint8_t* cg, const double* sigma0,
                             const double* G, int E, double* cval, cudaStream_t st) {
    if (nc == 0) return cudaSuccess;
    k_fill_cval<<<148 * 8, kThreads, 0, st>>>(nc, celem, cg, sigma0, G, (long long)E, cval);
    return cudaGetLastError();
}

cudaError_t launch_assemble_V_gather(const GatherData& gd, int N, const int32_t* sp, const int32_t* sc,
                                     const int32_t* diag, const ElemData& el, const double* T, double alpha,
                                     const uint8_t* bc, const double* g, double* vals, float* vals32, double* b,
                                     int row_lift, cudaStream_t st) {
    k_sigma_factor<<<blocks_for(el.E), kThreads, 0, st>>>(el.E, el.nodes, T, alpha, gd.ework);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_assemble_V_gather<<<blocks_for(N), kThreads, 0, st>>>(N, sp, sc, diag, gd.goff, gd.gcnt, gd.cval, gd.celem,
                                                            gd.ework, bc, g, vals, vals32, b, row_lift);
    return cudaGetLastError();
}

cudaError_t launch_rhs_T_gather(const GatherData& gd, int N, const ElemData& el, const double* T_sigma,
                                const double* T_old, const double* V, const uint8_t* bc, const double* g,
                                const double* bconst, double alpha, double c_mass, double* b, cudaStream_t st) {
    k_rhsT_elem<<<blocks_for(el.E), kThreads, 0, st>>>(el, T_sigma, T_old, V, alpha, c_mass * (1.0 / 20.0),
                                                        gd.ework);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_rhsT_gather<<<blocks_for(N), kThreads, 0, st>>>(N, gd.ioff, gd.icnt, gd.ielem, gd.ework, gd.mT, bconst, T_old,
                                                      bc, g, b);
    return cudaGetLastError();
}

cudaError_t launch_node_mass(const GatherData& gd, int N, const double* vol, double c_mass, cudaStream_t st) {
    k_node_mass<<<blocks_for(N), kThreads, 0, st>>>(N, gd.ioff, gd.icnt, gd.ielem, vol, c_mass, gd.mT);
    return cudaGetLastError();
}

cudaError_t launch_coupled(const ElemData& el, int e0, int e1, const int32_t* list, const double* V, const double* T,
                           const double* T_old, double alpha, double c_dt, double perf, double T_a, double* vals4,
                           double* R, cudaStream_t st) {
    if (e1 <= e0) return cudaSuccess;
    k_coupled<<<blocks_for(e1 - e0), kThreads, 0, st>>>(el, e0, e1, list, V, T, T_old, alpha, c_dt, perf, T_a, vals4,
                                                         R);
    return cudaGetLastError();
}

cudaError_t launch_coupled_dirichlet(int N, int sell, const int32_t* rp, const int32_t* diag, const uint8_t* bcV,
                                     const uint8_t* bcT, const double* gV, const double* gT, const double* V,
                                     const double* T, double* vals4, double* R, cudaStream_t st) {
    k_coupled_dirichlet<<<blocks_for(N), kThreads, 0, st>>>(N, sell, rp, diag, bcV, bcT, gV, gT, V, T, vals4, R);
    return cudaGetLastError();
}

cudaError_t launch_newton_update(int N, const double* delta, double* V, double* T, cudaStream_t st) {
    k_newton_update<<<blocks_for(N), kThreads, 0, st>>>(N, delta, V, T);
    return cudaGetLastError();
}

cudaError_t launch_max_abs_diff(int N, const double* a, const double* b, double* out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), st);
    if (e != cudaSuccess) return e;
    k_max_abs_diff<<<148 * 4, kThreads, 0, st>>>(N, a, b, reinterpret_cast<unsigned long long*>(out));
    return cudaGetLastError();
}

}  // namespace rafem
