// Differentiation form: element and node passes of the discrete adjoint of the lagged time step.
//
// One step (Sec. II-A main loop, lagged coefficients) maps T^n to T^{n+1}:
//   sigma_e = sigma0_e f_e,  f_e = 1 + alpha (Tbar^n_e - 37)
//   K(sigma) V = 0 (lifted)                         -> V^{n+1}
//   F_a = sum_e sigma_e V_e^T G_e V_e / 4           (Joule source, G_e = vol_e grad(phi) grad(phi)^T)
//   A_T T^{n+1} = (rho_c/dt) M T^n + perf T_a M 1 + F (lifted)
// Given lam = dL/dT^{n+1} (zero on the thermal Dirichlet rows), the backward step is
//   A_T mu = lam                                     (A_T symmetric)
//   s_e = mean of mu over the element's nodes
//   h_a = sum_e 2 s_e sigma_e (G_e V_e)_a on free potential rows   ->   K nu = h
//   g_e = (s_e V_e - nu_e)^T G_e V_e                 (= dL/dsigma_e)
//   dL/dsigma0_e += g_e f_e,   dL/dk_e += -mu_e^T G_e T^{n+1}_e
//   dL/dT^n_a = (rho_c/dt) (M mu)_a + sum_e alpha sigma0_e g_e / 4
// The element passes below compute the per-element terms; node passes sum them over the node->element
// incidence (entries 4 e + a), so every value is written once and no atomics are used.
#include <cuda_runtime.h>

#include "internal.h"

namespace rafem {

namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// (G x)_a for the 10-entry symmetric layout (00,11,22,33,01,02,03,12,13,23)
__device__ __forceinline__ void gmul(const double* G, const double* x, double* y) {
    y[0] = G[0] * x[0] + G[4] * x[1] + G[5] * x[2] + G[6] * x[3];
    y[1] = G[4] * x[0] + G[1] * x[1] + G[7] * x[2] + G[8] * x[3];
    y[2] = G[5] * x[0] + G[7] * x[1] + G[2] * x[2] + G[9] * x[3];
    y[3] = G[6] * x[0] + G[8] * x[1] + G[9] * x[2] + G[3] * x[3];
}

struct ElemLoad {
    int n[4];
    double G[10];
};

__device__ __forceinline__ void load_elem(const ElemData& el, int e, ElemLoad& L) {
    const size_t E = (size_t)el.E;
#pragma unroll
    for (int a = 0; a < 4; ++a) L.n[a] = __ldg(el.nodes + a * E + e);
#pragma unroll
    for (int q = 0; q < 10; ++q) L.G[q] = __ldg(el.G + q * E + e);
}

// ew[a][e] = 2 s_e sigma_e (G_e V_e)_a
__global__ void __launch_bounds__(kThreads) k_adj_elem_h(ElemData el, const double* __restrict__ Tn,
                                                         const double* __restrict__ V, const double* __restrict__ mu,
                                                         double alpha, double* __restrict__ ew) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= el.E) return;
    ElemLoad L;
    load_elem(el, e, L);
    double v[4], ts = 0.0, ms = 0.0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        v[a] = V[L.n[a]];
        ts += Tn[L.n[a]];
        ms += mu[L.n[a]];
    }
    const double sig = __ldg(el.sigma0 + e) * (1.0 + alpha * (0.25 * ts - 37.0));
    const double c = 2.0 * (0.25 * ms) * sig;
    double gv[4];
    gmul(L.G, v, gv);
    const size_t E = (size_t)el.E;
#pragma unroll
    for (int a = 0; a < 4; ++a) ew[a * E + e] = c * gv[a];
}

// h_i = sum over incident (e, a) of ew[a][e] (+ extra_i), 0 on Dirichlet rows
__global__ void __launch_bounds__(kThreads) k_adj_node_h(int N, long long E, const int32_t* __restrict__ ioff,
                                                         const int32_t* __restrict__ icnt,
                                                         const int32_t* __restrict__ ielem,
                                                         const double* __restrict__ ew, const uint8_t* __restrict__ bc,
                                                         const double* __restrict__ extra, double* __restrict__ h) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= N) return;
    if (bc[row]) {
        h[row] = 0.0;
        return;
    }
    const int s = row >> 5, lane = row & 31;
    const int off = __ldg(ioff + s) + lane, P = __ldg(icnt + s);
    double acc = extra ? extra[row] : 0.0;
    for (int m = 0; m < P; ++m) {
        const int v = __ldg(ielem + off + 32 * m);
        if (v >= 0) acc += ew[(long long)(v & 3) * E + (v >> 2)];
    }
    h[row] = acc;
}

// Parameter gradients of one step and the element term of dL/dT^n:
//   g_e = (s_e V_e - nu_e)^T G_e V_e;  gs_e += g_e f_e;  gk_e -= mu_e^T G_e T1_e
//   w_e = c_mass vol_e/20 sum_b mu_b + alpha sigma0_e g_e / 4
__global__ void __launch_bounds__(kThreads) k_adj_elem_g(ElemData el, const double* __restrict__ Tn,
                                                         const double* __restrict__ V, const double* __restrict__ T1,
                                                         const double* __restrict__ mu, const double* __restrict__ nu,
                                                         double alpha, double c_mass, double* __restrict__ gs,
                                                         double* __restrict__ gk, double* __restrict__ w) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= el.E) return;
    ElemLoad L;
    load_elem(el, e, L);
    double v[4], t1[4], m[4], x[4], ts = 0.0, ms = 0.0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int n = L.n[a];
        v[a] = V[n];
        t1[a] = T1[n];
        m[a] = mu[n];
        x[a] = nu[n];
        ts += Tn[n];
        ms += m[a];
    }
    const double sig0 = __ldg(el.sigma0 + e), vol = __ldg(el.vol + e);
    const double f = 1.0 + alpha * (0.25 * ts - 37.0);
    const double s = 0.25 * ms;
    double gv[4], gt[4];
    gmul(L.G, v, gv);
    gmul(L.G, t1, gt);
    double g = 0.0, kt = 0.0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        g += (s * v[a] - x[a]) * gv[a];
        kt += m[a] * gt[a];
    }
    gs[e] += g * f;
    gk[e] -= kt;
    w[e] = c_mass * vol * (1.0 / 20.0) * ms + 0.25 * alpha * sig0 * g;
}

// lam_i = mT_i mu_i + sum over incident elements of w_e; Dirichlet rows 0 when zero_dirichlet
__global__ void __launch_bounds__(kThreads) k_adj_node_lambda(int N, const int32_t* __restrict__ ioff,
                                                              const int32_t* __restrict__ icnt,
                                                              const int32_t* __restrict__ ielem,
                                                              const double* __restrict__ w,
                                                              const double* __restrict__ mT,
                                                              const double* __restrict__ mu,
                                                              const uint8_t* __restrict__ bc, int zero_dirichlet,
                                                              double* __restrict__ lam) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= N) return;
    if (zero_dirichlet && bc[row]) {
        lam[row] = 0.0;
        return;
    }
    const int s = row >> 5, lane = row & 31;
    const int off = __ldg(ioff + s) + lane, P = __ldg(icnt + s);
    double acc = mT[row] * mu[row];
    for (int m = 0; m < P; ++m) {
        const int v = __ldg(ielem + off + 32 * m);
        if (v >= 0) acc += w[v >> 2];
    }
    lam[row] = acc;
}

__global__ void k_mask(int N, const uint8_t* __restrict__ bc, const double* __restrict__ in, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) out[i] = bc[i] ? 0.0 : in[i];
}

// out[perm[i]] = in[i] (scatter = 1) or out[i] = in[perm[i]] (scatter = 0)
__global__ void k_permute(int n, const int32_t* __restrict__ perm, const double* __restrict__ in,
                          double* __restrict__ out, int scatter) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (scatter)
        out[perm[i]] = in[i];
    else
        out[i] = in[perm[i]];
}

// Initial guess of an adjoint solve: polynomial extrapolation (order q, see the forward predictor) of the last
// solutions of the backward sweep; x holds the newest and is overwritten, the history shifts.
__global__ void k_adj_extrapolate(int N, double* __restrict__ x, double* __restrict__ h1, double* __restrict__ h2,
                                  int q) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double t = x[i], t1 = h1[i], t2 = h2[i];
    if (q >= 2)
        x[i] = 3.0 * (t - t1) + t2;
    else if (q == 1)
        x[i] = 2.0 * t - t1;
    h2[i] = t1;
    h1[i] = t;
}

// Sum of the Krylov iterations of one adjoint solve (maximum over instances) and the worst status.
__global__ void k_adj_count(const InstState* __restrict__ inst, int n_inst, const GridBarrier* __restrict__ bar,
                            int32_t* __restrict__ acc /* [iters_V, iters_T, status] */, int slot) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int it = 0, st = 0;
    for (int i = 0; i < n_inst; ++i) {
        it = max(it, inst[i].iters);
        const int s = bar->err ? bar->err : inst[i].status;
        if (s < 0 || st < 0)
            st = s < st ? s : st;
        else
            st = s > st ? s : st;
    }
    acc[slot] += it;
    const int s0 = acc[2];
    if (st < 0 || s0 < 0)
        acc[2] = st < s0 ? st : s0;
    else
        acc[2] = st > s0 ? st : s0;
}

}  // namespace

cudaError_t launch_adj_h(const ElemData& el, const GatherData& gd, int N, const double* Tn, const double* V,
                         const double* mu, double alpha, const uint8_t* bcV, const double* extra, double* ew4,
                         double* h, cudaStream_t st) {
    if (el.E > 0) k_adj_elem_h<<<blocks_for(el.E), kThreads, 0, st>>>(el, Tn, V, mu, alpha, ew4);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_adj_node_h<<<blocks_for(N), kThreads, 0, st>>>(N, el.E, gd.ioff, gd.icnt, gd.ielem, ew4, bcV, extra, h);
    return cudaGetLastError();
}

cudaError_t launch_adj_g(const ElemData& el, const GatherData& gd, int N, const double* Tn, const double* V,
                         const double* T1, const double* mu, const double* nu, double alpha, double c_mass,
                         const uint8_t* bcT, int zero_dirichlet, double* gs, double* gk, double* w, double* lam,
                         cudaStream_t st) {
    if (el.E > 0) k_adj_elem_g<<<blocks_for(el.E), kThreads, 0, st>>>(el, Tn, V, T1, mu, nu, alpha, c_mass, gs, gk, w);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_adj_node_lambda<<<blocks_for(N), kThreads, 0, st>>>(N, gd.ioff, gd.icnt, gd.ielem, w, gd.mT, mu, bcT,
                                                          zero_dirichlet, lam);
    return cudaGetLastError();
}

cudaError_t launch_mask(int N, const uint8_t* bc, const double* in, double* out, cudaStream_t st) {
    k_mask<<<blocks_for(N), kThreads, 0, st>>>(N, bc, in, out);
    return cudaGetLastError();
}

cudaError_t launch_permute(int n, const int32_t* perm, const double* in, double* out, int scatter, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_permute<<<blocks_for(n), kThreads, 0, st>>>(n, perm, in, out, scatter);
    return cudaGetLastError();
}

cudaError_t launch_adj_extrapolate(int N, double* x, double* h1, double* h2, int q, cudaStream_t st) {
    k_adj_extrapolate<<<blocks_for(N), kThreads, 0, st>>>(N, x, h1, h2, q);
    return cudaGetLastError();
}

cudaError_t launch_adj_count(const InstState* inst, int n_inst, const GridBarrier* bar, int32_t* acc, int slot,
                             cudaStream_t st) {
    k_adj_count<<<1, 32, 0, st>>>(inst, n_inst, bar, acc, slot);
    return cudaGetLastError();
}

}  // namespace rafem
