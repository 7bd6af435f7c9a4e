// Building blocks of the persistent SELL-32 solvers, shared by the CG family (krylov.cu), GMRES(m) (gmres.cu) and
// BiCGSTAB (bicgstab.cu): the block shape (16 consumer warps + one producer warp), the shared-memory ring that the
// producer fills with bulk copies (cp.async.bulk, completion on mbarriers) of groups of SELL-32 slices while the
// consumers compute on earlier groups, the SpMV over one tile of rows with a row epilogue ("emitter"), vectorised
// row-local passes and fixed-order block sums. Every wait is bounded: it gives up after the solver's wait limit,
// records RAFEM_ERR_TIMEOUT in the launch's barrier word and raises the block's abort flag.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "grid_sync.cuh"
#include "internal.h"

namespace rafem {
namespace sell {

constexpr int kConsumerWarps = 16;
constexpr int kBlock = (kConsumerWarps + 1) * 32;  // + one producer warp that issues the bulk copies
constexpr int kWarps = kBlock / 32;

// TMA staging of SELL-32 slices: groups of consecutive slices are copied into a ring of kSlots shared-memory
// slots of kSlotBytes (full/empty mbarrier pair per slot). A group holds as many slices as fit a slot at 16
// entries per row (8 for FP32 values with 16-bit columns, 4 for FP64 values), so every slot carries ~24 KB.
constexpr int kSlots = 8;
constexpr int kSlotBytes = 24576;
constexpr int kRingBytes = kSlots * kSlotBytes;
// Where a SELL entry's column comes from: a per-entry array streamed with the values through the ring (int32
// columns, or int16 offsets to the row), or one offset pattern shared by the 32 rows of each slice (nothing
// streamed: the column of slot k of row r is r + pattern[k], clamped to the rows; rows without that neighbour hold
// a zero there).
template <typename T>
struct EntryCols {
    const T* c;
};
struct SliceCols {
    const int32_t* off;   // [slices] first offset of each slice's pattern in pool
    const int32_t* pool;  // the distinct patterns
    int n;                // rows (columns are clamped to [0, n))
};
template <class C>
struct ColBytes;  // bytes streamed per entry
template <>
struct ColBytes<EntryCols<int32_t>> {
    static constexpr int v = 4;
};
template <>
struct ColBytes<EntryCols<int16_t>> {
    static constexpr int v = 2;
};
template <>
struct ColBytes<SliceCols> {
    static constexpr int v = 0;
};

template <typename VT, class C>
constexpr int group_slices() {
    return kSlotBytes / (32 * 16 * (int)(sizeof(VT) + ColBytes<C>::v)) >= 8 ? 8 : 4;
}

// Loads of data written by other blocks during the kernel go through L2 (L1 is not coherent).
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }

// The matrix is streamed once per SpMV: loaded with an L2 evict-first policy (and no L1 allocation) so that
// the Krylov vectors, which every phase touches again, stay resident in L2.
__device__ __forceinline__ unsigned long long policy_stream() {
    unsigned long long p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ double ldm(const double* p, unsigned long long pol) {
    double v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float ldm(const float* p, unsigned long long pol) {
    float v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ int ldm(const int* p, unsigned long long pol) {
    int v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}

// ---- mbarrier + bulk-copy primitives (shared memory addresses are 32-bit shared-window offsets) ----------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// Bulk copy global -> shared; both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, unsigned long long* bar,
                                          unsigned long long pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

// W consecutive values loaded/stored as one vector access (W = 1, 2 for double; 1, 4 for float).
template <typename T, int W>
struct Vec {
    T v[W];
};
template <typename T, int W>
__device__ __forceinline__ Vec<T, W> ldv(const T* p) {
    Vec<T, W> r;
    if constexpr (W == 1) {
        r.v[0] = __ldcg(p);
    } else if constexpr (sizeof(T) == 8 && W == 2) {
        double2 q = __ldcg(reinterpret_cast<const double2*>(p));
        r.v[0] = q.x;
        r.v[1] = q.y;
    } else {
        static_assert(sizeof(T) == 4 && W == 4, "vector width");
        float4 q = __ldcg(reinterpret_cast<const float4*>(p));
        r.v[0] = q.x;
        r.v[1] = q.y;
        r.v[2] = q.z;
        r.v[3] = q.w;
    }
    return r;
}
template <typename T, int W>
__device__ __forceinline__ void stv(T* p, const Vec<T, W>& r) {
    if constexpr (W == 1) {
        p[0] = r.v[0];
    } else if constexpr (sizeof(T) == 8 && W == 2) {
        *reinterpret_cast<double2*>(p) = make_double2(r.v[0], r.v[1]);
    } else {
        *reinterpret_cast<float4*>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
    }
}

// Visit rows [r0, r1) of a tile: aligned groups of W rows as f.template operator()<W>(i), the unaligned head
// and tail one row at a time.
template <int W, class F>
__device__ __forceinline__ void for_rows(int r0, int r1, const F& f) {
    int a0 = (r0 + W - 1) / W * W;
    if (a0 > r1) a0 = r1;
    const int a1 = a0 + (r1 - a0) / W * W;
    for (int i = r0 + threadIdx.x; i < a0; i += kBlock) f.template operator()<1>(i);
    int i = a0 + W * threadIdx.x;
    for (; i + W * kBlock < a1; i += 2 * W * kBlock) f.template pair<W>(i, i + W * kBlock);
    if (i < a1) f.template operator()<W>(i);
    for (int j = a1 + threadIdx.x; j < r1; j += kBlock) f.template operator()<1>(j);
}

// Block-wide sum of NQ (<= 2) values with a fixed order; result valid in thread 0. Every thread stages its
// values in shared memory and one warp per quantity adds them up: the block issues ~kWarps + 5 add
// instructions per quantity instead of 5 per warp, which matters for FP64 (B300 retires ~2 FP64 FMAs per
// clock per SM).
constexpr int kSumMax = 2;
template <int NQ, typename T>
__device__ __forceinline__ void block_sum(T (&v)[NQ], T* sm /* [kSumMax * kBlock] */) {
    static_assert(NQ <= kSumMax, "block_sum handles at most kSumMax values");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) sm[q * kBlock + threadIdx.x] = v[q];
    __syncthreads();
    if (warp < NQ) {
        T acc = sm[warp * kBlock + lane];
#pragma unroll
        for (int k = 1; k < kWarps; ++k) acc += sm[warp * kBlock + 32 * k + lane];
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        __syncwarp();
        if (lane == 0) sm[warp * kBlock] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < NQ; ++q) v[q] = sm[q * kBlock];
    __syncthreads();
}

// ---- SpMV over the rows of one tile -------------------------------------------------------------------------
// An emitter provides pre(row) -> P (row-local loads issued before the row's products, so they overlap the
// gathers) and fin(row, value, P) (consumes y_row = sum_k A_rk x_k).

// Ring of shared-memory slots receiving bulk copies of SELL-32 slice groups. Group J (counted over the whole
// kernel) lives in slot J % kSlots; full[slot] completes when its bytes have landed, empty[slot] when the
// consumer warps of the group are done with it.
struct Ring {
    unsigned char* data;        // kSlots x kSlotBytes: values, then columns
    unsigned long long* full;   // [kSlots], arrival count 1 + transaction bytes
    unsigned long long* empty;  // [kSlots], arrival count kConsumerWarps
    int* st_n;                  // [kSlots] slices in the group; negative = group too large, read directly
    int* abort;                 // shared flag: a wait gave up, stop waiting
    unsigned base;              // groups issued before the current SpMV (identical in every thread)
};

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_n(unsigned long long* bar, unsigned n) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(n) : "memory");
}

// Bounded wait; gives up (recording RAFEM_ERR_TIMEOUT and raising the block's abort flag) after the spin
// limit, and returns at once while the abort flag is up.
// Ctl: any launch-argument type with spin_limit_ns (wall-clock limit) and bar (the launch's GridBarrier*).
template <class Ctl>
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity, const Ctl& a,
                                                  int* abort) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    long long spins = 0;
    while (!mbar_try_wait(bar, parity)) {
        if ((++spins & 63) == 0) {
            if (*(volatile int*)abort) return false;
            if ((long long)(globaltimer() - t0) > a.spin_limit_ns || spins > (1LL << 34)) {
                raise_barrier_error(a.bar, RAFEM_ERR_TIMEOUT);
                atomicExch(abort, 1);
                return false;
            }
        }
    }
    return true;
}

// Column of a SELL entry: stored directly (int32) or as a 16-bit delta to the row.
__device__ __forceinline__ int col_of(int32_t c, int) { return c; }
__device__ __forceinline__ int col_of(int16_t d, int row) { return row + (int)d; }
__device__ __forceinline__ int32_t ldm_col(const int32_t* p, unsigned long long pol) { return ldm(p, pol); }
__device__ __forceinline__ int16_t ldm_col(const int16_t* p, unsigned long long) { return __ldg(p); }

__device__ __forceinline__ int pattern_col(const SliceCols& cs, const int32_t* pat, int q, int row) {
    return min(max(row + __ldg(pat + q), 0), cs.n - 1);
}

template <typename VT, typename AT, class C, class Emit>
__device__ __forceinline__ void slice_direct(const int32_t* sp, const C& cs, const VT* A, const VT* xin, int slice,
                                             int r1, const Emit& em, unsigned long long pol) {
    const int lane = threadIdx.x & 31;
    const int row = (slice << 5) + lane;
    const int base = __ldg(sp + slice), w = (__ldg(sp + slice + 1) - base) >> 5;
    AT acc = AT(0);
    if constexpr (ColBytes<C>::v == 0) {
        const int32_t* pat = cs.pool + __ldg(cs.off + slice);
        for (int k = 0; k < w; ++k)
            acc = fma((AT)ldm(A + base + 32 * k + lane, pol), (AT)ldcg(xin + pattern_col(cs, pat, k, row)), acc);
    } else {
        for (int k = 0; k < w; ++k)
            acc = fma((AT)ldm(A + base + 32 * k + lane, pol),
                      (AT)ldcg(xin + col_of(ldm_col(cs.c + base + 32 * k + lane, pol), row)), acc);
    }
    if (row < r1) em.fin(row, acc, em.pre(row));
}

// SELL-32 SpMV over rows [r0, r1) of one tile (r0 a multiple of 32). The producer warp streams slice groups
// into the ring; consumer warps take one slice each, team by team, and never synchronise the whole block.
// Returns false when a wait gave up (the error is recorded in the barrier word).
template <typename VT, typename AT, class C, class Emit, class Ctl>
__device__ __forceinline__ bool sell_tile(const Ctl& a, Ring& g, const int32_t* __restrict__ sp, const C& cs,
                                          const VT* __restrict__ A, const VT* xin, int r0, int r1, const Emit& em) {
    constexpr int kCB = ColBytes<C>::v;
    const unsigned long long pol = policy_stream();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s_begin = r0 >> 5, s_end = (r1 + 31) >> 5;
    constexpr int kG = group_slices<VT, C>();
    constexpr int kCap = kG * 32 * 16;                 // entries per slot
    constexpr int kTeamsG = kConsumerWarps / kG;
    const int ngroups = (s_end - s_begin + kG - 1) / kG;
    bool ok = true;
    int issued = 0;  // producer lane: groups whose copies were issued in this call
    if (warp == kConsumerWarps) {
        if (lane == 0) {
            for (int j = 0; j < ngroups && ok; ++j) {
                const unsigned J = g.base + j;
                const int slot = (int)(J % kSlots);
                if (J >= (unsigned)kSlots) ok = mbar_wait_bounded(&g.empty[slot], ((J / kSlots) - 1) & 1, a, g.abort);
                if (!ok) break;
                issued = j + 1;
                const int s = s_begin + j * kG;
                const int ns = min(kG, s_end - s);
                const int base = __ldg(sp + s), endp = __ldg(sp + s + ns);
                const unsigned nb = (unsigned)(endp - base);
                if (nb > (unsigned)kCap) {
                    g.st_n[slot] = -ns;
                    mbar_arrive(&g.full[slot]);
                } else {
                    g.st_n[slot] = ns;
                    unsigned char* dst = g.data + (size_t)slot * kSlotBytes;
                    fence_proxy_async();
                    mbar_arrive_tx(&g.full[slot], nb * (unsigned)(sizeof(VT) + kCB));
                    bulk_copy(dst, A + base, nb * (unsigned)sizeof(VT), &g.full[slot], pol);
                    if constexpr (kCB > 0)
                        bulk_copy(dst + (size_t)kCap * sizeof(VT), cs.c + base, nb * (unsigned)kCB, &g.full[slot], pol);
                }
            }
        }
    } else {
        const int team = warp / kG, member = warp % kG;
        for (int j = team; j < ngroups; j += kTeamsG) {
            const unsigned J = g.base + j;
            const int slot = (int)(J % kSlots);
            if (!mbar_wait_bounded(&g.full[slot], (J / kSlots) & 1, a, g.abort)) {
                ok = false;
                break;
            }
            const int n = g.st_n[slot];
            const int slice = s_begin + j * kG + member;
            if (n > 0 && member < n) {
                const int row = (slice << 5) + lane;
                const bool valid = row < r1;
                const int gb = __ldg(sp + s_begin + j * kG);
                const int off = __ldg(sp + slice) - gb;
                const int w = (__ldg(sp + slice + 1) - __ldg(sp + slice)) >> 5;
                const unsigned char* base = g.data + (size_t)slot * kSlotBytes;
                const VT* av = reinterpret_cast<const VT*>(base) + off + lane;
                // column of slot q of this row: from the streamed entry columns, or from the slice's pattern
                const int32_t* pat = nullptr;
                if constexpr (kCB == 0) pat = cs.pool + __ldg(cs.off + slice);
                auto colq = [&](int q) -> int {
                    if constexpr (kCB == 0) {
                        return pattern_col(cs, pat, q, row);
                    } else {
                        using T = typename std::remove_cv<typename std::remove_pointer<decltype(cs.c)>::type>::type;
                        const T* cv = reinterpret_cast<const T*>(base + (size_t)kCap * sizeof(VT)) + off + lane;
                        return col_of(cv[32 * q], row);
                    }
                };
                const auto pre = em.pre(valid ? row : r0);
                AT acc = AT(0);
                if (w <= 16) {
                    // one batch of gathers for the whole row: a single L2 round trip per slice
                    VT x[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) x[q] = q < w ? ldcg(xin + colq(q)) : VT(0);
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        if (q < w) acc = fma((AT)av[32 * q], (AT)x[q], acc);
                } else {
                    int k = 0;
                    for (; k + 8 <= w; k += 8) {
                        VT x[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) x[q] = ldcg(xin + colq(k + q));
#pragma unroll
                        for (int q = 0; q < 8; ++q) acc = fma((AT)av[32 * (k + q)], (AT)x[q], acc);
                    }
                    for (; k < w; ++k) acc = fma((AT)av[32 * k], (AT)ldcg(xin + colq(k)), acc);
                }
                if (valid) em.fin(row, acc, pre);
            } else if (n < 0 && member < -n) {
                slice_direct<VT, AT, C>(sp, cs, A, xin, slice, r1, em, pol);
            }
            __syncwarp();
            // the empty barrier expects kConsumerWarps arrivals per use: each of the kG warps of the team adds
            // kConsumerWarps / kG
            if (lane == 0) mbar_arrive_n(&g.empty[slot], kConsumerWarps / kG);
        }
    }
    const unsigned J0 = g.base;
    g.base += (unsigned)ngroups;
    if (__syncthreads_and(ok)) return true;
    // A wait gave up somewhere in the block: before the kernel exits, the producer lane waits for the copies that
    // may still be landing in shared memory. Only the last min(kSlots, issued) groups can be in flight (an
    // earlier group's slot was refilled only after its consumers had waited for its bytes), and each of them is
    // the newest user of its slot, so its full barrier's phase is unambiguous. Copies always complete, so one
    // overall deadline (kDrainNs, independent of the configurable wait limit) bounds the drain.
    if (warp == kConsumerWarps && lane == 0) {
        constexpr long long kDrainNs = 2000000000LL;
        const unsigned long long t0 = globaltimer();
        for (int j = max(0, issued - kSlots); j < issued; ++j) {
            const unsigned J = J0 + j;
            while (!mbar_try_wait(&g.full[J % kSlots], (J / kSlots) & 1) &&
                   (long long)(globaltimer() - t0) < kDrainNs) {
            }
        }
    }
    __syncthreads();
    return false;
}

// CSR SpMV with L lanes per row; pre/fin run on lane 0 of the row's group.
template <int L, typename VT, typename AT, class Emit>
__device__ __forceinline__ void csr_tile(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                         const VT* __restrict__ A, const VT* xin, int r0, int r1, const Emit& em) {
    const unsigned long long pol = policy_stream();
    const int lane = threadIdx.x & (L - 1);
    const int grp = threadIdx.x / L, ngrp = kBlock / L;
    const unsigned mask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << ((threadIdx.x & 31) & ~(L - 1)));
    for (int row = r0 + grp; row < r1; row += ngrp) {
        const int s = __ldg(rp + row), e = __ldg(rp + row + 1);
        AT acc = AT(0);
        for (int k = s + lane; k < e; k += L) acc = fma((AT)ldm(A + k, pol), (AT)ldcg(xin + ldm(ci + k, pol)), acc);
#pragma unroll
        for (int o = L / 2; o; o >>= 1) acc += __shfl_xor_sync(mask, acc, o, L);
        if (lane == 0) em.fin(row, acc, em.pre(row));
    }
}

// Block-uniform ring set-up at kernel start (SELL-32 kernels).
#define RAFEM_RING_SETUP(L_)                                                           \
    extern __shared__ __align__(128) unsigned char ring_data[];                       \
    __shared__ unsigned long long ring_full[kSlots], ring_empty[kSlots];              \
    __shared__ int ring_n[kSlots], ring_abort;                                        \
    Ring ring{ring_data, ring_full, ring_empty, ring_n, &ring_abort, 0u};             \
    if constexpr ((L_) <= 3) {                                                        \
        if (threadIdx.x == 0) {                                                       \
            for (int q = 0; q < kSlots; ++q) {                                        \
                mbar_init(&ring_full[q], 1);                                          \
                mbar_init(&ring_empty[q], kConsumerWarps);                            \
            }                                                                         \
            ring_abort = 0;                                                           \
            fence_proxy_async();                                                      \
        }                                                                             \
        __syncthreads();                                                              \
    }


}  // namespace sell
}  // namespace rafem
