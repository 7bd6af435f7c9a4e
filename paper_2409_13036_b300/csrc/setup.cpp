// Host-side, once-per-mesh setup of the fixed sparse structure (integer graph work, OpenMP).
//
// The paper reuses analysis work because the global matrix pattern never changes between steps (Sec. III-B,
// the reused column permutation). Here everything that depends only on connectivity is built once:
//   - the CSR pattern of the node graph (row i holds every node sharing an element with i, sorted),
//   - the element -> CSR slot map (16 slots per tetrahedron),
//   - a greedy element colouring in which no two elements of one colour share a node, so that one colour's
//     element matrices can be scattered into the global matrix without atomics (Sec. III-A assembles by
//     mapping threads to disjoint matrix regions to avoid races),
//   - first/last-writer flags per slot in colour order (the first writer stores instead of adding, which
//     removes a per-step zeroing pass; the last writer also emits the FP32 copy of the finished value).
#include "setup.h"

#include <algorithm>
#include <map>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace rafem {

int validate_mesh(int N, int E, const int32_t* tets, const double* xyz, std::vector<int8_t>& orient,
                  double* vol_min, double* vol_max) {
    if (N < 4 || E < 1) return -1;
    int bad_index = 0, bad_vol = 0;
    double vmin = INFINITY, vmax = 0.0;
    orient.assign(E, 1);
#pragma omp parallel for reduction(+ : bad_index, bad_vol) reduction(min : vmin) reduction(max : vmax) schedule(static)
    for (int64_t e = 0; e < E; ++e) {
        const int32_t* t = tets + 4 * e;
        bool ok = true;
        for (int a = 0; a < 4; ++a)
            if (t[a] < 0 || t[a] >= N) ok = false;
        for (int a = 0; a < 4 && ok; ++a)
            for (int b = a + 1; b < 4; ++b)
                if (t[a] == t[b]) ok = false;
        if (!ok) { bad_index++; continue; }
        double e1[3], e2[3], e3[3];
        for (int c = 0; c < 3; ++c) {
            e1[c] = xyz[3 * t[1] + c] - xyz[3 * t[0] + c];
            e2[c] = xyz[3 * t[2] + c] - xyz[3 * t[0] + c];
            e3[c] = xyz[3 * t[3] + c] - xyz[3 * t[0] + c];
        }
        double det = e1[0] * (e2[1] * e3[2] - e2[2] * e3[1]) - e1[1] * (e2[0] * e3[2] - e2[2] * e3[0]) +
                     e1[2] * (e2[0] * e3[1] - e2[1] * e3[0]);
        double scale = 0;
        for (int c = 0; c < 3; ++c) scale = std::max({scale, std::fabs(e1[c]), std::fabs(e2[c]), std::fabs(e3[c])});
        if (!(std::fabs(det) > 1e-14 * scale * scale * scale) || !std::isfinite(det)) bad_vol++;
        orient[e] = det > 0 ? 1 : -1;
        vmin = std::min(vmin, std::fabs(det) / 6.0);
        vmax = std::max(vmax, std::fabs(det) / 6.0);
    }
    if (vol_min) *vol_min = vmin;
    if (vol_max) *vol_max = vmax;
    if (bad_index) return -1;
    if (bad_vol) return -2;
    return 0;
}

void build_pattern(int N, int E, const int32_t* tets, std::vector<int32_t>& row_ptr, std::vector<int32_t>& col) {
    // node -> element incidence
    std::vector<int32_t> cnt(N + 1, 0);
    for (int64_t i = 0; i < 4LL * E; ++i) cnt[tets[i] + 1]++;
    for (int i = 0; i < N; ++i) cnt[i + 1] += cnt[i];
    std::vector<int32_t> inc(4LL * E);
    {
        std::vector<int32_t> pos(cnt.begin(), cnt.end() - 1);
        for (int64_t e = 0; e < E; ++e)
            for (int a = 0; a < 4; ++a) inc[pos[tets[4 * e + a]]++] = (int32_t)e;
    }
    // per-row unique neighbour lists: count pass, then fill pass
    std::vector<int32_t> len(N, 0);
#pragma omp parallel
    {
        std::vector<int32_t> buf;
#pragma omp for schedule(dynamic, 1024)
        for (int i = 0; i < N; ++i) {
            buf.clear();
            buf.push_back(i);  // every row stores its diagonal, also for a node that no element touches
            for (int32_t q = cnt[i]; q < cnt[i + 1]; ++q)
                for (int a = 0; a < 4; ++a) buf.push_back(tets[4LL * inc[q] + a]);
            std::sort(buf.begin(), buf.end());
            len[i] = (int32_t)(std::unique(buf.begin(), buf.end()) - buf.begin());
        }
    }
    row_ptr.assign(N + 1, 0);
    for (int i = 0; i < N; ++i) row_ptr[i + 1] = row_ptr[i] + len[i];
    col.assign(row_ptr[N], 0);
#pragma omp parallel
    {
        std::vector<int32_t> buf;
#pragma omp for schedule(dynamic, 1024)
        for (int i = 0; i < N; ++i) {
            buf.clear();
            buf.push_back(i);
            for (int32_t q = cnt[i]; q < cnt[i + 1]; ++q)
                for (int a = 0; a < 4; ++a) buf.push_back(tets[4LL * inc[q] + a]);
            std::sort(buf.begin(), buf.end());
            int n = (int)(std::unique(buf.begin(), buf.end()) - buf.begin());
            std::copy(buf.begin(), buf.begin() + n, col.begin() + row_ptr[i]);
        }
    }
}

int color_elements(int N, int E, const int32_t* tets, std::vector<int32_t>& color) {
    // Greedy: each element takes the lowest colour not used by any element already coloured that shares one
    // of its nodes. Node masks hold up to 256 colours.
    const int W = 4;
    std::vector<uint64_t> used((size_t)N * W, 0);
    color.assign(E, -1);
    int ncol = 0;
    for (int64_t e = 0; e < E; ++e) {
        uint64_t m[W] = {0, 0, 0, 0};
        for (int a = 0; a < 4; ++a)
            for (int w = 0; w < W; ++w) m[w] |= used[(size_t)tets[4 * e + a] * W + w];
        int c = -1;
        for (int w = 0; w < W && c < 0; ++w)
            if (~m[w]) c = 64 * w + __builtin_ctzll(~m[w]);
        if (c < 0) return -1;
        color[e] = c;
        ncol = std::max(ncol, c + 1);
        for (int a = 0; a < 4; ++a) used[(size_t)tets[4 * e + a] * W + c / 64] |= 1ULL << (c % 64);
    }
    return ncol;
}

void build_slots(int E, const int32_t* tets, const std::vector<int32_t>& row_ptr, const std::vector<int32_t>& col,
                 const std::vector<int64_t>& order, std::vector<int32_t>& slots) {
    // slots is SoA over the colour-sorted element order: slots[(a*4+b)*E + e'] for element order[e'].
    slots.assign(16LL * E, 0);
#pragma omp parallel for schedule(static)
    for (int64_t ep = 0; ep < E; ++ep) {
        const int32_t* t = tets + 4 * order[ep];
        for (int a = 0; a < 4; ++a) {
            const int32_t* rb = col.data() + row_ptr[t[a]];
            const int32_t* re = col.data() + row_ptr[t[a] + 1];
            for (int b = 0; b < 4; ++b) {
                const int32_t* f = std::lower_bound(rb, re, t[b]);
                slots[(int64_t)(a * 4 + b) * E + ep] = (int32_t)(f - col.data());
            }
        }
    }
    // first / last writer in execution order (colour-sorted element order, any order inside a colour is
    // race-free because elements of one colour share no node and hence no slot)
    const int64_t nnz = (int64_t)col.size();
    std::vector<int64_t> first(nnz, -1), last(nnz, -1);
    for (int64_t ep = 0; ep < E; ++ep)
        for (int q = 0; q < 16; ++q) {
            int32_t s = slots[(int64_t)q * E + ep];
            int64_t id = ep * 16 + q;
            if (first[s] < 0) first[s] = id;
            last[s] = id;
        }
#pragma omp parallel for schedule(static)
    for (int64_t ep = 0; ep < E; ++ep)
        for (int q = 0; q < 16; ++q) {
            int32_t& s = slots[(int64_t)q * E + ep];
            int64_t id = ep * 16 + q;
            int32_t code = s;
            if (first[s] == id) code |= SLOT_FIRST;
            if (last[s] == id) code |= SLOT_LAST;
            s = code;
        }
}

void build_sell(int N, const std::vector<int32_t>& row_ptr, const std::vector<int32_t>& col,
                std::vector<int32_t>& slice_ptr, std::vector<int32_t>& sell_col, std::vector<int32_t>& csr_to_sell) {
    const int S = (N + SELL_C - 1) / SELL_C;
    slice_ptr.assign(S + 1, 0);
    for (int s = 0; s < S; ++s) {
        int w = 0;
        for (int r = s * SELL_C; r < std::min(N, (s + 1) * SELL_C); ++r) w = std::max(w, row_ptr[r + 1] - row_ptr[r]);
        slice_ptr[s + 1] = slice_ptr[s] + w * SELL_C;
    }
    sell_col.assign(slice_ptr[S], 0);
    csr_to_sell.assign(col.size(), 0);
#pragma omp parallel for schedule(static)
    for (int s = 0; s < S; ++s) {
        const int w = (slice_ptr[s + 1] - slice_ptr[s]) / SELL_C;
        for (int l = 0; l < SELL_C; ++l) {
            const int r = s * SELL_C + l;
            const int len = r < N ? row_ptr[r + 1] - row_ptr[r] : 0;
            for (int k = 0; k < w; ++k) {
                const int pos = slice_ptr[s] + k * SELL_C + l;
                if (k < len) {
                    sell_col[pos] = col[row_ptr[r] + k];
                    csr_to_sell[row_ptr[r] + k] = pos;
                } else {
                    sell_col[pos] = std::min(r, N - 1);
                }
            }
        }
    }
}

bool build_sell_patterns(int N, const std::vector<int32_t>& row_ptr, const std::vector<int32_t>& col,
                         std::vector<int32_t>& slice_ptr, std::vector<int32_t>& sell_col,
                         std::vector<int32_t>& csr_to_sell, std::vector<int32_t>& pat_off,
                         std::vector<int32_t>& pat_pool) {
    const int S = (N + SELL_C - 1) / SELL_C;
    std::vector<std::vector<int32_t>> pats(S);
    int64_t wide = 0, plain = 0;  // stored entries with shared patterns / with per-row slots
#pragma omp parallel for schedule(static) reduction(+ : wide, plain)
    for (int s = 0; s < S; ++s) {
        std::vector<int32_t>& u = pats[s];
        int w = 0;
        for (int r = s * SELL_C; r < std::min(N, (s + 1) * SELL_C); ++r) {
            w = std::max(w, row_ptr[r + 1] - row_ptr[r]);
            for (int32_t q = row_ptr[r]; q < row_ptr[r + 1]; ++q) u.push_back(col[q] - r);
        }
        std::sort(u.begin(), u.end());
        u.erase(std::unique(u.begin(), u.end()), u.end());
        wide += (int64_t)u.size();
        plain += w;
    }
    if (wide * 50 > plain * 51) return false;  // the shared patterns may add at most 2% of stored entries
    slice_ptr.assign(S + 1, 0);
    for (int s = 0; s < S; ++s) slice_ptr[s + 1] = slice_ptr[s] + (int32_t)pats[s].size() * SELL_C;
    // distinct patterns, each stored once in the pool
    pat_off.assign(S, 0);
    pat_pool.clear();
    std::map<std::vector<int32_t>, int32_t> seen;
    for (int s = 0; s < S; ++s) {
        auto it = seen.find(pats[s]);
        if (it == seen.end()) {
            it = seen.emplace(pats[s], (int32_t)pat_pool.size()).first;
            pat_pool.insert(pat_pool.end(), pats[s].begin(), pats[s].end());
        }
        pat_off[s] = it->second;
    }
    sell_col.assign(slice_ptr[S], 0);
    csr_to_sell.assign(col.size(), 0);
#pragma omp parallel for schedule(static)
    for (int s = 0; s < S; ++s) {
        const std::vector<int32_t>& u = pats[s];
        const int w = (int)u.size();
        for (int l = 0; l < SELL_C; ++l) {
            const int r = s * SELL_C + l;
            for (int k = 0; k < w; ++k) sell_col[slice_ptr[s] + k * SELL_C + l] = std::min(r, N - 1);
            if (r >= N) continue;
            for (int32_t q = row_ptr[r]; q < row_ptr[r + 1]; ++q) {
                const int k = (int)(std::lower_bound(u.begin(), u.end(), col[q] - r) - u.begin());
                const int pos = slice_ptr[s] + k * SELL_C + l;
                sell_col[pos] = col[q];
                csr_to_sell[q] = pos;
            }
        }
    }
    return true;
}

namespace {
int local_gidx(int a, int b) {
    if (a == b) return a;
    const int lo = std::min(a, b), hi = std::max(a, b);
    return lo == 0 ? 3 + hi : (lo == 1 ? 5 + hi : 9);
}
}  // namespace

void build_gather(int N, int E, const std::vector<int32_t>& row_ptr, const std::vector<int32_t>& col,
                  const std::vector<int32_t>& csr_slots, const std::vector<int32_t>& slice_ptr,
                  const std::vector<int32_t>& csr_to_sell, std::vector<int32_t>& gather_off,
                  std::vector<int32_t>& gather_cnt, std::vector<int32_t>& celem, std::vector<uint8_t>& cgidx,
                  std::vector<uint8_t>* cab) {
    (void)row_ptr;
    (void)N;
    const int64_t nnz = (int64_t)col.size();
    std::vector<int64_t> sell_to_csr(slice_ptr.back(), -1);  // CSR entry at each SELL position, -1 padding
    for (int64_t q = 0; q < nnz; ++q) sell_to_csr[csr_to_sell[q]] = q;
    std::vector<int32_t> cnt(nnz, 0);
    for (int64_t ep = 0; ep < E; ++ep)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b)
                if (a != b) cnt[csr_slots[(int64_t)(a * 4 + b) * E + ep] & SLOT_MASK]++;
    const int S = (int)slice_ptr.size() - 1;
    const int64_t Q = (int64_t)slice_ptr[S] / SELL_C;
    gather_off.assign(Q, 0);
    gather_cnt.assign(Q, 0);
    std::vector<int64_t> pos(nnz, -1);  // list start of each CSR entry (lane included)
    int64_t total = 0;
    for (int s = 0; s < S; ++s) {
        const int w = (slice_ptr[s + 1] - slice_ptr[s]) / SELL_C;
        const int64_t q0 = slice_ptr[s] / SELL_C;
        for (int k = 0; k < w; ++k) {
            int P = 0;
            for (int l = 0; l < SELL_C; ++l) {
                const int64_t e = sell_to_csr[slice_ptr[s] + (int64_t)k * SELL_C + l];
                if (e >= 0) P = std::max(P, cnt[e]);
            }
            gather_off[q0 + k] = (int32_t)total;
            gather_cnt[q0 + k] = P;
            for (int l = 0; l < SELL_C; ++l) {
                const int64_t e = sell_to_csr[slice_ptr[s] + (int64_t)k * SELL_C + l];
                if (e >= 0) pos[e] = total + l;
            }
            total += (int64_t)P * SELL_C;
        }
    }
    celem.assign(total, 0);
    cgidx.assign(total, 255);
    if (cab) cab->assign(total, 255);
    std::vector<int32_t> fill(nnz, 0);
    for (int64_t ep = 0; ep < E; ++ep)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                if (a == b) continue;
                const int32_t p = csr_slots[(int64_t)(a * 4 + b) * E + ep] & SLOT_MASK;
                const int64_t at = pos[p] + (int64_t)SELL_C * fill[p]++;
                celem[at] = (int32_t)ep;
                cgidx[at] = (uint8_t)local_gidx(a, b);
                if (cab) (*cab)[at] = (uint8_t)(4 * a + b);
            }
}

void build_incidence(int N, int E, const std::vector<int32_t>& nodes_soa, std::vector<int32_t>& inc_off,
                     std::vector<int32_t>& inc_cnt, std::vector<int32_t>& inc_elem) {
    std::vector<int32_t> cnt(N, 0);
    for (int64_t q = 0; q < 4LL * E; ++q) cnt[nodes_soa[q]]++;
    const int S = (N + SELL_C - 1) / SELL_C;
    inc_off.assign(S, 0);
    inc_cnt.assign(S, 0);
    int64_t total = 0;
    for (int s = 0; s < S; ++s) {
        int P = 0;
        for (int r = s * SELL_C; r < std::min(N, (s + 1) * SELL_C); ++r) P = std::max(P, cnt[r]);
        inc_off[s] = (int32_t)total;
        inc_cnt[s] = P;
        total += (int64_t)P * SELL_C;
    }
    inc_elem.assign(total, -1);
    std::vector<int32_t> fill(N, 0);
    for (int a = 0; a < 4; ++a)
        for (int64_t ep = 0; ep < E; ++ep) {
            const int r = nodes_soa[(int64_t)a * E + ep];
            const int s = r / SELL_C, l = r % SELL_C;
            inc_elem[inc_off[s] + (int64_t)SELL_C * fill[r]++ + l] = (int32_t)(4 * ep + a);
        }
}

}  // namespace rafem

namespace rafem {

int build_ilu(int N, const std::vector<int32_t>& rp, const std::vector<int32_t>& col, int order, IluHost& out) {
    // dependency levels in the given numbering: lev(i) = 1 + the largest level of an earlier neighbour
    std::vector<int32_t> lev(N, 0);
    int n_dep = 0, gap = 0;
    for (int i = 0; i < N; ++i) {
        int lv = 0;
        for (int32_t q = rp[i]; q < rp[i + 1]; ++q)
            if (col[q] < i) lv = std::max(lv, lev[col[q]] + 1);
        lev[i] = lv;
        n_dep = std::max(n_dep, lv + 1);
        for (int32_t q = rp[i]; q < rp[i + 1]; ++q)
            if (col[q] < i) gap = std::max(gap, lv - lev[col[q]]);
    }
    std::vector<int32_t> key;
    int n_levels = 0;
    if (order == 1) {
        key = lev;
        n_levels = n_dep;
    } else {
        // colours: neighbours are at most `gap` levels apart, so lev mod (gap + 1) is a proper colouring; the greedy
        // colouring (smallest colour unused by an earlier neighbour, nodes in index order) is taken when it needs
        // fewer colours
        std::vector<int32_t> greedy(N, 0), mark;
        int n_greedy = 0;
        for (int i = 0; i < N; ++i) {
            for (int32_t q = rp[i]; q < rp[i + 1]; ++q) {
                const int j = col[q];
                if (j < i) {
                    const int c = greedy[j];
                    if ((int)mark.size() <= c) mark.resize(c + 1, -1);
                    mark[c] = i;
                }
            }
            int c = 0;
            while (c < (int)mark.size() && mark[c] == i) ++c;
            greedy[i] = c;
            n_greedy = std::max(n_greedy, c + 1);
        }
        const int n_mod = std::min(gap + 1, n_dep);
        if (n_mod <= n_greedy) {
            key.resize(N);
            for (int i = 0; i < N; ++i) key[i] = lev[i] % n_mod;
            n_levels = n_mod;
        } else {
            key = std::move(greedy);
            n_levels = n_greedy;
        }
    }
    for (int i = 0; i < N; ++i)
        if (rp[i + 1] - rp[i] > 255) return -1;
    // padded level-contiguous numbering: level l occupies [lvl[l], lvl[l+1]), a multiple of 32 rows
    std::vector<int64_t> cnt(n_levels, 0);
    for (int i = 0; i < N; ++i) cnt[key[i]]++;
    out.n_levels = n_levels;
    out.lvl.assign(n_levels + 1, 0);
    for (int l = 0; l < n_levels; ++l) {
        const int64_t next = out.lvl[l] + (cnt[l] + SELL_C - 1) / SELL_C * SELL_C;
        if (next > INT32_MAX / 2) return -1;
        out.lvl[l + 1] = (int32_t)next;
    }
    const int Np = out.lvl[n_levels];
    out.Np = Np;
    out.perm.assign(Np, -1);
    std::vector<int32_t> pos(N), fill(out.lvl.begin(), out.lvl.end() - 1);
    for (int i = 0; i < N; ++i) {
        const int r = fill[key[i]]++;
        out.perm[r] = i;
        pos[i] = r;
    }
    // rows of P A P^T with columns in the new numbering, sorted; SELL-32 over the padded rows
    out.rlen.assign(Np, 1);
    out.dk.assign(Np, 0);
    const int S = Np / SELL_C;
    out.sp.assign(S + 1, 0);
    for (int s = 0; s < S; ++s) {
        int w = 1;
        for (int r = s * SELL_C; r < (s + 1) * SELL_C; ++r)
            if (out.perm[r] >= 0) w = std::max(w, rp[out.perm[r] + 1] - rp[out.perm[r]]);
        out.sp[s + 1] = out.sp[s] + w * SELL_C;
    }
    out.sc.assign(out.sp[S], 0);
    out.pmap.assign(out.sp[S], -1);
#pragma omp parallel for schedule(static)
    for (int s = 0; s < S; ++s) {
        const int w = (out.sp[s + 1] - out.sp[s]) / SELL_C;
        std::vector<std::pair<int32_t, int32_t>> row;
        for (int l = 0; l < SELL_C; ++l) {
            const int r = s * SELL_C + l;
            const int old = out.perm[r];
            row.clear();
            if (old >= 0) {
                for (int32_t q = rp[old]; q < rp[old + 1]; ++q) row.emplace_back(pos[col[q]], q);
                std::sort(row.begin(), row.end());
            } else {
                row.emplace_back(r, -2);  // dummy row: unit diagonal
            }
            out.rlen[r] = (uint8_t)row.size();
            for (int k = 0; k < w; ++k) {
                const int64_t at = out.sp[s] + (int64_t)k * SELL_C + l;
                if (k < (int)row.size()) {
                    out.sc[at] = row[k].first;
                    out.pmap[at] = row[k].second;
                    if (row[k].first == r) out.dk[r] = (uint8_t)k;
                } else {
                    out.sc[at] = r;
                    out.pmap[at] = -1;
                }
            }
        }
    }
    return 0;
}

namespace {
// SELL-32 layout of one row set of the padded ILU numbering (CSR rp/col over Np rows, sorted columns, src = the
// combined-layout position of each entry): shared slice patterns where possible, else per-entry columns.
void ilu_part_layout(int Np, const std::vector<int32_t>& rp, const std::vector<int32_t>& col,
                     const std::vector<int32_t>& src, IluPart& out) {
    std::vector<int32_t> map;
    out.patterns = build_sell_patterns(Np, rp, col, out.sp, out.sc, map, out.pat_off, out.pat_pool);
    if (!out.patterns) {
        out.pat_off.clear();
        out.pat_pool.clear();
        build_sell(Np, rp, col, out.sp, out.sc, map);
    }
    out.src.assign(out.sc.size(), -1);
    for (size_t q = 0; q < col.size(); ++q) out.src[map[q]] = src[q];
}
}  // namespace

void build_ilu_ring(const IluHost& ih, IluRingHost& out) {
    const int Np = ih.Np, S = Np / SELL_C;
    // rows of P A P^T in the padded numbering: full, strictly lower, strictly upper (sorted columns)
    std::vector<int32_t> rpA(Np + 1, 0), rpL(Np + 1, 0), rpU(Np + 1, 0);
    for (int r = 0; r < Np; ++r) {
        rpA[r + 1] = rpA[r] + ih.rlen[r];
        rpL[r + 1] = rpL[r] + ih.dk[r];
        rpU[r + 1] = rpU[r] + ih.rlen[r] - ih.dk[r] - 1;
    }
    std::vector<int32_t> cA(rpA[Np]), sA(rpA[Np]), cL(rpL[Np]), sL(rpL[Np]), cU(rpU[Np]), sU(rpU[Np]);
#pragma omp parallel for schedule(static)
    for (int sl = 0; sl < S; ++sl)
        for (int l = 0; l < SELL_C; ++l) {
            const int r = sl * SELL_C + l;
            int a = rpA[r], lo = rpL[r], up = rpU[r];
            for (int k = 0; k < ih.rlen[r]; ++k) {
                const int32_t at = ih.sp[sl] + k * SELL_C + l;
                cA[a] = ih.sc[at];
                sA[a++] = at;
                if (k < ih.dk[r]) {
                    cL[lo] = ih.sc[at];
                    sL[lo++] = at;
                } else if (k > ih.dk[r]) {
                    cU[up] = ih.sc[at];
                    sU[up++] = at;
                }
            }
        }
    ilu_part_layout(Np, rpA, cA, sA, out.A);
    ilu_part_layout(Np, rpL, cL, sL, out.L);
    ilu_part_layout(Np, rpU, cU, sU, out.U);
}

}  // namespace rafem

namespace rafem {

int reorder_rcm(int N, int E, const int32_t* tets, std::vector<int32_t>& perm) {
    std::vector<int32_t> rp, col;
    build_pattern(N, E, tets, rp, col);
    std::vector<int32_t> deg(N);
    for (int i = 0; i < N; ++i) deg[i] = rp[i + 1] - rp[i] - 1;  // the pattern stores the diagonal
    std::vector<char> seen(N, 0);
    std::vector<int32_t> order;
    order.reserve(N);
    std::vector<int32_t> level(N, -1), nb;
    // breadth-first level structure from s over the unvisited component; returns (eccentricity, last level)
    auto bfs_levels = [&](int s, std::vector<int32_t>& last) {
        std::vector<int32_t> cur{s}, next, touched{s};
        level[s] = 0;
        int ecc = 0;
        while (true) {
            next.clear();
            for (int u : cur)
                for (int32_t q = rp[u]; q < rp[u + 1]; ++q) {
                    const int v = col[q];
                    if (v == u || seen[v] || level[v] >= 0) continue;
                    level[v] = ecc + 1;
                    next.push_back(v);
                    touched.push_back(v);
                }
            if (next.empty()) break;
            ++ecc;
            cur.swap(next);
        }
        last = cur;
        for (int v : touched) level[v] = -1;
        return ecc;
    };
    for (int first = 0; first < N; ++first) {
        if (seen[first]) continue;
        // start: the smallest-degree unvisited node of this component (lowest index on ties) ...
        int s = first;
        {
            // collect the component by a plain traversal (level[] marks members, cleared afterwards)
            std::vector<int32_t> comp{first};
            level[first] = 0;
            for (size_t h = 0; h < comp.size(); ++h) {
                const int u = comp[h];
                for (int32_t q = rp[u]; q < rp[u + 1]; ++q) {
                    const int v = col[q];
                    if (v == u || seen[v] || level[v] >= 0) continue;
                    level[v] = 0;
                    comp.push_back(v);
                }
            }
            for (int v : comp) {
                level[v] = -1;
                if (deg[v] < deg[s] || (deg[v] == deg[s] && v < s)) s = v;
            }
        }
        // ... moved to a pseudo-peripheral node: the smallest-degree node of the last level while that increases
        // the eccentricity
        std::vector<int32_t> last;
        int ecc = bfs_levels(s, last);
        while (true) {
            int c = last[0];
            for (int v : last)
                if (deg[v] < deg[c] || (deg[v] == deg[c] && v < c)) c = v;
            std::vector<int32_t> last2;
            const int e2 = bfs_levels(c, last2);
            if (e2 <= ecc) break;
            s = c;
            ecc = e2;
            last.swap(last2);
        }
        // Cuthill-McKee: breadth first from s, unvisited neighbours in increasing (degree, index)
        const size_t h0 = order.size();
        order.push_back(s);
        seen[s] = 1;
        for (size_t h = h0; h < order.size(); ++h) {
            const int u = order[h];
            nb.clear();
            for (int32_t q = rp[u]; q < rp[u + 1]; ++q) {
                const int v = col[q];
                if (!seen[v]) nb.push_back(v);
            }
            std::sort(nb.begin(), nb.end(), [&](int a, int b) { return deg[a] != deg[b] ? deg[a] < deg[b] : a < b; });
            for (int v : nb) {
                seen[v] = 1;
                order.push_back(v);
            }
        }
    }
    perm.assign(order.rbegin(), order.rend());
    return 0;
}

}  // namespace rafem
