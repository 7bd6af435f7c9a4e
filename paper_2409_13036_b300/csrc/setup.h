// Host-side setup of the fixed sparse structure (see setup.cpp).
#pragma once
#include <cstdint>
#include <vector>

namespace rafem {

// Slot-code flags stored in the element -> CSR slot map (slot index in the low 29 bits).
constexpr int32_t SLOT_FIRST = 1 << 30;   // this element is the first writer of the slot: store, do not add
constexpr int32_t SLOT_LAST = 1 << 29;    // this element is the last writer of the slot: emit the FP32 copy
constexpr int32_t SLOT_MASK = (1 << 29) - 1;

// 0 ok, -1 bad index / repeated node, -2 degenerate element. orient[e] = sign of the element's volume.
int validate_mesh(int N, int E, const int32_t* tets, const double* xyz, std::vector<int8_t>& orient,
                  double* vol_min = nullptr, double* vol_max = nullptr);

// CSR pattern of the node graph: row i lists every node sharing an element with i (itself included), sorted.
void build_pattern(int N, int E, const int32_t* tets, std::vector<int32_t>& row_ptr, std::vector<int32_t>& col);

// Greedy element colouring (no two elements of a colour share a node). Returns the colour count or -1.
int color_elements(int N, int E, const int32_t* tets, std::vector<int32_t>& color);

// Element -> slot map over the element order `order` (SoA [16][E]), with first/last-writer flags.
void build_slots(int E, const int32_t* tets, const std::vector<int32_t>& row_ptr, const std::vector<int32_t>& col,
                 const std::vector<int64_t>& order, std::vector<int32_t>& slots);

// SELL-C layout (C = 32, no sorting) of a CSR pattern: slice s holds rows [32s, 32s+32), padded to the longest
// row of the slice and stored column-major (entry k of lane l at slice_ptr[s] + 32k + l). Padding entries get
// column min(row, N-1) and are never written. csr_to_sell maps each CSR position to its SELL position.
constexpr int SELL_C = 32;
void build_sell(int N, const std::vector<int32_t>& row_ptr, const std::vector<int32_t>& col,
                std::vector<int32_t>& slice_ptr, std::vector<int32_t>& sell_col, std::vector<int32_t>& csr_to_sell);

// SELL-C layout whose slices share one column pattern per slice: the entries of slice s sit at the slots of the
// sorted union of the column offsets (col - row) of its rows, slot k of every row holding offset pat[k] (rows
// without that neighbour store a padding entry there, column min(row, N-1), never written). Used only when the
// patterns add at most 2% to the stored entries of build_sell's layout (lattice numberings: a few slices that mix
// the ends of two lattice lines widen, under 0.4% on the cube meshes; none when the lines hold a multiple of 32
// nodes). The patterns are stored once each in pat_pool; pat_off[s] is slice s's first offset there. Returns false
// (outputs unspecified) otherwise.
bool build_sell_patterns(int N, const std::vector<int32_t>& row_ptr, const std::vector<int32_t>& col,
                         std::vector<int32_t>& slice_ptr, std::vector<int32_t>& sell_col,
                         std::vector<int32_t>& csr_to_sell, std::vector<int32_t>& pat_off,
                         std::vector<int32_t>& pat_pool);

// Row-owner ("gather") assembly of the pure stiffness matrix sigma(T)-weighted sum_e sigma0_e G_e on the SELL-32
// layout (either SELL builder; csr_to_sell maps CSR positions to SELL positions). For every off-diagonal SELL entry
// the elements sharing that edge are listed with the index of
// G_e[a][b]; entries of one (slice, column) group are stored column-major with the group padded to the longest
// list among its 32 rows: contribution m of lane l of group q lives at gather_off[q] + 32 m + l, and the group has
// gather_cnt[q] contributions (0 for groups holding only diagonal or padding entries). Padding contributions
// carry gidx = 255. csr_slots are the element->CSR slot codes (flags allowed) over the sorted element order.
// With cab non-null it also receives, per contribution, the local vertices of the row (a) and of the column (b) as
// 4 a + b (255 for padding), which the coupled Jacobian needs because its blocks are not symmetric in (a, b).
void build_gather(int N, int E, const std::vector<int32_t>& row_ptr, const std::vector<int32_t>& col,
                  const std::vector<int32_t>& csr_slots, const std::vector<int32_t>& slice_ptr,
                  const std::vector<int32_t>& csr_to_sell, std::vector<int32_t>& gather_off,
                  std::vector<int32_t>& gather_cnt, std::vector<int32_t>& celem, std::vector<uint8_t>& cgidx,
                  std::vector<uint8_t>* cab = nullptr);

// Node -> element incidence (sorted element order) in the SELL-32 slice layout: entry m of row 32 s + l at
// inc_off[s] + 32 m + l for m < inc_cnt[s] holds 4 e + a (element e, local vertex a); -1 marks padding.
// Requires 4 E < 2^31.
void build_incidence(int N, int E, const std::vector<int32_t>& nodes_soa, std::vector<int32_t>& inc_off,
                     std::vector<int32_t>& inc_cnt, std::vector<int32_t>& inc_elem);

// ILU(0) layout: a symmetric permutation P in which the rows of one level never depend on each other, levels
// stored contiguously and each padded to a multiple of 32 rows (dummy rows carry a unit diagonal), and P A P^T in
// SELL-32 with 32-bit columns (new numbering). With the dependency levels lev(i) = 1 + max lev(j) over earlier
// neighbours j and g the largest level gap along an edge: order 1 uses the levels themselves; order 0 uses the
// colouring lev mod (g + 1) (neighbours are 1..g levels apart, so it is proper; 4 colours on the Kuhn lattice),
// or the greedy colouring (smallest colour unused by an earlier neighbour, nodes in index order) when that needs
// fewer colours. Within a level rows keep their original order.
struct IluHost {
    int Np = 0, n_levels = 0;
    std::vector<int32_t> lvl;    // [n_levels + 1] first padded row of each level
    std::vector<int32_t> perm;   // [Np] original row of each padded row, -1 for a dummy row
    std::vector<int32_t> sp;     // [Np/32 + 1] slice pointers
    std::vector<int32_t> sc;     // columns (new numbering); padding entries point at their own row
    std::vector<int32_t> pmap;   // source CSR position of each entry; -1 padding (0), -2 dummy diagonal (1)
    std::vector<uint8_t> rlen;   // entries per row
    std::vector<uint8_t> dk;     // index of the diagonal within the row
};
// Returns 0, or -1 when a row has more than 255 entries or the padded size overflows.
int build_ilu(int N, const std::vector<int32_t>& rp, const std::vector<int32_t>& col, int order, IluHost& out);

// Layouts of the ILU(0) solver that streams its matrices through the shared-memory ring: P A P^T, the strictly
// lower factor L and the strictly upper part of U, each a SELL-32 layout over the padded numbering of IluHost (one
// column pattern per slice where that widens no slice, else per-entry columns). src maps every position to its
// position in IluHost's combined layout (where the system and its factors are stored), -1 for padding.
struct IluPart {
    bool patterns = false;
    std::vector<int32_t> sp, sc, pat_off, pat_pool, src;
};
struct IluRingHost {
    IluPart A, L, U;
};
void build_ilu_ring(const IluHost& ih, IluRingHost& out);

// Reverse Cuthill-McKee order of the node graph: perm[new] = old. Per connected component (taken in order of its
// lowest node): start at the component's smallest-degree node (lowest index on ties), move to the smallest-degree
// node of the last breadth-first level while that increases the eccentricity, then number breadth first with the
// unvisited neighbours of each node in increasing (degree, index); the whole order is reversed at the end.
int reorder_rcm(int N, int E, const int32_t* tets, std::vector<int32_t>& perm);

}  // namespace rafem
