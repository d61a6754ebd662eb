// Internal data structures shared by the host analysis, the device factorization and the
// device sweep of the PEERS library.  Not part of the C ABI.
#pragma once

#include <cstdint>
#include <memory>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "peers.h"

#ifdef __CUDACC__
#define PEERS_HD __host__ __device__
#else
#define PEERS_HD
#endif

namespace peers {

// Width of a column block: the factorization's panel blocks, the sweep's diagonal-block
// inverses and the sweep's update steps all use it, so every query's arithmetic is blocked
// identically whatever tile it lands in.
constexpr int kBlock = 32;
// Rows x columns of one trailing-update tile of the factorization (halved for launches that
// would have fewer than kTrailFewTiles tiles).
constexpr int kTile = 64;
constexpr int64_t kTrailFewTiles = 148 * 4;
// Supernodes of one column block whose front has at most this many rows are factored whole
// by one CTA in shared memory (assembly, children's update matrices, L D L^T, write-back).
constexpr int kFactorFuseN = 96;
// CUDA streams over which independent subtrees are spread (factorization, selected inversion).
constexpr int kLanes = 4;

// One group of the factorization: the supernodes of one level in one lane (lane -1: the part
// above the lanes' subtrees, on the context's stream).  fuse_sn[fuse_b, fuse_e) are factored
// whole, fac_sn[fac_b, fac_e) (widest first) by the blocked kernels over nblocks column
// blocks, with trailing-update tiles trail_*[trail_base + J] and extend-add ranks
// ea_off[ea_b .. ea_e].
struct FactorGroup {
  int32_t lane, level;
  int32_t fuse_b, fuse_e, fac_b, fac_e;
  int32_t nblocks;
  int64_t trail_base;
  int64_t ea_b, ea_e;
  bool split;   // each block's update is split (see Symbolic::split_off) over three streams
};
// Largest number of queries one sweep tile (one CTA) carries.
constexpr int kQMax = 32;
// Shared-memory budget of one sweep CTA for its query fronts (bytes).
constexpr int64_t kSweepSmemBudget = 200 * 1024;

// Largest dynamic shared memory of one CTA on sm_103a (bytes).
constexpr int64_t kMaxSmem = 232448;
// CTAs of a sweep launch over fronts kept in global memory (supernodes whose front does not
// fit one CTA's shared memory): a persistent grid, each CTA with its own front scratch.
constexpr int kSpillGrid = 296;

// Row stride (in queries) of a sweep CTA's shared front: a multiple of 4, at least 4.
PEERS_HD inline int64_t sweep_qstride(int64_t Q) { return Q < 4 ? 4 : (Q + 3) / 4 * 4; }
// Dynamic shared memory of a sweep CTA for a front of N rows and Q queries: the front
// itself plus the block's y values and y^2/d terms.
PEERS_HD inline int64_t sweep_smem_bytes(int64_t N, int64_t Q) {
  return (N + 2 * kBlock) * sweep_qstride(Q) * 8;
}

// Front-size classes of the sweep's tile policy: rows N of a supernode's front in
// [0,128), [128,512), [512,2048), [2048,inf).
constexpr int kSizeClasses = 4;
inline int size_class(int64_t N) { return N < 128 ? 0 : N < 512 ? 1 : N < 2048 ? 2 : 3; }

// One unit of sweep work at supernode s.
//   kind 0 (range): the query slots [q0, q0+nq) of the sorted order.  src >= 0: they arrive
//     from child supernode src (their carries are scattered through src's relative map);
//     src == -1: they start at s (seeded with +1 at qa, -1 at qb).
//   kind 1 (list): nq entries ldesc[q0 .. q0+nq) of the two-branch walk (see SweepDesc).
//   kind 2 (combine): finish the two-branch queries [q0, q0+nq) of a wave (multi-graph
//     launches only; single-graph sweeps use a separate combine launch).
// g selects the graph/wave argument block in multi-graph launches (0 otherwise).
struct SweepItem {
  int32_t s;
  int32_t src;
  int32_t q0;
  int32_t nq;
  int32_t j0;   // first column block (block-aligned) with a non-zero right-hand side
  int32_t kind;
  int32_t g;
  int32_t spill;   // 1: the tile's fronts live in the CTA's global scratch, not shared memory
};

// One query step of the two-branch walk (a listed pair whose endpoints' etree paths meet
// only above the lower endpoint's supernode).  The front of slot `a` comes from child `src_a`
// (or its seed when src_a == -1); when `b` >= 0 the carry of slot b from child src_b is added
// (the two branches merge here); when b == -1 and seed_b >= 0, -1 is added at local row
// seed_b (the upper endpoint's column lies in this supernode).  The result goes to slot a.
struct SweepDesc {
  int32_t a, src_a, b, src_b, seed_b;
};

// One wave of the sweep: the queries [q_begin, q_end) of the sorted order, walked to the
// root level by level.  items[level_ptr[l] .. level_ptr[l+1]) are the level's items.
// Allocator whose value-initialising construct() default-initialises instead: a vector of
// trivially constructible elements that is sized and then filled is not zeroed first.
template <class T>
struct NoInitAlloc : std::allocator<T> {
  template <class U>
  struct rebind { using other = NoInitAlloc<U>; };
  NoInitAlloc() = default;
  template <class U>
  NoInitAlloc(const NoInitAlloc<U> &) noexcept {}
  template <class U>
  void construct(U *p) noexcept { ::new (static_cast<void *>(p)) U; }
  template <class U, class... Args>
  void construct(U *p, Args &&...args) {
    ::new (static_cast<void *>(p)) U(std::forward<Args>(args)...);
  }
};

struct SweepWave {
  int64_t q_begin, q_end;
  int64_t two_begin = 0, two_end = 0;   // two-branch queries finished by this wave (combine)
  std::vector<int64_t> level_ptr;
  std::vector<int64_t> level_smem;   // dynamic shared memory of the level's launch
  // the first level_nspill[l] items of level l have spill == 1 and run in their own launch
  // (dynamic shared memory level_spill_smem[l])
  std::vector<int64_t> level_nspill, level_spill_smem;
  std::vector<SweepItem, NoInitAlloc<SweepItem>> items;   // filled level by level once sized
};

struct Symbolic {
  // ---- graph ----
  int64_t n = 0;        // graph nodes
  int64_t nr = 0;       // reduced nodes (n - 1)
  int32_t ground = 0;
  int64_t nnz_csr = 0;  // stored CSR entries of the input graph
  // reduced node r <-> graph node: graph = r + (r >= ground)
  std::vector<int32_t> perm;   // elimination position k -> reduced node
  std::vector<int32_t> iperm;  // reduced node -> elimination position

  // ---- supernodes (postorder; columns of supernode s are [first[s], first[s+1])) ----
  int32_t nsuper = 0;
  std::vector<int32_t> first;       // nsuper + 1
  std::vector<int32_t> parent;      // nsuper
  std::vector<int32_t> nb;          // below-diagonal row count
  std::vector<int32_t> level;       // height above the leaves
  std::vector<int32_t> fdesc;       // first (lowest-numbered) supernode of the subtree
  std::vector<int32_t> child_ptr, child_list;   // children in increasing order
  std::vector<int64_t> rows_off;    // nsuper + 1: B_s = rows[rows_off[s] .. rows_off[s+1])
  // row indices (elimination positions) of each B_s, ascending
  std::vector<int32_t, NoInitAlloc<int32_t>> rows;
  std::vector<int32_t, NoInitAlloc<int32_t>> rmap;   // parallel to rows: local row in the parent
  std::vector<int32_t> col2sn;      // column -> supernode
  int32_t nlevels = 0;
  std::vector<int32_t> level_ptr;   // nlevels + 1
  std::vector<int32_t> level_sn;    // supernodes by level, each level sorted by n_c descending

  // ---- device layout of the factor ----
  std::vector<int64_t> panel_off;   // panel of s: (n_c+n_b) x n_c column-major, ld = n_c+n_b
  int64_t panel_total = 0;
  std::vector<int64_t> tinv_off;    // diagonal-block inverses of s: block J at +kBlock^2 * J
  int64_t tinv_total = 0;
  std::vector<int64_t> u_off;       // update matrix of s: n_b x n_b column-major
  int64_t u_total = 0;
  // assembly of L_r into the panels: entry e goes to panel[a_dest[e]].  Entries are the
  // strictly-lower entries followed by the nr diagonal entries.  a_src[e] is the CSR index
  // of the conductance of an off-diagonal entry.
  std::vector<int64_t, NoInitAlloc<int64_t>> a_dest;
  std::vector<int64_t, NoInitAlloc<int64_t>> a_src;
  int64_t nnz_lower = 0;
  // diagonal of the reduced node r = sum of the conductances of CSR row g(r)
  std::vector<int64_t, NoInitAlloc<int64_t>> csr_indptr;  // copy of the input indptr (degrees)
  std::vector<double, NoInitAlloc<double>> w0;           // conductances given to analyze
  // lanes (see kLanes): per supernode its depth below its root and its lane (-1: top part)
  std::vector<int32_t> depth, lane_of;
  int32_t nlanes = 0;
  bool one_stream = false;   // peers_options.one_stream: no lanes, no split column blocks
  // factorization schedule: groups in issue order, over the supernode lists fuse_sn (factored
  // whole in one CTA, see kFactorFuseN) and fac_sn (blocked kernels)
  std::vector<FactorGroup> fgroups;
  std::vector<int32_t> fuse_sn, fac_sn;
  // trailing-update tiles: for (group g, block J) the active supernodes are the first
  // na = trail_na[tp] of the group's blocked supernodes; trail_prefix[trail_off[tp] + i] is the
  // tile prefix of the i-th active supernode (na + 1 entries).  tp = fgroups[g].trail_base + J.
  std::vector<int64_t> trail_off, trail_na;
  std::vector<int32_t> trail_ts;    // tile size of each (group, block): kTile or kTile / 2
  std::vector<int64_t> trail_prefix;
  // split of (group, block J) for groups of more than one column block (split_off[tp] < 0:
  // not split), three parts of the block's update that together are its whole trailing
  // update: "next", block J + 1's columns (one column of kTile / 2 tiles per supernode, next_na
  // supernodes); "panel rest", the panel's columns after block J + 1 (tiles of pr_ts); and "U",
  // the update matrix (triangle of tiles of up_ts).  Their tile prefixes over the block's na
  // active supernodes (next_na for "next") start at trail_prefix[split_off[tp]], then
  // + next_na + 1, then + next_na + na + 2.
  std::vector<int64_t> split_off, next_na;
  std::vector<int32_t> pr_ts, up_ts;
  // extend-add schedule: for group g and child rank r (ea_b <= r < ea_e), pairs
  // (parent, child) in ea_pairs[2 ea_off[r] .. 2 ea_off[r + 1])
  std::vector<int64_t> ea_off;
  std::vector<int32_t> ea_pairs;    // (parent, child) interleaved
  int64_t factor_fma = 0;

  // ---- queries ----
  int64_t nq = 0;                   // as given
  int64_t nq_trivial = 0;
  int64_t nq_two = 0;
  int64_t nsorted = 0;              // non-trivial queries, sorted by (start supernode, lo)
  std::vector<int64_t, NoInitAlloc<int64_t>> qorig;   // sorted slot -> user query index
  // local seed rows (+1 at qa, -1 at qb; qb = -1: none)
  std::vector<int32_t, NoInitAlloc<int32_t>> qa, qb;
  std::vector<int64_t> qbeg;        // nsuper + 1: first slot whose start supernode is >= s
  std::vector<int32_t> qtile;       // tile size (queries per CTA) per supernode
  int32_t qcap[kSizeClasses] = {kQMax, kQMax, kQMax, kQMax};   // tile caps in use
  int64_t carry_budget = 0;         // bytes of carried fronts per wave
  // shared memory of a sweep CTA: the tile is sized for front_budget bytes of fronts, and a
  // supernode whose smallest tile still needs more than front_limit bytes keeps its fronts in
  // global memory (spill[s] = 1, kSpillGrid CTAs x spill_stride doubles of scratch)
  int64_t front_budget = kSweepSmemBudget, front_limit = kMaxSmem;
  std::vector<char> spill;
  int64_t spill_stride = 0;
  std::vector<int32_t> two_lo, two_hi;   // two-branch queries (elimination positions)
  std::vector<int64_t> two_idx;          // and their user indices
  int32_t nbmax = 0;
  std::vector<SweepWave> waves;
  // two-branch walk: step descriptors, and per such query (user index, slot a, slot b of a
  // branch that ends in another etree root or -1) for the final combine
  std::vector<SweepDesc> ldesc;
  std::vector<int64_t> two_user;
  std::vector<int32_t> two_a, two_b;
  int64_t carry_slots = 0;          // slots of the carry buffer (largest wave)
  int64_t walk_entries = 0, walk_fma = 0;
  int64_t front_bytes = 0;   // query-front bytes one sweep reads and writes between levels
  double t_order = 0, t_symbolic = 0, t_queries = 0;
};

// Host analysis (analyze.cpp).  Returns a PEERS_* status and fills `err`.
int analyze(Symbolic &S, int64_t n, const int64_t *indptr, const int32_t *indices,
            const double *w, int32_t ground, int64_t nq, const int32_t *qu, const int32_t *qv,
            const double *coords, int dim, const peers_options &opt, std::string &err);

// Queries per sweep CTA for a front of N rows under the plan's shared-memory budget and the
// size class's cap (analyze.cpp).
int32_t sweep_tile(const Symbolic &S, int64_t N, int32_t cap);

// (Re)builds the sweep's tiles and waves of an analysed plan (analyze.cpp).
int build_sweep_plan(Symbolic &S, const int32_t *qcap, std::string &err);
// Caps the host threads of the analyses the calling thread runs (0: no cap).
void set_host_thread_cap(int cap);

// Conductance-dependent assembly values (off-diagonals -w, then diagonals = degrees) in the
// order of a_dest, for conductances w (CSR layout of the analysed graph).
void assembly_values(const Symbolic &S, const double *w, std::vector<double> &vals);

inline int32_t sn_nc(const Symbolic &S, int32_t s) { return S.first[s + 1] - S.first[s]; }

}  // namespace peers
