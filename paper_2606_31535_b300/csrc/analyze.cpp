// Host analysis of the PEERS library: validation, grounding, fill-reducing ordering,
// elimination tree, supernodes, factorization schedule and query grouping.
//
// Paper correspondence (PEERS, arXiv 2606.31535):
//   - grounding and the reduced Laplacian: §II-A (eq. 1, and the text after it), §IV-A;
//   - fill-reducing ordering (the paper uses AMD in Alg. 8 step 1 and nested dissection in
//     its analysis, Def. 1-2, Lemma 2): nested dissection here, by coordinates or by BFS
//     level structures;
//   - elimination tree (Lemma 1: y = L^{-1} b is non-zero only on etree paths);
//   - query graph (§III-G): each query is mapped to its permuted endpoints and grouped by the
//     supernode where its etree path starts.
// Everything here is integer work on the CPU; no device is touched.  The large steps run on
// up to kPlanThreads host threads, and no result depends on how many.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <condition_variable>
#include <cstdlib>
#include <exception>
#include <mutex>
#include <new>
#include <numeric>
#include <system_error>
#include <thread>

#include "internal.h"

namespace peers {
namespace {

using Clock = std::chrono::steady_clock;
double since(Clock::time_point t0) {
  return std::chrono::duration<double>(Clock::now() - t0).count();
}

// Host threads for the large analysis steps: the hardware's count, at most kPlanThreads, at
// most PEERS_ANALYSIS_THREADS when that is set to a positive number, and at most the calling
// thread's cap (set_host_thread_cap).  No result depends on the count.
constexpr int kPlanThreads = 8;
thread_local int t_thread_cap = 0;
int plan_threads() {
  unsigned t = std::min<unsigned>(std::thread::hardware_concurrency(), kPlanThreads);
  if (const char *e = std::getenv("PEERS_ANALYSIS_THREADS")) {
    const long v = std::strtol(e, nullptr, 10);
    if (v > 0) t = std::min<unsigned>(t, static_cast<unsigned>(v));
  }
  if (t_thread_cap > 0) t = std::min<unsigned>(t, static_cast<unsigned>(t_thread_cap));
  return static_cast<int>(std::max(1u, t));
}

// Runs f(0) .. f(nthreads - 1), each on a host thread of its own (inline for one).  If the
// system starts no more threads, the calling thread runs the remaining calls itself.  An
// exception thrown by a call (a failed allocation) is rethrown here after every thread has
// been joined.
template <class F>
void run_threads(int nthreads, F &&f) {
  if (nthreads <= 1) {
    f(0);
    return;
  }
  std::vector<std::exception_ptr> errs(static_cast<size_t>(nthreads));
  auto call = [&f, &errs](int t) {
    try {
      f(t);
    } catch (...) {
      errs[t] = std::current_exception();
    }
  };
  std::vector<std::thread> pool;
  pool.reserve(static_cast<size_t>(nthreads));
  int started = 0;
  for (; started < nthreads; ++started) {
    try {
      pool.emplace_back(call, started);
    } catch (const std::system_error &) {
      break;
    }
  }
  for (int t = started; t < nthreads; ++t) call(t);
  for (std::thread &th : pool) th.join();
  for (const std::exception_ptr &e : errs)
    if (e) std::rethrow_exception(e);
}

// Runs f(lo, hi) over contiguous chunks of [0, count): one chunk per host thread when count
// is large, else one chunk.
template <class F>
void chunked(int64_t count, F &&f) {
  const int nt = count >= (int64_t(1) << 18) ? plan_threads() : 1;
  run_threads(nt, [&](int c) { f(count * c / nt, count * (c + 1) / nt); });
}

// ------------------------------------------------------------------------- validation

int validate(int64_t n, const int64_t *indptr, const int32_t *indices, const double *w,
             int32_t ground, std::string &err) {
  if (n < 2) { err = "a graph needs at least two nodes"; return PEERS_EINVAL; }
  if (n > INT32_MAX - 1) { err = "more than 2^31-2 nodes"; return PEERS_EINVAL; }
  if (!indptr || !indices || !w) { err = "null graph array"; return PEERS_EINVAL; }
  if (ground < 0 || ground >= n) { err = "ground node out of range"; return PEERS_EINVAL; }
  if (indptr[0] != 0) { err = "indptr[0] must be 0"; return PEERS_EINVAL; }
  for (int64_t i = 0; i < n; ++i)
    if (indptr[i + 1] < indptr[i]) { err = "indptr is not non-decreasing"; return PEERS_EINVAL; }
  const int64_t nnz = indptr[n];
  // The row checks run over contiguous row chunks, one per host thread, in three passes (entry
  // values; duplicates; symmetry).  Each chunk keeps its first failure, and the first chunk
  // that failed reports: the error a pass over the rows in order meets first.
  const int nchunks = nnz >= (int64_t(1) << 20) ? plan_threads() : 1;
  std::vector<std::string> errs(static_cast<size_t>(nchunks));
  std::vector<int> codes(static_cast<size_t>(nchunks), PEERS_OK);
  auto pass = [&](auto &&check_row) -> int {
    run_threads(nchunks, [&](int c) {
      const int64_t r0 = n * c / nchunks, r1 = n * (c + 1) / nchunks;
      for (int64_t i = r0; i < r1; ++i)
        if (!check_row(i, errs[c])) { codes[c] = PEERS_EINVAL; return; }
    });
    for (int c = 0; c < nchunks; ++c)
      if (codes[c] != PEERS_OK) { err = errs[c]; return codes[c]; }
    return PEERS_OK;
  };
  int rc = pass([&](int64_t i, std::string &e) {
    for (int64_t p = indptr[i]; p < indptr[i + 1]; ++p) {
      int64_t j = indices[p];
      if (j < 0 || j >= n) { e = "column index out of range"; return false; }
      if (j == i) { e = "self-loop at node " + std::to_string(i); return false; }
      if (!(w[p] > 0.0) || !std::isfinite(w[p])) {
        e = "conductance must be positive and finite (entry " + std::to_string(p) + ")";
        return false;
      }
    }
    return true;
  });
  if (rc != PEERS_OK) return rc;
  // per-row copies sorted by column, for the duplicate and symmetry checks
  struct Entry { int32_t j; double w; };
  std::vector<Entry, NoInitAlloc<Entry>> srt(static_cast<size_t>(nnz));
  rc = pass([&](int64_t i, std::string &e) {
    for (int64_t p = indptr[i]; p < indptr[i + 1]; ++p) srt[p] = Entry{indices[p], w[p]};
    std::sort(srt.begin() + indptr[i], srt.begin() + indptr[i + 1],
              [](const Entry &a, const Entry &b) { return a.j < b.j; });
    for (int64_t p = indptr[i] + 1; p < indptr[i + 1]; ++p)
      if (srt[p].j == srt[p - 1].j) {
        e = "duplicate edge in row " + std::to_string(i);
        return false;
      }
    return true;
  });
  if (rc != PEERS_OK) return rc;
  rc = pass([&](int64_t i, std::string &e) {
    for (int64_t p = indptr[i]; p < indptr[i + 1]; ++p) {
      const int32_t j = srt[p].j;
      auto b = srt.begin() + indptr[j], en = srt.begin() + indptr[j + 1];
      auto it = std::lower_bound(b, en, i, [](const Entry &a, int64_t c) { return a.j < c; });
      if (it == en || it->j != i) { e = "CSR is not symmetric"; return false; }
      if (it->w != srt[p].w) {
        e = "conductances of (u,v) and (v,u) differ";
        return false;
      }
    }
    return true;
  });
  if (rc != PEERS_OK) return rc;
  // connectivity is checked on the elimination tree, once the analysis has it
  return PEERS_OK;
}

// Adjacency of the reduced graph (ground removed, no diagonal), reduced numbering.
struct Adj {
  std::vector<int64_t> ptr;
  std::vector<int32_t, NoInitAlloc<int32_t>> idx;
};

Adj reduced_adjacency(int64_t n, const int64_t *indptr, const int32_t *indices, int32_t g) {
  Adj A;
  const int64_t nr = n - 1;
  A.ptr.assign(static_cast<size_t>(nr + 1), 0);
  chunked(n, [&](int64_t i0, int64_t i1) {
    for (int64_t i = i0; i < i1; ++i) {
      if (i == g) continue;
      int64_t c = 0;
      for (int64_t p = indptr[i]; p < indptr[i + 1]; ++p) c += indices[p] != g;
      A.ptr[(i > g ? i - 1 : i) + 1] = c;
    }
  });
  for (int64_t r = 0; r < nr; ++r) A.ptr[r + 1] += A.ptr[r];
  A.idx.resize(static_cast<size_t>(A.ptr[nr]));
  chunked(n, [&](int64_t i0, int64_t i1) {
    for (int64_t i = i0; i < i1; ++i) {
      if (i == g) continue;
      int64_t q = A.ptr[i > g ? i - 1 : i];
      for (int64_t p = indptr[i]; p < indptr[i + 1]; ++p) {
        int32_t j = indices[p];
        if (j != g) A.idx[q++] = j > g ? j - 1 : j;
      }
    }
  });
  return A;
}

// ------------------------------------------------------------------------- orderings
//
// Both nested-dissection variants order in place: the task [lo, hi) of `work` is rewritten
// as [part A | part B | separator] and A and B become new tasks; the separator stays last
// (it is eliminated after both halves, the structure behind Def. 1 / Lemma 2).

struct NdTask { int64_t lo, hi; };

// Coordinate bisection: split at the median of the widest axis; the separator is the set of
// upper-side nodes with a lower-side neighbour.  A task's split depends only on its own nodes,
// so tasks run on up to kPlanThreads host threads with the same result as one: each task
// stamps its nodes with its own id, and a neighbour counts as lower-side only under the id of
// the task looking at it.
void order_coordinate_nd(const Adj &A, const double *xy, int dim, int leaf,
                         std::vector<int32_t> &work) {
  const int64_t nr = static_cast<int64_t>(A.ptr.size()) - 1;
  work.resize(static_cast<size_t>(nr));
  std::iota(work.begin(), work.end(), 0);
  std::vector<int8_t> side(static_cast<size_t>(nr), -1);
  std::vector<std::atomic<int32_t>> owner(static_cast<size_t>(nr));
  for (auto &o : owner) o.store(0, std::memory_order_relaxed);
  std::atomic<int32_t> next_id{1};
  constexpr int64_t kNdInner = int64_t(1) << 20;
  struct Scratch {
    std::vector<std::pair<double, int32_t>> keys;
    std::vector<double> vals, mn, mx;
    std::vector<int64_t> cnt;
    std::vector<int32_t> tmp;
    std::vector<char> sep;
  };
  // splits a task of fewer than kNdInner nodes into [A | B | separator] on the calling thread;
  // returns the new tasks (A and B) in kids
  auto split_small = [&](NdTask t, Scratch &sc, NdTask kids[2]) -> int {
    const int64_t cnt = t.hi - t.lo;
    if (cnt <= leaf) return 0;
    int axis = -1;
    double width = 0.0;
    for (int a = 0; a < dim; ++a) {
      double mn = INFINITY, mx = -INFINITY;
      for (int64_t i = t.lo; i < t.hi; ++i) {
        double c = xy[static_cast<int64_t>(work[i]) * dim + a];
        mn = std::min(mn, c);
        mx = std::max(mx, c);
      }
      if (mx - mn > width) { width = mx - mn; axis = a; }
    }
    if (axis < 0) return 0;   // all nodes coincide: keep as one block
    const int32_t id = next_id.fetch_add(1, std::memory_order_relaxed);
    auto &keys = sc.keys;
    keys.resize(static_cast<size_t>(cnt));
    for (int64_t i = 0; i < cnt; ++i) {
      const int32_t v = work[t.lo + i];
      keys[i] = {xy[static_cast<int64_t>(v) * dim + axis], v};
      owner[v].store(id, std::memory_order_relaxed);
    }
    std::nth_element(keys.begin(), keys.begin() + cnt / 2, keys.end());
    const double pivot = keys[cnt / 2].first;
    int64_t nlow = 0;
    for (auto &k : keys) nlow += k.first < pivot;
    const bool strict = nlow > 0;
    for (auto &k : keys) side[k.second] = (strict ? k.first < pivot : k.first <= pivot) ? 0 : 1;
    int64_t na = 0, nbu = 0;
    for (int64_t i = t.lo; i < t.hi; ++i) {
      int32_t v = work[i];
      if (side[v] == 1) {
        for (int64_t p = A.ptr[v]; p < A.ptr[v + 1]; ++p) {
          const int32_t u = A.idx[p];
          if (owner[u].load(std::memory_order_relaxed) == id && side[u] == 0) {
            side[v] = 2;
            break;
          }
        }
      }
    }
    for (int64_t i = t.lo; i < t.hi; ++i) {
      int sd = side[work[i]];
      na += sd == 0;
      nbu += sd == 1;
    }
    if (na == 0 || nbu == 0) {   // no proper split
      for (int64_t i = t.lo; i < t.hi; ++i) side[work[i]] = -1;
      return 0;
    }
    sc.tmp.assign(work.begin() + t.lo, work.begin() + t.hi);
    int64_t a = t.lo, b = t.lo + na, c = t.lo + na + nbu;
    for (int32_t v : sc.tmp) {
      int sd = side[v];
      (sd == 0 ? work[a++] : sd == 1 ? work[b++] : work[c++]) = v;
      side[v] = -1;
    }
    kids[0] = {t.lo, t.lo + na};
    kids[1] = {t.lo + na, t.lo + na + nbu};
    return 2;
  };
  // the same split for a task of at least kNdInner nodes (the first levels, which run few at a
  // time), each of its passes spread over host threads: chunk results are combined in chunk
  // order, and the median is taken as the value of rank cnt / 2 of the coordinates alone
  const int wide_threads = plan_threads();   // read on the calling thread (its cap applies)
  auto split_wide = [&](NdTask t, Scratch &sc, NdTask kids[2]) -> int {
    const int64_t cnt = t.hi - t.lo;
    const int nt = wide_threads;
    // f(chunk, i0, i1) over contiguous chunks of the task's range
    auto pfor = [&](auto &&f) {
      run_threads(nt, [&](int c) { f(c, t.lo + cnt * c / nt, t.lo + cnt * (c + 1) / nt); });
    };
    auto coord = [&](int64_t i, int a) { return xy[static_cast<int64_t>(work[i]) * dim + a]; };
    sc.mn.assign(static_cast<size_t>(nt) * dim, INFINITY);
    sc.mx.assign(static_cast<size_t>(nt) * dim, -INFINITY);
    pfor([&](int c, int64_t i0, int64_t i1) {
      for (int a = 0; a < dim; ++a) {
        double mn = INFINITY, mx = -INFINITY;
        for (int64_t i = i0; i < i1; ++i) {
          const double x = coord(i, a);
          mn = std::min(mn, x);
          mx = std::max(mx, x);
        }
        sc.mn[c * dim + a] = mn;
        sc.mx[c * dim + a] = mx;
      }
    });
    int axis = -1;
    double width = 0.0;
    for (int a = 0; a < dim; ++a) {
      double mn = INFINITY, mx = -INFINITY;
      for (int c = 0; c < nt; ++c) {
        mn = std::min(mn, sc.mn[c * dim + a]);
        mx = std::max(mx, sc.mx[c * dim + a]);
      }
      if (mx - mn > width) { width = mx - mn; axis = a; }
    }
    if (axis < 0) return 0;   // all nodes coincide: keep as one block
    const int32_t id = next_id.fetch_add(1, std::memory_order_relaxed);
    // the median coordinate along the axis: the value of rank cnt / 2
    sc.vals.resize(static_cast<size_t>(cnt));
    pfor([&](int, int64_t i0, int64_t i1) {
      for (int64_t i = i0; i < i1; ++i) {
        sc.vals[i - t.lo] = coord(i, axis);
        owner[work[i]].store(id, std::memory_order_relaxed);
      }
    });
    std::nth_element(sc.vals.begin(), sc.vals.begin() + cnt / 2, sc.vals.end());
    const double pivot = sc.vals[cnt / 2];
    sc.cnt.assign(static_cast<size_t>(nt) * 3, 0);
    pfor([&](int c, int64_t i0, int64_t i1) {
      int64_t k = 0;
      for (int64_t i = i0; i < i1; ++i) k += coord(i, axis) < pivot;
      sc.cnt[c * 3] = k;
    });
    int64_t nlow = 0;
    for (int c = 0; c < nt; ++c) nlow += sc.cnt[c * 3];
    const bool strict = nlow > 0;
    pfor([&](int, int64_t i0, int64_t i1) {
      for (int64_t i = i0; i < i1; ++i) {
        const double x = coord(i, axis);
        side[work[i]] = (strict ? x < pivot : x <= pivot) ? 0 : 1;
      }
    });
    // separator: upper-side nodes with a lower-side neighbour in this task
    sc.sep.resize(static_cast<size_t>(cnt));
    pfor([&](int, int64_t i0, int64_t i1) {
      for (int64_t i = i0; i < i1; ++i) {
        const int32_t v = work[i];
        char f = 0;
        if (side[v] == 1) {
          for (int64_t p = A.ptr[v]; p < A.ptr[v + 1]; ++p) {
            const int32_t u = A.idx[p];
            if (owner[u].load(std::memory_order_relaxed) == id && side[u] == 0) {
              f = 1;
              break;
            }
          }
        }
        sc.sep[i - t.lo] = f;
      }
    });
    pfor([&](int c, int64_t i0, int64_t i1) {
      int64_t k[3] = {0, 0, 0};
      for (int64_t i = i0; i < i1; ++i) {
        const int32_t v = work[i];
        if (sc.sep[i - t.lo]) side[v] = 2;
        k[side[v]]++;
      }
      for (int x = 0; x < 3; ++x) sc.cnt[c * 3 + x] = k[x];
    });
    int64_t na = 0, nbu = 0;
    for (int c = 0; c < nt; ++c) {
      na += sc.cnt[c * 3];
      nbu += sc.cnt[c * 3 + 1];
    }
    if (na == 0 || nbu == 0) {   // no proper split
      pfor([&](int, int64_t i0, int64_t i1) {
        for (int64_t i = i0; i < i1; ++i) side[work[i]] = -1;
      });
      return 0;
    }
    // [A | B | separator], each part in the task's order: chunk c's nodes of a part follow
    // those of the chunks before it
    int64_t at[3] = {t.lo, t.lo + na, t.lo + na + nbu};
    for (int c = 0; c < nt; ++c)
      for (int x = 0; x < 3; ++x) {
        const int64_t k = sc.cnt[c * 3 + x];
        sc.cnt[c * 3 + x] = at[x];
        at[x] += k;
      }
    sc.tmp.assign(work.begin() + t.lo, work.begin() + t.hi);
    pfor([&](int c, int64_t i0, int64_t i1) {
      int64_t pos[3] = {sc.cnt[c * 3], sc.cnt[c * 3 + 1], sc.cnt[c * 3 + 2]};
      for (int64_t i = i0; i < i1; ++i) {
        const int32_t v = sc.tmp[i - t.lo];
        work[pos[side[v]]++] = v;
        side[v] = -1;
      }
    });
    kids[0] = {t.lo, t.lo + na};
    kids[1] = {t.lo + na, t.lo + na + nbu};
    return 2;
  };
  auto split = [&](NdTask t, Scratch &sc, NdTask kids[2]) -> int {
    return t.hi - t.lo >= kNdInner ? split_wide(t, sc, kids) : split_small(t, sc, kids);
  };
  // a task of at most kNdLocal nodes is dissected whole by the thread that takes it
  constexpr int64_t kNdLocal = 1 << 14;
  auto run_local = [&](NdTask t, Scratch &sc) {
    std::vector<NdTask> stack{t};
    NdTask kids[2];
    while (!stack.empty()) {
      NdTask u = stack.back();
      stack.pop_back();
      const int k = split(u, sc, kids);
      for (int i = k - 1; i >= 0; --i) stack.push_back(kids[i]);
    }
  };
  const int nthreads = nr >= (int64_t(1) << 16) ? plan_threads() : 1;
  if (nthreads <= 1) {
    Scratch sc;
    run_local({0, nr}, sc);
    return;
  }
  std::mutex mu;
  std::condition_variable cv;
  std::vector<NdTask> queue{{0, nr}};
  int busy = 0;
  bool failed = false;   // a task threw: every thread stops
  run_threads(nthreads, [&](int) {
    Scratch sc;
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      cv.wait(lk, [&] { return failed || !queue.empty() || busy == 0; });
      if (failed || queue.empty()) return;   // nothing queued and nothing running: done
      const NdTask t = queue.back();
      queue.pop_back();
      ++busy;
      lk.unlock();
      NdTask kids[2];
      int k = 0;
      std::exception_ptr ex;
      try {
        if (t.hi - t.lo <= kNdLocal) run_local(t, sc);
        else k = split(t, sc, kids);
      } catch (...) {
        ex = std::current_exception();
      }
      lk.lock();
      if (ex) failed = true;
      else
        for (int i = 0; i < k; ++i) queue.push_back(kids[i]);
      --busy;
      cv.notify_all();
      if (ex) std::rethrow_exception(ex);
    }
  });
}

// BFS level-structure bisection for graphs without coordinates: from a pseudo-peripheral
// node, the level that splits the node count in half is the separator.  Disconnected task
// sets are split into their components first.
void order_bfs_nd(const Adj &A, int leaf, std::vector<int32_t> &work) {
  const int64_t nr = static_cast<int64_t>(A.ptr.size()) - 1;
  work.resize(static_cast<size_t>(nr));
  std::iota(work.begin(), work.end(), 0);
  std::vector<int64_t> stamp(static_cast<size_t>(nr), -1);
  std::vector<int32_t> lev(static_cast<size_t>(nr), -1);
  std::vector<int32_t> q(static_cast<size_t>(nr)), tmp;
  int64_t cur = 0;
  auto bfs = [&](int32_t src, int64_t st, int64_t &count) -> int32_t {
    // BFS within nodes stamped st; returns the last node reached, fills lev[]
    int64_t head = 0, tail = 0;
    q[tail++] = src;
    lev[src] = 0;
    stamp[src] = st + 1;   // visited marker: st + 1
    while (head < tail) {
      int32_t v = q[head++];
      for (int64_t p = A.ptr[v]; p < A.ptr[v + 1]; ++p) {
        int32_t u = A.idx[p];
        if (stamp[u] == st) { stamp[u] = st + 1; lev[u] = lev[v] + 1; q[tail++] = u; }
      }
    }
    count = tail;
    for (int64_t i = 0; i < tail; ++i) stamp[q[i]] = st;   // unvisit
    return q[tail - 1];
  };
  std::vector<NdTask> stack{{0, nr}};
  while (!stack.empty()) {
    NdTask t = stack.back();
    stack.pop_back();
    const int64_t cnt = t.hi - t.lo;
    if (cnt <= leaf) continue;
    const int64_t st = cur;
    cur += 2;
    for (int64_t i = t.lo; i < t.hi; ++i) stamp[work[i]] = st;
    int64_t reached = 0;
    int32_t far = bfs(work[t.lo], st, reached);
    if (reached < cnt) {   // split off the component of work[lo]
      tmp.assign(work.begin() + t.lo, work.begin() + t.hi);
      for (int64_t i = 0; i < reached; ++i) stamp[q[i]] = st + 1;
      int64_t a = t.lo, b = t.lo + reached;
      for (int32_t v : tmp) (stamp[v] == st + 1 ? work[a++] : work[b++]) = v;
      for (int32_t v : tmp) stamp[v] = -1;
      stack.push_back({t.lo + reached, t.hi});
      stack.push_back({t.lo, t.lo + reached});
      continue;
    }
    int32_t ecc = lev[far];
    for (int it = 0; it < 3; ++it) {   // pseudo-peripheral node
      int32_t nf = bfs(far, st, reached);
      if (lev[nf] <= ecc) break;
      ecc = lev[nf];
      far = nf;
    }
    bfs(far, st, reached);
    ecc = 0;
    for (int64_t i = t.lo; i < t.hi; ++i) ecc = std::max(ecc, lev[work[i]]);
    std::vector<int64_t> per(static_cast<size_t>(ecc + 2), 0);
    for (int64_t i = t.lo; i < t.hi; ++i) per[lev[work[i]]]++;
    int32_t k = 0;
    int64_t acc = 0;
    for (; k <= ecc; ++k) {
      acc += per[k];
      if (2 * acc >= cnt) break;
    }
    int64_t na = 0, nbu = 0;
    for (int64_t i = t.lo; i < t.hi; ++i) {
      int32_t l = lev[work[i]];
      na += l < k;
      nbu += l > k;
    }
    if (na == 0 || nbu == 0) {
      for (int64_t i = t.lo; i < t.hi; ++i) stamp[work[i]] = -1;
      continue;
    }
    tmp.assign(work.begin() + t.lo, work.begin() + t.hi);
    int64_t a = t.lo, b = t.lo + na, c = t.lo + na + nbu;
    for (int32_t v : tmp) {
      int32_t l = lev[v];
      (l < k ? work[a++] : l > k ? work[b++] : work[c++]) = v;
      stamp[v] = -1;
    }
    stack.push_back({t.lo + na, t.lo + na + nbu});
    stack.push_back({t.lo, t.lo + na});
  }
}

// ------------------------------------------------------------------------- etree

// Elimination tree of the permuted pattern by Liu's ancestor path compression.
void etree(const Adj &A, const std::vector<int32_t> &perm, const std::vector<int32_t> &iperm,
           std::vector<int32_t> &parent) {
  const int64_t nr = static_cast<int64_t>(perm.size());
  parent.assign(static_cast<size_t>(nr), -1);
  std::vector<int32_t> anc(static_cast<size_t>(nr), -1);
  for (int64_t k = 0; k < nr; ++k) {
    const int32_t v = perm[k];
    for (int64_t p = A.ptr[v]; p < A.ptr[v + 1]; ++p) {
      int32_t i = iperm[A.idx[p]];
      while (i != -1 && i < k) {
        int32_t next = anc[i];
        anc[i] = static_cast<int32_t>(k);
        if (next == -1) { parent[i] = static_cast<int32_t>(k); break; }
        i = next;
      }
    }
  }
}

int64_t tri(int64_t a) { return a * (a + 1) / 2; }

}  // namespace

void set_host_thread_cap(int cap) { t_thread_cap = cap; }

// ------------------------------------------------------------------------- assembly values

void assembly_values(const Symbolic &S, const double *w, std::vector<double> &vals) {
  vals.resize(S.a_dest.size());
  chunked(S.nnz_lower, [&](int64_t e0, int64_t e1) {
    for (int64_t e = e0; e < e1; ++e) vals[e] = -w[S.a_src[e]];
  });
  chunked(S.nr, [&](int64_t k0, int64_t k1) {
    for (int64_t k = k0; k < k1; ++k) {
      const int64_t r = S.perm[k];
      const int64_t gnode = r + (r >= S.ground);
      double deg = 0.0;
      for (int64_t p = S.csr_indptr[gnode]; p < S.csr_indptr[gnode + 1]; ++p) deg += w[p];
      vals[S.nnz_lower + k] = deg;
    }
  });
}

int32_t sweep_tile(const Symbolic &S, int64_t N, int32_t cap) {
  int64_t q = S.front_budget / (8 * (N + 2 * kBlock));
  q = std::min<int64_t>(q, cap);
  if (q >= 4) q -= q % 4;
  return static_cast<int32_t>(std::max<int64_t>(1, std::min<int64_t>(kQMax, q)));
}

namespace {

// Orders the items [b, e) of a wave's level l (sorted by cost) with the spilled ones first
// and records the level's launch shapes: shared memory of the regular launch, and the count
// and shared memory of the spilled items' launch.
void finish_level(const Symbolic &S, SweepWave &W, int32_t l, SweepItem *b, SweepItem *e) {
  auto spilled = [](const SweepItem &it) { return it.spill != 0; };
  if (std::any_of(b, e, spilled)) std::stable_partition(b, e, spilled);
  int64_t smem = 0, nspill = 0, spill_smem = 0;
  for (const SweepItem *pi = b; pi != e; ++pi) {
    const SweepItem &it = *pi;
    if (it.spill) {
      ++nspill;
      spill_smem = std::max(spill_smem, int64_t(2) * kBlock * sweep_qstride(it.nq) * 8);
    } else {
      smem = std::max(smem, sweep_smem_bytes(sn_nc(S, it.s) + S.nb[it.s], it.nq));
    }
  }
  W.level_smem[l] = smem;
  W.level_nspill[l] = nspill;
  W.level_spill_smem[l] = spill_smem;
}

}  // namespace

namespace {
int build_sweep_plan_impl(Symbolic &S, const int32_t *qcap, std::string &err);
}  // namespace

// Tiles, waves and the two-branch walk of an analysed plan for the given per-size-class
// tile caps (queries per CTA; 0 = the largest that fits).  Rebuilding it does not change the
// arithmetic of any query: blocks stay aligned to kBlock whatever the tile, and a front kept
// in global memory goes through exactly the same operations as one in shared memory.  A failed
// host allocation returns PEERS_ENOMEM (the plan is then unusable).
int build_sweep_plan(Symbolic &S, const int32_t *qcap, std::string &err) {
  try {
    return build_sweep_plan_impl(S, qcap, err);
  } catch (const std::bad_alloc &) {
    err = "host allocation while building the sweep plan";
    return PEERS_ENOMEM;
  }
}

namespace {
int build_sweep_plan_impl(Symbolic &S, const int32_t *qcap, std::string &err) {
  struct Two { int32_t lo, hi; int64_t idx; };
  const int32_t kInfCol = INT32_MAX;
  (void)kInfCol;
  // tile sizes: as many queries as fit the shared-memory budget, up to the size class's cap
  const int32_t ns = S.nsuper;
  for (int c = 0; c < kSizeClasses; ++c)
    S.qcap[c] = qcap && qcap[c] > 0 ? std::min<int32_t>(qcap[c], kQMax) : kQMax;
  S.qtile.assign(static_cast<size_t>(ns), 1);
  S.spill.assign(static_cast<size_t>(ns), 0);
  S.spill_stride = 0;
  for (int32_t s = 0; s < ns; ++s) {
    const int64_t N = sn_nc(S, s) + S.nb[s];
    const int32_t cap = S.qcap[size_class(N)];
    S.qtile[s] = sweep_tile(S, N, cap);
    if (sweep_smem_bytes(N, S.qtile[s]) > S.front_limit) {
      // the front does not fit one CTA's shared memory even for one query: keep the tile's
      // fronts in the CTA's global scratch and take the class's full tile
      S.qtile[s] = std::max<int32_t>(1, std::min<int32_t>(kQMax, cap));
      S.spill[s] = 1;
      S.spill_stride = std::max(S.spill_stride, N * sweep_qstride(S.qtile[s]));
    }
  }

  // waves: bound the carry buffer (per query in flight, one slot of nbmax doubles for its
  // carried front plus one double for its running sum)
  const int64_t budget = S.carry_budget;
  const int64_t slot_bytes = int64_t(8) * (int64_t(S.nbmax) + 1);
  int64_t per_wave = std::max<int64_t>(1, budget / slot_bytes);
  if (per_wave > INT32_MAX) per_wave = INT32_MAX;
  S.waves.clear();
  S.carry_slots = 0;
  S.walk_entries = 0;
  S.walk_fma = 0;
  S.front_bytes = 0;
  // the FMAs of one query's item at supernode s from column block j0 / kBlock on: suffix sums
  // over the supernode's blocks, so that an item's count is one lookup
  std::vector<int64_t> fma_off(static_cast<size_t>(ns) + 1, 0);
  for (int32_t s = 0; s < ns; ++s)
    fma_off[s + 1] = fma_off[s] + (sn_nc(S, s) + kBlock - 1) / kBlock + 1;
  std::vector<int64_t> fma_suf(static_cast<size_t>(fma_off[ns]), 0);
  for (int32_t s = 0; s < ns; ++s) {
    const int64_t nc = sn_nc(S, s), N = nc + S.nb[s];
    const int64_t nbk = fma_off[s + 1] - fma_off[s] - 1;
    for (int64_t jb = nbk - 1; jb >= 0; --jb) {
      const int64_t J = jb * kBlock, bw = std::min<int64_t>(kBlock, nc - J);
      fma_suf[fma_off[s] + jb] = bw * (bw - 1) / 2 + (N - J - bw) * bw + bw +
                                 fma_suf[fma_off[s] + jb + 1];
    }
  }
  auto item_fma = [&](int32_t s, int32_t j0) -> int64_t {
    const int64_t jb = j0 / kBlock, nbk = fma_off[s + 1] - fma_off[s] - 1;
    return jb >= nbk ? 0 : fma_suf[fma_off[s] + jb];
  };
  auto entries = [&](int32_t s, int64_t first_col) -> int64_t {
    const int64_t np = sn_nc(S, s) - first_col;
    return np * (np - 1) / 2 + int64_t(S.nb[s]) * np + np;
  };
  // position of each supernode in level_sn
  std::vector<int32_t> lpos(static_cast<size_t>(ns));
  for (int32_t i = 0; i < ns; ++i) lpos[S.level_sn[i]] = i;
  // the waves' query ranges (one empty wave when there are no queries)
  std::vector<std::pair<int64_t, int64_t>> ranges;
  for (int64_t w0 = 0; w0 < std::max<int64_t>(S.nsorted, 1); w0 += per_wave) {
    const int64_t w1 = std::min<int64_t>(S.nsorted, w0 + per_wave);
    if (w1 <= w0 && S.nsorted > 0) break;
    ranges.emplace_back(w0, w1);
    if (S.nsorted == 0) break;
  }
  const int64_t nw = static_cast<int64_t>(ranges.size());
  const int nthreads = S.nsorted >= (int64_t(1) << 16) ? plan_threads() : 1;
  struct LevelOut {
    int64_t walk_entries = 0, walk_fma = 0, front_bytes = 0;
  };
  struct WaveBuild {
    std::vector<int32_t> rel;       // positions in level_sn of the supernodes it can reach
    std::vector<int64_t> rel_ptr;   // nlevels + 1: level l's are rel[rel_ptr[l] .. [l + 1])
    std::vector<LevelOut> outs;
  };
  std::vector<SweepWave> waves(static_cast<size_t>(nw));
  std::vector<WaveBuild> wb(static_cast<size_t>(nw));
  // Each wave first finds the supernodes that can carry its items: the start supernodes
  // [s_lo, s_hi] of its queries and the ancestors of s_hi (every subtree that holds one of the
  // wave's queries is a range of supernodes meeting [s_lo, s_hi], so its root is in it or
  // above s_hi).  A counting pass then sizes each level's range of the wave's items.
  auto setup_wave = [&](int64_t w) {
    SweepWave &W = waves[w];
    WaveBuild &B = wb[w];
    W.q_begin = ranges[w].first;
    W.q_end = ranges[w].second;
    W.level_ptr.assign(static_cast<size_t>(S.nlevels) + 1, 0);
    W.level_smem.assign(static_cast<size_t>(S.nlevels), 0);
    W.level_nspill.assign(static_cast<size_t>(S.nlevels), 0);
    W.level_spill_smem.assign(static_cast<size_t>(S.nlevels), 0);
    if (W.q_end > W.q_begin) {
      const int32_t s_lo = static_cast<int32_t>(
          std::upper_bound(S.qbeg.begin() + 1, S.qbeg.end(), W.q_begin) - (S.qbeg.begin() + 1));
      const int32_t s_hi = static_cast<int32_t>(
          std::lower_bound(S.qbeg.begin(), S.qbeg.begin() + ns, W.q_end) - S.qbeg.begin()) - 1;
      for (int32_t x = s_lo; x <= s_hi; ++x) B.rel.push_back(lpos[x]);
      for (int32_t x = S.parent[s_hi]; x != -1; x = S.parent[x]) B.rel.push_back(lpos[x]);
      std::sort(B.rel.begin(), B.rel.end());
    }
    B.rel_ptr.resize(static_cast<size_t>(S.nlevels) + 1);
    for (int32_t l = 0; l <= S.nlevels; ++l)
      B.rel_ptr[l] = std::lower_bound(B.rel.begin(), B.rel.end(), S.level_ptr[l]) - B.rel.begin();
    for (int32_t l = 0; l < S.nlevels; ++l) {
      int64_t cnt = 0;
      for (int64_t r = B.rel_ptr[l]; r < B.rel_ptr[l + 1]; ++r) {
        const int32_t p = S.level_sn[B.rel[r]];
        const int64_t tile = S.qtile[p];
        auto tiles = [&](int64_t b, int64_t e) {
          b = std::max(b, W.q_begin);
          e = std::min(e, W.q_end);
          return e > b ? (e - b + tile - 1) / tile : 0;
        };
        for (int32_t c = S.child_ptr[p]; c < S.child_ptr[p + 1]; ++c) {
          const int32_t ch = S.child_list[c];
          cnt += tiles(S.qbeg[S.fdesc[ch]], S.qbeg[ch + 1]);
        }
        cnt += tiles(S.qbeg[p], S.qbeg[p + 1]);
      }
      W.level_ptr[l + 1] = W.level_ptr[l] + cnt;
    }
    W.items.resize(static_cast<size_t>(W.level_ptr[S.nlevels]));
    B.outs.assign(static_cast<size_t>(S.nlevels), LevelOut{});
  };
  // Then every (wave, level) is independent: it builds its items, ordered by cost (largest
  // first; ties in the order they are made), into its own range of the wave's items, and its
  // share of the walk counts.  They run on up to kPlanThreads host threads; the counts are
  // summed in wave and level order, so the plan is the same as one thread's.
  std::atomic<bool> miscount{false};
  auto build_level = [&](int64_t w, int32_t l) {
    SweepWave &W = waves[w];
    const WaveBuild &B = wb[w];
    LevelOut &o = wb[w].outs[l];
    const int64_t count = W.level_ptr[l + 1] - W.level_ptr[l];
    std::vector<int64_t, NoInitAlloc<int64_t>> keys;
    std::vector<SweepItem, NoInitAlloc<SweepItem>> made;
    keys.reserve(static_cast<size_t>(count));
    made.reserve(static_cast<size_t>(count));
    for (int64_t r = B.rel_ptr[l]; r < B.rel_ptr[l + 1]; ++r) {
      const int32_t p = S.level_sn[B.rel[r]];
      const int32_t tile = S.qtile[p];
      auto emit = [&](int32_t src, int64_t b, int64_t e) {
        b = std::max(b, W.q_begin);
        e = std::min(e, W.q_end);
        for (int64_t q = b; q < e; q += tile) {
          SweepItem it{};
          it.s = p;
          it.src = src;
          it.q0 = static_cast<int32_t>(q);
          it.nq = static_cast<int32_t>(std::min<int64_t>(tile, e - q));
          it.spill = S.spill[p];
          int32_t j0;
          if (src >= 0) {
            j0 = S.rmap[S.rows_off[src]];
            o.walk_entries += it.nq * entries(p, j0);
          } else {
            j0 = S.qa[q];
            for (int64_t k = q; k < q + it.nq; ++k) o.walk_entries += entries(p, S.qa[k]);
          }
          it.j0 = (j0 / kBlock) * kBlock;
          const int64_t f = it.nq * item_fma(p, it.j0);
          o.walk_fma += f;
          // fronts carried between levels: read from the child's carry, written for the parent
          o.front_bytes += int64_t(8) * it.nq * ((src >= 0 ? S.nb[src] : 0) + S.nb[p]);
          keys.push_back(f);
          made.push_back(it);
        }
      };
      for (int32_t c = S.child_ptr[p]; c < S.child_ptr[p + 1]; ++c) {
        const int32_t ch = S.child_list[c];
        emit(ch, S.qbeg[S.fdesc[ch]], S.qbeg[ch + 1]);
      }
      emit(-1, S.qbeg[p], S.qbeg[p + 1]);
    }
    if (static_cast<int64_t>(made.size()) != count) {
      miscount = true;
      return;
    }
    std::vector<int32_t> order(made.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t x, int32_t y) { return keys[x] > keys[y]; });
    SweepItem *dst = W.items.data() + W.level_ptr[l];
    for (int32_t x : order) *dst++ = made[x];
    finish_level(S, W, l, W.items.data() + W.level_ptr[l], dst);
  };
  {
    std::atomic<int64_t> next{0};
    run_threads(nthreads, [&](int) {
      for (int64_t w = next++; w < nw; w = next++) setup_wave(w);
    });
    const int64_t ntasks = nw * S.nlevels;
    std::atomic<int64_t> task{0};
    run_threads(nthreads, [&](int) {
      for (int64_t t = task++; t < ntasks; t = task++)
        build_level(t / S.nlevels, static_cast<int32_t>(t % S.nlevels));
    });
  }
  if (miscount) {
    err = "internal: sweep items disagree with their count";
    return PEERS_EINVAL;
  }
  for (int64_t w = 0; w < nw; ++w) {
    for (const LevelOut &o : wb[w].outs) {
      S.walk_entries += o.walk_entries;
      S.walk_fma += o.walk_fma;
      S.front_bytes += o.front_bytes;
    }
    S.carry_slots = std::max(S.carry_slots, waves[w].q_end - waves[w].q_begin);
    S.waves.push_back(std::move(waves[w]));
  }
  if (S.nsorted == 0 && S.nq_two > 0) S.waves.clear();

  // ---- two-branch walk (listed pairs whose etree paths merge above the start) ----
  // Slots nsorted + 2k (branch of the lower endpoint, continues after the merge) and
  // nsorted + 2k + 1 (branch of the upper endpoint, ends at the merge supernode).
  S.ldesc.clear();
  S.two_user.clear();
  S.two_a.clear();
  S.two_b.clear();
  if (S.nq_two > 0) {
    std::vector<int32_t> depth(static_cast<size_t>(ns), 0);
    for (int32_t s = ns - 1; s >= 0; --s)
      depth[s] = S.parent[s] == -1 ? 0 : depth[S.parent[s]] + 1;
    const int64_t per_two = std::max<int64_t>(1, per_wave / 2);
    const int32_t kInf = INT32_MAX;
    // rank of each supernode in (level, supernode) order, the order the steps run in
    std::vector<int32_t> rank(static_cast<size_t>(ns));
    {
      std::vector<int32_t> at(static_cast<size_t>(S.nlevels) + 1, 0);
      for (int32_t s = 0; s < ns; ++s) at[S.level[s] + 1]++;
      for (int32_t l = 0; l < S.nlevels; ++l) at[l + 1] += at[l];
      for (int32_t s = 0; s < ns; ++s) rank[s] = at[S.level[s]]++;
    }
    for (int64_t k0 = 0; k0 < S.nq_two; k0 += per_two) {
      const int64_t k1 = std::min<int64_t>(S.nq_two, k0 + per_two);
      // the steps of pair k, in the order they are made, each passed to emit(supernode, step);
      // the pair's merge supernode (lowest common ancestor of its two start supernodes, -1:
      // different trees) is merge[k - k0]
      std::vector<int32_t> merge(static_cast<size_t>(k1 - k0));
      auto walk = [&](int64_t k, auto &&emit) {
        const int32_t sa = S.col2sn[S.two_lo[k]], sb = S.col2sn[S.two_hi[k]];
        const int32_t A = static_cast<int32_t>(S.nsorted + 2 * k), B = A + 1;
        const int32_t m = merge[k - k0];
        int32_t prev = -1;
        for (int32_t p = sa; p != m; prev = p, p = S.parent[p])
          emit(p, SweepDesc{A, prev, -1, -1, -1});
        const int32_t child_a = prev;
        prev = -1;
        if (sb != m)
          for (int32_t p = sb; p != m; prev = p, p = S.parent[p])
            emit(p, SweepDesc{B, prev, -1, -1, -1});
        const int32_t child_b = prev;
        if (m != -1) {
          if (sb == m)
            emit(m, SweepDesc{A, child_a, -1, -1, S.two_hi[k] - S.first[m]});
          else
            emit(m, SweepDesc{A, child_a, B, child_b, -1});
          prev = m;
          for (int32_t p = S.parent[m]; p != -1; prev = p, p = S.parent[p])
            emit(p, SweepDesc{A, prev, -1, -1, -1});
        }
      };
      // the steps in (level, supernode) order, each supernode's in the order they are made:
      // one pass counts them per supernode, a second writes each to its place
      std::vector<int64_t> at(static_cast<size_t>(ns) + 1, 0);
      for (int64_t k = k0; k < k1; ++k) {
        const Two t{S.two_lo[k], S.two_hi[k], S.two_idx[k]};
        const int32_t sa = S.col2sn[t.lo], sb = S.col2sn[t.hi];
        const int32_t A = static_cast<int32_t>(S.nsorted + 2 * k), B = A + 1;
        S.qorig[A] = S.qorig[B] = t.idx;
        S.qa[A] = t.lo - S.first[sa];
        S.qb[A] = -1;
        S.qa[B] = -1;
        S.qb[B] = t.hi - S.first[sb];
        int32_t x = sa, y = sb;
        while (x != y && x != -1 && y != -1) {
          if (depth[x] >= depth[y]) x = S.parent[x]; else y = S.parent[y];
        }
        const int32_t m = (x == y) ? x : -1;
        merge[k - k0] = m;
        walk(k, [&](int32_t p, const SweepDesc &) { at[rank[p] + 1]++; });
        S.two_user.push_back(t.idx);
        S.two_a.push_back(A);
        S.two_b.push_back(m == -1 ? B : -1);
      }
      for (int32_t r = 0; r < ns; ++r) at[r + 1] += at[r];
      struct Step { int32_t s; SweepDesc d; };
      std::vector<Step, NoInitAlloc<Step>> steps(static_cast<size_t>(at[ns]));
      for (int64_t k = k0; k < k1; ++k)
        walk(k, [&](int32_t p, const SweepDesc &d) { steps[at[rank[p]]++] = Step{p, d}; });
      SweepWave W;
      W.q_begin = S.nsorted + 2 * k0;
      W.q_end = S.nsorted + 2 * k1;
      W.two_begin = k0;
      W.two_end = k1;
      S.carry_slots = std::max(S.carry_slots, W.q_end - W.q_begin);
      W.level_ptr.assign(static_cast<size_t>(S.nlevels) + 1, 0);
      W.level_smem.assign(static_cast<size_t>(S.nlevels), 0);
      W.level_nspill.assign(static_cast<size_t>(S.nlevels), 0);
      W.level_spill_smem.assign(static_cast<size_t>(S.nlevels), 0);
      auto first_row = [&](const SweepDesc &d) -> int32_t {
        int32_t r = kInf;
        if (d.src_a >= 0) r = S.rmap[S.rows_off[d.src_a]];
        else {
          if (S.qa[d.a] >= 0) r = std::min(r, S.qa[d.a]);
          if (S.qb[d.a] >= 0) r = std::min(r, S.qb[d.a]);
        }
        if (d.b >= 0) r = std::min(r, S.rmap[S.rows_off[d.src_b]]);
        else if (d.seed_b >= 0) r = std::min(r, d.seed_b);
        return r;
      };
      W.items.reserve(steps.size());
      size_t i = 0;
      for (int32_t l = 0; l < S.nlevels; ++l) {
        const size_t lb = W.items.size();
        while (i < steps.size() && S.level[steps[i].s] == l) {
          const int32_t p = steps[i].s;
          size_t e = i;
          while (e < steps.size() && steps[e].s == p) ++e;
          for (size_t c = i; c < e; c += S.qtile[p]) {
            const size_t ce = std::min(e, c + static_cast<size_t>(S.qtile[p]));
            SweepItem it{};
            it.s = p;
            it.src = -1;
            it.kind = 1;
            it.spill = S.spill[p];
            it.q0 = static_cast<int32_t>(S.ldesc.size());
            it.nq = static_cast<int32_t>(ce - c);
            int32_t j0 = kInf;
            for (size_t q = c; q < ce; ++q) {
              const int32_t fr = first_row(steps[q].d);
              j0 = std::min(j0, fr);
              S.walk_entries += entries(p, fr);
              S.ldesc.push_back(steps[q].d);
            }
            it.j0 = (j0 / kBlock) * kBlock;
            S.walk_fma += it.nq * item_fma(p, it.j0);
            W.items.push_back(it);
          }
          i = e;
        }
        finish_level(S, W, l, W.items.data() + lb, W.items.data() + W.items.size());
        W.level_ptr[l + 1] = static_cast<int64_t>(W.items.size());
      }
      S.waves.push_back(std::move(W));
    }
  }
  return PEERS_OK;
}
}  // namespace

// ------------------------------------------------------------------------- analyze

int analyze(Symbolic &S, int64_t n, const int64_t *indptr, const int32_t *indices,
            const double *w, int32_t ground, int64_t nq, const int32_t *qu, const int32_t *qv,
            const double *coords, int dim, const peers_options &opt, std::string &err) {
  int st = validate(n, indptr, indices, w, ground, err);
  if (st != PEERS_OK) return st;
  auto t0 = Clock::now();
  S.n = n;
  S.nr = n - 1;
  S.ground = ground;
  S.nnz_csr = indptr[n];
  S.csr_indptr.resize(static_cast<size_t>(n) + 1);
  S.w0.resize(static_cast<size_t>(indptr[n]));
  chunked(n + 1, [&](int64_t i0, int64_t i1) {
    std::copy(indptr + i0, indptr + i1, S.csr_indptr.begin() + i0);
  });
  chunked(indptr[n], [&](int64_t p0, int64_t p1) {
    std::copy(w + p0, w + p1, S.w0.begin() + p0);
  });
  const int64_t nr = S.nr;
  const int leaf = opt.nd_leaf > 0 ? opt.nd_leaf : 32;
  Adj A = reduced_adjacency(n, indptr, indices, ground);

  // ---- ordering ----
  std::vector<int32_t> perm;
  int mode = opt.ordering;
  if (mode == 0) mode = (coords && dim > 0) ? 1 : 2;
  if (mode == 1) {
    if (!coords || dim <= 0) { err = "coordinate ordering needs coords"; return PEERS_EINVAL; }
    std::vector<double> xy(static_cast<size_t>(nr) * dim);
    for (int64_t i = 0; i < n; ++i) {
      if (i == ground) continue;
      const int64_t r = i > ground ? i - 1 : i;
      for (int a = 0; a < dim; ++a) xy[r * dim + a] = coords[i * dim + a];
    }
    order_coordinate_nd(A, xy.data(), dim, leaf, perm);
  } else if (mode == 2) {
    order_bfs_nd(A, leaf, perm);
  } else if (mode == 3) {
    perm.resize(static_cast<size_t>(nr));
    std::iota(perm.begin(), perm.end(), 0);
  } else {
    err = "unknown ordering";
    return PEERS_EINVAL;
  }
  std::vector<int32_t> iperm(static_cast<size_t>(nr));
  for (int64_t k = 0; k < nr; ++k) iperm[perm[k]] = static_cast<int32_t>(k);

  // ---- etree, postorder ----
  std::vector<int32_t> par;
  etree(A, perm, iperm, par);
  {
    std::vector<int32_t> head(static_cast<size_t>(nr), -1), next(static_cast<size_t>(nr), -1);
    for (int64_t k = nr - 1; k >= 0; --k)
      if (par[k] != -1) { next[k] = head[par[k]]; head[par[k]] = static_cast<int32_t>(k); }
    std::vector<int32_t> post(static_cast<size_t>(nr)), stk;
    int64_t cnt = 0;
    for (int64_t r = 0; r < nr; ++r) {
      if (par[r] != -1) continue;
      stk.push_back(static_cast<int32_t>(r));
      while (!stk.empty()) {
        int32_t v = stk.back();
        if (head[v] != -1) {       // descend into the next unvisited child
          int32_t c = head[v];
          head[v] = next[c];
          stk.push_back(c);
        } else {
          post[v] = static_cast<int32_t>(cnt++);
          stk.pop_back();
        }
      }
    }
    std::vector<int32_t> perm2(static_cast<size_t>(nr)), par2(static_cast<size_t>(nr));
    for (int64_t k = 0; k < nr; ++k) {
      perm2[post[k]] = perm[k];
      par2[post[k]] = par[k] == -1 ? -1 : post[par[k]];
    }
    perm.swap(perm2);
    par.swap(par2);
    for (int64_t k = 0; k < nr; ++k) iperm[perm[k]] = static_cast<int32_t>(k);
  }
  // connectivity (the reduced Laplacian is SPD exactly when G is connected): the etree has one
  // tree per connected component of the reduced graph, and G is connected exactly when each
  // of them holds a neighbour of the ground
  {
    std::vector<char> reach(static_cast<size_t>(nr), 0);
    for (int64_t p = indptr[ground]; p < indptr[ground + 1]; ++p) {
      const int32_t j = indices[p];
      reach[iperm[j > ground ? j - 1 : j]] = 1;
    }
    for (int64_t k = 0; k < nr; ++k) {   // postorder: a subtree is complete when its root is met
      if (par[k] != -1) reach[par[k]] |= reach[k];
      else if (!reach[k]) { err = "graph is not connected"; return PEERS_ENOTCONNECTED; }
    }
  }
  S.t_order = since(t0);
  auto t1 = Clock::now();

  // ---- column counts (strictly lower) from the leaves of the row subtrees (Gilbert, Ng and
  //      Peyton).  Column j of L holds row i > j exactly when j lies in the row subtree of i,
  //      the union of the etree paths from row i's entries up to i.  The numbering is an etree
  //      postorder, so the subtree of j is the index range [fdesc[j], j].  Marks +1 at each
  //      leaf of a row subtree, -1 at the lowest common ancestor of consecutive leaves (found
  //      by path-compressed union-find over the finished subtrees) and -1 at the parent of
  //      every non-root make each column's count (with its diagonal) the sum of the marks over
  //      its subtree. ----
  std::vector<int64_t> cc(static_cast<size_t>(nr), 0);
  std::vector<int32_t> nchild(static_cast<size_t>(nr), 0);
  {
    std::vector<int32_t> fdesc(static_cast<size_t>(nr), -1);
    for (int64_t k = 0; k < nr; ++k) {
      cc[k] = fdesc[k] == -1 ? 1 : 0;   // an etree leaf starts with its own diagonal
      for (int32_t j = static_cast<int32_t>(k); j != -1 && fdesc[j] == -1; j = par[j])
        fdesc[j] = static_cast<int32_t>(k);
    }
    for (int64_t k = 0; k < nr; ++k)
      if (par[k] != -1) { cc[par[k]]--; nchild[par[k]]++; }
    std::vector<int32_t> anc(static_cast<size_t>(nr)), maxfirst(static_cast<size_t>(nr), -1),
        prevleaf(static_cast<size_t>(nr), -1);
    std::iota(anc.begin(), anc.end(), 0);
    auto find = [&](int32_t x) {
      int32_t r = x;
      while (anc[r] != r) r = anc[r];
      while (anc[x] != r) { const int32_t nx = anc[x]; anc[x] = r; x = nx; }
      return r;
    };
    // column j as a possible leaf of row i's subtree (rows' columns taken in increasing order)
    auto leaf_step = [&](int32_t i, int32_t j) {
      if (fdesc[j] <= maxfirst[i]) return;   // j is not a new leaf of row i's tree
      maxfirst[i] = fdesc[j];
      const int32_t jprev = prevleaf[i];
      prevleaf[i] = j;
      cc[j]++;
      if (jprev != -1) cc[find(jprev)]--;
    };
    // The row subtree of a row i lies in the etree subtree of i, so the etree subtrees of at
    // most nr / (4 nthreads) columns whose parent's subtree is larger take their own rows on
    // host threads of their own (the lowest common ancestors of their rows' leaves stay inside
    // them).  The rows above those subtrees follow on one thread, their (row, column) pairs in
    // increasing column order, over a fresh union-find that links every column before the
    // current one: the marks each row leaves do not depend on how the rows are split.
    const int nthreads = nr >= (int64_t(1) << 16) ? plan_threads() : 1;
    const int64_t cap = nthreads > 1 ? std::max<int64_t>(1, nr / (4 * nthreads)) : nr;
    auto big = [&](int64_t k) { return k - fdesc[k] + 1 > cap; };
    std::vector<int32_t> roots;
    for (int64_t k = 0; k < nr; ++k)
      if (!big(k) && (par[k] == -1 || big(par[k]))) roots.push_back(static_cast<int32_t>(k));
    std::atomic<size_t> next{0};
    run_threads(nthreads, [&](int) {
      for (size_t x = next++; x < roots.size(); x = next++) {
        const int32_t r = roots[x];
        for (int32_t j = fdesc[r]; j <= r; ++j) {
          const int32_t v = perm[j];
          for (int64_t p = A.ptr[v]; p < A.ptr[v + 1]; ++p) {
            const int32_t i = iperm[A.idx[p]];
            if (i > j && i <= r) leaf_step(i, j);
          }
          if (j != r) anc[j] = par[j];
        }
      }
    });
    std::vector<std::pair<int32_t, int32_t>> top;   // (column j, row i > j), row i above them
    for (int64_t k = 0; k < nr; ++k) {
      if (!big(k)) continue;
      const int32_t v = perm[k];
      for (int64_t p = A.ptr[v]; p < A.ptr[v + 1]; ++p) {
        const int32_t j = iperm[A.idx[p]];
        if (j < k) top.emplace_back(j, static_cast<int32_t>(k));
      }
    }
    if (!top.empty()) {
      std::sort(top.begin(), top.end());
      std::iota(anc.begin(), anc.end(), 0);
      int64_t linked = 0;
      for (const auto &pr : top) {
        for (; linked < pr.first; ++linked)
          if (par[linked] != -1) anc[linked] = par[linked];
        leaf_step(pr.second, pr.first);
      }
    }
    for (int64_t k = 0; k < nr; ++k)
      if (par[k] != -1) cc[par[k]] += cc[k];
    for (int64_t k = 0; k < nr; ++k) cc[k] -= 1;
  }

  // ---- fundamental supernodes ----
  std::vector<int32_t> ffirst;
  for (int64_t k = 0; k < nr; ++k) {
    bool join = k > 0 && par[k - 1] == k && cc[k - 1] == cc[k] + 1 && nchild[k] == 1;
    if (!join) ffirst.push_back(static_cast<int32_t>(k));
  }
  const int32_t nf = static_cast<int32_t>(ffirst.size());
  ffirst.push_back(static_cast<int32_t>(nr));
  std::vector<int32_t> fcol2sn(static_cast<size_t>(nr));
  for (int32_t s = 0; s < nf; ++s)
    for (int32_t k = ffirst[s]; k < ffirst[s + 1]; ++k) fcol2sn[k] = s;
  std::vector<int32_t> fparent(static_cast<size_t>(nf));
  for (int32_t s = 0; s < nf; ++s) {
    int32_t last = ffirst[s + 1] - 1;
    fparent[s] = par[last] == -1 ? -1 : fcol2sn[par[last]];
  }
  // |B_s| of a fundamental supernode: the column count of its last column
  std::vector<int64_t> fnb(static_cast<size_t>(nf));
  for (int32_t s = 0; s < nf; ++s) fnb[s] = cc[ffirst[s + 1] - 1];

  // ---- relaxed amalgamation: a supernode whose columns end right before its parent's
  //      (its parent's last child) joins the parent when the merge is small or adds few
  //      explicit zeros ----
  const int relax_small = opt.relax_small > 0 ? opt.relax_small : 8;
  const int relax_max = opt.relax_max > 0 ? opt.relax_max : 32;
  const double relax_frac = opt.relax_frac > 0 ? opt.relax_frac : 0.15;
  std::vector<int32_t> into(static_cast<size_t>(nf), -1), cfirst(ffirst.begin(), ffirst.end() - 1),
      ncols(static_cast<size_t>(nf));
  std::vector<int64_t> zeros(static_cast<size_t>(nf), 0);
  for (int32_t s = 0; s < nf; ++s) ncols[s] = ffirst[s + 1] - ffirst[s];
  for (int32_t s = 0; s < nf; ++s) {
    const int32_t p = fparent[s];
    if (p == -1 || cfirst[s] + ncols[s] != cfirst[p]) continue;
    const int64_t a = ncols[s], b = ncols[p];
    const int64_t nbs = fnb[s], nbp = fnb[p];
    const int64_t em = tri(a + b) + (a + b) * nbp;
    const int64_t zm = zeros[s] + zeros[p] + a * (b + nbp - nbs);
    if (a + b <= relax_small || (a + b <= relax_max && zm <= relax_frac * em)) {
      into[s] = p;
      cfirst[p] = cfirst[s];
      ncols[p] += static_cast<int32_t>(a);
      zeros[p] = zm;
    }
  }
  std::vector<int32_t> fin(static_cast<size_t>(nf), -1);   // fundamental -> final id
  int32_t ns = 0;
  for (int32_t s = 0; s < nf; ++s)
    if (into[s] == -1) fin[s] = ns++;
  S.nsuper = ns;
  S.first.assign(static_cast<size_t>(ns) + 1, 0);
  S.parent.assign(static_cast<size_t>(ns), -1);
  S.nb.assign(static_cast<size_t>(ns), 0);
  S.rows_off.assign(static_cast<size_t>(ns) + 1, 0);
  S.rows.clear();
  for (int32_t s = 0; s < nf; ++s) {
    if (into[s] != -1) continue;
    const int32_t f = fin[s];
    S.first[f] = cfirst[s];
    int32_t p = fparent[s];
    while (p != -1 && into[p] != -1) p = into[p];
    S.parent[f] = p == -1 ? -1 : fin[p];
    S.nb[f] = static_cast<int32_t>(fnb[s]);
    S.rows_off[f + 1] = S.rows_off[f] + fnb[s];
  }
  S.first[ns] = static_cast<int32_t>(nr);
  S.col2sn.assign(static_cast<size_t>(nr), 0);
  for (int32_t s = 0; s < ns; ++s)
    for (int32_t k = S.first[s]; k < S.first[s + 1]; ++k) S.col2sn[k] = s;
  // row structure B_s (rows past s's last column).  Row i belongs to B_s exactly when s lies
  // on the supernodal etree path from the supernode of one of row i's entries j < i up to
  // (not including) the supernode of i; rows are visited in increasing order, so each B_s
  // fills sorted, into the slot its column count sized.  The walks of a row stay inside the
  // subtree of its supernode, and rows above a subtree are greater than all of its rows, so
  // disjoint subtrees run on host threads of their own and the rows above them follow.
  {
    S.rows.clear();
    S.rows.resize(static_cast<size_t>(S.rows_off[ns]));   // every slot is written below
    std::vector<int64_t> fill(S.rows_off.begin(), S.rows_off.end() - 1);
    std::vector<int32_t> mk(static_cast<size_t>(ns), -1);
    auto run_rows = [&](int64_t i0, int64_t i1) -> bool {
      for (int64_t ii = i0; ii < i1; ++ii) {
        const int32_t i = static_cast<int32_t>(ii);
        mk[S.col2sn[i]] = i;
        const int32_t v = perm[i];
        for (int64_t p = A.ptr[v]; p < A.ptr[v + 1]; ++p) {
          const int32_t j = iperm[A.idx[p]];
          if (j >= i) continue;
          for (int32_t t = S.col2sn[j]; t != -1 && mk[t] != i; t = S.parent[t]) {
            if (fill[t] == S.rows_off[t + 1]) return false;
            mk[t] = i;
            S.rows[fill[t]++] = i;
          }
        }
      }
      return true;
    };
    bool ok = true;
    const int nthreads = nr >= (int64_t(1) << 16) ? plan_threads() : 1;
    if (nthreads <= 1) {
      ok = run_rows(0, nr);
    } else {
      // subtrees of at most nr / (4 nthreads) rows whose parent's subtree is larger; a subtree
      // of supernode s holds supernodes [sub[s], s] (postorder) and rows [first[sub[s]],
      // first[s + 1])
      std::vector<int32_t> sub(static_cast<size_t>(ns));
      std::iota(sub.begin(), sub.end(), 0);
      for (int32_t t = 0; t < ns; ++t)
        if (S.parent[t] != -1) sub[S.parent[t]] = std::min(sub[S.parent[t]], sub[t]);
      const int64_t cap = std::max<int64_t>(1, nr / (4 * nthreads));
      auto big = [&](int32_t t) { return S.first[t + 1] - S.first[sub[t]] > cap; };
      std::vector<int32_t> roots;
      for (int32_t t = 0; t < ns; ++t)
        if (!big(t) && (S.parent[t] == -1 || big(S.parent[t]))) roots.push_back(t);
      std::atomic<size_t> next{0};
      std::atomic<bool> good{true};
      run_threads(nthreads, [&](int) {
        for (size_t r = next++; r < roots.size(); r = next++)
          if (!run_rows(S.first[sub[roots[r]]], S.first[roots[r] + 1])) good = false;
      });
      ok = good;
      // the rows of the supernodes above those subtrees, in increasing order
      for (int32_t t = 0; t < ns && ok; ++t)
        if (big(t)) ok = run_rows(S.first[t], S.first[t + 1]);
    }
    for (int32_t t = 0; t < ns && ok; ++t) ok = fill[t] == S.rows_off[t + 1];
    if (!ok) {
      err = "internal: supernode structure disagrees with the column counts";
      return PEERS_EINVAL;
    }
  }
  S.perm = perm;
  S.iperm = iperm;

  // children, subtree starts, levels (height above the leaves)
  S.child_ptr.assign(static_cast<size_t>(ns) + 1, 0);
  for (int32_t s = 0; s < ns; ++s)
    if (S.parent[s] != -1) S.child_ptr[S.parent[s] + 1]++;
  for (int32_t s = 0; s < ns; ++s) S.child_ptr[s + 1] += S.child_ptr[s];
  S.child_list.assign(static_cast<size_t>(S.child_ptr[ns]), 0);
  {
    std::vector<int32_t> fill(S.child_ptr.begin(), S.child_ptr.end() - 1);
    for (int32_t s = 0; s < ns; ++s)
      if (S.parent[s] != -1) S.child_list[fill[S.parent[s]]++] = s;
  }
  S.fdesc.assign(static_cast<size_t>(ns), 0);
  S.level.assign(static_cast<size_t>(ns), 0);
  for (int32_t s = 0; s < ns; ++s) {
    S.fdesc[s] = s;
    for (int32_t c = S.child_ptr[s]; c < S.child_ptr[s + 1]; ++c) {
      const int32_t ch = S.child_list[c];
      S.fdesc[s] = std::min(S.fdesc[s], S.fdesc[ch]);
      S.level[s] = std::max(S.level[s], S.level[ch] + 1);
    }
  }
  S.nlevels = 0;
  for (int32_t s = 0; s < ns; ++s) S.nlevels = std::max(S.nlevels, S.level[s] + 1);
  S.level_ptr.assign(static_cast<size_t>(S.nlevels) + 1, 0);
  for (int32_t s = 0; s < ns; ++s) S.level_ptr[S.level[s] + 1]++;
  for (int32_t l = 0; l < S.nlevels; ++l) S.level_ptr[l + 1] += S.level_ptr[l];
  S.level_sn.assign(static_cast<size_t>(ns), 0);
  {
    std::vector<int32_t> fill(S.level_ptr.begin(), S.level_ptr.end() - 1);
    for (int32_t s = 0; s < ns; ++s) S.level_sn[fill[S.level[s]]++] = s;
    // levels sorted independently, on up to kPlanThreads host threads
    std::atomic<int32_t> next{0};
    run_threads(ns >= (1 << 16) ? plan_threads() : 1, [&](int) {
      for (int32_t l = next++; l < S.nlevels; l = next++)
        std::stable_sort(S.level_sn.begin() + S.level_ptr[l],
                         S.level_sn.begin() + S.level_ptr[l + 1],
                         [&](int32_t a, int32_t b) { return sn_nc(S, a) > sn_nc(S, b); });
    });
  }

  // relative maps into the parent front: rows of s (C_s then B_s) -> local index in parent.
  // A child's rows and its parent's are both ascending, so one forward search through the
  // parent's rows maps a child; children are mapped independently, over host-thread chunks.
  S.rmap.clear();
  S.rmap.resize(S.rows.size());   // every slot is written below
  {
    const int nchunks =
        static_cast<int64_t>(S.rows.size()) >= (int64_t(1) << 20) ? plan_threads() : 1;
    std::vector<const char *> bad(static_cast<size_t>(nchunks), nullptr);
    run_threads(nchunks, [&](int c) {
      for (int32_t s = static_cast<int32_t>(int64_t(ns) * c / nchunks);
           s < static_cast<int32_t>(int64_t(ns) * (c + 1) / nchunks); ++s) {
        const int32_t p = S.parent[s];
        if (p == -1) {
          std::fill(S.rmap.begin() + S.rows_off[s], S.rmap.begin() + S.rows_off[s + 1], -1);
          continue;
        }
        const int32_t pf = S.first[p], pnc = sn_nc(S, p);
        const auto pb = S.rows.begin() + S.rows_off[p], pe = S.rows.begin() + S.rows_off[p + 1];
        auto at = pb;
        for (int64_t t = S.rows_off[s]; t < S.rows_off[s + 1]; ++t) {
          const int32_t r = S.rows[t];
          if (r < pf) { bad[c] = "internal: row below the parent's first column"; return; }
          if (r < pf + pnc) { S.rmap[t] = r - pf; continue; }
          at = std::lower_bound(at, pe, r);
          if (at == pe || *at != r) { bad[c] = "internal: child row missing from parent"; return; }
          S.rmap[t] = pnc + static_cast<int32_t>(at - pb);
        }
      }
    });
    for (const char *m : bad)
      if (m) { err = m; return PEERS_EINVAL; }
  }

  // ---- device layout ----
  S.panel_off.assign(static_cast<size_t>(ns) + 1, 0);
  S.tinv_off.assign(static_cast<size_t>(ns) + 1, 0);
  S.u_off.assign(static_cast<size_t>(ns) + 1, 0);
  S.nbmax = 0;
  S.factor_fma = 0;
  for (int32_t s = 0; s < ns; ++s) {
    const int64_t nc = sn_nc(S, s), nbv = S.nb[s], N = nc + nbv;
    S.panel_off[s + 1] = S.panel_off[s] + N * nc;
    const int64_t nblk = (nc + kBlock - 1) / kBlock, bwl = nc - (nblk - 1) * kBlock;
    S.tinv_off[s + 1] = S.tinv_off[s] + (nblk - 1) * kBlock * kBlock + bwl * bwl;
    S.u_off[s + 1] = S.u_off[s] + nbv * nbv;
    S.nbmax = std::max<int32_t>(S.nbmax, static_cast<int32_t>(nbv));
    // dense partial LDL^T of an N x nc front: sum over columns k of (N-k-1)(N-k)/2
    for (int64_t k = 0; k < nc; ++k) S.factor_fma += (N - k - 1) * (N - k) / 2;
  }
  S.panel_total = S.panel_off[ns];
  S.tinv_total = S.tinv_off[ns];
  S.u_total = S.u_off[ns];

  // ---- assembly map of L_r into the panels ----
  {
    auto local_row = [&](int32_t s, int32_t i) -> int64_t {
      const int32_t f = S.first[s], nc = sn_nc(S, s);
      if (i < f + nc) return i - f;
      auto b = S.rows.begin() + S.rows_off[s], e = S.rows.begin() + S.rows_off[s + 1];
      auto it = std::lower_bound(b, e, i);
      if (it == e || *it != i) return -1;
      return nc + (it - b);
    };
    // rows in contiguous chunks, one per host thread: a first pass counts each chunk's lower
    // entries, a second writes them at the chunk's offset (the order of one pass over the rows)
    const int nchunks = indptr[n] >= (int64_t(1) << 20) ? plan_threads() : 1;
    std::vector<int64_t> off(static_cast<size_t>(nchunks) + 1, 0);
    std::vector<char> bad(static_cast<size_t>(nchunks), 0);
    auto row_of = [&](int64_t g) { return iperm[g > ground ? g - 1 : g]; };
    run_threads(nchunks, [&](int c) {
      int64_t cnt = 0;
      for (int64_t gi = n * c / nchunks; gi < n * (c + 1) / nchunks; ++gi) {
        if (gi == ground) continue;
        const int32_t i = row_of(gi);
        for (int64_t p = indptr[gi]; p < indptr[gi + 1]; ++p)
          cnt += indices[p] != ground && i > row_of(indices[p]);
      }
      off[c + 1] = cnt;
    });
    for (int c = 0; c < nchunks; ++c) off[c + 1] += off[c];
    S.nnz_lower = off[nchunks];
    S.a_dest.resize(static_cast<size_t>(S.nnz_lower + nr));
    S.a_src.resize(static_cast<size_t>(S.nnz_lower));
    run_threads(nchunks, [&](int c) {
      int64_t q = off[c];
      for (int64_t gi = n * c / nchunks; gi < n * (c + 1) / nchunks; ++gi) {
        if (gi == ground) continue;
        const int32_t i = row_of(gi);
        for (int64_t p = indptr[gi]; p < indptr[gi + 1]; ++p) {
          const int32_t gj = indices[p];
          if (gj == ground) continue;
          const int32_t j = row_of(gj);
          if (i <= j) continue;   // lower entry (row i > column j)
          const int32_t s = S.col2sn[j];
          const int64_t N = sn_nc(S, s) + S.nb[s];
          const int64_t lr = local_row(s, i);
          if (lr < 0) { bad[c] = 1; return; }
          S.a_dest[q] = S.panel_off[s] + static_cast<int64_t>(j - S.first[s]) * N + lr;
          S.a_src[q] = p;
          ++q;
        }
      }
    });
    for (int c = 0; c < nchunks; ++c)
      if (bad[c]) {
        err = "internal: matrix entry outside the supernode structure";
        return PEERS_EINVAL;
      }
    chunked(nr, [&](int64_t k0, int64_t k1) {
      for (int64_t k = k0; k < k1; ++k) {
        const int32_t s = S.col2sn[k];
        const int64_t N = sn_nc(S, s) + S.nb[s];
        const int64_t c = k - S.first[s];
        S.a_dest[S.nnz_lower + k] = S.panel_off[s] + c * N + c;
      }
    });
  }

  // ---- lanes: independent subtrees on separate CUDA streams ----
  // The supernodes at the first depth that has at least 2 kLanes of them root disjoint
  // subtrees; these are dealt to kLanes lanes, largest first (by N^2 n_c, the order of their
  // dense work), to the least loaded lane.  The factorization and the selected inversion run
  // each lane on its own stream, so that launches of different subtrees overlap and fill each
  // other's partial last waves; the supernodes above the cut (lane -1) run on the context's
  // stream.  A lane's arithmetic is that of the one-stream schedule, in the same order.
  S.depth.assign(static_cast<size_t>(ns), 0);
  for (int32_t s = ns - 1; s >= 0; --s)
    S.depth[s] = S.parent[s] == -1 ? 0 : S.depth[S.parent[s]] + 1;
  S.lane_of.assign(static_cast<size_t>(ns), -1);
  S.nlanes = 0;
  {
    int32_t maxd = 0;
    for (int32_t s = 0; s < ns; ++s) maxd = std::max(maxd, S.depth[s]);
    std::vector<int32_t> per_depth(static_cast<size_t>(maxd) + 1, 0);
    for (int32_t s = 0; s < ns; ++s) per_depth[S.depth[s]]++;
    int32_t cut = -1;
    for (int32_t d = 0; d <= maxd && cut < 0 && opt.one_stream == 0; ++d)
      if (per_depth[d] >= 2 * kLanes) cut = d;
    if (cut > 0) {
      std::vector<double> work(static_cast<size_t>(ns), 0.0);
      for (int32_t s = 0; s < ns; ++s) {
        const double nc = sn_nc(S, s), N = nc + S.nb[s];
        work[s] += N * N * nc;
        if (S.parent[s] != -1) work[S.parent[s]] += work[s];   // children precede parents
      }
      std::vector<int32_t> roots;
      for (int32_t s = 0; s < ns; ++s)
        if (S.depth[s] == cut) roots.push_back(s);
      std::stable_sort(roots.begin(), roots.end(),
                       [&](int32_t x, int32_t y) { return work[x] > work[y]; });
      std::vector<double> load(kLanes, 0.0);
      std::vector<int32_t> lane_root(static_cast<size_t>(ns), -1);
      for (int32_t r : roots) {
        const int32_t L = static_cast<int32_t>(std::min_element(load.begin(), load.end()) -
                                               load.begin());
        load[L] += work[r];
        lane_root[r] = L;
      }
      // every supernode below the cut follows its depth-`cut` ancestor (parents come later
      // in postorder, so walk from the top down)
      for (int32_t s = ns - 1; s >= 0; --s) {
        if (S.depth[s] == cut) S.lane_of[s] = lane_root[s];
        else if (S.depth[s] > cut) S.lane_of[s] = S.lane_of[S.parent[s]];
      }
      S.nlanes = kLanes;
    }
  }

  // ---- factorization schedule ----
  // Groups of supernodes of one level and one lane, in issue order: every level of every lane
  // (lanes interleaved level by level), then the levels of the top part.  In a group, small
  // one-block supernodes are factored whole by one CTA each; the rest by the blocked kernels,
  // column block by column block, widest first.
  S.fgroups.clear();
  S.fuse_sn.clear();
  S.fac_sn.clear();
  S.trail_off.clear();
  S.trail_na.clear();
  S.trail_ts.clear();
  S.trail_prefix.clear();
  S.split_off.clear();
  S.next_na.clear();
  S.pr_ts.clear();
  S.up_ts.clear();
  S.ea_off.clear();
  S.ea_pairs.clear();
  auto add_group = [&](int32_t lane, int32_t l) {
    FactorGroup G{};
    G.lane = lane;
    G.level = l;
    G.fuse_b = static_cast<int32_t>(S.fuse_sn.size());
    G.fac_b = static_cast<int32_t>(S.fac_sn.size());
    for (int32_t i = S.level_ptr[l]; i < S.level_ptr[l + 1]; ++i) {
      const int32_t s = S.level_sn[i];
      if (S.lane_of[s] != lane) continue;
      if (sn_nc(S, s) <= kBlock && sn_nc(S, s) + S.nb[s] <= kFactorFuseN)
        S.fuse_sn.push_back(s);
      else
        S.fac_sn.push_back(s);
    }
    G.fuse_e = static_cast<int32_t>(S.fuse_sn.size());
    G.fac_e = static_cast<int32_t>(S.fac_sn.size());
    if (G.fuse_e == G.fuse_b && G.fac_e == G.fac_b) return;
    const int32_t *ls = S.fac_sn.data() + G.fac_b;
    const int32_t cnt = G.fac_e - G.fac_b;
    G.nblocks = cnt > 0 ? (sn_nc(S, ls[0]) + kBlock - 1) / kBlock : 0;
    // groups of several column blocks: each block's update is split so that the next block's
    // chain (diagonal block, panel rows, next columns) does not wait for the bulk of it
    G.split = G.nblocks >= 2;
    G.trail_base = static_cast<int64_t>(S.trail_na.size());
    for (int32_t J = 0; J < G.nblocks; ++J) {
      int32_t na = 0;
      while (na < cnt && sn_nc(S, ls[na]) > J * kBlock) ++na;
      // tiles of one supernode's part of the update: the triangle of columns (and rows) from
      // `lo`, or (rect) the columns [lo, nc) over the rows from lo
      auto part_tiles = [&](int32_t i, int64_t lo, int64_t ts, bool rect) -> int64_t {
        const int64_t nc = sn_nc(S, ls[i]), N = nc + S.nb[ls[i]];
        const int64_t T = (N - lo + ts - 1) / ts;
        if (!rect) return T * (T + 1) / 2;
        const int64_t Tc = (nc - lo + ts - 1) / ts;
        return Tc * T - Tc * (Tc - 1) / 2;
      };
      auto t0_of = [&](int32_t i) { return std::min<int64_t>(sn_nc(S, ls[i]), (J + 1) * kBlock); };
      auto t1_of = [&](int32_t i) { return std::min<int64_t>(sn_nc(S, ls[i]), (J + 2) * kBlock); };
      auto nc_of = [&](int32_t i) { return static_cast<int64_t>(sn_nc(S, ls[i])); };
      // tiles of 64, or of 32 when 64-tiles would not give every SM a few of them
      auto pick_ts = [&](auto lo_of, bool rect) -> int64_t {
        int64_t acc = 0;
        for (int32_t i = 0; i < na; ++i) acc += part_tiles(i, lo_of(i), kTile, rect);
        return acc < kTrailFewTiles ? kTile / 2 : kTile;
      };
      auto push_prefix = [&](int32_t cnt_sn, auto lo_of, int64_t ts, bool rect) {
        int64_t acc = 0;
        S.trail_prefix.push_back(0);
        for (int32_t i = 0; i < cnt_sn; ++i) {
          acc += part_tiles(i, lo_of(i), ts, rect);
          S.trail_prefix.push_back(acc);
        }
      };
      const int64_t ts = pick_ts(t0_of, false);
      S.trail_off.push_back(static_cast<int64_t>(S.trail_prefix.size()));
      S.trail_na.push_back(na);
      S.trail_ts.push_back(static_cast<int32_t>(ts));
      push_prefix(na, t0_of, ts, false);
      if (G.split) {
        // next: one column of tiles per supernode that has a block J + 1
        int32_t nn = 0;
        while (nn < na && sn_nc(S, ls[nn]) > (J + 1) * kBlock) ++nn;
        S.split_off.push_back(static_cast<int64_t>(S.trail_prefix.size()));
        S.next_na.push_back(nn);
        int64_t acc = 0;
        S.trail_prefix.push_back(0);
        for (int32_t i = 0; i < nn; ++i) {
          const int64_t N = nc_of(i) + S.nb[ls[i]];
          acc += (N - t0_of(i) + kTile / 2 - 1) / (kTile / 2);
          S.trail_prefix.push_back(acc);
        }
        const int64_t pts = pick_ts(t1_of, true);
        S.pr_ts.push_back(static_cast<int32_t>(pts));
        push_prefix(na, t1_of, pts, true);
        const int64_t uts = pick_ts(nc_of, false);
        S.up_ts.push_back(static_cast<int32_t>(uts));
        push_prefix(na, nc_of, uts, false);
      } else {
        S.split_off.push_back(-1);
        S.next_na.push_back(0);
        S.pr_ts.push_back(0);
        S.up_ts.push_back(0);
      }
    }
    // extend-add of the blocked supernodes' children, one launch per child rank (the
    // supernodes factored whole add their children's update matrices themselves)
    int32_t maxc = 0;
    for (int32_t i = 0; i < cnt; ++i)
      maxc = std::max(maxc, S.child_ptr[ls[i] + 1] - S.child_ptr[ls[i]]);
    G.ea_b = static_cast<int64_t>(S.ea_off.size());
    for (int32_t r = 0; r < maxc; ++r) {
      S.ea_off.push_back(static_cast<int64_t>(S.ea_pairs.size() / 2));
      for (int32_t i = 0; i < cnt; ++i) {
        const int32_t s = ls[i];
        if (S.child_ptr[s] + r < S.child_ptr[s + 1]) {
          S.ea_pairs.push_back(s);
          S.ea_pairs.push_back(S.child_list[S.child_ptr[s] + r]);
        }
      }
    }
    G.ea_e = static_cast<int64_t>(S.ea_off.size());
    S.fgroups.push_back(G);
  };
  for (int32_t l = 0; l < S.nlevels; ++l)
    for (int32_t L = 0; L < S.nlanes; ++L) add_group(L, l);
  for (int32_t l = 0; l < S.nlevels; ++l) add_group(-1, l);
  S.ea_off.push_back(static_cast<int64_t>(S.ea_pairs.size() / 2));
  S.t_symbolic = since(t1);
  auto t2 = Clock::now();

  // ---- queries (§III-G: each query mapped to permuted endpoints, grouped by start) ----
  std::vector<int32_t, NoInitAlloc<int32_t>> eu, ev;
  const int32_t *QU = qu, *QV = qv;
  if (nq < 0 || !qu || !qv) {
    // all edges, u ascending then CSR order: each row chunk counts its edges (u < v), then
    // writes them from its prefix offset
    const int nt = n >= (int64_t(1) << 18) ? plan_threads() : 1;
    std::vector<int64_t> at(static_cast<size_t>(nt) + 1, 0);
    auto row_edges = [&](int c, auto &&put) {
      for (int64_t u = n * c / nt, u1 = n * (c + 1) / nt; u < u1; ++u)
        for (int64_t p = indptr[u]; p < indptr[u + 1]; ++p)
          if (indices[p] > u) put(u, indices[p]);
    };
    run_threads(nt, [&](int c) {
      int64_t k = 0;
      row_edges(c, [&](int64_t, int32_t) { ++k; });
      at[c + 1] = k;
    });
    for (int c = 0; c < nt; ++c) at[c + 1] += at[c];
    eu.resize(static_cast<size_t>(at[nt]));
    ev.resize(static_cast<size_t>(at[nt]));
    run_threads(nt, [&](int c) {
      int64_t k = at[c];
      row_edges(c, [&](int64_t u, int32_t v) {
        eu[k] = static_cast<int32_t>(u);
        ev[k++] = v;
      });
    });
    nq = at[nt];
    QU = eu.data();
    QV = ev.data();
  }
  S.nq = nq;
  struct Rec { int32_t s0, a, b; int64_t idx; };
  struct Two { int32_t lo, hi; int64_t idx; };
  auto pos = [&](int64_t u) -> int32_t {
    return u == ground ? -1 : iperm[u > ground ? u - 1 : u];
  };
  // Queries are mapped in contiguous chunks, one per host thread; each chunk keeps its records
  // in query order and counts them per start supernode.
  struct Chunk {
    std::vector<Rec> recs;
    std::vector<Two> twos;
    std::vector<int64_t> at;   // per start supernode: its count, then its first output slot
    int64_t trivial = 0;
    bool bad = false;
  };
  const int nchunks = nq >= (int64_t(1) << 16) ? plan_threads() : 1;
  std::vector<Chunk> chunks(static_cast<size_t>(nchunks));
  run_threads(nchunks, [&](int c) {
    Chunk &C = chunks[c];
    const int64_t i0 = nq * c / nchunks, i1 = nq * (c + 1) / nchunks;
    C.recs.reserve(static_cast<size_t>(i1 - i0));
    for (int64_t i = i0; i < i1; ++i) {
      const int64_t u = QU[i], v = QV[i];
      if (u < 0 || u >= n || v < 0 || v >= n) { C.bad = true; return; }
      if (u == v) { C.trivial++; continue; }
      int32_t pu = pos(u), pv = pos(v), lo, hi;
      if (pu < 0 || pv < 0) { lo = std::max(pu, pv); hi = -1; }
      else { lo = std::min(pu, pv); hi = std::max(pu, pv); }
      const int32_t s0 = S.col2sn[lo];
      const int32_t f = S.first[s0], nc = sn_nc(S, s0);
      int32_t b = -1;
      if (hi >= 0) {
        if (hi < f + nc) {
          b = hi - f;
        } else {
          auto rb = S.rows.begin() + S.rows_off[s0], re = S.rows.begin() + S.rows_off[s0 + 1];
          auto it = std::lower_bound(rb, re, hi);
          if (it == re || *it != hi) {   // paths meet above s0: two-branch walk
            C.twos.push_back({lo, hi, i});
            continue;
          }
          b = nc + static_cast<int32_t>(it - rb);
        }
      }
      C.recs.push_back({s0, lo - f, b, i});
    }
    C.at.assign(static_cast<size_t>(ns), 0);
    for (const Rec &r : C.recs) C.at[r.s0]++;
  });
  S.nq_trivial = 0;
  std::vector<Two> twos;
  for (const Chunk &C : chunks) {
    if (C.bad) { err = "query node out of range"; return PEERS_EINVAL; }
    S.nq_trivial += C.trivial;
    twos.insert(twos.end(), C.twos.begin(), C.twos.end());
  }
  S.nq_two = static_cast<int64_t>(twos.size());
  // ordered by (start supernode, a, b, query index): the chunks scatter their records into
  // groups by start supernode, then each group is sorted on its own (the order is total, so
  // this is the order one sort of all records gives)
  S.qbeg.assign(static_cast<size_t>(ns) + 1, 0);
  for (int32_t s = 0; s < ns; ++s) {
    int64_t next = S.qbeg[s];
    for (Chunk &C : chunks) {
      const int64_t k = C.at[s];
      C.at[s] = next;
      next += k;
    }
    S.qbeg[s + 1] = next;
  }
  std::vector<Rec, NoInitAlloc<Rec>> recs(static_cast<size_t>(S.qbeg[ns]));
  run_threads(nchunks, [&](int c) {
    Chunk &C = chunks[c];
    for (const Rec &r : C.recs) recs[C.at[r.s0]++] = r;
    std::vector<Rec>().swap(C.recs);
  });
  run_threads(nchunks, [&](int c) {
    // supernodes [s_begin, s_end) hold about a 1/nchunks share of the records
    auto first_at = [&](int k) -> int32_t {
      if (k == nchunks) return ns;
      const int64_t goal = S.qbeg[ns] * k / nchunks;
      return static_cast<int32_t>(std::lower_bound(S.qbeg.begin(), S.qbeg.end(), goal) -
                                  S.qbeg.begin());
    };
    const int32_t s_begin = std::min(first_at(c), ns), s_end = std::min(first_at(c + 1), ns);
    for (int32_t s = s_begin; s < s_end; ++s)
      std::sort(recs.begin() + S.qbeg[s], recs.begin() + S.qbeg[s + 1],
                [](const Rec &x, const Rec &y) {
                  if (x.a != y.a) return x.a < y.a;
                  if (x.b != y.b) return x.b < y.b;
                  return x.idx < y.idx;
                });
  });
  S.nsorted = static_cast<int64_t>(recs.size());
  const int64_t nslots = S.nsorted + 2 * S.nq_two;
  S.qorig.resize(static_cast<size_t>(nslots));
  S.qa.resize(static_cast<size_t>(nslots));
  S.qb.resize(static_cast<size_t>(nslots));
  chunked(static_cast<int64_t>(recs.size()), [&](int64_t k0, int64_t k1) {
    for (int64_t k = k0; k < k1; ++k) {
      S.qorig[k] = recs[k].idx;
      S.qa[k] = recs[k].a;
      S.qb[k] = recs[k].b;
    }
  });

  S.two_lo.resize(twos.size());
  S.two_hi.resize(twos.size());
  S.two_idx.resize(twos.size());
  for (size_t k = 0; k < twos.size(); ++k) {
    S.two_lo[k] = twos[k].lo;
    S.two_hi[k] = twos[k].hi;
    S.two_idx[k] = twos[k].idx;
  }
  S.carry_budget = opt.carry_budget > 0 ? opt.carry_budget : (int64_t(48) << 30);
  if (opt.front_smem > 0) S.front_budget = S.front_limit = std::min(opt.front_smem, kMaxSmem);
  S.one_stream = opt.one_stream != 0;
  int32_t caps[kSizeClasses];
  for (int c = 0; c < kSizeClasses; ++c) caps[c] = opt.qcap[c];
  st = build_sweep_plan(S, caps, err);
  if (st != PEERS_OK) return st;
  S.t_queries = since(t2);
  return PEERS_OK;
}

}  // namespace peers
