/*
 * CPU oracle for exact effective resistance.  TEST INFRASTRUCTURE ONLY: it is called by the
 * tests, by the bench's CPU-baseline leg and by the package smoke check, never by the
 * library's compute path, and it shares no code with the CUDA library.
 *
 * What it computes (PEERS, §II-A eq. 1-4 and §IV-A eq. 15-18):
 *   L_G = D - W is the graph Laplacian (eq. 1).  Grounding node g and deleting its row and
 *   column gives the SPD reduced Laplacian L_r.  The effective resistance of a pair (s,t)
 *   is R_st = (e_s - e_t)^T L_r^{-1} (e_s - e_t) (eq. 2 / eq. 15); when one endpoint is g its
 *   unit vector is dropped (eq. 4).  With L_r = L D L^T (unit lower L; the paper writes the
 *   equivalent L L^T form, eq. 3 and eq. 16) and L y = e_s - e_t, R_st = sum_k y_k^2 / d_k
 *   (eq. 17-18 with the diagonal scaling moved into D).
 *
 * How (each step plain and unblocked):
 *   1. an ordering of the oracle's own: coordinate nested dissection when coordinates are
 *      given (separators of §II-D, Def. 1), reverse Cuthill-McKee otherwise;
 *   2. elimination tree of the permuted L_r (Liu's path-compression algorithm);
 *   3. simplicial up-looking LDL^T: row k of L comes from one sparse unit-lower solve whose
 *      pattern is the union of etree paths from the row's non-zeros (Lemma 1's structure);
 *   4. per query, a sparse forward solve L y = b over the union of the etree paths of the two
 *      endpoints (the reach of b, as in the paper's LSolve, Alg. 2), then sum_k y_k^2/d_k in
 *      increasing k;
 *   5. a "full solve" mode: x = L_r^{-1} b by forward, diagonal and backward substitution over
 *      all n columns, R = b^T x, plus the residual ||L_r x - b||_inf against the unfactored
 *      matrix (checks the factor itself, not only the sum identity).
 * Queries run on POSIX threads, each with its own dense work vector.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_ENOTSPD (-3)

typedef struct oracle_factor {
  int64_t n;          /* reduced size (graph nodes minus the ground) */
  int32_t ground;     /* grounded graph node */
  int64_t n_graph;
  int32_t *perm;      /* perm[k] = reduced node eliminated k-th */
  int32_t *iperm;     /* iperm[reduced node] = elimination position */
  int32_t *parent;    /* etree parent (-1 = root) in elimination positions */
  int64_t *colp;      /* column pointers of strictly-lower L, by elimination position */
  int32_t *rowi;      /* row indices (ascending within a column) */
  double *val;        /* L values */
  double *d;          /* diagonal of D */
  /* reduced Laplacian in the original reduced numbering, full symmetric CSR */
  int64_t *ap;
  int32_t *ai;
  double *ax;
} oracle_factor;

/* ---------------------------------------------------------------- reduced Laplacian */

/* Builds L_r (eq. 1 with the ground's row and column removed) as symmetric CSR in the
 * reduced numbering r(i) = i - (i > g). */
static int build_reduced(int64_t n, const int64_t *indptr, const int32_t *indices, const double *w,
                         int32_t g, int64_t **ap_o, int32_t **ai_o, double **ax_o) {
  int64_t nr = n - 1;
  int64_t *ap = (int64_t *)calloc((size_t)nr + 1, sizeof(int64_t));
  if (!ap) return ORC_ENOMEM;
  for (int64_t i = 0; i < n; ++i) {
    if (i == g) continue;
    int64_t cnt = 1; /* diagonal */
    for (int64_t p = indptr[i]; p < indptr[i + 1]; ++p)
      if (indices[p] != g) cnt++;
    ap[(i > g ? i - 1 : i) + 1] = cnt;
  }
  for (int64_t i = 0; i < nr; ++i) ap[i + 1] += ap[i];
  int32_t *ai = (int32_t *)malloc(sizeof(int32_t) * (size_t)ap[nr]);
  double *ax = (double *)malloc(sizeof(double) * (size_t)ap[nr]);
  if (!ai || !ax) { free(ap); free(ai); free(ax); return ORC_ENOMEM; }
  for (int64_t i = 0; i < n; ++i) {
    if (i == g) continue;
    int64_t r = i > g ? i - 1 : i;
    int64_t q = ap[r];
    double deg = 0.0;
    for (int64_t p = indptr[i]; p < indptr[i + 1]; ++p) {
      int32_t j = indices[p];
      deg += w[p];                     /* the degree counts the edge to g as well */
      if (j == g) continue;
      ai[q] = j > g ? j - 1 : j;
      ax[q] = -w[p];
      q++;
    }
    ai[q] = (int32_t)r;
    ax[q] = deg;
  }
  *ap_o = ap; *ai_o = ai; *ax_o = ax;
  return ORC_OK;
}

/* ---------------------------------------------------------------- orderings */

/* Selection by plain sort of (coordinate, node) keys. */
typedef struct { double key; int32_t node; } keyed_t;
static int cmp_keyed(const void *a, const void *b) {
  const keyed_t *x = (const keyed_t *)a, *y = (const keyed_t *)b;
  if (x->key < y->key) return -1;
  if (x->key > y->key) return 1;
  return (x->node > y->node) - (x->node < y->node);
}

/* Coordinate nested dissection: split the node set at the median of its widest coordinate
 * axis, take as separator the nodes of the lower side that have a neighbour on the upper side,
 * order [lower minus separator, upper, separator] recursively.  Sets of at most LEAF nodes are
 * emitted as they are. */
#define ND_LEAF 8
static int order_coord_nd(int64_t nr, const int64_t *ap, const int32_t *ai, const double *coords,
                          int dim, int32_t *perm) {
  int32_t *work = (int32_t *)malloc(sizeof(int32_t) * (size_t)nr);
  int32_t *side = (int32_t *)malloc(sizeof(int32_t) * (size_t)nr);
  keyed_t *keys = (keyed_t *)malloc(sizeof(keyed_t) * (size_t)nr);
  /* explicit stack of tasks: (lo, hi, out_end) meaning "order work[lo:hi) into the output
   * positions ending at out_end" -- the output is filled from the back */
  int64_t cap = 1024, top = 0;
  int64_t *stk = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)cap);
  if (!work || !side || !keys || !stk) { free(work); free(side); free(keys); free(stk); return ORC_ENOMEM; }
  for (int64_t i = 0; i < nr; ++i) { work[i] = (int32_t)i; side[i] = -1; }
  stk[0] = 0; stk[1] = nr; stk[2] = nr; top = 1;
  while (top > 0) {
    top--;
    int64_t lo = stk[3 * top], hi = stk[3 * top + 1], out_end = stk[3 * top + 2];
    int64_t cnt = hi - lo;
    if (cnt <= 0) continue;
    if (cnt <= ND_LEAF) {
      for (int64_t i = 0; i < cnt; ++i) perm[out_end - cnt + i] = work[lo + i];
      continue;
    }
    /* widest axis */
    int axis = 0;
    double best = -1.0;
    for (int a = 0; a < dim; ++a) {
      double mn = INFINITY, mx = -INFINITY;
      for (int64_t i = lo; i < hi; ++i) {
        double c = coords[(int64_t)work[i] * dim + a];
        if (c < mn) mn = c;
        if (c > mx) mx = c;
      }
      if (mx - mn > best) { best = mx - mn; axis = a; }
    }
    if (best <= 0.0) {   /* all coincide: emit as a block */
      for (int64_t i = 0; i < cnt; ++i) perm[out_end - cnt + i] = work[lo + i];
      continue;
    }
    for (int64_t i = lo; i < hi; ++i) {
      keys[i - lo].key = coords[(int64_t)work[i] * dim + axis];
      keys[i - lo].node = work[i];
    }
    qsort(keys, (size_t)cnt, sizeof(keyed_t), cmp_keyed);
    double pivot = keys[cnt / 2].key;
    /* lower side: key < pivot (or <= pivot when that leaves it empty) */
    int strict = keys[0].key < pivot;
    for (int64_t i = 0; i < cnt; ++i) {
      int lower = strict ? (keys[i].key < pivot) : (keys[i].key <= pivot);
      side[keys[i].node] = lower ? 0 : 1;
    }
    /* separator: lower nodes adjacent to an upper node */
    int64_t nl = 0, nu = 0, ns = 0;
    for (int64_t i = 0; i < cnt; ++i) {
      int32_t v = keys[i].node;
      if (side[v] == 0) {
        int sep = 0;
        for (int64_t p = ap[v]; p < ap[v + 1]; ++p)
          if (side[ai[p]] == 1) { sep = 1; break; }
        if (sep) side[v] = 2;
      }
    }
    for (int64_t i = 0; i < cnt; ++i) {
      int s = side[keys[i].node];
      if (s == 0) nl++; else if (s == 1) nu++; else ns++;
    }
    if (nu == 0 || nl + ns == 0) {  /* cannot split */
      for (int64_t i = 0; i < cnt; ++i) { perm[out_end - cnt + i] = work[lo + i]; side[work[lo + i]] = -1; }
      continue;
    }
    /* rewrite work[lo:hi) as [lower | upper | separator] in key order */
    int64_t a = lo, b = lo + nl, c = lo + nl + nu;
    for (int64_t i = 0; i < cnt; ++i) {
      int32_t v = keys[i].node;
      int s = side[v];
      if (s == 0) work[a++] = v; else if (s == 1) work[b++] = v; else work[c++] = v;
      side[v] = -1;
    }
    /* separator goes last */
    for (int64_t i = 0; i < ns; ++i) perm[out_end - ns + i] = work[lo + nl + nu + i];
    if (top + 2 > cap) {
      cap *= 2;
      int64_t *ns_ = (int64_t *)realloc(stk, sizeof(int64_t) * 3 * (size_t)cap);
      if (!ns_) { free(work); free(side); free(keys); free(stk); return ORC_ENOMEM; }
      stk = ns_;
    }
    /* upper part ends right before the separator, lower part before the upper part */
    stk[3 * top] = lo + nl; stk[3 * top + 1] = lo + nl + nu; stk[3 * top + 2] = out_end - ns; top++;
    stk[3 * top] = lo; stk[3 * top + 1] = lo + nl; stk[3 * top + 2] = out_end - ns - nu; top++;
  }
  free(work); free(side); free(keys); free(stk);
  return ORC_OK;
}

/* Reverse Cuthill-McKee, component by component, each started from a minimum-degree node. */
static int order_rcm(int64_t nr, const int64_t *ap, const int32_t *ai, int32_t *perm) {
  char *seen = (char *)calloc((size_t)nr, 1);
  int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)nr);
  keyed_t *nb = (keyed_t *)malloc(sizeof(keyed_t) * (size_t)(nr + 1));
  if (!seen || !queue || !nb) { free(seen); free(queue); free(nb); return ORC_ENOMEM; }
  int64_t head = 0, tail = 0;
  for (;;) {
    int64_t start = -1, mindeg = INT64_MAX;
    for (int64_t i = 0; i < nr; ++i)
      if (!seen[i] && ap[i + 1] - ap[i] < mindeg) { mindeg = ap[i + 1] - ap[i]; start = i; }
    if (start < 0) break;
    seen[start] = 1;
    queue[tail++] = (int32_t)start;
    while (head < tail) {
      int32_t v = queue[head++];
      int64_t k = 0;
      for (int64_t p = ap[v]; p < ap[v + 1]; ++p) {
        int32_t u = ai[p];
        if (u == v || seen[u]) continue;
        seen[u] = 1;
        nb[k].key = (double)(ap[u + 1] - ap[u]);
        nb[k].node = u;
        k++;
      }
      qsort(nb, (size_t)k, sizeof(keyed_t), cmp_keyed);
      for (int64_t i = 0; i < k; ++i) queue[tail++] = nb[i].node;
    }
  }
  for (int64_t i = 0; i < nr; ++i) perm[i] = queue[nr - 1 - i];
  free(seen); free(queue); free(nb);
  return ORC_OK;
}

/* ---------------------------------------------------------------- factorization */

/* Row pattern of row k of L: the union of the etree paths from each i < k with
 * A(perm[i], perm[k]) != 0, stopped at k or at a node already marked for row k.  Written into
 * stack[top..k) in an order where every node precedes its etree ancestors.  Returns top. */
static int64_t row_pattern(const oracle_factor *F, int64_t k, int32_t *mark, int32_t *stack,
                           int32_t *path) {
  int64_t top = F->n;  /* stack is filled from the back of an n-sized buffer */
  int32_t vk = F->perm[k];
  mark[k] = (int32_t)k;
  for (int64_t p = F->ap[vk]; p < F->ap[vk + 1]; ++p) {
    int32_t i = F->iperm[F->ai[p]];
    if (i >= k) continue;
    int64_t len = 0;
    while (mark[i] != k) {
      path[len++] = i;
      mark[i] = (int32_t)k;
      i = F->parent[i];
    }
    /* push the path so that its bottom ends up first */
    while (len > 0) stack[--top] = path[--len];
  }
  return top;
}

static int factorize(oracle_factor *F) {
  int64_t n = F->n;
  int32_t *anc = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t *path = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  double *x = (double *)calloc((size_t)n, sizeof(double));
  F->parent = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  F->d = (double *)malloc(sizeof(double) * (size_t)n);
  F->colp = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
  if (!anc || !mark || !stack || !path || !cnt || !x || !F->parent || !F->d || !F->colp) {
    free(anc); free(mark); free(stack); free(path); free(cnt); free(x);
    return ORC_ENOMEM;
  }
  /* elimination tree (Liu): for each column k, climb from every lower-numbered neighbour */
  for (int64_t k = 0; k < n; ++k) {
    F->parent[k] = -1;
    anc[k] = -1;
    int32_t vk = F->perm[k];
    for (int64_t p = F->ap[vk]; p < F->ap[vk + 1]; ++p) {
      int32_t i = F->iperm[F->ai[p]];
      while (i != -1 && i < k) {
        int32_t next = anc[i];
        anc[i] = (int32_t)k;
        if (next == -1) { F->parent[i] = (int32_t)k; break; }
        i = next;
      }
    }
  }
  /* symbolic pass: column counts of L */
  for (int64_t k = 0; k < n; ++k) mark[k] = -1;
  for (int64_t k = 0; k < n; ++k) {
    int64_t top = row_pattern(F, k, mark, stack, path);
    for (int64_t t = top; t < n; ++t) cnt[stack[t]]++;
  }
  F->colp[0] = 0;
  for (int64_t j = 0; j < n; ++j) F->colp[j + 1] = F->colp[j] + cnt[j];
  int64_t nnz = F->colp[n];
  F->rowi = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  F->val = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  if (!F->rowi || !F->val) {
    free(anc); free(mark); free(stack); free(path); free(cnt); free(x);
    return ORC_ENOMEM;
  }
  /* numeric pass, row by row.  For row k: solve L[0:k,0:k] t = A[0:k,k] over the row pattern
   * (t_j = d_j L_kj), then L_kj = t_j / d_j and d_k = A_kk - sum_j L_kj t_j. */
  for (int64_t j = 0; j < n; ++j) cnt[j] = F->colp[j];   /* next free slot per column */
  for (int64_t k = 0; k < n; ++k) mark[k] = -1;
  int status = ORC_OK;
  for (int64_t k = 0; k < n && status == ORC_OK; ++k) {
    int64_t top = row_pattern(F, k, mark, stack, path);
    int32_t vk = F->perm[k];
    double dk = 0.0;
    for (int64_t p = F->ap[vk]; p < F->ap[vk + 1]; ++p) {
      int32_t i = F->iperm[F->ai[p]];
      if (i < k) x[i] = F->ax[p];
      else if (i == k) dk = F->ax[p];
    }
    for (int64_t t = top; t < n; ++t) {
      int32_t j = stack[t];
      double tj = x[j];
      x[j] = 0.0;
      /* t_i -= L_ij t_j for the rows i of column j already computed (all are < k) */
      for (int64_t p = F->colp[j]; p < cnt[j]; ++p) x[F->rowi[p]] -= F->val[p] * tj;
      double lkj = tj / F->d[j];
      dk -= lkj * tj;
      F->rowi[cnt[j]] = (int32_t)k;
      F->val[cnt[j]] = lkj;
      cnt[j]++;
    }
    if (!(dk > 0.0) || !isfinite(dk)) status = ORC_ENOTSPD;
    F->d[k] = dk;
  }
  free(anc); free(mark); free(stack); free(path); free(cnt); free(x);
  return status;
}

void oracle_free(oracle_factor *F) {
  if (!F) return;
  free(F->perm); free(F->iperm); free(F->parent); free(F->colp); free(F->rowi); free(F->val);
  free(F->d); free(F->ap); free(F->ai); free(F->ax);
  free(F);
}

/* Grounds node g of the CSR graph (n nodes, symmetric, weights per stored entry), orders the
 * reduced Laplacian (coordinate ND when coords != NULL, RCM otherwise) and factors it. */
int oracle_factorize(int64_t n, const int64_t *indptr, const int32_t *indices, const double *w,
                     int32_t ground, const double *coords, int dim, oracle_factor **out) {
  *out = NULL;
  if (n < 2 || ground < 0 || ground >= n) return ORC_EINVAL;
  oracle_factor *F = (oracle_factor *)calloc(1, sizeof(oracle_factor));
  if (!F) return ORC_ENOMEM;
  F->n = n - 1;
  F->n_graph = n;
  F->ground = ground;
  int st = build_reduced(n, indptr, indices, w, ground, &F->ap, &F->ai, &F->ax);
  if (st) { oracle_free(F); return st; }
  F->perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)F->n);
  F->iperm = (int32_t *)malloc(sizeof(int32_t) * (size_t)F->n);
  if (!F->perm || !F->iperm) { oracle_free(F); return ORC_ENOMEM; }
  if (coords && dim > 0) {
    /* coordinates of the reduced nodes */
    double *rc = (double *)malloc(sizeof(double) * (size_t)F->n * (size_t)dim);
    if (!rc) { oracle_free(F); return ORC_ENOMEM; }
    for (int64_t i = 0; i < n; ++i) {
      if (i == ground) continue;
      int64_t r = i > ground ? i - 1 : i;
      for (int a = 0; a < dim; ++a) rc[r * dim + a] = coords[i * dim + a];
    }
    st = order_coord_nd(F->n, F->ap, F->ai, rc, dim, F->perm);
    free(rc);
  } else {
    st = order_rcm(F->n, F->ap, F->ai, F->perm);
  }
  if (st) { oracle_free(F); return st; }
  for (int64_t k = 0; k < F->n; ++k) F->iperm[F->perm[k]] = (int32_t)k;
  st = factorize(F);
  if (st) { oracle_free(F); return st; }
  *out = F;
  return ORC_OK;
}

int64_t oracle_nnz_l(const oracle_factor *F) { return F->colp[F->n]; }
int64_t oracle_n(const oracle_factor *F) { return F->n; }

/* elimination position of graph node u, or -1 for the ground */
static int64_t position(const oracle_factor *F, int64_t u) {
  if (u == F->ground) return -1;
  return F->iperm[u > F->ground ? u - 1 : u];
}

/* ---------------------------------------------------------------- per-query path solve */

/* One query by the sparse forward solve over the union of the two etree paths. */
static double resistance_one(const oracle_factor *F, int64_t u, int64_t v, double *y, int32_t *sup) {
  if (u == v) return 0.0;
  int64_t a = position(F, u), b = position(F, v);
  int64_t len = 0;
  /* merge the two ascending etree paths */
  while (a != -1 || b != -1) {
    int64_t next;
    if (b == -1 || (a != -1 && a < b)) { next = a; a = F->parent[a]; }
    else if (a == -1 || b < a) { next = b; b = F->parent[b]; }
    else { next = a; a = F->parent[a]; b = F->parent[b]; }
    sup[len++] = (int32_t)next;
  }
  int64_t pu = position(F, u), pv = position(F, v);
  if (pu >= 0) y[pu] += 1.0;
  if (pv >= 0) y[pv] -= 1.0;
  double r = 0.0;
  for (int64_t t = 0; t < len; ++t) {
    int32_t j = sup[t];
    double yj = y[j];
    for (int64_t p = F->colp[j]; p < F->colp[j + 1]; ++p) y[F->rowi[p]] -= F->val[p] * yj;
    r += yj * yj / F->d[j];
  }
  for (int64_t t = 0; t < len; ++t) y[sup[t]] = 0.0;
  return r;
}

typedef struct {
  const oracle_factor *F;
  int64_t nq;
  const int32_t *qu, *qv;
  double *R;
  int64_t next;           /* shared work counter */
  pthread_mutex_t lock;
  int status;
} job_t;

#define CHUNK 64
static void *worker(void *arg) {
  job_t *J = (job_t *)arg;
  const oracle_factor *F = J->F;
  double *y = (double *)calloc((size_t)F->n, sizeof(double));
  int32_t *sup = (int32_t *)malloc(sizeof(int32_t) * (size_t)F->n);
  if (!y || !sup) {
    pthread_mutex_lock(&J->lock); J->status = ORC_ENOMEM; pthread_mutex_unlock(&J->lock);
    free(y); free(sup);
    return NULL;
  }
  for (;;) {
    pthread_mutex_lock(&J->lock);
    int64_t s = J->next;
    J->next += CHUNK;
    pthread_mutex_unlock(&J->lock);
    if (s >= J->nq) break;
    int64_t e = s + CHUNK < J->nq ? s + CHUNK : J->nq;
    for (int64_t q = s; q < e; ++q) J->R[q] = resistance_one(F, J->qu[q], J->qv[q], y, sup);
  }
  free(y); free(sup);
  return NULL;
}

/* R[q] for the pairs (qu[q], qv[q]) of graph nodes, on `threads` threads (<=0: 1). */
int oracle_resistance(const oracle_factor *F, int64_t nq, const int32_t *qu, const int32_t *qv,
                      int threads, double *R) {
  for (int64_t q = 0; q < nq; ++q)
    if (qu[q] < 0 || qu[q] >= F->n_graph || qv[q] < 0 || qv[q] >= F->n_graph) return ORC_EINVAL;
  if (threads < 1) threads = 1;
  job_t J;
  J.F = F; J.nq = nq; J.qu = qu; J.qv = qv; J.R = R; J.next = 0; J.status = ORC_OK;
  pthread_mutex_init(&J.lock, NULL);
  pthread_t *tid = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
  if (!tid) return ORC_ENOMEM;
  int started = 0;
  for (int t = 1; t < threads; ++t)
    if (pthread_create(&tid[t], NULL, worker, &J) == 0) started = t; else break;
  worker(&J);
  for (int t = 1; t <= started; ++t) pthread_join(tid[t], NULL);
  free(tid);
  pthread_mutex_destroy(&J.lock);
  return J.status;
}

/* ---------------------------------------------------------------- full-solve mode */

/* R = b^T L_r^{-1} b by a dense forward, diagonal and backward solve over all columns, and
 * resid = ||L_r x - b||_inf computed with the unfactored reduced Laplacian. */
int oracle_full_solve(const oracle_factor *F, int64_t u, int64_t v, double *R, double *resid) {
  int64_t n = F->n;
  double *y = (double *)calloc((size_t)n, sizeof(double));
  double *x = (double *)calloc((size_t)n, sizeof(double));
  double *b = (double *)calloc((size_t)n, sizeof(double));
  if (!y || !x || !b) { free(y); free(x); free(b); return ORC_ENOMEM; }
  if (u == v) { *R = 0.0; *resid = 0.0; free(y); free(x); free(b); return ORC_OK; }
  int64_t pu = position(F, u), pv = position(F, v);
  if (pu >= 0) y[pu] += 1.0;
  if (pv >= 0) y[pv] -= 1.0;
  for (int64_t j = 0; j < n; ++j) {          /* L y = P b */
    double yj = y[j];
    if (yj != 0.0)
      for (int64_t p = F->colp[j]; p < F->colp[j + 1]; ++p) y[F->rowi[p]] -= F->val[p] * yj;
  }
  for (int64_t j = 0; j < n; ++j) y[j] /= F->d[j];   /* D z = y */
  for (int64_t j = n - 1; j >= 0; --j) {     /* L^T x = z */
    double s = y[j];
    for (int64_t p = F->colp[j]; p < F->colp[j + 1]; ++p) s -= F->val[p] * y[F->rowi[p]];
    y[j] = s;
  }
  for (int64_t k = 0; k < n; ++k) x[F->perm[k]] = y[k];   /* back to the reduced numbering */
  int64_t ru = u == F->ground ? -1 : (u > F->ground ? u - 1 : u);
  int64_t rv = v == F->ground ? -1 : (v > F->ground ? v - 1 : v);
  if (ru >= 0) b[ru] += 1.0;
  if (rv >= 0) b[rv] -= 1.0;
  double r = 0.0, res = 0.0;
  if (ru >= 0) r += x[ru];
  if (rv >= 0) r -= x[rv];
  for (int64_t i = 0; i < n; ++i) {
    double s = -b[i];
    for (int64_t p = F->ap[i]; p < F->ap[i + 1]; ++p) s += F->ax[p] * x[F->ai[p]];
    if (fabs(s) > res) res = fabs(s);
  }
  *R = r;
  *resid = res;
  free(y); free(x); free(b);
  return ORC_OK;
}

/* Diagonal entries of D and the elimination tree, for structural tests. */
void oracle_export(const oracle_factor *F, double *d_out, int32_t *parent_out, int32_t *perm_out) {
  for (int64_t k = 0; k < F->n; ++k) {
    if (d_out) d_out[k] = F->d[k];
    if (parent_out) parent_out[k] = F->parent[k];
    if (perm_out) perm_out[k] = F->perm[k];
  }
}
