/*
 * lmf_oracle.c -- CPU oracle for batches of group-by aggregates over a natural join.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this file; the GPU library never links or calls it and
 * shares no code with it.
 *
 * What it computes is the plain definition of the problem statement (Sec. 1.1
 * and Eq. query of Sec. 2):
 *
 *   SELECT F_1..F_f, SUM(alpha_1), ..., SUM(alpha_l)
 *   FROM R_1 NATURAL JOIN ... NATURAL JOIN R_m  GROUP BY F_1..F_f
 *
 * with each alpha a product of factors: a power x^p of an attribute, or a
 * threshold indicator 1[x <= t] / 1[x > t] (the Kronecker deltas of Sec. 1.1;
 * the two operators follow the inlined code of App. C, "<=" and ">").
 *
 * Method, kept deliberately naive:
 *   1. The natural join is enumerated tuple by tuple.  Each non-root relation is
 *      joined to its parent in the join tree on *all* attributes the two share
 *      (Sec. 3.1: by the running-intersection property this is the natural join
 *      of all relations).  Matching child rows are found through a sorted index
 *      on the declared key attribute; remaining shared attributes are checked
 *      row by row.  The join is streamed, never stored.
 *   2. For every joined tuple and every aggregate, the product of the factors
 *      is evaluated literally and added to the cell of the tuple's group.
 *   3. Sums are kept in double precision with Neumaier compensation; products
 *      of indicators only (counts) are kept as exact int64.  Alongside every
 *      sum the oracle also keeps SUM(|value|), the scale used by the tests'
 *      error rule.
 *
 * Threads (OpenMP, optional): contiguous blocks of root rows, one private set of
 * accumulators per thread, combined in thread order, so a fixed thread count
 * gives bit-identical results.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_I32 = 0, ORC_F32 = 1, ORC_F64 = 2 };
enum { ORC_POW = 0, ORC_LE = 1, ORC_GT = 2 };

typedef struct {
  int64_t nrows;
  int32_t ncols;
  const int32_t* dtypes;       /* ORC_I32 / ORC_F32 / ORC_F64 per column */
  const void* const* data;     /* column arrays */
} orc_relation;

typedef struct {
  int32_t parent, child;       /* relation indices */
  int32_t n_eq;                /* attributes shared by parent and child */
  const int32_t* parent_cols;  /* [0] is the indexed key, int32 on both sides */
  const int32_t* child_cols;
} orc_edge;

typedef struct {
  int32_t n_group_by;
  const int32_t* gb_rel;
  const int32_t* gb_col;
  const int32_t* gb_dom;       /* values must lie in [0, dom) */
  int32_t n_factors;
  const int32_t* f_rel;
  const int32_t* f_col;
  const int32_t* f_kind;       /* ORC_POW / ORC_LE / ORC_GT */
  const int32_t* f_pow;        /* power for ORC_POW */
  const double* f_thr;         /* threshold for ORC_LE / ORC_GT */
  int32_t is_count;            /* 1 when no factor is a power: an exact count */
  int64_t offset;              /* first cell in the count or the sum arrays */
} orc_agg;

/* --------------------------------------------------------------------------- */
typedef struct {
  int32_t* keys;   /* sorted key values */
  int64_t* rows;   /* row id of each sorted entry */
  int64_t n;
} key_index;

static const orc_relation* g_sort_rel;
static int32_t g_sort_col;

static int cmp_rows(const void* a, const void* b) {
  const int32_t* k = (const int32_t*)g_sort_rel->data[g_sort_col];
  int64_t ra = *(const int64_t*)a, rb = *(const int64_t*)b;
  if (k[ra] != k[rb]) return k[ra] < k[rb] ? -1 : 1;
  return ra < rb ? -1 : (ra > rb);
}

static int build_index(const orc_relation* rel, int32_t col, key_index* ix) {
  ix->n = rel->nrows;
  ix->rows = (int64_t*)malloc(sizeof(int64_t) * (size_t)(rel->nrows + 1));
  ix->keys = (int32_t*)malloc(sizeof(int32_t) * (size_t)(rel->nrows + 1));
  if (!ix->rows || !ix->keys) return -1;
  for (int64_t i = 0; i < rel->nrows; ++i) ix->rows[i] = i;
  g_sort_rel = rel;
  g_sort_col = col;
  qsort(ix->rows, (size_t)rel->nrows, sizeof(int64_t), cmp_rows);
  const int32_t* k = (const int32_t*)rel->data[col];
  for (int64_t i = 0; i < rel->nrows; ++i) ix->keys[i] = k[ix->rows[i]];
  return 0;
}

/* first position with keys[pos] >= v */
static int64_t lower_bound(const key_index* ix, int32_t v) {
  int64_t lo = 0, hi = ix->n;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (ix->keys[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

static double value_at(const orc_relation* rel, int32_t col, int64_t row) {
  switch (rel->dtypes[col]) {
    case ORC_I32: return (double)((const int32_t*)rel->data[col])[row];
    case ORC_F32: return (double)((const float*)rel->data[col])[row];
    default: return ((const double*)rel->data[col])[row];
  }
}

/* --------------------------------------------------------------------------- */
typedef struct {
  double* sum;
  double* comp;
  double* abs;
  int64_t* cnt;
  int64_t join_size;
  int error;
} accum;

typedef struct {
  int nrel;
  const orc_relation* rels;
  const int32_t* order;        /* relations, parents before children */
  const int32_t* edge_of;      /* edge index of each non-root relation */
  const orc_edge* edges;
  const key_index* index;      /* per relation (non-root) */
  int nagg;
  const orc_agg* aggs;
} problem;

static void neumaier_add(double* s, double* c, double v) {
  double t = *s + v;
  if (fabs(*s) >= fabs(v)) *c += (*s - t) + v;
  else *c += (v - t) + *s;
  *s = t;
}

/* one joined tuple: cur[r] is the row of relation r */
static void emit(const problem* P, const int64_t* cur, accum* A) {
  A->join_size += 1;
  for (int a = 0; a < P->nagg; ++a) {
    const orc_agg* g = &P->aggs[a];
    double v = 1.0;
    int zero = 0;
    for (int f = 0; f < g->n_factors && !zero; ++f) {
      double x = value_at(&P->rels[g->f_rel[f]], g->f_col[f], cur[g->f_rel[f]]);
      if (g->f_kind[f] == ORC_POW) {
        double p = 1.0;
        for (int e = 0; e < g->f_pow[f]; ++e) p *= x;
        v *= p;
      } else if (g->f_kind[f] == ORC_LE) {
        if (!(x <= g->f_thr[f])) zero = 1;
      } else {
        if (!(x > g->f_thr[f])) zero = 1;
      }
    }
    if (zero) continue;
    int64_t cell = 0;
    for (int k = 0; k < g->n_group_by; ++k) {
      double xv = value_at(&P->rels[g->gb_rel[k]], g->gb_col[k], cur[g->gb_rel[k]]);
      int64_t iv = (int64_t)xv;
      if (xv != (double)iv || iv < 0 || iv >= g->gb_dom[k]) { A->error = 1; return; }
      cell = cell * g->gb_dom[k] + iv;
    }
    if (g->is_count) {
      A->cnt[g->offset + cell] += 1;
    } else {
      neumaier_add(&A->sum[g->offset + cell], &A->comp[g->offset + cell], v);
      A->abs[g->offset + cell] += fabs(v);
    }
  }
}

/* extend the partial tuple with the relation at position pos of the order */
static void extend(const problem* P, int pos, int64_t* cur, accum* A) {
  if (A->error) return;
  if (pos == P->nrel) { emit(P, cur, A); return; }
  int32_t r = P->order[pos];
  const orc_edge* e = &P->edges[P->edge_of[r]];
  const orc_relation* pr = &P->rels[e->parent];
  const orc_relation* cr = &P->rels[r];
  int32_t key = ((const int32_t*)pr->data[e->parent_cols[0]])[cur[e->parent]];
  const key_index* ix = &P->index[r];
  for (int64_t i = lower_bound(ix, key); i < ix->n && ix->keys[i] == key; ++i) {
    int64_t row = ix->rows[i];
    int ok = 1;
    for (int q = 1; q < e->n_eq && ok; ++q)
      ok = value_at(pr, e->parent_cols[q], cur[e->parent]) ==
           value_at(cr, e->child_cols[q], row);
    if (!ok) continue;
    cur[r] = row;
    extend(P, pos + 1, cur, A);
  }
}

/*
 * Evaluate the batch over the joined tuples that extend root rows
 * [root_begin, root_end).  Outputs are overwritten:
 *   out_sum/out_abs: n_sum_cells doubles (sum-type aggregates),
 *   out_cnt:         n_cnt_cells int64   (count-type aggregates),
 *   *out_join_size:  number of joined tuples enumerated.
 * Returns 0, -1 on a bad argument / allocation failure, -2 when a group-by
 * value is not an integer in [0, dom).
 */
int orc_evaluate(int nrel, const orc_relation* rels, int root, int nedge,
                 const orc_edge* edges, int nagg, const orc_agg* aggs,
                 int64_t n_sum_cells, int64_t n_cnt_cells,
                 int64_t root_begin, int64_t root_end, int nthreads,
                 double* out_sum, double* out_abs, int64_t* out_cnt,
                 int64_t* out_join_size) {
  if (nrel <= 0 || root < 0 || root >= nrel || nedge != nrel - 1) return -1;
  int32_t* order = (int32_t*)calloc((size_t)nrel, sizeof(int32_t));
  int32_t* edge_of = (int32_t*)calloc((size_t)nrel, sizeof(int32_t));
  key_index* index = (key_index*)calloc((size_t)nrel, sizeof(key_index));
  if (!order || !edge_of || !index) return -1;
  for (int r = 0; r < nrel; ++r) edge_of[r] = -1;
  for (int e = 0; e < nedge; ++e) {
    if (edges[e].child < 0 || edges[e].child >= nrel || edge_of[edges[e].child] != -1) return -1;
    edge_of[edges[e].child] = e;
  }
  /* breadth-first order from the root: every parent precedes its children */
  int head = 0, tail = 0;
  order[tail++] = root;
  while (head < tail) {
    int32_t p = order[head++];
    for (int e = 0; e < nedge; ++e)
      if (edges[e].parent == p) order[tail++] = edges[e].child;
  }
  if (tail != nrel) return -1;
  for (int r = 0; r < nrel; ++r)
    if (r != root && build_index(&rels[r], edges[edge_of[r]].child_cols[0], &index[r]) != 0)
      return -1;

  /* position 0 of the order is the root, handled by the row loop below */
  problem P = {nrel, rels, order, edge_of, edges, index, nagg, aggs};

  if (root_begin < 0) root_begin = 0;
  if (root_end > rels[root].nrows) root_end = rels[root].nrows;
  int nt = nthreads > 0 ? nthreads : 1;
#ifndef _OPENMP
  nt = 1;
#endif
  accum* acc = (accum*)calloc((size_t)nt, sizeof(accum));
  if (!acc) return -1;
  for (int t = 0; t < nt; ++t) {
    acc[t].sum = (double*)calloc((size_t)(n_sum_cells + 1), sizeof(double));
    acc[t].comp = (double*)calloc((size_t)(n_sum_cells + 1), sizeof(double));
    acc[t].abs = (double*)calloc((size_t)(n_sum_cells + 1), sizeof(double));
    acc[t].cnt = (int64_t*)calloc((size_t)(n_cnt_cells + 1), sizeof(int64_t));
    if (!acc[t].sum || !acc[t].comp || !acc[t].abs || !acc[t].cnt) return -1;
  }
  int64_t total = root_end > root_begin ? root_end - root_begin : 0;

#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
  {
    int t = 0;
#ifdef _OPENMP
    t = omp_get_thread_num();
#endif
    int64_t b = root_begin + total * t / nt, e = root_begin + total * (t + 1) / nt;
    int64_t* cur = (int64_t*)calloc((size_t)nrel, sizeof(int64_t));
    for (int64_t r = b; r < e && cur; ++r) {
      cur[root] = r;
      extend(&P, 1, cur, &acc[t]);
      if (acc[t].error) break;
    }
    free(cur);
  }

  int err = 0;
  for (int64_t i = 0; i < n_sum_cells; ++i) {
    double s = 0.0, c = 0.0, ab = 0.0;
    for (int t = 0; t < nt; ++t) {
      neumaier_add(&s, &c, acc[t].sum[i]);
      neumaier_add(&s, &c, acc[t].comp[i]);
      ab += acc[t].abs[i];
    }
    out_sum[i] = s + c;
    out_abs[i] = ab;
  }
  for (int64_t i = 0; i < n_cnt_cells; ++i) {
    int64_t s = 0;
    for (int t = 0; t < nt; ++t) s += acc[t].cnt[i];
    out_cnt[i] = s;
  }
  int64_t js = 0;
  for (int t = 0; t < nt; ++t) {
    js += acc[t].join_size;
    err |= acc[t].error;
    free(acc[t].sum); free(acc[t].comp); free(acc[t].abs); free(acc[t].cnt);
  }
  *out_join_size = js;
  free(acc);
  for (int r = 0; r < nrel; ++r) { free(index[r].keys); free(index[r].rows); }
  free(index); free(order); free(edge_of);
  return err ? -2 : 0;
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
