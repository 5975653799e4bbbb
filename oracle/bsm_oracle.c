/*
 * bsm_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct FP64 CPU implementation of the local
 * block-sparse multiply with on-the-fly norm filtering,
 *
 *     C = beta * C_in + alpha * sum_{k kept} A_ik * B_kj ,
 *
 * written from the paper's statement of the problem:
 *   - Sec. 2: matrices are stored as blocked CSR; elements are grouped into
 *     blocks by rows and columns; the result pattern is not fixed in advance but
 *     is determined by the computation, blocks below the threshold being skipped
 *     during the multiplication.
 *   - Sec. 2 (local multiplication): the local multiply is a set of block-wise
 *     small matrix products; a block product is only carried out when the
 *     product of the two block norms passes the threshold (on-the-fly filter).
 *   - Algorithm 1 / Algorithm 2: the operation is C = C + A.B; alpha and beta
 *     generalise it the way BLAS does.
 *   - Table 1: "FLOPs" count 2*m*n*k per block product actually executed
 *     (10 multiplies of a dense 60000^3 problem are 4.320e15 FLOPs).
 *
 * Only tests/, the smoke check and the CPU-baseline leg of the benchmark may
 * load this library. The GPU product path shares no code with it.
 *
 * Readings of points the paper leaves open (each is also a test case):
 *   - norm: Frobenius, accumulated column-major, element by element, each
 *     multiply and add rounded separately (this file is compiled with
 *     -ffp-contract=off), then the correctly rounded sqrt.
 *   - filter: a product (i,k,j) is dropped iff nrm(A_ik)*nrm(B_kj) < eps.
 *     A tie is kept, NaN is kept, eps <= 0 drops nothing.
 *   - alpha does not enter the filter.
 *   - beta == 0: C_in is ignored entirely (pattern and values), as in BLAS.
 *   - block values are column-major; zero-size blocks and duplicate blocks
 *     are errors.
 *   - sums over k run in ascending k, and inside one block product over the
 *     inner index in ascending order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define BSMO_OK 0
#define BSMO_ERR_INVALID_ARG -1
#define BSMO_ERR_DIM_MISMATCH -2
#define BSMO_ERR_DUPLICATE_BLOCK -3
#define BSMO_ERR_OUT_OF_RANGE -4
#define BSMO_ERR_NOMEM -6

typedef struct {
  int32_t nbr;              /* number of block rows */
  int32_t nbc;              /* number of block columns */
  const int32_t *row_sizes; /* [nbr] */
  const int32_t *col_sizes; /* [nbc] */
  int64_t nblk;             /* number of stored blocks */
  const int32_t *blk_row;   /* [nblk] */
  const int32_t *blk_col;   /* [nblk] */
  const double *values;     /* blocks in list order, each column-major */
} bsmo_matrix;

typedef struct {
  int64_t nblk;
  int64_t nnz;
  int32_t *blk_row; /* sorted by (row, col) */
  int32_t *blk_col;
  int64_t *blk_off; /* offset of each block in values */
  double *values;   /* NULL when only the pattern was asked for */
  int64_t candidates;
  int64_t kept;
  int64_t dropped;
  double flops; /* sum over kept products of 2*m*n*k */
} bsmo_result;

/* ------------------------------------------------------------------ */
/* The canonical block norm: Frobenius, column-major, no fused ops.    */
/* ------------------------------------------------------------------ */
double bsmo_block_norm(int32_t r, int32_t c, const double *x) {
  double s = 0.0;
  int64_t n = (int64_t)r * (int64_t)c;
  for (int64_t e = 0; e < n; e++) {
    double sq = x[e] * x[e];
    s = s + sq;
  }
  return sqrt(s);
}

/* ------------------------------------------------------------------ */
/* A row-indexed view of a block list, built by a plain sort.          */
/* ------------------------------------------------------------------ */
typedef struct {
  int32_t nbr, nbc;
  const int32_t *row_sizes, *col_sizes;
  int64_t nblk;
  int64_t *row_start; /* [nbr+1] into order[] */
  int64_t *order;     /* block ids sorted by (row, col) */
  int64_t *off;       /* value offset of block id (list order) */
  const int32_t *blk_row, *blk_col;
  const double *values;
  double *norm; /* canonical norm of block id */
} rowview;

static const int32_t *g_sort_row, *g_sort_col;
static int cmp_int32(const void *pa, const void *pb) {
  int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
  return (a > b) - (a < b);
}
static int cmp_rowcol(const void *pa, const void *pb) {
  int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
  if (g_sort_row[a] != g_sort_row[b]) return g_sort_row[a] < g_sort_row[b] ? -1 : 1;
  if (g_sort_col[a] != g_sort_col[b]) return g_sort_col[a] < g_sort_col[b] ? -1 : 1;
  return 0;
}

static void rowview_free(rowview *v) {
  free(v->row_start);
  free(v->order);
  free(v->off);
  free(v->norm);
  memset(v, 0, sizeof(*v));
}

static int rowview_build(const bsmo_matrix *m, int want_norms, rowview *v) {
  memset(v, 0, sizeof(*v));
  if (!m || m->nbr < 0 || m->nbc < 0 || m->nblk < 0) return BSMO_ERR_INVALID_ARG;
  if ((m->nbr > 0 && !m->row_sizes) || (m->nbc > 0 && !m->col_sizes)) return BSMO_ERR_INVALID_ARG;
  if (m->nblk > 0 && (!m->blk_row || !m->blk_col)) return BSMO_ERR_INVALID_ARG;
  for (int32_t i = 0; i < m->nbr; i++)
    if (m->row_sizes[i] <= 0) return BSMO_ERR_INVALID_ARG;
  for (int32_t j = 0; j < m->nbc; j++)
    if (m->col_sizes[j] <= 0) return BSMO_ERR_INVALID_ARG;
  v->nbr = m->nbr;
  v->nbc = m->nbc;
  v->row_sizes = m->row_sizes;
  v->col_sizes = m->col_sizes;
  v->nblk = m->nblk;
  v->blk_row = m->blk_row;
  v->blk_col = m->blk_col;
  v->values = m->values;
  v->row_start = (int64_t *)calloc((size_t)m->nbr + 1, sizeof(int64_t));
  v->order = (int64_t *)malloc(((size_t)m->nblk + 1) * sizeof(int64_t));
  v->off = (int64_t *)malloc(((size_t)m->nblk + 1) * sizeof(int64_t));
  if (!v->row_start || !v->order || !v->off) {
    rowview_free(v);
    return BSMO_ERR_NOMEM;
  }
  int64_t acc = 0;
  for (int64_t b = 0; b < m->nblk; b++) {
    int32_t i = m->blk_row[b], j = m->blk_col[b];
    if (i < 0 || i >= m->nbr || j < 0 || j >= m->nbc) {
      rowview_free(v);
      return BSMO_ERR_OUT_OF_RANGE;
    }
    v->off[b] = acc;
    acc += (int64_t)m->row_sizes[i] * (int64_t)m->col_sizes[j];
    v->order[b] = b;
  }
  if (m->nblk > 0 && !m->values && want_norms) {
    rowview_free(v);
    return BSMO_ERR_INVALID_ARG;
  }
  g_sort_row = m->blk_row;
  g_sort_col = m->blk_col;
  qsort(v->order, (size_t)m->nblk, sizeof(int64_t), cmp_rowcol);
  for (int64_t p = 1; p < m->nblk; p++) {
    if (cmp_rowcol(&v->order[p - 1], &v->order[p]) == 0) {
      rowview_free(v);
      return BSMO_ERR_DUPLICATE_BLOCK;
    }
  }
  for (int64_t p = 0; p < m->nblk; p++) v->row_start[m->blk_row[v->order[p]] + 1]++;
  for (int32_t i = 0; i < m->nbr; i++) v->row_start[i + 1] += v->row_start[i];
  if (want_norms) {
    v->norm = (double *)malloc(((size_t)m->nblk + 1) * sizeof(double));
    if (!v->norm) {
      rowview_free(v);
      return BSMO_ERR_NOMEM;
    }
    for (int64_t b = 0; b < m->nblk; b++)
      v->norm[b] = bsmo_block_norm(m->row_sizes[m->blk_row[b]], m->col_sizes[m->blk_col[b]],
                                   m->values + v->off[b]);
  }
  return BSMO_OK;
}

/* Find block (i, j) of a row view; returns the block id or -1. */
static int64_t rowview_find(const rowview *v, int32_t i, int32_t j) {
  int64_t lo = v->row_start[i], hi = v->row_start[i + 1];
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    int32_t cj = v->blk_col[v->order[mid]];
    if (cj == j) return v->order[mid];
    if (cj < j) lo = mid + 1;
    else hi = mid;
  }
  return -1;
}

/* The filter test of Sec. 2, with a tie and NaN kept. */
static int keep_product(double na, double nb, double eps) {
  double prod = na * nb;
  return !(prod < eps);
}

static int check_dims(const bsmo_matrix *A, const bsmo_matrix *B, const bsmo_matrix *Cin) {
  if (A->nbc != B->nbr) return BSMO_ERR_DIM_MISMATCH;
  for (int32_t k = 0; k < A->nbc; k++)
    if (A->col_sizes[k] != B->row_sizes[k]) return BSMO_ERR_DIM_MISMATCH;
  if (Cin) {
    if (Cin->nbr != A->nbr || Cin->nbc != B->nbc) return BSMO_ERR_DIM_MISMATCH;
    for (int32_t i = 0; i < A->nbr; i++)
      if (Cin->row_sizes[i] != A->row_sizes[i]) return BSMO_ERR_DIM_MISMATCH;
    for (int32_t j = 0; j < B->nbc; j++)
      if (Cin->col_sizes[j] != B->col_sizes[j]) return BSMO_ERR_DIM_MISMATCH;
  }
  return BSMO_OK;
}

/* Output of one C block row, kept apart so rows can run in any order. */
typedef struct {
  int64_t nblk;
  int32_t *cols;
  double *vals; /* blocks of this row, concatenated, column-major */
  int64_t nnz;
  int64_t candidates, kept, dropped;
  double flops;
  int err;
} rowout;

/*
 * One C block row i, by the definition: walk A's row i in ascending k, and
 * for each A_ik walk B's row k in ascending j (Gustavson's row-wise order).
 * Every (i,k,j) met is a candidate; the filter decides whether it is kept.
 * A kept product is added, element by element over the inner index, into a
 * per-(i,j) sum S_ij, so each S_ij accumulates over ascending k. The block is
 * in the pattern if at least one product was kept or, when beta != 0, if C_in
 * holds it. Finally C_ij = (beta*C_in_ij, or 0) + alpha*S_ij.
 */
static void do_row(const rowview *a, const rowview *b, const rowview *cin, double alpha,
                   double beta, double eps, int pattern_only, int32_t i, int64_t *slot,
                   rowout *out) {
  memset(out, 0, sizeof(*out));
  const int32_t m = a->row_sizes[i];
  const int32_t nbc = b->nbc;
  /* pass 1: the pattern of row i and the statistics */
  int64_t ntouched = 0;
  int32_t *touched = (int32_t *)malloc(((size_t)nbc + 1) * sizeof(int32_t));
  if (!touched) {
    out->err = BSMO_ERR_NOMEM;
    return;
  }
  for (int64_t p = a->row_start[i]; p < a->row_start[i + 1]; p++) {
    int64_t ab = a->order[p];
    int32_t k = a->blk_col[ab];
    for (int64_t q = b->row_start[k]; q < b->row_start[k + 1]; q++) {
      int64_t bb = b->order[q];
      int32_t j = b->blk_col[bb];
      out->candidates++;
      if (keep_product(a->norm[ab], b->norm[bb], eps)) {
        out->kept++;
        out->flops += 2.0 * (double)m * (double)a->col_sizes[k] * (double)b->col_sizes[j];
        if (slot[j] < 0) {
          slot[j] = 0;
          touched[ntouched++] = j;
        }
      } else {
        out->dropped++;
      }
    }
  }
  if (cin && beta != 0.0) {
    for (int64_t p = cin->row_start[i]; p < cin->row_start[i + 1]; p++) {
      int32_t j = cin->blk_col[cin->order[p]];
      if (slot[j] < 0) {
        slot[j] = 0;
        touched[ntouched++] = j;
      }
    }
  }
  /* ascending column order */
  qsort(touched, (size_t)ntouched, sizeof(int32_t), cmp_int32);
  int32_t *cols = (int32_t *)malloc(((size_t)ntouched + 1) * sizeof(int32_t));
  int64_t *coff = (int64_t *)malloc(((size_t)ntouched + 1) * sizeof(int64_t));
  if (!cols || !coff) {
    for (int64_t t = 0; t < ntouched; t++) slot[touched[t]] = -1;
    free(touched);
    free(cols);
    free(coff);
    out->err = BSMO_ERR_NOMEM;
    return;
  }
  int64_t nb = 0, nnz = 0;
  for (int64_t t = 0; t < ntouched; t++) {
    int32_t j = touched[t];
    slot[j] = nb;
    cols[nb] = j;
    coff[nb] = nnz;
    nnz += (int64_t)m * (int64_t)b->col_sizes[j];
    nb++;
  }
  free(touched);
  out->nblk = nb;
  out->cols = cols;
  out->nnz = nnz;
  if (!pattern_only) {
    double *S = (double *)calloc((size_t)nnz + 1, sizeof(double));
    double *V = (double *)calloc((size_t)nnz + 1, sizeof(double));
    if (!S || !V) {
      free(S);
      free(V);
      free(coff);
      out->err = BSMO_ERR_NOMEM;
      for (int32_t j = 0; j < nbc; j++) slot[j] = -1;
      return;
    }
    /* pass 2: the sums S_ij, over ascending k, inner index ascending */
    for (int64_t p = a->row_start[i]; p < a->row_start[i + 1]; p++) {
      int64_t ab = a->order[p];
      int32_t k = a->blk_col[ab];
      int32_t s = a->col_sizes[k];
      const double *Ab = a->values + a->off[ab]; /* m x s, column-major */
      for (int64_t q = b->row_start[k]; q < b->row_start[k + 1]; q++) {
        int64_t bb = b->order[q];
        if (!keep_product(a->norm[ab], b->norm[bb], eps)) continue;
        int32_t j = b->blk_col[bb];
        int32_t n = b->col_sizes[j];
        const double *Bb = b->values + b->off[bb]; /* s x n, column-major */
        double *Sb = S + coff[slot[j]];            /* m x n, column-major */
        for (int32_t c = 0; c < n; c++)
          for (int32_t r = 0; r < m; r++)
            for (int32_t l = 0; l < s; l++) {
              double t = Ab[r + (int64_t)l * m] * Bb[l + (int64_t)c * s];
              Sb[r + (int64_t)c * m] = Sb[r + (int64_t)c * m] + t;
            }
      }
    }
    /* C_ij = (beta*C_in_ij or 0) + alpha*S_ij */
    for (int64_t t = 0; t < nb; t++) {
      int32_t j = cols[t];
      int64_t len = (int64_t)m * (int64_t)b->col_sizes[j];
      int64_t src = (cin && beta != 0.0) ? rowview_find(cin, i, j) : -1;
      for (int64_t e = 0; e < len; e++) {
        double base = (src >= 0) ? beta * cin->values[cin->off[src] + e] : 0.0;
        V[coff[t] + e] = base + alpha * S[coff[t] + e];
      }
    }
    free(S);
    out->vals = V;
  }
  free(coff);
  for (int32_t t = 0; t < (int32_t)nb; t++) slot[cols[t]] = -1;
}

/*
 * Full multiply over the C block rows [row_begin, row_end) (the whole matrix
 * when row_end <= row_begin). pattern_only skips the numeric sums. nthreads > 1
 * spreads independent C block rows over OpenMP threads; the arithmetic of each
 * row is unchanged, so results do not depend on the thread count.
 */
int bsmo_multiply(const bsmo_matrix *A, const bsmo_matrix *B, const bsmo_matrix *Cin,
                  double alpha, double beta, double eps, int32_t row_begin, int32_t row_end,
                  int32_t pattern_only, int32_t nthreads, bsmo_result *res) {
  if (!A || !B || !res) return BSMO_ERR_INVALID_ARG;
  memset(res, 0, sizeof(*res));
  int err;
  rowview a, b, cin;
  memset(&cin, 0, sizeof(cin));
  if ((err = rowview_build(A, 1, &a)) != BSMO_OK) return err;
  if ((err = rowview_build(B, 1, &b)) != BSMO_OK) {
    rowview_free(&a);
    return err;
  }
  const int use_cin = (Cin != NULL) && (beta != 0.0);
  if (use_cin && (err = rowview_build(Cin, 0, &cin)) != BSMO_OK) {
    rowview_free(&a);
    rowview_free(&b);
    return err;
  }
  if ((err = check_dims(A, B, use_cin ? Cin : NULL)) != BSMO_OK) goto done;
  if (use_cin && Cin->nblk > 0 && !Cin->values) {
    err = BSMO_ERR_INVALID_ARG;
    goto done;
  }
  if (row_end <= row_begin) {
    row_begin = 0;
    row_end = A->nbr;
  }
  if (row_begin < 0 || row_end > A->nbr) {
    err = BSMO_ERR_INVALID_ARG;
    goto done;
  }
  {
    const int32_t nrows = row_end - row_begin;
    rowout *ro = (rowout *)calloc((size_t)nrows + 1, sizeof(rowout));
    if (!ro) {
      err = BSMO_ERR_NOMEM;
      goto done;
    }
    int nt = nthreads > 0 ? nthreads : 1;
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
    {
      int64_t *slot = (int64_t *)malloc(((size_t)B->nbc + 1) * sizeof(int64_t));
      if (slot) {
        for (int32_t j = 0; j < B->nbc; j++) slot[j] = -1;
      }
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
      for (int32_t t = 0; t < nrows; t++) {
        if (!slot) {
          ro[t].err = BSMO_ERR_NOMEM;
          continue;
        }
        do_row(&a, &b, use_cin ? &cin : NULL, alpha, beta, eps, pattern_only, row_begin + t,
               slot, &ro[t]);
      }
      free(slot);
    }
    (void)nt;
    int64_t nblk = 0, nnz = 0;
    for (int32_t t = 0; t < nrows; t++) {
      if (ro[t].err) err = ro[t].err;
      nblk += ro[t].nblk;
      nnz += ro[t].nnz;
    }
    if (err == BSMO_OK) {
      res->blk_row = (int32_t *)malloc(((size_t)nblk + 1) * sizeof(int32_t));
      res->blk_col = (int32_t *)malloc(((size_t)nblk + 1) * sizeof(int32_t));
      res->blk_off = (int64_t *)malloc(((size_t)nblk + 1) * sizeof(int64_t));
      if (!pattern_only) res->values = (double *)malloc(((size_t)nnz + 1) * sizeof(double));
      if (!res->blk_row || !res->blk_col || !res->blk_off || (!pattern_only && !res->values))
        err = BSMO_ERR_NOMEM;
    }
    if (err == BSMO_OK) {
      int64_t pb = 0, pv = 0;
      for (int32_t t = 0; t < nrows; t++) {
        int32_t i = row_begin + t;
        int64_t rv = 0;
        for (int64_t q = 0; q < ro[t].nblk; q++) {
          res->blk_row[pb] = i;
          res->blk_col[pb] = ro[t].cols[q];
          res->blk_off[pb] = pv + rv;
          rv += (int64_t)A->row_sizes[i] * (int64_t)B->col_sizes[ro[t].cols[q]];
          pb++;
        }
        if (!pattern_only && ro[t].nnz > 0)
          memcpy(res->values + pv, ro[t].vals, (size_t)ro[t].nnz * sizeof(double));
        pv += ro[t].nnz;
        res->candidates += ro[t].candidates;
        res->kept += ro[t].kept;
        res->dropped += ro[t].dropped;
        res->flops += ro[t].flops;
      }
      res->nblk = nblk;
      res->nnz = nnz;
    }
    for (int32_t t = 0; t < nrows; t++) {
      free(ro[t].cols);
      free(ro[t].vals);
    }
    free(ro);
  }
done:
  rowview_free(&a);
  rowview_free(&b);
  rowview_free(&cin);
  if (err != BSMO_OK) {
    free(res->blk_row);
    free(res->blk_col);
    free(res->blk_off);
    free(res->values);
    memset(res, 0, sizeof(*res));
  }
  return err;
}

void bsmo_free_result(bsmo_result *res) {
  if (!res) return;
  free(res->blk_row);
  free(res->blk_col);
  free(res->blk_off);
  free(res->values);
  memset(res, 0, sizeof(*res));
}

/* The canonical norms of every block of a matrix, in list order. */
int bsmo_norms(const bsmo_matrix *M, double *out) {
  if (!M || !out) return BSMO_ERR_INVALID_ARG;
  rowview v;
  int err = rowview_build(M, 1, &v);
  if (err != BSMO_OK) return err;
  for (int64_t b = 0; b < M->nblk; b++) out[b] = v.norm[b];
  rowview_free(&v);
  return BSMO_OK;
}

int bsmo_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Post-multiplication filter (Sec. 1: filtering after each multiply;  */
/* Sec. 2: blocks below the threshold are removed after the multiply). */
/* A block of M is dropped iff its canonical norm is below eps (a tie  */
/* and NaN are kept, eps <= 0 drops nothing). The kept blocks keep     */
/* their values; the result is sorted by (row, col).                   */
/* ------------------------------------------------------------------ */
int bsmo_post_filter(const bsmo_matrix *M, double eps, bsmo_result *res) {
  if (!M || !res) return BSMO_ERR_INVALID_ARG;
  memset(res, 0, sizeof(*res));
  rowview v;
  int err = rowview_build(M, 1, &v);
  if (err != BSMO_OK) return err;
  int64_t nb = 0, nnz = 0;
  for (int64_t p = 0; p < M->nblk; p++) {
    int64_t b = v.order[p];
    if (!(v.norm[b] < eps)) {
      nb++;
      nnz += (int64_t)M->row_sizes[M->blk_row[b]] * M->col_sizes[M->blk_col[b]];
    }
  }
  res->blk_row = (int32_t *)malloc(((size_t)nb + 1) * sizeof(int32_t));
  res->blk_col = (int32_t *)malloc(((size_t)nb + 1) * sizeof(int32_t));
  res->blk_off = (int64_t *)malloc(((size_t)nb + 1) * sizeof(int64_t));
  res->values = (double *)malloc(((size_t)nnz + 1) * sizeof(double));
  if (!res->blk_row || !res->blk_col || !res->blk_off || !res->values) {
    rowview_free(&v);
    bsmo_free_result(res);
    return BSMO_ERR_NOMEM;
  }
  int64_t q = 0, o = 0;
  for (int64_t p = 0; p < M->nblk; p++) {
    int64_t b = v.order[p];
    if (v.norm[b] < eps) continue;
    int64_t len = (int64_t)M->row_sizes[M->blk_row[b]] * M->col_sizes[M->blk_col[b]];
    res->blk_row[q] = M->blk_row[b];
    res->blk_col[q] = M->blk_col[b];
    res->blk_off[q] = o;
    memcpy(res->values + o, M->values + v.off[b], (size_t)len * sizeof(double));
    o += len;
    q++;
  }
  res->nblk = nb;
  res->nnz = nnz;
  rowview_free(&v);
  return BSMO_OK;
}

/* ------------------------------------------------------------------ */
/* Block-sparse accumulation C = beta*C_in + alpha*A (Algorithm 2: the */
/* partial C panels of the last ticks are summed into the final one).  */
/* Pattern: A's blocks, plus C_in's when beta != 0 (beta == 0 ignores  */
/* C_in, as for the multiply).                                         */
/* ------------------------------------------------------------------ */
int bsmo_add(const bsmo_matrix *A, const bsmo_matrix *Cin, double alpha, double beta,
             bsmo_result *res) {
  if (!A || !res) return BSMO_ERR_INVALID_ARG;
  memset(res, 0, sizeof(*res));
  const int use_cin = (Cin != NULL) && (beta != 0.0);
  rowview a, c;
  memset(&c, 0, sizeof(c));
  int err = rowview_build(A, 0, &a);
  if (err != BSMO_OK) return err;
  if (use_cin && (err = rowview_build(Cin, 0, &c)) != BSMO_OK) {
    rowview_free(&a);
    return err;
  }
  if (use_cin) {
    int bad = Cin->nbr != A->nbr || Cin->nbc != A->nbc;
    for (int32_t i = 0; !bad && i < A->nbr; i++) bad = Cin->row_sizes[i] != A->row_sizes[i];
    for (int32_t j = 0; !bad && j < A->nbc; j++) bad = Cin->col_sizes[j] != A->col_sizes[j];
    if (bad) {
      rowview_free(&a);
      rowview_free(&c);
      return BSMO_ERR_DIM_MISMATCH;
    }
  }
  /* upper bounds, then the merge of the two sorted rows */
  int64_t cap_b = A->nblk + (use_cin ? Cin->nblk : 0);
  int64_t cap_v = 0;
  for (int64_t b = 0; b < A->nblk; b++)
    cap_v += (int64_t)A->row_sizes[A->blk_row[b]] * A->col_sizes[A->blk_col[b]];
  if (use_cin)
    for (int64_t b = 0; b < Cin->nblk; b++)
      cap_v += (int64_t)Cin->row_sizes[Cin->blk_row[b]] * Cin->col_sizes[Cin->blk_col[b]];
  res->blk_row = (int32_t *)malloc(((size_t)cap_b + 1) * sizeof(int32_t));
  res->blk_col = (int32_t *)malloc(((size_t)cap_b + 1) * sizeof(int32_t));
  res->blk_off = (int64_t *)malloc(((size_t)cap_b + 1) * sizeof(int64_t));
  res->values = (double *)malloc(((size_t)cap_v + 1) * sizeof(double));
  if (!res->blk_row || !res->blk_col || !res->blk_off || !res->values) {
    rowview_free(&a);
    rowview_free(&c);
    bsmo_free_result(res);
    return BSMO_ERR_NOMEM;
  }
  int64_t q = 0, o = 0;
  for (int32_t i = 0; i < A->nbr; i++) {
    int64_t pa = a.row_start[i], ea = a.row_start[i + 1];
    int64_t pc = use_cin ? c.row_start[i] : 0, ec = use_cin ? c.row_start[i + 1] : 0;
    while (pa < ea || pc < ec) {
      int32_t ja = pa < ea ? A->blk_col[a.order[pa]] : INT32_MAX;
      int32_t jc = pc < ec ? Cin->blk_col[c.order[pc]] : INT32_MAX;
      int32_t j = ja < jc ? ja : jc;
      int64_t len = (int64_t)A->row_sizes[i] * A->col_sizes[j];
      const double *va = (ja == j) ? A->values + a.off[a.order[pa]] : NULL;
      const double *vc = (jc == j) ? Cin->values + c.off[c.order[pc]] : NULL;
      for (int64_t e = 0; e < len; e++) {
        double base = vc ? beta * vc[e] : 0.0;
        res->values[o + e] = va ? base + alpha * va[e] : base;
      }
      res->blk_row[q] = i;
      res->blk_col[q] = j;
      res->blk_off[q] = o;
      o += len;
      q++;
      if (ja == j) pa++;
      if (jc == j) pc++;
    }
  }
  res->nblk = q;
  res->nnz = o;
  rowview_free(&a);
  rowview_free(&c);
  return BSMO_OK;
}
