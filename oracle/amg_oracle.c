/*
 * amg_oracle.c -- plain, serial, FP64 CPU statement of the aggregation-AMG
 * preconditioned Krylov method of Ganesan & Shah, "SParSH-AMG: a library for
 * hybrid CPU-GPU algebraic multigrid and preconditioned iterative methods"
 * (arXiv 2007.00056).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA library is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load it.  It shares no code, header, table or constant
 * with the CUDA library, and the CUDA library never calls it.
 *
 * Style: every step follows the paper's definitions in the paper's order, with
 * no blocking, fusion or reordering.  Sums run in plain index order.  Build with
 * -O2 -ffp-contract=off so that no multiply-add is contracted.
 *
 * Readings of points the paper leaves open:
 *  - edge weight of {i,j}: w_ij = max(|a_ij|, |a_ji|), diagonal and explicit
 *    zeros skipped (Sec. 2.1.1 and Algorithm 3 put both directed entries in
 *    the edge list, so a pair is first met at the larger one);
 *  - ties between equal weights go to the smaller index: the total edge order
 *    is (w descending, min(i,j) ascending, max(i,j) ascending); as an option,
 *    the order Algorithm 3 prints (its edge list sorted lexicographically
 *    descending, so ties go to the larger index: w descending, max(i,j)
 *    descending, min(i,j) descending);
 *  - as an option outside the paper, the edge weight divided by
 *    sqrt(|a_ii| |a_jj|) (a diagonally scaled weight, computed as
 *    max(|a_ij|,|a_ji|) / sqrt(|a_ii| * |a_jj|));
 *  - aggregate number = rank of the aggregate's smallest member;
 *  - "2 passes": two pairwise matchings per level, the second one on the
 *    Galerkin product of the first (aggregates of up to four nodes);
 *  - Galerkin sum order: coarse row I, members ascending, each member's CSR
 *    entries in stored order, first contribution starts the sum;
 *  - Algorithm 4 (PCG) prints r_{j+1} = r_j + alpha A p_j; the sign is read as
 *    minus, and the loop runs while the relative residual exceeds tol;
 *  - Algorithm 5 (BiCG) is read as right-preconditioned BiCGStab with
 *    p_0 = r_0, rbar_0 = r_0 and p_{j+1} = r_{j+1} + beta (p_j - omega A p~_j);
 *  - the coarsest solve of Algorithm 1 is A_L^{-1} f_L by dense LU with partial
 *    pivoting, or, when A_L is too large for a dense factor, Jacobi-PCG to a
 *    relative residual of 1e-12 (the CG coarse solver of Sec. 4.2), in the
 *    textbook recurrence of preconditioned CG;
 *  - the W- and F-cycles, which Sec. 2 and Sec. 3 only name, take their
 *    textbook form: the coarse correction of level k is gamma = 2 cycles of
 *    level k+1 (W), or one F-cycle then one V-cycle of level k+1 (F), the
 *    first from a zero guess and the second from the first one's result; the
 *    coarsest level is solved once per coarse correction;
 *  - AMG as a solver (Sec. 3.1, Sec. 4.4) is the stationary iteration
 *    x_{j+1} = x_j + M^{-1}(b - A x_j) with M^{-1} one cycle from a zero
 *    guess, stopping once ||b - A x_j|| <= rtol ||b||;
 *  - the node-based matching's scan "alternately from the first and the last
 *    index" (Sec. 2.1.1) alternates per pairwise pass over the whole
 *    hierarchy (upward in passes 0, 2, 4, ..., downward in 1, 3, 5, ...),
 *    numbering aggregates in visit order as Algorithm 2's counter does.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_INVALID_ARG 1
#define ORC_ERR_INVALID_CSR 2
#define ORC_ERR_ZERO_DIAG 3
#define ORC_ERR_OOM 4
#define ORC_ERR_BREAKDOWN 5
#define ORC_ERR_NOT_CONVERGED 6

/* ------------------------------------------------------------------------ */
/* Basic CSR helpers                                                        */
/* ------------------------------------------------------------------------ */

/* y = A x, each row summed in stored order (the plain definition). */
void orc_spmv(int n, const int *rp, const int *ci, const double *val,
              const double *x, double *y) {
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) s += val[e] * x[ci[e]];
    y[i] = s;
  }
}

static double dot(int n, const double *a, const double *b) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

static double norm2(int n, const double *a) { return sqrt(dot(n, a, a)); }

/* Stored value a_ij, or 0 when (i,j) is not stored.  Columns are sorted. */
static double entry(const int *rp, const int *ci, const double *val, int i, int j) {
  int lo = rp[i], hi = rp[i + 1] - 1;
  while (lo <= hi) {
    int mid = lo + (hi - lo) / 2;
    if (ci[mid] == j) return val[mid];
    if (ci[mid] < j) lo = mid + 1; else hi = mid - 1;
  }
  return 0.0;
}

/* Checks the CSR conventions of the problem statement (Sec. 2: A is N x N,
 * stored in CSR, Sec. 2.1): row pointers start at 0 and do not decrease,
 * columns lie in [0,n) and are strictly ascending within each row. */
int orc_check_csr(int n, long long nnz, const int *rp, const int *ci) {
  if (n < 0 || nnz < 0) return ORC_ERR_INVALID_ARG;
  if (rp[0] != 0 || (long long)rp[n] != nnz) return ORC_ERR_INVALID_CSR;
  for (int i = 0; i < n; ++i) {
    if (rp[i + 1] < rp[i]) return ORC_ERR_INVALID_CSR;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      if (ci[e] < 0 || ci[e] >= n) return ORC_ERR_INVALID_CSR;
      if (e > rp[i] && ci[e] <= ci[e - 1]) return ORC_ERR_INVALID_CSR;
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Heavy-edge matching (Sec. 2.1)                                           */
/* ------------------------------------------------------------------------ */

typedef struct { double w; int u, v; } edge_t;

/* Total edge order: heavier first; equal weights -> smaller min endpoint,
 * then smaller max endpoint. */
static int edge_cmp(const void *pa, const void *pb) {
  const edge_t *a = (const edge_t *)pa, *b = (const edge_t *)pb;
  if (a->w > b->w) return -1;
  if (a->w < b->w) return 1;
  if (a->u != b->u) return a->u < b->u ? -1 : 1;
  if (a->v != b->v) return a->v < b->v ? -1 : 1;
  return 0;
}

/* Total edge order of Algorithm 3's lexicographically descending sort:
 * heavier first; equal weights -> larger max endpoint, then larger min. */
static int edge_cmp_desc(const void *pa, const void *pb) {
  const edge_t *a = (const edge_t *)pa, *b = (const edge_t *)pb;
  if (a->w > b->w) return -1;
  if (a->w < b->w) return 1;
  if (a->v != b->v) return a->v > b->v ? -1 : 1;
  if (a->u != b->u) return a->u > b->u ? -1 : 1;
  return 0;
}

/* |a_ii| of every row (0 when the diagonal is not stored). */
static double *abs_diag(int n, const int *rp, const int *ci, const double *val) {
  double *d = (double *)calloc((size_t)(n ? n : 1), sizeof(double));
  if (!d) return NULL;
  for (int i = 0; i < n; ++i)
    for (int e = rp[i]; e < rp[i + 1]; ++e)
      if (ci[e] == i) d[i] = fabs(val[e]);
  return d;
}

/* Weight of the directed entry a_ij: |a_ij|, or with edge_weight = 1
 * |a_ij| / sqrt(|a_ii| * |a_jj|). */
static double entry_weight(double a_ij, const double *d, int i, int j, int edge_weight) {
  if (edge_weight == 1) return fabs(a_ij) / sqrt(d[i] * d[j]);
  return fabs(a_ij);
}

/* Edge-based HEM (Sec. 2.1.2, Algorithm 3): list every stored off-diagonal
 * nonzero as an edge weighted |a_ij|, sort the list heaviest first, then walk
 * it and pair both endpoints whenever both are still unpaired.  Each directed
 * entry is listed, so the pair {i,j} is met first at max(|a_ij|,|a_ji|); the
 * later copy finds both ends taken and does nothing.  Ties use the total
 * order of edge_cmp (smaller index first).  mate[i] = partner or -1.
 * Returns the number of pairs, or -1 on allocation failure. */
int orc_match_greedy_opt(int n, const int *rp, const int *ci, const double *val, int tie_break,
                         int edge_weight, int *mate) {
  double *d = abs_diag(n, rp, ci, val);
  if (!d) return -1;
  long long m = 0;
  for (int i = 0; i < n; ++i)
    for (int e = rp[i]; e < rp[i + 1]; ++e)
      if (ci[e] != i && val[e] != 0.0) ++m;
  edge_t *T = (edge_t *)malloc((size_t)(m ? m : 1) * sizeof(edge_t));
  if (!T) { free(d); return -1; }
  long long t = 0;
  for (int i = 0; i < n; ++i)
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      int j = ci[e];
      if (j == i || val[e] == 0.0) continue;
      T[t].w = entry_weight(val[e], d, i, j, edge_weight);
      T[t].u = i < j ? i : j;
      T[t].v = i < j ? j : i;
      ++t;
    }
  qsort(T, (size_t)m, sizeof(edge_t), tie_break == 1 ? edge_cmp_desc : edge_cmp);
  for (int i = 0; i < n; ++i) mate[i] = -1;
  int pairs = 0;
  for (long long k = 0; k < m; ++k) {
    int u = T[k].u, v = T[k].v;
    if (mate[u] < 0 && mate[v] < 0) {
      mate[u] = v;
      mate[v] = u;
      ++pairs;
    }
  }
  free(T);
  free(d);
  return pairs;
}

int orc_match_greedy(int n, const int *rp, const int *ci, const double *val, int *mate) {
  return orc_match_greedy_opt(n, rp, ci, val, 0, 0, mate);
}

/* Weighted neighbour lists of the undirected graph of A (Sec. 2.1: A is the
 * adjacency matrix, a_ij the edge weight): neighbours of i are all j != i with
 * a_ij != 0 or a_ji != 0, weighted max(|a_ij|,|a_ji|).  Built by brute force
 * from both directions of every stored entry. */
typedef struct { int *rp; int *nb; double *w; } wgraph_t;

static int wgraph_build(int n, const int *rp, const int *ci, const double *val, int edge_weight, wgraph_t *g) {
  double *d = abs_diag(n, rp, ci, val);
  int *deg = (int *)calloc((size_t)n + 1, sizeof(int));
  if (!deg || !d) { free(deg); free(d); return -1; }
  for (int i = 0; i < n; ++i)
    for (int e = rp[i]; e < rp[i + 1]; ++e)
      if (ci[e] != i && val[e] != 0.0) { deg[i]++; deg[ci[e]]++; }
  /* upper bound on the list sizes (each pair may be listed twice) */
  g->rp = (int *)malloc(((size_t)n + 1) * sizeof(int));
  long long cap = 0;
  for (int i = 0; i < n; ++i) cap += deg[i];
  g->nb = (int *)malloc((size_t)(cap ? cap : 1) * sizeof(int));
  g->w = (double *)malloc((size_t)(cap ? cap : 1) * sizeof(double));
  int *fill = (int *)calloc((size_t)n + 1, sizeof(int));
  if (!g->rp || !g->nb || !g->w || !fill) { free(deg); free(fill); return -1; }
  long long *start = (long long *)malloc(((size_t)n + 1) * sizeof(long long));
  start[0] = 0;
  for (int i = 0; i < n; ++i) start[i + 1] = start[i] + deg[i];
  for (int i = 0; i < n; ++i)
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      int j = ci[e];
      if (j == i || val[e] == 0.0) continue;
      double a = entry_weight(val[e], d, i, j, edge_weight);
      /* add (i -> j) and (j -> i), keeping the larger weight for repeats */
      int ends[2][2] = {{i, j}, {j, i}};
      for (int s = 0; s < 2; ++s) {
        int p = ends[s][0], q = ends[s][1], found = 0;
        for (long long k = start[p]; k < start[p] + fill[p]; ++k)
          if (g->nb[k] == q) { if (a > g->w[k]) g->w[k] = a; found = 1; break; }
        if (!found) { g->nb[start[p] + fill[p]] = q; g->w[start[p] + fill[p]] = a; fill[p]++; }
      }
    }
  /* compact */
  long long o = 0;
  for (int i = 0; i < n; ++i) {
    g->rp[i] = (int)o;
    for (long long k = start[i]; k < start[i] + fill[i]; ++k) { g->nb[o] = g->nb[k]; g->w[o] = g->w[k]; ++o; }
  }
  g->rp[n] = (int)o;
  free(deg); free(fill); free(start); free(d);
  return 0;
}

static void wgraph_free(wgraph_t *g) { free(g->rp); free(g->nb); free(g->w); }

/* Matching by synchronous rounds of mutual-heaviest-neighbour handshakes: in
 * each round every unpaired node picks its heaviest unpaired neighbour
 * (equal weights -> smaller index; larger with tie_break = 1) using the state
 * at the start of the round;
 * two nodes that picked each other are paired.  Rounds repeat until a round
 * pairs nothing; nodes still unpaired stay single (Sec. 2.1.1: a node without
 * an unmatched neighbour becomes a coarse node by itself).  *rounds counts
 * every round run, the final empty one included.  Returns the number of
 * pairs, or -1 on allocation failure. */
int orc_match_rounds_opt(int n, const int *rp, const int *ci, const double *val, int tie_break, int edge_weight,
                         int *mate, int *rounds) {
  wgraph_t g;
  if (wgraph_build(n, rp, ci, val, edge_weight, &g)) return -1;
  int *pick = (int *)malloc((size_t)(n ? n : 1) * sizeof(int));
  for (int i = 0; i < n; ++i) mate[i] = -1;
  int pairs = 0, r = 0;
  for (;;) {
    ++r;
    for (int i = 0; i < n; ++i) {
      pick[i] = -1;
      if (mate[i] >= 0) continue;
      double best = 0.0;
      for (int k = g.rp[i]; k < g.rp[i + 1]; ++k) {
        int j = g.nb[k];
        if (mate[j] >= 0) continue;
        if (pick[i] < 0 || g.w[k] > best || (g.w[k] == best && (tie_break == 1 ? j > pick[i] : j < pick[i]))) {
          best = g.w[k];
          pick[i] = j;
        }
      }
    }
    int new_pairs = 0;
    for (int i = 0; i < n; ++i) {
      int j = pick[i];
      if (j > i && pick[j] == i) { mate[i] = j; mate[j] = i; ++new_pairs; }
    }
    pairs += new_pairs;
    if (new_pairs == 0) break;
  }
  if (rounds) *rounds = r;
  free(pick);
  wgraph_free(&g);
  return pairs;
}

int orc_match_rounds(int n, const int *rp, const int *ci, const double *val, int *mate, int *rounds) {
  return orc_match_rounds_opt(n, rp, ci, val, 0, 0, mate, rounds);
}

/* Node-based HEM as printed in Algorithm 2 (Sec. 2.1.1), kept only as a
 * cross-check: nodes are visited in index order; an unassigned node i takes,
 * among its unassigned neighbours j with a_ij != 0, the one of largest
 * |a_ij|, and on equal weights the last one met in the row (the test
 * max(k,|a_ij|) = |a_ij| accepts equality).  The printed listing scans row i
 * only.  agg receives the coarse numbers in visit order.  Returns N_c. */
int orc_nhem_dir(int n, const int *rp, const int *ci, const double *val, int descending, int *agg) {
  for (int i = 0; i < n; ++i) agg[i] = -1;
  int C = 0;
  for (int s = 0; s < n; ++s) {
    const int i = descending ? n - 1 - s : s;
    if (agg[i] >= 0) continue;
    double k = -1.0;
    int match = -1;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      int j = ci[e];
      if (j == i || agg[j] >= 0 || val[e] == 0.0) continue;
      double a = fabs(val[e]);
      if ((k > a ? k : a) == a) { k = a; match = j; }
    }
    agg[i] = C;
    if (match >= 0) agg[match] = C;
    ++C;
  }
  return C;
}

int orc_nhem(int n, const int *rp, const int *ci, const double *val, int *agg) {
  return orc_nhem_dir(n, rp, ci, val, 0, agg);
}

/* Aggregate numbering (Sec. 2.1.1, Algorithm 2's coarse counter C): every
 * aggregate (a pair or a single node) gets the rank of its smallest member,
 * i.e. aggregates are numbered in the order their smallest members appear.
 * This reproduces the column order of P in the worked example of Sec. 2.1.1.
 * Returns N_c. */
int orc_aggregates(int n, const int *mate, int *agg) {
  int C = 0;
  for (int i = 0; i < n; ++i) {
    if (mate[i] < 0 || i < mate[i]) agg[i] = C++;
  }
  for (int i = 0; i < n; ++i)
    if (mate[i] >= 0 && mate[i] < i) agg[i] = agg[mate[i]];
  return C;
}

/* Galerkin product A_c = P^T A P with the piecewise-constant P of Sec. 2.1.1
 * (P_iI = 1 iff agg[i] = I): (A_c)_IJ = sum of a_ij over i in I, j in J.  An
 * entry exists when at least one stored a_ij contributes, even if the sum is
 * 0.0.  Columns ascend.  Sum order: members i of I ascending, each row's
 * entries in stored order; the first contribution starts the sum.
 * ci_c/val_c must hold at least nnz(A) entries (nnz(A_c) <= nnz(A)).
 * Returns nnz(A_c), or -1 on allocation failure. */
long long orc_galerkin(int n, const int *rp, const int *ci, const double *val,
                       const int *agg, int nc, int *rp_c, int *ci_c, double *val_c) {
  /* member lists of every aggregate, members ascending */
  int *mcount = (int *)calloc((size_t)nc + 1, sizeof(int));
  int *mstart = (int *)malloc(((size_t)nc + 1) * sizeof(int));
  int *members = (int *)malloc((size_t)(n ? n : 1) * sizeof(int));
  int *fill = (int *)calloc((size_t)nc + 1, sizeof(int));
  /* per-row accumulator: position of coarse column J in the current row */
  int *slot = (int *)malloc((size_t)(nc ? nc : 1) * sizeof(int));
  if (!mcount || !mstart || !members || !fill || !slot) return -1;
  for (int i = 0; i < n; ++i) mcount[agg[i]]++;
  mstart[0] = 0;
  for (int I = 0; I < nc; ++I) mstart[I + 1] = mstart[I] + mcount[I];
  for (int i = 0; i < n; ++i) members[mstart[agg[i]] + fill[agg[i]]++] = i;
  for (int J = 0; J < nc; ++J) slot[J] = -1;

  long long out = 0;
  rp_c[0] = 0;
  for (int I = 0; I < nc; ++I) {
    long long row_begin = out;
    for (int m = mstart[I]; m < mstart[I + 1]; ++m) {
      int i = members[m];
      for (int e = rp[i]; e < rp[i + 1]; ++e) {
        int J = agg[ci[e]];
        if (slot[J] < 0) {
          slot[J] = (int)out;
          ci_c[out] = J;
          val_c[out] = val[e];
          ++out;
        } else {
          val_c[slot[J]] = val_c[slot[J]] + val[e];
        }
      }
    }
    /* sort the row by column (insertion sort keeps it plain) */
    for (long long a = row_begin + 1; a < out; ++a) {
      int cj = ci_c[a];
      double cv = val_c[a];
      long long b = a - 1;
      while (b >= row_begin && ci_c[b] > cj) { ci_c[b + 1] = ci_c[b]; val_c[b + 1] = val_c[b]; --b; }
      ci_c[b + 1] = cj;
      val_c[b + 1] = cv;
    }
    for (long long a = row_begin; a < out; ++a) slot[ci_c[a]] = -1;
    rp_c[I + 1] = (int)out;
  }
  free(mcount); free(mstart); free(members); free(fill); free(slot);
  return out;
}

/* ------------------------------------------------------------------------ */
/* Hierarchy (setup phase, Sec. 3)                                          */
/* ------------------------------------------------------------------------ */

typedef struct {
  int passes, max_levels, coarse_max;
  double stall_ratio, omega;
  int nu_pre, nu_post, coarse_solver; /* 0 auto, 1 dense LU, 2 CG */
  int matcher;                        /* 0 greedy EHEM order, 1 literal rounds, 2 node-based HEM
                                         (Algorithm 2) with alternating scan direction */
  int cycle;                          /* 0 V, 1 W, 2 F (Sec. 2 names all three) */
  int tie_break;                      /* 0 smaller index, 1 larger (Algorithm 3's order) */
  int edge_weight;                    /* 0 max(|a_ij|,|a_ji|), 1 / sqrt(|a_ii a_jj|) */
} orc_params;

typedef struct {
  int n;
  long long nnz;
  int *rp, *ci;
  double *val;
  double *diag;
  int *agg;   /* level k -> level k+1 (composed over the passes); NULL at the coarsest */
  int rounds[8];
} orc_level;

typedef struct {
  orc_params prm;
  int L;                 /* index of the coarsest level; levels 0..L */
  orc_level lev[32];
  int dense;             /* coarsest solved by dense LU */
  double *lu;            /* n_L x n_L, row-major, L below / U on and above the diagonal */
  int *piv;              /* row permutation: row k of PA is row piv[k] of A */
  /* V-cycle scratch, one per level */
  double *f[32], *x[32], *t[32];
  int coarse_cg_iters;   /* iterations of the last coarse CG solve */
} orc_hier;

static void level_free(orc_level *l) {
  free(l->rp); free(l->ci); free(l->val); free(l->diag); free(l->agg);
}

/* One pairwise pass: match, number, and form the Galerkin product. */
static int coarsen_pass(const orc_params *prm, int pass_index, int n, const int *rp, const int *ci,
                        const double *val, int *agg, int *nc_out, int **rp_c, int **ci_c, double **val_c,
                        long long *nnz_c, int *rounds) {
  int nc;
  if (prm->matcher == 2) {
    /* node-based HEM (Algorithm 2), its scan direction alternating from one
     * pass to the next: from the first index in passes 0, 2, 4, ..., from the
     * last index in passes 1, 3, 5, ... (counted over the whole hierarchy) */
    *rounds = 0;
    nc = orc_nhem_dir(n, rp, ci, val, pass_index % 2, agg);
  } else {
    int *mate = (int *)malloc((size_t)(n ? n : 1) * sizeof(int));
    if (!mate) return ORC_ERR_OOM;
    int r = 0;
    int pairs = prm->matcher == 1
                    ? orc_match_rounds_opt(n, rp, ci, val, prm->tie_break, prm->edge_weight, mate, &r)
                    : orc_match_greedy_opt(n, rp, ci, val, prm->tie_break, prm->edge_weight, mate);
    if (pairs < 0) { free(mate); return ORC_ERR_OOM; }
    *rounds = r;
    nc = orc_aggregates(n, mate, agg);
    free(mate);
  }
  long long nnz = rp[n];
  *rp_c = (int *)malloc(((size_t)nc + 1) * sizeof(int));
  *ci_c = (int *)malloc((size_t)(nnz ? nnz : 1) * sizeof(int));
  *val_c = (double *)malloc((size_t)(nnz ? nnz : 1) * sizeof(double));
  if (!*rp_c || !*ci_c || !*val_c) return ORC_ERR_OOM;
  *nnz_c = orc_galerkin(n, rp, ci, val, agg, nc, *rp_c, *ci_c, *val_c);
  if (*nnz_c < 0) return ORC_ERR_OOM;
  *nc_out = nc;
  return ORC_OK;
}

/* Dense LU with partial pivoting (the direct coarsest solve of Sec. 2 and
 * Algorithm 1; factor once at setup).  Pivot = largest |entry| in the column,
 * the smallest row index on ties. */
static int dense_lu(int n, double *a, int *piv) {
  for (int i = 0; i < n; ++i) piv[i] = i;
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(a[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (fabs(a[(size_t)i * n + k]) > best) { best = fabs(a[(size_t)i * n + k]); p = i; }
    if (best == 0.0) return ORC_ERR_BREAKDOWN;
    if (p != k) {
      for (int j = 0; j < n; ++j) { double t = a[(size_t)k * n + j]; a[(size_t)k * n + j] = a[(size_t)p * n + j]; a[(size_t)p * n + j] = t; }
      int t = piv[k]; piv[k] = piv[p]; piv[p] = t;
    }
    for (int i = k + 1; i < n; ++i) {
      double l = a[(size_t)i * n + k] / a[(size_t)k * n + k];
      a[(size_t)i * n + k] = l;
      for (int j = k + 1; j < n; ++j) a[(size_t)i * n + j] -= l * a[(size_t)k * n + j];
    }
  }
  return ORC_OK;
}

/* x = A^{-1} b from the factors: P A = L U, forward then back substitution. */
static void dense_lu_solve(int n, const double *lu, const int *piv, const double *b, double *x) {
  for (int i = 0; i < n; ++i) {
    double s = b[piv[i]];
    for (int j = 0; j < i; ++j) s -= lu[(size_t)i * n + j] * x[j];
    x[i] = s;
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int j = i + 1; j < n; ++j) s -= lu[(size_t)i * n + j] * x[j];
    x[i] = s / lu[(size_t)i * n + i];
  }
}

/* Stand-alone dense LU solve (used by the tests as a textbook pin). */
int orc_dense_solve(int n, const double *a_rowmajor, const double *b, double *x) {
  double *a = (double *)malloc((size_t)n * n * sizeof(double) + 8);
  int *piv = (int *)malloc((size_t)(n ? n : 1) * sizeof(int));
  memcpy(a, a_rowmajor, (size_t)n * n * sizeof(double));
  int st = dense_lu(n, a, piv);
  if (st == ORC_OK) dense_lu_solve(n, a, piv, b, x);
  free(a); free(piv);
  return st;
}

void orc_default_params(orc_params *p) {
  p->passes = 2;
  p->max_levels = 10;
  p->coarse_max = 4096;
  p->stall_ratio = 0.85;
  p->omega = 2.0 / 3.0;
  p->nu_pre = 1;
  p->nu_post = 1;
  p->coarse_solver = 0;
  p->matcher = 0;
  p->cycle = 0;
  p->tie_break = 0;
  p->edge_weight = 0;
}

void orc_destroy(orc_hier *h) {
  if (!h) return;
  for (int k = 0; k <= h->L; ++k) {
    level_free(&h->lev[k]);
    free(h->f[k]); free(h->x[k]); free(h->t[k]);
  }
  free(h->lu); free(h->piv);
  free(h);
}

static double *dup_d(const double *s, long long n) {
  double *d = (double *)malloc((size_t)(n ? n : 1) * sizeof(double));
  if (d && n) memcpy(d, s, (size_t)n * sizeof(double));
  return d;
}
static int *dup_i(const int *s, long long n) {
  int *d = (int *)malloc((size_t)(n ? n : 1) * sizeof(int));
  if (d && n) memcpy(d, s, (size_t)n * sizeof(int));
  return d;
}

/* Setup phase (Sec. 3): build the hierarchy A_0 = A, A_{k+1} = P_k^T A_k P_k
 * by `passes` pairwise HEM passes per level, stopping before a level whose size
 * ratio N_{k+1}/N_k exceeds stall_ratio, when N_k <= coarse_max, or at
 * max_levels levels (Table 2 gives 6 levels and a bounded coarsest size).
 * Then factor the coarsest matrix (dense LU) or leave it to CG. */
int orc_setup(int n, const int *rp, const int *ci, const double *val, const orc_params *prm,
              orc_hier **out) {
  *out = NULL;
  if (n <= 0) return ORC_ERR_INVALID_ARG;
  int st = orc_check_csr(n, rp[n], rp, ci);
  if (st) return st;
  orc_hier *h = (orc_hier *)calloc(1, sizeof(orc_hier));
  h->prm = *prm;
  orc_level *l0 = &h->lev[0];
  l0->n = n;
  l0->nnz = rp[n];
  l0->rp = dup_i(rp, (long long)n + 1);
  l0->ci = dup_i(ci, l0->nnz);
  l0->val = dup_d(val, l0->nnz);
  int k = 0;
  while (k + 1 < prm->max_levels && k + 1 < 32 && h->lev[k].n > prm->coarse_max) {
    orc_level *f = &h->lev[k];
    int cur_n = f->n;
    int *cur_rp = f->rp, *cur_ci = f->ci;
    double *cur_val = f->val;
    int *agg = (int *)malloc((size_t)cur_n * sizeof(int));
    for (int i = 0; i < cur_n; ++i) agg[i] = i;
    int owned = 0;
    int rounds[8] = {0};
    for (int p = 0; p < prm->passes && p < 8; ++p) {
      int *pagg = (int *)malloc((size_t)(cur_n ? cur_n : 1) * sizeof(int));
      int nc, *rpc, *cic;
      double *valc;
      long long nnzc;
      st = coarsen_pass(prm, k * prm->passes + p, cur_n, cur_rp, cur_ci, cur_val, pagg, &nc, &rpc, &cic, &valc,
                        &nnzc, &rounds[p]);
      if (st) { free(pagg); free(agg); orc_destroy(h); return st; }
      for (int i = 0; i < f->n; ++i) agg[i] = pagg[agg[i]];
      free(pagg);
      if (owned) { free(cur_rp); free(cur_ci); free(cur_val); }
      cur_n = nc; cur_rp = rpc; cur_ci = cic; cur_val = valc;
      owned = 1;
      (void)nnzc;
    }
    if ((double)cur_n / (double)f->n > prm->stall_ratio) {
      if (owned) { free(cur_rp); free(cur_ci); free(cur_val); }
      free(agg);
      break;
    }
    f->agg = agg;
    memcpy(f->rounds, rounds, sizeof(rounds));
    orc_level *c = &h->lev[k + 1];
    c->n = cur_n;
    c->nnz = cur_rp[cur_n];
    c->rp = cur_rp; c->ci = cur_ci; c->val = cur_val;
    ++k;
  }
  h->L = k;
  for (int j = 0; j <= h->L; ++j) {
    orc_level *l = &h->lev[j];
    l->diag = (double *)malloc((size_t)l->n * sizeof(double));
    for (int i = 0; i < l->n; ++i) {
      l->diag[i] = entry(l->rp, l->ci, l->val, i, i);
      if (l->diag[i] == 0.0) { orc_destroy(h); return ORC_ERR_ZERO_DIAG; }
    }
    h->f[j] = (double *)calloc((size_t)l->n, sizeof(double));
    h->x[j] = (double *)calloc((size_t)l->n, sizeof(double));
    h->t[j] = (double *)calloc((size_t)l->n, sizeof(double));
  }
  orc_level *cl = &h->lev[h->L];
  int dense = prm->coarse_solver == 1 || (prm->coarse_solver == 0 && cl->n <= prm->coarse_max);
  h->dense = dense;
  if (dense) {
    int m = cl->n;
    h->lu = (double *)calloc((size_t)m * m, sizeof(double));
    h->piv = (int *)malloc((size_t)m * sizeof(int));
    for (int i = 0; i < m; ++i)
      for (int e = cl->rp[i]; e < cl->rp[i + 1]; ++e) h->lu[(size_t)i * m + cl->ci[e]] = cl->val[e];
    st = dense_lu(m, h->lu, h->piv);
    if (st) { orc_destroy(h); return st; }
  }
  *out = h;
  return ORC_OK;
}

int orc_num_levels(const orc_hier *h) { return h->L + 1; }
int orc_dense_coarse(const orc_hier *h) { return h->dense; }
int orc_last_coarse_cg_iters(const orc_hier *h) { return h->coarse_cg_iters; }

int orc_level_info(const orc_hier *h, int k, int *n, long long *nnz, int *rounds) {
  if (k < 0 || k > h->L) return ORC_ERR_INVALID_ARG;
  *n = h->lev[k].n;
  *nnz = h->lev[k].nnz;
  if (rounds) memcpy(rounds, h->lev[k].rounds, sizeof(h->lev[k].rounds));
  return ORC_OK;
}

/* Copies level k's CSR and (k < L) its fine-to-coarse map. */
int orc_level_export(const orc_hier *h, int k, int *rp, int *ci, double *val, int *agg) {
  if (k < 0 || k > h->L) return ORC_ERR_INVALID_ARG;
  const orc_level *l = &h->lev[k];
  memcpy(rp, l->rp, ((size_t)l->n + 1) * sizeof(int));
  memcpy(ci, l->ci, (size_t)l->nnz * sizeof(int));
  memcpy(val, l->val, (size_t)l->nnz * sizeof(double));
  if (agg && k < h->L) memcpy(agg, l->agg, (size_t)l->n * sizeof(int));
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Solve phase                                                              */
/* ------------------------------------------------------------------------ */

/* Jacobi-preconditioned CG on the coarsest matrix from x = 0 until
 * ||r|| <= 1e-12 ||f|| or 1000 iterations (CG as the coarse solver, Sec. 4.2),
 * in the textbook recurrence of preconditioned CG with M = D (the diagonal):
 *   r = f, z = D^-1 r, p = z;  repeat: q = A p, alpha = (r,z)/(p,q),
 *   x += alpha p, r -= alpha q, stop if ||r|| is small enough,
 *   z = D^-1 r, beta = (r,z)_new/(r,z)_old, p = z + beta p. */
static int coarse_cg(orc_hier *h, const double *f, double *x) {
  const orc_level *l = &h->lev[h->L];
  int n = l->n;
  double *r = (double *)malloc((size_t)n * sizeof(double));
  double *z = (double *)malloc((size_t)n * sizeof(double));
  double *p = (double *)malloc((size_t)n * sizeof(double));
  double *q = (double *)malloc((size_t)n * sizeof(double));
  for (int i = 0; i < n; ++i) { x[i] = 0.0; r[i] = f[i]; }
  double fn = norm2(n, f);
  int it = 0;
  if (fn > 0.0) {
    for (int i = 0; i < n; ++i) { z[i] = r[i] / l->diag[i]; p[i] = z[i]; }
    double rz = dot(n, r, z);
    for (it = 1; it <= 1000; ++it) {
      orc_spmv(n, l->rp, l->ci, l->val, p, q);
      double alpha = rz / dot(n, p, q);
      if (!isfinite(alpha)) break;
      for (int i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
      if (norm2(n, r) <= 1e-12 * fn) break;
      for (int i = 0; i < n; ++i) z[i] = r[i] / l->diag[i];
      double rz_new = dot(n, r, z);
      double beta = rz_new / rz;
      rz = rz_new;
      for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    if (it > 1000) it = 1000;
  }
  h->coarse_cg_iters = it;
  free(r); free(z); free(p); free(q);
  return ORC_OK;
}

/* Coarsest solve x_L = A_L^{-1} f_L (Algorithm 1, "solve the system exactly"). */
static void coarse_solve(orc_hier *h, const double *f, double *x) {
  if (h->dense) dense_lu_solve(h->lev[h->L].n, h->lu, h->piv, f, x);
  else coarse_cg(h, f, x);
}

/* One damped-Jacobi sweep x <- x + omega D^{-1} (f - A x) (smoother S_k of
 * Sec. 2, damped Jacobi with the configured omega). */
static void jacobi_sweep(const orc_level *l, double omega, const double *f, double *x, double *t) {
  orc_spmv(l->n, l->rp, l->ci, l->val, x, t);
  for (int i = 0; i < l->n; ++i) x[i] = x[i] + omega * (f[i] - t[i]) / l->diag[i];
}

/* Multigrid cycle of level k on A_k x = f_k (Algorithm 1 and its W- and
 * F-cycle variants).  zero_guess = 1 starts from x_k = 0 as Algorithm 1
 * does; zero_guess = 0 starts from the x passed in.  kind: 0 V, 1 W, 2 F.
 * The coarsest level is solved, not cycled, and ignores the guess. */
static void mg_cycle(orc_hier *h, int k, const double *f, double *x, int kind, int zero_guess) {
  if (k == h->L) { coarse_solve(h, f, x); return; }
  const orc_level *l = &h->lev[k];
  const orc_params *p = &h->prm;
  double *t = h->t[k];
  /* presmoothing */
  if (zero_guess)
    for (int i = 0; i < l->n; ++i) x[i] = 0.0;
  for (int s = 0; s < p->nu_pre; ++s) jacobi_sweep(l, p->omega, f, x, t);
  /* residual r_k = f_k - A_k x_k */
  orc_spmv(l->n, l->rp, l->ci, l->val, x, t);
  for (int i = 0; i < l->n; ++i) t[i] = f[i] - t[i];
  /* restriction f_{k+1} = P_k^T r_k: sum over each aggregate, members ascending */
  int nc = h->lev[k + 1].n;
  double *fc = h->f[k + 1], *xc = h->x[k + 1];
  char *seen = (char *)calloc((size_t)nc, 1);
  for (int i = 0; i < l->n; ++i) {
    int I = l->agg[i];
    if (!seen[I]) { fc[I] = t[i]; seen[I] = 1; }
    else fc[I] = fc[I] + t[i];
  }
  free(seen);
  /* coarse correction x_{k+1} ~ A_{k+1}^{-1} f_{k+1}: the exact solve at the
   * coarsest level, else one (V), two (W) or an F- then a V- (F) cycle of
   * level k+1, the first from zero, the second from the first one's result */
  mg_cycle(h, k + 1, fc, xc, kind, 1);
  if (k + 1 < h->L && kind == 1) mg_cycle(h, k + 1, fc, xc, 1, 0);
  if (k + 1 < h->L && kind == 2) mg_cycle(h, k + 1, fc, xc, 0, 0);
  /* prolongation x_k += P_k x_{k+1} */
  for (int i = 0; i < l->n; ++i) x[i] = x[i] + xc[l->agg[i]];
  /* postsmoothing */
  for (int s = 0; s < p->nu_post; ++s) jacobi_sweep(l, p->omega, f, x, t);
}

/* z = M^{-1} r: one cycle of the configured kind from the zero guess (the
 * preconditioner of Algorithms 4 and 5; a V-cycle by default). */
int orc_vcycle(orc_hier *h, const double *r, double *z) {
  mg_cycle(h, 0, r, z, h->prm.cycle, 1);
  return ORC_OK;
}

typedef struct {
  int iterations;
  double rel_res_recurrence;
  double rel_res_true;
  int status;
} orc_info;

static double true_rel_res(const orc_level *l, const double *b, const double *x, double bn) {
  double *t = (double *)malloc((size_t)l->n * sizeof(double));
  orc_spmv(l->n, l->rp, l->ci, l->val, x, t);
  for (int i = 0; i < l->n; ++i) t[i] = b[i] - t[i];
  double r = norm2(l->n, t) / bn;
  free(t);
  return r;
}

/* Optional record of the search directions of orc_pcg, for tests of the CG
 * recurrence: while set, iteration j (1-based, j <= trace_max) stores its
 * direction p_j at trace[(j - 1) n .. j n - 1].  Not thread-safe. */
static double *pcg_trace = NULL;
static int pcg_trace_max = 0;
void orc_set_pcg_trace(double *trace, int max_vectors) {
  pcg_trace = trace;
  pcg_trace_max = trace ? max_vectors : 0;
}

/* AMG-preconditioned CG (Sec. 3.2, Algorithm 4), with the sign of the
 * residual update read as r_{j+1} = r_j - alpha A p_j.  x holds x_0 on entry.
 * Stops once ||r_j|| <= rtol ||b|| (checked after each residual update).
 * flexible = 1 uses beta = (z_{j+1}, r_{j+1} - r_j)/(z_j, r_j) (flexible CG),
 * flexible = 0 the printed beta = (r_{j+1}, z_{j+1})/(r_j, z_j). */
int orc_pcg(orc_hier *h, const double *b, double *x, double rtol, int max_iter, int flexible,
            orc_info *info) {
  const orc_level *l = &h->lev[0];
  int n = l->n;
  double *r = (double *)malloc((size_t)n * sizeof(double));
  double *rold = (double *)malloc((size_t)n * sizeof(double));
  double *z = (double *)malloc((size_t)n * sizeof(double));
  double *p = (double *)malloc((size_t)n * sizeof(double));
  double *q = (double *)malloc((size_t)n * sizeof(double));
  double bn = norm2(n, b);
  info->iterations = 0;
  info->status = ORC_OK;
  if (bn == 0.0) {
    for (int i = 0; i < n; ++i) x[i] = 0.0;
    info->rel_res_recurrence = info->rel_res_true = 0.0;
    free(r); free(rold); free(z); free(p); free(q);
    return ORC_OK;
  }
  orc_spmv(n, l->rp, l->ci, l->val, x, q);
  for (int i = 0; i < n; ++i) r[i] = b[i] - q[i];
  double rel = norm2(n, r) / bn;
  int st = ORC_ERR_NOT_CONVERGED;
  if (rel <= rtol) st = ORC_OK;
  int it = 0;
  if (st != ORC_OK) {
    orc_vcycle(h, r, z);
    for (int i = 0; i < n; ++i) p[i] = z[i];
    double rz = dot(n, r, z);
    for (it = 1; it <= max_iter; ++it) {
      if (it <= pcg_trace_max) memcpy(pcg_trace + (size_t)(it - 1) * n, p, (size_t)n * sizeof(double));
      orc_spmv(n, l->rp, l->ci, l->val, p, q);
      double pq = dot(n, p, q);
      if (pq == 0.0 || !isfinite(pq) || !isfinite(rz)) { st = ORC_ERR_BREAKDOWN; break; }
      double alpha = rz / pq;
      for (int i = 0; i < n; ++i) x[i] = x[i] + alpha * p[i];
      if (flexible) memcpy(rold, r, (size_t)n * sizeof(double));
      for (int i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];
      rel = norm2(n, r) / bn;
      if (rel <= rtol) { st = ORC_OK; break; }
      if (it == max_iter) break;
      orc_vcycle(h, r, z);
      double rz_new = dot(n, r, z);
      double beta;
      if (flexible) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += z[i] * (r[i] - rold[i]);
        beta = s / rz;
      } else {
        beta = rz_new / rz;
      }
      rz = rz_new;
      for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    if (it > max_iter) it = max_iter;
  }
  info->iterations = it;
  info->rel_res_recurrence = rel;
  info->rel_res_true = true_rel_res(l, b, x, bn);
  info->status = st;
  free(r); free(rold); free(z); free(p); free(q);
  return st;
}

/* AMG as a solver (Sec. 3.1, Sec. 4.4): the stationary iteration
 * x_{j+1} = x_j + M^{-1}(b - A x_j), M^{-1} one cycle of the configured kind
 * from the zero guess.  x holds x_0 on entry.  Stops once
 * ||b - A x_j|| <= rtol ||b|| (the residual recomputed from x_j after every
 * cycle) or after max_iter cycles. */
int orc_amg_solve(orc_hier *h, const double *b, double *x, double rtol, int max_iter, orc_info *info) {
  const orc_level *l = &h->lev[0];
  int n = l->n;
  double *r = (double *)malloc((size_t)n * sizeof(double));
  double *z = (double *)malloc((size_t)n * sizeof(double));
  double bn = norm2(n, b);
  info->iterations = 0;
  info->status = ORC_OK;
  if (bn == 0.0) {
    for (int i = 0; i < n; ++i) x[i] = 0.0;
    info->rel_res_recurrence = info->rel_res_true = 0.0;
    free(r); free(z);
    return ORC_OK;
  }
  orc_spmv(n, l->rp, l->ci, l->val, x, r);
  for (int i = 0; i < n; ++i) r[i] = b[i] - r[i];
  double rel = norm2(n, r) / bn;
  int st = rel <= rtol ? ORC_OK : ORC_ERR_NOT_CONVERGED;
  int it = 0;
  while (st != ORC_OK && it < max_iter) {
    orc_vcycle(h, r, z);
    for (int i = 0; i < n; ++i) x[i] = x[i] + z[i];
    orc_spmv(n, l->rp, l->ci, l->val, x, r);
    for (int i = 0; i < n; ++i) r[i] = b[i] - r[i];
    ++it;
    rel = norm2(n, r) / bn;
    if (rel <= rtol) st = ORC_OK;
    else if (!isfinite(rel)) st = ORC_ERR_BREAKDOWN;
    if (st == ORC_ERR_BREAKDOWN) break;
  }
  info->iterations = it;
  info->rel_res_recurrence = rel;
  info->rel_res_true = rel;
  info->status = st;
  free(r); free(z);
  return st;
}

/* AMG-preconditioned BiCGStab (Sec. 3.2, Algorithm 5), right preconditioned:
 * p~ = M^{-1} p, s = r - alpha A p~, s~ = M^{-1} s, omega = (A s~, s)/(A s~, A s~),
 * x += alpha p~ + omega s~, r = s - omega A s~, beta = (r_{j+1},rbar)/(r_j,rbar)
 * * alpha/omega, p = r + beta (p - omega A p~).  rbar = r_0, p_0 = r_0.
 * If ||s|| <= rtol ||b|| the half step x += alpha p~ ends the iteration. */
int orc_bicgstab(orc_hier *h, const double *b, double *x, double rtol, int max_iter, orc_info *info) {
  const orc_level *l = &h->lev[0];
  int n = l->n;
  double *r = (double *)malloc((size_t)n * sizeof(double));
  double *rb = (double *)malloc((size_t)n * sizeof(double));
  double *p = (double *)malloc((size_t)n * sizeof(double));
  double *ph = (double *)malloc((size_t)n * sizeof(double));
  double *v = (double *)malloc((size_t)n * sizeof(double));
  double *s = (double *)malloc((size_t)n * sizeof(double));
  double *sh = (double *)malloc((size_t)n * sizeof(double));
  double *t = (double *)malloc((size_t)n * sizeof(double));
  double bn = norm2(n, b);
  info->iterations = 0;
  info->status = ORC_OK;
  int st = ORC_ERR_NOT_CONVERGED;
  double rel = 0.0;
  int it = 0;
  if (bn == 0.0) {
    for (int i = 0; i < n; ++i) x[i] = 0.0;
    st = ORC_OK;
    goto done;
  }
  orc_spmv(n, l->rp, l->ci, l->val, x, t);
  for (int i = 0; i < n; ++i) { r[i] = b[i] - t[i]; rb[i] = r[i]; p[i] = r[i]; }
  rel = norm2(n, r) / bn;
  if (rel <= rtol) { st = ORC_OK; goto done; }
  double rho = dot(n, r, rb);
  for (it = 1; it <= max_iter; ++it) {
    if (fabs(rho) < 1e-300 || !isfinite(rho)) { st = ORC_ERR_BREAKDOWN; break; }
    orc_vcycle(h, p, ph);
    orc_spmv(n, l->rp, l->ci, l->val, ph, v);
    double rv = dot(n, v, rb);
    if (fabs(rv) < 1e-300 || !isfinite(rv)) { st = ORC_ERR_BREAKDOWN; break; }
    double alpha = rho / rv;
    for (int i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
    double srel = norm2(n, s) / bn;
    if (srel <= rtol) {
      for (int i = 0; i < n; ++i) x[i] = x[i] + alpha * ph[i];
      rel = srel;
      st = ORC_OK;
      break;
    }
    orc_vcycle(h, s, sh);
    orc_spmv(n, l->rp, l->ci, l->val, sh, t);
    double tt = dot(n, t, t);
    if (tt == 0.0 || !isfinite(tt)) { st = ORC_ERR_BREAKDOWN; break; }
    double omega = dot(n, t, s) / tt;
    for (int i = 0; i < n; ++i) {
      x[i] = x[i] + alpha * ph[i] + omega * sh[i];
      r[i] = s[i] - omega * t[i];
    }
    rel = norm2(n, r) / bn;
    if (rel <= rtol) { st = ORC_OK; break; }
    if (fabs(omega) < 1e-300) { st = ORC_ERR_BREAKDOWN; break; }
    if (it == max_iter) break;
    double rho_new = dot(n, r, rb);
    double beta = (rho_new / rho) * (alpha / omega);
    rho = rho_new;
    for (int i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
  }
  if (it > max_iter) it = max_iter;
done:
  info->iterations = it;
  info->rel_res_recurrence = rel;
  info->rel_res_true = bn == 0.0 ? 0.0 : true_rel_res(l, b, x, bn);
  info->status = st;
  free(r); free(rb); free(p); free(ph); free(v); free(s); free(sh); free(t);
  return st;
}
