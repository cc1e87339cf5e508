/*
 * ot_oracle.c -- plain, slow, single-threaded CPU oracle for the exact
 * assignment problem.  TEST INFRASTRUCTURE ONLY: nothing in the product
 * library links or calls this file; only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load it.  It shares no code, header or
 * constant with the CUDA path.
 *
 * Problem (paper, Sec. 1, Eq. 1 with r and c all-ones, i.e. the assignment
 * problem): given an n x m integer cost matrix C (n <= m), find an injective
 * map sigma: [n] -> [m] minimising sum_i C[i][sigma(i)].
 *
 * Functions:
 *   oracle_brute_force   the plain definition: enumerate every injective map
 *                        (n <= 8, m <= 10).
 *   oracle_km            Kuhn-Munkres (Hungarian) in its shortest-augmenting-
 *                        path form, one root row at a time, eager dual updates
 *                        (paper, Sec. 2.3 "Variations of the Hungarian
 *                        algorithm" and Sec. 4.1 "KM and variants": the exact
 *                        O(n^3) KM the paper benchmarks).
 *   oracle_bkm           batched KM (paper, Sec. 2.3 "Batched KM"): route a
 *                        maximal set of vertex-disjoint augmenting paths in
 *                        the tight-edge graph, repeat until there is none,
 *                        then adjust the duals across the cut between the
 *                        rows and columns reachable from free rows, exactly
 *                        as KM adjusts them.  Exact mode: scaling factor 1.
 *   oracle_check_certificate   LP-duality certificate of optimality.
 *   oracle_auction       the auction algorithm with epsilon-scaling (paper,
 *                        Sec. 2.3.3 and Sec. 4.1 "Auction"), exact for
 *                        integer costs; readings at the function.
 *
 * Tie-breaks where the paper is silent: rows are rooted in index order, the
 * minimum slack picks the lowest column index, a slack entry is replaced only
 * on a strictly smaller value.  INF = 2^62.
 *
 * Dual convention: u (rows), v (columns), feasibility u_i + v_j <= C[i][j],
 * v_j <= 0, tight (equality) on matched pairs, v_j = 0 on unmatched columns.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_INF ((int64_t)1 << 62)

#define AT(C, ldc, i, j) ((int64_t)(C)[(int64_t)(i) * (ldc) + (j)])

/* ------------------------------------------------------------------ */
/* brute force: the plain definition of OPT                            */
/* ------------------------------------------------------------------ */

static void bf_rec(const int32_t *C, int64_t ldc, int n, int m, int row,
                   int64_t partial, int *used, int *cur, int64_t *best,
                   int32_t *best_assign) {
  if (row == n) {
    if (partial < *best) {
      *best = partial;
      for (int i = 0; i < n; ++i) best_assign[i] = cur[i];
    }
    return;
  }
  for (int j = 0; j < m; ++j) {
    if (used[j]) continue;
    used[j] = 1;
    cur[row] = j;
    bf_rec(C, ldc, n, m, row + 1, partial + AT(C, ldc, row, j), used, cur,
           best, best_assign);
    used[j] = 0;
  }
}

/* Returns OPT; row_to_col receives the first optimal map in lexicographic
 * enumeration order.  Returns INT64_MIN on bad sizes. */
int64_t oracle_brute_force(const int32_t *C, int64_t ldc, int n, int m,
                           int32_t *row_to_col) {
  if (n < 0 || n > 8 || m < n || m > 10) return INT64_MIN;
  int used[16] = {0}, cur[16] = {0};
  int64_t best = INT64_MAX;
  if (n == 0) return 0;
  bf_rec(C, ldc, n, m, 0, 0, used, cur, &best, row_to_col);
  return best;
}

/* ------------------------------------------------------------------ */
/* Kuhn-Munkres, shortest augmenting path, eager duals                 */
/* ------------------------------------------------------------------ */

/* stats[0] = row scans (tree-growing steps), stats[1] = cost bytes read
 * (4 bytes per reduced cost evaluated, i.e. per column outside the tree at
 * each scan), stats[2] = augmentations.  Returns the optimal cost, or
 * INT64_MIN on bad arguments / allocation failure. */
int64_t oracle_km(const int32_t *C, int64_t ldc, int n, int m,
                  int32_t *row_to_col, int64_t *u, int64_t *v,
                  int64_t *stats) {
  if (n < 0 || m < n || (n > 0 && ldc < m)) return INT64_MIN;
  int64_t steps = 0, bytes = 0, augs = 0;
  for (int i = 0; i < n; ++i) { u[i] = 0; row_to_col[i] = -1; }
  for (int j = 0; j < m; ++j) v[j] = 0;
  int32_t *col_to_row = malloc(sizeof(int32_t) * (m ? m : 1));
  int64_t *slack = malloc(sizeof(int64_t) * (m ? m : 1));
  int32_t *pred = malloc(sizeof(int32_t) * (m ? m : 1));   /* row */
  char *in_tree = malloc(m ? m : 1);
  if (!col_to_row || !slack || !pred || !in_tree) {
    free(col_to_row); free(slack); free(pred); free(in_tree);
    return INT64_MIN;
  }
  for (int j = 0; j < m; ++j) col_to_row[j] = -1;

  for (int r = 0; r < n; ++r) {
    for (int j = 0; j < m; ++j) { slack[j] = OR_INF; pred[j] = -1; in_tree[j] = 0; }
    int i = r;            /* row most recently added to the tree */
    int jfree = -1;
    while (jfree < 0) {
      /* scan row i: reduced costs against the current duals */
      steps++;
      for (int j = 0; j < m; ++j) {
        if (in_tree[j]) continue;
        int64_t rc = AT(C, ldc, i, j) - u[i] - v[j];
        bytes += 4;
        if (rc < slack[j]) { slack[j] = rc; pred[j] = i; }
      }
      /* minimum slack outside the tree, lowest column on ties */
      int64_t delta = OR_INF;
      int jstar = -1;
      for (int j = 0; j < m; ++j)
        if (!in_tree[j] && slack[j] < delta) { delta = slack[j]; jstar = j; }
      /* dual adjustment: tree rows up, tree columns down, slacks down */
      u[r] += delta;
      for (int j = 0; j < m; ++j) {
        if (in_tree[j]) { u[col_to_row[j]] += delta; v[j] -= delta; }
        else slack[j] -= delta;
      }
      if (jstar < 0) break;   /* unreachable for n <= m: some column is outside T */
      in_tree[jstar] = 1;
      if (col_to_row[jstar] < 0) jfree = jstar;
      else i = col_to_row[jstar];
    }
    /* augment: flip the alternating path that ends at jfree */
    augs++;
    int j = jfree;
    while (j >= 0) {
      int pi = pred[j];
      int prev = row_to_col[pi];        /* -1 for the root r */
      row_to_col[pi] = j;
      col_to_row[j] = pi;
      j = prev;
    }
  }
  int64_t cost = 0;
  for (int i = 0; i < n; ++i) cost += AT(C, ldc, i, row_to_col[i]);
  if (stats) { stats[0] = steps; stats[1] = bytes; stats[2] = augs; }
  free(col_to_row); free(slack); free(pred); free(in_tree);
  return cost;
}

/* ------------------------------------------------------------------ */
/* batched KM (exact, scaling factor 1)                                */
/* ------------------------------------------------------------------ */

typedef struct {
  const int32_t *C; int64_t ldc; int n, m;
  int64_t *u, *v;
  int32_t *row_to_col, *col_to_row;
  int32_t *layer;      /* BFS layer of each row, -1 = unreached */
  int32_t *queue;
  char *col_dead;      /* column already used by a path in this phase */
  int64_t bytes;
} bkm_state;

static int tight(const bkm_state *s, int i, int j) {
  return AT(s->C, s->ldc, i, j) - s->u[i] - s->v[j] == 0;
}

/* Hopcroft-Karp layering over tight edges from all free rows.  Returns the
 * length (in rows) of the shortest augmenting path, or -1 if none. */
static int hk_bfs(bkm_state *s) {
  int n = s->n, m = s->m, head = 0, tail = 0, found = -1;
  for (int i = 0; i < n; ++i) {
    if (s->row_to_col[i] < 0) { s->layer[i] = 0; s->queue[tail++] = i; }
    else s->layer[i] = -1;
  }
  while (head < tail) {
    int i = s->queue[head++];
    if (found >= 0 && s->layer[i] >= found) continue;
    for (int j = 0; j < m; ++j) {
      s->bytes += 4;
      if (!tight(s, i, j)) continue;
      int k = s->col_to_row[j];
      if (k < 0) { if (found < 0) found = s->layer[i]; }
      else if (s->layer[k] < 0) { s->layer[k] = s->layer[i] + 1; s->queue[tail++] = k; }
    }
  }
  return found;
}

/* DFS along the layers, columns in increasing order; a column is used by
 * at most one path per phase and rows that fail are cut from the layering. */
static int hk_dfs(bkm_state *s, int i, int last) {
  for (int j = 0; j < s->m; ++j) {
    if (s->col_dead[j] || !tight(s, i, j)) continue;
    int k = s->col_to_row[j];
    if (k < 0) {
      if (s->layer[i] != last) continue;
      s->col_dead[j] = 1;
      s->row_to_col[i] = j; s->col_to_row[j] = i;
      return 1;
    }
    if (s->layer[k] != s->layer[i] + 1) continue;
    s->col_dead[j] = 1;
    if (hk_dfs(s, k, last)) { s->row_to_col[i] = j; s->col_to_row[j] = i; return 1; }
  }
  s->layer[i] = -1;
  return 0;
}

/* stats[0] = dual adjustments (rounds), stats[1] = HK phases,
 * stats[2] = augmentations, stats[3] = cost bytes evaluated. */
int64_t oracle_bkm(const int32_t *C, int64_t ldc, int n, int m,
                   int32_t *row_to_col, int64_t *u, int64_t *v,
                   int64_t *stats) {
  if (n < 0 || m < n || (n > 0 && ldc < m)) return INT64_MIN;
  bkm_state s;
  s.C = C; s.ldc = ldc; s.n = n; s.m = m; s.u = u; s.v = v;
  s.row_to_col = row_to_col; s.bytes = 0;
  s.col_to_row = malloc(sizeof(int32_t) * (m ? m : 1));
  s.layer = malloc(sizeof(int32_t) * (n ? n : 1));
  s.queue = malloc(sizeof(int32_t) * (n ? n : 1));
  s.col_dead = malloc(m ? m : 1);
  char *in_S = malloc(n ? n : 1), *in_T = malloc(m ? m : 1);
  int32_t *q = malloc(sizeof(int32_t) * (n ? n : 1));
  if (!s.col_to_row || !s.layer || !s.queue || !s.col_dead || !in_S || !in_T || !q) {
    free(s.col_to_row); free(s.layer); free(s.queue); free(s.col_dead);
    free(in_S); free(in_T); free(q);
    return INT64_MIN;
  }
  int64_t rounds = 0, phases = 0, augs = 0;
  /* initial duals: row minima, zero column potentials */
  for (int i = 0; i < n; ++i) {
    int64_t mn = OR_INF;
    for (int j = 0; j < m; ++j) { int64_t c = AT(C, ldc, i, j); if (c < mn) mn = c; }
    s.bytes += 4 * (int64_t)m;
    u[i] = mn; row_to_col[i] = -1;
  }
  for (int j = 0; j < m; ++j) { v[j] = 0; s.col_to_row[j] = -1; }
  int matched = 0;

  for (;;) {
    /* maximal augmentation in the tight graph, repeated until none exists */
    for (;;) {
      int last = hk_bfs(&s);
      if (last < 0) break;
      phases++;
      memset(s.col_dead, 0, m);
      for (int i = 0; i < n; ++i)
        if (row_to_col[i] < 0 && s.layer[i] == 0)
          if (hk_dfs(&s, i, last)) { augs++; matched++; }
    }
    if (matched == n) break;
    /* cut: rows/columns reachable from free rows along alternating tight paths */
    int head = 0, tail = 0;
    for (int i = 0; i < n; ++i) { in_S[i] = row_to_col[i] < 0; if (in_S[i]) q[tail++] = i; }
    memset(in_T, 0, m);
    while (head < tail) {
      int i = q[head++];
      for (int j = 0; j < m; ++j) {
        s.bytes += 4;
        if (in_T[j] || !tight(&s, i, j)) continue;
        in_T[j] = 1;
        int k = s.col_to_row[j];   /* matched: no augmenting path remains */
        if (k >= 0 && !in_S[k]) { in_S[k] = 1; q[tail++] = k; }
      }
    }
    /* delta = min reduced cost from S to columns outside T */
    int64_t delta = OR_INF;
    for (int i = 0; i < n; ++i) {
      if (!in_S[i]) continue;
      for (int j = 0; j < m; ++j) {
        if (in_T[j]) continue;
        s.bytes += 4;
        int64_t rc = AT(C, ldc, i, j) - u[i] - v[j];
        if (rc < delta) delta = rc;
      }
    }
    rounds++;
    for (int i = 0; i < n; ++i) if (in_S[i]) u[i] += delta;
    for (int j = 0; j < m; ++j) if (in_T[j]) v[j] -= delta;
  }
  int64_t cost = 0;
  for (int i = 0; i < n; ++i) cost += AT(C, ldc, i, row_to_col[i]);
  if (stats) { stats[0] = rounds; stats[1] = phases; stats[2] = augs; stats[3] = s.bytes; }
  free(s.col_to_row); free(s.layer); free(s.queue); free(s.col_dead);
  free(in_S); free(in_T); free(q);
  return cost;
}

/* ------------------------------------------------------------------ */
/* LP-duality certificate                                              */
/* ------------------------------------------------------------------ */

/* Returns 0 when (row_to_col, u, v, cost) is a proven optimum:
 *   1  row_to_col out of range
 *   2  two rows share a column
 *   3  dual infeasible: u_i + v_j > C[i][j] for some (i, j)
 *   4  matched pair not tight
 *   5  v_j > 0 for some column (n < m), or v_j != 0 on an unmatched column
 *   6  cost != sum of matched costs
 *   7  cost != sum(u) + sum(v)
 *   8  bad sizes / allocation failure
 * Weak duality makes 0 a proof of optimality. */
int oracle_check_certificate(const int32_t *C, int64_t ldc, int n, int m,
                             const int32_t *row_to_col, const int64_t *u,
                             const int64_t *v, int64_t cost) {
  if (n < 0 || m < n || (n > 0 && ldc < m)) return 8;
  char *seen = calloc(m ? m : 1, 1);
  if (!seen) return 8;
  int rc = 0;
  for (int i = 0; i < n && !rc; ++i) {
    int j = row_to_col[i];
    if (j < 0 || j >= m) rc = 1;
    else if (seen[j]) rc = 2;
    else seen[j] = 1;
  }
  for (int i = 0; i < n && !rc; ++i)
    for (int j = 0; j < m; ++j)
      if (u[i] + v[j] > AT(C, ldc, i, j)) { rc = 3; break; }
  for (int i = 0; i < n && !rc; ++i)
    if (u[i] + v[row_to_col[i]] != AT(C, ldc, i, row_to_col[i])) rc = 4;
  if (!rc && m > n)
    for (int j = 0; j < m; ++j)
      if (v[j] > 0 || (!seen[j] && v[j] != 0)) { rc = 5; break; }
  if (!rc) {
    int64_t prim = 0, dual = 0;
    for (int i = 0; i < n; ++i) prim += AT(C, ldc, i, row_to_col[i]);
    for (int i = 0; i < n; ++i) dual += u[i];
    for (int j = 0; j < m; ++j) dual += v[j];
    if (prim != cost) rc = 6;
    else if (dual != cost) rc = 7;
  }
  free(seen);
  return rc;
}

/* ------------------------------------------------------------------------
 * oracle_auction: the auction algorithm with epsilon-scaling (paper,
 * Sec. 2.3.3 "The auction algorithm" and Sec. 4.1 "Auction": bidders raise
 * object prices until every bidder holds an object that is within epsilon
 * of its best; with integral costs the result is exact once epsilon is
 * below 1/n; epsilon-scaling lowers epsilon in stages, "AuctionScaled").
 *
 * Readings (the paper gives no schedule or parallel form):
 *   - Minimisation form: bidder i values object j at w_ij = C'[i][j] + p_j
 *     and bids for the object of lowest w (lowest index on ties), raising
 *     its price by (second-lowest w - lowest w) + eps (by eps when m = 1).
 *   - Exactness: costs are shifted to start at 0 and multiplied by N + 1
 *     (N = m bidders after padding), and the last stage runs at eps = 1;
 *     an eps-optimal assignment of the scaled problem is then within
 *     N < N + 1 of the scaled optimum, and every assignment's scaled cost is
 *     a multiple of N + 1, so it is optimal ("epsilon < 1/n").
 *   - n < m: m - n dummy bidders whose costs are all 0 (a constant row does
 *     not change which assignment of the real rows is optimal).
 *   - Parallel (Jacobi) rounds, the parallel bidding the paper mentions:
 *     every unassigned bidder bids against the prices at the start of the
 *     round; an object that received bids goes to the highest bid (lowest
 *     bidder index on ties), takes that bid as its price and releases its
 *     previous holder.  The outcome of a round does not depend on the
 *     order in which the bids are computed.
 *   - Schedule: eps_0 = max(1, R' / 8) with R' = (N + 1) (max C - min C);
 *     each later stage divides eps by 4 (at least 1), keeps the prices and
 *     restarts with every bidder unassigned; the stage at eps = 1 is last.
 *
 * Outputs row_to_col[n], the final prices p[m] (scaled units) and stats:
 * [0] stages, [1] rounds, [2] bids (all bidders), [3] bids of real rows.
 * Returns the cost under C (int64), INT64_MIN on bad sizes, allocation
 * failure or a scaled range above 2^50.
 * ---------------------------------------------------------------------- */
int64_t oracle_auction(const int32_t *C, int64_t ldc, int n, int m, int32_t *row_to_col,
                       int64_t *prices, int64_t *stats) {
  if (n < 0 || m < n || (n > 0 && ldc < m)) return INT64_MIN;
  int64_t st[4] = {0, 0, 0, 0};
  if (n == 0) {
    if (prices) memset(prices, 0, sizeof(int64_t) * (size_t)m);
    if (stats) memcpy(stats, st, sizeof(st));
    return 0;
  }
  const int N = m;
  int64_t cmin = C[0], cmax = C[0];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) {
      const int64_t c = C[(int64_t)i * ldc + j];
      if (c < cmin) cmin = c;
      if (c > cmax) cmax = c;
    }
  const int64_t scale = (int64_t)N + 1;
  const int64_t range = (cmax - cmin) * scale;
  if (range > ((int64_t)1 << 50)) return INT64_MIN;
  int64_t *p = calloc((size_t)N, sizeof(int64_t));
  int32_t *holder = malloc(sizeof(int32_t) * (size_t)N);  /* object -> bidder or -1 */
  int32_t *held = malloc(sizeof(int32_t) * (size_t)N);    /* bidder -> object or -1 */
  int32_t *bid_obj = malloc(sizeof(int32_t) * (size_t)N); /* -1: no bid this round */
  int64_t *bid_amt = malloc(sizeof(int64_t) * (size_t)N);
  int32_t *win = malloc(sizeof(int32_t) * (size_t)N);     /* object -> best bidder */
  if (!p || !holder || !held || !bid_obj || !bid_amt || !win) {
    free(p); free(holder); free(held); free(bid_obj); free(bid_amt); free(win);
    return INT64_MIN;
  }
  int64_t eps = range / 8;
  if (eps < 1) eps = 1;
  for (;;) {
    ++st[0];
    for (int k = 0; k < N; ++k) holder[k] = held[k] = -1;
    for (;;) {
      /* every unassigned bidder bids against the round-start prices */
      int bidders = 0;
      for (int i = 0; i < N; ++i) {
        bid_obj[i] = -1;
        if (held[i] >= 0) continue;
        int j1 = -1;
        int64_t w1 = OR_INF, w2 = OR_INF;
        for (int j = 0; j < N; ++j) {
          const int64_t c = i < n ? (C[(int64_t)i * ldc + j] - cmin) * scale : 0;
          const int64_t w = c + p[j];
          if (w < w1) {
            w2 = w1;
            w1 = w;
            j1 = j;
          } else if (w < w2) {
            w2 = w;
          }
        }
        if (N == 1) w2 = w1;
        bid_obj[i] = j1;
        bid_amt[i] = p[j1] + (w2 - w1) + eps;
        ++bidders;
        ++st[2];
        if (i < n) ++st[3];
      }
      if (bidders == 0) break;
      ++st[1];
      /* highest bid per object, lowest bidder index among equal bids */
      for (int j = 0; j < N; ++j) win[j] = -1;
      for (int i = 0; i < N; ++i) {
        const int j = bid_obj[i];
        if (j >= 0 && (win[j] < 0 || bid_amt[i] > bid_amt[win[j]])) win[j] = i;
      }
      /* the winner takes the object at its bid; the previous holder is
         released and bids in the next round */
      for (int j = 0; j < N; ++j) {
        if (win[j] < 0) continue;
        p[j] = bid_amt[win[j]];
        if (holder[j] >= 0) held[holder[j]] = -1;
        holder[j] = win[j];
        held[win[j]] = j;
      }
    }
    if (eps == 1) break;
    eps /= 4;
    if (eps < 1) eps = 1;
  }
  int64_t cost = 0;
  for (int i = 0; i < n; ++i) {
    row_to_col[i] = held[i];
    cost += C[(int64_t)i * ldc + held[i]];
  }
  if (prices) memcpy(prices, p, sizeof(int64_t) * (size_t)N);
  if (stats) memcpy(stats, st, sizeof(st));
  free(p); free(holder); free(held); free(bid_obj); free(bid_amt); free(win);
  return cost;
}
