/*
 * gabp_oracle.c -- plain, slow, FP64 CPU reference of Gaussian belief propagation
 * (GaBP) for A x = b with A sparse and symmetric.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the GPU solver is
 * checked against.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may build, load or call it.  It shares no code, header,
 * table or helper with the CUDA solver.
 *
 * What it computes (paper: Bickson, "Gaussian Belief Propagation: Theory and
 * Application"):
 *
 *   orc_gabp_naive      Algorithm 1 ("naive GaBP"), parallel (synchronous)
 *                       schedule: two message stores, the previous round's and
 *                       the current round's (Sec. "The Gaussian BP Algorithm",
 *                       the paragraph on parallel vs serial scheduling).  Every
 *                       message i->j is rebuilt from the explicit sum over
 *                       N(i)\j (eq_prec, eq_mean, eq_prec_message, eq_mean_message),
 *                       in the (precision P, mean mu) parameterisation.
 *   orc_gabp_broadcast  Algorithm 2 ("broadcast GaBP"): every node first forms
 *                       its aggregate P~_i, mu~_i over all of N(i); each message
 *                       then subtracts the reverse message j->i
 *                       (Sec. "GaBP Broadcast Variant").
 *   orc_gabp_serial     Algorithm 1's message rules under the serial schedule
 *                       (same paragraph: ONE message store, so messages sent
 *                       earlier in a sweep are seen by the nodes that fire later).
 *                       A sweep fires the nodes colour by colour (colour 0 first)
 *                       and, within a colour, in index order; nodes of one colour
 *                       share no edge, so this is one sequential order.  Firing
 *                       node i rebuilds every message i -> j from the current
 *                       messages into i.
 *   orc_colour_greedy   the colouring used by the serial sweeps: nodes in index
 *                       order, each taking the smallest colour not used by a
 *                       lower-indexed neighbour.
 *
 * Message storage: the input is the FULL symmetric CSR (diagonal included,
 * columns sorted within rows).  For row i, the slot p with col[p] = k != i holds
 * the message k -> i (P_ki, mu_ki).  The diagonal slots hold nothing.
 *
 * Stopping rules (the paper is not uniform here):
 *   stop_rule 0: after round t's messages are computed, form the tentative
 *                marginal means x_t (Alg. 1 step 4) and stop when
 *                ||b - A x_t||_2 <= tol * ||b||_2 ;
 *   stop_rule 1: stop when every message changed by less than tol in absolute
 *                value between rounds t-1 and t (the rule of the paper's
 *                numerical-examples chapter).
 * Either way the run also stops at t = max_iter.  With b = 0 the answer is
 * x = 0 after 0 rounds.
 *
 * Return codes: 0 converged, 1 not converged within max_iter, 2 diverged
 * (a non-finite value appeared), 3 breakdown (a cavity precision P_{i\j} or a
 * marginal precision P_i is exactly zero; the paper's Matlab listing asserts
 * the same), -1 invalid input.
 *
 * Threads: the same file is also built with OpenMP (for the host-cores timing
 * baseline).  The row loops of the parallel schedule then run on all cores:
 * every row writes only its own outputs and the slots that receive its
 * messages, so the arithmetic per message is unchanged; only the order of the
 * residual and norm sums differs.  The serial schedule stays sequential.
 * Without OpenMP the pragmas are ignored.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_NOT_CONVERGED 1
#define ORC_DIVERGED 2
#define ORC_BREAKDOWN 3
#define ORC_INVALID (-1)

/* slot of column k in row i, or -1 (linear scan: slow and obviously right) */
static long slot_of(const int *rowptr, const int *col, int i, int k) {
  for (long p = rowptr[i]; p < rowptr[i + 1]; ++p)
    if (col[p] == k) return p;
  return -1;
}

/* A_ii, or 0 if row i stores no diagonal entry */
static double diag_entry(const int *rowptr, const int *col, const double *val, int i) {
  long p = slot_of(rowptr, col, i, i);
  return p < 0 ? 0.0 : val[p];
}

/* Input checks: one nonzero diagonal per row, symmetric pattern and values,
 * no stored zero off the diagonal. */
static int check_input(int n, const int *rowptr, const int *col, const double *val) {
  if (n < 0) return ORC_INVALID;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1024) reduction(| : bad)
  for (int i = 0; i < n; ++i) {
    if (diag_entry(rowptr, col, val, i) == 0.0) bad = 1;
    for (long p = rowptr[i]; p < rowptr[i + 1] && !bad; ++p) {
      int k = col[p];
      if (k < 0 || k >= n) { bad = 1; break; }
      if (k == i) continue;
      if (val[p] == 0.0) { bad = 1; break; }
      long q = slot_of(rowptr, col, k, i);
      if (q < 0 || val[q] != val[p]) bad = 1;
    }
  }
  return bad ? ORC_INVALID : ORC_OK;
}

/* Alg. 1 step 4: marginal precision P_i = P_ii + sum_k P_ki and marginal mean
 * mu_i = (P_ii mu_ii + sum_k P_ki mu_ki) / P_i over all k in N(i). */
static int infer(int n, const int *rowptr, const int *col, const double *val, const double *b,
                 const double *Pm, const double *Mm, double *x, double *Pi) {
  int broken = 0;
#pragma omp parallel for schedule(static) reduction(| : broken)
  for (int i = 0; i < n; ++i) {
    double Pii = diag_entry(rowptr, col, val, i);
    double muii = b[i] / Pii;
    double P = Pii, num = Pii * muii;
    for (long p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      if (col[p] == i) continue;
      P += Pm[p];
      num += Pm[p] * Mm[p];
    }
    if (P == 0.0) {
      broken = 1;
      continue;
    }
    Pi[i] = P;
    x[i] = num / P;
  }
  return broken ? ORC_BREAKDOWN : ORC_OK;
}

/* ||b - A x||_2 and ||b||_2 over the full matrix */
static void residual(int n, const int *rowptr, const int *col, const double *val, const double *b,
                     const double *x, double *rnorm, double *bnorm) {
  double rr = 0.0, bb = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : rr, bb)
  for (int i = 0; i < n; ++i) {
    double ax = 0.0;
    for (long p = rowptr[i]; p < rowptr[i + 1]; ++p) ax += val[p] * x[col[p]];
    double r = b[i] - ax;
    rr += r * r;
    bb += b[i] * b[i];
  }
  *rnorm = sqrt(rr);
  *bnorm = sqrt(bb);
}

static int all_finite(long m, const double *a) {
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (long p = 0; p < m; ++p)
    if (!isfinite(a[p])) bad = 1;
  return !bad;
}

/* One synchronous round of Algorithm 1: from the round t-1 store (Po, Mo)
 * compute every message i -> j into the round t store (Pn, Mn). */
static int round_naive(int n, const int *rowptr, const int *col, const double *val, const double *b,
                       const double *Po, const double *Mo, double *Pn, double *Mn) {
  int broken = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(| : broken)
  for (int i = 0; i < n; ++i) {
    double Pii = diag_entry(rowptr, col, val, i); /* P_ii = A_ii */
    double muii = b[i] / Pii;                       /* mu_ii = b_i / A_ii */
    for (long q = rowptr[i]; q < rowptr[i + 1]; ++q) {
      int j = col[q];
      if (j == i) continue;
      /* eq_prec / eq_mean: cavity over N(i) \ j */
      double Pcav = Pii;
      double hcav = Pii * muii;
      for (long p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        int k = col[p];
        if (k == i || k == j) continue;
        Pcav += Po[p];
        hcav += Po[p] * Mo[p];
      }
      if (Pcav == 0.0) {
        broken = 1;
        continue;
      }
      double Aij = val[q];
      long dst = slot_of(rowptr, col, j, i); /* row j's slot that receives i -> j */
      Pn[dst] = -Aij * Aij / Pcav;           /* Alg. 1: P_ij = -A_ij^2 / P_{i\j} */
      Mn[dst] = hcav / Aij;                  /* Alg. 1: mu_ij = P_{i\j} mu_{i\j} / A_ij */
    }
  }
  return broken ? ORC_BREAKDOWN : ORC_OK;
}

/* One synchronous round of Algorithm 2: aggregates first, then each message
 * subtracts the reverse message j -> i. */
static int round_broadcast(int n, const int *rowptr, const int *col, const double *val, const double *b,
                           const double *Po, const double *Mo, double *Pn, double *Mn,
                           double *Ptil, double *Mtil) {
  int broken = 0;
#pragma omp parallel for schedule(static) reduction(| : broken)
  for (int i = 0; i < n; ++i) {
    double Pii = diag_entry(rowptr, col, val, i);
    double muii = b[i] / Pii;
    double P = Pii, num = Pii * muii;
    for (long p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      if (col[p] == i) continue;
      P += Po[p];
      num += Po[p] * Mo[p];
    }
    if (P == 0.0) broken = 1; /* mu~_i = P~_i^{-1}(...) needs P~_i != 0 */
    Ptil[i] = P;
    Mtil[i] = num / P;
  }
  if (broken) return ORC_BREAKDOWN;
#pragma omp parallel for schedule(dynamic, 256) reduction(| : broken)
  for (int i = 0; i < n; ++i) {
    for (long q = rowptr[i]; q < rowptr[i + 1]; ++q) {
      int j = col[q];
      if (j == i) continue;
      double Pji = Po[q], muji = Mo[q]; /* message j -> i lives in row i, slot q */
      double Pcav = Ptil[i] - Pji;      /* P_{i\j} = P~_i - P_ji */
      if (Pcav == 0.0) {
        broken = 1;
        continue;
      }
      double Aij = val[q];
      long dst = slot_of(rowptr, col, j, i);
      Pn[dst] = -Aij * Aij / Pcav;                        /* Alg. 2 */
      Mn[dst] = (Ptil[i] * Mtil[i] - Pji * muji) / Aij;   /* Alg. 2 */
    }
  }
  return broken ? ORC_BREAKDOWN : ORC_OK;
}

/* Greedy colouring in index order; returns the number of colours. */
int orc_colour_greedy(int n, const int *rowptr, const int *col, int *colour) {
  int ncol = 0;
  int *used = calloc((size_t)n + 1, sizeof(int)); /* used[c] == i + 1: colour c taken by a lower neighbour of i */
  if (!used) return -1;
  for (int i = 0; i < n; ++i) {
    for (long p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      int k = col[p];
      if (k < i) used[colour[k]] = i + 1;
    }
    int c = 0;
    while (used[c] == i + 1) ++c;
    colour[i] = c;
    if (c + 1 > ncol) ncol = c + 1;
  }
  free(used);
  return ncol;
}

/* One serial sweep: nodes fire colour by colour, each node rebuilding its
 * outgoing messages (Algorithm 1's rules, cavity sums over N(i)\j) from the
 * CURRENT store, which it updates in place. */
static int sweep_serial(int n, const int *rowptr, const int *col, const double *val, const double *b,
                        const int *colour, int ncol, double *Pm, double *Mm) {
  for (int c = 0; c < ncol; ++c) {
    for (int i = 0; i < n; ++i) {
      if (colour[i] != c) continue;
      double Pii = diag_entry(rowptr, col, val, i);
      double muii = b[i] / Pii;
      for (long q = rowptr[i]; q < rowptr[i + 1]; ++q) {
        int j = col[q];
        if (j == i) continue;
        double Pcav = Pii, hcav = Pii * muii;
        for (long p = rowptr[i]; p < rowptr[i + 1]; ++p) {
          int k = col[p];
          if (k == i || k == j) continue;
          Pcav += Pm[p];
          hcav += Pm[p] * Mm[p];
        }
        if (Pcav == 0.0) return ORC_BREAKDOWN;
        double Aij = val[q];
        long dst = slot_of(rowptr, col, j, i); /* row j's slot that receives i -> j */
        Pm[dst] = -Aij * Aij / Pcav;
        Mm[dst] = hcav / Aij;
      }
    }
  }
  return ORC_OK;
}

static int run(int variant, int n, const int *rowptr, const int *col, const double *val, const double *b,
               int max_iter, double tol, int stop_rule, double *x, double *Pi, int *iters,
               double *relres, double *Pmsg, double *Mmsg, int checked) {
  int rc = checked ? check_input(n, rowptr, col, val) : ORC_OK;
  if (rc != ORC_OK) return rc;
  long nnz = rowptr[n];
  int *colour = NULL, ncol = 0;
  if (variant == 2) {
    colour = calloc((size_t)n + 1, sizeof(int));
    if (!colour) return ORC_INVALID;
    ncol = orc_colour_greedy(n, rowptr, col, colour);
  }
  double *Po = calloc(nnz + 1, sizeof(double)), *Mo = calloc(nnz + 1, sizeof(double));
  double *Pn = calloc(nnz + 1, sizeof(double)), *Mn = calloc(nnz + 1, sizeof(double));
  double *Pt = calloc(n + 1, sizeof(double)), *Mt = calloc(n + 1, sizeof(double));
  if (!Po || !Mo || !Pn || !Mn || !Pt || !Mt) { rc = ORC_INVALID; goto done; }

  double rn, bn;
  residual(n, rowptr, col, val, b, Mt /* zeros */, &rn, &bn);
  *iters = 0;
  /* Alg. 1 step 1: all messages start at P = 0, mu = 0 (calloc). */
  rc = infer(n, rowptr, col, val, b, Po, Mo, x, Pi);
  if (rc != ORC_OK) goto done;
  if (bn == 0.0) {
    for (int i = 0; i < n; ++i) x[i] = 0.0;
    *relres = 0.0;
    rc = ORC_OK;
    goto done;
  }
  residual(n, rowptr, col, val, b, x, &rn, &bn);
  *relres = rn / bn;
  rc = ORC_NOT_CONVERGED;
  for (int t = 1; t <= max_iter; ++t) {
    int r;
    if (variant == 2) { /* serial: Pn/Mn keep the previous sweep for the change test */
      memcpy(Pn, Po, nnz * sizeof(double));
      memcpy(Mn, Mo, nnz * sizeof(double));
      r = sweep_serial(n, rowptr, col, val, b, colour, ncol, Pn, Mn);
    } else {
      r = variant == 0 ? round_naive(n, rowptr, col, val, b, Po, Mo, Pn, Mn)
                       : round_broadcast(n, rowptr, col, val, b, Po, Mo, Pn, Mn, Pt, Mt);
    }
    if (r != ORC_OK) { rc = r; *iters = t; break; }
    double maxchange = 0.0;
#pragma omp parallel for schedule(static) reduction(max : maxchange)
    for (long p = 0; p < nnz; ++p) {
      double dP = fabs(Pn[p] - Po[p]), dM = fabs(Mn[p] - Mo[p]);
      if (dP > maxchange) maxchange = dP;
      if (dM > maxchange) maxchange = dM;
    }
    double *tp = Po; Po = Pn; Pn = tp;
    tp = Mo; Mo = Mn; Mn = tp;
    *iters = t;
    r = infer(n, rowptr, col, val, b, Po, Mo, x, Pi);
    if (r != ORC_OK) { rc = r; break; }
    if (!all_finite(nnz, Po) || !all_finite(nnz, Mo) || !all_finite(n, x)) { rc = ORC_DIVERGED; break; }
    residual(n, rowptr, col, val, b, x, &rn, &bn);
    *relres = rn / bn;
    if (!isfinite(rn)) { rc = ORC_DIVERGED; break; }
    if (stop_rule == 0 ? (rn <= tol * bn) : (maxchange < tol)) { rc = ORC_OK; break; }
  }
  if (Pmsg) memcpy(Pmsg, Po, nnz * sizeof(double));
  if (Mmsg) memcpy(Mmsg, Mo, nnz * sizeof(double));
done:
  free(Po); free(Mo); free(Pn); free(Mn); free(Pt); free(Mt); free(colour);
  return rc;
}

/* Exported entry points.  x, Pi: [n].  Pmsg, Mmsg: [nnz] in the input's slot
 * order (message col[p] -> row), may be NULL.  relres receives the relative
 * residual of the last x_t formed. */
int orc_gabp_naive(int n, const int *rowptr, const int *col, const double *val, const double *b,
                   int max_iter, double tol, int stop_rule, double *x, double *Pi, int *iters,
                   double *relres, double *Pmsg, double *Mmsg) {
  *relres = NAN;
  return run(0, n, rowptr, col, val, b, max_iter, tol, stop_rule, x, Pi, iters, relres, Pmsg, Mmsg, 1);
}

int orc_gabp_broadcast(int n, const int *rowptr, const int *col, const double *val, const double *b,
                       int max_iter, double tol, int stop_rule, double *x, double *Pi, int *iters,
                       double *relres, double *Pmsg, double *Mmsg) {
  *relres = NAN;
  return run(1, n, rowptr, col, val, b, max_iter, tol, stop_rule, x, Pi, iters, relres, Pmsg, Mmsg, 1);
}

/* As orc_gabp_broadcast without the input checks (the caller has checked the matrix with a
 * checked call before): the timing baseline times the rounds alone. */
int orc_gabp_broadcast_unchecked(int n, const int *rowptr, const int *col, const double *val, const double *b,
                                 int max_iter, double tol, int stop_rule, double *x, double *Pi, int *iters,
                                 double *relres, double *Pmsg, double *Mmsg) {
  *relres = NAN;
  return run(1, n, rowptr, col, val, b, max_iter, tol, stop_rule, x, Pi, iters, relres, Pmsg, Mmsg, 0);
}

/* Threads the OpenMP build uses (1 without OpenMP). */
int orc_threads(void) {
#ifdef _OPENMP
  int t = 1;
#pragma omp parallel
#pragma omp single
  t = omp_get_num_threads();
  return t;
#else
  return 1;
#endif
}

int orc_gabp_serial(int n, const int *rowptr, const int *col, const double *val, const double *b,
                    int max_iter, double tol, int stop_rule, double *x, double *Pi, int *iters,
                    double *relres, double *Pmsg, double *Mmsg) {
  *relres = NAN;
  return run(2, n, rowptr, col, val, b, max_iter, tol, stop_rule, x, Pi, iters, relres, Pmsg, Mmsg, 1);
}
