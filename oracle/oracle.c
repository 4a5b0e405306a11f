/*
 * FP64 CPU oracle for the per-frame illumination decomposition solve of
 * "Real-Time Global Illumination Decomposition of Videos" (Sec. 5 and Sec. 6).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code with the CUDA library.
 *
 * Style: plain, slow, FP64.  Every energy term is written as the list of
 * its least-squares residual rows (value f and the sparse Jacobian row a_j), in
 * the order the paper lists the terms.  The Gauss-Newton normal-equation
 * products J^T J p, -J^T F and diag(J^T J) are then the textbook sums over those
 * rows, so a reader can check each term against its equation by eye.
 *
 * Order of the FP64 sums (fixed, whatever the thread count, so results are the
 * same bit for bit on 1 or many threads; OpenMP only spreads the work for the
 * benchmark's timing): the residual rows are visited in stripes of OR_STRIPE
 * image rows, all even stripes first, then all odd ones, each stripe in row
 * order.  A row generated at image row y touches unknowns of rows y - 3 .. y + 3
 * only (the widest reach is the consistency pairs' radius 3), so two stripes of
 * one phase never touch the same unknown and may run at once.  Dot products
 * and per-term energies are summed per fixed chunk (stripe), then over the
 * chunks in order.
 *
 * Unknowns per pixel (V = K + 4): r_R, r_G, r_B (r = ln R, the log reflectance
 * of eq:clustering-term) and T_0..T_K (eq:imageformation).  Layout [V][H][W].
 *
 * Readings of points the paper leaves open (each is a flag or a fixed choice):
 *   - the intensity |S| in the monochrome prior is the channel mean;
 *   - image gradients are forward differences with no residual across the
 *     border; the reflectance gradient norm groups (d/dx, d/dy) x RGB;
 *   - the consistency prior (only cited to earlier work in Sec. 5.1) pairs every
 *     pixel with a fixed set of random offsets, soft chromaticity closeness
 *     weight exp(-|C(x)-C(y)|^2 / tau^2), squared l2;
 *   - IRLS weights use the same eps = 0.002 for every reweighted term and no
 *     1/2 factor unless irls_half is set;
 *   - the non-negativity weight is 0 only for T > 0, as printed (T >= 0 if
 *     nonneg_strict is cleared);
 *   - in eq:basecolorrefinement b_k is the initially estimated base colour and
 *     Delta b_k the whole refinement, re-solved at every dense step against the
 *     current layers; the refined colours are b_k + Delta b_k.  The chromaticity
 *     regulariser is taken literally, i.e. it equals |Delta b_k|^2;
 *   - R_cluster stays the clustering's output (colours b_init) unless
 *     rcluster_follows_b is set.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_STRIPE 8   /* image rows per stripe (> 2 x 3, the widest reach of a row) */
#define OR_CHUNK 4096 /* elements per partial sum of a dot product */

/* Threads used by the parallel loops (timing only; results do not depend on it). */
void or_set_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : 1);
#else
  (void)n;
#endif
}
int or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

typedef struct {
  int H, W, K;
  double lambda_data, lambda_clustering, lambda_rsparsity, p, lambda_rconsistency,
      lambda_monochrome, lambda_isparsity, lambda_smoothness, lambda_nonneg,
      lambda_IR, lambda_CR, eps;
  int nonneg_strict; /* 1: weight 0 only for T > 0 (as printed); 0: for T >= 0 */
  int irls_half;     /* 1: majorise-minimise 1/2 factor on IRLS weights */
  int n_spatial, n_temporal;
  const int *off_spatial;  /* n_spatial x (dy, dx) */
  const int *off_temporal; /* n_temporal x (dy, dx) */
  const double *I;         /* 3 x H x W */
  const unsigned char *labels; /* H x W, base colour index k-1 */
  const double *b;         /* K x 3: b_1..b_K (b_0 is white) */
  const double *wsr;       /* H x W soft-Retinex weight */
  const double *omega_s;   /* n_spatial x H x W pair weights */
  const double *omega_t;   /* n_temporal x H x W, NULL: no temporal pairs */
  const double *rprev;     /* 3 x H x W previous frame's r, NULL: none */
  const double *b_init;    /* K x 3 initial (clustered) base colours, the anchor of
                              eq:basecolorrefinement and the colours of R_cluster */
  int rcluster_follows_b;  /* 1: r_cluster = ln b (current); 0: ln b_init */
} or_problem;

enum { T_DATA, T_CLUSTER, T_RSPARSE, T_RCONSIST, T_MONO, T_ISPARSE, T_SMOOTH, T_NONNEG, N_TERMS };
#define ALL_TERMS 0xffu
#define OR_MAXNZ 24

typedef struct {
  int term;
  double f;
  int n;
  long j[OR_MAXNZ];
  double a[OR_MAXNZ];
} or_row;

typedef void (*or_visit_fn)(const or_row *, void *);

/* b_k for k = 0..K; b_0 = (1, 1, 1) is the white illuminant (Sec. 3). */
static double base(const or_problem *pb, int k, int c) { return k == 0 ? 1.0 : pb->b[(k - 1) * 3 + c]; }

static long P_of(const or_problem *pb) { return (long)pb->H * pb->W; }
static long idx(const or_problem *pb, int v, int y, int x) { return (long)v * P_of(pb) + (long)y * pb->W + x; }
static int inside(const or_problem *pb, int y, int x) { return y >= 0 && y < pb->H && x >= 0 && x < pb->W; }

/* S_c(x) = sum_{k=0..K} b_kc T_k(x), eq:imageformation. */
static double shading(const or_problem *pb, const double *X, int c, int y, int x) {
  double s = 0;
  for (int k = 0; k <= pb->K; k++) s += base(pb, k, c) * X[idx(pb, 3 + k, y, x)];
  return s;
}

/* r_cluster(x) = ln of the clustered reflectance R_cluster(x) (Sec. 4.1): the
 * initial colour of the pixel's cluster (or the refined one, by flag). */
static double rcluster(const or_problem *pb, int c, int y, int x) {
  int k = pb->labels[(long)y * pb->W + x];
  return log(pb->rcluster_follows_b ? pb->b[k * 3 + c] : pb->b_init[k * 3 + c]);
}

static void row_begin(or_row *r, int term, double f) { r->term = term; r->f = f; r->n = 0; }
static void row_add(or_row *r, long j, double a) { r->j[r->n] = j; r->a[r->n] = a; r->n++; }

/* IRLS weight of an l_p residual norm (Sec. 5.3): lambda * (|g_old| + eps)^(p-2). */
static double irls(const or_problem *pb, double lambda, double gnorm_old, double p) {
  double w = lambda * pow(gnorm_old + pb->eps, p - 2.0);
  return pb->irls_half ? 0.5 * w : w;
}

static const int DIRS[2][2] = {{0, 1}, {1, 0}}; /* forward differences along x and y */

/*
 * Enumerate every residual row of the (IRLS-reweighted) decomposition energy
 * eq:giv-energy at state X; the reweighting constants come from state Xw.
 */
static void or_rows_range(const or_problem *pb, const double *X, const double *Xw, unsigned mask, or_visit_fn fn,
                          void *ctx, int y_begin, int y_end) {
  const int W = pb->W, K = pb->K;
  or_row row;
  for (int y = y_begin; y < y_end; y++)
    for (int x = 0; x < W; x++) {
      /* E_data, eq:data-term: sqrt(l_data) (I_c - R_c S_c), R_c = exp(r_c). */
      if (mask & (1u << T_DATA)) {
        double sl = sqrt(pb->lambda_data);
        for (int c = 0; c < 3; c++) {
          double R = exp(X[idx(pb, c, y, x)]);
          double S = shading(pb, X, c, y, x);
          double Ic = pb->I[idx(pb, c, y, x)];
          row_begin(&row, T_DATA, sl * (Ic - R * S));
          row_add(&row, idx(pb, c, y, x), -sl * R * S);
          for (int k = 0; k <= K; k++) row_add(&row, idx(pb, 3 + k, y, x), -sl * R * base(pb, k, c));
          fn(&row, ctx);
        }
      }
      /* E_clustering, eq:clustering-term: sqrt(l_cl) (r_c - r_cluster,c). */
      if (mask & (1u << T_CLUSTER)) {
        double sl = sqrt(pb->lambda_clustering);
        for (int c = 0; c < 3; c++) {
          row_begin(&row, T_CLUSTER, sl * (X[idx(pb, c, y, x)] - rcluster(pb, c, y, x)));
          row_add(&row, idx(pb, c, y, x), sl);
          fn(&row, ctx);
        }
      }
      /* E_r-sparsity, eq:reflectance-sparsity-term, IRLS on |grad r|_2^p. */
      if (mask & (1u << T_RSPARSE)) {
        double g2 = 0;
        for (int d = 0; d < 2; d++) {
          int ny = y + DIRS[d][0], nx = x + DIRS[d][1];
          if (!inside(pb, ny, nx)) continue;
          for (int c = 0; c < 3; c++) {
            double g = Xw[idx(pb, c, ny, nx)] - Xw[idx(pb, c, y, x)];
            g2 += g * g;
          }
        }
        double sw = sqrt(irls(pb, pb->lambda_rsparsity, sqrt(g2), pb->p));
        for (int d = 0; d < 2; d++) {
          int ny = y + DIRS[d][0], nx = x + DIRS[d][1];
          if (!inside(pb, ny, nx)) continue;
          for (int c = 0; c < 3; c++) {
            row_begin(&row, T_RSPARSE, sw * (X[idx(pb, c, ny, nx)] - X[idx(pb, c, y, x)]));
            row_add(&row, idx(pb, c, ny, nx), sw);
            row_add(&row, idx(pb, c, y, x), -sw);
            fn(&row, ctx);
          }
        }
      }
      /* E_r-consistency (Sec. 5.1): random spatial pairs, and temporal pairs to the previous frame. */
      if (mask & (1u << T_RCONSIST)) {
        for (int j = 0; j < pb->n_spatial; j++) {
          int ny = y + pb->off_spatial[2 * j], nx = x + pb->off_spatial[2 * j + 1];
          if (!inside(pb, ny, nx)) continue;
          double sw = sqrt(pb->lambda_rconsistency * pb->omega_s[(long)j * P_of(pb) + (long)y * W + x]);
          for (int c = 0; c < 3; c++) {
            row_begin(&row, T_RCONSIST, sw * (X[idx(pb, c, y, x)] - X[idx(pb, c, ny, nx)]));
            row_add(&row, idx(pb, c, y, x), sw);
            row_add(&row, idx(pb, c, ny, nx), -sw);
            fn(&row, ctx);
          }
        }
        if (pb->omega_t && pb->rprev)
          for (int j = 0; j < pb->n_temporal; j++) {
            int ny = y + pb->off_temporal[2 * j], nx = x + pb->off_temporal[2 * j + 1];
            if (!inside(pb, ny, nx)) continue;
            double sw = sqrt(pb->lambda_rconsistency * pb->omega_t[(long)j * P_of(pb) + (long)y * W + x]);
            for (int c = 0; c < 3; c++) {
              row_begin(&row, T_RCONSIST, sw * (X[idx(pb, c, y, x)] - pb->rprev[idx(pb, c, ny, nx)]));
              row_add(&row, idx(pb, c, y, x), sw);
              fn(&row, ctx);
            }
          }
      }
      /* E_monochrome (Sec. 5.2): sqrt(l_mono w_SR) (S_c - |S|), |S| = channel mean of S. */
      if (mask & (1u << T_MONO)) {
        double sw = sqrt(pb->lambda_monochrome * pb->wsr[(long)y * W + x]);
        double Sbar = 0;
        for (int c = 0; c < 3; c++) Sbar += shading(pb, X, c, y, x) / 3.0;
        for (int c = 0; c < 3; c++) {
          row_begin(&row, T_MONO, sw * (shading(pb, X, c, y, x) - Sbar));
          for (int k = 0; k <= K; k++) {
            double bbar = (base(pb, k, 0) + base(pb, k, 1) + base(pb, k, 2)) / 3.0;
            row_add(&row, idx(pb, 3 + k, y, x), sw * (base(pb, k, c) - bbar));
          }
          fn(&row, ctx);
        }
      }
      /* E_i-sparsity, eq:shading-sparsity-term: l1 of T_1..T_K, IRLS. */
      if (mask & (1u << T_ISPARSE))
        for (int k = 1; k <= K; k++) {
          double sw = sqrt(irls(pb, pb->lambda_isparsity, fabs(Xw[idx(pb, 3 + k, y, x)]), 1.0));
          row_begin(&row, T_ISPARSE, sw * X[idx(pb, 3 + k, y, x)]);
          row_add(&row, idx(pb, 3 + k, y, x), sw);
          fn(&row, ctx);
        }
      /* E_smoothness, eq:smoothness-term: anisotropic l1 of grad T_k, k = 0..K, IRLS. */
      if (mask & (1u << T_SMOOTH))
        for (int k = 0; k <= K; k++)
          for (int d = 0; d < 2; d++) {
            int ny = y + DIRS[d][0], nx = x + DIRS[d][1];
            if (!inside(pb, ny, nx)) continue;
            double gold = Xw[idx(pb, 3 + k, ny, nx)] - Xw[idx(pb, 3 + k, y, x)];
            double sw = sqrt(irls(pb, pb->lambda_smoothness, fabs(gold), 1.0));
            row_begin(&row, T_SMOOTH, sw * (X[idx(pb, 3 + k, ny, nx)] - X[idx(pb, 3 + k, y, x)]));
            row_add(&row, idx(pb, 3 + k, ny, nx), sw);
            row_add(&row, idx(pb, 3 + k, y, x), -sw);
            fn(&row, ctx);
          }
      /* E_non-neg, eq:nonnegativityterm, reweighted as w_k T_k^2 (Sec. 5.3.1). */
      if (mask & (1u << T_NONNEG))
        for (int k = 0; k <= K; k++) {
          double Told = Xw[idx(pb, 3 + k, y, x)];
          int free_ = pb->nonneg_strict ? (Told > 0) : (Told >= 0);
          double w = free_ ? 0.0 : 1.0 / (fabs(Told) + pb->eps);
          if (pb->irls_half) w *= 0.5;
          double sw = sqrt(pb->lambda_nonneg * w);
          row_begin(&row, T_NONNEG, sw * X[idx(pb, 3 + k, y, x)]);
          row_add(&row, idx(pb, 3 + k, y, x), sw);
          fn(&row, ctx);
        }
    }
}

/* Every row in image-row order (visitors whose result depends on the order). */
static void or_rows(const or_problem *pb, const double *X, const double *Xw, unsigned mask, or_visit_fn fn, void *ctx) {
  or_rows_range(pb, X, Xw, mask, fn, ctx, 0, pb->H);
}

/* Every row, in the striped order described at the top of the file; for
 * visitors that only add into the unknowns the row touches. */
static void or_rows_striped(const or_problem *pb, const double *X, const double *Xw, unsigned mask, or_visit_fn fn,
                            void *ctx) {
  const int ns = (pb->H + OR_STRIPE - 1) / OR_STRIPE;
  for (int phase = 0; phase < 2; phase++) {
#pragma omp parallel for schedule(static)
    for (int st = phase; st < ns; st += 2) {
      const int y1 = (st + 1) * OR_STRIPE < pb->H ? (st + 1) * OR_STRIPE : pb->H;
      or_rows_range(pb, X, Xw, mask, fn, ctx, st * OR_STRIPE, y1);
    }
  }
}

/* ---------------- normal-equation products over the rows ---------------- */

typedef struct { const double *p; double *q; } apply_ctx;
static void visit_apply(const or_row *r, void *vc) {
  apply_ctx *c = (apply_ctx *)vc;
  double s = 0;
  for (int i = 0; i < r->n; i++) s += r->a[i] * c->p[r->j[i]];
  for (int i = 0; i < r->n; i++) c->q[r->j[i]] += r->a[i] * s;
}

static void visit_rhs(const or_row *r, void *vc) {
  double *g = (double *)vc;
  for (int i = 0; i < r->n; i++) g[r->j[i]] -= r->a[i] * r->f;
}

static void visit_diag(const or_row *r, void *vc) {
  double *d = (double *)vc;
  for (int i = 0; i < r->n; i++) d[r->j[i]] += r->a[i] * r->a[i];
}

static void visit_sq(const or_row *r, void *vc) { ((double *)vc)[r->term] += r->f * r->f; }

typedef struct { double *F; long n, cap; int *term; } res_ctx;
static void visit_res(const or_row *r, void *vc) {
  res_ctx *c = (res_ctx *)vc;
  if (c->n < c->cap) {
    c->F[c->n] = r->f;
    if (c->term) c->term[c->n] = r->term;
  }
  c->n++;
}

static long nvar(const or_problem *pb) { return (long)(pb->K + 4) * P_of(pb); }

/* q = J^T J p (Gauss-Newton normal matrix, eq:optimization). */
void or_apply(const or_problem *pb, const double *X, const double *Xw, unsigned mask, const double *p, double *q) {
  memset(q, 0, sizeof(double) * nvar(pb));
  apply_ctx c = {p, q};
  or_rows_striped(pb, X, Xw, mask, visit_apply, &c);
}

/* g = -J^T F (right-hand side of the normal equations). */
void or_rhs(const or_problem *pb, const double *X, const double *Xw, unsigned mask, double *g) {
  memset(g, 0, sizeof(double) * nvar(pb));
  or_rows_striped(pb, X, Xw, mask, visit_rhs, g);
}

/* d = diag(J^T J), the Jacobi preconditioner's inverse. */
void or_diag(const or_problem *pb, const double *X, const double *Xw, unsigned mask, double *d) {
  memset(d, 0, sizeof(double) * nvar(pb));
  or_rows_striped(pb, X, Xw, mask, visit_diag, d);
}

/* Per-term sum of squared residuals |F_t|^2 (the IRLS surrogate energy). */
void or_surrogate(const or_problem *pb, const double *X, const double *Xw, unsigned mask, double *E) {
  memset(E, 0, sizeof(double) * N_TERMS);
  or_rows(pb, X, Xw, mask, visit_sq, E);
}

/* Stacked residual vector F; returns the row count (writes at most cap). */
long or_residuals(const or_problem *pb, const double *X, const double *Xw, unsigned mask, double *F, int *term, long cap) {
  res_ctx c = {F, 0, cap, term};
  or_rows(pb, X, Xw, mask, visit_res, &c);
  return c.n;
}

/* ---------------- exact energy (Sec. 5, eq:giv-energy) ---------------- */

/* E[0..7] = E_data, E_clustering, E_r-sparsity, E_r-consistency, E_monochrome,
 * E_i-sparsity, E_smoothness, E_non-neg, each as its equation defines it
 * (the l1 / l_p / max terms exactly, not their IRLS surrogates). */
static void or_energy_range(const or_problem *pb, const double *X, double *E, int y_begin, int y_end) {
  const int W = pb->W, K = pb->K;
  for (int y = y_begin; y < y_end; y++)
    for (int x = 0; x < W; x++) {
      long px = (long)y * W + x;
      double S[3], Sbar = 0;
      for (int c = 0; c < 3; c++) { S[c] = shading(pb, X, c, y, x); Sbar += S[c] / 3.0; }
      for (int c = 0; c < 3; c++) {
        double e = pb->I[idx(pb, c, y, x)] - exp(X[idx(pb, c, y, x)]) * S[c];
        E[T_DATA] += pb->lambda_data * e * e;
        double d = X[idx(pb, c, y, x)] - rcluster(pb, c, y, x);
        E[T_CLUSTER] += pb->lambda_clustering * d * d;
        E[T_MONO] += pb->lambda_monochrome * pb->wsr[px] * (S[c] - Sbar) * (S[c] - Sbar);
      }
      double g2 = 0;
      for (int d = 0; d < 2; d++) {
        int ny = y + DIRS[d][0], nx = x + DIRS[d][1];
        if (!inside(pb, ny, nx)) continue;
        for (int c = 0; c < 3; c++) {
          double g = X[idx(pb, c, ny, nx)] - X[idx(pb, c, y, x)];
          g2 += g * g;
        }
      }
      E[T_RSPARSE] += pb->lambda_rsparsity * pow(sqrt(g2), pb->p);
      for (int j = 0; j < pb->n_spatial; j++) {
        int ny = y + pb->off_spatial[2 * j], nx = x + pb->off_spatial[2 * j + 1];
        if (!inside(pb, ny, nx)) continue;
        for (int c = 0; c < 3; c++) {
          double d = X[idx(pb, c, y, x)] - X[idx(pb, c, ny, nx)];
          E[T_RCONSIST] += pb->lambda_rconsistency * pb->omega_s[(long)j * P_of(pb) + px] * d * d;
        }
      }
      if (pb->omega_t && pb->rprev)
        for (int j = 0; j < pb->n_temporal; j++) {
          int ny = y + pb->off_temporal[2 * j], nx = x + pb->off_temporal[2 * j + 1];
          if (!inside(pb, ny, nx)) continue;
          for (int c = 0; c < 3; c++) {
            double d = X[idx(pb, c, y, x)] - pb->rprev[idx(pb, c, ny, nx)];
            E[T_RCONSIST] += pb->lambda_rconsistency * pb->omega_t[(long)j * P_of(pb) + px] * d * d;
          }
        }
      for (int k = 1; k <= K; k++) E[T_ISPARSE] += pb->lambda_isparsity * fabs(X[idx(pb, 3 + k, y, x)]);
      for (int k = 0; k <= K; k++) {
        for (int d = 0; d < 2; d++) {
          int ny = y + DIRS[d][0], nx = x + DIRS[d][1];
          if (!inside(pb, ny, nx)) continue;
          E[T_SMOOTH] += pb->lambda_smoothness * fabs(X[idx(pb, 3 + k, ny, nx)] - X[idx(pb, 3 + k, y, x)]);
        }
        E[T_NONNEG] += pb->lambda_nonneg * fmax(-X[idx(pb, 3 + k, y, x)], 0.0);
      }
    }
}

void or_energy(const or_problem *pb, const double *X, double *E) {
  const int ns = (pb->H + OR_STRIPE - 1) / OR_STRIPE;
  double *part = calloc((size_t)ns * N_TERMS, sizeof(double));
#pragma omp parallel for schedule(static)
  for (int st = 0; st < ns; st++) {
    const int y1 = (st + 1) * OR_STRIPE < pb->H ? (st + 1) * OR_STRIPE : pb->H;
    or_energy_range(pb, X, part + (long)st * N_TERMS, st * OR_STRIPE, y1);
  }
  memset(E, 0, sizeof(double) * N_TERMS);
  for (int st = 0; st < ns; st++)
    for (int t = 0; t < N_TERMS; t++) E[t] += part[(long)st * N_TERMS + t];
  free(part);
}

/* ---------------- Gauss-Newton step with Jacobi-PCG (Sec. 6) ---------------- */

static double dot(const double *a, const double *b, long n) {
  const long nc = (n + OR_CHUNK - 1) / OR_CHUNK;
  double *part = malloc(sizeof(double) * (nc > 0 ? nc : 1));
#pragma omp parallel for schedule(static)
  for (long c = 0; c < nc; c++) {
    double s = 0;
    const long e = (c + 1) * OR_CHUNK < n ? (c + 1) * OR_CHUNK : n;
    for (long i = c * OR_CHUNK; i < e; i++) s += a[i] * b[i];
    part[c] = s;
  }
  double s = 0;
  for (long c = 0; c < nc; c++) s += part[c];
  free(part);
  return s;
}

/*
 * Solve J^T J delta = -J^T F at X by exactly M steps of textbook preconditioned
 * conjugate gradient (Sec. 6.1: "16 steps of ... preconditioned conjugate
 * gradient"), Jacobi preconditioner M^-1 = diag(J^T J)^-1, delta_0 = 0, no early
 * exit.  A zero denominator makes that step's alpha (or beta) zero.
 * rz[m] (length M + 1) receives rho_m = <r_m, z_m>; may be NULL.
 */
void or_pcg(const or_problem *pb, const double *X, int M, double *delta, double *rz) {
  long n = nvar(pb);
  double *g = malloc(sizeof(double) * n), *d = malloc(sizeof(double) * n);
  double *r = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n);
  double *p = malloc(sizeof(double) * n), *q = malloc(sizeof(double) * n);
  or_rhs(pb, X, X, ALL_TERMS, g);
  or_diag(pb, X, X, ALL_TERMS, d);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; i++) {
    delta[i] = 0;
    r[i] = g[i];
    z[i] = r[i] / d[i];
    p[i] = z[i];
  }
  double rho = dot(r, z, n);
  if (rz) rz[0] = rho;
  for (int m = 1; m <= M; m++) {
    or_apply(pb, X, X, ALL_TERMS, p, q);
    double pq = dot(p, q, n);
    double alpha = pq != 0 ? rho / pq : 0.0;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
      delta[i] += alpha * p[i];
      r[i] -= alpha * q[i];
      z[i] = r[i] / d[i];
    }
    double rho_new = dot(r, z, n);
    double beta = rho != 0 ? rho_new / rho : 0.0;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
    rho = rho_new;
    if (rz) rz[m] = rho;
  }
  free(g); free(d); free(r); free(z); free(p); free(q);
}

/* One Gauss-Newton step X <- X + delta* (eq:optimization), delta* from or_pcg. */
void or_gn_step(const or_problem *pb, double *X, int M) {
  long n = nvar(pb);
  double *delta = malloc(sizeof(double) * n);
  or_pcg(pb, X, M, delta, NULL);
  for (long i = 0; i < n; i++) X[i] += delta[i];
  free(delta);
}

/* ---------------- preconditioner and PCG variants (Sec. 6.1 leaves the preconditioner unnamed) ---------------- */

/*
 * Per-pixel V x V diagonal blocks of J^T J: B[x][u][v] = sum over the rows of
 * a_(u,x) a_(v,x), both entries of one row at the same pixel x.  B is (P, V, V),
 * row-major per pixel.  The diagonal of B is or_diag's d.
 */
typedef struct { double *B; long P; int V; } block_ctx;
static void visit_block(const or_row *r, void *vc) {
  block_ctx *c = (block_ctx *)vc;
  for (int i = 0; i < r->n; i++)
    for (int j = 0; j < r->n; j++) {
      long xi = r->j[i] % c->P, xj = r->j[j] % c->P;
      if (xi != xj) continue;
      int u = (int)(r->j[i] / c->P), v = (int)(r->j[j] / c->P);
      c->B[(xi * c->V + u) * c->V + v] += r->a[i] * r->a[j];
    }
}

void or_block_diag(const or_problem *pb, const double *X, const double *Xw, unsigned mask, double *B) {
  const int V = pb->K + 4;
  memset(B, 0, sizeof(double) * P_of(pb) * V * V);
  block_ctx c = {B, P_of(pb), V};
  or_rows_striped(pb, X, Xw, mask, visit_block, &c);
}

/* Cholesky factor (lower, in place, row-major n x n) of an SPD matrix; returns 0 on a non-positive pivot. */
static int cholesky(double *A, int n) {
  for (int j = 0; j < n; j++) {
    double s = A[j * n + j];
    for (int k = 0; k < j; k++) s -= A[j * n + k] * A[j * n + k];
    if (!(s > 0)) return 0;
    A[j * n + j] = sqrt(s);
    for (int i = j + 1; i < n; i++) {
      double t = A[i * n + j];
      for (int k = 0; k < j; k++) t -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = t / A[j * n + j];
    }
  }
  return 1;
}

/* Solve L L^T z = r with the factor from cholesky(). */
static void chol_solve(const double *L, int n, const double *r, double *z) {
  for (int i = 0; i < n; i++) {
    double t = r[i];
    for (int k = 0; k < i; k++) t -= L[i * n + k] * z[k];
    z[i] = t / L[i * n + i];
  }
  for (int i = n - 1; i >= 0; i--) {
    double t = z[i];
    for (int k = i + 1; k < n; k++) t -= L[k * n + i] * z[k];
    z[i] = t / L[i * n + i];
  }
}

/* The preconditioner step z = M^-1 r: Jacobi (block == 0: d = diag J^T J) or
 * block-Jacobi (block == 1: Lb = the per-pixel Cholesky factors of or_block_diag). */
typedef struct { int block; long P; int V; const double *d, *Lb; } precond;
static void precond_apply(const precond *m, const double *r, double *z) {
  if (!m->block) {
    for (long i = 0; i < m->P * m->V; i++) z[i] = r[i] / m->d[i];
    return;
  }
  double rv[32], zv[32];
  for (long x = 0; x < m->P; x++) {
    for (int v = 0; v < m->V; v++) rv[v] = r[v * m->P + x];
    chol_solve(m->Lb + x * m->V * m->V, m->V, rv, zv);
    for (int v = 0; v < m->V; v++) z[v * m->P + x] = zv[v];
  }
}

/*
 * M steps of preconditioned CG on J^T J delta = -J^T F at X, delta_0 = 0, no early
 * exit, in one of two preconditioners (block: 0 Jacobi, 1 block-Jacobi) and two
 * recurrences (single_reduction: 0 the textbook two-reduction recurrence, as in
 * or_pcg; 1 the single-reduction recurrence of Chronopoulos and Gear (1989),
 * which carries s = A p and takes <r,u> and <A u,u> from one reduction, u = M^-1 r:
 *   beta = gamma / gamma_old, alpha = gamma / (delta - beta gamma / alpha_old),
 *   p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s, u = M^-1 r, w = A u).
 * In exact arithmetic both recurrences give the same iterates.  rz[m] = <r_m, z_m>
 * (length M + 1, may be NULL).  Returns 0 if a block is not positive definite.
 */
int or_pcg_variant(const or_problem *pb, const double *X, int M, int block, int single_reduction, double *delta,
                   double *rz) {
  const long n = nvar(pb), P = P_of(pb);
  const int V = pb->K + 4;
  double *g = malloc(sizeof(double) * n), *d = malloc(sizeof(double) * n);
  double *r = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n);
  double *p = malloc(sizeof(double) * n), *q = malloc(sizeof(double) * n);
  double *w = malloc(sizeof(double) * n), *Lb = NULL;
  int ok = 1;
  or_rhs(pb, X, X, ALL_TERMS, g);
  or_diag(pb, X, X, ALL_TERMS, d);
  if (block) {
    Lb = malloc(sizeof(double) * P * V * V);
    or_block_diag(pb, X, X, ALL_TERMS, Lb);
    for (long x = 0; x < P && ok; x++) ok = cholesky(Lb + x * V * V, V);
  }
  precond m = {block, P, V, d, Lb};
  for (long i = 0; i < n; i++) {
    delta[i] = 0;
    r[i] = g[i];
  }
  if (ok && !single_reduction) {
    precond_apply(&m, r, z);
    for (long i = 0; i < n; i++) p[i] = z[i];
    double rho = dot(r, z, n);
    if (rz) rz[0] = rho;
    for (int it = 1; it <= M; it++) {
      or_apply(pb, X, X, ALL_TERMS, p, q);
      double pq = dot(p, q, n);
      double alpha = pq != 0 ? rho / pq : 0.0;
      for (long i = 0; i < n; i++) {
        delta[i] += alpha * p[i];
        r[i] -= alpha * q[i];
      }
      precond_apply(&m, r, z);
      double rho_new = dot(r, z, n);
      double beta = rho != 0 ? rho_new / rho : 0.0;
      for (long i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
      rho = rho_new;
      if (rz) rz[it] = rho;
    }
  } else if (ok) {
    /* z holds u = M^-1 r, w = A u, q holds s = A p */
    precond_apply(&m, r, z);
    or_apply(pb, X, X, ALL_TERMS, z, w);
    double gamma = dot(r, z, n), dl = dot(w, z, n);
    double alpha = dl != 0 ? gamma / dl : 0.0, beta = 0.0, gamma_old = gamma;
    if (rz) rz[0] = gamma;
    for (long i = 0; i < n; i++) p[i] = q[i] = 0;
    for (int it = 1; it <= M; it++) {
      for (long i = 0; i < n; i++) {
        p[i] = z[i] + beta * p[i];
        q[i] = w[i] + beta * q[i];
        delta[i] += alpha * p[i];
        r[i] -= alpha * q[i];
      }
      precond_apply(&m, r, z);
      or_apply(pb, X, X, ALL_TERMS, z, w);
      gamma = dot(r, z, n);
      dl = dot(w, z, n);
      if (rz) rz[it] = gamma;
      beta = gamma_old != 0 ? gamma / gamma_old : 0.0;
      double den = dl - (alpha != 0 ? beta * gamma / alpha : 0.0);
      alpha = den != 0 ? gamma / den : 0.0;
      gamma_old = gamma;
    }
  }
  free(g); free(d); free(r); free(z); free(p); free(q); free(w); free(Lb);
  return ok;
}

/* ---------------- dense step: base-colour refinement (Sec. 5.4) ---------------- */

/*
 * Normal equations of E_refine (eq:basecolorrefinement) in the unknowns
 * Delta b_k, k = 1..K (b_0 stays white), at fixed layers X, with b_k the initial
 * estimate b_init (the refined colours are b_init + Delta b).  The data residual
 * of channel c involves only Delta b_{.,c}, and both regularisers are diagonal,
 * so the 3K x 3K system is three K x K blocks: A[c][k][l], g[c][k]
 * (A is (3, K, K) row-major, g is (3, K); g = -J^T F).
 */
static void or_dense_range(const or_problem *pb, const double *X, double *A, double *g, int y_begin, int y_end) {
  const int W = pb->W, K = pb->K;
  double sl = sqrt(pb->lambda_data);
  double a[64];
  for (int y = y_begin; y < y_end; y++)
    for (int x = 0; x < W; x++)
      for (int c = 0; c < 3; c++) {
        double R = exp(X[idx(pb, c, y, x)]);
        double S0 = X[idx(pb, 3, y, x)]; /* b_0 T_0 with b_0 white */
        for (int k = 1; k <= K; k++) S0 += pb->b_init[(k - 1) * 3 + c] * X[idx(pb, 3 + k, y, x)];
        double f = sl * (pb->I[idx(pb, c, y, x)] - R * S0);
        for (int k = 1; k <= K; k++) a[k - 1] = -sl * R * X[idx(pb, 3 + k, y, x)];
        for (int k = 0; k < K; k++) {
          g[c * K + k] -= a[k] * f;
          for (int l = 0; l < K; l++) A[(c * K + k) * K + l] += a[k] * a[l];
        }
      }
}

void or_dense_normal(const or_problem *pb, const double *X, double *A, double *g) {
  const int K = pb->K, ns = (pb->H + OR_STRIPE - 1) / OR_STRIPE, na = 3 * K * K + 3 * K;
  double *part = calloc((size_t)ns * na, sizeof(double));
#pragma omp parallel for schedule(static)
  for (int st = 0; st < ns; st++) {
    const int y1 = (st + 1) * OR_STRIPE < pb->H ? (st + 1) * OR_STRIPE : pb->H;
    or_dense_range(pb, X, part + (long)st * na, part + (long)st * na + 3 * K * K, st * OR_STRIPE, y1);
  }
  memset(A, 0, sizeof(double) * 3 * K * K);
  memset(g, 0, sizeof(double) * 3 * K);
  for (int st = 0; st < ns; st++) {
    for (int i = 0; i < 3 * K * K; i++) A[i] += part[(long)st * na + i];
    for (int i = 0; i < 3 * K; i++) g[i] += part[(long)st * na + 3 * K * K + i];
  }
  free(part);
  /* Intensity regulariser sqrt(l_IR) Delta b_kc and chromaticity regulariser
   * sqrt(l_CR) ((C(b_k) + Delta b_k) - C(b_k))_c: both residuals are zero at
   * Delta b = 0 with unit Jacobian, adding l_IR + l_CR to the diagonal. */
  for (int c = 0; c < 3; c++)
    for (int k = 0; k < K; k++) A[(c * K + k) * K + k] += pb->lambda_IR + pb->lambda_CR;
}

/* ---------------- per-frame precompute ---------------- */

/*
 * Chromaticity C = I / (I_R + I_G + I_B + 1e-6) (Sec. 4.1), soft-Retinex weight
 * w_SR = 1 - exp(-sharpness * dC) with dC the largest chromaticity difference to
 * an in-image 4-neighbour (Sec. 5.2), and the consistency pair weights
 * omega(x, y) = exp(-|C(x) - C'(y)|^2 / tau^2) (0 if y is outside the image),
 * spatial (C' = C) and temporal (C' = chromaticity of Iprev; skipped if NULL).
 */
void or_precompute(int H, int W, const double *I, const double *Iprev, int n_s, const int *off_s, int n_t,
                   const int *off_t, double tau, double sharpness, double *C, double *wsr, double *omega_s,
                   double *omega_t) {
  long P = (long)H * W;
  double *Cp = Iprev ? malloc(sizeof(double) * 3 * P) : NULL;
#pragma omp parallel for schedule(static)
  for (long i = 0; i < P; i++) {
    double s = I[i] + I[P + i] + I[2 * P + i] + 1e-6;
    for (int c = 0; c < 3; c++) C[c * P + i] = I[c * P + i] / s;
    if (Cp) {
      double sp = Iprev[i] + Iprev[P + i] + Iprev[2 * P + i] + 1e-6;
      for (int c = 0; c < 3; c++) Cp[c * P + i] = Iprev[c * P + i] / sp;
    }
  }
  static const int N4[4][2] = {{0, 1}, {0, -1}, {1, 0}, {-1, 0}};
#pragma omp parallel for schedule(static)
  for (int y = 0; y < H; y++)
    for (int x = 0; x < W; x++) {
      long i = (long)y * W + x;
      double dC = 0;
      for (int n = 0; n < 4; n++) {
        int ny = y + N4[n][0], nx = x + N4[n][1];
        if (ny < 0 || ny >= H || nx < 0 || nx >= W) continue;
        long jn = (long)ny * W + nx;
        double d2 = 0;
        for (int c = 0; c < 3; c++) d2 += (C[c * P + jn] - C[c * P + i]) * (C[c * P + jn] - C[c * P + i]);
        if (sqrt(d2) > dC) dC = sqrt(d2);
      }
      wsr[i] = 1.0 - exp(-sharpness * dC);
      for (int j = 0; j < n_s; j++) {
        int ny = y + off_s[2 * j], nx = x + off_s[2 * j + 1];
        double w = 0;
        if (ny >= 0 && ny < H && nx >= 0 && nx < W) {
          long jn = (long)ny * W + nx;
          double d2 = 0;
          for (int c = 0; c < 3; c++) d2 += (C[c * P + i] - C[c * P + jn]) * (C[c * P + i] - C[c * P + jn]);
          w = exp(-d2 / (tau * tau));
        }
        omega_s[j * P + i] = w;
      }
      if (Cp && omega_t)
        for (int j = 0; j < n_t; j++) {
          int ny = y + off_t[2 * j], nx = x + off_t[2 * j + 1];
          double w = 0;
          if (ny >= 0 && ny < H && nx >= 0 && nx < W) {
            long jn = (long)ny * W + nx;
            double d2 = 0;
            for (int c = 0; c < 3; c++) d2 += (C[c * P + i] - Cp[c * P + jn]) * (C[c * P + i] - Cp[c * P + jn]);
            w = exp(-d2 / (tau * tau));
          }
          omega_t[j * P + i] = w;
        }
    }
  free(Cp);
}

/*
 * Cold start: r = r_cluster (Sec. 4.1 uses R_cluster to initialise R),
 * T_0 = mean_c I / mean_c R_cluster, T_k = 0 for k >= 1 (the paper does not
 * state the initial T).
 */
void or_init_cold(const or_problem *pb, double *X) {
  const int H = pb->H, W = pb->W, K = pb->K;
  for (int y = 0; y < H; y++)
    for (int x = 0; x < W; x++) {
      double mi = 0, mr = 0;
      for (int c = 0; c < 3; c++) {
        X[idx(pb, c, y, x)] = rcluster(pb, c, y, x);
        mi += pb->I[idx(pb, c, y, x)] / 3.0;
        mr += exp(rcluster(pb, c, y, x)) / 3.0;
      }
      X[idx(pb, 3, y, x)] = mi / mr;
      for (int k = 1; k <= K; k++) X[idx(pb, 3 + k, y, x)] = 0.0;
    }
}
