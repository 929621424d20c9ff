/*
 * oracle.c -- plain, slow FP64 reference for the GWAS sequence of generalized
 * least-squares problems (Fabregat-Traver, Aulchenko, Bientinesi, "Solving
 * Sequences of Generalized Least-Squares Problems on Multi-threaded
 * Architectures", Eq. 1):
 *
 *     b_i := (X_i^T M^{-1} X_i)^{-1} X_i^T M^{-1} y,   1 <= i <= m,
 *     X_i = (X_L | x_Ri),  M SPD (n x n),  X_L n x (p-1),  x_Ri n x 1.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The GPU product path
 * never calls, links or includes it, and it shares no code, header, table or
 * constant with the GPU path.
 *
 * What it computes, step by step (no blocking, no fusion):
 *   1. L L^T = M, unblocked left-looking Cholesky         (Alg. 5 line 1, potrf)
 *   2. y~ = L^{-1} y, X~_L = L^{-1} X_L, one column at a
 *      time by forward substitution                      (Alg. 5 lines 2 and 4)
 *   3. per SNP i, on its own:
 *        x~ = L^{-1} x_Ri by forward substitution         (Alg. 5 line 3, one column)
 *        S_i = [X~_L x~]^T [X~_L x~], the full p x p Gram (Alg. 3 line 4, syrk;
 *                                                         Fig. 1 blocks, none reused)
 *        r_i = [X~_L x~]^T y~                             (Alg. 3 line 5, gemv)
 *        b_i = S_i^{-1} r_i by an unpivoted Cholesky of
 *              S_i and two triangular solves              (Alg. 3 line 6, posv)
 *
 * Readings where the paper is silent (conventions it leaves open, taken here):
 *   - storage is column-major with leading dimensions (LAPACK convention);
 *   - only the lower triangle of M is read;
 *   - b_i lists the X_L coefficients first and the SNP coefficient last;
 *   - p = 1 means X_L is empty;
 *   - a pivot d_j of S_i with d_j <= tau * S_i[j][j] (the diagonal entry before
 *     elimination) marks S_i as not SPD: b_i is set to NaN and status[i] = 1;
 *     tau is a parameter so that each precision path is checked against the
 *     same rule;
 *   - sums run in ascending index order; the file is compiled with
 *     -ffp-contract=off so that every product is rounded before it is added.
 *
 * The threads only split independent work (rows of one Cholesky column, whole
 * SNPs); they never change the order of any sum.
 */
#include <math.h>
#include <pthread.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define COLMAJ(a, ld, i, j) ((a)[(size_t)(j) * (size_t)(ld) + (size_t)(i)])

/* ------------------------------------------------------------------------- */
/* Tiny barrier (pthread_barrier_t is optional in POSIX; this one is plain).  */
/* ------------------------------------------------------------------------- */
typedef struct {
  pthread_mutex_t mu;
  pthread_cond_t cv;
  int count, waiting, phase;
} oracle_barrier_t;

static void barrier_init(oracle_barrier_t* b, int count) {
  pthread_mutex_init(&b->mu, NULL);
  pthread_cond_init(&b->cv, NULL);
  b->count = count;
  b->waiting = 0;
  b->phase = 0;
}

static void barrier_destroy(oracle_barrier_t* b) {
  pthread_mutex_destroy(&b->mu);
  pthread_cond_destroy(&b->cv);
}

static void barrier_wait(oracle_barrier_t* b) {
  pthread_mutex_lock(&b->mu);
  int phase = b->phase;
  if (++b->waiting == b->count) {
    b->waiting = 0;
    b->phase++;
    pthread_cond_broadcast(&b->cv);
  } else {
    while (phase == b->phase) pthread_cond_wait(&b->cv, &b->mu);
  }
  pthread_mutex_unlock(&b->mu);
}

/* ------------------------------------------------------------------------- */
/* Step 1: Cholesky factorization L L^T = M (Alg. 5 line 1).                  */
/*                                                                           */
/* Left-looking column form: for column j,                                   */
/*   v_i = M_ij - sum_{k<j} L_ik L_jk      (i >= j, k ascending)              */
/*   L_jj = sqrt(v_j),  L_ij = v_i / L_jj  (i > j).                           */
/* Fails at the first j with v_j <= 0 (returned 1-based, as LAPACK potrf).    */
/* ------------------------------------------------------------------------- */
typedef struct {
  int64_t n;
  const double* M;
  int64_t ldm;
  double* L;
  int64_t ldl;
  double* v;        /* length n scratch: column being formed */
  int tid, nthreads;
  oracle_barrier_t* bar;
  volatile int64_t* info;
} potrf_job_t;

static void* potrf_worker(void* arg) {
  potrf_job_t* jb = (potrf_job_t*)arg;
  const int64_t n = jb->n;
  double* L = jb->L;
  const int64_t ldl = jb->ldl;
  double* v = jb->v;
  for (int64_t j = 0; j < n; ++j) {
    /* rows [j, n) split across threads */
    int64_t rows = n - j;
    int64_t lo = j + rows * jb->tid / jb->nthreads;
    int64_t hi = j + rows * (jb->tid + 1) / jb->nthreads;
    for (int64_t i = lo; i < hi; ++i) v[i] = COLMAJ(jb->M, jb->ldm, i, j);
    for (int64_t k = 0; k < j; ++k) {
      const double ljk = COLMAJ(L, ldl, j, k);
      for (int64_t i = lo; i < hi; ++i) v[i] -= COLMAJ(L, ldl, i, k) * ljk;
    }
    barrier_wait(jb->bar);
    if (!(v[j] > 0.0)) {
      /* every thread sees the same v[j]: all stop at the same column */
      if (jb->tid == 0) *jb->info = j + 1;
      return NULL;
    }
    const double ljj = sqrt(v[j]);
    for (int64_t i = lo; i < hi; ++i) COLMAJ(L, ldl, i, j) = (i == j) ? ljj : v[i] / ljj;
    barrier_wait(jb->bar);
  }
  return NULL;
}

int64_t gls_oracle_potrf(int64_t n, const double* M, int64_t ldm, double* L, int64_t ldl,
                         int32_t nthreads) {
  if (n <= 0) return 0;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) COLMAJ(L, ldl, i, j) = 0.0;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if ((int64_t)nthreads > n) nthreads = (int32_t)n;
  double* v = (double*)malloc(sizeof(double) * (size_t)n);
  if (!v) return -1;
  volatile int64_t info = 0;
  oracle_barrier_t bar;
  barrier_init(&bar, nthreads);
  potrf_job_t* jobs = (potrf_job_t*)malloc(sizeof(potrf_job_t) * (size_t)nthreads);
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
  for (int t = 0; t < nthreads; ++t) {
    jobs[t] = (potrf_job_t){n, M, ldm, L, ldl, v, t, nthreads, &bar, &info};
  }
  for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, potrf_worker, &jobs[t]);
  potrf_worker(&jobs[0]);
  for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
  barrier_destroy(&bar);
  free(th);
  free(jobs);
  free(v);
  return info;
}

/* ------------------------------------------------------------------------- */
/* Step 2/3: forward substitution L x = b, overwriting b (trsv, Table 1).     */
/* Column-oriented: x_j = b_j / L_jj, then b_i -= L_ij x_j for i > j.         */
/* ------------------------------------------------------------------------- */
void gls_oracle_trsv(int64_t n, const double* L, int64_t ldl, double* x) {
  for (int64_t j = 0; j < n; ++j) {
    const double xj = x[j] / COLMAJ(L, ldl, j, j);
    x[j] = xj;
    for (int64_t i = j + 1; i < n; ++i) x[i] -= COLMAJ(L, ldl, i, j) * xj;
  }
}

/* ------------------------------------------------------------------------- */
/* Step 3 tail: b = S^{-1} r for one p x p SPD system (posv, Alg. 3 line 6).  */
/* S is p x p column-major (lower triangle used), destroyed.  Returns 0, or   */
/* 1 when a pivot d_j <= tau * S_jj (S not numerically SPD).                  */
/* ------------------------------------------------------------------------- */
static int posv_small(int p, double* S, const double* r, double tau, double* b) {
  /* unpivoted Cholesky S = R R^T, R lower, stored over S */
  for (int j = 0; j < p; ++j) {
    const double sjj = COLMAJ(S, p, j, j);
    double d = sjj;
    for (int k = 0; k < j; ++k) d -= COLMAJ(S, p, j, k) * COLMAJ(S, p, j, k);
    if (!(d > tau * sjj)) return 1;
    const double rjj = sqrt(d);
    COLMAJ(S, p, j, j) = rjj;
    for (int i = j + 1; i < p; ++i) {
      double s = COLMAJ(S, p, i, j);
      for (int k = 0; k < j; ++k) s -= COLMAJ(S, p, i, k) * COLMAJ(S, p, j, k);
      COLMAJ(S, p, i, j) = s / rjj;
    }
  }
  /* R z = r */
  for (int i = 0; i < p; ++i) {
    double s = r[i];
    for (int k = 0; k < i; ++k) s -= COLMAJ(S, p, i, k) * b[k];
    b[i] = s / COLMAJ(S, p, i, i);
  }
  /* R^T b = z */
  for (int i = p - 1; i >= 0; --i) {
    double s = b[i];
    for (int k = i + 1; k < p; ++k) s -= COLMAJ(S, p, k, i) * b[k];
    b[i] = s / COLMAJ(S, p, i, i);
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* The whole sequence (Eq. 1).                                                */
/* ------------------------------------------------------------------------- */
typedef struct {
  int64_t n;
  int32_t p;
  const double* L;
  const double* XLt; /* n x (p-1), whitened, ld = n */
  const double* yt;  /* n, whitened */
  const int8_t* XR;
  int64_t ldxr;
  double* B;
  int64_t ldb;
  int32_t* status;
  double tau;
  int64_t first, last; /* SNP range [first, last) */
} snp_job_t;

static void* snp_worker(void* arg) {
  snp_job_t* jb = (snp_job_t*)arg;
  const int64_t n = jb->n;
  const int p = jb->p;
  double* xt = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* S = (double*)malloc(sizeof(double) * (size_t)p * (size_t)p);
  double* r = (double*)malloc(sizeof(double) * (size_t)p);
  double* b = (double*)malloc(sizeof(double) * (size_t)p);
  for (int64_t s = jb->first; s < jb->last; ++s) {
    const int8_t* x = jb->XR + (size_t)s * (size_t)jb->ldxr;
    for (int64_t t = 0; t < n; ++t) xt[t] = (double)x[t];
    gls_oracle_trsv(n, jb->L, n, xt);
    /* columns of X~_i: 0..p-2 from X~_L, p-1 is x~ */
    for (int a = 0; a < p; ++a) {
      const double* ca = (a < p - 1) ? jb->XLt + (size_t)a * (size_t)n : xt;
      for (int c = 0; c <= a; ++c) {
        const double* cc = (c < p - 1) ? jb->XLt + (size_t)c * (size_t)n : xt;
        double acc = 0.0;
        for (int64_t t = 0; t < n; ++t) acc += ca[t] * cc[t];
        COLMAJ(S, p, a, c) = acc;
        COLMAJ(S, p, c, a) = acc;
      }
      double acc = 0.0;
      for (int64_t t = 0; t < n; ++t) acc += ca[t] * jb->yt[t];
      r[a] = acc;
    }
    double* out = jb->B + (size_t)s * (size_t)jb->ldb;
    int st = posv_small(p, S, r, jb->tau, b);
    if (st == 0) {
      for (int a = 0; a < p; ++a) out[a] = b[a];
    } else {
      for (int a = 0; a < p; ++a) out[a] = NAN;
    }
    if (jb->status) jb->status[s] = st;
  }
  free(xt);
  free(S);
  free(r);
  free(b);
  return NULL;
}

/*
 * Steps 2-3 for a given factor: L is n x n lower (ld = n) with L L^T = M.
 * Arguments and outputs as for gls_oracle_gls below.  Returns 0, or -1 on a
 * bad argument / allocation failure.
 */
int64_t gls_oracle_gls_factored(int64_t n, int32_t p, const double* L, const double* XL,
                                int64_t ldxl, const double* y, int64_t k, const int8_t* XR,
                                int64_t ldxr, double* B, int64_t ldb, int32_t* status, double tau,
                                int32_t nthreads) {
  if (n < 1 || p < 1 || k < 0 || ldxr < n || ldb < p || L == NULL) return -1;
  if (p > 1 && (XL == NULL || ldxl < n)) return -1;
  if (nthreads < 1) nthreads = 1;
  double* XLt = (double*)malloc(sizeof(double) * (size_t)n * (size_t)(p > 1 ? p - 1 : 1));
  double* yt = (double*)malloc(sizeof(double) * (size_t)n);
  if (!XLt || !yt) {
    free(XLt);
    free(yt);
    return -1;
  }
  /* y~ = L^{-1} y, X~_L = L^{-1} X_L (Alg. 5 lines 2 and 4) */
  for (int64_t t = 0; t < n; ++t) yt[t] = y[t];
  gls_oracle_trsv(n, L, n, yt);
  for (int c = 0; c < p - 1; ++c) {
    double* col = XLt + (size_t)c * (size_t)n;
    for (int64_t t = 0; t < n; ++t) col[t] = COLMAJ(XL, ldxl, t, c);
    gls_oracle_trsv(n, L, n, col);
  }
  int T = nthreads;
  if ((int64_t)T > k) T = (int)(k > 0 ? k : 1);
  snp_job_t* jobs = (snp_job_t*)malloc(sizeof(snp_job_t) * (size_t)T);
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)T);
  for (int t = 0; t < T; ++t) {
    jobs[t] = (snp_job_t){n, p, L, XLt, yt, XR, ldxr, B, ldb, status, tau,
                          k * t / T, k * (t + 1) / T};
  }
  for (int t = 1; t < T; ++t) pthread_create(&th[t], NULL, snp_worker, &jobs[t]);
  snp_worker(&jobs[0]);
  for (int t = 1; t < T; ++t) pthread_join(th[t], NULL);
  free(th);
  free(jobs);
  free(XLt);
  free(yt);
  return 0;
}

/*
 * Full reference: returns 0, the 1-based failing pivot of M (B untouched), or
 * -1 on a bad argument / allocation failure.
 *   M      n x n, ldm >= n, lower triangle read
 *   XL     n x (p-1), ldxl >= n (ignored when p == 1)
 *   y      n
 *   XR     n x k int8, ldxr >= n
 *   B      p x k, ldb >= p (output)
 *   status k int32 (output, may be NULL): 0 ok, 1 S_i not SPD (b_i = NaN)
 */
int64_t gls_oracle_gls(int64_t n, int32_t p, const double* M, int64_t ldm, const double* XL,
                       int64_t ldxl, const double* y, int64_t k, const int8_t* XR, int64_t ldxr,
                       double* B, int64_t ldb, int32_t* status, double tau, int32_t nthreads) {
  if (n < 1 || p < 1 || k < 0 || ldm < n || ldxr < n || ldb < p) return -1;
  if (p > 1 && (XL == NULL || ldxl < n)) return -1;
  if (nthreads < 1) nthreads = 1;
  double* L = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
  if (!L) return -1;
  int64_t info = gls_oracle_potrf(n, M, ldm, L, n, nthreads);
  if (info == 0)
    info = gls_oracle_gls_factored(n, p, L, XL, ldxl, y, k, XR, ldxr, B, ldb, status, tau,
                                   nthreads);
  free(L);
  return info;
}

/*
 * Same as gls_oracle_gls, for a chosen subset of SNP columns: SNP idx[j] of XR
 * is solved into column j of B (and status[j]).  Used to check full-size runs
 * on sampled outputs without solving every SNP.
 */
int64_t gls_oracle_gls_sampled(int64_t n, int32_t p, const double* M, int64_t ldm,
                               const double* XL, int64_t ldxl, const double* y, int64_t nidx,
                               const int64_t* idx, const int8_t* XR, int64_t ldxr, double* B,
                               int64_t ldb, int32_t* status, double tau, int32_t nthreads) {
  if (nidx < 0 || (nidx > 0 && idx == NULL)) return -1;
  int8_t* sub = (int8_t*)malloc((size_t)(nidx > 0 ? nidx : 1) * (size_t)n);
  if (!sub) return -1;
  for (int64_t j = 0; j < nidx; ++j)
    memcpy(sub + (size_t)j * (size_t)n, XR + (size_t)idx[j] * (size_t)ldxr, (size_t)n);
  int64_t r = gls_oracle_gls(n, p, M, ldm, XL, ldxl, y, nidx, sub, n, B, ldb, status, tau,
                             nthreads);
  free(sub);
  return r;
}
