// variants.cu -- kernels of the paper's comparison algorithms for a sequence
// of GLS problems (Section 2), binary64, for the cost comparison of Table 2.
// The library's own path is Alg. 5 (hp-gwas); these are the others:
//
//   Alg. 3 (black-box): each problem on its own: potrf of M, trsm of
//       X_i = (X_L | x_Ri), trsv of y, syrk, gemv, posv.  Cost ~ n^3 per problem.
//   Alg. 4 (seq-gls): potrf of M and trsv of y once; per problem the trsm of
//       the whole X_i (p columns), syrk, gemv, posv.  Cost ~ n^2 p per problem.
//   Alg. 6 (gwfgls, GenABEL): the explicit inverse M^{-1} and W_L = M^{-1} X_L
//       once; per problem w = M^{-1} x_Ri with the full (not triangular)
//       inverse, S_i = (W_L | w)^T (X_L | x_Ri) formed entry by entry without
//       using its symmetry, b_i = (W_L | w)^T y, and an LU solve (gesv).
//       Cost ~ 2 n^2 per problem.
//
// The triangular solves with L are applied as products with Z = L^{-1} (the
// library's factor gives both), which costs the same n^2 per column.  Every
// kernel sums in a fixed order, so results do not depend on launch shapes.
#include <math.h>

#include "common.cuh"
#include "variants.cuh"

namespace gls {
namespace {

constexpr double kNaN = __builtin_nan("");

// R = [X_L | x_j | y] (mode 0, one SNP: p + 1 columns) or, for the g SNPs
// j0 .. j0+g-1, [X_L | x_j] side by side (mode 1: p columns each), npad rows,
// rows >= n zero.  x_j is converted from int8.
__global__ void __launch_bounds__(256) rhs_kernel(const double* __restrict__ XL, int64_t ldxl,
                                                  const double* __restrict__ y,
                                                  const int8_t* __restrict__ XR, int64_t ldxr,
                                                  int64_t j0, int g, int64_t n, int64_t npad,
                                                  int p, int mode, double* __restrict__ R,
                                                  int64_t ldr) {
  const int q = p - 1;
  const int cols = mode == 0 ? p + 1 : p * g;
  const int64_t total = npad * cols;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx % npad;
    const int c = (int)(idx / npad);
    double v = 0.0;
    if (r < n) {
      const int s = mode == 0 ? 0 : c / p;      // SNP of this column
      const int cc = mode == 0 ? c : c % p;     // column within (X_L | x_j [| y])
      if (cc < q) v = XL[r + (int64_t)cc * ldxl];
      else if (cc == q) v = (double)XR[r + (j0 + s) * ldxr];
      else v = y[r];
    }
    R[r + (int64_t)c * ldr] = v;
  }
}

// Alg. 3/4 per problem: S = X~^T X~ (p x p) and r = X~^T y~ from the whitened
// columns X~ = W[:, s*cstride .. s*cstride + p) of SNP s and y~, then the
// Cholesky solve of S b = r (posv).  One CTA per SNP; each sum over the n rows
// is a fixed-stride loop per thread and a fixed tree.  A pivot d <= tau S_jj
// marks S as not SPD: b = NaN, status 1.
__global__ void __launch_bounds__(256) gram_posv_kernel(const double* __restrict__ W,
                                                        int64_t ldw, int64_t n, int p,
                                                        int cstride,
                                                        const double* __restrict__ yt,
                                                        double tau, double* __restrict__ B,
                                                        int64_t ldb, int32_t* __restrict__ status) {
  __shared__ double red[256];
  __shared__ double S[kVarMaxP * (kVarMaxP + 1)];  // column-major p x (p + 1): [S | r]
  __shared__ double L[kVarMaxP * kVarMaxP];
  __shared__ double z[kVarMaxP];
  const int s = blockIdx.x;
  const double* X = W + (int64_t)s * cstride * ldw;
  const int npairs = p * (p + 1) / 2 + p;
  for (int e = 0; e < npairs; ++e) {
    int a, c;  // e < p(p+1)/2: pair (a >= c) of S; else r_a
    const double* u;
    const double* v;
    if (e < p * (p + 1) / 2) {
      a = 0;
      while ((a + 1) * (a + 2) / 2 <= e) ++a;
      c = e - a * (a + 1) / 2;
      u = X + (int64_t)a * ldw;
      v = X + (int64_t)c * ldw;
    } else {
      a = e - p * (p + 1) / 2;
      c = p;
      u = X + (int64_t)a * ldw;
      v = yt;
    }
    double acc = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) acc = fma(u[r], v[r], acc);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      S[a + c * p] = red[0];
      if (c < p) S[c + a * p] = red[0];
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  bool ok = true;
  for (int j = 0; j < p && ok; ++j) {
    double d = S[j + j * p];
    for (int c = 0; c < j; ++c) d -= L[j + c * p] * L[j + c * p];
    if (!(d > tau * S[j + j * p])) {
      ok = false;
      break;
    }
    const double ljj = sqrt(d);
    L[j + j * p] = ljj;
    for (int i = j + 1; i < p; ++i) {
      double t = S[i + j * p];
      for (int c = 0; c < j; ++c) t -= L[i + c * p] * L[j + c * p];
      L[i + j * p] = t / ljj;
    }
  }
  double* out = B + (int64_t)s * ldb;
  if (!ok) {
    for (int a = 0; a < p; ++a) out[a] = kNaN;
    if (status) status[s] = 1;
    return;
  }
  for (int i = 0; i < p; ++i) {  // L z = r
    double t = S[i + p * p];
    for (int c = 0; c < i; ++c) t -= L[i + c * p] * z[c];
    z[i] = t / L[i + i * p];
  }
  for (int i = p - 1; i >= 0; --i) {  // L^T b = z
    double t = z[i];
    for (int c = i + 1; c < p; ++c) t -= L[c + i * p] * out[c];
    out[i] = t / L[i + i * p];
  }
  if (status) status[s] = 0;
}

// C (M x N, ldc) = A^T B with A (K x M, lda) and B (K x N, ldb), binary64.
// 64 x 64 tiles of C per CTA, K in chunks of 32 from shared memory, 4 x 4
// accumulators per thread; rows/columns beyond M, N and K are guarded.
__global__ void __launch_bounds__(256) gemm_tn_kernel(const double* __restrict__ A, int64_t lda,
                                                      const double* __restrict__ Bm,
                                                      int64_t ldbm, double* __restrict__ C,
                                                      int64_t ldc, int64_t M, int64_t N,
                                                      int64_t K) {
  __shared__ double As[32][65];
  __shared__ double Bs[32][65];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t i0 = (int64_t)blockIdx.x * 64, j0 = (int64_t)blockIdx.y * 64;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int64_t k0 = 0; k0 < K; k0 += 32) {
    for (int idx = threadIdx.x; idx < 32 * 64; idx += 256) {
      const int kk = idx % 32, c = idx / 32;
      const int64_t k = k0 + kk;
      As[kk][c] = (k < K && i0 + c < M) ? A[k + (i0 + c) * lda] : 0.0;
      Bs[kk][c] = (k < K && j0 + c < N) ? Bm[k + (j0 + c) * ldbm] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 32; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[kk][tx + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][ty + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t i = i0 + tx + 16 * a, j = j0 + ty + 16 * b;
      if (i < M && j < N) C[i + j * ldc] = acc[a][b];
    }
}

// Alg. 6 per block of SNPs: w = Minv x_j over all n rows (dense), and per
// 64-row block I the partial sums
//   P[I][a][j]         = sum_{r in I} w_r XL(r, a)    a < q      (w^T X_L)
//   P[I][q][j]         = sum_{r in I} w_r y_r                    (w^T y)
//   P[I][q + 1][j]     = sum_{r in I} w_r x_r                    (w^T x)
//   P[I][q + 2 + a][j] = sum_{r in I} WL(r, a) x_r    a < q      (W_L^T x)
// (2q + 2 rows per block); w is never stored.
__global__ void __launch_bounds__(256) dense_gram_kernel(
    const double* __restrict__ Minv, int64_t ldm, int64_t n, int nI,
    const int8_t* __restrict__ XR, int64_t ldxr, int64_t k, const double* __restrict__ XL,
    int64_t ldxl, const double* __restrict__ WL, int64_t ldwl, const double* __restrict__ y,
    int q, double* __restrict__ P, int64_t ldp) {
  // the two 32 x 64 staging tiles, then (after the products) the 64 x 64 x~ tile
  __shared__ double sm[2 * 32 * 64];
  double(*Zs)[64] = reinterpret_cast<double(*)[64]>(sm);
  double(*Xs)[64] = reinterpret_cast<double(*)[64]>(sm + 32 * 64);
  double(*T)[64] = reinterpret_cast<double(*)[64]>(sm);
  const int I = (int)blockIdx.y;
  const int64_t r0 = (int64_t)I * 64, j0 = (int64_t)blockIdx.x * 64;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int64_t c0 = 0; c0 < n; c0 += 32) {
    for (int idx = tid; idx < 32 * 64; idx += 256) {
      const int i = idx % 64, kk = idx / 64;
      const int64_t r = r0 + i, c = c0 + kk;
      Zs[kk][i] = (r < n && c < n) ? Minv[r + c * ldm] : 0.0;
      const int64_t jj = j0 + i;
      Xs[kk][i] = (jj < k && c < n) ? (double)XR[c + jj * ldxr] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 32; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = Zs[kk][tx + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Xs[kk][ty + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) T[tx + 16 * a][ty + 16 * b] = acc[a][b];
  __syncthreads();
  // thread -> one SNP j of the tile (tid < 64), rows of the block in order
  if (tid >= 64) return;
  const int64_t jj = j0 + tid;
  if (jj >= k) return;
  double part[2 * kVarMaxP + 2];
  const int nrows = 2 * q + 2;
  for (int a = 0; a < nrows; ++a) part[a] = 0.0;
  for (int i = 0; i < 64; ++i) {
    const int64_t r = r0 + i;
    if (r >= n) break;
    const double w = T[i][tid];
    const double x = (double)XR[r + jj * ldxr];
    for (int a = 0; a < q; ++a) part[a] = fma(w, XL[r + (int64_t)a * ldxl], part[a]);
    part[q] = fma(w, y[r], part[q]);
    part[q + 1] = fma(w, x, part[q + 1]);
    for (int a = 0; a < q; ++a) part[q + 2 + a] = fma(WL[r + (int64_t)a * ldwl], x, part[q + 2 + a]);
  }
  double* out = P + (int64_t)I * nrows * ldp + jj;
  for (int a = 0; a < nrows; ++a) out[(int64_t)a * ldp] = part[a];
}

// Alg. 6 per SNP: S = (W_L | w)^T (X_L | x) from the fixed block F = W_L^T X_L
// (q x q) and the per-SNP sums, r = (W_L^T y ; w^T y), then S b = r by LU with
// partial pivoting (gesv).  A pivot |u_jj| <= tau |S_jj| marks S as singular:
// b = NaN, status 1.  One thread per SNP.
__global__ void __launch_bounds__(128) gesv_kernel(const double* __restrict__ P, int64_t ldp,
                                                   int nI, int q, int64_t k,
                                                   const double* __restrict__ F, int ldf,
                                                   const double* __restrict__ bT, double tau,
                                                   double* __restrict__ B, int64_t ldb,
                                                   int32_t* __restrict__ status) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= k) return;
  const int p = q + 1, nrows = 2 * q + 2;
  double sum[2 * kVarMaxP + 2];
  for (int a = 0; a < nrows; ++a) sum[a] = 0.0;
  for (int I = 0; I < nI; ++I)
    for (int a = 0; a < nrows; ++a) sum[a] += P[((int64_t)I * nrows + a) * ldp + j];
  double S[kVarMaxP * kVarMaxP], r[kVarMaxP];
  for (int a = 0; a < q; ++a) {
    for (int c = 0; c < q; ++c) S[a + c * p] = F[a + c * ldf];  // W_L^T X_L
    S[a + q * p] = sum[q + 2 + a];                              // W_L^T x
    S[q + a * p] = sum[a];                                      // w^T X_L
    r[a] = bT[a];                                               // W_L^T y
  }
  S[q + q * p] = sum[q + 1];  // w^T x
  r[q] = sum[q];              // w^T y
  double diag[kVarMaxP];
  for (int a = 0; a < p; ++a) diag[a] = fabs(S[a + a * p]);
  double* out = B + j * ldb;
  for (int c = 0; c < p; ++c) {
    int piv = c;
    for (int a = c + 1; a < p; ++a)
      if (fabs(S[a + c * p]) > fabs(S[piv + c * p])) piv = a;
    if (piv != c) {
      for (int e = 0; e < p; ++e) {
        const double t = S[c + e * p];
        S[c + e * p] = S[piv + e * p];
        S[piv + e * p] = t;
      }
      const double t = r[c];
      r[c] = r[piv];
      r[piv] = t;
    }
    if (!(fabs(S[c + c * p]) > tau * diag[c])) {
      for (int a = 0; a < p; ++a) out[a] = kNaN;
      if (status) status[j] = 1;
      return;
    }
    for (int a = c + 1; a < p; ++a) {
      const double f = S[a + c * p] / S[c + c * p];
      for (int e = c + 1; e < p; ++e) S[a + e * p] -= f * S[c + e * p];
      r[a] -= f * r[c];
    }
  }
  for (int a = p - 1; a >= 0; --a) {
    double t = r[a];
    for (int e = a + 1; e < p; ++e) t -= S[a + e * p] * out[e];
    out[a] = t / S[a + a * p];
  }
  if (status) status[j] = 0;
}

inline unsigned grid1(int64_t total, int threads) {
  const int64_t g = ceil_div(total, threads);
  return (unsigned)(g > 65535 * 8 ? 65535 * 8 : (g < 1 ? 1 : g));
}

}  // namespace

void launch_variant_rhs(const double* XL, int64_t ldxl, const double* y, const int8_t* XR,
                        int64_t ldxr, int64_t j0, int g, int64_t n, int64_t npad, int p,
                        int mode, double* R, int64_t ldr, cudaStream_t st) {
  const int cols = mode == 0 ? p + 1 : p * g;
  rhs_kernel<<<grid1(npad * cols, 256), 256, 0, st>>>(XL, ldxl, y, XR, ldxr, j0, g, n, npad, p,
                                                      mode, R, ldr);
}

void launch_gram_posv(const double* W, int64_t ldw, int64_t n, int p, int cstride, int g,
                      const double* yt, double tau, double* B, int64_t ldb, int32_t* status,
                      cudaStream_t st) {
  gram_posv_kernel<<<(unsigned)g, 256, 0, st>>>(W, ldw, n, p, cstride, yt, tau, B, ldb, status);
}

void launch_gemm_tn(const double* A, int64_t lda, const double* B, int64_t ldb, double* C,
                    int64_t ldc, int64_t M, int64_t N, int64_t K, cudaStream_t st) {
  dim3 grid((unsigned)ceil_div(M, 64), (unsigned)ceil_div(N, 64));
  gemm_tn_kernel<<<grid, 256, 0, st>>>(A, lda, B, ldb, C, ldc, M, N, K);
}

void launch_dense_gram(const double* Minv, int64_t ldm, int64_t n, const int8_t* XR,
                       int64_t ldxr, int64_t k, const double* XL, int64_t ldxl,
                       const double* WL, int64_t ldwl, const double* y, int q, double* P,
                       int64_t ldp, cudaStream_t st) {
  const int nI = (int)ceil_div(n, 64);
  dim3 grid((unsigned)ceil_div(k, 64), (unsigned)nI);
  dense_gram_kernel<<<grid, 256, 0, st>>>(Minv, ldm, n, nI, XR, ldxr, k, XL, ldxl, WL, ldwl, y,
                                          q, P, ldp);
}

void launch_gesv(const double* P, int64_t ldp, int nI, int q, int64_t k, const double* F,
                 int ldf, const double* bT, double tau, double* B, int64_t ldb,
                 int32_t* status, cudaStream_t st) {
  gesv_kernel<<<(unsigned)ceil_div(k, 128), 128, 0, st>>>(P, ldp, nI, q, k, F, ldf, bT, tau, B,
                                                          ldb, status);
}

}  // namespace gls
