// variants.cuh -- launchers of the comparison algorithms' kernels (variants.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gls {

// Largest p the comparison paths take (their per-SNP p x p systems live in
// registers and local memory; the paper compares the algorithms at p = 4).
constexpr int kVarMaxP = 8;

// mode 0: R = [X_L | x_j0 | y] (p + 1 columns); mode 1: [X_L | x_j] for the
// g SNPs j0 .. j0+g-1 (p columns each).  npad rows, rows >= n zero.
void launch_variant_rhs(const double* XL, int64_t ldxl, const double* y, const int8_t* XR,
                        int64_t ldxr, int64_t j0, int g, int64_t n, int64_t npad, int p,
                        int mode, double* R, int64_t ldr, cudaStream_t st);
// Per SNP s < g: S = X~^T X~, r = X~^T y~ with X~ = W[:, s cstride .. + p), then posv.
void launch_gram_posv(const double* W, int64_t ldw, int64_t n, int p, int cstride, int g,
                      const double* yt, double tau, double* B, int64_t ldb, int32_t* status,
                      cudaStream_t st);
// C (M x N) = A^T B, binary64.
void launch_gemm_tn(const double* A, int64_t lda, const double* B, int64_t ldb, double* C,
                    int64_t ldc, int64_t M, int64_t N, int64_t K, cudaStream_t st);
// Alg. 6 block: per 64-row block partials of w^T X_L, w^T y, w^T x, W_L^T x
// (2q + 2 rows) with w = Minv x, for the k SNP columns of XR.
void launch_dense_gram(const double* Minv, int64_t ldm, int64_t n, const int8_t* XR,
                       int64_t ldxr, int64_t k, const double* XL, int64_t ldxl,
                       const double* WL, int64_t ldwl, const double* y, int q, double* P,
                       int64_t ldp, cudaStream_t st);
// Alg. 6 per SNP: assemble S and r from F = W_L^T X_L (q x q, ldf), b_T and
// the partials, then gesv.
void launch_gesv(const double* P, int64_t ldp, int nI, int q, int64_t k, const double* F,
                 int ldf, const double* bT, double tau, double* B, int64_t ldb,
                 int32_t* status, cudaStream_t st);

}  // namespace gls
