// common.cuh -- shared definitions for the GB300 GLS kernels and the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gls {

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// FP64 factor/solve tile edge: L, L^{-1} and the FP64 blocked solve use 64 x 64 tiles.
constexpr int kT = 64;
constexpr int kMaxP = 32;
// Columns of the whitened right-hand block [X_L | Y]: p - 1 covariates plus
// t phenotypes, q + t <= kMaxW.
constexpr int kMaxW = 32;
// Largest number of problems one batched launch serves.
constexpr int kMaxBatch = 64;

// Device-side status words of a plan (one int32 each).
enum FlagSlot : int {
  kFlagPotrf = 0,   // 1-based failing pivot of M (first one), 0 if none
  kFlagSTL = 1,     // 1-based failing pivot of S_TL, 0 if none
  kFlagKernel = 2,  // KernelError bits raised by a kernel
  kFlagWhere = 3,   // diagnostic: which wait gave up
  kFlagCount = 8
};

enum KernelError : int { kErrNone = 0, kErrTimeout = 1, kErrBounds = 2, kErrConfig = 4 };

// Pivot thresholds of the p x p solve: pivot d <= tau * S_jj marks S_i as not SPD.
constexpr double kTauFP64 = 9.313225746154785e-10;   // 2^-30
constexpr double kTauMixed = 1.52587890625e-05;      // 2^-16

// ---------------------------------------------------------------------------
// Kernel launchers (defined in the .cu files; all asynchronous on `st`).
// ---------------------------------------------------------------------------

// factor_fp64.cu
void launch_pad_lower(double* A, int64_t lda, int64_t n, int64_t npad, cudaStream_t st);
void launch_identity(double* Z, int64_t ldz, int64_t npad, cudaStream_t st);
cudaError_t potrf_trtri_fp64(double* A, double* Z, int64_t ld, int64_t npad, int* flags,
                             cudaStream_t st);
void launch_whiten(const double* Z, int64_t ldz, int64_t n, int64_t npad, const double* rhs,
                   int64_t ldr, int ncols, double* out, int64_t ldo, const int* flags,
                   cudaStream_t st);
// gram (ncols x ncols) = W^T W over the n rows of W (npad x ncols).
void launch_fixed_gram(const double* W, int64_t ld, int64_t n, int ncols, double* gram,
                       cudaStream_t st);
// R_TL R_TL^T = gram[0:q, 0:q]; zT (q x t) = R_TL^{-1} gram[0:q, q:q+t] (ld of gram: ldg).
void launch_small_chol(const double* gram, int ldg, int q, int t, double* RTL, double* zT,
                       int* flags, cudaStream_t st);

// trsm_fp64.cu
cudaError_t launch_trsm_gram_fp64(const double* Z, int64_t ldz, int64_t n, int64_t npad,
                                  const int8_t* XR, int64_t ldxr, int64_t k, const double* W,
                                  int64_t ldw, int p, double* partials, int64_t ldp,
                                  cudaStream_t st);

// plan.cu: replaces the calling thread's gls_last_error() text.
void set_last_error_text(const char* msg);

// solve_small.cu.  t phenotypes: b_ij goes to column i t + j of B.
// FP64 partials: per row block nw + 1 rows (S_BL: q, b_B: nw - q of which the
// first t are used, S_BR last).
void launch_assemble_solve(const double* partials, int64_t ldp, int nrowblocks, int p, int t,
                           int nw, int64_t k, const double* RTL, const double* zT, double tau,
                           double* B, int64_t ldb, int32_t* status, cudaStream_t st);
void launch_assemble_solve_split(const double* Glin, const double* Pbr, int64_t ldp,
                                 int nrowblocks, int p, int t, int64_t k, const double* RTL,
                                 const double* zT, double tau, double* B, int64_t ldb,
                                 int32_t* status, cudaStream_t st);

// genotypes.cu: 2-bit packed genotype columns (ldp bytes each) -> int8 X_R (ldx)
cudaError_t launch_unpack2(const uint8_t* xp, int64_t ldp, int64_t n, int64_t k, int8_t* x,
                           int64_t ldx, cudaStream_t st);

}  // namespace gls
