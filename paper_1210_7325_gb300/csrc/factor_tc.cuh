// factor_tc.cuh -- binary64 setup phase (Cholesky of M, L^{-1}, whitening) with
// its dense products evaluated exactly on tcgen05 tensor cores (factor_tc.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gls_gb300.h"

namespace gls {

struct TcFactor;

// Device bytes of the workspace tc_factor_create allocates for an npad x npad factor.
size_t tc_factor_bytes(int64_t npad);
gls_status_t tc_factor_create(TcFactor** out, int64_t npad);
void tc_factor_free(TcFactor* w);
const char* tc_factor_last_error();

// L L^T = A and Z = L^{-1} for the npad x npad column-major A (lower triangle
// read; npad a multiple of 64).  A is overwritten by L (zeros above the
// diagonal stay zero), Z must hold the identity on entry (only its upper
// triangle is kept).  A non-positive pivot records its 1-based index in
// flags[kFlagPotrf]; later kernels of the factor then do nothing.
cudaError_t tc_potrf_trtri(TcFactor* w, double* A, double* Z, int64_t ld, int64_t npad, int* flags,
                           cudaStream_t st);

// out (npad x ncols, ldo) = Z * rhs with Z lower triangular (ldz), rhs npad x ncols (ldr).
cudaError_t tc_lower_times(TcFactor* w, const double* Z, int64_t ldz, int64_t npad,
                           const double* rhs, int64_t ldr, int ncols, double* out, int64_t ldo,
                           int* flags, cudaStream_t st);

// out (npad x ncols, ldo) = Z^T * rhs with Z lower triangular.
cudaError_t tc_lower_t_times(TcFactor* w, const double* Z, int64_t ldz, int64_t npad,
                             const double* rhs, int64_t ldr, int ncols, double* out, int64_t ldo,
                             int* flags, cudaStream_t st);

// Kernels enqueued through this workspace so far (for the plan's launch count).
int64_t tc_launches(const TcFactor* w);

// Launcher of the binary64 64 x 64 diagonal-block Cholesky + inverse (factor_fp64.cu).
void launch_potrf_diag64(double* A, double* Z, int64_t ld, int64_t k0, int* flags,
                         cudaStream_t st);

}  // namespace gls
