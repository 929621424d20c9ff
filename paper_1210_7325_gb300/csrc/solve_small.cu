// solve_small.cu -- per-SNP assembly of the p x p system and its Cholesky solve
// (Alg. 5 line 11, posv; Fig. 1 partition of S_i and b_i).
//
//   S_i = [ S_TL     S_BL_i^T ]     r_i = [ b_T   ]
//         [ S_BL_i   S_BR_i   ]           [ b_B_i ]
//
// The Cholesky factor of S_i is [[R_TL, 0], [r^T, delta]] with
//   R_TL R_TL^T = S_TL  (fixed for the whole sequence, factored once in the setup),
//   R_TL r = S_BL_i,    delta^2 = S_BR_i - r^T r,
// so the per-SNP part of the unpivoted Cholesky is one triangular solve of
// length p-1 and one pivot; the two triangular solves of posv then give
//   z_B = (b_B_i - r^T z_T) / delta,  b_SNP = z_B / delta,
//   b_cov = R_TL^{-T} (z_T - r b_SNP),   with z_T = R_TL^{-1} b_T (fixed).
// A pivot delta^2 <= tau * S_BR_i marks S_i as not SPD: b_i = NaN, status 1.
// With t phenotypes (Eq. 1's index j <= t), S_i and its factor are shared and
// only b_B_ij and z_T,j differ: one factor per SNP, t pairs of triangular
// solves, b_ij written to column i t + j of B.
//
// The Gram entries arrive as per-row-block partials P[I][q][j] and are summed
// over I in ascending order (deterministic, independent of the launch shape).
#include <math.h>

#include "common.cuh"

namespace gls {
namespace {

// Shared by the t phenotypes of one SNP: the per-SNP part of the Cholesky of
// S_i (which does not depend on the phenotype).  s = S_BL_i (length q) becomes
// r = R_TL^{-1} S_BL_i in place; returns delta = sqrt(S_BR_i - r^T r), or 0
// when the pivot fails (delta^2 <= tau S_BR_i).
__device__ __forceinline__ double factor_one(double (&s)[kMaxW], double sigma, int q,
                                             const double* R, double tau) {
  for (int a = 0; a < q; ++a) {
    double t = s[a];
    for (int c = 0; c < a; ++c) t -= R[a + c * q] * s[c];
    s[a] = t / R[a + a * q];
  }
  double d = sigma;
  for (int a = 0; a < q; ++a) d -= s[a] * s[a];
  if (!(d > tau * sigma)) return 0.0;
  return sqrt(d);
}

// One right-hand side: rho = b_B_ij = y~_j^T x~_i, z = z_T of phenotype j;
// writes the p = q + 1 entries of b_ij (X_L coefficients, then the SNP's).
__device__ __forceinline__ void solve_rhs(const double (&r)[kMaxW], double delta, double rho,
                                          int q, const double* R, const double* z, double* out) {
  double zb = rho;
  for (int a = 0; a < q; ++a) zb -= r[a] * z[a];
  zb /= delta;
  const double bsnp = zb / delta;
  double bt[kMaxW];
  for (int a = 0; a < q; ++a) bt[a] = z[a] - r[a] * bsnp;
  for (int a = q - 1; a >= 0; --a) {
    double t = bt[a];
    for (int c = a + 1; c < q; ++c) t -= R[c + a * q] * bt[c];
    bt[a] = t / R[a + a * q];
  }
  for (int a = 0; a < q; ++a) out[a] = bt[a];
  out[q] = bsnp;
}

// The whole SNP: one factor, t solves into columns j t + jj of B; a failed
// pivot gives NaN for every phenotype and status 1.
__device__ __forceinline__ void solve_snp(double (&s)[kMaxW], const double* rho, int64_t rho_ld,
                                          double sigma, int p, int t, const double* R,
                                          const double* z, double tau, double* Bj, int64_t ldb,
                                          int32_t* status_j) {
  const int q = p - 1;
  const double delta = factor_one(s, sigma, q, R, tau);
  if (delta == 0.0) {
    for (int jj = 0; jj < t; ++jj)
      for (int a = 0; a < p; ++a) Bj[a + jj * ldb] = __longlong_as_double(0x7ff8000000000000ll);
    if (status_j) *status_j = 1;
    return;
  }
  for (int jj = 0; jj < t; ++jj)
    solve_rhs(s, delta, rho[jj * rho_ld], q, R, z + jj * q, Bj + jj * ldb);
  if (status_j) *status_j = 0;
}

// FP64 path: partials P[I][a][j] for a <= nw (S_BL, the b_B, S_BR last),
// summed over I in ascending order; the first t b_B rows are used.
__global__ void __launch_bounds__(128) assemble_solve_kernel(
    const double* __restrict__ P, int64_t ldp, int nI, int p, int t, int nw, int64_t k,
    const double* __restrict__ RTL, const double* __restrict__ zT, double tau,
    double* __restrict__ B, int64_t ldb, int32_t* __restrict__ status) {
  __shared__ double R[kMaxW * kMaxW];
  __shared__ double z[kMaxW * kMaxW];
  const int q = p - 1;
  for (int i = threadIdx.x; i < q * q; i += blockDim.x) R[i] = RTL[i];
  for (int i = threadIdx.x; i < q * t; i += blockDim.x) z[i] = zT[i];
  __syncthreads();
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= k) return;
  double s[kMaxW];
  double rho[kMaxW];
  double sigma = 0.0;
  for (int a = 0; a < q; ++a) s[a] = 0.0;
  for (int a = 0; a < t; ++a) rho[a] = 0.0;
  for (int I = 0; I < nI; ++I) {
    const double* pi = P + (int64_t)I * (nw + 1) * ldp + j;
    for (int a = 0; a < q; ++a) s[a] += pi[(int64_t)a * ldp];
    for (int a = 0; a < t; ++a) rho[a] += pi[(int64_t)(q + a) * ldp];
    sigma += pi[(int64_t)nw * ldp];
  }
  solve_snp(s, rho, 1, sigma, p, t, R, z, tau, B + j * t * ldb, ldb,
            status ? status + j : nullptr);
}

// Mixed path: S_BL and the t b_B arrive whole in Glin[a][j]; S_BR as
// row-block partials Pbr[I][j], summed over I in ascending order.
__global__ void __launch_bounds__(128) assemble_solve_split_kernel(
    const double* __restrict__ Glin, const double* __restrict__ Pbr, int64_t ldp, int nI, int p,
    int t, int64_t k, const double* __restrict__ RTL, const double* __restrict__ zT, double tau,
    double* __restrict__ B, int64_t ldb, int32_t* __restrict__ status) {
  __shared__ double R[kMaxW * kMaxW];
  __shared__ double z[kMaxW * kMaxW];
  const int q = p - 1;
  for (int i = threadIdx.x; i < q * q; i += blockDim.x) R[i] = RTL[i];
  for (int i = threadIdx.x; i < q * t; i += blockDim.x) z[i] = zT[i];
  __syncthreads();
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= k) return;
  double s[kMaxW];
  for (int a = 0; a < q; ++a) s[a] = Glin[(int64_t)a * ldp + j];
  double sigma = 0.0;
  for (int I = 0; I < nI; ++I) sigma += Pbr[(int64_t)I * ldp + j];
  solve_snp(s, Glin + (int64_t)q * ldp + j, ldp, sigma, p, t, R, z, tau, B + j * t * ldb, ldb,
            status ? status + j : nullptr);
}

}  // namespace

void launch_assemble_solve(const double* partials, int64_t ldp, int nI, int p, int t, int nw,
                           int64_t k, const double* RTL, const double* zT, double tau,
                           double* B, int64_t ldb, int32_t* status, cudaStream_t st) {
  if (k <= 0) return;
  assemble_solve_kernel<<<(unsigned)ceil_div(k, 128), 128, 0, st>>>(
      partials, ldp, nI, p, t, nw, k, RTL, zT, tau, B, ldb, status);
}

void launch_assemble_solve_split(const double* Glin, const double* Pbr, int64_t ldp, int nI,
                                 int p, int t, int64_t k, const double* RTL, const double* zT,
                                 double tau, double* B, int64_t ldb, int32_t* status,
                                 cudaStream_t st) {
  if (k <= 0) return;
  assemble_solve_split_kernel<<<(unsigned)ceil_div(k, 128), 128, 0, st>>>(
      Glin, Pbr, ldp, nI, p, t, k, RTL, zT, tau, B, ldb, status);
}

}  // namespace gls
