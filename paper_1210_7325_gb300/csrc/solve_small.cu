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
//
// The Gram entries arrive as per-row-block partials P[I][q][j] and are summed
// over I in ascending order (deterministic, independent of the launch shape).
#include <math.h>

#include "common.cuh"

namespace gls {
namespace {

// The per-SNP part of the Cholesky solve of S_i, given s = S_BL_i (length q),
// rho = b_B_i and sigma = S_BR_i.  R (q x q) and z (q) are R_TL and z_T.
__device__ __forceinline__ void solve_one(double (&s)[kMaxP], double rho, double sigma, int p,
                                          const double* R, const double* z, double tau,
                                          double* out, int32_t* status_j) {
  const int q = p - 1;
  // r = R_TL^{-1} S_BL (in place in s)
  for (int a = 0; a < q; ++a) {
    double t = s[a];
    for (int c = 0; c < a; ++c) t -= R[a + c * q] * s[c];
    s[a] = t / R[a + a * q];
  }
  double d = sigma;
  for (int a = 0; a < q; ++a) d -= s[a] * s[a];
  if (!(d > tau * sigma)) {
    for (int a = 0; a < p; ++a) out[a] = __longlong_as_double(0x7ff8000000000000ll);
    if (status_j) *status_j = 1;
    return;
  }
  const double delta = sqrt(d);
  double zb = rho;
  for (int a = 0; a < q; ++a) zb -= s[a] * z[a];
  zb /= delta;
  const double bsnp = zb / delta;
  double bt[kMaxP];
  for (int a = 0; a < q; ++a) bt[a] = z[a] - s[a] * bsnp;
  for (int a = q - 1; a >= 0; --a) {
    double t = bt[a];
    for (int c = a + 1; c < q; ++c) t -= R[c + a * q] * bt[c];
    bt[a] = t / R[a + a * q];
  }
  for (int a = 0; a < q; ++a) out[a] = bt[a];
  out[q] = bsnp;
  if (status_j) *status_j = 0;
}

// FP64 path: partials P[I][a][j] for a <= p (S_BL..., b_B, S_BR), summed over I
// in ascending order.
__global__ void __launch_bounds__(128) assemble_solve_kernel(
    const double* __restrict__ P, int64_t ldp, int nI, int p, int64_t k,
    const double* __restrict__ RTL, const double* __restrict__ zT, double tau,
    double* __restrict__ B, int64_t ldb, int32_t* __restrict__ status) {
  __shared__ double R[kMaxP * kMaxP];
  __shared__ double z[kMaxP];
  const int q = p - 1;
  for (int t = threadIdx.x; t < q * q; t += blockDim.x) R[t] = RTL[t];
  for (int t = threadIdx.x; t < q; t += blockDim.x) z[t] = zT[t];
  __syncthreads();
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= k) return;
  double s[kMaxP];
  double rho = 0.0, sigma = 0.0;
  for (int a = 0; a < q; ++a) s[a] = 0.0;
  for (int I = 0; I < nI; ++I) {
    const double* pi = P + (int64_t)I * (p + 1) * ldp + j;
    for (int a = 0; a < q; ++a) s[a] += pi[(int64_t)a * ldp];
    rho += pi[(int64_t)q * ldp];
    sigma += pi[(int64_t)p * ldp];
  }
  solve_one(s, rho, sigma, p, R, z, tau, B + j * ldb, status ? status + j : nullptr);
}

// Mixed path: S_BL and b_B arrive whole in Glin[a][j]; S_BR as row-block
// partials Pbr[I][j], summed over I in ascending order.
__global__ void __launch_bounds__(128) assemble_solve_split_kernel(
    const double* __restrict__ Glin, const double* __restrict__ Pbr, int64_t ldp, int nI, int p,
    int64_t k, const double* __restrict__ RTL, const double* __restrict__ zT, double tau,
    double* __restrict__ B, int64_t ldb, int32_t* __restrict__ status) {
  __shared__ double R[kMaxP * kMaxP];
  __shared__ double z[kMaxP];
  const int q = p - 1;
  for (int t = threadIdx.x; t < q * q; t += blockDim.x) R[t] = RTL[t];
  for (int t = threadIdx.x; t < q; t += blockDim.x) z[t] = zT[t];
  __syncthreads();
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= k) return;
  double s[kMaxP];
  for (int a = 0; a < q; ++a) s[a] = Glin[(int64_t)a * ldp + j];
  const double rho = Glin[(int64_t)q * ldp + j];
  double sigma = 0.0;
  for (int I = 0; I < nI; ++I) sigma += Pbr[(int64_t)I * ldp + j];
  solve_one(s, rho, sigma, p, R, z, tau, B + j * ldb, status ? status + j : nullptr);
}

}  // namespace

void launch_assemble_solve(const double* partials, int64_t ldp, int nI, int p, int64_t k,
                           const double* RTL, const double* zT, double tau, double* B,
                           int64_t ldb, int32_t* status, cudaStream_t st) {
  if (k <= 0) return;
  assemble_solve_kernel<<<(unsigned)ceil_div(k, 128), 128, 0, st>>>(
      partials, ldp, nI, p, k, RTL, zT, tau, B, ldb, status);
}

void launch_assemble_solve_split(const double* Glin, const double* Pbr, int64_t ldp, int nI,
                                 int p, int64_t k, const double* RTL, const double* zT,
                                 double tau, double* B, int64_t ldb, int32_t* status,
                                 cudaStream_t st) {
  if (k <= 0) return;
  assemble_solve_split_kernel<<<(unsigned)ceil_div(k, 128), 128, 0, st>>>(
      Glin, Pbr, ldp, nI, p, k, RTL, zT, tau, B, ldb, status);
}

}  // namespace gls
