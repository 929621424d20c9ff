// factor_fp64.cu -- setup phase of Alg. 5 (lines 1, 2, 4, 5, 6) in binary64.
//
//   L L^T = M                 blocked right-looking Cholesky on 64 x 64 tiles (potrf)
//   Z = L^{-1}                blocked triangular inverse, right-looking over block rows
//   [X~_L | y~] = Z [X_L | y] whitening of the covariates and the phenotype (trsm, trsv)
//   G = [X~_L | y~]^T [X~_L | y~]   gives S_TL = X~_L^T X~_L and b_T = X~_L^T y~ (syrk, gemv;
//                                     Fig. 1)
//   S_TL = R_TL R_TL^T, z_T = R_TL^{-1} b_T   leading block of every p x p Cholesky
//
// The matrices live in an npad x npad column-major array (npad = n rounded up
// to 64).  The padding is the identity, so the padded factor is diag(L, I) and
// the padded inverse is diag(L^{-1}, I): no tile needs a bounds check.
//
// GB300 note: binary64 arithmetic runs at a small fraction of the FP32 rate on
// this part, so these kernels aim at keeping the DFMA pipe busy (64 x 64 x 64
// tile products from shared memory, 16 accumulators per thread) rather than at
// memory traffic, which is negligible next to the n^3/3 flops.
#include <math.h>

#include "common.cuh"
#include "factor_tc.cuh"

namespace gls {
namespace {

constexpr int kLd = kT + 1;                         // padded shared-memory row (doubles)
constexpr size_t kTileSmem = 2 * kT * kLd * sizeof(double);

// In place on A (npad x npad, lda): keep the lower triangle of the n x n block,
// zero the strict upper triangle, identity on the padding.
__global__ void pad_lower_kernel(double* __restrict__ A, int64_t lda, int64_t n, int64_t npad) {
  const int64_t total = npad * npad;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = idx / npad, i = idx - j * npad;
    double* a = A + i + j * lda;
    if (i < j) {
      *a = 0.0;
    } else if (i >= n) {
      *a = (i == j) ? 1.0 : 0.0;
    }
  }
}

__global__ void identity_kernel(double* __restrict__ Z, int64_t ldz, int64_t npad) {
  const int64_t total = npad * npad;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = idx / npad, i = idx - j * npad;
    Z[i + j * ldz] = (i == j) ? 1.0 : 0.0;
  }
}

// 1/sqrt(d): the FP32 estimate refined by two binary64 Newton steps.
__device__ __forceinline__ double rsqrt_newton(double d) {
  if (d > 1e-30 && d < 1e30) {
    const double h = 0.5 * d;
    double r = (double)rsqrtf((float)d);
    r = r * fma(-h * r, r, 1.5);
    r = r * fma(-h * r, r, 1.5);
    return r;
  }
  return 1.0 / sqrt(d);
}

// Cholesky of the 64 x 64 diagonal block at (k0, k0) and its triangular
// inverse.  One CTA.  The block already carries every update of the earlier
// block columns.  A pivot <= 0 records its 1-based global index in
// flags[kFlagPotrf] (first failure wins) and stops.
//
// Right-looking over the 64 columns, the Cholesky and the inverse in the same
// sweep.  At column j the first 64 threads scale column j of L and row j of
// W = L^{-1} by r_j = 1/L_jj (one element each); then warps 1-15 apply the
// rank-1 updates S_il -= L_ij L_lj (j < l <= i, except S_{j+1,j+1}) and
// W_ic -= L_ij W_jc (c <= j < i), numbered densely so that every lane of every
// binary64 instruction does useful work, while thread 0 forms the next pivot
// d_{j+1} = S_{j+1,j+1} - L_{j+1,j}^2 and r_{j+1}.
// Dependent binary64 operations take about 64 cycles each on this part, so the
// pivot's chain (about 700 cycles) runs beside the column's update instead of
// before it.  The column loop is latency-bound, so the CTA has 16 warps: the
// more warps share a column's update, the more of its latency they hide.
constexpr int kLeafThreads = 512;

__global__ void __launch_bounds__(kLeafThreads) potrf_diag_kernel(double* __restrict__ A,
                                                         double* __restrict__ Z, int64_t ld,
                                                         int64_t k0, int* flags) {
  extern __shared__ double sm[];
  double(*S)[kLd] = reinterpret_cast<double(*)[kLd]>(sm);            // S[i][l], lower
  double(*W)[kLd] = reinterpret_cast<double(*)[kLd]>(sm + kT * kLd);  // W[i][c], lower
  __shared__ int fail;
  __shared__ double piv_d, piv_r;  // d_j and 1/sqrt(d_j) of the column to scale next
  // tri[q] = (a << 8) | b for the q-th entry (a, b), b <= a, of a lower triangle
  // numbered row by row; the trailing triangle of every column is a prefix
  __shared__ uint16_t tri[(kT - 1) * kT / 2];
  const int tid = threadIdx.x;
  if (*(volatile int*)&flags[kFlagPotrf] != 0) return;
  for (int idx = tid; idx < kT * kT; idx += blockDim.x) {
    const int i = idx % kT, l = idx / kT;  // unit stride along i (column-major A)
    S[i][l] = (i >= l) ? A[(k0 + i) + (k0 + l) * ld] : 0.0;
    W[i][l] = (i == l) ? 1.0 : 0.0;
  }
  for (int a = tid; a < kT - 1; a += blockDim.x)
    for (int b = 0; b <= a; ++b) tri[a * (a + 1) / 2 + b] = (uint16_t)((a << 8) | b);
  if (tid == 0) fail = 0;
  __syncthreads();
  if (tid == 0) {
    const double d = S[0][0];
    if (!(d > 0.0)) {
      fail = 1;
    } else {
      piv_d = d;
      piv_r = rsqrt_newton(d);
    }
  }
  __syncthreads();
  constexpr int kUpd = kLeafThreads - 32;  // threads of warps 1-15
  for (int j = 0; j < kT; ++j) {
    if (fail) break;
    // column j of L and row j of W: one element per thread of the first 64
    if (tid < kT) {
      const double r = piv_r;
      if (tid > j) S[tid][j] *= r;
      else W[j][tid] *= r;
      if (tid == 0) S[j][j] = piv_d * r;
    }
    __syncthreads();
    if (tid == 0) {
      // the next pivot; the update below leaves S_{j+1,j+1} to this thread
      if (j + 1 < kT) {
        const double l = S[j + 1][j];
        const double d = fma(-l, l, S[j + 1][j + 1]);
        if (!(d > 0.0)) {
          fail = j + 2;
        } else {
          piv_d = d;
          piv_r = rsqrt_newton(d);
        }
      }
    } else if (tid >= 32) {
      const int m = kT - 1 - j, ns = m * (m + 1) / 2, total = ns + m * (j + 1);
      const float rj = 1.0f / (float)(j + 1);
      for (int q0 = tid - 32 + 1; q0 < total; q0 += 4 * kUpd) {  // q = 0 is S_{j+1,j+1}
        double av[4], bv[4], lv[4];
        double* dst[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int q = q0 + u * kUpd;
          dst[u] = nullptr;
          if (q < total) {
            int i;
            if (q < ns) {
              const int e = tri[q];
              const int l = j + 1 + (e & 0xFF);
              i = j + 1 + (e >> 8);
              dst[u] = &S[i][l];
              bv[u] = S[l][j];
            } else {
              // (r + 1/2) / (j + 1) is at least 1/128 away from an integer, so
              // the FP32 quotient truncates to the exact row index
              const int r = q - ns, ip = (int)(((float)r + 0.5f) * rj), c = r - ip * (j + 1);
              i = j + 1 + ip;
              dst[u] = &W[i][c];
              bv[u] = W[j][c];
            }
            lv[u] = S[i][j];
            av[u] = *dst[u];
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (dst[u]) *dst[u] = fma(-lv[u], bv[u], av[u]);
      }
    }
    __syncthreads();
  }
  if (fail) {
    if (tid == 0) atomicCAS(&flags[kFlagPotrf], 0, (int)(k0 + fail));
    return;
  }
  for (int idx = tid; idx < kT * kT; idx += blockDim.x) {
    const int i = idx % kT, l = idx / kT;
    A[(k0 + i) + (k0 + l) * ld] = (i >= l) ? S[i][l] : 0.0;
    Z[(k0 + i) + (k0 + l) * ld] = (i >= l) ? W[i][l] : 0.0;
  }
}

enum GemmMode : int { kPanel = 0, kSyrk = 1, kTrtriRow = 2, kTrtriUpd = 3 };

// One 64 x 64 output tile, C = op(A) * op(B) (64-deep), or C -= ... .
//   kPanel    L_IK  = A_IK Z_KK^T            I > K        (panel solve by the block inverse)
//   kSyrk     L_IJ -= L_IK L_JK^T            K < J <= I   (trailing update)
//   kTrtriRow Z_KJ  = Z_KK B_KJ              J < K        (block row K of L^{-1}, in place)
//   kTrtriUpd B_IJ -= L_IK Z_KJ              I > K, J<=K  (right-hand sides of later rows)
// Both operands are staged whole in shared memory before any store, so the
// in-place modes are safe.
__global__ void __launch_bounds__(256) tile_gemm_kernel(double* __restrict__ L,
                                                        double* __restrict__ Z, int64_t ld,
                                                        int K, int mode, const int* flags) {
  if (*(volatile const int*)&flags[kFlagPotrf] != 0) return;
  extern __shared__ double sm[];
  double(*As)[kLd] = reinterpret_cast<double(*)[kLd]>(sm);           // As[i][k]
  double(*Bs)[kLd] = reinterpret_cast<double(*)[kLd]>(sm + kT * kLd);  // Bs[k][j]
  const int64_t bx = blockIdx.x;
  int64_t ti = 0, tj = 0;
  const double* Ab = nullptr;
  const double* Bb = nullptr;
  int64_t b_sk = 1, b_sj = ld;
  double* Cb = nullptr;
  bool sub = false;
  const int64_t K64 = (int64_t)K * kT;
  switch (mode) {
    case kPanel:
      ti = K + 1 + bx;
      tj = K;
      Ab = L + ti * kT + K64 * ld;
      Bb = Z + K64 + K64 * ld;  // B(k, j) = Z_KK(j, k)
      b_sk = ld;
      b_sj = 1;
      Cb = L + ti * kT + tj * kT * ld;
      break;
    case kSyrk: {
      int64_t a = (int64_t)((sqrt(8.0 * (double)bx + 1.0) - 1.0) * 0.5);
      while (a * (a + 1) / 2 > bx) --a;
      while ((a + 1) * (a + 2) / 2 <= bx) ++a;
      const int64_t b = bx - a * (a + 1) / 2;
      ti = K + 1 + a;
      tj = K + 1 + b;
      Ab = L + ti * kT + K64 * ld;
      Bb = L + tj * kT + K64 * ld;  // B(k, j) = L(J64 + j, K64 + k)
      b_sk = ld;
      b_sj = 1;
      Cb = L + ti * kT + tj * kT * ld;
      sub = true;
      break;
    }
    case kTrtriRow:
      ti = K;
      tj = bx;
      Ab = Z + K64 + K64 * ld;
      Bb = Z + K64 + tj * kT * ld;  // B(k, j) = Z(K64 + k, J64 + j)
      b_sk = 1;
      b_sj = ld;
      Cb = Z + ti * kT + tj * kT * ld;
      break;
    default:  // kTrtriUpd
      ti = K + 1 + bx / (K + 1);
      tj = bx % (K + 1);
      Ab = L + ti * kT + K64 * ld;
      Bb = Z + K64 + tj * kT * ld;
      b_sk = 1;
      b_sj = ld;
      Cb = Z + ti * kT + tj * kT * ld;
      sub = true;
      break;
  }
  const int tid = threadIdx.x;
  for (int idx = tid; idx < kT * kT; idx += blockDim.x) {
    const int i = idx % kT, k = idx / kT;  // unit stride along i (column-major)
    As[i][k] = Ab[i + (int64_t)k * ld];
  }
  for (int idx = tid; idx < kT * kT; idx += blockDim.x) {
    const int f = idx % kT, s = idx / kT;  // f walks the unit-stride index
    if (b_sj == 1) Bs[s][f] = Bb[(int64_t)s * b_sk + f];
    else Bs[f][s] = Bb[f + (int64_t)s * b_sj];
  }
  __syncthreads();
  const int tx = tid % 16, ty = tid / 16;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
#pragma unroll 4
  for (int k = 0; k < kT; ++k) {
    double av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = As[tx + 16 * a][k];
#pragma unroll
    for (int b = 0; b < 4; ++b) bv[b] = Bs[k][ty + 16 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      double* c = Cb + (tx + 16 * a) + (int64_t)(ty + 16 * b) * ld;
      *c = sub ? (*c - acc[a][b]) : acc[a][b];
    }
}

// out(r, q) = sum_{c <= r} Z(r, c) rhs(c, q) for r < npad, q < ncols (<= 32);
// rhs rows >= n count as zero.  One CTA per 64 rows, fixed summation order.
__global__ void __launch_bounds__(256) whiten_kernel(const double* __restrict__ Z, int64_t ldz,
                                                     int64_t n, const double* __restrict__ rhs,
                                                     int64_t ldr, int ncols,
                                                     double* __restrict__ out, int64_t ldo,
                                                     const int* flags) {
  if (*(volatile const int*)&flags[kFlagPotrf] != 0) return;
  extern __shared__ double sm[];
  double(*Zs)[kLd] = reinterpret_cast<double(*)[kLd]>(sm);     // Zs[c][i]
  double(*Rs)[kMaxP + 1] = reinterpret_cast<double(*)[kMaxP + 1]>(sm + kT * kLd);  // Rs[c][q]
  const int64_t r0 = (int64_t)blockIdx.x * kT;
  const int tid = threadIdx.x;
  const int i = tid % kT, qg = tid / kT;  // 4 column groups
  double acc[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) acc[t] = 0.0;
  for (int64_t c0 = 0; c0 < r0 + kT; c0 += kT) {
    for (int idx = tid; idx < kT * kT; idx += blockDim.x) {
      const int ii = idx % kT, cc = idx / kT;
      Zs[cc][ii] = Z[(r0 + ii) + (c0 + cc) * ldz];
    }
    for (int idx = tid; idx < kT * ncols; idx += blockDim.x) {
      const int cc = idx % kT, q = idx / kT;
      const int64_t c = c0 + cc;
      Rs[cc][q] = (c < n) ? rhs[c + q * ldr] : 0.0;
    }
    __syncthreads();
    for (int cc = 0; cc < kT; ++cc) {
      const double z = Zs[cc][i];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int q = qg + 4 * t;
        if (q < ncols) acc[t] = fma(z, Rs[cc][q], acc[t]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int q = qg + 4 * t;
    if (q < ncols) out[(r0 + i) + q * ldo] = acc[t];
  }
}

// G(a, c) = sum_{r < n} W(r, a) W(r, c) for the p columns of W (covariates
// and phenotypes); one CTA per pair a >= c, each thread summing a fixed stride
// in order, then a fixed tree.
__global__ void __launch_bounds__(256) fixed_gram_kernel(const double* __restrict__ W,
                                                         int64_t ld, int64_t n, int p,
                                                         double* __restrict__ G) {
  int64_t pr = blockIdx.x;
  int a = 0;
  while ((a + 1) * (a + 2) / 2 <= pr) ++a;
  const int c = (int)(pr - (int64_t)a * (a + 1) / 2);
  const double* wa = W + (int64_t)a * ld;
  const double* wc = W + (int64_t)c * ld;
  double s = 0.0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) s = fma(wa[r], wc[r], s);
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    G[a + (int64_t)c * p] = red[0];
    G[c + (int64_t)a * p] = red[0];
  }
}

// S_TL = G[0:q, 0:q] = R_TL R_TL^T (pivot rule d <= tau S_jj fails), and for
// each phenotype h < t, z_T,h = R_TL^{-1} b_T,h with b_T,h = G[0:q, q + h]
// (G is ldg x ldg).  One thread; q + t <= 32.
__global__ void small_chol_kernel(const double* __restrict__ G, int ldg, int q, int t,
                                  double* __restrict__ R, double* __restrict__ zT, int* flags) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (*(volatile int*)&flags[kFlagPotrf] != 0) return;
  const int64_t p = ldg;
  for (int j = 0; j < q; ++j) {
    const double sjj = G[j + (int64_t)j * p];
    double d = sjj;
    for (int k = 0; k < j; ++k) d -= R[j + k * q] * R[j + k * q];
    if (!(d > kTauFP64 * sjj)) {
      flags[kFlagSTL] = j + 1;
      return;
    }
    const double rjj = sqrt(d);
    R[j + j * q] = rjj;
    for (int i = j + 1; i < q; ++i) {
      double s = G[i + (int64_t)j * p];
      for (int k = 0; k < j; ++k) s -= R[i + k * q] * R[j + k * q];
      R[i + j * q] = s / rjj;
    }
    for (int i = 0; i < j; ++i) R[i + j * q] = 0.0;
  }
  for (int h = 0; h < t; ++h) {
    double* z = zT + (int64_t)h * q;
    for (int i = 0; i < q; ++i) {
      double s = G[i + (int64_t)(q + h) * p];
      for (int k = 0; k < i; ++k) s -= R[i + k * q] * z[k];
      z[i] = s / R[i + i * q];
    }
  }
}

inline int grid_for(int64_t total, int threads) {
  int64_t g = ceil_div(total, threads);
  return (int)(g > 65535 * 8 ? 65535 * 8 : (g < 1 ? 1 : g));
}

bool g_attrs_set = false;

cudaError_t set_attrs() {
  if (g_attrs_set) return cudaSuccess;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(potrf_diag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kTileSmem)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(tile_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kTileSmem)) != cudaSuccess)
    return e;
  const int wsm = (int)((kT * kLd + kT * (kMaxP + 1)) * sizeof(double));
  if ((e = cudaFuncSetAttribute(whiten_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                wsm)) != cudaSuccess)
    return e;
  g_attrs_set = true;
  return cudaSuccess;
}

}  // namespace

void launch_pad_lower(double* A, int64_t lda, int64_t n, int64_t npad, cudaStream_t st) {
  pad_lower_kernel<<<grid_for(npad * npad, 256), 256, 0, st>>>(A, lda, n, npad);
}

void launch_identity(double* Z, int64_t ldz, int64_t npad, cudaStream_t st) {
  identity_kernel<<<grid_for(npad * npad, 256), 256, 0, st>>>(Z, ldz, npad);
}

cudaError_t potrf_trtri_fp64(double* A, double* Z, int64_t ld, int64_t npad, int* flags,
                             cudaStream_t st) {
  cudaError_t e = set_attrs();
  if (e != cudaSuccess) return e;
  const int N = (int)(npad / kT);
  for (int K = 0; K < N; ++K) {
    potrf_diag_kernel<<<1, kLeafThreads, kTileSmem, st>>>(A, Z, ld, (int64_t)K * kT, flags);
    const int64_t m = N - K - 1;
    if (m > 0) {
      tile_gemm_kernel<<<(unsigned)m, 256, kTileSmem, st>>>(A, Z, ld, K, kPanel, flags);
      tile_gemm_kernel<<<(unsigned)(m * (m + 1) / 2), 256, kTileSmem, st>>>(A, Z, ld, K, kSyrk,
                                                                            flags);
    }
  }
  for (int K = 0; K < N; ++K) {
    if (K > 0) tile_gemm_kernel<<<(unsigned)K, 256, kTileSmem, st>>>(A, Z, ld, K, kTrtriRow, flags);
    const int64_t m = N - K - 1;
    if (m > 0)
      tile_gemm_kernel<<<(unsigned)(m * (K + 1)), 256, kTileSmem, st>>>(A, Z, ld, K, kTrtriUpd,
                                                                        flags);
  }
  return cudaGetLastError();
}

void launch_potrf_diag64(double* A, double* Z, int64_t ld, int64_t k0, int* flags,
                         cudaStream_t st) {
  if (set_attrs() != cudaSuccess) return;
  potrf_diag_kernel<<<1, kLeafThreads, kTileSmem, st>>>(A, Z, ld, k0, flags);
}

void launch_whiten(const double* Z, int64_t ldz, int64_t n, int64_t npad, const double* rhs,
                   int64_t ldr, int ncols, double* out, int64_t ldo, const int* flags,
                   cudaStream_t st) {
  if (set_attrs() != cudaSuccess) return;
  const size_t smem = (kT * kLd + kT * (kMaxP + 1)) * sizeof(double);
  whiten_kernel<<<(unsigned)(npad / kT), 256, smem, st>>>(Z, ldz, n, rhs, ldr, ncols, out, ldo,
                                                          flags);
}

void launch_fixed_gram(const double* W, int64_t ld, int64_t n, int p, double* gram,
                       cudaStream_t st) {
  fixed_gram_kernel<<<(unsigned)(p * (p + 1) / 2), 256, 0, st>>>(W, ld, n, p, gram);
}

void launch_small_chol(const double* gram, int ldg, int q, int t, double* RTL, double* zT,
                       int* flags, cudaStream_t st) {
  small_chol_kernel<<<1, 32, 0, st>>>(gram, ldg, q, t, RTL, zT, flags);
}

}  // namespace gls
