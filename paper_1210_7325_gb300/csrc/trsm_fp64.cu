// trsm_fp64.cu -- binary64 blocked triangular solve of a block of SNP columns with
// the Gram epilogue fused in (Alg. 5 lines 3 and 8-10).
//
// For a 64-row block I and a 64-SNP tile J:
//   X~[I, J] = sum_{K <= I} Z[I, K] X[K, J]      Z = L^{-1} (lower, from the setup)
// and, without ever storing X~, the per-SNP Gram partials over the rows of I:
//   P[I][q][j] = sum_{r in I} W(r, q) x~(r, j)   q < p   (W = [X~_L | y~]: S_BL, b_B)
//   P[I][p][j] = sum_{r in I} x~(r, j)^2                 (S_BR)
// The partials are summed over I in a fixed order by the assemble kernel.
//
// Using the block inverse turns the blocked solve into independent tile
// products: there is no dependency chain between row blocks, so every
// (I, J) tile is its own CTA (heaviest rows first).
#include "common.cuh"

namespace gls {
namespace {

constexpr int TR = 64;  // rows per tile
constexpr int TS = 64;  // SNPs per tile
constexpr int KC = 32;  // K chunk

struct Smem {
  double Zs[KC][TR];          // Zs[kk][i] = Z(r0 + i, c0 + kk)
  double Xs[KC][TS];          // Xs[kk][j] = X(c0 + kk, j0 + j)
  double T[TR][TS + 1];       // x~ tile
  double Ws[TR][kMaxP + 1];   // W rows of the tile
};

__global__ void __launch_bounds__(256) trsm_gram_fp64_kernel(
    const double* __restrict__ Z, int64_t ldz, int64_t n, int nI, const int8_t* __restrict__ XR,
    int64_t ldxr, int64_t k, const double* __restrict__ W, int64_t ldw, int p,
    double* __restrict__ P, int64_t ldp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& s = *reinterpret_cast<Smem*>(smem_raw);
  const int I = nI - 1 - (int)blockIdx.y;
  const int64_t r0 = (int64_t)I * TR;
  const int64_t j0 = (int64_t)blockIdx.x * TS;
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;

  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;

  const int64_t kend = r0 + TR;  // Z is zero above the diagonal
  for (int64_t c0 = 0; c0 < kend; c0 += KC) {
    // Z chunk: 64 rows x 32 columns, column-major source -> coalesced along i
    for (int idx = tid; idx < TR * KC; idx += 256) {
      const int i = idx % TR, kk = idx / TR;
      s.Zs[kk][i] = Z[(r0 + i) + (c0 + kk) * ldz];
    }
    // genotype chunk: 32 rows x 64 SNPs; thread -> (SNP, 8 consecutive rows)
    {
      const int j = tid / 4, kk0 = (tid % 4) * 8;
      const int64_t jj = j0 + j;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int64_t c = c0 + kk0 + e;
        double v = 0.0;
        if (jj < k && c < n) v = (double)XR[c + jj * ldxr];
        s.Xs[kk0 + e][j] = v;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KC; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = s.Zs[kk][tx + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = s.Xs[kk][ty + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }

  // ---- Gram epilogue -------------------------------------------------------
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) s.T[tx + 16 * a][ty + 16 * b] = acc[a][b];
  for (int idx = tid; idx < TR * p; idx += 256) {
    const int i = idx % TR, q = idx / TR;
    s.Ws[i][q] = W[(r0 + i) + (int64_t)q * ldw];
  }
  __syncthreads();
  // thread -> (SNP j, row group g of 16 rows); the 4 groups of a SNP are adjacent lanes
  const int j = tid / 4, g = tid % 4;
  double part[kMaxP + 1];
#pragma unroll
  for (int q = 0; q <= kMaxP; ++q) part[q] = 0.0;
  for (int i = g * 16; i < g * 16 + 16; ++i) {
    const double x = s.T[i][j];
#pragma unroll
    for (int q = 0; q < kMaxP; ++q)
      if (q < p) part[q] = fma(s.Ws[i][q], x, part[q]);
    part[kMaxP] = fma(x, x, part[kMaxP]);
  }
#pragma unroll
  for (int q = 0; q <= kMaxP; ++q) {
    part[q] += __shfl_xor_sync(0xffffffffu, part[q], 1);
    part[q] += __shfl_xor_sync(0xffffffffu, part[q], 2);
  }
  const int64_t jj = j0 + j;
  if (g == 0 && jj < k) {
    double* out = P + (int64_t)I * (p + 1) * ldp + jj;
#pragma unroll
    for (int q = 0; q < kMaxP; ++q)
      if (q < p) out[(int64_t)q * ldp] = part[q];
    out[(int64_t)p * ldp] = part[kMaxP];
  }
}

bool g_attr = false;

}  // namespace

cudaError_t launch_trsm_gram_fp64(const double* Z, int64_t ldz, int64_t n, int64_t npad,
                                  const int8_t* XR, int64_t ldxr, int64_t k, const double* W,
                                  int64_t ldw, int p, double* partials, int64_t ldp,
                                  cudaStream_t st) {
  if (!g_attr) {
    cudaError_t e = cudaFuncSetAttribute(trsm_gram_fp64_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(Smem));
    if (e != cudaSuccess) return e;
    g_attr = true;
  }
  const int nI = (int)(npad / TR);
  dim3 grid((unsigned)ceil_div(k, TS), (unsigned)nI);
  trsm_gram_fp64_kernel<<<grid, 256, sizeof(Smem), st>>>(Z, ldz, n, nI, XR, ldxr, k, W, ldw, p,
                                                         partials, ldp);
  return cudaGetLastError();
}

int fp64_rows_per_tile() { return TR; }

}  // namespace gls
