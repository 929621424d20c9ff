// genotypes.cu -- 2-bit packed genotype blocks -> the int8 layout of X_R.
//
// A packed block holds k SNP columns of ldp bytes each (ldp >= ceil(n/4)).
// Genotype i of column j is the 2-bit code in bits 2 (i mod 4) .. 2 (i mod 4)
// + 1 of byte floor(i / 4) of the column (the first sample in the lowest
// bits), read as the value 0..3; the codes 0, 1, 2 are the genotype dosages
// of X_R.  Four genotypes per byte cut the host-to-device bytes of a block to
// a quarter of the int8 form.
#include <stdint.h>

#include <algorithm>

#include "common.cuh"

namespace gls {
namespace {

// One thread per packed byte: four int8 outputs (one 32-bit store when the
// output is 4-byte aligned).  Rows i >= n, the padding bits of a column's
// last byte, are not written.
__global__ void __launch_bounds__(256) unpack2_kernel(const uint8_t* __restrict__ xp,
                                                      int64_t ldp, int64_t n, int64_t k,
                                                      int8_t* __restrict__ x, int64_t ldx,
                                                      int vec) {
  const int64_t pb = (n + 3) / 4;
  const int64_t total = pb * k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = t / pb, b = t - j * pb;
    const uint32_t v = xp[j * ldp + b];
    const int64_t i0 = 4 * b;
    int8_t* dst = x + j * ldx + i0;
    if (vec && i0 + 4 <= n) {
      *reinterpret_cast<uint32_t*>(dst) = (v & 3u) | (((v >> 2) & 3u) << 8) |
                                          (((v >> 4) & 3u) << 16) | ((v >> 6) << 24);
    } else {
      for (int q = 0; q < 4 && i0 + q < n; ++q) dst[q] = (int8_t)((v >> (2 * q)) & 3u);
    }
  }
}

}  // namespace

cudaError_t launch_unpack2(const uint8_t* xp, int64_t ldp, int64_t n, int64_t k, int8_t* x,
                           int64_t ldx, cudaStream_t st) {
  if (n <= 0 || k <= 0) return cudaSuccess;
  const int64_t total = ceil_div(n, 4) * k;
  const int64_t grid = std::min<int64_t>(ceil_div(total, 256), 152 * 16);
  const int vec = ((ldx & 3) == 0 && (reinterpret_cast<uintptr_t>(x) & 3) == 0) ? 1 : 0;
  unpack2_kernel<<<(unsigned)grid, 256, 0, st>>>(xp, ldp, n, k, x, ldx, vec);
  return cudaGetLastError();
}

}  // namespace gls
