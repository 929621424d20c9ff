// static_solve.cu -- an allocation-free variant of the FP64 block solve
// (gls_solve_block_fp64_static in include/gls_gb300.h).
//
// Some callers cannot call cudaMalloc at all: code running where another
// allocator owns the device memory (a framework's caching pool), real-time
// loops that must not enter the driver's allocator, or embedding hosts that
// forbid it.  For them this entry point takes every input and output as a
// caller-owned device buffer and keeps its only scratch -- the per-row-block
// Gram partials of the blocked solve -- in a fixed file-scope device array.
//
// The array (kStaticPartials doubles, 4 MiB) is part of the library image:
// every GPU that loads the library holds its own copy until the process exits.
// Calls on the same device share that copy and it keeps the last call's
// contents; nothing in it has to start at zero, because each call writes every
// partial it later reads.  Two calls on one device whose kernels can overlap
// on the GPU (for example calls on different streams, or from different host
// threads) race on it: the caller orders them.  Calls on different devices
// use different copies.
#include <cuda.h>

#include <mutex>

#include "common.cuh"
#include "gls_gb300.h"

namespace {

constexpr int64_t kStaticPartials = 524288;  // doubles (4 MiB)
constexpr int TR = 64, TS = 64, KC = 32;
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_static_partials[kStaticPartials];

// Set-up state per device, valid for the context it was made in: a device
// reset (cudaDeviceReset) ends that context and reloads the library's module
// in the next one, which moves the array, so a new context id redoes the set-up.
struct DeviceSetup {
  unsigned long long ctx_id = 0;
  double* scratch = nullptr;  // device address of g_static_partials
};
std::mutex g_mu;
DeviceSetup g_setup[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Unique id of the calling thread's current context (0 if it cannot be read).
unsigned long long current_context_id() {
  static const CtxGetCurrentFn get_current = []() {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return static_cast<CtxGetCurrentFn>(nullptr);
    }
    return reinterpret_cast<CtxGetCurrentFn>(f);
  }();
  static const CtxGetIdFn get_id = []() {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return static_cast<CtxGetIdFn>(nullptr);
    }
    return reinterpret_cast<CtxGetIdFn>(f);
  }();
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx ||
      get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

struct Smem {
  double Zs[KC][TR];
  double Xs[KC][TS];
  double T[TR][TS + 1];
  double Ws[TR][gls::kMaxP + 1];
};

// Bounds-checked form of the FP64 blocked solve + Gram epilogue: Z is the
// caller's n x n L^{-1} (only c <= r is read), W the caller's n x p
// [X~_L | y~]; rows and columns beyond n count as zero.
__global__ void __launch_bounds__(256) trsm_gram_fp64_static_kernel(
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
  for (int64_t c0 = 0; c0 < r0 + TR; c0 += KC) {
    for (int idx = tid; idx < TR * KC; idx += 256) {
      const int i = idx % TR, kk = idx / TR;
      const int64_t r = r0 + i, c = c0 + kk;
      s.Zs[kk][i] = (r < n && c <= r) ? Z[r + c * ldz] : 0.0;
    }
    {
      const int j = tid / 4, kk0 = (tid % 4) * 8;
      const int64_t jj = j0 + j;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int64_t c = c0 + kk0 + e;
        s.Xs[kk0 + e][j] = (jj < k && c < n) ? (double)XR[c + jj * ldxr] : 0.0;
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
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) s.T[tx + 16 * a][ty + 16 * b] = acc[a][b];
  for (int idx = tid; idx < TR * p; idx += 256) {
    const int i = idx % TR, q = idx / TR;
    const int64_t r = r0 + i;
    s.Ws[i][q] = (r < n) ? W[r + (int64_t)q * ldw] : 0.0;
  }
  __syncthreads();
  const int j = tid / 4, g = tid % 4;
  double part[gls::kMaxP + 1];
#pragma unroll
  for (int q = 0; q <= gls::kMaxP; ++q) part[q] = 0.0;
  for (int i = g * 16; i < g * 16 + 16; ++i) {
    const double x = s.T[i][j];
#pragma unroll
    for (int q = 0; q < gls::kMaxP; ++q)
      if (q < p) part[q] = fma(s.Ws[i][q], x, part[q]);
    part[gls::kMaxP] = fma(x, x, part[gls::kMaxP]);
  }
#pragma unroll
  for (int q = 0; q <= gls::kMaxP; ++q) {
    part[q] += __shfl_xor_sync(0xffffffffu, part[q], 1);
    part[q] += __shfl_xor_sync(0xffffffffu, part[q], 2);
  }
  const int64_t jj = j0 + j;
  if (g == 0 && jj < k) {
    double* out = P + (int64_t)I * (p + 1) * ldp + jj;
#pragma unroll
    for (int q = 0; q < gls::kMaxP; ++q)
      if (q < p) out[(int64_t)q * ldp] = part[q];
    out[(int64_t)p * ldp] = part[gls::kMaxP];
  }
}

gls_status_t fail(gls_status_t st, const char* msg) {
  gls::set_last_error_text(msg);
  return st;
}

}  // namespace

extern "C" gls_status_t gls_solve_block_fp64_static(int64_t n, int32_t p, const double* Zinv,
                                                    int64_t ldz, const double* W, int64_t ldw,
                                                    const double* RTL, const double* zT,
                                                    const int8_t* XR, int64_t ldxr, int64_t k,
                                                    double* B, int64_t ldb, int32_t* snp_status,
                                                    void* stream) {
  gls::set_last_error_text("");
  if (n < 1 || p < 1 || p > gls::kMaxP || k < 0 || ldz < n || ldw < n || ldxr < n || ldb < p)
    return fail(GLS_ERR_INVALID_ARG, "bad size or leading dimension");
  if (k == 0) return GLS_OK;
  if (!Zinv || !W || !XR || !B || (p > 1 && (!RTL || !zT)))
    return fail(GLS_ERR_INVALID_ARG, "NULL input or output");
  const int nI = (int)gls::ceil_div(n, TR);
  if ((int64_t)nI * (p + 1) * k > kStaticPartials)
    return fail(GLS_ERR_INVALID_ARG,
                "ceil(n/64) * (p+1) * k exceeds the 524288-double (4 MiB) static scratch");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return fail(GLS_ERR_CUDA, "no current CUDA device");
  }
  // 0 when no context is current yet: the set-up below makes the primary one
  const unsigned long long ctx = current_context_id();
  double* scratch = nullptr;
  {
    // Once per device (and context), with that device current: the host-side
    // name of the array is not a device address; ask the runtime for it.
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceSetup& su = g_setup[dev];
    if (!su.scratch || ctx == 0 || su.ctx_id != ctx) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_static_partials) != cudaSuccess || !ptr) {
        cudaGetLastError();
        return fail(GLS_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
      }
      if (cudaFuncSetAttribute(trsm_gram_fp64_static_kernel,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)sizeof(Smem)) != cudaSuccess) {
        cudaGetLastError();
        return fail(GLS_ERR_CUDA, "cudaFuncSetAttribute failed");
      }
      su.scratch = static_cast<double*>(ptr);
      su.ctx_id = current_context_id();
    }
    scratch = su.scratch;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  dim3 grid((unsigned)gls::ceil_div(k, TS), (unsigned)nI);
  trsm_gram_fp64_static_kernel<<<grid, 256, sizeof(Smem), st>>>(Zinv, ldz, n, nI, XR, ldxr, k, W,
                                                                ldw, p, scratch, k);
  gls::launch_assemble_solve(scratch, k, nI, p, 1, p, k, RTL, zT, gls::kTauFP64, B, ldb,
                             snp_status, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(GLS_ERR_CUDA, cudaGetErrorString(e));
  return GLS_OK;
}
