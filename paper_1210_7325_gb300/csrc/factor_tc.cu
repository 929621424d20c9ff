// factor_tc.cu -- the binary64 setup phase of Alg. 5 (line 1: L L^T = M; the
// triangular inverse Z = L^{-1} used by the blocked solve; lines 2 and 4: the
// whitened covariates and phenotype) with every dense product evaluated
// exactly on tcgen05 tensor cores.
//
// Why.  Binary64 FMA throughput on this part is about 1/1500 of its BF16
// tensor-core rate, so an O(n^3) binary64 factor costs more than the whole
// O(n^2 m) mixed-precision SNP loop.  The products below are therefore split
// into exact integer slices and multiplied on the tensor cores (the error-free
// splitting of Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59 (2012)), and
// only the small diagonal blocks run in binary64 arithmetic.
//
// Slices.  For one operand row x_k (k in its K range) let 2^E bound max |x_k|
// and X_k = round(x_k 2^(56-E)), an integer with |X_k| <= 2^56.  Its balanced
// base-256 digits give X_k = sum_{t=0..6} a_t 2^(48-8t) with |a_0| <= 256 and
// |a_t| <= 128, and the slices s_t = a_t 2^(-8t) are exact in BF16, so
//     x_k = 2^(E-8) sum_t s_t + d_k,   |d_k| <= 2^(E-57).
// A product of two operands is then
//     sum_k x_k y_k = 2^(E_x + E_y - 16) sum_k sum_{t,u} s_t s'_u  (+ truncation),
// keeping the 28 slice pairs with t + u <= 6.  Pairs of equal level t + u
// share one FP32 tensor-memory accumulator.  Over a chunk of at most 128
// values of k the level-L sums are integer multiples of 2^(-8L) whose integer
// part stays below 2^24 for L <= 3 (level 0: 128 * 2^16; level 1:
// 2 * 128 * 2^15; level 2: 128 * (2 * 2^15 + 2^14); level 3:
// 128 * (2 * 2^15 + 2 * 2^14)), so the tensor core adds them exactly.  Levels
// 4..6 share a fifth accumulator whose weight is at most 2^-32 of level 0, so
// its FP32 rounding stays near 2^-56 of the result.  The epilogue converts the
// four exact levels of every chunk to one int64 (exact across chunks), keeps
// the tail in FP32, and rounds once to binary64 at the end: the result carries
// the slice truncation (about 2^-54 of max|x| max|y| per product), which is
// below the rounding error of a binary64 dot product.
//
// Algorithm.  A recursive Cholesky with inverse on the column-major npad x npad
// arrays (block sizes multiples of 64):
//     [A11    ]      L11 Z11  = factor(A11)
//     [A21 A22]  ->  L21      = A21 Z11^T           (L21 = A21 L11^{-T})
//                    A22     -= L21 L21^T           (trailing update)
//                    L22 Z22  = factor(A22)
//                    Z21      = -Z22 (L21 Z11)      (block of L^{-1})
// with the 64 x 64 leaves factored and inverted in binary64 (factor_fp64.cu).
// Every product has a long inner dimension, so the binary64 epilogue runs once
// per output element of each product rather than once per 64-deep update.
//
// Tensor-core kernel.  One persistent CTA per SM, 320 threads:
//   warp 0     TMA producer: per 32-deep stage, the 7 slices of a 128-row A tile
//              and of a 64-row B tile (64-byte swizzle), one mbarrier per stage
//   warp 1     TMEM allocator and the thread issuing tcgen05.mma (M = 128,
//              N = 64, K = 16, BF16 in, FP32 accumulate): 28 pairs x 2 per stage
//              into five accumulators; each accumulator has its own full/empty
//              barrier pair, so the epilogue drains level L of one 128-deep
//              chunk while the tensor core works on the later levels and the
//              next chunk
//   warps 2-9  epilogue: two warps per TMEM lane quarter, 32 columns each;
//              per chunk tcgen05.ld of the five accumulators into the int64 and
//              FP32 sums, per tile the binary64 result written to C
// Every mbarrier wait is bounded (1 s of %globaltimer); a timeout sets an error
// flag, drains what is in flight, frees tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>

#include "common.cuh"
#include "factor_tc.cuh"
#include "sm100.cuh"

namespace gls {

using namespace sm100;

namespace {

constexpr int kS = 7;                  // slices per binary64 operand
constexpr int OBM = 128;               // output rows per tile (TMEM lanes)
constexpr int OBN = 64;                // output columns per tile
constexpr int OBK = 32;                // K per stage: 32 x 16-bit = one 64-byte swizzle row
constexpr int kChunkStages = 4;        // exact chunks of 128
constexpr int kStages = 2;
constexpr int kAcc = 5;                // levels 0, 1, 2, 3 (exact) and the tail 4..6
constexpr uint32_t kTmemCols = 512;    // 5 accumulators x 64 columns (power-of-two allocation)
constexpr int kEpiWarps = 8;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kABytes = kS * OBM * OBK * 2;     // 57344
constexpr int kBBytes = kS * OBN * OBK * 2;     // 28672
constexpr int kStageBytes = kABytes + kBBytes;  // 86016 = 84 KiB
constexpr int kSmemBytes = kStages * kStageBytes + 1024 + 256;
constexpr uint64_t kWaitLimitNs = 1000000000ull;
constexpr uint64_t kDrainLimitNs = 100000000ull;
constexpr int kExpNonFinite = 4096;    // row exponent marking a row with Inf/NaN

enum KMode : int { kKFull = 0, kKLeJ = 1, kKGeJ = 2, kKLeI = 3, kKGeI = 4 };

thread_local std::string g_err;

struct OzParams {
  double* C;
  int64_t ldc;
  const int* eA;     // row exponents of the A operand
  const int* eB;     // row exponents of the B operand
  int64_t diag_off;  // lower: store only where row + diag_off >= col
  double alpha;
  int M, N, tilesI, tilesJ;
  int Kend, kmode, koff;
  int beta, lower;
  int* flags;        // plan status words: kFlagPotrf read, kFlagKernel / kFlagWhere written
};

__device__ __forceinline__ uint64_t umma_desc_sw64(uint32_t smem_addr) {
  uint64_t d = 0;
  d |= (uint64_t)((smem_addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;   // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512u >> 4) << 32;  // stride byte offset: 8 rows x 64 bytes
  d |= (uint64_t)1 << 46;            // descriptor version
  d |= (uint64_t)4 << 61;            // 64-byte swizzle
  return d;
}

__device__ __forceinline__ double pow2i(int e) {
  if (e >= -1022 && e <= 1023) return __longlong_as_double((long long)(e + 1023) << 52);
  return ldexp(1.0, e);
}

struct TileWork {
  int I, J, k0, k1;
  bool valid;
};

__device__ __forceinline__ TileWork tile_work(const OzParams& q, int t) {
  TileWork w;
  w.I = t / q.tilesJ;
  w.J = t - w.I * q.tilesJ;
  w.valid = !q.lower || ((int64_t)w.I * OBM + OBM - 1 + q.diag_off >= (int64_t)w.J * OBN);
  int k0 = 0, k1 = q.Kend;
  switch (q.kmode) {
    case kKLeJ: k1 = min(k1, (w.J + 1) * OBN + q.koff); break;
    case kKGeJ: k0 = w.J * OBN + q.koff; break;
    case kKLeI: k1 = min(k1, (w.I + 1) * OBM + q.koff); break;
    case kKGeI: k0 = w.I * OBM + q.koff; break;
    default: break;
  }
  k0 = max(k0, 0);
  if (k1 < k0) k1 = k0;
  w.k0 = k0;
  w.k1 = k1;
  return w;
}

__device__ void raise_error(int* eflags, int site) {
  atomicOr(&eflags[kFlagKernel], kErrTimeout);
  atomicExch(&eflags[kFlagWhere], 100 + site);
}

__device__ __forceinline__ bool epilogue_all(bool ok) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, 1, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)ok), "r"(32 * kEpiWarps)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ bool wait_drain(uint64_t* bar, uint32_t parity) {
  volatile int never = 0;
  return mbar_wait_bounded(bar, parity, &never, kDrainLimitNs);
}

__device__ __forceinline__ float f32(uint32_t v) { return __uint_as_float(v); }

__global__ void __launch_bounds__(kThreads, 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ OzParams q) {
  if (*(volatile const int*)&q.flags[kFlagPotrf] != 0) return;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + kStages * kStageBytes);
  uint64_t* empty = full + kStages;
  uint64_t* afull = empty + kStages;   // per accumulator: chunk's products complete
  uint64_t* aempty = afull + kAcc;     // per accumulator: drained by the epilogue
  uint64_t* drain = aempty + kAcc;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < kAcc; ++a) {
      mbar_init(&afull[a], 1);
      mbar_init(&aempty[a], kEpiWarps);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int ntiles = q.tilesI * q.tilesJ;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      tma_prefetch_desc(&tmA);
      tma_prefetch_desc(&tmB);
      uint32_t g = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const TileWork w = tile_work(q, t);
        if (!w.valid) continue;
        for (int k = w.k0; k < w.k1; k += OBK, ++g) {
          const int st = (int)(g % kStages);
          const uint32_t ph = g / kStages;
          if (!mbar_wait_bounded(&empty[st], (ph & 1) ^ 1, abort_flag, kWaitLimitNs)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&full[st], (uint32_t)kStageBytes);
          uint8_t* sb = base + (size_t)st * kStageBytes;
          tma_load_3d(sb, &tmA, &full[st], k, w.I * OBM, 0);
          tma_load_3d(sb + kABytes, &tmB, &full[st], k, w.J * OBN, 0);
        }
      }
      if (!ok) {
        raise_error(q.flags, 1);
        const uint32_t first = g > (uint32_t)kStages ? g - kStages : 0;
        for (uint32_t g2 = first; g2 < g; ++g2)
          wait_drain(&full[g2 % kStages], (g2 / kStages) & 1);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = umma_idesc_f16(OBM, OBN, true);
      uint32_t g = 0, cg = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const TileWork w = tile_work(q, t);
        if (!w.valid) continue;
        const int nk = (w.k1 - w.k0) / OBK;
        for (int s0 = 0; s0 < nk && ok; s0 += kChunkStages, ++cg) {
          const uint32_t par = cg & 1;
          const int ns = min(kChunkStages, nk - s0);
          for (int s = 0; s < ns && ok; ++s, ++g) {
            const int st = (int)(g % kStages);
            const uint32_t ph = g / kStages;
            if (!mbar_wait_bounded(&full[st], ph & 1, abort_flag, kWaitLimitNs)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(base + (size_t)st * kStageBytes);
            const uint32_t sbb = sa + kABytes;
#pragma unroll
            for (int kk = 0; kk < OBK / 16; ++kk) {
              const bool chunk_first = (s == 0) && (kk == 0);
              const bool chunk_last = (s == ns - 1) && (kk == OBK / 16 - 1);
#pragma unroll
              for (int lam = 0; lam < kS; ++lam) {
                const int acc = lam < kAcc - 1 ? lam : kAcc - 1;
                if (chunk_first && lam < kAcc) {
                  // the previous chunk's value of this accumulator has been read
                  if (!mbar_wait_bounded(&aempty[acc], par ^ 1, abort_flag, kWaitLimitNs)) {
                    ok = false;
                    break;
                  }
                  tc_fence_after();
                }
#pragma unroll
                for (int ta = 0; ta <= lam; ++ta) {
                  const int tb = lam - ta;
                  const bool fresh = chunk_first && ta == 0 && lam < kAcc;
                  umma_f16(tmem + (uint32_t)acc * OBN,
                           umma_desc_sw64(sa + ta * (OBM * OBK * 2) + kk * 32),
                           umma_desc_sw64(sbb + tb * (OBN * OBK * 2) + kk * 32), idesc,
                           fresh ? 0u : 1u);
                }
                if (chunk_last && (lam < kAcc - 1 || lam == kS - 1)) umma_commit(&afull[acc]);
              }
              if (!ok) break;
            }
            umma_commit(&empty[st]);
          }
        }
      }
      if (!ok) raise_error(q.flags, 2);
      umma_commit(drain);
      wait_drain(drain, 0);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;
    const int rl = quarter * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)half * 32;
    uint32_t cg = 0;
    bool alive = true;
    for (int t = blockIdx.x; t < ntiles && alive; t += gridDim.x) {
      const TileWork w = tile_work(q, t);
      if (!w.valid) continue;
      const int nk = (w.k1 - w.k0) / OBK;
      long long V[32];
      float tl[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        V[j] = 0;
        tl[j] = 0.f;
      }
      for (int s0 = 0; s0 < nk && alive; s0 += kChunkStages, ++cg) {
        const uint32_t par = cg & 1;
#pragma unroll
        for (int a = 0; a < kAcc; ++a) {
          const bool got = mbar_wait_bounded(&afull[a], par, abort_flag, kWaitLimitNs);
          if (!epilogue_all(got)) {
            if (!got && lane == 0) raise_error(q.flags, 3);
            alive = false;
            break;
          }
          tc_fence_after();
          uint32_t r[32];
          tmem_ld32(lane_base + (uint32_t)a * OBN, r);
          tmem_ld_wait(r);
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&aempty[a]);
          if (a < kAcc - 1) {
            // level a: an integer multiple of 2^(-8a); V counts units of 2^-24
            const float up = (float)(1u << (8 * a));
            const long long w = 1ll << (24 - 8 * a);
#pragma unroll
            for (int j = 0; j < 32; ++j) V[j] += (long long)__float2int_rn(f32(r[j]) * up) * w;
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) tl[j] += f32(r[j]);
          }
        }
      }
      if (!alive) break;
      const int64_t row = (int64_t)w.I * OBM + rl;
      if (row < q.M) {
        const int ea = q.eA[row];
        const int64_t col0 = (int64_t)w.J * OBN + half * 32;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int64_t col = col0 + j;
          if (col < q.N && (!q.lower || row + q.diag_off >= col)) {
            const int eb = q.eB[col];
            double d;
            if (ea == kExpNonFinite || eb == kExpNonFinite) {
              d = __longlong_as_double(0x7ff8000000000000ll);
            } else {
              const int e = ea + eb - 16;
              d = fma((double)V[j], pow2i(e - 24), (double)tl[j] * pow2i(e));
            }
            double* cp = q.C + row + col * q.ldc;
            *cp = q.beta ? fma(q.alpha, d, *cp) : q.alpha * d;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------- slicing
// Exponent E with max |x| < 2^E (frexp convention); 0 for an all-zero row.
__device__ __forceinline__ int row_exponent(double m, bool nonfinite) {
  if (nonfinite) return kExpNonFinite;
  if (!(m > 0.0)) return 0;
  const int ex = (int)((__double_as_longlong(m) >> 52) & 0x7FF);
  return ex == 0 ? -1022 : ex - 1022;
}

// The kS slices of x relative to 2^E (see the file header), as BF16 bits.
__device__ __forceinline__ void slice_value(double x, int E, uint16_t (&s)[kS]) {
  const long long bits = __double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7FF);
  long long X = 0;
  if (ex != 0 && ex != 0x7FF && E != kExpNonFinite) {
    const long long mant = (bits & 0xFFFFFFFFFFFFFll) | (1ll << 52);
    const int sh = ex - 1019 - E;  // X = mant * 2^sh, sh <= 3 because |x| < 2^E
    long long m;
    if (sh >= 0) m = mant << min(sh, 3);
    else if (sh > -63) m = (mant + (1ll << (-sh - 1))) >> (-sh);
    else m = 0;
    X = bits < 0 ? -m : m;
  }
  long long r = X;
#pragma unroll
  for (int t = 0; t < kS - 1; ++t) {
    const int sh = 48 - 8 * t;
    const long long a = (r + (1ll << (sh - 1))) >> sh;
    r -= a * (1ll << sh);
    s[t] = __bfloat16_as_ushort(__float2bfloat16_rn(ldexpf((float)a, -8 * t)));
  }
  s[kS - 1] = __bfloat16_as_ushort(__float2bfloat16_rn(ldexpf((float)r, -8 * (kS - 1))));
}

// Operand row i = source row i, k = source column k: x(i, k) = src[i + k ld],
// i < R, k < K; out[t][i][k] with row length kld (zeros for K <= k < kld).
// One CTA per 32 rows; lanes walk rows (coalesced reads), warps walk k, and
// the K-major slices are written through a shared-memory transpose.
__global__ void __launch_bounds__(256) slice_rows_kernel(const double* __restrict__ src,
                                                         int64_t ld, int64_t R, int64_t K,
                                                         int64_t kld, uint16_t* __restrict__ out,
                                                         int* __restrict__ expo,
                                                         const int* flags) {
  if (*(volatile const int*)&flags[kFlagPotrf] != 0) return;
  __shared__ double red[8][33];
  __shared__ int bad[8][33];
  __shared__ int Es[32];
  __shared__ __align__(16) uint16_t sh[kS][32][OBK + 8];
  const int l = threadIdx.x % 32, w = threadIdx.x / 32;
  const int64_t i = (int64_t)blockIdx.x * 32 + l;
  const bool iv = i < R;
  double m = 0.0;
  int nf = 0;
  if (iv)
    for (int64_t k = w; k < K; k += 8) {
      const double v = src[i + k * ld];
      nf |= !isfinite(v);
      m = fmax(m, fabs(v));
    }
  red[w][l] = m;
  bad[w][l] = nf;
  __syncthreads();
  if (w == 0) {
    for (int v = 1; v < 8; ++v) {
      m = fmax(m, red[v][l]);
      nf |= bad[v][l];
    }
    const int E = row_exponent(m, nf != 0);
    Es[l] = E;
    if (iv) expo[i] = E;
  }
  __syncthreads();
  const int E = Es[l];
  const size_t plane = (size_t)R * kld;
  for (int64_t k0 = 0; k0 < kld; k0 += OBK) {
#pragma unroll
    for (int e = 0; e < OBK / 8; ++e) {
      const int kk = w + 8 * e;
      const int64_t k = k0 + kk;
      uint16_t s[kS];
      slice_value((iv && k < K) ? src[i + k * ld] : 0.0, E, s);
#pragma unroll
      for (int t = 0; t < kS; ++t) sh[t][l][kk] = s[t];
    }
    __syncthreads();
    // kS slices x 32 rows x 4 uint4 (64 bytes per row)
    for (int idx = threadIdx.x; idx < kS * 32 * 4; idx += 256) {
      const int t = idx / 128, rr = (idx / 4) % 32, c4 = idx % 4;
      const int64_t ii = (int64_t)blockIdx.x * 32 + rr;
      if (ii < R) {
        const uint4 v = *reinterpret_cast<const uint4*>(&sh[t][rr][c4 * 8]);
        *reinterpret_cast<uint4*>(out + t * plane + ii * kld + k0 + c4 * 8) = v;
      }
    }
    __syncthreads();
  }
}

// Operand row i = source column i, k = source row k: x(i, k) = src[k + i ld].
// One warp per operand row.
__global__ void __launch_bounds__(256) slice_cols_kernel(const double* __restrict__ src,
                                                         int64_t ld, int64_t R, int64_t K,
                                                         int64_t kld, uint16_t* __restrict__ out,
                                                         int* __restrict__ expo,
                                                         const int* flags) {
  if (*(volatile const int*)&flags[kFlagPotrf] != 0) return;
  const int l = threadIdx.x % 32, w = threadIdx.x / 32;
  const int64_t i = (int64_t)blockIdx.x * 8 + w;
  if (i >= R) return;
  const double* col = src + i * ld;
  double m = 0.0;
  int nf = 0;
  for (int64_t k = l; k < K; k += 32) {
    const double v = col[k];
    nf |= !isfinite(v);
    m = fmax(m, fabs(v));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    nf |= __shfl_xor_sync(0xffffffffu, nf, o);
  }
  const int E = row_exponent(m, nf != 0);
  if (l == 0) expo[i] = E;
  const size_t plane = (size_t)R * kld;
  for (int64_t k = l; k < kld; k += 32) {
    uint16_t s[kS];
    slice_value(k < K ? col[k] : 0.0, E, s);
#pragma unroll
    for (int t = 0; t < kS; ++t) out[t * plane + i * kld + k] = s[t];
  }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() {
    cudaDriverEntryPointQueryResult qr;
    void* ptr = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &qr) != cudaSuccess ||
        qr != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return static_cast<PFN_cuTensorMapEncodeTiled_v12000>(nullptr);
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  }();
  return fn;
}

}  // namespace

// ------------------------------------------------------------------ workspace
struct TcFactor {
  int64_t npad = 0, half = 0;
  size_t cap = 0;             // elements per slice plane of SA / SB
  uint16_t* SA = nullptr;     // kS x cap
  uint16_t* SB = nullptr;     // kS x cap
  int* eA = nullptr;          // npad
  int* eB = nullptr;          // npad
  double* T = nullptr;        // half x half
  int num_sms = 1;
};

namespace {

int64_t half_of(int64_t npad) { return 64 * ceil_div(npad / 64, 2); }

// Elements per slice plane: the largest operand of the recursion (half x half)
// and at least one 128-row panel of the whitening products (128 x npad).
size_t plane_cap(int64_t npad) {
  const int64_t h = half_of(npad);
  return std::max((size_t)h * (size_t)round_up(h, OBK), (size_t)OBM * (size_t)npad);
}

bool g_smem_attr = false;

struct Operand {
  const uint16_t* slices;
  const int* expo;
  int64_t rows, kld;
};

cudaError_t enc_err(const char* what) {
  g_err = std::string("tensor map encode failed: ") + what;
  return cudaErrorInvalidValue;
}

cudaError_t encode(CUtensorMap* map, const Operand& o, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
  if (!enc) return enc_err("cuTensorMapEncodeTiled unavailable");
  cuuint64_t dims[3] = {(cuuint64_t)o.kld, (cuuint64_t)o.rows, (cuuint64_t)kS};
  cuuint64_t strides[2] = {(cuuint64_t)o.kld * 2, (cuuint64_t)o.rows * o.kld * 2};
  cuuint32_t box[3] = {OBK, (cuuint32_t)box_rows, kS};
  cuuint32_t es[3] = {1, 1, 1};
  if (enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<uint16_t*>(o.slices), dims,
          strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return enc_err("slices");
  return cudaSuccess;
}

// x(i, k) = src[i + k ld] (rows = true) or src[k + i ld] (rows = false).
cudaError_t slice(const double* src, int64_t ld, int64_t R, int64_t K, bool rows, uint16_t* out,
                  int* expo, const int* flags, cudaStream_t st) {
  const int64_t kld = round_up(K, OBK);
  if (rows)
    slice_rows_kernel<<<(unsigned)ceil_div(R, 32), 256, 0, st>>>(src, ld, R, K, kld, out, expo,
                                                                 flags);
  else
    slice_cols_kernel<<<(unsigned)ceil_div(R, 8), 256, 0, st>>>(src, ld, R, K, kld, out, expo,
                                                                flags);
  return cudaGetLastError();
}

// C (M x N, ldc) = alpha * A B^T + beta * C, A = M x K and B = N x K operands
// already sliced; kmode restricts each tile's K range to the structural nonzeros.
cudaError_t gemm(TcFactor* w, const Operand& A, const Operand& B, double* C, int64_t ldc, int M,
                 int N, int K, int kmode, int koff, double alpha, int beta, bool lower,
                 int64_t diag_off, int* flags, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (!g_smem_attr) {
    cudaError_t e = cudaFuncSetAttribute(oz_gemm_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    g_smem_attr = true;
  }
  CUtensorMap ta, tb;
  cudaError_t e;
  if ((e = encode(&ta, A, OBM)) != cudaSuccess) return e;
  if ((e = encode(&tb, B, OBN)) != cudaSuccess) return e;
  OzParams q;
  memset(&q, 0, sizeof(q));
  q.C = C;
  q.ldc = ldc;
  q.eA = A.expo;
  q.eB = B.expo;
  q.diag_off = diag_off;
  q.alpha = alpha;
  q.M = M;
  q.N = N;
  q.tilesI = (int)ceil_div(M, OBM);
  q.tilesJ = (int)ceil_div(N, OBN);
  q.Kend = K;
  q.kmode = kmode;
  q.koff = koff;
  q.beta = beta;
  q.lower = lower ? 1 : 0;
  q.flags = flags;
  const int tiles = q.tilesI * q.tilesJ;
  const int grid = std::max(1, std::min(w->num_sms, tiles));
  oz_gemm_kernel<<<grid, kThreads, kSmemBytes, st>>>(ta, tb, q);
  return cudaGetLastError();
}

#define TC_TRY(expr)                     \
  do {                                   \
    cudaError_t e_ = (expr);             \
    if (e_ != cudaSuccess) return e_;    \
  } while (0)

cudaError_t rec(TcFactor* w, double* A, double* Z, int64_t ld, int64_t r0, int64_t n, int* flags,
                cudaStream_t st) {
  if (n == 64) {
    launch_potrf_diag64(A, Z, ld, r0, flags, st);
    return cudaGetLastError();
  }
  const int64_t n1 = 64 * ((n / 64) / 2), n2 = n - n1;
  TC_TRY(rec(w, A, Z, ld, r0, n1, flags, st));
  double* A21 = A + (r0 + n1) + r0 * ld;
  double* A22 = A + (r0 + n1) + (r0 + n1) * ld;
  double* Z11 = Z + r0 + r0 * ld;
  double* Z21 = Z + (r0 + n1) + r0 * ld;
  double* Z22 = Z + (r0 + n1) + (r0 + n1) * ld;
  const Operand SA1{w->SA, w->eA, n2, round_up(n1, OBK)};
  const Operand SB1{w->SB, w->eB, n1, round_up(n1, OBK)};
  // L21 = A21 Z11^T (Z11 lower: column block J needs k < (J+1) 64)
  TC_TRY(slice(A21, ld, n2, n1, true, w->SA, w->eA, flags, st));
  TC_TRY(slice(Z11, ld, n1, n1, true, w->SB, w->eB, flags, st));
  TC_TRY(gemm(w, SA1, SB1, A21, ld, (int)n2, (int)n1, (int)n1, kKLeJ, 0, 1.0, 0, false, 0, flags,
              st));
  // A22 -= L21 L21^T (lower triangle)
  TC_TRY(slice(A21, ld, n2, n1, true, w->SA, w->eA, flags, st));
  const Operand SA1b{w->SA, w->eA, n2, round_up(n1, OBK)};
  TC_TRY(gemm(w, SA1, SA1b, A22, ld, (int)n2, (int)n2, (int)n1, kKFull, 0, -1.0, 1, true, 0,
              flags, st));
  TC_TRY(rec(w, A, Z, ld, r0 + n1, n2, flags, st));
  // T = L21 Z11 (Z11 lower: column j needs k >= j)
  TC_TRY(slice(A21, ld, n2, n1, true, w->SA, w->eA, flags, st));
  TC_TRY(slice(Z11, ld, n1, n1, false, w->SB, w->eB, flags, st));
  TC_TRY(gemm(w, SA1, SB1, w->T, n2, (int)n2, (int)n1, (int)n1, kKGeJ, 0, 1.0, 0, false, 0, flags,
              st));
  // Z21 = -Z22 T (Z22 lower: row block I needs k < (I+1) 128)
  const Operand SA2{w->SA, w->eA, n2, round_up(n2, OBK)};
  const Operand SB2{w->SB, w->eB, n1, round_up(n2, OBK)};
  TC_TRY(slice(Z22, ld, n2, n2, true, w->SA, w->eA, flags, st));
  TC_TRY(slice(w->T, n2, n1, n2, false, w->SB, w->eB, flags, st));
  TC_TRY(gemm(w, SA2, SB2, Z21, ld, (int)n2, (int)n1, (int)n2, kKLeI, 0, -1.0, 0, false, 0, flags,
              st));
  return cudaSuccess;
}

int64_t rec_launches(int64_t n) {
  if (n == 64) return 1;
  const int64_t n1 = 64 * ((n / 64) / 2), n2 = n - n1;
  return rec_launches(n1) + rec_launches(n2) + 11;
}

// Rows per panel so that rows x K fits one slice plane.
int64_t panel_rows(const TcFactor* w, int64_t K) {
  int64_t P = (int64_t)(w->cap / (size_t)round_up(K, OBK));
  P = (P / OBM) * OBM;
  return std::max<int64_t>(P, OBM);
}

}  // namespace

size_t tc_factor_bytes(int64_t npad) {
  const int64_t h = half_of(npad);
  return 2 * (size_t)kS * plane_cap(npad) * 2 + 2 * (size_t)npad * 4 + (size_t)h * h * 8;
}

const char* tc_factor_last_error() { return g_err.c_str(); }

void tc_factor_free(TcFactor* w) {
  if (!w) return;
  cudaFree(w->SA);
  cudaFree(w->SB);
  cudaFree(w->eA);
  cudaFree(w->eB);
  cudaFree(w->T);
  delete w;
}

gls_status_t tc_factor_create(TcFactor** out, int64_t npad) {
  *out = nullptr;
  if (npad % 128 != 0) {
    g_err = "npad must be a multiple of 128";
    return GLS_ERR_INVALID_ARG;
  }
  TcFactor* w = new TcFactor();
  w->npad = npad;
  w->half = half_of(npad);
  w->cap = plane_cap(npad);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&w->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaMalloc(&w->SA, (size_t)kS * w->cap * 2) != cudaSuccess ||
      cudaMalloc(&w->SB, (size_t)kS * w->cap * 2) != cudaSuccess ||
      cudaMalloc(&w->eA, (size_t)npad * 4) != cudaSuccess ||
      cudaMalloc(&w->eB, (size_t)npad * 4) != cudaSuccess ||
      cudaMalloc(&w->T, (size_t)w->half * w->half * 8) != cudaSuccess) {
    cudaGetLastError();
    tc_factor_free(w);
    g_err = "cudaMalloc of the tensor-core factor workspace failed";
    return GLS_ERR_OOM;
  }
  *out = w;
  return GLS_OK;
}

int64_t tc_potrf_trtri_launches(int64_t npad) { return rec_launches(npad); }

cudaError_t tc_potrf_trtri(TcFactor* w, double* A, double* Z, int64_t ld, int64_t npad, int* flags,
                           cudaStream_t st) {
  if (npad != w->npad) {
    g_err = "workspace size does not match npad";
    return cudaErrorInvalidValue;
  }
  TC_TRY(rec(w, A, Z, ld, 0, npad, flags, st));
  return cudaSuccess;
}

cudaError_t tc_lower_times(TcFactor* w, const double* Z, int64_t ldz, int64_t npad,
                           const double* rhs, int64_t ldr, int ncols, double* out, int64_t ldo,
                           int* flags, cudaStream_t st) {
  // out[i0 + i] = sum_{k <= i0 + i} Z[i0 + i][k] rhs[k], by row panels of Z
  const int64_t P = panel_rows(w, npad);
  for (int64_t i0 = 0; i0 < npad; i0 += P) {
    const int64_t rows = std::min(P, npad - i0), K = i0 + rows;
    TC_TRY(slice(Z + i0, ldz, rows, K, true, w->SA, w->eA, flags, st));
    TC_TRY(slice(rhs, ldr, ncols, K, false, w->SB, w->eB, flags, st));
    const Operand a{w->SA, w->eA, rows, round_up(K, OBK)};
    const Operand b{w->SB, w->eB, ncols, round_up(K, OBK)};
    TC_TRY(gemm(w, a, b, out + i0, ldo, (int)rows, ncols, (int)K, kKLeI, (int)i0, 1.0, 0, false,
                0, flags, st));
  }
  return cudaSuccess;
}

cudaError_t tc_lower_t_times(TcFactor* w, const double* Z, int64_t ldz, int64_t npad,
                             const double* rhs, int64_t ldr, int ncols, double* out, int64_t ldo,
                             int* flags, cudaStream_t st) {
  // out[c0 + i] = sum_{r >= c0 + i} Z[r][c0 + i] rhs[r], by column panels of Z
  const int64_t P = panel_rows(w, npad);
  for (int64_t c0 = 0; c0 < npad; c0 += P) {
    const int64_t rows = std::min(P, npad - c0), K = npad - c0;
    TC_TRY(slice(Z + c0 + c0 * ldz, ldz, rows, K, false, w->SA, w->eA, flags, st));
    TC_TRY(slice(rhs + c0, ldr, ncols, K, false, w->SB, w->eB, flags, st));
    const Operand a{w->SA, w->eA, rows, round_up(K, OBK)};
    const Operand b{w->SB, w->eB, ncols, round_up(K, OBK)};
    TC_TRY(gemm(w, a, b, out + c0, ldo, (int)rows, ncols, (int)K, kKGeI, 0, 1.0, 0, false, 0,
                flags, st));
  }
  return cudaSuccess;
}

}  // namespace gls
