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
// keeping the 28 slice pairs with t + u <= 6.  Each level t + u has its own
// FP32 tensor-memory accumulator (7 x BN columns).  Over a chunk of at most 128
// values of k the level-L sums are integer multiples of 2^(-8L) whose integer
// part stays below 2^24 for L <= 3 (level 0: 128 * 2^16; level 1:
// 2 * 128 * 2^15; level 2: 128 * (2 * 2^15 + 2^14); level 3:
// 128 * (2 * 2^15 + 2 * 2^14)), so the tensor core adds them exactly.  Levels
// 4..6 weigh at most 2^-32 of level 0, so FP32 rounding of their sums stays
// near 2^-56 of the result.  The epilogue converts the four exact levels of
// every chunk to one int64 (exact across chunks), adds the tail levels in
// FP32, and rounds once to binary64 at the end: the result carries
// the slice truncation (about 2^-54 of max|x| max|y| per product), which is
// below the rounding error of a binary64 dot product.
//
// Algorithm.  A recursive Cholesky with inverse on the column-major npad x npad
// arrays (block sizes multiples of 64):
//     [A11    ]      L11 Z11  = factor(A11)
//     [A21 A22]  ->  L21      = A21 Z11^T           (L21 = A21 L11^{-T})
//                    A22     -= L21 L21^T           (trailing update)
//                    T        = L21 Z11             (kept in the Z21 block)
//                    L22 Z22  = factor(A22)
//                    Z21      = -Z22 T              (block of L^{-1})
// with the 64 x 64 leaves factored and inverted in binary64 (factor_fp64.cu).
// Every product has a long inner dimension, so the binary64 epilogue runs once
// per output element of each product rather than once per 64-deep update.
//
// Tensor-core kernel.  One persistent CTA per SM, 320 threads, output tiles of
// 128 x BN (BN = 64; BN = 16 for products with few tiles, so that more SMs
// share their binary64 epilogue):
//   warp 0     TMA producer: per 16-deep stage, the 7 slices of a 128-row A tile
//              and of a BN-row B tile (32-byte swizzle), 5-6 stages in flight
//   warp 1     TMEM allocator and the thread issuing tcgen05.mma (M = 128,
//              K = 16, BF16 in, FP32 accumulate), the 28 pairs of a stage in
//              one of two orders.  The first stage of a 128-deep chunk goes
//              level by level (N = BN, 28 MMAs), each level waiting only for
//              the epilogue's drain of its own accumulator.  The other stages
//              multiply A slice t by B slices 0..6-t at once: those B slices
//              lie back to back in shared memory and the accumulators of
//              levels t..6 back to back in tensor memory, so one MMA of
//              N = c BN covers c pairs (c <= 256 / BN: 10 MMAs per stage for
//              BN = 64, 7 for BN = 16).  Each accumulator has its own
//              full/empty barrier pair, so the epilogue drains level L of a
//              chunk while the tensor core works on the later levels and the
//              next chunk
//   warps 2-9  epilogue: two warps per TMEM lane quarter, BN/2 columns each;
//              per chunk tcgen05.ld of the seven accumulators into the int64 and
//              FP32 sums, per tile the binary64 result written to C (three
//              binary64 operations per element; the power-of-two scale is an
//              exponent-field add)
// The slices are formed by one launch per product (both operands): row
// maxima, then integer digit extraction, 8 consecutive k per 16-byte store.
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
constexpr int OBK = 16;                // K per stage: 16 x 16-bit = one 32-byte swizzle row
constexpr int kChunkStages = 8;        // exact chunks of 128
constexpr int kKAlign = 32;            // operand rows are stored padded to a multiple of 32
constexpr int kAcc = kS;               // one accumulator per level t + u = 0..6
constexpr int kExact = 4;              // levels 0..3 are summed exactly
constexpr int kEpiWarps = 8;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr uint64_t kWaitLimitNs = 1000000000ull;
constexpr uint64_t kDrainLimitNs = 100000000ull;
constexpr int kExpNonFinite = 4096;    // row exponent marking a row with Inf/NaN

// Tile shapes: BN = 64 output columns for large products, BN = 16 for small
// ones (more CTAs share the binary64 epilogue of a few output tiles).
template <int BN>
struct Shape {
  static constexpr int kABytes = kS * OBM * OBK * 2;       // 28672
  static constexpr int kBBytes = kS * BN * OBK * 2;        // 14336 or 3584
  static constexpr int kStageBytes = kABytes + kBBytes;    // multiples of 512
  static constexpr int kStages = BN == 64 ? 5 : 6;
  static constexpr int kSmemBytes = kStages * kStageBytes + 1024 + 256;
  static constexpr uint32_t kTmemCols = BN == 64 ? 512 : 128;  // 7 accumulators x BN
  static constexpr int kCols = BN / 2;                     // columns per epilogue warp
  static constexpr int kASlice = OBM * OBK * 2;            // bytes of one A slice per stage
  static constexpr int kBSlice = BN * OBK * 2;             // bytes of one B slice per stage
  static constexpr int kPerMma = 256 / BN;                 // B slices one MMA can take (N <= 256)
  static_assert(kAcc * BN <= (int)kTmemCols, "accumulators exceed the tensor-memory allocation");
};

enum KMode : int { kKFull = 0, kKLeJ = 1, kKGeJ = 2, kKLeI = 3, kKGeI = 4 };

thread_local std::string g_err;

struct OzParams {
  double* C;
  int64_t ldc;
  const int* eA;     // row exponents of the A operand
  const int* eB;     // row exponents of the B operand
  int64_t diag_off;  // lower: store only where row + diag_off >= col
  int M, N, tilesI, tilesJ;
  int ntiles;        // tiles of the launch: tilesI x tilesJ, or the lower ones only
  int Kend, kmode, koff;
  int neg, beta, lower;  // C = (neg ? -1 : 1) A B^T + (beta ? C : 0)
  int* flags;        // plan status words: kFlagPotrf read, kFlagKernel / kFlagWhere written
};

__device__ __forceinline__ double pow2i(int e) {
  if (e >= -1022 && e <= 1023) return __longlong_as_double((long long)(e + 1023) << 52);
  return ldexp(1.0, e);
}

// d * 2^e: an exponent-field add while the result stays a normal number.
__device__ __forceinline__ double scale2(double d, int e) {
  const long long b = __double_as_longlong(d);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex != 0 && ex != 0x7FF && ex + e >= 1 && ex + e <= 2046)
    return __longlong_as_double(b + ((long long)e << 52));
  return d * pow2i(e);
}

struct TileWork {
  int I, J, k0, k1;
  bool valid;
};

// Valid tiles of block row I of a lower-triangular output: J = 0 .. count - 1.
template <int BN>
__device__ __forceinline__ int lower_count(const OzParams& q, int I) {
  const int64_t c = ((int64_t)I * OBM + OBM - 1 + q.diag_off) / BN + 1;
  return (int)(c < 0 ? 0 : (c > q.tilesJ ? q.tilesJ : c));
}

// Tile t of the launch, heaviest first: the persistent CTAs take tiles t,
// t + grid, ... so that the longest K ranges are spread over all of them
// first (a triangular operand's K range grows or shrinks with I or J), and a
// lower-triangular output lists only its valid tiles.
template <int BN>
__device__ __forceinline__ TileWork tile_work(const OzParams& q, int t) {
  TileWork w;
  w.valid = t < q.ntiles;
  switch (q.kmode) {
    case kKLeJ: w.J = q.tilesJ - 1 - t / q.tilesI; w.I = t % q.tilesI; break;
    case kKGeJ: w.J = t / q.tilesI; w.I = t % q.tilesI; break;
    case kKLeI: w.I = q.tilesI - 1 - t / q.tilesJ; w.J = t % q.tilesJ; break;
    case kKGeI: w.I = t / q.tilesJ; w.J = t % q.tilesJ; break;
    default:
      if (q.lower) {
        int I = 0, r = t;
        while (I < q.tilesI - 1 && r >= lower_count<BN>(q, I)) r -= lower_count<BN>(q, I++);
        w.I = I;
        w.J = r;
      } else {
        w.I = t / q.tilesJ;
        w.J = t % q.tilesJ;
      }
      break;
  }
  w.valid = w.valid && w.I >= 0 && w.I < q.tilesI && w.J >= 0 && w.J < q.tilesJ &&
            (!q.lower || ((int64_t)w.I * OBM + OBM - 1 + q.diag_off >= (int64_t)w.J * BN));
  int k0 = 0, k1 = q.Kend;
  switch (q.kmode) {
    case kKLeJ: k1 = min(k1, (w.J + 1) * BN + q.koff); break;
    case kKGeJ: k0 = w.J * BN + q.koff; break;
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

// One accumulator's columns of this warp (32 or 8), waited for.
__device__ __forceinline__ void ld_cols(uint32_t taddr, uint32_t (&r)[32]) {
  tmem_ld32(taddr, r);
  tmem_ld_wait(r);
}
__device__ __forceinline__ void ld_cols(uint32_t taddr, uint32_t (&r)[8]) {
  tmem_ld8(taddr, r);
  tmem_ld_wait8(r);
}

template <int BN>
__global__ void __launch_bounds__(kThreads, 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ OzParams q) {
  using Sh = Shape<BN>;
  constexpr int CW = Sh::kCols;
  if (*(volatile const int*)&q.flags[kFlagPotrf] != 0) return;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + Sh::kStages * Sh::kStageBytes);
  uint64_t* empty = full + Sh::kStages;
  uint64_t* afull = empty + Sh::kStages;  // per accumulator: chunk's products complete
  uint64_t* aempty = afull + kAcc;        // per accumulator: drained by the epilogue
  uint64_t* drain = aempty + kAcc;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int s = 0; s < Sh::kStages; ++s) {
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
    tmem_alloc(tmem_slot, Sh::kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int ntiles = q.ntiles;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      tma_prefetch_desc(&tmA);
      tma_prefetch_desc(&tmB);
      uint32_t g = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const TileWork w = tile_work<BN>(q, t);
        if (!w.valid) continue;
        for (int k = w.k0; k < w.k1; k += OBK, ++g) {
          const int st = (int)(g % Sh::kStages);
          const uint32_t ph = g / Sh::kStages;
          if (!mbar_wait_bounded(&empty[st], (ph & 1) ^ 1, abort_flag, kWaitLimitNs)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&full[st], (uint32_t)Sh::kStageBytes);
          uint8_t* sb = base + (size_t)st * Sh::kStageBytes;
          tma_load_3d(sb, &tmA, &full[st], k, w.I * OBM, 0);
          tma_load_3d(sb + Sh::kABytes, &tmB, &full[st], k, w.J * BN, 0);
        }
      }
      if (!ok) raise_error(q.flags, 1);
      // the loads already issued land before the CTA's shared memory goes away,
      // also when another warp gave up after the last load was issued (in a
      // run that completes they have landed already and this returns at once)
      const uint32_t first = g > (uint32_t)Sh::kStages ? g - Sh::kStages : 0;
      for (uint32_t g2 = first; g2 < g; ++g2)
        wait_drain(&full[g2 % Sh::kStages], (g2 / Sh::kStages) & 1);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = umma_idesc_f16(OBM, BN, true);
      uint32_t g = 0, cg = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const TileWork w = tile_work<BN>(q, t);
        if (!w.valid) continue;
        const int nk = (w.k1 - w.k0) / OBK;
        for (int s0 = 0; s0 < nk && ok; s0 += kChunkStages, ++cg) {
          const uint32_t par = cg & 1;
          const int ns = min(kChunkStages, nk - s0);
          for (int s = 0; s < ns && ok; ++s, ++g) {
            const int st = (int)(g % Sh::kStages);
            const uint32_t ph = g / Sh::kStages;
            if (!mbar_wait_bounded(&full[st], ph & 1, abort_flag, kWaitLimitNs)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(base + (size_t)st * Sh::kStageBytes);
            const uint32_t sbb = sa + Sh::kABytes;
            const bool chunk_first = s == 0;
            const bool chunk_last = s == ns - 1;
            if (chunk_first) {
              // level by level, so that each level waits only for the epilogue's
              // drain of its own accumulator from the previous chunk
#pragma unroll
              for (int lam = 0; lam < kS; ++lam) {
                if (!mbar_wait_bounded(&aempty[lam], par ^ 1, abort_flag, kWaitLimitNs)) {
                  ok = false;
                  break;
                }
                tc_fence_after();
#pragma unroll
                for (int ta = 0; ta <= lam; ++ta)
                  umma_f16(tmem + (uint32_t)(lam * BN), umma_desc_sw32(sa + ta * Sh::kASlice),
                           umma_desc_sw32(sbb + (lam - ta) * Sh::kBSlice), idesc,
                           ta == 0 ? 0u : 1u);
                if (chunk_last) umma_commit(&afull[lam]);
              }
            } else {
              // A slice ta against B slices 0..6-ta at once: the B slices lie back
              // to back in shared memory (one 8-row group every 256 bytes) and the
              // accumulators of levels ta..6 back to back in tensor memory, so one
              // MMA of N = c BN covers c consecutive pairs (c <= 256 / BN)
#pragma unroll
              for (int ta = 0; ta < kS; ++ta) {
#pragma unroll
                for (int u0 = 0; u0 < kS - ta; u0 += Sh::kPerMma) {
                  const int c = (kS - ta - u0) < Sh::kPerMma ? (kS - ta - u0) : Sh::kPerMma;
                  umma_f16(tmem + (uint32_t)((ta + u0) * BN),
                           umma_desc_sw32(sa + ta * Sh::kASlice),
                           umma_desc_sw32(sbb + u0 * Sh::kBSlice),
                           umma_idesc_f16(OBM, c * BN, true), 1u);
                }
                // level ta has had its last product (ta, 0)
                if (chunk_last) umma_commit(&afull[ta]);
              }
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
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * CW);
    uint32_t cg = 0;
    bool alive = true;
    for (int t = blockIdx.x; t < ntiles && alive; t += gridDim.x) {
      const TileWork w = tile_work<BN>(q, t);
      if (!w.valid) continue;
      const int nk = (w.k1 - w.k0) / OBK;
      long long V[CW];  // exact levels 0..3, in units of 2^-24 of level 0
      float tl[CW];     // levels 4..6 (weights <= 2^-32)
#pragma unroll
      for (int j = 0; j < CW; ++j) {
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
          uint32_t r[CW];
          ld_cols(lane_base + (uint32_t)(a * BN), r);
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&aempty[a]);
          if (a < kExact) {
            // level a: an integer multiple of 2^(-8a)
            const float up = (float)(1u << (8 * a));
            const long long wgt = 1ll << (24 - 8 * a);
#pragma unroll
            for (int j = 0; j < CW; ++j) V[j] += (long long)__float2int_rn(f32(r[j]) * up) * wgt;
          } else {
#pragma unroll
            for (int j = 0; j < CW; ++j) tl[j] += f32(r[j]);
          }
        }
      }
      if (!alive) break;
      const int64_t row = (int64_t)w.I * OBM + rl;
      if (row < q.M) {
        const int ea = q.eA[row];
        const int64_t col0 = (int64_t)w.J * BN + half * CW;
#pragma unroll
        for (int j = 0; j < CW; ++j) {
          const int64_t col = col0 + j;
          if (col < q.N && (!q.lower || row + q.diag_off >= col)) {
            const int eb = q.eB[col];
            double d;
            if (ea == kExpNonFinite || eb == kExpNonFinite) {
              d = __longlong_as_double(0x7ff8000000000000ll);
            } else {
              // 2^(ea + eb - 16) (V 2^-24 + tl), with tl 2^24 exact in FP32
              d = scale2((double)V[j] + (double)(tl[j] * 16777216.f), ea + eb - 40);
            }
            if (q.neg) d = -d;
            double* cp = q.C + row + col * q.ldc;
            *cp = q.beta ? *cp + d : d;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, Sh::kTmemCols);
}

// ---------------------------------------------------------------- small nodes
// Recursion nodes of at most kSmallNode rows hold few multiply-adds (n1 n2
// (n1 + n2) in all), so on the tensor path their cost is the latency of a
// slicing and a product launch each.  Here each product is one binary64
// launch spread over the SMs, one CTA per output row (column), with the
// usual binary64 rounding of a dot product.  A CTA first stages the row
// (column) of the operand that it overwrites in shared memory, which makes
// the in-place forms safe: no other CTA reads that row (column).
constexpr int kSmallNode = 384;
constexpr int kSmallThreads = 128;

enum SmallMode : int {
  kSmL21 = 0,   // L21 = A21 Z11^T in place: b(k, j) = Z11(j, k), k <= j
  kSmSyrk = 1,  // A22 -= L21 L21^T, lower: b(k, j) = L21(j, k), j <= i
  kSmT = 2      // T = L21 Z11 into the Z21 block: b(k, j) = Z11(k, j), k >= j
};

// C(i, j) (= or -=) sum_k a(i, k) b(k, j), one row i per CTA, a(i, k) =
// a[i + k ld] staged in shared memory; b as the mode says, from B.  Four
// partial sums break the dependent chain of binary64 FMAs.
__global__ void __launch_bounds__(kSmallThreads)
    small_rows_kernel(const double* a, double* C, const double* B, int64_t ld, int N, int K,
                      int mode, const int* flags) {
  if (*(volatile const int*)&flags[kFlagPotrf] != 0) return;
  __shared__ double row[kSmallNode];
  const int i = blockIdx.x;
  for (int k = threadIdx.x; k < K; k += blockDim.x) row[k] = a[i + (int64_t)k * ld];
  __syncthreads();
  const int jend = mode == kSmSyrk ? min(N, i + 1) : N;
  for (int j = threadIdx.x; j < jend; j += blockDim.x) {
    const int k0 = mode == kSmT ? j : 0;
    const int k1 = mode == kSmL21 ? min(K, j + 1) : K;
    // b(k, j) = B[j + k ld] (L21, Syrk) or B[k + j ld] (T)
    const int64_t sk = mode == kSmT ? 1 : ld, sj = mode == kSmT ? ld : 1;
    const double* bj = B + (int64_t)j * sj;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int k = k0;
    for (; k + 3 < k1; k += 4) {
      s0 = fma(row[k], bj[k * sk], s0);
      s1 = fma(row[k + 1], bj[(k + 1) * sk], s1);
      s2 = fma(row[k + 2], bj[(k + 2) * sk], s2);
      s3 = fma(row[k + 3], bj[(k + 3) * sk], s3);
    }
    for (; k < k1; ++k) s0 = fma(row[k], bj[k * sk], s0);
    const double acc = (s0 + s1) + (s2 + s3);
    double* c = C + i + (int64_t)j * ld;
    if (mode == kSmSyrk) *c -= acc;
    else *c = acc;
  }
}

// Z21 = -Z22 T with T held in the Z21 block (n2 x n1): one column j per CTA,
// staged before it is overwritten; Z22 lower, so row i needs k <= i.
__global__ void __launch_bounds__(kSmallThreads)
    small_z21_kernel(const double* __restrict__ Z22, double* Z21, int64_t ld, int n2,
                     const int* flags) {
  if (*(volatile const int*)&flags[kFlagPotrf] != 0) return;
  __shared__ double col[kSmallNode];
  const int j = blockIdx.x;
  double* zc = Z21 + (int64_t)j * ld;
  for (int k = threadIdx.x; k < n2; k += blockDim.x) col[k] = zc[k];
  __syncthreads();
  for (int i = threadIdx.x; i < n2; i += blockDim.x) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int k = 0;
    for (; k + 3 <= i; k += 4) {
      s0 = fma(Z22[i + (int64_t)k * ld], col[k], s0);
      s1 = fma(Z22[i + (int64_t)(k + 1) * ld], col[k + 1], s1);
      s2 = fma(Z22[i + (int64_t)(k + 2) * ld], col[k + 2], s2);
      s3 = fma(Z22[i + (int64_t)(k + 3) * ld], col[k + 3], s3);
    }
    for (; k <= i; ++k) s0 = fma(Z22[i + (int64_t)k * ld], col[k], s0);
    zc[i] = -((s0 + s1) + (s2 + s3));
  }
}

// ---------------------------------------------------------------- slicing
// The kS slices of x relative to 2^E (see the file header), as BF16 bits.
// BF16 bits of a 2^(-8t) for an integer |a| <= 256, a value BF16 holds
// exactly: the float of |a| from the 2^23 exponent trick (an integer OR and
// one FP32 subtraction), scaled by an exact power of two, its upper half
// taken (its lower half is zero) and the sign set.  Integer and FP32
// arithmetic only: the conversion instructions this replaces (integer to
// float, float to BF16, two per digit and seven digits per element) share a
// pipe a quarter as wide and bounded the slicing kernel.
__device__ __forceinline__ uint16_t bf16_digit(int a, int t) {
  const unsigned int m = (unsigned int)(a < 0 ? -a : a);
  const float f = (__uint_as_float(0x4B000000u | m) - 8388608.0f) *
                  __uint_as_float((uint32_t)(127 - 8 * t) << 23);
  return (uint16_t)((__float_as_uint(f) >> 16) | (a < 0 ? 0x8000u : 0u));
}

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
    s[t] = bf16_digit((int)a, t);
  }
  s[kS - 1] = bf16_digit((int)r, kS - 1);
}

// One operand to slice: x(i, k) = src[i + k ld] (rows mode, operand rows are
// source rows) or src[k + i ld] (columns mode), i < R, k < K; written as
// out[t][i][k], t < kS, row length kld (zeros for K <= k < kld), plus the row
// exponents expo[i].  nblocks CTAs: 32 rows each (rows mode) or 16 (columns).
struct SliceJob {
  const double* src;
  int64_t ld, R, K, kld;
  uint16_t* out;
  int* expo;
  // Null: every CTA forms its rows' maxima over the whole k range itself.
  // Otherwise the row maxima of |x| as bit patterns, written by rowmax_kernel.
  unsigned long long* maxbits;
  int rows_mode;
  int kspan;    // k per CTA (a multiple of 256), kld when maxbits is null
  int kblocks;  // CTAs per row band along k
  int nblocks;  // bands x kblocks
};

constexpr int kSliceWarps = 16;
constexpr unsigned long long kInfBits = 0x7FF0000000000000ull;

// |v| as a bit pattern (integer operations only: binary64 instructions are
// scarce on this part); Inf and NaN sort above every finite value.
__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}

// The row exponent E (max |x| < 2^E) from the bit pattern of max |x|.
__device__ __forceinline__ int exponent_of_bits(unsigned long long mb) {
  if (mb >= kInfBits) return kExpNonFinite;
  if (mb == 0) return 0;
  const int ex = (int)(mb >> 52);
  return ex == 0 ? -1022 : ex - 1022;
}

// 8 consecutive k (k0 .. k0+7) of one operand row: x(k) = base[k * stride],
// sliced and stored as one 16-byte vector per slice.
__device__ __forceinline__ void load8(const double* base, int64_t stride, int64_t K, int64_t k0,
                                      double (&x)[8]) {
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int64_t k = k0 + e;
    x[e] = k < K ? base[k * stride] : 0.0;
  }
}

// The slices of x (8 consecutive k from k0), one 16-byte store per slice:
// slice t of elements 2w and 2w+1 share word w of that store.
__device__ __forceinline__ void store8(const double (&x)[8], int64_t k0, int E, uint16_t* dst,
                                       size_t plane) {
  uint32_t o[kS][4];
#pragma unroll
  for (int e = 0; e < 8; e += 2) {
    uint16_t a[kS], b[kS];
    slice_value(x[e], E, a);
    slice_value(x[e + 1], E, b);
#pragma unroll
    for (int t = 0; t < kS; ++t) o[t][e / 2] = (uint32_t)a[t] | ((uint32_t)b[t] << 16);
  }
#pragma unroll
  for (int t = 0; t < kS; ++t)
    *reinterpret_cast<uint4*>(dst + t * plane + k0) = make_uint4(o[t][0], o[t][1], o[t][2], o[t][3]);
}

// k0 = first, first + step, ... < kend: each iteration's loads are issued
// before the previous iteration's values are sliced and stored, so a warp
// keeps two iterations of loads in flight (the kernel is bound by the latency
// of its loads, not by their bandwidth).
__device__ __forceinline__ void slice_span(const double* base, int64_t stride, int64_t K,
                                           int64_t first, int64_t kend, int64_t step, int E,
                                           uint16_t* dst, size_t plane) {
  if (first >= kend) return;
  double x[8];
  load8(base, stride, K, first, x);
  for (int64_t k0 = first; k0 < kend; k0 += step) {
    double xn[8];
    const bool more = k0 + step < kend;
    if (more) load8(base, stride, K, k0 + step, xn);
    store8(x, k0, E, dst, plane);
    if (more) {
#pragma unroll
      for (int e = 0; e < 8; ++e) x[e] = xn[e];
    }
  }
}

// Rows mode tile: 32 rows (lane = row, reads coalesced along the column-major
// source) x one k span; warps split the span.
__device__ void slice_rows_tile(const SliceJob& j, int band, int kb) {
  __shared__ unsigned long long red[kSliceWarps][33];
  __shared__ int Es[32];
  const int l = threadIdx.x % 32, w = threadIdx.x / 32;
  const int64_t i = (int64_t)band * 32 + l;
  const bool iv = i < j.R;
  const double* row = j.src + (iv ? i : 0);
  if (!j.maxbits) {
    unsigned long long m = 0;
    if (iv) {
#pragma unroll 8
      for (int64_t k = w; k < j.K; k += kSliceWarps) m = max(m, abs_bits(row[k * j.ld]));
    }
    red[w][l] = m;
    __syncthreads();
    if (w == 0) {
      for (int v = 1; v < kSliceWarps; ++v) m = max(m, red[v][l]);
      const int E = exponent_of_bits(m);
      Es[l] = E;
      if (iv) j.expo[i] = E;
    }
    __syncthreads();
  } else if (w == 0) {
    const int E = iv ? exponent_of_bits(j.maxbits[i]) : 0;
    Es[l] = E;
    if (iv && kb == 0) j.expo[i] = E;
  }
  if (j.maxbits) __syncthreads();
  if (!iv) return;
  const int E = Es[l];
  const size_t plane = (size_t)j.R * j.kld;
  uint16_t* dst = j.out + i * j.kld;
  const int64_t kend = min(j.kld, (int64_t)(kb + 1) * j.kspan);
  slice_span(row, j.ld, j.K, (int64_t)kb * j.kspan + w * 8, kend, 8 * kSliceWarps, E, dst, plane);
}

// Columns mode tile: 16 operand rows (one warp each, a contiguous source
// column) x one k span.
__device__ void slice_cols_tile(const SliceJob& j, int band, int kb) {
  const int l = threadIdx.x % 32, w = threadIdx.x / 32;
  const int64_t i = (int64_t)band * kSliceWarps + w;
  if (i >= j.R) return;
  const double* col = j.src + i * j.ld;
  int E;
  if (!j.maxbits) {
    unsigned long long m = 0;
#pragma unroll 4
    for (int64_t k = l; k < j.K; k += 32) m = max(m, abs_bits(col[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    E = exponent_of_bits(m);
  } else {
    E = exponent_of_bits(j.maxbits[i]);
  }
  if (l == 0 && kb == 0) j.expo[i] = E;
  const size_t plane = (size_t)j.R * j.kld;
  uint16_t* dst = j.out + i * j.kld;
  const int64_t kend = min(j.kld, (int64_t)(kb + 1) * j.kspan);
  slice_span(col, 1, j.K, (int64_t)kb * j.kspan + l * 8, kend, 256, E, dst, plane);
}

// Up to two operands in one launch: blocks [0, a.nblocks) slice a, the rest b.
__global__ void __launch_bounds__(32 * kSliceWarps) slice_kernel(const SliceJob a,
                                                                 const SliceJob b,
                                                                 const int* flags) {
  if (*(volatile const int*)&flags[kFlagPotrf] != 0) return;
  const bool first = (int)blockIdx.x < a.nblocks;
  const SliceJob& j = first ? a : b;
  const int bid = first ? (int)blockIdx.x : (int)blockIdx.x - a.nblocks;
  const int band = bid / j.kblocks, kb = bid - band * j.kblocks;
  if (j.rows_mode) slice_rows_tile(j, band, kb);
  else slice_cols_tile(j, band, kb);
}

// Row maxima of |x| (bit patterns, atomicMax into maxbits zeroed beforehand)
// over the same tiles as slice_kernel, for operands split along k.
__global__ void __launch_bounds__(32 * kSliceWarps) rowmax_kernel(const SliceJob a,
                                                                  const SliceJob b,
                                                                  const int* flags) {
  if (*(volatile const int*)&flags[kFlagPotrf] != 0) return;
  __shared__ unsigned long long red[kSliceWarps][33];
  const bool first = (int)blockIdx.x < a.nblocks;
  const SliceJob& j = first ? a : b;
  if (!j.maxbits) return;
  const int bid = first ? (int)blockIdx.x : (int)blockIdx.x - a.nblocks;
  const int band = bid / j.kblocks, kb = bid - band * j.kblocks;
  const int l = threadIdx.x % 32, w = threadIdx.x / 32;
  const int64_t k_lo = (int64_t)kb * j.kspan, k_hi = min(j.K, k_lo + j.kspan);
  if (j.rows_mode) {
    const int64_t i = (int64_t)band * 32 + l;
    unsigned long long m = 0;
    if (i < j.R) {
      const double* row = j.src + i;
#pragma unroll 8
      for (int64_t k = k_lo + w; k < k_hi; k += kSliceWarps) m = max(m, abs_bits(row[k * j.ld]));
    }
    red[w][l] = m;
    __syncthreads();
    if (w == 0 && i < j.R) {
      for (int v = 1; v < kSliceWarps; ++v) m = max(m, red[v][l]);
      atomicMax(&j.maxbits[i], m);
    }
  } else {
    const int64_t i = (int64_t)band * kSliceWarps + w;
    if (i >= j.R) return;
    const double* col = j.src + i * j.ld;
    unsigned long long m = 0;
#pragma unroll 4
    for (int64_t k = k_lo + l; k < k_hi; k += 32) m = max(m, abs_bits(col[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (l == 0) atomicMax(&j.maxbits[i], m);
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
  unsigned long long* maxA = nullptr;  // npad: row maxima of split operands
  unsigned long long* maxB = nullptr;
  int num_sms = 1;
  int64_t launches = 0;       // kernels enqueued so far
};

namespace {

int64_t half_of(int64_t npad) { return 64 * ceil_div(npad / 64, 2); }

// Elements per slice plane: the largest operand of the recursion (half x half)
// and at least one 128-row panel of the whitening products (128 x npad).
size_t plane_cap(int64_t npad) {
  const int64_t h = half_of(npad);
  return std::max((size_t)h * (size_t)round_up(h, kKAlign), (size_t)OBM * (size_t)npad);
}

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
          strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return enc_err("slices");
  return cudaSuccess;
}

// Operands of at least this many elements are split along k as well as rows:
// a row-maxima pass, then the slicing pass, each over (rows x 1024 k) tiles.
constexpr int64_t kSplitElems = (int64_t)1 << 21;
constexpr int kSplitSpan = 1024;

SliceJob job(const double* src, int64_t ld, int64_t R, int64_t K, bool rows, uint16_t* out,
             int* expo, unsigned long long* maxbuf) {
  SliceJob j;
  j.src = src;
  j.ld = ld;
  j.R = R;
  j.K = K;
  j.kld = round_up(K, kKAlign);
  j.out = out;
  j.expo = expo;
  j.rows_mode = rows ? 1 : 0;
  const bool split = R * j.kld >= kSplitElems;
  j.maxbits = split ? maxbuf : nullptr;
  j.kspan = split ? kSplitSpan : (int)j.kld;
  j.kblocks = split ? (int)ceil_div(j.kld, kSplitSpan) : 1;
  const int64_t bands = rows ? ceil_div(R, 32) : ceil_div(R, kSliceWarps);
  j.nblocks = R <= 0 ? 0 : (int)(bands * j.kblocks);
  return j;
}

// Slices one or two operands in one launch (b.nblocks may be 0).
cudaError_t slice2(TcFactor* w, const SliceJob& a, const SliceJob& b, const int* flags,
                   cudaStream_t st) {
  const int grid = a.nblocks + b.nblocks;
  if (grid == 0) return cudaSuccess;
  if ((a.nblocks && a.maxbits) || (b.nblocks && b.maxbits)) {
    for (const SliceJob* j : {&a, &b})
      if (j->nblocks && j->maxbits) {
        cudaError_t e = cudaMemsetAsync(j->maxbits, 0, (size_t)j->R * 8, st);
        if (e != cudaSuccess) return e;
      }
    rowmax_kernel<<<grid, 32 * kSliceWarps, 0, st>>>(a, b, flags);
    ++w->launches;
  }
  slice_kernel<<<grid, 32 * kSliceWarps, 0, st>>>(a, b, flags);
  ++w->launches;
  return cudaGetLastError();
}

template <int BN>
cudaError_t launch_gemm(TcFactor* w, const Operand& A, const Operand& B, OzParams q,
                        cudaStream_t st);

// C (M x N, ldc) = (neg ? -1 : 1) A B^T + (beta ? C : 0), A = M x K and B = N x K
// operands already sliced; kmode restricts each tile's K range to the
// structural nonzeros.  Products with few 128 x 64 tiles use 128 x 16 tiles.
cudaError_t gemm(TcFactor* w, const Operand& A, const Operand& B, double* C, int64_t ldc, int M,
                 int N, int K, int kmode, int koff, bool neg, int beta, bool lower,
                 int64_t diag_off, int* flags, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  OzParams q;
  memset(&q, 0, sizeof(q));
  q.C = C;
  q.ldc = ldc;
  q.eA = A.expo;
  q.eB = B.expo;
  q.diag_off = diag_off;
  q.M = M;
  q.N = N;
  q.tilesI = (int)ceil_div(M, OBM);
  q.Kend = K;
  q.kmode = kmode;
  q.koff = koff;
  q.neg = neg ? 1 : 0;
  q.beta = beta;
  q.lower = lower ? 1 : 0;
  q.flags = flags;
  const int64_t tiles64 = (int64_t)q.tilesI * ceil_div(N, 64);
  if (tiles64 * 4 <= w->num_sms) {
    q.tilesJ = (int)ceil_div(N, 16);
    return launch_gemm<16>(w, A, B, q, st);
  }
  q.tilesJ = (int)ceil_div(N, 64);
  return launch_gemm<64>(w, A, B, q, st);
}

template <int BN>
cudaError_t launch_gemm(TcFactor* w, const Operand& A, const Operand& B, OzParams q,
                        cudaStream_t st) {
  using Sh = Shape<BN>;
  static bool attr_done[64] = {};  // per instantiation and device
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr_done[dev]) {
    cudaError_t e = cudaFuncSetAttribute(oz_gemm_kernel<BN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Sh::kSmemBytes);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_done[dev] = true;
  }
  CUtensorMap ta, tb;
  cudaError_t e;
  if ((e = encode(&ta, A, OBM)) != cudaSuccess) return e;
  if ((e = encode(&tb, B, BN)) != cudaSuccess) return e;
  // tiles of the launch (the lower ones only for a lower-triangular output)
  int64_t tiles = (int64_t)q.tilesI * q.tilesJ;
  if (q.lower && q.kmode == kKFull) {  // tile_work lists only the valid ones then
    tiles = 0;
    for (int I = 0; I < q.tilesI; ++I) {
      const int64_t c = ((int64_t)I * OBM + OBM - 1 + q.diag_off) / BN + 1;
      tiles += c < 0 ? 0 : std::min<int64_t>(c, q.tilesJ);
    }
  }
  if (tiles == 0) return cudaSuccess;
  q.ntiles = (int)tiles;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(w->num_sms, tiles));
  oz_gemm_kernel<BN><<<grid, kThreads, Sh::kSmemBytes, st>>>(ta, tb, q);
  ++w->launches;
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
    ++w->launches;
    return cudaGetLastError();
  }
  const int64_t n1 = 64 * ((n / 64) / 2), n2 = n - n1;
  TC_TRY(rec(w, A, Z, ld, r0, n1, flags, st));
  double* A21 = A + (r0 + n1) + r0 * ld;
  double* A22 = A + (r0 + n1) + (r0 + n1) * ld;
  double* Z11 = Z + r0 + r0 * ld;
  double* Z21 = Z + (r0 + n1) + r0 * ld;
  double* Z22 = Z + (r0 + n1) + (r0 + n1) * ld;
  if (n <= kSmallNode) {
    const dim3 rows((unsigned)n2), cols((unsigned)n1);
    small_rows_kernel<<<rows, kSmallThreads, 0, st>>>(A21, A21, Z11, ld, (int)n1, (int)n1,
                                                      kSmL21, flags);
    small_rows_kernel<<<rows, kSmallThreads, 0, st>>>(A21, A22, A21, ld, (int)n2, (int)n1,
                                                      kSmSyrk, flags);
    small_rows_kernel<<<rows, kSmallThreads, 0, st>>>(A21, Z21, Z11, ld, (int)n1, (int)n1, kSmT,
                                                      flags);
    w->launches += 3;
    TC_TRY(cudaGetLastError());
    TC_TRY(rec(w, A, Z, ld, r0 + n1, n2, flags, st));
    small_z21_kernel<<<cols, kSmallThreads, 0, st>>>(Z22, Z21, ld, (int)n2, flags);
    ++w->launches;
    return cudaGetLastError();
  }
  const Operand SA1{w->SA, w->eA, n2, round_up(n1, kKAlign)};
  const Operand SB1{w->SB, w->eB, n1, round_up(n1, kKAlign)};
  // L21 = A21 Z11^T (Z11 lower: column block J needs k < (J+1) BN)
  TC_TRY(slice2(w, job(A21, ld, n2, n1, true, w->SA, w->eA, w->maxA),
                job(Z11, ld, n1, n1, true, w->SB, w->eB, w->maxB), flags, st));
  TC_TRY(gemm(w, SA1, SB1, A21, ld, (int)n2, (int)n1, (int)n1, kKLeJ, 0, false, 0, false, 0,
              flags, st));
  // One slicing of L21 serves both the trailing update and T = L21 Z11, which
  // does not depend on the factor of A22 and is formed before it.  T is kept
  // in the Z21 block (zero until Z21 = -Z22 T overwrites it below); the
  // recursion on A22 touches only A22 and Z22.
  TC_TRY(slice2(w, job(A21, ld, n2, n1, true, w->SA, w->eA, w->maxA),
                job(Z11, ld, n1, n1, false, w->SB, w->eB, w->maxB), flags, st));
  // A22 -= L21 L21^T (lower triangle)
  TC_TRY(gemm(w, SA1, SA1, A22, ld, (int)n2, (int)n2, (int)n1, kKFull, 0, true, 1, true, 0, flags,
              st));
  // T = L21 Z11 (Z11 lower: column j needs k >= j)
  TC_TRY(gemm(w, SA1, SB1, Z21, ld, (int)n2, (int)n1, (int)n1, kKGeJ, 0, false, 0, false, 0,
              flags, st));
  TC_TRY(rec(w, A, Z, ld, r0 + n1, n2, flags, st));
  // Z21 = -Z22 T (Z22 lower: row block I needs k < (I+1) 128); T's slices are
  // taken before the product overwrites it
  const Operand SA2{w->SA, w->eA, n2, round_up(n2, kKAlign)};
  const Operand SB2{w->SB, w->eB, n1, round_up(n2, kKAlign)};
  TC_TRY(slice2(w, job(Z22, ld, n2, n2, true, w->SA, w->eA, w->maxA),
                job(Z21, ld, n1, n2, false, w->SB, w->eB, w->maxB), flags, st));
  TC_TRY(gemm(w, SA2, SB2, Z21, ld, (int)n2, (int)n1, (int)n2, kKLeI, 0, true, 0, false, 0, flags,
              st));
  return cudaSuccess;
}

// Rows per panel so that rows x K fits one slice plane.
int64_t panel_rows(const TcFactor* w, int64_t K) {
  int64_t P = (int64_t)(w->cap / (size_t)round_up(K, kKAlign));
  P = (P / OBM) * OBM;
  return std::max<int64_t>(P, OBM);
}

}  // namespace

size_t tc_factor_bytes(int64_t npad) {
  return 2 * (size_t)kS * plane_cap(npad) * 2 + 2 * (size_t)npad * (4 + 8);
}

const char* tc_factor_last_error() { return g_err.c_str(); }

void tc_factor_free(TcFactor* w) {
  if (!w) return;
  cudaFree(w->SA);
  cudaFree(w->SB);
  cudaFree(w->eA);
  cudaFree(w->eB);
  cudaFree(w->maxA);
  cudaFree(w->maxB);
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
      cudaMalloc(&w->maxA, (size_t)npad * 8) != cudaSuccess ||
      cudaMalloc(&w->maxB, (size_t)npad * 8) != cudaSuccess) {
    cudaGetLastError();
    tc_factor_free(w);
    g_err = "cudaMalloc of the tensor-core factor workspace failed";
    return GLS_ERR_OOM;
  }
  *out = w;
  return GLS_OK;
}

int64_t tc_launches(const TcFactor* w) { return w->launches; }

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
    TC_TRY(slice2(w, job(Z + i0, ldz, rows, K, true, w->SA, w->eA, w->maxA),
                  job(rhs, ldr, ncols, K, false, w->SB, w->eB, w->maxB), flags, st));
    const Operand a{w->SA, w->eA, rows, round_up(K, kKAlign)};
    const Operand b{w->SB, w->eB, ncols, round_up(K, kKAlign)};
    TC_TRY(gemm(w, a, b, out + i0, ldo, (int)rows, ncols, (int)K, kKLeI, (int)i0, false, 0, false,
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
    TC_TRY(slice2(w, job(Z + c0 + c0 * ldz, ldz, rows, K, false, w->SA, w->eA, w->maxA),
                  job(rhs + c0, ldr, ncols, K, false, w->SB, w->eB, w->maxB), flags, st));
    const Operand a{w->SA, w->eA, rows, round_up(K, kKAlign)};
    const Operand b{w->SB, w->eB, ncols, round_up(K, kKAlign)};
    TC_TRY(gemm(w, a, b, out + c0, ldo, (int)rows, ncols, (int)K, kKGeI, 0, false, 0, false, 0,
                flags, st));
  }
  return cudaSuccess;
}

}  // namespace gls
