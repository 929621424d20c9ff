// trsm_mixed.cu -- mixed-precision blocked triangular solve of a block of SNP
// columns on tcgen05 tensor cores, with the Gram epilogue fused in
// (Alg. 5 lines 3 and 8-10; the grouped TRSM of Section 2).
//
// Blocked form.  With Z = L^{-1} (binary64, from the setup),
//     x~_I = Z_II x_I + sum_{K<I} Z_IK x_K,
// i.e. L_KK^{-1} applied to the diagonal block plus the off-diagonal updates.
// The genotype codes x are small integers, exact in BF16/FP16, so only Z is
// split.  For every row r of Z the entries left of its nd x nd diagonal block
// are written as
//     Z_rc = u_r (H_rc + R1_rc + R2_rc),   u_r = 2^(E_r - B),
// where 2^E_r bounds the row's largest such |Z_rc|, H_rc = rint(Z_rc / u_r) is an
// integer of at most B bits (B = 7 for BF16, 10 for FP16) and R1, R2 are the
// first two 16-bit float terms of the remainder (|R| <= 1/2).  Products of H
// with genotype codes are integers, so their FP32 tensor-core sum is exact
// while it stays below 2^24 in magnitude (any n <= 65536 for |x| <= 2 with
// BF16); the remainder terms are 2^-B smaller, so FP32 rounding in their sum
// is negligible.  Slice H accumulates in one TMEM accumulator, R1 + R2 in a
// second one.  The epilogue forms
//     x~_r = u_r (acc_H + acc_R) + d_r,   d_r = sum_{c in diag block} Z_rc x_c
// rounded once to FP32, and reduces S_BR = x~^T x~ over the tile's 128 rows in
// a compensated FP32 sum (see add_squares4), written as FP64 partials.  d_r
// is formed in FP32 as well, from the split
//     Z_rc = s_r k_rc + l_rc,   s_r = 2^(E_r - 12),   k_rc = rint(Z_rc / s_r),
// where 2^E_r bounds the row's diagonal-block entries: the integers k (|k| <=
// 2^12) times genotype codes sum exactly in FP32, the FP32 low parts l
// (|l| <= s_r / 2) carry the rest, and d_r = fma(sum k x, s_r, sum l x) is
// rounded once, to about the accuracy of rounding the exact d_r to FP32 (x~_r
// is rounded to FP32 right after anyway).  Binary64 arithmetic runs at a small
// fraction of the FP32 rate on this part, and the epilogue is not overlapped
// with the products.
//
// The other Gram entries of Fig. 1 are linear in x~, and
//     S_BL_i = X~_L^T x~_i = (Z^T X~_L)^T x_i,   b_B_i = y~^T x~_i = (Z^T y~)^T x_i,
// so they are computed from the exact genotypes with W = Z^T [X~_L | y~]
// (= M^{-1} [X_L | y], binary64, once per factor) split the same way as Z: one
// extra 128-row block of the A operand holds the p rows of W^T, its K range
// is all n, and its accumulators give the p products per SNP directly, with
// no cross-row reduction.  All S slices of those rows go through one product
// of N = 32 S, each slice into its own 32 accumulator columns, added once in
// the epilogue: sharing one FP32 sum inside the tensor core with the larger
// slice cost the low slices most of their bits.  (In FP32 those cross products lose accuracy to
// cancellation; through the exact split they keep about 2^-25 relative to
// each row's scale.)
//
// Kernel shape (one persistent CTA per SM, 320 threads):
//   warp 0      TMA producer: per stage the 128-SNP x 32 genotype tile and the S
//               slices of Z for the item's 256 rows (256 x 32 each), 64-byte
//               swizzled, one mbarrier
//   warp 1      TMEM allocator and the single thread issuing tcgen05.mma
//               (M = 128 SNPs, N = 256 rows of x~, K = 16) into one accumulator
//               pair (acc_H, acc_R: 256 columns each); genotypes are operand A.
//               N = 256 rather than 128 cuts the operand bytes the tensor core
//               reads from shared memory per multiply-add by a quarter and halves
//               the genotype bytes the TMA writes there: shared-memory bandwidth,
//               not the tensor rate, is what limits the 128 x 128 shape
//   warps 2-9   epilogue, one SNP per thread (its TMEM lane), two warps per lane
//               quarter, each taking one of the item's two 128-row blocks:
//               tcgen05.ld of 32 rows at a time, the 4 x 4 diagonal blocks (FP32 split)
//               from the SNP's own genotypes, and the S_BR sum in registers
// Work items (row-block pair I = blocks 2I and 2I+1, SNP tile J), I = 0..nP
// (nP = ceil(nI / 2); I = nP is the W^T block, issued with N = 32 S, and an
// odd last pair holds one block, issued with N = 128), run heaviest first in groups of `group`
// pairs x all SNP tiles, so the concurrently running CTAs share both the Z
// slices of a few row blocks and the genotype panels of a few dozen SNP tiles
// in L2.  The accumulators are single-buffered: the epilogue of an item is
// short next to its K loop (K = 256 (I + 1) deep), so the tensor core waits on
// it for a few percent of the time.
//
// One launch can serve many independent problems (scans with their own M, n,
// p and SNP block): each problem has a descriptor in device memory (its
// buffers), its TMA maps travel by value in the launch's parameters, and the
// by-value run parameters give each problem's block size and the prefix of
// its work items; the persistent CTAs walk the concatenated item list,
// largest problems first.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <stdio.h>

#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"
#include "mixed.cuh"
#include "sm100.cuh"

namespace gls {

using namespace sm100;

namespace {

constexpr int BM = 128;                 // rows of x~ per row block
constexpr int kPair = 2 * BM;           // rows of x~ per work item (MMA N)
constexpr int BN = 128;                 // SNPs per tile (MMA M, TMEM lanes)
constexpr int BK = 32;                  // K per stage: 32 x 16-bit = one 64-byte swizzle row
constexpr int kSliceBytes = kPair * BK * 2;  // one slice of Z for an item, per stage
constexpr int kXBytes = BN * BK * 2;         // the genotype tile, per stage
constexpr int kRowsBytes = kPair * (4 + 8 * 4 + 4);  // u_r, (k, l) of the diagonal blocks, s_r
constexpr int kEpiWarps = 8;             // two per TMEM lane quarter
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr uint32_t kTmemCols = 512;     // acc_H and acc_R, 256 columns each
constexpr uint32_t kAccR = 256;         // column of acc_R
constexpr int kMaxDynSmem = 232448;     // 227 KB
constexpr int kDiag = 4;                // nd: diagonal block edge
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // bounded waits give up after 1 s (default)
constexpr uint64_t kDrainLimitNs = 100000000ull;
constexpr int kDefaultGroup = 3;        // row-block pairs per rasterization group

// Z's slices (and the rows of W^T) are stored pre-tiled for plain bulk copies:
// per slice s, 256-row group g (row pair g of Z; g = nP holds the W^T rows)
// and 32-deep K stage kb, one 16 KB tile in the MMA's K-major layout without
// swizzling: core matrices of 8 rows x 8 values (128 contiguous bytes), the 4
// along K 128 bytes apart, groups of 8 rows 512 bytes apart.  A stage's slice
// then arrives as 128 long contiguous requests instead of 256 rows of 64
// bytes: the solve is bound by the rate of requests an SM sends to L2 (one
// 64-byte row per request through a tensor map, measured: halving the rows
// to 32 bytes doubled the requests and made it 58% slower).
constexpr int kTileElems = kPair * BK;   // 8192 16-bit values, 16 KB
constexpr uint32_t kCoreLbo = 128;       // bytes between core matrices adjacent along K
constexpr uint32_t kCoreSbo = 512;       // bytes between groups of 8 rows

__host__ __device__ __forceinline__ size_t tile_index(int s, int g, int64_t kb, int nG,
                                                      int64_t nKB) {
  return ((size_t)s * nG + g) * (size_t)nKB + (size_t)kb;
}
// Position of (row rr < 256, column kk < 32) inside a tile.
__host__ __device__ __forceinline__ int in_tile(int rr, int kk) {
  return (((rr >> 3) * 4 + (kk >> 3)) * 8 + (rr & 7)) * 8 + (kk & 7);
}

thread_local std::string g_err;

// Per-problem constants, in device memory.
struct ProblemDesc {
  const uint16_t* tiles;  // the pre-tiled slices of Z and W^T (see kTileElems)
  int64_t nKB;            // K stages per row: npad / 32
  int nG;                 // 256-row groups: row pairs plus the W^T group
  const uint16_t* x16;    // genotype operand, SNP-major [j][npad], zero rows >= n
  int bf16;               // its codes are BF16 (else FP16)
  const float* rowscale;  // u_r, npad + 128 rows
  const float* diagKL;    // npad x (k[4], l[4]): split diagonal blocks
  const float* diagS;     // npad: s_r
  double* Pbr;            // S_BR partials, nI x ldp
  double* Glin;           // S_BL and b_B, p x ldp
  int64_t npad, ldp;
  int nI, p;
  uint32_t idesc, idesc_half;  // MMA N = 256 (two row blocks) and N = 128 (one), BF16 or FP16
  uint32_t idesc_w;            // MMA N = 32 S: the W^T block's rows of all S slices
};

// The TMA map of every problem's genotype operand in a launch, passed by value
// as a __grid_constant__ parameter (8 KB for kMaxBatch problems): the TMA unit
// reads them from parameter space, so no map ever lives in global memory
// that the host writes and later frees and reuses.
struct MapSet {
  CUtensorMap tmB[kMaxBatch];  // genotype operand X16: (npad, kmax), 16-bit
};

// Per-launch values, by value: each problem's block size and item range.
struct RunParams {
  int nprob, total, group;
  int nJ[kMaxBatch];
  int item_begin[kMaxBatch + 1];
  int64_t k[kMaxBatch];
};

struct KConst {
  int S, stages;
  uint64_t wait_ns;  // limit of every pipeline wait
  int* flags;
  uint32_t off_rows, off_bar, stage_bytes;
};

// Work item t of one problem -> (row-block pair I, SNP tile J): groups of
// `group` pairs, heaviest first; within a group SNP tiles advance slowest.
__device__ __forceinline__ void decode_item(int t, int nIt, int nJ, int group, int& I, int& J) {
  const int per = group * nJ;
  const int full = nIt / group, tail = nIt - full * group;
  int g, ii;
  if (t < full * per) {
    g = t / per;
    const int rem = t - g * per;
    J = rem / group;
    ii = rem - J * group;
  } else {
    g = full;
    const int rem = t - full * per;
    J = rem / tail;
    ii = rem - J * tail;
  }
  I = nIt - 1 - (g * group + ii);
}

// Global item t -> problem index (the item ranges are in ascending order).
__device__ __forceinline__ int find_problem(const RunParams& run, int t) {
  int lo = 0, hi = run.nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (run.item_begin[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

struct Item {
  int pi, I, J, nI, nP;  // I == nP: the W^T block
  __device__ __forceinline__ bool lin() const { return I == nP; }
  // both row blocks of a pair exist (MMA N = 256); else N = 128
  __device__ __forceinline__ bool wide() const { return I < nP && 2 * I + 1 < nI; }
  // 16-bit K extent: rows left of the pair's end, or all of them for W^T
  __device__ __forceinline__ int kblocks() const {
    return (lin() ? nI : min(2 * I + 2, nI)) * (BM / BK);
  }
  __device__ __forceinline__ int row0() const { return lin() ? nI * BM : I * kPair; }
};

__device__ __forceinline__ Item item_at(const ProblemDesc* probs, const RunParams& run, int t) {
  Item w;
  w.pi = find_problem(run, t);
  w.nI = probs[w.pi].nI;
  w.nP = (w.nI + 1) >> 1;
  decode_item(t - run.item_begin[w.pi], w.nP + 1, run.nJ[w.pi], run.group, w.I, w.J);
  return w;
}

__device__ void raise_error(int* flags, int site) {
  atomicOr(&flags[kFlagKernel], kErrTimeout);
  atomicExch(&flags[kFlagWhere], site);
}

// True when every epilogue thread passes ok = true (named barrier 1).
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

// Four 16-bit genotype codes (two per word, low half first) as four signed
// bytes.  The codes hold integers, so each converts back exactly: BF16 widens
// to FP32 by a shift, FP16 through the half type.
__device__ __forceinline__ uint32_t codes_to_bytes(uint32_t w0, uint32_t w1, bool bf16) {
  const uint32_t h[4] = {w0 & 0xFFFFu, w0 >> 16, w1 & 0xFFFFu, w1 >> 16};
  uint32_t r = 0;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float f = bf16 ? __uint_as_float(h[e] << 16)
                         : __half2float(__ushort_as_half((unsigned short)h[e]));
    r |= (uint32_t)(uint8_t)(int8_t)__float2int_rz(f) << (8 * e);
  }
  return r;
}

// Signed byte k of w as a float: the byte (offset by 128) becomes the low
// mantissa bits of 2^23, and the subtraction is exact.
template <int k>
__device__ __forceinline__ float byte_to_float(uint32_t w_flipped) {
  return __int_as_float((int)__byte_perm(w_flipped, 0x4B000000u, 0x7540u + k)) - 8388736.0f;
}

__device__ __forceinline__ float two_sum(float a, float b, float& err) {
  const float s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
  return s;
}

// Adds the squares of four rows' values v = u (aH + aR) + d to the
// compensated sum (sum, comp): u is a power of two, d the diagonal-block term.
// Each value and its square are rounded once and the four squares summed in
// FP32; only that partial sum joins the running total through an error-free
// two-sum.  The per-row roundings are a few units in the last place of values
// whose FP32 tensor-core accumulation already carries a larger error, and
// being independent and unbiased they shrink against the total over n rows;
// the long sum across the rows is the part whose error would grow with n, and
// it is the part that is compensated.
__device__ __forceinline__ void add_squares4(const uint32_t* aH, const uint32_t* aR,
                                             const float* u, float d0, float d1, float d2,
                                             float d3, float& sum, float& comp) {
  const float h0 = fmaf(u[0], __fadd_rn(__uint_as_float(aH[0]), __uint_as_float(aR[0])), d0);
  const float h1 = fmaf(u[1], __fadd_rn(__uint_as_float(aH[1]), __uint_as_float(aR[1])), d1);
  const float h2 = fmaf(u[2], __fadd_rn(__uint_as_float(aH[2]), __uint_as_float(aR[2])), d2);
  const float h3 = fmaf(u[3], __fadd_rn(__uint_as_float(aH[3]), __uint_as_float(aR[3])), d3);
  const float q = __fadd_rn(fmaf(h0, h0, __fmul_rn(h1, h1)), fmaf(h2, h2, __fmul_rn(h3, h3)));
  float e;
  sum = two_sum(sum, q, e);
  comp = __fadd_rn(comp, e);
}

__global__ void __launch_bounds__(kThreads, 1)
    trsm_gram_mixed_kernel(const ProblemDesc* __restrict__ probs,
                           const __grid_constant__ RunParams run, const KConst kc,
                           const __grid_constant__ MapSet maps) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + kc.off_bar);
  uint64_t* empty = full + kc.stages;
  uint64_t* tfull = empty + kc.stages;
  uint64_t* tempty = tfull + 1;
  uint64_t* drain = tempty + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  // per-item row data, double-buffered: u_r, the split diagonal blocks (k[4], l[4]), s_r
  uint8_t* rows_base = base + kc.off_rows;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int S = kc.S, stages = kc.stages;
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, kEpiWarps);
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
  const int total = run.total;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
      int last_pi = -1;
      for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
        const Item w = item_at(probs, run, t);
        const ProblemDesc* pd = probs + w.pi;
        const CUtensorMap* tB = &maps.tmB[w.pi];
        if (w.pi != last_pi) {
          tma_prefetch_desc(tB);
          last_pi = w.pi;
        }
        // group I of the tiled slices (I = nP is the W^T group); an N = 128
        // product reads the first 128 rows of the tile only (its first 8 KB),
        // the W^T product its first 32 rows (2 KB) of every slice, landed
        // side by side so that one N = 32 S product covers all slices
        const uint16_t* tiles = pd->tiles;
        const int nG = pd->nG;
        const int64_t nKB = pd->nKB;
        const uint32_t slice_bytes = w.wide()  ? (uint32_t)kSliceBytes
                                     : w.lin() ? (uint32_t)kSliceBytes / 8
                                               : (uint32_t)kSliceBytes / 2;
        const int kblocks = w.kblocks();
        for (int kb = 0; kb < kblocks; ++kb, ++g) {
          const int st = (int)(g % stages);
          const uint32_t ph = g / stages;
          if (!mbar_wait_bounded(&empty[st], (ph & 1) ^ 1, abort_flag, kc.wait_ns)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&full[st], (uint32_t)S * slice_bytes + kXBytes);
          uint8_t* sb = base + (size_t)st * kc.stage_bytes;
          const uint32_t dst_stride = w.lin() ? slice_bytes : (uint32_t)kSliceBytes;
          for (int s = 0; s < S; ++s)
            bulk_load(sb + s * dst_stride, tiles + tile_index(s, w.I, kb, nG, nKB) * kTileElems,
                      slice_bytes, &full[st]);
          tma_load_2d(sb + S * kSliceBytes, tB, &full[st], kb * BK, w.J * BN);
        }
      }
      if (!ok) raise_error(kc.flags, 1);
      // the loads already issued land before the CTA's shared memory goes away,
      // also when another warp gave up after the last load was issued (in a
      // run that completes they have landed already and this returns at once)
      const uint32_t first = g > (uint32_t)stages ? g - stages : 0;
      for (uint32_t g2 = first; g2 < g; ++g2)
        wait_drain(&full[g2 % stages], (g2 / stages) & 1);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
      int it = 0;
      const uint32_t dH = tmem, dR = tmem + kAccR;
      for (int t = blockIdx.x; t < total && ok; t += gridDim.x, ++it) {
        const Item w = item_at(probs, run, t);
        const int kblocks = w.kblocks();
        const bool lin = w.lin();
        // the operand type is per problem: a batch may mix BF16 and FP16 plans
        const uint32_t idesc = w.wide()  ? probs[w.pi].idesc
                               : w.lin() ? probs[w.pi].idesc_w
                                         : probs[w.pi].idesc_half;
        // the epilogue has read the previous item's accumulators
        if (!mbar_wait_bounded(tempty, ((uint32_t)it & 1) ^ 1, abort_flag, kc.wait_ns)) {
          ok = false;
          break;
        }
        tc_fence_after();
        for (int kb = 0; kb < kblocks; ++kb, ++g) {
          const int st = (int)(g % stages);
          const uint32_t ph = g / stages;
          if (!mbar_wait_bounded(&full[st], ph & 1, abort_flag, kc.wait_ns)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sz = smem_u32(base + (size_t)st * kc.stage_bytes);  // Z slices
          const uint32_t sx = sz + (uint32_t)S * kSliceBytes;                 // genotypes
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            // genotypes: 64-byte swizzled rows (TMA); slices: untiled core
            // matrices, the second K = 16 half two core matrices further on
            const uint64_t adesc = umma_desc_sw64(sx + kk * 32);
            const uint32_t first = (kb | kk) != 0;
            // W^T: the S slices' 32 rows each side by side, one product; slice s
            // lands in accumulator columns 32 s .. 32 s + 31, so no slice's
            // products share a sum with another's
            umma_f16(dH, adesc, umma_desc_noswz(sz + kk * 2 * kCoreLbo, kCoreLbo, kCoreSbo), idesc,
                     first);
            if (!lin)
              for (int s = 1; s < S; ++s)
                umma_f16(dR, adesc,
                         umma_desc_noswz(sz + s * kSliceBytes + kk * 2 * kCoreLbo, kCoreLbo,
                                         kCoreSbo),
                         idesc, first | (s > 1));
          }
          umma_commit(&empty[st]);
        }
        if (ok) umma_commit(tfull);
      }
      if (!ok) raise_error(kc.flags, 2);
      // every issued MMA completes before the accumulators are released
      umma_commit(drain);
      wait_drain(drain, 0);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int quarter = warp & 3;            // TMEM lanes this warp may read
    const int half = (warp - 2) >> 2;        // which row block of the pair this warp handles
    const int lrow = quarter * 32 + lane;    // accumulator lane = SNP within the tile
    const int et = threadIdx.x - 64;         // 0..255
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    int it = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x, ++it) {
      const Item w = item_at(probs, run, t);
      const ProblemDesc* pd = probs + w.pi;
      const bool lin = w.lin();
      const int blk = 2 * w.I + half;        // this warp's row block
      const bool bv = !lin && blk < w.nI;
      const int p = pd->p;
      const int64_t kk_j = run.k[w.pi];
      const int64_t ldp = pd->ldp;
      const uint32_t ph = (uint32_t)it & 1;
      const int64_t j = (int64_t)w.J * BN + lrow;
      const bool jv = j < kk_j;
      float* su = reinterpret_cast<float*>(rows_base + ph * kRowsBytes);
      float* skl = su + kPair;           // row r: k[0..3], l[0..3]
      float* ss = skl + kPair * 8;
      {
        const int64_t r = (int64_t)w.row0() + et;
        if (lin) {
          if (et < BM) su[et] = pd->rowscale[r];
        } else if (r < pd->npad) {
          su[et] = pd->rowscale[r];
          const float4* src = reinterpret_cast<const float4*>(pd->diagKL + r * 8);
          reinterpret_cast<float4*>(skl)[et * 2] = src[0];
          reinterpret_cast<float4*>(skl)[et * 2 + 1] = src[1];
          ss[et] = pd->diagS[r];
        }
      }
      // this SNP's genotypes of this warp's 128 rows, as signed bytes, read
      // from the operand while the tile's products are still running
      uint4 xv[BM / 16];
#pragma unroll
      for (int i = 0; i < BM / 16; ++i) xv[i] = make_uint4(0, 0, 0, 0);
      if (bv && jv) {
        const uint4* src =
            reinterpret_cast<const uint4*>(pd->x16 + j * pd->npad + (int64_t)blk * BM);
        const bool b16 = pd->bf16 != 0;
#pragma unroll
        for (int i = 0; i < BM / 16; ++i) {
          const uint4 a = __ldg(src + 2 * i), b = __ldg(src + 2 * i + 1);
          xv[i] = make_uint4(codes_to_bytes(a.x, a.y, b16), codes_to_bytes(a.z, a.w, b16),
                             codes_to_bytes(b.x, b.y, b16), codes_to_bytes(b.z, b.w, b16));
        }
      }
      const bool got = mbar_wait_bounded(tfull, ph, abort_flag, kc.wait_ns);
      if (!epilogue_all(got)) {  // all epilogue threads leave together; also orders the row data
        if (!got && lane == 0) raise_error(kc.flags, 3);
        break;
      }
      tc_fence_after();
      if (lin) {
        // W^T block: column q < p holds (M^{-1}[X_L | y])_q^T x_j
        if (half == 0) {
          // slice 0 in columns 0 .. 31, slice s > 0 in 32 s .. 32 s + 31
          uint32_t aH[32], aR[32];
          float lo[32];
#pragma unroll
          for (int q = 0; q < 32; ++q) lo[q] = 0.f;
          for (int s = 1; s < S; ++s) {
            tmem_ld32(lane_base + 32u * (uint32_t)s, aR);
            tmem_ld_wait(aR);
#pragma unroll
            for (int q = 0; q < 32; ++q) lo[q] += __uint_as_float(aR[q]);
          }
          tmem_ld32(lane_base, aH);
          tmem_ld_wait(aH);
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(tempty);
          if (jv) {
#pragma unroll
            for (int q = 0; q < 32; ++q)
              if (q < p)
                pd->Glin[(int64_t)q * ldp + j] =
                    (double)su[q] *
                    ((double)__uint_as_float(aH[q]) + (double)lo[q]);
          }
        } else {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(tempty);
        }
        continue;
      }
      if (!bv) {  // the missing second block of an odd last pair
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty);
        continue;
      }
      float sum = 0.f, comp = 0.f;
#pragma unroll 1
      for (int c = 0; c < BM / 32; ++c) {  // 32-row chunk of this warp's block
        const uint32_t col = (uint32_t)(half * BM + c * 32);
        uint32_t aH[32], aR[32];
        tmem_ld32(lane_base + col, aH);
        tmem_ld32(lane_base + kAccR + col, aR);
        uint4 v0 = xv[0], v1 = xv[1];
#pragma unroll
        for (int q = 1; q < BM / 32; ++q)
          if (c == q) {
            v0 = xv[2 * q];
            v1 = xv[2 * q + 1];
          }
        tmem_ld_wait(aH);
        tmem_ld_fence(aR);
        if (c == BM / 32 - 1) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(tempty);
        }
#pragma unroll
        for (int g4 = 0; g4 < 8; ++g4) {
          // rows 4*g4 .. 4*g4+3 of this chunk form one diagonal block
          const uint4 v4 = g4 < 4 ? v0 : v1;
          const uint32_t wv = ((g4 & 3) == 0 ? v4.x : (g4 & 3) == 1 ? v4.y
                             : (g4 & 3) == 2 ? v4.z : v4.w) ^ 0x80808080u;
          const float x0 = byte_to_float<0>(wv), x1 = byte_to_float<1>(wv);
          const float x2 = byte_to_float<2>(wv), x3 = byte_to_float<3>(wv);
          const int rl = half * BM + c * 32 + g4 * 4;  // row within the pair
          const float* z = skl + rl * 8;               // row rl + i: k at 8i, l at 8i + 4
          const float4 s4 = *reinterpret_cast<const float4*>(ss + rl);
          // integer parts: exact; low parts: one rounding each; d = fma(k x, s, l x)
          const float d0 = fmaf(z[0] * x0, s4.x, z[4] * x0);
          const float d1 = fmaf(fmaf(z[9], x1, z[8] * x0), s4.y, fmaf(z[13], x1, z[12] * x0));
          const float d2 = fmaf(fmaf(z[18], x2, fmaf(z[17], x1, z[16] * x0)), s4.z,
                                fmaf(z[22], x2, fmaf(z[21], x1, z[20] * x0)));
          const float d3 =
              fmaf(fmaf(z[27], x3, fmaf(z[26], x2, fmaf(z[25], x1, z[24] * x0))), s4.w,
                   fmaf(z[31], x3, fmaf(z[30], x2, fmaf(z[29], x1, z[28] * x0))));
          add_squares4(aH + g4 * 4, aR + g4 * 4, su + rl, d0, d1, d2, d3, sum, comp);
        }
      }
      if (jv) pd->Pbr[(int64_t)blk * ldp + j] = (double)sum + (double)comp;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, kTmemCols);
}

// BF16 or FP16 bits of a genotype code c (|c| <= 128, exact in both): the
// float of |c| from the 2^23 exponent trick (an integer OR and one FP32
// subtraction), then its upper half (BF16) or its exponent rebased and
// mantissa shifted (FP16), and the sign.  Integer and FP32 arithmetic only,
// instead of two conversion instructions per code on a pipe a quarter as wide.
template <bool kBF16>
__device__ __forceinline__ uint32_t code16(int c) {
  const uint32_t m = (uint32_t)(c < 0 ? -c : c);
  const uint32_t fb = __float_as_uint(__uint_as_float(0x4B000000u | m) - 8388608.0f);
  uint32_t h;
  if (kBF16) h = fb >> 16;
  else h = m ? (fb >> 13) - (112u << 10) : 0u;
  return h | (c < 0 ? 0x8000u : 0u);
}

// X_R block (n x k int8, ldx) -> operand layout X16[j][c] (16-bit), c < npad
// (zero rows >= n).
template <bool kBF16>
__global__ void convert_x_kernel(const int8_t* __restrict__ x8, int64_t ldx, int64_t n,
                                 int64_t k, int64_t npad, uint16_t* __restrict__ x16) {
  const int64_t per_col = npad / 8;
  const int64_t total = k * per_col;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = idx / per_col;
    const int64_t c0 = (idx - j * per_col) * 8;
    uint16_t v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int64_t c = c0 + e;
      const int xi = (c < n) ? (int)x8[c + j * ldx] : 0;
      v[e] = (uint16_t)code16<kBF16>(xi);
    }
    uint4 w;
    w.x = (uint32_t)v[0] | ((uint32_t)v[1] << 16);
    w.y = (uint32_t)v[2] | ((uint32_t)v[3] << 16);
    w.z = (uint32_t)v[4] | ((uint32_t)v[5] << 16);
    w.w = (uint32_t)v[6] | ((uint32_t)v[7] << 16);
    *reinterpret_cast<uint4*>(x16 + j * npad + c0) = w;
  }
}

// The same output with 16 rows per thread and one 16-byte load of codes, for
// sources whose columns start on 16-byte boundaries.  Used for HBM sources
// and for pinned host memory read in place over the host link (the stream's
// direct path), where wide requests keep enough bytes in flight.
template <bool kBF16>
__global__ void __launch_bounds__(256) convert_x_wide_kernel(
    const int8_t* __restrict__ x8, int64_t ldx, int64_t n, int64_t k, int64_t npad,
    uint16_t* __restrict__ x16) {
  const int64_t per_col = npad / 16;
  const int64_t total = k * per_col;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = idx / per_col;
    const int64_t c0 = (idx - j * per_col) * 16;
    const int8_t* col = x8 + j * ldx;
    uint4 raw = make_uint4(0, 0, 0, 0);
    if (c0 + 16 <= n) {
      raw = *reinterpret_cast<const uint4*>(col + c0);
    } else if (c0 < n) {  // ragged end of the column: bytes, rows >= n stay zero
      uint32_t w[4] = {0, 0, 0, 0};
      for (int e = 0; e < 16 && c0 + e < n; ++e)
        w[e / 4] |= (uint32_t)(uint8_t)col[c0 + e] << (8 * (e % 4));
      raw = make_uint4(w[0], w[1], w[2], w[3]);
    }
    const uint32_t wv[4] = {raw.x, raw.y, raw.z, raw.w};
    uint32_t o[8];
#pragma unroll
    for (int e = 0; e < 16; e += 2) {
      const int a = (int)(int8_t)(wv[e / 4] >> (8 * (e % 4)));
      const int b = (int)(int8_t)(wv[e / 4] >> (8 * (e % 4 + 1)));
      const uint32_t va = code16<kBF16>(a);
      const uint32_t vb = code16<kBF16>(b);
      o[e / 2] = va | (vb << 16);
    }
    uint4* dst = reinterpret_cast<uint4*>(x16 + j * npad + c0);
    dst[0] = make_uint4(o[0], o[1], o[2], o[3]);
    dst[1] = make_uint4(o[4], o[5], o[6], o[7]);
  }
}

// The conversion of the next block beside a running solve, for sources whose
// columns start on 16-byte boundaries: up to kSideSms CTAs of 1024 threads,
// each thread with two 16-byte loads in flight (pinned host memory read over
// the host link needs bytes in flight).  A solve CTA (about 53.8K registers)
// and one of these (32K or more) never fit on one SM together, and the solve
// launch leaves as many SMs free as there are conversion CTAs, so the two
// kernels do not share SMs whichever starts first.
constexpr int kSideThreads = 1024;

template <bool kBF16>
__device__ __forceinline__ void convert16(uint4 raw, int64_t j, int64_t c0, int64_t npad,
                                          uint16_t* __restrict__ x16) {
  const uint32_t wv[4] = {raw.x, raw.y, raw.z, raw.w};
  uint32_t o[8];
#pragma unroll
  for (int e = 0; e < 16; e += 2) {
    const int a = (int)(int8_t)(wv[e / 4] >> (8 * (e % 4)));
    const int b = (int)(int8_t)(wv[e / 4] >> (8 * (e % 4 + 1)));
    o[e / 2] = code16<kBF16>(a) | (code16<kBF16>(b) << 16);
  }
  uint4* dst = reinterpret_cast<uint4*>(x16 + j * npad + c0);
  dst[0] = make_uint4(o[0], o[1], o[2], o[3]);
  dst[1] = make_uint4(o[4], o[5], o[6], o[7]);
}

template <bool kBF16>
__device__ __forceinline__ uint4 load16(const int8_t* __restrict__ x8, int64_t ldx, int64_t n,
                                        int64_t idx, int64_t per_col, int64_t* j, int64_t* c0) {
  *j = idx / per_col;
  *c0 = (idx - *j * per_col) * 16;
  const int8_t* col = x8 + *j * ldx;
  uint4 raw = make_uint4(0, 0, 0, 0);
  if (*c0 + 16 <= n) {
    raw = *reinterpret_cast<const uint4*>(col + *c0);
  } else if (*c0 < n) {  // ragged end of the column: bytes, rows >= n stay zero
    uint32_t w[4] = {0, 0, 0, 0};
    for (int e = 0; e < 16 && *c0 + e < n; ++e)
      w[e / 4] |= (uint32_t)(uint8_t)col[*c0 + e] << (8 * (e % 4));
    raw = make_uint4(w[0], w[1], w[2], w[3]);
  }
  return raw;
}

template <bool kBF16>
__global__ void __launch_bounds__(kSideThreads) convert_x_side_kernel(
    const int8_t* __restrict__ x8, int64_t ldx, int64_t n, int64_t k, int64_t npad,
    uint16_t* __restrict__ x16) {
  const int64_t per_col = npad / 16;
  const int64_t total = k * per_col;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += 2 * stride) {
    int64_t j0, c00, j1 = 0, c01 = 0;
    const uint4 r0 = load16<kBF16>(x8, ldx, n, idx, per_col, &j0, &c00);
    const bool two = idx + stride < total;
    uint4 r1 = make_uint4(0, 0, 0, 0);
    if (two) r1 = load16<kBF16>(x8, ldx, n, idx + stride, per_col, &j1, &c01);
    convert16<kBF16>(r0, j0, c00, npad, x16);
    if (two) convert16<kBF16>(r1, j1, c01, npad, x16);
  }
}

// The same output from 2-bit packed genotype columns (ldp bytes each; row i
// in bits 2 (i mod 4) .. 2 (i mod 4) + 1 of byte i / 4): the 8 rows of a
// thread are two packed bytes, so the block is read once, at a quarter of
// the int8 bytes, with no separate unpacking pass.
template <bool kBF16>
__global__ void convert_xp_kernel(const uint8_t* __restrict__ xp, int64_t ldp, int64_t n,
                                  int64_t k, int64_t npad, uint16_t* __restrict__ x16) {
  const int64_t per_col = npad / 8;
  const int64_t total = k * per_col;
  const int64_t nb = (n + 3) / 4;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = idx / per_col;
    const int64_t c0 = (idx - j * per_col) * 8;
    const int64_t b0 = c0 / 4;
    uint32_t w = 0;
    if (b0 < nb) w = xp[j * ldp + b0];
    if (b0 + 1 < nb) w |= (uint32_t)xp[j * ldp + b0 + 1] << 8;
    uint16_t v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int xi = (c0 + e < n) ? (int)((w >> (2 * e)) & 3u) : 0;
      v[e] = (uint16_t)code16<kBF16>(xi);
    }
    uint4 o;
    o.x = (uint32_t)v[0] | ((uint32_t)v[1] << 16);
    o.y = (uint32_t)v[2] | ((uint32_t)v[3] << 16);
    o.z = (uint32_t)v[4] | ((uint32_t)v[5] << 16);
    o.w = (uint32_t)v[6] | ((uint32_t)v[7] << 16);
    *reinterpret_cast<uint4*>(x16 + j * npad + c0) = o;
  }
}

template <bool kBF16>
__device__ __forceinline__ uint16_t to16(double v) {
  return kBF16 ? __bfloat16_as_ushort(__float2bfloat16_rn((float)v))
               : __half_as_ushort(__float2half_rn((float)v));
}
template <bool kBF16>
__device__ __forceinline__ double from16(uint16_t b) {
  return kBF16 ? (double)__bfloat162float(__ushort_as_bfloat16(b))
               : (double)__half2float(__ushort_as_half(b));
}

// Splits the part of each row of Z left of its diagonal block into S slices
// (see the file header); also writes u_r and the split diagonal blocks
// (k_rc, l_rc, s_r).
// One CTA per 32-row stripe; Z is read column-major (coalesced along rows) and
// the slices are written row-major through a shared-memory transpose.
template <bool kBF16>
__global__ void __launch_bounds__(256) split_kernel(const double* __restrict__ Z, int64_t ldz,
                                                    int64_t npad, int S, int bits, int naive,
                                                    int nG, uint16_t* __restrict__ tiles,
                                                    float* __restrict__ rowscale,
                                                    float* __restrict__ diagKL,
                                                    float* __restrict__ diagS) {
  __shared__ double red[8][33];
  __shared__ uint16_t sh[3][32][64 + 8];
  const int l = threadIdx.x % 32, w = threadIdx.x / 32;
  const int64_t r = (int64_t)blockIdx.x * 32 + l;
  const int64_t r0 = r - (r % kDiag);
  double m = 0.0;
  for (int64_t c = w; c < r0; c += 8) m = fmax(m, fabs(Z[r + c * ldz]));
  red[w][l] = m;
  __syncthreads();
  if (w == 0) {
    for (int v = 1; v < 8; ++v) m = fmax(m, red[v][l]);
    double u = 1.0;
    if (!naive && m > 0.0) {
      int e;
      frexp(m, &e);  // m < 2^e
      u = ldexp(1.0, e - bits);
    }
    red[0][l] = u;
    rowscale[r] = (float)u;
    double zd[kDiag], dm = 0.0;
#pragma unroll
    for (int q = 0; q < kDiag; ++q) {
      zd[q] = (r0 + q <= r) ? Z[r + (r0 + q) * ldz] : 0.0;
      dm = fmax(dm, fabs(zd[q]));
    }
    double sr = 0.0;
    if (dm > 0.0) {
      int e;
      frexp(dm, &e);  // dm < 2^e, so |k| <= 2^12
      sr = ldexp(1.0, e - 12);
    }
#pragma unroll
    for (int q = 0; q < kDiag; ++q) {
      const double k = sr > 0.0 ? rint(zd[q] / sr) : 0.0;
      diagKL[r * 8 + q] = (float)k;
      diagKL[r * 8 + 4 + q] = (float)(zd[q] - k * sr);
    }
    diagS[r] = (float)sr;
  }
  __syncthreads();
  const double inv_u = 1.0 / red[0][l];  // power of two: exact
  // The solve reads the rows of pair I = stripe / 256 up to column 256 (I + 1)
  // only; columns past that stay as the zeros the buffer was created with.
  // Chunks right of every row's diagonal block are zeros: no arithmetic.
  const int64_t stripe0 = (int64_t)blockIdx.x * 32;
  const int64_t cend = std::min<int64_t>(npad, (stripe0 / kPair + 1) * kPair);
  const int64_t czero = stripe0 + 31 - ((stripe0 + 31) % kDiag);  // largest r0 of the stripe
  for (int64_t c0 = 0; c0 < cend; c0 += 64) {
    if (c0 >= czero) {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int cc = w + 8 * e;
        sh[0][l][cc] = 0;
        sh[1][l][cc] = 0;
        sh[2][l][cc] = 0;
      }
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int cc = w + 8 * e;
        const int64_t c = c0 + cc;
        const double z = (c < r0) ? Z[r + c * ldz] * inv_u : 0.0;
        double h = naive ? from16<kBF16>(to16<kBF16>(z)) : rint(z);
        const double rem = z - h;
        const uint16_t s1 = to16<kBF16>(rem);
        const uint16_t s2 = to16<kBF16>(rem - from16<kBF16>(s1));
        sh[0][l][cc] = to16<kBF16>(h);
        sh[1][l][cc] = s1;
        sh[2][l][cc] = s2;
      }
    }
    __syncthreads();
    {
      // one 16-byte core-matrix row per thread, 8 threads per core matrix: a
      // warp writes 4 core matrices of one tile (512 contiguous bytes)
      const int r8 = threadIdx.x & 7, ch = (threadIdx.x >> 3) & 7, rl = (threadIdx.x >> 6) * 8 + r8;
      const int64_t row = stripe0 + rl;
      const int g = (int)(row / kPair), rr = (int)(row % kPair);
      const int64_t c = c0 + ch * 8;
      const int64_t nKB = npad / BK;
      for (int s = 0; s < S; ++s) {
        uint4 v;
        const uint16_t* src = &sh[s][rl][ch * 8];
        v.x = (uint32_t)src[0] | ((uint32_t)src[1] << 16);
        v.y = (uint32_t)src[2] | ((uint32_t)src[3] << 16);
        v.z = (uint32_t)src[4] | ((uint32_t)src[5] << 16);
        v.w = (uint32_t)src[6] | ((uint32_t)src[7] << 16);
        *reinterpret_cast<uint4*>(tiles + tile_index(s, g, c / BK, nG, nKB) * kTileElems +
                                  in_tile(rr, (int)(c % BK))) = v;
      }
    }
    __syncthreads();
  }
}

// W = Z^T Wt (= M^{-1} [X_L | y]), binary64: W(c, q) = sum_{r >= c} Z(r, c) Wt(r, q).
// One CTA per 64 columns c; Z is read column-major (coalesced along r).
__global__ void __launch_bounds__(256) wtrans_kernel(const double* __restrict__ Z, int64_t ldz,
                                                     int64_t npad, const double* __restrict__ Wt,
                                                     int64_t ldw, int p, double* __restrict__ W) {
  __shared__ double Zs[64][65];              // Zs[rr][cc]
  __shared__ double Rs[64][kMaxP + 1];       // Rs[rr][q]
  const int64_t c0 = (int64_t)blockIdx.x * 64;
  const int tid = threadIdx.x;
  const int cc = tid % 64, qg = tid / 64;
  double acc[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) acc[t] = 0.0;
  for (int64_t r0 = c0; r0 < npad; r0 += 64) {
    for (int idx = tid; idx < 64 * 64; idx += 256) {
      const int rr = idx % 64, c = idx / 64;
      Zs[rr][c] = Z[(r0 + rr) + (c0 + c) * ldz];
    }
    for (int idx = tid; idx < 64 * p; idx += 256) {
      const int rr = idx % 64, q = idx / 64;
      Rs[rr][q] = Wt[(r0 + rr) + (int64_t)q * ldw];
    }
    __syncthreads();
    for (int rr = 0; rr < 64; ++rr) {
      const double z = Zs[rr][cc];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int q = qg + 4 * t;
        if (q < p) acc[t] = fma(z, Rs[rr][q], acc[t]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int q = qg + 4 * t;
    if (q < p) W[(c0 + cc) + (int64_t)q * npad] = acc[t];
  }
}

// Splits row q of W^T (column q of W) into the slices of A-operand row npad + q,
// with its own scale u = 2^(E - bits) over the whole row.  One CTA per q.
template <bool kBF16>
__global__ void __launch_bounds__(256) split_w_kernel(const double* __restrict__ W, int64_t npad,
                                                      int bits, int naive, int nG,
                                                      uint16_t* __restrict__ tiles,
                                                      float* __restrict__ rowscale) {
  __shared__ double red[256];
  const int q = blockIdx.x;
  const double* w = W + (int64_t)q * npad;
  double m = 0.0;
  for (int64_t c = threadIdx.x; c < npad; c += blockDim.x) m = fmax(m, fabs(w[c]));
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  m = red[0];
  double u = 1.0;
  if (!naive && m > 0.0) {
    int e;
    frexp(m, &e);
    u = ldexp(1.0, e - bits);
  }
  const int64_t row = npad + q;
  if (threadIdx.x == 0) rowscale[row] = (float)u;
  const double inv_u = 1.0 / u;
  // row q of the W^T group (the last 256-row group of the tiles)
  const int64_t nKB = npad / BK;
  const int gW = nG - 1;
  for (int64_t c = threadIdx.x; c < npad; c += blockDim.x) {
    const double z = w[c] * inv_u;
    const double h = naive ? from16<kBF16>(to16<kBF16>(z)) : rint(z);
    const double rem = z - h;
    const uint16_t s1 = to16<kBF16>(rem);
    const uint16_t s2 = to16<kBF16>(rem - from16<kBF16>(s1));
    const int o = in_tile(q, (int)(c % BK));
    tiles[tile_index(0, gW, c / BK, nG, nKB) * kTileElems + o] = to16<kBF16>(h);
    tiles[tile_index(1, gW, c / BK, nG, nKB) * kTileElems + o] = s1;
    tiles[tile_index(2, gW, c / BK, nG, nKB) * kTileElems + o] = s2;
  }
}

// Looked up once; the initialisation of a function-local static is
// thread-safe, so plans created on several host threads share it.
PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() {
    cudaDriverEntryPointQueryResult q;
    void* ptr = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return static_cast<PFN_cuTensorMapEncodeTiled_v12000>(nullptr);
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  }();
  return fn;
}

}  // namespace

struct MixedState {
  int64_t n = 0, npad = 0, kmax = 0;
  int p = 1, S = 3, stages = 3, bits = 7;
  bool bf16 = true;
  bool naive = false;
  int num_sms = 1;
  uint16_t* slices = nullptr;  // 3 planes of nG x nKB tiles (see kTileElems)
  int nG = 1;                  // 256-row groups: row pairs plus the W^T group
  int64_t nKB = 1;             // 32-deep K stages per row
  float* rowscale = nullptr;   // npad + 128
  float* diagKL = nullptr;     // npad x 8: k[4], l[4] of the diagonal blocks
  float* diagS = nullptr;      // npad
  double* Wm = nullptr;        // W = M^{-1} [X_L | y], npad x p
  uint16_t* x16 = nullptr;     // kmax x npad
  ProblemDesc desc;            // host copy (buffers filled in by the plan per call)
  MapSet maps;                 // this problem's maps in slot 0 (single-problem launches)
  ProblemDesc* d_desc = nullptr;  // device copy used by single-problem launches
  double* d_Pbr = nullptr;     // buffers the device copy currently points to
  double* d_Glin = nullptr;
  // Genotype operand buffer 1 (mixed_add_buffer): a stream converts block j+1
  // into one buffer beside the solve of block j from the other.
  uint16_t* x16b = nullptr;
  ProblemDesc descb;
  MapSet mapsb;
  ProblemDesc* d_descb = nullptr;
  double* d_Pbrb = nullptr;
  double* d_Glinb = nullptr;
  KConst kc{};
  size_t smem = 0;
};

struct MixedBatch {
  std::vector<MixedState*> states;  // launch order (largest n first)
  std::vector<int> order;           // states[i] = input[order[i]]
  MapSet maps;                      // slot i: the maps of states[i]
  ProblemDesc* d_desc = nullptr;
  std::vector<double*> Pbr, Glin;
};

namespace {

size_t smem_bytes(int S, int stages) {
  const uint32_t stage_bytes = (uint32_t)S * kSliceBytes + kXBytes;
  const uint32_t epi = 2u * kRowsBytes;
  const uint32_t bars = 8 * (2 * stages + 3) + 16;
  return (size_t)stages * stage_bytes + epi + bars + 1024;
}

bool g_attr_done = false;

}  // namespace

size_t tiles_bytes(int64_t npad) {
  const int64_t nI = npad / BM;
  const int64_t nG = (nI + 1) / 2 + 1;
  return (size_t)3 * nG * (npad / BK) * kTileElems * 2;
}

size_t mixed_footprint(int64_t n, int64_t npad, int p, int64_t kmax, int split_terms) {
  (void)n;
  (void)split_terms;
  size_t b = tiles_bytes(npad);
  b += (size_t)(npad + 128) * 4 + (size_t)npad * (9 * 4 + 8 * p);
  b += (size_t)kmax * npad * 2 + sizeof(ProblemDesc);
  return b;
}

const char* mixed_last_error() { return g_err.c_str(); }

int mixed_diag_block(const MixedState*) { return kDiag; }

void mixed_free(MixedState* ms) {
  if (!ms) return;
  cudaFree(ms->slices);
  cudaFree(ms->rowscale);
  cudaFree(ms->diagKL);
  cudaFree(ms->diagS);
  cudaFree(ms->Wm);
  cudaFree(ms->x16);
  cudaFree(ms->d_desc);
  cudaFree(ms->x16b);
  cudaFree(ms->d_descb);
  delete ms;
}

namespace {

// The tensor map of a genotype operand buffer (kmax x npad 16-bit, boxes of
// BK x BN, 64-byte swizzle) into slot 0 of maps.
bool encode_x16(const MixedState* ms, uint16_t* x16, MapSet* maps) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
  if (!enc) return false;
  const CUtensorMapDataType dt =
      ms->bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  cuuint64_t dims[2] = {(cuuint64_t)ms->npad, (cuuint64_t)ms->kmax};
  cuuint64_t strides[1] = {(cuuint64_t)ms->npad * 2};
  cuuint32_t box[2] = {BK, BN};
  cuuint32_t es[2] = {1, 1};
  return enc(&maps->tmB[0], dt, 2, x16, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

gls_status_t mixed_add_buffer(MixedState* ms) {
  if (ms->x16b) return GLS_OK;
  const size_t cells = (size_t)ms->kmax * ms->npad;
  if (cudaMalloc(&ms->x16b, cells * 2) != cudaSuccess ||
      cudaMalloc(&ms->d_descb, sizeof(ProblemDesc)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(ms->x16b);
    cudaFree(ms->d_descb);
    ms->x16b = nullptr;
    ms->d_descb = nullptr;
    g_err = "cudaMalloc of the second genotype operand buffer failed";
    return GLS_ERR_OOM;
  }
  ms->descb = ms->desc;
  ms->descb.x16 = ms->x16b;
  ms->d_Pbrb = ms->d_Glinb = nullptr;  // the device copy is written on first use
  memset(&ms->mapsb, 0, sizeof(ms->mapsb));
  if (!encode_x16(ms, ms->x16b, &ms->mapsb)) {
    g_err = "tensor map encode (second genotype buffer) failed";
    return GLS_ERR_CUDA;
  }
  return GLS_OK;
}

size_t mixed_buffer_bytes(int64_t npad, int64_t kmax) { return (size_t)kmax * npad * 2; }

gls_status_t mixed_create(MixedState** out, int64_t n, int64_t npad, int p, int64_t kmax,
                          int precision, int split_terms, uint32_t flags, int32_t wait_limit_us,
                          cudaStream_t st) {
  *out = nullptr;
  if (npad % BM != 0) {
    g_err = "npad must be a multiple of 128";
    return GLS_ERR_INVALID_ARG;
  }
  if (npad > (int64_t)1 << 24 || kmax > ((int64_t)1 << 31) - BN) {
    g_err = "problem too large for 32-bit TMA coordinates";
    return GLS_ERR_INVALID_ARG;
  }
  MixedState* ms = new MixedState();
  ms->n = n;
  ms->npad = npad;
  ms->kmax = kmax;
  ms->p = p;
  ms->nG = (int)((npad / BM + 1) / 2 + 1);
  ms->nKB = npad / BK;
  // BF16 slices below kBf16MinN rows fall short of 1e-6 on b_i; FP16 slices
  // (three more bits per slice, same tensor rate) meet it at every size
  ms->bf16 = (precision == GLS_PREC_MIXED_BF16) && n >= kBf16MinN;
  ms->S = split_terms ? split_terms : 3;
  ms->bits = ms->bf16 ? 7 : 10;
  ms->naive = (flags & GLS_FLAG_NAIVE_SPLIT) != 0;
  auto fail = [&](gls_status_t s, const char* msg) {
    g_err = msg;
    mixed_free(ms);
    return s;
  };
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&ms->num_sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t rows = (size_t)npad + 128;
  if (cudaMalloc(&ms->slices, tiles_bytes(npad)) != cudaSuccess ||
      cudaMalloc(&ms->rowscale, rows * 4) != cudaSuccess ||
      cudaMalloc(&ms->diagKL, (size_t)npad * 8 * 4) != cudaSuccess ||
      cudaMalloc(&ms->diagS, (size_t)npad * 4) != cudaSuccess ||
      cudaMalloc(&ms->Wm, (size_t)npad * p * 8) != cudaSuccess ||
      cudaMalloc(&ms->x16, (size_t)kmax * npad * 2) != cudaSuccess ||
      cudaMalloc(&ms->d_desc, sizeof(ProblemDesc)) != cudaSuccess) {
    cudaGetLastError();
    return fail(GLS_ERR_OOM, "cudaMalloc of the mixed-precision operands failed");
  }
  // the W^T block's unused rows stay zero
  if (cudaMemsetAsync(ms->slices, 0, tiles_bytes(npad), st) != cudaSuccess ||
      cudaMemsetAsync(ms->rowscale, 0, rows * 4, st) != cudaSuccess) {
    cudaGetLastError();
    return fail(GLS_ERR_CUDA, "cudaMemset of the operand slices failed");
  }
  int stages = 6;
  while (stages > 2 && smem_bytes(ms->S, stages) > (size_t)kMaxDynSmem) --stages;
  if (smem_bytes(ms->S, stages) > (size_t)kMaxDynSmem)
    return fail(GLS_ERR_UNSUPPORTED, "shared-memory budget exceeded for this split");
  ms->stages = stages;
  ms->smem = smem_bytes(ms->S, stages);
  KConst& kc = ms->kc;
  kc.S = ms->S;
  kc.stages = stages;
  kc.wait_ns = wait_limit_us > 0 ? (uint64_t)wait_limit_us * 1000ull : kWaitLimitNs;
  kc.stage_bytes = (uint32_t)ms->S * kSliceBytes + kXBytes;
  kc.off_rows = (uint32_t)stages * kc.stage_bytes;
  kc.off_bar = kc.off_rows + 2u * kRowsBytes;
  if (!g_attr_done) {
    if (cudaFuncSetAttribute(trsm_gram_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kMaxDynSmem) != cudaSuccess) {
      cudaGetLastError();
      return fail(GLS_ERR_CUDA, "cudaFuncSetAttribute (shared memory) failed");
    }
    g_attr_done = true;
  }
  PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
  if (!enc) return fail(GLS_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is not available");
  const CUtensorMapDataType dt =
      ms->bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  ProblemDesc& d = ms->desc;
  memset(&d, 0, sizeof(d));
  memset(&ms->maps, 0, sizeof(ms->maps));
  (void)dt;
  if (!encode_x16(ms, ms->x16, &ms->maps))
    return fail(GLS_ERR_CUDA, "tensor map encode (genotypes) failed");
  d.tiles = ms->slices;
  d.nKB = ms->nKB;
  d.nG = ms->nG;
  d.x16 = ms->x16;
  d.bf16 = ms->bf16 ? 1 : 0;
  d.rowscale = ms->rowscale;
  d.diagKL = ms->diagKL;
  d.diagS = ms->diagS;
  d.npad = npad;
  d.nI = (int)(npad / BM);
  d.p = p;
  d.idesc = umma_idesc_f16(BN, kPair, ms->bf16);
  d.idesc_half = umma_idesc_f16(BN, BM, ms->bf16);
  d.idesc_w = umma_idesc_f16(BN, 32 * ms->S, ms->bf16);
  *out = ms;
  return GLS_OK;
}

double* mixed_w_buffer(MixedState* ms) { return ms->Wm; }

gls_status_t mixed_prepare(MixedState* ms, const double* Z, int64_t ldz, const double* Wt,
                           int64_t ldw, bool new_factor, bool w_ready, cudaStream_t st) {
  if (new_factor) {
    const unsigned grid = (unsigned)(ms->npad / 32);
    if (ms->bf16)
      split_kernel<true><<<grid, 256, 0, st>>>(Z, ldz, ms->npad, ms->S, ms->bits, ms->naive,
                                               ms->nG, ms->slices, ms->rowscale, ms->diagKL,
                                               ms->diagS);
    else
      split_kernel<false><<<grid, 256, 0, st>>>(Z, ldz, ms->npad, ms->S, ms->bits, ms->naive,
                                                ms->nG, ms->slices, ms->rowscale, ms->diagKL,
                                                ms->diagS);
  }
  if (!w_ready)
    wtrans_kernel<<<(unsigned)(ms->npad / 64), 256, 0, st>>>(Z, ldz, ms->npad, Wt, ldw, ms->p,
                                                             ms->Wm);
  if (ms->bf16)
    split_w_kernel<true><<<(unsigned)ms->p, 256, 0, st>>>(ms->Wm, ms->npad, ms->bits, ms->naive,
                                                         ms->nG, ms->slices, ms->rowscale);
  else
    split_w_kernel<false><<<(unsigned)ms->p, 256, 0, st>>>(ms->Wm, ms->npad, ms->bits, ms->naive,
                                                          ms->nG, ms->slices, ms->rowscale);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_err = std::string("mixed prepare: ") + cudaGetErrorString(e);
    return GLS_ERR_CUDA;
  }
  return GLS_OK;
}

cudaError_t mixed_convert(MixedState* ms, const int8_t* xr, int64_t ldxr, int64_t k,
                          cudaStream_t st, int buf, int side_ctas) {
  if (k <= 0) return cudaSuccess;
  if (buf != 0 && !ms->x16b) return cudaErrorInvalidValue;
  uint16_t* x16 = buf ? ms->x16b : ms->x16;
  const bool wide = ((uintptr_t)xr % 16) == 0 && (ldxr % 16) == 0;
  if (side_ctas > 0) {
    if (!wide) return cudaErrorInvalidValue;
    const unsigned grid = (unsigned)std::min(side_ctas, kSideSms);
    if (ms->bf16)
      convert_x_side_kernel<true>
          <<<grid, kSideThreads, 0, st>>>(xr, ldxr, ms->n, k, ms->npad, x16);
    else
      convert_x_side_kernel<false>
          <<<grid, kSideThreads, 0, st>>>(xr, ldxr, ms->n, k, ms->npad, x16);
    return cudaGetLastError();
  }
  if (wide) {
    const int64_t work = k * (ms->npad / 16);
    const unsigned grid =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(work, 256), ms->num_sms * 8));
    if (ms->bf16)
      convert_x_wide_kernel<true><<<grid, 256, 0, st>>>(xr, ldxr, ms->n, k, ms->npad, x16);
    else
      convert_x_wide_kernel<false><<<grid, 256, 0, st>>>(xr, ldxr, ms->n, k, ms->npad, x16);
    return cudaGetLastError();
  }
  const int64_t work = k * (ms->npad / 8);
  const unsigned cgrid = (unsigned)std::min<int64_t>(ceil_div(work, 256), 65535 * 4);
  if (ms->bf16)
    convert_x_kernel<true><<<cgrid, 256, 0, st>>>(xr, ldxr, ms->n, k, ms->npad, x16);
  else
    convert_x_kernel<false><<<cgrid, 256, 0, st>>>(xr, ldxr, ms->n, k, ms->npad, x16);
  return cudaGetLastError();
}

cudaError_t mixed_convert_packed(MixedState* ms, const uint8_t* xp, int64_t ldp, int64_t k,
                                 cudaStream_t st) {
  if (k <= 0) return cudaSuccess;
  const int64_t work = k * (ms->npad / 8);
  const unsigned cgrid = (unsigned)std::min<int64_t>(ceil_div(work, 256), 65535 * 4);
  if (ms->bf16)
    convert_xp_kernel<true><<<cgrid, 256, 0, st>>>(xp, ldp, ms->n, k, ms->npad, ms->x16);
  else
    convert_xp_kernel<false><<<cgrid, 256, 0, st>>>(xp, ldp, ms->n, k, ms->npad, ms->x16);
  return cudaGetLastError();
}

namespace {

// (row-block pairs + the W^T block) x SNP tiles
int items_of(const MixedState* ms, int64_t k) {
  return (int)(ceil_div(ms->npad / BM, 2) + 1) * (int)ceil_div(k, BN);
}

cudaError_t launch(const MixedState* ms0, const ProblemDesc* d_desc, const RunParams& run,
                   const MapSet& maps, int* flags, cudaStream_t st, int max_ctas = 0) {
  KConst kc = ms0->kc;
  kc.flags = flags;
  const int ctas = max_ctas > 0 ? std::min(max_ctas, ms0->num_sms) : ms0->num_sms;
  const int grid = std::min(ctas, std::max(run.total, 1));
  trsm_gram_mixed_kernel<<<grid, kThreads, ms0->smem, st>>>(d_desc, run, kc, maps);
  return cudaGetLastError();
}

}  // namespace

cudaError_t mixed_trsm_gram(MixedState* ms, const int8_t* xr, int64_t ldxr, int64_t k,
                            double* Pbr, double* Glin, int64_t ldp, int* flags, cudaStream_t st,
                            int buf, int side_sms) {
  (void)xr;
  (void)ldxr;
  if (k <= 0) return cudaSuccess;
  if (buf != 0 && !ms->x16b) return cudaErrorInvalidValue;
  ProblemDesc& d = buf ? ms->descb : ms->desc;
  ProblemDesc* dd = buf ? ms->d_descb : ms->d_desc;
  double*& dPbr = buf ? ms->d_Pbrb : ms->d_Pbr;
  double*& dGlin = buf ? ms->d_Glinb : ms->d_Glin;
  if (Pbr != dPbr || Glin != dGlin || d.ldp != ldp) {
    d.Pbr = Pbr;
    d.Glin = Glin;
    d.ldp = ldp;
    cudaError_t e = cudaMemcpyAsync(dd, &d, sizeof(ProblemDesc), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);  // the host copy may change on a later call
    if (e != cudaSuccess) return e;
    dPbr = Pbr;
    dGlin = Glin;
  }
  RunParams run;
  memset(&run, 0, sizeof(run));
  run.nprob = 1;
  run.group = kDefaultGroup;
  run.k[0] = k;
  run.nJ[0] = (int)ceil_div(k, BN);
  run.item_begin[0] = 0;
  run.total = run.item_begin[1] = items_of(ms, k);
  return launch(ms, dd, run, buf ? ms->mapsb : ms->maps, flags, st,
                side_sms > 0 ? ms->num_sms - side_sms : 0);
}

int mixed_split_terms(const MixedState* ms) { return ms->S; }
bool mixed_is_bf16(const MixedState* ms) { return ms->bf16; }
int64_t mixed_n(const MixedState* ms) { return ms->n; }

gls_status_t mixed_batch_create(MixedState* const* states, const double* const* Pbr,
                                const double* const* Glin, const int64_t* ldp, int count,
                                MixedBatch** out) {
  *out = nullptr;
  if (count < 1 || count > kMaxBatch) {
    g_err = "batch size must be in [1, " + std::to_string(kMaxBatch) + "]";
    return GLS_ERR_INVALID_ARG;
  }
  for (int i = 1; i < count; ++i)
    if (states[i]->S != states[0]->S) {
      g_err = "all plans of a batch need the same split_terms";
      return GLS_ERR_INVALID_ARG;
    }
  MixedBatch* b = new MixedBatch();
  b->order.resize(count);
  for (int i = 0; i < count; ++i) b->order[i] = i;
  std::stable_sort(b->order.begin(), b->order.end(),
                   [&](int a, int c) { return states[a]->n > states[c]->n; });
  std::vector<ProblemDesc> h(count);
  memset(&b->maps, 0, sizeof(b->maps));
  for (int i = 0; i < count; ++i) {
    const int o = b->order[i];
    b->states.push_back(states[o]);
    b->maps.tmB[i] = states[o]->maps.tmB[0];
    h[i] = states[o]->desc;
    h[i].Pbr = const_cast<double*>(Pbr[o]);
    h[i].Glin = const_cast<double*>(Glin[o]);
    h[i].ldp = ldp[o];
  }
  if (cudaMalloc(&b->d_desc, sizeof(ProblemDesc) * count) != cudaSuccess ||
      cudaMemcpy(b->d_desc, h.data(), sizeof(ProblemDesc) * count, cudaMemcpyHostToDevice) !=
          cudaSuccess) {
    cudaGetLastError();
    cudaFree(b->d_desc);
    delete b;
    g_err = "batch descriptor allocation failed";
    return GLS_ERR_OOM;
  }
  *out = b;
  return GLS_OK;
}

void mixed_batch_free(MixedBatch* b) {
  if (!b) return;
  cudaFree(b->d_desc);
  delete b;
}

cudaError_t mixed_batch_run(MixedBatch* b, const int64_t* k, int group, int* flags,
                            cudaStream_t st) {
  RunParams run;
  memset(&run, 0, sizeof(run));
  const int count = (int)b->states.size();
  run.nprob = count;
  run.group = group > 0 ? group : kDefaultGroup;
  int total = 0;
  for (int i = 0; i < count; ++i) {
    const int o = b->order[i];
    run.k[i] = k[o];
    run.nJ[i] = (int)ceil_div(k[o], BN);
    run.item_begin[i] = total;
    total += k[o] > 0 ? items_of(b->states[i], k[o]) : 0;
  }
  run.item_begin[count] = total;
  run.total = total;
  if (total == 0) return cudaSuccess;
  return launch(b->states[0], b->d_desc, run, b->maps, flags, st);
}

}  // namespace gls
