// mixed.cuh -- interface of the mixed-precision blocked triangular solve (tcgen05).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gls_gb300.h"

namespace gls {

struct MixedState;

// GLS_PREC_MIXED_BF16 plans with fewer rows use FP16 operand slices.
constexpr int64_t kBf16MinN = 2048;

// Device bytes the mixed path adds to a plan.
size_t mixed_footprint(int64_t n, int64_t npad, int p, int64_t kmax, int split_terms);

// Allocates the operand slices and encodes the TMA descriptors.  The solve's
// pipeline waits give up after wait_limit_us microseconds (0: one second).
gls_status_t mixed_create(MixedState** out, int64_t n, int64_t npad, int p, int64_t kmax,
                          int precision, int split_terms, uint32_t flags, int32_t wait_limit_us,
                          cudaStream_t st);
void mixed_free(MixedState* ms);
const char* mixed_last_error();

// After the FP64 setup: splits the off-diagonal part of Z = L^{-1} into
// tensor-core slices and keeps its diagonal blocks as exact FP32 splits
// (integer part and low part per entry; only when new_factor),
// then forms W = Z^T [X~_L | y~] = M^{-1} [X_L | y] in binary64 and splits W^T
// into the extra row block of the A operand.
// With w_ready, W has already been written to mixed_w_buffer(ms) by the caller.
gls_status_t mixed_prepare(MixedState* ms, const double* Z, int64_t ldz, const double* Wt,
                           int64_t ldw, bool new_factor, bool w_ready, cudaStream_t st);
// Device buffer (npad x p, column-major) holding W = M^{-1} [X_L | y].
double* mixed_w_buffer(MixedState* ms);

// Adds genotype operand buffer 1 (mixed_buffer_bytes more device memory), so
// that a stream can convert block j+1 into one buffer beside the solve of
// block j from the other.  OOM leaves the state usable with buffer 0 alone.
gls_status_t mixed_add_buffer(MixedState* ms);
size_t mixed_buffer_bytes(int64_t npad, int64_t kmax);
// SMs a conversion beside a solve occupies (reading pinned host memory over
// the host link).
constexpr int kSideSms = 8;

// One block, step 1: int8 genotypes -> the 16-bit operand layout read by TMA,
// into operand buffer buf.  With side_ctas > 0 the conversion runs as that
// many CTAs of 1024 threads, meant to run beside a solve launched with
// side_sms = side_ctas (columns on 16-byte boundaries only).
cudaError_t mixed_convert(MixedState* ms, const int8_t* xr, int64_t ldxr, int64_t k,
                          cudaStream_t st, int buf = 0, int side_ctas = 0);
// The same from 2-bit packed genotype columns (ldp bytes each, four codes a byte).
cudaError_t mixed_convert_packed(MixedState* ms, const uint8_t* xp, int64_t ldp, int64_t k,
                                 cudaStream_t st);
// One block, step 2: the persistent tcgen05 solve + Gram epilogue.  Writes the
// S_BR partials Pbr[I][j] (I < npad/128) and the linear Gram entries
// Glin[q][j] (q < p-1: S_BL, q = p-1: b_B), j < k, leading dimension ldp.
// The solve reads operand buffer buf; side_sms > 0 leaves that many SMs free
// for a conversion running beside it.
cudaError_t mixed_trsm_gram(MixedState* ms, const int8_t* xr, int64_t ldxr, int64_t k,
                            double* Pbr, double* Glin, int64_t ldp, int* flags,
                            cudaStream_t st, int buf = 0, int side_sms = 0);

// Size of the diagonal blocks kept out of the tensor-core slices.
int mixed_diag_block(const MixedState* ms);
int mixed_split_terms(const MixedState* ms);
bool mixed_is_bf16(const MixedState* ms);
int64_t mixed_n(const MixedState* ms);

// Several problems in one persistent launch.  Pbr / Glin / ldp are each
// problem's partial buffers (as for mixed_trsm_gram); all states need the same
// split (BF16 and FP16 operands may be mixed).  The genotypes of each problem must have been
// converted (mixed_convert) on the launch stream before mixed_batch_run.
struct MixedBatch;
gls_status_t mixed_batch_create(MixedState* const* states, const double* const* Pbr,
                                const double* const* Glin, const int64_t* ldp, int count,
                                MixedBatch** out);
void mixed_batch_free(MixedBatch* b);
// k[i]: SNPs of problem i in this launch (input order); group: row blocks per
// rasterization group (0 = default).
cudaError_t mixed_batch_run(MixedBatch* b, const int64_t* k, int group, int* flags,
                            cudaStream_t st);

}  // namespace gls
