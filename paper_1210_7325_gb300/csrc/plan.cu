// plan.cu -- the C ABI of include/gls_gb300.h: plan objects, the setup phase,
// one block of the SNP loop, and the double-buffered stream of Alg. 8.
#include <errno.h>
#include <fcntl.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "factor_tc.cuh"
#include "gls_gb300.h"
#include "mixed.cuh"
#include "variants.cuh"

namespace {

thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

#define GLS_CUDA(expr)                                                          \
  do {                                                                          \
    cudaError_t e_ = (expr);                                                    \
    if (e_ != cudaSuccess) {                                                    \
      set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                __LINE__);                                                      \
      return GLS_ERR_CUDA;                                                      \
    }                                                                           \
  } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) ok = true;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

enum class Mem { Device, Pinned, Pageable };

// Where p lives; for pinned host memory *dev (if given) receives the address
// kernels use for it (the runtime's device pointer of the mapping).
Mem classify(const void* p, const void** dev = nullptr) {
  if (dev) *dev = nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return Mem::Pageable;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return Mem::Device;
  if (a.type == cudaMemoryTypeHost) {
    if (dev) *dev = a.devicePointer;
    return Mem::Pinned;
  }
  return Mem::Pageable;
}

}  // namespace

namespace gls {
void set_last_error_text(const char* msg) { g_last_error = msg ? msg : ""; }
}  // namespace gls

namespace {
struct Capture;
struct ReplayCache;
}  // namespace

struct gls_plan {
  gls_plan_desc_t desc{};
  int device = 0;
  int64_t n = 0, npad = 0, kmax = 0;
  int p = 1;
  int t = 1;                // phenotypes the plan holds (desc.phenotypes)
  int t_active = 1;         // phenotypes of the last gls_factor
  int nw = 1;               // columns of [X_L | Y]: p - 1 + t
  int precision = GLS_PREC_FP64;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t ev_loaded[2]{}, ev_computed[2]{}, ev_stored[2]{}, ev_staged[2]{};
  // mixed streams reading pinned int8 in place: block j+1 is converted on cvt
  // into operand buffer (j+1) % 2 beside the solve of block j (first such call)
  cudaStream_t cvt = nullptr;
  cudaEvent_t ev_conv[2]{};

  double* A = nullptr;      // L, npad x npad
  double* Z = nullptr;      // L^{-1}, npad x npad
  double* Wrhs = nullptr;   // [X_L | Y], npad x nw
  double* Wt = nullptr;     // [X~_L | Y~], npad x nw
  double* gram = nullptr;   // nw x nw
  double* RTL = nullptr;    // (p-1) x (p-1)
  double* zT = nullptr;     // (p-1) x t
  int* flags = nullptr;     // kFlagCount
  int* h_flags = nullptr;   // pinned read-back of flags (an async copy the host can wait on)
  int8_t* xr[2]{};          // device staging of X_R blocks (ld = n)
  double* bdev[2]{};        // p x (t kmax)
  int32_t* sdev[2]{};       // kmax
  double* partials = nullptr;
  int64_t ldp = 0;
  int nI = 0;               // row blocks of the active path
  int8_t* h_xr[2]{};        // pinned staging for pageable inputs
  uint8_t* xp[2]{};         // device staging of 2-bit packed blocks (first packed call)
  uint8_t* h_xp[2]{};       // pinned staging for pageable packed inputs
  double* h_b[2]{};
  int32_t* h_s[2]{};
  uint8_t* h_ring[3]{};     // pinned slots of the file reader (first gls_solve_file)
  uint8_t* d_ring[3]{};     // their device addresses
  size_t ring_bytes = 0;
  cudaEvent_t ev_ring[3]{};
  gls::MixedState* mixed = nullptr;
  bool tc = false;          // factor on the tensor cores (exact slices)
  gls::TcFactor* tcf = nullptr;
  // device-time accounting (gls_plan_set_timing / gls_plan_stats)
  struct Slot {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
    double ms = 0.0;
    int64_t launches = 0;
    int64_t bytes = 0;  // copies only
  };
  bool timing = false;
  Slot t_trsm, t_convert, t_solve, t_factor, t_h2d, t_d2h;
  int64_t launches = 0;
  std::vector<cudaEvent_t> event_pool;
  bool has_factor = false;  // L and Z valid
  bool has_xl = false;      // X_L staged
  bool factored = false;    // ready for solves
  Capture* cap = nullptr;   // set while a launch sequence is being captured
  ReplayCache* replays = nullptr;  // captured launch sequences of this plan
};

namespace {

cudaEvent_t pool_event(gls_plan* pl) {
  if (!pl->event_pool.empty()) {
    cudaEvent_t e = pl->event_pool.back();
    pl->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// ------------------------------------------------------------------ CUDA graphs
// A launch sequence that repeats with the same arguments is captured as a CUDA
// graph the second time it is seen and replayed from then on: the factor of M
// on a plan (about 1500 launches at n = 10^4), one block of the SNP loop, one
// batched round.  The first run is eager, so one-off sequences (the rounds of a
// serving loop) cost no instantiation and first-use setup stays outside any
// capture.  Timing brackets inside a captured sequence become event-record
// nodes that get fresh events at every replay.
struct Capture {
  struct Mark {
    cudaEvent_t e0, e1;
    gls_plan::Slot* slot;
  };
  std::vector<cudaEvent_t> spare;  // created before the capture began
  std::vector<cudaEvent_t> used;
  std::vector<Mark> marks;
  cudaEvent_t take() {
    if (spare.empty()) return nullptr;
    cudaEvent_t e = spare.back();
    spare.pop_back();
    used.push_back(e);
    return e;
  }
};

struct Replay {
  struct Mark {
    cudaGraphNode_t n0 = nullptr, n1 = nullptr;
    gls_plan::Slot* slot = nullptr;
  };
  uint64_t key = 0, used = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> events;  // the placeholders the graph's event-record nodes name
  int64_t launches = 0;
  ~Replay() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (cudaEvent_t e : events) cudaEventDestroy(e);
  }
};

struct ReplayCache {
  static constexpr size_t kMaxGraphs = 48;  // least recently used beyond this are dropped
  static constexpr size_t kMaxSeen = 256;
  std::vector<std::unique_ptr<Replay>> items;
  std::vector<uint64_t> seen;  // keys run eagerly once
  uint64_t clock = 0;
  bool enabled = true;
};

// FNV-1a over 64-bit words.
struct KeyHash {
  uint64_t h = 1469598103934665603ull;
  KeyHash& operator<<(uint64_t v) {
    for (int i = 0; i < 8; ++i) {
      h ^= (v >> (8 * i)) & 0xFFu;
      h *= 1099511628211ull;
    }
    return *this;
  }
  KeyHash& operator<<(const void* p) { return *this << (uint64_t)(uintptr_t)p; }
};

// Brackets one kernel (or phase) with events on the plan's stream when timing
// is on; inside a capture the events become event-record nodes of the graph.
struct Timed {
  gls_plan* pl;
  gls_plan::Slot* slot;
  Capture* cap;
  cudaStream_t st;
  cudaEvent_t e0 = nullptr;
  // on pl->stream (inside a capture when one is open), or on `side`, a stream
  // that is never captured
  Timed(gls_plan* p, gls_plan::Slot* s, cudaStream_t side = nullptr)
      : pl(p), slot(s), cap(side ? nullptr : p->cap), st(side ? side : p->stream) {
    if (!pl->timing) return;
    e0 = cap ? cap->take() : pool_event(pl);
    if (e0) record(e0);
  }
  void record(cudaEvent_t e) {
    if (cap) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else cudaEventRecord(e, st);
  }
  void finish() {
    if (!e0) return;
    cudaEvent_t e1 = cap ? cap->take() : pool_event(pl);
    if (!e1) {
      if (!cap) pl->event_pool.push_back(e0);
    } else {
      record(e1);
      if (cap) cap->marks.push_back({e0, e1, slot});
      else slot->pending.emplace_back(e0, e1);
    }
    e0 = nullptr;
  }
  ~Timed() { finish(); }
};

gls_status_t launch_replay(gls_plan* pl, Replay& r) {
  if (pl->timing) {
    for (Replay::Mark& m : r.marks) {
      cudaEvent_t e0 = pool_event(pl), e1 = pool_event(pl);
      if (!e0 || !e1) {
        if (e0) pl->event_pool.push_back(e0);
        if (e1) pl->event_pool.push_back(e1);
        continue;
      }
      GLS_CUDA(cudaGraphExecEventRecordNodeSetEvent(r.exec, m.n0, e0));
      GLS_CUDA(cudaGraphExecEventRecordNodeSetEvent(r.exec, m.n1, e1));
      m.slot->pending.emplace_back(e0, e1);
    }
  }
  GLS_CUDA(cudaGraphLaunch(r.exec, pl->stream));
  pl->launches += r.launches;
  return GLS_OK;
}

// Runs body() (launches on pl->stream only, no host synchronisation) through
// the cache rc: eagerly the first time `key` is seen, captured and replayed
// from the second time on.  A failed capture runs body() eagerly and turns
// the cache off.
template <class F>
gls_status_t replayed(gls_plan* pl, ReplayCache* rc, uint64_t key, F&& body) {
  if (!rc || !rc->enabled || !pl->own_stream || (pl->desc.flags & GLS_FLAG_EAGER)) return body();
  key = (KeyHash() << key << (uint64_t)pl->timing).h;
  for (auto& r : rc->items)
    if (r->key == key) {
      r->used = ++rc->clock;
      return launch_replay(pl, *r);
    }
  if (std::find(rc->seen.begin(), rc->seen.end(), key) == rc->seen.end()) {
    if (rc->seen.size() >= ReplayCache::kMaxSeen) rc->seen.erase(rc->seen.begin());
    rc->seen.push_back(key);
    return body();
  }
  Capture cap;
  for (int i = 0; i < 8 && pl->timing; ++i) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      break;
    }
    cap.spare.push_back(e);
  }
  auto r = std::make_unique<Replay>();
  r->key = key;
  const int64_t l0 = pl->launches;
  bool ok = cudaStreamBeginCapture(pl->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  gls_status_t s = GLS_OK;
  if (ok) {
    pl->cap = &cap;
    s = body();
    pl->cap = nullptr;
    ok = cudaStreamEndCapture(pl->stream, &r->graph) == cudaSuccess && r->graph && s == GLS_OK;
  }
  r->launches = pl->launches - l0;
  pl->launches = l0;
  r->events = cap.used;
  r->events.insert(r->events.end(), cap.spare.begin(), cap.spare.end());
  if (ok) ok = cudaGraphInstantiate(&r->exec, r->graph, 0) == cudaSuccess;
  if (ok && !cap.marks.empty()) {
    size_t nn = 0;
    ok = cudaGraphGetNodes(r->graph, nullptr, &nn) == cudaSuccess;
    std::vector<cudaGraphNode_t> nodes(nn);
    if (ok && nn) ok = cudaGraphGetNodes(r->graph, nodes.data(), &nn) == cudaSuccess;
    auto node_of = [&](cudaEvent_t e) -> cudaGraphNode_t {
      for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        cudaEvent_t ev = nullptr;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeEventRecord &&
            cudaGraphEventRecordNodeGetEvent(nd, &ev) == cudaSuccess && ev == e)
          return nd;
      }
      return nullptr;
    };
    for (const Capture::Mark& m : cap.marks) {
      Replay::Mark rm;
      rm.n0 = node_of(m.e0);
      rm.n1 = node_of(m.e1);
      rm.slot = m.slot;
      if (!rm.n0 || !rm.n1) ok = false;
      r->marks.push_back(rm);
    }
  }
  if (!ok) {
    cudaGetLastError();
    rc->enabled = false;
    r.reset();
    return body();  // nothing ran during the capture
  }
  if (rc->items.size() >= ReplayCache::kMaxGraphs) {
    cudaStreamSynchronize(pl->stream);  // the evicted graph may still be running
    auto lru = std::min_element(rc->items.begin(), rc->items.end(),
                                [](const std::unique_ptr<Replay>& a,
                                   const std::unique_ptr<Replay>& b) { return a->used < b->used; });
    rc->items.erase(lru);
  }
  r->used = ++rc->clock;
  Replay& ref = *r;
  rc->items.push_back(std::move(r));
  return launch_replay(pl, ref);
}

// FP64 path: per 64-row block, nw + 1 partial sums per SNP (S_BL, b_B per
// phenotype, S_BR).  Mixed path: one S_BR partial per 128-row block per SNP,
// plus the nw linear Gram entries per SNP.
size_t partial_doubles(int precision, int64_t npad, int nw, int64_t kmax) {
  if (precision == GLS_PREC_FP64) return (size_t)(npad / gls::kT) * (nw + 1) * kmax;
  return (size_t)(npad / 128 + nw) * kmax;
}

int phenotypes_of(const gls_plan_desc_t& d) { return d.phenotypes > 0 ? d.phenotypes : 1; }

bool uses_tc_factor(const gls_plan_desc_t& d) {
  if (d.precision == GLS_PREC_FP64) return (d.flags & GLS_FLAG_FACTOR_TENSOR) != 0;
  return (d.flags & GLS_FLAG_FACTOR_NATIVE) == 0;
}

size_t footprint(const gls_plan_desc_t& d, int64_t* npad_out = nullptr) {
  const int64_t npad = gls::round_up(d.n, 128);
  if (npad_out) *npad_out = npad;
  const int p = d.p, t = phenotypes_of(d), nw = p - 1 + t;
  const int64_t kmax = d.max_block_snps;
  size_t bytes = 0;
  bytes += 2 * (size_t)npad * npad * sizeof(double);              // L, Z
  bytes += 2 * (size_t)npad * nw * sizeof(double);                // Wrhs, Wt
  bytes += (size_t)nw * nw * sizeof(double) + 2 * 32 * 32 * sizeof(double);
  bytes += 64;                                                    // flags
  bytes += 2 * (size_t)d.n * kmax;                                // X_R staging
  bytes += 2 * (size_t)kmax * ((size_t)p * t * sizeof(double) + sizeof(int32_t));
  bytes += partial_doubles(d.precision, npad, nw, kmax) * sizeof(double);  // Gram partials
  if (d.precision != GLS_PREC_FP64)
    bytes += gls::mixed_footprint(d.n, npad, nw, kmax, d.split_terms);
  if (uses_tc_factor(d)) bytes += gls::tc_factor_bytes(npad);
  return bytes;
}

gls_status_t validate_desc(const gls_plan_desc_t* d) {
  if (!d) {
    set_error("desc is NULL");
    return GLS_ERR_INVALID_ARG;
  }
  if (d->n < 1 || d->n > (int64_t)1 << 20) {
    set_error("n = %lld out of range", (long long)d->n);
    return GLS_ERR_INVALID_ARG;
  }
  if (d->p < 1 || d->p > gls::kMaxP) {
    set_error("p = %d out of range [1, %d]", d->p, gls::kMaxP);
    return GLS_ERR_INVALID_ARG;
  }
  if (d->max_block_snps < 1) {
    set_error("max_block_snps must be >= 1");
    return GLS_ERR_INVALID_ARG;
  }
  if (d->precision != GLS_PREC_FP64 && d->precision != GLS_PREC_MIXED_BF16 &&
      d->precision != GLS_PREC_MIXED_FP16) {
    set_error("unknown precision %d", d->precision);
    return GLS_ERR_INVALID_ARG;
  }
  if (!(d->split_terms == 0 || d->split_terms == 2 || d->split_terms == 3)) {
    set_error("split_terms must be 0, 2 or 3");
    return GLS_ERR_INVALID_ARG;
  }
  const uint32_t known = GLS_FLAG_NAIVE_SPLIT | GLS_FLAG_FACTOR_NATIVE | GLS_FLAG_FACTOR_TENSOR |
                         GLS_FLAG_EAGER | GLS_FLAG_STAGED_INPUT;
  if ((d->flags & ~known) != 0) {
    set_error("unknown flag bits 0x%x", d->flags);
    return GLS_ERR_INVALID_ARG;
  }
  if ((d->flags & GLS_FLAG_FACTOR_NATIVE) && (d->flags & GLS_FLAG_FACTOR_TENSOR)) {
    set_error("GLS_FLAG_FACTOR_NATIVE and GLS_FLAG_FACTOR_TENSOR exclude each other");
    return GLS_ERR_INVALID_ARG;
  }
  if (d->wait_limit_us < 0 || d->host_wait_ms < 0) {
    set_error("wait_limit_us and host_wait_ms must be >= 0");
    return GLS_ERR_INVALID_ARG;
  }
  if (d->phenotypes < 0 || d->p - 1 + phenotypes_of(*d) > gls::kMaxW) {
    set_error("phenotypes = %d: need p - 1 + phenotypes <= %d", d->phenotypes, gls::kMaxW);
    return GLS_ERR_INVALID_ARG;
  }
  for (int i = 0; i < 4; ++i)
    if (d->reserved[i] != 0) {
      set_error("reserved fields must be 0");
      return GLS_ERR_INVALID_ARG;
    }
  return GLS_OK;
}

void free_plan(gls_plan* pl) {
  if (!pl) return;
  if (pl->stream) cudaStreamSynchronize(pl->stream);
  if (pl->h2d) cudaStreamSynchronize(pl->h2d);
  if (pl->d2h) cudaStreamSynchronize(pl->d2h);
  delete pl->replays;
  pl->replays = nullptr;
  if (pl->mixed) gls::mixed_free(pl->mixed);
  if (pl->tcf) gls::tc_factor_free(pl->tcf);
  cudaFree(pl->A);
  cudaFree(pl->Z);
  cudaFree(pl->Wrhs);
  cudaFree(pl->Wt);
  cudaFree(pl->gram);
  cudaFree(pl->RTL);
  cudaFree(pl->zT);
  cudaFree(pl->flags);
  cudaFreeHost(pl->h_flags);
  cudaFree(pl->partials);
  for (int s = 0; s < 2; ++s) {
    cudaFree(pl->xr[s]);
    cudaFree(pl->bdev[s]);
    cudaFree(pl->sdev[s]);
    cudaFreeHost(pl->h_xr[s]);
    cudaFree(pl->xp[s]);
    cudaFreeHost(pl->h_xp[s]);
    cudaFreeHost(pl->h_b[s]);
    cudaFreeHost(pl->h_s[s]);
    if (pl->ev_loaded[s]) cudaEventDestroy(pl->ev_loaded[s]);
    if (pl->ev_computed[s]) cudaEventDestroy(pl->ev_computed[s]);
    if (pl->ev_stored[s]) cudaEventDestroy(pl->ev_stored[s]);
    if (pl->ev_staged[s]) cudaEventDestroy(pl->ev_staged[s]);
  }
  for (int s = 0; s < 3; ++s) {
    cudaFreeHost(pl->h_ring[s]);
    if (pl->ev_ring[s]) cudaEventDestroy(pl->ev_ring[s]);
  }
  for (gls_plan::Slot* sl :
       {&pl->t_trsm, &pl->t_convert, &pl->t_solve, &pl->t_factor, &pl->t_h2d, &pl->t_d2h})
    for (auto& pr : sl->pending) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  for (cudaEvent_t e : pl->event_pool) cudaEventDestroy(e);
  if (pl->h2d) cudaStreamDestroy(pl->h2d);
  if (pl->d2h) cudaStreamDestroy(pl->d2h);
  if (pl->cvt) cudaStreamDestroy(pl->cvt);
  for (cudaEvent_t e : pl->ev_conv)
    if (e) cudaEventDestroy(e);
  if (pl->own_stream && pl->stream) cudaStreamDestroy(pl->stream);
  cudaGetLastError();
  delete pl;
}

// A pitched copy, issued as one contiguous copy when both pitches equal the
// row width (the usual case for X_R blocks and b): one large transfer for the
// copy engine instead of a row-by-row description.
cudaError_t copy2d(void* dst, size_t dpitch, const void* src, size_t spitch, size_t width,
                   size_t height, cudaMemcpyKind kind, cudaStream_t st) {
  if (dpitch == width && spitch == width)
    return cudaMemcpyAsync(dst, src, width * height, kind, st);
  return cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, height, kind, st);
}

// A host<->device copy of the double-buffered stream on a side stream,
// bracketed by events when timing is on (its duration on that stream).
cudaError_t timed_copy(gls_plan* pl, gls_plan::Slot* slot, cudaStream_t side, size_t bytes,
                       cudaError_t (*issue)(void*), void* ctx) {
  cudaEvent_t e0 = pl->timing ? pool_event(pl) : nullptr;
  cudaEvent_t e1 = pl->timing ? pool_event(pl) : nullptr;
  if (e0 && e1) cudaEventRecord(e0, side);
  cudaError_t e = issue(ctx);
  if (e0 && e1) {
    cudaEventRecord(e1, side);
    slot->pending.emplace_back(e0, e1);
    slot->bytes += (int64_t)bytes;
  } else {
    if (e0) pl->event_pool.push_back(e0);
    if (e1) pl->event_pool.push_back(e1);
  }
  return e;
}

template <class T>
gls_status_t dev_alloc(T** p, size_t count) {
  if (cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    set_error("cudaMalloc of %zu bytes failed", count * sizeof(T));
    return GLS_ERR_OOM;
  }
  return GLS_OK;
}

template <class T>
gls_status_t host_alloc(T** p, size_t count) {
  if (cudaMallocHost((void**)p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    set_error("cudaMallocHost of %zu bytes failed", count * sizeof(T));
    return GLS_ERR_OOM;
  }
  return GLS_OK;
}

#define GLS_TRY(expr)              \
  do {                             \
    gls_status_t s_ = (expr);      \
    if (s_ != GLS_OK) return s_;   \
  } while (0)

// Waits on the host for the work queued on `st`.  With a deadline
// (desc.host_wait_ms > 0) it polls and gives up past it, the work still queued.
gls_status_t host_wait(gls_plan* pl, cudaStream_t st) {
  const int32_t limit_ms = pl->desc.host_wait_ms;
  if (limit_ms <= 0) {
    GLS_CUDA(cudaStreamSynchronize(st));
    return GLS_OK;
  }
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaStreamQuery(st);
    if (e == cudaSuccess) return GLS_OK;
    if (e != cudaErrorNotReady) {
      set_error("stream wait failed: %s", cudaGetErrorString(e));
      return GLS_ERR_CUDA;
    }
    if (std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(limit_ms)) {
      cudaGetLastError();
      set_error("host wait gave up after %d ms with the plan's work still queued; "
                "gls_synchronize or gls_destroy before reusing its buffers", limit_ms);
      return GLS_ERR_TIMEOUT;
    }
    std::this_thread::yield();
  }
}

gls_status_t check_flags(gls_plan* pl, int host_flags[gls::kFlagCount]) {
  // into pinned memory: a copy into pageable memory would itself block until
  // the stream is done, outside the deadline
  GLS_CUDA(cudaMemcpyAsync(pl->h_flags, pl->flags, sizeof(int) * gls::kFlagCount,
                           cudaMemcpyDeviceToHost, pl->stream));
  GLS_TRY(host_wait(pl, pl->stream));
  memcpy(host_flags, pl->h_flags, sizeof(int) * gls::kFlagCount);
  if (host_flags[gls::kFlagKernel] & gls::kErrTimeout) {
    set_error("a bounded device wait gave up (site %d)", host_flags[gls::kFlagWhere]);
    return GLS_ERR_TIMEOUT;
  }
  if (host_flags[gls::kFlagKernel] != 0) {
    set_error("kernel error bits 0x%x", host_flags[gls::kFlagKernel]);
    return GLS_ERR_CUDA;
  }
  return GLS_OK;
}

// Solves one block whose inputs/outputs are all device resident, on pl->stream.
// Mixed paths only: with xp set, the genotypes are 2-bit packed columns (ldp
// bytes each) converted straight to the tensor-core operand (xr unused).
// With `converted` the block's operand is already in buffer buf (xr unused);
// side_sms > 0 leaves that many SMs to a conversion running beside the solve.
gls_status_t run_block(gls_plan* pl, const int8_t* xr, int64_t ldxr, int64_t k, double* B,
                       int64_t ldb, int32_t* status, const uint8_t* xp = nullptr,
                       int64_t ldp = 0, int buf = 0, bool converted = false,
                       int side_sms = 0) {
  if (k == 0) return GLS_OK;
  if (pl->precision == GLS_PREC_FP64) {
    {
      Timed t(pl, &pl->t_trsm);
      GLS_CUDA(gls::launch_trsm_gram_fp64(pl->Z, pl->npad, pl->n, pl->npad, xr, ldxr, k, pl->Wt,
                                          pl->npad, pl->nw, pl->partials, pl->ldp, pl->stream));
    }
    Timed t(pl, &pl->t_solve);
    gls::launch_assemble_solve(pl->partials, pl->ldp, pl->nI, pl->p, pl->t_active, pl->nw, k,
                               pl->RTL, pl->zT, gls::kTauFP64, B, ldb, status, pl->stream);
    pl->launches += 2;
  } else {
    double* Pbr = pl->partials;                      // nI x ldp
    double* Glin = pl->partials + (int64_t)pl->nI * pl->ldp;  // p x ldp
    if (!converted) {
      Timed t(pl, &pl->t_convert);
      if (xp) GLS_CUDA(gls::mixed_convert_packed(pl->mixed, xp, ldp, k, pl->stream));
      else GLS_CUDA(gls::mixed_convert(pl->mixed, xr, ldxr, k, pl->stream));
      pl->launches += 1;
    }
    {
      Timed t(pl, &pl->t_trsm);
      GLS_CUDA(gls::mixed_trsm_gram(pl->mixed, xr, ldxr, k, Pbr, Glin, pl->ldp, pl->flags,
                                    pl->stream, buf, side_sms));
    }
    Timed t(pl, &pl->t_solve);
    gls::launch_assemble_solve_split(Glin, Pbr, pl->ldp, pl->nI, pl->p, pl->t_active, k, pl->RTL,
                                     pl->zT, gls::kTauMixed, B, ldb, status, pl->stream);
    pl->launches += 2;
  }
  GLS_CUDA(cudaGetLastError());
  return GLS_OK;
}

}  // namespace

extern "C" {

int32_t gls_version(void) { return 200; }  // 0.2.0: packed input, graph replay, factor flags

const char* gls_last_error(void) { return g_last_error.c_str(); }

const char* gls_status_string(gls_status_t s) {
  switch (s) {
    case GLS_OK: return "GLS_OK";
    case GLS_ERR_INVALID_ARG: return "GLS_ERR_INVALID_ARG";
    case GLS_ERR_NOT_SPD: return "GLS_ERR_NOT_SPD";
    case GLS_ERR_OOM: return "GLS_ERR_OOM";
    case GLS_ERR_CUDA: return "GLS_ERR_CUDA";
    case GLS_ERR_TIMEOUT: return "GLS_ERR_TIMEOUT";
    case GLS_ERR_STATE: return "GLS_ERR_STATE";
    case GLS_ERR_UNSUPPORTED: return "GLS_ERR_UNSUPPORTED";
    case GLS_ERR_COVARIATES_SINGULAR: return "GLS_ERR_COVARIATES_SINGULAR";
    case GLS_ERR_IO: return "GLS_ERR_IO";
  }
  return "GLS_ERR_UNKNOWN";
}

size_t gls_plan_footprint_bytes(const gls_plan_desc_t* desc) {
  if (validate_desc(desc) != GLS_OK) return 0;
  return footprint(*desc);
}

gls_status_t gls_plan_create(const gls_plan_desc_t* desc, gls_plan_t* out) {
  g_last_error.clear();
  if (!out) {
    set_error("out is NULL");
    return GLS_ERR_INVALID_ARG;
  }
  *out = nullptr;
  GLS_TRY(validate_desc(desc));
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    set_error("no CUDA device");
    return GLS_ERR_UNSUPPORTED;
  }
  if (desc->device < 0 || desc->device >= ndev) {
    set_error("device %d out of range", desc->device);
    return GLS_ERR_INVALID_ARG;
  }
  DeviceGuard guard(desc->device);
  if (!guard.ok) {
    set_error("cudaSetDevice(%d) failed", desc->device);
    return GLS_ERR_CUDA;
  }
  cudaDeviceProp prop;
  GLS_CUDA(cudaGetDeviceProperties(&prop, desc->device));
  if (!(prop.major == 10 && prop.minor == 3)) {
    set_error("device %d is sm_%d%d; this build targets sm_103a", desc->device, prop.major,
              prop.minor);
    return GLS_ERR_UNSUPPORTED;
  }
  gls_plan* pl = new gls_plan();
  pl->desc = *desc;
  pl->device = desc->device;
  pl->n = desc->n;
  pl->p = desc->p;
  pl->kmax = desc->max_block_snps;
  pl->precision = desc->precision;
  pl->t = pl->t_active = phenotypes_of(*desc);
  pl->nw = desc->p - 1 + pl->t;
  footprint(*desc, &pl->npad);
  const int64_t npad = pl->npad, n = pl->n, kmax = pl->kmax;
  const int p = pl->p, nw = pl->nw;
  pl->nI = (int)((pl->precision == GLS_PREC_FP64) ? npad / gls::kT : npad / 128);
  pl->ldp = kmax;

  auto fail = [&](gls_status_t s) {
    free_plan(pl);
    return s;
  };
  if (desc->stream) {
    pl->stream = (cudaStream_t)desc->stream;
  } else {
    if (cudaStreamCreateWithFlags(&pl->stream, cudaStreamNonBlocking) != cudaSuccess) {
      set_error("cudaStreamCreate failed");
      return fail(GLS_ERR_CUDA);
    }
    pl->own_stream = true;
  }
  pl->replays = new ReplayCache();
  if (cudaStreamCreateWithFlags(&pl->h2d, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&pl->d2h, cudaStreamNonBlocking) != cudaSuccess) {
    set_error("cudaStreamCreate failed");
    return fail(GLS_ERR_CUDA);
  }
  for (int s = 0; s < 2; ++s) {
    if (cudaEventCreateWithFlags(&pl->ev_loaded[s], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&pl->ev_computed[s], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&pl->ev_stored[s], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&pl->ev_staged[s], cudaEventDisableTiming) != cudaSuccess) {
      set_error("cudaEventCreate failed");
      return fail(GLS_ERR_CUDA);
    }
  }
  gls_status_t st;
  if ((st = dev_alloc(&pl->A, (size_t)npad * npad)) != GLS_OK) return fail(st);
  if ((st = dev_alloc(&pl->Z, (size_t)npad * npad)) != GLS_OK) return fail(st);
  if ((st = dev_alloc(&pl->Wrhs, (size_t)npad * nw)) != GLS_OK) return fail(st);
  if ((st = dev_alloc(&pl->Wt, (size_t)npad * nw)) != GLS_OK) return fail(st);
  if ((st = dev_alloc(&pl->gram, (size_t)nw * nw)) != GLS_OK) return fail(st);
  if ((st = dev_alloc(&pl->RTL, (size_t)32 * 32)) != GLS_OK) return fail(st);
  if ((st = dev_alloc(&pl->zT, (size_t)32 * 32)) != GLS_OK) return fail(st);
  if ((st = dev_alloc(&pl->flags, (size_t)gls::kFlagCount)) != GLS_OK) return fail(st);
  if ((st = host_alloc(&pl->h_flags, (size_t)gls::kFlagCount)) != GLS_OK) return fail(st);
  if ((st = dev_alloc(&pl->partials, partial_doubles(pl->precision, npad, nw, kmax))) != GLS_OK)
    return fail(st);
  for (int s = 0; s < 2; ++s) {
    if ((st = dev_alloc(&pl->xr[s], (size_t)n * kmax)) != GLS_OK) return fail(st);
    if ((st = dev_alloc(&pl->bdev[s], (size_t)p * pl->t * kmax)) != GLS_OK) return fail(st);
    if ((st = dev_alloc(&pl->sdev[s], (size_t)kmax)) != GLS_OK) return fail(st);
  }
  if (cudaMemsetAsync(pl->Wrhs, 0, sizeof(double) * npad * nw, pl->stream) != cudaSuccess ||
      cudaMemsetAsync(pl->flags, 0, sizeof(int) * gls::kFlagCount, pl->stream) != cudaSuccess) {
    set_error("cudaMemset failed");
    return fail(GLS_ERR_CUDA);
  }
  if (pl->precision != GLS_PREC_FP64) {
    if ((st = gls::mixed_create(&pl->mixed, n, npad, nw, kmax, pl->precision, desc->split_terms,
                                desc->flags, desc->wait_limit_us, pl->stream)) != GLS_OK) {
      set_error("%s", gls::mixed_last_error());
      return fail(st);
    }
  }
  pl->tc = uses_tc_factor(*desc);
  if (pl->tc) {
    if ((st = gls::tc_factor_create(&pl->tcf, npad)) != GLS_OK) {
      set_error("%s", gls::tc_factor_last_error());
      return fail(st);
    }
  }
  if (cudaStreamSynchronize(pl->stream) != cudaSuccess) {
    set_error("plan setup failed: %s", cudaGetErrorString(cudaGetLastError()));
    return fail(GLS_ERR_CUDA);
  }
  *out = pl;
  return GLS_OK;
}

gls_status_t gls_factor(gls_plan_t pl, const double* M, int64_t ldm, const double* XL,
                        int64_t ldxl, const double* y, int64_t* info) {
  return gls_factor_y(pl, M, ldm, XL, ldxl, y, pl ? pl->n : 1, 1, info);
}

gls_status_t gls_factor_y(gls_plan_t pl, const double* M, int64_t ldm, const double* XL,
                          int64_t ldxl, const double* Y, int64_t ldy, int32_t t,
                          int64_t* info) {
  g_last_error.clear();
  if (info) *info = 0;
  if (!pl) {
    set_error("plan is NULL");
    return GLS_ERR_INVALID_ARG;
  }
  if (!Y) {
    set_error("Y is NULL");
    return GLS_ERR_INVALID_ARG;
  }
  if (t < 1 || t > pl->t || ldy < pl->n) {
    set_error("t = %d outside [1, phenotypes = %d], or ldy < n", t, pl->t);
    return GLS_ERR_INVALID_ARG;
  }
  if (M && ldm < pl->n) {
    set_error("ldm < n");
    return GLS_ERR_INVALID_ARG;
  }
  if (!M && !pl->has_factor) {
    set_error("M == NULL but no earlier factor to keep");
    return GLS_ERR_STATE;
  }
  if (pl->p > 1) {
    if (XL && ldxl < pl->n) {
      set_error("ldxl < n");
      return GLS_ERR_INVALID_ARG;
    }
    if (!XL && !pl->has_xl) {
      set_error("XL is NULL but p > 1 and no earlier X_L to keep");
      return GLS_ERR_INVALID_ARG;
    }
  }
  DeviceGuard guard(pl->device);
  pl->factored = false;
  const int64_t n = pl->n, npad = pl->npad;
  const int p = pl->p, q = p - 1, nw = pl->nw;
  cudaStream_t st = pl->stream;
  Timed phase(pl, &pl->t_factor);
  GLS_CUDA(cudaMemsetAsync(pl->flags, 0, sizeof(int) * gls::kFlagCount, st));
  if (M) {
    pl->has_factor = false;
    GLS_CUDA(copy2d(pl->A, npad * sizeof(double), M, ldm * sizeof(double),
                               n * sizeof(double), n, cudaMemcpyDefault, st));
    // from here on the factor touches plan buffers only: one graph per plan
    GLS_TRY(replayed(pl, pl->replays, (KeyHash() << 1u).h, [&]() -> gls_status_t {
      gls::launch_pad_lower(pl->A, npad, n, npad, st);
      gls::launch_identity(pl->Z, npad, npad, st);
      if (pl->tc) {
        const int64_t tc0 = gls::tc_launches(pl->tcf);
        cudaError_t e = gls::tc_potrf_trtri(pl->tcf, pl->A, pl->Z, npad, npad, pl->flags, st);
        if (e != cudaSuccess) {
          set_error("tensor-core factor: %s %s", cudaGetErrorString(e),
                    gls::tc_factor_last_error());
          return GLS_ERR_CUDA;
        }
        pl->launches += 2 + gls::tc_launches(pl->tcf) - tc0;
      } else {
        const int64_t N = npad / gls::kT;
        GLS_CUDA(gls::potrf_trtri_fp64(pl->A, pl->Z, npad, npad, pl->flags, st));
        pl->launches += 2 + N + 4 * (N - 1);
      }
      return GLS_OK;
    }));
  }
  const int64_t tc_before = pl->tc ? gls::tc_launches(pl->tcf) : 0;
  if (p > 1 && XL) {
    GLS_CUDA(copy2d(pl->Wrhs, npad * sizeof(double), XL, ldxl * sizeof(double),
                               n * sizeof(double), p - 1, cudaMemcpyDefault, st));
    pl->has_xl = true;
  }
  GLS_CUDA(copy2d(pl->Wrhs + (int64_t)q * npad, npad * sizeof(double), Y, ldy * sizeof(double),
                  n * sizeof(double), t, cudaMemcpyDefault, st));
  if (q + t < nw)  // columns of phenotypes this call does not use: zero
    GLS_CUDA(cudaMemsetAsync(pl->Wrhs + (int64_t)(q + t) * npad, 0,
                             sizeof(double) * npad * (nw - q - t), st));
  if (pl->tc) {
    cudaError_t e = gls::tc_lower_times(pl->tcf, pl->Z, npad, npad, pl->Wrhs, npad, nw, pl->Wt,
                                        npad, pl->flags, st);
    if (e != cudaSuccess) {
      set_error("tensor-core whitening: %s %s", cudaGetErrorString(e),
                gls::tc_factor_last_error());
      return GLS_ERR_CUDA;
    }
  } else {
    gls::launch_whiten(pl->Z, npad, n, npad, pl->Wrhs, npad, nw, pl->Wt, npad, pl->flags, st);
  }
  gls::launch_fixed_gram(pl->Wt, npad, n, nw, pl->gram, st);
  if (p > 1) gls::launch_small_chol(pl->gram, nw, q, t, pl->RTL, pl->zT, pl->flags, st);
  pl->launches += (p > 1) ? 3 : 2;
  GLS_CUDA(cudaGetLastError());
  int hf[gls::kFlagCount];
  GLS_TRY(check_flags(pl, hf));
  if (hf[gls::kFlagPotrf] != 0) {
    if (info) *info = hf[gls::kFlagPotrf];
    set_error("M is not positive definite (pivot %d)", hf[gls::kFlagPotrf]);
    return GLS_ERR_NOT_SPD;
  }
  pl->has_factor = true;
  if (hf[gls::kFlagSTL] != 0) {
    if (info) *info = hf[gls::kFlagSTL];
    set_error("X~_L^T X~_L is not positive definite (pivot %d)", hf[gls::kFlagSTL]);
    return GLS_ERR_COVARIATES_SINGULAR;
  }
  if (pl->precision != GLS_PREC_FP64) {
    double* W = nullptr;  // M^{-1} [X_L | y] = Z^T [X~_L | y~]
    if (pl->tc) {
      W = gls::mixed_w_buffer(pl->mixed);
      cudaError_t e = gls::tc_lower_t_times(pl->tcf, pl->Z, npad, npad, pl->Wt, npad, nw, W, npad,
                                            pl->flags, st);
      if (e != cudaSuccess) {
        set_error("tensor-core W: %s %s", cudaGetErrorString(e), gls::tc_factor_last_error());
        return GLS_ERR_CUDA;
      }
    }
    GLS_TRY(gls::mixed_prepare(pl->mixed, pl->Z, npad, pl->Wt, npad, M != nullptr, W != nullptr,
                               st));
    pl->launches += (M != nullptr ? 1 : 0) + (W != nullptr ? 0 : 1) + 1;
  }
  phase.finish();
  if (pl->tc) pl->launches += gls::tc_launches(pl->tcf) - tc_before;
  if (pl->precision != GLS_PREC_FP64) GLS_TRY(check_flags(pl, hf));
  pl->t_active = t;
  pl->factored = true;
  return GLS_OK;
}

gls_status_t gls_plan_get_factor(gls_plan_t pl, double* L, int64_t ldl, double* Zinv,
                                 int64_t ldz) {
  g_last_error.clear();
  if (!pl) {
    set_error("plan is NULL");
    return GLS_ERR_INVALID_ARG;
  }
  if (!pl->has_factor) {
    set_error("no factor yet");
    return GLS_ERR_STATE;
  }
  if ((L && ldl < pl->n) || (Zinv && ldz < pl->n)) {
    set_error("leading dimension < n");
    return GLS_ERR_INVALID_ARG;
  }
  DeviceGuard guard(pl->device);
  const int64_t n = pl->n, npad = pl->npad;
  if (L)
    GLS_CUDA(copy2d(L, ldl * sizeof(double), pl->A, npad * sizeof(double),
                               n * sizeof(double), n, cudaMemcpyDefault, pl->stream));
  if (Zinv)
    GLS_CUDA(copy2d(Zinv, ldz * sizeof(double), pl->Z, npad * sizeof(double),
                               n * sizeof(double), n, cudaMemcpyDefault, pl->stream));
  return host_wait(pl, pl->stream);
}

gls_status_t gls_solve_block(gls_plan_t pl, const int8_t* XR, int64_t ldxr, int64_t k,
                             double* B, int64_t ldb, int32_t* snp_status) {
  g_last_error.clear();
  if (!pl) {
    set_error("plan is NULL");
    return GLS_ERR_INVALID_ARG;
  }
  if (!pl->factored) {
    set_error("gls_solve_block before a successful gls_factor");
    return GLS_ERR_STATE;
  }
  if (k < 0 || k > pl->kmax) {
    set_error("k = %lld outside [0, max_block_snps = %lld]", (long long)k, (long long)pl->kmax);
    return GLS_ERR_INVALID_ARG;
  }
  if (k == 0) return GLS_OK;
  if (!XR || !B || ldxr < pl->n || ldb < pl->p) {
    set_error("bad XR/B pointer or leading dimension");
    return GLS_ERR_INVALID_ARG;
  }
  DeviceGuard guard(pl->device);
  const Mem mx = classify(XR), mb = classify(B);
  const Mem ms = snp_status ? classify(snp_status) : Mem::Device;
  cudaStream_t st = pl->stream;
  const int8_t* xin = XR;
  int64_t ldin = ldxr;
  if (mx != Mem::Device) {
    GLS_CUDA(copy2d(pl->xr[0], pl->n, XR, ldxr, pl->n, k, cudaMemcpyHostToDevice, st));
    xin = pl->xr[0];
    ldin = pl->n;
  }
  double* bout = (mb == Mem::Device) ? B : pl->bdev[0];
  const int64_t ldout = (mb == Mem::Device) ? ldb : pl->p;
  int32_t* sout = snp_status ? ((ms == Mem::Device) ? snp_status : pl->sdev[0]) : nullptr;
  GLS_TRY(replayed(pl, pl->replays,
                   (KeyHash() << 2u << xin << ldin << k << bout << ldout << sout
                    << (uint64_t)pl->t_active).h,
                   [&]() { return run_block(pl, xin, ldin, k, bout, ldout, sout); }));
  const bool sync = (mx != Mem::Device) || (mb != Mem::Device) || (ms != Mem::Device);
  if (mb != Mem::Device)
    GLS_CUDA(copy2d(B, ldb * sizeof(double), bout, pl->p * sizeof(double),
                               pl->p * sizeof(double), k * pl->t_active, cudaMemcpyDeviceToHost,
                               st));
  if (snp_status && ms != Mem::Device)
    GLS_CUDA(cudaMemcpyAsync(snp_status, sout, k * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  if (sync) {
    int hf[gls::kFlagCount];
    GLS_TRY(check_flags(pl, hf));
  }
  return GLS_OK;
}

}  // extern "C"

namespace {

// Device staging of packed blocks (and pinned staging for pageable input),
// allocated by the first packed call.
gls_status_t packed_staging(gls_plan* pl, bool pinned) {
  const size_t bytes = (size_t)gls::ceil_div(pl->n, 4) * (size_t)pl->kmax;
  for (int s = 0; s < 2; ++s) {
    if (!pl->xp[s]) GLS_TRY(dev_alloc(&pl->xp[s], bytes));
    if (pinned && !pl->h_xp[s]) GLS_TRY(host_alloc(&pl->h_xp[s], bytes));
  }
  return GLS_OK;
}

// Block schedule of a stream of m SNPs: a short first block (its load is not
// overlapped), then doubling up to max_block_snps (Section 4.3); uniform:
// max_block_snps throughout.
std::vector<std::pair<int64_t, int64_t>> block_schedule(int64_t kmax, int64_t m,
                                                        bool uniform = false) {
  std::vector<std::pair<int64_t, int64_t>> blocks;
  int64_t kb = uniform ? kmax : std::min<int64_t>(kmax, std::max<int64_t>(256, kmax / 8));
  for (int64_t s0 = 0; s0 < m;) {
    const int64_t kk = std::min<int64_t>(kb, m - s0);
    blocks.emplace_back(s0, kk);
    s0 += kk;
    kb = std::min<int64_t>(kmax, kb * 2);
  }
  return blocks;
}

// The disk tier of Alg. 8: genotype blocks are read from a file into a ring of
// pinned host slots by a background thread, ahead of the GPU (the paper's
// async_read).  Block j goes to slot j mod kSlots once the GPU has finished
// reading the block that used that slot before: the compute thread records an
// event after that read and the reader waits for it.  Each block is read by up
// to 8 parallel pread calls (one per 64 MiB) so that page-cache and NVMe reads
// reach their bandwidth.
struct FileRing {
  static constexpr int kSlots = 3;
  int fd = -1;
  int64_t offset = 0, ldx = 0;
  std::vector<std::pair<int64_t, int64_t>> blocks;  // (first SNP, SNPs)
  uint8_t* slot[kSlots]{};                           // pinned, ldx x kmax bytes each
  cudaEvent_t released[kSlots]{};                    // the GPU has read the slot's block
  std::mutex mu;
  std::condition_variable cv;
  int64_t filled = -1;    // last block read into its slot
  int64_t recorded = -1;  // last block whose release event has been recorded
  bool stop = false;
  int err = 0;            // errno of a failed or short read
  std::thread th;

  void run() {
    for (size_t jb = 0; jb < blocks.size(); ++jb) {
      const int s = (int)(jb % kSlots);
      if (jb >= (size_t)kSlots) {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return stop || recorded >= (int64_t)jb - kSlots; });
        if (stop) return;
        lk.unlock();
        if (cudaEventSynchronize(released[s]) != cudaSuccess) {
          cudaGetLastError();
          fail(EIO);
          return;
        }
      }
      const int64_t bytes = blocks[jb].second * ldx;
      const off_t at = (off_t)(offset + blocks[jb].first * ldx);
      const int parts = (int)std::max<int64_t>(1, std::min<int64_t>(8, bytes >> 26));
      std::vector<std::thread> rd;
      std::atomic<int> rerr{0};
      for (int t = 0; t < parts; ++t) {
        const int64_t b0 = bytes * t / parts, b1 = bytes * (t + 1) / parts;
        rd.emplace_back([&, b0, b1]() {
          int64_t done = b0;
          while (done < b1) {
            const ssize_t r = pread(fd, slot[s] + done, (size_t)(b1 - done), at + done);
            if (r <= 0) {
              rerr = r == 0 ? EIO : errno;
              return;
            }
            done += r;
          }
        });
      }
      for (auto& t : rd) t.join();
      if (rerr) {
        fail(rerr);
        return;
      }
      std::lock_guard<std::mutex> lk(mu);
      filled = (int64_t)jb;
      cv.notify_all();
    }
  }
  void fail(int e) {
    std::lock_guard<std::mutex> lk(mu);
    err = e;
    cv.notify_all();
  }
  // Waits until block jb is in its slot; false on a read error.
  bool wait_filled(size_t jb) {
    std::unique_lock<std::mutex> lk(mu);
    cv.wait(lk, [&] { return err != 0 || filled >= (int64_t)jb; });
    return err == 0;
  }
  // After the GPU work that reads block jb has been enqueued on `st`.
  cudaError_t release(size_t jb, cudaStream_t st) {
    const cudaError_t e = cudaEventRecord(released[jb % kSlots], st);
    std::lock_guard<std::mutex> lk(mu);
    recorded = (int64_t)jb;
    cv.notify_all();
    return e;
  }
  void finish() {
    {
      std::lock_guard<std::mutex> lk(mu);
      stop = true;
      cv.notify_all();
    }
    if (th.joinable()) th.join();
  }
};

// The second genotype operand buffer, the conversion stream and its events
// of a mixed plan (first stream that converts beside its solves).  False when
// they cannot be had; the stream then converts every block in line.
bool ensure_side(gls_plan* pl) {
  if (pl->cvt) return true;
  if (gls::mixed_add_buffer(pl->mixed) != GLS_OK) return false;
  cudaStream_t st = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (st) cudaStreamDestroy(st);
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    return false;
  }
  pl->cvt = st;
  pl->ev_conv[0] = ev[0];
  pl->ev_conv[1] = ev[1];
  return true;
}

// The SNP stream of Alg. 8 for int8 (packed = false, ldx >= n) or 2-bit
// packed (packed = true, ldx >= ceil(n/4)) genotype columns X, or, with a
// ring, for the blocks the ring reads from a file (X unused; its slots are
// pinned host memory).
gls_status_t stream_impl(gls_plan* pl, const uint8_t* X, int64_t ldx, bool packed, int64_t m,
                         double* B, int64_t ldb, int32_t* snp_status,
                         FileRing* ring = nullptr) {
  DeviceGuard guard(pl->device);
  const int64_t n = pl->n, kmax = pl->kmax;
  const int p = pl->p, t = pl->t_active;  // b_ij of SNP i, phenotype j: column i t + j of B
  const int64_t width = packed ? gls::ceil_div(n, 4) : n;  // bytes per column
  const void* Xdev = nullptr;
  const Mem mx = ring ? Mem::Pinned : classify(X, &Xdev), mb = classify(B);
  if (ring) Xdev = pl->d_ring[0];
  const Mem ms = snp_status ? classify(snp_status) : Mem::Device;
  // Mixed plans read pinned int8 blocks in place: the conversion kernel loads
  // them over the host link through the mapping's device address, and the
  // copy engine (whose rate falls several-fold while kernels run) is idle.
  const bool direct = !packed && pl->precision != GLS_PREC_FP64 && mx == Mem::Pinned && Xdev &&
                      !(pl->desc.flags & GLS_FLAG_STAGED_INPUT);
  const bool staged = (mx != Mem::Device) && !direct;

  // device-resident input has no load to hide behind a short first block
  const std::vector<std::pair<int64_t, int64_t>> blocks =
      ring ? ring->blocks : block_schedule(kmax, m, mx == Mem::Device);
  // host and device addresses of block jb's first column (ld = ldx)
  auto src_host = [&](size_t jb) -> const uint8_t* {
    return ring ? ring->slot[jb % FileRing::kSlots] : X + blocks[jb].first * ldx;
  };
  auto src_dev = [&](size_t jb) -> const uint8_t* {
    return ring ? pl->d_ring[jb % FileRing::kSlots]
                : reinterpret_cast<const uint8_t*>(Xdev) + blocks[jb].first * ldx;
  };
  const bool pageable_in = (mx == Mem::Pageable);
  const bool out_b_host = (mb != Mem::Device);
  const bool out_s_host = snp_status && (ms != Mem::Device);
  const bool pageable_out = (mb == Mem::Pageable) || (snp_status && ms == Mem::Pageable);
  if (packed) GLS_TRY(packed_staging(pl, pageable_in));
  for (int s = 0; s < 2; ++s) {
    if (!packed && pageable_in && !pl->h_xr[s])
      GLS_TRY(host_alloc(&pl->h_xr[s], (size_t)n * kmax));
    if (pageable_out && !pl->h_b[s]) {
      GLS_TRY(host_alloc(&pl->h_b[s], (size_t)p * pl->t * kmax));
      GLS_TRY(host_alloc(&pl->h_s[s], (size_t)kmax));
    }
  }
  // where the H2D copy of block s lands, and its pinned staging if pageable
  auto dev_in = [&](int s) -> uint8_t* {
    return packed ? pl->xp[s] : reinterpret_cast<uint8_t*>(pl->xr[s]);
  };
  auto host_in = [&](int s) -> uint8_t* {
    return packed ? pl->h_xp[s] : reinterpret_cast<uint8_t*>(pl->h_xr[s]);
  };
  cudaStream_t cs = pl->stream;
  // Order the side streams after any earlier work on the compute stream.
  cudaEvent_t ev0 = pl->ev_computed[1];
  GLS_CUDA(cudaEventRecord(ev0, cs));
  GLS_CUDA(cudaStreamWaitEvent(pl->h2d, ev0, 0));
  GLS_CUDA(cudaStreamWaitEvent(pl->d2h, ev0, 0));
  GLS_CUDA(cudaEventRecord(pl->ev_computed[0], cs));
  GLS_CUDA(cudaEventRecord(pl->ev_stored[0], pl->d2h));
  GLS_CUDA(cudaEventRecord(pl->ev_stored[1], pl->d2h));
  GLS_CUDA(cudaEventRecord(pl->ev_staged[0], pl->h2d));
  GLS_CUDA(cudaEventRecord(pl->ev_staged[1], pl->h2d));

  auto issue_load = [&](size_t jb) -> gls_status_t {
    const int s = (int)(jb % 2);
    const int64_t s0 = blocks[jb].first, kb = blocks[jb].second;
    // device buffer s is free once the compute of block jb-2 is done
    GLS_CUDA(cudaStreamWaitEvent(pl->h2d, pl->ev_computed[s], 0));
    struct Copy {
      void* dst;
      const void* src;
      size_t ldsrc, width, cols;
      cudaStream_t st;
    };
    auto issue = [](void* c) -> cudaError_t {
      const Copy& q = *static_cast<const Copy*>(c);
      return copy2d(q.dst, q.width, q.src, q.ldsrc, q.width, q.cols, cudaMemcpyHostToDevice,
                    q.st);
    };
    if (ring && !ring->wait_filled(jb)) {
      set_error("reading genotype block %zu from the file failed: %s", jb, strerror(ring->err));
      return GLS_ERR_IO;
    }
    if (!pageable_in) {
      Copy q{dev_in(s), src_host(jb), (size_t)ldx, (size_t)width, (size_t)kb, pl->h2d};
      GLS_CUDA(timed_copy(pl, &pl->t_h2d, pl->h2d, (size_t)width * kb, issue, &q));
      if (ring) GLS_CUDA(ring->release(jb, pl->h2d));
    } else {
      GLS_CUDA(cudaEventSynchronize(pl->ev_staged[s]));  // pinned staging s is free
      for (int64_t c = 0; c < kb; ++c)
        memcpy(host_in(s) + c * width, X + (s0 + c) * ldx, (size_t)width);
      Copy q{dev_in(s), host_in(s), (size_t)width, (size_t)width, (size_t)kb, pl->h2d};
      GLS_CUDA(timed_copy(pl, &pl->t_h2d, pl->h2d, (size_t)width * kb, issue, &q));
      GLS_CUDA(cudaEventRecord(pl->ev_staged[s], pl->h2d));
    }
    GLS_CUDA(cudaEventRecord(pl->ev_loaded[s], pl->h2d));
    return GLS_OK;
  };
  auto finish_host = [&](size_t jb) -> gls_status_t {
    if (!pageable_out) return GLS_OK;
    const int s = (int)(jb % 2);
    const int64_t s0 = blocks[jb].first, kb = blocks[jb].second;
    GLS_CUDA(cudaEventSynchronize(pl->ev_stored[s]));
    if (mb == Mem::Pageable)
      for (int64_t c = 0; c < kb * t; ++c)
        memcpy(B + (s0 * t + c) * ldb, pl->h_b[s] + c * p, sizeof(double) * p);
    if (snp_status && ms == Mem::Pageable)
      memcpy(snp_status + s0, pl->h_s[s], sizeof(int32_t) * kb);
    return GLS_OK;
  };

  // Reading pinned int8 in place over the host link takes the conversion
  // several times longer than from HBM, so there block j+1 is converted beside
  // block j's solve: the solve leaves gls::kSideSms SMs free and the
  // conversion (that many CTAs of 1024 threads, which never share an SM with a
  // solve CTA) writes the other operand buffer there.  From HBM the
  // conversion stays in line: on 3 SMs it took longer than the solves it ran
  // beside (about 54 GB/s per SM), and 8 SMs cost the solve more than the
  // 0.5 ms per block the conversion takes on the whole GPU.
  const uint8_t* side_base = reinterpret_cast<const uint8_t*>(Xdev);
  const bool side = direct && !ring && blocks.size() >= 2 && side_base &&
                    (reinterpret_cast<uintptr_t>(side_base) % 16) == 0 && (ldx % 16) == 0 &&
                    ensure_side(pl);
  const int side_sms = gls::kSideSms;
  auto side_src = [&](size_t jb) -> const int8_t* {
    return reinterpret_cast<const int8_t*>(side_base + blocks[jb].first * ldx);
  };
  auto side_convert = [&](size_t jb) -> gls_status_t {
    const int b = (int)(jb % 2);
    // operand buffer b is free once block jb-2 is solved
    GLS_CUDA(cudaStreamWaitEvent(pl->cvt, pl->ev_computed[b], 0));
    {
      Timed tm(pl, &pl->t_convert, pl->cvt);
      GLS_CUDA(gls::mixed_convert(pl->mixed, side_src(jb), ldx, blocks[jb].second, pl->cvt, b,
                                  side_sms));
    }
    pl->launches += 1;
    GLS_CUDA(cudaEventRecord(pl->ev_conv[b], pl->cvt));
    return GLS_OK;
  };
  if (side) {  // block 0 has the GPU to itself
    Timed tm(pl, &pl->t_convert);
    GLS_CUDA(gls::mixed_convert(pl->mixed, side_src(0), ldx, blocks[0].second, cs, 0, 0));
    pl->launches += 1;
  }

  if (staged) GLS_TRY(issue_load(0));
  for (size_t jb = 0; jb < blocks.size(); ++jb) {
    const int s = (int)(jb % 2);
    const int64_t s0 = blocks[jb].first, kb = blocks[jb].second;
    if (staged && jb + 1 < blocks.size()) GLS_TRY(issue_load(jb + 1));
    // queued before block jb's solve, so that the two start together
    if (side && jb + 1 < blocks.size()) GLS_TRY(side_convert(jb + 1));
    if (side && jb >= 1) GLS_CUDA(cudaStreamWaitEvent(cs, pl->ev_conv[s], 0));
    if (direct && ring && !ring->wait_filled(jb)) {
      set_error("reading genotype block %zu from the file failed: %s", jb, strerror(ring->err));
      return GLS_ERR_IO;
    }
    if (staged) GLS_CUDA(cudaStreamWaitEvent(cs, pl->ev_loaded[s], 0));
    GLS_CUDA(cudaStreamWaitEvent(cs, pl->ev_stored[s], 0));  // output slot s copied out
    double* bout = out_b_host ? pl->bdev[s] : B + s0 * t * ldb;
    const int64_t ldout = out_b_host ? p : ldb;
    int32_t* sout = snp_status ? (out_s_host ? pl->sdev[s] : snp_status + s0) : nullptr;
    if (side) {
      const int free_sms = jb + 1 < blocks.size() ? side_sms : 0;
      GLS_TRY(replayed(pl, pl->replays,
                       (KeyHash() << 5u << (uint64_t)s << kb << bout << ldout << sout
                        << (uint64_t)t << (uint64_t)free_sms).h,
                       [&]() {
                         return run_block(pl, nullptr, 0, kb, bout, ldout, sout, nullptr, 0, s,
                                          true, free_sms);
                       }));
    } else if (packed && pl->precision != GLS_PREC_FP64) {
      // the mixed paths convert the packed codes straight to their operand
      const uint8_t* src = (mx == Mem::Device) ? X + s0 * ldx : pl->xp[s];
      const int64_t ld = (mx == Mem::Device) ? ldx : width;
      GLS_TRY(replayed(pl, pl->replays,
                       (KeyHash() << 3u << src << ld << kb << bout << ldout << sout
                        << (uint64_t)t).h,
                       [&]() {
                         return run_block(pl, nullptr, 0, kb, bout, ldout, sout, src, ld);
                       }));
    } else {
      const int8_t* xin;
      int64_t ldin;
      if (packed) {
        // unpack into the int8 staging of slot s (free: the compute stream is in order)
        const uint8_t* src = (mx == Mem::Device) ? X + s0 * ldx : pl->xp[s];
        GLS_CUDA(gls::launch_unpack2(src, (mx == Mem::Device) ? ldx : width, n, kb, pl->xr[s],
                                     n, cs));
        pl->launches += 1;
        xin = pl->xr[s];
        ldin = n;
      } else if (mx == Mem::Device || direct) {
        xin = direct ? reinterpret_cast<const int8_t*>(src_dev(jb))
                     : reinterpret_cast<const int8_t*>(X) + s0 * ldx;
        ldin = ldx;
      } else {
        xin = pl->xr[s];
        ldin = n;
      }
      GLS_TRY(replayed(pl, pl->replays,
                       (KeyHash() << 2u << xin << ldin << kb << bout << ldout << sout
                        << (uint64_t)t).h,
                       [&]() { return run_block(pl, xin, ldin, kb, bout, ldout, sout); }));
    }
    GLS_CUDA(cudaEventRecord(pl->ev_computed[s], cs));
    if (direct && ring) GLS_CUDA(ring->release(jb, cs));  // the conversion has read the slot
    if (out_b_host || out_s_host) {
      GLS_CUDA(cudaStreamWaitEvent(pl->d2h, pl->ev_computed[s], 0));
      if (out_b_host) {
        struct Copy {
          double* dst;
          size_t lddst;
          const double* src;
          size_t rows, cols;
          cudaStream_t st;
        };
        auto issue = [](void* c) -> cudaError_t {
          const Copy& q = *static_cast<const Copy*>(c);
          return copy2d(q.dst, q.lddst * sizeof(double), q.src, q.rows * sizeof(double),
                        q.rows * sizeof(double), q.cols, cudaMemcpyDeviceToHost, q.st);
        };
        Copy q = (mb == Mem::Pinned) ? Copy{B + s0 * t * ldb, (size_t)ldb, bout, (size_t)p,
                                            (size_t)(kb * t), pl->d2h}
                                     : Copy{pl->h_b[s], (size_t)p, bout, (size_t)p,
                                            (size_t)(kb * t), pl->d2h};
        GLS_CUDA(timed_copy(pl, &pl->t_d2h, pl->d2h, sizeof(double) * p * kb * t, issue, &q));
      }
      if (out_s_host) {
        int32_t* dst = (ms == Mem::Pinned) ? snp_status + s0 : pl->h_s[s];
        GLS_CUDA(cudaMemcpyAsync(dst, sout, sizeof(int32_t) * kb, cudaMemcpyDeviceToHost,
                                 pl->d2h));
      }
      GLS_CUDA(cudaEventRecord(pl->ev_stored[s], pl->d2h));
    }
    if (jb >= 1) GLS_TRY(finish_host(jb - 1));
  }
  GLS_TRY(finish_host(blocks.size() - 1));
  GLS_TRY(host_wait(pl, pl->h2d));
  GLS_TRY(host_wait(pl, pl->d2h));
  int hf[gls::kFlagCount];
  GLS_TRY(check_flags(pl, hf));
  return GLS_OK;
}

// Common argument checks of the two stream entry points.
gls_status_t stream_args(gls_plan* pl, const void* X, int64_t ldx, int64_t min_ld, int64_t m,
                         const double* B, int64_t ldb, const char* name) {
  if (!pl) {
    set_error("plan is NULL");
    return GLS_ERR_INVALID_ARG;
  }
  if (!pl->factored) {
    set_error("%s before a successful gls_factor", name);
    return GLS_ERR_STATE;
  }
  if (m < 0) {
    set_error("m < 0");
    return GLS_ERR_INVALID_ARG;
  }
  if (m > 0 && (!X || !B || ldx < min_ld || ldb < pl->p)) {
    set_error("bad XR/B pointer or leading dimension");
    return GLS_ERR_INVALID_ARG;
  }
  return GLS_OK;
}

}  // namespace

extern "C" {

gls_status_t gls_solve_stream(gls_plan_t pl, const int8_t* XR, int64_t ldxr, int64_t m,
                              double* B, int64_t ldb, int32_t* snp_status) {
  g_last_error.clear();
  GLS_TRY(stream_args(pl, XR, ldxr, pl ? pl->n : 0, m, B, ldb, "gls_solve_stream"));
  if (m == 0) return GLS_OK;
  return stream_impl(pl, reinterpret_cast<const uint8_t*>(XR), ldxr, false, m, B, ldb,
                     snp_status);
}

gls_status_t gls_solve_stream_packed(gls_plan_t pl, const uint8_t* XP, int64_t ldxp, int64_t m,
                                     double* B, int64_t ldb, int32_t* snp_status) {
  g_last_error.clear();
  GLS_TRY(stream_args(pl, XP, ldxp, pl ? gls::ceil_div(pl->n, 4) : 0, m, B, ldb,
                      "gls_solve_stream_packed"));
  if (m == 0) return GLS_OK;
  return stream_impl(pl, XP, ldxp, true, m, B, ldb, snp_status);
}

gls_status_t gls_solve_file(gls_plan_t pl, const char* path, int64_t offset, int32_t packed,
                            int64_t ldx, int64_t m, double* B, int64_t ldb,
                            int32_t* snp_status) {
  g_last_error.clear();
  if (!path || offset < 0) {
    set_error("path is NULL or offset < 0");
    return GLS_ERR_INVALID_ARG;
  }
  GLS_TRY(stream_args(pl, path, ldx, pl ? (packed ? gls::ceil_div(pl->n, 4) : pl->n) : 0, m, B,
                      ldb, "gls_solve_file"));
  if (m == 0) return GLS_OK;
  DeviceGuard guard(pl->device);
  // the ring's pinned slots and their events stay with the plan for later calls
  const size_t need = (size_t)ldx * (size_t)pl->kmax;
  if (pl->ring_bytes < need) {
    for (int s = 0; s < FileRing::kSlots; ++s) {
      cudaFreeHost(pl->h_ring[s]);
      pl->h_ring[s] = nullptr;
      pl->d_ring[s] = nullptr;
    }
    pl->ring_bytes = 0;
    for (int s = 0; s < FileRing::kSlots; ++s) {
      GLS_TRY(host_alloc(&pl->h_ring[s], need));
      GLS_CUDA(cudaHostGetDevicePointer((void**)&pl->d_ring[s], pl->h_ring[s], 0));
    }
    pl->ring_bytes = need;
  }
  for (int s = 0; s < FileRing::kSlots; ++s)
    if (!pl->ev_ring[s]) GLS_CUDA(cudaEventCreateWithFlags(&pl->ev_ring[s], cudaEventDisableTiming));
  const int fd = open(path, O_RDONLY | O_CLOEXEC);
  if (fd < 0) {
    set_error("cannot open %s: %s", path, strerror(errno));
    return GLS_ERR_IO;
  }
  struct stat sb;
  if (fstat(fd, &sb) != 0 || sb.st_size < offset + m * ldx) {
    set_error("%s holds fewer than offset + m * ldx = %lld bytes", path,
              (long long)(offset + m * ldx));
    close(fd);
    return GLS_ERR_IO;
  }
  posix_fadvise(fd, offset, m * ldx, POSIX_FADV_SEQUENTIAL);
  FileRing ring;
  ring.fd = fd;
  ring.offset = offset;
  ring.ldx = ldx;
  ring.blocks = block_schedule(pl->kmax, m);
  for (int s = 0; s < FileRing::kSlots; ++s) {
    ring.slot[s] = pl->h_ring[s];
    ring.released[s] = pl->ev_ring[s];
  }
  ring.th = std::thread([&ring]() { ring.run(); });
  gls_status_t st = stream_impl(pl, nullptr, ldx, packed != 0, m, B, ldb, snp_status, &ring);
  ring.finish();  // also stops a reader still waiting after an early return
  close(fd);
  if (st == GLS_OK && ring.err) {
    set_error("reading %s failed: %s", path, strerror(ring.err));
    st = GLS_ERR_IO;
  }
  return st;
}

gls_status_t gls_solve_block_packed(gls_plan_t pl, const uint8_t* XP, int64_t ldxp, int64_t k,
                                    double* B, int64_t ldb, int32_t* snp_status) {
  g_last_error.clear();
  if (!pl) {
    set_error("plan is NULL");
    return GLS_ERR_INVALID_ARG;
  }
  if (!pl->factored) {
    set_error("gls_solve_block_packed before a successful gls_factor");
    return GLS_ERR_STATE;
  }
  if (k < 0 || k > pl->kmax) {
    set_error("k = %lld outside [0, max_block_snps = %lld]", (long long)k, (long long)pl->kmax);
    return GLS_ERR_INVALID_ARG;
  }
  if (k == 0) return GLS_OK;
  const int64_t width = gls::ceil_div(pl->n, 4);
  if (!XP || !B || ldxp < width || ldb < pl->p) {
    set_error("bad XP/B pointer or leading dimension");
    return GLS_ERR_INVALID_ARG;
  }
  {
    DeviceGuard guard(pl->device);
    const Mem mx = classify(XP);
    GLS_TRY(packed_staging(pl, false));
    const uint8_t* src = XP;
    int64_t ld = ldxp;
    if (mx != Mem::Device) {
      GLS_CUDA(copy2d(pl->xp[0], width, XP, ldxp, width, k, cudaMemcpyHostToDevice, pl->stream));
      src = pl->xp[0];
      ld = width;
    }
    GLS_CUDA(gls::launch_unpack2(src, ld, pl->n, k, pl->xr[0], pl->n, pl->stream));
    pl->launches += 1;
  }
  // the unpacked block is device-resident int8: the int8 entry point from here
  return gls_solve_block(pl, pl->xr[0], pl->n, k, B, ldb, snp_status);
}

}  // extern "C"

struct gls_batch {
  std::vector<gls_plan*> plans;
  gls::MixedBatch* mb = nullptr;
  int* flags = nullptr;
  int* h_flags = nullptr;  // pinned read-back
  cudaEvent_t ev = nullptr;
  int device = 0;
  ReplayCache replays;  // rounds captured on the first plan's stream
};

extern "C" {

gls_status_t gls_batch_create(const gls_plan_t* plans, int32_t nplans, gls_batch_t* out) {
  g_last_error.clear();
  if (!out) {
    set_error("out is NULL");
    return GLS_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (!plans || nplans < 1 || nplans > gls::kMaxBatch) {
    set_error("nplans must be in [1, %d]", gls::kMaxBatch);
    return GLS_ERR_INVALID_ARG;
  }
  for (int i = 0; i < nplans; ++i) {
    if (!plans[i] || plans[i]->precision == GLS_PREC_FP64 || !plans[i]->mixed) {
      set_error("plan %d is NULL or not a mixed-precision plan", i);
      return GLS_ERR_INVALID_ARG;
    }
    if (plans[i]->device != plans[0]->device) {
      set_error("plans of a batch must share one device");
      return GLS_ERR_INVALID_ARG;
    }
  }
  DeviceGuard guard(plans[0]->device);
  std::vector<gls::MixedState*> st(nplans);
  std::vector<const double*> pbr(nplans), glin(nplans);
  std::vector<int64_t> ldp(nplans);
  for (int i = 0; i < nplans; ++i) {
    st[i] = plans[i]->mixed;
    pbr[i] = plans[i]->partials;
    glin[i] = plans[i]->partials + (int64_t)plans[i]->nI * plans[i]->ldp;
    ldp[i] = plans[i]->ldp;
  }
  gls_batch* b = new gls_batch();
  b->device = plans[0]->device;
  b->plans.assign(plans, plans + nplans);
  gls_status_t s = gls::mixed_batch_create(st.data(), pbr.data(), glin.data(), ldp.data(), nplans,
                                           &b->mb);
  if (s != GLS_OK) {
    set_error("%s", gls::mixed_last_error());
    delete b;
    return s;
  }
  if (cudaMalloc(&b->flags, sizeof(int) * gls::kFlagCount) != cudaSuccess ||
      cudaMemset(b->flags, 0, sizeof(int) * gls::kFlagCount) != cudaSuccess ||
      cudaMallocHost(&b->h_flags, sizeof(int) * gls::kFlagCount) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    gls::mixed_batch_free(b->mb);
    cudaFree(b->flags);
    cudaFreeHost(b->h_flags);
    delete b;
    set_error("batch allocation failed");
    return GLS_ERR_OOM;
  }
  *out = b;
  return GLS_OK;
}

gls_status_t gls_batch_solve(gls_batch_t b, const int8_t* const* XR, const int64_t* ldxr,
                             const int64_t* k, double* const* B, const int64_t* ldb,
                             int32_t* const* snp_status, int32_t group) {
  g_last_error.clear();
  if (!b || !XR || !ldxr || !k || !B || !ldb || group < 0) {
    set_error("NULL batch or argument array, or negative group");
    return GLS_ERR_INVALID_ARG;
  }
  const int count = (int)b->plans.size();
  for (int i = 0; i < count; ++i) {
    gls_plan* pl = b->plans[i];
    if (!pl->factored) {
      set_error("plan %d of the batch has no successful gls_factor", i);
      return GLS_ERR_STATE;
    }
    if (k[i] < 0 || k[i] > pl->kmax) {
      set_error("k[%d] = %lld outside [0, max_block_snps]", i, (long long)k[i]);
      return GLS_ERR_INVALID_ARG;
    }
    if (k[i] == 0) continue;
    if (!XR[i] || !B[i] || ldxr[i] < pl->n || ldb[i] < pl->p) {
      set_error("plan %d: bad XR/B pointer or leading dimension", i);
      return GLS_ERR_INVALID_ARG;
    }
    if (classify(XR[i]) != Mem::Device || classify(B[i]) != Mem::Device ||
        (snp_status && snp_status[i] && classify(snp_status[i]) != Mem::Device)) {
      set_error("plan %d: batched solves take device buffers only", i);
      return GLS_ERR_INVALID_ARG;
    }
  }
  DeviceGuard guard(b->device);
  gls_plan* p0 = b->plans[0];
  cudaStream_t st = p0->stream;
  // order after the work already queued on every plan's stream
  for (int i = 1; i < count; ++i) {
    GLS_CUDA(cudaEventRecord(b->ev, b->plans[i]->stream));
    GLS_CUDA(cudaStreamWaitEvent(st, b->ev, 0));
  }
  KeyHash key;
  key << 3u << (uint64_t)group;
  for (int i = 0; i < count; ++i)
    key << XR[i] << ldxr[i] << k[i] << B[i] << ldb[i]
        << (snp_status ? (const void*)snp_status[i] : nullptr) << (uint64_t)b->plans[i]->t_active;
  // one round: every conversion, the persistent solve over all scans, every
  // p x p assembly; captured as one graph when the same round repeats
  GLS_TRY(replayed(p0, &b->replays, key.h, [&]() -> gls_status_t {
    GLS_CUDA(cudaMemsetAsync(b->flags, 0, sizeof(int) * gls::kFlagCount, st));
    {
      Timed t(p0, &p0->t_convert);
      for (int i = 0; i < count; ++i) {
        if (k[i] == 0) continue;
        GLS_CUDA(gls::mixed_convert(b->plans[i]->mixed, XR[i], ldxr[i], k[i], st));
        p0->launches += 1;
      }
    }
    {
      Timed t(p0, &p0->t_trsm);
      GLS_CUDA(gls::mixed_batch_run(b->mb, k, group, b->flags, st));
      p0->launches += 1;
    }
    Timed t(p0, &p0->t_solve);
    for (int i = 0; i < count; ++i) {
      if (k[i] == 0) continue;
      gls_plan* pl = b->plans[i];
      gls::launch_assemble_solve_split(pl->partials + (int64_t)pl->nI * pl->ldp, pl->partials,
                                       pl->ldp, pl->nI, pl->p, pl->t_active, k[i], pl->RTL,
                                       pl->zT, gls::kTauMixed, B[i], ldb[i],
                                       snp_status ? snp_status[i] : nullptr, st);
      p0->launches += 1;
    }
    GLS_CUDA(cudaGetLastError());
    return GLS_OK;
  }));
  GLS_CUDA(cudaGetLastError());
  GLS_CUDA(cudaEventRecord(b->ev, st));
  for (int i = 1; i < count; ++i) GLS_CUDA(cudaStreamWaitEvent(b->plans[i]->stream, b->ev, 0));
  int hf[gls::kFlagCount];
  GLS_CUDA(cudaMemcpyAsync(b->h_flags, b->flags, sizeof(hf), cudaMemcpyDeviceToHost, st));
  GLS_TRY(host_wait(p0, st));
  memcpy(hf, b->h_flags, sizeof(hf));
  if (hf[gls::kFlagKernel] & gls::kErrTimeout) {
    set_error("a bounded device wait gave up (site %d)", hf[gls::kFlagWhere]);
    return GLS_ERR_TIMEOUT;
  }
  return GLS_OK;
}

gls_status_t gls_batch_destroy(gls_batch_t b) {
  g_last_error.clear();
  if (!b) return GLS_OK;
  DeviceGuard guard(b->device);
  if (!b->plans.empty()) cudaStreamSynchronize(b->plans[0]->stream);
  b->replays.items.clear();
  gls::mixed_batch_free(b->mb);
  cudaFree(b->flags);
  cudaFreeHost(b->h_flags);
  if (b->ev) cudaEventDestroy(b->ev);
  cudaGetLastError();
  delete b;
  return GLS_OK;
}

gls_status_t gls_synchronize(gls_plan_t pl) {
  g_last_error.clear();
  if (!pl) {
    set_error("plan is NULL");
    return GLS_ERR_INVALID_ARG;
  }
  DeviceGuard guard(pl->device);
  GLS_TRY(host_wait(pl, pl->h2d));
  GLS_TRY(host_wait(pl, pl->d2h));
  int hf[gls::kFlagCount];
  return check_flags(pl, hf);
}

void* gls_plan_stream(gls_plan_t pl) { return pl ? (void*)pl->stream : nullptr; }

int32_t gls_plan_operand_precision(gls_plan_t pl) {
  if (!pl) return -1;
  if (pl->precision == GLS_PREC_FP64) return GLS_PREC_FP64;
  return gls::mixed_is_bf16(pl->mixed) ? GLS_PREC_MIXED_BF16 : GLS_PREC_MIXED_FP16;
}

gls_status_t gls_plan_wait_event(gls_plan_t pl, void* event) {
  g_last_error.clear();
  if (!pl || !event) {
    set_error("plan or event is NULL");
    return GLS_ERR_INVALID_ARG;
  }
  DeviceGuard guard(pl->device);
  // every device input is read on the compute stream; the side streams of a
  // stream call start after the compute stream's earlier work
  GLS_CUDA(cudaStreamWaitEvent(pl->stream, (cudaEvent_t)event, 0));
  return GLS_OK;
}

gls_status_t gls_plan_set_timing(gls_plan_t pl, int32_t enable) {
  g_last_error.clear();
  if (!pl) {
    set_error("plan is NULL");
    return GLS_ERR_INVALID_ARG;
  }
  DeviceGuard guard(pl->device);
  GLS_CUDA(cudaStreamSynchronize(pl->stream));
  GLS_CUDA(cudaStreamSynchronize(pl->h2d));
  GLS_CUDA(cudaStreamSynchronize(pl->d2h));
  for (gls_plan::Slot* sl :
       {&pl->t_trsm, &pl->t_convert, &pl->t_solve, &pl->t_factor, &pl->t_h2d, &pl->t_d2h}) {
    for (auto& pr : sl->pending) {
      pl->event_pool.push_back(pr.first);
      pl->event_pool.push_back(pr.second);
    }
    sl->pending.clear();
    sl->ms = 0.0;
    sl->launches = 0;
    sl->bytes = 0;
  }
  pl->launches = 0;
  pl->timing = enable != 0;
  return GLS_OK;
}

gls_status_t gls_plan_stats(gls_plan_t pl, gls_stats_t* out) {
  g_last_error.clear();
  if (!pl || !out) {
    set_error("plan or out is NULL");
    return GLS_ERR_INVALID_ARG;
  }
  DeviceGuard guard(pl->device);
  GLS_CUDA(cudaStreamSynchronize(pl->stream));
  GLS_CUDA(cudaStreamSynchronize(pl->h2d));
  GLS_CUDA(cudaStreamSynchronize(pl->d2h));
  for (gls_plan::Slot* sl :
       {&pl->t_trsm, &pl->t_convert, &pl->t_solve, &pl->t_factor, &pl->t_h2d, &pl->t_d2h}) {
    for (auto& pr : sl->pending) {
      float ms = 0.f;
      GLS_CUDA(cudaEventElapsedTime(&ms, pr.first, pr.second));
      sl->ms += ms;
      sl->launches += 1;
      pl->event_pool.push_back(pr.first);
      pl->event_pool.push_back(pr.second);
    }
    sl->pending.clear();
  }
  out->launches = pl->launches;
  out->trsm_ms = pl->t_trsm.ms;
  out->trsm_launches = pl->t_trsm.launches;
  out->convert_ms = pl->t_convert.ms;
  out->convert_launches = pl->t_convert.launches;
  out->solve_ms = pl->t_solve.ms;
  out->solve_launches = pl->t_solve.launches;
  out->factor_ms = pl->t_factor.ms;
  out->factor_calls = pl->t_factor.launches;
  out->h2d_ms = pl->t_h2d.ms;
  out->h2d_bytes = pl->t_h2d.bytes;
  out->h2d_copies = pl->t_h2d.launches;
  out->d2h_ms = pl->t_d2h.ms;
  out->d2h_bytes = pl->t_d2h.bytes;
  out->d2h_copies = pl->t_d2h.launches;
  return GLS_OK;
}

gls_status_t gls_destroy(gls_plan_t pl) {
  g_last_error.clear();
  if (!pl) return GLS_OK;
  DeviceGuard guard(pl->device);
  free_plan(pl);
  return GLS_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ Alg. 3, 4, 6
namespace {

// Device workspace of one gls_solve_variant call, freed when it goes out of scope.
struct DevBuf {
  double* p = nullptr;
  ~DevBuf() { cudaFree(p); }
};

}  // namespace

extern "C" gls_status_t gls_solve_variant(gls_plan_t pl, int32_t algorithm, const double* M,
                                          int64_t ldm, const double* XL, int64_t ldxl,
                                          const double* y, const int8_t* XR, int64_t ldxr,
                                          int64_t k, double* B, int64_t ldb,
                                          int32_t* snp_status) {
  g_last_error.clear();
  if (!pl) {
    set_error("plan is NULL");
    return GLS_ERR_INVALID_ARG;
  }
  if (pl->precision != GLS_PREC_FP64 || pl->t != 1) {
    set_error("the comparison algorithms run on binary64 plans with one phenotype");
    return GLS_ERR_INVALID_ARG;
  }
  if (algorithm != GLS_ALG_BLACK_BOX && algorithm != GLS_ALG_SEQ_GLS &&
      algorithm != GLS_ALG_HP_GWAS && algorithm != GLS_ALG_GWFGLS) {
    set_error("unknown algorithm %d", algorithm);
    return GLS_ERR_INVALID_ARG;
  }
  const int64_t n = pl->n, npad = pl->npad;
  const int p = pl->p, q = p - 1;
  if (algorithm != GLS_ALG_HP_GWAS && p > gls::kVarMaxP) {
    set_error("the comparison algorithms take p <= %d", gls::kVarMaxP);
    return GLS_ERR_INVALID_ARG;
  }
  if (k < 0 || !M || !y || (q > 0 && !XL) || (k > 0 && (!XR || !B)) || ldm < n ||
      (q > 0 && ldxl < n) || ldxr < n || ldb < p) {
    set_error("bad size, pointer or leading dimension");
    return GLS_ERR_INVALID_ARG;
  }
  DeviceGuard guard(pl->device);
  for (const void* ptr : {(const void*)M, (const void*)XL, (const void*)y, (const void*)XR,
                          (const void*)B, (const void*)snp_status})
    if (ptr && classify(ptr) != Mem::Device) {
      set_error("the comparison algorithms take device buffers only");
      return GLS_ERR_INVALID_ARG;
    }
  if (k == 0) return GLS_OK;
  if (algorithm == GLS_ALG_HP_GWAS) {  // the library's own path, block by block
    GLS_TRY(gls_factor(pl, M, ldm, XL, ldxl, y, nullptr));
    for (int64_t j0 = 0; j0 < k; j0 += pl->kmax) {
      const int64_t kb = std::min(pl->kmax, k - j0);
      GLS_TRY(gls_solve_block(pl, XR + j0 * ldxr, ldxr, kb, B + j0 * ldb, ldb,
                              snp_status ? snp_status + j0 : nullptr));
    }
    return gls_synchronize(pl);
  }
  cudaStream_t st = pl->stream;
  pl->factored = pl->has_factor = false;  // A and Z are overwritten below
  GLS_CUDA(cudaMemsetAsync(pl->flags, 0, sizeof(int) * gls::kFlagCount, st));
  auto factor = [&]() -> gls_status_t {
    GLS_CUDA(copy2d(pl->A, npad * sizeof(double), M, ldm * sizeof(double), n * sizeof(double), n,
                    cudaMemcpyDeviceToDevice, st));
    gls::launch_pad_lower(pl->A, npad, n, npad, st);
    gls::launch_identity(pl->Z, npad, npad, st);
    GLS_CUDA(gls::potrf_trtri_fp64(pl->A, pl->Z, npad, npad, pl->flags, st));
    return GLS_OK;
  };
  auto alloc = [&](DevBuf& b, size_t count) -> gls_status_t {
    return dev_alloc(&b.p, count);
  };
  DevBuf R, Ws, yt, Mi, WL, F, bT, P;
  if (algorithm == GLS_ALG_BLACK_BOX) {
    // every problem from scratch: potrf of M, [X_L | x_j | y] whitened, syrk, gemv, posv
    GLS_TRY(alloc(R, (size_t)npad * (p + 1)));
    GLS_TRY(alloc(Ws, (size_t)npad * (p + 1)));
    for (int64_t j = 0; j < k; ++j) {
      GLS_TRY(factor());
      gls::launch_variant_rhs(XL, ldxl, y, XR, ldxr, j, 1, n, npad, p, 0, R.p, npad, st);
      gls::launch_whiten(pl->Z, npad, n, npad, R.p, npad, p + 1, Ws.p, npad, pl->flags, st);
      gls::launch_gram_posv(Ws.p, npad, n, p, 0, 1, Ws.p + (int64_t)p * npad, gls::kTauFP64,
                            B + j * ldb, ldb, snp_status ? snp_status + j : nullptr, st);
      GLS_CUDA(cudaGetLastError());
    }
  } else if (algorithm == GLS_ALG_SEQ_GLS) {
    // potrf and y~ once; per problem the whole X_i = [X_L | x_j] whitened
    const int g = std::max(1, gls::kMaxP / p);  // problems per whitening launch
    GLS_TRY(alloc(R, (size_t)npad * p * g));
    GLS_TRY(alloc(Ws, (size_t)npad * p * g));
    GLS_TRY(alloc(yt, (size_t)npad));
    GLS_TRY(factor());
    gls::launch_whiten(pl->Z, npad, n, npad, y, n, 1, yt.p, npad, pl->flags, st);
    for (int64_t j0 = 0; j0 < k; j0 += g) {
      const int gg = (int)std::min<int64_t>(g, k - j0);
      gls::launch_variant_rhs(XL, ldxl, y, XR, ldxr, j0, gg, n, npad, p, 1, R.p, npad, st);
      gls::launch_whiten(pl->Z, npad, n, npad, R.p, npad, p * gg, Ws.p, npad, pl->flags, st);
      gls::launch_gram_posv(Ws.p, npad, n, p, p, gg, yt.p, gls::kTauFP64, B + j0 * ldb, ldb,
                            snp_status ? snp_status + j0 : nullptr, st);
      GLS_CUDA(cudaGetLastError());
    }
  } else {  // GLS_ALG_GWFGLS
    // M^{-1} = Z^T Z and W_L = M^{-1} X_L once; per problem w = M^{-1} x_j, the
    // unsymmetric S = (W_L | w)^T (X_L | x_j), r = (W_L | w)^T y, gesv
    const int64_t kb_max = std::min<int64_t>(k, 16384);
    const int nI = (int)gls::ceil_div(n, 64);
    GLS_TRY(alloc(Mi, (size_t)npad * n));
    GLS_TRY(alloc(WL, (size_t)npad * std::max(q, 1)));
    GLS_TRY(alloc(F, (size_t)std::max(q * q, 1)));
    GLS_TRY(alloc(bT, (size_t)std::max(q, 1)));
    GLS_TRY(alloc(P, (size_t)nI * (2 * q + 2) * kb_max));
    GLS_TRY(factor());
    gls::launch_gemm_tn(pl->Z, npad, pl->Z, npad, Mi.p, npad, n, n, npad, st);
    if (q > 0) {
      gls::launch_gemm_tn(Mi.p, npad, XL, ldxl, WL.p, npad, n, q, n, st);
      gls::launch_gemm_tn(WL.p, npad, XL, ldxl, F.p, q, q, q, n, st);
      gls::launch_gemm_tn(WL.p, npad, y, n, bT.p, q, q, 1, n, st);
    }
    for (int64_t j0 = 0; j0 < k; j0 += kb_max) {
      const int64_t kb = std::min(kb_max, k - j0);
      gls::launch_dense_gram(Mi.p, npad, n, XR + j0 * ldxr, ldxr, kb, XL, ldxl, WL.p, npad, y,
                             q, P.p, kb, st);
      gls::launch_gesv(P.p, kb, nI, q, kb, F.p, std::max(q, 1), bT.p, gls::kTauFP64,
                       B + j0 * ldb, ldb, snp_status ? snp_status + j0 : nullptr, st);
      GLS_CUDA(cudaGetLastError());
    }
  }
  int hf[gls::kFlagCount];
  GLS_TRY(check_flags(pl, hf));
  if (hf[gls::kFlagPotrf] != 0) {
    set_error("M is not positive definite (pivot %d)", hf[gls::kFlagPotrf]);
    return GLS_ERR_NOT_SPD;
  }
  return GLS_OK;
}
