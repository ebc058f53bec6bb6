// The C ABI (include/stc.h): argument checks, the key plan, stream-ordered memory, and the
// order of the stages of one contraction.
#include <algorithm>
#include <atomic>
#include <memory>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <set>
#include <mutex>
#include <string>
#include <vector>

#include "launch.h"

using namespace stc;

// Autotuning of batches: per size bucket, each candidate is timed once with CUDA events around
// the accumulation kernels, read back without a sync on a later call of the same bucket; then
// the fastest is kept. A candidate sets three things: the group load factor (table sizes), the
// largest table a group may get in a warp of its own (group-per-warp granularity: groups above
// it take a CTA), and the expansion split of the CTA tables (products per lane per round).
struct TuneChoice {
  double alpha;
  int warp_max;  // slots of the largest warp-sized table used (256 or 1024)
  int depth;     // 0: the default expansion split, 1: half as many products per lane per round
};
constexpr TuneChoice kTune[] = {{0.5, 1024, 0}, {0.75, 1024, 0}, {0.9, 1024, 0}, {0.75, 256, 0}, {0.75, 1024, 1}};
constexpr int kTuneCand = 5;
constexpr TuneChoice kTuneDefault = {0.75, 1024, 0};
struct TuneEntry {
  int best = -1;
  float ms[kTuneCand] = {};
  bool done[kTuneCand] = {};
  bool pending[kTuneCand] = {};   // handed to a batch, not yet read back
  bool recorded[kTuneCand] = {};  // that batch has recorded both events
  cudaEvent_t ev0[kTuneCand] = {}, ev1[kTuneCand] = {};
};

struct stc_ctx {
  int device = 0;
  size_t budget = 0;  // 0 = no cap
  cudaMemPool_t pool = nullptr;
  std::atomic<size_t> held{0};
  std::atomic<int64_t> live_results{0};
  int sms = 0;
  std::mutex tune_mu;
  std::map<int, TuneEntry> tune;
  // Problem shapes (shape_signature) whose last run here averaged at least kRowsMinPerOutput
  // products per output cell with output rows of at most kLaneRowMax keys: AUTO then groups X
  // and takes the lane-private dense rows for them (the product count is only known after the
  // survey, and the one-global-table path for small output key spaces never waits for it).
  std::mutex rows_mu;
  std::set<uint64_t> rows_shapes;
};

namespace {
// Picks the load factor for a batch of this bucket; *measure is the candidate to time (or -1).
TuneChoice tune_pick(stc_ctx* ctx, int bucket, int* measure) {
  std::lock_guard<std::mutex> lk(ctx->tune_mu);
  TuneEntry& te = ctx->tune[bucket];
  *measure = -1;
  if (te.best >= 0) return kTune[te.best];
  // Only candidates whose batch has recorded both events are read: a batch of another thread
  // may still be between picking a candidate and recording its events (an event never
  // recorded reads as complete). A failed read is cleared so that it cannot surface as the
  // error of a later call on this thread, and the candidate is timed again.
  for (int c = 0; c < kTuneCand; c++) {
    if (!te.pending[c] || !te.recorded[c]) continue;
    const cudaError_t q = cudaEventQuery(te.ev1[c]);
    if (q == cudaErrorNotReady) {
      cudaGetLastError();
      continue;
    }
    const cudaError_t e = q == cudaSuccess ? cudaEventElapsedTime(&te.ms[c], te.ev0[c], te.ev1[c]) : q;
    if (e != cudaSuccess) cudaGetLastError();
    te.pending[c] = false;
    te.recorded[c] = false;
    te.done[c] = e == cudaSuccess;
  }
  int best = 0;
  bool all = true;
  for (int c = 0; c < kTuneCand; c++) {
    all = all && te.done[c];
    if (te.done[c] && te.ms[c] < te.ms[best]) best = c;
    if (te.done[c] && !te.done[best]) best = c;
  }
  if (all) {
    te.best = best;
    return kTune[best];
  }
  for (int c = 0; c < kTuneCand; c++) {
    if (!te.done[c] && !te.pending[c]) {
      if (!te.ev1[c]) {
        cudaEvent_t a = nullptr, b = nullptr;
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
          cudaGetLastError();
          if (a) cudaEventDestroy(a);
          return kTuneDefault;  // untimed
        }
        te.ev0[c] = a;
        te.ev1[c] = b;
      }
      *measure = c;
      te.pending[c] = true;
      te.recorded[c] = false;
      return kTune[c];
    }
  }
  return kTuneDefault;  // every remaining candidate is still being timed
}
void tune_mark(stc_ctx* ctx, int bucket, int cand, bool end, cudaStream_t s) {
  if (cand < 0) return;
  std::lock_guard<std::mutex> lk(ctx->tune_mu);
  TuneEntry& te = ctx->tune[bucket];
  if (cudaEventRecord(end ? te.ev1[cand] : te.ev0[cand], s) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  if (end) te.recorded[cand] = true;
}
// A batch that failed after picking a candidate gives it back.
void tune_abort(stc_ctx* ctx, int bucket, int cand) {
  if (cand < 0) return;
  std::lock_guard<std::mutex> lk(ctx->tune_mu);
  ctx->tune[bucket].pending[cand] = false;
  ctx->tune[bucket].recorded[cand] = false;
}
int log2_floor(uint64_t v) { return v ? 63 - __builtin_clzll(v) : 0; }
}  // namespace

// Device memory owned by one or more results (a batch's results share one block); returned to
// the context's pool, in the order of the stream it was made on, when the last owner goes.
struct DeviceBlock {
  stc_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<std::pair<void*, size_t>> parts;
  ~DeviceBlock();
};

struct stc_result {
  stc_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  int64_t nnz = 0;
  int32_t order = 0;
  std::vector<int64_t> shape;
  int32_t* coords = nullptr;  // coordinates, or with keys_form the output keys (2 words each)
  double* vals = nullptr;
  bool keys_form = false;
  std::shared_ptr<DeviceBlock> mem;
  stc_stats stats{};
};

namespace {

thread_local std::string g_last_error;

stc_status fail(stc_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

#define STC_CUDA(expr)                                                                          \
  do {                                                                                          \
    const cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess)                                                                      \
      return fail(STC_ERR_CUDA, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

#define STC_TRY(expr)                    \
  do {                                   \
    const stc_status s_ = (expr);        \
    if (s_ != STC_OK) return s_;         \
  } while (0)

// Makes the context's device current for the duration of a call, then restores the caller's.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && (prev == dev || cudaSetDevice(dev) == cudaSuccess)) ok = true;
  }
  ~DeviceGuard() {
    if (ok && prev >= 0) cudaSetDevice(prev);
  }
};

// Stream-ordered scratch from the context's pool. Everything still held when the arena
// dies is returned to the pool in stream order; `keep` hands a block to a result instead.
struct Arena {
  stc_ctx* ctx;
  cudaStream_t s;
  struct Block { void* p; size_t bytes; };
  std::vector<Block> blocks;
  Arena(stc_ctx* c, cudaStream_t st) : ctx(c), s(st) {}
  ~Arena() {
    for (auto& b : blocks) {
      cudaFreeAsync(b.p, s);
      ctx->held -= b.bytes;
    }
  }
  template <typename T>
  stc_status alloc(T** out, size_t count) {
    *out = nullptr;
    const size_t bytes = count * sizeof(T);
    if (bytes == 0) return STC_OK;
    const size_t after = ctx->held.fetch_add(bytes) + bytes;
    if (ctx->budget && after > ctx->budget) {
      ctx->held -= bytes;
      return fail(STC_ERR_OUT_OF_MEMORY, "request of %zu bytes exceeds the context budget (%zu of %zu held)", bytes,
                  after - bytes, ctx->budget);
    }
    void* p = nullptr;
    const cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, ctx->pool, s);
    if (e != cudaSuccess) {
      ctx->held -= bytes;
      cudaGetLastError();
      return fail(STC_ERR_OUT_OF_MEMORY, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    blocks.push_back({p, bytes});
    *out = static_cast<T*>(p);
    return STC_OK;
  }
  size_t keep(void* p) {
    for (size_t i = 0; i < blocks.size(); i++)
      if (blocks[i].p == p) {
        const size_t b = blocks[i].bytes;
        blocks.erase(blocks.begin() + i);
        return b;
      }
    return 0;
  }
};

bool is_pow2(uint64_t v) { return v && !(v & (v - 1)); }

// Output key spaces up to this size take the one-global-table strategy without a host read
// between the survey and the expansion: table and output sized from F (16 MB of table at most).
constexpr uint64_t kGlobalFromF = 1ull << 18;
// Lane-private dense rows (STC_ACC_ROWS): output rows of at most this many free keys, chosen by
// AUTO when the products average at least kRowsMinPerOutput per output cell.
constexpr uint64_t kLaneRowMax = 64;
constexpr uint64_t kRowsMinPerOutput = 64;
// Lanes that probe the one global table together when stc_opts.probe is 0.
constexpr int kDefaultProbe = 1;

// Moves the listed blocks from an arena into a shared block that results can own.
std::shared_ptr<DeviceBlock> adopt(Arena& ar, stc_ctx* ctx, cudaStream_t s, std::initializer_list<void*> ptrs) {
  auto blk = std::make_shared<DeviceBlock>();
  blk->ctx = ctx;
  blk->stream = s;
  for (void* p : ptrs)
    if (p) blk->parts.push_back({p, ar.keep(p)});
  return blk;
}

uint64_t pow2_at_least(uint64_t v) {
  uint64_t c = 1;
  while (c < v) c <<= 1;
  return c;
}

uint32_t log2_u64(uint64_t v) {
  uint32_t r = 0;
  while (v > 1) v >>= 1, r++;
  return r;
}

// The key plan of a contraction (Section 2.4.1 LN keys; the output mode order of Eq. 4).
struct Plan {
  KeyPlan kx{}, ky{};
  OutPlan op{};
  uint64_t K = 1, FX = 1, FY = 1, F = 1;
  int32_t oz = 0;
  int32_t ocols = 0;      // int32 words per output entry: oz, or 2 for a 64-bit output key
  bool keys_out = false;  // outputs are keys (row-major over the output shape), not coordinates
  std::vector<int64_t> zshape;
};

stc_status check_coo(const stc_coo* t, const char* name) {
  if (!t) return fail(STC_ERR_INVALID_ARG, "%s is NULL", name);
  if (t->order < 0 || t->order > STC_MAX_ORDER)
    return fail(STC_ERR_INVALID_ARG, "%s.order = %d outside 0..%d", name, t->order, STC_MAX_ORDER);
  if (t->order > 0 && !t->shape) return fail(STC_ERR_INVALID_ARG, "%s.shape is NULL", name);
  for (int j = 0; j < t->order; j++)
    if (t->shape[j] < 1 || t->shape[j] > (int64_t)1 << 31)
      return fail(STC_ERR_INVALID_ARG, "%s.shape[%d] = %lld outside 1..2^31", name, j, (long long)t->shape[j]);
  if (t->nnz < 0 || t->nnz > STC_MAX_NNZ)
    return fail(STC_ERR_INVALID_ARG, "%s.nnz = %lld outside 0..%lld", name, (long long)t->nnz, STC_MAX_NNZ);
  if (t->nnz > 0 && (!t->vals || (t->order > 0 && !t->coords)))
    return fail(STC_ERR_INVALID_ARG, "%s has nnz > 0 but NULL coords or vals", name);
  return STC_OK;
}

// keys_out: outputs as 64-bit keys. xfree_sizes: when X is the split form of a tensor in key
// form, the lengths of that tensor's free modes, which the output's X part then has (the split
// form's free key is already the row-major index over them).
stc_status make_plan(const stc_coo* X, const stc_coo* Y, int32_t m, const int32_t* cx, const int32_t* cy,
                     const int32_t* out_order, Plan& pl, bool keys_out = false,
                     const std::vector<int64_t>* xfree_sizes = nullptr) {
  STC_TRY(check_coo(X, "X"));
  STC_TRY(check_coo(Y, "Y"));
  if (m < 0 || m > X->order || m > Y->order)
    return fail(STC_ERR_INVALID_ARG, "ncontract = %d outside 0..min(%d, %d)", m, X->order, Y->order);
  if (m > 0 && (!cx || !cy)) return fail(STC_ERR_INVALID_ARG, "cx or cy is NULL");
  bool xc[STC_MAX_ORDER] = {}, yc[STC_MAX_ORDER] = {};
  for (int i = 0; i < m; i++) {
    if (cx[i] < 0 || cx[i] >= X->order || cy[i] < 0 || cy[i] >= Y->order)
      return fail(STC_ERR_INVALID_ARG, "contract pair %d = (%d, %d) out of range", i, cx[i], cy[i]);
    if (xc[cx[i]] || yc[cy[i]]) return fail(STC_ERR_INVALID_ARG, "a mode is listed twice in cx or cy");
    xc[cx[i]] = yc[cy[i]] = true;
  }
  for (int i = 0; i < m; i++)
    if (X->shape[cx[i]] != Y->shape[cy[i]])
      return fail(STC_ERR_SHAPE_MISMATCH, "X mode %d has length %lld but Y mode %d has length %lld", cx[i],
                  (long long)X->shape[cx[i]], cy[i], (long long)Y->shape[cy[i]]);

  pl.kx = KeyPlan{};
  pl.ky = KeyPlan{};
  pl.kx.order = X->order;
  pl.ky.order = Y->order;
  pl.kx.nseg = pl.ky.nseg = 1;
  for (int j = 0; j < X->order; j++) pl.kx.size[j] = X->shape[j];
  for (int j = 0; j < Y->order; j++) pl.ky.size[j] = Y->shape[j];

  // Contract key: row-major over the contract list, first listed pair most significant.
  unsigned __int128 acc = 1;
  for (int i = m - 1; i >= 0; i--) {
    pl.kx.cstride[cx[i]] = (uint64_t)acc;
    pl.ky.cstride[cy[i]] = (uint64_t)acc;
    acc *= (unsigned __int128)X->shape[cx[i]];
    if (acc > (unsigned __int128)UINT64_MAX) return fail(STC_ERR_KEY_OVERFLOW, "contract key space exceeds 2^64");
  }
  pl.K = (uint64_t)acc;

  // Free keys: row-major over the free modes in ascending order.
  std::vector<int> xf, yf;
  for (int j = 0; j < X->order; j++)
    if (!xc[j]) xf.push_back(j);
  for (int j = 0; j < Y->order; j++)
    if (!yc[j]) yf.push_back(j);
  acc = 1;
  for (int a = (int)xf.size() - 1; a >= 0; a--) {
    pl.kx.fstride[xf[a]] = (uint64_t)acc;
    acc *= (unsigned __int128)X->shape[xf[a]];
    if (acc > (unsigned __int128)UINT64_MAX) return fail(STC_ERR_KEY_OVERFLOW, "X free key space exceeds 2^64");
  }
  pl.FX = (uint64_t)acc;
  acc = 1;
  for (int b = (int)yf.size() - 1; b >= 0; b--) {
    pl.ky.fstride[yf[b]] = (uint64_t)acc;
    acc *= (unsigned __int128)Y->shape[yf[b]];
    if (acc > (unsigned __int128)UINT64_MAX) return fail(STC_ERR_KEY_OVERFLOW, "Y free key space exceeds 2^64");
  }
  pl.FY = (uint64_t)acc;
  const unsigned __int128 F = (unsigned __int128)pl.FX * pl.FY;
  // The all-ones key marks empty table slots, so the largest usable key is 2^64 - 2.
  if (F > (unsigned __int128)(UINT64_MAX - 1)) return fail(STC_ERR_KEY_OVERFLOW, "output key space exceeds 2^64 - 1");
  pl.F = (uint64_t)F;

  // Output: the concatenation (X free, Y free) is row-major in zkey = fX * FY + fY.
  std::vector<uint64_t> xs;
  if (xfree_sizes) {
    unsigned __int128 fx = 1;
    for (int64_t v : *xfree_sizes) xs.push_back((uint64_t)v), fx *= (unsigned __int128)v;
    if (fx > (unsigned __int128)pl.FX) return fail(STC_ERR_INVALID_ARG, "free modes do not fit the split key");
    const unsigned __int128 F2 = fx * pl.FY;
    if (F2 > (unsigned __int128)(UINT64_MAX - 1)) return fail(STC_ERR_KEY_OVERFLOW, "output key space exceeds 2^64 - 1");
    pl.F = (uint64_t)F2;
  } else {
    for (int a : xf) xs.push_back((uint64_t)X->shape[a]);
  }
  pl.oz = (int32_t)(xs.size() + yf.size());
  std::vector<uint64_t> csize(pl.oz), cstr(pl.oz);
  for (size_t a = 0; a < xs.size(); a++) csize[a] = xs[a];
  for (size_t b = 0; b < yf.size(); b++) csize[xs.size() + b] = (uint64_t)Y->shape[yf[b]];
  uint64_t st = 1;
  for (int t = pl.oz - 1; t >= 0; t--) {
    cstr[t] = st;
    st *= csize[t];
  }
  if (out_order) {
    std::vector<int> seen(pl.oz, 0);
    for (int q = 0; q < pl.oz; q++) {
      if (out_order[q] < 0 || out_order[q] >= pl.oz || seen[out_order[q]])
        return fail(STC_ERR_INVALID_ARG, "out_order is not a permutation of 0..%d", pl.oz - 1);
      seen[out_order[q]] = 1;
    }
  }
  pl.op = OutPlan{};
  pl.op.order = pl.oz;
  pl.op.pow2 = 1;
  pl.op.z32 = pl.F <= (1ull << 32);
  pl.op.ident = 1;
  pl.zshape.assign(pl.oz, 0);
  std::vector<int> pos_of(pl.oz);  // output position of concatenated mode t
  for (int q = 0; q < pl.oz; q++) {
    const int t = out_order ? out_order[q] : q;
    pos_of[t] = q;
    if (t != q) pl.op.ident = 0;
    pl.op.mod[q] = csize[t];
    pl.zshape[q] = (int64_t)csize[t];
    if (!is_pow2(csize[t])) pl.op.pow2 = 0;
  }
  for (int q = 0; q < pl.oz; q++) {
    const int t = out_order ? out_order[q] : q;
    pl.op.shift[q] = pl.op.pow2 ? log2_u64(cstr[t]) : 0;
  }
  // Digits least significant first: the last concatenated mode is the lowest digit.
  for (int j = 0; j < pl.oz; j++) {
    const int t = pl.oz - 1 - j;
    const uint64_t d = csize[t];
    const uint32_t l = d <= 1 ? 0 : 64 - (uint32_t)__builtin_clzll(d - 1);  // ceil(log2 d)
    const unsigned N = pl.op.z32 ? 32 : 64;
    const unsigned __int128 num = ((unsigned __int128)(((unsigned __int128)1 << l) - d)) << N;
    pl.op.magic[j] = (uint64_t)(num / d + 1);
    pl.op.dpos[j] = (uint8_t)pos_of[t];
    pl.op.dsh1[j] = (uint8_t)(l < 1 ? l : 1);
    pl.op.dsh2[j] = (uint8_t)(l > 1 ? l - 1 : 0);
  }
  pl.ocols = pl.oz;
  pl.keys_out = keys_out;
  if (keys_out) {
    // The key itself, written by every output writer as two 32-bit "coordinates": the low and
    // the high half of zkey (a power-of-two plan of radix 2^32), i.e. one little-endian uint64.
    if (!pl.op.ident) return fail(STC_ERR_INVALID_ARG, "output_keys needs the output modes in concatenation order");
    OutPlan k{};
    k.order = 2;
    k.pow2 = 1;
    k.z32 = 0;
    k.ident = 1;
    k.mod[0] = k.mod[1] = 1ull << 32;
    k.shift[0] = 0;
    k.shift[1] = 32;
    pl.op = k;
    pl.ocols = 2;
  }
  return STC_OK;
}

stc_status status_word(uint32_t st) {
  if (st & kStatCoordRange) return fail(STC_ERR_COORD_OUT_OF_RANGE, "an input coordinate is outside its mode");
  if (st & kStatTableFull) return fail(STC_ERR_TABLE_FULL, "an accumulation table overflowed");
  if (st & kStatOutOverflow) return fail(STC_ERR_TABLE_FULL, "output capacity exceeded");
  if (st & kStatTimeout) return fail(STC_ERR_TIMEOUT, "a bounded wait gave up");
  if (st & kStatTooLarge) return fail(STC_ERR_UNSUPPORTED, "one X free group needs a table above 2^31 slots");
  return STC_OK;
}

// Small device counters of one call, in one allocation so one memset clears them.
struct Counters {
  u64 P;           // products
  u64 nz;          // output entries written
  unsigned ns;     // survivors
  uint32_t status; // kStat* bits
};

// Per-stage CUDA events when timing is requested.
struct StageTimer {
  bool on = false;
  cudaStream_t s = nullptr;
  std::vector<cudaEvent_t> ev;
  int stage_of[16] = {};
  void start(bool enable, cudaStream_t st) {
    on = enable;
    s = st;
    if (on) mark(-1);
  }
  void mark(int stage) {
    if (!on) return;
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      on = false;
      return;
    }
    cudaEventRecord(e, s);
    if (ev.size() > 16) {
      cudaEventDestroy(e);
      return;
    }
    if (stage >= 0 && stage < 8 && !ev.empty()) stage_of[ev.size() - 1] = stage;
    ev.push_back(e);
  }
  void collect(stc_stats& stats) {
    if (!on) return;
    if (!ev.empty()) cudaEventSynchronize(ev.back());  // stage times are a diagnostic: wait for them
    for (size_t i = 1; i < ev.size(); i++) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[i - 1], ev[i]);
      const int st = stage_of[i - 1];
      stats.stage_ms[st] += ms;
      stats.nstages = std::max(stats.nstages, st + 1);
    }
  }
  ~StageTimer() {
    for (auto e : ev) cudaEventDestroy(e);
  }
};

// The device state shared by the counting pass and the contraction: Y grouped by contract
// key, and X surveyed against it.
struct Prepared {
  uint32_t* yoff = nullptr;  // [K + 1]
  void* yfk = nullptr;       // [nY], Y free keys in contract-key order (u32 when key32, else u64)
  bool key32 = false;
  double* yv = nullptr;      // [nY]
  Survivors sv{};
  Counters* ctr = nullptr;
  uint32_t* gcnt = nullptr;  // [FX] entries with a Y run per X free key (GROUPED only)
  bool dense = false;        // GROUPED without a survivor list (X re-read by the scatter)
  bool keep_ck = false;      // survivors keep their contract key (dense-row accumulation)
};

// How X is surveyed: a survivor list (GLOBAL), a survivor list plus per-group counts
// (GROUPED, few X entries have a Y run), or per-group counts alone (GROUPED, most do).
enum class Survey { kSurvivors, kSurvivorsGroups, kDenseGroups };

stc_status prepare(stc_ctx* ctx, Arena& ar, const stc_coo* X, const stc_coo* Y, const Plan& pl, Survey mode,
                   cudaStream_t s, StageTimer& tm, Prepared& pr) {
  const bool groups = mode != Survey::kSurvivors;
  const uint64_t bins = pl.K * pl.ky.nseg;
  if (pl.K > kMaxDirectBins || bins > kMaxDirectBins)
    return fail(STC_ERR_UNSUPPORTED, "contract key space %llu exceeds %llu bins", (unsigned long long)pl.K,
                (unsigned long long)kMaxDirectBins);
  const int64_t nX = X->nnz, nY = Y->nnz;
  STC_TRY(ar.alloc(&pr.ctr, 1));
  STC_CUDA(cudaMemsetAsync(pr.ctr, 0, sizeof(Counters), s));
  uint32_t* status = &pr.ctr->status;

  // Y: count per contract key, exclusive scan, scatter (Section 4.1.1 counting sort).
  uint32_t *ycnt = nullptr, *ycur = nullptr, *scr = nullptr;
  // The Y counts and, past them, the bitmap of contract keys with entries (one clearing).
  const uint64_t ne_words = (mode != Survey::kDenseGroups && pl.K <= kNonemptyMaxKeys) ? (pl.K + 31) / 32 : 0;
  STC_TRY(ar.alloc(&ycnt, bins + ne_words));
  STC_TRY(ar.alloc(&pr.yoff, bins + 1));
  STC_TRY(ar.alloc(&ycur, bins));
  STC_TRY(ar.alloc(&scr, (size_t)scan_scratch_elems((int64_t)bins)));
  pr.key32 = groups && pl.FY <= 0xffffffffull;
  if (pr.key32) {
    uint32_t* k32 = nullptr;
    STC_TRY(ar.alloc(&k32, (size_t)nY));
    pr.yfk = k32;
  } else {
    u64* k64 = nullptr;
    STC_TRY(ar.alloc(&k64, (size_t)nY));
    pr.yfk = k64;
  }
  STC_TRY(ar.alloc(&pr.yv, (size_t)nY));
  // X's arrays too, before any launch: the stages' events then enclose device work, not the
  // host's allocation calls.
  pr.sv.count = &pr.ctr->ns;
  if (groups) STC_TRY(ar.alloc(&pr.gcnt, pl.FX));
  pr.dense = mode == Survey::kDenseGroups;
  uint32_t* nonempty = nullptr;
  if (!pr.dense) {
    STC_TRY(ar.alloc(&pr.sv.fk, (size_t)nX));
    if (pr.keep_ck) STC_TRY(ar.alloc(&pr.sv.ck, (size_t)nX));
    STC_TRY(ar.alloc(&pr.sv.ystart, (size_t)nX));
    STC_TRY(ar.alloc(&pr.sv.w, (size_t)nX));
    STC_TRY(ar.alloc(&pr.sv.v, (size_t)nX));
    if (ne_words) nonempty = ycnt + bins;
  }
  STC_CUDA(cudaMemsetAsync(ycnt, 0, (bins + ne_words) * sizeof(uint32_t), s));
  STC_CUDA(launch_y_count(Y->coords, nY, pl.ky, ycnt, status, ctx->sms, s, nonempty));
  STC_CUDA(scan_u32(ycnt, pr.yoff, (int64_t)bins, scr, s));
  STC_CUDA(cudaMemcpyAsync(ycur, pr.yoff, bins * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  STC_CUDA(launch_y_scatter(Y->coords, Y->vals, nY, pl.ky, ycur, pr.yfk, pr.key32, pr.yv, ctx->sms, s));
  tm.mark(0);

  // X: find each entry's Y run and count the products exactly (Section 4.3).
  if (groups) STC_CUDA(cudaMemsetAsync(pr.gcnt, 0, pl.FX * sizeof(uint32_t), s));
  if (pr.dense) {
    STC_CUDA(launch_x_count(X->coords, nX, pl.kx, pr.yoff, &pr.ctr->P, pr.gcnt, status, ctx->sms, s));
  } else {
    STC_CUDA(launch_x_survey(X->coords, X->vals, nX, pl.kx, pr.yoff, pl.K, pr.sv, &pr.ctr->P, pr.gcnt, status,
                             nonempty, ctx->sms, s, nonempty != nullptr));
  }
  tm.mark(1);
  return STC_OK;
}

stc_status read_counters(const Prepared& pr, cudaStream_t s, Counters& h) {
  STC_CUDA(cudaMemcpyAsync(&h, pr.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s));
  STC_CUDA(cudaStreamSynchronize(s));
  return status_word(h.status);
}

// Peak device bytes of the GLOBAL strategy for these counts.
uint64_t global_bytes(const Plan& pl, int64_t nX, int64_t nY, uint64_t ns, uint64_t P, double alpha) {
  // Small output key spaces are sized from F itself (no host read of P), with a prefix over nX.
  const bool from_f = pl.F <= kGlobalFromF;
  const uint64_t target = from_f ? pl.F : std::min<uint64_t>(P, pl.F);
  if (from_f) ns = (uint64_t)nX;
  const uint64_t cap = pow2_at_least(std::max<uint64_t>(64, (uint64_t)((double)target / alpha) + 1));
  const uint64_t out_cap = std::min(target, cap);
  uint64_t b = sizeof(Counters) + pl.K * 4 * 3 + (uint64_t)scan_scratch_elems((int64_t)pl.K) * 4 + (pl.K + 31) / 32 * 4;
  b += (uint64_t)nY * 16 + (uint64_t)nX * 24;
  b += (ns + 1) * 8 + (uint64_t)scan_scratch_elems((int64_t)ns) * 8;
  b += cap * 16 + out_cap * (4ull * pl.ocols + 8);
  return b;
}


// Peak device bytes of the GROUPED strategy: Y grouped, X grouped (and, at worst, a survivor
// list), per-group arrays, and an output at its bound. Overflow-group tables are bounded by
// twice the output bound.
uint64_t grouped_bytes(const Plan& pl, int64_t nX, int64_t nY, uint64_t P) {
  const uint64_t out = std::min<uint64_t>(P, pl.F);
  uint64_t b = sizeof(Counters) + pl.K * 4 * 3 + (uint64_t)scan_scratch_elems((int64_t)pl.K) * 4 + (pl.K + 31) / 32 * 4;
  b += (uint64_t)nY * 16 + (uint64_t)nX * (24 + 16);
  b += pl.FX * (4 * 3) + std::min<uint64_t>(pl.FX, (uint64_t)nX) * 4 * (kMaxClasses + 5);
  b += out * (4ull * pl.ocols + 8);
  return b;
}

// Counters of the grouping and binning passes, read back with the first host sync.
struct GroupCounters {
  uint32_t count[kMaxClasses + 4];
  unsigned stream_nrec;  // streamed (group, segment) records
  u64 huge_slots;
  u64 out_cap;
  u64 stream_holes;      // positions of streamed reservations that hold no output
  u64 fill_counters[2];
};

// GROUPED strategy (Sections 4.1 and 4.3): survivors are counting-sorted by X free key,
// each group is binned by its table size, and the class kernels accumulate one group per
// CTA in shared memory and write its outputs directly.
stc_status contract_grouped(stc_ctx* ctx, Arena& ar, const stc_coo* X, const stc_coo* Y, const Plan& plan_in,
                            const stc_opts& o, cudaStream_t s, StageTimer& tm, stc_result* r) {
  const int64_t nX = X->nnz;
  Plan pl = plan_in;
  if (o.accumulator == STC_ACC_ROWS && pl.FY > kLaneRowMax)
    return fail(STC_ERR_INVALID_ARG, "the ROWS accumulator takes at most %llu Y free keys, not %llu",
                (unsigned long long)kLaneRowMax, (unsigned long long)pl.FY);
  // Bitmap rows: F_Y is swept in segments of `seg` free keys; Y is grouped per (contract key,
  // segment). Used when F_Y <= 2^20: for every group with the bitmap accumulator, for the
  // groups beyond the warp-sized hash classes with AUTO.
  bool dense_rows = false;
  uint32_t seg = 1, nseg = 1;
  if (pl.FY <= (1ull << 20) && (o.accumulator == STC_ACC_AUTO || o.accumulator == STC_ACC_DENSE)) {
    seg = (uint32_t)std::min<uint64_t>(kDenseSeg, pow2_at_least(std::max<uint64_t>(pl.FY, 64)));
    nseg = (uint32_t)((pl.FY + seg - 1) / seg);
    dense_rows = pl.K * nseg <= kMaxDirectBins;
  }
  if (dense_rows) {
    pl.ky.nseg = pl.kx.nseg = nseg;
    pl.ky.seg_shift = log2_u64(seg);
  }
  Prepared pr;
  pr.keep_ck = dense_rows;
  // Dense when Y's runs cover the contract keys on average: then nearly every X entry has a
  // run and a survivor list would only be written and read back.
  const Survey mode = ((uint64_t)Y->nnz >= pl.K) ? Survey::kDenseGroups : Survey::kSurvivorsGroups;
  STC_TRY(prepare(ctx, ar, X, Y, pl, mode, s, tm, pr));

  const bool wide = pl.FY > 0xffffffffull;
  const int ncls = wide ? kNumClasses64 : kNumClasses32;
  const ClassShape* shapes = wide ? kClassShapes64 : kClassShapes32;
  const double ga = (o.group_load_factor > 0.0) ? o.group_load_factor : 0.75;
  const uint64_t maxg = std::min<uint64_t>(pl.FX, (uint64_t)std::max<int64_t>(nX, 1));

  uint32_t *goff = nullptr, *gcur = nullptr, *scr = nullptr;
  GroupedX gx{};
  Bins b{};
  GroupCounters* gc = nullptr;
  STC_TRY(ar.alloc(&goff, pl.FX + 1));
  STC_TRY(ar.alloc(&gcur, pl.FX));
  STC_TRY(ar.alloc(&scr, (size_t)scan_scratch_elems((int64_t)pl.FX)));
  STC_TRY(ar.alloc(&gx.ystart, (size_t)nX));
  STC_TRY(ar.alloc(&gx.w, (size_t)nX));
  STC_TRY(ar.alloc(&gx.v, (size_t)nX));
  if (dense_rows) STC_TRY(ar.alloc(&gx.ck, (size_t)nX));
  STC_TRY(ar.alloc(&gc, 1));
  b.nclasses = ncls;
  for (int c = 0; c < ncls; c++) {
    b.tmax[c] = (u64)(ga * shapes[c].slots);
    STC_TRY(ar.alloc(&b.list[c], maxg));
  }
  if (dense_rows) {
    // With AUTO, groups that fit the warp classes keep their hash tables (a bitmap sweep costs
    // a fixed amount per segment).
    b.dense_min = o.accumulator == STC_ACC_DENSE ? 0 : (b.tmax[1] + 1) * nseg;
    b.stream_cap = dense_stream_cap();
    b.stash_cap = dense_stash_cap();
    for (int d = 0; d < 3; d++) STC_TRY(ar.alloc(&b.dense_list[d], maxg));
  }
  STC_TRY(ar.alloc(&b.huge_list, maxg));
  STC_TRY(ar.alloc(&b.huge_off, maxg));
  STC_TRY(ar.alloc(&b.huge_cap, maxg));
  b.count = gc->count;
  b.huge_slots = &gc->huge_slots;
  b.out_cap = &gc->out_cap;
  b.status = &pr.ctr->status;
  STC_CUDA(cudaMemsetAsync(gc, 0, sizeof(GroupCounters), s));
  STC_CUDA(scan_u32(pr.gcnt, goff, (int64_t)pl.FX, scr, s));
  STC_CUDA(cudaMemcpyAsync(gcur, goff, pl.FX * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  if (pr.dense) {
    STC_CUDA(launch_x_scatter_dense(X->coords, X->vals, nX, pl.kx, pr.yoff, gcur, gx, &pr.ctr->status, ctx->sms, s));
    STC_CUDA(cudaMemcpyAsync(&pr.ctr->ns, goff + pl.FX, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  } else {
    STC_CUDA(launch_x_group_scatter(pr.sv, gcur, gx, nX, ctx->sms, s));
  }
  STC_CUDA(launch_bin_groups(pl.FX, goff, gx.w, pl.FY, b, ctx->sms, s));
  tm.mark(2);

  Counters h{};
  GroupCounters hg{};
  STC_CUDA(cudaMemcpyAsync(&hg, gc, sizeof(GroupCounters), cudaMemcpyDeviceToHost, s));
  STC_TRY(read_counters(pr, s, h));
  tm.mark(3);
  r->stats.products = h.P;
  r->stats.survivors = h.ns;
  uint64_t groups = 0, dense_groups = 0;
  for (int c = 0; c < kMaxClasses + 4; c++) groups += hg.count[c];
  dense_groups = hg.count[kMaxClasses + 1] + hg.count[kMaxClasses + 2] + hg.count[kMaxClasses + 3];
  r->stats.groups = groups;
  r->stats.table_slots = hg.huge_slots;
  r->stats.accumulator = dense_groups == 0 ? STC_ACC_HASH : (dense_groups == groups ? STC_ACC_DENSE : STC_ACC_AUTO);
  if (h.P == 0) return STC_OK;
  // Lane-private dense rows: asked for, or (AUTO) output rows of at most 64 keys that receive
  // on average kRowsMinPerOutput products or more per output cell.
  const bool lane_rows = !wide && pl.FY <= kLaneRowMax &&
                         (o.accumulator == STC_ACC_ROWS ||
                          (o.accumulator == STC_ACC_AUTO && h.P >= kRowsMinPerOutput * pl.FX * pl.FY));
  if (lane_rows) r->stats.accumulator = STC_ACC_ROWS;

  const uint64_t out_cap = hg.out_cap;
  HugeGroups hh{};
  hh.count = lane_rows ? 0u : hg.count[kMaxClasses];
  hh.countp = gc->count + kMaxClasses;
  hh.list = b.huge_list;
  hh.off = b.huge_off;
  hh.cap = b.huge_cap;
  STC_TRY(ar.alloc(&r->coords, out_cap * (size_t)pl.ocols));
  STC_TRY(ar.alloc(&r->vals, out_cap));
  if (hh.count) {
    STC_TRY(ar.alloc(&hh.keys, hg.huge_slots));
    STC_TRY(ar.alloc(&hh.vals, hg.huge_slots));
    STC_CUDA(cudaMemsetAsync(hh.keys, 0xff, hg.huge_slots * sizeof(u64), s));
    STC_CUDA(cudaMemsetAsync(hh.vals, 0, hg.huge_slots * sizeof(double), s));
  }
  BatchOut hbo{};
  hbo.FY = pl.FY;
  hbo.out_cap = out_cap;
  hbo.coords = r->coords;
  hbo.vals = r->vals;
  hbo.op = pl.op;
  BatchOut* dbo = nullptr;
  STC_TRY(ar.alloc(&dbo, 1));
  STC_CUDA(cudaMemcpyAsync(dbo, &hbo, sizeof(BatchOut), cudaMemcpyHostToDevice, s));
  GroupArgs a{};
  a.goff = goff;
  a.gx = gx;
  a.yfk = pr.yfk;
  a.yv = pr.yv;
  a.FY = pl.FY;
  a.op = pl.op;
  a.coords = r->coords;
  a.vals = r->vals;
  a.out_cap = out_cap;
  a.nz = &pr.ctr->nz;
  a.status = &pr.ctr->status;
  a.bout = dbo;
  a.bnz = &pr.ctr->nz;
  if (lane_rows) {
    STC_CUDA(launch_group_lanerow(a, pl.FX, (uint32_t)pl.FY, ctx->sms, s));
  } else {
    const bool direct = !wide && out_cap < 0xffffffffull && o.accumulator != STC_ACC_HASH_SCAN;
    STC_CUDA(launch_group_classes(a, wide, direct, b, hg.count, ctx->sms, s));
    STC_CUDA(launch_group_huge(a, hh, wide, ctx->sms, s));
  }
  StreamArgs sa{};
  const uint32_t nstream = (dense_rows && !lane_rows) ? hg.count[kMaxClasses + 1] : 0u;
  if (dense_rows && !lane_rows) {
    // Streamed groups go last: every other kernel's outputs then lie below the final count.
    STC_CUDA(launch_group_dense(a, pr.yoff, nseg, seg, b.dense_list[2], hg.count[kMaxClasses + 3], b.dense_list[1],
                                hg.count[kMaxClasses + 2], ctx->sms, s));
    if (nstream) {
      STC_TRY(ar.alloc(&sa.rec, (size_t)nstream * nseg));
      sa.nrec = &gc->stream_nrec;
      sa.holes = &gc->stream_holes;
      const bool fixed_rows = !pl.op.pow2 && pl.op.ident && pl.op.order >= 2 && pl.op.order <= 8;
      STC_CUDA(launch_group_stream(a, pr.yoff, nseg, seg, b.dense_list[0], nstream, sa, fixed_rows, ctx->sms, s));
    }
  }
  tm.mark(4);
  u64 holes = 0;
  if (nstream) STC_CUDA(cudaMemcpyAsync(&holes, &gc->stream_holes, sizeof(u64), cudaMemcpyDeviceToHost, s));
  Counters h2{};
  STC_TRY(read_counters(pr, s, h2));
  r->nnz = (int64_t)(h2.nz - holes);
  if (holes) {
    if (holes >= (1ull << 32)) return fail(STC_ERR_UNSUPPORTED, "more than 2^32 repeated products in streamed groups");
    uint32_t* src_pos = nullptr;
    STC_TRY(ar.alloc(&src_pos, (size_t)holes));
    STC_CUDA(launch_stream_fill(sa.rec, sa.nrec, (u64)r->nnz, holes, src_pos, gc->fill_counters, r->coords,
                                r->vals, pl.ocols, &pr.ctr->status, ctx->sms, s));
    tm.mark(5);
  }
  r->stats.out_capacity = out_cap;
  r->mem = adopt(ar, ctx, s, {r->coords, r->vals});
  return STC_OK;
}

// AUTO: one global table when the output key space is small (the table stays in L2),
// per-group shared-memory tables when X's free keys can be counted directly.
// GROUPED pays per X free key (a counting sort over F_X bins) and per group (a table and an
// output reservation), so it needs groups with work in them: at most about two free keys per
// X entry, or up to sixteen when each X entry meets many Y entries (n_Y >= 16 K).
int pick_strategy(const Plan& pl, const stc_coo* X, const stc_coo* Y, int requested) {
  if (requested != STC_STRATEGY_AUTO) return requested;
  if (pl.F <= (1ull << 22)) return STC_STRATEGY_GLOBAL;
  if (pl.FX > kMaxDirectBins) return STC_STRATEGY_GLOBAL;
  const uint64_t nX = (uint64_t)X->nnz, nY = (uint64_t)Y->nnz;
  if (pl.FX <= 2 * nX + (1ull << 20)) return STC_STRATEGY_GROUPED;
  if (nY >= 16 * pl.K && pl.FX <= 16 * nX + (1ull << 20)) return STC_STRATEGY_GROUPED;
  return STC_STRATEGY_GLOBAL;
}

// FNV-1a over what fixes a contraction's shape: the operands' shapes and entry counts, the mode
// lists, the output order and form.
uint64_t shape_signature(const stc_coo* X, const stc_coo* Y, int32_t m, const int32_t* cx, const int32_t* cy,
                         const int32_t* out_order, int32_t oz, int32_t keys_out) {
  uint64_t h = 0xcbf29ce484222325ull;
  auto mix = [&](uint64_t v) {
    for (int i = 0; i < 8; i++) {
      h ^= (v >> (8 * i)) & 0xff;
      h *= 0x100000001b3ull;
    }
  };
  mix((uint64_t)X->order);
  for (int j = 0; j < X->order; j++) mix((uint64_t)X->shape[j]);
  mix((uint64_t)Y->order);
  for (int j = 0; j < Y->order; j++) mix((uint64_t)Y->shape[j]);
  mix((uint64_t)X->nnz);
  mix((uint64_t)Y->nnz);
  mix((uint64_t)m);
  for (int i = 0; i < m; i++) mix(((uint64_t)(uint32_t)cx[i] << 32) | (uint32_t)cy[i]);
  mix(out_order ? 1u : 0u);
  if (out_order)
    for (int q = 0; q < oz; q++) mix((uint64_t)(uint32_t)out_order[q]);
  mix((uint64_t)keys_out);
  return h;
}

bool rows_remembered(stc_ctx* ctx, uint64_t sig) {
  std::lock_guard<std::mutex> lk(ctx->rows_mu);
  return ctx->rows_shapes.count(sig) != 0;
}

void rows_note(stc_ctx* ctx, uint64_t sig, bool rows) {
  std::lock_guard<std::mutex> lk(ctx->rows_mu);
  if (!rows) {
    ctx->rows_shapes.erase(sig);
    return;
  }
  if (ctx->rows_shapes.size() >= 4096) ctx->rows_shapes.clear();  // a bound, not an eviction policy
  ctx->rows_shapes.insert(sig);
}

// Whether the contract keys are renumbered to dense ids before grouping (Section 4.1.2):
// always past the direct-counting limit, and under AUTO when the key space dwarfs the inputs
// (the K-bin histogram and scan would cost more than the renumbering).
bool use_dense_ids(const Plan& pl, const stc_coo* X, const stc_coo* Y, int mode) {
  if (pl.K > kMaxDirectBins) return true;
  if (pl.K <= 1 || mode == STC_IDS_DIRECT) return false;
  if (mode == STC_IDS_DENSE) return true;
  return pl.K > (1ull << 22) && pl.K > 8ull * (uint64_t)(X->nnz + Y->nnz);
}

// A contraction whose contract key space is too large to count directly, restated over
// dense ids (Section 4.1.2): the distinct contract keys of Y are numbered 0..D-1, and X and
// Y are rewritten with their free modes (ascending, lengths unchanged) followed by one
// paired mode of length D + 1 holding the id. X entries whose key Y lacks take the id D,
// which no Y entry has, so they form no products, as in Eq. 2. The free modes keep their
// order, so the output modes and out_order mean the same for the rewritten pair.
struct Relabelled {
  Arena ar;  // the rewritten coordinates
  StageTimer tm;
  std::vector<int64_t> xs, ys;
  stc_coo X{}, Y{};
  int32_t cx = 0, cy = 0;
  uint64_t ids = 0;  // D
  unsigned launches = 0;
  Relabelled(stc_ctx* c, cudaStream_t s) : ar(c, s) {}
};

stc_status relabel(stc_ctx* ctx, const stc_coo* X, const stc_coo* Y, const Plan& pl, bool record,
                   cudaStream_t s, Relabelled& rl) {
  rl.tm.start(record, s);
  const uint64_t slots = id_table_slots(Y->nnz);
  uint32_t fx = 0, fy = 0;
  int nfx = 0, nfy = 0;
  for (int j = 0; j < X->order; j++)
    if (pl.kx.cstride[j] == 0) fx |= 1u << j, rl.xs.push_back(X->shape[j]), nfx++;
  for (int j = 0; j < Y->order; j++)
    if (pl.ky.cstride[j] == 0) fy |= 1u << j, rl.ys.push_back(Y->shape[j]), nfy++;
  int32_t *xc = nullptr, *yc = nullptr;
  STC_TRY(rl.ar.alloc(&xc, (size_t)X->nnz * (nfx + 1)));
  STC_TRY(rl.ar.alloc(&yc, (size_t)Y->nnz * (nfy + 1)));
  uint32_t h[2] = {0, 0};
  {
    Arena tab(ctx, s);  // released (stream-ordered) once the rewrites are queued
    IdTable t{};
    uint32_t *scr = nullptr, *status = nullptr;
    t.slots = slots;
    STC_TRY(tab.alloc(&t.keys, slots));
    STC_TRY(tab.alloc(&t.flags, slots + 1));
    STC_TRY(tab.alloc(&t.prefix, slots + 2));
    STC_TRY(tab.alloc(&scr, (size_t)scan_scratch_elems((int64_t)slots + 1)));
    STC_TRY(tab.alloc(&status, 1));
    STC_CUDA(cudaMemsetAsync(t.keys, 0xff, slots * sizeof(u64), s));
    STC_CUDA(cudaMemsetAsync(t.flags + slots, 0, sizeof(uint32_t), s));
    STC_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t), s));
    STC_CUDA(launch_id_insert_rows(Y->coords, Y->nnz, pl.ky, t, status, ctx->sms, s));
    STC_CUDA(launch_id_number(t, scr, ctx->sms, s));
    STC_CUDA(launch_id_rewrite_rows(X->coords, X->nnz, pl.kx, fx, nfx, t, xc, status, ctx->sms, s));
    STC_CUDA(launch_id_rewrite_rows(Y->coords, Y->nnz, pl.ky, fy, nfy, t, yc, status, ctx->sms, s));
    STC_CUDA(cudaMemcpyAsync(&h[0], status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    STC_CUDA(cudaMemcpyAsync(&h[1], t.prefix + slots + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    STC_CUDA(cudaStreamSynchronize(s));
  }
  rl.tm.mark(0);
  STC_TRY(status_word(h[0]));
  rl.ids = h[1];
  if (rl.ids + 1 > kMaxDirectBins)
    return fail(STC_ERR_UNSUPPORTED, "Y has %llu distinct contract keys; at most 2^26 - 1 are supported",
                (unsigned long long)rl.ids);
  rl.xs.push_back((int64_t)rl.ids + 1);
  rl.ys.push_back((int64_t)rl.ids + 1);
  rl.X = stc_coo{nfx + 1, rl.xs.data(), X->nnz, xc, X->vals};
  rl.Y = stc_coo{nfy + 1, rl.ys.data(), Y->nnz, yc, Y->vals};
  rl.cx = nfx;
  rl.cy = nfy;
  rl.launches = take_launches();
  return STC_OK;
}

}  // namespace

DeviceBlock::~DeviceBlock() {
  DeviceGuard g(ctx->device);
  for (auto& p : parts) {
    cudaFreeAsync(p.first, stream);
    ctx->held -= p.second;
  }
}

namespace stc {
// Lets other translation units of the library set the calling thread's last error.
stc_status report_error(stc_status s, const char* msg) { return fail(s, "%s", msg); }
int ctx_device(const stc_ctx* ctx) { return ctx->device; }
// Results handed out by a server outlive its streams: their memory is returned on the legacy
// default stream instead (their data is complete when they are handed out).
void result_release_on_default_stream(stc_result* r) {
  if (!r) return;
  r->stream = nullptr;
  if (r->mem) r->mem->stream = nullptr;
}
}  // namespace stc

namespace {

// ---------------------------------------------------------------- batches
// The device state of one batch of problems: descriptors and every scratch array, all sized
// from totals the host knows before any kernel runs (entries of X and Y, contract-key bins,
// problems). Filled by batch_setup, consumed by the launch sequence that follows.
struct BatchDev {
  int32_t n = 0;
  std::vector<Plan> plans;
  std::vector<BatchOut> hbo;  // per problem: F_Y and the output plan (positions filled later)
  BatchArgs ba{};
  GroupedX gx{};
  Bins b{};
  GroupCounters* gc = nullptr;
  Counters* ctr = nullptr;
  u64* per = nullptr;          // [3n]: products, output bound, output count per problem
  uint32_t* gprob = nullptr;
  u64* gfk = nullptr;
  BatchOut* dbo = nullptr;     // [n]
  int32_t* doz = nullptr;      // [n] output order per problem
  u64* offs = nullptr;         // [2n + 2] value and coordinate offsets of a captured run
  BatchLayoutArgs* dargs = nullptr;
  bool wide = false;
  int depth = 0;  // expansion split of the CTA tables (TuneChoice::depth)
  int64_t total_x = 0, total_y = 0;
  int tune_bucket = 0;
};

// Plans, descriptors and scratch of a batch (no kernel runs; the descriptors are copied on s).
stc_status batch_setup(stc_ctx* ctx, int32_t n, const stc_problem* problems, Arena& ar, cudaStream_t s,
                       BatchDev& bd) {
  bd.n = n;
  bd.plans.assign(n, Plan{});
  std::vector<BatchProb> hb(n);
  std::vector<int64_t> xrow(n + 1, 0), yrow(n + 1, 0);
  std::vector<u64> fxoff(n + 1, 0);
  std::vector<int32_t> oz(n);
  unsigned __int128 bins = 0, fxsum = 0;
  bool key32 = true;
  for (int32_t i = 0; i < n; i++) {
    const stc_problem& q = problems[i];
    STC_TRY(make_plan(&q.X, &q.Y, q.ncontract, q.cx, q.cy, q.out_order, bd.plans[i]));
    const Plan& pl = bd.plans[i];
    if (pl.FY > 0xffffffffull) key32 = false;
    BatchProb& b = hb[i];
    b = BatchProb{};
    b.xc = q.X.coords;
    b.xv = q.X.vals;
    b.yc = q.Y.coords;
    b.yv = q.Y.vals;
    b.kx = pl.kx;
    b.ky = pl.ky;
    b.koff = (u64)bins;
    b.fxoff = (u64)fxsum;
    b.FY = pl.FY;
    oz[i] = pl.oz;
    bins += pl.K;
    fxsum += pl.FX;
    xrow[i + 1] = xrow[i] + q.X.nnz;
    yrow[i + 1] = yrow[i] + q.Y.nnz;
    fxoff[i + 1] = (u64)fxsum;
    if (bins > kMaxDirectBins) return fail(STC_ERR_UNSUPPORTED, "the batch's contract key spaces exceed 2^26 bins");
    if (fxsum >= ((unsigned __int128)1 << 63)) return fail(STC_ERR_KEY_OVERFLOW, "the batch's X free key spaces exceed 2^63");
    if (xrow[i + 1] > STC_MAX_NNZ || yrow[i + 1] > STC_MAX_NNZ)
      return fail(STC_ERR_INVALID_ARG, "the batch holds more than STC_MAX_NNZ entries of X or of Y");
  }
  bd.total_x = xrow[n];
  bd.total_y = yrow[n];
  bd.tune_bucket = log2_floor((uint64_t)(bd.total_x + bd.total_y)) * 32 + std::min(31, log2_floor((uint64_t)n));
  bd.hbo.assign(n, BatchOut{});
  for (int32_t i = 0; i < n; i++) {
    bd.hbo[i].FY = bd.plans[i].FY;
    bd.hbo[i].op = bd.plans[i].op;
  }

  BatchArgs& ba = bd.ba;
  ba = BatchArgs{};
  ba.n = n;
  ba.total_x = bd.total_x;
  ba.total_y = bd.total_y;
  ba.bins = (u64)bins;
  ba.key32 = key32;
  BatchProb* dpb = nullptr;
  int64_t *dxrow = nullptr, *dyrow = nullptr;
  u64* dfxoff = nullptr;
  STC_TRY(ar.alloc(&dpb, (size_t)n));
  STC_TRY(ar.alloc(&dxrow, (size_t)n + 1));
  STC_TRY(ar.alloc(&dyrow, (size_t)n + 1));
  STC_TRY(ar.alloc(&dfxoff, (size_t)n + 1));
  STC_TRY(ar.alloc(&bd.ctr, 1));
  STC_TRY(ar.alloc(&bd.per, 3 * (size_t)n));
  STC_TRY(ar.alloc(&bd.dbo, (size_t)n));
  STC_TRY(ar.alloc(&bd.doz, (size_t)n));
  STC_TRY(ar.alloc(&bd.offs, 2 * (size_t)n + 2));
  STC_TRY(ar.alloc(&bd.dargs, 1));
  STC_CUDA(cudaMemcpyAsync(dpb, hb.data(), n * sizeof(BatchProb), cudaMemcpyHostToDevice, s));
  STC_CUDA(cudaMemcpyAsync(dxrow, xrow.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  STC_CUDA(cudaMemcpyAsync(dyrow, yrow.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  STC_CUDA(cudaMemcpyAsync(dfxoff, fxoff.data(), (n + 1) * sizeof(u64), cudaMemcpyHostToDevice, s));
  STC_CUDA(cudaMemcpyAsync(bd.dbo, bd.hbo.data(), n * sizeof(BatchOut), cudaMemcpyHostToDevice, s));
  STC_CUDA(cudaMemcpyAsync(bd.doz, oz.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  ba.pb = dpb;
  ba.xrow = dxrow;
  ba.yrow = dyrow;
  ba.fxoff = dfxoff;
  ba.P = &bd.ctr->P;
  ba.Pp = bd.per;
  ba.pcap = bd.per + n;
  ba.status = &bd.ctr->status;

  const int64_t total_x = bd.total_x, total_y = bd.total_y;
  const u64 gcap = pow2_at_least(std::max<u64>(64, 2 * (u64)std::max<int64_t>(total_x, 1)));
  STC_TRY(ar.alloc(&ba.ycnt, ba.bins));
  STC_TRY(ar.alloc(&ba.yoff, ba.bins + 1));
  STC_TRY(ar.alloc(&ba.ycur, ba.bins));
  if (key32) {
    uint32_t* k = nullptr;
    STC_TRY(ar.alloc(&k, (size_t)total_y));
    ba.yfk = k;
    STC_TRY(ar.alloc(&ba.yuniq, (size_t)std::max<int64_t>(total_y, 1)));
  } else {
    u64* k = nullptr;
    STC_TRY(ar.alloc(&k, (size_t)total_y));
    ba.yfk = k;
  }
  STC_TRY(ar.alloc(&ba.yv, (size_t)total_y));
  STC_TRY(ar.alloc(&ba.sv.fk, (size_t)total_x));
  STC_TRY(ar.alloc(&ba.sv.ystart, (size_t)total_x));
  STC_TRY(ar.alloc(&ba.sv.w, (size_t)total_x));
  STC_TRY(ar.alloc(&ba.sv.v, (size_t)total_x));
  ba.sv.count = &bd.ctr->ns;
  STC_TRY(ar.alloc(&ba.idmap.keys, gcap));
  ba.idmap.mask = gcap - 1;
  STC_TRY(ar.alloc(&ba.gid, (size_t)total_x));
  STC_TRY(ar.alloc(&ba.gcnt, gcap));
  STC_TRY(ar.alloc(&ba.goff, gcap + 1));
  STC_TRY(ar.alloc(&ba.gcur, gcap));
  STC_TRY(ar.alloc(&ba.scan_scratch32, (size_t)std::max(scan_scratch_elems((int64_t)ba.bins),
                                                          scan_scratch_elems((int64_t)gcap))));

  // Grouped X, the class lists and counters.
  bd.wide = !key32;
  const int ncls = bd.wide ? kNumClasses64 : kNumClasses32;
  const size_t maxg = (size_t)std::max<int64_t>(total_x, 1);
  STC_TRY(ar.alloc(&bd.gx.ystart, maxg));
  STC_TRY(ar.alloc(&bd.gx.w, maxg));
  STC_TRY(ar.alloc(&bd.gx.v, maxg));
  STC_TRY(ar.alloc(&bd.gc, 1));
  STC_TRY(ar.alloc(&bd.gprob, gcap));
  STC_TRY(ar.alloc(&bd.gfk, gcap));
  Bins& b = bd.b;
  b = Bins{};
  b.nclasses = ncls;
  for (int c = 0; c < ncls; c++) STC_TRY(ar.alloc(&b.list[c], maxg));
  STC_TRY(ar.alloc(&b.huge_list, maxg));
  STC_TRY(ar.alloc(&b.huge_off, maxg));
  STC_TRY(ar.alloc(&b.huge_cap, maxg));
  b.count = bd.gc->count;
  b.huge_slots = &bd.gc->huge_slots;
  b.out_cap = &bd.gc->out_cap;
  b.status = &bd.ctr->status;
  return STC_OK;
}

// Class thresholds of a tuning choice: a group of bound t goes to the first class with
// t <= alpha * slots; with warp_max 256 the 1024-slot warp class takes no groups (its groups go
// to the CTA classes). depth selects the expansion split of the CTA tables.
void batch_set_choice(BatchDev& bd, const TuneChoice& ch) {
  const ClassShape* shapes = bd.wide ? kClassShapes64 : kClassShapes32;
  for (int c = 0; c < bd.b.nclasses; c++) bd.b.tmax[c] = (u64)(ch.alpha * shapes[c].slots);
  if (ch.warp_max < 1024) bd.b.tmax[1] = bd.b.tmax[0];
  bd.depth = ch.depth;
}

// The batch up to its per-group bins: counters cleared, Y grouped, X surveyed, grouped by
// (problem, X free key) and binned. Only enqueues work on s (no host reads).
stc_status batch_front(stc_ctx* ctx, BatchDev& bd, cudaStream_t s, StageTimer& tm) {
  BatchArgs& ba = bd.ba;
  const int32_t n = bd.n;
  STC_CUDA(cudaMemsetAsync(bd.ctr, 0, sizeof(Counters), s));
  STC_CUDA(cudaMemsetAsync(bd.per, 0, 3 * n * sizeof(u64), s));
  if (ba.bins) STC_CUDA(cudaMemsetAsync(ba.ycnt, 0, ba.bins * sizeof(uint32_t), s));
  STC_CUDA(cudaMemsetAsync(ba.idmap.keys, 0xff, (ba.idmap.mask + 1) * sizeof(u64), s));
  STC_CUDA(cudaMemsetAsync(ba.gcnt, 0, (ba.idmap.mask + 1) * sizeof(uint32_t), s));
  STC_CUDA(launch_batch_prepare(ba, ctx->sms, s));
  tm.mark(1);
  STC_CUDA(cudaMemsetAsync(bd.gc, 0, sizeof(GroupCounters), s));
  STC_CUDA(launch_batch_group(ba, bd.gx, bd.b, bd.gprob, bd.gfk, ctx->sms, s));
  tm.mark(2);
  return STC_OK;
}

// GroupArgs of the batch's accumulation kernels.
GroupArgs batch_group_args(const BatchDev& bd) {
  GroupArgs a{};
  a.goff = bd.ba.goff;
  a.gx = bd.gx;
  a.yfk = bd.ba.yfk;
  a.yv = bd.ba.yv;
  a.status = &bd.ctr->status;
  a.nz = &bd.ctr->nz;
  a.bout = bd.dbo;
  a.bnz = bd.per + 2 * bd.n;
  a.gprob = bd.gprob;
  a.gfk = bd.gfk;
  a.yuniq = bd.ba.yuniq;
  return a;
}

// One result per problem over a shared output block (offsets in elements).
void batch_results(stc_ctx* ctx, cudaStream_t s, const BatchDev& bd, const std::shared_ptr<DeviceBlock>& blk,
                   double* vals, int32_t* coords, const u64* voff, const u64* coff, const u64* hper,
                   const stc_stats& common, stc_result** outs) {
  const int32_t n = bd.n;
  for (int32_t i = 0; i < n; i++) {
    stc_result* r = new stc_result;
    r->ctx = ctx;
    r->stream = s;
    r->order = bd.plans[i].oz;
    r->shape = bd.plans[i].zshape;
    r->nnz = (int64_t)hper[2 * n + i];
    r->coords = coords ? coords + coff[i] : nullptr;
    r->vals = vals ? vals + voff[i] : nullptr;
    r->mem = blk;
    r->stats = common;
    r->stats.products = hper[i];
    r->stats.out_capacity = hper[n + i];
    ctx->live_results++;
    outs[i] = r;
  }
}

// Sizes one run of a batch needed, read back after it: what a captured run must provide.
struct BatchSizes {
  u64 vals = 0;     // output entries over all problems (sum of the exact bounds)
  u64 coords = 0;   // output coordinates over all problems
  u64 huge = 0;     // overflow-table slots
  u64 maxcap = 0;   // largest bound of one problem
};

// The rest of a batch with the host in the loop: the bins' counters are read back, one output
// block of the exact size is taken from `run`, the groups are accumulated, and the output
// counts are read back into hper[2n, 3n). bd.b.tmax must be set. tune_cand >= 0 times the
// accumulation for the autotuner.
stc_status batch_finish_eager(stc_ctx* ctx, BatchDev& bd, const stc_opts& o, Arena& run, cudaStream_t s,
                              StageTimer& tm, int tune_cand, bool* timed, std::vector<u64>& hper, BatchSizes& sz,
                              double** vals_out, int32_t** coords_out, std::vector<u64>& voff,
                              std::vector<u64>& coff) {
  const int32_t n = bd.n;
  Counters h{};
  GroupCounters hg{};
  hper.assign(3 * (size_t)n, 0);
  STC_CUDA(cudaMemcpyAsync(&hg, bd.gc, sizeof(GroupCounters), cudaMemcpyDeviceToHost, s));
  STC_CUDA(cudaMemcpyAsync(hper.data(), bd.per, 2 * n * sizeof(u64), cudaMemcpyDeviceToHost, s));
  STC_CUDA(cudaMemcpyAsync(&h, bd.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s));
  STC_CUDA(cudaStreamSynchronize(s));
  STC_TRY(status_word(h.status));
  tm.mark(3);

  // One output allocation: every problem's values, then every problem's coordinates.
  voff.assign(n + 1, 0);
  coff.assign(n + 1, 0);
  sz = BatchSizes{};
  for (int32_t i = 0; i < n; i++) {
    voff[i + 1] = voff[i] + hper[n + i];
    coff[i + 1] = coff[i] + hper[n + i] * (u64)bd.plans[i].oz;
    sz.maxcap = std::max<u64>(sz.maxcap, hper[n + i]);
  }
  sz.vals = voff[n];
  sz.coords = coff[n];
  sz.huge = hg.huge_slots;
  double* vals = nullptr;
  int32_t* coords = nullptr;
  STC_TRY(run.alloc(&vals, voff[n]));
  STC_TRY(run.alloc(&coords, coff[n]));
  std::vector<BatchOut> hbo = bd.hbo;
  for (int32_t i = 0; i < n; i++) {
    hbo[i].out_cap = hper[n + i];
    hbo[i].coords = coords ? coords + coff[i] : nullptr;
    hbo[i].vals = vals ? vals + voff[i] : nullptr;
  }
  STC_CUDA(cudaMemcpyAsync(bd.dbo, hbo.data(), n * sizeof(BatchOut), cudaMemcpyHostToDevice, s));
  HugeGroups hh{};
  hh.count = hg.count[kMaxClasses];
  hh.countp = bd.gc->count + kMaxClasses;
  hh.list = bd.b.huge_list;
  hh.off = bd.b.huge_off;
  hh.cap = bd.b.huge_cap;
  if (hh.count) {
    STC_TRY(run.alloc(&hh.keys, hg.huge_slots));
    STC_TRY(run.alloc(&hh.vals, hg.huge_slots));
    STC_CUDA(cudaMemsetAsync(hh.keys, 0xff, hg.huge_slots * sizeof(u64), s));
    STC_CUDA(cudaMemsetAsync(hh.vals, 0, hg.huge_slots * sizeof(double), s));
  }
  const GroupArgs a = batch_group_args(bd);
  if (h.P > 0) {
    const bool direct = !bd.wide && sz.maxcap < 0xffffffffull && o.accumulator != STC_ACC_HASH_SCAN;
    tune_mark(ctx, bd.tune_bucket, tune_cand, false, s);
    STC_CUDA(launch_group_classes(a, bd.wide, direct, bd.b, hg.count, ctx->sms, s, bd.depth));
    STC_CUDA(launch_group_huge(a, hh, bd.wide, ctx->sms, s));
    tune_mark(ctx, bd.tune_bucket, tune_cand, true, s);
    if (timed) *timed = true;
  }
  tm.mark(4);
  STC_CUDA(cudaMemcpyAsync(hper.data() + 2 * n, bd.per + 2 * n, n * sizeof(u64), cudaMemcpyDeviceToHost, s));
  Counters h2{};
  STC_CUDA(cudaMemcpyAsync(&h2, bd.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s));
  STC_CUDA(cudaStreamSynchronize(s));
  STC_TRY(status_word(h2.status));
  *vals_out = vals;
  *coords_out = coords;
  return STC_OK;
}

}  // namespace

// A prepared batch: the problems' descriptors and every scratch array held on the device
// across runs, and, once the load factor is settled, the whole launch sequence of a run
// captured in one CUDA graph that each later run replays.
struct stc_batch_plan {
  stc_ctx* ctx = nullptr;
  stc_opts opts{};
  int32_t n = 0;
  std::vector<stc_problem> probs;
  std::vector<std::vector<int64_t>> shapes;
  std::vector<std::vector<int32_t>> modes;
  cudaStream_t stream = nullptr;  // scratch allocation and graph capture
  std::unique_ptr<Arena> scratch;
  BatchDev bd;
  BatchSizes sizes{};
  TuneChoice choice{0.0, 1024, 0};  // the settled choice the graph was captured with (alpha 0: none)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  unsigned graph_launches = 0;
  u64* huge_keys = nullptr;
  double* huge_vals = nullptr;
  u64 huge_cap = 0;
  // pinned host mirrors written by the captured copies
  BatchLayoutArgs* h_args = nullptr;
  u64* h_per = nullptr;
  Counters* h_ctr = nullptr;
  u64* h_offs = nullptr;
  GroupCounters* h_gc = nullptr;
  int64_t runs = 0, graph_runs = 0;
};

namespace {

// Captures one run of the plan's batch on the plan's stream: the layout arguments copied in,
// the front of the batch, the device-side output layout, every class kernel with its count read
// on the device, and the copies of the counters the host reads after the run.
stc_status plan_capture(stc_batch_plan* pl) {
  BatchDev& bd = pl->bd;
  stc_ctx* ctx = pl->ctx;
  cudaStream_t ps = pl->stream;
  // The overflow groups' table is the plan's, sized by the last run.
  if (pl->sizes.huge > pl->huge_cap) {
    const u64 cap = std::max<u64>(pl->sizes.huge, 64);
    STC_TRY(pl->scratch->alloc(&pl->huge_keys, cap));
    STC_TRY(pl->scratch->alloc(&pl->huge_vals, cap));
    pl->huge_cap = cap;
    STC_CUDA(cudaStreamSynchronize(ps));
  }
  pl->h_args->huge_keys = pl->huge_keys;
  pl->h_args->huge_vals = pl->huge_vals;
  pl->h_args->huge_cap = pl->huge_cap;
  batch_set_choice(bd, pl->choice);
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  pl->exec = nullptr;
  pl->graph = nullptr;
  take_launches();
  STC_CUDA(cudaStreamBeginCapture(ps, cudaStreamCaptureModeThreadLocal));
  auto body = [&]() -> stc_status {
    StageTimer tm;
    const int32_t n = bd.n;
    STC_CUDA(cudaMemcpyAsync(bd.dargs, pl->h_args, sizeof(BatchLayoutArgs), cudaMemcpyHostToDevice, ps));
    STC_TRY(batch_front(ctx, bd, ps, tm));
    STC_CUDA(launch_batch_layout(n, bd.per + n, bd.doz, bd.dbo, bd.dargs, bd.offs, &bd.gc->huge_slots,
                                 bd.gc->count + kMaxClasses, &bd.ctr->status, ctx->sms, ps));
    const GroupArgs a = batch_group_args(bd);
    const bool direct =
        !bd.wide && pl->sizes.maxcap < 0x7fffffffull && pl->opts.accumulator != STC_ACC_HASH_SCAN;
    STC_CUDA(launch_group_classes(a, bd.wide, direct, bd.b, nullptr, ctx->sms, ps, bd.depth));
    HugeGroups hh{};
    hh.count = kCountOnDevice;
    hh.countp = bd.gc->count + kMaxClasses;
    hh.list = bd.b.huge_list;
    hh.off = bd.b.huge_off;
    hh.cap = bd.b.huge_cap;
    hh.keys = pl->huge_keys;
    hh.vals = pl->huge_vals;
    STC_CUDA(launch_group_huge(a, hh, bd.wide, ctx->sms, ps));
    STC_CUDA(cudaMemcpyAsync(pl->h_per, bd.per, 3 * n * sizeof(u64), cudaMemcpyDeviceToHost, ps));
    STC_CUDA(cudaMemcpyAsync(pl->h_ctr, bd.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, ps));
    STC_CUDA(cudaMemcpyAsync(pl->h_offs, bd.offs, (2 * n + 2) * sizeof(u64), cudaMemcpyDeviceToHost, ps));
    STC_CUDA(cudaMemcpyAsync(pl->h_gc, bd.gc, sizeof(GroupCounters), cudaMemcpyDeviceToHost, ps));
    return STC_OK;
  };
  const stc_status st = body();
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(ps, &g);  // ends the capture whatever happened
  if (st != STC_OK) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return st;
  }
  STC_CUDA(e);
  pl->graph = g;
  STC_CUDA(cudaGraphInstantiate(&pl->exec, g, 0));
  pl->graph_launches = take_launches();
  return STC_OK;
}

// One run with the host in the loop (the first runs, while the load factor is tuned, and any
// run whose sizes outgrew the captured layout). Captures the graph once the load factor is
// settled.
stc_status plan_run_eager(stc_batch_plan* pl, cudaStream_t s, stc_result** outs) {
  BatchDev& bd = pl->bd;
  stc_ctx* ctx = pl->ctx;
  int tune_cand = -1;
  const bool given = pl->opts.group_load_factor > 0.0;
  const TuneChoice ch =
      given ? TuneChoice{pl->opts.group_load_factor, 1024, 0} : tune_pick(ctx, bd.tune_bucket, &tune_cand);
  struct TuneGuard {
    stc_ctx* c;
    int b, k;
    bool armed = true;
    ~TuneGuard() {
      if (armed) tune_abort(c, b, k);
    }
  } tune_guard{ctx, bd.tune_bucket, tune_cand};
  batch_set_choice(bd, ch);
  Arena run(ctx, s);
  StageTimer tm;
  tm.start(pl->opts.record_times != 0, s);
  take_launches();
  STC_TRY(batch_front(ctx, bd, s, tm));
  std::vector<u64> hper, voff, coff;
  double* vals = nullptr;
  int32_t* coords = nullptr;
  bool timed = false;
  STC_TRY(batch_finish_eager(ctx, bd, pl->opts, run, s, tm, tune_cand, &timed, hper, pl->sizes, &vals, &coords, voff,
                             coff));
  if (timed) tune_guard.armed = false;
  stc_stats common{};
  tm.collect(common);
  common.launches = take_launches();
  common.strategy = STC_STRATEGY_GROUPED;
  common.accumulator = STC_ACC_HASH;
  auto blk = adopt(run, ctx, s, {vals, coords});
  batch_results(ctx, s, bd, blk, vals, coords, voff.data(), coff.data(), hper.data(), common, outs);
  // Capture once the choice is settled (given, or the tuner's pick for this bucket).
  TuneChoice settled{0.0, 1024, 0};
  if (given) {
    settled = ch;
  } else {
    int probe = -1;
    const TuneChoice pick = tune_pick(ctx, bd.tune_bucket, &probe);
    if (probe < 0) settled = pick;
    else tune_abort(ctx, bd.tune_bucket, probe);
  }
  const bool changed = settled.alpha != pl->choice.alpha || settled.warp_max != pl->choice.warp_max ||
                       settled.depth != pl->choice.depth;
  if (settled.alpha > 0.0 && (!pl->exec || changed || pl->sizes.huge > pl->huge_cap)) {
    pl->choice = settled;
    const stc_status st = plan_capture(pl);
    if (st != STC_OK) {
      // The results of this run stand; the plan keeps running with the host in the loop.
      cudaGetLastError();
      pl->exec = nullptr;
    }
  }
  return STC_OK;
}

}  // namespace

namespace {
stc_status contract_impl(stc_ctx* ctx, const stc_coo* X, const stc_coo* Y, int32_t m, const int32_t* cx,
                         const int32_t* cy, const int32_t* out_order, const stc_opts* opts, void* stream,
                         stc_result** out, const std::vector<int64_t>* xfree);
}  // namespace

extern "C" {

const char* stc_status_string(stc_status s) {
  switch (s) {
    case STC_OK: return "ok";
    case STC_ERR_INVALID_ARG: return "invalid argument";
    case STC_ERR_SHAPE_MISMATCH: return "paired modes have different lengths";
    case STC_ERR_KEY_OVERFLOW: return "key space exceeds 64 bits";
    case STC_ERR_OUT_OF_MEMORY: return "out of device memory or over budget";
    case STC_ERR_TABLE_FULL: return "accumulation table full";
    case STC_ERR_TIMEOUT: return "timeout";
    case STC_ERR_CUDA: return "CUDA error";
    case STC_ERR_COORD_OUT_OF_RANGE: return "coordinate out of range";
    case STC_ERR_UNSUPPORTED: return "unsupported";
    case STC_ERR_CANCELLED: return "cancelled";
  }
  return "unknown status";
}

const char* stc_last_error(void) { return g_last_error.c_str(); }

stc_status stc_create(stc_ctx** out, int device, size_t mem_budget_bytes) {
  if (!out) return fail(STC_ERR_INVALID_ARG, "ctx is NULL");
  *out = nullptr;
  int ndev = 0;
  STC_CUDA(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(STC_ERR_INVALID_ARG, "device %d of %d", device, ndev);
  DeviceGuard g(device);
  if (!g.ok) return fail(STC_ERR_CUDA, "cannot make device %d current", device);
  stc_ctx* c = new stc_ctx;
  c->device = device;
  c->budget = mem_budget_bytes;
  cudaError_t e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  if (e == cudaSuccess) e = cudaMemPoolCreate(&c->pool, &props);
  if (e == cudaSuccess) {
    uint64_t keep_all = UINT64_MAX;
    e = cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep_all);
  }
  if (e != cudaSuccess) {
    if (c->pool) cudaMemPoolDestroy(c->pool);
    delete c;
    return fail(STC_ERR_CUDA, "context set-up failed: %s", cudaGetErrorString(e));
  }
  *out = c;
  return STC_OK;
}

stc_status stc_destroy(stc_ctx* ctx) {
  if (!ctx) return fail(STC_ERR_INVALID_ARG, "ctx is NULL");
  if (ctx->live_results.load() != 0)
    return fail(STC_ERR_INVALID_ARG, "%lld results of this context are still alive",
                (long long)ctx->live_results.load());
  DeviceGuard g(ctx->device);
  cudaDeviceSynchronize();
  for (auto& kv : ctx->tune)
    for (int c = 0; c < kTuneCand; c++) {
      if (kv.second.ev0[c]) cudaEventDestroy(kv.second.ev0[c]);
      if (kv.second.ev1[c]) cudaEventDestroy(kv.second.ev1[c]);
    }
  cudaMemPoolDestroy(ctx->pool);
  delete ctx;
  return STC_OK;
}

stc_status stc_contract(stc_ctx* ctx, const stc_coo* X, const stc_coo* Y, int32_t m, const int32_t* cx,
                        const int32_t* cy, const int32_t* out_order, const stc_opts* opts, void* stream,
                        stc_result** out) {
  return contract_impl(ctx, X, Y, m, cx, cy, out_order, opts, stream, out, nullptr);
}

}  // extern "C"

namespace {
// stc_contract, and the contraction of the split form of a tensor in key form (xfree: the
// lengths of that tensor's free modes; the operands then keep their roles).
stc_status contract_impl(stc_ctx* ctx, const stc_coo* X, const stc_coo* Y, int32_t m, const int32_t* cx,
                         const int32_t* cy, const int32_t* out_order, const stc_opts* opts, void* stream,
                         stc_result** out, const std::vector<int64_t>* xfree) {
  if (!ctx || !out) return fail(STC_ERR_INVALID_ARG, "ctx or out is NULL");
  *out = nullptr;
  const stc_opts o = opts ? *opts : stc_opts{};
  Plan pl;
  STC_TRY(make_plan(X, Y, m, cx, cy, out_order, pl, o.output_keys != 0, xfree));
  const double alpha = (o.load_factor > 0.0) ? o.load_factor : 0.5;
  if (!(alpha > 0.0 && alpha <= 0.9)) return fail(STC_ERR_INVALID_ARG, "load_factor %g outside (0, 0.9]", alpha);
  if (o.strategy < 0 || o.strategy > STC_STRATEGY_GROUPED)
    return fail(STC_ERR_INVALID_ARG, "unknown strategy %d", o.strategy);
  if (o.accumulator < 0 || o.accumulator > STC_ACC_ROWS)
    return fail(STC_ERR_INVALID_ARG, "unknown accumulator %d", o.accumulator);
  if (o.group_load_factor < 0.0 || o.group_load_factor > 0.9)
    return fail(STC_ERR_INVALID_ARG, "group_load_factor %g outside (0, 0.9]", o.group_load_factor);
  if (o.contract_ids < 0 || o.contract_ids > STC_IDS_DENSE)
    return fail(STC_ERR_INVALID_ARG, "unknown contract_ids %d", o.contract_ids);
  if (o.operands < 0 || o.operands > STC_OPERANDS_SWAPPED)
    return fail(STC_ERR_INVALID_ARG, "unknown operands %d", o.operands);
  if (o.table_shrink < 0 || o.table_shrink > 30)
    return fail(STC_ERR_INVALID_ARG, "table_shrink %d outside 0..30", o.table_shrink);
  if (o.probe != 0 && o.probe != 1 && o.probe != 4 && o.probe != 8)
    return fail(STC_ERR_INVALID_ARG, "probe %d is none of 0, 1, 4, 8", o.probe);
  const int probe = o.probe ? o.probe : kDefaultProbe;
  // A swap permutes the output modes back, so outputs in key form keep the operands as given.
  if (!xfree && (o.operands == STC_OPERANDS_SWAPPED ||
                 (o.operands == STC_OPERANDS_AUTO && !o.output_keys && (uint64_t)Y->nnz > 4 * (uint64_t)X->nnz))) {
    // Y (x) X has output modes (Y free, X free); map each requested mode onto that order.
    const int nfx = X->order - m, nfy = Y->order - m;
    std::vector<int32_t> oo(nfx + nfy);
    for (int q = 0; q < nfx + nfy; q++) {
      const int t = out_order ? out_order[q] : q;
      oo[q] = t < nfx ? nfy + t : t - nfx;
    }
    stc_opts inner = o;
    inner.operands = STC_OPERANDS_AS_GIVEN;
    STC_TRY(stc_contract(ctx, Y, X, m, cy, cx, oo.data(), &inner, stream, out));
    (*out)->stats.swapped = 1;
    return STC_OK;
  }
  if (!xfree && use_dense_ids(pl, X, Y, o.contract_ids)) {
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(STC_ERR_CUDA, "cannot make device %d current", ctx->device);
    Relabelled rl(ctx, static_cast<cudaStream_t>(stream));
    take_launches();
    STC_TRY(relabel(ctx, X, Y, pl, o.record_times != 0, static_cast<cudaStream_t>(stream), rl));
    stc_opts inner = o;
    inner.contract_ids = STC_IDS_DIRECT;
    STC_TRY(stc_contract(ctx, &rl.X, &rl.Y, 1, &rl.cx, &rl.cy, out_order, &inner, stream, out));
    (*out)->stats.launches += rl.launches;
    (*out)->stats.contract_ids = rl.ids;
    rl.tm.collect((*out)->stats);
    return STC_OK;
  }
  int strategy = pick_strategy(pl, X, Y, o.strategy);
  // AUTO: a shape whose last run here was rows-heavy is grouped again (lane-private rows).
  const uint64_t sig = shape_signature(X, Y, m, cx, cy, out_order, pl.oz, o.output_keys);
  const bool rows_shape = o.strategy == STC_STRATEGY_AUTO && pl.FY <= kLaneRowMax && pl.FX <= kMaxDirectBins &&
                          (o.accumulator == STC_ACC_AUTO || o.accumulator == STC_ACC_ROWS);
  const bool by_memory = rows_shape && strategy == STC_STRATEGY_GLOBAL && rows_remembered(ctx, sig);
  if (by_memory) strategy = STC_STRATEGY_GROUPED;
  if (strategy == STC_STRATEGY_GROUPED && pl.FX > kMaxDirectBins)
    return fail(STC_ERR_UNSUPPORTED, "X free key space %llu exceeds %llu bins", (unsigned long long)pl.FX,
                (unsigned long long)kMaxDirectBins);

  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(STC_ERR_CUDA, "cannot make device %d current", ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Arena ar(ctx, s);
  StageTimer tm;
  tm.start(o.record_times != 0, s);
  take_launches();

  if (strategy == STC_STRATEGY_GROUPED) {
    stc_result* r = new stc_result;
    r->ctx = ctx;
    r->stream = s;
    r->order = pl.oz;
    r->keys_form = pl.keys_out;
    r->shape = pl.zshape;
    r->stats.strategy = STC_STRATEGY_GROUPED;
    const stc_status st = contract_grouped(ctx, ar, X, Y, pl, o, s, tm, r);
    if (st != STC_OK) {
      delete r;
      return st;
    }
    if (by_memory && r->stats.accumulator != STC_ACC_ROWS) rows_note(ctx, sig, false);
    tm.collect(r->stats);
    r->stats.launches = take_launches();
    ctx->live_results++;
    *out = r;
    return STC_OK;
  }

  Prepared pr;
  STC_TRY(prepare(ctx, ar, X, Y, pl, Survey::kSurvivors, s, tm, pr));
  if (pl.F <= kGlobalFromF && o.table_shrink == 0 && X->nnz > 0 && Y->nnz > 0) {
    // A small output key space: the table and the output are sized from F itself, and P and
    // the survivor count are read on the device, so the call waits once, at its end.
    const uint64_t cap = pow2_at_least(std::max<uint64_t>(64, (uint64_t)((double)pl.F / alpha) + 1));
    const uint64_t out_cap = std::min<uint64_t>(pl.F, cap);
    const int64_t nX = X->nnz;
    stc_result* r = new stc_result;
    r->ctx = ctx;
    r->stream = s;
    r->order = pl.oz;
    r->keys_form = pl.keys_out;
    r->shape = pl.zshape;
    r->stats.strategy = STC_STRATEGY_GLOBAL;
    auto run = [&]() -> stc_status {
      GlobalTable t{};
      u64 *wpre = nullptr, *wscr = nullptr;
      STC_TRY(ar.alloc(&t.keys, cap));
      STC_TRY(ar.alloc(&t.vals, cap));
      STC_TRY(ar.alloc(&wpre, (size_t)nX + 1));
      STC_TRY(ar.alloc(&wscr, (size_t)scan_scratch_elems(nX)));
      STC_TRY(ar.alloc(&r->coords, out_cap * (size_t)pl.ocols));
      STC_TRY(ar.alloc(&r->vals, out_cap));
      t.mask = cap - 1;
      STC_CUDA(cudaMemsetAsync(t.keys, 0xff, cap * sizeof(u64), s));
      STC_CUDA(cudaMemsetAsync(t.vals, 0, cap * sizeof(double), s));
      STC_CUDA(scan_u32_u64_dev(pr.sv.w, wpre, nX, &pr.ctr->ns, wscr, s));
      tm.mark(3);
      STC_CUDA(launch_expand_global_dev(wpre, &pr.ctr->ns, &pr.ctr->P, pr.sv, static_cast<const u64*>(pr.yfk), pr.yv,
                                        pl.FY, t, &pr.ctr->status, ctx->sms, s, probe));
      tm.mark(4);
      STC_CUDA(launch_compact_global(t, pl.op, r->coords, r->vals, out_cap, &pr.ctr->nz, &pr.ctr->status, ctx->sms,
                                     s));
      tm.mark(5);
      Counters h{};
      STC_TRY(read_counters(pr, s, h));
      r->nnz = (int64_t)h.nz;
      r->stats.products = h.P;
      r->stats.survivors = h.ns;
      r->stats.table_slots = cap;
      r->stats.out_capacity = out_cap;
      return STC_OK;
    };
    const stc_status st = run();
    if (st != STC_OK) {
      delete r;
      return st;
    }
    if (rows_shape && r->stats.products >= kRowsMinPerOutput * pl.F) rows_note(ctx, sig, true);
    r->mem = adopt(ar, ctx, s, {r->coords, r->vals});
    tm.collect(r->stats);
    r->stats.launches = take_launches();
    ctx->live_results++;
    *out = r;
    return STC_OK;
  }
  Counters h{};
  STC_TRY(read_counters(pr, s, h));
  tm.mark(3);
  if (rows_shape && h.P >= kRowsMinPerOutput * pl.F) rows_note(ctx, sig, true);

  stc_result* r = new stc_result;
  r->ctx = ctx;
  r->stream = s;
  r->order = pl.oz;
  r->keys_form = pl.keys_out;
  r->shape = pl.zshape;
  r->stats.products = h.P;
  r->stats.survivors = h.ns;
  r->stats.strategy = STC_STRATEGY_GLOBAL;

  if (h.P > 0) {
    const uint64_t target = std::min<uint64_t>(h.P, pl.F);
    const uint64_t cap = pow2_at_least(std::max<uint64_t>(64, (uint64_t)((double)target / alpha) + 1));
    const uint64_t out_cap = std::min(target, cap);
    // Fault injection (stc_opts.table_shrink): the first attempt uses a smaller table.
    const uint64_t first_cap = std::max<uint64_t>(64, o.table_shrink > 0 ? cap >> o.table_shrink : cap);
    GlobalTable t{};
    u64* wpre = nullptr;
    u64* wscr = nullptr;
    stc_status st = STC_OK;
    auto run = [&]() -> stc_status {
      STC_TRY(ar.alloc(&t.keys, cap));
      STC_TRY(ar.alloc(&t.vals, cap));
      STC_TRY(ar.alloc(&wpre, (size_t)h.ns + 1));
      STC_TRY(ar.alloc(&wscr, (size_t)scan_scratch_elems((int64_t)h.ns)));
      STC_TRY(ar.alloc(&r->coords, out_cap * (size_t)pl.ocols));
      STC_TRY(ar.alloc(&r->vals, out_cap));
      STC_CUDA(scan_u32_u64(pr.sv.w, wpre, (int64_t)h.ns, wscr, s));
      tm.mark(3);
      for (uint64_t c = first_cap;; c = cap) {
        t.mask = c - 1;
        STC_CUDA(cudaMemsetAsync(t.keys, 0xff, c * sizeof(u64), s));
        STC_CUDA(cudaMemsetAsync(t.vals, 0, c * sizeof(double), s));
        STC_CUDA(launch_expand_global(wpre, (int64_t)h.ns, h.P, pr.sv, static_cast<const u64*>(pr.yfk), pr.yv,
                                      pl.FY, t, &pr.ctr->status, ctx->sms, s, probe));
        tm.mark(4);
        STC_CUDA(launch_compact_global(t, pl.op, r->coords, r->vals, out_cap, &pr.ctr->nz, &pr.ctr->status,
                                       ctx->sms, s));
        tm.mark(5);
        Counters h2{};
        STC_CUDA(cudaMemcpyAsync(&h2, pr.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s));
        STC_CUDA(cudaStreamSynchronize(s));
        // A table that overflowed lost products: run the expansion again at full capacity
        // (the compaction wrote at most out_cap entries, all of them overwritten now).
        if (h2.status == kStatTableFull && c < cap) {
          STC_CUDA(cudaMemsetAsync(&pr.ctr->nz, 0, sizeof(u64), s));
          STC_CUDA(cudaMemsetAsync(&pr.ctr->status, 0, sizeof(uint32_t), s));
          r->stats.retries++;
          continue;
        }
        STC_TRY(status_word(h2.status));
        r->nnz = (int64_t)h2.nz;
        return STC_OK;
      }
    };
    st = run();
    if (st != STC_OK) {
      delete r;  // its blocks are still owned by the arena and are released with it
      return st;
    }
    r->mem = adopt(ar, ctx, s, {r->coords, r->vals});
    r->stats.out_capacity = out_cap;
    r->stats.table_slots = cap;
  }
  tm.collect(r->stats);
  r->stats.launches = take_launches();
  ctx->live_results++;
  *out = r;
  return STC_OK;
}


}  // namespace

extern "C" {

stc_status stc_contract_batch(stc_ctx* ctx, int32_t n, const stc_problem* problems, const stc_opts* opts,
                              void* stream, stc_result** outs) {
  if (!ctx || n < 0 || (n > 0 && (!problems || !outs))) return fail(STC_ERR_INVALID_ARG, "bad batch arguments");
  for (int32_t i = 0; i < n; i++) outs[i] = nullptr;
  if (n == 0) return STC_OK;
  const stc_opts o = opts ? *opts : stc_opts{};
  if (o.group_load_factor < 0.0 || o.group_load_factor > 0.9)
    return fail(STC_ERR_INVALID_ARG, "group_load_factor %g outside (0, 0.9]", o.group_load_factor);
  if (o.output_keys) return fail(STC_ERR_UNSUPPORTED, "batches return coordinates (output_keys is for stc_contract)");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(STC_ERR_CUDA, "cannot make device %d current", ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Arena ar(ctx, s);
  BatchDev bd;
  STC_TRY(batch_setup(ctx, n, problems, ar, s, bd));
  // Load factor: given, or picked by the autotuner for this size bucket (entries, problems).
  int tune_cand = -1;
  const TuneChoice ch =
      o.group_load_factor > 0.0 ? TuneChoice{o.group_load_factor, 1024, 0} : tune_pick(ctx, bd.tune_bucket, &tune_cand);
  struct TuneGuard {  // gives a picked candidate back if the batch fails before it is timed
    stc_ctx* c;
    int b, k;
    bool armed = true;
    ~TuneGuard() {
      if (armed) tune_abort(c, b, k);
    }
  } tune_guard{ctx, bd.tune_bucket, tune_cand};
  batch_set_choice(bd, ch);
  StageTimer tm;
  tm.start(o.record_times != 0, s);
  take_launches();
  STC_TRY(batch_front(ctx, bd, s, tm));
  std::vector<u64> hper, voff, coff;
  BatchSizes sz;
  double* vals = nullptr;
  int32_t* coords = nullptr;
  bool timed = false;
  STC_TRY(batch_finish_eager(ctx, bd, o, ar, s, tm, tune_cand, &timed, hper, sz, &vals, &coords, voff, coff));
  if (timed) tune_guard.armed = false;
  auto blk = adopt(ar, ctx, s, {vals, coords});
  stc_stats common{};
  tm.collect(common);
  common.launches = take_launches();
  common.strategy = STC_STRATEGY_GROUPED;
  common.accumulator = STC_ACC_HASH;
  batch_results(ctx, s, bd, blk, vals, coords, voff.data(), coff.data(), hper.data(), common, outs);
  return STC_OK;
}

stc_status stc_batch_plan_create(stc_ctx* ctx, int32_t n, const stc_problem* problems, const stc_opts* opts,
                                 stc_batch_plan** out) {
  if (!ctx || !out || n <= 0 || !problems) return fail(STC_ERR_INVALID_ARG, "bad batch plan arguments");
  *out = nullptr;
  const stc_opts o = opts ? *opts : stc_opts{};
  if (o.group_load_factor < 0.0 || o.group_load_factor > 0.9)
    return fail(STC_ERR_INVALID_ARG, "group_load_factor %g outside (0, 0.9]", o.group_load_factor);
  if (o.output_keys) return fail(STC_ERR_UNSUPPORTED, "batches return coordinates (output_keys is for stc_contract)");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(STC_ERR_CUDA, "cannot make device %d current", ctx->device);
  std::unique_ptr<stc_batch_plan> pl(new stc_batch_plan);
  pl->ctx = ctx;
  pl->opts = o;
  pl->n = n;
  // The problems' host arrays are copied; their device arrays are the caller's.
  pl->probs.assign(problems, problems + n);
  pl->shapes.resize(2 * (size_t)n);
  pl->modes.resize(3 * (size_t)n);
  for (int32_t i = 0; i < n; i++) {
    stc_problem& q = pl->probs[i];
    STC_TRY(check_coo(&q.X, "X"));
    STC_TRY(check_coo(&q.Y, "Y"));
    if (q.ncontract < 0 || q.ncontract > q.X.order || q.ncontract > q.Y.order || (q.ncontract && (!q.cx || !q.cy)))
      return fail(STC_ERR_INVALID_ARG, "problem %d: bad contract mode lists", i);
    pl->shapes[2 * i].assign(q.X.shape, q.X.shape + q.X.order);
    pl->shapes[2 * i + 1].assign(q.Y.shape, q.Y.shape + q.Y.order);
    pl->modes[3 * i].assign(q.cx, q.cx + q.ncontract);
    pl->modes[3 * i + 1].assign(q.cy, q.cy + q.ncontract);
    const int oz = (q.X.order - q.ncontract) + (q.Y.order - q.ncontract);
    if (q.out_order) pl->modes[3 * i + 2].assign(q.out_order, q.out_order + oz);
    q.X.shape = pl->shapes[2 * i].data();
    q.Y.shape = pl->shapes[2 * i + 1].data();
    q.cx = pl->modes[3 * i].data();
    q.cy = pl->modes[3 * i + 1].data();
    q.out_order = q.out_order ? pl->modes[3 * i + 2].data() : nullptr;
  }
  STC_CUDA(cudaStreamCreateWithFlags(&pl->stream, cudaStreamNonBlocking));
  pl->scratch.reset(new Arena(ctx, pl->stream));
  stc_status st = batch_setup(ctx, n, pl->probs.data(), *pl->scratch, pl->stream, pl->bd);
  cudaError_t e = cudaSuccess;
  if (st == STC_OK) {
    e = cudaMallocHost(&pl->h_args, sizeof(BatchLayoutArgs));
    if (e == cudaSuccess) e = cudaMallocHost(&pl->h_per, 3 * (size_t)n * sizeof(u64));
    if (e == cudaSuccess) e = cudaMallocHost(&pl->h_ctr, sizeof(Counters));
    if (e == cudaSuccess) e = cudaMallocHost(&pl->h_offs, (2 * (size_t)n + 2) * sizeof(u64));
    if (e == cudaSuccess) e = cudaMallocHost(&pl->h_gc, sizeof(GroupCounters));
    if (e == cudaSuccess) e = cudaStreamSynchronize(pl->stream);
    if (e != cudaSuccess) st = fail(STC_ERR_CUDA, "batch plan set-up failed: %s", cudaGetErrorString(e));
  }
  if (st != STC_OK) {
    stc_batch_plan_destroy(pl.release());
    return st;
  }
  *out = pl.release();
  return STC_OK;
}

stc_status stc_batch_plan_run(stc_batch_plan* pl, void* stream, stc_result** outs) {
  if (!pl || !outs) return fail(STC_ERR_INVALID_ARG, "plan or outs is NULL");
  for (int32_t i = 0; i < pl->n; i++) outs[i] = nullptr;
  stc_ctx* ctx = pl->ctx;
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(STC_ERR_CUDA, "cannot make device %d current", ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  pl->runs++;
  if (!pl->exec) return plan_run_eager(pl, s, outs);
  // Replay: one output block of the last run's exact size, the layout arguments written for
  // the graph's first copy, the graph, one wait.
  const int32_t n = pl->n;
  BatchDev& bd = pl->bd;
  const u64 vbytes = (pl->sizes.vals * 8 + 15) & ~15ull;
  const u64 bytes = vbytes + pl->sizes.coords * 4;
  Arena run(ctx, s);
  unsigned char* block = nullptr;
  STC_TRY(run.alloc(&block, (size_t)std::max<u64>(bytes, 16)));
  pl->h_args->out = block;
  pl->h_args->out_bytes = bytes;
  STC_CUDA(cudaGraphLaunch(pl->exec, s));
  STC_CUDA(cudaStreamSynchronize(s));
  const uint32_t status = pl->h_ctr->status;
  if (status & kStatOutOverflow) {
    // This run's bounds outgrew the captured layout (the inputs' contents changed): run it
    // again with the host in the loop, which also captures a layout of the new sizes.
    return plan_run_eager(pl, s, outs);
  }
  STC_TRY(status_word(status));
  pl->graph_runs++;
  const u64* offs = pl->h_offs;
  std::vector<u64> voff(offs, offs + n + 1), coff(offs + n + 1, offs + 2 * n + 2);
  double* vals = reinterpret_cast<double*>(block);
  int32_t* coords = reinterpret_cast<int32_t*>(block + vbytes);
  stc_stats common{};
  common.launches = pl->graph_launches;
  common.strategy = STC_STRATEGY_GROUPED;
  common.accumulator = STC_ACC_HASH;
  auto blk = adopt(run, ctx, s, {block});
  batch_results(ctx, s, bd, blk, vals, coords, voff.data(), coff.data(), pl->h_per, common, outs);
  return STC_OK;
}

stc_status stc_batch_plan_stats(const stc_batch_plan* pl, int64_t* runs, int64_t* graph_runs,
                                double* group_load_factor, int32_t* warp_table_max, int32_t* expansion_depth) {
  if (!pl) return fail(STC_ERR_INVALID_ARG, "plan is NULL");
  if (runs) *runs = pl->runs;
  if (graph_runs) *graph_runs = pl->graph_runs;
  if (group_load_factor) *group_load_factor = pl->exec ? pl->choice.alpha : 0.0;
  if (warp_table_max) *warp_table_max = pl->exec ? pl->choice.warp_max : 0;
  if (expansion_depth) *expansion_depth = pl->exec ? pl->choice.depth : 0;
  return STC_OK;
}

stc_status stc_batch_plan_destroy(stc_batch_plan* pl) {
  if (!pl) return STC_OK;
  DeviceGuard g(pl->ctx->device);
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  if (pl->stream) cudaStreamSynchronize(pl->stream);
  pl->scratch.reset();  // scratch goes back to the pool in the plan stream's order
  if (pl->stream) {
    cudaStreamSynchronize(pl->stream);
    cudaStreamDestroy(pl->stream);
  }
  if (pl->h_args) cudaFreeHost(pl->h_args);
  if (pl->h_per) cudaFreeHost(pl->h_per);
  if (pl->h_ctr) cudaFreeHost(pl->h_ctr);
  if (pl->h_offs) cudaFreeHost(pl->h_offs);
  if (pl->h_gc) cudaFreeHost(pl->h_gc);
  delete pl;
  return STC_OK;
}

stc_status stc_ctx_stats(const stc_ctx* ctx, uint64_t* held_bytes, int64_t* live_results) {
  if (!ctx) return fail(STC_ERR_INVALID_ARG, "ctx is NULL");
  if (held_bytes) *held_bytes = ctx->held.load();
  if (live_results) *live_results = ctx->live_results.load();
  return STC_OK;
}

stc_status stc_count(stc_ctx* ctx, const stc_coo* X, const stc_coo* Y, int32_t m, const int32_t* cx,
                     const int32_t* cy, void* stream, uint64_t* products, uint64_t* bytes_bound) {
  if (!ctx) return fail(STC_ERR_INVALID_ARG, "ctx is NULL");
  Plan pl;
  STC_TRY(make_plan(X, Y, m, cx, cy, nullptr, pl));
  // Bound the orientation stc_contract's AUTO operand order will run (P is the same).
  if ((uint64_t)Y->nnz > 4 * (uint64_t)X->nnz)
    return stc_count(ctx, Y, X, m, cy, cx, stream, products, bytes_bound);
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(STC_ERR_CUDA, "cannot make device %d current", ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (use_dense_ids(pl, X, Y, STC_IDS_AUTO)) {
    Relabelled rl(ctx, s);
    STC_TRY(relabel(ctx, X, Y, pl, false, s, rl));
    uint64_t b = 0;
    STC_TRY(stc_count(ctx, &rl.X, &rl.Y, 1, &rl.cx, &rl.cy, stream, products, bytes_bound ? &b : nullptr));
    // The rewritten coordinates stay held beside the id table, then beside the contraction.
    const uint64_t slots = id_table_slots(Y->nnz);
    const uint64_t table = 16 * slots + 4 * (uint64_t)scan_scratch_elems((int64_t)slots + 1) + 16;
    if (bytes_bound)
      *bytes_bound = std::max(b, table) + 4ull * (uint64_t)(rl.X.order * X->nnz + rl.Y.order * Y->nnz);
    return STC_OK;
  }
  Arena ar(ctx, s);
  StageTimer tm;
  Prepared pr;
  const int strategy = pick_strategy(pl, X, Y, STC_STRATEGY_AUTO);
  const bool dense = strategy == STC_STRATEGY_GROUPED && (uint64_t)Y->nnz >= pl.K;
  STC_TRY(prepare(ctx, ar, X, Y, pl, dense ? Survey::kDenseGroups : Survey::kSurvivors, s, tm, pr));
  Counters h{};
  STC_TRY(read_counters(pr, s, h));
  if (products) *products = h.P;
  if (bytes_bound)
    *bytes_bound = strategy == STC_STRATEGY_GROUPED ? grouped_bytes(pl, X->nnz, Y->nnz, h.P)
                                                    : global_bytes(pl, X->nnz, Y->nnz, h.ns, h.P, 0.5);
  return STC_OK;
}

stc_status stc_linearize(stc_ctx* ctx, const stc_coo* T, int32_t nmodes, const int32_t* modes, uint64_t* keys_out,
                         void* stream) {
  if (!ctx) return fail(STC_ERR_INVALID_ARG, "ctx is NULL");
  STC_TRY(check_coo(T, "T"));
  if (nmodes < 0 || nmodes > T->order || (nmodes > 0 && !modes))
    return fail(STC_ERR_INVALID_ARG, "bad mode list");
  if (T->nnz > 0 && !keys_out) return fail(STC_ERR_INVALID_ARG, "keys_out is NULL");
  KeyPlan p{};
  p.order = T->order;
  for (int j = 0; j < T->order; j++) p.size[j] = T->shape[j];
  bool seen[STC_MAX_ORDER] = {};
  unsigned __int128 acc = 1;
  for (int i = nmodes - 1; i >= 0; i--) {
    if (modes[i] < 0 || modes[i] >= T->order || seen[modes[i]]) return fail(STC_ERR_INVALID_ARG, "bad mode list");
    seen[modes[i]] = true;
    p.cstride[modes[i]] = (uint64_t)acc;
    acc *= (unsigned __int128)T->shape[modes[i]];
    if (acc > (unsigned __int128)UINT64_MAX) return fail(STC_ERR_KEY_OVERFLOW, "key space exceeds 2^64");
  }
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(STC_ERR_CUDA, "cannot make device %d current", ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Arena ar(ctx, s);
  uint32_t* status = nullptr;
  STC_TRY(ar.alloc(&status, 1));
  STC_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t), s));
  STC_CUDA(launch_linearize(T->coords, T->nnz, p, reinterpret_cast<u64*>(keys_out), status, ctx->sms, s));
  uint32_t h = 0;
  STC_CUDA(cudaMemcpyAsync(&h, status, sizeof(h), cudaMemcpyDeviceToHost, s));
  STC_CUDA(cudaStreamSynchronize(s));
  return status_word(h);
}

stc_status stc_group_keys(stc_ctx* ctx, const uint64_t* keys, int64_t n, uint64_t k, uint32_t* offsets_out,
                          uint32_t* perm_out, void* stream) {
  if (!ctx) return fail(STC_ERR_INVALID_ARG, "ctx is NULL");
  if (n < 0 || n > STC_MAX_NNZ) return fail(STC_ERR_INVALID_ARG, "n = %lld out of range", (long long)n);
  if (k > kMaxDirectBins) return fail(STC_ERR_UNSUPPORTED, "k = %llu exceeds 2^26", (unsigned long long)k);
  if (!offsets_out || (n > 0 && (!keys || !perm_out))) return fail(STC_ERR_INVALID_ARG, "NULL pointer");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(STC_ERR_CUDA, "cannot make device %d current", ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Arena ar(ctx, s);
  uint32_t *cnt = nullptr, *cur = nullptr, *scr = nullptr, *status = nullptr;
  STC_TRY(ar.alloc(&status, 1));
  STC_TRY(ar.alloc(&cnt, k));
  STC_TRY(ar.alloc(&cur, k));
  STC_TRY(ar.alloc(&scr, (size_t)scan_scratch_elems((int64_t)k)));
  STC_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t), s));
  if (k) STC_CUDA(cudaMemsetAsync(cnt, 0, k * sizeof(uint32_t), s));
  const u64* kk = reinterpret_cast<const u64*>(keys);
  STC_CUDA(launch_key_count(kk, n, k, cnt, status, ctx->sms, s));
  STC_CUDA(scan_u32(cnt, offsets_out, (int64_t)k, scr, s));
  if (k) STC_CUDA(cudaMemcpyAsync(cur, offsets_out, k * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  STC_CUDA(launch_key_scatter(kk, n, k, cur, perm_out, ctx->sms, s));
  uint32_t h = 0;
  STC_CUDA(cudaMemcpyAsync(&h, status, sizeof(h), cudaMemcpyDeviceToHost, s));
  STC_CUDA(cudaStreamSynchronize(s));
  return status_word(h);
}

stc_status stc_dense_ids(stc_ctx* ctx, const uint64_t* keys, int64_t n, uint32_t* ids_out, uint64_t* ndistinct,
                         void* stream) {
  if (!ctx) return fail(STC_ERR_INVALID_ARG, "ctx is NULL");
  if (n < 0 || n > STC_MAX_NNZ) return fail(STC_ERR_INVALID_ARG, "n = %lld out of range", (long long)n);
  if (!ndistinct || (n > 0 && (!keys || !ids_out))) return fail(STC_ERR_INVALID_ARG, "NULL pointer");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(STC_ERR_CUDA, "cannot make device %d current", ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Arena ar(ctx, s);
  IdTable t{};
  uint32_t *scr = nullptr, *status = nullptr;
  t.slots = id_table_slots(n);
  STC_TRY(ar.alloc(&t.keys, t.slots));
  STC_TRY(ar.alloc(&t.flags, t.slots + 1));
  STC_TRY(ar.alloc(&t.prefix, t.slots + 2));
  STC_TRY(ar.alloc(&scr, (size_t)scan_scratch_elems((int64_t)t.slots + 1)));
  STC_TRY(ar.alloc(&status, 1));
  STC_CUDA(cudaMemsetAsync(t.keys, 0xff, t.slots * sizeof(u64), s));
  STC_CUDA(cudaMemsetAsync(t.flags + t.slots, 0, sizeof(uint32_t), s));
  STC_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t), s));
  const u64* kk = reinterpret_cast<const u64*>(keys);
  STC_CUDA(launch_id_insert_keys(kk, n, t, status, ctx->sms, s));
  STC_CUDA(launch_id_number(t, scr, ctx->sms, s));
  STC_CUDA(launch_id_lookup_keys(kk, n, t, ids_out, ctx->sms, s));
  uint32_t h[2] = {0, 0};
  STC_CUDA(cudaMemcpyAsync(&h[0], status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  STC_CUDA(cudaMemcpyAsync(&h[1], t.prefix + t.slots + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  STC_CUDA(cudaStreamSynchronize(s));
  *ndistinct = h[1];
  return status_word(h[0]);
}

stc_status stc_result_info(const stc_result* r, int64_t* nnz, int32_t* order, const int64_t** shape) {
  if (!r) return fail(STC_ERR_INVALID_ARG, "result is NULL");
  if (nnz) *nnz = r->nnz;
  if (order) *order = r->order;
  if (shape) *shape = r->shape.empty() ? nullptr : r->shape.data();
  return STC_OK;
}

stc_status stc_result_data(const stc_result* r, const int32_t** coords, const double** vals) {
  if (!r) return fail(STC_ERR_INVALID_ARG, "result is NULL");
  if (coords) *coords = r->coords;
  if (vals) *vals = r->vals;
  return STC_OK;
}

stc_status stc_result_stats(const stc_result* r, stc_stats* stats) {
  if (!r || !stats) return fail(STC_ERR_INVALID_ARG, "NULL argument");
  *stats = r->stats;
  return STC_OK;
}

stc_status stc_result_as_coo(const stc_result* r, stc_coo* out) {
  if (!r || !out) return fail(STC_ERR_INVALID_ARG, "NULL argument");
  if (r->keys_form) return fail(STC_ERR_INVALID_ARG, "the result is in key form (stc_result_as_keyed)");
  out->order = r->order;
  out->shape = r->shape.empty() ? nullptr : r->shape.data();
  out->nnz = r->nnz;
  out->coords = r->coords;
  out->vals = r->vals;
  return STC_OK;
}

stc_status stc_result_keys(const stc_result* r, const uint64_t** keys) {
  if (!r || !keys) return fail(STC_ERR_INVALID_ARG, "NULL argument");
  *keys = r->keys_form ? reinterpret_cast<const uint64_t*>(r->coords) : nullptr;
  return STC_OK;
}

stc_status stc_result_as_keyed(const stc_result* r, stc_keyed* out) {
  if (!r || !out) return fail(STC_ERR_INVALID_ARG, "NULL argument");
  if (!r->keys_form) return fail(STC_ERR_INVALID_ARG, "the result holds coordinates, not keys");
  out->order = r->order;
  out->shape = r->shape.empty() ? nullptr : r->shape.data();
  out->nnz = r->nnz;
  out->keys = reinterpret_cast<const uint64_t*>(r->coords);
  out->vals = r->vals;
  return STC_OK;
}

stc_status stc_contract_keyed(stc_ctx* ctx, const stc_keyed* X, const stc_coo* Y, int32_t m, const int32_t* cx,
                              const int32_t* cy, const int32_t* out_order, const stc_opts* opts, void* stream,
                              stc_result** out) {
  if (!ctx || !out || !X) return fail(STC_ERR_INVALID_ARG, "ctx, X or out is NULL");
  *out = nullptr;
  if (X->order < 1 || X->order > STC_MAX_ORDER || !X->shape)
    return fail(STC_ERR_INVALID_ARG, "X.order = %d outside 1..%d", X->order, STC_MAX_ORDER);
  if (X->nnz < 0 || X->nnz > STC_MAX_NNZ || (X->nnz > 0 && (!X->keys || !X->vals)))
    return fail(STC_ERR_INVALID_ARG, "bad X.nnz, keys or vals");
  if (m < 0 || m > X->order || (m > 0 && (!cx || !cy))) return fail(STC_ERR_INVALID_ARG, "bad contract mode lists");
  for (int j = 0; j < X->order; j++)
    if (X->shape[j] < 1 || X->shape[j] > (int64_t)1 << 31)
      return fail(STC_ERR_INVALID_ARG, "X.shape[%d] = %lld outside 1..2^31", j, (long long)X->shape[j]);
  // The contracted modes: a contiguous block at the end (or the start) of X's modes, in order.
  bool trailing = true, leading = true;
  for (int i = 0; i < m; i++) {
    trailing = trailing && cx[i] == X->order - m + i;
    leading = leading && cx[i] == i;
  }
  if (!trailing && !leading)
    return fail(STC_ERR_INVALID_ARG, "X's contracted modes must be its last (or first) %d modes, in order", m);
  KeySplit ks{};
  ks.m = m;
  ks.trailing = trailing ? 1 : 0;
  unsigned __int128 K = 1, F = 1;
  std::vector<int64_t> xfree;
  for (int j = 0; j < X->order; j++) {
    const bool contracted = trailing ? j >= X->order - m : j < m;
    if (contracted) K *= (unsigned __int128)X->shape[j];
    else F *= (unsigned __int128)X->shape[j], xfree.push_back(X->shape[j]);
  }
  for (int i = 0; i < m; i++) ks.csize[i] = X->shape[cx[i]];
  if (K * F > (unsigned __int128)UINT64_MAX) return fail(STC_ERR_KEY_OVERFLOW, "X's key space exceeds 2^64");
  if (K > kMaxDirectBins) return fail(STC_ERR_UNSUPPORTED, "X's contract key space exceeds 2^26");
  ks.K = (u64)K;
  ks.F = (u64)F;
  ks.FL = std::min<u64>(ks.F, 1ull << 30);
  const u64 FH = (ks.F + ks.FL - 1) / ks.FL;
  if (FH > (1ull << 31)) return fail(STC_ERR_UNSUPPORTED, "X's free key space exceeds 2^61");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(STC_ERR_CUDA, "cannot make device %d current", ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Arena ar(ctx, s);
  int32_t* rows = nullptr;
  uint32_t* status = nullptr;
  STC_TRY(ar.alloc(&rows, (size_t)X->nnz * (2 + m)));
  STC_TRY(ar.alloc(&status, 1));
  STC_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t), s));
  take_launches();
  STC_CUDA(launch_keyed_split(reinterpret_cast<const u64*>(X->keys), X->nnz, ks, rows, status, ctx->sms, s));
  const unsigned split_launches = take_launches();
  // The split form: modes (free / FL, free % FL, contracted modes), its free key the original
  // free index, paired on its last m modes.
  std::vector<int64_t> shape2 = {(int64_t)FH, (int64_t)ks.FL};
  std::vector<int32_t> cx2(m);
  for (int i = 0; i < m; i++) shape2.push_back(ks.csize[i]), cx2[i] = 2 + i;
  const stc_coo X2{2 + m, shape2.data(), X->nnz, rows, X->vals};
  stc_opts o = opts ? *opts : stc_opts{};
  o.operands = STC_OPERANDS_AS_GIVEN;
  o.contract_ids = STC_IDS_DIRECT;
  STC_TRY(contract_impl(ctx, &X2, Y, m, cx2.data(), cy, out_order, &o, stream, out, &xfree));
  uint32_t h = 0;
  const cudaError_t e1 = cudaMemcpyAsync(&h, status, sizeof(h), cudaMemcpyDeviceToHost, s);
  const cudaError_t e2 = e1 == cudaSuccess ? cudaStreamSynchronize(s) : e1;
  const stc_status st = e2 != cudaSuccess ? fail(STC_ERR_CUDA, "%s", cudaGetErrorString(e2)) : status_word(h);
  if (st != STC_OK) {
    stc_result_free(*out);
    *out = nullptr;
    return st;
  }
  (*out)->stats.launches += split_launches;
  return STC_OK;
}

stc_status stc_result_free(stc_result* r) {
  if (!r) return STC_OK;
  r->ctx->live_results--;
  delete r;
  return STC_OK;
}

}  // extern "C"
