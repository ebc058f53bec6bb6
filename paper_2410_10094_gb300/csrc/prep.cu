// Input processing on the device: LN keys (Section 2.4.1), grouping of Y by contract key
// with a counting sort (Sections 4.1.1 and 4.2), and the survey of X that finds each
// entry's Y run and counts the products exactly (Section 4.3).
#include "launch.h"

namespace stc {

namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(int64_t n, int sms, int per_sm = 8) {
  const int64_t want = (n + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)sms * per_sm;
  return (unsigned)(want < cap ? want : cap);
}

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Warp-uniform grid-stride loop: every lane of a warp runs the same iterations, so warp
// collectives inside the body are safe. `i` is this lane's element (may be >= n).
#define STC_WARP_LOOP(i, n)                                                                      \
  for (int64_t base_ = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u), i = base_ + lane_id(); \
       base_ < (n); base_ += (int64_t)gridDim.x * blockDim.x, i = base_ + lane_id())

template <int ORDER, bool VEC>
__global__ void __launch_bounds__(kThreads) linearize_kernel(const int32_t* __restrict__ coords, int64_t n,
                                                             KeyPlan p, u64* __restrict__ keys,
                                                             uint32_t* status) {
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
    uint64_t ck, fk;
    if (!row_keys<ORDER, VEC>(coords, i, p, ck, fk)) atomicOr(status, kStatCoordRange);
    keys[i] = ck;
  }
}

__global__ void __launch_bounds__(kThreads) key_count_kernel(const u64* __restrict__ keys, int64_t n, u64 k,
                                                             uint32_t* __restrict__ cnt, uint32_t* status) {
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
    const u64 key = keys[i];
    if (key >= k) {
      atomicOr(status, kStatCoordRange);
      continue;
    }
    atomicAdd(cnt + key, 1u);
  }
}

__global__ void __launch_bounds__(kThreads) key_scatter_kernel(const u64* __restrict__ keys, int64_t n, u64 k,
                                                               uint32_t* __restrict__ cursor,
                                                               uint32_t* __restrict__ perm) {
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
    const u64 key = keys[i];
    if (key >= k) continue;
    const uint32_t pos = atomicAdd(cursor + key, 1u);
    perm[pos] = (uint32_t)i;
  }
}

// Row-streaming kernels take R rows per thread per step and issue all of their loads before
// using any, so each thread keeps R coordinate rows (and their lookups) in flight.
constexpr int kRows = 4;
// Row streams over X: at least this many CTAs per SM (keeps enough rows in flight).
#ifndef STC_X_MIN_BLOCKS
#define STC_X_MIN_BLOCKS 4
#endif
constexpr int kXMinBlocks = STC_X_MIN_BLOCKS;
#ifndef STC_STAGE_ROWS
#define STC_STAGE_ROWS 1
#endif
constexpr bool kStageRows = STC_STAGE_ROWS != 0;

template <int ORDER, bool VEC>
// With `nonempty` non-null, also sets bit c of it for every contract key c that has an entry
// (when the first entry of one of its bins is counted): the survey's bitmap of keys with a run.
__global__ void __launch_bounds__(kThreads) y_count_kernel(const int32_t* __restrict__ coords, int64_t n, KeyPlan p,
                                                           uint32_t* __restrict__ cnt, uint32_t* status,
                                                           uint32_t* __restrict__ nonempty) {
  const int64_t step = (int64_t)gridDim.x * kThreads * kRows;
  for (int64_t base = (int64_t)blockIdx.x * kThreads * kRows + threadIdx.x; base < n; base += step) {
    uint64_t ck[kRows], fk[kRows];
    bool ok[kRows];
#pragma unroll
    for (int r = 0; r < kRows; r++) {
      const int64_t i = base + (int64_t)r * kThreads;
      ok[r] = i < n ? row_keys<ORDER, VEC>(coords, i, p, ck[r], fk[r]) : true;
      if (i >= n) ck[r] = kEmpty64;
    }
#pragma unroll
    for (int r = 0; r < kRows; r++) {
      if (!ok[r]) {
        atomicOr(status, kStatCoordRange);
      } else if (ck[r] != kEmpty64) {
        uint32_t* const bin = cnt + ck[r] * p.nseg + (p.nseg > 1 ? (fk[r] >> p.seg_shift) : 0);
        if (nonempty) {
          if (atomicAdd(bin, 1u) == 0u) atomicOr(nonempty + (ck[r] >> 5), 1u << (ck[r] & 31));
        } else {
          atomicAdd(bin, 1u);
        }
      }
    }
  }
}

template <int ORDER, bool VEC, typename YK>
__global__ void __launch_bounds__(kThreads) y_scatter_kernel(const int32_t* __restrict__ coords,
                                                             const double* __restrict__ vals, int64_t n, KeyPlan p,
                                                             uint32_t* __restrict__ cursor, YK* __restrict__ yfk,
                                                             double* __restrict__ yv) {
  const int64_t step = (int64_t)gridDim.x * kThreads * kRows;
  for (int64_t base = (int64_t)blockIdx.x * kThreads * kRows + threadIdx.x; base < n; base += step) {
    uint64_t ck[kRows], fk[kRows];
    bool ok[kRows];
    double v[kRows];
#pragma unroll
    for (int r = 0; r < kRows; r++) {
      const int64_t i = base + (int64_t)r * kThreads;
      ok[r] = false;
      if (i < n) {
        ok[r] = row_keys<ORDER, VEC>(coords, i, p, ck[r], fk[r]);
        v[r] = __ldg(vals + i);
      }
    }
#pragma unroll
    for (int r = 0; r < kRows; r++) {
      if (!ok[r]) continue;
      const uint32_t pos = atomicAdd(cursor + ck[r] * p.nseg + (p.nseg > 1 ? (fk[r] >> p.seg_shift) : 0), 1u);
      yfk[pos] = (YK)fk[r];
      yv[pos] = v[r];
    }
  }
}

// Warp-uniform loop over blocks of 32 * kRows consecutive rows; lane l takes rows
// base + l + 32 r, so every load instruction of a warp reads consecutive rows.
#define STC_WARP_ROWS(base, n)                                                                   \
  for (int64_t base = ((int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5)) * 32 * kRows; \
       base < (n); base += (int64_t)gridDim.x * kThreads * kRows)

// Looks up each row's Y run: lo = first slot, w = length (0 when the key has no run or the
// row is invalid). Invalid coordinates raise kStatCoordRange.
// The coordinates of a warp's block of rows [base, base + 32 * kRows), read with 16-byte
// loads of the whole block (coalesced whatever the order) and handed out through shared
// memory: lane l receives rows base + l + 32 r.
template <int ORDER>
__device__ __forceinline__ void stage_rows(const int32_t* __restrict__ coords, int64_t base, int64_t n,
                                           int32_t (&c)[kRows][ORDER]) {
  constexpr int kInts = 32 * kRows * ORDER;
  __shared__ __align__(16) int32_t buf[kThreads / 32][kInts];
  int32_t* wb = buf[threadIdx.x >> 5];
  const int lane = (int)lane_id();
  const int rows = n - base < 32 * kRows ? (int)(n - base) : 32 * kRows;
  const int total = rows * ORDER;
  const int32_t* src = coords + base * ORDER;
  int k0 = 0;
  if ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
    const int nv = total >> 2;
    int4 t[(kInts / 4 + 31) / 32];
#pragma unroll
    for (int it = 0; it < (kInts / 4 + 31) / 32; it++) {
      const int k = lane + 32 * it;
      if (k < nv) t[it] = __ldg(reinterpret_cast<const int4*>(src) + k);
    }
#pragma unroll
    for (int it = 0; it < (kInts / 4 + 31) / 32; it++) {
      const int k = lane + 32 * it;
      if (k < nv) reinterpret_cast<int4*>(wb)[k] = t[it];
    }
    k0 = nv << 2;
  }
  for (int k = k0 + lane; k < total; k += 32) wb[k] = __ldg(src + k);
  __syncwarp();
#pragma unroll
  for (int r = 0; r < kRows; r++) {
    const int row = lane + 32 * r;
#pragma unroll
    for (int q = 0; q < ORDER; q++) c[r][q] = row < rows ? wb[row * ORDER + q] : 0;
  }
  __syncwarp();
}

// `nonempty` (shared memory, may be null) has bit c set when contract key c has a Y run: rows
// whose bit is clear skip the run lookup.
template <int ORDER, bool VEC>
__device__ __forceinline__ void rows_runs(const int32_t* __restrict__ coords, int64_t base, int64_t n,
                                          const KeyPlan& p, const uint32_t* __restrict__ yoff, uint64_t* fk,
                                          uint32_t* lo, uint32_t* w, uint32_t* status, uint64_t* ck,
                                          const uint32_t* nonempty = nullptr) {
  bool ok[kRows];
  if constexpr (kStageRows && !VEC && ORDER >= 3) {
    int32_t c[kRows][ORDER];
    stage_rows<ORDER>(coords, base, n, c);
#pragma unroll
    for (int r = 0; r < kRows; r++) {
      const int64_t i = base + lane_id() + 32 * r;
      ok[r] = false;
      if (i < n) {
        ok[r] = keys_of<ORDER>(c[r], p, ck[r], fk[r]);
        if (!ok[r]) atomicOr(status, kStatCoordRange);
      }
    }
  } else {
#pragma unroll
    for (int r = 0; r < kRows; r++) {
      const int64_t i = base + lane_id() + 32 * r;
      ok[r] = false;
      if (i < n) {
        ok[r] = row_keys<ORDER, VEC>(coords, i, p, ck[r], fk[r]);
        if (!ok[r]) atomicOr(status, kStatCoordRange);
      }
    }
  }
  if (nonempty) {
#pragma unroll
    for (int r = 0; r < kRows; r++)
      if (ok[r]) ok[r] = (nonempty[ck[r] >> 5] >> (ck[r] & 31)) & 1u;
  }
#pragma unroll
  for (int r = 0; r < kRows; r++) {
    lo[r] = 0;
    w[r] = 0;
    if (ok[r]) {
      lo[r] = __ldg(yoff + ck[r] * p.nseg);
      w[r] = __ldg(yoff + (ck[r] + 1) * p.nseg);
    }
  }
#pragma unroll
  for (int r = 0; r < kRows; r++) w[r] -= lo[r];
}

// Bit c of `bits` is set when contract key c has a Y run (any segment).
__global__ void __launch_bounds__(kThreads) nonempty_kernel(const uint32_t* __restrict__ yoff, u64 K, uint32_t nseg,
                                                            uint32_t* __restrict__ bits) {
  const u64 words = (K + 31) / 32;
  for (u64 wi = (u64)blockIdx.x * kThreads + threadIdx.x; wi < words; wi += (u64)gridDim.x * kThreads) {
    uint32_t b = 0;
    for (int j = 0; j < 32; j++) {
      const u64 c = wi * 32 + j;
      if (c < K && yoff[(c + 1) * nseg] > yoff[c * nseg]) b |= 1u << j;
    }
    bits[wi] = b;
  }
}

// A warp's share of a row stream read as whole blocks of 32 * kRows rows with 16-byte loads
// (coords 16-byte aligned): load() issues a block's loads, unpack() hands lane l the rows
// block + l + 32 r. Holding two of these keeps the next block's loads in flight while the
// current block is processed.
template <int ORDER>
struct RowBlock {
  static constexpr int kVec = 32 * kRows * ORDER / 4;  // int4 per block
  static constexpr int NV = (kVec + 31) / 32;
  int4 t[NV];
  __device__ __forceinline__ void load(const int32_t* __restrict__ coords, int64_t blk) {
    const int4* src = reinterpret_cast<const int4*>(coords + blk * (32 * kRows * ORDER));
    const int lane = (int)lane_id();
#pragma unroll
    for (int it = 0; it < NV; it++)
      if (lane + 32 * it < kVec) t[it] = __ldg(src + lane + 32 * it);
  }
  __device__ __forceinline__ void unpack(int4* wb, int32_t (&c)[kRows][ORDER]) const {
    const int lane = (int)lane_id();
    if constexpr (ORDER == 4) {
#pragma unroll
      for (int r = 0; r < kRows; r++) {
        c[r][0] = t[r].x; c[r][1] = t[r].y; c[r][2] = t[r].z; c[r][3] = t[r].w;
      }
    } else {
#pragma unroll
      for (int it = 0; it < NV; it++)
        if (lane + 32 * it < kVec) wb[lane + 32 * it] = t[it];
      __syncwarp();
      const int32_t* w32 = reinterpret_cast<const int32_t*>(wb);
#pragma unroll
      for (int r = 0; r < kRows; r++)
#pragma unroll
        for (int q = 0; q < ORDER; q++) c[r][q] = w32[(lane + 32 * r) * ORDER + q];
      __syncwarp();
    }
  }
};

template <int ORDER, bool VEC, bool GROUPS>
__global__ void __launch_bounds__(kThreads, 3) x_survey_kernel(const int32_t* __restrict__ coords,
                                                            const double* __restrict__ vals, int64_t n, KeyPlan p,
                                                            const uint32_t* __restrict__ yoff, Survivors sv,
                                                            u64* __restrict__ P, uint32_t* __restrict__ gcnt,
                                                            uint32_t* status, const uint32_t* __restrict__ nonempty,
                                                            uint32_t ne_words) {
  extern __shared__ __align__(16) uint32_t s_nonempty[];
  __shared__ u64 warp_p[kThreads / 32];
  if (ne_words) {
    for (uint32_t i = threadIdx.x; i < ne_words; i += kThreads) s_nonempty[i] = nonempty[i];
    __syncthreads();
  }
  const uint32_t* ne = ne_words ? s_nonempty : nullptr;
  // Survivors are gathered per warp in shared memory and appended 32 or more at a time: one
  // atomic on the shared survivor counter per flush instead of one per warp and row step. Their
  // runs and values are read at the flush, all lanes at once, so that with the bitmap the row
  // stream itself waits on no lookup.
  __shared__ u64 b_fk[kThreads / 32][64], b_row[kThreads / 32][64];
  __shared__ uint32_t b_ck[kThreads / 32][64];
  constexpr int OD = ORDER > 0 ? ORDER : 1;
  __shared__ int4 rowbuf[kThreads / 32][ORDER == 4 ? 1 : RowBlock<OD>::kVec];
  const unsigned lane = lane_id(), wq = threadIdx.x >> 5;
  uint32_t held = 0;  // warp-uniform
  u64 my_p = 0;
  auto flush = [&]() {
    __syncwarp();
    unsigned pos = 0;
    if (lane == 0) pos = atomicAdd(sv.count, held);
    pos = __shfl_sync(0xffffffffu, pos, 0);
    for (uint32_t k = lane; k < held; k += 32) {
      const uint32_t c = b_ck[wq][k];
      const u64 fk = b_fk[wq][k];
      const uint32_t lo = __ldg(yoff + (u64)c * p.nseg);
      const uint32_t w = __ldg(yoff + ((u64)c + 1) * p.nseg) - lo;
      const double v = __ldg(vals + b_row[wq][k]);
      sv.fk[pos + k] = fk;
      if (sv.ck) sv.ck[pos + k] = c;
      sv.ystart[pos + k] = lo;
      sv.w[pos + k] = w;
      sv.v[pos + k] = v;
      my_p += w;
      if (GROUPS) atomicAdd(gcnt + fk, 1u);
    }
    __syncwarp();
    held = 0;
  };
  // Rows [base, base + 32 * kRows) with their coordinates in c.
  auto process = [&](int64_t base, int32_t (&c)[kRows][OD]) {
    uint64_t fk[kRows], ck[kRows];
    bool live[kRows];
#pragma unroll
    for (int r = 0; r < kRows; r++) {
      live[r] = false;
      if (base + lane + 32 * r < n) {
        live[r] = keys_of<ORDER>(c[r], p, ck[r], fk[r]);
        if (!live[r]) atomicOr(status, kStatCoordRange);
        else if (ne) live[r] = (ne[ck[r] >> 5] >> (ck[r] & 31)) & 1u;
      }
    }
    if (!ne) {
#pragma unroll
      for (int r = 0; r < kRows; r++)
        if (live[r]) live[r] = __ldg(yoff + (ck[r] + 1) * p.nseg) > __ldg(yoff + ck[r] * p.nseg);
    }
#pragma unroll
    for (int r = 0; r < kRows; r++) {
      const unsigned m = __ballot_sync(0xffffffffu, live[r]);
      if (live[r]) {
        const uint32_t k = held + __popc(m & lanemask_lt());
        b_fk[wq][k] = fk[r];
        b_ck[wq][k] = (uint32_t)ck[r];
        b_row[wq][k] = (u64)(base + lane + 32 * r);
      }
      held += __popc(m);
      if (held >= 32) flush();
    }
  };
  const int64_t nw = (int64_t)gridDim.x * (kThreads / 32);
  int64_t blk = (int64_t)blockIdx.x * (kThreads / 32) + wq;
  if constexpr (ORDER > 0) {
    if ((reinterpret_cast<uintptr_t>(coords) & 15u) == 0) {
      // Whole blocks, two in flight per warp.
      const int64_t nfull = n / (32 * kRows);
      RowBlock<ORDER> cur, nxt;
      if (blk < nfull) cur.load(coords, blk);
      for (; blk < nfull; blk += nw) {
        if (blk + nw < nfull) nxt.load(coords, blk + nw);
        int32_t c[kRows][OD];
        cur.unpack(rowbuf[wq], c);
        process(blk * (32 * kRows), c);
        cur = nxt;
      }
    }
  }
  // The last partial block, or every block when the coordinates are not 16-byte aligned.
  for (; blk * (32 * kRows) < n; blk += nw) {
    int32_t c[kRows][OD];
    const int64_t base = blk * (32 * kRows);
#pragma unroll
    for (int r = 0; r < kRows; r++)
#pragma unroll
      for (int q = 0; q < ORDER; q++)
        c[r][q] = base + lane + 32 * r < n ? __ldg(coords + (base + lane + 32 * r) * ORDER + q) : 0;
    process(base, c);
  }
  if (held) flush();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_p += __shfl_down_sync(0xffffffffu, my_p, o);
  if (lane_id() == 0) warp_p[threadIdx.x >> 5] = my_p;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 t = 0;
    for (int k = 0; k < kThreads / 32; k++) t += warp_p[k];
    if (t) atomicAdd(P, t);
  }
}

// Dense X (most entries have a Y run): count entries per X free key and the products,
// without writing a survivor list.
template <int ORDER, bool VEC>
__global__ void __launch_bounds__(kThreads, kXMinBlocks) x_count_kernel(const int32_t* __restrict__ coords, int64_t n, KeyPlan p,
                                                           const uint32_t* __restrict__ yoff, u64* __restrict__ P,
                                                           uint32_t* __restrict__ gcnt, uint32_t* status) {
  __shared__ u64 warp_p[kThreads / 32];
  u64 my_p = 0;
  STC_WARP_ROWS(base, n) {
    uint64_t fk[kRows], ck[kRows];
    uint32_t lo[kRows], w[kRows];
    rows_runs<ORDER, VEC>(coords, base, n, p, yoff, fk, lo, w, status, ck);
#pragma unroll
    for (int r = 0; r < kRows; r++) {
      if (w[r] > 0) {
        my_p += w[r];
        atomicAdd(gcnt + fk[r], 1u);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_p += __shfl_down_sync(0xffffffffu, my_p, o);
  if (lane_id() == 0) warp_p[threadIdx.x >> 5] = my_p;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 t = 0;
    for (int k = 0; k < kThreads / 32; k++) t += warp_p[k];
    if (t) atomicAdd(P, t);
  }
}

// Dense X: read X again and place every entry with a Y run at its group's cursor.
template <int ORDER, bool VEC>
__global__ void __launch_bounds__(kThreads, kXMinBlocks) x_scatter_dense_kernel(const int32_t* __restrict__ coords,
                                                                   const double* __restrict__ vals, int64_t n,
                                                                   KeyPlan p, const uint32_t* __restrict__ yoff,
                                                                   uint32_t* __restrict__ gcur, GroupedX gx,
                                                                   uint32_t* status) {
  STC_WARP_ROWS(base, n) {
    uint64_t fk[kRows], ck[kRows];
    uint32_t lo[kRows], w[kRows];
    double v[kRows];
#pragma unroll
    for (int r = 0; r < kRows; r++) {
      const int64_t i = base + lane_id() + 32 * r;
      if (i < n) v[r] = __ldg(vals + i);
    }
    rows_runs<ORDER, VEC>(coords, base, n, p, yoff, fk, lo, w, status, ck);
#pragma unroll
    for (int r = 0; r < kRows; r++) {
      if (w[r] > 0) {
        const uint32_t pos = atomicAdd(gcur + fk[r], 1u);
        if (gx.ck) gx.ck[pos] = (uint32_t)ck[r];
        gx.ystart[pos] = lo[r];
        gx.w[pos] = w[r];
        gx.v[pos] = v[r];
      }
    }
  }
}

// ---- the survey with X's coordinates streamed through shared memory by bulk copies: one
// persistent CTA per SM, a ring of kSvStages chunks of coordinate rows filled by one producer
// thread (cp.async.bulk, completion counted on the stage's mbarrier) and consumed by
// kSvConsumers warps, which release each stage through a second mbarrier. The copies keep
// up to kSvStages chunks per SM in flight without holding them in registers. Rows whose
// contract key has a Y run (bitmap in shared memory) are appended to the survivor list as in
// x_survey_kernel. Needs 16-byte aligned coordinates and K <= kNonemptyMaxKeys.
#ifndef SV_CONSUMERS
#define SV_CONSUMERS 24
#endif
#ifndef SV_STAGES
#define SV_STAGES 6
#endif
#ifndef SV_ROWS
#define SV_ROWS 1536
#endif
constexpr int kSvConsumers = SV_CONSUMERS;
constexpr int kSvThreads = (kSvConsumers + 1) * 32;
constexpr int kSvStages = SV_STAGES;
template <int ORDER>
__host__ __device__ constexpr int sv_rows() {
  // rows per chunk: a multiple of 4 (16-byte chunk sizes) and of 32 * kSvConsumers
  return ORDER <= 4 || SV_ROWS / 2 < 32 * kSvConsumers ? SV_ROWS : SV_ROWS / 2;
}
template <int ORDER>
__host__ __device__ constexpr size_t sv_ring_bytes() {
  return (size_t)kSvStages * sv_rows<ORDER>() * ORDER * 4;
}

// Static shared memory of x_survey_bulk_kernel: the consumers' survivor buffers (free key,
// contract key, row), their product sums, the ring's mbarriers, the abort flag.
constexpr size_t kSvStatic = (size_t)kSvConsumers * 64 * (8 + 4 + 8) + (size_t)kSvConsumers * 8 +
                             (size_t)kSvStages * 16 + 256;  // + alignment
static_assert(sv_ring_bytes<4>() + kNonemptyMaxKeys / 8 + kSvStatic <= 227 * 1024 &&
                  sv_ring_bytes<8>() + kNonemptyMaxKeys / 8 + kSvStatic <= 227 * 1024,
              "the survey's ring, key bitmap and buffers fit one CTA's shared memory");

// KEY32: contract keys below 2^32, formed in 32-bit arithmetic; the free key (64-bit) is formed
// only for the rows that survive.
template <int ORDER, bool GROUPS, bool KEY32>
__global__ void __launch_bounds__(kSvThreads, 1) x_survey_bulk_kernel(const int32_t* __restrict__ coords,
                                                                     const double* __restrict__ vals, int64_t n,
                                                                     KeyPlan p, const uint32_t* __restrict__ yoff,
                                                                     Survivors sv, u64* __restrict__ P,
                                                                     uint32_t* __restrict__ gcnt, uint32_t* status,
                                                                     const uint32_t* __restrict__ nonempty,
                                                                     uint32_t ne_words) {
  constexpr int R = sv_rows<ORDER>();
  constexpr int RPW = R / kSvConsumers;  // rows of a chunk per consumer warp
  static_assert(R % 4 == 0 && RPW % 32 == 0, "chunk shape");
  extern __shared__ __align__(128) unsigned char smem[];
  int32_t* const ring = reinterpret_cast<int32_t*>(smem);
  uint32_t* const ne = reinterpret_cast<uint32_t*>(smem + sv_ring_bytes<ORDER>());
  __shared__ __align__(8) uint64_t full[kSvStages], empty[kSvStages];
  __shared__ u64 b_fk[kSvConsumers][64];
  __shared__ uint32_t b_ck[kSvConsumers][64];
  __shared__ u64 b_row[kSvConsumers][64];
  __shared__ u64 warp_p[kSvConsumers];
  __shared__ int s_abort;
  const unsigned lane = lane_id(), wq = threadIdx.x >> 5;
  const int64_t nchunks = n / R;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kSvStages; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kSvConsumers);
    }
    s_abort = 0;
    fence_mbar_init();
  }
  for (uint32_t i = threadIdx.x; i < ne_words; i += kSvThreads) ne[i] = nonempty[i];
  __syncthreads();

  if (wq == kSvConsumers) {
    // ---- producer: one thread issues the chunk copies of this CTA, kSvStages ahead.
    if (lane == 0) {
      int64_t issued = 0;
      for (int64_t k = 0;; k++) {
        const int64_t c = (int64_t)blockIdx.x + k * gridDim.x;
        if (c >= nchunks) break;
        const int st = (int)(k % kSvStages);
        const uint32_t round = (uint32_t)(k / kSvStages);
        if (round > 0 && !mbar_wait(&empty[st], (round - 1) & 1u)) {
          atomicOr(status, kStatTimeout);
          s_abort = 1;
          break;
        }
        if (s_abort) break;
        constexpr uint32_t bytes = (uint32_t)(R * ORDER * 4);
        mbar_arrive_expect_tx(&full[st], bytes);
        bulk_load(ring + (size_t)st * R * ORDER, coords + c * (int64_t)R * ORDER, bytes, &full[st]);
        issued = k + 1;
      }
      if (s_abort) {
        // Let the copies already issued land before the CTA exits (bounded).
        const int64_t k0 = issued > kSvStages ? issued - kSvStages : 0;
        for (int64_t k = k0; k < issued; k++) mbar_wait(&full[k % kSvStages], (uint32_t)(k / kSvStages) & 1u);
      }
    }
    return;
  }
  // ---- consumers.
  uint32_t held = 0;  // warp-uniform
  u64 my_p = 0;
  auto flush = [&]() {
    __syncwarp();
    unsigned pos = 0;
    if (lane == 0) pos = atomicAdd(sv.count, held);
    pos = __shfl_sync(0xffffffffu, pos, 0);
    for (uint32_t k = lane; k < held; k += 32) {
      const uint32_t c = b_ck[wq][k];
      const u64 fk = b_fk[wq][k];
      const uint32_t lo = __ldg(yoff + (u64)c * p.nseg);
      const uint32_t w = __ldg(yoff + ((u64)c + 1) * p.nseg) - lo;
      const double v = __ldg(vals + b_row[wq][k]);
      sv.fk[pos + k] = fk;
      if (sv.ck) sv.ck[pos + k] = c;
      sv.ystart[pos + k] = lo;
      sv.w[pos + k] = w;
      sv.v[pos + k] = v;
      my_p += w;
      if (GROUPS) atomicAdd(gcnt + fk, 1u);
    }
    __syncwarp();
    held = 0;
  };
  uint32_t cs32[ORDER > 0 ? ORDER : 1], sz32[ORDER > 0 ? ORDER : 1];
#pragma unroll
  for (int j = 0; j < ORDER; j++) {
    cs32[j] = (uint32_t)p.cstride[j];
    sz32[j] = (uint32_t)p.size[j];
  }
  // One row per lane: keys, the range check, the bitmap test, and the append of survivors.
  auto take = [&](const int32_t* c, int64_t row, bool in) {
    uint64_t ck = 0, fk = 0;
    bool live = false;
    if (in) {
      bool ok;
      if constexpr (KEY32) {
        uint32_t k = 0;
        ok = true;
#pragma unroll
        for (int j = 0; j < ORDER; j++) {
          ok &= (uint32_t)c[j] < sz32[j];
          k += (uint32_t)c[j] * cs32[j];
        }
        ck = k;
      } else {
        ok = keys_of<ORDER>(c, p, ck, fk);
      }
      if (!ok) atomicOr(status, kStatCoordRange);
      live = ok && ((ne[ck >> 5] >> (ck & 31)) & 1u);
      if (KEY32 && live) {
#pragma unroll
        for (int j = 0; j < ORDER; j++) fk += (uint64_t)(uint32_t)c[j] * p.fstride[j];
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, live);
    if (live) {
      const uint32_t k = held + __popc(m & lanemask_lt());
      b_fk[wq][k] = fk;
      b_ck[wq][k] = (uint32_t)ck;
      b_row[wq][k] = (u64)row;
    }
    held += __popc(m);
    if (held >= 32) flush();
  };
  bool aborted = false;
  for (int64_t k = 0;; k++) {
    const int64_t c = (int64_t)blockIdx.x + k * gridDim.x;
    if (c >= nchunks) break;
    const int st = (int)(k % kSvStages);
    if (!mbar_wait(&full[st], (uint32_t)(k / kSvStages) & 1u)) {
      atomicOr(status, kStatTimeout);
      s_abort = 1;
      aborted = true;
      break;
    }
    const int32_t* rows = ring + (size_t)st * R * ORDER;
#pragma unroll
    for (int i = 0; i < RPW / 32; i++) {
      const int r = (int)wq * RPW + i * 32 + (int)lane;
      int32_t cr[ORDER > 0 ? ORDER : 1];
#pragma unroll
      for (int j = 0; j < ORDER; j++) cr[j] = rows[r * ORDER + j];
      take(cr, c * R + r, true);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[st]);
  }
  // The rows after the last whole chunk, read directly by the last CTA.
  if (!aborted && blockIdx.x == gridDim.x - 1) {
    for (int64_t base = nchunks * R + (int64_t)wq * 32; base < n; base += 32 * kSvConsumers) {
      const int64_t row = base + lane;
      int32_t cr[ORDER > 0 ? ORDER : 1];
#pragma unroll
      for (int j = 0; j < ORDER; j++) cr[j] = row < n ? __ldg(coords + row * ORDER + j) : 0;
      take(cr, row, row < n);
    }
  }
  if (held) flush();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_p += __shfl_down_sync(0xffffffffu, my_p, o);
  if (lane == 0) warp_p[wq] = my_p;
  // Consumer warps only (the producer warp has returned): a named barrier over them.
  asm volatile("bar.sync 1, %0;" ::"n"(kSvConsumers * 32) : "memory");
  if (threadIdx.x == 0) {
    u64 t = 0;
    for (int k = 0; k < kSvConsumers; k++) t += warp_p[k];
    if (t) atomicAdd(P, t);
  }
}

// The split form of a tensor in key form (chains of contractions): row i = (f / FL, f % FL,
// c_1 .. c_m), where the key's free part f and contract part c are key / K and key % K when
// the contracted modes are the last ones, key % F and key / F when they are the first ones,
// and c_1 .. c_m are c's digits over the contracted modes' lengths, first most significant.
// The free part stays one number: the row-major index over the free modes.
__global__ void __launch_bounds__(kThreads) keyed_split_kernel(const u64* __restrict__ keys, int64_t n, KeySplit ks,
                                                               int32_t* __restrict__ out, uint32_t* status) {
  const int w = 2 + ks.m;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
    const u64 key = keys[i];
    int32_t* row = out + i * w;
    if (key / ks.F >= ks.K) {  // outside prod(shape)
      atomicOr(status, kStatCoordRange);
      for (int j = 0; j < w; j++) row[j] = 0;
      continue;
    }
    u64 f, c;
    if (ks.trailing) {
      f = key / ks.K;
      c = key - f * ks.K;
    } else {
      c = key / ks.F;
      f = key - c * ks.F;
    }
    const u64 fh = f / ks.FL;
    row[0] = (int32_t)fh;
    row[1] = (int32_t)(f - fh * ks.FL);
    for (int j = ks.m - 1; j >= 0; j--) {
      const u64 q = c / (u64)ks.csize[j];
      row[2 + j] = (int32_t)(c - q * (u64)ks.csize[j]);
      c = q;
    }
  }
}

// Runs `body.template operator()<ORDER, VEC>()` for the runtime order and alignment.
template <typename F>
cudaError_t dispatch_order(int order, bool vec, F&& body) {
  switch (order) {
    case 0: return body.template operator()<0, false>();
    case 1: return body.template operator()<1, false>();
    case 2: return vec ? body.template operator()<2, true>() : body.template operator()<2, false>();
    case 3: return body.template operator()<3, false>();
    case 4: return vec ? body.template operator()<4, true>() : body.template operator()<4, false>();
    case 5: return body.template operator()<5, false>();
    case 6: return body.template operator()<6, false>();
    case 7: return body.template operator()<7, false>();
    case 8: return body.template operator()<8, false>();
    default: return cudaErrorInvalidValue;
  }
}

inline bool vec_ok(const int32_t* coords, int order) {
  if (order == 4) return aligned16(coords);
  if (order == 2) return (reinterpret_cast<uintptr_t>(coords) & 7u) == 0;
  return false;
}

}  // namespace

cudaError_t launch_linearize(const int32_t* coords, int64_t n, const KeyPlan& p, u64* keys, uint32_t* status,
                             int sms, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const unsigned g = grid_for(n, sms);
  return dispatch_order(p.order, vec_ok(coords, p.order), [&]<int O, bool V>() {
    linearize_kernel<O, V><<<g, kThreads, 0, s>>>(coords, n, p, keys, status);
    note_launch();
    return cudaGetLastError();
  });
}

cudaError_t launch_key_count(const u64* keys, int64_t n, u64 k, uint32_t* cnt, uint32_t* status, int sms,
                             cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  key_count_kernel<<<grid_for(n, sms), kThreads, 0, s>>>(keys, n, k, cnt, status);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_key_scatter(const u64* keys, int64_t n, u64 k, uint32_t* cursor, uint32_t* perm, int sms,
                               cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  key_scatter_kernel<<<grid_for(n, sms), kThreads, 0, s>>>(keys, n, k, cursor, perm);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_y_count(const int32_t* coords, int64_t n, const KeyPlan& p, uint32_t* cnt, uint32_t* status,
                           int sms, cudaStream_t s, uint32_t* nonempty) {
  if (n <= 0) return cudaSuccess;
  const unsigned g = grid_for((n + kRows - 1) / kRows, sms);
  return dispatch_order(p.order, vec_ok(coords, p.order), [&]<int O, bool V>() {
    y_count_kernel<O, V><<<g, kThreads, 0, s>>>(coords, n, p, cnt, status, nonempty);
    note_launch();
    return cudaGetLastError();
  });
}

cudaError_t launch_y_scatter(const int32_t* coords, const double* vals, int64_t n, const KeyPlan& p,
                             uint32_t* cursor, void* yfk, bool key32, double* yv, int sms, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const unsigned g = grid_for((n + kRows - 1) / kRows, sms);
  return dispatch_order(p.order, vec_ok(coords, p.order), [&]<int O, bool V>() {
    if (key32)
      y_scatter_kernel<O, V, uint32_t>
          <<<g, kThreads, 0, s>>>(coords, vals, n, p, cursor, static_cast<uint32_t*>(yfk), yv);
    else
      y_scatter_kernel<O, V, u64><<<g, kThreads, 0, s>>>(coords, vals, n, p, cursor, static_cast<u64*>(yfk), yv);
    note_launch();
    return cudaGetLastError();
  });
}

cudaError_t launch_x_survey(const int32_t* coords, const double* vals, int64_t n, const KeyPlan& p,
                            const uint32_t* yoff, u64 K, Survivors sv, u64* P, uint32_t* gcnt, uint32_t* status,
                            uint32_t* nonempty, int sms, cudaStream_t s, bool nonempty_built) {
  if (n <= 0) return cudaSuccess;
  const unsigned g = grid_for((n + kRows - 1) / kRows, sms);
  const bool groups = gcnt != nullptr;
  const uint32_t ne_words = (nonempty && K <= kNonemptyMaxKeys) ? (uint32_t)((K + 31) / 32) : 0u;
  if (ne_words && !nonempty_built) {
    const unsigned gw = (unsigned)std::min<u64>((ne_words + kThreads - 1) / kThreads, (u64)sms * 8);
    nonempty_kernel<<<gw, kThreads, 0, s>>>(yoff, K, p.nseg, nonempty);
    note_launch();
  }
  const size_t smem = (size_t)ne_words * 4;
  if (ne_words && p.order >= 1 && aligned16(coords)) {
    // Coordinates streamed through shared memory by bulk copies, one persistent CTA per SM.
    return dispatch_order(p.order, false, [&]<int O, bool V>() {
      if constexpr (O == 0) {
        return cudaErrorInvalidValue;
      } else {
        // 32-bit contract keys when every contract stride and key fits (K <= 2^18 here).
        const bool k32 = K <= 0xffffffffull;
        auto kern = groups ? (k32 ? x_survey_bulk_kernel<O, true, true> : x_survey_bulk_kernel<O, true, false>)
                           : (k32 ? x_survey_bulk_kernel<O, false, true> : x_survey_bulk_kernel<O, false, false>);
        const size_t bytes = sv_ring_bytes<O>() + smem;
        // The limit is a property of the kernel, shared by every thread that launches it, so it
        // is set to the largest size any launch uses (the bitmap of kNonemptyMaxKeys keys), not
        // to this launch's: threads of a server launching with different key spaces at once
        // would otherwise lower it under one another's launches.
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(sv_ring_bytes<O>() + kNonemptyMaxKeys / 8));
        if (e != cudaSuccess) return e;
        const int64_t nchunks = n / sv_rows<O>();
        const unsigned gb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(sms, nchunks));
        kern<<<gb, kSvThreads, bytes, s>>>(coords, vals, n, p, yoff, sv, P, gcnt, status, nonempty, ne_words);
        note_launch();
        return cudaGetLastError();
      }
    });
  }
  return dispatch_order(p.order, vec_ok(coords, p.order), [&]<int O, bool V>() {
    auto kern = groups ? x_survey_kernel<O, V, true> : x_survey_kernel<O, V, false>;
    if (smem) {  // the largest size any launch uses, as above
      const cudaError_t e =
          cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kNonemptyMaxKeys / 8));
      if (e != cudaSuccess) return e;
    }
    kern<<<g, kThreads, smem, s>>>(coords, vals, n, p, yoff, sv, P, gcnt, status, nonempty, ne_words);
    note_launch();
    return cudaGetLastError();
  });
}

cudaError_t launch_x_count(const int32_t* coords, int64_t n, const KeyPlan& p, const uint32_t* yoff, u64* P,
                           uint32_t* gcnt, uint32_t* status, int sms, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const unsigned g = grid_for((n + kRows - 1) / kRows, sms);
  return dispatch_order(p.order, vec_ok(coords, p.order), [&]<int O, bool V>() {
    x_count_kernel<O, V><<<g, kThreads, 0, s>>>(coords, n, p, yoff, P, gcnt, status);
    note_launch();
    return cudaGetLastError();
  });
}

cudaError_t launch_x_scatter_dense(const int32_t* coords, const double* vals, int64_t n, const KeyPlan& p,
                                   const uint32_t* yoff, uint32_t* gcur, GroupedX gx, uint32_t* status, int sms,
                                   cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const unsigned g = grid_for((n + kRows - 1) / kRows, sms);
  return dispatch_order(p.order, vec_ok(coords, p.order), [&]<int O, bool V>() {
    x_scatter_dense_kernel<O, V><<<g, kThreads, 0, s>>>(coords, vals, n, p, yoff, gcur, gx, status);
    note_launch();
    return cudaGetLastError();
  });
}

cudaError_t launch_keyed_split(const u64* keys, int64_t n, const KeySplit& ks, int32_t* out, uint32_t* status,
                               int sms, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  keyed_split_kernel<<<grid_for(n, sms), kThreads, 0, s>>>(keys, n, ks, out, status);
  note_launch();
  return cudaGetLastError();
}

}  // namespace stc
