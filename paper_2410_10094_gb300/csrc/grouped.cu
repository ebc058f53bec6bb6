// Per-X-free-group accumulation (Sections 4.1, 4.3): X entries that share a free key form
// one group; its outputs can never collide with another group's (Section 2.4.2), so each
// group gets its own probing table, sized from the group's exact bound
// B_g = sum over its entries of count_Y[contract key], capped by the Y free key space.
//
// Device layout: survivors are scattered into group order (counting sort over the X free
// key, Section 4.1.1), groups are binned by table size class, and each class runs one
// persistent kernel whose CTAs take one group at a time with the table in shared memory.
// Groups too large for shared memory use a table region in global memory.
#include "launch.h"

namespace stc {

namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(int64_t n, int sms, int per_sm = 8) {
  const int64_t want = (n + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)sms * per_sm;
  return (unsigned)(want < 1 ? 1 : (want < cap ? want : cap));
}

template <typename KT>
__device__ __forceinline__ KT empty_key();
template <>
__device__ __forceinline__ uint32_t empty_key<uint32_t>() { return kEmpty32; }
template <>
__device__ __forceinline__ u64 empty_key<u64>() { return kEmpty64; }

__device__ __forceinline__ uint32_t slot_hash(uint32_t k) { return mix32(k); }
__device__ __forceinline__ uint32_t slot_hash(u64 k) { return (uint32_t)mix64(k); }

// ---------------------------------------------------------------- grouping of X

__global__ void __launch_bounds__(kThreads) x_group_scatter_kernel(Survivors sv, uint32_t* __restrict__ gcur,
                                                                   GroupedX gx) {
  const int64_t ns = (int64_t)*sv.count;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < ns; i += (int64_t)gridDim.x * kThreads) {
    const uint32_t pos = atomicAdd(gcur + sv.fk[i], 1u);
    if (gx.ck) gx.ck[pos] = sv.ck[i];
    gx.ystart[pos] = sv.ystart[i];
    gx.w[pos] = sv.w[i];
    gx.v[pos] = sv.v[i];
  }
}

// One warp per X free key g: the group's bound B_g (Section 4.3) is the sum of its entries'
// run lengths, read from the grouped X. Non-empty groups go to the first class whose table
// holds t = min(B_g, F_Y); larger ones get a region of the overflow table.
__global__ void __launch_bounds__(kThreads) bin_groups_kernel(u64 FX, const uint32_t* __restrict__ goff,
                                                              const uint32_t* __restrict__ gw, u64 FY, Bins b) {
  __shared__ u64 s_cap[kThreads / 32];
  const unsigned lane = lane_id();
  u64 my_cap = 0;
  for (u64 g = (u64)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5); g < FX;
       g += (u64)gridDim.x * (kThreads / 32)) {
    const uint32_t x0 = goff[g], x1 = goff[g + 1];
    if (x0 == x1) continue;
    u64 bnd = 0;
    for (uint32_t i = x0 + lane; i < x1; i += 32) bnd += gw[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bnd += __shfl_xor_sync(0xffffffffu, bnd, o);
    if (lane == 0) {
      const u64 t = bnd < FY ? bnd : FY;
      int c = 0;
      while (c < b.nclasses && t > b.tmax[c]) c++;
      if (b.dense_list[0] && t >= b.dense_min) {
        // Streamed groups reserve one output position per product (their repeats' records).
        const int d = (bnd <= b.stream_cap && 2 * bnd <= FY) ? 0 : (bnd <= b.stash_cap ? 2 : 1);
        my_cap += d == 0 ? bnd : t;
        const uint32_t idx = atomicAdd(b.count + kMaxClasses + 1 + d, 1u);
        b.dense_list[d][idx] = (uint32_t)g;
      } else if (c < b.nclasses) {
        my_cap += t;
        const uint32_t idx = atomicAdd(b.count + c, 1u);
        b.list[c][idx] = (uint32_t)g;
      } else if (t > (1ull << 30)) {
        atomicOr(b.status, kStatTooLarge);
      } else {
        my_cap += t;
        const uint32_t idx = atomicAdd(b.count + kMaxClasses, 1u);
        u64 cap = 64;
        while (cap < 2 * t) cap <<= 1;
        b.huge_list[idx] = (uint32_t)g;
        b.huge_off[idx] = atomicAdd(b.huge_slots, cap);
        b.huge_cap[idx] = cap;
      }
    }
  }
  if (lane == 0) s_cap[threadIdx.x >> 5] = my_cap;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 t = 0;
    for (int w = 0; w < kThreads / 32; w++) t += s_cap[w];
    if (t) atomicAdd(b.out_cap, t);
  }
}

// ---------------------------------------------------------------- accumulation

// Resolves group g's output target and reserves n output positions (thread 0 only). The
// problem's descriptor is read from global memory word by word.
__device__ __forceinline__ void resolve_target(const GroupArgs& a, u64 g, unsigned n, OutTarget& t) {
  const uint32_t p = a.gprob ? a.gprob[g] : 0u;
  const BatchOut* bo = a.bout + p;
  const u64 FY = bo->FY;
  t.FY = FY;
  t.zrow = (a.gfk ? a.gfk[g] : g) * FY;
  t.counter = a.bnz + p;
  t.base = n ? atomicAdd(a.bnz + p, (u64)n) : 0;
  t.cap = bo->out_cap;
  t.coords = bo->coords;
  t.vals = bo->vals;
  const u64* src = reinterpret_cast<const u64*>(&bo->op);
  u64* dst = reinterpret_cast<u64*>(&t.op);
#pragma unroll 1
  for (unsigned i = 0; i < sizeof(OutPlan) / sizeof(u64); i++) dst[i] = src[i];
}

// resolve_target by the 32 lanes of one warp (every lane calls it): the output plan is copied a
// word per lane rather than word by word, and only when the group's problem differs from the
// previous group's (a single contraction copies it once), so a group's set-up costs at most one
// round of loads. t.prob must hold kNoProb before the warp's first call.
__device__ __forceinline__ void resolve_target_warp(const GroupArgs& a, u64 g, unsigned n, OutTarget& t) {
  const unsigned lane = lane_id();
  uint32_t p = 0;
  if (lane == 0 && a.gprob) p = a.gprob[g];
  p = __shfl_sync(0xffffffffu, p, 0);
  const bool fresh = t.prob != p;
  __syncwarp();  // every lane has read t.prob before lane 0 rewrites it
  const BatchOut* bo = a.bout + p;
  if (fresh) {
    const u64* src = reinterpret_cast<const u64*>(&bo->op);
    u64* dst = reinterpret_cast<u64*>(&t.op);
    constexpr unsigned kWords = sizeof(OutPlan) / sizeof(u64);
    for (unsigned i = lane; i < kWords; i += 32) dst[i] = src[i];
  }
  if (lane == 0) {
    t.prob = p;
    const u64 FY = bo->FY;
    t.FY = FY;
    t.zrow = (a.gfk ? a.gfk[g] : g) * FY;
    t.counter = a.bnz + p;
    t.base = n ? atomicAdd(a.bnz + p, (u64)n) : 0;
    t.cap = bo->out_cap;
    t.coords = bo->coords;
    t.vals = bo->vals;
  }
  __syncwarp();
}

// Shared-memory staging of one chunk of a group's X entries: the exclusive prefix of their
// run lengths (products), the first slot of each run, and the X values.
template <int THREADS>
struct Chunk {
  u64 pre[THREADS + 1];
  uint32_t ystart[THREADS];
  double v[THREADS];
};

// Exclusive block scan of one u64 per thread into pre[0..THREADS], pre[THREADS] = total.
template <int THREADS>
__device__ __forceinline__ void block_scan(u64* pre, u64 w, u64* warp_tot) {
  constexpr int NW = THREADS / 32;
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  u64 x = w;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u64 y = __shfl_up_sync(0xffffffffu, x, o);
    if ((int)lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 run = 0;
    for (int k = 0; k < NW; k++) {
      const u64 t = warp_tot[k];
      warp_tot[k] = run;
      run += t;
    }
    pre[THREADS] = run;
  }
  __syncthreads();
  pre[threadIdx.x] = warp_tot[warp] + x - w;
}

template <int THREADS>
__device__ __forceinline__ void chunk_scan(Chunk<THREADS>& c, u64 w, u64* warp_tot) {
  block_scan<THREADS>(c.pre, w, warp_tot);
}

// Loads the chunk of X entries [c0, c0 + n) of a group and scans their run lengths.
template <int THREADS>
__device__ __forceinline__ void load_chunk(const GroupArgs& a, Chunk<THREADS>& c, u64* warp_tot, uint32_t c0,
                                           uint32_t n) {
  u64 w = 0;
  if (threadIdx.x < n) {
    const uint32_t xi = c0 + threadIdx.x;
    w = a.gx.w[xi];
    c.ystart[threadIdx.x] = a.gx.ystart[xi];
    c.v[threadIdx.x] = a.gx.v[xi];
  }
  chunk_scan<THREADS>(c, w, warp_tot);
  __syncthreads();
}

template <typename YK>
__device__ __forceinline__ u64 y_key(const void* yfk, u64 j) {
  return (u64)__ldg(static_cast<const YK*>(yfk) + j);
}

// ---- shared-memory tables: buckets of 16 bytes (4 32-bit keys or 2 64-bit keys) probed
// with one vector load; the first empty slot of the first bucket without the key is
// claimed with a compare-and-swap (linear probing over buckets, Section 2.3.1).

template <typename KT>
struct Bucket;
template <>
struct Bucket<uint32_t> {
  static constexpr int N = 4;
  uint32_t k[4];
};
template <>
struct Bucket<u64> {
  static constexpr int N = 2;
  u64 k[2];
};

// A fresh 16-byte read of bucket b (volatile: other threads claim slots concurrently).
template <typename KT>
__device__ __forceinline__ Bucket<KT> load_bucket(const KT* keys, uint32_t b) {
  Bucket<KT> out;
  const unsigned addr = (unsigned)__cvta_generic_to_shared(keys + (16 / sizeof(KT)) * b);
  if constexpr (sizeof(KT) == 4) {
    asm volatile("ld.volatile.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(out.k[0]), "=r"(out.k[1]), "=r"(out.k[2]), "=r"(out.k[3])
                 : "r"(addr)
                 : "memory");
  } else {
    asm volatile("ld.volatile.shared.v2.u64 {%0, %1}, [%2];" : "=l"(out.k[0]), "=l"(out.k[1]) : "r"(addr) : "memory");
  }
  return out;
}

// Returns the slot holding `key` after inserting it if absent, or -1 if the table is full.
// *claimed tells whether this call took a new slot.
template <typename KT, int SLOTS>
__device__ __forceinline__ int bucket_claim(KT* keys, KT key, bool* claimed) {
  constexpr int B = Bucket<KT>::N;
  constexpr uint32_t NB = SLOTS / B;
  uint32_t b = slot_hash(key) & (NB - 1);
  *claimed = false;
  for (uint32_t probe = 0; probe < NB;) {
    const Bucket<KT> bk = load_bucket<KT>(keys, b);
    int empty = -1;
#pragma unroll
    for (int i = B - 1; i >= 0; i--) {
      if (bk.k[i] == key) return (int)(b * B + i);
      if (bk.k[i] == empty_key<KT>()) empty = i;
    }
    if (empty < 0) {
      b = (b + 1) & (NB - 1);
      probe++;
      continue;
    }
    const KT prev = atomicCAS(keys + b * B + empty, empty_key<KT>(), key);
    if (prev == empty_key<KT>()) {
      *claimed = true;
      return (int)(b * B + empty);
    }
    if (prev == key) return (int)(b * B + empty);
    // Another key took that slot: look at the same bucket again.
  }
  return -1;
}

// One group: every product of its X entries goes into the shared-memory table. The chunk's
// product range is split evenly over the warps; a warp walks its share 32 products at a
// time (consecutive lanes read consecutive slots of a Y run), advancing the owning X entry
// with the chunk prefix instead of searching for it. The Y reads of D such steps are issued
// before any of their inserts.
//
// Values are settled without floating-point atomics in the common case: the product whose
// compare-and-swap claims a slot stores its value there; products that find their key already
// present keep their value and add it atomically after the round's barrier, when every
// claiming store is visible. Rounds are counted the same way in every warp so that the
// barrier is reached by all threads.
template <int SLOTS, int THREADS, typename KT, int D>
__device__ __forceinline__ void expand_group_smem(const GroupArgs& a, Chunk<THREADS>& c, u64* warp_tot,
                                                  uint32_t x0, uint32_t x1, KT* keys, double* vals,
                                                  unsigned* claims) {
  constexpr int NW = THREADS / 32;
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  for (uint32_t c0 = x0; c0 < x1; c0 += THREADS) {
    const uint32_t n = (x1 - c0 < (uint32_t)THREADS) ? x1 - c0 : (uint32_t)THREADS;
    load_chunk<THREADS>(a, c, warp_tot, c0, n);
    const u64 total = c.pre[n];
    const u64 lo = total * warp / NW, hi = total * (warp + 1) / NW;
    // Owner of product lo: the largest k with pre[k] <= lo.
    uint32_t own = 0;
    if (lo < hi) {
      uint32_t l = 0, h = n - 1;
      while (l < h) {
        const uint32_t mid = (l + h + 1) >> 1;
        if (c.pre[mid] <= lo) l = mid; else h = mid - 1;
      }
      own = l;
    }
    const u64 per = (total + NW - 1) / NW;
    const uint32_t rounds = (uint32_t)((per + 32 * D - 1) / (32 * D));
    const uint64_t keep = policy_evict_last();
    unsigned my_claims = 0;
    for (uint32_t r = 0; r < rounds; r++) {
      const u64 base = lo + (u64)r * 32 * D;
      KT key[D];
      double prod[D];
#pragma unroll
      for (int u = 0; u < D; u++) {
        const u64 p = base + (u64)u * 32 + lane;
        uint32_t k = own;
        key[u] = empty_key<KT>();
        if (p < hi) {
          while (c.pre[k + 1] <= p) k++;
          const u64 j = (u64)c.ystart[k] + (p - c.pre[k]);
          if constexpr (sizeof(KT) == 4)
            key[u] = (KT)ld_keep_u32(static_cast<const uint32_t*>(a.yfk) + j, keep);
          else
            key[u] = (KT)ld_keep_u64(static_cast<const uint64_t*>(a.yfk) + j, keep);
          prod[u] = __dmul_rn(c.v[k], ld_keep_f64(a.yv + j, keep));
        }
        own = __shfl_sync(0xffffffffu, k, 31);
      }
      int later[D];
#pragma unroll
      for (int u = 0; u < D; u++) {
        later[u] = -1;
        bool claimed = false;
        if (key[u] != empty_key<KT>()) {
          const int slot = bucket_claim<KT, SLOTS>(keys, key[u], &claimed);
          if (slot < 0) atomicOr(a.status, kStatTableFull);
          else if (claimed) vals[slot] = prod[u];
          else later[u] = slot;
        }
        my_claims += __popc(__ballot_sync(0xffffffffu, claimed));
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < D; u++)
        if (later[u] >= 0) atomicAdd(vals + later[u], prod[u]);
    }
    if (lane == 0 && my_claims) atomicAdd(claims, my_claims);
    __syncthreads();
  }
}

// Writes the occupied slots as COO output and empties them. One atomic reserves the group's
// output range; inside it, a warp takes 32 buckets at a time, reserves room for their occupied
// slots from a shared-memory cursor, and writes them so that the k-th entry of the warp is
// stored by lane k % 32 (consecutive lanes, consecutive positions: coalesced streaming stores).
template <int SLOTS, int THREADS, typename KT>
__device__ __forceinline__ void write_group_smem(const GroupArgs& a, u64 g, KT* keys, const double* vals,
                                                 unsigned* claims, unsigned* cursor, OutTarget& tg) {
  constexpr int B = Bucket<KT>::N;
  constexpr uint32_t NB = SLOTS / B;
  const unsigned lane = lane_id();
  if (threadIdx.x == 0) {
    resolve_target(a, g, *claims, tg);
    *cursor = 0;
  }
  __syncthreads();
  const u64 base = tg.base;
  const u64 zrow = tg.zrow;
  const uint64_t pol = policy_evict_first();
  for (uint32_t b0 = (threadIdx.x & ~31u); b0 < NB; b0 += THREADS) {
    const uint32_t b = b0 + lane;
    unsigned live = 0;
    if (b < NB) {
      const Bucket<KT> bk = load_bucket<KT>(keys, b);
#pragma unroll
      for (int i = 0; i < B; i++) live |= (bk.k[i] != empty_key<KT>()) ? (1u << i) : 0u;
    }
    const unsigned cnt = __popc(live);
    unsigned incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
      if ((int)lane >= o) incl += y;
    }
    const unsigned tot = __shfl_sync(0xffffffffu, incl, 31);
    if (tot == 0) continue;
    unsigned off = 0;
    if (lane == 0) off = atomicAdd(cursor, tot);
    off = __shfl_sync(0xffffffffu, off, 0);
    for (unsigned k0 = 0; k0 < tot; k0 += 32) {
      const unsigned k = k0 + lane;
      // Source lane: the first lane whose inclusive prefix exceeds k.
      unsigned src = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const unsigned probe = __shfl_sync(0xffffffffu, incl, src + step - 1);
        if (probe <= k) src += step;
      }
      const unsigned src_incl = __shfl_sync(0xffffffffu, incl, src);
      const unsigned src_live = __shfl_sync(0xffffffffu, live, src);
      const unsigned src_cnt = __popc(src_live);
      if (k < tot) {
        // Rank of this entry among the source bucket's occupied slots, then that slot.
        unsigned m = src_live;
        for (unsigned t = k - (src_incl - src_cnt); t > 0; t--) m &= m - 1;
        const uint32_t slot = (b0 + src) * B + (uint32_t)(__ffs(m) - 1);
        const u64 pos = base + off + k;
        if (pos < tg.cap)
          store_output(tg.coords, tg.vals, pos, zrow + (u64)keys[slot], vals[slot], tg.op, pol);
        else
          atomicOr(a.status, kStatOutOverflow);
      }
    }
    __syncwarp();
    if (live) {
      KT* kb = keys + b * B;
#pragma unroll
      for (int i = 0; i < B; i++) kb[i] = empty_key<KT>();
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *claims = 0;
}

// Persistent: CTA b takes groups b, b + grid, ... of its class list. The table is cleared
// once; write_group_smem empties it again after each group.
template <int SLOTS, int THREADS, typename KT>
__global__ void __launch_bounds__(THREADS) group_smem_kernel(GroupArgs a, const uint32_t* __restrict__ list,
                                                             const uint32_t* __restrict__ countp) {
  const uint32_t count = *countp;
  extern __shared__ __align__(16) unsigned char smem[];
  double* vals = reinterpret_cast<double*>(smem);
  KT* keys = reinterpret_cast<KT*>(vals + SLOTS);
  Chunk<THREADS>& c = *reinterpret_cast<Chunk<THREADS>*>(smem + SLOTS * (sizeof(double) + sizeof(KT)));
  __shared__ u64 warp_tot[THREADS / 32];
  __shared__ unsigned claims, cursor;
  __shared__ OutTarget tg;
  for (int i = threadIdx.x; i < SLOTS; i += THREADS) keys[i] = empty_key<KT>();
  if (threadIdx.x == 0) claims = 0;
  __syncthreads();
  for (uint32_t k = blockIdx.x; k < count; k += gridDim.x) {
    const uint32_t g = list[k];
    expand_group_smem<SLOTS, THREADS, KT, sizeof(KT) == 4 ? 8 : 4>(a, c, warp_tot, a.goff[g], a.goff[g + 1], keys,
                                                                   vals, &claims);
    write_group_smem<SLOTS, THREADS, KT>(a, g, keys, vals, &claims, &cursor, tg);
  }
}

// ---- overflow groups: a table region in global memory, scalar linear probing.

template <typename KT>
__device__ __forceinline__ bool probe_add(KT* keys, double* vals, uint32_t mask, KT key, double v) {
  uint32_t h = slot_hash(key) & mask;
  for (uint32_t probe = 0; probe <= mask; probe++) {
    KT cur = *reinterpret_cast<volatile KT*>(keys + h);
    if (cur == empty_key<KT>()) {
      const KT prev = atomicCAS(keys + h, empty_key<KT>(), key);
      cur = (prev == empty_key<KT>()) ? key : prev;
    }
    if (cur == key) {
      atomicAdd(vals + h, v);
      return true;
    }
    h = (h + 1) & mask;
  }
  return false;
}

template <int THREADS, typename YK>
__device__ __forceinline__ void expand_group_global(const GroupArgs& a, Chunk<THREADS>& c, u64* warp_tot,
                                                    uint32_t x0, uint32_t x1, u64* keys, double* vals,
                                                    uint32_t mask) {
  for (uint32_t c0 = x0; c0 < x1; c0 += THREADS) {
    const uint32_t n = (x1 - c0 < (uint32_t)THREADS) ? x1 - c0 : (uint32_t)THREADS;
    load_chunk<THREADS>(a, c, warp_tot, c0, n);
    const u64 total = c.pre[n];
    for (u64 p = threadIdx.x; p < total; p += THREADS) {
      uint32_t lo = 0, hi = n - 1;
      while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (c.pre[mid] <= p) lo = mid; else hi = mid - 1;
      }
      const u64 j = (u64)c.ystart[lo] + (p - c.pre[lo]);
      const u64 key = y_key<YK>(a.yfk, j);
      const double prod = __dmul_rn(c.v[lo], __ldg(a.yv + j));
      if (!probe_add<u64>(keys, vals, mask, key, prod)) atomicOr(a.status, kStatTableFull);
    }
    __syncthreads();
  }
}

template <int THREADS>
__device__ __forceinline__ void write_group_global(const GroupArgs& a, u64 g, const u64* keys,
                                                   const double* vals, uint32_t slots, uint32_t* warp_cnt,
                                                   u64* warp_base, OutTarget& tg) {
  constexpr int NW = THREADS / 32;
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  const uint32_t per = (slots + NW - 1) / NW;
  const uint32_t s0 = warp * per;
  const uint32_t s1 = (s0 + per < slots) ? s0 + per : slots;
  uint32_t cnt = 0;
  for (uint32_t i = s0 + lane; i < s1; i += 32) cnt += keys[i] != kEmpty64;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  if (lane == 0) warp_cnt[warp] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 tot = 0;
    for (int k = 0; k < NW; k++) tot += warp_cnt[k];
    resolve_target(a, g, (unsigned)tot, tg);
    u64 base = tg.base;
    for (int k = 0; k < NW; k++) {
      warp_base[k] = base;
      base += warp_cnt[k];
    }
  }
  __syncthreads();
  u64 run = warp_base[warp];
  const u64 zrow = tg.zrow;
  for (uint32_t i0 = s0; i0 < s1; i0 += 32) {
    const uint32_t i = i0 + lane;
    const u64 k = (i < s1) ? keys[i] : kEmpty64;
    const bool live = k != kEmpty64;
    const unsigned m = __ballot_sync(0xffffffffu, live);
    if (live) {
      const u64 pos = run + __popc(m & lanemask_lt());
      if (pos < tg.cap) {
        store_coords(zrow + k, tg.op, tg.coords + pos * (u64)tg.op.order);
        tg.vals[pos] = vals[i];
      } else {
        atomicOr(a.status, kStatOutOverflow);
      }
    }
    run += __popc(m);
  }
  __syncthreads();
}

// One CTA per overflow group; the table is that group's region of a global array (the host
// clears it before the launch).
template <int THREADS, typename YK>
__global__ void __launch_bounds__(THREADS) group_global_kernel(GroupArgs a, HugeGroups h) {
  __shared__ Chunk<THREADS> c;
  __shared__ u64 warp_tot[THREADS / 32];
  __shared__ uint32_t warp_cnt[THREADS / 32];
  __shared__ u64 warp_base[THREADS / 32];
  __shared__ OutTarget tg;
  const uint32_t count = *h.countp;
  for (uint32_t k = blockIdx.x; k < count; k += gridDim.x) {
    const uint32_t g = h.list[k];
    u64* keys = h.keys + h.off[k];
    double* vals = h.vals + h.off[k];
    const uint32_t cap = (uint32_t)h.cap[k];
    expand_group_global<THREADS, YK>(a, c, warp_tot, a.goff[g], a.goff[g + 1], keys, vals, cap - 1);
    write_group_global<THREADS>(a, g, keys, vals, cap, warp_cnt, warp_base, tg);
  }
}


// ---- bitmap rows: each group is swept one free-key segment at a time. Pass 1 sets, for
// every product, the bit of its free key in a bitmap over the segment. An exclusive scan of
// the words' population counts then ranks the keys present: the group's n outputs of the
// segment take n consecutive output positions in ascending free-key order, reserved with one
// atomic. Pass 2 forms the products again, finds each one's rank from its bitmap word and
// the word's prefix, and accumulates it into a compact value array indexed by rank, which is
// then written out with coalesced stores. No hashing or probing.
//
// Products are enumerated in slots of 32 consecutive Y entries of one X entry's run (one per
// lane, coalesced). In the common case (a group that fits one chunk, with at most kSlotCap
// slots per segment) the slots are listed in a table, and pass 1 also records, per slot, the
// lanes whose key had already been marked (repeats): pass 2 then stores every first product
// of a key without atomics and queues the repeats, which are added after one barrier.
// Otherwise (long groups, many repeats or more keys than the value array) the first product
// of a key is settled with a second bitmap in pass 2, repeats add after a per-round barrier,
// and pass 2 is run once per window of ranks that fits the value array.

constexpr uint32_t kSlotCap = 512;  // slot-table entries
constexpr uint32_t kRepCap = 512;   // queued repeats

template <int THREADS>
struct BitmapStage {
  uint32_t ys[THREADS];          // first Y slot of each entry's run in the current segment
  uint32_t len[THREADS];         // run length
  uint32_t ck[THREADS];          // contract key
  uint32_t sstart[THREADS + 4];  // exclusive prefix of the entries' slot counts
  double v[THREADS];             // X value
};

// Dynamic shared memory of the bitmap kernel, laid out for the widest segment (kDenseSeg
// free keys, kBitmapWords words), in order: the words {bits, rank of the word's first key};
// a region used either as the first-product bitmap or as the repeat masks and queue; the
// slot table; kBitmapVcap values and as many 16-bit keys; the stage.
constexpr uint32_t kBitmapWords = kDenseSeg / 32;
constexpr size_t kBitmapUnion = (size_t)kBitmapWords * 4 > (size_t)kSlotCap * 4 + (size_t)kRepCap * 12
                                    ? (size_t)kBitmapWords * 4
                                    : (size_t)kSlotCap * 4 + (size_t)kRepCap * 12;
constexpr size_t kBitmapFixed = (size_t)kBitmapWords * 8 + kBitmapUnion + (size_t)kSlotCap * 8;
template <int THREADS>
__host__ __device__ constexpr uint32_t bitmap_vcap() {
  return (uint32_t)((kBitmapSmemPerCta - kBitmapFixed - sizeof(BitmapStage<THREADS>)) / 10) & ~7u;
}
template <int THREADS>
__host__ __device__ constexpr size_t bitmap_smem() {
  return kBitmapFixed + (size_t)bitmap_vcap<THREADS>() * 10 + sizeof(BitmapStage<THREADS>);
}

// Runs of segment q of the n staged entries and the prefix of their slot counts; returns
// the chunk's slot count. Entries' ck and v must be staged.
template <int THREADS>
__device__ __forceinline__ uint32_t bitmap_runs(BitmapStage<THREADS>& st, u64* warp_tot,
                                                const uint32_t* __restrict__ yoff, uint32_t nseg, uint32_t q,
                                                uint32_t n, bool have_runs, uint32_t pf_ys, uint32_t pf_len) {
  uint32_t slots = 0;
  if (threadIdx.x < n) {
    uint32_t lo = pf_ys, len = pf_len;
    if (!have_runs) {
      const u64 b = (u64)st.ck[threadIdx.x] * nseg + q;
      lo = __ldg(yoff + b);
      len = __ldg(yoff + b + 1) - lo;
    }
    st.ys[threadIdx.x] = lo;
    st.len[threadIdx.x] = len;
    slots = (len + 31) >> 5;
  }
  constexpr int NW = THREADS / 32;
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  uint32_t x = slots;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if ((int)lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (threadIdx.x < 32) {
    const uint32_t t = (int)lane < NW ? (uint32_t)warp_tot[lane] : 0u;
    uint32_t inc = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if ((int)lane >= o) inc += y;
    }
    if ((int)lane < NW) warp_tot[lane] = inc - t;
    if (lane == 31) st.sstart[THREADS] = inc;
  }
  __syncthreads();
  st.sstart[threadIdx.x] = (uint32_t)warp_tot[warp] + x - slots;
  const uint32_t total = st.sstart[THREADS];
  __syncthreads();
  return total;
}

// A warp's walk over its share of the staged slots (chunks without a slot table). All lanes
// hold the same state.
template <int THREADS>
struct SlotWalk {
  uint32_t s, s_end;  // current slot and end of the warp's share
  uint32_t e;         // current entry
  uint32_t t0;        // offset of the current slot in the entry's run
  uint32_t ys, len;   // current entry's run
  __device__ __forceinline__ void seek(const BitmapStage<THREADS>& st, uint32_t n, uint32_t total) {
    constexpr int NW = THREADS / 32;
    const unsigned warp = threadIdx.x >> 5;
    s = (uint32_t)((u64)total * warp / NW);
    s_end = (uint32_t)((u64)total * (warp + 1) / NW);
    e = 0;
    t0 = 0;
    ys = len = 0;
    if (s < s_end) {
      uint32_t l = 0, h = n - 1;  // largest e with sstart[e] <= s
      while (l < h) {
        const uint32_t mid = (l + h + 1) >> 1;
        if (st.sstart[mid] <= s) l = mid; else h = mid - 1;
      }
      e = l;
      t0 = (s - st.sstart[e]) << 5;
      ys = st.ys[e];
      len = st.len[e];
    }
  }
  // The lane's product of the current slot: its Y slot j, and whether it exists. Advances.
  __device__ __forceinline__ bool next(const BitmapStage<THREADS>& st, uint32_t& j, uint32_t& entry) {
    const uint32_t lane = lane_id();
    const bool live = s < s_end;
    const bool ok = live && t0 + lane < len;
    j = ys + t0 + lane;
    entry = e;
    if (live) {
      s++;
      t0 += 32;
      if (t0 >= len && s < s_end) {
        t0 = 0;
        do {
          e++;
          len = st.len[e];
        } while (len == 0);
        ys = st.ys[e];
      }
    }
    return ok;
  }
};

// One product slot as the slot table holds it: the Y slot of lane 0, and the staged entry
// (high 16 bits) with the number of live lanes (low 16 bits).
__device__ __forceinline__ bool slot_lane(uint2 rec, uint32_t lane, uint32_t& j, uint32_t& e) {
  const bool ok = lane < (rec.y & 0xffffu);
  j = rec.x + (ok ? lane : 0u);
  e = rec.y >> 16;
  return ok;
}

template <int THREADS, int U1, int U2>
__global__ void __launch_bounds__(THREADS, 2) group_bitmap_kernel(GroupArgs a, const uint32_t* __restrict__ yoff,
                                                                  uint32_t nseg, uint32_t seg,
                                                                  const uint32_t* __restrict__ list, uint32_t count) {
  constexpr int NW = THREADS / 32;
  constexpr uint32_t vcap = bitmap_vcap<THREADS>();
  constexpr uint32_t uni_words = (uint32_t)(kBitmapUnion / 4);
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t nwords = seg >> 5;
  uint2* const bw = reinterpret_cast<uint2*>(smem);
  unsigned char* const uni = smem + (size_t)kBitmapWords * 8;
  uint32_t* const first = reinterpret_cast<uint32_t*>(uni);             // protocol mode
  uint32_t* const repmask = reinterpret_cast<uint32_t*>(uni);           // table mode: [kSlotCap]
  double* const rep_v = reinterpret_cast<double*>(uni + kSlotCap * 4);  // [kRepCap]
  uint32_t* const rep_r = reinterpret_cast<uint32_t*>(uni + kSlotCap * 4 + kRepCap * 8);  // [kRepCap]
  uint2* const stab = reinterpret_cast<uint2*>(uni + kBitmapUnion);
  double* const zv = reinterpret_cast<double*>(smem + kBitmapFixed);
  uint16_t* const zk = reinterpret_cast<uint16_t*>(smem + kBitmapFixed + (size_t)vcap * 8);
  BitmapStage<THREADS>& st = *reinterpret_cast<BitmapStage<THREADS>*>(smem + kBitmapFixed + (size_t)vcap * 10);
  __shared__ u64 warp_tot[NW];
  __shared__ OutTarget tg;
  __shared__ u64 gbase;
  __shared__ uint32_t s_n, s_reps, s_queued;
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  const uint64_t keep = policy_evict_last();
  const uint64_t pol = policy_evict_first();
  const uint32_t* yfk = static_cast<const uint32_t*>(a.yfk);
  u64 my_base = 0;
  for (uint32_t i = threadIdx.x; i < nwords; i += THREADS) bw[i] = make_uint2(0, 0);
  for (uint32_t i = threadIdx.x; i < uni_words; i += THREADS) first[i] = 0;
  // Prefetched staging of the next group (when it fits one chunk): its X entries' contract
  // keys and values, and with a single segment their runs.
  uint32_t pf_g = 0, pf_x0 = 0, pf_x1 = 0, pf_ck = 0, pf_ys = 0, pf_len = 0;
  double pf_v = 0.0;
  auto prefetch = [&](uint32_t gi) {
    if (gi >= count) return;
    pf_g = list[gi];
    pf_x0 = a.goff[pf_g];
    pf_x1 = a.goff[pf_g + 1];
    if (pf_x1 - pf_x0 <= (uint32_t)THREADS && threadIdx.x < pf_x1 - pf_x0) {
      pf_ck = a.gx.ck[pf_x0 + threadIdx.x];
      pf_v = a.gx.v[pf_x0 + threadIdx.x];
      if (nseg == 1) {
        pf_ys = __ldg(yoff + pf_ck);
        pf_len = __ldg(yoff + pf_ck + 1) - pf_ys;
      }
    }
  };
  prefetch(blockIdx.x);
  if (threadIdx.x < 32) {  // warp 0 resolves the targets: no plan cached yet
    if (threadIdx.x == 0) tg.prob = kNoProb;
    __syncwarp();
  }
  for (uint32_t gi = blockIdx.x; gi < count; gi += gridDim.x) {
    const uint32_t g = pf_g, x0 = pf_x0, x1 = pf_x1;
    const bool one_chunk = x1 - x0 <= (uint32_t)THREADS;
    if ((threadIdx.x >> 5) == 0) resolve_target_warp(a, g, 0, tg);  // warp 0; published by later barriers
    if (one_chunk && threadIdx.x < x1 - x0) {
      st.ck[threadIdx.x] = pf_ck;
      st.v[threadIdx.x] = pf_v;
    }
    const uint32_t r_ys = pf_ys, r_len = pf_len;
    bool fetched = false;
    for (uint32_t q = 0; q < nseg; q++) {
      // ---- pass 1: mark the free keys of the segment's products.
      uint32_t seg_slots = 0;
      bool table = false;
      for (uint32_t c0 = x0; c0 < x1; c0 += THREADS) {
        const uint32_t n = (x1 - c0 < (uint32_t)THREADS) ? x1 - c0 : (uint32_t)THREADS;
        if (!one_chunk) {
          __syncthreads();
          if (threadIdx.x < n) {
            st.ck[threadIdx.x] = a.gx.ck[c0 + threadIdx.x];
            st.v[threadIdx.x] = a.gx.v[c0 + threadIdx.x];
          }
        }
        const uint32_t total =
            bitmap_runs<THREADS>(st, warp_tot, yoff, nseg, q, n, one_chunk && nseg == 1, r_ys, r_len);
        seg_slots += total;
        if (total == 0) continue;
        table = one_chunk && total <= kSlotCap;
        if (table) {
          if (threadIdx.x < n) {
            const uint32_t s0 = st.sstart[threadIdx.x], ys = st.ys[threadIdx.x], len = st.len[threadIdx.x];
            for (uint32_t k = 0; k * 32 < len; k++) {
              const uint32_t live = len - k * 32 < 32 ? len - k * 32 : 32;
              stab[s0 + k] = make_uint2(ys + k * 32, (threadIdx.x << 16) | live);
            }
          }
          if (threadIdx.x == 0) s_reps = 0;
          __syncthreads();
          for (uint32_t sb = warp; sb < total; sb += NW * U1) {
            uint32_t fk[U1];
            bool ok[U1];
#pragma unroll
            for (int u = 0; u < U1; u++) {
              const uint32_t s = sb + u * NW;
              ok[u] = false;
              if (s < total) {
                uint32_t j, e;
                ok[u] = slot_lane(stab[s], lane, j, e);
                fk[u] = ld_keep_u32(yfk + j, keep) & (seg - 1);
              }
            }
#pragma unroll
            for (int u = 0; u < U1; u++) {
              const uint32_t s = sb + u * NW;
              if (s < total) {
                bool rep = false;
                if (ok[u]) {
                  const uint32_t bit = 1u << (fk[u] & 31);
                  rep = (atomicOr(&bw[fk[u] >> 5].x, bit) & bit) != 0;
                }
                const uint32_t m = __ballot_sync(0xffffffffu, rep);
                if (lane == 0) {
                  repmask[s] = m;
                  if (m) atomicAdd(&s_reps, (uint32_t)__popc(m));
                }
              }
            }
          }
        } else {
          SlotWalk<THREADS> sw;
          sw.seek(st, n, total);
          while (__any_sync(0xffffffffu, sw.s < sw.s_end)) {
            uint32_t fk[U1];
            bool ok[U1];
#pragma unroll
            for (int u = 0; u < U1; u++) {
              uint32_t j, e;
              ok[u] = sw.next(st, j, e);
              if (ok[u]) fk[u] = ld_keep_u32(yfk + j, keep) & (seg - 1);
            }
#pragma unroll
            for (int u = 0; u < U1; u++)
              if (ok[u]) atomicOr(&bw[fk[u] >> 5].x, 1u << (fk[u] & 31));
          }
        }
      }
      if (seg_slots == 0) continue;
      __syncthreads();
      // ---- ranks: exclusive scan of the words' population counts (a few consecutive words
      // per thread, then a block scan of the per-thread sums); one atomic reserves the outputs.
      {
        const uint32_t wpt = (nwords + THREADS - 1) / THREADS;
        const uint32_t w0 = threadIdx.x * wpt;
        const uint32_t w1 = w0 + wpt < nwords ? w0 + wpt : nwords;
        uint32_t sum = 0;
        for (uint32_t w = w0; w < w1; w++) sum += __popc(bw[w].x);
        uint32_t x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
          if ((int)lane >= o) x += y;
        }
        if (lane == 31) warp_tot[warp] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
          const uint32_t t = (int)lane < NW ? (uint32_t)warp_tot[lane] : 0u;
          uint32_t inc = t;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if ((int)lane >= o) inc += y;
          }
          if ((int)lane < NW) warp_tot[lane] = inc - t;
          if (lane == 31) {
            s_n = inc;
            s_queued = 0;
            my_base = inc ? atomicAdd(tg.counter, (u64)inc) : 0;  // consumed after pass 2
          }
        }
        __syncthreads();
        uint32_t rank = (uint32_t)warp_tot[warp] + x - sum;
        for (uint32_t w = w0; w < w1; w++) {
          bw[w].y = rank;
          rank += __popc(bw[w].x);
        }
      }
      // The next group's staging loads are issued here and land during pass 2 and the write.
      if (q + 1 == nseg) {
        prefetch(gi + gridDim.x);
        fetched = true;
      }
      __syncthreads();
      const uint32_t nkeys = s_n;
      const u64 zseg = tg.zrow + (u64)q * seg;
      const uint32_t tslots = st.sstart[THREADS];
      const bool queue = table && s_reps <= kRepCap && nkeys <= vcap;
      if (table && !queue) {
        for (uint32_t i = threadIdx.x; i < uni_words; i += THREADS) first[i] = 0;
        __syncthreads();
      }
      for (uint32_t r0 = 0; r0 < nkeys; r0 += vcap) {
        const uint32_t wn = nkeys - r0 < vcap ? nkeys - r0 : vcap;
        // ---- pass 2: accumulate the products whose rank falls in [r0, r0 + wn).
        if (queue) {
          // First products store; repeats are queued and added after the barrier.
          for (uint32_t sb = warp; sb < tslots; sb += NW * U2) {
#pragma unroll
            for (int u = 0; u < U2; u++) {
              const uint32_t s = sb + u * NW;
              if (s < tslots) {
                uint32_t j, e;
                const bool ok = slot_lane(stab[s], lane, j, e);
                const uint32_t rm = repmask[s];
                const uint32_t f = ld_keep_u32(yfk + j, keep) & (seg - 1);
                const double prod = __dmul_rn(st.v[e], ld_keep_f64(a.yv + j, keep));
                const uint2 wd = bw[f >> 5];
                const uint32_t bit = 1u << (f & 31);
                const uint32_t r = wd.y + __popc(wd.x & (bit - 1));
                const bool rep = (rm >> lane) & 1u;
                if (ok && !rep) {
                  zv[r] = prod;
                  zk[r] = (uint16_t)f;
                }
                if (rm) {
                  const uint32_t at = warp_reserve(rep, &s_queued);
                  if (rep) {
                    rep_r[at] = r;
                    rep_v[at] = prod;
                  }
                }
              }
            }
          }
          __syncthreads();
          const uint32_t nq = s_queued;
          for (uint32_t i = threadIdx.x; i < nq; i += THREADS) atomicAdd(zv + rep_r[i], rep_v[i]);
        } else {
          for (uint32_t c0 = x0; c0 < x1; c0 += THREADS) {
            const uint32_t n = (x1 - c0 < (uint32_t)THREADS) ? x1 - c0 : (uint32_t)THREADS;
            uint32_t total = tslots;
            if (!one_chunk) {
              __syncthreads();
              if (threadIdx.x < n) {
                st.ck[threadIdx.x] = a.gx.ck[c0 + threadIdx.x];
                st.v[threadIdx.x] = a.gx.v[c0 + threadIdx.x];
              }
              total = bitmap_runs<THREADS>(st, warp_tot, yoff, nseg, q, n, false, 0, 0);
            }
            if (total == 0) continue;
            // The first product of a key (first to set its bit in `first`) stores; the others
            // add after the round's barrier. Every warp runs the same number of rounds.
            SlotWalk<THREADS> sw;
            if (!table) sw.seek(st, n, total);
            const uint32_t per = (total + NW - 1) / NW;
            const uint32_t rounds = (per + U2 - 1) / U2;
            for (uint32_t rd = 0; rd < rounds; rd++) {
              uint32_t slot[U2];
              double prod[U2];
              bool later[U2];
#pragma unroll
              for (int u = 0; u < U2; u++) {
                uint32_t j = 0, e = 0;
                bool ok = false;
                later[u] = false;
                if (table) {
                  const uint32_t s = warp + NW * (rd * U2 + u);
                  if (s < total) ok = slot_lane(stab[s], lane, j, e);
                } else {
                  ok = sw.next(st, j, e);
                }
                if (ok) {
                  const uint32_t f = ld_keep_u32(yfk + j, keep) & (seg - 1);
                  prod[u] = __dmul_rn(st.v[e], ld_keep_f64(a.yv + j, keep));
                  const uint2 wd = bw[f >> 5];
                  const uint32_t bit = 1u << (f & 31);
                  slot[u] = wd.y + __popc(wd.x & (bit - 1)) - r0;
                  if (slot[u] < wn) {
                    if (atomicOr(first + (f >> 5), bit) & bit) {
                      later[u] = true;
                    } else {
                      zv[slot[u]] = prod[u];
                      zk[slot[u]] = (uint16_t)f;
                    }
                  }
                }
              }
              __syncthreads();
#pragma unroll
              for (int u = 0; u < U2; u++)
                if (later[u]) atomicAdd(zv + slot[u], prod[u]);
            }
          }
        }
        if (threadIdx.x == 31) gbase = my_base;
        __syncthreads();
        // ---- write the window: consecutive threads, consecutive output positions.
        const u64 pbase = gbase + r0;
        const u64 cap = tg.cap;
        int32_t* const coords = tg.coords;
        double* const vals = tg.vals;
        if (tg.op.order == 4 && tg.op.pow2 && ((reinterpret_cast<uintptr_t>(coords) & 15u) == 0)) {
          // Coordinates are below 2^31: 32-bit masks.
          const uint32_t s0 = tg.op.shift[0], s1 = tg.op.shift[1], s2 = tg.op.shift[2], s3 = tg.op.shift[3];
          const uint32_t m0 = (uint32_t)tg.op.mod[0] - 1, m1 = (uint32_t)tg.op.mod[1] - 1,
                         m2 = (uint32_t)tg.op.mod[2] - 1, m3 = (uint32_t)tg.op.mod[3] - 1;
          for (uint32_t i = threadIdx.x; i < wn; i += THREADS) {
            const u64 pos = pbase + i;
            const u64 z = zseg + zk[i];
            if (pos < cap) {
              const int4 cv = make_int4((int32_t)((uint32_t)(z >> s0) & m0), (int32_t)((uint32_t)(z >> s1) & m1),
                                        (int32_t)((uint32_t)(z >> s2) & m2), (int32_t)((uint32_t)(z >> s3) & m3));
              st_stream_v4(coords + pos * 4, cv, pol);
              st_stream_f64(vals + pos, zv[i], pol);
            } else {
              atomicOr(a.status, kStatOutOverflow);
            }
          }
        } else {
          for (uint32_t i = threadIdx.x; i < wn; i += THREADS) {
            const u64 pos = pbase + i;
            if (pos < cap)
              store_output(coords, vals, pos, zseg + zk[i], zv[i], tg.op, pol);
            else
              atomicOr(a.status, kStatOutOverflow);
          }
        }
        if (r0 + vcap < nkeys) __syncthreads();
      }
      for (uint32_t i = threadIdx.x; i < nwords; i += THREADS) bw[i] = make_uint2(0, 0);
      for (uint32_t i = threadIdx.x; i < uni_words; i += THREADS) first[i] = 0;
      __syncthreads();
    }
    if (!fetched) prefetch(gi + gridDim.x);
  }
}


// ---- product stash: groups whose product count fits the stash (the common case of the
// bitmap path). Pass 1 forms every product once (Y key and value read together, one round
// trip) and marks its free key in a bitmap over the segment: the first product of a key is
// the one that finds its bit clear. First products take consecutive places at the front of
// the stash (their order is the group's output order); repeats take places from the back
// and mark their key in a second bitmap. After pass 1 the group's output count is the number
// of first products, reserved with one atomic. First products of keys that never repeat are
// written out at once; repeated keys are ranked by a scan over the second bitmap, their first
// products record their place in a rank-indexed map, every repeat adds its value there, and
// those outputs are written last. Products are enumerated in slots of up to 32 consecutive Y
// entries of one X entry's run (one per lane, coalesced), listed in a slot table.

#ifndef STASH_THREADS
#define STASH_THREADS 512
#endif
#ifndef STASH_U
#define STASH_U 3
#endif
#ifndef STASH_PIPE
#define STASH_PIPE 1
#endif
constexpr bool kStashPipe = STASH_PIPE != 0;
constexpr int kStashThreads = STASH_THREADS;
constexpr uint32_t kStashMaxEntries = kStashThreads;  // X entries staged per chunk
// Shared memory (widest segment, kBitmapWords words), in order: key bitmap, repeat bitmap,
// slot table, X values of the chunk, then per product a value, a key and a map byte pair
// for every two products (repeat rank -> place of the key's first product).
__host__ __device__ constexpr uint32_t stash_slots(uint32_t cap) { return cap / 32 + kStashMaxEntries; }
__host__ __device__ constexpr size_t stash_smem(uint32_t cap) {
  return (size_t)kBitmapWords * 8 + (size_t)stash_slots(cap) * 8 + (size_t)kStashMaxEntries * 8 +
         (size_t)cap * 10 + (size_t)cap;
}
__host__ __device__ constexpr uint32_t stash_cap() {
  uint32_t c = 16384;
  while (stash_smem(c) > kBitmapSmemPerCta - 256) c -= 32;
  return c;
}
constexpr uint32_t kStashCap = stash_cap();  // products of one group segment
constexpr uint32_t kStashSlots = stash_slots(kStashCap);
constexpr size_t kStashSmem = stash_smem(kStashCap);
static_assert(kStashCap >= 4096 && kStashCap < 65536 && kStashCap % 32 == 0, "stash capacity");

// Block-wide exclusive scan of one u32 per thread (THREADS threads); returns the exclusive
// prefix and sets *total. Two barriers; warp_tot must hold THREADS / 32 + 1 entries.
template <int THREADS>
__device__ __forceinline__ uint32_t block_exscan_u32(uint32_t v, uint32_t* total, u64* warp_tot) {
  constexpr int NW = THREADS / 32;
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if ((int)lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (threadIdx.x < 32) {
    const uint32_t t = (int)lane < NW ? (uint32_t)warp_tot[lane] : 0u;
    uint32_t inc = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if ((int)lane >= o) inc += y;
    }
    if ((int)lane < NW) warp_tot[lane] = inc - t;
    if (lane == 31) warp_tot[NW] = inc;
  }
  __syncthreads();
  *total = (uint32_t)warp_tot[NW];
  return (uint32_t)warp_tot[warp] + x - v;
}

template <int U>
__global__ void __launch_bounds__(kStashThreads, 2) group_stash_kernel(GroupArgs a, const uint32_t* __restrict__ yoff,
                                                                      uint32_t nseg, uint32_t seg,
                                                                      const uint32_t* __restrict__ list,
                                                                      uint32_t count) {
  constexpr int T = kStashThreads, NW = T / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t nwords = seg >> 5;
  uint32_t* const bits = reinterpret_cast<uint32_t*>(smem);             // key marks, then repeat ranks
  uint32_t* const rbits = bits + kBitmapWords;                          // keys met again
  uint2* const stab = reinterpret_cast<uint2*>(rbits + kBitmapWords);  // slot table
  double* const sx = reinterpret_cast<double*>(stab + kStashSlots);    // X values of the chunk
  double* const pv = sx + kStashMaxEntries;                             // stashed products
  uint16_t* const pk = reinterpret_cast<uint16_t*>(pv + kStashCap);    // stashed keys
  uint16_t* const map = pk + kStashCap;                                 // repeat rank -> first place
  __shared__ u64 warp_tot[NW + 1];
  __shared__ OutTarget tg;
  __shared__ u64 s_gbase;
  __shared__ uint32_t s_cnt;
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  const uint32_t lt = lanemask_lt();
  const uint64_t keep = policy_evict_last();
  const uint64_t pol = policy_evict_first();
  const uint32_t* yfk = static_cast<const uint32_t*>(a.yfk);
  for (uint32_t i = threadIdx.x; i < 2 * kBitmapWords; i += T) bits[i] = 0;
  if (threadIdx.x == 0) s_cnt = 0;
  // Prefetched staging of the next group (when it fits one chunk): its X entries' contract
  // keys and values, and with a single segment their runs.
  uint32_t pf_g = 0, pf_x0 = 0, pf_x1 = 0, pf_ck = 0, pf_ys = 0, pf_ye = 0;
  double pf_v = 0.0;
  auto prefetch = [&](uint32_t gi) {
    if (gi >= count) return;
    pf_g = list[gi];
    pf_x0 = a.goff[pf_g];
    pf_x1 = a.goff[pf_g + 1];
    if (pf_x1 - pf_x0 <= (uint32_t)T && threadIdx.x < pf_x1 - pf_x0) {
      pf_ck = a.gx.ck[pf_x0 + threadIdx.x];
      pf_v = a.gx.v[pf_x0 + threadIdx.x];
      if (nseg == 1) {
        pf_ys = __ldg(yoff + pf_ck);
        pf_ye = __ldg(yoff + pf_ck + 1);
      }
    }
  };
  prefetch(blockIdx.x);
  if (threadIdx.x < 32) {  // warp 0 resolves the targets: no plan cached yet
    if (threadIdx.x == 0) tg.prob = kNoProb;
    __syncwarp();
  }
  for (uint32_t gi = blockIdx.x; gi < count; gi += gridDim.x) {
    const uint32_t g = pf_g, x0 = pf_x0, x1 = pf_x1;
    const bool one_chunk = x1 - x0 <= (uint32_t)T;
    if ((threadIdx.x >> 5) == 0) resolve_target_warp(a, g, 0, tg);  // warp 0; published by later barriers
    const uint32_t my_ck = pf_ck, my_ys = pf_ys, my_ye = pf_ye;
    const double my_v = pf_v;
    prefetch(gi + gridDim.x);
    for (uint32_t q = 0; q < nseg; q++) {
      // ---- pass 1, one chunk of X entries at a time.
      for (uint32_t c0 = x0; c0 < x1; c0 += T) {
        const uint32_t n = (x1 - c0 < (uint32_t)T) ? x1 - c0 : (uint32_t)T;
        uint32_t ys = 0, len = 0;
        if (threadIdx.x < n) {
          sx[threadIdx.x] = one_chunk ? my_v : a.gx.v[c0 + threadIdx.x];
          if (one_chunk && nseg == 1) {
            ys = my_ys;
            len = my_ye - my_ys;
          } else {
            const uint32_t ck = one_chunk ? my_ck : a.gx.ck[c0 + threadIdx.x];
            const u64 b = (u64)ck * nseg + q;
            ys = __ldg(yoff + b);
            len = __ldg(yoff + b + 1) - ys;
          }
        }
        uint32_t S;
        uint32_t s = block_exscan_u32<T>((len + 31) >> 5, &S, warp_tot);
        if (threadIdx.x < n) {
          for (uint32_t k = 0; k < len; k += 32, s++) {
            const uint32_t live = len - k < 32 ? len - k : 32;
            stab[s] = make_uint2(ys + k, live | (threadIdx.x << 8));
          }
        }
        __syncthreads();
        // Slot batches of U per warp; the next batch's Y loads are issued before the current
        // batch is claimed, so two batches of loads are in flight per warp.
        uint32_t fA[U], eA[U];
        double yA[U];
        bool okA[U], inA[U];
        auto issue = [&](uint32_t sbase, uint32_t (&f)[U], uint32_t (&e)[U], double (&y)[U], bool (&ok)[U],
                         bool (&in)[U]) {
#pragma unroll
          for (int u = 0; u < U; u++) {
            const uint32_t si = sbase + u * NW;
            in[u] = si < S;
            ok[u] = false;
            if (in[u]) {
              const uint2 rec = stab[si];
              ok[u] = lane < (rec.y & 255u);
              const uint32_t j = rec.x + (ok[u] ? lane : 0u);
              e[u] = rec.y >> 8;
              f[u] = ld_keep_u32(yfk + j, keep);
              y[u] = ld_keep_f64(a.yv + j, keep);
            }
          }
        };
        issue(warp, fA, eA, yA, okA, inA);
        for (uint32_t sb = warp; sb < S; sb += NW * U) {
          uint32_t fB[U], eB[U];
          double yB[U];
          bool okB[U], inB[U];
          if (kStashPipe) issue(sb + NW * U, fB, eB, yB, okB, inB);
#pragma unroll
          for (int u = 0; u < U; u++) {
            if (inA[u]) {
              const uint32_t f = fA[u] & (seg - 1);
              const double prod = __dmul_rn(sx[eA[u]], yA[u]);
              const uint32_t w = f >> 5, bit = 1u << (f & 31);
              bool first = false;
              if (okA[u]) {
                first = (atomicOr(bits + w, bit) & bit) == 0;
                if (!first) atomicOr(rbits + w, bit);
              }
              const uint32_t fm = __ballot_sync(0xffffffffu, first);
              const uint32_t rm = __ballot_sync(0xffffffffu, okA[u] && !first);
              // One packed counter: first products in the low half, repeats in the high half.
              uint32_t base = 0;
              if (lane == 0) base = atomicAdd(&s_cnt, (uint32_t)__popc(fm) | ((uint32_t)__popc(rm) << 16));
              base = __shfl_sync(0xffffffffu, base, 0);
              if (okA[u]) {
                const uint32_t at = first ? (base & 0xffffu) + __popc(fm & lt)
                                          : kStashCap - 1 - ((base >> 16) + __popc(rm & lt));
                pk[at] = (uint16_t)f;
                pv[at] = prod;
              }
            }
          }
          if (!kStashPipe) {
            issue(sb + NW * U, fB, eB, yB, okB, inB);
          }
#pragma unroll
          for (int u = 0; u < U; u++) {
            fA[u] = fB[u];
            eA[u] = eB[u];
            yA[u] = yB[u];
            okA[u] = okB[u];
            inA[u] = inB[u];
          }
        }
        if (!one_chunk) __syncthreads();
      }
      __syncthreads();
      const uint32_t nkeys = s_cnt & 0xffffu, reps = s_cnt >> 16;
      if (nkeys == 0) continue;
      // Thread 31 reserves the outputs; the result is published by the barrier before the write.
      u64 my_base = 0;
      if (threadIdx.x == 31) my_base = atomicAdd(tg.counter, (u64)nkeys);
      uint32_t nrep_keys = 0;
      if (reps) {
        // Rank the repeated keys; the key marks are no longer needed and hold the ranks.
        const uint32_t wpt = (nwords + T - 1) / T;
        const uint32_t w0 = threadIdx.x * wpt, w1 = w0 + wpt < nwords ? w0 + wpt : nwords;
        uint32_t sum = 0;
        for (uint32_t w = w0; w < w1; w++) sum += __popc(rbits[w]);
        uint32_t r = block_exscan_u32<T>(sum, &nrep_keys, warp_tot);
        for (uint32_t w = w0; w < w1; w++) {
          bits[w] = r;
          r += __popc(rbits[w]);
        }
      }
      if (threadIdx.x == 31) s_gbase = my_base;
      __syncthreads();
      const u64 gb = s_gbase;
      const u64 zseg = tg.zrow + (u64)q * seg;
      const u64 cap = tg.cap;
      int32_t* const coords = tg.coords;
      double* const vals = tg.vals;
      const bool v4 = tg.op.order == 4 && tg.op.pow2 && ((reinterpret_cast<uintptr_t>(coords) & 15u) == 0);
      const uint32_t s0 = tg.op.shift[0], s1 = tg.op.shift[1], s2 = tg.op.shift[2], s3 = tg.op.shift[3];
      const uint32_t m0 = (uint32_t)tg.op.mod[0] - 1, m1 = (uint32_t)tg.op.mod[1] - 1,
                     m2 = (uint32_t)tg.op.mod[2] - 1, m3 = (uint32_t)tg.op.mod[3] - 1;
      auto write = [&](uint32_t i) {
        const u64 pos = gb + i;
        const u64 z = zseg + pk[i];
        if (pos >= cap) {
          atomicOr(a.status, kStatOutOverflow);
        } else if (v4) {
          // Coordinates are below 2^31: 32-bit masks.
          const int4 cv = make_int4((int32_t)((uint32_t)(z >> s0) & m0), (int32_t)((uint32_t)(z >> s1) & m1),
                                    (int32_t)((uint32_t)(z >> s2) & m2), (int32_t)((uint32_t)(z >> s3) & m3));
          st_stream_v4(coords + pos * 4, cv, pol);
          st_stream_f64(vals + pos, pv[i], pol);
        } else {
          store_output(coords, vals, pos, z, pv[i], tg.op, pol);
        }
      };
      // ---- write the keys met once; record the places of repeated keys' first products.
      for (uint32_t i = threadIdx.x; i < nkeys; i += T) {
        if (reps) {
          const uint32_t f = pk[i], w = f >> 5, bit = 1u << (f & 31), rw = rbits[w];
          if (rw & bit) {
            map[bits[w] + __popc(rw & (bit - 1))] = (uint16_t)i;
            continue;
          }
        }
        write(i);
      }
      if (reps) {
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < reps; k += T) {
          const uint32_t at = kStashCap - 1 - k;
          const uint32_t f = pk[at], w = f >> 5, bit = 1u << (f & 31);
          atomicAdd(pv + map[bits[w] + __popc(rbits[w] & (bit - 1))], pv[at]);
        }
        __syncthreads();
        for (uint32_t r = threadIdx.x; r < nrep_keys; r += T) write(map[r]);
      }
      // ---- clear the bitmaps for the next segment or group.
      for (uint32_t i = threadIdx.x; i < nwords / 4; i += T) {
        reinterpret_cast<uint4*>(bits)[i] = make_uint4(0, 0, 0, 0);
        reinterpret_cast<uint4*>(rbits)[i] = make_uint4(0, 0, 0, 0);
      }
      if (nwords < 4 && threadIdx.x < nwords) bits[threadIdx.x] = rbits[threadIdx.x] = 0;
      if (threadIdx.x == 0) s_cnt = 0;
      __syncthreads();
    }
  }
}


// ---- output streaming: groups whose product count fits kStreamCap (the common case of the
// bitmap path). Each group segment reserves as many output positions as it has products.
// Pass 1 forms every product once and marks its free key in a bitmap over the segment; the
// first product of a key (the one that finds its bit clear) writes its output entry at once,
// at the next place from the front of the reservation. A repeat writes its key and value as
// a temporary record at the next place from the back and marks its key in a second bitmap.
// After a block barrier (which orders the block's own stores before its later reads and
// atomics) the repeated keys are ranked, their first products' places looked up, and every
// repeat adds its value to that entry with an L2 atomic. The back of the reservation (the repeats' records) becomes a hole; after all
// groups, holes below the final output count are filled with the entries above it.

#ifndef STREAM_U
#define STREAM_U 3
#endif
#ifndef STREAM_MINB
#define STREAM_MINB 4
#endif
constexpr int kStreamThreads = 256;
constexpr uint32_t kStreamEntries = 256;  // X entries staged per chunk
constexpr uint32_t kStreamCap = 8192;     // products of one group segment
constexpr uint32_t kStreamSlots = kStreamCap / 32 + kStreamEntries;
// Shared memory: key bitmap, repeat bitmap, slot table, X values, first-product keys, and the
// rank -> place map of the repeated keys.
static_assert(kStreamCap % 4 == 0, "the fix-up reads the first-product keys four at a time");
constexpr size_t kStreamSmem = (size_t)kBitmapWords * 8 + (size_t)kStreamSlots * 8 + (size_t)kStreamEntries * 8 +
                               (size_t)kStreamCap * 2 + (size_t)kStreamCap;

// FIXED: output rows of 2..8 coordinates in concatenation order with some length not a power
// of two, decoded into registers and stored in pairs (store_row_fixed); a separate
// instantiation so that the power-of-two kernel keeps its own code.
template <int U, bool FIXED>
__global__ void __launch_bounds__(kStreamThreads, STREAM_MINB) group_stream_kernel(GroupArgs a, const uint32_t* __restrict__ yoff,
                                                                        uint32_t nseg, uint32_t seg,
                                                                        const uint32_t* __restrict__ list,
                                                                        uint32_t count, StreamArgs sa) {
  constexpr int T = kStreamThreads, NW = T / 32;
  constexpr uint32_t CH = kStreamEntries;
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t nwords = seg >> 5;
  uint32_t* const bits = reinterpret_cast<uint32_t*>(smem);              // key marks, then repeat ranks
  uint32_t* const rbits = bits + kBitmapWords;                           // keys met again
  uint2* const stab = reinterpret_cast<uint2*>(rbits + kBitmapWords);   // slot table
  double* const sx = reinterpret_cast<double*>(stab + kStreamSlots);    // X values of the chunk
  uint16_t* const pk = reinterpret_cast<uint16_t*>(sx + CH);            // keys of the first products
  uint16_t* const map = pk + kStreamCap;                                 // repeat rank -> first place
  __shared__ u64 warp_tot[NW + 1];
  __shared__ OutTarget tg;
  __shared__ u64 s_gbase;
  __shared__ uint32_t s_cnt;
  // Order-4 power-of-two outputs: each coordinate is either constant over the segment or a bit
  // field of the segment-relative free key fy = q * seg + fk; coordinate = cst | (fy >> sh) & mk.
  __shared__ int4 s_cst;
  __shared__ uint4 s_sh, s_mk;
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  const uint32_t lt = lanemask_lt();
  const uint64_t keep = policy_evict_last();
  const uint64_t pol = policy_evict_first();
  const uint32_t* yfk = static_cast<const uint32_t*>(a.yfk);
  for (uint32_t i = threadIdx.x; i < 2 * kBitmapWords; i += T) bits[i] = 0;
  if (threadIdx.x == 0) s_cnt = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) *sa.nrec = count * nseg;  // one record per (group, segment)
  // Prefetched staging of the next group (when it fits one chunk).
  uint32_t pf_g = 0, pf_x0 = 0, pf_x1 = 0, pf_ck = 0, pf_ys = 0, pf_ye = 0;
  double pf_v = 0.0;
  auto prefetch = [&](uint32_t gi) {
    if (gi >= count) return;
    pf_g = list[gi];
    pf_x0 = a.goff[pf_g];
    pf_x1 = a.goff[pf_g + 1];
    if (pf_x1 - pf_x0 <= CH && threadIdx.x < pf_x1 - pf_x0) {
      pf_ck = a.gx.ck[pf_x0 + threadIdx.x];
      pf_v = a.gx.v[pf_x0 + threadIdx.x];
      if (nseg == 1) {
        pf_ys = __ldg(yoff + pf_ck);
        pf_ye = __ldg(yoff + pf_ck + 1);
      }
    }
  };
  prefetch(blockIdx.x);
  if (threadIdx.x < 32) {  // warp 0 resolves the targets: no plan cached yet
    if (threadIdx.x == 0) tg.prob = kNoProb;
    __syncwarp();
  }
  for (uint32_t gi = blockIdx.x; gi < count; gi += gridDim.x) {
    const uint32_t g = pf_g, x0 = pf_x0, x1 = pf_x1;
    const bool one_chunk = x1 - x0 <= CH;
    if ((threadIdx.x >> 5) == 0) resolve_target_warp(a, g, 0, tg);  // warp 0; published by later barriers
    const uint32_t my_ck = pf_ck, my_ys = pf_ys, my_ye = pf_ye;
    const double my_v = pf_v;
    prefetch(gi + gridDim.x);
    for (uint32_t q = 0; q < nseg; q++) {
      if (threadIdx.x == 0 && tg.op.order == 4 && tg.op.pow2) {
        // Published by the staging scan's barriers below.
        const uint32_t b = 63 - __clzll(tg.FY);
        uint32_t c[4], sh[4], mk[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
          const uint32_t sk = tg.op.shift[k], mkk = (uint32_t)tg.op.mod[k] - 1;
          const bool cst = sk >= b;
          c[k] = cst ? (uint32_t)(tg.zrow >> sk) & mkk : 0u;
          sh[k] = cst ? 0u : sk;
          mk[k] = cst ? 0u : mkk;
        }
        s_cst = make_int4((int32_t)c[0], (int32_t)c[1], (int32_t)c[2], (int32_t)c[3]);
        s_sh = make_uint4(sh[0], sh[1], sh[2], sh[3]);
        s_mk = make_uint4(mk[0], mk[1], mk[2], mk[3]);
      }
      // The segment's products, reserved up front (a separate count pass for long groups).
      uint32_t Pq = 0;
      if (!one_chunk) {
        for (uint32_t c0 = x0; c0 < x1; c0 += CH) {
          const uint32_t n = (x1 - c0 < CH) ? x1 - c0 : CH;
          uint32_t len = 0;
          if (threadIdx.x < n) {
            const u64 b = (u64)a.gx.ck[c0 + threadIdx.x] * nseg + q;
            len = __ldg(yoff + b + 1) - __ldg(yoff + b);
          }
          uint32_t tot;
          block_exscan_u32<T>(len, &tot, warp_tot);
          Pq += tot;
        }
        if (Pq == 0) {
          if (threadIdx.x == 0) sa.rec[(u64)gi * nseg + q] = StreamRec{0, 0, 0};
          continue;
        }
        if (threadIdx.x == 0) s_gbase = atomicAdd(tg.counter, (u64)Pq);
      }
      // ---- pass 1, one chunk of X entries at a time.
      for (uint32_t c0 = x0; c0 < x1; c0 += CH) {
        const uint32_t n = (x1 - c0 < CH) ? x1 - c0 : CH;
        uint32_t ys = 0, len = 0;
        if (threadIdx.x < n) {
          sx[threadIdx.x] = one_chunk ? my_v : a.gx.v[c0 + threadIdx.x];
          if (one_chunk && nseg == 1) {
            ys = my_ys;
            len = my_ye - my_ys;
          } else {
            const uint32_t ck = one_chunk ? my_ck : a.gx.ck[c0 + threadIdx.x];
            const u64 b = (u64)ck * nseg + q;
            ys = __ldg(yoff + b);
            len = __ldg(yoff + b + 1) - ys;
          }
        }
        // Products (high bits) and slots (low 12 bits) before each entry, in one scan; a
        // one-chunk group reserves its outputs between the scan's two barriers.
        const uint32_t nslot = (len + 31) >> 5;
        uint32_t x = (len << 12) | nslot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
          if ((int)lane >= o) x += y;
        }
        if (lane == 31) warp_tot[warp] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
          const uint32_t t = (int)lane < NW ? (uint32_t)warp_tot[lane] : 0u;
          uint32_t inc = t;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if ((int)lane >= o) inc += y;
          }
          if ((int)lane < NW) warp_tot[lane] = inc - t;
          if (lane == 31) {
            warp_tot[NW] = inc;
            if (one_chunk && (inc >> 12)) s_gbase = atomicAdd(tg.counter, (u64)(inc >> 12));
          }
        }
        __syncthreads();
        const uint32_t tot = (uint32_t)warp_tot[NW], S = tot & 4095u;
        if (one_chunk) Pq = tot >> 12;
        {
          uint32_t s = ((uint32_t)warp_tot[warp] + x - ((len << 12) | nslot)) & 4095u;
          if (threadIdx.x < n) {
            for (uint32_t k = 0; k < len; k += 32, s++) {
              const uint32_t live = len - k < 32 ? len - k : 32;
              stab[s] = make_uint2(ys + k, live | (threadIdx.x << 8));
            }
          }
        }
        __syncthreads();
        if (Pq == 0) continue;
        const u64 gbase = s_gbase;
        const u64 zseg = tg.zrow + (u64)q * seg;
        int32_t* const coords = tg.coords;
        double* const vals = tg.vals;
        const int oz = tg.op.order;
        const bool v4 = oz == 4 && tg.op.pow2 && ((reinterpret_cast<uintptr_t>(coords) & 15u) == 0);
        for (uint32_t sb = warp; sb < S; sb += NW * U) {
          uint32_t f[U], e[U];
          double y[U];
          bool ok[U], in[U];
#pragma unroll
          for (int u = 0; u < U; u++) {
            const uint32_t si = sb + u * NW;
            in[u] = si < S;
            ok[u] = false;
            if (in[u]) {
              const uint2 rec = stab[si];
              ok[u] = lane < (rec.y & 255u);
              const uint32_t j = rec.x + (ok[u] ? lane : 0u);
              e[u] = rec.y >> 8;
              f[u] = ld_keep_u32(yfk + j, keep);
              y[u] = ld_keep_f64(a.yv + j, keep);
            }
          }
#pragma unroll
          for (int u = 0; u < U; u++) {
            if (in[u]) {
              const uint32_t fk = f[u] & (seg - 1);
              const double prod = __dmul_rn(sx[e[u]], y[u]);
              const uint32_t w = fk >> 5, bit = 1u << (fk & 31);
              bool first = false;
              if (ok[u]) {
                first = (atomicOr(bits + w, bit) & bit) == 0;
                if (!first) atomicOr(rbits + w, bit);
              }
              const uint32_t fm = __ballot_sync(0xffffffffu, first);
              const uint32_t rm = __ballot_sync(0xffffffffu, ok[u] && !first);
              uint32_t base = 0;
              if (lane == 0) base = atomicAdd(&s_cnt, (uint32_t)__popc(fm) | ((uint32_t)__popc(rm) << 16));
              base = __shfl_sync(0xffffffffu, base, 0);
              if (ok[u]) {
                if (first) {
                  const uint32_t place = (base & 0xffffu) + __popc(fm & lt);
                  pk[place] = (uint16_t)fk;
                  const u64 pos = gbase + place;
                  if (v4) {
                    const uint32_t fy = q * seg + fk;
                    const int4 cb = s_cst;
                    const uint4 sh = s_sh, mk = s_mk;
                    const int4 cv = make_int4(cb.x | (int32_t)((fy >> sh.x) & mk.x), cb.y | (int32_t)((fy >> sh.y) & mk.y),
                                              cb.z | (int32_t)((fy >> sh.z) & mk.z), cb.w | (int32_t)((fy >> sh.w) & mk.w));
                    st_stream_v4(coords + pos * 4, cv, pol);
                    vals[pos] = prod;  // default policy: a repeat may still add to it
                  } else {
                    store_output<FIXED>(coords, vals, pos, zseg + fk, prod, tg.op, pol);
                  }
                } else {
                  const u64 pos = gbase + Pq - 1 - ((base >> 16) + __popc(rm & lt));
                  if (oz) coords[pos * oz] = (int32_t)fk;
                  vals[pos] = prod;
                }
              }
            }
          }
        }
        if (!one_chunk) __syncthreads();
      }
      if (Pq == 0) {
        if (threadIdx.x == 0) sa.rec[(u64)gi * nseg + q] = StreamRec{0, 0, 0};
        continue;
      }
      // The block barrier orders every thread's earlier global stores (first products, repeats'
      // records) before the later reads and atomics of the block's threads, which are the only
      // ones that touch this group's reservation; no device-wide fence is needed.
      __syncthreads();
      const uint32_t nkeys = s_cnt & 0xffffu, reps = s_cnt >> 16;
      if (reps) {
        const u64 gbase = s_gbase;
        // Rank the repeated keys; the key marks are no longer needed and hold the ranks.
        const uint32_t wpt = (nwords + T - 1) / T;
        const uint32_t w0 = threadIdx.x * wpt, w1 = w0 + wpt < nwords ? w0 + wpt : nwords;
        uint32_t sum = 0;
        for (uint32_t w = w0; w < w1; w++) sum += __popc(rbits[w]);
        uint32_t nrk;
        uint32_t r = block_exscan_u32<T>(sum, &nrk, warp_tot);
        for (uint32_t w = w0; w < w1; w++) {
          bits[w] = r;
          r += __popc(rbits[w]);
        }
        __syncthreads();
        // Four first-product keys per 8-byte load (pk holds kStreamCap entries, so reading up
        // to the next multiple of four stays inside it; entries past nkeys are skipped).
        for (uint32_t q = threadIdx.x; q < (nkeys + 3) / 4; q += T) {
          const uint2 four = reinterpret_cast<const uint2*>(pk)[q];
#pragma unroll
          for (int t = 0; t < 4; t++) {
            const uint32_t i = q * 4 + t;
            const uint32_t fk = ((t < 2 ? four.x : four.y) >> ((t & 1) * 16)) & 0xffffu;
            const uint32_t w = fk >> 5, bit = 1u << (fk & 31), rw = rbits[w];
            if (i < nkeys && (rw & bit)) map[bits[w] + __popc(rw & (bit - 1))] = (uint16_t)i;
          }
        }
        __syncthreads();
        const int oz = tg.op.order;
        for (uint32_t k = threadIdx.x; k < reps; k += T) {
          const u64 pos = gbase + Pq - 1 - k;
          const uint32_t fk = oz ? (uint32_t)__ldcg(tg.coords + pos * oz) : 0u;
          const double v = __ldcg(tg.vals + pos);
          const uint32_t w = fk >> 5, bit = 1u << (fk & 31);
          atomicAdd(tg.vals + gbase + map[bits[w] + __popc(rbits[w] & (bit - 1))], v);
        }
        if (threadIdx.x == 0) atomicAdd(sa.holes, (u64)reps);
        __syncthreads();  // the lookups above read the bitmaps cleared below
      }
      // Every streamed segment is recorded, at its own index (list position, segment): those
      // whose outputs end above the final count are the sources of the hole filling, whatever
      // their repeats.
      if (threadIdx.x == 0) sa.rec[(u64)gi * nseg + q] = StreamRec{s_gbase, nkeys, Pq};
      // ---- clear the bitmaps for the next segment or group.
      for (uint32_t i = threadIdx.x; i < nwords / 4; i += T) {
        reinterpret_cast<uint4*>(bits)[i] = make_uint4(0, 0, 0, 0);
        reinterpret_cast<uint4*>(rbits)[i] = make_uint4(0, 0, 0, 0);
      }
      if (nwords < 4 && threadIdx.x < nwords) bits[threadIdx.x] = rbits[threadIdx.x] = 0;
      if (threadIdx.x == 0) s_cnt = 0;
      __syncthreads();
    }
  }
}

// Hole filling after the streaming kernel (its reservations are the last ones, so every
// other kernel's outputs lie below the final count). Sources: the entries of streamed
// segments at positions >= nnz; holes: the repeats' records below nnz. Both are numbered
// through atomic counters; hole k receives source k.
__global__ void __launch_bounds__(256) stream_sources_kernel(const StreamRec* __restrict__ rec,
                                                             const unsigned* __restrict__ nrec, u64 nnz,
                                                             uint32_t* __restrict__ src_pos, u64* __restrict__ src_count) {
  const unsigned lane = lane_id();
  const unsigned nr = *nrec;
  for (unsigned i = blockIdx.x * 8 + (threadIdx.x >> 5); i < nr; i += gridDim.x * 8) {
    const StreamRec r = rec[i];
    const u64 lo = r.base > nnz ? r.base : nnz, hi = r.base + r.firsts;
    if (lo >= hi) continue;
    u64 k0 = 0;
    if (lane == 0) k0 = atomicAdd(src_count, hi - lo);
    k0 = __shfl_sync(0xffffffffu, k0, 0);
    for (u64 p = lo + lane; p < hi; p += 32) src_pos[k0 + (p - lo)] = (uint32_t)(p - nnz);
  }
}

__global__ void __launch_bounds__(256) stream_fill_kernel(const StreamRec* __restrict__ rec,
                                                          const unsigned* __restrict__ nrec, u64 nnz,
                                                          const uint32_t* __restrict__ src_pos, u64 nsrc,
                                                          u64* __restrict__ hole_count, int32_t* __restrict__ coords,
                                                          double* __restrict__ vals, int oz, uint32_t* status) {
  const unsigned lane = lane_id();
  const unsigned nr = *nrec;
  for (unsigned i = blockIdx.x * 8 + (threadIdx.x >> 5); i < nr; i += gridDim.x * 8) {
    const StreamRec r = rec[i];
    const u64 lo = r.base + r.firsts, hi0 = r.base + r.products, hi = hi0 < nnz ? hi0 : nnz;
    if (lo >= hi) continue;
    u64 k0 = 0;
    if (lane == 0) k0 = atomicAdd(hole_count, hi - lo);
    k0 = __shfl_sync(0xffffffffu, k0, 0);
    for (u64 h = lo + lane; h < hi; h += 32) {
      const u64 k = k0 + (h - lo);
      if (k >= nsrc) {
        atomicOr(status, kStatOutOverflow);
        continue;
      }
      const u64 s = nnz + src_pos[k];
      if (oz == 4 && ((reinterpret_cast<uintptr_t>(coords) & 15u) == 0)) {
        reinterpret_cast<int4*>(coords)[h] = reinterpret_cast<const int4*>(coords)[s];
      } else {
        for (int q = 0; q < oz; q++) coords[h * oz + q] = coords[s * oz + q];
      }
      vals[h] = vals[s];
    }
  }
}


// ---- small groups: one warp per group, each warp with its own table (group-per-warp
// granularity). Everything a group needs stays inside its warp, so warp-level
// synchronisation replaces block barriers and warps progress independently.

template <int SLOTS, typename KT>
struct alignas(16) WarpSlice {
  double vals[SLOTS];
  KT keys[SLOTS];
  u64 pre[33];
  uint32_t ystart[32];
  double v[32];
  OutTarget tg;
};

static_assert(sizeof(WarpSlice<256, uint32_t>) % 16 == 0 && sizeof(WarpSlice<1024, uint32_t>) % 16 == 0 &&
                  sizeof(WarpSlice<256, u64>) % 16 == 0 && sizeof(WarpSlice<1024, u64>) % 16 == 0,
              "per-warp slices must keep the key buckets 16-byte aligned");

template <int SLOTS, typename KT, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) group_warp_kernel(GroupArgs a, const uint32_t* __restrict__ list,
                                                                const uint32_t* __restrict__ countp) {
  const uint32_t count = *countp;
  constexpr int B = Bucket<KT>::N;
  constexpr uint32_t NB = SLOTS / B;
  constexpr int D = 4;
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  WarpSlice<SLOTS, KT>& ws = reinterpret_cast<WarpSlice<SLOTS, KT>*>(smem)[warp];
  for (uint32_t i = lane; i < SLOTS; i += 32) ws.keys[i] = empty_key<KT>();
  if (lane == 0) ws.tg.prob = kNoProb;
  __syncwarp();
  const uint64_t keep = policy_evict_last();
  const uint64_t pol = policy_evict_first();
  for (uint32_t k = blockIdx.x * WARPS + warp; k < count; k += gridDim.x * WARPS) {
    const uint32_t g = list[k];
    const uint32_t x0 = a.goff[g], x1 = a.goff[g + 1];
    if (a.yuniq != nullptr && x1 - x0 == 1 && a.yuniq[a.gx.ystart[x0]]) {
      // One X entry over a run of all-different free keys: every product is an output of its
      // own, written as the run scaled by x, without the table.
      const uint32_t ys = a.gx.ystart[x0], len = a.gx.w[x0];
      const double xv = a.gx.v[x0];
      resolve_target_warp(a, g, len, ws.tg);
      for (uint32_t j = lane; j < len; j += 32) {
        u64 key;
        if constexpr (sizeof(KT) == 4)
          key = ld_keep_u32(static_cast<const uint32_t*>(a.yfk) + ys + j, keep);
        else
          key = ld_keep_u64(static_cast<const uint64_t*>(a.yfk) + ys + j, keep);
        const double prod = __dmul_rn(xv, ld_keep_f64(a.yv + ys + j, keep));
        const u64 pos = ws.tg.base + j;
        if (pos < ws.tg.cap)
          store_output(ws.tg.coords, ws.tg.vals, pos, ws.tg.zrow + key, prod, ws.tg.op, pol);
        else
          atomicOr(a.status, kStatOutOverflow);
      }
      __syncwarp();  // ws.tg is rewritten for the next group
      continue;
    }
    unsigned claims = 0;
    for (uint32_t c0 = x0; c0 < x1; c0 += 32) {
      const uint32_t n = (x1 - c0 < 32u) ? x1 - c0 : 32u;
      u64 w = 0;
      if (lane < n) {
        w = a.gx.w[c0 + lane];
        ws.ystart[lane] = a.gx.ystart[c0 + lane];
        ws.v[lane] = a.gx.v[c0 + lane];
      }
      u64 incl = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const u64 y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += y;
      }
      ws.pre[lane] = incl - w;
      const u64 total = __shfl_sync(0xffffffffu, incl, 31);
      if (lane == 0) ws.pre[32] = total;
      __syncwarp();
      // pre[n] must bound the walk: entries at or past n have w = 0, so pre[n..32] = total.
      uint32_t own = 0;
      for (u64 base = 0; base < total; base += 32 * D) {
        KT key[D];
        double prod[D];
#pragma unroll
        for (int u = 0; u < D; u++) {
          const u64 p = base + (u64)u * 32 + lane;
          uint32_t kk = own;
          key[u] = empty_key<KT>();
          if (p < total) {
            while (ws.pre[kk + 1] <= p) kk++;
            const u64 j = (u64)ws.ystart[kk] + (p - ws.pre[kk]);
            if constexpr (sizeof(KT) == 4)
              key[u] = (KT)ld_keep_u32(static_cast<const uint32_t*>(a.yfk) + j, keep);
            else
              key[u] = (KT)ld_keep_u64(static_cast<const uint64_t*>(a.yfk) + j, keep);
            prod[u] = __dmul_rn(ws.v[kk], ld_keep_f64(a.yv + j, keep));
          }
          own = __shfl_sync(0xffffffffu, kk, 31);
        }
        int later[D];
#pragma unroll
        for (int u = 0; u < D; u++) {
          later[u] = -1;
          bool claimed = false;
          if (key[u] != empty_key<KT>()) {
            const int slot = bucket_claim<KT, SLOTS>(ws.keys, key[u], &claimed);
            if (slot < 0) atomicOr(a.status, kStatTableFull);
            else if (claimed) ws.vals[slot] = prod[u];
            else later[u] = slot;
          }
          claims += __popc(__ballot_sync(0xffffffffu, claimed));
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < D; u++)
          if (later[u] >= 0) atomicAdd(ws.vals + later[u], prod[u]);
        __syncwarp();
      }
    }
    // Write the group's occupied slots, consecutive lanes storing consecutive outputs.
    resolve_target_warp(a, g, claims, ws.tg);
    unsigned off = 0;
    for (uint32_t b0 = 0; b0 < NB; b0 += 32) {
      const uint32_t b = b0 + lane;
      unsigned live = 0;
      if (b < NB) {
        const Bucket<KT> bk = load_bucket<KT>(ws.keys, b);
#pragma unroll
        for (int i = 0; i < B; i++) live |= (bk.k[i] != empty_key<KT>()) ? (1u << i) : 0u;
      }
      const unsigned cnt = __popc(live);
      unsigned incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += y;
      }
      const unsigned tot = __shfl_sync(0xffffffffu, incl, 31);
      for (unsigned k0 = 0; k0 < tot; k0 += 32) {
        const unsigned kq = k0 + lane;
        unsigned src = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const unsigned probe = __shfl_sync(0xffffffffu, incl, src + step - 1);
          if (probe <= kq) src += step;
        }
        const unsigned src_incl = __shfl_sync(0xffffffffu, incl, src);
        const unsigned src_live = __shfl_sync(0xffffffffu, live, src);
        if (kq < tot) {
          unsigned m = src_live;
          for (unsigned t = kq - (src_incl - __popc(src_live)); t > 0; t--) m &= m - 1;
          const uint32_t slot = (b0 + src) * B + (uint32_t)(__ffs(m) - 1);
          const u64 pos = ws.tg.base + off + kq;
          if (pos < ws.tg.cap)
            store_output(ws.tg.coords, ws.tg.vals, pos, ws.tg.zrow + (u64)ws.keys[slot], ws.vals[slot], ws.tg.op,
                         pol);
          else
            atomicOr(a.status, kStatOutOverflow);
        }
      }
      off += tot;
      __syncwarp();
      if (live) {
        KT* kb = ws.keys + b * B;
#pragma unroll
        for (int i = 0; i < B; i++) kb[i] = empty_key<KT>();
      }
    }
    __syncwarp();
  }
}

template <int SLOTS, typename KT>
cudaError_t launch_warp_class(const GroupArgs& a, const uint32_t* list, const uint32_t* countp, uint32_t count, int sms,
                              cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  constexpr int WARPS = 8;
  const size_t smem = WARPS * sizeof(WarpSlice<SLOTS, KT>);
  auto kern = group_warp_kernel<SLOTS, KT, WARPS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const uint32_t need = count == kCountOnDevice ? count : (count + WARPS - 1) / WARPS;
  const uint32_t cap = (uint32_t)(sms * per_sm);
  kern<<<need < cap ? need : cap, WARPS * 32, smem, s>>>(a, list, countp);
  note_launch();
  return cudaGetLastError();
}


// ---- small groups with direct output: one warp per group, each warp with its own table of
// 32-bit keys and output positions (no values in shared memory). A product that claims a new
// key writes its output entry at once: the round's claims are counted with ballots, one
// atomic on the problem's output counter reserves their positions, and consecutive claimers
// store at consecutive positions. Products whose key is already claimed add their value to
// that entry in global memory after the warp synchronises, which makes the claiming stores of
// the warp's lanes visible to its later atomics (only this warp touches the group's entries).
// Afterwards the table is cleared with vector stores: no scan of its slots writes the output.
template <int SLOTS>
struct alignas(16) WarpDirectSlice {
  uint32_t keys[SLOTS];
  uint32_t spos[SLOTS];  // output position of the key in the slot (within its problem's output)
  u64 pre[33];
  uint32_t ystart[32];
  double v[32];
  OutTarget tg;
};

template <int SLOTS, int WARPS, int D>
__global__ void __launch_bounds__(WARPS * 32) group_warp_direct_kernel(GroupArgs a,
                                                                       const uint32_t* __restrict__ list,
                                                                       const uint32_t* __restrict__ countp) {
  const uint32_t count = *countp;
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  const uint32_t lt = lanemask_lt();
  WarpDirectSlice<SLOTS>& ws = reinterpret_cast<WarpDirectSlice<SLOTS>*>(smem)[warp];
  for (uint32_t i = lane; i < SLOTS / 4; i += 32)
    reinterpret_cast<uint4*>(ws.keys)[i] = make_uint4(kEmpty32, kEmpty32, kEmpty32, kEmpty32);
  if (lane == 0) ws.tg.prob = kNoProb;
  __syncwarp();
  const uint64_t keep = policy_evict_last();
  const uint64_t pol = policy_evict_first();
  const uint32_t* yfk = static_cast<const uint32_t*>(a.yfk);
  for (uint32_t k = blockIdx.x * WARPS + warp; k < count; k += gridDim.x * WARPS) {
    const uint32_t g = list[k];
    const uint32_t x0 = a.goff[g], x1 = a.goff[g + 1];
    // One X entry over a run of all-different free keys: the run scaled by x, no table.
    const bool single = a.yuniq != nullptr && x1 - x0 == 1 && a.yuniq[a.gx.ystart[x0]];
    resolve_target_warp(a, g, single ? a.gx.w[x0] : 0u, ws.tg);
    const u64 cap = ws.tg.cap;
    if (single) {
      const uint32_t ys = a.gx.ystart[x0], len = a.gx.w[x0];
      const double xv = a.gx.v[x0];
      for (uint32_t j = lane; j < len; j += 32) {
        const uint32_t key = ld_keep_u32(yfk + ys + j, keep);
        const double prod = __dmul_rn(xv, ld_keep_f64(a.yv + ys + j, keep));
        const u64 pos = ws.tg.base + j;
        if (pos < cap)
          store_output(ws.tg.coords, ws.tg.vals, pos, ws.tg.zrow + (u64)key, prod, ws.tg.op, pol);
        else
          atomicOr(a.status, kStatOutOverflow);
      }
      __syncwarp();  // ws.tg is rewritten for the next group
      continue;
    }
    for (uint32_t c0 = x0; c0 < x1; c0 += 32) {
      const uint32_t n = (x1 - c0 < 32u) ? x1 - c0 : 32u;
      u64 w = 0;
      if (lane < n) {
        w = a.gx.w[c0 + lane];
        ws.ystart[lane] = a.gx.ystart[c0 + lane];
        ws.v[lane] = a.gx.v[c0 + lane];
      }
      u64 incl = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const u64 y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += y;
      }
      ws.pre[lane] = incl - w;
      const u64 total = __shfl_sync(0xffffffffu, incl, 31);
      if (lane == 0) ws.pre[32] = total;
      __syncwarp();
      // Entries at or past n have w = 0, so pre[n..32] = total bounds the walk.
      uint32_t own = 0;
      for (u64 base = 0; base < total; base += 32 * D) {
        uint32_t key[D];
        double prod[D];
#pragma unroll
        for (int u = 0; u < D; u++) {
          const u64 p = base + (u64)u * 32 + lane;
          uint32_t kk = own;
          key[u] = kEmpty32;
          if (p < total) {
            while (ws.pre[kk + 1] <= p) kk++;
            const u64 j = (u64)ws.ystart[kk] + (p - ws.pre[kk]);
            key[u] = ld_keep_u32(yfk + j, keep);
            prod[u] = __dmul_rn(ws.v[kk], ld_keep_f64(a.yv + j, keep));
          }
          own = __shfl_sync(0xffffffffu, kk, 31);
        }
        int slot[D];
        bool mine[D];
        uint32_t m[D];
        uint32_t nclaim = 0;
#pragma unroll
        for (int u = 0; u < D; u++) {
          slot[u] = -1;
          mine[u] = false;
          if (key[u] != kEmpty32) {
            slot[u] = bucket_claim<uint32_t, SLOTS>(ws.keys, key[u], &mine[u]);
            if (slot[u] < 0) atomicOr(a.status, kStatTableFull);
          }
          m[u] = __ballot_sync(0xffffffffu, mine[u]);
          nclaim += __popc(m[u]);
        }
        u64 rb = 0;
        if (nclaim) {
          if (lane == 0) rb = atomicAdd(ws.tg.counter, (u64)nclaim);
          rb = __shfl_sync(0xffffffffu, rb, 0);
        }
        uint32_t off = 0;
#pragma unroll
        for (int u = 0; u < D; u++) {
          if (mine[u]) {
            const u64 pos = rb + off + __popc(m[u] & lt);
            ws.spos[slot[u]] = (uint32_t)pos;
            if (pos < cap)
              store_output(ws.tg.coords, ws.tg.vals, pos, ws.tg.zrow + (u64)key[u], prod[u], ws.tg.op, pol);
            else
              atomicOr(a.status, kStatOutOverflow);
          }
          off += __popc(m[u]);
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < D; u++) {
          if (slot[u] >= 0 && !mine[u]) {
            const u64 pos = ws.spos[slot[u]];
            if (pos < cap) atomicAdd(ws.tg.vals + pos, prod[u]);
          }
        }
      }
      __syncwarp();  // the chunk's staging is rewritten by the next chunk
    }
    for (uint32_t i = lane; i < SLOTS / 4; i += 32)
      reinterpret_cast<uint4*>(ws.keys)[i] = make_uint4(kEmpty32, kEmpty32, kEmpty32, kEmpty32);
    __syncwarp();
  }
}

template <int SLOTS, int D>
cudaError_t launch_warp_direct_class(const GroupArgs& a, const uint32_t* list, const uint32_t* countp, uint32_t count,
                                     int sms, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  constexpr int WARPS = 8;
  const size_t smem = WARPS * sizeof(WarpDirectSlice<SLOTS>);
  auto kern = group_warp_direct_kernel<SLOTS, WARPS, D>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const uint32_t need = count == kCountOnDevice ? count : (count + WARPS - 1) / WARPS;
  const uint32_t cap = (uint32_t)(sms * per_sm);
  kern<<<need < cap ? need : cap, WARPS * 32, smem, s>>>(a, list, countp);
  note_launch();
  return cudaGetLastError();
}

// ---- direct output: a product that claims a new key writes its output entry at once.
// The table holds keys and output positions only. A claimer takes a rank inside its round
// (warp-aggregated); after the round's claims are counted, one atomic per round reserves the
// output positions, and claimers store their entry at base + rank (consecutive lanes,
// consecutive positions). Products whose key was already present add their value to that
// entry in global memory after a block barrier, which makes the claiming stores of the
// block's threads visible to the block's later atomics (only this block touches the group's
// entries). No values are kept in shared memory and no table scan writes the output.
template <int SLOTS, int THREADS, int D, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) group_direct_kernel(GroupArgs a, const uint32_t* __restrict__ list,
                                                                     const uint32_t* __restrict__ countp) {
  const uint32_t count = *countp;
  constexpr int NW = THREADS / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* keys = reinterpret_cast<uint32_t*>(smem);
  uint32_t* spos = keys + SLOTS;
  Chunk<THREADS>& c = *reinterpret_cast<Chunk<THREADS>*>(smem + 2 * SLOTS * sizeof(uint32_t));
  __shared__ u64 warp_tot[NW];
  __shared__ unsigned round_claims;
  __shared__ u64 round_base;
  __shared__ OutTarget tg;
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  for (uint32_t i = threadIdx.x; i < SLOTS / 4; i += THREADS)
    reinterpret_cast<uint4*>(keys)[i] = make_uint4(kEmpty32, kEmpty32, kEmpty32, kEmpty32);
  if (threadIdx.x == 0) round_claims = 0;
  const uint64_t keep = policy_evict_last();
  const uint64_t pol = policy_evict_first();
  if (threadIdx.x < 32) {  // warp 0 resolves the targets: no plan cached yet
    if (threadIdx.x == 0) tg.prob = kNoProb;
    __syncwarp();
  }
  for (uint32_t gi = blockIdx.x; gi < count; gi += gridDim.x) {
    const uint32_t g = list[gi];
    const uint32_t x0 = a.goff[g], x1 = a.goff[g + 1];
    // One X entry over a run of all-different free keys: the run scaled by x, no table.
    const bool single = a.yuniq != nullptr && x1 - x0 == 1 && a.yuniq[a.gx.ystart[x0]];
    if (warp == 0) resolve_target_warp(a, g, single ? a.gx.w[x0] : 0u, tg);  // published by the next barrier
    if (single) {
      __syncthreads();
      const uint32_t ys = a.gx.ystart[x0], len = a.gx.w[x0];
      const double xv = a.gx.v[x0];
      for (uint32_t j = threadIdx.x; j < len; j += THREADS) {
        const uint32_t key = ld_keep_u32(static_cast<const uint32_t*>(a.yfk) + ys + j, keep);
        const double prod = __dmul_rn(xv, ld_keep_f64(a.yv + ys + j, keep));
        const u64 pos = tg.base + j;
        if (pos < tg.cap)
          store_output(tg.coords, tg.vals, pos, tg.zrow + (u64)key, prod, tg.op, pol);
        else
          atomicOr(a.status, kStatOutOverflow);
      }
      __syncthreads();  // tg is rewritten for the next group
      continue;
    }
    for (uint32_t c0 = x0; c0 < x1; c0 += THREADS) {
      const uint32_t n = (x1 - c0 < (uint32_t)THREADS) ? x1 - c0 : (uint32_t)THREADS;
      load_chunk<THREADS>(a, c, warp_tot, c0, n);  // its barriers also publish tg
      const u64 total = c.pre[n];
      const u64 lo = total * warp / NW, hi = total * (warp + 1) / NW;
      uint32_t own = 0;
      if (lo < hi) {
        uint32_t l = 0, h = n - 1;
        while (l < h) {
          const uint32_t mid = (l + h + 1) >> 1;
          if (c.pre[mid] <= lo) l = mid; else h = mid - 1;
        }
        own = l;
      }
      const u64 per = (total + NW - 1) / NW;
      const uint32_t rounds = (uint32_t)((per + 32 * D - 1) / (32 * D));
      for (uint32_t r = 0; r < rounds; r++) {
        const u64 base = lo + (u64)r * 32 * D;
        uint32_t key[D];
        double prod[D];
#pragma unroll
        for (int u = 0; u < D; u++) {
          const u64 p = base + (u64)u * 32 + lane;
          uint32_t k = own;
          key[u] = kEmpty32;
          if (p < hi) {
            while (c.pre[k + 1] <= p) k++;
            const u64 j = (u64)c.ystart[k] + (p - c.pre[k]);
            key[u] = ld_keep_u32(static_cast<const uint32_t*>(a.yfk) + j, keep);
            prod[u] = __dmul_rn(c.v[k], ld_keep_f64(a.yv + j, keep));
          }
          own = __shfl_sync(0xffffffffu, k, 31);
        }
        int slot[D];
        unsigned rank[D];
        bool mine[D];
#pragma unroll
        for (int u = 0; u < D; u++) {
          slot[u] = -1;
          mine[u] = false;
          if (key[u] != kEmpty32) {
            slot[u] = bucket_claim<uint32_t, SLOTS>(keys, key[u], &mine[u]);
            if (slot[u] < 0) atomicOr(a.status, kStatTableFull);
          }
          const unsigned m = __ballot_sync(0xffffffffu, mine[u]);
          unsigned wbase = 0;
          if (m) {
            const int leader = __ffs(m) - 1;
            if ((int)lane == leader) wbase = atomicAdd(&round_claims, (unsigned)__popc(m));
            wbase = __shfl_sync(0xffffffffu, wbase, leader);
          }
          rank[u] = wbase + __popc(m & lanemask_lt());
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          const unsigned nclaim = round_claims;
          round_base = nclaim ? atomicAdd(tg.counter, (u64)nclaim) : 0;
          round_claims = 0;
        }
        __syncthreads();
        const u64 rb = round_base;
#pragma unroll
        for (int u = 0; u < D; u++) {
          if (mine[u]) {
            const u64 pos = rb + rank[u];
            spos[slot[u]] = (uint32_t)pos;
            if (pos < tg.cap)
              store_output(tg.coords, tg.vals, pos, tg.zrow + (u64)key[u], prod[u], tg.op, pol);
            else
              atomicOr(a.status, kStatOutOverflow);
          }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < D; u++) {
          if (slot[u] >= 0 && !mine[u]) {
            const u64 pos = spos[slot[u]];
            if (pos < tg.cap) atomicAdd(tg.vals + pos, prod[u]);
          }
        }
      }
      __syncthreads();
    }
    for (uint32_t i = threadIdx.x; i < SLOTS / 4; i += THREADS)
      reinterpret_cast<uint4*>(keys)[i] = make_uint4(kEmpty32, kEmpty32, kEmpty32, kEmpty32);
    __syncthreads();
  }
}

template <int SLOTS, int THREADS, int D, int MINB>
cudaError_t launch_direct_class(const GroupArgs& a, const uint32_t* list, const uint32_t* countp, uint32_t count,
                                int sms, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const size_t smem = 2 * SLOTS * sizeof(uint32_t) + sizeof(Chunk<THREADS>);
  auto kern = group_direct_kernel<SLOTS, THREADS, D, MINB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const uint32_t cap = (uint32_t)(sms * per_sm);
  kern<<<count < cap ? count : cap, THREADS, smem, s>>>(a, list, countp);
  note_launch();
  return cudaGetLastError();
}

template <int SLOTS, int THREADS, typename KT>
cudaError_t launch_class(const GroupArgs& a, const uint32_t* list, const uint32_t* countp, uint32_t count, int sms,
                         cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const size_t smem = SLOTS * (sizeof(double) + sizeof(KT)) + sizeof(Chunk<THREADS>);
  auto kern = group_smem_kernel<SLOTS, THREADS, KT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const uint32_t cap = (uint32_t)(sms * per_sm);
  kern<<<count < cap ? count : cap, THREADS, smem, s>>>(a, list, countp);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

// Table classes: slots and threads per group (32 = one warp per group). The binning threshold
// of class c is tmax[c] = floor(alpha * slots_c), alpha set by the host (default 0.75).
const ClassShape kClassShapes32[] = {{256, 32}, {1024, 32}, {4096, 256}, {8192, 512}, {16384, 1024}};
const ClassShape kClassShapes64[] = {{256, 32}, {1024, 32}, {4096, 256}, {8192, 512}};
const int kNumClasses32 = 5;
const int kNumClasses64 = 4;

cudaError_t launch_x_group_scatter(Survivors sv, uint32_t* gcur, GroupedX gx, int64_t max_ns, int sms,
                                   cudaStream_t s) {
  if (max_ns <= 0) return cudaSuccess;
  x_group_scatter_kernel<<<grid_for(max_ns, sms), kThreads, 0, s>>>(sv, gcur, gx);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bin_groups(u64 FX, const uint32_t* goff, const uint32_t* gw, u64 FY, const Bins& b, int sms,
                              cudaStream_t s) {
  if (FX == 0) return cudaSuccess;
  bin_groups_kernel<<<grid_for((int64_t)FX * 32, sms), kThreads, 0, s>>>(FX, goff, gw, FY, b);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_group_classes(const GroupArgs& a, bool wide_keys, bool direct, const Bins& b,
                                 const uint32_t* counts, int sms, cudaStream_t s, int depth) {
  cudaError_t e = cudaSuccess;
  // Host counts size the grids (a class without groups is not launched); without them
  // (counts == nullptr) each class kernel runs a full persistent grid and reads its count.
  uint32_t h[kMaxClasses];
  for (int c = 0; c < kMaxClasses; c++) h[c] = counts ? counts[c] : kCountOnDevice;
  const uint32_t* d = b.count;
  if (!wide_keys && direct) {
    // The expansion split: products each lane forms per round before the claims of the round.
    if (depth == 0) {
      if ((e = launch_warp_direct_class<256, 4>(a, b.list[0], d + 0, h[0], sms, s))) return e;
      if ((e = launch_warp_direct_class<1024, 4>(a, b.list[1], d + 1, h[1], sms, s))) return e;
    } else {
      if ((e = launch_warp_direct_class<256, 2>(a, b.list[0], d + 0, h[0], sms, s))) return e;
      if ((e = launch_warp_direct_class<1024, 2>(a, b.list[1], d + 1, h[1], sms, s))) return e;
    }
    if (depth == 0) {
      if ((e = launch_direct_class<4096, 256, 6, 4>(a, b.list[2], d + 2, h[2], sms, s))) return e;
      if ((e = launch_direct_class<8192, 512, 6, 2>(a, b.list[3], d + 3, h[3], sms, s))) return e;
      if ((e = launch_direct_class<16384, 1024, 4, 1>(a, b.list[4], d + 4, h[4], sms, s))) return e;
    } else {
      if ((e = launch_direct_class<4096, 256, 3, 4>(a, b.list[2], d + 2, h[2], sms, s))) return e;
      if ((e = launch_direct_class<8192, 512, 3, 2>(a, b.list[3], d + 3, h[3], sms, s))) return e;
      if ((e = launch_direct_class<16384, 1024, 2, 1>(a, b.list[4], d + 4, h[4], sms, s))) return e;
    }
  } else if (!wide_keys) {
    if ((e = launch_warp_class<256, uint32_t>(a, b.list[0], d + 0, h[0], sms, s))) return e;
    if ((e = launch_warp_class<1024, uint32_t>(a, b.list[1], d + 1, h[1], sms, s))) return e;
    if ((e = launch_class<4096, 256, uint32_t>(a, b.list[2], d + 2, h[2], sms, s))) return e;
    if ((e = launch_class<8192, 512, uint32_t>(a, b.list[3], d + 3, h[3], sms, s))) return e;
    if ((e = launch_class<16384, 1024, uint32_t>(a, b.list[4], d + 4, h[4], sms, s))) return e;
  } else {
    if ((e = launch_warp_class<256, u64>(a, b.list[0], d + 0, h[0], sms, s))) return e;
    if ((e = launch_warp_class<1024, u64>(a, b.list[1], d + 1, h[1], sms, s))) return e;
    if ((e = launch_class<4096, 256, u64>(a, b.list[2], d + 2, h[2], sms, s))) return e;
    if ((e = launch_class<8192, 512, u64>(a, b.list[3], d + 3, h[3], sms, s))) return e;
  }
  return cudaSuccess;
}

// ---- lane-private dense rows: output rows of at most kRowMax free keys (F_Y <= 64) that
// receive many products each (both operands' contract keys skewed). One warp per group (X free
// key); every lane owns a row of F_Y doubles in shared memory and adds its products into it, a
// rounded product and then a rounded add as everywhere else, with no atomics; a 64-bit mask per
// lane records the keys the lane has met. At the end the 32 rows are summed column by column
// in lane order (a lane that never met a key adds an exact zero, so an output of one or two
// products is the same sum as in any other accumulator), the masks are combined, and the
// group's outputs are written in key order after one reservation.
constexpr uint32_t kRowMax = 64;
constexpr uint32_t kRowStride = kRowMax + 1;  // odd stride in doubles: a column spreads over banks
constexpr int kRowWarps = 4;
constexpr int kRowD = 4;  // products per lane per round, loaded before any of them is added
constexpr size_t kRowSmem = (size_t)kRowWarps * 32 * kRowStride * sizeof(double);

__global__ void __launch_bounds__(kRowWarps * 32) group_lanerow_kernel(GroupArgs a, u64 ngroups, uint32_t FY) {
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  double* const rows = reinterpret_cast<double*>(smem) + (size_t)warp * 32 * kRowStride;
  double* const myrow = rows + (size_t)lane * kRowStride;
  __shared__ u64 s_pre[kRowWarps][33];
  __shared__ uint32_t s_ys[kRowWarps][32];
  __shared__ double s_v[kRowWarps][32];
  __shared__ OutTarget s_tg[kRowWarps];
  OutTarget& tg = s_tg[warp];
  u64* const pre = s_pre[warp];
  uint32_t* const ysv = s_ys[warp];
  double* const xv = s_v[warp];
  for (uint32_t c = 0; c < kRowMax; c++) myrow[c] = 0.0;
  if (lane == 0) tg.prob = kNoProb;
  __syncwarp();
  const uint64_t keep = policy_evict_last();
  const uint64_t pol = policy_evict_first();
  const uint32_t* yfk = static_cast<const uint32_t*>(a.yfk);
  for (u64 g = (u64)blockIdx.x * kRowWarps + warp; g < ngroups; g += (u64)gridDim.x * kRowWarps) {
    const uint32_t x0 = a.goff[g], x1 = a.goff[g + 1];
    if (x0 == x1) continue;  // uniform over the warp
    u64 seen = 0;
    for (uint32_t c0 = x0; c0 < x1; c0 += 32) {
      const uint32_t n = (x1 - c0 < 32u) ? x1 - c0 : 32u;
      u64 w = 0;
      if (lane < n) {
        w = a.gx.w[c0 + lane];
        ysv[lane] = a.gx.ystart[c0 + lane];
        xv[lane] = a.gx.v[c0 + lane];
      }
      u64 incl = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const u64 y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += y;
      }
      pre[lane] = incl - w;
      const u64 total = __shfl_sync(0xffffffffu, incl, 31);
      if (lane == 0) pre[32] = total;
      __syncwarp();
      // Entries at or past n have w = 0, so pre[n..32] = total bounds the walk.
      uint32_t own = 0;
      for (u64 base = 0; base < total; base += 32 * kRowD) {
        uint32_t fk[kRowD];
        double prod[kRowD];
#pragma unroll
        for (int u = 0; u < kRowD; u++) {
          const u64 p = base + (u64)u * 32 + lane;
          uint32_t kk = own;
          fk[u] = kRowMax;  // no product
          if (p < total) {
            while (pre[kk + 1] <= p) kk++;
            const u64 j = (u64)ysv[kk] + (p - pre[kk]);
            fk[u] = ld_keep_u32(yfk + j, keep);
            prod[u] = __dmul_rn(xv[kk], ld_keep_f64(a.yv + j, keep));
          }
          own = __shfl_sync(0xffffffffu, kk, 31);
        }
#pragma unroll
        for (int u = 0; u < kRowD; u++) {
          if (fk[u] < FY) {
            myrow[fk[u]] = __dadd_rn(myrow[fk[u]], prod[u]);
            seen |= 1ull << fk[u];
          }
        }
      }
      __syncwarp();  // the chunk's staging is rewritten by the next chunk
    }
    const u64 any = (u64)__reduce_or_sync(0xffffffffu, (uint32_t)seen) |
                    ((u64)__reduce_or_sync(0xffffffffu, (uint32_t)(seen >> 32)) << 32);
    resolve_target_warp(a, g, (unsigned)__popcll(any), tg);  // also orders the rows' stores
    for (uint32_t c = lane; c < FY; c += 32) {
      if ((any >> c) & 1ull) {
        double sum = 0.0;
        for (int l = 0; l < 32; l++) sum = __dadd_rn(sum, rows[(size_t)l * kRowStride + c]);
        const u64 pos = tg.base + (u64)__popcll(any & ((1ull << c) - 1ull));
        if (pos < tg.cap)
          store_output(tg.coords, tg.vals, pos, tg.zrow + c, sum, tg.op, pol);
        else
          atomicOr(a.status, kStatOutOverflow);
      }
    }
    __syncwarp();  // every column is summed before the rows are cleared
    for (uint32_t c = 0; c < FY; c++) myrow[c] = 0.0;
    __syncwarp();
  }
}

cudaError_t launch_group_lanerow(const GroupArgs& a, u64 ngroups, uint32_t FY, int sms, cudaStream_t s) {
  if (ngroups == 0) return cudaSuccess;
  if (FY == 0 || FY > kRowMax) return cudaErrorInvalidValue;
  auto kern = group_lanerow_kernel;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRowSmem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRowWarps * 32, kRowSmem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const u64 want = (ngroups + kRowWarps - 1) / kRowWarps, cap = (u64)sms * per_sm;
  kern<<<(unsigned)(want < cap ? want : cap), kRowWarps * 32, kRowSmem, s>>>(a, ngroups, FY);
  note_launch();
  return cudaGetLastError();
}

uint32_t dense_stash_cap() { return kStashCap; }
uint32_t dense_stream_cap() { return kStreamCap; }

cudaError_t launch_group_stream(const GroupArgs& a, const uint32_t* yoff, uint32_t nseg, uint32_t seg,
                                const uint32_t* list, uint32_t count, StreamArgs sa, bool fixed_rows, int sms,
                                cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  if (seg < 64 || seg > kDenseSeg) return cudaErrorInvalidValue;
  constexpr int U = STREAM_U;
  auto kern = fixed_rows ? group_stream_kernel<U, true> : group_stream_kernel<U, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStreamSmem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kStreamThreads, kStreamSmem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const uint32_t cap = (uint32_t)(sms * per_sm);
  kern<<<count < cap ? count : cap, kStreamThreads, kStreamSmem, s>>>(a, yoff, nseg, seg, list, count, sa);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_stream_fill(const StreamRec* rec, const unsigned* nrec, u64 nnz, u64 holes_total, uint32_t* src_pos,
                               u64* counters2, int32_t* coords, double* vals, int oz, uint32_t* status, int sms,
                               cudaStream_t s) {
  if (holes_total == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(counters2, 0, 2 * sizeof(u64), s);
  if (e != cudaSuccess) return e;
  const unsigned g = (unsigned)sms * 8;
  stream_sources_kernel<<<g, 256, 0, s>>>(rec, nrec, nnz, src_pos, counters2);
  stream_fill_kernel<<<g, 256, 0, s>>>(rec, nrec, nnz, src_pos, holes_total, counters2 + 1, coords, vals, oz, status);
  note_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_group_dense(const GroupArgs& a, const uint32_t* yoff, uint32_t nseg, uint32_t seg,
                               const uint32_t* stash_list, uint32_t stash_count, const uint32_t* rank_list,
                               uint32_t rank_count, int sms, cudaStream_t s) {
  if (seg < 64 || seg > kDenseSeg) return cudaErrorInvalidValue;
  cudaError_t e = cudaSuccess;
  if (stash_count) {
    constexpr int U = STASH_U;
    auto kern = group_stash_kernel<U>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStashSmem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kStashThreads, kStashSmem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const uint32_t cap = (uint32_t)(sms * per_sm);
    kern<<<stash_count < cap ? stash_count : cap, kStashThreads, kStashSmem, s>>>(a, yoff, nseg, seg, stash_list,
                                                                                  stash_count);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (rank_count) {
    constexpr int T = 512, U1 = 4, U2 = 2;
    static_assert(bitmap_smem<T>() <= kBitmapSmemPerCta && bitmap_vcap<T>() >= 4096, "bitmap layout");
    const size_t smem = bitmap_smem<T>();
    auto kern = group_bitmap_kernel<T, U1, U2>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const uint32_t cap = (uint32_t)(sms * per_sm);
    kern<<<rank_count < cap ? rank_count : cap, T, smem, s>>>(a, yoff, nseg, seg, rank_list, rank_count);
    note_launch();
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t launch_group_huge(const GroupArgs& a, const HugeGroups& h, bool wide_keys, int sms, cudaStream_t s) {
  if (h.count == 0) return cudaSuccess;  // h.count == kCountOnDevice: unknown on the host
  const uint32_t cap = (uint32_t)sms * 2;
  if (wide_keys)
    group_global_kernel<512, u64><<<h.count < cap ? h.count : cap, 512, 0, s>>>(a, h);
  else
    group_global_kernel<512, uint32_t><<<h.count < cap ? h.count : cap, 512, 0, s>>>(a, h);
  note_launch();
  return cudaGetLastError();
}

}  // namespace stc
