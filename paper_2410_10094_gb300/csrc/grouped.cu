// Per-X-free-group accumulation (Sections 4.1, 4.3): X entries that share a free key form
// one group; its outputs can never collide with another group's (Section 2.3.2), so each
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
      my_cap += t;
      int c = 0;
      while (c < b.nclasses && t > b.tmax[c]) c++;
      if (c < b.nclasses) {
        const uint32_t idx = atomicAdd(b.count + c, 1u);
        b.list[c][idx] = (uint32_t)g;
      } else if (t > (1ull << 30)) {
        atomicOr(b.status, kStatTooLarge);
      } else {
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
// claimed with a compare-and-swap (linear probing over buckets, Section 2.2.1).

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
                                                             uint32_t count) {
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
  for (uint32_t k = blockIdx.x; k < h.count; k += gridDim.x) {
    const uint32_t g = h.list[k];
    u64* keys = h.keys + h.off[k];
    double* vals = h.vals + h.off[k];
    const uint32_t cap = (uint32_t)h.cap[k];
    expand_group_global<THREADS, YK>(a, c, warp_tot, a.goff[g], a.goff[g + 1], keys, vals, cap - 1);
    write_group_global<THREADS>(a, g, keys, vals, cap, warp_cnt, warp_base, tg);
  }
}


// ---- dense rows: one free-key segment of one group at a time, accumulated in a dense
// shared-memory array indexed by the free key (no hashing, no probing). Ownership of a slot
// is settled without atomics: each product writes its id into the slot's tag unless the slot
// is already owned; after a barrier the product whose id survived stores its value, and the
// others (rare when outputs seldom repeat) add theirs atomically after a second barrier.

template <int THREADS>
struct DenseChunk {
  u64 pre[THREADS + 1];
  uint32_t ck[THREADS];
  uint32_t ystart[THREADS];
  double v[THREADS];
};

template <int THREADS>
__device__ __forceinline__ void dense_stage(const GroupArgs& a, DenseChunk<THREADS>& c, uint32_t c0, uint32_t n) {
  if (threadIdx.x < n) {
    c.ck[threadIdx.x] = a.gx.ck[c0 + threadIdx.x];
    c.v[threadIdx.x] = a.gx.v[c0 + threadIdx.x];
  }
}

// Expands segment q of the staged entries into the dense accumulator.
template <int THREADS, int D>
__device__ __forceinline__ void dense_expand(const GroupArgs& a, DenseChunk<THREADS>& c, u64* warp_tot,
                                             const uint32_t* __restrict__ yoff, uint32_t nseg, uint32_t q,
                                             uint32_t seg, uint32_t n, double* acc, uint16_t* tag,
                                             unsigned* winners) {
  constexpr int NW = THREADS / 32;
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  u64 w = 0;
  if (threadIdx.x < n) {
    const u64 b = (u64)c.ck[threadIdx.x] * nseg + q;
    const uint32_t lo = __ldg(yoff + b);
    c.ystart[threadIdx.x] = lo;
    w = __ldg(yoff + b + 1) - lo;
  }
  block_scan<THREADS>(c.pre, w, warp_tot);
  __syncthreads();
  const u64 total = c.pre[n];
  if (total == 0) return;
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
  const uint32_t* yfk = static_cast<const uint32_t*>(a.yfk);
  const u64 per = (total + NW - 1) / NW;
  const uint32_t rounds = (uint32_t)((per + 32 * D - 1) / (32 * D));
  unsigned my_win = 0;
  for (uint32_t r = 0; r < rounds; r++) {
    const u64 base = lo + (u64)r * 32 * D;
    uint32_t slot[D];
    double prod[D];
    int st[D];  // 0 nothing, 1 candidate owner, 2 adds later
#pragma unroll
    for (int u = 0; u < D; u++) {
      const u64 p = base + (u64)u * 32 + lane;
      uint32_t k = own;
      st[u] = 0;
      if (p < hi) {
        while (c.pre[k + 1] <= p) k++;
        const u64 j = (u64)c.ystart[k] + (p - c.pre[k]);
        slot[u] = __ldg(yfk + j) & (seg - 1);
        prod[u] = __dmul_rn(c.v[k], __ldg(a.yv + j));
        st[u] = 1;
      }
      own = __shfl_sync(0xffffffffu, k, 31);
    }
#pragma unroll
    for (int u = 0; u < D; u++) {
      if (st[u] == 1) {
        volatile uint16_t* t = tag + slot[u];
        if (*t != 0) st[u] = 2;
        else *t = (uint16_t)(threadIdx.x * D + u + 1);
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < D; u++) {
      bool won = false;
      if (st[u] == 1) {
        if (tag[slot[u]] == (uint16_t)(threadIdx.x * D + u + 1)) {
          acc[slot[u]] = prod[u];
          won = true;
        } else {
          st[u] = 2;
        }
      }
      my_win += __popc(__ballot_sync(0xffffffffu, won));
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < D; u++)
      if (st[u] == 2) atomicAdd(acc + slot[u], prod[u]);
  }
  if (lane == 0 && my_win) atomicAdd(winners, my_win);
}

// Writes segment q of group g (its owned slots, in free-key order within each warp's slice)
// and frees the tags.
template <int THREADS>
__device__ __forceinline__ void dense_write(const GroupArgs& a, u64 g, uint32_t q, uint32_t seg, const double* acc,
                                            uint16_t* tag, unsigned* winners, unsigned* cursor, u64* gbase) {
  const unsigned lane = lane_id();
  if (threadIdx.x == 0) {
    const unsigned n = *winners;
    *gbase = n ? atomicAdd(a.nz, (u64)n) : 0;
    *cursor = 0;
    *winners = 0;
  }
  __syncthreads();
  const u64 base = *gbase;
  const u64 zrow = g * a.FY + (u64)q * seg;
  const int oz = a.op.order;
  for (uint32_t blk = 0; blk < seg; blk += THREADS * 8) {
    const uint32_t s0 = blk + threadIdx.x * 8;
    uint4 tv = make_uint4(0, 0, 0, 0);
    if (s0 < seg) tv = *reinterpret_cast<const uint4*>(tag + s0);
    const uint32_t words[4] = {tv.x, tv.y, tv.z, tv.w};
    unsigned live = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) live |= ((words[i >> 1] >> (16 * (i & 1))) & 0xffffu) ? (1u << i) : 0u;
    const unsigned cnt = __popc(live);
    unsigned pre = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, pre, o);
      if ((int)lane >= o) pre += y;
    }
    const unsigned tot = __shfl_sync(0xffffffffu, pre, 31);
    unsigned off = 0;
    if (lane == 0 && tot) off = atomicAdd(cursor, tot);
    off = __shfl_sync(0xffffffffu, off, 0) + pre - cnt;
    if (live) {
      for (unsigned m = live; m; m &= m - 1) {
        const int i = __ffs(m) - 1;
        {
          const u64 pos = base + off++;
          if (pos < a.out_cap) {
            const u64 z = zrow + s0 + i;
            int32_t* dst = a.coords + pos * (u64)oz;
            if (oz == 4 && a.op.pow2 && ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0)) {
              int4 cv;
              cv.x = (int32_t)((z >> a.op.shift[0]) & (a.op.mod[0] - 1));
              cv.y = (int32_t)((z >> a.op.shift[1]) & (a.op.mod[1] - 1));
              cv.z = (int32_t)((z >> a.op.shift[2]) & (a.op.mod[2] - 1));
              cv.w = (int32_t)((z >> a.op.shift[3]) & (a.op.mod[3] - 1));
              __stcs(reinterpret_cast<int4*>(dst), cv);
            } else {
              for (int qq = 0; qq < oz; qq++) __stcs(dst + qq, out_coord(z, a.op, qq));
            }
            __stcs(a.vals + pos, acc[s0 + i]);
          } else {
            atomicOr(a.status, kStatOutOverflow);
          }
        }
      }
      *reinterpret_cast<uint4*>(tag + s0) = make_uint4(0, 0, 0, 0);
    }
  }
  __syncthreads();
}

// Persistent over the group list; every group is swept one free-key segment at a time.
template <int THREADS, int D>
__global__ void __launch_bounds__(THREADS) group_dense_kernel(GroupArgs a, const uint32_t* __restrict__ yoff,
                                                              uint32_t nseg, uint32_t seg,
                                                              const uint32_t* __restrict__ list, uint32_t count) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* acc = reinterpret_cast<double*>(smem);
  uint16_t* tag = reinterpret_cast<uint16_t*>(acc + kDenseSeg);
  DenseChunk<THREADS>& c = *reinterpret_cast<DenseChunk<THREADS>*>(tag + kDenseSeg);
  __shared__ u64 warp_tot[THREADS / 32];
  __shared__ unsigned winners, cursor;
  __shared__ u64 gbase;
  for (uint32_t i = threadIdx.x; i < kDenseSeg / 8; i += THREADS)
    reinterpret_cast<uint4*>(tag)[i] = make_uint4(0, 0, 0, 0);
  if (threadIdx.x == 0) winners = 0;
  __syncthreads();
  for (uint32_t k = blockIdx.x; k < count; k += gridDim.x) {
    const uint32_t g = list[k];
    const uint32_t x0 = a.goff[g], x1 = a.goff[g + 1];
    const bool one_chunk = x1 - x0 <= (uint32_t)THREADS;
    if (one_chunk) dense_stage<THREADS>(a, c, x0, x1 - x0);
    for (uint32_t q = 0; q < nseg; q++) {
      for (uint32_t c0 = x0; c0 < x1; c0 += THREADS) {
        const uint32_t n = (x1 - c0 < (uint32_t)THREADS) ? x1 - c0 : (uint32_t)THREADS;
        if (!one_chunk) dense_stage<THREADS>(a, c, c0, n);
        dense_expand<THREADS, D>(a, c, warp_tot, yoff, nseg, q, seg, n, acc, tag, &winners);
        __syncthreads();
      }
      dense_write<THREADS>(a, g, q, seg, acc, tag, &winners, &cursor, &gbase);
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
                                                                uint32_t count) {
  constexpr int B = Bucket<KT>::N;
  constexpr uint32_t NB = SLOTS / B;
  constexpr int D = 4;
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  WarpSlice<SLOTS, KT>& ws = reinterpret_cast<WarpSlice<SLOTS, KT>*>(smem)[warp];
  for (uint32_t i = lane; i < SLOTS; i += 32) ws.keys[i] = empty_key<KT>();
  __syncwarp();
  const uint64_t keep = policy_evict_last();
  const uint64_t pol = policy_evict_first();
  for (uint32_t k = blockIdx.x * WARPS + warp; k < count; k += gridDim.x * WARPS) {
    const uint32_t g = list[k];
    const uint32_t x0 = a.goff[g], x1 = a.goff[g + 1];
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
    if (lane == 0) resolve_target(a, g, claims, ws.tg);
    __syncwarp();
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
cudaError_t launch_warp_class(const GroupArgs& a, const uint32_t* list, uint32_t count, int sms, cudaStream_t s) {
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
  const uint32_t need = (count + WARPS - 1) / WARPS;
  const uint32_t cap = (uint32_t)(sms * per_sm);
  kern<<<need < cap ? need : cap, WARPS * 32, smem, s>>>(a, list, count);
  note_launch();
  return cudaGetLastError();
}


// ---- direct output: a product that claims a new key writes its output entry at once.
// The table holds keys and output positions only. A claimer takes a rank inside its round
// (warp-aggregated); after the round's claims are counted, one atomic per round reserves the
// output positions, and claimers store their entry at base + rank (consecutive lanes,
// consecutive positions). Products whose key was already present add their value to that
// entry in global memory after a device-scope fence and a barrier, when the claiming store
// is visible. No values are kept in shared memory and no table scan writes the output.
template <int SLOTS, int THREADS, int D, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) group_direct_kernel(GroupArgs a, const uint32_t* __restrict__ list,
                                                                     uint32_t count) {
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
  for (uint32_t gi = blockIdx.x; gi < count; gi += gridDim.x) {
    const uint32_t g = list[gi];
    if (threadIdx.x == 0) resolve_target(a, g, 0, tg);
    const uint32_t x0 = a.goff[g], x1 = a.goff[g + 1];
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
        __threadfence();
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
cudaError_t launch_direct_class(const GroupArgs& a, const uint32_t* list, uint32_t count, int sms, cudaStream_t s) {
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
  kern<<<count < cap ? count : cap, THREADS, smem, s>>>(a, list, count);
  note_launch();
  return cudaGetLastError();
}

template <int SLOTS, int THREADS, typename KT>
cudaError_t launch_class(const GroupArgs& a, const uint32_t* list, uint32_t count, int sms, cudaStream_t s) {
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
  kern<<<count < cap ? count : cap, THREADS, smem, s>>>(a, list, count);
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
                                 const uint32_t* counts, int sms, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (!wide_keys && direct) {
    if ((e = launch_warp_class<256, uint32_t>(a, b.list[0], counts[0], sms, s))) return e;
    if ((e = launch_warp_class<1024, uint32_t>(a, b.list[1], counts[1], sms, s))) return e;
    if ((e = launch_direct_class<4096, 256, 6, 4>(a, b.list[2], counts[2], sms, s))) return e;
    if ((e = launch_direct_class<8192, 512, 6, 2>(a, b.list[3], counts[3], sms, s))) return e;
    if ((e = launch_direct_class<16384, 1024, 4, 1>(a, b.list[4], counts[4], sms, s))) return e;
  } else if (!wide_keys) {
    if ((e = launch_warp_class<256, uint32_t>(a, b.list[0], counts[0], sms, s))) return e;
    if ((e = launch_warp_class<1024, uint32_t>(a, b.list[1], counts[1], sms, s))) return e;
    if ((e = launch_class<4096, 256, uint32_t>(a, b.list[2], counts[2], sms, s))) return e;
    if ((e = launch_class<8192, 512, uint32_t>(a, b.list[3], counts[3], sms, s))) return e;
    if ((e = launch_class<16384, 1024, uint32_t>(a, b.list[4], counts[4], sms, s))) return e;
  } else {
    if ((e = launch_warp_class<256, u64>(a, b.list[0], counts[0], sms, s))) return e;
    if ((e = launch_warp_class<1024, u64>(a, b.list[1], counts[1], sms, s))) return e;
    if ((e = launch_class<4096, 256, u64>(a, b.list[2], counts[2], sms, s))) return e;
    if ((e = launch_class<8192, 512, u64>(a, b.list[3], counts[3], sms, s))) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_group_dense(const GroupArgs& a, const uint32_t* yoff, uint32_t nseg, uint32_t seg,
                               const uint32_t* list, uint32_t count, int sms, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  constexpr int T = 512, D = 4;
  const size_t smem = kDenseSeg * (sizeof(double) + sizeof(uint16_t)) + sizeof(DenseChunk<T>);
  auto kern = group_dense_kernel<T, D>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const uint32_t cap = (uint32_t)(sms * per_sm);
  kern<<<count < cap ? count : cap, T, smem, s>>>(a, yoff, nseg, seg, list, count);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_group_huge(const GroupArgs& a, const HugeGroups& h, bool wide_keys, int sms, cudaStream_t s) {
  if (h.count == 0) return cudaSuccess;
  const uint32_t cap = (uint32_t)sms * 2;
  if (wide_keys)
    group_global_kernel<512, u64><<<h.count < cap ? h.count : cap, 512, 0, s>>>(a, h);
  else
    group_global_kernel<512, uint32_t><<<h.count < cap ? h.count : cap, 512, 0, s>>>(a, h);
  note_launch();
  return cudaGetLastError();
}

}  // namespace stc
