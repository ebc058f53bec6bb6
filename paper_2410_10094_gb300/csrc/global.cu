// Contraction and accumulation into one device-wide open-addressing table (Section 2.4.2
// contraction; Section 4.3 probing table sized from the exact product count), followed
// by the writeback of occupied slots as COO output (Section 2.5).
//
// This is the "leave X ungrouped" form noted at the end of Section 4.4: every product
// goes to one global table keyed on the full output key. It is chosen when the output
// key space is small enough for the whole table to stay in L2.
#include "launch.h"

namespace stc {

namespace {

constexpr int kExThreads = 256;
constexpr int kExTile = 2048;  // products per merge-path tile
constexpr int kCpThreads = 256;

// Linear probing (Section 2.3.1) with a compare-and-swap claim of empty slots. A slot's key
// only ever changes from empty to its final key, so a stale read can only show "empty"
// and is then settled by the CAS. The probe sequence is bounded by the table size.
__device__ __forceinline__ void table_add(u64* __restrict__ keys, double* __restrict__ vals, u64 mask, u64 key,
                                          double v, uint32_t* status) {
  u64 slot = mix64(key) & mask;
  for (u64 probe = 0; probe <= mask; probe++) {
    u64 cur = __ldcg(keys + slot);
    if (cur == kEmpty64) {
      const u64 prev = atomicCAS(keys + slot, kEmpty64, key);
      cur = (prev == kEmpty64) ? key : prev;
    }
    if (cur == key) {
      atomicAdd(vals + slot, v);
      return;
    }
    slot = (slot + 1) & mask;
  }
  atomicOr(status, kStatTableFull);
}

// Cooperative probing: a tile of G consecutive lanes inserts its lanes' keys one at a time.
// The table is read as buckets of G consecutive slots (G·8 contiguous bytes of the key array,
// one 32-byte sector for G = 4); every lane of the tile reads one slot of the bucket and two
// ballots tell the whole tile whether the key is there and where the first free slot is. A
// key is placed in the first free slot of the first bucket of its probe sequence that has
// one, so a key is found in the bucket where it would be placed: the invariant of linear
// probing (Section 2.3.1) over buckets instead of slots. A lost claim reads the bucket again.
// Every lane of the warp calls this (`has` false for lanes without a product); `done` and the
// ballots' masks are uniform over a tile, so the tile's lanes stay converged where they
// exchange values.
template <int G>
__device__ __forceinline__ void table_add_coop(u64* __restrict__ keys, double* __restrict__ vals, u64 mask, bool has,
                                               u64 key, double v, uint32_t* status) {
  constexpr unsigned kFull = 0xffffffffu;
  const unsigned lane = lane_id();
  const unsigned base = lane & ~(unsigned)(G - 1);
  const unsigned tmask = (G == 32) ? kFull : (((1u << G) - 1u) << base);
  const unsigned r = lane - base;
  const u64 bmask = mask / G;  // buckets - 1 (the capacity is a power of two >= G)
  bool todo = has;
  while (__any_sync(kFull, todo)) {
    const unsigned pend = __ballot_sync(kFull, todo) & tmask;
    const int src = pend ? __ffs(pend) - 1 : (int)lane;
    const u64 k = __shfl_sync(kFull, key, src);
    const double x = __shfl_sync(kFull, v, src);
    if ((int)lane == src) todo = false;
    bool done = pend == 0;
    u64 b = (mix64(k) & mask) / G;
    u64 steps = 0;
    while (__any_sync(kFull, !done)) {
      const u64 cur = done ? kEmpty64 : __ldcg(keys + b * G + r);
      const unsigned hit = __ballot_sync(kFull, !done && cur == k) & tmask;
      const unsigned emp = __ballot_sync(kFull, !done && cur == kEmpty64) & tmask;
      if (done) continue;
      if (hit) {
        if ((int)lane == __ffs(hit) - 1) atomicAdd(vals + b * G + r, x);
        done = true;
      } else if (emp) {
        const int e = __ffs(emp) - 1;
        u64 prev = 0;
        if ((int)lane == e) prev = atomicCAS(keys + b * G + r, kEmpty64, k);
        prev = __shfl_sync(tmask, prev, e);
        if (prev == kEmpty64 || prev == k) {
          if ((int)lane == e) atomicAdd(vals + b * G + r, x);
          done = true;
        }
      } else {
        b = (b + 1) & bmask;
        if (++steps > bmask) {
          if (lane == base) atomicOr(status, kStatTableFull);
          done = true;
        }
      }
    }
  }
}

// Each CTA takes tiles of kExTile consecutive products. Products are numbered by the
// survivors' exclusive prefix `wpre`: survivor s owns products [wpre[s], wpre[s+1]), its
// r-th product pairs it with slot ystart[s] + r of its Y run. Within a tile, thread t
// handles products t, t+256, ...; consecutive threads read consecutive Y slots.
// With dP / dns non-null, P and the survivor count are read on the device (the grid then is a
// persistent one sized by the host without them). G = 1: each lane probes on its own
// (table_add); G > 1: tiles of G lanes probe buckets together (table_add_coop). The loop over
// a tile's products is uniform over each warp, so all lanes reach the cooperative probe.
template <int G>
__global__ void __launch_bounds__(kExThreads) expand_global_kernel(
    const u64* __restrict__ wpre, int64_t ns, u64 P, const u64* __restrict__ sfk, const uint32_t* __restrict__ systart,
    const double* __restrict__ sv, const u64* __restrict__ yfk, const double* __restrict__ yv, u64 FY,
    GlobalTable t, uint32_t* status, const u64* dP, const unsigned* dns) {
  if (dP) P = *dP;
  if (dns) ns = (int64_t)*dns;
  if (P == 0 || ns <= 0) return;
  __shared__ u64 s_pre[kExTile + 1];
  __shared__ int64_t s_lo;
  __shared__ int s_n;
  const u64 ntiles = (P + kExTile - 1) / kExTile;
  for (u64 tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const u64 p0 = tile * kExTile;
    const u64 p1 = (p0 + kExTile < P) ? p0 + kExTile : P;
    if (threadIdx.x == 0) {
      // Largest s with wpre[s] <= p0, then largest s with wpre[s] <= p1 - 1.
      int64_t a = 0, b = ns - 1;
      while (a < b) {
        const int64_t mid = (a + b + 1) >> 1;
        if (wpre[mid] <= p0) a = mid; else b = mid - 1;
      }
      int64_t c = a, d = ns - 1;
      while (c < d) {
        const int64_t mid = (c + d + 1) >> 1;
        if (wpre[mid] <= p1 - 1) c = mid; else d = mid - 1;
      }
      s_lo = a;
      s_n = (int)(c - a + 1);
    }
    __syncthreads();
    const int64_t lo = s_lo;
    const int n = s_n;
    for (int k = threadIdx.x; k <= n; k += kExThreads) s_pre[k] = wpre[lo + k];
    __syncthreads();
    for (u64 g0 = p0 + (threadIdx.x & ~31u); g0 < p1; g0 += kExThreads) {
      const u64 g = g0 + lane_id();
      const bool has = g < p1;
      u64 key = 0;
      double prod = 0.0;
      if (has) {
        int a = 0, b = n - 1;
        while (a < b) {
          const int mid = (a + b + 1) >> 1;
          if (s_pre[mid] <= g) a = mid; else b = mid - 1;
        }
        const int64_t s = lo + a;
        const u64 j = (u64)__ldg(systart + s) + (g - s_pre[a]);
        key = __ldg(sfk + s) * FY + __ldg(yfk + j);
        prod = __dmul_rn(__ldg(sv + s), __ldg(yv + j));
      }
      if (G == 1) {
        if (has) table_add(t.keys, t.vals, t.mask, key, prod, status);
      } else {
        table_add_coop<G>(t.keys, t.vals, t.mask, has, key, prod, status);
      }
    }
    __syncthreads();
  }
}

// Each CTA takes 2048 consecutive slots at a time (8 per thread, coalesced), ranks the
// occupied ones with a block scan and reserves their output positions with one atomic.
constexpr int kCpItems = 8;
__global__ void __launch_bounds__(kCpThreads) compact_global_kernel(GlobalTable t, OutPlan op,
                                                                    int32_t* __restrict__ coords,
                                                                    double* __restrict__ vals, u64 out_cap,
                                                                    u64* __restrict__ nz, uint32_t* status) {
  constexpr int NW = kCpThreads / 32;
  __shared__ uint32_t s_warp[NW + 1];
  __shared__ u64 s_base;
  const int64_t cap = (int64_t)t.mask + 1;
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  for (int64_t base = (int64_t)blockIdx.x * kCpThreads * kCpItems; base < cap;
       base += (int64_t)gridDim.x * kCpThreads * kCpItems) {
    u64 k[kCpItems];
    uint32_t cnt = 0;
#pragma unroll
    for (int it = 0; it < kCpItems; it++) {
      const int64_t i = base + (int64_t)it * kCpThreads + threadIdx.x;
      k[it] = i < cap ? __ldcs(t.keys + i) : kEmpty64;
      cnt += k[it] != kEmpty64;
    }
    uint32_t x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if ((int)lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t run = 0;
      for (int w = 0; w < NW; w++) {
        const uint32_t v = s_warp[w];
        s_warp[w] = run;
        run += v;
      }
      s_base = run ? atomicAdd(nz, (u64)run) : 0;
    }
    __syncthreads();
    u64 pos = s_base + s_warp[warp] + x - cnt;
#pragma unroll
    for (int it = 0; it < kCpItems; it++) {
      if (k[it] == kEmpty64) continue;
      if (pos < out_cap) {
        const int64_t i = base + (int64_t)it * kCpThreads + threadIdx.x;
        store_coords(k[it], op, coords + pos * (u64)op.order);
        vals[pos] = __ldcs(t.vals + i);
      } else {
        atomicOr(status, kStatOutOverflow);
      }
      pos++;
    }
    __syncthreads();  // s_warp and s_base are rewritten by the next round
  }
}

}  // namespace

namespace {
using ExpandKernel = void (*)(const u64*, int64_t, u64, const u64*, const uint32_t*, const double*, const u64*,
                              const double*, u64, GlobalTable, uint32_t*, const u64*, const unsigned*);
ExpandKernel expand_for(int probe) {
  switch (probe) {
    case 4: return expand_global_kernel<4>;
    case 8: return expand_global_kernel<8>;
    default: return expand_global_kernel<1>;
  }
}
}  // namespace

cudaError_t launch_expand_global(const u64* wpre, int64_t ns, u64 P, Survivors sv, const u64* yfk, const double* yv,
                                 u64 FY, GlobalTable t, uint32_t* status, int sms, cudaStream_t s, int probe) {
  if (P == 0 || ns <= 0) return cudaSuccess;
  const u64 ntiles = (P + kExTile - 1) / kExTile;
  const u64 cap = (u64)sms * 8;
  const unsigned g = (unsigned)(ntiles < cap ? ntiles : cap);
  expand_for(probe)<<<g, kExThreads, 0, s>>>(wpre, ns, P, sv.fk, sv.ystart, sv.v, yfk, yv, FY, t, status, nullptr,
                                             nullptr);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_expand_global_dev(const u64* wpre, const unsigned* dns, const u64* dP, Survivors sv, const u64* yfk,
                                     const double* yv, u64 FY, GlobalTable t, uint32_t* status, int sms,
                                     cudaStream_t s, int probe) {
  expand_for(probe)<<<(unsigned)sms * 8, kExThreads, 0, s>>>(wpre, 0, 0, sv.fk, sv.ystart, sv.v, yfk, yv, FY, t,
                                                             status, dP, dns);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_compact_global(GlobalTable t, const OutPlan& op, int32_t* coords, double* vals, u64 out_cap,
                                  u64* nz, uint32_t* status, int sms, cudaStream_t s) {
  const u64 cap = t.mask + 1;
  const u64 want = (cap + kCpThreads * kCpItems - 1) / (kCpThreads * kCpItems);
  const u64 lim = (u64)sms * 8;
  compact_global_kernel<<<(unsigned)(want < lim ? want : lim), kCpThreads, 0, s>>>(t, op, coords, vals, out_cap, nz,
                                                                                  status);
  note_launch();
  return cudaGetLastError();
}

}  // namespace stc
