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
    gx.ystart[pos] = sv.ystart[i];
    gx.w[pos] = sv.w[i];
    gx.v[pos] = sv.v[i];
  }
}

// One thread per X free key: non-empty groups go to the first class whose table holds
// their bound t = min(B_g, F_Y); larger ones get a region of the overflow table.
__global__ void __launch_bounds__(kThreads) bin_groups_kernel(u64 FX, const uint32_t* __restrict__ gcnt,
                                                              const u64* __restrict__ gbound, u64 FY, Bins b) {
  __shared__ u64 s_cap[kThreads / 32];
  u64 my_cap = 0;
  for (int64_t base = (int64_t)blockIdx.x * kThreads + (threadIdx.x & ~31u); base < (int64_t)FX;
       base += (int64_t)gridDim.x * kThreads) {
    const int64_t g = base + lane_id();
    if (g < (int64_t)FX && gcnt[g] != 0) {
      const u64 bnd = gbound[g];
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
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_cap += __shfl_down_sync(0xffffffffu, my_cap, o);
  if (lane_id() == 0) s_cap[threadIdx.x >> 5] = my_cap;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 t = 0;
    for (int w = 0; w < kThreads / 32; w++) t += s_cap[w];
    if (t) atomicAdd(b.out_cap, t);
  }
}

// ---------------------------------------------------------------- accumulation

// Shared-memory staging of one chunk of a group's X entries: the exclusive prefix of their
// run lengths (products), the first slot of each run, and the X values.
template <int THREADS>
struct Chunk {
  u64 pre[THREADS + 1];
  uint32_t ystart[THREADS];
  double v[THREADS];
};

// Exclusive block scan of one u64 per thread into c.pre[0..THREADS], c.pre[THREADS] = total.
template <int THREADS>
__device__ __forceinline__ void chunk_scan(Chunk<THREADS>& c, u64 w, u64* warp_tot) {
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
    c.pre[THREADS] = run;
  }
  __syncthreads();
  c.pre[threadIdx.x] = warp_tot[warp] + x - w;
}

// Insert (key, v) into a linear-probing table of mask+1 slots: claim an empty slot with a
// compare-and-swap, or find the key, then add v to the slot's value.
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

// Expands every product of group g's X entries [x0, x1) into the table. Products of a chunk
// of THREADS X entries are spread over the threads in order (consecutive threads read
// consecutive slots of a Y run); the owning X entry of product p is found by binary search
// in the chunk's prefix.
template <int THREADS, typename KT>
__device__ __forceinline__ void expand_group(const GroupArgs& a, Chunk<THREADS>& c, u64* warp_tot, uint32_t x0,
                                             uint32_t x1, KT* keys, double* vals, uint32_t mask) {
  for (uint32_t c0 = x0; c0 < x1; c0 += THREADS) {
    const uint32_t n = (x1 - c0 < (uint32_t)THREADS) ? x1 - c0 : (uint32_t)THREADS;
    const uint32_t xi = c0 + threadIdx.x;
    u64 w = 0;
    if (threadIdx.x < n) {
      w = a.gx.w[xi];
      c.ystart[threadIdx.x] = a.gx.ystart[xi];
      c.v[threadIdx.x] = a.gx.v[xi];
    }
    chunk_scan<THREADS>(c, w, warp_tot);
    __syncthreads();
    const u64 total = c.pre[THREADS];
    for (u64 p = threadIdx.x; p < total; p += THREADS) {
      uint32_t lo = 0, hi = n - 1;
      while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (c.pre[mid] <= p) lo = mid; else hi = mid - 1;
      }
      const u64 j = (u64)c.ystart[lo] + (p - c.pre[lo]);
      const KT key = (KT)__ldg(a.yfk + j);
      const double prod = __dmul_rn(c.v[lo], __ldg(a.yv + j));
      if (!probe_add<KT>(keys, vals, mask, key, prod)) atomicOr(a.status, kStatTableFull);
    }
    __syncthreads();
  }
}

// Writes the occupied slots of group g's table as COO output and empties the table for
// the next group. Each warp owns a contiguous slice of the table; one atomic per group
// reserves the group's output range.
template <int THREADS, typename KT>
__device__ __forceinline__ void write_group(const GroupArgs& a, u64 g, KT* keys, double* vals, uint32_t slots,
                                            uint32_t* warp_cnt, u64* warp_base) {
  constexpr int NW = THREADS / 32;
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  const uint32_t per = (slots + NW - 1) / NW;
  const uint32_t s0 = warp * per;
  const uint32_t s1 = (s0 + per < slots) ? s0 + per : slots;
  uint32_t cnt = 0;
  for (uint32_t i = s0 + lane; i < s1; i += 32) cnt += keys[i] != empty_key<KT>();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  if (lane == 0) warp_cnt[warp] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 tot = 0;
    for (int k = 0; k < NW; k++) tot += warp_cnt[k];
    u64 base = tot ? atomicAdd(a.nz, tot) : 0;
    for (int k = 0; k < NW; k++) {
      warp_base[k] = base;
      base += warp_cnt[k];
    }
  }
  __syncthreads();
  u64 run = warp_base[warp];
  const u64 gbase = g * a.FY;
  for (uint32_t i0 = s0; i0 < s1; i0 += 32) {
    const uint32_t i = i0 + lane;
    KT k = empty_key<KT>();
    if (i < s1) k = keys[i];
    const bool live = k != empty_key<KT>();
    const unsigned m = __ballot_sync(0xffffffffu, live);
    if (live) {
      const u64 pos = run + __popc(m & lanemask_lt());
      if (pos < a.out_cap) {
        store_coords(gbase + (u64)k, a.op, a.coords + pos * (u64)a.op.order);
        a.vals[pos] = vals[i];
      } else {
        atomicOr(a.status, kStatOutOverflow);
      }
      keys[i] = empty_key<KT>();
      vals[i] = 0.0;
    }
    run += __popc(m);
  }
  __syncthreads();
}

// Persistent: CTA b takes groups b, b + grid, ... of its class list. The shared-memory
// table is cleared once; write_group leaves it empty again after each group.
template <int SLOTS, int THREADS, typename KT>
__global__ void __launch_bounds__(THREADS) group_smem_kernel(GroupArgs a, const uint32_t* __restrict__ list,
                                                             uint32_t count) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* vals = reinterpret_cast<double*>(smem);
  KT* keys = reinterpret_cast<KT*>(vals + SLOTS);
  Chunk<THREADS>& c = *reinterpret_cast<Chunk<THREADS>*>(smem + SLOTS * (sizeof(double) + sizeof(KT)));
  __shared__ u64 warp_tot[THREADS / 32];
  __shared__ uint32_t warp_cnt[THREADS / 32];
  __shared__ u64 warp_base[THREADS / 32];
  for (int i = threadIdx.x; i < SLOTS; i += THREADS) {
    keys[i] = empty_key<KT>();
    vals[i] = 0.0;
  }
  __syncthreads();
  for (uint32_t k = blockIdx.x; k < count; k += gridDim.x) {
    const uint32_t g = list[k];
    const uint32_t x0 = a.goff[g], x1 = a.goff[g + 1];
    expand_group<THREADS, KT>(a, c, warp_tot, x0, x1, keys, vals, SLOTS - 1);
    write_group<THREADS, KT>(a, g, keys, vals, SLOTS, warp_cnt, warp_base);
  }
}

// Groups whose table does not fit in shared memory: one CTA per group, the table a region
// of a global array (cleared by the host before the launch).
template <int THREADS>
__global__ void __launch_bounds__(THREADS) group_global_kernel(GroupArgs a, HugeGroups h) {
  __shared__ Chunk<THREADS> c;
  __shared__ u64 warp_tot[THREADS / 32];
  __shared__ uint32_t warp_cnt[THREADS / 32];
  __shared__ u64 warp_base[THREADS / 32];
  for (uint32_t k = blockIdx.x; k < h.count; k += gridDim.x) {
    const uint32_t g = h.list[k];
    u64* keys = h.keys + h.off[k];
    double* vals = h.vals + h.off[k];
    const uint32_t cap = (uint32_t)h.cap[k];
    expand_group<THREADS, u64>(a, c, warp_tot, a.goff[g], a.goff[g + 1], keys, vals, cap - 1);
    __threadfence_block();
    write_group<THREADS, u64>(a, g, keys, vals, cap, warp_cnt, warp_base);
  }
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

// Table classes: slots and threads per CTA. The binning threshold of class c is
// tmax[c] = floor(alpha_c * slots_c) (set by the host; default alpha 0.5).
const ClassShape kClassShapes32[] = {{128, 64}, {1024, 128}, {4096, 256}, {8192, 512}, {16384, 1024}};
const ClassShape kClassShapes64[] = {{128, 64}, {1024, 128}, {4096, 256}, {8192, 512}};
const int kNumClasses32 = 5;
const int kNumClasses64 = 4;

cudaError_t launch_x_group_scatter(Survivors sv, uint32_t* gcur, GroupedX gx, int64_t max_ns, int sms,
                                   cudaStream_t s) {
  if (max_ns <= 0) return cudaSuccess;
  x_group_scatter_kernel<<<grid_for(max_ns, sms), kThreads, 0, s>>>(sv, gcur, gx);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bin_groups(u64 FX, const uint32_t* gcnt, const u64* gbound, u64 FY, const Bins& b, int sms,
                              cudaStream_t s) {
  if (FX == 0) return cudaSuccess;
  bin_groups_kernel<<<grid_for((int64_t)FX, sms), kThreads, 0, s>>>(FX, gcnt, gbound, FY, b);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_group_classes(const GroupArgs& a, bool wide_keys, const Bins& b, const uint32_t* counts,
                                 int sms, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (!wide_keys) {
    if ((e = launch_class<128, 64, uint32_t>(a, b.list[0], counts[0], sms, s))) return e;
    if ((e = launch_class<1024, 128, uint32_t>(a, b.list[1], counts[1], sms, s))) return e;
    if ((e = launch_class<4096, 256, uint32_t>(a, b.list[2], counts[2], sms, s))) return e;
    if ((e = launch_class<8192, 512, uint32_t>(a, b.list[3], counts[3], sms, s))) return e;
    if ((e = launch_class<16384, 1024, uint32_t>(a, b.list[4], counts[4], sms, s))) return e;
  } else {
    if ((e = launch_class<128, 64, u64>(a, b.list[0], counts[0], sms, s))) return e;
    if ((e = launch_class<1024, 128, u64>(a, b.list[1], counts[1], sms, s))) return e;
    if ((e = launch_class<4096, 256, u64>(a, b.list[2], counts[2], sms, s))) return e;
    if ((e = launch_class<8192, 512, u64>(a, b.list[3], counts[3], sms, s))) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_group_huge(const GroupArgs& a, const HugeGroups& h, int sms, cudaStream_t s) {
  if (h.count == 0) return cudaSuccess;
  const uint32_t cap = (uint32_t)sms * 2;
  group_global_kernel<512><<<h.count < cap ? h.count : cap, 512, 0, s>>>(a, h);
  note_launch();
  return cudaGetLastError();
}

}  // namespace stc
