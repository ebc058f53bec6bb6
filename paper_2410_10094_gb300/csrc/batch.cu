// Batches of independent contractions that share every pass: the inputs of all problems are
// processed as one flattened row space (each row finds its problem by binary search over the
// row offsets), Y is grouped over the concatenation of all problems' contract-key bins, and
// X's survivors are grouped by (problem, X free key). Because the problems' X free key spaces
// together are far too large to count directly, each distinct (problem, free key) pair gets a
// small number through a probing table, in order of first sight (Section 4.1.2, Fig. 7).
// The per-group accumulation then runs in the same class kernels as a single contraction.
#include "launch.h"

namespace stc {

namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(int64_t n, int sms, int per_sm = 8) {
  const int64_t want = (n + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)sms * per_sm;
  return (unsigned)(want < 1 ? 1 : (want < cap ? want : cap));
}

// The problem owning flattened row r: the largest p with off[p] <= r (off has n + 1 entries).
__device__ __forceinline__ int row_problem(const int64_t* __restrict__ off, int n, int64_t r) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= r) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int key_problem(const u64* __restrict__ off, int n, u64 key) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= key) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Contract and free keys of row i of a tensor whose order is only known at run time.
__device__ __forceinline__ bool row_keys_any(const int32_t* __restrict__ coords, int64_t i, const KeyPlan& p,
                                             uint64_t& ck, uint64_t& fk) {
  bool ok = true;
  ck = 0;
  fk = 0;
  for (int j = 0; j < p.order; j++) {
    const int32_t c = __ldg(coords + i * p.order + j);
    ok &= (c >= 0) & ((int64_t)c < p.size[j]);
    ck += (uint64_t)(uint32_t)c * p.cstride[j];
    fk += (uint64_t)(uint32_t)c * p.fstride[j];
  }
  return ok;
}

__global__ void __launch_bounds__(kThreads) y_count_batch_kernel(const BatchProb* __restrict__ pb,
                                                                 const int64_t* __restrict__ yrow, int n,
                                                                 int64_t total, uint32_t* __restrict__ cnt,
                                                                 uint32_t* status) {
  for (int64_t r = (int64_t)blockIdx.x * kThreads + threadIdx.x; r < total; r += (int64_t)gridDim.x * kThreads) {
    const int p = row_problem(yrow, n, r);
    const BatchProb& q = pb[p];
    uint64_t ck, fk;
    if (!row_keys_any(q.yc, r - yrow[p], q.ky, ck, fk)) {
      atomicOr(status, kStatCoordRange);
      continue;
    }
    atomicAdd(cnt + q.koff + ck, 1u);
  }
}

template <typename YK>
__global__ void __launch_bounds__(kThreads) y_scatter_batch_kernel(const BatchProb* __restrict__ pb,
                                                                   const int64_t* __restrict__ yrow, int n,
                                                                   int64_t total, uint32_t* __restrict__ cursor,
                                                                   YK* __restrict__ yfk, double* __restrict__ yv) {
  for (int64_t r = (int64_t)blockIdx.x * kThreads + threadIdx.x; r < total; r += (int64_t)gridDim.x * kThreads) {
    const int p = row_problem(yrow, n, r);
    const BatchProb& q = pb[p];
    const int64_t i = r - yrow[p];
    uint64_t ck, fk;
    if (!row_keys_any(q.yc, i, q.ky, ck, fk)) continue;
    const uint32_t pos = atomicAdd(cursor + q.koff + ck, 1u);
    yfk[pos] = (YK)fk;
    yv[pos] = __ldg(q.yv + i);
  }
}

// Marks the Y runs (the entries of one contract-key bin) whose free keys are all different:
// yuniq[first entry of the run] = 1, else 0. One warp per run, with a table of kUniqSlots keys
// in shared memory (linear probing, one compare-and-swap per entry); runs longer than half the
// table are set to 0 here and decided by run_unique_long_kernel up to kUniqLongMax entries (the
// longer ones keep the table path). The table is cleared after every run.
constexpr int kUniqWarps = 8;
constexpr uint32_t kUniqSlots = 1024;
__global__ void __launch_bounds__(kUniqWarps * 32) run_unique_kernel(const uint32_t* __restrict__ yoff, u64 bins,
                                                                    const uint32_t* __restrict__ yfk,
                                                                    uint8_t* __restrict__ yuniq) {
  __shared__ __align__(16) uint32_t tab[kUniqWarps][kUniqSlots];
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  uint32_t* const t = tab[warp];
  for (uint32_t i = lane; i < kUniqSlots / 4; i += 32)
    reinterpret_cast<uint4*>(t)[i] = make_uint4(kEmpty32, kEmpty32, kEmpty32, kEmpty32);
  __syncwarp();
  for (u64 b = (u64)blockIdx.x * kUniqWarps + warp; b < bins; b += (u64)gridDim.x * kUniqWarps) {
    const uint32_t s0 = yoff[b], len = yoff[b + 1] - s0;
    if (len <= 1) {
      if (len == 1 && lane == 0) yuniq[s0] = 1;
      continue;
    }
    if (len > kUniqSlots / 2) {
      if (lane == 0) yuniq[s0] = 0;
      continue;
    }
    bool dup = false;
    for (uint32_t j = lane; j < len; j += 32) {
      const uint32_t key = yfk[s0 + j];
      uint32_t h = (key * 0x9E3779B1u) >> 22;  // 10 bits: kUniqSlots slots
      for (uint32_t probe = 0; probe < kUniqSlots; probe++) {
        const uint32_t prev = atomicCAS(t + h, kEmpty32, key);
        if (prev == kEmpty32) break;
        if (prev == key) {
          dup = true;
          break;
        }
        h = (h + 1) & (kUniqSlots - 1);
      }
    }
    const bool any = __any_sync(0xffffffffu, dup);
    if (lane == 0) yuniq[s0] = any ? 0 : 1;
    __syncwarp();
    for (uint32_t i = lane; i < kUniqSlots / 4; i += 32)
      reinterpret_cast<uint4*>(t)[i] = make_uint4(kEmpty32, kEmpty32, kEmpty32, kEmpty32);
    __syncwarp();
  }
}
static_assert(kUniqSlots == 1024, "the hash above takes 10 bits");

// The same for the runs run_unique_kernel leaves unmarked (kUniqSlots / 2 < length <=
// kUniqLongMax): one CTA per run with a table of 2 * kUniqLongMax keys in shared memory.
constexpr int kUniqLongThreads = 256;
constexpr uint32_t kUniqLongMax = 4096;
constexpr uint32_t kUniqLongSlots = 2 * kUniqLongMax;
__global__ void __launch_bounds__(kUniqLongThreads) run_unique_long_kernel(const uint32_t* __restrict__ yoff, u64 bins,
                                                                          const uint32_t* __restrict__ yfk,
                                                                          uint8_t* __restrict__ yuniq) {
  __shared__ __align__(16) uint32_t t[kUniqLongSlots];
  __shared__ int s_dup;
  for (uint32_t i = threadIdx.x; i < kUniqLongSlots / 4; i += kUniqLongThreads)
    reinterpret_cast<uint4*>(t)[i] = make_uint4(kEmpty32, kEmpty32, kEmpty32, kEmpty32);
  if (threadIdx.x == 0) s_dup = 0;
  __syncthreads();
  for (u64 b = blockIdx.x; b < bins; b += gridDim.x) {
    const uint32_t s0 = yoff[b], len = yoff[b + 1] - s0;
    if (len <= kUniqSlots / 2 || len > kUniqLongMax) continue;  // uniform over the CTA
    for (uint32_t j = threadIdx.x; j < len; j += kUniqLongThreads) {
      const uint32_t key = yfk[s0 + j];
      uint32_t h = (key * 0x9E3779B1u) >> 19;  // 13 bits: kUniqLongSlots slots
      for (uint32_t probe = 0; probe < kUniqLongSlots; probe++) {
        const uint32_t prev = atomicCAS(t + h, kEmpty32, key);
        if (prev == kEmpty32) break;
        if (prev == key) {
          s_dup = 1;
          break;
        }
        h = (h + 1) & (kUniqLongSlots - 1);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      yuniq[s0] = s_dup ? 0 : 1;
      s_dup = 0;
    }
    for (uint32_t i = threadIdx.x; i < kUniqLongSlots / 4; i += kUniqLongThreads)
      reinterpret_cast<uint4*>(t)[i] = make_uint4(kEmpty32, kEmpty32, kEmpty32, kEmpty32);
    __syncthreads();
  }
}
static_assert(kUniqLongSlots == 8192, "the hash above takes 13 bits");

// Survivors of all problems: their combined group key fxoff[p] + fX, Y run, value; the
// product count per problem and in total.
__global__ void __launch_bounds__(kThreads) x_survey_batch_kernel(const BatchProb* __restrict__ pb,
                                                                  const int64_t* __restrict__ xrow, int n,
                                                                  int64_t total, const uint32_t* __restrict__ yoff,
                                                                  Survivors sv, u64* __restrict__ P,
                                                                  u64* __restrict__ Pp, uint32_t* status) {
  for (int64_t base = (int64_t)blockIdx.x * kThreads + (threadIdx.x & ~31u); base < total;
       base += (int64_t)gridDim.x * kThreads) {
    const int64_t r = base + lane_id();
    bool live = false;
    u64 gkey = 0;
    uint32_t lo = 0, w = 0;
    int p = 0;
    if (r < total) {
      p = row_problem(xrow, n, r);
      const BatchProb& q = pb[p];
      uint64_t ck, fk;
      if (!row_keys_any(q.xc, r - xrow[p], q.kx, ck, fk)) {
        atomicOr(status, kStatCoordRange);
      } else {
        lo = __ldg(yoff + q.koff + ck);
        w = __ldg(yoff + q.koff + ck + 1) - lo;
        live = w > 0;
        gkey = q.fxoff + fk;
      }
    }
    const unsigned pos = warp_reserve<unsigned>(live, sv.count);
    if (live) {
      sv.fk[pos] = gkey;
      sv.ystart[pos] = lo;
      sv.w[pos] = w;
      sv.v[pos] = __ldg(pb[p].xv + (r - xrow[p]));
    }
    // Products per problem: rows are in problem order, so a warp spans few problems; one
    // atomic per (warp, problem).
    unsigned todo = __ballot_sync(0xffffffffu, live);
    while (todo) {
      const int leader = __ffs(todo) - 1;
      const int pl = __shfl_sync(0xffffffffu, p, leader);
      const bool mine = live && p == pl;
      u64 sum = mine ? (u64)w : 0ull;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      if ((int)lane_id() == leader) {
        atomicAdd(Pp + pl, sum);
        atomicAdd(P, sum);
      }
      todo &= ~__ballot_sync(0xffffffffu, mine);
    }
  }
}

// The small-number map (Section 4.1.2) on the GPU: every distinct group key claims a slot of
// a probing table, and a group's number is its slot. Numbers are then sparse in [0, table
// size) rather than dense in order of first sight (which would serialise on one counter);
// empty slots are empty groups and are skipped.
__global__ void __launch_bounds__(kThreads) idmap_insert_kernel(Survivors sv, IdMap m, uint32_t* status) {
  const int64_t ns = (int64_t)*sv.count;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < ns; i += (int64_t)gridDim.x * kThreads) {
    const u64 key = sv.fk[i];
    u64 slot = mix64(key) & m.mask;
    bool done = false;
    for (u64 probe = 0; probe <= m.mask; probe++) {
      u64 cur = __ldcg(m.keys + slot);
      if (cur == kEmpty64) {
        const u64 prev = atomicCAS(m.keys + slot, kEmpty64, key);
        cur = (prev == kEmpty64) ? key : prev;
      }
      if (cur == key) {
        done = true;
        break;
      }
      slot = (slot + 1) & m.mask;
    }
    if (!done) atomicOr(status, kStatTableFull);
  }
}

// Second pass (a separate launch, so the table is complete): each survivor finds its key's
// slot, which is its group number, and is counted in its group.
__global__ void __launch_bounds__(kThreads) idmap_lookup_kernel(Survivors sv, IdMap m, uint32_t* __restrict__ gid,
                                                                uint32_t* __restrict__ gcnt) {
  const int64_t ns = (int64_t)*sv.count;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < ns; i += (int64_t)gridDim.x * kThreads) {
    const u64 key = sv.fk[i];
    u64 slot = mix64(key) & m.mask;
    for (u64 probe = 0; probe <= m.mask; probe++) {
      if (__ldcg(m.keys + slot) == key) {
        gid[i] = (uint32_t)slot;
        atomicAdd(gcnt + slot, 1u);
        break;
      }
      slot = (slot + 1) & m.mask;
    }
  }
}

__global__ void __launch_bounds__(kThreads) batch_group_scatter_kernel(Survivors sv, const uint32_t* __restrict__ gid,
                                                                       uint32_t* __restrict__ gcur, GroupedX gx) {
  const int64_t ns = (int64_t)*sv.count;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < ns; i += (int64_t)gridDim.x * kThreads) {
    const uint32_t pos = atomicAdd(gcur + gid[i], 1u);
    gx.ystart[pos] = sv.ystart[i];
    gx.w[pos] = sv.w[i];
    gx.v[pos] = sv.v[i];
  }
}

// One thread per group: its bound (sum of its entries' run lengths; groups here are mostly a
// single X entry), its problem and X free key, its class. Appends to the class lists are
// aggregated per warp; each problem's output bound sums min(B_g, F_Y) over its groups.
__global__ void __launch_bounds__(kThreads) bin_batch_kernel(u64 G, const uint32_t* __restrict__ goff,
                                                             const uint32_t* __restrict__ gw,
                                                             const u64* __restrict__ gkey,
                                                             const u64* __restrict__ fxoff, int n,
                                                             const BatchProb* __restrict__ pb, Bins b,
                                                             uint32_t* __restrict__ gprob, u64* __restrict__ gfk,
                                                             u64* __restrict__ pcap) {
  __shared__ u64 s_cap[kThreads / 32];
  const unsigned lane = lane_id();
  u64 my_cap = 0;
  for (u64 base = (u64)blockIdx.x * kThreads + (threadIdx.x & ~31u); base < G; base += (u64)gridDim.x * kThreads) {
    const u64 g = base + lane;
    int cls = -1;
    int p = -1;
    u64 t = 0;
    if (g < G && goff[g] != goff[g + 1]) {
      u64 bnd = 0;
      for (uint32_t i = goff[g]; i < goff[g + 1]; i++) bnd += gw[i];
      const u64 key = gkey[g];
      p = key_problem(fxoff, n, key);
      gprob[g] = (uint32_t)p;
      gfk[g] = key - fxoff[p];
      const u64 FY = pb[p].FY;
      t = bnd < FY ? bnd : FY;
      my_cap += t;
      cls = 0;
      while (cls < b.nclasses && t > b.tmax[cls]) cls++;
      if (cls == b.nclasses && t > (1ull << 30)) {
        atomicOr(b.status, kStatTooLarge);
        cls = -1;
      }
    }
    for (int c = 0; c <= b.nclasses; c++) {
      const bool in = cls == c;
      const uint32_t pos = warp_reserve<uint32_t>(in, b.count + (c < b.nclasses ? c : kMaxClasses));
      if (in) {
        if (c < b.nclasses) {
          b.list[c][pos] = (uint32_t)g;
        } else {
          u64 cap = 64;
          while (cap < 2 * t) cap <<= 1;
          b.huge_list[pos] = (uint32_t)g;
          b.huge_off[pos] = atomicAdd(b.huge_slots, cap);
          b.huge_cap[pos] = cap;
        }
      }
    }
    // Output bound per problem, one atomic per (warp, problem).
    unsigned todo = __ballot_sync(0xffffffffu, p >= 0);
    while (todo) {
      const int leader = __ffs(todo) - 1;
      const int pl = __shfl_sync(0xffffffffu, p, leader);
      const bool mine = p == pl;
      u64 sum = mine ? t : 0ull;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      if ((int)lane == leader) atomicAdd(pcap + pl, sum);
      todo &= ~__ballot_sync(0xffffffffu, mine);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_cap += __shfl_down_sync(0xffffffffu, my_cap, o);
  if (lane == 0) s_cap[threadIdx.x >> 5] = my_cap;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 tot = 0;
    for (int w = 0; w < kThreads / 32; w++) tot += s_cap[w];
    if (tot) atomicAdd(b.out_cap, tot);
  }
}

// Output layout of a captured batch, on the device: every problem's output region is placed
// in the run's output block by an exclusive scan of the exact bounds (values first, then
// coordinates, 16-byte aligned), and the overflow groups' table is cleared. When the block
// or the table is too small for this run's bounds, nothing is placed (every capacity 0, no
// overflow group runs) and the status word says so; the host then runs the batch again with
// the sizes it reads back.
constexpr int kLayoutThreads = 1024;
__global__ void __launch_bounds__(kLayoutThreads) batch_layout_kernel(int n, const u64* __restrict__ pcap,
                                                                      const int32_t* __restrict__ oz,
                                                                      BatchOut* __restrict__ bo,
                                                                      const BatchLayoutArgs* __restrict__ args,
                                                                      u64* __restrict__ offs, const u64* huge_slots,
                                                                      uint32_t* huge_count, uint32_t* status) {
  __shared__ u64 s_tot[2][kLayoutThreads / 32 + 1];
  const int per = (n + kLayoutThreads - 1) / kLayoutThreads;
  const int i0 = (int)threadIdx.x * per, i1 = i0 + per < n ? i0 + per : n;
  u64 sv = 0, sc = 0;
  for (int i = i0; i < i1; i++) {
    sv += pcap[i];
    sc += pcap[i] * (u64)oz[i];
  }
  // Block exclusive scans of the two sums.
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  u64 xv = sv, xc = sc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u64 a = __shfl_up_sync(0xffffffffu, xv, o), c = __shfl_up_sync(0xffffffffu, xc, o);
    if ((int)lane >= o) xv += a, xc += c;
  }
  if (lane == 31) s_tot[0][warp] = xv, s_tot[1][warp] = xc;
  __syncthreads();
  if (threadIdx.x < 32) {
    constexpr int NW = kLayoutThreads / 32;
    u64 tv = (int)lane < NW ? s_tot[0][lane] : 0, tc = (int)lane < NW ? s_tot[1][lane] : 0;
    u64 iv = tv, ic = tc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u64 a = __shfl_up_sync(0xffffffffu, iv, o), c = __shfl_up_sync(0xffffffffu, ic, o);
      if ((int)lane >= o) iv += a, ic += c;
    }
    if ((int)lane < NW) s_tot[0][lane] = iv - tv, s_tot[1][lane] = ic - tc;
    if (lane == 31) s_tot[0][NW] = iv, s_tot[1][NW] = ic;
  }
  __syncthreads();
  constexpr int NW = kLayoutThreads / 32;
  const u64 tot_v = s_tot[0][NW], tot_c = s_tot[1][NW];
  const u64 vbytes = (tot_v * 8 + 15) & ~15ull;
  const bool fits = vbytes + tot_c * 4 <= args->out_bytes && *huge_slots <= args->huge_cap;
  u64 ov = s_tot[0][warp] + xv - sv, oc = s_tot[1][warp] + xc - sc;
  double* const vbase = reinterpret_cast<double*>(args->out);
  int32_t* const cbase = reinterpret_cast<int32_t*>(args->out + vbytes);
  for (int i = i0; i < i1; i++) {
    offs[i] = ov;
    offs[n + 1 + i] = oc;
    bo[i].out_cap = fits ? pcap[i] : 0;
    bo[i].vals = fits ? vbase + ov : nullptr;
    bo[i].coords = fits ? cbase + oc : nullptr;
    ov += pcap[i];
    oc += pcap[i] * (u64)oz[i];
  }
  if (threadIdx.x == 0) {
    offs[n] = tot_v;
    offs[2 * n + 1] = tot_c;
    if (!fits) {
      atomicOr(status, kStatOutOverflow);
      *huge_count = 0;
    }
  }
}

// Clears the slots the overflow groups' table uses in this run (after batch_layout_kernel,
// which leaves no overflow groups when the run's layout did not fit).
__global__ void __launch_bounds__(kThreads) batch_clear_huge_kernel(const BatchLayoutArgs* __restrict__ args,
                                                                    const u64* huge_slots,
                                                                    const uint32_t* huge_count) {
  if (*huge_count == 0) return;
  const u64 hs = *huge_slots < args->huge_cap ? *huge_slots : args->huge_cap;
  u64* const keys = args->huge_keys;
  double* const vals = args->huge_vals;
  for (u64 k = (u64)blockIdx.x * kThreads + threadIdx.x; k < hs; k += (u64)gridDim.x * kThreads) {
    keys[k] = kEmpty64;
    vals[k] = 0.0;
  }
}

}  // namespace

cudaError_t launch_batch_prepare(const BatchArgs& ba, int sms, cudaStream_t s) {
  if (ba.total_y > 0) {
    y_count_batch_kernel<<<grid_for(ba.total_y, sms), kThreads, 0, s>>>(ba.pb, ba.yrow, ba.n, ba.total_y, ba.ycnt,
                                                                       ba.status);
    note_launch();
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = scan_u32(ba.ycnt, ba.yoff, (int64_t)ba.bins, ba.scan_scratch32, s);
  if (e != cudaSuccess) return e;
  if (ba.bins) {
    e = cudaMemcpyAsync(ba.ycur, ba.yoff, ba.bins * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  if (ba.total_y > 0) {
    if (ba.key32) {
      y_scatter_batch_kernel<uint32_t><<<grid_for(ba.total_y, sms), kThreads, 0, s>>>(
          ba.pb, ba.yrow, ba.n, ba.total_y, ba.ycur, static_cast<uint32_t*>(ba.yfk), ba.yv);
      if (ba.yuniq && ba.bins) {
        const u64 want = (ba.bins + kUniqWarps - 1) / kUniqWarps, cap = (u64)sms * 8;
        run_unique_kernel<<<(unsigned)(want < cap ? want : cap), kUniqWarps * 32, 0, s>>>(
            ba.yoff, ba.bins, static_cast<const uint32_t*>(ba.yfk), ba.yuniq);
        const u64 lcap = (u64)sms * 4;
        run_unique_long_kernel<<<(unsigned)(ba.bins < lcap ? ba.bins : lcap), kUniqLongThreads, 0, s>>>(
            ba.yoff, ba.bins, static_cast<const uint32_t*>(ba.yfk), ba.yuniq);
        note_launch(2);
      }
    } else
      y_scatter_batch_kernel<u64><<<grid_for(ba.total_y, sms), kThreads, 0, s>>>(
          ba.pb, ba.yrow, ba.n, ba.total_y, ba.ycur, static_cast<u64*>(ba.yfk), ba.yv);
    note_launch();
  }
  if (ba.total_x > 0) {
    x_survey_batch_kernel<<<grid_for(ba.total_x, sms), kThreads, 0, s>>>(ba.pb, ba.xrow, ba.n, ba.total_x, ba.yoff,
                                                                        ba.sv, ba.P, ba.Pp, ba.status);
    note_launch();
    idmap_insert_kernel<<<grid_for(ba.total_x, sms), kThreads, 0, s>>>(ba.sv, ba.idmap, ba.status);
    idmap_lookup_kernel<<<grid_for(ba.total_x, sms), kThreads, 0, s>>>(ba.sv, ba.idmap, ba.gid, ba.gcnt);
    note_launch(2);
  }
  return cudaGetLastError();
}

cudaError_t launch_batch_group(const BatchArgs& ba, GroupedX gx, const Bins& b, uint32_t* gprob, u64* gfk,
                               int sms, cudaStream_t s) {
  const int64_t G = (int64_t)ba.idmap.mask + 1;
  cudaError_t e = scan_u32(ba.gcnt, ba.goff, G, ba.scan_scratch32, s);
  if (e != cudaSuccess) return e;
  if (ba.total_x <= 0) return cudaSuccess;
  e = cudaMemcpyAsync(ba.gcur, ba.goff, (size_t)G * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  batch_group_scatter_kernel<<<grid_for(ba.total_x, sms), kThreads, 0, s>>>(ba.sv, ba.gid, ba.gcur, gx);
  bin_batch_kernel<<<grid_for(G, sms), kThreads, 0, s>>>((u64)G, ba.goff, gx.w, ba.idmap.keys, ba.fxoff, ba.n, ba.pb,
                                                         b, gprob, gfk, ba.pcap);
  note_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_batch_layout(int n, const u64* pcap, const int32_t* oz, BatchOut* bo, const BatchLayoutArgs* args,
                                u64* offs, const u64* huge_slots, uint32_t* huge_count, uint32_t* status, int sms,
                                cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  batch_layout_kernel<<<1, kLayoutThreads, 0, s>>>(n, pcap, oz, bo, args, offs, huge_slots, huge_count, status);
  batch_clear_huge_kernel<<<(unsigned)sms * 8, kThreads, 0, s>>>(args, huge_slots, huge_count);
  note_launch(2);
  return cudaGetLastError();
}

}  // namespace stc
