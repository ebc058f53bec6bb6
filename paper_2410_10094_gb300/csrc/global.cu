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

// Each CTA takes tiles of kExTile consecutive products. Products are numbered by the
// survivors' exclusive prefix `wpre`: survivor s owns products [wpre[s], wpre[s+1]), its
// r-th product pairs it with slot ystart[s] + r of its Y run. Within a tile, thread t
// handles products t, t+256, ...; consecutive threads read consecutive Y slots.
// With dP / dns non-null, P and the survivor count are read on the device (the grid then is a
// persistent one sized by the host without them).
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
    for (u64 g = p0 + threadIdx.x; g < p1; g += kExThreads) {
      int a = 0, b = n - 1;
      while (a < b) {
        const int mid = (a + b + 1) >> 1;
        if (s_pre[mid] <= g) a = mid; else b = mid - 1;
      }
      const int64_t s = lo + a;
      const u64 j = (u64)__ldg(systart + s) + (g - s_pre[a]);
      const u64 key = __ldg(sfk + s) * FY + __ldg(yfk + j);
      const double prod = __dmul_rn(__ldg(sv + s), __ldg(yv + j));
      table_add(t.keys, t.vals, t.mask, key, prod, status);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kCpThreads) compact_global_kernel(GlobalTable t, OutPlan op,
                                                                    int32_t* __restrict__ coords,
                                                                    double* __restrict__ vals, u64 out_cap,
                                                                    u64* __restrict__ nz, uint32_t* status) {
  const int64_t cap = (int64_t)t.mask + 1;
  for (int64_t base = (int64_t)blockIdx.x * kCpThreads + (threadIdx.x & ~31u); base < cap;
       base += (int64_t)gridDim.x * kCpThreads) {
    const int64_t i = base + lane_id();
    const u64 k = i < cap ? __ldcs(t.keys + i) : kEmpty64;
    const bool live = k != kEmpty64;
    const u64 pos = warp_reserve<u64>(live, nz);
    if (live) {
      if (pos < out_cap) {
        store_coords(k, op, coords + pos * (u64)op.order);
        vals[pos] = __ldcs(t.vals + i);
      } else {
        atomicOr(status, kStatOutOverflow);
      }
    }
  }
}

}  // namespace

cudaError_t launch_expand_global(const u64* wpre, int64_t ns, u64 P, Survivors sv, const u64* yfk, const double* yv,
                                 u64 FY, GlobalTable t, uint32_t* status, int sms, cudaStream_t s) {
  if (P == 0 || ns <= 0) return cudaSuccess;
  const u64 ntiles = (P + kExTile - 1) / kExTile;
  const u64 cap = (u64)sms * 8;
  const unsigned g = (unsigned)(ntiles < cap ? ntiles : cap);
  expand_global_kernel<<<g, kExThreads, 0, s>>>(wpre, ns, P, sv.fk, sv.ystart, sv.v, yfk, yv, FY, t, status, nullptr,
                                                nullptr);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_expand_global_dev(const u64* wpre, const unsigned* dns, const u64* dP, Survivors sv, const u64* yfk,
                                     const double* yv, u64 FY, GlobalTable t, uint32_t* status, int sms,
                                     cudaStream_t s) {
  expand_global_kernel<<<(unsigned)sms * 8, kExThreads, 0, s>>>(wpre, 0, 0, sv.fk, sv.ystart, sv.v, yfk, yv, FY, t,
                                                                status, dP, dns);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_compact_global(GlobalTable t, const OutPlan& op, int32_t* coords, double* vals, u64 out_cap,
                                  u64* nz, uint32_t* status, int sms, cudaStream_t s) {
  const u64 cap = t.mask + 1;
  const u64 want = (cap + kCpThreads - 1) / kCpThreads;
  const u64 lim = (u64)sms * 8;
  compact_global_kernel<<<(unsigned)(want < lim ? want : lim), kCpThreads, 0, s>>>(t, op, coords, vals, out_cap, nz,
                                                                                  status);
  note_launch();
  return cudaGetLastError();
}

}  // namespace stc
