// Dense ids for keys whose space is too large to count directly (Section 4.1.2, Fig. 7).
//
// The paper gives each distinct key the next unused small number while it scans the keys
// in order, so that a counting sort over the ids costs O(n). On the device the distinct
// keys are first collected in an open-addressing table (linear probing, load <= 1/2); the
// id of a key is then the number of occupied slots before its own slot, a prefix sum over
// the table. The ids are dense in [0, D) and equal keys share one id, which is all a
// grouping needs; which key receives which number differs from the sequential first-seen
// order. The all-ones key, which marks empty slots, is tracked by one extra flag placed
// after the last slot, so every 64-bit key is allowed.
#include "launch.h"

namespace stc {

namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(int64_t n, int sms, int per_sm = 8) {
  const int64_t want = (n + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)sms * per_sm;
  return (unsigned)(want < cap ? want : cap);
}

// Inserts key (not all-ones); false if the probe ran through the whole table.
__device__ __forceinline__ bool id_insert(u64* keys, u64 mask, u64 key) {
  u64 h = mix64(key) & mask;
  for (u64 probe = 0; probe <= mask; probe++) {
    const u64 cur = *reinterpret_cast<volatile u64*>(keys + h);
    if (cur == key) return true;
    if (cur == kEmpty64) {
      const u64 old = atomicCAS(keys + h, kEmpty64, key);
      if (old == kEmpty64 || old == key) return true;
    }
    h = (h + 1) & mask;
  }
  return false;
}

// Slot of key (not all-ones) in a table no longer written to, or -1 when it is absent.
__device__ __forceinline__ int64_t id_slot(const u64* __restrict__ keys, u64 mask, u64 key) {
  u64 h = mix64(key) & mask;
  for (u64 probe = 0; probe <= mask; probe++) {
    const u64 cur = __ldg(keys + h);
    if (cur == key) return (int64_t)h;
    if (cur == kEmpty64) return -1;
    h = (h + 1) & mask;
  }
  return -1;
}

// Id of key, or the count D of distinct keys when the table lacks it.
__device__ __forceinline__ uint32_t id_of(const IdTable& t, u64 key) {
  if (key == kEmpty64) return t.flags[t.slots] ? __ldg(t.prefix + t.slots) : __ldg(t.prefix + t.slots + 1);
  const int64_t h = id_slot(t.keys, t.slots - 1, key);
  return __ldg(t.prefix + (h >= 0 ? (u64)h : t.slots + 1));
}

// Contract key of coordinate row i (any order). False if a coordinate is outside its mode.
__device__ __forceinline__ bool row_ckey(const int32_t* __restrict__ coords, int64_t i, const KeyPlan& p, u64& ck) {
  bool ok = true;
  ck = 0;
  const int32_t* c = coords + i * p.order;
  for (int j = 0; j < p.order; j++) {
    const int32_t v = __ldg(c + j);
    ok &= (v >= 0) & ((int64_t)v < p.size[j]);
    ck += (u64)(uint32_t)v * p.cstride[j];
  }
  return ok;
}

__global__ void __launch_bounds__(kThreads) id_insert_keys_kernel(const u64* __restrict__ keys, int64_t n,
                                                                  IdTable t, uint32_t* status) {
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
    const u64 key = keys[i];
    if (key == kEmpty64)
      t.flags[t.slots] = 1u;
    else if (!id_insert(t.keys, t.slots - 1, key))
      atomicOr(status, kStatTableFull);
  }
}

__global__ void __launch_bounds__(kThreads) id_insert_rows_kernel(const int32_t* __restrict__ coords, int64_t n,
                                                                  KeyPlan p, IdTable t, uint32_t* status) {
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
    u64 ck;
    if (!row_ckey(coords, i, p, ck)) {
      atomicOr(status, kStatCoordRange);
      continue;
    }
    // A contract key is below K <= 2^64 - 1, so it is never the all-ones marker.
    if (!id_insert(t.keys, t.slots - 1, ck)) atomicOr(status, kStatTableFull);
  }
}

// flags[i] = 1 for an occupied slot; flags[slots] was set by the insert when it saw the
// all-ones key.
__global__ void __launch_bounds__(kThreads) id_flags_kernel(IdTable t) {
  for (u64 i = (u64)blockIdx.x * kThreads + threadIdx.x; i < t.slots; i += (u64)gridDim.x * kThreads)
    t.flags[i] = t.keys[i] != kEmpty64 ? 1u : 0u;
}

__global__ void __launch_bounds__(kThreads) id_lookup_keys_kernel(const u64* __restrict__ keys, int64_t n,
                                                                  IdTable t, uint32_t* __restrict__ ids) {
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
    ids[i] = id_of(t, keys[i]);
}

// Row i of out = (the free coordinates of row i in ascending mode order, the id of its
// contract key); rows whose key the table lacks get the id D.
__global__ void __launch_bounds__(kThreads) id_rewrite_rows_kernel(const int32_t* __restrict__ coords, int64_t n,
                                                                   KeyPlan p, uint32_t fmask, int nf, IdTable t,
                                                                   int32_t* __restrict__ out, uint32_t* status) {
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
    u64 ck;
    if (!row_ckey(coords, i, p, ck)) atomicOr(status, kStatCoordRange);
    int32_t* o = out + i * (int64_t)(nf + 1);
    int a = 0;
    for (int j = 0; j < p.order; j++)
      if ((fmask >> j) & 1u) o[a++] = __ldg(coords + i * p.order + j);
    o[nf] = (int32_t)id_of(t, ck);
  }
}

}  // namespace

uint64_t id_table_slots(int64_t n) {
  uint64_t s = 64;
  while (s < 2 * (uint64_t)(n > 0 ? n : 1)) s <<= 1;
  return s;
}

cudaError_t launch_id_insert_keys(const u64* keys, int64_t n, const IdTable& t, uint32_t* status, int sms,
                                  cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  id_insert_keys_kernel<<<grid_for(n, sms), kThreads, 0, s>>>(keys, n, t, status);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_id_insert_rows(const int32_t* coords, int64_t n, const KeyPlan& p, const IdTable& t,
                                  uint32_t* status, int sms, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  id_insert_rows_kernel<<<grid_for(n, sms), kThreads, 0, s>>>(coords, n, p, t, status);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_id_number(const IdTable& t, uint32_t* scratch, int sms, cudaStream_t s) {
  id_flags_kernel<<<grid_for((int64_t)t.slots, sms), kThreads, 0, s>>>(t);
  note_launch();
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return scan_u32(t.flags, t.prefix, (int64_t)t.slots + 1, scratch, s);
}

cudaError_t launch_id_lookup_keys(const u64* keys, int64_t n, const IdTable& t, uint32_t* ids, int sms,
                                  cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  id_lookup_keys_kernel<<<grid_for(n, sms), kThreads, 0, s>>>(keys, n, t, ids);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_id_rewrite_rows(const int32_t* coords, int64_t n, const KeyPlan& p, uint32_t fmask, int nf,
                                   const IdTable& t, int32_t* out, uint32_t* status, int sms, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  id_rewrite_rows_kernel<<<grid_for(n, sms), kThreads, 0, s>>>(coords, n, p, fmask, nf, t, out, status);
  note_launch();
  return cudaGetLastError();
}

}  // namespace stc
