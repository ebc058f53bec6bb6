// Input processing on the device: LN keys (Section 2.3.1), grouping of Y by contract key
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

template <int ORDER, bool VEC>
__global__ void __launch_bounds__(kThreads) y_count_kernel(const int32_t* __restrict__ coords, int64_t n, KeyPlan p,
                                                           uint32_t* __restrict__ cnt, uint32_t* status) {
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
      if (!ok[r]) atomicOr(status, kStatCoordRange);
      else if (ck[r] != kEmpty64) atomicAdd(cnt + ck[r] * p.nseg + (p.nseg > 1 ? (fk[r] >> p.seg_shift) : 0), 1u);
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
template <int ORDER, bool VEC>
__device__ __forceinline__ void rows_runs(const int32_t* __restrict__ coords, int64_t base, int64_t n,
                                          const KeyPlan& p, const uint32_t* __restrict__ yoff, uint64_t* fk,
                                          uint32_t* lo, uint32_t* w, uint32_t* status, uint64_t* ck) {
  bool ok[kRows];
#pragma unroll
  for (int r = 0; r < kRows; r++) {
    const int64_t i = base + lane_id() + 32 * r;
    ok[r] = false;
    if (i < n) {
      ok[r] = row_keys<ORDER, VEC>(coords, i, p, ck[r], fk[r]);
      if (!ok[r]) atomicOr(status, kStatCoordRange);
    }
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

template <int ORDER, bool VEC, bool GROUPS>
__global__ void __launch_bounds__(kThreads) x_survey_kernel(const int32_t* __restrict__ coords,
                                                            const double* __restrict__ vals, int64_t n, KeyPlan p,
                                                            const uint32_t* __restrict__ yoff, Survivors sv,
                                                            u64* __restrict__ P, uint32_t* __restrict__ gcnt,
                                                            uint32_t* status) {
  __shared__ u64 warp_p[kThreads / 32];
  u64 my_p = 0;
  STC_WARP_ROWS(base, n) {
    uint64_t fk[kRows], ck[kRows];
    uint32_t lo[kRows], w[kRows];
    rows_runs<ORDER, VEC>(coords, base, n, p, yoff, fk, lo, w, status, ck);
#pragma unroll
    for (int r = 0; r < kRows; r++) {
      const bool live = w[r] > 0;
      const unsigned pos = warp_reserve<unsigned>(live, sv.count);
      if (live) {
        const int64_t i = base + lane_id() + 32 * r;
        sv.fk[pos] = fk[r];
        if (sv.ck) sv.ck[pos] = (uint32_t)ck[r];
        sv.ystart[pos] = lo[r];
        sv.w[pos] = w[r];
        sv.v[pos] = __ldg(vals + i);
        my_p += w[r];
        if (GROUPS) atomicAdd(gcnt + fk[r], 1u);
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

// Dense X (most entries have a Y run): count entries per X free key and the products,
// without writing a survivor list.
template <int ORDER, bool VEC>
__global__ void __launch_bounds__(kThreads) x_count_kernel(const int32_t* __restrict__ coords, int64_t n, KeyPlan p,
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
__global__ void __launch_bounds__(kThreads) x_scatter_dense_kernel(const int32_t* __restrict__ coords,
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
                           int sms, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const unsigned g = grid_for((n + kRows - 1) / kRows, sms);
  return dispatch_order(p.order, vec_ok(coords, p.order), [&]<int O, bool V>() {
    y_count_kernel<O, V><<<g, kThreads, 0, s>>>(coords, n, p, cnt, status);
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
                            const uint32_t* yoff, Survivors sv, u64* P, uint32_t* gcnt, uint32_t* status, int sms,
                            cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const unsigned g = grid_for((n + kRows - 1) / kRows, sms);
  const bool groups = gcnt != nullptr;
  return dispatch_order(p.order, vec_ok(coords, p.order), [&]<int O, bool V>() {
    if (groups)
      x_survey_kernel<O, V, true><<<g, kThreads, 0, s>>>(coords, vals, n, p, yoff, sv, P, gcnt, status);
    else
      x_survey_kernel<O, V, false><<<g, kThreads, 0, s>>>(coords, vals, n, p, yoff, sv, P, gcnt, status);
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

}  // namespace stc
