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

template <int ORDER, bool VEC>
__global__ void __launch_bounds__(kThreads) y_count_kernel(const int32_t* __restrict__ coords, int64_t n, KeyPlan p,
                                                           uint32_t* __restrict__ cnt, uint32_t* status) {
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
    uint64_t ck, fk;
    if (!row_keys<ORDER, VEC>(coords, i, p, ck, fk)) {
      atomicOr(status, kStatCoordRange);
      continue;
    }
    atomicAdd(cnt + ck, 1u);
  }
}

template <int ORDER, bool VEC>
__global__ void __launch_bounds__(kThreads) y_scatter_kernel(const int32_t* __restrict__ coords,
                                                             const double* __restrict__ vals, int64_t n, KeyPlan p,
                                                             uint32_t* __restrict__ cursor, u64* __restrict__ yfk,
                                                             double* __restrict__ yv) {
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
    uint64_t ck, fk;
    if (!row_keys<ORDER, VEC>(coords, i, p, ck, fk)) continue;
    const uint32_t pos = atomicAdd(cursor + ck, 1u);
    yfk[pos] = fk;
    yv[pos] = __ldg(vals + i);
  }
}

template <int ORDER, bool VEC, bool GROUPS>
__global__ void __launch_bounds__(kThreads) x_survey_kernel(const int32_t* __restrict__ coords,
                                                            const double* __restrict__ vals, int64_t n, KeyPlan p,
                                                            const uint32_t* __restrict__ yoff, Survivors sv,
                                                            u64* __restrict__ P, uint32_t* __restrict__ gcnt,
                                                            u64* __restrict__ gbound, uint32_t* status) {
  __shared__ u64 warp_p[kThreads / 32];
  u64 my_p = 0;
  STC_WARP_LOOP(i, n) {
    bool live = false;
    uint64_t ck = 0, fk = 0;
    uint32_t lo = 0, w = 0;
    if (i < n) {
      if (!row_keys<ORDER, VEC>(coords, i, p, ck, fk)) {
        atomicOr(status, kStatCoordRange);
      } else {
        lo = __ldg(yoff + ck);
        w = __ldg(yoff + ck + 1) - lo;
        live = w > 0;
      }
    }
    const unsigned pos = warp_reserve<unsigned>(live, sv.count);
    if (live) {
      sv.fk[pos] = fk;
      sv.ystart[pos] = lo;
      sv.w[pos] = w;
      sv.v[pos] = __ldg(vals + i);
      my_p += w;
      if (GROUPS) {
        atomicAdd(gcnt + fk, 1u);
        atomicAdd(gbound + fk, (u64)w);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_p += __shfl_down_sync(0xffffffffu, my_p, o);
  if (lane_id() == 0) warp_p[threadIdx.x >> 5] = my_p;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 t = 0;
    for (int w = 0; w < kThreads / 32; w++) t += warp_p[w];
    if (t) atomicAdd(P, t);
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
  const unsigned g = grid_for(n, sms);
  return dispatch_order(p.order, vec_ok(coords, p.order), [&]<int O, bool V>() {
    y_count_kernel<O, V><<<g, kThreads, 0, s>>>(coords, n, p, cnt, status);
    note_launch();
    return cudaGetLastError();
  });
}

cudaError_t launch_y_scatter(const int32_t* coords, const double* vals, int64_t n, const KeyPlan& p,
                             uint32_t* cursor, u64* yfk, double* yv, int sms, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const unsigned g = grid_for(n, sms);
  return dispatch_order(p.order, vec_ok(coords, p.order), [&]<int O, bool V>() {
    y_scatter_kernel<O, V><<<g, kThreads, 0, s>>>(coords, vals, n, p, cursor, yfk, yv);
    note_launch();
    return cudaGetLastError();
  });
}

cudaError_t launch_x_survey(const int32_t* coords, const double* vals, int64_t n, const KeyPlan& p,
                            const uint32_t* yoff, Survivors sv, u64* P, uint32_t* gcnt, u64* gbound,
                            uint32_t* status, int sms, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const unsigned g = grid_for(n, sms);
  const bool groups = gcnt != nullptr;
  return dispatch_order(p.order, vec_ok(coords, p.order), [&]<int O, bool V>() {
    if (groups)
      x_survey_kernel<O, V, true><<<g, kThreads, 0, s>>>(coords, vals, n, p, yoff, sv, P, gcnt, gbound, status);
    else
      x_survey_kernel<O, V, false><<<g, kThreads, 0, s>>>(coords, vals, n, p, yoff, sv, P, gcnt, gbound, status);
    note_launch();
    return cudaGetLastError();
  });
}

}  // namespace stc
