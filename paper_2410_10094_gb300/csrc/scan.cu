// Device-wide exclusive prefix sums (tile reduce, recursive scan of tile sums, tile scan).
// Used for the cumulative-sum step of the counting sort (Section 4.1.1) and for the
// survivors' product prefix that drives the merge-path split.
#include "launch.h"

namespace stc {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;
constexpr int kWarps = kThreads / 32;

// Exclusive scan of one value per thread across the block; `total` receives the sum.
template <typename T>
__device__ T block_exclusive_scan(T v, T& total, T* warp_sums) {
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, x, o);
    if ((int)lane >= o) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T w = lane < (unsigned)kWarps ? warp_sums[lane] : T(0);
#pragma unroll
    for (int o = 1; o < kWarps; o <<= 1) {
      const T y = __shfl_up_sync(0xffffffffu, w, o);
      if ((int)lane >= o) w += y;
    }
    if (lane < (unsigned)kWarps) warp_sums[lane] = w;
  }
  __syncthreads();
  const T before = warp ? warp_sums[warp - 1] : T(0);
  total = warp_sums[kWarps - 1];
  __syncthreads();
  return before + x - v;
}

// With `dn` the scan's length is min(*dn, n), read on the device (n bounds it and sizes the
// grid); tiles past it sum to zero.
template <typename TI, typename TO>
__global__ void __launch_bounds__(kThreads) tile_sums_kernel(const TI* __restrict__ in, int64_t n,
                                                             TO* __restrict__ sums, const unsigned* dn) {
  if (dn && (int64_t)*dn < n) n = (int64_t)*dn;
  __shared__ TO warp_sums[kWarps];
  const int64_t base = (int64_t)blockIdx.x * kTile;
  if (base >= n) {  // a tile past the end (device-side length): its sum is zero
    if (threadIdx.x == 0) sums[blockIdx.x] = TO(0);
    return;
  }
  TO acc = 0;
#pragma unroll
  for (int k = 0; k < kItems; k++) {
    const int64_t i = base + k * kThreads + threadIdx.x;
    if (i < n) acc += (TO)in[i];
  }
  TO total;
  block_exclusive_scan<TO>(acc, total, warp_sums);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(kThreads) tile_scan_kernel(const TI* __restrict__ in, int64_t n,
                                                             TO* __restrict__ out,
                                                             const TO* __restrict__ tile_offsets, const unsigned* dn) {
  if (dn && (int64_t)*dn < n) n = (int64_t)*dn;
  // Padded so that thread t's run of kItems consecutive elements spreads over banks.
  __shared__ TO tile[kTile + kTile / 32];
  __shared__ TO warp_sums[kWarps];
  auto at = [](int e) { return e + (e >> 5); };
  const int64_t base = (int64_t)blockIdx.x * kTile;
  // A tile past the end writes nothing (the tile starting exactly at the end writes the total).
  if (base > n) return;
#pragma unroll
  for (int k = 0; k < kItems; k++) {
    const int e = k * kThreads + threadIdx.x;
    const int64_t i = base + e;
    tile[at(e)] = i < n ? (TO)in[i] : TO(0);
  }
  __syncthreads();
  TO loc[kItems];
  TO sum = 0;
#pragma unroll
  for (int k = 0; k < kItems; k++) {
    loc[k] = tile[at(threadIdx.x * kItems + k)];
    sum += loc[k];
  }
  TO total;
  const TO ex = block_exclusive_scan<TO>(sum, total, warp_sums);
  const TO off = tile_offsets ? tile_offsets[blockIdx.x] : TO(0);
  TO run = off + ex;
#pragma unroll
  for (int k = 0; k < kItems; k++) {
    tile[at(threadIdx.x * kItems + k)] = run;
    run += loc[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kItems; k++) {
    const int e = k * kThreads + threadIdx.x;
    const int64_t i = base + e;
    if (i < n) out[i] = tile[at(e)];
  }
  // The total goes after the last element, written by the tile that holds position n (the
  // last tile when n is one past its end).
  if (threadIdx.x == 0 && ((base <= n && n < base + kTile) || (blockIdx.x == gridDim.x - 1 && n >= base + kTile)))
    out[n] = off + total;
}

template <typename TI, typename TO>
cudaError_t exclusive_scan(const TI* in, TO* out, int64_t n, TO* scratch, cudaStream_t s,
                           const unsigned* dn = nullptr) {
  if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(TO), s);
  const int64_t nb = (n + kTile - 1) / kTile;
  if (nb == 1) {
    tile_scan_kernel<TI, TO><<<1, kThreads, 0, s>>>(in, n, out, nullptr, dn);
    note_launch();
    return cudaGetLastError();
  }
  TO* sums = scratch;
  TO* offs = scratch + nb;
  tile_sums_kernel<TI, TO><<<(unsigned)nb, kThreads, 0, s>>>(in, n, sums, dn);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = exclusive_scan<TO, TO>(sums, offs, nb, scratch + 2 * nb + 1, s);
  if (e != cudaSuccess) return e;
  tile_scan_kernel<TI, TO><<<(unsigned)nb, kThreads, 0, s>>>(in, n, out, offs, dn);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

namespace {
thread_local unsigned t_launches = 0;
}
void note_launch(unsigned n) { t_launches += n; }
unsigned take_launches() {
  const unsigned n = t_launches;
  t_launches = 0;
  return n;
}

int64_t scan_scratch_elems(int64_t n) {
  const int64_t nb = (n + kTile - 1) / kTile;
  if (nb <= 1) return 0;
  return 2 * nb + 1 + scan_scratch_elems(nb);
}

cudaError_t scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* scratch, cudaStream_t s) {
  return exclusive_scan<uint32_t, uint32_t>(in, out, n, scratch, s);
}
cudaError_t scan_u32_u64(const uint32_t* in, u64* out, int64_t n, u64* scratch, cudaStream_t s) {
  return exclusive_scan<uint32_t, u64>(in, out, n, scratch, s);
}
cudaError_t scan_u32_u64_dev(const uint32_t* in, u64* out, int64_t nmax, const unsigned* dn, u64* scratch,
                             cudaStream_t s) {
  return exclusive_scan<uint32_t, u64>(in, out, nmax, scratch, s, dn);
}
cudaError_t scan_u64(const u64* in, u64* out, int64_t n, u64* scratch, cudaStream_t s) {
  return exclusive_scan<u64, u64>(in, out, n, scratch, s);
}

}  // namespace stc
