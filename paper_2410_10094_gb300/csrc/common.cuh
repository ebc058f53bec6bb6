// Internal definitions shared by the library's CUDA translation units: key plans, status
// bits, hashing, warp helpers. Nothing here is part of the public ABI (include/stc.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "stc.h"

namespace stc {

constexpr int kMaxOrder = STC_MAX_ORDER;
constexpr int kMaxOutOrder = 2 * STC_MAX_ORDER;
constexpr uint64_t kEmpty64 = ~0ull;       // empty slot of a 64-bit-key table
constexpr uint32_t kEmpty32 = ~0u;         // empty slot of a 32-bit-key table
constexpr uint64_t kMaxDirectBins = 1ull << 26;  // largest key space grouped by direct counting

// Bits a kernel raises in the device status word; the host maps them to stc_status.
enum : uint32_t {
  kStatCoordRange = 1u,   // an input coordinate was out of range (entry skipped)
  kStatTableFull = 2u,    // a probe sequence ran through the whole table
  kStatOutOverflow = 4u,  // an output position past the allocated capacity (entry dropped)
  kStatTimeout = 8u,      // a bounded wait gave up
  kStatTooLarge = 16u,    // one group's table would exceed 2^31 slots
};

// How one input tensor's coordinates map to its two keys (Section 2.4.1, the LN key):
// ckey = sum_j coord[j] * cstride[j] (contract modes, in the order of the contract list),
// fkey = sum_j coord[j] * fstride[j] (free modes, ascending). A mode has a nonzero stride
// in exactly one of the two. size[] bounds-checks each coordinate.
//
// Y may be grouped by (contract key, free-key segment): with nseg > 1 the bin of a Y entry is
// ckey * nseg + (fkey >> seg_shift), and an X entry's runs are the nseg consecutive bins
// starting at ckey * nseg.
struct KeyPlan {
  int32_t order;
  uint32_t nseg;       // free-key segments per contract key (1 = plain grouping)
  uint32_t seg_shift;  // log2 of the segment width
  uint32_t pad_;
  int64_t size[kMaxOrder];
  uint64_t cstride[kMaxOrder];
  uint64_t fstride[kMaxOrder];
};

// How an output key zkey = fX * F_Y + fY decodes into output coordinates. zkey is a
// mixed-radix number whose digits, least significant first, are the output coordinates at
// positions dpos[0], dpos[1], ...; digit j has radix mod[dpos[j]]. When every length is a
// power of two, output mode q is simply (zkey >> shift[q]) & (mod[q] - 1). Otherwise the
// digits are peeled off by repeated division, each division by an invariant radix done with
// a multiply-high (Granlund and Montgomery, PLDI 1994, Section 4): with l = ceil(log2 d),
// m = floor(2^N (2^l - d) / d) + 1 and t = mulhi(m, n), n / d = (t + ((n - t) >> sh1)) >> sh2
// where sh1 = min(l, 1), sh2 = max(l - 1, 0), for every N-bit n. N = 32 when z32 (every
// output key below 2^32), else 64.
struct OutPlan {
  int32_t order;
  int32_t pow2;
  int32_t z32;
  int32_t ident;                 // output modes in concatenation order (no permutation)
  uint64_t mod[kMaxOutOrder];    // length of output mode q
  uint32_t shift[kMaxOutOrder];  // power-of-two plans: bit offset of output mode q
  uint64_t magic[kMaxOutOrder];  // multiplier m of digit j
  uint8_t dpos[kMaxOutOrder];    // output position of digit j
  uint8_t dsh1[kMaxOutOrder];
  uint8_t dsh2[kMaxOutOrder];
  uint8_t pad2_[kMaxOutOrder];
};

// MurmurHash3's 64-bit finaliser (fmix64, Austin Appleby, public domain): a bijective
// mixer, so distinct keys never share a home slot pattern by construction of the key.
__device__ __forceinline__ uint64_t mix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

// MurmurHash3's 32-bit finaliser (fmix32).
__device__ __forceinline__ uint32_t mix32(uint32_t k) {
  k ^= k >> 16;
  k *= 0x85ebca6bu;
  k ^= k >> 13;
  k *= 0xc2b2ae35u;
  k ^= k >> 16;
  return k;
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Contract and free keys of one coordinate row. Returns false if any coordinate is outside
// its mode.
template <int ORDER>
__device__ __forceinline__ bool keys_of(const int32_t* c, const KeyPlan& p, uint64_t& ck, uint64_t& fk) {
  bool ok = true;
  ck = 0;
  fk = 0;
#pragma unroll
  for (int j = 0; j < ORDER; j++) {
    ok &= (c[j] >= 0) & ((int64_t)c[j] < p.size[j]);
    ck += (uint64_t)(uint32_t)c[j] * p.cstride[j];
    fk += (uint64_t)(uint32_t)c[j] * p.fstride[j];
  }
  return ok;
}

// Reads coordinate row i of a [n][ORDER] int32 array and forms its contract and free
// keys. Returns false if any coordinate is outside its mode.
template <int ORDER, bool VEC>
__device__ __forceinline__ bool row_keys(const int32_t* __restrict__ coords, int64_t i,
                                         const KeyPlan& p, uint64_t& ck, uint64_t& fk) {
  int32_t c[ORDER > 0 ? ORDER : 1];
  if constexpr (ORDER == 4 && VEC) {
    const int4 v = __ldg(reinterpret_cast<const int4*>(coords) + i);
    c[0] = v.x; c[1] = v.y; c[2] = v.z; c[3] = v.w;
  } else if constexpr (ORDER == 2 && VEC) {
    const int2 v = __ldg(reinterpret_cast<const int2*>(coords) + i);
    c[0] = v.x; c[1] = v.y;
  } else {
#pragma unroll
    for (int j = 0; j < ORDER; j++) c[j] = __ldg(coords + i * ORDER + j);
  }
  return keys_of<ORDER>(c, p, ck, fk);
}

// Peels the digits of zkey off (least significant first) and hands each output coordinate
// to put(q, c). Used when the plan is not all powers of two.
template <typename Put>
__device__ __forceinline__ void decode_digits(uint64_t zkey, const OutPlan& op, Put&& put) {
  if (op.z32) {
    uint32_t z = (uint32_t)zkey;
#pragma unroll 1
    for (int j = 0; j < op.order; j++) {
      const uint32_t t = __umulhi(z, (uint32_t)op.magic[j]);
      const uint32_t q = (t + ((z - t) >> op.dsh1[j])) >> op.dsh2[j];
      const int p = op.dpos[j];
      put(p, (int32_t)(z - q * (uint32_t)op.mod[p]));
      z = q;
    }
  } else {
    uint64_t z = zkey;
#pragma unroll 1
    for (int j = 0; j < op.order; j++) {
      const uint64_t t = __umul64hi(z, op.magic[j]);
      const uint64_t q = (t + ((z - t) >> op.dsh1[j])) >> op.dsh2[j];
      const int p = op.dpos[j];
      put(p, (int32_t)(z - q * op.mod[p]));
      z = q;
    }
  }
}

// Output coordinate q of an output key (power-of-two plans).
__device__ __forceinline__ int32_t out_coord_pow2(uint64_t zkey, const OutPlan& op, int q) {
  return (int32_t)((zkey >> op.shift[q]) & (op.mod[q] - 1));
}

// Writes the output coordinates of zkey to dst[0..order).
__device__ __forceinline__ void store_coords(uint64_t zkey, const OutPlan& op, int32_t* __restrict__ dst) {
  if (op.order == 4 && op.pow2 && ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0)) {
    int4 v;
    v.x = (int32_t)((zkey >> op.shift[0]) & (op.mod[0] - 1));
    v.y = (int32_t)((zkey >> op.shift[1]) & (op.mod[1] - 1));
    v.z = (int32_t)((zkey >> op.shift[2]) & (op.mod[2] - 1));
    v.w = (int32_t)((zkey >> op.shift[3]) & (op.mod[3] - 1));
    *reinterpret_cast<int4*>(dst) = v;
    return;
  }
  if (op.pow2) {
#pragma unroll 1
    for (int q = 0; q < op.order; q++) dst[q] = out_coord_pow2(zkey, op, q);
    return;
  }
  decode_digits(zkey, op, [&](int q, int32_t c) { dst[q] = c; });
}

// L2 cache policies (PTX createpolicy): data read again soon (Y runs) is kept with
// evict_last; output written once is streamed with evict_first.
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint32_t ld_keep_u32(const uint32_t* ptr, uint64_t pol) {
  uint32_t v;
  asm volatile("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(ptr), "l"(pol));
  return v;
}
__device__ __forceinline__ uint64_t ld_keep_u64(const uint64_t* ptr, uint64_t pol) {
  uint64_t v;
  asm volatile("ld.global.nc.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(ptr), "l"(pol));
  return v;
}
__device__ __forceinline__ double ld_keep_f64(const double* ptr, uint64_t pol) {
  double v;
  asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(ptr), "l"(pol));
  return v;
}
__device__ __forceinline__ void st_stream_v4(int32_t* ptr, int4 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.s32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(ptr), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void st_stream_s32(int32_t* ptr, int32_t v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.s32 [%0], %1, %2;" ::"l"(ptr), "r"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_stream_f64(double* ptr, double v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(ptr), "d"(v), "l"(pol) : "memory");
}

// Output rows of O coordinates in concatenation order, not all lengths powers of two: the
// digits are decoded into registers (digit j is coordinate O-1-j) and stored in pairs with
// 8-byte stores where the row allows.
template <int O>
__device__ __forceinline__ void store_row_fixed(int32_t* __restrict__ dst, uint64_t zkey, const OutPlan& op,
                                                uint64_t pol) {
  int32_t c[O];
  if (op.z32) {
    uint32_t z = (uint32_t)zkey;
#pragma unroll
    for (int j = 0; j < O; j++) {
      const uint32_t t = __umulhi(z, (uint32_t)op.magic[j]);
      const uint32_t q = (t + ((z - t) >> op.dsh1[j])) >> op.dsh2[j];
      c[O - 1 - j] = (int32_t)(z - q * (uint32_t)op.mod[O - 1 - j]);
      z = q;
    }
  } else {
    uint64_t z = zkey;
#pragma unroll
    for (int j = 0; j < O; j++) {
      const uint64_t t = __umul64hi(z, op.magic[j]);
      const uint64_t q = (t + ((z - t) >> op.dsh1[j])) >> op.dsh2[j];
      c[O - 1 - j] = (int32_t)(z - q * op.mod[O - 1 - j]);
      z = q;
    }
  }
  const int first = (reinterpret_cast<uintptr_t>(dst) & 7u) ? 1 : 0;  // 0 or 1 single store first
  if (first) st_stream_s32(dst, c[0], pol);
#pragma unroll
  for (int k = 0; k < O; k++) {
    if (k < first || ((k - first) & 1)) continue;
    if (k + 1 < O) {
      asm volatile("st.global.L2::cache_hint.v2.s32 [%0], {%1, %2}, %3;" ::"l"(dst + k), "r"(c[k]), "r"(c[k + 1]),
                   "l"(pol)
                   : "memory");
    } else {
      st_stream_s32(dst + k, c[k], pol);
    }
  }
}

// Writes output entry `pos` (coordinates decoded from zkey, and its value) with streaming stores.
// FIXED = false leaves out the register-decoded rows of store_row_fixed (a smaller body for
// kernels whose hot path is the power-of-two one).
template <bool FIXED = true>
__device__ __forceinline__ void store_output(int32_t* __restrict__ coords, double* __restrict__ vals, unsigned long long pos,
                                             uint64_t zkey, double v, const OutPlan& op, uint64_t pol) {
  int32_t* dst = coords + pos * (uint64_t)op.order;
  if (op.order == 4 && op.pow2 && ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0)) {
    int4 cv;
    cv.x = (int32_t)((zkey >> op.shift[0]) & (op.mod[0] - 1));
    cv.y = (int32_t)((zkey >> op.shift[1]) & (op.mod[1] - 1));
    cv.z = (int32_t)((zkey >> op.shift[2]) & (op.mod[2] - 1));
    cv.w = (int32_t)((zkey >> op.shift[3]) & (op.mod[3] - 1));
    st_stream_v4(dst, cv, pol);
  } else if (op.pow2) {
    for (int q = 0; q < op.order; q++) st_stream_s32(dst + q, out_coord_pow2(zkey, op, q), pol);
  } else if (FIXED && op.ident && op.order >= 2 && op.order <= 8) {
    switch (op.order) {
      case 2: store_row_fixed<2>(dst, zkey, op, pol); break;
      case 3: store_row_fixed<3>(dst, zkey, op, pol); break;
      case 4: store_row_fixed<4>(dst, zkey, op, pol); break;
      case 5: store_row_fixed<5>(dst, zkey, op, pol); break;
      case 6: store_row_fixed<6>(dst, zkey, op, pol); break;
      case 7: store_row_fixed<7>(dst, zkey, op, pol); break;
      default: store_row_fixed<8>(dst, zkey, op, pol); break;
    }
  } else {
    decode_digits(zkey, op, [&](int q, int32_t c) { st_stream_s32(dst + q, c, pol); });
  }
  st_stream_f64(vals + pos, v, pol);
}

// ---- asynchronous bulk copies (the TMA engine's untiled form) into shared memory, completed
// on an mbarrier. All addresses are 16-byte aligned and sizes multiples of 16 bytes.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// Makes barrier initialisation visible to the asynchronous (bulk copy) proxy.
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// One try of a wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Bounded wait: gives up after about `limit` tries (each try itself suspends for a while)
// and returns false, so that a copy that never lands cannot hang the kernel.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit = 1u << 24) {
  for (uint32_t i = 0; i < limit; i++)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// Copies `bytes` from global memory to shared memory; completion is counted on `bar`.
__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst_smem)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Warp-aggregated reservation of `pred ? 1 : 0` slots from a global counter. All 32 lanes
// must call it together. Returns this lane's position (meaningful only where pred).
template <typename T>
__device__ __forceinline__ T warp_reserve(bool pred, T* counter) {
  const unsigned mask = __ballot_sync(0xffffffffu, pred);
  T base = 0;
  if (mask) {
    const int leader = __ffs(mask) - 1;
    if ((int)lane_id() == leader) base = atomicAdd(counter, (T)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
  }
  return base + (T)__popc(mask & lanemask_lt());
}

}  // namespace stc
