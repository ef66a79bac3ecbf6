// Shared device-side definitions of the HISA engine (sm_103a).
//
// Tuples of a binary relation are stored as packed codes
//     code = (inst << 2b) | (c0 << b) | c1
// in the column order of the index (Section 4.2: the join column first, then
// the others), where b is the bit width of the active domain and inst is the
// instance id of a batched run (0 otherwise).  Sorting codes as unsigned
// integers is the lexicographic order of Section 4.2; the join key of an index
// is code >> b.  Codes are 32-bit when inst_bits + 2b <= 32, else 64-bit.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hisa {

// ---- device-resident control block ---------------------------------------------------

enum : int { kMaxBufs = 160, kMaxCnts = 160 };

// Device error codes (DevState::error).
enum : uint32_t {
  kDevOk = 0,
  kDevTimeout = 1,      // a bounded wait on another tile ran out
  kDevProbeLimit = 2,   // hash probe sequence exceeded the table size
  kDevBadState = 3,
};

struct DBuf {
  void* ptr;
  uint64_t cap;  // capacity in elements
};

// Everything a kernel needs that changes between iterations lives here, so a
// captured launch sequence stays valid while buffers swap and grow.
struct DevState {
  DBuf buf[kMaxBufs];
  uint64_t cnt[kMaxCnts];
  uint64_t need[kMaxBufs];     // required capacity when a stage overflowed
  uint32_t overflow;           // bit s set: stage s must be re-run after regrow
  uint32_t error;              // kDev* code
  uint32_t epoch;              // tag of the current look-back chain
  uint32_t go;                 // fixpoint loop condition
  uint32_t iter;               // iterations committed
  uint32_t max_iters;
  uint32_t tile_ctr[16];       // per-kernel tile counters (reset by ctrl kernels)
  uint64_t aux[16];
};

// ---- look-back status words: [63:44] epoch | [43:42] flag | [41:0] value --------------

enum : uint64_t { kFlagAgg = 1, kFlagIncl = 2 };
__device__ __forceinline__ uint64_t lb_pack(uint32_t epoch, uint64_t flag, uint64_t v) {
  return (uint64_t(epoch & 0xFFFFF) << 44) | (flag << 42) | (v & ((1ull << 42) - 1));
}
__device__ __forceinline__ uint64_t lb_flag(uint64_t w, uint32_t epoch) {
  return (uint32_t(w >> 44) == (epoch & 0xFFFFF)) ? ((w >> 42) & 3) : 0;
}
__device__ __forceinline__ uint64_t lb_value(uint64_t w) { return w & ((1ull << 42) - 1); }

// A look-back word carries its value, flag and epoch in one 64-bit word and no
// other data depends on it, so single-copy-atomic relaxed accesses suffice (no
// fence per publish).
__device__ __forceinline__ void st_release(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_acquire(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Polls allowed while waiting on a predecessor tile before the kernel gives up,
// records kDevTimeout and continues with a zero contribution (results are then
// invalid and the host reports HISA_ERR_DEVICE_TIMEOUT).  The look-back
// routines take the limit as an argument (this value by default), so that a
// check can make a wait run out after a few polls.
constexpr uint32_t kSpinLimit = 1u << 22;

// Warp-cooperative decoupled look-back (Merrill & Garland, "Single-pass
// parallel prefix scan with decoupled look-back", 2016).  Called by one full
// warp; returns the exclusive prefix of `tile` and publishes its inclusive one.
__device__ __forceinline__ uint64_t lookback_warp(uint64_t* status, uint64_t tile, uint64_t local,
                                                  uint32_t epoch, uint32_t* err, uint32_t spin_limit = kSpinLimit) {
  const int lane = threadIdx.x & 31;
  if (tile == 0) {
    if (lane == 0) st_release(&status[0], lb_pack(epoch, kFlagIncl, local));
    return 0;
  }
  if (lane == 0) st_release(&status[tile], lb_pack(epoch, kFlagAgg, local));
  uint64_t excl = 0;
  int64_t pos = int64_t(tile) - 1;
  uint32_t spins = 0;
  while (true) {
    const int64_t j = pos - lane;
    uint64_t w = 0, f = kFlagIncl, v = 0;
    if (j >= 0) {
      w = ld_acquire(&status[j]);
      f = lb_flag(w, epoch);
      v = lb_value(w);
    }
    if (__any_sync(0xffffffffu, f == 0)) {
      if (++spins > spin_limit) {
        if (lane == 0) atomicExch(err, kDevTimeout);
        break;
      }
      __nanosleep(64);
      continue;
    }
    const uint32_t incl = __ballot_sync(0xffffffffu, f == kFlagIncl);
    const int stop = incl ? __ffs(incl) - 1 : 31;   // closest inclusive predecessor
    uint64_t part = (lane <= stop) ? v : 0;
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    excl += part;
    if (incl) break;
    pos -= 32;
  }
  if (lane == 0) st_release(&status[tile], lb_pack(epoch, kFlagIncl, excl + local));
  return excl;
}

// Split form of the per-digit look-back: publish the tile's aggregate as soon
// as it is known, resolve the prefix later.
__device__ __forceinline__ void lookback_publish(uint64_t* status, uint64_t tile, uint64_t stride, uint64_t local,
                                                 uint32_t epoch) {
  st_release(&status[tile * stride], lb_pack(epoch, tile == 0 ? kFlagIncl : kFlagAgg, local));
}
__device__ __forceinline__ uint64_t lookback_resolve(uint64_t* status, uint64_t tile, uint64_t stride, uint64_t local,
                                                     uint32_t epoch, uint32_t* err, uint32_t spin_limit = kSpinLimit);

// Single-thread look-back for per-digit chains (radix sort: one thread per
// digit).  Eight predecessor words are read per round trip, so a walk over
// tiles that only published their aggregate costs 1/8 of the latency.
constexpr int kLookbackBatch = 8;
__device__ __forceinline__ uint64_t lookback_thread(uint64_t* status, uint64_t tile, uint64_t stride,
                                                    uint64_t local, uint32_t epoch, uint32_t* err,
                                                    uint32_t spin_limit = kSpinLimit) {
  if (tile == 0) {
    st_release(&status[0], lb_pack(epoch, kFlagIncl, local));
    return 0;
  }
  st_release(&status[tile * stride], lb_pack(epoch, kFlagAgg, local));
  uint64_t excl = 0;
  int64_t j = int64_t(tile) - 1;
  uint32_t spins = 0;
  while (true) {
    uint64_t w[kLookbackBatch];
#pragma unroll
    for (int b = 0; b < kLookbackBatch; ++b)
      w[b] = (j - b >= 0) ? ld_acquire(&status[uint64_t(j - b) * stride]) : lb_pack(epoch, kFlagIncl, 0);
    int used = 0;
    bool done = false;
#pragma unroll
    for (int b = 0; b < kLookbackBatch; ++b) {
      if (done || used < b) break;           // stopped earlier in this batch
      const uint64_t f = lb_flag(w[b], epoch);
      if (f == 0) break;                     // not published yet: re-read from here
      excl += lb_value(w[b]);
      ++used;
      if (f == kFlagIncl) done = true;
    }
    if (done) break;
    j -= used;
    if (used == 0) {
      if (++spins > spin_limit) {
        atomicExch(err, kDevTimeout);
        break;
      }
      __nanosleep(32);
    }
  }
  st_release(&status[tile * stride], lb_pack(epoch, kFlagIncl, excl + local));
  return excl;
}

__device__ __forceinline__ uint64_t lookback_resolve(uint64_t* status, uint64_t tile, uint64_t stride, uint64_t local,
                                                     uint32_t epoch, uint32_t* err, uint32_t spin_limit) {
  if (tile == 0) return 0;
  uint64_t excl = 0;
  int64_t j = int64_t(tile) - 1;
  uint32_t spins = 0;
  while (true) {
    uint64_t w[kLookbackBatch];
#pragma unroll
    for (int b = 0; b < kLookbackBatch; ++b)
      w[b] = (j - b >= 0) ? ld_acquire(&status[uint64_t(j - b) * stride]) : lb_pack(epoch, kFlagIncl, 0);
    int used = 0;
    bool done = false;
#pragma unroll
    for (int b = 0; b < kLookbackBatch; ++b) {
      if (done || used < b) break;
      const uint64_t f = lb_flag(w[b], epoch);
      if (f == 0) break;
      excl += lb_value(w[b]);
      ++used;
      if (f == kFlagIncl) done = true;
    }
    if (done) break;
    j -= used;
    if (used == 0) {
      if (++spins > spin_limit) {
        atomicExch(err, kDevTimeout);
        break;
      }
      __nanosleep(32);
    }
  }
  st_release(&status[tile * stride], lb_pack(epoch, kFlagIncl, excl + local));
  return excl;
}

// ---- small helpers --------------------------------------------------------------------

__host__ __device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  // MurmurHash3 finaliser (Appleby): full avalanche of a 32-bit key.
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

// Exclusive sum in place over v[0, n) by one CTA (blockDim.x a multiple of
// 32, at most 1024); returns the total to every thread.  Each warp takes a
// contiguous range, read coalesced with kB loads in flight per lane: the
// pass over HBM/L2 is bound by bandwidth, not by one load's latency per
// chunk.  smem holds >= 33 entries.
__device__ __forceinline__ uint64_t cta_scan_inplace(uint64_t* v, uint64_t n, uint64_t* smem) {
  constexpr int kB = 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint64_t wper = (((n + nw - 1) / nw) + 31) & ~31ull;
  const uint64_t w0 = min(n, uint64_t(warp) * wper), w1 = min(n, w0 + wper);
  uint64_t sum = 0;
  for (uint64_t base = w0; base < w1; base += 32 * kB) {
    uint64_t x[kB];
#pragma unroll
    for (int i = 0; i < kB; ++i) {
      const uint64_t g = base + uint64_t(i) * 32 + lane;
      x[i] = g < w1 ? v[g] : 0;
    }
#pragma unroll
    for (int i = 0; i < kB; ++i) sum += x[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane == 0) smem[warp] = sum;
  __syncthreads();
  if (warp == 0) {
    const uint64_t x0 = lane < nw ? smem[lane] : 0;
    uint64_t x = x0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    smem[lane] = x - x0;
    if (lane == 31) smem[32] = x;
  }
  __syncthreads();
  uint64_t carry = smem[warp];
  for (uint64_t base = w0; base < w1; base += 32 * kB) {
    uint64_t x[kB];
#pragma unroll
    for (int i = 0; i < kB; ++i) {
      const uint64_t g = base + uint64_t(i) * 32 + lane;
      x[i] = g < w1 ? v[g] : 0;
    }
#pragma unroll
    for (int i = 0; i < kB; ++i) {
      uint64_t incl = x[i];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const uint64_t g = base + uint64_t(i) * 32 + lane;
      if (g < w1) v[g] = carry + incl - x[i];
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  const uint64_t total = smem[32];
  __syncthreads();   // smem may be reused after return
  return total;
}

template <typename T>
__device__ __forceinline__ T block_exclusive_sum(T v, T* smem_warp, T* total) {
  // Exclusive sum over the block; smem_warp holds >= 32 entries.
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = (blockDim.x + 31) >> 5;
  T x = v;
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T w = lane < nwarps ? smem_warp[lane] : T(0);
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nwarps) smem_warp[lane] = w;  // inclusive warp prefix
  }
  __syncthreads();
  const T warp_excl = warp ? smem_warp[warp - 1] : T(0);
  if (total) *total = smem_warp[nwarps - 1];
  __syncthreads();
  return warp_excl + x - v;
}

template <typename K>
struct KeyTraits;
template <>
struct KeyTraits<uint32_t> { static constexpr int bits = 32; };
template <>
struct KeyTraits<uint64_t> { static constexpr int bits = 64; };

}  // namespace hisa
