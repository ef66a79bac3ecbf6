// LSD radix sort of packed tuple codes (Section 4.2 "Construction": the sorted
// index is built by a least-significant-first sort; here one 8-bit digit per
// pass over the packed code instead of one stable sort per column).
//
// One pass is a single "onesweep" kernel (Adinets & Merrill, "Onesweep: a
// faster least significant digit radix sort for GPUs", 2022): each CTA takes
// the next tile of keys, ranks them stably inside the tile (a warp finds the
// lanes that hold the same digit through a word per digit in shared memory,
// one atomic OR per key; one digit counter set per warp), learns the tile's
// global offset per digit by decoupled look-back over the previous tiles,
// stages the tile in shared memory in digit order and writes it out.  The digit histograms of all passes
// come from one earlier read (or are fused into the kernel that produced the
// keys), so a pass reads and writes every key exactly once.
#pragma once
#include "common.cuh"

namespace hisa {

constexpr int kRadixBits = 8;
constexpr int kRadixDigits = 1 << kRadixBits;
constexpr int kRadixThreads = 256;   // one thread per digit in the per-tile scans
constexpr int kRadixWarps = kRadixThreads / 32;

// Keys per thread of a tile: a default and a smaller alternative per code
// width (the tile is chosen per context, hisa_config.radix_items); status
// buffers are sized for the smaller tile, so either fits.
template <typename K>
struct RadixCfg;
template <>
struct RadixCfg<uint32_t> { static constexpr int items = 24, items_alt = 16; };
template <>
struct RadixCfg<uint64_t> { static constexpr int items = 12, items_alt = 8; };

template <typename K>
__host__ __device__ constexpr int radix_tile() { return kRadixThreads * RadixCfg<K>::items_alt; }

// Dynamic shared memory of one pass: two tile buffers (the one being ranked,
// which then holds the tile in digit order, and the next tile's TMA target).
template <typename K, int ITEMS>
__host__ __device__ constexpr int radix_dyn_smem() { return 2 * kRadixThreads * ITEMS * int(sizeof(K)); }

struct RadixPassArgs {
  DevState* st;
  int in_buf, out_buf;   // key buffers (slots)
  int n_cnt;             // cnt slot holding the number of keys
  int hist_buf;          // u64 [passes][256] digit histograms
  int status_buf;        // u64 [tiles][256] look-back words
  int pass;              // pass index (histogram row)
  int shift;             // bit offset of this pass's digit
  int ctr;               // tile counter index
  int skip_mask;         // st->overflow bits that cancel this launch
  int stage_bit;         // overflow bit raised when a buffer is too small
  int items = 0;         // keys per thread (0: RadixCfg<K>::items; else items or items_alt)
};

// Digit histograms of all passes in one read of the keys.
struct RadixHistArgs {
  DevState* st;
  int in_buf, n_cnt, hist_buf;
  int passes;
  int skip_mask;
};

template <typename K>
__global__ void __launch_bounds__(256) k_radix_hist(RadixHistArgs a) {
  __shared__ uint32_t h[8][kRadixDigits];
  DevState* st = a.st;
  if (st->overflow & a.skip_mask) return;
  const K* in = static_cast<const K*>(st->buf[a.in_buf].ptr);
  const uint64_t n = st->cnt[a.n_cnt];
  for (int i = threadIdx.x; i < a.passes * kRadixDigits; i += blockDim.x) (&h[0][0])[i] = 0;
  __syncthreads();
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
    const K k = in[i];
    for (int p = 0; p < a.passes; ++p) atomicAdd(&h[p][(k >> (p * kRadixBits)) & 0xFF], 1u);
  }
  __syncthreads();
  unsigned long long* g = static_cast<unsigned long long*>(st->buf[a.hist_buf].ptr);
  for (int i = threadIdx.x; i < a.passes * kRadixDigits; i += blockDim.x) {
    const uint32_t v = (&h[0][0])[i];
    if (v) atomicAdd(&g[i], (unsigned long long)v);
  }
}

// ---- mbarrier / bulk-copy helpers (sm_90+ PTX) --------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ void mbar_init(uint64_t* m, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* m, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(smem_u32(m)), "r"(parity)
      : "memory");
  return ok != 0;
}
// 1-D bulk copy global -> shared (TMA engine); both addresses 16-byte aligned,
// size a multiple of 16; completion is signalled on the mbarrier.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* m) {
  asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(m))
               : "memory");
}
// Bounded wait for the mbarrier phase `parity`; false if the limit ran out.
constexpr uint32_t kMbarWaitLimit = 1u << 26;
__device__ __forceinline__ bool mbar_wait(uint64_t* m, uint32_t parity, uint32_t limit = kMbarWaitLimit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(m, parity)) return true;
  return false;
}

// One LSD pass.  Per tile: (1) the keys arrive in shared memory (bulk copy
// issued one tile ahead, so a CTA's next tile loads while it ranks the
// current one); (2) per-warp digit counts by shared atomics; (3) the tile's
// per-digit counts are published for the look-back at once, before ranking,
// so successors rarely wait; (4) stable ranks: for 32 keys of a warp at a
// time, every lane ORs its lane bit into its digit's match word (a word per
// digit per warp, all zero between steps), so the word read back is the set of
// lanes holding the same digit; the lowest of them advances the warp's running
// offset of that digit and clears the word, and every key goes straight to its
// position in the tile's digit order (written over the consumed input buffer).
// One shared atomic per key does the work of eight warp ballots and runs about
// 2.6 times faster on sm_103a; (5) look-back gives each digit run's global
// start, checked against the key count once per digit; (6) the tile is
// written out digit run by digit run.
template <typename K, int ITEMS>
__global__ void __launch_bounds__(kRadixThreads, 3) k_radix_pass(RadixPassArgs a) {
  constexpr int TILE = kRadixThreads * ITEMS;
  extern __shared__ __align__(128) unsigned char radix_dyn[];
  K* s_buf[2] = {reinterpret_cast<K*>(radix_dyn), reinterpret_cast<K*>(radix_dyn) + TILE};
  __shared__ uint32_t s_wh[kRadixWarps][kRadixDigits];     // per-warp counts, then tile positions
  __shared__ uint32_t s_match[kRadixWarps][kRadixDigits];  // lanes holding each digit (rank step)
  __shared__ int s_bad;
  __shared__ uint64_t s_gdelta[kRadixDigits];           // global position - tile position, per digit
  __shared__ uint64_t s_bucket[kRadixDigits];           // global start of each digit bucket
  __shared__ uint64_t s_scan[32];
  __shared__ uint32_t s_tile[2];
  __shared__ __align__(8) uint64_t s_mbar[2];

  DevState* st = a.st;
  if (st->overflow & a.skip_mask) return;
  const uint64_t n = st->cnt[a.n_cnt];
  if (n == 0) return;
  const uint64_t ntiles = (n + TILE - 1) / TILE;
  if (st->buf[a.status_buf].cap < ntiles * kRadixDigits || st->buf[a.out_buf].cap < n) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      atomicOr(&st->overflow, 1u << a.stage_bit);
      atomicMax((unsigned long long*)&st->need[a.status_buf], (unsigned long long)(ntiles * kRadixDigits));
      atomicMax((unsigned long long*)&st->need[a.out_buf], (unsigned long long)n);
    }
    return;
  }
  const K* in = static_cast<const K*>(st->buf[a.in_buf].ptr);
  K* out = static_cast<K*>(st->buf[a.out_buf].ptr);
  uint64_t* status = static_cast<uint64_t*>(st->buf[a.status_buf].ptr);
  const uint64_t* hist = static_cast<const uint64_t*>(st->buf[a.hist_buf].ptr) + a.pass * kRadixDigits;
  const uint32_t epoch = st->epoch;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lt_mask = (1u << lane) - 1;
  const uint32_t shift = uint32_t(a.shift);
  const bool aligned = (reinterpret_cast<uintptr_t>(in) & 15) == 0;

  {  // bucket starts of this pass: exclusive scan of the digit histogram
    uint64_t tot;
    s_bucket[tid] = block_exclusive_sum<uint64_t>(hist[tid], s_scan, &tot);
  }
#pragma unroll
  for (int w = 0; w < kRadixWarps; ++w) s_match[w][tid] = 0;
  if (tid == 0) {
    mbar_init(&s_mbar[0], 1);
    mbar_init(&s_mbar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  // thread 0: bulk-load tile t into buffer b when it is a whole, aligned tile
  auto prefetch = [&](uint64_t t, int b) {
    if (t < ntiles && aligned && n - t * TILE >= uint64_t(TILE)) {
      mbar_expect_tx(&s_mbar[b], TILE * sizeof(K));
      bulk_load(s_buf[b], in + t * TILE, TILE * sizeof(K), &s_mbar[b]);
    }
  };
  if (tid == 0) {
    const uint32_t t = atomicAdd(&st->tile_ctr[a.ctr], 1u);
    s_tile[0] = t;
    prefetch(t, 0);
  }
  uint32_t parity0 = 0, parity1 = 0;
  int b = 0;
  while (true) {
    __syncthreads();   // s_tile[b] visible; the other buffer is no longer read
    const uint64_t tile = s_tile[b];
    if (tile >= ntiles) break;
    if (tid == 0) {
      const uint32_t t = atomicAdd(&st->tile_ctr[a.ctr], 1u);
      s_tile[b ^ 1] = t;
      prefetch(t, b ^ 1);
    }
    const uint64_t t0 = tile * TILE;
    const uint32_t tile_n = uint32_t(min(uint64_t(TILE), n - t0));
    K* sk = s_buf[b];
    if (aligned && tile_n == TILE) {
      const uint32_t par = b ? parity1 : parity0;
      if (!mbar_wait(&s_mbar[b], par)) atomicExch(&st->error, kDevTimeout);
      if (b) parity1 ^= 1; else parity0 ^= 1;
    } else {
      for (uint32_t i = tid; i < tile_n; i += kRadixThreads) sk[i] = in[t0 + i];
    }
#pragma unroll
    for (int w = 0; w < kRadixWarps; ++w) s_wh[w][tid] = 0;
    __syncthreads();
    // warp-striped arrangement: item k of lane l is tile key warp*32*ITEMS + k*32 + l,
    // so processing items in order keeps the tile's key order (stable ranks)
    K key[ITEMS];
    const uint32_t wofs = uint32_t(warp) * 32 * ITEMS + lane;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const uint32_t i = wofs + k * 32;
      key[k] = i < tile_n ? sk[i] : K(0);
      if (i < tile_n) atomicAdd(&s_wh[warp][uint32_t(key[k] >> shift) & 0xFF], 1u);
    }
    __syncthreads();
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < kRadixWarps; ++w) {
      const uint32_t c = s_wh[w][tid];
      s_wh[w][tid] = cnt;
      cnt += c;
    }
    lookback_publish(status + tid, tile, kRadixDigits, cnt, epoch);
    uint64_t tot;
    const uint32_t excl = uint32_t(block_exclusive_sum<uint64_t>(cnt, s_scan, &tot));
#pragma unroll
    for (int w = 0; w < kRadixWarps; ++w) s_wh[w][tid] += excl;
    __syncthreads();   // every key is in registers: the buffer takes the ranked tile
    uint32_t* match = s_match[warp];
    uint32_t* wh = s_wh[warp];
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const bool valid = wofs + k * 32 < tile_n;
      const uint32_t d = uint32_t(key[k] >> shift) & 0xFF;
      if (valid) atomicOr(&match[d], 1u << lane);
      __syncwarp();
      uint32_t peers = 0, base = 0;
      if (valid) {
        peers = match[d];
        base = wh[d];
      }
      __syncwarp();
      const uint32_t before = __popc(peers & lt_mask);
      if (valid && before == 0) {   // the lowest lane of the digit: advance and clear
        wh[d] = base + __popc(peers);
        match[d] = 0;
      }
      __syncwarp();
      if (valid) sk[base + before] = key[k];
    }
    // global offset of this tile's run of digit `tid`, checked once per digit
    const uint64_t prev = lookback_resolve(status + tid, tile, kRadixDigits, cnt, epoch, &st->error);
    const uint64_t gstart = s_bucket[tid] + prev;
    s_gdelta[tid] = gstart - excl;
    if (tid == 0) s_bad = 0;
    __syncthreads();
    if (gstart + cnt > n) s_bad = 1;   // histogram and keys disagree
    __syncthreads();
    if (s_bad) {
      if (tid == 0) atomicExch(&st->error, kDevBadState);
    } else if (tile_n == TILE) {
#pragma unroll 4
      for (int k = 0; k < ITEMS; ++k) {
        const uint32_t i = uint32_t(tid) + uint32_t(k) * kRadixThreads;
        const K v = sk[i];
        out[s_gdelta[uint32_t(v >> shift) & 0xFF] + i] = v;
      }
    } else {
      for (uint32_t i = tid; i < tile_n; i += kRadixThreads) {
        const K v = sk[i];
        out[s_gdelta[uint32_t(v >> shift) & 0xFF] + i] = v;
      }
    }
    b ^= 1;
  }
}

}  // namespace hisa
