// LSD radix sort of packed tuple codes (Section 4.2 "Construction": the sorted
// index is built by a least-significant-first sort; here one 8-bit digit per
// pass over the packed code instead of one stable sort per column).
//
// One pass is a single "onesweep" kernel (Adinets & Merrill, "Onesweep: a
// faster least significant digit radix sort for GPUs", 2022): each CTA takes
// the next tile of keys, ranks them stably inside the tile with warp match
// (one digit counter set per warp), learns the tile's global offset per digit
// by decoupled look-back over the previous tiles, stages the tile in shared
// memory in digit order and writes it out.  The digit histograms of all passes
// come from one earlier read (or are fused into the kernel that produced the
// keys), so a pass reads and writes every key exactly once.
#pragma once
#include "common.cuh"

namespace hisa {

constexpr int kRadixBits = 8;
constexpr int kRadixDigits = 1 << kRadixBits;
constexpr int kRadixThreads = 256;   // one thread per digit in the per-tile scans
constexpr int kRadixWarps = kRadixThreads / 32;

template <typename K>
struct RadixCfg;
template <>
struct RadixCfg<uint32_t> { static constexpr int items = 16; };
template <>
struct RadixCfg<uint64_t> { static constexpr int items = 12; };

template <typename K>
__host__ __device__ constexpr int radix_tile() { return kRadixThreads * RadixCfg<K>::items; }

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

template <typename K>
__global__ void __launch_bounds__(kRadixThreads) k_radix_pass(RadixPassArgs a) {
  constexpr int ITEMS = RadixCfg<K>::items;
  constexpr int TILE = kRadixThreads * ITEMS;
  __shared__ K s_keys[TILE];
  __shared__ uint32_t s_wh[kRadixWarps][kRadixDigits];  // per-warp counts, then offsets
  __shared__ uint32_t s_excl[kRadixDigits];             // tile-local digit start
  __shared__ uint64_t s_gbase[kRadixDigits];            // global start of the tile's digit run
  __shared__ uint64_t s_bucket[kRadixDigits];           // global start of each digit bucket
  __shared__ uint64_t s_scan[32];
  __shared__ uint32_t s_tile;

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

  {  // bucket starts of this pass: exclusive scan of the digit histogram
    uint64_t tot;
    const uint64_t e = block_exclusive_sum<uint64_t>(hist[tid], s_scan, &tot);
    s_bucket[tid] = e;
  }

  while (true) {
    if (tid == 0) s_tile = atomicAdd(&st->tile_ctr[a.ctr], 1u);
    for (int w = 0; w < kRadixWarps; ++w) s_wh[w][tid] = 0;
    __syncthreads();
    const uint64_t tile = s_tile;
    if (tile >= ntiles) break;
    const uint64_t t0 = tile * TILE;

    K key[ITEMS];
    uint32_t rank[ITEMS];
    uint32_t dig[ITEMS];
    // warp-striped arrangement: item k of lane l is key t0 + warp*32*ITEMS + k*32 + l,
    // so processing items in order keeps the tile's key order (stable ranks)
    const uint64_t wbase = t0 + uint64_t(warp) * 32 * ITEMS + lane;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const uint64_t i = wbase + k * 32;
      const bool valid = i < n;
      key[k] = valid ? in[i] : K(0);
      dig[k] = valid ? uint32_t((key[k] >> a.shift) & 0xFF) : 256u;
    }
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const uint32_t d = dig[k];
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      const uint32_t before = __popc(peers & lt_mask);
      uint32_t base = 0;
      if (d < 256) base = s_wh[warp][d];
      __syncwarp();
      if (d < 256 && before == 0) s_wh[warp][d] = base + __popc(peers);
      __syncwarp();
      rank[k] = base + before;
    }
    __syncthreads();
    // per digit: offsets of each warp inside the tile's digit run
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < kRadixWarps; ++w) {
      const uint32_t c = s_wh[w][tid];
      s_wh[w][tid] = cnt;
      cnt += c;
    }
    {
      uint64_t tot;
      const uint64_t e = block_exclusive_sum<uint64_t>(cnt, s_scan, &tot);
      s_excl[tid] = uint32_t(e);
    }
    // global offset of this tile's run of digit `tid`
    const uint64_t prev = lookback_thread(status + tid, tile, kRadixDigits, cnt, epoch, &st->error);
    s_gbase[tid] = s_bucket[tid] + prev;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const uint32_t d = dig[k];
      if (d < 256) s_keys[s_excl[d] + s_wh[warp][d] + rank[k]] = key[k];
    }
    __syncthreads();
    const uint32_t valid_n = uint32_t(min(uint64_t(TILE), n - t0));
    for (uint32_t i = tid; i < valid_n; i += kRadixThreads) {
      const K k = s_keys[i];
      const uint32_t d = uint32_t((k >> a.shift) & 0xFF);
      const uint64_t pos = s_gbase[d] + (i - s_excl[d]);
      if (pos < n) out[pos] = k;
      else atomicExch(&st->error, kDevBadState);   // histogram and keys disagree
    }
    __syncthreads();
  }
}

}  // namespace hisa
