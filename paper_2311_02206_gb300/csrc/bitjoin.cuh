// Semi-naive evaluation of a linear recursive rule on bit matrices.
//
// For a program whose one IDB relation R is defined by non-recursive rules
// R(x, y) <- E_i(x, y) and one recursive rule R(x, z) <- B(x, y), R(y, z)
// (REACH, Section 1), over a domain of at most 2^16 values, R's full and
// delta are kept as bit matrices over (first column, second column): row x
// holds bit z for every tuple (x, z).  One iteration of Section 5.1 is then
//
//   new[x]    = OR over the tuples (x, y) of B of delta[y]   (Algorithm 3's
//               join: the run of B's tuples with first column x, each
//               selecting a whole row of delta, 2^b tuples per row OR)
//   delta'[x] = new[x] AND NOT full[x]                        (populating delta)
//   full[x]  |= delta'[x]                                      (merge)
//
// with |delta'| counted by popcount.  The rows are in the declared column
// order, so reading R is writing the rows' bits in order.  Each row keeps a
// mask of its non-zero 32-word chunks, so sparse deltas cost little: a warp
// owns whole chunks and skips those of a delta row that are empty.
#pragma once
#include "common.cuh"

namespace hisa {

constexpr int kBitThreads = 256;
constexpr int kBitMaxBits = 16;   // 2^(2b) bits per matrix: 512 MB at b = 16

__host__ __device__ constexpr uint64_t bit_nwords(int b) { return b >= 5 ? (1ull << (b - 5)) : 1ull; }
__host__ __device__ constexpr uint64_t bit_nchunks(int b) { return b >= 10 ? (1ull << (b - 10)) : 1ull; }
__host__ __device__ constexpr uint64_t bit_mwords(int b) { return b >= 15 ? (1ull << (b - 15)) : 1ull; }

// The tuples of codes (c0 << b) | c1 set in a matrix (rows c0) and in its
// chunk masks; idempotent.
struct BitInitArgs {
  const void* codes;   // K [n]
  uint64_t n;
  int b;
  uint32_t* M;         // 2^b rows of bit_nwords(b) words
  uint32_t* mask;      // 2^b rows of bit_mwords(b) words
  uint32_t* M2;        // optional second matrix set alike (null: none)
};

template <typename K>
__global__ void k_bit_init(BitInitArgs a) {
  const K* codes = static_cast<const K*>(a.codes);
  const uint64_t nw = bit_nwords(a.b), mw = bit_mwords(a.b);
  const uint32_t vmask = (1u << a.b) - 1;
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < a.n; i += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t c = uint64_t(codes[i]);
    const uint64_t x = (c >> a.b) & vmask;
    const uint32_t z = uint32_t(c) & vmask;
    const uint32_t bit = 1u << (z & 31);
    atomicOr(&a.M[x * nw + (z >> 5)], bit);
    if (a.M2) atomicOr(&a.M2[x * nw + (z >> 5)], bit);
    const uint32_t chunk = z >> 10;
    atomicOr(&a.mask[x * mw + (chunk >> 5)], 1u << (chunk & 31));
  }
}

// Bits set in a matrix, summed into *total.
struct BitCountArgs {
  const uint32_t* M;
  uint64_t words;
  unsigned long long* total;
};
static __global__ void k_bit_count(BitCountArgs a) {
  unsigned long long c = 0;
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < a.words; i += uint64_t(gridDim.x) * blockDim.x)
    c += __popc(a.M[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(a.total, c);
}

// One iteration, over work items (row x, segment of at most kBitSeg of its
// B tuples): a hub's thousands of tuples are spread over many CTAs.  Items
// are handed out by an atomic counter, the heaviest rows' first.  A CTA's
// warp w owns the chunks w, w + 8, ... of the row (a chunk is 32 words, a
// word per lane) and ORs the delta rows its segment's tuples select, chunk
// by chunk where the delta row's chunk is non-empty, four tuples' loads in
// flight.  A row of one segment is finished by its CTA: the difference with
// full, full ORed, delta' and the row's chunk mask written, bits counted.  A
// row of several segments ORs each partial row into its accumulator (one per
// such row); the CTA that completes the row (an arrival counter) takes the
// accumulator back, leaving it and the counter zeroed, and finishes the row.
constexpr int kBitSeg = 64;
struct BitJoinArgs {
  const uint64_t* first;   // B's run of first column x: codes [first[x], first[x + 1])
  const void* bcodes;      // B's codes (K), sorted
  const uint64_t* items;   // (x << 32) | segment
  uint64_t nitems;
  const uint32_t* hslot;   // row -> its accumulator (rows of several segments; else unused)
  uint32_t* hacc;          // accumulators, zero between launches
  uint32_t* hdone;         // arrival counters, zero between launches
  const uint32_t* D;       // delta
  const uint32_t* Dmask;
  uint32_t* D2;            // delta' (only the chunks its mask marks are written)
  uint32_t* D2mask;        // zeroed before the launch; written for the rows with B tuples
  uint32_t* R;             // full
  unsigned long long* total;
  unsigned long long* loads;   // delta chunks read (128 B each), for the byte count
  uint32_t* ctr;           // item counter, zeroed before the launch
  int b;
};

constexpr int kBitChunksPerWarp = (1 << (kBitMaxBits - 10)) / (kBitThreads / 32);   // 8 at b = 16

template <typename K>
__global__ void __launch_bounds__(kBitThreads) k_bitjoin(BitJoinArgs a) {
  __shared__ uint32_t s_mask[1 << (kBitMaxBits - 15)];
  __shared__ uint64_t s_item;
  __shared__ int s_last;
  __shared__ unsigned long long s_cnt;
  const K* bc = static_cast<const K*>(a.bcodes);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int nwarps = kBitThreads / 32;
  const uint64_t nw = bit_nwords(a.b), nch = bit_nchunks(a.b), mw = bit_mwords(a.b);
  const uint32_t vmask = (1u << a.b) - 1;
  // words of a chunk that exist (rows of fewer than 32 words: b < 10)
  const uint32_t cw = nw < 32 ? uint32_t(nw) : 32u;
  if (threadIdx.x == 0) s_cnt = 0;
  uint32_t nloads = 0;
  while (true) {
    if (threadIdx.x == 0) {
      const uint32_t i = atomicAdd(a.ctr, 1u);
      s_item = i < a.nitems ? a.items[i] : ~0ull;
    }
    if (threadIdx.x < mw) s_mask[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t item = s_item;
    if (item == ~0ull) break;
    const uint32_t x = uint32_t(item >> 32), seg = uint32_t(item);
    const uint64_t f0 = a.first[x], f1 = a.first[x + 1];
    const uint64_t e0 = f0 + uint64_t(seg) * kBitSeg, e1 = min(f1, e0 + kBitSeg);
    const uint32_t nseg = uint32_t((f1 - f0 + kBitSeg - 1) / kBitSeg);
    uint32_t acc[kBitChunksPerWarp];
#pragma unroll
    for (int k = 0; k < kBitChunksPerWarp; ++k) acc[k] = 0;
    for (uint64_t e = e0; e < e1; e += 4) {
      uint64_t y[4];
      uint32_t m0[4], m1[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) y[u] = e + u < e1 ? uint64_t(bc[e + u]) & vmask : ~0ull;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        m0[u] = y[u] != ~0ull ? a.Dmask[y[u] * mw] : 0u;
        m1[u] = y[u] != ~0ull && mw > 1 ? a.Dmask[y[u] * mw + 1] : 0u;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
#pragma unroll
        for (int k = 0; k < kBitChunksPerWarp; ++k) {
          const uint64_t c = uint64_t(warp) + uint64_t(k) * nwarps;
          if (c >= nch) break;
          const uint32_t mword = c < 32 ? m0[u] : m1[u];
          if ((mword >> (c & 31)) & 1u) {
            if (lane < cw) acc[k] |= a.D[y[u] * nw + c * 32 + lane];
            ++nloads;
          }
        }
      }
    }
    if (nseg > 1) {   // a partial row: into the row's accumulator; the last arrival finishes it
      uint32_t* h = a.hacc + uint64_t(a.hslot[x]) * nw;
#pragma unroll
      for (int k = 0; k < kBitChunksPerWarp; ++k) {
        const uint64_t c = uint64_t(warp) + uint64_t(k) * nwarps;
        if (c >= nch) break;
        if (lane < cw && acc[k]) atomicOr(&h[c * 32 + lane], acc[k]);
      }
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) s_last = atomicAdd(&a.hdone[a.hslot[x]], 1u) == nseg - 1;
      __syncthreads();
      if (!s_last) continue;
      __threadfence();
#pragma unroll
      for (int k = 0; k < kBitChunksPerWarp; ++k) {
        const uint64_t c = uint64_t(warp) + uint64_t(k) * nwarps;
        if (c >= nch) break;
        if (lane < cw) {
          acc[k] = __ldcg(&h[c * 32 + lane]);
          h[c * 32 + lane] = 0;
        }
      }
      if (threadIdx.x == 0) a.hdone[a.hslot[x]] = 0;
    }
    uint32_t cnt = 0;
#pragma unroll
    for (int k = 0; k < kBitChunksPerWarp; ++k) {
      const uint64_t c = uint64_t(warp) + uint64_t(k) * nwarps;
      if (c >= nch) break;
      uint32_t d = 0;
      if (acc[k]) {   // new bits of this word: not yet in full
        uint32_t* rw = a.R + uint64_t(x) * nw + c * 32 + lane;
        d = acc[k] & ~*rw;
        if (d) *rw |= d;
      }
      if (__ballot_sync(0xffffffffu, d != 0u)) {
        if (lane < cw) a.D2[uint64_t(x) * nw + c * 32 + lane] = d;
        if (lane == 0) atomicOr(&s_mask[c >> 5], 1u << (c & 31));
      }
      cnt += __popc(d);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0 && cnt) atomicAdd(&s_cnt, (unsigned long long)cnt);
    __syncthreads();
    if (threadIdx.x < mw) a.D2mask[uint64_t(x) * mw + threadIdx.x] = s_mask[threadIdx.x];
    __syncthreads();   // s_mask and s_item are rewritten for the next item
  }
  if (threadIdx.x == 0 && s_cnt) atomicAdd(a.total, s_cnt);
  if (lane == 0 && nloads) atomicAdd(a.loads, (unsigned long long)nloads);
}

}  // namespace hisa
