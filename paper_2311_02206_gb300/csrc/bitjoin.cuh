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

constexpr int kBitSeg = 64;                                                 // B tuples per work item
constexpr int kBitBatch = 8;                                                // items a warp takes at once
constexpr int kBitGroups = 8;                                               // chunk groups of a row
constexpr int kBitChunksPerWarp = (1 << (kBitMaxBits - 10)) / kBitGroups;   // 8 at b = 16
__host__ __device__ constexpr uint32_t bit_groups(int b) {
  return bit_nchunks(b) < kBitGroups ? uint32_t(bit_nchunks(b)) : uint32_t(kBitGroups);
}

// The tuples of codes (c0 << b) | c1 set in a matrix (rows c0) and in its
// chunk masks; idempotent.
struct BitInitArgs {
  const void* codes;   // K [n]
  uint64_t n;
  int b;
  uint32_t* M;         // 2^b rows of bit_nwords(b) words
  uint32_t* mask;      // 2^b rows of bit_mwords(b) words
  uint32_t* M2;        // optional second matrix set alike (null: none)
  unsigned long long* total;   // bits newly set in M (null: not counted)
};

template <typename K>
__global__ void k_bit_init(BitInitArgs a) {
  const K* codes = static_cast<const K*>(a.codes);
  const uint64_t nw = bit_nwords(a.b), mw = bit_mwords(a.b);
  const uint32_t vmask = (1u << a.b) - 1;
  uint32_t fresh = 0;
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < a.n; i += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t c = uint64_t(codes[i]);
    const uint64_t x = (c >> a.b) & vmask;
    const uint32_t z = uint32_t(c) & vmask;
    const uint32_t bit = 1u << (z & 31);
    fresh += (atomicOr(&a.M[x * nw + (z >> 5)], bit) & bit) ? 0u : 1u;
    if (a.M2) atomicOr(&a.M2[x * nw + (z >> 5)], bit);
    const uint32_t chunk = z >> 10;
    atomicOr(&a.mask[x * mw + (chunk >> 5)], 1u << (chunk & 31));
  }
  if (a.total) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fresh += __shfl_xor_sync(0xffffffffu, fresh, o);
    if ((threadIdx.x & 31) == 0 && fresh) atomicAdd(a.total, (unsigned long long)fresh);
  }
}

// The work items, built on the device: per row its item count (segments x
// groups) and, for a row of several segments, an accumulator slot; a one-CTA
// scan; every row's items written at its offset (rows in order: the hubs of
// an R-MAT graph are its first rows).
struct BitItemsArgs {
  const uint64_t* first;
  uint64_t* offs;          // rows + 1; offs[rows] = the number of items
  uint64_t* items;
  uint32_t* hslot;
  uint32_t* nheavy;        // zeroed before the launch
  int b;
  // rows to work this iteration (a bit each; null: every row with B tuples,
  // and the rows of several segments get their accumulators)
  const uint32_t* todo;
};
static __global__ void k_bit_items_count(BitItemsArgs a) {
  const uint64_t rows = 1ull << a.b;
  for (uint64_t x = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; x < rows; x += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t nseg = (a.first[x + 1] - a.first[x] + kBitSeg - 1) / kBitSeg;
    if (a.todo) {
      a.offs[x] = ((a.todo[x >> 5] >> (x & 31)) & 1u) ? nseg * bit_groups(a.b) : 0;
    } else {
      a.offs[x] = nseg * bit_groups(a.b);
      if (nseg > 1) a.hslot[x] = atomicAdd(a.nheavy, 1u);
    }
  }
}

// The rows an iteration must work: every x with a B tuple (x, y) whose delta
// row y is non-empty (its chunk mask); a thread per B tuple.  Rows whose B
// tuples all select empty delta rows derive nothing.
struct BitTodoArgs {
  const uint32_t* Dmask;
  const void* bcodes;      // B's codes (K): (x << b) | y
  uint64_t n;
  uint32_t* todo;          // zeroed before the launch
  int b;
};
template <typename K>
__global__ void k_bit_todo(BitTodoArgs a) {
  const uint64_t mw = bit_mwords(a.b);
  const uint32_t vmask = (1u << a.b) - 1;
  const K* bc = static_cast<const K*>(a.bcodes);
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < a.n; i += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t c = uint64_t(bc[i]);
    const uint64_t y = c & vmask;
    uint32_t any = a.Dmask[y * mw];
    if (mw > 1) any |= a.Dmask[y * mw + 1];
    if (!any) continue;
    const uint32_t x = uint32_t(c >> a.b) & vmask;
    const uint32_t bit = 1u << (x & 31);
    if (!(a.todo[x >> 5] & bit)) atomicOr(&a.todo[x >> 5], bit);
  }
}
static __global__ void __launch_bounds__(1024) k_bit_items_scan(BitItemsArgs a) {
  __shared__ uint64_t s_scan[33];
  const uint64_t rows = 1ull << a.b;
  const uint64_t total = cta_scan_inplace(a.offs, rows, s_scan);
  if (threadIdx.x == 0) a.offs[rows] = total;
}
static __global__ void k_bit_items_write(BitItemsArgs a) {
  const uint64_t rows = 1ull << a.b;
  const uint32_t ng = bit_groups(a.b);
  for (uint64_t x = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; x < rows; x += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t n = a.offs[x + 1] - a.offs[x];
    for (uint64_t i = 0; i < n; ++i)
      a.items[a.offs[x] + i] = (x << 32) | ((i / ng) << 8) | (i % ng);
  }
}

struct BitJoinArgs {
  const uint64_t* first;   // B's run of first column x: codes [first[x], first[x + 1])
  const void* bcodes;      // B's codes (K), sorted
  const uint64_t* items;   // (x << 32) | (segment << 8) | group
  const uint64_t* nitems;  // device: the number of items
  const uint32_t* hslot;   // row -> its accumulator (rows of several segments; else unused)
  uint32_t* hacc;          // accumulators (a row each), zero between launches
  uint32_t* hdone;         // arrival counters (kBitGroups per accumulator), zero between launches
  const uint32_t* D;       // delta
  const uint32_t* Dmask;
  uint32_t* D2;            // delta' (only the chunks its mask marks are written)
  uint32_t* D2mask;        // zeroed before the launch
  uint32_t* R;             // full
  unsigned long long* total;
  unsigned long long* loads;   // delta chunks read (128 B each), for the byte count
  uint32_t* ctr;           // item counter, zeroed before the launch
  int b;
};

// Bits k = 0..7 of the result: mask bit g + 8k of row y (the chunks of group
// g); rows of one or two mask words.
__device__ __forceinline__ uint32_t group_bits(const uint32_t* mask, uint64_t y, uint64_t mw, uint32_t g) {
  const uint64_t m = mw > 1 ? *reinterpret_cast<const unsigned long long*>(mask + y * mw) : uint64_t(mask[y * mw]);
  return uint32_t((((m >> g) & 0x0101010101010101ull) * 0x0102040810204080ull) >> 56);
}

template <typename K>
__global__ void __launch_bounds__(kBitThreads) k_bitjoin(BitJoinArgs a) {
  const K* bc = static_cast<const K*>(a.bcodes);
  const int lane = threadIdx.x & 31;
  const uint64_t nw = bit_nwords(a.b), nch = bit_nchunks(a.b), mw = bit_mwords(a.b);
  const uint32_t vmask = (1u << a.b) - 1;
  const uint32_t cw = nw < 32 ? uint32_t(nw) : 32u;   // words of a chunk (b < 10: fewer than 32)
  unsigned long long cnt = 0, nloads = 0;
  const uint64_t nitems = *a.nitems;
  uint32_t next = 0, left = 0;   // this warp's batch of items
  while (true) {
    if (left == 0) {   // kBitBatch items per atomic: the counter is no bottleneck
      uint32_t i0 = 0;
      if (lane == 0) i0 = atomicAdd(a.ctr, uint32_t(kBitBatch));
      next = __shfl_sync(0xffffffffu, i0, 0);
      left = kBitBatch;
    }
    if (next >= nitems) break;
    const uint64_t item = a.items[next];
    ++next;
    --left;
    const uint32_t x = uint32_t(item >> 32), seg = uint32_t(item >> 8) & 0xFFFFFFu, g = uint32_t(item) & 0xFFu;
    const uint64_t f0 = a.first[x], f1 = a.first[x + 1];
    const uint64_t e0 = f0 + uint64_t(seg) * kBitSeg, e1 = min(f1, e0 + kBitSeg);
    const uint32_t nseg = uint32_t((f1 - f0 + kBitSeg - 1) / kBitSeg);
    uint32_t acc[kBitChunksPerWarp];
#pragma unroll
    for (int k = 0; k < kBitChunksPerWarp; ++k) acc[k] = 0;
    // chunks of this group that exist (k with g + 8k < nch) and lanes that hold a word
    uint32_t live = 0;
    for (int k = 0; k < kBitChunksPerWarp; ++k)
      if (uint64_t(g) + uint64_t(k) * kBitGroups < nch) live |= 1u << k;
    if (lane >= cw) live = 0;
    for (uint64_t e = e0; e < e1; e += 2) {
      const bool ok1 = e + 1 < e1;
      const uint64_t y0 = uint64_t(bc[e]) & vmask;
      const uint64_t y1 = ok1 ? uint64_t(bc[e + 1]) & vmask : 0;
      // this group's chunks g, g + 8, ... of each delta row's mask as the
      // bits of one byte (every eighth mask bit gathered by a multiply)
      const uint32_t s0 = group_bits(a.Dmask, y0, mw, g) & live;
      const uint32_t s1 = ok1 ? group_bits(a.Dmask, y1, mw, g) & live : 0u;
      uint32_t v0[kBitChunksPerWarp], v1[kBitChunksPerWarp];
#pragma unroll
      for (int k = 0; k < kBitChunksPerWarp; ++k) {   // every load issued before any is used
        const uint64_t c = uint64_t(g) + uint64_t(k) * kBitGroups;
        v0[k] = (s0 >> k) & 1u ? a.D[y0 * nw + c * 32 + lane] : 0u;
        v1[k] = (s1 >> k) & 1u ? a.D[y1 * nw + c * 32 + lane] : 0u;
      }
      if (lane == 0) nloads += __popc(s0) + __popc(s1);
#pragma unroll
      for (int k = 0; k < kBitChunksPerWarp; ++k) acc[k] |= v0[k] | v1[k];
    }
    if (nseg > 1) {   // a partial row: into the row's accumulator; the last arrival finishes the group
      const uint32_t hs = a.hslot[x];
      uint32_t* h = a.hacc + uint64_t(hs) * nw;
#pragma unroll
      for (int k = 0; k < kBitChunksPerWarp; ++k) {
        const uint64_t c = uint64_t(g) + uint64_t(k) * kBitGroups;
        if (c < nch && lane < cw && acc[k]) atomicOr(&h[c * 32 + lane], acc[k]);
      }
      __threadfence();
      __syncwarp();
      uint32_t last = 0;
      if (lane == 0) last = atomicAdd(&a.hdone[uint64_t(hs) * kBitGroups + g], 1u) == nseg - 1;
      last = __shfl_sync(0xffffffffu, last, 0);
      if (!last) continue;
      __threadfence();
#pragma unroll
      for (int k = 0; k < kBitChunksPerWarp; ++k) {
        const uint64_t c = uint64_t(g) + uint64_t(k) * kBitGroups;
        if (c < nch && lane < cw) {
          acc[k] = __ldcg(&h[c * 32 + lane]);
          h[c * 32 + lane] = 0;
        }
      }
      if (lane == 0) a.hdone[uint64_t(hs) * kBitGroups + g] = 0;
    }
#pragma unroll
    for (int k = 0; k < kBitChunksPerWarp; ++k) {
      const uint64_t c = uint64_t(g) + uint64_t(k) * kBitGroups;
      if (c >= nch) break;
      uint32_t d = 0;
      if (acc[k]) {   // new bits of this word: not yet in full
        uint32_t* rw = a.R + uint64_t(x) * nw + c * 32 + lane;
        d = acc[k] & ~*rw;
        if (d) *rw |= d;
      }
      if (__ballot_sync(0xffffffffu, d != 0u)) {
        if (lane < cw) a.D2[uint64_t(x) * nw + c * 32 + lane] = d;
        if (lane == 0) atomicOr(&a.D2mask[uint64_t(x) * mw + (c >> 5)], 1u << (c & 31));
      }
      cnt += __popc(d);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane == 0 && cnt) atomicAdd(a.total, cnt);
  if (lane == 0 && nloads) atomicAdd(a.loads, nloads);
}

// The same iteration with 16-byte loads, for rows of whole 32-word chunks
// (b >= 10): lane l holds words 4 (l mod 8) .. + 3 of chunk k = 4p + l / 8 of
// the group (p = 0, 1), so one warp load covers four chunks and a B tuple's
// eight chunks take two loads instead of eight.
__device__ __forceinline__ void or4(uint4& a, const uint4& v) {
  a.x |= v.x;
  a.y |= v.y;
  a.z |= v.z;
  a.w |= v.w;
}
__device__ __forceinline__ bool any4(const uint4& v) { return (v.x | v.y | v.z | v.w) != 0u; }

template <typename K>
__global__ void __launch_bounds__(kBitThreads) k_bitjoin_vec(BitJoinArgs a) {
  const K* bc = static_cast<const K*>(a.bcodes);
  const int lane = threadIdx.x & 31, sub = lane >> 3, w4 = (lane & 7) * 4;
  const uint64_t nw = bit_nwords(a.b), nch = bit_nchunks(a.b), mw = bit_mwords(a.b);
  const uint32_t vmask = (1u << a.b) - 1;
  unsigned long long cnt = 0, nloads = 0;
  const uint64_t nitems = *a.nitems;
  uint32_t next = 0, left = 0;   // this warp's batch of items
  while (true) {
    if (left == 0) {
      uint32_t i0 = 0;
      if (lane == 0) i0 = atomicAdd(a.ctr, uint32_t(kBitBatch));
      next = __shfl_sync(0xffffffffu, i0, 0);
      left = kBitBatch;
    }
    if (next >= nitems) break;
    const uint64_t item = a.items[next];
    ++next;
    --left;
    const uint32_t x = uint32_t(item >> 32), seg = uint32_t(item >> 8) & 0xFFFFFFu, g = uint32_t(item) & 0xFFu;
    const uint64_t f0 = a.first[x], f1 = a.first[x + 1];
    const uint64_t e0 = f0 + uint64_t(seg) * kBitSeg, e1 = min(f1, e0 + kBitSeg);
    const uint32_t nseg = uint32_t((f1 - f0 + kBitSeg - 1) / kBitSeg);
    // this lane's two chunks (k = sub, 4 + sub) and whether they exist
    const uint64_t c0 = uint64_t(g) + uint64_t(sub) * kBitGroups, c1 = c0 + 4ull * kBitGroups;
    const uint32_t live = (c0 < nch ? 1u : 0u) | (c1 < nch ? 2u : 0u);
    uint4 acc0 = make_uint4(0, 0, 0, 0), acc1 = make_uint4(0, 0, 0, 0);
    for (uint64_t e = e0; e < e1; e += 2) {
      const bool ok1 = e + 1 < e1;
      const uint64_t y0 = uint64_t(bc[e]) & vmask;
      const uint64_t y1 = ok1 ? uint64_t(bc[e + 1]) & vmask : 0;
      const uint32_t sa = group_bits(a.Dmask, y0, mw, g);
      const uint32_t sb = ok1 ? group_bits(a.Dmask, y1, mw, g) : 0u;
      // bits 0, 1: this lane's chunks of the two delta rows
      const uint32_t m0 = (((sa >> sub) & 1u) | (((sa >> (4 + sub)) & 1u) << 1)) & live;
      const uint32_t m1 = (((sb >> sub) & 1u) | (((sb >> (4 + sub)) & 1u) << 1)) & live;
      const uint4 z = make_uint4(0, 0, 0, 0);
      const uint4 v00 = m0 & 1u ? *reinterpret_cast<const uint4*>(a.D + y0 * nw + c0 * 32 + w4) : z;
      const uint4 v01 = m0 & 2u ? *reinterpret_cast<const uint4*>(a.D + y0 * nw + c1 * 32 + w4) : z;
      const uint4 v10 = m1 & 1u ? *reinterpret_cast<const uint4*>(a.D + y1 * nw + c0 * 32 + w4) : z;
      const uint4 v11 = m1 & 2u ? *reinterpret_cast<const uint4*>(a.D + y1 * nw + c1 * 32 + w4) : z;
      if (lane == 0) nloads += __popc(sa & 0xFFu) + __popc(sb & 0xFFu);
      or4(acc0, v00);
      or4(acc0, v10);
      or4(acc1, v01);
      or4(acc1, v11);
    }
    if (nseg > 1) {   // a partial row: into the row's accumulator; the last arrival finishes the group
      const uint32_t hs = a.hslot[x];
      uint32_t* h = a.hacc + uint64_t(hs) * nw;
      const uint32_t* p0 = &acc0.x;
      const uint32_t* p1 = &acc1.x;
      for (int q = 0; q < 4; ++q) {
        if ((live & 1u) && p0[q]) atomicOr(&h[c0 * 32 + w4 + q], p0[q]);
        if ((live & 2u) && p1[q]) atomicOr(&h[c1 * 32 + w4 + q], p1[q]);
      }
      __threadfence();
      __syncwarp();
      uint32_t last = 0;
      if (lane == 0) last = atomicAdd(&a.hdone[uint64_t(hs) * kBitGroups + g], 1u) == nseg - 1;
      last = __shfl_sync(0xffffffffu, last, 0);
      if (!last) continue;
      __threadfence();
      uint32_t* q0 = &acc0.x;
      uint32_t* q1 = &acc1.x;
      for (int q = 0; q < 4; ++q) {
        if (live & 1u) {
          q0[q] = __ldcg(&h[c0 * 32 + w4 + q]);
          h[c0 * 32 + w4 + q] = 0;
        }
        if (live & 2u) {
          q1[q] = __ldcg(&h[c1 * 32 + w4 + q]);
          h[c1 * 32 + w4 + q] = 0;
        }
      }
      if (lane == 0) a.hdone[uint64_t(hs) * kBitGroups + g] = 0;
    }
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      if (!__any_sync(0xffffffffu, (live >> p) & 1u)) break;
      const uint64_t c = p ? c1 : c0;
      const uint4 ac = p ? acc1 : acc0;
      uint4 d = make_uint4(0, 0, 0, 0);
      if (((live >> p) & 1u) && any4(ac)) {   // new bits of these words: not yet in full
        uint4* rw = reinterpret_cast<uint4*>(a.R + uint64_t(x) * nw + c * 32 + w4);
        const uint4 r = *rw;
        d = make_uint4(ac.x & ~r.x, ac.y & ~r.y, ac.z & ~r.z, ac.w & ~r.w);
        if (any4(d)) *rw = make_uint4(r.x | d.x, r.y | d.y, r.z | d.z, r.w | d.w);
      }
      // a chunk is the 8 lanes of one quarter of the warp
      const uint32_t bal = __ballot_sync(0xffffffffu, any4(d));
      if ((bal >> (sub * 8)) & 0xFFu) {
        *reinterpret_cast<uint4*>(a.D2 + uint64_t(x) * nw + c * 32 + w4) = d;
        if ((lane & 7) == 0) atomicOr(&a.D2mask[uint64_t(x) * mw + (c >> 5)], 1u << (c & 31));
      }
      cnt += __popc(d.x) + __popc(d.y) + __popc(d.z) + __popc(d.w);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane == 0 && cnt) atomicAdd(a.total, cnt);
  if (lane == 0 && nloads) atomicAdd(a.loads, nloads);
}

}  // namespace hisa
