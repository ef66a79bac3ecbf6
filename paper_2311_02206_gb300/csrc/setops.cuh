// Populate delta and merge full/delta in one pass over merge-path tiles.
//
// Inputs: full (A, sorted, no duplicates) and new (B, sorted, may repeat).
// Outputs: delta = distinct(B) \ A (Section 5.1 "Populating delta", a set
// difference; the adjacent-duplicate test of Section 4.2 "Deduplication"
// removes repeats of B) and full' = A U delta (Section 4.2/5.1 "Merge", the
// merge-path merge of Green, McColl & Bader 2012 that Thrust provides).
//
// The merged sequence of A and B (ties: the A element first) is cut into
// tiles of C elements; a partition kernel finds each tile's split (a_t, b_t)
// by merge-path search.  Within a tile every thread merges ITEMS elements; a
// B element is kept iff it differs from the previous B element and from the
// last A element merged before it (the largest A element <= it).  Kept counts
// are scanned across tiles by decoupled look-back; an A element at index i
// lands at full'[i + kept before it], a kept B element at delta[d] and
// full'[d + A elements before it].  Both outputs are staged in shared memory
// and written coalesced.  Either output can be switched off: delta only
// gives "unique \ full" (or plain unique when A is empty), full' only would
// be a set union.
#pragma once
#include "common.cuh"

namespace hisa {

template <typename K>
struct SetopCfg;
// Items per thread: odd, so that the threads' merge positions (about
// tid * items / 2 into each input) fall on different shared-memory banks.
template <>
struct SetopCfg<uint32_t> { static constexpr int items = 15; };
template <>
struct SetopCfg<uint64_t> { static constexpr int items = 7; };
constexpr int kSetopThreads = 256;
template <typename K>
__host__ __device__ constexpr int setop_tile() { return kSetopThreads * SetopCfg<K>::items; }

struct SetopArgs {
  DevState* st;
  int a_buf, a_cnt;        // full
  int b_buf, b_cnt;        // sorted new
  int split_buf;           // u64 [tiles + 1]
  int status_buf;          // u64 [tiles]
  int d_buf, d_cnt;        // delta out (-1: none)
  int f_buf, f_cnt;        // full' out (-1: none)
  int ctr;
  int skip_mask;           // st->overflow bits that cancel this launch
  int stage_bit;           // overflow bit raised when an output is too small
  int gate1;               // 1 + cnt slot that must be non-zero for the launch to run (0: always)
};

__device__ __forceinline__ bool gated_off(const DevState* st, int gate1) {
  return gate1 > 0 && st->cnt[gate1 - 1] == 0;
}

// Number of A elements among the first d merged elements (ties take A first).
template <typename K>
__device__ __forceinline__ uint64_t merge_path(const K* A, uint64_t na, const K* B, uint64_t nb, uint64_t d) {
  uint64_t lo = d > nb ? d - nb : 0;
  uint64_t hi = d < na ? d : na;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (A[mid] <= B[d - 1 - mid]) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

template <typename K>
__global__ void k_setop_partition(SetopArgs a) {
  constexpr int C = setop_tile<K>();
  DevState* st = a.st;
  if ((st->overflow & a.skip_mask) || gated_off(st, a.gate1)) return;
  const uint64_t na = st->cnt[a.a_cnt], nb = st->cnt[a.b_cnt];
  const uint64_t D = na + nb;
  const uint64_t ntiles = (D + C - 1) / C;
  const K* A = static_cast<const K*>(st->buf[a.a_buf].ptr);
  const K* B = static_cast<const K*>(st->buf[a.b_buf].ptr);
  uint64_t* split = static_cast<uint64_t*>(st->buf[a.split_buf].ptr);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // capacity of the per-tile scratch (checked before any tile runs)
    if (st->buf[a.split_buf].cap < ntiles + 1 || st->buf[a.status_buf].cap < ntiles) {
      atomicOr(&st->overflow, 1u << a.stage_bit);
      atomicMax((unsigned long long*)&st->need[a.split_buf], (unsigned long long)(ntiles + 1));
      atomicMax((unsigned long long*)&st->need[a.status_buf], (unsigned long long)ntiles);
    }
    if (a.d_cnt >= 0) st->cnt[a.d_cnt] = 0;
    if (a.f_cnt >= 0) st->cnt[a.f_cnt] = na;
  }
  if (st->buf[a.split_buf].cap < ntiles + 1) return;
  for (uint64_t t = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; t <= ntiles;
       t += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t d = min(t * C, D);
    split[t] = merge_path(A, na, B, nb, d);
  }
}

template <typename K>
__global__ void __launch_bounds__(kSetopThreads, 5) k_setop(SetopArgs a) {
  constexpr int ITEMS = SetopCfg<K>::items;
  constexpr int C = kSetopThreads * ITEMS;
  __shared__ K s_in[C];     // A part then B part; reused for the full' tile
  __shared__ K s_d[C];      // delta tile
  __shared__ uint64_t s_scan[32];
  __shared__ uint64_t s_dbase;
  __shared__ uint32_t s_tile;
  __shared__ K s_prevA, s_prevB;
  __shared__ int s_hasA, s_hasB;

  DevState* st = a.st;
  if ((st->overflow & a.skip_mask) || gated_off(st, a.gate1)) return;
  const uint64_t na = st->cnt[a.a_cnt], nb = st->cnt[a.b_cnt];
  if (nb == 0) return;   // nothing new: delta stays empty, full' is not needed
  const uint64_t D = na + nb;
  const uint64_t ntiles = (D + C - 1) / C;
  if (st->buf[a.split_buf].cap < ntiles + 1 || st->buf[a.status_buf].cap < ntiles) return;
  const K* A = static_cast<const K*>(st->buf[a.a_buf].ptr);
  const K* B = static_cast<const K*>(st->buf[a.b_buf].ptr);
  const uint64_t* split = static_cast<const uint64_t*>(st->buf[a.split_buf].ptr);
  uint64_t* status = static_cast<uint64_t*>(st->buf[a.status_buf].ptr);
  K* dout = a.d_buf >= 0 ? static_cast<K*>(st->buf[a.d_buf].ptr) : nullptr;
  K* fout = a.f_buf >= 0 ? static_cast<K*>(st->buf[a.f_buf].ptr) : nullptr;
  const uint64_t dcap = a.d_buf >= 0 ? st->buf[a.d_buf].cap : 0;
  const uint64_t fcap = a.f_buf >= 0 ? st->buf[a.f_buf].cap : 0;
  const uint32_t epoch = st->epoch;
  const int tid = threadIdx.x;

  while (true) {
    if (tid == 0) s_tile = atomicAdd(&st->tile_ctr[a.ctr], 1u);
    __syncthreads();
    const uint64_t tile = s_tile;
    if (tile >= ntiles) break;
    const uint64_t d0 = tile * C, d1 = min(d0 + C, D);
    const uint64_t a0 = split[tile], a1 = split[tile + 1];
    const uint64_t b0 = d0 - a0, b1 = d1 - a1;
    const int nA = int(a1 - a0), nB = int(b1 - b0), nT = nA + nB;
    {   // the tile's A part, then its B part, into shared memory: every load of
        // a thread is in flight before the first store (coalesced, ITEMS each)
      K v[ITEMS];
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) {
        const int i = tid + k * kSetopThreads;
        v[k] = i < nA ? A[a0 + i] : (i < nT ? B[b0 + (i - nA)] : K(0));
      }
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) {
        const int i = tid + k * kSetopThreads;
        if (i < nT) s_in[i] = v[k];
      }
    }
    if (tid == 0) {
      s_hasA = a0 > 0;
      if (a0 > 0) s_prevA = A[a0 - 1];
      s_hasB = b0 > 0;
      if (b0 > 0) s_prevB = B[b0 - 1];
    }
    __syncthreads();
    const K* sA = s_in;
    const K* sB = s_in + nA;
    // this thread's slice of the tile's merged sequence
    const int dt = min(tid * ITEMS, nT);
    int ai, bi;
    {
      int lo = max(0, dt - nB), hi = min(dt, nA);
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (sA[mid] <= sB[dt - 1 - mid]) lo = mid + 1;
        else hi = mid;
      }
      ai = lo;
      bi = dt - lo;
    }
    const int ai0 = ai;
    K val[ITEMS];
    uint32_t kind = 0;   // bit k: item k is a kept B element
    uint32_t isA = 0;    // bit k: item k is an A element
    const int nmine = max(0, min(ITEMS, nT - dt));
    const int nitems = nmine;
    // heads of A and B and the last element merged from each, kept in
    // registers; a step is branch-free: both heads are compared, the taken one
    // is replaced by one shared-memory load (A and B are adjacent in s_in)
    bool hasA = ai < nA, hasB = bi < nB;
    K va = hasA ? sA[ai] : K(0), vb = hasB ? sB[bi] : K(0);
    bool hasPrevA = ai > 0 || s_hasA, hasPrevB = bi > 0 || s_hasB;
    K pa = ai > 0 ? sA[ai - 1] : s_prevA;
    K pb = bi > 0 ? sB[bi - 1] : s_prevB;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      if (k >= nmine) break;
      const bool takeA = !hasB || (hasA && va <= vb);
      const bool keep = !takeA && !(hasPrevB && pb == vb) && !(hasPrevA && pa == vb);
      val[k] = takeA ? va : vb;
      isA |= uint32_t(takeA) << k;
      kind |= uint32_t(keep) << k;
      pa = takeA ? va : pa;
      pb = takeA ? pb : vb;
      hasPrevA = hasPrevA || takeA;
      hasPrevB = hasPrevB || !takeA;
      ai += takeA;
      bi += !takeA;
      const int nx = takeA ? ai : nA + bi;   // the taken side's next element
      const K v = s_in[min(nx, C - 1)];
      va = takeA ? v : va;
      vb = takeA ? vb : v;
      hasA = ai < nA;
      hasB = bi < nB;
    }
    const int kept = __popc(kind);
    uint64_t tile_kept;
    const uint32_t kexcl = uint32_t(block_exclusive_sum<uint64_t>(kept, s_scan, &tile_kept));
    if (tid < 32) {
      const uint64_t db = lookback_warp(status, tile, tile_kept, epoch, &st->error);
      if (tid == 0) s_dbase = db;
    }
    __syncthreads();   // s_in is free: every thread holds its items in registers
    const uint64_t dbase = s_dbase;
    // stage outputs: full' tile index = A items before + kept before
    int fa = ai0, kk = int(kexcl);
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      if (k >= nitems) break;
      if (isA & (1u << k)) {
        s_in[fa + kk] = val[k];
        ++fa;
      } else if (kind & (1u << k)) {
        s_in[fa + kk] = val[k];
        s_d[kk] = val[k];
        ++kk;
      }
    }
    __syncthreads();
    const int nF = nA + int(tile_kept);
    if (fout) {
      const uint64_t f0 = a0 + dbase;
      for (int i = tid; i < nF; i += kSetopThreads)
        if (f0 + i < fcap) fout[f0 + i] = s_in[i];
    }
    if (dout) {
      for (int i = tid; i < int(tile_kept); i += kSetopThreads)
        if (dbase + i < dcap) dout[dbase + i] = s_d[i];
    }
    if (tile == ntiles - 1 && tid == 0) {
      const uint64_t nd = dbase + tile_kept;
      const uint64_t nf = na + nd;
      if (a.d_cnt >= 0) st->cnt[a.d_cnt] = nd;
      if (a.f_cnt >= 0) st->cnt[a.f_cnt] = nf;
      bool over = false;
      if (dout && nd > dcap) {
        atomicMax((unsigned long long*)&st->need[a.d_buf], (unsigned long long)nd);
        over = true;
      }
      if (fout && nf > fcap) {
        atomicMax((unsigned long long*)&st->need[a.f_buf], (unsigned long long)nf);
        over = true;
      }
      if (over) atomicOr(&st->overflow, 1u << a.stage_bit);
    }
    __syncthreads();
  }
}

// ---- difference by sorted probes (log-structured full) ------------------------------
//
// C = adjacent-unique(B) \ A for a sorted B (with repeats) and a sorted,
// duplicate-free A that is much larger than B.  Only B is streamed: every
// thread locates its first item in A by binary search inside the A-range of
// its tile, then gallops forward for the following (ascending) items, so A
// is read only where B's items fall (Section 5.1 "populating delta" against
// the large level of a log-structured full).  Kept items are compacted in
// order through a decoupled look-back over the tiles.

struct DiffArgs {
  DevState* st;
  int a_buf, a_cnt;        // sorted, unique
  int b_buf, b_cnt;        // sorted, repeats allowed
  int out_buf, out_cnt;    // C, written from 0
  int status_buf;          // u64 [tiles] look-back
  int ctr;
  int skip_mask, stage_bit;
  int gate1;               // as in SetopArgs
};

constexpr int kDiffThreads = 256;
constexpr int kDiffItems = 8;
constexpr int kDiffTile = kDiffThreads * kDiffItems;

// First position in A[lo, hi) holding a value >= x.
template <typename K>
__device__ __forceinline__ uint64_t lower_bound_k(const K* A, uint64_t lo, uint64_t hi, K x) {
  while (lo < hi) {
    const uint64_t m = (lo + hi) >> 1;
    if (A[m] < x) lo = m + 1;
    else hi = m;
  }
  return lo;
}

template <typename K>
__global__ void __launch_bounds__(kDiffThreads) k_diff_probe(DiffArgs a) {
  __shared__ K s_b[kDiffTile];
  __shared__ uint64_t s_scan[32];
  __shared__ uint64_t s_base, s_lo, s_hi;
  __shared__ uint32_t s_tile;
  __shared__ K s_prev;
  __shared__ int s_has_prev;
  DevState* st = a.st;
  if ((st->overflow & a.skip_mask) || gated_off(st, a.gate1)) return;
  const uint64_t na = st->cnt[a.a_cnt], nb = st->cnt[a.b_cnt];
  if (nb == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) st->cnt[a.out_cnt] = 0;
    return;
  }
  const uint64_t ntiles = (nb + kDiffTile - 1) / kDiffTile;
  if (st->buf[a.status_buf].cap < ntiles) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      atomicMax((unsigned long long*)&st->need[a.status_buf], (unsigned long long)ntiles);
      atomicOr(&st->overflow, 1u << a.stage_bit);
    }
    return;
  }
  const K* A = static_cast<const K*>(st->buf[a.a_buf].ptr);
  const K* B = static_cast<const K*>(st->buf[a.b_buf].ptr);
  K* out = static_cast<K*>(st->buf[a.out_buf].ptr);
  const uint64_t ocap = st->buf[a.out_buf].cap;
  uint64_t* status = static_cast<uint64_t*>(st->buf[a.status_buf].ptr);
  const uint32_t epoch = st->epoch;
  const int tid = threadIdx.x;
  while (true) {
    if (tid == 0) s_tile = atomicAdd(&st->tile_ctr[a.ctr], 1u);
    __syncthreads();
    const uint64_t tile = s_tile;
    if (tile >= ntiles) break;
    const uint64_t b0 = tile * kDiffTile;
    const int nT = int(min(uint64_t(kDiffTile), nb - b0));
    for (int i = tid; i < nT; i += kDiffThreads) s_b[i] = B[b0 + i];
    if (tid == 0) {
      s_has_prev = b0 > 0;
      if (b0 > 0) s_prev = B[b0 - 1];
    }
    __syncthreads();
    if (tid == 0) s_lo = lower_bound_k(A, 0, na, s_b[0]);
    if (tid == 32) {   // one past the last A value <= the tile's largest item
      const K last = s_b[nT - 1];
      uint64_t lo = 0, hi = na;
      while (lo < hi) {
        const uint64_t m = (lo + hi) >> 1;
        if (A[m] <= last) lo = m + 1;
        else hi = m;
      }
      s_hi = lo;
    }
    __syncthreads();
    const uint64_t lo = s_lo, hi = s_hi;
    const int i0 = tid * kDiffItems;
    const int nmine = max(0, min(kDiffItems, nT - i0));
    uint32_t keep = 0;
    if (nmine > 0) {
      uint64_t p = lower_bound_k(A, lo, hi, s_b[i0]);
      bool hp = i0 > 0 || s_has_prev;
      K prev = i0 > 0 ? s_b[i0 - 1] : s_prev;
#pragma unroll
      for (int k = 0; k < kDiffItems; ++k) {
        if (k >= nmine) break;
        const K x = s_b[i0 + k];
        if (!(hp && prev == x)) {
          // gallop from p to the first A value >= x
          if (p < hi && A[p] < x) {
            uint64_t step = 1, q = p;
            while (q + step < hi && A[q + step] < x) {
              q += step;
              step <<= 1;
            }
            p = lower_bound_k(A, q + 1, min(hi, q + step + 1), x);
          }
          if (!(p < hi && A[p] == x)) keep |= 1u << k;
        }
        prev = x;
        hp = true;
      }
    }
    const uint32_t kept = __popc(keep);
    uint64_t tile_kept;
    const uint64_t kexcl = block_exclusive_sum<uint64_t>(kept, s_scan, &tile_kept);
    if (tid < 32) {
      const uint64_t base = lookback_warp(status, tile, tile_kept, epoch, &st->error);
      if (tid == 0) s_base = base;
    }
    __syncthreads();
    // compact in order: kept items of this thread go to s_b[kexcl ...]; every
    // thread reads its items into registers first
    K v[kDiffItems];
#pragma unroll
    for (int k = 0; k < kDiffItems; ++k)
      if (k < nmine) v[k] = s_b[i0 + k];
    __syncthreads();
    int w = int(kexcl);
#pragma unroll
    for (int k = 0; k < kDiffItems; ++k)
      if (keep & (1u << k)) s_b[w++] = v[k];
    __syncthreads();
    const uint64_t base = s_base;
    for (int i = tid; i < int(tile_kept); i += kDiffThreads)
      if (base + i < ocap) out[base + i] = s_b[i];
    if (tile == ntiles - 1 && tid == 0) {
      const uint64_t n = base + tile_kept;
      st->cnt[a.out_cnt] = n;
      if (n > ocap) {
        atomicMax((unsigned long long*)&st->need[a.out_buf], (unsigned long long)n);
        atomicOr(&st->overflow, 1u << a.stage_bit);
      }
    }
    __syncthreads();
  }
}

}  // namespace hisa
