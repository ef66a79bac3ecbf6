// Range index over sorted runs and the binary join (Section 4.3, Algorithm 2,
// Algorithm 3, Section 5.1 "Implementing Joins").
//
// Index: for every run of equal join keys (code >> b) in a sorted code array,
// one open-addressing slot {key, length, begin} placed by linear probing from
// fmix32(key).  Unlike the paper's table, the slot stores the key itself
// rather than only its hash (two keys with equal hashes stay distinct) and the
// run length next to its smallest position, so a probe returns the whole range
// and no atomic-min loop is needed: only run heads are inserted.
//
// Join, outer scanned and inner range-probed as in Algorithm 3, in two passes:
//   count: one probe per outer tuple gives its number of results; the counts
//          are scanned (decoupled look-back) into absolute output offsets;
//   write: the outputs are cut into equal chunks; each CTA finds the outer
//          tuples covering its chunk (precomputed by a partition kernel),
//          stages them with their probe results in shared memory and every
//          thread writes outputs j by a binary search of the staged offsets,
//          so a skewed run is spread over many threads instead of one.
// Filters x != y / x == y are folded into the exact counts: against a value
// fixed per outer tuple they keep or drop the whole run, against the inner
// tuple's other column they remove or keep one position, found by binary
// search in the run (the run's other column is sorted and distinct).
#pragma once
#include "common.cuh"

namespace hisa {

struct Slot {
  uint32_t key;
  uint32_t len;    // 0 = empty slot
  uint64_t begin;
};

// Sources of a result column or filter operand.
enum : int { kSrcOuter0 = 0, kSrcOuter1 = 1, kSrcKey = 2, kSrcOther = 3 };
enum : int { kFiltNone = 0, kFiltNeq = 1, kFiltEq = 2 };

struct IndexArgs {
  DevState* st;
  int keys_buf, keys_cnt;   // sorted codes
  int table_buf;            // Slot[cap], cap a power of two, zeroed; or the direct array
  int b;                    // domain bits: key = code >> b
  int runs_cnt;             // cnt slot receiving the number of runs (-1: none)
  int skip_mask;
  int direct;               // > 0: direct-addressed index over `direct` key bits (below)
};

struct JoinArgs {
  DevState* st;
  int outer_buf, outer_cnt;
  int has_inner;
  int inner_buf, inner_cnt, table_buf;
  int b;                     // domain bits
  int outer_kcol;            // outer column holding the join value
  int proj0, proj1;          // sources of the result columns
  int nfilt;
  int fop[2], fa[2], fb[2];  // filters: op, operand sources
  int offs_buf;              // u64 [n_outer + 1] absolute result offsets
  int status_buf;            // u64 [tiles] look-back
  int starts_buf;            // u64 [chunks + 1] first outer of each write chunk
  int out_buf, out_cnt;      // results appended at cnt[out_cnt]
  int total_cnt;             // cnt slot receiving this join's number of results
  int hist_buf, hist_passes; // fused digit histogram of the results (-1: none)
  int ctr;
  int skip_mask, stage_bit;
  int index_direct;          // the inner index is direct-addressed (k_index_direct)
};

constexpr int kJoinThreads = 256;
constexpr int kJoinItems = 8;
constexpr int kJoinTile = kJoinThreads * kJoinItems;   // outer tuples per count tile
// results per write chunk: 16 per thread for 4-byte codes, 8 for 8-byte ones
// (the chunk is staged in shared memory); the smaller one sizes the buffers
// of chunk starts
template <typename K>
__host__ __device__ constexpr int join_chunk() { return kJoinThreads * (sizeof(K) == 4 ? 16 : 8); }
constexpr int kJoinChunkMin = kJoinThreads * 8;

// instance id of a batched code (0 when the two columns fill the code)
template <typename K>
__device__ __forceinline__ uint64_t inst_of(K code, int b) {
  return 2 * b >= 64 ? 0ull : (uint64_t(code) >> (2 * b));
}
__device__ __forceinline__ uint32_t join_key(uint64_t inst, uint32_t v, int b) {
  return b >= 32 ? v : uint32_t((inst << b) | v);
}

template <typename K>
__device__ __forceinline__ uint32_t colv(K code, int c, int b) {
  const uint64_t m = (b >= 32) ? 0xFFFFFFFFull : ((1ull << b) - 1);
  return c == 0 ? uint32_t((uint64_t(code) >> b) & m) : uint32_t(uint64_t(code) & m);
}

__device__ __forceinline__ bool probe(const Slot* table, uint64_t mask, uint32_t key, uint64_t* begin,
                                      uint32_t* len, uint32_t* err) {
  uint64_t h = fmix32(key) & mask;
  for (uint64_t p = 0; p <= mask; ++p) {
    const uint4 s = *reinterpret_cast<const uint4*>(&table[h]);
    if (s.y == 0) return false;
    if (s.x == key) {
      *begin = (uint64_t(s.w) << 32) | s.z;
      *len = s.y;
      return true;
    }
    h = (h + 1) & mask;
  }
  atomicExch(err, kDevProbeLimit);
  return false;
}

// Direct-addressed run index, for key domains of at most 2^kDirectMaxBits
// values: u64 first[k] for every key k in [0, 2^bits], so the run of key k is
// [first[k], first[k+1]) -- one probe instead of a hash-slot walk.  Built by
// a lower-bound search per key over the sorted codes.
constexpr int kDirectMaxBits = 20;

__device__ __forceinline__ bool probe_run(const void* table, uint64_t mask, int direct, uint32_t key,
                                          uint64_t* begin, uint32_t* len, uint32_t* err) {
  if (direct) {
    const uint64_t* first = static_cast<const uint64_t*>(table);
    const uint64_t b0 = first[key], b1 = first[key + 1];
    *begin = b0;
    *len = uint32_t(b1 - b0);
    return b1 > b0;
  }
  return probe(static_cast<const Slot*>(table), mask, key, begin, len, err);
}

template <typename K>
__global__ void k_index_direct(IndexArgs a) {
  DevState* st = a.st;
  if (st->overflow & a.skip_mask) return;
  const K* keys = static_cast<const K*>(st->buf[a.keys_buf].ptr);
  const uint64_t n = st->cnt[a.keys_cnt];
  uint64_t* first = static_cast<uint64_t*>(st->buf[a.table_buf].ptr);
  const uint64_t nk = 1ull << a.direct;
  for (uint64_t k = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; k <= nk; k += uint64_t(gridDim.x) * blockDim.x) {
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
      const uint64_t m = (lo + hi) >> 1;
      if ((uint64_t(keys[m]) >> a.b) < k) lo = m + 1;
      else hi = m;
    }
    first[k] = lo;
  }
}

// First position in inner[lo, lo+len) whose other column is >= v.
template <typename K>
__device__ __forceinline__ uint32_t run_lower_bound(const K* inner, uint64_t lo, uint32_t len, uint32_t v, int b) {
  uint32_t l = 0, h = len;
  while (l < h) {
    const uint32_t m = (l + h) >> 1;
    if (colv(inner[lo + m], 1, b) < v) l = m + 1;
    else h = m;
  }
  return l;
}

// ---- index build -------------------------------------------------------------------

template <typename K>
__global__ void k_index_build(IndexArgs a) {
  DevState* st = a.st;
  if (st->overflow & a.skip_mask) return;
  const K* keys = static_cast<const K*>(st->buf[a.keys_buf].ptr);
  const uint64_t n = st->cnt[a.keys_cnt];
  Slot* table = static_cast<Slot*>(st->buf[a.table_buf].ptr);
  const uint64_t mask = st->buf[a.table_buf].cap - 1;
  uint32_t runs = 0;
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t k = uint64_t(keys[i]) >> a.b;
    if (i > 0 && (uint64_t(keys[i - 1]) >> a.b) == k) continue;
    // run head: gallop to the end of the run
    uint64_t step = 1, lo = i, hi = i + 1;
    while (hi < n && (uint64_t(keys[hi]) >> a.b) == k) {
      lo = hi;
      hi = min(n, hi + step);
      step <<= 1;
    }
    while (lo + 1 < hi) {  // keys[lo] has key k; keys[hi] (if < n) does not
      const uint64_t m = (lo + hi) >> 1;
      if ((uint64_t(keys[m]) >> a.b) == k) lo = m;
      else hi = m;
    }
    const uint64_t len = hi - i;
    ++runs;
    uint64_t h = fmix32(uint32_t(k)) & mask;
    const unsigned long long word = (unsigned long long)(uint32_t(k)) | ((unsigned long long)len << 32);
    for (uint64_t p = 0; p <= mask; ++p) {
      unsigned long long* w = reinterpret_cast<unsigned long long*>(&table[h]);
      if (atomicCAS(w, 0ull, word) == 0ull) {
        table[h].begin = i;
        break;
      }
      h = (h + 1) & mask;
      if (p == mask) atomicExch(&st->error, kDevProbeLimit);
    }
  }
  if (a.runs_cnt >= 0) {
    for (int o = 16; o > 0; o >>= 1) runs += __shfl_xor_sync(0xffffffffu, runs, o);
    if ((threadIdx.x & 31) == 0 && runs) atomicAdd((unsigned long long*)&st->cnt[a.runs_cnt], (unsigned long long)runs);
  }
}

// ---- join: per-outer probe ---------------------------------------------------------

struct Probe {
  uint64_t begin;
  uint32_t cnt;   // number of results
  uint32_t hole;  // run position removed (neq) or the only one kept (eq); 0xFFFFFFFF = none
  uint32_t mode;  // 0 = whole run [minus hole], 1 = single position `hole`
};

template <typename K>
__device__ __forceinline__ uint32_t src_value(int src, K outer, uint32_t key, int b, bool* fixed) {
  *fixed = src != kSrcOther;
  if (src == kSrcOuter0) return colv(outer, 0, b);
  if (src == kSrcOuter1) return colv(outer, 1, b);
  return key;  // kSrcKey (kSrcOther handled by the caller)
}

template <typename K>
__device__ __forceinline__ Probe do_probe(const JoinArgs& a, K code, const K* inner, const Slot* table,
                                          uint64_t mask, uint32_t* err) {
  Probe p{0, 0, 0xFFFFFFFFu, 0};
  const uint32_t v = colv(code, a.outer_kcol, a.b);
  uint32_t len = 1;
  if (a.has_inner) {
    const uint32_t key = join_key(inst_of(code, a.b), v, a.b);
    if (!probe_run(table, mask, a.index_direct, key, &p.begin, &len, err)) return p;
  }
  // filters (at most two; unrolled so the argument arrays stay in registers)
#pragma unroll
  for (int f = 0; f < 2; ++f) {
    if (f >= a.nfilt) break;
    const int s0 = a.fa[f], s1 = a.fb[f];
    if (s0 == kSrcOther && s1 == kSrcOther) {
      if (a.fop[f] == kFiltNeq) return p;  // x != x never holds
      continue;
    }
    if (s0 != kSrcOther && s1 != kSrcOther) {
      bool fx;
      const uint32_t x = src_value(s0, code, v, a.b, &fx), y = src_value(s1, code, v, a.b, &fx);
      if ((a.fop[f] == kFiltNeq) == (x == y)) return p;
      continue;
    }
    // one operand is the inner tuple's other column
    bool fx;
    const uint32_t x = src_value(s0 == kSrcOther ? s1 : s0, code, v, a.b, &fx);
    const uint32_t pos = run_lower_bound(inner, p.begin, len, x, a.b);
    const bool present = pos < len && colv(inner[p.begin + pos], 1, a.b) == x;
    if (a.fop[f] == kFiltEq) {
      if (!present || (p.mode == 0 && p.hole != 0xFFFFFFFFu && p.hole == pos)) return p;
      if (p.mode == 1 && p.hole != pos) return p;
      p.mode = 1;
      p.hole = pos;
      len = 1;
    } else if (present) {
      if (p.mode == 1) {
        if (p.hole == pos) return p;
      } else {
        p.hole = pos;
      }
    }
  }
  if (p.mode == 1) {
    p.cnt = 1;
  } else {
    p.cnt = len - (p.hole != 0xFFFFFFFFu ? 1 : 0);
  }
  return p;
}

// result r (0-based among this outer's results) -> inner position
__device__ __forceinline__ uint64_t result_pos(const Probe& p, uint32_t r) {
  if (p.mode == 1) return p.begin + p.hole;
  return p.begin + ((p.hole != 0xFFFFFFFFu && r >= p.hole) ? r + 1 : r);
}

template <typename K>
__device__ __forceinline__ K project(const JoinArgs& a, K outer, K inner_code, bool has_inner) {
  const int b = a.b;
  const uint32_t o0 = colv(outer, 0, b), o1 = colv(outer, 1, b);
  const uint32_t key = colv(outer, a.outer_kcol, b);
  const uint32_t oth = has_inner ? colv(inner_code, 1, b) : 0;
  auto pick = [&](int s) -> uint32_t { return s == kSrcOuter0 ? o0 : s == kSrcOuter1 ? o1 : s == kSrcKey ? key : oth; };
  const uint64_t hi = 2 * b >= 64 ? 0ull : (inst_of(outer, b) << (2 * b));
  return K(hi | (uint64_t(pick(a.proj0)) << b) | uint64_t(pick(a.proj1)));
}

template <typename K>
__global__ void __launch_bounds__(kJoinThreads) k_join_count(JoinArgs a) {
  __shared__ K s_code[kJoinTile];
  __shared__ uint64_t s_off[kJoinTile];
  __shared__ uint64_t s_scan[32];
  __shared__ uint64_t s_base;
  __shared__ uint32_t s_tile;
  DevState* st = a.st;
  if (st->overflow & a.skip_mask) return;
  const uint64_t n = st->cnt[a.outer_cnt];
  const uint64_t ntiles = (n + kJoinTile - 1) / kJoinTile;
  if (st->buf[a.offs_buf].cap < n + 1 || st->buf[a.status_buf].cap < ntiles) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      atomicOr(&st->overflow, 1u << a.stage_bit);
      atomicMax((unsigned long long*)&st->need[a.offs_buf], (unsigned long long)(n + 1));
      atomicMax((unsigned long long*)&st->need[a.status_buf], (unsigned long long)ntiles);
    }
    return;
  }
  const K* outer = static_cast<const K*>(st->buf[a.outer_buf].ptr);
  const K* inner = a.has_inner ? static_cast<const K*>(st->buf[a.inner_buf].ptr) : nullptr;
  const Slot* table = a.has_inner ? static_cast<const Slot*>(st->buf[a.table_buf].ptr) : nullptr;
  const uint64_t mask = a.has_inner ? st->buf[a.table_buf].cap - 1 : 0;
  uint64_t* offs = static_cast<uint64_t*>(st->buf[a.offs_buf].ptr);
  uint64_t* status = static_cast<uint64_t*>(st->buf[a.status_buf].ptr);
  const uint32_t epoch = st->epoch;
  const int tid = threadIdx.x;
  if (n == 0) {
    if (blockIdx.x == 0 && tid == 0) {
      offs[0] = 0;
      st->cnt[a.total_cnt] = 0;
    }
    return;
  }
  while (true) {
    if (tid == 0) s_tile = atomicAdd(&st->tile_ctr[a.ctr], 1u);
    __syncthreads();
    const uint64_t tile = s_tile;
    if (tile >= ntiles) break;
    const uint64_t t0 = tile * kJoinTile;
    const int nv = int(min(uint64_t(kJoinTile), n - t0));
    for (int i = tid; i < nv; i += kJoinThreads) s_code[i] = outer[t0 + i];
    __syncthreads();
    uint32_t c[kJoinItems];
    uint64_t sum = 0;
#pragma unroll
    for (int k = 0; k < kJoinItems; ++k) {
      const int i = tid * kJoinItems + k;
      c[k] = 0;
      if (i < nv) c[k] = do_probe<K>(a, s_code[i], inner, table, mask, &st->error).cnt;
      sum += c[k];
    }
    uint64_t tot;
    uint64_t ex = block_exclusive_sum<uint64_t>(sum, s_scan, &tot);
    if (tid < 32) {
      const uint64_t base = lookback_warp(status, tile, tot, epoch, &st->error);
      if (tid == 0) s_base = base;
    }
    __syncthreads();
    ex += s_base;
#pragma unroll
    for (int k = 0; k < kJoinItems; ++k) {
      s_off[tid * kJoinItems + k] = ex;
      ex += c[k];
    }
    __syncthreads();
    for (int i = tid; i < nv; i += kJoinThreads) offs[t0 + i] = s_off[i];
    if (tile == ntiles - 1 && tid == 0) {
      const uint64_t total = s_base + tot;
      offs[n] = total;
      st->cnt[a.total_cnt] = total;
      const uint64_t need = st->cnt[a.out_cnt] + total;
      if (need > st->buf[a.out_buf].cap) {
        atomicOr(&st->overflow, 1u << a.stage_bit);
        atomicMax((unsigned long long*)&st->need[a.out_buf], (unsigned long long)need);
      }
    }
    __syncthreads();
  }
}

// starts[c] = index of the outer tuple whose result range holds result c * chunk
template <typename K>
__global__ void k_join_partition(JoinArgs a) {
  DevState* st = a.st;
  if (st->overflow & a.skip_mask) return;
  const uint64_t n = st->cnt[a.outer_cnt];
  const uint64_t total = st->cnt[a.total_cnt];
  const uint64_t nchunks = (total + join_chunk<K>() - 1) / join_chunk<K>();
  if (st->buf[a.starts_buf].cap < nchunks + 1) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      atomicOr(&st->overflow, 1u << a.stage_bit);
      atomicMax((unsigned long long*)&st->need[a.starts_buf], (unsigned long long)(nchunks + 1));
    }
    return;
  }
  const uint64_t* offs = static_cast<const uint64_t*>(st->buf[a.offs_buf].ptr);
  uint64_t* starts = static_cast<uint64_t*>(st->buf[a.starts_buf].ptr);
  for (uint64_t c = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; c <= nchunks; c += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t o = min(c * join_chunk<K>(), total);
    // largest i in [0, n] with offs[i] <= o  (offs is non-decreasing, offs[0] = 0)
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
      const uint64_t m = (lo + hi + 1) >> 1;
      if (offs[m] <= o) lo = m;
      else hi = m - 1;
    }
    starts[c] = lo;
  }
}

template <typename K>
__global__ void __launch_bounds__(kJoinThreads) k_join_write(JoinArgs a) {
  constexpr int S = kJoinThreads;          // outer tuples staged per batch
  constexpr int IPT = join_chunk<K>() / kJoinThreads;   // consecutive results per thread
  __shared__ uint64_t s_off[S + 1];        // result offset of each staged outer tuple
  __shared__ uint64_t s_begin[S];          // first inner position of its range
  __shared__ uint32_t s_hole[S];           // see Probe::hole
  __shared__ uint32_t s_mode[S];
  __shared__ K s_code[S];
  // the chunk's results, for coalesced stores; one pad word per 32 keeps the
  // per-thread runs of IPT consecutive results on distinct banks
  __shared__ K s_out[join_chunk<K>() + join_chunk<K>() / 32];
  __shared__ uint32_t s_hist[8][256];   // the CTA's digit counts of up to eight passes
  DevState* st = a.st;
  if (st->overflow & a.skip_mask) return;
  const uint64_t n = st->cnt[a.outer_cnt];
  const uint64_t total = st->cnt[a.total_cnt];
  if (total == 0) return;
  const uint64_t nchunks = (total + join_chunk<K>() - 1) / join_chunk<K>();
  const K* outer = static_cast<const K*>(st->buf[a.outer_buf].ptr);
  const K* inner = a.has_inner ? static_cast<const K*>(st->buf[a.inner_buf].ptr) : nullptr;
  const uint64_t n_inner = a.has_inner ? st->cnt[a.inner_cnt] : 0;
  const Slot* table = a.has_inner ? static_cast<const Slot*>(st->buf[a.table_buf].ptr) : nullptr;
  const uint64_t mask = a.has_inner ? st->buf[a.table_buf].cap - 1 : 0;
  const uint64_t* offs = static_cast<const uint64_t*>(st->buf[a.offs_buf].ptr);
  const uint64_t* starts = static_cast<const uint64_t*>(st->buf[a.starts_buf].ptr);
  K* out = static_cast<K*>(st->buf[a.out_buf].ptr) + st->cnt[a.out_cnt];
  const int tid = threadIdx.x;
  const int passes = a.hist_buf >= 0 ? min(a.hist_passes, 8) : 0;
  // the histogram of up to 8 digit passes: every thread counts the digits of
  // its own consecutive results, one atomic per run of equal digits (the high
  // digits of one outer tuple's results rarely change); the CTA's counts are
  // added to the global histogram once, at the end
  unsigned long long* ghist = passes ? static_cast<unsigned long long*>(st->buf[a.hist_buf].ptr) : nullptr;
  for (int i = tid; i < passes * 256; i += kJoinThreads) (&s_hist[0][0])[i] = 0;
  for (uint64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const uint64_t o0 = ch * join_chunk<K>(), o1 = min(o0 + join_chunk<K>(), total);
    uint64_t s = starts[ch];
    const uint64_t last = starts[ch + 1];   // outer holding result o1 (or n)
    while (true) {
      __syncthreads();
      const uint64_t i = s + tid;
      if (i <= last && i < n) {
        s_off[tid] = offs[i];
        const K code = outer[i];
        s_code[tid] = code;
        const Probe p = do_probe<K>(a, code, inner, table, mask, &st->error);
        s_begin[tid] = p.begin;
        s_hole[tid] = p.hole;
        s_mode[tid] = p.mode;
      } else {
        s_off[tid] = ~0ull;
      }
      if (tid == 0) {
        const uint64_t e = s + S;
        s_off[S] = e <= n ? offs[e] : total;
        if (e > last) s_off[S] = ~0ull;
      }
      __syncthreads();
      const uint64_t lo = max(o0, s_off[0]);
      const uint64_t hi_batch = min(s_off[S], total);
      const uint64_t hi = min(o1, hi_batch);
      // this thread's results: IPT consecutive ones of the chunk
      const uint64_t j0 = o0 + uint64_t(tid) * IPT;
      uint64_t j = max(j0, lo);
      const uint64_t jend = min(j0 + IPT, hi);
      if (j < jend) {
        int l = 0, h = S - 1;   // staged outer with s_off[l] <= j < s_off[l+1]
        while (l < h) {
          const int m = (l + h + 1) >> 1;
          if (s_off[m] <= j) l = m;
          else h = m - 1;
        }
        // the results of one outer tuple differ only in the inner tuple's
        // other column: the outer's part of the code is formed once per outer
        const bool in0 = a.proj0 == kSrcOther, in1 = a.proj1 == kSrcOther;
        const uint64_t vmask = a.b >= 32 ? 0xFFFFFFFFull : ((1ull << a.b) - 1);
        while (j < jend) {   // one outer tuple's share of this thread's results
          const uint64_t seg_end = min(jend, s_off[l + 1]);
          const uint32_t r0 = uint32_t(j - s_off[l]);
          const uint32_t nres = uint32_t(seg_end - j);
          const K fixed = project<K>(a, s_code[l], K(0), false);
          const uint64_t begin = s_begin[l];
          const uint32_t hole = s_hole[l], mode = s_mode[l];
          const uint32_t q0 = uint32_t(j - o0);
          if (a.has_inner) {
            // inner positions rise with the result index: check the last one
            const uint32_t rl = r0 + nres - 1;
            const uint64_t last = mode == 1 ? begin + hole : begin + rl + (rl >= hole ? 1 : 0);
            if (nres && last >= n_inner) {   // offsets and probes disagree
              atomicExch(&st->error, kDevBadState);
            } else {
              for (uint32_t t = 0; t < nres; ++t) {
                const uint32_t r = r0 + t;
                const uint64_t ip = mode == 1 ? begin + hole : begin + r + (r >= hole ? 1 : 0);
                const K oth = K(uint64_t(inner[ip]) & vmask);
                const uint32_t q = q0 + t;
                s_out[q + (q >> 5)] = fixed | (in0 ? K(oth << a.b) : K(0)) | (in1 ? oth : K(0));
              }
            }
          } else {
            for (uint32_t t = 0; t < nres; ++t) {
              const uint32_t q = q0 + t;
              s_out[q + (q >> 5)] = fixed;
            }
          }
          j = seg_end;
          ++l;
        }
      }
      if (hi_batch >= o1 || s + S > last) break;
      s += S;
    }
    __syncthreads();
    const uint32_t cn = uint32_t(o1 - o0);
    for (uint32_t t = tid; t < cn; t += kJoinThreads) out[o0 + t] = s_out[t + (t >> 5)];
    if (passes) {
      const uint32_t q0 = uint32_t(tid) * IPT, q1 = min(q0 + IPT, cn);
      for (int q = 0; q < passes; ++q) {
        uint32_t run_d = 0xFFFFFFFFu, run_n = 0;
        for (uint32_t t = q0; t < q1; ++t) {
          const uint32_t d = uint32_t(uint64_t(s_out[t + (t >> 5)]) >> (8 * q)) & 0xFF;
          if (d != run_d) {
            if (run_n) atomicAdd(&s_hist[q][run_d], run_n);
            run_d = d;
            run_n = 0;
          }
          ++run_n;
        }
        if (run_n) atomicAdd(&s_hist[q][run_d], run_n);
      }
    }
    __syncthreads();   // s_out is rewritten by the next chunk
  }
  if (passes) {
    __syncthreads();
    for (int i = tid; i < passes * 256; i += kJoinThreads) {
      const uint32_t c = (&s_hist[0][0])[i];
      if (c) atomicAdd(&ghist[i], (unsigned long long)c);
    }
  }
}

}  // namespace hisa
