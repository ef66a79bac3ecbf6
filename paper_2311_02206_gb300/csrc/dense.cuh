// Grouped join with dense-domain deduplication: the join of Algorithm 3 and
// the sort + unique of new (Section 4.2) in one pass, for a join step whose
// results are grouped by a column of the outer relation.
//
// Applies when the outer (a delta) is stored as (g, k) -- g the column the
// result keeps, k the join column -- and the result is (g, o) with o the
// inner relation's other column, as in REACH's recursive rule with Reach
// stored target-first.  The outer tuples of one g are contiguous, so one CTA
// takes a whole group: every outer (g, k) probes the inner index on k and
// marks the inner run's o values in a shared-memory bitmap over the active
// domain (2^b bits); the group's results are then the set bits in ascending
// order.  Groups are placed by their offsets in group order, so
// new comes out sorted and duplicate-free, and no raw result is ever written
// to HBM (they were 8.5x the distinct ones on R-MAT 16).  Three launches:
// mark (each group's bitmap and count, groups in any order), scan (offsets),
// emit (each group's set bits at its offset).
#pragma once
#include "common.cuh"
#include "join.cuh"

namespace hisa {

// Start position of every run of equal g = code >> b in a sorted code array,
// compacted in order; cnt[out_cnt] = number of groups and out[groups] = n
// (k_group_compact, from a direct index of the array by g).
struct GroupArgs {
  DevState* st;
  int in_buf, in_cnt;
  int b;
  int out_buf, out_cnt;   // u64 starts
  int status_buf;         // u64 [tiles] look-back
  int ctr;
  int skip_mask, stage_bit;
  // k_group_compact only, when unit_size > 0: the dense join's work units
  // per group (see DenseArgs), computed in the same pass
  int units_buf, done_buf, mslot_buf, unit_size;
  int bmm_buf, bm_words;   // multi-unit bitmaps: capacity checked here, bm_words per group
  // k_group_compact: with indirect, first[g] is read as vals[in[g]] (a
  // gathered Tmp's starts: vals = offsets per inner tuple, in = the inner's
  // direct index by the kept value)
  int indirect, vals_buf;
  // k_group_compact with units: bit g of this u32 bitmap set = group g is
  // pulled: it gets no units; its index goes to plist (count in cnt[pull_cnt])
  int pull_bm_buf = -1, plist_buf = -1, pull_cnt = -1;
};

// A two-step rule variant H(x, y) <- A(x, a), delta(a, c), B(c, y) -- delta
// joined on its first stored column with the inner atom A, the Tmp relation
// keeping A's other column x first and delta's second column c -- gathered
// straight into Tmp grouped by x, in place of the join and the sort of Tmp
// by x that the dense join needs (Section 4.1's join of delta with an inner
// relation, its results grouped by the kept column):
//   len:    per tuple (x, a) of A (sorted by x): |delta(a, .)| -> pre
//   scan:   pre -> exclusive offsets, the total is |Tmp| (capacity check)
//   gather: delta(a, .)'s second column, x prepended, copied to Tmp at pre
// Tmp's group starts are then pre[first_A(x)] (k_group_compact, indirect).
struct ChainArgs {
  DevState* st;
  int a_buf, a_cnt;           // A's codes sorted by x: x in the high half, a in the low half
  int delta_buf, delta_cnt;   // delta sorted by its first stored column
  int dfirst_buf;             // direct index of delta by its high half (2^b + 1 entries)
  int pre_buf;                // u64 [|A| + 1]
  int tmp_buf, tmp_cnt;
  int b;
  int skip_mask, stage_bit;
  // optional (tfirst_buf >= 0): Tmp's direct index by x, tfirst[x] =
  // pre[afirst[x]] (afirst: A's direct index by x), for a next step that
  // probes Tmp by x (an inverted dense join)
  int afirst_buf, tfirst_buf;
};

template <typename K>
__global__ void k_chain_first(ChainArgs a) {
  DevState* st = a.st;
  if (st->overflow & a.skip_mask) return;
  const uint64_t* af = static_cast<const uint64_t*>(st->buf[a.afirst_buf].ptr);
  const uint64_t* pre = static_cast<const uint64_t*>(st->buf[a.pre_buf].ptr);
  uint64_t* tf = static_cast<uint64_t*>(st->buf[a.tfirst_buf].ptr);
  const uint64_t nk = 1ull << a.b;
  for (uint64_t k = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; k <= nk; k += uint64_t(gridDim.x) * blockDim.x)
    tf[k] = pre[af[k]];
}

template <typename K>
__global__ void k_chain_len(ChainArgs a) {
  DevState* st = a.st;
  if (st->overflow & a.skip_mask) return;
  const uint64_t na = st->cnt[a.a_cnt];
  if (st->buf[a.pre_buf].cap < na + 1) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      atomicMax((unsigned long long*)&st->need[a.pre_buf], (unsigned long long)(na + 1));
      atomicOr(&st->overflow, 1u << a.stage_bit);
    }
    return;
  }
  const K* A = static_cast<const K*>(st->buf[a.a_buf].ptr);
  const uint64_t* df = static_cast<const uint64_t*>(st->buf[a.dfirst_buf].ptr);
  uint64_t* pre = static_cast<uint64_t*>(st->buf[a.pre_buf].ptr);
  for (uint64_t j = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; j < na; j += uint64_t(gridDim.x) * blockDim.x) {
    const uint32_t av = colv(A[j], 1, a.b);
    pre[j] = df[av + 1] - df[av];
  }
}

template <typename K>
__global__ void __launch_bounds__(1024) k_chain_scan(ChainArgs a) {
  __shared__ uint64_t s_scan[33];
  DevState* st = a.st;
  if (st->overflow & a.skip_mask) return;
  const uint64_t na = st->cnt[a.a_cnt];
  uint64_t* pre = static_cast<uint64_t*>(st->buf[a.pre_buf].ptr);
  const uint64_t total = cta_scan_inplace(pre, na, s_scan);
  if (threadIdx.x == 0) {
    pre[na] = total;
    st->cnt[a.tmp_cnt] = total;
    if (total > st->buf[a.tmp_buf].cap) {
      atomicMax((unsigned long long*)&st->need[a.tmp_buf], (unsigned long long)total);
      atomicOr(&st->overflow, 1u << a.stage_bit);
    }
  }
}

// A warp per tuple of A: its delta run copied (coalesced) behind pre[j].
template <typename K>
__global__ void k_chain_gather(ChainArgs a) {
  DevState* st = a.st;
  if (st->overflow & a.skip_mask) return;
  const uint64_t na = st->cnt[a.a_cnt];
  const K* A = static_cast<const K*>(st->buf[a.a_buf].ptr);
  const K* delta = static_cast<const K*>(st->buf[a.delta_buf].ptr);
  const uint64_t* df = static_cast<const uint64_t*>(st->buf[a.dfirst_buf].ptr);
  const uint64_t* pre = static_cast<const uint64_t*>(st->buf[a.pre_buf].ptr);
  K* tmp = static_cast<K*>(st->buf[a.tmp_buf].ptr);
  const int lane = threadIdx.x & 31;
  const uint64_t nw = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  for (uint64_t j = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5; j < na; j += nw) {
    const K code = A[j];
    const uint32_t av = colv(code, 1, a.b);
    const uint64_t hi = uint64_t(colv(code, 0, a.b)) << a.b;
    const uint64_t d0 = df[av], n = df[av + 1] - d0, o = pre[j];
    for (uint64_t i = lane; i < n; i += 32) tmp[o + i] = K(hi | colv(delta[d0 + i], 1, a.b));
  }
}

struct DenseArgs {
  DevState* st;
  int outer_buf, outer_cnt;     // (g, k) codes, sorted
  int groups_buf, groups_cnt;   // group starts (GroupArgs output)
  int inner_buf, table_buf;     // inner codes (k, o) and their run index
  int b;
  int out_buf, out_cnt;         // results appended after cnt[out_cnt] (read only)
  int total_cnt;                // receives the number of results
  int raw_cnt;                  // cnt slot accumulating raw (pre-dedup) results
  int bm_buf;                   // u32 [groups][2^b / 32]: each group's bitmap
  int offs_buf;                 // u64 [groups]: result count, then its offset
  int ctr;
  int skip_mask, stage_bit;
  int index_direct;             // the inner index is direct-addressed
  // full of the head relation (append-only: one sorted, duplicate-free level
  // per iteration) with each level's direct index by the kept column: their
  // tuples are removed from each group's bitmap, so the join writes
  // delta = new \ full itself (-1: no difference)
  int full_buf, lvidx_buf, nlv_cnt;
  int drop_self;                // the rule's filter kept != other: drop bit g in group g
  // work units: a group of more than unit_size outer tuples is marked by
  // several CTAs (first unit of group g: units[g], total in units[groups]);
  // done[g] counts its finished units; such a group's CTAs OR their marks
  // into its slot mslot[g] of bmm (multi-unit bitmaps, left zeroed; count
  // in mslot[groups])
  int units_buf, done_buf;
  int unit_size;
  int mslot_buf, bmm_buf;
  int units_ready;              // computed by the group compaction (else k_dense_units runs)
  // pull mode (pull_inner_buf >= 0; a direct inner index, b <= kPullMaxBits):
  // a group listed in plist is worked the other way round by k_dense_pull
  // (one CTA per group; it has no units in k_dense_mark).  Its delta values k go into a frontier bitmap F, full's
  // tuples of the group into a bitmap V, and every candidate o (a value with
  // inner tuples, not in V) walks its inner tuples (o, k') -- the inner
  // relation sorted by its other column, with a direct index by it -- until
  // one k' is in F: o is then new.  Same results as marking the inner runs of
  // the delta values (the direction-optimizing traversal of Beamer et al.,
  // 2012, applied per group).  Each group's finish chooses the next
  // iteration's mode: pull when the inner runs the next delta would mark
  // (sum of their lengths) exceed pull_k16 / 16 times the candidates left
  // (|other values| - |full_g| - |next delta|) plus the next delta's size.
  int pull_inner_buf = -1, pull_index_buf = -1;   // inner codes (o, k) sorted; direct index by o
  int pull_out_buf = -1;                // u32 [2^b / 32]: values o with inner tuples
  int pull_bm_buf = -1;                 // u32 [2^b / 32]: bit g = group g pulls (this and next iteration)
  int fcnt_buf = -1;                    // u32 [2^b]: |full_g| (kept by the append of each level, or by the emit)
  int nout_cnt = -1;                    // cnt slot: number of values o with inner tuples
  int pull_first_buf = -1;              // u32 [2^b]: each o's first k (PullOutArgs)
  int tdeg_buf = -1;                    // u32 [2^b]: each k's run length in the push-ordered inner
  int plist_buf = -1, pull_cnt = -1;    // pulled groups (indices, written by the group compaction)
  int pull_raw_cnt = -1;                // cnt slot: codes the pull kernel read (delta, full, inner tuples)
  // full kept as a bit matrix (fbm_buf >= 0; b <= kMatrixMaxBits): row g holds
  // bit o for every (g, o) in full, 2^b bits per row.  The difference against
  // full is then one AND-NOT of the group's row; full_buf is -1.
  int fbm_buf = -1;
  // batched runs: the row of (instance, g) is the code shifted right by b,
  // masked to row_bits bits (instance bits + b; 0: b).  fbm_or = 0 leaves the
  // matrix to the tail (k_matrix_codes takes each committed delta), so an
  // iteration that is run again never finds its own tuples in full.
  int row_bits = 0;
  int fbm_or = 1;
  // the previous iteration's group bitmaps (the bitmap slots are swapped after
  // every committed iteration) and, per kept value, its group index there
  // (written by the emit): from iteration 3 on the pull kernel copies a
  // group's frontier from there instead of reading its delta codes
  int prev_bm_buf = -1, prev_gi_buf = -1;
  uint32_t pull_k16 = 64;
};

// two bitmaps (frontier and full) of 2^b bits in shared memory
constexpr int kPullMaxBits = 16;
// a full kept as a bit matrix: 2^(2b) bits (512 MB at b = 16)
constexpr int kMatrixMaxBits = 16;
// default switch point, x16: a group pulls when the inner runs its next delta
// would mark exceed 4x its candidates plus the delta's size (R-MAT 16 with
// full as a bit matrix: 23.3 / 23.5 / 27.3 ms per fixpoint at 4 / 8 / 16)
constexpr uint32_t kPullK16 = 64;

// Values o with inner tuples (a non-empty run in the direct index by o), as a
// bitmap, and their number (added to cnt[nout_cnt]).
// (pull mode needs b <= 16, so the inner codes are 32-bit)
struct PullOutArgs {
  DevState* st;
  int index_buf;       // u64 [2^b + 1] direct index of the pull-ordered inner by o
  int inner_buf;       // u32 codes (o, k), sorted
  int top_index_buf;   // u64 [2^b + 1] direct index of the push-ordered inner by k
  int b;
  int out_buf;         // u32 [2^b / 32]: values o with inner tuples
  int first_buf;       // u32 [2^b]: o's first (smallest) k, 0xFFFFFFFF when none
  int tdeg_buf;        // u32 [2^b]: length of k's run in the push-ordered inner
  int nout_cnt;
};

// The values (low b bits) of the sorted codes src[r0 .. r1) into the bitmap
// `bm`, by the calling warp and the other warps of the CTA (warp of nwarps):
// each lane takes eight consecutive codes (a warp reads 1 KB per step, all
// eight loads in flight), ORs the bits of neighbours that share a word in
// registers and issues one shared-memory atomic per distinct word.
template <typename K>
__device__ __forceinline__ void sorted_run_to_bitmap(uint32_t* bm, const K* src, uint64_t r0, uint64_t r1,
                                                     uint32_t vmask, int warp, int nwarps) {
  const int lane = threadIdx.x & 31;
  for (uint64_t i = r0 + (uint64_t(warp) * 32 + lane) * 8; i < r1; i += uint64_t(nwarps) * 256) {
    uint32_t v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = i + u < r1 ? uint32_t(src[i + u]) & vmask : 0xFFFFFFFFu;
    uint32_t cw = v[0] >> 5, acc = 0;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (v[u] == 0xFFFFFFFFu) break;
      if ((v[u] >> 5) != cw) {
        if (acc & ~bm[cw]) atomicOr(&bm[cw], acc);
        cw = v[u] >> 5;
        acc = 0;
      }
      acc |= 1u << (v[u] & 31);
    }
    if (acc && (acc & ~bm[cw])) atomicOr(&bm[cw], acc);
  }
}

constexpr int kDenseThreads = 128;
constexpr int kDenseCtasPerSm = 16;   // latency-bound (L2 probes and run reads): full occupancy
constexpr int kDenseMaxBits = 18;   // bitmap of 2^18 bits = 32 KB of shared memory
// an inverted dense join reads all of its inner relation every iteration:
// only over domains of at most 2^14 values (inner relations of <= 2^28 tuples)
constexpr int kInvertMaxBits = 14;

// Group starts by one pass over a sorted array (heads of runs of equal
// g = code >> b, compacted in order by a decoupled look-back over tiles): for
// key spaces too large for a direct index (batched runs).
constexpr int kGroupThreads = 256, kGroupItems = 8, kGroupTile = kGroupThreads * kGroupItems;
template <typename K>
__global__ void __launch_bounds__(kGroupThreads) k_group_starts(GroupArgs a) {
  __shared__ uint64_t s_scan[32];
  __shared__ uint64_t s_base;
  __shared__ uint32_t s_tile;
  DevState* st = a.st;
  if (st->overflow & a.skip_mask) return;
  const uint64_t n = st->cnt[a.in_cnt];
  uint64_t* out = static_cast<uint64_t*>(st->buf[a.out_buf].ptr);
  const uint64_t ocap = st->buf[a.out_buf].cap;
  if (n == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st->cnt[a.out_cnt] = 0;
      if (ocap >= 1) out[0] = 0;
    }
    return;
  }
  const uint64_t ntiles = (n + kGroupTile - 1) / kGroupTile;
  if (st->buf[a.status_buf].cap < ntiles) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      atomicMax((unsigned long long*)&st->need[a.status_buf], (unsigned long long)ntiles);
      atomicOr(&st->overflow, 1u << a.stage_bit);
    }
    return;
  }
  const K* in = static_cast<const K*>(st->buf[a.in_buf].ptr);
  uint64_t* status = static_cast<uint64_t*>(st->buf[a.status_buf].ptr);
  const uint32_t epoch = st->epoch;
  const int tid = threadIdx.x;
  while (true) {
    if (tid == 0) s_tile = atomicAdd(&st->tile_ctr[a.ctr], 1u);
    __syncthreads();
    const uint64_t tile = s_tile;
    if (tile >= ntiles) break;
    const uint64_t i0 = tile * kGroupTile + uint64_t(tid) * kGroupItems;
    uint32_t heads = 0;
    uint64_t prev = i0 > 0 && i0 <= n ? uint64_t(in[i0 - 1]) >> a.b : ~0ull;
#pragma unroll
    for (int k = 0; k < kGroupItems; ++k) {
      const uint64_t i = i0 + k;
      if (i >= n) break;
      const uint64_t g = uint64_t(in[i]) >> a.b;
      if (i == 0 || g != prev) heads |= 1u << k;
      prev = g;
    }
    uint64_t tile_heads;
    const uint64_t excl = block_exclusive_sum<uint64_t>(__popc(heads), s_scan, &tile_heads);
    if (tid < 32) {
      const uint64_t base = lookback_warp(status, tile, tile_heads, epoch, &st->error);
      if (tid == 0) s_base = base;
    }
    __syncthreads();
    uint64_t w = s_base + excl;
#pragma unroll
    for (int k = 0; k < kGroupItems; ++k)
      if (heads & (1u << k)) {
        if (w < ocap) out[w] = i0 + k;
        ++w;
      }
    if (tile == ntiles - 1 && tid == 0) {
      const uint64_t total = s_base + tile_heads;
      st->cnt[a.out_cnt] = total;
      if (total + 1 <= ocap) out[total] = n;   // sentinel: end of the last group
      else {
        atomicMax((unsigned long long*)&st->need[a.out_buf], (unsigned long long)(total + 1));
        atomicOr(&st->overflow, 1u << a.stage_bit);
      }
    }
    __syncthreads();
  }
}

// A full kept as a bit matrix takes the new tuples of iterations >= 2 in the
// grouped join's emit (k_dense_emit: each group's bitmap ORed into the row of
// its kept value, |full_g| recounted from the row); a delta of iteration 1
// (from the sort + unique) goes in by codes here, idempotently, so a tail
// re-run after a buffer grew repeats it safely.
struct MatrixArgs {
  DevState* st;
  int groups_buf, groups_cnt;   // group starts into the outer relation
  int outer_buf;                // the outer codes (kept value in the high half)
  int bm_buf;                   // u32 [groups][2^b / 32]: each group's new tuples
  int codes_buf, codes_cnt;     // k_matrix_codes: codes (kept value high) to add
  int b;
  int fbm_buf, fcnt_buf;
  int skip_mask;
  int gate1;                    // k_matrix_codes runs only when cnt[gate1 - 1] != 0 (0: always)
  int row_bits = 0;             // bits of a row index (instance bits + b; 0: b)
};
// The same from codes (kept value in the high half): iteration 1's delta.
template <typename K>
__global__ void k_matrix_codes(MatrixArgs a) {
  DevState* st = a.st;
  if ((st->overflow & a.skip_mask) || (a.gate1 > 0 && st->cnt[a.gate1 - 1] == 0)) return;
  const uint64_t n = st->cnt[a.codes_cnt];
  const K* codes = static_cast<const K*>(st->buf[a.codes_buf].ptr);
  uint32_t* fbm = static_cast<uint32_t*>(st->buf[a.fbm_buf].ptr);
  uint32_t* fcnt = static_cast<uint32_t*>(st->buf[a.fcnt_buf].ptr);
  const uint32_t vmask = (1u << a.b) - 1;
  const uint64_t rmask = a.row_bits > 0 ? (1ull << a.row_bits) - 1 : uint64_t(vmask);
  const uint64_t nwords = a.b >= 5 ? (1ull << (a.b - 5)) : 1;
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t g = (uint64_t(codes[i]) >> a.b) & rmask;
    const uint32_t o = uint32_t(codes[i]) & vmask;
    const uint32_t bit = 1u << (o & 31);
    if (!(atomicOr(&fbm[uint64_t(g) * nwords + (o >> 5)], bit) & bit)) atomicAdd(&fcnt[g], 1u);
  }
}

// The end of a group in either direction: its bitmap `res` (the group's new
// delta) stored to its slot gbm (coalesced) and cleared, with `also` (null or
// a second bitmap) cleared beside it, its size into counts[gi].  With pull
// mode on, the inner-run lengths of the set bits are summed (what a push pass
// would mark next iteration) and the group's next mode is chosen: pull when
// that sum exceeds pull_k16 / 16 times its remaining candidates plus the
// delta's size.  Called by every thread of the CTA (blockDim.x threads).
template <typename K>
__device__ __forceinline__ void dense_finish(const DenseArgs& a, DevState* st, uint32_t* res, uint32_t* also,
                                             uint32_t* gbm, uint64_t gi, uint32_t g, int nwords,
                                             unsigned long long* s_cnt, unsigned long long* s_td) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nthreads = blockDim.x;
  const bool pull_on = a.pull_inner_buf >= 0;
  uint32_t mine = 0;
  for (int j0 = warp * 32; j0 < nwords; j0 += nthreads) {   // warp-uniform
    const int j = j0 + lane;
    const uint32_t w = j < nwords ? res[j] : 0u;
    if (j < nwords) gbm[j] = w;
    mine += __popc(w);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  if (lane == 0 && mine) atomicAdd(s_cnt, (unsigned long long)mine);
  __syncthreads();
  // the next delta's inner-run total, only where pulling could pay: the
  // delta is at least 1/16 of the candidates left (a word at a time, a lane
  // per bit, coalesced)
  uint64_t cand = 0;
  bool weigh = false;
  if (pull_on) {
    const uint64_t nout = st->cnt[a.nout_cnt];
    const uint64_t full_after = uint64_t(static_cast<const uint32_t*>(st->buf[a.fcnt_buf].ptr)[g]) + *s_cnt;
    cand = nout > full_after ? nout - full_after : 0;
    weigh = 16ull * *s_cnt >= cand && *s_cnt > 0;
  }
  unsigned long long td = 0;
  const uint32_t* tdeg = weigh ? static_cast<const uint32_t*>(st->buf[a.tdeg_buf].ptr) : nullptr;
  for (int j0 = warp * 32; j0 < nwords; j0 += nthreads) {   // warp-uniform
    const int j = j0 + lane;
    const uint32_t w = j < nwords ? res[j] : 0u;
    if (j < nwords) {
      res[j] = 0;
      if (also) also[j] = 0;
    }
    if (weigh)   // eight words' loads in flight
      for (uint32_t any = __ballot_sync(0xffffffffu, w != 0u); any;) {
        uint32_t t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int jl = any ? __ffs(any) - 1 : -1;
          any = any ? any & (any - 1) : 0u;
          const uint32_t ww = __shfl_sync(0xffffffffu, w, jl & 31);
          t[u] = jl >= 0 && ((ww >> lane) & 1u) ? tdeg[uint32_t(j0 + jl) * 32 + uint32_t(lane)] : 0u;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) td += t[u];
      }
  }
  if (weigh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) td += __shfl_xor_sync(0xffffffffu, td, o);
    if (lane == 0 && td) atomicAdd(s_td, td);
  }
  __syncthreads();
  if (tid == 0) {
    static_cast<uint64_t*>(st->buf[a.offs_buf].ptr)[gi] = *s_cnt;
    if (pull_on) {
      const bool pull_next = weigh && 16ull * *s_td > uint64_t(a.pull_k16) * cand + 16ull * *s_cnt;
      uint32_t* pbm = static_cast<uint32_t*>(st->buf[a.pull_bm_buf].ptr);
      if (pull_next) atomicOr(&pbm[g >> 5], 1u << (g & 31));
      else atomicAnd(&pbm[g >> 5], ~(1u << (g & 31)));
    }
    *s_cnt = 0;   // read again only after the next group's first barrier
    *s_td = 0;
  }
}

// Phase 0 (one CTA): units per group (ceil(size / unit_size)) -> first unit
// of each group, total units in units[groups]; done counters cleared.
template <typename K>
__global__ void k_dense_units(DenseArgs a) {
  __shared__ uint64_t s_scan[32];
  DevState* st = a.st;
  if (st->overflow & a.skip_mask) return;
  const uint64_t ngroups = st->cnt[a.groups_cnt];
  if (st->buf[a.units_buf].cap < ngroups + 1 || st->buf[a.done_buf].cap < ngroups) {
    if (threadIdx.x == 0) {
      atomicMax((unsigned long long*)&st->need[a.units_buf], (unsigned long long)(ngroups + 1));
      atomicMax((unsigned long long*)&st->need[a.done_buf], (unsigned long long)ngroups);
      atomicOr(&st->overflow, 1u << a.stage_bit);
    }
    return;
  }
  if (st->buf[a.mslot_buf].cap < ngroups + 1) {
    if (threadIdx.x == 0) {
      atomicMax((unsigned long long*)&st->need[a.mslot_buf], (unsigned long long)(ngroups + 1));
      atomicOr(&st->overflow, 1u << a.stage_bit);
    }
    return;
  }
  const uint64_t* gs = static_cast<const uint64_t*>(st->buf[a.groups_buf].ptr);
  uint64_t* units = static_cast<uint64_t*>(st->buf[a.units_buf].ptr);
  uint32_t* done = static_cast<uint32_t*>(st->buf[a.done_buf].ptr);
  uint32_t* mslot = static_cast<uint32_t*>(st->buf[a.mslot_buf].ptr);
  uint64_t carry = 0, mcarry = 0;
  for (uint64_t c0 = 0; c0 < ngroups; c0 += blockDim.x) {
    const uint64_t g = c0 + threadIdx.x;
    const uint64_t nu = g < ngroups ? (gs[g + 1] - gs[g] + a.unit_size - 1) / a.unit_size : 0;
    uint64_t tot, mtot;
    const uint64_t ex = block_exclusive_sum<uint64_t>(nu, s_scan, &tot);
    const uint64_t mex = block_exclusive_sum<uint64_t>(nu > 1 ? 1 : 0, s_scan, &mtot);
    if (g < ngroups) {
      units[g] = carry + ex;
      done[g] = 0;
      mslot[g] = uint32_t(mcarry + mex);
    }
    carry += tot;
    mcarry += mtot;
  }
  if (threadIdx.x == 0) {
    units[ngroups] = carry;
    mslot[ngroups] = uint32_t(mcarry);
    const uint64_t nwords = a.b >= 5 ? (1ull << (a.b - 5)) : 1;
    if (st->buf[a.bmm_buf].cap < mcarry * nwords) {
      atomicMax((unsigned long long*)&st->need[a.bmm_buf], (unsigned long long)(mcarry * nwords));
      atomicOr(&st->overflow, 1u << a.stage_bit);
    }
  }
}

// Phase 1: one unit per CTA (taken in any order, so a large group delays no
// other and is spread over several CTAs): mark the inner runs of the unit's
// outer tuples -- a warp takes 32 outer tuples at once (32 probes in
// flight), then its lanes stride over the concatenation of their runs, each
// element finding its run by a binary search over the warp's inclusive
// run-length prefix.  A group of one unit is finished by its CTA (set
// difference, count, store); the units of a larger group OR their bitmaps
// into the group's (zeroed) bitmap in HBM and the last one to finish
// finishes the group.
template <typename K>
__global__ void __launch_bounds__(kDenseThreads, kDenseCtasPerSm) k_dense_mark(DenseArgs a) {
  extern __shared__ __align__(16) uint32_t s_bm[];   // 2^b bits
  __shared__ unsigned long long s_cnt;
  __shared__ uint64_t s_unit[3];   // the unit's outer range [start, end) and its group
  __shared__ uint32_t s_nu;        // units in that group
  __shared__ int s_last;
  __shared__ unsigned long long s_td;
  DevState* st = a.st;
  if (st->overflow & a.skip_mask) return;
  const uint64_t ngroups = st->cnt[a.groups_cnt];
  if (ngroups == 0) return;
  const int nwords = a.b >= 5 ? (1 << (a.b - 5)) : 1;
  // (the multi-unit bitmaps' capacity is checked where the units are made)
  if (st->buf[a.bm_buf].cap < ngroups * uint64_t(nwords) || st->buf[a.offs_buf].cap < ngroups + 1) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      atomicMax((unsigned long long*)&st->need[a.bm_buf], (unsigned long long)(ngroups * uint64_t(nwords)));
      atomicMax((unsigned long long*)&st->need[a.offs_buf], (unsigned long long)(ngroups + 1));
      atomicOr(&st->overflow, 1u << a.stage_bit);
    }
    return;
  }
  const K* outer = static_cast<const K*>(st->buf[a.outer_buf].ptr);
  const uint64_t* gs = static_cast<const uint64_t*>(st->buf[a.groups_buf].ptr);
  const K* inner = static_cast<const K*>(st->buf[a.inner_buf].ptr);
  const Slot* table = static_cast<const Slot*>(st->buf[a.table_buf].ptr);
  const uint64_t tmask = st->buf[a.table_buf].cap - 1;
  uint32_t* bm = static_cast<uint32_t*>(st->buf[a.bm_buf].ptr);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int nwarps = kDenseThreads / 32;
  const uint32_t vmask = a.b >= 32 ? 0xFFFFFFFFu : ((1u << a.b) - 1);
  for (int j = tid; j < nwords; j += kDenseThreads) s_bm[j] = 0;
  if (tid == 0) {
    s_cnt = 0;
    s_td = 0;
  }
  unsigned long long raw = 0;
  while (true) {
    // one thread finds the unit (its group: the last g with units[g] <= ui)
    // and hands it to the CTA through shared memory, which keeps the
    // marking loop's registers as they are without units
    if (tid == 0) {
      const uint64_t* units = static_cast<const uint64_t*>(st->buf[a.units_buf].ptr);
      const uint64_t ui = atomicAdd(&st->tile_ctr[a.ctr], 1u);
      uint64_t gi = ~0ull;
      if (ui < units[ngroups]) {
        uint64_t lo = 0, hi = ngroups;
        while (hi - lo > 1) {
          const uint64_t m = (lo + hi) >> 1;
          if (units[m] <= ui) lo = m;
          else hi = m;
        }
        gi = lo;
        const uint64_t s = gs[gi] + (ui - units[gi]) * uint64_t(a.unit_size);
        s_unit[0] = s;
        s_unit[1] = min(gs[gi + 1], s + uint64_t(a.unit_size));
        s_nu = uint32_t(units[gi + 1] - units[gi]);
      }
      s_unit[2] = gi;
    }
    __syncthreads();
    if (s_unit[2] == ~0ull) break;
    const uint64_t gi = s_unit[2];
    uint32_t* gbm = bm + gi * uint64_t(nwords);
    // a unit spans at most unit_size (< 2^31) outer tuples: 32-bit offsets
    const K* uo = outer + s_unit[0];
    const uint32_t un = uint32_t(s_unit[1] - s_unit[0]);
    for (uint32_t ob = uint32_t(warp) * 32; ob < un; ob += uint32_t(nwarps) * 32) {
      const uint32_t o = ob + lane;
      uint64_t begin = 0;
      uint32_t len = 0;
      if (o < un) {
        const K code = uo[o];
        const uint32_t key = join_key(inst_of(code, a.b), colv(code, 1, a.b), a.b);
        if (!probe_run(table, tmask, a.index_direct, key, &begin, &len, &st->error)) len = 0;
      }
      // runs of at least 32 values are walked by the whole warp one after
      // another: coalesced, no per-value search for the run, and a sorted
      // run's neighbouring values mostly share a bitmap word
      for (uint32_t lm = __ballot_sync(0xffffffffu, len >= 32); lm; lm &= lm - 1) {
        const int l = __ffs(lm) - 1;
        const uint64_t rb = __shfl_sync(0xffffffffu, begin, l);
        const uint32_t rn = __shfl_sync(0xffffffffu, len, l);
        if (lane == 0) raw += rn;
        for (uint32_t i0 = 0; i0 < rn; i0 += 128) {
          uint32_t v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const uint32_t i = i0 + uint32_t(u) * 32 + lane;
            v[u] = i < rn ? uint32_t(inner[rb + i]) & vmask : 0xFFFFFFFFu;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (v[u] == 0xFFFFFFFFu) continue;
            const uint32_t bit = 1u << (v[u] & 31);
            if (!(s_bm[v[u] >> 5] & bit)) atomicOr(&s_bm[v[u] >> 5], bit);
          }
        }
      }
      if (len >= 32) len = 0;
      // the short runs concatenated: each value finds its run by a binary
      // search over the warp's inclusive run-length prefix
      uint32_t incl = len;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
      }
      const uint32_t excl = incl - len;
      const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
      if (lane == 0) raw += total;
      // four elements per lane per step: all four loads are in flight
      // before any is marked
      for (uint32_t q0 = 0; q0 < total; q0 += 128) {
        uint32_t v[4];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const uint32_t q = q0 + uint32_t(u) * 32 + lane;
          int owner = 0;   // lanes whose inclusive prefix is <= q
#pragma unroll
          for (int step = 16; step >= 1; step >>= 1) {
            const uint32_t x = __shfl_sync(0xffffffffu, incl, owner + step - 1);
            if (x <= q) owner += step;
          }
          const uint64_t ob_begin = __shfl_sync(0xffffffffu, begin, owner & 31);
          const uint32_t ob_excl = __shfl_sync(0xffffffffu, excl, owner & 31);
          ok[u] = q < total;
          v[u] = ok[u] ? uint32_t(inner[ob_begin + (q - ob_excl)]) & vmask : 0u;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (!ok[u]) continue;
          const uint32_t bit = 1u << (v[u] & 31);
          // most values are marked already (many outer tuples share inner
          // values): a plain read skips the serialised same-word atomics
          if (!(s_bm[v[u] >> 5] & bit)) atomicOr(&s_bm[v[u] >> 5], bit);
        }
      }
    }
    __syncthreads();
    if (s_nu > 1) {
      // this unit's marks into the group's multi-unit bitmap; the last unit
      // takes it back (leaving it zeroed) and finishes the group
      const uint32_t nu = s_nu;
      uint32_t* done = static_cast<uint32_t*>(st->buf[a.done_buf].ptr);
      uint32_t* mbm = static_cast<uint32_t*>(st->buf[a.bmm_buf].ptr) +
                      uint64_t(static_cast<const uint32_t*>(st->buf[a.mslot_buf].ptr)[gi]) * nwords;
      for (int j = tid; j < nwords; j += kDenseThreads) {
        const uint32_t w = s_bm[j];
        if (w) atomicOr(&mbm[j], w);
        s_bm[j] = 0;
      }
      __threadfence();
      __syncthreads();
      if (tid == 0) s_last = atomicAdd(&done[gi], 1u) == nu - 1;
      __syncthreads();
      if (!s_last) continue;
      __threadfence();
      for (int j = tid; j < nwords; j += kDenseThreads) {
        s_bm[j] = __ldcg(&mbm[j]);
        mbm[j] = 0;
      }
      __syncthreads();
    }
    // set difference against full (Section 5.1 "populating delta"): clear the
    // bits of the group's tuples already in full; every level holds the kept
    // value first, so each contributes one contiguous run
    if (a.drop_self && tid == 0) {
      const uint32_t g = uint32_t(uint64_t(outer[gs[gi]]) >> a.b) & vmask;
      atomicAnd(&s_bm[g >> 5], ~(1u << (g & 31)));
    }
    if (a.fbm_buf >= 0) {   // full as a bit matrix: clear the bits of the group's row
      const uint64_t rmask = a.row_bits > 0 ? (1ull << a.row_bits) - 1 : uint64_t(vmask);
      const uint64_t g = (uint64_t(outer[gs[gi]]) >> a.b) & rmask;
      const uint32_t* row = static_cast<const uint32_t*>(st->buf[a.fbm_buf].ptr) + g * uint64_t(nwords);
      for (int j = tid; j < nwords; j += kDenseThreads) {   // atomic: the filter above may clear a bit too
        const uint32_t f = row[j];
        if (s_bm[j] & f) atomicAnd(&s_bm[j], ~f);
      }
    }
    if (a.full_buf >= 0) {
      const uint64_t nlv = st->cnt[a.nlv_cnt], nk = (1ull << a.b) + 1;
      const uint64_t* lvidx = static_cast<const uint64_t*>(st->buf[a.lvidx_buf].ptr);
      const K* fl = static_cast<const K*>(st->buf[a.full_buf].ptr);
      const uint64_t g = uint64_t(outer[gs[gi]]) >> a.b;
      for (uint64_t lv = 0; lv < nlv; ++lv) {
        const uint64_t r0 = lvidx[lv * nk + g], r1 = lvidx[lv * nk + g + 1];
        if (r1 - r0 <= 4 * kDenseThreads) {   // a short run: one pass
          for (uint64_t i = r0 + tid; i < r1; i += kDenseThreads) {
            const uint32_t v = uint32_t(fl[i]) & vmask;
            const uint32_t bit = 1u << (v & 31);
            if (s_bm[v >> 5] & bit) atomicAnd(&s_bm[v >> 5], ~bit);
          }
          continue;
        }
        // eight loads in flight per thread: the level runs come from HBM
        for (uint64_t i0 = r0 + tid; i0 < r1; i0 += 8 * kDenseThreads) {
          uint32_t v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const uint64_t i = i0 + uint64_t(u) * kDenseThreads;
            v[u] = i < r1 ? uint32_t(fl[i]) & vmask : 0xFFFFFFFFu;
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            if (v[u] == 0xFFFFFFFFu) continue;
            const uint32_t bit = 1u << (v[u] & 31);
            if (s_bm[v[u] >> 5] & bit) atomicAnd(&s_bm[v[u] >> 5], ~bit);
          }
        }
      }
    }
    __syncthreads();
    dense_finish<K>(a, st, s_bm, nullptr, gbm, gi, uint32_t(uint64_t(outer[gs[gi]]) >> a.b) & vmask, nwords, &s_cnt,
                    &s_td);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) raw += __shfl_xor_sync(0xffffffffu, raw, o);
  if (lane == 0 && raw) atomicAdd((unsigned long long*)&st->cnt[a.raw_cnt], raw);
}

// Pull mode (see DenseArgs): one CTA per listed group.  The group's delta
// values go into a frontier bitmap F and full's tuples of the group into V
// (both sorted, so a warp combines the bits of one word before its atomic);
// every candidate -- a value with inner tuples, not in V -- is new if one of
// its inner tuples (o, k) has k in F.  A warp takes a candidate word at a time,
// a lane per candidate: its first inner tuple (the smallest k, precomputed;
// coalesced over the word) decides most of them, eight words in flight; then
// each lane scans the rest of the runs of its own word's undecided candidates,
// four tuples at a time until one k is in F, 32 words at once.
constexpr int kPullCtasPerSm = 10;   // two bitmaps of up to 8 KB each; 48 registers
template <typename K>
__global__ void __launch_bounds__(kDenseThreads, kPullCtasPerSm) k_dense_pull(DenseArgs a) {
  extern __shared__ __align__(16) uint32_t s_bm[];   // F, then V (2^b bits each)
  __shared__ unsigned long long s_cnt, s_td;
  __shared__ uint64_t s_gi;
  DevState* st = a.st;
  if ((st->overflow & a.skip_mask) || a.pull_inner_buf < 0) return;
  const uint64_t ngroups = st->cnt[a.groups_cnt];
  const uint64_t npull = st->cnt[a.pull_cnt];
  const int nwords = a.b >= 5 ? (1 << (a.b - 5)) : 1;
  if (npull == 0 || st->buf[a.bm_buf].cap < ngroups * uint64_t(nwords) || st->buf[a.offs_buf].cap < ngroups + 1)
    return;   // (k_dense_mark reports the capacities; this launch follows it)
  const K* outer = static_cast<const K*>(st->buf[a.outer_buf].ptr);
  const uint64_t* gs = static_cast<const uint64_t*>(st->buf[a.groups_buf].ptr);
  const uint32_t* plist = static_cast<const uint32_t*>(st->buf[a.plist_buf].ptr);
  const K* pin = static_cast<const K*>(st->buf[a.pull_inner_buf].ptr);
  const uint64_t* pidx = static_cast<const uint64_t*>(st->buf[a.pull_index_buf].ptr);
  const uint32_t* outbm = static_cast<const uint32_t*>(st->buf[a.pull_out_buf].ptr);
  const uint32_t* firstk = static_cast<const uint32_t*>(st->buf[a.pull_first_buf].ptr);
  uint32_t* bm = static_cast<uint32_t*>(st->buf[a.bm_buf].ptr);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int nwarps = kDenseThreads / 32;
  const uint32_t vmask = (1u << a.b) - 1;
  uint32_t* F = s_bm;
  uint32_t* V = s_bm + nwords;
  for (int j = tid; j < 2 * nwords; j += kDenseThreads) s_bm[j] = 0;
  if (tid == 0) {
    s_cnt = 0;
    s_td = 0;
  }
  unsigned long long raw = 0;
  while (true) {
    if (tid == 0) {
      const uint64_t i = atomicAdd(&st->tile_ctr[a.ctr + 1], 1u);
      s_gi = i < npull ? uint64_t(plist[i]) : ~0ull;
    }
    __syncthreads();
    const uint64_t gi = s_gi;
    if (gi == ~0ull) break;
    const uint64_t o0 = gs[gi], o1 = gs[gi + 1];
    const uint32_t g = uint32_t(uint64_t(outer[o0]) >> a.b) & vmask;
    if (tid == 0) raw += o1 - o0;
    if (a.prev_bm_buf >= 0 && st->iter >= 2) {   // the delta as last iteration's bitmap of the group
      const uint32_t pgi = static_cast<const uint32_t*>(st->buf[a.prev_gi_buf].ptr)[g];
      const uint32_t* src = static_cast<const uint32_t*>(st->buf[a.prev_bm_buf].ptr) + uint64_t(pgi) * nwords;
      for (int j = tid; j < nwords; j += kDenseThreads) F[j] = src[j];
    } else {
      sorted_run_to_bitmap<K>(F, outer, o0, o1, vmask, warp, nwarps);
    }
    if (a.full_buf >= 0) {
      const uint64_t nlv = st->cnt[a.nlv_cnt], nk = (1ull << a.b) + 1;
      const uint64_t* lvidx = static_cast<const uint64_t*>(st->buf[a.lvidx_buf].ptr);
      const K* fl = static_cast<const K*>(st->buf[a.full_buf].ptr);
      for (uint64_t lv = 0; lv < nlv; ++lv) {
        const uint64_t r0 = lvidx[lv * nk + g], r1 = lvidx[lv * nk + g + 1];
        if (tid == 0) raw += r1 - r0;
        sorted_run_to_bitmap<K>(V, fl, r0, r1, vmask, warp, nwarps);
      }
    }
    __syncthreads();
    const uint32_t* frow = a.fbm_buf >= 0 ? static_cast<const uint32_t*>(st->buf[a.fbm_buf].ptr) + g * uint64_t(nwords)
                                          : V;   // full of the group as bits
    for (int base = warp * 32; base < nwords; base += nwarps * 32) {
      const int wl = base + lane;
      const uint32_t cm_l = wl < nwords ? (outbm[wl] & ~frow[wl]) : 0u;
      uint32_t any = __ballot_sync(0xffffffffu, cm_l != 0u);
      uint32_t r_l = 0, m_l = 0;   // this lane's word: hits, and misses of the first tuple
      // first tuples: a word at a time, a lane per candidate, eight words in flight
      while (any) {
        int jl[8];
        uint32_t kf[8];
        bool mine[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          jl[u] = any ? __ffs(any) - 1 : -1;
          any = any ? any & (any - 1) : 0u;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const uint32_t cm = __shfl_sync(0xffffffffu, cm_l, jl[u] & 31);
          mine[u] = jl[u] >= 0 && ((cm >> lane) & 1u);
          kf[u] = mine[u] ? firstk[uint32_t(base + jl[u]) * 32 + uint32_t(lane)] : 0u;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const bool hit = mine[u] && ((F[kf[u] >> 5] >> (kf[u] & 31)) & 1u);
          raw += mine[u];
          const uint32_t hb = __ballot_sync(0xffffffffu, hit), mb = __ballot_sync(0xffffffffu, mine[u] && !hit);
          if (lane == jl[u]) {
            r_l = hb;
            m_l = mb;
          }
        }
      }
      // the misses: every lane scans the rest of its own word's candidates'
      // runs, four tuples at a time, the 32 words of the warp at once
      for (uint32_t mm = m_l; mm; mm &= mm - 1) {
        const uint32_t bit = uint32_t(__ffs(mm) - 1);
        const uint32_t o = uint32_t(wl) * 32 + bit;
        uint64_t p = pidx[o] + 1;
        const uint64_t pe = pidx[o + 1];
        bool hit = false;
        while (p < pe && !hit) {
          uint32_t k[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) k[q] = p + q < pe ? uint32_t(pin[p + q]) & vmask : 0xFFFFFFFFu;
#pragma unroll
          for (int q = 0; q < 4; ++q) hit = hit || (k[q] != 0xFFFFFFFFu && ((F[k[q] >> 5] >> (k[q] & 31)) & 1u));
          raw += min(uint64_t(4), pe - p);
          p += 4;
        }
        if (hit) r_l |= 1u << bit;
      }
      if (wl < nwords) V[wl] = r_l;   // the results replace the word of V
    }
    __syncthreads();
    if (a.drop_self && tid == 0) V[g >> 5] &= ~(1u << (g & 31));
    __syncthreads();
    dense_finish<K>(a, st, V, F, bm + gi * uint64_t(nwords), gi, g, nwords, &s_cnt, &s_td);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) raw += __shfl_xor_sync(0xffffffffu, raw, o);
  if (lane == 0 && raw) atomicAdd((unsigned long long*)&st->cnt[a.pull_raw_cnt], raw);
}

// Phase 2 (one CTA): counts -> exclusive offsets; total and capacity check.
template <typename K>
__global__ void __launch_bounds__(1024) k_dense_scan(DenseArgs a) {
  __shared__ uint64_t s_scan[33];
  DevState* st = a.st;
  if (st->overflow & a.skip_mask) return;
  const uint64_t ngroups = st->cnt[a.groups_cnt];
  uint64_t* offs = static_cast<uint64_t*>(st->buf[a.offs_buf].ptr);
  const uint64_t carry = cta_scan_inplace(offs, ngroups, s_scan);
  if (threadIdx.x == 0) {
    st->cnt[a.total_cnt] = carry;
    const uint64_t out0 = st->cnt[a.out_cnt];
    if (out0 + carry > st->buf[a.out_buf].cap) {
      atomicMax((unsigned long long*)&st->need[a.out_buf], (unsigned long long)(out0 + carry));
      atomicOr(&st->overflow, 1u << a.stage_bit);
    }
  }
}

// Phase 3: each group's set bits, in order, at its offset (groups in any
// order).  Each warp owns a contiguous quarter of the group's bitmap: a first
// coalesced pass counts its bits (the warps' counts give their bases), a
// second pass takes 32 words per step, stages the step's values in shared
// memory and writes them out coalesced.
template <typename K>
__global__ void __launch_bounds__(kDenseThreads) k_dense_emit(DenseArgs a) {
  constexpr int nwarps = kDenseThreads / 32;
  __shared__ K s_stage[nwarps][32 * 32];          // one 32-word step of a warp
  __shared__ uint32_t s_wtot[nwarps];
  DevState* st = a.st;
  if (st->overflow & a.skip_mask) return;
  const uint64_t ngroups = st->cnt[a.groups_cnt];
  const int nwords = a.b >= 5 ? (1 << (a.b - 5)) : 1;
  const int wrange = (nwords + nwarps - 1) / nwarps;        // words per warp
  const K* outer = static_cast<const K*>(st->buf[a.outer_buf].ptr);
  const uint64_t* gs = static_cast<const uint64_t*>(st->buf[a.groups_buf].ptr);
  const uint32_t* bm = static_cast<const uint32_t*>(st->buf[a.bm_buf].ptr);
  const uint64_t* offs = static_cast<const uint64_t*>(st->buf[a.offs_buf].ptr);
  K* out = static_cast<K*>(st->buf[a.out_buf].ptr) + st->cnt[a.out_cnt];
  // a full kept as a bit matrix takes the group's new tuples here, and |full_g|
  // grows by their count: this launch runs once per committed iteration (only
  // when the join stage did not overflow, and nothing after it in that stage
  // can: the matrix is kept for single-relation programs only)
  uint32_t* fbm = a.fbm_buf >= 0 && a.fbm_or ? static_cast<uint32_t*>(st->buf[a.fbm_buf].ptr) : nullptr;
  uint32_t* fcnt = fbm ? static_cast<uint32_t*>(st->buf[a.fcnt_buf].ptr) : nullptr;
  const uint32_t vmask = a.b >= 32 ? 0xFFFFFFFFu : ((1u << a.b) - 1);
  const uint64_t rmask = a.row_bits > 0 ? (1ull << a.row_bits) - 1 : uint64_t(vmask);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (uint64_t gi = blockIdx.x; gi < ngroups; gi += gridDim.x) {
    const uint64_t gcode = uint64_t(outer[gs[gi]]) >> a.b;   // (inst, g): the result's high part
    const uint32_t* gbm = bm + gi * uint64_t(nwords);
    uint32_t* row = fbm ? fbm + (gcode & rmask) * nwords : nullptr;
    const int w0 = warp * wrange, w1 = min(nwords, w0 + wrange);
    uint32_t cnt = 0;
    for (int j = w0 + lane; j < w1; j += 32) {
      const uint32_t x = gbm[j];
      cnt += __popc(x);
      if (row && x) row[j] |= x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0) s_wtot[warp] = cnt;
    __syncthreads();
    if (row && tid == 0) {
      uint32_t t = 0;
      for (int w = 0; w < nwarps; ++w) t += s_wtot[w];
      fcnt[gcode & rmask] += t;
    }
    if (a.prev_gi_buf >= 0 && tid == 0)
      static_cast<uint32_t*>(st->buf[a.prev_gi_buf].ptr)[uint32_t(gcode) & vmask] = uint32_t(gi);
    uint64_t base = offs[gi];
    for (int w = 0; w < warp; ++w) base += s_wtot[w];
    for (int j0 = w0; j0 < w1; j0 += 32) {
      const int j = j0 + lane;
      const uint32_t bits = j < w1 ? gbm[j] : 0u;
      const uint32_t c = __popc(bits);
      uint32_t incl = c;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
      }
      const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
      if (tot == 0) continue;
      uint32_t pos = incl - c;
      const uint32_t vbase = uint32_t(j) * 32u;
      uint32_t rest = bits;
      while (rest) {
        const int t = __ffs(rest) - 1;
        rest &= rest - 1;
        s_stage[warp][pos++] = K((gcode << a.b) | uint64_t(vbase + uint32_t(t)));
      }
      __syncwarp();
      for (uint32_t i = lane; i < tot; i += 32) out[base + i] = s_stage[warp][i];
      __syncwarp();
      base += tot;
    }

    __syncthreads();   // s_wtot is rewritten by the next group
  }
}

// Reading an append-only full (one sorted level per iteration, every level
// keeping the group column first, levels disjoint) in lexicographic order
// without sorting it: a CTA per group value g marks the group's runs of all
// levels in a shared bitmap and writes its set bits in order, decoded into
// the two output columns, at the group's offset sum over levels of
// lvidx[lv][g] - lvidx[lv][0].  Reads full once and writes the output once
// (coalesced), so a read into page-locked host columns runs at the host
// link's rate.
struct LevelsReadArgs {
  DevState* st;
  int full_buf, lvidx_buf, nlv_cnt;
  int b;
  uint32_t* out0;   // device or host-mapped; |full| entries each
  uint32_t* out1;
};
constexpr int kLevelsChunk = kDenseThreads;   // levels whose run bounds are staged at once

template <typename K>
__global__ void __launch_bounds__(kDenseThreads) k_levels_read(LevelsReadArgs a) {
  constexpr int nwarps = kDenseThreads / 32;
  extern __shared__ __align__(16) uint32_t s_dyn[];   // bitmap (2^b bits), then the warps' staging
  __shared__ uint64_t s_r0[kLevelsChunk], s_r1[kLevelsChunk];
  __shared__ unsigned long long s_off, s_cnt;
  __shared__ uint32_t s_wtot[nwarps];
  DevState* st = a.st;
  const int nwords = a.b >= 5 ? (1 << (a.b - 5)) : 1;
  uint32_t* s_bm = s_dyn;
  uint32_t* s_stage = s_dyn + nwords;   // [nwarps][1024]
  const uint64_t nk1 = (1ull << a.b) + 1, ng = 1ull << a.b;
  const uint64_t nlv = st->cnt[a.nlv_cnt];
  const uint64_t* lvidx = static_cast<const uint64_t*>(st->buf[a.lvidx_buf].ptr);
  const K* fl = static_cast<const K*>(st->buf[a.full_buf].ptr);
  const uint32_t vmask = a.b >= 32 ? 0xFFFFFFFFu : ((1u << a.b) - 1);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int j = tid; j < nwords; j += kDenseThreads) s_bm[j] = 0;
  if (tid == 0) s_off = s_cnt = 0;
  __syncthreads();
  for (uint64_t g = blockIdx.x; g < ng; g += gridDim.x) {
    // mark every level's run of g (levels staged kLevelsChunk at a time)
    for (uint64_t l0 = 0; l0 < nlv; l0 += kLevelsChunk) {
      const uint64_t lv = l0 + tid;
      unsigned long long off = 0, cnt = 0;
      if (lv < nlv) {
        const uint64_t r0 = lvidx[lv * nk1 + g], r1 = lvidx[lv * nk1 + g + 1];
        s_r0[tid] = r0;
        s_r1[tid] = r1;
        off = r0 - lvidx[lv * nk1];
        cnt = r1 - r0;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        off += __shfl_xor_sync(0xffffffffu, off, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
      }
      if (lane == 0 && (off || cnt)) {
        atomicAdd(&s_off, off);
        atomicAdd(&s_cnt, cnt);
      }
      __syncthreads();
      const int nl = int(min(uint64_t(kLevelsChunk), nlv - l0));
      for (int l = 0; l < nl; ++l)
        for (uint64_t i = s_r0[l] + tid; i < s_r1[l]; i += kDenseThreads) {
          const uint32_t v = uint32_t(fl[i]) & vmask;
          atomicOr(&s_bm[v >> 5], 1u << (v & 31));
        }
      __syncthreads();
    }
    const uint64_t base0 = s_off, total = s_cnt;
    if (total) {
      // emit: each warp owns a contiguous part of the bitmap; count, then
      // 32 words per step staged and written coalesced; words cleared
      const int wrange = (nwords + nwarps - 1) / nwarps;
      const int w0 = min(nwords, warp * wrange), w1 = min(nwords, w0 + wrange);
      uint32_t c = 0;
      for (int j = w0 + lane; j < w1; j += 32) c += __popc(s_bm[j]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
      if (lane == 0) s_wtot[warp] = c;
      __syncthreads();
      uint64_t base = base0;
      for (int w = 0; w < warp; ++w) base += s_wtot[w];
      uint32_t* stage = s_stage + warp * 1024;
      for (int j0 = w0; j0 < w1; j0 += 32) {
        const int j = j0 + lane;
        const uint32_t bits = j < w1 ? s_bm[j] : 0u;
        if (j < w1) s_bm[j] = 0;
        const uint32_t pc = __popc(bits);
        uint32_t incl = pc;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
          if (lane >= d) incl += y;
        }
        const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
        if (tot == 0) continue;
        uint32_t pos = incl - pc;
        uint32_t rest = bits;
        while (rest) {
          const int t = __ffs(rest) - 1;
          rest &= rest - 1;
          stage[pos++] = uint32_t(j) * 32u + uint32_t(t);
        }
        __syncwarp();
        for (uint32_t i = lane; i < tot; i += 32) {
          a.out0[base + i] = uint32_t(g);
          a.out1[base + i] = stage[i];
        }
        __syncwarp();
        base += tot;
      }
    }
    __syncthreads();   // s_wtot, s_off, s_cnt reused by the next group
    if (tid == 0) s_off = s_cnt = 0;
    __syncthreads();
  }
}

}  // namespace hisa
