// Control kernels: stage bookkeeping, the iteration commit (fixpoint test) and
// buffer zeroing.  All read and write only the device-resident DevState, so a
// captured iteration replays without host involvement.
#include "kernels.cuh"

namespace hisa {

__global__ void k_ctl(CtlArgs a) {
  DevState* st = a.st;
  if (st->overflow & a.skip_mask) return;
  for (int i = 0; i < a.n; ++i) {
    const CtlCmd c = a.cmd[i];
    if (c.op == kCtlZeroSmall) {
      uint64_t* p = static_cast<uint64_t*>(st->buf[c.a].ptr);
      for (long long j = threadIdx.x; j < c.b; j += blockDim.x) p[j] = 0;
      continue;
    }
    if (threadIdx.x != 0) continue;
    switch (c.op) {
      case kCtlEpoch: st->epoch = st->epoch + 1; break;
      case kCtlResetCtr: st->tile_ctr[c.a] = 0; break;
      case kCtlSetCnt: st->cnt[c.a] = uint64_t(c.b); break;
      case kCtlAddCnt: st->cnt[c.a] += st->cnt[c.b]; break;
      case kCtlCopyCnt: st->cnt[c.a] = st->cnt[c.b]; break;
      case kCtlSwapIfCnt:
        if (st->cnt[c.c] > 0) {
          const DBuf t = st->buf[c.a];
          st->buf[c.a] = st->buf[c.b];
          st->buf[c.b] = t;
          st->cnt[c.a] = st->cnt[c.b];
        }
        break;
      case kCtlCheckTable: {
        // runs * 1024 <= cap * lf1024, else ask for a larger power of two
        const uint64_t runs = st->cnt[c.b], cap = st->buf[c.a].cap;
        if (runs * 1024ull > cap * uint64_t(c.c)) {
          atomicMax((unsigned long long*)&st->need[c.a], (unsigned long long)((runs * 1024ull) / uint64_t(c.c) + 1));
          atomicOr(&st->overflow, 1u);
        }
        break;
      }
      case kCtlMergeGate: {
        // log-structured full: the small level is merged into the large one
        // once it holds more than 1/ratio of it, or before new is merged
        // straight into the large level
        const uint64_t small = st->cnt[c.b], large = st->cnt[int(c.c >> 32)];
        const bool forced = st->cnt[int((c.c >> 16) & 0xFFFF)] != 0;
        st->cnt[c.a] = (small * uint64_t(c.c & 0xFFFF) > large || forced) ? small : 0;
        break;
      }
      case kCtlBigFlag:
        st->cnt[c.a] = st->cnt[c.b] * uint64_t(c.c & 0xFFFF) > st->cnt[int(c.c >> 16)] ? 1 : 0;
        break;
      case kCtlNot:
        st->cnt[c.a] = st->cnt[c.b] ? 0 : 1;
        break;
      case kCtlSwap: {
        const DBuf t = st->buf[c.a];
        st->buf[c.a] = st->buf[int(c.b)];
        st->buf[int(c.b)] = t;
        break;
      }
      case kCtlZeroIfCnt:
        if (st->cnt[c.c] > 0) st->cnt[c.a] = 0;
        break;
      default: st->error = kDevBadState; break;
    }
  }
}

// End of an iteration (Section 5.1 "Merging Full with Delta and Clearing New"
// and the fixpoint check): unless a stage overflowed, the new full and delta
// versions become current, |delta_k| is appended to each relation's history,
// and the loop continues while some delta is non-empty.
__global__ void k_commit(CommitArgs a) {
  DevState* st = a.st;
  if (threadIdx.x != 0) return;
  if (st->overflow || st->error) {
    st->go = 0;
    return;
  }
  bool any = false;
  const uint32_t it = st->iter;
  for (int r = 0; r < a.nrel; ++r) {
    const uint64_t nd = st->cnt[a.delta_next[r]];
    if (nd > 0 && a.append_nlv1[r] > 0) {
      // delta was appended to full as a new level
      st->cnt[a.full[r]] += nd;
      const uint64_t lv = ++st->cnt[a.append_nlv1[r] - 1];
      if (lv >= uint64_t(a.max_levels)) st->aux[2] = 1;   // the host merges the levels
      any = true;
    } else if (nd > 0) {
      const bool alt = a.alt_flag1[r] > 0 && st->cnt[a.alt_flag1[r] - 1] != 0;
      const int f = alt ? a.alt_full[r] : a.full[r], fn = alt ? a.alt_full_next[r] : a.full_next[r];
      DBuf t = st->buf[f];
      st->buf[f] = st->buf[fn];
      st->buf[fn] = t;
      st->cnt[f] = st->cnt[fn];
      any = true;
    }
    DBuf t = st->buf[a.delta[r]];
    st->buf[a.delta[r]] = st->buf[a.delta_next[r]];
    st->buf[a.delta_next[r]] = t;
    st->cnt[a.delta[r]] = nd;
    DBuf h = st->buf[a.history[r]];
    if (it < h.cap) static_cast<uint64_t*>(h.ptr)[it] = nd;
    st->aux[1] += st->cnt[a.fresh[r]];   // tuples joined (|new| before dedup)
  }
  st->iter = it + 1;
  st->go = (any || a.force) && st->iter < st->max_iters && !st->aux[2] ? 1u : 0u;
  if (any) st->aux[0] = st->iter;   // last iteration that produced a tuple
}

__global__ void k_zero(ZeroArgs a) {
  DevState* st = a.st;
  if (st->overflow & a.skip_mask) return;
  const uint64_t words = st->buf[a.buf].cap * uint64_t(a.elem_bytes) / 16;
  uint4* p = static_cast<uint4*>(st->buf[a.buf].ptr);
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < words; i += uint64_t(gridDim.x) * blockDim.x)
    p[i] = make_uint4(0, 0, 0, 0);
}

__global__ void k_fill_u32(uint32_t* p, uint64_t n, uint32_t v) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x)
    p[i] = v;
}
void launch_fill_u32(uint32_t* p, uint64_t n, uint32_t v, const Grid& g, cudaStream_t s) {
  HISA_LAUNCH(kKZero, s, (k_fill_u32<<<g.small, 256, 0, s>>>(p, n, v)));
}

// Group starts from a direct index over the delta's kept column (first[g]
// for g in [0, 2^bits], GroupArgs::in_buf): the non-empty groups' starts in
// order, then the sentinel n.  One CTA walks the 2^bits keys.
__global__ void k_group_compact(GroupArgs a, int bits) {
  __shared__ uint64_t s_scan[32];
  DevState* st = a.st;
  if (st->overflow & a.skip_mask) return;
  const uint64_t* first = static_cast<const uint64_t*>(st->buf[a.in_buf].ptr);
  uint64_t* out = static_cast<uint64_t*>(st->buf[a.out_buf].ptr);
  const uint64_t ocap = st->buf[a.out_buf].cap;
  const uint64_t nk = 1ull << bits;
  uint64_t carry = 0;
  for (uint64_t c0 = 0; c0 < nk; c0 += blockDim.x) {
    const uint64_t g = c0 + threadIdx.x;
    const bool head = g < nk && first[g + 1] > first[g];
    uint64_t tot;
    const uint64_t ex = block_exclusive_sum<uint64_t>(head ? 1 : 0, s_scan, &tot);
    if (head && carry + ex < ocap) out[carry + ex] = first[g];
    carry += tot;
  }
  if (threadIdx.x == 0) {
    st->cnt[a.out_cnt] = carry;
    if (carry + 1 <= ocap) out[carry] = first[nk];
    else {
      atomicMax((unsigned long long*)&st->need[a.out_buf], (unsigned long long)(carry + 1));
      atomicOr(&st->overflow, 1u << a.stage_bit);
    }
  }
}

void launch_ctl(const CtlArgs& a, cudaStream_t s) { HISA_LAUNCH(kKCtl, s, (k_ctl<<<1, 256, 0, s>>>(a))); }
void launch_group_compact(const GroupArgs& a, int bits, cudaStream_t s) {
  HISA_LAUNCH(kKGroups, s, (k_group_compact<<<1, 1024, 0, s>>>(a, bits)));
}
void launch_commit(const CommitArgs& a, cudaStream_t s) { HISA_LAUNCH(kKCommit, s, (k_commit<<<1, 32, 0, s>>>(a))); }
void launch_zero(const ZeroArgs& a, const Grid& g, cudaStream_t s) {
  HISA_LAUNCH(kKZero, s, (k_zero<<<g.small, 256, 0, s>>>(a)));
}

const char* const kKernelNames[kKindCount] = {
    "encode", "decode", "count_runs", "radix_hist", "radix_pass", "setop_partition", "setop_diff_merge",
    "index_build", "join_count", "join_partition", "join_write", "ctl", "commit", "zero", "swap_cols", "setop_diff_probe", "group_compact", "join_dense_mark", "join_dense_scan", "join_dense_emit", "append_level"};

thread_local KernelTimer* g_timer = nullptr;
thread_local uint64_t g_launches = 0;

cudaEvent_t KernelTimer::get() {
  if (used == pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    pool.push_back(e);
  }
  return pool[used++];
}
void KernelTimer::begin(int kind, cudaStream_t s) {
  Rec r{kind, get(), get()};
  cudaEventRecord(r.a, s);
  recs.push_back(r);
}
void KernelTimer::end(cudaStream_t s) { cudaEventRecord(recs.back().b, s); }
void KernelTimer::truncate(size_t n) {
  if (n < recs.size()) {
    recs.resize(n);
    used = 2 * n;
  }
}
void KernelTimer::reset() {
  recs.clear();
  used = 0;
}
KernelTimer::~KernelTimer() {
  for (auto e : pool) cudaEventDestroy(e);
}

}  // namespace hisa
