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
    if (nd > 0 && a.add_full[r]) {
      // delta was ORed into full's bit matrix
      st->cnt[a.full[r]] += nd;
      any = true;
    } else if (nd > 0 && a.append_nlv1[r] > 0) {
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
// order, then the sentinel n.  One CTA: each warp takes a contiguous range of
// keys, read coalesced with eight loads in flight per lane, counts it, and
// after a scan over the warps' counts writes it.
__global__ void __launch_bounds__(1024) k_group_compact(GroupArgs a, int bits) {
  __shared__ uint64_t s_gm[33], s_nu[33], s_pl[33];
  constexpr int kB = 8;   // 32-key chunks loaded before any is used
  DevState* st = a.st;
  if (st->overflow & a.skip_mask) return;
  const uint64_t* first = static_cast<const uint64_t*>(st->buf[a.in_buf].ptr);
  const uint64_t* vals = a.indirect ? static_cast<const uint64_t*>(st->buf[a.vals_buf].ptr) : nullptr;
  auto F = [&](uint64_t g) { return vals ? vals[first[g]] : first[g]; };
  uint64_t* out = static_cast<uint64_t*>(st->buf[a.out_buf].ptr);
  const uint64_t ocap = st->buf[a.out_buf].cap;
  const uint64_t nk = 1ull << bits;
  // with unit_size: the dense join's units per group, their first unit, the
  // multi-unit slot (k_dense_units' outputs) in the same pass
  const bool units_on = a.unit_size > 0;
  const uint64_t usz = units_on ? uint64_t(a.unit_size) : 1;
  uint64_t* units = units_on ? static_cast<uint64_t*>(st->buf[a.units_buf].ptr) : nullptr;
  uint32_t* done = units_on ? static_cast<uint32_t*>(st->buf[a.done_buf].ptr) : nullptr;
  uint32_t* mslot = units_on ? static_cast<uint32_t*>(st->buf[a.mslot_buf].ptr) : nullptr;
  const uint64_t ucap = units_on ? min(st->buf[a.units_buf].cap, min(st->buf[a.done_buf].cap, st->buf[a.mslot_buf].cap))
                                 : 0;
  // pulled groups (dense.cuh, pull mode) are one unit each
  const uint32_t* pbm = units_on && a.pull_bm_buf >= 0 ? static_cast<const uint32_t*>(st->buf[a.pull_bm_buf].ptr)
                                                       : nullptr;
  auto pulled = [&](uint64_t g) { return pbm && ((pbm[g >> 5] >> (g & 31)) & 1u); };
  uint32_t* plist = pbm ? static_cast<uint32_t*>(st->buf[a.plist_buf].ptr) : nullptr;
  const uint64_t pcap = pbm ? st->buf[a.plist_buf].cap : 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint64_t wper = (((nk + nw - 1) / nw) + 31) & ~31ull;
  const uint64_t w0 = min(nk, uint64_t(warp) * wper), w1 = min(nk, w0 + wper);
  // pass 1: groups and multi-unit groups (packed, each < 2^32), units,
  // pulled groups
  uint64_t gm = 0, nus = 0, npl = 0;
  for (uint64_t base = w0; base < w1; base += 32 * kB) {
    uint64_t f0[kB], f1[kB];
#pragma unroll
    for (int i = 0; i < kB; ++i) {
      const uint64_t g = base + uint64_t(i) * 32 + lane;
      f0[i] = g < w1 ? F(g) : 0;
      f1[i] = g < w1 ? F(g + 1) : 0;
    }
#pragma unroll
    for (int i = 0; i < kB; ++i)
      if (f1[i] > f0[i]) {
        const bool pg = pulled(base + uint64_t(i) * 32 + lane);
        const uint64_t nu = pg ? 0 : (f1[i] - f0[i] + usz - 1) / usz;
        gm += 1 + (uint64_t(nu > 1) << 32);
        nus += nu;
        npl += pg;
      }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    gm += __shfl_xor_sync(0xffffffffu, gm, o);
    nus += __shfl_xor_sync(0xffffffffu, nus, o);
    npl += __shfl_xor_sync(0xffffffffu, npl, o);
  }
  if (lane == 0) {
    s_gm[warp] = gm;
    s_nu[warp] = nus;
    s_pl[warp] = npl;
  }
  __syncthreads();
  if (warp == 0) {   // exclusive scan over the warps; totals in [32]
    uint64_t x = lane < nw ? s_gm[lane] : 0, y = lane < nw ? s_nu[lane] : 0, z = lane < nw ? s_pl[lane] : 0;
    const uint64_t x0 = x, y0 = y, z0 = z;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t xs = __shfl_up_sync(0xffffffffu, x, o), ys = __shfl_up_sync(0xffffffffu, y, o),
                     zs = __shfl_up_sync(0xffffffffu, z, o);
      if (lane >= o) {
        x += xs;
        y += ys;
        z += zs;
      }
    }
    s_gm[lane] = x - x0;
    s_nu[lane] = y - y0;
    s_pl[lane] = z - z0;
    if (lane == 31) {
      s_gm[32] = x;
      s_nu[32] = y;
      s_pl[32] = z;
    }
  }
  __syncthreads();
  // pass 2: write the groups' starts (and units) at their ranks
  uint64_t c = s_gm[warp] & 0xFFFFFFFFull, m = s_gm[warp] >> 32, u = s_nu[warp], pl = s_pl[warp];
  const uint32_t lt = (1u << lane) - 1;
  for (uint64_t base = w0; base < w1; base += 32 * kB) {
    uint64_t f0[kB], f1[kB];
#pragma unroll
    for (int i = 0; i < kB; ++i) {
      const uint64_t g = base + uint64_t(i) * 32 + lane;
      f0[i] = g < w1 ? F(g) : 0;
      f1[i] = g < w1 ? F(g + 1) : 0;
    }
#pragma unroll
    for (int i = 0; i < kB; ++i) {
      const bool head = f1[i] > f0[i];
      const uint32_t hb = __ballot_sync(0xffffffffu, head);
      const uint64_t pos = c + __popc(hb & lt);
      if (head && pos < ocap) out[pos] = f0[i];
      if (units_on) {
        const bool pg = head && pulled(base + uint64_t(i) * 32 + lane);
        const uint64_t nu = !head || pg ? 0 : (f1[i] - f0[i] + usz - 1) / usz;
        const uint32_t pb = __ballot_sync(0xffffffffu, pg);
        if (pg && pl + __popc(pb & lt) < pcap) plist[pl + __popc(pb & lt)] = uint32_t(pos);
        pl += __popc(pb);
        const uint32_t mb = __ballot_sync(0xffffffffu, nu > 1);
        uint64_t incl = nu;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        if (head && pos + 1 < ucap) {
          units[pos] = u + incl - nu;
          done[pos] = 0;
          mslot[pos] = uint32_t(m + __popc(mb & lt));
        }
        u += __shfl_sync(0xffffffffu, incl, 31);
        m += __popc(mb);
      }
      c += __popc(hb);
    }
  }
  if (threadIdx.x == 0) {
    const uint64_t carry = s_gm[32] & 0xFFFFFFFFull, mcarry = s_gm[32] >> 32, nu_tot = s_nu[32];
    st->cnt[a.out_cnt] = carry;
    bool over = false;
    if (carry + 1 <= ocap) out[carry] = F(nk);
    else {
      atomicMax((unsigned long long*)&st->need[a.out_buf], (unsigned long long)(carry + 1));
      over = true;
    }
    if (pbm) {
      st->cnt[a.pull_cnt] = s_pl[32];
      if (s_pl[32] > pcap) {
        atomicMax((unsigned long long*)&st->need[a.plist_buf], (unsigned long long)s_pl[32]);
        over = true;
      }
    }
    if (units_on) {
      if (carry + 1 < ucap) {
        units[carry] = nu_tot;
        mslot[carry] = uint32_t(mcarry);
        if (st->buf[a.bmm_buf].cap < mcarry * uint64_t(a.bm_words)) {
          atomicMax((unsigned long long*)&st->need[a.bmm_buf], (unsigned long long)(mcarry * uint64_t(a.bm_words)));
          over = true;
        }
      } else {
        atomicMax((unsigned long long*)&st->need[a.units_buf], (unsigned long long)(carry + 2));
        atomicMax((unsigned long long*)&st->need[a.done_buf], (unsigned long long)(carry + 2));
        atomicMax((unsigned long long*)&st->need[a.mslot_buf], (unsigned long long)(carry + 2));
        over = true;
      }
    }
    if (over) atomicOr(&st->overflow, 1u << a.stage_bit);
  }
}

// dense.cuh, pull mode: the bitmap of values with inner tuples and their count
__global__ void k_pull_out(PullOutArgs a) {
  DevState* st = a.st;
  const uint64_t* first = static_cast<const uint64_t*>(st->buf[a.index_buf].ptr);
  const uint64_t* tfirst = static_cast<const uint64_t*>(st->buf[a.top_index_buf].ptr);
  const uint32_t* inner = static_cast<const uint32_t*>(st->buf[a.inner_buf].ptr);
  uint32_t* out = static_cast<uint32_t*>(st->buf[a.out_buf].ptr);
  uint32_t* fk = static_cast<uint32_t*>(st->buf[a.first_buf].ptr);
  uint32_t* tdeg = static_cast<uint32_t*>(st->buf[a.tdeg_buf].ptr);
  const uint64_t nwords = a.b >= 5 ? (1ull << (a.b - 5)) : 1;
  const uint64_t nk = 1ull << a.b;
  const uint32_t mask = uint32_t(nk - 1);
  unsigned long long cnt = 0;
  for (uint64_t w = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; w < nwords;
       w += uint64_t(gridDim.x) * blockDim.x) {
    uint32_t bits = 0;
    for (uint32_t i = 0; i < 32; ++i) {
      const uint64_t o = w * 32 + i;
      if (o >= nk) break;
      const uint64_t f0 = first[o], f1 = first[o + 1];
      if (f1 > f0) bits |= 1u << i;
      fk[o] = f1 > f0 ? inner[f0] & mask : 0xFFFFFFFFu;
      tdeg[o] = uint32_t(tfirst[o + 1] - tfirst[o]);
    }
    out[w] = bits;
    cnt += __popc(bits);
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd((unsigned long long*)&st->cnt[a.nout_cnt], cnt);
}

void launch_pull_out(const PullOutArgs& a, const Grid& g, cudaStream_t s) {
  HISA_LAUNCH(kKIndex, s, (k_pull_out<<<g.small, 256, 0, s>>>(a)));
}
void launch_ctl(const CtlArgs& a, cudaStream_t s) { HISA_LAUNCH(kKCtl, s, (k_ctl<<<1, 256, 0, s>>>(a))); }
void launch_group_compact(const GroupArgs& a, int bits, cudaStream_t s) {
  HISA_LAUNCH(kKGroups, s, (k_group_compact<<<1, 1024, 0, s>>>(a, bits)));
}
void launch_commit(const CommitArgs& a, cudaStream_t s) { HISA_LAUNCH(kKCommit, s, (k_commit<<<1, 32, 0, s>>>(a))); }
void launch_zero(const ZeroArgs& a, const Grid& g, cudaStream_t s) {
  HISA_LAUNCH(kKZero, s, (k_zero<<<g.small, 256, 0, s>>>(a)));
}

void launch_matrix_transpose(const MatrixTransposeArgs& t, const Grid& g, cudaStream_t s) {
  HISA_LAUNCH(kKDecode, s, (k_matrix_transpose<<<g.sms * 8, 256, 0, s>>>(t)));
}
void launch_bit_items(const BitItemsArgs& a, const Grid& g, cudaStream_t s) {
  HISA_LAUNCH(kKBitInit, s, (k_bit_items_count<<<g.small, 256, 0, s>>>(a)));
  HISA_LAUNCH(kKBitInit, s, (k_bit_items_scan<<<1, 1024, 0, s>>>(a)));
  HISA_LAUNCH(kKBitInit, s, (k_bit_items_write<<<g.small, 256, 0, s>>>(a)));
}

const char* const kKernelNames[kKindCount] = {
    "encode", "decode", "count_runs", "radix_hist", "radix_pass", "setop_partition", "setop_diff_merge",
    "index_build", "join_count", "join_partition", "join_write", "ctl", "commit", "zero", "swap_cols", "setop_diff_probe", "group_compact", "join_dense_mark", "join_dense_scan", "join_dense_emit", "append_level", "chain_len", "chain_scan", "chain_gather", "join_dense_pull", "matrix_merge", "matrix_diff", "bit_join", "bit_init"};

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
