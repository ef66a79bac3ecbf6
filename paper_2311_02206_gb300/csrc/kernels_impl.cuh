// Kernel bodies of the conversion/control kernels and the launcher templates.
// Included once per code width by kernels_u32.cu / kernels_u64.cu.
#pragma once
#include "kernels.cuh"

namespace hisa {

template <typename K>
__global__ void k_encode(EncodeArgs a) {
  DevState* st = a.st;
  K* out = static_cast<K*>(st->buf[a.out_buf].ptr) + st->cnt[a.out_cnt];
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < a.n; i += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t x = a.c0[i], y = a.c1[i];
    const uint64_t inst = a.inst ? (uint64_t(a.inst[i]) << (2 * a.b)) : a.inst_code;
    out[i] = K(inst | (a.order == 0 ? ((x << a.b) | y) : ((y << a.b) | x)));
  }
}

template <typename K>
__global__ void k_decode(DecodeArgs a) {
  DevState* st = a.st;
  const K* in = static_cast<const K*>(st->buf[a.in_buf].ptr);
  const uint64_t m = a.b >= 32 ? 0xFFFFFFFFull : ((1ull << a.b) - 1);
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < a.count; i += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t c = in[a.begin + i];
    const uint32_t hi = uint32_t((c >> a.b) & m), lo = uint32_t(c & m);
    a.c0[i] = a.order == 0 ? hi : lo;
    a.c1[i] = a.order == 0 ? lo : hi;
  }
}

template <typename K>
__global__ void k_count_runs(RunsArgs a) {
  DevState* st = a.st;
  if (st->overflow & a.skip_mask) return;
  const K* keys = static_cast<const K*>(st->buf[a.keys_buf].ptr);
  const uint64_t n = st->cnt[a.keys_cnt];
  uint32_t runs = 0;
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x)
    runs += (i == 0 || (uint64_t(keys[i - 1]) >> a.b) != (uint64_t(keys[i]) >> a.b));
  for (int o = 16; o > 0; o >>= 1) runs += __shfl_xor_sync(0xffffffffu, runs, o);
  if ((threadIdx.x & 31) == 0 && runs) atomicAdd((unsigned long long*)&st->cnt[a.out_cnt], (unsigned long long)runs);
}

// (inst, c0, c1) -> (inst, c1, c0): the reverse-order copy of a delta, sorted
// afterwards and merged into the reverse-order full of an IDB relation.
template <typename K>
__global__ void k_swap_cols(SwapArgs a) {
  DevState* st = a.st;
  if (st->overflow & a.skip_mask) return;
  const uint64_t n = st->cnt[a.in_cnt];
  if (n > st->buf[a.out_buf].cap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      atomicMax((unsigned long long*)&st->need[a.out_buf], (unsigned long long)n);
      atomicOr(&st->overflow, 1u << a.stage_bit);
    }
    return;
  }
  const K* in = static_cast<const K*>(st->buf[a.in_buf].ptr);
  K* out = static_cast<K*>(st->buf[a.out_buf].ptr);
  const uint64_t m = a.b >= 32 ? 0xFFFFFFFFull : ((1ull << a.b) - 1);
  const uint64_t im = 2 * a.b >= 64 ? 0ull : ~((1ull << (2 * a.b)) - 1);
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t c = in[i];
    out[i] = K((c & im) | ((c & m) << a.b) | ((c >> a.b) & m));
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) st->cnt[a.out_cnt] = n;
}

// Counts of each instance id in a sorted code array: every thread walks a
// contiguous stretch and adds one count per run of equal ids.
template <typename K>
__global__ void k_inst_hist(InstArgs a) {
  DevState* st = a.st;
  const K* c = static_cast<const K*>(st->buf[a.buf].ptr);
  const uint64_t n = st->cnt[a.cnt];
  const uint64_t nth = uint64_t(gridDim.x) * blockDim.x;
  const uint64_t per = (n + nth - 1) / nth;
  const uint64_t lo = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) * per;
  const uint64_t hi = min(n, lo + per);
  if (lo >= hi) return;
  uint64_t cur = uint64_t(c[lo]) >> a.shift, run = 0;
  for (uint64_t i = lo; i < hi; ++i) {
    const uint64_t id = uint64_t(c[i]) >> a.shift;
    if (id != cur) {
      if (cur < a.ninst) atomicAdd(&a.out[cur], (unsigned long long)run);
      cur = id;
      run = 0;
    }
    ++run;
  }
  if (cur < a.ninst) atomicAdd(&a.out[cur], (unsigned long long)run);
}

// out[i] = first position whose instance id is >= i, for i in [0, ninst].
template <typename K>
__global__ void k_inst_bounds(InstArgs a) {
  DevState* st = a.st;
  const K* c = static_cast<const K*>(st->buf[a.buf].ptr);
  const uint64_t n = st->cnt[a.cnt];
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i <= a.ninst; i += uint64_t(gridDim.x) * blockDim.x) {
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
      const uint64_t m = (lo + hi) >> 1;
      if ((uint64_t(c[m]) >> a.shift) < i) lo = m + 1;
      else hi = m;
    }
    a.out[i] = lo;
  }
}

template <typename K>
void launch_inst_hist(const InstArgs& a, const Grid& g, cudaStream_t s) {
  HISA_LAUNCH(kKCtl, s, (k_inst_hist<K><<<g.small, 256, 0, s>>>(a)));
}
template <typename K>
void launch_inst_bounds(const InstArgs& a, const Grid& g, cudaStream_t s) {
  HISA_LAUNCH(kKCtl, s, (k_inst_bounds<K><<<g.small, 256, 0, s>>>(a)));
}

template <typename K>
__global__ void k_append(AppendArgs a) {
  DevState* st = a.st;
  if (st->overflow & a.skip_mask) return;
  const uint64_t n = st->cnt[a.src_cnt];
  if (n == 0) return;
  const uint64_t base = st->cnt[a.full_cnt], lv = st->cnt[a.nlv_cnt];
  const uint64_t nk = (1ull << a.bits) + 1;
  if (base + n > st->buf[a.full_buf].cap || (lv + 1) * nk > st->buf[a.lvidx_buf].cap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      atomicMax((unsigned long long*)&st->need[a.full_buf], (unsigned long long)(base + n));
      atomicMax((unsigned long long*)&st->need[a.lvidx_buf], (unsigned long long)((lv + 1) * nk));
      atomicOr(&st->overflow, 1u << a.stage_bit);
    }
    return;
  }
  const K* src = static_cast<const K*>(st->buf[a.src_buf].ptr);
  K* full = static_cast<K*>(st->buf[a.full_buf].ptr) + base;
  uint64_t* idx = static_cast<uint64_t*>(st->buf[a.lvidx_buf].ptr) + lv * nk;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += stride) full[i] = src[i];
  uint32_t* fcnt = a.fcnt_buf >= 0 ? static_cast<uint32_t*>(st->buf[a.fcnt_buf].ptr) : nullptr;
  auto lower = [&](uint64_t k) {
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
      const uint64_t m = (lo + hi) >> 1;
      if ((uint64_t(src[m]) >> a.b) < k) lo = m + 1;
      else hi = m;
    }
    return lo;
  };
  for (uint64_t k = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; k < nk; k += stride) {
    const uint64_t lo = lower(k);
    idx[k] = base + lo;
    if (fcnt && k + 1 < nk) fcnt[k] += uint32_t(lower(k + 1) - lo);
  }
}

template <typename K>
void launch_group_starts(const GroupArgs& a, const Grid& g, cudaStream_t s) {
  CtlArgs c{};
  c.st = a.st;
  c.skip_mask = a.skip_mask;
  c.n = 2;
  c.cmd[0] = {kCtlEpoch, 0, 0};
  c.cmd[1] = {kCtlResetCtr, a.ctr, 0};
  launch_ctl(c, s);
  HISA_LAUNCH(kKGroups, s, (k_group_starts<K><<<g.setop, kGroupThreads, 0, s>>>(a)));
}
template <typename K>
void launch_chain(const ChainArgs& a, const Grid& g, cudaStream_t s) {
  HISA_LAUNCH(kKChainLen, s, (k_chain_len<K><<<g.small * 2, 256, 0, s>>>(a)));
  HISA_LAUNCH(kKChainScan, s, (k_chain_scan<K><<<1, 1024, 0, s>>>(a)));
  HISA_LAUNCH(kKChainGather, s, (k_chain_gather<K><<<g.join, 256, 0, s>>>(a)));
  if (a.tfirst_buf >= 0) HISA_LAUNCH(kKChainScan, s, (k_chain_first<K><<<g.small, 256, 0, s>>>(a)));
}
template <typename K>
void launch_levels_read(const LevelsReadArgs& a, const Grid& g, cudaStream_t s) {
  const size_t nwords = a.b >= 5 ? (size_t(1) << (a.b - 5)) : 1;
  const size_t smem = (nwords + (kDenseThreads / 32) * 1024) * 4;
  // the bitmap of an 18-bit domain and the staging exceed the default 48 KB
  cudaFuncSetAttribute(k_levels_read<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  HISA_LAUNCH(kKDecode, s, (k_levels_read<K><<<g.sms * 8, kDenseThreads, smem, s>>>(a)));
}
template <typename K>
void launch_levels_transpose(const LevelsTransposeArgs& a, const Grid& g, cudaStream_t s) {
  const size_t tile = (size_t(1) << a.b) * 2;   // 2^b 16-bit columns
  cudaFuncSetAttribute(k_levels_transpose<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(tile));
  HISA_LAUNCH(kKDecode, s, (k_levels_transpose<K><<<g.sms, 1024, tile, s>>>(a)));
  HISA_LAUNCH(kKDecode, s, (k_rows_count<K><<<g.small, 256, 0, s>>>(a)));
  HISA_LAUNCH(kKDecode, s, (k_rows_scan<K><<<1, 1024, 0, s>>>(a)));
  HISA_LAUNCH(kKDecode, s, (k_rows_emit<K><<<g.sms * 8, kDenseThreads, 0, s>>>(a)));
}
template <typename K>
void launch_matrix_codes(const MatrixArgs& a, const Grid& g, cudaStream_t s) {
  HISA_LAUNCH(kKMatrix, s, (k_matrix_codes<K><<<g.small, 256, 0, s>>>(a)));
}
template <typename K>
void launch_matrix_diff(const MatrixDiffArgs& a, const Grid& g, cudaStream_t s) {
  CtlArgs c{};
  c.st = a.st;
  c.skip_mask = a.skip_mask;
  c.n = 2;
  c.cmd[0] = {kCtlEpoch, 0, 0};
  c.cmd[1] = {kCtlResetCtr, a.ctr, 0};
  launch_ctl(c, s);
  HISA_LAUNCH(kKMatrixDiff, s, (k_matrix_diff<K><<<g.setop, kDiffThreads, 0, s>>>(a)));
}
template <typename K>
void launch_bit_init(const BitInitArgs& a, const Grid& g, cudaStream_t s) {
  HISA_LAUNCH(kKBitInit, s, (k_bit_init<K><<<g.small, 256, 0, s>>>(a)));
}
template <typename K>
void launch_bit_todo(const BitTodoArgs& a, const Grid& g, cudaStream_t s) {
  HISA_LAUNCH(kKBitInit, s, (k_bit_todo<K><<<g.small, 256, 0, s>>>(a)));
}
template <typename K>
void launch_bitjoin(const BitJoinArgs& a, const Grid& g, cudaStream_t s) {
  if (a.b >= 10) HISA_LAUNCH(kKBitJoin, s, (k_bitjoin_vec<K><<<g.sms * 8, kBitThreads, 0, s>>>(a)));
  else HISA_LAUNCH(kKBitJoin, s, (k_bitjoin<K><<<g.sms * 8, kBitThreads, 0, s>>>(a)));
}
template <typename K>
void launch_matrix_extract(const MatrixExtractArgs& a, const Grid& g, cudaStream_t s) {
  HISA_LAUNCH(kKDecode, s, (k_matrix_extract_counts<<<g.small, 256, 0, s>>>(a)));
  HISA_LAUNCH(kKDecode, s, (k_matrix_extract_scan<<<1, 1024, 0, s>>>(a)));
  HISA_LAUNCH(kKDecode, s, (k_matrix_extract<K><<<g.sms * 8, kDenseThreads, 0, s>>>(a)));
}
template <typename K>
void launch_matrix_read(const MatrixTransposeArgs& t, const LevelsTransposeArgs& a, bool transpose, const Grid& g,
                        cudaStream_t s) {
  if (transpose) HISA_LAUNCH(kKDecode, s, (k_matrix_transpose<<<g.sms * 8, 256, 0, s>>>(t)));
  HISA_LAUNCH(kKDecode, s, (k_rows_count<K><<<g.small, 256, 0, s>>>(a)));
  HISA_LAUNCH(kKDecode, s, (k_rows_scan<K><<<1, 1024, 0, s>>>(a)));
  HISA_LAUNCH(kKDecode, s, (k_rows_emit<K><<<g.sms * 8, kDenseThreads, 0, s>>>(a)));
}
template <typename K>
void launch_append(const AppendArgs& a, const Grid& g, cudaStream_t s) {
  HISA_LAUNCH(kKAppend, s, (k_append<K><<<g.small * 2, 256, 0, s>>>(a)));
}

template <typename K>
void launch_encode(const EncodeArgs& a, const Grid& g, cudaStream_t s) {
  HISA_LAUNCH(kKEncode, s, (k_encode<K><<<g.small, 256, 0, s>>>(a)));
}
template <typename K>
void launch_decode(const DecodeArgs& a, const Grid& g, cudaStream_t s) {
  HISA_LAUNCH(kKDecode, s, (k_decode<K><<<g.small, 256, 0, s>>>(a)));
}
template <typename K>
void launch_count_runs(const RunsArgs& a, const Grid& g, cudaStream_t s) {
  HISA_LAUNCH(kKRuns, s, (k_count_runs<K><<<g.small, 256, 0, s>>>(a)));
}
template <typename K>
void launch_swap(const SwapArgs& a, const Grid& g, cudaStream_t s) {
  HISA_LAUNCH(kKSwap, s, (k_swap_cols<K><<<g.small, 256, 0, s>>>(a)));
}
template <typename K>
void launch_radix_hist(const RadixHistArgs& a, const Grid& g, cudaStream_t s) {
  HISA_LAUNCH(kKHist, s, (k_radix_hist<K><<<g.small, 256, 0, s>>>(a)));
}
template <typename K, int ITEMS>
void launch_radix_pass_items(const RadixPassArgs& a, const Grid& g, cudaStream_t s) {
  static bool attr = false;   // the tiles exceed the default 48 KB of dynamic shared memory
  if (!attr) {
    cudaFuncSetAttribute(k_radix_pass<K, ITEMS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         radix_dyn_smem<K, ITEMS>());
    attr = true;
  }
  HISA_LAUNCH(kKRadixPass, s, (k_radix_pass<K, ITEMS><<<g.radix, kRadixThreads, radix_dyn_smem<K, ITEMS>(), s>>>(a)));
}
template <typename K>
void launch_radix_pass(const RadixPassArgs& a, const Grid& g, cudaStream_t s) {
  CtlArgs c{};
  c.st = a.st;
  c.skip_mask = a.skip_mask;
  c.n = 2;
  c.cmd[0] = {kCtlEpoch, 0, 0};
  c.cmd[1] = {kCtlResetCtr, a.ctr, 0};
  launch_ctl(c, s);
  if (a.items == RadixCfg<K>::items_alt) launch_radix_pass_items<K, RadixCfg<K>::items_alt>(a, g, s);
  else launch_radix_pass_items<K, RadixCfg<K>::items>(a, g, s);
}
template <typename K>
void launch_setop(const SetopArgs& a, const Grid& g, cudaStream_t s) {
  CtlArgs c{};
  c.st = a.st;
  c.skip_mask = a.skip_mask;
  c.n = 2;
  c.cmd[0] = {kCtlEpoch, 0, 0};
  c.cmd[1] = {kCtlResetCtr, a.ctr, 0};
  launch_ctl(c, s);
  HISA_LAUNCH(kKSetopPartition, s, (k_setop_partition<K><<<g.small, 256, 0, s>>>(a)));
  HISA_LAUNCH(kKSetop, s, (k_setop<K><<<g.setop, kSetopThreads, 0, s>>>(a)));
}
template <typename K>
void launch_diff(const DiffArgs& a, const Grid& g, cudaStream_t s) {
  CtlArgs c{};
  c.st = a.st;
  c.skip_mask = a.skip_mask;
  c.n = 2;
  c.cmd[0] = {kCtlEpoch, 0, 0};
  c.cmd[1] = {kCtlResetCtr, a.ctr, 0};
  launch_ctl(c, s);
  HISA_LAUNCH(kKDiffProbe, s, (k_diff_probe<K><<<g.setop, kDiffThreads, 0, s>>>(a)));
}
template <typename K>
void launch_join_dense(const DenseArgs& a, const Grid& g, cudaStream_t s) {
  CtlArgs c{};
  c.st = a.st;
  c.skip_mask = a.skip_mask;
  c.n = 3;
  c.cmd[0] = {kCtlEpoch, 0, 0};
  c.cmd[1] = {kCtlResetCtr, a.ctr, 0};
  c.cmd[2] = {kCtlResetCtr, a.ctr + 1, 0};   // the pull kernel's group counter
  launch_ctl(c, s);
  const size_t smem = size_t(a.b >= 5 ? (1u << (a.b - 5)) : 1u) * 4;   // one bitmap of 2^b bits
  if (!a.units_ready) HISA_LAUNCH(kKDenseScan, s, (k_dense_units<K><<<1, 1024, 0, s>>>(a)));
  HISA_LAUNCH(kKJoinDense, s, (k_dense_mark<K><<<g.sms * kDenseCtasPerSm, kDenseThreads, smem, s>>>(a)));
  if (a.pull_inner_buf >= 0)   // pulled groups: frontier and full bitmaps
    HISA_LAUNCH(kKJoinPull, s, (k_dense_pull<K><<<g.sms * kPullCtasPerSm, kDenseThreads, 2 * smem, s>>>(a)));
  HISA_LAUNCH(kKDenseScan, s, (k_dense_scan<K><<<1, 1024, 0, s>>>(a)));
  HISA_LAUNCH(kKDenseEmit, s, (k_dense_emit<K><<<g.sms * kDenseCtasPerSm, kDenseThreads, 0, s>>>(a)));
  CtlArgs d{};
  d.st = a.st;
  d.skip_mask = a.skip_mask;
  d.n = 1;
  d.cmd[0] = {kCtlAddCnt, a.out_cnt, a.total_cnt};
  launch_ctl(d, s);
}
template <typename K>
void launch_index(const IndexArgs& a, const Grid& g, cudaStream_t s) {
  if (a.direct) HISA_LAUNCH(kKIndex, s, (k_index_direct<K><<<g.small, 256, 0, s>>>(a)));
  else HISA_LAUNCH(kKIndex, s, (k_index_build<K><<<g.small, 256, 0, s>>>(a)));
}
template <typename K>
void launch_join(const JoinArgs& a, const Grid& g, cudaStream_t s) {
  CtlArgs c{};
  c.st = a.st;
  c.skip_mask = a.skip_mask;
  c.n = 2;
  c.cmd[0] = {kCtlEpoch, 0, 0};
  c.cmd[1] = {kCtlResetCtr, a.ctr, 0};
  launch_ctl(c, s);
  HISA_LAUNCH(kKJoinCount, s, (k_join_count<K><<<g.join, kJoinThreads, 0, s>>>(a)));
  HISA_LAUNCH(kKJoinPartition, s, (k_join_partition<K><<<g.small, 256, 0, s>>>(a)));
  HISA_LAUNCH(kKJoinWrite, s, (k_join_write<K><<<g.join, kJoinThreads, 0, s>>>(a)));
  CtlArgs d{};
  d.st = a.st;
  d.skip_mask = a.skip_mask;
  d.n = 1;
  d.cmd[0] = {kCtlAddCnt, a.out_cnt, a.total_cnt};
  launch_ctl(d, s);
}

template <typename K>
void launch_join_count(const JoinArgs& a, const Grid& g, cudaStream_t s) {
  HISA_LAUNCH(kKJoinCount, s, (k_join_count<K><<<g.join, kJoinThreads, 0, s>>>(a)));
}
template <typename K>
void launch_join_write(const JoinArgs& a, const Grid& g, cudaStream_t s) {
  HISA_LAUNCH(kKJoinPartition, s, (k_join_partition<K><<<g.small, 256, 0, s>>>(a)));
  HISA_LAUNCH(kKJoinWrite, s, (k_join_write<K><<<g.join, kJoinThreads, 0, s>>>(a)));
}

#define HISA_INSTANTIATE(K)                                                              \
  template void launch_encode<K>(const EncodeArgs&, const Grid&, cudaStream_t);          \
  template void launch_decode<K>(const DecodeArgs&, const Grid&, cudaStream_t);          \
  template void launch_count_runs<K>(const RunsArgs&, const Grid&, cudaStream_t);        \
  template void launch_swap<K>(const SwapArgs&, const Grid&, cudaStream_t);              \
  template void launch_diff<K>(const DiffArgs&, const Grid&, cudaStream_t);              \
  template void launch_append<K>(const AppendArgs&, const Grid&, cudaStream_t);          \
  template void launch_group_starts<K>(const GroupArgs&, const Grid&, cudaStream_t);     \
  template void launch_join_dense<K>(const DenseArgs&, const Grid&, cudaStream_t);       \
  template void launch_chain<K>(const ChainArgs&, const Grid&, cudaStream_t);            \
  template void launch_levels_read<K>(const LevelsReadArgs&, const Grid&, cudaStream_t);  \
  template void launch_levels_transpose<K>(const LevelsTransposeArgs&, const Grid&, cudaStream_t); \
  template void launch_matrix_codes<K>(const MatrixArgs&, const Grid&, cudaStream_t);    \
  template void launch_matrix_diff<K>(const MatrixDiffArgs&, const Grid&, cudaStream_t); \
  template void launch_bit_init<K>(const BitInitArgs&, const Grid&, cudaStream_t);       \
  template void launch_bitjoin<K>(const BitJoinArgs&, const Grid&, cudaStream_t);        \
  template void launch_bit_todo<K>(const BitTodoArgs&, const Grid&, cudaStream_t);      \
  template void launch_matrix_extract<K>(const MatrixExtractArgs&, const Grid&, cudaStream_t); \
  template void launch_matrix_read<K>(const MatrixTransposeArgs&, const LevelsTransposeArgs&, bool, const Grid&, \
                                      cudaStream_t);                                     \
  template void launch_radix_hist<K>(const RadixHistArgs&, const Grid&, cudaStream_t);   \
  template void launch_radix_pass<K>(const RadixPassArgs&, const Grid&, cudaStream_t);   \
  template void launch_setop<K>(const SetopArgs&, const Grid&, cudaStream_t);            \
  template void launch_index<K>(const IndexArgs&, const Grid&, cudaStream_t);            \
  template void launch_inst_hist<K>(const InstArgs&, const Grid&, cudaStream_t);          \
  template void launch_inst_bounds<K>(const InstArgs&, const Grid&, cudaStream_t);        \
  template void launch_join<K>(const JoinArgs&, const Grid&, cudaStream_t);              \
  template void launch_join_count<K>(const JoinArgs&, const Grid&, cudaStream_t);        \
  template void launch_join_write<K>(const JoinArgs&, const Grid&, cudaStream_t);

}  // namespace hisa
