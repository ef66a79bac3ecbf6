// Control, commit and conversion kernels plus the host-side launchers of every
// kernel of the engine.  The launchers are templates over the code width K and
// are instantiated for uint32_t and uint64_t in kernels_u32.cu / kernels_u64.cu.
#pragma once
#include "common.cuh"
#include "join.cuh"
#include "radix.cuh"
#include "setops.cuh"
#include "dense.cuh"
#include "read.cuh"
#include "matrix.cuh"
#include "bitjoin.cuh"
#include <vector>

namespace hisa {

// ---- control commands (one tiny launch between stages) -------------------------------

enum : int {
  kCtlEpoch = 1,     // epoch++
  kCtlResetCtr,      // tile_ctr[a] = 0
  kCtlSetCnt,        // cnt[a] = b
  kCtlAddCnt,        // cnt[a] += cnt[b]
  kCtlCopyCnt,       // cnt[a] = cnt[b]
  kCtlZeroSmall,     // zero the first b u64 words of buffer a
  kCtlSwapIfCnt,     // if cnt[c] > 0: exchange buffers a and b, cnt[a] = cnt[b]
  kCtlCheckTable,    // hash table a must hold cnt[b] runs at load factor c / 1024
  kCtlMergeGate,     // cnt[a] = cnt[b] if cnt[b] * r > cnt[L] or cnt[F] != 0, else 0;
                     //   c = (L << 32) | (F << 16) | r
  kCtlBigFlag,       // cnt[a] = (cnt[b] * (c & 0xFFFF) > cnt[c >> 16]) ? 1 : 0
  kCtlNot,           // cnt[a] = cnt[b] ? 0 : 1
  kCtlSwap,          // exchange buffers a and b (counts untouched)
  kCtlZeroIfCnt,     // if cnt[c] > 0: cnt[a] = 0
};

struct CtlCmd {
  int op, a;
  long long b;
  long long c;
};
constexpr int kMaxCtl = 24;
struct CtlArgs {
  DevState* st;
  int n;
  int skip_mask;
  CtlCmd cmd[kMaxCtl];
};

struct CommitArgs {
  DevState* st;
  int nrel;
  int full[8], full_next[8], delta[8], delta_next[8], history[8], fresh[8];
  // a second (full, full_next) pair swapped instead when cnt[alt_flag1 - 1]
  // is non-zero (log-structured full: delta merged into the large level)
  int alt_full[8], alt_full_next[8], alt_flag1[8];
  // append-only full (dense-join relations): 1 + cnt slot of its level count
  // (0: not append-only); the commit adds delta's size to full's count and
  // one level, and asks the host to compact past max_levels
  int append_nlv1[8];
  // full kept as a bit matrix: the commit only adds delta's size to full's count
  int add_full[8];
  int max_levels;
  int force;   // commit even when no delta is non-empty (first iteration)
};

// Appends a sorted, duplicate-free delta to an append-only full as a new
// level: copies it behind full's cnt tuples and writes the level's direct
// index (first position of every kept value g in [0, 2^bits], absolute in
// full).  Counts are bumped by the commit, so a re-run rewrites the same
// places.
struct AppendArgs {
  DevState* st;
  int src_buf, src_cnt;
  int full_buf, full_cnt;
  int lvidx_buf, nlv_cnt;   // u64 [levels][2^bits + 1]
  int b, bits;
  int skip_mask, stage_bit;
  int fcnt_buf = -1;        // u32 [2^bits]: tuples of full per kept value, grown by the new level's runs
};

struct EncodeArgs {
  DevState* st;
  const uint32_t* c0;
  const uint32_t* c1;
  uint64_t n;
  int out_buf, out_cnt;
  int b;
  int order;   // 0: (c0, c1); 1: (c1, c0)
  uint64_t inst_code;  // instance id << 2b, or 0
  const uint32_t* inst;  // per-tuple instance ids (batched runs), or null
};

// Per-instance counts of a sorted code array (instance id = code >> 2b).
struct InstArgs {
  DevState* st;
  int buf, cnt;
  int shift;              // 2b
  uint32_t ninst;         // instance slots
  unsigned long long* out;   // [ninst] counts (added to) or [ninst + 1] bounds
};

struct DecodeArgs {
  DevState* st;
  int in_buf, in_cnt;
  uint32_t* c0;
  uint32_t* c1;
  int b;
  int order;
  uint64_t begin, count;
};

struct ZeroArgs {
  DevState* st;
  int buf;
  int elem_bytes;
  int skip_mask;
};

struct RunsArgs {
  DevState* st;
  int keys_buf, keys_cnt, b, out_cnt;
  int skip_mask;
};

// Column exchange of packed codes: (inst, c0, c1) -> (inst, c1, c0).
struct SwapArgs {
  DevState* st;
  int in_buf, in_cnt;
  int out_buf, out_cnt;   // written from 0; cnt[out_cnt] = cnt[in_cnt]
  int b;
  int skip_mask, stage_bit;
};

// ---- launch accounting -----------------------------------------------------------------

enum KernelKind : int {
  kKEncode, kKDecode, kKRuns, kKHist, kKRadixPass, kKSetopPartition, kKSetop, kKIndex,
  kKJoinCount, kKJoinPartition, kKJoinWrite, kKCtl, kKCommit, kKZero, kKSwap, kKDiffProbe, kKGroups, kKJoinDense, kKDenseScan, kKDenseEmit, kKAppend, kKChainLen, kKChainScan, kKChainGather, kKJoinPull, kKMatrix, kKMatrixDiff, kKBitJoin, kKBitInit, kKindCount
};
extern const char* const kKernelNames[kKindCount];

// CUDA-event timer around every kernel launch (host-driven loop only).
struct KernelTimer {
  struct Rec { int kind; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  cudaEvent_t get();
  void begin(int kind, cudaStream_t s);
  void end(cudaStream_t s);
  void truncate(size_t n);   // drop records from n on (an iteration that was re-run)
  void reset();
  ~KernelTimer();
};
extern thread_local KernelTimer* g_timer;
extern thread_local uint64_t g_launches;

#define HISA_LAUNCH(kind, s, stmt)            \
  do {                                        \
    if (g_timer) g_timer->begin((kind), (s)); \
    stmt;                                     \
    ++g_launches;                             \
    if (g_timer) g_timer->end((s));           \
  } while (0)

// ---- launchers ------------------------------------------------------------------------

struct Grid {
  int sms = 152;
  int radix = 152 * 4;
  int setop = 152 * 4;
  int join = 152 * 4;
  int small = 152 * 2;
};

void launch_ctl(const CtlArgs& a, cudaStream_t s);
void launch_commit(const CommitArgs& a, cudaStream_t s);
void launch_zero(const ZeroArgs& a, const Grid& g, cudaStream_t s);

template <typename K> void launch_encode(const EncodeArgs& a, const Grid& g, cudaStream_t s);
template <typename K> void launch_decode(const DecodeArgs& a, const Grid& g, cudaStream_t s);
template <typename K> void launch_radix_hist(const RadixHistArgs& a, const Grid& g, cudaStream_t s);
template <typename K> void launch_radix_pass(const RadixPassArgs& a, const Grid& g, cudaStream_t s);
template <typename K> void launch_setop(const SetopArgs& a, const Grid& g, cudaStream_t s);   // partition + merge
template <typename K> void launch_index(const IndexArgs& a, const Grid& g, cudaStream_t s);
template <typename K> void launch_count_runs(const RunsArgs& a, const Grid& g, cudaStream_t s);
template <typename K> void launch_swap(const SwapArgs& a, const Grid& g, cudaStream_t s);
template <typename K> void launch_diff(const DiffArgs& a, const Grid& g, cudaStream_t s);
void launch_group_compact(const GroupArgs& a, int bits, cudaStream_t s);
void launch_pull_out(const PullOutArgs& a, const Grid& g, cudaStream_t s);
template <typename K> void launch_group_starts(const GroupArgs& a, const Grid& g, cudaStream_t s);
template <typename K> void launch_append(const AppendArgs& a, const Grid& g, cudaStream_t s);
template <typename K> void launch_join_dense(const DenseArgs& a, const Grid& g, cudaStream_t s);
template <typename K> void launch_chain(const ChainArgs& a, const Grid& g, cudaStream_t s);   // len + scan + gather
template <typename K> void launch_levels_read(const LevelsReadArgs& a, const Grid& g, cudaStream_t s);
template <typename K> void launch_levels_transpose(const LevelsTransposeArgs& a, const Grid& g, cudaStream_t s);
template <typename K> void launch_matrix_codes(const MatrixArgs& a, const Grid& g, cudaStream_t s);
template <typename K> void launch_matrix_diff(const MatrixDiffArgs& a, const Grid& g, cudaStream_t s);
template <typename K> void launch_bit_init(const BitInitArgs& a, const Grid& g, cudaStream_t s);
void launch_bit_items(const BitItemsArgs& a, const Grid& g, cudaStream_t s);
template <typename K> void launch_bitjoin(const BitJoinArgs& a, const Grid& g, cudaStream_t s);
template <typename K> void launch_bit_todo(const BitTodoArgs& a, const Grid& g, cudaStream_t s);
template <typename K> void launch_matrix_extract(const MatrixExtractArgs& a, const Grid& g, cudaStream_t s);
void launch_matrix_transpose(const MatrixTransposeArgs& t, const Grid& g, cudaStream_t s);
// a full kept as a bit matrix read in the declared order: transposed (order 1)
// or read as it is (order 0), then its rows counted, scanned and written
template <typename K> void launch_matrix_read(const MatrixTransposeArgs& t, const LevelsTransposeArgs& a, bool transpose,
                                              const Grid& g, cudaStream_t s);
template <typename K> void launch_inst_hist(const InstArgs& a, const Grid& g, cudaStream_t s);
template <typename K> void launch_inst_bounds(const InstArgs& a, const Grid& g, cudaStream_t s);
void launch_fill_u32(uint32_t* p, uint64_t n, uint32_t v, const Grid& g, cudaStream_t s);
template <typename K> void launch_join(const JoinArgs& a, const Grid& g, cudaStream_t s);     // count + partition + write
template <typename K> void launch_join_count(const JoinArgs& a, const Grid& g, cudaStream_t s);
template <typename K> void launch_join_write(const JoinArgs& a, const Grid& g, cudaStream_t s);  // partition + write

}  // namespace hisa
