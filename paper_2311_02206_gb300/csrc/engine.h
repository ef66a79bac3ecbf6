// Engine state behind the C-ABI (include/hisa.h).
#pragma once
#include <chrono>
#include <deque>
#include <map>
#include <string>
#include <unordered_map>
#include <vector>

#include "hisa.h"
#include "kernels.cuh"

namespace hisa {

struct Relation {
  std::string name;
  uint32_t arity = 2;
  bool idb = false;
  // EDB staging: raw columns as loaded
  uint32_t* stage[2] = {nullptr, nullptr};
  uint32_t* stage_inst = nullptr;   // instance id of each staged tuple
  uint64_t staged = 0, stage_cap = 0;
  uint32_t max_value = 0;
  // slots (see DevState::buf): sorted codes in column order (c0,c1) and (c1,c0),
  // and a run index over each order's first column
  int base = -1, rev = -1;
  int table[2] = {-1, -1};
  bool need_idx[2] = {false, false};
  // IDB versions (full == base)
  int full = -1, full_next = -1, delta = -1, delta_next = -1;
  int fresh = -1, fresh_alt = -1;   // "new" and its radix ping-pong partner
  int hist = -1;                    // digit histograms of new
  // an IDB relation probed as an inner relation: its full in reverse order
  // (kept as full's mirror by merging each sorted, column-swapped delta) and
  // the sort buffers of that delta; run counts feeding the index rebuilds
  int rev_next = -1, rswap = -1, rswap_alt = -1;
  int runs_cnt[2] = {-1, -1};
  // log-structured full (HISA_FLAG_LOG_FULL): full holds the large level,
  // l1 the small one that absorbs each delta; newp = new minus the large level;
  // gate = |l1| when l1 is due to be merged into full, else 0
  bool log = false;
  bool dense_head = false;   // its writer in iterations >= 2 is a dense join (writes delta itself)
  // append-only full (dense_head relations): one sorted level per iteration,
  // lvidx = each level's direct index by the kept column, nlv = levels
  bool append = false;
  int lvidx = -1, nlv = -1;
  int sortf = -1;   // 1 unless a dense join wrote this iteration's delta itself
  int order = 0;   // storage order of an IDB relation: 0 = (c0, c1), 1 = (c1, c0)
  int l1 = -1, l1_next = -1, newp = -1, gate = -1;
  int bigf = -1, smallf = -1;   // this iteration merges new straight into full / probes it
  int history = -1;                 // |delta_k| per iteration
  std::vector<uint64_t> delta_counts;
  // pull mode of its grouped bitmap join (dense.cuh): the inner relation
  // sorted by its other column and that order's direct index; the values with
  // inner tuples (bitmap, and their number in cnt[nout]); the groups that pull
  // next iteration (bitmap); |full_g| per kept value g
  bool pull = false;
  int pull_inner = -1, pull_index = -1;
  int pull_out = -1, nout = -1, pull_bm = -1, fcnt = -1;
  int pull_first = -1, tdeg = -1;   // each o's first k; each k's push-run length
  int push_index = -1;              // the push-ordered inner's direct index by k
  // full kept as a bit matrix (HISA_FLAG_LEVELS off): row g, bit o for (g, o)
  bool mfull = false;
  int fbm = -1;
};

// One binary join (or a one-atom projection) of a compiled rule variant.
struct StepPlan {
  int outer_slot, outer_cnt, outer_kcol;
  bool has_inner;
  int inner_rel, inner_col;
  int proj0, proj1;
  int nfilt, fop[2], fa[2], fb[2];
  bool to_tmp;
  int out_rel;
  bool dense;   // grouped join with bitmap deduplication (dense.cuh)
  bool resort;  // its outer (a delta stored join column first) is exchanged and sorted by the kept column first
  bool chain;   // a first step whose Tmp is gathered grouped by its kept column (ChainArgs)
  bool invert;  // a dense join run the other way round: the inner (sorted by the kept column) is
                // the grouped outer, delta (directly indexed by the join column) the probed side
};

struct Op {
  enum Kind { CTL, JOIN, PASS, HIST, SETOP, COMMIT, RUNS, INDEX, ZERO, SWAP, DIFF, DENSE, GCOMPACT, APPEND, GROUPS, CHAIN,
              MCODES, MDIFF } kind;
  CtlArgs ctl;
  JoinArgs join;
  RadixPassArgs pass;
  RadixHistArgs hist;
  SetopArgs setop;
  CommitArgs commit;
  RunsArgs runs;
  IndexArgs index;
  ZeroArgs zero;
  SwapArgs swap;
  DiffArgs diff;
  GroupArgs groups;
  AppendArgs append;
  DenseArgs dense;
  ChainArgs chain;
  MatrixArgs matrix;
  MatrixDiffArgs mdiff;
};

struct Scratch {
  int empty, hist, radix_status, split, setop_status, offs, join_status, starts, tmp_a, tmp_b;
  int runs, total, tmp_cnt;   // count-only slots
  int groups, dense_status;   // group starts of a delta and the dense join's per-group counts/offsets
  int dense_bm;               // the dense join's per-group bitmaps
  int tmp_hist;               // digit histograms of a Tmp relation sorted before a dense join
  int gather;                 // an instance's codes from both levels of a log-structured full
  int mrows;                  // u64 row offsets of a bit-matrix read-out (matrix.cuh)
  int mslots;                 // u32 instance slots whose blocks a read-out takes
  int dense_first;            // direct index of a delta by its kept column (group starts)
  int dense_units, dense_done;  // the dense join's first unit per group and finished-unit counters
  int dense_mslot, dense_bmm;   // multi-unit groups' bitmap slot and those bitmaps (kept zeroed)
  int chain_dfirst, chain_pre;  // a gathered Tmp: delta's direct index, offsets per inner tuple
  int chain_tfirst;             // a gathered Tmp's direct index by its kept column
  int dense_plist = -1, pull_cnt = -1;   // pulled groups of the grouped bitmap join, and their count
  int pull_raw_cnt = -1;                 // codes read by the pull kernel
  int dense_bm_prev = -1, prev_gi = -1;   // the previous iteration's group bitmaps; group index per value
  int read_m = -1, read_rows = -1;  // reading a column-swapped append-only full: its bit matrix, row offsets
  int read_s0 = -1, read_s1 = -1;   // and its device staging columns (kept across reads)

  int group_cnt, raw_cnt;     // count-only slots
};

// One request of the serving loop: the EDB tuples of an independent instance.
struct Request {
  uint64_t ticket = 0;
  uint32_t rel = 0;
  std::vector<uint32_t> c0, c1;
  uint64_t est_bytes = 0;
  int slot = -1;
  bool done = false;
  uint32_t* dev_edges = nullptr;                                        // c0 then c1 on the device
  uint64_t n = 0;
  std::map<int, std::vector<uint64_t>> deltas;                          // IDB rel -> |delta_k|
  std::map<int, std::pair<void*, uint64_t>> result;                     // IDB rel -> codes on the device
};

class Engine {
 public:
  ~Engine();
  hisa_status init(const hisa_config& c);
  hisa_status declare(const char* name, uint32_t arity, int is_idb, uint32_t* id);
  hisa_status load(uint32_t rid, const uint32_t* const* cols, uint64_t n, int on_device);
  hisa_status reset_edb();
  hisa_status add_rule(const hisa_rule* r);
  hisa_status run(hisa_run_stats* stats);
  hisa_status relation_size(uint32_t rid, uint64_t* n);
  hisa_status read_relation(uint32_t rid, uint32_t* const* cols, uint64_t cap, uint64_t* n, int on_device);
  hisa_status delta_counts(uint32_t rid, uint64_t* out, uint32_t cap, uint32_t* n_iters);
  // batched instances (serve.cu)
  hisa_status load_instance(uint32_t rid, uint32_t inst, const uint32_t* const* cols, uint64_t n, int on_device);
  hisa_status instance_size(uint32_t rid, uint32_t inst, uint64_t* n);
  hisa_status read_instance(uint32_t rid, uint32_t inst, uint32_t* const* cols, uint64_t cap, uint64_t* n,
                            int on_device);
  hisa_status instance_delta_counts(uint32_t rid, uint32_t inst, uint64_t* out, uint32_t cap, uint32_t* n_iters);
  hisa_status serve_open(uint32_t max_instances, uint32_t max_value, uint64_t budget);
  hisa_status serve_submit(uint32_t rid, const uint32_t* const* cols, uint64_t n, uint64_t* ticket);
  hisa_status serve_step(uint32_t max_iters, hisa_serve_stats* st);
  hisa_status serve_poll(uint64_t ticket, int* done);
  hisa_status serve_retired(uint64_t* tickets, uint32_t cap, uint32_t* n);
  hisa_status serve_result(uint64_t ticket, uint32_t rid, uint32_t* const* cols, uint64_t cap, uint64_t* n,
                           uint64_t* deltas, uint32_t dcap, uint32_t* n_iters, int on_device);
  hisa_status serve_release(uint64_t ticket);
  hisa_status ctx_fail(hisa_status s, const char* what, const char* detail);
  uint32_t load_inst = 0;   // instance id given to tuples by the next load

  std::string last_error;

 private:
  hisa_status dev_alloc(size_t bytes, void** out);
  void dev_free(void* p);
  // The read scratch (bit matrix, row offsets, staging columns) stays
  // allocated between reads; an allocation that would exceed the budget, or
  // that the allocator refuses, first releases it (never during a read).
  bool release_read_scratch();
  bool reading = false;
  int new_slot(int elem_bytes);
  hisa_status ensure(int id, uint64_t cap);
  hisa_status upload();
  hisa_status download();
  hisa_status check_launch(const char* what);
  hisa_status device_max(const uint32_t* a, const uint32_t* b, uint64_t n, uint32_t* mx);
  hisa_status compile();
  // bit-matrix evaluation of a program of REACH's shape (bitjoin.cuh)
  bool detect_bitjoin();
  hisa_status run_bitjoin(hisa_run_stats* stats, std::chrono::steady_clock::time_point t0);
  bool bitjoin = false;
  int bj_rel = -1, bj_inner = -1;   // R and B of R(x, z) <- B(x, y), R(y, z)
  std::vector<int> bj_base;         // E of the rules R(x, y) <- E(x, y)
  int bj_first = -1, bj_d = -1, bj_d2 = -1, bj_dm = -1, bj_dm2 = -1, bj_tot = -1, bj_ctr = -1;
  int bj_items = -1, bj_hslot = -1, bj_hacc = -1, bj_hdone = -1, bj_todo = -1, bj_items2 = -1, bj_offs2 = -1;
  hisa_status plan_variant(const hisa_rule& R, int delta_atom, std::vector<StepPlan>& out);
  void emit_join(std::vector<Op>& ops, const StepPlan& sp);
  void emit_dense(std::vector<Op>& ops, const StepPlan& sp, bool chain_groups = false, int inner_buf = -1,
                  int table_buf = -1);
  void emit_invert(std::vector<Op>& ops, const StepPlan& sp, bool tmp_probe);
  int sorted_by_other(const StepPlan& sp) const;
  void emit_chain(std::vector<Op>& ops, const StepPlan& sp, bool tmp_index);
  hisa_status plan_all();
  void emit_head(std::vector<Op>& ops, const std::vector<std::vector<StepPlan>>& plans, bool idb_inner);
  void emit_idb_index(std::vector<Op>& ops);
  void emit_sort(std::vector<Op>& ops, int in, int alt, int cnt, int hist, int skip_mask, int stage_bit);
  void emit_tail(std::vector<Op>& ops, bool force);
  void emit_level_merge(std::vector<Op>& ops, const Relation& R, bool force);
  hisa_status merge_levels();
  hisa_status compact_levels();
  template <typename K> hisa_status exec_t(const std::vector<Op>& ops);
  hisa_status exec(const std::vector<Op>& ops);
  template <typename K> hisa_status prepare_rel_t(Relation& r, int order, int slot);
  hisa_status prepare_edb();
  hisa_status regrow();
  hisa_status grow_keep(int id, uint64_t cap, uint64_t keep);
  hisa_status init_run_state();
  hisa_status run_loop(hisa_run_stats* stats, std::chrono::steady_clock::time_point t0);
  hisa_status iterate_once(const std::vector<Op>& ops);
  hisa_status collect_inst_rows(std::vector<std::vector<uint64_t>>& rows);
  hisa_status inst_bounds(int slot, std::vector<uint64_t>& bounds);
  hisa_status decode_range(int slot, uint64_t begin, uint64_t count, std::vector<uint32_t>& c0,
                           std::vector<uint32_t>& c1);
  hisa_status rebuild_serving_edb(const std::vector<uint64_t>& admitted);
  hisa_status retire(const std::vector<uint64_t>& tickets);
  // codes of bit-matrix rows [row0, row0 + nrows) of R, stored order, into
  // `slot` from position `at` (the slot must hold them)
  hisa_status matrix_rows_out(const Relation& R, uint64_t row0, uint64_t nrows, int slot, uint64_t at,
                              const std::vector<uint32_t>* blocks = nullptr);
  uint64_t inst_total(size_t idb_index, uint32_t inst) const;   // sum of an instance's delta sizes
  hisa_status compact_dead();
  hisa_status compact(int slot, int next, const std::vector<uint64_t>& bnd, const std::vector<bool>& drop);
  hisa_status declared_order(int slot, uint64_t begin, uint64_t count, int* out);
  hisa_status resort(int slot, uint64_t begin, uint64_t count, bool swap, int* out);
  hisa_status launch_graph();
  hisa_status build_graph();
  hisa_status launch_once();   // one iteration of opsN as a CUDA graph (batched / served loops)

  hisa_config cfg{};
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaMemPool_t pool = nullptr;
  Grid grid;
  DevState hs{};                 // host mirror of the device state
  DevState* hs_pinned = nullptr; // staging for transfers
  DevState* dst = nullptr;       // device copy
  int nslots = 0;
  int slot_elem[kMaxBufs] = {};
  bool slot_zero[kMaxBufs] = {};   // zero on allocation (look-back status words)
  bool slot_pow2[kMaxBufs] = {};   // capacity must be a power of two (hash tables)
  std::unordered_map<void*, size_t> allocs;
  std::vector<uint64_t> submit_seen;   // serve_submit's distinct-value bitmap (kept cleared)
  uint64_t bytes_in_use = 0, peak_bytes = 0;
  uint32_t regrows = 0;
  Scratch sc{};
  std::vector<Relation> rels;
  std::vector<hisa_rule> rules;
  std::vector<int> idb;
  std::vector<std::vector<StepPlan>> plan1, planN;
  std::vector<Op> ops1, opsN, tail;
  bool compiled = false, edb_dirty = true, ran = false;
  int b = 1;           // domain bits
  bool wide = false;   // 64-bit codes
  int passes = 1;      // radix passes over 2b bits
  int direct_bits = 0; // > 0: run indexes are direct-addressed over this many key bits
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  bool graph_stale = true;
  cudaGraph_t once_graph = nullptr;
  cudaGraphExec_t once_exec = nullptr;
  bool once_stale = true;
  hisa_run_stats last_stats{};
  KernelTimer timer;
  // batched instances: codes carry an instance id above the two columns
  bool batched = false;
  uint32_t max_inst = 0;
  int inst_bits = 0;
  int inst_row = -1;          // slot: per-instance counts of one iteration
  int inst_bnd = -1;          // slot: per-instance bounds of a sorted array
  std::vector<std::vector<std::vector<uint64_t>>> inst_hist;   // [idb][inst] -> |delta_k| per iteration
  // serving session
  bool serving = false;
  int fixed_b = 0, fixed_inst_bits = 0;
  uint32_t serve_slots = 0;
  uint64_t serve_budget = 0, active_bytes = 0, next_ticket = 1;
  std::vector<uint64_t> slot_owner;                  // ticket per slot, 0 = free
  std::vector<char> slot_dirty;                      // a retired instance's tuples still in full
  uint64_t dead_tuples = 0;                          // tuples of retired, not yet compacted instances
  uint64_t dead_bytes = 0;                           // their admission estimates, released at compaction
  bool edb_restage = true;                           // the staged EDB still holds retired instances' tuples
  std::unordered_map<uint64_t, Request> reqs;
  std::deque<uint64_t> pending;
  std::vector<uint64_t> last_retired;   // tickets retired by the latest serve_step
  std::vector<Op> ops_admit;
  int res_slot = -1;          // slot aliasing a request's result codes while they are decoded
  struct KStat { uint64_t launches; double ms, bytes; };
  KStat kstat[kKindCount] = {};
  uint64_t body_kernels = 0;   // kernels in one captured iteration

 public:
  hisa_status kernel_stats(hisa_kernel_stat* out, uint32_t cap, uint32_t* n);
};

}  // namespace hisa
