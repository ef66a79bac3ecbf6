// Batched instances and the serving loop (continuous batching) of the engine.
//
// Many independent fixpoint instances share one run: every code carries its
// instance id above the two columns, so the packed relations are the union of
// the instances and every kernel of the iteration works on all of them at
// once (one launch per stage for the whole instance table).  Joins probe keys
// (instance, value), so instances never meet.  A serving session admits new
// instances at iteration boundaries (their non-recursive rules run in that
// iteration next to everyone else's recursive ones), and retires each
// instance whose delta becomes empty: its tuples are copied out and its range
// of the sorted relations is cut out.
#include <algorithm>
#include <chrono>
#include <cstring>

#include "engine.h"

namespace hisa {

#define CU(call)                                                                           \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) return ctx_fail(HISA_ERR_CUDA, #call, cudaGetErrorString(e_)); \
  } while (0)

static uint32_t instance_slots(uint32_t max_inst) { return max_inst + 1; }

hisa_status Engine::load_instance(uint32_t rid, uint32_t inst, const uint32_t* const* cols, uint64_t n,
                                  int on_device) {
  if (serving) return ctx_fail(HISA_ERR_STATE, "load during a serving session", nullptr);
  if (inst >= (1u << 24)) return ctx_fail(HISA_ERR_INVALID_ARG, "instance id too large", nullptr);
  load_inst = inst;
  hisa_status s = load(rid, cols, n, on_device);
  load_inst = 0;
  if (s) return s;
  batched = true;
  max_inst = std::max(max_inst, inst);
  return HISA_OK;
}

// Per-instance counts of delta (after the commit) of every IDB relation.
hisa_status Engine::collect_inst_rows(std::vector<std::vector<uint64_t>>& rows) {
  const uint32_t ninst = serving ? serve_slots : instance_slots(max_inst);
  hisa_status s;
  if ((s = ensure(inst_row, ninst)) || (s = upload())) return s;
  rows.assign(idb.size(), std::vector<uint64_t>(ninst, 0));
  for (size_t i = 0; i < idb.size(); ++i) {
    const Relation& R = rels[idb[i]];
    CU(cudaMemsetAsync(hs.buf[inst_row].ptr, 0, ninst * 8, stream));
    InstArgs a{dst, R.delta, R.delta, 2 * b, ninst, static_cast<unsigned long long*>(hs.buf[inst_row].ptr)};
    if (wide) launch_inst_hist<uint64_t>(a, grid, stream);
    else launch_inst_hist<uint32_t>(a, grid, stream);
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(rows[i].data(), hs.buf[inst_row].ptr, ninst * 8, cudaMemcpyDeviceToHost, stream));
  }
  CU(cudaStreamSynchronize(stream));
  return HISA_OK;
}

// bounds[i] = first position of instance i in the sorted array of `slot`.
hisa_status Engine::inst_bounds(int slot, std::vector<uint64_t>& bounds) {
  const uint32_t ninst = serving ? serve_slots : instance_slots(max_inst);
  hisa_status s;
  if ((s = ensure(inst_bnd, ninst + 1)) || (s = upload())) return s;
  InstArgs a{dst, slot, slot, 2 * b, ninst, static_cast<unsigned long long*>(hs.buf[inst_bnd].ptr)};
  if (wide) launch_inst_bounds<uint64_t>(a, grid, stream);
  else launch_inst_bounds<uint32_t>(a, grid, stream);
  CU(cudaGetLastError());
  bounds.assign(ninst + 1, 0);
  CU(cudaMemcpyAsync(bounds.data(), hs.buf[inst_bnd].ptr, (ninst + 1) * 8, cudaMemcpyDeviceToHost, stream));
  CU(cudaStreamSynchronize(stream));
  return HISA_OK;
}

hisa_status Engine::decode_range(int slot, uint64_t begin, uint64_t count, std::vector<uint32_t>& c0,
                                 std::vector<uint32_t>& c1) {
  c0.assign(count, 0);
  c1.assign(count, 0);
  if (count == 0) return HISA_OK;
  void *t0, *t1;
  hisa_status s;
  if ((s = dev_alloc(count * 4, &t0)) || (s = dev_alloc(count * 4, &t1))) return s;
  DecodeArgs a{dst, slot, slot, static_cast<uint32_t*>(t0), static_cast<uint32_t*>(t1), b, 0, begin, count};
  if (wide) launch_decode<uint64_t>(a, grid, stream);
  else launch_decode<uint32_t>(a, grid, stream);
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(c0.data(), t0, count * 4, cudaMemcpyDeviceToHost, stream));
  CU(cudaMemcpyAsync(c1.data(), t1, count * 4, cudaMemcpyDeviceToHost, stream));
  dev_free(t0);
  dev_free(t1);
  CU(cudaStreamSynchronize(stream));
  return HISA_OK;
}

// With `blocks`, the rows are those of the listed instance slots' blocks, in
// list order (nrows = blocks->size() << b); row0 is unused.
hisa_status Engine::matrix_rows_out(const Relation& R, uint64_t row0, uint64_t nrows, int slot, uint64_t at,
                                    const std::vector<uint32_t>* blocks) {
  hisa_status s;
  if (blocks) nrows = uint64_t(blocks->size()) << b;
  if ((s = ensure(sc.mrows, nrows + 1))) return s;
  const uint64_t kb = wide ? 8 : 4;
  MatrixExtractArgs a{static_cast<const uint32_t*>(hs.buf[R.fbm].ptr), static_cast<const uint32_t*>(hs.buf[R.fcnt].ptr),
                      row0, nrows, b, static_cast<uint64_t*>(hs.buf[sc.mrows].ptr),
                      static_cast<char*>(hs.buf[slot].ptr) + at * kb};
  if (blocks) {
    if (blocks->empty()) return HISA_OK;
    if ((s = ensure(sc.mslots, blocks->size()))) return s;
    CU(cudaMemcpyAsync(hs.buf[sc.mslots].ptr, blocks->data(), blocks->size() * 4, cudaMemcpyHostToDevice, stream));
    a.slots = static_cast<const uint32_t*>(hs.buf[sc.mslots].ptr);
  }
  if (wide) launch_matrix_extract<uint64_t>(a, grid, stream);
  else launch_matrix_extract<uint32_t>(a, grid, stream);
  CU(cudaGetLastError());
  return HISA_OK;
}

uint64_t Engine::inst_total(size_t i, uint32_t inst) const {
  uint64_t t = 0;
  if (i < inst_hist.size() && inst < inst_hist[i].size())
    for (uint64_t d : inst_hist[i][inst]) t += d;
  return t;
}

static int find_idb(const std::vector<int>& idb, uint32_t rid) {
  for (size_t i = 0; i < idb.size(); ++i)
    if (uint32_t(idb[i]) == rid) return int(i);
  return -1;
}

hisa_status Engine::instance_size(uint32_t rid, uint32_t inst, uint64_t* n) {
  if (!n || rid >= rels.size()) return ctx_fail(HISA_ERR_INVALID_ARG, "instance_size", nullptr);
  if (!batched || inst > max_inst) return ctx_fail(HISA_ERR_INVALID_ARG, "no such instance", nullptr);
  const Relation& r = rels[rid];
  if ((r.idb && !ran) || (!r.idb && edb_dirty)) return ctx_fail(HISA_ERR_STATE, "relation not evaluated yet", nullptr);
  if (r.idb && r.mfull) {   // full as a bit matrix: the instance's deltas are disjoint
    *n = inst_total(size_t(find_idb(idb, rid)), inst);
    return HISA_OK;
  }
  std::vector<uint64_t> bnd;
  hisa_status s = inst_bounds(r.idb ? r.full : r.base, bnd);
  if (s) return s;
  *n = bnd[inst + 1] - bnd[inst];
  return HISA_OK;
}

// Codes [begin, begin + count) of `slot`, stored (c1, c0), exchanged and
// sorted into the declared column order; *out receives the slot holding them
// from position 0 (scratch, valid until the next run).
hisa_status Engine::declared_order(int slot, uint64_t begin, uint64_t count, int* out) {
  return resort(slot, begin, count, true, out);
}

// The same, with or without the column exchange.
hisa_status Engine::resort(int slot, uint64_t begin, uint64_t count, bool swap, int* out) {
  const uint64_t kb = wide ? 8 : 4;
  const int kt = wide ? radix_tile<uint64_t>() : radix_tile<uint32_t>();
  hisa_status s;
  if ((s = ensure(sc.tmp_a, count)) || (s = ensure(sc.tmp_b, count)) ||
      (s = ensure(sc.radix_status, (count / kt + 2) * kRadixDigits)))
    return s;
  if (res_slot < 0) res_slot = new_slot(int(kb));
  hs.buf[res_slot] = {static_cast<char*>(hs.buf[slot].ptr) + begin * kb, count};
  hs.cnt[res_slot] = count;
  if ((s = upload())) return s;
  std::vector<Op> ops;
  if (swap) {
    Op w{};
    w.kind = Op::SWAP;
    w.swap = SwapArgs{dst, res_slot, res_slot, sc.tmp_a, sc.tmp_cnt, b, 0, 0};
    ops.push_back(w);
  } else {
    CU(cudaMemcpyAsync(hs.buf[sc.tmp_a].ptr, hs.buf[res_slot].ptr, count * kb, cudaMemcpyDeviceToDevice, stream));
    Op c{};
    c.kind = Op::CTL;
    c.ctl.st = dst;
    c.ctl.cmd[c.ctl.n++] = {kCtlSetCnt, sc.tmp_cnt, (long long)count, 0};
    ops.push_back(c);
  }
  Op z{};
  z.kind = Op::CTL;
  z.ctl.st = dst;
  z.ctl.cmd[z.ctl.n++] = {kCtlZeroSmall, sc.hist, 8 * 256, 0};
  ops.push_back(z);
  Op h{};
  h.kind = Op::HIST;
  h.hist = RadixHistArgs{dst, sc.tmp_a, sc.tmp_cnt, sc.hist, passes, 0};
  ops.push_back(h);
  emit_sort(ops, sc.tmp_a, sc.tmp_b, sc.tmp_cnt, sc.hist, 0, 0);
  if ((s = exec(ops)) || (s = download())) return s;
  hs.buf[res_slot] = {nullptr, 0};
  hs.cnt[res_slot] = 0;
  if (hs.overflow || hs.error) return ctx_fail(HISA_ERR_CUDA, "re-sort into the declared column order", nullptr);
  *out = (passes & 1) ? sc.tmp_b : sc.tmp_a;
  return upload();
}

hisa_status Engine::read_instance(uint32_t rid, uint32_t inst, uint32_t* const* cols, uint64_t cap, uint64_t* n,
                                  int on_device) {
  if (!cols || !n || rid >= rels.size()) return ctx_fail(HISA_ERR_INVALID_ARG, "read_instance", nullptr);
  if (!batched || inst > max_inst) return ctx_fail(HISA_ERR_INVALID_ARG, "no such instance", nullptr);
  const Relation& r = rels[rid];
  if ((r.idb && !ran) || (!r.idb && edb_dirty)) return ctx_fail(HISA_ERR_STATE, "relation not evaluated yet", nullptr);
  int slot = r.idb ? r.full : r.base;
  hisa_status s;
  uint64_t lo = 0, cnt = 0;
  if (r.idb && r.mfull) {   // the instance's block of matrix rows, read out as codes
    cnt = inst_total(size_t(find_idb(idb, rid)), inst);
    *n = cnt;
    if (cap < cnt) return ctx_fail(HISA_ERR_CAPACITY, "read_instance: buffer too small", nullptr);
    if (cnt == 0) return HISA_OK;
    if ((s = ensure(sc.gather, cnt)) || (s = matrix_rows_out(r, uint64_t(inst) << b, 1ull << b, sc.gather, 0)))
      return s;
    slot = sc.gather;
  } else {
    std::vector<uint64_t> bnd;
    if ((s = inst_bounds(slot, bnd))) return s;
    lo = bnd[inst];
    cnt = bnd[inst + 1] - bnd[inst];
    *n = cnt;
    if (cap < cnt) return ctx_fail(HISA_ERR_CAPACITY, "read_instance: buffer too small", nullptr);
    if (cnt == 0) return HISA_OK;
  }
  int src = slot;
  if (r.idb && r.order == 1) {   // stored (c1, c0): into the declared order
    if ((s = declared_order(slot, lo, cnt, &src))) return s;
    lo = 0;
  }
  if (on_device) {
    DecodeArgs a{dst, src, src, cols[0], cols[1], b, 0, lo, cnt};
    if (wide) launch_decode<uint64_t>(a, grid, stream);
    else launch_decode<uint32_t>(a, grid, stream);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(stream));
    return HISA_OK;
  }
  std::vector<uint32_t> c0, c1;
  if ((s = decode_range(src, lo, cnt, c0, c1))) return s;
  std::memcpy(cols[0], c0.data(), cnt * 4);
  std::memcpy(cols[1], c1.data(), cnt * 4);
  return HISA_OK;
}

hisa_status Engine::instance_delta_counts(uint32_t rid, uint32_t inst, uint64_t* out, uint32_t cap,
                                          uint32_t* n_iters) {
  if (!n_iters || rid >= rels.size()) return ctx_fail(HISA_ERR_INVALID_ARG, "instance_delta_counts", nullptr);
  const int i = find_idb(idb, rid);
  if (i < 0 || !batched || !ran) return ctx_fail(HISA_ERR_INVALID_ARG, "not an evaluated IDB relation", nullptr);
  if (size_t(i) >= inst_hist.size() || inst >= inst_hist[i].size()) {
    *n_iters = 0;
    return HISA_OK;
  }
  const auto& h = inst_hist[i][inst];
  uint32_t K = uint32_t(h.size());
  while (K > 0 && h[K - 1] == 0) --K;
  *n_iters = K;
  for (uint32_t k = 0; k < K && k < cap && out; ++k) out[k] = h[k];
  if (cap < K) return ctx_fail(HISA_ERR_CAPACITY, "instance_delta_counts: buffer too small", nullptr);
  return HISA_OK;
}

// ---- serving --------------------------------------------------------------------------

hisa_status Engine::serve_open(uint32_t max_instances, uint32_t max_value, uint64_t budget) {
  if (serving) return ctx_fail(HISA_ERR_STATE, "serving session already open", nullptr);
  if (max_instances == 0 || rules.empty()) return ctx_fail(HISA_ERR_INVALID_ARG, "serve_open", nullptr);
  for (auto& r : rels)
    if (!r.idb && r.staged) return ctx_fail(HISA_ERR_STATE, "EDB tuples loaded before serve_open", nullptr);
  int bb = 1;
  while (bb < 32 && (uint64_t(max_value) >> bb) != 0) ++bb;
  int ib = 1;
  while (ib < 32 && (uint64_t(max_instances - 1) >> ib) != 0) ++ib;
  if (ib + bb > 32) return ctx_fail(HISA_ERR_UNSUPPORTED, "instance bits + domain bits exceed 32", nullptr);
  serving = true;
  batched = true;
  fixed_b = bb;
  fixed_inst_bits = ib;
  serve_slots = max_instances;
  max_inst = max_instances - 1;
  serve_budget = budget ? budget : cfg.hbm_budget_bytes;
  active_bytes = 0;
  slot_owner.assign(max_instances, 0);
  slot_dirty.assign(max_instances, 0);
  dead_tuples = 0;
  dead_bytes = 0;
  edb_restage = true;
  hisa_status s;
  if ((s = compile())) return s;
  // plans: ordinary iterations, and admission iterations that also run the
  // non-recursive rules (for the instances admitted at that boundary)
  ops1.clear();
  opsN.clear();
  tail.clear();
  ops_admit.clear();
  std::vector<std::vector<StepPlan>> both = plan1;
  both.insert(both.end(), planN.begin(), planN.end());
  emit_head(ops_admit, both, true);
  emit_tail(ops_admit, false);
  emit_head(opsN, planN, true);
  emit_tail(opsN, false);
  emit_tail(tail, false);
  if ((s = init_run_state())) return s;
  for (int r : idb) rels[r].delta_counts.clear();
  ran = true;
  return HISA_OK;
}

hisa_status Engine::serve_submit(uint32_t rid, const uint32_t* const* cols, uint64_t n, uint64_t* ticket) {
  if (!serving) return ctx_fail(HISA_ERR_STATE, "no serving session", nullptr);
  if (rid >= rels.size() || rels[rid].idb || !ticket || (n && (!cols || !cols[0] || !cols[1])))
    return ctx_fail(HISA_ERR_INVALID_ARG, "serve_submit", nullptr);
  Request q;
  q.ticket = next_ticket++;
  q.rel = rid;
  // distinct values, by a bitmap over the session's fixed domain (2^b values)
  if (submit_seen.size() != (size_t(1) << fixed_b) / 64 + 1) submit_seen.assign((size_t(1) << fixed_b) / 64 + 1, 0);
  uint64_t distinct = 0;
  for (int c = 0; c < 2 && n; ++c)
    for (uint64_t i = 0; i < n; ++i) {
      const uint32_t v = cols[c][i];
      if ((uint64_t(v) >> fixed_b) != 0) {
        std::fill(submit_seen.begin(), submit_seen.end(), 0);
        return ctx_fail(HISA_ERR_INVALID_ARG, "value above max_value", nullptr);
      }
      uint64_t& w = submit_seen[v >> 6];
      const uint64_t bit = 1ull << (v & 63);
      distinct += (w & bit) ? 0 : 1;
      w |= bit;
    }
  for (int c = 0; c < 2 && n; ++c)   // clear only the words that were set
    for (uint64_t i = 0; i < n; ++i) submit_seen[cols[c][i] >> 6] = 0;
  // worst case of a binary IDB relation over these values, in both versions
  q.est_bytes = distinct * distinct * (wide ? 8 : 4) * 2 + n * 64;
  q.n = n;
  if (n) {   // the request's tuples move to the device once (the caller's arrays may go)
    void* p;
    hisa_status s = dev_alloc(2 * n * 4, &p);
    if (s) return s;
    q.dev_edges = static_cast<uint32_t*>(p);
    CU(cudaMemcpyAsync(q.dev_edges, cols[0], n * 4, cudaMemcpyHostToDevice, stream));
    CU(cudaMemcpyAsync(q.dev_edges + n, cols[1], n * 4, cudaMemcpyHostToDevice, stream));
    CU(cudaStreamSynchronize(stream));
  }
  *ticket = q.ticket;
  pending.push_back(q.ticket);
  reqs.emplace(q.ticket, std::move(q));
  return HISA_OK;
}

// The EDB of a serving session: the tuples of the active requests, tagged
// with their slots, then sorted and indexed again (after admissions).  The
// newly admitted requests' tuples are appended to the staged ones; the
// staging is rebuilt from the active requests only after a compaction (a
// retired instance's staged tuples join nothing meanwhile: its delta is
// empty and instance ids keep codes apart).
hisa_status Engine::rebuild_serving_edb(const std::vector<uint64_t>& admitted) {
  std::vector<uint64_t> add;
  if (edb_restage) {
    for (auto& r : rels)
      if (!r.idb) r.staged = 0;
    for (uint32_t slot = 0; slot < serve_slots; ++slot)
      if (slot_owner[slot]) add.push_back(slot_owner[slot]);
    edb_restage = false;
  } else {
    add = admitted;
  }
  for (uint64_t t : add) {
    Request& q = reqs[t];
    if (!q.n) continue;
    const uint32_t* cols[2] = {q.dev_edges, q.dev_edges + q.n};
    load_inst = uint32_t(q.slot);
    hisa_status s = load(q.rel, cols, q.n, 1);
    load_inst = 0;
    if (s) return s;
  }
  return prepare_edb();
}

// Keeps the instance ranges of `slot` (bounds `bnd`) not marked in `drop`:
// the kept runs are copied into `next`, which then becomes `slot`.
hisa_status Engine::compact(int slot, int next, const std::vector<uint64_t>& bnd, const std::vector<bool>& drop) {
  const uint64_t kb = wide ? 8 : 4;
  const uint64_t n = hs.cnt[slot];
  hisa_status s;
  if ((s = ensure(next, std::max<uint64_t>(n, 1)))) return s;
  uint64_t w = 0;
  uint32_t i = 0;
  while (i < serve_slots) {
    if (drop[i]) {
      ++i;
      continue;
    }
    uint32_t j = i;
    while (j < serve_slots && !drop[j]) ++j;
    const uint64_t lo = bnd[i], hi = bnd[j];
    if (hi > lo)
      CU(cudaMemcpyAsync(static_cast<char*>(hs.buf[next].ptr) + w * kb, static_cast<char*>(hs.buf[slot].ptr) + lo * kb,
                         (hi - lo) * kb, cudaMemcpyDeviceToDevice, stream));
    w += hi - lo;
    i = j;
  }
  std::swap(hs.buf[slot], hs.buf[next]);
  hs.cnt[slot] = w;
  hs.cnt[next] = 0;
  return HISA_OK;
}

// Removes the tuples of retired instances from full (both levels) and its
// mirror.  Deferred until a slot is reused or the dead tuples are half of the
// live ones: a retired instance's tuples join nothing (its delta is empty and
// instance ids keep codes apart), so they only cost merge traffic meanwhile.
hisa_status Engine::compact_dead() {
  hisa_status s;
  std::vector<bool> drop(serve_slots, false);
  bool any = false;
  for (uint32_t i = 0; i < serve_slots; ++i)
    if (slot_dirty[i]) drop[i] = any = true;
  if (!any) return HISA_OK;
  for (int r : idb) {
    Relation& R = rels[r];
    if (R.mfull) {   // clear the retired instances' blocks of rows
      const uint64_t nw = b >= 5 ? (1ull << (b - 5)) : 1ull;
      for (uint32_t i = 0; i < serve_slots; ++i) {
        if (!drop[i]) continue;
        const uint64_t row0 = uint64_t(i) << b;
        CU(cudaMemsetAsync(static_cast<uint32_t*>(hs.buf[R.fbm].ptr) + row0 * nw, 0, (1ull << b) * nw * 4, stream));
        CU(cudaMemsetAsync(static_cast<uint32_t*>(hs.buf[R.fcnt].ptr) + row0, 0, (1ull << b) * 4, stream));
      }
      hs.cnt[R.full] -= std::min(hs.cnt[R.full], dead_tuples);   // (the only IDB relation)
      continue;
    }
    std::vector<uint64_t> bnd;
    if ((s = inst_bounds(R.full, bnd)) || (s = compact(R.full, R.full_next, bnd, drop))) return s;
    if (R.log && ((s = inst_bounds(R.l1, bnd)) || (s = compact(R.l1, R.l1_next, bnd, drop)))) return s;
    if (R.need_idx[1] && ((s = inst_bounds(R.rev, bnd)) || (s = compact(R.rev, R.rev_next, bnd, drop)))) return s;
  }
  std::fill(slot_dirty.begin(), slot_dirty.end(), 0);
  dead_tuples = 0;
  active_bytes -= std::min(active_bytes, dead_bytes);
  dead_bytes = 0;
  edb_restage = true;
  return upload();
}

// Copies out the tuples of finished requests (they leave full lazily).
hisa_status Engine::retire(const std::vector<uint64_t>& tickets) {
  if (tickets.empty()) return HISA_OK;
  hisa_status s;
  for (int r : idb) {
    Relation& R = rels[r];
    const uint64_t kb = wide ? 8 : 4;
    if (R.mfull) {
      // each finished instance's block of rows read out as codes (its size is
      // the sum of its delta sizes), sorted into the declared column order,
      // copied aside; the block is cleared when the slot is compacted
      uint64_t total = 0;
      std::vector<uint64_t> cnt(tickets.size(), 0);
      for (size_t k = 0; k < tickets.size(); ++k) {
        for (uint64_t d : reqs[tickets[k]].deltas[r]) cnt[k] += d;
        total += cnt[k];
      }
      if (total > 0) {
        if ((s = ensure(sc.gather, total))) return s;
        int src = sc.gather;
        if (R.order == 1 && b >= 8) {
          // stored column-swapped: each block transposed (256 x 256-bit tiles)
          // and its rows read out in the declared order, no sort
          const uint64_t nw = 1ull << (b - 5);
          if ((s = ensure(sc.read_m, (1ull << b) * nw)) || (s = ensure(sc.mrows, (1ull << b) + 1))) return s;
          uint64_t w = 0;
          for (size_t k = 0; k < tickets.size(); ++k) {
            if (!cnt[k]) continue;
            const uint64_t slot = uint64_t(reqs[tickets[k]].slot);
            uint32_t* tm = static_cast<uint32_t*>(hs.buf[sc.read_m].ptr);
            launch_matrix_transpose(MatrixTransposeArgs{static_cast<const uint32_t*>(hs.buf[R.fbm].ptr) +
                                                            (slot << b) * nw, tm, b},
                                    grid, stream);
            MatrixExtractArgs xa{tm, nullptr, 0, 1ull << b, b, static_cast<uint64_t*>(hs.buf[sc.mrows].ptr),
                                 static_cast<char*>(hs.buf[sc.gather].ptr) + w * kb};
            xa.standalone = true;
            xa.code_row0 = slot << b;
            if (wide) launch_matrix_extract<uint64_t>(xa, grid, stream);
            else launch_matrix_extract<uint32_t>(xa, grid, stream);
            CU(cudaGetLastError());
            w += cnt[k];
          }
        } else {
          std::vector<uint32_t> blocks;   // one read-out of all finished blocks, in slot order
          for (size_t k = 0; k < tickets.size(); ++k)
            if (cnt[k]) blocks.push_back(uint32_t(reqs[tickets[k]].slot));
          if ((s = matrix_rows_out(R, 0, 0, sc.gather, 0, &blocks))) return s;
          // (stored in the declared order: the rows are sorted already)
          if (R.order == 1 && (s = resort(sc.gather, 0, total, true, &src))) return s;
        }
        hs.cnt[src] = total;
        uint64_t at = 0;
        for (size_t k = 0; k < tickets.size(); ++k) {   // instances stay in slot order
          Request& q = reqs[tickets[k]];
          void* p = nullptr;
          if (cnt[k]) {
            if ((s = dev_alloc(cnt[k] * kb, &p))) return s;
            CU(cudaMemcpyAsync(p, static_cast<char*>(hs.buf[src].ptr) + at * kb, cnt[k] * kb,
                               cudaMemcpyDeviceToDevice, stream));
          }
          q.result[r] = {p, cnt[k]};
          at += cnt[k];
        }
      } else {
        for (uint64_t t : tickets) reqs[t].result[r] = {nullptr, 0};
      }
      // the rows stay until the slot's compaction: an admission iteration
      // derives a retired instance's first tuples again from its staged EDB,
      // and its full must still remove them
      dead_tuples += total;
      continue;
    }
    std::vector<uint64_t> bnd, bnd1;
    if ((s = inst_bounds(R.full, bnd))) return s;
    if (R.log && (s = inst_bounds(R.l1, bnd1))) return s;
    if (!R.log && R.order == 0) {   // one sorted array in the declared order: copy the ranges
      for (uint64_t t : tickets) {
        Request& q = reqs[t];
        const uint64_t lo = bnd[q.slot], cnt = bnd[q.slot + 1] - bnd[q.slot];
        void* p = nullptr;
        if (cnt) {   // the finished instance's codes, copied aside on the device
          if ((s = dev_alloc(cnt * kb, &p))) return s;
          CU(cudaMemcpyAsync(p, static_cast<char*>(hs.buf[R.full].ptr) + lo * kb, cnt * kb,
                             cudaMemcpyDeviceToDevice, stream));
        }
        q.result[r] = {p, cnt};
        dead_tuples += cnt;
      }
      continue;
    }
    // else every finished instance's codes from both levels are gathered and
    // sorted together (instance ids keep them apart), then cut by instance
    uint64_t total = 0;
    for (uint64_t t : tickets) {
      const Request& q = reqs[t];
      total += bnd[q.slot + 1] - bnd[q.slot];
      if (R.log) total += bnd1[q.slot + 1] - bnd1[q.slot];
    }
    if (total == 0) {
      for (uint64_t t : tickets) reqs[t].result[r] = {nullptr, 0};
      continue;
    }
    if ((s = ensure(sc.gather, total))) return s;
    char* g = static_cast<char*>(hs.buf[sc.gather].ptr);
    uint64_t w = 0;
    for (uint64_t t : tickets) {
      const Request& q = reqs[t];
      for (int lv = 0; lv < (R.log ? 2 : 1); ++lv) {
        const std::vector<uint64_t>& bb = lv ? bnd1 : bnd;
        const uint64_t lo = bb[q.slot], cnt = bb[q.slot + 1] - bb[q.slot];
        if (cnt)
          CU(cudaMemcpyAsync(g + w * kb, static_cast<char*>(hs.buf[lv ? R.l1 : R.full].ptr) + lo * kb, cnt * kb,
                             cudaMemcpyDeviceToDevice, stream));
        w += cnt;
      }
    }
    int src = -1;
    if ((s = resort(sc.gather, 0, total, R.order == 1, &src))) return s;
    hs.cnt[src] = total;
    std::vector<uint64_t> sb;
    if ((s = inst_bounds(src, sb))) return s;
    for (uint64_t t : tickets) {
      Request& q = reqs[t];
      const uint64_t lo = sb[q.slot], cnt = sb[q.slot + 1] - sb[q.slot];
      void* p = nullptr;
      if (cnt) {
        if ((s = dev_alloc(cnt * kb, &p))) return s;
        CU(cudaMemcpyAsync(p, static_cast<char*>(hs.buf[src].ptr) + lo * kb, cnt * kb, cudaMemcpyDeviceToDevice,
                           stream));
      }
      q.result[r] = {p, cnt};
      dead_tuples += cnt;
    }
  }
  for (uint64_t t : tickets) {
    Request& q = reqs[t];
    slot_owner[q.slot] = 0;
    slot_dirty[q.slot] = 1;   // its tuples leave full at the next compaction
    dead_bytes += q.est_bytes;   // still in memory until the compaction
    q.done = true;
    dev_free(q.dev_edges);
    q.dev_edges = nullptr;
  }
  return upload();
}

hisa_status Engine::serve_step(uint32_t max_iters, hisa_serve_stats* st) {
  if (!serving) return ctx_fail(HISA_ERR_STATE, "no serving session", nullptr);
  hisa_serve_stats out{};
  hisa_status s;
  last_retired.clear();
  // phase clock: with HISA_FLAG_PHASE_TIMES a phase ends with a synchronisation
  const bool sync_phases = (cfg.flags & HISA_FLAG_PHASE_TIMES) != 0;
  auto tick = std::chrono::steady_clock::now();
  auto phase = [&](double& acc) {
    if (sync_phases) cudaStreamSynchronize(stream);
    const auto now = std::chrono::steady_clock::now();
    acc += std::chrono::duration<double, std::milli>(now - tick).count();
    tick = now;
  };
  auto compact_timed = [&]() {
    phase(out.ms_admit);   // what came before belongs to the caller's phase
    const hisa_status r = compact_dead();
    phase(out.ms_compact);
    return r;
  };
  for (uint32_t it = 0; it < std::max(max_iters, 1u); ++it) {
    // admission at the iteration boundary: free slot and budget
    std::vector<uint64_t> admitted;
    // an admission iteration re-stages and re-indexes the EDB and runs the
    // non-recursive rules: while the budget is three-quarters used, wait
    // for a quarter to free up so admissions come in groups
    const bool busy = serve_budget && active_bytes > serve_budget / 4 * 3 &&
                      std::any_of(slot_owner.begin(), slot_owner.end(), [](uint64_t t) { return t != 0; });
    while (!pending.empty() && !busy) {
      const uint64_t t = pending.front();
      Request& q = reqs[t];
      auto clean_free = [&] {
        for (uint32_t i = 0; i < serve_slots; ++i)
          if (!slot_owner[i] && !slot_dirty[i]) return slot_owner.begin() + i;
        return slot_owner.end();
      };
      auto free_slot = clean_free();
      if (free_slot == slot_owner.end() &&
          std::find(slot_owner.begin(), slot_owner.end(), 0ull) != slot_owner.end()) {
        if ((s = compact_timed())) return s;   // a retired slot is reused: its tuples go first
        free_slot = clean_free();
      }
      if (free_slot == slot_owner.end()) break;
      if (serve_budget && active_bytes + q.est_bytes > serve_budget && dead_bytes > 0) {
        if ((s = compact_timed())) return s;   // retired instances' memory counts until it is freed
      }
      if (serve_budget && active_bytes + q.est_bytes > serve_budget && active_bytes > 0) break;
      q.slot = int(free_slot - slot_owner.begin());
      *free_slot = t;
      active_bytes += q.est_bytes;
      admitted.push_back(t);
      pending.pop_front();
    }
    out.admitted += uint32_t(admitted.size());
    if (!admitted.empty() && (s = rebuild_serving_edb(admitted))) return s;
    phase(out.ms_admit);
    const bool any_active = std::any_of(slot_owner.begin(), slot_owner.end(), [](uint64_t t) { return t != 0; });
    if (!any_active) break;
    // one iteration of the shared fixpoint
    if ((s = iterate_once(admitted.empty() ? opsN : ops_admit))) return s;
    ++out.iterations;
    phase(out.ms_iterate);
    std::vector<std::vector<uint64_t>> rows;
    if ((s = collect_inst_rows(rows))) return s;
    phase(out.ms_rows);
    std::vector<uint64_t> finished;
    for (uint32_t slot = 0; slot < serve_slots; ++slot) {
      const uint64_t t = slot_owner[slot];
      if (!t) continue;
      Request& q = reqs[t];
      bool empty = true;
      for (size_t i = 0; i < idb.size(); ++i) {
        q.deltas[idb[i]].push_back(rows[i][slot]);
        if (rows[i][slot]) empty = false;
      }
      if (empty) finished.push_back(t);
    }
    for (uint64_t t : finished)
      for (auto& kv : reqs[t].deltas) {
        auto& v = kv.second;
        while (!v.empty() && v.back() == 0) v.pop_back();
      }
    if ((s = retire(finished))) return s;
    out.retired += uint32_t(finished.size());
    last_retired.insert(last_retired.end(), finished.begin(), finished.end());
    phase(out.ms_retire);
    uint64_t live = 0;
    for (int r : idb) live += hs.cnt[rels[r].full] + (rels[r].log ? hs.cnt[rels[r].l1] : 0);
    if (dead_tuples * 2 > live) {
      if ((s = compact_dead())) return s;
      phase(out.ms_compact);
    }
  }
  out.pending = uint32_t(pending.size());
  out.active = uint32_t(std::count_if(slot_owner.begin(), slot_owner.end(), [](uint64_t t) { return t != 0; }));
  if (st) *st = out;
  return HISA_OK;
}

hisa_status Engine::serve_retired(uint64_t* tickets, uint32_t cap, uint32_t* n) {
  if (!serving) return ctx_fail(HISA_ERR_STATE, "no serving session", nullptr);
  *n = uint32_t(last_retired.size());
  for (uint32_t i = 0; tickets && i < cap && i < last_retired.size(); ++i) tickets[i] = last_retired[i];
  if (tickets && cap < last_retired.size()) return ctx_fail(HISA_ERR_CAPACITY, "serve_retired: buffer too small", nullptr);
  return HISA_OK;
}

hisa_status Engine::serve_poll(uint64_t ticket, int* done) {
  auto it = reqs.find(ticket);
  if (it == reqs.end() || !done) return ctx_fail(HISA_ERR_INVALID_ARG, "unknown ticket", nullptr);
  *done = it->second.done ? 1 : 0;
  return HISA_OK;
}

hisa_status Engine::serve_result(uint64_t ticket, uint32_t rid, uint32_t* const* cols, uint64_t cap, uint64_t* n,
                                 uint64_t* deltas, uint32_t dcap, uint32_t* n_iters, int on_device) {
  auto it = reqs.find(ticket);
  if (it == reqs.end() || !n) return ctx_fail(HISA_ERR_INVALID_ARG, "unknown ticket", nullptr);
  Request& q = it->second;
  if (!q.done) return ctx_fail(HISA_ERR_STATE, "request not complete", nullptr);
  auto r = q.result.find(int(rid));
  const uint64_t size = r == q.result.end() ? 0 : r->second.second;
  *n = size;
  const auto& dv = q.deltas[int(rid)];
  if (n_iters) *n_iters = uint32_t(dv.size());
  for (uint32_t k = 0; deltas && k < dv.size() && k < dcap; ++k) deltas[k] = dv[k];
  if (cap < size || (deltas && dcap < dv.size()))
    return ctx_fail(HISA_ERR_CAPACITY, "serve_result: buffer too small", nullptr);
  if (!size || !cols) return HISA_OK;
  // decode the stored codes through a slot that aliases them
  if (res_slot < 0) res_slot = new_slot(wide ? 8 : 4);
  hs.buf[res_slot] = {r->second.first, size};
  hs.cnt[res_slot] = size;
  hisa_status s = upload();
  if (s) return s;
  uint32_t *d0 = cols[0], *d1 = cols[1];
  void *t0 = nullptr, *t1 = nullptr;
  if (!on_device) {
    if ((s = dev_alloc(size * 4, &t0)) || (s = dev_alloc(size * 4, &t1))) return s;
    d0 = static_cast<uint32_t*>(t0);
    d1 = static_cast<uint32_t*>(t1);
  }
  DecodeArgs a{dst, res_slot, res_slot, d0, d1, b, 0, 0, size};
  if (wide) launch_decode<uint64_t>(a, grid, stream);
  else launch_decode<uint32_t>(a, grid, stream);
  CU(cudaGetLastError());
  if (!on_device) {
    CU(cudaMemcpyAsync(cols[0], d0, size * 4, cudaMemcpyDeviceToHost, stream));
    CU(cudaMemcpyAsync(cols[1], d1, size * 4, cudaMemcpyDeviceToHost, stream));
    dev_free(t0);
    dev_free(t1);
  }
  CU(cudaStreamSynchronize(stream));
  hs.buf[res_slot] = {nullptr, 0};
  hs.cnt[res_slot] = 0;
  return upload();
}

hisa_status Engine::serve_release(uint64_t ticket) {
  auto it = reqs.find(ticket);
  if (it == reqs.end()) return ctx_fail(HISA_ERR_INVALID_ARG, "unknown ticket", nullptr);
  if (!it->second.done) return ctx_fail(HISA_ERR_STATE, "request not complete", nullptr);
  for (auto& kv : it->second.result) dev_free(kv.second.first);
  reqs.erase(it);
  return HISA_OK;
}

}  // namespace hisa
