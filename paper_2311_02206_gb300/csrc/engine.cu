// Host side of the engine: relation store, rule compiler, eager buffer
// management and the semi-naive fixpoint driver behind include/hisa.h.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "engine.h"

namespace hisa {

// ---- errors ---------------------------------------------------------------------------

#define CU(call)                                                                  \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) return ctx_fail(HISA_ERR_CUDA, #call, cudaGetErrorString(e_)); \
  } while (0)

hisa_status Engine::ctx_fail(hisa_status s, const char* what, const char* detail) {
  char buf[512];
  snprintf(buf, sizeof buf, "%s%s%s", what ? what : "", detail ? ": " : "", detail ? detail : "");
  last_error = buf;
  return s;
}

// ---- memory ---------------------------------------------------------------------------

hisa_status Engine::dev_alloc(size_t bytes, void** out) {
  *out = nullptr;
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  if (cfg.hbm_budget_bytes && bytes_in_use + bytes > cfg.hbm_budget_bytes &&
      (!release_read_scratch() || bytes_in_use + bytes > cfg.hbm_budget_bytes))
    return ctx_fail(HISA_ERR_OOM, "HBM budget exceeded", nullptr);
  void* p = nullptr;
  for (int attempt = 0; !p; ++attempt) {
    if (cfg.alloc) {
      p = cfg.alloc(bytes, stream, cfg.user);
      if (!p && (attempt || !release_read_scratch()))
        return ctx_fail(HISA_ERR_OOM, "allocator hook returned NULL", nullptr);
    } else {
      cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, pool, stream);
      if (e != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        if (attempt || !release_read_scratch())
          return ctx_fail(HISA_ERR_OOM, "cudaMallocFromPoolAsync", cudaGetErrorString(e));
      }
    }
  }
  allocs[p] = bytes;
  bytes_in_use += bytes;
  peak_bytes = std::max(peak_bytes, bytes_in_use);
  *out = p;
  return HISA_OK;
}

void Engine::dev_free(void* p) {
  if (!p) return;
  auto it = allocs.find(p);
  if (it == allocs.end()) return;
  if (cfg.free) cfg.free(p, it->second, stream, cfg.user);
  else cudaFreeAsync(p, stream);
  bytes_in_use -= it->second;
  allocs.erase(it);
}

bool Engine::release_read_scratch() {
  if (reading) return false;
  bool freed = false;
  for (int id : {sc.read_m, sc.read_rows, sc.read_s0, sc.read_s1}) {
    if (id < 0 || !hs.buf[id].ptr) continue;
    dev_free(hs.buf[id].ptr);
    hs.buf[id] = {nullptr, 0};
    freed = true;
  }
  return freed;
}

int Engine::new_slot(int elem_bytes) {
  const int id = nslots++;
  slot_elem[id] = elem_bytes;
  hs.buf[id] = {nullptr, 0};
  hs.cnt[id] = 0;
  return id;
}

// Grows slot `id` to at least `cap` elements (contents are not kept: the old
// buffer is released first, so growth never holds both).
hisa_status Engine::ensure(int id, uint64_t cap) {
  if (hs.buf[id].cap >= cap && hs.buf[id].ptr) return HISA_OK;
  dev_free(hs.buf[id].ptr);
  hs.buf[id] = {nullptr, 0};
  void* p;
  hisa_status s = dev_alloc(size_t(std::max<uint64_t>(cap, 1)) * slot_elem[id], &p);
  if (s) return s;
  hs.buf[id] = {p, std::max<uint64_t>(cap, 1)};
  if (slot_zero[id]) {
    // look-back words: a recycled allocation may hold words of another
    // context whose epoch tags collide with ours; zero means "not published"
    CU(cudaMemsetAsync(p, 0, size_t(std::max<uint64_t>(cap, 1)) * slot_elem[id], stream));
  }
  return HISA_OK;
}

hisa_status Engine::upload() {
  std::memcpy(hs_pinned, &hs, sizeof(DevState));
  CU(cudaMemcpyAsync(dst, hs_pinned, sizeof(DevState), cudaMemcpyHostToDevice, stream));
  CU(cudaStreamSynchronize(stream));   // hs_pinned is reused by the next transfer
  return HISA_OK;
}

hisa_status Engine::download() {
  CU(cudaMemcpyAsync(hs_pinned, dst, sizeof(DevState), cudaMemcpyDeviceToHost, stream));
  CU(cudaStreamSynchronize(stream));
  std::memcpy(&hs, hs_pinned, sizeof(DevState));
  return HISA_OK;
}

hisa_status Engine::check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return ctx_fail(HISA_ERR_CUDA, what, cudaGetErrorString(e));
  return HISA_OK;
}

// ---- lifecycle ------------------------------------------------------------------------

hisa_status Engine::init(const hisa_config& c) {
  cfg = c;
  if (cfg.load_factor <= 0.f || cfg.load_factor > 0.95f) cfg.load_factor = 0.8f;
  if (cfg.ebm_k <= 0.f) cfg.ebm_k = 2.f;
  if (cfg.max_iters == 0) cfg.max_iters = 1000000;
  if (!(cfg.pull_ratio > 0.f) || cfg.pull_ratio > 4096.f) cfg.pull_ratio = float(kPullK16) / 16.f;
  // tuning knobs outside their ranges fall back to the defaults
  if (cfg.radix_items != 0 && cfg.radix_items != uint32_t(RadixCfg<uint32_t>::items) &&
      cfg.radix_items != uint32_t(RadixCfg<uint32_t>::items_alt) && cfg.radix_items != uint32_t(RadixCfg<uint64_t>::items) &&
      cfg.radix_items != uint32_t(RadixCfg<uint64_t>::items_alt))
    cfg.radix_items = 0;
  if (cfg.dense_unit != 0 && (cfg.dense_unit < 64 || cfg.dense_unit > (1u << 20))) cfg.dense_unit = 0;
  if (cfg.device >= 0) CU(cudaSetDevice(cfg.device));
  CU(cudaGetDevice(&device));
  stream = static_cast<cudaStream_t>(cfg.cuda_stream);
  int sms = 0;
  CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  grid.sms = sms;
  // persistent grids: resident CTAs per SM from the kernels' footprints
  grid.radix = sms * 3;
  grid.setop = sms * 5;
  grid.join = sms * 4;
  grid.small = sms * 4;
  if (!cfg.alloc) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    CU(cudaMemPoolCreate(&pool, &props));
    uint64_t thr = ~0ull;
    CU(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
  }
  CU(cudaMallocHost(&hs_pinned, sizeof(DevState)));
  std::memset(&hs, 0, sizeof hs);
  void* p;
  hisa_status s = dev_alloc(sizeof(DevState), &p);
  if (s) return s;
  dst = static_cast<DevState*>(p);
  // shared scratch
  sc.empty = new_slot(8);
  sc.hist = new_slot(8);
  sc.radix_status = new_slot(8);
  sc.split = new_slot(8);
  sc.setop_status = new_slot(8);
  sc.offs = new_slot(8);
  sc.join_status = new_slot(8);
  sc.starts = new_slot(8);
  sc.tmp_a = new_slot(8);
  sc.tmp_b = new_slot(8);
  sc.runs = nslots++;
  sc.total = nslots++;
  sc.tmp_cnt = nslots++;
  sc.groups = new_slot(8);
  sc.dense_status = new_slot(8);
  sc.dense_bm = new_slot(4);
  sc.tmp_hist = new_slot(8);
  sc.gather = new_slot(4);
  sc.mrows = new_slot(8);
  sc.mslots = new_slot(4);
  sc.dense_first = new_slot(8);
  sc.dense_units = new_slot(8);
  sc.dense_done = new_slot(4);
  sc.dense_mslot = new_slot(4);
  sc.dense_bmm = new_slot(4);
  sc.chain_dfirst = new_slot(8);
  sc.chain_pre = new_slot(8);
  sc.chain_tfirst = new_slot(8);
  sc.dense_plist = new_slot(4);
  sc.pull_cnt = nslots++;
  sc.pull_raw_cnt = nslots++;
  sc.dense_bm_prev = new_slot(4);
  sc.prev_gi = new_slot(4);
  sc.read_m = new_slot(4);
  sc.read_rows = new_slot(8);
  sc.read_s0 = new_slot(4);
  sc.read_s1 = new_slot(4);
  sc.group_cnt = nslots++;
  sc.raw_cnt = nslots++;
  slot_zero[sc.radix_status] = slot_zero[sc.setop_status] = slot_zero[sc.join_status] = true;
  slot_zero[sc.dense_status] = true;
  slot_zero[sc.dense_bmm] = true;   // split groups' units OR into these; each is zeroed again after use
  if ((s = ensure(sc.empty, 1)) || (s = ensure(sc.hist, 8 * 256))) return s;
  return upload();
}

Engine::~Engine() {
  if (stream || dst) cudaStreamSynchronize(stream);
  if (graph_exec) cudaGraphExecDestroy(graph_exec);
  if (graph) cudaGraphDestroy(graph);
  if (once_exec) cudaGraphExecDestroy(once_exec);
  if (once_graph) cudaGraphDestroy(once_graph);
  for (auto& kv : std::vector<std::pair<void*, size_t>>(allocs.begin(), allocs.end())) dev_free(kv.first);
  if (stream) cudaStreamSynchronize(stream);
  if (pool) cudaMemPoolDestroy(pool);
  if (hs_pinned) cudaFreeHost(hs_pinned);
}

// ---- relations --------------------------------------------------------------------------

hisa_status Engine::declare(const char* name, uint32_t arity, int is_idb, uint32_t* id) {
  if (!name || !id || std::strlen(name) > 63) return ctx_fail(HISA_ERR_INVALID_ARG, "relation name", nullptr);
  if (arity != 2) return ctx_fail(HISA_ERR_ARITY, "only binary relations are evaluated", nullptr);
  for (auto& r : rels)
    if (r.name == name) return ctx_fail(HISA_ERR_INVALID_ARG, "duplicate relation", name);
  if (rels.size() >= 8) return ctx_fail(HISA_ERR_UNSUPPORTED, "at most 8 relations", nullptr);
  Relation r;
  r.name = name;
  r.arity = arity;
  r.idb = is_idb != 0;
  rels.push_back(r);
  *id = uint32_t(rels.size() - 1);
  compiled = false;
  return HISA_OK;
}

hisa_status Engine::load(uint32_t rid, const uint32_t* const* cols, uint64_t n, int on_device) {
  if (rid >= rels.size() || !cols) return ctx_fail(HISA_ERR_INVALID_ARG, "load: relation", nullptr);
  Relation& r = rels[rid];
  if (r.idb) return ctx_fail(HISA_ERR_STATE, "load into an IDB relation", r.name.c_str());
  if (n == 0) return HISA_OK;
  if (!cols[0] || !cols[1]) return ctx_fail(HISA_ERR_INVALID_ARG, "load: null column", nullptr);
  // staging: raw columns appended into one device buffer per column
  const uint64_t need = r.staged + n;
  if (need > r.stage_cap) {
    const uint64_t cap = std::max<uint64_t>(need, r.stage_cap * 2);
    void *a, *b, *c;
    hisa_status s;
    if ((s = dev_alloc(cap * 4, &a)) || (s = dev_alloc(cap * 4, &b)) || (s = dev_alloc(cap * 4, &c))) return s;
    if (r.staged) {
      CU(cudaMemcpyAsync(a, r.stage[0], r.staged * 4, cudaMemcpyDeviceToDevice, stream));
      CU(cudaMemcpyAsync(b, r.stage[1], r.staged * 4, cudaMemcpyDeviceToDevice, stream));
      CU(cudaMemcpyAsync(c, r.stage_inst, r.staged * 4, cudaMemcpyDeviceToDevice, stream));
    }
    dev_free(r.stage[0]);
    dev_free(r.stage[1]);
    dev_free(r.stage_inst);
    r.stage[0] = static_cast<uint32_t*>(a);
    r.stage[1] = static_cast<uint32_t*>(b);
    r.stage_inst = static_cast<uint32_t*>(c);
    r.stage_cap = cap;
  }
  launch_fill_u32(r.stage_inst + r.staged, n, load_inst, grid, stream);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  for (int c = 0; c < 2; ++c)
    CU(cudaMemcpyAsync(r.stage[c] + r.staged, cols[c], n * 4, kind, stream));
  // active-domain bound for the code width (fixed up front in a serving session)
  uint32_t mx = 0;
  if (serving) {
  } else if (!on_device) {
    for (int c = 0; c < 2; ++c)
      for (uint64_t i = 0; i < n; ++i) mx = std::max(mx, cols[c][i]);
  } else {
    hisa_status s = device_max(r.stage[0] + r.staged, r.stage[1] + r.staged, n, &mx);
    if (s) return s;
  }
  r.max_value = std::max(r.max_value, mx);
  r.staged += n;
  edb_dirty = true;
  return HISA_OK;
}

hisa_status Engine::reset_edb() {
  for (auto& r : rels) {
    if (r.idb) continue;
    r.staged = 0;
    r.max_value = 0;
  }
  edb_dirty = true;
  compiled = false;
  return HISA_OK;
}

hisa_status Engine::add_rule(const hisa_rule* rule) {
  if (!rule) return ctx_fail(HISA_ERR_INVALID_ARG, "null rule", nullptr);
  const hisa_rule& R = *rule;
  if (R.n_body < 1 || R.n_body > 3 || R.n_neq > 2) return ctx_fail(HISA_ERR_INVALID_ARG, "rule shape", nullptr);
  auto ok_atom = [&](const hisa_atom& a) { return a.rel < rels.size() && a.var[0] < 16 && a.var[1] < 16; };
  if (!ok_atom(R.head) || !rels[R.head.rel].idb) return ctx_fail(HISA_ERR_INVALID_ARG, "rule head", nullptr);
  for (uint32_t i = 0; i < R.n_body; ++i)
    if (!ok_atom(R.body[i])) return ctx_fail(HISA_ERR_INVALID_ARG, "rule body atom", nullptr);
  auto bound = [&](uint32_t v) {
    for (uint32_t i = 0; i < R.n_body; ++i)
      if (R.body[i].var[0] == v || R.body[i].var[1] == v) return true;
    return false;
  };
  for (int c = 0; c < 2; ++c)
    if (!bound(R.head.var[c])) return ctx_fail(HISA_ERR_INVALID_ARG, "unbound head variable", nullptr);
  for (uint32_t f = 0; f < R.n_neq; ++f)
    if (!bound(R.neq[f][0]) || !bound(R.neq[f][1]))
      return ctx_fail(HISA_ERR_INVALID_ARG, "unbound filter variable", nullptr);
  rules.push_back(R);
  compiled = false;
  return HISA_OK;
}

// ---- rule compilation -------------------------------------------------------------------

// Plans one semi-naive variant of a rule: the body atom `delta_atom` (or the
// first atom of a non-recursive rule) is the scanned outer relation; every
// further atom is joined as a range-probed inner relation (Algorithm 3); with
// three atoms the first join writes the temporarily materialized Tmp relation
// (Section 5.2), keeping only the columns later steps need.
hisa_status Engine::plan_variant(const hisa_rule& R, int delta_atom, std::vector<StepPlan>& out) {
  const int nb = int(R.n_body);
  std::vector<int> rest;
  const int first = delta_atom >= 0 ? delta_atom : 0;
  for (int j = 0; j < nb; ++j)
    if (j != first) rest.push_back(j);
  // current tuple: its two columns and the variables they carry
  // the code's high half holds the relation's first stored column
  const Relation& r0 = rels[R.body[first].rel];
  int cur_var[2] = {int(R.body[first].var[r0.order]), int(R.body[first].var[1 - r0.order])};
  int cur_slot, cur_cnt;
  if (delta_atom >= 0) {
    cur_slot = r0.delta;
    cur_cnt = r0.delta;
  } else {
    cur_slot = r0.idb ? r0.full : r0.base;
    cur_cnt = cur_slot;
  }
  std::vector<bool> applied(R.n_neq, false);
  bool first_step = true;
  while (true) {
    StepPlan sp{};
    sp.outer_slot = cur_slot;
    sp.outer_cnt = cur_cnt;
    int src_of[16];
    for (int& v : src_of) v = -1;
    src_of[cur_var[0]] = kSrcOuter0;
    if (src_of[cur_var[1]] < 0) src_of[cur_var[1]] = kSrcOuter1;
    auto add_filter = [&](int op, int a, int b) -> bool {
      if (sp.nfilt >= 2) return false;
      sp.fop[sp.nfilt] = op;
      sp.fa[sp.nfilt] = a;
      sp.fb[sp.nfilt] = b;
      ++sp.nfilt;
      return true;
    };
    // a repeated variable in the current tuple (e.g. Tgt(t,t)) is an equality filter
    if (first_step && cur_var[0] == cur_var[1] && !add_filter(kFiltEq, kSrcOuter0, kSrcOuter1))
      return ctx_fail(HISA_ERR_UNSUPPORTED, "too many filters in one join step", nullptr);
    if (!rest.empty()) {
      // next atom: the first remaining one sharing a variable with the current tuple
      int pick = -1, jv = -1;
      for (size_t q = 0; q < rest.size() && pick < 0; ++q) {
        const hisa_atom& A = R.body[rest[q]];
        for (int c = 0; c < 2; ++c)
          if (src_of[A.var[c]] >= 0) {
            pick = int(q);
            jv = int(A.var[c]);
            break;
          }
      }
      if (pick < 0) return ctx_fail(HISA_ERR_UNSUPPORTED, "rule needs a cross product", nullptr);
      const hisa_atom& A = R.body[rest[pick]];
      rest.erase(rest.begin() + pick);
      const int c = int(A.var[0]) == jv ? 0 : 1;
      const int ov = int(A.var[1 - c]);
      if (ov != jv && src_of[ov] >= 0)
        return ctx_fail(HISA_ERR_UNSUPPORTED, "join on two columns", nullptr);
      // an IDB inner relation is read from full (its first stored column) or
      // from its reverse-order mirror, indexed again every iteration
      Relation& ir = rels[A.rel];
      const int scol = ir.order == 0 ? c : 1 - c;
      ir.need_idx[scol] = true;
      sp.has_inner = true;
      sp.inner_rel = int(A.rel);
      sp.inner_col = scol;
      sp.outer_kcol = src_of[jv] == kSrcOuter0 ? 0 : 1;
      src_of[jv] = src_of[jv];  // the key equals the outer value
      if (ov == jv) {
        if (!add_filter(kFiltEq, kSrcKey, kSrcOther)) return ctx_fail(HISA_ERR_UNSUPPORTED, "filters", nullptr);
      } else {
        src_of[ov] = kSrcOther;
      }
    } else {
      sp.has_inner = false;
      sp.outer_kcol = 0;
    }
    // filters whose variables are all available now
    int other_filters = 0;
    for (uint32_t f = 0; f < R.n_neq; ++f) {
      if (applied[f]) continue;
      const int a = src_of[R.neq[f][0]], b = src_of[R.neq[f][1]];
      if (a < 0 || b < 0) continue;
      if (a == kSrcOther || b == kSrcOther) ++other_filters;
      if (other_filters > 1 || !add_filter(kFiltNeq, a, b))
        return ctx_fail(HISA_ERR_UNSUPPORTED, "too many filters in one join step", nullptr);
      applied[f] = true;
    }
    if (rest.empty()) {
      const int ho = rels[R.head.rel].order;
      sp.proj0 = src_of[R.head.var[ho]];
      sp.proj1 = src_of[R.head.var[1 - ho]];
      sp.out_rel = int(R.head.rel);
      sp.to_tmp = false;
      out.push_back(sp);
      return HISA_OK;
    }
    // Tmp: the variables still needed (remaining atoms, head, pending filters)
    std::vector<int> need;
    auto want = [&](int v) {
      if (src_of[v] >= 0 && std::find(need.begin(), need.end(), v) == need.end()) need.push_back(v);
    };
    for (int j : rest) {
      want(int(R.body[j].var[0]));
      want(int(R.body[j].var[1]));
    }
    want(int(R.head.var[0]));
    want(int(R.head.var[1]));
    for (uint32_t f = 0; f < R.n_neq; ++f)
      if (!applied[f]) {
        want(int(R.neq[f][0]));
        want(int(R.neq[f][1]));
      }
    if (need.size() > 2) return ctx_fail(HISA_ERR_UNSUPPORTED, "Tmp relation needs more than two columns", nullptr);
    if (need.size() == 1) need.push_back(need[0]);
    // the head's first stored variable first: the final join then keeps the
    // high half of Tmp (what the grouped bitmap join needs), and any join
    // reads either half
    if (need[1] == int(R.head.var[rels[R.head.rel].order])) std::swap(need[0], need[1]);
    sp.proj0 = src_of[need[0]];
    sp.proj1 = src_of[need[1]];
    sp.to_tmp = true;
    sp.out_rel = -1;
    out.push_back(sp);
    cur_var[0] = need[0];
    cur_var[1] = need[1];
    cur_slot = sc.tmp_a;
    cur_cnt = sc.tmp_cnt;
    first_step = false;
  }
}

hisa_status Engine::compile() {
  // code width from the active domain (Datalog without constants or arithmetic
  // derives values only from EDB values)
  uint32_t mx = 0;
  for (auto& r : rels) mx = std::max(mx, r.max_value);
  b = 1;
  while (b < 32 && (uint64_t(mx) >> b) != 0) ++b;
  inst_bits = 0;
  if (batched) {
    inst_bits = 1;
    while (inst_bits < 32 && (uint64_t(max_inst) >> inst_bits) != 0) ++inst_bits;
  }
  if (serving) {   // a serving session fixes the widths up front
    b = fixed_b;
    inst_bits = fixed_inst_bits;
  }
  if (inst_bits + b > 32)
    return ctx_fail(HISA_ERR_UNSUPPORTED, "instance bits + domain bits exceed the 32-bit join key", nullptr);
  wide = 2 * b + inst_bits > 32;
  direct_bits = (b + inst_bits <= kDirectMaxBits && !(cfg.flags & HISA_FLAG_HASH_INDEX)) ? b + inst_bits : 0;
  passes = (2 * b + inst_bits + 7) / 8;
  const int kb = wide ? 8 : 4;
  if (inst_row < 0) {
    inst_row = new_slot(8);
    inst_bnd = new_slot(8);
  }
  // slots of every relation (kept across runs; element width may change)
  for (auto& r : rels) {
    r.need_idx[0] = r.need_idx[1] = false;
    if (r.base < 0) {
      r.base = new_slot(kb);
      r.rev = new_slot(kb);
      r.table[0] = new_slot(16);
      r.table[1] = new_slot(16);
      slot_pow2[r.table[0]] = slot_pow2[r.table[1]] = true;
      if (r.idb) {
        r.full = r.base;
        r.full_next = new_slot(kb);
        r.delta = new_slot(kb);
        r.delta_next = new_slot(kb);
        r.fresh = new_slot(kb);
        r.fresh_alt = new_slot(kb);
        r.hist = new_slot(8);
        r.history = new_slot(8);
        r.rev_next = new_slot(kb);
        r.rswap = new_slot(kb);
        r.rswap_alt = new_slot(kb);
        r.runs_cnt[0] = nslots++;
        r.runs_cnt[1] = nslots++;
        r.l1 = new_slot(kb);
        r.l1_next = new_slot(kb);
        r.newp = new_slot(kb);
        r.gate = nslots++;
        r.bigf = nslots++;
        r.smallf = nslots++;
        r.lvidx = new_slot(8);
        r.nlv = nslots++;
        r.sortf = nslots++;
      }
    }
    for (int id : {r.base, r.rev, r.full_next, r.delta, r.delta_next, r.fresh, r.fresh_alt, r.rev_next, r.rswap,
                   r.rswap_alt, r.l1, r.l1_next, r.newp})
      if (id >= 0 && slot_elem[id] != kb) {
        dev_free(hs.buf[id].ptr);
        hs.buf[id] = {nullptr, 0};
        slot_elem[id] = kb;
      }
  }
  if (slot_elem[sc.tmp_a] != kb || slot_elem[sc.gather] != kb) {
    for (int id : {sc.tmp_a, sc.tmp_b, sc.gather}) {
      dev_free(hs.buf[id].ptr);
      hs.buf[id] = {nullptr, 0};
      slot_elem[id] = kb;
    }
  }
  idb.clear();
  for (size_t i = 0; i < rels.size(); ++i)
    if (rels[i].idb) idb.push_back(int(i));
  if (idb.empty()) return ctx_fail(HISA_ERR_INVALID_ARG, "no IDB relation", nullptr);
  hisa_status s;
  for (int r : idb) rels[r].order = 0;
  if ((s = plan_all())) return s;
  // grouped join with bitmap deduplication: an IDB relation R whose only
  // writer in iterations >= 2 is one binary join of delta_R with an EDB
  // relation is stored with the non-join column first, so delta's tuples
  // of one kept value are contiguous (dense.cuh)
  const bool dense_on = !(cfg.flags & HISA_FLAG_NO_DENSE) && b <= kDenseMaxBits;
  auto writers = [&](int r) {
    std::vector<const std::vector<StepPlan>*> w;
    for (auto& v : planN)
      if (!v.empty() && !v.back().to_tmp && v.back().out_rel == r) w.push_back(&v);
    return w;
  };
  // the last step of a one- or two-step variant: delta (or Tmp, sorted by
  // its kept column first) joined with an EDB relation on its low half,
  // keeping the high half and the inner's other column, with at most the
  // filter kept != other
  auto dense_ok = [&](const std::vector<StepPlan>& v, int r) {
    if (v.empty() || v.size() > 2) return false;
    const StepPlan& sp = v.back();
    const bool outer_ok = v.size() == 1 ? sp.outer_slot == rels[r].delta : sp.outer_slot == sc.tmp_a;
    const bool filt_ok = sp.nfilt == 0 ||
                         (sp.nfilt == 1 && sp.fop[0] == kFiltNeq &&
                          ((sp.fa[0] == kSrcOuter0 && sp.fb[0] == kSrcOther) ||
                           (sp.fa[0] == kSrcOther && sp.fb[0] == kSrcOuter0)));
    // and nothing probes r (its full becomes append-only levels, not one
    // sorted array an index could be built over)
    return outer_ok && filt_ok && sp.out_rel == r && sp.has_inner && !rels[sp.inner_rel].idb &&
           sp.outer_kcol == 1 && sp.proj0 == kSrcOuter0 && sp.proj1 == kSrcOther && !rels[r].need_idx[0] &&
           !rels[r].need_idx[1];
  };
  bool reorder = false;
  if (dense_on)
    for (int r : idb) {
      auto w = writers(r);
      if (w.size() != 1 || w[0]->size() != 1) continue;
      const StepPlan& sp = (*w[0])[0];
      if (sp.outer_slot != rels[r].delta || !sp.has_inner || rels[sp.inner_rel].idb || sp.nfilt ||
          rels[r].need_idx[0] || rels[r].need_idx[1])
        continue;
      if (sp.outer_kcol == 0) {   // join column first in (c0, c1): store (c1, c0)
        rels[r].order = 1;
        reorder = true;
      }
    }
  if (reorder && (s = plan_all())) return s;
  for (int r : idb) {
    auto w = writers(r);
    const bool ok = dense_on && w.size() == 1 && dense_ok(*w[0], r);
    if (!ok && rels[r].order) {   // the reordered plan does not fit: back to (c0, c1)
      rels[r].order = 0;
      if ((s = plan_all())) return s;
    }
  }
  for (auto& v : planN)
    for (auto& sp : v) sp.dense = sp.resort = false;
  for (int r : idb) rels[r].dense_head = rels[r].append = false;
  if (dense_on)
    for (int r : idb) {
      auto w = writers(r);
      if (w.size() == 1 && dense_ok(*w[0], r)) {
        for (auto& v : planN)
          if (&v == w[0]) v.back().dense = true;
        rels[r].dense_head = true;
        rels[r].append = !batched;   // batched runs keep one sorted full (retirement cuts it by instance)
      }
    }
  // any other writer's last step of the right shape (the head keeps one
  // column of the outer and the inner's other column, at most the filter
  // kept != other) joins densely too, into new beside the other writers;
  // a delta outer stored join column first is exchanged and sorted by the
  // kept column first (Tmp already holds the head's first variable first)
  if (dense_on)
    for (auto& v : planN) {
      StepPlan& sp = v.back();
      if (sp.dense || sp.to_tmp || !sp.has_inner || rels[sp.out_rel].append) continue;
      const bool tmp = v.size() > 1;
      const int kept = sp.outer_kcol == 0 ? kSrcOuter1 : kSrcOuter0;
      if (tmp && sp.outer_kcol != 1) continue;
      if (sp.proj0 != kept || sp.proj1 != kSrcOther) continue;
      const bool filt_ok = sp.nfilt == 0 ||
                           (sp.nfilt == 1 && sp.fop[0] == kFiltNeq &&
                            ((sp.fa[0] == kept && sp.fb[0] == kSrcOther) ||
                             (sp.fa[0] == kSrcOther && sp.fb[0] == kept)));
      if (!filt_ok) continue;
      sp.dense = true;
      sp.resort = !tmp && sp.outer_kcol == 0;
    }
  // a two-step variant whose first step joins a delta on its first stored
  // column and keeps the inner's other column x first and delta's second
  // column, and whose second step is dense: Tmp is gathered grouped by x
  // (ChainArgs) instead of joined and sorted.  The inner must be stored x
  // first: an EDB relation builds that copy, an IDB one must keep it anyway.
  //
  // A one-step variant H(x, y) <- A(x, z), delta(z, y) (the head keeps the
  // inner's other column first and delta's second column) joins densely the
  // other way round: A sorted by x is the grouped outer and delta, directly
  // indexed by z, the probed side (StepPlan::invert); so does a second step
  // of that shape over a gathered Tmp.  Each iteration reads all of A, so
  // only over small domains (|A| <= 2^(2 * kInvertMaxBits)).
  auto invertible = [&](const StepPlan& sp) {
    if (sp.dense || sp.to_tmp || !sp.has_inner || sp.out_rel < 0 || rels[sp.out_rel].append) return false;
    if (sp.outer_kcol != 0 || sp.proj0 != kSrcOther || sp.proj1 != kSrcOuter1) return false;
    const bool filt_ok = sp.nfilt == 0 ||
                         (sp.nfilt == 1 && sp.fop[0] == kFiltNeq &&
                          ((sp.fa[0] == kSrcOther && sp.fb[0] == kSrcOuter1) ||
                           (sp.fa[0] == kSrcOuter1 && sp.fb[0] == kSrcOther)));
    const Relation& A = rels[sp.inner_rel];
    return filt_ok && !(A.idb && sp.inner_col == 0 && !A.need_idx[1]);   // x second: its (c1, c0) order kept
  };
  const bool gather_on = dense_on && !(cfg.flags & HISA_FLAG_NO_CHAIN) && inst_bits == 0 && b <= kDirectMaxBits;
  const bool invert_on = gather_on && b <= kInvertMaxBits;
  for (auto& v : planN)
    for (auto& sp : v) sp.chain = sp.invert = false;
  if (gather_on)
    for (auto& v : planN) {
      if (v.size() != 2 || v[1].outer_slot != sc.tmp_a) continue;
      const bool inv2 = !v[1].dense && invert_on && invertible(v[1]);
      if (!v[1].dense && !inv2) continue;
      StepPlan& s1 = v[0];
      bool delta_outer = false;
      for (int r : idb) delta_outer = delta_outer || s1.outer_slot == rels[r].delta;
      if (!delta_outer || !s1.has_inner || s1.nfilt || s1.outer_kcol != 0 || s1.proj0 != kSrcOther ||
          s1.proj1 != kSrcOuter1)
        continue;
      Relation& A = rels[s1.inner_rel];
      const int xcol = 1 - s1.inner_col;
      if (A.idb && !A.need_idx[xcol]) continue;
      s1.chain = true;
      A.need_idx[xcol] = true;
      if (inv2) {
        v[1].invert = v[1].dense = true;
        Relation& A2 = rels[v[1].inner_rel];
        if (!A2.idb && v[1].inner_col == 0) A2.need_idx[1] = true;   // an EDB relation builds its (c1, c0) copy
      }
    }
  if (invert_on)
    for (auto& v : planN) {
      if (v.size() != 1) continue;
      StepPlan& sp = v[0];
      bool delta_outer = false;
      for (int r : idb) delta_outer = delta_outer || sp.outer_slot == rels[r].delta;
      if (!delta_outer || !invertible(sp)) continue;
      sp.invert = sp.dense = true;
      Relation& A = rels[sp.inner_rel];
      if (!A.idb && sp.inner_col == 0) A.need_idx[1] = true;   // an EDB relation builds its (c1, c0) copy
    }
  // full as a bit matrix (dense.cuh) for the one IDB relation of a program
  // whose writer is the grouped bitmap join: the join is then the last step
  // of every iteration's join stage, so the matrix takes its delta after it
  // without any later overflow of that stage re-running the iteration
  for (int r : idb) {
    Relation& R = rels[r];
    R.mfull = R.append && idb.size() == 1 && b >= 8 && b <= kMatrixMaxBits && !(cfg.flags & HISA_FLAG_LEVELS);
    // batched and served runs (matrix.cuh): row (instance, g), when the matrix
    // of all instance slots fits; the dense join then writes new like any
    // other writer and the tail takes delta = unique(new) \ full by bit tests
    if (batched && R.dense_head && idb.size() == 1 && b <= kMatrixMaxBits && !(cfg.flags & HISA_FLAG_LEVELS) &&
        inst_bits + 2 * b <= 40 && (1ull << (inst_bits + 2 * b)) / 8 <= kBatchMatrixMaxBytes)
      R.mfull = true;
    if (R.mfull && R.fbm < 0) R.fbm = new_slot(4);
    if (R.mfull && R.fcnt < 0) R.fcnt = new_slot(4);
  }
  // pull mode (dense.cuh) for a relation written only by a one-step grouped
  // bitmap join of its delta with an EDB relation (REACH's recursive rule):
  // the inner relation is also sorted and directly indexed by its other column
  const bool pull_on = dense_on && !(cfg.flags & HISA_FLAG_NO_PULL) && !batched && inst_bits == 0 &&
                       direct_bits > 0 && b <= kPullMaxBits;
  for (int r : idb) {
    Relation& R = rels[r];
    R.pull = false;
    if (!pull_on || !R.append) continue;
    auto w = writers(r);
    if (w.size() != 1 || w[0]->size() != 1) continue;
    const StepPlan& sp = (*w[0])[0];
    if (!sp.dense || sp.invert || sp.chain || sp.outer_slot != R.delta || !sp.has_inner || rels[sp.inner_rel].idb)
      continue;
    Relation& I = rels[sp.inner_rel];
    const int ocol = 1 - sp.inner_col;
    I.need_idx[ocol] = true;
    R.pull = true;
    R.pull_inner = ocol == 0 ? I.base : I.rev;
    R.pull_index = I.table[ocol];
    R.push_index = I.table[sp.inner_col];
    if (R.pull_out < 0) {
      R.pull_out = new_slot(4);
      R.pull_bm = new_slot(4);
      if (R.fcnt < 0) R.fcnt = new_slot(4);
      R.pull_first = new_slot(4);
      R.tdeg = new_slot(4);
      R.nout = nslots++;
    }
  }
  // log-structured full where nothing probes full (it is only differenced
  // and merged): REACH and SG, not CSPA's inner IDB atoms nor batched runs
  for (int r : idb) {
    Relation& R = rels[r];
    R.log = (cfg.flags & HISA_FLAG_LOG_FULL) && !R.need_idx[0] && !R.need_idx[1] && !R.append && !R.mfull;
  }
  bitjoin = detect_bitjoin();
  if (bitjoin) {   // full is kept as a bit matrix in the declared column order
    Relation& R = rels[bj_rel];
    R.order = 0;
    R.mfull = true;
    if (R.fbm < 0) R.fbm = new_slot(4);
    if (bj_first < 0) {
      bj_first = new_slot(8);
      bj_d = new_slot(4);
      bj_d2 = new_slot(4);
      bj_dm = new_slot(4);
      bj_dm2 = new_slot(4);
      bj_tot = new_slot(8);
      bj_ctr = new_slot(4);
      bj_items = new_slot(8);
      bj_hslot = new_slot(4);
      bj_hacc = new_slot(4);
      bj_hdone = new_slot(4);
      bj_todo = new_slot(4);
      bj_items2 = new_slot(8);
      bj_offs2 = new_slot(8);
    }
  }
  compiled = true;
  graph_stale = true;
  once_stale = true;
  return HISA_OK;
}

// A program of REACH's shape (bitjoin.cuh): one binary IDB relation R, rules
// R(x, y) <- E(x, y) with E an EDB relation, and exactly one recursive rule
// R(x, z) <- B(x, y), R(y, z) with B an EDB relation (either body order), no
// filters; a domain of at most 2^16 values; no batching and no flag that asks
// for another path.
bool Engine::detect_bitjoin() {
  bj_base.clear();
  bj_rel = bj_inner = -1;
  if (batched || serving || idb.size() != 1 || b > kBitMaxBits) return false;
  if (cfg.flags & (HISA_FLAG_NO_BITJOIN | HISA_FLAG_NO_DENSE | HISA_FLAG_NO_PULL | HISA_FLAG_LEVELS)) return false;
  const uint32_t r = uint32_t(idb[0]);
  int recursive = 0;
  for (const hisa_rule& q : rules) {
    if (q.head.rel != r || q.n_neq != 0) return false;
    if (q.n_body == 1) {
      const hisa_atom& e = q.body[0];
      if (e.rel == r || rels[e.rel].idb) return false;
      if (q.head.var[0] == q.head.var[1] || e.var[0] != q.head.var[0] || e.var[1] != q.head.var[1]) return false;
      bj_base.push_back(int(e.rel));
    } else if (q.n_body == 2) {
      const int ri = q.body[0].rel == r ? 0 : 1;
      const hisa_atom& ra = q.body[ri];
      const hisa_atom& ba = q.body[1 - ri];
      if (ra.rel != r || ba.rel == r || rels[ba.rel].idb) return false;
      const uint32_t x = ba.var[0], y = ba.var[1], z = ra.var[1];
      if (x == y || y == z || x == z || ra.var[0] != y || q.head.var[0] != x || q.head.var[1] != z) return false;
      bj_inner = int(ba.rel);
      ++recursive;
    } else {
      return false;
    }
  }
  if (recursive != 1 || bj_base.empty()) return false;
  bj_rel = int(r);
  return true;
}

// The fixpoint of a program of REACH's shape on bit matrices (bitjoin.cuh):
// iteration 1 sets delta = full = the union of the E relations; every later
// iteration ORs, per tuple (x, y) of B, delta's row y into row x, keeps the
// bits not in full as delta' and ORs them into full, until delta' is empty.
hisa_status Engine::run_bitjoin(hisa_run_stats* stats, std::chrono::steady_clock::time_point t0) {
  hisa_status s;
  Relation& R = rels[bj_rel];
  const Relation& B = rels[bj_inner];
  const uint64_t rows = 1ull << b, nw = bit_nwords(b), mw = bit_mwords(b);
  const bool timing = cfg.flags & HISA_FLAG_PHASE_TIMES;
  std::memset(kstat, 0, sizeof kstat);
  timer.reset();
  struct TimerGuard {
    explicit TimerGuard(KernelTimer* t) { g_timer = t; }
    ~TimerGuard() { g_timer = nullptr; }
  } tg(timing ? &timer : nullptr);
  const uint64_t launches0 = g_launches;
  if ((s = ensure(R.fbm, rows * nw)) || (s = ensure(bj_d, rows * nw)) || (s = ensure(bj_d2, rows * nw)) ||
      (s = ensure(bj_dm, rows * mw)) || (s = ensure(bj_dm2, rows * mw)) || (s = ensure(bj_first, rows + 1)) ||
      (s = ensure(bj_tot, 2)) || (s = ensure(bj_ctr, 1)))
    return s;
  CU(cudaMemsetAsync(hs.buf[R.fbm].ptr, 0, rows * nw * 4, stream));
  CU(cudaMemsetAsync(hs.buf[bj_d].ptr, 0, rows * nw * 4, stream));
  CU(cudaMemsetAsync(hs.buf[bj_dm].ptr, 0, rows * mw * 4, stream));
  if ((s = upload())) return s;
  // B's run of each first column: a direct index over its sorted codes
  if ((s = ensure(bj_todo, (rows + 31) / 32))) return s;
  if ((s = upload())) return s;
  {
    std::vector<Op> ops(1);
    ops[0].kind = Op::INDEX;
    ops[0].index = IndexArgs{dst, B.base, B.base, bj_first, b, -1, 0, b};
    if ((s = exec(ops))) return s;
  }
  // work items (row, segment of at most kBitSeg B tuples, chunk group), built
  // on the device; a row of several segments gets an accumulator (at most
  // min(rows, |B| / (kBitSeg + 1) + 1) of them)
  const uint64_t nb = hs.cnt[B.base];
  const uint64_t nh = std::min<uint64_t>(rows, nb / (kBitSeg + 1) + 1);
  const uint64_t max_items = (nb / kBitSeg + rows) * bit_groups(b) + 1;
  if ((s = ensure(bj_items, max_items)) || (s = ensure(bj_hslot, rows + 1)) || (s = ensure(bj_hacc, nh * nw)) ||
      (s = ensure(bj_hdone, nh * kBitGroups)) || (s = ensure(sc.mrows, rows + 1)))
    return s;
  CU(cudaMemsetAsync(hs.buf[bj_hacc].ptr, 0, nh * nw * 4, stream));
  CU(cudaMemsetAsync(hs.buf[bj_hdone].ptr, 0, nh * kBitGroups * 4, stream));
  uint32_t* nheavy = static_cast<uint32_t*>(hs.buf[bj_hslot].ptr) + rows;
  CU(cudaMemsetAsync(nheavy, 0, 4, stream));
  uint64_t* item_offs = static_cast<uint64_t*>(hs.buf[sc.mrows].ptr);
  BitItemsArgs ita{static_cast<const uint64_t*>(hs.buf[bj_first].ptr), item_offs,
                   static_cast<uint64_t*>(hs.buf[bj_items].ptr), static_cast<uint32_t*>(hs.buf[bj_hslot].ptr),
                   nheavy, b, nullptr};
  launch_bit_items(ita, grid, stream);   // every row with B tuples, and the accumulator slots
  if ((s = check_launch("bit items"))) return s;
  // a sparse delta (below 256 bits per row on average): only the rows with a
  // B tuple selecting a non-empty delta row are worked, from items made for
  // the iteration; a dense one takes every row's items
  if ((s = ensure(bj_items2, max_items)) || (s = ensure(bj_offs2, rows + 1))) return s;
  uint32_t* todo = static_cast<uint32_t*>(hs.buf[bj_todo].ptr);
  BitItemsArgs itb = ita;
  itb.offs = static_cast<uint64_t*>(hs.buf[bj_offs2].ptr);
  itb.items = static_cast<uint64_t*>(hs.buf[bj_items2].ptr);
  itb.todo = todo;
  const uint64_t sparse_below = rows * 256;
  auto* tot = static_cast<unsigned long long*>(hs.buf[bj_tot].ptr);
  uint32_t* D = static_cast<uint32_t*>(hs.buf[bj_d].ptr);
  uint32_t* D2 = static_cast<uint32_t*>(hs.buf[bj_d2].ptr);
  uint32_t* Dm = static_cast<uint32_t*>(hs.buf[bj_dm].ptr);
  uint32_t* Dm2 = static_cast<uint32_t*>(hs.buf[bj_dm2].ptr);
  uint32_t* F = static_cast<uint32_t*>(hs.buf[R.fbm].ptr);
  // iteration 1: the non-recursive rules (|delta_1| counts the bits they set)
  CU(cudaMemsetAsync(tot, 0, 16, stream));
  for (int e : bj_base) {
    const Relation& E = rels[e];
    if (!hs.cnt[E.base]) continue;
    BitInitArgs ia{hs.buf[E.base].ptr, hs.cnt[E.base], b, D, Dm, F, tot};
    if (wide) launch_bit_init<uint64_t>(ia, grid, stream);
    else launch_bit_init<uint32_t>(ia, grid, stream);
    if ((s = check_launch("bit init"))) return s;
  }
  unsigned long long h[2] = {0, 0};
  CU(cudaMemcpyAsync(h, tot, 16, cudaMemcpyDeviceToHost, stream));
  CU(cudaStreamSynchronize(stream));
  std::vector<uint64_t> hist;
  if (h[0]) hist.push_back(h[0]);
  const double kb = wide ? 8.0 : 4.0;
  kstat[kKBitInit].bytes += double(hs.cnt[B.base]) * kb + double(rows * nw) * 4.0;
  uint32_t iters_run = 1;
  uint64_t d = h[0];
  while (d > 0 && iters_run < cfg.max_iters) {
    const bool sparse = d < sparse_below;
    if (sparse) {   // this iteration's rows: those with a B tuple selecting a non-empty delta row
      CU(cudaMemsetAsync(todo, 0, (rows + 31) / 32 * 4, stream));
      if (wide) launch_bit_todo<uint64_t>(BitTodoArgs{Dm, hs.buf[B.base].ptr, nb, todo, b}, grid, stream);
      else launch_bit_todo<uint32_t>(BitTodoArgs{Dm, hs.buf[B.base].ptr, nb, todo, b}, grid, stream);
      launch_bit_items(itb, grid, stream);
      if ((s = check_launch("bit items"))) return s;
    }
    const BitItemsArgs& it = sparse ? itb : ita;
    CU(cudaMemsetAsync(tot, 0, 16, stream));
    CU(cudaMemsetAsync(hs.buf[bj_ctr].ptr, 0, 4, stream));
    CU(cudaMemsetAsync(Dm2, 0, rows * mw * 4, stream));
    BitJoinArgs ja{static_cast<const uint64_t*>(hs.buf[bj_first].ptr),
                   hs.buf[B.base].ptr,
                   it.items,
                   it.offs + rows,
                   static_cast<const uint32_t*>(hs.buf[bj_hslot].ptr),
                   static_cast<uint32_t*>(hs.buf[bj_hacc].ptr),
                   static_cast<uint32_t*>(hs.buf[bj_hdone].ptr),
                   D, Dm, D2, Dm2, F, tot, tot + 1, static_cast<uint32_t*>(hs.buf[bj_ctr].ptr), b};
    if (wide) launch_bitjoin<uint64_t>(ja, grid, stream);
    else launch_bitjoin<uint32_t>(ja, grid, stream);
    if ((s = check_launch("bit join"))) return s;
    CU(cudaMemcpyAsync(h, tot, 16, cudaMemcpyDeviceToHost, stream));
    CU(cudaStreamSynchronize(stream));
    ++iters_run;
    d = h[0];
    // bytes: B read, the delta chunks selected, full's row read and delta'
    // written where new bits arrived (at most), the masks
    kstat[kKBitJoin].bytes += double(hs.cnt[B.base]) * kb + double(h[1]) * 128.0 + double(d) * 1.0 +
                              double(rows * mw) * 8.0 + double(rows + 1) * 8.0;
    if (d) hist.push_back(d);
    std::swap(D, D2);
    std::swap(Dm, Dm2);
  }
  if (d > 0) return ctx_fail(HISA_ERR_NOT_CONVERGED, "max_iters reached", nullptr);
  uint64_t total = 0;
  for (uint64_t x : hist) total += x;
  hs.cnt[R.full] = total;
  R.delta_counts = hist;
  if ((s = upload())) return s;
  if (timing) {
    CU(cudaStreamSynchronize(stream));
    for (auto& rc : timer.recs) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, rc.a, rc.b);
      kstat[rc.kind].ms += ms;
      kstat[rc.kind].launches += 1;
    }
    timer.reset();
  }
  last_stats.kernel_launches = g_launches - launches0;
  last_stats.tuples_joined = total;
  last_stats.iterations = uint32_t(hist.size());
  last_stats.iterations_run = iters_run;
  last_stats.regrows = 0;
  last_stats.graph_launches = 0;
  last_stats.peak_bytes = peak_bytes;
  last_stats.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = last_stats;
  ran = true;
  return HISA_OK;
}

// Semi-naive variants (Section 2): iteration 1 runs the rules without IDB
// atoms; later iterations run each rule once per IDB atom, that atom read
// from delta and the others from full.
hisa_status Engine::plan_all() {
  plan1.clear();
  planN.clear();
  for (auto& r : rels) r.need_idx[0] = r.need_idx[1] = false;
  for (auto& R : rules) {
    std::vector<int> idb_atoms;
    for (uint32_t j = 0; j < R.n_body; ++j)
      if (rels[R.body[j].rel].idb) idb_atoms.push_back(int(j));
    hisa_status s;
    if (idb_atoms.empty()) {
      std::vector<StepPlan> v;
      if ((s = plan_variant(R, -1, v))) return s;
      plan1.push_back(v);
    } else {
      for (int j : idb_atoms) {
        std::vector<StepPlan> v;
        if ((s = plan_variant(R, j, v))) return s;
        planN.push_back(v);
      }
    }
  }
  return HISA_OK;
}

// ---- op emission ------------------------------------------------------------------------

void Engine::emit_join(std::vector<Op>& ops, const StepPlan& sp) {
  Op o{};
  o.kind = Op::JOIN;
  JoinArgs& a = o.join;
  a.st = dst;
  a.outer_buf = sp.outer_slot;
  a.outer_cnt = sp.outer_cnt;
  a.has_inner = sp.has_inner;
  if (sp.has_inner) {
    const Relation& ir = rels[sp.inner_rel];
    a.inner_buf = sp.inner_col == 0 ? ir.base : ir.rev;
    a.inner_cnt = a.inner_buf;
    a.table_buf = ir.table[sp.inner_col];
  }
  a.b = b;
  a.outer_kcol = sp.outer_kcol;
  a.proj0 = sp.proj0;
  a.proj1 = sp.proj1;
  a.nfilt = sp.nfilt;
  for (int f = 0; f < 2; ++f) {
    a.fop[f] = sp.fop[f];
    a.fa[f] = sp.fa[f];
    a.fb[f] = sp.fb[f];
  }
  a.offs_buf = sc.offs;
  a.status_buf = sc.join_status;
  a.starts_buf = sc.starts;
  if (sp.to_tmp) {
    a.out_buf = sc.tmp_a;
    a.out_cnt = sc.tmp_cnt;
    a.hist_buf = -1;
  } else {
    const Relation& hr = rels[sp.out_rel];
    a.out_buf = hr.fresh;
    a.out_cnt = hr.fresh;
    a.hist_buf = hr.hist;
    a.hist_passes = passes;
  }
  a.total_cnt = sc.total;
  a.ctr = 0;
  a.skip_mask = 1;
  a.stage_bit = 0;
  a.index_direct = direct_bits > 0;
  ops.push_back(o);
}

// Indexes of the IDB relations probed as inner relations, for the iteration
// about to run (Algorithm 2 over the current full; Section 4.2 orders the
// columns join column first).  Column 1 is served by the reverse-order mirror
// of full: the delta of the last iteration, columns exchanged and sorted,
// merged into it (delta and full are disjoint, so the merge drops nothing).
// Every step is idempotent, so an iteration re-run after a regrow repeats it
// safely.
void Engine::emit_idb_index(std::vector<Op>& ops) {
  auto ctl = [&](std::initializer_list<CtlCmd> cmds) {
    Op c{};
    c.kind = Op::CTL;
    c.ctl.st = dst;
    c.ctl.skip_mask = 1;
    for (const CtlCmd& x : cmds) c.ctl.cmd[c.ctl.n++] = x;
    ops.push_back(c);
  };
  const long long lf1024 = std::max(1LL, (long long)(cfg.load_factor * 1024.f));
  for (int r : idb) {
    const Relation& R = rels[r];
    if (R.need_idx[1]) {
      Op w{};
      w.kind = Op::SWAP;
      w.swap = SwapArgs{dst, R.delta, R.delta, R.rswap, R.rswap, b, 1, 0};
      ops.push_back(w);
      ctl({{kCtlZeroSmall, sc.hist, 8 * 256, 0}});
      Op h{};
      h.kind = Op::HIST;
      h.hist = RadixHistArgs{dst, R.rswap, R.rswap, sc.hist, passes, 1};
      ops.push_back(h);
      emit_sort(ops, R.rswap, R.rswap_alt, R.rswap, sc.hist, 1, 0);
      Op m{};
      m.kind = Op::SETOP;
      SetopArgs& a = m.setop;
      a.st = dst;
      a.a_buf = R.rev;
      a.a_cnt = R.rev;
      a.b_buf = (passes & 1) ? R.rswap_alt : R.rswap;
      a.b_cnt = R.rswap;
      a.split_buf = sc.split;
      a.status_buf = sc.setop_status;
      a.d_buf = -1;
      a.d_cnt = -1;
      a.f_buf = R.rev_next;
      a.f_cnt = R.rev_next;
      a.ctr = 2;
      a.skip_mask = 1;
      a.stage_bit = 0;
      ops.push_back(m);
      ctl({{kCtlSwapIfCnt, R.rev, R.rev_next, R.rswap}});
    }
    for (int col = 0; col < 2; ++col) {
      if (!R.need_idx[col]) continue;
      const int keys = col == 0 ? R.full : R.rev;
      if (direct_bits) {
        Op i{};
        i.kind = Op::INDEX;
        i.index = IndexArgs{dst, keys, keys, R.table[col], b, -1, 1, direct_bits};
        ops.push_back(i);
        continue;
      }
      ctl({{kCtlSetCnt, R.runs_cnt[col], 0, 0}});
      Op u{};
      u.kind = Op::RUNS;
      u.runs = RunsArgs{dst, keys, keys, b, R.runs_cnt[col], 1};
      ops.push_back(u);
      ctl({{kCtlCheckTable, R.table[col], R.runs_cnt[col], lf1024}});
      Op z{};
      z.kind = Op::ZERO;
      z.zero = ZeroArgs{dst, R.table[col], 16, 1};
      ops.push_back(z);
      Op i{};
      i.kind = Op::INDEX;
      i.index = IndexArgs{dst, keys, keys, R.table[col], b, -1, 1};
      ops.push_back(i);
    }
  }
}

// Tmp of a two-step variant gathered grouped by its kept column x: delta's
// direct index by its first stored column (the join value), the inner's
// direct index by x (into dense_first, read by the dense join's group
// compaction through chain_pre), then len + scan + gather (ChainArgs).
void Engine::emit_chain(std::vector<Op>& ops, const StepPlan& sp, bool tmp_index) {
  const int abuf = sorted_by_other(sp);   // stored x first
  Op x{};
  x.kind = Op::INDEX;
  x.index = IndexArgs{dst, sp.outer_slot, sp.outer_cnt, sc.chain_dfirst, b, -1, 1, b};
  ops.push_back(x);
  Op y{};
  y.kind = Op::INDEX;
  y.index = IndexArgs{dst, abuf, abuf, sc.dense_first, b, -1, 1, b};
  ops.push_back(y);
  Op c{};
  c.kind = Op::CHAIN;
  c.chain = ChainArgs{dst, abuf, abuf, sp.outer_slot, sp.outer_cnt, sc.chain_dfirst, sc.chain_pre, sc.tmp_a,
                      sc.tmp_cnt, b, 1, 0, sc.dense_first, tmp_index ? sc.chain_tfirst : -1};
  ops.push_back(c);
}

// The slot of a step's inner relation sorted by its other (non-join) column.
int Engine::sorted_by_other(const StepPlan& sp) const {
  const Relation& A = rels[sp.inner_rel];
  return sp.inner_col == 1 ? A.base : A.rev;
}

// An inverted dense join (StepPlan::invert): delta's direct index by its
// first stored column (the join value), then the grouped bitmap join with
// the inner sorted by its other column as the outer and delta as the inner.
void Engine::emit_invert(std::vector<Op>& ops, const StepPlan& sp, bool tmp_probe) {
  // a gathered Tmp comes with its direct index (emit_chain); a delta is indexed here
  if (!tmp_probe) {
    Op x{};
    x.kind = Op::INDEX;
    x.index = IndexArgs{dst, sp.outer_slot, sp.outer_cnt, sc.chain_dfirst, b, -1, 1, b};
    ops.push_back(x);
  }
  StepPlan d = sp;
  d.outer_slot = d.outer_cnt = sorted_by_other(sp);
  d.outer_kcol = 1;
  d.proj0 = kSrcOuter0;
  emit_dense(ops, d, false, sp.outer_slot, tmp_probe ? sc.chain_tfirst : sc.chain_dfirst);
}

void Engine::emit_dense(std::vector<Op>& ops, const StepPlan& sp, bool chain_groups, int inner_buf,
                        int table_buf) {
  const Relation& ir = rels[sp.inner_rel];
  const Relation& hr = rels[sp.out_rel];
  // group starts: a direct index of delta by the kept column, compacted to
  // the non-empty groups; one pass over delta when instance ids make the key
  // space too large for a direct index; for a gathered Tmp, its offsets at
  // the inner's direct index (emit_chain)
  if (chain_groups) {
    Op g{};
    g.kind = Op::GCOMPACT;
    g.groups = GroupArgs{dst, sc.dense_first, sp.outer_cnt, b, sc.groups, sc.group_cnt, sc.join_status, 3, 1, 0};
    g.groups.indirect = 1;
    g.groups.vals_buf = sc.chain_pre;
    ops.push_back(g);
  } else if (b + inst_bits <= kDirectMaxBits) {
    Op x{};
    x.kind = Op::INDEX;
    x.index = IndexArgs{dst, sp.outer_slot, sp.outer_cnt, sc.dense_first, b, -1, 1, b + inst_bits};
    ops.push_back(x);
    Op g{};
    g.kind = Op::GCOMPACT;
    g.groups = GroupArgs{dst, sc.dense_first, sp.outer_cnt, b + inst_bits, sc.groups, sc.group_cnt, sc.join_status, 3, 1, 0};
    ops.push_back(g);
  } else {
    Op g{};
    g.kind = Op::GROUPS;
    g.groups = GroupArgs{dst, sp.outer_slot, sp.outer_cnt, b, sc.groups, sc.group_cnt, sc.join_status, 3, 1, 0};
    ops.push_back(g);
  }
  // with an append-only full the join writes delta itself, into delta_next
  const int out = hr.append ? hr.delta_next : hr.fresh;
  // a unit holds enough outer tuples to outweigh its bitmap
  const int unit_size = cfg.dense_unit ? int(cfg.dense_unit)
                                       : int(std::max<uint64_t>(256, std::min<uint64_t>(32768, 16ull << (b >= 5 ? b - 5 : 0))));
  const bool units_ready = b + inst_bits <= kDirectMaxBits;
  const bool pull = hr.pull && !chain_groups && inner_buf < 0 && units_ready;
  if (units_ready) {
    GroupArgs& ga = ops.back().groups;
    ga.units_buf = sc.dense_units;
    ga.done_buf = sc.dense_done;
    ga.mslot_buf = sc.dense_mslot;
    ga.unit_size = unit_size;
    ga.bmm_buf = sc.dense_bmm;
    ga.bm_words = b >= 5 ? 1 << (b - 5) : 1;
    if (pull) {
      ga.pull_bm_buf = hr.pull_bm;
      ga.plist_buf = sc.dense_plist;
      ga.pull_cnt = sc.pull_cnt;
    }
  }
  Op d{};
  d.kind = Op::DENSE;
  d.dense = DenseArgs{dst, sp.outer_slot, sp.outer_cnt, sc.groups, sc.group_cnt,
                      inner_buf >= 0 ? inner_buf : sp.inner_col == 0 ? ir.base : ir.rev,
                      table_buf >= 0 ? table_buf : ir.table[sp.inner_col], b,
                      out, out, sc.total, sc.raw_cnt, sc.dense_bm, sc.dense_status, 4, 1, 0,
                      inner_buf >= 0 || direct_bits > 0, hr.append && !hr.mfull ? hr.full : -1, hr.lvidx, hr.nlv,
                      sp.nfilt > 0,
                      sc.dense_units, sc.dense_done, unit_size, sc.dense_mslot, sc.dense_bmm, units_ready};
  if (hr.mfull) {   // the emit ORs the groups' new tuples into full's bit matrix
    d.dense.fbm_buf = hr.fbm;
    d.dense.fcnt_buf = hr.fcnt;
    d.dense.row_bits = b + inst_bits;
    d.dense.fbm_or = batched ? 0 : 1;   // batched: the tail adds the committed delta
  }
  if (pull) {
    DenseArgs& da = d.dense;
    da.pull_inner_buf = hr.pull_inner;
    da.pull_index_buf = hr.pull_index;
    da.pull_out_buf = hr.pull_out;
    da.pull_bm_buf = hr.pull_bm;
    da.fcnt_buf = hr.fcnt;
    da.nout_cnt = hr.nout;
    da.pull_first_buf = hr.pull_first;
    da.tdeg_buf = hr.tdeg;
    da.plist_buf = sc.dense_plist;
    da.pull_cnt = sc.pull_cnt;
    da.pull_raw_cnt = sc.pull_raw_cnt;
    da.prev_bm_buf = sc.dense_bm_prev;
    da.prev_gi_buf = sc.prev_gi;
    da.pull_k16 = uint32_t(cfg.pull_ratio * 16.f + 0.5f);
  }
  ops.push_back(d);
  if (hr.append) {   // no unique pass in the tail; |new| (statistics) = |delta|
    Op f{};
    f.kind = Op::CTL;
    f.ctl.st = dst;
    f.ctl.skip_mask = 1;
    f.ctl.cmd[f.ctl.n++] = {kCtlSetCnt, hr.sortf, 0, 0};
    f.ctl.cmd[f.ctl.n++] = {kCtlCopyCnt, hr.fresh, hr.delta_next, 0};
    ops.push_back(f);
  }
}

// Join stage of one iteration: clear new, run every variant, sort each new.
void Engine::emit_head(std::vector<Op>& ops, const std::vector<std::vector<StepPlan>>& plans, bool idb_inner) {
  Op c{};
  c.kind = Op::CTL;
  c.ctl.st = dst;
  c.ctl.skip_mask = 1;
  auto cmd = [&](CtlCmd x) {   // a full command list goes out as its own launch
    if (c.ctl.n == kMaxCtl) {
      ops.push_back(c);
      c.ctl.n = 0;
    }
    c.ctl.cmd[c.ctl.n++] = x;
  };
  for (int r : idb) {
    cmd({kCtlSetCnt, rels[r].fresh, 0});
    cmd({kCtlZeroSmall, rels[r].hist, 8 * 256});
    if (rels[r].append) {
      cmd({kCtlSetCnt, rels[r].delta_next, 0});
      cmd({kCtlSetCnt, rels[r].sortf, 1});
    }
  }
  cmd({kCtlSetCnt, sc.raw_cnt, 0});
  cmd({kCtlSetCnt, sc.pull_raw_cnt, 0});
  ops.push_back(c);
  if (idb_inner) emit_idb_index(ops);
  for (auto& v : plans) {
    const bool tmp_dense = v.size() > 1 && v.back().dense;
    const bool chain = v.size() > 1 && v[0].chain;
    if (v.size() > 1) {
      Op t{};
      t.kind = Op::CTL;
      t.ctl.st = dst;
      t.ctl.skip_mask = 1;
      t.ctl.cmd[t.ctl.n++] = {kCtlSetCnt, sc.tmp_cnt, 0};
      if (tmp_dense && !chain) t.ctl.cmd[t.ctl.n++] = {kCtlZeroSmall, sc.tmp_hist, 8 * 256};
      ops.push_back(t);
    }
    for (auto& sp : v) {
      if (sp.chain) {
        emit_chain(ops, sp, v.size() > 1 && v[1].invert);
      } else if (sp.invert) {
        emit_invert(ops, sp, chain);
      } else if (sp.dense && sp.outer_slot == sc.tmp_a && chain) {
        emit_dense(ops, sp, true);   // Tmp gathered grouped by its kept column
      } else if (sp.dense && sp.outer_slot == sc.tmp_a) {
        // Tmp sorted (kept column first) so its groups are contiguous
        emit_sort(ops, sc.tmp_a, sc.tmp_b, sc.tmp_cnt, sc.tmp_hist, 1, 0);
        StepPlan d = sp;
        d.outer_slot = (passes & 1) ? sc.tmp_b : sc.tmp_a;
        emit_dense(ops, d);
      } else if (sp.dense && sp.resort) {
        // delta (join column first) exchanged into Tmp's buffers and sorted
        // kept column first
        Op w{};
        w.kind = Op::SWAP;
        w.swap = SwapArgs{dst, sp.outer_slot, sp.outer_cnt, sc.tmp_a, sc.tmp_cnt, b, 1, 0};
        ops.push_back(w);
        Op z{};
        z.kind = Op::CTL;
        z.ctl.st = dst;
        z.ctl.skip_mask = 1;
        z.ctl.cmd[z.ctl.n++] = {kCtlZeroSmall, sc.tmp_hist, 8 * 256, 0};
        ops.push_back(z);
        Op h{};
        h.kind = Op::HIST;
        h.hist = RadixHistArgs{dst, sc.tmp_a, sc.tmp_cnt, sc.tmp_hist, passes, 1};
        ops.push_back(h);
        emit_sort(ops, sc.tmp_a, sc.tmp_b, sc.tmp_cnt, sc.tmp_hist, 1, 0);
        StepPlan d = sp;
        d.outer_slot = (passes & 1) ? sc.tmp_b : sc.tmp_a;
        d.outer_cnt = sc.tmp_cnt;
        d.outer_kcol = 1;
        d.proj0 = kSrcOuter0;
        emit_dense(ops, d);
      } else if (sp.dense) {
        emit_dense(ops, sp);
      } else {
        emit_join(ops, sp);
        if (sp.to_tmp && tmp_dense) ops.back().join.hist_buf = sc.tmp_hist, ops.back().join.hist_passes = passes;
      }
    }
  }
  // sort each new, unless every writer of it is a dense join (sorted and
  // duplicate-free already); the sorted new always ends in `fresh`
  for (int r : idb) {
    int writers_n = 0;
    bool all_dense = true, any_dense = false;
    for (auto& v : plans)
      if (!v.empty() && !v.back().to_tmp && v.back().out_rel == r) {
        ++writers_n;
        all_dense = all_dense && v.back().dense;
        any_dense = any_dense || v.back().dense;
      }
    // one dense writer: new is sorted and duplicate-free already; several
    // writers' outputs are sorted (and deduplicated) together
    if (writers_n == 1 && all_dense) continue;
    const Relation& R = rels[r];
    if (any_dense) {
      // a dense join wrote part of new without digit histograms (a serving
      // admission iteration runs it beside the non-recursive rules): count
      // all of new again
      Op z{};
      z.kind = Op::CTL;
      z.ctl.st = dst;
      z.ctl.skip_mask = 1;
      z.ctl.cmd[z.ctl.n++] = {kCtlZeroSmall, R.hist, 8 * 256, 0};
      ops.push_back(z);
      Op h{};
      h.kind = Op::HIST;
      h.hist = RadixHistArgs{dst, R.fresh, R.fresh, R.hist, passes, 1};
      ops.push_back(h);
    }
    emit_sort(ops, R.fresh, R.fresh_alt, R.fresh, R.hist, 1, 0);
    if (passes & 1) {
      Op w{};
      w.kind = Op::CTL;
      w.ctl.st = dst;
      w.ctl.skip_mask = 1;
      w.ctl.cmd[w.ctl.n++] = {kCtlSwap, R.fresh, R.fresh_alt, 0};
      ops.push_back(w);
    }
  }
}

// LSD passes ping-ponging between `in` and `alt`; the result lands in `in`
// for an even number of passes, else in `alt`.
void Engine::emit_sort(std::vector<Op>& ops, int in, int alt, int cnt, int hist, int skip_mask, int stage_bit) {
  for (int p = 0; p < passes; ++p) {
    Op o{};
    o.kind = Op::PASS;
    RadixPassArgs& a = o.pass;
    a.st = dst;
    a.in_buf = (p & 1) ? alt : in;
    a.out_buf = (p & 1) ? in : alt;
    a.n_cnt = cnt;
    a.hist_buf = hist;
    a.status_buf = sc.radix_status;
    a.pass = p;
    a.shift = 8 * p;
    a.ctr = 1;
    a.skip_mask = skip_mask;
    a.stage_bit = stage_bit;
    a.items = int(cfg.radix_items);
    ops.push_back(o);
  }
}

// Log-structured full, step 0.  When new is large against the large level
// (|new| * kBigRatio > |full|) probing it costs more than streaming full, so
// this iteration merges new straight into full (bigf) after the small level
// has been folded in; otherwise new is probed (smallf).  The small level is
// merged into the large one when it has grown past 1/kLevelRatio of it, when
// bigf is set, or always (`force`); both levels are sorted and disjoint, so
// the merge drops nothing.  Idempotent: a re-run finds the small level empty
// and takes the same decision.
constexpr int kLevelRatio = 8;
constexpr int kMaxLevels = 128;   // levels of an append-only full before the host merges them
constexpr int kBigRatio = 2;
void Engine::emit_level_merge(std::vector<Op>& ops, const Relation& R, bool force) {
  Op g{};
  g.kind = Op::CTL;
  g.ctl.st = dst;
  g.ctl.skip_mask = 3;
  if (force) {
    g.ctl.cmd[g.ctl.n++] = {kCtlCopyCnt, R.gate, R.l1, 0};
  } else {
    g.ctl.cmd[g.ctl.n++] = {kCtlBigFlag, R.bigf, R.fresh, ((long long)R.full << 16) | kBigRatio};
    g.ctl.cmd[g.ctl.n++] = {kCtlNot, R.smallf, R.bigf, 0};
    g.ctl.cmd[g.ctl.n++] = {kCtlMergeGate, R.gate, R.l1,
                            ((long long)R.full << 32) | ((long long)R.bigf << 16) | kLevelRatio};
  }
  ops.push_back(g);
  Op m{};
  m.kind = Op::SETOP;
  SetopArgs& a = m.setop;
  a.st = dst;
  a.a_buf = R.full;
  a.a_cnt = R.full;
  a.b_buf = R.l1;
  a.b_cnt = R.gate;
  a.split_buf = sc.split;
  a.status_buf = sc.setop_status;
  a.d_buf = -1;
  a.d_cnt = -1;
  a.f_buf = R.full_next;
  a.f_cnt = R.full_next;
  a.ctr = 2;
  a.skip_mask = 3;
  a.stage_bit = 1;
  ops.push_back(m);
  Op c{};
  c.kind = Op::CTL;
  c.ctl.st = dst;
  c.ctl.skip_mask = 3;
  c.ctl.cmd[c.ctl.n++] = {kCtlSwapIfCnt, R.full, R.full_next, R.gate};
  c.ctl.cmd[c.ctl.n++] = {kCtlZeroIfCnt, R.l1, 0, R.gate};
  ops.push_back(c);
}

// Populate delta, merge, commit.  With a log-structured full: level merge,
// new minus the large level by sorted probes, then difference and merge
// against the small level (which becomes l1 at the commit).
void Engine::emit_tail(std::vector<Op>& ops, bool force) {
  for (int r : idb) {
    const Relation& R = rels[r];
    if (R.append) {
      // delta = unique(new) (the dense join already removed full's tuples; in
      // iteration 1 full is empty), appended to full as a new level
      Op o{};
      o.kind = Op::SETOP;
      SetopArgs& a = o.setop;
      a.st = dst;
      a.a_buf = sc.empty;
      a.a_cnt = sc.empty;
      a.b_buf = R.fresh;
      a.b_cnt = R.fresh;
      a.split_buf = sc.split;
      a.status_buf = sc.setop_status;
      a.d_buf = R.delta_next;
      a.d_cnt = R.delta_next;
      a.f_buf = -1;
      a.f_cnt = -1;
      a.ctr = 2;
      a.skip_mask = 3;
      a.stage_bit = 1;
      a.gate1 = R.sortf + 1;   // skipped when the dense join wrote delta
      ops.push_back(o);
      if (R.mfull) {   // a delta from the unique (iteration 1) into full's bit matrix
        Op m{};
        m.kind = Op::MCODES;
        m.matrix = MatrixArgs{dst, -1, -1, -1, -1, R.delta_next, R.delta_next, b, R.fbm, R.fcnt, 3, R.sortf + 1};
        ops.push_back(m);
        continue;
      }
      Op p{};
      p.kind = Op::APPEND;
      p.append = AppendArgs{dst, R.delta_next, R.delta_next, R.full, R.full, R.lvidx, R.nlv, b, b, 3, 1};
      if (R.pull) p.append.fcnt_buf = R.fcnt;
      ops.push_back(p);
      continue;
    }
    if (R.mfull) {
      // batched runs (matrix.cuh): delta = unique(new) \ full by bit tests,
      // then delta ORed into the rows; full's count grows at the commit
      Op d{};
      d.kind = Op::MDIFF;
      d.mdiff = MatrixDiffArgs{dst, R.fresh, R.fresh, R.delta_next, R.delta_next, sc.setop_status, R.fbm, b,
                               b + inst_bits, 2, 3, 1};
      ops.push_back(d);
      Op m{};
      m.kind = Op::MCODES;
      m.matrix = MatrixArgs{dst, -1, -1, -1, -1, R.delta_next, R.delta_next, b, R.fbm, R.fcnt, 3, 0, b + inst_bits};
      ops.push_back(m);
      continue;
    }
    if (R.log) {
      const int sorted_new = R.fresh;
      emit_level_merge(ops, R, false);
      // large new: difference + merge against the large level (commit swaps it)
      Op big{};
      big.kind = Op::SETOP;
      SetopArgs& m = big.setop;
      m.st = dst;
      m.a_buf = R.full;
      m.a_cnt = R.full;
      m.b_buf = sorted_new;
      m.b_cnt = R.fresh;
      m.split_buf = sc.split;
      m.status_buf = sc.setop_status;
      m.d_buf = R.delta_next;
      m.d_cnt = R.delta_next;
      m.f_buf = R.full_next;
      m.f_cnt = R.full_next;
      m.ctr = 2;
      m.skip_mask = 3;
      m.stage_bit = 1;
      m.gate1 = R.bigf + 1;
      ops.push_back(big);
      // small new: probe the large level, then difference + merge against
      // the small one
      Op d{};
      d.kind = Op::DIFF;
      d.diff = DiffArgs{dst, R.full, R.full, sorted_new, R.fresh, R.newp, R.newp, sc.setop_status, 2, 3, 1,
                        R.smallf + 1};
      ops.push_back(d);
      Op o{};
      o.kind = Op::SETOP;
      SetopArgs& a = o.setop;
      a.gate1 = R.smallf + 1;
      a.st = dst;
      a.a_buf = R.l1;
      a.a_cnt = R.l1;
      a.b_buf = R.newp;
      a.b_cnt = R.newp;
      a.split_buf = sc.split;
      a.status_buf = sc.setop_status;
      a.d_buf = R.delta_next;
      a.d_cnt = R.delta_next;
      a.f_buf = R.l1_next;
      a.f_cnt = R.l1_next;
      a.ctr = 2;
      a.skip_mask = 3;
      a.stage_bit = 1;
      ops.push_back(o);
      continue;
    }
    Op o{};
    o.kind = Op::SETOP;
    SetopArgs& a = o.setop;
    a.st = dst;
    a.a_buf = R.full;
    a.a_cnt = R.full;
    a.b_buf = R.fresh;   // sorted new (emit_head leaves it there)
    a.b_cnt = R.fresh;
    a.split_buf = sc.split;
    a.status_buf = sc.setop_status;
    a.d_buf = R.delta_next;
    a.d_cnt = R.delta_next;
    a.f_buf = R.full_next;
    a.f_cnt = R.full_next;
    a.ctr = 2;
    a.skip_mask = 3;
    a.stage_bit = 1;
    ops.push_back(o);
  }
  bool any_pull = false;
  for (int r : idb) any_pull = any_pull || rels[r].pull;
  if (any_pull) {   // this iteration's group bitmaps become the previous ones (after a clean stage only)
    Op w{};
    w.kind = Op::CTL;
    w.ctl.st = dst;
    w.ctl.skip_mask = 3;
    w.ctl.cmd[w.ctl.n++] = {kCtlSwap, sc.dense_bm, sc.dense_bm_prev, 0};
    ops.push_back(w);
  }
  Op c{};
  c.kind = Op::COMMIT;
  c.commit.st = dst;
  c.commit.nrel = int(idb.size());
  for (size_t i = 0; i < idb.size(); ++i) {
    const Relation& R = rels[idb[i]];
    c.commit.full[i] = R.log ? R.l1 : R.full;          // the level that absorbed delta
    c.commit.full_next[i] = R.log ? R.l1_next : R.full_next;
    c.commit.alt_full[i] = R.full;
    c.commit.alt_full_next[i] = R.full_next;
    c.commit.alt_flag1[i] = R.log ? R.bigf + 1 : 0;
    c.commit.delta[i] = R.delta;
    c.commit.delta_next[i] = R.delta_next;
    c.commit.history[i] = R.history;
    c.commit.fresh[i] = R.fresh;
    c.commit.append_nlv1[i] = R.append && !R.mfull ? R.nlv + 1 : 0;
    c.commit.add_full[i] = R.mfull ? 1 : 0;
  }
  c.commit.max_levels = kMaxLevels;
  c.commit.force = force;
  ops.push_back(c);
}

template <typename K>
hisa_status Engine::exec_t(const std::vector<Op>& ops) {
  for (const Op& o : ops) {
    switch (o.kind) {
      case Op::CTL: launch_ctl(o.ctl, stream); break;
      case Op::JOIN: launch_join<K>(o.join, grid, stream); break;
      case Op::PASS: launch_radix_pass<K>(o.pass, grid, stream); break;
      case Op::HIST: launch_radix_hist<K>(o.hist, grid, stream); break;
      case Op::SETOP: launch_setop<K>(o.setop, grid, stream); break;
      case Op::COMMIT: launch_commit(o.commit, stream); break;
      case Op::RUNS: launch_count_runs<K>(o.runs, grid, stream); break;
      case Op::INDEX: launch_index<K>(o.index, grid, stream); break;
      case Op::ZERO: launch_zero(o.zero, grid, stream); break;
      case Op::SWAP: launch_swap<K>(o.swap, grid, stream); break;
      case Op::DIFF: launch_diff<K>(o.diff, grid, stream); break;
      case Op::GCOMPACT: launch_group_compact(o.groups, o.groups.b, stream); break;
      case Op::APPEND: launch_append<K>(o.append, grid, stream); break;
      case Op::GROUPS: launch_group_starts<K>(o.groups, grid, stream); break;
      case Op::DENSE: launch_join_dense<K>(o.dense, grid, stream); break;
      case Op::CHAIN: launch_chain<K>(o.chain, grid, stream); break;
      case Op::MCODES: launch_matrix_codes<K>(o.matrix, grid, stream); break;
      case Op::MDIFF: launch_matrix_diff<K>(o.mdiff, grid, stream); break;
    }
  }
  return check_launch("kernel launch");
}

hisa_status Engine::exec(const std::vector<Op>& ops) {
  return wide ? exec_t<uint64_t>(ops) : exec_t<uint32_t>(ops);
}

// ---- EDB preparation (Algorithm 1 + Algorithm 2 for every index) ------------------------

template <typename K>
hisa_status Engine::prepare_rel_t(Relation& r, int order, int slot) {
  const uint64_t n = r.staged;
  hisa_status s;
  if ((s = ensure(sc.tmp_a, n)) || (s = ensure(sc.tmp_b, n)) || (s = ensure(slot, n))) return s;
  if ((s = ensure(sc.radix_status, ((n + radix_tile<K>() - 1) / radix_tile<K>()) * 256 + 1))) return s;
  const uint64_t st_tiles = (n + setop_tile<K>() - 1) / setop_tile<K>() + 2;
  if ((s = ensure(sc.split, st_tiles)) || (s = ensure(sc.setop_status, st_tiles))) return s;
  hs.cnt[sc.tmp_a] = n;
  hs.cnt[sc.empty] = 0;
  if ((s = upload())) return s;
  EncodeArgs e{dst, r.stage[0], r.stage[1], n, sc.tmp_a, sc.empty, b, order, 0, batched ? r.stage_inst : nullptr};
  launch_encode<K>(e, grid, stream);
  CtlArgs z{};
  z.st = dst;
  z.n = 1;
  z.cmd[0] = {kCtlZeroSmall, sc.hist, 8 * 256};
  launch_ctl(z, stream);
  RadixHistArgs h{dst, sc.tmp_a, sc.tmp_a, sc.hist, passes, 0};
  launch_radix_hist<K>(h, grid, stream);
  std::vector<Op> ops;
  emit_sort(ops, sc.tmp_a, sc.tmp_b, sc.tmp_a, sc.hist, 0, 0);
  Op u{};
  u.kind = Op::SETOP;
  SetopArgs& a = u.setop;
  a.st = dst;
  a.a_buf = sc.empty;
  a.a_cnt = sc.empty;
  a.b_buf = (passes & 1) ? sc.tmp_b : sc.tmp_a;
  a.b_cnt = sc.tmp_a;
  a.split_buf = sc.split;
  a.status_buf = sc.setop_status;
  a.d_buf = slot;
  a.d_cnt = slot;
  a.f_buf = -1;
  a.f_cnt = -1;
  a.ctr = 2;
  a.skip_mask = 0;
  a.stage_bit = 1;
  ops.push_back(u);
  if ((s = exec_t<K>(ops))) return s;
  if ((s = download())) return s;
  if (hs.overflow || hs.error) return ctx_fail(HISA_ERR_CUDA, "EDB preparation overflowed", nullptr);
  // run index of the join column: direct-addressed over a small key domain
  if (r.need_idx[order] && direct_bits) {
    if ((s = ensure(r.table[order], ((1ull << direct_bits) + 2) / 2 + 1)) || (s = upload())) return s;
    IndexArgs ia{dst, slot, slot, r.table[order], b, -1, 0, direct_bits};
    launch_index<K>(ia, grid, stream);
    if ((s = check_launch("index build"))) return s;
  } else if (r.need_idx[order]) {   // else hashed over its runs
    hs.cnt[sc.runs] = 0;
    if ((s = upload())) return s;
    RunsArgs ra{dst, slot, slot, b, sc.runs, 0};
    launch_count_runs<K>(ra, grid, stream);
    if ((s = download())) return s;
    const uint64_t runs = hs.cnt[sc.runs];
    uint64_t cap = 16;
    while (double(cap) * cfg.load_factor < double(runs)) cap <<= 1;
    if ((s = ensure(r.table[order], cap))) return s;
    hs.buf[r.table[order]].cap = cap;  // power of two for the probe mask
    if ((s = upload())) return s;
    ZeroArgs za{dst, r.table[order], 16, 0};
    launch_zero(za, grid, stream);
    IndexArgs ia{dst, slot, slot, r.table[order], b, -1, 0};
    launch_index<K>(ia, grid, stream);
    if ((s = check_launch("index build"))) return s;
    if ((s = download())) return s;
    if (hs.error) return ctx_fail(HISA_ERR_CUDA, "index build", "probe limit");
  }
  return HISA_OK;
}

hisa_status Engine::prepare_edb() {
  hisa_status s;
  // a run that failed (an allocation refused during a regrow, say) leaves its
  // overflow bits, needs and error code in the host mirror of the device
  // state; uploaded again, they would make every kernel here skip its work
  hs.overflow = 0;
  hs.error = 0;
  std::memset(hs.need, 0, sizeof hs.need);
  for (auto& r : rels) {
    if (r.idb) continue;
    for (int order = 0; order < 2; ++order) {
      if (order == 1 && !r.need_idx[1]) continue;
      const int slot = order == 0 ? r.base : r.rev;
      s = wide ? prepare_rel_t<uint64_t>(r, order, slot) : prepare_rel_t<uint32_t>(r, order, slot);
      if (s) return s;
    }
  }
  edb_dirty = false;
  return HISA_OK;
}

// ---- growth (Section 5.3) ----------------------------------------------------------------

// Grows slot `id` to `cap` elements keeping its first `keep` elements.
hisa_status Engine::grow_keep(int id, uint64_t cap, uint64_t keep) {
  if (hs.buf[id].cap >= cap && hs.buf[id].ptr) return HISA_OK;
  void* p;
  hisa_status s = dev_alloc(size_t(cap) * slot_elem[id], &p);
  if (s) return s;
  if (keep && hs.buf[id].ptr)
    CU(cudaMemcpyAsync(p, hs.buf[id].ptr, size_t(keep) * slot_elem[id], cudaMemcpyDeviceToDevice, stream));
  dev_free(hs.buf[id].ptr);
  hs.buf[id] = {p, cap};
  return HISA_OK;
}

hisa_status Engine::regrow() {
  static const bool debug = std::getenv("HISA_DEBUG") != nullptr;
  if (debug) {
    std::fprintf(stderr, "[hisa] iter %u overflow %u:", hs.iter, hs.overflow);
    for (int id = 0; id < nslots; ++id)
      if (hs.need[id]) std::fprintf(stderr, " slot %d need %llu cap %llu", id, (unsigned long long)hs.need[id],
                                    (unsigned long long)hs.buf[id].cap);
    std::fprintf(stderr, "\n");
  }
  for (int id = 0; id < nslots; ++id) {
    const uint64_t need = hs.need[id];
    if (need == 0 || need <= hs.buf[id].cap) continue;
    // an append-only full and its level indexes are live: grow them in place
    bool kept = false;
    for (int r : idb) {
      const Relation& R = rels[r];
      if (!R.append || (id != R.full && id != R.lvidx)) continue;
      const uint64_t live = id == R.full ? hs.cnt[R.full] : hs.cnt[R.nlv] * ((1ull << b) + 1);
      const uint64_t grow = id == R.full ? std::max(uint64_t(cfg.ebm_k * double(need - live)), need / 4) : need;
      hisa_status s = grow_keep(id, need + grow + 1024, live);
      if (s) return s;
      ++regrows;
      kept = true;
    }
    if (kept) continue;
    uint64_t cap = need + need / 8 + 1024;
    if (slot_pow2[id]) {   // hash table: the probe mask needs a power of two
      cap = 16;
      while (cap < need) cap <<= 1;
    }
    int partner = -1, live = -1;
    for (int r : idb) {
      const Relation& R = rels[r];
      if (id == R.full_next || id == R.full || id == R.rev_next || id == R.rev || id == R.l1 || id == R.l1_next) {
        // eager buffer management: full + k * delta, and at least a quarter more
        const bool rv = id == R.rev_next || id == R.rev;
        const bool small = id == R.l1 || id == R.l1_next;
        const int cur = rv ? R.rev : small ? R.l1 : R.full;
        const uint64_t delta = need > hs.cnt[cur] ? need - hs.cnt[cur] : need;
        cap = need + std::max(uint64_t(cfg.ebm_k * double(delta)), need / 4) + 1024;
        partner = rv      ? (id == R.rev_next ? R.rev : R.rev_next)
                  : small ? (id == R.l1_next ? R.l1 : R.l1_next)
                          : (id == R.full_next ? R.full : R.full_next);
        live = cur;
      } else if (id == R.delta_next || id == R.delta) {
        cap = need + need / 4 + 1024;
        partner = id == R.delta_next ? R.delta : R.delta_next;
        live = R.delta;
      }
    }
    hisa_status s = ensure(id, cap);
    if (s) return s;
    // the two versions swap every iteration: grow the partner too (keeping the
    // live version's tuples), or the next iteration overflows again
    if (partner >= 0 && (s = grow_keep(partner, cap, partner == live ? hs.cnt[live] : 0))) return s;
    ++regrows;
  }
  // scratch whose size follows from the same counts grows in the same step, so
  // one growth event costs one re-run (only when the join stage re-runs: after
  // a merge-stage overflow the radix buffers hold the sorted new tuples)
  const int kt = wide ? radix_tile<uint64_t>() : radix_tile<uint32_t>();
  const int ks = wide ? setop_tile<uint64_t>() : setop_tile<uint32_t>();
  uint64_t new_cap = 0, full_cap = 0, delta_cap = 0;
  for (int r : idb) {
    const Relation& R = rels[r];
    new_cap = std::max({new_cap, hs.buf[R.fresh].cap, hs.buf[R.fresh_alt].cap});
    full_cap = std::max({full_cap, hs.cnt[R.full], hs.buf[R.full_next].cap});
    delta_cap = std::max({delta_cap, hs.buf[R.delta].cap, hs.buf[R.delta_next].cap});
    if (R.log) full_cap = std::max({full_cap, hs.cnt[R.full] + hs.buf[R.l1].cap, hs.buf[R.l1_next].cap});
  }
  hisa_status s;
  if (hs.overflow & 1) {
    for (int r : idb) {
      const Relation& R = rels[r];
      if ((s = ensure(R.fresh, new_cap)) || (s = ensure(R.fresh_alt, new_cap))) return s;
      // the column-swapped delta sorted into the reverse-order mirror
      if (R.need_idx[1] && ((s = ensure(R.rswap, delta_cap)) || (s = ensure(R.rswap_alt, delta_cap)))) return s;
    }
    // radix look-back words for new, the swapped delta and a sorted Tmp; Tmp's
    // sort partner; the join's write chunks
    if ((s = ensure(sc.radix_status, (std::max({new_cap, delta_cap, hs.buf[sc.tmp_a].cap}) / kt + 2) * kRadixDigits)) ||
        (s = ensure(sc.tmp_b, hs.buf[sc.tmp_a].cap)) || (s = ensure(sc.starts, new_cap / kJoinChunkMin + 2)))
      return s;
  }
  for (int r : idb) {   // new minus the large level holds at most |new|
    const Relation& R = rels[r];
    if (R.log && (s = ensure(R.newp, new_cap))) return s;
  }
  // next iterations: delta is the outer relation of the joins; full + new is merged
  if ((s = ensure(sc.offs, delta_cap + 1)) || (s = ensure(sc.join_status, delta_cap / kJoinTile + 2))) return s;
  if ((s = ensure(sc.groups, std::min<uint64_t>(delta_cap, 1ull << (b + inst_bits)) + 2)) ||
      (s = ensure(sc.dense_status, std::min<uint64_t>(delta_cap, 1ull << (b + inst_bits)) + 2)) ||
      (s = ensure(sc.dense_units, std::min<uint64_t>(delta_cap, 1ull << (b + inst_bits)) + 2)) ||
      (s = ensure(sc.dense_done, std::min<uint64_t>(delta_cap, 1ull << (b + inst_bits)) + 2)) ||
      (s = ensure(sc.dense_mslot, std::min<uint64_t>(delta_cap, 1ull << (b + inst_bits)) + 2)))
    return s;
  if ((s = ensure(sc.split, (full_cap + std::max(new_cap, delta_cap)) / ks + 2)) ||
      (s = ensure(sc.setop_status,
                  std::max((full_cap + std::max(new_cap, delta_cap)) / ks, new_cap / kDiffTile) + 2)))
    return s;
  std::memset(hs.need, 0, sizeof hs.need);
  hs.overflow = 0;
  return HISA_OK;
}

// ---- the fixpoint loop ---------------------------------------------------------------------

hisa_status Engine::run(hisa_run_stats* stats) {
  auto t0 = std::chrono::steady_clock::now();
  hisa_status s;
  if (!compiled || edb_dirty) {
    if ((s = compile())) return s;
    double ms = 0;
    auto e0 = std::chrono::steady_clock::now();
    if ((s = prepare_edb())) return s;
    ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - e0).count();
    last_stats.ms_edb = ms;
    // plans
    ops1.clear();
    opsN.clear();
    tail.clear();
    emit_head(ops1, plan1, false);
    emit_tail(ops1, false);
    emit_head(opsN, planN, true);
    emit_tail(opsN, false);
    emit_tail(tail, false);
  } else {
    last_stats.ms_edb = 0;
  }
  const double ms_edb = last_stats.ms_edb;
  last_stats = hisa_run_stats{};
  last_stats.ms_edb = ms_edb;
  regrows = 0;
  if (bitjoin) return run_bitjoin(stats, t0);
  if ((s = init_run_state())) return s;
  return run_loop(stats, t0);
}

// Fresh IDB state: empty versions with initial capacities, counters reset.
hisa_status Engine::init_run_state() {
  hisa_status s;
  // initial capacities: a multiple of the EDB size
  uint64_t nedb = 1024;
  for (auto& r : rels)
    if (!r.idb) nedb = std::max<uint64_t>(nedb, r.staged);
  const int kt = wide ? radix_tile<uint64_t>() : radix_tile<uint32_t>();
  for (int r : idb) {
    Relation& R = rels[r];
    for (int id : {R.full, R.full_next, R.delta, R.delta_next, R.fresh, R.fresh_alt})
      if ((s = ensure(id, 4 * nedb))) return s;
    if ((s = ensure(R.hist, 8 * 256)) || (s = ensure(R.history, std::min<uint64_t>(cfg.max_iters + 1, 1u << 20))))
      return s;
    for (int id : {R.full, R.full_next, R.delta, R.delta_next, R.fresh}) hs.cnt[id] = 0;
    if (R.need_idx[1]) {
      for (int id : {R.rev, R.rev_next, R.rswap, R.rswap_alt})
        if ((s = ensure(id, 4 * nedb))) return s;
      hs.cnt[R.rev] = hs.cnt[R.rev_next] = hs.cnt[R.rswap] = 0;
    }
    if (R.append) {
      if ((s = ensure(R.lvidx, 8 * ((1ull << b) + 1)))) return s;
      hs.cnt[R.nlv] = 0;
      hs.cnt[R.sortf] = 1;
    }
    if (R.log) {
      for (int id : {R.l1, R.l1_next, R.newp})
        if ((s = ensure(id, 4 * nedb))) return s;
      hs.cnt[R.l1] = hs.cnt[R.l1_next] = hs.cnt[R.newp] = hs.cnt[R.gate] = 0;
      hs.cnt[R.bigf] = hs.cnt[R.smallf] = 0;
    }
    for (int col = 0; col < 2; ++col) {
      if (!R.need_idx[col]) continue;
      uint64_t cap = 1024;
      if (direct_bits) cap = ((1ull << direct_bits) + 2) / 2 + 1;
      else
        while (double(cap) * cfg.load_factor < double(nedb)) cap <<= 1;
      if ((s = ensure(R.table[col], cap))) return s;
      hs.cnt[R.runs_cnt[col]] = 0;
    }
  }
  hs.cnt[sc.tmp_cnt] = 0;
  hs.cnt[sc.raw_cnt] = hs.cnt[sc.group_cnt] = hs.cnt[sc.pull_raw_cnt] = 0;
  if (b + inst_bits <= kDirectMaxBits && (s = ensure(sc.dense_first, (1ull << (b + inst_bits)) + 2))) return s;
  bool any_chain = false;
  for (auto& v : planN) any_chain = any_chain || (!v.empty() && (v[0].chain || v[0].invert));
  if (any_chain && ((s = ensure(sc.chain_dfirst, (1ull << b) + 2)) || (s = ensure(sc.chain_pre, 4 * nedb + 2)) ||
                    (s = ensure(sc.chain_tfirst, (1ull << b) + 2))))
    return s;
  if ((s = ensure(sc.tmp_hist, 8 * 256)) || (s = ensure(sc.tmp_b, 4 * nedb))) return s;
  if ((s = ensure(sc.groups, std::min<uint64_t>(4 * nedb, 1ull << (b + inst_bits)) + 2)) ||
      (s = ensure(sc.dense_status, std::min<uint64_t>(4 * nedb, 1ull << (b + inst_bits)) + 2)) ||
      (s = ensure(sc.dense_units, std::min<uint64_t>(4 * nedb, 1ull << (b + inst_bits)) + 2)) ||
      (s = ensure(sc.dense_done, std::min<uint64_t>(4 * nedb, 1ull << (b + inst_bits)) + 2)) ||
      (s = ensure(sc.dense_mslot, std::min<uint64_t>(4 * nedb, 1ull << (b + inst_bits)) + 2)))
    return s;
  bool any_pull = false;
  for (int r : idb) any_pull = any_pull || rels[r].pull;
  if (any_pull && ((s = ensure(sc.dense_plist, std::min<uint64_t>(4 * nedb, 1ull << b) + 2)) ||
                   (s = ensure(sc.prev_gi, 1ull << b))))
    return s;
  if (any_pull) {   // the two group-bitmap slots swap every iteration: the same capacity for both
    const uint64_t cap = std::max(hs.buf[sc.dense_bm].cap, hs.buf[sc.dense_bm_prev].cap);
    if (cap && ((s = ensure(sc.dense_bm, cap)) || (s = ensure(sc.dense_bm_prev, cap)))) return s;
  }
  if ((s = ensure(sc.radix_status, (4 * nedb / kt + 2) * 256)) || (s = ensure(sc.offs, 4 * nedb + 1)) ||
      (s = ensure(sc.join_status, 4 * nedb / kJoinTile + 2)) || (s = ensure(sc.starts, 4 * nedb / kJoinChunkMin + 2)) ||
      (s = ensure(sc.split, 8 * nedb / 2048 + 2)) || (s = ensure(sc.setop_status, 8 * nedb / 2048 + 2)) ||
      (s = ensure(sc.tmp_a, 4 * nedb)))
    return s;
  // look-back words carry a 20-bit epoch tag: clear them well before it wraps
  if (hs.epoch > (1u << 20) - (1u << 16)) {
    for (int id : {sc.radix_status, sc.setop_status, sc.join_status})
      if (hs.buf[id].ptr) CU(cudaMemsetAsync(hs.buf[id].ptr, 0, hs.buf[id].cap * 8, stream));
    hs.epoch = 0;
  }
  hs.iter = 0;
  hs.go = 1;
  hs.overflow = 0;
  hs.error = 0;
  hs.max_iters = cfg.max_iters;
  hs.aux[0] = 0;
  hs.aux[1] = 0;
  std::memset(hs.need, 0, sizeof hs.need);
  inst_hist.assign(idb.size(), {});
  for (int r : idb) {
    Relation& R = rels[r];
    if (!R.mfull) continue;
    // one row per (instance slot, value): 2^(inst_bits + b) rows of 2^b bits
    const uint64_t rows = 1ull << (b + (batched ? inst_bits : 0));
    const uint64_t words = rows * (b >= 5 ? (1ull << (b - 5)) : 1ull);
    if ((s = ensure(R.fbm, words)) || (s = ensure(R.fcnt, rows))) return s;
    CU(cudaMemsetAsync(hs.buf[R.fbm].ptr, 0, words * 4, stream));
    CU(cudaMemsetAsync(hs.buf[R.fcnt].ptr, 0, rows * 4, stream));
  }
  for (int r : idb) {
    Relation& R = rels[r];
    if (!R.pull) continue;
    const uint64_t nw = b >= 5 ? (1ull << (b - 5)) : 1;
    if ((s = ensure(R.fcnt, 1ull << b)) || (s = ensure(R.pull_bm, nw)) || (s = ensure(R.pull_out, nw)) ||
        (s = ensure(R.pull_first, 1ull << b)) || (s = ensure(R.tdeg, 1ull << b)))
      return s;
    CU(cudaMemsetAsync(hs.buf[R.fcnt].ptr, 0, (1ull << b) * 4, stream));
    CU(cudaMemsetAsync(hs.buf[R.pull_bm].ptr, 0, nw * 4, stream));   // iteration 2 marks (push)
    hs.cnt[R.nout] = 0;
  }
  if ((s = upload())) return s;
  for (int r : idb) {
    const Relation& R = rels[r];
    if (!R.pull) continue;
    PullOutArgs pa{dst, R.pull_index, R.pull_inner, R.push_index, b, R.pull_out, R.pull_first, R.tdeg, R.nout};
    launch_pull_out(pa, grid, stream);
    if ((s = check_launch("pull out"))) return s;
  }
  return HISA_OK;
}

hisa_status Engine::run_loop(hisa_run_stats* stats, std::chrono::steady_clock::time_point t0) {
  hisa_status s;
  uint32_t graph_launches = 0;
  int guard = 0;
  uint32_t last_iter = hs.iter;
  const bool timing = cfg.flags & HISA_FLAG_PHASE_TIMES;
  const double kb = wide ? 8.0 : 4.0;
  std::memset(kstat, 0, sizeof kstat);
  timer.reset();
  struct TimerGuard {
    explicit TimerGuard(KernelTimer* t) { g_timer = t; }
    ~TimerGuard() { g_timer = nullptr; }
  } tg(timing ? &timer : nullptr);
  const uint64_t launches0 = g_launches;
  uint64_t graph_kernels = 0;
  while (true) {
    const bool first = hs.iter == 0;
    const bool use_graph = !first && (cfg.flags & HISA_FLAG_GRAPH) && !timing && !batched;
    // batched runs read per-instance counts after every iteration: one
    // iteration per graph launch
    const bool use_once = !first && (cfg.flags & HISA_FLAG_GRAPH) && !timing && batched;
    const size_t rec0 = timer.recs.size();
    std::vector<uint64_t> m_prev, d_prev, l_prev;
    for (int r : idb) {
      m_prev.push_back(hs.cnt[rels[r].full]);
      d_prev.push_back(hs.cnt[rels[r].delta]);
      l_prev.push_back(rels[r].log ? hs.cnt[rels[r].l1] : 0);
    }
    const uint32_t iter0 = hs.iter;
    if (use_graph) {
      if ((s = launch_graph())) return s;
      ++graph_launches;
    } else if (use_once) {
      if ((s = launch_once())) return s;
      ++graph_launches;
      graph_kernels += body_kernels;
    } else {
      if ((s = exec(first ? ops1 : opsN))) return s;
    }
    if ((s = download())) return s;
    if (use_graph) graph_kernels += body_kernels * (hs.iter - iter0 + (hs.overflow ? 1 : 0));
    if (timing) {
      if (hs.overflow) {
        timer.truncate(rec0);   // the iteration re-runs: keep only clean ones
      } else {
        // algorithmic bytes of this iteration's kernels (counts read back above)
        for (size_t i = 0; i < idb.size(); ++i) {
          const Relation& R = rels[idb[i]];
          const double nn = double(hs.cnt[R.fresh]), nd = double(hs.cnt[R.delta]);
          const double m = double(m_prev[i]), dp = double(d_prev[i]);
          bool dense = false, via_tmp = false;
          const StepPlan* chain = nullptr;
          for (auto& v : planN)
            if (!first && !v.empty() && v.back().dense && v.back().out_rel == idb[i]) {
              dense = true;
              via_tmp = v.size() > 1;
              if (v[0].chain) chain = &v[0];
            }
          if (chain) {
            // Tmp gathered: delta's index; per inner tuple read it and two
            // index entries, write its offset; scan; gather reads the inner
            // tuple, its index entries and offset, the delta run, writes Tmp
            const double tm = double(hs.cnt[sc.tmp_cnt]);
            const Relation& A = rels[chain->inner_rel];
            const double na = double(hs.cnt[chain->inner_col == 1 ? A.base : A.rev]);
            kstat[kKIndex].bytes += 8.0 * double((1u << b) + 1) * 2.0;
            kstat[kKChainLen].bytes += na * (kb + 16.0 + 8.0);
            kstat[kKChainScan].bytes += 16.0 * na;
            kstat[kKChainGather].bytes += na * (kb + 24.0) + 2.0 * tm * kb;
          } else if (via_tmp) {   // first join into Tmp, Tmp sorted by its kept column
            const double tm = double(hs.cnt[sc.tmp_cnt]);
            kstat[kKJoinWrite].bytes += 2.0 * tm * kb + dp * (kb + 8.0);
            kstat[kKJoinCount].bytes += dp * (kb + 8.0 + 16.0);
            kstat[kKRadixPass].bytes += passes * 2.0 * tm * kb;
          }
          if (dense) {
            // group starts: direct index of delta, compaction; mark: read delta, probe,
            // read the inner runs (raw results), write the bitmaps; scan:
            // counts; emit: read the bitmaps, write new
            const double raw = double(hs.cnt[sc.raw_cnt]), ng = double(hs.cnt[sc.group_cnt]);
            const double bmb = ng * double(b >= 5 ? (1u << (b - 5)) : 1u) * 4.0;
            kstat[kKIndex].bytes += 8.0 * double(1u << b);
            kstat[kKGroups].bytes += 16.0 * double(1u << b) + 8.0 * ng;
            // (+ the full levels' runs read for the set difference)
            // (+ full: its row of the bit matrix, or the levels' runs of the group)
            kstat[kKJoinDense].bytes += dp * (kb + 16.0) + raw * kb + bmb + (R.mfull ? bmb : m * kb);
            // pulled groups: their delta, full's runs and the inner tuples they
            // scanned (the push term above still counts full for every group)
            kstat[kKJoinPull].bytes += double(hs.cnt[sc.pull_raw_cnt]) * kb;
            kstat[kKDenseScan].bytes += 16.0 * ng;
            kstat[kKDenseEmit].bytes += bmb + nn * kb;
          } else {
            kstat[kKRadixPass].bytes += passes * 2.0 * nn * kb;
          }
          if (R.append) {
            // unique of new into delta, then delta copied behind full with its
            // level index
            if (nn > 0 && !dense) kstat[kKSetop].bytes += (nn + nd) * kb;
            if (nd > 0 && !R.mfull) kstat[kKAppend].bytes += 2.0 * nd * kb + 8.0 * double((1u << b) + 1);
            if (nd > 0 && R.mfull && !dense) kstat[kKMatrix].bytes += nd * kb + 8.0 * nd;
          } else if (R.mfull) {
            // bit tests of new (one matrix word each), delta written; delta ORed in
            if (nn > 0) kstat[kKMatrixDiff].bytes += nn * (kb + 4.0) + nd * kb;
            if (nd > 0) kstat[kKMatrix].bytes += nd * (kb + 8.0);
          } else if (R.log && hs.cnt[R.bigf]) {
            // small level folded in, then new merged into the large level
            const double lp = double(l_prev[i]);
            if (lp > 0) kstat[kKSetop].bytes += 2.0 * (m + lp) * kb;
            if (nn > 0) kstat[kKSetop].bytes += (m + lp + nn) * kb + (m + lp + 2.0 * nd) * kb;
          } else if (R.log) {
            // level merge (when the large level changed), new minus the large
            // level (read new, write new'), small-level difference + merge
            const double m_after = double(hs.cnt[R.full]), np = double(hs.cnt[R.newp]);
            const double l1 = m_after != m ? 0.0 : double(l_prev[i]);
            if (m_after != m) kstat[kKSetop].bytes += 2.0 * m_after * kb;
            if (nn > 0) {
              kstat[kKDiffProbe].bytes += (nn + np) * kb;
              kstat[kKSetop].bytes += (l1 + np) * kb + (l1 + 2.0 * nd) * kb;
            }
          } else if (nn > 0) {
            kstat[kKSetop].bytes += (m + nn) * kb + (m + 2.0 * nd) * kb;
          }
          if (!dense) {
            kstat[kKJoinWrite].bytes += 2.0 * nn * kb + dp * (kb + 8.0);
            kstat[kKJoinCount].bytes += dp * (kb + 8.0 + 16.0);
          }
          // inner-relation upkeep at the head of this iteration
          if (!first && R.need_idx[1]) {
            kstat[kKSwap].bytes += 2.0 * dp * kb;
            kstat[kKRadixPass].bytes += passes * 2.0 * dp * kb;
            kstat[kKSetop].bytes += 2.0 * m * kb;
          }
          for (int col = 0; col < 2 && !first; ++col) {
            if (!R.need_idx[col]) continue;
            kstat[kKRuns].bytes += m * kb;
            kstat[kKIndex].bytes += m * kb + double(hs.cnt[R.runs_cnt[col]]) * 16.0;
            kstat[kKZero].bytes += double(hs.buf[R.table[col]].cap) * 16.0;
          }
        }
      }
    }
    if (hs.error) {
      return ctx_fail(hs.error == kDevTimeout ? HISA_ERR_DEVICE_TIMEOUT : HISA_ERR_CUDA, "device error",
                      hs.error == kDevTimeout ? "bounded wait expired" : "probe limit / bad state");
    }
    if (hs.iter != last_iter) {   // progress: an iteration committed (launch or tail re-run)
      guard = 0;
      last_iter = hs.iter;
    }
    if (hs.overflow) {
      if (++guard > 16) {
        std::string m = "overflow bits " + std::to_string(hs.overflow) + " iter " + std::to_string(hs.iter) + ":";
        for (int id = 0; id < nslots; ++id)
          if (hs.need[id])
            m += " slot " + std::to_string(id) + " need " + std::to_string(hs.need[id]) + " cap " +
                 std::to_string(hs.buf[id].cap);
        return ctx_fail(HISA_ERR_OOM, "buffers keep overflowing", m.c_str());
      }
      const uint32_t bits = hs.overflow;
      if ((s = regrow())) return s;
      if ((s = upload())) return s;
      if (bits & 1) continue;       // join/sort stage: re-run the whole iteration
      const size_t rec1 = timer.recs.size();
      if ((s = exec(tail))) return s;   // only the set-difference/merge stage
      if ((s = download())) return s;
      if (timing) timer.truncate(rec1);
      if (hs.overflow) {
        const uint32_t bits2 = hs.overflow;
        if ((s = regrow())) return s;
        if ((s = upload())) return s;
        (void)bits2;
        continue;
      }
    }
    if (batched && !hs.overflow && hs.iter != iter0) {
      // per-instance |delta| of the iteration just committed
      std::vector<std::vector<uint64_t>> rows;
      if ((s = collect_inst_rows(rows))) return s;
      for (size_t i = 0; i < idb.size(); ++i) {
        auto& h = inst_hist[i];
        if (h.size() < rows[i].size()) h.resize(rows[i].size());
        for (size_t q = 0; q < rows[i].size(); ++q) h[q].push_back(rows[i][q]);
      }
    }
    if (!hs.go) {
      if (hs.aux[2]) {   // an append-only full reached kMaxLevels: merge its levels, go on
        if ((s = compact_levels())) return s;
        hs.aux[2] = 0;
        hs.go = 1;
        if ((s = upload())) return s;
        continue;
      }
      break;
    }
  }
  if ((s = merge_levels())) return s;
  if (hs.iter >= cfg.max_iters && hs.aux[0] == hs.iter)
    return ctx_fail(HISA_ERR_NOT_CONVERGED, "max_iters reached", nullptr);
  // delta histories
  const uint32_t K = uint32_t(hs.aux[0]);
  for (int r : idb) {
    Relation& R = rels[r];
    R.delta_counts.assign(K, 0);
    if (K) CU(cudaMemcpyAsync(R.delta_counts.data(), hs.buf[R.history].ptr, K * 8, cudaMemcpyDeviceToHost, stream));
  }
  CU(cudaStreamSynchronize(stream));
  if (timing) {
    for (auto& rc : timer.recs) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, rc.a, rc.b);
      kstat[rc.kind].ms += ms;
      kstat[rc.kind].launches += 1;
    }
    timer.reset();
  }
  last_stats.kernel_launches = (g_launches - launches0) + graph_kernels;
  last_stats.tuples_joined = hs.aux[1];
  last_stats.iterations = K;
  last_stats.iterations_run = hs.iter;
  last_stats.regrows = regrows;
  last_stats.graph_launches = graph_launches;
  last_stats.peak_bytes = peak_bytes;
  last_stats.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = last_stats;
  ran = true;
  return HISA_OK;
}

// End of a run with a log-structured full: the small level is merged into the
// large one, so full holds the whole relation for reading.
hisa_status Engine::merge_levels() {
  std::vector<Op> ops;
  std::vector<double> before;
  for (int r : idb)
    if (rels[r].log) {
      emit_level_merge(ops, rels[r], true);
      before.push_back(double(hs.cnt[rels[r].full] + hs.cnt[rels[r].l1]));
    }
  if (ops.empty()) return HISA_OK;
  hisa_status s;
  for (int guard = 0; guard < 16; ++guard) {
    if ((s = exec(ops)) || (s = download())) return s;
    if (hs.error) return ctx_fail(HISA_ERR_CUDA, "device error", "level merge");
    if (!hs.overflow) {
      for (double n : before) kstat[kKSetop].bytes += 2.0 * n * (wide ? 8.0 : 4.0);
      return HISA_OK;
    }
    if ((s = regrow()) || (s = upload())) return s;
  }
  return ctx_fail(HISA_ERR_OOM, "buffers keep overflowing", "level merge");
}

// An append-only full with kMaxLevels levels: sort it (its levels are
// disjoint, so the sort leaves it duplicate-free) and index it as one level.
hisa_status Engine::compact_levels() {
  hisa_status s;
  for (int r : idb) {
    Relation& R = rels[r];
    if (!R.append || hs.cnt[R.nlv] <= 1) continue;
    const uint64_t n = hs.cnt[R.full];
    const int kt = wide ? radix_tile<uint64_t>() : radix_tile<uint32_t>();
    if ((s = ensure(R.full_next, n)) || (s = ensure(sc.radix_status, (n / kt + 2) * kRadixDigits))) return s;
    if ((s = upload())) return s;
    std::vector<Op> ops;
    Op z{};
    z.kind = Op::CTL;
    z.ctl.st = dst;
    z.ctl.cmd[z.ctl.n++] = {kCtlZeroSmall, sc.hist, 8 * 256, 0};
    ops.push_back(z);
    Op h{};
    h.kind = Op::HIST;
    h.hist = RadixHistArgs{dst, R.full, R.full, sc.hist, passes, 0};
    ops.push_back(h);
    emit_sort(ops, R.full, R.full_next, R.full, sc.hist, 0, 0);
    if (passes & 1) {
      Op w{};
      w.kind = Op::CTL;
      w.ctl.st = dst;
      w.ctl.cmd[w.ctl.n++] = {kCtlSwap, R.full, R.full_next, 0};
      ops.push_back(w);
    }
    Op x{};
    x.kind = Op::INDEX;
    x.index = IndexArgs{dst, R.full, R.full, R.lvidx, b, -1, 0, b};
    ops.push_back(x);
    if ((s = exec(ops)) || (s = download())) return s;
    if (hs.overflow || hs.error) return ctx_fail(HISA_ERR_CUDA, "level merge of an append-only full", nullptr);
    hs.cnt[R.nlv] = 1;
  }
  return upload();
}

// Runs one iteration with `ops` (host-driven) until it commits, growing
// buffers and re-running the overflowed stage as needed.
hisa_status Engine::iterate_once(const std::vector<Op>& ops) {
  hisa_status s;
  bool rerun_all = true;
  for (int guard = 0; guard < 16; ++guard) {
    if (guard == 0 && &ops == &opsN && (cfg.flags & HISA_FLAG_GRAPH) && !(cfg.flags & HISA_FLAG_PHASE_TIMES)) {
      if ((s = launch_once())) return s;
    } else if ((s = exec(rerun_all ? ops : tail))) {
      return s;
    }
    if ((s = download())) return s;
    if (hs.error)
      return ctx_fail(hs.error == kDevTimeout ? HISA_ERR_DEVICE_TIMEOUT : HISA_ERR_CUDA, "device error",
                      hs.error == kDevTimeout ? "bounded wait expired" : "probe limit / bad state");
    if (!hs.overflow) return HISA_OK;
    rerun_all = (hs.overflow & 1) != 0;
    if ((s = regrow()) || (s = upload())) return s;
  }
  return ctx_fail(HISA_ERR_OOM, "buffers keep overflowing", nullptr);
}

hisa_status Engine::launch_graph() {
  // the device-side loop: iterations repeat while DevState::go is set
  if (!graph_exec || graph_stale) {
    hisa_status s = build_graph();
    if (s) return s;
  }
  CU(cudaGraphLaunch(graph_exec, stream));
  return HISA_OK;
}

hisa_status Engine::launch_once() {
  if (!once_exec || once_stale) {
    if (once_exec) {
      cudaGraphExecDestroy(once_exec);
      once_exec = nullptr;
    }
    if (once_graph) {
      cudaGraphDestroy(once_graph);
      once_graph = nullptr;
    }
    cudaStream_t cs;
    CU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaStream_t saved = stream;
    stream = cs;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      stream = saved;
      cudaStreamDestroy(cs);
      return ctx_fail(HISA_ERR_CUDA, "cudaStreamBeginCapture", cudaGetErrorString(e));
    }
    const uint64_t l0 = g_launches;
    hisa_status s = exec(opsN);
    body_kernels = g_launches - l0;
    g_launches = l0;
    e = cudaStreamEndCapture(cs, &once_graph);
    stream = saved;
    cudaStreamDestroy(cs);
    if (s) return s;
    if (e != cudaSuccess) return ctx_fail(HISA_ERR_CUDA, "cudaStreamEndCapture", cudaGetErrorString(e));
    CU(cudaGraphInstantiate(&once_exec, once_graph, 0));
    once_stale = false;
  }
  CU(cudaGraphLaunch(once_exec, stream));
  return HISA_OK;
}

__global__ void k_set_cond(DevState* st, cudaGraphConditionalHandle h) {
  cudaGraphSetConditional(h, st->go ? 1u : 0u);
}

hisa_status Engine::build_graph() {
  if (graph_exec) {
    cudaGraphExecDestroy(graph_exec);
    graph_exec = nullptr;
  }
  if (graph) {
    cudaGraphDestroy(graph);
    graph = nullptr;
  }
  CU(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle handle;
  CU(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  CU(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  cudaStream_t cs;
  CU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaStream_t saved = stream;
  stream = cs;
  cudaError_t e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    stream = saved;
    cudaStreamDestroy(cs);
    return ctx_fail(HISA_ERR_CUDA, "cudaStreamBeginCaptureToGraph", cudaGetErrorString(e));
  }
  const uint64_t l0 = g_launches;
  hisa_status s = exec(opsN);
  k_set_cond<<<1, 1, 0, cs>>>(dst, handle);
  body_kernels = g_launches - l0 + 1;
  g_launches = l0;
  cudaGraph_t captured;
  e = cudaStreamEndCapture(cs, &captured);
  stream = saved;
  cudaStreamDestroy(cs);
  if (s) return s;
  if (e != cudaSuccess) return ctx_fail(HISA_ERR_CUDA, "cudaStreamEndCapture", cudaGetErrorString(e));
  CU(cudaGraphInstantiate(&graph_exec, graph, 0));
  graph_stale = false;
  return HISA_OK;
}

// ---- reading results ----------------------------------------------------------------------

hisa_status Engine::relation_size(uint32_t rid, uint64_t* n) {
  if (rid >= rels.size() || !n) return ctx_fail(HISA_ERR_INVALID_ARG, "relation_size", nullptr);
  const Relation& r = rels[rid];
  if (r.idb) *n = ran ? hs.cnt[r.full] : 0;
  else *n = r.base >= 0 && !edb_dirty ? hs.cnt[r.base] : r.staged;
  return HISA_OK;
}

hisa_status Engine::read_relation(uint32_t rid, uint32_t* const* cols, uint64_t cap, uint64_t* n, int on_device) {
  if (rid >= rels.size() || !cols || !n) return ctx_fail(HISA_ERR_INVALID_ARG, "read_relation", nullptr);
  const Relation& r = rels[rid];
  if (r.base < 0 || (!r.idb && edb_dirty) || (r.idb && !ran))
    return ctx_fail(HISA_ERR_STATE, "relation not evaluated yet", nullptr);
  const uint64_t size = hs.cnt[r.idb ? r.full : r.base];
  *n = size;
  if (cap < size) return ctx_fail(HISA_ERR_CAPACITY, "read_relation: buffer too small", nullptr);
  if (size == 0) return HISA_OK;
  struct ReadGuard {   // the read scratch is in use until this call returns
    bool& f;
    explicit ReadGuard(bool& x) : f(x) { f = true; }
    ~ReadGuard() { f = false; }
  } guard(reading);
  uint32_t* d0 = cols[0];
  uint32_t* d1 = cols[1];
  void *t0 = nullptr, *t1 = nullptr;
  hisa_status s;
  int src = r.idb ? r.full : r.base;
  // a full kept as a bit matrix: its rows written in order, transposed first
  // when stored column-swapped (the row matrix is needed then: no fallback)
  const bool matrix = r.idb && r.mfull && !batched;
  // a batched run's matrix (rows per instance): its rows read out as codes in
  // the stored order, then handled like a sorted full
  const bool bmat = r.idb && r.mfull && batched;
  int codes = r.full;
  if (bmat) {
    if ((s = ensure(sc.gather, size)) ||
        (s = matrix_rows_out(r, 0, 1ull << (b + inst_bits), sc.gather, 0)))
      return s;
    codes = sc.gather;
    hs.cnt[sc.gather] = size;
  }
  if (matrix && (((s = ensure(sc.read_rows, (1ull << b) + 1))) ||
                 (r.order == 1 && (s = ensure(sc.read_m, (1ull << (2 * b)) / 32)))))
    return s;
  // an append-only full stored in declared order: its levels merged by
  // group straight into the columns (k_levels_read), no sort
  const bool levels = r.idb && r.append && !matrix && r.order == 0;
  // stored column-swapped: transposed through a bit matrix over the domain
  // (k_levels_transpose; 2^(2b) bits), no sort
  bool transposed = r.idb && r.append && !matrix && r.order == 1 && b >= 8 && b <= 16;
  if (transposed && (ensure(sc.read_m, (1ull << (2 * b)) / 32) || ensure(sc.read_rows, (1ull << b) + 1))) {
    transposed = false;   // the matrix does not fit (budget): sort instead
    last_error.clear();
  }
  if (r.idb && (r.order == 1 || r.append || bmat) && !levels && !transposed && !matrix) {
    // stored (c1, c0), or as unmerged levels: (exchange the columns and) sort,
    // so the caller gets the lexicographic order of the declared columns
    const int kt = wide ? radix_tile<uint64_t>() : radix_tile<uint32_t>();
    if ((s = ensure(sc.tmp_a, size)) || (s = ensure(sc.tmp_b, size)) ||
        (s = ensure(sc.radix_status, (size / kt + 2) * kRadixDigits)))
      return s;
    if ((s = upload())) return s;
    std::vector<Op> ops;
    if (r.order == 1) {
      Op w{};
      w.kind = Op::SWAP;
      w.swap = SwapArgs{dst, codes, codes, sc.tmp_a, sc.tmp_cnt, b, 0, 0};
      ops.push_back(w);
    } else {
      CU(cudaMemcpyAsync(hs.buf[sc.tmp_a].ptr, hs.buf[codes].ptr, size * (wide ? 8 : 4), cudaMemcpyDeviceToDevice,
                         stream));
      Op c{};
      c.kind = Op::CTL;
      c.ctl.st = dst;
      c.ctl.cmd[c.ctl.n++] = {kCtlSetCnt, sc.tmp_cnt, (long long)size, 0};
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
    if (hs.overflow || hs.error) return ctx_fail(HISA_ERR_CUDA, "read_relation: re-sort", nullptr);
    src = (passes & 1) ? sc.tmp_b : sc.tmp_a;
  }
  // page-locked host columns are written by the decode kernel itself (over
  // the host link, no device staging and no separate copy); pageable ones
  // go through device buffers and a copy
  bool mapped = false;
  if (!on_device) {
    cudaPointerAttributes pa0{}, pa1{};
    if (cudaPointerGetAttributes(&pa0, cols[0]) == cudaSuccess &&
        cudaPointerGetAttributes(&pa1, cols[1]) == cudaSuccess && pa0.type == cudaMemoryTypeHost &&
        pa1.type == cudaMemoryTypeHost && pa0.devicePointer && pa1.devicePointer) {
      // the row emit of a transposed read writes the host link slower than
      // the copy engine does: stage in device memory (kept for the next
      // read) when it fits
      if ((transposed || matrix) && ensure(sc.read_s0, size) == HISA_OK && ensure(sc.read_s1, size) == HISA_OK) {
        d0 = static_cast<uint32_t*>(hs.buf[sc.read_s0].ptr);
        d1 = static_cast<uint32_t*>(hs.buf[sc.read_s1].ptr);
      } else {
        last_error.clear();
        d0 = static_cast<uint32_t*>(pa0.devicePointer);
        d1 = static_cast<uint32_t*>(pa1.devicePointer);
        mapped = true;
      }
    } else {
      cudaGetLastError();
      if ((s = dev_alloc(size * 4, &t0)) || (s = dev_alloc(size * 4, &t1))) return s;
      d0 = static_cast<uint32_t*>(t0);
      d1 = static_cast<uint32_t*>(t1);
    }
  }
  if (matrix) {
    uint32_t* fbm = static_cast<uint32_t*>(hs.buf[r.fbm].ptr);
    uint32_t* m = r.order == 1 ? static_cast<uint32_t*>(hs.buf[sc.read_m].ptr) : fbm;
    LevelsTransposeArgs ta{dst, -1, -1, -1, b, m, static_cast<uint64_t*>(hs.buf[sc.read_rows].ptr), d0, d1};
    MatrixTransposeArgs mt{fbm, m, b};
    if (wide) launch_matrix_read<uint64_t>(mt, ta, r.order == 1, grid, stream);
    else launch_matrix_read<uint32_t>(mt, ta, r.order == 1, grid, stream);
  } else if (transposed) {
    LevelsTransposeArgs ta{dst, r.full, r.lvidx, r.nlv, b, static_cast<uint32_t*>(hs.buf[sc.read_m].ptr),
                           static_cast<uint64_t*>(hs.buf[sc.read_rows].ptr), d0, d1};
    if (wide) launch_levels_transpose<uint64_t>(ta, grid, stream);
    else launch_levels_transpose<uint32_t>(ta, grid, stream);
  } else if (levels) {
    LevelsReadArgs la{dst, r.full, r.lvidx, r.nlv, b, d0, d1};
    if (wide) launch_levels_read<uint64_t>(la, grid, stream);
    else launch_levels_read<uint32_t>(la, grid, stream);
  } else {
    DecodeArgs a{dst, src, 0, d0, d1, b, 0, 0, size};
    if (wide) launch_decode<uint64_t>(a, grid, stream);
    else launch_decode<uint32_t>(a, grid, stream);
  }
  if ((s = check_launch("decode"))) return s;
  if (!on_device && !mapped) {
    CU(cudaMemcpyAsync(cols[0], d0, size * 4, cudaMemcpyDeviceToHost, stream));
    CU(cudaMemcpyAsync(cols[1], d1, size * 4, cudaMemcpyDeviceToHost, stream));
    dev_free(t0);
    dev_free(t1);
  }
  CU(cudaStreamSynchronize(stream));
  return HISA_OK;
}

hisa_status Engine::delta_counts(uint32_t rid, uint64_t* out, uint32_t cap, uint32_t* n_iters) {
  if (rid >= rels.size() || !n_iters) return ctx_fail(HISA_ERR_INVALID_ARG, "delta_counts", nullptr);
  const Relation& r = rels[rid];
  if (!r.idb) return ctx_fail(HISA_ERR_INVALID_ARG, "delta_counts of an EDB relation", nullptr);
  const uint32_t K = uint32_t(r.delta_counts.size());
  *n_iters = K;
  for (uint32_t i = 0; i < K && i < cap && out; ++i) out[i] = r.delta_counts[i];
  if (cap < K) return ctx_fail(HISA_ERR_CAPACITY, "delta_counts: buffer too small", nullptr);
  return HISA_OK;
}

__global__ void k_max2(const uint32_t* a, const uint32_t* b, uint64_t n, uint32_t* out) {
  uint32_t m = 0;
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x)
    m = max(m, max(a[i], b[i]));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

hisa_status Engine::device_max(const uint32_t* a, const uint32_t* b2, uint64_t n, uint32_t* mx) {
  void* p;
  hisa_status s = dev_alloc(4, &p);
  if (s) return s;
  CU(cudaMemsetAsync(p, 0, 4, stream));
  k_max2<<<grid.small, 256, 0, stream>>>(a, b2, n, static_cast<uint32_t*>(p));
  if ((s = check_launch("max"))) return s;
  CU(cudaMemcpyAsync(hs_pinned, p, 4, cudaMemcpyDeviceToHost, stream));
  CU(cudaStreamSynchronize(stream));
  std::memcpy(mx, hs_pinned, 4);
  dev_free(p);
  return HISA_OK;
}

}  // namespace hisa

namespace hisa {

hisa_status Engine::kernel_stats(hisa_kernel_stat* out, uint32_t cap, uint32_t* n) {
  if (!n) return ctx_fail(HISA_ERR_INVALID_ARG, "kernel_stats", nullptr);
  uint32_t k = 0;
  for (int i = 0; i < kKindCount; ++i) {
    if (!kstat[i].launches) continue;
    if (out && k < cap) {
      hisa_kernel_stat& o = out[k];
      std::memset(&o, 0, sizeof o);
      std::snprintf(o.name, sizeof o.name, "%s", kKernelNames[i]);
      o.launches = kstat[i].launches;
      o.ms = kstat[i].ms;
      o.bytes = kstat[i].bytes;
    }
    ++k;
  }
  *n = k;
  if (out && cap < k) return ctx_fail(HISA_ERR_CAPACITY, "kernel_stats: buffer too small", nullptr);
  return HISA_OK;
}

}  // namespace hisa
