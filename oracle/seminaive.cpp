// CPU oracle: plain semi-naive Datalog evaluation over std::set.
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
// cpu_baseline / reference legs of bench.py may load this library.  It shares
// no code, header, table or helper with the CUDA path.
//
// What it computes (Section 2, "Semi-naive evaluation"; Section 5.1 and its
// evaluation-workflow figure):
//   * every relation has the versions full, delta and new;
//   * iteration 1 evaluates the rules whose body names no IDB relation
//     (their output is the first delta);
//   * iteration k >= 2 evaluates every rule whose body names an IDB relation,
//     once per IDB body atom i, with atom i read from delta_{k-1} and every
//     other atom read from full_{k-1} (which already holds delta_{k-1});
//     all rules read the same snapshot, merges happen after all rules ran;
//   * delta_k = new \ full_{k-1}  ("populating delta": a set difference);
//     full_k = full_{k-1} U delta_k ("merge full/delta"); new is cleared;
//   * stop when every delta is empty (the fixpoint).
// A body is evaluated as a nested-loop join: the delta atom is scanned first
// (the outer relation of Algorithm 3), every later atom is range-queried on its
// already-bound columns (the inner relation), atoms sharing a bound variable
// taken first.  Filters x != y are checked on
// the complete binding.  Relations are sets: loading drops duplicate tuples.
//
// Delta-count convention: counts[k-1] = |delta_k| for k = 1..K, where K is the
// last iteration in which some relation gained a tuple; iteration K+1 runs and
// finds nothing.
#ifndef ORACLE_PLANT
#define ORACLE_PLANT 0
#endif
#include <cstdint>
#include <cstring>
#include <set>
#include <utility>
#include <vector>

namespace {

using Tup = std::pair<uint32_t, uint32_t>;
using TupSet = std::set<Tup>;

struct Rel {
  bool idb = false;
  TupSet full, full_rev;    // full_rev holds (c1, c0) for lookups on column 1
  TupSet delta, delta_rev;
  TupSet fresh;             // "new"
  std::vector<uint64_t> counts;
};

struct Atom { int rel; int var[2]; };
struct Rule {
  Atom head;
  std::vector<Atom> body;
  std::vector<std::pair<int, int>> neq;
};

enum { kMaxVars = 16 };

struct Program {
  std::vector<Rel> rels;
  std::vector<Rule> rules;
  int iterations_run = 0;
};

struct Binding { int64_t v[kMaxVars]; };

// Evaluate body atoms order[pos..] under binding b; atom order[0] is the scanned
// (outer) atom.  use_delta[j] selects delta instead of full for body atom j.
void eval_atoms(Program& P, const Rule& R, const std::vector<int>& order,
                const std::vector<bool>& use_delta, size_t pos, Binding& b) {
  if (pos == order.size()) {
#if ORACLE_PLANT != 3  // planted mistake 3: filters ignored
    for (auto& f : R.neq)
      if (b.v[f.first] == b.v[f.second]) return;
#endif
#if ORACLE_PLANT == 2  // planted mistake: head columns swapped
    Tup out{(uint32_t)b.v[R.head.var[1]], (uint32_t)b.v[R.head.var[0]]};
#else
    Tup out{(uint32_t)b.v[R.head.var[0]], (uint32_t)b.v[R.head.var[1]]};
#endif
    P.rels[R.head.rel].fresh.insert(out);
    return;
  }
  const int j = order[pos];
  const Atom& A = R.body[j];
  Rel& rel = P.rels[A.rel];
  const TupSet& fwd = use_delta[j] ? rel.delta : rel.full;
  const TupSet& rev = use_delta[j] ? rel.delta_rev : rel.full_rev;
  const int x = A.var[0], y = A.var[1];
  const bool bx = b.v[x] >= 0, by = b.v[y] >= 0;

  auto visit = [&](uint32_t c0, uint32_t c1) {
    // bind, checking repeated variables and earlier bindings
    Binding nb = b;
    if (nb.v[x] >= 0 && nb.v[x] != (int64_t)c0) return;
    nb.v[x] = c0;
    if (nb.v[y] >= 0 && nb.v[y] != (int64_t)c1) return;
    nb.v[y] = c1;
    eval_atoms(P, R, order, use_delta, pos + 1, nb);
  };

  if (bx) {
    const uint32_t k = (uint32_t)b.v[x];
    for (auto it = fwd.lower_bound({k, 0u}); it != fwd.end() && it->first == k; ++it)
      visit(it->first, it->second);
  } else if (by) {
    const uint32_t k = (uint32_t)b.v[y];
    for (auto it = rev.lower_bound({k, 0u}); it != rev.end() && it->first == k; ++it)
      visit(it->second, it->first);
  } else {
    for (auto& t : fwd) visit(t.first, t.second);
  }
}

// Atom order: the delta atom (else the first atom) is scanned; each further
// position takes the first remaining atom that shares a variable already bound,
// so it is range-queried rather than scanned (the order changes the cost, not
// the set of bindings).
void eval_rule(Program& P, const Rule& R, int delta_atom) {
  const int nb = (int)R.body.size();
  std::vector<int> order;
  std::vector<bool> use_delta(nb, false), used(nb, false);
  bool bound[kMaxVars] = {};
  auto take = [&](int j) {
    order.push_back(j);
    used[j] = true;
    bound[R.body[j].var[0]] = bound[R.body[j].var[1]] = true;
  };
  if (delta_atom >= 0) {
    use_delta[delta_atom] = true;
    take(delta_atom);
  }
  while ((int)order.size() < nb) {
    int pick = -1;
    for (int j = 0; j < nb && pick < 0; ++j)
      if (!used[j] && (bound[R.body[j].var[0]] || bound[R.body[j].var[1]])) pick = j;
    for (int j = 0; j < nb && pick < 0; ++j)
      if (!used[j]) pick = j;
    take(pick);
  }
  Binding b;
  for (auto& v : b.v) v = -1;
  eval_atoms(P, R, order, use_delta, 0, b);
}

bool rule_is_recursive(const Program& P, const Rule& R) {
  for (auto& a : R.body)
    if (P.rels[a.rel].idb) return true;
  return false;
}

// Populate delta (set difference), merge into full, clear new.  Returns true if
// some relation gained a tuple.
bool finish_iteration(Program& P) {
  bool any = false;
  for (auto& r : P.rels) {
    if (!r.idb) continue;
    r.delta.clear();
    r.delta_rev.clear();
    for (auto& t : r.fresh)
#if ORACLE_PLANT == 1  // planted mistake: no set difference against full
      r.delta.insert(t);
#else
      if (!r.full.count(t)) r.delta.insert(t);
#endif
    for (auto& t : r.delta) {
      r.full.insert(t);
      r.full_rev.insert({t.second, t.first});
      r.delta_rev.insert({t.second, t.first});
    }
#if ORACLE_PLANT == 4  // planted mistake: counts new instead of delta
    r.counts.push_back(r.fresh.size());
#else
    r.counts.push_back(r.delta.size());
#endif
    r.fresh.clear();
    if (!r.delta.empty()) any = true;
  }
  return any;
}

}  // namespace

extern "C" {

void* oracle_new() { return new Program(); }

void oracle_free(void* h) { delete static_cast<Program*>(h); }

int oracle_add_relation(void* h, int is_idb) {
  auto* P = static_cast<Program*>(h);
  P->rels.emplace_back();
  P->rels.back().idb = is_idb != 0;
  return (int)P->rels.size() - 1;
}

int oracle_load(void* h, int rel, const uint32_t* c0, const uint32_t* c1, uint64_t n) {
  auto* P = static_cast<Program*>(h);
  if (rel < 0 || rel >= (int)P->rels.size()) return -1;
  Rel& r = P->rels[rel];
  for (uint64_t i = 0; i < n; ++i) {
    r.full.insert({c0[i], c1[i]});
    r.full_rev.insert({c1[i], c0[i]});
  }
  return 0;
}

// desc: head_rel, hv0, hv1, n_body, (rel, v0, v1) * n_body, n_neq, (a, b) * n_neq
int oracle_add_rule(void* h, const int32_t* d, int len) {
  auto* P = static_cast<Program*>(h);
  Rule R;
  int p = 0;
  auto get = [&](int32_t& out) { if (p >= len) return false; out = d[p++]; return true; };
  int32_t nb, nn, t;
  if (!get(t)) return -1;
  R.head.rel = t;
  if (!get(t)) return -1;
  R.head.var[0] = t;
  if (!get(t)) return -1;
  R.head.var[1] = t;
  if (!get(nb) || nb < 1) return -1;
  for (int i = 0; i < nb; ++i) {
    Atom a;
    if (!get(a.rel) || !get(a.var[0]) || !get(a.var[1])) return -1;
    R.body.push_back(a);
  }
  if (!get(nn)) return -1;
  for (int i = 0; i < nn; ++i) {
    int32_t a, b;
    if (!get(a) || !get(b)) return -1;
    R.neq.push_back({a, b});
  }
  auto okrel = [&](int r) { return r >= 0 && r < (int)P->rels.size(); };
  auto okvar = [&](int v) { return v >= 0 && v < kMaxVars; };
  if (!okrel(R.head.rel) || !P->rels[R.head.rel].idb) return -2;
  for (auto& a : R.body)
    if (!okrel(a.rel) || !okvar(a.var[0]) || !okvar(a.var[1])) return -2;
  for (int hv : R.head.var) {
    bool found = false;
    for (auto& a : R.body) found |= (a.var[0] == hv || a.var[1] == hv);
    if (!okvar(hv) || !found) return -3;  // head variables must be bound by the body
  }
  P->rules.push_back(R);
  return (int)P->rules.size() - 1;
}

// Runs to the fixpoint.  Returns K (the number of iterations that produced a
// tuple) or -1 if max_iters iterations ran without reaching the fixpoint.
int oracle_run(void* h, uint32_t max_iters) {
  auto* P = static_cast<Program*>(h);
  // iteration 1: non-recursive rules
  for (auto& R : P->rules)
    if (!rule_is_recursive(*P, R)) eval_rule(*P, R, -1);
  int k = 1;
  bool any = finish_iteration(*P);
  int last = any ? 1 : 0;
  while (any) {
    if ((uint32_t)k >= max_iters) return -1;
    ++k;
    for (auto& R : P->rules) {
      if (!rule_is_recursive(*P, R)) continue;
      for (int j = 0; j < (int)R.body.size(); ++j) {
        if (!P->rels[R.body[j].rel].idb) continue;
        eval_rule(*P, R, j);
#if ORACLE_PLANT == 5  // planted mistake: only the first IDB atom is ever the delta atom
        break;
#endif
      }
    }
    any = finish_iteration(*P);
    if (any) last = k;
  }
  P->iterations_run = k;
  // trim every relation's history to K entries
  for (auto& r : P->rels)
    if (r.idb) r.counts.resize(last);
  return last;
}

uint64_t oracle_size(void* h, int rel) {
  return static_cast<Program*>(h)->rels[rel].full.size();
}

int oracle_read(void* h, int rel, uint32_t* c0, uint32_t* c1) {
  auto& r = static_cast<Program*>(h)->rels[rel];
  uint64_t i = 0;
  for (auto& t : r.full) {  // std::set order = lexicographic (c0, c1)
    c0[i] = t.first;
    c1[i] = t.second;
    ++i;
  }
  return 0;
}

int oracle_delta_counts(void* h, int rel, uint64_t* out, int cap) {
  auto& r = static_cast<Program*>(h)->rels[rel];
  int n = (int)r.counts.size();
  for (int i = 0; i < n && i < cap; ++i) out[i] = r.counts[i];
  return n;
}

}  // extern "C"
