"""Second, independent CPU evaluator: naive iteration of the immediate-consequence
operator, in pure Python sets (tiny inputs only).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  It shares no code with the
semi-naive oracle: every round it re-evaluates every rule on the whole current
database (Section 2: rules are applied until no new fact is derived).  Under the
reading that all rules of one iteration read the same snapshot, the tuples new
in naive round k are exactly semi-naive's delta_k, so this evaluator also pins
the per-iteration delta counts.
"""
from __future__ import annotations


def _matches(body, db, neq):
    """All variable bindings satisfying every atom of ``body`` over ``db``."""
    envs = [{}]
    for rel, (x, y) in body:
        nxt = []
        for env in envs:
            for (a, b) in db[rel]:
                e = dict(env)
                if e.setdefault(x, a) != a:
                    continue
                if e.setdefault(y, b) != b:
                    continue
                nxt.append(e)
        envs = nxt
    return [e for e in envs if all(e[p] != e[q] for p, q in neq)]


def naive(relations: dict, rules: list, edb: dict, max_rounds: int = 10_000):
    """Returns (idb name -> sorted list of tuples, idb name -> delta counts)."""
    db = {name: set() for name in relations}
    for name, (c0, c1) in edb.items():
        db[name] = {(int(a), int(b)) for a, b in zip(c0, c1)}
    counts = {n: [] for n, k in relations.items() if k == "idb"}
    for _ in range(max_rounds):
        derived = {n: set() for n in counts}
        for (hrel, (hx, hy)), body, neq in rules:
            for e in _matches(body, db, neq):
                derived[hrel].add((e[hx], e[hy]))
        fresh = {n: derived[n] - db[n] for n in counts}
        if not any(fresh.values()):
            break
        for n in counts:
            db[n] |= fresh[n]
            counts[n].append(len(fresh[n]))
    else:
        raise RuntimeError("no fixpoint within max_rounds")
    return {n: sorted(db[n]) for n in counts}, counts
