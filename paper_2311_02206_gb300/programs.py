"""The Datalog programs evaluated by the engine, its tests and the benchmark.

Plain data only: ``relations`` maps a relation name to ``"edb"`` (loaded) or
``"idb"`` (derived); ``rules`` is a list of ``(head, body, neq)`` where
``head`` and each body atom are ``(relation, (var, var))`` and ``neq`` lists
pairs of variables that must differ.  Nothing here evaluates anything: the
CUDA engine (through ``hisa.Context.program``) and the CPU oracle both read
these texts, as they both read the seeded EDB generators of ``workloads``.
"""

# REACH, Section 1: Reach(from,to) <- Edge(from,to); Reach(from,to) <- Edge(from,mid), Reach(mid,to).
REACH = (
    {"Edge": "edb", "Reach": "idb"},
    [
        (("Reach", ("f", "t")), [("Edge", ("f", "t"))], []),
        (("Reach", ("f", "t")), [("Edge", ("f", "m")), ("Reach", ("m", "t"))], []),
    ],
)

# SG, Section 2: both rules carry x != y.
SG = (
    {"Edge": "edb", "SG": "idb"},
    [
        (("SG", ("x", "y")), [("Edge", ("p", "x")), ("Edge", ("p", "y"))], [("x", "y")]),
        (("SG", ("x", "y")), [("Edge", ("a", "x")), ("SG", ("a", "b")), ("Edge", ("b", "y"))], [("x", "y")]),
    ],
)

# SG as the workload description prints it: the filter on the first rule only
# (on a DAG whose nodes have several parents, rule 2 then also derives SG(x,x)).
SG_LITERAL = (
    {"Edge": "edb", "SG": "idb"},
    [
        (("SG", ("x", "y")), [("Edge", ("p", "x")), ("Edge", ("p", "y"))], [("x", "y")]),
        (("SG", ("x", "y")), [("Edge", ("a", "x")), ("SG", ("a", "b")), ("Edge", ("b", "y"))], []),
    ],
)


# A context-sensitive points-to style program over Assign / Dereference (written
# for this project; the paper elides its CSPA query, stating only that five rules
# initialise and five mutually recursive rules propagate, that the first
# recursive rule makes ValueFlow transitive and that the second makes two values
# flowing into the same variable aliases).  ValueFlow(a, b): the value of b flows
# into a; Assign(a, b): a = b; Dereference(a, b): a is the dereference of b.
CSPA = (
    {"Assign": "edb", "Dereference": "edb", "ValueFlow": "idb", "MemoryAlias": "idb", "ValueAlias": "idb"},
    [
        (("ValueFlow", ("y", "x")), [("Assign", ("y", "x"))], []),
        (("ValueFlow", ("x", "x")), [("Assign", ("x", "y"))], []),
        (("ValueFlow", ("x", "x")), [("Assign", ("y", "x"))], []),
        (("MemoryAlias", ("x", "x")), [("Assign", ("y", "x"))], []),
        (("MemoryAlias", ("x", "x")), [("Assign", ("x", "y"))], []),
        (("ValueFlow", ("x", "y")), [("ValueFlow", ("x", "z")), ("ValueFlow", ("z", "y"))], []),
        (("ValueAlias", ("x", "y")), [("ValueFlow", ("z", "x")), ("ValueFlow", ("z", "y"))], []),
        (("ValueFlow", ("x", "y")), [("Assign", ("x", "z")), ("MemoryAlias", ("z", "y"))], []),
        (("MemoryAlias", ("x", "w")), [("Dereference", ("y", "x")), ("ValueAlias", ("y", "z")),
                                       ("Dereference", ("z", "w"))], []),
        (("ValueAlias", ("x", "y")), [("ValueFlow", ("z", "x")), ("MemoryAlias", ("z", "w")),
                                      ("ValueFlow", ("w", "y"))], []),
    ],
)
