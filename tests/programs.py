"""Datalog programs used by the oracle pins and the GPU parity tests, beyond
the paper's REACH, SG and the points-to program held by the oracle package."""
import oracle

# non-linear closure: both body atoms are IDB (column 0 and column 1 lookups)
TC_NONLINEAR = ({"E": "edb", "T": "idb"}, [
    (("T", ("x", "y")), [("E", ("x", "y"))], []),
    (("T", ("x", "z")), [("T", ("x", "y")), ("T", ("y", "z"))], []),
])

# mutual recursion over two IDB relations, a column-1 lookup and a filter
MUTUAL = ({"A": "edb", "B": "edb", "P": "idb", "Q": "idb"}, [
    (("P", ("x", "y")), [("A", ("x", "y"))], []),
    (("Q", ("y", "x")), [("B", ("x", "y"))], []),
    (("P", ("x", "z")), [("Q", ("x", "y")), ("P", ("y", "z"))], []),
    (("Q", ("x", "z")), [("P", ("y", "x")), ("B", ("y", "z"))], [("x", "z")]),
    (("Q", ("x", "x")), [("P", ("x", "w")), ("Q", ("w", "v"))], []),
])

# a recursive rule whose head keeps the inner atom's other column first and
# filters x != y (the engine runs it as an inverted grouped bitmap join with
# its filter over small domains), and a rule reading R's delta on its second
# column
INVERTED = ({"E": "edb", "R": "idb", "S": "idb"}, [
    (("R", ("x", "y")), [("E", ("x", "y"))], []),
    (("R", ("x", "y")), [("E", ("x", "z")), ("R", ("z", "y"))], [("x", "y")]),
    (("S", ("x", "y")), [("R", ("x", "z")), ("E", ("z", "y"))], []),
])

PROGRAMS = {
    "reach": oracle.REACH,
    "sg": oracle.SG,
    "tc_nonlinear": TC_NONLINEAR,
    "mutual": MUTUAL,
    "inverted": INVERTED,
}
