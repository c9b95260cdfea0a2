"""Generate the 5x5 median comparator network used by stage B (median_net.cuh).

The median of step 7 (arXiv 1802.00036, Section IV-7) is taken over every
5x5 window.  A thread computes a block of 2 output rows x BC output columns
from the 6 x (BC + 4) input values under it, sharing work between the
windows of the block:

* vertical: for every input column, the four rows common to both output
  rows are sorted once (5 compare-exchanges), then the top row and the
  bottom row are each inserted, giving the sorted 5-column of each output
  row (insertion of y into sorted w0..w3: out0 = min(w0, y),
  out_i = max(w_{i-1}, min(w_i, y)), out4 = max(w3, y));
* horizontal: the sorted columns of adjacent pairs are merged (Batcher's
  odd-even merge), the two pairs common to two neighbouring outputs are
  merged into the sorted 20 values of their four shared columns, and each
  output's median is the 13th smallest of those 20 and of its fifth sorted
  column, by the selection identity for two sorted lists
  kth(A u B) = min over i + j = k of max(a_i, b_j);
* every min/max whose result no output needs is pruned, and a min (max)
  whose only use is another min (max) is fused into a 3-input min (max),
  which issues at the same rate as the 2-input form on sm_103a.

The network description is verified here (and by the test suite) with the
0-1 principle: a comparator network selects the k-th smallest of its inputs
for all real inputs iff it does so for all 0/1 inputs.  Each output depends
on its own 25 inputs only, so each output is checked on all 2^25 binary
windows.

Run ``python gen_median.py`` to rewrite median_net.cuh.
"""
from __future__ import annotations

import os
import sys

import numpy as np

ROWS = 6          # input rows per block (2 output rows + 2 + 2)


class Net:
    """Straight-line min/max program over wires (SSA)."""

    def __init__(self):
        self.ops = []          # (kind, args...) ; kind in in/min/max/min3/max3
        self.names = {}

    def inp(self, name):
        self.ops.append(("in",))
        self.names[len(self.ops) - 1] = name
        return len(self.ops) - 1

    def op(self, kind, *args):
        self.ops.append((kind,) + tuple(args))
        return len(self.ops) - 1

    def ce(self, a, b):
        return self.op("min", a, b), self.op("max", a, b)


def oe_merge(net, A, B):
    """Batcher's odd-even merge of sorted wire lists A and B."""
    if not A:
        return list(B)
    if not B:
        return list(A)
    if len(A) == 1 and len(B) == 1:
        return list(net.ce(A[0], B[0]))
    E = oe_merge(net, A[0::2], B[0::2])
    O = oe_merge(net, A[1::2], B[1::2])
    res = [E[0]]
    for i in range(max(len(E) - 1, len(O))):
        if i < len(O) and i + 1 < len(E):
            res += list(net.ce(O[i], E[i + 1]))
        elif i < len(O):
            res.append(O[i])
        else:
            res.append(E[i + 1])
    return res


def sort4(net, a, b, c, d):
    """Optimal 4-sorter (5 compare-exchanges)."""
    a, b = net.ce(a, b)
    c, d = net.ce(c, d)
    a, c = net.ce(a, c)
    b, d = net.ce(b, d)
    b, c = net.ce(b, c)
    return [a, b, c, d]


def insert1(net, w, y):
    """Insert y into sorted w (len 4) -> sorted 5."""
    out = [net.op("min", w[0], y)]
    for i in range(1, len(w)):
        out.append(net.op("max", w[i - 1], net.op("min", w[i], y)))
    out.append(net.op("max", w[-1], y))
    return out


def build(BC: int):
    """Network for a 2 x BC output block; inputs x[r][j], r < 6, j < BC + 4."""
    assert BC % 2 == 0 and BC >= 2
    net = Net()
    NC = BC + 4
    x = [[net.inp(f"x[{r}][{j}]") for j in range(NC)] for r in range(ROWS)]
    outs = {}
    for row in range(2):
        pass
    # vertical: sorted 5-columns for output rows 0 (input rows 0..4) and 1 (1..5)
    S = [[None] * NC for _ in range(2)]
    for j in range(NC):
        core = sort4(net, x[1][j], x[2][j], x[3][j], x[4][j])
        S[0][j] = insert1(net, core, x[0][j])
        S[1][j] = insert1(net, core, x[5][j])
    # horizontal, per output row
    for row in range(2):
        pairs = {}

        def P(j):
            if j not in pairs:
                pairs[j] = oe_merge(net, S[row][j], S[row][j + 1])
            return pairs[j]

        for o in range(0, BC, 2):
            core = oe_merge(net, P(o + 1), P(o + 3))        # columns o+1 .. o+4
            for oo, extra in ((o, S[row][o]), (o + 1, S[row][o + 5])):
                terms = [core[12]]
                for j in range(1, 6):
                    terms.append(net.op("max", core[12 - j], extra[j - 1]))
                m = terms[0]
                for t in terms[1:]:
                    m = net.op("min", m, t)
                outs[(row, oo)] = m
    return net, x, outs


def prune_and_fuse(net, outs):
    """Keep only ops that reach an output; fuse single-use min/max chains."""
    need = set(outs.values())
    for i in range(len(net.ops) - 1, -1, -1):
        if i in need and net.ops[i][0] != "in":
            need.update(net.ops[i][1:])
    uses = {}
    for i in sorted(need):
        for a in net.ops[i][1:]:
            uses[a] = uses.get(a, 0) + 1
    out_set = set(outs.values())
    ops = {i: list(net.ops[i]) for i in need}
    fused_away = set()
    for i in sorted(need):
        k = ops[i][0]
        if k not in ("min", "max"):
            continue
        a, b = ops[i][1:]
        # fold one operand that is a single-use 2-input op of the same kind
        for inner, other in ((a, b), (b, a)):
            if (ops[inner][0] == k and uses.get(inner, 0) == 1 and inner not in out_set
                    and inner not in fused_away):
                ops[i] = [k + "3", ops[inner][1], ops[inner][2], other]
                fused_away.add(inner)
                break
    order = [i for i in sorted(need) if i not in fused_away]
    return order, ops


def evaluate_bits(order, ops, inputs_bits, outs_wanted):
    """Evaluate the network on packed 0/1 inputs (numpy uint64 words)."""
    val = dict(inputs_bits)
    for i in order:
        k = ops[i][0]
        if k == "in":
            continue
        a = [val[j] for j in ops[i][1:]]
        if k in ("min", "min3"):
            v = a[0]
            for t in a[1:]:
                v = v & t
        else:
            v = a[0]
            for t in a[1:]:
                v = v | t
        val[i] = v
    return {o: val[o] for o in outs_wanted}


def output_cone(order, ops, wire):
    """The ops (in order) that the output `wire` depends on."""
    need = {wire}
    for i in reversed(order):
        if i in need:
            need.update(ops[i][1:])
    return [i for i in order if i in need]


def verify(BC: int, outputs=None, chunk_bits: int = 20) -> int:
    """0-1 principle, exhaustively, for the chosen outputs of the block (all
    by default).  Each output's cone must read only its own 25 inputs; it is
    then evaluated on all 2^25 binary windows.  Returns windows checked."""
    net, x, outs = build(BC)
    order, ops = prune_and_fuse(net, outs)
    checked = 0
    # bit patterns of the 2^chunk_bits low cases, one packed array per input bit
    low = np.arange(1 << chunk_bits, dtype=np.uint64)
    low_bits = [np.packbits(((low >> np.uint64(b)) & np.uint64(1)).astype(np.uint8),
                            bitorder="little").view(np.uint64) for b in range(chunk_bits)]
    low_pop = sum(((low >> np.uint64(b)) & np.uint64(1)) for b in range(chunk_bits)).astype(np.int64)
    zeros = np.zeros_like(low_bits[0])
    for key, wire in sorted(outs.items()):
        if outputs is not None and key not in outputs:
            continue
        row, o = key
        win = [x[row + dr][o + dc] for dr in range(5) for dc in range(5)]
        cone = output_cone(order, ops, wire)
        reads = {a for i in cone for a in ops[i][1:] if ops[a][0] == "in"}
        assert reads <= set(win), f"output {key} reads outside its window"
        for chunk in range(1 << (25 - chunk_bits)):
            bits = {}
            for b, w in enumerate(win):
                if b < chunk_bits:
                    bits[w] = low_bits[b]
                else:
                    bits[w] = ~zeros if (chunk >> (b - chunk_bits)) & 1 else zeros
            pop = low_pop + bin(chunk).count("1")
            want = np.packbits((pop >= 13).astype(np.uint8), bitorder="little").view(np.uint64)
            got = evaluate_bits(cone, ops, bits, [wire])[wire]
            if not np.array_equal(got, want):
                raise AssertionError(f"median network wrong for output {key}")
            checked += 1 << chunk_bits
    return checked


def count(BC: int):
    net, x, outs = build(BC)
    order, ops = prune_and_fuse(net, outs)
    n = sum(1 for i in order if ops[i][0] != "in")
    return n, n / (2 * BC)


def emit(BC: int) -> str:
    net, x, outs = build(BC)
    order, ops = prune_and_fuse(net, outs)
    lines = []
    NC = BC + 4
    n_ops, per = count(BC)
    lines.append(f"// median of every 5x5 window of a 2 x {BC} output block: {n_ops} min/max")
    lines.append(f"// instructions ({per:.1f} per output).  x[r][j]: input rows r = 0..5")
    lines.append(f"// (output row 0 is input row 2), columns j = 0..{NC - 1} (output column o")
    lines.append("// is input column o + 2); m[row][o]: the medians.")
    lines.append("template <class T, class Ops>")
    lines.append(f"__device__ __forceinline__ void median_block_2x{BC}(const T (&x)[6][{NC}], T (&m)[2][{BC}])")
    lines.append("{")
    name = {}
    for i in order:
        k = ops[i][0]
        if k == "in":
            name[i] = net.names[i]
            continue
        args = ", ".join(name[a] for a in ops[i][1:])
        fn = {"min": "Ops::min2", "max": "Ops::max2", "min3": "Ops::min3", "max3": "Ops::max3"}[k]
        name[i] = f"t{i}"
        lines.append(f"    const T t{i} = {fn}({args});")
    for (row, o), w in sorted(outs.items()):
        lines.append(f"    m[{row}][{o}] = {name[w]};")
    lines.append("}")
    return "\n".join(lines) + "\n"


HEADER = """// median_net.cuh -- GENERATED by gen_median.py; do not edit.
//
// 5x5 median (arXiv 1802.00036, Section IV-7) of a 2-row block of outputs
// as a pruned, shared comparator network (sorted columns, merged pairs and
// quads, two-list selection).  Verified exhaustively with the 0-1 principle
// by gen_median.py and tests/test_median_network.py.
#pragma once

"""


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "median_net.cuh")
    text = HEADER + "\n".join(emit(bc) for bc in (8,))
    with open(out, "w") as fh:
        fh.write(text)
    for bc in (2, 4, 8):
        print("BC", bc, "ops %d, per output %.2f" % count(bc))
    if "--verify" in sys.argv:
        print("checked", verify(8))


if __name__ == "__main__":
    main()
