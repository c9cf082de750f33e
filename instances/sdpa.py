"""SDPA sparse text format ("dat-s") for the problem data, with a content hash.

The format (the input format of the SDPA family, to which the paper's SDPA-C belongs):

    "comment lines start with a double quote or an asterisk
    m                      number of constraint matrices F_1..F_m
    nBlock                 number of diagonal blocks
    s_1 s_2 ...            block sizes; a negative size -k is a diagonal (LP) block of order k
    c_1 ... c_m
    k b i j v              entry (i, j), i <= j, 1-based, of block b of F_k (k = 0..m)

Punctuation `{ } ( ) ,` between numbers is ignored.  SDPA's pair is

    (SDPA primal) min c^T x  s.t.  sum_k F_k x_k - F_0 psd,
    (SDPA dual)   max F_0 . Y  s.t.  F_k . Y = c_k,  Y psd,

and the SDPA dual is the paper's (P) (Sec. 1) with A_0 = -F_0, A_k = F_k, b = c (the library's
`form = 0` applies the same map); the optima differ in sign.  Several blocks are placed on the
diagonal of one matrix of order sum |s_b| (a diagonal block contributes its diagonal entries), so
E splits along the blocks.  Reading and writing only move numbers; nothing of the method is
computed here.
"""
import hashlib
import re

import numpy as np

from .problems import _pack

_SEP = re.compile(r"[{}(),]")


def to_text(inst):
    """The instance as one SDPA block of order n: F_0 = -A_0, F_k = A_k, c = b."""
    lines = ['"' + inst.name, str(inst.m), "1", str(inst.n),
             " ".join(repr(float(x)) for x in inst.b)]
    for k, i, j, v in zip(inst.mat, inst.row, inst.col, inst.val):
        fv = -float(v) if k == 0 else float(v)
        lines.append(f"{int(k)} 1 {int(i) + 1} {int(j) + 1} {fv!r}")
    return "\n".join(lines) + "\n"


def content_hash(text):
    return hashlib.sha256(text.encode("utf-8")).hexdigest()


def write(inst, path):
    """Write the instance; returns the SHA-256 of the file's bytes."""
    text = to_text(inst)
    with open(path, "w", encoding="utf-8") as f:
        f.write(text)
    return content_hash(text)


def parse(text, name="sdpa"):
    """An SDPInstance (paper notation) from SDPA sparse text.  Raises ValueError on malformed
    input, on a duplicate (k, block, i, j) and on an off-diagonal entry of a diagonal block."""
    toks = []
    for line in text.splitlines():
        s = line.strip()
        if not s or s[0] in "\"*":
            continue
        toks.append(_SEP.sub(" ", s).split())
    if len(toks) < 4:
        raise ValueError("SDPA text: header incomplete")
    m = int(toks[0][0])
    nblock = int(toks[1][0])
    sizes = [int(float(x)) for x in toks[2]]
    if len(sizes) != nblock or m < 1 or any(s == 0 for s in sizes):
        raise ValueError("SDPA text: bad m, nBlock or block sizes")
    # c may wrap over several lines: take numbers until m are read
    c, r = [], 3
    while len(c) < m:
        if r >= len(toks):
            raise ValueError("SDPA text: c has fewer than m entries")
        c.extend(float(x) for x in toks[r])
        r += 1
    if len(c) != m:
        raise ValueError("SDPA text: c has more than m entries")
    offs = np.concatenate([[0], np.cumsum([abs(s) for s in sizes])]).astype(int)
    n = int(offs[-1])
    ent = {}
    for t in toks[r:]:
        if len(t) != 5:
            raise ValueError(f"SDPA text: entry line {' '.join(t)!r} does not have 5 fields")
        k, b, i, j = (int(x) for x in t[:4])
        v = float(t[4])
        if not (0 <= k <= m and 1 <= b <= nblock):
            raise ValueError(f"SDPA text: matrix {k} or block {b} out of range")
        sz = abs(sizes[b - 1])
        if not (1 <= i <= sz and 1 <= j <= sz):
            raise ValueError(f"SDPA text: index ({i}, {j}) outside block {b} of order {sz}")
        if sizes[b - 1] < 0 and i != j:
            raise ValueError(f"SDPA text: off-diagonal entry in diagonal block {b}")
        i, j = min(i, j), max(i, j)
        key = (k, int(offs[b - 1]) + i - 1, int(offs[b - 1]) + j - 1)
        if key in ent:
            raise ValueError(f"SDPA text: duplicate entry (matrix {k}, block {b}, {i}, {j})")
        ent[key] = -v if k == 0 else v
    return _pack(name, n, m, np.array(c), ent,
                 meta={"kind": "sdpa", "block_sizes": sizes, "block_offsets": offs.tolist()})


def read(path, name=None):
    """(instance, SHA-256 of the file's bytes)."""
    with open(path, "r", encoding="utf-8") as f:
        text = f.read()
    return parse(text, name or path), content_hash(text)


NAMED = ("grid_maxcut_100", "block_arrow_2020", "block_arrow_1020", "ring_maxcut_20000")


def main(argv=None):
    """python -m instances.sdpa DIR [NAME ...]: writes the named workloads as DIR/NAME.dat-s and
    prints `sha256  NAME.dat-s` lines (the format of instances/workloads.sha256)."""
    import os
    import sys
    from .problems import workload
    args = sys.argv[1:] if argv is None else argv
    if not args:
        print(main.__doc__)
        return 2
    out, names = args[0], args[1:] or NAMED
    os.makedirs(out, exist_ok=True)
    for nm in names:
        h = write(workload(nm), os.path.join(out, nm + ".dat-s"))
        print(f"{h}  {nm}.dat-s")
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
