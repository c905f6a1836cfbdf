"""Two-dimensional random circuits and their compilation onto a 1D MPS path
(App. A of arXiv:2312.02667: RQC-2D, the ABCD pattern, recompilation of the C
and D layers with SWAP gates).

Input preparation only: this module builds gate lists; it holds no step of
pTEBD itself.

Lattice qubit (x, y), 0 <= x < Lx, 0 <= y < Ly.  Physical layers follow the
pattern A B C D A B C D ...:
  A: pairs (x, y)-(x, y+1) with y even,   B: the same with y odd,
  C: pairs (x, y)-(x+1, y) with x even,   D: the same with x odd,
with no gate on an edge qubit that has no partner (odd Lx or Ly).  Every pair
gets a Haar-random U(4) (the single-qubit gates of RQC-2D are absorbed), acting
as U[(2 s' + t'), (2 s + t)] with s the first qubit of the pair ((x, y) above).

MPS path: column by column, position(x, y) = x * Ly + y, so A and B gates act
on neighbouring path sites.  A C layer and the D layer after it are compiled
together into 3 (Ly - 1) + 2 layers of nearest-neighbour gates, the compiled
depth the paper states:
  1. Ly - 1 layers of SWAPs interleave each column pair (x, x+1), x even, so
     that (x, y) and (x+1, y) become neighbours;
  2. the C gates;
  3. Ly - 1 layers of SWAPs regroup the qubits so that the D pairs are
     neighbours (column 0 back in front, (x, x+1) interleaved for x odd);
  4. the D gates;
  5. Ly - 1 layers of SWAPs restore the column order.
The SWAP networks are odd-even transposition networks towards the target
order (empty layers dropped); each one takes exactly Ly - 1 layers.
"""
from __future__ import annotations

import numpy as np

from .inputs import _rng, haar_u4

__all__ = ["position", "physical_layers", "compile_layers", "compiled_depth", "SWAP"]

SWAP = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)


def position(lx: int, ly: int) -> dict:
    """Path position of every lattice qubit."""
    return {(x, y): x * ly + y for x in range(lx) for y in range(ly)}


def _pairs(kind: str, lx: int, ly: int) -> list:
    if kind in "AB":
        y0 = 0 if kind == "A" else 1
        return [((x, y), (x, y + 1)) for x in range(lx) for y in range(y0, ly - 1, 2)]
    x0 = 0 if kind == "C" else 1
    return [((x, y), (x + 1, y)) for x in range(x0, lx - 1, 2) for y in range(ly)]


def physical_layers(seed: int, lx: int, ly: int, depth: int):
    """[(kind, [(q1, q2, U), ...]), ...] for `depth` physical layers (a
    multiple of 4) of the ABCD pattern with Haar-random U(4) gates."""
    if depth % 4:
        raise ValueError("the ABCD pattern needs a depth that is a multiple of 4")
    out = []
    for l in range(depth):
        kind = "ABCD"[l % 4]
        rng = _rng(seed, 0x2D, lx, ly, l)
        out.append((kind, [(q1, q2, haar_u4(rng)) for q1, q2 in _pairs(kind, lx, ly)]))
    return out


def _layout_base(lx, ly):
    return [(x, y) for x in range(lx) for y in range(ly)]


def _layout_interleaved(lx, ly, first):
    """Columns (x, x+1) interleaved for x = first, first + 2, ...; others whole."""
    out = []
    x = 0
    while x < lx:
        if x >= first and (x - first) % 2 == 0 and x + 1 < lx:
            for y in range(ly):
                out += [(x, y), (x + 1, y)]
            x += 2
        else:
            out += [(x, y) for y in range(ly)]
            x += 1
    return out


def _transposition_network(start: list, target: list) -> list:
    """Layers of adjacent swaps (odd-even transposition towards `target`,
    empty layers dropped, the starting parity with fewer layers)."""
    tpos = {q: i for i, q in enumerate(target)}
    best = None
    for p0 in (0, 1):
        arr = list(start)
        parity, layers, idle = p0, [], 0
        while any(tpos[q] != i for i, q in enumerate(arr)):
            sw = []
            for i in range(parity, len(arr) - 1, 2):
                if tpos[arr[i]] > tpos[arr[i + 1]]:
                    arr[i], arr[i + 1] = arr[i + 1], arr[i]
                    sw.append(i)
            if sw:
                layers.append(sw)
                idle = 0
            else:
                idle += 1
                if idle > 2:
                    layers = None
                    break
            parity ^= 1
        if layers is not None and (best is None or len(layers) < len(best)):
            best = layers
    return best


def _gate_layer(arr: list, gates) -> tuple:
    """Bonds and oriented gates of one layer of neighbour gates."""
    where = {q: i for i, q in enumerate(arr)}
    bonds, us = [], []
    for q1, q2, u in gates:
        p1, p2 = where[q1], where[q2]
        if abs(p1 - p2) != 1:
            raise RuntimeError(f"{q1} and {q2} are not neighbours on the path")
        bonds.append(min(p1, p2))
        us.append(u if p1 < p2 else SWAP @ u @ SWAP)
    order = np.argsort(bonds)
    return [int(bonds[i]) for i in order], np.stack([us[i] for i in order]) if us else np.zeros((0, 4, 4), complex)


def compile_layers(lx: int, ly: int, layers) -> list:
    """Compiled layers [(bonds, gates[n,4,4]), ...] on path positions.  The
    qubit order on the path is the column order before and after every
    compiled C/D block."""
    out = []
    base = _layout_base(lx, ly)
    i = 0
    while i < len(layers):
        kind, gates = layers[i]
        if kind in "AB":
            out.append(_gate_layer(base, gates))
            i += 1
            continue
        if kind != "C" or i + 1 >= len(layers) or layers[i + 1][0] != "D":
            raise ValueError("a C layer must be followed by a D layer")
        cint = _layout_interleaved(lx, ly, 0)
        dint = _layout_interleaved(lx, ly, 1)
        arr = list(base)
        for target, g in ((cint, gates), (dint, layers[i + 1][1])):
            for sw in _transposition_network(arr, target):
                for p in sw:
                    arr[p], arr[p + 1] = arr[p + 1], arr[p]
                out.append((list(sw), np.stack([SWAP] * len(sw))))
            out.append(_gate_layer(arr, g))
        for sw in _transposition_network(arr, base):
            for p in sw:
                arr[p], arr[p + 1] = arr[p + 1], arr[p]
            out.append((list(sw), np.stack([SWAP] * len(sw))))
        assert arr == base
        i += 2
    return out


def compiled_depth(lx: int, ly: int, physical_depth: int) -> int:
    """Number of compiled layers for `physical_depth` layers of ABCD."""
    cd_pairs = physical_depth // 4
    ab = physical_depth - 2 * cd_pairs
    per_pair = sum(1 for _ in compile_layers(lx, ly, [("C", []), ("D", [])]))
    return ab + cd_pairs * per_pair
