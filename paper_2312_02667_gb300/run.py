"""Run one of the paper's circuits through the GPU library and print one JSON
line per layer (arXiv:2312.02667, Algorithm 1 with the IPMC).

    python -m paper_2312_02667_gb300.run --family rqc1d --n 101 --depth 200 --chi 64
    python -m paper_2312_02667_gb300.run --family rqc2d --lx 12 --ly 12 --depth 40 --chi 32 --g 1

Each line: layer index, the bonds it gated, the running sums of the discarded
weights (gated bonds and tSU steps) and of ln nu, the largest bond dimension,
and the wall time of the layer (synchronised).  With --norm-every k the
stabilised norm n* (full contraction) and n = n* / prod nu are added every k
layers.  A final line gives the totals; --samples draws bit strings from the
final state (after ptebd_canonicalize when --canonicalize is given).
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np


def build_layers(args):
    from . import circuits, circuits2d, inputs
    fam = args.family
    if fam == "haar1d":
        return args.n, [(b, g) for _, b, g in inputs.brickwork_circuit(args.seed, args.n, args.depth)]
    if fam == "rqc1d":
        return args.n, [(b, g) for _, b, g in circuits.rqc1d_circuit(args.seed, args.n, args.depth)]
    if fam == "pqc1d":
        return args.n, [(b, g) for _, b, g in circuits.pqc1d_circuit(args.seed, args.n, args.depth)]
    lx, ly = args.lx, args.ly
    if fam == "haar2d":
        phys = circuits2d.physical_layers(args.seed, lx, ly, args.depth)
    elif fam == "rqc2d":
        phys = circuits.fuse_2d(circuits.rqc2d_physical(args.seed, lx, ly, args.depth), lx, ly)
    elif fam == "pqc2d":
        phys = circuits.fuse_2d(circuits.pqc2d_physical(args.seed, lx, ly, args.depth), lx, ly)
    else:
        raise SystemExit(f"unknown family {fam}")
    return lx * ly, circuits2d.compile_layers(lx, ly, phys)


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("--family", default="rqc1d", choices=["haar1d", "rqc1d", "pqc1d", "haar2d", "rqc2d", "pqc2d"])
    p.add_argument("--n", type=int, default=101, help="qubits (1D families)")
    p.add_argument("--lx", type=int, default=6)
    p.add_argument("--ly", type=int, default=6)
    p.add_argument("--depth", type=int, default=20, help="physical layers")
    p.add_argument("--chi", type=int, default=64)
    p.add_argument("--g", type=int, default=0, help="PtSU steps after every layer")
    p.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    p.add_argument("--cutoff", type=float, default=1e-12)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--norm-every", type=int, default=0)
    p.add_argument("--canonicalize", action="store_true")
    p.add_argument("--samples", type=int, default=0)
    args = p.parse_args(argv)

    from . import ptebd
    n, layers = build_layers(args)
    st = ptebd.State(n, args.chi, args.precision, cutoff=args.cutoff, g=args.g)
    out = sys.stdout
    t_all = time.perf_counter()
    for i, (bonds, gates) in enumerate(layers):
        t0 = time.perf_counter()
        st.apply_bonds(bonds, gates)
        st.sync()
        dt = time.perf_counter() - t0
        eps, lognu = st.trunc_error()
        row = {"layer": i, "gated": len(bonds), "eps_total": eps, "log_nu_total": lognu,
               "max_chi": int(np.max(st.chi())), "ms": 1e3 * dt}
        if args.norm_every and ((i + 1) % args.norm_every == 0 or i + 1 == len(layers)):
            n_star = st.norm()
            row["n_star"] = n_star
            row["n"] = n_star * float(np.exp(-lognu))
        out.write(json.dumps(row) + "\n")
    total = {"family": args.family, "qubits": n, "layers": len(layers), "chi_max": args.chi, "g": args.g,
             "precision": args.precision, "wall_s": time.perf_counter() - t_all}
    eps, lognu = st.trunc_error()
    total.update({"eps_total": eps, "log_nu_total": lognu, "n_star": st.norm()})
    if args.canonicalize:
        st.canonicalize()
        total["canonicalized"] = True
    if args.samples:
        rng = np.random.default_rng(args.seed)
        bits = st.sample(rng.random((args.samples, n)))
        total["samples"] = ["".join(str(int(b)) for b in row) for row in bits[: min(8, args.samples)]]
        total["mean_bit"] = float(bits.mean())
    out.write(json.dumps(total) + "\n")


if __name__ == "__main__":
    main()
