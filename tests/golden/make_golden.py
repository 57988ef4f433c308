"""Writes the stored expected values under tests/golden/.

Calls only ``oracle.exact`` (mpmath brute force) on inputs from
``dqmc_inputs``; nothing here comes from the CUDA path.

single_n16_mpmath.txt -- 4x4 periodic lattice, t=1, U=4, dtau=0.1, beta=8
(M=80), Hirsch +-1 field of seed 2003_05286*1000 + 100 + 0: the exact
G = [1 + B_80...B_1]^{-1} (Eq. (etgf)) and log|det(1 + B_80...B_1)| with its
sign, from the naive product at the precision oracle.exact.required_dps picks.
First row: logdet, sign; then the 256 entries of G in row-major order.

single_n16_displaced_mpmath.txt -- the same instance: G(tau_l, 0) = B_l...B_1 G_1
and G(0, tau_l) = -(1 - G_1)(B_l...B_1)^{-1} (both cases of Eq. (tdgf_propagate))
for l = 10, 40, 70, from the same naive products.  One block per (function, l):
a header line "t0 <l>" or "0t <l>", then 256 entries row-major.

batch_n64_229_displaced_mpmath.txt -- instance 229 of the 8x8, U=4, beta=40
(M=400) batch (seed 2003_05286*1000 + 200 + 229), an ill-conditioned field
(|G(tau,0)| up to ~1e4): G(tau_l, 0) = B_l...B_1 G_1 for l = 10, 50, 80 from
the naive product at the precision oracle.exact.required_dps picks.  Blocks
"t0 <l>" of 4096 entries row-major.  Slow (minutes): written only with the
argument "n64".

Run from the repository root:  python tests/golden/make_golden.py [n64]
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import dqmc_inputs as di  # noqa: E402
from oracle import exact as ex  # noqa: E402


def main():
    inst = di.single_n16()
    bf = ex.BruteForce(inst.K, inst.dtau, inst.V)
    G, ld, s = bf.greens(1)
    G = bf.to_numpy(G)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "single_n16_mpmath.txt")
    with open(out, "w") as f:
        f.write(f"# mpmath dps={bf.dps}; first row: logdet sign; then G row-major\n")
        f.write(f"{float(ld):.17e} {s:d}\n")
        for v in G.ravel():
            f.write(f"{v:.17e}\n")
    print("wrote", out, "dps", bf.dps)

    mp = bf.mp
    G1 = bf.greens(1)[0]
    one_minus = mp.eye(bf.N) - G1
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                       "single_n16_displaced_mpmath.txt")
    with open(out, "w") as f:
        f.write(f"# mpmath dps={bf.dps}; blocks 't0 l' = G(tau_l, 0), '0t l' = G(0, tau_l)\n")
        for l in (10, 40, 70):
            C = bf.chain(range(1, l + 1))
            for name, A in (("t0", C * G1), ("0t", -(one_minus * mp.inverse(C)))):
                f.write(f"{name} {l}\n")
                for v in bf.to_numpy(A).ravel():
                    f.write(f"{v:.17e}\n")
    print("wrote", out)


def main_n64():
    inst = di.batch_n64_tdisplaced(229)
    bf = ex.BruteForce(inst.K, inst.dtau, inst.V)
    G1 = bf.greens(1)[0]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                       "batch_n64_229_displaced_mpmath.txt")
    with open(out, "w") as f:
        f.write(f"# mpmath dps={bf.dps}; blocks 't0 l' = G(tau_l, 0) of instance 229\n")
        for l in (10, 50, 80):
            A = bf.chain(range(1, l + 1)) * G1
            f.write(f"t0 {l}\n")
            for v in bf.to_numpy(A).ravel():
                f.write(f"{v:.17e}\n")
    print("wrote", out, "dps", bf.dps)


if __name__ == "__main__":
    if len(sys.argv) > 1 and sys.argv[1] == "n64":
        main_n64()
    else:
        main()
