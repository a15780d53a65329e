"""Write the stored expected values of tests/golden/ from the oracle alone.

    python tests/golden/make_golden.py

* cbc_s100_m10.txt: the CBC generating vector (Sec. 3.2 cites Nuyens-Cools;
  reading A13) for s = 100 coordinates and 2^10 points, with the criterion
  after each component.
* lattice_bits_problem2.txt: shifted lattice-sequence bits (Sec. 3.2, reading
  A11) and the normals (Phi^-1 of the 53-bit midpoint map, reading A12) of
  the 6-level lattice problem (seed 20180616) at a few (level, shift, index),
  first 8 coordinates.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402


def main():
    z, e2 = O.cbc(100, 10)
    with open(os.path.join(HERE, "cbc_s100_m10.txt"), "w") as f:
        f.write("# CBC generating vector, s = 100, N = 2^10, gamma_j = j^-2 (oracle or_cbc)\n")
        f.write("# j z_j criterion_after_j\n")
        for j in range(100):
            f.write(f"{j} {int(z[j])} {float(e2[j]).hex()}\n")
    cfg = W.LATTICE_6LEVEL
    orc = O.Oracle(n_levels=cfg["n_levels"], n0=cfg["n0"], s=cfg["s"], sampler="lattice", seed=cfg["seed"],
                   R=cfg["R"], genvec=z, log2_nmax=cfg["log2_nmax"])
    with open(os.path.join(HERE, "lattice_bits_problem2.txt"), "w") as f:
        f.write(f"# 6-level lattice problem: s = 100, seed {cfg['seed']}, 2^10 points; first 8 coordinates\n")
        f.write("# level shift index coordinate bits(hex) normal(hex float)\n")
        for (lv, r, n) in [(0, 0, 0), (0, 3, 1), (2, 7, 5), (5, 15, 31), (3, 1, 100)]:
            y = orc.normals(lv, r, n)
            for j in range(8):
                bits = O.lattice_bits(z[j], n, O.shift_bits(cfg["seed"], lv, r, j))
                f.write(f"{lv} {r} {n} {j} {bits:016x} {float(y[j]).hex()}\n")


if __name__ == "__main__":
    main()
