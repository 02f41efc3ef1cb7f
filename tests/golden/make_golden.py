"""Writes the oracle's golden rollout summaries in this folder.

Calls only ``oracle`` (and the seeded input generators for its inputs). The
paper prints no MPM state to compare against, so these files are regression
fixtures of the oracle itself: a change to them must name, in its commit
message, the passage or reading that justifies the changed arithmetic.

Usage: python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2302_04659_gb300 import scenes  # noqa: E402


def summary(s, m):
    ke = 0.5 * m * (s.v ** 2).sum()
    com = s.x.mean(1)
    mom = m * s.v.sum(1)
    lo, hi = s.x.min(1), s.x.max(1)
    fdev = np.abs(s.F - np.eye(3).reshape(9, 1)).mean() if s.F is not None else 0.0
    return np.concatenate([com, mom, [ke], lo, hi, [fdev]])


def cube_floor_rollout():
    sc = scenes.cube_scene("floor")
    P = oracle.Params(n=sc.n, dt=sc.dt, p_vol=sc.material.p_vol)
    s = oracle.State.from_arrays(sc.x, sc.v, sc.C, sc.F)
    m = P.c().p_mass
    rows = []
    for k in range(50):
        oracle.substep(P, s)
        if (k + 1) % 10 == 0:
            rows.append([k + 1] + list(summary(s, m)))
    return np.array(rows)


def main():
    rows = cube_floor_rollout()
    header = ("oracle rollout of the 32^3 / 8,192-particle plasticine cube on the sticky floor "
              "(dt 2e-4, E 5e3, nu 0.3, yield 50, rho 1e3), written by tests/golden/make_golden.py\n"
              "substep com_x com_y com_z p_x p_y p_z kinetic_energy min_x min_y min_z max_x max_y max_z mean|F-I|")
    np.savetxt(os.path.join(HERE, "cube_floor_rollout.txt"), rows, fmt="%.17g", header=header)


if __name__ == "__main__":
    main()
