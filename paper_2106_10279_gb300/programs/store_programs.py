"""Build the programs that take minutes to construct and store their
structure next to this file (process.build_program then loads them):

    python -m paper_2106_10279_gb300.programs.store_programs

gg -> tt~ggg: 1240 diagrams, 3712 operations, a 120 x 120 colour matrix;
about ten minutes of Python.  The stored structure keeps masses as flavour
names and couplings by kind, so any m_t, alpha_s and alpha can be loaded.
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from paper_2106_10279_gb300 import process as P  # noqa: E402

STORED = {"gg_ttxggg": [("g", True), ("g", True), ("t", False), ("t~", False), ("g", False), ("g", False),
                        ("g", False)]}


def main():
    for name, legs in STORED.items():
        path = os.path.join(HERE, name + ".json")
        if os.path.exists(path):
            os.rename(path, path + ".old")        # build from scratch, not from the store
        t = time.time()
        masses = {"t": 173.0}
        prog = P.build_program(name, legs, masses, 0.118, 1 / 128)
        P.store_program(prog, masses, path)
        if os.path.exists(path + ".old"):
            os.remove(path + ".old")
        print(f"{name}: {prog.n_diagrams} diagrams, {len(prog.ops)} ops, {prog.colour_num.shape[0]} flows, "
              f"{time.time() - t:.0f} s")


if __name__ == "__main__":
    main()
