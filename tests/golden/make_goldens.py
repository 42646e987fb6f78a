"""Write the stored expected values under tests/golden/ that are too slow to
recompute in the CPU test suite.  Calls only the oracle package.

    python tests/golden/make_goldens.py [--rows 7,8,9] [--jobs 3]

table1_irreducible.txt: for each Table I row (sl, ll), whether the trinomial
x^ll + x^sl + 1 is irreducible over GF(2) (oracle.gf2_trinomial_irreducible).
For the Mersenne exponents ll of Table I irreducible implies primitive, which
is what gives the additive generator its maximal period (Sec. II.D).
"""
import argparse
import os
import sys
import time
from concurrent.futures import ProcessPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))


def _rows():
    out = []
    with open(os.path.join(HERE, "table1_lags.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                r, sl, ll = map(int, line.split())
                out.append((r, sl, ll))
    return out


def _check(args):
    r, sl, ll = args
    import oracle
    t0 = time.time()
    ok = oracle.gf2_trinomial_irreducible(ll, sl)
    return r, sl, ll, ok, time.time() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rows", default="0,1,2,3,4,5,6,7,8,9")
    ap.add_argument("--jobs", type=int, default=4)
    a = ap.parse_args()
    want = {int(x) for x in a.rows.split(",")}
    import oracle
    oracle.build()
    todo = [row for row in _rows() if row[0] in want]
    path = os.path.join(HERE, "table1_irreducible.txt")
    known = {}
    if os.path.exists(path):
        with open(path) as f:
            for line in f:
                if line.strip() and not line.startswith("#"):
                    r, sl, ll, ok = line.split()[:4]
                    known[int(r)] = (int(sl), int(ll), int(ok))
    import multiprocessing as mp
    with ProcessPoolExecutor(a.jobs, mp_context=mp.get_context("spawn")) as ex:
        for r, sl, ll, ok, dt in ex.map(_check, todo):
            known[r] = (sl, ll, int(ok))
            print(f"row {r}: x^{ll} + x^{sl} + 1 irreducible={ok} ({dt:.0f} s)", flush=True)
    with open(path, "w") as f:
        f.write("# Written by tests/golden/make_goldens.py (oracle.gf2_trinomial_irreducible).\n")
        f.write("# row sl ll irreducible(1/0) for x^ll + x^sl + 1 over GF(2), Table I rows.\n")
        for r in sorted(known):
            sl, ll, ok = known[r]
            f.write(f"{r} {sl} {ll} {ok}\n")


if __name__ == "__main__":
    main()
