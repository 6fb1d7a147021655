"""Write tests/golden/jet512x256x256.json from a full FP64 CPU-oracle solve of
the 512x256x256 jet (L = (2, 1, 1), periodic x, walls y and z, rho 1000/1,
dt = 5e-5; Sec. 3.7, Eq. poisson).

Calls only the oracle and the seeded input generator, through the same
record writer as the 256^3 drop field: the checksum of C, the oracle's
iterations, residuals and Lanczos extremes, its own error bound, and p at
4096 seeded cells and u at 4096 seeded faces.
Run:  python tests/golden/make_jet512_golden.py  (about an hour on 8 cores).
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
import make_drops256_golden as mk  # noqa: E402


def main(out=None):
    out = out or os.path.join(HERE, "jet512x256x256.json")
    mk.solve_and_store(mk.pi.config3(), out, [301, 512])


if __name__ == "__main__":
    main()
