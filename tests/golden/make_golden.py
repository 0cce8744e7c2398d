"""Write the oracle-derived golden files of tests/golden/ (calls only oracle/)."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

if __name__ == "__main__":
    om = oracle.sample_frequencies(64, 0.1, 0)
    with open(os.path.join(HERE, "omega_m64_eps0.1_seed0.txt"), "w") as f:
        f.write("# oracle.sample_frequencies(m=64, eps=0.1, seed=0), default sigma/R; hex floats, one frequency per row\n")
        for row in om:
            f.write(" ".join(float(x).hex() for x in row) + "\n")
