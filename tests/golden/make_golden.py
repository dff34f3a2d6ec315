"""Write the stored oracle fixtures under tests/golden/.

Calls only the FP64 oracle (and the seeded input generator).  The fixture is
a regression guard for the oracle itself: Eq. 1-3 with the Sec. II.A default
gene on a 4 x 5 torus, x ~ U[-1, 1] (seed 0), u = v = x, T = 10.
Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import rdcnn_inputs as inp  # noqa: E402


def main():
    params = inp.default_params()
    x = inp.uniform_field(0, 4, 5)
    u, v = oracle.run(x, x, params, 10)
    out = {
        "cite": "Eq. 1-3, Sec. II.A defaults; toroidal boundary (Sec. II.B-II.C); written by oracle only",
        "seed": 0, "T": 10, "params": params,
        "u": [[float(repr_) for repr_ in row] for row in u.tolist()],
        "v": [[float(repr_) for repr_ in row] for row in v.tolist()],
    }
    with open(os.path.join(HERE, "oracle_4x5_T10.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
