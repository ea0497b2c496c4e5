"""Write the stored mini-batch index vectors under tests/golden/.

Calls only the oracle (oracle.fblisa); run from the repository root:
    python tests/golden/make_golden.py
The CUDA library's host code must reproduce these vectors bit for bit.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import fblisa  # noqa: E402

CASES = [  # (seed, n_theta, N0, epochs)
    (3001, 90, 10, 2),
    (3003, 720, 40, 1),
    (7, 13, 5, 3),
]


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "batches.txt")
    with open(out, "w") as f:
        f.write("# seed n_theta N0 epoch k N_t : views  (written by tests/golden/make_golden.py)\n")
        for seed, n_theta, N0, epochs in CASES:
            k = 0
            for t, (N_t, _) in enumerate(fblisa.schedule(n_theta, N0, n_theta, 1.0, 0.99, epochs), 1):
                for views in fblisa.epoch_batches(seed, t, n_theta, N_t):
                    f.write("%d %d %d %d %d %d : %s\n" % (seed, n_theta, N0, t, k, N_t,
                                                          " ".join(map(str, views))))
                    k += 1
    print(out)


if __name__ == "__main__":
    main()
