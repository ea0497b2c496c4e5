"""The oracle's schedule against the values the paper prints for Case 3.

Fixture: tests/golden/paper_case3.txt (Sec. 3 "Compared Methods", "Experimental
Setup" and the discussion of Fig. 2).  The paper states the batch starts at
N_0 = 8 and reaches 13 without ever reaching full batch during the 240 s run;
it does not state the iteration count, so the check is that 13 is reached and
that full batch is not reached within the whole window in which the batch is
13 (under the reading "n" = n_theta and C = M).
"""
import os

from oracle import fblisa

HERE = os.path.dirname(os.path.abspath(__file__))


def _read(name):
    vals = {}
    with open(os.path.join(HERE, "golden", name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_case3_growth_8_to_13_never_full_batch():
    p = _read("paper_case3.txt")
    n = int(p["n_theta"])
    sched = fblisa.schedule(n, int(p["N0"]), n, p["M"], p["eps_base"], 60)
    Ns = [N for N, it in sched for _ in range(it)]  # batch size per iteration
    assert Ns[0] == int(p["batch_first"])
    last = int(p["batch_last"])
    assert last in Ns
    window_end = Ns.index(last + 1)
    assert all(N < n for N in Ns[:window_end]) == (p["full_batch_reached"] == 0)
    assert Ns[:window_end] == sorted(Ns[:window_end])


def test_stored_batches_reproduce():
    with open(os.path.join(HERE, "golden", "batches.txt")) as f:
        rows = [ln.split(":") for ln in f if not ln.startswith("#")]
    seen = {}
    for head, views in rows:
        seed, n_theta, N0, t, k, N_t = map(int, head.split())
        key = (seed, n_theta, t, N_t)
        if key not in seen:
            seen[key] = fblisa.epoch_batches(seed, t, n_theta, N_t)
            base = k
        assert seen[key][k - base] == [int(v) for v in views.split()]
