"""Write the oracle's farthest-point picks on the full-size workloads.

The full-size FPS parity tests compare the CUDA picks with these, index for
index, and the CPU baseline triangulates these landmarks to time the oracle
on the workload's own complex. Every stored value comes from the oracle alone
(oracle.fps: greedy k-centre of §3.2 with binary32 keys and lowest-index
ties) run on the seeded generator's cloud; nothing here touches the CUDA path.
One oracle iteration is a pass over X, so the 5,000,000-point shape mix with
10,000 picks takes about 20 minutes on one core, the 1M-point clouds with
2,000 picks about a minute.

Output: fps_<workload>_oracle.txt beside this script. Header lines start with
'#': the generator call, the SHA-256 of the cloud's float32 bytes (readers
check it first, so a host whose numpy draws a different cloud is reported as
such), n_landmarks, start, the SHA-256 of the picked keys' binary32 bytes and
the last key's bits. Then one picked row of X per line, in pick order.

    python tests/golden/make_fps_golden.py torus-1M shapes-5M swisscheese-1M swisscheese4d-1M swisscheese5d-1M
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2509_22432_b300 import data  # noqa: E402

# workload -> (generator call as text, generator, n_landmarks)
WORKLOADS = {
    "torus-1M": ("data.torus_cloud(1_000_000, seed=2)", lambda: data.torus_cloud(1_000_000, seed=2), 2000),
    "shapes-5M": ("data.shape_mix_cloud(5_000_000, seed=3)", lambda: data.shape_mix_cloud(5_000_000, seed=3),
                  10_000),
    "swisscheese-1M": ("data.swisscheese_cloud(1_000_000, seed=6)",
                       lambda: data.swisscheese_cloud(1_000_000, seed=6), 2000),
    # the scaling study in the ambient dimension (§5.3, Fig. 4c: |X| = 1M, |L| = 1k)
    "swisscheese4d-1M": ("data.swisscheese_cloud(1_000_000, seed=6, dim=4)",
                         lambda: data.swisscheese_cloud(1_000_000, seed=6, dim=4), 1000),
    "swisscheese5d-1M": ("data.swisscheese_cloud(1_000_000, seed=6, dim=5)",
                         lambda: data.swisscheese_cloud(1_000_000, seed=6, dim=5), 1000),
}
START = 0


def path_of(workload: str) -> str:
    return os.path.join(HERE, f"fps_{workload}_oracle.txt")


def cloud_sha256(X: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(X, np.float32).tobytes()).hexdigest()


def read(workload: str) -> dict:
    """Parse a golden file: header fields and the picked rows (int64)."""
    head, rows = {}, []
    with open(path_of(workload)) as f:
        for line in f:
            if line.startswith("#"):
                parts = line[1:].split()
                if len(parts) == 2:
                    head[parts[0]] = parts[1]
            elif line.strip():
                rows.append(int(line))
    head["idx"] = np.array(rows, dtype=np.int64)
    return head


def write(workload: str) -> None:
    call, gen, n_l = WORKLOADS[workload]
    X = gen()
    t0 = time.time()
    idx, key = oracle.fps(X, n_l, START)
    key_sha = hashlib.sha256(np.ascontiguousarray(key, np.float32).tobytes()).hexdigest()
    out = path_of(workload)
    with open(out + ".tmp", "w") as f:
        f.write(f"# oracle.fps picks on {call} (written by make_fps_golden.py)\n")
        f.write(f"# x_sha256 {cloud_sha256(X)}\n")
        f.write(f"# n_landmarks {n_l}\n")
        f.write(f"# start {START}\n")
        f.write(f"# key_sha256 {key_sha}\n")
        f.write(f"# last_key_hex {int(np.float32(key[-1]).view(np.uint32)):08x}\n")
        for i in idx:
            f.write(f"{int(i)}\n")
    os.replace(out + ".tmp", out)
    print(f"wrote {out} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    for w in sys.argv[1:] or list(WORKLOADS):
        write(w)
