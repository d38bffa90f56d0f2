"""Writes the oracle's diagram of a full-size configuration as a digest:
``tests/golden/<name>_oracle.json``.

    python -m tests.golden.make_oracle_digest noise256_f32
    python -m tests.golden.make_oracle_digest mixture512_u16

The field is generated on the CPU by ``synthfields.config_field`` and its
bytes' SHA-256 is recorded.  The pairs come from ``oracle.fastpairs`` (the
standard reduction in fast mode, pinned equal to the textbook reduction):
per dimension, the count of finite pairs and of infinite classes and the
SHA-256 of the canonical row list -- int64 rows (dim, birth simplex, death
simplex, birth vertex, death vertex, infinite flag) sorted by (birth, death)
-- which a test computes the same way from the GPU's pairs.  Only oracle/
and synthfields are called.  The 512^3 recipe takes about an hour and some
25 GB of RAM on one core; 256^3 noise about six minutes.
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synthfields as sf  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def canonical(rows6: np.ndarray) -> dict:
    """Per-dimension counts and SHA-256 of int64 rows (dim, birth, death,
    birth_vertex, death_vertex, infinite) sorted by (birth, death)."""
    import hashlib
    out = {}
    for d in range(3):
        r = rows6[rows6[:, 0] == d]
        r = r[np.lexsort((r[:, 2], r[:, 1]))]
        out[str(d)] = {"finite": int((r[:, 5] == 0).sum()), "infinite": int((r[:, 5] == 1).sum()),
                       "sha256": hashlib.sha256(np.ascontiguousarray(r, np.int64).tobytes())
                       .hexdigest()}
    return out


def main(name: str):
    t0 = time.time()
    v = sf.config_field(name)
    shape, dtype, recipe = sf.CONFIGS[name]
    field_sha = sf.sha256(v)
    t1 = time.time()
    rows = oracle.fastpairs(v)
    t2 = time.time()
    doc = {
        "source": "oracle.fastpairs (standard reduction, fast mode) on synthfields.config_field"
                  f"({name!r}) generated on the CPU; written by tests/golden/make_oracle_digest.py",
        "config": name, "shape_xyz": list(shape), "dtype": np.dtype(dtype).name, "recipe": recipe,
        "field_sha256": field_sha,
        "dims": canonical(np.ascontiguousarray(rows[:, :6], np.int64)),
        "oracle_seconds": round(t2 - t1, 1), "generation_seconds": round(t1 - t0, 1),
    }
    path = os.path.join(HERE, f"{name}_oracle.json")
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")
    print(path, json.dumps(doc["dims"]))


if __name__ == "__main__":
    main(sys.argv[1])
