"""Comparison helpers for the parity tests (CUDA path vs the oracle)."""
import numpy as np


def oracle_rows_to_set(rows):
    """{(dim, birth, death, birth_vertex, death_vertex, essential)}"""
    return {(int(r[0]), int(r[1]), int(r[2]), int(r[3]), int(r[4]), int(r[5])) for r in rows}


def gpu_to_set(diag):
    out = set()
    for d in range(3):
        for p in diag[d]:
            out.add((int(p["dim"]), int(p["birth_simplex"]), int(p["death_simplex"]),
                     int(p["birth_vertex"]), int(p["death_vertex"]), int(p["essential"])))
    return out


def raw_bits(values, v):
    flat = values.reshape(-1)
    if flat.dtype == np.uint16:
        return int(flat[v])
    if flat.dtype == np.float32:
        return int(flat[v:v + 1].view(np.uint32)[0])
    return int(flat[v:v + 1].view(np.uint64)[0])


def check_bits(values, diag):
    """Birth/death bits are the raw bits of the maximum vertices' values; an
    infinite class dies at the maximum value."""
    flat = values.reshape(-1)
    vmax = flat.max()
    if flat.dtype.kind == "f" and vmax == 0:
        vmax = flat.dtype.type(0.0)
    maxbits = raw_bits(np.array([vmax], dtype=flat.dtype), 0)
    for d in range(3):
        for p in diag[d]:
            assert int(p["birth_bits"]) == raw_bits(values, int(p["birth_vertex"]))
            if p["essential"]:
                assert int(p["death_bits"]) == maxbits
            else:
                assert int(p["death_bits"]) == raw_bits(values, int(p["death_vertex"]))


def compare(values, diag, rows):
    got, want = gpu_to_set(diag), oracle_rows_to_set(rows)
    missing, extra = want - got, got - want
    assert not missing and not extra, (
        f"{len(missing)} missing e.g. {sorted(missing)[:5]}; {len(extra)} extra e.g. {sorted(extra)[:5]}")
    n = sum(len(diag[d]) for d in range(3))
    assert n == len(got), "duplicate pairs"
    check_bits(values, diag)
