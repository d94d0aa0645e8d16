"""The hand-worked z_top cases of tests/golden/block_ztop.txt (App. D, the
height of the highest part within a block) as scenes, shared by the oracle
pin and the GPU check."""
import math
import pathlib

import torch

from paper_2312_16457_gb300 import synth


def ztop_golden_cases():
    """(R, C, zlo, zhi, kind, k, z_top) rows of tests/golden/block_ztop.txt."""
    rows = []
    for ln in (pathlib.Path(__file__).parent / "golden" / "block_ztop.txt").read_text().splitlines():
        if not ln.strip() or ln.startswith("#"):
            continue
        t = ln.split()
        rows.append((int(t[0]), int(t[1]), float(t[2]), float(t[3]), t[4], None if t[5] == "-" else int(t[5]),
                     float(t[6])))
    return rows


def ztop_case_scene(R, C, zlo, zhi, kind, k):
    """One block over [0, 1]^2 x [zlo, zhi] whose dense vertices follow the
    fixture's kind: density 20 there (ch0 = ln 20), 1e-4 elsewhere."""
    g = torch.zeros(R, R, R, 8)
    g[..., 0] = math.log(1e-4)
    if kind == "vertex":
        g[k, 1, R - 1, 0] = math.log(20.0)
    elif kind == "slab":
        g[: k + 1, :, :, 0] = math.log(20.0)
    pl = [torch.zeros(4, 4, 8) for _ in range(3)]
    blk = synth.Block((0.0, 0.0, zlo), (1.0, 1.0, zhi), R, 4, grid=g, planes=pl)
    return synth.Scene([blk], (0.0, 0.0, zlo), (1.0, 1.0, zhi), occ_cell=C)
