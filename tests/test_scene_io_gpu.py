"""Packed scene files (cow_save_scene / cow_load_scene): a context loaded
from the file renders exactly what the saved one rendered, for dense and
brick-sparse grids, FP8 storage with its scales, unbounded blocks and LOD
links, and for blocks written from their host copies under a budget."""
import os

import numpy as np
import pytest
import torch

from paper_2312_16457_gb300 import cow, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2312_16457_gb300 import build

    build.build()
    torch.cuda.set_device(0)


def _views(ctx, sc):
    cams = [synth.camera((-3.5, -5.0, 3.5), (0.2, 0.3, -0.9), 48, 30, 60.0),
            synth.camera((2.0, 2.5, 1.0), (-1.0, -0.5, -0.8), 33, 27, 70.0)]
    if sc.n_levels > 1:
        return cams, [ctx.select_lod(c, sc.lod_thresh) for c in cams]
    return cams, [ctx.sort_blocks(c, list(range(len(sc.blocks)))) for c in cams]


@pytest.mark.parametrize("storage,bricks", [("bf16", False), ("fp8", False), ("fp8_bf16d", True), ("fp32", True)])
def test_saved_scene_renders_the_same(tmp_path, storage, bricks):
    sc = synth.city_scene(41, 4, 2.0, [(20, 24), (12, 16)], **synth.SPARSE_CITY)
    ctx = cow.Context(sc, storage, bricks=bricks)
    cams, ids = _views(ctx, sc)
    mlp = synth.mlp_weights(4)
    ref = ctx.render(cams, ids, mlp, nsamp=True)
    path = str(tmp_path / "scene.cow")
    ctx.save(path)
    assert os.path.getsize(path) > 0
    ld = cow.Context.load(path, scene=sc)
    assert ld.n_blocks == len(sc.blocks)
    for i in range(len(sc.blocks)):
        assert ld.ztop(i) == ctx.ztop(i)
        assert ld.block_bytes(i) == ctx.block_bytes(i)
        assert np.array_equal(ld.occupancy(i), ctx.occupancy(i))
    got = ld.render(cams, [ld.select_lod(c, sc.lod_thresh) for c in cams], mlp, nsamp=True)
    ld.sync_check()
    for x, y in zip(ref, got):
        assert torch.equal(x, y)
    ld.close()
    ctx.close()


def test_saved_scene_unbounded_and_budget(tmp_path):
    sc, cams, mlp = synth.workload_unbounded(R=24, P=32, width=40, height=24)
    ctx = cow.Context(sc, "fp16")
    ids = [ctx.sort_blocks(cams[0], list(range(4)))]
    ref = ctx.render(cams, ids, mlp, nsamp=True)
    ctx.set_residency(ctx.block_bytes(0) + ctx.block_bytes(1))  # every block unloaded on entry
    path = str(tmp_path / "unb.cow")
    ctx.save(path)  # written from the pinned host copies
    ld = cow.Context.load(path, scene=sc)
    got = ld.render(cams, ids, mlp, nsamp=True)
    ld.sync_check()
    for x, y in zip(ref, got):
        assert torch.equal(x, y)
    ctx.set_residency(0)
    ld.close()
    ctx.close()


def test_load_rejects_foreign_files(tmp_path):
    p = tmp_path / "junk.cow"
    p.write_bytes(b"not a scene" * 10)
    with pytest.raises(cow.CowError, match="packed scene"):
        cow.Context.load(str(p))
    sc = synth.city_scene(41, 2, 2.0, [(8, 8)])
    ctx = cow.Context(sc, "bf16")
    full = tmp_path / "s.cow"
    ctx.save(str(full))
    data = full.read_bytes()
    (tmp_path / "cut.cow").write_bytes(data[: len(data) // 2])
    with pytest.raises(cow.CowError, match="truncated"):
        cow.Context.load(str(tmp_path / "cut.cow"))
    ctx.close()


def _sections(data):
    """(data start, per block (offsets, bytes) of its 8 sections) of a packed
    scene file: header 40 bytes, 320-byte block records, the JSON manifest,
    then the arrays from the next 256-byte boundary."""
    import struct

    n_blocks = struct.unpack_from("<i", data, 12)[0]
    json_bytes = struct.unpack_from("<Q", data, 32)[0]
    data0 = (40 + 320 * n_blocks + json_bytes + 255) & ~255
    blocks = []
    for i in range(n_blocks):
        base = 40 + 320 * i
        blocks.append((struct.unpack_from("<8Q", data, base + 192), struct.unpack_from("<8Q", data, base + 256)))
    return data0, blocks


def test_load_rejects_inconsistent_occupancy_and_bricks(tmp_path):
    """A file whose coarse occupancy is not the OR of its fine cells, or whose
    brick table leaves an occupied brick unstored, is refused: the kernels
    trust both (they skip coarse cells without reading fine ones, and read an
    occupied cell's brick without testing its slot)."""
    import struct

    sc = synth.city_scene(43, 2, 2.0, [(20, 24)], **synth.SPARSE_CITY)
    ctx = cow.Context(sc, "bf16", bricks=True)
    path = tmp_path / "s.cow"
    ctx.save(str(path))
    ctx.close()
    data = bytearray(path.read_bytes())
    data0, blocks = _sections(bytes(data))
    ok = cow.Context.load(str(path))  # the file as saved loads
    ok.close()
    # a block with a stored brick: clear that brick's coarse bit
    for off, nbytes in blocks:
        tab = np.frombuffer(bytes(data[data0 + off[6]: data0 + off[6] + nbytes[6]]), dtype=np.int32)
        stored = np.nonzero(tab >= 0)[0]
        if len(stored):
            k = int(stored[0])
            bad = bytearray(data)
            w = data0 + off[5] + 4 * (k >> 5)
            struct.pack_into("<I", bad, w, struct.unpack_from("<I", bad, w)[0] & ~(1 << (k & 31)))
            (tmp_path / "occ2.cow").write_bytes(bytes(bad))
            with pytest.raises(cow.CowError, match="inconsistent"):
                cow.Context.load(str(tmp_path / "occ2.cow"))
            bad = bytearray(data)
            struct.pack_into("<i", bad, data0 + off[6] + 4 * k, -1)
            (tmp_path / "tab.cow").write_bytes(bytes(bad))
            with pytest.raises(cow.CowError, match="inconsistent"):
                cow.Context.load(str(tmp_path / "tab.cow"))
            break
    else:
        pytest.fail("no stored brick in the scene")
