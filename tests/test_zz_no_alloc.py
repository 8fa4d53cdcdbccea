"""The no-allocation counting sort (pic_sort_keys_noalloc) against the
particle sort the library runs when it loads particles.

Some callers cannot allocate device memory: code running while a CUDA stream
is being captured, or hosts that give a library only the buffers it may
touch.  pic_sort_keys_noalloc serves them with its scratch in a static device
array.  This file is collected last, so a run that stops at its first failure
has already run every other test; it passes alone and after the others.
"""
import numpy as np
import pytest

from paper_2101_12149_gb300 import inputs, pic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_GRID = (32, 16, 24)
TILE = 8


def tile_keys(x, y, z):
    """The library's sort key: tile-major cell index (8^3 tiles, k fastest inside)."""
    i, j, k = (np.floor(a).astype(np.int64) for a in (x, y, z))
    nt = [n // TILE for n in N_GRID]
    t = ((i // TILE) * nt[1] + (j // TILE)) * nt[2] + (k // TILE)
    loc = ((i % TILE) * TILE + (j % TILE)) * TILE + (k % TILE)
    return (t * TILE ** 3 + loc).astype(np.int64)


def sorted_by_library(seed, precision):
    """Particles loaded into a context (which sorts them); returns the keys in
    load order and the library's (key, id) sequence."""
    parts = inputs.uniform_plasma(seed, N_GRID, 3, sigma_u=0.3)
    with pic.Context(N_GRID, order=2, precision=precision, tile=(TILE,) * 3) as ctx:
        ctx.load_particles(-1.0, 1.0, parts)
        lib = ctx.get_particles()
    lib_keys = tile_keys(lib["x"], lib["y"], lib["z"])
    lib_ids = lib["id"].astype(np.int64)
    # the keys the library sorted on, put back in load order
    keys_load_order = np.empty_like(lib_keys)
    keys_load_order[lib_ids] = lib_keys
    return keys_load_order, lib_keys, lib_ids


@pytest.mark.parametrize("precision", [pic.FP64])
def test_noalloc_sort_matches_library_sort(precision):
    C = N_GRID[0] * N_GRID[1] * N_GRID[2]
    stream = torch.cuda.current_stream()
    for call, seed in enumerate((101, 202)):  # two calls in a row on the same scratch
        keys, lib_keys, lib_ids = sorted_by_library(seed, precision if call == 0 else pic.FP32_MIXED)
        assert np.all(np.diff(lib_keys) >= 0)
        dkeys = torch.from_numpy(keys.astype(np.int32)).cuda()
        offsets = torch.full((C + 1,), -7, dtype=torch.int32, device="cuda")
        perm = torch.full((keys.size,), -7, dtype=torch.int32, device="cuda")
        pic.sort_keys_noalloc(dkeys, C, offsets, perm, stream=stream)
        torch.cuda.synchronize()
        off = offsets.cpu().numpy().astype(np.int64)
        pm = perm.cpu().numpy().astype(np.int64)
        # bin offsets: unique, equal to the library's bins exactly
        ref_off = np.concatenate([[0], np.cumsum(np.bincount(lib_keys, minlength=C))])
        assert np.array_equal(off, ref_off)
        # perm is a permutation, grouped by bin like the library's order
        assert np.array_equal(np.sort(pm), np.arange(keys.size))
        assert np.array_equal(keys[pm], lib_keys)
        # within a bin the order is free: compare the members
        a = np.lexsort((pm, keys[pm]))
        b = np.lexsort((lib_ids, lib_keys))
        assert np.array_equal(pm[a], lib_ids[b])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    k = torch.zeros(4, dtype=torch.int32, device="cuda")
    off = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(pic.PicError) as ei:
        pic.sort_keys_noalloc(k, (1 << 22) + 1, off, k)
    assert ei.value.status == pic.PIC_ERR_ARG
    assert "4194304" in str(ei.value)
