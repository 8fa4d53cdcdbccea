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


def _check_sort(keys_np, nbins, off, pm):
    """offsets are the exclusive prefix sum of the histogram; perm is a
    permutation that groups the keys by bin in ascending bin order."""
    ref_off = np.concatenate([[0], np.cumsum(np.bincount(keys_np, minlength=nbins))])
    assert np.array_equal(off, ref_off)
    assert np.array_equal(np.sort(pm), np.arange(keys_np.size))
    assert np.all(np.diff(keys_np[pm]) >= 0)


def test_noalloc_at_the_bin_limit():
    """nbins = 4,194,304, the scratch limit: 1,024 scan chunks, so each
    chunk's look-back spans many 32-chunk windows; then a smaller call on the
    same scratch, whose counts must start from zero again."""
    nbins = 1 << 22
    rng = np.random.default_rng(7)
    stream = torch.cuda.current_stream()
    for nb, n in ((nbins, 3_000_000), (5000, 20_000)):
        keys_np = rng.integers(0, nb, size=n).astype(np.int64)
        keys_np[:1000] = nb - 1  # a crowded last bin
        keys = torch.from_numpy(keys_np.astype(np.int32)).cuda()
        off = torch.full((nb + 1,), -7, dtype=torch.int32, device="cuda")
        perm = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        pic.sort_keys_noalloc(keys, nb, off, perm, stream=stream)
        torch.cuda.synchronize()
        _check_sort(keys_np, nb, off.cpu().numpy().astype(np.int64), perm.cpu().numpy().astype(np.int64))


def test_noalloc_empty_and_out_of_range_keys():
    """n = 0 gives all-zero offsets (two scan chunks at nbins = 5000); a key
    equal to nbins is rejected with PIC_ERR_ARG; a valid call afterwards
    sorts correctly (the scratch is cleared after an error)."""
    nb = 5000
    off = torch.full((nb + 1,), -7, dtype=torch.int32, device="cuda")
    empty = torch.zeros(0, dtype=torch.int32, device="cuda")
    pic.sort_keys_noalloc(empty, nb, off, empty)
    torch.cuda.synchronize()
    assert np.array_equal(off.cpu().numpy(), np.zeros(nb + 1, dtype=np.int32))

    rng = np.random.default_rng(8)
    keys_np = rng.integers(0, nb, size=4000).astype(np.int64)
    bad = keys_np.copy()
    bad[123] = nb
    perm = torch.zeros(bad.size, dtype=torch.int32, device="cuda")
    with pytest.raises(pic.PicError) as ei:
        pic.sort_keys_noalloc(torch.from_numpy(bad.astype(np.int32)).cuda(), nb, off, perm)
    assert ei.value.status == pic.PIC_ERR_ARG
    assert "outside" in str(ei.value)

    keys = torch.from_numpy(keys_np.astype(np.int32)).cuda()
    pic.sort_keys_noalloc(keys, nb, off, perm)
    torch.cuda.synchronize()
    _check_sort(keys_np, nb, off.cpu().numpy().astype(np.int64), perm.cpu().numpy().astype(np.int64))
