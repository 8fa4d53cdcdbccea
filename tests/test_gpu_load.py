"""pic_load_particles from the three kinds of source memory gives the same
particles bit for bit: device arrays, pinned host arrays (read by the load
kernel directly) and pageable host arrays (staged in chunks of 2^23
particles; this load takes two chunks)."""
import numpy as np
import pytest

from paper_2101_12149_gb300 import inputs, pic

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [pic.FP32_MIXED, pic.FP64])
def test_device_pinned_and_pageable_loads_agree(precision):
    import torch
    n = (128, 128, 68)                      # 8 ppc: 8,912,896 particles > 2^23
    parts = inputs.uniform_plasma(7, n, 8, sigma_u=0.1)
    # a few positions outside the box (wrapped on load) and on its faces
    parts["x"][:3] = [-0.25, 128.0, 300.5]
    parts["z"][3:5] = [68.0, -68.0]
    pinned = {k: torch.from_numpy(v).pin_memory() for k, v in parts.items()}
    device = {k: torch.from_numpy(v).cuda() for k, v in parts.items()}
    out = []
    for src in (device, pinned, parts):
        with pic.Context(n, order=3, precision=precision) as c:
            c.load_particles(-1.0, 1.0, src)
            out.append(c.get_particles())
    for o in out[1:]:
        for k in pic.PARTICLE_KEYS + ("id",):
            assert np.array_equal(o[k], out[0][k]), k
    assert out[0]["id"].size == parts["x"].size
    assert np.all((out[0]["x"] >= 0) & (out[0]["x"] < 128))
