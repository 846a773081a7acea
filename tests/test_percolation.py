"""Site percolation on the GPU against the oracle (Supplemental Material).

Largest clusters are integers: the GPU union-find must equal the oracle's
breadth-first search exactly, for given masks and for masks drawn on the
device from the Philox stream (reproduced here with the oracle's Philox)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1501_05630_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1501_05630_gb300 import build, icmpt
    build.build()
    torch.cuda.set_device(0)
    ctx = icmpt.Context(0)
    yield icmpt, ctx
    ctx.close()


@pytest.mark.parametrize("kind,L", [(O.SQUARE2D, 6), (O.SQUARE2D, 32), (O.CUBIC3D, 4), (O.CUBIC3D, 8),
                                    (O.CHIMERA, 1), (O.CHIMERA, 3), (O.CHIMERA, 16), (O.CHIMERA, 48)])
def test_largest_clusters_equal_oracle(env, kind, L):
    icmpt, ctx = env
    g = O.Geometry(kind, L)
    masks = np.concatenate([I.site_masks(g.N, p, 31 + L, 25) for p in (0.0, 0.2, 0.31, 0.39, 0.59, 0.8, 1.0)])
    got = icmpt.largest_clusters(ctx, kind, L, masks)
    assert np.array_equal(got, O.largest_clusters(g, masks))


def _philox_masks(g, p, seed, n):
    key = [seed & 0xFFFFFFFF, seed >> 32]
    thr = int(p * 2 ** 32) if p < 1 else 2 ** 32 - 1
    m = np.zeros((n, g.N), dtype=np.uint8)
    for a in range(n):
        for i in range(g.N):
            m[a, i] = O.philox([i, a, 0, 5 << 24], key)[0] < thr
    return m


@pytest.mark.parametrize("kind,L,p", [(O.CHIMERA, 3, 0.3866), (O.SQUARE2D, 8, 0.5927), (O.CUBIC3D, 4, 0.3116)])
def test_device_random_masks_follow_the_philox_stream(env, kind, L, p):
    icmpt, ctx = env
    g = O.Geometry(kind, L)
    seed = 0x1501056300000005
    got = icmpt.largest_clusters_random(ctx, kind, L, p, seed, 12)
    assert np.array_equal(got, O.largest_clusters(g, _philox_masks(g, p, seed, 12)))
    assert np.all(icmpt.largest_clusters_random(ctx, kind, L, 1.0, seed, 3) == g.N)
    assert np.all(icmpt.largest_clusters_random(ctx, kind, L, 0.0, seed, 3) == 0)
