"""The tile-shape autotuner: picks a valid shape by timing, caches it, and the
tuned shape leaves results unchanged."""
import json

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(tmp_path_factory):
    import os

    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_0711_gb300 import _build, coulps
    _build.build()
    coulps.load()
    coulps.use_torch_allocator()
    os.environ["COULPS_TUNE_CACHE"] = str(tmp_path_factory.mktemp("tune") / "tune.json")
    return torch, coulps, torch.cuda.Stream()


def test_tune_lattice_and_cache(env):
    torch, coulps, stream = env
    import os

    from paper_1403_0711_gb300 import autotune, inputs
    L = (48, 40, 36)
    lat = coulps.Lattice(L, n_chains=4, precision=coulps.F32, seed=3, stream=stream)
    best = autotune.tune_lattice(lat, reps=2)
    assert best in autotune.candidates(L, coulps.F32)
    assert lat.info()["ty"] == best[0] and lat.info()["dz"] == best[1]
    cache = json.loads(open(os.environ["COULPS_TUNE_CACHE"]).read())
    assert any(v["tile"] == list(best) for v in cache.values())
    # cached: same answer without timing again
    assert autotune.tune_shape(L, 4, coulps.F32, reps=2, stream=stream) == best
    # results do not depend on the tuned shape
    sites, q = inputs.uniform_q(L, 30, seed=1)
    ch = coulps.Charges(lat, sites, q, log_capacity=3)
    ch.run(1, 3, 1, 2)
    lat2 = coulps.Lattice(L, n_chains=4, precision=coulps.F32, seed=3, stream=stream)
    ch2 = coulps.Charges(lat2, sites, q, log_capacity=3)
    ch2.run(1, 3, 1, 2)
    for k in range(4):
        assert np.array_equal(lat.field(k), lat2.field(k))
    for o in (ch, ch2, lat, lat2):
        o.close()


def test_tune_batch(env):
    torch, coulps, stream = env
    from paper_1403_0711_gb300 import autotune, inputs
    systems = inputs.batch_systems(6, seed=2, edges=(32, 48))
    b = coulps.Batch([L for L, _, _ in systems], precision=coulps.F32, seed=1, stream=stream)
    best = autotune.tune_batch(b, reps=1)
    tiles = b.tiles()
    for (L, _, _), t in zip(systems, tiles):
        assert tuple(t) == tuple(best[L])
    b.close()
