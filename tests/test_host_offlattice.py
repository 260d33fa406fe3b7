"""Host logic of the off-lattice sets, through the C ABI on the CPU (no
device): the near-pair builder (cell grid) against the oracle's brute-force
pair set, and the corner offsets, weights and gradients against the oracle's
trilinear corners."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def cl():
    from paper_1403_0711_gb300 import _build, coulps
    _build.build()
    coulps.load()
    return coulps


def _pairs_of_csr(ptr, nbr):
    n = len(ptr) - 1
    out = set()
    for i in range(n):
        lst = list(nbr[ptr[i]:ptr[i + 1]])
        assert lst == sorted(lst) and i not in lst
        for j in lst:
            out.add((min(i, j), max(i, j)))
    return out


@pytest.mark.parametrize("n,rc,box,seed", [(0, 1.0, 5, 0), (1, 1.0, 5, 1), (2, 10.0, 3, 2),
                                           (50, 1.5, 8, 3), (300, 2.2, 20, 4), (200, 0.0, 6, 5),
                                           (120, 50.0, 9, 6), (400, 0.7, 4, 7)])
def test_near_pairs_match_brute_force(cl, n, rc, box, seed):
    from oracle import offlattice as off
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, box, (n, 3))
    if n >= 10:  # a tight cluster and coincident particles
        pos[:5] = pos[0] + rng.uniform(-0.05, 0.05, (5, 3))
        pos[5] = pos[6]
    ptr, nbr = cl.near_pairs(pos, rc)
    assert len(ptr) == n + 1 and ptr[0] == 0 and len(nbr) == ptr[-1]
    got = _pairs_of_csr(ptr, nbr)
    want = {tuple(p) for p in off.near_pairs(pos, rc)} if n else set()
    assert got == want
    assert 2 * len(want) == len(nbr)  # both directions


def test_near_pairs_rejects_bad_input(cl):
    with pytest.raises(cl.CoulpsError):
        cl.near_pairs([[0, 0, np.nan]], 1.0)
    with pytest.raises(cl.CoulpsError):
        cl.near_pairs([[0, 0, 0]], -1.0)


def _layout(L, precision):
    es = 4 if precision == 0 else 8
    wq = (L[0] + 7) // 8
    align = 32 // es
    W = (4 * wq + align - 1) // align * align
    return W, L[2] * L[1] * W


@pytest.mark.parametrize("L,prec", [((6, 5, 4), 0), ((13, 2, 7), 1), ((128, 128, 128), 0),
                                    ((2, 2, 2), 0), ((33, 17, 9), 1)])
def test_corners_match_oracle(cl, L, prec):
    from oracle import offlattice as off
    from paper_1403_0711_gb300 import inputs
    pos, _ = inputs.off_lattice(L, 40, seed=sum(L))
    offs, w, g = cl.offlattice_corners(L, prec, pos)
    sites, w_o, g_o = off.corners(L, pos)
    assert np.abs(w - w_o).max() < 1e-15 and np.abs(g - g_o).max() < 1e-15
    W, ce = _layout(L, prec)
    colour = offs // ce
    rem = offs % ce
    z, y, h = rem // (L[1] * W), (rem // W) % L[1], rem % W
    x = 2 * h + ((colour + y + z) & 1)
    assert np.array_equal(np.stack([x, y, z], axis=-1), sites)
    assert np.array_equal(colour, sites.sum(axis=-1) & 1)


def test_corners_reject_bad_input(cl):
    for L, pos in (((6, 5, 4), [[5.0001, 1, 1]]), ((6, 5, 4), [[-1e-9, 1, 1]]),
                   ((6, 1, 4), [[1, 0, 1]]), ((6, 5, 4), [[np.inf, 1, 1]])):
        with pytest.raises(cl.CoulpsError):
            cl.offlattice_corners(L, 0, pos)
