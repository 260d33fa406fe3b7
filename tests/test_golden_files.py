"""The stored expected values under tests/golden/ are what the oracle
computes now (the small and fast entries are recomputed here; the 128^3
entries of e_lat.txt take minutes and are checked only for their format)."""
import numpy as np


def _rows(name):
    from pathlib import Path
    p = Path(__file__).resolve().parent / "golden" / name
    return [ln.split() for ln in p.read_text().splitlines() if ln and not ln.startswith("#")]


def test_e_lat_small_entries_recomputed(orc):
    from paper_1403_0711_gb300 import inputs
    rows = {r[0]: r for r in _rows("e_lat.txt")}
    for name in ("plain_16c_n8_pm", "cube_16c_n8_q1"):
        r = rows[name]
        L = tuple(int(v) for v in r[1:4])
        sites, q = (inputs.plus_minus(L, int(r[5]), int(r[6])) if r[4] == "plus_minus"
                    else inputs.cube(L, round(int(r[5]) ** (1 / 3))))
        assert abs(orc.e_lat(L, sites, q, "dense") - float(r[8])) < 1e-12 * abs(float(r[8]))
        assert abs(orc.coulomb_direct(sites, q) - float(r[9])) < 1e-12 * abs(float(r[9]))
    for r in rows.values():
        assert len(r) == 10 and np.isfinite(float(r[8])) and np.isfinite(float(r[9]))


def test_offlattice_entries_recomputed(orc):
    from oracle import offlattice as off
    from paper_1403_0711_gb300 import inputs
    for r in _rows("offlattice.txt"):
        L = tuple(int(v) for v in r[1:4])
        side, seed, jitter, rc = int(r[4]), int(r[5]), float(r[6]), float(r[7])
        pos, q = inputs.off_lattice_cube(L, side, seed, jitter)
        pairs = off.near_pairs(pos, rc)
        assert len(pairs) == int(r[8])
        want = [off.far_energy_solve(L, pos, q, pairs), off.near_direct_energy(pos, q, pairs),
                off.far_energy_solve(L, pos, q, pairs[:0]), orc.coulomb_direct(pos, q)]
        for w, got in zip(want, r[9:13]):
            assert abs(w - float(got)) < 1e-12 * max(1.0, abs(w))
