"""Write tests/golden/e_lat.txt: exact lattice energies E_lat of the seeded
workloads, computed by the FP64 oracle only (DST-I spectral solve for G rho,
heat-kernel quadrature for G_ii; dense Cholesky where the box is small), and
tests/golden/offlattice.txt: the off-lattice cube's exact energies (trilinear
weights, near pairs within r_c left out and their continuum terms).

Run from the repository root:  python tests/golden/make_golden.py [--offlattice-only]
"""
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

from oracle import offlattice, oracle  # noqa: E402
from paper_1403_0711_gb300 import inputs  # noqa: E402

OFF_CASES = [
    # name, L, cube side, seed, jitter, r_c
    ("offcube_128c_n8_q1", (128, 128, 128), 2, 0, 0.3, 1.5),
]

CASES = [
    # name, L, generator, N, seed, method  (two_body: the seed column holds n_x)
    ("plain_16c_n8_pm", (16, 16, 16), "plus_minus", 8, 1, "dense"),
    ("bench_128c_n4096_pm", (128, 128, 128), "plus_minus", 4096, 1, "dst"),
    ("cube_16c_n8_q1", (16, 16, 16), "cube", 8, 0, "dense"),
    ("cube_128c_n8_q1", (128, 128, 128), "cube", 8, 0, "dst"),
    # the paper's Fig. 2 cubes (q = 1, N = 2^3 .. 32^3 at the centre of 128^3)
    ("cube_128c_n64_q1", (128, 128, 128), "cube", 64, 0, "dst"),
    ("cube_128c_n512_q1", (128, 128, 128), "cube", 512, 0, "dst"),
    ("cube_128c_n4096_q1", (128, 128, 128), "cube", 4096, 0, "dst"),
    ("cube_128c_n32768_q1", (128, 128, 128), "cube", 32768, 0, "dst"),
] + [
    # the paper's Fig. 1 pairs: one charge at (L/2, L/2, L/2), the other at (n_x, L/2, L/2)
    (f"twobody_128c_nx{nx}", (128, 128, 128), "two_body", 2, nx, "dst")
    for nx in (65, 66, 68, 72, 80, 96, 112, 127)
]


def charges(gen, L, n, seed):
    if gen == "plus_minus":
        return inputs.plus_minus(L, n, seed)
    if gen == "cube":
        side = round(n ** (1 / 3))
        return inputs.cube(L, side)
    if gen == "two_body":
        return inputs.two_body(L, seed)
    raise ValueError(gen)


def main_offlattice():
    lines = ["# name Lx Ly Lz side seed jitter r_c n_pairs E_far E_direct E_plain continuum_Eq_s1",
             "# E_far: mean of the sample with the near pairs left out; E_direct: their",
             "# continuum terms; E_plain: the interpolated lattice energy with no pairs left out",
             "# written by tests/golden/make_golden.py (FP64 oracle only)"]
    for name, L, side, seed, jitter, rc in OFF_CASES:
        pos, q = inputs.off_lattice_cube(L, side, seed, jitter)
        pairs = offlattice.near_pairs(pos, rc)
        e_far = offlattice.far_energy_solve(L, pos, q, pairs)
        e_dir = offlattice.near_direct_energy(pos, q, pairs)
        e_plain = offlattice.far_energy_solve(L, pos, q, pairs[:0])
        cont = oracle.coulomb_direct(pos, q)
        lines.append(f"{name} {L[0]} {L[1]} {L[2]} {side} {seed} {jitter} {rc} {len(pairs)} "
                     f"{e_far:.15e} {e_dir:.15e} {e_plain:.15e} {cont:.15e}")
        print(lines[-1], flush=True)
    (Path(__file__).resolve().parent / "offlattice.txt").write_text("\n".join(lines) + "\n")


def main():
    main_offlattice()
    if "--offlattice-only" in sys.argv:
        return
    lines = ["# name Lx Ly Lz generator N seed method E_lat continuum_Eq_s1",
             "# written by tests/golden/make_golden.py (FP64 oracle only)"]
    for name, L, gen, n, seed, method in CASES:
        sites, q = charges(gen, L, n, seed)
        e = oracle.e_lat(L, sites, q, method)
        cont = oracle.coulomb_direct(sites, q)
        lines.append(f"{name} {L[0]} {L[1]} {L[2]} {gen} {n} {seed} {method} {e:.15e} {cont:.15e}")
        print(lines[-1], flush=True)
    (Path(__file__).resolve().parent / "e_lat.txt").write_text("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
