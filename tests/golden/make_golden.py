"""Write tests/golden/e_lat.txt: exact lattice energies E_lat of the seeded
workloads, computed by the FP64 oracle only (DST-I spectral solve for G rho,
heat-kernel quadrature for G_ii; dense Cholesky where the box is small).

Run from the repository root:  python tests/golden/make_golden.py
"""
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

from oracle import oracle  # noqa: E402
from paper_1403_0711_gb300 import inputs  # noqa: E402

CASES = [
    # name, L, generator, N, seed, method
    ("plain_16c_n8_pm", (16, 16, 16), "plus_minus", 8, 1, "dense"),
    ("bench_128c_n4096_pm", (128, 128, 128), "plus_minus", 4096, 1, "dst"),
    ("cube_16c_n8_q1", (16, 16, 16), "cube", 8, 0, "dense"),
    ("cube_128c_n8_q1", (128, 128, 128), "cube", 8, 0, "dst"),
]


def charges(gen, L, n, seed):
    if gen == "plus_minus":
        return inputs.plus_minus(L, n, seed)
    if gen == "cube":
        side = round(n ** (1 / 3))
        return inputs.cube(L, side)
    raise ValueError(gen)


def main():
    lines = ["# name Lx Ly Lz generator N seed method E_lat continuum_Eq_s1",
             "# written by tests/golden/make_golden.py (FP64 oracle only)"]
    for name, L, gen, n, seed, method in CASES:
        sites, q = charges(gen, L, n, seed)
        e = oracle.e_lat(L, sites, q, method)
        cont = oracle.coulomb_direct(sites, q) if n <= 4096 else float("nan")
        lines.append(f"{name} {L[0]} {L[1]} {L[2]} {gen} {n} {seed} {method} {e:.15e} {cont:.15e}")
        print(lines[-1], flush=True)
    (Path(__file__).resolve().parent / "e_lat.txt").write_text("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
