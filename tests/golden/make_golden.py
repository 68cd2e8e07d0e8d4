"""Writes the oracle's expected values for small fixed inputs.

Calls only ``oracle/`` (and the seeded scene generators).  Run from the
repository root:  python tests/golden/make_golden.py
The fixtures pin the oracle against accidental change and give the GPU
parity tests fixed expected values that were never produced by the GPU.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1409_7474_gb300 import scenes  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def fixture_inputs():
    """Small inputs: a 12 x 16 rectangle scene and a circle LSF."""
    img, truth, _ = scenes.rect_scene(12, 16, 6, 4, noise=0.05, seed_pos=3,
                                      seed_noise=4)
    phi0 = scenes.circle_phi(12, 16, radius=4.0)
    return img, phi0


def main():
    img, phi0 = fixture_inputs()
    g = oracle.edge_indicator(img, 1.0, 9, 255.0)
    cases = {
        "region_step1": oracle.evolve(img, phi0, "region", iterations=1)[0],
        "region_step5": oracle.evolve(img, phi0, "region", iterations=5)[0],
        "edge_indicator": g,
        "edge_step3": oracle.evolve(img, -phi0, "edge", g=g, iterations=3)[0],
    }
    for name, arr in cases.items():
        path = os.path.join(HERE, f"oracle_{name}_12x16.txt")
        with open(path, "w") as f:
            f.write(f"# oracle output '{name}' for tests/golden/make_golden.py"
                    " fixture_inputs(); 12 rows x 16 columns, %.17g\n")
            np.savetxt(f, arr, fmt="%.17g")
        print("wrote", path)


if __name__ == "__main__":
    main()
