"""Write the stored expected values under tests/golden/ (calls only oracle/).

fomlr_2x2x3x2.txt : x = sum_i omega_i (A^2 - sigma_i)^{-1} A b (Algorithm 1 without
                    deflation, A^2 reading of eq. (6.2)), for the seeded inputs listed in
                    its header, computed by the FP64 oracle to tol 1e-13.
kenney_laub_s4.txt: sigma_i, omega_i of eq. (6.2) for s = 4, c = 1.
Run: python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
import seeded_inputs as si  # noqa: E402

DIMS, MU, SPREAD, GSEED, BSEED, S, C, K = (2, 2, 3, 2), 0.3, 0.7, 77, 78, 8, 0.5, 12


def main():
    U = si.random_su3_links(DIMS, SPREAD, GSEED)
    b = si.gaussian_field(DIMS, BSEED)
    sigma, omega = O.kenney_laub(S, C)
    x, rep, _ = O.fom_lr(DIMS, U, b, MU, sigma, omega, k=K, tol=1e-13, max_cycles=5000)
    assert rep["converged"]
    with open(os.path.join(HERE, "fomlr_2x2x3x2.txt"), "w") as f:
        f.write("# Algorithm 1 (restarted multishift FOM, no deflation), A^2 reading of eq. (6.2)\n")
        f.write(f"# dims={DIMS} mu={MU} spread={SPREAD} gauge_seed={GSEED} source_seed={BSEED} "
                f"s={S} c={C} k={K} tol=1e-13 cycles={rep['cycles']}\n")
        for z in x:
            f.write(f"{z.real:.17e} {z.imag:.17e}\n")
    sig4, om4 = O.kenney_laub(4, 1.0)
    with open(os.path.join(HERE, "kenney_laub_s4.txt"), "w") as f:
        f.write("# eq. (6.2): sigma_i = -tan^2(theta_i), omega_i = sec^2(theta_i)/s, theta_i = pi(i-1/2)/(2s); s=4 c=1\n")
        for a, w in zip(sig4, om4):
            f.write(f"{a:.17e} {w:.17e}\n")


if __name__ == "__main__":
    main()
