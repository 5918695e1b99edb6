"""The synthetic analogues of the paper's plaintext experiments at the paper's
sizes (a few minutes on one core): Table empirical_T on 20 inputs of 151,936
logits, Fig. 5 on 30 inputs of 50,257 logits x 1,000 draws, Fig. 3 on 100
inputs of 50,257 logits.  Prints the tables recorded in the design notes.
Run from the repository root:  python tests/synthetic_experiments.py
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

from test_synthetic_experiments import below_mean_fractions, convergence_table, violation_rates  # noqa: E402


def main():
    tab = convergence_table(151936, range(1000, 1020))
    print("convergence (151,936 logits, 20 inputs): T, best (p, c), mean max Z, max max Z")
    for T, (mean, mx, p, c) in sorted(tab.items()):
        print(f"  T={T}  (p, c) = ({p}, {c})  {mean:.7f}  {mx:.7f}")
    v = violation_rates(50257, range(3000, 3030), draws=1000)
    print("violation rate (p = 0.9, 50,257 logits, 30 inputs x 1,000 draws):")
    print(f"  Gumbel-max {100 * v[:, 0].mean():.2f} % +- {100 * v[:, 0].std():.2f} % "
          f"(1 - nucleus mass {100 * v[:, 2].mean():.2f} %); Beta cut {100 * v[:, 1].mean():.2f} %")
    fr = below_mean_fractions(50257, range(2000, 2100))
    print("fraction below the mean, (p, c) = (19, 27), T = 3 (50,257 logits, 100 inputs):")
    for t in range(fr.shape[1]):
        print(f"  t={t + 1}  {fr[:, t].mean():.5f} +- {fr[:, t].std():.5f}")


if __name__ == "__main__":
    main()
