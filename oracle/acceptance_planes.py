"""Acceptance planes per site word of the sweep, counted by the oracle.

A site word draws its random stream lazily (Sec. 2 step 3 reading: 32
same-colour sites share each Philox word; the proposal takes B words, the
acceptance words follow and are drawn only while a site of the word is
undecided), so the number of Philox calls the oracle's sweep draws for a word
is the number that word's deepest site needs, in whole calls of four words.
This script runs a constant-step schedule (by default the plain at-scale one:
q = 10, L = 64, beta 0 -> 1.6 in 200 steps, theta = 10) on a sample of the
population with the oracle and prints, per step, the mean acceptance planes per
site word: 4 x (calls per word) - B.  It uses only the oracle.

    python oracle/acceptance_planes.py [R_sample [q L K beta_end theta]] > profiles/acceptance_planes_q<q>-L<L>.txt
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402


def main(R=64, q=10, L=64, K=200, beta_end=1.6, theta=10, seed=1):
    B = oracle.state_bits(q)
    words = 2 * oracle.colour_words(L) * theta  # site-word updates per replica and step
    betas = np.array([beta_end * i / K for i in range(K + 1)])
    spins = oracle.init_random(q, L, 0, R, seed)
    E = np.array([oracle.energy(s) for s in spins], dtype=np.int32)
    args = f"{R}" if (q, L, K, beta_end, theta) == (10, 64, 200, 1.6, 10) else f"{R} {q} {L} {K} {beta_end} {theta}"
    print(f"# command: python oracle/acceptance_planes.py {args} > profiles/acceptance_planes_q{q}-L{L}.txt")
    print(f"# acceptance planes per site word, oracle count: q={q} L={L} R={R} (a sample of the population)")
    print(f"# theta={theta}, beta 0 -> {beta_end} in {K} steps, nearest-integer resampling, seed {seed}")
    print("# step beta planes_per_word")
    for i in range(1, K + 1):
        r, _, _, _ = oracle.copy_numbers(E, betas[i] - betas[i - 1], R, oracle.NEAREST_INT, i, seed)
        spins = spins[oracle.parents(r)]
        calls = 0
        new = []
        for slot, s in enumerate(spins):
            s2, c = oracle.sweep_replica(q, s, betas[i], theta, i, slot, seed, with_calls=True)
            new.append(s2)
            calls += c
        spins = np.array(new)
        E = np.array([oracle.energy(s) for s in spins], dtype=np.int32)
        print(f"{i} {betas[i]:.6f} {4.0 * calls / (len(spins) * words) - B:.4f}", flush=True)


if __name__ == "__main__":
    a = sys.argv[1:]
    kw = {}
    if a:
        kw["R"] = int(a[0])
    if len(a) >= 6:
        kw.update(q=int(a[1]), L=int(a[2]), K=int(a[3]), beta_end=float(a[4]), theta=int(a[5]))
    main(**kw)
