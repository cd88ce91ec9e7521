"""Writes tests/golden/tiny_oracle.json from the FP64 oracle (and the seeded inputs).

The paper prints no worked example, so this fixture is a regression record of
the oracle on the tiny workload (64x64 pixels, 8 frames, 4 coils, R=4,
lambda=0.01, mu=0.1, rho=0.5): J(0..K) for both priors, ||x|| and the ADMM
residuals of the last iteration.
Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synthdata  # noqa: E402


def main():
    shape = dict(Nx=64, Ny=64, Nt=8, Nc=4)
    iters = 50
    case = synthdata.make_case("tiny", **shape)
    P = oracle.make_problem(case)
    out = dict(shape, iters=iters, lam=case.lam, mu=case.mu, rho=case.rho,
               source="oracle (FP64) on synthdata tiny workload, seed 1")
    for prior in ("tv", "dft"):
        x, info = P.solve(prior, case.lam, case.mu, case.rho, iters)
        out[prior] = dict(J=[float(v) for v in info["J"]], xnorm=float(np.linalg.norm(x)),
                          primal_res=float(info["primal_res"]), dual_res=float(info["dual_res"]))
    with open(os.path.join(HERE, "tiny_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
