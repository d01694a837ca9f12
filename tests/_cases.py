"""Small seeded parity cases shared by the GPU tests (inputs only)."""
import numpy as np

import workloads as W

# name -> dict(N, npml, nb, overlap, medium, cuts)
CASES = {
    # the tiny configuration: 128^2, 2x2 boxes of width 104
    "tiny": dict(N=128, npml=16, nb=2, overlap=8, medium="homogeneous", cuts=None, seed=0),
    # ragged: uneven cuts, odd box widths (GEMV tail), random medium, 3x3 boxes
    "ragged": dict(N=100, npml=8, nb=3, overlap=5, medium="random", cuts=[8, 8 + 29, 8 + 71, 108], seed=5),
    # 4x4 boxes over three layers
    "layers4": dict(N=128, npml=16, nb=4, overlap=8, medium="three_layer", cuts=None, seed=1),
    # boxes wider than 128 (160, 178, 150): the factorisation's bottom-right block and
    # ragged last panels; 178 is the widest box that needs a 178 x 178 Schur block
    "wide": dict(N=360, npml=16, nb=3, overlap=8, medium="random", cuts=[16, 136, 266, 376], seed=9),
}


def velocity(case):
    N, npml = case["N"], case["npml"]
    if case["medium"] == "homogeneous":
        return W.velocity_homogeneous(N, npml)
    if case["medium"] == "three_layer":
        return W.velocity_three_layer(N, npml)
    return W.velocity_random_field(N, npml, seed=case["seed"])


def omega(case, c):
    return 2 * np.pi * float(c.min()) * case["N"] / 10.0


def cuts(case):
    return case["cuts"] if case["cuts"] is not None else W.even_cuts(case["N"], case["npml"], case["nb"])
