"""Writes the stored expected values under tests/golden/ from the FP64 oracle.

The paper prints no worked numerical example of the layer, so these fixtures
are the oracle's own outputs on small seeded inputs (Eq. 1-2 with the box
mean of A and b, Sec. 3.2-3.3, and the gradients of Algorithm 1): a
regression record of the pinned oracle that the CPU tests re-derive and the
GPU tests compare the kernels against without running the oracle.  This
script calls only oracle/ and the seeded input generators.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

CASES = {
    # name: (N, C, h_l, w_l, f, r, eps, seed)
    "small_f2_r1": (1, 1, 5, 4, 2, 1, 1e-2, 5),
    "small_f4_r2": (1, 1, 4, 4, 4, 2, 1e-3, 6),
}


def make(name, N, C, hl, wl, f, r, eps, seed):
    d = synth.photo_like(seed, N, C, hl, wl, f)
    R = synth.upstream_grad(seed + 100, d["I_h"].shape)
    p, il, ih = (d[k].numpy() for k in ("p_l", "I_l", "I_h"))
    O = oracle.forward(p, il, ih, r, eps)
    dp, dil, dih = oracle.backward(R.numpy(), p, il, ih, r, eps)
    return {
        "what": "FP64 oracle outputs (Eq. 1-2 with the box mean of A and b; Algorithm 1 gradients of "
                "sum(O_h * R)) on seeded inputs; written by tests/golden/make_golden.py",
        "N": N, "C": C, "h_l": hl, "w_l": wl, "h": hl * f, "w": wl * f, "r": r, "eps": eps,
        "inputs": {"p_l": p.tolist(), "I_l": il.tolist(), "I_h": ih.tolist(), "R": R.numpy().tolist()},
        "expected": {"O_h": O.tolist(), "dp_l": dp.tolist(), "dI_l": dil.tolist(), "dI_h": dih.tolist()},
    }


if __name__ == "__main__":
    for name, args in CASES.items():
        with open(os.path.join(HERE, name + ".json"), "w") as f:
            json.dump(make(name, *args), f)
        print("wrote", name)
