"""Writes precision_reduced.json: the FP64 oracle's BSGD-TV trajectory on the
reduced precision workload (synth.PRECISION_REDUCED: the 512^3 / 720 x 512^2
configuration at 1/8 resolution, 16 x 16 blocks, lambda = 1e-3, Algorithm 4),
kept as the image after every epoch at seeded sample voxels, with the step mu
(rho / max_J ||A^J||^2 by the oracle's power iteration) and the data's norm.

Calls only oracle/ (and the seeded input generators); run from the repository
root:  python tests/golden/make_precision_reduced.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import bsgd as OB  # noqa: E402
from oracle import projector as OP  # noqa: E402
from paper_1903_11874_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "precision_reduced.json")


def main():
    w = synth.PRECISION_REDUCED
    og = OP.Geometry(**w["geometry"])
    xt = synth.precision_reduced_phantom().reshape(-1).astype(np.float64)
    y = OP.fp(og, xt).reshape(-1).astype(np.float32).astype(np.float64)
    mu = OB.step_strip(og, w["N"], w["rho"], w["power_iters"])
    prm = OB.Params(w["M"], w["N"], 1 / w["M"], 1 / w["N"], mu, seed=w["seed"],
                    tv_lambda=w["tv_lambda"], tv_iters=w["tv_iters"])
    idx = synth.sample_indices(og.n_cols, w["n_samples"], w["sample_seed"])
    st = OB.BSGDState(og, y, prm)
    per_epoch, norms, resid = [], [], []
    for _ in range(w["epochs"]):
        for _ in range(prm.epoch_len):
            st.step()
        per_epoch.append([float("%.10e" % v) for v in st.x[idx]])
        norms.append(float(np.linalg.norm(st.x)))
        resid.append(st.residual_norm())
    out = {
        "what": "FP64 oracle (oracle/bsgd.py, Algorithm 4 with the prox weight of Eq. (TVequ)) "
                "on synth.PRECISION_REDUCED: image at the sample voxels after each epoch",
        "mu": mu, "y_norm": float(np.linalg.norm(y)), "sample_indices": [int(i) for i in idx],
        "x_samples": per_epoch, "x_norm": norms, "residual_norm": resid,
    }
    with open(OUT, "w") as f:
        json.dump(out, f, separators=(",", ":"))


if __name__ == "__main__":
    main()
