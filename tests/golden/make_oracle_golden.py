"""Writes oracle_small_cases.json: outputs of the FP64 oracle (and nothing else) on small
seeded cases, so that any later change to the oracle's arithmetic shows up in
tests/test_oracle_golden.py and has to be justified by the passage of the paper it follows.

    python tests/golden/make_oracle_golden.py

Cases (arXiv 2501.13382):
  fan_latlong    take-off grid of Sec. 3.3 (Tables 2-3 ranges), 4 x 8 cells: directions, weights
  open_plane     beam summation (Eq. 3 with the beam of Eq. 1 / Eq. 2) of the 1,024-ray open
                 plane at 500 Hz, 16 seeded receivers of the 64 x 64 grid
  city_trace     ray tracing with specular reflection (Sec. 2, Sec. 3.1) of 256 rays through
                 the synthetic city: segment count, per-ray counts, hit primitives
  city_sum       the same trace summed at 8 receivers, 2 frequencies, SEGMENT window
  city_adjoint   gradients of Re sum conj(g) p (derivatives of Eq. 1) for that sum
  city_lossy     the same sum with the atmosphere of the paper's Tables 2-3 (20 C, 70 %,
                 1 atm; ISO 9613-1 absorption) and a porous ground (Delany-Bazley, 200 kPa s
                 m^-2) under hard buildings
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O                      # noqa: E402
from paper_2501_13382_gb300 import inputs as I      # noqa: E402


def cases():
    out = {}
    d, w = O.fan_latlong(4, 8, (0.0, 180.0), (0.0, 360.0))
    out["fan_latlong"] = {"dirs": d.tolist(), "weights": w.tolist()}

    wl = I.open_plane_small()
    idx = I.receiver_subset(wl.receivers, 16, seed=3)
    tr = O.trace(wl.scene, wl.sources[0])
    p = O.gbs_sum(tr, wl.receivers[idx], wl.freqs, wl.beam_b[0], wl.scene.c, wl.scene.gamma,
                  window=wl.window, cutoff=wl.cutoff)
    out["open_plane"] = {"receivers": idx.tolist(), "re": p.real.tolist(), "im": p.imag.tolist()}

    sc, _ = I.city_scene(I.SEED_BASE + 3)
    src = I.Source(np.array([0.0, 0.0, 5.0]), 256, 8, 1000.0)
    tc = O.trace(sc, src)
    out["city_trace"] = {"n_segments": int(tc.n_seg), "counts": np.diff(tc.ray_off).tolist(),
                         "hit": tc.hit.tolist()}
    recv = I.receiver_grid(4, 100.0, 1.5)[[0, 3, 5, 6, 9, 10, 12, 15]]
    freqs, b = [500.0, 1000.0], [30.0, 45.0]
    pc = O.gbs_sum(tc, recv, freqs, b, sc.c, sc.gamma, window=I.WINDOW_SEGMENT)
    out["city_sum"] = {"receivers": recv.tolist(), "freqs": freqs, "b": b,
                       "re": pc.real.tolist(), "im": pc.imag.tolist()}
    g = np.conj(pc) * (1.0 + 0.5j)
    dg, dw, db = O.gbs_adjoint(tc, recv, freqs, b, sc.c, sc.gamma, g, window=I.WINDOW_SEGMENT)
    out["city_adjoint"] = {"grad_gamma": dg.tolist(), "grad_weight_sum": float(dw.sum()),
                           "grad_weight_norm": float(np.linalg.norm(dw)), "grad_b": db.tolist()}
    absorb = O.air_absorption(freqs, 20.0, 70.0, 101.325)
    sigma = np.full(sc.n_materials, -10.0)
    sigma[0] = 200.0
    pl = O.gbs_sum(tc, recv, freqs, b, sc.c, sc.gamma, window=I.WINDOW_SEGMENT,
                   absorption=absorb, sigma=sigma, scene=sc)
    out["city_lossy"] = {"absorption": absorb.tolist(), "re": pl.real.tolist(),
                         "im": pl.imag.tolist()}
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_small_cases.json"), "w") as f:
        json.dump(cases(), f, indent=0)
    print("wrote", os.path.join(HERE, "oracle_small_cases.json"))
