"""What the rank predictor gains in assembly, on fresh meshes.

Trains the predictor on the probe logs of plain assemblies (the crater
bowl and seeded fBm terrains of 5k-80k facets, the meshes the batching
workload uses), then assembles fresh meshes twice, once on the plain probe
path and once with the predictor, and reports per mesh: assembly time,
probe time, probes run, probes skipped by the predictor, compressed bytes,
and the relative difference of the two matrices' products with E (both
paths meet the tolerance, so it stays below 2 tol).

    python -m paper_2209_07632_gb300.predictor_eval [--quick]

Prints one JSON line.  --quick uses smaller meshes (for a fast check).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--epochs", type=int, default=30)
    a = ap.parse_args()
    import torch

    import synth
    from paper_2209_07632_gb300 import vf

    tol = 1e-3
    train_sides = [51, 70, 90, 120] if a.quick else [51, 80, 110, 140, 170, 200]
    t0 = time.time()
    Xs, ys = [], []
    v, f = synth.cap_bowl_mesh()
    prob = vf.build_problem(v, f, tol=tol, precisions=("fp32",))
    X, y = vf.vf_hmat_probe_log(prob.hmat)
    Xs.append(X)
    ys.append(y)
    for k, side in enumerate(train_sides):
        v, f = synth.fbm_dem_mesh(n=side, seed=100 + k, crater_diameter=1000.0 if k % 2 == 0 else None)
        prob = vf.build_problem(v, f, tol=tol, precisions=("fp32",))
        X, y = vf.vf_hmat_probe_log(prob.hmat)
        Xs.append(X)
        ys.append(y)
        del prob
    X, y = np.concatenate(Xs), np.concatenate(ys)
    t_data = time.time() - t0
    p = vf.vf_predictor_create(seed=1)
    t1 = time.time()
    loss = vf.vf_predictor_train(p, X, y, epochs=a.epochs, batch=512, lr=2e-3)
    t_train = time.time() - t1
    cls, _ = vf.vf_predictor_predict(p, X)
    train_acc = float(np.mean(cls == y))

    evals = []
    cases = [("fbm256_seed3" if not a.quick else "fbm100_seed3", "quad",
              synth.fbm_dem_mesh(n=256 if not a.quick else 100, spacing=10.0, seed=3, crater_diameter=None)),
             ("gaussian_sphere_l6" if not a.quick else "gaussian_sphere_l5", "oct",
              synth.gaussian_sphere_mesh(level=6 if not a.quick else 5))]
    for name, kind, (v, f) in cases:
        m = vf.vf_mesh_create(v, f)
        t = vf.vf_partition(m, kind, 64)
        res = {"mesh": name, "facets": m.n, "tree": kind}
        out = {}
        for label, pred in (("plain", None), ("predictor", p)):
            torch.cuda.synchronize()
            s0 = time.time()
            h, st = vf.vf_assemble(m, t, tol=tol, precisions=("fp32",), predictor=pred)
            torch.cuda.synchronize()
            wall = time.time() - s0
            res[label] = {"assembly_s": round(wall, 3), "t_probe_s": round(st["t_probe"], 3),
                          "probes": st["probes"], "probes_failed": st["probes_failed"],
                          "probes_predicted_skip": st["probes_predicted_skip"],
                          "predictor_audits": st["predictor_audits"],
                          "predictor_audit_wins": st["predictor_audit_wins"],
                          "predictor_fallbacks": st["predictor_fallbacks"],
                          "bytes_fp32": vf.vf_hmat_bytes(h, "fp32"), "blocks": st["nblocks"]}
            dirs = synth.sun_directions(8, 10.0)
            E = torch.empty((8, m.n), device="cuda")
            vf.vf_mesh_insolation(m, dirs, 1365.0, E)
            Y = torch.empty_like(E)
            vf.vf_apply(h, E, Y)
            out[label] = Y.double()
            del h
        d = ((out["predictor"] - out["plain"]).norm(dim=1) / out["plain"].norm(dim=1)).max().item()
        res["apply_rel_diff_vs_plain"] = d
        res["probe_time_ratio"] = round(res["predictor"]["t_probe_s"] / max(res["plain"]["t_probe_s"], 1e-9), 3)
        res["bytes_ratio"] = round(res["predictor"]["bytes_fp32"] / res["plain"]["bytes_fp32"], 4)
        evals.append(res)
    print(json.dumps({"train": {"samples": int(len(y)), "class_counts": np.bincount(y, minlength=6).tolist(),
                                "final_loss": loss, "train_accuracy": train_acc, "data_s": round(t_data, 1),
                                "train_s": round(t_train, 2), "epochs": a.epochs},
                      "tol": tol, "eval": evals}))


if __name__ == "__main__":
    main()
