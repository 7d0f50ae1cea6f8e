"""Train the ensemble surrogate for one RVE class on solves of this library.

Training data: macro Gauss points drawn like the batched workload (T ~ U(20,60)
C, moisture ~ U(0,1.5) wt%, t = 10^U(0,4) h), plus --n-aged points of long
exposure (T ~ U(40,60) C, moisture ~ U(0,1.5) wt%, t = 10^U(2,4) h), whose
strongly degraded states the workload distribution reaches only thinly but a
macro structure held hot for long fills; each is solved by the batched
mixed-precision PCG (`macro_update_gauss_points`).  Held-out points from other
seeds, of both kinds, measure the error.  Everything (solves, training,
inference) runs on the GPU through librve.

    python -m paper_1610_03484_gb300.train_surrogate --n-train 20000 --n-aged 6000 --n-test 2000 \
        --out paper_1610_03484_gb300/surrogate_24x24x8_p2.npz
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import rve_inputs as ri  # noqa: E402

import paper_1610_03484_gb300 as rve  # noqa: E402

DEFAULT_OUT = os.path.join(HERE, "surrogate_24x24x8_p2.npz")
TAU = 5e-3          # ensemble-spread gate: larger spread -> fallback to the PCG solve


def rel_err(P, R):
    P = P.reshape(len(P), -1)
    R = R.reshape(len(R), -1)
    return np.linalg.norm(P - R, axis=1) / np.linalg.norm(R, axis=1)


def solve(ctx, mesh, T, c, t):
    Cg, Kg, Dg, st, stats, rc = ctx.macro_update([mesh], T, c, t, np.zeros(len(T), np.int32))
    if not (st == 0).all():
        raise RuntimeError("some training solves did not converge")
    return Cg, Kg, Dg


def load_class(ctx, grid=(24, 24, 8), p=2):
    xyz, tets, phase, tangent = ri.weave_rve(*grid)
    mesh = ctx.mesh_load(xyz, tets, p, phase, tangent)
    mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
    mesh.set_bc(rve.BC_PERIODIC)
    return mesh


def load_surrogate(ctx, path=DEFAULT_OUT):
    z = np.load(path)
    s = rve.Surrogate(ctx, members=int(z["members"]), seed=0)
    s.set_params(z["params"])
    return s


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-train", type=int, default=20000)
    ap.add_argument("--n-aged", type=int, default=6000)
    ap.add_argument("--n-test", type=int, default=2000)
    ap.add_argument("--members", type=int, default=4)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--rtol", type=float, default=1e-7)
    ap.add_argument("--out", default=DEFAULT_OUT)
    args = ap.parse_args(argv)
    ctx = rve.Context(precision=rve.PREC_MIXED, rtol=args.rtol, inner_rtol=min(1e-5, args.rtol))
    mesh = load_class(ctx)
    T, c, t, _, _ = ri.gauss_point_states(args.n_train, seed=3)
    if args.n_aged > 0:
        Ta, ca, ta = ri.aged_states(args.n_aged, seed=13)
        T, c, t = np.concatenate([T, Ta]), np.concatenate([c, ca]), np.concatenate([t, ta])
    Th, ch, th, _, _ = ri.gauss_point_states(args.n_test, seed=4)
    Tq, cq, tq = ri.aged_states(max(1, args.n_test // 4), seed=14)
    t0 = time.perf_counter()
    Cg, Kg, Dg = solve(ctx, mesh, T, c, t)
    t_solve = time.perf_counter() - t0
    Ch, Kh, Dh = solve(ctx, mesh, Th, ch, th)
    Cq, Kq, Dq = solve(ctx, mesh, Tq, cq, tq)
    feat = ctx.features(mesh, T, c, t)
    feat_h = ctx.features(mesh, Th, ch, th)
    feat_q = ctx.features(mesh, Tq, cq, tq)
    s = rve.Surrogate(ctx, members=args.members, seed=7)
    t0 = time.perf_counter()
    hist = s.train(feat, Cg, Kg, Dg, epochs=args.epochs, batch=args.batch, lr=args.lr, seed=5)
    t_train = time.perf_counter() - t0
    Cp, Kp, Dp, spread = s.predict(feat_h)
    errs = np.stack([rel_err(Cp, Ch), rel_err(Kp, Kh), rel_err(Dp, Dh)], axis=1)
    gated = spread <= TAU
    Cpq, Kpq, Dpq, spread_q = s.predict(feat_q)
    errs_q = np.stack([rel_err(Cpq, Cq), rel_err(Kpq, Kq), rel_err(Dpq, Dq)], axis=1)
    gated_q = spread_q <= TAU
    report = {
        "class": "24x24x8 p=2 plain weave, periodic", "n_train": args.n_train, "n_aged": args.n_aged,
        "n_test": args.n_test,
        "members": args.members, "epochs": args.epochs, "solve_s": t_solve, "train_s": t_train,
        "loss_first": float(hist[0]), "loss_last": float(hist[-1]),
        "heldout_rel_err_max": errs.max(axis=0).tolist(), "heldout_rel_err_median": np.median(errs, axis=0).tolist(),
        "gate_tau": TAU, "gated_frac": float(gated.mean()),
        "gated_rel_err_max": errs[gated].max(axis=0).tolist() if gated.any() else None,
        "aged_heldout": {"n": int(len(Tq)), "rel_err_max": errs_q.max(axis=0).tolist(),
                         "gated_frac": float(gated_q.mean()),
                         "gated_rel_err_max": errs_q[gated_q].max(axis=0).tolist() if gated_q.any() else None},
    }
    np.savez_compressed(args.out, params=s.get_params(), members=args.members, report=json.dumps(report))
    print(json.dumps(report))
    return report


if __name__ == "__main__":
    main()
