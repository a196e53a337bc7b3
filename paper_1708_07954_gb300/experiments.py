"""The paper's convergence experiments, re-run on the synthetic workloads on one GPU.

    python -m paper_1708_07954_gb300.experiments blocks   # Sec. 4: points / cameras per update step
    python -m paper_1708_07954_gb300.experiments loss     # Sec. 4.1: squared vs Huber misfit
    python -m paper_1708_07954_gb300.experiments rho      # Sec. 4: the consensus penalty
    python -m paper_1708_07954_gb300.experiments solver   # Sec. 3.1: Gauss-Newton vs L-BFGS local solves

Each line printed is one JSON record.  Everything runs through the library's
public API (dba.Solver, dba.BlockSolver); the datasets of the paper are not
used (synthetic scenes from scenes.py stand in for them).
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import sys

from . import build, dba
from . import scenes as S


def _emit(rec):
    print(json.dumps(rec), flush=True)


def block_sweep(n_pts=500000, pis=(1, 8, 32, 64), kappas=(1, 2, 4), target=0.5, max_iters=400, precision=None,
                profile_iters=10):
    """Points and cameras per update step (Sec. 3.1.4, Eq. 14; Sec. 4 sweeps both):
    blocks and copies, device time per iteration, iterations and device time until
    rmse_gt <= target.  The per-observation path (dba.Solver) is the pi = kappa = 1
    reference line."""
    sc = S.scene2(n_pts=n_pts)
    prec = dba.DBA_PREC_F32_LOCAL if precision is None else precision
    with dba.Solver(sc, precision=prec) as s:
        prof = s.profile(profile_iters)
    with dba.Solver(sc, precision=prec) as s:
        m = s.iterate_until(max_iters, target)
    _emit({"experiment": "blocks", "workload": sc.name, "n_obs": sc.n_obs, "path": "per-observation tiles",
           "pi": 1, "kappa": 1, "ms_per_iter": sum(prof.values()), "kernels_ms": prof, "iters": m["iters_done"],
           "seconds": m["seconds"], "rmse_gt": m["rmse_gt"], "reached": m["rmse_gt"] <= target})
    for pi in pis:
        for kappa in kappas:
            with dba.BlockSolver(sc, pi, kappa, precision=prec) as s:
                lay = s.layout()
                lay["blocks_per_size_class"] = s.size_classes()
                prof = s.profile(profile_iters)
            with dba.BlockSolver(sc, pi, kappa, precision=prec) as s:
                m = s.iterate_until(max_iters, target)
            _emit({"experiment": "blocks", "workload": sc.name, "n_obs": sc.n_obs, "path": "blocks", "pi": pi,
                   "kappa": kappa, **lay, "ms_per_iter": sum(prof.values()), "kernels_ms": prof,
                   "iters": m["iters_done"], "seconds": m["seconds"], "rmse_gt": m["rmse_gt"],
                   "reached": m["rmse_gt"] <= target})


def loss_comparison(n_pts=100000, iters=(5, 10, 20, 40, 80, 160), target=0.5, outliers=(0.0, 0.05)):
    """Squared vs Huber misfit (Sec. 4.1 reports faster convergence of the reprojection
    error with the robust loss): rmse_gt after a number of iterations and iterations to
    the target, with and without gross outliers in the pixels."""
    for frac in outliers:
        sc = S.scene2(n_pts=n_pts, outlier_frac=frac)
        for name, loss in (("l2", dba.DBA_LOSS_L2), ("huber", dba.DBA_LOSS_HUBER)):
            scl = dataclasses.replace(sc, loss=loss)
            curve = {}
            with dba.Solver(scl) as s:
                done = 0
                for k in iters:
                    m = s.iterate(k - done)
                    done = k
                    curve[k] = m["rmse_gt"]
            with dba.Solver(scl) as s:
                m = s.iterate_until(max(iters), target)
            _emit({"experiment": "loss", "workload": sc.name, "outlier_frac": frac, "loss": name,
                   "rmse_gt_after": curve, "iters_to_target": m["iters_done"] if m["rmse_gt"] <= target else None,
                   "target_px": target})


def rho_sweep(n_pts=100000, factors=(0.25, 0.5, 1.0, 2.0, 4.0), iters=(10, 50, 200, 1000), target=0.5):
    """The consensus penalty (Sec. 4: a higher rho converged faster on the paper's data;
    Thm. 1 asks for rho large enough): each block's penalty set to `factor` times its
    data curvature; rmse_gt along the run, iterations to the target."""
    sc = S.scene2(n_pts=n_pts)
    for f in factors:
        rx, ry, ra = S.default_rho(sc, f)
        curve = {}
        with dba.Solver(sc, rho_x=rx, rho_y=ry, rho_angle=ra) as s:
            done = 0
            for k in iters:
                m = s.iterate(k - done)
                done = k
                curve[k] = {"rmse_gt": m["rmse_gt"], "primal_res": m["primal_res"]}
        with dba.Solver(sc, rho_x=rx, rho_y=ry, rho_angle=ra) as s:
            m = s.iterate_until(max(iters), target)
        _emit({"experiment": "rho", "workload": sc.name, "rho_factor": f, "curve": curve,
               "iters_to_target": m["iters_done"] if m["rmse_gt"] <= target else None, "target_px": target})


def solver_comparison(n_pts=500000, steps=(1, 2, 5, 10), target=0.5, max_iters=400, profile_iters=10):
    """Local solver of Eq. (9) (Sec. 3.1: Gauss-Newton for l2, L-BFGS for Huber), Huber
    workload 2: device time per iteration and iterations / device time to the target for
    1-10 inner iterations of each."""
    sc = S.scene2(n_pts=n_pts)
    for name, solver in (("gauss-newton", dba.DBA_SOLVER_GN), ("l-bfgs", dba.DBA_SOLVER_LBFGS)):
        for k in steps:
            with dba.Solver(sc, inner_steps=k, local_solver=solver) as s:
                prof = s.profile(profile_iters)
            with dba.Solver(sc, inner_steps=k, local_solver=solver) as s:
                m = s.iterate_until(max_iters, target)
            _emit({"experiment": "solver", "workload": sc.name, "solver": name, "inner_steps": k,
                   "ms_per_iter": sum(prof.values()), "kernels_ms": prof, "iters": m["iters_done"],
                   "seconds": m["seconds"], "rmse_gt": m["rmse_gt"], "reached": m["rmse_gt"] <= target})


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("which", choices=["blocks", "loss", "rho", "solver"])
    ap.add_argument("--n-pts", type=int, default=None)
    args = ap.parse_args(argv)
    build.build()
    dba.load()
    kw = {} if args.n_pts is None else {"n_pts": args.n_pts}
    {"blocks": block_sweep, "loss": loss_comparison, "rho": rho_sweep,
     "solver": solver_comparison}[args.which](**kw)
    return 0


if __name__ == "__main__":
    sys.exit(main())
