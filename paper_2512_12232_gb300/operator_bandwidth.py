"""Bandwidth of the stand-alone matrix-free Q4 operator (pf_apply_timing) on a batch of
seeded five-cylinder grids, one JSON line per precision:

    python -m paper_2512_12232_gb300.operator_bandwidth --nx 4096 --ny 2048 \\
        --deltas 0.25,0.5,1.0 --reps 20 --precision mixed

Each measurement runs three untimed launches and then `reps` timed ones on the handle's
own padded vectors; the algorithmic bytes are p read and y written at every node, one
tag byte per node and the stored coefficients of the cells that need them."""
import argparse
import json
import os


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--nx", type=int, default=4096)
    ap.add_argument("--ny", type=int, default=2048)
    ap.add_argument("--sweeps", type=int, default=200)
    ap.add_argument("--deltas", default="0.25,0.5,1.0", help="gap ratios, one grid each")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--precision", choices=["mixed", "fp64", "both"], default="both")
    args = ap.parse_args(argv)
    from . import api, workloads as W
    cases = [W.five_cylinder_case(float(d), args.nx, args.ny, args.sweeps) for d in args.deltas.split(",")]
    precs = {"mixed": [("fp32", api.PF_MIXED)], "fp64": [("fp64", api.PF_FP64)],
             "both": [("fp32", api.PF_MIXED), ("fp64", api.PF_FP64)]}[args.precision]
    peak = None
    try:
        with open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                               "MEASURED_PEAKS.json")) as f:
            peak = json.load(f).get("hbm_gbs")
    except (OSError, ValueError):
        pass
    with api.batch_build(cases) as g:
        nodes = sum(g.stats(v)["n_nodes"] for v in range(len(cases)))
        for name, pr in precs:
            us, by = g.apply_timing(pr, reps=args.reps)
            gbs = by / us / 1e3
            print(json.dumps({"operator": name, "grids": len(cases), "nx": args.nx, "ny": args.ny, "nodes": nodes,
                              "us_per_apply": us, "algorithmic_bytes": by, "GB/s": gbs,
                              "frac_of_measured_hbm": gbs / peak if peak else None}))


if __name__ == "__main__":
    main()
