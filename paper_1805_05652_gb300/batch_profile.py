"""Phase profile of an uneven batch: plans the uneven workload's instances
(optionally only one window and one N_SFT range), runs the batch once phase
by phase through fmap_batch_profile (direct launches, outside the graph, so
a profiler sees every phase kernel as an ordinary launch) and prints the
device milliseconds of each phase.

    python -m paper_1805_05652_gb300.batch_profile --instances 256 \\
        --window exp --n-sft 4822 9000
"""

import argparse
import json


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--instances", type=int, default=256,
                    help="instances of the uneven workload to draw before filtering")
    ap.add_argument("--window", choices=["rect", "exp", "both"], default="both")
    ap.add_argument("--n-sft", type=int, nargs=2, default=(0, 1 << 30), metavar=("MIN", "MAX"),
                    help="keep instances with MIN <= N_SFT <= MAX")
    ap.add_argument("--budget-gb", type=float, default=24.0)
    args = ap.parse_args(argv)

    import torch
    import synth

    from . import Batch, build

    build()
    dev = torch.device("cuda", 0)
    keep = {"rect": (synth.RECT,), "exp": (synth.EXP,), "both": (synth.RECT, synth.EXP)}
    specs = [s for s in synth.config_uneven(n_instances=args.instances)
             if s["window"] in keep[args.window] and args.n_sft[0] <= s["n_sft"] <= args.n_sft[1]]
    insts = [synth.instance_from_spec(s) for s in specs]
    items = [(i.grid, torch.from_numpy(i.t).to(dev), torch.from_numpy(i.antenna).to(dev),
              torch.from_numpy(i.fafb).to(dev)) for i in insts]
    batch = Batch(items, want_map=True, workspace_budget=int(args.budget_gb * (1 << 30)),
                  autotune=False)
    phases = batch.profile()
    torch.cuda.synchronize()
    print(json.dumps({"instances": len(insts), "info": batch.info(), "status": batch.status(),
                      "phases_ms": {k: round(v, 3) for k, v in phases.items()}}))
    batch.close()


if __name__ == "__main__":
    main()
