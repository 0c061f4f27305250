"""Write the shipped tuning table: the autotuner's choice (ftoep_autotune: block length x
scheduler x internal streams) for the benchmark workloads, keyed like the user cache
(ftoep.tuning_key: device name and the multiset of (N bucket, M bucket, precision, kind,
space)).  Run on the GPU the table is for:

    python -m paper_1710_11593_gb300.tune_table [output.json]

ftoep.autotune_cached reads this table (read-only) when the user's cache has no entry.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

TABLE = os.path.join(HERE, "tuned_gb300.json")


def workloads():
    from paper_1710_11593_gb300 import ftoep, workloads as wl
    out = {}
    batch = wl.config_batched()
    for prec, name in ((ftoep.MIXED, "batched512_mixed"), (ftoep.FP64, "batched512_fp64")):
        out[name] = [ftoep.ProblemSpec(p.kind, p.gamma, p.N, p.M, p.space, prec) for p in batch]
    d = wl.config_diffusion()
    out["diffusion_fp64"] = [ftoep.ProblemSpec(d.kind, d.gamma, d.N, d.M, d.space, ftoep.FP64)]
    w = wl.config_wave()
    out["wave_mixed"] = [ftoep.ProblemSpec(w.kind, w.gamma, w.N, w.M, w.space, ftoep.MIXED)]
    return out


def main(path=TABLE):
    import torch
    from paper_1710_11593_gb300 import ftoep
    ftoep.load()
    device = torch.cuda.get_device_name()
    table = {}
    for name, specs in workloads().items():
        tuning = ftoep.ftoep_autotune(specs)
        table[ftoep.tuning_key(specs, device)] = dict(tuning, workload=name)
        print(name, tuning, flush=True)
    with open(path, "w") as fh:
        json.dump(table, fh, indent=1, sort_keys=True)
    return 0


if __name__ == "__main__":
    sys.exit(main(*sys.argv[1:]))
