"""Long evolutions of the benchmark shells: the mixed path beside the plain FP64
path, with the constraint norms tracked.

    python -m paper_1104_3408_gb300.evolve [--workload ks_33x48x96] [--steps N] [--every K]

Workloads (inputs.WORKLOADS): the 33 x 48 x 96 shell with 50 fields (1000 RK4
steps by default) and the 65 x 96 x 192 shell with 58 fields (200 steps).
Each path: shell created, gauge source from the state (H_a = -Gamma_a,
eq. gauge; written into the state for 58 fields), initial data filtered once
(the per-substep filter placement of Sec. 2.5 then keeps the state in the
filter's range), then `steps` RK4 steps (cffyn_rk4_step, one CUDA graph per
step) in chunks of `every`.  After each chunk: the RMS of the constraints
C_iab = d_i g_ab - Phi_iab and C_a = H_a + Gamma_a (App. A.1,
cffyn_constraint_norms) on both paths, and the max-norm difference of the two
states relative to the FP64 one.  Prints one JSON line.  Every step runs in the
CUDA library; torch holds the arrays and reduces the state difference.
"""

import argparse
import json
import sys
import time

from . import cffyn, inputs


def _shell(w, precision):
    return cffyn.Shell(w["n_r"], w["n_theta"], w["n_phi"], w["r_in"], w["r_out"], w["L"],
                       n_fields=w["n_fields"], precision=precision)


def _prepare(sh, u0, device):
    import torch
    u = torch.from_numpy(u0).to(device)
    sh.init_gauge_from_state(u)
    uf = torch.empty_like(u)
    sh.filter(u, uf)
    return uf


def run(workload="ks_33x48x96", steps=None, every=10, fp64=True, device="cuda"):
    import torch
    w = dict(inputs.WORKLOADS[workload])
    steps = steps or w["steps"]
    u0 = inputs.kerr_schild_state(w["n_r"], w["n_theta"], w["n_phi"], w["r_in"], w["r_out"],
                                  n_fields=w["n_fields"], amp=w["amp"], ell=w["ell"], seed=w["seed"])
    paths = {"mixed": cffyn.MIXED}
    if fp64:
        paths["fp64"] = cffyn.FP64
    shells = {k: _shell(w, p) for k, p in paths.items()}
    dt = w["lam"] / 0.25 * shells["mixed"].default_dt()
    states = {k: _prepare(sh, u0, device) for k, sh in shells.items()}
    rec = {k: {"constraint_norms": [[0] + list(sh.constraint_norms(states[k]))], "seconds": 0.0}
           for k, sh in shells.items()}
    diff = []
    done = 0
    while done < steps:
        k = min(every, steps - done)
        for name, sh in shells.items():
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sh.rk4_step(states[name], dt, k)
            torch.cuda.synchronize()
            rec[name]["seconds"] += time.perf_counter() - t0
        done += k
        for name, sh in shells.items():
            rec[name]["constraint_norms"].append([done] + list(sh.constraint_norms(states[name])))
        if fp64:
            a, b = states["mixed"], states["fp64"]
            diff.append([done, float((a - b).abs().max() / b.abs().max())])
    out = {"workload": workload, "n_r": w["n_r"], "n_theta": w["n_theta"], "n_phi": w["n_phi"],
           "n_fields": w["n_fields"], "L": w["L"], "dt": dt, "steps": steps, "every": every}
    for name in shells:
        r = rec[name]
        out[name] = {"ms_per_step_wall": 1e3 * r["seconds"] / steps,
                     "constraint_norms": r["constraint_norms"]}
    if fp64:
        out["rel_diff_mixed_vs_fp64"] = diff
    for sh in shells.values():
        sh.destroy()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", default="ks_33x48x96",
                    choices=["ks_9x12x24", "ks_33x48x96", "ks_65x96x192_58f"])
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--every", type=int, default=10)
    ap.add_argument("--no-fp64", action="store_true")
    a = ap.parse_args(argv)
    cffyn.load()
    print(json.dumps(run(a.workload, a.steps, a.every, not a.no_fp64)), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
