"""Row-group tuner of the split-precision operator launches.

For every shell shape it tunes, each family of tensor-core operator launches
(0 d_r, 1 d_theta with d_phi, 2 phi analysis, 3 projections, 4 phi
synthesis) is tried with 48 and with 96 operator rows per block (48: two
blocks per SM and more row groups; 96: one block per SM), one family after
the other, keeping the faster choice: whole RK4 steps of the shell are timed
with CUDA events on the launching stream (median of the timed steps, L2
flushed before each).  A family whose operator has at most 48 rows keeps 48.
With --write-table the choices are written as the C table
(csrc/tile_table.h) that every new shell of a listed shape takes at
creation; the library needs a rebuild to pick it up.

    python -m paper_1104_3408_gb300.tune [--steps K] [--write-table PATH]

Prints one JSON line per shape (times of every candidate, the choice).
"""

import argparse
import json
import os
import statistics
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FAMILIES = ["d_r", "d_theta_phi", "dft_fwd", "project", "dft_inv"]


def default_shapes():
    """(n_r, n_theta, L, n_fields, r_out) of the benchmarked shells: the
    33 x 48 x 96 and 9 x 12 x 24 shells, the 58-field 65 x 96 x 192 shell and
    the twelve shapes of the uneven-shell batch (L = n_theta - 2)."""
    shapes = [(33, 48, 46, 50, 11.0), (9, 12, 10, 50, 11.0), (65, 96, 94, 58, 41.0)]
    for nt in (16, 24, 32, 48):
        for nr in (17, 25, 33):
            if (nr, nt) != (33, 48):
                shapes.append((nr, nt, nt - 2, 50, 11.0))
    return shapes


def family_rows(n_r, N, L):
    """Operator rows of each family: n_r, 2N, 2L + 1, N, 2N."""
    return [n_r, 2 * N, 2 * L + 1, N, 2 * N]


def time_steps(sh, u, torch, steps, flush):
    st = torch.cuda.current_stream()
    v = u.clone()
    for _ in range(2):
        sh.rk4_step(v, 0.0, 1)
    ts = []
    for _ in range(steps):
        flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        sh.rk4_step(v, 0.0, 1)
        b.record(st)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def tune_shape(cf, inputs, torch, shape, steps, flush):
    n_r, N, L, nf, r_out = shape
    sh = cf.Shell(n_r, N, 2 * N, 1.8, r_out, L, n_fields=nf, precision=cf.MIXED)
    u = torch.from_numpy(inputs.kerr_schild_state(n_r, N, 2 * N, 1.8, r_out, n_fields=nf, amp=1e-4,
                                                  ell=4, seed=0)).cuda()
    sh.init_gauge_from_state(u)
    v = torch.empty_like(u)
    sh.filter(u, v)
    for w in range(len(FAMILIES)):          # start from the rule
        sh.set_operator_rows(w, 0)
    rows = []
    times = {}
    for w, P in enumerate(family_rows(n_r, N, L)):
        if P <= 48:
            sh.set_operator_rows(w, 48)
            rows.append(48)
            continue
        t = {}
        for r in (48, 96):
            sh.set_operator_rows(w, r)
            t[r] = time_steps(sh, v, torch, steps, flush)
        best = min(t, key=t.get)
        sh.set_operator_rows(w, best)
        rows.append(best)
        times[FAMILIES[w]] = t
    rule = []
    for w, P in enumerate(family_rows(n_r, N, L)):
        rule.append(48 if P <= 48 else 96)
    sh.destroy()
    return {"n_r": n_r, "n_theta": N, "L": L, "n_fields": nf, "rows": rows, "rule": rule,
            "ms_per_step": times}


def table_text(results):
    """The C table of the chosen row-group sizes (csrc/tile_table.h)."""
    lines = [
        "// Row-group sizes of the split-precision operator launches, chosen per shell",
        "// shape by timing both candidates (48 or 96 operator rows per CTA) on GB300:",
        "// written by `python -m paper_1104_3408_gb300.tune --write-table`, which",
        "// times whole RK4 steps of each shape with CUDA events for every candidate",
        "// of every operator family and keeps the fastest.  Shapes not listed take",
        "// the rule (48 rows up to 48 operator rows, else 96).  Families: d_r,",
        "// d_theta + d_phi, phi analysis, projections, phi synthesis.",
        "#pragma once",
        "",
        "namespace cffyn {",
        "",
        "struct TileEntry {",
        "  int n_r, n_theta, L, n_fields, filter_kind;",
        "  int rows[5];",
        "};",
        "",
        "static const TileEntry kTileTable[] = {",
    ]
    for r in results:
        rows = ", ".join(str(x) for x in r["rows"])
        lines.append(f"    {{{r['n_r']}, {r['n_theta']}, {r['L']}, {r['n_fields']}, 0, {{{rows}}}}},")
    lines += ["    {0, 0, 0, 0, 0, {0, 0, 0, 0, 0}},  // end of table", "};", "", "}  // namespace cffyn", ""]
    return "\n".join(lines)


def write_table(results, path):
    with open(path, "w") as fh:
        fh.write(table_text(results))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=7)
    ap.add_argument("--write-table", default=None)
    args = ap.parse_args()
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1104_3408_gb300 import cffyn, inputs
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    results = []
    for shape in default_shapes():
        r = tune_shape(cffyn, inputs, torch, shape, args.steps, flush)
        results.append(r)
        print(json.dumps(r), flush=True)
        torch.cuda.empty_cache()
    if args.write_table:
        write_table(results, args.write_table)


if __name__ == "__main__":
    main()
