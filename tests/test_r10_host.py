"""Host logic of the R10 study driver (paper_1104_3408_gb300.r10), with the
GPU runs replaced by a fake: the Courant-factor ladder of Tab. dtfac stops at
the first failing factor and reports the bracket, and run summaries keep the
monitored series.  CPU only."""

import math

from paper_1104_3408_gb300 import r10


class _Args:
    ladder = "4.0,4.5,5.0,5.5,6.0"
    n_r = [25]
    n_theta = 9
    t_end = 100.0
    precision = "mixed"


def test_dtfac_ladder_brackets_the_limit(monkeypatch):
    calls = []

    def fake_run_one(n_r, n_theta, t_end, courant=4.0, precision=None, sample_steps=20, **kw):
        calls.append(courant)
        failed = 12.5 if courant > 5.2 else None
        return dict(failed_at=failed, t=t_end if failed is None else failed, rhs_gtt_final=1e-12,
                    seconds=0.0)

    monkeypatch.setattr(r10, "run_one", fake_run_one)
    out = []
    r10.study_dtfac(_Args(), lambda study, rec: out.append((study, rec)))
    assert [c for c in calls] == [4.0, 4.5, 5.0, 5.5]      # stops after the first failure
    (study, rec), = out
    assert study == "dtfac" and rec["grid"] == "25x9x18"
    assert rec["largest_stable"] == 5.0 and rec["smallest_unstable"] == 5.5
    assert rec["paper_lambda_max"] == 6.1


def test_summary_keeps_first_last_and_late_values():
    series = [(0.0, 1e-16), (1.0, 3e-4), (2.0, 1e-4), (8.0, 2e-6), (9.0, 1e-6), (10.0, 5e-7)]
    s = r10._summary(dict(series=series, t=10.0, dt=0.5, steps=20, failed_at=None, seconds=1.0))
    assert s["rhs_gtt_first"] == 3e-4 and s["rhs_gtt_final"] == 5e-7
    assert s["rhs_gtt_max"] == 3e-4 and s["rhs_gtt_late_max"] == 2e-6
    assert s["series_log10"][0] == (0.0, round(math.log10(1e-16), 3))
