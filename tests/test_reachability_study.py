"""The oracle-side reachability study runs (CPU only, a few evaluations of each optimizer).

The study itself (hundreds of evaluations per instance) stands behind the warm-start reading of
the design notes; this keeps the committed script runnable and its output well formed.
"""
import contextlib
import io
import math
import re

import pytest

from oracle import reachability_study as R


@pytest.mark.parametrize("optimizer", ["adam", "lbfgsb"])
def test_study_runs_and_reports(optimizer):
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        R.main(["--family", "local", "--instance", "0", "--optimizer", optimizer, "--evals", "3"])
    m = re.search(r"done local 0 %s: (\d+) evaluations, final F ([0-9.]+), first F >= 0.999 at evaluation (-?\d+)"
                  % optimizer, buf.getvalue())
    assert m, buf.getvalue()
    n, F = int(m.group(1)), float(m.group(2))
    assert n >= 3 and math.isfinite(F) and 0.0 <= F <= 1.0
