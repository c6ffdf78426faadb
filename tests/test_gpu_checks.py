"""The checking build (GV_CHECKS: index and state checks in the kernels that
record GV_ERR_INTERNAL instead of trapping) runs every kernel variant clean,
with integer results identical to the release build's."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2005_00949_gb300 import workloads as W

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cases():
    mixed = W.pbps_mixed(120).subset(120)
    mixed.primaries["E"] = np.minimum(mixed.primaries["E"], 5000.0)
    em3 = W.with_msc(W.with_field(W.pblar_testem3(40, 2000.0), 4.0, 1))
    return [
        ("mixed", mixed, {}),
        ("mixed_fp64", mixed, {"precision": 1}),
        ("nosort", mixed, {"process_sort": 0, "claim_chunks": 1}),
        ("merged_scoring", mixed, {"scoring": 1}),
        ("local_stack", mixed, {"local_stack": 1, "tail_steps_per_claim": 8}),
        ("split", mixed, {"pipeline": 1}),
        ("one_event", mixed, {"mode": 1}),
        ("msc_field", em3, {}),
        ("rejection_integral", W.with_integral(W.with_rejection(mixed)), {}),
        ("cells", W.wsi_cells(20, 20_000.0), {}),
    ]


_RUN = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
sys.path.insert(0, sys.argv[1] + "/tests")
import numpy as np
from paper_2005_00949_gb300 import gv
from test_gpu_checks import _cases
out = {}
for name, wl, kw in _cases():
    ctx = gv.Context(wl, gv.gv_default_config(stack_capacity=1 << 21, per_event_counts=1, **kw))
    try:
        r = ctx.transport(wl, per_event=True)
        out[name] = {"status": r["status"], "counts": r["counts"][:, :11].tolist()}
    except gv.GvError as e:
        out[name] = {"status": str(e)}
    ctx.close()
print(json.dumps(out))
"""


def test_checking_build_runs_clean_and_matches_release():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2005_00949_gb300 import build, gv
    lib = build.build(checks=True, out=os.path.join(ROOT, "paper_2005_00949_gb300", "libgv_checks.so"))
    env = dict(os.environ, GV_LIB=lib)
    res = subprocess.run([sys.executable, "-c", _RUN, ROOT], capture_output=True, text=True, env=env,
                         timeout=900)
    assert res.returncode == 0, res.stderr[-3000:]
    checked = json.loads(res.stdout.strip().splitlines()[-1])
    for name, wl, kw in _cases():
        assert checked[name]["status"] == 0, (name, checked[name]["status"])
        ctx = gv.Context(wl, gv.gv_default_config(stack_capacity=1 << 21, per_event_counts=1, **kw))
        r = ctx.transport(wl, per_event=True)
        ctx.close()
        assert np.array_equal(np.array(checked[name]["counts"]), r["counts"][:, :11]), name
