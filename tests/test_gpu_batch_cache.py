"""The batch tuner's file cache (fe_batch_tune_cached): a choice timed in one process is read back
by the next one without timing, keyed by device and batch shape, also through FEASM_TUNE_CACHE."""
from __future__ import annotations

import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
sys.path.insert(0, {root!r})
import numpy as np
from paper_1305_3122_gb300 import feasm, meshgen
from tests.gpu_common import assert_values_close
meshes = meshgen.batch_meshes({seed}, count={count}, lo=16, hi=96)
fm = [feasm.Mesh(m.q, m.me) for m in meshes]
fp = [feasm.Pattern(x) for x in fm]
b = feasm.Batch(fm, fp)
block, tile = b.tune(cache={cache!r})
S, M = b.assemble()
S = [t.clone() for t in S]
M = [t.clone() for t in M]
Sp, Mp = b.assemble_plain()
for p, x, y, u, v in zip(fp, S, Sp, M, Mp):
    rp = p.row_ptr.cpu().numpy()
    assert_values_close(rp, x.cpu().numpy(), y.cpu().numpy())
    assert_values_close(rp, u.cpu().numpy(), v.cpu().numpy())
print(json.dumps({{"from_cache": b.from_cache, "config": list(b.config()), "block": block, "tile": tile}}))
"""


def _run(seed, count, cache, env_cache=None):
    env = dict(os.environ)
    env.pop("FEASM_TUNE_CACHE", None)
    if env_cache is not None:
        env["FEASM_TUNE_CACHE"] = env_cache
    code = CHILD.format(root=ROOT, seed=seed, count=count, cache=cache)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_tuning_cache_across_processes(tmp_path):
    path = str(tmp_path / "tune.json")
    first = _run(11, 24, path)
    assert not first["from_cache"]
    assert os.path.exists(path)
    with open(path) as f:
        entries = json.load(f)                        # the file is JSON
    assert len(entries) == 1
    (key, choice), = entries.items()
    assert "|n24|" in key
    assert [choice["variant"], choice["block"], choice["tile"]] == first["config"]
    # a second process: the same choice, read back without timing
    second = _run(11, 24, path)
    assert second["from_cache"] and second["config"] == first["config"]
    # the path from the environment
    third = _run(11, 24, "", env_cache=path)
    assert third["from_cache"] and third["config"] == first["config"]
    # another batch shape is timed and added beside the first entry
    other = _run(12, 10, path)
    assert not other["from_cache"]
    with open(path) as f:
        assert len(json.load(f)) == 2
    again = _run(12, 10, path)
    assert again["from_cache"] and again["config"] == other["config"]


def test_tuning_cache_rejects_unwritable_path(tmp_path):
    from paper_1305_3122_gb300 import feasm, meshgen
    meshes = meshgen.batch_meshes(13, count=3, lo=16, hi=24)
    fm = [feasm.Mesh(m.q, m.me) for m in meshes]
    fp = [feasm.Pattern(x) for x in fm]
    b = feasm.Batch(fm, fp)
    with pytest.raises(feasm.FeasmError) as e:
        b.tune(cache=str(tmp_path / "no_such_dir" / "tune.json"))
    assert e.value.status == 1
    # an unreadable or absent file is just an empty cache
    b2 = feasm.Batch(fm, fp)
    b2.tune(cache=str(tmp_path / "fresh.json"))
    assert not b2.from_cache
    assert np.all([t.numel() > 0 for t in b2.S])
