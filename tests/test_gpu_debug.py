"""The debug build of the library (libpt_debug.so) on every sweep path: in its kernels every
spin-word, count-buffer and trace index is checked before the access and every store of a
half sweep tags its word, so that an out-of-range index or a word stored twice in one half
sweep is recorded (never trapped) and reported through pt_debug_report. These checks stand in
for a memory and race checker on small cases.

The cases run in a child process that loads the debug build (PT_LIBRARY=debug): the plain
path (persistent with a cooperative grid, with a cluster grid, with the plane in shared
memory, with a band of rows per CTA; one launch per half sweep; ferro, field and antiferromagnetic modes; traced), every
batch strategy (dealt, queued, dataflow, cluster) and the allocation-free batch entry point on
a mix of problems, a traced problem in a batch with the batched read, single-spin flips with
both kernels, and a checkpoint round trip. Each must end with no failed check, with every spin
word stored by its own half sweep of the last sweep, and equal to the oracle. Two planted
mistakes -- a word stored twice, a neighbour index past its colour -- must each be caught."""
from __future__ import annotations

import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def outcome():
    from paper_2512_03825_b300 import build as B
    B.build(debug=True)
    env = dict(os.environ, PT_LIBRARY="debug")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "helpers", "debug_paths.py")],
                       capture_output=True, text=True, env=env, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_every_path_passes_the_checks_and_equals_the_oracle(outcome):
    bad = [c for c in outcome["cases"] if not c["ok"]]
    assert not bad, bad
    names = {c["case"] for c in outcome["cases"]}
    for expect in ("persistent cooperative L128 R32", "persistent cluster L32 R40",
                   "persistent shared-memory plane L16 R8", "launches generic L24 R37",
                   "batch dealt", "batch queued", "batch dataflow", "batch cluster",
                   "batch static", "flip shared + sweeps", "flip global + sweeps",
                   "checkpoint load + sweeps", "bands L128 R32", "bands generic uneven L90 R40",
                   "traced bands"):
        assert expect in names


def test_planted_double_write_is_caught(outcome):
    got = outcome["planted"]["1"]
    assert got["report"]["violations"] >= 1
    assert got["report"]["first_kind"] == 3  # a spin word stored twice in one half sweep
    assert got["synchronize_rc"] == -7       # PT_EINTERNAL: the problem is poisoned
    assert "debug build" in got["message"]


def test_planted_index_past_the_colour_is_caught(outcome):
    got = outcome["planted"]["2"]
    assert got["report"]["violations"] >= 1
    assert got["report"]["first_kind"] == 1  # a spin-word load outside its plane and colour
    assert got["synchronize_rc"] == -7
