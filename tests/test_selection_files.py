"""Host-only checks of variant selection across processes: the selection
table and cost-model files round-trip through the C ABI, malformed files
are rejected without side effects, the selector modes decide which source
a class's choice comes from, and the environment settings are applied in a
fresh process.  No GPU: the cost model is installed while the mode is not
MODEL, so it is not evaluated here (the GPU test does that)."""
from __future__ import annotations

import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1304_7053_gb300 import sbgemm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
S, D, C, Z, H, B = range(6)


@pytest.fixture(autouse=True)
def clean_state():
    sbgemm.set_selector(sbgemm.SELECTOR_TABLE)
    sbgemm.clear_choices()
    yield
    sbgemm.set_selector(sbgemm.SELECTOR_TABLE)
    sbgemm.clear_choices()


ENTRIES = [(S, 10, 10, 10, 0, 0, 1, 5, 4), (D, 16, 16, 16, 1, 0, 0, 6, 3),
           (H, 12, 12, 12, 0, 0, 1, 6, 0), (C, 9, 16, 9, 1, 0, 0, 5, 6)]


def test_table_file_round_trip(tmp_path):
    L = sbgemm.lib()
    for e in ENTRIES:
        assert L.sbgemm_set_choice(*e) == 0
    p = str(tmp_path / "table.txt")
    sbgemm.save_table(p)
    lines = open(p).read().splitlines()
    assert lines[0] == "sbgemm-table 1" and lines[1].startswith("device ")
    sbgemm.clear_choices()
    for e in ENTRIES:
        assert L.sbgemm_get_choice(*e[:8]) == L.sbgemm_default_variant(e[0], e[1], e[2], e[3], e[6], e[7])
    sbgemm.load_table(p)
    for e in ENTRIES:
        assert L.sbgemm_get_choice(*e[:8]) == e[8]
    p2 = str(tmp_path / "table2.txt")
    sbgemm.save_table(p2)
    assert open(p2).read() == open(p).read()


@pytest.mark.parametrize("body", [
    "sbgemm-table 2\n",                                    # unknown version
    "not a table\n0 10 10 10 0 0 1 5 4\n",                # no header
    "sbgemm-table 1\n0 10 10 10 0 0 1 5 99\n",            # variant out of range
    "sbgemm-table 1\n0 17 10 10 0 0 1 5 0\n",             # m out of range
    "sbgemm-table 1\n0 10 10 10 0 0 1 9 0\n",             # size class out of range
    "sbgemm-table 1\n0 10 10 10 0 0 1 5\n",               # missing field
    "sbgemm-table 1\n0 10 10 10 0 0 1 5 2 7\n",           # extra field
])
def test_malformed_table_is_rejected_and_adds_nothing(tmp_path, body):
    p = str(tmp_path / "bad.txt")
    # a valid entry first: nothing of the file may be added
    open(p, "w").write(body if not body.startswith("sbgemm-table 1") else
                       body.replace("sbgemm-table 1\n", "sbgemm-table 1\n3 8 8 8 0 0 0 5 5\n"))
    assert sbgemm.lib().sbgemm_load_table(p.encode()) == -9
    assert sbgemm.lib().sbgemm_get_choice(Z, 8, 8, 8, 0, 0, 0, 5) == \
        sbgemm.lib().sbgemm_default_variant(Z, 8, 8, 8, 0, 5)
    assert sbgemm.lib().sbgemm_load_table(str(tmp_path / "missing.txt").encode()) == -9


def test_selector_modes():
    L = sbgemm.lib()
    assert L.sbgemm_set_choice(S, 10, 10, 10, 0, 0, 1, 5, 4) == 0
    assert L.sbgemm_get_choice(S, 10, 10, 10, 0, 0, 1, 5) == 4
    sbgemm.set_selector(sbgemm.SELECTOR_DEFAULT)
    assert L.sbgemm_get_choice(S, 10, 10, 10, 0, 0, 1, 5) == L.sbgemm_default_variant(S, 10, 10, 10, 1, 5)
    assert sbgemm.get_selector()[0] == sbgemm.SELECTOR_DEFAULT
    sbgemm.set_selector(sbgemm.SELECTOR_TABLE)
    assert L.sbgemm_get_choice(S, 10, 10, 10, 0, 0, 1, 5) == 4
    assert L.sbgemm_set_selector(7) == -5
    # the built-in rule itself
    assert L.sbgemm_default_variant(H, 16, 16, 16, 1, 6) == 7
    assert L.sbgemm_default_variant(H, 12, 12, 12, 1, 6) == 7
    assert L.sbgemm_default_variant(C, 10, 10, 10, 1, 6) == 2
    assert L.sbgemm_default_variant(S, 10, 10, 10, 1, 5) == 2
    assert L.sbgemm_default_variant(S, 10, 10, 10, 1, 6) == 0
    assert L.sbgemm_default_variant(D, 10, 10, 10, 1, 5) == 0
    assert L.sbgemm_default_variant(S, 7, 3, 11, 1, 5) == 0
    assert L.sbgemm_default_variant(S, 17, 3, 11, 1, 5) == -1
    # real fp64 on the tensor cores: m = n = k >= 13, 12 with beta != 0, 16 x 8 x 16
    assert L.sbgemm_default_variant(D, 16, 16, 16, 0, 5) == 7
    assert L.sbgemm_default_variant(D, 13, 13, 13, 1, 5) == 7
    assert L.sbgemm_default_variant(D, 13, 13, 13, 0, 5) == 7
    assert L.sbgemm_default_variant(D, 12, 12, 12, 0, 5) == 7
    assert L.sbgemm_default_variant(D, 12, 12, 12, 1, 5) == 0
    assert L.sbgemm_default_variant(D, 11, 11, 11, 0, 5) == 0
    assert L.sbgemm_default_variant(D, 16, 8, 16, 0, 6) == 7
    assert L.sbgemm_default_variant(D, 9, 16, 9, 0, 6) == 0


def _params(seed=3):
    n = int(sbgemm.lib().sbgemm_mlp_param_count(16, 64, 9))
    return ((np.arange(n) * 2654435761 % 1000003) / 1000003.0 - 0.5).astype(np.float32)


MARGINS6 = {"s": 0.05, "d": 1.0, "c": 0.0, "z": 0.02, "h": 0.1, "b": 0.2}


def test_cost_model_file_round_trip(tmp_path):
    p = _params()
    sbgemm.set_cost_model(16, 64, 9, p, -2.5, 1.25, MARGINS6)
    f1 = str(tmp_path / "model.txt")
    sbgemm.save_cost_model(f1)
    txt = open(f1).read().split("\n")
    assert txt[0] == "sbgemm-cost-model 2" and txt[1].startswith("device ")
    assert txt[2] == "features 16 hidden 64 outputs 9"
    assert txt[3] == "log_time_mean -2.5 log_time_std 1.25"
    assert [float(x) for x in txt[4].split()[1:]] == [MARGINS6[d] for d in "sdczhb"]
    vals = np.array(" ".join(txt[6:]).split(), dtype=np.float32)
    assert np.array_equal(vals, p)                        # 9 digits: exact for fp32
    sbgemm.load_cost_model(f1)
    f2 = str(tmp_path / "model2.txt")
    sbgemm.save_cost_model(f2)
    assert open(f2).read() == open(f1).read()
    # a version-1 file (one margin for every type) loads and saves as version 2
    lines = open(f1).read().split("\n")
    lines[0] = "sbgemm-cost-model 1"
    lines[3] = lines[3] + " margin 0.125"
    del lines[4]
    f3 = str(tmp_path / "model_v1.txt")
    open(f3, "w").write("\n".join(lines))
    sbgemm.load_cost_model(f3)
    sbgemm.save_cost_model(f2)
    assert open(f2).read().split("\n")[4] == "margins" + " 0.125" * 6


def test_cost_model_rejections(tmp_path):
    L = sbgemm.lib()
    p = _params()
    addr = p.ctypes.data
    m0 = np.zeros(6)
    assert L.sbgemm_set_cost_model(15, 64, 9, addr, 0.0, 1.0, m0.ctypes.data) == -5   # F must be 16
    assert L.sbgemm_set_cost_model(16, 64, 9, addr, 0.0, 0.0, m0.ctypes.data) == -5   # std > 0
    for bad_margin in (1.5, -0.1, np.nan):
        mb = np.zeros(6)
        mb[3] = bad_margin
        assert L.sbgemm_set_cost_model(16, 64, 9, addr, 0.0, 1.0, mb.ctypes.data) == -5
    assert L.sbgemm_set_cost_model(16, 64, 9, addr, 0.0, 1.0, None) == -4       # margins NULL
    assert L.sbgemm_set_cost_model(16, 64, 9, addr, 0.0, 1.0, np.ones(6).ctypes.data) == 0
    q = p.copy()
    q[5] = np.nan
    assert L.sbgemm_set_cost_model(16, 64, 9, q.ctypes.data, 0.0, 1.0, m0.ctypes.data) == -5
    sbgemm.set_cost_model(16, 64, 9, p, 0.0, 1.0, 0.0)
    good = str(tmp_path / "m.txt")
    sbgemm.save_cost_model(good)
    text = open(good).read()
    n = int(L.sbgemm_mlp_param_count(16, 64, 9))
    for bad in (text.replace(f"params {n}", f"params {n - 1}"),        # count mismatch
                text.replace("sbgemm-cost-model 2", "sbgemm-cost-model 3"),
                text.replace("margins 0 0 0 0 0 0", "margins 0 0 0 0 0"),  # five margins
                text.replace("margins 0 0 0 0 0 0", "margins 0 0 0 0 0 2"),  # margin above 1
                text.rsplit("\n", 2)[0] + "\n",                          # truncated
                text + "1.0\n"):                                         # trailing value
        assert bad != text
        f = str(tmp_path / "bad.txt")
        open(f, "w").write(bad)
        assert L.sbgemm_load_cost_model(f.encode()) == -9


def test_environment_settings_in_a_fresh_process(tmp_path):
    L = sbgemm.lib()
    assert L.sbgemm_set_choice(S, 10, 10, 10, 0, 0, 1, 5, 4) == 0
    p = str(tmp_path / "t.txt")
    sbgemm.save_table(p)
    code = ("import json, sys; sys.path.insert(0, %r)\n"
            "from paper_1304_7053_gb300 import sbgemm\n"
            "L = sbgemm.lib()\n"
            "print(json.dumps([sbgemm.get_selector(), L.sbgemm_get_choice(0, 10, 10, 10, 0, 0, 1, 5)]))"
            % ROOT)

    def run(**env):
        e = {k: v for k, v in os.environ.items() if not k.startswith("SBGEMM_")}
        e.update(env)
        r = subprocess.run([sys.executable, "-c", code], env=e, capture_output=True, text=True,
                           timeout=120)
        assert r.returncode == 0, r.stderr
        return json.loads(r.stdout.strip().splitlines()[-1])

    dflt = L.sbgemm_default_variant(S, 10, 10, 10, 1, 5)
    assert run() == [[1, 0], dflt]
    assert run(SBGEMM_TABLE=p) == [[1, 0], 4]
    assert run(SBGEMM_TABLE=p, SBGEMM_SELECTOR="default") == [[0, 0], dflt]
    assert run(SBGEMM_TABLE=str(tmp_path / "none.txt")) == [[1, -9], dflt]
    assert run(SBGEMM_SELECTOR="model") == [[1, -5], dflt]        # no model: mode unchanged
