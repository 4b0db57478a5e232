"""Tuned and learned choices reach dispatch, in this process and in a fresh
one: a cost model and a selection table written to files are loaded
through the environment settings of a new process, the choices it reports
and the variants its calls run follow table > model > built-in rule, and
the results stay oracle-exact on integer inputs.  The library's own
evaluation of an installed network agrees with the trainer's."""
from __future__ import annotations

import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1304_7053_gb300 import inputs, sbgemm, selector

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
D = 1

CHILD = r'''
import json, sys
sys.path.insert(0, ROOT)
import numpy as np
from paper_1304_7053_gb300 import inputs, sbgemm
from tests import gpu_helpers as H
L = sbgemm.lib()
out = {"selector": sbgemm.get_selector(),
       "choice_m10": L.sbgemm_get_choice(1, 10, 10, 10, 0, 0, 1, 3),
       "choice_m12": L.sbgemm_get_choice(1, 12, 12, 12, 0, 0, 1, 3),
       "choice_generic": L.sbgemm_get_choice(0, 7, 3, 11, 0, 0, 1, 3)}
ran = {}
for m in (10, 12):
    b = inputs.UniformBatch("d", "N", "N", m, m, m, 5003, seed=m, int_valued=True)
    got = H.run_gpu(b, 1.5, 0.0)
    ran[m] = L.sbgemm_last_variant()
    H.assert_parity(b, got, H.oracle_ref(b, 1.5, 0.0), 1.5, 0.0, exact=True)
out["ran_m10"], out["ran_m12"] = ran[10], ran[12]
sbgemm.set_selector(sbgemm.SELECTOR_TABLE)
b = inputs.UniformBatch("d", "N", "N", 10, 10, 10, 5003, seed=10, int_valued=True)
H.run_gpu(b, 1.5, 0.0)
out["ran_m10_table_mode"] = L.sbgemm_last_variant()
print(json.dumps(out))
'''


def test_fresh_process_applies_table_and_cost_model(tmp_path):
    F, Hd, V = 16, 64, 9
    n = int(sbgemm.lib().sbgemm_mlp_param_count(F, Hd, V))
    p = np.zeros(n, dtype=np.float32)
    p[n - V + 4] = -3.0               # output bias: variant 4 predicted e^3 times faster
    model = str(tmp_path / "model.txt")
    table = str(tmp_path / "table.txt")
    sbgemm.set_selector(sbgemm.SELECTOR_TABLE)
    sbgemm.clear_choices()
    sbgemm.set_cost_model(F, Hd, V, p, 0.0, 1.0, 0.05)
    sbgemm.save_cost_model(model)
    sbgemm.lib().sbgemm_set_choice(D, 12, 12, 12, 0, 0, 1, 3, 3)
    sbgemm.save_table(table)
    sbgemm.clear_choices()
    env = {k: v for k, v in os.environ.items() if not k.startswith("SBGEMM_")}
    env.update(SBGEMM_COST_MODEL=model, SBGEMM_TABLE=table, SBGEMM_SELECTOR="model")
    r = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT))], env=env,
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["selector"] == [sbgemm.SELECTOR_MODEL, 0]
    assert out["choice_m10"] == 4 and out["ran_m10"] == 4          # the model's choice
    assert out["choice_m12"] == 3 and out["ran_m12"] == 3          # the table wins
    assert out["choice_generic"] == 0                                # fp32: one variant only
    assert out["ran_m10_table_mode"] == sbgemm.default_variant("d", 10, 10, 10, 1, 3)


def test_library_evaluation_matches_trainer():
    """A network trained on synthetic per-variant times, installed in the
    library: for every class with a choice the library's pick equals the
    trainer's ``choose`` on the same features, up to near-ties."""
    rng = inputs.uniform(5, 4000)
    classes = selector.random_classes(300, seed=3)
    feats = np.stack([selector.features(*c) for c in classes])
    # synthetic times: a smooth function of the features plus per-variant offsets
    base = 0.01 * (1 + feats[:, :3].sum(1))[:, None]
    off = 1.0 + 0.3 * np.sin(np.arange(selector.NVAR)[None, :] * (1 + feats[:, 3:4]))
    times = base * off * (1 + 0.01 * rng[:len(classes) * selector.NVAR].reshape(len(classes), -1))
    nv = np.array([sbgemm.num_variants(c[0], c[1], c[2], c[3]) for c in classes])
    times = np.where(np.arange(selector.NVAR)[None, :] < nv[:, None], times, np.nan)
    net = selector.CostModel(seed=1)
    net.fit(feats, times, steps=300)
    margins = {"s": 0.02, "d": 0.0, "c": 0.05, "z": 1.0, "h": 0.1, "b": 0.02}
    sbgemm.clear_choices()
    net.install(margins)
    sbgemm.set_selector(sbgemm.SELECTOR_MODEL)
    try:
        checked = 0
        for dt in selector.DTYPES:
            for m, nn, k in ((8, 8, 8), (10, 10, 10), (16, 16, 16), (4, 16, 4), (16, 16, 15)):
                for ta, tb, bz, sc in ((0, 0, 1, 3), (1, 0, 0, 5), (0, 1, 1, 6)):
                    f = selector.features(dt, m, nn, k, ta, tb, 0, bz, 10 ** (sc + 0.5))[None, :]
                    nvalid = np.array([sbgemm.num_variants(dt, m, nn, k)])
                    dflt = np.array([sbgemm.default_variant(dt, m, nn, k, bz, sc)])
                    margin = margins[dt]
                    want = int(net.choose(f, nvalid, margins, dflt, [dt])[0])
                    got = sbgemm.get_choice(dt, m, nn, k, ta, tb, bz, sc)
                    if got != want:
                        pr = net.predict_rel(f)[0]
                        assert abs(pr[got] - pr[want]) <= 1e-4 * pr[want] or \
                            abs(pr[got] - pr[dflt[0]] * (1 - margin)) <= 1e-4 * pr[got], (dt, m, got, want)
                    checked += 1
        assert checked == 6 * 5 * 3
    finally:
        sbgemm.set_selector(sbgemm.SELECTOR_TABLE)
