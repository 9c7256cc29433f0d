"""The stored oracle samples (tests/golden/) are well formed and match the
workloads they name; the generator script calls only the oracle and the input
generators."""
import json
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def test_full_run_samples_well_formed():
    with open(os.path.join(HERE, "golden", "full_run_samples.json")) as fh:
        d = json.load(fh)
    runs = {r["name"]: r for r in d["runs"]}
    assert set(runs) == {"vortex_256_p3_200", "perturbed_vortex_256_p2_400"}
    for r in runs.values():
        n_modes = (r["p"] + 1) * (r["p"] + 2) // 2
        assert r["shape"] == [2 * r["n"] ** 2, 4, n_modes]
        size = int(np.prod(r["shape"]))
        idx = np.array(r["index"])
        assert idx.size == len(r["value"]) == 1024 and np.all(np.diff(idx) > 0)
        assert idx[0] >= 0 and idx[-1] < size
        assert np.all(np.isfinite(r["value"])) and r["l2_norm"] > 0 and len(r["totals"]) == 4
        assert r["dt"] > 0 and r["steps"] in (200, 400)


def test_generator_uses_only_the_oracle():
    src = open(os.path.join(HERE, "golden", "make_full_run_samples.py")).read()
    imports = set(re.findall(r"^\s*(?:from|import)\s+([\w.]+)", src, flags=re.M))
    assert imports <= {"json", "os", "sys", "numpy", "oracle", "paper_1601_07944_gb300"}
    assert "from paper_1601_07944_gb300 import inputs as I" in src
    assert "dg" not in re.findall(r"from paper_1601_07944_gb300 import (\w+)", src)
