"""The checked build (libbcm_check.so: index checks on the grid tables in every kernel
that reads them, NaN in every shared-memory tile before it is staged) on grids that
exercise each staged-tile path: same-level, domain and 2:1 faces, FP32 and FP64, the
persistent streaming and two-launch PCG, the multigrid levels, QUICK + Crank-Nicolson
and graph steps.  No check fails (a failure is BCM_E_BOUNDS), no NaN of an unstaged
tile value reaches a result, and the results equal those of the default build."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def run(out, checked):
    env = dict(os.environ)
    env.pop("BCM_CHECK", None)
    if checked:
        env["BCM_CHECK"] = "1"
    r = subprocess.run([sys.executable, os.path.join(HERE, "check_cases.py"), out], env=env,
                       cwd=ROOT, capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert ("libbcm_check.so" in r.stdout) == checked, r.stdout
    return np.load(out)


def test_checked_build_passes_its_checks_and_matches_default(tmp_path):
    sys.path.insert(0, ROOT)
    from paper_1808_04099_gb300 import _build
    _build.build(check=True)  # compiled here, before the timed subprocesses
    plain = run(str(tmp_path / "plain.npz"), False)
    checked = run(str(tmp_path / "checked.npz"), True)
    assert sorted(plain.files) == sorted(checked.files)
    for name in plain.files:
        a, b = plain[name], checked[name]
        assert np.all(np.isfinite(b)), name
        den = np.linalg.norm(a)
        assert np.linalg.norm(a - b) <= 1e-13 * den, (name, np.linalg.norm(a - b) / den)
