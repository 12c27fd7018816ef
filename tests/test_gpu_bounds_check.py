"""The index-checked build (SAA_BOUNDS_CHECK, libsaa_bounds.so).

A child process loads the checked library (SAA_BOUNDS_CHECK=1) and runs the
tensor-core value, gradient and streamed paths on shapes that cover every
cluster size of the gradient kernel and both streamed precisions.  Its
results must equal the normal build's bit for bit (the checks change no
arithmetic) with the error word clear, and its index-check self-test must be
flagged on the next sync, with the context still usable afterwards.  The
self-test stores past the declared capacity of an array twice that size, so
even a build without the checks writes nowhere it should not."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from helpers import make
from paper_2404_11631_gb300 import inputs

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [("eval", 128, 20_000, 256, "f16x3"), ("eval", 256, 5_000, 64, "bf16x3"), ("eval", 64, 3_001, 5, "f16x3"),
         ("grad", 1024, 4_096, 64, "f16x3"), ("grad", 300, 3_000, 17, "f16x3"), ("grad", 130, 2_000, 9, "bf16x3"),
         ("samples", 128, 20_000, 64, "f16x3"), ("samples", 100, 9_999, 33, "fp8x")]


def run_cases(out_path):
    """Runs CASES with whichever library saa.lib() loads; saves every output."""
    from paper_2404_11631_gb300 import saa
    res = {"checked": np.array([saa.saa_bounds_check_enabled()])}
    for n, (kind, d, N, K, prec) in enumerate(CASES):
        X = torch.tensor(inputs.decisions(K, d, seed=d), device="cuda")
        if kind == "samples":
            R, inst = inputs.sample_matrix(N, d, seed=d)
            R64 = R.astype(np.float64)
            out = saa.saa_eval_samples(torch.from_numpy(R).cuda(), X, 0.5, prec,
                                       center=torch.tensor(R64.mean(axis=0), device="cuda"),
                                       sigma=torch.tensor(R64.std(axis=0) + 1e-30, device="cuda"))
        else:
            gp, op, inst = make(d, N, seed=d)
            out = saa.saa_eval(gp, X, prec) if kind == "eval" else saa.saa_grad(gp, X, prec)
        saa.saa_ctx_sync()
        for k, v in out.items():
            if torch.is_tensor(v) and k != "ws":
                res[f"{n}_{k}"] = v.cpu().numpy()
    np.savez(out_path, **res)


CHILD = r"""
import os, sys
sys.path.insert(0, sys.argv[1])
sys.path.insert(0, os.path.join(sys.argv[1], "tests"))
from test_gpu_bounds_check import run_cases
from paper_2404_11631_gb300 import saa
run_cases(sys.argv[2])
saa.saa_selftest_bounds()
try:
    saa.saa_ctx_sync()
    print("SELFTEST not flagged")
except saa.SAAError as e:
    print("SELFTEST status", e.status)
saa.saa_ctx_sync()   # the word was cleared: the context is usable
print("AFTER ok")
"""


def test_checked_build_matches_and_flags(tmp_path):
    from paper_2404_11631_gb300 import saa
    ref_path, chk_path = str(tmp_path / "ref.npz"), str(tmp_path / "chk.npz")
    run_cases(ref_path)
    env = dict(os.environ, SAA_BOUNDS_CHECK="1")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, chk_path], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    assert f"SELFTEST status {saa.SAA_EDEVICE}" in r.stdout, r.stdout
    assert "AFTER ok" in r.stdout
    ref, chk = np.load(ref_path), np.load(chk_path)
    assert int(ref["checked"][0]) == 0 and int(chk["checked"][0]) == 1
    keys = [k for k in ref.files if k != "checked"]
    assert keys and sorted(keys) == sorted(k for k in chk.files if k != "checked")
    for k in keys:
        assert np.array_equal(ref[k], chk[k]), k


def test_normal_build_refuses_the_selftest():
    from paper_2404_11631_gb300 import saa
    assert not saa.saa_bounds_check_enabled()
    with pytest.raises(saa.SAAError) as e:
        saa.saa_selftest_bounds()
    assert e.value.status == saa.SAA_EUNSUPPORTED
