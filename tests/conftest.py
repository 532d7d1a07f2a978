"""Shared pytest configuration: the ``gpu`` marker and repository paths."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")


#: worst achieved error per result over the session: name -> (error, tolerance, what it is relative to)
_ERRORS = {}


def record_error(result, err, tol, relative_to):
    """Keep the worst error of ``result`` against the FP64 oracle seen in this session; the
    summary at the end lists every result with its tolerance (and a JSON copy goes to the file
    named by the environment variable SXE_PARITY_REPORT, if set)."""
    err = float(err)
    prev = _ERRORS.get(result)
    if prev is None or err > prev[0]:
        _ERRORS[result] = (err, float(tol), relative_to)
    return err


def pytest_terminal_summary(terminalreporter):
    if not _ERRORS:
        return
    import json
    tr = terminalreporter
    tr.write_sep("-", "worst achieved error against the FP64 oracle, per result")
    for name in sorted(_ERRORS):
        err, tol, rel = _ERRORS[name]
        tr.write_line("%-66s %10.3g  tol %8.3g  (%.3f of tol)  vs %s" % (name, err, tol, err / tol if tol else 0.0, rel))
    path = os.environ.get("SXE_PARITY_REPORT")
    if path:
        with open(path, "w") as fh:
            json.dump({k: {"error": v[0], "tolerance": v[1], "relative_to": v[2]} for k, v in sorted(_ERRORS.items())},
                      fh, indent=1)


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def cuda_lib():
    """Build (if needed) and load libsimplexenc on the GPU; fails loudly without CUDA."""
    import torch
    from paper_2311_15439_gb300 import build, _lib
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    _lib.lib()
    return _lib


def rel_err(got, want, den, floor=1e-30):
    """max |got - want| / (den + floor): error measured against the sum of absolute terms."""
    import numpy as np
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    return float(np.max(np.abs(got - want) / (np.asarray(den, dtype=np.float64) + floor))) if got.size else 0.0


#: tolerance of an encoding value against sum_k |w_k H_k|, by output dtype: binary32
#: accumulation of at most 32 terms (1e-5, the stated FP32 bar), or one final rounding
#: to fp16 (unit roundoff 2^-11 -> 2e-3) / bf16 (2^-8 -> 5e-3).
ENC_TOL = {"f32": 1e-5, "f16": 2e-3, "bf16": 5e-3}
#: absolute part of the same bound: below 2^-14 fp16 is subnormal with spacing 2^-24, so
#: one rounding errs by up to 2^-25 regardless of the value (bf16 and binary32 keep the
#: binary32 exponent range: no floor needed at these magnitudes).
ENC_ATOL = {"f32": 0.0, "f16": 2.0 ** -25, "bf16": 0.0}


def worst_ratio(got, want, den, tol, atol=0.0):
    """max |got - want| / (tol * den + atol): <= 1 means within the bound everywhere."""
    import numpy as np
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    bound = tol * np.asarray(den, dtype=np.float64) + atol
    err = np.abs(got - want)
    return float(np.max(np.where(bound > 0, err / np.where(bound > 0, bound, 1.0), np.where(err > 0, np.inf, 0.0))))
