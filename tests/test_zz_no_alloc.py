"""fram_sdsn_static: the SDSN entry point for callers that cannot allocate
device memory (their memory belongs to another allocator, or they cannot
afford cudaFree's device-wide synchronisation).  It must give the same result
as fram_sdsn, which runs the same kernel with context-owned scratch, on two
calls in a row (the static scratch keeps the previous call's contents), and
must reject sizes beyond its static limit with a message.

This file is collected last so that a failure here, under ``-x``, comes after
every other test has run.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import paper_2508_00887_gb300 as fr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2508_00887_gb300 import build
    build.build()
    fr.load()
    return torch


@pytest.fixture(scope="module")
def ctx(torch_cuda):
    c = fr.fram_create(0, 0, torch_cuda.cuda.current_stream().cuda_stream)
    yield c
    fr.fram_destroy(c)


def relF(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("n,theta,cap", [(300, 10.0, 200), (1000, 2.0, 50), (97, 2.0, 5000),
                                         (fr.FRAM_SDSN_STATIC_MAX_N, 2.0, 20)])
def test_static_matches_context_entry_twice(torch_cuda, ctx, n, theta, cap):
    torch = torch_cuda
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):                      # two calls in a row share the scratch
        X = np.random.default_rng(100 * n + call).random((n, n)) ** 2
        Xd = torch.from_numpy(X).cuda()
        D_ref = torch.empty_like(Xd)
        D_sta = torch.empty_like(Xd)
        _, sw_ref, g_ref = fr.fram_sdsn(ctx, n, Xd, D_ref, theta, 1e-14, cap)
        st, sw, g, msg = fr.fram_sdsn_static(n, Xd, D_sta, theta, 1e-14, cap, stream)
        assert st == fr.FRAM_OK and msg == ""
        assert sw == sw_ref
        assert relF(D_sta.cpu().numpy(), D_ref.cpu().numpy()) <= 1e-12
        assert abs(g - g_ref) <= 1e-12 * max(1.0, abs(g_ref))


def test_static_rejects_sizes_beyond_limit(torch_cuda):
    torch = torch_cuda
    n = fr.FRAM_SDSN_STATIC_MAX_N + 1
    X = torch.zeros(1, dtype=torch.float64, device="cuda")   # never read: rejected first
    st, _, _, msg = fr.fram_sdsn_static(n, X, X, 2.0, check=False)
    assert st == fr.FRAM_ERR_INVALID
    assert "static scratch limit" in msg and str(fr.FRAM_SDSN_STATIC_MAX_N) in msg


def test_static_in_place(torch_cuda, ctx):
    # D == X: the result overwrites the input, as for fram_sdsn.
    torch = torch_cuda
    n = 1000
    X = np.random.default_rng(77).random((n, n)) ** 2
    Xd = torch.from_numpy(X).cuda()
    D_ref = torch.empty_like(Xd)
    _, sw_ref, g_ref = fr.fram_sdsn(ctx, n, Xd, D_ref, 10.0, 1e-14, 100)
    st, sw, g, _ = fr.fram_sdsn_static(n, Xd, Xd, 10.0, 1e-14, 100,
                                       torch.cuda.current_stream().cuda_stream)
    assert st == fr.FRAM_OK and sw == sw_ref
    assert relF(Xd.cpu().numpy(), D_ref.cpu().numpy()) <= 1e-12
    assert abs(g - g_ref) <= 1e-12 * max(1.0, abs(g_ref))


_FRESH = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import paper_2508_00887_gb300 as fr
fr.load()
n = int(sys.argv[2])
X = torch.from_numpy(np.random.default_rng(5).random((n, n)) ** 2).cuda()
D = torch.empty_like(X)
# the first library call of this process: no context exists
st, sw, g, msg = fr.fram_sdsn_static(n, X, D, 2.0, 1e-14, 40)
assert st == fr.FRAM_OK, msg
np.save(sys.argv[3], D.cpu().numpy())
print(sw, repr(g))
"""


def test_static_needs_no_context(torch_cuda, ctx, tmp_path):
    # A fresh process whose first and only library call is fram_sdsn_static
    # (no fram_create anywhere) gives fram_sdsn's result.
    torch = torch_cuda
    n = 600
    out = tmp_path / "d.npy"
    r = subprocess.run([sys.executable, "-c", _FRESH, ROOT, str(n), str(out)],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    sw, g = r.stdout.split()
    X = torch.from_numpy(np.random.default_rng(5).random((n, n)) ** 2).cuda()
    D_ref = torch.empty_like(X)
    _, sw_ref, g_ref = fr.fram_sdsn(ctx, n, X, D_ref, 2.0, 1e-14, 40)
    assert int(sw) == sw_ref
    assert relF(np.load(out), D_ref.cpu().numpy()) <= 1e-12
    assert abs(float(g) - g_ref) <= 1e-12 * max(1.0, abs(g_ref))
