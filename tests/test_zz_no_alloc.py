"""The allocation-free panel factorization (hpl_panel_getrf_noalloc).

It serves callers that cannot allocate device memory when they call the
library -- for example a process that hands all GPU memory to its own pool at
start-up.  The tests call the entry point through the C ABI (ctypes): twice in
a row against the workspace-based hpl_panel_getrf, and directly against the
oracle, with the tolerance of the panel parity tests.  It is collected last so a failing run
that stops at the first failure has run every other test already, and it needs
no state from other tests.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest
import torch

from tests import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import __graft_entry__ as g
    g.build()
    import paper_2304_10397_gb300 as H
    assert torch.cuda.is_available()
    return H


def _dev(H, A, ld):
    T = H.colmajor(A.shape[0], A.shape[1], ld=ld)
    T.copy_(torch.from_numpy(np.ascontiguousarray(A)))
    return T


def test_noalloc_panel_matches_workspace_entry(H):
    L = H.load_library()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (m, w) in enumerate([(4096, 384), (20000, 512)]):
        A = inputs.uniform((m, w), seed=900 + call)
        # the existing entry point (workspace-based)
        ref = _dev(H, A, m + 1)
        ipiv_ref, info_ref = H.panel_getrf(ref)
        H.sync_check()
        # the new entry point, through the C ABI
        got = _dev(H, A, m + 1)
        ipiv = torch.zeros(w, device="cuda", dtype=torch.int32)
        info = torch.full((1,), 7, device="cuda", dtype=torch.int32)
        rc = L.hpl_panel_getrf_noalloc(C.c_int64(m), C.c_int64(w), C.c_void_p(got.data_ptr()), C.c_int64(m + 1),
                                       C.c_void_p(ipiv.data_ptr()), C.c_void_p(info.data_ptr()), stream)
        assert rc == 0, L.hpl_last_error()
        torch.cuda.synchronize()
        assert int(info.item()) == 0 == int(info_ref.item())
        assert np.array_equal(ipiv.cpu().numpy(), ipiv_ref.cpu().numpy()[:w])
        R = ref.cpu().numpy()
        G = got.cpu().numpy()
        assert np.max(np.abs(G - R)) <= 1e-11 * max(1.0, np.max(np.abs(R)))


@pytest.mark.parametrize("m,w", [(3000, 384), (517, 100), (7, 1)])
def test_noalloc_panel_vs_oracle(H, m, w):
    # directly against the oracle: its unblocked partial-pivoting LU replays
    # the GPU's pivots under the 1e-13 near-tie rule (a tie may go either
    # way), then the factors agree to the panel parity bar
    import oracle as O
    L = H.load_library()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    A = inputs.uniform((m, w), seed=31 * m + w)
    got = _dev(H, A, m + 3)
    ipiv = torch.zeros(w, device="cuda", dtype=torch.int32)
    info = torch.full((1,), 7, device="cuda", dtype=torch.int32)
    rc = L.hpl_panel_getrf_noalloc(C.c_int64(m), C.c_int64(w), C.c_void_p(got.data_ptr()), C.c_int64(m + 3),
                                   C.c_void_p(ipiv.data_ptr()), C.c_void_p(info.data_ptr()), stream)
    assert rc == 0, L.hpl_last_error()
    torch.cuda.synchronize()
    gp = ipiv.cpu().numpy()[:w]
    LU, oipiv, oinfo, st, mism = O.getrf(A, replay=gp, rtol=1e-13)
    assert st == 0, "pivot of column %d differs beyond the tie tolerance" % (-st - 1)
    assert np.array_equal(oipiv, gp)
    assert int(info.item()) == oinfo == 0
    G = got.cpu().numpy()[:m, :w]
    assert np.max(np.abs(G - LU)) <= 1e-11 * max(1.0, np.max(np.abs(LU)))


def test_noalloc_rejects_width_beyond_its_scratch(H):
    L = H.load_library()
    L.hpl_last_error.restype = C.c_char_p
    m, w = 2048, 1025
    A = H.colmajor(m, w)
    ipiv = torch.zeros(w, device="cuda", dtype=torch.int32)
    info = torch.zeros(1, device="cuda", dtype=torch.int32)
    rc = L.hpl_panel_getrf_noalloc(C.c_int64(m), C.c_int64(w), C.c_void_p(A.data_ptr()), C.c_int64(m),
                                   C.c_void_p(ipiv.data_ptr()), C.c_void_p(info.data_ptr()),
                                   C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -2 and b"1024" in L.hpl_last_error()


_FRESH = r"""
import ctypes as C, json, sys
sys.path.insert(0, sys.argv[1])
import torch
import paper_2304_10397_gb300 as H
torch.cuda.set_device(0)
L = H.load_library()
m, w = 8192, 256
A = H.colmajor(m, w)
A.uniform_(-0.5, 0.5)
ipiv = torch.zeros(w, device="cuda", dtype=torch.int32)
info = torch.zeros(1, device="cuda", dtype=torch.int32)
stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
frees, rcs, infos = [], [], []
for call in range(3):
    A.uniform_(-0.5, 0.5)
    rcs.append(L.hpl_panel_getrf_noalloc(C.c_int64(m), C.c_int64(w), C.c_void_p(A.data_ptr()), C.c_int64(m),
                                         C.c_void_p(ipiv.data_ptr()), C.c_void_p(info.data_ptr()), stream))
    torch.cuda.synchronize()
    infos.append(int(info.item()))
    frees.append(torch.cuda.mem_get_info()[0])
print(json.dumps({"free0": free0, "frees": frees, "rcs": rcs, "infos": infos,
                  "workspace_bytes": int(L.hpl_workspace_bytes())}))
"""


def test_noalloc_allocates_nothing_in_a_fresh_process(H):
    # Run in a process of its own, where this entry point is the library's
    # first call: the library must take no workspace (hpl_workspace_bytes
    # stays 0) and the device's free memory must not move from call to call.
    # The first call may load the library's module (code and the static
    # scratch array), which is the only change allowed, and is small.
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FRESH, root], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["rcs"] == [0, 0, 0] and out["infos"] == [0, 0, 0]
    assert out["workspace_bytes"] == 0
    assert out["frees"][0] == out["frees"][1] == out["frees"][2]
    assert out["free0"] - out["frees"][0] <= 64 << 20, out
