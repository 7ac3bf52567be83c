"""Pins for the oracle's Philox4x32-10 stream (Salmon et al., SC 2011).

The reference values come from Triton's own Philox4x32 routine, run in
Triton's CPU interpreter in a child process: a library implementation that
shares nothing with the oracle."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle

_TRITON_SCRIPT = r"""
import json, os, sys
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl
from triton.language.random import philox

@triton.jit
def k(c_ptr, out_ptr, seed, N: tl.constexpr):
    i = tl.arange(0, N)
    c0 = tl.load(c_ptr + 4 * i + 0).to(tl.uint32, bitcast=True)
    c1 = tl.load(c_ptr + 4 * i + 1).to(tl.uint32, bitcast=True)
    c2 = tl.load(c_ptr + 4 * i + 2).to(tl.uint32, bitcast=True)
    c3 = tl.load(c_ptr + 4 * i + 3).to(tl.uint32, bitcast=True)
    r0, r1, r2, r3 = philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + 4 * i + 0, r0.to(tl.int32, bitcast=True))
    tl.store(out_ptr + 4 * i + 1, r1.to(tl.int32, bitcast=True))
    tl.store(out_ptr + 4 * i + 2, r2.to(tl.int32, bitcast=True))
    tl.store(out_ptr + 4 * i + 3, r3.to(tl.int32, bitcast=True))

cases = json.loads(sys.stdin.read())
res = []
for seed, ctrs in cases:
    c = torch.tensor(np.array(ctrs, dtype=np.uint32).view(np.int32).reshape(-1))
    out = torch.zeros_like(c)
    k[(1,)](c, out, seed, N=len(ctrs))
    res.append(out.numpy().view(np.uint32).reshape(-1, 4).tolist())
print(json.dumps(res))
"""


def _cases():
    rng = np.random.default_rng(11)
    seeds = [0, 1, 0xFFFFFFFF, 0x123456789ABCDEF0, int(rng.integers(0, 2**63))]
    out = []
    for s in seeds:
        ctrs = rng.integers(0, 2**32, size=(16, 4), dtype=np.uint64)
        ctrs[0] = 0
        ctrs[1] = [2**32 - 1] * 4
        ctrs[2] = [5, 0, 0, 0]
        ctrs[3] = [0, 0, 0, 7]
        out.append([s, ctrs.tolist()])
    return out


def test_philox_matches_triton_reference():
    pytest.importorskip("triton")
    cases = _cases()
    env = dict(os.environ, TRITON_INTERPRET="1")
    p = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(cases), capture_output=True,
                       text=True, env=env, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    ref = json.loads(p.stdout.strip().splitlines()[-1])
    for (seed, ctrs), expect in zip(cases, ref):
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for c, e in zip(ctrs, expect):
            got = oracle.philox(c, key)
            assert [int(x) for x in got] == e, (seed, c)


def test_philox_uniform_bins():
    # 2^14 draws of lane 0 from consecutive counters: 64-bin chi-square.
    key = [12345, 678]
    vals = np.array([oracle.philox([i, 0, 3, 0], key)[0] for i in range(1 << 14)], np.uint64)
    u = (vals >> np.uint64(8)).astype(np.float64) / 2.0**24
    hist, _ = np.histogram(u, bins=64, range=(0.0, 1.0))
    expect = len(u) / 64
    chi2 = float(np.sum((hist - expect) ** 2 / expect))
    assert chi2 < 120.0   # 63 dof: p ~ 1e-5
