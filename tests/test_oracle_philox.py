"""Pin the oracle's Philox4x32-10 to an independent library implementation.

Triton ships a Philox4x32 (``tl.philox_impl``); run in its CPU interpreter it
gives the reference blocks for random counters and keys. Runs in a child
process because the interpreter switch must be set before triton loads."""
import json
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle

CHILD = textwrap.dedent(r"""
    import os, sys, json
    os.environ["TRITON_INTERPRET"] = "1"
    import numpy as np, torch, triton, triton.language as tl

    @triton.jit
    def k(c0, c1, c2, c3, k0, k1, o0, o1, o2, o3, N: tl.constexpr):
        i = tl.arange(0, N)
        a = tl.load(c0 + i); b = tl.load(c1 + i); c = tl.load(c2 + i); d = tl.load(c3 + i)
        x0 = tl.load(k0 + i); x1 = tl.load(k1 + i)
        r0, r1, r2, r3 = tl.philox_impl(a, b, c, d, x0, x1, 10)
        tl.store(o0 + i, r0); tl.store(o1 + i, r1); tl.store(o2 + i, r2); tl.store(o3 + i, r3)

    inp = np.array(json.loads(sys.stdin.read()), dtype=np.uint64).astype(np.uint32)
    N = inp.shape[0]
    cols = [torch.from_numpy(inp[:, j].copy()) for j in range(6)]
    outs = [torch.zeros(N, dtype=torch.uint32) for _ in range(4)]
    k[(1,)](*cols, *outs, N=N)
    print(json.dumps(np.stack([o.numpy() for o in outs], 1).astype(np.uint64).tolist()))
""")


def test_philox_matches_library_implementation():
    pytest.importorskip("triton")
    rng = np.random.default_rng(20110523)
    inp = rng.integers(0, 2**32, size=(64, 6), dtype=np.uint64)
    inp[0] = 0
    inp[1] = 2**32 - 1
    proc = subprocess.run([sys.executable, "-c", CHILD], input=json.dumps(inp.tolist()),
                          capture_output=True, text=True, timeout=600)
    if proc.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + proc.stderr[-300:])
    ref = np.array(json.loads(proc.stdout.strip().splitlines()[-1]), dtype=np.uint64)
    for i in range(inp.shape[0]):
        got = oracle.philox(inp[i, :4], inp[i, 4:6])
        assert got.astype(np.uint64).tolist() == ref[i].tolist(), i


def test_philox_uniformity():
    # words of consecutive counters are uniform and their bits balanced
    words = np.array([oracle.philox([i, 7, 3, 0], [0x5EED, 0]) for i in range(4000)],
                     dtype=np.uint64)
    u = words.astype(np.float64) / 2**32
    assert abs(u.mean() - 0.5) < 4 * np.sqrt(1 / 12 / u.size)
    bits = np.unpackbits(words.astype(np.uint32).view(np.uint8))
    assert abs(bits.mean() - 0.5) < 4 * 0.5 / np.sqrt(bits.size)
