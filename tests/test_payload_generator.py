"""The SplitMix64 payload generator of served requests (host side).

Pinned to the published reference outputs of SplitMix64 from state 0
(tests/golden/splitmix64_seed0.txt); the payload mappings give the stated
ranges exactly (int32 on [0, 65536), float32 multiples of 2^-24 on [0, 1)).
The device implementation is compared with this one in test_gpu_serve.py.
"""
import os

import numpy as np

from signals import Request, payload_from_bits, request_payload, splitmix64

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed0.txt")


def test_splitmix64_reference_outputs():
    want = [int(l, 16) for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    got = splitmix64(0, len(want))
    assert [int(v) for v in got] == want
    # offsets continue the same stream
    assert [int(v) for v in splitmix64(0, 2, offset=2)] == want[2:4]


def test_payload_ranges_and_exactness():
    z = splitmix64(99, 200_000)
    xi = payload_from_bits(z, "int32")
    assert xi.dtype == np.int32 and xi.min() >= 0 and xi.max() < 65536
    xf = payload_from_bits(z, "float32")
    assert xf.dtype == np.float32 and xf.min() >= 0.0 and xf.max() < 1.0
    scaled = xf.astype(np.float64) * 2 ** 24
    assert np.array_equal(scaled, np.floor(scaled))
    assert np.array_equal(scaled.astype(np.int64), (z >> np.uint64(40)).astype(np.int64))
    # roughly uniform: every 1/16 bucket holds 1/16 +- 1 %
    h = np.bincount((xf * 16).astype(np.int64), minlength=16) / xf.size
    assert np.all(np.abs(h - 1 / 16) < 0.01)


def test_request_payload_is_deterministic():
    r = Request(rid=3, arrival_s=0.0, n=1000, k=5, dtype="float32", seed=2 ** 63 + 1)
    assert np.array_equal(request_payload(r), request_payload(r))
    r2 = Request(rid=3, arrival_s=0.0, n=1000, k=5, dtype="float32", seed=2 ** 63 + 2)
    assert not np.array_equal(request_payload(r), request_payload(r2))
